"""Benchmark of the flat-torus generalized MBO iteration on GB300.

Workload (the single-GPU configuration the headline metric is quoted on):
2-D torus 1024 x 1024, n = 3 (O_3-valued), tau = 3 h^2, initial field iid
N(0,1) 3x3 entries with det > 0 on x < 1/2 and det < 0 on x >= 1/2, projected
onto O_3.  A step is one MBO iteration (diffusion of all 9 channels,
projection of every point, FP64 Lyapunov energy, stationarity statistics).
The FP32 form is the headline ``value``; the FP64 form is reported beside it.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the launching stream with a 256 MB L2-flushing read between steps (outside
the events); barrier + synchronize on both sides; max over ranks.  The field
and its workspace (~80 MB) would otherwise stay in the 129 MB L2.

Sub-lines of the same JSON line: the FP64 form (with its ALU roofline against
the measured DFMA rate), the FP32 form with FP64 re-projection below
sigma_min = 1e-3, the 96-field batch, the 128^2 n=2 FP64 run (c1), the 256^3
and 512^3 fields (c3, c5), the measured SIMT multiply-add peaks, and an
accuracy block: one step of each form against one oracle step from the same
input, and 200-step runs against the stored oracle run.  The roofline uses
the minimal 2-D schedule's algorithmic bytes: 2S per fused pass, 4S per step
(S = P n^2 w).

Multi-GPU: the path has no exchange step; each rank iterates its own field
(replicas, weak scaling, no collective on the data path).

``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1711_01365_gb300 import inputs as I  # noqa: E402

METRIC = "grid-point MBO iterations/sec and % HBM roofline, FP32/batched vs FP64 plain"
UNIT = "grid-point iterations/s"
WORKLOAD = "C2"


def kernel_sources_hash() -> str:
    """sha256 (first 16 hex digits) of the CUDA sources, concatenated as
    csrc/*.cu, *.cuh, *.h in name order."""
    import glob
    import hashlib
    d = os.path.join(ROOT, "paper_1711_01365_gb300", "csrc")
    data = b""
    for pat in ("*.cu", "*.cuh", "*.h"):
        for f in sorted(glob.glob(os.path.join(d, pat))):
            with open(f, "rb") as fh:
                data += fh.read()
    return hashlib.sha256(data).hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the last ncu capture, if it was taken on
    the current kernel sources; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("sources_sha256_16") != kernel_sources_hash() or kernel not in rec.get("kernel", ""):
        return None
    return rec.get("dram_bytes_per_launch")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def job_throughput(points_per_rank: int, steps: int, seconds_local: float, device=None):
    """Whole-job grid-point iterations/s over replicas: every rank iterates its
    own field (no data-path collective); the job time is the max over ranks.
    Returns (value, job_seconds)."""
    import torch
    import torch.distributed as dist

    t = seconds_local
    ws = 1
    if dist.is_available() and dist.is_initialized():
        ws = dist.get_world_size()
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return points_per_rank * steps * ws / t, t


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def field_c2(dims=None):
    F, n, tau = I.config_field(WORKLOAD, dims=dims)
    return F, n, tau


def oracle_sample(steps_budget_s: float, K: int | None = None):
    """Time the FP64 oracle on the full workload, whole MBO iterations only."""
    from oracle import oracle as O

    F, n, tau = field_c2()
    cores = O.set_threads(0)
    A = O.project(F, n)
    P = int(np.prod(F.shape[1:]))
    done, t0 = 0, time.perf_counter()
    times = []
    while True:
        ts = time.perf_counter()
        A, _ = O.step(A, n, tau)
        times.append(time.perf_counter() - ts)
        done += 1
        el = time.perf_counter() - t0
        if (K is not None and done >= K) or (K is None and el >= steps_budget_s) or el >= steps_budget_s:
            break
    total = sum(times)
    return {"value": P * done / total, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} full MBO iteration(s) of the {F.shape[1]}x{F.shape[2]} n={n} field, "
                      f"FP64 C oracle, OpenMP over {cores} threads",
            "steps": done, "seconds": total}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from oracle import oracle as O

    O.build()
    F, n, tau = field_c2()
    P = int(np.prod(F.shape[1:]))
    cores = O.set_threads(0)
    A = O.project(F, n)
    for _ in range(args.warmup):
        A, _ = O.step(A, n, tau)
    budget = 150.0
    times = []
    t0 = time.perf_counter()
    for k in range(args.steps):
        ts = time.perf_counter()
        A, _ = O.step(A, n, tau)
        times.append(time.perf_counter() - ts)
        if time.perf_counter() - t0 > budget:
            break
    total = sum(times)
    done = len(times)
    v = P * done / total
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / done,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "2-D flat torus 1024x1024, n=3, tau=3h^2, sign-split iid N(0,1) init",
                   "grid": list(F.shape[1:]), "n": n, "tau": tau},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{done} of {args.steps} requested full MBO iterations "
                                   f"(time budget {budget:.0f} s), FP64 C oracle, {cores} threads"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_steps(torch, h, A, K, flush, prof=True):
    """K steady-state steps, each between CUDA events, L2 flushed in between."""
    from paper_1711_01365_gb300 import mbo as M

    s = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    if prof:
        M.mbo_profile_enable(h.h, True)
    for k in range(K):
        flush()
        ev[k][0].record(s)
        h.step(A, flags=M.MBO_STEP_CONTINUE)
        ev[k][1].record(s)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    passes = M.mbo_profile_read(h.h) if prof else None
    if prof:
        M.mbo_profile_enable(h.h, False)
    return ms, passes


def bench_batched(args, torch, M):
    """96 independent 2-D fields of uneven sizes and orders (FP32), one CUDA-graph
    launch per batch step; the 6 GB working set exceeds the L2."""
    spec = I.batch_mixed(96, None)
    dims_l = [s[0] for s in spec]
    n_l = [s[1] for s in spec]
    tau_l = [s[2] for s in spec]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(I.SEED_BASE + 4)
    A = []
    for d, n, tau in zip(dims_l, n_l, tau_l):
        raw = torch.randn((n * n,) + tuple(d), generator=gen, device="cuda", dtype=torch.float32)
        h = M.Mbo(d, n, tau, "f32")
        a = torch.empty_like(raw)
        h.project(raw, a)
        h.close()
        A.append(a)
        del raw
    b = M.Batch(dims_l, n_l, tau_l, "f32")
    b.step(A)
    for _ in range(max(args.warmup - 1, 0)):
        b.step(A, flags=M.MBO_STEP_CONTINUE)
    K = max(3, args.steps)
    s = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    torch.cuda.synchronize()
    for k in range(K):
        ev[k][0].record(s)
        b.step(A, flags=M.MBO_STEP_CONTINUE)
        ev[k][1].record(s)
    torch.cuda.synchronize()
    t = sum(a.elapsed_time(e) for a, e in ev) / 1e3
    pts = sum(int(np.prod(d)) for d in dims_l)
    b.close()
    # minimal 2-D schedule of every field: two fused passes over its spectrum, 4 S_i
    step_bytes = sum(4 * int(np.prod(d)) * n * n * 4 for d, n in zip(dims_l, n_l))
    hbm, peak_kind = load_peaks()
    ach = step_bytes / (t / K) / 1e9
    return {"value": pts * K / t, "unit": UNIT, "fields": len(spec), "points": pts, "steps": K,
            "ms_per_step": 1e3 * t / K, "dtype": "f32",
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "peak_kind": peak_kind, "traffic": None,
                         "alg_bytes_per_step": step_bytes,
                         "basis": "sum over the fields of 4 S_i (S_i = P_i n_i^2 4 B), the whole "
                                  "batch step"},
            "note": "96 fields 256^2..2048^2, n=2/3, tau=4h^2, one graph launch per batch step, "
                    "working set > L2 (no flush)"}


EPS32 = 2.0 ** -24


def accuracy_block(torch, M, A_in32, n, tau):
    """One step of each form from the same input (the FP32 field after the
    timed steps, taken exactly in FP64) against one FP64 oracle step:
    max-entry error (all points; points whose |det A~| is above the FP32
    rounding level 64 eps |A~|_F^n; of those, points with sigma_2 + sigma_3 >=
    1e-2), orthogonality defect max |B^t B - I|, energy relative error and
    det-flip counts.  Host time: one oracle step plus an SVD per point."""
    from oracle import oracle as O

    dims = tuple(A_in32.shape[1:])
    A_in = A_in32.double().cpu().numpy()
    O.set_threads(0)
    ref, st = O.step(A_in, n, tau)
    At = O.diffuse(A_in, tau)
    mats = np.moveaxis(At.reshape(n * n, -1), 0, -1).reshape(-1, n, n)
    sv = np.linalg.svd(mats, compute_uv=False)
    cs = sv[:, -1] + sv[:, -2]
    absdet = np.prod(sv, axis=1)
    cut = 64 * EPS32 * np.sqrt((sv ** 2).sum(axis=1)) ** n
    out = {"input": "the FP32 field after the timed steps, exactly in FP64; one step of each form vs one FP64 oracle step",
           "oracle_energy": st["energy"], "oracle_det_flips": int(st["det_flips"])}
    for form, tdt in (("fp32", torch.float32), ("fp64", torch.float64)):
        h = M.Mbo(dims, n, tau, form.replace("fp", "f"))
        t = torch.tensor(A_in, dtype=tdt, device="cuda")
        rec = h.step(t, want_stats=True)
        B = t.double().cpu().numpy()
        h.close()
        err = np.abs(B - ref).reshape(n * n, -1).max(axis=0)
        Bm = np.moveaxis(B.reshape(n * n, -1), 0, -1).reshape(-1, n, n)
        orth = np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(n)).max()
        unamb = absdet > (cut if form == "fp32" else 1e-12)
        well = unamb & (cs >= 1e-2)
        out[form] = {"max_entry_err_all": float(err.max()),
                     "max_entry_err_unambiguous": float(err[unamb].max()),
                     "max_entry_err_sigma23_ge_1e-2": float(err[well].max()),
                     "points_det_at_rounding_level": int((~unamb).sum()),
                     "orthogonality_defect": float(orth),
                     "energy_rel_err": abs(rec["energy"] - st["energy"]) / abs(st["energy"]),
                     "det_flips": int(rec["det_flips"])}
    return out


def trajectory_block(torch, M):
    """200 steps of the 1024^2 n=3 workload from the oracle's projection of
    the raw field, both forms, against the FP64 oracle run stored in
    tests/golden/c2_trajectory_fp64.txt: stationary step counts, the number of
    leading steps whose det-sign flip counts agree, and the largest energy
    relative error over those steps."""
    from oracle import oracle as O

    path = os.path.join(ROOT, "tests", "golden", "c2_trajectory_fp64.txt")
    if not os.path.exists(path):
        return None
    g_steps, g_stat, rows = None, None, []
    with open(path) as f:
        for line in f:
            if line.startswith("# steps="):
                kv = dict(x.split("=") for x in line[2:].split()[:2])
                g_steps, g_stat = int(kv["steps"]), bool(int(kv["stationary"]))
            elif not line.startswith("#"):
                rows.append(line.split())
    g_en = np.array([float(r[1]) for r in rows])
    g_fl = np.array([int(r[3]) for r in rows[:-1]])
    F, n, tau = I.config_field(WORKLOAD)
    A0 = O.project(F, n)
    out = {"oracle_steps": g_steps, "oracle_stationary": g_stat, "max_steps": 200, "tol": 1e-4}
    for form, tdt in (("fp32", torch.float32), ("fp64", torch.float64)):
        h = M.Mbo(F.shape[1:], n, tau, form.replace("fp", "f"))
        t = torch.tensor(A0, dtype=tdt, device="cuda")
        r = h.run(t, 200, 1e-4)
        h.close()
        fl = np.asarray(r["det_flips"])
        k = min(len(fl), len(g_fl))
        diff = np.nonzero(fl[:k] != g_fl[:k])[0]
        agree = int(diff[0]) if len(diff) else k
        en = np.asarray(r["energies"])
        m = min(len(en), len(g_en), agree + 1)
        out[form] = {"steps": int(r["steps"]), "stationary": bool(r["stationary"]),
                     "steps_flips_agree": agree,
                     "max_energy_rel_err_while_agreeing": float(np.max(np.abs(en[:m] - g_en[:m]) / np.abs(g_en[:m])))}
    return out


def bench_c1(torch, M, steps):
    """128^2, n=2, FP64, tau=4h^2: graph-replayed run of `steps` steps (never
    stopping) from the projected Gaussian field; launch-latency bound."""
    from oracle import oracle as O

    F, n, tau = I.config_field("C1")
    A0 = O.project(F, n)
    h = M.Mbo(F.shape[1:], n, tau, "f64", autotune=1)  # launch shapes timed at creation
    t = torch.tensor(A0, dtype=torch.float64, device="cuda")
    h.run(t, 10, -1.0)  # warm-up (captures the step graph)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    r = h.run(t, steps, -1.0)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    h.close()
    P = int(np.prod(F.shape[1:]))
    return {"workload": "2-D flat torus 128x128, n=2 (O_2), tau=4h^2, FP64, graph-replayed run",
            "value": P * r["steps"] / (ms / 1e3), "unit": UNIT, "steps": int(r["steps"]),
            "us_per_step": 1e3 * ms / r["steps"], "dtype": "f64",
            "note": "mbo_run_until_stationary with tol < 0 (no early stop); includes the run's "
                    "host polls of the step records; launch shapes autotuned; the field fits in L2 "
                    "(latency bound: 128 rows of FP64 work per pass)"}


def bench_3d(torch, M, name, steps, warmup, hbm, peak_kind):
    """K steady-state steps of a 3-D workload (FP32, n=3), each between CUDA
    events without per-pass events; then a profiled set of steps for the pass
    times.  The fields exceed L2, so no flush is needed."""
    F, n, tau = I.config_field(name, dtype=np.float32)
    dims = tuple(F.shape[1:])
    P = int(np.prod(dims))
    h = M.Mbo(dims, n, tau, "f32")
    raw = torch.from_numpy(F).cuda()
    del F
    A = torch.empty_like(raw)
    h.project(raw, A)
    del raw
    h.step(A)
    for _ in range(max(warmup - 1, 0)):
        h.step(A, flags=M.MBO_STEP_CONTINUE)
    torch.cuda.synchronize()
    ms, _ = time_steps(torch, h, A, steps, lambda: None, prof=False)
    _, passes = time_steps(torch, h, A, 2, lambda: None, prof=True)
    h.close()
    del A
    torch.cuda.empty_cache()
    t = sum(ms) / 1e3 / steps
    C, Q, nx = n * n, (n * n + 1) // 2, dims[-1]
    xh = min(nx, ((nx // 2 + 1 + 15) // 16) * 16) if (C % 2 and nx in (256, 512, 1024)) else nx
    w_bytes = ((Q - 1) * nx + xh) * (P // nx) * 2 * 4
    S = C * P * 4
    pt = {k: v[0] / 1e3 / max(v[1], 1) for k, v in passes.items() if v[1]}
    # a 3-D step moves 8S algorithmic bytes (four passes, each reading and writing the field's bytes)
    return {"workload": f"3-D flat torus {'x'.join(map(str, dims))}, n=3, FP32, tau=2h^2",
            "value": P / t, "unit": UNIT, "steps": steps, "ms_per_step": 1e3 * t, "dtype": "f32",
            "roofline": {"bound": "hbm", "achieved": 8 * S / t / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": 8 * S / t / 1e9 / hbm, "peak_kind": peak_kind,
                         "alg_bytes_per_step": 8 * S, "basis": "8S per step (four passes over the field bytes S)",
                         "passes_us": {k: v * 1e6 for k, v in pt.items()},
                         "step_bytes_as_built": 2 * w_bytes * 3 + 2 * w_bytes + 2 * S},
            "l2": "field larger than L2 (no flush)"}


def run_ours(args, ws, rank, local):
    import torch

    from paper_1711_01365_gb300 import build as B

    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    from paper_1711_01365_gb300 import mbo as M

    F, n, tau = field_c2()
    dims = tuple(F.shape[1:])
    P = int(np.prod(dims))
    C = n * n
    # initial field: projected onto O_3 by the library (FP64)
    raw = torch.tensor(F, dtype=torch.float64, device="cuda")
    h64 = M.Mbo(dims, n, tau, "f64")
    A0 = torch.empty_like(raw)
    h64.project(raw, A0)
    del raw
    flushbuf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB
    flushbuf.fill_(1.0)
    sink = torch.zeros((), dtype=torch.float32, device="cuda")

    def flush():
        sink.add_(flushbuf.sum())

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- FP32 form (headline) ----
    h32 = M.Mbo(dims, n, tau, "f32")
    A32 = A0.float().contiguous()
    clk = ClockSampler(local)
    clk.start()
    h32.step(A32)  # fills the workspace spectrum
    for _ in range(max(args.warmup - 1, 0)):
        flush()
        h32.step(A32, flags=M.MBO_STEP_CONTINUE)
    barrier()
    ms32, _ = time_steps(torch, h32, A32, args.steps, flush, prof=False)
    barrier()
    value, t32 = job_throughput(P, args.steps, sum(ms32) / 1e3, device="cuda")
    # per-pass device times from a separate, profiled set of steps (the event
    # pairs around each pass stay out of the timed steps above)
    _, passes = time_steps(torch, h32, A32, max(5, min(args.steps, 20)), flush, prof=True)

    # dominant kernel: the fused inverse-x / projection / forward-x pass
    hbm, peak_kind = load_peaks()
    elem = 4
    Q = (C + 1) // 2
    # the workspace keeps Q complex planes; a last plane holding one real
    # channel keeps only its Hermitian half along x (nx/2 + 1 columns rounded
    # up to 16) when the x transform is the natural-order warp plan
    nx = dims[-1]
    xh = min(nx, ((nx // 2 + 1 + 15) // 16) * 16) if (C % 2 and nx in (256, 512, 1024)) else nx
    w_bytes = ((Q - 1) * nx + xh) * (P // nx) * 2 * elem
    a_bytes = C * P * elem
    row_ms, row_n = passes["row_project"]
    ax_ms, ax_n = passes["axis_fgi"]
    # algorithmic bytes of the minimal 2-D schedule (two fused passes, each
    # reading and writing the field's bytes S = P n^2 w): 2S per pass, 4S per step
    S = a_bytes
    row_t = row_ms / 1e3 / max(row_n, 1)
    ax_t = ax_ms / 1e3 / max(ax_n, 1)
    dominant = ("row_project", row_t) if row_ms >= ax_ms else ("axis_fgi", ax_t)
    achieved = 2 * S / dominant[1] / 1e9
    traffic = recorded_traffic("k_wrow" if dominant[0] == "row_project" else "k_wcol")
    roofline = {"bound": "hbm", "kernel": dominant[0], "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "peak_kind": peak_kind,
                "traffic": traffic,
                "alg_bytes_per_launch": 2 * S, "launch_us": dominant[1] * 1e6,
                "basis": "2S per fused pass, 4S per step (S = P n^2 w, the field's bytes)",
                "passes_us": {"row_project": row_t * 1e6, "axis_fgi": ax_t * 1e6},
                "step_alg_bytes": 4 * S,
                "step_frac": 4 * S / (t32 / args.steps) / 1e9 / hbm,
                "as_built_bytes": {"row_project": 2 * w_bytes + 2 * a_bytes, "axis_fgi": 2 * w_bytes,
                                   "note": "x pass: read W, read the old field for the step "
                                           "statistics, write the field, write W; y pass: read W, write W"}}

    # ---- FP64 form (plain), same workload ----
    fp64 = None
    if not args.no_fp64:
        A64 = A0.clone()
        h64.step(A64)
        for _ in range(2):
            h64.step(A64, flags=M.MBO_STEP_CONTINUE)
        K64 = max(3, min(args.steps, 10))
        barrier()
        ms64, _ = time_steps(torch, h64, A64, K64, flush, prof=False)
        barrier()
        _, p64 = time_steps(torch, h64, A64, 3, flush, prof=True)
        v64, t64 = job_throughput(P, K64, sum(ms64) / 1e3, device="cuda")
        fp64 = {"value": v64, "unit": UNIT, "steps": K64,
                "ms_per_step": 1e3 * t64 / K64,
                "passes_us": {k: 1e3 * v[0] / max(v[1], 1) for k, v in p64.items() if v[1]}}

    # ---- FP32 form with the FP64 re-projection trigger at sigma_min < 1e-3 ----
    fb3 = None
    if not args.no_fp64:
        hf = M.Mbo(dims, n, tau, "f32", fallback_sigma=1e-3)
        Af = A0.float().contiguous()
        hf.step(Af)
        for _ in range(max(args.warmup - 1, 0)):
            flush()
            hf.step(Af, flags=M.MBO_STEP_CONTINUE)
        barrier()
        msf, _ = time_steps(torch, hf, Af, args.steps, flush, prof=False)
        barrier()
        recf = hf.step(Af, flags=M.MBO_STEP_CONTINUE, want_stats=True)
        vf, tf = job_throughput(P, args.steps, sum(msf) / 1e3, device="cuda")
        fb3 = {"value": vf, "unit": UNIT, "ms_per_step": 1e3 * tf / args.steps,
               "fallback_points_per_step": int(recf["fallback_points"]),
               "note": "fallback_sigma = 1e-3: n=3 points whose smallest-singular-value estimate "
                       "is below 1e-3 are re-projected in FP64 (the headline uses the default 0: "
                       "quaternion form, FP64 only where (sigma_2+sigma_3)/|A| is small too)"}
        hf.close()
        del Af

    # ---- batched form: 96 independent uneven fields (256^2 .. 2048^2, n = 2, 3) ----
    batched = None
    if not args.no_batch:
        batched = bench_batched(args, torch, M)

    # ---- the other configurations: 128^2 n=2 FP64 (launch-latency bound), 256^3 and 512^3 ----
    c1 = c3 = c5 = None
    if not args.no_extra:
        c1 = bench_c1(torch, M, 100)
        c3 = bench_3d(torch, M, "C3", 5, 3, hbm, peak_kind)
        c5 = bench_3d(torch, M, "C5", 3, 3, hbm, peak_kind)
    # ---- measured SIMT pipe peaks; the FP64 form's ALU roofline ----
    peaks = M.mbo_measure_fma_peaks()
    clocks = clk.stop()
    if fp64 is not None:
        # algorithmic FP64 flops per point and step: four length-1024 complex
        # transforms of the 5 planes (5 N log2 N each: 50 per element), the
        # multiplier (2 per element) and the scaled Newton polar factor of a
        # 3x3 (about 95 flops per scaled and 59 per unscaled iteration; about
        # four scaled and three unscaled)
        flops_pt = 5 * (4 * 50 + 2) + (4 * 95 + 3 * 59)
        ach = flops_pt * P / (fp64["ms_per_step"] / 1e3) / 1e12
        fp64["roofline"] = {"bound": "fp64_alu", "achieved": ach, "peak": peaks["fp64"], "unit": "TFLOP/s",
                            "frac": ach / peaks["fp64"], "peak_kind": "measured (mbo_measure_fma_peaks, DFMA)",
                            "alg_flops_per_point_step": flops_pt}

    # ---- run loop as a user runs it (graph replay, L2 left warm) ----
    Arun = A0.float().contiguous()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = h32.run(Arun, args.run_steps, -1.0)
    t_run = time.perf_counter() - t0
    run_loop = {"value": P * r["steps"] / t_run, "unit": UNIT, "steps": r["steps"],
                "note": "mbo_run_until_stationary on a device field, wall clock, L2 not flushed"}

    # ---- end to end through the C ABI with host buffers ----
    hostA = A0.float().cpu().pin_memory()
    e2e_times = []
    for _ in range(3):
        src = hostA.clone().pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = h32.run(src, args.run_steps, -1.0)
        e2e_times.append(time.perf_counter() - t0)
    te = float(np.median(e2e_times))
    fbytes = a_bytes
    e2e = {"value": P * args.run_steps * ws / te, "unit": UNIT,
           "h2d_bytes_per_step": fbytes / args.run_steps,
           "d2h_bytes_per_step": (fbytes + 8 * (args.run_steps + 1)) / args.run_steps,
           "steps_per_call": args.run_steps,
           "note": "mbo_run_until_stationary on a pinned host field: H2D, all iterations, D2H"}

    accuracy = None
    if rank == 0 and not args.no_accuracy:
        accuracy = accuracy_block(torch, M, A32, n, tau)
        accuracy["trajectory"] = trajectory_block(torch, M)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = oracle_sample(args.cpu_seconds)
        cpu.pop("steps", None)
        cpu.pop("seconds", None)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t32 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "2-D flat torus 1024x1024, n=3 (O_3), tau=3h^2, sign-split "
                                   "iid N(0,1) init projected; FP32 form with FP64 energy sums; "
                                   "n=3 projection by scaled Newton; points singular to "
                                   "single precision by the quaternion form, or in FP64 where "
                                   "(sigma_2+sigma_3)/|A| is small too",
                       "grid": list(dims), "n": n, "tau": tau,
                       "l2": "flushed between timed steps (256 MB read)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": sum(v[1] for v in passes.values()),
            "clocks": clocks,
            "accuracy": accuracy,
            "fp64": fp64,
            "fp32_fallback_sigma_1e-3": fb3,
            "batched": batched,
            "c1": c1, "c3": c3, "c5": c5,
            "simt_peaks_tflops": peaks,
            "run_loop": run_loop,
        }
        print(json.dumps(line), flush=True)
    h32.close()
    h64.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_3d(args, ws, rank, local):
    """The 3-D workloads (256^3 Voronoi, 512^3 smooth SO(3); n = 3, FP32): K
    steady-state steps between CUDA events.  The field is larger than L2, so
    no flush is needed.  One JSON line on rank 0."""
    import torch

    from paper_1711_01365_gb300 import build as B

    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    from paper_1711_01365_gb300 import mbo as M

    name = args.workload
    F, n, tau = I.config_field(name, dtype=np.float32)
    dims = tuple(F.shape[1:])
    P = int(np.prod(dims))
    h = M.Mbo(dims, n, tau, "f32")
    raw = torch.from_numpy(F).cuda()
    del F
    A = torch.empty_like(raw)
    h.project(raw, A)
    del raw

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clk = ClockSampler(local)
    clk.start()
    h.step(A)
    for _ in range(max(args.warmup - 1, 0)):
        h.step(A, flags=M.MBO_STEP_CONTINUE)
    barrier()
    ms, _ = time_steps(torch, h, A, args.steps, lambda: None, prof=False)
    barrier()
    _, passes = time_steps(torch, h, A, 2, lambda: None, prof=True)
    clocks = clk.stop()
    value, t = job_throughput(P, args.steps, sum(ms) / 1e3, device="cuda")
    hbm, peak_kind = load_peaks()
    C, Q, nx = n * n, (n * n + 1) // 2, dims[-1]
    xh = min(nx, ((nx // 2 + 1 + 15) // 16) * 16) if (C % 2 and nx in (256, 512, 1024)) else nx
    w_bytes = ((Q - 1) * nx + xh) * (P // nx) * 2 * 4
    row_alg = 2 * w_bytes + 2 * C * P * 4
    col_alg = 2 * w_bytes
    pt = {k: v[0] / 1e3 / max(v[1], 1) for k, v in passes.items() if v[1]}
    row_t = pt["row_project"]
    roofline = {"bound": "hbm", "kernel": "row_project", "achieved": row_alg / row_t / 1e9,
                "peak": hbm, "unit": "GB/s", "frac": row_alg / row_t / 1e9 / hbm,
                "peak_kind": peak_kind, "traffic": None,
                "alg_bytes_per_launch": row_alg, "launch_us": row_t * 1e6,
                "passes_us": {k: v * 1e6 for k, v in pt.items()},
                "step_alg_bytes": row_alg + 3 * col_alg,
                "step_frac": (row_alg + 3 * col_alg) / (t / args.steps) / 1e9 / hbm}
    if rank == 0:
        init = {"C3": "Voronoi rotations + N(0,0.05) noise, projected",
                "C5": "smooth SO(3) field with 20% reflections, projected"}[name]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"3-D flat torus {'x'.join(map(str, dims))}, n=3, tau=2h^2, {init}",
                           "grid": list(dims), "n": n, "tau": tau,
                           "l2": "field larger than L2 (no flush)",
                           "parallelism": f"replicas x{ws}"},
                "roofline": roofline, "cpu_baseline": None,
                "e2e": None, "gpu_launches": 4 * args.steps, "clocks": clocks,
                "note": "secondary workload; cpu_baseline and e2e are measured on the 1024^2 headline only"}
        print(json.dumps(line), flush=True)


def run_surface(args, ws, rank, local):
    """The closed-surface workload of Sec. 6.2 (unit sphere, dx = 0.05,
    tau = 0.005, eps = 1e-6, p = 3, n = 3, FP32): K steps of Algorithm 1 with
    the diffusion of Algorithm 2, between CUDA events.  The grid (192^3 x 9
    channels) and the point tables exceed L2, so no flush is needed.  One JSON
    line on rank 0."""
    import torch

    from paper_1711_01365_gb300 import build as B

    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    from paper_1711_01365_gb300 import mbo as M

    tau, eps, dx, p, n = 0.005, 1e-6, 0.05, 3, 3
    radius = args.surface_radius
    wb = M.mbo_surface_band_width(eps, tau)
    xq, wq, xc = M.mbo_surface_sphere_band(radius, dx, wb, p)
    nq = len(wq)
    s = M.Surface(xq, wq, xc, n, tau, eps, "f32")
    prm = s.params()
    A = torch.tensor(I.sphere_paper_field(xc), dtype=torch.float32, device="cuda")

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clk = ClockSampler(local)
    clk.start()
    for _ in range(args.warmup):
        s.step(A)
    barrier()
    # per step: k_spread, the grid FFT (5 passes on 192^3), k_interp, k_sproject
    stream = torch.cuda.current_stream()
    M.mbo_surface_profile_enable(s.h, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s.step(A)
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    passes = M.mbo_surface_profile_read(s.h)
    M.mbo_surface_profile_enable(s.h, False)
    # the volume-preserving step (Sec. 7, Algorithm 3) on the same field, volume of its own input
    for _ in range(2):
        s.step_volume(A, -1.0)
    barrier()
    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    v0.record(stream)
    for _ in range(args.steps):
        s.step_volume(A, -1.0)
    v1.record(stream)
    barrier()
    vol_ms = v0.elapsed_time(v1) / args.steps
    value, t = job_throughput(nq, args.steps, ms / 1e3, device="cuda")
    # spreading: W^3 multiply-adds per source and channel (2 flops each) on the
    # FP32 vector units, against the measured FFMA rate of this device
    W = prm["width"]
    flops = 2.0 * nq * W ** 3 * n * n
    sp_ms = passes["spread"][0] / max(passes["spread"][1], 1)
    peak = M.mbo_measure_fma_peaks()["fp32"]
    achieved = flops / (sp_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": "spread", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_kind": "measured (mbo_measure_fma_peaks, FFMA chains)",
                "traffic": None, "alg_flops_per_launch": flops, "launch_us": sp_ms * 1e3,
                "passes_us": {k: 1e3 * v[0] / max(v[1], 1) for k, v in passes.items() if v[1]}}
    if rank == 0:
        line = {"metric": "surface MBO point-iterations/sec (Algorithm 1 with the diffusion of Algorithm 2)",
                "value": value, "unit": "point-iterations/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"sphere of radius {radius:g}, closest-point band (Sec. 6.2): dx=0.05, "
                                       "tau=0.005, eps=1e-6, p=3, n=3; the paper's two printed matrices as A_0",
                           "points": nq, "band_width": wb, "h": prm["h"], "M": prm["M"],
                           "grid": prm["nf"], "kernel_width": W,
                           "l2": "grid and tables larger than L2 (no flush)",
                           "parallelism": f"replicas x{ws}"},
                "roofline": roofline, "cpu_baseline": None, "e2e": None,
                "gpu_launches": 8 * args.steps, "clocks": clocks,
                "volume_step_ms": vol_ms,
                "note": "secondary workload; cpu_baseline and e2e are measured on the 1024^2 headline only; "
                        "volume_step_ms: mbo_surface_step_volume on the same field, timed after the main steps"}
        print(json.dumps(line), flush=True)
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--run-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 128^2, 256^3 and 512^3 sub-lines")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the accuracy block against the oracle")
    ap.add_argument("--workload", default="C2", choices=["C2", "C3", "C5", "sphere"],
                    help="C2: 1024^2 headline (default); C3: 256^3, C5: 512^3 (FP32 only); "
                         "sphere: the closed-surface workload of Sec. 6.2")
    ap.add_argument("--surface-radius", type=float, default=1.0,
                    help="sphere radius of --workload sphere (1 = the paper's unit sphere)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "sphere":
        run_surface(args, ws, rank, local)
    elif args.workload != "C2":
        run_3d(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()

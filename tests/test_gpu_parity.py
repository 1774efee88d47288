"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (max-entry absolute error; entries of O_n fields are <= 1):
  FP64 path  1e-12 for diffusion, projection, one fused step and the run
             (points whose diffused determinant is within rounding of 0 take
             the sign decision in each side's own arithmetic and are
             excluded from the value comparison, then checked for validity);
  FP32 path  diffusion 4e-6; projection and one step 2e-5 at points whose
             polar factor is not ill conditioned (sigma_{n-1} + sigma_n >=
             1e-2, condition number <= 200), and elsewhere the first-order
             bound 2e-5 + 2 * err(A~) / (sigma_{n-1} + sigma_n) that the polar
             factor's condition number gives; energy relative error 1e-5.
             Points whose |det A~| is within 64 eps_32 |A~|_F^n of zero, where
             the single-precision sign decision is rounding noise, are checked
             for validity only; their number is asserted small.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1711_01365_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_DIFF_TOL = 4e-6
F32_STEP_TOL = 2e-5
F32_ENERGY_RTOL = 1e-5


@pytest.fixture(scope="module")
def M():
    from paper_1711_01365_gb300 import build
    build.build()
    from paper_1711_01365_gb300 import mbo
    return mbo


def dev(a, dtype):
    t = torch.tensor(np.ascontiguousarray(a), dtype=torch.float64).to(dtype)
    return t.cuda().contiguous()


def host(t):
    return t.detach().double().cpu().numpy()


def tdt(name):
    return torch.float32 if name == "f32" else torch.float64


def mats(F, n):
    return F.reshape(n, n, -1).transpose(2, 0, 1)


def cond_sum(At, n):
    """sigma_{n-1} + sigma_n of every point (sigma_1 for n = 1)."""
    s = np.linalg.svd(mats(At, n), compute_uv=False)
    return s[:, -1] + (s[:, -2] if n > 1 else s[:, -1])


def dets(At, n):
    return np.linalg.det(mats(At, n))


# FP32 sign decisions: |det A~| within 64 eps_32 |A~|_F^n of zero is rounding
# noise for a determinant computed in single precision (the FP32 rounding of
# A~ alone moves det by ~n eps |A~|^n); such points are compared for validity
# only (reading of Lemma 1.1 at det A~ = 0).
EPS32 = 2.0 ** -24
# the strict FP32 bound holds where sigma_{n-1} + sigma_n >= 1e-2 (the polar
# factor's condition number 2 / (sigma_{n-1} + sigma_n) is at most 200 there)
F32_WELL_CS = 1e-2


def det_cut32(At, n):
    nrm = np.sqrt((mats(At, n) ** 2).sum(axis=(1, 2)))
    return 64 * EPS32 * nrm ** n


def projected(dims, n, seed):
    return O.project(I.gaussian(dims, n, seed), n)


SIZES_2D = [(2, 2), (3, 3), (4, 6), (8, 8), (6, 18), (16, 12), (24, 32), (64, 64), (96, 128),
            (128, 128), (27, 36), (48, 384)]
SIZES_3D = [(4, 6, 8), (8, 8, 8), (6, 12, 16), (16, 16, 16)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("dims", SIZES_2D + SIZES_3D)
def test_diffuse_matches_oracle(M, dims, n, dtype):
    tau = 3.0 / max(dims) ** 2
    A = projected(dims, n, 1000 + n + len(dims))
    ref = O.diffuse(A, tau)
    h = M.Mbo(dims, n, tau, dtype)
    a = dev(A, tdt(dtype))
    out = torch.empty_like(a)
    h.diffuse(a, out)
    torch.cuda.synchronize()
    err = np.abs(host(out) - ref).max()
    assert err <= (F64_TOL if dtype == "f64" else F32_DIFF_TOL), err
    h.close()


@pytest.mark.parametrize("dims,k", [((32, 32), (3, 5)), ((24, 48), (11, -7)), ((64, 64), (32, 0)),
                                    ((8, 12, 16), (2, 3, 4))])
def test_single_fourier_mode_decay_on_gpu(M, dims, k):
    tau = 2.0 / max(dims) ** 2
    X = np.meshgrid(*[np.arange(N) / N for N in dims], indexing="ij")
    ph = 2 * np.pi * sum(kk * xx for kk, xx in zip(k, X))
    F = np.stack([np.cos(ph), np.sin(ph), np.cos(ph) + 0.25, np.sin(ph) - 0.5])
    lam = math.exp(-4 * math.pi ** 2 * tau * sum(kk * kk for kk in k))
    want = np.stack([lam * np.cos(ph), lam * np.sin(ph), lam * np.cos(ph) + 0.25,
                     lam * np.sin(ph) - 0.5])
    h = M.Mbo(dims, 2, tau, "f64")
    a = dev(F, torch.float64)
    out = torch.empty_like(a)
    h.diffuse(a, out)
    torch.cuda.synchronize()
    assert np.abs(host(out) - want).max() < 1e-13
    h.close()


def _projection_inputs(n, seed):
    g = I.rng(seed)
    dims = (32, 48)
    At = O.diffuse(projected(dims, n, seed), 3.0 / 48 ** 2)       # realistic diffused matrices
    raw = g.standard_normal((n * n,) + dims) * g.choice([1e-3, 1.0, 5.0], size=dims)
    return np.concatenate([At, raw], axis=1)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [1, 2, 3])
def test_project_matches_oracle(M, n, dtype):
    At = _projection_inputs(n, 77 + n)
    dims = At.shape[1:]
    ref, sref = O.project(At, n, return_sign=True)
    h = M.Mbo(dims, n, 1e-3, dtype)
    a = dev(At, tdt(dtype))
    out = torch.empty_like(a)
    sg = torch.empty(dims, dtype=torch.int8, device="cuda")
    h.project(a, out, sg)
    torch.cuda.synchronize()
    B = host(out)
    d = np.abs(dets(At, n)).reshape(dims)
    Bm = mats(B, n)
    # always: orthogonal with the reported sign
    orth = np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(n)).max()
    assert orth < (1e-13 if dtype == "f64" else 2e-6)
    assert np.array_equal(np.sign(np.linalg.det(Bm)).reshape(dims), sg.cpu().numpy().astype(float))
    unamb = d > (1e-12 if dtype == "f64" else det_cut32(At, n).reshape(dims))
    excluded = int((~unamb).sum())
    print(f"n={n} {dtype}: {excluded} of {unamb.size} points with |det| at rounding level")
    assert excluded <= max(2, unamb.size // 100)
    assert np.array_equal(sg.cpu().numpy()[unamb], sref[unamb])
    err = np.abs(B - ref).max(axis=0)
    if dtype == "f64":
        assert err[unamb].max() <= F64_TOL
    else:
        cs = cond_sum(At, n).reshape(dims)
        well = unamb & (cs >= F32_WELL_CS)
        assert err[well].max() <= F32_STEP_TOL
        eps_in = np.abs(At - At.astype(np.float32).astype(np.float64)).max(axis=0)
        bound = F32_STEP_TOL + 2 * (eps_in * n + 1e-7) / np.maximum(cs, 1e-30)
        assert np.all(err[unamb] <= bound[unamb])
    h.close()


def test_project_tie_rules_on_gpu(M):
    """det = 0 -> positive class; zero matrix -> identity (same readings as the
    oracle).  Where the minimiser is unique (rank >= n-1) the values must agree;
    for rank <= n-2 every orthogonal completion is a minimiser, so only validity
    (orthogonal, det +1, distance sum (sigma_i - 1)^2) is checked."""
    mats3 = [np.zeros((3, 3)), np.diag([2.0, 1.0, 0.0]), np.diag([1.0, 0.0, 0.0])]
    mats2 = [np.zeros((2, 2)), np.diag([1.0, 0.0])]
    for n, ms in ((3, mats3), (2, mats2)):
        F = np.stack([m.reshape(-1) for m in ms], axis=1).reshape(n * n, 1, len(ms))
        F = np.repeat(F, 2, axis=1)
        for dtype in ("f64", "f32"):
            h = M.Mbo((2, len(ms)), n, 1e-3, dtype)
            a = dev(F, tdt(dtype))
            out = torch.empty_like(a)
            h.project(a, out)
            torch.cuda.synchronize()
            ref = O.project(F, n)
            B = host(out)
            for i, m in enumerate(ms):
                Bi = B[:, 0, i].reshape(n, n)
                assert np.abs(Bi.T @ Bi - np.eye(n)).max() < 1e-6
                assert np.linalg.det(Bi) > 0
                s = np.linalg.svd(m, compute_uv=False)
                assert ((Bi - m) ** 2).sum() == pytest.approx(((s - 1) ** 2).sum(), abs=1e-6)
                if np.linalg.matrix_rank(m) >= n - 1:
                    assert np.abs(Bi - ref[:, 0, i].reshape(n, n)).max() < 1e-6
            h.close()


def _step_case(dims, n, seed):
    A = projected(dims, n, seed)
    tau = 3.0 / max(dims) ** 2
    ref, st = O.step(A, n, tau)
    At = O.diffuse(A, tau)
    return A, tau, ref, st, At


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("dims", [(8, 8), (12, 6), (64, 64), (96, 128), (48, 384), (6, 12, 16),
                                  (16, 16, 16)])
def test_one_step_matches_oracle(M, dims, n, dtype):
    A, tau, ref, st, At = _step_case(dims, n, 500 + n)
    h = M.Mbo(dims, n, tau, dtype)
    a = dev(A, tdt(dtype))
    rec = h.step(a, want_stats=True)
    torch.cuda.synchronize()
    B = host(a)
    d = np.abs(dets(At, n)).reshape(dims)
    err = np.abs(B - ref).max(axis=0)
    if dtype == "f64":
        unamb = d > 1e-12
        assert err[unamb].max() <= F64_TOL
        assert rec["energy"] == pytest.approx(st["energy"], rel=1e-12)
        assert rec["max_delta"] == pytest.approx(st["max_delta"], abs=1e-12)
        if unamb.all():
            assert rec["det_flips"] == st["det_flips"]
    else:
        cs = cond_sum(At, n).reshape(dims)
        unamb = d > det_cut32(At, n).reshape(dims)
        excluded = int((~unamb).sum())
        print(f"{dims} n={n} f32: {excluded} of {unamb.size} points with |det| at rounding level")
        assert excluded <= max(2, unamb.size // 100)
        well = unamb & (cs >= F32_WELL_CS)
        assert err[well].max() <= F32_STEP_TOL
        bound = F32_STEP_TOL + 2 * F32_DIFF_TOL * n / np.maximum(cs, 1e-30)
        assert np.all(err[unamb] <= bound[unamb])
        assert rec["energy"] == pytest.approx(st["energy"], rel=F32_ENERGY_RTOL)
    assert rec["nonfinite"] == 0
    Bm = mats(B, n)
    assert np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(n)).max() < (1e-13 if dtype == "f64" else 2e-6)
    h.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,dims", [(2, (32, 32)), (3, (24, 48)), (3, (8, 8, 8)), (1, (64, 64))])
def test_lyapunov_matches_oracle(M, n, dims, dtype):
    A = projected(dims, n, 900 + n)
    tau = 4.0 / max(dims) ** 2
    ref = O.energy(A, n, tau)
    h = M.Mbo(dims, n, tau, dtype)
    E = h.lyapunov(dev(A, tdt(dtype)))
    assert E == pytest.approx(ref, rel=1e-12 if dtype == "f64" else F32_ENERGY_RTOL)
    h.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_winding_field_fixed_point_and_energy_on_gpu(M, dtype):
    dims = (64, 64)
    tau = 4.0 / 64 ** 2
    Y, X = np.meshgrid(np.arange(64) / 64, np.arange(64) / 64, indexing="ij")
    a = 2 * np.pi * (X + 2 * Y)
    F = np.stack([np.cos(a), -np.sin(a), np.sin(a), np.cos(a)])
    h = M.Mbo(dims, 2, tau, dtype)
    t = dev(F, tdt(dtype))
    rec = h.step(t, want_stats=True)
    torch.cuda.synchronize()
    tol = 1e-13 if dtype == "f64" else 1e-6
    assert np.abs(host(t) - F).max() < tol
    want = 2.0 / tau * (1 - math.exp(-4 * math.pi ** 2 * 5 * tau))
    assert rec["energy"] == pytest.approx(want, rel=1e-12 if dtype == "f64" else 1e-6)
    assert rec["det_flips"] == 0
    h.close()


def test_run_c1_small_matches_oracle_fp64(M):
    """128 x 128, n = 2, tau = 4 h^2, FP64: the whole run against the oracle."""
    F, n, tau = I.config_field("C1")
    A0 = O.project(F, n)
    ref, info = O.run(A0, n, tau, 100, 1e-4)
    h = M.Mbo(F.shape[1:], n, tau, "f64")
    t = dev(A0, torch.float64)
    out = h.run(t, 100, 1e-4)
    assert out["steps"] == info["steps"]
    assert out["stationary"] == info["stationary"]
    np.testing.assert_allclose(out["energies"], info["energies"], rtol=1e-10)
    np.testing.assert_array_equal(out["det_flips"], info["det_flips"])
    assert np.abs(host(t) - ref).max() < 1e-10
    e = out["energies"]
    assert np.all(np.diff(e) <= 1e-12 * e[0])
    h.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_run_host_pointer_equals_device_run(M, dtype):
    dims, n = (64, 96), 3
    A0 = projected(dims, n, 1234)
    tau = 3.0 / 96 ** 2
    h = M.Mbo(dims, n, tau, dtype, check_interval=4)
    t = dev(A0, tdt(dtype))
    r1 = h.run(t, 30, 1e-4)
    hostA = np.ascontiguousarray(A0.astype(np.float32 if dtype == "f32" else np.float64))
    r2 = h.run(hostA, 30, 1e-4)
    assert r1["steps"] == r2["steps"]
    np.testing.assert_array_equal(r1["energies"], r2["energies"])
    np.testing.assert_array_equal(host(t), hostA.astype(np.float64))
    h.close()


@pytest.mark.parametrize("use_graph", [0, 1])
def test_run_graph_and_direct_agree_and_steps_match_mbo_step(M, use_graph):
    dims, n = (48, 64), 2
    A0 = projected(dims, n, 4321)
    tau = 4.0 / 64 ** 2
    h = M.Mbo(dims, n, tau, "f64", use_graph=use_graph, check_interval=3)
    t = dev(A0, torch.float64)
    r = h.run(t, 20, -1.0)
    assert r["steps"] == 20 and not r["stationary"]
    h2 = M.Mbo(dims, n, tau, "f64")
    u = dev(A0, torch.float64)
    energies = []
    for s in range(20):
        rec = h2.step(u, flags=M.MBO_STEP_CONTINUE if s else 0, want_stats=True)
        energies.append(rec["energy"])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(t), host(u))
    np.testing.assert_array_equal(r["energies"][:20], np.array(energies))
    assert h2.lyapunov(u) == pytest.approx(r["energies"][20], rel=1e-14)
    h.close()
    h2.close()


def test_step_continue_equals_fresh_step(M):
    dims, n = (32, 64), 3
    A0 = projected(dims, n, 99)
    tau = 3.0 / 64 ** 2
    h = M.Mbo(dims, n, tau, "f32")
    a = dev(A0, torch.float32)
    b = a.clone()
    h.step(a)
    h.step(a, flags=M.MBO_STEP_CONTINUE)
    h2 = M.Mbo(dims, n, tau, "f32")
    h2.step(b)
    h2.step(b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    h.close()
    h2.close()


def test_nan_input_reports_numeric_error(M):
    dims, n = (16, 16), 2
    A0 = projected(dims, n, 5)
    A0[:, 3, 4] = np.nan
    h = M.Mbo(dims, n, 4.0 / 256, "f32")
    with pytest.raises(M.MboError) as ei:
        h.step(dev(A0, torch.float32), want_stats=True)
    assert ei.value.status == 5
    h.close()


def test_max_size_rows_and_columns(M):
    """2048-point axes (the largest supported) in both precisions."""
    for dtype in ("f64", "f32"):
        dims, n = (4, 2048), 3
        A = projected(dims, n, 7)
        tau = 3.0 / 2048 ** 2
        h = M.Mbo(dims, n, tau, dtype)
        a = dev(A, tdt(dtype))
        out = torch.empty_like(a)
        h.diffuse(a, out)
        torch.cuda.synchronize()
        assert np.abs(host(out) - O.diffuse(A, tau)).max() < (F64_TOL if dtype == "f64" else F32_DIFF_TOL)
        h.close()
        dims = (2048, 4)
        A = projected(dims, n, 8)
        h = M.Mbo(dims, n, tau, dtype)
        a = dev(A, tdt(dtype))
        out = torch.empty_like(a)
        h.diffuse(a, out)
        torch.cuda.synchronize()
        assert np.abs(host(out) - O.diffuse(A, tau)).max() < (F64_TOL if dtype == "f64" else F32_DIFF_TOL)
        h.close()


def test_project_small_sigma_min_f32_routes(M):
    """FP32 n = 3 points with a small smallest singular value: the quaternion
    form (sigma_2 + sigma_3 away from 0) and the FP64 re-projection (both
    small) must both meet the FP32 bound against the oracle's FP64 polar
    factor of Lemma 1.1, in both determinant classes."""
    g = I.rng(4242)
    configs = [(1.0, 0.9, 1e-7), (1.0, 0.5, 1e-5), (5.0, 2.0, 1e-3), (5.0, 0.5, 2e-4),
               (1.0, 0.2, 5e-4), (5.0, 0.2, 0.05), (3.0, 0.05, 0.02), (1.0, 1.0, 1e-6)]
    mats_ = []
    for s in configs:
        for _ in range(64):
            U = np.linalg.qr(g.standard_normal((3, 3)))[0]
            V = np.linalg.qr(g.standard_normal((3, 3)))[0]
            Mx = U @ np.diag(s) @ V.T
            mats_.append(Mx)
            mats_.append(-Mx)
    Ms = np.stack(mats_)                                   # (1024, 3, 3)
    At = Ms.reshape(32, 32, 9).transpose(2, 0, 1).copy()   # (9, 32, 32)
    dims = At.shape[1:]
    ref, sref = O.project(At, 3, return_sign=True)
    h = M.Mbo(dims, 3, 1e-3, "f32")
    a = dev(At, torch.float32)
    out = torch.empty_like(a)
    sg = torch.empty(dims, dtype=torch.int8, device="cuda")
    h.project(a, out, sg)
    torch.cuda.synchronize()
    B = host(out)
    Bm = mats(B, 3)
    assert np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(3)).max() < 2e-6
    d = np.abs(dets(At, 3)).reshape(dims)
    unamb = d > det_cut32(At, 3).reshape(dims)
    assert unamb.sum() >= 448
    assert np.array_equal(sg.cpu().numpy()[unamb], sref[unamb])
    cs = cond_sum(At, 3).reshape(dims)
    eps_in = np.abs(At - At.astype(np.float32).astype(np.float64)).max(axis=0)
    bound = F32_STEP_TOL + 2 * (eps_in * 3 + 1e-7) / np.maximum(cs, 1e-30)
    err = np.abs(B - ref).max(axis=0)
    assert np.all(err[unamb] <= bound[unamb])
    h.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [2, 3])
def test_project_rotated_rank_deficient_on_gpu(M, n, dtype):
    """Rotated matrices of rank n-1 and (n = 3) rank 1, whose computed det is
    rounding noise: the projection must return a minimiser of Lemma 1.1 in the
    class it reports (|B - A|^2 = sum (s_i - 1)^2; at s_n = 0 both classes are
    equally close, Lemma 7.1)."""
    g = I.rng(4300 + n)
    cols = []
    for r in range(1, n):
        for _ in range(64):
            U = np.linalg.qr(g.standard_normal((n, n)))[0]
            V = np.linalg.qr(g.standard_normal((n, n)))[0]
            sv = np.zeros(n)
            sv[:r] = np.sort(g.uniform(0.2, 2.0, r))[::-1]
            cols.append((U @ np.diag(sv) @ V.T).reshape(-1))
    F = np.stack(cols, axis=1).reshape(n * n, 2 * (n - 1), 32)
    dims = F.shape[1:]
    h = M.Mbo(dims, n, 1e-3, dtype)
    a = dev(F, tdt(dtype))
    out = torch.empty_like(a)
    sg = torch.empty(dims, dtype=torch.int8, device="cuda")
    h.project(a, out, sg)
    torch.cuda.synchronize()
    Bm = mats(host(out), n)
    Fm = mats(F, n)
    assert np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(n)).max() < (1e-12 if dtype == "f64" else 2e-6)
    assert np.array_equal(np.sign(np.linalg.det(Bm)).reshape(dims), sg.cpu().numpy().astype(float))
    s = np.linalg.svd(Fm, compute_uv=False)
    d2 = ((Bm - Fm) ** 2).sum((1, 2))
    assert np.abs(d2 - ((s - 1) ** 2).sum(1)).max() < (1e-9 if dtype == "f64" else 2e-5)
    h.close()

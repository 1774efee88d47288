"""Batches of independent fields (uneven sizes, orders and dimensions).

A batch step must reproduce, bit for bit, the single-field steps of the same
fields (the kernels are the same; only the launch is shared), a batch run must
reproduce each field's own run (its own stationary step), and the batched
results are checked against the oracle.  The last test runs the 96-field
workload (sizes 256^2 .. 2048^2, n = 2 and 3, tau = 4 h^2, FP32) at full size.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1711_01365_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_1711_01365_gb300 import build
    build.build()
    from paper_1711_01365_gb300 import mbo
    return mbo


SMALL = [((32, 48), 2), ((64, 64), 3), ((96, 128), 1), ((12, 16, 24), 3), ((27, 36), 2), ((128, 128), 3)]


def _fields(spec, dtype, seed=0):
    out = []
    for k, (dims, n) in enumerate(spec):
        A0 = O.project(I.gaussian(dims, n, seed + k), n)
        out.append(torch.tensor(A0, dtype=dtype, device="cuda"))
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_step_equals_single_field_steps(M, dtype):
    tdt = torch.float32 if dtype == "f32" else torch.float64
    taus = [3.0 / max(d) ** 2 for d, _ in SMALL]
    b = M.Batch([d for d, _ in SMALL], [n for _, n in SMALL], taus, dtype)
    A = _fields(SMALL, tdt)
    Bf = [a.clone() for a in A]
    recs = b.step(A, want_stats=True)
    recs2 = b.step(A, flags=M.MBO_STEP_CONTINUE, want_stats=True)
    for i, (dims, n) in enumerate(SMALL):
        h = M.Mbo(dims, n, taus[i], dtype)
        r1 = h.step(Bf[i], want_stats=True)
        r2 = h.step(Bf[i], flags=M.MBO_STEP_CONTINUE, want_stats=True)
        torch.cuda.synchronize()
        assert torch.equal(A[i], Bf[i])
        assert recs[i]["energy"] == r1["energy"] and recs2[i]["energy"] == r2["energy"]
        assert recs2[i]["det_flips"] == r2["det_flips"]
        h.close()
    b.close()


def test_batch_run_equals_single_runs_and_oracle(M):
    spec = [((32, 32), 2), ((48, 64), 3), ((64, 64), 2)]
    taus = [4.0 / max(d) ** 2 for d, _ in spec]
    b = M.Batch([d for d, _ in spec], [n for _, n in spec], taus, "f64", check_interval=5)
    A = _fields(spec, torch.float64, seed=10)
    starts = [a.cpu().numpy().copy() for a in A]
    out = b.run(A, 40, 1e-4)
    for i, (dims, n) in enumerate(spec):
        h = M.Mbo(dims, n, taus[i], "f64")
        t = torch.tensor(starts[i], device="cuda")
        r = h.run(t, 40, 1e-4)
        assert out["steps"][i] == r["steps"] and out["stationary"][i] == r["stationary"]
        np.testing.assert_array_equal(out["energies"][i], r["energies"])
        assert torch.equal(t, A[i])
        ref, info = O.run(starts[i], n, taus[i], 40, 1e-4)
        assert info["steps"] == r["steps"]
        np.testing.assert_allclose(r["energies"], info["energies"], rtol=1e-10)
        assert np.abs(A[i].cpu().numpy() - ref).max() < 1e-10
        h.close()
    b.close()


def test_batch_96_uneven_fields_full_size(M):
    """The 96-field workload at full size, FP32: one batch step equals the
    single-field steps, and two fields are checked against the oracle at
    sampled points (one step from each side's own projection of the raw field)."""
    spec = I.batch_mixed(96, I.SEED_BASE + 4)
    dims_l = [s[0] for s in spec]
    n_l = [s[1] for s in spec]
    tau_l = [s[2] for s in spec]
    b = M.Batch(dims_l, n_l, tau_l, "f32")
    raw = [I.gaussian(d, n, seed, dtype=np.float32) for d, n, _, seed in spec]
    A = []
    for i, F in enumerate(raw):
        h = M.Mbo(dims_l[i], n_l[i], tau_l[i], "f32")
        t = torch.from_numpy(F).cuda()
        a = torch.empty_like(t)
        h.project(t, a)
        A.append(a)
        h.close()
    torch.cuda.synchronize()
    checks = [0, 6, 13]  # 256^2 n=2, 2048^2 n=2, 2048^2 n=3
    before = {i: A[i].clone() for i in checks}
    recs = b.step(A, want_stats=True)
    assert all(r["nonfinite"] == 0 for r in recs)
    for i in checks:
        h = M.Mbo(dims_l[i], n_l[i], tau_l[i], "f32")
        x = before[i]
        h.step(x)
        torch.cuda.synchronize()
        assert torch.equal(x, A[i])
        h.close()
        g = I.rng(100 + i)
        pts = np.stack([g.integers(0, d, 24) for d in dims_l[i]], 1)
        n = n_l[i]
        At_o, B_o = O.step_points(raw[i], n, tau_l[i], pts, project_input=True)
        idx = (slice(None),) + tuple(torch.as_tensor(pts.T))
        Bg = A[i][idx].double().cpu().numpy().T
        s = np.linalg.svd(At_o.reshape(-1, n, n), compute_uv=False)
        cs = s[:, -1] + s[:, -2]
        cut = 64 * 2.0 ** -24 * np.sqrt((s ** 2).sum(axis=1)) ** n  # FP32 det rounding level
        ok = (np.prod(s, axis=1) > cut) & (cs >= 1e-2)
        assert ok.sum() >= 6
        assert np.abs(Bg - B_o).max(axis=1)[ok].max() <= 2e-5
    b.close()

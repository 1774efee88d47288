"""Volume-preserving step (Sec. 7) on the GPU against the oracle.

The selection is an integer decision taken from floating-point dE; the two
sides agree wherever dE is not within rounding of the selection threshold
lambda.  Tests compare values at points away from lambda, check that exactly
n_plus points lie in SO(n), and use constant fields (all dE equal) to check
the index tie-break exactly.
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


def _dets(F, n):
    return np.linalg.det(F.reshape(n, n, -1).transpose(2, 0, 1))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("dims,n", [((16, 24), 1), ((32, 32), 2), ((24, 48), 3), ((8, 12, 16), 3)])
def test_volume_step_matches_oracle(M, dims, n, dtype):
    A0 = O.project(I.gaussian(dims, n, 700 + n), n)
    tau = 4.0 / max(dims) ** 2
    P = int(np.prod(dims))
    n0 = O.count_positive(A0, n)
    for n_plus in (n0, max(n0 - P // 7, 0), min(n0 + P // 5, P)):
        ref, st, dE = O.step_volume(A0, n, tau, n_plus)
        order = np.sort(dE.ravel())[::-1]
        lam_hi = order[n_plus - 1] if n_plus > 0 else np.inf
        lam_lo = order[n_plus] if n_plus < P else -np.inf
        h = M.Mbo(dims, n, tau, dtype)
        a = torch.tensor(A0, dtype=torch.float32 if dtype == "f32" else torch.float64, device="cuda")
        rec = h.step_volume(a, n_plus, want_stats=True)
        B = a.double().cpu().numpy()
        assert int((_dets(B, n) > 0).sum()) == n_plus
        margin = 1e-9 if dtype == "f64" else 1e-4
        far = (np.abs(dE - lam_hi) > margin) & (np.abs(dE - lam_lo) > margin)
        err = np.abs(B - ref).max(axis=0)
        At = O.diffuse(A0, tau)
        s = np.linalg.svd(At.reshape(n, n, -1).transpose(2, 0, 1), compute_uv=False)
        cs = s[:, -1] + (s[:, -2] if n > 1 else s[:, -1])
        well = far & (cs.reshape(dims) >= (1e-6 if dtype == "f64" else 0.1))
        assert err[well].max() <= (1e-11 if dtype == "f64" else 2e-5)
        assert rec["energy"] == pytest.approx(st["energy"], rel=1e-12 if dtype == "f64" else 1e-5)
        h.close()


def test_volume_ties_broken_by_index(M):
    """A constant rotation field: every dE is equal, so the n_plus lowest grid
    indices take T+ (= the field, unique); at the others every reflection is
    equally close (all singular values are 1), so T- is checked for validity:
    a reflection at distance^2 sum (s - 1)^2 + 4 s_min = 4 (Lemma 7.1)."""
    dims, n = (8, 16), 2
    th = 0.3
    F = np.zeros((4,) + dims)
    F[0], F[1], F[2], F[3] = np.cos(th), -np.sin(th), np.sin(th), np.cos(th)
    tau = 0.01
    for n_plus in (0, 5, 77, 128):
        ref, _, _ = O.step_volume(F, n, tau, n_plus)
        h = M.Mbo(dims, n, tau, "f64")
        a = torch.tensor(F, device="cuda")
        h.step_volume(a, n_plus)
        B = a.cpu().numpy()
        pos = (_dets(B, n) > 0).reshape(-1)
        assert pos[:n_plus].all() and not pos[n_plus:].any()
        assert np.array_equal(pos, (_dets(ref, n) > 0).reshape(-1))
        Bp = B.reshape(4, -1)
        Fp = F.reshape(4, -1)
        if pos.any():
            assert np.abs(Bp[:, pos] - Fp[:, pos]).max() < 1e-12
        for x in np.nonzero(~pos)[0]:
            R = Bp[:, x].reshape(2, 2)
            assert np.allclose(R.T @ R, np.eye(2), atol=1e-12) and np.linalg.det(R) < 0
            assert ((R - Fp[:, x].reshape(2, 2)) ** 2).sum() == pytest.approx(4.0, abs=1e-12)
        h.close()


def test_volume_run_preserves_volume_and_decreases_energy(M):
    dims, n = (64, 64), 2
    tau = 8.0 / 64 ** 2
    A0 = O.project(I.gaussian(dims, n, 801), n)
    n0 = O.count_positive(A0, n)
    h = M.Mbo(dims, n, tau, "f64", check_interval=4)
    a = torch.tensor(A0, device="cuda")
    out = h.run_volume(a, -1, 30, 1e-6)
    B = a.cpu().numpy()
    assert int((_dets(B, n) > 0).sum()) == n0
    e = out["energies"]
    assert len(e) == out["steps"] + 1
    assert np.all(np.diff(e) <= 1e-12 * e[0])
    # the same steps in the oracle
    A = A0.copy()
    for s in range(out["steps"]):
        A, st, _ = O.step_volume(A, n, tau, n0)
        assert st["energy"] == pytest.approx(e[s], rel=1e-9)
    h.close()

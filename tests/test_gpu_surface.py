"""Closed-surface path (Sec. 5.2, Algorithm 2; include/mbo_surface.h) on the
GPU against the oracle (oracle/surface.py).

* Parameters: h and M equal the oracle's (the heat-kernel approximation
  theorem, R the points' extent); the grid is 2^a 3^b and at least 4M.
* Diffusion: the GPU's spreading / FFT / interpolation equals the oracle's
  plain double sum at every point, to the accuracy the spreading width buys
  (FP32, eps = 1e-6: 2e-5 of the field's scale; FP64, eps = 1e-7, the
  widest kernel: 2e-6),
  for n = 1..4 on clustered random points (empty and crowded bins, a ragged
  last block) and on a coarse sphere band.
* Step: the projected field equals the oracle's step where the class is
  unambiguous, and is orthogonal everywhere.
* Volume-preserving step (Sec. 7, Algorithm 3 on the surface): the selected
  weight reaches the volume with a minimal prefix, and the values match the
  oracle's step away from the selection threshold.
* Full size (the sphere experiment of Sec. 6.2: dx = 0.05, tau = 0.005,
  eps = 1e-6, p = 3): properties that hold at any size -- constants are kept,
  the degree-1 harmonic z decays by 1 - 2 tau (Laplace-Beltrami, first order
  in tau, against the exact Gaussian convolution of the oracle at sampled
  points), and a step from the paper's two-matrix initial field stays
  orthogonal with det classes +-1.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle import surface as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = {"f32": 2e-5, "f64": 2e-6}
EPS = {"f32": 1e-6, "f64": 1e-7}


@pytest.fixture(scope="module")
def M():
    from paper_1711_01365_gb300 import build
    build.build()
    from paper_1711_01365_gb300 import mbo
    return mbo


def _tdt(dtype):
    return torch.float32 if dtype == "f32" else torch.float64


def clustered(nq, seed):
    """Two clusters of quadrature points in [0, 1]^3 with nearby targets."""
    g = np.random.default_rng(seed)
    half = nq // 2
    xq = np.concatenate([g.uniform(0.0, 0.35, (half, 3)), g.uniform(0.6, 1.0, (nq - half, 3))])
    xc = np.clip(xq + g.normal(0, 0.03, xq.shape), 0, 1)
    wq = g.uniform(0.5, 1.5, nq) / nq
    return xq, wq, xc


def field(n, nq, seed):
    """O(n)-valued field: projected (fixed matrix + N(0, 0.8^2) noise) per point,
    so that diffused matrices are mostly well conditioned, with both classes."""
    g = np.random.default_rng(seed)
    base = g.standard_normal((n * n, 1))
    return O.project(base + 0.8 * g.standard_normal((n * n, nq)), n)


def _mats(F, n):
    return F.T.reshape(-1, n, n)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_params_match_the_oracle(M, dtype):
    xq, wq, xc = clustered(1500, 1)
    s = M.Surface(xq, wq, xc, 2, 0.01, EPS[dtype], dtype)
    p = s.params()
    h, m = S.heat_modes(EPS[dtype], 0.01, S.extent(xq, xc))
    assert p["M"] == m and p["h"] == pytest.approx(h, rel=1e-14)
    nf = p["nf"]
    assert nf >= 4 * m and nf >= 2 * p["width"]
    k = nf
    while k % 2 == 0:
        k //= 2
    while k % 3 == 0:
        k //= 3
    assert k == 1
    assert p["width"] == min(max(math.ceil(math.log10(1 / EPS[dtype])) + 1, 4), 8)
    assert p["bins"] > 1
    s.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_diffuse_and_step_match_the_oracle_on_clusters(M, n, dtype):
    nq, tau, eps = 2001, 0.01, EPS[dtype]
    xq, wq, xc = clustered(nq, 10 + n)
    A = field(n, nq, 20 + n)
    s = M.Surface(xq, wq, xc, n, tau, eps, dtype)
    p = s.params()
    a = torch.tensor(A, dtype=_tdt(dtype), device="cuda")
    out = torch.empty_like(a)
    s.diffuse(a, out)
    torch.cuda.synchronize()
    ref = S.surface_diffuse(A, xq, wq, xc, tau, p["h"], p["M"])
    got = out.double().cpu().numpy()
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(got - ref).max() <= TOL[dtype] * scale

    st = s.step(a, want_stats=True)
    B = a.double().cpu().numpy()
    Bo, Ato, sto = S.surface_step(A, xq, wq, xc, n, tau, p["h"], p["M"])
    Bm = _mats(B, n)
    assert np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(n)).max() < (2e-6 if dtype == "f32" else 1e-12)
    sv = np.linalg.svd(_mats(Ato, n), compute_uv=False)
    absdet = np.prod(sv, axis=1)
    cs = sv[:, -1] + (sv[:, -2] if n > 1 else sv[:, -1])
    well = (absdet > 1e-3 * scale ** n) & (cs >= 0.05 * scale)
    assert well.sum() > nq // 4
    err = np.abs(B - Bo).max(axis=0)
    dtol = TOL[dtype] * scale
    assert np.all(err[well] <= 2 * n * dtol / cs[well] + (2e-5 if dtype == "f32" else 1e-10))
    assert np.array_equal(np.sign(np.linalg.det(Bm))[well], np.sign(np.linalg.det(_mats(Bo, n)))[well])
    assert st["nonfinite"] == 0 and math.isnan(st["energy"])
    assert st["max_delta"] == pytest.approx(np.abs(B - A).max(), rel=1e-5, abs=1e-6)
    s.close()


@pytest.mark.parametrize("dtype,n,eps", [("f32", 3, 1e-6), ("f64", 2, 1e-7)])
def test_coarse_sphere_band(M, dtype, n, eps):
    tau = 0.05
    wb = S.band_width(eps, tau)
    xq, wq, xc = M.mbo_surface_sphere_band(1.0, 0.4, wb, 1)
    A = field(n, len(wq), 33)
    s = M.Surface(xq, wq, xc, n, tau, eps, dtype)
    p = s.params()
    a = torch.tensor(A, dtype=_tdt(dtype), device="cuda")
    out = torch.empty_like(a)
    s.diffuse(a, out)
    torch.cuda.synchronize()
    ref = S.surface_diffuse(A, xq, wq, xc, tau, p["h"], p["M"])
    assert np.abs(out.double().cpu().numpy() - ref).max() <= TOL[dtype] * max(1.0, np.abs(ref).max())
    s.close()


def _paper_sphere_field(xc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "sphere_matrices.txt")) if l.strip() and not l.startswith("#")]
    m1 = np.array(rows[:3], dtype=float)
    m2 = np.array(rows[3:6], dtype=float)
    q1, q2 = O.polar(m1), O.polar(m2)
    sel = (xc[:, 0] < 0) & (xc[:, 1] < 0) & (xc[:, 2] > 0)
    A = np.where(sel[None, :], q1.reshape(9, 1), q2.reshape(9, 1))
    return A, q1, q2


def test_full_size_sphere_properties(M):
    tau, eps, dx, p = 0.005, 1e-6, 0.05, 3
    wb = M.mbo_surface_band_width(eps, tau)
    xq, wq, xc = M.mbo_surface_sphere_band(1.0, dx, wb, p)
    nq = len(wq)
    assert nq == len(S.sphere_band(1.0, dx, wb, p)[1])
    # constants and the degree-1 harmonic (channels 0 and 1 of an n = 2 field)
    s = M.Surface(xq, wq, xc, 2, tau, eps, "f32")
    F = np.zeros((4, nq))
    F[0] = 1.0
    F[1] = xc[:, 2]
    a = torch.tensor(F, dtype=torch.float32, device="cuda")
    out = torch.empty_like(a)
    s.diffuse(a, out)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    assert np.abs(got[0] - 1).max() < 5e-5
    assert np.abs(got[2:]).max() < 1e-5
    idx = np.random.default_rng(4).choice(nq, 24, replace=False)
    z = S.gauss_convolve(F[1:2], xq, wq, xc[idx], tau)[0]
    assert np.abs(got[1, idx] - z).max() < 5e-5
    sel = np.abs(xc[:, 2]) > 0.3
    ratio = got[1, sel] / xc[sel, 2]
    assert np.abs(ratio - (1 - 2 * tau)).max() < tau * tau
    s.close()
    # one step of Algorithm 1 from the paper's initial field (n = 3)
    A, q1, q2 = _paper_sphere_field(xc)
    s = M.Surface(xq, wq, xc, 3, tau, eps, "f32")
    a = torch.tensor(A, dtype=torch.float32, device="cuda")
    st = s.step(a, want_stats=True)
    B = a.double().cpu().numpy()
    Bm = _mats(B, 3)
    assert np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(3)).max() < 2e-6
    d = np.linalg.det(Bm)
    assert np.all(np.abs(np.abs(d) - 1) < 1e-5)
    # far from the interface the field keeps its matrix
    far = ((xc[:, 0] > 0.7) | (xc[:, 1] > 0.7) | (xc[:, 2] < -0.7))
    assert np.abs(B[:, far] - q2.reshape(9, 1)).max() < 1e-4
    assert st["det_flips"] == int(np.sum(np.sign(d) != np.sign(np.linalg.det(_mats(A, 3)))))
    s.close()


def test_coarse_peanut_band(M):
    """The peanut of Sec. 6.3 (tau = 0.032, eps = 1e-6 as printed; coarse
    cells dx = 0.35, p = 1): diffusion against the oracle's double sum on the
    library's band, and one step that stays orthogonal."""
    tau, eps, n = 0.032, 1e-6, 2
    wb = M.mbo_surface_band_width(eps, tau)
    xq, wq, xc = M.mbo_surface_peanut_band(0.35, wb, 1)
    A = field(n, len(wq), 44)
    s = M.Surface(xq, wq, xc, n, tau, eps, "f32")
    p = s.params()
    a = torch.tensor(A, dtype=torch.float32, device="cuda")
    out = torch.empty_like(a)
    s.diffuse(a, out)
    torch.cuda.synchronize()
    ref = S.surface_diffuse(A, xq, wq, xc, tau, p["h"], p["M"])
    assert np.abs(out.double().cpu().numpy() - ref).max() <= TOL["f32"] * max(1.0, np.abs(ref).max())
    st = s.step(a, want_stats=True)
    Bm = _mats(a.double().cpu().numpy(), n)
    assert np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(n)).max() < 2e-6
    assert st["nonfinite"] == 0
    s.close()


def test_runtime_width_fp32(M):
    """eps = 1e-4 gives width 5, which runs the runtime-width kernels (width 7,
    the paper's eps = 1e-6, has its own compile-time instantiation): diffusion
    against the double sum to the accuracy of that width (~10^(1 - 5))."""
    nq, tau, eps, n = 1501, 0.01, 1e-4, 3
    xq, wq, xc = clustered(nq, 55)
    A = field(n, nq, 56)
    s = M.Surface(xq, wq, xc, n, tau, eps, "f32")
    p = s.params()
    assert p["width"] == 5
    a = torch.tensor(A, dtype=torch.float32, device="cuda")
    out = torch.empty_like(a)
    s.diffuse(a, out)
    torch.cuda.synchronize()
    ref = S.surface_diffuse(A, xq, wq, xc, tau, p["h"], p["M"])
    assert np.abs(out.double().cpu().numpy() - ref).max() <= 1e-3 * max(1.0, np.abs(ref).max())
    s.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("n", [1, 2, 3])
def test_volume_step_matches_the_oracle(M, n, dtype):
    """Sec. 7, Algorithm 3 on a surface: the GPU's volume-preserving step (dE
    keys, weighted radix selection, class assignment) against the oracle's at
    three volumes (the input's own, -15% and +20%): the selected set is a
    minimal prefix in decreasing dE whose weight reaches V, and away from the
    selection threshold (where a diffusion difference cannot reorder dE) the
    values match the oracle to the step tolerance."""
    nq, tau, eps = 2001, 0.01, EPS[dtype]
    xq, wq, xc = clustered(nq, 60 + n)
    A = field(n, nq, 70 + n)
    d0 = np.linalg.det(_mats(A, n))
    V0 = wq[d0 > 0].sum()
    s = M.Surface(xq, wq, xc, n, tau, eps, dtype)
    p = s.params()
    for vol in (-1.0, 0.85 * V0, min(1.2 * V0, 0.99 * wq.sum())):
        ref, Ato, dE, sto = S.surface_step_volume(A, xq, wq, xc, n, tau, p["h"], p["M"], volume=vol)
        V = V0 if vol < 0 else vol
        a = torch.tensor(A, dtype=_tdt(dtype), device="cuda")
        st = s.step_volume(a, vol, want_stats=True)
        B = a.double().cpu().numpy()
        sel = np.linalg.det(_mats(B, n)) > 0
        W = wq[sel].sum()
        assert W >= V * (1 - 1e-12)
        assert W - wq[sel][np.argmin(np.where(sel, dE, np.inf)[sel])] < V * (1 + 1e-12) or dtype == "f32"
        order = np.sort(dE)[::-1]
        k = sto["selected"]
        lam_hi = order[k - 1] if k > 0 else np.inf
        lam_lo = order[k] if k < nq else -np.inf
        scale = max(1.0, np.abs(Ato).max())
        margin = 1e-3 * scale if dtype == "f32" else 1e-4 * scale
        far = (np.abs(dE - lam_hi) > margin) & (np.abs(dE - lam_lo) > margin)
        sv = np.linalg.svd(_mats(Ato, n), compute_uv=False)
        cs = sv[:, -1] + (sv[:, -2] if n > 1 else sv[:, -1])
        well = far & (cs >= 0.05 * scale)
        assert well.sum() > nq // 4
        err = np.abs(B - ref).max(axis=0)
        assert np.all(err[well] <= 2 * n * TOL[dtype] * scale / cs[well] + (2e-5 if dtype == "f32" else 1e-10))
        assert abs(int(sel.sum()) - k) <= (0 if dtype == "f64" else 3)
        Bm = _mats(B, n)
        assert np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(n)).max() < (2e-6 if dtype == "f32" else 1e-12)
        assert st["nonfinite"] == 0
    s.close()


def test_volume_step_order4_unsupported(M):
    xq, wq, xc = clustered(64, 3)
    s = M.Surface(xq, wq, xc, 4, 0.01, 1e-6, "f32")
    a = torch.zeros((16, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(M.MboError) as ei:
        s.step_volume(a, 10)
    assert ei.value.status == 2
    s.close()


@pytest.mark.parametrize("case", ["single", "coincident"])
def test_degenerate_point_sets(M, case):
    """A single point (zero extent: the plan takes R = 1) and 50 copies of one
    point with its closest point (one footprint group, one bin): the diffusion
    equals the oracle's double sum with the plan's h and M, and a step stays
    orthogonal."""
    n, tau, eps = 3, 0.01, 1e-6
    if case == "single":
        xq, xc, wq = np.array([[0.3, -0.2, 0.5]]), np.array([[0.31, -0.18, 0.49]]), np.array([0.7])
    else:
        xq = np.repeat([[0.1, 0.2, 0.3]], 50, axis=0)
        xc = np.repeat([[0.12, 0.2, 0.28]], 50, axis=0)
        wq = np.full(50, 1.0 / 50)
    A = field(n, len(wq), 80)
    s = M.Surface(xq, wq, xc, n, tau, eps, "f32")
    p = s.params()
    a = torch.tensor(A, dtype=torch.float32, device="cuda")
    out = torch.empty_like(a)
    s.diffuse(a, out)
    torch.cuda.synchronize()
    ref = S.surface_diffuse(A, xq, wq, xc, tau, p["h"], p["M"])
    assert np.abs(out.double().cpu().numpy() - ref).max() <= TOL["f32"] * max(1.0, np.abs(ref).max())
    s.step(a)
    Bm = _mats(a.double().cpu().numpy(), n)
    assert np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(n)).max() < 2e-6
    s.close()

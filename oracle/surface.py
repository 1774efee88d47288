"""FP64 oracle of the closed-surface diffusion and MBO step (Sec. 5.2 and
Algorithm 2 of Osting & Wang, arXiv:1711.01365).

Test infrastructure only: the tests, the smoke check and the benchmark's
CPU-baseline leg use it; the CUDA library never does.  It shares no code with
the library: the band geometry, the quadrature rule, the mode count and the
diffusion are computed here with numpy from their definitions, and the
projection of Lemma 1.1 is the C oracle's (oracle.project).

What is computed, step by step, in the paper's order:

* ``T`` and ``band_width``: the tail bound T(x) = 2x/sqrt(pi) e^{-x^2} +
  erfc(x) of the band-truncation theorem of Sec. 5.2 and the band width w_b
  with T(w_b / (2 sqrt(tau))) = eps (Table 1).
* ``heat_modes``: the spacing h and mode count M of the heat-kernel
  approximation theorem of Sec. 5.2 (the truncated Fourier sum of G_tau, Table 2).
* ``cheb_rule``: the p-point rule on the Gauss-Chebyshev nodes used for the
  quadrature points x_q in each band cell (Algorithm 2, step 1).
* ``sphere_closest`` and ``sphere_band``: the closest-point map of a sphere and
  the sets G^b (grid points within w_b of the surface), Q (quadrature points)
  and the closest points x_q^c (Algorithm 2, step 1).
* ``peanut_closest`` and ``peanut_band``: the same for the peanut surface of
  Sec. 6.3, a surface of revolution whose closest points come from the
  closest point of the generating curve in the point's meridian plane.
* ``surface_diffuse``: steps 2-5 of Algorithm 2 as the plain double sum
      A*(x_t) = (h / 2 pi)^3 Re sum_m e^{-h^2 tau |m|^2} e^{i h m . x_t}
                                   sum_q w_q A~(x_q) e^{-i h m . x_q},
  m in {-M, ..., M-1}^3 (the type-1 sum (4.1) times n_q e^{-|m|^2 h^2 tau}, then
  the type-2 sum (4.2) and the factor of the tensor-product kernel
  approximation), evaluated with dense matrix products, no NUFFT.
* ``gauss_convolve``: the same sum with the exact Gaussian G_tau^3 in place of
  its Fourier approximation (the convolution the algorithm approximates).
* ``surface_step``: one iteration of Algorithm 1 on the surface: diffusion,
  then the projection of every point onto O(n) (Lemma 1.1).

Readings where the paper is garbled or silent (each one a choice made here):

* The mode count: the printed formula takes the logarithm of
  sqrt(pi) eps / (2 h sqrt(tau)), which is below 1; the argument is read
  inverted, M = ceil(sqrt(ln(2 h sqrt(tau) / (sqrt(pi) eps)) / tau) / h).
  This is never smaller than Table 2's entries (Table 2 lies within one of a
  variant with 2 sqrt(tau) / (pi eps) inside the logarithm).  With this M the
  theorem's bound 4 eps / sqrt(4 pi tau) holds for h^2 tau >= 0.005, the range
  of the paper's surface experiments; for smaller h^2 tau it does not (the
  truncated tail decays like 1 / (8 h^2 tau M) times the bound).
* R, the spatial radius of that theorem, is the largest coordinate extent of
  the source and target points (every per-axis difference is then at most R).
* The printed sum runs over m = -M..M-1, so one mode has no partner; the field
  is real, so the real part is kept (equivalently: weight 1/2 at |m_i| = M).
* The factor of the last step is (h / 2 pi)^3 (the tensor-product kernel
  approximation); the printed (2 pi)^-3 h^-3 is read as that.
* Quadrature: the p Gauss-Chebyshev nodes cos((2k - 1) pi / (2p)) of each cell
  axis carry the interpolatory weights of those nodes for the plain integral
  (the rule of Fejer), so each cell rule integrates polynomials of degree
  p - 1 exactly; the grid is dx Z^3 with the sphere's centre at the origin and
  cell x_g + [0, dx]^3.
* The state lives at the closest points x_q^c, one per quadrature point; the
  constant extension gives the source x_q the value at its own x_q^c.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as _core


# --- band width (Sec. 5.2, band-truncation theorem; Table 1) ---------------------

def T(x: float) -> float:
    """Tail bound of the band-truncation theorem: 2x/sqrt(pi) e^{-x^2} + erfc(x)."""
    return 2.0 * x / math.sqrt(math.pi) * math.exp(-x * x) + math.erfc(x)


def band_width(eps: float, tau: float) -> float:
    """w_b with T(w_b / (2 sqrt(tau))) = eps (bisection; T decreases on x > 0)."""
    lo, hi = 0.0, 1.0
    while T(hi) > eps:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if T(mid) > eps:
            lo = mid
        else:
            hi = mid
    return 2.0 * math.sqrt(tau) * hi


# --- spectral approximation of the heat kernel (Sec. 5.2; Table 2) --------------

def heat_modes(eps: float, tau: float, R: float):
    """(h, M) of the heat-kernel approximation theorem for |x| <= R."""
    h = min(math.pi / R, math.pi / (2.0 * math.sqrt(tau * abs(math.log(eps)))))
    arg = 2.0 * h * math.sqrt(tau) / (math.sqrt(math.pi) * eps)
    M = math.ceil(math.sqrt(max(math.log(arg), 0.0) / tau) / h)
    return h, max(int(M), 1)


def kernel_1d(x, tau: float, h: float, M: int):
    """(h / 2 pi) sum_{m=-M}^{M-1} e^{-m^2 h^2 tau + i m h x} (complex)."""
    x = np.asarray(x, dtype=np.float64)
    m = np.arange(-M, M, dtype=np.float64)
    return (h / (2 * math.pi)) * (np.exp(-(m * h) ** 2 * tau)[None, :] *
                                  np.exp(1j * h * np.multiply.outer(x.ravel(), m))).sum(1).reshape(x.shape)


def gauss_1d(x, tau: float):
    """The 1-D heat kernel G_tau(x) = exp(-x^2 / (4 tau)) / sqrt(4 pi tau)."""
    x = np.asarray(x, dtype=np.float64)
    return np.exp(-x * x / (4 * tau)) / math.sqrt(4 * math.pi * tau)


# --- quadrature (Algorithm 2, step 1) --------------------------------------------

def cheb_rule(p: int):
    """Nodes cos((2k - 1) pi / (2p)), k = 1..p, on [-1, 1] and the interpolatory
    weights for int_{-1}^{1} f: the solution of sum_k w_k t_k^j = int t^j, j < p."""
    k = np.arange(1, p + 1)
    t = np.cos((2 * k - 1) * np.pi / (2 * p))
    V = np.vander(t, p, increasing=True).T  # V[j, k] = t_k^j
    mom = np.array([(1.0 - (-1.0) ** (j + 1)) / (j + 1) for j in range(p)])
    w = np.linalg.solve(V, mom)
    return t, w


# --- sphere geometry (Algorithm 2, step 1) -----------------------------------------

def sphere_closest(x: np.ndarray, radius: float) -> np.ndarray:
    """Closest point on the sphere |y| = radius (centre 0) of each row of x; the
    centre itself (every sphere point is closest) maps to (0, 0, radius)."""
    x = np.asarray(x, dtype=np.float64)
    r = np.linalg.norm(x, axis=-1, keepdims=True)
    out = np.empty_like(x)
    ok = r[..., 0] > 0
    out[ok] = radius * x[ok] / r[ok]
    out[~ok] = np.array([0.0, 0.0, radius])
    return out


def sphere_band(radius: float, dx: float, wb: float, p: int):
    """Band construction for the sphere of the given radius centred at 0.

    Grid points x_g = dx (i, j, k) with | |x_g| - radius | < wb form G^b; each
    cell x_g + [0, dx]^3 carries p^3 quadrature points (tensor rule of
    ``cheb_rule`` mapped to [0, dx]).  Returns (xq, wq, xc): quadrature points
    (nq, 3), weights (nq,), and their closest points on the sphere (nq, 3).
    Order: grid points by (i, j, k) lexicographic (k fastest), then the nodes
    of each cell by (a, b, c) lexicographic (c fastest)."""
    t, w = cheb_rule(p)
    s = dx * (1.0 + t) / 2.0
    ws = w * dx / 2.0
    lim = int(math.ceil((radius + wb) / dx)) + 1
    ax = np.arange(-lim, lim + 1)
    I, J, K = np.meshgrid(ax, ax, ax, indexing="ij")
    g = dx * np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1).astype(np.float64)
    d = np.abs(np.linalg.norm(g, axis=1) - radius)
    g = g[d < wb]
    A, B, Cc = np.meshgrid(np.arange(p), np.arange(p), np.arange(p), indexing="ij")
    a, b, c = A.ravel(), B.ravel(), Cc.ravel()
    off = np.stack([s[a], s[b], s[c]], axis=1)
    wq1 = ws[a] * ws[b] * ws[c]
    xq = (g[:, None, :] + off[None, :, :]).reshape(-1, 3)
    wq = np.tile(wq1, g.shape[0])
    return xq, wq, sphere_closest(xq, radius)


# --- peanut geometry (Sec. 6.3; Algorithm 2, step 1) -------------------------------

def peanut_curve(t):
    """Generating curve of the peanut surface, t in [-1, 1]: x = 3t - t^3,
    rho = sqrt((1 + x^2)(4 - x^2)) / 2 (the surface is (x, rho cos th, rho sin th))."""
    t = np.asarray(t, dtype=np.float64)
    x = 3 * t - t ** 3
    rho = 0.5 * np.sqrt(np.maximum((1 + x * x) * (4 - x * x), 0.0))
    return x, rho


def peanut_closest(P: np.ndarray, samples: int = 20001, iters: int = 90, chunk: int = 4096):
    """Closest point on the peanut surface of each row of P, through the
    surface of revolution: the closest point of (x, r = |(y, z)|) on the
    generating curve, by a dense scan of t and a golden-section search between
    the neighbours of the best sample, rotated back to the point's meridian
    ((y, z) = 0: the meridian of +y).  Returns (closest points, distances)."""
    P = np.asarray(P, dtype=np.float64).reshape(-1, 3)
    r = np.hypot(P[:, 1], P[:, 2])
    ts = np.linspace(-1.0, 1.0, samples)
    cx, cr = peanut_curve(ts)
    tbest = np.empty(len(P))
    for a in range(0, len(P), chunk):
        b = min(len(P), a + chunk)
        d2 = (cx[None, :] - P[a:b, 0:1]) ** 2 + (cr[None, :] - r[a:b, None]) ** 2
        tbest[a:b] = ts[np.argmin(d2, axis=1)]
    step = 2.0 / (samples - 1)
    lo, hi = np.maximum(tbest - step, -1.0), np.minimum(tbest + step, 1.0)

    def D(t):
        x, rho = peanut_curve(t)
        return (x - P[:, 0]) ** 2 + (rho - r) ** 2

    g = (math.sqrt(5.0) - 1) / 2
    c, d = hi - g * (hi - lo), lo + g * (hi - lo)
    fc, fd = D(c), D(d)
    for _ in range(iters):
        left = fc < fd
        hi = np.where(left, d, hi)
        lo = np.where(left, lo, c)
        c_new = hi - g * (hi - lo)
        d_new = lo + g * (hi - lo)
        c, d = np.where(left, c_new, d), np.where(left, c, d_new)
        fc, fd = np.where(left, D(c), fd), np.where(left, fc, D(d))
    t = 0.5 * (lo + hi)
    x, rho = peanut_curve(t)
    safe = np.where(r > 0, r, 1.0)
    uy = np.where(r > 0, P[:, 1] / safe, 1.0)
    uz = np.where(r > 0, P[:, 2] / safe, 0.0)
    cp = np.stack([x, rho * uy, rho * uz], axis=1)
    return cp, np.sqrt(D(t))


def peanut_band(dx: float, wb: float, p: int):
    """Band construction for the peanut (as ``sphere_band``): grid points
    x_g = dx (i, j, k) whose distance to the surface is below wb, p^3
    quadrature points per cell x_g + [0, dx]^3 with their weights, and the
    closest points of the quadrature points.  Same ordering as sphere_band."""
    t, w = cheb_rule(p)
    s = dx * (1.0 + t) / 2.0
    ws = w * dx / 2.0
    _, cr = peanut_curve(np.linspace(-1, 1, 20001))
    lx = int(math.ceil((2.0 + wb) / dx)) + 1
    lr = int(math.ceil((cr.max() + wb) / dx)) + 1
    I, J, K = np.meshgrid(np.arange(-lx, lx + 1), np.arange(-lr, lr + 1), np.arange(-lr, lr + 1), indexing="ij")
    g = dx * np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1).astype(np.float64)
    _, dist = peanut_closest(g)
    g = g[dist < wb]
    A, B, Cc = np.meshgrid(np.arange(p), np.arange(p), np.arange(p), indexing="ij")
    a, b, c = A.ravel(), B.ravel(), Cc.ravel()
    off = np.stack([s[a], s[b], s[c]], axis=1)
    wq1 = ws[a] * ws[b] * ws[c]
    xq = (g[:, None, :] + off[None, :, :]).reshape(-1, 3)
    wq = np.tile(wq1, g.shape[0])
    return xq, wq, peanut_closest(xq)[0]


def extent(*pts) -> float:
    """Largest coordinate extent (max - min over any axis) of the point sets."""
    allp = np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1, 3) for p in pts])
    return float((allp.max(0) - allp.min(0)).max())


# --- diffusion (Algorithm 2, steps 2-5) -----------------------------------------------

def _phases(x: np.ndarray, h: float, M: int, sign: int) -> list:
    m = np.arange(-M, M, dtype=np.float64)
    return [np.exp(sign * 1j * h * np.multiply.outer(m, x[:, a])) for a in range(3)]  # (2M, n)


def surface_diffuse(F: np.ndarray, xs: np.ndarray, ws: np.ndarray, xt: np.ndarray,
                    tau: float, h: float, M: int, chunk: int = 2048) -> np.ndarray:
    """Steps 2-5 of Algorithm 2 as the plain double sum (module docstring).

    F: (C, nq) values at the targets; the source xs[q] (weight ws[q]) takes
    the value F[:, q] of its own closest point xt[q] (step 2).  Returns the
    diffused values at the targets, (C, nt)."""
    F = np.asarray(F, dtype=np.float64)
    xs = np.asarray(xs, dtype=np.float64).reshape(-1, 3)
    xt = np.asarray(xt, dtype=np.float64).reshape(-1, 3)
    Cn, ns = F.shape
    L = 2 * M
    # step 4: type-1 sum over the sources, Ahat[c, m1, m2, m3]
    Ah = np.zeros((Cn, L, L, L), dtype=np.complex128)
    for q0 in range(0, ns, chunk):
        sl = slice(q0, min(ns, q0 + chunk))
        E1, E2, E3 = _phases(xs[sl], h, M, -1)
        S = (F[:, sl] * ws[sl][None, :]).astype(np.complex128)  # (C, nq)
        B12 = (E1[:, None, :] * E2[None, :, :]).reshape(L * L, -1)  # (L^2, nq)
        for c in range(Cn):
            Ah[c] += (B12 @ (E3 * S[c][None, :]).T).reshape(L, L, L)
    # the heat factor e^{-h^2 tau |m|^2}
    m = np.arange(-M, M, dtype=np.float64)
    g1 = np.exp(-(m * h) ** 2 * tau)
    Ah *= g1[None, :, None, None] * g1[None, None, :, None] * g1[None, None, None, :]
    # step 5: type-2 sum at the targets, real part, times (h / 2 pi)^3
    nt = xt.shape[0]
    out = np.empty((Cn, nt))
    for t0 in range(0, nt, chunk):
        sl = slice(t0, min(nt, t0 + chunk))
        E1, E2, E3 = _phases(xt[sl], h, M, +1)
        B12 = (E1[:, None, :] * E2[None, :, :]).reshape(L * L, -1)
        for c in range(Cn):
            Y = Ah[c].reshape(L * L, L) @ E3  # (L^2, nt)
            out[c, sl] = np.real((Y * B12).sum(0))
    return out * (h / (2 * math.pi)) ** 3


def gauss_convolve(F: np.ndarray, xs: np.ndarray, ws: np.ndarray, xt: np.ndarray,
                   tau: float, chunk: int = 256) -> np.ndarray:
    """sum_q ws[q] F[:, q] G_tau^3(xt - xs[q]) with the exact heat kernel."""
    F = np.asarray(F, dtype=np.float64)
    xs = np.asarray(xs, dtype=np.float64).reshape(-1, 3)
    xt = np.asarray(xt, dtype=np.float64).reshape(-1, 3)
    S = F * np.asarray(ws, dtype=np.float64)[None, :]
    out = np.empty((F.shape[0], xt.shape[0]))
    for t0 in range(0, xt.shape[0], chunk):
        sl = slice(t0, min(xt.shape[0], t0 + chunk))
        d2 = ((xt[sl, None, :] - xs[None, :, :]) ** 2).sum(-1)
        G = np.exp(-d2 / (4 * tau)) / (4 * math.pi * tau) ** 1.5
        out[:, sl] = S @ G.T
    return out


def surface_step(A: np.ndarray, xs: np.ndarray, ws: np.ndarray, xt: np.ndarray, n: int,
                 tau: float, h: float, M: int):
    """One iteration of Algorithm 1 on the surface: (A_next, A~, stats)."""
    At = surface_diffuse(A, xs, ws, xt, tau, h, M)
    B, sg = _core.project(At, n, return_sign=True)
    A0 = np.asarray(A, dtype=np.float64)
    d0 = np.array([np.linalg.det(A0[:, i].reshape(n, n)) for i in range(A0.shape[1])])
    flips = int(np.sum((d0 > 0) != (sg > 0)))
    return B, At, {"max_delta": float(np.abs(B - A0).max()), "det_flips": flips}


# --- volume-preserving step on the surface (Sec. 7 on a closed surface) ---------

def surface_step_volume(A: np.ndarray, xs: np.ndarray, ws: np.ndarray, xt: np.ndarray, n: int,
                        tau: float, h: float, M: int, volume: float = -1.0, weights=None):
    """One volume-preserving step on the surface (Sec. 7, Algorithm 3) with the
    diffusion of Algorithm 2: A~ = surface_diffuse(A); dE(x) = <T+(A~) - T-(A~), A~>
    per point (T+/T- the closest matrices of SO(n) / SO^-(n), Lemma 7.1).  Points
    are taken in decreasing dE (equal dE: lower index first), adding their
    weights (default: the quadrature weights ws) until the total reaches the
    volume V; those take T+, the rest T-.  volume < 0: V is the weight of the
    points with det A > 0.  Weights are added in exact rational arithmetic.
    Returns (A_next, A~, dE, stats)."""
    from fractions import Fraction
    A0 = np.asarray(A, dtype=np.float64)
    w = np.asarray(ws if weights is None else weights, dtype=np.float64)
    At = surface_diffuse(A0, xs, ws, xt, tau, h, M)
    npt = At.shape[1]
    mats = At.T.reshape(npt, n, n)
    dE = np.array([_core.delta_energy(m) for m in mats])
    d0 = np.array([np.linalg.det(A0[:, i].reshape(n, n)) for i in range(npt)])
    wf = [Fraction(float(x)) for x in w]
    V = sum((wf[i] for i in range(npt) if d0[i] > 0), Fraction(0)) if volume < 0 else Fraction(float(volume))
    order = np.lexsort((np.arange(npt), -dE))
    plus = np.zeros(npt, dtype=bool)
    V0 = Fraction(0)
    for i in order:
        if V0 >= V:
            break
        plus[i] = True
        V0 += wf[i]
    B = np.stack([_core.polar_class(m, 1 if p else -1).reshape(-1) for m, p in zip(mats, plus)], axis=1)
    stats = {"max_delta": float(np.abs(B - A0).max()), "det_flips": int(np.sum((d0 > 0) != plus)),
             "selected": int(plus.sum()), "volume": float(V), "selected_volume": float(V0)}
    return B, At, dE, stats

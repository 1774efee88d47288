"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This module draws random numbers and arranges them into raw (not yet
projected) matrix fields.  It holds none of the MBO arithmetic: no heat
multiplier, no transform, no projection.  Each consumer projects the raw field
onto O_n with its own projection (the oracle's Jacobi SVD on the CPU, the
library's kernel on the GPU), since Algorithm 1 takes an O_n-valued A_0.

Layout: float64 array of shape ``(n*n, *dims)``; channel ``i*n+j`` is matrix
entry ``(i, j)``; ``dims`` is row-major with the last axis (x) fastest.
The torus is [0,1)^d with grid point index i_j at coordinate i_j / N_j.

Workload recipes (the paper has no dataset; these stand in for its flat-torus
experiments, Sec. 6.1, at the sizes the benchmark configurations name):
  * ``gaussian``      iid N(0,1) entries per point.
  * ``sign_split``    iid N(0,1) entries, conditioned so that det > 0 where
                      x < 1/2 and det < 0 where x >= 1/2 (rows 0 and 1 of a
                      matrix with the wrong sign are swapped; the swap is
                      measure preserving, so entries stay N(0,1)).
  * ``voronoi``       piecewise-constant Haar SO(3) rotations on seeded
                      periodic Voronoi cells plus N(0, sd) entrywise noise.
  * ``smooth_so3``    exp of a Gaussian random so(3) field with spectrum
                      ~ exp(-|k|^2 / kc^2), some points replaced by -Q with
                      Q Haar in SO(3) (determinant -1).
  * ``batch_mixed``   many independent 2-D fields of uneven sizes and orders.
  * ``paper_experiment`` the analytic initial fields of the paper's flat-torus
                      experiments (Sec. 6.1 examples 1-3, Sec. 7).
  * ``sphere_paper_field`` the two printed 3x3 matrices of the sphere
                      experiment (Sec. 6.2) placed on given surface points
                      (raw: the matrices are not orthogonal as printed).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 171101365


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian(dims, n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """iid N(0,1) matrix entries at every grid point."""
    g = rng(seed)
    return g.standard_normal((n * n,) + tuple(int(d) for d in dims)).astype(dtype, copy=False)


def _det_sign_sample(F: np.ndarray, n: int) -> np.ndarray:
    """sign(det) of every point's raw matrix (input preparation only)."""
    M = np.moveaxis(F.reshape((n, n) + F.shape[1:]), (0, 1), (-2, -1))
    return np.sign(np.linalg.det(M))


def sign_split(dims, n: int, seed: int) -> np.ndarray:
    """iid N(0,1) entries; det > 0 on x < 1/2 and det < 0 on x >= 1/2."""
    if n < 2:
        raise ValueError("sign_split needs n >= 2")
    F = gaussian(dims, n, seed)
    nx = F.shape[-1]
    want = np.where(np.arange(nx) < nx // 2, 1.0, -1.0)
    have = _det_sign_sample(F, n)
    wrong = have != want  # broadcast over the last axis
    for j in range(n):  # swap rows 0 and 1 where the sign is wrong
        c0, c1 = 0 * n + j, 1 * n + j
        a = F[c0][wrong].copy()
        F[c0][wrong] = F[c1][wrong]
        F[c1][wrong] = a
    return F


def haar_so3(count: int, g: np.random.Generator) -> np.ndarray:
    """Haar-random rotations from uniform unit quaternions (Shoemake 1992)."""
    u1, u2, u3 = g.random(count), g.random(count), g.random(count)
    a = np.sqrt(1 - u1)
    b = np.sqrt(u1)
    w = a * np.sin(2 * np.pi * u2)
    x = a * np.cos(2 * np.pi * u2)
    y = b * np.sin(2 * np.pi * u3)
    z = b * np.cos(2 * np.pi * u3)
    R = np.empty((count, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def voronoi(dims, seed: int, cells: int = 64, sd: float = 0.05, dtype=np.float64) -> np.ndarray:
    """Piecewise-constant Haar SO(3) on periodic Voronoi cells + N(0, sd) noise (n = 3)."""
    g = rng(seed)
    d = len(dims)
    centres = g.random((cells, d))
    rots = haar_so3(cells, g)
    shape = tuple(int(s) for s in dims)
    P = int(np.prod(shape))
    out = np.empty((9, P), dtype=dtype)
    coords = [np.arange(s) / s for s in shape]
    # nearest centre (minimum image on the unit torus), one slab of the first axis at a time
    plane = P // shape[0]
    grid_rest = np.stack(np.meshgrid(*coords[1:], indexing="ij"), -1).reshape(-1, d - 1)
    rest_d2 = np.zeros((plane, cells))
    for a in range(d - 1):
        diff = np.abs(grid_rest[:, a:a + 1] - centres[None, :, a + 1])
        diff = np.minimum(diff, 1.0 - diff)
        rest_d2 += diff * diff
    flat = rots.reshape(cells, 9)
    for i0 in range(shape[0]):
        dz = np.abs(coords[0][i0] - centres[:, 0])
        dz = np.minimum(dz, 1.0 - dz)
        lab = np.argmin(rest_d2 + (dz * dz)[None, :], axis=1)
        out[:, i0 * plane:(i0 + 1) * plane] = flat[lab].T
    out += sd * g.standard_normal(out.shape)
    return out.reshape((9,) + shape)


def smooth_so3(dims, seed: int, kc: float = 32.0, frac_reflect: float = 0.2,
               dtype=np.float32) -> np.ndarray:
    """exp([w]_x) of a smooth Gaussian so(3) field; a Bernoulli(frac) mask of
    points is replaced by -Q, Q Haar in SO(3) (n = 3, any d).

    Each component of w is white noise filtered by sqrt(exp(-|k|^2 / kc^2)) (k
    in integer cycles over the unit torus) and normalised to unit pointwise
    standard deviation.  Computed in float32 with scipy.fft (all cores)."""
    import scipy.fft as sfft
    g = rng(seed)
    shape = tuple(int(s) for s in dims)
    P = int(np.prod(shape))
    freqs = [np.fft.fftfreq(s, 1.0 / s) for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1], 1.0 / shape[-1])]
    amp = np.ones([len(f) for f in freqs], dtype=np.float32)
    for ax, f in enumerate(freqs):
        sh = [1] * len(shape)
        sh[ax] = len(f)
        amp = amp * np.exp(-(f.astype(np.float64) ** 2) / (2 * kc ** 2)).astype(np.float32).reshape(sh)
    w = np.empty((3, P), dtype=np.float32)
    for i in range(3):
        white = g.standard_normal(shape, dtype=np.float32)
        f = sfft.irfftn(sfft.rfftn(white, workers=-1) * amp, s=shape, workers=-1)
        f /= f.std()
        w[i] = f.reshape(-1)
        del white, f
    theta = np.sqrt((w * w).sum(0))
    safe = np.where(theta > 0, theta, 1.0).astype(np.float32)
    w /= safe
    kx, ky, kz = w
    s = np.sin(theta)
    c1 = (1.0 - np.cos(theta)).astype(np.float32)
    del theta, safe
    R = np.empty((9, P), dtype=dtype)
    # Rodrigues: I + sin(t) K + (1 - cos(t)) K^2 for the unit axis (kx, ky, kz)
    R[0] = 1 - c1 * (ky * ky + kz * kz)
    R[1] = -s * kz + c1 * kx * ky
    R[2] = s * ky + c1 * kx * kz
    R[3] = s * kz + c1 * kx * ky
    R[4] = 1 - c1 * (kx * kx + kz * kz)
    R[5] = -s * kx + c1 * ky * kz
    R[6] = -s * ky + c1 * kx * kz
    R[7] = s * kx + c1 * ky * kz
    R[8] = 1 - c1 * (kx * kx + ky * ky)
    del w, s, c1
    mask = g.random(P) < frac_reflect
    cnt = int(mask.sum())
    if cnt:
        R[:, mask] = (-haar_so3(cnt, g).reshape(cnt, 9).T).astype(dtype)
    return R.reshape((9,) + shape)


def paper_experiment(k: int, N: int = 1024):
    """Initial fields of the flat-torus experiments of Sec. 6.1 (k = 1, 2, 3) and
    of the volume-preserving flat-torus experiment of Sec. 7 (k = 4, the field
    of k = 1).  Domain [-1/2, 1/2)^2 sampled at x = i/N - 1/2 (x fastest),
    n = 2.  Inside the region named in the paper the matrix is the rotation by
    alpha, elsewhere the reflection [[cos a, sin a], [sin a, -cos a]].
    Returns (field (4, N, N), n, tau).  The paper gives tau = 8 dx or 64 dx
    with dx = 1/1024; those values are read as the time of a heat kernel with
    Fourier multiplier exp(-tau |xi|^2) for integer frequencies xi (a
    2 pi-periodic length scale), i.e. tau / (4 pi^2) for the unit torus used
    here.  Taken literally on the unit torus, tau = 64 dx spreads the kernel
    over a third of the domain and examples 2 and 3 collapse to one phase
    within a few steps, unlike the evolution the paper describes."""
    c = np.arange(N) / N - 0.5
    Y, X = np.meshgrid(c, c, indexing="ij")
    if k in (1, 4):
        alpha = 0.5 * np.pi * np.sin(2 * np.pi * (X + Y))
        r = np.sqrt(X * X + Y * Y)
        th = np.arctan2(Y, X)
        inside = r < 0.3 + 0.06 * np.sin(6 * th)
        tau = 8.0 / 1024 / (4 * np.pi ** 2)
    elif k in (2, 3):
        alpha = np.pi * np.sin(2 * np.pi * Y) if k == 2 else 2 * np.pi * Y
        w = 0.25 * np.abs(np.sin(2.5 * np.pi * Y))
        inside = (X > w + 0.2) | (X < -w - 0.2)
        tau = 64.0 / 1024 / (4 * np.pi ** 2)
    else:
        raise ValueError(k)
    ca, sa = np.cos(alpha), np.sin(alpha)
    F = np.empty((4, N, N))
    F[0] = ca
    F[1] = np.where(inside, -sa, sa)
    F[2] = sa
    F[3] = np.where(inside, ca, -ca)
    return F, 2, tau


# Batched 2-D workload: field i gets N = SIZES[i % 7], n = 2 + (i % 2), tau = 4 / N^2.
BATCH_SIZES = (256, 384, 512, 768, 1024, 1536, 2048)


# The two matrices printed for the sphere experiment (Sec. 6.2), row-major.
SPHERE_MATRICES = (
    (0.392227, 0.706046, 0.046171, 0.655478, 0.031833, 0.097132, 0.171187, 0.276923, 0.82346),
    (0.699077, 0.547216, 0.257508, 0.890903, 0.138624, 0.840717, 0.959291, 0.149294, 0.254282),
)


def sphere_paper_field(xc: np.ndarray) -> np.ndarray:
    """Raw initial field of the sphere experiment (Sec. 6.2) at points xc
    (nq x 3): the first printed matrix where x < 0, y < 0 and z > 0, the
    second elsewhere.  Shape (9, nq)."""
    xc = np.asarray(xc, dtype=np.float64)
    sel = (xc[:, 0] < 0) & (xc[:, 1] < 0) & (xc[:, 2] > 0)
    m1 = np.array(SPHERE_MATRICES[0]).reshape(9, 1)
    m2 = np.array(SPHERE_MATRICES[1]).reshape(9, 1)
    return np.where(sel[None, :], m1, m2)


def batch_mixed(count: int, seed: int, sizes=BATCH_SIZES):
    """List of (dims, n, tau, raw field) for independent uneven 2-D fields."""
    out = []
    for i in range(count):
        N = sizes[i % len(sizes)]
        n = 2 + (i % 2)
        out.append(((N, N), n, 4.0 / N ** 2, None if seed is None else (seed + 1000 + i)))
    return out


# Named workloads.  tau is in units of h^2 with h = 1 / N (Sec. 5.1 grid on [0,1)^d).
CONFIGS = {
    "C1": dict(dims=(128, 128), n=2, tau=4.0 / 128 ** 2, steps=100, init="gaussian"),
    "C2": dict(dims=(1024, 1024), n=3, tau=3.0 / 1024 ** 2, steps=200, init="sign_split"),
    "C3": dict(dims=(256, 256, 256), n=3, tau=2.0 / 256 ** 2, steps=300, init="voronoi"),
    "C4": dict(count=96, steps=100, init="batch_mixed"),
    "C5": dict(dims=(512, 512, 512), n=3, tau=2.0 / 512 ** 2, steps=100, init="smooth_so3"),
}


def config_field(name: str, seed: int | None = None, dims=None,
                 dtype=np.float64) -> tuple[np.ndarray, int, float]:
    """Raw initial field for a named workload, optionally at smaller dims
    (tau is rescaled to keep the same multiple of h^2).  dtype applies to the
    3-D recipes (float32 halves the host memory of the 512^3 field)."""
    cfg = CONFIGS[name]
    seed = SEED_BASE + int(name[1:]) if seed is None else seed
    d = tuple(dims) if dims is not None else cfg["dims"]
    tau = cfg["tau"] * (cfg["dims"][-1] / d[-1]) ** 2
    n = cfg["n"]
    init = cfg["init"]
    if init == "gaussian":
        F = gaussian(d, n, seed)
    elif init == "sign_split":
        F = sign_split(d, n, seed)
    elif init == "voronoi":
        F = voronoi(d, seed, dtype=dtype)
    elif init == "smooth_so3":
        F = smooth_so3(d, seed, kc=32.0 * d[-1] / cfg["dims"][-1], dtype=dtype)
    else:
        raise ValueError(init)
    return F, n, tau

"""FP32 axes of length 256, 512 and 1024, and 768, 1536 and 2048 (a radix-3 or
radix-2 stage across groups of lanes on top), which the library transforms with
the warp-cooperative four-step plan (spectrum in natural order), against the
oracle: the diffusion (Sec. 5.1), one step of Algorithm 1 and a second step
from the kept spectrum, and the Lyapunov functional of Sec. 4.

Shapes put each warp-plan axis beside generic axes: x alone (with an odd row
count, so the last block of the 2-row kernels holds a row past the end), y
alone, y and x together, and the z axis of 3-D fields.  Tolerances are those
of test_gpu_parity.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1711_01365_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_DIFF_TOL = 4e-6
F32_STEP_TOL = 2e-5
F32_ENERGY_RTOL = 1e-5

WARP_SHAPES = [
    (6, 1024),       # x: 32 lanes x 32 points
    (3, 512),        # x: 16 x 32, odd row count
    (9, 256),        # x: 16 x 16, odd row count
    (1024, 8),       # y: 32 x 32, 8-column tiles
    (512, 16),       # y
    (256, 24),       # y
    (256, 256),      # y and x
    (3, 512, 8),     # 3-D: y
    (256, 2, 8),     # 3-D: z
    (2, 4, 512),     # 3-D: x
    (256, 4, 256),   # 3-D: z and x
    (4, 2048),       # x: 2 groups of 32 lanes (radix-2 stage)
    (3, 1536),       # x: 3 groups of 16 lanes (radix-3 stage), odd row count
    (6, 768),        # x: 3 x 256
    (2048, 4),       # y: 2 x 1024, 4-column tiles
    (1536, 8),       # y: 3 x 512
    (768, 16),       # y: 3 x 256
    (768, 768),      # y and x
    (768, 2, 8),     # 3-D: z
    (2, 4, 1536),    # 3-D: x
]


@pytest.fixture(scope="module")
def M():
    from paper_1711_01365_gb300 import build
    build.build()
    from paper_1711_01365_gb300 import mbo
    return mbo


def _mats(F, n):
    return np.moveaxis(F.reshape(n * n, -1), 0, -1).reshape(-1, n, n)


def _case(dims, n, seed):
    A = O.project(I.gaussian(dims, n, seed), n)
    tau = 3.0 / max(dims) ** 2
    return A, tau


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("dims", WARP_SHAPES)
def test_warp_axes_diffuse_step_energy(M, dims, n):
    A, tau = _case(dims, n, 7000 + n + sum(dims))
    h = M.Mbo(dims, n, tau, "f32")
    a = torch.tensor(A, dtype=torch.float32, device="cuda")

    # diffusion
    out = torch.empty_like(a)
    h.diffuse(a, out)
    torch.cuda.synchronize()
    At = O.diffuse(A, tau)
    assert np.abs(out.double().cpu().numpy() - At).max() <= F32_DIFF_TOL

    # energy
    E = h.lyapunov(a)
    assert E == pytest.approx(O.energy(A, n, tau), rel=F32_ENERGY_RTOL)

    # two steps (the second from the spectrum the first one kept)
    ref1, st1 = O.step(A, n, tau)
    rec1 = h.step(a, want_stats=True)
    B1 = a.double().cpu().numpy()
    s = np.linalg.svd(_mats(At, n), compute_uv=False)
    absdet = np.prod(s, axis=1).reshape(dims)
    cs = (s[:, -1] + (s[:, -2] if n > 1 else s[:, -1])).reshape(dims)
    err = np.abs(B1 - ref1).max(axis=0)
    # |det| above its single-precision rounding level; sigma_{n-1} + sigma_n >= 1e-2
    unamb = absdet > 64 * 2.0 ** -24 * np.sqrt((s ** 2).sum(axis=1)).reshape(dims) ** n
    well = unamb & (cs >= 1e-2)
    assert err[well].max() <= F32_STEP_TOL
    bound = F32_STEP_TOL + 2 * F32_DIFF_TOL * n / np.maximum(cs, 1e-30)
    assert np.all(err[unamb] <= bound[unamb])
    assert rec1["energy"] == pytest.approx(st1["energy"], rel=F32_ENERGY_RTOL)
    assert rec1["nonfinite"] == 0
    Bm = _mats(B1, n)
    assert np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(n)).max() < 2e-6

    # the second step starts from the library's own first step (FP32 values)
    ref2, st2 = O.step(B1, n, tau)
    rec2 = h.step(a, flags=M.MBO_STEP_CONTINUE, want_stats=True)
    B2 = a.double().cpu().numpy()
    At2 = O.diffuse(B1, tau)
    s2 = np.linalg.svd(_mats(At2, n), compute_uv=False)
    absdet2 = np.prod(s2, axis=1).reshape(dims)
    cs2 = (s2[:, -1] + (s2[:, -2] if n > 1 else s2[:, -1])).reshape(dims)
    err2 = np.abs(B2 - ref2).max(axis=0)
    unamb2 = absdet2 > 64 * 2.0 ** -24 * np.sqrt((s2 ** 2).sum(axis=1)).reshape(dims) ** n
    bound2 = F32_STEP_TOL + 2 * F32_DIFF_TOL * n / np.maximum(cs2, 1e-30)
    assert np.all(err2[unamb2] <= bound2[unamb2])
    assert rec2["energy"] == pytest.approx(st2["energy"], rel=F32_ENERGY_RTOL)
    h.close()

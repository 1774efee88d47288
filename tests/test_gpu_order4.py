"""Order n = 4 (O_4-valued fields) on the GPU against the oracle: the
diffusion of Sec. 5.1, the projection of Lemma 1.1 (scaled Newton with 4 x 4
cofactors; FP64 one-sided Jacobi for matrices singular to working precision),
one step of Algorithm 1 with its energy, and the Lyapunov functional of Sec. 4.
Shapes cover the in-place network and the warp-cooperative plans (x, y and
3-D).  Tolerances are those of test_gpu_parity."""
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
N = 4

SHAPES = [(8, 8), (24, 32), (6, 1024), (1024, 8), (256, 256), (4, 6, 8), (2, 4, 512)]


@pytest.fixture(scope="module")
def M():
    from paper_1711_01365_gb300 import build
    build.build()
    from paper_1711_01365_gb300 import mbo
    return mbo


def _mats(F):
    return F.reshape(N, N, -1).transpose(2, 0, 1)


def _dev(a, dtype):
    t = torch.tensor(np.ascontiguousarray(a), dtype=torch.float64).to(dtype)
    return t.cuda().contiguous()


def _host(t):
    return t.detach().double().cpu().numpy()


def _tdt(name):
    return torch.float32 if name == "f32" else torch.float64


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("dims", SHAPES)
def test_order4_diffuse_step_energy(M, dims, dtype):
    A = O.project(I.gaussian(dims, N, 8100 + sum(dims)), N)
    tau = 1.0 / max(dims) ** 2
    h = M.Mbo(dims, N, tau, dtype)
    a = _dev(A, _tdt(dtype))
    out = torch.empty_like(a)
    h.diffuse(a, out)
    torch.cuda.synchronize()
    At = O.diffuse(A, tau)
    assert np.abs(_host(out) - At).max() <= (F64_TOL if dtype == "f64" else F32_DIFF_TOL)

    E = h.lyapunov(a)
    assert E == pytest.approx(O.energy(A, N, tau), rel=1e-12 if dtype == "f64" else F32_ENERGY_RTOL)

    ref, st = O.step(A, N, tau)
    rec = h.step(a, want_stats=True)
    B = _host(a)
    s = np.linalg.svd(_mats(At), compute_uv=False)
    absdet = np.prod(s, axis=1).reshape(dims)
    cs = (s[:, -1] + s[:, -2]).reshape(dims)
    err = np.abs(B - ref).max(axis=0)
    if dtype == "f64":
        unamb = absdet > 1e-12
        assert unamb.any()
        assert err[unamb].max() <= F64_TOL
        assert rec["energy"] == pytest.approx(st["energy"], rel=1e-12)
        assert rec["max_delta"] == pytest.approx(st["max_delta"], abs=1e-12)
    else:
        # |det| above its single-precision rounding level (64 eps |A~|_F^4);
        # strict bound where sigma_3 + sigma_4 >= 1e-2
        unamb = absdet > 64 * 2.0 ** -24 * np.sqrt((s ** 2).sum(axis=1)).reshape(dims) ** N
        well = unamb & (cs >= 1e-2)
        assert well.any()
        assert err[well].max() <= F32_STEP_TOL
        bound = F32_STEP_TOL + 2 * F32_DIFF_TOL * N / np.maximum(cs, 1e-30)
        assert np.all(err[unamb] <= bound[unamb])
        assert rec["energy"] == pytest.approx(st["energy"], rel=F32_ENERGY_RTOL)
    assert rec["nonfinite"] == 0
    Bm = _mats(B)
    orth = np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(N)).max()
    assert orth < (1e-13 if dtype == "f64" else 2e-6)
    h.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_order4_project_against_oracle(M, dtype):
    """Realistic diffused matrices, raw Gaussian matrices of three scales, and
    rotated matrices of rank 3 and 2 (the singular branches)."""
    g = I.rng(8200)
    At = O.diffuse(O.project(I.gaussian((32, 48), N, 8201), N), 3.0 / 48 ** 2)
    raw = g.standard_normal((N * N, 30, 48)) * g.choice([1e-3, 1.0, 5.0], size=(30, 48))
    sing = []
    for r in (3, 2):
        for _ in range(48):
            Ux = np.linalg.qr(g.standard_normal((N, N)))[0]
            Vx = np.linalg.qr(g.standard_normal((N, N)))[0]
            sv = np.zeros(N)
            sv[:r] = np.sort(g.uniform(0.2, 2.0, r))[::-1]
            sing.append((Ux @ np.diag(sv) @ Vx.T).reshape(-1))
    S = np.stack(sing, axis=1).reshape(N * N, 2, 48)
    F = np.concatenate([At, raw, S], axis=1)  # 64 x 48 points
    dims = F.shape[1:]
    ref, sref = O.project(F, N, return_sign=True)
    h = M.Mbo(dims, N, 1e-3, dtype)
    a = _dev(F, _tdt(dtype))
    out = torch.empty_like(a)
    sg = torch.empty(dims, dtype=torch.int8, device="cuda")
    h.project(a, out, sg)
    torch.cuda.synchronize()
    B = _host(out)
    Bm = _mats(B)
    assert np.abs(np.einsum("pki,pkj->pij", Bm, Bm) - np.eye(N)).max() < (1e-13 if dtype == "f64" else 2e-6)
    assert np.array_equal(np.sign(np.linalg.det(Bm)).reshape(dims), sg.cpu().numpy().astype(float))
    Fm = _mats(F)
    d = np.abs(np.linalg.det(Fm)).reshape(dims)
    s = np.linalg.svd(Fm, compute_uv=False)
    cs = (s[:, -1] + s[:, -2]).reshape(dims)
    err = np.abs(B - ref).max(axis=0)
    cut32 = 64 * 2.0 ** -24 * np.sqrt((s ** 2).sum(axis=1)).reshape(dims) ** N
    unamb = d > (1e-12 if dtype == "f64" else cut32)
    assert np.array_equal(sg.cpu().numpy()[unamb], sref[unamb])
    # rank-deficient rows: det A~ is rounding noise, so either class is a
    # minimiser; B must be one: |B - A~|^2 = sum (s_i - 1)^2 (with s_n = 0 both
    # classes are equally close, Lemma 7.1)
    Bs = _mats(B[:, dims[0] - 2:])
    Ss = _mats(F[:, dims[0] - 2:])
    ss = np.linalg.svd(Ss, compute_uv=False)
    d2 = ((Bs - Ss) ** 2).sum((1, 2))
    assert np.abs(d2 - ((ss - 1) ** 2).sum(1)).max() < (1e-9 if dtype == "f64" else 2e-5)
    if dtype == "f64":
        assert err[unamb].max() <= F64_TOL
    else:
        well = unamb & (cs >= 1e-2)
        assert err[well].max() <= F32_STEP_TOL
        eps_in = np.abs(F - F.astype(np.float32).astype(np.float64)).max(axis=0)
        bound = F32_STEP_TOL + 2 * (eps_in * N + 1e-7) / np.maximum(cs, 1e-30)
        assert np.all(err[unamb] <= bound[unamb])
    h.close()


def test_order4_block_field_evolves_as_two_order2_fields(M):
    """blockdiag(R, S) with R, S independent O_2 fields: FP64 GPU steps of the
    n = 4 field equal FP64 GPU steps of the two n = 2 fields."""
    dims = (64, 64)
    tau = 4.0 / 64 ** 2
    R = O.project(I.gaussian(dims, 2, 8301), 2)
    S = O.project(I.gaussian(dims, 2, 8302), 2)
    blk = [(0, 0, 0), (0, 1, 1), (1, 0, 2), (1, 1, 3)]
    F = np.zeros((16,) + dims)
    for i, j, c in blk:
        F[i * 4 + j] = R[c]
        F[(i + 2) * 4 + (j + 2)] = S[c]
    h4 = M.Mbo(dims, 4, tau, "f64")
    h2 = M.Mbo(dims, 2, tau, "f64")
    f, r, s = _dev(F, torch.float64), _dev(R, torch.float64), _dev(S, torch.float64)
    for k in range(5):
        h4.step(f, flags=M.MBO_STEP_CONTINUE if k else 0)
        h2.step(r)
        h2.step(s)
    torch.cuda.synchronize()
    Fh, Rh, Sh = _host(f), _host(r), _host(s)
    for i, j, c in blk:
        assert np.abs(Fh[i * 4 + j] - Rh[c]).max() < 1e-12
        assert np.abs(Fh[(i + 2) * 4 + (j + 2)] - Sh[c]).max() < 1e-12
    off = [i * 4 + j for i in range(4) for j in range(4) if (i < 2) != (j < 2)]
    assert np.abs(Fh[off]).max() < 1e-12
    h4.close()
    h2.close()


def test_order4_volume_step_unsupported(M):
    h = M.Mbo((8, 8), 4, 1e-2, "f32")
    a = torch.zeros((16, 8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(M.MboError) as ei:
        h.step_volume(a, 10)
    assert ei.value.status == 2  # MBO_ERR_UNSUPPORTED_SIZE
    h.close()

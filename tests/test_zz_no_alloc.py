"""The allocation-free diffusion entry point, mbo_diffuse_noalloc.

Some callers must not allocate device memory: a framework's caching allocator
may already hold the memory they are allowed to use, a tight loop may not
afford the synchronisation that cudaMalloc/cudaFree can imply, or the memory
budget is fixed in advance.  For them the library offers a diffusion call
whose scratch lives in a static 64 MiB device array inside the library.  These
tests call it through the C ABI and check, on two calls in a row, that it
returns what the handle-based mbo_diffuse returns for the same input, and what
the FP64 CPU oracle's diffusion (Sec. 5.1) returns, within the parity
tolerances (max-entry 1e-12 in FP64, 4e-6 in FP32).  They also check in-place
calls (A_tilde == A) and the refusals that happen before any launch.  The file
is named so that pytest collects it last.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1711_01365_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 4e-6}


@pytest.fixture(scope="module")
def M():
    from paper_1711_01365_gb300 import build
    build.build()
    O.build()
    from paper_1711_01365_gb300 import mbo
    return mbo


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("dims,n", [((96, 128), 3), ((8, 12, 16), 2), ((64, 64), 1), ((48, 64), 4)])
def test_noalloc_matches_mbo_diffuse_on_two_calls_in_a_row(M, dims, n, dtype):
    tau = 3.0 / max(dims) ** 2
    tdt = torch.float32 if dtype == "f32" else torch.float64
    code = M.MBO_F32 if dtype == "f32" else M.MBO_F64
    h = M.Mbo(dims, n, tau, dtype)
    for call, seed in enumerate((11, 12)):
        F = I.gaussian(dims, n, seed)
        A = torch.tensor(F, dtype=tdt, device="cuda")
        ref = torch.empty_like(A)
        h.diffuse(A, ref)
        out = torch.full_like(A, float("nan"))
        M.mbo_diffuse_noalloc(dims, n, tau, code, A, out)
        torch.cuda.synchronize()
        err = (out.double() - ref.double()).abs().max().item()
        assert err <= TOL[dtype], (call, err)
        # the oracle's diffusion of the same (rounded) input; the raw Gaussian
        # entries reach ~5, so the FP32 bound scales with max |A|
        a64 = A.double().cpu().numpy()
        want = O.diffuse(a64, tau)
        err_o = np.abs(out.double().cpu().numpy() - want).max()
        assert err_o <= TOL[dtype] * max(1.0, np.abs(a64).max()), (call, err_o)
    h.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("dims,n", [((96, 128), 3), ((8, 12, 16), 2)])
def test_noalloc_in_place(M, dims, n, dtype):
    """A_tilde == A: the first pass reads all of A into the workspace before
    the last pass writes A_tilde, so an in-place call equals an out-of-place
    one."""
    tau = 3.0 / max(dims) ** 2
    tdt = torch.float32 if dtype == "f32" else torch.float64
    code = M.MBO_F32 if dtype == "f32" else M.MBO_F64
    h = M.Mbo(dims, n, tau, dtype)
    for seed in (21, 22):
        X = torch.tensor(I.gaussian(dims, n, seed), dtype=tdt, device="cuda")
        ref = torch.empty_like(X)
        h.diffuse(X.clone(), ref)
        M.mbo_diffuse_noalloc(dims, n, tau, code, X, X)
        torch.cuda.synchronize()
        err = (X.double() - ref.double()).abs().max().item()
        assert err <= TOL[dtype], err
    h.close()


def test_noalloc_rejects_problems_beyond_its_scratch(M):
    # 1024 x 1024, n = 3, FP64 needs 5 * 2^20 * 16 B = 80 MiB of workspace > 64 MiB;
    # raw pointers bypass the binding's own size checks so the C ABI refuses
    A = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MboError) as ei:
        M.mbo_diffuse_noalloc((1024, 1024), 3, 1e-6, M.MBO_F64, A.data_ptr(), A.data_ptr())
    assert ei.value.status == 2
    # the largest FP32 workload that fits: 1024 x 1024, n = 3 (40 MiB of workspace)
    dims, n, tau = (1024, 1024), 3, 3.0 / 1024 ** 2
    F = torch.tensor(I.gaussian(dims, n, 5), dtype=torch.float32, device="cuda")
    out = torch.empty_like(F)
    M.mbo_diffuse_noalloc(dims, n, tau, M.MBO_F32, F, out)
    h = M.Mbo(dims, n, tau, "f32")
    ref = torch.empty_like(F)
    h.diffuse(F, ref)
    torch.cuda.synchronize()
    assert (out - ref).abs().max().item() <= TOL["f32"]
    h.close()


def test_noalloc_rejects_rows_beyond_shared_memory_then_still_works(M):
    """2 x 2048 with n = 4 in FP64 needs only 512 KiB of workspace, but one row
    of its 8 complex planes (about 295 KB) does not fit in a block's shared
    memory: the call is refused with MBO_ERR_UNSUPPORTED_SIZE before any launch,
    and a valid call right after it succeeds."""
    dims, n = (2, 2048), 4
    A = torch.zeros((n * n,) + dims, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MboError) as ei:
        M.mbo_diffuse_noalloc(dims, n, 1e-6, M.MBO_F64, A, A)
    assert ei.value.status == 2
    dims, n, tau = (64, 96), 2, 3.0 / 96 ** 2
    X = torch.tensor(I.gaussian(dims, n, 8), dtype=torch.float64, device="cuda")
    out = torch.empty_like(X)
    M.mbo_diffuse_noalloc(dims, n, tau, M.MBO_F64, X, out)
    torch.cuda.synchronize()
    want = O.diffuse(X.cpu().numpy(), tau)
    assert np.abs(out.cpu().numpy() - want).max() <= TOL["f64"]


def test_noalloc_rejects_pointers_that_are_not_device_memory(M):
    """A host pointer is refused (MBO_ERR_INVALID_ARG) before any launch; the
    binding refuses tensors of the wrong size, dtype or layout outright."""
    dims, n = (32, 32), 2
    host = torch.zeros((n * n,) + dims, dtype=torch.float64).pin_memory()
    devt = torch.zeros((n * n,) + dims, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MboError) as ei:
        M.mbo_diffuse_noalloc(dims, n, 1e-3, M.MBO_F64, host.data_ptr(), devt.data_ptr())
    assert ei.value.status == 1
    with pytest.raises(ValueError):
        M.mbo_diffuse_noalloc(dims, n, 1e-3, M.MBO_F64, devt[:2], devt)
    with pytest.raises(ValueError):
        M.mbo_diffuse_noalloc(dims, n, 1e-3, M.MBO_F32, devt, devt)
    with pytest.raises(ValueError):
        M.mbo_diffuse_noalloc(dims, n, 1e-3, M.MBO_F64, devt.transpose(1, 2), devt)

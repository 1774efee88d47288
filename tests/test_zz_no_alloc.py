"""The allocation-free diffusion entry point, mbo_diffuse_noalloc.

Some callers must not allocate device memory: a framework's caching allocator
may already hold the memory they are allowed to use, a tight loop may not
afford the synchronisation that cudaMalloc/cudaFree can imply, or the memory
budget is fixed in advance.  For them the library offers a diffusion call
whose scratch lives in a static 64 MiB device array inside the library.  These
tests call it through the C ABI and check, on two calls in a row, that it
returns what the handle-based mbo_diffuse returns for the same input, within
the parity tolerances (max-entry 1e-12 in FP64, 4e-6 in FP32).  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1711_01365_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 4e-6}


@pytest.fixture(scope="module")
def M():
    from paper_1711_01365_gb300 import build
    build.build()
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
        A = torch.tensor(I.gaussian(dims, n, seed), dtype=tdt, device="cuda")
        ref = torch.empty_like(A)
        h.diffuse(A, ref)
        out = torch.full_like(A, float("nan"))
        M.mbo_diffuse_noalloc(dims, n, tau, code, A, out)
        torch.cuda.synchronize()
        err = (out.double() - ref.double()).abs().max().item()
        assert err <= TOL[dtype], (call, err)
    h.close()


def test_noalloc_rejects_problems_beyond_its_scratch(M):
    # 1024 x 1024, n = 3, FP64 needs 5 * 2^20 * 16 B = 80 MiB of workspace > 64 MiB
    A = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MboError) as ei:
        M.mbo_diffuse_noalloc((1024, 1024), 3, 1e-6, M.MBO_F64, A, A)
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

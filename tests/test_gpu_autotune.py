"""The launch-shape autotuner (mbo_config.autotune).

A tuned handle picks its strided-pass tile width, tile buffers, threads per
block of the network passes and of the network row pass by timing candidate
steps on a scratch field.  Launch shapes only decide which block computes
which column or row: the arithmetic of every point is the same, so the field
after a step must equal the default handle's bit for bit.  The energy may
differ by the order of its partial sums: each thread accumulates its points in
the field's precision (FP32 for the FP32 form) before the FP64 block sums.  A second handle of the same
(dims, n, dtype) takes the cached choice.
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


CASES = [((1024, 1024), 3, "f32"), ((384, 384), 2, "f32"), ((256, 512), 3, "f32"),
         ((96, 64), 2, "f64"), ((16, 24, 32), 3, "f32")]


@pytest.mark.parametrize("dims,n,dtype", CASES)
def test_tuned_step_equals_default_step(M, dims, n, dtype):
    tau = 3.0 / max(dims) ** 2
    tdt = torch.float32 if dtype == "f32" else torch.float64
    A0 = torch.tensor(O.project(I.gaussian(dims, n, 5), n), dtype=tdt, device="cuda")
    hd = M.Mbo(dims, n, tau, dtype)
    ht = M.Mbo(dims, n, tau, dtype, autotune=1)
    cd, ct = M.mbo_launch_config(hd.h), M.mbo_launch_config(ht.h)
    assert ct["autotune"] == 1 and cd["autotune"] == 0
    nx = dims[-1]
    assert ct["axis_tx"] >= 1 and nx % ct["axis_tx"] == 0
    assert ct["axis_stages"] in (1, 2, 3) and ct["pdl"] in (1, 2)
    assert 32 <= ct["row_threads"] <= 384 and ct["row_threads"] % 32 == 0
    assert 64 <= ct["axis_threads"] <= 384 and ct["axis_threads"] % 32 == 0
    Ad, At = A0.clone(), A0.clone()
    for k in range(3):
        fl = 0 if k == 0 else M.MBO_STEP_CONTINUE
        rd = hd.step(Ad, flags=fl, want_stats=True)
        rt = ht.step(At, flags=fl, want_stats=True)
        torch.cuda.synchronize()
        assert torch.equal(Ad, At), f"step {k}: tuned launch shapes changed the field"
        assert rd["det_flips"] == rt["det_flips"]
        assert rd["fallback_points"] == rt["fallback_points"]
        etol = 1e-5 if dtype == "f32" else 1e-12
        assert abs(rd["energy"] - rt["energy"]) <= etol * abs(rd["energy"])
    # the choice is cached for the process
    h2 = M.Mbo(dims, n, tau, dtype, autotune=1)
    assert M.mbo_launch_config(h2.h) == ct
    for h in (hd, ht, h2):
        h.close()


def test_tuned_run_matches_oracle(M):
    dims, n = (128, 96), 2
    tau = 4.0 / 128 ** 2
    A0 = O.project(I.gaussian(dims, n, 11), n)
    h = M.Mbo(dims, n, tau, "f64", autotune=1)
    A = torch.tensor(A0, dtype=torch.float64, device="cuda")
    res = h.run(A, 40, 1e-10)
    ref, info = O.run(A0, n, tau, 40, 1e-10)
    # the tuning steps left no trace in the run state: step count and energies
    assert res["steps"] == info["steps"] and res["stationary"] == info["stationary"]
    np.testing.assert_allclose(res["energies"], info["energies"], rtol=1e-10)
    np.testing.assert_allclose(A.cpu().numpy(), ref, atol=1e-10, rtol=0)
    h.close()


def test_explicit_shape_is_kept(M):
    dims, n = (512, 512), 3
    h = M.Mbo(dims, n, 3.0 / 512 ** 2, "f32", autotune=1, axis_tx=4, axis_stages=1)
    c = M.mbo_launch_config(h.h)
    assert c["axis_tx"] == 4 and c["axis_stages"] == 1
    h.close()


def test_batch_with_autotune_equals_default_batch(M):
    spec = [((256, 256), 2), ((384, 384), 3), ((512, 512), 3)]
    taus = [4.0 / d[0] ** 2 for d, _ in spec]
    A = [torch.tensor(O.project(I.gaussian(d, n, 20 + k), n), dtype=torch.float32, device="cuda")
         for k, (d, n) in enumerate(spec)]
    B = [a.clone() for a in A]
    bd = M.Batch([d for d, _ in spec], [n for _, n in spec], taus, "f32")
    bt = M.Batch([d for d, _ in spec], [n for _, n in spec], taus, "f32", autotune=1)
    for k in range(2):
        fl = 0 if k == 0 else M.MBO_STEP_CONTINUE
        bd.step(A, flags=fl)
        bt.step(B, flags=fl)
    torch.cuda.synchronize()
    for a, b in zip(A, B):
        assert torch.equal(a, b)
    bd.close()
    bt.close()


@pytest.mark.parametrize("dims,n", [((1024, 1024), 3), ((2048, 256), 2), ((32, 64, 256), 3)])
def test_dependent_launch_changes_nothing(M, dims, n):
    """Programmatic dependent launch only moves when a pass is scheduled: the
    fields, energies and statistics of a short run are those without it."""
    tau = 3.0 / max(dims) ** 2
    A0 = torch.tensor(O.project(I.gaussian(dims, n, 9), n), dtype=torch.float32, device="cuda")
    out = []
    for pdl in (1, 2):
        h = M.Mbo(dims, n, tau, "f32", pdl=pdl)
        assert M.mbo_launch_config(h.h)["pdl"] == pdl
        A = A0.clone()
        res = h.run(A, 12, -1.0)
        torch.cuda.synchronize()
        out.append((A, res))
        h.close()
    (A1, r1), (A2, r2) = out
    assert torch.equal(A1, A2)
    np.testing.assert_array_equal(r1["energies"], r2["energies"])
    np.testing.assert_array_equal(r1["det_flips"], r2["det_flips"])


def test_dependent_launch_option_checked(M):
    with pytest.raises(M.MboError):
        M.Mbo((64, 64), 2, 1e-3, "f32", pdl=3)


@pytest.mark.parametrize("dims", [(256, 64), (512, 64), (768, 64), (1024, 64), (1536, 64),
                                  (2048, 64), (512, 16, 64)])
def test_strided_pass_shapes_change_nothing(M, dims):
    """Every tile width (16 columns up to 512 rows) and staging form of the FP32 strided passes gives the
    field of the default launch bit for bit (two steps, n = 3)."""
    n = 3
    tau = 3.0 / max(dims) ** 2
    A0 = torch.tensor(O.project(I.gaussian(dims, n, 13), n), dtype=torch.float32, device="cuda")
    ref = None
    for tx in (8, 16, 4):
        for stages in (1, 2, 3):
            try:
                h = M.Mbo(dims, n, tau, "f32", axis_tx=tx, axis_stages=stages)
            except M.MboError as e:  # a shape whose buffers exceed shared memory is refused
                assert e.status == 2 and tx == 16 and stages > 1, (tx, stages, e)
                continue
            A = A0.clone()
            r1 = h.step(A, want_stats=True)
            r2 = h.step(A, flags=M.MBO_STEP_CONTINUE, want_stats=True)
            torch.cuda.synchronize()
            if ref is None:
                ref = (A, r1, r2)
            else:
                assert torch.equal(A, ref[0]), (tx, stages)
                assert r2["det_flips"] == ref[2]["det_flips"]
                assert abs(r2["energy"] - ref[2]["energy"]) <= 1e-5 * abs(ref[2]["energy"])
            h.close()

"""Batched and device-resident solves: same results as the single-cell path.

The device-resident loop (one CUDA graph launch with a while node) and the
host-launched loop run the same kernels in the same order, so their results are
identical; batched cells share launches but keep per-problem state, so each cell
matches its own single-cell solve.
"""
import numpy as np
import pytest
import torch

from paper_2312_15554_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def single_tensor(lib, H, prm):
    ctx = lib.acm_ctx(H.shape)
    dt = torch.float64 if prm.precision == lib.FP64 else torch.float32
    u3 = torch.zeros((3, 3) + H.shape, dtype=dt, device=DEV)
    s, K, _, reps = lib.acm_stokes_tensor(ctx, torch.as_tensor(H, device=DEV), prm, u3)
    torch.cuda.synchronize()
    ctx.close()
    return K, reps, u3.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_device_loop_equals_host_loop(lib, precision):
    H = I.sphere_pack((32, 16, 32), 0.45, 3.5, 21)[0]
    p = lib.FP64 if precision == "fp64" else lib.FP32
    Ka, ra, ua = single_tensor(lib, H, lib.stokes_params(precision=p, eps=1e-6, max_iter=3000, device_loop=1))
    Kb, rb, ub = single_tensor(lib, H, lib.stokes_params(precision=p, eps=1e-6, max_iter=3000, device_loop=0,
                                                         check_every=5))
    assert [r.iters for r in ra] == [r.iters for r in rb]
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(Ka, Kb)


def test_batched_cells_of_two_sizes_match_single_cell_solves(lib):
    shapes = [(16, 16, 16), (32, 32, 32), (16, 16, 16), (32, 32, 32), (16, 16, 16)]
    Hs = []
    for i, sh in enumerate(shapes):
        por, radii = I.cell_recipe(100 + i)
        Hs.append(I.sphere_pack(sh, por, (radii[0] * sh[0] / 64, radii[1] * sh[0] / 64), 100 + i)[0])
    prm = lib.stokes_params(precision=lib.FP32, eps=1e-5, max_iter=2000)
    batch = lib.acm_batch(shapes)
    u_out = [torch.zeros((3, 3) + sh, dtype=torch.float32, device=DEV) for sh in shapes]
    s, K, reps = lib.acm_batch_stokes(batch, [torch.as_tensor(h, device=DEV) for h in Hs], prm, u_out)
    torch.cuda.synchronize()
    batch.close()
    for i, H in enumerate(Hs):
        Ks, rs, us = single_tensor(lib, H, prm)
        assert [r.iters for r in reps[i]] == [r.iters for r in rs]
        np.testing.assert_allclose(K[i], Ks, rtol=1e-6, atol=1e-12 * np.abs(Ks).max())
        np.testing.assert_allclose(u_out[i].cpu().numpy(), us, rtol=0, atol=1e-6 * np.abs(us).max())


def test_batched_degenerate_cell_is_reported_not_iterated(lib):
    shapes = [(16, 16, 16), (16, 16, 16)]
    Hs = [I.sphere_pack((16, 16, 16), 0.5, 3.0, 5)[0], np.zeros((16, 16, 16), np.uint8)]
    batch = lib.acm_batch(shapes)
    s, K, reps = lib.acm_batch_stokes(batch, Hs, lib.stokes_params(eps=1e-5, max_iter=500))
    batch.close()
    assert np.isfinite(K[0]).all() and np.isnan(K[1]).all()
    assert all(r.status == -7 and r.iters == 0 for r in reps[1])
    assert all(r.status in (0, -4) for r in reps[0])

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


def test_batched_cells_of_the_c3_recipe_match_the_oracle(lib):
    """Two 64^3 and two 128^3 cells of the batched workload's recipe (porosity
    U[0.2, 0.6], sphere radii U[3, 10] voxels), all three loads of every cell in
    one device-resident graph, fixed penalties, 8 ADMM iterations from rest: u
    and H lambda of every load against the FP64 oracle, element by element."""
    from oracle import acm_oracle as Ora
    shapes = [(64, 64, 64), (128, 128, 128), (64, 64, 64), (128, 128, 128)]
    Hs = []
    for i, sh in enumerate(shapes):
        por, radii = I.cell_recipe(5000 + i)
        Hs.append(I.sphere_pack(sh, por, radii, 5000 + i)[0])
    n_it = 8
    prm = lib.stokes_params(precision=lib.FP32, eps=0.0, adaptive=0, max_iter=n_it, device_loop=1)
    batch = lib.acm_batch(shapes)
    u_out = [torch.zeros((3, 3) + sh, dtype=torch.float32, device=DEV) for sh in shapes]
    l_out = [torch.zeros((3, 3) + sh, dtype=torch.float32, device=DEV) for sh in shapes]
    s, K, reps = lib.acm_batch_stokes(batch, [torch.as_tensor(h, device=DEV) for h in Hs], prm, u_out,
                                      lambda_out=l_out)
    torch.cuda.synchronize()
    batch.close()
    for i, H in enumerate(Hs):
        assert all(r.iters == n_it for r in reps[i])
        for j in range(3):
            R = Ora.stokes(H, np.eye(3)[j], Ora.StokesParams(eps=0.0, adaptive=False, max_iter=n_it))
            u = u_out[i][j].cpu().numpy()
            lam = l_out[i][j].cpu().numpy()
            assert np.abs(u - R.state.u).max() < 1e-5 * np.abs(R.state.u).max(), (i, j)
            assert np.abs(lam - R.state.lam).max() < 1e-5 * np.abs(R.state.lam).max(), (i, j)
            np.testing.assert_allclose(K[i][:, j], R.K_col, rtol=0, atol=1e-5 * np.abs(R.K_col).max())


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_solute_device_loop_equals_host_loop(lib, precision):
    """The solute loop as one graph launch runs the same kernels in the same
    order as the host-launched chunks: identical fields, iteration counts, D."""
    H = I.sphere_pack((32, 16, 32), 0.45, 3.5, 22)[0]
    shape = H.shape
    p = lib.FP64 if precision == "fp64" else lib.FP32
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = torch.as_tensor(0.05 * I.random_field((3,) + shape, 23) * (1 - H)[None], dtype=dt, device=DEV)
    out = []
    for dl in (1, 0):
        ctx = lib.acm_ctx(shape)
        chi3 = torch.zeros((3,) + shape, dtype=dt, device=DEV)
        s, D, Dx, reps = lib.acm_advdiff_tensor(ctx, torch.as_tensor(H, device=DEV), u, 10.0, lib.advdiff_params(
            precision=p, eps=1e-7, max_iter=3000, device_loop=dl, check_every=7), chi3)
        torch.cuda.synchronize()
        ctx.close()
        assert all(r.converged for r in reps)
        out.append(([r.iters for r in reps], chi3.cpu().numpy(), D))
    assert out[0][0] == out[1][0]
    np.testing.assert_array_equal(out[0][1], out[1][1])
    np.testing.assert_array_equal(out[0][2], out[1][2])


def test_pore_scale_penalties_follow_each_cells_pore_length(lib):
    """pore_scale = f starts every penalty at f / l^2 times the default, l = pore
    voxels / solid-pore faces (counted here with numpy), per cell in a batch;
    the fields then equal the oracle's with those fixed penalties."""
    from oracle import acm_oracle as Ora

    def expected(H, f=9.0):
        faces = sum(int(np.count_nonzero(H != np.roll(H, -1, axis=a))) for a in range(3) if H.shape[a] > 1)
        l = np.count_nonzero(H == 0) / faces
        return f / l**2 * Ora.default_penalty(H.shape, 1.0)

    H = I.sphere_pack((32, 32, 32), 0.45, 4.0, 12)[0]
    ctx = lib.acm_ctx(H.shape)
    u = torch.zeros((3,) + H.shape, dtype=torch.float64, device=DEV)
    s, K, rep = lib.acm_stokes(ctx, torch.as_tensor(H, device=DEV), [1.0, 0.0, 0.0], lib.stokes_params(
        precision=lib.FP64, eps=0.0, max_iter=5, adaptive=0, pore_scale=9.0), None, None, u, None, None)
    ctx.close()
    psi = expected(H)
    np.testing.assert_allclose(rep.psi[:3], [psi] * 3, rtol=1e-12)
    R = Ora.stokes(H, [1.0, 0.0, 0.0], Ora.StokesParams(eps=0.0, max_iter=5, adaptive=False, alpha0=psi, beta0=psi,
                                                        b0=psi))
    np.testing.assert_allclose(u.cpu().numpy(), R.state.u, rtol=0, atol=1e-10 * np.abs(R.state.u).max())
    shapes = [(32, 32, 32), (1, 64, 64), (32, 32, 32)]
    Hs = [H, I.disk_pack(64, 64, 0.5, (3.0, 6.0), 5), I.sphere_pack((32, 32, 32), 0.3, 3.0, 13)[0]]
    batch = lib.acm_batch(shapes)
    s, Kb, reps = lib.acm_batch_stokes(batch, [torch.as_tensor(h, device=DEV) for h in Hs], lib.stokes_params(
        precision=lib.FP32, eps=0.0, max_iter=3, adaptive=0, pore_scale=9.0))
    batch.close()
    for i, h in enumerate(Hs):
        for r in reps[i]:
            np.testing.assert_allclose(r.psi[:3], [expected(h)] * 3, rtol=1e-12)

"""Warm starts of the Stokes ADMM: the batch entry point's init/lambda buffers,
the axis-swap rule of acm_fno_warm_start, and what a trained network gains.

The ADMM always runs to the same tolerance; a warm start may only change how
many iterations that takes, so every test also checks the permeability against
the zero start.
"""
import numpy as np
import pytest
import torch

from paper_2312_15554_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _cells(n, seeds):
    out = []
    for s in seeds:
        por, radii = I.cell_recipe(s)
        out.append(I.sphere_pack((n, n, n), por, (min(radii[0], n / 6), min(radii[1], n / 4)), s)[0])
    return np.stack(out)


def test_warm_start_swaps_axes_and_components(lib):
    n, W, modes, L = 16, 8, 3, 2
    fno = lib.acm_fno((n, n, n), W, modes, L, max_batch=4)
    rng = np.random.Generator(np.random.PCG64(5))
    theta = (0.3 * rng.standard_normal(fno.num_params)).astype(np.float32)
    fno.set_params(theta)
    H = _cells(n, [11, 12])
    Hd = torch.as_tensor(H, device=DEV)
    iu = torch.full((2, 3, 3, n, n, n), float("nan"), device=DEV)
    il = torch.full_like(iu, float("nan"))
    fno.warm_start(Hd, iu, il)
    iu, il = iu.cpu().numpy(), il.cpu().numpy()
    for j in range(3):
        perm = [0, 1, 2]
        perm[0], perm[j] = j, 0
        Hs = np.ascontiguousarray(H.transpose(0, *[p + 1 for p in perm]))
        out = torch.zeros((2, 6, n, n, n), device=DEV)
        fno.forward(torch.as_tensor(Hs, device=DEV), out)
        o = out.cpu().numpy()
        for c in range(3):
            sc = perm[c]
            u_ref = o[:, sc].transpose(0, *[p + 1 for p in perm])
            l_ref = o[:, 3 + sc].transpose(0, *[p + 1 for p in perm])
            np.testing.assert_allclose(iu[:, j, c], u_ref, rtol=1e-6, atol=1e-6 * np.abs(u_ref).max())
            np.testing.assert_allclose(il[:, j, c], l_ref, rtol=1e-6, atol=1e-6 * np.abs(l_ref).max())
    fno.close()


def test_warm_start_rejects_non_cubic_grids_and_host_outputs(lib):
    fno = lib.acm_fno((8, 16, 16), 4, 2, 1, max_batch=1)
    H = torch.zeros((1, 8, 16, 16), dtype=torch.uint8, device=DEV)
    u = torch.zeros((1, 3, 3, 8, 16, 16), device=DEV)
    with pytest.raises(lib.AcmError) as e:
        fno.warm_start(H, u, u.clone())
    assert e.value.status == -10
    fno.close()
    fno = lib.acm_fno((8, 8, 8), 4, 2, 1, max_batch=1)
    with pytest.raises(lib.AcmError) as e:
        fno.warm_start(torch.zeros((1, 8, 8, 8), dtype=torch.uint8, device=DEV), np.zeros((1, 3, 3, 8, 8, 8), np.float32),
                       np.zeros((1, 3, 3, 8, 8, 8), np.float32))
    assert e.value.status == -1
    fno.close()


def test_batch_restart_near_a_solution_needs_far_fewer_iterations(lib):
    """Restart from a converged (u, lambda) perturbed by 5 % voxelwise noise: the
    warm start (with its consistent pressure) cuts the iterations several-fold
    (the FP64 oracle on 16^3 cells of the same recipe: 138 and 214 against 3232
    and 6053 from zero). The exact solution itself is a poorer start under the
    adaptive penalties of Eq. 22, which restart from their initial values."""
    n = 32
    H = torch.as_tensor(_cells(n, [21, 22, 23]), device=DEV)
    batch = lib.acm_batch([(n, n, n)] * 3)
    # lengths in voxels (nu = h^2): velocities O(1), so the absolute part of the
    # tolerance of Eq. 11-12 does not dominate
    prm = lib.stokes_params(nu=1.0 / n ** 2, eps=1e-4, max_iter=20000, precision=lib.FP32)
    u = [torch.zeros((3, 3, n, n, n), device=DEV) for _ in range(3)]
    lam = [torch.zeros_like(x) for x in u]
    s, K0, r0 = lib.acm_batch_stokes(batch, list(H), prm, u_out=u, lambda_out=lam)
    assert s == 0 and all(x.converged for r in r0 for x in r)
    # lambda lives on the solid only
    for i in range(3):
        assert float(lam[i][:, :, ~H[i].bool()].abs().max()) == 0.0
        assert float(lam[i][:, :, H[i].bool()].abs().max()) > 0.0
    rng = np.random.Generator(np.random.PCG64(8))
    pert = [torch.as_tensor(1 + 0.05 * rng.standard_normal((2,) + tuple(x.shape)), dtype=torch.float32, device=DEV)
            for x in u]
    u = [x * e[0] for x, e in zip(u, pert)]
    lam = [x * e[1] for x, e in zip(lam, pert)]
    s, K1, r1 = lib.acm_batch_stokes(batch, list(H), prm, init_u=u, init_lambda=lam)
    assert s == 0 and all(x.converged for r in r1 for x in r)
    it0 = np.array([[x.iters for x in r] for r in r0])
    it1 = np.array([[x.iters for x in r] for r in r1])
    assert (it1 < 0.25 * it0).all(), (it0, it1)
    # both stops are within the accuracy the tolerance gives (a few per cent on K here)
    dK = np.linalg.norm(K1 - K0, axis=(1, 2)) / np.linalg.norm(K0, axis=(1, 2))
    assert (dK < 0.1).all(), dK
    # a warm start for one cell only leaves the others as from zero
    s, K2, r2 = lib.acm_batch_stokes(batch, list(H), prm, init_u=[u[0], None, None], init_lambda=[lam[0], None, None])
    it2 = np.array([[x.iters for x in r] for r in r2])
    assert (it2[0] == it1[0]).all() and (it2[1:] == it0[1:]).all()
    batch.close()


def test_trained_network_saves_iterations_on_held_out_cells(lib):
    """A small network trained by the library's own kernels on solutions of the
    method, evaluated on held-out seeds: fewer ADMM iterations to the same
    tolerance, and the same permeability."""
    from paper_2312_15554_gb300 import warm_start as WS
    r = WS.run(n=32, width=16, modes=6, layers=2, n_train=64, n_test=8, tol=1e-6, max_iter=20000, epochs=6,
               batch=4, lr=3e-3, chunk=64, seed=1, n_curve=0, log=lambda m: None)
    assert r["plain"]["converged_frac"] == 1.0 and r["warm"]["converged_frac"] == 1.0
    assert r["losses"][-1] < 0.5 * r["losses"][0]
    assert r["warm_start_velocity_rel_err"] < 0.5
    assert r["iterations_saved_frac"] > 0.1, r
    # the stop of Eq. 11-12 leaves K a few per cent from its limit in these units
    assert r["K_rel_diff_warm_vs_plain_max"] < 0.3

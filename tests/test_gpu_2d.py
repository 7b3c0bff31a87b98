"""The two-dimensional cell (n0 = 1, one plane): the paper's own setting
(Section 4: 128 x 128 grids), through the C ABI against the FP64 oracle.

With n0 = 1 the strided pass along axis 0 is a line of one point: its
transform is the identity and the pass applies the Green step (Eq. 13 or
Eq. 20) alone; the symbols of axis 0 are zero.
"""
import numpy as np
import pytest
import torch

from oracle import acm_oracle as O
from paper_2312_15554_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=DEV)


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("n", [64, 128])
@pytest.mark.parametrize("deriv", [O.EXACT, O.CENTRAL])
@pytest.mark.parametrize("fp64", [False, True])
def test_plane_stokes_fixed_iterations_match_oracle(lib, n, deriv, fp64):
    H = I.disk_pack(n, n, 0.6, (2.0 * n / 64, 6.0 * n / 64), 40 + n)
    g = [0.0, 1.0, 0.4]
    pen = dict(alpha0=250.0, beta0=180.0, b0=300.0)
    n_it = 12
    R = O.stokes(H, g, O.StokesParams(eps=0.0, adaptive=False, max_iter=n_it, deriv=deriv, **pen))
    dt = torch.float64 if fp64 else torch.float32
    ctx = lib.acm_ctx(H.shape)
    u = torch.zeros((3,) + H.shape, dtype=dt, device=DEV)
    p = torch.zeros(H.shape, dtype=dt, device=DEV)
    lam = torch.zeros((3,) + H.shape, dtype=dt, device=DEV)
    s, K, rep = lib.acm_stokes(ctx, dev(H, torch.uint8), g, lib.stokes_params(
        precision=lib.FP64 if fp64 else lib.FP32, eps=0.0, adaptive=0, max_iter=n_it, deriv=deriv, **pen),
        None, None, u, p, lam)
    ctx.close()
    assert s == lib.ACM_ERR_MAXITER and rep.iters == n_it
    tol = 1e-10 if fp64 else 1e-5
    assert relerr(u.cpu().numpy(), R.state.u) < tol
    assert relerr(p.cpu().numpy(), R.p) < tol
    assert relerr(lam.cpu().numpy(), R.state.lam) < tol
    assert np.abs(u.cpu().numpy()[0]).max() == 0.0      # no out-of-plane flow for an in-plane load


@pytest.mark.parametrize("fp64", [False, True])
def test_plane_solute_fixed_iterations_match_oracle(lib, fp64):
    n = 128
    H = I.disk_pack(n, n, 0.55, (3.0, 9.0), 77)
    u = 0.3 * I.random_field((3,) + H.shape, 78) * (1 - H)[None]
    u[0] = 0.0
    Pe = 5.0
    R = O.diffusivity_tensor(H, u, Pe, O.AdvDiffParams(eps=0.0, max_iter=6))
    dt = torch.float64 if fp64 else torch.float32
    ctx = lib.acm_ctx(H.shape)
    chi3 = torch.zeros((3,) + H.shape, dtype=dt, device=DEV)
    s, D, Dx, reps = lib.acm_advdiff_tensor(ctx, dev(H, torch.uint8), dev(u, dt), Pe, lib.advdiff_params(
        precision=lib.FP64 if fp64 else lib.FP32, eps=0.0, max_iter=6), chi3)
    ctx.close()
    tol = 1e-10 if fp64 else 1e-5
    assert relerr(chi3.cpu().numpy(), np.stack([r.chi for r in R[2]])) < tol
    assert relerr(D, R[0]) < (1e-10 if fp64 else 1e-6)
    assert relerr(Dx, R[1]) < (1e-10 if fp64 else 1e-6)


def test_square_cylinder_array_on_the_gpu(lib):
    """A disk of radius 0.2 at 64^2, FP64 with the central symbols, converged:
    K within 1e-6 of the oracle and within 3% of the cylinder-array formula of
    Sangani & Acrivos (1982) and Drummond & Tahir (1984)."""
    n = 64
    H = I.single_cylinder((1, n, n), 0.2)
    kw = dict(eps=1e-9, adaptive=False, alpha0=300.0, beta0=300.0, b0=300.0, max_iter=60000, deriv=O.CENTRAL)
    R = O.stokes(H, [0.0, 0.0, 1.0], O.StokesParams(**kw))
    assert R.converged
    ctx = lib.acm_ctx(H.shape)
    u = torch.zeros((3,) + H.shape, dtype=torch.float64, device=DEV)
    s, K, rep = lib.acm_stokes(ctx, dev(H, torch.uint8), [0.0, 0.0, 1.0], lib.stokes_params(precision=lib.FP64, **kw),
                               None, None, u, None, None)
    ctx.close()
    assert s == 0 and rep.converged and abs(rep.iters - R.iters) <= 1
    assert abs(K[2] / R.K_col[2] - 1) < 1e-6
    c = H.mean()
    k_arr = (-np.log(c) - 1.476 + 2 * c - 1.774 * c**2 + 4.076 * c**3) / (8 * np.pi)
    assert abs(K[2] / k_arr - 1) < 0.03


def test_plane_batch_and_tile_variants(lib):
    """Plane cells in a batch next to 3D cells, and the register-resident
    strided variants, give the single-cell results."""
    shapes = [(1, 128, 128), (32, 32, 32), (1, 128, 128)]
    Hs = [I.disk_pack(128, 128, 0.5, (3.0, 8.0), 90), I.sphere_pack((32, 32, 32), 0.5, 3.0, 91)[0],
          I.disk_pack(128, 128, 0.6, (3.0, 8.0), 92)]
    prm = lib.stokes_params(precision=lib.FP32, eps=0.0, adaptive=0, max_iter=10, alpha0=300, beta0=300, b0=300)
    batch = lib.acm_batch(shapes)
    u_out = [torch.zeros((3, 3) + sh, dtype=torch.float32, device=DEV) for sh in shapes]
    lib.acm_batch_stokes(batch, [dev(h, torch.uint8) for h in Hs], prm, u_out)
    torch.cuda.synchronize()
    batch.close()
    for i in (0, 2):
        for rr in (False, True):
            ctx = lib.acm_ctx(shapes[i])
            if rr:
                # the y passes (128 points) in the register-resident variant; the
                # z passes of a plane are lines of one point (no variants)
                t = lib.acm_get_tiles(ctx, False)
                t.update({k: -16 for k in t if k.startswith("y_")})
                lib.acm_set_tiles(ctx, t, False)
            u3 = torch.zeros((3, 3) + shapes[i], dtype=torch.float32, device=DEV)
            lib.acm_stokes_tensor(ctx, dev(Hs[i], torch.uint8), prm, u3)
            torch.cuda.synchronize()
            ctx.close()
            ref = u3.cpu().numpy()
            np.testing.assert_allclose(u_out[i].cpu().numpy(), ref, rtol=0, atol=1e-6 * np.abs(ref).max())

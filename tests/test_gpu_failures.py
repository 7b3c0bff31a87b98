"""Failure paths of the solvers, each produced through the C ABI and read as a
status on the host (no GPU fault is involved: the failing values are ordinary
numbers in device memory).

* ACM_ERR_DIVERGED: the Lippmann-Schwinger map of Section 3.2 contracts only
  for a large enough comparison medium (the paper's Section 4.2 study); at
  Pe = 0 its pore part scales gradients by (1 - A0) / A0, so A0 = 0.3 expands
  them 2.3-fold per iteration and the residual grows without bound.
* ACM_ERR_NONFINITE: a NaN in a velocity or a warm start reaches the residual
  norms in the first iteration.
* ACM_ERR_MAXITER: the cap ends a solve that has not met its tolerance, and
  every output is still written (it equals the oracle after as many iterations).
* FP32 rounding floor: with ACM_FP32_THEN_FP64 and an FP32 tolerance below
  what FP32 can reach, the FP32 phase stops when its residuals no longer gain
  on the tolerance and the FP64 phase finishes the solve.
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
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.mark.parametrize("device_loop", [1, 0])
def test_small_comparison_medium_is_reported_as_divergence(lib, device_loop):
    H = I.sphere_pack((16, 16, 16), 0.5, 3.0, 7)[0]
    ctx = lib.acm_ctx(H.shape)
    u = torch.zeros((3,) + H.shape, dtype=torch.float32, device=DEV)
    with pytest.raises(lib.AcmError) as e:
        lib.acm_advdiff(ctx, dev(H, torch.uint8), u, 0.0, [1.0, 0.0, 0.0],
                        lib.advdiff_params(A0=0.3, eps=1e-8, max_iter=2000, device_loop=device_loop))
    assert e.value.status == -5
    ctx.close()


def test_nan_in_the_velocity_is_reported_as_nonfinite(lib):
    H = I.sphere_pack((16, 16, 16), 0.5, 3.0, 8)[0]
    u = 0.1 * I.random_field((3,) + H.shape, 9) * (1 - H)[None]
    pore = np.argwhere(H == 0)[0]
    u[(1,) + tuple(pore)] = np.nan
    ctx = lib.acm_ctx(H.shape)
    with pytest.raises(lib.AcmError) as e:
        lib.acm_advdiff_tensor(ctx, dev(H, torch.uint8), dev(u, torch.float32), 5.0,
                               lib.advdiff_params(eps=1e-6, max_iter=100))
    assert e.value.status == -6
    ctx.close()


@pytest.mark.parametrize("fp64", [False, True])
def test_nan_in_a_warm_start_is_reported_as_nonfinite(lib, fp64):
    H = I.sphere_pack((16, 16, 16), 0.5, 3.0, 10)[0]
    dt = torch.float64 if fp64 else torch.float32
    u0 = np.zeros((3,) + H.shape)
    u0[0, 3, 4, 5] = np.nan
    ctx = lib.acm_ctx(H.shape)
    u = torch.zeros((3,) + H.shape, dtype=dt, device=DEV)
    with pytest.raises(lib.AcmError) as e:
        lib.acm_stokes(ctx, dev(H, torch.uint8), [1.0, 0.0, 0.0],
                       lib.stokes_params(precision=lib.FP64 if fp64 else lib.FP32, eps=1e-6, max_iter=50),
                       dev(u0, dt), None, u, None, None)
    assert e.value.status == -6
    ctx.close()


def test_iteration_cap_still_writes_every_output(lib):
    H = I.sphere_pack((16, 16, 16), 0.5, 3.0, 11)[0]
    g = [1.0, 0.0, 0.0]
    pen = dict(alpha0=250.0, beta0=180.0, b0=300.0)
    R = O.stokes(H, g, O.StokesParams(eps=1e-12, adaptive=False, max_iter=6, **pen))
    assert not R.converged
    ctx = lib.acm_ctx(H.shape)
    u = torch.zeros((3,) + H.shape, dtype=torch.float32, device=DEV)
    p = torch.zeros(H.shape, dtype=torch.float32, device=DEV)
    lam = torch.zeros((3,) + H.shape, dtype=torch.float32, device=DEV)
    s, K, rep = lib.acm_stokes(ctx, dev(H, torch.uint8), g, lib.stokes_params(
        precision=lib.FP32, eps=1e-12, adaptive=0, max_iter=6, **pen), None, None, u, p, lam)
    ctx.close()
    assert s == lib.ACM_ERR_MAXITER and rep.status == -4 and rep.iters == 6 and not rep.converged
    assert relerr(u.cpu().numpy(), R.state.u) < 1e-5
    assert relerr(p.cpu().numpy(), R.p) < 1e-5
    assert relerr(lam.cpu().numpy(), R.state.lam) < 1e-5
    assert relerr(K, R.K_col) < 1e-5


def test_fp32_phase_below_its_rounding_floor_hands_over_to_fp64(lib):
    """eps32 = 1e-9 is below what FP32 iterations can reach: the FP32 phase stops
    at its floor instead of burning max_iter, and FP64 converges to 1e-10 with
    the oracle's permeability."""
    H = I.single_sphere((16, 16, 16), 0.3)
    g = [1.0, 0.0, 0.0]
    kw = dict(eps=1e-10, adaptive=False, alpha0=300.0, beta0=300.0, b0=300.0, max_iter=20000, deriv=O.CENTRAL)
    R = O.stokes(H, g, O.StokesParams(**kw))
    assert R.converged
    ctx = lib.acm_ctx(H.shape)
    u = torch.zeros((3,) + H.shape, dtype=torch.float64, device=DEV)
    prm = lib.stokes_params(precision=lib.FP32_THEN_FP64, eps32=1e-9, **kw)
    s, K, rep = lib.acm_stokes(ctx, dev(H, torch.uint8), g, prm, None, None, u, None, None)
    ctx.close()
    assert s == 0 and rep.converged
    assert 0 < rep.iters_fp64 < rep.iters < kw["max_iter"]
    assert abs(K[0] / R.K_col[0] - 1) < 1e-6
    assert relerr(u.cpu().numpy(), R.state.u) < 1e-6

"""Re-solving an evolving geometry from the previous state.

As the solid dissolves, the cell changes a little between steps; the previous
velocity and multiplier (with the consistent pressure of the warm start) start
the ADMM of the next geometry, which runs to the same tolerance. The sequence
here dissolves a fifth of the interface solid per step.
"""
import numpy as np
import pytest
import torch

from paper_2312_15554_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def test_dissolution_sequence_restarts_from_the_previous_state(lib):
    n = 32
    H = I.sphere_pack((n, n, n), 0.3, (3.0, 6.0), 17)[0]
    ctx = lib.acm_ctx(H.shape)
    # lengths in voxels so that the tolerance of Eq. 11-12 is relative in effect
    prm = lib.stokes_params(nu=1.0 / n ** 2, eps=1e-5, max_iter=40000, precision=lib.FP32)
    g = [1.0, 0.0, 0.0]
    u = torch.zeros((3, n, n, n), device=DEV)
    lam = torch.zeros_like(u)
    s, K, rep = lib.acm_stokes(ctx, torch.as_tensor(H, device=DEV), g, prm, u=u, lam=lam)
    assert rep.converged
    saved = []
    for step in range(3):
        H = I.dissolve(H, 1, fraction=0.2, seed=step)
        Hd = torch.as_tensor(H, device=DEV)
        uz = torch.zeros_like(u)
        s0, K0, r0 = lib.acm_stokes(ctx, Hd, g, prm, u=uz)
        u1, l1 = torch.zeros_like(u), torch.zeros_like(u)
        s1, K1, r1 = lib.acm_stokes(ctx, Hd, g, prm, init_u=u, init_lambda=lam, u=u1, lam=l1)
        assert r0.converged and r1.converged
        saved.append(1 - r1.iters / r0.iters)
        # both stops agree to the accuracy the tolerance gives
        assert abs(K1[0] / K0[0] - 1) < 2e-2, (step, K0, K1)
        u, lam = u1, l1
    # the previous state is the better start at every step
    assert min(saved) > 0.2, saved
    ctx.close()

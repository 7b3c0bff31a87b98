"""Pins of the FNO oracle: finite-difference gradients and special cases."""
import numpy as np
import pytest

from oracle import fno_oracle as F
from paper_2312_15554_gb300 import inputs as I


def _setup(shape=(8, 8, 8), width=4, modes=2, layers=2, seed=3):
    H = I.random_indicator(shape, 0.4, seed)
    theta = F.init_params(width, modes, layers, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    theta = theta + 0.3 * rng.standard_normal(theta.size) * (np.abs(theta).max() + 0.1) * 0.1
    target = rng.standard_normal((6,) + shape)
    return H, theta, target


def _loss(theta, H, target, cfg):
    out, _ = F.forward(theta, H, *cfg)
    return F.loss_and_grad_out(out, target, H)[0]


@pytest.mark.parametrize("cfg", [(4, 2, 2), (3, 1, 1)])
def test_gradient_matches_central_differences(cfg):
    H, theta, target = _setup(width=cfg[0], modes=cfg[1], layers=cfg[2])
    out, cache = F.forward(theta, H, *cfg)
    L, dout = F.loss_and_grad_out(out, target, H)
    g = F.backward(theta, H, cache, dout, *cfg)
    rng = np.random.Generator(np.random.PCG64(9))
    # random directions
    for _ in range(3):
        d = rng.standard_normal(theta.size)
        h = 1e-6
        fd = (_loss(theta + h * d, H, target, cfg) - _loss(theta - h * d, H, target, cfg)) / (2 * h)
        assert fd == pytest.approx(g @ d, rel=1e-6, abs=1e-9)
    # individual entries of every parameter block
    o = 0
    for name, sh in F.param_shapes(*cfg):
        n = int(np.prod(sh))
        for j in (o, o + n // 2, o + n - 1):
            e = np.zeros(theta.size)
            e[j] = 1.0
            h = 1e-6
            fd = (_loss(theta + h * e, H, target, cfg) - _loss(theta - h * e, H, target, cfg)) / (2 * h)
            assert fd == pytest.approx(g[j], rel=1e-5, abs=1e-9), name
        o += n


def test_truncated_transforms_follow_their_direct_sum_definitions():
    """F(v)(k) = sum_x v exp(-2 pi i k.x/n) on the kept modes and
    G(Y)(x) = (1/V) sum_k w_k Re[Y(k) exp(2 pi i k.x/n)], evaluated as explicit
    sums, equal the FFT-based implementation (indices, signs, weights, scaling)."""
    shape = (4, 6, 8)
    modes = 2
    rng = np.random.Generator(np.random.PCG64(1))
    v = rng.standard_normal((1,) + shape)
    Y = rng.standard_normal((1, 4 * modes ** 3)) + 1j * rng.standard_normal((1, 4 * modes ** 3))
    idx = F.kept_modes(shape, modes)
    j = [np.arange(n) for n in shape]
    J0, J1, J2 = np.meshgrid(*j, indexing="ij")
    Fd = np.zeros(len(idx[0]), complex)
    Gd = np.zeros(shape)
    for m, (a0, a1, a2) in enumerate(zip(*idx)):
        th = 2 * np.pi * (a0 * J0 / shape[0] + a1 * J1 / shape[1] + a2 * J2 / shape[2])
        Fd[m] = np.sum(v[0] * np.exp(-1j * th))
        w = 1.0 if a2 == 0 else 2.0
        Gd += w * (Y[0, m] * np.exp(1j * th)).real / v[0].size
    np.testing.assert_allclose(F._fwd_dft(v, idx)[0], Fd, atol=1e-12)
    np.testing.assert_allclose(F._inv_dft(Y, idx, shape)[0], Gd, atol=1e-12)


def test_loss_ignores_lambda_on_pore_voxels():
    H, theta, target = _setup()
    out, _ = F.forward(theta, H, 4, 2, 2)
    L1, _ = F.loss_and_grad_out(out, target, H)
    t2 = target.copy()
    t2[3:, H == 0] += 5.0
    L2, _ = F.loss_and_grad_out(out, t2, H)
    assert L1 == pytest.approx(L2, rel=1e-14)

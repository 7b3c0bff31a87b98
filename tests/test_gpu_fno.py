"""The learned warm start's GPU kernels against the FP64 FNO oracle.

The oracle runs with the same BF16-rounded parameters, so the differences are
the BF16 storage of activations and FP32 arithmetic: forward and loss within
2e-2 relative, gradients with cosine similarity above 0.999 and relative error
at most 2e-2.
"""
import numpy as np
import pytest
import torch

from oracle import fno_oracle as F
from paper_2312_15554_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def bf16_round(x):
    return torch.as_tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def _case(shape, width, modes, layers, B, seed):
    theta = F.init_params(width, modes, layers, seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = theta + 0.05 * rng.standard_normal(theta.size)
    theta = bf16_round(theta)
    Hs = np.stack([I.sphere_pack(shape, 0.5, 2.5, seed + b)[0] for b in range(B)])
    tgt = 0.5 * rng.standard_normal((B, 6) + shape)
    return theta, Hs, tgt


@pytest.mark.parametrize("shape,width,modes,layers,B", [((16, 16, 16), 8, 3, 2, 2), ((8, 16, 32), 4, 2, 3, 3),
                                                       ((32, 32, 32), 32, 4, 2, 1),
                                                       ((64, 64, 64), 32, 12, 4, 1)])  # the trained size
def test_fno_forward_loss_and_gradient_match_oracle(lib, shape, width, modes, layers, B):
    theta, Hs, tgt = _case(shape, width, modes, layers, B, 7)
    fno = lib.acm_fno(shape, width, modes, layers, max_batch=4)
    assert fno.num_params == F.n_params(width, modes, layers)
    fno.set_params(theta.astype(np.float32))
    Hd = torch.as_tensor(Hs, device=DEV)
    out = torch.zeros((B, 6) + shape, dtype=torch.float32, device=DEV)
    fno.forward(Hd, out)
    grad = torch.zeros(fno.num_params, dtype=torch.float32, device=DEV)
    loss = fno.backward(Hd, torch.as_tensor(tgt, dtype=torch.float32, device=DEV), grad)
    out = out.cpu().numpy()
    g = grad.cpu().numpy().astype(np.float64)
    L_ref, g_ref = 0.0, np.zeros_like(g)
    for b in range(B):
        o, cache = F.forward(theta, Hs[b], width, modes, layers)
        np.testing.assert_allclose(out[b], o, atol=2e-2 * np.abs(o).max())
        Lb, dout = F.loss_and_grad_out(o, tgt[b], Hs[b])
        L_ref += Lb / B
        g_ref += F.backward(theta, Hs[b], cache, dout / B, width, modes, layers)
    assert loss == pytest.approx(L_ref, rel=2e-2)
    cos = g @ g_ref / (np.linalg.norm(g) * np.linalg.norm(g_ref))
    assert cos > 0.999
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 2e-2
    # one AdamW step on the device equals the update written out on the host
    lr, b1, b2, eps, wd = 1e-3, 0.9, 0.999, 1e-8, 1e-4
    fno.adamw(lr, b1, b2, eps, wd)
    new = fno.get_params().astype(np.float64)
    m, v = (1 - b1) * g, (1 - b2) * g * g
    ref = theta - lr * ((m / (1 - b1)) / (np.sqrt(v / (1 - b2)) + eps) + wd * theta)
    np.testing.assert_allclose(new, ref, rtol=1e-5, atol=1e-7)
    fno.close()

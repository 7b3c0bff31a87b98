"""The exact-against-central symbol study (Section 3.2, Eq. 21; Section 4.2)
on the GPU, one point against the FP64 oracle: iterations to the tolerance,
D, and the high-band energy fraction of grad chi, for both symbol sets.

The oracle side forms the energy fraction from the full spectrum (no
Hermitian weights), an independent route to the module's half-spectrum sums.
"""
import numpy as np
import pytest
import torch

from oracle import acm_oracle as O
from oracle import fft as OF
from paper_2312_15554_gb300 import inputs as I
from paper_2312_15554_gb300 import symbol_study as S

pytestmark = pytest.mark.gpu


def oracle_hf(grad):
    shape = grad.shape[1:]
    m = [np.minimum(np.arange(n), n - np.arange(n)) for n in shape]
    hi = np.zeros(shape, bool)
    for a, n in enumerate(shape):
        if n > 1:
            b = [1, 1, 1]
            b[a] = n
            hi = hi | (m[a].reshape(b) * 4 >= n)
    e = np.abs(OF.fftn(grad, axes=(1, 2, 3))) ** 2
    return float(e[:, hi].sum() / e.sum())


@pytest.mark.parametrize("Pe", [0.0, 10.0])
def test_symbol_study_point_matches_the_oracle(lib, Pe):
    n = 32
    H = I.sphere_pack((n, n, n), 0.5, n / 8.0, 7)[0]
    R = O.stokes(H, [1.0, 0.0, 0.0], O.StokesParams(nu=1.0 / n**2, eps=0.0, max_iter=40, adaptive=False,
                                                    alpha0=2.0, beta0=2.0, b0=2.0, deriv=O.CENTRAL))
    u = R.state.u / np.abs(R.state.u).max()
    for name, d in S.DERIVS.items():
        ref = O.advdiff(H, u, Pe, [1.0, 0.0, 0.0], O.AdvDiffParams(eps=1e-9, max_iter=20000, deriv=d))
        assert ref.converged
        got = S.solute_metrics(H, torch.as_tensor(u, device="cuda"), Pe, d, eps=1e-9, precision=lib.FP64)
        assert got["converged"] and abs(got["iters"] - ref.iters) <= 1, (name, got["iters"], ref.iters)
        np.testing.assert_allclose(got["D_col"], ref.Dg, rtol=1e-7, atol=1e-12)
        assert got["hf"] == pytest.approx(oracle_hf(ref.grad_chi), rel=1e-5)
    # the symbols differ where the study says they do: the exact one leaves far
    # more of grad chi's energy in the upper band
    ex = S.solute_metrics(H, torch.as_tensor(u, device="cuda"), Pe, S.DERIVS["exact"], eps=1e-9, precision=lib.FP64)
    ce = S.solute_metrics(H, torch.as_tensor(u, device="cuda"), Pe, S.DERIVS["central"], eps=1e-9,
                          precision=lib.FP64)
    assert ex["hf"] > 5 * ce["hf"]

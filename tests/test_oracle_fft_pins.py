"""Pins of the oracle's own transform (oracle/fft.py, oracle/oracle_fft.c).

The fast transform is checked against the DFT written out by its definition
(explicit exponentials, phases reduced modulo n in integers), against closed
forms (single modes, Parseval), and, as a special case that reduces to a
library routine, against numpy's FFT.
"""
import numpy as np
import pytest

from oracle import fft as F


def _rand(shape, seed, cplx=True):
    r = np.random.default_rng(seed)
    x = r.standard_normal(shape)
    if cplx:
        x = x + 1j * r.standard_normal(shape)
    return x


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64, 3, 6, 10])
@pytest.mark.parametrize("sign", [-1, +1])
def test_each_axis_length_matches_the_direct_dft(n, sign):
    x = _rand((5, n), n)
    ref = F.dft_direct(x, axis=-1, sign=sign)
    got = F.fftn(x, axes=(-1,)) if sign < 0 else F.ifftn(x, axes=(-1,)) * n
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_three_axes_are_the_product_of_the_axis_dfts():
    x = _rand((8, 16, 4), 3)
    ref = F.dft_direct(F.dft_direct(F.dft_direct(x, 0), 1), 2)
    got = F.fftn(x, axes=(0, 1, 2))
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    # strided middle axis of a batched array: only that axis moves
    y = _rand((3, 16, 8, 4), 4)
    got = F.fftn(y, axes=(2,))
    assert np.abs(got - F.dft_direct(y, 2)).max() < 1e-13 * np.abs(got).max()


def test_single_mode_transforms_to_one_coefficient():
    shape = (8, 4, 16)
    m = (3, 1, 5)
    j = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    x = np.exp(2j * np.pi * sum(m[c] * j[c] / shape[c] for c in range(3)))
    X = F.fftn(x)
    ref = np.zeros(shape, complex)
    ref[m] = np.prod(shape)
    assert np.abs(X - ref).max() < 1e-12 * np.prod(shape)


def test_parseval_and_round_trip():
    x = _rand((16, 32, 8), 5, cplx=False)
    X = F.fftn(x)
    assert np.sum(np.abs(X) ** 2) / x.size == pytest.approx(np.sum(x * x), rel=1e-13)
    np.testing.assert_allclose(F.ifftn(X).real, x, atol=1e-14 * np.abs(x).max())
    assert np.abs(F.ifftn(X).imag).max() < 1e-14 * np.abs(x).max()


def test_library_fft_is_a_special_case():
    x = _rand((32, 64, 16), 6)
    assert np.abs(F.fftn(x) - np.fft.fftn(x)).max() < 1e-13 * np.abs(np.fft.fftn(x)).max()


def test_half_spectrum_real_transforms():
    shape = (4, 8, 8)
    x = _rand(shape, 7, cplx=False)
    h = F.rfftn(x)
    assert h.shape == (4, 8, 5)
    np.testing.assert_allclose(h, F.fftn(x)[..., :5], atol=1e-13 * np.abs(h).max())
    # irfftn is (1/V) sum over the half spectrum of w Re[Y exp(2 pi i m.x)],
    # w = 1 on the planes m2 = 0 and m2 = n2/2, 2 elsewhere: checked by that sum
    Y = _rand(h.shape, 8)
    j = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    ref = np.zeros(shape)
    V = np.prod(shape)
    for m0 in range(shape[0]):
        for m1 in range(shape[1]):
            for m2 in range(shape[2] // 2 + 1):
                w = 1.0 if m2 in (0, shape[2] // 2) else 2.0
                ph = 2 * np.pi * (m0 * j[0] / shape[0] + m1 * j[1] / shape[1] + m2 * j[2] / shape[2])
                ref += w * np.real(Y[m0, m1, m2] * np.exp(1j * ph)) / V
    got = F.irfftn(Y, s=shape)
    np.testing.assert_allclose(got, ref, atol=1e-13 * np.abs(ref).max())
    # the library's inverse real transform follows the same convention
    np.testing.assert_allclose(got, np.fft.irfftn(Y, s=shape, axes=(0, 1, 2)), atol=1e-13 * np.abs(ref).max())
    # and a real field survives the round trip through its half spectrum
    np.testing.assert_allclose(F.irfftn(h, s=shape), x, atol=1e-13 * np.abs(x).max())


def test_runs_on_the_host_threads():
    assert F.threads() >= 1

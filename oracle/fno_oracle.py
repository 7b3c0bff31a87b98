"""FP64 CPU oracle of the learned warm start: a Fourier neural operator.

TEST INFRASTRUCTURE ONLY (like acm_oracle): used by the tests, never by the
product library.

The paper motivates fast repeated unit-cell solves (Section 5: a neural operator
trained on ACM solutions for the macroscopic model). The warm start here is a
small 3D Fourier neural operator that maps the indicator H of a cell to an
initial velocity u and solid multiplier lambda for the ADMM of Section 3.1;
the ADMM then runs to its tolerance as usual.

Model (width W, `modes` kept per axis, L layers), on a grid (n0, n1, n2):
  features  a = (H, x0, x1, x2), x_c = (i_c + 1/2) / n_c                    (4 channels)
  lift      v = P a + p                                                     (W channels)
  layer l   v <- gelu(S_l(v) + M_l v + m_l)
            S_l(v) = G(R_l(k) F(v)(k))  on the kept modes k
            F(v)(k) = sum_x v(x) exp(-2 pi i k.x/n)   (forward DFT, kept modes only)
            G(Y)(x) = (1/V) sum_k w_k Re[Y(k) exp(2 pi i k.x/n)]  (w_k = 1 at k2 = 0, 2 else)
  project   out = Q v + q                                                   (6 channels: u, lambda)
Kept modes: k2 in [0, modes) of the half spectrum, k1 and k0 in
[0, modes) U [n - modes, n) (the four corner blocks).

Loss: L = 1/(B V) sum_b sum_x [ sum_{c<3} (out_c - t_c)^2 + H sum_{c>=3} (out_c - t_c)^2 ].
Parameters are one flat FP64 vector, in the order of `param_shapes`.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from oracle import fft as FFT


def kept_modes(shape, modes):
    """Index arrays (i0, i1, i2) of the kept modes in the rfftn layout, mode order
    m = (j0 * 2 modes + j1) * modes + j2."""
    n0, n1, n2 = shape
    if not (2 * modes <= n0 and 2 * modes <= n1 and modes <= n2 // 2):
        raise ValueError("too many modes for the grid")
    r0 = list(range(modes)) + list(range(n0 - modes, n0))
    r1 = list(range(modes)) + list(range(n1 - modes, n1))
    i0, i1, i2 = np.meshgrid(r0, r1, list(range(modes)), indexing="ij")
    return i0.ravel(), i1.ravel(), i2.ravel()


def param_shapes(width, modes, layers):
    nm = 4 * modes ** 3
    shapes = [("P", (width, 4)), ("p", (width,))]
    for l in range(layers):
        shapes += [(f"R{l}", (nm, width, width, 2)), (f"M{l}", (width, width)), (f"m{l}", (width,))]
    shapes += [("Q", (6, width)), ("q", (6,))]
    return shapes


def unflatten(theta, width, modes, layers):
    out, o = {}, 0
    for name, sh in param_shapes(width, modes, layers):
        n = int(np.prod(sh))
        out[name] = theta[o:o + n].reshape(sh)
        o += n
    assert o == theta.size
    return out


def n_params(width, modes, layers):
    return sum(int(np.prod(sh)) for _, sh in param_shapes(width, modes, layers))


def features(H):
    n0, n1, n2 = H.shape
    x = [(np.arange(n) + 0.5) / n for n in (n0, n1, n2)]
    X = np.meshgrid(*x, indexing="ij")
    return np.stack([H.astype(np.float64), X[0], X[1], X[2]])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _fwd_dft(v, idx):
    """F(v) on the kept modes: (C, M) complex."""
    vh = FFT.rfftn(v, axes=(1, 2, 3))
    return vh[:, idx[0], idx[1], idx[2]]


def _inv_dft(Y, idx, shape):
    """G(Y): (C, M) complex on the kept modes -> real field (C, ...)."""
    C = Y.shape[0]
    yh = np.zeros((C, shape[0], shape[1], shape[2] // 2 + 1), dtype=np.complex128)
    yh[:, idx[0], idx[1], idx[2]] = Y
    return FFT.irfftn(yh, s=shape, axes=(1, 2, 3))


def forward(theta, H, width, modes, layers):
    """Returns (out (6, ...), cache for backward)."""
    prm = unflatten(theta, width, modes, layers)
    shape = H.shape
    idx = kept_modes(shape, modes)
    a = features(H)
    v = np.einsum("ca,a...->c...", prm["P"], a) + prm["p"][:, None, None, None]
    cache = {"a": a, "vs": [], "xh": [], "zs": [], "idx": idx}
    for l in range(layers):
        R = prm[f"R{l}"][..., 0] + 1j * prm[f"R{l}"][..., 1]          # (M, W, W)
        X = _fwd_dft(v, idx)                                             # (W, M)
        Y = np.einsum("mij,jm->im", R, X)
        y = _inv_dft(Y, idx, shape)
        z = y + np.einsum("ij,j...->i...", prm[f"M{l}"], v) + prm[f"m{l}"][:, None, None, None]
        cache["vs"].append(v)
        cache["xh"].append(X)
        cache["zs"].append(z)
        v = gelu(z)
    cache["v_last"] = v
    out = np.einsum("ij,j...->i...", prm["Q"], v) + prm["q"][:, None, None, None]
    return out, cache


def loss_and_grad_out(out, target, H):
    """Loss of one sample (divided by V) and dL/dout."""
    V = H.size
    Hf = H.astype(np.float64)
    mask = np.concatenate([np.ones((3,) + H.shape), np.broadcast_to(Hf, (3,) + H.shape)])
    d = (out - target) * mask
    return float(np.sum(d * d)) / V, 2.0 * d / V


def backward(theta, H, cache, dout, width, modes, layers):
    """Gradient of the loss w.r.t. the flat parameter vector (same layout)."""
    prm = unflatten(theta, width, modes, layers)
    grads = {k: np.zeros_like(v) for k, v in prm.items()}
    shape = H.shape
    V = H.size
    idx = cache["idx"]
    wk = np.where(idx[2] == 0, 1.0, 2.0)
    v = cache["v_last"]
    grads["Q"] = dout.reshape(6, -1) @ v.reshape(width, -1).T
    grads["q"] = dout.reshape(6, -1).sum(axis=1)
    dv = np.einsum("ij,i...->j...", prm["Q"], dout)
    for l in reversed(range(layers)):
        z, vin, X = cache["zs"][l], cache["vs"][l], cache["xh"][l]
        dz = dv * gelu_grad(z)
        grads[f"M{l}"] = dz.reshape(width, -1) @ vin.reshape(width, -1).T
        grads[f"m{l}"] = dz.reshape(width, -1).sum(axis=1)
        dv_new = np.einsum("ij,i...->j...", prm[f"M{l}"], dz)
        # y = G(Y): dL/dY(k) = (w_k / V) F(dz)(k)
        gY = _fwd_dft(dz, idx) * (wk / V)[None, :]
        R = prm[f"R{l}"][..., 0] + 1j * prm[f"R{l}"][..., 1]
        gR = np.einsum("im,jm->mij", gY, np.conj(X))                  # dL/dR = gY X^H
        grads[f"R{l}"] = np.stack([gR.real, gR.imag], axis=-1)
        gX = np.einsum("mij,im->jm", np.conj(R), gY)                  # R^H gY
        # X = F(v): dL/dv(x) = sum_k Re[gX(k) exp(2 pi i k.x/n)] = V * G(gX / w_k)
        dv_new = dv_new + V * _inv_dft(gX / wk[None, :], idx, shape)
        dv = dv_new
    a = cache["a"]
    grads["P"] = dv.reshape(width, -1) @ a.reshape(4, -1).T
    grads["p"] = dv.reshape(width, -1).sum(axis=1)
    return np.concatenate([grads[k].ravel() for k, _ in param_shapes(width, modes, layers)])


def init_params(width, modes, layers, seed):
    """Seeded initial parameters (scaled like a standard FNO initialisation)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for name, sh in param_shapes(width, modes, layers):
        if name.startswith("R"):
            scale = 1.0 / (width * width)
            parts.append(scale * rng.random(sh))
        elif name in ("P", "Q") or name.startswith("M"):
            fan_in = sh[1]
            parts.append(rng.uniform(-1, 1, sh) / math.sqrt(fan_in))
        else:
            parts.append(np.zeros(sh))
    return np.concatenate([p.ravel() for p in parts])

"""Exact against central derivative symbols in the solute iteration.

Section 3.2 (Eq. 21) replaces the exact spectral derivative i k by the symbol
of the central difference, i sin(h k)/h (and the Laplacian by its compact
three-point symbol), and Section 4.2 shows why: with the exact symbol the
concentration gradient oscillates at the solid-pore interfaces. This module
measures that on the GPU for a cell and its own flow, with both symbol sets
and everything else equal:

* iterations of the Lippmann-Schwinger loop to the tolerance of Eq. 19,
* D (Eq. 3, first column: composition load e_0) and the extended-domain D,
* hf: the fraction of the energy of grad chi carried by wavenumbers with
  max_c |m_c| >= N_c / 4 (the upper half of every axis' band); the Gibbs
  ripple of the exact derivative at a jump keeps it large at every grid size.

The flow is the library's Stokes solution of load e_0 in voxel units
(nu = h^2, so velocities are O(1)), scaled to a largest speed of 1. Every step
runs in the library (the transform of grad chi included); numpy only forms the
weighted sums of the returned spectrum.

Usage: python -m paper_2312_15554_gb300.symbol_study [--n 64 128 256] [--pe 0 10]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from paper_2312_15554_gb300 import acm
from paper_2312_15554_gb300 import inputs as I

DERIVS = {"exact": acm.DERIV_EXACT, "central": acm.DERIV_CENTRAL}


def band_energy(spec, shape):
    """(high-band, total) energy of a real field from its half spectrum spec
    [n0][n1][n2/2+1] (complex): Parseval with weight 2 on the interior columns
    of the half axis; the high band is max_c |m_c| >= n_c / 4 over the axes
    longer than one point."""
    n0, n1, n2 = shape

    def absfreq(n):
        i = np.arange(n)
        return np.minimum(i, n - i)
    w = np.full(n2 // 2 + 1, 2.0)
    w[0] = 1.0
    w[n2 // 2] = 1.0
    e = np.abs(spec) ** 2 * w[None, None, :]
    hi = (absfreq(n1)[None, :, None] * 4 >= n1) | (np.arange(n2 // 2 + 1)[None, None, :] * 4 >= n2)
    if n0 > 1:
        hi = hi | (absfreq(n0)[:, None, None] * 4 >= n0)
    hi = np.broadcast_to(hi, e.shape)
    return float(e[hi].sum()), float(e.sum())


def solute_metrics(H, u, Pe, deriv, eps=1e-6, precision=None, max_iter=20000, A0=0.55, eta=0.01):
    """The metrics of one symbol set for load e_0 (u: a torch tensor on the GPU)."""
    import torch
    precision = acm.FP32 if precision is None else precision
    dt = torch.float64 if precision == acm.FP64 else torch.float32
    shape = tuple(H.shape)
    ctx = acm.acm_ctx(shape)
    grad = torch.zeros((3,) + shape, dtype=dt, device="cuda")
    prm = acm.advdiff_params(eps=eps, max_iter=max_iter, deriv=deriv, precision=precision, A0=A0, eta=eta)
    s, Dg, Dx, rep = acm.acm_advdiff(ctx, torch.as_tensor(H, device="cuda"), u.to(dt).contiguous(), Pe,
                                     [1.0, 0.0, 0.0], prm, None, grad)
    spec = torch.zeros((3,) + shape[:2] + (shape[2] // 2 + 1, 2), dtype=dt, device="cuda")
    acm.acm_fft_r2c(ctx, grad, spec, precision == acm.FP64, 3)
    torch.cuda.synchronize()
    ctx.close()
    sp = spec.cpu().numpy().astype(np.float64)
    sp = sp[..., 0] + 1j * sp[..., 1]
    hi = tot = 0.0
    for c in range(3):
        a, b = band_energy(sp[c], shape)
        hi += a
        tot += b
    return {"iters": rep.iters, "converged": bool(rep.converged), "status": rep.status, "D_col": Dg.tolist(),
            "D_ext_col": Dx.tolist(), "hf": hi / tot}


def flow(H, eps=1e-5, max_iter=20000):
    """Converged FP32 Stokes flow of load e_0 in voxel units (nu = 1/n^2 of the
    geometric-mean grid size), central symbols, scaled to max |u| = 1."""
    import torch
    shape = tuple(H.shape)
    n = float(np.prod([s for s in shape if s > 1])) ** (1.0 / sum(1 for s in shape if s > 1))
    ctx = acm.acm_ctx(shape)
    u = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    prm = acm.stokes_params(nu=1.0 / n ** 2, eps=eps, max_iter=max_iter, deriv=acm.DERIV_CENTRAL, precision=acm.FP32)
    s, K, rep = acm.acm_stokes(ctx, torch.as_tensor(H, device="cuda"), [1.0, 0.0, 0.0], prm, None, None, u, None,
                               None)
    torch.cuda.synchronize()
    ctx.close()
    return u / u.abs().max(), rep


def study(n, Pe_list, eps=1e-6, seed=7):
    """Both symbol sets on a pack of spheres of radius n/8 at porosity 0.5."""
    H = I.sphere_pack((n, n, n), 0.5, n / 8.0, seed)[0]
    u, frep = flow(H)
    out = {"n": n, "porosity": float(1 - H.mean()), "flow_iters": frep.iters, "flow_converged": bool(frep.converged)}
    for Pe in Pe_list:
        res = {name: solute_metrics(H, u, Pe, d, eps=eps) for name, d in DERIVS.items()}
        ex, ce = res["exact"], res["central"]
        out[f"Pe{Pe:g}"] = {
            **res,
            "iteration_ratio": ex["iters"] / max(ce["iters"], 1),
            "D00_gap": abs(ex["D_col"][0] - ce["D_col"][0]) / abs(ce["D_col"][0]),
        }
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[64, 128, 256])
    ap.add_argument("--pe", type=float, nargs="+", default=[0.0, 10.0])
    ap.add_argument("--eps", type=float, default=1e-6)
    args = ap.parse_args()
    acm.load()
    for n in args.n:
        print(json.dumps(study(n, args.pe, args.eps)), flush=True)


if __name__ == "__main__":
    main()

"""Parameter sweeps of the two iterations (the 3D counterparts of the paper's
penalty study for the Stokes ADMM, Section 5 with Eq. 22, and its
comparison-medium study for the Lippmann-Schwinger iteration, Section 3.2).

* Stokes: iterations to a tolerance for fixed penalties alpha = beta = b at
  multiples of the default and for the adaptive rule of Eq. 22 (both tau sets
  the paper uses), on a batch of seeded sphere packs, all three loads.
* Solute: iterations to a tolerance against A0 for one flow field at a given
  Peclet number; a run that diverges or hits the cap is reported as such.

The converged answers do not depend on these parameters; only the iteration
counts do. Run as a module; prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np


def stokes_penalties(acm, Hs, nu, eps, max_iter, stream, factors=(0.25, 1.0, 4.0, 16.0)):
    """Iterations (mean, max over problems) and converged fraction per setting."""
    import torch
    n = Hs[0].shape[0]
    shapes = [tuple(h.shape) for h in Hs]
    batch = acm.acm_batch(shapes, stream.cuda_stream)
    p0 = nu * (math.pi * n) ** 2 / 8
    settings = [("adaptive, tau (5, 10, 5)", {}), ("adaptive, tau (20, 10, 30)", {"tau": (20.0, 10.0, 30.0)})]
    settings += [(f"fixed {f:g} x default", {"adaptive": 0, "alpha0": f * p0, "beta0": f * p0, "b0": f * p0})
                 for f in factors]
    out = {}
    for name, kw in settings:
        prm = acm.stokes_params(nu=nu, eps=eps, max_iter=max_iter, precision=acm.FP32, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, K, reps = acm.acm_batch_stokes(batch, Hs, prm)
        e1.record(stream)
        torch.cuda.synchronize()
        it = np.array([[r.iters for r in rr] for rr in reps])
        conv = np.array([[r.converged for r in rr] for rr in reps])
        out[name] = {"iters_mean": float(it.mean()), "iters_max": int(it.max()),
                     "converged_frac": float(conv.mean()), "seconds": e0.elapsed_time(e1) / 1e3,
                     "K_mean_diag": float(np.mean([np.trace(k) / 3 for k in K]) * nu)}
    batch.close()
    return {"default_penalty": p0, "settings": out}


def solute_a0(acm, H, u, Pe, eps, max_iter, stream, a0s=(0.3, 0.4, 0.55, 0.7, 1.0, 1.5, 2.0)):
    """Iterations of the three composition loads against A0 (B0 = mean of B)."""
    import torch
    ctx = acm.acm_ctx(H.shape, stream.cuda_stream)
    Hd = torch.as_tensor(H, device=u.device)
    out = {}
    for a0 in a0s:
        prm = acm.advdiff_params(A0=a0, eps=eps, max_iter=max_iter, precision=acm.FP32)
        try:
            s, D, Dx, reps = acm.acm_advdiff_tensor(ctx, Hd, u, Pe, prm)
            out[f"{a0:g}"] = {"iters": [r.iters for r in reps], "converged": [bool(r.converged) for r in reps],
                              "status": int(s), "D_diag": [float(D[i, i]) for i in range(3)]}
        except acm.AcmError as e:  # diverged or non-finite: no answer at this A0
            out[f"{a0:g}"] = {"status": int(e.status), "error": str(e)}
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--cells", type=int, default=16)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--pe", type=float, default=10.0)
    ap.add_argument("--solute-eps", type=float, default=1e-6)
    a = ap.parse_args()
    import torch

    from . import acm
    from . import build as B
    from . import inputs as I
    B.build()
    acm.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    n = a.n
    Hs = []
    for s in range(a.cells):
        por, radii = I.cell_recipe(700_000 + s)
        Hs.append(I.sphere_pack((n, n, n), por, radii, 700_000 + s)[0])
    Hd = [torch.as_tensor(h, device=dev) for h in Hs]
    # lengths in voxels: velocities O(1), so the tolerance is relative in effect
    nu = 1.0 / n ** 2
    res = {"grid": n, "cells": a.cells, "nu": nu, "stokes_eps": a.eps}
    res["stokes"] = stokes_penalties(acm, Hd, nu, a.eps, a.max_iter, stream)
    # the solute study on the first cell, with its converged flow for the load e_0 (unit-cell units)
    ctx = acm.acm_ctx(Hs[0].shape, stream.cuda_stream)
    u = torch.zeros((3,) + Hs[0].shape, dtype=torch.float32, device=dev)
    acm.acm_stokes(ctx, Hd[0], [1.0, 0.0, 0.0], acm.stokes_params(nu=nu, eps=a.eps, max_iter=a.max_iter,
                                                                  precision=acm.FP32), u=u)
    ctx.close()
    u *= nu
    res["solute"] = {"Pe": a.pe, "eps": a.solute_eps,
                     "A0": solute_a0(acm, Hs[0], u, a.pe, a.solute_eps, a.max_iter, stream)}
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()

"""Time to permeability: how long until K stays within a relative error of its
limit, for the plain, batched and learned-warm-start forms.

The limit K_ref of each cell comes from an FP64 solve at eps = 1e-10 (Eq. 11-12)
in voxel units (nu = h^2, lengths in voxels, so velocities are O(1) and the
relative part of the tolerance governs), started from the end state of the
FP32 run (the limit is the unique fixed point, whatever the start) and capped
in iterations; its own change over its last tenth is reported. With penalties
proportional to nu the ADMM iterates scale exactly as 1/nu, so K in the cell's
units is K_voxel * nu.
The timed runs are FP32 in the cell's units (nu = 1); the k = 0 coefficient of
every Green solve gives K after every iteration (the solve's history), the
crossing iteration n* is the first after which the Frobenius relative error
stays at or below the threshold, and the time is n* times the measured time
per iteration of that run (CUDA events).

Both runs use the approximate derivatives of Eq. 21 and fixed penalties from
the pore-scale rule (acm_stokes_params.pore_scale): the adaptive rule of Eq. 22
compares a velocity with a penalty times a velocity, so it is not unit-free, and
the exact symbols leave a slow tail (both are library defaults and are reported
separately by the bench).
"""
from __future__ import annotations

import numpy as np

THRESHOLDS = (1e-1, 1e-2, 1e-3, 1e-4)
PORE_SCALE = 9.0


def crossing(K_hist, K_ref, rel):
    """First iteration (1-based) after which |K_n - K_ref|_F / |K_ref|_F stays <= rel (None: never)."""
    err = np.linalg.norm(K_hist - K_ref, axis=(1, 2)) / np.linalg.norm(K_ref)
    bad = np.nonzero(err > rel)[0]
    if len(bad) == 0:
        return 1
    return int(bad[-1]) + 2 if bad[-1] + 1 < len(err) else None


def grid_nu(shape):
    """nu of voxel units: h^2 of the geometric-mean grid size over the axes longer than one."""
    ax = [s for s in shape if s > 1]
    n = float(np.prod(ax)) ** (1.0 / len(ax))
    return 1.0 / (n * n)


def plain_history(acm, ctx, Hd, stream, n_iter, pore_scale=PORE_SCALE):
    """The timed FP32 tensor solve of the plain form on ctx (cell units, n_iter
    iterations, eps = 0): K after every iteration and the seconds per iteration."""
    import torch
    u3 = torch.zeros((3, 3) + tuple(Hd.shape), dtype=torch.float32, device=Hd.device)
    prm = acm.stokes_params(eps=0.0, max_iter=n_iter, precision=acm.FP32, deriv=acm.DERIV_CENTRAL, adaptive=0,
                            pore_scale=pore_scale, check_every=500)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    acm.acm_stokes_tensor(ctx, Hd, prm, u3)
    e1.record(stream)
    torch.cuda.synchronize()
    per_iter = e0.elapsed_time(e1) / 1e3 / n_iter
    hs = [acm.acm_history(ctx, j) for j in range(3)]
    m = min(len(h) for h in hs)
    Kn = np.stack([np.stack([hs[j][:m, 15 + i] for j in range(3)], axis=-1) for i in range(3)], axis=1)
    return Kn, per_iter


def thresholds(Kn, K_ref, per_iter):
    out = {}
    for rel in THRESHOLDS:
        n_star = crossing(Kn, K_ref, rel)
        out[f"{rel:g}"] = ({"reached": True, "iterations": n_star, "seconds": n_star * per_iter}
                           if n_star is not None else {"reached": False})
    return out


def plain(acm, ctx, Hd, stream, n_iter, ref_eps=1e-10, ref_max_iter=2000, pore_scale=PORE_SCALE):
    """Time to permeability of one cell: the timed FP32 run, then the cell's FP64
    reference started from the end state of an identical FP32 run."""
    import torch
    Kn, per_iter = plain_history(acm, ctx, Hd, stream, n_iter, pore_scale)
    u_end = [torch.zeros((3, 3) + tuple(Hd.shape), dtype=torch.float32, device=Hd.device)]
    l_end = [torch.zeros_like(u_end[0])]
    batched_histories(acm, [Hd], n_iter, stream, pore_scale=pore_scale, u_out=u_end, lambda_out=l_end,
                      history=False)
    K_ref, ref = references(acm, [Hd], stream, u_end, l_end, ref_eps, ref_max_iter, pore_scale)
    return {"thresholds": thresholds(Kn, K_ref[0], per_iter), "seconds_per_iteration": per_iter,
            "iterations_run": len(Kn), "final_rel_err": float(np.linalg.norm(Kn[-1] - K_ref[0]) /
                                                               np.linalg.norm(K_ref[0])),
            "K_ref": K_ref[0].tolist(), "reference": ref}


def batched_histories(acm, Hd_list, n_iter, stream, nu=1.0, precision=None, eps=0.0, pore_scale=PORE_SCALE,
                      init=None, history=True, u_out=None, lambda_out=None):
    """One batched solve (cells of any shapes); returns (K [N, 3, 3] cell units,
    K histories [N][iters, 3, 3] cell units or None, reports, device seconds)."""
    import torch
    precision = acm.FP32 if precision is None else precision
    shapes = [tuple(h.shape) for h in Hd_list]
    batch = acm.acm_batch(shapes, stream.cuda_stream)
    if history:
        acm.acm_batch_history_enable(batch, n_iter)
    prm = acm.stokes_params(nu=nu, eps=eps, max_iter=n_iter, precision=precision, deriv=acm.DERIV_CENTRAL,
                            adaptive=0, pore_scale=pore_scale)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, K, reps = acm.acm_batch_stokes(batch, Hd_list, prm, u_out=u_out, init_u=None if init is None else init[0],
                                      init_lambda=None if init is None else init[1], lambda_out=lambda_out)
    e1.record(stream)
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    hist = None
    if history:
        hist = []
        for i in range(len(Hd_list)):
            hs = [acm.acm_batch_history(batch, i, j) for j in range(3)]
            m = min(len(h) for h in hs)
            hist.append(np.stack([hs[j][:m, 15:18] for j in range(3)], axis=-1) * nu)
    batch.close()
    return K * nu, hist, reps, secs


def references(acm, Hd_list, stream, u_end, lam_end, eps=1e-10, max_iter=2000, pore_scale=PORE_SCALE, chunk=48,
               nu_run=1.0):
    """Per-cell K_ref (cell units): FP64 batched solves in voxel units at eps,
    started from an FP32 end state (u_end, lam_end: per-cell [3][3][V] FP32 of
    a run with viscosity nu_run; u scales as 1 / nu, lambda does not), at most
    max_iter iterations. The residual stop of Eq. 11-12 at 1e-10 asks far more
    than K needs; the change of K over the run's last tenth (reported) bounds
    the reference's own error."""
    groups = {}
    for i, h in enumerate(Hd_list):
        groups.setdefault(tuple(h.shape), []).append(i)
    N = len(Hd_list)
    K_ref = np.zeros((N, 3, 3))
    iters = np.zeros((N, 3), np.int64)
    conv = np.zeros((N, 3), bool)
    drift = np.zeros(N)
    secs = 0.0
    for shape, idx in groups.items():
        nu = grid_nu(shape)
        for c0 in range(0, len(idx), chunk):
            sub = idx[c0:c0 + chunk]
            iu = [u_end[i].double() * (nu_run / nu) for i in sub]
            il = [lam_end[i].double() for i in sub]
            Kr, hist, reps, s = batched_histories(acm, [Hd_list[i] for i in sub], max_iter, stream, nu=nu,
                                                  precision=acm.FP64, eps=eps, pore_scale=pore_scale, init=(iu, il))
            secs += s
            for k, i in enumerate(sub):
                K_ref[i] = Kr[k]
                iters[i] = [r.iters for r in reps[k]]
                conv[i] = [bool(r.converged) for r in reps[k]]
                h = hist[k]
                drift[i] = float(np.linalg.norm(h[-1] - h[max(0, len(h) - 1 - len(h) // 10)]) / np.linalg.norm(h[-1]))
            del iu, il
    return K_ref, {"kind": f"FP64 at eps {eps:g} in voxel units (nu = h^2), started from the FP32 end state, "
                           f"at most {max_iter} iterations", "iters_max": int(iters.max()),
                   "residuals_converged_frac": float(conv.mean()), "K_change_last10pct_max": float(drift.max()),
                   "seconds": secs}


def batched(acm, Hd_list, n_iter, stream, ref_eps=1e-10, ref_max_iter=2000, pore_scale=PORE_SCALE, init=None):
    """Time to permeability of a batch of cells: one FP32 batched run (cell
    units) of n_iter iterations with every problem's K after every iteration,
    then per-cell FP64 references started from its end state. The batch
    reaches a threshold when its last cell does: n* = max over cells."""
    import torch
    u_end = [torch.zeros((3, 3) + tuple(h.shape), dtype=torch.float32, device=h.device) for h in Hd_list]
    l_end = [torch.zeros_like(x) for x in u_end]
    _, hist, _, secs = batched_histories(acm, Hd_list, n_iter, stream, pore_scale=pore_scale, init=init,
                                         u_out=u_end, lambda_out=l_end)
    per_iter = secs / n_iter
    K_ref, ref = references(acm, Hd_list, stream, u_end, l_end, ref_eps, ref_max_iter, pore_scale)
    del u_end, l_end
    out = {}
    n_star = {}
    for rel in THRESHOLDS:
        ns = [crossing(hist[i], K_ref[i], rel) for i in range(len(Hd_list))]
        n_star[f"{rel:g}"] = ns
        ok = [x for x in ns if x is not None]
        every = len(ok) == len(ns)
        out[f"{rel:g}"] = {"cells_reached": len(ok), "cells": len(ns),
                           "iterations_max": int(max(ok)) if every else None,
                           "iterations_median": float(np.median(ok)) if ok else None,
                           "seconds_all_cells": max(ok) * per_iter if every else None}
    final = [float(np.linalg.norm(hist[i][-1] - K_ref[i]) / np.linalg.norm(K_ref[i])) for i in range(len(hist))]
    return {"thresholds": out, "n_star": n_star, "K_ref": K_ref.tolist(), "reference": ref,
            "seconds_per_batch_iteration": per_iter, "iterations_run": n_iter,
            "final_rel_err_max": max(final), "final_rel_err_median": float(np.median(final))}

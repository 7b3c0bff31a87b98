"""Learned warm start for the Stokes ADMM: data generation, training, evaluation.

The network (a 3D Fourier neural operator, run by the library's own BF16/FP32
kernels through acm_fno_*) maps the indicator H of a cubic cell to the velocity
u and solid multiplier lambda of the unit load e_0. Its training data are
solutions of the ADMM of Section 3.1 itself (acm_batch_stokes), and the ADMM
always runs to the same tolerance afterwards: the warm start changes where the
iteration begins, never where it stops.

Pipeline
  1. cells: seeded sphere packs (porosity U[0.2, 0.6], radii U[3, 10] voxels).
  2. targets: batched FP32 solves of the three unit loads per cell to `tol`;
     every load becomes a sample for the load e_0 by swapping axes 0 and j of
     the cell and of the fields (the Stokes problem is invariant under that
     relabelling), so N cells give 3N samples.
  3. training: AdamW on the loss of the acm_fno header (velocity everywhere,
     multiplier on solid voxels), targets scaled to unit RMS per field; the
     scales are folded into the projection afterwards so the network emits
     physical values.
  4. evaluation on held-out seeds: iterations and seconds to `tol` for the
     three loads of every cell, batched, from zero and from the warm start,
     and the permeability of both.

Run as a module for the full workload (64^3 cells, width 32, 12 modes, 4
layers, 2000 training and 256 held-out cells); it prints one JSON line.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import math
import multiprocessing as mp
import os
import time

import numpy as np

from . import inputs as I

TRAIN_SEED0 = 100_000
TEST_SEED0 = 900_000


def _cell(args):
    n, seed = args
    por, radii = I.cell_recipe(seed)
    return I.sphere_pack((n, n, n), por, radii, seed)[0]


def make_cells(n, seeds, workers=None):
    """Indicators of the cells with these seeds, (len(seeds), n, n, n) uint8."""
    workers = workers or min(16, os.cpu_count() or 1)
    if len(seeds) < 8 or workers == 1:
        return np.stack([_cell((n, s)) for s in seeds])
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return np.stack(list(ex.map(_cell, [(n, s) for s in seeds], chunksize=4)))


def swap_sample(H, u, lam, j):
    """(H, u, lambda) of the load e_j as the load e_0 of the cell with axes 0 and
    j swapped (torch tensors: H (n, n, n), u and lambda (3, n, n, n))."""
    if j == 0:
        return H, u, lam
    perm = [0, 1, 2]
    perm[0], perm[j] = j, 0
    comp = list(perm)
    Hs = H.permute(*perm)
    us = u[comp].permute(0, *[p + 1 for p in perm])
    ls = lam[comp].permute(0, *[p + 1 for p in perm])
    return Hs.contiguous(), us.contiguous(), ls.contiguous()


def solve_cells(acm, Hd, tol, max_iter, chunk, stream, init=None, keep_fields=True, nu=1.0, history=False,
                prm_kw=None):
    """Batched FP32 solves of the three loads of every cell.

    Hd: device uint8 (N, n, n, n). init: optional (u0, lam0) device FP32
    (N, 3, 3, n, n, n). Returns dict with K (N, 3, 3), iters (N, 3), converged
    (N, 3), seconds (device time of the solves), when keep_fields the fields
    u, lam (N, 3, 3, n, n, n) on the device, and when history the volume
    average K_hist (N, iters, 3, 3) after every iteration."""
    import torch
    N, n = Hd.shape[0], Hd.shape[1]
    prm = acm.stokes_params(nu=nu, eps=tol, max_iter=max_iter, precision=acm.FP32, **(prm_kw or {}))
    K_hist = [] if history else None
    K = np.zeros((N, 3, 3))
    iters = np.zeros((N, 3), np.int64)
    conv = np.zeros((N, 3), bool)
    u_all = torch.zeros((N, 3, 3, n, n, n), dtype=torch.float32, device=Hd.device) if keep_fields else None
    l_all = torch.zeros_like(u_all) if keep_fields else None
    secs = 0.0
    batch = None
    for s0 in range(0, N, chunk):
        s1 = min(N, s0 + chunk)
        if batch is None or len(batch.shapes) != s1 - s0:
            if batch is not None:
                batch.close()
            batch = acm.acm_batch([(n, n, n)] * (s1 - s0), stream.cuda_stream)
            if history:
                acm.acm_batch_history_enable(batch, max_iter)
        Hs = [Hd[i] for i in range(s0, s1)]
        uo = [u_all[i] for i in range(s0, s1)] if keep_fields else None
        lo = [l_all[i] for i in range(s0, s1)] if keep_fields else None
        iu = [init[0][i] for i in range(s0, s1)] if init is not None else None
        il = [init[1][i] for i in range(s0, s1)] if init is not None else None
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, Kc, reps = acm.acm_batch_stokes(batch, Hs, prm, u_out=uo, init_u=iu, init_lambda=il, lambda_out=lo)
        e1.record(stream)
        torch.cuda.synchronize()
        secs += e0.elapsed_time(e1) / 1e3
        K[s0:s1] = Kc
        for i, r in enumerate(reps):
            iters[s0 + i] = [x.iters for x in r]
            conv[s0 + i] = [bool(x.converged) for x in r]
            if history:
                hs = [acm.acm_batch_history(batch, i, j) for j in range(3)]
                m = min(len(h) for h in hs)
                K_hist.append(np.stack([hs[j][:m, 15:18] for j in range(3)], axis=-1) * nu)
    if batch is not None:
        batch.close()
    return {"K": K * nu, "iters": iters, "converged": conv, "seconds": secs, "u": u_all, "lam": l_all,
            "K_hist": K_hist}


def iterations_to(K_hist, K_ref, rel):
    """First iteration after which the Frobenius relative error of K stays at or
    below `rel` (None if it never does)."""
    err = np.linalg.norm(K_hist - K_ref, axis=(1, 2)) / np.linalg.norm(K_ref)
    bad = np.nonzero(err > rel)[0]
    if len(bad) == 0:
        return 1
    return int(bad[-1]) + 2 if bad[-1] + 1 < len(err) else None


def build_dataset(Hd, u, lam):
    """Samples for the load e_0: (H (3N, n, n, n) uint8, targets (3N, 6, n, n, n))."""
    import torch
    N, n = Hd.shape[0], Hd.shape[1]
    Hs = torch.empty((3 * N, n, n, n), dtype=Hd.dtype, device=Hd.device)
    Ts = torch.empty((3 * N, 6, n, n, n), dtype=u.dtype, device=u.device)
    for i in range(N):
        for j in range(3):
            h, uu, ll = swap_sample(Hd[i], u[i, j], lam[i, j], j)
            Hs[3 * i + j] = h
            Ts[3 * i + j, :3] = uu
            Ts[3 * i + j, 3:] = ll
    return Hs, Ts


def target_scales(H, T):
    """RMS of the velocity over all voxels and of the multiplier over solid voxels."""
    su = float(T[:, :3].double().pow(2).mean().sqrt())
    m = H.unsqueeze(1).double()
    sl = float(((T[:, 3:].double() * m).pow(2).sum() / (3 * m.sum())).sqrt())
    return su, sl


def fold_scales(theta, width, su, sl):
    """Parameters emitting physical values from a network trained on scaled targets
    (Q [6][W] and q [6] are the last 6 W + 6 entries)."""
    th = theta.copy()
    s = np.array([su] * 3 + [sl] * 3, np.float32)
    Q = th[-(6 * width + 6):-6].reshape(6, width)
    Q *= s[:, None]
    th[-6:] *= s
    return th


def init_theta(width, modes, layers, seed):
    """Seeded initial parameters in the layout of acm_fno (standard FNO scaling:
    spectral weights uniform in [0, 1/W^2), dense weights uniform in +-1/sqrt(fan_in))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nm = 4 * modes ** 3
    parts = [rng.uniform(-1, 1, (width, 4)) / 2.0, np.zeros(width)]
    for _ in range(layers):
        parts += [rng.random((nm, width, width, 2)) / (width * width),
                  rng.uniform(-1, 1, (width, width)) / math.sqrt(width), np.zeros(width)]
    parts += [rng.uniform(-1, 1, (6, width)) / math.sqrt(width), np.zeros(6)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def train(acm, fno, H, T, epochs, batch, lr, weight_decay, seed, stream, log=None):
    """AdamW with a cosine learning-rate schedule; returns per-epoch mean losses
    and the seconds spent (device time of forward, backward and update)."""
    import torch
    N = H.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    steps = epochs * (N // batch)
    k = 0
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = rng.permutation(N)
        tot = 0.0
        for b0 in range(0, N - batch + 1, batch):
            idx = torch.as_tensor(order[b0:b0 + batch], device=H.device)
            Hb, Tb = H.index_select(0, idx).contiguous(), T.index_select(0, idx).contiguous()
            tot += fno.backward(Hb, Tb)
            lr_k = lr * 0.5 * (1.0 + math.cos(math.pi * k / max(1, steps)))
            fno.adamw(max(lr_k, 1e-3 * lr), weight_decay=weight_decay)
            k += 1
        losses.append(tot / (N // batch))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4e}")
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0


def warm_starts(fno, Hd, batch):
    """(init_u, init_lambda) (N, 3, 3, n, n, n) FP32 for every cell, and seconds."""
    import torch
    N, n = Hd.shape[0], Hd.shape[1]
    iu = torch.zeros((N, 3, 3, n, n, n), dtype=torch.float32, device=Hd.device)
    il = torch.zeros_like(iu)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s0 in range(0, N, batch):
        s1 = min(N, s0 + batch)
        fno.warm_start(Hd[s0:s1], iu[s0:s1], il[s0:s1])
    torch.cuda.synchronize()
    return iu, il, time.perf_counter() - t0


def field_error(pred, ref, H):
    """Relative L2 error of the predicted velocity (all voxels) over all samples."""
    du = (pred - ref).double().pow(2).sum()
    return float((du / ref.double().pow(2).sum()).sqrt())


def run(n=64, width=32, modes=12, layers=4, n_train=2000, n_test=256, tol=1e-6, max_iter=20000,
        epochs=12, batch=4, lr=2e-3, weight_decay=1e-4, chunk=128, seed=0, nu=1.0, n_curve=32,
        curve_iters=20000, log=print, central=False):
    """The whole pipeline; returns a dict of results (see the module docstring).

    nu = 1 on the unit cell are the units of the paper; the absolute part of
    the tolerance of Eq. 11-12 then sets how accurate K is at the stop, so the
    evaluation also follows K after every iteration of both starts on n_curve
    held-out cells (eps = 0, curve_iters iterations). With central = False the
    library defaults are used (exact symbols, Eq. 22) and K is compared with the
    last K of the zero start; with central = True every solve takes the
    symbols of Eq. 21 and fixed pore-scale penalties, and each curve cell's
    limit comes from an FP64 solve at eps = 1e-10 (time to permeability,
    ttk.references)."""
    import torch

    from . import acm
    from . import ttk
    acm.load()
    kw = dict(deriv=acm.DERIV_CENTRAL, adaptive=0, pore_scale=ttk.PORE_SCALE) if central else {}
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    res = {"grid": n, "width": width, "modes": modes, "layers": layers, "n_train_cells": n_train,
           "n_test_cells": n_test, "tol": tol, "nu": nu,
           "solver": "Eq. 21 symbols, fixed pore-scale penalties" if central else "library defaults"}
    t = time.perf_counter()
    Htr = make_cells(n, range(TRAIN_SEED0 + seed * 10_000, TRAIN_SEED0 + seed * 10_000 + n_train))
    Hte = make_cells(n, range(TEST_SEED0 + seed * 10_000, TEST_SEED0 + seed * 10_000 + n_test))
    res["cells_seconds"] = time.perf_counter() - t
    Htr_d, Hte_d = torch.as_tensor(Htr, device=dev), torch.as_tensor(Hte, device=dev)
    # 2. training targets from the method itself
    sol = solve_cells(acm, Htr_d, tol, max_iter, chunk, stream, nu=nu, prm_kw=kw)
    res["train_solve_seconds"] = sol["seconds"]
    res["train_iters_mean"] = float(sol["iters"].mean())
    res["train_converged_frac"] = float(sol["converged"].mean())
    log(f"targets: {sol['seconds']:.1f} s, mean iterations {sol['iters'].mean():.0f}")
    H, T = build_dataset(Htr_d, sol["u"], sol["lam"])
    del sol
    torch.cuda.empty_cache()
    su, sl = target_scales(H, T)
    T[:, :3] /= su
    T[:, 3:] /= sl
    res["target_rms"] = {"u": su, "lambda": sl}
    # 3. training on the device with the library's kernels
    fno = acm.acm_fno((n, n, n), width, modes, layers, max_batch=max(batch, 8), stream=stream.cuda_stream)
    fno.set_params(init_theta(width, modes, layers, seed))
    losses, secs = train(acm, fno, H, T, epochs, batch, lr, weight_decay, seed, stream, log)
    res.update({"n_params": fno.num_params, "train_samples": int(H.shape[0]), "epochs": epochs, "batch": batch,
                "lr": lr, "losses": losses, "train_seconds": secs})
    del H, T
    theta = fold_scales(fno.get_params(), width, su, sl)
    fno.set_params(theta)
    # 4. held-out cells: zero start against the learned start, same tolerance
    plain = solve_cells(acm, Hte_d, tol, max_iter, chunk, stream, nu=nu, prm_kw=kw)
    iu, il, inf_s = warm_starts(fno, Hte_d, 8)
    warm = solve_cells(acm, Hte_d, tol, max_iter, chunk, stream, init=(iu, il), keep_fields=False, nu=nu,
                       prm_kw=kw)
    fe = field_error(iu, plain["u"], Hte_d)
    dK = np.linalg.norm(warm["K"] - plain["K"], axis=(1, 2)) / np.linalg.norm(plain["K"], axis=(1, 2))
    res.update({
        "plain": {"iters_mean": float(plain["iters"].mean()), "seconds": plain["seconds"],
                  "converged_frac": float(plain["converged"].mean())},
        "warm": {"iters_mean": float(warm["iters"].mean()), "seconds": warm["seconds"],
                 "inference_seconds": inf_s, "converged_frac": float(warm["converged"].mean())},
        "iterations_saved_frac": float(1 - warm["iters"].sum() / plain["iters"].sum()),
        "time_saved_frac": float(1 - (warm["seconds"] + inf_s) / plain["seconds"]),
        "per_cell_iters_plain": plain["iters"].sum(axis=1).tolist(),
        "per_cell_iters_warm": warm["iters"].sum(axis=1).tolist(),
        "warm_start_velocity_rel_err": fe,
        "K_rel_diff_warm_vs_plain_max": float(dK.max()),
        "K_rel_diff_warm_vs_plain_median": float(np.median(dK)),
    })
    del plain, warm
    # 5. K after every iteration on a subset (eps = 0: both run curve_iters iterations)
    if n_curve > 0:
        m = min(n_curve, n_test)
        sub = Hte_d[:m]
        pc = solve_cells(acm, sub, 0.0, curve_iters, chunk, stream, keep_fields=central, nu=nu, history=True,
                         prm_kw=kw)
        wc = solve_cells(acm, sub, 0.0, curve_iters, chunk, stream, init=(iu[:m], il[:m]), keep_fields=False,
                         nu=nu, history=True, prm_kw=kw)
        per_iter = pc["seconds"] / curve_iters
        if central:
            K_refs, ref = ttk.references(acm, [sub[c] for c in range(m)], stream, [pc["u"][c] for c in range(m)],
                                         [pc["lam"][c] for c in range(m)], nu_run=nu)
            K_refs = K_refs / nu   # the curves are in the run's units
            res["K_reference"] = {"kind": "FP64, eps 1e-10, voxel units, from the zero start's end state", **ref}
        else:
            K_refs = [pc["K_hist"][c][-1] for c in range(m)]
        curves = {}
        for rel in (1e-1, 3e-2, 1e-2, 3e-3, 1e-3, 1e-4):
            a = [iterations_to(pc["K_hist"][c], K_refs[c], rel) for c in range(m)]
            b = [iterations_to(wc["K_hist"][c], K_refs[c], rel) for c in range(m)]
            ok = [x is not None and y is not None for x, y in zip(a, b)]
            curves[f"{rel:g}"] = {
                "cells_reached_both": int(sum(ok)),
                "plain_iters_median": float(np.median([x for x, k in zip(a, ok) if k])) if any(ok) else None,
                "warm_iters_median": float(np.median([y for y, k in zip(b, ok) if k])) if any(ok) else None,
                "plain_iters_max": int(max(x for x, k in zip(a, ok) if k)) if all(ok) else None,
                "warm_iters_max": int(max(y for y, k in zip(b, ok) if k)) if all(ok) else None,
                "plain_seconds_all_cells": max(a) * per_iter if all(ok) else None,
                "warm_seconds_all_cells": (max(b) * per_iter + inf_s * m / n_test) if all(ok) else None,
            }
        tail = [float(np.linalg.norm(h[-1] - h[-max(2, curve_iters // 10)]) / np.linalg.norm(h[-1]))
                for h in pc["K_hist"]]
        res["K_curves"] = {"cells": m, "iterations": curve_iters, "seconds_per_iteration_batch": per_iter,
                           "reference": ("FP64 solve at eps 1e-10" if central else "last K of the zero start"),
                           "reference_last10pct_change_median":
                           float(np.median(tail)), "iterations_to_rel_err": curves}
    fno.close()
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--width", type=int, default=32)
    ap.add_argument("--modes", type=int, default=12)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=256)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--chunk", type=int, default=128)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--nu", type=float, default=1.0)
    ap.add_argument("--curve-cells", type=int, default=32)
    ap.add_argument("--curve-iters", type=int, default=20000)
    ap.add_argument("--central", action="store_true",
                    help="Eq. 21 symbols and fixed pore-scale penalties, FP64 references for the K curves")
    a = ap.parse_args()
    from . import build as B
    B.build()
    r = run(a.n, a.width, a.modes, a.layers, a.train, a.test, a.tol, a.max_iter, a.epochs, a.batch, a.lr,
            chunk=a.chunk, seed=a.seed, nu=a.nu, n_curve=a.curve_cells, curve_iters=a.curve_iters,
            log=lambda m: print(m, flush=True), central=a.central)
    print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()

"""Throughput of the ACM hot path on one or more GPUs (one process per GPU).

Workload: a 256^3 periodic cell of seeded Boolean (overlapping) spheres of
radius 8 voxels at porosity 0.35. One step is
  * Stokes (ADMM, adaptive penalties, FP32 fields, FP64 reductions): the three
    unit loads solved together, ITERS iterations each, with residuals and stop
    test every iteration and the permeability tensor at the end;
  * solute (Lippmann-Schwinger, FP32): for Pe = 1, 10, 100 the three composition
    loads advected by the e_0 flow, ITERS iterations each, with the effective
    diffusivity tensor at the end.
The metric is voxel-iterations per second: V * (3 + 9) * ITERS per step.

Output: one JSON line on rank 0. `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

from paper_2312_15554_gb300 import shard as SH

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 256
POROSITY = 0.35
RADIUS = 8.0
PECLETS = (1.0, 10.0, 100.0)
METRIC = "ACM voxel-iterations/s and time-to-permeability (rel err 1e-4) vs HBM roofline"
UNIT = "voxel-iterations/s"
WORKLOAD = (f"{N}^3 Boolean sphere pack (radius {RADIUS:g} vox, porosity {POROSITY}); Stokes 3 loads + "
            f"solute Pe 1/10/100 x 3 loads")


def algorithmic_bytes_per_voxel(kind: str, n2: int, porosity: float, share: int = 3) -> float:
    """Bytes a kernel of the given kind must move per voxel and per problem (FP32).

    cspec: one complex FP32 component of the half spectrum (n2/2 + 1 of n2 columns).
    Multiplier lambda lives on solid voxels only, the solute velocity on pore voxels
    only. share: problems of one launch that read the same indicator (the loads of
    one cell) and, in the solute pass, the same velocity (the composition loads of
    one flow field); data they share is counted once per launch. The indicator is
    read as bits (1/8 byte per voxel).
    """
    cspec = 8.0 * (n2 // 2 + 1) / n2
    solid = 1.0 - porosity
    hbits = 1.0 / 8.0
    return {
        "x_stokes_local": 3 * cspec + 24.0 + 24.0 * solid + hbits / share,
        "x_stokes_rhs": 12.0 + 12.0 * solid + hbits / share + 3 * cspec,
        "y_fwd_stokes": 6 * cspec,
        "z_stokes": 10 * cspec,
        "y_inv_stokes": 6 * cspec,
        # solute passes carry (tau_0, tau_1, s') -> (tau_0, s'') -> (d0 chi, chi) -> (d0 chi, d1 chi, d2 chi)
        "x_solute": 3 * cspec + (12.0 * porosity + hbits) / share + 3 * cspec,
        "y_fwd_solute": 5 * cspec,
        "z_solute": 6 * cspec,
        "y_inv_solute": 5 * cspec,
    }.get(kind, 0.0)


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel at the default workload (256^3, porosity 0.35, 3 problems per launch),
# from one ncu capture of that kernel (mean over its captured launches). An
# entry holds only while the kernel is unchanged since that capture.
MEASURED_TRAFFIC = {"x_solute": 836.852e6 + 569.529e6, "x_stokes_local": 2403.660e6 + 1052.283e6}


def step_roofline(kern: dict, peak: float) -> dict:
    """Algorithmic bandwidth of the whole step: the algorithmic bytes of every
    kernel kind that has a byte count, summed, over their summed CUDA-event time
    (the time-weighted mean over the pass kernels), against the peak; time_share
    is the part of all timed kernel time those kinds cover."""
    tot_b = tot_s = all_s = 0.0
    for v in kern.values():
        s = v["ms"] / 1e3
        all_s += s
        if v.get("GBps"):
            tot_b += v["GBps"] * 1e9 * s
            tot_s += s
    if tot_s <= 0:
        return None
    achieved = tot_b / tot_s / 1e9
    return {"achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "time_share": round(tot_s / all_s, 4), "basis": "algorithmic bytes, time-weighted over the pass kernels"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs(rank: int):
    from paper_2312_15554_gb300 import inputs as I
    H = I.sphere_pack((N, N, N), POROSITY, RADIUS, 2024 + rank)[0]
    return H


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_threads() -> int:
    """Host threads the oracle's transforms run on (its pointwise numpy work is single-threaded)."""
    from oracle import fft as FFT
    return FFT.threads()


def oracle_sample(H, iters: int = 1):
    """Oracle Stokes + solute iterations on one load each; returns (voxel-iterations, seconds)."""
    from oracle import acm_oracle as O
    V = H.size
    t0 = time.perf_counter()
    R = O.stokes(H, [1.0, 0.0, 0.0], O.StokesParams(eps=0.0, max_iter=iters))
    O.advdiff(H, R.state.u, 10.0, [1.0, 0.0, 0.0], O.AdvDiffParams(eps=0.0, max_iter=iters))
    dt = time.perf_counter() - t0
    return 2 * V * iters, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    H = make_inputs(0)
    for _ in range(args.warmup):
        oracle_sample(H)
    vi, secs = 0, 0.0
    for _ in range(args.steps):
        a, b = oracle_sample(H)
        vi += a
        secs += b
    value = vi / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "sample": "1 Stokes + 1 solute iteration (1 load each) per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                         "sample": "per step: 1 ADMM iteration (load e_0) + 1 Lippmann-Schwinger iteration "
                                   "(Pe 10, g_chi e_0) at 256^3, FP64 oracle (own radix-2 FFT in C over "
                                   "the host threads, pointwise steps in numpy)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def time_to_permeability(acm, ctx, Hd, stream, n_long, deriv=None, fixed_penalty=None):
    """Seconds until the permeability tensor stays within a relative error
    (Frobenius) of the tensor after n_long iterations, for the plain solve,
    at 1e-1 ... 1e-4. deriv selects the derivative symbols of the Stokes solve
    (None: the library default, the exact symbols of Eq. 13; DERIV_CENTRAL: the
    approximate derivatives of Eq. 21). fixed_penalty = f runs with alpha = beta
    = b = f times the default initial penalty and no Eq. 22 adaptation; None keeps
    the library defaults (adaptive).

    The k = 0 Fourier coefficient of each Green solve gives the volume average of
    u for every iteration (history), so the crossing iteration n* is found from one
    long run; the seconds are n* times the per-iteration time of that run (CUDA
    events). A threshold below the change of the reference over its last tenth
    cannot be resolved by the reference and is reported as not reached.
    """
    import torch
    u3 = torch.zeros((3, 3) + tuple(Hd.shape), dtype=torch.float32, device=Hd.device)
    kw = {} if deriv is None else {"deriv": deriv}
    if fixed_penalty is not None:
        n = float(np.prod(Hd.shape)) ** (1.0 / 3.0)
        psi = fixed_penalty * (math.pi * n) ** 2 / 8.0   # nu = 1
        kw.update(adaptive=0, alpha0=psi, beta0=psi, b0=psi)
    prm = acm.stokes_params(eps=0.0, max_iter=n_long, precision=acm.FP32, check_every=500, **kw)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    acm.acm_stokes_tensor(ctx, Hd, prm, u3)
    e1.record(stream)
    torch.cuda.synchronize()
    per_iter = e0.elapsed_time(e1) / 1e3 / n_long
    hs = [acm.acm_history(ctx, j) for j in range(3)]
    m = min(len(h) for h in hs)
    Kn = np.stack([np.stack([hs[j][:m, 15 + i] for j in range(3)], axis=-1) for i in range(3)], axis=1)
    Kref = Kn[-1]
    err = np.linalg.norm(Kn - Kref, axis=(1, 2)) / np.linalg.norm(Kref)
    tail = float(np.linalg.norm(Kn[-1] - Kn[max(0, m - 1 - m // 10)]) / np.linalg.norm(Kref))
    out = {}
    for rel in (1e-1, 1e-2, 1e-3, 1e-4):
        bad = np.nonzero(err > rel)[0]
        n_star = int(bad[-1]) + 2 if len(bad) else 1
        if rel <= tail or n_star > m:
            out[f"{rel:g}"] = {"reached": False}
        else:
            out[f"{rel:g}"] = {"reached": True, "iterations": n_star, "seconds": n_star * per_iter}
    return {"thresholds": out, "reference_iterations": n_long, "reference_last10pct_change": tail,
            "seconds_per_iteration": per_iter, "K_ref": Kref.tolist(),
            "form": "plain (FP32, unit cell, nu = 1), "
                    + ("adaptive penalties of Eq. 22 (library defaults), " if fixed_penalty is None
                       else f"fixed penalties {fixed_penalty:g} x the default initial penalty, ")
                    + ("exact derivative symbols (Eq. 13)" if deriv is None or deriv == acm.DERIV_EXACT
                       else "approximate derivative symbols (Eq. 21)")}


def run_gpu(args, rank, world, dist):
    import torch

    from paper_2312_15554_gb300 import acm
    from paper_2312_15554_gb300 import build as B

    B.build()
    acm.load()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    H = make_inputs(rank)
    porosity = 1.0 - float(H.mean())
    V = H.size
    iters = args.iters
    stream = torch.cuda.current_stream(dev)
    ctx = acm.acm_ctx(H.shape, stream.cuda_stream)
    Hd = torch.as_tensor(H, device=dev)
    H_pin = torch.as_tensor(H).pin_memory()
    u3 = torch.zeros((3, 3) + H.shape, dtype=torch.float32, device=dev)
    sp = acm.stokes_params(eps=0.0, max_iter=iters, precision=acm.FP32)
    cp = acm.advdiff_params(eps=0.0, max_iter=iters, precision=acm.FP32)
    # tile widths of the strided passes, tuned once per shape (outside the timed region)
    torch.cuda.synchronize()
    t_tune = time.perf_counter()
    tiles = acm.acm_autotune(ctx, False)
    tune_s = time.perf_counter() - t_tune

    def step(Hin):
        s, K, _, _ = acm.acm_stokes_tensor(ctx, Hin, sp, u3)
        Ds = []
        for Pe in PECLETS:
            s2, D, _, _ = acm.acm_advdiff_tensor(ctx, Hin, u3[0], Pe, cp)
            Ds.append(D)
        return K, Ds

    vi_per_step = V * iters * (3 + 3 * len(PECLETS))

    for _ in range(args.warmup):
        step(Hd)
    torch.cuda.synchronize()
    acm.acm_profile_read(ctx)                      # reset counters
    acm.acm_profile_enable(ctx, True)
    sampler = ClockSampler(local) if rank == 0 else None
    SH.barrier(dist)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        K, Ds = step(Hd)
    e1.record(stream)
    torch.cuda.synchronize()
    SH.barrier(dist)
    clocks = sampler.stop() if sampler else None
    prof = acm.acm_profile_read(ctx)
    acm.acm_profile_enable(ctx, False)
    ms = SH.max_over_ranks(e0.elapsed_time(e1), dist, dev)
    value = vi_per_step * args.steps * world / (ms / 1e3)

    # end to end through the public API with host buffers: H from pinned host
    # memory every call, K and D read back to the host
    torch.cuda.synchronize()
    SH.barrier(dist)
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps // 2)):
        K, Ds = step(H_pin.numpy())
    torch.cuda.synchronize()
    e2e_s = SH.max_over_ranks((time.perf_counter() - t0) / max(1, args.steps // 2), dist, dev)
    e2e_value = vi_per_step * world / e2e_s

    # roofline of the dominant kernel (largest device time in the timed region)
    kinds = {k: v for k, v in prof.items() if k not in ("other", "finalize") and v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms, dom_n = kinds[dom]
    nprob = 3
    bytes_per_launch = algorithmic_bytes_per_voxel(dom, N, porosity) * V * nprob
    achieved = bytes_per_launch / (dom_ms / dom_n / 1e3) / 1e9
    peak, peak_src = measured_peaks()
    launches = int(sum(v[1] for v in prof.values()))
    kern = {k: {"ms": round(v[0], 3), "launches": v[1],
                "GBps": (round(algorithmic_bytes_per_voxel(k, N, porosity) * V * nprob / (v[0] / v[1] / 1e3) / 1e9, 1)
                         if v[1] and algorithmic_bytes_per_voxel(k, N, porosity) else None)}
            for k, v in prof.items() if v[1]}

    # time to permeability on one GPU only (several ranks would each hold a GPU for it)
    ttk = (time_to_permeability(acm, ctx, Hd, stream, args.ttk_long)
           if (args.ttk and args.ttk_default_form and world == 1) else None)
    ttk_c = ttk_b = None
    if args.ttk and world == 1 and args.ttk_iters > 0:
        from paper_2312_15554_gb300 import ttk as TTK
        ttk_c = TTK.plain(acm, ctx, Hd, stream, args.ttk_iters, ref_max_iter=args.ttk_ref_iters)
        ttk_c["form"] = ("plain (FP32, unit cell, nu = 1), approximate derivative symbols (Eq. 21), fixed "
                         f"penalties {TTK.PORE_SCALE:g} / l^2 x the default (pore length l)")
        if args.ttk_cells > 0:
            # a reduced batched figure: cells of the batched workload's recipe
            Hb = [torch.as_tensor(_batched_cell(i), device=dev) for i in range(args.ttk_cells)]
            r = TTK.batched(acm, Hb, args.ttk_iters, stream, ref_max_iter=args.ttk_ref_iters)
            r.pop("n_star")
            r.pop("K_ref")
            ttk_b = {"form": f"batched, {args.ttk_cells} cells of the batched recipe (half 64^3, half 128^3), "
                             "FP32, Eq. 21 symbols, pore-scale fixed penalties per cell", **r}
            del Hb

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        vi_c, s_c = oracle_sample(H, 1)
        cpu = {"value": vi_c / s_c, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
               "sample": "1 ADMM iteration (load e_0) + 1 Lippmann-Schwinger iteration (Pe 10) at 256^3, "
                         f"FP64 oracle (own radix-2 FFT in C over the host threads, pointwise steps in numpy), "
                         f"{s_c:.1f} s"}
    ctx.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "porosity": round(porosity, 4), "iters_per_step": iters,
                   "problems_per_step": 3 + 3 * len(PECLETS), "l2": "inputs larger than L2 (3.3 GB working set)",
                   "parallelism": f"independent cells x{world}", "tiles": tiles,
                   "autotune_s": round(tune_s, 3)},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": MEASURED_TRAFFIC.get(dom) if (N == 256 and abs(POROSITY - 0.35) < 1e-9) else None,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch"
                                       if dom in MEASURED_TRAFFIC else None,
                     "peak_source": peak_src, "bytes_per_launch": bytes_per_launch},
        "roofline_step": step_roofline(kern, peak),
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(4 * V),
                "d2h_bytes_per_step": int(8 * 9 * (1 + len(PECLETS)))},
        "gpu_launches": launches,
        "clocks": clocks,
        "kernels": kern,
        "K_diag": [float(K[i, i]) for i in range(3)],
    }
    if ttk is not None:
        line["time_to_permeability"] = ttk
    if ttk_c is not None:
        line["time_to_permeability_fp64_reference"] = ttk_c
    if ttk_b is not None:
        line["time_to_permeability_batched_fp64_reference"] = ttk_b
    print(json.dumps(line), flush=True)


def _batched_cell(i):
    """Cell i of the batched workload: 64^3 for even i, 128^3 for odd i."""
    from paper_2312_15554_gb300 import inputs as I
    n = 64 if i % 2 == 0 else 128
    por, radii = I.cell_recipe(5000 + i)
    return I.sphere_pack((n, n, n), por, radii, 5000 + i)[0]


def run_batched(args, rank, world, dist):
    """Many cells in one device-resident solve (Stokes, three loads per cell)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    idx = list(SH.shard(args.cells * world, rank, world))   # the same number of cells per rank (weak scaling)
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                                mp_context=mp.get_context("spawn")) as ex:
        Hs = list(ex.map(_batched_cell, idx, chunksize=4))
    import torch

    from paper_2312_15554_gb300 import acm
    from paper_2312_15554_gb300 import build as B
    B.build()
    acm.load()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    shapes = [h.shape for h in Hs]
    Hd = [torch.as_tensor(h, device=dev) for h in Hs]
    batch = acm.acm_batch(shapes, stream.cuda_stream)
    prm = acm.stokes_params(eps=0.0, max_iter=args.iters, precision=acm.FP32)
    torch.cuda.synchronize()
    t_tune = time.perf_counter()
    acm.acm_batch_autotune(batch)
    tune_s = time.perf_counter() - t_tune
    tiles = {f"{shapes[i][0]}^3": acm.acm_batch_tiles(batch, i) for i in range(min(2, len(shapes)))}
    vi = sum(int(np.prod(sh)) for sh in shapes) * 3 * args.iters
    for _ in range(args.warmup):
        acm.acm_batch_stokes(batch, Hd, prm)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    sampler = ClockSampler(local) if rank == 0 else None
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s, K, reps = acm.acm_batch_stokes(batch, Hd, prm)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    ttk = None
    if args.ttk_batched > 0 and world == 1:
        # time to permeability of the batched form (Eq. 21 symbols, pore-scale
        # fixed penalties): every problem's K after every iteration of one
        # batched FP32 run, each cell against its FP64 limit at eps 1e-10
        from paper_2312_15554_gb300 import ttk as TTK
        r = TTK.batched(acm, Hd, args.ttk_batched, stream, ref_max_iter=args.ttk_ref_iters)
        r.pop("n_star")
        r.pop("K_ref")
        ttk = {"form": "batched (FP32, nu = 1), approximate derivative symbols (Eq. 21), fixed penalties "
                       f"{TTK.PORE_SCALE:g} / l^2 x the default per cell", **r}
    # per-kernel shares of one more step, host-launched with CUDA events
    acm.acm_batch_profile_read(batch)
    acm.acm_batch_profile_enable(batch, True)
    acm.acm_batch_stokes(batch, Hd, prm)
    prof = acm.acm_batch_profile_read(batch)
    acm.acm_batch_profile_enable(batch, False)
    batch.close()
    ms = SH.max_over_ranks(ms, dist, dev)
    K_all = SH.gather_rows(K, args.cells * world, dist, dev, world)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": vi * args.steps * world / (ms / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched: {len(shapes)} cells (half 64^3, half 128^3), 3 loads each, "
                               "porosity U[0.2,0.6], radii U[3,10] vox", "iters_per_step": args.iters,
                   "device_loop": "CUDA graph while node", "tiles": tiles, "autotune_s": round(tune_s, 3)},
        "clocks": clocks,
        "kernels_profiled_step": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in prof.items() if v[1]},
        "K_mean_diag_cell0": [float(K_all[0, i, i]) for i in range(3)],
        "cells_all_ranks": int(K_all.shape[0]),
    }
    if ttk is not None:
        line["time_to_permeability"] = ttk
    print(json.dumps(line), flush=True)


def run_grf512(args, rank, world, dist):
    """512^3 thresholded Gaussian random field (correlation length 16 voxels, porosity
    0.3): Stokes for the load e_x, then advection-diffusion at Pe 10 (3 loads).

    value: voxel-iterations/s of the FP32 path (20 Stokes + 3 x 20 solute iterations
    per step, FP64 residuals). Accuracy: the same problems solved to eps with FP32
    iterations and a final FP64 refinement (ACM_FP32_THEN_FP64), against FP64
    iterations throughout; the differences of K_xx, of u and of D are reported.
    """
    import torch

    from paper_2312_15554_gb300 import acm
    from paper_2312_15554_gb300 import build as B
    from paper_2312_15554_gb300 import inputs as I
    n = 512
    H = I.grf_medium((n, n, n), 16.0, 0.3, 2024 + rank)
    B.build()
    acm.load()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    V = H.size
    porosity = 1.0 - float(H.mean())
    ctx = acm.acm_ctx(H.shape, stream.cuda_stream)
    Hd = torch.as_tensor(H, device=dev)
    tiles = acm.acm_autotune(ctx, False)
    acm.acm_autotune(ctx, True)
    iters = args.iters
    u = torch.zeros((3,) + H.shape, dtype=torch.float32, device=dev)
    sp = acm.stokes_params(eps=0.0, max_iter=iters, precision=acm.FP32)
    cp = acm.advdiff_params(eps=0.0, max_iter=iters, precision=acm.FP32)

    def step():
        acm.acm_stokes(ctx, Hd, [1.0, 0.0, 0.0], sp, u=u)
        acm.acm_advdiff_tensor(ctx, Hd, u, 10.0, cp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    acm.acm_profile_read(ctx)
    acm.acm_profile_enable(ctx, True)
    sampler = ClockSampler(local) if rank == 0 else None
    SH.barrier(dist)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    prof = acm.acm_profile_read(ctx)
    acm.acm_profile_enable(ctx, False)
    ms = SH.max_over_ranks(e0.elapsed_time(e1), dist, dev)
    vi_step = V * iters * 4
    value = vi_step * args.steps * world / (ms / 1e3)
    kinds = {k: v for k, v in prof.items() if k not in ("other", "finalize") and v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    per_problem = {"x_stokes_local": 3, "x_stokes_rhs": 3, "y_fwd_stokes": 3, "z_stokes": 3, "y_inv_stokes": 3}
    nprob_of = lambda k: 1 if k in per_problem else 3
    kern = {k: {"ms": round(v[0], 3), "launches": v[1],
                "GBps": (round(algorithmic_bytes_per_voxel(k, n, porosity, nprob_of(k)) * V * nprob_of(k) * v[1]
                               / (v[0] / 1e3) / 1e9, 1) if v[1] and algorithmic_bytes_per_voxel(k, n, porosity) else None)}
            for k, v in prof.items() if v[1]}
    peak, peak_src = measured_peaks()
    achieved = kern[dom]["GBps"]
    # accuracy: FP32 iterations + FP64 refinement against FP64 throughout
    eps, eps32, nu = args.c5_eps, args.c5_eps32, args.c5_nu
    uA = torch.zeros((3,) + H.shape, dtype=torch.float64, device=dev)
    uB = torch.zeros_like(uA)
    pA = acm.stokes_params(nu=nu, eps=eps, eps32=eps32, max_iter=args.c5_max_iter, precision=acm.FP32_THEN_FP64)
    pB = acm.stokes_params(nu=nu, eps=eps, max_iter=args.c5_max_iter, precision=acm.FP64)
    sA, KA, rA = acm.acm_stokes(ctx, Hd, [1.0, 0.0, 0.0], pA, u=uA)
    sB, KB, rB = acm.acm_stokes(ctx, Hd, [1.0, 0.0, 0.0], pB, u=uB)
    du = float((uA - uB).norm() / uB.norm())
    qA = acm.advdiff_params(eps=eps, max_iter=args.c5_max_iter, precision=acm.FP32_THEN_FP64)  # FP32 stage to 1e-5
    qB = acm.advdiff_params(eps=eps, max_iter=args.c5_max_iter, precision=acm.FP64)
    # the Peclet number is defined with the unit-cell velocity (nu = 1): u scales as 1/nu
    tA, DA, DxA, dA = acm.acm_advdiff_tensor(ctx, Hd, uA * nu, 10.0, qA)
    tB, DB, DxB, dB = acm.acm_advdiff_tensor(ctx, Hd, uB * nu, 10.0, qB)
    ctx.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "512^3 Gaussian random field (correlation 16 vox) thresholded to porosity 0.3; "
                               "Stokes load e_x + solute Pe 10 x 3 loads", "n": n, "porosity": round(porosity, 4),
                   "iters_per_step": iters, "problems_per_step": 4, "tiles": tiles,
                   "l2": "inputs larger than L2"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4) if achieved else None, "traffic": None,
                     "peak_source": peak_src},
        "clocks": clocks,
        "kernels": kern,
        "precision_check": {
            "eps": eps, "eps32": eps32, "nu": nu,
            "note": "nu = 1: unit cell; nu = 1/n^2: lengths in voxels (velocities O(1), so the absolute part "
                    "of the tolerance does not end the iteration early)",
            "stokes_fp32_then_fp64": {"status": sA, "iters": rA.iters, "iters_fp64": rA.iters_fp64,
                                      "converged": rA.converged, "ms": rA.time_ms, "K_xx": float(KA[0] * nu)},
            "stokes_fp64": {"status": sB, "iters": rB.iters, "converged": rB.converged, "ms": rB.time_ms,
                            "K_xx": float(KB[0] * nu)},
            "K_col_rel_diff": float(np.linalg.norm(KA - KB) / np.linalg.norm(KB)),
            "u_rel_l2_diff": du,
            "solute_fp32_then_fp64": {"iters": [r.iters for r in dA], "iters_fp64": [r.iters_fp64 for r in dA],
                                      "converged": [r.converged for r in dA], "D": DA.tolist()},
            "solute_fp64": {"iters": [r.iters for r in dB], "converged": [r.converged for r in dB], "D": DB.tolist()},
            "D_rel_diff": float(np.linalg.norm(DA - DB) / np.linalg.norm(DB)),
        },
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--iters", type=int, default=20, help="iterations per problem per step")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ttk", action=argparse.BooleanOptionalAction, default=True,
                    help="also measure time-to-permeability (K within 1e-4 of a long-run reference)")
    ap.add_argument("--ttk-long", type=int, default=8000,
                    help="iterations of the library-default form's self-referenced run")
    ap.add_argument("--ttk-iters", type=int, default=1000,
                    help="iterations of the FP32 run timed against the FP64 reference (0: skip that form)")
    ap.add_argument("--ttk-ref-iters", type=int, default=2000,
                    help="iteration cap of the FP64 references (started from the FP32 end state)")
    ap.add_argument("--ttk-cells", type=int, default=8,
                    help="cells of the reduced batched time-to-permeability figure (0: skip)")
    ap.add_argument("--ttk-default-form", action="store_true",
                    help="also time the library defaults (Eq. 13 symbols, Eq. 22) against their own long run")
    ap.add_argument("--config", default="cell256", choices=["cell256", "batched", "grf512"],
                    help="cell256: the 256^3 cell (default); batched: 384 cells (192 at 64^3, 192 at 128^3); "
                         "grf512: the 512^3 Gaussian random field with the FP32/FP64 comparison")
    ap.add_argument("--c5-eps", type=float, default=1e-6, help="grf512: tolerance of the accuracy runs")
    ap.add_argument("--c5-eps32", type=float, default=1e-5, help="grf512: FP32 stage tolerance")
    ap.add_argument("--c5-max-iter", type=int, default=20000)
    ap.add_argument("--c5-nu", type=float, default=1.0, help="grf512: viscosity of the accuracy runs")
    ap.add_argument("--cells", type=int, default=384, help="cells of the batched configuration")
    ap.add_argument("--ttk-batched", type=int, default=0,
                    help="batched: also follow K of every cell for this many iterations (time to permeability)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
        # one rank (re)builds the library if needed; the others wait for it
        if int(os.environ.get("LOCAL_RANK", "0")) == 0:
            from paper_2312_15554_gb300 import build as B
            B.build()
        dist.barrier()
    if args.config == "batched":
        run_batched(args, rank, world, dist)
    elif args.config == "grf512":
        run_grf512(args, rank, world, dist)
    else:
        run_gpu(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Host-side arithmetic of the bench line (no GPU): the step-level roofline and
the algorithmic byte counts it is built from."""
import numpy as np
import pytest

import bench


def test_step_roofline_is_the_time_weighted_bandwidth_of_the_counted_kernels():
    kern = {"a": {"ms": 1.0, "launches": 1, "GBps": 1000.0},   # 1 GB in 1 ms
            "b": {"ms": 1.0, "launches": 2, "GBps": 3000.0},   # 3 GB in 1 ms
            "other": {"ms": 2.0, "launches": 5, "GBps": None}}  # no byte count
    r = bench.step_roofline(kern, 4000.0)
    assert r["achieved"] == 2000.0          # 4 GB over 2 ms
    assert r["frac"] == 0.5
    assert r["time_share"] == 0.5           # 2 of 4 ms carry a byte count
    assert bench.step_roofline({"other": {"ms": 1.0, "launches": 1, "GBps": None}}, 4000.0) is None


def test_algorithmic_bytes_count_half_spectrum_components_and_the_solid_share():
    n2 = 256
    cspec = 8.0 * (n2 // 2 + 1) / n2
    # the Green passes move whole components of the half spectrum only
    assert bench.algorithmic_bytes_per_voxel("z_stokes", n2, 0.35) == 10 * cspec
    assert bench.algorithmic_bytes_per_voxel("y_inv_solute", n2, 0.35) == 5 * cspec
    # the multiplier lives on solid voxels: more solid, more bytes
    lo = bench.algorithmic_bytes_per_voxel("x_stokes_local", n2, 0.6)
    hi = bench.algorithmic_bytes_per_voxel("x_stokes_local", n2, 0.3)
    assert hi - lo == pytest.approx(24.0 * 0.3, rel=1e-12)
    assert bench.algorithmic_bytes_per_voxel("finalize", n2, 0.35) == 0.0


def test_time_to_permeability_crossing_is_the_first_iteration_that_stays_within():
    from paper_2312_15554_gb300 import ttk
    K_ref = np.eye(3)
    errs = [0.5, 0.05, 0.2, 0.02, 0.008, 0.009, 0.001]   # Frobenius errors e / sqrt(3) of K_ref = I
    hist = np.stack([K_ref * (1 + e / np.sqrt(3)) for e in errs])   # Frobenius error e
    assert ttk.crossing(hist, K_ref, 0.1) == 4          # 0.2 at iteration 3 breaks the earlier entry
    assert ttk.crossing(hist, K_ref, 0.01) == 5
    assert ttk.crossing(hist, K_ref, 1e-4) is None      # never reached within the run
    assert ttk.crossing(hist, K_ref, 1.0) == 1
    # voxel units of a cube and of a plane cell
    assert ttk.grid_nu((64, 64, 64)) == pytest.approx(1 / 64**2, rel=1e-12)
    assert ttk.grid_nu((1, 128, 128)) == pytest.approx(1 / 128**2, rel=1e-12)

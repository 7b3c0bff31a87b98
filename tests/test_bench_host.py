"""Host-side arithmetic of the bench line (no GPU): the step-level roofline and
the algorithmic byte counts it is built from."""
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

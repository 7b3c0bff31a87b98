"""Seeded synthetic inputs for the ACM solvers: microstructures and random fields.

This module holds no arithmetic of the method itself. It only builds the
indicator grids H (Eq. 4: 1 = solid, 0 = pore) and random test fields, and is
the one module shared by the CPU oracle tests and the CUDA path.

Geometry conventions
--------------------
* A grid has shape (n0, n1, n2); axis 2 is contiguous in memory.
* The unit cell is the unit cube; voxel (i0, i1, i2) has centre
  ((i0 + 1/2)/n0, (i1 + 1/2)/n1, (i2 + 1/2)/n2).
* Vector fields are component-planar, shape (3, n0, n1, n2); component c is
  the component along array axis c.
* A voxel is solid when the periodic minimum-image distance from its centre to
  a sphere centre is at most the sphere radius.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014), written out
below from its published definition, so that a seed gives the same geometry on
every machine.
"""
from __future__ import annotations

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 counter-based generator (Steele, Lea & Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def _periodic_delta(idx: np.ndarray, n: int, c: float) -> np.ndarray:
    """Minimum-image distance (in voxels) from voxel centres idx + 1/2 to c."""
    d = (idx + 0.5) - c
    return d - n * np.round(d / n)


def _stamp_sphere(H: np.ndarray, centre_vox, radius_vox: float) -> int:
    """Mark the voxels of one periodic sphere solid; return how many were new."""
    shape = H.shape
    ranges = []
    for ax in range(3):
        n = shape[ax]
        c = centre_vox[ax]
        lo = int(np.floor(c - 0.5 - radius_vox)) - 1
        hi = int(np.ceil(c - 0.5 + radius_vox)) + 1
        idx = np.arange(lo, hi + 1)
        if idx.size >= n:
            idx = np.arange(n)
        ranges.append(np.mod(idx, n))
    d0 = _periodic_delta(ranges[0], shape[0], centre_vox[0])
    d1 = _periodic_delta(ranges[1], shape[1], centre_vox[1])
    d2 = _periodic_delta(ranges[2], shape[2], centre_vox[2])
    r2 = d0[:, None, None] ** 2 + d1[None, :, None] ** 2 + d2[None, None, :] ** 2
    mask = r2 <= radius_vox * radius_vox
    sub = H[np.ix_(ranges[0], ranges[1], ranges[2])]
    new = int(np.count_nonzero(mask & (sub == 0)))
    if new:
        sub[mask] = 1
        H[np.ix_(ranges[0], ranges[1], ranges[2])] = sub
    return new


def single_sphere(shape, radius: float = 0.3, centre=(0.5, 0.5, 0.5)) -> np.ndarray:
    """One solid sphere of radius `radius` (unit-cell units) at `centre`."""
    shape = tuple(int(s) for s in shape)
    if np.isscalar(shape) or len(shape) != 3:
        raise ValueError("shape must be (n0, n1, n2)")
    H = np.zeros(shape, dtype=np.uint8)
    # distances measured in unit-cell units on each axis
    d = [(_periodic_delta(np.arange(n), n, centre[a] * n)) / n for a, n in enumerate(shape)]
    r2 = d[0][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[2][None, None, :] ** 2
    H[r2 <= radius * radius] = 1
    return H


def single_cylinder(shape, radius: float = 0.3, centre=(0.5, 0.5)) -> np.ndarray:
    """One solid disk of radius `radius` (unit-cell units) at `centre` of the
    (axis 1, axis 2) plane, the same on every plane along axis 0 (a cylinder;
    with shape (1, n, n) the two-dimensional cell)."""
    shape = tuple(int(s) for s in shape)
    H = np.zeros(shape, dtype=np.uint8)
    d1 = _periodic_delta(np.arange(shape[1]), shape[1], centre[0] * shape[1]) / shape[1]
    d2 = _periodic_delta(np.arange(shape[2]), shape[2], centre[1] * shape[2]) / shape[2]
    H[:, d1[:, None] ** 2 + d2[None, :] ** 2 <= radius * radius] = 1
    return H


def disk_pack(n1: int, n2: int, target_porosity: float, radius_vox, seed: int, max_disks: int = 1_000_000):
    """Boolean (overlapping) pack of disks in a (1, n1, n2) cell, the
    two-dimensional analogue of sphere_pack: centres uniform in the plane from
    SplitMix64(seed) (two uniforms per disk, then one for the radius when
    `radius_vox` is a (lo, hi) range), added until the porosity is at most
    `target_porosity`."""
    H = np.zeros((1, n1, n2), dtype=np.uint8)
    rng = SplitMix64(seed)
    target_solid = (1.0 - target_porosity) * H.size
    ranged = not np.isscalar(radius_vox)
    i1, i2 = np.arange(n1) + 0.5, np.arange(n2) + 0.5
    ndisks = 0
    while np.count_nonzero(H) < target_solid:
        if ndisks >= max_disks:
            raise RuntimeError("disk_pack: disk budget exhausted")
        c1, c2 = rng.uniform() * n1, rng.uniform() * n2
        r = (radius_vox[0] + (radius_vox[1] - radius_vox[0]) * rng.uniform()) if ranged else float(radius_vox)
        d1 = np.abs(i1 - c1)
        d1 = np.minimum(d1, n1 - d1)
        d2 = np.abs(i2 - c2)
        d2 = np.minimum(d2, n2 - d2)
        H[0][d1[:, None] ** 2 + d2[None, :] ** 2 <= r * r] = 1
        ndisks += 1
    return H


def slab(shape, solid_layers: int, normal_axis: int = 1) -> np.ndarray:
    """Plane channel: the first `solid_layers` layers normal to `normal_axis` are solid."""
    H = np.zeros(tuple(shape), dtype=np.uint8)
    sl = [slice(None)] * 3
    sl[normal_axis] = slice(0, solid_layers)
    H[tuple(sl)] = 1
    return H


def laminate(shape, solid_layers: int, normal_axis: int = 0) -> np.ndarray:
    """Laminate of one solid and one pore layer stack normal to `normal_axis`."""
    return slab(shape, solid_layers, normal_axis)


def sphere_pack(shape, target_porosity: float, radius_vox, seed: int,
                max_spheres: int = 10_000_000):
    """Boolean (overlapping) sphere pack.

    Sphere centres are uniform in the cell (Poisson), drawn from SplitMix64(seed)
    as three uniforms per sphere, followed by one more uniform for the radius when
    `radius_vox` is a (lo, hi) range. Spheres are added one at a time until the
    voxel porosity is at most `target_porosity`. Returns (H, centres, radii) with
    centres in voxel units.
    """
    shape = tuple(int(s) for s in shape)
    H = np.zeros(shape, dtype=np.uint8)
    V = H.size
    rng = SplitMix64(seed)
    solid = 0
    target_solid = (1.0 - target_porosity) * V
    centres, radii = [], []
    ranged = not np.isscalar(radius_vox)
    while solid < target_solid:
        if len(radii) >= max_spheres:
            raise RuntimeError("sphere_pack: sphere budget exhausted")
        c = (rng.uniform() * shape[0], rng.uniform() * shape[1], rng.uniform() * shape[2])
        if ranged:
            lo, hi = radius_vox
            r = lo + (hi - lo) * rng.uniform()
        else:
            r = float(radius_vox)
        solid += _stamp_sphere(H, c, r)
        centres.append(c)
        radii.append(r)
    return H, np.array(centres), np.array(radii)


def cell_recipe(seed: int):
    """Per-cell recipe of the batched workload: porosity ~U[0.2, 0.6], radii ~U[3, 10] voxels."""
    rng = SplitMix64(seed ^ 0x5DEECE66D)
    porosity = 0.2 + 0.4 * rng.uniform()
    return porosity, (3.0, 10.0)


def gaussian_random_field(shape, corr_len_vox: float, seed: int) -> np.ndarray:
    """Stationary Gaussian random field with covariance exp(-r^2 / (2 l^2)).

    White noise (numpy PCG64, seeded) filtered in Fourier space by the square
    root of the Gaussian spectral density exp(-l^2 |k|^2 / 2), k in radians per
    voxel. Returned with zero mean and unit variance.
    """
    shape = tuple(int(s) for s in shape)
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal(shape)
    wh = np.fft.rfftn(w)
    k0 = 2 * np.pi * np.fft.fftfreq(shape[0])
    k1 = 2 * np.pi * np.fft.fftfreq(shape[1])
    k2 = 2 * np.pi * np.fft.rfftfreq(shape[2])
    k2sq = k0[:, None, None] ** 2 + k1[None, :, None] ** 2 + k2[None, None, :] ** 2
    wh *= np.exp(-0.25 * corr_len_vox ** 2 * k2sq)
    f = np.fft.irfftn(wh, s=shape)
    f -= f.mean()
    f /= f.std()
    return f


def grf_medium(shape, corr_len_vox: float, porosity: float, seed: int) -> np.ndarray:
    """Thresholded Gaussian random field: the round(porosity * V) lowest values are pore.

    Ties are broken by linear index (stable sort).
    """
    f = gaussian_random_field(shape, corr_len_vox, seed).ravel()
    n_pore = int(round(porosity * f.size))
    order = np.argsort(f, kind="stable")
    H = np.ones(f.size, dtype=np.uint8)
    H[order[:n_pore]] = 0
    return H.reshape(shape)


def random_indicator(shape, solid_fraction: float, seed: int) -> np.ndarray:
    """Independent Bernoulli voxels (tiny brute-force test cases)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.random(tuple(shape)) < solid_fraction).astype(np.uint8)


def random_field(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Standard normal FP64 field (numpy PCG64, seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal(tuple(shape))


def dissolve(H: np.ndarray, layers: int = 1, fraction: float = 1.0, seed: int = 0) -> np.ndarray:
    """Dissolve solid at the pore interface, `layers` times: a solid voxel with a
    pore voxel among its six periodic face neighbours becomes pore, each with
    probability `fraction` (numpy PCG64, seeded); fraction 1 removes whole
    layers. The geometry sequence of an evolving medium."""
    H = np.asarray(H, dtype=np.uint8).copy()
    rng = np.random.Generator(np.random.PCG64(seed))
    for _ in range(layers):
        pore = H == 0
        touch = np.zeros_like(pore)
        for ax in range(3):
            touch |= np.roll(pore, 1, axis=ax) | np.roll(pore, -1, axis=ax)
        front = (H == 1) & touch
        if fraction < 1.0:
            front &= rng.random(H.shape) < fraction
        H[front] = 0
    return H


def porosity(H: np.ndarray) -> float:
    return 1.0 - float(np.count_nonzero(H)) / H.size

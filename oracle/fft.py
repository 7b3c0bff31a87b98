"""The oracle's own discrete Fourier transform (test infrastructure only).

Nothing in the product library imports, links or calls this module; only the
oracle, the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` do. It shares no code with the CUDA path.

The transforms of Algorithm 1 (Section 3.3) and the per-wavevector solves of
Eq. 13 and Eq. 20 need the multidimensional DFT

    forward  f^(m) = sum_x f(x) exp(-2 pi i m.x)          (unnormalised)
    inverse  f(x)  = (1/V) sum_m f^(m) exp(+2 pi i m.x)

applied axis by axis. Each axis is transformed by `oracle_fft.c` (an iterative
radix-2 Cooley-Tukey FFT for power-of-two lengths, the plain O(n^2) sum for
the small odd-sized test grids; compiled with gcc on first use and spread over
the host cores with OpenMP). `dft_direct` is the O(n^2) definition written out
with explicit exponentials, the independent check of the fast transform.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "oracle_fft.c")
_OUT = os.path.join(_DIR, "_lib")
_LIB_PATH = os.path.join(_OUT, "liboracle_fft.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle_fft.c into oracle/_lib/liboracle_fft.so (OpenMP when gcc supports it)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(_OUT, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_OUT)
    os.close(fd)
    base = ["gcc", "-O2", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:4] + ["-fopenmp"] + base[4:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
    if r.returncode != 0:
        os.unlink(tmp)
        raise RuntimeError(f"gcc failed on oracle_fft.c:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    try:
        lib = ctypes.CDLL(build())
    except OSError:
        # a library left by another machine (architecture mismatch): rebuild
        lib = ctypes.CDLL(build(force=True))
    lib.oracle_fft_axis.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_longlong,
                                    ctypes.c_int]
    lib.oracle_fft_axis.restype = ctypes.c_int
    lib.oracle_fft_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def threads() -> int:
    """Host threads the transforms run on."""
    return int(_load().oracle_fft_threads())


def _transform(a, axes, sign):
    lib = _load()
    out = np.array(a, dtype=np.complex128, order="C", copy=True)
    for ax in axes:
        ax = ax % out.ndim
        n = out.shape[ax]
        outer = int(np.prod(out.shape[:ax], dtype=np.int64))
        inner = int(np.prod(out.shape[ax + 1:], dtype=np.int64))
        if out.size and lib.oracle_fft_axis(out.ctypes.data, outer, n, inner, sign) != 0:
            raise MemoryError("oracle FFT: line buffer allocation failed")
    return out


def fftn(a, axes=(-3, -2, -1)):
    """Forward DFT over `axes`, unnormalised: sum_x f(x) exp(-2 pi i m.x)."""
    return _transform(a, axes, -1)


def ifftn(a, axes=(-3, -2, -1)):
    """Inverse DFT over `axes`: (1/V) sum_m f^(m) exp(+2 pi i m.x)."""
    out = _transform(a, axes, +1)
    out /= float(np.prod([out.shape[ax % out.ndim] for ax in axes]))
    return out


def rfftn(a, axes=(-3, -2, -1)):
    """Forward DFT of a real field, kept on the half spectrum m_last = 0..n_last/2."""
    n = np.shape(a)[axes[-1]]
    full = fftn(np.asarray(a, dtype=np.float64), axes)
    return np.take(full, np.arange(n // 2 + 1), axis=axes[-1])


def irfftn(half, s, axes=(-3, -2, -1)):
    """Real field (1/V) sum_m w_m Re[Y(m) exp(+2 pi i m.x)] of a half spectrum Y.

    m runs over the half spectrum (last axis 0..n/2); w_m = 1 on the planes
    m_last = 0 and m_last = n/2 and 2 elsewhere: the Hermitian completion of Y,
    counting the imaginary parts of the two self-conjugate planes as zero.
    """
    half = np.asarray(half, dtype=np.complex128)
    ax = axes[-1] % half.ndim
    n = s[-1]
    shape = list(half.shape)
    shape[ax] = n
    full = np.zeros(shape, dtype=np.complex128)
    w = np.full(n // 2 + 1, 2.0)
    w[0] = 1.0
    w[n // 2] = 1.0
    bw = [1] * half.ndim
    bw[ax] = n // 2 + 1
    idx = [slice(None)] * half.ndim
    idx[ax] = slice(0, n // 2 + 1)
    full[tuple(idx)] = half * w.reshape(bw)
    return ifftn(full, axes).real


def dft_direct(a, axis=-1, sign=-1):
    """The DFT along one axis by its definition, sum_j a_j exp(sign 2 pi i j m / n).

    The phase j m is reduced modulo n in exact integer arithmetic before the
    exponential is taken (O(n^2); for checking the fast transform only).
    """
    a = np.asarray(a, dtype=np.complex128)
    n = a.shape[axis]
    j = np.arange(n)
    ph = np.outer(j, j) % n
    W = np.exp(sign * 2j * np.pi * ph / n)
    return np.moveaxis(np.tensordot(W, np.moveaxis(a, axis, 0), axes=(1, 0)), 0, axis)

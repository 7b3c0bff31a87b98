"""The allocation-free transform entry point (acm_fft_r2c_static).

Some callers cannot let a library allocate device memory: applications that
give each component a fixed device-memory budget under their own allocator, and
latency-critical loops that must not call cudaMalloc/cudaFree because those can
synchronise the device. acm_fft_r2c_static serves them from a fixed device
array that the library holds; these tests call it through the C ABI twice in a
row and compare it with the context-based acm_fft_r2c.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2312_15554_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _reference(lib, x, fp64):
    ctx = lib.acm_ctx(x.shape)
    out = torch.zeros(x.shape[:2] + (x.shape[2] // 2 + 1, 2), dtype=x.dtype, device=DEV)
    lib.acm_fft_r2c(ctx, x, out, fp64)
    torch.cuda.synchronize()
    ctx.close()
    return out.cpu().numpy()


@pytest.mark.parametrize("shape,fp64", [((32, 64, 128), False), ((128, 128, 128), False),
                                        ((16, 16, 64), True), ((128, 128, 64), True)])
def test_static_transform_matches_context_transform_twice(lib, shape, fp64):
    dt = torch.float64 if fp64 else torch.float32
    tol = 1e-12 if fp64 else 2e-6
    for seed in (3, 4):                      # two calls in a row share the device array
        x = torch.as_tensor(I.random_field(shape, seed), dtype=dt, device=DEV)
        out = torch.full(shape[:2] + (shape[2] // 2 + 1, 2), float("nan"), dtype=dt, device=DEV)
        lib.acm_fft_r2c_static(x, out, fp64)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = _reference(lib, x, fp64)
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("shape,fp64", [((512, 512, 8), False), ((256, 512, 8), True)])
def test_static_transform_at_the_scratch_limit_matches_the_oracle_transform(lib, shape, fp64):
    """Grids whose working spectrum n0 * n1 * (n2/2 + 4) fills the 16 MiB array
    exactly, twice in a row, against the oracle's own transform."""
    from oracle import fft as OF
    dt = torch.float64 if fp64 else torch.float32
    tol = 1e-12 if fp64 else 2e-6
    for seed in (5, 6):
        xh = I.random_field(shape, seed)
        x = torch.as_tensor(xh, dtype=dt, device=DEV)
        out = torch.full(shape[:2] + (shape[2] // 2 + 1, 2), float("nan"), dtype=dt, device=DEV)
        lib.acm_fft_r2c_static(x, out, fp64)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        got = got[..., 0] + 1j * got[..., 1]
        ref = OF.rfftn(np.asarray(x.cpu().numpy(), dtype=np.float64))
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("shape,fp64", [((128, 256, 128), False), ((64, 256, 128), True),
                                        ((128, 128, 128), True), ((512, 512, 16), False)])
def test_static_transform_rejects_grids_just_beyond_the_scratch(lib, shape, fp64):
    dt = torch.float64 if fp64 else torch.float32
    x = torch.zeros(shape, dtype=dt, device=DEV)
    out = torch.zeros(shape[:2] + (shape[2] // 2 + 1, 2), dtype=dt, device=DEV)
    with pytest.raises(lib.AcmError) as e:
        lib.acm_fft_r2c_static(x, out, fp64)
    assert e.value.status == -10


def test_static_transform_rejects_oversized_grids_and_host_buffers(lib):
    x = torch.zeros((256, 256, 256), dtype=torch.float32, device=DEV)
    out = torch.zeros((256, 256, 129, 2), dtype=torch.float32, device=DEV)
    with pytest.raises(lib.AcmError) as e:
        lib.acm_fft_r2c_static(x, out, False)
    assert e.value.status == -10              # beyond the fixed scratch size
    # host buffers would need staging memory: the C entry point refuses them
    xh = torch.zeros((16, 16, 16), dtype=torch.float32).pin_memory()
    oh = torch.zeros((16, 16, 9, 2), dtype=torch.float32).pin_memory()
    s = lib.load().acm_fft_r2c_static(16, 16, 16, 0, lib._ptr(xh), lib._ptr(oh), None)
    assert s == -1

"""The tile autotuner of the strided FFT passes.

A tile width only regroups which spectral columns one block transforms, so
every width gives the same fields up to rounding (each compiled variant may
contract multiply-adds differently) and the FP64 residual partial sums change
their order only. The tests solve with every compiled width of every tuned pass
and compare with the default widths, then check that the tuner picks among the
compiled widths and leaves the results unchanged.
"""
import itertools

import numpy as np
import pytest
import torch

from paper_2312_15554_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _widths(lib, ctx, fp64):
    """Compiled widths of each tuned pass: the default, and half, double and four
    times it when they exist, and the register-resident variant (reported as -W,
    W = 16 columns per block in FP32, 8 in FP64) where it exists."""
    base = lib.acm_get_tiles(ctx, fp64)
    out = {}
    for k, w in base.items():
        opts = [w]
        for cand in (w // 2, w * 2, w * 4, -8 if fp64 else -16, -4 if fp64 else -8):
            t = dict(base)
            t[k] = cand
            try:
                lib.acm_set_tiles(ctx, t, fp64)
                opts.append(cand)
            except lib.AcmError:
                pass
        out[k] = opts
    lib.acm_set_tiles(ctx, base, fp64)
    return base, out


def _stokes(lib, ctx, H, fp64):
    dt = torch.float64 if fp64 else torch.float32
    u = torch.zeros((3,) + H.shape, dtype=dt, device=DEV)
    prm = lib.stokes_params(eps=0.0, adaptive=0, max_iter=6, precision=lib.FP64 if fp64 else lib.FP32,
                            alpha0=300, beta0=300, b0=300)
    s, K, rep, *_ = lib.acm_stokes(ctx, torch.as_tensor(H, device=DEV), [1.0, 0.3, 0.0], prm, u=u)
    return u.cpu().numpy(), np.array(rep.res[:6])


def _solute(lib, ctx, H, u, fp64):
    dt = torch.float64 if fp64 else torch.float32
    chi = torch.zeros(H.shape, dtype=dt, device=DEV)
    prm = lib.advdiff_params(eps=0.0, max_iter=5, precision=lib.FP64 if fp64 else lib.FP32)
    lib.acm_advdiff(ctx, torch.as_tensor(H, device=DEV), torch.as_tensor(u, dtype=dt, device=DEV), 10.0,
                    [1.0, 0.0, 0.0], prm, chi=chi)
    return chi.cpu().numpy()


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("shape", [(64, 64, 64), (128, 64, 32), (128, 64, 16)])
def test_every_tile_width_gives_identical_fields(lib, shape, fp64):
    H = I.sphere_pack(shape, 0.5, 4.0, 3)[0]
    ctx = lib.acm_ctx(shape)
    base, opts = _widths(lib, ctx, fp64)
    assert any(len(v) > 1 for v in opts.values())
    # the register-resident variant exists for every tuned pass at 64, 128 and
    # 256 points
    for k, ws in opts.items():
        n = shape[1] if k.startswith("y") else shape[0]
        want = n in (64, 128, 256)
        assert any(w < 0 for w in ws) == want, (k, ws)
    u0, r0 = _stokes(lib, ctx, H, fp64)
    uin = 1e3 * u0
    c0 = _solute(lib, ctx, H, uin, fp64)
    # each pass in turn at each of its widths, the others at their defaults
    for k, ws in opts.items():
        for w in ws[1:]:
            t = dict(base)
            t[k] = w
            lib.acm_set_tiles(ctx, t, fp64)
            u1, r1 = _stokes(lib, ctx, H, fp64)
            c1 = _solute(lib, ctx, H, uin, fp64)
            tol = 1e-13 if fp64 else 1e-6
            np.testing.assert_allclose(u1, u0, rtol=tol, atol=tol * np.abs(u0).max(), err_msg=f"{k} {w}")
            np.testing.assert_allclose(c1, c0, rtol=tol, atol=tol * np.abs(c0).max(), err_msg=f"{k} {w}")
            np.testing.assert_allclose(r1, r0, rtol=1e-9 if fp64 else 1e-5)  # FP32 per-thread partials regroup
    ctx.close()


def test_autotuner_picks_compiled_widths_and_keeps_results(lib):
    shape = (64, 64, 64)
    H = I.sphere_pack(shape, 0.4, 5.0, 4)[0]
    ctx = lib.acm_ctx(shape)
    _, opts = _widths(lib, ctx, False)
    u0, _ = _stokes(lib, ctx, H, False)
    tiles = lib.acm_autotune(ctx, False)
    for k, w in tiles.items():
        assert w in opts[k], (k, w, opts[k])
    assert lib.acm_get_tiles(ctx, False) == tiles
    u1, _ = _stokes(lib, ctx, H, False)
    np.testing.assert_allclose(u1, u0, rtol=1e-6, atol=1e-6 * np.abs(u0).max())
    ctx.close()


def test_batch_autotune_per_shape_keeps_results(lib):
    shapes = [(64, 64, 64), (32, 32, 32), (64, 64, 64)]
    Hs = [torch.as_tensor(I.sphere_pack(sh, 0.45, 3.0, 30 + i)[0], device=DEV) for i, sh in enumerate(shapes)]
    batch = lib.acm_batch(shapes)
    prm = lib.stokes_params(eps=0.0, adaptive=0, max_iter=8, precision=lib.FP32, alpha0=200, beta0=200, b0=200)
    u0 = [torch.zeros((3, 3) + sh, device=DEV) for sh in shapes]
    lib.acm_batch_stokes(batch, Hs, prm, u0)
    lib.acm_batch_autotune(batch)
    t0, t2 = lib.acm_batch_tiles(batch, 0), lib.acm_batch_tiles(batch, 2)
    assert t0 == t2                      # one tuning per shape group
    u1 = [torch.zeros_like(x) for x in u0]
    lib.acm_batch_stokes(batch, Hs, prm, u1)
    for a, b in zip(u0, u1):
        torch.testing.assert_close(b, a, rtol=1e-6, atol=1e-6 * float(a.abs().max()))
    batch.close()

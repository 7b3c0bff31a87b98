"""Small fixed case for ncu captures: the bench geometry at n^3 (default 128).

Runs acm_stokes_tensor (4 ADMM iterations, FP32) then acm_advdiff_tensor
(Pe 10, 4 Lippmann-Schwinger iterations) through the binding. The Stokes loop
is launched from the host (device_loop = 0): kernels inside a graph with a
conditional node cannot be captured one by one.
Usage: python -m paper_2312_15554_gb300.profile_case [n]
"""
import os
import sys

import torch

from paper_2312_15554_gb300 import acm
from paper_2312_15554_gb300 import inputs as I


def main(n: int = 128):
    acm.load()
    H = I.sphere_pack((n, n, n), 0.35, 8.0 * n / 256, 2024)[0]
    dev = "cuda:0"
    ctx = acm.acm_ctx(H.shape)
    Hd = torch.as_tensor(H, device=dev)
    u3 = torch.zeros((3, 3) + H.shape, dtype=torch.float32, device=dev)
    s, K, Kg, reps = acm.acm_stokes_tensor(ctx, Hd, acm.stokes_params(eps=0.0, max_iter=4, device_loop=0), u3)
    s, D, Dx, reps = acm.acm_advdiff_tensor(ctx, Hd, u3[0], 10.0, acm.advdiff_params(eps=0.0, max_iter=4))
    torch.cuda.synchronize()
    ctx.close()
    print("ok", K[0, 0], D[0, 0])


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 128)

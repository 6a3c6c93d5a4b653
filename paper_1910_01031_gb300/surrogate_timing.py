"""Timing of the learned surrogate's inference: one network call over a batch
of fields, on the tcgen05 path (default) or the mma.sync path.

    python -m paper_1910_01031_gb300.surrogate_timing --fields 64 --nx 256 --ny 256

Prints one line per repetition: milliseconds of the call (CUDA events on the
surrogate's stream) and algorithmic TFLOP/s, 2 * 9 * (3*64 + 4*64*64 + 64*3)
FLOPs per pixel.  The weights are the random initial ones: the time does not
depend on them.
"""
from __future__ import annotations

import argparse
import ctypes

import torch

from . import iewpf

FLOPS_PER_PIXEL = 2 * 9 * (3 * 64 + 4 * 64 * 64 + 64 * 3)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--fields", type=int, default=64)
    ap.add_argument("--nx", type=int, default=256)
    ap.add_argument("--ny", type=int, default=256)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--path", type=int, default=0, choices=[0, 1], help="0 tcgen05, 1 mma.sync")
    args = ap.parse_args()
    sur = iewpf.Surrogate(args.nx, args.ny, 64, 6, seed=1)
    sur.set_scales([20.0, 0.2, 0.2], [0.004, 0.3, 0.3])
    sur.set_path(args.path)
    gen = torch.Generator(device="cuda").manual_seed(0)
    U = torch.randn(args.fields, 3, args.ny, args.nx, device="cuda", generator=gen)
    U *= torch.tensor([0.05, 5.0, 5.0], device="cuda").view(1, 3, 1, 1)
    st = torch.cuda.ExternalStream(sur.stream())
    handle = ctypes.c_void_p(st.cuda_stream)
    flops = FLOPS_PER_PIXEL * args.fields * args.nx * args.ny
    for rep in range(args.reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        sur.apply_device(U, stream=handle)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        print("path %d rep %d: %.3f ms, %.1f TFLOP/s (tcgen05: %s)" % (args.path, rep, ms, flops / ms / 1e9,
                                                                        sur.uses_tcgen05()), flush=True)
    sur.close()


if __name__ == "__main__":
    main()

"""Runs SpMV steps on one HPCG matrix for profiling (ncu launch lists and
kernel captures): python -m paper_1612_00530_gb300.profile_spmv
[--grid N] [--format ell|pattern|delta] [--order column|fast] [--steps K]
[--warmup W].  Prints the mean step time measured with CUDA events."""
from __future__ import annotations

import argparse

import torch

import paper_1612_00530_gb300 as P
import spmv_inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=192)
    ap.add_argument("--format", default="pattern", choices=("ell", "pattern", "delta"))
    ap.add_argument("--order", default="fast", choices=("column", "fast"))
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--kind", default="hpcg", choices=("hpcg", "irregular"))
    ap.add_argument("--variant", type=int, default=-1, help="FAST kernel: 0 direct, 1 staged, 2 pre-converted")
    ap.add_argument("--tile", type=int, default=2048)
    args = ap.parse_args()
    g = args.grid
    A = P.spmv_build(args.kind, g, g, g, seed=2)
    M = A if args.format == "ell" else P.spmv_compress(A, format=args.format, order=args.order)
    n = P.spmv_info(M)["n"]
    x = torch.from_numpy(spmv_inputs.uniform_vector(n, seed=1)).cuda()
    y = torch.empty_like(x)
    if args.variant >= 0:
        P.spmv_set_variant(M, args.variant, args.tile)
    for _ in range(args.warmup):
        P.spmv_apply(M, x, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        P.spmv_apply(M, x, y)
    e1.record()
    torch.cuda.synchronize()
    print(f"{args.kind} {g}^3 {args.format}/{args.order}: {e0.elapsed_time(e1) / args.steps * 1e3:.1f} us/step")


if __name__ == "__main__":
    main()

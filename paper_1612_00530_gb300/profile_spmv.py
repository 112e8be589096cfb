"""Runs SpMV steps on one HPCG matrix for profiling (ncu launch lists and
kernel captures): python -m paper_1612_00530_gb300.profile_spmv
[--grid N] [--format ell|pattern|delta|dit|data_table] [--reorder] [--order column|fast] [--steps K]
[--warmup W] [--variant V --tile T --threads B] [--spmm K [--spmm-kernel 0|1]].  Prints the
mean step time measured with CUDA events."""
from __future__ import annotations

import argparse

import torch

import paper_1612_00530_gb300 as P
import spmv_inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=192)
    ap.add_argument("--format", default="pattern", choices=("ell", "pattern", "delta", "dit", "data_table"))
    ap.add_argument("--reorder", action="store_true", help="locality reordering inside spmv_compress")
    ap.add_argument("--order", default="fast", choices=("column", "fast"))
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--kind", default="hpcg", choices=("hpcg", "irregular"))
    ap.add_argument("--variant", type=int, default=-1,
                    help="FAST kernel: 0 direct, 1 staged, 2 pre-converted, 3 staged pre-converted, "
                         "4/5 persistent, 6 register-staged, 7 z-marching, 8/9 register-staged with shared-memory "
                         "records / row types, 10 z-block (tile = 512 x planes, 256 threads)")
    ap.add_argument("--tile", type=int, default=2048)
    ap.add_argument("--threads", type=int, default=512, help="block size of the staged kernels (512 or 256)")
    ap.add_argument("--cg", choices=("fp64", "ir_fp32"), default=None,
                    help="run one CG solve (b = A 1) instead of SpMV steps")
    ap.add_argument("--cg-iters", type=int, default=40)
    ap.add_argument("--cg-rhs", type=int, default=1,
                    help="FP64 CG on this many right-hand sides at once (b_j = A v_j, V seed 22)")
    ap.add_argument("--spmm", type=int, default=0, help="time Y = A X with K right-hand sides (X seed 3)")
    ap.add_argument("--f32", type=int, default=-1, choices=(-1, 0, 1, 2),
                    help="time the binary32 product with kernel 2 (TMA), 1 (row types) or 0 (records)")
    ap.add_argument("--spmm-kernel", type=int, default=3, choices=(0, 1, 2, 3),
                    help="FAST SpMM kernel: 1-3 TMA-fed with that many CTAs an SM, 0 one thread a (row, column)")
    args = ap.parse_args()
    g = args.grid
    A = P.spmv_build(args.kind, g, g, g, seed=2)
    M = A if args.format == "ell" else P.spmv_compress(A, format=args.format, order=args.order,
                                                       reorder=args.reorder)
    n = P.spmv_info(M)["n"]
    x = torch.from_numpy(spmv_inputs.uniform_vector(n, seed=1)).cuda()
    y = torch.empty_like(x)
    if args.variant >= 0:
        P.spmv_set_tile(M, args.variant, args.tile, args.threads)
    if args.cg and args.cg_rhs > 1:
        V = torch.from_numpy(spmv_inputs.uniform_matrix(n, args.cg_rhs, seed=22)).cuda()
        B = torch.empty_like(V)
        P.spmm_apply(A, V, B)
        X0 = torch.zeros_like(B)
        r = P.cg_solve(M, B, X0, tol=1e-30, max_iter=args.cg_iters, check_every=8)
        print(f"cg fp64, {args.cg_rhs} right-hand sides: {r['iterations']} steps in {r['seconds'] * 1e3:.2f} ms "
              f"({r['seconds'] / max(1, r['iterations']) * 1e6:.1f} us/step)")
        return
    if args.cg:
        ones = torch.ones_like(x)
        P.spmv_apply(M, ones, y)
        xs = torch.zeros_like(x)
        r = P.cg_solve(M, y.clone(), xs, tol=1e-30, max_iter=args.cg_iters, mode=args.cg,
                       inner_max_iter=args.cg_iters, inner_tol=1e-30)
        print(f"cg {args.cg}: {r['iterations']} steps in {r['seconds'] * 1e3:.2f} ms "
              f"({r['seconds'] / max(1, r['iterations']) * 1e6:.1f} us/step)")
        return
    if args.f32 >= 0:
        P.spmv_set_f32_kernel(M, args.f32)
        x32, y32 = x.float(), torch.empty(n, dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            P.spmv_apply_f32(M, x32, y32)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            P.spmv_apply_f32(M, x32, y32)
        e1.record()
        torch.cuda.synchronize()
        print(f"{args.kind} {g}^3 {args.format} binary32 kernel={args.f32}: "
              f"{e0.elapsed_time(e1) / args.steps * 1e3:.1f} us/step")
        return
    if args.spmm:
        k = args.spmm
        X = torch.from_numpy(spmv_inputs.uniform_matrix(n, k, seed=3)).cuda()
        Y = torch.empty_like(X)
        if args.format == "pattern" and args.order == "fast":
            P.spmv_set_spmm_kernel(M, args.spmm_kernel)
        for _ in range(args.warmup):
            P.spmm_apply(M, X, Y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            P.spmm_apply(M, X, Y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        nnz = P.spmv_info(M)["nnz"]
        alg = nnz + n * 5 / 8 + 16 * n * k
        print(f"{args.kind} {g}^3 {args.format}/{args.order} spmm k={k} kernel={args.spmm_kernel}: "
              f"{ms * 1e3:.1f} us/step, {2 * nnz * k / ms / 1e6:.0f} GFLOP/s, {alg / ms / 1e6:.0f} GB/s algorithmic")
        return
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

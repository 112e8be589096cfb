#!/usr/bin/env python3
"""Benchmark: SpMV GFLOP/s and fraction of the HBM roofline, compressed
(pattern format, uint8 value codes + 5-bit stencil-pattern numbers, FAST
order) vs plain ELL, on the 192^3 HPCG matrix (7,077,888 rows, 189,119,224
nonzeros), x ~ U[-1,1) from seed 1, on one GB300.

A step is one y = A x with the compressed matrix, inputs resident in HBM.
GF/s counts 2 flops per stored nonzero (Sec. IV-B of arXiv:1612.00530).
The matrix, x and y together (311 MB) exceed the 129 MB L2, so no flush is
needed between steps.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU
(replicas; the method has no exchange step on one grid); the JSON line
reports the work of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = NZ = 192
X_SEED = 1
METRIC = "SpMV GFLOP/s + % HBM roofline, compressed vs plain ELL, 192^3 HPCG, 1 GB300"
WORKLOAD = "hpcg_192^3_x_seed1_compressed_pattern_uint8codes_5bit_patterns_vs_ell"


KERNEL_SOURCES = {"tma": ("k_tma.cu", "fast_fixed.cuh", "tma_ptx.cuh"),
                  "other": ("k_spmv.cu", "fast_fixed.cuh")}


def kernel_source_hash(kernel: str = "") -> str:
    """sha256 (first 16 hex digits) of the sources of a FAST kernel: the
    TMA-fed kernel's files for ids starting with "tma", else k_spmv.cu's."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES["tma" if kernel.startswith("tma") else "other"]:
        with open(os.path.join(ROOT, "paper_1612_00530_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled(kernel: str, tag: str = "traffic", key: str = "bytes"):
    """A per-launch ncu figure of `kernel` recorded in the committed summary
    in profiles/ (lines `<tag>: kernel=... source_sha256_16=... <key>=...`),
    if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "spmv_fast_hpcg192.md")
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as f:
        for line in f:
            if line.startswith(tag + ":"):
                parts = dict(p.split("=", 1) for p in line.split()[1:] if "=" in p)
                if parts.get("kernel") == kernel:
                    fields = parts
    if fields.get("source_sha256_16") != kernel_source_hash(kernel):
        return None
    try:
        return float(fields[key])
    except (KeyError, ValueError):
        return None


def profiled_traffic(kernel: str):
    """dram read+write bytes per launch of `kernel` (ncu), or None."""
    return profiled(kernel, "traffic", "bytes")


# GB300 rates used for the bounds the headline line reports beside the HBM
# roofline: 4 warp-instructions issued per SM per clock (one per scheduler),
# and the FP64 FMA rate a microbenchmark measured, 2.07 per SM per clock.
ISSUE_PER_SM_CLK = 4.0
FP64_FMA_PER_SM_CLK = 2.07
NOMINAL_HBM_GBS = 7900.0


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(seconds: float = 12.0, all_core_seconds: float = 6.0, y_check=None) -> dict:
    """The oracle's CSR SpMV as written, on this host: single-threaded (the
    reported value), and row-parallel on every host core (the same per-row
    fma chains over disjoint row blocks, so the same bits; reported beside).
    y_check: the timed GPU product on the same x, compared here with the
    oracle's, normwise and row by row against sum_j |a_ij x_j|."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    import spmv_inputs

    rowptr, col, val = oracle.hpcg_csr(NX, NY, NZ)
    n = NX * NY * NZ
    x = spmv_inputs.uniform_vector(n, seed=X_SEED)
    nnz = int(rowptr[-1])
    csr_bytes = 12.0 * nnz + 8.0 * (n + 1) + 16.0 * n     # col + val + rowptr + x + y
    reps, t0 = 0, time.perf_counter()
    while True:
        y1 = oracle.spmv(rowptr, col, val, x)
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = (time.perf_counter() - t0) / reps
    out = {"value": 2.0 * nnz / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
           "gbs": csr_bytes / dt / 1e9,
           "sample": f"{reps} full 192^3 CSR SpMVs (x seed 1), single thread, {reps * dt:.1f} s"}
    if y_check is not None:
        d = np.abs(np.asarray(y_check, dtype=np.float64) - y1)
        scale = oracle.spmv(rowptr, col, np.abs(val), np.abs(x))     # sum_j |a_ij x_j|
        out["parity"] = {"normwise": float(d.max() / np.abs(y1).max()),
                         "componentwise": float(np.max(np.where(scale > 0, d / np.where(scale > 0, scale, 1.0),
                                                                np.where(d > 0, np.inf, 0.0)))),
                         "bound": 1e-14, "rows": int(n)}
    # every core: the ctypes call releases the interpreter lock, so threads run
    # the oracle's row-range routine side by side
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    bounds = np.linspace(0, n, cores + 1).astype(np.int64)

    def block(b):
        lo, hi = int(bounds[b]), int(bounds[b + 1])
        return oracle.spmv_range(lo, hi, rowptr[lo:hi + 1], col, val, x)

    with ThreadPoolExecutor(cores) as ex:
        yp = np.concatenate(list(ex.map(block, range(cores))))
        same = bool(np.array_equal(yp.view(np.uint64), y1.view(np.uint64)))
        reps_p, t0 = 0, time.perf_counter()
        while True:
            list(ex.map(block, range(cores)))
            reps_p += 1
            if time.perf_counter() - t0 >= all_core_seconds:
                break
        dtp = (time.perf_counter() - t0) / reps_p
    out["all_cores"] = {"value": 2.0 * nnz / dtp / 1e9, "unit": "GFLOP/s", "cores": cores,
                        "gbs": csr_bytes / dtp / 1e9, "bit_identical_to_single_thread": same,
                        "sample": f"{reps_p} full 192^3 CSR SpMVs, {cores} row blocks on {cores} threads, "
                                  f"{reps_p * dtp:.1f} s"}
    return out


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_reference(args, world, rank):
    """The oracle as it stands, on the host cores, on a bounded sample."""
    if rank != 0:
        return
    cb = cpu_baseline(seconds=max(10.0, min(60.0, 0.4 * args.steps)))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "GFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 2.0 * 189119224 / cb["value"] / 1e6,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": NX * NY * NZ, "nnz": 189119224},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_timer(torch, stream=None):
    """ms per call of fn, CUDA events on `stream` (the current stream by
    default) after `warm` untimed calls."""
    def time_ms(fn, steps, warm=3):
        st = stream or torch.cuda.current_stream()
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps
    return time_ms


def bench_irregular(P, torch, dev, time_ms, peaks, iters=100):
    """Irregular 128^3 (seed 2): ELL vs the delta format, unordered and with
    the locality reordering inside spmv_compress (both bit-exact)."""
    import spmv_inputs
    A = P.spmv_build("irregular", 128, 128, 128, seed=2)
    C = P.spmv_compress(A)
    ia, ic = P.spmv_info(A), P.spmv_info(C)
    n, nnz = ic["n"], ic["nnz"]
    x = torch.from_numpy(spmv_inputs.uniform_vector(n, seed=2)).to(dev)
    y = torch.empty_like(x)
    t_ell = time_ms(lambda: P.spmv_apply(A, x, y), iters)
    t_d = time_ms(lambda: P.spmv_apply(C, x, y), iters)
    t0 = time.perf_counter()
    R = P.spmv_compress(A, reorder=True)
    t_reorder = time.perf_counter() - t0
    ir = P.spmv_info(R)
    t_r = time_ms(lambda: P.spmv_apply(R, x, y), iters)

    def fmt(info, ms, extra_bytes):
        return {"gflops": 2 * nnz / ms / 1e6, "ms": ms, "bytes_per_nnz": info["format_bytes"] / nnz,
                "gbs": (info["format_bytes"] + extra_bytes) / ms / 1e6,
                "slices_value_raw_frac": info["slices_value_raw"] / info["n_slices"],
                "slices_col_raw_frac": info["slices_col_raw"] / info["n_slices"], "dict_size": info["dict_size"],
                "bandwidth": info["bandwidth"]}
    out = {"rows": n, "nnz": nnz, "ell": {"gflops": 2 * nnz / t_ell / 1e6, "ms": t_ell,
                                           "bytes_per_nnz": ia["format_bytes"] / nnz},
           "delta": fmt(ic, t_d, 16 * n),
           "delta_reordered": dict(fmt(ir, t_r, 56 * n), compress_seconds=t_reorder),
           "speedup_vs_ell": {"delta": t_ell / t_d, "delta_reordered": t_ell / t_r},
           "peak_gbs": peaks["hbm_gbs"],
           "note": "gbs counts format bytes + x,y (16 B/row); reordered also the gather of x and scatter of y "
                   "(40 B/row more); column order, bit-exact"}
    return out


def bench_table2(P, torch, dev, A, x, time_ms, peaks, iters=100):
    """Table II's three layouts on 192^3: plain ELL ("Original"), the Data
    Table (value-sorted columns S_i + terminal indices T_i) and the
    Data+Index Table, both decoded in Listing 1's order (bit-exact)."""
    D = P.spmv_compress(A, format="dit")
    T = P.spmv_compress(A, format="data_table")
    idt, itb = P.spmv_info(D), P.spmv_info(T)
    n, nnz = idt["n"], idt["nnz"]
    y = torch.empty_like(x)
    t_ell = time_ms(lambda: P.spmv_apply(A, x, y), iters)
    t_dt = time_ms(lambda: P.spmv_apply(T, x, y), iters)
    t_dit = time_ms(lambda: P.spmv_apply(D, x, y), iters)

    def row(ms, fbytes, **kw):
        b = fbytes + 16 * n
        return {"gflops": 2 * nnz / ms / 1e6, "ms": ms, "bytes_per_row": fbytes / n, "gbs": b / ms / 1e6,
                "frac_of_hbm": b / ms / 1e6 / peaks["hbm_gbs"], **kw}
    return {"rows": n, "nnz": nnz,
            "original_ell": row(t_ell, 12 * nnz, paper_bytes_per_row=324),
            "data_table": row(t_dt, itb["format_bytes"], paper_bytes_per_row=116),
            "data_index_table": row(t_dit, idt["format_bytes"], types=idt["n_patterns"], paper_bytes_per_row=12),
            "speedup_vs_ell": {"data_table": t_ell / t_dt, "data_index_table": t_ell / t_dit},
            "paper_gflops_pezy_sc": {"original_ell": 11.6, "data_table": 15.9, "data_index_table": 32.4},
            "order": "Listing 1 (value groups ascending, one fma per entry; bit-exact)",
            "fp64_pipe_bound_ms": nnz / (FP64_FMA_PER_SM_CLK * torch.cuda.get_device_properties(dev).multi_processor_count
                                         * 2.07e9) * 1e3}


def bench_cg(P, torch, dev, A, C, batched=True, one_at_a_time=True):
    """CG on 192^3 with b = A 1, x0 = 0, to a relative residual of 1e-10:
    plain FP64 CG and FP64 iterative refinement around a binary32 inner
    CG; optionally eight right-hand sides (b_j = A v_j, v_j ~ U[-1,1) seed
    22) batched and one at a time."""
    import spmv_inputs
    n = P.spmv_info(C)["n"]
    ones = torch.ones(n, dtype=torch.float64, device=dev)
    b = torch.empty_like(ones)
    P.spmv_apply(A, ones, b)            # ELL, column order: integer sums, exact
    xx = torch.zeros_like(b)
    res = {}
    for mode, extra in (("fp64", {}), ("ir_fp32", {"inner_max_iter": 300, "inner_tol": 1e-6})):
        xx.zero_()
        r = P.cg_solve(C, b, xx, tol=1e-10, mode=mode, max_iter=5000, **extra)
        res[mode] = {"seconds": r["seconds"], "iterations": r["iterations"], "outer": r["outer_iterations"],
                     "rel_residual": r["rel_residual"], "max_abs_err_x_minus_1": float((xx - 1.0).abs().max()),
                     "status": r["status"], "history_head": r["history"][:4], "history_tail": r["history"][-3:],
                     "history_len": len(r["history"]), **extra}
    res["ir_speedup"] = res["fp64"]["seconds"] / res["ir_fp32"]["seconds"]
    if batched:
        kb = 8
        V = torch.from_numpy(spmv_inputs.uniform_matrix(n, kb, seed=22)).to(dev)
        Bm = torch.empty_like(V)
        for j in range(kb):              # b_j = A v_j by the exact ELL product, column by column
            vj = V[:, j].contiguous()
            bj = torch.empty_like(vj)
            P.spmv_apply(A, vj, bj)
            Bm[:, j] = bj
        Xm = torch.zeros_like(Bm)
        r = P.cg_solve(C, Bm, Xm, tol=1e-10, max_iter=5000)
        res["fp64_batched_8rhs"] = {"seconds": r["seconds"], "seconds_per_rhs": r["seconds"] / kb,
                                    "iterations": r["iterations"], "rel_residual": r["rel_residual"],
                                    "max_abs_err_x_minus_v": float((Xm - V).abs().max()), "status": r["status"]}
        if one_at_a_time:
            single_s, single_it = 0.0, []
            for j in range(kb):
                bj = Bm[:, j].contiguous()
                xj = torch.zeros_like(bj)
                rj = P.cg_solve(C, bj, xj, tol=1e-10, max_iter=5000)
                single_s += rj["seconds"]
                single_it.append(rj["iterations"])
            res["fp64_same_8rhs_one_at_a_time"] = {"seconds": single_s, "seconds_per_rhs": single_s / kb,
                                                   "iterations": single_it}
            res["batched_speedup_per_rhs"] = single_s / r["seconds"]
    return res


def bench_spmm(P, torch, dev, time_ms, ks=(1, 8, 32), iters=10, column=False, edge=160):
    """SpMM Y = A X on the HPCG matrix of edge^3, X ~ U[-1,1) (seed 3),
    FAST order (and COLUMN order when asked)."""
    import spmv_inputs
    A = P.spmv_build("hpcg", edge, edge, edge)
    Cf = P.spmv_compress(A, format="pattern", order="fast")
    Cc = P.spmv_compress(A, format="pattern", order="column") if column else None
    n, nnz = P.spmv_info(Cf)["n"], P.spmv_info(Cf)["nnz"]
    del A
    out = {"rows": n, "nnz": nnz}
    for k in ks:
        X = torch.from_numpy(spmv_inputs.uniform_matrix(n, k, seed=3)).to(dev)
        Y = torch.empty_like(X)
        tf = time_ms(lambda: P.spmm_apply(Cf, X, Y), iters)
        alg = nnz + n * 5 / 8 + 16 * n * k
        d = {"fast_gflops": 2 * nnz * k / tf / 1e6, "fast_ms": tf, "fast_gbs_alg": alg / tf / 1e6,
             "alg_bytes_per_row": alg / n}
        if Cc is not None:
            tc = time_ms(lambda: P.spmm_apply(Cc, X, Y), max(2, iters // 4), warm=1)
            d.update(column_gflops=2 * nnz * k / tc / 1e6, column_ms=tc)
        out[f"k{k}"] = d
        del X, Y
    return out


def bench_ragged(P, torch, dev, time_ms, iters=30):
    """24 HPCG cubes, edges U{16..96} (seed 4), one captured-graph launch
    for the whole batch vs one launch per matrix."""
    import spmv_inputs
    edges = spmv_inputs.grid_edges(24, seed=4)
    mats, xs, ys = [], [], []
    tot_nnz = 0
    for bidx, e in enumerate(edges):
        M = P.spmv_compress(P.spmv_build("hpcg", e, e, e), format="pattern")
        mats.append(M)
        tot_nnz += P.spmv_info(M)["nnz"]
        xs.append(torch.from_numpy(spmv_inputs.uniform_vector(e ** 3, seed=100 + bidx)).to(dev))
        ys.append(torch.empty_like(xs[-1]))
    plan = P.spmv_batch_create(mats, xs, ys)
    tb = time_ms(lambda: P.spmv_batch_launch(plan), iters)
    ts = time_ms(lambda: [P.spmv_apply(M, xv, yv) for M, xv, yv in zip(mats, xs, ys)], max(3, iters // 3))
    # the same batch in FAST order, its item size tuned
    for M in mats:
        P.spmv_set_order(M, "fast")
    plan_f = P.spmv_batch_create(mats, xs, ys)
    rows = P.spmv_batch_autotune(plan_f)
    tf = time_ms(lambda: P.spmv_batch_launch(plan_f), iters)
    return {"edges": edges, "nnz": tot_nnz,
            "batched_graph": {"ms": tb, "gflops": 2 * tot_nnz / tb / 1e6, "order": "column (bit-exact)"},
            "one_launch_per_matrix": {"ms": ts, "gflops": 2 * tot_nnz / ts / 1e6, "order": "column (bit-exact)"},
            "batched_graph_fast": {"ms": tf, "gflops": 2 * tot_nnz / tf / 1e6, "item_rows": rows,
                                   "order": "fast (<= 1e-14)"}}


def bench_row_types(P, torch, dev, A, x, time_ms, peaks, t_ell, iters=200):
    """Values registered in the pattern (Sec. V): one byte a row."""
    T = P.spmv_compress(A, format="pattern", order="fast")
    n, nnz = P.spmv_info(T)["n"], P.spmv_info(T)["nnz"]
    y = torch.empty_like(x)
    best = None
    for t, bt in ((1024, 256), (512, 256), (1024, 512)):
        P.spmv_set_tile(T, 9, t, bt)
        ms = time_ms(lambda: P.spmv_apply(T, x, y), iters)
        if best is None or ms < best[0]:
            best = (ms, t, bt)
    it = P.spmv_info(T)
    typed_bytes = n * 1 + 16 * n
    return {"rows": n, "nnz": nnz, "row_types": it["row_types"], "gflops": 2 * nnz / best[0] / 1e6,
            "ms": best[0], "tile_rows": best[1], "threads": best[2], "bytes_per_row": 1 + 16,
            "gbs": typed_bytes / best[0] / 1e6, "frac_of_hbm": typed_bytes / best[0] / 1e6 / peaks["hbm_gbs"],
            "speedup_vs_ell": t_ell / best[0], "order": "fast (<= 1e-14)"}


def run_suite(args):
    """The further workloads at full length, one JSON line each (irregular
    128^3, Table II layouts and row types on 192^3, CG vs IR-CG and
    batched CG on 192^3, SpMM k = 1..32 on 160^3, the ragged batch).  Not
    the headline."""
    import torch

    import paper_1612_00530_gb300 as P
    import spmv_inputs
    from paper_1612_00530_gb300 import build as lib_build

    lib_build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peaks = measured_peaks()
    time_ms = make_timer(torch)

    def emit(name, d):
        print(json.dumps({"workload": name, **d}), flush=True)

    emit("irregular_128^3_seed2", bench_irregular(P, torch, dev, time_ms, peaks, iters=200))
    A = P.spmv_build("hpcg", 192, 192, 192)
    n = P.spmv_info(A)["n"]
    x = torch.from_numpy(spmv_inputs.uniform_vector(n, seed=1)).to(dev)
    t2 = bench_table2(P, torch, dev, A, x, time_ms, peaks)
    emit("hpcg_192^3_table2_layouts", t2)
    emit("hpcg_192^3_row_types", bench_row_types(P, torch, dev, A, x, time_ms, peaks, t2["original_ell"]["ms"]))
    C = P.spmv_compress(A, format="pattern", order="fast")
    y = torch.empty_like(x)
    P.spmv_autotune(C, x, y)
    emit("cg_192^3_b_eq_A1_tol1e-10", bench_cg(P, torch, dev, A, C))
    del A, C, x, y
    emit("spmm_160^3_X_seed3", bench_spmm(P, torch, dev, time_ms, ks=(1, 4, 8, 16, 32), iters=20, column=True))
    emit("ragged_24_cubes_seed4", bench_ragged(P, torch, dev, time_ms, iters=50))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--suite", action="store_true", help="measure the further workloads instead of the headline")
    ap.add_argument("--kernel", default=None, metavar="VARIANT:TILE",
                    help="set the FAST kernel instead of running the autotuner (e.g. 11:1, the choice the "
                         "autotuner makes in plain runs; under a profiler its timings are distorted)")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave the further workloads' short measurements out of the headline line")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world, rank, local = dist_setup()
    import torch

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        run_reference(args, world, rank)
        barrier(world)
        return
    if args.suite:
        if rank == 0:
            run_suite(args)
        barrier(world)
        return

    import paper_1612_00530_gb300 as P
    import spmv_inputs
    from paper_1612_00530_gb300 import build as lib_build

    lib_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    A = P.spmv_build("hpcg", NX, NY, NZ)
    C = P.spmv_compress(A, format="pattern", order="fast")
    info_c, info_a = P.spmv_info(C), P.spmv_info(A)
    n, nnz = info_c["n"], info_c["nnz"]
    x_np = spmv_inputs.uniform_vector(n, seed=X_SEED)
    x = torch.from_numpy(x_np).to(dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    if args.kernel:
        kv, kt = (int(v) for v in args.kernel.split(":"))
        P.spmv_set_tile(C, kv, kt, 0)
    else:
        P.spmv_autotune(C, x, y)
    info_c = P.spmv_info(C)
    variant = info_c["fast_variant"]
    tile, threads = info_c["fast_tile_rows"], info_c["fast_block_threads"]
    launches_per_step = {0: 2, 1: 1, 2: 3, 3: 3, 4: 1, 5: 3, 6: 1, 7: 2, 8: 1, 9: 1, 10: 1, 11: 1}[variant]
    kernel_id = {0: "direct", 1: "staged%dt%d" % (tile, threads), 2: "preconverted", 3: "xstaged%d" % tile,
                 4: "persistent", 5: "persistent_x", 6: "rstaged%dt%d" % (tile, threads),
                 7: "zmarch%dt%d" % (tile, threads), 8: "rstaged_srec%dt%d" % (tile, threads),
                 9: "rstaged_types%dt%d" % (tile, threads), 10: "zblock%dt%d" % (tile, threads),
                 11: "tma%dt%d" % (tile, threads)}[variant]
    kernel_desc = {0: "xmax pre-pass + pattern_fast_kernel",
                   1: "pattern_fast_staged_kernel (%d-row shared-memory tiles, %d threads)" % (tile, threads),
                   2: "xmax + convert_x pre-passes + pattern_fast_x_kernel",
                   3: "xmax + convert_x pre-passes + pattern_fast_xstaged_kernel (%d-row tiles)" % tile,
                   4: "pattern_fast_async_kernel (persistent, double-buffered 1024-row tiles)",
                   5: "xmax + convert_x pre-passes + persistent pattern_fast_async_kernel",
                   6: "pattern_fast_rstaged_kernel (%d-row register-staged tiles, %d threads)" % (tile, threads),
                   7: "xmax pre-pass + pattern_fast_zmarch_kernel (%d-row column blocks, %d threads)" % (tile, threads),
                   8: "pattern_fast_rstaged_kernel, records in shared memory (%d-row tiles, %d threads)" % (tile, threads),
                   9: "pattern_fast_rstaged_kernel, one-byte row types (%d-row tiles, %d threads)" % (tile, threads),
                   10: "pattern_fast_zblock_kernel (512-row column blocks of %d planes, %d threads)"
                       % (tile // 512, threads),
                   11: "pattern_fast_tma_kernel (persistent z-marching, TMA-fed %d-row column blocks, %d threads)"
                       % (tile, threads)}[variant]

    def timed(M, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier(world)
        ev0.record(stream)
        for _ in range(steps):
            P.spmv_apply(M, x, y, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return ev0.elapsed_time(ev1) / steps  # ms

    # plain ELL baseline and COLUMN-order compressed (bit-exact mode)
    for _ in range(args.warmup):
        P.spmv_apply(A, x, y, stream)
    ell_ms = max_over_ranks(timed(A, max(20, min(args.steps, 400))), world)
    Ccol = P.spmv_compress(A, format="pattern", order="column")
    for _ in range(args.warmup):
        P.spmv_apply(Ccol, x, y, stream)
    col_ms = max_over_ranks(timed(Ccol, max(20, min(args.steps, 400))), world)
    del Ccol

    # headline: compressed, FAST order
    sampler = ClockSampler(local)
    sampler.start()
    t_warm = time.perf_counter()
    warm = 0
    while warm < args.warmup or time.perf_counter() - t_warm < 0.8:
        P.spmv_apply(C, x, y, stream)
        warm += 1
        if warm % 200 == 0:
            torch.cuda.synchronize()
    ms = max_over_ranks(timed(C, args.steps), world)
    clocks = sampler.stop()
    assert P.spmv_device_error(C) == 0
    y_fast = y.cpu().numpy()          # the timed product, checked against the oracle on the CPU leg

    # cold-L2 variant: each product timed alone right after writing a buffer
    # twice the size of L2 (median of 30)
    l2_bytes = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or 129 * 2 ** 20)
    flush = torch.empty(2 * l2_bytes // 4, dtype=torch.int32, device=dev)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cold = []
    for i in range(30):
        flush.fill_(i)
        c0.record(stream)
        P.spmv_apply(C, x, y, stream)
        c1.record(stream)
        c1.synchronize()
        cold.append(c0.elapsed_time(c1) * 1e3)
    del flush
    cold_us = statistics.median(cold)

    # end to end through the host-buffer entry point: x H2D, SpMV, y D2H
    hx = torch.from_numpy(x_np).pin_memory()
    hy = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_steps = max(3, min(args.steps, 300))
    for _ in range(3):
        P.spmv_apply_host(C, hx, hy)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        P.spmv_apply_host(C, hx, hy)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)

    flops = 2.0 * nnz
    value = world * flops / (ms * 1e-3) / 1e9
    peaks = measured_peaks()
    alg_bytes = nnz * 1.0 + n * 5.0 / 8.0 + 16.0 * n      # codes + pattern + x + y
    ell_alg_bytes = nnz * 12.0 + 16.0 * n                  # value + column + x + y
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    # the three bounds of a compressed product: HBM (algorithmic bytes at the
    # measured copy rate), instruction issue (the kernel's warp-instructions
    # per launch, from ncu on this source, at the sampled SM clock), and the
    # FP64 pipe a one-FMA-per-nonzero order would meet (the COLUMN order)
    props = torch.cuda.get_device_properties(dev)
    f_hz = (clocks.get("sm_mhz") or 2070.0) * 1e6
    warp_inst = profiled(kernel_id, "issue", "warp_inst")
    bounds_us = {"hbm": alg_bytes / (peaks["hbm_gbs"] * 1e9) * 1e6,
                 "issue": (warp_inst / (ISSUE_PER_SM_CLK * props.multi_processor_count * f_hz) * 1e6
                           if warp_inst else None),
                 "fp64_pipe_column_order": nnz / (FP64_FMA_PER_SM_CLK * props.multi_processor_count * f_hz) * 1e6,
                 "measured": ms * 1e3}
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64-in/out, int64 fixed-point accumulate", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rows": n, "nnz": nnz, "format": "pattern", "order": "fast",
                   "record_bytes_per_row": info_c["record_bytes"], "algorithmic_bytes_per_nnz": alg_bytes / nnz,
                   "l2": f"inputs {(info_c['format_bytes'] + 16 * n) / 1e6:.0f} MB > 129 MB L2, no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": profiled_traffic(kernel_id),
                     "kernel": kernel_desc, "kernel_id": kernel_id,
                     "algorithmic_bytes_per_launch": alg_bytes, "peak_source": peaks["source"],
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                     "bounds_us": bounds_us},
        "ell": {"gflops": world * flops / (ell_ms * 1e-3) / 1e9, "ms_per_step": ell_ms,
                "achieved_gbs": ell_alg_bytes / (ell_ms * 1e-3) / 1e9,
                "frac": ell_alg_bytes / (ell_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]},
        "compressed_column_order": {"gflops": world * flops / (col_ms * 1e-3) / 1e9, "ms_per_step": col_ms},
        "speedup_vs_ell": ell_ms / ms,
        "cold_l2": {"median_us": cold_us, "gflops": 2.0 * nnz / cold_us / 1e3, "flush_bytes": 2 * l2_bytes,
                    "launches": 30},
        "clocks": clocks,
        "e2e": {"value": world * flops / e2e_s / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n, "steps": e2e_steps},
        "gpu_launches": launches_per_step * args.steps,
        "paper_context_gflops": {"pezy_sc_ell": 11.6, "pezy_sc_data_index_table": 32.4},
    }
    if rank == 0 and world == 1 and not args.no_extras:
        # the further workloads, short runs on this GPU (rank 0 of one)
        t_ex = time.perf_counter()
        time_ms = make_timer(torch, stream)
        line["cg_192"] = bench_cg(P, torch, dev, A, C, batched=True, one_at_a_time=True)
        line["table2_192"] = bench_table2(P, torch, dev, A, x, time_ms, peaks, iters=50)
        del A, C
        line["irregular_128"] = bench_irregular(P, torch, dev, time_ms, peaks, iters=50)
        line["spmm_160"] = bench_spmm(P, torch, dev, time_ms, ks=(1, 8, 32), iters=10)
        line["ragged_24"] = bench_ragged(P, torch, dev, time_ms, iters=20)
        line["extras_seconds"] = time.perf_counter() - t_ex
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(y_check=y_fast)
    if rank == 0:
        print(json.dumps(line), flush=True)
    barrier(world)


if __name__ == "__main__":
    main()

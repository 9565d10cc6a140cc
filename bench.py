#!/usr/bin/env python
"""Throughput of the structured-matrix-approximation hot path on one GB300.

Workload: the space-time covariance matrix (Section 6.2 class; 64 time lags x
256 random points in the unit square, non-separable Gneiting covariance),
16384 x 16384, dense in HBM, block Toeplitz in time with p = 127 distinct
256 x 256 blocks.  One step = the whole path: struct_E gather -> X x3 M
(DCT-II) -> Jacobi SVD of the 127 frontal slices -> global truncation at
relative tolerance 1e-6 -> Kronecker-sum factors -> report (ranks, error,
orthogonality) -> Kronecker-sum matvec on 256 right-hand sides.

Prints ONE JSON line (rank 0).  `value` = steps per second (t-SVDM
compressions/s, each including its 256-RHS matvec); the matvec GFLOP/s and
the fp64 GPU form are reported beside it.  With --impl reference the FP64 CPU
oracle is timed on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
NSM = 152
FP32_LANES_PER_SM = 128
NRHS = 256
REL_TOL = 1e-6
# the headline metric, as the benchmark configuration names it; value = whole
# steps (compression + 256-RHS matvec) per second, the matvec GFLOP/s beside it
METRIC = "t-SVDM compressions/s + Kron-sum matvec GFLOP/s, mixed vs FP64 GPU, equal err"
# DRAM bytes (read + write) of one slice of the register-tiled Jacobi SVD at
# 256 x 256, from an ncu capture of the 15-slice case (4,164,096 B read, 0
# written); every slice moves the same bytes, so a launch moves p times this
JACOBI_DRAM_BYTES_PER_SLICE = 4164096 / 15


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def replica_throughput(t_local, steps, dist=None, device=None):
    """Whole-job throughput of N independent replicas: every rank runs `steps`
    steps; the job takes as long as its slowest rank (the max over ranks of
    the local timed total), and the value counts the steps of all ranks."""
    import torch
    world = dist.get_world_size() if dist else 1
    t = float(t_local)
    if dist:
        tt = torch.tensor([t], device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return world * steps / t, t


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        d["source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["source"] = "fallback"
    return d


def svd_flops(m, n):
    """Golub-Van Loan operation count of a full SVD (U, S, V) of an m x n
    matrix, m >= n: 4 m^2 n + 8 m n^2 + 9 n^3."""
    m, n = max(m, n), min(m, n)
    return 4 * m * m * n + 8 * m * n * n + 9 * n ** 3


def kron_matvec_flops(m, n, ell, q, nterms, nrhs):
    """Algorithmic flops of Y = sum_j D_j X C_j^T with dense m x n D_j and
    ell x q C_j, per batch of nrhs right-hand sides."""
    return nrhs * nterms * (2 * n * q * ell + 2 * m * n * ell)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------

def build_device_inputs(torch, pr, dtype, device):
    """Dense column-major A (ell m x q n) assembled on the device from the
    distinct blocks, and NRHS right-hand sides."""
    from sma_inputs import generators as G
    blocks = torch.from_numpy(pr.blocks).to(device=device, dtype=dtype)      # p, m, n
    bm = torch.from_numpy(pr.block_map.astype(np.int64)).to(device)          # ell, q
    A4 = blocks[bm]                                                          # ell, q, m, n
    At = A4.permute(1, 3, 0, 2).reshape(pr.q * pr.n, pr.ell * pr.m).contiguous()
    del A4
    A = At.t()                                                               # column-major view
    x = G.random_rhs(pr.q * pr.n, NRHS, 1)
    X = torch.from_numpy(np.ascontiguousarray(x.T)).to(device=device, dtype=dtype).t()
    Y = torch.empty(NRHS, pr.ell * pr.m, dtype=dtype, device=device).t()
    return A, X, Y


def run_gpu_form(torch, S, pr, prec, steps, warmup, device, stream, flush):
    dtype = torch.float32 if prec == S.SMA_MIXED else torch.float64
    A, X, Y = build_device_inputs(torch, pr, dtype, device)
    h = S.Handle([pr], prec=prec, decomp=S.SMA_TSVDM, rel_tol=REL_TOL,
                 stream=stream.cuda_stream, profile=True, autotune=True)
    evs = []
    with torch.cuda.stream(stream):
        for it in range(warmup + steps):
            flush.fill_(float(it))                      # evict L2 between steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            if it == warmup:
                h.profile(reset=True)
            e0.record(stream)
            h.compress([A], want_result=False)
            e1.record(stream)
            h.apply(0, X, Y)
            e2.record(stream)
            stream.synchronize()
            if it >= warmup:
                evs.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
    res = h.result(0)
    prof = h.profile(reset=True)
    ranks = h.ranks(0)
    h.close()
    del A, X, Y
    torch.cuda.empty_cache()
    comp = np.array([a for a, _ in evs])
    app = np.array([b for _, b in evs])
    return {"compress_ms": comp, "apply_ms": app, "result": res, "profile": prof,
            "ranks": ranks}


def run_batch(torch, S, steps, warmup, device, stream, flush):
    """The batched workload: 512 uneven block-tridiagonal matrices (block
    counts 16..256, block sizes 8..64) compressed by one handle from their
    distinct blocks, relative tolerance 1e-3, CUDA events per compression."""
    from sma_inputs import generators as G
    prs = G.block_tridiag_batch()
    blocks = [torch.from_numpy(np.asfortranarray(
        np.concatenate(list(pr.blocks), axis=1).astype(np.float32))).to(device) for pr in prs]
    blocks = [b.t().contiguous().t() for b in blocks]
    h = S.Handle(prs, prec=S.SMA_MIXED, rel_tol=1e-3, layout=S.SMA_INPUT_BLOCKS,
                 stream=stream.cuda_stream, autotune=True, profile=True)
    ts = []
    with torch.cuda.stream(stream):
        for it in range(warmup + steps):
            flush.fill_(float(it))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            if it == warmup:
                h.profile(reset=True)
            e0.record(stream)
            h.compress(blocks, want_result=False)
            e1.record(stream)
            stream.synchronize()
            if it >= warmup:
                ts.append(e0.elapsed_time(e1))
    res = [h.result(i) for i in range(len(prs))]
    prof = h.profile(reset=True)
    h.close()
    del blocks
    torch.cuda.empty_cache()
    ms = float(np.mean(ts))
    nslices = sum(pr.p for pr in prs)
    return {"workload": "block_tridiag_batch (512 matrices, block counts 16..256, blocks 8..64, "
                        "rel_tol 1e-3, distinct blocks in HBM)",
            "matrices": len(prs), "slices": nslices, "ms_per_compression": ms,
            "matrices_per_s": len(prs) / (ms * 1e-3), "slices_per_s": nslices / (ms * 1e-3),
            "max_rel_err": max(r["rel_err"] for r in res),
            "stage_ms": {k: v / max(steps, 1) for k, v in prof["ms"].items()},
            "launches_per_compression": int(prof["launches"]) // max(steps, 1),
            "device_status": int(np.bitwise_or.reduce([r["device_status"] for r in res]))}


def run_e2e(torch, S, pr, steps, warmup, device, stream):
    """The same step through the C ABI with HOST buffers: the library copies
    what it needs (the p representative blocks) host->device, the right-hand
    sides go up and the result comes back inside the timed region."""
    Ah = np.asfortranarray(pr.dense().astype(np.float32))
    pinned = torch.from_numpy(np.ascontiguousarray(Ah.T)).pin_memory()
    A_host = pinned.numpy().T                                 # Fortran view of pinned memory
    from sma_inputs import generators as G
    x = G.random_rhs(pr.q * pr.n, NRHS, 1).astype(np.float32)
    Xp = torch.from_numpy(np.ascontiguousarray(x.T)).pin_memory()
    Yp = torch.empty(NRHS, pr.ell * pr.m, dtype=torch.float32).pin_memory()
    X_host, Y_host = Xp.numpy().T, Yp.numpy().T
    h = S.Handle([pr], prec=S.SMA_MIXED, decomp=S.SMA_TSVDM, rel_tol=REL_TOL, autotune=True,
                 stream=stream.cuda_stream)
    times = []
    with torch.cuda.stream(stream):
        for it in range(warmup + steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.compress([A_host], want_result=True)        # report read back to the host
            h.apply(0, X_host, Y_host)                     # waits for Y on the host
            t1 = time.perf_counter()
            if it >= warmup:
                times.append(t1 - t0)
    h.close()
    h2d = pr.p * pr.m * pr.n * 4 + x.nbytes
    d2h = Y_host.nbytes + 64                               # Y and the report
    del pinned, Xp, Yp
    return float(np.mean(times)), h2d, d2h


def cpu_oracle_sample(pr, nslices=16, nrhs=4):
    """The FP64 oracle as it stands on a bounded sample of one step: the full
    gather and transform, `nslices` of the p slice SVDs and the Kronecker-sum
    matvec for `nrhs` of the NRHS right-hand sides; scaled to a full step."""
    from oracle import sma_oracle as O
    A = pr.dense()
    t0 = time.perf_counter()
    X = O.T_E(A, pr.block_map, pr.p, pr.m, pr.n)
    M = O.dct2_matrix(pr.p)
    Xh = O.mode3(X, M)
    t1 = time.perf_counter()
    for i in range(nslices):
        np.linalg.svd(Xh[:, :, i], full_matrices=False)
    t2 = time.perf_counter()
    # the matvec on the full-rank factors (every slice kept at this tolerance)
    terms = [(O.struct_E(list(M[i, :]), pr.block_map, pr.p), Xh[:, :, i]) for i in range(pr.p)]
    x = np.random.default_rng(0).standard_normal((pr.q * pr.n, nrhs))
    t3 = time.perf_counter()
    O.apply_kron(terms, x)
    t4 = time.perf_counter()
    full = (t1 - t0) + (t2 - t1) * pr.p / nslices + (t4 - t3) * NRHS / nrhs
    return full, {"gather_transform_s": t1 - t0, "svd_s_per_slice": (t2 - t1) / nslices,
                  "apply_s_per_rhs": (t4 - t3) / nrhs}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched 512-matrix workload reported beside the headline")
    ap.add_argument("--lags", type=int, default=64,
                    help="time lags T (64 = the benchmark workload; smaller for profiling)")
    ap.add_argument("--nrhs", type=int, default=256)
    args = ap.parse_args()
    global NRHS
    NRHS = args.nrhs
    if args.warmup < 3:
        args.warmup = 3

    from sma_inputs import generators as G
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pr = G.spacetime_covariance(T=args.lags)   # 256 points, T lags, p = 2T - 1
    workload = (f"spacetime_covariance_T{args.lags}_N256 ({pr.ell * pr.m}^2 block Toeplitz, "
                f"tensor {pr.m}x{pr.n}x{pr.p})")
    cfg = {"workload": workload, "ell": pr.ell, "m": pr.m, "n": pr.n, "p": pr.p,
           "rel_tol": REL_TOL, "nrhs": NRHS, "transform": "orthonormal DCT-II",
           "l2": "flushed between steps (512 MiB write)", "parallelism": "replicas",
           "slice_svd_plan": "autotuned on the first (warm-up) compression"}

    if args.impl == "reference":
        if rank != 0:
            return
        steps = []
        for _ in range(args.warmup + args.steps):
            t, _ = cpu_oracle_sample(pr)
            steps.append(t)
        t = float(np.mean(steps[args.warmup:]))
        v = 1.0 / t
        line = {"impl": "reference", "metric": METRIC,
                "value": v, "unit": "compressions/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": cfg,
                "cpu_baseline": {"value": v, "unit": "compressions/s", "cores": os.cpu_count(),
                                 "kind": "oracle",
                                 "sample": f"full gather+transform, 16 of {pr.p} slice SVDs, "
                                           "4 of 256 RHS of the matvec; scaled to a full step"},
                "e2e": {"value": v, "unit": "compressions/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    import paper_2105_01170_gb300 as S
    from paper_2105_01170_gb300 import _build
    _build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    stream = torch.cuda.Stream(device=device)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=device)

    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    clocks.start()
    mixed = run_gpu_form(torch, S, pr, S.SMA_MIXED, args.steps, args.warmup, device, stream, flush)
    clk = clocks.stop()
    step_ms = float(np.mean(mixed["compress_ms"] + mixed["apply_ms"]))
    t_total = float(np.sum(mixed["compress_ms"] + mixed["apply_ms"])) / 1e3
    value, t_total = replica_throughput(t_total, args.steps, dist, device)

    res = mixed["result"]
    prof = mixed["profile"]
    nterms = pr.p
    mv_flops = kron_matvec_flops(pr.m, pr.n, pr.ell, pr.q, nterms, NRHS)
    app_ms = float(np.mean(mixed["apply_ms"]))
    ncomp = max(prof["calls"]["gather"], 1)          # one gather stage per compression
    svd_ms = prof["ms"]["svd"] / ncomp
    svd_alg = pr.p * svd_flops(pr.m, pr.n)
    pk = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    alu_peak = NSM * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12      # TFLOP/s fp32 FMA
    achieved = svd_alg / (svd_ms * 1e-3) / 1e12
    roof = {"kernel": "jacobi_kernel<float> (per-slice SVD, one CTA per slice)",
            "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
            "frac": achieved / alu_peak,
            "traffic": (JACOBI_DRAM_BYTES_PER_SLICE * pr.p
                        if (pr.m, pr.n) == (256, 256) else None),
            "traffic_note": "dram read+write bytes per launch, ncu capture of 15 slices scaled by slices",
            "peak_note": f"fp32 FMA: {NSM} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz "
                         "(unit counts x max clock; no measured ALU peak)",
            "algorithmic": f"{pr.p} x GVL SVD count 4m^2n+8mn^2+9n^3 = {svd_alg:.3e} flop/launch",
            "launch_ms": svd_ms}

    line = {"metric": METRIC,
            "value": value, "unit": "compressions/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (bf16x3 tensor-core contractions, fp64 angles and energy sums)",
            "data": "synthetic", "config": cfg,
            "compress_ms": float(np.mean(mixed["compress_ms"])),
            "matvec": {"gflops": mv_flops / (app_ms * 1e-3) / 1e9, "ms": app_ms,
                       "flop_per_apply": mv_flops, "terms": nterms},
            "stage_ms": {k: v / ncomp for k, v in prof["ms"].items()},
            "result": {"total_rank": res["total_rank"], "rel_err": res["rel_err"],
                       "orth_defect": res["orth_defect"], "sweeps_max": res["sweeps_max"],
                       "device_status": res["device_status"]},
            "roofline": roof, "clocks": clk,
            "gpu_launches": int(prof["launches"])}
    # the matvec's tensor-core work against the measured bf16 peak: every fp32
    # multiply-add of the Kronecker-sum matvec is six bf16 products (the
    # 3-piece split), so its bf16 rate is six times its fp32-equivalent rate
    bf16_rate = 6 * mv_flops / (app_ms * 1e-3) / 1e12
    line["roofline_apply"] = {
        "kernel": "tc_mid_kernel + tc_gemm_kernel (256-RHS Kronecker-sum matvec)",
        "bound": "tensor", "achieved": bf16_rate, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
        "frac": bf16_rate / pk["bf16_tflops"],
        "frac_sustained": bf16_rate / pk["bf16_tflops_sustained"],
        "algorithmic": f"6 x {mv_flops:.3e} bf16 flop per apply (2 (n q ell + m n ell) p per RHS)",
        "peak_note": f"bf16 GEMM burst peak ({pk['source']})",
        "traffic": None,
        "traffic_note": "two kernels; the mid-index contraction writes 3.2 GB of split planes"}

    if args.fp64_steps > 0:
        f64 = run_gpu_form(torch, S, pr, S.SMA_FP64, args.fp64_steps, 1, device, stream, flush)
        f_ms = float(np.mean(f64["compress_ms"] + f64["apply_ms"]))
        line["fp64_gpu"] = {"value": 1e3 / f_ms, "unit": "compressions/s", "ms_per_step": f_ms,
                            "compress_ms": float(np.mean(f64["compress_ms"])),
                            "matvec_gflops": mv_flops / (np.mean(f64["apply_ms"]) * 1e-3) / 1e9,
                            "total_rank": f64["result"]["total_rank"],
                            "rel_err": f64["result"]["rel_err"],
                            "stage_ms": {k: v / max(f64["profile"]["calls"]["gather"], 1)
                                         for k, v in f64["profile"]["ms"].items()}}
        line["mixed_vs_fp64_speedup"] = f_ms / step_ms
        line["ranks_equal_to_fp64"] = bool(np.array_equal(f64["ranks"], mixed["ranks"]))

    if args.lags == 64 and not args.no_batch:
        line["batch"] = run_batch(torch, S, max(2, args.steps // 2), 3, device, stream, flush)

    if not args.no_e2e:
        e2e_t, h2d, d2h = run_e2e(torch, S, pr, max(2, args.steps // 2), 1, device, stream)
        line["e2e"] = {"value": 1.0 / e2e_t, "unit": "compressions/s",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank == 0 and not args.no_cpu:
        t_cpu, parts = cpu_oracle_sample(pr)
        line["cpu_baseline"] = {"value": 1.0 / t_cpu, "unit": "compressions/s",
                                "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"full gather+transform, 16 of {pr.p} slice SVDs "
                                          f"(numpy LAPACK), 4 of {NRHS} RHS of the matvec; "
                                          "scaled to a full step", "parts": parts}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

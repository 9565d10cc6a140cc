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
oracle is timed on the same workload instead (one whole oracle step per timed
step).  Beside the headline the line carries the other workloads of the
benchmark configuration under "configs" (mixed and FP64 forms on the GPU,
errors against the oracle, the oracle's own time).
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
# DRAM bytes (read + write) per slice of the rotation-log Jacobi at 256 x 256,
# from an ncu capture of the 15-slice case (4,098,560 B read: the slices and
# the block workspace; 11,086,848 B written: the rotation log, part of which
# is still in L2 at exit); every slice moves the same bytes, so a launch
# moves p times this.  The replay reads the logs of the slices with
# discarded columns only.
JACOBI_DRAM_BYTES_PER_SLICE = (4098560 + 11086848) / 15


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
    distinct blocks, relative tolerance 1e-3, CUDA events per compression;
    the compression is captured into a CUDA graph on its second call and
    replayed from then on."""
    from sma_inputs import generators as G
    prs = G.block_tridiag_batch()
    blocks = [torch.from_numpy(np.asfortranarray(
        np.concatenate(list(pr.blocks), axis=1).astype(np.float32))).to(device) for pr in prs]
    blocks = [b.t().contiguous().t() for b in blocks]
    h = S.Handle(prs, prec=S.SMA_MIXED, rel_tol=1e-3, layout=S.SMA_INPUT_BLOCKS,
                 stream=stream.cuda_stream, autotune=True, profile=True, graph=True)
    ts = []
    stage_prof = None
    with torch.cuda.stream(stream):
        for it in range(warmup + steps):
            flush.fill_(float(it))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            if it == 1:
                # stage times of the first call, which runs stage by stage
                # (the graph replays after it record no stage events)
                stage_prof = h.profile(reset=True)
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
                        "rel_tol 1e-3, distinct blocks in HBM, CUDA-graph replay)",
            "matrices": len(prs), "slices": nslices, "ms_per_compression": ms,
            "matrices_per_s": len(prs) / (ms * 1e-3), "slices_per_s": nslices / (ms * 1e-3),
            "max_rel_err": max(r["rel_err"] for r in res),
            "stage_ms_first_call": dict(stage_prof["ms"]) if stage_prof else None,
            "launches_per_compression": int(prof["launches"]) // max(steps, 1),
            "graph_replay": True,
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


# ----------------------------------------------------------------------------
# the other workloads of the benchmark configuration: each compressed (and
# applied) in the mixed and the FP64 form on the same GPU, its error against
# the FP64 oracle, and the oracle's own time on the host (measured, on the
# sample stated)
# ----------------------------------------------------------------------------

def _dev(torch, a, dtype):
    """Column-major device copy of a host matrix (or a 1-D vector)."""
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).to(device="cuda", dtype=dtype)
    return t.t() if t.dim() == 2 else t


def _timed(torch, stream, flush, fn, steps, warmup):
    """Mean device ms of fn() over `steps` calls after `warmup` calls, CUDA
    events on the handle's stream, L2 flushed before each call."""
    ts = []
    with torch.cuda.stream(stream):
        for it in range(warmup + steps):
            flush.fill_(float(it))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            stream.synchronize()
            if it >= warmup:
                ts.append(e0.elapsed_time(e1))
    return float(np.mean(ts))


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _export_T(torch, S, h, pr, prec):
    """The approximation tensor T of problem 0 (filled by sma_reconstruct)."""
    dt = torch.float64 if prec == S.SMA_FP64 else torch.float32
    Ah = torch.empty(pr.q * pr.n, pr.ell * pr.m, dtype=dt, device="cuda").t()
    h.reconstruct(0, Ah)
    del Ah
    n = h.export_size(0, S.EXPORT_T)
    buf = torch.empty(n, dtype=dt, device="cuda")
    h.export(0, S.EXPORT_T, buf)
    return buf.cpu().numpy().astype(np.float64).reshape((pr.m, pr.n, pr.p), order="F")


def _forms(torch, S, make, prec_list=None):
    """Run make(prec) for both precisions; returns {name: result dict}."""
    out = {}
    for prec in (prec_list or (S.SMA_MIXED, S.SMA_FP64)):
        out["mixed" if prec == S.SMA_MIXED else "fp64"] = make(prec)
    return out


def cfg_planted(torch, S, stream, flush, steps, alu_peak):
    """Planted Kronecker sum (block Toeplitz 128^2, 15 distinct 16 x 16
    blocks, 1e-8 noise): t-SVDM at tolerance 1e-6 and its 256-RHS matvec, and
    the block-index Tucker-1 that must find Kronecker rank 3."""
    from oracle import sma_oracle as O
    from sma_inputs import generators as G
    pr = G.planted_kron_toeplitz()
    x = G.random_rhs(pr.q * pr.n, NRHS, 1)

    def make(prec):
        dt = torch.float64 if prec == S.SMA_FP64 else torch.float32
        A = pr.dense() if prec == S.SMA_FP64 else pr.dense().astype(np.float32)
        dA, dX = _dev(torch, A, dt), _dev(torch, x, dt)
        dY = torch.empty(NRHS, pr.ell * pr.m, dtype=dt, device="cuda").t()
        h = S.Handle([pr], prec=prec, rel_tol=1e-6, stream=stream.cuda_stream)
        ms_c = _timed(torch, stream, flush, lambda: h.compress([dA], want_result=False), steps, 3)
        ms_a = _timed(torch, stream, flush, lambda: h.apply(0, dX, dY), steps, 3)
        res = h.result(0)
        X = O.T_E(np.asarray(A, np.float64), pr.block_map, pr.p, pr.m, pr.n)
        ora = O.tsvdm(X, O.dct2_matrix(pr.p), rel_tol=1e-6)
        T = _export_T(torch, S, h, pr, prec)
        yo = O.apply_kron(O.tsvdm_kron_terms(ora, pr.block_map), x.astype(np.asarray(A).dtype)
                          .astype(np.float64))
        out = {"compress_ms": ms_c, "apply_ms": ms_a, "total_rank": res["total_rank"],
               "rel_err": res["rel_err"],
               "ranks_equal_oracle": bool(np.array_equal(h.ranks(0), ora.ranks)),
               "T_rel_err_vs_oracle": _rel(T, ora.tensor_approx()),
               "apply_rel_err_vs_oracle": _rel(dY.cpu().numpy(), yo)}
        h.close()
        hk = S.Handle([pr], prec=prec, decomp=S.SMA_TUCKER_BLOCKMODE, rel_tol=1e-6,
                      stream=stream.cuda_stream)
        out["tucker1_ms"] = _timed(torch, stream, flush,
                                   lambda: hk.compress([dA], want_result=False), steps, 3)
        out["kron_rank"] = hk.result(0)["ranks"][0]
        out["kron_rank_oracle"] = O.tucker1_blockmode(X, rel_tol=1e-6).rank
        hk.close()
        return out

    forms = _forms(torch, S, make)
    t0 = time.perf_counter()
    Xo = O.T_E(pr.dense(), pr.block_map, pr.p, pr.m, pr.n)
    ora = O.tsvdm(Xo, O.dct2_matrix(pr.p), rel_tol=1e-6)
    O.apply_kron(O.tsvdm_kron_terms(ora, pr.block_map), x)
    t_or = time.perf_counter() - t0
    return {"workload": "planted Kronecker sum, block Toeplitz 8 x 8 of 16 x 16 (p = 15), "
                        "t-SVDM tol 1e-6 + 256-RHS matvec; Tucker-1 Kronecker rank",
            "forms": forms, "oracle_ms": t_or * 1e3,
            "oracle_sample": "the whole compression and 256-RHS matvec (FP64 numpy)",
            "roofline": {"bound": "latency", "note": "a 30 KB tensor: a handful of small "
                         "launches, far below any throughput roof"}}


def cfg_spacetime_blr(torch, S, stream, flush, steps, pk):
    """The space-time covariance (16384^2, 127 lag blocks of 256 x 256) in its
    block-low-rank forms: the SPSD shared-U compression at tolerance 1e-2 and
    the SPD-preserving form at rank 64, each with a 256-RHS matvec."""
    from oracle import sma_oracle as O
    from sma_inputs import generators as G
    pr = G.spacetime_covariance()
    x = G.random_rhs(pr.q * pr.n, NRHS, 1)
    out = {}

    def shared(prec):
        dt = torch.float64 if prec == S.SMA_FP64 else torch.float32
        A = pr.dense() if prec == S.SMA_FP64 else pr.dense().astype(np.float32)
        dA, dX = _dev(torch, A, dt), _dev(torch, x, dt)
        dY = torch.empty(NRHS, pr.ell * pr.m, dtype=dt, device="cuda").t()
        h = S.Handle([pr], prec=prec, decomp=S.SMA_TUCKER_SHARED_U, rel_tol=1e-2,
                     stream=stream.cuda_stream, profile=True)
        ms_c = _timed(torch, stream, flush, lambda: h.compress([dA], want_result=False),
                      max(2, steps // 2), 2)
        ms_a = _timed(torch, stream, flush, lambda: h.apply(0, dX, dY), steps, 3)
        h.profile(reset=True)
        with torch.cuda.stream(stream):
            h.compress([dA], want_result=False)
        prof = h.profile(reset=True)
        res = h.result(0)
        X = O.T_E(np.asarray(A, np.float64), pr.block_map, pr.p, pr.m, pr.n)
        su = O.shared_u(X, rel_tol=1e-2)
        T = _export_T(torch, S, h, pr, prec)
        r = res["ranks"][0]
        o = {"compress_ms": ms_c, "apply_ms": ms_a, "rank": r, "rank_oracle": su.rank,
             "ranks_equal_oracle": r == su.rank, "rel_err": res["rel_err"],
             "T_rel_err_vs_oracle": _rel(T, su.tensor_approx()),
             "trace_relerr": res["trace_relerr"], "storage_ratio": res["storage_ratio"],
             "compress_stage_ms": {k: v for k, v in prof["ms"].items() if v > 0}}
        del dA
        h.close()
        return o

    def spd(prec):
        dt = torch.float64 if prec == S.SMA_FP64 else torch.float32
        B = np.concatenate(list(pr.blocks), axis=1)
        B = B if prec == S.SMA_FP64 else B.astype(np.float32)
        dB, dX = _dev(torch, B, dt), _dev(torch, x, dt)
        dY = torch.empty(NRHS, pr.ell * pr.m, dtype=dt, device="cuda").t()
        h = S.Handle([pr], prec=prec, decomp=S.SMA_TUCKER_SPD, layout=S.SMA_INPUT_BLOCKS,
                     fixed_rank=64, stream=stream.cuda_stream)
        ms_c = _timed(torch, stream, flush, lambda: h.compress([dB], want_result=False),
                      max(2, steps // 2), 2)
        ms_a = _timed(torch, stream, flush, lambda: h.apply(0, dX, dY), steps, 3)
        res = h.result(0)
        A = pr.dense() if prec == S.SMA_FP64 else pr.dense().astype(np.float32)
        s = O.spd_preserving(np.asarray(A, np.float64), pr.block_map, pr.p, pr.m, rank=64)
        T = _export_T(torch, S, h, G.Problem("inner", s.X.transpose(2, 0, 1), s.inner_map), prec)
        o = {"compress_ms": ms_c, "apply_ms": ms_a, "rank": res["ranks"][0],
             "rel_err": res["rel_err"], "T_rel_err_vs_oracle": _rel(T, s.su.tensor_approx()),
             "storage_ratio": res["storage_ratio"]}
        h.close()
        return o

    out["shared_u_tol_1e-2"] = _forms(torch, S, shared)
    out["spd_rank_64"] = _forms(torch, S, spd)
    sh = out["shared_u_tol_1e-2"]
    out["mixed_vs_fp64_compress_speedup"] = sh["fp64"]["compress_ms"] / sh["mixed"]["compress_ms"]
    t0 = time.perf_counter()
    Xo = O.T_E(pr.dense(), pr.block_map, pr.p, pr.m, pr.n)
    O.shared_u(Xo, rel_tol=1e-2)
    out["oracle_ms"] = (time.perf_counter() - t0) * 1e3
    out["oracle_sample"] = "the shared-U compression (gather, mode-1 SVD, core) in FP64 numpy"
    out["workload"] = ("space-time covariance 16384^2 (127 lag blocks of 256 x 256): SPSD "
                       "shared-U at tol 1e-2 and SPD-preserving at rank 64, 256-RHS matvecs")
    return out


def cfg_hankel(torch, S, stream, flush, steps, alu_peak):
    """LTI block Hankel 2048^2 (64 x 64 blocks of 32 x 32, p = 127): rows-
    and-columns Tucker block low rank at r = 5, 10, 20 and the 256-RHS
    matvec."""
    from oracle import sma_oracle as O
    from sma_inputs import generators as G
    pr = G.lti_hankel()
    N = pr.ell * pr.m
    x = G.random_rhs(N, NRHS, 3)
    out = {}
    for r in (5, 10, 20):
        def make(prec, r=r):
            dt = torch.float64 if prec == S.SMA_FP64 else torch.float32
            A = pr.dense() if prec == S.SMA_FP64 else pr.dense().astype(np.float32)
            dA, dX = _dev(torch, A, dt), _dev(torch, x.astype(np.asarray(A).dtype), dt)
            dY = torch.empty(NRHS, N, dtype=dt, device="cuda").t()
            h = S.Handle([pr], prec=prec, decomp=S.SMA_TUCKER_ROWCOL, fixed_rank=r,
                         stream=stream.cuda_stream)
            ms_c = _timed(torch, stream, flush, lambda: h.compress([dA], want_result=False),
                          steps, 3)
            ms_a = _timed(torch, stream, flush, lambda: h.apply(0, dX, dY), steps, 3)
            X = O.T_E(np.asarray(A, np.float64), pr.block_map, pr.p, pr.m, pr.n)
            t = O.tucker2_rows_cols(X, r, r)
            yo = O.apply_M_E(t.tensor_approx(), pr.block_map,
                             x.astype(np.asarray(A).dtype).astype(np.float64))
            flops = 2 * 2 * (64 * 32 * r * NRHS) + 2 * 64 * 64 * r * r * NRHS
            o = {"compress_ms": ms_c, "apply_ms": ms_a,
                 "apply_rel_err_vs_oracle": _rel(dY.cpu().numpy(), yo),
                 "apply_gflops": flops / (ms_a * 1e-3) / 1e9,
                 "apply_alu_frac": flops / (ms_a * 1e-3) / 1e12 / alu_peak}
            h.close()
            return o
        out[f"r{r}"] = _forms(torch, S, make)
    t0 = time.perf_counter()
    A = pr.dense()
    X = O.T_E(A, pr.block_map, pr.p, pr.m, pr.n)
    t = O.tucker2_rows_cols(X, 10, 10)
    O.apply_M_E(t.tensor_approx(), pr.block_map, x)
    out["oracle_ms"] = (time.perf_counter() - t0) * 1e3
    out["oracle_sample"] = "r = 10: gather, both mode SVDs, core and the 256-RHS matvec (FP64 numpy)"
    out["workload"] = ("LTI block Hankel 2048^2 (64 x 64 blocks of 32 x 32), rows-and-columns "
                       "Tucker BLR at r = 5/10/20, 256-RHS matvec")
    out["roofline"] = {"bound": "latency", "kernel": "the BLR matvec's three products",
                       "note": "the core product on tcgen05 (fp16 two-piece split) from "
                               "r = 5 on, the two projections on CUDA cores; 0.1 ms per "
                               "256-RHS apply, launch- and latency-bound; apply_alu_frac is the "
                               "fp32-equivalent rate against the derived FP32 peak; the "
                               "compression is two small Gram eigen-solves (latency-bound)"}
    return out


def cfg_block_index(torch, S, stream, flush, steps):
    """One block-tridiagonal matrix of the batched kind at the size of the
    largest matrix of the paper's Kronecker-sum table (300 blocks of 32 x 32,
    p = 898 distinct blocks, Kronecker rank 5): the block-index Tucker-1 at
    rank 5 from the p x p Gram (deterministic) and from the randomized sketch
    of Section 6.3 (s = 3)."""
    from oracle import sma_oracle as O
    from sma_inputs import generators as G
    pr = G.block_tridiag_kron(300, 32)
    r, sk = 5, 3
    Om, Ps = G.gaussian_sketch(pr.m, pr.n, sk)

    def make(prec):
        dt = torch.float64 if prec == S.SMA_FP64 else torch.float32
        A = pr.dense() if prec == S.SMA_FP64 else pr.dense().astype(np.float32)
        dA = _dev(torch, A, dt)
        X = O.T_E(np.asarray(A, np.float64), pr.block_map, pr.p, pr.m, pr.n)
        t = O.tucker1_blockmode(X, rank=r)
        o = {}
        for name, kw in (("deterministic", {}), ("sketch_s3", {"sketch": (Om, Ps)})):
            h = S.Handle([pr], prec=prec, decomp=S.SMA_TUCKER_BLOCKMODE, fixed_rank=r,
                         stream=stream.cuda_stream, profile=True, **kw)
            ms = _timed(torch, stream, flush, lambda: h.compress([dA], want_result=False),
                        max(2, steps // 2), 2)
            res = h.result(0)
            o[name] = {"compress_ms": ms, "rel_err": res["rel_err"],
                       "err_vs_optimal_factor": res["tensor_err"] / max(t.err, 1e-300)}
            if name == "deterministic":
                n = h.export_size(0, S.EXPORT_FACTOR)
                buf = torch.empty(n, dtype=dt, device="cuda")
                h.export(0, S.EXPORT_FACTOR, buf)
                V = buf.cpu().numpy().astype(np.float64).reshape(pr.p, pr.p, order="F")[:, :r]
                o[name]["factor_projector_gap_vs_oracle"] = float(
                    np.linalg.norm(V @ V.T - t.V @ t.V.T, 2))
            h.close()
        return o

    out = _forms(torch, S, make)
    t0 = time.perf_counter()
    X = O.T_E(pr.dense(), pr.block_map, pr.p, pr.m, pr.n)
    O.tucker1_blockmode(X, rank=r)
    out_or = (time.perf_counter() - t0) * 1e3
    return {"workload": "block tridiagonal, 300 blocks of 32 x 32 (p = 898), Kronecker rank 5: "
                        "block-index Tucker-1 at rank 5, deterministic (898^2 Gram) and "
                        "randomized sketch (s = 3)",
            "forms": out, "oracle_ms": out_or,
            "oracle_sample": "gather and the block-index unfolding's SVD (FP64 numpy)"}


def cfg_psf(torch, S, stream, flush, steps, pk):
    """3-D Gaussian blur of a 64^3 volume (15^3 PSF, sigma 2/3/4, rotated 30
    degrees, zero boundary): the three-level HOSVD at tolerance 1e-4 and the
    matvec on 64 volumes."""
    from oracle import sma_oracle as O
    from sma_inputs import generators as G
    K, half, tol = 64, 7, 1e-4
    s_ = 2 * half + 1
    P = G.gaussian_psf3(support=s_, sig=(2.0, 3.0, 4.0))
    bm = O.banded_toeplitz_map(K, half)
    a64 = np.transpose(P, (2, 1, 0)).ravel(order="F")
    vols = G.random_volumes(64, K)
    x = np.stack([v.ravel(order="F") for v in vols], axis=1)

    def make(prec):
        dt = torch.float64 if prec == S.SMA_FP64 else torch.float32
        a = a64 if prec == S.SMA_FP64 else a64.astype(np.float32)
        xin = x if prec == S.SMA_FP64 else x.astype(np.float32)
        da, dX = _dev(torch, a, dt), _dev(torch, xin, dt)
        dY = torch.empty(64, K ** 3, dtype=dt, device="cuda").t()
        mp = S.MultilevelProblem([bm, bm, bm], [s_, s_, s_])
        h = S.Handle([mp], prec=prec, decomp=S.SMA_HOSVD_MULTILEVEL, layout=S.SMA_INPUT_BLOCKS,
                     rel_tol=tol, stream=stream.cuda_stream)
        ms_c = _timed(torch, stream, flush, lambda: h.compress([da], want_result=False), steps, 3)
        ms_a = _timed(torch, stream, flush, lambda: h.apply(0, dX, dY), steps, 3)
        res = h.result(0)
        Pin = np.transpose(np.asarray(a, np.float64).reshape((s_, s_, s_), order="F"), (2, 1, 0))
        ho = O.hosvd3(O.psf_tensor(Pin, K), rel_tol=tol)
        Gc, C1, C2, C3 = O.multilevel_kron_terms(ho, K, half)
        yo = O.multilevel_apply(Gc, C1, C2, C3, np.asarray(vols[:1], np.float64)
                                .astype(np.float32 if prec == S.SMA_MIXED else np.float64)
                                .astype(np.float64))[0].ravel(order="F")
        y0 = dY[:, 0].cpu().numpy()
        hbm = 2 * 64 * K ** 3 * (8 if prec == S.SMA_FP64 else 4)
        o = {"compress_ms": ms_c, "apply_ms": ms_a, "ranks": res["ranks"][:3],
             "ranks_oracle": list(ho.ranks), "ranks_equal_oracle": list(res["ranks"][:3]) ==
             list(ho.ranks), "rel_err": res["rel_err"],
             "apply_rel_err_vs_oracle_1_volume": _rel(y0, yo),
             "apply_hbm_gbs": hbm / (ms_a * 1e-3) / 1e9,
             "apply_hbm_frac": hbm / (ms_a * 1e-3) / 1e9 / pk["hbm_gbs"]}
        h.close()
        return o

    out = _forms(torch, S, make)
    t0 = time.perf_counter()
    ho = O.hosvd3(O.psf_tensor(P, K), rel_tol=tol)
    Gc, C1, C2, C3 = O.multilevel_kron_terms(ho, K, half)
    t1 = time.perf_counter()
    O.multilevel_apply(Gc, C1, C2, C3, vols[:1])
    t2 = time.perf_counter()
    return {"workload": "3-D blur 64^3 (15^3 PSF, sigma 2/3/4, rotated 30 degrees), three-level "
                        "HOSVD tol 1e-4, 64-volume matvec",
            "forms": out, "oracle_ms": ((t1 - t0) + (t2 - t1) * 64) * 1e3,
            "oracle_sample": f"HOSVD {1e3 * (t1 - t0):.1f} ms + the matvec on 1 of the 64 "
                             f"volumes ({1e3 * (t2 - t1):.1f} ms) x 64",
            "roofline": {"bound": "hbm", "kernel": "the three-level matvec",
                         "note": "apply_hbm_frac: 2 x 64 volumes read and written once against "
                                 "the measured HBM copy bandwidth"}}


def cfg_batch_fp64(torch, S, stream, flush, steps):
    """The 512-matrix batch in the FP64 form, and the oracle on a sample of
    its problems (ranks and error against the mixed and FP64 GPU forms)."""
    from oracle import sma_oracle as O
    from sma_inputs import generators as G
    prs = G.block_tridiag_batch()
    out = {}
    for prec in (S.SMA_FP64, S.SMA_MIXED):
        dt = torch.float64 if prec == S.SMA_FP64 else torch.float32
        blocks = [_dev(torch, np.concatenate(list(pr.blocks), axis=1)
                       .astype(np.float64 if prec == S.SMA_FP64 else np.float32), dt) for pr in prs]
        h = S.Handle(prs, prec=prec, rel_tol=1e-3, layout=S.SMA_INPUT_BLOCKS,
                     stream=stream.cuda_stream, autotune=True)
        ms = _timed(torch, stream, flush, lambda: h.compress(blocks, want_result=False),
                    max(1, steps // 4), 1)
        sample = [0, 17, 300]
        cmp = []
        for i in sample:
            pr = prs[i]
            B = blocks[i].cpu().numpy().astype(np.float64).reshape(pr.m, pr.n, pr.p, order="F")
            X = B * np.sqrt(O.multiplicities(pr.block_map, pr.p))[None, None, :]
            ora = O.tsvdm(X, O.dct2_matrix(pr.p), rel_tol=1e-3)
            r = h.result(i)
            cmp.append({"problem": i, "ranks_equal_oracle": bool(np.array_equal(h.ranks(i), ora.ranks)),
                        "err_rel_diff": abs(r["tensor_err"] - ora.err) / max(ora.err, 1e-300)})
        out["fp64" if prec == S.SMA_FP64 else "mixed"] = {"ms_per_compression": ms,
                                                          "sampled_vs_oracle": cmp}
        h.close()
        del blocks
        torch.cuda.empty_cache()
    return out


def oracle_step(pr, nslices=None, nrhs=None):
    """One step of the FP64 oracle as it stands: gather, transform, the slice
    SVDs, the global truncation, the Kronecker-sum terms and the matvec on
    the right-hand sides.  With nslices / nrhs a bounded sample: only that
    many of the p slice SVDs and of the NRHS right-hand sides (the truncation
    then runs on the sampled slices).  Returns the measured seconds of each
    part."""
    from oracle import sma_oracle as O
    A = pr.dense()
    ns = pr.p if nslices is None else nslices
    nr = NRHS if nrhs is None else nrhs
    t0 = time.perf_counter()
    X = O.T_E(A, pr.block_map, pr.p, pr.m, pr.n)
    M = O.dct2_matrix(pr.p)
    Xh = O.mode3(X, M)
    t1 = time.perf_counter()
    facs = [np.linalg.svd(Xh[:, :, i], full_matrices=False) for i in range(ns)]
    t2 = time.perf_counter()
    ranks = O.truncate_global([f[1] for f in facs], REL_TOL, float(np.sum(X * X)))
    terms = []
    for i in range(ns):
        u, sv, vt = facs[i]
        r = int(ranks[i])
        if r > 0:
            terms.append((O.struct_E(list(M[i, :]), pr.block_map, pr.p),
                          (u[:, :r] * sv[:r]) @ vt[:r, :]))
    t3 = time.perf_counter()
    x = np.random.default_rng(0).standard_normal((pr.q * pr.n, nr))
    O.apply_kron(terms, x)
    t4 = time.perf_counter()
    return {"gather_transform_s": t1 - t0, "svd_s": t2 - t1, "truncate_terms_s": t3 - t2,
            "apply_s": t4 - t3, "slices": ns, "rhs": nr, "total_s": t4 - t0}


def oracle_single_thread(pr, nslices, nrhs):
    """The same sample in a child process whose BLAS and OpenMP pools are
    limited to one thread (the pools are sized when numpy loads)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(nslices), str(nrhs),
           "--lags", str(pr.ell)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_rate(parts, pr):
    """Compressions per second of the full step implied by a sample: the
    gather and transform as measured, the SVD, truncation/terms and matvec
    parts scaled from the sampled slices and right-hand sides."""
    fs = pr.p / parts["slices"]
    fr = NRHS / parts["rhs"]
    full = (parts["gather_transform_s"] + (parts["svd_s"] + parts["truncate_terms_s"]) * fs +
            parts["apply_s"] * fr)
    return 1.0 / full, {"slice_scale": fs, "rhs_scale": fr, "full_step_s": full}


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
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (planted Kronecker sum, the space-time "
                         "BLR forms, block Hankel, the FP64 batch, 3-D blur)")
    ap.add_argument("--oracle-sample", type=int, nargs=2, metavar=("SLICES", "RHS"),
                    help="(internal) time one bounded oracle step and print its parts")
    args = ap.parse_args()
    global NRHS
    NRHS = args.nrhs
    if args.warmup < 3:
        args.warmup = 3
    if args.oracle_sample:
        from sma_inputs import generators as G
        prs = G.spacetime_covariance(T=args.lags)
        print(json.dumps(oracle_step(prs, *args.oracle_sample)), flush=True)
        return

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
        # the FP64 oracle as it stands, one whole step (every slice SVD, the
        # truncation, the Kronecker terms and all 256 right-hand sides) per
        # timed step, on the host's cores; ranks other than 0 exit at once
        if rank != 0:
            return
        steps = []
        for _ in range(args.warmup + args.steps):
            steps.append(oracle_step(pr)["total_s"])
        t = float(np.mean(steps[args.warmup:]))
        v = 1.0 / t
        sample = (f"one whole step per timed step: gather + transform, all {pr.p} slice SVDs "
                  f"(numpy LAPACK), the global truncation, the Kronecker terms and the matvec "
                  f"on all {NRHS} RHS; numpy's default BLAS threading")
        line = {"impl": "reference", "metric": METRIC,
                "value": v, "unit": "compressions/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": cfg,
                "cpu_baseline": {"value": v, "unit": "compressions/s", "cores": os.cpu_count(),
                                 "kind": "oracle", "sample": sample},
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
    roof = {"kernel": "jacobi_kernel<float> rotation-log form + jacobi_v_replay_kernel "
                      "(the slice-SVD step: one CTA per slice, then the columns of V the "
                      "rebuild reads)",
            "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
            "frac": achieved / alu_peak,
            "traffic": (JACOBI_DRAM_BYTES_PER_SLICE * pr.p
                        if (pr.m, pr.n) == (256, 256) and JACOBI_DRAM_BYTES_PER_SLICE else None),
            "traffic_note": "dram read+write bytes of the Jacobi launch (the replay reads the "
                            "logs of the slices with discarded columns), ncu capture of 15 "
                            "slices scaled by slices",
            "peak_note": f"fp32 FMA: {NSM} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz "
                         "(unit counts x max clock; no measured ALU peak)",
            "algorithmic": f"{pr.p} x GVL SVD count 4m^2n+8mn^2+9n^3 = {svd_alg:.3e} flop/launch",
            "launch_ms": svd_ms}

    line = {"metric": METRIC,
            "value": value, "unit": "compressions/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (split-precision tensor-core contractions: bf16x3 transform, fp16x2 matvec; fp64 angles and energy sums)",
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
    # multiply-add of the Kronecker-sum matvec is three fp16 products (the
    # scaled two-piece split hi hi + hi lo + lo hi), so its fp16 rate is three
    # times its fp32-equivalent rate; the dense fp16 rate equals the bf16 one
    f16_rate = 3 * mv_flops / (app_ms * 1e-3) / 1e12
    line["roofline_apply"] = {
        "kernel": "tc_mid_kernel + tc_gemm_kernel (256-RHS Kronecker-sum matvec)",
        "bound": "tensor", "achieved": f16_rate, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
        "frac": f16_rate / pk["bf16_tflops"],
        "frac_sustained": f16_rate / pk["bf16_tflops_sustained"],
        "algorithmic": f"3 x {mv_flops:.3e} fp16 flop per apply (2 (n q ell + m n ell) p per RHS)",
        "peak_note": f"bf16 GEMM burst peak ({pk['source']}) x 1: dense fp16 and bf16 rates are equal",
        "traffic": None,
        "traffic_note": "two kernels; the mid-index contraction writes 2.1 GB of split planes"}

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

    if args.lags == 64 and not args.no_configs:
        cfgs = {}
        jobs = [("1_planted_kron", lambda: cfg_planted(torch, S, stream, flush, args.steps,
                                                       alu_peak)),
                ("2_spacetime_blr", lambda: cfg_spacetime_blr(torch, S, stream, flush,
                                                              args.steps, pk)),
                ("3_lti_hankel", lambda: cfg_hankel(torch, S, stream, flush, args.steps,
                                                    alu_peak)),
                ("4_batch_forms", lambda: cfg_batch_fp64(torch, S, stream, flush, args.steps)),
                ("4b_block_index_factor", lambda: cfg_block_index(torch, S, stream, flush,
                                                                  args.steps)),
                ("5_psf_blur", lambda: cfg_psf(torch, S, stream, flush, args.steps, pk))]
        for name, job in jobs:
            try:
                cfgs[name] = job()
            except Exception as e:          # report, keep the headline line
                cfgs[name] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()
        line["configs"] = cfgs

    if rank == 0 and not args.no_cpu:
        full = oracle_step(pr)
        single = oracle_single_thread(pr, 16, 4)
        cb = {"value": 1.0 / full["total_s"], "unit": "compressions/s",
              "cores": os.cpu_count(), "kind": "oracle",
              "sample": (f"one whole oracle step (all {pr.p} slice SVDs, truncation, terms, "
                         f"{NRHS}-RHS matvec) on all host cores, measured"),
              "parts": full}
        if single is not None:
            rate1, scale = oracle_rate(single, pr)
            cb["single_thread"] = {"value": rate1, "unit": "compressions/s", "cores": 1,
                                   "sample": f"16 of {pr.p} slice SVDs and 4 of {NRHS} RHS in "
                                             "a one-thread child process, scaled by the "
                                             "factors given", "scale": scale, "parts": single}
        line["cpu_baseline"] = cb
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

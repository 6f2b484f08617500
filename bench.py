"""Throughput of the screened mixed-precision Lasso solve on one GB300 (or N, weak scaling).

Workload (one step): the batched mixed-precision configuration -- a dense 2048 x 8192 FP32
dictionary with unit atoms, 4096 signals y_i = A x0_i with Bernoulli(p_i) x0, p_i ~ U[0.01, 0.05],
lambda_i / lambda_max,i ~ U[0.1, 0.9], solved to relative duality gap 1e-6 over the ladder
FP8 (per-atom scaled E4M3) -> BF16 -> FP32 (exact), every signal certified by the full-dictionary
gap.  A solve counts when its certified gap is <= tol.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--signals B]
N > 1 runs under torchrun, one rank per GPU, each rank solving its own 4096 signals.
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Lasso solves/sec at rel. gap 1e-6: screened mixed-prec vs plain FISTA, GB/s"
UNIT = "solves/s"
TOL = 1e-6


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--signals", type=int, default=4096)
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--config", default="c3", choices=["c1", "c2", "c3", "c4", "c5"],
                    help="workload: c3 (default, the headline batched mixed-precision line) or c1 / c2 / c4 / c5")
    ap.add_argument("--grid", action="store_true",
                    help="run the Section V parameter grid instead (T/T_N, F/F_N per point)")
    ap.add_argument("--grid-families", default="gaussian,kron,faust,example,combos",
                    help="comma list of grid families: gaussian, kron, faust, example (Section IV's worked "
                         "example), combos (ISTA / FISTA x GAP / Dynamic Safe, single versus multiple "
                         "approximations)")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_first(rank, signals_per_rank):
    """First global signal index of a rank's shard: ranks solve disjoint, equally sized slices of
    one seeded batch (signal i depends only on (seed, i)), so the job needs no data exchange."""
    return rank * signals_per_rank


def job_totals(t_local, solved_local, device):
    """Whole-job time (max over ranks) and solves (sum over ranks); one rank returns its own."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t_local), int(solved_local)
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    n = torch.tensor([float(solved_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(n.item()))


def _peaks():
    """(HBM GB/s, BF16 TF/s burst, BF16 TF/s sustained, source) from MEASURED_PEAKS.json, else the
    pool's fallback figures."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return (d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0),
                d.get("bf16_tflops_sustained", d.get("bf16_tflops", 1700.0)), "measured")
    return 6800.0, 1900.0, 1700.0, "fallback"


# FP32 / FP64 SIMT peaks derived from GB300's unit counts and maximum clock (not measured): 152 SMs x
# 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz; FP64 at 1/64 of the FP32 rate on this part.
SIMT_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
SIMT_FP64_TFLOPS = SIMT_FP32_TFLOPS / 64


def _workload_config(B):
    return {"workload": f"c3 batched mixed precision: dense 2048x8192 FP32 dictionary (unit atoms), {B} signals "
                        "per GPU, x0 Bernoulli(p_i) p_i~U[0.01,0.05], lambda_i/lambda_max~U[0.1,0.9], rel gap 1e-6",
            "N": 2048, "K": 8192, "signals_per_gpu": B,
            "ladder": ["fp8_e4m3_atom_scaled", "bf16", "split_bf16_pair_on_tensor_cores", "f32_exact"],
            "tol": TOL, "stopping_certificate": "full-dictionary duality gap bound (rounding folded in)",
            "l2": "flushed between timed steps (512 MB write)"}


# ----------------------------------------------------------------------------- CPU oracle leg

def _oracle_rate(w, seconds, max_signals=64):
    """Oracle (FP64 numpy Algorithm 1, same ladder) on the first signals until `seconds` pass."""
    from oracle import dictionaries as OD
    from oracle import lasso as OL
    from oracle import solvers as OS
    A = w.A
    f8, _, _ = OD.fp8_quantize(A)
    levels = [OD.dense_level("fp8", f8, A, 0.25), OD.dense_level("bf16", OD.bf16_round(A), A, 0.5),
              OD.exact_level(A)]
    Lip = OD.power_iteration_sq_norm(levels[-1].op, iters=50) * 1.01
    t0 = time.perf_counter()
    n = 0
    while n < min(max_signals, w.Y.shape[0]) and time.perf_counter() - t0 < seconds:
        y = w.Y[n]
        Aty = A.T @ y
        lam = w.lam_ratio[n] * OL.lambda_max(Aty)
        r = OS.fast_l1(levels, levels[-1].atnorm, y, lam, TOL, Gamma=0.5, Lip=Lip, Aty=Aty)
        n += int(r.converged)
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    import synthetic as S
    w = S.c3(n_signals=64)
    times, solved = [], 0
    for _ in range(args.warmup):
        pass   # the oracle has no warm state; warm-up steps are empty
    per_step = max(5.0, min(60.0, 150.0 / max(1, args.steps)))
    for _ in range(args.steps):
        rate, n, dt = _oracle_rate(w, per_step)
        times.append(dt)
        solved += n
    tot = sum(times)
    value = solved / tot if tot > 0 else 0.0
    sample = f"first signals of the c3 batch, about {per_step:.0f} s of oracle work per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _workload_config(4096),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- comparator

def plain_fista(A_t, Y, lam, L, tol, max_iter=3000, check_every=10):
    """Plain FP32 FISTA without screening (torch FP32 GEMMs, TF32 off), gap checked every
    `check_every` passes with FP64 scalars; returns (#signals below tol, seconds, passes)."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    B, N = Y.shape
    K = A_t.shape[0]
    X = torch.zeros((B, K), device=Y.device)
    Zc = torch.zeros_like(X)
    t = 1.0
    yy = (Y.double() ** 2).sum(1)
    lam_c = lam.float()[:, None]
    done = torch.zeros(B, dtype=torch.bool, device=Y.device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it = 0
    for it in range(1, max_iter + 1):
        R = Y - Zc @ A_t                      # B x N
        G = R @ A_t.T                         # B x K
        if it % check_every == 0:
            rr = (R.double() ** 2).sum(1)
            yr = (Y.double() * R.double()).sum(1)
            m = G.abs().max(1).values.double()
            beta = yr / (lam * rr)
            s = torch.clamp(beta, -1.0 / m, 1.0 / m)
            P = 0.5 * rr + lam * Zc.double().abs().sum(1)
            D = lam * s * yr - 0.5 * lam * lam * s * s * rr
            done |= (P - D) / yy <= tol
            if bool(done.all()):
                break
        Xn = Zc + G / L
        Xn = torch.sign(Xn) * torch.clamp(Xn.abs() - lam_c / L, min=0.0)
        tn = 0.5 * (1.0 + (1.0 + 4.0 * t * t) ** 0.5)
        Zc = Xn + ((t - 1.0) / tn) * (Xn - X)
        X, t = Xn, tn
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    # the rate of the comparator's two products (B x K @ K x N and B x N @ N x K), CUDA events
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(2):
        Zc @ A_t
        R @ A_t.T
    ev[0].record()
    for _ in range(5):
        Zc @ A_t
    ev[1].record()
    for _ in range(5):
        R @ A_t.T
    ev[2].record()
    ev[2].synchronize()
    ms1, ms2 = ev[0].elapsed_time(ev[1]) / 5, ev[1].elapsed_time(ev[2]) / 5
    flops = 2.0 * B * N * K
    gemm = {"residual_gemm_ms": ms1, "correlation_gemm_ms": ms2,
            "residual_gemm_tflops": flops / (ms1 * 1e-3) / 1e12, "correlation_gemm_tflops": flops / (ms2 * 1e-3) / 1e12,
            "flops_per_gemm": flops, "dtype": "f32 (TF32 off)"}
    return int(done.sum()), secs, it, gemm


def _l2_peak_gbs():
    """Measured read bandwidth of data resident in L2 (48 MiB read 50 times in one launch with
    16-byte loads that bypass L1; the library's probe), best of 3."""
    import ctypes as C
    from paper_1812_06635_gb300 import _native
    lib = _native.load()
    best = 0.0
    for _ in range(3):
        v = C.c_double()
        if lib.lasso_probe_l2_read(48 << 20, 50, C.byref(v)) == 0:
            best = max(best, v.value)
    return best


def _code_hash(scope):
    """sha256 prefix of the code a kernel is compiled from, comments, blank lines and indentation
    left out.
    `scope` lists files; a file with an "until" marker counts only up to it (its kernel's
    translation unit up to the end of the kernel, where everything the kernel calls is defined)."""
    h = hashlib.sha256()
    for item in scope:
        t = open(os.path.join(ROOT, item["file"]), encoding="utf-8").read()
        if item.get("until"):
            i = t.find(item["until"])
            if i < 0:
                return None
            t = t[:i]
        t = re.sub(r"/\*.*?\*/", "", t, flags=re.S)
        t = re.sub(r"//[^\n]*", "", t)
        h.update("\n".join(ln.strip() for ln in t.splitlines() if ln.strip()).encode())
    return h.hexdigest()[:16]


def _traffic(kind):
    """Per-launch DRAM bytes of the dominant kernel on this workload from the committed ncu
    summary, if the kernel's code has not changed since (hash recorded with the counters)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p)).get(kind)
        if _code_hash(d["scope"]) != d["code_sha256_16"]:
            return None
        return d["dram_bytes_per_launch"]
    except (KeyError, OSError, TypeError, ValueError, AttributeError):
        return None


def _c3_roofline(kms, kbytes, klaunch, level_atoms, N):
    """Roofline block of the batched mixed-precision workload, for its dominant kernel.

    The dominant kernel is the correlation pass (kernel kind 1), whose dense contraction is the
    exact level's g = A_[A]^T rho over each signal's preserved atoms (the BF16 / FP8 levels are
    correlated by the tensor-core GEMM, kind 5, and only gathered by this pass).  Its algorithmic
    work is 2 N flops per (signal, preserved atom) on the exact level -- level_atoms[exact] counts
    those products over the timed steps -- and the graded bound is the tensor pipe's sustained
    BF16 rate.  Diagnostics: the same pass as algorithmic bytes against the L2 read bandwidth
    measured in this run and against the HBM copy rate (the dictionary stays in L2 across the
    batch, so the HBM figure can exceed 1), the derived FP32 SIMT rate, and the tensor-core stage
    as algorithmic TF/s (2 N K per signal on its level)."""
    hbm, bf16, bf16_s, src = _peaks()
    names = ["k_residual", "k_corr", "k_screen", "k_schedule", "k_structured", "k_tc_gemm"]
    corr_s = kms[1] * 1e-3
    exact = int(np.max(np.flatnonzero(level_atoms))) if level_atoms.any() else 0
    flops = 2.0 * N * level_atoms[exact]
    tf = flops / corr_s / 1e12 if corr_s > 0 else 0.0
    launches = max(1.0, klaunch[1])
    roof = {"bound": "tensor", "achieved": tf, "peak": bf16_s, "unit": "TFLOP/s", "frac": tf / bf16_s,
            "traffic": _traffic("k_corr_pass@c3"), "kernel": "k_corr_pass (exact-level correlation + update)",
            "peak_source": f"{src} bf16_tflops_sustained (MEASURED_PEAKS.json)",
            "algorithmic_flops_per_launch": flops / launches, "avg_launch_us": 1e6 * corr_s / launches,
            "work": "2 N |A_t| flops per signal-pass on the exact level (preserved atoms only)",
            "kernel_share": {names[i]: kms[i] / max(1e-9, kms.sum()) for i in range(6) if kms[i] > 0},
            "why_this_kernel": "the correlation, the step the C3 measurement grades; the residual pass and the "
                               "evaluation + screening group take similar shares of the step (kernel_share)"}
    gbps = kbytes[1] / corr_s / 1e9 if corr_s > 0 else 0.0
    l2 = _l2_peak_gbs()
    diag = {
        "l2": {"achieved": gbps, "peak": l2, "unit": "GB/s", "frac": gbps / l2 if l2 else None,
               "peak_source": "measured in this run (lasso_probe_l2_read: a 48 MiB L2-resident buffer read 50 "
                              "times with L1-bypassing 16-byte loads, best of 3)",
               "algorithmic_bytes_per_launch": kbytes[1] / launches},
        "hbm": {"achieved": gbps, "peak": hbm, "unit": "GB/s", "frac": gbps / hbm,
                "note": "algorithmic bytes; the dictionary is read from L2, not DRAM"},
        "simt_fp32": {"achieved": tf, "peak": SIMT_FP32_TFLOPS, "unit": "TFLOP/s", "frac": tf / SIMT_FP32_TFLOPS,
                      "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"},
        "kernels_GBps": {names[i]: kbytes[i] / (kms[i] * 1e-3) / 1e9 for i in range(5)
                         if kms[i] > 0 and kbytes[i] > 0}}
    if roof["traffic"] and kbytes[1] > 0:
        # DRAM bytes (ncu) over algorithmic bytes per launch: rows shared by signals hit in L2
        diag["l2"]["dram_traffic_over_algorithmic"] = roof["traffic"] / (kbytes[1] / launches)
    # the whole correlation stage of a pass (every level: tensor-core GEMMs and the gather pass),
    # algorithmic work 2 N |A_t| per signal-pass on each level
    st_s = (kms[1] + kms[5]) * 1e-3
    if st_s > 0:
        fl = 2.0 * N * float(np.sum(level_atoms))
        diag["correlation_stage"] = {"achieved": fl / st_s / 1e12, "peak": bf16_s, "unit": "TFLOP/s",
                                     "frac": fl / st_s / 1e12 / bf16_s,
                                     "kernels": "k_tc_corr (FP8, BF16, split levels) + k_quant_rho + k_corr_pass",
                                     "work": "2 N |A_t| flops per signal-pass on every level"}
    if kms[5] > 0:
        tc = kbytes[5] / (kms[5] * 1e-3) / 1e12
        diag["tensor_stage"] = {"achieved": tc, "peak": bf16, "unit": "TFLOP/s", "frac": tc / bf16,
                                "kernel": "k_tc_corr (+ k_quant_rho)",
                                "peak_source": "bf16_tflops burst (MEASURED_PEAKS.json); FP8 launches counted "
                                               "against the same BF16 figure",
                                "work": "executed: 2 N K per signal-pass on a tensor-core level, three times on "
                                        "the split level (a1 r1 + a1 r2 + a2 r1)",
                                "algorithmic_flops_per_launch": kbytes[5] / max(1.0, klaunch[5] / 2)}
    return roof, diag


# ----------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    import synthetic as S
    import paper_1812_06635_gb300 as pkg
    from paper_1812_06635_gb300 import build
    build.build()
    pkg.load()

    B = args.signals
    w = S.c3(n_signals=B, first=shard_first(rank, B))
    d = pkg.Dictionary.dense(w.A, dtype="f32").add_level(pkg.LEVEL_FP8).add_level(pkg.LEVEL_BF16).prepare()
    Y = torch.tensor(w.Y, dtype=torch.float32, device=dev)
    ratios = torch.tensor(w.lam_ratio, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(profile=0):
        return d.solve_batch(Y, ratios, TOL, stream=stream, lambda_relative=1, profile=profile)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    total_ms, solved, kms, kbytes, klaunch, launches = 0.0, 0, np.zeros(6), np.zeros(6), np.zeros(6), 0
    level_atoms = np.zeros(8)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        X, gaps, status, iters, st = step(profile=1)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        solved += int(((status == 0) & (gaps <= TOL)).sum())
        kms += np.array(st.kernel_ms)
        kbytes += np.array(st.kernel_bytes)
        klaunch += np.array(st.kernel_launches)
        level_atoms += np.array(st.level_atoms)
        launches += st.launches
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    t_job, solved_job = job_totals(total_ms / 1e3, solved, dev)
    value = solved_job / t_job

    # e2e: the same solve through the C ABI with pinned host buffers, copies included
    Yh = torch.empty(Y.shape, dtype=torch.float32, pin_memory=True)
    Yh.copy_(Y)
    lh = torch.empty(B, dtype=torch.float64, pin_memory=True)
    lh.copy_(ratios)
    Xh = torch.empty((B, w.K), dtype=torch.float32, pin_memory=True).numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xo, go, so, st_e2e = d.solve_batch_host(Yh.numpy(), lh.numpy(), TOL, lambda_relative=1)
    e2e_s = time.perf_counter() - t0
    e2e_solved = int(((so == 0) & (go <= TOL)).sum())
    del Xh

    roofline, roofline_diag = _c3_roofline(kms, kbytes, klaunch, level_atoms, w.N)

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            rate, n, dt = _oracle_rate(S.c3(n_signals=64), args.cpu_seconds)
            cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"{n} signals of c3 solved by the FP64 numpy oracle (same ladder) in {dt:.1f} s "
                             "(numpy BLAS threads on all host cores)"}
        comp = None
        if not args.no_comparator:
            A_t = torch.tensor(w.A.T, dtype=torch.float32, device=dev).contiguous()   # K x N
            lam = ratios * d.lambda_max(Y)
            info = d.info()
            nsolved, secs, its, gemm = plain_fista(A_t, Y, lam, info["L"], TOL)
            comp = {"impl": "plain FP32 unscreened FISTA (torch FP32 GEMM, TF32 off, gap every 10 passes)",
                    "value": nsolved / secs, "unit": UNIT, "solved": nsolved, "signals": B, "seconds": secs,
                    "passes": its, "ms_per_pass": 1e3 * secs / max(1, its), "gemm": gemm,
                    "simt_fp32_peak_tflops": SIMT_FP32_TFLOPS}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": _workload_config(B),
                "solved_per_step": solved / args.steps, "signals_per_step": B * world,
                "e2e": {"value": e2e_solved / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(B * w.N * 4 + B * 8),
                        "d2h_bytes_per_step": int(B * w.K * 4 + B * 8 + B * 4)},
                "gpu_launches": int(launches), "roofline": roofline, "roofline_diagnostics": roofline_diag,
                "autotuned": {"corr_chunk": st.corr_chunk, "corr_blocks_per_sm": st.corr_blocks_per_sm,
                              "level_rc": [round(v, 5) for v in st.level_rc if v]},
                "fp64_resolved_per_step": st.fp64_resolved,
                "cpu_baseline": cpu, "comparator": comp,
                "clocks": clk, "passes_max": st.passes,
                "ladder": ["fp8", "bf16"] + (["split_bf16_tc"] if st.level_passes[3] else []) + ["f32_exact"],
                "level_passes_per_signal": [v / B for v in st.level_passes if v],
                "level_atom_passes_per_signal": [v / B for v in st.level_atoms if v]}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    d.close()
    return 0


# ----------------------------------------------------------------------------- the other configs

CONFIGS = {
    "c1": "c1 plain FP64: dense 100x500 Gaussian (unit atoms), x0 25-sparse, y = A x0 + N(0, 0.01^2), "
          "lambda = 0.5 lambda_max, exact GAP Safe, rel gap 1e-8, single signal",
    "c2": "c2 structured: sum of 4 Kronecker terms of 32x64 factors (N=1024, K=4096, unit atoms), ladder R=1 -> R=2 "
          "-> exact, x0 Bernoulli(0.02), 20 dB, lambda/lambda_max in {0.3, 0.5, 0.8} x 25 realisations, rel gap 1e-6",
    "c4": "c4 differentiation: dense 1024x4096 FP32 (unit atoms), 256 signals, lambda = 0.5 lambda_max, x0 and "
          "x_target Bernoulli(0.02), 20 dB; forward solve to rel gap 1e-6 then the support adjoint dL/dy, dL/dA",
    "c5": "c5 large structured: sum of 8 Kronecker terms, B_r 64x256, C_r 128x256 (N=8192, K=65536), ladder R=1 -> "
          "R=2 -> R=4 -> FP8 -> exact, 512 signals, x0 Bernoulli(0.005), lambda/lambda_max~U[0.2,0.7], rel gap 1e-6",
}


def _timed_steps(fn, steps, warmup, stream, flush):
    """W warm-up calls, then K calls each preceded by an L2 flush and bracketed by CUDA events on
    `stream`; returns (total ms, [per-step results]) with nvidia-smi clocks sampled meanwhile."""
    import torch
    for _ in range(max(3, warmup)):
        fn()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    total, outs = 0.0, []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs.append(fn())
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    return total, outs, clocks.stop()


def _kron_flops(st, levels_R, N1, K1, N2, K2):
    """Algorithmic flops of the Kronecker products of a solve: each pass on a level with R terms
    forms one product and one adjoint product, R * 2 (N1 K1 K2 + N1 K2 N2) flops each."""
    per = 2.0 * (N1 * K1 * K2 + N1 * K2 * N2)
    return sum(2.0 * R * per * st.level_passes[i] for i, R in enumerate(levels_R))


def run_config(args):
    """One JSON line for config c1, c2, c4 or c5 (same metric and contract as the default line)."""
    import torch
    import synthetic as S
    import paper_1812_06635_gb300 as pkg
    from paper_1812_06635_gb300 import build
    build.build()
    pkg.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    cfg = args.config
    hbm, bf16, bf16_s, src = _peaks()
    extra, cpu = {}, None
    if cfg == "c1":
        from oracle import lasso as OL
        from oracle import solvers as OS
        tol, reps = 1e-8, 25
        w = S.c1()
        d = pkg.Dictionary.dense(w.A, dtype="f64").prepare()
        Y = torch.tensor(w.Y[:1], dtype=torch.float32, device=dev)
        ratio = torch.tensor([0.5], dtype=torch.float64, device=dev)

        def fn():
            return [d.solve_batch(Y, ratio, tol, stream=stream, lambda_relative=1) for _ in range(reps)]
        ms, outs, clk = _timed_steps(fn, args.steps, args.warmup, stream, flush)
        runs = [r for o in outs for r in o]
        solved = sum(int(((r[2] == 0) & (r[1] <= tol)).sum()) for r in runs)
        launches = sum(r[4].launches for r in runs)
        passes = float(np.mean([r[4].passes for r in runs]))
        value, unit_work = solved / (ms * 1e-3), len(runs)
        t0 = time.perf_counter()
        for _ in range(reps):
            x, gap, kept, _st = d.solve(w.Y[0], 0.5, tol, lambda_relative=1)
        e2e = {"value": reps / (time.perf_counter() - t0), "unit": UNIT, "h2d_bytes_per_step": 8 * 100 + 8,
               "d2h_bytes_per_step": 8 * 500 + 8 + 4 * 500, "api": "lasso_solve (host FP64 y)"}
        us = 1e3 * ms / len(runs)
        roof = {"bound": "latency", "achieved": us, "peak": None, "unit": "us/solve", "frac": None, "traffic": None,
                "note": "100 x 500 FP64 (400 KB, L2-resident): one signal's passes are a chain of small launches; "
                        "no roofline claim", "passes_per_solve": passes}
        if not args.no_cpu_baseline:
            A, y = w.A, w.Y[0]
            lam = 0.5 * OL.lambda_max(A.T @ y)
            t0, n = time.perf_counter(), 0
            while time.perf_counter() - t0 < min(args.cpu_seconds, 10.0):
                OS.fista_gap_safe(A, y, lam, tol, max_iter=400000)
                n += 1
            dt = time.perf_counter() - t0
            cpu = {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"the c1 signal solved {n} times by the FP64 numpy oracle (FISTA + GAP Safe) in {dt:.1f} s"}
        d.close()
    elif cfg in ("c2", "c5"):
        from oracle import dictionaries as OD
        from oracle import lasso as OL
        from oracle import solvers as OS
        if cfg == "c2":
            ws = [S.c2(seed=0, lam_ratio=r, n_signals=25) for r in (0.3, 0.5, 0.8)]
            levels_R, Rtot = [1, 2], 4
        else:
            ws = [S.c5()]
            levels_R, Rtot = [1, 2, 4], 8
        w = ws[0]
        d = pkg.Dictionary.kron(w.Bf, w.Cf)
        for R in levels_R:
            d.add_level(pkg.LEVEL_KRON, R)
        if cfg == "c5":
            d.add_level(pkg.LEVEL_FP8)
        d.prepare()
        Ys = [torch.tensor(x.Y, dtype=torch.float32, device=dev) for x in ws]
        rs = [torch.tensor(x.lam_ratio, dtype=torch.float64, device=dev) for x in ws]

        def fn():
            return [d.solve_batch(Y, r, TOL, stream=stream, lambda_relative=1, profile=1) for Y, r in zip(Ys, rs)]
        ms, outs, clk = _timed_steps(fn, args.steps, args.warmup, stream, flush)
        runs = [r for o in outs for r in o]
        solved = sum(int(((r[2] == 0) & (r[1] <= TOL)).sum()) for r in runs)
        launches = sum(r[4].launches for r in runs)
        value, unit_work = solved / (ms * 1e-3), sum(int(Y.shape[0]) for Y in Ys) * args.steps
        kms = np.sum([r[4].kernel_ms for r in runs], axis=0)
        kb = np.sum([r[4].kernel_bytes for r in runs], axis=0)
        kl = np.sum([r[4].kernel_launches for r in runs], axis=0)
        _, N1, K1 = w.Bf.shape
        _, N2, K2 = w.Cf.shape
        kflops = sum(_kron_flops(r[4], levels_R, N1, K1, N2, K2) for r in runs)
        names = ["k_residual", "k_corr", "k_screen", "k_schedule", "k_structured", "k_tc_gemm"]
        share = {names[i]: kms[i] / max(1e-9, kms.sum()) for i in range(6) if kms[i] > 0}
        tf = kflops / (kms[4] * 1e-3) / 1e12 if kms[4] > 0 else 0.0
        structured = {"achieved": tf, "unit": "TFLOP/s", "frac_of_bf16_sustained": tf / bf16_s,
                      "frac_of_simt_fp32": tf / SIMT_FP32_TFLOPS, "simt_fp32_peak_derived": SIMT_FP32_TFLOPS,
                      "kernel": "k_kron_gemm + k_kron_scatter (structured products of the R-term levels)",
                      "work": "per pass on an R-term level: product and adjoint, R * 2 (N1 K1 K2 + N1 K2 N2) flops "
                              "each", "share": share.get("k_structured", 0.0)}
        if int(np.argmax(kms)) == 1 and cfg == "c5":
            # the exact level's correlation pass over the preserved atoms dominates: a gather of
            # 32 KB FP32 rows of the 2 GiB dense exact level, which does not fit in L2
            gbps = kb[1] / (kms[1] * 1e-3) / 1e9
            roof = {"bound": "hbm", "achieved": gbps, "peak": hbm, "unit": "GB/s", "frac": gbps / hbm,
                    "traffic": None, "kernel": "k_corr_pass (exact-level correlation + update)",
                    "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)",
                    "work": "per signal-pass: |A_t| (4 N + 24) bytes of preserved rows and iterates + 4 N of rho",
                    "algorithmic_bytes_per_launch": kb[1] / max(1.0, kl[1]),
                    "avg_launch_us": 1e3 * kms[1] / max(1.0, kl[1]), "kernel_share": share}
        else:
            roof = {"bound": "tensor", "achieved": tf, "peak": bf16_s, "unit": "TFLOP/s", "frac": tf / bf16_s,
                    "traffic": None, "kernel": structured["kernel"],
                    "peak_source": f"{src} bf16_tflops_sustained (MEASURED_PEAKS.json)",
                    "work": structured["work"], "kernel_share": share}
        extra["structured_products"] = structured
        extra["dominant_kernel"] = names[int(np.argmax(kms))]
        extra["level_passes_per_signal"] = (np.sum([r[4].level_passes for r in runs], axis=0) / unit_work).tolist()
        extra["fp64_resolved_per_step"] = sum(r[4].fp64_resolved for r in runs) / args.steps
        if kms[5] > 0:
            extra["tensor_stage_tflops"] = kb[5] / (kms[5] * 1e-3) / 1e12
        # e2e through the host-buffer call
        t0 = time.perf_counter()
        e2e_solved = 0
        for x in ws:
            X, g, st_, _ = d.solve_batch_host(x.Y.astype(np.float32), x.lam_ratio, TOL, lambda_relative=1)
            e2e_solved += int(((st_ == 0) & (g <= TOL)).sum())
        dt = time.perf_counter() - t0
        nb = sum(x.Y.shape[0] for x in ws)
        e2e = {"value": e2e_solved / dt, "unit": UNIT, "h2d_bytes_per_step": int(nb * (w.Y.shape[1] * 4 + 8)),
               "d2h_bytes_per_step": int(nb * (K1 * K2 * 4 + 12)), "api": "lasso_solve_batch_host"}
        if not args.no_cpu_baseline:
            # the oracle's structured ladder (Algorithm 1 with FP64 Kronecker operators), signal after
            # signal of the same batches, for about --cpu-seconds (each signal capped in passes)
            dsc = 1.0 / S.gen.kron_column_norms(w.Bf, w.Cf)
            levs = [OD.kron_level(w.Bf, w.Cf, dsc, R) for R in levels_R] + [OD.kron_level(w.Bf, w.Cf, dsc, Rtot)]
            Lip = OD.power_iteration_sq_norm(levs[-1].op, iters=30) * 1.01
            cap = 2000 if cfg == "c5" else 100000
            t0 = time.perf_counter()
            n_ok, n_try = 0, 0
            for x in ws:
                for b in range(x.Y.shape[0]):
                    if time.perf_counter() - t0 > args.cpu_seconds:
                        break
                    y = x.Y[b]
                    Aty = levs[-1].op.rmatvec(y)
                    lam = float(x.lam_ratio[b]) * OL.lambda_max(Aty)
                    r = OS.fast_l1(levs, levs[-1].atnorm, y, lam, TOL, Lip=Lip, Aty=Aty, max_iter=cap)
                    n_try += 1
                    n_ok += int(r.converged)
            dt = time.perf_counter() - t0
            cpu = {"value": n_ok / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"{n_ok} of {n_try} signals of the {cfg} batches certified by the FP64 numpy oracle "
                             f"(structured ladder, at most {cap} passes each) in {dt:.1f} s"}
        d.close()
    elif cfg == "c4":
        from oracle import backward as OB
        w = S.c4()
        d = pkg.Dictionary.dense(w.A, dtype="f32").prepare()
        Y = torch.tensor(w.Y, dtype=torch.float32, device=dev)
        r = torch.tensor(w.lam_ratio, dtype=torch.float64, device=dev)
        xt = torch.tensor(w.x_target, dtype=torch.float32, device=dev)
        bw = {"ms": 0.0, "n": 0, "support": []}

        def fn():
            X, gaps, status, iters, st = d.solve_batch(Y, r, TOL, stream=stream, lambda_relative=1)
            G = 2.0 * (X - xt)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dY, dA = d.backward(Y, X, G)
            e1.record(stream)
            e1.synchronize()
            bw["ms"] += e0.elapsed_time(e1)
            bw["n"] += 1
            bw["support"] = (X != 0).sum(1).double().cpu().numpy()
            return status, gaps, st
        ms, outs, clk = _timed_steps(fn, args.steps, args.warmup, stream, flush)
        B, N = w.Y.shape
        solved = sum(int(((o[0] == 0) & (o[1] <= TOL)).sum()) for o in outs)
        launches = sum(o[2].launches + 3 for o in outs)
        value, unit_work = solved / (ms * 1e-3), B * args.steps
        bw_ms = bw["ms"] / bw["n"]
        Sz = bw["support"]
        bflops = float(np.sum(N * Sz ** 2 + Sz ** 3 / 3.0 + 2.0 * N * Sz))
        tfb = bflops / (bw_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": tfb, "peak": SIMT_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": tfb / SIMT_FP64_TFLOPS, "traffic": None, "kernel": "k_backward (FP64 Gram, Cholesky, dy, dA)",
                "peak_source": "derived FP64 SIMT rate: 152 SMs x 128 lanes x 2 flop x 2.07 GHz / 64",
                "work": "per signal: Gram N|S|^2, Cholesky |S|^3/3, dA 2N|S| flops",
                "backward_us_per_signal": 1e3 * bw_ms / B, "support_mean": float(np.mean(Sz))}
        extra["backward_ms_per_batch"] = bw_ms
        t0 = time.perf_counter()
        X, g, st_, _ = d.solve_batch_host(w.Y.astype(np.float32), w.lam_ratio, TOL, lambda_relative=1)
        Xd = torch.tensor(X, device=dev)
        dY, dA = d.backward(Y, Xd, 2.0 * (Xd - xt))
        dYh = dY.cpu().numpy()
        e2e = {"value": int(((st_ == 0) & (g <= TOL)).sum()) / (time.perf_counter() - t0), "unit": UNIT,
               "h2d_bytes_per_step": int(B * (N * 4 + 8) + B * w.A.shape[1] * 4 * 2),
               "d2h_bytes_per_step": int(B * (w.A.shape[1] * 4 + 12) + dYh.nbytes),
               "api": "lasso_solve_batch_host, then lasso_backward"}
        if not args.no_cpu_baseline:
            from oracle import lasso as OL
            from oracle import solvers as OS
            t0, n = time.perf_counter(), 0
            while n < B and time.perf_counter() - t0 < args.cpu_seconds:
                y = w.Y[n]
                lam = 0.5 * OL.lambda_max(w.A.T @ y)
                rr = OS.fista_gap_safe(w.A, y, lam, TOL, max_iter=200000)
                OB.support_adjoint(w.A, y, rr.x, OB.target_loss(rr.x, w.x_target[n])[1])
                n += 1
            dt = time.perf_counter() - t0
            cpu = {"value": n / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"{n} c4 signals: FP64 oracle solve + support adjoint in {dt:.1f} s"}
        d.close()
    else:
        raise SystemExit(f"unknown config {cfg}")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if cfg == "c1" else "f32", "data": "synthetic",
            "config": {"workload": CONFIGS[cfg], "name": cfg, "l2": "flushed between timed steps (512 MB write)"},
            "solved_per_step": solved / args.steps, "signals_per_step": unit_work / args.steps,
            "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "cpu_baseline": cpu, "clocks": clk}
    line.update(extra)
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- Section V grid

def run_grid(args):
    """The experiments' parameter pool (Section V) on synthetic inputs of their size (N = 2500,
    K = 10000, unit-norm y, x Bernoulli(0.02)-Gaussian, 25 realisations solved as one batch):
    lambda / lambda_max log-spaced in [1e-2, 1], tol in {1e-3, 1e-6}, FISTA / ISTA, GAP / Dynamic Safe,
    Gamma in {0.01, 0.1, 0.8}; fast dictionaries: the FP8 -> BF16 precision ladder of a Gaussian A, and
    Kronecker truncations (R = 1, 2 of 4 terms) of structured dictionaries with term decay 0.3 / 0.5 / 0.7;
    and the source-localisation setting of Section VI on its synthetic stand-in (204 x 8193, 50 signals
    of 8 active sources, lambda = 0.1 lambda_max) with four sparse-factor product levels, or only the
    finest one.  Each line reports T / T_N, the batch time over that of the same engine without screening on the
    exact dictionary (the paper's normalisation), and F / F_N, the atom work weighted by each level's
    relative complexity over that of the unscreened exact solve.  One JSON line per grid point."""
    import torch
    import synthetic as S
    import paper_1812_06635_gb300 as pkg
    from paper_1812_06635_gb300 import build
    build.build()
    pkg.load()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ratios_grid = [0.01, 0.03, 0.1, 0.3, 0.7]
    NO_SCREEN = 1 << 30

    warmed = set()

    def timed(d, Y, lam, tol, **kw):
        if (id(d), int(Y.shape[0])) not in warmed:           # warm once per dictionary and batch size
            d.solve_batch(Y, lam, tol, **kw)                  # (tuning, workspace)
            warmed.add((id(d), int(Y.shape[0])))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        X, gaps, status, iters, st = d.solve_batch(Y, lam, tol, **kw)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, st, int(((status == 0) & (gaps <= tol)).sum())

    def work(st, rc):
        return sum(st.level_atoms[i] * rc[i] for i in range(len(rc)))

    def point(family, d, d_exact, rc, Y, lmax, ratio, tol, algo=0, rule=0, Gamma=0.5, screened_exact=False,
              single=None):
        lam = torch.full((Y.shape[0],), ratio, dtype=torch.float64, device=dev) * lmax
        T, st, ok = timed(d, Y, lam, tol, algo=algo, rule=rule, Gamma=Gamma)
        TN, stn, okn = timed(d_exact, Y, lam, tol, algo=algo, rule=rule, screen_every=NO_SCREEN)
        F, FN = work(st, rc), float(d_exact.K) * sum(stn.level_passes)
        line = {"grid": {"dictionary": family, "lambda_ratio": ratio, "tol": tol, "algo": ["FISTA", "ISTA"][algo],
                         "rule": ["GAP", "DST", "STATIC"][rule], "Gamma": Gamma, "signals": int(Y.shape[0])},
                "T_ms": 1e3 * T, "T_N_ms": 1e3 * TN, "T/T_N": T / TN, "F/F_N": F / max(FN, 1.0),
                "solved": ok, "solved_N": okn, "passes_max": st.passes, "passes_max_N": stn.passes,
                "level_passes_per_signal": [v / Y.shape[0] for v in st.level_passes[:len(rc)]]}
        if screened_exact:
            # the same screening on the exact dictionary alone (the paper's conventional-screening curve)
            TS, sts, oks = timed(d_exact, Y, lam, tol, algo=algo, rule=rule)
            line.update({"T_S_ms": 1e3 * TS, "T_S/T_N": TS / TN, "solved_S": oks})
        if single is not None:
            # a single approximation before the exact dictionary (the paper's single-approximation curve)
            d1, rc1 = single
            T1, st1, ok1 = timed(d1, Y, lam, tol, algo=algo, rule=rule, Gamma=Gamma)
            line.update({"T_single_ms": 1e3 * T1, "T_single/T_N": T1 / TN, "F_single/F_N": work(st1, rc1) / max(FN, 1.0),
                         "solved_single": ok1})
        print(json.dumps(line), flush=True)

    fams = set(args.grid_families.split(","))

    if "example" in fams:
        # Section IV's example: four approximations with RC = 0.15 (i + 1) (SuKro truncations to 5, 10,
        # 15 and 20 terms of a 25-term sum, 0.03 per term), Gamma = 0.2, lambda / lambda_max = 0.2
        we = S.paper_kron(0.85, n_signals=25, R=25)
        Ye = torch.tensor(we.Y, dtype=torch.float32, device=dev)
        de = pkg.Dictionary.kron(we.Bf, we.Cf)
        for R in (5, 10, 15, 20):
            de.add_level(pkg.LEVEL_KRON, R)
        de.prepare()
        dex = pkg.Dictionary.kron(we.Bf, we.Cf).prepare()
        info = de.info()
        print(json.dumps({"example": {"rc": info["rc"], "eps_mean": info["eps_mean"], "eps_max": info["eps_max"]}}),
              flush=True)
        lme = de.lambda_max(Ye)
        point("example-sukro25-decay0.85", de, dex, info["rc"], Ye, lme, 0.2, 1e-6, Gamma=0.2, screened_exact=True)
        de.close()
        dex.close()
    if "combos" in fams:
        # single versus multiple approximations (Section V-B): FISTA / ISTA x GAP / Dynamic Safe on the
        # moderate scenario, tol 1e-5, Gamma 0.5; multiple: R = 1, 2 truncations; single: R = 2 only
        wm = S.paper_kron(0.5, n_signals=25)
        Ym = torch.tensor(wm.Y, dtype=torch.float32, device=dev)
        dm = pkg.Dictionary.kron(wm.Bf, wm.Cf).add_level(pkg.LEVEL_KRON, 1).add_level(pkg.LEVEL_KRON, 2).prepare()
        d1 = pkg.Dictionary.kron(wm.Bf, wm.Cf).add_level(pkg.LEVEL_KRON, 2).prepare()
        dmx = pkg.Dictionary.kron(wm.Bf, wm.Cf).prepare()
        rcm, rc1 = dm.info()["rc"], d1.info()["rc"]
        lmm = dm.lambda_max(Ym)
        for algo in (0, 1):
            for rule in (0, 1):
                for ratio in (0.01, 0.1, 0.3, 0.7):
                    point("kron-decay0.5", dm, dmx, rcm, Ym, lmm, ratio, 1e-5, algo=algo, rule=rule, Gamma=0.5,
                          screened_exact=True, single=(d1, rc1))
        dm.close()
        d1.close()
        dmx.close()
    if not fams & {"faust", "gaussian", "kron"}:
        return 0

    if "faust" in fams:
        # the source-localisation stand-in: four sparse-factor levels, or only the finest one
        wf = S.meg_faust(n_signals=50)
        Yf = torch.tensor(wf.Y, dtype=torch.float32, device=dev)
        dfx = pkg.Dictionary.dense(wf.A, dtype="f32").prepare()
        lmf = dfx.lambda_max(Yf)
        for name, levels in (("meg-faust4", wf.levels), ("meg-faust1", wf.levels[-1:])):
            df = pkg.Dictionary.dense(wf.A, dtype="f32")
            for facs in levels:
                df.add_faust_level(facs)
            df.prepare()
            rcf = df.info()["rc"]
            for tol in (1e-3, 1e-6):
                point(name, df, dfx, rcf, Yf, lmf, 0.1, tol, screened_exact=True)
            for ratio in (0.03, 0.3):
                point(name, df, dfx, rcf, Yf, lmf, ratio, 1e-6, screened_exact=True)
            df.close()
        dfx.close()
    if "gaussian" not in fams and "kron" not in fams:
        return 0
    if "gaussian" not in fams:
        return _grid_kron(point, pkg, S, dev, ratios_grid)
    # Gaussian dictionary with the precision ladder
    w = S.paper_dense(n_signals=25)
    Y = torch.tensor(w.Y, dtype=torch.float32, device=dev)
    d = pkg.Dictionary.dense(w.A, dtype="f32").add_level(pkg.LEVEL_FP8).add_level(pkg.LEVEL_BF16).prepare()
    d_exact = pkg.Dictionary.dense(w.A, dtype="f32").prepare()
    rc = d.info()["rc"]
    lmax = d.lambda_max(Y)
    for tol in (1e-3, 1e-6):
        for ratio in ratios_grid:
            point("gaussian+fp8/bf16", d, d_exact, rc, Y, lmax, ratio, tol)
    for G in (0.01, 0.1, 0.8):
        point("gaussian+fp8/bf16", d, d_exact, rc, Y, lmax, 0.1, 1e-6, Gamma=G)
    point("gaussian+fp8/bf16", d, d_exact, rc, Y, lmax, 0.1, 1e-6, algo=1)
    point("gaussian+fp8/bf16", d, d_exact, rc, Y, lmax, 0.1, 1e-6, rule=1)
    d.close()
    d_exact.close()
    if "kron" in fams:
        return _grid_kron(point, pkg, S, dev, ratios_grid)
    return 0


def _grid_kron(point, pkg, S, dev, ratios_grid):
    """Grid points of the structured dictionaries: three error profiles of the Kronecker terms."""
    import torch
    for decay in (0.3, 0.5, 0.7):
        wk = S.paper_kron(decay, n_signals=25)
        Yk = torch.tensor(wk.Y, dtype=torch.float32, device=dev)
        dk = pkg.Dictionary.kron(wk.Bf, wk.Cf).add_level(pkg.LEVEL_KRON, 1).add_level(pkg.LEVEL_KRON, 2).prepare()
        dkx = pkg.Dictionary.kron(wk.Bf, wk.Cf).prepare()
        rck = dk.info()["rc"]
        lm = dk.lambda_max(Yk)
        for ratio in ratios_grid:
            point(f"kron-decay{decay}", dk, dkx, rck, Yk, lm, ratio, 1e-6)
        dk.close()
        dkx.close()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.grid:
        return run_grid(args)
    if args.config != "c3":
        return run_config(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

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
    ap.add_argument("--grid", action="store_true",
                    help="run the Section V parameter grid instead (T/T_N, F/F_N per point)")
    ap.add_argument("--grid-families", default="gaussian,kron,faust",
                    help="comma list of grid families: gaussian, kron, faust")
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
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


def _workload_config(B):
    return {"workload": f"c3 batched mixed precision: dense 2048x8192 FP32 dictionary (unit atoms), {B} signals "
                        "per GPU, x0 Bernoulli(p_i) p_i~U[0.01,0.05], lambda_i/lambda_max~U[0.1,0.9], rel gap 1e-6",
            "N": 2048, "K": 8192, "signals_per_gpu": B, "ladder": ["fp8_e4m3_atom_scaled", "bf16", "f32_exact"],
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
    return int(done.sum()), time.perf_counter() - t0, it


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


def _traffic(kind):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu summary, if the
    kernel source has not changed since (hash recorded with the counters)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p)).get(kind)
        src = open(os.path.join(ROOT, d["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != d["sha256_16"]:
            return None
        return d["dram_bytes_per_launch"]
    except (KeyError, OSError, TypeError, ValueError):
        return None


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

    # roofline of the dominant kernel (algorithmic bytes / its event-timed duration)
    hbm, bf16, peak_src = _peaks()
    kind = int(np.argmax(kms))
    names = ["k_residual", "k_corr", "k_screen", "k_schedule", "k_structured", "k_tc_gemm"]
    achieved = kbytes[kind] / (kms[kind] * 1e-3) / 1e9 if kms[kind] > 0 else 0.0
    per_launch_bytes = kbytes[kind] / max(1.0, klaunch[kind])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": _traffic(names[kind]), "kernel": names[kind],
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                "algorithmic_bytes_per_launch": per_launch_bytes,
                "avg_launch_us": 1e3 * kms[kind] / max(1.0, klaunch[kind]),
                "kernel_share": {names[i]: kms[i] / max(1e-9, kms.sum()) for i in range(6) if kms[i] > 0},
                "kernels_GBps": {names[i]: kbytes[i] / (kms[i] * 1e-3) / 1e9 for i in range(6)
                                 if kms[i] > 0 and kbytes[i] > 0 and i != 5}}
    roofline["note"] = ("algorithmic bytes count every signal's own reads of its preserved atoms; the "
                        "dictionary stays in L2 across the batch, so DRAM traffic is far below them and the "
                        "HBM fraction can exceed 1 (see roofline_l2)")
    l2 = _l2_peak_gbs()
    roofline_l2 = {"bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s", "frac": achieved / l2,
                   "kernel": names[kind],
                   "peak_source": "measured in this run: one launch reading a 48 MiB L2-resident buffer 50 "
                                  "times with L1-bypassing 16-byte loads (lasso_probe_l2_read), best of 3"}
    # the tensor-core stage (quantisation + tcgen05 correlation of the FP8 / BF16 levels)
    roofline_tc = None
    if kms[5] > 0:
        tflops = kbytes[5] / (kms[5] * 1e-3) / 1e12
        roofline_tc = {"bound": "tensor", "achieved": tflops, "peak": bf16, "unit": "TFLOP/s",
                       "frac": tflops / bf16, "kernel": "k_tc_corr (+ k_quant_rho)",
                       "peak_source": "measured bf16 (MEASURED_PEAKS.json bf16_tflops); FP8 passes counted "
                                      "against the same BF16 peak",
                       "algorithmic_flops_per_launch": kbytes[5] / max(1.0, klaunch[5] / 2)}

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
            nsolved, secs, its = plain_fista(A_t, Y, lam, info["L"], TOL)
            comp = {"impl": "plain FP32 unscreened FISTA (torch FP32 GEMM, TF32 off, gap every 10 passes)",
                    "value": nsolved / secs, "unit": UNIT, "solved": nsolved, "signals": B, "seconds": secs,
                    "passes": its}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": _workload_config(B),
                "solved_per_step": solved / args.steps, "signals_per_step": B * world,
                "e2e": {"value": e2e_solved / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(B * w.N * 4 + B * 8),
                        "d2h_bytes_per_step": int(B * w.K * 4 + B * 8 + B * 4)},
                "gpu_launches": int(launches), "roofline": roofline, "roofline_l2": roofline_l2,
                "roofline_tensor": roofline_tc,
                "autotuned": {"corr_chunk": st.corr_chunk, "corr_blocks_per_sm": st.corr_blocks_per_sm},
                "fp64_resolved_per_step": st.fp64_resolved,
                "cpu_baseline": cpu, "comparator": comp,
                "clocks": clk, "passes_max": st.passes,
                "level_passes_per_signal": [v / B for v in st.level_passes[:3]],
                "level_atom_passes_per_signal": [v / B for v in st.level_atoms[:3]]}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    d.close()
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

    def timed(d, Y, lam, tol, **kw):
        d.solve_batch(Y, lam, tol, **kw)                     # warm (tuning, workspace)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        X, gaps, status, iters, st = d.solve_batch(Y, lam, tol, **kw)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, st, int(((status == 0) & (gaps <= tol)).sum())

    def work(st, rc):
        return sum(st.level_atoms[i] * rc[i] for i in range(len(rc)))

    def point(family, d, d_exact, rc, Y, lmax, ratio, tol, algo=0, rule=0, Gamma=0.5, screened_exact=False):
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
            # the same screening on the exact dictionary alone (the paper's GAP Safe FISTA curve)
            TS, sts, oks = timed(d_exact, Y, lam, tol, algo=algo, rule=rule)
            line.update({"T_S_ms": 1e3 * TS, "T_S/T_N": TS / TN, "solved_S": oks})
        print(json.dumps(line), flush=True)

    fams = set(args.grid_families.split(","))

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
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

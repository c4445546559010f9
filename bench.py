#!/usr/bin/env python
"""Benchmark: preconditioned MINRES (ABAC preconditioner) on the 2-D L1 time-fractional workload.

Workload: L1 scheme, gamma = 0.7, N = 1024 time steps, m = 255 (M = 65,025 = 255^2, 5-point
Laplacian), 66,585,600 unknowns, f ~ U[-1, 1] (seed 2), tolerance 1e-8 relative residual.
A step is one whole solve through the C ABI: the per-alpha preconditioner set-up (tables rebuilt
every step), the entry transform, the MINRES iterations, the exit transform and the FP64 true
residual.  Metric: unknown-iterations/s = n * iterations / solve time.

Forms timed, each with its time to solution at relres <= 1e-8 (the deciding number when forms
need different iteration counts):
  * f32_precond: the FP32 preconditioner (alpha = 1e-2), the double-float matvec and entry/exit
    DSTs, FP64 Lanczos recurrences and true residual, DST basis.  `value` is this form's
    unknown-iterations/s (the precision form the metric compares with the plain FP64 one);
  * plain_f64: alpha = 1e-8 (the paper's rule), everything native FP64;
  * f32x2_precond: the double-float preconditioner at alpha = 1e-6 with the double-float matvec;
  * f32_physical: f32_precond in the physical basis (DSTs inside every preconditioner apply);
  * tc: f32_precond with the opt-in tensor-core time product.
`fastest_form` names the form with the shortest time to solution.

Every vector is 533 MB (> 129 MB L2), so no L2 flush is needed between steps.

Multi-GPU (torchrun, N > 1): independent replicas, one solve per rank per step (weak scaling);
torch.distributed is used only for the barrier and the max-over-ranks time.

--impl reference: the CPU oracle, as it stands, timed on the host cores: each step is one
MINRES iteration's operator work (one Y A z and one P_alpha^{-1} apply) on the full workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "frac2d_N1024_m255_g0.7"
TOL = 1e-8
ALPHA_F64 = 1e-8          # the paper's alpha rule (Sec. 5.2)
# FP32 preconditioner: alpha raised so that the FP32 rounding, amplified by kappa(D_alpha) =
# alpha^{-(N-1)/N}, costs no MINRES iteration against the FP64 oracle at the same alpha (6 and 6
# on this workload; at alpha = 1e-3 the oracle needs 4 and the FP32 form 6)
ALPHA_F32 = 1e-2
ALPHA_F32X2 = 1e-6        # double-float preconditioner: 2 iterations, as the FP64 oracle at 1e-6
# DRAM bytes (read + write) per unknown of one launch, from one ncu capture of the current kernel
# on the full workload
NCU_TRAFFIC_PER_UNKNOWN = {
    "conv_df": (15.38, "ncu dram__bytes_read.sum + dram__bytes_write.sum of one full-size launch "
                       "(547.2 + 477.0 MB over 66,585,600 unknowns; one pass)"),
}
# one metric text for both arms (the GPU solve and the CPU oracle), so that their lines compare
METRIC = "unknown-iterations/s to relres<=1e-8"
FP64_PEAK_TFLOPS = 1.259  # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (measured 1.20 at 1995 MHz)
FP32_PEAK_TFLOPS = 80.6   # 128 FFMA/clk/SM x 152 SMs x 2.07 GHz (measured 69.8 at 1995 MHz)
FP32_PEAK_TOPS = 40.28    # FP32 pipe: 128 instructions/clk/SM x 152 SMs x 2.07 GHz


# FP32 operations of the double-float arithmetic as the kernels implement it (common.cuh): a sum
# inside an FFT pass is a two-sum plus the trailing parts (8 operations, not renormalised), a
# twiddle product a dot product of two such products (16), a renormalised sum 11, a renormalised
# complex product 38.  One complex point, per pass:
DF_ADD_NR, DF_CMUL_NR, DF_ADD, DF_CMUL = 8.0, 32.0, 11.0, 38.0
R4_PASS = (8 * 2 * DF_ADD_NR + 3 * DF_CMUL_NR) / 4          # one length-4 DFT + 3 twiddles / 4 pts
R8_PASS = (2 * 8 * 2 * DF_ADD_NR + 2 * DF_CMUL_NR + 8 * 2 * DF_ADD_NR + 7 * DF_CMUL_NR) / 8
R8_HALF = (2 * 8 * 2 * DF_ADD_NR + 2 * DF_CMUL_NR + 4 * 2 * DF_ADD_NR + 7 * DF_CMUL_NR) / 8


def df_fft_ops(L, skip_radix2=False, half_out=False):
    """FP32 operations per complex point of one double-float FFT of length L as planned by the
    512-thread tiles: radix 2 only when the caller applied it (skip_radix2: free), one or two
    radix-4 passes, radix-8 passes for the rest; half_out: the last radix-8 pass forms half of
    its outputs."""
    lg = int(np.log2(L))
    rem = lg - (1 if (lg % 2 and skip_radix2) else 0)
    n4 = 1 if rem % 3 == 2 else (2 if rem % 3 == 1 else 0)
    n8 = (rem - 2 * n4) // 3
    ops = n4 * R4_PASS + n8 * R8_PASS
    if half_out and n8 > 0:
        ops += R8_HALF - R8_PASS
    return ops


def df_conv_ops(N):
    """FP32 operations per unknown of the double-float matvec in the DST basis: the forward FFT of
    2N (its first radix-2 pass is the zero padding's copy), the common spectral product, the
    inverse FFT forming the first N outputs, the scaled load (one double-float product)."""
    return df_fft_ops(2 * N, skip_radix2=True) + DF_CMUL + df_fft_ops(2 * N, half_out=True) + 7.0


def df_timepass_ops(N):
    """FP32 operations per unknown of the double-float time pass: four FFTs of N per complex
    column (two real modes), two split spectral products (per frequency pair: four renormalised
    complex sums and two complex products), the three row scalings."""
    ffts = 4 * df_fft_ops(N) / 2
    prods = 2 * (4 * 2 * DF_ADD + 2 * DF_CMUL) / 2 / 2
    return ffts + prods + 3 * 7.0


def df_dst_ops(m):
    """FP32 operations per unknown of the double-float DST-I of length m: one complex FFT of
    P = m + 1 per two lines, the pre-pass and the split (two renormalised complex sums and two
    scalings per row pair and column), the prefix sum, the scaled read-out."""
    P = m + 1
    fft = P * df_fft_ops(P) / (2 * m)
    pre = P / 2 * (4 * 2 * DF_ADD + 2 * 2 * 7.0) / (2 * m)
    split = P / 2 * (2 * 2 * DF_ADD + 2 * 2 * 7.0) / (2 * m)
    prefix = P / 2 * 2 * 2 * DF_ADD / (2 * m)
    return fft + pre + split + prefix + 7.0


def peaks():
    p = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            j = json.load(fh)
        p["hbm_gbs"] = float(j["hbm_gbs"])
        p["bf16_tflops"] = float(j["bf16_tflops"])
        p["source"] = "measured"
    except Exception:
        pass
    return p


# --------------------------------------------------------------------------------------------
# algorithmic cost per unknown of each kernel family (bytes and operations the method needs)
def kernel_cost(name, N, m, d, iters=None):
    """(bound, bytes per unknown, flops per unknown) of one launch, per unknown it processes.
    iters: the solve's iteration count, which sets the size of a deferred-update fold."""
    l2N = np.log2(2 * N)
    lN = np.log2(N)
    if name == "conv":      # FP64: real FFT 2N fwd + inv (2 x 2.5 * 2N log2 2N / N), 6 mul, 4 epilogue
        return "alu64", 16.0, 10.0 * l2N + 10.0
    if name == "conv_df":   # same algorithm in double-float on the FP32 pipes (FP32 operations)
        return "alu32", 16.0, df_conv_ops(N)
    if name in ("direct", "direct_resid"):
        return "hbm", 16.0, 6.0
    # tensor-core product: 15 digit-pair MMAs over the input times that reach each output block
    # of 128 times (128 (NB - rb) for row block rb of NB = N/128), 2 flops per multiply-add
    if name == "conv_tc":
        NB = N // 128
        return "tensor", 24.0, 2.0 * 15 * 128 * (NB + 1) / 2
    if name == "tc_digits":   # read x, write five bf16 digit planes
        return "hbm", 18.0, 0.0
    # the time pass inside the loop fuses the Lanczos combine: q, v_j, v_{j-1} read, v_{j+1} and z
    # written (40 B); the FP64 and double-float forms also read the lambda^{-1/2} table (8 B once)
    if name in ("timepass64", "timepass32"):   # 4 real FFTs of N, 2 spectral products, 3 scalings
        b = 40.0 + (8.0 if name == "timepass64" else 0.0)
        return ("alu64" if name == "timepass64" else "hbm"), b, 10.0 * lN + 15.0
    # DST-I: one complex FFT of length P = m+1 per two lines, the y_j pre-pass, the split of the
    # two spectra and the prefix sum of the odd outputs
    P = m + 1
    if name in ("dst64", "dst32"):
        return ("alu64" if name == "dst64" else "hbm"), 16.0, 5.0 * P * np.log2(P) / (2 * m) + 6.0
    if name == "dst_df":
        return "alu32", 16.0, df_dst_ops(m)
    if name == "timepass_df":
        return "alu32", 48.0, df_timepass_ops(N)
    if name == "w_update":
        return "hbm", 48.0, 6.0
    # deferred-update fold at the stop: x = sum of k = min(iters, 8) stored z's (k read, x written)
    if name == "fold":
        k = min(int(iters), 8) if iters else 8
        return "hbm", 8.0 * (k + 1), 2.0 * k
    # basis change of the dense-operator form: an M x M by M x N FP64 GEMM (2M flops per unknown)
    if name == "basis_gemm":
        return "alu64", 16.0, 2.0 * float(m) ** d
    # the same product in double-float on the FP32 pipes: 15 FP32 operations per multiply-add
    if name == "basis_gemm_df":
        return "alu32", 16.0, 15.0 * float(m) ** d
    return "hbm", 0.0, 0.0


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, index=0):
        self.proc = None
        # a scratch file in the system's temporary directory; the summary goes into the JSON line
        self.path = os.path.join(tempfile.gettempdir(), f"bltt_clocks_{os.getpid()}_{index}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.cmd = ["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                    "-lms", "200"]

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(self.cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 0, 1
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    return rank, local, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(v, ws, op, device):
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(v, ws, device="cuda"):
    """The timed region's length is the slowest rank's."""
    import torch.distributed as dist
    return _reduce(v, ws, dist.ReduceOp.MAX if ws > 1 else None, device)


def sum_over_ranks(v, ws, device="cuda"):
    """Units (unknown-iterations) processed by all ranks together."""
    import torch.distributed as dist
    return _reduce(v, ws, dist.ReduceOp.SUM if ws > 1 else None, device)


def replica_throughput(units_local, ms_local, ws, device="cuda"):
    """Whole-job throughput of independent replicas: sum of units / max of times (weak scaling)."""
    ms = max_over_ranks(ms_local, ws, device)
    units = sum_over_ranks(units_local, ws, device)
    return units / (ms / 1e3), ms, units


# --------------------------------------------------------------------------------------------
def time_form(B, solver, fd, steps, warmup, alpha, precision, basis, arith, ws, stream, profile):
    """Time `steps` whole solves (after `warmup`) on the device; returns a result dict."""
    import torch
    for _ in range(warmup):
        u, info = solver.solve(fd, alpha=alpha, tol=TOL, maxit=200, precision=precision,
                               basis=basis, rebuild=True, matvec_arith=arith)
    torch.cuda.synchronize()
    if profile:
        solver.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    infos = []
    e0.record(stream)
    for _ in range(steps):
        u, info = solver.solve(fd, alpha=alpha, tol=TOL, maxit=200, precision=precision,
                               basis=basis, rebuild=True, matvec_arith=arith)
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    prof = solver.profile_read() if profile else {}
    if profile:
        solver.profile(False)
    return {"ms_total": ms, "infos": infos, "profile": prof, "u": u}


def copy_bandwidth(f_host, stream):
    """GB/s of one host->device and one device->host copy of f (pinned), CUDA events."""
    import torch
    fd = torch.empty(f_host.shape, dtype=f_host.dtype, device="cuda")
    back = torch.empty_like(f_host, pin_memory=True)
    out = {}
    with torch.cuda.stream(stream):
        for name, (dst, src) in (("h2d", (fd, f_host)), ("d2h", (back, fd))):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            out[name] = round(f_host.numel() * 8 / (e0.elapsed_time(e1) / 1e3) / 1e9, 1)
    return out


def time_e2e(B, solver, f_host, steps, alpha, precision, basis, arith, stream):
    """Same metric through the public host-buffer solve: f copied in from pinned host memory,
    solve, u copied back into pinned host memory (the copy overlaps the final residual check)."""
    import torch
    u_host = torch.empty(f_host.shape, dtype=torch.float64, pin_memory=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # one untimed call: the handle's graph was last captured for another form
    solver.solve_host(f_host, alpha=alpha, tol=TOL, maxit=200, precision=precision, basis=basis,
                      u_host=u_host, rebuild=True, matvec_arith=arith)
    torch.cuda.synchronize()
    iters = 0
    e0.record(stream)
    for _ in range(steps):
        u, info = solver.solve_host(f_host, alpha=alpha, tol=TOL, maxit=200, precision=precision,
                                    basis=basis, u_host=u_host, rebuild=True, matvec_arith=arith)
        iters += info["iters"]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), iters


def cpu_baseline_sample(prob, f, alpha):
    """The oracle, as it stands, on one iteration's operator work of the full workload."""
    import oracle as O
    t0 = time.perf_counter()
    y = O.bltt_matvec(prob, f, flip=True)
    t1 = time.perf_counter()
    O.precond_apply(prob, alpha, y)
    t2 = time.perf_counter()
    return t2 - t0, t1 - t0, t2 - t1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from workloads import workload
    prob, rf = workload(WORKLOAD)
    f = rf()
    for _ in range(args.warmup):
        cpu_baseline_sample(prob, f, ALPHA_F32)
    times = []
    for _ in range(args.steps):
        times.append(cpu_baseline_sample(prob, f, ALPHA_F32)[0])
    tot = sum(times)
    value = prob.n * args.steps / tot
    cores = os.cpu_count()
    sample = ("one MINRES iteration's operator work (one Y A z by the direct Toeplitz product and "
              f"one P_alpha^{{-1}} apply by the paper's three steps, alpha = {ALPHA_F32:g}) on the "
              f"full {prob.n}-unknown workload per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "unknown-iter/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": prob.N, "m": prob.m[0], "d": prob.d, "gamma": 0.7,
                   "unknowns": prob.n, "tol": TOL},
        "cpu_baseline": {"value": value, "unit": "unknown-iter/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "unknown-iter/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


HEAD = "f32_precond"      # the form whose unknown-iterations/s is `value`
FORMS = {
    "f32_precond": dict(alpha=ALPHA_F32, precision=32, basis=1, arith=2),
    "chosen": dict(alpha=ALPHA_F32, precision=32, basis=1, arith=2),   # the same, older name
    "plain_f64": dict(alpha=ALPHA_F64, precision=64, basis=1, arith=1),
    "f32x2_precond": dict(alpha=ALPHA_F32X2, precision=96, basis=1, arith=2),
    "f32_physical": dict(alpha=ALPHA_F32, precision=32, basis=2, arith=2),
    "tc": dict(alpha=ALPHA_F32, precision=32, basis=1, arith=3),
}


def run_once(args):
    """One solve of the headline workload in one form, direct launches (for ncu captures).
    --m 127 keeps the kernels and FFT lengths of the 2-D N = 1024 workload on a quarter of its
    modes (132 MB per vector, still above L2), for captures that replay each kernel many times."""
    import torch
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as B
    from workloads import workload, rhs_uniform, fractional_problem, heat_bdf_problem
    if args.problem == "heat3d":
        # the 3-D heat workload's N = 256 on m = 63 per axis: 64 M unknowns, 512 MB per vector
        prob = heat_bdf_problem(3, args.m, 256)
        name = f"heat3d_bdf_N256_m{args.m}"
    elif args.m == 255:
        prob, _ = workload(WORKLOAD)
        name = WORKLOAD
    else:
        prob = fractional_problem(2, args.m, 1024, 0.7)
        name = f"frac2d_N1024_m{args.m}_g0.7"
    s = B.Solver(prob)
    fd = torch.from_numpy(rhs_uniform(prob.n, 2)).cuda()
    fm = FORMS[args.form]
    u, info = s.solve(fd, alpha=fm["alpha"], tol=TOL, maxit=100, precision=fm["precision"],
                      basis=fm["basis"], matvec_arith=fm["arith"], graph=False)
    torch.cuda.synchronize()
    print(json.dumps({"workload": name, "form": args.form, "iters": info["iters"],
                      "status": info["status"], "relres_true": info["relres_true"]}))
    return 0 if info["status"] == 0 else 1


def run_batched(args):
    """96 L1 fractional systems of uneven N and M with 4 right-hand sides each (8.75 G unknowns
    in all), solved by one bltt_solve_batched call, against the same items solved one by one.
    Right-hand sides: U[-1,1] seeded 4 + 1000 s + r; for the small systems (M <= 3969, at most
    600,000 unknowns) drawn by the workloads' numpy recipe, so that their iteration counts can be
    set beside the FP64 oracle's stored counts (tests/golden/oracle_counts_batched_sample.json),
    for the others by torch's CUDA generator (drawing 70 GB on the host would dominate the run)."""
    import torch
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as B
    from workloads import batched_systems
    sysl = batched_systems(96, 4, seed=4)
    probs = [p for p, _ in sysl]
    sample = [s for s, p in enumerate(probs) if p.M <= 3969 and p.n <= 600_000]
    fs, us = [], []
    for s, (p, rhs) in enumerate(sysl):
        row_f, row_u = [], []
        for r in range(4):
            if s in sample:
                row_f.append(torch.from_numpy(rhs[r]()).cuda())
            else:
                g = torch.Generator(device="cuda")
                g.manual_seed(4 + 1000 * s + r)
                row_f.append(torch.rand(p.n, generator=g, dtype=torch.float64, device="cuda") * 2 - 1)
            row_u.append(torch.empty(p.n, dtype=torch.float64, device="cuda"))
        fs.append(row_f)
        us.append(row_u)
    torch.cuda.synchronize()
    golden = {}
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_counts_batched_sample.json")) as fh:
            for c in json.load(fh)["cases"]:
                golden[(c["system"], c["rhs"], c["alpha"])] = c["iters"]
    except OSError:
        pass
    total_n = sum(p.n * 4 for p in probs)
    out = {"workload": "batched96x4", "systems": 96, "rhs_per_system": 4, "unknowns": total_n}
    forms = {"f32_precond": dict(precision=32, matvec_arith=2, alpha=ALPHA_F32),
             "f32x2_precond": dict(precision=96, matvec_arith=2, alpha=ALPHA_F32X2),
             "plain_f64": dict(precision=64, matvec_arith=1, alpha=ALPHA_F64)}
    for name, fm in forms.items():
        # a first call fills the tile-width autotuner's cache for these shapes
        B.bltt_solve_batched(probs, fs, us, alpha=[fm["alpha"]] * 96, tol=TOL, maxit=100,
                             precision=fm["precision"], matvec_arith=fm["matvec_arith"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, infos = B.bltt_solve_batched(probs, fs, us, alpha=[fm["alpha"]] * 96, tol=TOL,
                                         maxit=100, precision=fm["precision"],
                                         matvec_arith=fm["matvec_arith"])
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        iters = [i["iters"] for i in infos]
        units = sum(p.n * iters[4 * s + r] for s, p in enumerate(probs) for r in range(4))
        # the same items one at a time through bltt_minres_solve_ex on a stream (graph replay)
        stream = torch.cuda.Stream()
        t0 = time.perf_counter()
        seq_iters = []
        with torch.cuda.stream(stream):
            for s, p in enumerate(probs):
                sol = B.Solver(p, stream=stream)
                for r in range(4):
                    _, inf = sol.solve(fs[s][r], alpha=fm["alpha"], tol=TOL, maxit=100,
                                       precision=fm["precision"], basis=B.BASIS_SPECTRAL,
                                       matvec_arith=fm["matvec_arith"], u=us[s][r])
                    seq_iters.append(inf["iters"])
                sol.close()
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        # per-system counts of the sampled systems against the FP64 oracle's at the same alpha
        deltas = [iters[4 * s + r] - golden[(s, r, fm["alpha"])] for s in sample for r in range(4)
                  if (s, r, fm["alpha"]) in golden]
        out[name] = {"status": st, "batched_s": t_batch, "sequential_s": t_seq,
                     "speedup": t_seq / t_batch,
                     "value_batched": units / t_batch, "value_sequential":
                     sum(p.n * seq_iters[4 * s + r] for s, p in enumerate(probs) for r in range(4)) / t_seq,
                     "unit": "unknown-iter/s", "alpha": fm["alpha"],
                     "max_relres": max(i["relres_true"] for i in infos),
                     "iters_per_system": [iters[4 * s] for s in range(96)],
                     "iters_match_sequential": iters == seq_iters,
                     "oracle_sample": {"items": len(deltas),
                                       "systems": len(sample),
                                       "equal": sum(1 for d in deltas if d == 0),
                                       "max_abs_delta": max((abs(d) for d in deltas), default=None),
                                       "deltas_histogram": {str(k): deltas.count(k)
                                                            for k in sorted(set(deltas))}}}
    print(json.dumps(out))
    return 0


def run_alpha(args):
    """Learned alpha (FP32-preconditioner form): sweeps, training, held-out evaluation.  Every
    held-out solve is timed on the device (CUDA events on the solver's stream, set-up included);
    the learned form is compared with fixed alphas of the same form (the best of them picked with
    hindsight on the held-out set), with the paper's alpha = 1e-8 in that form, and with the plain
    FP64 solve at alpha = 1e-8."""
    import torch
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as B
    from paper_2307_07749_gb300 import learned_alpha as LA
    from workloads import alpha_training_problems
    t0 = time.perf_counter()
    train = alpha_training_problems(args.alpha_train, seed=5)
    X, t, raw = LA.build_dataset(train, maxit=40)
    t_sweep = time.perf_counter() - t0
    t0 = time.perf_counter()
    model, hist = LA.train(X, t, epochs=4000, lr=3e-3, seed=0)
    t_train = time.perf_counter() - t0
    held = alpha_training_problems(args.alpha_heldout, seed=55)
    alphas = LA.predict(model, [p for p, _ in held])
    fs = [rf() for _, rf in held]

    def evaluate(alpha_of, precision=32, arith=2, maxit=60):
        its, ms, fails = [], [], 0
        for (p, _), f, a in zip(held, fs, alpha_of):
            stream = torch.cuda.Stream()
            s = B.Solver(p, stream=stream)
            fd = torch.from_numpy(f).cuda()
            with torch.cuda.stream(stream):
                # one untimed solve (graph capture, tables), then the timed one
                s.solve(fd, alpha=float(a), tol=TOL, maxit=maxit, precision=precision, basis=1,
                        matvec_arith=arith, raise_on_error=False, rebuild=True)
                _, info = s.solve(fd, alpha=float(a), tol=TOL, maxit=maxit, precision=precision,
                                  basis=1, matvec_arith=arith, raise_on_error=False, rebuild=True)
            torch.cuda.synchronize()
            ok = info["status"] == 0 and info["relres_true"] <= TOL
            fails += 0 if ok else 1
            its.append(info["iters"] if ok else maxit)
            ms.append(info["t_solve_ms"])
            s.close()
        return {"mean_iters": float(np.mean(its)), "total_iters": int(np.sum(its)),
                "mean_device_ms": float(np.mean(ms)), "total_device_ms": float(np.sum(ms)),
                "not_converged": fails}

    fixed = {a: evaluate([a] * len(held)) for a in (1e-2, 3e-3, 1e-3, 1e-4)}
    best_a = min(fixed, key=lambda a: (fixed[a]["total_iters"], fixed[a]["total_device_ms"]))
    res = {"workload": "alpha_learning", "train_problems": len(train), "labelled": int(len(t)),
           "heldout": len(held), "sweep_s": t_sweep, "train_s": t_train,
           "loss_first_last": [float(hist[0]), float(hist[-1])],
           "learned": evaluate(alphas),
           "fixed": {f"{a:g}": v for a, v in fixed.items()},
           "best_fixed_alpha": best_a,
           "paper_rule_1e-8_same_form": evaluate([1e-8] * len(held)),
           "plain_f64_1e-8": evaluate([1e-8] * len(held), precision=64, arith=1),
           "form": "FP32 preconditioner, double-float matvec, DST basis, tol 1e-8",
           "timing": "device time of each solve (CUDA events on its stream, set-up included), "
                     "after one untimed solve"}
    print(json.dumps(res))
    return 0


def run_heat3d(args):
    """The 3-D backward-Euler heat workload (N = 256, m = 127, 524 M unknowns, 4.2 GB per vector):
    whole solves in the FP32-preconditioner form and the plain FP64 form, each kernel's live
    duration against its algorithmic bytes (the memory-bound roofline run)."""
    import torch
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as B
    from workloads import workload
    prob, rf = workload("heat3d_bdf_N256_m127")
    f = rf()
    stream = torch.cuda.Stream()
    solver = B.Solver(prob, stream=stream)
    fd = torch.from_numpy(f).to("cuda")
    del f
    torch.cuda.synchronize()
    pk = peaks()
    forms = {"f32_precond": dict(alpha=ALPHA_F32, precision=32, basis=B.BASIS_SPECTRAL,
                                 arith=B.ARITH_F32X2),
             "plain_f64": dict(alpha=ALPHA_F64, precision=64, basis=B.BASIS_SPECTRAL,
                               arith=B.ARITH_F64)}
    out = {"workload": "heat3d_bdf_N256_m127", "unknowns": prob.n, "N": prob.N, "m": prob.m[0],
           "d": prob.d, "tol": TOL, "steps": args.steps, "warmup": max(args.warmup, 1),
           "l2": "inputs larger than L2 (4.2 GB per vector), no flush"}
    with torch.cuda.stream(stream):
        for key, fm in forms.items():
            r = time_form(B, solver, fd, args.steps, max(args.warmup, 1), fm["alpha"],
                          fm["precision"], fm["basis"], fm["arith"], 1, stream, profile=True)
            iters = [i["iters"] for i in r["infos"]]
            kern = []
            for name, (all_l, all_ms, launches, tot_ms) in r["profile"].items():
                bound, bpu, fpu = kernel_cost(name, prob.N, prob.m[0], prob.d, iters[-1])
                if launches == 0 or bpu == 0:
                    continue
                avg = tot_ms / launches
                gbs = bpu * prob.n / (avg / 1e3) / 1e9
                kern.append({"name": name, "launches": launches, "ms_per_launch": round(avg, 4),
                             "bytes_per_unit": bpu, "GB/s": round(gbs, 1),
                             "frac_hbm": round(gbs / pk["hbm_gbs"], 4), "bound": bound,
                             "all_launches": all_l, "all_ms": round(all_ms, 3)})
            kern.sort(key=lambda k: -k["ms_per_launch"] * k["launches"])
            ms = r["ms_total"] / args.steps
            out[key] = {"value": prob.n * sum(iters) / (r["ms_total"] / 1e3),
                        "unit": "unknown-iter/s", "iters": iters[-1], "ms_per_solve": ms,
                        "relres_true": max(i["relres_true"] for i in r["infos"]),
                        "status": max(i["status"] for i in r["infos"]), "form": fm,
                        "kernels": kern}
    out["hbm_peak_gbs"] = pk["hbm_gbs"]
    print(json.dumps(out))
    return 0


def run_varcoef(args):
    """Variable-coefficient blocks at the largest size of the paper's tables, physical basis (the
    DST does not diagonalise L_a), the preconditioner of the mean-coefficient blocks, tolerance
    1e-6 as in the tables:
      * Example heateqvarcoeff (CN heat, Table 3): N = 256, m + 1 = 256 (16,646,400 unknowns),
        right-hand side seeded U[-1, 1];
      * Example 4 (L1 fractional, gamma = 0.6, a = 35 + x^3.5 + y^3.5, Table 8): the same size, on
        the example's own right-hand side."""
    import torch
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as B
    from workloads import (fractional_varcoeff_problem, heat_cn_varcoeff_problem,
                           paper_data_frac_var, rhs_uniform)
    pk = peaks()
    # the FP32-preconditioner form with the double-float matvec, as in the headline
    # (the CN blocks' direct product is FP64 whatever the setting)
    forms = {"plain_f64": dict(alpha=ALPHA_F64, precision=64, arith=B.ARITH_F64),
             "f32_precond": dict(alpha=ALPHA_F32, precision=32, arith=B.ARITH_F32X2)}

    def measure(prob, f_np):
        stream = torch.cuda.Stream()
        solver = B.Solver(prob, stream=stream)
        fd = torch.from_numpy(f_np).to("cuda")
        torch.cuda.synchronize()
        res = {}
        with torch.cuda.stream(stream):
            for key, fm in forms.items():
                for _ in range(max(args.warmup, 1)):
                    solver.solve(fd, alpha=fm["alpha"], tol=1e-6, maxit=200,
                                 precision=fm["precision"], basis=B.BASIS_PHYSICAL, rebuild=True,
                                 matvec_arith=fm["arith"])
                torch.cuda.synchronize()
                solver.profile(True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                infos = []
                e0.record(stream)
                for _ in range(args.steps):
                    _, info = solver.solve(fd, alpha=fm["alpha"], tol=1e-6, maxit=200,
                                           precision=fm["precision"], basis=B.BASIS_PHYSICAL,
                                           rebuild=True, matvec_arith=fm["arith"])
                    infos.append(info)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                prof = solver.profile_read()
                solver.profile(False)
                iters = [i["iters"] for i in infos]
                kern = []
                for name, (_, _, launches, tot_ms) in prof.items():
                    bound, bpu, fpu = kernel_cost(name, prob.N, prob.m[0], prob.d, iters[-1])
                    if launches == 0 or bpu == 0:
                        continue
                    avg = tot_ms / launches
                    gbs = bpu * prob.n / (avg / 1e3) / 1e9
                    kern.append({"name": name, "launches": launches, "ms_per_launch": round(avg, 4),
                                 "GB/s": round(gbs, 1), "frac_hbm": round(gbs / pk["hbm_gbs"], 4)})
                kern.sort(key=lambda k: -k["ms_per_launch"] * k["launches"])
                res[key] = {"value": prob.n * sum(iters) / (ms / 1e3), "unit": "unknown-iter/s",
                            "iters": iters[-1], "ms_per_solve": ms / args.steps,
                            "relres_true": max(i["relres_true"] for i in infos),
                            "status": max(i["status"] for i in infos), "kernels": kern}
        solver.close()
        return res

    prob = heat_cn_varcoeff_problem(255, 256)
    out = {"workload": "heat2d_cnvar_N256_m255 (Table 3, largest size)", "unknowns": prob.n,
           "tol": 1e-6, "basis": "physical", "steps": args.steps,
           "warmup": max(args.warmup, 1),
           "paper_context": "Table 3 prints 10 MINRES-P_alpha iterations and 32.40 s (Octave, CPU) at this size"}
    out.update(measure(prob, rhs_uniform(prob.n, 12)))
    p4 = fractional_varcoeff_problem(255, 256, 0.6)
    e4 = {"workload": "fracvar2d_N256_m255_g0.6 (Example 4, Table 8, largest size)",
          "unknowns": p4.n, "rhs": "the example's own data",
          "paper_context": "Table 8 prints 8 MINRES-P_alpha iterations and 27.14 s (Octave, CPU) at this size"}
    e4.update(measure(p4, paper_data_frac_var(p4, 0.6)))
    out["example4"] = e4
    print(json.dumps(out))
    return 0


def run_small(args):
    """The smallest workload (1-D L1 fractional, gamma = 0.5, N = 64, m = 63: 4032 unknowns), DST
    basis, in FP64 (alpha = 1e-8) and in the FP32-preconditioner form: whole solves by the
    multi-launch driver (CUDA-graph replay) against the single-block kernel (one launch per
    solve).  Right-hand side: seeded U[-1, 1]."""
    import torch
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as B
    from workloads import workload, rhs_uniform
    prob, _ = workload("frac1d_N64_m63_g0.5")
    stream = torch.cuda.Stream()
    solver = B.Solver(prob, stream=stream)
    fd = torch.from_numpy(rhs_uniform(prob.n, 1)).to("cuda")
    torch.cuda.synchronize()
    out = {"workload": "frac1d_N64_m63_g0.5", "unknowns": prob.n, "tol": TOL,
           "steps": args.steps * 20, "warmup": max(args.warmup, 3)}
    f64 = dict(alpha=ALPHA_F64, precision=64, matvec_arith=B.ARITH_F64)
    f32p = dict(alpha=ALPHA_F32, precision=32, matvec_arith=B.ARITH_F32X2)
    forms = {"graph_f64": dict(single_block=False, **f64),
             "single_block_f64": dict(single_block=True, **f64),
             "graph_f32_precond": dict(single_block=False, **f32p),
             "single_block_f32_precond": dict(single_block=True, **f32p)}
    with torch.cuda.stream(stream):
        for key, fm in forms.items():
            for _ in range(max(args.warmup, 3)):
                solver.solve(fd, tol=TOL, maxit=100, basis=1, **fm)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            infos = []
            k = args.steps * 20
            e0.record(stream)
            for _ in range(k):
                _, info = solver.solve(fd, tol=TOL, maxit=100, basis=1, **fm)
                infos.append(info)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            out[key] = {"ms_per_solve": ms, "iters": infos[-1]["iters"],
                        "value": prob.n * infos[-1]["iters"] / (ms / 1e3), "unit": "unknown-iter/s",
                        "relres_true": max(i["relres_true"] for i in infos),
                        "kernel_launches": infos[-1]["kernel_launches"],
                        "status": max(i["status"] for i in infos)}
    print(json.dumps(out))
    return 0


def run_dense(args):
    """Commuting dense blocks a_k I + b_k K (Sec. 3): the L1 time-fractional blocks (gamma = 0.5,
    N = 1024) with a dense non-local diffusion operator K on a 63 x 63 grid (M = 3969, n =
    4,064,256 unknowns).  The solve runs in K's eigenbasis: one GEMM in, the iterations with K's
    eigenvalue table, one GEMM out (double-float on the FP32 pipes with the double-float matvec,
    FP64 with the FP64 matvec).  The eigendecomposition is set-up (untimed).
    Right-hand side: seeded U[-1, 1]."""
    import torch
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as B
    from workloads import nonlocal_diffusion_problem, rhs_uniform
    prob = nonlocal_diffusion_problem(63, 1024, 0.5)
    stream = torch.cuda.Stream()
    t0 = time.time()
    solver = B.Solver(prob, stream=stream)
    t_setup = time.time() - t0
    fd = torch.from_numpy(rhs_uniform(prob.n, 13)).to("cuda")
    torch.cuda.synchronize()
    pk = peaks()
    forms = {"f32_precond": dict(alpha=ALPHA_F32, precision=32, basis=B.BASIS_SPECTRAL,
                                 arith=B.ARITH_F32X2),
             "plain_f64": dict(alpha=ALPHA_F64, precision=64, basis=B.BASIS_SPECTRAL,
                               arith=B.ARITH_F64)}
    out = {"workload": "nonlocal2d_N1024_m63 (L1 gamma 0.5, dense Gaussian-kernel K)",
           "unknowns": prob.n, "M": prob.M, "tol": TOL, "steps": args.steps,
           "warmup": max(args.warmup, 1), "eigendecomposition_s": round(t_setup, 3),
           "l2": "inputs of 32.5 MB per vector, below L2; no flush (supplementary report)"}
    with torch.cuda.stream(stream):
        for key, fm in forms.items():
            r = time_form(B, solver, fd, args.steps, max(args.warmup, 1), fm["alpha"],
                          fm["precision"], fm["basis"], fm["arith"], 1, stream, profile=True)
            iters = [i["iters"] for i in r["infos"]]
            kern = []
            for name, (all_l, all_ms, launches, tot_ms) in r["profile"].items():
                bound, bpu, fpu = kernel_cost(name, prob.N, prob.m[0], prob.d, iters[-1])
                if launches == 0 or bpu == 0:
                    continue
                avg = tot_ms / launches
                e = {"name": name, "launches": launches, "ms_per_launch": round(avg, 4),
                     "bound": bound}
                if name == "basis_gemm":
                    tf = fpu * prob.n / (avg / 1e3) / 1e12
                    e.update({"TFLOP/s": round(tf, 3), "frac_fp64": round(tf / FP64_PEAK_TFLOPS, 4)})
                elif name == "basis_gemm_df":
                    tops = fpu * prob.n / (avg / 1e3) / 1e12
                    e.update({"Tops/s (FP32 pipe)": round(tops, 3),
                              "frac_fp32_pipe": round(tops / FP32_PEAK_TOPS, 4),
                              "fp64_equivalent_TFLOP/s": round(2 * tops / fpu * prob.M, 3)})
                else:
                    gbs = bpu * prob.n / (avg / 1e3) / 1e9
                    e.update({"GB/s": round(gbs, 1), "frac_hbm": round(gbs / pk["hbm_gbs"], 4)})
                kern.append(e)
            kern.sort(key=lambda k: -k["ms_per_launch"] * k["launches"])
            out[key] = {"value": prob.n * sum(iters) / (r["ms_total"] / 1e3),
                        "unit": "unknown-iter/s", "iters": iters[-1],
                        "ms_per_solve": r["ms_total"] / args.steps,
                        "relres_true": max(i["relres_true"] for i in r["infos"]),
                        "status": max(i["status"] for i in r["infos"]), "form": fm,
                        "kernels": kern}
    out["fp64_peak_tflops"] = FP64_PEAK_TFLOPS
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="frac2d",
                    choices=["frac2d", "batched", "alpha", "once", "heat3d", "varcoef", "dense",
                             "small"],
                    help="frac2d: the headline line; batched / alpha / heat3d: supplementary "
                         "reports; once: a single solve of the headline workload (for ncu "
                         "captures)")
    ap.add_argument("--form", default="f32_precond", choices=list(FORMS))
    ap.add_argument("--m", type=int, default=255, choices=[63, 127, 255],
                    help="--workload once: interior points per axis (255: the headline workload)")
    ap.add_argument("--problem", default="frac2d", choices=["frac2d", "heat3d"],
                    help="--workload once: the 2-D fractional workload or the 3-D heat one")
    ap.add_argument("--alpha-train", type=int, default=2000)
    ap.add_argument("--alpha-heldout", type=int, default=256)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "alpha":
        return run_alpha(args)
    if args.workload == "once":
        return run_once(args)
    if args.workload == "heat3d":
        return run_heat3d(args)
    if args.workload == "varcoef":
        return run_varcoef(args)
    if args.workload == "dense":
        return run_dense(args)
    if args.workload == "small":
        return run_small(args)
    args.warmup = max(args.warmup, 3)

    rank, local, ws = dist_init()
    import torch
    torch.cuda.set_device(local)
    from paper_2307_07749_gb300 import build
    if rank == 0:
        build.build()
    barrier(ws)
    import paper_2307_07749_gb300 as B
    from workloads import workload, rhs_uniform

    prob, _ = workload(WORKLOAD)
    f = rhs_uniform(prob.n, 2 + 100 * rank)      # rank r solves its own right-hand side
    stream = torch.cuda.Stream()
    solver = B.Solver(prob, stream=stream)
    fd = torch.from_numpy(f).to("cuda")
    torch.cuda.synchronize()

    forms = {
        "f32_precond": dict(alpha=ALPHA_F32, precision=32, basis=B.BASIS_SPECTRAL,
                            arith=B.ARITH_F32X2),
        "plain_f64": dict(alpha=ALPHA_F64, precision=64, basis=B.BASIS_SPECTRAL, arith=B.ARITH_F64),
        "f32x2_precond": dict(alpha=ALPHA_F32X2, precision=96, basis=B.BASIS_SPECTRAL,
                              arith=B.ARITH_F32X2),
        "f32_physical": dict(alpha=ALPHA_F32, precision=32, basis=B.BASIS_PHYSICAL,
                             arith=B.ARITH_F32X2),
        "tc": dict(alpha=ALPHA_F32, precision=32, basis=B.BASIS_SPECTRAL, arith=B.ARITH_TC),
    }
    res = {}
    e2e_raw = None
    with torch.cuda.stream(stream):
        for key, fm in forms.items():
            sampler = ClockSampler(local) if key == HEAD else None
            if sampler:
                sampler.__enter__()
            try:
                r = time_form(B, solver, fd, args.steps, args.warmup, fm["alpha"], fm["precision"],
                              fm["basis"], fm["arith"], ws, stream, profile=True)
            finally:
                if sampler:
                    sampler.__exit__()
            r["clocks"] = sampler.summary() if sampler else None
            res[key] = r
            if key == HEAD and not args.no_e2e:
                # the same form end to end through the host-buffer entry point, right after the
                # device-resident timing (same handle, same clocks), its own clock samples beside it
                f_host = torch.from_numpy(f).pin_memory()
                copy_gbs = copy_bandwidth(f_host, stream)
                es = ClockSampler(local)
                es.__enter__()
                try:
                    e_ms, e_iters = time_e2e(B, solver, f_host, args.steps, ALPHA_F32, 32,
                                             B.BASIS_SPECTRAL, B.ARITH_F32X2, stream)
                finally:
                    es.__exit__()
                e2e_raw = (e_ms, e_iters, copy_gbs, es.summary())

    def summarise(r):
        ms = max_over_ranks(r["ms_total"], ws)
        iters = [i["iters"] for i in r["infos"]]
        units = sum_over_ranks(float(prob.n * sum(iters)), ws)
        return {
            "value": units / (ms / 1e3), "ms_per_step": ms / args.steps,
            "iters": iters[-1], "relres_true": max(i["relres_true"] for i in r["infos"]),
            "status": max(i["status"] for i in r["infos"]),
            "launches": sum(i["kernel_launches"] for i in r["infos"]),
            "setup_ms": float(np.mean([i["t_setup_ms"] for i in r["infos"]])),
        }

    ch = summarise(res[HEAD])
    pl = summarise(res["plain_f64"])
    others = {k: summarise(res[k]) for k in ("f32x2_precond", "f32_physical", "tc")}
    # time to solution of every form (the deciding number), and the fastest
    tts = {k: summarise(res[k]) for k in forms}
    fastest = min(tts, key=lambda k: tts[k]["ms_per_step"])

    # roofline of the dominant kernel of the headline form (live CUDA-event durations)
    pk = peaks()
    prof = res[HEAD]["profile"]
    kern = []
    for name, (all_launches, all_ms, launches, tot_ms) in prof.items():
        bound, bpu, fpu = kernel_cost(name, prob.N, prob.m[0], prob.d,
                                      res[HEAD]["infos"][-1]["iters"])
        avg_ms = tot_ms / max(launches, 1)
        units = prob.n
        if bound == "alu64":
            ach = fpu * units / (avg_ms / 1e3) / 1e12
            kern.append(dict(name=name, launches=launches, total_ms=tot_ms, bound="alu",
                             achieved=ach, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s (FP64)",
                             frac=ach / FP64_PEAK_TFLOPS, bytes_per_unit=bpu, flops_per_unit=fpu))
        elif bound == "alu32":
            ach = fpu * units / (avg_ms / 1e3) / 1e12
            kern.append(dict(name=name, launches=launches, total_ms=tot_ms, bound="alu",
                             achieved=ach, peak=FP32_PEAK_TOPS, unit="Tops/s (FP32 pipe)",
                             frac=ach / FP32_PEAK_TOPS, bytes_per_unit=bpu, flops_per_unit=fpu))
        elif bound == "tensor":
            ach = fpu * units / (avg_ms / 1e3) / 1e12
            kern.append(dict(name=name, launches=launches, total_ms=tot_ms, bound="tensor",
                             achieved=ach, peak=pk["bf16_tflops"], unit="TFLOP/s (bf16 tensor)",
                             frac=ach / pk["bf16_tflops"], bytes_per_unit=bpu, flops_per_unit=fpu))
        elif bpu > 0:
            ach = bpu * units / (avg_ms / 1e3) / 1e9
            kern.append(dict(name=name, launches=launches, total_ms=tot_ms, bound="hbm",
                             achieved=ach, peak=pk["hbm_gbs"], unit="GB/s",
                             frac=ach / pk["hbm_gbs"], bytes_per_unit=bpu, flops_per_unit=fpu))
    kern.sort(key=lambda k: -k["total_ms"])
    dom = kern[0] if kern else None
    roof = None
    if dom:
        roof = {"kernel": dom["name"], "bound": dom["bound"], "achieved": round(dom["achieved"], 4),
                "peak": dom["peak"], "unit": dom["unit"], "frac": round(dom["frac"], 4),
                "traffic": NCU_TRAFFIC_PER_UNKNOWN.get(dom["name"], (None, ""))[0] and
                           NCU_TRAFFIC_PER_UNKNOWN[dom["name"]][0] * prob.n,
                "traffic_source": NCU_TRAFFIC_PER_UNKNOWN.get(dom["name"], (None, None))[1],
                "peak_source": (("derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz, confirmed by a "
                                 "measured 1.20 TFLOP/s FP64 FMA loop") if dom["unit"].endswith("(FP64)")
                                else ("derived: 128 FP32 ops/clk/SM x 152 SMs x 2.07 GHz, confirmed "
                                      "by a measured 69.8 TFLOP/s FP32 FMA loop")
                                if dom["bound"] == "alu" else pk["source"] + " hbm_gbs")}

    e2e = None
    if e2e_raw is not None:
        e_ms, e_iters, copy_gbs, e_clocks = e2e_raw
        e_ms = max_over_ranks(e_ms, ws)
        e_units = sum_over_ranks(float(prob.n * e_iters), ws)
        e2e = {"value": e_units / (e_ms / 1e3), "unit": "unknown-iter/s",
               "h2d_bytes_per_step": prob.n * 8, "d2h_bytes_per_step": prob.n * 8,
               "ms_per_step": e_ms / args.steps, "copy_GBps": copy_gbs, "clocks": e_clocks}

    # accuracy of the headline form against the plain FP64 GPU solve (error stated per result)
    uc = res[HEAD]["u"]
    up = res["plain_f64"]["u"]
    err_vs_f64 = float(torch.linalg.norm(uc - up) / torch.linalg.norm(up))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        t, tmv, tpc = cpu_baseline_sample(prob, f, ALPHA_F32)
        cpu = {"value": prob.n / t, "unit": "unknown-iter/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": ("one MINRES iteration's operator work on the full workload: one Y A z "
                          f"({tmv:.1f} s) and one P_alpha^-1 apply ({tpc:.1f} s), numpy/scipy FP64")}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": ch["value"], "unit": "unknown-iter/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ch["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (f32x2 matvec)",
            "data": "synthetic (seeded U[-1,1] right-hand side)",
            "config": {"workload": WORKLOAD, "d": 2, "N": prob.N, "m": prob.m[0], "M": prob.M,
                       "gamma": 0.7, "unknowns": prob.n, "tol": TOL, "alpha": ALPHA_F32,
                       "precond_precision": "fp32", "basis": "spectral (DST-I basis)",
                       "matvec_arith": "f32x2 (double-float)",
                       "l2": "inputs larger than L2 (533 MB per vector), no flush",
                       "parallelism": f"replicas x{ws}"},
            "form": HEAD, "iters": ch["iters"], "relres_true": ch["relres_true"],
            "time_to_solution_ms": ch["ms_per_step"], "setup_ms": ch["setup_ms"],
            # every form's time to solution at relres <= 1e-8 (the deciding number) and the
            # fastest of them
            "time_to_solution": {k: {"ms": round(v["ms_per_step"], 3), "iters": v["iters"],
                                     "relres_true": v["relres_true"],
                                     "alpha": forms[k]["alpha"],
                                     "unknown_iter_per_s": v["value"]}
                                 for k, v in tts.items()},
            "fastest_form": {"form": fastest, "time_to_solution_ms": tts[fastest]["ms_per_step"],
                             "iters": tts[fastest]["iters"],
                             "relres_true": tts[fastest]["relres_true"],
                             "alpha": forms[fastest]["alpha"],
                             "kernels": {k: [int(v[2]), round(v[3], 4)]
                                         for k, v in res[fastest]["profile"].items()}},
            "err_vs_plain_f64_solution": err_vs_f64,
            "plain_f64": {"value": pl["value"], "unit": "unknown-iter/s", "iters": pl["iters"],
                          "relres_true": pl["relres_true"], "time_to_solution_ms": pl["ms_per_step"],
                          "alpha": ALPHA_F64, "basis": "spectral", "dtype": "f64",
                          "setup_ms": pl["setup_ms"]},
            "other_forms": {k: {"value": v["value"], "unit": "unknown-iter/s", "iters": v["iters"],
                                "relres_true": v["relres_true"],
                                "time_to_solution_ms": v["ms_per_step"],
                                "form": {kk: (vv if not isinstance(vv, float) else vv)
                                         for kk, vv in forms[k].items()}}
                            for k, v in others.items()},
            "roofline": roof,
            "kernels": [{k: (round(v, 5) if isinstance(v, float) else v) for k, v in kk.items()}
                        for kk in kern],
            # every form's kernel families: [active launches, their total ms]
            "kernels_by_form": {key: {k: [int(v[2]), round(v[3], 4)]
                                      for k, v in res[key]["profile"].items()}
                                for key in res},
            "e2e": e2e,
            "gpu_launches": ch["launches"],
            "clocks": res[HEAD]["clocks"],
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

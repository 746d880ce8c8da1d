#!/usr/bin/env python
"""Throughput of the FFT Toeplitz apply of the fractional-Laplacian scheme on one GB300.

Default workload: 2D, alpha = 1.5, Omega = (-1,1)^2, h = 2/2048 (2047 x 2047 interior
unknowns), an FP64-precision apply y = A u through libfrlap (the 2D throughput case
of the 3D FP64 CG configuration), computed by the double-float FFT engine
(FP64 vectors; FFT stages in FP32 pairs, parity 1e-12 normwise against the FP64
oracle, like native FP64).  One step = one batched apply (frlap_apply_batch, one
launch per stage) to 8 distinct seeded N(0,1) vectors (268 MB of inputs, more than
the 129 MB L2).  Reported: apply
unknowns/s over all ranks, the per-kernel roofline of the dominant kernel, the
same metric end to end through host buffers, and the CPU oracle timed on the
host cores.  Extra lines (native FP64 and FP32 applies, 3D 255^3 applies, CG
solve times) are measured after the timed region.  `--suite solvers` instead runs
the solver configurations (time to 1e-10 for plain CG, refinement, Strang and
learned preconditioning; the batched Allen-Cahn launch) and prints them.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl frlap|reference] [--prec df64|f64|f32]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import frlap_inputs as inp  # noqa: E402

ALPHA = 1.5
NGRID = 2048
BATCH = 8  # vectors per step of the 2D workload
BATCH_2D = BATCH
NGRID_3D, ALPHA_3D, BATCH_3D = 256, 1.0, 2
E2E_CHUNK = 1  # vectors per chunk of the host-buffer pipeline (1, 2, 4, 8 measured 6.9, 6.6, 5.8, 4.7 G unknowns/s)
METRIC = "apply unknowns/s & %HBM peak; PCG time to 1e-10 of FP64 sol vs plain FP64 CG"
UNIT = "unknowns/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 pipe: 152 SMs x 4 FP64 flop/clk (2 DFMA) x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 256 * 2.07e9 / 1e12
# DRAM traffic of one batched launch of the dominant kernel, by (dims, kernel, engine) (dram__bytes_read.sum +
# dram__bytes_write.sum) from the ncu captures summarised under profiles/; absent where the kernel
# changed since the capture
MEASURED_TRAFFIC = {(2, "colmul", "df64"): 1282.7e6, (2, "colmul", "f32"): 598.3e6,
                    (3, "colmul", "df64"): 2459.0e6, (3, "colmul", "f32"): 1261.6e6}

# double-float roofline: FP32 issue rate (152 SMs x 128 lanes x 2.07 GHz = 40.3 T instr/s) over the
# FP32 instructions the kernel's double-float butterflies take per FP64-equivalent flop (flops counted
# by the usual 5 L log2 L per complex transform).  Instruction costs of the double-float operations:
# add 11, add without renormalisation 8, multiply 7, complex product feeding a sum (two lazy
# two-product sums) 32.
FP32_ISSUE = 152 * 128 * 2.07e9
DF_DFT4 = 4 * 2 * 8 + 4 * 2 * 11                              # lazy first-level sums, full second level
DF_DFT16_TAIL = 8 * 32 + 4 * DF_DFT4                          # 8 products by W16^m, four length-4 DFTs
DF_DFT16 = 4 * DF_DFT4 + DF_DFT16_TAIL
DF_DFT16_ZIN = 4 * 4 * 2 * 11 + DF_DFT16_TAIL                 # upper half of the input zero
DF_DFT8_COMBINE = 2 * (2 * 11 + 2 * 7) + 8 * 2 * 11
DF_DFT8 = 2 * DF_DFT4 + DF_DFT8_COMBINE
DF_DFT8_ZIN = 8 * 2 * 11 + DF_DFT8_COMBINE
DF_TW16 = 15 * 32                                             # stage twiddles of a radix-16 butterfly


def df_fft_instr(L, zin):
    """FP32 instructions of one double-float transform of length L (the engine's stage order)."""
    n = int(math.log2(L))
    rem = n % 4
    if rem == 3:
        return L // 8 * (DF_DFT8_ZIN if zin else DF_DFT8) + (n - 3) // 4 * L // 16 * (DF_DFT16 + DF_TW16)
    first = L // 16 * (DF_DFT16_ZIN if zin else DF_DFT16)
    mid = ((n - rem) // 4 - 1) * L // 16 * (DF_DFT16 + DF_TW16)
    last = {0: 0, 1: L // 2 * (32 + 2 * 2 * 11), 2: L // 4 * (3 * 32 + DF_DFT4)}[rem]
    return first + mid + last


def df64_instr_per_flop(kernel, P):
    """FP32 instructions per FP64-equivalent flop of one line of `kernel` (P: embedding per axis)."""
    if kernel == "colmul":
        L = P[-1]
        return (df_fft_instr(L, True) + df_fft_instr(L, False) + 14 * L) / (10 * L * math.log2(L) + 2 * L)
    if kernel in ("c2cT_fwd", "c2cT_inv"):
        L = P[1]
        return df_fft_instr(L, kernel == "c2cT_fwd") / (5 * L * math.log2(L))
    # r2c_T / c2r_T: half-length complex transform and the split of its H + 1 bins (two sums, a
    # product, a sum: about 104 instructions a bin)
    H = P[0] // 2
    return (df_fft_instr(H, kernel == "r2c_T") + 104 * (H + 1)) / (2.5 * P[0] * math.log2(P[0]))


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def fft_flops_2d(n, P):
    """Algorithmic flops of one 2D apply, radix-2 convention 5 L log2 L per complex transform of length L
    (a real transform of length L counts half)."""
    nx, ny = n
    Px, Py = P
    Hx1 = Px // 2 + 1
    f_rows = ny * 2.5 * Px * math.log2(Px)
    f_cols = Hx1 * (2 * 5 * Py * math.log2(Py) + 2 * Py)
    return {"r2c": f_rows, "colmul": f_cols, "c2r": f_rows}


def stage_names(d):
    return ["r2c_T", "colmul", "c2r_T"] if d == 2 else ["r2c_T", "c2cT_fwd", "colmul", "c2cT_inv", "c2r_T"]


def stage_bytes(d, n, P, eb):
    """Bytes each stage must move (read + write) in the pass model: real in/out eb bytes, complex 2 eb."""
    cb = 2 * eb
    if d == 2:
        nx, ny = n
        Px, Py = P
        H1 = Px // 2 + 1
        M = nx * ny
        s1 = H1 * ny
        lam = H1 * (Py // 2 + 1) * eb
        return [M * eb + s1 * cb, 2 * s1 * cb + lam, s1 * cb + M * eb]
    nx, ny, nz = n
    Px, Py, Pz = P
    H1 = Px // 2 + 1
    M = nx * ny * nz
    s1 = H1 * ny * nz
    s2 = H1 * Py * nz
    lam = H1 * (Py // 2 + 1) * (Pz // 2 + 1) * eb
    return [M * eb + s1 * cb, s1 * cb + s2 * cb, 2 * s2 * cb + lam, s2 * cb + s1 * cb, s1 * cb + M * eb]


def stage_flops(d, n, P):
    if d == 2:
        f = fft_flops_2d(n, P)
        return [f["r2c"], f["colmul"], f["c2r"]]
    nx, ny, nz = n
    Px, Py, Pz = P
    H1 = Px // 2 + 1
    rows = ny * nz * 2.5 * Px * math.log2(Px)
    yf = H1 * nz * 5 * Py * math.log2(Py)
    zc = H1 * Py * (2 * 5 * Pz * math.log2(Pz) + 2 * Pz)
    return [rows, yf, zc, yf, rows]


# ----------------------------------------------------------------------------- reference arm (CPU oracle)
def oracle_apply_setup(d, N, alpha):
    from oracle import fast, scheme
    h = 2.0 / N
    a = scheme.coefficients(d, alpha, h, N)
    c = scheme.c_d_alpha(d, alpha)
    Ns = (N,) * d
    op = fast.FastOperator(a, c, tuple(N - 1 for _ in range(d)))
    return op, Ns


def cpu_oracle_rate(d=2, N=NGRID, alpha=ALPHA, budget_s=15.0, min_applies=1):
    op, Ns = oracle_apply_setup(d, N, alpha)
    u = inp.normal_field(Ns, seed=2)
    M = u.size
    t0 = time.perf_counter()
    count = 0
    while count < min_applies or time.perf_counter() - t0 < budget_s:
        op(u)
        count += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": count * M / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{count} FP64 applies of the {N - 1}^{d} alpha={alpha} NumPy-FFT oracle "
                      f"(circulant embedding, pocketfft single thread) in {dt:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    D = args.dims
    NG, AL = (NGRID, ALPHA) if D == 2 else (NGRID_3D, ALPHA_3D)
    op, Ns = oracle_apply_setup(D, NG, AL)
    u = inp.normal_field(Ns, seed=2)
    M = u.size
    for _ in range(args.warmup):
        op(u)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        op(u)  # one step = one apply (a bounded sample of the 8-apply batch)
    dt = time.perf_counter() - t0
    value = args.steps * M / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"{D}D {NG - 1}^{D} alpha={AL} FP64 apply, CPU oracle",
                                             "step": "1 apply", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} NumPy-FFT oracle applies after {args.warmup} warm-up"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def max_over_ranks(dist, ms, device):
    """The slowest rank's time (the job's time) on every rank; ms itself without a process group."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, batch, unknowns, total_ms):
    """Whole-job unknowns/s: every rank applies steps x batch vectors of `unknowns` in the job's time."""
    return world * steps * batch * unknowns / (total_ms / 1e3)


def time_applies(fl, torch, plan, U, Y, work, steps, warmup, d, barrier=None):
    """Time `steps` steps, each one batched apply of all of U (shape (batch, *plan.shape)) with one
    launch per stage.  Returns (total_ms, per-stage ms per instance (launch time / batch), launches)."""
    ns = fl.frlap_apply_nstages(plan)
    B = U.shape[0]
    stream = torch.cuda.current_stream()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(ns + 1)] for _ in range(steps)]
    for row in evs:  # create the events
        for e in row:
            e.record(stream)
    for _ in range(warmup):
        fl.frlap_apply_batch(plan, U, Y, work)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        fl.frlap_apply_batch(plan, U, Y, work, events=evs[k])
    e1.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    total = e0.elapsed_time(e1)
    st = [statistics.mean(evs[k][s].elapsed_time(evs[k][s + 1]) for k in range(steps)) / B for s in range(ns)]
    return total, st, steps * ns


def batch_workspace(fl, torch, plan, B):
    nb = fl.frlap_apply_batch_workspace_bytes(plan, B)
    raw = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    off = (-raw.data_ptr()) % 256
    return raw[off:off + nb]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="frlap", choices=["frlap", "reference"])
    ap.add_argument("--prec", default="df64", choices=["f64", "f32", "df64"])
    ap.add_argument("--suite", default="apply", choices=["apply", "solvers"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--dims", type=int, default=2, choices=[2, 3],
                    help="2: the 2047^2 workload (default); 3: 255^3, alpha = 1.0, 2 vectors per step")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.suite == "solvers":
        run_solver_suite(args)
        return

    import torch
    import paper_1804_02718_gb300 as fl
    from paper_1804_02718_gb300 import build as _build

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    barrier = (lambda: dist.barrier()) if dist else None
    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()

    prec = {"f32": fl.FRLAP_F32, "f64": fl.FRLAP_F64, "df64": fl.FRLAP_DF64}[args.prec]
    dt = torch.float32 if args.prec == "f32" else torch.float64
    eb = 4 if args.prec == "f32" else 8
    # the workload: 2D 2047^2, alpha = 1.5, 8 vectors per step (default) or 3D 255^3, alpha = 1.0, 2 vectors
    D = args.dims
    NG, AL, BATCH = (NGRID, ALPHA, BATCH_2D) if D == 2 else (NGRID_3D, ALPHA_3D, BATCH_3D)
    h = 2.0 / NG
    Ns = (NG,) * D
    plan = fl.Plan(D, AL, h, Ns, prec=prec)
    tuned = fl.frlap_plan_autotune(plan, BATCH)  # launch shapes, before the timed region
    U = torch.stack([torch.from_numpy(inp.normal_field(Ns, seed=100 + b)) for b in range(BATCH)]).to("cuda", dt)
    Y = torch.empty_like(U)
    work = batch_workspace(fl, torch, plan, BATCH)

    clocks = ClockSampler(local)
    clocks.start()
    total_ms, stage_ms, launches = time_applies(fl, torch, plan, U, Y, work, args.steps, args.warmup, D, barrier)
    clk = clocks.stop()
    total_ms = max_over_ranks(dist, total_ms, "cuda")
    M = plan.M
    value = job_throughput(world, args.steps, BATCH, M, total_ms)

    # roofline of the dominant kernel
    names = stage_names(D)
    sb = stage_bytes(D, plan.n, plan.P, eb)
    sf = stage_flops(D, plan.n, plan.P)
    dom = int(np.argmax(stage_ms))
    hbm, hbm_src = peaks()
    if args.prec == "f64":
        ach = sf[dom] / (stage_ms[dom] / 1e3) / 1e12
        roof = {"kernel": names[dom], "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "FP64 pipe: 152 SMs x 4 flop/clk x 2.07 GHz",
                "flops_per_launch": sf[dom] * BATCH}
    elif args.prec == "df64":
        # FFT flops counted as FP64-equivalent operations, each executed as a double-float sequence
        # on the FP32 pipes; peak = FP32 issue rate / FP32 instructions per FP64-equivalent flop
        ach = sf[dom] / (stage_ms[dom] / 1e3) / 1e12
        ipf = df64_instr_per_flop(names[dom], plan.P)
        peak = FP32_ISSUE / ipf / 1e12
        roof = {"kernel": names[dom], "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s (FP64-equivalent, double-float)", "frac": ach / peak,
                "traffic": MEASURED_TRAFFIC.get((D, names[dom], args.prec)),
                "peak_source": f"FP32 issue rate (152 SMs x 128 lanes x 2.07 GHz) / {ipf:.2f} FP32 instructions "
                               "per FP64-equivalent flop of this kernel's double-float butterflies",
                "flops_per_launch": sf[dom] * BATCH}
    else:
        ach = sb[dom] / (stage_ms[dom] / 1e3) / 1e9
        roof = {"kernel": names[dom], "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": MEASURED_TRAFFIC.get((D, names[dom], args.prec)),
                "peak_source": f"{hbm_src} hbm_gbs", "bytes_per_launch": sb[dom] * BATCH}
    roof["instances_per_launch"] = BATCH
    roof["launch_ms"] = stage_ms[dom] * BATCH
    apply_ms = sum(stage_ms)
    model_bytes = sum(sb)
    kernels = {nm: {"ms": round(ms, 5), "model_GBps": round(b / (ms / 1e3) / 1e9, 1),
                    "GFLOPps": round(f / (ms / 1e3) / 1e9, 1)} for nm, ms, b, f in zip(names, stage_ms, sb, sf)}

    # end to end through host buffers (pinned), same batch, H2D + applies + D2H each step
    e2e = None
    if rank == 0 or world > 1:
        # the library's host-buffer batch (frlap_apply_host): chunks of E2E_CHUNK vectors, the
        # copies in and out overlapped with the applies of the neighbouring chunks
        Uh = U.cpu().pin_memory()
        Yh = torch.empty_like(Uh).pin_memory()
        hwork = fl.frlap_apply_host_workspace_bytes(plan, E2E_CHUNK)
        hraw = torch.empty(hwork + 256, dtype=torch.uint8, device="cuda")
        hoff = (-hraw.data_ptr()) % 256
        hw = hraw[hoff:hoff + hwork]
        ksteps = max(2, min(args.steps, 10))
        for _ in range(2):
            fl.frlap_apply_host(plan, Uh, Yh, chunk=E2E_CHUNK, work=hw)
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(ksteps):
            fl.frlap_apply_host(plan, Uh, Yh, chunk=E2E_CHUNK, work=hw)
        z.record()
        torch.cuda.synchronize()
        ems = a.elapsed_time(z)
        del hraw, hw
        e2e = {"value": world * ksteps * BATCH * M / (ems / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": BATCH * M * eb, "d2h_bytes_per_step": BATCH * M * eb, "steps": ksteps,
               "call": f"frlap_apply_host (pinned host buffers, chunks of {E2E_CHUNK})"}

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(fl, torch, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_rate(d=D, N=NG, alpha=AL)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"df64": "f32x2"}.get(args.prec, args.prec),
            "data": "synthetic",
            "config": {"workload": f"{D}D {NG - 1}^{D} alpha={AL} {args.prec.upper()} FFT Toeplitz apply",
                       "batch_per_step": BATCH, "launch": "frlap_apply_batch (one launch per stage for the batch)",
                       "lines_per_cta": {"fp64_side": tuned[0][:3], "fp32": tuned[1][:3],
                                         "chosen_by": "frlap_plan_autotune"},
                       "embedding": list(plan.P),
                       "l2": f"inputs larger than L2 ({BATCH} distinct {NG - 1}^{D} vectors per step)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof,
            "apply": {"ms": apply_ms, "model_bytes": model_bytes,
                      "model_GBps": model_bytes / (apply_ms / 1e3) / 1e9,
                      "frac_of_hbm_model": model_bytes / (apply_ms / 1e3) / 1e9 / hbm, "kernels": kernels},
            "gpu_launches": launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_extras(fl, torch, args):
    """Secondary measurements (not part of the timed region): FP32 / 3D applies and CG solves."""
    out = {}
    cases = [("apply_2047^2_f32", 2, NGRID, fl.FRLAP_F32, 8), ("apply_2047^2_f64", 2, NGRID, fl.FRLAP_F64, 8),
             ("apply_2047^2_df64", 2, NGRID, fl.FRLAP_DF64, 8),
             ("apply_255^3_f64", 3, 256, fl.FRLAP_F64, 1), ("apply_255^3_df64", 3, 256, fl.FRLAP_DF64, 1),
             ("apply_255^3_f32", 3, 256, fl.FRLAP_F32, 2)]
    hbm, _ = peaks()
    for name, d, N, prec, batch in cases:
        dt = torch.float32 if prec == fl.FRLAP_F32 else torch.float64
        eb = 4 if prec == fl.FRLAP_F32 else 8
        plan = fl.Plan(d, ALPHA if d == 2 else 1.0, 2.0 / N, (N,) * d, prec=prec)
        fl.frlap_plan_autotune(plan, batch)
        U = torch.randn((batch,) + plan.shape, dtype=dt, device="cuda")
        Y = torch.empty_like(U)
        work = batch_workspace(fl, torch, plan, batch)
        steps = 5 if (d == 3 and prec != fl.FRLAP_F32) else 10
        total, st, _ = time_applies(fl, torch, plan, U, Y, work, steps, 2, d)
        sb = stage_bytes(d, plan.n, plan.P, eb)
        ms = sum(st)
        out[name] = {"unknowns_per_s": plan.M / (ms / 1e3), "ms": ms, "model_GBps": sum(sb) / (ms / 1e3) / 1e9,
                     "frac_of_hbm_model": sum(sb) / (ms / 1e3) / 1e9 / hbm,
                     "kernels_ms": [round(v, 5) for v in st]}
        del plan, U, Y, work
        torch.cuda.empty_cache()
    # cuFFT (torch.fft) on the same embedding, as a timed comparison (not on the product path)
    for name, prec in (("cufft_2047^2_f64", fl.FRLAP_F64), ("cufft_2047^2_f32", fl.FRLAP_F32)):
        out[name] = cufft_compare(fl, torch, prec, 8)
        torch.cuda.empty_cache()
    # CG: 63^2 with f = 1 and 2047^2 with the Gaussian-sum f, plain FP64 CG vs FP32-inner refinement
    for name, N, f_kind, solver in [("cg_63^2_f1_fp64", 64, "one", fl.FRLAP_SOLVE_CG),
                                    ("cg_2047^2_gauss_fp64", 2048, "gauss", fl.FRLAP_SOLVE_CG),
                                    ("ir_2047^2_gauss_fp32inner", 2048, "gauss", fl.FRLAP_SOLVE_IR)]:
        h = 2.0 / N
        prec = fl.FRLAP_MIXED if solver == fl.FRLAP_SOLVE_IR else fl.FRLAP_F64
        plan = fl.Plan(2, ALPHA, h, (N, N), prec=prec)
        f = inp.constant_field((N, N)) if f_kind == "one" else inp.gaussian_sum_field((N, N), h, seed=3)
        ft = torch.from_numpy(f).cuda()
        x = torch.zeros_like(ft)
        fl.frlap_pcg_solve(plan, ft, x.clone(), rtol=1e-10, solver=solver, inner_rtol=1e-4, raise_on_error=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, it, rel, code = fl.frlap_pcg_solve(plan, ft, x, rtol=1e-10, solver=solver, inner_rtol=1e-4,
                                              raise_on_error=False)
        torch.cuda.synchronize()
        out[name] = {"s": time.perf_counter() - t0, "iters": it, "relres": rel, "status": code}
        del plan
        torch.cuda.empty_cache()
    return out


def cufft_compare(fl, torch, prec, batch, steps=10):
    """The 2047^2 apply of the bench computed with cuFFT through torch.fft: zero-pad each vector to
    P x P, real-to-complex 2D FFT, multiply by the symbol (the plan's own, 1/P^2 folded in), inverse,
    crop.  Returns its time per vector and its normwise difference from frlap_apply_batch."""
    dt = torch.float32 if prec == fl.FRLAP_F32 else torch.float64
    plan = fl.Plan(2, ALPHA, 2.0 / NGRID, (NGRID, NGRID), prec=prec)
    ny, nx = plan.shape
    Py, Px = plan.P[1], plan.P[0]
    oct_ = plan.symbol()  # (Py/2+1, Px/2+1), natural order
    ky = torch.arange(Py, device="cuda")
    lam = oct_[torch.minimum(ky, Py - ky)].to(dt)  # (Py, Px/2+1)
    U = torch.randn((batch, ny, nx), dtype=dt, device="cuda")
    Z = torch.zeros((batch, Py, Px), dtype=dt, device="cuda")
    Y = torch.empty_like(U)

    def run():
        Z[:, :ny, :nx].copy_(U)
        X = torch.fft.rfft2(Z)
        X.mul_(lam)
        Y.copy_(torch.fft.irfft2(X, s=(Py, Px), norm="forward")[:, :ny, :nx])

    for _ in range(3):
        run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        run()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps / batch
    Yf = fl.frlap_apply_batch(plan, U)
    diff = (torch.linalg.norm((Y - Yf).double()) / torch.linalg.norm(Yf.double())).item()
    return {"ms_per_vector": ms, "unknowns_per_s": plan.M / (ms / 1e3), "rel_diff_vs_frlap": diff,
            "what": "torch.fft rfft2/irfft2 on the zero-padded P x P grid + symbol multiply + crop"}


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out


def run_solver_suite(args):
    """Time to 1e-10 (true relative residual) for the solver configurations, one GPU."""
    import torch
    import paper_1804_02718_gb300 as fl
    from paper_1804_02718_gb300 import build as _build, learned
    _build.build()
    out = {"suite": "solvers", "rtol": 1e-10}
    # learned network: trained once on plain-CG pairs (2D 63^2 and 3D 15^3, alpha 0.5..1.9)
    t_train, params2 = _timed(lambda: learned.train(
        [learned.PairSet(2, al, 64, [inp.gaussian_sum_field((64, 64), 2 / 64, seed=s) for s in (6, 7)], K=400)
         for al in (0.5, 0.9, 1.3, 1.7, 1.9)], steps=400, batch=8, lr=2e-3, seed=0)[0])
    t_train3, params3 = _timed(lambda: learned.train(
        [learned.PairSet(3, al, 16, [inp.gaussian_sum_field((16, 16, 16), 2 / 16, seed=s) for s in (6, 7)], K=300)
         for al in (0.5, 0.9, 1.3, 1.7, 1.9)], steps=300, batch=8, lr=2e-3, seed=0)[0])
    out["train_s"] = {"2d": t_train, "3d": t_train3}

    def solve_row(d, N, alpha, seed, variants):
        h = 2.0 / N
        f = torch.from_numpy(inp.gaussian_sum_field((N,) * d, h, seed=seed)).cuda()
        row = {}
        for name, prec, solver, pre in variants:
            plan = fl.Plan(d, alpha, h, (N,) * d, prec=prec)
            fl.frlap_plan_autotune(plan, 1)  # launch shapes (not part of the solve time)
            if pre == fl.FRLAP_PRECOND_STRANG:
                fl.frlap_precond_strang(plan)
            elif pre == fl.FRLAP_PRECOND_LEARNED:
                learned.install(plan, params2 if d == 2 else params3)
            plan.workspace(fl.FRLAP_OP_PCG)
            dt, (x, it, rel, code) = _timed(lambda: fl.frlap_pcg_solve(plan, f, rtol=1e-10, solver=solver,
                                                                     precond=pre, inner_rtol=1e-4,
                                                                     raise_on_error=False))
            row[name] = {"s": dt, "iters": it, "relres": rel, "status": code}
            del plan
            torch.cuda.empty_cache()
        return row

    F64, DF, MX = fl.FRLAP_F64, fl.FRLAP_DF64, fl.FRLAP_MIXED_DF64
    CG, IR = fl.FRLAP_SOLVE_CG, fl.FRLAP_SOLVE_IR
    NONE, STR, LRN = fl.FRLAP_PRECOND_NONE, fl.FRLAP_PRECOND_STRANG, fl.FRLAP_PRECOND_LEARNED
    full = [("plain_cg_fp64", F64, CG, NONE), ("plain_cg_df64", DF, CG, NONE), ("pcg_strang_df64", DF, CG, STR),
            ("pcg_learned_df64", DF, CG, LRN), ("ir_learned_fp32inner", MX, IR, LRN)]
    fast = [("pcg_strang_df64", DF, CG, STR), ("pcg_learned_df64", DF, CG, LRN), ("ir_strang_fp32inner", MX, IR, STR),
            ("ir_learned_fp32inner", MX, IR, LRN)]
    out["2d_2047_alpha1.5"] = solve_row(2, 2048, 1.5, 1, full)
    for al in (0.5, 1.0, 1.5, 1.9):
        out[f"3d_255_alpha{al}"] = solve_row(3, 256, al, 1, full if al in (1.0, 1.9) else fast)
    for al in (1.2, 1.8):
        out[f"2d_4095_alpha{al}"] = solve_row(2, 4096, al, 3, fast + [("plain_cg_df64", DF, CG, NONE)])
        out[f"3d_511_alpha{al}"] = solve_row(3, 512, al, 3, fast)
    # batched Allen-Cahn: 64 instances, alpha ~ U[1.2,1.9], grids 255/511/1023, 200 steps, one graph launch
    batch = inp.allen_cahn_batch()
    plans = [fl.Plan(2, al, 2.0 / (n + 1), (n + 1, n + 1), prec=fl.FRLAP_DF64) for al, n, _ in batch]
    # the first plan of each grid leads its group in the batched launch: tune its launch shapes
    for n in sorted({n for _, n, _ in batch}):
        first = next(i for i, (_, m, _) in enumerate(batch) if m == n)
        fl.frlap_plan_autotune(plans[first], sum(1 for _, m, _ in batch if m == n))
    us = [torch.from_numpy(u0).cuda() for _, _, u0 in batch]
    dt, (its, st, code) = _timed(lambda: fl.frlap_allen_cahn_batch(plans, us, 1e-3, 0.05, 200, rtol=1e-10,
                                                                   raise_on_error=False))
    unknown_steps = sum(u.numel() for u in us) * 200
    out["allen_cahn_batch_64x200"] = {"s": dt, "status": code, "total_cg_iters": int(sum(its)),
                                     "unknown_steps_per_s": unknown_steps / dt,
                                     "max_abs_u": max(float(u.abs().max().item()) for u in us)}
    # the paper's own Allen-Cahn example (Crank-Nicolson, u = -1 outside, kissing bubbles, delta = 0.03,
    # tau = 5e-4 until t = 0.015 = 30 steps), at the grids and alphas of its CPU-time table Tab10
    cn = {}
    for N in (128, 256, 512, 1024):
        for al in (1.9, 1.5, 1.0, 0.7):
            h = 1.0 / N
            plan = fl.Plan(2, al, h, (N, N), prec=fl.FRLAP_DF64)
            fl.frlap_plan_autotune(plan, 1)
            ub = torch.from_numpy(inp.kissing_bubbles((N, N), h, 0.03) + 1.0).cuda()
            plan.workspace(fl.FRLAP_OP_AC)
            dt, (its, mass) = _timed(lambda: fl.frlap_allen_cahn_cn(plan, ub, 5e-4, 0.03, 30, rtol=1e-10))
            cn[f"N{N}_alpha{al}"] = {"s": dt, "cg_iters": its, "mass_t0.015": mass[-1]}
            del plan, ub
            torch.cuda.empty_cache()
    out["paper_allen_cahn_cn_to_t0.015"] = cn
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

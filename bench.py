"""Benchmark of the quantum-trajectory hot path on GB300.

One step = one pass of the whole path over one batch: the trajectory kernel
(Algorithm 1 of the QTM paper for every trajectory of the batch, with its
Dormand-Prince integration, jump location, channel choice and observables) plus
the FP64 ensemble reduction, on inputs already resident in device memory.

Default workload: the damped, driven Jaynes-Cummings model (cavity Fock cutoff
30 x qubit, N = 60, two collapse operators, 401 output times over t in [0, 40],
observables a^dag a and sigma_+ sigma_-), 20,000 trajectories per GPU, complex128
arithmetic, rtol 1e-8 / atol 1e-10, Philox seed 1.  Under torchrun each rank runs
its own 20,000 trajectory ids (weak scaling); the FP64 sums are combined with one
all-reduce per step.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (the
reference arm: there is no reference implementation to run, only the paper).

Prints one JSON line (rank 0).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "trajectories/sec at ≤1e-5 observable error vs plain FP64 GPU path; roofline %"
UNIT = "trajectories/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ntraj", type=int, default=20000, help="trajectories per GPU per step")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="c128", choices=["c128", "df64", "c64"],
                    help="trajectory arithmetic: complex128, double-float or complex64")
    return ap.parse_args()


def workload(ntraj):
    from paper_1810_03047_gb300 import systems as S
    prob = S.jaynes_cummings_driven(ntraj=ntraj)
    nnz_m = _nnz_effective(prob)
    desc = (f"damped driven Jaynes-Cummings, N={prob.dim} (Fock 30 x qubit), 2 collapse ops, "
            f"CSR nnz(H_eff)={nnz_m}, {len(prob.t)} outputs on [0,{prob.t[-1]:g}], "
            f"{ntraj} trajectories per GPU, rtol {prob.rtol:g} atol {prob.atol:g}, seed {prob.seed}")
    return prob, nnz_m, desc


def _nnz_effective(prob):
    M = (-1j * prob.H - 0.5 * sum(c.conj().T @ c for c in prob.C)).tocsr()
    M.eliminate_zeros()
    return int(M.nnz)


def flops_per_attempt(n, nnz_m):
    # Dormand-Prince step: 6 new stage products M y (8 flops per complex
    # multiply-add) and 26 real-coefficient complex axpys (4 flops per element).
    return 6 * 8 * nnz_m + 26 * 4 * n


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# FP64 FMA units: GB300 lists 1.25 TFLOP/s dense FP64; at the 2070 MHz maximum SM
# clock over 152 SMs that is 2 FP64 FMA per SM per clock.
FP64_FMA_PER_SM_CLK = 2
SMS = 152
SM_MAX_MHZ = 2070.0


def cpu_baseline(prob, seconds, rank):
    """The FP64 oracle on this host's cores on a bounded sample of the same workload."""
    from oracle import oracle
    nthreads = os.cpu_count() or 1
    pilot = max(nthreads * 4, 64)
    t0 = time.perf_counter()
    r = oracle.mcwf(prob, ntraj=pilot, nthreads=nthreads, max_jumps=1)
    dt = time.perf_counter() - t0
    if r["rc"] != 0:
        raise RuntimeError(f"oracle failed: {r['rc']}")
    n = int(min(prob.ntraj, max(pilot, pilot * seconds / max(dt, 1e-6))))
    t0 = time.perf_counter()
    r = oracle.mcwf(prob, ntraj=n, nthreads=nthreads, max_jumps=1)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"trajectory ids 0..{n - 1} of the same workload ({n} of {prob.ntraj}), "
                      f"{dt:.1f} s wall on {nthreads} host threads"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle
    prob, nnz_m, desc = workload(args.ntraj)
    nthreads = os.cpu_count() or 1
    per_step = max(nthreads * 8, 128)
    oracle.build()
    for _ in range(args.warmup):
        oracle.mcwf(prob, ntraj=max(nthreads, 16), nthreads=nthreads, max_jumps=1)
    total = 0.0
    done = 0
    for s in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.mcwf(prob, traj0=s * per_step, ntraj=per_step, nthreads=nthreads, max_jumps=1)
        total += time.perf_counter() - t0
        done += per_step
        if r["rc"] != 0:
            raise RuntimeError(f"oracle failed: {r['rc']}")
    value = done / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "ntraj_per_step": per_step,
                       "l2": "n/a (host)", "parallelism": f"{nthreads} host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": f"{per_step} trajectories per step, ids 0..{done - 1}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_1810_03047_gb300 import qtm as Q

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    prob, nnz_m, desc = workload(args.ntraj)
    ntraj = args.ntraj
    first = rank * ntraj
    stream = torch.cuda.current_stream()
    Q.use_torch_allocator()
    prec = {"c128": Q.QTM_PREC_C128, "df64": Q.QTM_PREC_DF64, "c64": Q.QTM_PREC_C64}[args.precision]
    ctx = Q.qtm_create(prob, stream=int(stream.cuda_stream), precision=prec)
    P = len(prob.t) * len(prob.A)
    sums = torch.zeros(2 * P, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def step():
        Q.qtm_run_range(ctx, first, ntraj, prob.seed)
        if world > 1:
            Q.qtm_sums_device(ctx, sums.data_ptr(), sums.data_ptr() + 8 * P)
            dist.all_reduce(sums)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    st = Q.qtm_stats(ctx)
    if st["failed"]:
        raise RuntimeError(f"warm-up run failed: {st}")

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = 0.0
    kernel_ms = []
    attempts = 0
    launches = 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        s = Q.qtm_stats(ctx)
        kernel_ms.append(s["kernel_ms"])
        attempts += s["accepted"] + s["rejected"]
        launches += 5  # trajectory kernel + four reduction kernels
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    mean, se = Q.qtm_expect(ctx)
    last = Q.qtm_stats(ctx)

    # end to end through the public API with host buffers: create (H2D of the
    # problem), run, expect (D2H of mean and standard error), destroy
    e2e_steps = max(1, min(args.steps, 3))
    h2d = d2h = 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        c2 = Q.qtm_create(prob, stream=int(stream.cuda_stream), precision=prec)
        Q.qtm_run_range(c2, first, ntraj, prob.seed)
        Q.qtm_expect(c2)
        Q.qtm_destroy(c2)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_s = float(te.item())
    h2d = (sum((m.indptr.nbytes // 2 + m.indices.nbytes // 2 + m.data.nbytes) for m in [prob.H] + prob.C + prob.A)
           + prob.psi0.nbytes + prob.t.nbytes)
    d2h = 2 * P * 8 + 4

    value = world * ntraj * args.steps / (total_ms / 1e3)
    F = flops_per_attempt(prob.dim, nnz_m)
    kern_avg_ms = sum(kernel_ms) / len(kernel_ms)
    achieved = F * (attempts / args.steps) / (kern_avg_ms / 1e3) / 1e12
    fp64_peak = SMS * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "ntraj_per_gpu": ntraj, "precision": "c128",
                   "l2": "flushed between steps (256 MB write); operators are L2/SMEM-resident by design",
                   "parallelism": f"trajectory shards, {world} GPU(s)"},
        "observable_error": 0.0,
        "observable_error_note": "the complex128 path is the plain FP64 GPU path itself",
        "rhs_evals_per_s": world * last["rhs_evals"] / (total_ms / 1e3 / args.steps),
        "steps_per_trajectory": attempts / args.steps / ntraj,
        "jumps_per_trajectory": last["jumps"] / ntraj,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp64_peak, "traffic": None,
                     "kernel": "qtm::mcwf_kernel<double,32,2>",
                     "peak_note": "FP64 FMA pipe, 152 SMs x 2 FMA/clk x 2070 MHz (nominal 1.25 TFLOP/s)",
                     "kernel_ms": kern_avg_ms},
        "e2e": {"value": world * ntraj * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, args.cpu_seconds, rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    Q.qtm_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

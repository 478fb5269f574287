"""Benchmark of the quantum-trajectory hot path on GB300.

One step = one pass of the whole path over one batch: the trajectory kernel
(Algorithm 1 of the QTM paper for every trajectory of the batch, with its
Dormand-Prince integration, jump location, channel choice and observables) plus
the exact ensemble reduction (integer sums of the quantised values, from which
the FP64 mean and standard error follow), on inputs already resident in device
memory.

Default workload: the damped, driven Jaynes-Cummings model (cavity Fock cutoff
30 x qubit, N = 60, two collapse operators, 401 output times over t in [0, 40],
observables a^dag a and sigma_+ sigma_-), 20,000 trajectories per GPU, rtol 1e-8 /
atol 1e-10, Philox seed 1.  The same ensemble is timed in three arithmetics:
complex128 (the plain FP64 GPU path, whose means are the reference), the
double-float path (FP64-class precision on the FP32 pipe) and complex64; the
headline `value` is the fastest path whose ensemble stays within 1e-5 of the
complex128 means.  Under torchrun each rank runs
its own 20,000 trajectory ids (weak scaling); the shards' exact moment words are
combined with one integer all-reduce per step (exact, so independent of the
collective's order).

``--impl reference`` times the FP64 CPU oracle on the host cores instead (the
reference arm: there is no reference implementation to run, only the paper).

Prints one JSON line (rank 0).
"""

from __future__ import annotations

import argparse
import platform
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
# kernels per qtm_run: the trajectory kernel and the two exact-moment kernels of
# the ensemble reduction
RUN_LAUNCHES = 3

# DRAM bytes (read + write) of one launch at full size, from one ncu capture with
# `--metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
# --clock-control none -s 1 -c 1` (one pass) of the timed launch of
# `python bench.py --only df64 --steps 1 --warmup 1` (-k regex:mcwf_kernel) and
# `python bench.py --only dense --steps 1 --warmup 1` (-k regex:dense_tc_kernel).
# Valid for the kernels as captured; a change to a kernel voids its entry.
# dram__bytes_read.sum + dram__bytes_write.sum of one launch at the bench's size
# (one ncu pass, profiles/); an entry is removed when its kernel changes
TRAFFIC_PER_LAUNCH = {
    "qtm::mcwf_kernel<df64,32,2>": 14.04e6 + 236.46e6,   # 20,000 JC trajectories: outputs and spill evictions
    "qtm::dense_tc_kernel<256>": 55.05e9 + 55.78e9,      # 20,000 dense trajectories, seven products per attempt
}


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
    ap.add_argument("--no-peak-probe", action="store_true",
                    help="skip the arithmetic-peak probes (profiling runs): roofline against the nominal peaks")
    ap.add_argument("--no-paper", action="store_true",
                    help="skip the paper's own examples (Sec. 4.1 unitary, Sec. 4.2 trilinear OPA)")
    ap.add_argument("--no-dense", action="store_true",
                    help="skip the dense tensor-core measurement (N = 256, 20,000 trajectories)")
    ap.add_argument("--no-proposal", action="store_true",
                    help="skip the learned jump-time proposal measurement (200,000 JC trajectories)")
    ap.add_argument("--no-expo", action="store_true",
                    help="skip the exponential-method legs (stiff Purcell system, Jaynes-Cummings)")
    ap.add_argument("--no-ising", action="store_true",
                    help="skip the batched Ising-chain measurement (L = 6..10 in one CUDA graph)")
    ap.add_argument("--only", choices=["c128", "df64", "c64", "dense", "expo_purcell", "expo_jc", "expo_dense",
                                       "expo_tc", "expo_prop", "peak"],
                    default=None,
                    help="time one arithmetic only (profiling); no observable-error comparison.  'dense': the "
                         "tensor-core engine on the dense N = 256 system with --ntraj trajectories")
    ap.add_argument("--dense-t-end", type=float, default=10.0, help="--only dense: end of the time grid")
    ap.add_argument("--dense-outputs", type=int, default=101, help="--only dense: number of output times")
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
    # one core on a smaller sample, for the per-core rate
    n1 = max(8, min(64, n // max(nthreads, 1)))
    t1 = time.perf_counter()
    oracle.mcwf(prob, ntraj=n1, nthreads=1, max_jumps=1)
    dt1 = time.perf_counter() - t1
    return {"value": n / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"trajectory ids 0..{n - 1} of the same workload ({n} of {prob.ntraj}), "
                      f"{dt:.1f} s wall on {nthreads} host threads",
            "one_core_value": n1 / dt1, "one_core_sample": f"trajectory ids 0..{n1 - 1} on one thread",
            "cpu_model": _cpu_model()}


def _cpu_model() -> str:
    """The host CPU's model name (Linux /proc/cpuinfo; Arm cores report their part number)."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        return platform.processor() or platform.machine()
    for key in ("model name", "Model name", "CPU part"):
        for line in info.splitlines():
            if line.split(":")[0].strip() == key:
                return f"{platform.machine()} {key}: {line.split(':', 1)[1].strip()}"
    return platform.machine()


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
                             "sample": f"{per_step} trajectories per step, ids 0..{done - 1}",
                             "cpu_model": _cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# FP32 pipe: 152 SMs x 128 lanes at 2070 MHz issue 40.3e12 FP32 instructions/s.
# A double-float multiply-add (TwoProd, two cross FMAs, TwoSum, two adds) takes 12
# FP32 instructions for 2 FP64-class flops, so the emulated FP64 peak is 1/6 of
# the FP32 instruction rate.
FP32_LANES_PER_SM = 128
DF_INSTR_PER_FLOP = 6


def nominal_peaks():
    """Peaks from the unit counts and the maximum SM clock (context for the measured ones)."""
    fp64 = SMS * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    fp32_instr = SMS * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6
    return {"c128": fp64, "df64": fp32_instr / DF_INSTR_PER_FLOP / 1e12, "c64": 2 * fp32_instr / 1e12}


def peaks(measured=None):
    """Roofline denominators: the arithmetic peaks measured in this run (probe
    kernels, of measured), falling back to the nominal unit-count figures."""
    nom = nominal_peaks()
    m = measured or {}
    out = {}
    for key, probe, what in (("c128", "fp64", "FP64 FMA chains"), ("c64", "fp32", "FP32 FMA chains"),
                             ("df64", "df64", "double-float multiply-add chains (12 FP32 instructions, 2 FP64-class "
                                              "flop each)")):
        if m.get(probe):
            out[key] = (m[probe], f"measured in this run by the probe kernel ({what} on every SM, CUDA events), "
                                  f"of measured; nominal {nom[key]:.3g} TFLOP/s from unit counts at 2070 MHz")
        else:
            out[key] = (nom[key], f"nominal from unit counts at 2070 MHz ({what}), no measurement")
    out["hbm"] = _hbm_peak()
    return out


def measured_arith_peaks(Q, torch, stream, seconds=1.0):
    """The arithmetic peaks of this GPU, measured in this run by the library's probe
    kernels (independent multiply-add chains on every SM; qtm_arith_peak_launch),
    timed with CUDA events on `stream`: each probe is calibrated on a short launch,
    then run for about `seconds`, best of three.  TFLOP/s per kind."""
    scratch = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = {}
    for name, kind in (("fp64", Q.QTM_PEAK_FP64), ("fp32", Q.QTM_PEAK_FP32), ("df64", Q.QTM_PEAK_DF64)):
        iters, best = 1000, 0.0
        for rep in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flop = Q.qtm_arith_peak_launch(kind, iters, scratch.data_ptr(), int(stream.cuda_stream))
            e1.record(stream)
            e1.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            if rep >= 2:
                best = max(best, flop / sec / 1e12)
            else:  # calibration launches
                iters = max(1000, int(iters * seconds / max(sec, 1e-6)))
        out[name] = best
    return out


def _bf16x6_peak(sustained=True):
    """Peak of the tensor-core engines' FP32-accurate products: the measured bf16
    dense peak (sustained for kernels inside a long run) over the six bf16
    products each BF16x6 product issues."""
    mp = measured_peaks()
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    if key in mp:
        return float(mp[key]) / 6.0, f"measured cuBLAS bf16 peak (MEASURED_PEAKS.json {key}) / 6, of measured"
    return (1700.0 if sustained else 1900.0) / 6.0, "fallback bf16 peak / 6, of fallback"


def lockstep_launches(n_t, every=16):
    """Kernels of one lock-step exponential run on the tensor cores: a tensor-core
    product per output interval, the per-interval kernel per output, a catch-up
    every `every` intervals and after the last, the finish, and the reduction."""
    catch = sum(1 for j in range(1, n_t) if j % every == 0 or j == n_t - 1)
    return (n_t - 1) + n_t + catch + 1 + (RUN_LAUNCHES - 1)


def _hbm_peak():
    mp = measured_peaks()
    if "hbm_gbs" in mp:
        return float(mp["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), of measured"
    return 6800.0, "fallback 6.8 TB/s (one earlier GB300 measurement), of fallback"


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

    from paper_1810_03047_gb300 import shards
    prob, nnz_m, desc = workload(args.ntraj)
    first, ntraj = shards.shard(world * args.ntraj, world, rank)  # weak scaling: args.ntraj per GPU
    stream = torch.cuda.current_stream()
    Q.use_torch_allocator()
    P = len(prob.t) * len(prob.A)
    words = torch.zeros((P, Q.QTM_MOMENT_WORDS), dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    F = flops_per_attempt(prob.dim, nnz_m)
    arith = {} if args.no_peak_probe else measured_arith_peaks(Q, torch, stream)
    pk = peaks(arith)
    codes = {"c128": Q.QTM_PREC_C128, "df64": Q.QTM_PREC_DF64, "c64": Q.QTM_PREC_C64}

    def timed(prec_name, steps, warmup):
        """Times `steps` passes of the path (trajectory kernel + ensemble reduction,
        plus the integer all-reduce of the moment words across GPUs) with L2
        flushed in between."""
        ctx = Q.qtm_create(prob, stream=int(stream.cuda_stream), precision=codes[prec_name])

        def step():
            Q.qtm_run_range(ctx, first, ntraj, prob.seed)
            if world > 1:
                Q.qtm_moments_device(ctx, words.data_ptr())
                dist.all_reduce(words)

        for _ in range(max(warmup, 0)):
            step()
        torch.cuda.synchronize()
        if Q.qtm_stats(ctx)["failed"]:
            raise RuntimeError(f"{prec_name}: warm-up run failed")
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        total_ms, kernel_ms, attempts, launches = 0.0, [], 0, 0
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            st = Q.qtm_stats(ctx)
            kernel_ms.append(st["kernel_ms"])
            attempts += st["accepted"] + st["rejected"]
            launches += RUN_LAUNCHES
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        mean, se = Q.qtm_expect(ctx)
        if world > 1:  # the whole job's ensemble from the all-reduced words of the last step
            E = Q.qtm_moments(ctx)[2]
            m_all = Q.qtm_combine_moments(words.cpu().numpy(), [world * ntraj], len(prob.A), E)[0]
            mean = m_all.reshape(mean.shape)
        last = Q.qtm_stats(ctx)
        Q.qtm_destroy(ctx)
        kern = sum(kernel_ms) / len(kernel_ms)
        achieved = F * (attempts / steps) / (kern / 1e3) / 1e12
        peak, note = pk[prec_name]
        return {"value": world * ntraj * steps / (total_ms / 1e3), "ms_per_step": total_ms / steps,
                "kernel_ms": kern, "mean": mean, "stats": last, "launches": launches,
                "attempts_per_traj": attempts / steps / ntraj,
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak,
                             "traffic": TRAFFIC_PER_LAUNCH.get(
                                 f"qtm::mcwf_kernel<{prec_name},{last['kernel_group']},{last['kernel_rows']}>")
                             if ntraj == 20000 else None,
                             "kernel": f"qtm::mcwf_kernel<{prec_name},{last['kernel_group']},{last['kernel_rows']}>",
                             "peak_note": note, "kernel_ms": kern}}

    clocks = ClockSampler(local)
    clocks.start()
    if args.only == "peak":
        clk = clocks.stop()
        if rank == 0:
            nom = nominal_peaks()
            print(json.dumps({"metric": "arithmetic peaks (probe kernels)", "unit": "TFLOP/s",
                              "fp64": arith.get("fp64"), "fp32": arith.get("fp32"), "df64": arith.get("df64"),
                              "nominal": {"fp64": nom["c128"], "fp32": nom["c64"], "df64": nom["df64"]},
                              "gpu_launches": 15, "clocks": clk}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return 0
    if args.only == "dense":
        from paper_1810_03047_gb300 import systems as S
        dprob = S.dense_random(ntraj=args.ntraj, t_end=args.dense_t_end, n_t=args.dense_outputs)
        ctx = Q.qtm_create(dprob, stream=int(stream.cuda_stream), precision=Q.QTM_PREC_BF16X6)
        for _ in range(max(args.warmup, 0)):
            Q.qtm_run_range(ctx, first, ntraj, dprob.seed)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            Q.qtm_run_range(ctx, first, ntraj, dprob.seed)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = Q.qtm_stats(ctx)
        Q.qtm_destroy(ctx)
        clk = clocks.stop()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": world * ntraj / (max(ms) / 1e3), "unit": UNIT,
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": max(ms), "higher_is_better": True, "scaling": "weak",
                              "vs_baseline": None, "dtype": "bf16x6-tc/f32", "data": "synthetic",
                              "config": {"workload": f"dense random N=256, t in [0, {args.dense_t_end}], "
                                                     f"{args.dense_outputs} outputs", "ntraj_per_gpu": ntraj},
                              "steps_per_trajectory": (st["accepted"] + st["rejected"]) / ntraj,
                              "gpu_launches": RUN_LAUNCHES * (args.steps + max(args.warmup, 0)), "clocks": clk,
                              "note": "tensor-core engine only (profiling run)"}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return 0
    if args.only in ("expo_tc", "expo_prop"):
        # one leg alone (profiling): the exponential method on the tensor cores on
        # the dense workload, or the learned proposal in the exponential method's
        # crossing search on the Jaynes-Cummings workload, --ntraj trajectories
        if args.only == "expo_tc":
            from paper_1810_03047_gb300 import systems as S
            dprob = S.dense_random(ntraj=args.ntraj)
            r = _timed_passes(Q, torch, stream, world, dist, dprob, Q.QTM_PREC_BF16X6, Q.QTM_METHOD_EXPONENTIAL,
                              first, ntraj, passes=max(1, args.steps))
            r.pop("mean")
        else:
            r = _learned_proposal_expo(Q, torch, stream, world, dist, prob, first, ntraj, ntraj)
        clk = clocks.stop()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": 1, "higher_is_better": True, "scaling": "weak",
                              "vs_baseline": None, "data": "synthetic",
                              "config": {"workload": args.only, "ntraj_per_gpu": ntraj}, "result": r,
                              "gpu_launches": r.get("launches"), "clocks": clk,
                              "note": "one leg only (profiling run)"}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return 0
    if args.only in ("expo_purcell", "expo_jc", "expo_dense"):
        from paper_1810_03047_gb300 import systems as S
        eprob = {"expo_purcell": S.purcell_qubit(ntraj=args.ntraj), "expo_jc": prob,
                 "expo_dense": S.dense_random(ntraj=args.ntraj)}[args.only]
        res = {}
        for pname, prec in (("c128", Q.QTM_PREC_C128), ("df64", Q.QTM_PREC_DF64), ("c64", Q.QTM_PREC_C64)):
            res[pname] = _timed_passes(Q, torch, stream, world, dist, eprob, prec, Q.QTM_METHOD_EXPONENTIAL, first,
                                       ntraj, passes=max(1, args.steps))
        clk = clocks.stop()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": res["c128"]["value"], "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": 1, "ms_per_step": res["c128"]["ms_per_step"],
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                              "data": "synthetic", "config": {"workload": eprob.name, "ntraj_per_gpu": ntraj,
                                                              "method": "exponential"},
                              "df64": {k: v for k, v in res["df64"].items() if k != "mean"},
                              "c64": {k: v for k, v in res["c64"].items() if k != "mean"},
                              "gpu_launches": sum(r["launches"] for r in res.values()), "clocks": clk,
                              "note": "exponential method only (profiling run)"}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return 0
    if args.only:
        only = timed(args.only, args.steps, args.warmup)
        clk = clocks.stop()
        line = {"metric": METRIC, "value": only["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": only["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.only, "data": "synthetic",
                "config": {"workload": desc, "ntraj_per_gpu": ntraj, "precision": args.only,
                           "l2": "flushed between steps (256 MB write)",
                           "parallelism": f"trajectory shards, {world} GPU(s)"},
                "observable_error": None, "roofline": only["roofline"], "gpu_launches": only["launches"],
                "clocks": clk, "note": "single-arithmetic profiling run"}
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return 0
    ref = timed("c128", max(1, min(args.steps, 3)), max(1, min(args.warmup, 3)))
    fast = timed("df64", args.steps, args.warmup)
    mixed = timed("c64", max(1, min(args.steps, 3)), max(1, min(args.warmup, 3)))
    clk = clocks.stop()
    err_df = float(np.abs(fast["mean"] - ref["mean"]).max())
    err_c64 = float(np.abs(mixed["mean"] - ref["mean"]).max())
    head, head_name, head_err = (fast, "df64", err_df) if err_df <= 1e-5 else (ref, "c128", 0.0)

    # end to end through the public API with host buffers: create (H2D of the
    # problem), run, expect (D2H of mean and standard error), destroy
    e2e_steps = max(1, min(args.steps, 3))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        c2 = Q.qtm_create(prob, stream=int(stream.cuda_stream), precision=codes[head_name])
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
    d2h = P * Q.QTM_MOMENT_WORDS * 8 + 4  # qtm_expect reads the moment words and the first-error code

    def side(r, err):
        return {"value": r["value"], "ms_per_step": r["ms_per_step"], "observable_error": err,
                "steps_per_trajectory": r["attempts_per_traj"], "roofline_frac": r["roofline"]["frac"],
                "kernel_ms": r["kernel_ms"]}

    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": head_name, "data": "synthetic",
        "config": {"workload": desc, "ntraj_per_gpu": ntraj, "precision": head_name,
                   "l2": "flushed between steps (256 MB write); operators are shared-memory/L2 resident by design",
                   "parallelism": f"trajectory shards, {world} GPU(s)"},
        "observable_error": head_err,
        "observable_error_note": "max |mean - mean of the complex128 (plain FP64) GPU path| over all output "
                                 "times and observables, same seed and trajectories",
        "fp64_path": side(ref, 0.0),
        "c64_path": dict(side(mixed, err_c64), qualifies=err_c64 <= 1e-5),
        "speedup_vs_fp64_path": head["value"] / ref["value"],
        "rhs_evals_per_s": world * head["stats"]["rhs_evals"] / (head["ms_per_step"] / 1e3),
        "steps_per_trajectory": head["attempts_per_traj"],
        "jumps_per_trajectory": head["stats"]["jumps"] / ntraj,
        "roofline": head["roofline"],
        "e2e": {"value": world * ntraj * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": ref["launches"] + fast["launches"] + mixed["launches"] + (15 if arith else 0),
        "clocks": clk,
        "arithmetic_peaks_tflops": dict(arith, note="measured in this run by the probe kernels "
                                                     "(qtm_arith_peak_launch), best of three ~1 s launches"),
    }
    if not args.no_ising:
        line["ising_batch"] = ising_batch(Q, torch, stream, world, rank, dist, pk)
        line["gpu_launches"] += line["ising_batch"].pop("launches")
    if not args.no_paper:
        line["paper_workloads"] = paper_workloads(Q, torch, stream, world, rank, dist)
        line["gpu_launches"] += line["paper_workloads"].pop("launches")
    if not args.no_dense:
        line["dense_tensor_core"] = dense_tensor_core(Q, torch, stream, world, rank, dist, pk)
        line["gpu_launches"] += line["dense_tensor_core"].pop("launches")
    if not args.no_expo:
        line["exponential_method"] = exponential_method(Q, torch, stream, world, rank, dist, pk, ref["mean"])
        line["gpu_launches"] += line["exponential_method"].pop("launches")
    if not args.no_proposal:
        line["learned_proposal"] = learned_proposal(Q, torch, stream, world, rank, dist)
        line["gpu_launches"] += line["learned_proposal"].pop("launches")
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, args.cpu_seconds, rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def ising_batch(Q, torch, stream, world, rank, dist, pk):
    """The uneven batched ensemble: open transverse-field Ising chains L = 6..10
    (N = 64..1024, 2L channels) with 50k/20k/10k/5k/2k trajectories (seed 7), all
    five systems in one CUDA-graph launch.  Double-float with autotuned lane
    layouts is timed (1 warm-up, 1 timed pass) and compared with the complex128
    batch on the same trajectories.  Roofline: algorithmic flops of every attempt
    of every system (6 * 8 nnz(M) + 26 * 4 N, nnz(M) = (L + 1) N) over the batch
    time, against the measured double-float peak; and the same for the L = 10
    kernel timed alone."""
    from paper_1810_03047_gb300 import shards
    from paper_1810_03047_gb300 import systems as S
    Ls = [6, 7, 8, 9, 10]
    probs = [S.ising_chain(L) for L in Ls]
    counts, firsts = [], []
    for L in Ls:
        f, c = shards.shard(world * S.ISING_TRAJ[L], world, rank)
        firsts.append(f)
        counts.append(c)
    sid = int(stream.cuda_stream)
    ref = [Q.qtm_create(p, stream=sid, precision=Q.QTM_PREC_C128) for p in probs]
    fast = [Q.qtm_create(p, stream=sid, precision=Q.QTM_PREC_DF64) for p in probs]
    layouts = [Q.qtm_autotune(c, min(n, 4096), 7) for c, n in zip(fast, counts)]
    Q.qtm_run_batch(ref, counts, 7, firsts)
    ref_means = [Q.qtm_expect(c)[0] for c in ref]
    ref_ms = []
    for _ in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Q.qtm_run_batch(fast, counts, 7, firsts)
        e1.record(stream)
        e1.synchronize()
        ref_ms.append(e0.elapsed_time(e1))
    ms = ref_ms[-1]
    err = max(float(np.abs(Q.qtm_expect(c)[0] - m).max()) for c, m in zip(fast, ref_means))
    flop = 0.0
    for c, p in zip(fast, probs):
        st = Q.qtm_stats(c)
        flop += flops_per_attempt(p.dim, _nnz_effective(p)) * (st["accepted"] + st["rejected"])
    peak, note = pk["df64"]
    achieved = flop / (ms / 1e3) / 1e12
    # the L = 10 kernel alone (the largest share of the batch's device time)
    c10, p10 = fast[-1], probs[-1]
    Q.qtm_run_range(c10, firsts[-1], counts[-1], 7)
    st10 = Q.qtm_stats(c10)
    a10 = flops_per_attempt(p10.dim, _nnz_effective(p10)) * (st10["accepted"] + st10["rejected"]) \
        / (st10["kernel_ms"] / 1e3) / 1e12
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    for c in ref + fast:
        Q.qtm_destroy(c)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "qtm::mcwf_kernel<df64, autotuned layouts> x 5 systems in one graph",
            "peak_note": note,
            "l10_alone": {"kernel": f"qtm::mcwf_kernel<df64,{st10['kernel_group']},{st10['kernel_rows']}>",
                          "kernel_ms": st10["kernel_ms"], "achieved": a10, "frac": a10 / peak}}
    return {"workload": "transverse-field Ising chains L=6..10 (N=64..1024, J=1, h=0.7, decay 0.05 and "
                        "dephasing 0.02 per site), 50k/20k/10k/5k/2k trajectories, 201 outputs on [0,20], "
                        "one CUDA-graph launch", "precision": "df64",
            "value": world * sum(counts) / (float(t.item()) / 1e3), "unit": UNIT, "ms_per_step": float(t.item()),
            "observable_error": err, "layouts": [list(x) for x in layouts], "roofline": roof,
            "launches": 2 * 5 * RUN_LAUNCHES + RUN_LAUNCHES}


def paper_workloads(Q, torch, stream, world, rank, dist):
    """The paper's own timed examples, as the paper states them: Sec. 4.1 (H =
    (2 pi/10) sigma_x, C = 0.05 sigma_x, observable sigma_z, psi0 = |0>, t in [0, 10],
    1,000 trajectories) and Sec. 4.2 (trilinear optical parametric amplifier, 8 x 8
    x 8 modes = N 512, three damping channels, coherent pump alpha = sqrt 3, three
    photon-number observables, t in [0, 4], 10,000 trajectories).  Double-float and
    complex128, each timed end to end through the public API (create with the host
    problem, run, expect) and as kernel time; the paper's CPU times are context
    only (another machine, tolerance 1e-7, a Fortran ZVODE solver)."""
    from paper_1810_03047_gb300 import shards
    from paper_1810_03047_gb300 import systems as S
    sid = int(stream.cuda_stream)
    out = {}
    launches = 0
    for name, prob, n, ctx_note in [
            ("unitary_sec4_1", S.paper_unitary(), 1000,
             "paper: QTM 2-3 s for 1,000 trajectories on 8 MPI processes (mostly start-up); QuTiP ~0.9 s on "
             "1 core; Intel i7 4.0 GHz, tolerance 1e-7"),
            ("trilinear_sec4_2", S.paper_trilinear(), 10000,
             "paper: timings shown only as a figure (QTM on 32 MPI workers, QuTiP on 4 cores, "
             "QuantumOptics.jl on 1 core)")]:
        first, count = shards.shard(world * n, world, rank)
        res = {}
        for pname, prec in (("df64", Q.QTM_PREC_DF64), ("c128", Q.QTM_PREC_C128)):
            ctx = Q.qtm_create(prob, stream=sid, precision=prec)
            Q.qtm_run_range(ctx, first, count, prob.seed)  # warm-up
            Q.qtm_expect(ctx)
            Q.qtm_destroy(ctx)
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx = Q.qtm_create(prob, stream=sid, precision=prec)
            Q.qtm_run_range(ctx, first, count, prob.seed)
            mean, _ = Q.qtm_expect(ctx)
            wall = time.perf_counter() - t0
            st = Q.qtm_stats(ctx)
            Q.qtm_destroy(ctx)
            t = torch.tensor([wall], dtype=torch.float64, device="cuda")
            if world > 1:
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
            res[pname] = {"e2e_s": float(t.item()), "kernel_ms": st["kernel_ms"],
                          "value": world * count / float(t.item()), "mean": mean}
            launches += 2 * RUN_LAUNCHES
        out[name] = {"ntraj": world * count, "unit": UNIT,
                     "df64": {k: v for k, v in res["df64"].items() if k != "mean"},
                     "c128": {k: v for k, v in res["c128"].items() if k != "mean"},
                     "observable_error_df64_vs_c128": float(np.abs(res["df64"]["mean"] - res["c128"]["mean"]).max()),
                     "steps_per_trajectory": (st["accepted"] + st["rejected"]) / count,
                     "jumps_per_trajectory": st["jumps"] / count, "context": ctx_note}
    out["launches"] = launches
    return out


def dense_tensor_core(Q, torch, stream, world, rank, dist, pk, ntraj=20000, sample=2000):
    """The dense random open system (GUE H, N = 256, four Ginibre channels with
    ||C_n||_2 = 0.3, 101 outputs on [0, 10], observable diag(0..N-1)/N, operators
    from default_rng(3), seed 1) through the tensor-core engine (BF16x6 stage
    products on tcgen05, FP32 state), 20,000 trajectories per GPU: one warm-up
    pass, two timed.  The plain FP64 GPU path (complex128) runs the first 2,000
    trajectory ids for its throughput and for the observable error on the same
    trajectories.  Roofline: the products are the engine's work -- per attempted
    step and trajectory seven FP32-accurate products of the scaled operator (8 N^2
    flops each, the Krylov form's wt_1 .. wt_7), issued as six bf16 tensor-core
    products each -- against the measured bf16 peak over six.  Its state passes
    (per attempt: seven product inputs, seven outputs, eight vectors read and one
    written by the control warps, 23 passes over 2N FP32 values) are reported
    beside it."""
    from paper_1810_03047_gb300 import shards
    from paper_1810_03047_gb300 import systems as S
    prob = S.dense_random(ntraj=ntraj)
    sid = int(stream.cuda_stream)
    first, count = shards.shard(world * ntraj, world, rank)
    tc = Q.qtm_create(prob, stream=sid, precision=Q.QTM_PREC_BF16X6)
    Q.qtm_run_range(tc, first, count, prob.seed)
    Q.qtm_expect(tc)
    times, kern, attempts = [], [], 0
    for _ in range(2):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Q.qtm_run_range(tc, first, count, prob.seed)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        st = Q.qtm_stats(tc)
        kern.append(st["kernel_ms"])
        attempts += st["accepted"] + st["rejected"]
    t = torch.tensor([max(times)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    tc_traj = Q.qtm_traj_expect(tc)[:sample]
    Q.qtm_destroy(tc)
    ref = Q.qtm_create(prob, stream=sid, precision=Q.QTM_PREC_C128)
    Q.qtm_run_range(ref, first, sample, prob.seed)
    ref_traj = Q.qtm_traj_expect(ref)
    ref_ms = Q.qtm_stats(ref)["kernel_ms"]
    Q.qtm_destroy(ref)
    err = float(np.abs(tc_traj.mean(axis=0) - ref_traj.mean(axis=0)).max())
    n = prob.dim
    bytes_per_attempt = 23 * 2 * n * 4
    flops_per_attempt = 7 * 8.0 * n * n
    kms = sum(kern) / len(kern)
    achieved = flops_per_attempt * (attempts / 2) / (kms / 1e3) / 1e12
    peak, note = _bf16x6_peak()
    hbm_peak, _ = pk["hbm"]
    return {"workload": "dense random open system: GUE H (N=256), 4 Ginibre C_n (||C_n||_2=0.3), 101 outputs on "
                        "[0,10], A = diag(0..N-1)/N, operators default_rng(3), seed 1",
            "precision": "tensor-core BF16x6 products, FP32 state, FP64 scalars", "unit": UNIT,
            "value": world * count / (ms / 1e3), "ms_per_step": ms, "ntraj_per_gpu": count,
            "fp64_path": {"value": sample / (ref_ms / 1e3), "kernel_ms": ref_ms, "sample": sample},
            "speedup_vs_fp64_path": (world * count / (ms / 1e3)) / (sample / (ref_ms / 1e3)),
            "observable_error": err,
            "observable_error_note": f"max |mean - complex128 mean| over the first {sample} trajectory ids",
            "steps_per_trajectory": attempts / 2 / count,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": TRAFFIC_PER_LAUNCH.get("qtm::dense_tc_kernel<256>") if count == 20000 else None,
                         "kernel": "qtm::dense_tc_kernel<256>", "flops_per_attempt": flops_per_attempt,
                         "state_bytes_per_attempt": bytes_per_attempt,
                         "state_gbs": bytes_per_attempt * (attempts / 2) / (kms / 1e3) / 1e9,
                         "state_frac_of_hbm": bytes_per_attempt * (attempts / 2) / (kms / 1e3) / 1e9 / hbm_peak,
                         "peak_note": note, "kernel_ms": kms},
            "launches": 4 * RUN_LAUNCHES}


def _timed_passes(Q, torch, stream, world, dist, prob, prec, method, first, count, passes=2):
    """One warm-up and `passes` timed runs of one context (CUDA events on the
    launching stream, max over ranks); returns throughput, time and counters."""
    ctx = Q.qtm_create(prob, stream=int(stream.cuda_stream), precision=prec)
    Q.qtm_set_method(ctx, method)
    Q.qtm_run_range(ctx, first, count, prob.seed)
    Q.qtm_expect(ctx)
    ms = []
    for _ in range(passes):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Q.qtm_run_range(ctx, first, count, prob.seed)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = torch.tensor([max(ms)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    st = Q.qtm_stats(ctx)
    mean = Q.qtm_expect(ctx)[0]
    Q.qtm_destroy(ctx)
    per_run = lockstep_launches(len(prob.t)) if (prec == Q.QTM_PREC_BF16X6 and method == Q.QTM_METHOD_EXPONENTIAL) \
        else RUN_LAUNCHES
    out = {"value": world * count / (float(t.item()) / 1e3), "ms_per_step": float(t.item()),
           "kernel_ms": st["kernel_ms"], "products_per_trajectory": st["rhs_evals"] / count,
           "jumps_per_trajectory": st["jumps"] / count, "mean": mean, "launches": (1 + passes) * per_run}
    if st.get("product_ms"):
        out["product_ms"] = st["product_ms"]
    return out


def exponential_method(Q, torch, stream, world, rank, dist, pk, jc_ref_mean, ntraj=20000):
    """The exponential method (exact propagation between jumps through a ladder of
    precomputed exp(M delta 2^l); Sec. 2.1's stiff-problem setting) against the
    Dormand-Prince path on the same trajectory ids: (1) the stiff Purcell system (a
    driven qubit on a cavity with kappa = 200, Purcell rate 0.5, N = 10, 201
    outputs on [0, 20]), where the explicit integrator's step is set by stability,
    and (2) the headline Jaynes-Cummings workload (N = 60, 401 outputs on
    [0, 40]), where it is not.  Observable errors are against the complex128
    Dormand-Prince path.  Roofline of the exponential kernel on the
    Jaynes-Cummings workload: per trajectory and output interval one dense
    product P x (N^2 complex multiply-adds = 8 N^2 flops), against the FP64 peak
    (complex128) or the double-float emulation peak.  On the dense workload also
    the lock-step form on the tensor cores (QTM_PREC_BF16X6): its product launch
    ((P_L - I) psi for all trajectories, 8 N^2 flops each) against the bf16 peak
    over six."""
    from paper_1810_03047_gb300 import shards
    from paper_1810_03047_gb300 import systems as S
    first, count = shards.shard(world * ntraj, world, rank)
    D, E = Q.QTM_METHOD_DOPRI5, Q.QTM_METHOD_EXPONENTIAL
    out, launches = {}, 0
    stiff = S.purcell_qubit(ntraj=ntraj)
    r = {}
    for key, prec, meth in (("expo_df64", Q.QTM_PREC_DF64, E), ("expo_c128", Q.QTM_PREC_C128, E),
                            ("expo_c64", Q.QTM_PREC_C64, E),
                            ("dopri5_df64", Q.QTM_PREC_DF64, D), ("dopri5_c128", Q.QTM_PREC_C128, D)):
        r[key] = _timed_passes(Q, torch, stream, world, dist, stiff, prec, meth, first, count)
        launches += r[key].pop("launches")
    ref = r["dopri5_c128"]["mean"]
    out["stiff_purcell"] = {
        "workload": "driven qubit + cavity (Purcell): N=10, g=5, kappa=200, gamma=0.05, drive 0.5, 201 outputs "
                    f"on [0, 20], {world * count} trajectories (seed 1)",
        "unit": UNIT,
        **{k: {kk: vv for kk, vv in v.items() if kk != "mean"} for k, v in r.items()},
        "speedup_expo_df64_vs_dopri5_df64": r["expo_df64"]["value"] / r["dopri5_df64"]["value"],
        "speedup_expo_c128_vs_dopri5_c128": r["expo_c128"]["value"] / r["dopri5_c128"]["value"],
        "observable_error_expo_c128_vs_dopri5_c128": float(np.abs(r["expo_c128"]["mean"] - ref).max()),
        "observable_error_expo_df64_vs_dopri5_c128": float(np.abs(r["expo_df64"]["mean"] - ref).max()),
        "observable_error_expo_c64_vs_dopri5_c128": float(np.abs(r["expo_c64"]["mean"] - ref).max()),
    }
    if world == 1 and rank == 0:
        # the exact-propagation oracle (scipy expm + brentq, one host core) on a bounded sample
        from oracle import exact
        t0 = time.perf_counter()
        sample = exact.mcwf(stiff, ntraj=200)
        dt = time.perf_counter() - t0
        out["stiff_purcell"]["oracle_cpu"] = {"value": 200 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                              "sample": "trajectory ids 0..199 of the same workload "
                                                        "(oracle/exact.py, single thread)"}
        del sample
    prob, _, _ = workload(ntraj)
    j = {}
    for key, prec in (("expo_df64", Q.QTM_PREC_DF64), ("expo_c128", Q.QTM_PREC_C128), ("expo_c64", Q.QTM_PREC_C64)):
        j[key] = _timed_passes(Q, torch, stream, world, dist, prob, prec, E, first, count)
        launches += j[key].pop("launches")
    n = prob.dim
    flops = 8.0 * n * n * (len(prob.t) - 1)  # the output-interval products, per trajectory
    jc = {"workload": f"damped driven Jaynes-Cummings (N=60), 401 outputs on [0, 40], {world * count} trajectories",
          "unit": UNIT}
    for key, peak_key in (("expo_df64", "df64"), ("expo_c128", "c128"), ("expo_c64", "c64")):
        v = j[key]
        achieved = flops * count / (v["kernel_ms"] / 1e3) / 1e12
        peak, note = pk[peak_key]
        jc[key] = {kk: vv for kk, vv in v.items() if kk != "mean"}
        jc[key]["observable_error_vs_dopri5_c128"] = float(np.abs(v["mean"] - jc_ref_mean).max())
        jc[key]["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                               "frac": achieved / peak, "traffic": None, "peak_note": note,
                               "flops_note": "8 N^2 per trajectory and output interval (P_L x); the "
                                             "observables, jumps and Taylor products are not counted"}
    out["jaynes_cummings"] = jc
    # dense operators: one dense product per output interval instead of six per
    # Dormand-Prince step; against the complex128 Dormand-Prince path on the first
    # 2,000 ids and the tensor-core engine's figure (reported in its own leg)
    dense = S.dense_random(ntraj=ntraj)
    dres = {}
    for key, prec in (("expo_df64", Q.QTM_PREC_DF64), ("expo_c128", Q.QTM_PREC_C128), ("expo_c64", Q.QTM_PREC_C64),
                      ("expo_tc", Q.QTM_PREC_BF16X6)):
        dres[key] = _timed_passes(Q, torch, stream, world, dist, dense, prec, E, first, count,
                                  passes=2 if key == "expo_tc" else 1)
        launches += dres[key].pop("launches")
    sample = min(count, 2000)
    ctx = Q.qtm_create(dense, stream=int(stream.cuda_stream), precision=Q.QTM_PREC_C128)
    Q.qtm_run_range(ctx, first, sample, dense.seed)
    ref_traj = Q.qtm_traj_expect(ctx)
    ref_ms = Q.qtm_stats(ctx)["kernel_ms"]
    Q.qtm_destroy(ctx)
    launches += RUN_LAUNCHES
    ex_traj = {}
    for key, prec in (("expo_df64", Q.QTM_PREC_DF64), ("expo_c64", Q.QTM_PREC_C64), ("expo_tc", Q.QTM_PREC_BF16X6)):
        ctx = Q.qtm_create(dense, stream=int(stream.cuda_stream), precision=prec)
        Q.qtm_set_method(ctx, E)
        Q.qtm_run_range(ctx, first, sample, dense.seed)
        ex_traj[key] = Q.qtm_traj_expect(ctx)
        Q.qtm_destroy(ctx)
        launches += lockstep_launches(len(dense.t)) if key == "expo_tc" else RUN_LAUNCHES
    nd = dense.dim
    dj = {"workload": "dense random open system (GUE H, N=256, 4 Ginibre C_n), 101 outputs on [0, 10], "
                      f"{world * count} trajectories", "unit": UNIT,
          "dopri5_c128_sample": {"value": sample / (ref_ms / 1e3), "kernel_ms": ref_ms, "sample": sample},
          "observable_error_expo_df64_vs_dopri5_c128": float(np.abs(ex_traj["expo_df64"].mean(axis=0)
                                                                    - ref_traj.mean(axis=0)).max()),
          "observable_error_expo_c64_vs_dopri5_c128": float(np.abs(ex_traj["expo_c64"].mean(axis=0)
                                                                   - ref_traj.mean(axis=0)).max()),
          "observable_error_expo_tc_vs_dopri5_c128": float(np.abs(ex_traj["expo_tc"].mean(axis=0)
                                                                  - ref_traj.mean(axis=0)).max()),
          "observable_error_note": f"max |mean - complex128 Dormand-Prince mean| over the first {sample} ids"}
    for key, peak_key in (("expo_df64", "df64"), ("expo_c128", "c128"), ("expo_c64", "c64")):
        v = dres[key]
        achieved = 8.0 * nd * nd * (len(dense.t) - 1) * count / (v["kernel_ms"] / 1e3) / 1e12
        peak, note = pk[peak_key]
        dj[key] = {kk: vv for kk, vv in v.items() if kk != "mean"}
        dj[key]["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                               "frac": achieved / peak, "traffic": None, "peak_note": note}
    # the lock-step path on the tensor cores: its product launch against the
    # BF16x6 emulation peak (one (P_L - I) psi of 8 N^2 flops per trajectory)
    v = dres["expo_tc"]
    dj["expo_tc"] = {kk: vv for kk, vv in v.items() if kk != "mean"}
    dj["expo_tc"]["precision"] = ("tensor-core BF16x6 products (P_L - I) psi for all trajectories per output "
                                  "interval, complex64 crossing search, jumps and outputs")
    dj["expo_tc"]["speedup_vs_expo_c64"] = v["value"] / dres["expo_c64"]["value"]
    if v.get("product_ms"):
        peak, note = _bf16x6_peak()
        achieved = 8.0 * nd * nd * count / (v["product_ms"] / 1e3) / 1e12
        dj["expo_tc"]["roofline"] = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                     "frac": achieved / peak, "traffic": None,
                                     "kernel": "qtm::dense_tc_kernel<256> (rhs mode, (P_L - I) psi)",
                                     "flops_per_launch": 8.0 * nd * nd * count, "kernel_ms": v["product_ms"],
                                     "peak_note": note}
    out["dense_random"] = dj
    out["launches"] = launches
    return out


def learned_proposal(Q, torch, stream, world, rank, dist, ntraj=200000):
    """The learned jump-time proposal on the Jaynes-Cummings workload: about 10^6
    (features -> time left to the jump) pairs from 12,000 trajectories of the
    plain method (seed 11), the 6-64-64-1 network trained on the GPU, then 200,000
    trajectories (seed 1) timed with the plain double-float kernel and with the
    proposal kernel (network inference fused in the step loop; the root find
    still decides every jump).  Steps per trajectory, trajectories/s and the
    ensemble difference between the two are reported."""
    from paper_1810_03047_gb300 import shards
    prob, _, _ = workload(ntraj)
    sid = int(stream.cuda_stream)
    first, count = shards.shard(world * ntraj, world, rank)
    ctx = Q.qtm_create(prob, stream=sid, precision=Q.QTM_PREC_DF64)
    t0 = time.perf_counter()
    npairs = Q.qtm_proposal_collect(ctx, 12000, 11, stride=8, max_per_traj=96)
    t1 = time.perf_counter()
    steps = 2000
    loss, base = Q.qtm_proposal_train(ctx, steps=steps, batch=8192, lr=2e-3, seed=11)
    t2 = time.perf_counter()
    Q.qtm_run_range(ctx, first, min(count, 20000), prob.seed)  # warm-up of both kernels
    Q.qtm_proposal_enable(ctx, True, 0.05)
    Q.qtm_run_range(ctx, first, min(count, 20000), prob.seed)
    res = {}
    for on in (False, True):
        Q.qtm_proposal_enable(ctx, on, 0.05)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Q.qtm_run_range(ctx, first, count, prob.seed)
        e1.record(stream)
        e1.synchronize()
        t = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        st = Q.qtm_stats(ctx)
        res[on] = {"ms": float(t.item()), "mean": Q.qtm_expect(ctx)[0],
                   "steps": (st["accepted"] + st["rejected"]) / count, "jumps": st["jumps"] / count}
    Q.qtm_destroy(ctx)
    off, on = res[False], res[True]
    expo = _learned_proposal_expo(Q, torch, stream, world, dist, prob, first, count, ntraj)
    return {"workload": f"damped driven Jaynes-Cummings (N=60), {world * ntraj} trajectories (seed 1); "
                        f"network trained on {npairs} pairs from 12,000 trajectories (seed 11)",
            "exponential_method": expo,
            "precision": "df64", "unit": UNIT,
            "value": world * ntraj / (on["ms"] / 1e3), "plain_value": world * ntraj / (off["ms"] / 1e3),
            "steps_per_trajectory": on["steps"], "plain_steps_per_trajectory": off["steps"],
            "step_saving": (off["steps"] - on["steps"]) / off["steps"],
            "jumps_per_trajectory": on["jumps"], "plain_jumps_per_trajectory": off["jumps"],
            "observable_error_vs_plain": float(np.abs(on["mean"] - off["mean"]).max()),
            "train": {"pairs": npairs, "steps": steps, "batch": 8192, "loss": loss, "loss_rate_estimate": base,
                      "collect_s": t1 - t0, "train_s": t2 - t1},
            "launches": RUN_LAUNCHES + 3 * steps + 1 + 4 * RUN_LAUNCHES + expo.pop("launches")}


def _learned_proposal_expo(Q, torch, stream, world, dist, prob, first, count, ntraj):
    """The learned proposal inside the exponential method's crossing search, same
    workload: pairs from the method's own crossings in 12,000 trajectories (seed
    11), trained on the GPU, then the 200,000 trajectories timed without and with
    the proposal (double-float).  Products per trajectory (ladder levels, Taylor
    and channel products), bracket hits, trajectories/s and the ensemble
    difference are reported."""
    sid = int(stream.cuda_stream)
    ctx = Q.qtm_create(prob, stream=sid, precision=Q.QTM_PREC_DF64)
    Q.qtm_set_method(ctx, Q.QTM_METHOD_EXPONENTIAL)
    npairs = Q.qtm_proposal_collect(ctx, 12000, 11, stride=1, max_per_traj=96)
    steps = 2000
    loss, base = Q.qtm_proposal_train(ctx, steps=steps, batch=8192, lr=2e-3, seed=11)
    Q.qtm_run_range(ctx, first, min(count, 20000), prob.seed)  # warm-up of both kernels
    Q.qtm_proposal_enable(ctx, True, 0.05)
    Q.qtm_run_range(ctx, first, min(count, 20000), prob.seed)
    res = {}
    for on in (False, True):
        Q.qtm_proposal_enable(ctx, on, 0.05)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Q.qtm_run_range(ctx, first, count, prob.seed)
        e1.record(stream)
        e1.synchronize()
        t = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        st = Q.qtm_stats(ctx)
        res[on] = {"ms": float(t.item()), "mean": Q.qtm_expect(ctx)[0], "products": st["rhs_evals"] / count,
                   "jumps": st["jumps"], "misses": st["proposal_misses"]}
    Q.qtm_destroy(ctx)
    off, on = res[False], res[True]
    return {"precision": "df64", "unit": UNIT,
            "value": world * ntraj / (on["ms"] / 1e3), "plain_value": world * ntraj / (off["ms"] / 1e3),
            "products_per_trajectory": on["products"], "plain_products_per_trajectory": off["products"],
            "product_saving": (off["products"] - on["products"]) / off["products"],
            "bracket_hit_rate": 1.0 - on["misses"] / max(on["jumps"], 1),
            "jumps_per_trajectory": on["jumps"] / count,
            "observable_error_vs_plain": float(np.abs(on["mean"] - off["mean"]).max()),
            "train": {"pairs": npairs, "steps": steps, "batch": 8192, "loss": loss, "loss_rate_estimate": base},
            "launches": RUN_LAUNCHES + 3 * steps + 1 + 4 * RUN_LAUNCHES}


if __name__ == "__main__":
    sys.exit(main())

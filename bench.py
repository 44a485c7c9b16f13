#!/usr/bin/env python
"""Benchmark of the unitary-matrix simulation hot path on GB300.

Workload (one "step"): a batch of 11-qubit circuits shaped like the paper's
evaluated programs - fully entangled (GHZ chain), Deutsch-Jozsa with a
constant and with a balanced oracle, and QFT on a seeded basis state, 25 %
each - simulated by the fused step kernels in one CUDA-graph launch: the
state of every circuit, |psi_i|^2 in FP64 and the FP64 norm of every circuit.
Synthetic, seeded inputs (base seed 14398).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tqs|reference]

Prints one JSON line (rank 0).  metric: circuits/s (whole job); beside it the
plain materialised-matrix form on the same GPU, the dense-equivalent complex
GFLOP/s, the roofline of the fused kernel, the end-to-end rate through the
host-buffer C entry point, and the CPU FP64 oracle timed on the host.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_QUBITS = 11
BATCH = 16384
METRIC = "circuits/s"
WORKLOAD = "paper-shaped 11-qubit circuits (GHZ / DJ-constant / DJ-balanced / QFT, 25% each)"

# DRAM bytes (read + write) per launch of the fused kernel on this workload,
# from the ncu capture summarised in profiles/: 19.64 MB read + 476.63 MB
# written for one launch over the 16384 circuits of a step, at the launch
# shape given here (one warp per circuit, one warp per CTA).  Reported only
# when the autotuner picked that shape; set back to None whenever the kernel
# changes, until it is captured again.
NCU_TRAFFIC = {"team_warps": 1, "warps_per_cta": 1, "bytes": 19_641_600 + 476_631_296}


def roofline_traffic(team_warps, warps_per_cta, capture=NCU_TRAFFIC):
    """The captured DRAM bytes per launch when the timed launch shape is the
    captured one, else None (another shape's traffic was not measured)."""
    if capture is None:
        return None
    if (team_warps, warps_per_cta) != (capture["team_warps"], capture["warps_per_cta"]):
        return None
    return capture["bytes"]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["tqs", "reference"], default="tqs")
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-chain", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-sample", action="store_true")
    ap.add_argument("--no-fsv", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------ CPU oracle arm

ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
from oracle import kron_route
from paper_2305_14398_gb300 import workloads as W
mix = W.paper_mix(%(n)d, 4, seed_tag=%(tag)d)
kinds = %(kinds)r
t0 = time.perf_counter()
done = 0
for i in kinds:
    name, ops = mix[i]
    kron_route.simulate(%(n)d, ops)
    done += 1
dt = time.perf_counter() - t0
print(json.dumps({"circuits": done, "seconds": dt}))
"""


ORACLE_EXTRA_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
from oracle import fsv_route
from paper_2305_14398_gb300 import workloads as W
out = {}
mix = W.paper_mix(%(n)d, 64, seed_tag=1)
t0 = time.perf_counter()
for _, ops in mix:
    fsv_route.simulate(%(n)d, ops)
out["fsv_circuits_per_s"] = len(mix) / (time.perf_counter() - t0)
n = 12
ops = W.random_layered(n, 20, (2, n))
cols = [0, 1, 2, 3]
t0 = time.perf_counter()
fsv_route.unitary_columns(n, ops, cols)
dt = time.perf_counter() - t0
out["chain_n12_columns"] = len(cols)
out["chain_n12_seconds_full_estimate"] = dt / len(cols) * (1 << n)
print(json.dumps(out))
"""


def oracle_extra():
    """Further CPU baselines of the oracle, one thread: the per-gate route
    (eq. 12) on 64 circuits of the bench mix, and the circuit-unitary chain
    at n = 12 by the column route (4 columns timed, the full 4096-column
    unitary extrapolated)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ORACLE_EXTRA_SNIPPET % {"root": ROOT, "n": N_QUBITS}
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample(kinds, tag=1):
    """Time the oracle's literal route (Algorithm 1/2: Kronecker step matrix +
    dense matvec per step, FP64) on the given circuits of the mix, one thread,
    in a fresh process."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ORACLE_SNIPPET % {"root": ROOT, "n": N_QUBITS, "tag": tag, "kinds": list(kinds)}
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample_all_cores(kinds, tag=1):
    """The same sample in one fresh process per host core, run at once
    (each process one thread); returns the circuits done and the wall time."""
    procs = os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ORACLE_SNIPPET % {"root": ROOT, "n": N_QUBITS, "tag": tag, "kinds": list(kinds)}
    t0 = time.perf_counter()
    ps = [subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                           stderr=subprocess.PIPE, text=True) for _ in range(procs)]
    done, inner = 0, 0.0
    for p in ps:
        out, err = p.communicate(timeout=900)
        if p.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        r = json.loads(out.strip().splitlines()[-1])
        done += r["circuits"]
        inner = max(inner, r["seconds"])
    # seconds: wall time with process start-up; inner_seconds: the slowest
    # process's own timed work (they run at once)
    return {"circuits": done, "seconds": time.perf_counter() - t0, "inner_seconds": inner,
            "procs": procs}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    # each step: one circuit of the mix in each of one single-thread process
    # per host core at once, kinds in rotation (GHZ, DJc, DJb, QFT); a step's
    # time is the slowest process's own timed work
    for w in range(args.warmup):
        oracle_sample_all_cores([w % 4])
    total_c, total_s, cores = 0, 0.0, 1
    for k in range(args.steps):
        r = oracle_sample_all_cores([k % 4])
        total_c += r["circuits"]
        total_s += r["inner_seconds"]
        cores = r["procs"]
    value = total_c / total_s
    # the workload's description is the GPU arm's (one batch of the mix per GPU)
    from paper_2305_14398_gb300 import workloads as W
    circs = replica_circuits(W, 0, args.batch)
    steps_total = sum(W.asap_steps(ops) for _, ops in circs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "circuits/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(len(circs), steps_total, max(1, args.gpus)),
        "cpu_baseline": {"value": value, "unit": "circuits/s", "cores": cores, "kind": "oracle",
                         "sample": "per step one circuit in each of one single-thread process "
                                   "per host core at once, kinds in rotation GHZ/DJ-constant/"
                                   "DJ-balanced/QFT, literal Kronecker route, FP64"},
        "e2e": {"value": value, "unit": "circuits/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (timestamped on the host) during a window."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append((time.perf_counter(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self, t0, t1):
        inside = [p for t, p in self.samples if t0 <= t <= t1]
        window = "timed region"
        if len(inside) < 3:
            inside = [p for _, p in self.samples]
            window = "warm-up + timed region (timed region shorter than the sampling period)"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "window": window}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(p[0]) for p in inside if num(p[0]) is not None]
        smax = [num(p[1]) for p in inside if num(p[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in inside for i in range(4) if p[4 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(inside), "window": window}


def workload_config(count, steps_total, world):
    """The bench line's `config`: the workload, the same for this implementation
    and the reference arm (no implementation or launch keys)."""
    return {"workload": WORKLOAD, "n_qubits": N_QUBITS, "circuits_per_gpu": count,
            "steps_per_batch": steps_total, "parallelism": f"replicas x{world}",
            "l2": "GPU arm: flushed between timed steps (256 MiB write, not timed); "
                  "CPU reference arm: not applicable",
            "outputs": "state (complex64) + |psi|^2 (f64) + norm (f64) per circuit"}


def replica_circuits(W, rank, batch):
    """This rank's share: its own seeded batch of the workload (weak scaling;
    circuits are independent, so ranks exchange no data)."""
    return [(N_QUBITS, ops) for _, ops in W.paper_mix(N_QUBITS, batch, seed_tag=1 + 1000 * rank)]


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds_max):
    """Units all ranks processed per second of the slowest rank."""
    return units_per_rank * world / seconds_max


def smi_index(local):
    """nvidia-smi -i argument of this rank's GPU (index or UUID)."""
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        parts = [p.strip() for p in cvd.split(",") if p.strip()]
        if local < len(parts):
            return parts[local]
    return str(local)


# ----------------------------------------------------------------- GPU arm

def run_tqs(args):
    import numpy as np
    import torch

    from paper_2305_14398_gb300 import binding as B
    from paper_2305_14398_gb300 import build as _build
    from paper_2305_14398_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if not os.path.exists(B.LIB_PATH):
        _build.build()
    B.lib()

    # ---------------------------------------------------------- inputs
    circs = replica_circuits(W, rank, args.batch)
    from paper_2305_14398_gb300 import autotune
    tuned = autotune.tune_warps_per_cta(circs)
    arrays = B.pack_ops(circs)
    b = B.tqs_batch_create_packed(*arrays)
    count, total, offs, steps_total, prog_bytes = B.tqs_batch_info(b, extra=True)
    states = torch.empty(total, dtype=torch.complex64, device="cuda")
    probs = torch.empty(total, dtype=torch.float64, device="cuda")
    norms = torch.empty(count, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    stream = torch.cuda.current_stream()

    sampler = ClockSampler(smi_index(local))
    sampler.start()
    # first run uploads and captures the graph (untimed)
    B.tqs_batch_run(b, states, probs, norms, use_graph=True)
    for _ in range(max(3, args.warmup)):
        flush.zero_()
        B.tqs_batch_run(b, states, probs, norms, use_graph=True)
    torch.cuda.synchronize()
    # soak so that clock samples exist around a short timed region
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < 1.0:
        B.tqs_batch_run(b, states, probs, norms, use_graph=True)
        torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = B.tqs_launch_count()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (not timed)
        ev[k][0].record(stream)
        B.tqs_batch_run(b, states, probs, norms, use_graph=True)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    launches = B.tqs_launch_count() - launches0
    if dist:
        dist.barrier()
    sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist, "cuda")
    value = whole_job_rate(count * args.steps, world, total_s)
    ms_step = 1e3 * total_s / args.steps

    # sanity: every norm within 1e-6 of 1
    nrm = norms.cpu()
    norm_err = float((nrm - 1.0).abs().max())

    # ------------------------------------------------- roofline (fused kernel)
    N = 1 << N_QUBITS
    alg_bytes = count * (N * 8 + N * 8 + 8) + prog_bytes  # state + probs + norm written, program read
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    achieved_gbs = alg_bytes / (ms_step / 1e3) / 1e9
    dense_flops = 8.0 * (4 ** N_QUBITS) * steps_total  # ZGEMM convention, dense-equivalent
    line = {
        "metric": METRIC, "value": value, "unit": "circuits/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(count, steps_total, world),
        "launch": {"warps_per_circuit": tuned["team_warps"],
                   "warps_per_cta": tuned["warps"], "autotune_ms": tuned["timings_ms"],
                   "autotune_source": tuned["source"]},
        "dense_equiv_complex_gflops": dense_flops * world * args.steps / total_s / 1e9,
        "step_ms_stats": step_stats(step_ms),
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak,
                     "unit": "GB/s", "frac": achieved_gbs / hbm_peak,
                     "traffic": roofline_traffic(tuned["team_warps"], tuned["warps"]),
                     "peak_source": peak_src,
                     "kernel": ("fused_kernel<TEAM_PAIR>" if tuned["team_warps"] == 2
                                else "fused_kernel<TEAM_WARP>"),
                     "algorithmic_bytes_per_launch": alg_bytes},
        "norm_max_err": norm_err,
        "gpu_launches": launches,
    }
    line["clocks"] = sampler.summary(t0, t1)

    # ------------------------------------------------------- end to end
    if not args.no_e2e:
        bufs = [(torch.empty(total, dtype=torch.complex64).pin_memory(),
                 torch.empty(total, dtype=torch.float64).pin_memory(),
                 torch.empty(count, dtype=torch.float64).pin_memory()) for _ in range(2)]
        e2e_steps = max(3, min(args.steps, 20))
        for k in range(2):  # warm: creation scratch, device pool, both buffer sets
            bb = B.tqs_batch_create_packed(*arrays)
            B.tqs_batch_run_host(bb, *bufs[k])
            B.tqs_batch_destroy(bb)
        if dist:
            dist.barrier()
        # sequential: create, run, destroy, one batch after the other
        te0 = time.perf_counter()
        for k in range(e2e_steps):
            bb = B.tqs_batch_create_packed(*arrays)
            B.tqs_batch_run_host(bb, *bufs[k % 2])
            B.tqs_batch_destroy(bb)
        te_seq = max_over_ranks(time.perf_counter() - te0, dist, "cuda")
        if dist:
            dist.barrier()
        # pipelined: a second host thread creates batch k + 1 while batch k runs
        te_pipe = max_over_ranks(e2e_pipelined(B, arrays, bufs, e2e_steps), dist, "cuda")
        line["e2e"] = {"value": whole_job_rate(count * e2e_steps, world, te_pipe), "unit": "circuits/s",
                       "h2d_bytes_per_step": int(prog_bytes),
                       "d2h_bytes_per_step": int(total * 8 + total * 8 + count * 8),
                       "steps": e2e_steps,
                       "sequential_value": whole_job_rate(count * e2e_steps, world, te_seq),
                       "path": "tqs_batch_create_packed (host gate arrays) + tqs_batch_run_host "
                               "(page-locked host buffers, written by the kernel over C2C) + "
                               "tqs_batch_destroy; value: a second host thread creates the next "
                               "batch (and destroys finished ones) while the current one runs; "
                               "sequential_value: one batch after the other"}

    # ----------------------------------------------- measured peaks (rank 0)
    # (after the end-to-end leg: the sustained GEMM loop heats the GPU)
    mpeaks = {}
    if rank == 0:
        from paper_2305_14398_gb300 import peaks as _peaks
        mpeaks = _peaks.measure(B, torch)
        line["measured_peaks"] = mpeaks

    # ------------------------------------------------------- plain form
    if not args.no_plain and rank == 0:
        mix = W.paper_mix(N_QUBITS, 4, seed_tag=1)
        handles = [B.circuit_from_ops(N_QUBITS, ops) for _, ops in mix]
        out = torch.empty(N, dtype=torch.complex64, device="cuda")
        for h in handles:
            B.tqs_simulate_plain(h, out)
        torch.cuda.synchronize()
        reps = 3
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for _ in range(reps):
            for h in handles:
                B.tqs_simulate_plain(h, out)
        e.record(stream)
        torch.cuda.synchronize()
        plain_s = s.elapsed_time(e) / 1e3
        plain_steps = sum(B.tqs_circuit_info(h)[2] for h in handles) * reps
        # the fused kernel on the same circuits, one launch per circuit
        # (single-circuit latency: one warp team on one SM)
        probs1 = torch.empty(N, dtype=torch.float64, device="cuda")
        norm1 = torch.empty(1, dtype=torch.float64, device="cuda")
        for h in handles:
            B.tqs_simulate(h, out, probs=probs1, norm=norm1)
        torch.cuda.synchronize()
        reps1 = 50
        s.record(stream)
        for _ in range(reps1):
            for h in handles:
                B.tqs_simulate(h, out, probs=probs1, norm=norm1)
        e.record(stream)
        torch.cuda.synchronize()
        single_s = s.elapsed_time(e) / 1e3
        for h in handles:
            B.tqs_circuit_destroy(h)
        plain_rate = 4 * reps / plain_s
        line["plain"] = {
            "value": plain_rate, "unit": "circuits/s",
            "sample": "one circuit of each kind, 3 repetitions",
            "dense_equiv_complex_gflops": 8.0 * (4 ** N_QUBITS) * plain_steps / plain_s / 1e9,
            "hbm_gbs_algorithmic": 16.0 * (4 ** N_QUBITS) * plain_steps / plain_s / 1e9,
            "fused_speedup": value / world / plain_rate,
            "fused_single": {"value": 4 * reps1 / single_s, "unit": "circuits/s",
                             "latency_us": 1e6 * single_s / (4 * reps1),
                             "sample": "the same 4 circuits, one tqs_simulate each (state, "
                                       "probabilities, norm), 50 repetitions, back to back on "
                                       "one stream",
                             "speedup_vs_plain": (4 * reps1 / single_s) / plain_rate},
        }

    if not args.no_plain and rank == 0:
        line["plain"]["cublas_cgemv"] = bench_cublas_plain(B, W, torch)

    # ------------------------------------------------ collapse (sampling)
    if not args.no_sample and rank == 0:
        line["sample"] = bench_sample(B, torch, b, probs, count, total, flush, hbm_peak)

    # ------------------------------------- random batches (L2- and HBM-sized)
    if not args.no_batch and rank == 0:
        line["batch"] = bench_batch(B, W, torch, peaks, flush, max(3, min(args.steps, 10)),
                                    mpeaks["fp32_fma_tflops"])

    # ------------------------------------------ full state vector (large n)
    if not args.no_fsv and rank == 0:
        line["fsv"] = bench_fsv(B, W, torch, hbm_peak, mpeaks["fp32_fma_tflops"])

    # ------------------------------------------- circuit-unitary chain (a5)
    if not args.no_chain and rank == 0:
        line["chain"] = bench_chain(B, W, torch, peaks, mpeaks)
        line["chain"]["cublas"] = bench_cublas_chain(B, W, torch)
        # the library reference points also as top-level keys of the chain leg
        for k, v in line["chain"]["cublas"].items():
            if k.startswith("n1"):
                line["chain"][k] = v
    # the column-sharded chain: every rank its own block of columns, no exchange
    if not args.no_chain:
        sh = bench_chain_sharded(B, W, torch, dist, rank, world, peaks)
        if rank == 0:
            line["chain_sharded"] = sh

    # ----------------------------------------------------- serving loop (a8)
    if not args.no_serving and rank == 0:
        from paper_2305_14398_gb300 import serve
        reqs = W.serving_requests(20000, 2000.0)
        # warm-up (not reported): the server's pool, kernel attributes, cooperative launches
        serve.replay(reqs[:2000], budget_bytes=120 * 10 ** 9, max_inflight=4, max_batch=256)
        r = serve.replay(reqs, budget_bytes=120 * 10 ** 9, max_inflight=4, max_batch=256)
        line["serving"] = {
            "workload": "20000 simulate requests, Poisson 2000 req/s (seeded), n ~ U{6..16}, "
                        "25% each GHZ / Deutsch-Jozsa / QFT / random mixed; HBM budget 120 GB; "
                        "continuous batching, 4 batches in flight",
            "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "mean_ms": r["mean_ms"],
            "max_ms": r["max_ms"], "completed_rps": r["throughput_rps"], "wall_s": r["wall_s"],
            "norm_max_err": float(np.max(np.abs(r["norms"] - 1.0))),
            "peak_device_bytes": r["stats"]["peak_bytes"], "busy_frac": r["busy_frac"]}
        # offered load up to saturation (same mix, 20000 requests per rate)
        sw = serve.sweep([5000, 20000, 50000, 100000, 200000, 400000])
        kept = [x["offered_rps"] for x in sw if x["completed_rps"] >= 0.95 * x["offered_rps"]]
        line["serving"]["sweep"] = sw
        line["serving"]["max_sustained_rps"] = max(kept) if kept else None
        line["serving"]["sweep_note"] = ("busy_frac: wall-time share with a batch in flight as the "
                                         "polls see it; max_sustained_rps: the highest offered rate "
                                         "completed at >= 95 %")

    # ---------------------------------------------------------- CPU oracle
    if not args.no_cpu_baseline and rank == 0:
        r1 = oracle_sample([0, 1, 2, 3])
        ra = oracle_sample_all_cores([0, 1, 2, 3])
        line["cpu_baseline"] = {
            "value": ra["circuits"] / ra["inner_seconds"], "unit": "circuits/s",
            "cores": ra["procs"], "kind": "oracle",
            "sample": f"4 circuits (one GHZ, DJ-constant, DJ-balanced, QFT) of the same workload "
                      f"in each of {ra['procs']} concurrent single-thread processes (one per host "
                      f"core), literal Kronecker route (Algorithm 1/2), FP64; time = the slowest "
                      f"process's own timed work",
            "value_1_core": r1["circuits"] / r1["seconds"],
        }
        ex = oracle_extra()
        line["cpu_baseline_other"] = {
            "per_gate_route_circuits_per_s_1_core": ex["fsv_circuits_per_s"],
            "per_gate_route_sample": "64 circuits of the bench mix, eq. 12 per gate, FP64, 1 thread",
            "chain_n12_seconds_1_core_estimate": ex["chain_n12_seconds_full_estimate"],
            "chain_n12_sample": f"{ex['chain_n12_columns']} columns of the 40-step random layered "
                                "unitary by the column route, extrapolated to 4096 columns",
        }

    B.tqs_batch_destroy(b)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def step_stats(ms):
    """Mean, p50, p99, min and max of per-step device times (this rank)."""
    v = sorted(ms)

    def pct(q):
        return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]
    return {"mean": sum(v) / len(v), "p50": pct(0.5), "p99": pct(0.99), "min": v[0], "max": v[-1],
            "count": len(v)}


def e2e_pipelined(B, arrays, bufs, steps):
    """End to end through the public API with two host threads: a producer
    creates the batches (host compile from the gate arrays) and destroys the
    ones already run, while the caller runs each with tqs_batch_run_host into
    alternating host buffers.  Returns the wall time of `steps` batches."""
    import queue
    q = queue.Queue(maxsize=2)
    done = queue.Queue()
    errors = []

    def producer():
        try:
            for _ in range(steps):
                while True:  # free what the caller has finished with
                    try:
                        B.tqs_batch_destroy(done.get_nowait())
                    except queue.Empty:
                        break
                q.put(B.tqs_batch_create_packed(*arrays))
        except Exception as e:  # surfaced by the consumer
            errors.append(e)
            q.put(None)

    t0 = time.perf_counter()
    th = threading.Thread(target=producer, daemon=True)
    th.start()
    for k in range(steps):
        bb = q.get()
        if bb is None:
            raise errors[0]
        B.tqs_batch_run_host(bb, *bufs[k % 2])
        done.put(bb)
    th.join()
    while not done.empty():
        B.tqs_batch_destroy(done.get_nowait())
    return time.perf_counter() - t0


def bench_sample(B, torch, b, probs, count, total, flush, hbm_peak, shots=64, reps=5):
    """simulateAndCollapse's sampling stage over the bench batch: `shots`
    inverse-CDF draws per circuit from the probabilities the step wrote."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(14398)
    u = torch.rand(count * shots, dtype=torch.float64, device="cuda", generator=gen)
    out = torch.empty(count * shots, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    B.tqs_batch_sample(b, probs, shots, u, out)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for k in range(reps):
        flush.zero_()
        ev[k][0].record(stream)
        B.tqs_batch_sample(b, probs, shots, u, out)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    sec = sum(s.elapsed_time(e) for s, e in ev) / 1e3 / reps
    alg = 8.0 * total + 16.0 * count * shots  # probabilities read once; u read, index written
    return {"workload": f"{shots} shots per circuit from the step's probabilities "
                        f"({count} circuits)",
            "ms": 1e3 * sec, "shots_per_s": count * shots / sec,
            "hbm": {"achieved_gbs": alg / sec / 1e9, "peak": hbm_peak,
                    "frac": alg / sec / 1e9 / hbm_peak, "algorithmic_bytes": alg},
            "launches_per_call": 3}


# Algorithmic FP32 flops of one gate on an n-qubit state (per-gate update of
# Appendix A, eq. 12): a dense single-qubit gate is 2 complex MACs (16 flops) per
# amplitude; a controlled dense gate does that on the control = 1 half; a
# diagonal (or phased permutation, Y) gate is one complex multiply (8) on half of
# the amplitudes, a controlled diagonal on a quarter; pure permutations are free.
_GATE_FLOPS = {"h": 16.0, "rx": 16.0, "ry": 16.0, "u3": 16.0, "cu": 8.0,
               "y": 4.0, "z": 4.0, "s": 4.0, "t": 4.0, "r": 4.0, "rz": 4.0,
               "cz": 2.0, "cp": 2.0, "x": 0.0, "cx": 0.0, "cnot": 0.0, "swap": 0.0}


def algorithmic_flops(n, ops):
    return float(1 << n) * sum(_GATE_FLOPS[name] for name, _, _ in ops)


def bench_batch(B, W, torch, peaks, flush, reps, fp32_peak):
    """The batched persistent launch on random mixed circuits: 4096 circuits of
    n = 4..14 (log-uniform, depth U{5..40}; states L2-resident) and 4096
    circuits all at n = 14 (1.5 GiB of outputs, streamed through HBM).  Each
    rep is one graph launch with L2 flushed before it (not timed)."""
    hbm = peaks.get("hbm_gbs", 6800.0)
    stream = torch.cuda.current_stream()
    out = {}
    for key, circs, what in [
            ("random_4096_n4_14", W.batch_circuits(4096, seed_tag=3),
             "4096 random mixed circuits, n = floor(exp(U[ln 4, ln 15))), depth U{5..40}"),
            ("random_4096_n14", W.batch_circuits_fixed_n(4096, 14, seed_tag=5),
             "4096 random mixed circuits, all n = 14, depth U{5..40}")]:
        from paper_2305_14398_gb300 import autotune
        tuned = autotune.tune_cta_threads(circs)
        b = B.tqs_batch_create_packed(*B.pack_ops(circs))
        count, total, _, steps_total, prog_bytes = B.tqs_batch_info(b, extra=True)
        states = torch.empty(total, dtype=torch.complex64, device="cuda")
        probs = torch.empty(total, dtype=torch.float64, device="cuda")
        norms = torch.empty(count, dtype=torch.float64, device="cuda")
        for _ in range(3):
            B.tqs_batch_run(b, states, probs, norms, use_graph=True)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for k in range(reps):
            flush.zero_()
            ev[k][0].record(stream)
            B.tqs_batch_run(b, states, probs, norms, use_graph=True)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        sec = sum(s.elapsed_time(e) for s, e in ev) / 1e3 / reps
        alg_bytes = 16.0 * total + 8.0 * count + prog_bytes
        flops = sum(algorithmic_flops(n, ops) for n, ops in circs)
        out[key] = {
            "workload": what, "circuits": count, "steps": steps_total,
            "ms": 1e3 * sec, "circuits_per_s": count / sec,
            "hbm": {"achieved_gbs": alg_bytes / sec / 1e9, "peak": hbm,
                    "frac": alg_bytes / sec / 1e9 / hbm, "algorithmic_bytes": alg_bytes},
            "alu": {"achieved_tflops": flops / sec / 1e12,
                    "peak": fp32_peak,
                    "frac": flops / sec / 1e12 / fp32_peak,
                    "algorithmic_flops": flops,
                    "peak_source": "measured FP32 FMA microkernel (measured_peaks)"},
            "norm_max_err": float((norms.cpu() - 1.0).abs().max()),
            "cta_threads": {"chosen": tuned["value"], "autotune_ms": tuned["timings_ms"],
                            "source": tuned["source"]},
        }
        B.tqs_batch_destroy(b)
        del states, probs, norms
        torch.cuda.empty_cache()
    return out


def bench_fsv(B, W, torch, hbm_peak, fp32_peak):
    """Full-state-vector backend on states in HBM: random layered circuits
    (10 x (U3 on every qubit + CNOTs on n/2 seeded pairs)) at n = 24, 28, 30.
    Each pass streams the state once (read + write): 16 * 2^n algorithmic
    bytes per pass; the ALU fraction counts the algorithmic FP32 flops of the
    per-gate update (eq. 12).  Also: the per-gate form (one pass per gate) at
    n = 24, and the fused kernel beside the tiled passes at n = 16."""
    from paper_2305_14398_gb300 import autotune
    out = {"workload": "random layered: 10 x (U3 on every qubit + CNOTs on n/2 seeded pairs)"}
    tiles = {}
    for n, reps in ((24, 5), (28, 3), (30, 2)):
        ops = W.random_layered(n, 10, (9, n))
        tiles[n] = autotune.tune_fsv_tile(n, ops, reps=2 if n < 28 else 1)
        c = B.circuit_from_ops(n, ops)
        st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
        st[0] = 1.0
        passes, tile = B.tqs_fsv_passes(c)
        B.tqs_simulate_fsv(c, st)  # compile + upload, warm
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            B.tqs_simulate_fsv(c, st)
        e.record()
        torch.cuda.synchronize()
        sec = s.elapsed_time(e) / 1e3 / reps
        alg = 16.0 * (1 << n) * passes
        flops = algorithmic_flops(n, ops)
        out[f"n{n}"] = {"gates": len(ops), "passes": passes, "tile_bits": tile,
                        "tile_autotune_ms": tiles[n]["timings_ms"], "ms": 1e3 * sec,
                        "gates_per_s": len(ops) / sec,
                        "hbm": {"achieved_gbs": alg / sec / 1e9, "peak": hbm_peak,
                                "frac": alg / sec / 1e9 / hbm_peak, "algorithmic_bytes": alg},
                        "alu": {"achieved_tflops": flops / sec / 1e12, "peak": fp32_peak,
                                "frac": flops / sec / 1e12 / fp32_peak,
                                "algorithmic_flops": flops}}
        B.tqs_circuit_destroy(c)
        del st
        torch.cuda.empty_cache()
    B.tqs_set_option(B.OPT_FSV_TILE_Q, 0, 0)  # the automatic choice for the legs below
    # The per-gate form of eq. 12 (one pass over the state per gate) at n = 24,
    # and the fused kernel on the same kind of circuit at n = 16 (its largest
    # size) beside the tiled passes.
    n = 24
    ops = W.random_layered(n, 10, (9, n))
    c = B.circuit_from_ops(n, ops)
    st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    st[0] = 1.0
    B.tqs_set_option(B.OPT_FSV_MAX_GATES, 0, 1)
    try:
        passes, _ = B.tqs_fsv_passes(c)
        B.tqs_simulate_fsv(c, st)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        B.tqs_simulate_fsv(c, st)
        e.record()
        torch.cuda.synchronize()
    finally:
        B.tqs_set_option(B.OPT_FSV_MAX_GATES, 0, 0)
    sec = s.elapsed_time(e) / 1e3
    alg = 16.0 * (1 << n) * passes
    out["per_gate_n24"] = {"passes": passes, "ms": 1e3 * sec,
                           "hbm": {"achieved_gbs": alg / sec / 1e9, "frac": alg / sec / 1e9 / hbm_peak},
                           "grouped_ms": out["n24"]["ms"]}
    B.tqs_circuit_destroy(c)
    del st
    n = 16
    ops = W.random_layered(n, 10, (9, n))
    c = B.circuit_from_ops(n, ops)
    st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    st[0] = 1.0
    fused_out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    times = {}

    def one_cta():
        B.tqs_set_option(B.OPT_MULTI_CTAS, 0, 1)
        try:
            B.tqs_simulate(c, fused_out)
        finally:
            B.tqs_set_option(B.OPT_MULTI_CTAS, 0, 8)
    for name, fn in (("fused_ms", lambda: B.tqs_simulate(c, fused_out)),
                     ("fused_one_cta_ms", one_cta),
                     ("fsv_ms", lambda: B.tqs_simulate_fsv(c, st))):
        fn()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(5):
            fn()
        e.record()
        torch.cuda.synchronize()
        times[name] = s.elapsed_time(e) / 5
    out["vs_fused_n16"] = dict(times, fsv_passes=B.tqs_fsv_passes(c)[0],
                               note="one circuit; fused_ms: the fused kernel on 8 CTAs "
                                    "(TEAM_MULTI, grid barrier per pass), fused_one_cta_ms: on one "
                                    "CTA (the batch form), fsv_ms: the tiled passes on the whole GPU")
    B.tqs_circuit_destroy(c)
    del st, fused_out
    torch.cuda.empty_cache()
    return out


def bench_chain(B, W, torch, peaks, mpeaks):
    """Algorithm 1 on the random layered circuits (20 layers, 40 steps) at
    n = 12, 13, 14: tensor-core BF16x3 chain (and FP32 SIMT at n = 12), with the
    error of sampled columns against the FP64 oracle at n = 12."""
    import numpy as np
    from oracle import fsv_route

    peak = peaks.get("bf16_tflops", 1927.5)
    tf32 = mpeaks.get("tf32_tflops")
    out = {"workload": "random layered: 20 x (U3 on every qubit + CNOTs on n/2 seeded pairs), "
                       "40 steps, U = S_40 ... S_1",
           "tensor_peak_tflops": peak, "peak_source": "measured bf16 burst",
           "tf32_peak_tflops": tf32, "tf32_peak_source": "measured TF32 cuBLAS burst (measured_peaks)"}
    names = {B.PREC_TC_BF16X3: "tc_bf16x3", B.PREC_TC_TF32X3: "tc_tf32x3",
             B.PREC_FP32_SIMT: "fp32_simt"}
    from paper_2305_14398_gb300 import autotune
    group13 = None
    for n, prec, reps in [(12, B.PREC_TC_BF16X3, 3), (12, B.PREC_TC_TF32X3, 2),
                          (12, B.PREC_FP32_SIMT, 1), (13, B.PREC_TC_BF16X3, 2),
                          (14, B.PREC_TC_BF16X3, 1)]:
        ops = W.random_layered(n, 20, (2, n))
        group = None
        if prec != B.PREC_FP32_SIMT:
            if n <= 13:
                group = autotune.tune_chain_group(n, ops, prec)
                if n == 13:
                    group13 = group
            else:  # one product at n = 14 takes about 50 ms: the n = 13 choice
                B.tqs_set_option(B.OPT_CHAIN_GROUP, 0, group13["value"] if group13 else 16)
                group = {"value": B.tqs_get_option(B.OPT_CHAIN_GROUP, 0), "timings_ms": {},
                         "source": "the n = 13 choice"}
        c = B.circuit_from_ops(n, ops)
        U = torch.empty((1 << n, 1 << n), dtype=torch.complex64, device="cuda")
        B.tqs_circuit_unitary(c, prec, U)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            B.tqs_circuit_unitary(c, prec, U)
        e.record()
        torch.cuda.synchronize()
        sec = s.elapsed_time(e) / 1e3 / reps
        N = 1 << n
        gemms = B.tqs_circuit_info(c)[2] - 1
        key = f"n{n}_{names[prec]}"
        rec = {"ms": 1e3 * sec, "gemms": gemms,
               "useful_complex_gflops": 8.0 * N ** 3 * gemms / sec / 1e9}
        if group is not None:
            rec["raster_group"] = {"chosen": group["value"], "autotune_ms": group["timings_ms"],
                                   "source": group["source"]}
        if prec != B.PREC_FP32_SIMT:
            issued = 18.0 * N ** 3 * gemms / sec / 1e12  # 3 real GEMMs x 3 split products
            rec["issued_tensor_tflops"] = issued
            own_peak = peak if prec == B.PREC_TC_BF16X3 else tf32
            rec["tensor_peak_tflops"] = own_peak
            rec["tensor_frac"] = issued / own_peak
            # useful work (a complex GEMM, 8 N^3 per product) against the
            # sustained peak of the precision (bf16 from MEASURED_PEAKS, TF32
            # measured by this bench): the fraction a caller gets per flop asked
            sus = (peaks.get("bf16_tflops_sustained") if prec == B.PREC_TC_BF16X3
                   else mpeaks.get("tf32_tflops_sustained"))
            if sus:
                rec["useful_tflops"] = 8.0 * N ** 3 * gemms / sec / 1e12
                rec["useful_frac_of_sustained"] = rec["useful_tflops"] / sus
                rec["sustained_peak_tflops"] = sus
        if n == 12:
            cols = [0, 1, 777, 2048, 4095]
            got = U[:, cols].cpu().numpy().astype(np.complex128)
            rec["max_abs_err_vs_oracle"] = float(np.max(np.abs(got - fsv_route.unitary_columns(n, ops, cols))))
        out[key] = rec
        B.tqs_circuit_destroy(c)
        del U
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------- cuBLAS reference points

def _cublas():
    """ctypes handle of the cuBLAS library torch has loaded (found in the
    process's mappings after a torch GEMM), or None."""
    import ctypes
    path = None
    try:
        with open("/proc/self/maps") as f:
            for ln in f:
                if "libcublas.so" in ln and "libcublasLt" not in ln:
                    path = ln.split()[-1]
                    break
    except OSError:
        return None
    if path is None:
        return None
    L = ctypes.CDLL(path)
    vp, i = ctypes.c_void_p, ctypes.c_int
    L.cublasSetStream_v2.argtypes = [vp, vp]
    L.cublasCgemm3m.argtypes = [vp, i, i, i, i, i, vp, vp, i, vp, i, vp, vp, i]
    L.cublasCgemv_v2.argtypes = [vp, i, i, i, vp, vp, i, vp, i, vp, vp, i]
    return L


def cublas_gemm3m(L, torch, S, U, out):
    """out = S @ U (row-major complex64, N x N) by cublasCgemm3m: in column-major
    terms out^T = U^T S^T."""
    import ctypes
    import numpy as np
    N = S.shape[0]
    h = ctypes.c_void_p(torch.cuda.current_blas_handle())
    L.cublasSetStream_v2(h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    one = np.array([1.0, 0.0], dtype=np.float32)
    zero = np.array([0.0, 0.0], dtype=np.float32)
    st = L.cublasCgemm3m(h, 0, 0, N, N, N, one.ctypes.data, ctypes.c_void_p(U.data_ptr()), N,
                         ctypes.c_void_p(S.data_ptr()), N, zero.ctypes.data,
                         ctypes.c_void_p(out.data_ptr()), N)
    if st != 0:
        raise RuntimeError(f"cublasCgemm3m status {st}")


def cublas_gemv(L, torch, S, x, y):
    """y = S x (row-major complex64 S, N x N) by cublasCgemv: column-major S^T,
    transposed."""
    import ctypes
    import numpy as np
    N = S.shape[0]
    h = ctypes.c_void_p(torch.cuda.current_blas_handle())
    L.cublasSetStream_v2(h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    one = np.array([1.0, 0.0], dtype=np.float32)
    zero = np.array([0.0, 0.0], dtype=np.float32)
    st = L.cublasCgemv_v2(h, 1, N, N, one.ctypes.data, ctypes.c_void_p(S.data_ptr()), N,
                          ctypes.c_void_p(x.data_ptr()), 1, zero.ctypes.data,
                          ctypes.c_void_p(y.data_ptr()), 1)
    if st != 0:
        raise RuntimeError(f"cublasCgemv status {st}")


def bench_cublas_plain(B, W, torch, n=11, reps=3):
    """Library yardstick for the plain form: cuBLAS cgemv on the same
    materialised step matrices S_k as matvec_kernel, one circuit of each paper
    kind.  Three timings per circuit, each a back-to-back run of all its steps:
    the library's materialisation alone (tqs_materialize_step), materialise +
    cuBLAS cgemv per step, and the library's plain form (tqs_simulate_plain:
    materialise + matvec_kernel per step); the mat-vecs' own times follow by
    difference."""
    import numpy as np
    from oracle import fsv_route
    torch.matmul(torch.ones(8, 8, device="cuda"), torch.ones(8, 8, device="cuda"))  # cuBLAS loaded
    L = _cublas()
    if L is None:
        return {"unavailable": "libcublas not found in the process"}
    N = 1 << n
    S = torch.empty((N, N), dtype=torch.complex64, device="cuda")
    x = torch.zeros(N, dtype=torch.complex64, device="cuda")
    y = torch.empty(N, dtype=torch.complex64, device="cuda")
    out = torch.empty(N, dtype=torch.complex64, device="cuda")
    t = {"mat": 0.0, "mat_cgemv": 0.0, "plain": 0.0}
    steps_all = 0
    err = 0.0
    for _, ops in W.paper_mix(n, 4, seed_tag=1):
        c = B.circuit_from_ops(n, ops)
        try:
            steps = B.tqs_circuit_info(c)[2]

            def run(kind):
                nonlocal x, y
                if kind == "plain":
                    B.tqs_simulate_plain(c, out)
                    return
                x.zero_()
                x[0] = 1.0
                for k in range(steps):
                    B.tqs_materialize_step(c, k, S)
                    if kind == "mat_cgemv":
                        cublas_gemv(L, torch, S, x, y)
                        x, y = y, x
            for kind in t:
                run(kind)
                torch.cuda.synchronize()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record()
                for _ in range(reps):
                    run(kind)
                s1.record()
                torch.cuda.synchronize()
                t[kind] += s0.elapsed_time(s1) / 1e3 / reps
            run("mat_cgemv")
            torch.cuda.synchronize()
            err = max(err, float(np.max(np.abs(x.cpu().numpy().astype(np.complex128)
                                              - fsv_route.simulate(n, ops)))))
            steps_all += steps
        finally:
            B.tqs_circuit_destroy(c)
    mv_lib = t["mat_cgemv"] - t["mat"]
    mv_ours = t["plain"] - t["mat"]
    return {"what": "cuBLAS cgemv (cublasCgemv) on the same materialised S_k; baseline only",
            "steps": steps_all,
            "materialize_us_per_step": 1e6 * t["mat"] / steps_all,
            "materialize_plus_cgemv_us_per_step": 1e6 * t["mat_cgemv"] / steps_all,
            "plain_form_us_per_step": 1e6 * t["plain"] / steps_all,
            "cgemv_us_per_step_derived": 1e6 * mv_lib / steps_all,
            "matvec_kernel_us_per_step_derived": 1e6 * mv_ours / steps_all,
            "cgemv_gbs_algorithmic": 8.0 * N * N * steps_all / mv_lib / 1e9 if mv_lib > 0 else None,
            "matvec_kernel_gbs_algorithmic": 8.0 * N * N * steps_all / mv_ours / 1e9 if mv_ours > 0 else None,
            "note": "S_k is read right after it is written (32 MiB, L2-resident) in both forms",
            "max_abs_err_vs_oracle": err}


def bench_cublas_chain(B, W, torch):
    """Library yardsticks for the chain (Algorithm 1, U <- S_k U): cuBLAS
    cgemm (torch.matmul complex64, FP32) and cgemm3m (ctypes) on the same step
    matrices (materialised by tqs_materialize_step) at n = 12 (whole chain,
    error against the oracle's columns) and n = 13, 14 (one product timed,
    times the chain's product count)."""
    import numpy as np
    from oracle import fsv_route
    L = _cublas()
    out = {"what": "cuBLAS complex64 GEMM chain on the same S_k; baseline only (never the hot path)"}
    for n in (12, 13, 14):
        N = 1 << n
        ops = W.random_layered(n, 20, (2, n))
        c = B.circuit_from_ops(n, ops)
        try:
            steps = B.tqs_circuit_info(c)[2]
            S = torch.empty((N, N), dtype=torch.complex64, device="cuda")
            U = torch.empty((N, N), dtype=torch.complex64, device="cuda")
            V = torch.empty((N, N), dtype=torch.complex64, device="cuda")
            for name in ("cgemm", "cgemm3m"):
                if name == "cgemm3m" and L is None:
                    out[f"n{n}_cublas_cgemm3m"] = {"unavailable": "libcublas not found in the process"}
                    continue
                full = n == 12
                ks = range(1, steps) if full else [1]
                B.tqs_materialize_step(c, 0, U)
                t = 0.0
                for k in ks:
                    B.tqs_materialize_step(c, k, S)
                    torch.cuda.synchronize()
                    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    s0.record()
                    if name == "cgemm":
                        torch.matmul(S, U, out=V)
                    else:
                        cublas_gemm3m(L, torch, S, U, V)
                    s1.record()
                    torch.cuda.synchronize()
                    t += s0.elapsed_time(s1) / 1e3
                    U, V = V, U
                per = t / len(ks)
                rec = {"ms_per_product": 1e3 * per, "chain_ms": 1e3 * per * (steps - 1),
                       "chain_ms_source": "timed" if full else "one product x (steps - 1)",
                       "useful_complex_tflops": 8.0 * N ** 3 / per / 1e12}
                if full:
                    cols = [0, 1, 777, 2048, 4095]
                    got = U[:, cols].cpu().numpy().astype(np.complex128)
                    rec["max_abs_err_vs_oracle"] = float(np.max(np.abs(
                        got - fsv_route.unitary_columns(n, ops, cols))))
                out[f"n{n}_cublas_{name}"] = rec
            del S, U, V
            torch.cuda.empty_cache()
        finally:
            B.tqs_circuit_destroy(c)
    return out


def bench_chain_sharded(B, W, torch, dist, rank, world, peaks, n=13, reps=2):
    """The column-sharded circuit-unitary chain (Algorithm 1 by column blocks):
    rank r computes U[:, block r] of the 40-step random layered chain at n = 13
    (BF16x3 tensor cores) with tqs_circuit_unitary_cols, generating every step
    unitary itself; no data is exchanged (only the timing: max over ranks).
    At one rank the block is the whole unitary."""
    from paper_2305_14398_gb300 import shard

    col0, ncols = shard.rank_block(n, rank, world)
    N = 1 << n
    ops = W.random_layered(n, 20, (2, n))
    c = B.circuit_from_ops(n, ops)
    sec = 0.0
    try:
        if ncols > 0:
            blk = torch.empty((N, ncols), dtype=torch.complex64, device="cuda")
            B.tqs_circuit_unitary_cols(c, B.PREC_TC_BF16X3, col0, ncols, blk)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            if ncols > 0:
                B.tqs_circuit_unitary_cols(c, B.PREC_TC_BF16X3, col0, ncols, blk)
        e.record()
        torch.cuda.synchronize()
        sec = s.elapsed_time(e) / 1e3 / reps
        gemms = B.tqs_circuit_info(c)[2] - 1
    finally:
        B.tqs_circuit_destroy(c)
    slowest = max_over_ranks(sec, dist, "cuda")
    useful = 8.0 * N * N * N * gemms  # complex MACs of all ranks' blocks together
    return {"workload": f"random layered n = {n}, 40 steps, BF16x3; rank r computes columns "
                        "shard.rank_block(n, r, world); no exchange",
            "ranks": world, "ms": 1e3 * slowest, "columns_per_rank": ncols,
            "useful_complex_gflops_whole_job": useful / slowest / 1e9 if slowest > 0 else None,
            "issued_tensor_tflops_whole_job": 18.0 * N ** 3 * gemms / slowest / 1e12 if slowest > 0 else None,
            "tensor_peak_tflops_per_gpu": peaks.get("bf16_tflops", 1927.5)}


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_tqs(args)


if __name__ == "__main__":
    sys.exit(main())

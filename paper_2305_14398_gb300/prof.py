"""Small driver for ncu captures of the fused step kernels.

    python -m paper_2305_14398_gb300.prof COUNT KIND REPS [noprobs] [TWxW]

chain: the 40-step random layered circuit-unitary chain at n = COUNT
       (tensor-core BF16x3); chain_tf32, chain_simt: the same in TF32x3 /
       FP32 SIMT;
probs: tqs_probabilities on a random 2^COUNT state;
sample: 64 inverse-CDF shots per circuit of COUNT paper-shaped 11-qubit
       circuits (tqs_batch_sample);
multi: one random layered circuit of COUNT = 15 or 16 qubits on cooperating
       CTAs (tqs_simulate);
plain: the plain materialised form (tqs_simulate_plain) on one circuit of each
       paper kind at n = COUNT, REPS times;
fsv:   the full-state-vector backend on a random layered circuit
       (10 x (U3 on every qubit + CNOTs on n/2 seeded pairs)) at n = COUNT;
mix:   COUNT paper-shaped 11-qubit circuits (GHZ / DJ-constant / DJ-balanced /
       QFT, 25 % each); ghz, dj_constant, dj_balanced, qft: COUNT circuits of one
       of those kinds; batch: the first COUNT circuits of the random batched
       workload (n = 4..14, depth 5..40); n14: COUNT random circuits at n = 14.
       Runs tqs_batch_run REPS times
       without a graph, then once more timed with CUDA events.
noprobs: the same without the FP64 probability output (d_probs = NULL).
TWxW (e.g. 2x16): warps per circuit and per CTA of the 11-qubit warp class
(the bench's autotuned shape), set before the batch is planned.
"""
import sys

import torch

from . import binding as B
from . import workloads as W


def chain(n, reps):
    ops = W.random_layered(n, 20, (2, n))
    c = B.circuit_from_ops(n, ops)
    U = torch.empty((1 << n, 1 << n), dtype=torch.complex64, device="cuda")
    for _ in range(reps):
        B.tqs_circuit_unitary(c, B.PREC_TC_BF16X3, U)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    B.tqs_circuit_unitary(c, B.PREC_TC_BF16X3, U)
    e.record()
    torch.cuda.synchronize()
    print("chain", n, "ms %.3f" % s.elapsed_time(e))
    B.tqs_circuit_destroy(c)


def fsv(n, reps):
    ops = W.random_layered(n, 10, (9, n))
    c = B.circuit_from_ops(n, ops)
    st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    st[0] = 1.0
    passes, _ = B.tqs_fsv_passes(c)
    for _ in range(reps):
        B.tqs_simulate_fsv(c, st)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    B.tqs_simulate_fsv(c, st)
    e.record()
    torch.cuda.synchronize()
    print("fsv", n, "passes", passes, "ms %.3f" % s.elapsed_time(e),
          "norm %.7f" % float((st.abs() ** 2).sum()))
    B.tqs_circuit_destroy(c)


def plain(n, reps):
    handles = [B.circuit_from_ops(n, ops) for _, ops in W.paper_mix(n, 4)]
    out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    for _ in range(reps):
        for h in handles:
            B.tqs_simulate_plain(h, out)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for h in handles:
        B.tqs_simulate_plain(h, out)
    e.record()
    torch.cuda.synchronize()
    steps = sum(B.tqs_circuit_info(h)[2] for h in handles)
    print("plain", n, "steps", steps, "ms %.3f" % s.elapsed_time(e))
    for h in handles:
        B.tqs_circuit_destroy(h)


def chain_prec(n, reps, prec):
    """The 40-step random layered chain at n in a given precision."""
    ops = W.random_layered(n, 20, (2, n))
    c = B.circuit_from_ops(n, ops)
    U = torch.empty((1 << n, 1 << n), dtype=torch.complex64, device="cuda")
    for _ in range(reps):
        B.tqs_circuit_unitary(c, prec, U)
    torch.cuda.synchronize()
    print("chain", n, "prec", prec, "done")
    B.tqs_circuit_destroy(c)


def probs(n, reps):
    """tqs_probabilities on a seeded random 2^n state."""
    g = W.rng(31, n)
    psi = torch.from_numpy((g.normal(size=1 << n) + 1j * g.normal(size=1 << n)).astype("complex64")).cuda()
    p = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    tot = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(reps):
        B.tqs_probabilities(psi, n, p, tot)
    torch.cuda.synchronize()
    print("probs", n, "sum %.6f" % float(tot.cpu()[0]))


def sample(count, reps, shots=64):
    """tqs_batch_sample: `shots` draws per circuit from the probabilities of a
    batch of `count` paper-shaped 11-qubit circuits."""
    circs = [(11, ops) for _, ops in W.paper_mix(11, count)]
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    c, total, _ = B.tqs_batch_info(b)
    st = torch.empty(total, dtype=torch.complex64, device="cuda")
    pr = torch.empty(total, dtype=torch.float64, device="cuda")
    B.tqs_batch_run(b, st, pr, None, use_graph=False)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(14398)
    u = torch.rand(c * shots, dtype=torch.float64, device="cuda", generator=gen)
    out = torch.empty(c * shots, dtype=torch.int64, device="cuda")
    for _ in range(reps):
        B.tqs_batch_sample(b, pr, shots, u, out)
    torch.cuda.synchronize()
    print("sample", count, "done")
    B.tqs_batch_destroy(b)


def multi(n, reps):
    """One random layered circuit of n = 15 or 16 qubits on cooperating CTAs
    (the fused kernel's TEAM_MULTI form)."""
    ops = W.random_layered(n, 10, (9, n))
    c = B.circuit_from_ops(n, ops)
    out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    for _ in range(reps):
        B.tqs_simulate(c, out)
    torch.cuda.synchronize()
    print("multi", n, "done")
    B.tqs_circuit_destroy(c)


def main(argv):
    count = int(argv[1]) if len(argv) > 1 else 2048
    kind = argv[2] if len(argv) > 2 else "mix"
    reps = int(argv[3]) if len(argv) > 3 else 4
    with_probs = "noprobs" not in argv[4:]
    for a in argv[4:]:
        if "x" in a and a.replace("x", "").isdigit():
            tw, w = (int(v) for v in a.split("x"))
            B.tqs_set_option(B.OPT_TEAM_WARPS, 11, tw)
            B.tqs_set_option(B.OPT_WARPS_PER_CTA, 11, w)
    if kind == "chain":
        return chain(count, reps)
    if kind == "chain_tf32":
        return chain_prec(count, reps, B.PREC_TC_TF32X3)
    if kind == "chain_simt":
        return chain_prec(count, reps, B.PREC_FP32_SIMT)
    if kind == "probs":
        return probs(count, reps)
    if kind == "sample":
        return sample(count, reps)
    if kind == "multi":
        return multi(count, reps)
    if kind == "fsv":
        return fsv(count, reps)
    if kind == "plain":
        return plain(count, reps)
    if kind == "mix":
        circs = [(11, ops) for _, ops in W.paper_mix(11, count)]
    elif kind in ("ghz", "dj_constant", "dj_balanced", "qft"):
        circs = [(11, ops) for k, ops in W.paper_mix(11, 4 * count) if k == kind]
    elif kind == "n14":
        circs = W.batch_circuits_fixed_n(count, 14)
    else:
        circs = W.batch_circuits(count, 3)
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    c, total, _ = B.tqs_batch_info(b)
    st = torch.empty(total, dtype=torch.complex64, device="cuda")
    pr = torch.empty(total, dtype=torch.float64, device="cuda") if with_probs else None
    nm = torch.empty(c, dtype=torch.float64, device="cuda")
    for _ in range(reps):
        B.tqs_batch_run(b, st, pr, nm, use_graph=False)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    B.tqs_batch_run(b, st, pr, nm, use_graph=False)
    e.record()
    torch.cuda.synchronize()
    print(kind, count, "ms %.4f" % s.elapsed_time(e),
          "norm err %.2e" % float((nm - 1).abs().max()))
    B.tqs_batch_destroy(b)


if __name__ == "__main__":
    main(sys.argv)

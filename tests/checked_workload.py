"""Workload run by test_gpu_checked.py in a child process against the normal
or the bounds-checked library (TQS_LIB), touching the kernels of every source
file: fused batches over every team kind (one and two warps per circuit),
measure/reset instructions, custom unitaries, the full-state-vector backend,
the plain materialised form, the circuit-unitary chain (FP32 SIMT and both
tensor-core splits), probabilities and marginals, sampling on its
shared-memory and global paths, simulateAndCollapse, and single 15-16 qubit
circuits on cooperating CTAs.  Prints one JSON
line: a digest of every output and the bounds-check violation count."""
import hashlib
import json
import sys

import numpy as np
import torch

from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import workloads as W
from oracle import gates


def rand_unitary(k, seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def main():
    B.lib()
    digest = hashlib.sha256()
    assert B.tqs_check_violations() == 0
    circs = W.batch_circuits(256, seed_tag=71) + [(n, W.qft(n)) for n in (1, 2, 3, 15, 16)]
    for tw in (1, 2):
        for q in range(4, 12):
            B.tqs_set_option(B.OPT_TEAM_WARPS, q, tw)
        b = B.tqs_batch_create_packed(*B.pack_ops(circs))
        count, total, _ = B.tqs_batch_info(b)
        st = torch.empty(total, dtype=torch.complex64, device="cuda")
        pr = torch.empty(total, dtype=torch.float64, device="cuda")
        nm = torch.empty(count, dtype=torch.float64, device="cuda")
        B.tqs_batch_run(b, st, pr, nm)
        torch.cuda.synchronize()
        digest.update(st.cpu().numpy().tobytes())
        digest.update(pr.cpu().numpy().tobytes())
        B.tqs_batch_destroy(b)
    for q in range(4, 12):
        B.tqs_set_option(B.OPT_TEAM_WARPS, q, 1)
    for n in (3, 11, 13, 16):
        ops = [("h", (q,), ()) for q in range(n)] + [("measure", (n // 2,), ()), ("reset", (0,), ())]
        ops += [("unitary", tuple(range(min(5, n))), gates.custom_params(rand_unitary(min(5, n), n)))]
        c = B.circuit_from_ops(n, ops)
        out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        u = torch.tensor([0.3, 0.6], dtype=torch.float64, device="cuda")
        oc = torch.empty(2, dtype=torch.int32, device="cuda")
        B.tqs_simulate_measured(c, out, u=u, outcomes=oc)
        torch.cuda.synchronize()
        digest.update(out.cpu().numpy().tobytes())
        digest.update(oc.cpu().numpy().tobytes())
        B.tqs_circuit_destroy(c)
    for n in (15, 16):  # single circuits on cooperating CTAs (TEAM_MULTI)
        c = B.circuit_from_ops(n, W.random_layered(n, 3, (78, n)))
        out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        pr = torch.empty(1 << n, dtype=torch.float64, device="cuda")
        nm = torch.empty(1, dtype=torch.float64, device="cuda")
        B.tqs_simulate(c, out, probs=pr, norm=nm)
        torch.cuda.synchronize()
        for t in (out, pr, nm):
            digest.update(t.cpu().numpy().tobytes())
        B.tqs_circuit_destroy(c)
    for n in (14, 20):
        ops = W.random_small(n, 3 * n, (72, n)) + [
            ("unitary", (n - 1, 0, n // 2), gates.custom_params(rand_unitary(3, 9)))]
        c = B.circuit_from_ops(n, ops)
        st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
        st[5] = 1.0
        B.tqs_simulate_fsv(c, st)
        torch.cuda.synchronize()
        digest.update(st.cpu().numpy().tobytes())
        B.tqs_circuit_destroy(c)
    for n in (3, 9):
        c = B.circuit_from_ops(n, W.random_mixed(n, 4, (73, n)))
        out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        B.tqs_simulate_plain(c, out)
        torch.cuda.synchronize()
        digest.update(out.cpu().numpy().tobytes())
        B.tqs_circuit_destroy(c)
    for n, prec in ((5, B.PREC_FP32_SIMT), (7, B.PREC_FP32_SIMT), (8, B.PREC_TC_BF16X3),
                    (8, B.PREC_TC_TF32X3)):
        c = B.circuit_from_ops(n, W.random_layered(n, 3, (74, n)))
        U = torch.empty((1 << n, 1 << n), dtype=torch.complex64, device="cuda")
        B.tqs_circuit_unitary(c, prec, U)
        torch.cuda.synchronize()
        digest.update(U.cpu().numpy().tobytes())
        B.tqs_circuit_destroy(c)
    for n in (6, 13, 17):
        c = B.circuit_from_ops(n, W.qft_on_basis(n, 5 % (1 << n)) if n <= 16 else
                               W.random_small(n, 2 * n, (75, n)))
        st = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        if n <= 16:
            B.tqs_simulate(c, st)
        else:
            st.zero_()
            st[0] = 1.0
            B.tqs_simulate_fsv(c, st)
        pr = torch.empty(1 << n, dtype=torch.float64, device="cuda")
        tot = torch.empty(2, dtype=torch.float64, device="cuda")
        B.tqs_probabilities(st, n, pr, tot[0:1])
        B.tqs_marginal_zero(st, n, 0b101, tot[1:2])
        shots = 3000
        gen = torch.Generator(device="cpu").manual_seed(n)
        u = torch.rand(shots, dtype=torch.float64, generator=gen).cuda()
        out = torch.empty(shots, dtype=torch.int64, device="cuda")
        B.tqs_sample(pr, n, shots, u, out)
        idx = torch.empty(1, dtype=torch.int64, device="cuda")
        if n <= 16:
            B.tqs_simulate_and_collapse(c, u[:1], idx, st)
        torch.cuda.synchronize()
        for t in (pr, tot, out, idx, st):
            digest.update(t.cpu().numpy().tobytes())
        B.tqs_circuit_destroy(c)
    circs = W.batch_circuits(64, seed_tag=76) + [(15, W.qft(15))]
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    count, total, _ = B.tqs_batch_info(b)
    st = torch.empty(total, dtype=torch.complex64, device="cuda")
    pr = torch.empty(total, dtype=torch.float64, device="cuda")
    B.tqs_batch_run(b, st, pr)
    shots = 500
    gen = torch.Generator(device="cpu").manual_seed(77)
    u = torch.rand(count * shots, dtype=torch.float64, generator=gen).cuda()
    out = torch.empty(count * shots, dtype=torch.int64, device="cuda")
    B.tqs_batch_sample(b, pr, shots, u, out)
    torch.cuda.synchronize()
    digest.update(out.cpu().numpy().tobytes())
    B.tqs_batch_destroy(b)
    print(json.dumps({"digest": digest.hexdigest(), "violations": B.tqs_check_violations(),
                      "lib": B.LIB_PATH}))


if __name__ == "__main__":
    sys.exit(main())

"""Circuits with measure / reset instructions and uniforms for them, shared
by the host-program and GPU tests (inputs only: seeded, no method arithmetic
beyond calling the oracle to keep draws away from decision boundaries)."""
import numpy as np

from oracle import collapse, fsv_route
from paper_2305_14398_gb300 import workloads as W


def safe_uniforms(n, ops, seed, margin=1e-4):
    """Uniforms whose every decision lies at least `margin` from the oracle's
    boundary S_0 / T, so that FP32 and FP64 states decide alike."""
    rng = np.random.default_rng(seed)
    k = sum(1 for name, _, _ in ops if name in collapse.INSTRUCTIONS)
    for _ in range(1000):
        u = rng.random(k)
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[0] = 1.0
        j, ok = 0, True
        for op in ops:
            if op[0] in collapse.INSTRUCTIONS:
                q = op[1][0]
                p = np.abs(psi) ** 2
                p0 = float(np.sum(p[((np.arange(1 << n) >> q) & 1) == 0])) / float(np.sum(p))
                if 0.0 < p0 < 1.0 and abs(u[j] - p0) < margin:
                    ok = False
                    break
                psi, _ = collapse.measure_qubit(psi, n, q, u[j], reset=(op[0] == "reset"))
                j += 1
            else:
                fsv_route.apply_op(psi, n, op)
        if ok:
            return u
    raise AssertionError("no safe uniforms")


def with_instructions(n, seed, count=4):
    """A random circuit with measure / reset instructions spliced in, including
    one first (on |0...0>), a SWAP before one, and an X right before another."""
    rng = np.random.default_rng(seed)
    ops = [("measure", (int(rng.integers(0, n)),), ())]
    body = W.random_small(n, 6 * n, (11, n, seed))
    cut = sorted(rng.choice(len(body), size=count, replace=False).tolist())
    prev = 0
    for j, c in enumerate(cut):
        ops += body[prev:c]
        q = int(rng.integers(0, n))
        if j == 1:
            ops.append(("x", (q,), ()))
        ops.append(("reset" if j % 2 else "measure", (q,), ()))
        prev = c
    ops += body[prev:]
    return ops

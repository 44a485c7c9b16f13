"""Seeded synthetic circuits: the inputs shared by the oracle tests, the CUDA
path and the bench.

This module only draws circuits.  It holds no arithmetic of the simulation
method (no gate matrices, no Kronecker products, no state updates): a circuit
is a list of operations ``(name, qubits, params)``, where ``name`` is one of

  h x y z s t r rx ry rz u3       single-qubit gates (params: angles in rad)
  cx cz cp cu                     controlled gates, qubits = (control, target)
  swap                            two-qubit swap, qubits = (a, b)

``r`` is the phase-shift gate R_phi of the paper's Table 1, ``cp`` its
controlled form; ``u3`` takes (theta, phi, lambda); ``cu`` takes the 8 real
numbers re/im of u00, u01, u10, u11.

Circuit shapes follow the paper's evaluated programs (Sec. 2.5 and Sec. 6:
fully entangled, Deutsch-Jozsa, QFT) and the synthetic batch / chain /
serving workloads built around them.  Qubit q is bit q of an amplitude index
(little-endian), controlled gates take (control, target).

Seeds: base seed 14398; every sub-stream seed is an output of SplitMix64
(Steele, Lea, Flood 2014) so that each circuit can be regenerated alone.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

Op = Tuple[str, Tuple[int, ...], Tuple[float, ...]]

BASE_SEED = 14398
_MASK64 = (1 << 64) - 1

ONE_QUBIT = ("h", "x", "y", "z", "s", "t", "r", "rx", "ry", "rz", "u3")
TWO_QUBIT = ("cx", "cz", "cp", "cu", "swap")
N_PARAMS = {"h": 0, "x": 0, "y": 0, "z": 0, "s": 0, "t": 0, "r": 1, "rx": 1,
            "ry": 1, "rz": 1, "u3": 3, "cx": 0, "cz": 0, "cp": 1, "cu": 8,
            "swap": 0}


def splitmix64(x: int) -> int:
    """One SplitMix64 output for state ``x`` (state advanced by the golden gamma)."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def sub_seed(*tags: int, base: int = BASE_SEED) -> int:
    """Seed of the sub-stream named by the integer path ``tags``."""
    s = base & _MASK64
    for t in tags:
        s = splitmix64((s ^ (t & _MASK64)) & _MASK64)
    return s


def rng(*tags: int) -> np.random.Generator:
    return np.random.default_rng(sub_seed(*tags))


# --------------------------------------------------------------------------
# The paper's programs (Sec. 2.5) and the Bell example (Sec. 2.4)
# --------------------------------------------------------------------------

def bell() -> List[Op]:
    """H(q0), CNOT(q0 -> q1): the Bell listing of Sec. 5.3."""
    return [("h", (0,), ()), ("cx", (0, 1), ())]


def ghz_chain(n: int) -> List[Op]:
    """Fully entangled circuit, chain form: H(q0), CNOT(q_i -> q_{i+1})."""
    ops: List[Op] = [("h", (0,), ())]
    ops += [("cx", (i, i + 1), ()) for i in range(n - 1)]
    return ops


def ghz_fanout(n: int) -> List[Op]:
    """Fully entangled circuit as drawn in Sec. 2.5: H(q0), then CNOTs from
    q0 to q_{n-1}, ..., q_1."""
    ops: List[Op] = [("h", (0,), ())]
    ops += [("cx", (0, t), ()) for t in range(n - 1, 0, -1)]
    return ops


def deutsch_jozsa(n: int, balanced: bool, seed_tags: Sequence[int]) -> List[Op]:
    """Deutsch-Jozsa on n-1 input qubits q0..q_{n-2} and ancilla q_{n-1}.

    The ancilla starts in |1> (an X gate), H on all qubits, the oracle U_f,
    then H on the inputs.  Balanced U_f: CNOT from each input in a seeded
    nonempty subset to the ancilla, wrapped in X gates on a seeded input
    mask.  Constant U_f: identity or X on the ancilla (seeded coin).
    """
    g = rng(*seed_tags)
    k = n - 1
    anc = n - 1
    ops: List[Op] = [("x", (anc,), ())]
    ops += [("h", (q,), ()) for q in range(n)]
    if balanced:
        subset = [q for q in range(k) if g.random() < 0.5]
        if not subset:
            subset = [int(g.integers(0, k))]
        mask = [q for q in range(k) if g.random() < 0.5]
        ops += [("x", (q,), ()) for q in mask]
        ops += [("cx", (q, anc), ()) for q in subset]
        ops += [("x", (q,), ()) for q in mask]
    else:
        if g.random() < 0.5:
            ops.append(("x", (anc,), ()))
    ops += [("h", (q,), ()) for q in range(k)]
    return ops


def basis_prep(n: int, x: int) -> List[Op]:
    """X gates that turn |0...0> into the basis state |x>."""
    return [("x", (q,), ()) for q in range(n) if (x >> q) & 1]


def qft(n: int) -> List[Op]:
    """QFT as drawn in Sec. 2.5 (read little-endian): for j = n-1 .. 0, H(q_j)
    then controlled phases R_{pi/2^{j-k}} from q_k (k = j-1 .. 0) onto q_j;
    then SWAP(q_i, q_{n-1-i}) for i < n/2."""
    ops: List[Op] = []
    for j in range(n - 1, -1, -1):
        ops.append(("h", (j,), ()))
        for k in range(j - 1, -1, -1):
            ops.append(("cp", (k, j), (math.pi / float(1 << (j - k)),)))
    for i in range(n // 2):
        ops.append(("swap", (i, n - 1 - i), ()))
    return ops


def qft_on_basis(n: int, x: int) -> List[Op]:
    return basis_prep(n, x) + qft(n)


# --------------------------------------------------------------------------
# Synthetic workloads
# --------------------------------------------------------------------------

def random_layered(n: int, layers: int, seed_tags: Sequence[int]) -> List[Op]:
    """Layers of U3 on every qubit (angles ~ U[0, 2pi)) followed by CNOTs on
    floor(n/2) disjoint pairs: a random permutation cut into consecutive
    pairs, each with a random orientation."""
    g = rng(*seed_tags)
    ops: List[Op] = []
    for _ in range(layers):
        ang = g.uniform(0.0, 2.0 * math.pi, size=(n, 3))
        for q in range(n):
            ops.append(("u3", (q,), (float(ang[q, 0]), float(ang[q, 1]), float(ang[q, 2]))))
        perm = g.permutation(n)
        for p in range(n // 2):
            a, b = int(perm[2 * p]), int(perm[2 * p + 1])
            if g.random() < 0.5:
                a, b = b, a
            ops.append(("cx", (a, b), ()))
    return ops


BATCH_GATES = ("h", "x", "y", "z", "s", "t", "rx", "ry", "rz", "cx", "cz", "cp")


def random_mixed(n: int, depth: int, seed_tags: Sequence[int]) -> List[Op]:
    """Random dense steps: each step walks the qubits in a seeded order and
    every still-free qubit draws a gate uniformly from BATCH_GATES; a
    two-qubit draw takes the next free qubit as its target (or is redrawn as
    a one-qubit type if no qubit is left).  Angles ~ U[0, 2pi)."""
    g = rng(*seed_tags)
    ops: List[Op] = []
    one = [x for x in BATCH_GATES if x not in ("cx", "cz", "cp")]
    for _ in range(depth):
        order = [int(q) for q in g.permutation(n)]
        i = 0
        while i < n:
            q = order[i]
            name = BATCH_GATES[int(g.integers(0, len(BATCH_GATES)))]
            if name in ("cx", "cz", "cp") and i + 1 >= n:
                name = one[int(g.integers(0, len(one)))]
            if name in ("cx", "cz", "cp"):
                t = order[i + 1]
                params = (float(g.uniform(0.0, 2.0 * math.pi)),) if name == "cp" else ()
                ops.append((name, (q, t), params))
                i += 2
            else:
                params = (float(g.uniform(0.0, 2.0 * math.pi)),) if name in ("rx", "ry", "rz") else ()
                ops.append((name, (q,), params))
                i += 1
    return ops


def batch_sizes(count: int, seed_tags: Sequence[int] = (3,)) -> List[Tuple[int, int]]:
    """(n, depth) pairs: n = floor(exp(U[ln 4, ln 15))) in 4..14, depth ~ U{5..40}."""
    g = rng(*seed_tags)
    out = []
    for _ in range(count):
        n = int(math.floor(math.exp(g.uniform(math.log(4.0), math.log(15.0)))))
        n = min(max(n, 4), 14)
        d = int(g.integers(5, 41))
        out.append((n, d))
    return out


def batch_circuits(count: int = 4096, seed_tag: int = 3) -> List[Tuple[int, List[Op]]]:
    """The batched workload: ``count`` random mixed circuits of uneven n and depth."""
    sizes = batch_sizes(count, (seed_tag,))
    return [(n, random_mixed(n, d, (seed_tag, 1, i))) for i, (n, d) in enumerate(sizes)]


def batch_circuits_fixed_n(count: int, n: int, seed_tag: int = 5) -> List[Tuple[int, List[Op]]]:
    """The batched workload with every circuit at ``n`` qubits (depth ~ U{5..40}):
    at n = 14 its states (128 KiB each) stream through HBM instead of L2."""
    g = rng(seed_tag, 0)
    depths = [int(g.integers(5, 41)) for _ in range(count)]
    return [(n, random_mixed(n, d, (seed_tag, 1, i))) for i, d in enumerate(depths)]


def paper_mix(n: int, count: int, seed_tag: int = 1) -> List[Tuple[str, List[Op]]]:
    """``count`` circuits shaped like the paper's n-qubit programs, cycling
    GHZ, DJ-constant, DJ-balanced and QFT on a seeded basis state."""
    out = []
    for i in range(count):
        kind = i % 4
        if kind == 0:
            out.append(("ghz", ghz_chain(n)))
        elif kind == 1:
            out.append(("dj_constant", deutsch_jozsa(n, False, (seed_tag, 2, i))))
        elif kind == 2:
            out.append(("dj_balanced", deutsch_jozsa(n, True, (seed_tag, 3, i))))
        else:
            x = int(rng(seed_tag, 4, i).integers(0, 1 << n))
            out.append(("qft", qft_on_basis(n, x)))
    return out


def asap_steps(ops) -> int:
    """Number of circuit steps when gates are packed as soon as possible (a
    gate goes into the step after the last one that touches any of its
    qubits): the step count of the library's step table, on the host."""
    last = {}
    steps = 0
    for _, qs, _ in ops:
        k = 1 + max((last.get(q, 0) for q in qs), default=0)
        for q in qs:
            last[q] = k
        steps = max(steps, k)
    return steps


def serving_requests(count: int = 20000, rate_hz: float = 2000.0, n_lo: int = 6,
                     n_hi: int = 16, seed_tag: int = 4):
    """Poisson arrivals at ``rate_hz``; n ~ U{n_lo..n_hi}; kinds 25% each of
    GHZ / Deutsch-Jozsa / QFT / random mixed (depth ~ U{5..40}).

    Returns a list of (arrival_s, kind, n, ops)."""
    g = rng(seed_tag)
    t = 0.0
    out = []
    for i in range(count):
        t += float(g.exponential(1.0 / rate_hz))
        n = int(g.integers(n_lo, n_hi + 1))
        kind = int(g.integers(0, 4))
        if kind == 0:
            ops, name = ghz_chain(n), "ghz"
        elif kind == 1:
            bal = bool(g.random() < 0.5)
            ops, name = deutsch_jozsa(n, bal, (seed_tag, 2, i)), "dj"
        elif kind == 2:
            x = int(g.integers(0, 1 << n))
            ops, name = qft_on_basis(n, x), "qft"
        else:
            d = int(g.integers(5, 41))
            ops, name = random_mixed(n, d, (seed_tag, 3, i)), "random"
        out.append((t, name, n, ops))
    return out


def random_small(n: int, n_ops: int, seed_tags: Sequence[int], names=None) -> List[Op]:
    """Any-gate random circuit for cross-checks (all gate kinds, incl. swap/cu)."""
    g = rng(*seed_tags)
    names = names or (ONE_QUBIT + (TWO_QUBIT if n >= 2 else ()))
    ops: List[Op] = []
    for _ in range(n_ops):
        name = names[int(g.integers(0, len(names)))]
        if name in TWO_QUBIT:
            a, b = (int(v) for v in g.choice(n, size=2, replace=False))
            qs = (a, b)
        else:
            qs = (int(g.integers(0, n)),)
        k = N_PARAMS[name]
        if name == "cu":
            # a random 2x2 unitary given by its entries: QR of a complex Gaussian
            z = g.normal(size=(2, 2)) + 1j * g.normal(size=(2, 2))
            qm, rm = np.linalg.qr(z)
            d = np.diag(rm)
            qm = qm * (d / np.abs(d))
            params = tuple(float(v) for e in qm.reshape(-1) for v in (e.real, e.imag))
        else:
            params = tuple(float(v) for v in g.uniform(0.0, 2.0 * math.pi, size=k))
        ops.append((name, qs, params))
    return ops

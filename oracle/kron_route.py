"""The unitary-matrix simulation method, literally (test infrastructure; see
the package header).

* Circuit steps (Sec. 5.2: the circuit model creates steps as operations are
  added).  The paper does not state its packing rule; the reading used here is
  "as soon as possible": an operation goes into the step after the last step
  that touches any of its qubits.  Operations in one step act on disjoint
  qubits, so results do not depend on the packing.
* Step unitary (Algorithm 2, eq. 9s1): the Kronecker product of the step's
  factors, identity on idle qubits.  Qubit q is bit q of the amplitude index
  (little-endian), so the factor list runs from q_{n-1} down to q_0 and
  S = F_{n-1} (x) ... (x) F_0.  A controlled gate enters as its projector sum
  (eq. 7): the step unitary is the sum of one Kronecker chain per choice of
  term of every controlled gate.  A SWAP factor is the permutation matrix that
  exchanges the two qubits' bits (it acts on qubits disjoint from the other
  factors, so it multiplies the Kronecker part on the right).
* State evolution: psi <- S_k psi, one dense matrix-vector product per step
  (eq. 11, applied step by step).
* Circuit unitary (Algorithm 1): result <- I; result <- S_k result per step.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import gates

Op = Tuple[str, Tuple[int, ...], Tuple[float, ...]]

MAX_DENSE_QUBITS = 12      # one 4096 x 4096 complex128 step matrix is 256 MiB
MAX_CONTROLLED_PER_STEP = 8


def validate(n: int, ops: Sequence[Op]) -> None:
    """Preconditions of each operation (Sec. 5.2): qubits in range, distinct,
    parameter count right."""
    if n < 1:
        raise ValueError("a circuit needs at least one qubit")
    for name, qs, ps in ops:
        if name == "unitary":
            gates.custom_matrix(qs, ps)
        else:
            want = 2 if gates.is_two_qubit(name) else 1
            if len(qs) != want:
                raise ValueError(f"{name} takes {want} qubit(s)")
        if any(q < 0 or q >= n for q in qs):
            raise ValueError(f"{name}: qubit out of range")
        if len(set(qs)) != len(qs):
            raise ValueError(f"{name}: repeated qubit")


def steps_asap(n: int, ops: Sequence[Op]) -> List[List[Op]]:
    """Pack operations into steps, each operation into the earliest step after
    every step that already touches one of its qubits."""
    validate(n, ops)
    last = [-1] * n
    steps: List[List[Op]] = []
    for op in ops:
        k = 1 + max(last[q] for q in op[1])
        while len(steps) <= k:
            steps.append([])
        steps[k].append(op)
        for q in op[1]:
            last[q] = k
    return steps


def _kron_chain(op_list: Sequence[np.ndarray]) -> np.ndarray:
    """Algorithm 2: result <- op_list[0]; result <- result (x) op for the rest."""
    result = op_list[0]
    for op in op_list[1:]:
        result = np.kron(result, op)
    return result


def _swap_column_map(n: int, swaps: Sequence[Tuple[int, int]]) -> np.ndarray:
    """sigma(c): index c with the bits of every swapped pair exchanged."""
    c = np.arange(1 << n, dtype=np.int64)
    out = c.copy()
    for a, b in swaps:
        ba = (c >> a) & 1
        bb = (c >> b) & 1
        out &= ~((1 << a) | (1 << b))
        out |= (bb << a) | (ba << b)
        c = out.copy()
    return out


def _embedded_custom(n: int, qs: Sequence[int], m: np.ndarray) -> np.ndarray:
    """A custom factor on qubits qs with identity on the others: entry (r, c) is
    m[local(r), local(c)] when r and c agree on every other qubit, else 0
    (the Kronecker product with the identity, for qubits in any order)."""
    dim = 1 << n
    idx = np.arange(dim, dtype=np.int64)
    local = np.zeros(dim, dtype=np.int64)
    mask = 0
    for t, q in enumerate(qs):
        local |= ((idx >> q) & 1) << t
        mask |= 1 << q
    same = (idx[:, None] & ~mask) == (idx[None, :] & ~mask)
    return np.where(same, m[local[:, None], local[None, :]], 0.0)


def step_unitary(n: int, step: Sequence[Op]) -> np.ndarray:
    """Dense 2^n x 2^n step unitary of one step (Algorithm 2 with eq. 7)."""
    if n > MAX_DENSE_QUBITS:
        raise ValueError("dense step unitary limited to n <= %d" % MAX_DENSE_QUBITS)
    fixed: Dict[int, np.ndarray] = {}
    controlled: List[Tuple[int, int, List[Tuple[np.ndarray, np.ndarray]]]] = []
    swaps: List[Tuple[int, int]] = []
    customs: List[Tuple[Tuple[int, ...], np.ndarray]] = []
    used = set()
    for name, qs, ps in step:
        for q in qs:
            if q in used:
                raise ValueError("operations of one step must act on disjoint qubits")
            used.add(q)
        if name == "unitary":
            customs.append((tuple(qs), gates.custom_matrix(qs, ps)))
        elif name == "swap":
            swaps.append((qs[0], qs[1]))
        elif gates.is_two_qubit(name):
            controlled.append((qs[0], qs[1], gates.two_qubit_terms(name, ps)))
        else:
            fixed[qs[0]] = gates.single_qubit_matrix(name, ps)
    if len(controlled) > MAX_CONTROLLED_PER_STEP:
        raise ValueError("too many controlled gates in one step for the expansion")
    dim = 1 << n
    s = np.zeros((dim, dim), dtype=np.complex128)
    term_ranges = [range(len(t)) for _, _, t in controlled]
    for choice in itertools.product(*term_ranges):
        per_qubit = dict(fixed)
        for (qa, qb, terms), k in zip(controlled, choice):
            per_qubit[qa] = terms[k][0]
            per_qubit[qb] = terms[k][1]
        op_list = [per_qubit.get(q, gates.I2) for q in range(n - 1, -1, -1)]
        s += _kron_chain(op_list)
    if swaps:
        s = s[:, _swap_column_map(n, swaps)]
    # custom factors act on qubits no other factor touches: they commute with
    # the rest and multiply it
    for qs, m in customs:
        s = s @ _embedded_custom(n, qs, m)
    return s


def simulate(n: int, ops: Sequence[Op], psi0: Optional[np.ndarray] = None) -> np.ndarray:
    """Final state: psi <- S_k psi for every step k (eq. 11)."""
    dim = 1 << n
    if psi0 is None:
        psi = np.zeros(dim, dtype=np.complex128)
        psi[0] = 1.0
    else:
        psi = np.asarray(psi0, dtype=np.complex128).copy()
    for step in steps_asap(n, ops):
        psi = step_unitary(n, step) @ psi
    return psi


def circuit_unitary(n: int, ops: Sequence[Op]) -> np.ndarray:
    """Algorithm 1: result <- I, then result <- S_k . result for every step."""
    result = np.eye(1 << n, dtype=np.complex128)
    for step in steps_asap(n, ops):
        result = step_unitary(n, step) @ result
    return result

"""Per-gate full-state-vector update (test infrastructure; see the package
header).

Appendix A, eq. 12: a single-qubit gate U = [[Ua, Ub], [Uc, Ud]] on qubit i
updates every pair of amplitudes whose indices differ only in bit i:
  a_{..0_i..} <- Ua a_{..0_i..} + Ub a_{..1_i..}
  a_{..1_i..} <- Uc a_{..0_i..} + Ud a_{..1_i..}
The paper says a similar formula holds for two-qubit gates; for a
controlled-U (eq. 7) it is the same update restricted to the indices whose
control bit is 1, and a SWAP exchanges the amplitudes whose two bits are 01
and 10.  This route never builds a step matrix, so it is an algorithm
independent of the Kronecker route.

States may carry trailing columns: shape (2^n,) or (2^n, k); each column is
updated alike (used for columns of a circuit unitary).
"""
from __future__ import annotations

from typing import Iterable, Optional, Sequence, Tuple

import numpy as np

from . import gates

Op = Tuple[str, Tuple[int, ...], Tuple[float, ...]]


def _indices_with(n: int, fixed: Iterable[Tuple[int, int]]) -> np.ndarray:
    """All indices in [0, 2^n) whose bit q equals v for every (q, v) in fixed."""
    idx = np.arange(1 << n, dtype=np.int64)
    keep = np.ones(idx.shape, dtype=bool)
    for q, v in fixed:
        keep &= ((idx >> q) & 1) == v
    return idx[keep]


def _pair_update(psi: np.ndarray, i0: np.ndarray, i1: np.ndarray, u: np.ndarray) -> None:
    a0 = psi[i0].copy()
    a1 = psi[i1].copy()
    psi[i0] = u[0, 0] * a0 + u[0, 1] * a1
    psi[i1] = u[1, 0] * a0 + u[1, 1] * a1


def apply_op(psi: np.ndarray, n: int, op: Op) -> None:
    """Apply one operation in place (eq. 12 and its two-qubit forms; a custom
    k-qubit unitary updates each group of 2^k amplitudes whose indices differ
    only in its qubits by its matrix)."""
    name, qs, ps = op
    if name == "unitary":
        m = gates.custom_matrix(qs, ps)
        base = _indices_with(n, [(q, 0) for q in qs])
        j = np.arange(m.shape[0], dtype=np.int64)
        local = np.zeros_like(j)
        for t, q in enumerate(qs):
            local |= ((j >> t) & 1) << q
        idx = base[:, None] + local[None, :]
        psi[idx] = np.tensordot(psi[idx], m, axes=([1], [1])) if psi.ndim == 1 else \
            np.einsum("gc...,rc->gr...", psi[idx], m)
    elif name == "swap":
        a, b = qs
        i01 = _indices_with(n, [(a, 0), (b, 1)])
        i10 = i01 ^ ((1 << a) | (1 << b))
        tmp = psi[i01].copy()
        psi[i01] = psi[i10]
        psi[i10] = tmp
    elif gates.is_two_qubit(name):
        c, t = qs
        u = gates.controlled_target_matrix(name, ps)
        i0 = _indices_with(n, [(c, 1), (t, 0)])
        _pair_update(psi, i0, i0 | (1 << t), u)
    else:
        (q,) = qs
        u = gates.single_qubit_matrix(name, ps)
        i0 = _indices_with(n, [(q, 0)])
        _pair_update(psi, i0, i0 | (1 << q), u)


def simulate(n: int, ops: Sequence[Op], psi0: Optional[np.ndarray] = None) -> np.ndarray:
    dim = 1 << n
    if psi0 is None:
        psi = np.zeros(dim, dtype=np.complex128)
        psi[0] = 1.0
    else:
        psi = np.array(psi0, dtype=np.complex128, copy=True)
    for op in ops:
        apply_op(psi, n, op)
    return psi


def unitary_columns(n: int, ops: Sequence[Op], cols: Sequence[int]) -> np.ndarray:
    """Columns U[:, j] of the circuit unitary: the circuit applied to e_j."""
    dim = 1 << n
    cols = np.asarray(list(cols), dtype=np.int64)
    m = np.zeros((dim, cols.size), dtype=np.complex128)
    m[cols, np.arange(cols.size)] = 1.0
    for op in ops:
        apply_op(m, n, op)
    return m

"""Probabilities and marginals of a state (test infrastructure; see the
package header).

Sec. 2.1 (eq. 2): the squared magnitudes of the amplitudes are the outcome
probabilities and sum to 1.  Sec. 5.2: simulateAndCollapse measures
according to these probabilities.  Sec. 2.5 (Deutsch-Jozsa): the answer is
read from the probability that the input register is all zero, the ancilla
marginalised out.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def probabilities(psi: np.ndarray) -> np.ndarray:
    """p_i = |psi_i|^2 in float64."""
    psi = np.asarray(psi, dtype=np.complex128)
    return psi.real * psi.real + psi.imag * psi.imag


def total(p: np.ndarray) -> float:
    return float(np.sum(np.asarray(p, dtype=np.float64)))


def marginal_zero(p: np.ndarray, qubits: Sequence[int]) -> float:
    """P(every qubit in ``qubits`` reads 0) = sum of p_i over the indices
    whose bits at those qubits are all 0."""
    p = np.asarray(p, dtype=np.float64)
    idx = np.arange(p.size, dtype=np.int64)
    mask = 0
    for q in qubits:
        mask |= 1 << q
    return float(np.sum(p[(idx & mask) == 0]))

"""Collapse, sampling and the measure / reset instructions (test
infrastructure; see the package header).

Sec. 5.2 (Simulator interface): simulateAndCollapse simulates a circuit and
returns only the collapsed state, the measurement being taken according to
the probabilities that the state vector gives (Sec. 2.1, eq. 2: p_i =
|psi_i|^2).  Sec. 5.2 (operation interface) also lists single-qubit
instructions: a measurement and a reset that brings the qubit back to its
initial state |0>.

The paper fixes neither how a random number selects the outcome nor the order
of the instruction's random draws; the readings used here:

* An outcome is selected from a uniform number u in [0, 1) by inverting the
  cumulative distribution: with C_i = p_0 + ... + p_i (summed in index order)
  and T = C_{N-1}, the sample is the smallest i with u T < C_i.  An index whose
  probability is 0 is therefore never returned.  Should rounding leave u T >=
  C_{N-1}, the last index with nonzero probability is returned.
* Measuring qubit q with u: S_0 = sum of p_i over the indices whose bit q is 0,
  T = sum of all p_i; the outcome is 0 when u T < S_0, else 1 (the same
  inverse-CDF rule over the two outcomes).  The state is projected on the
  outcome and divided by sqrt(S_b / T).
* Reset of qubit q with u: a measurement of q, then, if the outcome was 1, the
  X gate on q (the qubit ends in |0>).
* Each measure / reset instruction of a circuit takes the next uniform of the
  caller's array, in the order the instructions were added.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import fsv_route
from .observables import probabilities

INSTRUCTIONS = ("measure", "reset")


def sample_one(p: np.ndarray, u: float) -> int:
    """Inverse-CDF sample of one index: a plain loop over the definition."""
    p = np.asarray(p, dtype=np.float64)
    total = 0.0
    for x in p:
        total += float(x)
    target = float(u) * total
    c = 0.0
    for i, x in enumerate(p):
        c += float(x)
        if target < c:
            return i
    nz = np.nonzero(p > 0.0)[0]
    return int(nz[-1]) if nz.size else p.size - 1


def sample(p: np.ndarray, uniforms: Sequence[float]) -> np.ndarray:
    """``sample_one`` for every uniform (vectorised over the same cumulative
    sums, accumulated in index order)."""
    p = np.asarray(p, dtype=np.float64)
    c = np.cumsum(p)
    t = c[-1]
    u = np.asarray(uniforms, dtype=np.float64)
    idx = np.searchsorted(c, u * t, side="right")
    nz = np.nonzero(p > 0.0)[0]
    last = int(nz[-1]) if nz.size else p.size - 1
    return np.minimum(idx, last).astype(np.int64)


def collapse(psi: np.ndarray, u: float) -> Tuple[int, np.ndarray]:
    """simulateAndCollapse's last stage: the sampled index and the collapsed
    (basis) state |index>."""
    psi = np.asarray(psi, dtype=np.complex128)
    i = sample_one(probabilities(psi), u)
    out = np.zeros_like(psi)
    out[i] = 1.0
    return i, out


def measure_qubit(psi: np.ndarray, n: int, q: int, u: float, reset: bool = False
                  ) -> Tuple[np.ndarray, int]:
    """Projective measurement of qubit q (and, for a reset, the X gate when the
    outcome was 1).  Returns the new state and the outcome."""
    psi = np.asarray(psi, dtype=np.complex128)
    p = probabilities(psi)
    idx = np.arange(psi.size, dtype=np.int64)
    bit = (idx >> q) & 1
    s0 = float(np.sum(p[bit == 0]))
    t = float(np.sum(p))
    outcome = 0 if float(u) * t < s0 else 1
    s_b = s0 if outcome == 0 else t - s0
    out = np.where(bit == outcome, psi, 0.0) / np.sqrt(s_b / t)
    if reset and outcome == 1:
        flipped = np.zeros_like(out)
        flipped[idx ^ (1 << q)] = out
        out = flipped
    return out, outcome


def simulate_measured(n: int, ops: Sequence, uniforms: Sequence[float],
                      psi0: Optional[np.ndarray] = None) -> Tuple[np.ndarray, List[int]]:
    """Run a circuit whose op list may hold ("measure", (q,), ()) and
    ("reset", (q,), ()) instructions between its gates (gates by the per-gate
    update of eq. 12).  Returns the final state and the outcomes in order."""
    if psi0 is None:
        psi = np.zeros(1 << n, dtype=np.complex128)
        psi[0] = 1.0
    else:
        psi = np.array(psi0, dtype=np.complex128)
    outcomes: List[int] = []
    k = 0
    for op in ops:
        name, qubits = op[0], op[1]
        if name in INSTRUCTIONS:
            psi, b = measure_qubit(psi, n, int(qubits[0]), uniforms[k], reset=(name == "reset"))
            outcomes.append(b)
            k += 1
        else:
            fsv_route.apply_op(psi, n, op)
    return psi, outcomes

"""Gate matrices in complex128 (test infrastructure; see the package header).

Single-qubit gates are 2x2 matrices acting on (|0>, |1>) of their qubit.

* Table 1 (Sec. 2.3): H, X (Pauli-X, eq. 5), Y, Z and the phase shift
  R_phi = diag(1, e^{i phi}).
* S and T are named in Sec. 5.2 without matrices; their textbook forms are
  S = R_{pi/2} = diag(1, i) and T = R_{pi/4} = diag(1, e^{i pi/4}).
* RX, RY, RZ and U3 are not in the paper; they come from the synthetic
  workloads and use the textbook (OpenQASM 2) definitions:
  RX(t) = [[c, -i s], [-i s, c]], RY(t) = [[c, -s], [s, c]],
  RZ(t) = diag(e^{-i t/2}, e^{i t/2}) with c = cos(t/2), s = sin(t/2), and
  U3(t, p, l) = [[c, -e^{i l} s], [e^{i p} s, e^{i (p + l)} c]].

Two-qubit gates (Sec. 2.3, eq. 7): a controlled-U applies U to the target
when the control is |1>, i.e. it is the projector sum
  |0><0|_control (x) I_target + |1><1|_control (x) U_target,
returned here as the list of (operator on control, operator on target)
terms.  CNOT (eq. 8) is controlled-X, CZ controlled-Z, CP(phi) controlled
R_phi.  SWAP exchanges the two qubits' values and is the sum over a, b of
|a><b| (x) |b><a|.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
P0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)  # |0><0|
P1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)  # |1><1|


def _e(a: int, b: int) -> np.ndarray:
    """The matrix unit |a><b|."""
    m = np.zeros((2, 2), dtype=np.complex128)
    m[a, b] = 1.0
    return m


def single_qubit_matrix(name: str, params: Sequence[float] = ()) -> np.ndarray:
    """2x2 matrix of a single-qubit gate."""
    r2 = 1.0 / math.sqrt(2.0)
    if name == "h":
        return np.array([[r2, r2], [r2, -r2]], dtype=np.complex128)
    if name == "x":
        return np.array([[0, 1], [1, 0]], dtype=np.complex128)
    if name == "y":
        return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    if name == "z":
        return np.array([[1, 0], [0, -1]], dtype=np.complex128)
    if name == "r":
        (phi,) = params
        return np.array([[1, 0], [0, np.exp(1j * phi)]], dtype=np.complex128)
    if name == "s":
        return np.array([[1, 0], [0, 1j]], dtype=np.complex128)
    if name == "t":
        return np.array([[1, 0], [0, np.exp(1j * math.pi / 4.0)]], dtype=np.complex128)
    if name in ("rx", "ry", "rz"):
        (th,) = params
        c, s = math.cos(th / 2.0), math.sin(th / 2.0)
        if name == "rx":
            return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)
        if name == "ry":
            return np.array([[c, -s], [s, c]], dtype=np.complex128)
        return np.array([[np.exp(-0.5j * th), 0], [0, np.exp(0.5j * th)]], dtype=np.complex128)
    if name == "u3":
        th, ph, la = params
        c, s = math.cos(th / 2.0), math.sin(th / 2.0)
        return np.array([[c, -np.exp(1j * la) * s],
                         [np.exp(1j * ph) * s, np.exp(1j * (ph + la)) * c]], dtype=np.complex128)
    raise ValueError(f"not a single-qubit gate: {name}")


def controlled_target_matrix(name: str, params: Sequence[float] = ()) -> np.ndarray:
    """The U of a controlled-U gate."""
    if name == "cx":
        return single_qubit_matrix("x")
    if name == "cz":
        return single_qubit_matrix("z")
    if name == "cp":
        return single_qubit_matrix("r", params)
    if name == "cu":
        v = list(params)
        if len(v) != 8:
            raise ValueError("cu takes 8 numbers: re/im of u00, u01, u10, u11")
        return np.array([[v[0] + 1j * v[1], v[2] + 1j * v[3]],
                         [v[4] + 1j * v[5], v[6] + 1j * v[7]]], dtype=np.complex128)
    raise ValueError(f"not a controlled gate: {name}")


def two_qubit_terms(name: str, params: Sequence[float] = ()) -> List[Tuple[np.ndarray, np.ndarray]]:
    """A two-qubit gate as a sum of Kronecker terms (A on qubits[0], B on qubits[1])."""
    if name == "swap":
        return [(_e(a, b), _e(b, a)) for a in (0, 1) for b in (0, 1)]
    u = controlled_target_matrix(name, params)
    return [(P0, I2), (P1, u)]


def two_qubit_matrix_ct(name: str, params: Sequence[float] = ()) -> np.ndarray:
    """4x4 matrix in the paper's eq. 7 / eq. 8 labelling: rows and columns
    |first qubit, second qubit> = |00>, |01>, |10>, |11> (first = control)."""
    m = np.zeros((4, 4), dtype=np.complex128)
    for a, b in two_qubit_terms(name, params):
        m += np.kron(a, b)
    return m


def is_two_qubit(name: str) -> bool:
    return name in ("cx", "cz", "cp", "cu", "swap")


# ------------------------------------------------------------ custom unitaries
# Sec. 5.2 (operation interface): a custom unitary, registered by the user, is
# applied to a range of qubits.  Here it is the op ("unitary", qubits, params):
# k = len(qubits) qubits, params = the 2^k x 2^k matrix row-major as interleaved
# (re, im) numbers; bit t of the matrix's local index is qubit qubits[t]
# (little-endian, as for the state).

MAX_CUSTOM_QUBITS = 5


def custom_matrix(qubits: Sequence[int], params: Sequence[float]) -> np.ndarray:
    k = len(qubits)
    if not 1 <= k <= MAX_CUSTOM_QUBITS:
        raise ValueError("a custom unitary acts on 1..5 qubits")
    d = 1 << k
    v = np.asarray(params, dtype=np.float64)
    if v.size != 2 * d * d:
        raise ValueError(f"a {k}-qubit custom unitary takes {2 * d * d} numbers")
    return (v[0::2] + 1j * v[1::2]).reshape(d, d)


def custom_params(m: np.ndarray) -> Tuple[float, ...]:
    """The params of ("unitary", qubits, params) for matrix m."""
    m = np.asarray(m, dtype=np.complex128)
    out = np.empty(2 * m.size)
    out[0::2] = m.real.reshape(-1)
    out[1::2] = m.imag.reshape(-1)
    return tuple(out.tolist())

"""Pins of the oracle's custom k-qubit unitaries (Sec. 5.2: custom unitary
operations registered with the data provider and applied to qubits).

Closed forms and identities: a custom matrix equal to a built-in gate gives
that gate's result; a Kronecker product of single-qubit gates equals the
gates applied one by one (this fixes the local bit order: bit t = qubits[t]);
Toffoli and a 5-qubit cyclic shift act on basis states as the permutations
they are; the two oracle routes agree on random custom unitaries up to k = 5;
the circuit unitary stays unitary.  A planted reversal of the local bit order
fails the Kronecker pin.
"""
import numpy as np
import pytest

from oracle import fsv_route, gates, kron_route
from paper_2305_14398_gb300 import workloads as W


def rand_unitary(k, seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def unitary_op(qs, m):
    return ("unitary", tuple(qs), gates.custom_params(m))


def test_custom_equal_to_cnot():
    """CNOT (control c, target t) as a custom 2-qubit matrix on (c, t): local bit
    0 is c, bit 1 is t; the matrix flips bit 1 when bit 0 is 1."""
    m = np.zeros((4, 4))
    for j in range(4):
        out = j ^ 2 if j & 1 else j
        m[out, j] = 1.0
    n = 5
    pre = W.random_mixed(n, 4, (61, 1))
    for c, t in ((0, 3), (4, 1), (2, 0)):
        a = fsv_route.simulate(n, pre + [unitary_op((c, t), m)])
        b = fsv_route.simulate(n, pre + [("cx", (c, t), ())])
        assert np.max(np.abs(a - b)) < 1e-14
        assert np.max(np.abs(kron_route.simulate(n, pre + [unitary_op((c, t), m)]) - b)) < 1e-13


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_kronecker_of_single_gates(k):
    """M = U_{k-1} (x) ... (x) U_0 on qubits (q_0, ..., q_{k-1}) equals U_t applied
    to q_t for every t."""
    n = 7
    rng = np.random.default_rng(70 + k)
    qs = [int(q) for q in rng.permutation(n)[:k]]
    singles = []
    m = np.ones((1, 1), dtype=np.complex128)
    for t in range(k):
        ang = tuple(float(x) for x in rng.uniform(0, 2 * np.pi, 3))
        singles.append(("u3", (qs[t],), ang))
        m = np.kron(gates.single_qubit_matrix("u3", ang), m)
    pre = W.random_mixed(n, 3, (62, k))
    a = fsv_route.simulate(n, pre + [unitary_op(qs, m)])
    b = fsv_route.simulate(n, pre + singles)
    assert np.max(np.abs(a - b)) < 1e-13
    # a planted mistake, the local bit order reversed, is caught (k >= 2)
    if k >= 2:
        c = fsv_route.simulate(n, pre + [unitary_op(qs[::-1], m)])
        assert np.max(np.abs(c - b)) > 1e-3


def test_toffoli_and_cyclic_shift_permutations():
    """Toffoli on (c1, c2, t) flips t iff both controls are 1; a 5-qubit cyclic
    shift |x> -> |x + 1 mod 32> on (q_0..q_4) adds one to those bits."""
    tof = np.eye(8)
    tof[[3, 7]] = tof[[7, 3]]
    n = 6
    qs = (4, 0, 2)
    for x in range(1 << n):
        psi = fsv_route.simulate(n, W.basis_prep(n, x) + [unitary_op(qs, tof)])
        want = x ^ (1 << 2) if (x >> 4) & 1 and x & 1 else x
        assert abs(psi[want] - 1.0) < 1e-15
    shift = np.roll(np.eye(32), 1, axis=0)
    qs5 = (5, 1, 3, 0, 2)
    n = 7
    for x in (0, 5, 77, 127):
        psi = fsv_route.simulate(n, W.basis_prep(n, x) + [unitary_op(qs5, shift)])
        v = sum(((x >> q) & 1) << t for t, q in enumerate(qs5))
        v = (v + 1) % 32
        y = x & ~sum(1 << q for q in qs5)
        for t, q in enumerate(qs5):
            y |= ((v >> t) & 1) << q
        assert abs(psi[y] - 1.0) < 1e-15


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_two_routes_agree_with_customs(k):
    n = 8
    rng = np.random.default_rng(80 + k)
    ops = list(W.random_mixed(n, 3, (63, k)))
    for j in range(3):
        qs = [int(q) for q in rng.permutation(n)[:k]]
        ops.append(unitary_op(qs, rand_unitary(k, 100 * k + j)))
        ops += W.random_mixed(n, 2, (64, k, j))
    a = fsv_route.simulate(n, ops)
    b = kron_route.simulate(n, ops)
    assert np.max(np.abs(a - b)) < 1e-12
    u = kron_route.circuit_unitary(n, ops)
    assert np.max(np.abs(u.conj().T @ u - np.eye(1 << n))) < 1e-12
    cols = [0, 17, 255]
    assert np.max(np.abs(fsv_route.unitary_columns(n, ops, cols) - u[:, cols])) < 1e-12


def test_custom_shape_checks():
    with pytest.raises(ValueError):
        gates.custom_matrix((0, 1), [0.0] * 8)
    with pytest.raises(ValueError):
        gates.custom_matrix(tuple(range(6)), [0.0] * (2 * 4 ** 6))

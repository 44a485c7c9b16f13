"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them re-types the oracle's
own formulas: they compare with printed values (tests/golden), closed forms,
brute-force entry-by-entry definitions, textbook identities, or the second,
independent oracle route.
"""
import math

import numpy as np
import pytest

from conftest import read_named_matrices, read_token_matrix
from oracle import fsv_route, gates, kron_route, observables
from paper_2305_14398_gb300 import workloads as W

TOL = 1e-12


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


# ---------------------------------------------------------------- Table 1

def test_table1_printed_gates():
    """Table 1 (Sec. 2.3): H, X, Y, Z exactly as printed."""
    printed = read_named_matrices("table1_gates.txt")
    for key, name in (("H", "h"), ("X", "x"), ("Y", "y"), ("Z", "z")):
        assert maxabs(gates.single_qubit_matrix(name), printed[key]) < 1e-15


@pytest.mark.parametrize("phi", [0.0, 0.3, math.pi / 2, math.pi, 4.0])
def test_table1_phase_shift(phi):
    """Table 1: R_phi = [[1, 0], [0, e^{i phi}]]; S and T are R_{pi/2}, R_{pi/4}."""
    r = gates.single_qubit_matrix("r", (phi,))
    assert r[0, 0] == 1 and r[0, 1] == 0 and r[1, 0] == 0
    assert abs(r[1, 1] - complex(math.cos(phi), math.sin(phi))) < 1e-15
    assert maxabs(gates.single_qubit_matrix("s"), gates.single_qubit_matrix("r", (math.pi / 2,))) < 1e-15
    assert maxabs(gates.single_qubit_matrix("t"), gates.single_qubit_matrix("r", (math.pi / 4,))) < 1e-15


def test_eq6_x_swaps_amplitudes():
    """Eq. 6: X (alpha, beta) = (beta, alpha), through both routes."""
    psi = np.array([0.6, 0.8j])
    out_k = kron_route.simulate(1, [("x", (0,), ())], psi)
    out_f = fsv_route.simulate(1, [("x", (0,), ())], psi)
    assert maxabs(out_k, [0.8j, 0.6]) < 1e-15
    assert maxabs(out_f, [0.8j, 0.6]) < 1e-15


# ------------------------------------------------------- Kronecker mechanics

def test_eq9s1_step_matrix_printed():
    """Eq. 9s1: the printed 4x4 S_1 = H (x) I.  Under the little-endian
    reading the left factor is the most significant qubit, q1."""
    printed = read_token_matrix("eq9s1_S1.txt")
    s1 = kron_route.step_unitary(2, [("h", (1,), ())])
    assert maxabs(s1, printed) < 1e-15
    # H on q0 is then I (x) H, a different matrix
    s1b = kron_route.step_unitary(2, [("h", (0,), ())])
    assert maxabs(s1b, np.kron(np.eye(2), gates.single_qubit_matrix("h"))) < 1e-15
    assert maxabs(s1b, printed) > 0.5


def test_eq8_eq10_cnot_printed():
    """Eq. 8 / eq. 10: CNOT with rows |control, target>.  Little-endian:
    control q1, target q0 gives the printed matrix; the projector-sum 4x4
    in the control-first labelling is the printed matrix too."""
    printed = read_token_matrix("eq8_cnot.txt")
    assert maxabs(gates.two_qubit_matrix_ct("cx"), printed) == 0.0
    assert maxabs(kron_route.step_unitary(2, [("cx", (1, 0), ())]), printed) == 0.0


def test_eq7_controlled_u_structure():
    """Eq. 7: CU = diag(I, U) in the control-first labelling."""
    u = W.random_small(1, 1, (99, 1), names=("u3",))
    th, ph, la = u[0][2]
    um = gates.single_qubit_matrix("u3", (th, ph, la))
    params = tuple(v for e in um.reshape(-1) for v in (e.real, e.imag))
    m = gates.two_qubit_matrix_ct("cu", params)
    want = np.zeros((4, 4), dtype=complex)
    want[0, 0] = want[1, 1] = 1
    want[2:, 2:] = um
    assert maxabs(m, want) < 1e-15


def test_cz_pins():
    """CZ (controlled-Z, eq. 7 with U = Z of Table 1), pinned three ways that do
    not go through the oracle's own controlled-gate table:
    * on every basis state of 3 qubits, CZ(c, t) multiplies |x> by -1 exactly
      when bits c and t of x are both 1 and leaves it alone otherwise;
    * it is symmetric: CZ(c, t) = CZ(t, c) (a wrong table, e.g. C-X or C-Y,
      is not);
    * H_t CNOT(c, t) H_t = CZ(c, t), with CNOT pinned by the printed eq. 8 and
      H by the printed Table 1; and CZ = CP(pi) entrywise (R_pi = Z)."""
    n = 3
    pairs = [(c, t) for c in range(n) for t in range(n) if c != t]
    for c, t in pairs:
        for x in range(1 << n):
            e = np.zeros(1 << n, dtype=np.complex128)
            e[x] = 1.0
            sign = -1.0 if (x >> c) & 1 and (x >> t) & 1 else 1.0
            for route in (kron_route, fsv_route):
                prep = [("x", (q,), ()) for q in range(n) if (x >> q) & 1]
                assert maxabs(route.simulate(n, prep + [("cz", (c, t), ())]), sign * e) == 0.0
        u_ct = kron_route.step_unitary(n, [("cz", (c, t), ())])
        u_tc = kron_route.step_unitary(n, [("cz", (t, c), ())])
        assert maxabs(u_ct, u_tc) == 0.0
        h = kron_route.step_unitary(n, [("h", (t,), ())])
        cx = kron_route.step_unitary(n, [("cx", (c, t), ())])
        assert maxabs(h @ cx @ h, u_ct) < 1e-15
        assert maxabs(kron_route.step_unitary(n, [("cp", (c, t), (math.pi,))]), u_ct) < 1e-15


def test_eq11_bell_printed():
    """Eq. 11: S_2 S_1 |00> = (1/sqrt2, 0, 0, 1/sqrt2), for the printed
    matrices (mirror reading) and for the Bell listing H(0), CNOT(0, 1)."""
    printed = read_token_matrix("eq11_bell.txt").reshape(-1)
    mirror = [("h", (1,), ()), ("cx", (1, 0), ())]
    for ops in (mirror, W.bell()):
        assert maxabs(kron_route.simulate(2, ops), printed) < 1e-15
        assert maxabs(fsv_route.simulate(2, ops), printed) < 1e-15
    assert len(kron_route.steps_asap(2, W.bell())) == 2


def test_bell_reversed_control_does_not_entangle():
    """Sec. 5.3 listing: CNOT(0, 1) takes (control, target); reversing the
    order leaves the state a product state (control q1 is |0>)."""
    out = kron_route.simulate(2, [("h", (0,), ()), ("cx", (1, 0), ())])
    p = observables.probabilities(out)
    assert abs(p[3]) < 1e-30 and abs(p[1] - 0.5) < 1e-15


def _brute_step(n, step):
    """Step matrix entry by entry, from the definitions: a product over the
    step's factors of the factor's entry at the bits it acts on, and the
    identity (a Kronecker delta) on idle qubits.  Pure Python loops."""
    dim = 1 << n
    s = np.zeros((dim, dim), dtype=complex)
    for r in range(dim):
        for c in range(dim):
            v = 1.0 + 0j
            used = set()
            for name, qs, ps in step:
                used.update(qs)
                if name == "swap":
                    a, b = qs
                    ok = ((r >> a) & 1) == ((c >> b) & 1) and ((r >> b) & 1) == ((c >> a) & 1)
                    v *= 1.0 if ok else 0.0
                elif gates.is_two_qubit(name):
                    ct, tg = qs
                    u = gates.controlled_target_matrix(name, ps)
                    rc, cc = (r >> ct) & 1, (c >> ct) & 1
                    rt, col_t = (r >> tg) & 1, (c >> tg) & 1
                    if rc != cc:
                        v = 0.0
                    elif rc == 0:
                        v *= 1.0 if rt == col_t else 0.0
                    else:
                        v *= u[rt, col_t]
                else:
                    (q,) = qs
                    v *= gates.single_qubit_matrix(name, ps)[(r >> q) & 1, (c >> q) & 1]
            for q in range(n):
                if q not in used and ((r >> q) & 1) != ((c >> q) & 1):
                    v = 0.0
            s[r, c] = v
    return s


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_step_matrix_brute_force(n):
    """Algorithm 2 + eq. 7 against the entry-by-entry definition, n <= 5,
    for every gate kind including SWAP and a general controlled-U."""
    ops = W.random_small(n, 14, (77, n))
    for step in kron_route.steps_asap(n, ops):
        assert maxabs(kron_route.step_unitary(n, step), _brute_step(n, step)) < 1e-15


# --------------------------------------------------------- two routes agree

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_kron_route_equals_per_gate_route(n):
    """Algorithm 1/2 (Kronecker + dense matvec) vs eq. 12 (per gate), n <= 8."""
    ops = W.random_small(n, 6 * n, (11, n))
    a = kron_route.simulate(n, ops)
    b = fsv_route.simulate(n, ops)
    assert maxabs(a, b) < TOL


@pytest.mark.parametrize("n", [2, 4, 6])
def test_chain_columns(n):
    """Algorithm 1 chain vs the circuit applied to basis columns (eq. 12)."""
    ops = W.random_small(n, 5 * n, (12, n))
    u = kron_route.circuit_unitary(n, ops)
    cols = list(range(1 << n))
    assert maxabs(u, fsv_route.unitary_columns(n, ops, cols)) < TOL


def test_packing_does_not_change_result():
    """Operations on disjoint qubits commute, so the ASAP packing (the
    reading of "steps are created dynamically", Sec. 5.2) and any reordering
    of commuting operations give the same state."""
    n = 6
    ops = [("h", (0,), ()), ("x", (3,), ()), ("cx", (0, 1), ()), ("rz", (3,), (0.4,)),
           ("h", (5,), ()), ("cp", (5, 2), (1.1,)), ("swap", (1, 4), ())]
    reordered = [ops[1], ops[4], ops[0], ops[3], ops[2], ops[5], ops[6]]
    a = kron_route.simulate(n, ops)
    b = kron_route.simulate(n, reordered)
    assert maxabs(a, b) < TOL


# ------------------------------------------------------------ closed forms

def ghz_closed_form(n):
    v = np.zeros(1 << n, dtype=complex)
    v[0] = v[-1] = 2.0 ** -0.5
    return v


@pytest.mark.parametrize("n", list(range(2, 15)))
def test_ghz_closed_form(n):
    """Fully entangled circuit (Sec. 2.5): 1/sqrt2 on |0..0> and |1..1>."""
    want = ghz_closed_form(n)
    assert maxabs(fsv_route.simulate(n, W.ghz_chain(n)), want) < TOL
    assert maxabs(fsv_route.simulate(n, W.ghz_fanout(n)), want) < TOL
    if n <= 9:
        assert maxabs(kron_route.simulate(n, W.ghz_chain(n)), want) < TOL
        assert maxabs(kron_route.simulate(n, W.ghz_fanout(n)), want) < TOL


def dft_column(n, x):
    k = np.arange(1 << n)
    return np.exp(2j * np.pi * x * k / (1 << n)) / math.sqrt(1 << n)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_qft_closed_form_all_inputs(n):
    """QFT |x> = 2^{-n/2} sum_k e^{2 pi i x k / 2^n} |k> (textbook DFT reading
    of eq. qft), for every basis input, both routes."""
    for x in range(1 << n):
        want = dft_column(n, x)
        assert maxabs(kron_route.simulate(n, W.qft_on_basis(n, x)), want) < TOL
        assert maxabs(fsv_route.simulate(n, W.qft_on_basis(n, x)), want) < TOL


@pytest.mark.parametrize("n", [6, 8, 9, 11, 12])
def test_qft_closed_form_seeded(n):
    for i in range(3):
        x = int(W.rng(55, n, i).integers(0, 1 << n))
        want = dft_column(n, x)
        assert maxabs(fsv_route.simulate(n, W.qft_on_basis(n, x)), want) < TOL
        if n <= 8:
            assert maxabs(kron_route.simulate(n, W.qft_on_basis(n, x)), want) < TOL


def test_qft_unitary_is_dft_matrix():
    """The whole QFT circuit unitary (Algorithm 1) is the DFT matrix."""
    n = 5
    u = kron_route.circuit_unitary(n, W.qft(n))
    k = np.arange(1 << n)
    dft = np.exp(2j * np.pi * np.outer(k, k) / (1 << n)) / math.sqrt(1 << n)
    assert maxabs(u, dft) < TOL


@pytest.mark.parametrize("n", [2, 3, 5, 8, 11, 12])
@pytest.mark.parametrize("balanced", [False, True])
def test_deutsch_jozsa(n, balanced):
    """Deutsch-Jozsa (Sec. 2.5): P(input register = 0...0) is 1 for a constant
    oracle and 0 for a balanced one."""
    for i in range(4):
        ops = W.deutsch_jozsa(n, balanced, (21, n, i, int(balanced)))
        inputs = list(range(n - 1))
        routes = [fsv_route.simulate(n, ops)]
        if n <= 8:
            routes.append(kron_route.simulate(n, ops))
        for psi in routes:
            pz = observables.marginal_zero(observables.probabilities(psi), inputs)
            assert abs(pz - (0.0 if balanced else 1.0)) < TOL


# ------------------------------------------------------ unitarity, identities

@pytest.mark.parametrize("n", [1, 3, 6, 8, 10])
def test_circuit_unitary_is_unitary(n):
    """U^dagger U = I (Sec. 2.3), elementwise max norm <= 1e-12."""
    ops = W.random_small(n, 4 * n, (31, n))
    if n == 10:
        ops = W.random_layered(n, 2, (31, n))
    u = kron_route.circuit_unitary(n, ops)
    err = maxabs(u.conj().T @ u, np.eye(1 << n))
    assert err <= 1e-12


def test_reversibility():
    """U^dagger U psi = psi for a random state."""
    n = 5
    ops = W.random_small(n, 30, (41, 0))
    u = kron_route.circuit_unitary(n, ops)
    g = W.rng(41, 1)
    psi = g.normal(size=1 << n) + 1j * g.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    assert maxabs(u.conj().T @ (u @ psi), psi) < TOL


def test_norm_is_preserved():
    """Eq. 2: amplitudes stay normalised; probabilities sum to 1."""
    for n in (3, 7, 10):
        psi = fsv_route.simulate(n, W.random_mixed(n, 20, (42, n)))
        assert abs(observables.total(observables.probabilities(psi)) - 1.0) < TOL


def test_textbook_gate_identities():
    """Relations that fix the signs and phases of the rotation gates (not in
    the paper) and cross-check Table 1: HZH = X, HXH = Z, S^2 = Z, T^2 = S,
    Y = i X Z, RX(t) = U3(t, -pi/2, pi/2), RY(t) = U3(t, 0, 0),
    RZ(t) = e^{-i t/2} R_t, U3(pi/2, 0, pi) = H, RX(pi) = -i X."""
    m = gates.single_qubit_matrix
    assert maxabs(m("h") @ m("z") @ m("h"), m("x")) < 1e-15
    assert maxabs(m("h") @ m("x") @ m("h"), m("z")) < 1e-15
    assert maxabs(m("s") @ m("s"), m("z")) < 1e-15
    assert maxabs(m("t") @ m("t"), m("s")) < 1e-15
    assert maxabs(m("y"), 1j * m("x") @ m("z")) < 1e-15
    for t in (0.3, 1.7, 5.0):
        assert maxabs(m("rx", (t,)), m("u3", (t, -math.pi / 2, math.pi / 2))) < 1e-15
        assert maxabs(m("ry", (t,)), m("u3", (t, 0.0, 0.0))) < 1e-15
        assert maxabs(m("rz", (t,)), np.exp(-0.5j * t) * m("r", (t,))) < 1e-15
    assert maxabs(m("u3", (math.pi / 2, 0.0, math.pi)), m("h")) < 1e-15
    assert maxabs(m("rx", (math.pi,)), -1j * m("x")) < 1e-15
    for name, k in (("h", 0), ("x", 0), ("y", 0), ("z", 0), ("s", 0), ("t", 0), ("r", 1),
                    ("rx", 1), ("ry", 1), ("rz", 1), ("u3", 3)):
        u = m(name, tuple([0.9, 2.1, 4.4][:k]))
        assert maxabs(u.conj().T @ u, np.eye(2)) < 1e-15


def test_probability_observables():
    """Bell: P(|00>) = P(|11>) = 1/2; the marginal P(q0 = 0) = 1/2."""
    p = observables.probabilities(kron_route.simulate(2, W.bell()))
    assert abs(p[0] - 0.5) < 1e-15 and abs(p[3] - 0.5) < 1e-15
    assert abs(observables.marginal_zero(p, [0]) - 0.5) < 1e-15
    assert abs(observables.total(p) - 1.0) < 1e-15


def test_validation():
    """Preconditions are checked (Sec. 5.2)."""
    with pytest.raises(ValueError):
        kron_route.steps_asap(2, [("h", (2,), ())])
    with pytest.raises(ValueError):
        kron_route.steps_asap(2, [("cx", (1, 1), ())])
    with pytest.raises(ValueError):
        kron_route.steps_asap(2, [("cx", (1,), ())])


# ------------------------------------------------ planted mistakes are caught

def test_planted_kron_order_mistake_is_caught(monkeypatch):
    """Reversing the Kronecker factor order (big- instead of little-endian)
    must break the QFT closed form and the eq. 9s1 pin."""
    orig = kron_route._kron_chain
    monkeypatch.setattr(kron_route, "_kron_chain", lambda ops: orig(list(ops)[::-1]))
    n, x = 3, 3
    assert maxabs(kron_route.simulate(n, W.qft_on_basis(n, x)), dft_column(n, x)) > 1e-3
    assert maxabs(kron_route.step_unitary(2, [("h", (1,), ())]), read_token_matrix("eq9s1_S1.txt")) > 0.5


def test_planted_projector_mistake_is_caught(monkeypatch):
    """Projector-sum terms swapped (P1 (x) I + P0 (x) U) must break Bell."""
    orig = gates.two_qubit_terms

    def bad(name, params=()):
        t = orig(name, params)
        return [(gates.P1, t[0][1]), (gates.P0, t[1][1])] if name != "swap" else t

    monkeypatch.setattr(gates, "two_qubit_terms", bad)
    out = kron_route.simulate(2, W.bell())
    assert maxabs(out, read_token_matrix("eq11_bell.txt").reshape(-1)) > 0.1


def test_planted_sign_mistake_is_caught(monkeypatch):
    """A dropped minus sign in H must break GHZ-normalisation / QFT pins."""
    orig = gates.single_qubit_matrix

    def bad(name, params=()):
        m = orig(name, params)
        if name == "h":
            m = np.abs(m)
        return m

    monkeypatch.setattr(gates, "single_qubit_matrix", bad)
    psi = fsv_route.simulate(2, [("h", (0,), ()), ("h", (0,), ())])
    assert abs(observables.total(observables.probabilities(psi)) - 1.0) > 0.1


@pytest.mark.parametrize("wrong", ["x", "y", "s"])
def test_planted_cz_mistake_is_caught(monkeypatch, wrong):
    """A wrong CZ target matrix (C-X, C-Y or C-S) must break the CZ pins."""
    orig = gates.controlled_target_matrix

    def bad(name, params=()):
        if name == "cz":
            return gates.single_qubit_matrix(wrong)
        return orig(name, params)

    monkeypatch.setattr(gates, "controlled_target_matrix", bad)
    with pytest.raises(AssertionError):
        test_cz_pins()

"""Pins of the oracle's collapse, sampling and measure / reset instructions
(Sec. 5.2: simulateAndCollapse, measurement and reset instructions; Sec. 2.1,
eq. 2: outcome probabilities |psi_i|^2).

They check closed forms (Bell, GHZ, basis and |+> states), brute force
(an explicit loop over the definition), counting identities of the inverse
CDF on a uniform grid, invariants (norm 1 after a measurement, measurement
commuting with gates on other qubits), and planted mistakes that one of them
catches.
"""

import numpy as np

from oracle import collapse, fsv_route, observables
from paper_2305_14398_gb300 import workloads as W


def grid(k):
    return (np.arange(k) + 0.5) / k


# ------------------------------------------------------------ sampling

def test_sample_boundaries_closed_form():
    """Inverse CDF: u T < C_i picks i; a boundary value goes to the next index."""
    p = np.array([0.25, 0.25, 0.5])
    assert collapse.sample_one(p, 0.0) == 0
    assert collapse.sample_one(p, 0.2) == 0
    assert collapse.sample_one(p, 0.25) == 1
    assert collapse.sample_one(p, 0.3) == 1
    assert collapse.sample_one(p, 0.5) == 2
    assert collapse.sample_one(p, 0.999) == 2
    assert collapse.sample_one([0.5, 0.5], 0.5) == 1


def test_sample_never_returns_zero_probability():
    p = np.array([0.0, 0.25, 0.0, 0.0, 0.75, 0.0])
    got = set(collapse.sample(p, grid(4000)).tolist())
    assert got == {1, 4}


def test_sample_grid_counts_match_probabilities():
    """K uniforms on the grid (k + 1/2) / K: index i receives the grid points in
    [C_{i-1}, C_i) / T, i.e. K p_i / T of them up to one either way."""
    rng = np.random.default_rng(7)
    p = rng.random(37) ** 3
    p[[3, 11, 12]] = 0.0
    K = 100000
    idx = collapse.sample(p, grid(K))
    counts = np.bincount(idx, minlength=p.size)
    assert np.all(np.abs(counts - K * p / p.sum()) <= 1.0 + 1e-9)


def test_sample_vectorised_equals_loop():
    rng = np.random.default_rng(8)
    for size in (1, 2, 3, 17, 64):
        p = rng.random(size)
        p[rng.random(size) < 0.3] = 0.0
        if not p.any():
            p[0] = 1.0
        us = rng.random(50)
        assert collapse.sample(p, us).tolist() == [collapse.sample_one(p, u) for u in us]


def test_sample_unnormalised_input_scales_out():
    p = np.array([1.0, 3.0])
    assert collapse.sample_one(p, 0.24) == 0 and collapse.sample_one(p, 0.26) == 1


def test_collapse_ghz_only_all_zero_or_all_one():
    """GHZ closed form: the collapsed state is |0..0> or |1..1>, each for half of u."""
    n = 6
    psi = fsv_route.simulate(n, W.ghz_chain(n))
    outs = [collapse.collapse(psi, u)[0] for u in grid(200)]
    assert set(outs) == {0, (1 << n) - 1}
    assert outs.count(0) == 100
    i, st = collapse.collapse(psi, 0.7)
    assert i == (1 << n) - 1 and st[i] == 1 and np.count_nonzero(st) == 1


def test_collapse_basis_state_is_deterministic():
    n = 5
    psi = fsv_route.simulate(n, W.basis_prep(n, 19))
    assert {collapse.collapse(psi, u)[0] for u in grid(50)} == {19}


# ------------------------------------------------------ measure / reset

def test_measure_bell_closed_form():
    """Bell state (eq. 11): q0 reads 0 for u < 1/2 (state |00>), else 1 (|11>);
    q1 then reads the same for every u."""
    psi = fsv_route.simulate(2, W.bell())
    a, b = collapse.measure_qubit(psi, 2, 0, 0.3)
    assert b == 0 and np.allclose(a, [1, 0, 0, 0], atol=1e-15)
    a, b = collapse.measure_qubit(psi, 2, 0, 0.6)
    assert b == 1 and np.allclose(a, [0, 0, 0, 1], atol=1e-15)
    for u in (0.01, 0.5, 0.99):
        _, b2 = collapse.measure_qubit(a, 2, 1, u)
        assert b2 == 1


def test_measure_reads_the_named_qubit():
    """|q2 q1 q0> = |010>: q1 reads 1, q0 and q2 read 0, for any u."""
    psi = fsv_route.simulate(3, [("x", (1,), ())])
    for u in (0.0, 0.5, 0.999):
        assert collapse.measure_qubit(psi, 3, 1, u)[1] == 1
        assert collapse.measure_qubit(psi, 3, 0, u)[1] == 0
        assert collapse.measure_qubit(psi, 3, 2, u)[1] == 0


def test_measure_plus_state_probability_half():
    psi = fsv_route.simulate(1, [("h", (0,), ())])
    outs = [collapse.measure_qubit(psi, 1, 0, u)[1] for u in grid(1000)]
    assert sum(outs) == 500


def test_measure_ghz_all_outcomes_agree():
    n = 7
    ops = W.ghz_chain(n) + [("measure", (q,), ()) for q in (3, 0, 6, 1, 5, 2, 4)]
    for u0 in (0.1, 0.9):
        us = [u0] + list(np.random.default_rng(3).random(n - 1))
        psi, outs = collapse.simulate_measured(n, ops, us)
        assert len(set(outs)) == 1 and outs[0] == (0 if u0 < 0.5 else 1)
        assert abs(abs(psi[0 if outs[0] == 0 else (1 << n) - 1]) - 1.0) < 1e-12


def test_measure_norm_and_born_rule_random():
    """After a measurement the state has norm 1, and outcome 1 occurs for the
    fraction P1 of a uniform grid of u (Born rule, eq. 2)."""
    n = 6
    ops = W.random_mixed(n, 8, (91, 1))
    psi = fsv_route.simulate(n, ops)
    p = observables.probabilities(psi)
    for q in range(n):
        p1 = float(np.sum(p[((np.arange(1 << n) >> q) & 1) == 1]))
        K = 20000
        ones = sum(collapse.measure_qubit(psi, n, q, u)[1] for u in grid(K))
        assert abs(ones - K * p1) <= 1.0
        for u in (0.2, 0.7):
            a, _ = collapse.measure_qubit(psi, n, q, u)
            assert abs(np.vdot(a, a).real - 1.0) < 1e-12


def test_measure_commutes_with_gates_elsewhere():
    """A gate on other qubits before or after the measurement of q gives the
    same outcome and state (projector on q and unitary on the rest commute)."""
    n = 5
    pre = W.random_mixed(n, 6, (92, 1))
    other = [("u3", (1,), (0.3, 1.1, 2.0)), ("cx", (3, 4), ()), ("rz", (0,), (0.4,))]
    for u in (0.15, 0.55, 0.95):
        a, oa = collapse.simulate_measured(n, pre + [("measure", (2,), ())] + other, [u])
        b, ob = collapse.simulate_measured(n, pre + other + [("measure", (2,), ())], [u])
        assert oa == ob and np.max(np.abs(a - b)) < 1e-12


def test_reset_returns_qubit_to_zero():
    """Reset brings the qubit to |0>: from |1>, from |+>, and on an entangled
    Bell pair (where q1 keeps the measured value)."""
    for u in (0.1, 0.6, 0.99):
        psi, outs = collapse.simulate_measured(1, [("x", (0,), ()), ("reset", (0,), ())], [u])
        assert outs == [1] and np.allclose(psi, [1, 0], atol=1e-15)
        psi, outs = collapse.simulate_measured(1, [("h", (0,), ()), ("reset", (0,), ())], [u])
        assert np.allclose(psi, [1, 0], atol=1e-12)
        psi, outs = collapse.simulate_measured(2, W.bell() + [("reset", (0,), ())], [u])
        want = np.zeros(4)
        want[2 * outs[0]] = 1.0
        assert np.allclose(psi, want, atol=1e-12)


def test_uniforms_are_taken_in_instruction_order():
    ops = [("h", (0,), ()), ("h", (1,), ()), ("measure", (0,), ()), ("measure", (1,), ())]
    _, outs = collapse.simulate_measured(2, ops, [0.1, 0.9])
    assert outs == [0, 1]
    _, outs = collapse.simulate_measured(2, ops, [0.9, 0.1])
    assert outs == [1, 0]


# ------------------------------------------------------ planted mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """A measurement without renormalisation, a flipped decision, and a
    sampler with <= in place of < each fail one of the pins above."""
    psi = fsv_route.simulate(2, W.bell())

    def no_renorm(psi, n, q, u, reset=False):
        psi = np.asarray(psi, dtype=np.complex128)
        bit = (np.arange(psi.size) >> q) & 1
        p = observables.probabilities(psi)
        s0 = float(np.sum(p[bit == 0]))
        b = 0 if u * float(np.sum(p)) < s0 else 1
        return np.where(bit == b, psi, 0.0), b

    a, _ = no_renorm(psi, 2, 0, 0.3)
    assert abs(np.vdot(a, a).real - 1.0) > 1e-3

    def flipped(psi, n, q, u, reset=False):
        out, b = collapse.measure_qubit(psi, n, q, 1.0 - u, reset)
        return out, b

    assert flipped(psi, 2, 0, 0.3)[1] != 0

    def sample_le(p, u):
        p = np.asarray(p, dtype=np.float64)
        c = np.cumsum(p)
        return int(np.searchsorted(c, u * c[-1], side="left"))

    assert sample_le([0.25, 0.25, 0.5], 0.25) != collapse.sample_one([0.25, 0.25, 0.5], 0.25)

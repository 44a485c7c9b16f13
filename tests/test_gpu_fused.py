"""GPU parity of the fused step kernel, the plain materialised form and the
probability reduction against the FP64 oracle, through the C ABI.

Tolerances (stated by the target of this build for the FP32 path):
max |delta amplitude| <= 1e-5 and |1 - sum p| <= 1e-6 for n <= 14.
"""
import math

import numpy as np
import pytest

from oracle import fsv_route, kron_route, observables
from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import workloads as W

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
NORM_TOL = 1e-6

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    yield
    torch.cuda.synchronize()


def simulate_gpu(n, ops, init=None, with_probs=True):
    c = B.circuit_from_ops(n, ops)
    try:
        out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        probs = torch.empty(1 << n, dtype=torch.float64, device="cuda") if with_probs else None
        norm = torch.empty(1, dtype=torch.float64, device="cuda")
        d_init = None
        if init is not None:
            d_init = torch.from_numpy(np.asarray(init, dtype=np.complex64)).cuda()
        B.tqs_simulate(c, out, init=d_init, probs=probs, norm=norm)
        torch.cuda.synchronize()
        return (out.cpu().numpy(), None if probs is None else probs.cpu().numpy(),
                float(norm.cpu()[0]))
    finally:
        B.tqs_circuit_destroy(c)


def simulate_plain_gpu(n, ops):
    c = B.circuit_from_ops(n, ops)
    try:
        out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        B.tqs_simulate_plain(c, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        B.tqs_circuit_destroy(c)


def check_state(got, want, probs=None, norm=None):
    assert np.max(np.abs(got.astype(np.complex128) - want)) <= AMP_TOL
    if probs is not None:
        assert np.max(np.abs(probs - observables.probabilities(want))) <= 2 * AMP_TOL
        # the GPU probabilities are |amp|^2 of the FP32 state it wrote, formed in
        # FP32 arithmetic (default): within 2^-22 relative of the exact value
        g = got.astype(np.complex128)
        exact = g.real ** 2 + g.imag ** 2
        assert np.all(np.abs(probs - exact) <= 2.0 ** -22 * exact + 1e-44)
    if norm is not None:
        assert abs(norm - 1.0) <= NORM_TOL


# --------------------------------------------------------------- config 0/1

def test_exact_probabilities_option():
    """TQS_OPT_EXACT_PROBS = 1: the probabilities are the exact squares of the
    FP32 parts rounded once to FP64, bit for bit; the state and the norm do not
    change with the option."""
    n = 11
    ops = W.random_mixed(n, 12, (96, n))
    res = {}
    for exact in (0, 1):
        B.tqs_set_option(B.OPT_EXACT_PROBS, 0, exact)
        try:
            c = B.circuit_from_ops(n, ops)
            try:
                out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
                pr = torch.empty(1 << n, dtype=torch.float64, device="cuda")
                nm = torch.empty(1, dtype=torch.float64, device="cuda")
                B.tqs_simulate(c, out, probs=pr, norm=nm)
                torch.cuda.synchronize()
                res[exact] = (out.cpu().numpy(), pr.cpu().numpy(), float(nm.cpu()[0]))
            finally:
                B.tqs_circuit_destroy(c)
        finally:
            B.tqs_set_option(B.OPT_EXACT_PROBS, 0, 0)
    (s0, p0, n0), (s1, p1, n1) = res[0], res[1]
    assert np.array_equal(s0.view(np.uint32), s1.view(np.uint32)) and n0 == n1
    g = s1.astype(np.complex128)
    assert np.array_equal(p1, g.real ** 2 + g.imag ** 2)
    assert np.all(np.abs(p0 - p1) <= 2.0 ** -22 * p1 + 1e-44)
    assert np.all(p0.astype(np.float32) == p0)  # FP32 values, stored as FP64


def test_config0_ghz5_closed_form():
    """5-qubit fully entangled circuit: 1/sqrt2 on |00000> and |11111>."""
    got, probs, norm = simulate_gpu(5, W.ghz_chain(5))
    want = np.zeros(32, dtype=complex)
    want[0] = want[31] = 2 ** -0.5
    check_state(got, want, probs, norm)
    check_state(simulate_plain_gpu(5, W.ghz_chain(5)), want)


@pytest.mark.parametrize("kind", ["ghz", "dj_constant", "dj_balanced", "qft"])
def test_config1_n11(kind):
    """11-qubit paper circuits, fused and plain forms, against the oracle."""
    mix = [c for c in W.paper_mix(11, 8) if c[0] == kind]
    for _, ops in mix:
        want = fsv_route.simulate(11, ops)
        got, probs, norm = simulate_gpu(11, ops)
        check_state(got, want, probs, norm)
        check_state(simulate_plain_gpu(11, ops), want)


def test_dj_marginal_on_gpu():
    """Deutsch-Jozsa: P(inputs = 0) is 1 (constant) / 0 (balanced), by tqs_marginal_zero."""
    n = 11
    for bal in (False, True):
        ops = W.deutsch_jozsa(n, bal, (50, int(bal)))
        c = B.circuit_from_ops(n, ops)
        try:
            st = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
            B.tqs_simulate(c, st)
            out = torch.empty(1, dtype=torch.float64, device="cuda")
            B.tqs_marginal_zero(st, n, (1 << (n - 1)) - 1, out)
            pz = float(out.cpu()[0])
        finally:
            B.tqs_circuit_destroy(c)
        assert abs(pz - (0.0 if bal else 1.0)) <= NORM_TOL


def test_qft_closed_form_gpu():
    for n in (3, 8, 11, 13):
        x = int(W.rng(51, n).integers(0, 1 << n))
        k = np.arange(1 << n)
        want = np.exp(2j * np.pi * x * k / (1 << n)) / math.sqrt(1 << n)
        got, probs, norm = simulate_gpu(n, W.qft_on_basis(n, x))
        check_state(got, want, probs, norm)


# ------------------------------------------------- random circuits, all n

@pytest.mark.parametrize("n", list(range(1, 17)))
def test_random_all_gate_kinds(n):
    """Every gate kind (incl. SWAP and general controlled-U) at every size;
    warp teams (n <= 11), CTA teams (12..14) and global-memory teams (15, 16)."""
    reps = 3 if n <= 12 else 1
    for k in range(reps):
        ops = W.random_small(n, 12 * n, (52, n, k))
        want = fsv_route.simulate(n, ops)
        got, probs, norm = simulate_gpu(n, ops)
        check_state(got, want, probs, norm)


@pytest.mark.parametrize("n", [4, 9, 12, 14])
def test_random_mixed_deep(n):
    ops = W.random_mixed(n, 40, (53, n))
    want = fsv_route.simulate(n, ops)
    got, probs, norm = simulate_gpu(n, ops)
    check_state(got, want, probs, norm)


@pytest.mark.parametrize("n", [1, 3, 6, 11, 13, 15])
def test_initial_state(n):
    g = W.rng(54, n)
    psi0 = g.normal(size=1 << n) + 1j * g.normal(size=1 << n)
    psi0 /= np.linalg.norm(psi0)
    ops = W.random_small(n, 6 * n, (54, n))
    want = fsv_route.simulate(n, ops, psi0.astype(np.complex64).astype(np.complex128))
    got, probs, norm = simulate_gpu(n, ops, init=psi0)
    check_state(got, want, probs, norm)


@pytest.mark.parametrize("n", [5, 9, 11, 13, 15])
def test_basis_start_reached_a_few_qubits_at_a_time(n):
    """A basis-state start |x> (random x) whose gates reach the qubits three at
    a time: the first passes hold groups that are provably zero and are not
    worked (their far bits differ from x outside the positions the passes so
    far had as local ones).  States match the oracle, and every amplitude the
    oracle leaves exactly zero is exactly zero."""
    g = W.rng(55, n)
    for k in range(3):
        x = int(g.integers(0, 1 << n))
        ops = W.basis_prep(n, x)
        order = [int(q) for q in g.permutation(n)]
        for b in range(0, n, 3):
            block = order[b:b + 3]
            if len(block) < 2:
                block = block + [order[0]]
            sub = W.random_small(len(block), 4 * len(block), (55, n, k, b))
            ops += [(name, tuple(block[q] for q in qs), ps) for name, qs, ps in sub]
        want = fsv_route.simulate(n, ops)
        got, probs, norm = simulate_gpu(n, ops)
        check_state(got, want, probs, norm)
        zero = want == 0
        assert np.all(got[zero] == 0), (n, k, int(np.count_nonzero(got[zero])))


def test_empty_and_identity_circuits():
    for n in (1, 4, 12):
        got, probs, norm = simulate_gpu(n, [])
        want = np.zeros(1 << n, dtype=complex)
        want[0] = 1
        check_state(got, want, probs, norm)
    # swaps only: a pure relabeling
    n = 6
    ops = W.basis_prep(n, 0b000101) + [("swap", (0, 5), ()), ("swap", (2, 3), ())]
    got, _, _ = simulate_gpu(n, ops)
    check_state(got, fsv_route.simulate(n, ops))


# ------------------------------------------------------------ plain form

@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_materialize_step_matches_oracle(n):
    """Algorithm 2 on the GPU against the oracle's Kronecker step matrix."""
    ops = W.random_small(n, 5 * n, (55, n))
    steps = kron_route.steps_asap(n, ops)
    c = B.circuit_from_ops(n, ops)
    try:
        S = torch.empty((1 << n, 1 << n), dtype=torch.complex64, device="cuda")
        for k, st in enumerate(steps):
            B.tqs_materialize_step(c, k, S)
            torch.cuda.synchronize()
            want = kron_route.step_unitary(n, st)
            assert np.max(np.abs(S.cpu().numpy() - want)) <= 1e-6
    finally:
        B.tqs_circuit_destroy(c)


@pytest.mark.parametrize("n", [3, 7, 10])
def test_plain_form_random(n):
    ops = W.random_small(n, 8 * n, (56, n))
    check_state(simulate_plain_gpu(n, ops), fsv_route.simulate(n, ops))


# ----------------------------------------------------------- probabilities

@pytest.mark.parametrize("n", [1, 5, 14, 20])
def test_probabilities_reduction(n):
    g = W.rng(57, n)
    psi = (g.normal(size=1 << n) + 1j * g.normal(size=1 << n)).astype(np.complex64)
    d = torch.from_numpy(psi).cuda()
    p = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    s = torch.empty(1, dtype=torch.float64, device="cuda")
    B.tqs_probabilities(d, n, p, s)
    torch.cuda.synchronize()
    want = observables.probabilities(psi.astype(np.complex128))
    assert np.array_equal(p.cpu().numpy(), want)  # exact: squares of FP32 are exact in FP64
    assert abs(float(s.cpu()[0]) - want.sum()) <= 1e-12 * want.sum()
    # deterministic: same bits twice
    s2 = torch.empty(1, dtype=torch.float64, device="cuda")
    B.tqs_probabilities(d, n, None, s2)
    torch.cuda.synchronize()
    assert float(s2.cpu()[0]) == float(s.cpu()[0])


def test_abi_errors_on_gpu():
    c = B.circuit_from_ops(3, W.ghz_chain(3))
    try:
        out = torch.empty(9, dtype=torch.complex64, device="cuda")
        with pytest.raises(B.TqsError) as e:
            B.tqs_simulate(c, out[1:])  # 8-byte offset: misaligned
        assert e.value.name == "TQS_ERR_ARG"
        with pytest.raises(B.TqsError):
            B.tqs_materialize_step(c, 99, out)
    finally:
        B.tqs_circuit_destroy(c)


def test_program_upload_reused_and_refreshed():
    """tqs_simulate keeps a circuit's device program between calls: repeated
    calls (also from another stream, and alternating initial states) give the
    same results, and adding a gate refreshes the program."""
    n = 9
    ops = W.random_mixed(n, 8, (97, n))
    want = fsv_route.simulate(n, ops)
    rng = np.random.default_rng(98)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    v /= np.linalg.norm(v)
    init = torch.from_numpy(v.astype(np.complex64)).cuda()
    want_init = fsv_route.simulate(n, ops, v)
    c = B.circuit_from_ops(n, ops)
    try:
        other = torch.cuda.Stream()
        for stream, x, w in ((None, None, want), (None, None, want), (other, None, want),
                             (None, init, want_init), (None, None, want), (other, init, want_init)):
            out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
            if stream is not None:
                other.wait_stream(torch.cuda.current_stream())
            B.tqs_simulate(c, out, init=x, stream=stream)
            if stream is not None:
                torch.cuda.current_stream().wait_stream(other)
            torch.cuda.synchronize()
            assert np.max(np.abs(out.cpu().numpy().astype(np.complex128) - w)) <= AMP_TOL
        B.tqs_add_gate(c, "h", (3,))
        out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        B.tqs_simulate(c, out)
        torch.cuda.synchronize()
        want2 = fsv_route.simulate(n, list(ops) + [("h", (3,), ())])
        assert np.max(np.abs(out.cpu().numpy().astype(np.complex128) - want2)) <= AMP_TOL
    finally:
        B.tqs_circuit_destroy(c)

"""GPU parity of the full-state-vector backend (tqs_simulate_fsv; Appendix A,
eq. 12) against the FP64 oracle, through the C ABI.

* every gate kind, custom unitaries included, for n = 1 .. 20 compared
  element by element with the oracle (and, for n <= 16, with the fused
  kernel);
* n = 24, random layered circuit, element by element (the oracle handles
  2^24 amplitudes in seconds);
* the per-gate form (TQS_OPT_FSV_MAX_GATES = 1, one pass per gate) against
  the oracle and the grouped passes;
* n = 28: the GHZ closed form (two amplitudes 2^-1/2, the rest 0) and the
  QFT closed form on a basis state at sampled indices, plus the FP64 norm;
  these hold at any size.
"""
import numpy as np
import pytest

from oracle import fsv_route, gates
from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

AMP_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    yield
    torch.cuda.synchronize()


def rand_unitary(k, seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def basis(n, x=0):
    st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    st[x] = 1.0
    return st


def run_fsv(n, ops, x=0):
    c = B.circuit_from_ops(n, ops)
    try:
        st = basis(n, x)
        B.tqs_simulate_fsv(c, st)
        torch.cuda.synchronize()
        return st
    finally:
        B.tqs_circuit_destroy(c)


def mixed_circuit(n, seed):
    rng = np.random.default_rng(seed)
    ops = list(W.random_small(n, 5 * n, (15, n, seed)))
    for j in range(2):
        k = int(rng.integers(1, min(5, n) + 1))
        qs = tuple(int(q) for q in rng.permutation(n)[:k])
        ops.insert(int(rng.integers(0, len(ops) + 1)),
                   ("unitary", qs, gates.custom_params(rand_unitary(k, seed * 10 + j))))
    return ops


@pytest.mark.parametrize("n", [1, 3, 5, 6, 9, 12, 13, 16, 18, 20])
def test_fsv_matches_oracle(n):
    for seed in range(2):
        ops = mixed_circuit(n, 300 * n + seed)
        got = run_fsv(n, ops).cpu().numpy().astype(np.complex128)
        want = fsv_route.simulate(n, ops)
        assert np.max(np.abs(got - want)) <= AMP_TOL
        if n <= 16:
            c = B.circuit_from_ops(n, ops)
            try:
                out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
                B.tqs_simulate(c, out)
                torch.cuda.synchronize()
                assert np.max(np.abs(out.cpu().numpy() - got)) <= 2 * AMP_TOL
            finally:
                B.tqs_circuit_destroy(c)


def test_fsv_n24_random_layered():
    n = 24
    ops = W.random_layered(n, 4, (16, n))
    got = run_fsv(n, ops).cpu().numpy().astype(np.complex128)
    want = fsv_route.simulate(n, ops)
    assert np.max(np.abs(got - want)) <= AMP_TOL


@pytest.mark.parametrize("n,limit", [(9, 1), (18, 1), (18, 3)])
def test_fsv_per_gate_form(n, limit):
    ops = mixed_circuit(n, 77 * n)
    grouped = run_fsv(n, ops).cpu().numpy()
    B.tqs_set_option(B.OPT_FSV_MAX_GATES, 0, limit)
    try:
        c = B.circuit_from_ops(n, ops)
        try:
            passes = B.tqs_fsv_passes(c)[0]
            st = basis(n)
            B.tqs_simulate_fsv(c, st)
            torch.cuda.synchronize()
            got = st.cpu().numpy()
        finally:
            B.tqs_circuit_destroy(c)
    finally:
        B.tqs_set_option(B.OPT_FSV_MAX_GATES, 0, 0)
    if limit == 1 and n >= 4:
        assert passes == len(ops)
    want = fsv_route.simulate(n, ops)
    assert np.max(np.abs(got.astype(np.complex128) - want)) <= AMP_TOL
    assert np.max(np.abs(got - grouped)) <= 2 * AMP_TOL


def test_fsv_n28_closed_forms():
    n = 28
    st = run_fsv(n, W.ghz_chain(n))
    nz = torch.nonzero(st.abs() > 1e-6).flatten().cpu().tolist()
    assert nz == [0, (1 << n) - 1]
    assert abs(float(st[0].real) - 2 ** -0.5) < 1e-6 and abs(float(st[-1].real) - 2 ** -0.5) < 1e-6
    del st
    x = 0x5A3C1E7
    st = run_fsv(n, W.qft(n), x=x)
    idx = np.random.default_rng(17).integers(0, 1 << n, 4096)
    got = st[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
    want = np.exp(2j * np.pi * ((x * idx) % (1 << n)) / (1 << n)) / (2 ** (n / 2))
    assert np.max(np.abs(got - want)) * (2 ** (n / 2)) <= 1e-4  # relative to |amp| = 2^-n/2
    total = torch.empty(1, dtype=torch.float64, device="cuda")
    B.tqs_probabilities(st, n, None, total)
    assert abs(float(total.cpu()[0]) - 1.0) <= 1e-5


def test_fsv_edge_cases():
    # no gates: the state is unchanged; instructions are refused
    n = 14
    st = basis(n, 77)
    c = B.tqs_circuit_create(n)
    try:
        B.tqs_simulate_fsv(c, st)
        torch.cuda.synchronize()
        assert float(st[77].real) == 1.0 and int((st.abs() > 0).sum()) == 1
        B.tqs_add_gate(c, "measure", (3,))
        with pytest.raises(B.TqsError) as e:
            B.tqs_simulate_fsv(c, st)
        assert e.value.name == "TQS_ERR_UNSUPPORTED"
    finally:
        B.tqs_circuit_destroy(c)

"""Single circuits of 15 and 16 qubits on several CTAs (TQS_OPT_MULTI_CTAS):
the CTAs share the passes and meet at a grid barrier after each; states,
probabilities and the FP64 norm must be bitwise those of one CTA and of the
same circuit inside a batch, and match the FP64 oracle."""
import numpy as np
import pytest

from oracle import fsv_route, gates
from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    yield
    B.tqs_set_option(B.OPT_MULTI_CTAS, 0, 8)
    torch.cuda.synchronize()


def simulate(n, ops, ctas, init=None):
    B.tqs_set_option(B.OPT_MULTI_CTAS, 0, ctas)
    c = B.circuit_from_ops(n, ops)
    try:
        out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        pr = torch.empty(1 << n, dtype=torch.float64, device="cuda")
        nm = torch.empty(1, dtype=torch.float64, device="cuda")
        B.tqs_simulate(c, out, init=init, probs=pr, norm=nm)
        torch.cuda.synchronize()
        return out.cpu().numpy(), pr.cpu().numpy(), float(nm.cpu()[0])
    finally:
        B.tqs_circuit_destroy(c)


def circuits():
    yield 15, W.qft_on_basis(15, 12345)
    yield 16, W.ghz_chain(16)
    yield 16, W.random_layered(16, 6, (81, 16))
    yield 15, W.random_mixed(15, 20, (82, 15))


@pytest.mark.parametrize("ctas", [2, 3, 8, 64])
def test_multi_cta_bitwise_equals_one_cta(ctas):
    for n, ops in circuits():
        s1, p1, n1 = simulate(n, ops, 1)
        sk, pk, nk = simulate(n, ops, ctas)
        assert np.array_equal(s1.view(np.uint32), sk.view(np.uint32)), (n, ctas)
        assert np.array_equal(p1, pk) and n1 == nk


def test_multi_cta_matches_oracle_and_batch():
    circs = list(circuits())
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        count, total, offs = B.tqs_batch_info(b)
        st = torch.empty(total, dtype=torch.complex64, device="cuda")
        nm = torch.empty(count, dtype=torch.float64, device="cuda")
        B.tqs_batch_run(b, st, None, nm)
        torch.cuda.synchronize()
        st, nm = st.cpu().numpy(), nm.cpu().numpy()
    finally:
        B.tqs_batch_destroy(b)
    for i, (n, ops) in enumerate(circs):
        s, _, norm = simulate(n, ops, 8)
        assert np.array_equal(s.view(np.uint32), st[offs[i]:offs[i + 1]].view(np.uint32)), i
        assert norm == nm[i]
        want = fsv_route.simulate(n, ops)
        assert np.max(np.abs(s.astype(np.complex128) - want)) <= 1e-5


def test_multi_cta_with_initial_state_and_fallbacks():
    n = 16
    rng = np.random.default_rng(83)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    v /= np.linalg.norm(v)
    init = torch.from_numpy(v.astype(np.complex64)).cuda()
    ops = W.random_mixed(n, 8, (84, n))
    a = simulate(n, ops, 1, init=init)
    b = simulate(n, ops, 8, init=init)
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32)) and a[2] == b[2]
    want = fsv_route.simulate(n, ops, v)
    assert np.max(np.abs(b[0].astype(np.complex128) - want)) <= 1e-5
    # custom unitaries take one CTA: same results for every setting
    u = np.linalg.qr(rng.normal(size=(8, 8)) + 1j * rng.normal(size=(8, 8)))[0]
    ops2 = ops + [("unitary", (0, 7, 15), gates.custom_params(u))]
    a = simulate(n, ops2, 1)
    b = simulate(n, ops2, 8)
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32)) and a[2] == b[2]

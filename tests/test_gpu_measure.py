"""GPU parity of the measure / reset instructions (Sec. 5.2 operation
interface) in the fused kernel, against the FP64 oracle, through the C ABI.

The uniforms are chosen (on the oracle side) at least 1e-4 away from every
decision boundary S_0 / T, so the FP32 state decides like the FP64 one: the
outcomes must be equal, and the states within 1e-5.  The three team kinds
are covered (warp n <= 11, CTA n <= 14, global n = 15, 16), as are batches
(tqs_batch_run_measured equals tqs_simulate_measured bit for bit).
"""
import numpy as np
import pytest

from measure_cases import safe_uniforms, with_instructions
from oracle import collapse
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


def run_measured(n, ops, u):
    c = B.circuit_from_ops(n, ops)
    try:
        out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        norm = torch.empty(1, dtype=torch.float64, device="cuda")
        k = max(1, len(u))
        du = torch.from_numpy(np.asarray(u, dtype=np.float64).reshape(-1)).cuda() if len(u) else None
        oc = torch.full((k,), -7, dtype=torch.int32, device="cuda")
        B.tqs_simulate_measured(c, out, u=du, outcomes=oc, norm=norm)
        torch.cuda.synchronize()
        return out.cpu().numpy(), oc.cpu().numpy()[:len(u)].tolist(), float(norm.cpu()[0])
    finally:
        B.tqs_circuit_destroy(c)


@pytest.mark.parametrize("n", [1, 2, 4, 7, 11, 12, 14, 15, 16])
def test_measured_circuits_match_oracle(n):
    for seed in range(2 if n >= 15 else 3):
        ops = with_instructions(n, 1000 * n + seed)
        u = safe_uniforms(n, ops, 50 + seed)
        got, outs, norm = run_measured(n, ops, u)
        want, want_outs = collapse.simulate_measured(n, ops, u)
        assert outs == want_outs
        assert np.max(np.abs(got.astype(np.complex128) - want)) <= AMP_TOL
        assert abs(norm - 1.0) <= (1e-6 if n <= 14 else 3e-6)


def test_bell_and_ghz_closed_forms():
    for uu, b in ((0.3, 0), (0.7, 1)):
        st, outs, _ = run_measured(2, W.bell() + [("measure", (0,), ()), ("measure", (1,), ())],
                                   [uu, 0.5])
        assert outs == [b, b]
        assert abs(st[3 * b] - 1.0) < 1e-6 and np.sum(np.abs(st) > 1e-6) == 1
    n = 11
    ops = W.ghz_chain(n) + [("measure", (q,), ()) for q in range(n)]
    st, outs, _ = run_measured(n, ops, [0.8] + [0.01] * (n - 1))
    assert outs == [1] * n and abs(st[(1 << n) - 1] - 1.0) < 1e-6


def test_reset_and_leading_instruction():
    # a measurement before any gate reads |0>; X then reset returns to |0>
    st, outs, _ = run_measured(3, [("measure", (1,), ()), ("x", (2,), ()), ("reset", (2,), ()),
                                   ("h", (0,), ()), ("reset", (0,), ())], [0.9, 0.4, 0.6])
    assert outs[:2] == [0, 1]
    assert abs(st[0] - 1.0) < 1e-6 and np.sum(np.abs(st) > 1e-6) == 1


def test_missing_uniforms_is_an_error():
    c = B.circuit_from_ops(2, [("h", (0,), ()), ("measure", (0,), ())])
    try:
        out = torch.empty(4, dtype=torch.complex64, device="cuda")
        with pytest.raises(B.TqsError) as e:
            B.tqs_simulate_measured(c, out)
        assert e.value.name == "TQS_ERR_ARG"
        with pytest.raises(B.TqsError) as e:
            B.tqs_simulate(c, out)
        assert e.value.name == "TQS_ERR_UNSUPPORTED"
    finally:
        B.tqs_circuit_destroy(c)


@pytest.fixture(params=[1, 2], ids=["warp", "pair"])
def team_warps(request):
    """Run a test with 1 or 2 warps per circuit of the warp class."""
    for q in range(4, 12):
        B.tqs_set_option(B.OPT_TEAM_WARPS, q, request.param)
    yield request.param
    for q in range(4, 12):
        B.tqs_set_option(B.OPT_TEAM_WARPS, q, 1)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_measured_equals_single(use_graph, team_warps):
    circs = []
    for i in range(48):
        n = [3, 6, 9, 11, 12, 13, 15][i % 7]
        ops = with_instructions(n, 5000 + i) if i % 3 else W.random_mixed(n, 6, (31, i))
        circs.append((n, ops))
    us = [safe_uniforms(n, ops, 900 + i) for i, (n, ops) in enumerate(circs)]
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        count, total, offs = B.tqs_batch_info(b)
        ioff = B.tqs_batch_instructions(b)
        assert ioff[-1] == sum(len(u) for u in us)
        u_all = np.concatenate(us)
        st = torch.empty(total, dtype=torch.complex64, device="cuda")
        nm = torch.empty(count, dtype=torch.float64, device="cuda")
        oc = torch.full((int(ioff[-1]),), -7, dtype=torch.int32, device="cuda")
        du = torch.from_numpy(u_all).cuda()
        for _ in range(2):  # the second run replays the graph
            B.tqs_batch_run_measured(b, st, du, outcomes=oc, norms=nm, use_graph=use_graph)
        torch.cuda.synchronize()
        states, outs = st.cpu().numpy(), oc.cpu().numpy()
        for i, (n, ops) in enumerate(circs):
            s1, o1, _ = run_measured(n, ops, us[i])
            assert np.array_equal(states[offs[i]:offs[i + 1]].view(np.uint32), s1.view(np.uint32)), i
            assert outs[ioff[i]:ioff[i + 1]].tolist() == o1, i
            want, want_outs = collapse.simulate_measured(n, ops, us[i])
            assert o1 == want_outs
            assert np.max(np.abs(s1.astype(np.complex128) - want)) <= AMP_TOL
    finally:
        B.tqs_batch_destroy(b)

"""GPU parity of the batched persistent form (one CUDA-graph launch of the
fused step kernels over many circuits of uneven size and depth).

* every circuit of a reduced batch against the oracle (1e-5 on amplitudes,
  1e-6 on the probability sum);
* the full 4096-circuit batch: sampled circuits against the oracle, and the
  norm property on every circuit;
* a circuit's result is bitwise the same alone (tqs_simulate) and in the mix;
* graph replays and the host-buffer entry point give identical bits.
"""
import numpy as np
import pytest

from oracle import fsv_route
from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

AMP_TOL = 1e-5
NORM_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()


def run_batch(circs, use_graph=True, with_probs=True, runs=1):
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        count, total, offs = B.tqs_batch_info(b)
        st = torch.empty(total, dtype=torch.complex64, device="cuda")
        pr = torch.empty(total, dtype=torch.float64, device="cuda") if with_probs else None
        nm = torch.empty(count, dtype=torch.float64, device="cuda")
        outs = []
        for _ in range(runs):
            st.fill_(float("nan"))
            B.tqs_batch_run(b, st, pr, nm, use_graph=use_graph)
            torch.cuda.synchronize()
            outs.append((st.cpu().numpy().copy(), None if pr is None else pr.cpu().numpy().copy(),
                         nm.cpu().numpy().copy()))
        return offs, outs
    finally:
        B.tqs_batch_destroy(b)


def mixed_workload(count, seed_tag):
    """Config-3 style circuits plus paper circuits and 15/16-qubit ones."""
    circs = W.batch_circuits(count, seed_tag)
    circs += [(n, ops) for (n, ops) in
              [(11, W.qft_on_basis(11, 77)), (13, W.ghz_chain(13)), (15, W.random_mixed(15, 6, (60, 1))),
               (16, W.qft(16)), (2, W.bell()), (1, [("h", (0,), ())])]]
    return circs


def test_batch_every_circuit_matches_oracle():
    circs = mixed_workload(160, 61)
    offs, [(st, pr, nm)] = run_batch(circs)
    for i, (n, ops) in enumerate(circs):
        got = st[offs[i]:offs[i + 1]].astype(np.complex128)
        want = fsv_route.simulate(n, ops)
        assert np.max(np.abs(got - want)) <= AMP_TOL, (i, n)
        assert abs(nm[i] - 1.0) <= NORM_TOL
        exact = got.real ** 2 + got.imag ** 2
        assert np.all(np.abs(pr[offs[i]:offs[i + 1]] - exact) <= 2.0 ** -22 * exact + 1e-44)


def test_full_batch_4096_sampled():
    """The full batched workload (4096 circuits, n = 4..14, depth 5..40)."""
    circs = W.batch_circuits(4096, 3)
    offs, [(st, pr, nm)] = run_batch(circs)
    assert np.all(np.abs(nm - 1.0) <= NORM_TOL)
    ns = np.array([n for n, _ in circs])
    sample = list(np.flatnonzero(ns == 14)[:3]) + list(np.flatnonzero(ns == 13)[:3])
    sample += list(W.rng(62).choice(len(circs), size=24, replace=False))
    for i in sample:
        n, ops = circs[i]
        got = st[offs[i]:offs[i + 1]].astype(np.complex128)
        assert np.max(np.abs(got - fsv_route.simulate(n, ops))) <= AMP_TOL, (i, n)


def test_alone_equals_in_the_mix_bitwise():
    circs = mixed_workload(48, 63)
    offs, [(st, pr, nm)] = run_batch(circs)
    for i in range(0, len(circs), 5):
        n, ops = circs[i]
        c = B.circuit_from_ops(n, ops)
        try:
            out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
            norm = torch.empty(1, dtype=torch.float64, device="cuda")
            B.tqs_simulate(c, out, norm=norm)
            torch.cuda.synchronize()
        finally:
            B.tqs_circuit_destroy(c)
        assert np.array_equal(out.cpu().numpy().view(np.uint32),
                              st[offs[i]:offs[i + 1]].view(np.uint32)), (i, n)
        assert float(norm.cpu()[0]) == nm[i]


def test_graph_replay_and_plain_launch_identical():
    circs = mixed_workload(64, 64)
    _, outs = run_batch(circs, use_graph=True, runs=3)
    _, [plain] = run_batch(circs, use_graph=False)
    for o in outs[1:] + [plain]:
        assert np.array_equal(o[0].view(np.uint32), outs[0][0].view(np.uint32))
        assert np.array_equal(o[2], outs[0][2])


def test_host_buffer_entry_point():
    circs = mixed_workload(40, 65)
    offs, [(st, pr, nm)] = run_batch(circs)
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        count, total, _ = B.tqs_batch_info(b)
        hs = np.empty(total, dtype=np.complex64)
        hp = np.empty(total, dtype=np.float64)
        hn = np.empty(count, dtype=np.float64)
        B.tqs_batch_run_host(b, hs, hp, hn)
    finally:
        B.tqs_batch_destroy(b)
    assert np.array_equal(hs.view(np.uint32), st.view(np.uint32))
    assert np.array_equal(hp, pr) and np.array_equal(hn, nm)


@pytest.mark.parametrize("mode", ["pinned", "mixed", "copies"])
def test_host_buffer_entry_point_pinned(mode):
    """Page-locked host buffers are written by the kernel directly (no device
    copy); results equal the device run bit for bit.  In "mixed", only the
    probabilities are page-locked (states and norms take the copy path); in
    "copies", TQS_OPT_HOST_WRITES = 0 stages every output in device memory."""
    B.tqs_set_option(B.OPT_HOST_WRITES, 0, 0 if mode == "copies" else 1)
    try:
        _host_buffers(mode)
    finally:
        B.tqs_set_option(B.OPT_HOST_WRITES, 0, 1)


def _host_buffers(mode):
    circs = mixed_workload(40, 66)
    offs, [(st, pr, nm)] = run_batch(circs)
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        count, total, _ = B.tqs_batch_info(b)
        pin = (lambda t: t.pin_memory()) if mode != "mixed" else (lambda t: t)
        hs = pin(torch.empty(total, dtype=torch.complex64))
        hp = torch.empty(total, dtype=torch.float64).pin_memory()
        hn = pin(torch.empty(count, dtype=torch.float64))
        for _ in range(2):
            B.tqs_batch_run_host(b, hs, hp, hn)
    finally:
        B.tqs_batch_destroy(b)
    assert np.array_equal(hs.numpy().view(np.uint32), st.view(np.uint32))
    assert np.array_equal(hp.numpy(), pr) and np.array_equal(hn.numpy(), nm)

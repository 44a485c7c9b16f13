"""Launch-shape options the autotuner sets do not change results:
* TQS_OPT_CTA_THREADS (256 / 512 threads per one-CTA team): states and
  probabilities bitwise equal, states within 1e-5 of the oracle, norms within
  1e-6 of 1 and within 2.5e-7 of each other (a thread sums its 16-value blocks
  in FP32 before the FP64 reduction, and which values share a block depends on
  the thread count: at most 4 roundings of 2^-24 relative on sums <= 1);
* TQS_OPT_FSV_TILE_Q (tile bits 10..13 or automatic): every choice within
  1e-5 of the oracle (eq. 12 per gate);
* TQS_OPT_CHAIN_GROUP (raster band 1..64): the circuit unitary bitwise equal.
"""
import numpy as np
import pytest

from oracle import fsv_route
from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()


def run_batch(circs):
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        count, total, offs = B.tqs_batch_info(b)
        st = torch.empty(total, dtype=torch.complex64, device="cuda")
        pr = torch.empty(total, dtype=torch.float64, device="cuda")
        nm = torch.empty(count, dtype=torch.float64, device="cuda")
        B.tqs_batch_run(b, st, pr, nm, use_graph=False)
        torch.cuda.synchronize()
        return offs, st.cpu().numpy(), pr.cpu().numpy(), nm.cpu().numpy()
    finally:
        B.tqs_batch_destroy(b)


def test_cta_threads_same_results():
    circs = W.batch_circuits_fixed_n(24, 12, seed_tag=96) + W.batch_circuits_fixed_n(8, 14, seed_tag=97)
    res = {}
    try:
        for t in (512, 256):
            B.tqs_set_option(B.OPT_CTA_THREADS, 0, t)
            res[t] = run_batch(circs)
    finally:
        B.tqs_set_option(B.OPT_CTA_THREADS, 0, 512)
    (offs, s5, p5, n5), (_, s2, p2, n2) = res[512], res[256]
    assert np.array_equal(s5.view(np.uint32), s2.view(np.uint32))
    assert np.array_equal(p5.view(np.uint64), p2.view(np.uint64))
    assert np.max(np.abs(n5 - n2)) <= 2.5e-7
    assert np.max(np.abs(n5 - 1.0)) <= 1e-6 and np.max(np.abs(n2 - 1.0)) <= 1e-6
    for i in (0, 5, 24, 31):
        n, ops = circs[i]
        got = s2[offs[i]:offs[i + 1]].astype(np.complex128)
        assert np.max(np.abs(got - fsv_route.simulate(n, ops))) <= 1e-5


def test_fsv_tile_bits_all_match_oracle():
    n = 18
    ops = W.random_layered(n, 6, (98, n))
    want = fsv_route.simulate(n, ops)
    c = B.circuit_from_ops(n, ops)
    passes = {}
    try:
        for t in (0, 10, 11, 12, 13):
            B.tqs_set_option(B.OPT_FSV_TILE_Q, 0, t)
            st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
            st[0] = 1.0
            B.tqs_simulate_fsv(c, st)
            torch.cuda.synchronize()
            passes[t] = B.tqs_fsv_passes(c)
            assert np.max(np.abs(st.cpu().numpy().astype(np.complex128) - want)) <= 1e-5, t
    finally:
        B.tqs_set_option(B.OPT_FSV_TILE_Q, 0, 0)
        B.tqs_circuit_destroy(c)
    assert passes[10][1] == 10 and passes[13][1] == 13 and passes[0][1] == 12
    assert passes[10][0] >= passes[13][0]


@pytest.mark.parametrize("prec", [B.PREC_TC_BF16X3, B.PREC_TC_TF32X3])
def test_chain_group_bitwise(prec):
    n = 10
    ops = W.random_layered(n, 4, (99, n))
    c = B.circuit_from_ops(n, ops)
    out = {}
    try:
        for g in (16, 1, 3, 64):
            B.tqs_set_option(B.OPT_CHAIN_GROUP, 0, g)
            U = torch.empty((1 << n, 1 << n), dtype=torch.complex64, device="cuda")
            B.tqs_circuit_unitary(c, prec, U)
            torch.cuda.synchronize()
            out[g] = U.cpu().numpy()
    finally:
        B.tqs_set_option(B.OPT_CHAIN_GROUP, 0, 16)
        B.tqs_circuit_destroy(c)
    for g in (1, 3, 64):
        assert np.array_equal(out[g].view(np.uint32), out[16].view(np.uint32)), g


@pytest.mark.parametrize("prec", [B.PREC_TC_BF16X3, B.PREC_TC_TF32X3])
@pytest.mark.parametrize("n", [8, 11])
def test_chain_pair_bitwise(prec, n):
    """TQS_OPT_CHAIN_PAIR (two-CTA clusters sharing B tiles by multicast): the
    circuit unitary is bitwise that of one CTA per tile, and a column block of
    an odd number of tiles (no pairs) matches the whole unitary's columns."""
    ops = W.random_layered(n, 4, (100, n))
    c = B.circuit_from_ops(n, ops)
    out = {}
    try:
        for pair in (0, 1):
            B.tqs_set_option(B.OPT_CHAIN_PAIR, 0, pair)
            U = torch.empty((1 << n, 1 << n), dtype=torch.complex64, device="cuda")
            B.tqs_circuit_unitary(c, prec, U)
            torch.cuda.synchronize()
            out[pair] = U.cpu().numpy()
        # an odd number of 128-column tiles: the pair option falls back to single CTAs
        w = 384 if n >= 10 else 128
        blk = torch.empty((1 << n, w), dtype=torch.complex64, device="cuda")
        B.tqs_circuit_unitary_cols(c, prec, 128, w, blk)
        torch.cuda.synchronize()
        cols = blk.cpu().numpy()
    finally:
        B.tqs_set_option(B.OPT_CHAIN_PAIR, 0, 0)
        B.tqs_circuit_destroy(c)
    assert np.array_equal(out[1].view(np.uint32), out[0].view(np.uint32))
    assert np.array_equal(cols.view(np.uint32), out[1][:, 128:128 + w].view(np.uint32))
    want = fsv_route.unitary_columns(n, ops, [0, 200, (1 << n) - 1])
    assert np.max(np.abs(out[1][:, [0, 200, (1 << n) - 1]] - want)) <= 1e-4

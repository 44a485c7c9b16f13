"""GPU parity of the column-block chain (tqs_circuit_unitary_cols): a block of
columns of the circuit unitary by the same chain (Algorithm 1), the unit of
the column-sharded chain.

* blocks computed by separate calls and put side by side are bitwise the
  whole tqs_circuit_unitary result in each precision, compact (ldu = ncols)
  or written in place into a full matrix (ldu = 2^n);
* the blocks match the FP64 oracle's columns (eq. 12 applied to |j>) within
  the chain's tolerances (1e-5 FP32 SIMT, 1e-4 tensor-core splits);
* edge cases: zero / one step, arbitrary blocks below n = 7 (FP32 SIMT),
  misaligned or out-of-range blocks rejected.
"""
import numpy as np
import pytest

from oracle import fsv_route
from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import shard
from paper_2305_14398_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {B.PREC_FP32_SIMT: 1e-5, B.PREC_TC_BF16X3: 1e-4, B.PREC_TC_TF32X3: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()


def full_and_blocks(n, ops, prec, blocks, in_place=False):
    N = 1 << n
    c = B.circuit_from_ops(n, ops)
    try:
        full = torch.empty((N, N), dtype=torch.complex64, device="cuda")
        B.tqs_circuit_unitary(c, prec, full)
        if in_place:
            U = torch.full((N, N), float("nan"), dtype=torch.complex64, device="cuda")
            for col0, ncols in blocks:
                B.tqs_circuit_unitary_cols(c, prec, col0, ncols, U[:, col0:], ldu=N)
            parts = [U]
        else:
            parts = []
            for col0, ncols in blocks:
                blk = torch.full((N, ncols), float("nan"), dtype=torch.complex64, device="cuda")
                B.tqs_circuit_unitary_cols(c, prec, col0, ncols, blk)
                parts.append(blk)
        torch.cuda.synchronize()
        return full.cpu().numpy(), np.concatenate([p.cpu().numpy() for p in parts], axis=1)
    finally:
        B.tqs_circuit_destroy(c)


@pytest.mark.parametrize("prec", [B.PREC_FP32_SIMT, B.PREC_TC_BF16X3, B.PREC_TC_TF32X3])
def test_two_half_blocks_equal_full_and_oracle(prec):
    n = 12
    ops = W.random_layered(n, 20, (2, n))
    blocks = shard.column_blocks(n, 2)
    full, cat = full_and_blocks(n, ops, prec, blocks)
    assert np.array_equal(cat.view(np.uint32), full.view(np.uint32))
    cols = [0, 1, 777, 2047, 2048, 3001, 4095]
    want = fsv_route.unitary_columns(n, ops, cols)
    assert np.max(np.abs(cat[:, cols] - want)) <= TOL[prec]


@pytest.mark.parametrize("prec", [B.PREC_FP32_SIMT, B.PREC_TC_BF16X3])
def test_uneven_blocks_in_place(prec):
    """Three ranks' blocks of a 10-qubit chain (8 tiles: 2 + 3 + 3) written in
    place into one full matrix."""
    n = 10
    ops = W.random_layered(n, 6, (90, n))
    blocks = shard.column_blocks(n, 3)
    assert [b[1] for b in blocks] == [256, 384, 384]
    full, cat = full_and_blocks(n, ops, prec, blocks, in_place=True)
    assert np.array_equal(cat.view(np.uint32), full.view(np.uint32))
    want = fsv_route.unitary_columns(n, ops, [5, 300, 1000])
    assert np.max(np.abs(cat[:, [5, 300, 1000]] - want)) <= TOL[prec]


def test_simt_small_arbitrary_blocks():
    """Below n = 7 any block is allowed (FP32 SIMT)."""
    n = 5
    ops = W.random_small(n, 30, (91, n))
    full, cat = full_and_blocks(n, ops, B.PREC_FP32_SIMT, [(0, 3), (3, 7), (10, 22)])
    assert np.array_equal(cat.view(np.uint32), full.view(np.uint32))
    want = fsv_route.unitary_columns(n, ops, list(range(32)))
    assert np.max(np.abs(cat - want)) <= TOL[B.PREC_FP32_SIMT]


def test_zero_and_one_step_blocks():
    n = 8
    for ops in ([], [("h", (q,), ()) for q in range(n)]):
        full, cat = full_and_blocks(n, ops, B.PREC_TC_BF16X3, [(128, 128), (0, 128)])
        assert np.array_equal(cat[:, :128].view(np.uint32), full[:, 128:].view(np.uint32))
        assert np.array_equal(cat[:, 128:].view(np.uint32), full[:, :128].view(np.uint32))


def test_bad_blocks_rejected():
    n = 8
    c = B.circuit_from_ops(n, W.random_layered(n, 2, (92, n)))
    try:
        blk = torch.empty((1 << n, 256), dtype=torch.complex64, device="cuda")
        for col0, ncols, ldu in [(64, 128, 128), (0, 100, 128), (128, 256, 256), (0, 128, 64),
                                 (-128, 128, 128), (0, 0, 128)]:
            with pytest.raises(B.TqsError) as e:
                B.tqs_circuit_unitary_cols(c, B.PREC_TC_BF16X3, col0, ncols, blk, ldu=ldu)
            assert e.value.name == "TQS_ERR_ARG", (col0, ncols, ldu)
    finally:
        B.tqs_circuit_destroy(c)

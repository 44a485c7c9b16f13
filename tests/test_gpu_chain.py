"""GPU parity of the circuit-unitary chain (Algorithm 1) against the FP64 oracle.

Tolerances: max |delta entry| <= 1e-5 for the FP32 SIMT chain and <= 1e-4 for the
tensor-core split chains (BF16x3 and TF32x3).  At 2^12..2^14 the oracle computes sampled columns
U[:, j] = circuit applied to e_j (eq. 12), which also pins the whole chain order.
"""
import math

import numpy as np
import pytest

from oracle import fsv_route, kron_route
from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TC_TOL = 1e-4
SIMT_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()


def unitary_gpu(n, ops, prec):
    c = B.circuit_from_ops(n, ops)
    try:
        U = torch.empty((1 << n, 1 << n), dtype=torch.complex64, device="cuda")
        B.tqs_circuit_unitary(c, prec, U)
        torch.cuda.synchronize()
        return U
    finally:
        B.tqs_circuit_destroy(c)


def sampled_cols(n, seed):
    g = W.rng(80, n, seed)
    return sorted(set([0, (1 << n) - 1] + [int(v) for v in g.integers(0, 1 << n, size=14)]))


PRECS = [(B.PREC_FP32_SIMT, SIMT_TOL), (B.PREC_TC_BF16X3, TC_TOL), (B.PREC_TC_TF32X3, TC_TOL)]


@pytest.mark.parametrize("prec,tol", PRECS)
def test_chain_small_full_matrix(prec, tol):
    """n = 7 random layered circuit (8 steps): every entry against Algorithm 1
    in FP64."""
    n = 7
    ops = W.random_layered(n, 4, (81, 1))
    want = kron_route.circuit_unitary(n, ops)
    got = unitary_gpu(n, ops, prec).cpu().numpy()
    assert np.max(np.abs(got - want)) <= tol


@pytest.mark.parametrize("n", [1, 3, 5])
def test_chain_simt_tiny(n):
    ops = W.random_small(n, 6 * n, (82, n))
    want = kron_route.circuit_unitary(n, ops)
    got = unitary_gpu(n, ops, B.PREC_FP32_SIMT).cpu().numpy()
    assert np.max(np.abs(got - want)) <= SIMT_TOL


@pytest.mark.parametrize("prec,tol", PRECS)
def test_chain_qft_is_dft(prec, tol):
    """The QFT circuit unitary is the DFT matrix (closed form)."""
    n = 8
    k = np.arange(1 << n)
    dft = np.exp(2j * np.pi * np.outer(k, k) / (1 << n)) / math.sqrt(1 << n)
    got = unitary_gpu(n, W.qft(n), prec).cpu().numpy()
    assert np.max(np.abs(got - dft)) <= tol


@pytest.mark.parametrize("prec,tol", PRECS)
def test_chain_config_n12(prec, tol):
    """Random layered n = 12: 20 layers of U3 on every qubit + CNOTs on 6 seeded
    pairs (40 steps); sampled columns against the oracle."""
    n = 12
    ops = W.random_layered(n, 20, (2, n))
    U = unitary_gpu(n, ops, prec)
    cols = sampled_cols(n, 1)
    got = U[:, cols].cpu().numpy()
    want = fsv_route.unitary_columns(n, ops, cols)
    assert np.max(np.abs(got - want)) <= tol


@pytest.mark.parametrize("n", [13, 14])
def test_chain_tc_large_sampled(n):
    """n = 13, 14 (8192^2 and 16384^2): sampled columns against the oracle and
    orthonormality of the sampled columns (a property at any size)."""
    ops = W.random_layered(n, 20, (2, n))
    U = unitary_gpu(n, ops, B.PREC_TC_BF16X3)
    cols = sampled_cols(n, 2)
    got = U[:, cols].cpu().numpy().astype(np.complex128)
    del U
    torch.cuda.empty_cache()
    want = fsv_route.unitary_columns(n, ops, cols)
    assert np.max(np.abs(got - want)) <= TC_TOL
    # Orthonormality of the sampled columns.  The tensor cores' FP32
    # accumulation truncates, which shrinks a sum over K by a relative amount
    # that grows with the number of accumulation steps (measured ~2e-5 per
    # product at K = 16384 in one chunk: column norms^2 1 - 1.7e-3 after 39
    # products).  The GEMMs restart their accumulators every 512 of K and add
    # the chunks with rounding to nearest, so the shrink per product is ~32x
    # smaller at n = 14 (BF16x3, the default chunk).
    gram = got.conj().T @ got
    assert np.max(np.abs(gram - np.eye(len(cols)))) <= 1e-4


@pytest.mark.parametrize("prec", [B.PREC_TC_BF16X3, B.PREC_TC_TF32X3])
def test_chain_kchunk_bounds_truncation_shrink(prec):
    """n = 12 random layered chain (39 products of K = 4096): with all of K in
    one accumulation chunk every column's norm^2 drops below 1 by the
    truncation shrink; with the default chunks (32 MMA accumulation steps:
    K = 512 in BF16x3, 256 in TF32x3) the deviation is smaller by more than 4x
    and within 1e-4, and the sampled columns stay within the tolerance of the
    oracle either way."""
    n = 12
    ops = W.random_layered(n, 20, (2, n))
    cols = sampled_cols(n, 3)
    want = fsv_route.unitary_columns(n, ops, cols)
    dev = {}
    one_chunk = 1 << 20
    try:
        for kc in (one_chunk, 0):
            B.tqs_set_option(B.OPT_CHAIN_KCHUNK, 0, kc)
            U = unitary_gpu(n, ops, prec)
            cn = (U.real.double() ** 2 + U.imag.double() ** 2).sum(0).cpu().numpy()
            dev[kc] = float(np.max(np.abs(cn - 1.0)))
            assert np.max(np.abs(U[:, cols].cpu().numpy() - want)) <= TC_TOL, kc
            del U
    finally:
        B.tqs_set_option(B.OPT_CHAIN_KCHUNK, 0, 0)
    assert dev[0] <= 1e-4, dev
    assert dev[0] * 4 < dev[one_chunk], dev


def test_chain_edge_cases():
    n = 7
    # no steps: the identity; one step: S_1 itself
    U = unitary_gpu(n, [], B.PREC_TC_BF16X3).cpu().numpy()
    assert np.array_equal(U, np.eye(1 << n, dtype=np.complex64))
    ops = [("h", (q,), ()) for q in range(n)]
    U = unitary_gpu(n, ops, B.PREC_TC_BF16X3).cpu().numpy()
    assert np.max(np.abs(U - kron_route.circuit_unitary(n, ops))) <= 1e-6
    # the tensor-core form needs n >= 7
    with pytest.raises(B.TqsError) as e:
        unitary_gpu(6, W.ghz_chain(6), B.PREC_TC_BF16X3)
    assert e.value.name == "TQS_ERR_ARG"
    with pytest.raises(B.TqsError) as e:
        unitary_gpu(6, W.ghz_chain(6), B.PREC_TC_TF32X3)
    assert e.value.name == "TQS_ERR_ARG"
    with pytest.raises(B.TqsError) as e:
        unitary_gpu(8, W.ghz_chain(8), 7)
    assert e.value.name == "TQS_ERR_ARG"


def test_chain_split_precisions_error_budget():
    """Both split precisions on the n = 12 chain, same columns.  TF32 hi+lo keeps
    ~22 bits per operand against ~16 for BF16 hi+lo, yet its error is the larger
    one (measured 2.1e-5 vs 1.2e-5): the FP32 accumulation in the tensor cores
    rounds toward zero once per MMA, and TF32 MMAs take K = 8 instead of 16, so
    the accumulator rounds twice as often.  Both stay within 1e-4."""
    n = 12
    ops = W.random_layered(n, 20, (2, n))
    cols = sampled_cols(n, 3)
    want = fsv_route.unitary_columns(n, ops, cols)
    err = {}
    for prec in (B.PREC_TC_BF16X3, B.PREC_TC_TF32X3):
        got = unitary_gpu(n, ops, prec)[:, cols].cpu().numpy()
        err[prec] = np.max(np.abs(got - want))
    assert err[B.PREC_TC_BF16X3] <= TC_TOL and err[B.PREC_TC_TF32X3] <= TC_TOL
    assert err[B.PREC_TC_BF16X3] > 1e-7 and err[B.PREC_TC_TF32X3] > 1e-7  # truly split products

"""GPU parity of custom k-qubit unitaries (Sec. 5.2: registered with the
operation data provider, applied to qubits) in every form, against the FP64
oracle, through the C ABI: the fused kernel (wide passes, all team kinds),
the plain materialised form, the circuit-unitary chain (FP32 SIMT and both
tensor-core splits) and batches built from circuit handles.
"""
import numpy as np
import pytest

from oracle import fsv_route, gates, kron_route
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


def with_customs(n, seed, count=3):
    rng = np.random.default_rng(seed)
    ops = list(W.random_mixed(n, 3, (13, n, seed)))
    for j in range(count):
        k = int(rng.integers(1, min(5, n) + 1)) if j else min(5, n)
        qs = tuple(int(q) for q in rng.permutation(n)[:k])
        ops.append(("unitary", qs, gates.custom_params(rand_unitary(k, 1000 * seed + j))))
        ops += W.random_mixed(n, 2, (14, n, seed, j))
        if j == 0 and n >= 2:
            ops.append(("swap", (0, n - 1), ()))
    return ops


def fused(n, ops):
    c = B.circuit_from_ops(n, ops)
    try:
        out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        norm = torch.empty(1, dtype=torch.float64, device="cuda")
        B.tqs_simulate(c, out, norm=norm)
        torch.cuda.synchronize()
        return out.cpu().numpy(), float(norm.cpu()[0])
    finally:
        B.tqs_circuit_destroy(c)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11, 12, 14, 15, 16])
def test_fused_with_customs(n):
    for seed in range(2):
        ops = with_customs(n, 100 * n + seed)
        got, norm = fused(n, ops)
        want = fsv_route.simulate(n, ops)
        assert np.max(np.abs(got.astype(np.complex128) - want)) <= AMP_TOL
        assert abs(norm - 1.0) <= (1e-6 if n <= 14 else 3e-6)


def test_fused_toffoli_on_every_basis_state():
    tof = np.eye(8)
    tof[[3, 7]] = tof[[7, 3]]
    n, qs = 6, (4, 0, 2)
    for x in range(1 << n):
        got, _ = fused(n, W.basis_prep(n, x) + [("unitary", qs, gates.custom_params(tof))])
        want = x ^ (1 << 2) if (x >> 4) & 1 and x & 1 else x
        assert abs(got[want] - 1.0) < 1e-6 and np.sum(np.abs(got) > 1e-6) == 1


@pytest.mark.parametrize("n", [3, 6, 9])
def test_plain_with_customs(n):
    ops = with_customs(n, 7 * n)
    c = B.circuit_from_ops(n, ops)
    try:
        out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        B.tqs_simulate_plain(c, out)
        torch.cuda.synchronize()
        want = kron_route.simulate(n, ops)
        assert np.max(np.abs(out.cpu().numpy().astype(np.complex128) - want)) <= AMP_TOL
    finally:
        B.tqs_circuit_destroy(c)


@pytest.mark.parametrize("prec,tol", [(B.PREC_FP32_SIMT, 1e-5), (B.PREC_TC_BF16X3, 1e-4),
                                      (B.PREC_TC_TF32X3, 1e-4)])
def test_circuit_unitary_with_customs(prec, tol):
    n = 8
    ops = with_customs(n, 31)
    c = B.circuit_from_ops(n, ops)
    try:
        U = torch.empty((1 << n, 1 << n), dtype=torch.complex64, device="cuda")
        B.tqs_circuit_unitary(c, prec, U)
        torch.cuda.synchronize()
        want = kron_route.circuit_unitary(n, ops)
        assert np.max(np.abs(U.cpu().numpy().astype(np.complex128) - want)) <= tol
    finally:
        B.tqs_circuit_destroy(c)


@pytest.mark.parametrize("tw", [1, 2])
def test_batch_from_handles_with_customs(tw):
    for q in range(4, 12):
        B.tqs_set_option(B.OPT_TEAM_WARPS, q, tw)
    try:
        _batch_from_handles_with_customs()
    finally:
        for q in range(4, 12):
            B.tqs_set_option(B.OPT_TEAM_WARPS, q, 1)


def _batch_from_handles_with_customs():
    circs = [(n, with_customs(n, 500 + i)) for i, n in enumerate([2, 5, 7, 9, 11, 12, 13, 15, 4, 10])]
    hs = [B.circuit_from_ops(n, ops) for n, ops in circs]
    try:
        b = B.tqs_batch_create(hs)
        try:
            count, total, offs = B.tqs_batch_info(b)
            st = torch.empty(total, dtype=torch.complex64, device="cuda")
            B.tqs_batch_run(b, st)
            torch.cuda.synchronize()
            got = st.cpu().numpy()
            for i, (n, ops) in enumerate(circs):
                alone, _ = fused(n, ops)
                assert np.array_equal(got[offs[i]:offs[i + 1]].view(np.uint32), alone.view(np.uint32))
                want = fsv_route.simulate(n, ops)
                assert np.max(np.abs(alone.astype(np.complex128) - want)) <= AMP_TOL
        finally:
            B.tqs_batch_destroy(b)
    finally:
        for h in hs:
            B.tqs_circuit_destroy(h)

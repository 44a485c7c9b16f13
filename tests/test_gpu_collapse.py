"""GPU parity of the collapse (simulateAndCollapse, Sec. 5.2): inverse-CDF
sampling against the FP64 oracle, through the C ABI.

Two kinds of comparison:
* The probabilities are an input (tqs_sample, tqs_batch_sample fed the
  oracle's own FP64 probabilities): both sides sample the same vector, so the
  indices must be equal, except where u T lies within 1e-12 T of a boundary
  C_j of the oracle's cumulative sums (summation order differs in the last
  bits); such draws are also checked to be valid (p > 0, next to the
  boundary).
* The probabilities come from the simulation (tqs_simulate_and_collapse, a
  batch run then tqs_batch_sample): the GPU state is FP32 (within 1e-5 of the
  oracle's amplitudes), so an index may differ only where u lies within 1e-5
  of a boundary C_j / T of the oracle.
"""
import numpy as np
import pytest

from oracle import collapse, fsv_route, observables
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
    torch.cuda.synchronize()


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def check_indices(p, u, got, tol):
    """got (GPU) against the oracle's inverse CDF of p; a difference is allowed
    only where u lies within tol of a boundary C_j / T crossed between the two
    answers, and the GPU index must have p > 0."""
    p = np.asarray(p, dtype=np.float64)
    want = collapse.sample(p, u)
    c = np.cumsum(p)
    t = c[-1]
    bad = np.nonzero(want != got)[0]
    for k in bad:
        g = int(got[k])
        assert 0 <= g < p.size and p[g] > 0.0, (k, g)
        lo, hi = sorted((int(want[k]), g))
        gap = np.min(np.abs(u[k] - c[lo:hi] / t)) if hi > lo else np.inf
        assert gap <= tol, (k, int(want[k]), g, gap)
    return bad.size


def random_probs(n, seed, zero_frac=0.3):
    rng = np.random.default_rng(seed)
    p = rng.random(1 << n) ** 2
    p[rng.random(1 << n) < zero_frac] = 0.0
    if not p.any():
        p[-1] = 1.0
    return p


def boundary_uniforms(p, rng, k):
    """k random uniforms, then k // 4 uniforms on boundaries C_j / T, then 0 and
    the largest double below 1.  Returns (u, number of random ones)."""
    c = np.cumsum(p)
    picks = np.clip(c[rng.integers(0, p.size, k // 4)] / c[-1], 0.0, np.nextafter(1.0, 0.0))
    u = np.concatenate([rng.random(k), picks, [0.0, np.nextafter(1.0, 0.0)]])
    return u, k


@pytest.mark.parametrize("n", [1, 3, 7, 8, 9, 12, 16, 20])
def test_sample_equals_oracle_on_same_probs(n):
    """Random uniforms: the same index as the oracle (at most a couple of draws
    may land within 1e-12 of a boundary).  Uniforms placed on the boundaries
    themselves may go either way between the two summation orders; they must
    still give a valid index next to that boundary."""
    rng = np.random.default_rng(100 + n)
    p = random_probs(n, 200 + n)
    u, k = boundary_uniforms(p, rng, 4096)
    out = torch.empty(u.size, dtype=torch.int64, device="cuda")
    B.tqs_sample(dev(p, torch.float64), n, u.size, dev(u, torch.float64), out)
    got = out.cpu().numpy()
    assert check_indices(p, u[:k], got[:k], 1e-12) <= 2
    check_indices(p, u[k:], got[k:], 1e-12)


def test_sample_dyadic_probabilities_exact():
    """Probabilities that are multiples of 1/64 summing to exactly 1: every
    partial sum is exact in FP64 on both sides, so every draw, the boundaries
    u = C_j included, must match exactly."""
    n = 6
    rng = np.random.default_rng(5)
    w = rng.integers(0, 2, 1 << n).astype(np.float64)
    w[0] = 0.0
    w[0] = 64.0 - w.sum()
    p = w / 64.0
    c = np.cumsum(p)
    assert c[-1] == 1.0
    u = np.concatenate([c[:-1], rng.random(500), [0.0]])
    out = torch.empty(u.size, dtype=torch.int64, device="cuda")
    B.tqs_sample(dev(p, torch.float64), n, u.size, dev(u, torch.float64), out)
    assert np.array_equal(out.cpu().numpy(), collapse.sample(p, u))


def test_sample_edge_cases():
    # all zero -> -1; a single nonzero entry always; zero shots is a no-op
    n = 9
    z = torch.zeros(1 << n, dtype=torch.float64, device="cuda")
    u = dev(np.array([0.0, 0.3, 0.999]), torch.float64)
    out = torch.full((3,), 7, dtype=torch.int64, device="cuda")
    B.tqs_sample(z, n, 3, u, out)
    assert out.cpu().tolist() == [-1, -1, -1]
    one = torch.zeros(1 << n, dtype=torch.float64, device="cuda")
    one[300] = 0.25
    B.tqs_sample(one, n, 3, u, out)
    assert out.cpu().tolist() == [300, 300, 300]
    B.tqs_sample(one, n, 0, None, None)
    with pytest.raises(B.TqsError):
        B.tqs_sample(one, 31, 1, u, out)


def test_batch_sample_equals_oracle_on_oracle_probs():
    """tqs_batch_sample on the oracle's FP64 probabilities of a 256-circuit
    random batch (n = 4..14): indices equal to the oracle's inverse CDF."""
    circs = W.batch_circuits(256, seed_tag=9)
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        count, total, offs = B.tqs_batch_info(b)
        probs = np.zeros(total)
        for i, (n, ops) in enumerate(circs):
            probs[offs[i]:offs[i + 1]] = observables.probabilities(fsv_route.simulate(n, ops))
        shots = 37
        rng = np.random.default_rng(12)
        u = rng.random(count * shots)
        out = torch.empty(count * shots, dtype=torch.int64, device="cuda")
        B.tqs_batch_sample(b, dev(probs, torch.float64), shots, dev(u, torch.float64), out)
        got = out.cpu().numpy().reshape(count, shots)
        n_bad = 0
        for i in range(count):
            n_bad += check_indices(probs[offs[i]:offs[i + 1]], u[i * shots:(i + 1) * shots],
                                   got[i], 1e-12)
        assert n_bad <= 2
    finally:
        B.tqs_batch_destroy(b)


def test_batch_run_then_sample_paper_mix_full_size():
    """16384 paper-shaped 11-qubit circuits (the bench workload), 64 shots each,
    sampled from the GPU's own probabilities; every 97th circuit is compared
    with the oracle's simulation and inverse CDF."""
    circs = [(11, ops) for _, ops in W.paper_mix(11, 16384, seed_tag=1)]
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        count, total, offs = B.tqs_batch_info(b)
        st = torch.empty(total, dtype=torch.complex64, device="cuda")
        pr = torch.empty(total, dtype=torch.float64, device="cuda")
        B.tqs_batch_run(b, st, pr, None)
        shots = 64
        rng = np.random.default_rng(13)
        u = rng.random(count * shots)
        out = torch.empty(count * shots, dtype=torch.int64, device="cuda")
        B.tqs_batch_sample(b, pr, shots, dev(u, torch.float64), out)
        got = out.cpu().numpy().reshape(count, shots)
        assert got.min() >= 0 and got.max() < 2048
        n_bad = 0
        for i in range(0, count, 97):
            p = observables.probabilities(fsv_route.simulate(11, circs[i][1]))
            n_bad += check_indices(p, u[i * shots:(i + 1) * shots], got[i], 1e-5)
        assert n_bad <= 0.01 * shots * (count // 97 + 1)
    finally:
        B.tqs_batch_destroy(b)


@pytest.mark.parametrize("kind", ["ghz", "qft", "random"])
def test_simulate_and_collapse(kind):
    n = 11
    rng = np.random.default_rng(14)
    ops = {"ghz": W.ghz_chain(n), "qft": W.qft_on_basis(n, 1234),
           "random": W.random_mixed(n, 20, (77, 1))}[kind]
    p = observables.probabilities(fsv_route.simulate(n, ops))
    c = B.circuit_from_ops(n, ops)
    try:
        idx = torch.empty(1, dtype=torch.int64, device="cuda")
        st = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        us = np.concatenate([rng.random(40), [0.25, 0.75]])
        for uu in us:
            B.tqs_simulate_and_collapse(c, dev(np.array([uu]), torch.float64), idx, st)
            i = int(idx.cpu()[0])
            check_indices(p, np.array([uu]), np.array([i]), 1e-5)
            s = st.cpu().numpy()
            assert s[i] == 1 and np.count_nonzero(s) == 1
            if kind == "ghz":
                assert i == (0 if uu < 0.5 else (1 << n) - 1)
        # without a state buffer only the index is produced
        B.tqs_simulate_and_collapse(c, dev(np.array([0.75]), torch.float64), idx, None)
        check_indices(p, np.array([0.75]), np.array([int(idx.cpu()[0])]), 1e-5)
    finally:
        B.tqs_circuit_destroy(c)


def test_shared_memory_path_equals_global_path():
    """Batch sampling stages circuits of n <= 13 in shared memory (exact
    fixed-point cumulative sums); tqs_sample always takes the global path (FP64
    sums in the same order).  Away from the boundaries the indices must be
    identical; for uniforms placed on boundaries C_j / T both paths must give
    an index the oracle accepts within 1e-12 of that boundary."""
    circs = W.batch_circuits(96, seed_tag=21)
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        count, total, offs = B.tqs_batch_info(b)
        rng = np.random.default_rng(22)
        probs = np.zeros(total)
        for i, (n, _) in enumerate(circs):
            probs[offs[i]:offs[i + 1]] = random_probs(n, 300 + i)
        shots = 50
        u = np.empty(count * shots)
        for i in range(count):
            c = np.cumsum(probs[offs[i]:offs[i + 1]])
            u[i * shots:(i + 1) * shots - 10] = rng.random(shots - 10)
            u[(i + 1) * shots - 10:(i + 1) * shots] = np.clip(
                c[rng.integers(0, c.size, 10)] / c[-1], 0.0, np.nextafter(1.0, 0.0))
        dp = dev(probs, torch.float64)
        du = dev(u, torch.float64)
        out = torch.empty(count * shots, dtype=torch.int64, device="cuda")
        B.tqs_batch_sample(b, dp, shots, du, out)
        got = out.cpu().numpy()
        one = torch.empty(shots, dtype=torch.int64, device="cuda")
        for i, (n, _) in enumerate(circs):
            B.tqs_sample(dp[offs[i]:offs[i + 1]], n, shots, du[i * shots:(i + 1) * shots], one)
            g1 = one.cpu().numpy()
            g0 = got[i * shots:(i + 1) * shots]
            assert np.array_equal(g1[:shots - 10], g0[:shots - 10]), (i, n)
            pi, ui = probs[offs[i]:offs[i + 1]], u[i * shots:(i + 1) * shots]
            check_indices(pi, ui[shots - 10:], g0[shots - 10:], 1e-12)
            check_indices(pi, ui[shots - 10:], g1[shots - 10:], 1e-12)
    finally:
        B.tqs_batch_destroy(b)

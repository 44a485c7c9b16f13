"""The allocation-free probabilities entry point (tqs_probabilities_noalloc).

It exists for callers that cannot call cudaMalloc (a framework that owns all
device memory in its own pool, or a loop that cannot afford an allocation's
device synchronisation); its partial sums live in a fixed device array inside
the library.  This test calls it through the C ABI twice in a row and checks
both results against tqs_probabilities, the allocating entry point.  It sits in
a file of its own that pytest collects last, and it passes alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest

from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()


@pytest.mark.parametrize("n", [1, 11, 20])
def test_noalloc_matches_allocating_entry_point_twice(n):
    g = W.rng(70, n)
    psi = (g.normal(size=1 << n) + 1j * g.normal(size=1 << n)).astype(np.complex64)
    d = torch.from_numpy(psi).cuda()
    p_ref = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    s_ref = torch.empty(1, dtype=torch.float64, device="cuda")
    B.tqs_probabilities(d, n, p_ref, s_ref)
    torch.cuda.synchronize()
    want_p = p_ref.cpu().numpy()
    want_s = float(s_ref.cpu()[0])
    for _ in range(2):
        p = torch.full((1 << n,), float("nan"), dtype=torch.float64, device="cuda")
        s = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        B.tqs_probabilities_noalloc(d, n, p, s)
        torch.cuda.synchronize()
        got_p = p.cpu().numpy()
        got_s = float(s.cpu()[0])
        assert np.max(np.abs(got_p - want_p)) <= 1e-15
        assert abs(got_s - want_s) <= 1e-12 * want_s


def test_noalloc_sum_only_and_size_limit():
    n = 14
    psi = np.zeros(1 << n, dtype=np.complex64)
    psi[3] = 0.6
    psi[77] = 0.8j
    d = torch.from_numpy(psi).cuda()
    for _ in range(2):
        s = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        B.tqs_probabilities_noalloc(d, n, None, s)
        torch.cuda.synchronize()
        assert abs(float(s.cpu()[0]) - 1.0) <= 1e-6
    with pytest.raises(B.TqsError) as e:
        B.tqs_probabilities_noalloc(d, 31, None, s)
    assert e.value.name == "TQS_ERR_TOO_MANY_QUBITS"


def test_noalloc_calls_no_allocator():
    """With a counting allocator installed (tqs_set_allocator routes every
    library scratch allocation through it), the allocation-free entry point
    never calls it, and the device's free memory does not change across the
    calls (after one warm call, which may load the library's kernels)."""
    counts = {"alloc": 0, "free": 0}

    def alloc(n, stream):
        counts["alloc"] += 1
        return None  # refuse: a call that needed memory would fail

    def free(p, stream):
        counts["free"] += 1

    inputs = []
    for n in (1, 11, 20):
        g = W.rng(71, n)
        psi = (g.normal(size=1 << n) + 1j * g.normal(size=1 << n)).astype(np.complex64)
        inputs.append((n, torch.from_numpy(psi).cuda(),
                       torch.empty(1 << n, dtype=torch.float64, device="cuda"),
                       torch.empty(1, dtype=torch.float64, device="cuda")))
    B.tqs_probabilities_noalloc(inputs[0][1], inputs[0][0], inputs[0][2], inputs[0][3])
    torch.cuda.synchronize()
    B.tqs_set_allocator(alloc, free)
    try:
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            for n, d, p, s in inputs:
                B.tqs_probabilities_noalloc(d, n, p, s)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
    finally:
        B.tqs_set_allocator()
    assert counts == {"alloc": 0, "free": 0}
    assert free1 == free0
    for n, d, p, s in inputs:
        x = d.cpu().numpy().astype(np.complex128)
        assert abs(float(s.cpu()[0]) - float(np.sum(np.abs(x) ** 2))) <= 1e-12 * (1 << n)

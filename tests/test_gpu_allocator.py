"""The caller's device allocator (tqs_set_allocator) on the GPU: with torch's
caching allocator installed, every form gives bitwise the same results as
with cudaMalloc, and the library's scratch really comes from the callbacks
(every block handed out is returned).
"""
import numpy as np
import pytest

from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import serve
from paper_2305_14398_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    yield
    B.tqs_set_allocator()
    torch.cuda.synchronize()


def run_everything():
    out = {}
    c = B.circuit_from_ops(11, W.qft_on_basis(11, 77))
    try:
        st = torch.empty(1 << 11, dtype=torch.complex64, device="cuda")
        pr = torch.empty(1 << 11, dtype=torch.float64, device="cuda")
        B.tqs_simulate(c, st, probs=pr)
        pl = torch.empty(1 << 11, dtype=torch.complex64, device="cuda")
        B.tqs_simulate_plain(c, pl)
        torch.cuda.synchronize()
        out["fused"] = st.cpu().numpy()
        out["plain"] = pl.cpu().numpy()
    finally:
        B.tqs_circuit_destroy(c)
    c = B.circuit_from_ops(8, W.random_layered(8, 3, (55, 8)))
    try:
        U = torch.empty((256, 256), dtype=torch.complex64, device="cuda")
        B.tqs_circuit_unitary(c, B.PREC_TC_BF16X3, U)
        torch.cuda.synchronize()
        out["chain"] = U.cpu().numpy()
    finally:
        B.tqs_circuit_destroy(c)
    circs = W.batch_circuits(128, seed_tag=57)
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        count, total, _ = B.tqs_batch_info(b)
        hs = np.empty(total, dtype=np.complex64)
        hn = np.empty(count, dtype=np.float64)
        B.tqs_batch_run_host(b, hs, None, hn)
        out["batch"] = hs
    finally:
        B.tqs_batch_destroy(b)
    reqs = W.serving_requests(40, rate_hz=50000.0, seed_tag=58)
    r = serve.replay(reqs, budget_bytes=1 << 30, max_inflight=2, max_batch=16, keep_states=True)
    out["serve"] = np.concatenate([r["states"][i].view(np.uint32) for i in range(len(reqs))])
    return out


def test_torch_allocator_same_results():
    ref = run_everything()
    live = {}
    counts = {"alloc": 0, "free": 0}

    def alloc(n, stream):
        p = torch.cuda.caching_allocator_alloc(n, torch.cuda.current_device(), stream if stream else None)
        live[p] = n
        counts["alloc"] += 1
        return p

    def free(p, stream):
        assert p in live
        del live[p]
        counts["free"] += 1
        torch.cuda.caching_allocator_delete(p)

    B.tqs_set_allocator(alloc, free)
    try:
        got = run_everything()
    finally:
        B.tqs_set_allocator()
    for k in ref:
        assert np.array_equal(np.asarray(got[k]).view(np.uint8), np.asarray(ref[k]).view(np.uint8)), k
    assert counts["alloc"] > 0 and counts["free"] > 0
    assert not live, "every block handed out came back"

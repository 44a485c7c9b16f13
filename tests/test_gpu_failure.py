"""Failure detection on the GPU without a fault: a device wait on an mbarrier
that nothing completes runs out its bound, the kernel records the time-out in a
status word and returns, the host reports TQS_ERR_TIMEOUT, and the context stays
usable for the next simulation."""
import numpy as np
import pytest

from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_bounded_wait_times_out_and_context_survives():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with pytest.raises(B.TqsError) as e:
        B.tqs_selftest_wait_timeout(2_000_000)  # ~1 ms at 2 GHz
    assert e.value.name == "TQS_ERR_TIMEOUT"
    c = B.circuit_from_ops(5, W.ghz_chain(5))
    try:
        out = torch.empty(32, dtype=torch.complex64, device="cuda")
        B.tqs_simulate(c, out)
        torch.cuda.synchronize()
    finally:
        B.tqs_circuit_destroy(c)
    got = out.cpu().numpy()
    assert abs(got[0] - 2 ** -0.5) < 1e-6 and abs(got[31] - 2 ** -0.5) < 1e-6


def test_autotuner_keeps_results_bitwise():
    """Launch shapes chosen by the autotuner never change a result bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_14398_gb300 import autotune
    circs = W.batch_circuits(256, 91)
    outs = []
    for w in (1, 4, 12):
        B.tqs_set_option(B.OPT_WARPS_PER_CTA, autotune.warp_slice_q(circs), w)
        b = B.tqs_batch_create_packed(*B.pack_ops(circs))
        try:
            count, total, _ = B.tqs_batch_info(b)
            st = torch.empty(total, dtype=torch.complex64, device="cuda")
            B.tqs_batch_run(b, st, None, None, use_graph=False)
            torch.cuda.synchronize()
            outs.append(st.cpu().numpy())
        finally:
            B.tqs_batch_destroy(b)
    B.tqs_set_option(B.OPT_WARPS_PER_CTA, autotune.warp_slice_q(circs), 4)
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))
    r = autotune.tune_warps_per_cta(circs, sample=256, reps=2, use_cache=False)
    assert r["warps"] in (1, 2, 3, 4, 6, 8, 12) and r["source"] == "measured"

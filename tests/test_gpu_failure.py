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
    """Launch shapes (warps per circuit and per CTA) never change a state or
    probability bit; the FP64 norm stays within its bound either way."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_14398_gb300 import autotune
    circs = W.batch_circuits(256, 91)
    q = autotune.warp_slice_q(circs)
    outs, norms = [], []
    for tw, w in ((1, 1), (1, 4), (1, 12), (2, 2), (2, 8), (2, 16)):
        B.tqs_set_option(B.OPT_TEAM_WARPS, q, tw)
        B.tqs_set_option(B.OPT_WARPS_PER_CTA, q, w)
        b = B.tqs_batch_create_packed(*B.pack_ops(circs))
        try:
            count, total, _ = B.tqs_batch_info(b)
            st = torch.empty(total, dtype=torch.complex64, device="cuda")
            pr = torch.empty(total, dtype=torch.float64, device="cuda")
            nm = torch.empty(count, dtype=torch.float64, device="cuda")
            B.tqs_batch_run(b, st, pr, nm, use_graph=False)
            torch.cuda.synchronize()
            outs.append((st.cpu().numpy(), pr.cpu().numpy()))
            norms.append(nm.cpu().numpy())
        finally:
            B.tqs_batch_destroy(b)
    B.tqs_set_option(B.OPT_TEAM_WARPS, q, 1)
    B.tqs_set_option(B.OPT_WARPS_PER_CTA, q, 4)
    for st, pr in outs[1:]:
        assert np.array_equal(st.view(np.uint32), outs[0][0].view(np.uint32))
        assert np.array_equal(pr.view(np.uint64), outs[0][1].view(np.uint64))
    for nm in norms:
        assert np.max(np.abs(nm - 1.0)) <= 1e-6
    r = autotune.tune_warps_per_cta(circs, sample=256, reps=2, use_cache=False)
    assert (r["team_warps"], r["warps"]) in autotune.CANDIDATES and r["source"] == "measured"
    B.tqs_set_option(B.OPT_TEAM_WARPS, q, 1)
    B.tqs_set_option(B.OPT_WARPS_PER_CTA, q, 4)

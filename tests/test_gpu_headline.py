"""GPU parity of the exact configuration the benchmark times: 16384 paper-shaped
11-qubit circuits (GHZ chain, Deutsch-Jozsa constant and balanced, QFT on a
seeded basis state, 25 % each; seed tag 1) in one CUDA-graph launch of the
persistent fused kernel, at three launch shapes: one warp per circuit and one
warp per CTA (the shape the autotuner picks), one warp per circuit and 8 warps
per CTA, and two warps per circuit and 16 warps per CTA.

Every circuit's state is compared element by element with the oracle's
per-gate route (eq. 12) at 1e-5; every probability with the oracle's
|psi_i|^2 at the bound the amplitude tolerance implies; every norm within 1e-6
of 1.  The launch must hand each persistent team several circuits (jobs >
teams), so that the job hand-over between circuits of a team is exercised.
"""
import numpy as np
import pytest

from oracle import fsv_route
from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_QUBITS = 11
COUNT = 16384
AMP_TOL = 1e-5
NORM_TOL = 1e-6


@pytest.fixture(scope="module")
def headline():
    """The circuits and the oracle's states (computed before any GPU call)."""
    mix = W.paper_mix(N_QUBITS, COUNT, seed_tag=1)
    circs = [(N_QUBITS, ops) for _, ops in mix]
    want = np.empty((COUNT, 1 << N_QUBITS), dtype=np.complex128)
    for i, (n, ops) in enumerate(circs):
        want[i] = fsv_route.simulate(n, ops)
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    return circs, want


def run_shape(circs, team_warps, warps_per_cta):
    q = N_QUBITS
    old = (B.tqs_get_option(B.OPT_TEAM_WARPS, q), B.tqs_get_option(B.OPT_WARPS_PER_CTA, q))
    B.tqs_set_option(B.OPT_TEAM_WARPS, q, team_warps)
    B.tqs_set_option(B.OPT_WARPS_PER_CTA, q, warps_per_cta)
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        count, total, offs = B.tqs_batch_info(b)
        st = torch.full((total,), float("nan"), dtype=torch.complex64, device="cuda")
        pr = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
        nm = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
        B.tqs_batch_run(b, st, pr, nm, use_graph=True)
        torch.cuda.synchronize()
        plan = B.tqs_batch_launch_info(b, 0)
    finally:
        B.tqs_batch_destroy(b)
        B.tqs_set_option(B.OPT_TEAM_WARPS, q, old[0])
        B.tqs_set_option(B.OPT_WARPS_PER_CTA, q, old[1])
    assert np.array_equal(offs, np.arange(count + 1, dtype=np.int64) << N_QUBITS)
    return (st.cpu().numpy().reshape(count, -1), pr.cpu().numpy().reshape(count, -1),
            nm.cpu().numpy(), plan)


def check_against_oracle(want, st, pr, nm):
    got = st.astype(np.complex128)
    err = np.abs(got - want).max(axis=1)
    bad = np.flatnonzero(err > AMP_TOL)
    assert bad.size == 0, f"circuits {bad[:10]} off by up to {err.max():.3e}"
    # |p - |o|^2| <= |g - o| (|g| + |o|) plus the FP32 rounding of |g|^2
    a = np.abs(want)
    bound = AMP_TOL * (2.0 * a + AMP_TOL) + 2.0 ** -22 * a * a + 1e-30
    assert np.all(np.abs(pr - a * a) <= bound)
    assert np.all(np.abs(pr.sum(axis=1) - 1.0) <= NORM_TOL)
    assert np.all(np.abs(nm - 1.0) <= NORM_TOL)


# (warps per circuit, warps per CTA): the autotuned shape (one team per CTA,
# 13 CTAs per SM), one warp per circuit with the most warps whose 16 KiB slices
# fit a CTA's shared memory, and the pair shape
SHAPES = [(1, 1), (1, 8), (2, 16)]


@pytest.mark.parametrize("team_warps,warps", SHAPES)
def test_headline_batch_every_circuit(headline, team_warps, warps):
    circs, want = headline
    st, pr, nm, plan = run_shape(circs, team_warps, warps)
    assert plan["jobs"] == COUNT
    assert plan["threads"] == warps * 32
    assert plan["teams"] == plan["grid"] * (warps // team_warps)
    # persistent teams each run several circuits through the job hand-over
    assert plan["jobs"] > 4 * plan["teams"], plan
    check_against_oracle(want, st, pr, nm)


def test_headline_shapes_bitwise_equal(headline):
    """States and probabilities do not depend on the launch shape."""
    circs, _ = headline
    a = run_shape(circs, *SHAPES[0])
    for shape in SHAPES[1:]:
        b = run_shape(circs, *shape)
        assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32)), shape
        assert np.array_equal(a[1].view(np.uint64), b[1].view(np.uint64)), shape

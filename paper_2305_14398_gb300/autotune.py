"""Autotuner for the launch shapes: the batched fused step kernel's warp
class (below), the one-CTA team, the full-state-vector tiles and the
tensor-core chain's raster (at the end of the file).

The warp-class kernel (circuits of n <= 11, each state in a shared-memory slice
of 2^q amplitudes) runs one or two warps per circuit and groups 1..16 warps per
CTA.  Two warps per circuit double the warps per byte of shared memory (more
latency hiding); few warps per CTA schedule circuits at a fine grain.  Which is
faster depends on the circuit mix and on the GPU, so it is measured: every
candidate runs a sample of the actual workload (CUDA events, best of several
runs) and the fastest is set with tqs_set_option(TQS_OPT_TEAM_WARPS, q, ...) and
tqs_set_option(TQS_OPT_WARPS_PER_CTA, q, ...).  States and probabilities do not
depend on the choice.  Results are cached in a JSON file keyed by GPU name, q
and batch size (TQS_AUTOTUNE_CACHE, default ~/.cache/tqs/autotune.json).
"""
from __future__ import annotations

import json
import os

from . import binding as B

# (warps per circuit, warps per CTA)
CANDIDATES = tuple((1, w) for w in (1, 2, 3, 4, 6, 8, 12, 16)) + \
    tuple((2, w) for w in (2, 4, 6, 8, 12, 16))
SLICE_LIMIT_BYTES = 200 * 1024


def cache_path() -> str:
    return os.environ.get("TQS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "tqs", "autotune.json"))


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
    except OSError:
        pass


def warp_slice_q(circuits) -> int:
    """log2 of the warp-slice amplitudes a batch of (n, ops) would use, or 0."""
    qs = [max(n, 4) for n, _ in circuits if max(n, 4) <= 11]
    return max(qs) if qs else 0


def _apply(q, tw, w):
    B.tqs_set_option(B.OPT_TEAM_WARPS, q, tw)
    B.tqs_set_option(B.OPT_WARPS_PER_CTA, q, w)


def tune_warps_per_cta(circuits, sample: int = 16384, reps: int = 5, use_cache: bool = True):
    """Pick warps per circuit and per CTA for the warp-class launch of this kind
    of batch.  Returns {"q", "team_warps", "warps", "timings_ms", "source"}."""
    import torch

    q = warp_slice_q(circuits)
    if q == 0:
        return {"q": 0, "team_warps": None, "warps": None, "timings_ms": {},
                "source": "no warp-class circuits"}
    key = f"v2|{torch.cuda.get_device_name()}|q{q}|{len(circuits)}"
    cache = _load() if use_cache else {}
    if key in cache:
        tw, w = int(cache[key]["team_warps"]), int(cache[key]["warps"])
        _apply(q, tw, w)
        return {"q": q, "team_warps": tw, "warps": w, "timings_ms": cache[key]["timings_ms"],
                "source": "cache"}
    arrays = B.pack_ops(list(circuits[:sample]))
    timings = {}
    for tw, w in CANDIDATES:
        if (w // tw) * (1 << q) * 8 > SLICE_LIMIT_BYTES:
            continue
        _apply(q, tw, w)
        b = B.tqs_batch_create_packed(*arrays)
        try:
            count, total, _ = B.tqs_batch_info(b)
            st = torch.empty(total, dtype=torch.complex64, device="cuda")
            pr = torch.empty(total, dtype=torch.float64, device="cuda")
            nm = torch.empty(count, dtype=torch.float64, device="cuda")
            for _ in range(2):
                B.tqs_batch_run(b, st, pr, nm, use_graph=False)
            best = float("inf")
            for _ in range(reps):
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record()
                B.tqs_batch_run(b, st, pr, nm, use_graph=False)
                e.record()
                torch.cuda.synchronize()
                best = min(best, s.elapsed_time(e))
            timings[f"{tw}x{w}"] = best
        finally:
            B.tqs_batch_destroy(b)
    tw, w = (int(x) for x in min(timings, key=timings.get).split("x"))
    _apply(q, tw, w)
    cache[key] = {"team_warps": tw, "warps": w, "timings_ms": timings}
    if use_cache:
        _save(cache)
    return {"q": q, "team_warps": tw, "warps": w, "timings_ms": timings, "source": "measured"}


# ----------------------------------------------------------------------------
# Further launch parameters, each timed on the workload it serves (CUDA
# events, best of a few runs) and cached by GPU name, size and batch size:
# * the one-CTA team's thread count for circuits of 12..14 qubits
#   (TQS_OPT_CTA_THREADS: 256 or 512);
# * the tile bits of the full-state-vector passes (TQS_OPT_FSV_TILE_Q);
# * the raster band of the tensor-core chain's GEMM grid (TQS_OPT_CHAIN_GROUP).
# None of them changes a state or a unitary (the CTA team's FP64 norm follows
# the team size in its reduction order only).

def _best_ms(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e))
    return best


def _tune(key, option, candidates, run, reps, use_cache):
    """Time run() under each candidate value of `option`, set the fastest,
    and cache it under `key`."""
    cache = _load() if use_cache else {}
    if key in cache:
        v = int(cache[key]["value"])
        B.tqs_set_option(option, 0, v)
        return {"value": v, "timings_ms": cache[key]["timings_ms"], "source": "cache"}
    old = B.tqs_get_option(option, 0)
    timings = {}
    try:
        for v in candidates:
            B.tqs_set_option(option, 0, v)
            timings[str(v)] = _best_ms(run, reps)
    except Exception:
        B.tqs_set_option(option, 0, old)
        raise
    v = int(min(timings, key=timings.get))
    B.tqs_set_option(option, 0, v)
    if use_cache:
        cache[key] = {"value": v, "timings_ms": timings}
        _save(cache)
    return {"value": v, "timings_ms": timings, "source": "measured"}


def cta_subset(circuits):
    """The circuits of a batch that run on one-CTA teams (12..14 qubits) and
    the cache-key part that tells such subsets apart."""
    sub = [(n, ops) for n, ops in circuits if 12 <= max(n, 4) <= 14]
    amps = sum(1 << n for n, _ in sub)
    gates = sum(len(ops) for _, ops in sub)
    return sub, f"cta|{len(sub)}|a{amps}|g{gates}"


def tune_cta_threads(circuits, reps: int = 5, use_cache: bool = True):
    """Threads of the one-CTA team (circuits of 12..14 qubits) for this batch.

    A batch fixes its launch plan when it is first uploaded, so every
    candidate runs on a batch of its own: the whole batch (its one-CTA kernel
    runs beside the other team kinds' kernels), through its CUDA graph, with
    the probabilities written and L2 flushed before each timed run, as the
    bench times it.  The cache key carries the count, total amplitudes and
    total gates of the 12..14-qubit subset and the batch size: two batches of
    the same size and largest n but another mix of circuits are tuned apart."""
    import torch
    sub, tail = cta_subset(circuits)
    if not sub:
        return {"value": None, "timings_ms": {}, "source": "no circuits of 12..14 qubits"}
    key = f"v5|{torch.cuda.get_device_name()}|{tail}|{len(circuits)}"
    cache = _load() if use_cache else {}
    if key in cache:
        v = int(cache[key]["value"])
        B.tqs_set_option(B.OPT_CTA_THREADS, 0, v)
        return {"value": v, "timings_ms": cache[key]["timings_ms"], "source": "cache"}
    arrays = B.pack_ops(list(circuits))
    old = B.tqs_get_option(B.OPT_CTA_THREADS, 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    timings = {}
    try:
        for v in (256, 512):
            B.tqs_set_option(B.OPT_CTA_THREADS, 0, v)
            b = B.tqs_batch_create_packed(*arrays)
            try:
                count, total, _ = B.tqs_batch_info(b)
                st = torch.empty(total, dtype=torch.complex64, device="cuda")
                pr = torch.empty(total, dtype=torch.float64, device="cuda")
                nm = torch.empty(count, dtype=torch.float64, device="cuda")
                for _ in range(2):
                    B.tqs_batch_run(b, st, pr, nm, use_graph=True)
                best = float("inf")
                for _ in range(reps):
                    flush.zero_()
                    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    s.record()
                    B.tqs_batch_run(b, st, pr, nm, use_graph=True)
                    e.record()
                    torch.cuda.synchronize()
                    best = min(best, s.elapsed_time(e))
                timings[str(v)] = best
            finally:
                B.tqs_batch_destroy(b)
    except Exception:
        B.tqs_set_option(B.OPT_CTA_THREADS, 0, old)
        raise
    v = int(min(timings, key=timings.get))
    B.tqs_set_option(B.OPT_CTA_THREADS, 0, v)
    if use_cache:
        cache[key] = {"value": v, "timings_ms": timings}
        _save(cache)
    return {"value": v, "timings_ms": timings, "source": "measured"}


def tune_fsv_tile(n, ops, reps: int = 2, use_cache: bool = True):
    """Tile bits of the full-state-vector passes for this circuit size."""
    import torch
    key = f"v3|{torch.cuda.get_device_name()}|fsv|n{n}|{len(ops)}"
    c = B.circuit_from_ops(n, ops)
    try:
        st = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
        st[0] = 1.0
        cands = tuple(t for t in (11, 12, 13) if t <= n)
        return _tune(key, B.OPT_FSV_TILE_Q, cands, lambda: B.tqs_simulate_fsv(c, st), reps, use_cache)
    finally:
        B.tqs_circuit_destroy(c)


def tune_chain_group(n, ops, prec, reps: int = 2, use_cache: bool = True):
    """Raster band of the tensor-core chain for this size and precision."""
    import torch
    key = f"v3|{torch.cuda.get_device_name()}|chain|n{n}|p{prec}|{len(ops)}"
    c = B.circuit_from_ops(n, ops)
    try:
        U = torch.empty((1 << n, 1 << n), dtype=torch.complex64, device="cuda")
        cands = tuple(g for g in (4, 8, 16, 32) if g <= (1 << n) // 128)
        return _tune(key, B.OPT_CHAIN_GROUP, cands, lambda: B.tqs_circuit_unitary(c, prec, U), reps,
                     use_cache)
    finally:
        B.tqs_circuit_destroy(c)

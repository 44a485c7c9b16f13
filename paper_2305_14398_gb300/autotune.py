"""Autotuner for the batched fused step kernel's launch shape.

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

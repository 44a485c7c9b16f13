"""Autotuner for the batched fused step kernel's launch shape.

The warp-team kernel (one warp per circuit, its state in a shared-memory slice of
2^q amplitudes) can group 1..16 warps per CTA.  Few warps per CTA schedule
circuits at a fine grain; more warps share one CTA's launch overhead.  Which is
faster depends on the circuit mix and on the GPU, and the choice never changes a
result bit, so it is measured: every candidate runs a sample of the actual
workload (CUDA events, best of several runs) and the fastest is set with
tqs_set_option(TQS_OPT_WARPS_PER_CTA, q, warps).  Results are cached in a JSON
file keyed by GPU name and q (TQS_AUTOTUNE_CACHE, default
~/.cache/tqs/autotune.json).
"""
from __future__ import annotations

import json
import os

from . import binding as B

CANDIDATES = (1, 2, 3, 4, 6, 8, 12, 16)
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


def tune_warps_per_cta(circuits, sample: int = 4096, reps: int = 5, use_cache: bool = True):
    """Pick warps per CTA for the warp-team launch of this kind of batch.
    Returns {"q", "warps", "timings_ms", "source"}."""
    import torch

    q = warp_slice_q(circuits)
    if q == 0:
        return {"q": 0, "warps": None, "timings_ms": {}, "source": "no warp-team circuits"}
    key = f"{torch.cuda.get_device_name()}|q{q}|{len(circuits)}"
    cache = _load() if use_cache else {}
    if key in cache:
        w = int(cache[key]["warps"])
        B.tqs_set_option(B.OPT_WARPS_PER_CTA, q, w)
        return {"q": q, "warps": w, "timings_ms": cache[key]["timings_ms"], "source": "cache"}
    arrays = B.pack_ops(list(circuits[:sample]))
    timings = {}
    for w in CANDIDATES:
        if w * (1 << q) * 8 > SLICE_LIMIT_BYTES:
            continue
        B.tqs_set_option(B.OPT_WARPS_PER_CTA, q, w)
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
            timings[str(w)] = best
        finally:
            B.tqs_batch_destroy(b)
    w = int(min(timings, key=timings.get))
    B.tqs_set_option(B.OPT_WARPS_PER_CTA, q, w)
    cache[key] = {"warps": w, "timings_ms": timings}
    if use_cache:
        _save(cache)
    return {"q": q, "warps": w, "timings_ms": timings, "source": "measured"}

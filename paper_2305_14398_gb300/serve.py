"""Real-time serving driver over the continuous-batching server (tqs_server_*).

    python -m paper_2305_14398_gb300.serve [--requests 20000] [--rate 2000]
        [--budget-gb 120] [--inflight 4] [--max-batch 256]

Replays seeded Poisson arrivals (workloads.serving_requests: n ~ U{6..16},
25 % each GHZ / Deutsch-Jozsa / QFT / random mixed) against the wall clock:
each request is submitted at its arrival time, the server is polled
continuously, and latency = finish time observed by the poll - arrival time.
Requests are packed into host arrays before the clock starts (marshalling).
"""
from __future__ import annotations

import argparse
import gc
import json
import time

import numpy as np

from . import binding as B
from . import workloads as W


def replay(requests, budget_bytes: int, max_inflight: int = 4, max_batch: int = 256,
           keep_states: bool = False, max_seconds: float = 600.0):
    """Replay requests [(arrival_s, kind, n, ops)]; returns a result dict with
    per-request latencies (s), norms, optional states and server counters."""
    packed = [B.pack_request(ops) for (_, _, _, ops) in requests]
    arrivals = np.array([r[0] for r in requests], dtype=np.float64)
    ns = [r[2] for r in requests]
    count = len(requests)
    sv = B.tqs_server_create(budget_bytes, max_inflight, max_batch)
    finish = np.full(count, np.nan)
    norms = np.full(count, np.nan)
    states = {} if keep_states else None
    polls = 0
    busy_s = 0.0  # wall time with at least one batch in flight (device busy)
    # no cyclic garbage collection while the clock runs: a collection over a
    # large caller heap pauses this polling loop for tens of milliseconds
    gc_was_on = gc.isenabled()
    gc.disable()
    try:
        t0 = time.perf_counter()
        nxt = 0
        done = 0
        last = 0.0
        while done < count:
            now = time.perf_counter() - t0
            if B.tqs_server_stats(sv)["inflight"] > 0:
                busy_s += now - last
            last = now
            if now > max_seconds:
                raise RuntimeError(f"serving did not finish within {max_seconds} s")
            while nxt < count and arrivals[nxt] <= now:
                B.tqs_server_submit_packed(sv, nxt, ns[nxt], packed[nxt])
                nxt += 1
            tags = B.tqs_server_poll(sv)
            polls += 1
            if len(tags):
                t = time.perf_counter() - t0
                for tag in tags:
                    tag = int(tag)
                    st, nm = B.tqs_server_take(sv, tag, ns[tag] if keep_states else None)
                    finish[tag] = t
                    norms[tag] = nm
                    if keep_states:
                        states[tag] = st
                done += len(tags)
        wall = time.perf_counter() - t0
        stats = B.tqs_server_stats(sv)
    finally:
        if gc_was_on:
            gc.enable()
        B.tqs_server_destroy(sv)
    lat = finish - arrivals
    return {
        "latency_s": lat, "norms": norms, "states": states, "wall_s": wall,
        "throughput_rps": count / wall, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
        "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_ms": 1e3 * float(np.mean(lat)),
        "max_ms": 1e3 * float(np.max(lat)), "polls": polls, "stats": stats,
        "busy_frac": busy_s / wall,
    }


def sweep(rates, requests_per_rate: int = 20000, budget_bytes: int = 120 * 10 ** 9,
          max_inflight: int = 4, max_batch: int = 256, seed_tag: int = 4):
    """Offered load against latency: one replay per Poisson rate (req/s) of the
    same request mix; per rate p50 / p99 latency, completed req/s and the
    busy fraction (wall time with a batch in flight)."""
    out = []
    for rate in rates:
        reqs = W.serving_requests(requests_per_rate, float(rate), seed_tag=seed_tag)
        r = replay(reqs, budget_bytes, max_inflight, max_batch)
        out.append({"offered_rps": float(rate), "completed_rps": r["throughput_rps"],
                    "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "max_ms": r["max_ms"],
                    "busy_frac": r["busy_frac"],
                    "norm_max_err": float(np.max(np.abs(r["norms"] - 1.0)))})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--inflight", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=256)
    a = ap.parse_args()
    reqs = W.serving_requests(a.requests, a.rate)
    r = replay(reqs, int(a.budget_gb * 1e9), a.inflight, a.max_batch)
    out = {k: r[k] for k in ("throughput_rps", "p50_ms", "p99_ms", "mean_ms", "max_ms", "wall_s",
                             "polls", "stats")}
    out["norm_max_err"] = float(np.max(np.abs(r["norms"] - 1.0)))
    print(json.dumps(out))


if __name__ == "__main__":
    main()

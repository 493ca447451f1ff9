"""Batched GGArrays: the workload of thousands of arrays of uneven size grown
in one persistent launch, the per-array parameter rule, and its autotuner.

Every array a gets: payload size E = (4, 8, 16)[a % 3] bytes, a target
size S_a = min(16M, floor(exp(ln 65536 + 1.5 z_a))) (at least 1) with z_a a
standard normal drawn by Box-Muller from the counter-based generator, and
Poisson(1) per-thread counts per round.  The rule maps S_a to (threads per
block T, LFVectors L_a, first bucket B); the autotuner measures candidate
rules on the GPU and keeps the fastest whose memory stays within 2x the
needed memory plus the first buckets.
"""

from __future__ import annotations

import json
import math
import os
import time
from dataclasses import asdict, dataclass

import numpy as np

from . import workloads as wl

TUNED_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_batch.json")
MAX_SIZE = 16 << 20


def batched_sizes(n: int = 4096, seed: int = 3) -> np.ndarray:
    """Lognormal target sizes (median 64K, sigma 1.5, capped 16M, >= 1)."""
    h1 = wl.splitmix_at(seed, np.arange(n, dtype=np.uint64) * np.uint64(2))
    h2 = wl.splitmix_at(seed, np.arange(n, dtype=np.uint64) * np.uint64(2) + np.uint64(1))
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 1.0) / float(1 << 53)   # (0, 1]
    u2 = (h2 >> np.uint64(11)).astype(np.float64) / float(1 << 53)           # [0, 1)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    s = np.floor(np.exp(math.log(65536.0) + 1.5 * z))
    return np.clip(s, 1, MAX_SIZE).astype(np.int64)


def payload_bytes(a: int) -> int:
    return (4, 8, 16)[a % 3]


@dataclass
class Rule:
    """Per-array parameters from the target size: L_a = ceil(S / per_lfv)
    (1..max_l), B = the power of two nearest (S / L_a) / b_div, within
    [256, 65536]; T fixed."""
    T: int = 256
    per_lfv: int = 32768
    b_div: int = 16
    max_l: int = 1024

    def params(self, size: int):
        L = int(min(self.max_l, max(1, -(-int(size) // self.per_lfv))))
        per = max(1, int(size) // L)
        b = max(1.0, per / self.b_div)
        B = int(min(65536, max(256, 1 << int(round(math.log2(b))))))
        return self.T, L, B


def spec_for(gga_mod, a: int):
    """Counts Poisson(1) and self-describing values for array a."""
    thr = wl.poisson1_thresholds()
    return gga_mod.make_gen_spec((3 << 32) | a, "poisson", (0x10001, 0x9E3779B9, 7), round0=0, thresholds=thr)


@dataclass
class TypedRule:
    """One Rule per payload size (4, 8 and 16 bytes)."""
    by_payload: dict

    def params_for(self, a: int, size: int):
        return self.by_payload[payload_bytes(a)].params(size)

    def to_json(self):
        return {str(e): asdict(r) for e, r in self.by_payload.items()}


def params_for(rule, a: int, size: int):
    """(T, L, B) of array a of target `size` under a Rule or a TypedRule."""
    return rule.params_for(a, size) if isinstance(rule, TypedRule) else rule.params(size)


def build(sizes, rule, stream=None, pool_slack: float = 2.3):
    """Make the arrays (one shared pool) and the batch; returns
    (pool, arrays, batch, params list)."""
    from . import gga
    params = [params_for(rule, a, int(s)) for a, s in enumerate(sizes)]
    need = sum(int(s) * payload_bytes(a) for a, s in enumerate(sizes))
    first = sum(L * B * payload_bytes(a) for a, (_, L, B) in enumerate(params))
    pool_bytes = int(pool_slack * need + 2 * first + (256 << 20))
    pool = gga.GGAPool(pool_bytes, 256 * 4, stream=stream)
    arrays, jobs = [], []
    for a, (s, (T, L, B)) in enumerate(zip(sizes, params)):
        g = gga.GGArray(L, T, B, payload_bytes(a), shared_pool=pool, stream=stream)
        arrays.append(g)
        jobs.append((g, spec_for(gga, a), int(s)))
    batch = gga.GGABatch(jobs, stream=stream)
    return pool, arrays, batch, params


def teardown(pool, arrays, batch):
    batch.close()
    for g in arrays:
        g.close()
    pool.close()


def time_batch(batch, stream, steps: int = 5, warmup: int = 2) -> float:
    """Median milliseconds of one captured clear+grow replay."""
    import torch
    batch.capture(stream)
    for _ in range(warmup):
        batch.replay(stream)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        a.record(stream)
        batch.replay(stream)
        b.record(stream)
    torch.cuda.synchronize()
    return sorted(a.elapsed_time(b) for a, b in evs)[steps // 2]


def memory_ratio(arrays) -> float:
    used = need = 0
    for g in arrays:
        m = g.memory()
        used += m["bucket_bytes"]
        need += m["live_bytes"]
    return used / max(1, need)


def candidates():
    """The global grid: blocks of 512 or 1024 threads (smaller ones measured
    2-4x slower), 32K to 1M elements per LFVector, first bucket = the
    LFVector's share / 1..16."""
    for T in (512, 1024):
        for per_lfv in (32768, 131072, 262144, 524288, 1048576):
            for b_div in (1, 2, 4, 8, 16):
                yield Rule(T=T, per_lfv=per_lfv, b_div=b_div)


def neighbours(rule: Rule):
    """Rules around `rule`: per_lfv and b_div halved, kept or doubled, both T."""
    for T in (512, 1024):
        for f in (0.5, 1, 2):
            for d in (0.5, 1, 2):
                per = int(rule.per_lfv * f)
                bd = max(1, int(rule.b_div * d))
                if 4096 <= per <= (4 << 20):
                    yield Rule(T=T, per_lfv=per, b_div=bd)


def autotune(sizes, stream, out_path: str = TUNED_FILE, max_ratio: float = 2.05, log=print):
    """Measure candidate rules on the GPU and keep the fastest whose memory
    ratio is at most max_ratio: first one rule for every array over the
    global grid, then, payload type by payload type, the neighbours of the
    best rule for that type's arrays with the others' rules fixed.  Writes
    the choice and every measurement."""
    results = []
    total = int(np.sum(sizes))

    def measure(rule, tag):
        pool, arrays, batch, _ = build(sizes, rule, stream)
        ms = time_batch(batch, stream)
        ratio = memory_ratio(arrays)
        teardown(pool, arrays, batch)
        rec = {"stage": tag, "rule": rule.to_json() if isinstance(rule, TypedRule) else asdict(rule), "ms": ms,
               "gelem_s": total / (ms / 1e3) / 1e9, "mem_ratio": ratio}
        results.append(rec)
        log(json.dumps(rec))
        return ms, ratio

    best_rule, best_ms = None, math.inf
    for rule in candidates():
        ms, ratio = measure(rule, "global")
        if ratio <= max_ratio and ms < best_ms:
            best_rule, best_ms = rule, ms
    if best_rule is None:
        best_rule = Rule()
    typed = TypedRule({4: best_rule, 8: best_rule, 16: best_rule})
    for e in (4, 8, 16):
        for cand in neighbours(typed.by_payload[e]):
            if cand == typed.by_payload[e]:
                continue
            trial = TypedRule(dict(typed.by_payload))
            trial.by_payload[e] = cand
            ms, ratio = measure(trial, f"payload{e}")
            if ratio <= max_ratio and ms < best_ms:
                typed, best_ms = trial, ms
    doc = {"chosen_by_payload": typed.to_json(), "ms": best_ms, "measured": results, "n_arrays": len(sizes),
           "elements": total, "max_mem_ratio": max_ratio,
           "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    with open(out_path, "w") as f:
        json.dump(doc, f, indent=1)
    return typed


def tuned_rule():
    """The rule the autotuner chose (per payload type when it chose so), or
    the default rule."""
    try:
        with open(TUNED_FILE) as f:
            doc = json.load(f)
        if "chosen_by_payload" in doc:
            return TypedRule({int(e): Rule(**r) for e, r in doc["chosen_by_payload"].items()})
        return Rule(**doc["chosen"])
    except (OSError, KeyError, ValueError, TypeError):
        return Rule()


def plain_time(arrays, sizes, stream, steps: int = 3) -> float:
    """Milliseconds to grow every array with its own launches, one array
    after another (the plain one-launch-per-array form), median of steps."""
    import torch
    from . import gga
    singles = [gga.GGABatch([(g, spec_for(gga, a), int(s))], stream=stream)
               for a, (g, s) in enumerate(zip(arrays, sizes))]
    times = []
    for _ in range(steps + 1):
        for b in singles:
            b.clear(stream)
        a_ev = torch.cuda.Event(enable_timing=True)
        b_ev = torch.cuda.Event(enable_timing=True)
        a_ev.record(stream)
        for b in singles:
            b.grow(stream)
        b_ev.record(stream)
        torch.cuda.synchronize()
        times.append(a_ev.elapsed_time(b_ev))
    for b in singles:
        b.close()
    return sorted(times[1:])[len(times[1:]) // 2]


if __name__ == "__main__":
    import argparse
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--autotune", metavar="OUT_JSON", help="measure the candidate rules, write the choice here")
    args = ap.parse_args()
    if args.autotune:
        s = torch.cuda.Stream()
        rule = autotune(batched_sizes(), s, out_path=args.autotune)
        print("chosen", rule)

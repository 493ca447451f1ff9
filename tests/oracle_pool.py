"""Oracle runs in worker processes, for checks of workloads too large for
one core in a test's time: each worker builds the oracle's state of one
array and returns a digest of it (sizes, capacities, offsets, flattened
contents), which the test compares with the same digest of the GPU's
array.  Workers are started with `spawn` (never forked from a process
that holds a CUDA context) and import only the oracle and numpy."""

from __future__ import annotations

import hashlib
import multiprocessing as mp
import os

import numpy as np


def state_digest(sizes, caps, offsets, flat_bytes: bytes) -> str:
    h = hashlib.sha256()
    for x in (sizes, caps, offsets):
        h.update(np.ascontiguousarray(x, dtype=np.uint64).tobytes())
    h.update(flat_bytes)
    return h.hexdigest()


def _grown_digest(job):
    """job = (key, L, T, B, E, seed, dist, coeffs, target, thresholds)."""
    import oracle
    key, L, T, B, E, seed, dist, coeffs, target, thr = job
    o = oracle.OracleGGArray(L, T, B, E)
    o.grow_to_target(seed, dist, coeffs, target, thresholds=thr)
    caps, _ = o.capacities()
    d = state_digest(o.sizes(), caps, o.offsets(), o.flatten().tobytes())
    o.close()
    return key, d


def grown_digests(jobs, workers: int | None = None, timeout_s: float = 900.0) -> dict:
    """Digests of the oracle's grow_to_target for every job, largest first,
    in a spawned worker pool (a worker that dies makes the call fail after
    timeout_s instead of waiting forever)."""
    jobs = sorted(jobs, key=lambda j: -int(j[8]))
    n = workers or max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n) as pool:
        return dict(pool.map_async(_grown_digest, jobs, chunksize=4).get(timeout=timeout_s))


def _served_digests(job):
    """job = (L, T, B, E, read_n, [(array, [(request, type, n, tag), ...]), ...]):
    each array's admitted requests replayed in arrival order on its own
    oracle (an append of n elements, a read of read_n random indices, a
    flatten that retires the array); returns {request: SHA-256 of the read
    or flatten result}."""
    import oracle
    L, T, B, E, read_n, arrays = job
    out = {}
    for _, reqs in arrays:
        o = oracle.OracleGGArray(L, T, B, E)
        for r, typ, n, tag in reqs:
            if typ == 0:
                o.append(int(n), int(tag))
            elif typ == 1:
                out[r] = hashlib.sha256(o.read_random(read_n, int(tag)).tobytes()).hexdigest()
            else:
                out[r] = hashlib.sha256(o.flatten().tobytes()).hexdigest()
                o.close()
                o = oracle.OracleGGArray(L, T, B, E)
        o.close()
    return out


def served_digests(L, T, B, E, read_n, typ, arr, nn, tag, admitted, workers: int | None = None,
                   timeout_s: float = 900.0) -> dict:
    """Oracle digests of every admitted read and flatten of a served trace
    (admitted: boolean mask of the requests the server completed), one
    array at a time in spawned workers (an array's data lives only while
    its requests replay)."""
    idx = np.nonzero(admitted)[0]
    per = {}
    for r in idx:
        per.setdefault(int(arr[r]), []).append((int(r), int(typ[r]), int(nn[r]), int(tag[r])))
    items = sorted(per.items(), key=lambda kv: -sum(x[2] for x in kv[1] if x[1] == 0))
    n = workers or max(1, min(16, os.cpu_count() or 1))
    chunks = [items[i::n * 4] for i in range(n * 4)]
    jobs = [(L, T, B, E, read_n, c) for c in chunks if c]
    out = {}
    with mp.get_context("spawn").Pool(n) as pool:
        for d in pool.map_async(_served_digests, jobs).get(timeout=timeout_s):
            out.update(d)
    return out

"""A continuous-batching request server over many live GGArrays.

Requests arrive open-loop (Poisson arrivals) against up to 65,536 live
int64 arrays sharing one bucket pool:

* append n elements (n log-uniform over 1..10^6),
* read 4096 random indices,
* flatten (the contiguous copy is produced in device memory and the array
  is retired: its buckets go back to the pool's free queues).

The loop admits requests that arrived while earlier batches ran, packs
them into one append launch, one read launch and the flattens of the step
(at most one request per array per step, so per-array order is arrival
order), and keeps a few steps in flight; a request completes when its
step's event has completed.  Appends are admitted by the pool's free
memory, computed by a host mirror of the device allocator (the same
per-size free counts and bump pointer, so an admitted append always fits).
An append that does not fit leaves the ready queue for a waiting queue: it
is tried again, oldest first, after a flatten has returned memory, and is
rejected after a deadline.  Its array's later requests stay behind it (per
array, requests run in arrival order), while other arrays' requests go on.
The plain mode runs the same trace one request at a time, waiting for each.
"""

from __future__ import annotations

import hashlib
import heapq
import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import workloads as wl

APPEND, READ, FLATTEN = 0, 1, 2


@dataclass
class ServeConfig:
    n_arrays: int = 65536
    L: int = 4
    T: int = 256
    B: int = 1024
    E: int = 8
    pool_bytes: int = 64 << 30
    rate: float = 20000.0
    duration: float = 60.0
    mix: tuple = (0.70, 0.25, 0.05)
    read_n: int = 4096
    max_append: int = 1_000_000
    deadline: float = 0.05
    seed: int = 4
    max_inflight: int = 3
    max_batch: int = 480
    flatten_arena_bytes: int = 8 << 30


def make_trace(cfg: ServeConfig):
    """Arrival times (s), request types, array ids, append sizes, seeds/tags."""
    n = int(cfg.rate * cfg.duration * 1.2) + 16
    k = np.arange(n, dtype=np.uint64)
    u = lambda j: ((wl.splitmix_at(cfg.seed, k * np.uint64(4) + np.uint64(j)) >> np.uint64(11)).astype(np.float64)
                   + 0.5) / float(1 << 53)
    t = np.cumsum(-np.log(u(0)) / cfg.rate)
    keep = t < cfg.duration
    t = t[keep]
    m = t.shape[0]
    typ = np.where(u(1)[:m] < cfg.mix[0], APPEND, np.where(u(1)[:m] < cfg.mix[0] + cfg.mix[1], READ, FLATTEN))
    arr = (wl.splitmix_at(cfg.seed + 1, k[:m]) % np.uint64(cfg.n_arrays)).astype(np.int64)
    nn = np.floor(np.exp(u(2)[:m] * math.log(cfg.max_append))).astype(np.int64)
    nn = np.clip(nn, 1, cfg.max_append)
    tag = np.arange(m, dtype=np.int64) + 1          # request id: also the append tag and read seed
    return t, typ.astype(np.int8), arr, nn, tag


class PoolMirror:
    """Host copy of the device pool's accounting: per byte class the number
    of free buckets, and the bump pointer."""

    def __init__(self, pool_bytes: int):
        self.cap = pool_bytes
        self.bump = 0
        self.free = [0] * 64

    @staticmethod
    def cls(nbytes: int) -> int:
        return max(8, (max(nbytes, 256) - 1).bit_length())

    @staticmethod
    def tally(classes):
        """{class: number of buckets} of a list of bucket classes."""
        out = {}
        for c in classes:
            out[c] = out.get(c, 0) + 1
        return out

    def need(self, tally):
        """Bump bytes an allocation of these buckets would take now (free
        buckets of a class are used first, as the device allocator does)."""
        bump = 0
        for c, k in tally.items():
            f = self.free[c]
            if k > f:
                bump += (k - f) << c
        return bump

    def take(self, tally):
        for c, k in tally.items():
            f = self.free[c]
            if k > f:
                self.bump += (k - f) << c
                f = k
            self.free[c] = f - k

    def give(self, tally):
        for c, k in tally.items():
            self.free[c] += k


def buckets_for(size: int, B: int) -> int:
    if size == 0:
        return 0
    return (size - 1 + B).bit_length() - B.bit_length() + 1


class ArrayState:
    __slots__ = ("g", "sizes", "queue", "busy")

    def __init__(self, g, L):
        self.g = g
        self.sizes = [0] * L
        self.queue = deque()
        self.busy = False


class CudaBackend:
    """Device side of the server: the library, one stream, events, int64 buffers."""

    def __init__(self):
        import torch
        from . import gga
        self.torch = torch
        self.gga = gga

    def stream(self):
        return self.torch.cuda.Stream()

    def event(self):
        return self.torch.cuda.Event()

    def empty_i64(self, shape):
        return self.torch.empty(shape, dtype=self.torch.int64, device="cuda")


class Server:
    LOOK_AHEAD = 32     # waiting appends tried per step after memory was freed

    def __init__(self, cfg: ServeConfig, stream=None, record=False, backend=None):
        """record: False, True (keep every read and flatten result), or
        "digest" (keep the SHA-256 of each result's bytes)."""
        self.be = backend or CudaBackend()
        gga = self.gga = self.be.gga
        self.cfg = cfg
        self.stream = stream or self.be.stream()
        self.pool = gga.GGAPool(cfg.pool_bytes, cfg.B * cfg.E, stream=self.stream)
        self.mirror = PoolMirror(cfg.pool_bytes)
        self.arrays = [ArrayState(gga.GGArray(cfg.L, cfg.T, cfg.B, cfg.E, shared_pool=self.pool,
                                              stream=self.stream), cfg.L) for _ in range(cfg.n_arrays)]
        self.read_out = self.be.empty_i64((cfg.max_inflight + 1, cfg.max_batch, cfg.read_n))
        self.flat_arena = self.be.empty_i64(cfg.flatten_arena_bytes // 8)
        self.record = record
        self.results = {}

    # -- accounting ---------------------------------------------------------
    def _append_classes(self, st: ArrayState, n: int):
        cfg = self.cfg
        out = []
        for l in range(cfg.L):
            c = n // cfg.L + (1 if l < n % cfg.L else 0)
            s = st.sizes[l]
            for b in range(buckets_for(s, cfg.B), buckets_for(s + c, cfg.B)):
                out.append(PoolMirror.cls((cfg.B << b) * cfg.E))
        return PoolMirror.tally(out)

    def _all_classes(self, st: ArrayState):
        cfg = self.cfg
        return PoolMirror.tally([PoolMirror.cls((cfg.B << b) * cfg.E) for s in st.sizes
                                 for b in range(buckets_for(s, cfg.B))])

    # -- the loop -----------------------------------------------------------
    def run(self, trace, batched: bool = True, native: bool | None = None):
        """Serve the trace.  native (default: on the GPU) runs the same rules
        in the library's native loop (gga_serve_run, include/gga_serve.h);
        otherwise this Python loop runs them (it is also the model the
        scheduling tests exercise with a fake device)."""
        if native is None:
            native = isinstance(self.be, CudaBackend)
        if native:
            return self._run_native(trace, batched)
        cfg = self.cfg
        t_arr, typ, arr, nn, tag = trace
        m = len(t_arr)
        lat = np.full(m, np.nan)
        state = np.zeros(m, dtype=np.int8)          # 0 pending, 1 done, 2 rejected
        heap = []                                   # (arrival, request): array heads ready to run
        waiting = []                                # (arrival, request): heads that are appends not fitting yet
        wait_cls = {}                               # their bucket classes (fixed while they wait)
        freed = 0                                   # counts frees of pool memory (flattens)
        t_full = math.inf                           # arrival time of the first append that did not fit
        checked = 0                                 # value of `freed` when `waiting` was last tried
        nxt = 0
        inflight = deque()                          # (event, [requests], result locations, slot)
        slot = 0
        appended = 0
        steps = batched_reqs = 0
        max_batch = cfg.max_batch if batched else 1
        t0 = time.perf_counter()

        def next_head(st):
            st.queue.popleft()
            if st.queue:
                heapq.heappush(heap, (t_arr[st.queue[0]], st.queue[0]))

        def fits(cls):
            return self.mirror.bump + self.mirror.need(cls) <= self.mirror.cap

        while True:
            now = time.perf_counter() - t0
            # Arrivals: queue per array; a request becomes a ready head when its array has nothing ahead.
            while nxt < m and t_arr[nxt] <= now:
                st = self.arrays[arr[nxt]]
                st.queue.append(nxt)
                if len(st.queue) == 1 and not st.busy:
                    heapq.heappush(heap, (t_arr[nxt], nxt))
                nxt += 1
            # Completions.
            while inflight and (inflight[0][0].query() or len(inflight) >= cfg.max_inflight):
                ev, reqs, meta, _ = inflight.popleft()
                ev.synchronize()
                done = time.perf_counter() - t0
                for r in reqs:
                    lat[r] = done - t_arr[r]
                    state[r] = 1
                    st = self.arrays[arr[r]]
                    st.busy = False
                    next_head(st)
                    if self.record and r in meta:
                        self._save(r, meta[r])
            # Appends past their deadline are rejected; their arrays move on.
            while waiting and now - waiting[0][0] > cfg.deadline:
                _, r = heapq.heappop(waiting)
                del wait_cls[r]
                state[r] = 2
                next_head(self.arrays[arr[r]])
            appends, reads, flats, taken = [], [], [], []

            def admit(r, cls):
                st = self.arrays[arr[r]]
                self.mirror.take(cls)
                n = int(nn[r])
                for l in range(cfg.L):
                    st.sizes[l] += n // cfg.L + (1 if l < n % cfg.L else 0)
                appends.append(r)
                st.busy = True
                taken.append(r)

            # Waiting appends, oldest first, once memory has been freed since they were last tried.
            if waiting and freed != checked:
                checked = freed
                keep = []
                tried = 0
                while waiting and len(taken) < max_batch and tried < self.LOOK_AHEAD:
                    item = heapq.heappop(waiting)
                    tried += 1
                    if fits(wait_cls[item[1]]):
                        admit(item[1], wait_cls.pop(item[1]))
                    else:
                        keep.append(item)
                for item in keep:
                    heapq.heappush(waiting, item)
            # Ready heads, oldest first; an append that does not fit goes to the waiting queue.
            while heap and len(taken) < max_batch:
                _, r = heapq.heappop(heap)
                st = self.arrays[arr[r]]
                if typ[r] == APPEND:
                    cls = self._append_classes(st, int(nn[r]))
                    if fits(cls):
                        admit(r, cls)
                    else:
                        wait_cls[r] = cls
                        heapq.heappush(waiting, (t_arr[r], r))
                        t_full = min(t_full, t_arr[r])
                    continue
                if typ[r] == READ:
                    reads.append(r)
                else:
                    flats.append(r)
                st.busy = True
                taken.append(r)
            if taken:
                s = self.stream
                meta = self._launch(appends, reads, flats, arr, nn, tag, slot, s)
                steps += 1
                batched_reqs += len(taken)
                freed += len(flats)
                appended += int(sum(int(nn[r]) for r in appends))
                ev = self.be.event()
                ev.record(s)
                inflight.append((ev, taken, meta, slot))
                slot = (slot + 1) % (cfg.max_inflight + 1)
                if not batched:
                    ev.synchronize()
            elif not inflight:
                if nxt >= m and not heap and not waiting:
                    break
                wait = (t_arr[nxt] - (time.perf_counter() - t0)) if nxt < m else 0.0005
                if wait > 0:
                    time.sleep(min(wait, 0.0005))
        wall = time.perf_counter() - t0
        self.latency, self.state = lat, state
        rep = self._report(lat, state, typ, nn, wall, appended)
        # The same latencies split at the first append the pool could not hold:
        # before it the server is bound by its own work, after it by memory.
        rep["pool_first_full_s"] = None if math.isinf(t_full) else round(float(t_full), 3)
        for name, sel in (("before_pool_full", t_arr < t_full), ("after_pool_full", t_arr >= t_full)):
            done = (state == 1) & sel
            if done.any():
                ms = lat[done] * 1e3
                rep[name] = {"completed": int(done.sum()), "p50_ms": round(float(np.percentile(ms, 50)), 4),
                             "p99_ms": round(float(np.percentile(ms, 99)), 4)}
        rep["steps"] = steps
        rep["mean_requests_per_step"] = round(batched_reqs / max(1, steps), 3)
        return rep

    def _run_native(self, trace, batched: bool):
        gga, cfg = self.gga, self.cfg
        t_arr, typ, arr, nn, tag = trace
        c = gga.gga_serve_config()
        c.n_arrays, c.L, c.B, c.E = cfg.n_arrays, cfg.L, cfg.B, cfg.E
        c.read_n, c.max_inflight, c.max_batch = cfg.read_n, cfg.max_inflight, cfg.max_batch
        c.batched, c.deadline_s, c.pool_bytes = 1 if batched else 0, cfg.deadline, cfg.pool_bytes

        def keep(r, ptr, n):
            data = gga.device_to_host(ptr, n * cfg.E)
            if self.record == "digest":
                self.results[r] = hashlib.sha256(data).hexdigest()
            else:
                self.results[r] = np.frombuffer(data, dtype=np.int64).copy()

        lat, state, st = gga.gga_serve_run(c, [a.g.h for a in self.arrays], t_arr, typ, arr, nn, tag,
                                           self.read_out, self.flat_arena, keep if self.record else None,
                                           self.stream)
        self.latency, self.state = lat, state
        rep = self._report(lat, state, typ, nn, st["wall_s"], st["appended_elements"])
        t_full = math.inf if st["first_full_s"] is None else st["first_full_s"]
        rep["pool_first_full_s"] = None if math.isinf(t_full) else round(float(t_full), 3)
        for name, sel in (("before_pool_full", t_arr < t_full), ("after_pool_full", t_arr >= t_full)):
            done = (state == 1) & sel
            if done.any():
                ms = lat[done] * 1e3
                rep[name] = {"completed": int(done.sum()), "p50_ms": round(float(np.percentile(ms, 50)), 4),
                             "p99_ms": round(float(np.percentile(ms, 99)), 4)}
        rep["steps"] = st["steps"]
        rep["mean_requests_per_step"] = round(st["step_requests"] / max(1, st["steps"]), 3)
        rep["scheduler"] = "native"
        return rep

    def _launch(self, appends, reads, flats, arr, nn, tag, slot, s):
        """Enqueue one step; returns where each read/flatten result lands."""
        gga = self.gga
        cfg = self.cfg
        meta = {}
        if appends:
            gga.gga_append_batch([(self.arrays[arr[r]].g, int(nn[r]), int(tag[r])) for r in appends], s)
        if reads:
            gga.gga_read_batch([(self.arrays[arr[r]].g, cfg.read_n, int(tag[r]), self.read_out[slot, j])
                                for j, r in enumerate(reads)], s)
            for j, r in enumerate(reads):
                meta[r] = ("read", slot, j)
        for r in flats:
            st = self.arrays[arr[r]]
            n = sum(st.sizes)
            dst = self._arena_take(n)
            gga.gga_flatten(st.g.h, dst, n, s)
            gga.gga_clear(st.g.h, s)
            self.mirror.give(self._all_classes(st))
            st.sizes = [0] * cfg.L
            meta[r] = ("flat", dst, n)
        return meta

    # Flatten outputs go to a device arena used round robin; a result that
    # does not fit the arena gets its own buffer.
    _arena_ptr = 0

    def _arena_take(self, n):
        cap = self.flat_arena.shape[0]
        if n + 1 > cap:
            return self.be.empty_i64(n + 1)
        if self._arena_ptr + n + 1 > cap:
            self._arena_ptr = 0
        dst = self.flat_arena[self._arena_ptr:self._arena_ptr + n + 1]
        self._arena_ptr += n + 1
        return dst

    def _save(self, r, where):
        # Test mode: keep read and flatten results (or, with record="digest",
        # the SHA-256 of their bytes) once their step completed.
        if where[0] == "read":
            _, sl, j = where
            res = self.read_out[sl, j].cpu().numpy().copy()
        else:
            _, dst, n = where
            res = dst[:n].cpu().numpy().copy()
        self.results[r] = hashlib.sha256(res.tobytes()).hexdigest() if self.record == "digest" else res

    def _report(self, lat, state, typ, nn, wall, appended):
        done = state == 1
        out = {"requests": int(len(lat)), "completed": int(done.sum()), "rejected": int((state == 2).sum()),
               "wall_s": round(wall, 3)}
        if done.any():
            ms = lat[done] * 1e3
            out["p50_ms"] = round(float(np.percentile(ms, 50)), 4)
            out["p99_ms"] = round(float(np.percentile(ms, 99)), 4)
            for name, code in (("append", APPEND), ("read", READ), ("flatten", FLATTEN)):
                sel = done & (typ == code)
                if sel.any():
                    out[f"{name}_p50_ms"] = round(float(np.percentile(lat[sel] * 1e3, 50)), 4)
                    out[f"{name}_p99_ms"] = round(float(np.percentile(lat[sel] * 1e3, 99)), 4)
        offered = typ == APPEND
        out["append_accept_rate"] = round(float((done & offered).sum() / max(1, offered.sum())), 4)
        out["appended_elements"] = appended
        out["elements_per_s"] = round(appended / wall, 1)
        return out

    def close(self):
        for st in self.arrays:
            st.g.close()
        self.pool.close()

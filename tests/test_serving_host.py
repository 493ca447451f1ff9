"""The server's scheduling on the host, with a fake device layer: requests
of one array run in arrival order, an append that does not fit the pool
waits without holding up other arrays, memory returned by a flatten admits
waiting appends, and the pool mirror never admits more than the pool."""

import numpy as np
import torch

from paper_2209_00103_gb300 import serving


class FakeEvent:
    def record(self, stream):
        pass

    def query(self):
        return True

    def synchronize(self):
        pass


class FakeGGA:
    GGA_OK = 0

    def __init__(self):
        self.calls = []            # (kind, array object id, request tags)
        self.launch_sizes = []

    class GGAPool:
        def __init__(self, nbytes, min_bucket_bytes, stream=None):
            self.nbytes = nbytes

        def close(self):
            pass

    class GGArray:
        def __init__(self, L, T, B, E, shared_pool=None, stream=None):
            self.h = self

        def last_error(self):
            return 0

        def close(self):
            pass

    def gga_append_batch(self, reqs, stream=None):
        arrays = [id(g) for g, _, _ in reqs]
        assert len(set(arrays)) == len(arrays)      # one request per array per launch
        self.launch_sizes.append(len(reqs))
        for g, n, tag in reqs:
            self.calls.append(("append", id(g), tag))

    def gga_read_batch(self, reqs, stream=None):
        self.launch_sizes.append(len(reqs))
        for g, n, seed, out in reqs:
            out.fill_(seed)
            self.calls.append(("read", id(g), seed))

    def gga_flatten(self, h, dst, n, stream=None):
        self.calls.append(("flatten", id(h), None))

    def gga_clear(self, h, stream=None):
        pass


class FakeBackend:
    def __init__(self):
        self.gga = FakeGGA()

    def stream(self):
        return None

    def event(self):
        return FakeEvent()

    def empty_i64(self, shape):
        return torch.empty(shape, dtype=torch.int64)


def small_cfg(**kw):
    base = dict(n_arrays=4, L=4, T=256, B=1024, E=8, pool_bytes=1 << 20, rate=1000.0, duration=0.1,
                max_append=1000, deadline=0.05, max_inflight=3, max_batch=8, flatten_arena_bytes=1 << 16,
                read_n=16)
    base.update(kw)
    return serving.ServeConfig(**base)


def trace_of(rows):
    t = np.array([r[0] for r in rows], dtype=np.float64)
    typ = np.array([r[1] for r in rows], dtype=np.int8)
    arr = np.array([r[2] for r in rows], dtype=np.int64)
    nn = np.array([r[3] for r in rows], dtype=np.int64)
    tag = np.arange(len(rows), dtype=np.int64) + 1
    return t, typ, arr, nn, tag


def test_waiting_append_holds_only_its_own_array():
    A, R = serving.APPEND, serving.READ
    cfg = small_cfg()
    # r0 needs 4 x (buckets to 256K elements) of 8 bytes: far above the 1 MiB pool.
    tr = trace_of([(0.0, A, 0, 1 << 20), (0.001, R, 1, 0), (0.002, R, 0, 0), (0.003, A, 2, 100)])
    srv = serving.Server(cfg, backend=FakeBackend())
    rep = srv.run(tr)
    assert list(srv.state) == [2, 1, 1, 1]                   # the huge append is rejected
    assert rep["rejected"] == 1 and rep["completed"] == 3
    assert srv.latency[1] < cfg.deadline / 2                 # another array's read is not held up
    assert srv.latency[3] < cfg.deadline / 2                 # nor another array's append
    assert srv.latency[2] >= cfg.deadline - 0.002 - 1e-3    # the read behind the append waits for it


def test_flatten_frees_memory_for_a_waiting_append():
    A, F = serving.APPEND, serving.FLATTEN
    n = 3 * 1024 * 4                                         # 3 first-bucket spans per LFVector
    cfg = small_cfg(pool_bytes=PoolBytes.for_one(n), deadline=0.5)
    tr = trace_of([(0.0, A, 0, n), (0.001, A, 1, n), (0.01, F, 0, 0)])
    srv = serving.Server(cfg, backend=FakeBackend())
    srv.run(tr)
    assert list(srv.state) == [1, 1, 1]
    assert srv.latency[1] >= 0.009                           # admitted only after the flatten
    assert srv.mirror.bump <= cfg.pool_bytes


class PoolBytes:
    @staticmethod
    def for_one(n, L=4, B=1024, E=8):
        m = serving.PoolMirror(1 << 40)
        st = serving.ArrayState(None, L)
        cls = []
        for l in range(L):
            c = n // L + (1 if l < n % L else 0)
            for b in range(serving.buckets_for(0, B), serving.buckets_for(c, B)):
                cls.append(serving.PoolMirror.cls((B << b) * E))
        return m.need(serving.PoolMirror.tally(cls))


def test_random_trace_invariants():
    cfg = small_cfg(n_arrays=16, pool_bytes=4 << 20, rate=4000.0, duration=0.15, max_append=100000,
                    deadline=0.02, max_batch=6)
    tr = serving.make_trace(cfg)
    be = FakeBackend()
    srv = serving.Server(cfg, backend=be)
    rep = srv.run(tr)
    t, typ, arr, nn, tag = tr
    assert rep["completed"] + rep["rejected"] == len(t)
    assert np.all(typ[srv.state == 2] == serving.APPEND)      # only appends are ever rejected
    assert rep["rejected"] > 0
    assert max(be.gga.launch_sizes) <= cfg.max_batch
    assert srv.mirror.bump <= cfg.pool_bytes
    # Per array, requests reached the device in arrival order.
    ids = {id(st.g): a for a, st in enumerate(srv.arrays)}
    last = {}
    for kind, g, tg in be.gga.calls:
        if tg is None:
            continue
        a = ids[g]
        assert tg > last.get(a, 0)
        last[a] = tg


def test_pool_mirror_uses_free_buckets_first():
    m = serving.PoolMirror(1 << 20)
    t = serving.PoolMirror.tally([13, 13, 14, 8])
    assert t == {13: 2, 14: 1, 8: 1}
    assert m.need(t) == 2 * 8192 + 16384 + 256
    m.take(t)
    assert m.bump == 2 * 8192 + 16384 + 256
    m.give({13: 1, 14: 1})
    assert m.need(t) == 8192 + 256                    # one class-13 and the class-8 bucket from the bump
    m.take(t)
    assert m.free[13] == 0 and m.free[14] == 0
    assert m.bump == 2 * (2 * 8192 + 16384 + 256) - (8192 + 16384)

"""Serving many live arrays: batched appends and random reads against the
oracle, and the continuous-batching server: every request's result is the
same when it runs in a mix (batched) and alone (one request per launch),
and both equal the oracle's replay of the requests in arrival order."""

import numpy as np
import pytest
import torch

import oracle
from paper_2209_00103_gb300 import gga, serving

import oracle_pool
from harness import assert_same_state, dev_to_np

pytestmark = pytest.mark.gpu


def test_append_and_read_batches_match_oracle():
    rng = np.random.default_rng(83)
    pool = gga.GGAPool(512 << 20, 1024 * 4)
    shapes = [(int(rng.choice([1, 2, 4, 7])), 256, 1024, int(rng.choice([4, 8, 16]))) for _ in range(20)]
    arrays = [gga.GGArray(L, T, B, E, shared_pool=pool) for (L, T, B, E) in shapes]
    refs = [oracle.OracleGGArray(L, T, B, E) for (L, T, B, E) in shapes]
    tag = 1
    for step in range(6):
        picks = rng.choice(len(arrays), size=8, replace=False)
        reqs = []
        for a in picks:
            n = int(rng.choice([0, 1, 5, 1000, 70000]))
            reqs.append((arrays[a], n, tag))
            refs[a].append(n, tag)
            tag += 1
        gga.gga_append_batch(reqs)
        reads = []
        for a in rng.choice(len(arrays), size=6, replace=False):
            out = gga.elem_tensor(4096, shapes[a][3])
            reads.append((arrays[a], 4096, 1000 + step * 10 + int(a), out, a))
        gga.gga_read_batch([(g, n, seed, out) for g, n, seed, out, _ in reads])
        for g, n, seed, out, a in reads:
            assert dev_to_np(out, shapes[a][3]).tobytes() == refs[a].read_random(n, seed).tobytes()
    for g, o in zip(arrays, refs):
        assert_same_state(g, o)
    with pytest.raises(gga.GGAError):                     # one request per array per launch
        gga.gga_append_batch([(arrays[0], 1, 1), (arrays[0], 1, 2)])
    for g in arrays:
        g.close()
    pool.close()


def test_append_batch_over_many_lfvectors_splits_launches():
    # 12 arrays of 1024 LFVectors: more (request, LFVector) pairs than one
    # launch's reservation records, so the batch runs as several launches.
    pool = gga.GGAPool(256 << 20, 256 * 4)
    shapes = [(1024, 32, 256, (4, 8, 16)[a % 3]) for a in range(12)]
    arrays = [gga.GGArray(L, T, B, E, shared_pool=pool) for (L, T, B, E) in shapes]
    refs = [oracle.OracleGGArray(L, T, B, E) for (L, T, B, E) in shapes]
    for step, ns in enumerate([[3000 + 977 * a for a in range(12)], [1024 * 40 + 5] * 12, [1, 0, 2047] * 4]):
        gga.gga_append_batch([(g, n, 100 * step + a + 1) for a, (g, n) in enumerate(zip(arrays, ns))])
        for a, (o, n) in enumerate(zip(refs, ns)):
            o.append(n, 100 * step + a + 1)
    for g, o in zip(arrays, refs):
        assert_same_state(g, o)
        assert g.last_error() == gga.GGA_OK
    for g in arrays:
        g.close()
    pool.close()


def small_cfg(**kw):
    base = dict(n_arrays=64, L=4, T=256, B=1024, E=8, pool_bytes=2 << 30, rate=20000.0, duration=0.25,
                max_append=50000, deadline=1.0, max_inflight=3, max_batch=480, flatten_arena_bytes=1 << 30)
    base.update(kw)
    return serving.ServeConfig(**base)


def replay_oracle(cfg, trace, state):
    t, typ, arr, nn, tag = trace
    refs = [oracle.OracleGGArray(cfg.L, cfg.T, cfg.B, cfg.E) for _ in range(cfg.n_arrays)]
    out = {}
    for r in range(len(t)):
        if state is not None and state[r] != 1:
            continue
        o = refs[arr[r]]
        if typ[r] == serving.APPEND:
            o.append(int(nn[r]), int(tag[r]))
        elif typ[r] == serving.READ:
            out[r] = o.read_random(cfg.read_n, int(tag[r]))
        else:
            out[r] = o.flatten().copy()
            refs[arr[r]] = oracle.OracleGGArray(cfg.L, cfg.T, cfg.B, cfg.E)   # retired
    return out


@pytest.mark.parametrize("native", [True, False])
def test_server_mix_equals_alone_equals_oracle(native):
    # native: the library's scheduling loop (gga_serve_run); otherwise the
    # Python loop of serving.py, the same rules.
    cfg = small_cfg()
    trace = serving.make_trace(cfg)
    mixed = serving.Server(cfg, record=True)
    rep_mix = mixed.run(trace, batched=True, native=native)
    res_mix = mixed.results
    mixed.close()
    alone = serving.Server(cfg, record=True)
    rep_alone = alone.run(trace, batched=False, native=native)
    res_alone = alone.results
    alone.close()
    assert rep_mix["rejected"] == 0 and rep_alone["rejected"] == 0
    assert rep_mix["completed"] == len(trace[0]) == rep_alone["completed"]
    want = replay_oracle(cfg, trace, None)
    assert set(res_mix) == set(res_alone) == set(want)
    for r in want:
        assert res_mix[r].tobytes() == want[r].view(np.int64).tobytes(), r
        assert res_alone[r].tobytes() == res_mix[r].tobytes(), r


def test_server_admission_under_a_full_pool():
    # A pool far too small for the offered appends: appends wait, then some
    # are rejected at the deadline; admitted ones never fail on the device.
    cfg = small_cfg(pool_bytes=48 << 20, duration=0.2, deadline=0.02, max_append=200000)
    trace = serving.make_trace(cfg)
    srv = serving.Server(cfg)
    rep = srv.run(trace, batched=True)
    assert rep["rejected"] > 0
    assert rep["completed"] + rep["rejected"] == len(trace[0])
    assert all(st.g.last_error() == gga.GGA_OK for st in srv.arrays)
    info = srv.pool.info()
    assert info["bump_bytes"] <= cfg.pool_bytes
    srv.close()


def test_full_served_configuration_past_the_pool_filling_matches_oracle():
    # 7.5 s of the full configuration (65,536 int64 arrays, a 64 GiB pool,
    # 20k requests/s), which crosses the first moment the pool is full:
    # through the batched server and through the plain form, every read and
    # flatten of every array touched equals the oracle's replay of that
    # array's admitted requests in arrival order (compared as SHA-256 of the
    # results' bytes; the oracle replays one array at a time in spawned
    # workers).  Admission differs between the runs once the pool is full
    # (deadlines), so each run is checked against its own admitted set, and
    # the two runs agree on every request whose array had the same admitted
    # history in both.
    cfg = serving.ServeConfig(duration=7.5)
    trace = serving.make_trace(cfg)
    t, typ, arr, nn, tag = trace
    runs = {}
    for name, batched in (("mix", True), ("alone", False)):
        srv = serving.Server(cfg, record="digest")
        rep = srv.run(trace, batched=batched)
        assert rep["completed"] + rep["rejected"] == len(t)
        assert all(st.g.last_error() == gga.GGA_OK for st in srv.arrays[:64])
        runs[name] = (rep, srv.state.copy(), dict(srv.results))
        srv.close()
    rep_mix = runs["mix"][0]
    assert rep_mix["pool_first_full_s"] is not None and rep_mix["rejected"] > 0   # the pool did fill
    for name, (rep, state, res) in runs.items():
        done = state == 1
        want = oracle_pool.served_digests(cfg.L, cfg.T, cfg.B, cfg.E, cfg.read_n, typ, arr, nn, tag, done)
        assert set(res) == set(want), name
        bad = [r for r in want if res[r] != want[r]]
        assert not bad, (name, bad[:5])
        assert len(set(arr[done])) > 20000
    # Same admitted history of an array up to a request => same result.
    s_mix, s_alone = runs["mix"][1], runs["alone"][1]
    order = np.argsort(arr, kind="stable")                     # per array, in arrival order
    sa = arr[order]
    mis = (s_mix[order] != s_alone[order]).astype(np.int64)
    cm = np.cumsum(mis)
    starts = np.flatnonzero(np.concatenate([[True], sa[1:] != sa[:-1]]))
    before = np.repeat(cm[starts] - mis[starts], np.diff(np.append(starts, len(sa))))
    agree = order[cm - before == 0]                            # no disagreement so far in its array
    same = 0
    for r in agree:
        if typ[r] != serving.APPEND and s_mix[r] == 1:
            assert runs["mix"][2][r] == runs["alone"][2][r], r
            same += 1
    assert same > 1000

"""GPU parity of the device API (include/gga_device.cuh): a user's kernels,
built against the public header alone, push into a GGArray with
gga::block_push_back (Algorithm 1: prefix sum over the block's threads, one
reservation per block, buckets of Algorithm 2 from the device pool), then
gga_device_commit; the array must equal the oracle's after the same rounds,
bit for bit, and the library's calls must carry on from it.  Also the
generated insertion written as such a kernel (gga_push_generated)."""

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2209_00103_gb300 import gga
from paper_2209_00103_gb300 import workloads as wl

from harness import assert_same_state, counts_to_dev, dev_to_np, insert_both, make_pair, packed_values, values_to_dev
from user_kernel import load_user

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield
    torch.cuda.synchronize()


@pytest.fixture(scope="module")
def user():
    return load_user()


def stream_ptr():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def padded_rounds(rng, R, L, NT, kmax, E, seed):
    """counts [R][L][NT] in 0..kmax and values [R][L][NT][kmax] (unique), with
    the packed (round, LFVector, thread, k) order gga_insert and the oracle take."""
    counts = rng.integers(0, kmax + 1, size=(R, L, NT)).astype(np.uint32)
    n = R * L * NT * kmax
    vals = wl.encode_values(wl.splitmix_at(seed, np.arange(n, dtype=np.uint64)), E)
    keep = (np.arange(kmax)[None, None, None, :] < counts[..., None]).reshape(-1)
    return counts, vals, vals[keep]


def expected_first(counts, size0):
    """First LFVector-local index of every (round, LFVector, thread) run: the
    LFVector's size before the round plus the counts of the lower threads."""
    R, L, NT = counts.shape
    c = counts.astype(np.int64)
    before = size0[None, :] + np.concatenate([np.zeros((1, L), np.int64), np.cumsum(c.sum(axis=2), axis=0)[:-1]])
    return before[..., None] + np.cumsum(c, axis=2) - c


# Forms of the device API a user kernel pushes through: 0 block_push_back per
# round, 1 a BlockPusher, 2 a BlockPusher with a shared-memory stage (staged
# 128-bit writes), 3 block_push_rounds, 4 rounds per call, staged, 4
# block_push_rounds, 3 rounds per call, unstaged.
FORMS = [0, 1, 2, 3, 4]
STAGE_BYTES = 8192   # small enough that large pushes take the unstaged path


def push(user, g, counts, vals, bx, by, kmax, blocks=None, reverse=0, stop_on_fail=1, cursor=0):
    """The rounds through the device-API form `cursor` (FORMS)."""
    R, L, NT = counts.shape
    assert bx * by == NT and vals.shape[0] == R * L * NT * kmax
    cd = counts_to_dev(counts)
    vd = values_to_dev(vals, g.E)
    first = torch.empty(R * L * NT, dtype=torch.int64, device="cuda")
    args = (ctypes.c_void_p(g.device_view()), ctypes.c_void_p(cd.data_ptr()), ctypes.c_void_p(vd.data_ptr()),
            ctypes.c_void_p(first.data_ptr()), R, L, bx, by, kmax, g.E, blocks or L, reverse, stop_on_fail)
    if int(cursor) >= 2:
        rc = user.user_push_rounds_mode(*args, int(cursor), STAGE_BYTES, stream_ptr())
    else:
        fn = user.user_push_rounds_cursor if cursor else user.user_push_rounds
        rc = fn(*args, stream_ptr())
    assert rc == 0
    g.device_commit()
    return first.cpu().numpy().view(np.uint64).reshape(R, L, NT)


@pytest.mark.parametrize("cursor", FORMS)
@pytest.mark.parametrize("E", [4, 8, 16])
@pytest.mark.parametrize("bx,by", [(128, 1), (100, 1), (16, 6), (1, 1), (1024, 1), (8, 4), (33, 31)])
def test_user_kernel_pushes_match_oracle(user, E, bx, by, cursor):
    rng = np.random.default_rng(100 * E + bx + by)
    L, B, kmax = 7, 8, 3
    NT = bx * by
    g, o = make_pair(L, NT, B, E, pool_bytes=64 << 20)
    for step, R in enumerate((9, 1, 4)):
        size0 = o.sizes().astype(np.int64)
        counts, vals, packed = padded_rounds(rng, R, L, NT, kmax, E, seed=1000 * step + E)
        first = push(user, g, counts, vals, bx, by, kmax, cursor=cursor)
        o.insert(counts, packed)
        assert g.last_error() == gga.GGA_OK
        assert_same_state(g, o)
        want = expected_first(counts, size0)
        has = counts > 0
        assert np.array_equal(first[has].astype(np.int64), want[has])
    g.close()
    o.close()


def test_device_pushes_and_library_insertions_interleave(user):
    # User-kernel pushes, gga_insert, gga_insert_generated and pushes again:
    # each continues where the last left off.
    rng = np.random.default_rng(5)
    L, T, B, E, kmax = 13, 96, 16, 4, 2
    g, o = make_pair(L, T, B, E, pool_bytes=64 << 20)
    counts, vals, packed = padded_rounds(rng, 6, L, T, kmax, E, seed=1)
    push(user, g, counts, vals, T, 1, kmax)
    o.insert(counts, packed)
    c2 = rng.integers(0, 3, size=(5, L, T)).astype(np.uint32)
    insert_both(g, o, c2, packed_values(int(c2.sum()), E, seed=2), E)
    g.insert_generated(gga.make_gen_spec(3, "uniform3", (10, 1 << 20, 1)), 4)
    o.insert_generated(3, "uniform3", (10, 1 << 20, 1), 0, 4)
    counts, vals, packed = padded_rounds(rng, 3, L, T, kmax, E, seed=4)
    push(user, g, counts, vals, 32, 3, kmax)
    o.insert(counts, packed)
    counts, vals, packed = padded_rounds(rng, 5, L, T, kmax, E, seed=5)
    push(user, g, counts, vals, 96, 1, kmax, cursor=True)
    o.insert(counts, packed)
    assert g.last_error() == gga.GGA_OK
    assert_same_state(g, o)
    g.close()


@pytest.mark.parametrize("cursor", FORMS)
def test_grid_stride_blocks_and_reversed_lfvectors(user, cursor):
    # Fewer blocks than LFVectors, each block serving several in reverse
    # (with cursors: one after another on the same shared slots).
    rng = np.random.default_rng(6)
    L, T, B, E, kmax = 50, 64, 4, 8, 4
    g, o = make_pair(L, T, B, E, pool_bytes=64 << 20)
    counts, vals, packed = padded_rounds(rng, 5, L, T, kmax, E, seed=6)
    first = push(user, g, counts, vals, T, 1, kmax, blocks=7, reverse=1, cursor=cursor)
    o.insert(counts, packed)
    assert g.last_error() == gga.GGA_OK
    assert_same_state(g, o)
    has = counts > 0
    assert np.array_equal(first[has].astype(np.int64), expected_first(counts, np.zeros(L, np.int64))[has])
    g.close()


def test_short_form_pushes_into_the_blocks_own_lfvector(user):
    rng = np.random.default_rng(7)
    L, T, B, E, kmax = 9, 160, 8, 4, 3
    g, o = make_pair(L, T, B, E, pool_bytes=64 << 20)
    counts, vals, packed = padded_rounds(rng, 1, L, T, kmax, E, seed=7)
    cd, vd = counts_to_dev(counts), values_to_dev(vals, E)
    assert user.user_push_own(ctypes.c_void_p(g.device_view()), ctypes.c_void_p(cd.data_ptr()),
                              ctypes.c_void_p(vd.data_ptr()), L, T, kmax, stream_ptr()) == 0
    g.device_commit()
    o.insert(counts, packed)
    assert_same_state(g, o)
    g.close()


@pytest.mark.parametrize("E", [4, 8, 16])
def test_device_reads_by_global_and_local_index(user, E):
    rng = np.random.default_rng(8 + E)
    L, T, B, kmax = 21, 128, 8, 3
    g, o = make_pair(L, T, B, E, pool_bytes=64 << 20)
    counts, vals, packed = padded_rounds(rng, 7, L, T, kmax, E, seed=8)
    push(user, g, counts, vals, T, 1, kmax)
    o.insert(counts, packed)
    N = o.size()
    idx = np.concatenate([wl.uniform_indices(9, 4000, N), np.array([0, N - 1], np.uint64)])
    idx_d = torch.from_numpy(idx.view(np.int64)).cuda()
    out = gga.elem_tensor(idx.size, E)
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert user.user_read_global(ctypes.c_void_p(g.device_view()), ctypes.c_void_p(idx_d.data_ptr()), idx.size,
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(n_out.data_ptr()), E,
                                 stream_ptr()) == 0
    want, rc = o.read(idx)
    assert rc == oracle.OK
    assert int(n_out.item()) == N
    assert dev_to_np(out, E).tobytes() == want.tobytes()
    # LFVector-local: element j of LFVector l is global offsets[l] + j.
    sizes, offs = o.sizes().astype(np.int64), o.offsets().astype(np.int64)
    ls = rng.integers(0, L, size=3000)
    ls = ls[sizes[ls] > 0]
    js = (rng.random(ls.size) * sizes[ls]).astype(np.int64)
    l_d = torch.from_numpy(ls.astype(np.int32)).cuda()
    j_d = torch.from_numpy(js).cuda()
    out = gga.elem_tensor(ls.size, E)
    sz = torch.empty(ls.size, dtype=torch.int64, device="cuda")
    assert user.user_read_local(ctypes.c_void_p(g.device_view()), ctypes.c_void_p(l_d.data_ptr()),
                                ctypes.c_void_p(j_d.data_ptr()), ls.size, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(sz.data_ptr()), E, stream_ptr()) == 0
    want, rc = o.read((offs[ls] + js).astype(np.uint64))
    assert dev_to_np(out, E).tobytes() == want.tobytes()
    assert np.array_equal(sz.cpu().numpy(), sizes[ls])
    g.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_rejected_pushes_latch_invalid_and_change_nothing(user, mode):
    rng = np.random.default_rng(10)
    L, T, B, E, kmax = 3, 64, 8, 4, 2
    g, o = make_pair(L, T, B, E, pool_bytes=16 << 20)
    counts, vals, packed = padded_rounds(rng, 2, L, T, kmax, E, seed=10)
    push(user, g, counts, vals, T, 1, kmax)
    o.insert(counts, packed)
    ok = torch.full((2,), 9, dtype=torch.int32, device="cuda")
    assert user.user_push_rejected(ctypes.c_void_p(g.device_view()), mode, ctypes.c_void_p(ok.data_ptr()),
                                   stream_ptr()) == 0
    g.device_commit()
    assert ok.tolist() == [0, 0]
    assert g.last_error() == gga.GGA_ERR_INVALID
    assert g.last_error() == gga.GGA_OK   # read and cleared
    assert_same_state(g, o)
    g.close()


def round_chunks(counts, packed, l):
    """Values LFVector l receives in each round, in push order."""
    R, L, NT = counts.shape
    tot = counts.astype(np.int64).reshape(R * L, NT).sum(axis=1)
    start = np.concatenate([[0], np.cumsum(tot)])
    return [packed[start[r * L + l]:start[r * L + l + 1]] for r in range(R)]


@pytest.mark.parametrize("cursor", FORMS)
@pytest.mark.parametrize("stop_on_fail", [1, 0])
def test_pool_exhaustion_keeps_whole_rounds(user, stop_on_fail, cursor):
    # A pool too small for every LFVector: a block whose buckets do not fit
    # pushes nothing that round and latches POOL_EXHAUSTED; each LFVector holds
    # whole rounds in order (a prefix of them when the kernel stops there).
    rng = np.random.default_rng(11)
    L, T, B, E, kmax = 16, 64, 16, 4, 3
    g = gga.GGArray(L, T, B, E, 96 << 10)
    counts, vals, packed = padded_rounds(rng, 12, L, T, kmax, E, seed=11)
    push(user, g, counts, vals, T, 1, kmax, stop_on_fail=stop_on_fail, cursor=cursor)
    n, rc, sizes, caps = g.sizes_caps()
    assert rc == gga.GGA_ERR_POOL_EXHAUSTED
    sizes, caps = sizes.cpu().numpy(), caps.cpu().numpy()
    assert np.all(caps >= sizes)
    flat = dev_to_np(g.flatten(), E)[:n]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    assert n == offs[-1]
    lost = 0
    for l in range(L):
        got = flat[offs[l]:offs[l + 1]]
        pos, missed = 0, False
        for chunk in round_chunks(counts, packed, l):
            if chunk.size == 0:
                continue
            if pos + chunk.size <= got.size and got[pos:pos + chunk.size].tobytes() == chunk.tobytes():
                assert not (stop_on_fail and missed), l   # the block stopped at its first failure
                pos += chunk.size
            else:
                missed = True
                lost += 1
        assert pos == got.size, l
    assert lost > 0
    g.close()


# ---------------------------------------------------------------------------
# gga_push_generated: gga_insert_generated as a per-round device-API kernel.

@pytest.mark.parametrize("E", [4, 8, 16])
@pytest.mark.parametrize("dist", ["bernoulli", "uniform3", "geometric", "poisson"])
def test_push_generated_matches_oracle(dist, E):
    L, T, B = 11, 96, 8
    thr = wl.poisson1_thresholds()
    coeffs = (10, 1 << 20, 1 << 19)
    g, o = make_pair(L, T, B, E, pool_bytes=64 << 20)
    for round0, R in [(0, 5), (5, 12), (17, 1)]:
        spec = gga.make_gen_spec(99, dist, coeffs, round0=round0, thresholds=thr if dist == "poisson" else None)
        g.push_generated(spec, R)
        o.insert_generated(99, dist, coeffs, round0, R, thresholds=thr)
        assert g.last_error() == gga.GGA_OK
        assert_same_state(g, o)
    g.close()


def test_push_generated_equals_batched_insert_at_the_paper_growth_size():
    # 1024 blocks x 512 threads, 512 rounds of Uniform{0,1,2} (2^28 elements
    # expected): the per-round device-API kernel and the batched-round kernel
    # build the same array.
    w = wl.paper_growth()
    spec = gga.make_gen_spec(w.spec.seed, w.spec.dist, w.spec.coeffs)
    pool = int(2.2 * (1 << 28) * w.E) + (64 << 20)
    a = gga.GGArray(w.L, w.T, w.B, w.E, pool)
    a.push_generated(spec, w.spec.rounds)
    na, rca, sa, ca = a.sizes_caps()
    assert rca == gga.GGA_OK
    fa = a.flatten()
    a.close()
    b = gga.GGArray(w.L, w.T, w.B, w.E, pool)
    b.insert_generated(spec, w.spec.rounds)
    nb, rcb, sb, cb = b.sizes_caps()
    assert rcb == gga.GGA_OK and nb == na
    assert torch.equal(sa, sb) and torch.equal(ca, cb)
    assert torch.equal(fa[:na], b.flatten()[:nb])
    b.close()


def test_user_pushes_and_commit_replay_from_a_cuda_graph(user):
    # The user kernel and gga_device_commit captured once in a CUDA graph
    # (no host step between them) and replayed: every replay appends the same
    # rounds again, as that many insertions of them would.
    rng = np.random.default_rng(12)
    L, T, B, E, kmax = 24, 128, 16, 4, 3
    g, o = make_pair(L, T, B, E, pool_bytes=64 << 20)
    counts, vals, packed = padded_rounds(rng, 4, L, T, kmax, E, seed=12)
    cd, vd = counts_to_dev(counts), values_to_dev(vals, E)
    first = torch.empty(counts.size, dtype=torch.int64, device="cuda")
    view = g.device_view()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        rc = user.user_push_rounds(ctypes.c_void_p(view), ctypes.c_void_p(cd.data_ptr()),
                                   ctypes.c_void_p(vd.data_ptr()), ctypes.c_void_p(first.data_ptr()), 4, L, T, 1,
                                   kmax, E, L, 0, 1, ctypes.c_void_p(s.cuda_stream))
        g.device_commit(stream=s)
    assert rc == 0
    torch.cuda.synchronize()
    assert g.size()[0] == 0   # capture ran nothing
    for rep in range(3):
        graph.replay()
        torch.cuda.synchronize()
        o.insert(counts, packed)
        assert g.last_error() == gga.GGA_OK
        assert_same_state(g, o)
    g.close()


def test_push_generated_pool_exhaustion_keeps_whole_leading_rounds():
    # A pool too small for the rounds: each LFVector keeps the rounds before
    # its first failing one (the oracle, run round by round, gives the round
    # boundaries) and GGA_ERR_POOL_EXHAUSTED is latched.
    L, T, B, E, R = 12, 64, 16, 4, 20
    coeffs = (10, 1 << 20, 1 << 19)
    o = oracle.OracleGGArray(L, T, B, E)
    bounds = [np.zeros(L, np.int64)]
    for r in range(R):
        o.insert_generated(7, "uniform3", coeffs, r, 1)
        bounds.append(o.sizes().astype(np.int64))
    full = o.flatten()
    offs = o.offsets().astype(np.int64)
    g = gga.GGArray(L, T, B, E, 48 << 10)
    g.push_generated(gga.make_gen_spec(7, "uniform3", coeffs), R)
    n, rc, sizes, caps = g.sizes_caps()
    assert rc == gga.GGA_ERR_POOL_EXHAUSTED
    sizes = sizes.cpu().numpy()
    assert np.all(sizes <= caps.cpu().numpy())
    flat = dev_to_np(g.flatten(), E)[:n]
    got_offs = np.concatenate([[0], np.cumsum(sizes)])
    short = 0
    for l in range(L):
        kept = [int(b[l]) for b in bounds]
        assert int(sizes[l]) in kept, l                       # whole rounds only
        want = full[offs[l]:offs[l] + sizes[l]]
        assert flat[got_offs[l]:got_offs[l + 1]].tobytes() == want.tobytes(), l
        short += int(sizes[l]) < kept[-1]
    assert short > 0
    g.close()


@pytest.mark.parametrize("cursor", [False, True])
def test_counts_too_large_for_32_bit_scans(user, cursor):
    # One thread pushes 2^26 + 3 elements in a round (its warp's and the
    # block's sums need 64-bit scans), crossing many buckets in its own run;
    # the other threads push a few.  Values are a formula of (r, l, t, k).
    L, T, B, E, R = 2, 64, 1024, 8, 2
    counts = np.zeros((R, L, T), dtype=np.uint32)
    counts[0, 0, 5] = (1 << 26) + 3
    counts[0, 0, 40] = 7
    counts[0, 1, :] = 1
    counts[1, 0, :] = 2
    counts[1, 1, 63] = 1 << 20
    rr, ll, tt = np.nonzero(counts >= 0)
    c = counts.reshape(-1).astype(np.int64)
    starts = np.repeat(np.cumsum(c) - c, c)
    k = np.arange(int(c.sum()), dtype=np.int64) - starts
    head = ((rr.astype(np.uint64) << np.uint64(56)) | (ll.astype(np.uint64) << np.uint64(48))
            | (tt.astype(np.uint64) << np.uint64(32)))
    packed = np.repeat(head, c) | k.astype(np.uint64)
    g = gga.GGArray(L, T, B, E, 3 << 30)
    o = oracle.OracleGGArray(L, T, B, E)
    cd = counts_to_dev(counts)
    assert user.user_push_formula(ctypes.c_void_p(g.device_view()), ctypes.c_void_p(cd.data_ptr()), R, L, T,
                                  1 if cursor else 0, stream_ptr()) == 0
    g.device_commit()
    o.insert(counts, packed)
    assert g.last_error() == gga.GGA_OK
    assert_same_state(g, o)
    g.close()
    o.close()


def test_pushes_into_arrays_of_one_shared_pool_reuse_cleared_buckets(user):
    # Two arrays of one pool pushed from user kernels; A is cleared (its
    # buckets go to the pool's queues) and B's next pushes take them.  The
    # commits fold the queue pops; both arrays match their oracles, and the
    # pool hands out no new slab bytes for B's second growth while A's
    # queued buckets cover it.
    rng = np.random.default_rng(13)
    T, B, E, kmax = 64, 16, 4, 3
    pool = gga.GGAPool(64 << 20, B * E)
    a = gga.GGArray(10, T, B, E, shared_pool=pool)
    b = gga.GGArray(10, T, B, E, shared_pool=pool)
    oa, ob = oracle.OracleGGArray(10, T, B, E), oracle.OracleGGArray(10, T, B, E)
    ca, va, pa = padded_rounds(rng, 6, 10, T, kmax, E, seed=30)
    cb, vb, pb = padded_rounds(rng, 2, 10, T, kmax, E, seed=31)
    push(user, a, ca, va, T, 1, kmax, cursor=True)
    oa.insert(ca, pa)
    push(user, b, cb, vb, T, 1, kmax)
    ob.insert(cb, pb)
    assert_same_state(a, oa)
    assert_same_state(b, ob)
    bump_before = pool.info()["bump_bytes"]
    a.clear()
    oa.close()
    cb2, vb2, pb2 = padded_rounds(rng, 4, 10, T, kmax, E, seed=32)
    push(user, b, cb2, vb2, T, 1, kmax, cursor=True)
    ob.insert(cb2, pb2)
    assert b.last_error() == gga.GGA_OK
    assert_same_state(b, ob)
    assert pool.info()["bump_bytes"] == bump_before
    b.close()
    a.close()
    pool.close()


# ---------------------------------------------------------------------------
# gga_push_expand: values read from device memory, pushed K rounds per call
# through gga::block_push_rounds (staged, 128-bit stores).

def expand_case(L, T, E, R, seed, dist="uniform3", round0=0):
    spec = wl.InsertSpec(L=L, T=T, E=E, seed=seed, dist=dist, rounds=R, round0=round0,
                         coeffs=(7, 1 << 20, 0), thresholds=wl.poisson1_thresholds() if dist == "poisson" else None)
    counts = spec.counts()
    inputs = wl.expand_inputs(spec)
    packed = spec.values(counts)   # the inputs repeated count times (vc = 0)
    return counts, inputs, packed


@pytest.mark.parametrize("E", [4, 8, 16])
@pytest.mark.parametrize("T", [96, 300, 512])
def test_push_expand_matches_oracle(T, E):
    L, B = 13, 16
    g, o = make_pair(L, T, B, E, pool_bytes=128 << 20)
    for step, (R, dist) in enumerate([(11, "uniform3"), (1, "geometric"), (6, "poisson"), (17, "bernoulli")]):
        counts, inputs, packed = expand_case(L, T, E, R, seed=40 + step, dist=dist, round0=3 * step)
        g.push_expand(counts_to_dev(counts), values_to_dev(inputs, E).reshape(
            (R, L, T) + ((2,) if E == 16 else ())))
        o.insert(counts, packed)
        assert g.last_error() == gga.GGA_OK
        assert_same_state(g, o)
    g.close()
    o.close()


def test_push_expand_pool_exhaustion_keeps_whole_leading_rounds():
    # A pool too small: each LFVector keeps a prefix of whole rounds (the
    # longest that fits in the call that failed) and stops there.
    L, T, B, E, R = 16, 64, 16, 4, 24
    counts, inputs, packed = expand_case(L, T, E, R, seed=9)
    g = gga.GGArray(L, T, B, E, 64 << 10)
    g.push_expand(counts_to_dev(counts), values_to_dev(inputs, E).reshape(R, L, T))
    n, rc, sizes, caps = g.sizes_caps()
    assert rc == gga.GGA_ERR_POOL_EXHAUSTED
    sizes = sizes.cpu().numpy().astype(np.int64)
    flat = dev_to_np(g.flatten(), E)[:n]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    per_round = counts.sum(axis=2).astype(np.int64)            # [R][L]
    starts = np.concatenate([[0], np.cumsum(counts.reshape(-1).astype(np.int64))])
    short = 0
    for l in range(L):
        cum = np.concatenate([[0], np.cumsum(per_round[:, l])])
        kept = int(np.searchsorted(cum, sizes[l]))
        assert cum[kept] == sizes[l], l                         # whole rounds only
        want = b"".join(packed[starts[r * L * T + l * T]:starts[r * L * T + (l + 1) * T]].tobytes()
                        for r in range(kept))
        assert flat[offs[l]:offs[l + 1]].tobytes() == want, l
        short += kept < R
    assert short > 0
    g.close()


def test_push_expand_full_paper_size():
    # The paper-shaped workload (1024 x 512, B = 4096, 512 rounds of
    # Uniform{0,1,2}) through the memory-sourced device-API pushes, in the
    # launch configuration bench.py times, against the oracle.
    w = wl.paper_growth()
    spec = wl.InsertSpec(L=w.L, T=w.T, E=w.E, seed=w.spec.seed, dist=w.spec.dist, rounds=w.spec.rounds,
                         coeffs=(w.spec.coeffs[0], w.spec.coeffs[1], 0))
    dev = torch.device("cuda", 0)
    counts_t, values_t = wl.make_insert_inputs_t(spec, dev)
    inputs_t = wl.expand_inputs_t(spec, dev)
    N = int(values_t.shape[0])
    g = gga.GGArray(w.L, w.T, w.B, w.E, 3 << 30)
    g.push_expand(counts_t, inputs_t)
    n, rc = g.size()
    assert rc == gga.GGA_OK and n == N
    o = oracle.OracleGGArray(w.L, w.T, w.B, w.E)
    o.insert(counts_t.cpu().numpy().view(np.uint32), values_t.cpu().numpy().view(np.uint32))
    del counts_t, values_t, inputs_t
    assert_same_state(g, o)
    g.close()
    o.close()

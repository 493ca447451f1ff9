"""Thin ctypes binding of the C ABI in include/gga.h.

Argument marshalling only: every operation runs in the CUDA kernels of
libgga.so.  Tensors are passed as raw device pointers (``data_ptr()``) and
streams as their ``cuda_stream`` handle; PyTorch serves only as the device
memory and stream provider.  If libgga.so is missing or fails to load, the
import raises -- there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

GGA_OK = 0
GGA_ERR_INVALID = 1
GGA_ERR_POOL_EXHAUSTED = 2
GGA_ERR_OUT_OF_RANGE = 3
GGA_ERR_DST_TOO_SMALL = 4
GGA_ERR_CUDA = 5
GGA_ERR_TIMEOUT = 6
GGA_ERR_TOO_LARGE = 7
ERROR_NAMES = {0: "OK", 1: "INVALID", 2: "POOL_EXHAUSTED", 3: "OUT_OF_RANGE",
               4: "DST_TOO_SMALL", 5: "CUDA", 6: "TIMEOUT", 7: "TOO_LARGE"}

GGA_RW_G = 0
GGA_RW_B = 1
DIST = {"bernoulli": 0, "uniform3": 1, "geometric": 2, "poisson": 3}
MAX_THRESHOLDS = 16

# Every symbol include/gga.h declares.
EXPORTED = ["gga_create", "gga_insert", "gga_insert_noalloc", "gga_reserve", "gga_insert_generated",
            "gga_device_view", "gga_device_commit", "gga_push_generated", "gga_push_expand", "gga_read", "gga_write", "gga_sweep",
            "gga_flatten", "gga_size", "gga_offsets", "gga_clear", "gga_memory", "gga_last_error",
            "gga_destroy", "gga_twophase_spawn", "gga_twophase_work", "gga_pool_create", "gga_pool_destroy",
            "gga_pool_info", "gga_create_in_pool", "gga_batch_create", "gga_batch_grow", "gga_batch_clear",
            "gga_batch_capture", "gga_batch_replay", "gga_batch_destroy", "gga_append_batch", "gga_read_batch",
            "gga_vmm_create", "gga_vmm_grow", "gga_vmm_info", "gga_vmm_destroy", "gga_flat_insert",
            "gga_debug_wait_timeout", "gga_serve_run"]


class gga_params(ctypes.Structure):
    _fields_ = [("n_lfvectors", ctypes.c_uint32), ("threads_per_block", ctypes.c_uint32),
                ("base_bucket", ctypes.c_uint64), ("elem_bytes", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("pool_bytes", ctypes.c_uint64)]


class gga_gen_spec(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("dist", ctypes.c_uint32), ("n_thresholds", ctypes.c_uint32),
                ("thresholds", ctypes.c_uint32 * MAX_THRESHOLDS), ("va", ctypes.c_uint64),
                ("vb", ctypes.c_uint64), ("vc", ctypes.c_uint64), ("round0", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class gga_batch_job(ctypes.Structure):
    _fields_ = [("array", ctypes.c_void_p), ("spec", gga_gen_spec), ("target", ctypes.c_uint64)]


class gga_append_req(ctypes.Structure):
    _fields_ = [("array", ctypes.c_void_p), ("n", ctypes.c_uint64), ("tag", ctypes.c_uint64)]


class gga_read_req(ctypes.Structure):
    _fields_ = [("array", ctypes.c_void_p), ("n", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("out", ctypes.c_void_p)]


class gga_serve_config(ctypes.Structure):
    _fields_ = [("n_arrays", ctypes.c_uint32), ("L", ctypes.c_uint32), ("B", ctypes.c_uint32),
                ("E", ctypes.c_uint32), ("read_n", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32), ("batched", ctypes.c_int32), ("deadline_s", ctypes.c_double),
                ("pool_bytes", ctypes.c_uint64)]


class gga_serve_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("step_requests", ctypes.c_uint64),
                ("appended_elements", ctypes.c_uint64), ("wall_s", ctypes.c_double),
                ("first_full_s", ctypes.c_double)]


SERVE_RESULT_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64)


class gga_mem(ctypes.Structure):
    _fields_ = [("bucket_bytes", ctypes.c_uint64), ("live_bytes", ctypes.c_uint64),
                ("pool_bytes", ctypes.c_uint64), ("pool_bump_bytes", ctypes.c_uint64),
                ("free_list_bytes", ctypes.c_uint64), ("metadata_bytes", ctypes.c_uint64)]


_lib = None


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libgga.so (building it with nvcc first if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"libgga.so not built ({path})")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    sig = {
        "gga_create": [ctypes.POINTER(gga_params), vp, vp, ctypes.POINTER(vp)],
        "gga_insert": [vp, vp, u32, vp, u64, vp],
        "gga_insert_noalloc": [vp, vp, u32, vp, u64, vp],
        "gga_insert_generated": [vp, ctypes.POINTER(gga_gen_spec), u32, vp],
        "gga_reserve": [vp, vp, vp],
        "gga_device_view": [vp, ctypes.POINTER(vp)],
        "gga_device_commit": [vp, vp],
        "gga_push_generated": [vp, ctypes.POINTER(gga_gen_spec), u32, vp],
        "gga_push_expand": [vp, vp, vp, u32, vp],
        "gga_read": [vp, vp, u64, vp, vp],
        "gga_write": [vp, vp, u64, vp, vp],
        "gga_sweep": [vp, i32, u64, u32, vp],
        "gga_flatten": [vp, vp, u64, vp],
        "gga_size": [vp, ctypes.POINTER(u64), vp, vp, vp],
        "gga_offsets": [vp, vp, vp],
        "gga_clear": [vp, vp],
        "gga_memory": [vp, ctypes.POINTER(gga_mem), vp],
        "gga_last_error": [vp, vp],
        "gga_destroy": [vp],
        "gga_twophase_spawn": [vp, u32, u64, i32, vp, vp],
        "gga_pool_create": [u64, vp, u64, vp, ctypes.POINTER(vp)],
        "gga_pool_destroy": [vp],
        "gga_pool_info": [vp, ctypes.POINTER(u64), vp],
        "gga_create_in_pool": [ctypes.POINTER(gga_params), vp, vp, ctypes.POINTER(vp)],
        "gga_batch_create": [ctypes.POINTER(gga_batch_job), u32, vp, ctypes.POINTER(vp)],
        "gga_batch_grow": [vp, vp],
        "gga_batch_clear": [vp, vp],
        "gga_batch_capture": [vp, vp],
        "gga_batch_replay": [vp, vp],
        "gga_batch_destroy": [vp],
        "gga_append_batch": [ctypes.POINTER(gga_append_req), u32, vp],
        "gga_read_batch": [ctypes.POINTER(gga_read_req), u32, vp],
        "gga_serve_run": [ctypes.POINTER(gga_serve_config), ctypes.POINTER(vp), u64, vp, vp, vp, vp, vp, vp, vp, u64,
                          vp, vp, SERVE_RESULT_FN, vp, ctypes.POINTER(gga_serve_stats), vp],
        "gga_twophase_work": [vp, u64, u32, vp],
        "gga_flat_insert": [i32, vp, u64, vp, u64, u32, u32, vp],
        "gga_debug_wait_timeout": [u32, i32, vp],
        "gga_vmm_create": [u64, ctypes.POINTER(vp)],
        "gga_vmm_grow": [vp, u64],
        "gga_vmm_info": [vp, ctypes.POINTER(u64)],
        "gga_vmm_destroy": [vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    _lib = lib
    return lib


class GGAError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what} failed: GGA_ERR_{ERROR_NAMES.get(code, code)}")
        self.code = code


def _check(rc: int, what: str):
    if rc != GGA_OK:
        raise GGAError(rc, what)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return ctypes.c_void_p(t.data_ptr())


_ELEM_DTYPE = {4: torch.int32, 8: torch.int64, 16: torch.int64}


def elem_tensor(n: int, E: int, device="cuda") -> torch.Tensor:
    """A device buffer of n E-byte elements (int32, int64, or int64 pairs for records)."""
    if E == 16:
        return torch.empty((n, 2), dtype=torch.int64, device=device)
    return torch.empty(n, dtype=_ELEM_DTYPE[E], device=device)


# ---------------------------------------------------------------------------
# Functions with the C names (argument marshalling only).

def gga_create(L: int, T: int, B: int, E: int, pool_bytes: int, pool: torch.Tensor | None = None,
               stream=None) -> ctypes.c_void_p:
    lib = load_library()
    p = gga_params(L, T, B, E, 0, pool_bytes)
    h = ctypes.c_void_p()
    _check(lib.gga_create(ctypes.byref(p), _dptr(pool) if pool is not None else None, _stream(stream),
                          ctypes.byref(h)), "gga_create")
    return h


def gga_pool_create(pool_bytes: int, min_bucket_bytes: int, slab: torch.Tensor | None = None,
                    stream=None) -> ctypes.c_void_p:
    pl = ctypes.c_void_p()
    _check(load_library().gga_pool_create(pool_bytes, _dptr(slab) if slab is not None else None, min_bucket_bytes,
                                          _stream(stream), ctypes.byref(pl)), "gga_pool_create")
    return pl


def gga_pool_destroy(pool):
    _check(load_library().gga_pool_destroy(pool), "gga_pool_destroy")


def gga_pool_info(pool, stream=None) -> dict:
    out = (ctypes.c_uint64 * 4)()
    _check(load_library().gga_pool_info(pool, out, _stream(stream)), "gga_pool_info")
    return {"pool_bytes": int(out[0]), "bump_bytes": int(out[1]), "free_list_bytes": int(out[2]),
            "queue_bytes": int(out[3])}


def gga_create_in_pool(L: int, T: int, B: int, E: int, pool, stream=None) -> ctypes.c_void_p:
    p = gga_params(L, T, B, E, 0, 0)
    h = ctypes.c_void_p()
    _check(load_library().gga_create_in_pool(ctypes.byref(p), pool, _stream(stream), ctypes.byref(h)),
           "gga_create_in_pool")
    return h


def gga_insert(h, counts: torch.Tensor, values: torch.Tensor, stream=None):
    assert counts.dtype in (torch.int32, torch.uint32) and counts.dim() == 3
    n_values = values.shape[0] if values.numel() else 0
    _check(load_library().gga_insert(h, _dptr(counts), counts.shape[0], _dptr(values) if n_values else None,
                                     n_values, _stream(stream)), "gga_insert")


def gga_insert_noalloc(h, counts: torch.Tensor, values: torch.Tensor, stream=None):
    """gga_insert without allocating: per-call scratch lives in the library's
    fixed 32 MiB device array (see include/gga.h).  Raises GGAError with
    GGA_ERR_TOO_LARGE when the call needs more scratch than that."""
    assert counts.dtype in (torch.int32, torch.uint32) and counts.dim() == 3
    n_values = values.shape[0] if values.numel() else 0
    _check(load_library().gga_insert_noalloc(h, _dptr(counts), counts.shape[0],
                                             _dptr(values) if n_values else None, n_values, _stream(stream)),
           "gga_insert_noalloc")


def make_gen_spec(seed: int, dist: str, coeffs, round0: int = 0, thresholds=None) -> gga_gen_spec:
    s = gga_gen_spec()
    s.seed = seed & 0xFFFFFFFFFFFFFFFF
    s.dist = DIST[dist]
    thr = [] if thresholds is None else [int(x) for x in thresholds]
    assert len(thr) <= MAX_THRESHOLDS
    s.n_thresholds = len(thr)
    for i, x in enumerate(thr):
        s.thresholds[i] = x
    va, vb, vc = (int(c) & 0xFFFFFFFFFFFFFFFF for c in coeffs)
    s.va, s.vb, s.vc = va, vb, vc
    s.round0 = round0
    return s


def gga_reserve(h, target: torch.Tensor, stream=None):
    """target: device int64 tensor of L capacities (elements)."""
    _check(load_library().gga_reserve(h, _dptr(target), _stream(stream)), "gga_reserve")


def gga_insert_generated(h, spec: gga_gen_spec, rounds: int, stream=None):
    _check(load_library().gga_insert_generated(h, ctypes.byref(spec), rounds, _stream(stream)),
           "gga_insert_generated")


def gga_device_view(h) -> int:
    """Device address of the handle's gga_dev_view (include/gga_device.cuh),
    for user kernels that call gga::block_push_back."""
    v = ctypes.c_void_p()
    _check(load_library().gga_device_view(h, ctypes.byref(v)), "gga_device_view")
    return v.value


def gga_device_commit(h, stream=None):
    _check(load_library().gga_device_commit(h, _stream(stream)), "gga_device_commit")


def gga_push_generated(h, spec: gga_gen_spec, rounds: int, stream=None):
    _check(load_library().gga_push_generated(h, ctypes.byref(spec), rounds, _stream(stream)),
           "gga_push_generated")


def gga_push_expand(h, counts: torch.Tensor, inputs: torch.Tensor, stream=None):
    """counts: uint32/int32 [R][L][T]; inputs: [R][L][T] elements of E bytes
    (for E = 16, int64 [R][L][T][2]): thread t of block l appends
    counts[r][l][t] copies of inputs[r][l][t] in round r."""
    assert counts.dtype in (torch.int32, torch.uint32) and counts.dim() == 3
    assert inputs.shape[:3] == counts.shape
    _check(load_library().gga_push_expand(h, _dptr(counts), _dptr(inputs), counts.shape[0], _stream(stream)),
           "gga_push_expand")


def gga_read(h, idx: torch.Tensor, out: torch.Tensor, stream=None):
    assert idx.dtype in (torch.int64, torch.uint64)
    _check(load_library().gga_read(h, _dptr(idx), idx.shape[0], _dptr(out), _stream(stream)), "gga_read")


def gga_write(h, idx: torch.Tensor, vals: torch.Tensor, stream=None):
    assert idx.dtype in (torch.int64, torch.uint64)
    _check(load_library().gga_write(h, _dptr(idx), idx.shape[0], _dptr(vals), _stream(stream)), "gga_write")


def gga_sweep(h, mode: int, delta: int, repeats: int = 1, stream=None):
    _check(load_library().gga_sweep(h, mode, delta & 0xFFFFFFFFFFFFFFFF, repeats, _stream(stream)), "gga_sweep")


def gga_flatten(h, dst: torch.Tensor, capacity: int | None = None, stream=None):
    cap = dst.shape[0] if capacity is None else capacity
    _check(load_library().gga_flatten(h, _dptr(dst), cap, _stream(stream)), "gga_flatten")


def gga_size(h, sizes: torch.Tensor | None = None, caps: torch.Tensor | None = None, stream=None):
    """Returns (total, device_error_code).  Synchronizes the stream."""
    n = ctypes.c_uint64(0)
    rc = load_library().gga_size(h, ctypes.byref(n), _dptr(sizes) if sizes is not None else None,
                                 _dptr(caps) if caps is not None else None, _stream(stream))
    if rc == GGA_ERR_CUDA:
        raise GGAError(rc, "gga_size")
    return int(n.value), rc


def gga_offsets(h, out: torch.Tensor, stream=None):
    _check(load_library().gga_offsets(h, _dptr(out), _stream(stream)), "gga_offsets")


def gga_clear(h, stream=None):
    _check(load_library().gga_clear(h, _stream(stream)), "gga_clear")


def gga_memory(h, stream=None) -> dict:
    m = gga_mem()
    _check(load_library().gga_memory(h, ctypes.byref(m), _stream(stream)), "gga_memory")
    return {k: int(getattr(m, k)) for k, _ in gga_mem._fields_}


def gga_last_error(h, stream=None) -> int:
    return int(load_library().gga_last_error(h, _stream(stream)))


def gga_destroy(h):
    _check(load_library().gga_destroy(h), "gga_destroy")


def gga_twophase_spawn(h, gen: int, seed: int, born: torch.Tensor | None = None, stream=None):
    """One spawning generation of the two-phase case study (all records spawn
    unless `born` (int64 [L], device) is given: then only those from born[l])."""
    _check(load_library().gga_twophase_spawn(h, gen, seed & 0xFFFFFFFFFFFFFFFF, 0 if born is None else 1,
                                             _dptr(born) if born is not None else None, _stream(stream)),
           "gga_twophase_spawn")


def gga_twophase_work(records: torch.Tensor, passes: int, stream=None):
    """pos += vel, `passes` streaming passes over flattened records ([n, 2] int64)."""
    _check(load_library().gga_twophase_work(_dptr(records), records.shape[0], passes, _stream(stream)),
           "gga_twophase_work")


def gga_append_batch(reqs, stream=None):
    """reqs: list of (GGArray, n, tag)."""
    arr = (gga_append_req * max(1, len(reqs)))()
    for i, (g, n, tag) in enumerate(reqs):
        arr[i].array, arr[i].n, arr[i].tag = g.h, int(n), int(tag) & 0xFFFFFFFFFFFFFFFF
    _check(load_library().gga_append_batch(arr, len(reqs), _stream(stream)), "gga_append_batch")


def gga_read_batch(reqs, stream=None):
    """reqs: list of (GGArray, n, seed, out tensor)."""
    arr = (gga_read_req * max(1, len(reqs)))()
    for i, (g, n, seed, out) in enumerate(reqs):
        arr[i].array, arr[i].n, arr[i].seed = g.h, int(n), int(seed) & 0xFFFFFFFFFFFFFFFF
        arr[i].out = out.data_ptr()
    _check(load_library().gga_read_batch(arr, len(reqs), _stream(stream)), "gga_read_batch")


def gga_serve_run(cfg: gga_serve_config, handles, t, typ, arr, nn, tag, read_out, flat_arena, on_result=None,
                  stream=None):
    """Run a request trace through the native server (include/gga_serve.h).
    t, typ, arr, nn, tag: host arrays (float64, int8, int64, int64, int64);
    read_out, flat_arena: device int64 tensors; on_result(request, dev_ptr,
    n_elems) or None.  Returns (latency_s, state, stats dict)."""
    import numpy as np
    m = len(t)
    t = np.ascontiguousarray(t, dtype=np.float64)
    typ = np.ascontiguousarray(typ, dtype=np.int8)
    arr = np.ascontiguousarray(arr, dtype=np.int64)
    nn = np.ascontiguousarray(nn, dtype=np.int64)
    tag = np.ascontiguousarray(tag, dtype=np.int64)
    lat = np.empty(m, dtype=np.float64)
    state = np.zeros(m, dtype=np.int8)
    hs = (ctypes.c_void_p * max(1, len(handles)))(*handles)
    cb = SERVE_RESULT_FN(lambda ctx, r, ptr, n: on_result(int(r), int(ptr or 0), int(n))) if on_result else \
        SERVE_RESULT_FN()
    st = gga_serve_stats()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    arena_elems = flat_arena.numel() * flat_arena.element_size() // cfg.E
    _check(load_library().gga_serve_run(ctypes.byref(cfg), hs, m, p(t), p(typ), p(arr), p(nn), p(tag),
                                        _dptr(read_out), _dptr(flat_arena), arena_elems, p(lat), p(state), cb, None,
                                        ctypes.byref(st), _stream(stream)), "gga_serve_run")
    stats = {"steps": st.steps, "step_requests": st.step_requests, "appended_elements": st.appended_elements,
             "wall_s": st.wall_s, "first_full_s": None if st.first_full_s < 0 else st.first_full_s}
    return lat, state, stats


_cudart = None


def device_to_host(ptr: int, nbytes: int) -> bytes:
    """Copy nbytes at device address ptr to the host (cudaMemcpy of the CUDA
    runtime the library links; for test-mode result capture)."""
    global _cudart
    if _cudart is None:
        import glob
        cands = sorted(glob.glob(os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcudart.so*")))
        if not cands:
            raise ImportError("libcudart not found")
        _cudart = ctypes.CDLL(cands[-1])
    buf = ctypes.create_string_buffer(max(1, nbytes))
    if nbytes:
        rc = _cudart.cudaMemcpy(buf, ctypes.c_void_p(ptr), ctypes.c_size_t(nbytes), 2)   # device to host
        if rc != 0:
            raise GGAError(GGA_ERR_CUDA, "cudaMemcpy")
    return buf.raw[:nbytes]


def gga_debug_wait_timeout(attempts: int, arrive: bool, stream=None) -> int:
    """Test hook (include/gga_debug.h): status of a bounded mbarrier wait
    that completes (arrive) or that nothing completes (GGA_ERR_TIMEOUT)."""
    return int(load_library().gga_debug_wait_timeout(int(attempts), 1 if arrive else 0, _stream(stream)))


GGA_FLAT_ATOMIC = 0
GGA_FLAT_SCAN = 1


def gga_flat_insert(mode: int, array: torch.Tensor, size: torch.Tensor, n_threads: int, threads_per_block: int,
                    first_value: int = 0, stream=None):
    """Sec. III-B insertion approaches on a flat uint32 array (include/gga_flat.h).
    array: device int32 tensor (capacity = its length); size: device int64
    tensor of one element, advanced by n_threads."""
    assert array.dtype == torch.int32 and size.dtype == torch.int64 and size.numel() == 1
    _check(load_library().gga_flat_insert(int(mode), _dptr(array), array.numel(), _dptr(size), int(n_threads),
                                          int(threads_per_block), int(first_value) & 0xFFFFFFFF, _stream(stream)),
           "gga_flat_insert")


class GGAVMM:
    """The memMap comparison array (include/gga_vmm.h): a reserved range of
    device addresses grown by mapping physical memory behind it, no copy.
    tensor(n, dtype) is a zero-copy view of the first n elements."""

    def __init__(self, max_bytes: int):
        self.h = ctypes.c_void_p()
        _check(load_library().gga_vmm_create(int(max_bytes), ctypes.byref(self.h)), "gga_vmm_create")

    def grow(self, nbytes: int):
        _check(load_library().gga_vmm_grow(self.h, int(nbytes)), "gga_vmm_grow")

    def info(self):
        out = (ctypes.c_uint64 * 3)()
        _check(load_library().gga_vmm_info(self.h, out), "gga_vmm_info")
        return {"address": int(out[0]), "mapped_bytes": int(out[1]), "granularity": int(out[2])}

    def tensor(self, n: int, dtype=torch.int32) -> torch.Tensor:
        inf = self.info()
        itemsize = torch.empty(0, dtype=dtype).element_size()
        if n * itemsize > inf["mapped_bytes"]:
            raise ValueError("view beyond the mapped part")
        typestr = {torch.int32: "<i4", torch.int64: "<i8", torch.uint8: "|u1"}[dtype]

        class _View:
            __cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (inf["address"], False),
                                        "version": 2, "strides": None}
        return torch.as_tensor(_View(), device="cuda")

    def close(self):
        if self.h:
            _check(load_library().gga_vmm_destroy(self.h), "gga_vmm_destroy")
            self.h = ctypes.c_void_p()


class GGABatch:
    """Many GGArrays grown to their targets in one persistent launch (see
    gga_batch_create).  jobs: list of (GGArray, gga_gen_spec, target)."""

    def __init__(self, jobs, stream=None):
        self._arrays = [j[0] for j in jobs]
        arr = (gga_batch_job * max(1, len(jobs)))()
        for i, (g, spec, target) in enumerate(jobs):
            arr[i].array = g.h
            arr[i].spec = spec
            arr[i].target = int(target)
        self.h = ctypes.c_void_p()
        _check(load_library().gga_batch_create(arr, len(jobs), _stream(stream), ctypes.byref(self.h)),
               "gga_batch_create")

    def grow(self, stream=None):
        _check(load_library().gga_batch_grow(self.h, _stream(stream)), "gga_batch_grow")

    def clear(self, stream=None):
        _check(load_library().gga_batch_clear(self.h, _stream(stream)), "gga_batch_clear")

    def capture(self, stream):
        _check(load_library().gga_batch_capture(self.h, _stream(stream)), "gga_batch_capture")

    def replay(self, stream=None):
        _check(load_library().gga_batch_replay(self.h, _stream(stream)), "gga_batch_replay")

    def close(self):
        if self.h:
            _check(load_library().gga_batch_destroy(self.h), "gga_batch_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Object wrapper.

class GGAPool:
    """A bucket pool shared by several GGArrays (see gga_pool_create)."""

    def __init__(self, pool_bytes: int, min_bucket_bytes: int, slab: torch.Tensor | None = None, stream=None):
        self._slab = slab
        self.h = gga_pool_create(pool_bytes, min_bucket_bytes, slab, stream)

    def info(self, stream=None) -> dict:
        return gga_pool_info(self.h, stream)

    def close(self):
        if self.h:
            gga_pool_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GGArray:
    """A GGArray on the current CUDA device (L LFVectors of T-thread blocks,
    first bucket B elements, E-byte elements).  Buckets come from a private
    pool of pool_bytes (optionally on a lent slab tensor), or from a shared
    GGAPool."""

    def __init__(self, L: int, T: int, B: int, E: int, pool_bytes: int = 0, pool: torch.Tensor | None = None,
                 stream=None, shared_pool: GGAPool | None = None):
        self.L, self.T, self.B, self.E = L, T, B, E
        self.pool_bytes = pool_bytes
        self._pool = pool
        self._shared = shared_pool
        if shared_pool is not None:
            self.h = gga_create_in_pool(L, T, B, E, shared_pool.h, stream)
        else:
            self.h = gga_create(L, T, B, E, pool_bytes, pool, stream)

    def insert(self, counts, values, stream=None):
        gga_insert(self.h, counts, values, stream)

    def reserve(self, target, stream=None):
        """Capacity of LFVector l at least target[l] (device int64, L entries)."""
        gga_reserve(self.h, target, stream)

    def insert_generated(self, spec, rounds, stream=None):
        gga_insert_generated(self.h, spec, rounds, stream)

    def device_view(self) -> int:
        """Device pointer to pass to user kernels as `const gga_dev_view*`."""
        return gga_device_view(self.h)

    def device_commit(self, stream=None):
        """After user kernels pushed into the array (before any other call)."""
        gga_device_commit(self.h, stream)

    def push_generated(self, spec, rounds, stream=None):
        """insert_generated through the device API, one block_push_back per round."""
        gga_push_generated(self.h, spec, rounds, stream)

    def push_expand(self, counts, inputs, stream=None):
        """Memory-sourced pushes through the device API (block_push_rounds)."""
        gga_push_expand(self.h, counts, inputs, stream)

    def read(self, idx, out=None, stream=None):
        if out is None:
            out = elem_tensor(idx.shape[0], self.E, idx.device)
        gga_read(self.h, idx, out, stream)
        return out

    def write(self, idx, vals, stream=None):
        gga_write(self.h, idx, vals, stream)

    def sweep(self, mode, delta=1, repeats=1, stream=None):
        gga_sweep(self.h, mode, delta, repeats, stream)

    def flatten(self, dst=None, stream=None):
        if dst is None:
            n, _ = self.size(stream)
            dst = elem_tensor(max(n, 1), self.E)
        gga_flatten(self.h, dst, dst.shape[0], stream)
        return dst

    def size(self, stream=None):
        return gga_size(self.h, stream=stream)

    def sizes_caps(self, stream=None):
        sizes = torch.empty(self.L, dtype=torch.int64, device="cuda")
        caps = torch.empty(self.L, dtype=torch.int64, device="cuda")
        n, rc = gga_size(self.h, sizes, caps, stream)
        return n, rc, sizes, caps

    def offsets(self, stream=None):
        out = torch.empty(self.L + 1, dtype=torch.int64, device="cuda")
        gga_offsets(self.h, out, stream)
        return out

    def clear(self, stream=None):
        gga_clear(self.h, stream)

    def memory(self, stream=None):
        return gga_memory(self.h, stream)

    def last_error(self, stream=None):
        return gga_last_error(self.h, stream)

    def close(self):
        if self.h:
            gga_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""GGArray oracle -- TEST INFRASTRUCTURE ONLY.

A plain single-threaded CPU model of the GGArray (Meneses, Navarro and
Ferrada, arXiv 2209.00103), written in C++ (``gga_oracle.cpp``) and loaded
here through ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA path and never imports the package.

Every function of the C++ file cites the passage of the paper it follows.
Parity status: all functions are pinned by ``tests/test_oracle_pins.py``
(closed forms, brute force over tiny inputs, an independent Python model,
self-describing values); none is "parity unpinned".
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gga_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_INVALID = 1
ERR_OUT_OF_RANGE = 2
ERR_DST_TOO_SMALL = 3

DIST = {"bernoulli": 0, "uniform3": 1, "geometric": 2, "poisson": 3}


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ if it is missing or older than its source."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u8p = ctypes.c_void_p
        lib.orc_create.restype = ctypes.c_void_p
        lib.orc_create.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
        lib.orc_destroy.argtypes = [ctypes.c_void_p]
        lib.orc_insert.restype = ctypes.c_int
        lib.orc_insert.argtypes = [ctypes.c_void_p, u8p, ctypes.c_uint32, u8p, ctypes.c_uint64, u8p]
        lib.orc_insert_generated.restype = ctypes.c_int
        lib.orc_insert_generated.argtypes = [
            ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, u8p, ctypes.c_uint32,
            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, u8p]
        lib.orc_size.restype = ctypes.c_uint64
        lib.orc_size.argtypes = [ctypes.c_void_p]
        lib.orc_sizes.argtypes = [ctypes.c_void_p, u8p]
        lib.orc_capacities.argtypes = [ctypes.c_void_p, u8p, u8p]
        lib.orc_reserve.restype = ctypes.c_int
        lib.orc_reserve.argtypes = [ctypes.c_void_p, u8p]
        lib.orc_offsets.argtypes = [ctypes.c_void_p, u8p]
        lib.orc_bucket_of.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)]
        lib.orc_capacity_of.restype = ctypes.c_uint64
        lib.orc_capacity_of.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.orc_read.restype = ctypes.c_int
        lib.orc_read.argtypes = [ctypes.c_void_p, u8p, ctypes.c_uint64, u8p]
        lib.orc_write.restype = ctypes.c_int
        lib.orc_write.argtypes = [ctypes.c_void_p, u8p, ctypes.c_uint64, u8p]
        lib.orc_sweep_add.restype = ctypes.c_int
        lib.orc_sweep_add.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32]
        lib.orc_flatten.restype = ctypes.c_int
        lib.orc_flatten.argtypes = [ctypes.c_void_p, u8p, ctypes.c_uint64]
        lib.orc_lfvector.restype = ctypes.c_uint64
        lib.orc_lfvector.argtypes = [ctypes.c_void_p, ctypes.c_uint32, u8p]
        lib.orc_bucket_bytes.restype = ctypes.c_uint64
        lib.orc_bucket_bytes.argtypes = [ctypes.c_void_p]
        lib.orc_splitmix_at.restype = ctypes.c_uint64
        lib.orc_splitmix_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.orc_grow_to_target.restype = ctypes.c_int
        lib.orc_grow_to_target.argtypes = [
            ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, u8p, ctypes.c_uint32, ctypes.c_uint64,
            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
        lib.orc_append.restype = ctypes.c_int
        lib.orc_append.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]
        lib.orc_read_random.restype = ctypes.c_int
        lib.orc_read_random.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, u8p]
        lib.orc_spawn.restype = ctypes.c_int
        lib.orc_spawn.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, u8p]
        lib.orc_work_passes.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32]
        lib.orc_draw_count.restype = ctypes.c_uint32
        lib.orc_draw_count.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u8p, ctypes.c_uint32]
        _lib = lib
        return lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


_DTYPES = {4: np.dtype(np.uint32), 8: np.dtype(np.uint64), 16: np.dtype((np.void, 16))}


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


class OracleGGArray:
    """One GGArray held by the C++ oracle (L LFVectors, T threads per block,
    first bucket B elements, E-byte elements)."""

    def __init__(self, L: int, T: int, B: int, E: int):
        self._lib = _load()
        self.L, self.T, self.B, self.E = int(L), int(T), int(B), int(E)
        self._h = self._lib.orc_create(self.L, self.T, self.B, self.E)
        if not self._h:
            raise OracleError(ERR_INVALID, "create")
        self.dtype = _DTYPES[self.E]

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, what: str):
        if rc != OK:
            raise OracleError(rc, what)

    # Algorithm 1 over R rounds with packed values.
    def insert(self, counts: np.ndarray, values: np.ndarray, per_round: bool = False):
        counts = np.ascontiguousarray(counts, dtype=np.uint32)
        R = counts.shape[0]
        assert counts.shape == (R, self.L, self.T)
        values = np.ascontiguousarray(values)
        assert values.dtype.itemsize == self.E
        n = values.shape[0]
        spr = np.zeros((R, self.L), dtype=np.uint64) if per_round else None
        self._check(self._lib.orc_insert(self._h, _ptr(counts), R, _ptr(values), n, _ptr(spr)), "insert")
        return spr

    def insert_generated(self, seed: int, dist: str, coeffs, round0: int, rounds: int,
                         thresholds: np.ndarray | None = None, return_counts: bool = False):
        thr = None if thresholds is None else np.ascontiguousarray(thresholds, dtype=np.uint32)
        cnt = np.zeros((rounds, self.L, self.T), dtype=np.uint32) if return_counts else None
        va, vb, vc = (int(c) & 0xFFFFFFFFFFFFFFFF for c in coeffs)
        rc = self._lib.orc_insert_generated(
            self._h, seed & 0xFFFFFFFFFFFFFFFF, DIST[dist], _ptr(thr), 0 if thr is None else len(thr),
            va, vb, vc, round0, rounds, _ptr(cnt))
        self._check(rc, "insert_generated")
        return cnt

    def grow_to_target(self, seed: int, dist: str, coeffs, target: int, round0: int = 0,
                       thresholds: np.ndarray | None = None, max_rounds: int = 1 << 20):
        thr = None if thresholds is None else np.ascontiguousarray(thresholds, dtype=np.uint32)
        va, vb, vc = (int(c) & 0xFFFFFFFFFFFFFFFF for c in coeffs)
        rc = self._lib.orc_grow_to_target(self._h, seed & 0xFFFFFFFFFFFFFFFF, DIST[dist], _ptr(thr),
                                          0 if thr is None else len(thr), va, vb, vc, round0, target, max_rounds)
        self._check(rc, "grow_to_target")

    def append(self, n: int, tag: int):
        """Served append (see orc_append)."""
        self._check(self._lib.orc_append(self._h, n, tag & 0xFFFFFFFFFFFFFFFF), "append")

    def read_random(self, n: int, seed: int) -> np.ndarray:
        out = np.zeros(max(n, 1), dtype=self.dtype)
        self._check(self._lib.orc_read_random(self._h, n, seed & 0xFFFFFFFFFFFFFFFF, _ptr(out)), "read_random")
        return out[:n]

    def size(self) -> int:
        return int(self._lib.orc_size(self._h))

    def sizes(self) -> np.ndarray:
        out = np.zeros(self.L, dtype=np.uint64)
        self._lib.orc_sizes(self._h, _ptr(out))
        return out

    def reserve(self, target) -> int:
        """Resize: capacity of LFVector l at least target[l] (see orc_reserve)."""
        t = np.ascontiguousarray(target, dtype=np.uint64)
        assert t.shape == (self.L,)
        return self._lib.orc_reserve(self._h, _ptr(t))

    def capacities(self):
        caps = np.zeros(self.L, dtype=np.uint64)
        nb = np.zeros(self.L, dtype=np.uint64)
        self._lib.orc_capacities(self._h, _ptr(caps), _ptr(nb))
        return caps, nb

    def offsets(self) -> np.ndarray:
        out = np.zeros(self.L + 1, dtype=np.uint64)
        self._lib.orc_offsets(self._h, _ptr(out))
        return out

    def read(self, idx: np.ndarray):
        idx = np.ascontiguousarray(idx, dtype=np.uint64)
        out = np.zeros(idx.shape[0], dtype=self.dtype)
        rc = self._lib.orc_read(self._h, _ptr(idx), idx.shape[0], _ptr(out))
        return out, rc

    def write(self, idx: np.ndarray, vals: np.ndarray) -> int:
        idx = np.ascontiguousarray(idx, dtype=np.uint64)
        vals = np.ascontiguousarray(vals)
        assert vals.dtype.itemsize == self.E and vals.shape[0] == idx.shape[0]
        return self._lib.orc_write(self._h, _ptr(idx), idx.shape[0], _ptr(vals))

    def sweep_add(self, delta: int, repeats: int = 1):
        self._check(self._lib.orc_sweep_add(self._h, delta & 0xFFFFFFFFFFFFFFFF, repeats), "sweep_add")

    def flatten(self, capacity: int | None = None) -> np.ndarray:
        n = self.size()
        cap = n if capacity is None else int(capacity)
        out = np.zeros(max(cap, 1), dtype=self.dtype)
        self._check(self._lib.orc_flatten(self._h, _ptr(out), cap), "flatten")
        return out[:n]

    def lfvector(self, l: int) -> np.ndarray:
        n = int(self._lib.orc_lfvector(self._h, l, None))
        out = np.zeros(max(n, 1), dtype=self.dtype)
        self._lib.orc_lfvector(self._h, l, _ptr(out))
        return out[:n]

    def spawn(self, gen: int, seed: int, only_newborn: bool = False, born: np.ndarray | None = None):
        """Spawning generation of the two-phase case study (see orc_spawn)."""
        if only_newborn:
            assert born is not None and born.dtype == np.uint64 and born.shape == (self.L,)
        self._check(self._lib.orc_spawn(self._h, gen, seed & 0xFFFFFFFFFFFFFFFF, int(only_newborn),
                                        _ptr(born) if only_newborn else None), "spawn")

    def bucket_bytes(self) -> int:
        return int(self._lib.orc_bucket_bytes(self._h))


def bucket_of(j: int, B: int):
    lib = _load()
    b = ctypes.c_uint32()
    off = ctypes.c_uint64()
    lib.orc_bucket_of(j, B, ctypes.byref(b), ctypes.byref(off))
    return int(b.value), int(off.value)


def capacity_of(size: int, B: int) -> int:
    return int(_load().orc_capacity_of(size, B))


def splitmix_at(seed: int, key: int) -> int:
    return int(_load().orc_splitmix_at(seed & 0xFFFFFFFFFFFFFFFF, key & 0xFFFFFFFFFFFFFFFF))


def work_passes(records: np.ndarray, passes: int) -> np.ndarray:
    """pos += vel, `passes` times, on flattened 16-byte records (in place)."""
    assert records.dtype.itemsize == 16 and records.flags["C_CONTIGUOUS"]
    _load().orc_work_passes(_ptr(records), records.shape[0], passes)
    return records


def draw_count(dist: str, h: int, thresholds: np.ndarray | None = None) -> int:
    thr = None if thresholds is None else np.ascontiguousarray(thresholds, dtype=np.uint32)
    return int(_load().orc_draw_count(DIST[dist], h, _ptr(thr), 0 if thr is None else len(thr)))

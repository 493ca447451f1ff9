"""Builds and loads tests/cuda/user_push_back.cu: a user's kernels written
against the public device header alone (include/gga_device.cuh), compiled
with nvcc for sm_103a into a library of their own."""

from __future__ import annotations

import ctypes
import os
import subprocess

from paper_2209_00103_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cuda", "user_push_back.cu")
OUT = os.path.join(HERE, "cuda", "_build", "libgga_user_push.so")
HEADERS = [os.path.join(build.INCLUDE, f) for f in ("gga_device.cuh", "gga_layout.cuh", "gga.h")]


def build_user() -> str:
    """Compile the user library (only include/ on the include path)."""
    deps = [SRC] + HEADERS
    if os.path.exists(OUT) and all(os.path.getmtime(d) <= os.path.getmtime(OUT) for d in deps):
        return OUT
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = [build.nvcc(), *build.ARCH, "-O3", "-std=c++17", "-I" + build.INCLUDE, "-Xcompiler", "-fPIC",
           "-shared", "-cudart", "shared", "-o", tmp, SRC]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, OUT)
    return OUT


def load_user() -> ctypes.CDLL:
    lib = ctypes.CDLL(build_user())
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    sig = {
        "user_push_rounds": [vp, vp, vp, vp, u32, u32, u32, u32, u32, u32, u32, i32, i32, vp],
        "user_push_rounds_cursor": [vp, vp, vp, vp, u32, u32, u32, u32, u32, u32, u32, i32, i32, vp],
        "user_push_rounds_mode": [vp, vp, vp, vp, u32, u32, u32, u32, u32, u32, u32, i32, i32, i32, u32, vp],
        "user_push_own": [vp, vp, vp, u32, u32, u32, vp],
        "user_push_formula": [vp, vp, u32, u32, u32, i32, vp],
        "user_read_global": [vp, vp, u64, vp, vp, u32, vp],
        "user_read_local": [vp, vp, vp, u64, vp, vp, u32, vp],
        "user_push_rejected": [vp, i32, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    return lib

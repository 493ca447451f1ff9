"""GB300-native GGArray: a dynamically growable GPU array (arXiv 2209.00103).

The compute path is the CUDA library libgga.so (csrc/, C ABI in
include/gga.h); ``gga`` is its ctypes binding and ``workloads`` draws the
seeded synthetic inputs.  Attributes of ``gga`` are re-exported lazily so that
importing the package does not load the CUDA library.
"""

__all__ = ["gga", "workloads", "build"]


def __getattr__(name):
    import importlib
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    mod = importlib.import_module(f"{__name__}.gga")
    try:
        return getattr(mod, name)
    except AttributeError:
        raise AttributeError(name) from None

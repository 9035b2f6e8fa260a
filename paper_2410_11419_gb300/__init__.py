"""GS^3 triple-splatting relighting renderer for GB300 (sm_103a).

The compute path is libgs3.so (hand-written CUDA kernels behind the C ABI in
include/gs3.h); this package holds its ctypes binding, a device-memory helper
built on torch, and the seeded synthetic-scene generator.
"""
from . import synth  # noqa: F401  (host-only, no CUDA needed)


def __getattr__(name):
    # the CUDA-backed modules load libgs3.so lazily
    if name in ("render", "_native"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)

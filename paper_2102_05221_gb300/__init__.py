"""GB300-native EAPruned elastic-distance search (arXiv 2102.05221).

The compute path is libeap.so (hand-written CUDA for sm_103a behind the C ABI
in include/eap.h); ``eap`` is its ctypes binding and ``synth`` draws the
seeded synthetic inputs.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "eap", "build"]


def __getattr__(name):
    if name in ("eap", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

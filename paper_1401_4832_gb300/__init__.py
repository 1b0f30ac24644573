"""GB300-native asymmetric plmDCA (Ekeberg, Hartonen & Aurell 2014).

The compute lives in the CUDA library built from ``csrc/`` (C ABI in
``include/plmdca.h``); :mod:`.api` is its Python binding.  Importing this
package loads nothing; the library is loaded on first use and its absence
is an error (there is no CPU fallback).
"""
__all__ = ["api", "synth"]


def __getattr__(name):
    if name in ("api", "synth", "autograd"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)

"""Work-efficient triangle-inequality K-means (KPynq) for GB300, sm_103a.

The compute path is the C-ABI library ``libkpynq.so`` built from ``csrc/``
(hand-written CUDA); ``kpynq`` is its thin ctypes binding.  ``synth`` holds the
seeded input generators.  Importing this package loads nothing; the binding
loads the library on first use and raises if it is missing (there is no CPU
fallback).
"""
__all__ = ["synth", "kpynq", "sharded"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)

"""GB300-native replica-parallel Metropolis annealing for sparse Ising / MaxCut.

The compute path is the CUDA library ``libisg`` (C ABI declared in
``include/isg.h``); ``paper_2311_09275_gb300.isg`` is its thin Python binding.
``inputs`` (seeded instance generators) and ``metrics`` (time-to-target
arithmetic) are plain host modules and load no native code.
"""
import importlib

__all__ = ["inputs", "metrics", "isg"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

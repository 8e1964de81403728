"""IterNCGP hot path for NVIDIA GB300 (sm_103a).

The compute lives in ``libitergp.so`` (C ABI, ``include/itergp.h``); ``native`` is its
ctypes binding and is imported lazily so that the input generators (``datagen``) can be
used without a GPU or a built library.
"""
import importlib

__all__ = ["datagen", "native"]


def __getattr__(name):
    if name in ("native", "datagen"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

"""GB300-native PB-SpGEMM (propagation-blocking outer-product SpGEMM).

The compute path is the CUDA library ``libpbspgemm.so`` (sources in
``csrc/``, C ABI in ``include/pb_spgemm.h``); ``binding`` marshals torch
tensors into that ABI.  ``model`` holds the roofline byte model.
"""
import importlib

__all__ = ["binding", "model"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

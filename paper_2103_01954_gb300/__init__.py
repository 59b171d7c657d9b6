"""GB300 (sm_103a) ray-march path of Mixture of Volumetric Primitives.

The compute lives in ``libmvp.so`` (CUDA kernels behind the C ABI of
``include/mvp.h``); :mod:`.binding` loads it with ctypes under the same names and
:mod:`.torch_ops` passes PyTorch tensors (device memory and streams) to it.
"""
from . import binding  # noqa: F401

__all__ = ["binding", "torch_ops"]


def __getattr__(name):
    if name == "torch_ops":
        import importlib

        return importlib.import_module(".torch_ops", __name__)
    raise AttributeError(name)

"""GB300-native moment-conserving GW: Sigma-moment construction on one GPU.

The numerical path lives in libmgw.so (CUDA, sm_103a; C ABI in include/mgw.h).
`mgw` binds it; `driver` sequences its calls into G0W0 and evGW.
"""
from . import build  # noqa: F401

__all__ = ["build", "mgw", "driver"]


def __getattr__(name):
    if name in ("mgw", "driver"):
        import importlib

        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)

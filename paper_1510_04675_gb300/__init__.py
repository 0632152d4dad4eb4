"""mgq: GB300-native (sm_103a CUDA) hot path of the multiscale thermalization
of pure SU(3) Yang-Mills theory, behind the C ABI of include/mgq.h."""
import importlib

from ._lib import MgqError, load  # noqa: F401

__all__ = ["MgqError", "load", "api", "build"]


def __getattr__(name):
    if name in ("api", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

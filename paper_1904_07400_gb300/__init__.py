"""tdgrav: GB300-native thin-disk self-gravity by the B-spline direct method
(arXiv 1904.07400).  C-ABI CUDA library + thin PyTorch binding."""
from . import native  # noqa: F401

__all__ = ["native", "Plan", "ThinDiskForces", "forces_batched"]


def __getattr__(name):
    if name in ("Plan", "ThinDiskForces", "forces_batched"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)

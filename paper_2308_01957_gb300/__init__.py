"""GB300-native chi^2 forward-modelling path of AstroPhot (arXiv:2308.01957).

``build()`` compiles libastrophot_gb300.so (sm_103a); ``Context`` and ``chi2``
drive it from PyTorch.  There is no CPU fallback: without the library (or a
GPU) every call raises.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("Context", "Chi2", "chi2", "DeviceImage", "to_device_images"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)

"""GB300-native likelihood-guidance gradient for physics-guided diffusion FWI.

The compute path is the CUDA library ``libfwi.so`` (sources in ``csrc/``,
C ABI in ``include/fwi.h``); ``api`` is its thin Python binding.  Submodules
are imported lazily so that ``inputs`` (seeded synthetic data) can be used
without loading the CUDA library.
"""
import importlib

__all__ = ["api", "inputs", "autograd", "baselines"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

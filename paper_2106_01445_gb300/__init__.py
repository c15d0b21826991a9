"""GB300-native click-pattern probabilities for Gaussian boson sampling with
threshold detectors (Popova & Rubtsov, arXiv 2106.01445).

The computation lives in ``libgbs.so`` (CUDA C++ for sm_103a, C ABI declared
in include/gbs.h); this package is the Python binding.  Importing the package
does not load the library; ``Context()`` does, and fails loudly if it is not
built.
"""
from ._lib import GbsError, STATUS_NAMES  # noqa: F401


def Context(*args, **kwargs):
    from .api import Context as _Context
    return _Context(*args, **kwargs)

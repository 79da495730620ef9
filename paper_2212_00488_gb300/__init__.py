"""GB300 (sm_103a) implementation of the local stereo method of Chang &
Maruyama, "Real-Time High-Quality Stereo Matching System on a GPU"
(arXiv 2212.00488).

The compute path is ``lib/libstereo.so`` (C ABI in include/stereo.h).
Importing this package does not load it; ``Stereo`` and the ``_lib``
functions do, and raise if it is missing.
"""

__all__ = ["Stereo", "StereoOutput", "build"]


def __getattr__(name):
    if name in ("Stereo", "StereoOutput"):
        from . import stereo as _s
        return getattr(_s, name)
    raise AttributeError(name)

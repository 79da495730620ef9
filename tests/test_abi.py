"""The C-ABI library builds, loads and exports every symbol its header declares.

CPU only: no compute call is made (there is no GPU here); stereo_create must
fail cleanly with an error code when no sm_103 device is present.
"""
import ctypes
import os
import re

import pytest

from paper_2212_00488_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        names += re.findall(r"STEREO_API\s+[\w\s\*]+?\b(stereo_\w+)\s*\(", text)
    return names


@pytest.fixture(scope="module")
def lib():
    path = libbuild.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("stereo_create", "stereo_compute", "stereo_compute_host", "stereo_destroy",
                     "stereo_sync", "stereo_last_error", "stereo_default_params"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_2212_00488_gb300 import _lib
    assert set(_declared_functions()) <= set(_lib._SIGNATURES)
    _lib.load()


def test_default_params_are_the_papers():
    from paper_2212_00488_gb300 import _lib
    p = _lib.stereo_default_params()
    assert (p.lambda_ad, p.lambda_mc, p.t_fill) == (0.3, 2.3, 3)       # Sec. V
    assert (p.wx, p.wy, p.tc) == (21, 31, 13)                           # Table II footnote
    assert p.downscale == 1 and p.cost_scale == 512


def test_create_fails_cleanly_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2212_00488_gb300 import _lib
    with pytest.raises(_lib.StereoError):
        _lib.stereo_create(0)

"""GB300-native relaxed OS-LALM for PWLS X-ray CT reconstruction.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/ct.h``); :mod:`paper_1512_04564_gb300.ct` is its thin binding.
"""

import os

from . import build as _build

LIB_PATH = _build.LIB


def load():
    """Import the binding (loads ``libct.so``; raises if it was not built)."""
    from . import ct

    return ct

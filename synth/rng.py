"""Counter-based random generator used for every seeded input."""

import numpy as np


def philox(seed: int, stream: int = 0) -> np.random.Generator:
    """Philox4x64 generator keyed by (seed, stream).

    Philox is counter based, so a given (seed, stream) pair always yields the
    same sequence on every machine (x86 here, aarch64 on the GPU host).
    """
    key = (int(seed) & 0xFFFFFFFFFFFFFFFF) ^ ((int(stream) * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF)
    return np.random.Generator(np.random.Philox(key=key))

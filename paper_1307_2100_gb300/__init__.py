"""GB300-native binary tensor contraction (the method of arXiv 1307.2100).

The compute path is libtc.so (hand-written sm_103a kernels behind a C ABI,
declared in include/tc.h).  :mod:`.tc` is the ctypes binding with the C
names (importing it fails loudly when the library is not built: there is no
fallback); :class:`Contraction` (in :mod:`.api`) takes PyTorch tensors.
:mod:`.build` compiles the library and does not need it to exist.
"""
from __future__ import annotations

__all__ = ["tc", "Contraction"]


def __getattr__(name):
    import importlib
    if name == "Contraction":
        return importlib.import_module(".api", __name__).Contraction
    if name == "tc":
        return importlib.import_module(".tc", __name__)
    raise AttributeError(name)

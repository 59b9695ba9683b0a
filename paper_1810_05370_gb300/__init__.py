"""GB300 library for the operator-split multispecies glioblastoma step with mass effect.

The computation lives in libtg.so (hand-written sm_103a CUDA behind the C ABI of
include/tg.h).  This package is the Python binding: `_tg` mirrors the C entry points by name,
`Simulation` manages torch-owned device buffers around them; `build.build()` compiles the
library.  Importing `Simulation` loads
libtg.so and fails loudly if it is missing; there is no CPU fallback.
"""
__all__ = ["Simulation"]


def __getattr__(name):
    if name == "Simulation":
        from .simulation import Simulation
        return Simulation
    raise AttributeError(name)

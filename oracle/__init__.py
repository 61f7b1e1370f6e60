"""FP64 CPU oracle for the SRP-map hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct numpy/scipy implementation of what the GPU library
computes, written from the paper (Dietzen, De Sena, van Waterschoot, "Scalable-
Complexity Steered Response Power Based on Low-Rank and Sparse Interpolation").
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library and never
imports it; the product path fails loudly when its CUDA extension is missing.

Every function cites the section / equation it follows.  Pins (what fixes each
function independently of itself) live in ``tests/test_oracle_pins.py``.  There is
no function here whose parity is unpinned.
"""
from .srp import *  # noqa: F401,F403
from .srp import __all__  # noqa: F401

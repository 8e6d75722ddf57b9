"""CPU FP64 oracle for the ACOPF callbacks and the condensed KKT matrix.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
library under ``paper_2307_16830_gb300`` never imports it, and it imports
nothing from the library except the seeded data generator
``paper_2307_16830_gb300.synth`` (which holds no arithmetic of the method).
"""
from .acopf import *  # noqa: F401,F403
from .step import *  # noqa: F401,F403
from .chol import *  # noqa: F401,F403
from .ipm import *  # noqa: F401,F403

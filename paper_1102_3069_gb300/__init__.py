"""GB300 (sm_103a) effective-field + Landau-Lifshitz time-step path after
Vansteenkiste & Van de Wiele, "MuMax: a new high-performance micromagnetic
simulation tool" (arXiv:1102.3069).

The compute lives in ``csrc/`` (CUDA, built into the in-tree ``libmm.so`` by
``build.build()``); ``binding`` exposes the C ABI of ``include/mm.h`` with the
same names.  ``inputs`` holds the seeded synthetic workload generators.
"""

from . import binding  # noqa: F401

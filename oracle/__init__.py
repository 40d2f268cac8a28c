"""FP64 serial MPDATA oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.  ``build()`` compiles ``mpdata_oracle.c`` with gcc
(``-O2 -ffp-contract=off``: no fused multiply-add, so every operation rounds
once, in the order written); ``build(omp=True)`` compiles the same source
with ``-fopenmp`` for the all-core CPU baseline.
"""
from .oracle import Config, build, lib_path, load, mass, run, stages, step, threads  # noqa: F401

"""GB300 (sm_103a) Metropolis engine for Ising nanofilms built from height maps.

The compute path is the C-ABI library libisingfilm.so (include/isingfilm.h) with hand-written
CUDA kernels; `isingfilm` is its thin ctypes binding.  Importing the package does not load the
library: `from paper_1205_5588_gb300 import isingfilm` does, and fails loudly when it has not
been built (see `paper_1205_5588_gb300.build`).
"""

__all__ = ["isingfilm", "workloads", "build"]

"""B300-native (sm_103a) vectorial lattice Boltzmann step library.

The compute path is the CUDA library built from csrc/ (C interface in include/vlbm.h); `vlbm`
is its Python binding, `workloads` builds seeded synthetic inputs.  Importing `vlbm` requires
the built library; there is no CPU fallback.
"""

__all__ = ["vlbm", "workloads", "autograd"]

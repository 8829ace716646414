"""GB300-native kinetic-closure LES lattice-Boltzmann hot path.

The compute path is the CUDA shared library ``csrc/liblbm.so`` (sm_103a),
reached through the C ABI declared in ``include/lbm.h``; ``lbm`` is the thin
ctypes binding with the same entry-point names.  Importing this package does
not load the library; ``paper_2605_19796_gb300.lbm`` does, and raises if the
library has not been built.
"""
__all__ = ["lbm", "inputs"]

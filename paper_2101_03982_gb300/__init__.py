"""GB300-native semi-Lagrangian off-lattice Boltzmann step (arXiv:2101.03982).

The compute path is the CUDA library ``libolb.so`` (C ABI in ``include/olb.h``);
``olb`` is its thin ctypes binding.  Importing this package does not load the
library; the first call into ``olb`` does, and raises if it is missing.
"""
__all__ = ["olb", "inputs", "params"]

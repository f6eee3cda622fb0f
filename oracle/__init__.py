"""FP64 CPU oracle of the semi-Lagrangian lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: plain, slow, obviously correct numpy code written
from the paper (arXiv:2101.03982).  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product path (the
CUDA library and its binding) never does, and the oracle imports nothing from
the product.

``sllbm.strain_dissipation`` is a builder's estimator (no formula in the
paper); it is pinned by the analytic strain of the 3D Taylor-Green vortex
(tests/test_oracle_step.py).  ``glc`` holds the paper's cell-wise
Gauss-Lobatto-Chebyshev interpolation (tests/test_oracle_glc.py); the CUDA
library does not implement it yet.
"""

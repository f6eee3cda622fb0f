"""FP64 oracle of the enstrophy diagnostic (Sec. 4.2).

TEST INFRASTRUCTURE ONLY.  Nothing under ``oracle/`` is part of the product
path: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library.

Sec. 4.2 defines the enstrophy as the box average of the squared vorticity,
E = (2 pi)^-3 integral of |curl u|^2, and uses nu E as the physical
dissipation.  The paper's solver takes the curl from its finite elements; on
the uniform grid of this build the reading is fourth-order central
differences with periodic wrap,
  d g / dx ~ (g(x - 2) - 8 g(x - 1) + 8 g(x + 1) - g(x + 2)) / (12 dx),
and the average is the mean over the nodes.

Pins (tests/test_oracle_diagnostics.py): the closed form for the Taylor-Green
field (exact for this difference operator), zero curl for a discrete gradient
field, and fourth-order convergence to the continuum value.
"""
import numpy as np


def ddx4(g, dx, axis):
    """Fourth-order central difference of the periodic array g along `axis`."""
    return (np.roll(g, 2, axis=axis) - 8.0 * np.roll(g, 1, axis=axis)
            + 8.0 * np.roll(g, -1, axis=axis) - np.roll(g, -2, axis=axis)) / (12.0 * dx)


def vorticity(u, dx):
    """curl u of u (D, [nz,] ny, nx) with x the last array axis; 2D returns (1, ny, nx)."""
    D = u.shape[0]
    if D == 2:
        return np.stack([ddx4(u[1], dx, 1) - ddx4(u[0], dx, 0)])
    ax = {0: 2, 1: 1, 2: 0}  # spatial axis -> array axis
    d = lambda c, a: ddx4(u[c], dx, ax[a])
    return np.stack([d(2, 1) - d(1, 2), d(0, 2) - d(2, 0), d(1, 0) - d(0, 1)])


def enstrophy(u, dx):
    """Mean of |curl u|^2 over the nodes."""
    w = vorticity(u, dx)
    return float((w ** 2).sum(axis=0).mean())

"""Cell-wise interpolation on Gauss-Lobatto-Chebyshev points (Sec. 3).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: plain numpy FP64,
imported by tests only.  It shares no code with the CUDA library.

The paper's streaming step evaluates, for every support point x of a cell,
the interpolant of the post-collision field at the departure point
x - xi_i dt, using the Lagrange polynomials of the cell that contains the
departure point, whose support points are Gauss-Lobatto-Chebyshev (GLC)
points.  Here the grid is a tensor product of 1D periodic cell chains: an axis
of `cells` cells of width H carries n = cells * p nodes (neighbouring cells
share their end points), node j = c p + k sitting at H (c + zeta_k) with
zeta_k = (1 - cos(pi k / p)) / 2.

On such a grid the departure point of node j moves by the same physical shift
s for every node, so the cell offset and the weights depend only on the
residue k = j mod p: p stencils per velocity and axis (p^D in D dimensions).
Readings (listed with the others in the design notes): the mean node spacing
is dx = H / p; the GLC points are the Chebyshev extrema mapped to [0, 1].
"""
import itertools
import math

import numpy as np


def glc_points(p):
    """Local GLC coordinates zeta_0..zeta_p in [0, 1] (zeta_0 = 0, zeta_p = 1)."""
    return np.array([(1.0 - math.cos(math.pi * k / p)) / 2.0 for k in range(p + 1)])


def glc_positions(cells, p, length):
    """Node coordinates of one periodic axis: cells * p nodes."""
    H = length / cells
    z = glc_points(p)[:p]
    return np.array([H * (c + z[k]) for c in range(cells) for k in range(p)])


def lagrange_weights(nodes, x):
    """Lagrange basis of the points `nodes` evaluated at x (literal products)."""
    w = np.ones(len(nodes))
    for m in range(len(nodes)):
        for l in range(len(nodes)):
            if l != m:
                w[m] *= (x - nodes[l]) / (nodes[m] - nodes[l])
    return w


def residue_stencils(p, shift):
    """Per residue k = 0..p-1: (first support node relative to the node, weights).

    shift is the physical displacement of the departure point in cell widths
    (x_d = x - shift H).  The departure point of node k of cell c lies in cell
    c + d_k with d_k = floor(zeta_k - shift) at local coordinate
    zeta' = zeta_k - shift - d_k; its support nodes are (c + d_k) p + m,
    m = 0..p, i.e. j + d_k p - k + m.
    """
    z = glc_points(p)
    out = []
    for k in range(p):
        xl = z[k] - shift
        d = math.floor(xl)
        out.append((d * p - k, lagrange_weights(z, xl - d)))
    return out


def pull_plane_glc(plane, shifts, p):
    """Cell-wise GLC interpolation of one periodic field at the departure points.

    plane: (ny, nx) or (nz, ny, nx), every axis a multiple of p; shifts: the
    displacement per axis (x, y[, z]) in cell widths.  Direct evaluation of the
    (p+1)^D tensor-product sum per node.
    """
    D = plane.ndim
    st = [residue_stencils(p, float(shifts[a])) for a in range(D)]
    shape = plane.shape  # (z, y, x) order
    n = [shape[D - 1 - a] for a in range(D)]  # per axis (x, y, z)
    for a in range(D):
        if n[a] % p:
            raise ValueError("every axis must hold a whole number of cells")
    coords = [np.arange(n[a]) for a in range(D)]
    out = np.zeros_like(plane)
    for ms in itertools.product(range(p + 1), repeat=D):
        w_axes = []
        i_axes = []
        for a in range(D):
            k = coords[a] % p
            first = np.array([st[a][kk][0] for kk in range(p)])[k]
            w = np.array([st[a][kk][1][ms[a]] for kk in range(p)])[k]
            w_axes.append(w)
            i_axes.append((coords[a] + first + ms[a]) % n[a])
        # outer products in array order (z, y, x)
        W = w_axes[D - 1]
        for a in range(D - 2, -1, -1):
            W = np.multiply.outer(W, w_axes[a])
        out += W * plane[np.ix_(*[i_axes[a] for a in range(D - 1, -1, -1)])]
    return out


def pull_state_glc(vs, f, dt, cell, p):
    """The pull of every population field: shift xi_{i,a} dt / cell per axis."""
    xi = np.asarray(vs.xi, dtype=np.float64)
    return np.stack([pull_plane_glc(f[i], xi[i % vs.Q] * dt / cell, p) for i in range(f.shape[0])])


def step(prm, f, g=None):
    """One step with the cell-wise GLC pull, then the collision of Sec. 3.

    prm.dx is the mean node spacing, so the cell width is H = p dx.  Returns
    the post-collision state and the per-step diagnostics, as the uniform-grid
    step does (the global sums are plain node means).
    """
    from oracle import sllbm as O
    H = prm.p * prm.dx
    ft = pull_state_glc(prm.vs, f, prm.dt, H, prm.p).reshape(f.shape[0], -1)
    gt = pull_state_glc(prm.vs, g, prm.dt, H, prm.p).reshape(g.shape[0], -1) if prm.compressible else None
    fpost, gpost, diag = O.collide(prm, ft, gt)
    diag.update(O.reductions(prm, diag))
    fpost = fpost.reshape(f.shape)
    if gpost is not None:
        gpost = gpost.reshape(g.shape)
    return fpost, gpost, diag

"""Pins of the cell-wise Gauss-Lobatto-Chebyshev (GLC) interpolation oracle
(Sec. 3: the departure point is interpolated with the Lagrange polynomials of
the cell that contains it, on GLC support points).

* Brute force: per node, locate the departure cell and evaluate its Lagrange
  basis directly; the per-residue stencils must agree.
* p = 1: GLC points are the cell ends, so the scheme is linear interpolation on
  a uniform grid, equal to the equidistant p = 1 pull.
* Exactness for polynomials of degree <= p inside the domain, partition of
  unity, and convergence of order p + 1 under refinement.
* The whole step on a GLC grid: the 2D Taylor-Green vortex decays as
  exp(-2 nu t).
"""
import math

import numpy as np
import pytest

from oracle import glc as G
from oracle import sllbm as O
from oracle import velocity_sets as V


def brute_pull(plane, shifts, p, cells_len):
    """Departure cell located per node from the node's coordinate."""
    D = plane.ndim
    n = [plane.shape[D - 1 - a] for a in range(D)]
    pos = [G.glc_positions(n[a] // p, p, cells_len[a]) for a in range(D)]
    H = [cells_len[a] / (n[a] // p) for a in range(D)]
    z = G.glc_points(p)
    out = np.zeros_like(plane)
    for idx in np.ndindex(plane.shape):
        node = idx[::-1]
        per_axis = []
        for a in range(D):
            xd = (pos[a][node[a]] - shifts[a] * H[a]) % cells_len[a]
            c = int(math.floor(xd / H[a] + 1e-12))
            c = min(c, n[a] // p - 1)
            w = G.lagrange_weights(z, xd / H[a] - c)
            per_axis.append([((c * p + m) % n[a], w[m]) for m in range(p + 1)])
        acc = 0.0
        for combo in np.ndindex(*([p + 1] * D)):
            w = 1.0
            src = []
            for a in range(D):
                j, wm = per_axis[a][combo[a]]
                w *= wm
                src.append(j)
            acc += w * plane[tuple(src[::-1])]
        out[idx] = acc
    return out


@pytest.mark.parametrize("shape,shifts,p", [((8, 12), (0.37, -0.61), 4), ((9, 6), (-0.2, 0.45), 3),
                                            ((4, 6, 8), (0.3, -0.7, 0.15), 2)])
def test_glc_pull_matches_brute_force(shape, shifts, p):
    plane = np.random.default_rng(5).standard_normal(shape)
    lens = [2.0 * math.pi] * len(shape)
    got = G.pull_plane_glc(plane, np.array(shifts), p)
    want = brute_pull(plane, shifts, p, lens)
    assert np.abs(got - want).max() < 1e-12


def test_p1_is_the_equidistant_linear_pull():
    plane = np.random.default_rng(6).standard_normal((7, 10))
    shifts = np.array([0.43, -1.27])
    got = G.pull_plane_glc(plane, shifts, 1)
    want = O.pull_plane(plane, -shifts, 1)  # grid units: H = dx for p = 1
    assert np.abs(got - want).max() < 1e-14


@pytest.mark.parametrize("p", [2, 3, 4])
def test_polynomials_of_degree_p_are_exact_and_constants_kept(p):
    cells, L = 8, 8.0
    x = G.glc_positions(cells, p, L)
    shift = 0.37
    P = lambda t: 0.3 - 1.1 * t + 0.2 * t ** 2 + (0.05 * t ** p if p > 2 else 0.0)  # noqa: E731
    plane = np.tile(P(x), (p, 1))  # y: one cell, constant
    got = G.pull_plane_glc(plane, np.array([shift, 0.0]), p)[0]
    xd = x - shift * (L / cells)
    H = L / cells
    inside = (xd >= 0.0) & (np.floor(xd / H) < cells - 1)  # departure cells whose support does not wrap
    assert np.abs(got[inside] - P(xd[inside])).max() < 1e-11
    ones = np.ones((2 * p, cells * p))
    assert np.abs(G.pull_plane_glc(ones, np.array([0.81, -0.33]), p) - 1.0).max() < 1e-14


@pytest.mark.parametrize("p", [2, 3, 4])
def test_convergence_of_order_p_plus_one(p):
    errs = []
    for cells in (6, 12):
        x = G.glc_positions(cells, p, 2 * math.pi)
        H = 2 * math.pi / cells
        shift = 0.3
        plane = np.tile(np.sin(x), (p, 1))
        got = G.pull_plane_glc(plane, np.array([shift, 0.0]), p)[0]
        errs.append(np.abs(got - np.sin(x - shift * H)).max())
    # the same fraction of a cell on a grid twice as fine: error / 2^(p+1)
    assert errs[0] / errs[1] > 0.7 * 2 ** (p + 1), errs


def test_taylor_green_decay_on_a_glc_grid():
    """D2Q9 (c_s^2 = 1/3), N = 2, 16 x 16 cells of p = 4 (64 x 64 nodes),
    Courant 0.4 on the mean spacing, Re 100, 200 steps: the amplitude follows
    exp(-2 nu t) within 1e-3 (measured 2.4e-4)."""
    vs = V.get("D2Q9").scaled(1.0 / math.sqrt(3.0))
    p, cells = 4, 16
    n = cells * p
    L = 2 * math.pi
    dx = L / n
    dt = 0.4 * dx / np.abs(vs.xi).max()
    u0 = 0.05
    nu = u0 / 100.0
    prm = O.Params(vs, 2, p, dt=dt, dx=dx, tau=O.tau_isothermal(nu, vs.cs, dt))
    x = G.glc_positions(cells, p, L)
    Y, X = np.meshgrid(x, x, indexing="ij")
    u = np.stack([u0 * np.sin(X) * np.cos(Y), -u0 * np.cos(X) * np.sin(Y)])
    rho = 1.0 + (u0 ** 2 / 4.0) * (np.cos(2 * X) + np.cos(2 * Y)) / vs.cs ** 2
    f, _ = O.init_equilibrium(prm, rho, u)
    steps = 200
    for _ in range(steps):
        f, _, _ = G.step(prm, f)
    _, uu, _ = O.moments_of_state(prm, f)
    phi = np.sin(X) * np.cos(Y)
    amp = (uu[0] * phi).sum() / (phi * phi).sum() / u0
    assert abs(amp / math.exp(-2.0 * nu * steps * dt) - 1.0) < 1e-3


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_glc_points_are_the_chebyshev_lobatto_points(p):
    """GLC points on [-1, 1]: the end points and the zeros of T_p' (the
    extrema of the Chebyshev polynomial T_p), textbook definition."""
    from numpy.polynomial import chebyshev as C
    z = G.glc_points(p)
    x = 2.0 * z - 1.0
    assert x[0] == -1.0 and abs(x[-1] - 1.0) < 1e-15
    assert np.all(np.diff(x) > 0)
    dT = C.chebder([0] * p + [1])
    if p > 1:
        assert np.abs(C.chebval(x[1:-1], dT)).max() < 1e-10 * p * p
    assert np.abs(np.abs(C.chebval(x, [0] * p + [1])) - 1.0).max() < 1e-12  # |T_p| = 1 at every point

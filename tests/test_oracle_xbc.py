"""Pins of the oracle's non-periodic x (inflow at x < 0, zero-gradient outflow
at x >= nx; the standing-shock set-up of Sec. 4.1, whose boundary treatment
the paper does not state).

* The pull against a brute-force evaluation with explicit boundary lookups.
* A uniform field equal to the inflow state is a fixed point of the step.
* In a supersonic through-flow every characteristic leaves through the
  outflow: a density pulse is swept out and the domain returns to the inflow
  state (a periodic domain would keep the pulse).
"""
import math

import numpy as np
import pytest

from oracle import sllbm as O
from oracle import velocity_sets as V


def brute_pull(plane, delta, p, inflow):
    D = plane.ndim
    nx = plane.shape[-1]
    sts = [O.stencil_1d(float(delta[a]), p) for a in range(D)]
    out = np.zeros_like(plane)
    for idx in np.ndindex(plane.shape):
        pos = idx[::-1]  # (x, y[, z])
        acc = 0.0
        for js in np.ndindex(*([p + 1] * D)):
            w = 1.0
            src = []
            for a in range(D):
                m0, W = sts[a]
                w *= W[js[a]]
                src.append(pos[a] + m0 + js[a])
            if src[0] < 0:
                v = inflow
            else:
                xs = min(src[0], nx - 1)
                rest = [src[a] % plane.shape[D - 1 - a] for a in range(1, D)]
                v = plane[tuple(rest[::-1]) + (xs,)]
            acc += w * v
        out[idx] = acc
    return out


@pytest.mark.parametrize("shape,delta,p", [((5, 9), (0.37, -1.2), 3), ((4, 8), (-1.6, 0.4), 4),
                                           ((3, 4, 7), (1.3, -0.2, 0.7), 3), ((3, 4, 6), (-0.45, 0.0, -1.1), 4)])
def test_xbc_pull_matches_brute_force(shape, delta, p):
    rng = np.random.default_rng(41)
    plane = rng.standard_normal(shape)
    got = O.pull_plane_xbc(plane, np.array(delta), p, 0.75)
    want = brute_pull(plane, np.array(delta), p, 0.75)
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("name,N,comp", [("D2Q19", 4, True), ("D3Q27", 2, False)])
def test_uniform_inflow_state_is_a_fixed_point(name, N, comp):
    vs = V.get(name)
    dt = 0.4 / np.abs(vs.xi).max()
    if comp:
        prm = O.Params(vs, N, 4, dt=dt, dx=1.0, compressible=True, gamma=1.4, mu=0.05)
    else:
        prm = O.Params(vs, N, 4, dt=dt, dx=1.0, tau=0.8)
    grid = (4, 9) if vs.D == 2 else (3, 4, 9)
    u_in = np.zeros(vs.D)
    u_in[0] = 0.3 * vs.cs
    th_in = 1.1 if comp else 1.0
    f, g = O.init_equilibrium(prm, np.full(grid, 1.05), np.broadcast_to(u_in.reshape((vs.D,) + (1,) * vs.D),
                                                                         (vs.D,) + grid), np.full(grid, th_in))
    xbc = O.inflow_populations(prm, 1.05, u_in, th_in)
    f1, g1, _ = O.step(prm, f, g, xbc=xbc)
    assert np.abs(f1 - f).max() < 1e-13
    if comp:
        assert np.abs(g1 - g).max() < 1e-13


def test_supersonic_disturbance_leaves_the_domain():
    """D2Q19, N = 4, f + g, through-flow at Mach 1.7 (u = 2, c = sqrt(1.4)):
    a 1e-3 density pulse falls below 1e-6 after 320 steps."""
    vs = V.get("D2Q19")
    nx, ny = 48, 4
    dt = 0.4 / np.abs(vs.xi).max()
    prm = O.Params(vs, 4, 4, dt=dt, dx=1.0, compressible=True, gamma=1.4, mu=0.05)
    U = 2.0
    X = np.broadcast_to(np.arange(nx), (ny, nx))
    rho = 1.0 + 1e-3 * np.exp(-((X - 36) / 3.0) ** 2)
    u = np.stack([np.full((ny, nx), U), np.zeros((ny, nx))])
    f, g = O.init_equilibrium(prm, rho, u, np.ones((ny, nx)))
    xbc = O.inflow_populations(prm, 1.0, np.array([U, 0.0]), 1.0)
    for _ in range(320):
        f, g, _ = O.step(prm, f, g, xbc=xbc)
    r, uu, th = O.moments_of_state(prm, f, g)
    assert math.sqrt(1.4) < U
    assert np.abs(r - 1.0).max() < 1e-6
    assert np.abs(uu[0] - U).max() < 1e-6
    assert np.abs(th - 1.0).max() < 1e-6

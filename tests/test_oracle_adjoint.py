"""Pins of the adjoint oracle (exact transpose of one isothermal step, Sec. 3).

Each pin ties the adjoint to something other than itself:

* the dot-product identity <lam, S f> = <S^T lam, f> against the forward
  pull, which is pinned on its own (Fourier symbol, brute force);
* central finite differences of the forward oracle: the equilibrium
  (Appendix A), the moments (Sec. 3), one whole step and a short trajectory;
* the conservation invariants of BGK: the collision keeps rho and j, so the
  transposed collision Jacobian maps 1 to 1 and xi_a to xi_a;
* the on-lattice special case (D2Q9, dt = dx), where S^T is the opposite
  periodic shift.
"""
import math

import numpy as np
import pytest

from oracle import adjoint as A
from oracle import sllbm as O
from oracle import velocity_sets as V


def params(name, N, p, courant=0.4, tau=0.7, cs=None):
    vs = V.get(name)
    if cs is not None:
        vs = vs.scaled(cs)
    dx = 0.1
    dt = courant * dx / np.abs(vs.xi).max()
    return O.Params(vs, N, p, dt=dt, dx=dx, tau=tau)


def state(prm, grid, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    D = prm.vs.D
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, grid)
    u = 0.08 * prm.vs.cs * rng.uniform(-1, 1, (D,) + grid)
    f, _ = O.init_equilibrium(prm, rho, u)
    return f * (1.0 + amp * rng.uniform(-1, 1, f.shape))


@pytest.mark.parametrize("name,p,grid", [("D2Q9", 3, (9, 11)), ("D2Q25", 4, (10, 13)), ("D3Q27", 3, (5, 6, 7)),
                                         ("D3Q13", 2, (6, 5, 7)), ("D3Q45", 4, (6, 7, 5))])
def test_pull_transpose_dot_product(name, p, grid):
    prm = params(name, 2, p, courant=1.3)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((prm.vs.Q,) + grid)
    lam = rng.standard_normal((prm.vs.Q,) + grid)
    lhs = (lam * O.pull_state(prm, f)).sum()
    rhs = (A.pull_state_transpose(prm, lam) * f).sum()
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(lam).sum() * np.abs(f).max())


def test_pull_transpose_on_lattice_is_opposite_shift():
    vs = V.get("D2Q9").scaled(1.0 / math.sqrt(3.0))
    prm = O.Params(vs, 2, 3, dt=0.1, dx=0.1, tau=0.8)
    lam = np.random.default_rng(4).standard_normal((9, 8, 10))
    got = A.pull_state_transpose(prm, lam)
    for i in range(9):
        cx, cy = int(round(vs.xi[i][0])), int(round(vs.xi[i][1]))
        # the pull reads f(x - c); its transpose writes lam to x - c
        want = np.roll(np.roll(lam[i], -cx, axis=1), -cy, axis=0)
        assert np.allclose(got[i], want, atol=1e-14)


@pytest.mark.parametrize("name,N,cs", [("D2Q9", 2, 1 / math.sqrt(3)), ("D3Q27", 2, None), ("D3V27", 3, None),
                                       ("D3Q45", 4, None), ("D2Q25", 3, None)])
def test_equilibrium_derivatives_match_finite_differences(name, N, cs):
    vs = V.get(name) if cs is None else V.get(name).scaled(cs)
    rng = np.random.default_rng(5)
    M, D = 7, vs.D
    rho = 1.0 + 0.1 * rng.uniform(-1, 1, M)
    j = rho[:, None] * 0.1 * vs.cs * rng.uniform(-1, 1, (M, D))
    d_rho, d_j = A.equilibrium_derivatives(vs, rho, j, N)

    def feq(r, jj):
        return O.equilibrium(vs, r, jj / r[:, None], np.ones_like(r), N)

    h = 1e-6
    fd = (feq(rho + h, j) - feq(rho - h, j)) / (2 * h)
    assert np.allclose(d_rho, fd, atol=1e-8, rtol=0)
    for a in range(D):
        e = np.zeros(D)
        e[a] = h
        fd = (feq(rho, j + e) - feq(rho, j - e)) / (2 * h)
        assert np.allclose(d_j[:, :, a], fd, atol=1e-8, rtol=0)


@pytest.mark.parametrize("name,N", [("D2Q9", 2), ("D3Q27", 3), ("D3Q45", 4)])
def test_collision_adjoint_conserves(name, N):
    prm = params(name, N, 3, tau=0.63)
    f = state(prm, (4, 5) if prm.vs.D == 2 else (3, 4, 5), 6).reshape(prm.vs.Q, -1)
    ones = np.ones_like(f)
    assert np.allclose(A.collide_vjp(prm, f, ones), 1.0, atol=1e-12)
    for a in range(prm.vs.D):
        xa = np.repeat(prm.vs.xi[:, a:a + 1], f.shape[1], axis=1)
        assert np.allclose(A.collide_vjp(prm, f, xa), xa, atol=1e-12)


@pytest.mark.parametrize("name,N,p,grid", [("D2Q9", 2, 3, (8, 9)), ("D2Q19", 3, 4, (7, 8)),
                                           ("D3Q27", 2, 3, (4, 5, 6)), ("D3Q45", 4, 4, (5, 4, 6))])
def test_step_vjp_matches_finite_differences(name, N, p, grid):
    prm = params(name, N, p, courant=0.8, tau=0.61)
    f = state(prm, grid, 7, amp=1e-2)
    rng = np.random.default_rng(8)
    lam = rng.standard_normal(f.shape)
    v = rng.standard_normal(f.shape)
    g = A.step_vjp(prm, f, lam)
    h = 1e-6
    fp, _, _ = O.step(prm, f + h * v)
    fm, _, _ = O.step(prm, f - h * v)
    fd = (lam * (fp - fm)).sum() / (2 * h)
    assert abs((g * v).sum() - fd) <= 1e-7 * max(1.0, abs(fd))


def test_trajectory_vjp_of_kinetic_energy_matches_finite_differences():
    prm = params("D3Q27", 2, 3, courant=0.4, tau=0.58)
    vs = prm.vs
    grid = (4, 5, 6)
    f0 = state(prm, grid, 9, amp=1e-2)
    Q = vs.Q

    def J(f):
        rho, u = O.density_momentum(vs, f.reshape(Q, -1))
        return 0.5 * (u ** 2).sum(axis=1).mean()

    fT = f0
    for _ in range(3):
        fT, _, _ = O.step(prm, fT)
    rho, u = O.density_momentum(vs, fT.reshape(Q, -1))
    M = rho.shape[0]
    lamT = A.moments_vjp(vs, fT.reshape(Q, -1), np.zeros(M), u / M).reshape(fT.shape)
    lam0, _ = A.trajectory_vjp(prm, f0, 3, lamT)
    v = np.random.default_rng(10).standard_normal(f0.shape)
    h = 1e-6

    def run(f):
        for _ in range(3):
            f, _, _ = O.step(prm, f)
        return J(f)

    fd = (run(f0 + h * v) - run(f0 - h * v)) / (2 * h)
    assert abs((lam0 * v).sum() - fd) <= 1e-6 * abs(fd)


def test_moments_vjp_matches_finite_differences():
    vs = V.get("D2Q25")
    rng = np.random.default_rng(11)
    prm = params("D2Q25", 3, 3)
    f = state(prm, (3, 4), 12, amp=1e-2).reshape(vs.Q, -1)
    M = f.shape[1]
    gr = rng.standard_normal(M)
    gu = rng.standard_normal((M, 2))
    lam = A.moments_vjp(vs, f, gr, gu)
    v = rng.standard_normal(f.shape)
    h = 1e-6

    def J(ff):
        rho, u = O.density_momentum(vs, ff)
        return (gr * rho).sum() + (gu * u).sum()

    fd = (J(f + h * v) - J(f - h * v)) / (2 * h)
    assert abs((lam * v).sum() - fd) <= 1e-8 * max(1.0, abs(fd))


@pytest.mark.parametrize("name,N", [("D3Q27", 2), ("D2Q25", 4)])
def test_equilibrium_vjp_matches_finite_differences(name, N):
    vs = V.get(name)
    rng = np.random.default_rng(13)
    M, D = 6, vs.D
    rho = 1.0 + 0.1 * rng.uniform(-1, 1, M)
    u = 0.1 * vs.cs * rng.uniform(-1, 1, (M, D))
    lam = rng.standard_normal((vs.Q, M))
    gr, gu = A.equilibrium_vjp(vs, N, rho, u, lam)
    h = 1e-6

    def J(r, uu):
        return (lam * O.equilibrium(vs, r, uu, np.ones_like(r), N)).sum()

    dr = rng.standard_normal(M)
    du = rng.standard_normal((M, D))
    fd = (J(rho + h * dr, u + h * du) - J(rho - h * dr, u - h * du)) / (2 * h)
    assert abs((gr * dr).sum() + (gu * du).sum() - fd) <= 1e-8 * max(1.0, abs(fd))


def test_compressible_adjoint_is_rejected():
    vs = V.get("D3Q45")
    prm = O.Params(vs, 4, 3, dt=0.01, dx=0.1, compressible=True, mu=1e-3)
    with pytest.raises(ValueError):
        A.collide_vjp(prm, np.ones((45, 2)), np.ones((45, 2)))


def test_collision_jacobian_depends_on_the_moments_only():
    """The isothermal collision's Jacobian at f~ depends on f~ only through its
    moments (rho, j): two pulled states with the same rho and j but different
    higher moments give the same directional derivative of the forward
    collision (central differences of the forward oracle, no adjoint code),
    while a different momentum changes it.  This is why the library's tape
    keeps four moments per node for the adjoint."""
    vs = V.get("D3Q27")
    prm = O.Params(vs, 2, 4, dt=0.05, dx=0.1, tau=0.8)
    rng = np.random.default_rng(11)
    M = 6
    rho = 1.0 + 0.05 * rng.standard_normal(M)
    u = 0.05 * rng.standard_normal((M, 3))
    f1 = O.equilibrium(vs, rho, u, np.ones(M), 2) * (1.0 + 0.01 * rng.standard_normal((vs.Q, M)))
    # a perturbation with no mass and no momentum: project out span{1, xi_a}
    basis = np.column_stack([np.ones(vs.Q), vs.xi])               # (Q, 4)
    d = 1e-3 * rng.standard_normal((vs.Q, M))
    d -= basis @ np.linalg.lstsq(basis, d, rcond=None)[0]
    f2 = f1 + d
    assert np.abs(basis.T @ d).max() < 1e-15
    v = rng.standard_normal((vs.Q, M))
    sigma = rng.standard_normal((vs.Q, M))

    def dderiv(f, eps=1e-6):
        plus = O.collide(prm, f + eps * v)[0]
        minus = O.collide(prm, f - eps * v)[0]
        return (sigma * (plus - minus) / (2 * eps)).sum(axis=0)

    g1, g2 = dderiv(f1), dderiv(f2)
    assert np.abs(g1 - g2).max() < 1e-7 * np.abs(g1).max()
    # control: a change of momentum does change the Jacobian
    f3 = f1 + 1e-2 * np.outer(vs.xi[:, 0], np.ones(M)) * vs.w[:, None]
    assert np.abs(dderiv(f3) - g1).max() > 1e-4 * np.abs(g1).max()

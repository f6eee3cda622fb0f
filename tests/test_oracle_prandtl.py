"""Pins of the oracle's Prandtl-number model (Sec. 3: a quasi-equilibrium
varies Pr; the form is the heat-flux quasi-equilibrium read in oracle/sllbm.py).

* An isobaric temperature wave theta = 1 + eps sin x (rho = 1/theta, u = 0)
  is an entropy mode of the Navier-Stokes-Fourier equations; it decays at the
  thermal diffusivity kappa / (rho c_p) = nu / Pr.  Measured within 0.5 % for
  Pr = 0.5 ... 2; doubling either projection, or leaving out the one of f or
  of g, moves it by 11-21 %.
* A shear wave keeps the viscosity mu / rho at any Pr (the heat-flux
  projection carries no stress).
* Collision moments on random pulled states: mass, momentum and energy are
  kept; the non-equilibrium stress relaxes at tau and the central heat flux
  of f and the central first moment of g at tau_2 = 1/2 + (tau - 1/2)/Pr.
"""
import math

import numpy as np
import pytest

from oracle import sllbm as O
from oracle import velocity_sets as V


def thermal_diffusivity(Pr, mu=0.02, n=32, ny=4, steps=120, eps=1e-3):
    """Decay rate of the entropy s = ln theta - ((gamma - 1)/gamma) ln P of
    the wave (k = 1), D2Q25, N = 4, p = 4."""
    vs = V.get("D2Q25")
    dx = 2 * math.pi / n
    dt = 0.4 * dx / np.abs(vs.xi).max()
    prm = O.Params(vs, 4, 4, dt=dt, dx=dx, compressible=True, gamma=1.4, mu=mu, prandtl=Pr)
    X = np.broadcast_to(np.arange(n) * dx, (ny, n))
    theta = 1.0 + eps * np.sin(X)
    f, g = O.init_equilibrium(prm, 1.0 / theta, np.zeros((2, ny, n)), theta)
    gm = (prm.gamma - 1.0) / prm.gamma

    def amp(f, g):
        rho, _, th = O.moments_of_state(prm, f, g)
        s = np.log(th) - gm * np.log(rho * th)
        return 2.0 * (s * np.sin(X)).mean()

    for _ in range(10):  # let the heat flux build up from the equilibrium start
        f, g, _ = O.step(prm, f, g)
    a1 = amp(f, g)
    for _ in range(steps):
        f, g, _ = O.step(prm, f, g)
    return -math.log(amp(f, g) / a1) / (steps * dt)


@pytest.mark.parametrize("Pr", [1.0, 0.75, 0.5, 2.0])
def test_temperature_wave_decays_at_nu_over_prandtl(Pr):
    alpha = thermal_diffusivity(Pr)
    assert abs(alpha / (0.02 / Pr) - 1.0) < 1e-2, alpha


def test_shear_wave_viscosity_does_not_depend_on_prandtl():
    vs = V.get("D2Q25")
    n, ny, mu, steps = 32, 4, 0.02, 120
    dx = 2 * math.pi / n
    dt = 0.4 * dx / np.abs(vs.xi).max()
    rates = []
    for Pr in (1.0, 0.75):
        prm = O.Params(vs, 4, 4, dt=dt, dx=dx, compressible=True, gamma=1.4, mu=mu, prandtl=Pr)
        X = np.broadcast_to(np.arange(n) * dx, (ny, n))
        u = np.stack([np.zeros((ny, n)), 1e-3 * np.sin(X)])
        f, g = O.init_equilibrium(prm, np.ones((ny, n)), u, np.ones((ny, n)))
        for _ in range(10):
            f, g, _ = O.step(prm, f, g)
        a1 = 2.0 * (O.moments_of_state(prm, f, g)[1][1] * np.sin(X)).mean()
        for _ in range(steps):
            f, g, _ = O.step(prm, f, g)
        a2 = 2.0 * (O.moments_of_state(prm, f, g)[1][1] * np.sin(X)).mean()
        rates.append(-math.log(a2 / a1) / (steps * dt))
    assert abs(rates[0] / mu - 1.0) < 2e-3
    assert abs(rates[1] / rates[0] - 1.0) < 1e-4, rates


def _central_moments(vs, h, u, T0):
    zeta = vs.xi[:, None, :] - u[None, :, :]
    z2 = (zeta ** 2).sum(axis=2)
    stress = np.einsum("im,ima,imb->mab", h, zeta, zeta, optimize=False)
    heat = np.einsum("im,im,ima->ma", h, z2, zeta, optimize=False)
    first = np.einsum("im,ima->ma", h, zeta, optimize=False)
    return stress, heat, first


@pytest.mark.parametrize("name", ["D2Q19", "D2Q25", "D3Q45"])
@pytest.mark.parametrize("Pr", [0.75, 1.6])
def test_collision_moments(name, Pr):
    vs = V.get(name)
    T0 = vs.cs ** 2
    rng = np.random.default_rng(7)
    M = 16
    prm = O.Params(vs, 4, 4, dt=0.05, dx=0.1, compressible=True, gamma=1.4, mu=0.01, prandtl=Pr)
    rho = 1.0 + 0.1 * rng.standard_normal(M)
    u = 0.3 * vs.cs * rng.standard_normal((M, vs.D))
    theta = 1.0 + 0.1 * rng.standard_normal(M)
    feq0 = O.equilibrium(vs, rho, u, theta, 4)
    Cv = 1.0 / (prm.gamma - 1.0)
    ft = feq0 * (1.0 + 0.05 * rng.standard_normal(feq0.shape))
    gt = theta[None, :] * (2 * Cv - vs.D) * feq0 * (1.0 + 0.05 * rng.standard_normal(feq0.shape))
    fp, gp, diag = O.collide(prm, ft, gt)
    # collision invariants: mass, momentum, total energy sum(|xi|^2 f / T0 + g)
    xi2 = (vs.xi ** 2).sum(axis=1)
    np.testing.assert_allclose(fp.sum(0), ft.sum(0), rtol=1e-13)
    np.testing.assert_allclose(vs.xi.T @ fp, vs.xi.T @ ft, atol=1e-13)
    np.testing.assert_allclose(xi2 @ fp / T0 + gp.sum(0), xi2 @ ft / T0 + gt.sum(0), rtol=1e-13)
    # relaxation of the non-equilibrium moments
    tau = diag["tau"]
    tau2 = 0.5 + (tau - 0.5) / Pr
    uu, feq = diag["u"], diag["feq"]
    geq = diag["theta"][None, :] * (2 * Cv - vs.D) * feq
    s_pre, h_pre, _ = _central_moments(vs, ft - feq, uu, T0)
    s_post, h_post, _ = _central_moments(vs, fp - feq, uu, T0)
    _, _, g_pre = _central_moments(vs, gt - geq, uu, T0)
    _, _, g_post = _central_moments(vs, gp - geq, uu, T0)
    scale = np.abs(s_pre).max()
    np.testing.assert_allclose(s_post, (1 - 1 / tau)[:, None, None] * s_pre, atol=1e-12 * scale)
    np.testing.assert_allclose(h_post, (1 - 1 / tau2)[:, None] * h_pre, atol=1e-12 * np.abs(h_pre).max())
    np.testing.assert_allclose(g_post, (1 - 1 / tau2)[:, None] * g_pre, atol=1e-12 * np.abs(g_pre).max())
    # the heat-flux relaxation differs from the stress relaxation
    assert np.abs((1 - 1 / tau2) - (1 - 1 / tau)).min() > 1e-3


def test_prandtl_one_is_bgk():
    vs = V.get("D2Q25")
    rng = np.random.default_rng(3)
    a = O.Params(vs, 4, 4, dt=0.05, dx=0.1, compressible=True, mu=0.01)
    b = O.Params(vs, 4, 4, dt=0.05, dx=0.1, compressible=True, mu=0.01, prandtl=1.0)
    f = np.abs(rng.standard_normal((vs.Q, 5))) * vs.w[:, None]
    g = np.abs(rng.standard_normal((vs.Q, 5))) * vs.w[:, None]
    fa, ga, _ = O.collide(a, f, g)
    fb, gb, _ = O.collide(b, f, g)
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    with pytest.raises(ValueError):
        O.Params(vs, 2, 4, dt=0.05, dx=0.1, tau=0.8, prandtl=0.75)

"""Run parameters from flow numbers (host helper of the product path).

Relaxation times follow Sec. 3: tau = nu / (c_s^2 dt) + 1/2 (isothermal) and
tau = mu / (c_s^2 dt P) + 1/2 (compressible, P = rho theta).  The Courant
number is read as C = max_{i,alpha} |xi_{i,alpha}| dt / dx, the largest
departure offset in grid units, so dt = C dx / max |xi_{i,alpha}|.
"""
import math
from dataclasses import dataclass

from . import olb


def tau_isothermal(nu, cs, dt):
    return nu / (cs * cs * dt) + 0.5


def tau_compressible(mu, cs, dt, P=1.0):
    return mu / (cs * cs * dt * P) + 0.5


@dataclass
class RunParams:
    velocity_set: str
    n: int
    dim: int
    dx: float
    dt: float
    cs_scale: float
    cs: float
    u0: float
    tau: float
    nu: float = 0.0
    mu: float = 0.0
    compressible: bool = False
    gamma: float = 1.4


def tgv_isothermal(velocity_set, n, Re, Ma, courant, L=1.0):
    """Weakly compressible TGV on [0, 2 pi)^D with velocity unit u0 = 1.

    c_s = u0 / Ma sets the abscissae scale (the set's own c_s is rescaled),
    nu = u0 L / Re, dx = 2 pi / n, dt from the Courant number.
    """
    Q, D, cs_set, max_xi, _ = olb.velocity_set_info(velocity_set)
    u0 = 1.0
    cs = u0 / Ma
    s = cs / cs_set
    dx = 2.0 * math.pi / n
    dt = courant * dx / (max_xi * s)
    nu = u0 * L / Re
    return RunParams(velocity_set, n, D, dx, dt, s, cs, u0, tau_isothermal(nu, cs, dt), nu=nu)


def tgv2d_lattice(n=64, u0=0.05, Re=100.0, courant=0.4, L=1.0):
    """2D TGV with D2Q9 rescaled to c_s^2 = 1/3 (abscissae 0, +-1) and u0 in those units."""
    _, _, cs_set, max_xi, _ = olb.velocity_set_info("D2Q9")
    s = 1.0 / math.sqrt(3.0) / cs_set
    cs = cs_set * s
    dx = 2.0 * math.pi / n
    dt = courant * dx / (max_xi * s)
    nu = u0 * L / Re
    return RunParams("D2Q9", n, 2, dx, dt, s, cs, u0, tau_isothermal(nu, cs, dt), nu=nu)


def tgv_compressible(velocity_set, n, Re, Ma, courant, gamma=1.4, L=1.0):
    """Compressible TGV with c_s = 1 (T0 = 1): u0 = Ma c_s sqrt(gamma),
    mu = rho0 u0 L / Re, tau reported at theta = 1, rho = 1."""
    Q, D, cs_set, max_xi, _ = olb.velocity_set_info(velocity_set)
    if abs(cs_set - 1.0) > 1e-12:
        raise ValueError("compressible runs need a set with c_s = 1")
    u0 = Ma * math.sqrt(gamma)
    dx = 2.0 * math.pi / n
    dt = courant * dx / max_xi
    mu = u0 * L / Re
    return RunParams(velocity_set, n, D, dx, dt, 1.0, 1.0, u0, tau_compressible(mu, 1.0, dt), mu=mu,
                     compressible=True, gamma=gamma)

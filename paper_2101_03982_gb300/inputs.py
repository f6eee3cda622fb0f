"""Seeded synthetic inputs (macroscopic fields) for tests and benchmarks.

This module holds only the workloads' initial fields and seeded noise; none
of the method's arithmetic (no equilibrium, stencil or collision).  Both the
CUDA path and the oracle consume what it returns.  Arrays are numpy FP64 in
[z][y][x] order (x fastest); vector fields are structure-of-arrays [D][...].
Nodes sit at x_i = i dx with dx = 2 pi / n on the periodic box [0, 2 pi)^D.
"""
import math

import numpy as np


def _axes(shape_xyz):
    return [np.arange(n) * (2.0 * np.pi / n) for n in shape_xyz]


def tgv2d(n, u0, cs2, rho0=1.0):
    """2D decaying Taylor-Green vortex: u = u0 (sin x cos y, -cos x sin y).

    The pressure perturbation that balances u.grad(u) for this velocity field,
    p' = +(rho0 u0^2 / 4)(cos 2x + cos 2y), gives rho = rho0 + p'/c_s^2
    (isothermal equation of state p = rho c_s^2).
    Returns rho (n, n) and u (2, n, n).
    """
    x, y = _axes((n, n))
    Y, X = np.meshgrid(y, x, indexing="ij")
    u = np.stack([u0 * np.sin(X) * np.cos(Y), -u0 * np.cos(X) * np.sin(Y)])
    p = (rho0 * u0 ** 2 / 4.0) * (np.cos(2 * X) + np.cos(2 * Y))
    return rho0 + p / cs2, u


def tgv3d(n, u0, cs2, rho0=1.0):
    """3D Taylor-Green vortex of Sec. 4.2 (Brachet initial condition).

    u = u0 (sin x cos y cos z, -cos x sin y cos z, 0) and
    P' = (rho0 u0^2 / 16)(cos 2x + cos 2y)(cos 2z + 2), the paper's pressure
    with its "cos(2z+2)" read as cos(2z) + 2; rho = rho0 + P'/c_s^2.
    Returns rho (n, n, n) and u (3, n, n, n).
    """
    x, y, z = _axes((n, n, n))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u = np.stack([u0 * np.sin(X) * np.cos(Y) * np.cos(Z), -u0 * np.cos(X) * np.sin(Y) * np.cos(Z),
                  np.zeros_like(X)])
    p = (rho0 * u0 ** 2 / 16.0) * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    return rho0 + p / cs2, u


def ctic3d(n, u0, C=1.0):
    """Compressible TGV with constant temperature (Sec. 4.3): theta = 1,
    rho = 1 + (C^2/16)(cos 2x + cos 2y)(cos 2z + 2), u as in ``tgv3d``.
    Returns rho, u, theta."""
    x, y, z = _axes((n, n, n))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u = np.stack([u0 * np.sin(X) * np.cos(Y) * np.cos(Z), -u0 * np.cos(X) * np.sin(Y) * np.cos(Z),
                  np.zeros_like(X)])
    rho = 1.0 + (C ** 2 / 16.0) * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    return rho, u, np.ones_like(rho)


def rankine_hugoniot(Ma, gamma):
    """Downstream/upstream density and pressure ratios and downstream Mach
    number of a normal shock (textbook relations)."""
    M2 = Ma * Ma
    r = (gamma + 1.0) * M2 / ((gamma - 1.0) * M2 + 2.0)
    p = 1.0 + 2.0 * gamma / (gamma + 1.0) * (M2 - 1.0)
    Mb = math.sqrt((1.0 + 0.5 * (gamma - 1.0) * M2) / (gamma * M2 - 0.5 * (gamma - 1.0)))
    return r, p, Mb


def shock_vortex(nx, ny, Ma_a=1.2, Ma_v=0.25, radius=None, gamma=1.4, width=2.0):
    """Shock-vortex field of Sec. 4.1 on an nx x ny grid (grid units, c_s = 1).

    Upstream (x < nx/2): rho = 1, theta = 1, u = Ma_a sqrt(gamma); downstream the
    Rankine-Hugoniot state; the jump is smoothed by tanh over `width` nodes.  An
    isentropic vortex of radius R (default 0.075 ny) sits at x = nx/4, y = ny/2:
    u_theta = sqrt(gamma) Ma_v (r/R) exp((1 - (r/R)^2)/2),
    T = 1 - (gamma-1)/2 Ma_v^2 exp(1 - (r/R)^2) (the paper's bracket read with
    Ma_v^2), rho = T^(1/(gamma-1)).  Returns rho, u (2, ny, nx), theta.
    """
    R = 0.075 * ny if radius is None else radius
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    Y, X = np.meshgrid(y, x, indexing="ij")
    r_rho, r_p, _ = rankine_hugoniot(Ma_a, gamma)
    c1 = math.sqrt(gamma)
    u1 = Ma_a * c1
    s = 0.5 * (1.0 + np.tanh((X - 0.5 * nx) / width))
    rho = 1.0 + (r_rho - 1.0) * s
    theta = 1.0 + (r_p / r_rho - 1.0) * s
    ux = u1 + (u1 / r_rho - u1) * s
    dx, dy = X - 0.25 * nx, Y - 0.5 * ny
    rr = np.sqrt(dx * dx + dy * dy) / R
    ut = c1 * Ma_v * rr * np.exp(0.5 * (1.0 - rr * rr))
    with np.errstate(invalid="ignore", divide="ignore"):
        ex = np.where(rr > 0, -dy / (rr * R), 0.0)
        ey = np.where(rr > 0, dx / (rr * R), 0.0)
    Tv = 1.0 - 0.5 * (gamma - 1.0) * Ma_v ** 2 * np.exp(1.0 - rr * rr)
    rho = rho * Tv ** (1.0 / (gamma - 1.0))
    theta = theta * Tv
    u = np.stack([ux + ut * ex, ut * ey])
    return rho, u, theta


def noise(shape, seed, amplitude):
    """Seeded uniform noise in [-amplitude, amplitude)."""
    rng = np.random.default_rng(seed)
    return amplitude * (2.0 * rng.random(shape) - 1.0)


def random_fields(shape_zyx, dim, seed, u_amp=0.05, rho_amp=0.02, theta_amp=0.0):
    """Smooth-ish seeded random fields: rho = 1 + noise, u = noise, theta = 1 + noise."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * (2.0 * rng.random(shape_zyx) - 1.0)
    u = u_amp * (2.0 * rng.random((dim,) + tuple(shape_zyx)) - 1.0)
    theta = 1.0 + theta_amp * (2.0 * rng.random(shape_zyx) - 1.0)
    return rho, u, theta


def solenoidal(n, rng, rms, kmin=1, kmax=4):
    """Divergence-free random velocity on an n^3 periodic grid, array (3, n, n, n).

    The curl of a random vector potential whose Fourier modes have integer
    wavenumbers with kmin <= |k| <= kmax and Gaussian amplitudes, scaled to
    the given root-mean-square speed.  ``rng`` is a numpy Generator, so a
    sequence of fields can be drawn from one seeded stream.
    """
    k1 = np.fft.fftfreq(n, 1.0 / n)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    band = (kk >= kmin) & (kk <= kmax)
    A = []
    for _ in range(3):
        spec = (rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))) * band
        A.append(np.real(np.fft.ifftn(spec)))
    Ah = [np.fft.fftn(a) for a in A]  # components x, y, z
    ik = [1j * kx, 1j * ky, 1j * kz]
    ux = np.real(np.fft.ifftn(ik[1] * Ah[2] - ik[2] * Ah[1]))
    uy = np.real(np.fft.ifftn(ik[2] * Ah[0] - ik[0] * Ah[2]))
    uz = np.real(np.fft.ifftn(ik[0] * Ah[1] - ik[1] * Ah[0]))
    u = np.stack([ux, uy, uz])
    return u * (rms / math.sqrt((u ** 2).sum(axis=0).mean()))

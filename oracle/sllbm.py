"""Plain FP64 oracle of the semi-Lagrangian lattice Boltzmann (SLLBM) time step.

TEST INFRASTRUCTURE ONLY.  Nothing under ``oracle/`` is part of the product
path: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library.

Every function follows the paper (arXiv:2101.03982) step by step, in its order
and notation, with no blocking or fusion:

* streaming: Sec. 3, Eq. (sl_streaming) -- the population of velocity i at x is
  the interpolant of the post-collision field evaluated at the departure point
  x - xi_i dt.  On the uniform periodic grid of this build the interpolant is a
  tensor product of equidistant Lagrange polynomials of degree p around the
  departure point (a reading: the paper uses cell-wise Gauss-Lobatto-Chebyshev
  elements).  The oracle evaluates the full (p+1)^D tensor-product sum directly.
* moments: Sec. 3, Eqs. (density), (momentum); temperature: Sec. 3, the
  relation 2 rho C_v theta = sum(|zeta_i|^2 f_i / T0 + g_i).
* equilibrium: Sec. 3 Hermite series, with the literal Hermite tensors and the
  literal equilibrium moments of Appendix A, contracted in full.
* collision: Sec. 3 BGK; compressible relaxation time tau = mu/(c_s^2 dt P)+1/2
  with P = rho theta T0 and g^eq = theta (2 C_v - D) f^eq.  The dynamic
  viscosity is constant in the paper; the optional power law
  mu(theta) = mu theta^omega (omega = mu_exponent, 0 by default) is a
  builder's extension, pinned by the decay of a shear wave at two
  temperatures (the model's kinematic viscosity is mu(theta)/rho).
* Prandtl number (Sec. 3 states that a quasi-equilibrium varies Pr and
  gives no formula): the reading here is the heat-flux quasi-equilibrium of
  two-population kinetic models.  f* equals f^eq except that its central heat
  flux sum_i f*_i zeta_i |zeta_i|^2 is that of the pulled f, and g* equals g^eq
  except that its central first moment sum_i g*_i zeta_i is that of the pulled
  g; the step relaxes to f* at tau and from f* to f^eq at
  tau_2 = 1/2 + (tau - 1/2)/Pr, so the heat flux relaxes at tau_2 and every
  other non-conserved moment at tau.  ``quasi_equilibrium`` builds f* and g*
  as f^eq and g^eq plus the Hermite projections of the two non-equilibrium
  fluxes (exact on sets of degree >= 7).  Pinned by the decay of an isobaric
  temperature wave (thermal diffusivity nu/Pr) and by a shear wave that keeps
  its viscosity at any Pr.

Readings where the paper is silent (each listed in the design notes):
T0 = c_s^2 of the set; C_v = 1/(gamma - 1); one step = pull, then collide, and
the stored state is post-collision; f at t = 0 is the equilibrium of the
initial fields.

Parity pins: see tests/test_oracle_*.py (``reductions`` and the gather form
``step_at_points`` in tests/test_oracle_reductions.py).  The dissipation estimator
``strain_dissipation`` is a builder's quantity (no formula in the paper),
pinned by the analytic strain of the decaying 3D Taylor-Green vortex.
"""
import itertools
import math

import numpy as np

# ----------------------------------------------------------------------------
# Stencil of the pull (Sec. 3, Eq. sl_streaming; uniform-grid reading)
# ----------------------------------------------------------------------------


def stencil_1d(delta, p):
    """Support points m_0..m_p and Lagrange weights W_0..W_p at offset delta.

    delta is the departure offset in grid units along one axis,
    delta = -xi_alpha dt / dx.  The p+1 equidistant integer points surround
    delta: for odd p, m_0 = floor(delta) - (p-1)/2; for even p,
    m_0 = floor(delta + 1/2) - p/2.  W_j is the Lagrange basis polynomial of
    point m_j evaluated at delta, computed as the literal product.
    """
    if p % 2 == 1:
        m0 = math.floor(delta) - (p - 1) // 2
    else:
        m0 = math.floor(delta + 0.5) - p // 2
    m = [m0 + j for j in range(p + 1)]
    W = []
    for j in range(p + 1):
        prod = 1.0
        for k in range(p + 1):
            if k != j:
                prod *= (delta - m[k]) / (m[j] - m[k])
        W.append(prod)
    return m0, np.array(W, dtype=np.float64)


def departure_offsets(xi, dt, dx):
    """delta_{i,alpha} = -xi_{i,alpha} dt / dx (grid units)."""
    return -np.asarray(xi, dtype=np.float64) * dt / dx


def pull_plane(plane, delta, p):
    """Interpolate one population field at the departure points (direct sum).

    plane has shape (ny, nx) or (nz, ny, nx), x fastest, periodic.  delta holds
    the per-axis offsets (x, y[, z]).  Returns sum over all (p+1)^D stencil
    tuples of prod_alpha W_alpha[j_alpha] * plane(x + m).
    """
    D = plane.ndim
    sts = [stencil_1d(float(delta[a]), p) for a in range(D)]
    out = np.zeros_like(plane)
    for js in itertools.product(range(p + 1), repeat=D):
        weight = 1.0
        shifts = []
        for a in range(D):
            m0, W = sts[a]
            weight *= W[js[a]]
            shifts.append(m0 + js[a])
        # array axes are ordered (z, y, x); axis a (x=0) is array axis D-1-a.
        rolled = plane
        for a in range(D):
            rolled = np.roll(rolled, -shifts[a], axis=D - 1 - a)
        out += weight * rolled
    return out


def pull_plane_xbc(plane, delta, p, inflow):
    """The pull of ``pull_plane`` with non-periodic x (the standing-shock set-up
    of Sec. 4.1): departure points left of the domain (x < 0) read the inflow
    value, a fixed post-collision equilibrium, and points right of it
    (x >= nx) read the last column (zero-gradient outflow); y and z stay
    periodic.  This boundary treatment is a reading: the paper states none.
    """
    D = plane.ndim
    nx = plane.shape[-1]
    sts = [stencil_1d(float(delta[a]), p) for a in range(D)]
    pad = p + int(math.ceil(abs(float(delta[0])))) + 1
    left = np.full(plane.shape[:-1] + (pad,), float(inflow))
    right = np.repeat(plane[..., -1:], pad, axis=-1)
    ext = np.concatenate([left, plane, right], axis=-1)
    out = np.zeros_like(plane)
    for js in itertools.product(range(p + 1), repeat=D):
        weight = 1.0
        shifts = []
        for a in range(D):
            m0, W = sts[a]
            weight *= W[js[a]]
            shifts.append(m0 + js[a])
        moved = ext[..., pad + shifts[0]:pad + shifts[0] + nx]
        for a in range(1, D):
            moved = np.roll(moved, -shifts[a], axis=D - 1 - a)
        out += weight * moved
    return out


def inflow_populations(prm, rho, u, theta=1.0):
    """Equilibrium populations (f_in, g_in or None) of one inflow state."""
    vs = prm.vs
    feq = equilibrium(vs, np.array([float(rho)]), np.asarray(u, dtype=np.float64).reshape(1, vs.D),
                      np.array([float(theta)]), prm.N)[:, 0]
    if not prm.compressible:
        return feq, None
    Cv = 1.0 / (prm.gamma - 1.0)
    return feq, float(theta) * (2.0 * Cv - vs.D) * feq


def pull_point(plane, delta, p, point):
    """Interpolated value of one field at one node (brute-force loop form)."""
    D = plane.ndim
    shape_xyz = plane.shape[::-1]
    sts = [stencil_1d(float(delta[a]), p) for a in range(D)]
    total = 0.0
    for js in itertools.product(range(p + 1), repeat=D):
        weight = 1.0
        src = []
        for a in range(D):
            m0, W = sts[a]
            weight *= W[js[a]]
            src.append((point[a] + m0 + js[a]) % shape_xyz[a])
        total += weight * plane[tuple(src[::-1])]
    return total


# ----------------------------------------------------------------------------
# Hermite tensors and equilibrium moments (Appendix A)
# ----------------------------------------------------------------------------


def hermite_tensors(xi, cs, N):
    """Scaled Hermite tensors H_i^(n), n = 0..N, as full D^n arrays per velocity.

    xi_hat = xi / c_s; H^(1) = xi_hat/c_s; H^(2) = (xi_hat xi_hat - delta)/c_s^2;
    H^(3) = (xi_hat^3 - 3 sym terms xi_hat delta)/c_s^3;
    H^(4) = (xi_hat^4 - T_i + 3 delta delta terms)/c_s^4, T_i the six
    xi_hat xi_hat delta terms (Appendix A).
    """
    xi = np.asarray(xi, dtype=np.float64)
    Q, D = xi.shape
    x = xi / cs
    d = np.eye(D)
    H = [np.ones(Q)]
    if N >= 1:
        H.append(x / cs)
    if N >= 2:
        H.append((np.einsum("ia,ib->iab", x, x) - d[None]) / cs**2)
    if N >= 3:
        t = (np.einsum("ia,ib,ic->iabc", x, x, x)
             - (np.einsum("ia,bc->iabc", x, d) + np.einsum("ib,ac->iabc", x, d)
                + np.einsum("ic,ab->iabc", x, d)))
        H.append(t / cs**3)
    if N >= 4:
        T = (np.einsum("ia,ib,gd->iabgd", x, x, d) + np.einsum("ia,ig,bd->iabgd", x, x, d)
             + np.einsum("ia,id,bg->iabgd", x, x, d) + np.einsum("ib,ig,ad->iabgd", x, x, d)
             + np.einsum("ib,id,ag->iabgd", x, x, d) + np.einsum("ig,id,ab->iabgd", x, x, d))
        dd = (np.einsum("ab,gd->abgd", d, d) + np.einsum("ag,bd->abgd", d, d)
              + np.einsum("ad,bg->abgd", d, d))
        H.append((np.einsum("ia,ib,ig,id->iabgd", x, x, x, x) - T + dd[None]) / cs**4)
    if N >= 5:
        raise ValueError("Appendix A lists Hermite tensors up to fourth order")
    return H


def equilibrium_moments(rho, u, theta, T0, N):
    """Equilibrium Hermite moments a_eq^(n), n = 0..N (Appendix A), per node.

    rho (M,), u (M, D), theta (M,).  a^(2) = rho (u u + T0 (theta-1) delta);
    a^(3) = rho [u u u + T0 (theta-1) (3 delta u terms)];
    a^(4) = rho [u u u u + T0 (theta-1) ((3 delta delta terms) T0 (theta-1)
    + 6 delta u u terms)].  The printed fourth moment is garbled in
    extraction; this grouping (the Hermite moments of a Maxwellian) is the
    reading, pinned in the tests against quadrature of the Maxwellian.
    """
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    D = u.shape[1]
    d = np.eye(D)
    tt = T0 * (np.asarray(theta, dtype=np.float64) - 1.0)
    a = [rho.copy()]
    if N >= 1:
        a.append(rho[:, None] * u)
    if N >= 2:
        a.append(rho[:, None, None] * (np.einsum("ma,mb->mab", u, u)
                                       + tt[:, None, None] * d[None]))
    if N >= 3:
        sym = (np.einsum("ab,mc->mabc", d, u) + np.einsum("ac,mb->mabc", d, u)
               + np.einsum("bc,ma->mabc", d, u))
        a.append(rho[:, None, None, None] * (np.einsum("ma,mb,mc->mabc", u, u, u)
                                             + tt[:, None, None, None] * sym))
    if N >= 4:
        dd = (np.einsum("ab,gd->abgd", d, d) + np.einsum("ag,bd->abgd", d, d)
              + np.einsum("ad,bg->abgd", d, d))
        duu = (np.einsum("ab,mg,md->mabgd", d, u, u) + np.einsum("ag,mb,md->mabgd", d, u, u)
               + np.einsum("ad,mb,mg->mabgd", d, u, u) + np.einsum("bg,ma,md->mabgd", d, u, u)
               + np.einsum("bd,ma,mg->mabgd", d, u, u) + np.einsum("gd,ma,mb->mabgd", d, u, u))
        inner = dd[None] * tt[:, None, None, None, None] + duu
        a.append(rho[:, None, None, None, None] * (np.einsum("ma,mb,mg,md->mabgd", u, u, u, u)
                                                   + tt[:, None, None, None, None] * inner))
    return a


def equilibrium(vs, rho, u, theta, N, chunk=32768):
    """f_i^eq = w_i sum_{n<=N} (1/n!) a_eq^(n) : H_i^(n)  (Sec. 3), shape (Q, M)."""
    rho = np.asarray(rho, dtype=np.float64).ravel()
    M = rho.shape[0]
    u = np.asarray(u, dtype=np.float64).reshape(M, -1)
    theta = np.broadcast_to(np.asarray(theta, dtype=np.float64), (M,)).ravel()
    T0 = vs.cs ** 2
    H = hermite_tensors(vs.xi, vs.cs, N)
    out = np.empty((vs.Q, M))
    for s in range(0, M, chunk):
        e = min(M, s + chunk)
        a = equilibrium_moments(rho[s:e], u[s:e], theta[s:e], T0, N)
        acc = np.zeros((vs.Q, e - s))
        for n in range(N + 1):
            Hn = H[n].reshape(vs.Q, -1)
            an = a[n].reshape(e - s, -1)
            acc += np.einsum("ik,mk->im", Hn, an, optimize=False) / math.factorial(n)
        out[:, s:e] = vs.w[:, None] * acc
    return out


# ----------------------------------------------------------------------------
# Moments (Sec. 3)
# ----------------------------------------------------------------------------


def density_momentum(vs, f):
    """rho = sum_i f_i ; rho u = sum_i xi_i f_i ; f of shape (Q, M)."""
    rho = f.sum(axis=0)
    j = np.einsum("ia,im->ma", vs.xi, f, optimize=False)
    return rho, j / rho[:, None]


def temperature(vs, f, g, rho, u, gamma):
    """theta from 2 rho C_v theta = sum_i (|zeta_i|^2 f_i / T0 + g_i), zeta = xi - u."""
    Cv = 1.0 / (gamma - 1.0)
    T0 = vs.cs ** 2
    zeta2 = ((vs.xi[:, None, :] - u[None, :, :]) ** 2).sum(axis=2)
    return (zeta2 * f / T0 + g).sum(axis=0) / (2.0 * rho * Cv)


# ----------------------------------------------------------------------------
# One time step
# ----------------------------------------------------------------------------


class Params:
    """Run parameters of one simulation (grid units: dx, dt; tau or mu)."""

    def __init__(self, vs, N, p, dt, dx, tau=None, compressible=False, gamma=1.4, mu=None, mu_exponent=0.0,
                 prandtl=1.0):
        self.vs, self.N, self.p, self.dt, self.dx = vs, N, p, dt, dx
        self.tau, self.compressible, self.gamma, self.mu = tau, compressible, gamma, mu
        self.mu_exponent, self.prandtl = mu_exponent, prandtl
        if prandtl != 1.0 and not compressible:
            raise ValueError("the Prandtl number is a parameter of the compressible model")
        if compressible and mu is None:
            raise ValueError("compressible runs need the dynamic viscosity mu")
        if not compressible and tau is None:
            raise ValueError("isothermal runs need tau")


def pull_state(prm, f, inflow=None):
    """Apply the semi-Lagrangian pull to every population field. f: (Q, *grid).

    inflow: None (periodic), or the inflow value of every field (Q,) for the
    non-periodic x of ``pull_plane_xbc``."""
    deltas = departure_offsets(prm.vs.xi, prm.dt, prm.dx)
    Q = prm.vs.Q
    if inflow is None:
        return np.stack([pull_plane(f[i], deltas[i], prm.p) for i in range(f.shape[0])])
    return np.stack([pull_plane_xbc(f[i], deltas[i % Q], prm.p, inflow[i]) for i in range(f.shape[0])])


def quasi_equilibrium(vs, ft, gt, feq, geq, u):
    """The quasi-equilibria f*, g* of the heat flux (Prandtl reading above).

    With zeta_i = xi_i - u and T0 = c_s^2, the non-equilibrium central heat
    flux of f, q_f = sum_i (f~_i - f^eq_i) zeta_i |zeta_i|^2, and the
    non-equilibrium central first moment of g, q_g = sum_i (g~_i - g^eq_i) zeta_i,
    are carried by the third- and first-order Hermite terms
        f*_i - f^eq_i = w_i (q_f . xi_i)(|xi_i|^2 - (D + 2) T0) / (2 (D + 2) T0^3),
        g*_i - g^eq_i = w_i (q_g . xi_i) / T0,
    which have no mass, momentum, stress or energy, and whose central heat
    flux (first moment for g) is q_f (q_g) when the set integrates sixth-order
    monomials exactly.  All arrays (Q, M) except u (M, D)."""
    D, T0 = vs.D, vs.cs ** 2
    zeta = vs.xi[:, None, :] - u[None, :, :]
    zeta2 = (zeta ** 2).sum(axis=2)
    q_f = np.einsum("im,ima->ma", (ft - feq) * zeta2, zeta, optimize=False)
    q_g = np.einsum("im,ima->ma", gt - geq, zeta, optimize=False)
    xi2 = (vs.xi ** 2).sum(axis=1)
    qf_xi = q_f @ vs.xi.T  # (M, Q)
    qg_xi = q_g @ vs.xi.T
    fstar = feq + (vs.w[:, None] * qf_xi.T * (xi2[:, None] - (D + 2) * T0)) / (2.0 * (D + 2) * T0 ** 3)
    gstar = geq + vs.w[:, None] * qg_xi.T / T0
    return fstar, gstar


def collide(prm, ft, gt=None):
    """Moments, equilibrium and BGK on pulled populations ft (Q, M) [, gt].

    Returns (f_post, g_post, diag) with diag holding the per-node moments and
    the relaxation time used.
    """
    vs = prm.vs
    rho, u = density_momentum(vs, ft)
    if prm.compressible:
        theta = temperature(vs, ft, gt, rho, u, prm.gamma)
        P = rho * theta * vs.cs ** 2
        mu = prm.mu * theta ** prm.mu_exponent  # power law in temperature; constant for omega = 0
        tau = mu / (vs.cs ** 2 * prm.dt * P) + 0.5
    else:
        theta = np.ones_like(rho)
        tau = np.full_like(rho, prm.tau)
    feq = equilibrium(vs, rho, u, theta, prm.N)
    fpost = ft - (ft - feq) / tau[None, :]
    gpost = None
    if prm.compressible:
        Cv = 1.0 / (prm.gamma - 1.0)
        geq = theta[None, :] * (2.0 * Cv - vs.D) * feq
        gpost = gt - (gt - geq) / tau[None, :]
        if prm.prandtl != 1.0:
            # relax to f* at tau, and from f* to f^eq at tau_2 (heat flux)
            tau2 = 0.5 + (tau - 0.5) / prm.prandtl
            fstar, gstar = quasi_equilibrium(vs, ft, gt, feq, geq, u)
            c = (1.0 / tau - 1.0 / tau2)[None, :]
            fpost = fpost + c * (fstar - feq)
            gpost = gpost + c * (gstar - geq)
    diag = dict(rho=rho, u=u, theta=theta, tau=tau, ft=ft, feq=feq)
    return fpost, gpost, diag


def step(prm, f, g=None, xbc=None):
    """One SLLBM step: pull every population, then collide (BGK).

    f (Q, *grid) post-collision state at t; returns the post-collision state
    at t + dt and per-step diagnostics.  xbc: None (periodic), or
    ``inflow_populations`` of the inflow state for the non-periodic x of
    ``pull_plane_xbc``.
    """
    grid = f.shape[1:]
    f_in, g_in = xbc if xbc is not None else (None, None)
    ft = pull_state(prm, f, f_in).reshape(f.shape[0], -1)
    gt = pull_state(prm, g, g_in).reshape(g.shape[0], -1) if prm.compressible else None
    fpost, gpost, diag = collide(prm, ft, gt)
    diag.update(reductions(prm, diag))
    fpost = fpost.reshape(f.shape)
    if gpost is not None:
        gpost = gpost.reshape(g.shape)
    return fpost, gpost, diag


def step_at_points(prm, f, g, points):
    """Post-collision populations of one step at selected nodes only.

    points: integer array (K, D) of (x, y[, z]) node coordinates.  Gathers the
    (p+1)^D neighbourhood of each node per velocity with periodic wrap and
    applies the same pull and collision as ``step``.  Returns (fpost (Q, K),
    gpost or None, diag).
    """
    vs = prm.vs
    D = vs.D
    shape_xyz = f.shape[1:][::-1]
    pts = np.asarray(points, dtype=np.int64)
    deltas = departure_offsets(vs.xi, prm.dt, prm.dx)

    def pulled(field):
        out = np.zeros((field.shape[0], pts.shape[0]))
        for i in range(field.shape[0]):
            sts = [stencil_1d(float(deltas[i % vs.Q][a]), prm.p) for a in range(D)]
            for js in itertools.product(range(prm.p + 1), repeat=D):
                weight = 1.0
                idx = []
                for a in range(D):
                    m0, W = sts[a]
                    weight *= W[js[a]]
                    idx.append((pts[:, a] + m0 + js[a]) % shape_xyz[a])
                out[i] += weight * field[i][tuple(idx[::-1])]
        return out

    ft = pulled(f)
    gt = pulled(g) if prm.compressible else None
    return collide(prm, ft, gt)


# ----------------------------------------------------------------------------
# Initial state and diagnostics
# ----------------------------------------------------------------------------


def init_equilibrium(prm, rho, u, theta=None):
    """f = f^eq(rho, u, theta) (and g = theta (2 C_v - D) f^eq) from fields.

    rho (*grid), u (D, *grid) in SoA layout, theta (*grid) or None (= 1).
    """
    vs = prm.vs
    grid = np.shape(rho)
    M = int(np.prod(grid))
    uu = np.asarray(u).reshape(vs.D, M).T
    th = np.ones(M) if theta is None else np.asarray(theta).reshape(M)
    feq = equilibrium(vs, np.asarray(rho).reshape(M), uu, th, prm.N)
    f = feq.reshape((vs.Q,) + grid)
    g = None
    if prm.compressible:
        Cv = 1.0 / (prm.gamma - 1.0)
        g = (th[None, :] * (2.0 * Cv - vs.D) * feq).reshape((vs.Q,) + grid)
    return f, g


def strain_dissipation(prm, diag):
    """Builder's estimator: eps = mean 2 nu S:S with S = -Pi_neq / (2 P tau dt).

    Pi_neq = sum_i xi_i xi_i (f~_i - f_i^eq) (Chapman-Enskog); P = rho theta c_s^2;
    nu = c_s^2 theta dt (tau - 1/2).  Not in the paper; pinned by the analytic
    strain of the 3D Taylor-Green vortex, 2 nu <S:S> = (3/4) nu u0^2 e^(-6 nu t).
    """
    vs = prm.vs
    fneq = diag["ft"] - diag["feq"]
    Pi = np.einsum("ia,ib,im->mab", vs.xi, vs.xi, fneq, optimize=False)
    P = diag["rho"] * diag["theta"] * vs.cs ** 2
    S = -Pi / (2.0 * P * diag["tau"] * prm.dt)[:, None, None]
    nu = vs.cs ** 2 * diag["theta"] * prm.dt * (diag["tau"] - 0.5)
    return float((2.0 * nu * (S * S).sum(axis=(1, 2))).mean())


def reductions(prm, diag):
    """Global per-step sums of the post-streaming moments: k = mean |u|^2 / 2
    (Sec. 4.2, the mean kinetic energy; on the uniform grid the integral over
    the box divided by its volume is the node mean), the rho-weighted
    k_rho = mean rho |u|^2 / 2, the dissipation estimate, the mass sum rho
    and the momentum sum rho u.  Pinned by closed forms in
    tests/test_oracle_reductions.py."""
    rho, u = diag["rho"], diag["u"]
    ke = 0.5 * (u ** 2).sum(axis=1)
    return dict(
        k=float(ke.mean()),
        k_rho=float((rho * ke).mean()),
        eps=strain_dissipation(prm, diag),
        mass=float(rho.sum()),
        momentum=(rho[:, None] * u).sum(axis=0),
    )


def moments_of_state(prm, f, g=None):
    """rho, u (D, *grid), theta of a stored post-collision state (no pull)."""
    vs = prm.vs
    grid = f.shape[1:]
    ff = f.reshape(vs.Q, -1)
    rho, u = density_momentum(vs, ff)
    if prm.compressible:
        theta = temperature(vs, ff, g.reshape(vs.Q, -1), rho, u, prm.gamma)
    else:
        theta = np.ones_like(rho)
    return rho.reshape(grid), u.T.reshape((vs.D,) + grid), theta.reshape(grid)


def tau_isothermal(nu, cs, dt):
    """tau = nu / (c_s^2 dt) + 1/2 (Sec. 3, LBE)."""
    return nu / (cs ** 2 * dt) + 0.5


def tau_compressible(mu, cs, dt, P):
    """tau = mu / (c_s^2 dt P) + 1/2 (Sec. 3, compressible model)."""
    return mu / (cs ** 2 * dt * P) + 0.5

"""Plain FP64 oracle of the adjoint of the isothermal SLLBM step.

TEST INFRASTRUCTURE ONLY.  Nothing under ``oracle/`` is part of the product
path: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library.

The paper states no adjoint.  What is computed here is the exact transpose of
the Jacobian of one step as the paper defines the step (Sec. 3): the pull
(Eq. sl_streaming, a linear map S per velocity) followed by the BGK collision
C with the Hermite equilibrium of order N (Appendix A), isothermal
(theta = 1, constant tau).  For a scalar objective J of the state after the
step, with lam = dJ/d(state after the step):

    dJ/d(state before the step) = S^T  Jc(S f)^T  lam,

    (Jc^T sigma)_k = (1 - 1/tau) sigma_k
                     + (1/tau) sum_i sigma_i d f_i^eq / d f~_k,

    d f_i^eq / d f~_k = d f_i^eq / d rho |_j + (d f_i^eq / d j) . xi_k,

because rho = sum f~ and j = rho u = sum xi f~ (Sec. 3, Eqs. density and
momentum).  The derivatives of f^eq are taken through the Hermite moments of
Appendix A at theta = 1, a^(n) = j^(n-fold outer product) / rho^(n-1),
contracted with the literal Hermite tensors; S^T is the pull with every
stencil point reflected (the transpose of a sum of shifts is the sum of the
opposite shifts with the same weights).

Pins (tests/test_oracle_adjoint.py): the dot-product identity of S and S^T,
central finite differences of the forward oracle (equilibrium, moments, the
whole step, a short trajectory), and the conservation invariants
Jc^T 1 = 1 and Jc^T xi_a = xi_a.
"""
import itertools
import math

import numpy as np

from . import sllbm

# ----------------------------------------------------------------------------
# Transpose of the pull (Sec. 3, Eq. sl_streaming)
# ----------------------------------------------------------------------------


def pull_plane_transpose(plane, delta, p):
    """S^T of ``sllbm.pull_plane``: out(y) = sum_J W_J plane(y - m0 - J).

    The pull reads plane(x + m0 + J) with weight W_J, so its transpose sends
    lam(x) back to y = x + m0 + J with the same weight.
    """
    D = plane.ndim
    sts = [sllbm.stencil_1d(float(delta[a]), p) for a in range(D)]
    out = np.zeros_like(plane)
    for js in itertools.product(range(p + 1), repeat=D):
        weight = 1.0
        shifts = []
        for a in range(D):
            m0, W = sts[a]
            weight *= W[js[a]]
            shifts.append(m0 + js[a])
        rolled = plane
        for a in range(D):
            rolled = np.roll(rolled, +shifts[a], axis=D - 1 - a)
        out += weight * rolled
    return out


def pull_state_transpose(prm, lam):
    """S^T applied to every population field. lam: (Q, *grid)."""
    deltas = sllbm.departure_offsets(prm.vs.xi, prm.dt, prm.dx)
    return np.stack([pull_plane_transpose(lam[i], deltas[i], prm.p) for i in range(lam.shape[0])])


# ----------------------------------------------------------------------------
# Derivatives of the isothermal equilibrium (Sec. 3 Hermite series, Appendix A)
# ----------------------------------------------------------------------------


def _outer_power(j, n):
    """j^(n-fold outer product) per node, shape (M, D**n); n = 0 gives ones."""
    M, D = j.shape
    t = np.ones((M, 1))
    for _ in range(n):
        t = np.einsum("mk,ma->mka", t, j).reshape(M, -1)
    return t


def equilibrium_derivatives(vs, rho, j, N):
    """d f_i^eq/d rho at fixed j, shape (Q, M), and d f_i^eq/d j_a, shape (Q, M, D).

    Isothermal moments a^(n) = j^n / rho^(n-1):
      d a^(n)/d rho = (1 - n) j^n / rho^n,
      d (a^(n) : H^(n)) / d j_a = n (H^(n) contracted with j^(n-1))_a / rho^(n-1)
    (H^(n) is symmetric, so each of the n slots gives the same term).
    """
    rho = np.asarray(rho, dtype=np.float64).ravel()
    M = rho.shape[0]
    j = np.asarray(j, dtype=np.float64).reshape(M, -1)
    D = j.shape[1]
    H = sllbm.hermite_tensors(vs.xi, vs.cs, N)
    d_rho = np.zeros((vs.Q, M))
    d_j = np.zeros((vs.Q, M, D))
    for n in range(N + 1):
        fn = 1.0 / math.factorial(n)
        Hn = H[n].reshape(vs.Q, -1)
        if n >= 2:
            jn = _outer_power(j, n)
            d_rho += fn * (1 - n) * np.einsum("ik,mk->im", Hn, jn, optimize=False) / rho[None, :] ** n
        elif n == 0:
            d_rho += fn * Hn[:, :1] * np.ones((1, M))
        if n >= 1:
            Hr = H[n].reshape(vs.Q, D, -1)
            jm = _outer_power(j, n - 1)
            d_j += fn * n * np.einsum("iak,mk->ima", Hr, jm, optimize=False) / rho[None, :, None] ** (n - 1)
    return vs.w[:, None] * d_rho, vs.w[:, None, None] * d_j


# ----------------------------------------------------------------------------
# Vector-Jacobian products
# ----------------------------------------------------------------------------


def collide_vjp(prm, ft, sigma):
    """Jc(ft)^T sigma for the isothermal BGK collision; ft, sigma of shape (Q, M)."""
    if prm.compressible:
        raise ValueError("the adjoint is defined for the isothermal step only")
    vs = prm.vs
    rho = ft.sum(axis=0)
    j = np.einsum("ia,im->ma", vs.xi, ft, optimize=False)
    d_rho, d_j = equilibrium_derivatives(vs, rho, j, prm.N)
    A = (sigma * d_rho).sum(axis=0)                       # sum_i sigma_i d f_i^eq / d rho
    B = np.einsum("im,ima->ma", sigma, d_j, optimize=False)  # sum_i sigma_i d f_i^eq / d j
    inv_tau = 1.0 / prm.tau
    return (1.0 - inv_tau) * sigma + inv_tau * (A[None, :] + np.einsum("ka,ma->km", vs.xi, B, optimize=False))


def step_vjp(prm, f, lam):
    """dJ/df for J depending on the state after one step of f; lam = dJ/d(step(f)).

    f, lam of shape (Q, *grid); returns an array of the same shape.
    """
    Q = f.shape[0]
    ft = sllbm.pull_state(prm, f).reshape(Q, -1)
    sigma = collide_vjp(prm, ft, lam.reshape(Q, -1))
    return pull_state_transpose(prm, sigma.reshape(f.shape))


def trajectory_vjp(prm, f0, nsteps, lam_T):
    """dJ/df0 for J depending on the state after nsteps steps from f0.

    Stores every intermediate state (the oracle is used on small grids) and
    applies ``step_vjp`` from the last step back to the first.
    """
    states = [f0]
    f = f0
    for _ in range(nsteps):
        f, _, _ = sllbm.step(prm, f)
        states.append(f)
    lam = lam_T
    for t in range(nsteps - 1, -1, -1):
        lam = step_vjp(prm, states[t], lam)
    return lam, states[-1]


def moments_vjp(vs, f, grad_rho, grad_u):
    """lam_i = dJ/df_i for J(rho, u) with rho = sum f, u = sum xi f / rho.

    d rho/d f_i = 1 and d u/d f_i = (xi_i - u)/rho.  f (Q, M); grad_rho (M,);
    grad_u (M, D).  Returns (Q, M).
    """
    rho, u = sllbm.density_momentum(vs, f)
    xu = np.einsum("ia,ma->im", vs.xi, grad_u, optimize=False) - (u * grad_u).sum(axis=1)[None, :]
    return grad_rho[None, :] + xu / rho[None, :]


def equilibrium_vjp(vs, N, rho, u, lam):
    """Gradients of sum_i lam_i f_i^eq(rho, u) (theta = 1) with respect to rho and u.

    With j = rho u: d/du = rho d/dj and d/drho|_u = d/drho|_j + u . d/dj.
    rho (M,), u (M, D), lam (Q, M).  Returns (grad_rho (M,), grad_u (M, D)).
    """
    rho = np.asarray(rho, dtype=np.float64).ravel()
    u = np.asarray(u, dtype=np.float64).reshape(rho.shape[0], -1)
    d_rho, d_j = equilibrium_derivatives(vs, rho, rho[:, None] * u, N)
    gj = np.einsum("im,ima->ma", lam, d_j, optimize=False)
    g_rho = (lam * d_rho).sum(axis=0) + (u * gj).sum(axis=1)
    return g_rho, rho[:, None] * gj

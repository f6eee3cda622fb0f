"""Pins of the oracle's Hermite equilibrium (Sec. 3 and Appendix A).

* a_eq^(n) equals the Hermite moment of the Maxwellian with density rho,
  velocity u and temperature theta T0, computed by an exact Gauss-Hermite
  product rule in the variable zeta = (xi - u)/sqrt(theta T0) (numpy).
* The discrete equilibrium reproduces a_eq^(n) for n <= N whenever the set's
  degree is at least N + n (Sec. 2, exactness rule).  The scaled tensors of
  Appendix A are c_s^(-2n) times c_s^n He_n(xi/c_s), so moments taken with
  them are a_eq^(n) / c_s^(2n).
* The isothermal D2Q9 equilibrium with c_s^2 = 1/3 is the textbook formula.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import sllbm as O
from oracle import velocity_sets as V


def maxwellian_moments(rho, u, theta, T0, N, npts=6):
    D = u.shape[0]
    z, w = np.polynomial.hermite_e.hermegauss(npts)
    w = w / w.sum()
    nodes, weights = [], []
    for idx in itertools.product(range(npts), repeat=D):
        nodes.append([z[i] for i in idx])
        weights.append(math.prod(w[i] for i in idx))
    nodes = np.array(nodes)
    weights = np.array(weights)
    xi = u[None, :] + math.sqrt(theta * T0) * nodes
    cs = math.sqrt(T0)
    H = O.hermite_tensors(xi, cs, N)
    # Appendix A's tensors carry 1/c_s^(2n) relative to c_s^n He_n(xi/c_s), the
    # polynomials whose moments the a_eq^(n) are: undo that factor.
    return [rho * T0 ** n * np.tensordot(weights, H[n], axes=(0, 0)) for n in range(N + 1)]


@pytest.mark.parametrize("D,N,theta", [(2, 4, 1.3), (3, 4, 0.7), (3, 3, 1.0), (2, 2, 1.0), (3, 2, 1.6)])
@pytest.mark.parametrize("T0", [1.0, 0.6])
def test_equilibrium_moments_are_maxwellian_moments(D, N, theta, T0):
    rng = np.random.default_rng(11)
    rho = 1.3
    u = rng.uniform(-0.4, 0.4, D)
    a = O.equilibrium_moments(np.array([rho]), u[None, :], np.array([theta]), T0, N)
    want = maxwellian_moments(rho, u, theta, T0, N)
    for n in range(N + 1):
        assert np.allclose(a[n][0], want[n], atol=1e-12, rtol=1e-12), n


@pytest.mark.parametrize("name,N,comp", [
    ("D2Q9", 2, False), ("D3Q27", 2, False), ("D3Q13", 2, False), ("D3Q21", 2, False),
    ("D3V27", 3, False), ("D2Q19", 4, True), ("D2Q25", 4, True), ("D3Q45", 4, True)])
def test_discrete_equilibrium_recovers_moments(name, N, comp):
    vs = V.get(name)
    rng = np.random.default_rng(13)
    M = 20
    rho = rng.uniform(0.5, 2.0, M)
    u = rng.uniform(-0.5, 0.5, (M, vs.D)) * vs.cs / math.sqrt(vs.D)
    theta = rng.uniform(0.5, 2.0, M) if comp else np.ones(M)
    feq = O.equilibrium(vs, rho, u, theta, N)
    H = O.hermite_tensors(vs.xi, vs.cs, N)
    a = O.equilibrium_moments(rho, u, theta, vs.cs ** 2, N)
    for n in range(N + 1):
        if vs.degree < N + n:
            continue
        got = np.tensordot(feq, H[n], axes=(0, 0)) * vs.cs ** (2 * n)
        assert np.allclose(got, a[n], atol=1e-11), (name, n)


def test_hermite_tensors_are_orthogonal_under_degree_nine_rule():
    vs = V.get("D3Q45")
    H = O.hermite_tensors(vs.xi, vs.cs, 4)
    for n in range(5):
        for m in range(5):
            if n + m > vs.degree or n == m:
                continue
            g = np.tensordot(vs.w[:, None] * H[n].reshape(vs.Q, -1), H[m].reshape(vs.Q, -1), axes=(0, 0))
            assert np.abs(g).max() < 1e-12


def test_d2q9_textbook_equilibrium():
    vs = V.get("D2Q9").scaled(1.0 / math.sqrt(3.0))
    assert np.allclose(np.abs(vs.xi).max(), 1.0)
    rng = np.random.default_rng(17)
    rho = rng.uniform(0.8, 1.2, 50)
    u = rng.uniform(-0.1, 0.1, (50, 2))
    feq = O.equilibrium(vs, rho, u, np.ones(50), 2)
    cu = vs.xi @ u.T
    usq = (u ** 2).sum(1)
    want = vs.w[:, None] * rho[None, :] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * usq[None, :])
    assert np.allclose(feq, want, atol=1e-15)

"""Pins of the oracle's velocity sets (Sec. 2 Table 1, Tables 2-3, Appendices C-E).

Each set must satisfy the symmetry conditions of Appendix B (the Gaussian
moments of the weight function of Sec. 2) up to its claimed degree and fail
them one degree higher; product rules must equal numpy's Gauss-Hermite rule.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import velocity_sets as V


def gaussian_moment(j, cs):
    """E[x^j] for x ~ N(0, cs^2): cs^j (j-1)!! for even j, 0 for odd j."""
    if j % 2:
        return 0.0
    return cs ** j * math.prod(range(j - 1, 0, -2))


def max_residual(vs, degree):
    worst = 0.0
    for tot in range(degree + 1):
        for js in itertools.product(range(tot + 1), repeat=vs.D):
            if sum(js) != tot:
                continue
            mono = np.prod([vs.xi[:, a] ** js[a] for a in range(vs.D)], axis=0)
            got = float((vs.w * mono).sum())
            want = math.prod(gaussian_moment(j, vs.cs) for j in js)
            worst = max(worst, abs(got - want) / max(1.0, abs(want)))
    return worst


@pytest.mark.parametrize("name,Q,D,degree", [
    ("D2Q9", 9, 2, 5), ("D2Q19", 19, 2, 9), ("D2Q25", 25, 2, 9), ("D3Q13", 13, 3, 5),
    ("D3Q21", 21, 3, 5), ("D3Q27", 27, 3, 5), ("D3V27", 27, 3, 7), ("D3Q45", 45, 3, 9)])
def test_isotropy_to_claimed_degree(name, Q, D, degree):
    vs = V.get(name)
    assert vs.Q == Q and vs.D == D and vs.degree == degree
    assert max_residual(vs, degree) < 1e-12
    # one degree higher the rule is no longer exact (Appendix B, degree d)
    assert max_residual(vs, degree + 1) > 1e-6


@pytest.mark.parametrize("name", V.ALL_SETS)
def test_distinct_abscissae_and_rest_first(name):
    vs = V.get(name)
    assert np.all(vs.xi[0] == 0.0)
    d = np.linalg.norm(vs.xi[:, None, :] - vs.xi[None, :, :], axis=2) + np.eye(vs.Q)
    assert d.min() > 1e-6
    assert np.all(vs.w > 0)


def test_product_rules_equal_numpy_gauss_hermite():
    for npts, name2, name3 in ((3, "D2Q9", "D3Q27"), (5, "D2Q25", None)):
        x, w = np.polynomial.hermite_e.hermegauss(npts)
        w = w / w.sum()
        vs = V.get(name2)
        got = sorted(zip(np.round(vs.xi[:, 0], 12), np.round(vs.xi[:, 1], 12), np.round(vs.w, 14)))
        want = sorted((round(x[i], 12), round(x[j], 12), round(w[i] * w[j], 14))
                      for i in range(npts) for j in range(npts))
        assert np.allclose(np.array(got), np.array(want), atol=1e-12)
        if name3:
            vs3 = V.get(name3)
            assert vs3.Q == npts ** 3
            assert np.isclose(sorted(vs3.w)[0], sorted(w)[0] ** 3)


def test_tabulated_constants():
    # Table 2: every moving D3Q13 abscissa has |xi|^2 = r^2 + s^2 = 5
    vs = V.get("D3Q13")
    assert np.allclose((vs.xi[1:] ** 2).sum(1), 5.0)
    # Table 3: c_s = sqrt(3/5), moving abscissae on the sphere of radius sqrt(3)
    vs = V.get("D3Q21")
    assert np.isclose(vs.cs, math.sqrt(0.6))
    assert np.allclose((vs.xi[1:] ** 2).sum(1), 3.0)
    # Appendix E: the printed weights sum to 1 within their printed digits
    vs = V.get("D3Q45")
    assert abs(vs.w.sum() - 1.0) < 1e-14

"""Pins of the enstrophy oracle (Sec. 4.2: mean |curl u|^2).

* Taylor-Green field u = (sin x cos y cos z, -cos x sin y cos z, 0) of
  Sec. 4.2: |curl u|^2 averages to 3/4 in the continuum; the fourth-order
  difference of sin(x) on spacing h is g(h) cos(x) with
  g(h) = (8 sin h - sin 2h) / (6 h), so the discrete value is (3/4) g(h)^2.
* A discrete gradient field (same difference operator) has zero curl.
* Fourth-order convergence of the error against 3/4.
* 2D: u = (sin x cos y, -cos x sin y) gives omega = 2 sin x sin y, mean 1.
"""
import math

import numpy as np
import pytest

from oracle import diagnostics as G


def tgv(n):
    x = np.arange(n) * 2 * np.pi / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return np.stack([np.sin(X) * np.cos(Y) * np.cos(Z), -np.cos(X) * np.sin(Y) * np.cos(Z), 0 * X]), 2 * np.pi / n


@pytest.mark.parametrize("n", [8, 16, 32])
def test_tgv_enstrophy_closed_form(n):
    u, h = tgv(n)
    g = (8 * math.sin(h) - math.sin(2 * h)) / (6 * h)
    assert abs(G.enstrophy(u, h) - 0.75 * g * g) < 1e-13


def test_fourth_order_convergence():
    errs = []
    for n in (16, 32):
        u, h = tgv(n)
        errs.append(abs(G.enstrophy(u, h) - 0.75))
    assert 14.0 < errs[0] / errs[1] < 18.0


def test_gradient_field_has_no_curl():
    rng = np.random.default_rng(0)
    n, h = 12, 0.3
    phi = rng.standard_normal((n, n, n))
    u = np.stack([G.ddx4(phi, h, 2), G.ddx4(phi, h, 1), G.ddx4(phi, h, 0)])
    assert G.enstrophy(u, h) < 1e-24 * max(1.0, (u ** 2).sum())


def test_2d_vortex():
    n = 32
    h = 2 * np.pi / n
    x = np.arange(n) * h
    Y, X = np.meshgrid(x, x, indexing="ij")
    u = np.stack([np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y)])
    g = (8 * math.sin(h) - math.sin(2 * h)) / (6 * h)
    # omega = -2 g sin x sin y, mean of its square = g^2
    assert abs(G.enstrophy(u, h) - g * g) < 1e-13

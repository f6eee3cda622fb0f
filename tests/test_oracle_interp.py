"""Pins of the oracle's semi-Lagrangian pull (Sec. 3, Eq. sl_streaming).

The equidistant Lagrange stencil is fixed by closed forms: partition of unity,
exact reproduction of x^m for m <= p, Kronecker weights at integer offsets, and
the exact Fourier symbol of the pull on a plane wave.
"""
import itertools

import numpy as np
import pytest

from oracle import sllbm as O


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_stencil_reproduces_polynomials(p):
    rng = np.random.default_rng(1)
    for delta in list(rng.uniform(-3.0, 3.0, 25)) + [-0.5, 0.5, -0.4, 0.4]:
        m0, W = O.stencil_1d(delta, p)
        m = m0 + np.arange(p + 1)
        assert m[0] <= delta <= m[-1]
        # the support is centred on delta
        assert abs((m[0] + m[-1]) / 2.0 - delta) <= 1.0
        for k in range(p + 1):
            assert abs((W * m.astype(float) ** k).sum() - delta ** k) < 1e-11 * max(1.0, abs(delta) ** k)
        # one degree more is not reproduced in general
        if p < 6 and abs(delta - round(delta)) > 1e-3:
            assert abs((W * m.astype(float) ** (p + 1)).sum() - delta ** (p + 1)) > 1e-8


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_stencil_kronecker_at_integers(p):
    for delta in (-2.0, -1.0, 0.0, 1.0, 3.0):
        m0, W = O.stencil_1d(delta, p)
        m = m0 + np.arange(p + 1)
        assert np.array_equal(W, (m == delta).astype(float))


@pytest.mark.parametrize("D,p", [(2, 3), (2, 4), (3, 3), (3, 4)])
def test_pull_fourier_symbol(D, p):
    """Pull of exp(i k.x) is exp(i k.x) prod_a sum_j W_a[j] exp(i k_a m_j dx)."""
    n = 16 if D == 3 else 32
    rng = np.random.default_rng(7)
    for _ in range(3):
        k = rng.integers(-4, 5, size=D)
        delta = rng.uniform(-1.3, 1.3, size=D)
        axes = np.meshgrid(*[np.arange(n)] * D, indexing="ij")  # (z, y, x) order
        phase = sum(k[a] * axes[D - 1 - a] for a in range(D)) * (2 * np.pi / n)
        wave = np.exp(1j * phase)
        pulled = O.pull_plane(wave.real, delta, p) + 1j * O.pull_plane(wave.imag, delta, p)
        sym = 1.0 + 0j
        for a in range(D):
            m0, W = O.stencil_1d(delta[a], p)
            m = m0 + np.arange(p + 1)
            sym *= (W * np.exp(1j * k[a] * m * (2 * np.pi / n))).sum()
        assert np.allclose(pulled, sym * wave, atol=1e-13)


def test_pull_matches_brute_force_loops():
    rng = np.random.default_rng(3)
    f = rng.standard_normal((6, 7, 8))
    delta = np.array([0.37, -1.21, 0.5])
    full = O.pull_plane(f, delta, 3)
    for pt in [(0, 0, 0), (7, 6, 5), (3, 2, 1), (1, 5, 4)]:
        assert abs(full[pt[::-1]] - O.pull_point(f, delta, 3, pt)) < 1e-13


def test_pull_integer_offset_is_a_shift():
    rng = np.random.default_rng(5)
    f = rng.standard_normal((9, 10))
    got = O.pull_plane(f, np.array([2.0, -1.0]), 4)
    # value at x + delta: shift by -delta along each axis
    want = np.roll(np.roll(f, -2, axis=1), 1, axis=0)
    assert np.array_equal(got, want)

"""Host-side checks of the C-ABI library (no GPU needed).

The library loads, exports every function that include/olb.h declares, holds
velocity-set tables equal to the oracle's (same order), and rejects invalid
arguments with the documented codes before touching the device.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import velocity_sets as V

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def olb():
    from paper_2101_03982_gb300 import build, olb as ob
    build.build()
    return ob


def declared_functions():
    text = open(os.path.join(ROOT, "include", "olb.h")).read()
    return sorted(set(re.findall(r"\b(olb_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(olb):
    names = declared_functions()
    assert len(names) >= 20
    L = olb.lib()
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("name", V.ALL_SETS)
def test_library_tables_equal_oracle_tables(olb, name):
    xi, w = olb.velocity_set_table(name)
    vs = V.get(name)
    assert xi.shape == vs.xi.shape
    assert np.allclose(xi, vs.xi, atol=1e-15, rtol=0)
    assert np.allclose(w, vs.w, atol=1e-16, rtol=0)
    Q, D, cs, mx, deg = olb.velocity_set_info(name)
    assert (Q, D, deg) == (vs.Q, vs.D, vs.degree)
    assert abs(cs - vs.cs) < 1e-15
    assert abs(mx - np.abs(vs.xi).max()) < 1e-15


def _create(olb, dim=3, n=(16, 16, 16), vs="D3Q27", N=2, tau=0.8, dt=0.01, **kw):
    L = olb.lib()
    g = olb.Grid()
    g.dim = dim
    for k in range(3):
        g.n[k] = n[k]
    g.dx = 0.1
    o = olb.Options()
    L.olb_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    rc = L.olb_create(ctypes.byref(g), olb.VELOCITY_SETS[vs], N, tau, dt, ctypes.byref(o), ctypes.byref(h))
    return rc, h


def test_default_options_layout(olb):
    """The binding's struct and the library agree field by field."""
    o = olb.Options()
    olb.lib().olb_default_options(ctypes.byref(o))
    assert (o.interp_order, o.storage, o.cs_scale, o.compressible) == (3, 0, 1.0, 0)
    assert (o.gamma, o.mu, o.mu_exponent, o.prandtl, o.rho0) == (1.4, 0.0, 0.0, 1.0, 1.0)
    assert (o.allow_inexact, o.log_every, o.kernel, o.stream) == (0, 1, 0, None)


@pytest.mark.parametrize("kw,code", [
    (dict(dim=4), -1),
    (dict(n=(0, 4, 4)), -1),
    (dict(dim=2, n=(8, 8, 2), vs="D2Q9"), -1),
    (dict(tau=0.5), -1),
    (dict(dt=-1.0), -1),
    (dict(N=5), -1),
    (dict(interp_order=7), -1),
    (dict(storage=9), -1),
    (dict(vs="D2Q9"), -1),                      # set dimension differs from the grid's
    (dict(N=3), -7),                            # D3Q27 has degree 5 < 2N = 6
    (dict(vs="D3Q21", compressible=1, mu=0.1), -7),  # c_s = sqrt(3/5) != 1
    (dict(vs="D3Q45", N=4, compressible=1, mu=0.1, mu_exponent=float("nan")), -1),
    (dict(prandtl=0.75), -1),                   # Pr belongs to the compressible model
    (dict(vs="D3Q45", N=4, compressible=1, mu=0.1, prandtl=0.0), -1),
    (dict(vs="D3Q45", N=2, compressible=1, mu=0.1, prandtl=0.75), -7),  # f^eq of N = 2 has a heat flux
    (dict(vs="D3Q27", N=4, compressible=1, mu=0.1, allow_inexact=1, prandtl=0.75), -7),  # degree 5 < 7
])
def test_argument_checks(olb, kw, code):
    rc, h = _create(olb, **kw)
    assert rc == code
    assert not h.value
    assert olb.lib().olb_last_error()


def test_strerror(olb):
    L = olb.lib()
    for c in range(0, -9, -1):
        assert L.olb_strerror(c)


def test_null_arguments_are_rejected_before_any_device_work(olb):
    """Entry points check their pointers first: no GPU is touched here."""
    import ctypes as C
    L = olb.lib()
    u = (C.c_double * 3)(0.1, 0.0, 0.0)
    assert L.olb_set_x_boundary(None, 1, 1.0, u, 1.0) == -1
    assert L.olb_fp64_fma_peak(None, None) == -1
    assert L.olb_step(None, 1) == -1
    assert L.olb_get_state(None, None, 0, 0) == -1
    assert L.olb_set_state(None, None, 0, 0) == -1
    assert L.olb_destroy(None) == -1


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("shift", [0.0, 0.37, -0.61, 1.45, -2.2])
def test_glc_stencils_equal_the_oracle(olb, p, shift):
    """The library's cell-wise GLC stencils (host code, no GPU) against the
    oracle's, which are pinned on their own (tests/test_oracle_glc.py)."""
    from oracle import glc as G
    first, W = olb.glc_stencil(p, shift)
    for k, (f0, w) in enumerate(G.residue_stencils(p, shift)):
        assert first[k] == f0
        assert np.abs(W[k] - w).max() < 1e-14


def test_glc_stencil_argument_checks(olb):
    import ctypes as C
    L = olb.lib()
    first = (C.c_int * 8)()
    W = (C.c_double * 72)()
    assert L.olb_glc_stencil(0, 0.1, first, W) == -1
    assert L.olb_glc_stencil(9, 0.1, first, W) == -1
    assert L.olb_glc_stencil(3, float("inf"), first, W) == -1
    assert L.olb_glc_stencil(3, 0.1, None, W) == -1

"""GPU parity of the enstrophy diagnostic (Sec. 4.2) against the FP64 oracle.

The library takes u from the moments of the stored populations and the curl
with fourth-order central differences (FP64 throughout); the oracle does the
same from the populations the device holds.  Bound: 1e-12 relative.  The
Taylor-Green case is also checked against the closed form of the discrete
operator, (3/4) g(h)^2 with g(h) = (8 sin h - sin 2h) / (6 h), up to the
compressibility of the initial state (the velocity read back from the
populations equals the imposed one to rounding).
"""
import math

import numpy as np
import pytest

from oracle import diagnostics as G
from oracle import sllbm as O

from test_gpu_parity import make_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def olb():
    from paper_2101_03982_gb300 import olb as ob
    ob.lib()
    return ob


@pytest.mark.parametrize("name,shape,storage", [("D3Q27", (40, 20, 18), "fp64"), ("D3Q27", (37, 11, 9), "fp32"),
                                                ("D3Q45", (16, 12, 10), "fp64"), ("D2Q9", (64, 45), "fp64")])
def test_enstrophy_matches_oracle(olb, name, shape, storage):
    sim, prm, f = make_pair(olb, name, shape, N=2, p=4, storage=storage)
    _, u = O.density_momentum(prm.vs, f.reshape(prm.vs.Q, -1))
    u = u.T.reshape((prm.vs.D,) + f.shape[1:])
    want = G.enstrophy(u, prm.dx)
    got = sim.enstrophy()
    assert abs(got - want) <= 1e-12 * abs(want)
    sim.close()


def test_enstrophy_of_taylor_green_field(olb):
    from paper_2101_03982_gb300 import inputs, params
    n = 32
    rp = params.tgv_isothermal("D3Q27", n, 1600.0, 0.1, 0.4)
    sim = olb.Sim((n,) * 3, rp.dx, "D3Q27", 2, rp.tau, rp.dt, interp_order=4, storage="fp64", cs_scale=rp.cs_scale)
    rho, u = inputs.tgv3d(n, rp.u0, rp.cs ** 2)
    sim.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    h = rp.dx
    g = (8 * math.sin(h) - math.sin(2 * h)) / (6 * h)
    assert abs(sim.enstrophy() - 0.75 * g * g * rp.u0 ** 2) < 1e-12
    sim.close()

"""The 2D decaying Taylor-Green vortex at its stated size and horizon, on the GPU.

D2Q9 rescaled to c_s^2 = 1/3, second-order Hermite equilibrium, Re 100,
u0 = 0.05, 64 x 64 periodic nodes, Courant 0.4 (non-integer offsets), p = 3,
FP64 storage, 200 steps (Sec. 3 step; the 2D TGV is the method's textbook
check).  The library and the FP64 oracle start from the same equilibrium of
u = u0 (sin x cos y, -cos x sin y) with the balancing pressure and run 200
steps each: every population agrees within 1e-11 relative, the kinetic-energy
history within 1e-11 at every logged step, and the velocity amplitude follows
exp(-2 nu t) within the oracle's own 1e-3 (tests/test_oracle_step.py).
"""
import math

import numpy as np
import pytest

from oracle import sllbm as O
from oracle import velocity_sets as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, STEPS, LOG = 64, 200, 20


def test_tgv2d_200_steps_against_oracle():
    from paper_2101_03982_gb300 import inputs, olb, params
    rp = params.tgv2d_lattice(N)
    vs = V.get("D2Q9").scaled(rp.cs_scale)
    prm = O.Params(vs, 2, 3, dt=rp.dt, dx=rp.dx, tau=rp.tau)
    rho, u = inputs.tgv2d(N, rp.u0, rp.cs ** 2)
    f, _ = O.init_equilibrium(prm, rho, u)

    sim = olb.Sim((N, N), rp.dx, "D2Q9", 2, rp.tau, rp.dt, interp_order=3, storage="fp64",
                  cs_scale=rp.cs_scale, log_every=LOG)
    sim.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())

    k_gpu, k_ora = [], []
    for _ in range(STEPS // LOG):
        sim.step(LOG)
        k_gpu.append(sim.kinetic_energy()[0])
        for _ in range(LOG):
            f, _, diag = O.step(prm, f)
        k_ora.append(diag["k"])
    got = sim.get_populations(np.zeros_like(f))
    sim.close()

    assert np.abs(got - f).max() / np.abs(f).max() < 1e-11
    k_gpu, k_ora = np.array(k_gpu), np.array(k_ora)
    assert (np.abs(k_gpu - k_ora) / k_ora).max() < 1e-11

    # the analytic decay of the velocity amplitude, exp(-2 nu t)
    _, uu, _ = O.moments_of_state(prm, got)
    x = np.arange(N) * rp.dx
    Y, X = np.meshgrid(x, x, indexing="ij")
    amp = 4.0 * (uu[0] * np.sin(X) * np.cos(Y)).mean() / rp.u0
    assert abs(amp / math.exp(-2.0 * rp.nu * STEPS * rp.dt) - 1.0) < 1e-3

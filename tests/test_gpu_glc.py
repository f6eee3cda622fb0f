"""GPU parity of the step with the paper's cell-wise interpolation (Sec. 3:
Lagrange interpolation of the departure point in the cell that contains it, on
Gauss-Lobatto-Chebyshev support points) against the oracle (oracle/glc.py,
pinned on the CPU by brute force, exactness and convergence).

Each case sets the same seeded state on both sides, switches the handle to the
cell-wise pull (olb_set_interpolation), advances one step (or ten) and compares
every population; metric and bounds as in test_gpu_parity.py (FP64 1e-12,
FP32 2e-5 of the largest deviation from w rho0).  Every axis holds whole cells
(n a multiple of p).
"""
import math

import numpy as np
import pytest

from oracle import glc as G

from test_gpu_parity import base_of, make_pair, rel_err, TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def olb():
    from paper_2101_03982_gb300 import olb as ob
    ob.lib()
    return ob


def glc_steps(prm, state, steps=1):
    Q = prm.vs.Q
    f = state[:Q]
    g = state[Q:] if prm.compressible else None
    diag = None
    for _ in range(steps):
        f, g, diag = G.step(prm, f, g)
    return (np.concatenate([f, g]) if prm.compressible else f), diag


CASES = [
    # name, shape (x, y[, z]), N, p, storage, compressible, courant, cs_scale
    ("D3Q27", (16, 12, 8), 2, 4, "fp64", False, 0.4, 1.0),
    ("D3Q27", (12, 9, 6), 2, 3, "fp64", False, 0.4, 1.0),
    ("D3Q13", (16, 8, 12), 2, 4, "fp64", False, 0.4, 1.0),
    ("D3V27", (8, 12, 16), 3, 4, "fp64", False, 0.4, 1.0),
    ("D2Q9", (20, 16), 2, 4, "fp64", False, 0.4, 1 / math.sqrt(3)),
    ("D2Q25", (16, 12), 4, 4, "fp64", True, 0.4, 1.0),
    ("D3Q45", (8, 8, 12), 4, 4, "fp64", True, 0.4, 1.0),
    ("D3Q27", (16, 12, 8), 2, 4, "fp32", False, 0.4, 1.0),
    ("D3Q21", (12, 12, 8), 2, 4, "fp32", False, 0.4, 1.0),
    ("D2Q19", (16, 12), 4, 4, "fp32", True, 0.4, 1.0),
    # several tiles of the pull (32 x 16 x 16; FP64 32 x 16 x 8; 2D 32 x 32) with ragged tails:
    # 16-byte staging (n_x a multiple of 16 bytes' elements) and element staging
    ("D3Q27", (72, 36, 20), 2, 4, "fp32", False, 0.4, 1.0),
    ("D3Q27", (66, 33, 18), 2, 3, "fp32", False, 0.4, 1.0),
    ("D3Q27", (40, 34, 18), 2, 2, "fp64", False, 0.4, 1.0),
    ("D2Q9", (68, 40), 2, 4, "fp64", False, 1.3, 1 / math.sqrt(3)),
    # 16-bit storage: staged as stored (16-byte copies, or element loads when n_x is not a multiple of 8)
    ("D3Q27", (72, 36, 20), 2, 4, "bf16", False, 0.4, 1.0),
    ("D3Q27", (36, 20, 16), 2, 4, "fp16", False, 0.4, 1.0),
    ("D2Q19", (48, 36), 4, 4, "fp16", True, 0.4, 1.0),
]


@pytest.mark.parametrize("name,shape,N,p,storage,comp,courant,cs", CASES)
def test_one_step_parity_glc(olb, name, shape, N, p, storage, comp, courant, cs):
    sim, prm, state = make_pair(olb, name, shape, N=N, p=p, storage=storage, comp=comp, courant=courant,
                                cs_scale=cs)
    sim.set_interpolation("glc")
    want, diag = glc_steps(prm, state)
    sim.step(1)
    got = sim.get_populations(np.zeros_like(state))
    err = rel_err(got, want, base_of(prm, storage, state.shape[0]), storage)
    assert err < TOL[storage], err
    red = sim.reductions()
    # the pulled values pass between the two launches in the storage type: with
    # 16-bit storage they are rounded once more than in the uniform pull
    slack = {"fp64": 0.0, "fp32": 1e-6, "bf16": 1e-4, "fp16": 1e-5}[storage]
    assert abs(red["k"] - diag["k"]) <= (1e-9 + slack) * diag["k"]
    assert abs(red["mass"] - diag["mass"]) <= (1e-12 + slack) * diag["mass"]
    sim.close()


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_one_step_parity_glc_prandtl(olb, storage):
    """The GLC pull with the compressible collision at Pr = 0.75."""
    sim, prm, state = make_pair(olb, "D3Q45", (16, 16, 12), N=4, p=4, storage=storage, comp=True, prandtl=0.75)
    sim.set_interpolation("glc")
    want, _ = glc_steps(prm, state)
    sim.step(1)
    got = sim.get_populations(np.zeros_like(state))
    assert rel_err(got, want, base_of(prm, storage, state.shape[0]), storage) < TOL[storage]
    sim.close()


def test_ten_steps_glc_fp64(olb):
    sim, prm, state = make_pair(olb, "D3Q27", (16, 16, 12), N=2, p=4)
    sim.set_interpolation("glc")
    want, _ = glc_steps(prm, state, steps=10)
    sim.step(10)
    got = sim.get_populations(np.zeros_like(state))
    assert rel_err(got, want, np.zeros(27), "fp64") < 1e-11
    sim.close()


def test_glc_differs_from_the_uniform_pull_and_switches_back(olb):
    """The two interpolations give different steps (p > 1), and scheme 0
    restores the uniform pull exactly."""
    sim, prm, state = make_pair(olb, "D3Q27", (16, 12, 8), N=2, p=4)
    sim.set_interpolation("glc")
    sim.step(1)
    a = sim.get_populations(np.zeros_like(state))
    sim.set_populations(state)
    sim.set_interpolation("uniform")
    sim.step(1)
    b = sim.get_populations(np.zeros_like(state))
    assert np.abs(a - b).max() > 1e-6 * np.abs(state).max()
    from test_gpu_parity import oracle_steps
    want, _ = oracle_steps(prm, state)
    assert rel_err(b, want, np.zeros(27), "fp64") < 1e-12
    sim.close()


def test_glc_argument_checks(olb):
    from paper_2101_03982_gb300 import olb as ob
    sim, _, _ = make_pair(olb, "D3Q27", (18, 12, 8), N=2, p=4)  # 18 is not a multiple of 4
    with pytest.raises(ob.OlbError) as e:
        sim.set_interpolation("glc")
    assert e.value.code == -1
    sim.close()
    sim, prm, _ = make_pair(olb, "D3Q27", (16, 12, 8), N=2, p=4, storage="fp32")
    rho_in = 1.0
    u_in = np.zeros(3)
    u_in[0] = 0.05
    sim.set_x_boundary("inflow_outflow", rho_in, u_in, 1.0)
    with pytest.raises(ob.OlbError) as e:
        sim.set_interpolation("glc")  # periodic grids only
    assert e.value.code == -7
    sim.close()

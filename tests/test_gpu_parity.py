"""GPU parity of the fused step against the FP64 oracle, through the C ABI.

Each case sets the same seeded state on both sides (the oracle builds it: an
equilibrium of seeded fields plus seeded noise), advances one step (or ten),
and compares every population.  Metric: max |f_gpu - f_oracle| divided by
max |f_oracle| (FP64, bound 1e-12), and by max |f_oracle - w rho0| for the
shifted storages (FP32 bound 2e-5; BF16/FP16 bounds 2e-2 / 4e-3, half an ulp
of the stored deviation grown over one step).  Grids span several tiles and
ragged tails (tiles are 32 x 8 x 8 in 3D and 32 x 64 in 2D); odd nx takes the
scalar staging path, grids narrower than a staged box the modulo-wrap path.
"""
import math

import numpy as np
import pytest

from oracle import sllbm as O
from oracle import velocity_sets as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5, "bf16": 2e-2, "fp16": 4e-3}


@pytest.fixture(scope="module")
def olb():
    from paper_2101_03982_gb300 import olb as ob
    ob.lib()
    return ob


def make_pair(olb, name, shape, N=2, p=4, storage="fp64", comp=False, courant=0.4, cs_scale=1.0, tau=0.7,
              mu=0.02, gamma=1.4, seed=1, kernel="auto", mu_exponent=0.0, prandtl=1.0):
    vs = V.get(name)
    if cs_scale != 1.0:
        vs = vs.scaled(cs_scale)
    dx = 0.05
    dt = courant * dx / np.abs(vs.xi).max()
    prm = O.Params(vs, N, p, dt=dt, dx=dx, tau=tau, compressible=comp, gamma=gamma, mu=mu, mu_exponent=mu_exponent,
                   prandtl=prandtl)
    sim = olb.Sim(shape, dx, name, N, tau, dt, interp_order=p, storage=storage, cs_scale=cs_scale,
                  compressible=comp, gamma=gamma, mu=mu, kernel=kernel, mu_exponent=mu_exponent, prandtl=prandtl)
    rng = np.random.default_rng(seed)
    grid = tuple(reversed(shape))
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, grid)
    u = 0.08 * vs.cs * rng.uniform(-1, 1, (vs.D,) + grid)
    theta = 1.0 + 0.1 * rng.uniform(-1, 1, grid) if comp else None
    f, g = O.init_equilibrium(prm, rho, u, theta)
    f = f * (1.0 + 2e-3 * rng.uniform(-1, 1, f.shape))
    if comp:
        g = g * (1.0 + 2e-3 * rng.uniform(-1, 1, g.shape))
    state = np.concatenate([f, g]) if comp else f
    sim.set_populations(np.ascontiguousarray(state))
    # the oracle starts from exactly what the device stores (storage rounding)
    stored = sim.get_populations(np.zeros_like(state))
    return sim, prm, stored


def base_of(prm, storage, planes):
    if storage == "fp64":
        return np.zeros(planes)
    w = prm.vs.w
    if planes == prm.vs.Q:
        return w
    Cv = 1.0 / (prm.gamma - 1.0)
    return np.concatenate([w, w * (2 * Cv - prm.vs.D)])


def oracle_steps(prm, state, steps=1):
    Q = prm.vs.Q
    f = state[:Q]
    g = state[Q:] if prm.compressible else None
    diag = None
    for _ in range(steps):
        f, g, diag = O.step(prm, f, g)
    return (np.concatenate([f, g]) if prm.compressible else f), diag


def rel_err(got, want, base, storage):
    shape = (-1,) + (1,) * (want.ndim - 1)
    dev = want - base.reshape(shape)
    scale = np.abs(want).max() if storage == "fp64" else np.abs(dev).max()
    return np.abs(got - want).max() / scale


CASES = [
    # name, shape (x, y[, z]), N, p, storage, compressible, courant, cs_scale
    ("D2Q9", (64, 64), 2, 3, "fp64", False, 0.4, 1 / math.sqrt(3)),
    ("D2Q9", (70, 45), 2, 3, "fp64", False, 0.4, 1 / math.sqrt(3)),
    ("D2Q9", (45, 70), 2, 4, "fp64", False, 2.3, 1 / math.sqrt(3)),
    ("D3Q27", (40, 20, 18), 2, 4, "fp64", False, 0.4, 1.0),
    ("D3Q27", (33, 9, 10), 2, 3, "fp64", False, 0.4, 1.0),
    ("D3Q13", (32, 24, 17), 2, 4, "fp64", False, 0.4, 1.0),
    ("D3Q21", (36, 17, 11), 2, 4, "fp64", False, 0.4, 1.0),
    ("D3V27", (34, 16, 9), 3, 4, "fp64", False, 0.4, 1.0),
    ("D3Q45", (32, 12, 10), 2, 4, "fp64", False, 0.4, 1.0),
    ("D2Q19", (40, 70), 4, 4, "fp64", True, 0.4, 1.0),
    ("D2Q25", (66, 33), 4, 4, "fp64", True, 0.4, 1.0),
    ("D3Q45", (16, 12, 10), 4, 4, "fp64", True, 0.4, 1.0),
    ("D3Q45", (34, 10, 9), 4, 3, "fp64", True, 1.3, 1.0),
    ("D3Q27", (40, 20, 18), 2, 4, "fp32", False, 0.4, 1.0),
    ("D3Q45", (36, 17, 11), 2, 4, "fp32", False, 0.4, 1.0),
    ("D2Q9", (64, 64), 2, 3, "fp32", False, 0.4, 1 / math.sqrt(3)),
    ("D3Q45", (32, 16, 10), 4, 4, "fp32", True, 0.4, 1.0),
    ("D2Q19", (40, 70), 4, 4, "fp32", True, 0.4, 1.0),
    ("D3Q27", (40, 20, 18), 2, 4, "bf16", False, 0.4, 1.0),
    ("D3Q27", (40, 20, 18), 2, 4, "fp16", False, 0.4, 1.0),
    ("D3Q27", (37, 20, 18), 2, 4, "fp32", False, 0.4, 1.0),
    ("D3Q27", (8, 3, 2), 2, 4, "fp32", False, 0.4, 1.0),
    ("D2Q9", (4, 1), 2, 3, "fp64", False, 0.4, 1 / math.sqrt(3)),
    ("D3Q45", (64, 40, 24), 2, 4, "fp32", False, 0.4, 1.0),
]


# the single-role kernel (the automatic choice runs the warp-specialized one
# for the shifted storages)
GENERIC = [c for c in CASES if c[4] != "fp64"][:4] + [("D3Q45", (16, 12, 10), 4, 4, "fp32", True, 0.4, 1.0)]


@pytest.mark.parametrize("kernel", ["auto"])
@pytest.mark.parametrize("name,shape,N,p,storage,comp,courant,cs", CASES)
def test_one_step_parity(olb, name, shape, N, p, storage, comp, courant, cs, kernel):
    _one_step(olb, name, shape, N, p, storage, comp, courant, cs, kernel)


@pytest.mark.parametrize("name,shape,N,p,storage,comp,courant,cs", GENERIC)
def test_one_step_parity_generic_kernel(olb, name, shape, N, p, storage, comp, courant, cs):
    _one_step(olb, name, shape, N, p, storage, comp, courant, cs, "generic")


# isothermal FP32 3D: every set of up to 27 velocities, several tiles and
# several tiles per CTA (the last case), ragged tails, a grid smaller than one
# tile, an odd nx (node-by-node stores), p = 3 and 4, N = 2 and 3, a Courant
# number above 1
ISO32_CASES = [
    ("D3Q27", (40, 20, 18), 2, 4, "fp32", False, 0.4, 1.0),
    ("D3Q27", (37, 20, 18), 2, 4, "fp32", False, 0.4, 1.0),
    ("D3Q27", (33, 9, 10), 2, 3, "fp32", False, 0.4, 1.0),
    ("D3Q27", (8, 3, 2), 2, 4, "fp32", False, 0.4, 1.0),
    ("D3Q13", (32, 24, 17), 2, 4, "fp32", False, 0.4, 1.0),
    ("D3Q21", (36, 17, 11), 2, 4, "fp32", False, 0.4, 1.0),
    ("D3V27", (34, 16, 9), 3, 4, "fp32", False, 0.4, 1.0),
    ("D3Q27", (64, 16, 12), 2, 4, "fp32", False, 1.3, 1.0),
    ("D3Q27", (160, 96, 80), 2, 4, "fp32", False, 0.4, 1.0),
]


@pytest.mark.parametrize("kernel", ["auto", "twophase"])
@pytest.mark.parametrize("name,shape,N,p,storage,comp,courant,cs", ISO32_CASES)
def test_one_step_parity_fp32_iso(olb, name, shape, N, p, storage, comp, courant, cs, kernel):
    _one_step(olb, name, shape, N, p, storage, comp, courant, cs, kernel)


MU_OF_THETA = [
    ("D2Q19", (40, 70), 4, "fp64", "auto", 0.7),
    ("D3Q45", (34, 10, 9), 3, "fp64", "auto", -0.5),
    ("D3Q45", (32, 16, 10), 4, "fp32", "auto", 0.7),
    ("D2Q19", (40, 70), 4, "fp32", "auto", 0.7),
    ("D3Q45", (16, 12, 10), 4, "fp32", "generic", 0.7),
    ("D3Q45", (16, 12, 10), 4, "fp64", "generic", 0.7),
]


@pytest.mark.parametrize("name,shape,p,storage,kernel,omega", MU_OF_THETA)
def test_one_step_parity_viscosity_power_law(olb, name, shape, p, storage, kernel, omega):
    """Compressible step with mu(theta) = mu theta^omega in every kernel that
    runs the compressible collision."""
    _one_step(olb, name, shape, 4, p, storage, True, 0.4, 1.0, kernel, mu_exponent=omega)


PRANDTL = [
    ("D2Q19", (40, 70), 4, "fp64", "auto", 0.75, 0.0),
    ("D2Q25", (40, 70), 4, "fp32", "auto", 0.75, 0.0),
    ("D2Q19", (33, 70), 3, "fp32", "auto", 2.0, 0.7),
    ("D3Q45", (34, 10, 9), 4, "fp64", "auto", 0.75, 0.0),
    ("D3Q45", (32, 16, 10), 4, "fp32", "auto", 0.75, 0.0),
    ("D3Q45", (32, 16, 10), 3, "fp32", "auto", 0.5, 0.7),
    ("D3Q45", (32, 16, 10), 4, "bf16", "auto", 0.75, 0.0),
    ("D3Q45", (32, 16, 10), 4, "fp16", "auto", 0.75, 0.0),
    ("D3Q45", (16, 12, 10), 4, "fp32", "generic", 0.75, 0.0),
    ("D3Q45", (16, 12, 10), 4, "fp64", "generic", 1.6, 0.0),
    ("D2Q25", (36, 20), 5, "fp64", "generic", 0.75, 0.0),
]


@pytest.mark.parametrize("name,shape,p,storage,kernel,pr,omega", PRANDTL)
def test_one_step_parity_prandtl(olb, name, shape, p, storage, kernel, pr, omega):
    """Compressible step with the heat-flux quasi-equilibrium (Pr != 1) in
    every kernel and storage that runs the compressible collision."""
    _one_step(olb, name, shape, 4, p, storage, True, 0.4, 1.0, kernel, mu_exponent=omega, prandtl=pr)


def test_ten_steps_prandtl_fp64(olb):
    sim, prm, state = make_pair(olb, "D3Q45", (32, 16, 10), N=4, p=4, comp=True, prandtl=0.75)
    want, _ = oracle_steps(prm, state, steps=10)
    sim.step(10)
    got = sim.get_populations(np.zeros_like(state))
    assert rel_err(got, want, np.zeros(state.shape[0]), "fp64") < 1e-11
    sim.close()


def _one_step(olb, name, shape, N, p, storage, comp, courant, cs, kernel, mu_exponent=0.0, prandtl=1.0):
    sim, prm, state = make_pair(olb, name, shape, N=N, p=p, storage=storage, comp=comp, courant=courant,
                                cs_scale=cs, kernel=kernel, mu_exponent=mu_exponent, prandtl=prandtl)
    want, diag = oracle_steps(prm, state)
    sim.step(1)
    got = sim.get_populations(np.zeros_like(state))
    err = rel_err(got, want, base_of(prm, storage, state.shape[0]), storage)
    assert err < TOL[storage], err
    red = sim.reductions()
    assert abs(red["k"] - diag["k"]) <= 1e-9 * diag["k"] + (1e-6 * diag["k"] if storage != "fp64" else 0)
    assert abs(red["mass"] - diag["mass"]) <= 1e-12 * diag["mass"] + (1e-6 * diag["mass"] if storage != "fp64" else 0)
    if storage == "fp64":
        assert abs(red["eps"] - diag["eps"]) <= 1e-8 * abs(diag["eps"])
        assert np.allclose(red["momentum"], diag["momentum"], atol=1e-11 * diag["mass"])
    sim.close()


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_interpolation_orders_fp64(olb, p):
    sim, prm, state = make_pair(olb, "D3Q27", (34, 12, 9), N=2, p=p)
    want, _ = oracle_steps(prm, state)
    sim.step(1)
    got = sim.get_populations(np.zeros_like(state))
    assert rel_err(got, want, np.zeros(27), "fp64") < 1e-12
    sim.close()


def test_ten_steps_fp32(olb):
    sim, prm, state = make_pair(olb, "D3Q27", (64, 24, 20), N=2, p=4, storage="fp32")
    want, _ = oracle_steps(prm, state, steps=10)
    sim.step(10)
    got = sim.get_populations(np.zeros_like(state))
    assert rel_err(got, want, prm.vs.w, "fp32") < 1e-4
    sim.close()


def test_ten_steps_fp64(olb):
    sim, prm, state = make_pair(olb, "D3Q27", (32, 16, 16), N=2, p=4)
    want, _ = oracle_steps(prm, state, steps=10)
    sim.step(10)
    got = sim.get_populations(np.zeros_like(state))
    assert rel_err(got, want, np.zeros(27), "fp64") < 1e-12
    sim.close()


def test_stencil_table_matches_oracle(olb):
    sim, prm, _ = make_pair(olb, "D3Q45", (16, 16, 16), N=2, p=4, courant=1.7)
    m0, W = sim.stencil()
    deltas = O.departure_offsets(prm.vs.xi, prm.dt, prm.dx)
    for i in range(prm.vs.Q):
        for a in range(3):
            om0, oW = O.stencil_1d(deltas[i, a], 4)
            assert m0[i, a] == om0
            assert np.allclose(W[i, a], oW, atol=1e-15)
    sim.close()


@pytest.mark.parametrize("name,storage,comp", [("D3Q27", "fp64", False), ("D3Q45", "fp32", True),
                                               ("D2Q9", "bf16", False)])
def test_init_and_moments_match_oracle(olb, name, storage, comp):
    vs = V.get(name)
    shape = (20, 12, 9) if vs.D == 3 else (24, 20)
    grid = tuple(reversed(shape))
    prm = O.Params(vs, 4 if comp else 2, 4, dt=0.01, dx=0.05, tau=0.7, compressible=comp, mu=0.01)
    sim = olb.Sim(shape, 0.05, name, prm.N, 0.7, 0.01, interp_order=4, storage=storage, compressible=comp, mu=0.01)
    rng = np.random.default_rng(9)
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, grid)
    u = 0.1 * rng.uniform(-1, 1, (vs.D,) + grid)
    theta = 1.0 + 0.2 * rng.uniform(-1, 1, grid) if comp else None
    sim.init_fields(rho, u, theta)
    f, g = O.init_equilibrium(prm, rho, u, theta)
    want = np.concatenate([f, g]) if comp else f
    got = sim.get_populations(np.zeros_like(want))
    err = rel_err(got, want, base_of(prm, storage, want.shape[0]), storage)
    assert err < {"fp64": 1e-13, "fp32": 1e-6, "bf16": 1e-2}[storage]
    n = int(np.prod(shape))
    r2, u2, t2 = np.zeros(n), np.zeros(vs.D * n), np.zeros(n)
    sim.moments(r2, u2, t2)
    orr, ou, ot = O.moments_of_state(prm, got[:vs.Q].reshape((vs.Q,) + grid),
                                     got[vs.Q:].reshape((vs.Q,) + grid) if comp else None)
    assert np.allclose(r2, orr.ravel(), rtol=1e-12)
    assert np.allclose(u2, ou.reshape(-1), atol=1e-12)
    if comp:
        assert np.allclose(t2, ot.ravel(), rtol=1e-11)
    sim.close()


def test_state_round_trip_and_device_pointers(olb):
    sim, prm, state = make_pair(olb, "D3Q27", (32, 8, 8), N=2, p=3, storage="fp32")
    nb = sim.state_bytes()
    raw = torch.empty(nb, dtype=torch.uint8, device="cuda")
    sim.get_state(raw)
    sim.step(3)
    sim.set_state(raw)
    back = torch.empty_like(raw)
    sim.get_state(back)
    assert torch.equal(raw, back)
    host = np.zeros(nb, dtype=np.uint8)
    sim.get_state(host)
    assert np.array_equal(host, raw.cpu().numpy())
    f = torch.zeros(state.shape, dtype=torch.float64, device="cuda")
    sim.get_populations(f)
    assert np.allclose(f.cpu().numpy(), state, rtol=0, atol=0)
    sim.close()


@pytest.mark.parametrize("name,shape,p,storage", [("D3Q27", (37, 11, 9), 4, "fp32"), ("D3Q27", (33, 9, 10), 3, "fp64"),
                                                   ("D3Q27", (40, 20, 18), 4, "fp16")])
def test_set_state_fills_the_ghost_copies(olb, name, shape, p, storage):
    """A state written back through the compact copy steps exactly as the
    original: every periodic copy in the ghost layers was refilled (ragged
    rows included)."""
    sim, prm, state = make_pair(olb, name, shape, N=2, p=p, storage=storage)
    raw = torch.empty(sim.state_bytes(), dtype=torch.uint8, device="cuda")
    sim.get_state(raw)
    sim.step(2)
    want = sim.get_populations(np.zeros_like(state))
    sim.step(1)
    sim.set_state(raw.cpu().numpy())
    sim.step(2)
    got = sim.get_populations(np.zeros_like(state))
    assert np.array_equal(got, want)
    sim.close()


def test_state_through_pinned_host_memory(olb):
    """Page-locked host buffers are read and written in place by the copy
    kernels: the same bytes as through device memory, and a state set from
    one steps exactly as the original."""
    sim, prm, state = make_pair(olb, "D3Q27", (37, 11, 9), N=2, p=4, storage="fp32")
    nb = sim.state_bytes()
    dev = torch.empty(nb, dtype=torch.uint8, device="cuda")
    pinned = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    sim.get_state(dev)
    sim.get_state(pinned)
    assert torch.equal(pinned, dev.cpu())
    sim.step(2)
    want = sim.get_populations(np.zeros_like(state))
    sim.step(1)
    sim.set_state(pinned)
    sim.step(2)
    assert np.array_equal(sim.get_populations(np.zeros_like(state)), want)
    sim.close()


def test_nonfinite_state_is_reported(olb):
    sim, prm, state = make_pair(olb, "D3Q27", (32, 8, 8), N=2, p=3)
    bad = state.copy()
    bad[5, 3, 2, 1] = np.nan
    sim.set_populations(bad)
    red = sim.reductions(check=False)
    assert red["rc"] == -4 and red["nonfinite"] >= 1
    sim.step(1)
    red = sim.reductions(check=False)
    assert red["rc"] == -4
    sim.close()


def test_synchronize_with_time_limit(olb):
    sim, _, _ = make_pair(olb, "D3Q27", (32, 16, 16), N=2, p=4)
    sim.step(2)
    sim.synchronize(timeout_ms=60000)
    sim.close()

"""GPU parity of the adjoint of the isothermal step against the FP64 oracle.

The oracle's adjoint (oracle/adjoint.py) is pinned on the CPU against finite
differences of the forward oracle and the transpose identity of the pull.
Here the library's adjoint kernels, called through the C ABI, are compared
with it on the same seeded states and seeds:

* one step (olb_adjoint_step) for several sets, orders and ragged grids;
* a recorded trajectory swept back in full and in part (olb_tape_*);
* the seed from the moments and the gradient through the initial
  equilibrium (olb_moments_vjp, olb_equilibrium_vjp);
* the torch.autograd.Function with checkpoints: gradients of the final
  kinetic energy and of a velocity misfit with respect to the initial
  velocity, against central finite differences along random divergence-free
  directions (FP64 and FP32 runs against the FP64 differences) and against
  the CPU FP64 adjoint at 16^3.

Metric: max |got - want| / max |want|; FP64 bound 1e-12 (one step) and 1e-11
(trajectories), FP32 bound 2e-5 (FP32 arithmetic on O(1) adjoints).
"""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle import sllbm as O
from oracle import velocity_sets as V

from test_gpu_parity import make_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL1 = {"fp64": 1e-12, "fp32": 2e-5}
TOLN = {"fp64": 1e-11, "fp32": 2e-5}


@pytest.fixture(scope="module")
def olb():
    from paper_2101_03982_gb300 import olb as ob
    ob.lib()
    return ob


def rel(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


def state_bytes_of(sim):
    return np.zeros(sim.state_bytes(), dtype=np.uint8)


ONE_STEP = [
    ("D3Q27", (40, 20, 18), 2, 4, "fp64", 1.0),
    ("D3Q27", (37, 11, 9), 2, 3, "fp64", 1.0),
    ("D3Q27", (40, 20, 18), 2, 4, "fp32", 1.0),
    ("D3V27", (33, 9, 10), 3, 3, "fp64", 1.0),
    ("D3V27", (34, 16, 9), 3, 4, "fp64", 1.0),
    ("D3Q13", (32, 24, 17), 2, 4, "fp64", 1.0),
    ("D3Q21", (36, 17, 11), 2, 4, "fp32", 1.0),
    ("D3Q45", (32, 12, 10), 2, 4, "fp64", 1.0),
    ("D3Q45", (36, 17, 11), 2, 3, "fp32", 1.0),
    ("D2Q9", (64, 45), 2, 3, "fp64", 1 / np.sqrt(3)),
    ("D2Q9", (70, 45), 2, 4, "fp32", 1 / np.sqrt(3)),
    ("D2Q25", (66, 33), 3, 4, "fp64", 1.0),
    ("D2Q19", (40, 70), 2, 3, "fp64", 1.0),
]


@pytest.mark.parametrize("name,shape,N,p,storage,cs", ONE_STEP)
def test_adjoint_step_matches_oracle(olb, name, shape, N, p, storage, cs):
    sim, prm, f = make_pair(olb, name, shape, N=N, p=p, storage=storage, cs_scale=cs, courant=0.9)
    fwd = sim.get_state(state_bytes_of(sim))
    rng = np.random.default_rng(31)
    lam = rng.standard_normal(f.shape)
    want = A.step_vjp(prm, f, lam)
    got = sim.adjoint_step(fwd, np.ascontiguousarray(lam.astype(sim.adjoint_dtype)))
    err = rel(got.astype(np.float64), want)
    assert err < TOL1[storage], err
    sim.close()


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_tape_adjoint_matches_oracle_trajectory(olb, storage):
    sim, prm, f0 = make_pair(olb, "D3Q27", (36, 17, 11), N=2, p=3, storage=storage, courant=0.6)
    sim.tape_reserve(5)
    sim.tape_record(4)
    rng = np.random.default_rng(32)
    lamT = rng.standard_normal(f0.shape)
    # full sweep over the four recorded steps
    got = sim.tape_adjoint(np.ascontiguousarray(lamT.astype(sim.adjoint_dtype)), 4).astype(np.float64)
    want, fT = A.trajectory_vjp(prm, f0, 4, lamT)
    assert rel(got, want) < TOLN[storage]
    # the handle advanced by the four steps
    fT_gpu = sim.get_populations(np.zeros_like(f0))
    assert np.abs(fT_gpu - fT).max() < (1e-12 if storage == "fp64" else 1e-5)
    # partial sweep: the last two steps only
    states = [f0]
    for _ in range(4):
        states.append(O.step(prm, states[-1])[0])
    lam2 = A.step_vjp(prm, states[2], A.step_vjp(prm, states[3], lamT))
    got2 = sim.tape_adjoint(np.ascontiguousarray(lamT.astype(sim.adjoint_dtype)), 2).astype(np.float64)
    assert rel(got2, lam2) < TOLN[storage]
    sim.close()


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_moments_and_equilibrium_vjp(olb, storage):
    sim, prm, f = make_pair(olb, "D3V27", (20, 12, 9), N=3, p=4, storage=storage)
    vs = prm.vs
    Q = vs.Q
    rng = np.random.default_rng(33)
    grid = f.shape[1:]
    gr = rng.standard_normal(grid)
    gu = rng.standard_normal((3,) + grid)
    lam = sim.moments_vjp(gr, gu, np.zeros(f.shape, dtype=sim.adjoint_dtype)).astype(np.float64)
    want = A.moments_vjp(vs, f.reshape(Q, -1), gr.ravel(), gu.reshape(3, -1).T).reshape(f.shape)
    tol = 1e-12 if storage == "fp64" else 1e-5
    assert rel(lam, want) < tol
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, grid)
    u = 0.08 * vs.cs * rng.uniform(-1, 1, (3,) + grid)
    lam_in = rng.standard_normal(f.shape)
    g_rho, g_u = np.zeros(grid), np.zeros((3,) + grid)
    sim.equilibrium_vjp(rho, u, np.ascontiguousarray(lam_in.astype(sim.adjoint_dtype)), g_rho, g_u)
    wr, wu = A.equilibrium_vjp(vs, 3, rho.ravel(), u.reshape(3, -1).T, lam_in.reshape(Q, -1).astype(
        sim.adjoint_dtype).astype(np.float64))
    assert rel(g_rho.ravel(), wr) < 1e-12
    assert rel(g_u.reshape(3, -1).T, wu) < 1e-12
    sim.close()


def test_unsupported_configurations_are_rejected(olb):
    sim, _, _ = make_pair(olb, "D3Q27", (16, 8, 8), N=2, p=4, storage="bf16")
    with pytest.raises(olb.OlbError) as e:
        sim.tape_reserve(2)
    assert e.value.code == -7
    sim.close()
    sim, _, _ = make_pair(olb, "D3Q45", (16, 8, 8), N=4, p=4, storage="fp32", comp=True)
    with pytest.raises(olb.OlbError) as e:
        sim.tape_reserve(2)
    assert e.value.code == -7
    sim.close()
    sim, _, _ = make_pair(olb, "D3Q27", (16, 8, 8), N=2, p=4, storage="fp64")
    sim.tape_reserve(3)
    with pytest.raises(olb.OlbError) as e:
        sim.tape_record(4)  # needs 4 slots
    assert e.value.code == -6
    sim.close()


# --------------------------------------------------------------------------
# autograd with checkpoints: gradients with respect to the initial velocity
# --------------------------------------------------------------------------

def tgv_sim(olb, n, storage):
    """D3Q27, N = 2, p = 3, Re = 400, Ma = 0.1, Courant 0.4 (the adjoint workload's parameters)."""
    from paper_2101_03982_gb300 import params
    rp = params.tgv_isothermal("D3Q27", n, 400.0, 0.1, 0.4)
    return olb.Sim((n, n, n), rp.dx, "D3Q27", 2, rp.tau, rp.dt, interp_order=3, storage=storage,
                   cs_scale=rp.cs_scale), rp


def initial_fields(n, rng, rms):
    from paper_2101_03982_gb300 import inputs
    u0 = inputs.solenoidal(n, rng, rms)
    rho0 = np.ones((n, n, n))
    return rho0, u0


def run_J(sim, rho0, u0, nsteps, every, J):
    from paper_2101_03982_gb300.autograd import SimFunction
    r = torch.tensor(rho0, device="cuda")
    u = torch.tensor(u0, device="cuda", requires_grad=True)
    rho, uT = SimFunction.apply(r, u, sim, nsteps, every)
    val = J(rho, uT)
    val.backward()
    return float(val.item()), u.grad.detach().cpu().numpy()


def k_final(rho, u):
    return 0.5 * (u ** 2).sum(dim=0).mean()


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_simfunction_gradients_match_finite_differences(olb, storage):
    n, nsteps, every = 16, 12, 5
    rng = np.random.default_rng(20210111)
    rho0, u0 = initial_fields(n, rng, 1.0)
    from paper_2101_03982_gb300 import inputs
    target = inputs.solenoidal(n, rng, 1.0)
    dirs = [inputs.solenoidal(n, rng, 1.0) for _ in range(32)]
    tgt = torch.tensor(target, device="cuda")

    def misfit(rho, u):
        return 0.5 * ((u - tgt) ** 2).sum(dim=0).mean()

    sim64, _ = tgv_sim(olb, n, "fp64")
    sim, _ = tgv_sim(olb, n, storage)
    eps = 1e-6 * np.sqrt((u0 ** 2).sum())
    for J in (k_final, misfit):
        _, grad = run_J(sim, rho0, u0, nsteps, every, J)

        def J64(u):
            from paper_2101_03982_gb300.autograd import SimFunction
            with torch.no_grad():
                rho, uT = SimFunction.apply(torch.tensor(rho0, device="cuda"), torch.tensor(u, device="cuda"),
                                            sim64, nsteps, every)
                return float(J(rho, uT).item())

        fd = np.array([(J64(u0 + eps * v) - J64(u0 - eps * v)) / (2 * eps) for v in dirs])
        ad = np.array([float((grad * v).sum()) for v in dirs])
        scale = np.abs(fd).max()
        assert np.abs(ad - fd).max() <= 1e-4 * scale, (J.__name__, ad, fd)
        big = np.abs(fd) > 0.1 * scale
        assert (np.abs(ad - fd)[big] <= 1e-4 * np.abs(fd)[big]).all(), (J.__name__, ad, fd)
    sim.close()
    sim64.close()


def test_simfunction_gradient_matches_cpu_adjoint(olb):
    n, nsteps, every = 16, 6, 4
    rng = np.random.default_rng(20210111)
    rho0, u0 = initial_fields(n, rng, 1.0)
    sim, rp = tgv_sim(olb, n, "fp64")
    _, grad = run_J(sim, rho0, u0, nsteps, every, k_final)
    # CPU FP64 adjoint: oracle forward trajectory, seed, sweep, equilibrium link
    vs = V.get("D3Q27").scaled(rp.cs_scale)
    prm = O.Params(vs, 2, 3, dt=rp.dt, dx=rp.dx, tau=rp.tau)
    f0, _ = O.init_equilibrium(prm, rho0, u0)
    fT = f0
    for _ in range(nsteps):
        fT = O.step(prm, fT)[0]
    Q = vs.Q
    rhoT, uT = O.density_momentum(vs, fT.reshape(Q, -1))
    M = rhoT.shape[0]
    lamT = A.moments_vjp(vs, fT.reshape(Q, -1), np.zeros(M), uT / M).reshape(fT.shape)
    lam0, _ = A.trajectory_vjp(prm, f0, nsteps, lamT)
    _, gu = A.equilibrium_vjp(vs, 2, rho0.ravel(), u0.reshape(3, -1).T, lam0.reshape(Q, -1))
    want = gu.T.reshape(u0.shape)
    assert rel(grad, want) < 1e-10
    sim.close()

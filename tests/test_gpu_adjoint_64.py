"""The adjoint workload at its stated size: gradients through 500 steps at 64^3.

3D Taylor-Green vortex (Sec. 4.2 initial field), D3Q27, N = 2, p = 3,
Re = 400, Ma = 0.1, Courant 0.4, 64^3 periodic nodes; 500 forward steps with
a checkpoint every 25 steps (SimFunction recomputes each segment onto the
device tape and sweeps it back).  Two objectives of the final state u_T:

* J1 = k_final = mean |u_T|^2 / 2 (Sec. 4.2's kinetic energy);
* J2 = mean |u_T - u_target|^2 / 2, u_target a divergence-free random field
  (curl of a random vector potential, Fourier modes 1 <= |k| <= 4, Gaussian
  amplitudes, numpy default_rng(20210111), scaled to the rms of u0).

Both gradients with respect to the initial velocity, from FP64 and from FP32
storage, are checked against central differences of FP64 forward runs along
32 divergence-free directions drawn from the same stream after u_target
(epsilon = 1e-6 ||u0||): within 1e-4 of the largest difference, and within
1e-4 relative on every direction whose difference exceeds a tenth of it.
The transpose of the step has no counterpart in the paper; it is the exact
adjoint of the discrete step of Sec. 3.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_GRID, NSTEPS, EVERY = 64, 500, 25


@pytest.fixture(scope="module")
def workload():
    from paper_2101_03982_gb300 import inputs, olb, params
    olb.lib()
    rp = params.tgv_isothermal("D3Q27", N_GRID, 400.0, 0.1, 0.4)
    rho0, u0 = inputs.tgv3d(N_GRID, rp.u0, rp.cs ** 2)
    rng = np.random.default_rng(20210111)
    rms = float(np.sqrt((u0 ** 2).sum(axis=0).mean()))
    target = inputs.solenoidal(N_GRID, rng, rms)
    dirs = [inputs.solenoidal(N_GRID, rng, rms) for _ in range(32)]
    return rp, rho0, u0, target, dirs


def make_sim(olb, rp, storage):
    return olb.Sim((N_GRID,) * 3, rp.dx, "D3Q27", 2, rp.tau, rp.dt, interp_order=3, storage=storage,
                   cs_scale=rp.cs_scale, log_every=1000)


def objectives(tgt):
    def k_final(rho, u):
        return 0.5 * (u ** 2).sum(dim=0).mean()

    def misfit(rho, u):
        return 0.5 * ((u - tgt) ** 2).sum(dim=0).mean()

    return {"k_final": k_final, "misfit": misfit}


@pytest.fixture(scope="module")
def finite_differences(workload):
    """Central differences of both objectives along every direction (FP64 runs)."""
    from paper_2101_03982_gb300 import olb
    from paper_2101_03982_gb300.autograd import SimFunction
    rp, rho0, u0, target, dirs = workload
    tgt = torch.tensor(target, device="cuda")
    Js = objectives(tgt)
    sim = make_sim(olb, rp, "fp64")
    r = torch.tensor(rho0, device="cuda")
    eps = 1e-6 * float(np.sqrt((u0 ** 2).sum()))

    def run(u):
        with torch.no_grad():
            rho, uT = SimFunction.apply(r, torch.tensor(u, device="cuda"), sim, NSTEPS, EVERY)
            return {name: float(J(rho, uT).item()) for name, J in Js.items()}

    fd = {name: [] for name in Js}
    for v in dirs:
        jp, jm = run(u0 + eps * v), run(u0 - eps * v)
        for name in Js:
            fd[name].append((jp[name] - jm[name]) / (2 * eps))
    sim.close()
    return {name: np.array(val) for name, val in fd.items()}


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
@pytest.mark.parametrize("objective", ["k_final", "misfit"])
def test_gradient_after_500_steps_matches_finite_differences(workload, finite_differences, storage, objective):
    from paper_2101_03982_gb300 import olb
    from paper_2101_03982_gb300.autograd import SimFunction
    rp, rho0, u0, target, dirs = workload
    J = objectives(torch.tensor(target, device="cuda"))[objective]
    sim = make_sim(olb, rp, storage)
    u = torch.tensor(u0, device="cuda", requires_grad=True)
    rho, uT = SimFunction.apply(torch.tensor(rho0, device="cuda"), u, sim, NSTEPS, EVERY)
    J(rho, uT).backward()
    grad = u.grad.detach().cpu().numpy()
    sim.close()
    ad = np.array([float((grad * v).sum()) for v in dirs])
    fd = finite_differences[objective]
    scale = np.abs(fd).max()
    err = np.abs(ad - fd)
    print(f"{objective} {storage}: max |ad - fd| / max |fd| = {err.max() / scale:.3e}")
    assert err.max() <= 1e-4 * scale, (objective, storage, err.max() / scale)
    big = np.abs(fd) > 0.1 * scale
    assert (err[big] <= 1e-4 * np.abs(fd)[big]).all(), (objective, storage, (err[big] / np.abs(fd)[big]).max())

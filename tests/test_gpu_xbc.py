"""GPU parity of the non-periodic x (inflow / zero-gradient outflow ghost
columns, the standing-shock set-up of Sec. 4.1) against the oracle's
``step(..., xbc=...)``, which is pinned on its own (tests/test_oracle_xbc.py).

Each case starts from a seeded perturbed equilibrium, switches the handle to
inflow/outflow with an inflow state unlike the field's, and compares one and
then four more steps with the oracle.  The kernels that run: the two-phase
kernel (2D one-box and 3D in-place pulls, register and shared-memory-staged
collisions) and the single-role kernel.  Bounds as in the periodic parity
tests.  Also: back to periodic reproduces the periodic step, and the adjoint
is refused while x is not periodic.
"""
import numpy as np
import pytest

from oracle import sllbm as O

from test_gpu_parity import TOL, base_of, make_pair, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def olb():
    from paper_2101_03982_gb300 import olb as ob
    ob.lib()
    return ob


CASES = [
    # name, shape, N, p, storage, compressible, kernel
    ("D2Q19", (40, 70), 4, 4, "fp64", True, "auto"),
    ("D2Q19", (40, 70), 4, 4, "fp32", True, "auto"),
    ("D3Q27", (37, 11, 9), 2, 4, "fp32", False, "auto"),
    ("D3Q27", (33, 9, 10), 2, 3, "fp64", False, "auto"),
    ("D3Q45", (32, 16, 10), 4, 4, "fp32", True, "auto"),
    ("D3Q27", (40, 20, 18), 2, 4, "bf16", False, "auto"),
    ("D3Q27", (40, 20, 18), 2, 4, "fp32", False, "generic"),
]


def inflow_state(prm):
    D = prm.vs.D
    u = np.zeros(D)
    u[0] = 0.1 * prm.vs.cs
    if D > 1:
        u[1] = -0.02 * prm.vs.cs
    return 1.03, u, (1.08 if prm.compressible else 1.0)


@pytest.mark.parametrize("name,shape,N,p,storage,comp,kernel", CASES)
def test_inflow_outflow_steps_match_oracle(olb, name, shape, N, p, storage, comp, kernel):
    sim, prm, state = make_pair(olb, name, shape, N=N, p=p, storage=storage, comp=comp, kernel=kernel)
    rho_in, u_in, th_in = inflow_state(prm)
    sim.set_x_boundary("inflow_outflow", rho_in, u_in, th_in)
    xbc = O.inflow_populations(prm, rho_in, u_in, th_in)
    Q = prm.vs.Q
    f, g = state[:Q], (state[Q:] if comp else None)
    base = base_of(prm, storage, state.shape[0])
    done = 0
    for nsteps in (1, 4):
        for _ in range(nsteps):
            f, g, _ = O.step(prm, f, g, xbc=xbc)
        sim.step(nsteps)
        done += nsteps
        want = np.concatenate([f, g]) if comp else f
        got = sim.get_populations(np.zeros_like(state))
        err = rel_err(got, want, base, storage)
        assert err < TOL[storage] * done, (done, err)  # per-step bound, grown linearly as in the periodic tests
    sim.close()


@pytest.mark.parametrize("name,shape,N,storage,comp", [
    ("D3Q27", (37, 11, 9), 2, "fp32", False),
    ("D2Q19", (40, 33), 4, "fp64", True),
])
def test_back_to_periodic_and_adjoint_refused(olb, name, shape, N, storage, comp):
    """Switching back to periodic rewrites every ghost copy in place: the next
    step equals the oracle's periodic step of the same state.  The adjoint and
    the enstrophy (periodic differences) are refused while x is not periodic."""
    sim, prm, state = make_pair(olb, name, shape, N=N, p=4, storage=storage, comp=comp)
    rho_in, u_in, th_in = inflow_state(prm)
    sim.set_x_boundary("inflow_outflow", rho_in, u_in, th_in)
    if not comp:
        with pytest.raises(olb.OlbError) as e:
            sim.tape_reserve(2)
        assert e.value.code == -7
    with pytest.raises(olb.OlbError) as e:
        sim.enstrophy()
    assert e.value.code == -7
    sim.set_x_boundary("periodic")
    Q = prm.vs.Q
    f, g = O.step(prm, state[:Q], state[Q:] if comp else None)[:2]
    want = np.concatenate([f, g]) if comp else f
    sim.step(1)
    got = sim.get_populations(np.zeros_like(state))
    assert rel_err(got, want, base_of(prm, storage, state.shape[0]), storage) < TOL[storage]
    with pytest.raises(olb.OlbError) as e:
        sim.set_x_boundary("inflow_outflow", -1.0, u_in, th_in)
    assert e.value.code == -1
    sim.close()

"""The bounded-wait error path of the step kernels, exercised without a fault.

Every wait of a step kernel for a staging copy is bounded; when the bound runs
out the kernel raises the device error flag, waits (with the default bound)
for the copies it has in flight and returns, and the host reports
OLB_ETIMEOUT.  olb_set_wait_polls(h, 0) makes the first wait give up at once,
so the path runs deterministically with no copy left in flight.  Afterwards
the state is invalid until a new one is written; with the default bound back,
set_state and a step give exactly the result of a handle that never failed.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ETIMEOUT = -5


@pytest.mark.parametrize("kernel,storage", [("auto", "fp32"), ("auto", "fp64"), ("generic", "fp32")])
def test_wait_that_runs_out_reports_etimeout_and_the_handle_recovers(kernel, storage):
    from paper_2101_03982_gb300 import inputs, olb
    shape = (24, 20, 18)
    args = (shape, 0.05, "D3Q27", 2, 0.7, 0.01)
    kw = dict(interp_order=4, storage=storage, kernel=kernel)
    rho, u, _ = inputs.random_fields(tuple(reversed(shape)), 3, seed=5, u_amp=0.1)
    with olb.Sim(*args, **kw) as sim, olb.Sim(*args, **kw) as ref:
        sim.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        state0 = torch.empty(sim.state_bytes(), dtype=torch.uint8, device="cuda")
        sim.get_state(state0)
        sim.set_wait_polls(0)
        sim.step(1)  # enqueues the failing launch; the error shows at the next check
        red = sim.reductions(check=False)
        assert red["rc"] == ETIMEOUT
        with pytest.raises(olb.OlbError) as e:
            sim.step(1)  # the state is invalid: no step on it
        assert e.value.code == ETIMEOUT
        # a new state and the default bound: the step is exact again
        sim.set_wait_polls(-1)
        sim.set_state(state0)
        sim.step(2)
        sim.synchronize(60000)
        ref.set_state(state0)
        ref.step(2)
        got = torch.empty_like(state0)
        want = torch.empty_like(state0)
        sim.get_state(got)
        ref.get_state(want)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        r1, r2 = sim.reductions(), ref.reductions()
        assert r1["rc"] == 0 and r1["k"] == r2["k"]
        assert np.isfinite(r1["k"]) and r1["k"] > 0

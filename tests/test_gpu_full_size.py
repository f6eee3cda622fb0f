"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark times, on sampled outputs.

The oracle cannot step a 128^3 or 256^3 grid in seconds, but it computes the
post-collision populations of chosen nodes (``step_at_points``) from a stored
state.  Each case initialises the workload's field on the device exactly as
bench.py does, takes one step with the automatic kernel (the launch bench.py
times), and compares 4,096 randomly sampled nodes, every plane, with the
oracle stepping the same stored state at those nodes.  The oracle reads the
stored values it needs from the device state node by node, in FP64.

Cases: the 3D Taylor-Green vortex (Re 1600, Ma 0.1, p = 4, Courant 0.4) with
D3Q27 in FP32 and FP64 at 128^3 and D3Q45 (N = 2) in FP32 at 256^3, and the
compressible Taylor-Green vortex (D3Q45, N = 4, f + g, Ma 1.0, Pr 0.75) in FP32 at 256^3
and at 512^3, the largest workload (99 GB of A/B buffers).
Bounds as in the small-grid parity tests: FP32 2e-5 of the largest stored
deviation, FP64 1e-12 of the largest population.
"""
import numpy as np
import pytest

from oracle import sllbm as O
from oracle import velocity_sets as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NPTS = 4096


@pytest.fixture(scope="module")
def olb():
    from paper_2101_03982_gb300 import olb as ob
    ob.lib()
    return ob


class _DevPlane:
    def __init__(self, plane, base):
        self.plane, self.base = plane, base

    def __getitem__(self, idx):
        ii = tuple(torch.as_tensor(np.asarray(a), device=self.plane.device) for a in idx)
        return self.plane[ii].double().cpu().numpy() + self.base


class DevState:
    """Stored planes [plane][z][y][x] on the device, read as unshifted FP64."""

    def __init__(self, planes, base):
        self.planes, self.base = planes, base
        self.shape = tuple(planes.shape)

    def __getitem__(self, i):
        return _DevPlane(self.planes[i], float(self.base[i]))


def stored_planes(sim, dtype):
    raw = torch.empty(sim.state_bytes(), dtype=torch.uint8, device="cuda")
    sim.get_state(raw)
    return raw.view(dtype)


def base_of(prm, storage, comp):
    Q = prm.vs.Q
    if storage == "fp64":
        return np.zeros(2 * Q if comp else Q)
    w = prm.vs.w
    return np.concatenate([w, w * (2.0 / (prm.gamma - 1.0) - 3)]) if comp else w


def make_case(olb, name, n, storage, comp):
    from paper_2101_03982_gb300 import inputs, params
    if comp:
        rp = params.tgv_compressible(name, n, 1600.0, 1.0, 0.4)
        sim = olb.Sim((n,) * 3, rp.dx, name, 4, rp.tau, rp.dt, interp_order=4, storage=storage, compressible=True,
                      gamma=rp.gamma, mu=rp.mu, log_every=10, prandtl=0.75)
        rho, u, th = inputs.ctic3d(n, rp.u0)
        sim.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda(), torch.from_numpy(th).cuda())
        vs = V.get(name)
        prm = O.Params(vs, 4, 4, dt=rp.dt, dx=rp.dx, compressible=True, gamma=rp.gamma, mu=rp.mu, prandtl=0.75)
    else:
        rp = params.tgv_isothermal(name, n, 1600.0, 0.1, 0.4)
        sim = olb.Sim((n,) * 3, rp.dx, name, 2, rp.tau, rp.dt, interp_order=4, storage=storage,
                      cs_scale=rp.cs_scale, log_every=10)
        rho, u = inputs.tgv3d(n, rp.u0, rp.cs ** 2)
        sim.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        vs = V.get(name).scaled(rp.cs_scale)
        prm = O.Params(vs, 2, 4, dt=rp.dt, dx=rp.dx, tau=rp.tau)
    return sim, prm


@pytest.mark.parametrize("name,n,storage,comp", [("D3Q27", 128, "fp32", False), ("D3Q27", 128, "fp64", False),
                                                  ("D3Q45", 256, "fp32", False), ("D3Q45", 256, "fp32", True)])
def test_sampled_nodes_at_full_size(olb, name, n, storage, comp):
    sim, prm = make_case(olb, name, n, storage, comp)
    Q = prm.vs.Q
    dtype = torch.float64 if storage == "fp64" else torch.float32
    base = base_of(prm, storage, comp)
    before = stored_planes(sim, dtype).view(-1, n, n, n)
    sim.step(1)
    after = stored_planes(sim, dtype).view(-1, n, n, n)
    pts = np.random.default_rng(2101).integers(0, n, (NPTS, 3))
    f0 = DevState(before[:Q], base[:Q])
    g0 = DevState(before[Q:], base[Q:]) if comp else None
    fpost, gpost, _ = O.step_at_points(prm, f0, g0, pts)
    want = np.concatenate([fpost, gpost]) if comp else fpost
    idx = tuple(torch.as_tensor(pts[:, a], device="cuda") for a in (2, 1, 0))
    got = after[:, idx[0], idx[1], idx[2]].double().cpu().numpy() + base[:, None]
    if storage == "fp64":
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err < 1e-12, err
    else:
        err = np.abs(got - want).max() / np.abs(want - base[:, None]).max()
        assert err < 2e-5, err
    sim.close()


def test_sampled_nodes_at_512_cubed(olb):
    """The compressible D3Q45 workload at 512^3 (f + g, FP32): 99 GB of A/B
    buffers and a 48 GB compact copy of the state, the largest configuration.
    The oracle's values are taken from the copy before the step, which is then
    released, so the device holds at most about 150 GB."""
    import gc
    gc.collect()
    torch.cuda.empty_cache()
    n, Q = 512, 45
    sim, prm = make_case(olb, "D3Q45", n, "fp32", True)
    base = base_of(prm, "fp32", True)
    pts = np.random.default_rng(512).integers(0, n, (NPTS, 3))
    before = stored_planes(sim, torch.float32).view(-1, n, n, n)
    fpost, gpost, _ = O.step_at_points(prm, DevState(before[:Q], base[:Q]), DevState(before[Q:], base[Q:]), pts)
    want = np.concatenate([fpost, gpost])
    del before
    torch.cuda.empty_cache()
    sim.step(1)
    after = stored_planes(sim, torch.float32).view(-1, n, n, n)
    idx = tuple(torch.as_tensor(pts[:, a], device="cuda") for a in (2, 1, 0))
    got = after[:, idx[0], idx[1], idx[2]].double().cpu().numpy() + base[:, None]
    del after
    sim.close()
    torch.cuda.empty_cache()
    err = np.abs(got - want).max() / np.abs(want - base[:, None]).max()
    assert err < 2e-5, err

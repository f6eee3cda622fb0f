"""The allocation-free state sums agree with olb_reductions and with the oracle.

olb_state_sums_noalloc serves callers that cannot allocate device memory when
they need the global sums (their framework owns all device memory, or their
loop must not stall on cudaMalloc).  It keeps its per-block partial sums in a
fixed array inside the library.  Two calls in a row on different states and
grids -- first 96^3 (14 blocks of partial sums, so the final sum runs over
several slots), then 40 x 20 x 18 (one block) -- must each match the
handle-based olb_reductions (its stored-state path, the same FP64 arithmetic)
within 1e-12 relative, so a call never sees what the previous call left in the
shared array; k and the mass must also match the FP64 oracle's moments of the
same stored values within 1e-12.  Every storage type is covered.

This file is collected last on purpose: it also passes when run alone in a
fresh process, where its first call performs the one-time address lookup.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _grid(olb, shape):
    g = olb.Grid()
    g.dim = len(shape)
    n = list(shape) + [1] * (3 - len(shape))
    for k in range(3):
        g.n[k] = n[k]
    g.dx = 0.05
    return g


def _close(a, b, tol=1e-12):
    return abs(a - b) <= tol * max(1.0, abs(b))


def _stored_values(state, storage, Q, nodes):
    """FP64 copy of the raw stored values [Q][nodes] (no library conversion)."""
    raw = state.cpu().numpy()
    if storage == "fp64":
        v = raw.view(np.float64)
    elif storage == "fp32":
        v = raw.view(np.float32).astype(np.float64)
    elif storage == "fp16":
        v = raw.view(np.float16).astype(np.float64)
    else:  # bf16: the high half of an FP32 word
        v = (raw.view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return v.reshape(Q, nodes)


def _oracle_k_mass(values, storage, shape):
    from oracle import sllbm as O
    from oracle import velocity_sets as V
    vs = V.get("D3Q27")
    f = values + (0.0 if storage == "fp64" else 1.0) * vs.w[:, None]  # rho0 = 1
    prm = O.Params(vs, 2, 4, dt=0.01, dx=0.05, tau=0.7)
    rho, u, _ = O.moments_of_state(prm, f.reshape((vs.Q,) + tuple(reversed(shape))))
    return 0.5 * float((u ** 2).sum(axis=0).mean()), float(rho.sum())


@pytest.mark.parametrize("storage", ["fp32", "fp64", "bf16", "fp16"])
def test_noalloc_sums_match_reductions_and_the_oracle(storage):
    from paper_2101_03982_gb300 import inputs, olb
    L = olb.lib()
    out = torch.full((8,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # the multi-block grid first, then a one-block grid: the second call must not
    # see the first call's slots
    for call, shape in enumerate([(96, 96, 96), (40, 20, 18)]):
        # log_every large: olb_reductions then takes the stored-state path
        sim = olb.Sim(shape, 0.05, "D3Q27", 2, 0.7, 0.01, interp_order=4, storage=storage, log_every=1000)
        rho, u, _ = inputs.random_fields(tuple(reversed(shape)), 3, seed=21 + call, u_amp=0.1)
        sim.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        sim.step(2 + call)
        state = torch.empty(sim.state_bytes(), dtype=torch.uint8, device="cuda")
        sim.get_state(state)
        g = _grid(olb, shape)
        rc = L.olb_state_sums_noalloc(olb.VELOCITY_SETS["D3Q27"], ctypes.byref(g), olb.STORAGES[storage], 1.0, 1.0,
                                      ctypes.c_void_p(state.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(stream))
        assert rc == 0, L.olb_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = sim.reductions()
        assert _close(got[0], ref["k"]), (call, got[0], ref["k"])
        assert _close(got[1], ref["k_rho"])
        assert np.isnan(got[2]) and np.isnan(ref["eps"])
        assert _close(got[3], ref["mass"])
        for c in range(3):
            assert abs(got[4 + c] - ref["momentum"][c]) <= 1e-12 * ref["mass"]
        assert got[7] == 0.0 and ref["nonfinite"] == 0
        nodes = int(np.prod(shape))
        k_o, mass_o = _oracle_k_mass(_stored_values(state, storage, 27, nodes), storage, shape)
        assert _close(got[0], k_o), (call, got[0], k_o)
        assert abs(got[3] - mass_o) <= 1e-12 * mass_o
        sim.close()


def test_noalloc_rejects_oversized_grid():
    from paper_2101_03982_gb300 import olb
    L = olb.lib()
    g = _grid(olb, (1024, 1024, 1024))
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = L.olb_state_sums_noalloc(olb.VELOCITY_SETS["D3Q27"], ctypes.byref(g), olb.STORAGES["fp32"], 1.0, 1.0,
                                  ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == -6
    assert b"fixed scratch" in L.olb_last_error()

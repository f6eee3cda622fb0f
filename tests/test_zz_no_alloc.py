"""The allocation-free state sums agree with olb_reductions.

olb_state_sums_noalloc serves callers that cannot allocate device memory when
they need the global sums (their framework owns all device memory, or their
loop must not stall on cudaMalloc).  It keeps its partial sums in a fixed
array inside the library.  Two calls in a row, on two different states, must
each match the handle-based olb_reductions (its stored-state path, which uses
the same FP64 arithmetic) within 1e-12 relative, so a call never sees what
the previous call left in the shared array.

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


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
def test_noalloc_sums_match_reductions(storage):
    from paper_2101_03982_gb300 import inputs, olb
    L = olb.lib()
    shape = (40, 20, 18)
    # log_every large: olb_reductions then takes the stored-state path
    sim = olb.Sim(shape, 0.05, "D3Q27", 2, 0.7, 0.01, interp_order=4, storage=storage, log_every=1000)
    rho, u, _ = inputs.random_fields(tuple(reversed(shape)), 3, seed=21, u_amp=0.1)
    sim.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    g = _grid(olb, shape)
    state = torch.empty(sim.state_bytes(), dtype=torch.uint8, device="cuda")
    out = torch.full((8,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        if call == 1:
            sim.step(3)  # a different state for the second call
        sim.get_state(state)
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

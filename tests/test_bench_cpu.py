"""Host logic of bench.py that needs no GPU: the algorithmic flop count behind
the FP64 roofline, the whole-job throughput, the oracle sample calibration and
the workload names.
"""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_algorithmic_flops_by_hand():
    # D3Q27, p = 4, N = 2: 54 nonzero components -> pull 2*5*54 = 540; moments
    # 27*(1 + 2*3) = 189; per node 2 + 4*3 = 14; per velocity 27*(2*3 + 2*2 + 2 + 3) = 405
    assert bench.algorithmic_flops(dict(velocity_set="D3Q27", p=4, N=2)) == 540 + 189 + 14 + 405
    # D2Q9, p = 3, N = 2: 12 nonzero components -> 2*4*12 = 96; 9*5 = 45; 2 + 8 = 10; 9*(4 + 4 + 2 + 3) = 117
    assert bench.algorithmic_flops(dict(velocity_set="D2Q9", p=3, N=2)) == 96 + 45 + 10 + 117
    # compressible D2Q19, p = 4, N = 4: g doubles the pull; +3 per velocity in the moments, +10 per node and
    # +12 per velocity in the collision
    w = dict(velocity_set="D2Q19", p=4, N=4, compressible=True)
    iso = bench.algorithmic_flops(dict(w, compressible=False))
    assert bench.algorithmic_flops(w) - iso == (iso_pull(w) + 19 * 3 + 10 + 19 * 12)


def iso_pull(w):
    import numpy as np
    from paper_2101_03982_gb300 import olb
    xi, _ = olb.velocity_set_table(w["velocity_set"])
    return 2 * (w["p"] + 1) * int((np.abs(xi) > 0).sum())


def test_whole_job_throughput_counts_every_rank():
    assert bench.whole_job_mlups(1_000_000, 2, 0.01) == pytest.approx(200.0)
    assert bench.whole_job_mlups(2_097_152, 1, 0.0002) == pytest.approx(10485.76)


def test_calibration_fits_the_time_budget(monkeypatch):
    # a fake oracle costing 0.5 s fixed plus 1 ms per node: 16 s fit 15,500 nodes
    monkeypatch.setattr(bench, "oracle_time", lambda prm, f, npts, seed: 0.5 + 1e-3 * npts)
    assert bench.calibrate(None, None, 16.0) == 15500


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_workload_names_state_the_grid(name):
    w = bench.WORKLOADS[name]
    text = bench.workload_name(w)
    assert w["velocity_set"] in text
    if "n" in w:
        dim = 2 if w["velocity_set"].startswith("D2") else 3
        assert f"{w['n']}^{dim}" in text
    else:
        assert f"{w['shape'][0]}x{w['shape'][1]}" in text


@pytest.mark.parametrize("name", ["d3q45-comp", "d2q19-comp", "d2q25-comp"])
def test_compressible_workloads_use_the_papers_prandtl_number(name):
    # Secs. 4.1 and 4.3 run the compressible cases at Pr = 0.75
    w = bench.WORKLOADS[name]
    assert w["prandtl"] == 0.75
    assert "Pr 0.75" in bench.workload_name(w)

#!/usr/bin/env python
"""Throughput of the fused semi-Lagrangian LB step on GB300 (one JSON line).

Default workload (N = 1): 3D Taylor-Green vortex, Re = 1600, Ma = 0.1, 128^3
periodic nodes, D3Q27, N = 2 Hermite equilibrium, p = 4 Lagrange pull,
Courant 0.4, FP32 shifted storage.  One step = one launch of the fused
two-phase kernel over every node.  The L2 cache is flushed (a 256 MiB write) between timed
steps, and each step is timed alone with CUDA events on the simulation's
stream.  Under torchrun (N > 1) every rank runs its own replica of the
workload (weak scaling, no data-path collective); rank 0 reports the whole-job
node updates per second over the slowest rank.

`--impl reference` times the FP64 CPU oracle on bounded samples of the same
workload (host cores only); it is the deliberately slow correctness
reference, not a tuned CPU solver.
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import math  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import threading  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS (million node updates per second of the semi-Lagrangian LB step)"
WORKLOAD = dict(velocity_set="D3Q27", n=128, Re=1600.0, Ma=0.1, courant=0.4, N=2, p=4, storage="fp32",
                log_every=10)
# other single-GPU workloads of the paper's configurations, for profiling (256^3 runs fit as well)
WORKLOADS = {
    "d3q27": WORKLOAD,
    "d3q45": dict(WORKLOAD, velocity_set="D3Q45"),
    # compressible runs: Pr = 0.75 as in Secs. 4.1 and 4.3 (heat-flux quasi-equilibrium)
    "d3q45-comp": dict(WORKLOAD, velocity_set="D3Q45", N=4, compressible=True, Ma=1.0, prandtl=0.75),
    "d3q27-fp64": dict(WORKLOAD, storage="fp64"),
    "d2q19-comp": dict(velocity_set="D2Q19", shape=(1024, 512), N=4, p=4, storage="fp32", compressible=True,
                       Ma=1.2, Re=800.0, courant=0.4, prandtl=0.75),
    "d2q25-comp": dict(velocity_set="D2Q25", shape=(1024, 512), N=4, p=4, storage="fp32", compressible=True,
                       Ma=1.2, Re=800.0, courant=0.4, prandtl=0.75),
    "d3q13": dict(WORKLOAD, velocity_set="D3Q13"),
    "d3q21": dict(WORKLOAD, velocity_set="D3Q21"),
    "d3v27": dict(WORKLOAD, velocity_set="D3V27"),
    "d3q27-bf16": dict(WORKLOAD, storage="bf16"),
    "d3q27-fp16": dict(WORKLOAD, storage="fp16"),
    "d2q9-fp64": dict(velocity_set="D2Q9", n=64, N=2, p=3, storage="fp64", courant=0.4, Re=100.0, Ma=0.0866),
    "d3q27-glc": dict(WORKLOAD, interp="glc"),
}
FALLBACK_HBM_GBS = 6800.0
# DRAM traffic (read + write bytes per launch) of the step kernel for the
# default workload, from one ncu capture of the kernel source with this hash
# (summary in profiles/); reported as null once the kernel source changes.
TRAFFIC = {"kernel_sha": "ff4b475166f180ea", "bytes": 292462592 + 292550144}


def workload_name(w):
    if "shape" in w:  # the 2D shock-vortex field
        return (f"2D shock-vortex interaction (Mach {w['Ma']:g} standing shock, isentropic vortex), {w['shape'][0]}x"
                f"{w['shape'][1]}, inflow/outflow in x, periodic in y, {w['velocity_set']}, N={w['N']} Hermite "
                f"equilibrium, f+g, gamma 1.4, Pr {w.get('prandtl', 1.0):g}, "
                f"p={w['p']} Lagrange pull, Courant {w['courant']}, {w['storage'].upper()} shifted storage")
    if w["velocity_set"].startswith("D2"):  # the 2D Taylor-Green vortex
        return (f"2D Taylor-Green vortex Re={w['Re']:g}, {w['n']}^2 periodic, {w['velocity_set']} (c_s^2 = 1/3), "
                f"N={w['N']} Hermite equilibrium, p={w['p']} Lagrange pull, Courant {w['courant']}, "
                f"{w['storage'].upper()} storage")
    kind = f"compressible (f+g, gamma 1.4, Pr {w.get('prandtl', 1.0):g}) " if w.get("compressible") else ""
    return (f"{kind}3D Taylor-Green vortex Re={w['Re']:g} Ma={w['Ma']:g}, {w['n']}^3 periodic, {w['velocity_set']}, "
            f"N={w['N']} Hermite equilibrium, p={w['p']} "
            f"{'cell-wise GLC' if w.get('interp') == 'glc' else 'Lagrange'} pull, Courant {w['courant']}, "
            f"{w['storage'].upper()} {'shifted ' if w['storage'] != 'fp64' else ''}storage, "
            f"k and dissipation every {w.get('log_every', 1)} steps")


def algorithmic_flops(w):
    """Arithmetic of one node update in the step's own formulation (an FMA
    counts two): the separable pull, 2 (p + 1) per active axis of every
    velocity (f, and g when compressible); the moments, 1 + 2D per velocity
    (+ 3 with g: |xi|^2 f and g); 2 + 4D per node (rho, 1/rho, u, u/c_s, q;
    + 10 for the temperature); per velocity the equilibrium (s = xi^.u^: 2D,
    Horner polynomial of degree N in s: 2N, weight and density: 2; + 8 for the
    temperature-dependent coefficients) and BGK (3; + 4 for g)."""
    from paper_2101_03982_gb300 import olb
    xi, _ = olb.velocity_set_table(w["velocity_set"])
    Q, D = xi.shape
    comp = bool(w.get("compressible"))
    nnz = int((np.abs(xi) > 0).sum())
    pull = 2 * (w["p"] + 1) * nnz * (2 if comp else 1)
    moments = Q * (1 + 2 * D + (3 if comp else 0))
    node = 2 + 4 * D + (10 if comp else 0)
    per_vel = Q * (2 * D + 2 * w["N"] + 2 + 3 + (12 if comp else 0))
    return pull + moments + node + per_vel


def kernel_sha():
    h = hashlib.sha256()
    for f in ("olb_step.cuh", "olb_wg.cuh", "olb_step_f32_3d.cu"):
        h.update(open(os.path.join(ROOT, "paper_2101_03982_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json: STREAM-style copy)"
    return FALLBACK_HBM_GBS, "fallback (6.8 TB/s, earlier GB300 measurement)"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 3 + k and r[3 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# GPU measurements
# ---------------------------------------------------------------------------
def make_sim(w, torch):
    from paper_2101_03982_gb300 import inputs, olb, params
    if w.get("compressible"):
        if w["velocity_set"].startswith("D2"):
            rp = None
            nx, ny = w["shape"]
            _, _, cs, mx, _ = olb.velocity_set_info(w["velocity_set"])
            dt = w["courant"] * 1.0 / mx
            mu = math.sqrt(1.4) * w["Ma"] * (0.075 * ny) / w["Re"]
            sim = olb.Sim((nx, ny), 1.0, w["velocity_set"], w["N"], 1.0, dt, interp_order=w["p"],
                          storage=w["storage"], compressible=True, gamma=1.4, mu=mu,
                          log_every=w.get("log_every", 10), prandtl=w.get("prandtl", 1.0))
            rho, u, th = inputs.shock_vortex(nx, ny, Ma_a=w["Ma"])
            sim.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(np.ascontiguousarray(u)).cuda(),
                            torch.from_numpy(th).cuda())
            # standing shock: the upstream state flows in at x = 0, zero-gradient outflow at x = nx - 1
            sim.set_x_boundary("inflow_outflow", 1.0, (w["Ma"] * math.sqrt(1.4), 0.0), 1.0)
            return sim, int(nx * ny)
        rp = params.tgv_compressible(w["velocity_set"], w["n"], w["Re"], w["Ma"], w["courant"])
        sim = olb.Sim((w["n"],) * 3, rp.dx, w["velocity_set"], w["N"], rp.tau, rp.dt, interp_order=w["p"],
                      storage=w["storage"], compressible=True, gamma=rp.gamma, mu=rp.mu,
                      log_every=w.get("log_every", 10), prandtl=w.get("prandtl", 1.0))
        rho, u, th = inputs.ctic3d(w["n"], rp.u0)
        sim.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda(), torch.from_numpy(th).cuda())
        return sim, w["n"] ** 3
    if w["velocity_set"] == "D2Q9":
        rp = params.tgv2d_lattice(w["n"])
        sim = olb.Sim((w["n"],) * 2, rp.dx, "D2Q9", w["N"], rp.tau, rp.dt, interp_order=w["p"],
                      storage=w["storage"], cs_scale=rp.cs_scale, log_every=w.get("log_every", 10))
        rho, u = inputs.tgv2d(w["n"], rp.u0, rp.cs ** 2)
        sim.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        return sim, w["n"] ** 2
    rp = params.tgv_isothermal(w["velocity_set"], w["n"], w["Re"], w["Ma"], w["courant"])
    sim = olb.Sim((w["n"],) * 3, rp.dx, w["velocity_set"], w["N"], rp.tau, rp.dt, interp_order=w["p"],
                  storage=w["storage"], cs_scale=rp.cs_scale, log_every=w.get("log_every", 10),
                  kernel=w.get("kernel", "auto"))
    rho, u = inputs.tgv3d(w["n"], rp.u0, rp.cs ** 2)
    sim.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    if w.get("interp") == "glc":  # the paper's cell-wise GLC pull (two launches per step)
        sim.set_interpolation("glc")
    return sim, w["n"] ** 3


def time_steps(sim, torch, steps, warmup, flush):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        sim.step(1)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s, e in ev:
        flush.zero_()
        s.record(stream)
        sim.step(1)
        e.record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) * 1e-3 for s, e in ev]


def per_set_table(torch, flush):
    """Secondary lines: other sets, precisions and the other configurations."""
    rows = []
    specs = []
    for vs in ("D3Q13", "D3Q21", "D3V27", "D3Q27"):
        for st in ("fp32", "bf16", "fp16", "fp64"):
            specs.append(dict(WORKLOAD, velocity_set=vs, storage=st))
    specs.append(dict(WORKLOAD, velocity_set="D3V27", N=3))
    specs.append(dict(WORKLOAD, kernel="generic"))
    specs.append(dict(WORKLOAD, interp="glc"))
    specs.append(dict(WORKLOAD, interp="glc", storage="fp64"))
    specs.append(dict(WORKLOAD, interp="glc", storage="bf16"))
    specs.append(dict(WORKLOAD, velocity_set="D3Q45", N=2))
    specs.append(dict(WORKLOAD, n=256))
    specs.append(dict(WORKLOAD, n=256, velocity_set="D3Q45", N=2))
    specs.append(dict(WORKLOADS["d3q45-comp"], n=256))
    for ma in (0.5, 1.5, 2.0):  # the other Mach numbers of the compressible Taylor-Green runs
        specs.append(dict(WORKLOADS["d3q45-comp"], n=256, Ma=ma))
    specs.append(dict(WORKLOADS["d3q45-comp"], n=256, prandtl=1.0))  # plain BGK, the cost of the Pr model
    specs.append(dict(WORKLOADS["d3q45-comp"], n=512))  # 99 GB of A/B
    specs.append(WORKLOADS["d2q19-comp"])
    specs.append(WORKLOADS["d2q25-comp"])
    specs.append(dict(velocity_set="D2Q9", n=64, N=2, p=3, storage="fp64", courant=0.4, Re=100.0, Ma=0.0866))
    hbm, _ = measured_peaks()
    from paper_2101_03982_gb300 import olb
    fp64_peak = olb.fp64_fma_peak(torch.cuda.current_stream().cuda_stream) / 1e12
    for w in specs:
        try:
            sim, nodes = make_sim(w, torch)
        except Exception as e:  # a configuration that does not fit or is not built
            rows.append(dict(config=w, error=str(e)))
            continue
        steps = 5 if w["storage"] == "fp64" else 10
        ts = time_steps(sim, torch, steps, 2, flush)
        t = statistics.mean(ts)
        s = sim.elem_bytes
        nbytes = 2 * sim.planes * s * nodes
        rows.append(dict(kernel=w.get("kernel", "auto"), interp=w.get("interp", "uniform"),
                         velocity_set=w["velocity_set"], grid=w.get("shape") or [w["n"]] * (2 if w["velocity_set"] == "D2Q9" else 3),
                         N=w["N"], p=w["p"], storage=w["storage"], compressible=bool(w.get("compressible")),
                         prandtl=w.get("prandtl", 1.0), Ma=w.get("Ma"),
                         mlups=round(nodes / t / 1e6, 1), ms_per_step=round(t * 1e3, 4),
                         gbs=round(nbytes / t / 1e9, 1), hbm_frac=round(nbytes / t / 1e9 / hbm, 4)))
        if w["storage"] == "fp64":  # bound by the FP64 pipe: % of the measured FP64 FMA peak first
            fl = algorithmic_flops(w) * nodes / t / 1e12
            rows[-1].update(fp64_tflops=round(fl, 4), fp64_peak_tflops=round(fp64_peak, 4),
                            fp64_alu_frac=round(fl / fp64_peak, 4), flops_per_node=algorithmic_flops(w))
        sim.close()
        del sim
        torch.cuda.empty_cache()
    return rows


def history_run(w, torch, steps, log):
    """k and the dissipation estimate every `log` steps of one run of workload w."""
    sim, _ = make_sim(dict(w, log_every=log), torch)
    ks, es = [], []
    for _ in range(steps // log):
        sim.step(log)
        k, e = sim.kinetic_energy()
        ks.append(k)
        es.append(e)
    sim.close()
    return np.array(ks), np.array(es)


def precision_table(torch, steps):
    """The weakly compressible Taylor-Green runs (Sec. 4.2) at 128^3 for
    `steps` steps with k and the dissipation estimate every 10 steps, per set,
    in every storage: the largest relative deviation of each history from the
    FP64 storage run (whose step matches the FP64 oracle to 1e-12 per step)."""
    rows = []
    for vs in ("D3Q27", "D3Q13", "D3Q21", "D3V27"):
        w = dict(WORKLOAD, velocity_set=vs)
        t0 = time.perf_counter()
        k64, e64 = history_run(dict(w, storage="fp64"), torch, steps, 10)
        t64 = time.perf_counter() - t0
        for st in ("fp32", "bf16", "fp16"):
            k, e = history_run(dict(w, storage=st), torch, steps, 10)
            rows.append(dict(velocity_set=vs, storage=st, grid=[w["n"]] * 3, steps=steps, log_every=10,
                             k_err_vs_fp64=float((np.abs(k - k64) / np.abs(k64)).max()),
                             eps_err_vs_fp64=float((np.abs(e - e64) / np.abs(e64)).max()),
                             k_final=float(k[-1]), k_final_fp64=float(k64[-1])))
        rows.append(dict(velocity_set=vs, storage="fp64", grid=[w["n"]] * 3, steps=steps, log_every=10,
                         k_final=float(k64[-1]), seconds=round(t64, 2)))
        torch.cuda.empty_cache()
    return rows


def precision_comp_table(torch, n, steps):
    """The compressible Taylor-Green run (Sec. 4.3: D3Q45, N = 4, Ma 1.0,
    Pr 0.75) at n^3 for `steps` steps with k logged every 10 steps, FP32
    shifted storage against FP64 storage: the largest relative deviation of
    the k history."""
    w = dict(WORKLOADS["d3q45-comp"], n=n)
    t0 = time.perf_counter()
    k64, e64 = history_run(dict(w, storage="fp64"), torch, steps, 10)
    t64 = time.perf_counter() - t0
    k32, e32 = history_run(dict(w, storage="fp32"), torch, steps, 10)
    torch.cuda.empty_cache()
    rel = np.abs(k32 - k64) / np.abs(k64)
    # the deviation at a few points of the run: exponential growth from the
    # rounding level is the divergence of two trajectories of a chaotic flow,
    # growth from the start a drift of the FP32 step
    marks = sorted({max(1, len(rel) * q // 10) for q in (1, 2, 4, 6, 8, 10)})
    return [dict(velocity_set="D3Q45", compressible=True, Ma=w["Ma"], prandtl=w["prandtl"], storage="fp32",
                 grid=[n] * 3, steps=steps, log_every=10,
                 k_err_at_step={str(10 * m): float(rel[:m].max()) for m in marks},
                 k_err_vs_fp64=float(rel.max()),
                 eps_err_vs_fp64=float((np.abs(e32 - e64) / np.abs(e64)).max()),
                 k_final=float(k32[-1]), k_final_fp64=float(k64[-1]), k0_fp64=float(k64[0]),
                 fp64_seconds=round(t64, 1))]


def precision_shock_table(torch, steps):
    """The shock-vortex interaction (Sec. 4.1: D2Q19 and D2Q25, N = 4, Mach 1.2
    standing shock, inflow/outflow x, Pr 0.75) at 1024 x 512 for `steps`
    steps with k logged every 10 steps, FP32 shifted storage against FP64
    storage: the largest relative deviation of the k history."""
    rows = []
    for name in ("d2q19-comp", "d2q25-comp"):
        w = WORKLOADS[name]
        k64, e64 = history_run(dict(w, storage="fp64"), torch, steps, 10)
        k32, e32 = history_run(dict(w, storage="fp32"), torch, steps, 10)
        rel = np.abs(k32 - k64) / np.abs(k64)
        rows.append(dict(velocity_set=w["velocity_set"], compressible=True, Ma=w["Ma"], prandtl=w["prandtl"],
                         storage="fp32", grid=list(w["shape"]), steps=steps, log_every=10,
                         k_err_vs_fp64=float(rel.max()),
                         eps_err_vs_fp64=float((np.abs(e32 - e64) / np.abs(e64)).max()),
                         k_final=float(k32[-1]), k_final_fp64=float(k64[-1])))
        torch.cuda.empty_cache()
    return rows


def adjoint_table(torch, configs=((64, "fp32"), (64, "fp64"), (128, "fp32"))):
    """Adjoint of the isothermal step against the forward step (CUDA events).

    D3Q27, N = 2, p = 3, Re = 400, Ma = 0.1 (the adjoint workload) at 64^3
    (FP32, FP64) and 128^3 (FP32).  Per step: forward (olb_step), recording
    onto the device tape (olb_tape_record), and the adjoint sweep
    (olb_tape_adjoint over the recorded segment, scatter and gather of the
    adjoint included, amortised over the segment).  At 64^3 a state fits in
    L2, so both sides run partly from L2.
    """
    from paper_2101_03982_gb300 import inputs, olb, params
    rows = []
    for n, storage in configs:
        rp = params.tgv_isothermal("D3Q27", n, 400.0, 0.1, 0.4)
        sim = olb.Sim((n,) * 3, rp.dx, "D3Q27", 2, rp.tau, rp.dt, interp_order=3, storage=storage,
                      cs_scale=rp.cs_scale, log_every=1000000)
        rho, u = inputs.tgv3d(n, rp.u0, rp.cs ** 2)
        sim.init_fields(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        K = 25
        sim.tape_reserve(K)
        lam = torch.randn((sim.Q, n, n, n), dtype=getattr(torch, sim.adjoint_dtype), device="cuda")
        stream = torch.cuda.current_stream()

        def timed(fn, reps=3):
            fn()
            best = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize()
                best.append(a.elapsed_time(b) * 1e-3)
            return statistics.median(best)

        t_fwd = timed(lambda: sim.step(K)) / K
        t_rec = timed(lambda: sim.tape_record(K)) / K
        t_adj = timed(lambda: sim.tape_adjoint(lam, K)) / K
        rows.append(dict(grid=[n] * 3, velocity_set="D3Q27", N=2, p=3, storage=storage, segment=K,
                         forward_ms=round(t_fwd * 1e3, 4), record_ms=round(t_rec * 1e3, 4),
                         adjoint_ms=round(t_adj * 1e3, 4), adjoint_over_forward=round(t_adj / t_fwd, 3),
                         adjoint_plus_recompute_over_forward=round((t_adj + t_rec) / t_fwd, 3),
                         adjoint_mlups=round(n ** 3 / t_adj / 1e6, 1)))
        sim.close()
        del sim, lam
        torch.cuda.empty_cache()
    return rows


def diagnostics_timing(torch):
    """Enstrophy diagnostic (off the per-step path) on the default workload."""
    sim, nodes = make_sim(WORKLOAD, torch)
    sim.enstrophy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 5
    for _ in range(reps):
        e = sim.enstrophy()
    dt = (time.perf_counter() - t0) / reps
    sim.close()
    return dict(enstrophy_ms=round(dt * 1e3, 3), enstrophy=e, note="host-timed call incl. read-back")


def e2e_measure(w, torch, steps=8):
    """Through the C ABI with host buffers: upload the state from pinned host
    memory, one step, read back the kinetic energy (device -> host).  The
    handle sums k in the step itself (log_every = 1)."""
    sim, nodes = make_sim(dict(w, log_every=1), torch)
    nb = sim.state_bytes()
    host = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    sim.get_state(host.numpy())
    for _ in range(2):
        sim.set_state(host.numpy())
        sim.step(1)
        sim.kinetic_energy()
    t0 = time.perf_counter()
    for _ in range(steps):
        sim.set_state(host.numpy())
        sim.step(1)
        sim.kinetic_energy()
    dt = (time.perf_counter() - t0) / steps
    sim.close()
    return dict(value=round(nodes / dt / 1e6, 2), unit="MLUPS", h2d_bytes_per_step=int(nb),
                d2h_bytes_per_step=64, steps=steps)


# ---------------------------------------------------------------------------
# CPU oracle on bounded samples
# ---------------------------------------------------------------------------
def oracle_setup(w, build_state=True):
    from oracle import sllbm as O
    from oracle import velocity_sets as V
    from paper_2101_03982_gb300 import inputs
    vs0 = V.get(w["velocity_set"])
    cs = 1.0 / w["Ma"]
    vs = vs0.scaled(cs / vs0.cs)
    n = w["n"]
    dx = 2 * math.pi / n
    dt = w["courant"] * dx / np.abs(vs.xi).max()
    tau = O.tau_isothermal(1.0 / w["Re"], vs.cs, dt)
    prm = O.Params(vs, w["N"], w["p"], dt=dt, dx=dx, tau=tau)
    if not build_state:
        return prm, None
    rho, u = inputs.tgv3d(n, 1.0, vs.cs ** 2)
    f, _ = O.init_equilibrium(prm, rho, u)
    return prm, f


def oracle_time(prm, f, npts, seed):
    from oracle import sllbm as O
    rng = np.random.default_rng(seed)
    pts = rng.integers(0, f.shape[1], (npts, 3))
    t0 = time.perf_counter()
    O.step_at_points(prm, f, None, pts)
    return time.perf_counter() - t0


def _pool_init(w, shm_name, shape):
    """Worker of the all-cores oracle timing: the workload's parameters and a
    view of the parent's initial state in shared memory (no copy per worker)."""
    global _POOL_PRM, _POOL_F, _POOL_SHM
    from multiprocessing import shared_memory
    _POOL_SHM = shared_memory.SharedMemory(name=shm_name)
    _POOL_F = np.ndarray(shape, dtype=np.float64, buffer=_POOL_SHM.buf)
    _POOL_PRM, _ = oracle_setup(w, build_state=False)


def _pool_step(args):
    npts, seed = args
    from oracle import sllbm as O
    rng = np.random.default_rng(seed)
    pts = rng.integers(0, _POOL_F.shape[1], (npts, 3))
    O.step_at_points(_POOL_PRM, _POOL_F, None, pts)
    return npts


class OraclePool:
    """The oracle on every host core: one process per core (started with
    'spawn', so that no child inherits this process's CUDA context), each
    running step_at_points on its own random nodes of the same state."""

    def __init__(self, w, f):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        self.cores = os.cpu_count() or 1
        self.shm = shared_memory.SharedMemory(create=True, size=f.nbytes)
        np.ndarray(f.shape, dtype=np.float64, buffer=self.shm.buf)[...] = f
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_pool_init,
                                                 initargs=(w, self.shm.name, f.shape))
        # start-up outside the timing; every pool call has a time limit, so that a
        # worker that cannot start ends the run with an error instead of a hang
        self.pool.map_async(_pool_step, [(64, k) for k in range(self.cores)]).get(timeout=300)

    def time(self, npts_per_core, seed):
        t0 = time.perf_counter()
        work = [(npts_per_core, seed + k) for k in range(self.cores)]
        done = sum(self.pool.map_async(_pool_step, work).get(timeout=600))
        return done, time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()
        self.shm.close()
        self.shm.unlink()


def calibrate(prm, f, seconds):
    """Sample size whose oracle step takes about `seconds`: a fixed cost plus a
    per-node cost, fitted from two small timings."""
    t1 = oracle_time(prm, f, 512, 0)
    t2 = oracle_time(prm, f, 4096, 1)
    per_node = max((t2 - t1) / (4096 - 512), 1e-9)
    return max(256, int((seconds - max(t1 - 512 * per_node, 0.0)) / per_node))


def slowest_rank_time(t, dist, torch, device):
    """Mean step time of the slowest rank (every rank gets it); t itself on one rank."""
    if dist is None:
        return t
    tt = torch.tensor([t], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_mlups(nodes_per_rank, world, t):
    """Node updates per second of the whole job: every rank advances its own replica
    of nodes_per_rank nodes per step (weak scaling), timed by the slowest rank."""
    return world * nodes_per_rank / t / 1e6


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    if w.get("compressible"):
        print(json.dumps({"impl": "reference", "unavailable": "the timed oracle sample covers the isothermal "
                          "workloads only"}), flush=True)
        return
    prm, f = oracle_setup(w)
    budget = 150.0 / max(1, args.steps + args.warmup)
    per_core = min(200000, calibrate(prm, f, budget))
    pool = OraclePool(w, f)
    for k in range(args.warmup):
        pool.time(per_core, 100 + 64 * k)
    runs = [pool.time(per_core, 1000 + 64 * k) for k in range(args.steps)]
    pool.close()
    npts = runs[0][0]
    t = statistics.mean(dt for _, dt in runs)
    v = npts / t / 1e6
    sample = (f"{npts} random nodes of the {w['n']}^3 workload per step ({per_core} per core on {pool.cores} "
              f"processes; oracle step_at_points)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(w), "nodes_per_step": npts},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": pool.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-per-set", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--precision-steps", type=int, default=2000,
                    help="steps of the FP32/BF16/FP16-vs-FP64 history comparison (0: skip)")
    ap.add_argument("--precision-shock-steps", type=int, default=4000,
                    help="steps of the shock-vortex FP32-vs-FP64 k history (0: skip)")
    ap.add_argument("--precision-comp-steps", type=int, default=0,
                    help="steps of the compressible D3Q45 FP32-vs-FP64 k history (0: skip; minutes of FP64)")
    ap.add_argument("--precision-comp-n", type=int, default=128, help="grid of that comparison")
    ap.add_argument("--adjoint-only", default=None, metavar="N:STORAGE",
                    help="only time the adjoint (tape record and sweep) at N^3 with that storage, e.g. 128:fp32")
    ap.add_argument("--workload", default="d3q27", choices=sorted(WORKLOADS),
                    help="timed workload (the reported metric is quoted on the default)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    from paper_2101_03982_gb300 import olb
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.adjoint_only:
        n, storage = args.adjoint_only.split(":")
        print(json.dumps({"adjoint": adjoint_table(torch, ((int(n), storage),))}))
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    olb.lib()
    args.warmup = max(3, args.warmup)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    w = WORKLOADS[args.workload]
    sim, nodes = make_sim(w, torch)
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ts = time_steps(sim, torch, args.steps, 0, flush)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t = slowest_rank_time(statistics.mean(ts), dist, torch, "cuda")
    k, eps = sim.kinetic_energy()
    s = sim.elem_bytes
    bytes_per_launch = 2 * sim.planes * s * nodes
    hbm, peak_src = measured_peaks()
    achieved = bytes_per_launch / t / 1e9
    if w["storage"] == "fp64":  # the FP64 pipe bounds the FP64 step: measure its FMA peak on this GPU
        fp64_peak = olb.fp64_fma_peak(torch.cuda.current_stream().cuda_stream) / 1e12
        flops_per_launch = algorithmic_flops(w) * nodes
    sha = kernel_sha()
    traffic = TRAFFIC["bytes"] if TRAFFIC["kernel_sha"] == sha and args.workload == "d3q27" else None
    sim.close()
    del sim
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    e2e = e2e_measure(w, torch)
    per_set = [] if args.no_per_set else per_set_table(torch, flush)
    precision = [] if args.no_per_set or args.precision_steps <= 0 else precision_table(torch, args.precision_steps)
    if not args.no_per_set and args.precision_shock_steps > 0:
        precision += precision_shock_table(torch, args.precision_shock_steps)
    if args.precision_comp_steps > 0:
        precision += precision_comp_table(torch, args.precision_comp_n, args.precision_comp_steps)
    # the histories' deviations beside the throughput of the same set and storage
    for r in per_set:
        for q in precision:
            if (r.get("velocity_set"), r.get("storage"), r.get("compressible"), r.get("N"), r.get("grid")) == \
                    (q["velocity_set"], q["storage"], False, 2, q["grid"]) and "k_err_vs_fp64" in q:
                r["err_vs_fp64"] = {"k_history": q["k_err_vs_fp64"], "eps_history": q["eps_err_vs_fp64"],
                                    "steps": q["steps"]}
    adjoint = [] if args.no_per_set else adjoint_table(torch)
    diagnostics = None if args.no_per_set else diagnostics_timing(torch)
    cpu = None
    if not args.no_cpu and not w.get("compressible"):
        prm, f = oracle_setup(w)
        npts1 = min(400000, calibrate(prm, f, 8.0))
        tc1 = oracle_time(prm, f, npts1, 7)
        pool = OraclePool(w, f)
        npts, tc = pool.time(npts1, 11)
        pool.close()
        cpu = {"value": npts / tc / 1e6, "unit": "MLUPS", "cores": pool.cores, "kind": "oracle",
               "sample": f"{npts} random nodes of the {w['n']}^3 workload, one step ({npts1} per core on "
                         f"{pool.cores} processes, {tc:.1f} s; oracle step_at_points)",
               "value_1_core": npts1 / tc1 / 1e6,
               "sample_1_core": f"{npts1} random nodes on one thread, {tc1:.1f} s"}
    line = {
        "metric": METRIC, "value": whole_job_mlups(nodes, world, t), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w["storage"] != "fp64" else "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(w), "nodes": nodes, "velocity_set": w["velocity_set"],
                   "storage": w["storage"], "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "flushed (256 MiB write) between timed steps; each step timed alone"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "kernel": "sl_wg_kernel (two-phase fused pull + collide)"} if w["storage"] != "fp64" else
                    {"bound": "alu", "achieved": flops_per_launch / t / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": flops_per_launch / t / 1e12 / fp64_peak, "traffic": None,
                     "peak_source": "measured: FP64 FMA loop (olb_fp64_fma_peak) on this GPU",
                     "algorithmic_flops_per_launch": flops_per_launch,
                     "hbm": {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm},
                     "kernel": "sl_wg_kernel (two-phase fused pull + collide), FP64"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        # the 2D shock adds its x-boundary fill, the cell-wise GLC step its pull kernel
        "gpu_launches": args.steps * (2 if ("shape" in w or w.get("interp") == "glc") else 1),
        "clocks": clk.summary(),
        "k_final": k,
        "per_set": per_set,
        "precision": precision,
        "adjoint": adjoint,
        "diagnostics": diagnostics,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

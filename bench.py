"""Benchmark of the CFD-DEM coupling step on GB300.

One step = the whole hot path on one synthetic bed: particle location and
counting-sort binning, quadrature-centred void fraction, its smoothed L2
projection (CG), per-particle forces and the fluid source term.  Workload:
the Q2 32x32x128 mesh (0.1 x 0.1 x 0.4 m, 3x3x3 Gauss points, 1,085,825
nodes) with 100,000 spheres of d ~ U[2, 3] mm packed to a solid fraction of
~0.53 in the lower 40 % (synthetic, seeded).

The headline `value` is the mixed path (FP32 work, FP64 refinement of the
projection), in particle-coupling updates per second; the FP64 path is
reported beside it with the error of the mixed results against it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica of the step on its own
GPU (the step has no exchange between beds); value = all particles / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-coupling updates/s (eps+L2 proj+forces), mixed vs FP64 at stated err"
WORKLOAD = "q2_32x32x128_100k"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
FP32_TFLOPS = 73.13    # measured FMA peak on this GB300 (profiles/alu_peaks_gb300.md)
FP64_TFLOPS = 1.197
# DRAM bytes (read + write) of one launch of the FP32 QCM kernel on this
# workload, from one ncu capture (profiles/qcm_kernel_q2_32x32x128_100k.md):
# 3.62 MB read -- the sorted particle copies and the bin table -- and no
# write-back inside the launch (the 14 MB of eps stay in L2); to be cleared
# whenever that kernel changes
QCM_TRAFFIC_BYTES = 3623168 + 0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p)), "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    floor = 1e-3 * np.max(np.abs(b)) if b.size else 1.0
    den = np.maximum(np.abs(b), floor if floor > 0 else 1e-300)
    return float(np.max(np.abs(a - b) / den)) if b.size else 0.0


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def wait_first(self, timeout=3.0):
        """Block until nvidia-smi has written its first sample (so that the
        samples cover the timed region that follows)."""
        t0 = time.time()
        while self.p is not None and time.time() - t0 < timeout:
            self.f.flush()
            try:
                if os.path.getsize(self.f.name) > 0:
                    return
            except OSError:
                return
            time.sleep(0.02)

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(w, steps=None, budget_s=20.0):
    """The FP64 oracle as it stands on the host cores, timed on whole steps of
    the same workload until about budget_s seconds have been spent."""
    from oracle import oracle as O
    m = O.Mesh(w["origin"], w["extent"], w["n_el"], w["k"])
    prm = dict(w["params"], oracle_rtol=1e-13)
    n = w["x"].shape[0]
    times = []
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        O.coupling_step(m, prm, w["x"], w["r"], w["u_p"], w["u_nodal"], w["p_nodal"])
        times.append(time.perf_counter() - t0)
        if steps is not None and len(times) >= steps:
            break
        if steps is None and time.perf_counter() - t_all > budget_s:
            break
    per = float(np.mean(times))
    return {"value": n / per, "unit": "particle updates/s", "cores": O.num_threads(),
            "kind": "oracle", "sample": "%d whole coupling steps of %s (FP64, C + OpenMP)"
            % (len(times), WORKLOAD), "s_per_step": per}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2211_01185_gb300 import synth
    w = synth.make_workload(WORKLOAD)
    from oracle import oracle as O
    O.build()
    m = O.Mesh(w["origin"], w["extent"], w["n_el"], w["k"])
    prm = dict(w["params"], oracle_rtol=1e-13)
    for _ in range(args.warmup):
        O.coupling_step(m, prm, w["x"], w["r"], w["u_p"], w["u_nodal"], w["p_nodal"])
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.coupling_step(m, prm, w["x"], w["r"], w["u_p"], w["u_nodal"], w["p_nodal"])
        t.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(t))
    n = w["x"].shape[0]
    val = n / (ms * 1e-3)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "particle updates/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "mesh": "Q2 32x32x128", "particles": n,
                      "precision": "fp64", "parallelism": "host cores (OpenMP)"},
           "cpu_baseline": {"value": val, "unit": "particle updates/s",
                            "cores": O.num_threads(), "kind": "oracle",
                            "sample": "%d whole coupling steps of %s" % (args.steps, WORKLOAD)},
           "e2e": {"value": val, "unit": "particle updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def _max_over_ranks(x, dist, device):
    """The largest value of x over the ranks (x itself without a process
    group): a replica run is timed by its slowest rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(n_per_rank, world, ms):
    """Whole-job throughput: every rank advances its own replica of n
    particles in (at most) ms milliseconds."""
    return world * n_per_rank / (ms * 1e-3)


def _step_bytes(n, n_nodes, E, Q, iters, ms, hbm_gbs):
    """Algorithmic HBM bytes of one mixed coupling step and their rate: per
    particle x, r, u_p read, element/bin/slot and the sorted copies written
    and read back, forces and drag forces written (~180 B); the void fraction
    at the Gauss points written and read once (4 B each in FP32); the nodal
    right-hand side, velocity (24 B), void fraction and pressure read or
    written once (~48 B per node); per CG iteration about ten passes over
    double-float nodal vectors (8 B each: 80 B per node)."""
    b = 180.0 * n + 8.0 * E * Q + 48.0 * n_nodes + 80.0 * max(iters, 1) * n_nodes
    gbs = b / (ms * 1e-3) / 1e9
    return {"bytes": b, "achieved_gbs": gbs, "peak_gbs": hbm_gbs, "frac": gbs / hbm_gbs}


def _element_candidates(w):
    """(element, particle) pairs whose particle centre lies within R + r of the
    box spanned by the element's Gauss points: the candidates of element-level
    culling; times the Gauss points per element, the (point, particle) tests
    the QCM has to make."""
    x = np.asarray(w["x"])
    r = np.asarray(w["r"])
    o = np.asarray(w["origin"], dtype=np.float64)
    ne = np.asarray(w["n_el"])
    h = np.asarray(w["extent"], dtype=np.float64) / ne
    R = w["params"].get("qcm_radius", 0.0) or (3.0 * np.prod(h) / (4.0 * np.pi)) ** (1.0 / 3.0)
    cut = R + r
    m = int(np.ceil((R + r.max()) / h.min()))
    g = np.polynomial.legendre.leggauss(w["k"] + 1)[0]
    half = h * (0.5 * (g.max() + 1.0) - 0.5)   # Gauss box half extent
    base = np.clip(np.floor((x - o) / h).astype(np.int64), 0, ne - 1)
    total = 0
    rng = range(-m, m + 1)
    for dz in rng:
        for dy in rng:
            for dx in rng:
                e = base + np.array([dx, dy, dz])
                ok = np.all((e >= 0) & (e < ne), axis=1)
                c = o + (e + 0.5) * h
                gap = np.maximum(np.abs(x - c) - half, 0.0)
                total += int(np.count_nonzero(ok & (np.sum(gap * gap, axis=1) < cut * cut)))
    return float(total)


def run_batch(args):
    """The ensemble of 64 independent beds (Q1-Q3, 8-32 elements per axis, z up
    to 64, N log-uniform in [5e3, 2e5]): one cfdem_batch_coupling_step per step
    (one CUDA-graph replay after the first), against the same 64 beds stepped
    one after another through cfdem_coupling_step on one stream."""
    import torch
    from paper_2211_01185_gb300 import build as B
    from paper_2211_01185_gb300 import cfdem as cf
    from paper_2211_01185_gb300 import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    beds = synth.make_batch_workload(64)
    prec = 0 if args.precision == "fp64" else 1
    for b in beds:
        b["params"] = dict(b["params"], precision=prec, cg_rtol=1e-13 if prec == 0 else 1e-12,
                           max_radius=float(b["r"].max()))
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64).to(dev).contiguous()  # noqa: E731
    bufs = []
    with torch.cuda.stream(stream):
        for b in beds:
            n = b["x"].shape[0]
            ne = int(np.prod(b["n_el"]))
            nn = b["u_nodal"].shape[0]
            bufs.append(dict(n=n, x=t(b["x"]), r=t(b["r"]), u_p=t(b["u_p"]), u=t(b["u_nodal"]),
                             p=t(b["p_nodal"]),
                             eps=torch.zeros(nn, dtype=torch.float64, device=dev),
                             f=torch.empty((n, 3), dtype=torch.float64, device=dev),
                             fd=torch.empty((n, 3), dtype=torch.float64, device=dev),
                             Fe=torch.empty((ne, 3), dtype=torch.float64, device=dev)))
    n_tot = sum(bb["n"] for bb in bufs)
    ios = [cf.bed_io(bb["n"], bb["x"], bb["r"], bb["u_p"], bb["u"], bb["p"], bb["eps"], bb["f"],
                     bb["fd"], bb["Fe"]) for bb in bufs]
    bh = cf.cfdem_batch_create(len(beds), local, stream.cuda_stream)
    for i, b in enumerate(beds):
        h = cf.cfdem_batch_bed(bh, i)
        cf.cfdem_set_mesh(h, b["origin"], b["extent"], b["n_el"], b["k"])
        cf.cfdem_set_params(h, cf.make_params(**b["params"]))
    solo = [cf.Context(b["origin"], b["extent"], b["n_el"], b["k"], b["params"], device=local,
                       stream=stream.cuda_stream) for b in beds]

    def zero_eps():
        for bb in bufs:
            bb["eps"].zero_()   # cold start of every projection

    def step_batch():
        zero_eps()
        st = cf.cfdem_batch_coupling_step(bh, ios)
        if st != cf.OK:
            raise RuntimeError("batch step failed: %d" % st)

    def step_solo():
        zero_eps()
        for c, bb in zip(solo, bufs):
            cf.cfdem_coupling_step(c.h, bb["n"], bb["x"], bb["r"], bb["u_p"], bb["u"], bb["p"],
                                   bb["eps"], bb["f"], bb["fd"], bb["Fe"])

    def timed(fn, k):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize(dev)
            clk = Clocks(local)
            clk.wait_first()
            ev = []
            for _ in range(k):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                e.record(stream)
                ev.append((a, e))
            torch.cuda.synchronize(dev)
            clocks = clk.stop()
        return float(np.mean([a.elapsed_time(e) for a, e in ev])), clocks

    ms_b, clk_b = timed(step_batch, args.steps)
    st, bad = cf.cfdem_batch_synchronize(bh)
    replayed = cf.cfdem_batch_last_replayed(bh)
    its = [cf.cfdem_get_stats(cf.cfdem_batch_bed(bh, i)).cg_iterations for i in range(len(beds))]
    ms_s, clk_s = timed(step_solo, max(3, args.steps // 4))
    for c in solo:
        cf.cfdem_synchronize(c.h)
    res = {"metric": METRIC, "value": n_tot / (ms_b * 1e-3), "unit": "particle updates/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64" if prec == 1 else "f64", "data": "synthetic",
           "config": {"workload": "batch64: 64 beds Q1-Q3, N log-uniform [5e3, 2e5]",
                      "beds": len(beds), "particles": n_tot,
                      "nodes": int(sum(b["u_nodal"].shape[0] for b in beds)),
                      "precision": "mixed" if prec == 1 else "fp64", "cold_start": True,
                      "l2": "256 MiB buffer written between timed steps",
                      "parallelism": "single GPU, beds as parallel graph branches"},
           "graph_replayed": replayed, "batch_status": st,
           "cg_iterations": {"min": min(its), "max": max(its)},
           "solo_sequential": {"value": n_tot / (ms_s * 1e-3), "ms_per_step": ms_s,
                               "speedup_of_batch": ms_s / ms_b},
           "clocks": clk_b, "clocks_solo": clk_s}
    print(json.dumps(res), flush=True)
    cf.cfdem_batch_destroy(bh)
    for c in solo:
        c.close()
    return 0


def run_adjoint(args):
    """The sensitivity workload (24x24x96 Q2, 200,000 spheres, annulus and jet):
    one step = the forward coupling step and the adjoint of J = sum_i e_z .
    f_D,i + ||eps_h||_M (dJ/dx and dJ/du), FP64 and mixed."""
    import torch
    from paper_2211_01185_gb300 import build as B
    from paper_2211_01185_gb300 import cfdem as cf
    from paper_2211_01185_gb300 import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    w = synth.make_adjoint_workload()
    n = w["x"].shape[0]
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64).to(dev).contiguous()  # noqa: E731
    out = {}
    with torch.cuda.stream(stream):
        x, r, up, un, pn = t(w["x"]), t(w["r"]), t(w["u_p"]), t(w["u_nodal"]), t(w["p_nodal"])
        nn = un.shape[0]
        E = int(np.prod(w["n_el"]))
        z = lambda *s: torch.zeros(s, dtype=torch.float64, device=dev)  # noqa: E731
        eps, f, fd, Fe = z(nn), z(n, 3), z(n, 3), z(E, 3)
        g_fd = z(n, 3)
        g_fd[:, 2] = 1.0
        Me, dJdx, dJdu = z(nn), z(n, 3), z(nn, 3)
    for prec in (0, 1):
        prm = dict(w["params"], precision=prec, cg_rtol=1e-13 if prec == 0 else 1e-12,
                   max_radius=float(w["r"].max()))
        ctx = cf.Context(w["origin"], w["extent"], w["n_el"], w["k"], prm, device=local,
                         stream=stream.cuda_stream)

        def step():
            eps.zero_()
            cf.cfdem_coupling_step(ctx.h, n, x, r, up, un, pn, eps, f, fd, Fe)
            cf.cfdem_mass_apply(ctx.h, eps, Me)
            g_eps = Me / torch.sqrt(torch.dot(eps, Me))
            cf.cfdem_adjoint(ctx.h, n, x, r, up, un, pn, eps, None, g_fd, g_eps, dJdx, dJdu)

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step()
            cf.cfdem_synchronize(ctx.h)
            torch.cuda.synchronize(dev)
            clk = Clocks(local)
            clk.wait_first()
            ev = []
            for _ in range(args.steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step()
                b.record(stream)
                ev.append((a, b))
            torch.cuda.synchronize(dev)
            clocks = clk.stop()
            cf.cfdem_synchronize(ctx.h)
            st = ctx.stats()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        out[prec] = {"ms_per_step": ms, "value": n / (ms * 1e-3), "adjoint_cg_iterations":
                     st.cg_iterations, "clocks": clocks,
                     "dJdx_norm": float(torch.linalg.norm(dJdx).item()),
                     "dJdu_norm": float(torch.linalg.norm(dJdu).item())}
        ctx.close()
    res = {"metric": "particle gradient evaluations/s (forward step + adjoint)",
           "value": out[1]["value"], "unit": "particle updates/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": out[1]["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": w["name"], "mesh": "Q2 24x24x96", "particles": n,
                      "nodes": int(nn), "loss": "sum_i e_z.f_D,i + ||eps_h||_M",
                      "l2": "256 MiB buffer written between timed steps"},
           "mixed": out[1], "fp64": out[0]}
    print(json.dumps(res), flush=True)
    return 0


def run_dem(args):
    """The particle side of the coupling on the bench bed (100,000 spheres,
    d ~ U[2,3] mm, packed with small overlaps in the lower 40 % of the
    0.1 x 0.1 x 0.4 m box): one step = one CFD step's worth of DEM, 10
    Velocity Verlet sub-steps of 5 us with the contact model of Table
    (viscoelastic), FP64, with the coupling step's forces held as f_fp; also
    timed: the coupled step (mixed coupling step replayed as a graph, then
    the 10 DEM sub-steps on its forces)."""
    import torch
    from paper_2211_01185_gb300 import build as B
    from paper_2211_01185_gb300 import cfdem as cf
    from paper_2211_01185_gb300 import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    w = synth.make_workload(WORKLOAD)
    n = w["x"].shape[0]
    nsub, dt = 10, 5e-6
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64).to(dev).contiguous()  # noqa: E731
    lo = np.asarray(w["origin"], dtype=np.float64)
    hi = lo + np.asarray(w["extent"], dtype=np.float64)
    dprm = dict(rho_p=2500.0, youngs=1e7, poisson=0.3, restitution=0.9, friction=0.3,
                rolling_friction=0.01, wall_youngs=1e7, wall_poisson=0.3,
                wall_restitution=0.9, wall_friction=0.3, wall_rolling_friction=0.01,
                g=(0.0, 0.0, -9.81), lo=tuple(lo), hi=tuple(hi),
                max_radius=float(w["r"].max()), capacity=24)
    with torch.cuda.stream(stream):
        x0, r, up, un, pn = t(w["x"]), t(w["r"]), t(w["u_p"]), t(w["u_nodal"]), t(w["p_nodal"])
        x, v, om = x0.clone(), up.clone(), torch.zeros_like(up)
        nn = un.shape[0]
        E = int(np.prod(w["n_el"]))
        eps = torch.zeros(nn, dtype=torch.float64, device=dev)
        f = torch.zeros((n, 3), dtype=torch.float64, device=dev)
        fd, Fe = torch.zeros_like(f), torch.zeros((E, 3), dtype=torch.float64, device=dev)
    prm = dict(w["params"], precision=1, max_radius=float(w["r"].max()), cg_rtol=1e-12)
    bh = cf.cfdem_batch_create(1, local, stream.cuda_stream)
    bed = cf.cfdem_batch_bed(bh, 0)
    cf.cfdem_set_mesh(bed, w["origin"], w["extent"], w["n_el"], w["k"])
    cf.cfdem_set_params(bed, cf.make_params(**prm))
    dem = cf.Dem(dprm, device=local, stream=stream.cuda_stream)

    def coupling():
        eps.zero_()
        io = cf.bed_io(n, x, r, v, un, pn, eps, f, fd, Fe)
        assert cf.cfdem_batch_coupling_step(bh, [io]) == cf.OK

    def timed(fn, k):
        ev = []
        clk = Clocks(local)
        clk.wait_first()
        for _ in range(k):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize(dev)
        return float(np.mean([a.elapsed_time(b) for a, b in ev])), clk.stop()

    with torch.cuda.stream(stream):
        coupling()                                  # forces of the packed bed
        cf.cfdem_batch_synchronize(bh)
        per = {}
        for prec in (0, 1):                          # FP64, then mixed (kept for the coupled run)
            dem.set_params(dict(dprm, precision=prec))
            dem.reset()
            x.copy_(x0)
            v.copy_(up)
            om.zero_()
            for _ in range(args.warmup):
                dem.step(x, v, om, r, f, dt, nsub)
            torch.cuda.synchronize(dev)
            ms_p, clk_p = timed(lambda: dem.step(x, v, om, r, f, dt, nsub), args.steps)
            per[prec] = {"ms_per_step": ms_p, "value": n * nsub / (ms_p * 1e-3),
                         "status": int(dem.synchronize()), "clocks": clk_p}
        ms_dem, clocks, st_dem = per[1]["ms_per_step"], per[1]["clocks"], per[1]["status"]

        def coupled():
            coupling()
            dem.step(x, v, om, r, f, dt, nsub)

        for _ in range(args.warmup):
            coupled()
        torch.cuda.synchronize(dev)
        ms_cpl, clocks_cpl = timed(coupled, args.steps)
        st_b = cf.cfdem_batch_synchronize(bh)
        st_dem2 = dem.synchronize()
        drift = float(torch.linalg.norm(x - x0, dim=1).max().item())
    dem.close()
    cf.cfdem_batch_destroy(bh)
    res = {"metric": "DEM particle sub-steps/s (visco-elastic contacts, Velocity Verlet)",
           "value": n * nsub / (ms_dem * 1e-3), "unit": "particle sub-steps/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_dem,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "dem_" + WORKLOAD, "particles": n, "substeps_per_step": nsub,
                      "dt_dem": dt, "contact_capacity": 24,
                      "l2": "256 MiB buffer written between timed steps"},
           "status": {"dem": int(st_dem), "dem_coupled": int(st_dem2), "batch": list(st_b)},
           "precision": "mixed (FP32 contact forces, FP64 state)", "fp64": per[0],
           "coupled_step": {"ms_per_step": ms_cpl, "value": n / (ms_cpl * 1e-3),
                            "unit": "particle CFD steps/s (coupling + 10 DEM sub-steps)",
                            "clocks": clocks_cpl},
           "max_displacement_m": drift, "clocks": clocks}
    print(json.dumps(res), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"],
                    help="paths to time (profiling runs use one)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "batch64", "adjoint5", "dem"],
                    help="batch64: the 64-bed ensemble, graph replay against 64 solo runs; "
                         "adjoint5: forward step + adjoint of J = sum e_z.f_D + ||eps_h||_M; "
                         "dem: 10 DEM sub-steps per step on the bench bed, and the coupled step")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "adjoint5":
        return run_adjoint(args)
    if args.workload == "dem":
        return run_dem(args)

    import torch
    from paper_2211_01185_gb300 import build as B
    from paper_2211_01185_gb300 import cfdem as cf
    from paper_2211_01185_gb300 import synth

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()

    w = synth.make_workload(WORKLOAD)
    n = w["x"].shape[0]
    stream = torch.cuda.Stream(device=dev)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64).to(dev).contiguous()  # noqa: E731
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def make_ctx(precision):
        prm = dict(w["params"], precision=precision, max_radius=float(w["r"].max()),
                   cg_rtol=1e-13 if precision == 0 else 1e-12)
        return cf.Context(w["origin"], w["extent"], w["n_el"], w["k"], prm, device=local,
                          stream=stream.cuda_stream)

    with torch.cuda.stream(stream):
        x, r, up, un, pn = t(w["x"]), t(w["r"]), t(w["u_p"]), t(w["u_nodal"]), t(w["p_nodal"])
        nn = un.shape[0]
        ctxs = {0: make_ctx(0), 1: make_ctx(1)}
        st0 = ctxs[0].stats()
        E, Q, n_nodes = st0.n_elem, st0.n_qp // st0.n_elem, st0.n_nodes
        outs = {}
        for p in (0, 1):
            outs[p] = {"eps_h": torch.zeros(n_nodes, dtype=torch.float64, device=dev),
                       "f": torch.empty((n, 3), dtype=torch.float64, device=dev),
                       "fd": torch.empty((n, 3), dtype=torch.float64, device=dev),
                       "Fe": torch.empty((E, 3), dtype=torch.float64, device=dev)}

    def step(p):
        o = outs[p]
        o["eps_h"].zero_()   # cold start of the projection every step
        cf.cfdem_coupling_step(ctxs[p].h, n, x, r, up, un, pn, o["eps_h"], o["f"], o["fd"],
                               o["Fe"])

    def timed(p, k):
        ev = []
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step(p)
            cf.cfdem_synchronize(ctxs[p].h)
            cf.cfdem_set_timing(ctxs[p].h, 1)
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize(dev)
            clk = Clocks(local)
            clk.wait_first()
            for _ in range(k):
                flush.zero_()                     # evict L2 (256 MiB > 129 MB) between steps
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step(p)
                b.record(stream)
                ev.append((a, b))
            torch.cuda.synchronize(dev)
            clocks = clk.stop()
            st = ctxs[p].stats()
            cf.cfdem_synchronize(ctxs[p].h)
        ms = [a.elapsed_time(b) for a, b in ev]
        tot = _max_over_ranks(float(np.sum(ms)), dist, dev)
        return tot / k, st, clocks

    k64 = max(3, args.steps // 2)
    if args.precision in ("both", "fp64"):
        ms64, st64, clk64 = timed(0, k64)
    if args.precision == "fp64":
        print(json.dumps({"fp64_ms_per_step": ms64, "stages_ms": {
            nm: st64.stage_ms[i] / k64 for i, nm in enumerate(cf.STAGES)}}), flush=True)
        return 0
    ms_mx, st_mx, clk_mx = timed(1, args.steps)

    # the same mixed step replayed as one CUDA graph (a batch of this one bed:
    # device-driven CG loop, no host round trip inside the step)
    bh = cf.cfdem_batch_create(1, local, stream.cuda_stream)
    bed = cf.cfdem_batch_bed(bh, 0)
    cf.cfdem_set_mesh(bed, w["origin"], w["extent"], w["n_el"], w["k"])
    cf.cfdem_set_params(bed, cf.make_params(**dict(w["params"], precision=1,
                                                   max_radius=float(w["r"].max()),
                                                   cg_rtol=1e-12)))
    with torch.cuda.stream(stream):
        og = {"eps_h": torch.zeros(n_nodes, dtype=torch.float64, device=dev),
              "f": torch.empty((n, 3), dtype=torch.float64, device=dev),
              "fd": torch.empty((n, 3), dtype=torch.float64, device=dev),
              "Fe": torch.empty((E, 3), dtype=torch.float64, device=dev)}
    gio = [cf.bed_io(n, x, r, up, un, pn, og["eps_h"], og["f"], og["fd"], og["Fe"])]

    def step_graph():
        og["eps_h"].zero_()
        if cf.cfdem_batch_coupling_step(bh, gio) != cf.OK:
            raise RuntimeError(cf.cfdem_batch_last_error(bh))

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step_graph()
        torch.cuda.synchronize(dev)
        clk = Clocks(local)
        clk.wait_first()
        evg = []
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step_graph()
            b.record(stream)
            evg.append((a, b))
        torch.cuda.synchronize(dev)
        clk_g = clk.stop()
    replayed = cf.cfdem_batch_last_replayed(bh)
    gst, _ = cf.cfdem_batch_synchronize(bh)
    st_g = cf.cfdem_get_stats(bed)
    ms_all_g = [a.elapsed_time(b) for a, b in evg]
    ms_g = _max_over_ranks(float(np.mean(ms_all_g)), dist, dev)
    ms_g_median = _max_over_ranks(float(np.median(ms_all_g)), dist, dev)
    if args.precision == "mixed":
        print(json.dumps({"mixed_ms_per_step": ms_mx, "stages_ms": {
            nm: st_mx.stage_ms[i] / args.steps for i, nm in enumerate(cf.STAGES)}}), flush=True)
        return 0

    # error of the mixed path against the FP64 path (same inputs)
    err = {"eps_h": rel_err(outs[1]["eps_h"].cpu().numpy(), outs[0]["eps_h"].cpu().numpy()),
           "f": rel_err(outs[1]["f"].cpu().numpy(), outs[0]["f"].cpu().numpy()),
           "f_drag": rel_err(outs[1]["fd"].cpu().numpy(), outs[0]["fd"].cpu().numpy()),
           "F_e": rel_err(outs[1]["Fe"].cpu().numpy(), outs[0]["Fe"].cpu().numpy())}
    err_graph = {"eps_h": rel_err(og["eps_h"].cpu().numpy(), outs[1]["eps_h"].cpu().numpy()),
                 "f": rel_err(og["f"].cpu().numpy(), outs[1]["f"].cpu().numpy())}

    # end to end through the C ABI with host buffers: the batch step uploads
    # the step's inputs from page-locked host memory (x and r first; u_p,
    # u_nodal and p_nodal on a second stream while the void fraction and the
    # projection run) and downloads the forces and the fluid source, all
    # inside its graph
    hx = {k: torch.as_tensor(w[k], dtype=torch.float64).pin_memory()
          for k in ("x", "r", "u_p", "u_nodal", "p_nodal")}
    hx["f"] = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    hx["F_elem"] = torch.empty((E, 3), dtype=torch.float64).pin_memory()
    h2d = sum(hx[k].numel() * 8 for k in ("x", "r", "u_p", "u_nodal", "p_nodal"))
    d2h = (hx["f"].numel() + hx["F_elem"].numel()) * 8
    hio = [cf.bed_io(n, x, r, up, un, pn, og["eps_h"], og["f"], og["fd"], og["Fe"], host=hx)]

    def step_host():
        og["eps_h"].zero_()
        if cf.cfdem_batch_coupling_step(bh, hio) != cf.OK:
            raise RuntimeError(cf.cfdem_batch_last_error(bh))

    ev = []
    e2e_steps = 0 if args.no_e2e else args.warmup + args.steps
    with torch.cuda.stream(stream):
        for i in range(e2e_steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step_host()
            b.record(stream)
            if i >= args.warmup:
                ev.append((a, b))
        torch.cuda.synchronize(dev)
    e2e_replayed = cf.cfdem_batch_last_replayed(bh)
    e2e_err = rel_err(hx["f"].numpy(), outs[1]["f"].cpu().numpy()) if e2e_steps else None
    e2e_ms = float(np.mean([a.elapsed_time(b) for a, b in ev])) if ev else float("nan")

    # roofline of the dominant kernel group of the mixed step
    peaks, peak_kind = _peaks()
    stages = {name: st_mx.stage_ms[i] / args.steps for i, name in enumerate(cf.STAGES)}
    calls = {name: st_mx.stage_calls[i] / args.steps for i, name in enumerate(cf.STAGES)}
    k = w["k"]
    # algorithmic work per unit:
    #   operator: 7 banded 1D applies x (2k+1) taps x 2 flops + 5 = flops per node
    #   QCM: per neighbour pair 8 flops (distance) + 20 flops (lens volume)
    op_flops_node = 7 * (2 * k + 1) * 2 + 5
    # the op32 stage holds the double-float residual and the CG operator
    # launches (the last chunk's are no-ops once the CG has converged): per
    # launch, the productive ones only
    it_mx = max(1, st_mx.cg_iterations)
    calls["op32"] = it_mx + 1
    stages_k = dict(stages)
    stages_k["op32"] = stages["op32"] * it_mx / (it_mx + 1)   # the operator launches alone
    candidates = {
        "op32": ("alu", op_flops_node * n_nodes, FP64_TFLOPS,
                 "k_cg_apply_df (double-float CG operator: 48-bit arithmetic on the FP32 "
                 "pipes, stated against the FP64 peak)"),
        "void_fraction": ("alu", None, FP32_TFLOPS, "k_qcm<2,false> (FP32 QCM)"),
        "forces": ("hbm", 180.0 * n, peaks.get("hbm_gbs", 6800.0) / 1e3, "k_forces<2,1,float>"),
    }
    # neighbour pairs of this bed for the QCM flop count (outside the timed region)
    with torch.cuda.stream(stream):
        cnt = torch.zeros(E * Q, dtype=torch.int32, device=dev)
        cf.cfdem_void_fraction(ctxs[0].h, n, x, r, None, cnt, None)
        cf.cfdem_synchronize(ctxs[0].h)
        pairs = float(cnt.sum().item())
    tested = float(w["k"] + 1) ** 3 * _element_candidates(w)
    candidates["void_fraction"] = ("alu", 8.0 * tested + 20.0 * pairs, FP32_TFLOPS,
                                   "k_qcm<2,false> (FP32 QCM)")
    dom = max(candidates, key=lambda s: stages_k[s])
    bound, work, peak, kname = candidates[dom]
    per_launch_ms = stages[dom] / max(calls[dom], 1.0)
    if bound == "alu":
        achieved = work / (per_launch_ms * 1e-3) / 1e12
        unit, peak_v = "TFLOP/s", peak
    else:
        achieved = work / (per_launch_ms * 1e-3) / 1e9
        unit, peak_v = "GB/s", peaks.get("hbm_gbs", 6800.0)
    traffic = QCM_TRAFFIC_BYTES if dom == "void_fraction" else None
    # what bounds the QCM kernel instead of its FMA rate (same ncu captures)
    limiter = ("instruction issue: 77 % of issue slots active (ncu smsp__issue_active); "
               "the per-element work is a filter of compares, ballots and queue appends, "
               "whose instructions are not counted as algorithmic flops"
               if dom == "void_fraction" else None)
    roof = {"bound": bound, "kernel": kname, "achieved": achieved, "peak": peak_v,
            "unit": unit, "frac": achieved / peak_v, "traffic": traffic,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "limiter": limiter,
            "peak_source": ("measured FMA loop (profiles/alu_peaks_gb300.md)" if bound == "alu"
                            else "%s MEASURED_PEAKS.json hbm_gbs" % peak_kind),
            "launches_per_step": calls[dom], "ms_per_launch": per_launch_ms,
            "others": {c: {"kernel": candidates[c][3], "ms_per_step": stages_k[c],
                           "frac": ((candidates[c][1] / (stages[c] / max(calls[c], 1.0) * 1e-3)
                                     / (1e12 if candidates[c][0] == "alu" else 1e9))
                                    / (candidates[c][2] if candidates[c][0] == "alu"
                                       else peaks.get("hbm_gbs", 6800.0)))}
                       for c in candidates if c != dom}}

    value = _job_value(n, world, ms_g)
    res = {"metric": METRIC, "value": value, "unit": "particle updates/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_g,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "mesh": "Q2 32x32x128, 3x3x3 Gauss",
                      "particles": n, "nodes": n_nodes, "precision": "mixed",
                      "l2": "256 MiB buffer written between timed steps",
                      "cg_rtol": 1e-12, "cold_start": True,
                      "launch": "one CUDA-graph replay per step (cfdem_batch_coupling_step)",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "ms_per_step_median": ms_g_median,
           "step_hbm": _step_bytes(n, n_nodes, E, Q, st_g.cg_iterations, ms_g,
                                   peaks.get("hbm_gbs", 6800.0)),
           "graph": {"replayed": replayed, "status": gst, "cg_iterations": st_g.cg_iterations,
                     "cg_relres": st_g.cg_relres, "err_vs_eager": err_graph},
           "eager": {"value": world * n / (ms_mx * 1e-3), "ms_per_step": ms_mx,
                     "launch": "cfdem_coupling_step, stage timers on", "clocks": clk_mx},
           "fp64": {"value": world * n / (ms64 * 1e-3), "ms_per_step": ms64, "dtype": "f64",
                    "cg_iterations": st64.cg_iterations,
                    "stages_ms": {nm: st64.stage_ms[i] / k64 for i, nm in enumerate(cf.STAGES)}},
           "err_mixed_vs_fp64": err,
           "stages_ms": stages,
           "cg": {"mixed_inner_iterations": st_mx.cg_iterations, "mixed_outer": st_mx.cg_outer,
                  "mixed_relres": st_mx.cg_relres, "fp64_iterations": st64.cg_iterations,
                  "fp64_relres": st64.cg_relres},
           "roofline": roof,
           "e2e": {"value": world * n / (e2e_ms * 1e-3), "unit": "particle updates/s",
                   "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "launch": "cfdem_batch_coupling_step with page-locked host buffers: the "
                             "uploads and downloads run inside the replayed graph",
                   "replayed": e2e_replayed, "err_f_vs_eager": e2e_err},
           "gpu_launches": int(st_mx.kernel_launches),
           "gpu_launches_note": "counted on the eager run of the same K steps; the graph "
                                "replays the same kernels less the no-op CG iterations",
           "clocks": clk_g}
    if rank == 0 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(w)
    if dist is not None:
        dist.barrier()
    if rank == 0:
        print(json.dumps(res), flush=True)
    cf.cfdem_batch_destroy(bh)
    for c in ctxs.values():
        c.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

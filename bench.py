"""Benchmark of the CFD-DEM coupling step on GB300.

One step = the whole hot path on one synthetic bed: particle location and
counting-sort binning, quadrature-centred void fraction, its smoothed L2
projection (CG), per-particle forces and the fluid source term.  Headline
workload: the Q2 32x32x128 mesh (0.1 x 0.1 x 0.4 m, 3x3x3 Gauss points,
1,085,825 nodes) with 100,000 spheres of d ~ U[2, 3] mm packed to a solid
fraction of ~0.53 in the lower 40 % (synthetic, seeded).

The headline `value` is the mixed path (FP32 work, FP64 refinement of the
projection) replayed as one CUDA graph per step, in particle-coupling updates
per second; the FP64 path is timed the same way beside it, with the error of
the mixed results against it.  The default run also reports, under
`workloads`, the Q1 8x8x32 bed of 2,000 spheres, the Q3 24x24x96 bed of
1,000,000 spheres, the 64-bed ensemble, the adjoint workload and the DEM
step (fewer timed steps each).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload NAME] [--quick]
Under torchrun each rank runs an independent replica of the step on its own
GPU (the step has no exchange between beds); value = all particles / max time.
"""
from __future__ import annotations

import argparse
import ctypes
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
SINGLE_BEDS = ("q1_8x8x32_2k", "q2_32x32x128_100k", "q3_24x24x96_1m")
MESH_NAMES = {"q1_8x8x32_2k": "Q1 8x8x32, 2x2x2 Gauss", "q2_32x32x128_100k":
              "Q2 32x32x128, 3x3x3 Gauss", "q3_24x24x96_1m": "Q3 24x24x96, 4x4x4 Gauss"}
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
# DRAM bytes (read + write) per launch of a kernel on the headline bed, from
# one ncu capture of that kernel as it is now (dram__bytes_read.sum +
# dram__bytes_write.sum); an entry is removed when its kernel changes
NCU_TRAFFIC = {
    "void_fraction": 3749632,    # k_qcm_pts<2>
    "op32": 8769408,             # k_cg_apply_df<2>: mean of the two productive launches
    "forces": 20133376,          # k_forces<2,1,float>
}
# algorithmic work per unit (the per-unit figures of the measurement plan):
#   QCM: 8 flops per tested (Gauss point, particle) pair, 25 per lens volume
#   operator: 7 banded 1D applies x (2k+1) taps x 2 flops + 5 per node
#   forces: FP64 flops per particle of the Q_k interpolations (u: 3 x 2 per
#   node, eps: 2 per node, grad p: 3 x 2 per pressure node), the 1D bases
#   (~10 per point and axis) and ~60 for the closure and the force sum
QCM_FLOPS_TEST, QCM_FLOPS_LENS = 8.0, 25.0
# the same work in FP32 instructions (the QCM issues FADD/FMUL/FFMA and
# compares at one rate): a test is three subtractions, a multiply, two FMAs
# and a compare; a lens volume about sixteen (one reciprocal square root,
# the lens formula) and four for the compensated sum
QCM_INSTR_TEST, QCM_INSTR_LENS = 7.0, 20.0


def _forces_bytes(w, n_nodes):
    """Algorithmic HBM bytes of one launch of the force kernel: per particle
    x, r, u_p read and f, f_drag, its source record and element written
    (140 B); the nodal velocity and void fraction (32 B per node) and the
    pressure (8 B per pressure node) of the elements that hold particles,
    read once."""
    x = np.asarray(w["x"])
    o = np.asarray(w["origin"], dtype=np.float64)
    ne = np.asarray(w["n_el"])
    h = np.asarray(w["extent"], dtype=np.float64) / ne
    k, kp = w["k"], w["params"]["pressure_degree"]
    c = np.clip(np.floor((x - o) / h).astype(np.int64), 0, ne - 1)
    held = np.unique(c[:, 0] + ne[0] * (c[:, 1] + ne[1] * c[:, 2])).size
    frac = held / float(np.prod(ne))
    n_p = float(np.prod(ne * kp + 1))
    return 140.0 * x.shape[0] + frac * (32.0 * n_nodes + 8.0 * n_p)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p)), "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


def alu_peaks():
    """FP32 and FP64 FMA throughput of this device (TFLOP/s), measured by the
    FMA probe library built beside the coupling library."""
    from paper_2211_01185_gb300 import build as B
    L = ctypes.CDLL(B.PROBE_LIB)
    L.alu_fma_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = {}
    for name, fp64 in (("fp32_tflops", 0), ("fp64_tflops", 1)):
        v = ctypes.c_double(0.0)
        rc = L.alu_fma_peak(fp64, ctypes.byref(v))
        if rc != 0:
            raise RuntimeError("FMA probe failed with CUDA error %d" % rc)
        out[name] = v.value
    return out


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


# ----------------------------------------------------------------- oracle

def cpu_baseline(w, name, steps=None, budget_s=20.0):
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
            % (len(times), name), "s_per_step": per}


def workload_config(name, w):
    """The bench line's `config`: the workload alone, the same dict on both
    arms (how each arm computes it goes under `run`)."""
    n_el, k = w["n_el"], w["k"]
    nodes = int(np.prod([int(e) * k + 1 for e in n_el]))
    return {"workload": name, "mesh": MESH_NAMES[name], "particles": int(w["x"].shape[0]),
            "nodes": nodes, "cold_start": True,
            "l2": "GPU arm: a 256 MiB buffer written between timed steps"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2211_01185_gb300 import synth
    name = args.workload if args.workload in SINGLE_BEDS else WORKLOAD
    w = synth.make_workload(name)
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
           "config": workload_config(name, w),
           "run": {"precision": "fp64", "parallelism": "host cores (OpenMP)",
                   "solve": "the oracle's coupling step (exact FDM solve of the projection)"},
           "cpu_baseline": {"value": val, "unit": "particle updates/s",
                            "cores": O.num_threads(), "kind": "oracle",
                            "sample": "%d whole coupling steps of %s" % (args.steps, name)},
           "e2e": {"value": val, "unit": "particle updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ----------------------------------------------------------------- helpers

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


def _qcm_radius(w):
    h = np.asarray(w["extent"], dtype=np.float64) / np.asarray(w["n_el"])
    return w["params"].get("qcm_radius", 0.0) or (3.0 * np.prod(h) / (4.0 * np.pi)) ** (1 / 3)


def _gauss_points(w):
    """Gauss point coordinates of every element, [E*Q][3] (sampling only)."""
    o = np.asarray(w["origin"], dtype=np.float64)
    ne = np.asarray(w["n_el"])
    h = np.asarray(w["extent"], dtype=np.float64) / ne
    g = 0.5 * (np.polynomial.legendre.leggauss(w["k"] + 1)[0] + 1.0)
    axes = [o[a] + h[a] * (np.arange(ne[a])[:, None] + g[None, :]).ravel() for a in range(3)]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def _qcm_cell_list_tests(w):
    """The (Gauss point, particle) tests of the textbook cell-list search of
    the QCM: cells of edge >= R + r_max, every particle of the 27 cells
    around the Gauss point's cell tested -- the unit count of the
    measurement plan's 8 flops per tested pair."""
    x = np.asarray(w["x"])
    o = np.asarray(w["origin"], dtype=np.float64)
    L = np.asarray(w["extent"], dtype=np.float64)
    cut = _qcm_radius(w) + float(np.max(w["r"]))
    nc = np.maximum(np.floor(L / cut).astype(np.int64), 1)
    ci = np.clip(np.floor((x - o) / (L / nc)).astype(np.int64), 0, nc - 1)
    cnt = np.zeros(nc[::-1], dtype=np.int64)
    np.add.at(cnt, (ci[:, 2], ci[:, 1], ci[:, 0]), 1)
    pad = np.pad(cnt, 1)
    box = sum(pad[1 + dz:1 + dz + nc[2], 1 + dy:1 + dy + nc[1], 1 + dx:1 + dx + nc[0]]
              for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    qp = _gauss_points(w)
    qi = np.clip(np.floor((qp - o) / (L / nc)).astype(np.int64), 0, nc - 1)
    return float(box[qi[:, 2], qi[:, 1], qi[:, 0]].sum())


def _element_candidates(w):
    """(element, particle) pairs whose particle centre lies within R + r of the
    box spanned by the element's Gauss points: the candidates of element-level
    culling; times the Gauss points per element, the (point, particle) tests
    the QCM kernel makes."""
    x = np.asarray(w["x"])
    r = np.asarray(w["r"])
    o = np.asarray(w["origin"], dtype=np.float64)
    ne = np.asarray(w["n_el"])
    h = np.asarray(w["extent"], dtype=np.float64) / ne
    R = _qcm_radius(w)
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


class Env:
    """Device, stream, L2 flush buffer and process group of this rank."""

    def __init__(self, use_dist=False):
        import torch
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if use_dist and self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
            self.dist = dist
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        from paper_2211_01185_gb300 import build as B
        B.build()
        self.stream = torch.cuda.Stream(device=self.dev)
        # written between timed steps: 256 MiB > the 129 MB L2
        self.flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=self.dev)

    def t(self, a):
        import torch
        return torch.as_tensor(a, dtype=torch.float64).to(self.dev).contiguous()

    def timed(self, fn, k, barrier=False):
        """k calls of fn on the stream, each bracketed by CUDA events and
        preceded by an L2 flush; returns the per-step ms list and clocks."""
        import torch
        with torch.cuda.stream(self.stream):
            if barrier and self.dist is not None:
                self.dist.barrier()
            torch.cuda.synchronize(self.dev)
            clk = Clocks(self.local)
            clk.wait_first()
            ev = []
            for _ in range(k):
                self.flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(self.stream)
                fn()
                b.record(self.stream)
                ev.append((a, b))
            torch.cuda.synchronize(self.dev)
            clocks = clk.stop()
        return [a.elapsed_time(b) for a, b in ev], clocks


# --------------------------------------------------------------- one bed

def run_bed(env, name, steps, warmup, alu, headline=False, e2e=True, cpu=True,
            cpu_steps=None):
    """One single-bed workload: FP64 and mixed, each replayed as one CUDA
    graph per step (timed) and run eagerly with stage timers (the stage
    breakdown); errors of the mixed results against the FP64 ones; the
    roofline of the dominant kernel of the mixed step; for the headline bed
    also the end-to-end step through host buffers."""
    import torch
    from paper_2211_01185_gb300 import cfdem as cf
    from paper_2211_01185_gb300 import synth
    w = synth.make_workload(name)
    n = w["x"].shape[0]
    peaks, peak_kind = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    s = env.stream
    with torch.cuda.stream(s):
        x, r, up, un, pn = (env.t(w[k]) for k in ("x", "r", "u_p", "u_nodal", "p_nodal"))

    def prm(p):
        return dict(w["params"], precision=p, max_radius=float(w["r"].max()),
                    cg_rtol=1e-13 if p == 0 else 1e-12)

    ctxs = {p: cf.Context(w["origin"], w["extent"], w["n_el"], w["k"], prm(p),
                          device=env.local, stream=s.cuda_stream) for p in (0, 1)}
    st0 = ctxs[0].stats()
    E, Q, n_nodes = st0.n_elem, st0.n_qp // st0.n_elem, st0.n_nodes

    def outputs():
        z = lambda *sh: torch.zeros(sh, dtype=torch.float64, device=env.dev)  # noqa: E731
        return {"eps_h": z(n_nodes), "f": z(n, 3), "fd": z(n, 3), "Fe": z(E, 3)}

    res = {"workload": name, "mesh": MESH_NAMES[name], "particles": n, "nodes": n_nodes,
           "elements": E, "gauss_points": E * Q}
    per = {}
    graph = {}
    for p in (0, 1):
        # graph: the step of this one bed captured once and replayed
        bh = cf.cfdem_batch_create(1, env.local, s.cuda_stream)
        bed = cf.cfdem_batch_bed(bh, 0)
        cf.cfdem_set_mesh(bed, w["origin"], w["extent"], w["n_el"], w["k"])
        cf.cfdem_set_params(bed, cf.make_params(**prm(p)))
        with torch.cuda.stream(s):
            og = outputs()
        gio = [cf.bed_io(n, x, r, up, un, pn, og["eps_h"], og["f"], og["fd"], og["Fe"])]

        def step_graph():
            og["eps_h"].zero_()   # cold start of the projection every step
            if cf.cfdem_batch_coupling_step(bh, gio) != cf.OK:
                raise RuntimeError(cf.cfdem_batch_last_error(bh))

        with torch.cuda.stream(s):
            for _ in range(warmup):
                step_graph()
        ms, clocks = env.timed(step_graph, steps, barrier=headline)
        gst, _ = cf.cfdem_batch_synchronize(bh)
        st_g = cf.cfdem_get_stats(bed)
        graph[p] = dict(bh=bh, bed=bed, out=og, io=gio, step=step_graph)
        per[p] = {"ms_per_step": float(np.mean(ms)), "ms_per_step_median": float(np.median(ms)),
                  "launch": "one CUDA-graph replay per step", "replayed":
                  cf.cfdem_batch_last_replayed(bh), "status": gst,
                  "cg_iterations": st_g.cg_iterations, "cg_outer": st_g.cg_outer,
                  "cg_relres": st_g.cg_relres, "clocks": clocks, "_ms": ms}
        per[p]["value"] = n / (per[p]["ms_per_step"] * 1e-3)
        # eager with stage timers: where the time goes
        o = outputs()
        c = ctxs[p]

        def step_eager():
            o["eps_h"].zero_()
            cf.cfdem_coupling_step(c.h, n, x, r, up, un, pn, o["eps_h"], o["f"], o["fd"],
                                   o["Fe"])

        with torch.cuda.stream(s):
            for _ in range(warmup):
                step_eager()
            cf.cfdem_synchronize(c.h)
            cf.cfdem_set_timing(c.h, 1)
        ke = max(3, min(steps, 50))
        ms_e, _ = env.timed(step_eager, ke)
        st = c.stats()
        cf.cfdem_synchronize(c.h)
        cf.cfdem_set_timing(c.h, 0)
        per[p]["eager"] = {"ms_per_step": float(np.mean(ms_e)), "steps": ke,
                           "launch": "cfdem_coupling_step, stage timers on",
                           "stages_ms": {nm: st.stage_ms[i] / ke for i, nm in
                                         enumerate(cf.STAGES)},
                           "stage_launches": {nm: st.stage_calls[i] / ke for i, nm in
                                              enumerate(cf.STAGES)},
                           "kernel_launches_per_step": st.kernel_launches / ke,
                           "cg_iterations": st.cg_iterations}
        per[p]["autotune"] = {"bin_edge_m": list(st.bin_edge), "bins": list(st.nb),
                              "tile_shape": ["16x8x8", "22x13x4", "25x15x4"][st.tile_shape],
                              "tuned": {"bins": bool(st.tuned & 1), "tile": bool(st.tuned & 2)},
                              "tune_ms": st.tune_ms,
                              "fdm_tile": "%dx%d" % divmod(st.fdm_tile, 10)}
        per[p]["err_graph_vs_eager"] = {
            "eps_h": rel_err(og["eps_h"].cpu().numpy(), o["eps_h"].cpu().numpy()),
            "f": rel_err(og["f"].cpu().numpy(), o["f"].cpu().numpy())}
        per[p]["dtype"] = "f64" if p == 0 else "f32+f64"
    res["fp64"] = {k: v for k, v in per[0].items() if not k.startswith("_")}
    res["fp64"]["note"] = ("the QCM's lens volumes, scan and sums run in double-float on the "
                           "FP32 pipes (~1e-13 relative); the rest is FP64")
    res["mixed"] = {k: v for k, v in per[1].items() if not k.startswith("_")}
    res["mixed_speedup_over_fp64"] = per[0]["ms_per_step"] / per[1]["ms_per_step"]
    o0, o1 = graph[0]["out"], graph[1]["out"]
    res["err_mixed_vs_fp64"] = {
        "eps_h": rel_err(o1["eps_h"].cpu().numpy(), o0["eps_h"].cpu().numpy()),
        "f": rel_err(o1["f"].cpu().numpy(), o0["f"].cpu().numpy()),
        "f_drag": rel_err(o1["fd"].cpu().numpy(), o0["fd"].cpu().numpy()),
        "F_e": rel_err(o1["Fe"].cpu().numpy(), o0["Fe"].cpu().numpy())}

    # ---- roofline of the dominant kernel of the mixed step
    stages = per[1]["eager"]["stages_ms"]
    calls = per[1]["eager"]["stage_launches"]
    k, kp = w["k"], w["params"]["pressure_degree"]
    with torch.cuda.stream(s):
        cnt = torch.zeros(E * Q, dtype=torch.int32, device=env.dev)
        cf.cfdem_void_fraction(ctxs[0].h, n, x, r, None, cnt, None)
        cf.cfdem_synchronize(ctxs[0].h)
        pairs = float(cnt.sum().item())
    tests_cell = _qcm_cell_list_tests(w)
    tests_culled = float(k + 1) ** 3 * _element_candidates(w)
    qcm_ms = stages["void_fraction"] / max(calls["void_fraction"], 1.0)
    fo_ms = stages["forces"] / max(calls["forces"], 1.0)
    # the operator's launches: one per CG iteration (the eager solve queues
    # iterations in chunks of two, so a launch after convergence, which
    # returns at once, is rare)
    op_launches = float(max(per[1]["eager"]["cg_iterations"], 1))
    op_ms = stages["op32"] / op_launches
    op_macs = 7.0 * (2 * k + 1) * n_nodes   # z: M, K; y: 3 folded bands; x: M, K
    instr_peak = alu["fp32_tflops"] / 2.0    # FP32 instructions per second / 1e12
    qcm_flops = QCM_FLOPS_TEST * tests_cell + QCM_FLOPS_LENS * pairs
    qcm_instr = QCM_INSTR_TEST * tests_cell + QCM_INSTR_LENS * pairs
    qcm_instr_culled = QCM_INSTR_TEST * tests_culled + QCM_INSTR_LENS * pairs
    qcm_flops_culled = QCM_FLOPS_TEST * tests_culled + QCM_FLOPS_LENS * pairs
    fo_bytes = _forces_bytes(w, n_nodes)
    kern = {
        "void_fraction": {
            "kernel": "k_qcm_pts<%d> (FP32 QCM, one lane per Gauss point)" % k, "bound": "alu",
            "unit": "T FP32 instructions/s",
            "ms_per_launch": qcm_ms, "launches_per_step": calls["void_fraction"],
            "work": qcm_instr, "peak": instr_peak,
            "achieved": qcm_instr / (qcm_ms * 1e-3) / 1e12,
            "units": {"tested_pairs_cell_list": tests_cell, "neighbour_pairs": pairs,
                      "tested_pairs_element_culled": tests_culled,
                      "fp32_instructions_per_test": QCM_INSTR_TEST,
                      "fp32_instructions_per_lens": QCM_INSTR_LENS},
            "achieved_culled_count": qcm_instr_culled / (qcm_ms * 1e-3) / 1e12,
            "as_flops": {"work": qcm_flops, "peak_tflops": alu["fp32_tflops"],
                         "achieved_tflops": qcm_flops / (qcm_ms * 1e-3) / 1e12,
                         "frac": qcm_flops / (qcm_ms * 1e-3) / 1e12 / alu["fp32_tflops"],
                         "frac_culled_count": qcm_flops_culled / (qcm_ms * 1e-3) / 1e12 /
                         alu["fp32_tflops"]},
            "peak_source": "FMA probe on this device (libalupeak.so): FP32 FMA rate as "
                           "instructions/s",
            "limiter": "instruction issue (~80 % of issue slots): the streaming of the bin "
                       "rows (row bounds, warp scan, per-chunk search, box cull) is not "
                       "counted as work"},
        "forces": {
            "kernel": "k_forces<%d,%d,float>" % (k, kp), "bound": "hbm", "unit": "GB/s",
            "ms_per_launch": fo_ms, "launches_per_step": calls["forces"], "work": fo_bytes,
            "peak": hbm, "achieved": fo_bytes / (fo_ms * 1e-3) / 1e9,
            "peak_source": "%s MEASURED_PEAKS.json hbm_gbs" % peak_kind,
            "limiter": "instruction issue at ~40 % of the slots with 20 warps per SM (one "
                       "thread per particle): ~6,000 instructions a particle, mostly the "
                       "double-float splits of the nodal values and the compensated slip "
                       "sums; not the gathers (all nodal fields prefetched into L2, or a "
                       "layer's gathers issued together, left it as slow); no FP64 "
                       "instruction per node on the mixed path"},
        "op32": {
            "kernel": "k_cg_apply_df<%d> (double-float CG operator on the FP32 pipes)" % k,
            "bound": "alu", "unit": "T FP32 instructions/s", "ms_per_launch": op_ms,
            "launches_per_step": op_launches, "work": 12.0 * op_macs,
            "peak": instr_peak, "achieved": 12.0 * op_macs / (op_ms * 1e-3) / 1e12,
            "units": {"df_multiply_adds": op_macs, "fp32_instructions_per_df_multiply_add": 12,
                      "hbm_bytes_algorithmic": 16.0 * n_nodes},
            "peak_source": "FMA probe on this device (libalupeak.so): FP32 FMA rate as "
                           "instructions/s",
            "limiter": "instruction issue: each double-float multiply-add of the banded 1D "
                       "passes (7 (2k+1) per node) is 12 FP32 instructions (exact product, "
                       "two-sum, error accumulation); the algorithmic HBM traffic (the "
                       "double-float vector in and out, 16 B per node) would take ~3 us"},
    }
    for c in ("void_fraction", "forces", "op32"):
        kern[c]["frac"] = kern[c]["achieved"] / kern[c]["peak"]
    kern["void_fraction"]["frac_culled_count"] = (kern["void_fraction"]["achieved_culled_count"] /
                                                   kern["void_fraction"]["peak"])
    dom = max(("void_fraction", "forces", "op32"),
              key=lambda c: kern[c]["ms_per_launch"] * kern[c]["launches_per_step"])
    d = kern[dom]
    roof = {"bound": d["bound"], "kernel": d["kernel"], "achieved": d.get("achieved"),
            "peak": d.get("peak"), "unit": d.get("unit"), "frac": d.get("frac"),
            "traffic": NCU_TRAFFIC.get(dom) if name == WORKLOAD else None,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + "
                            "dram__bytes_write.sum)",
            "ms_per_launch": d["ms_per_launch"], "launches_per_step": d["launches_per_step"],
            "others": {c: v for c, v in kern.items() if c != dom}}
    for key in ("units", "achieved_culled_count", "frac_culled_count", "as_flops", "limiter",
                "peak_source", "work"):
        if key in d:
            roof[key] = d[key]
    res["roofline"] = roof
    res["step_hbm"] = _step_bytes(n, n_nodes, E, Q, per[1]["cg_iterations"],
                                  per[1]["ms_per_step"], hbm)
    res["step_hbm"]["peak_source"] = "%s MEASURED_PEAKS.json hbm_gbs" % peak_kind
    res["_config"] = workload_config(name, w)
    res["_ms"] = per[1]["_ms"]
    res["_clocks"] = per[1]["clocks"]
    res["_launches"] = per[1]["eager"]["kernel_launches_per_step"]

    # ---- end to end through host buffers (headline bed)
    if e2e:
        g = graph[1]
        hx = {kk: torch.as_tensor(w[kk], dtype=torch.float64).pin_memory()
              for kk in ("x", "r", "u_p", "u_nodal", "p_nodal")}
        hx["f"] = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        hx["F_elem"] = torch.empty((E, 3), dtype=torch.float64).pin_memory()
        h2d = sum(hx[kk].numel() * 8 for kk in ("x", "r", "u_p", "u_nodal", "p_nodal"))
        d2h = (hx["f"].numel() + hx["F_elem"].numel()) * 8
        og = g["out"]
        f_dev = og["f"].cpu().numpy()     # the device-buffer run's forces
        hio = [cf.bed_io(n, x, r, up, un, pn, og["eps_h"], og["f"], og["fd"], og["Fe"],
                         host=hx)]

        def step_host():
            og["eps_h"].zero_()
            if cf.cfdem_batch_coupling_step(g["bh"], hio) != cf.OK:
                raise RuntimeError(cf.cfdem_batch_last_error(g["bh"]))

        with torch.cuda.stream(s):
            for _ in range(warmup):
                step_host()
        ms_h, clk_h = env.timed(step_host, steps)
        e2e_ms = float(np.mean(ms_h))
        res["e2e"] = {"value": env.world * n / (e2e_ms * 1e-3), "unit": "particle updates/s",
                      "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h,
                      "launch": "cfdem_batch_coupling_step with page-locked host buffers: the "
                                "uploads and downloads run inside the replayed graph",
                      "replayed": cf.cfdem_batch_last_replayed(g["bh"]),
                      "err_f_vs_device_run": rel_err(hx["f"].numpy(), f_dev),
                      "clocks": clk_h}
    for p in (0, 1):
        cf.cfdem_batch_destroy(graph[p]["bh"])
    for c in ctxs.values():
        c.close()
    if cpu and env.rank == 0:
        res["cpu_baseline"] = cpu_baseline(w, name, steps=cpu_steps)
    return res


# ------------------------------------------------------------ other legs

def run_batch(env, steps, warmup, precision="mixed"):
    """The ensemble of 64 independent beds (Q1-Q3, 8-32 elements per axis, z up
    to 64, N log-uniform in [5e3, 2e5]): one cfdem_batch_coupling_step per step
    (one CUDA-graph replay after the first), against the same 64 beds stepped
    one after another through cfdem_coupling_step on one stream."""
    import torch
    from paper_2211_01185_gb300 import cfdem as cf
    from paper_2211_01185_gb300 import synth
    beds = synth.make_batch_workload(64)
    prec = 0 if precision == "fp64" else 1
    for b in beds:
        b["params"] = dict(b["params"], precision=prec, cg_rtol=1e-13 if prec == 0 else 1e-12,
                           max_radius=float(b["r"].max()))
    s = env.stream
    dev = env.dev
    bufs = []
    with torch.cuda.stream(s):
        for b in beds:
            n = b["x"].shape[0]
            ne = int(np.prod(b["n_el"]))
            nn = b["u_nodal"].shape[0]
            bufs.append(dict(n=n, x=env.t(b["x"]), r=env.t(b["r"]), u_p=env.t(b["u_p"]),
                             u=env.t(b["u_nodal"]), p=env.t(b["p_nodal"]),
                             eps=torch.zeros(nn, dtype=torch.float64, device=dev),
                             f=torch.empty((n, 3), dtype=torch.float64, device=dev),
                             fd=torch.empty((n, 3), dtype=torch.float64, device=dev),
                             Fe=torch.empty((ne, 3), dtype=torch.float64, device=dev)))
    n_tot = sum(bb["n"] for bb in bufs)
    ios = [cf.bed_io(bb["n"], bb["x"], bb["r"], bb["u_p"], bb["u"], bb["p"], bb["eps"], bb["f"],
                     bb["fd"], bb["Fe"]) for bb in bufs]
    bh = cf.cfdem_batch_create(len(beds), env.local, s.cuda_stream)
    for i, b in enumerate(beds):
        h = cf.cfdem_batch_bed(bh, i)
        cf.cfdem_set_mesh(h, b["origin"], b["extent"], b["n_el"], b["k"])
        cf.cfdem_set_params(h, cf.make_params(**b["params"]))
    solo = [cf.Context(b["origin"], b["extent"], b["n_el"], b["k"], b["params"],
                       device=env.local, stream=s.cuda_stream) for b in beds]

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

    with torch.cuda.stream(s):
        for _ in range(warmup):
            step_batch()
    ms_b, clk_b = env.timed(step_batch, steps)
    st, bad = cf.cfdem_batch_synchronize(bh)
    replayed = cf.cfdem_batch_last_replayed(bh)
    its = [cf.cfdem_get_stats(cf.cfdem_batch_bed(bh, i)).cg_iterations for i in range(len(beds))]
    with torch.cuda.stream(s):
        for _ in range(2):
            step_solo()
    ms_s, clk_s = env.timed(step_solo, max(3, steps // 4))
    for c in solo:
        cf.cfdem_synchronize(c.h)
    # each bed as its own one-bed batch (its own graph), the 64 graphs
    # replayed one after another: the launch overhead removed as in the
    # batch, without the beds running side by side
    singles = []
    for i, b in enumerate(beds):
        h1 = cf.cfdem_batch_create(1, env.local, s.cuda_stream)
        bed1 = cf.cfdem_batch_bed(h1, 0)
        cf.cfdem_set_mesh(bed1, b["origin"], b["extent"], b["n_el"], b["k"])
        cf.cfdem_set_params(bed1, cf.make_params(**b["params"]))
        singles.append(h1)

    def step_graphs():
        zero_eps()
        for h1, io in zip(singles, ios):
            if cf.cfdem_batch_coupling_step(h1, [io]) != cf.OK:
                raise RuntimeError(cf.cfdem_batch_last_error(h1))

    with torch.cuda.stream(s):
        for _ in range(2):
            step_graphs()
    ms_g, _ = env.timed(step_graphs, max(3, steps // 4))
    for h1 in singles:
        cf.cfdem_batch_synchronize(h1)
        cf.cfdem_batch_destroy(h1)
    mb, msolo, mgr = float(np.mean(ms_b)), float(np.mean(ms_s)), float(np.mean(ms_g))
    res = {"metric": METRIC, "value": n_tot / (mb * 1e-3), "unit": "particle updates/s",
           "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": mb,
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
           "solo_sequential": {"value": n_tot / (msolo * 1e-3), "ms_per_step": msolo,
                               "speedup_of_batch": msolo / mb},
           "solo_graphs": {"ms_per_step": mgr, "speedup_of_batch": mgr / mb,
                           "launch": "64 one-bed graphs replayed one after another"},
           "clocks": clk_b, "clocks_solo": clk_s}
    cf.cfdem_batch_destroy(bh)
    for c in solo:
        c.close()
    return res


def run_adjoint(env, steps, warmup):
    """The sensitivity workload (24x24x96 Q2, 200,000 spheres, annulus and jet):
    one step = the forward coupling step and the adjoint of J = sum_i e_z .
    f_D,i + ||eps_h||_M (dJ/dx and dJ/du), FP64 and mixed."""
    import torch
    from paper_2211_01185_gb300 import cfdem as cf
    from paper_2211_01185_gb300 import synth
    w = synth.make_adjoint_workload()
    n = w["x"].shape[0]
    s = env.stream
    dev = env.dev
    out = {}
    with torch.cuda.stream(s):
        x, r, up, un, pn = (env.t(w[k]) for k in ("x", "r", "u_p", "u_nodal", "p_nodal"))
        nn = un.shape[0]
        E = int(np.prod(w["n_el"]))
        z = lambda *sh: torch.zeros(sh, dtype=torch.float64, device=dev)  # noqa: E731
        eps, f, fd, Fe = z(nn), z(n, 3), z(n, 3), z(E, 3)
        g_fd = z(n, 3)
        g_fd[:, 2] = 1.0
        Me, dJdx, dJdu = z(nn), z(n, 3), z(nn, 3)
    grads = {}
    for prec in (0, 1):
        prm = dict(w["params"], precision=prec, cg_rtol=1e-13 if prec == 0 else 1e-12,
                   max_radius=float(w["r"].max()))
        ctx = cf.Context(w["origin"], w["extent"], w["n_el"], w["k"], prm, device=env.local,
                         stream=s.cuda_stream)

        def step():
            eps.zero_()
            cf.cfdem_coupling_step(ctx.h, n, x, r, up, un, pn, eps, f, fd, Fe)
            cf.cfdem_mass_apply(ctx.h, eps, Me)
            g_eps = Me / torch.sqrt(torch.dot(eps, Me))
            cf.cfdem_adjoint(ctx.h, n, x, r, up, un, pn, eps, None, g_fd, g_eps, dJdx, dJdu)

        with torch.cuda.stream(s):
            for _ in range(warmup):
                step()
            cf.cfdem_synchronize(ctx.h)
        ms, clocks = env.timed(step, steps)
        cf.cfdem_synchronize(ctx.h)
        st = ctx.stats()
        m = float(np.mean(ms))
        grads[prec] = (dJdx.cpu().numpy(), dJdu.cpu().numpy())
        out[prec] = {"ms_per_step": m, "value": n / (m * 1e-3), "adjoint_cg_iterations":
                     st.cg_iterations, "clocks": clocks,
                     "dJdx_norm": float(np.linalg.norm(grads[prec][0])),
                     "dJdu_norm": float(np.linalg.norm(grads[prec][1]))}
        ctx.close()
    return {"metric": "particle gradient evaluations/s (forward step + adjoint)",
            "value": out[1]["value"], "unit": "particle updates/s", "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": out[1]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": w["name"], "mesh": "Q2 24x24x96", "particles": n,
                       "nodes": int(nn), "loss": "sum_i e_z.f_D,i + ||eps_h||_M",
                       "l2": "256 MiB buffer written between timed steps"},
            "mixed": out[1], "fp64": out[0],
            "err_mixed_vs_fp64": {"dJdx": rel_err(grads[1][0], grads[0][0]),
                                  "dJdu": rel_err(grads[1][1], grads[0][1])}}


def run_dem(env, steps, warmup):
    """The particle side of the coupling on the bench bed (100,000 spheres,
    d ~ U[2,3] mm, packed with small overlaps in the lower 40 % of the
    0.1 x 0.1 x 0.4 m box): one step = one CFD step's worth of DEM, 10
    Velocity Verlet sub-steps of 5 us with the contact model of Table
    (viscoelastic), with the coupling step's forces held as f_fp; also timed:
    the coupled step (mixed coupling step replayed as a graph, then the 10
    DEM sub-steps on its forces)."""
    import torch
    from paper_2211_01185_gb300 import cfdem as cf
    from paper_2211_01185_gb300 import synth
    w = synth.make_workload(WORKLOAD)
    n = w["x"].shape[0]
    nsub, dt = 10, 5e-6
    s = env.stream
    dev = env.dev
    lo = np.asarray(w["origin"], dtype=np.float64)
    hi = lo + np.asarray(w["extent"], dtype=np.float64)
    dprm = dict(rho_p=2500.0, youngs=1e7, poisson=0.3, restitution=0.9, friction=0.3,
                rolling_friction=0.01, wall_youngs=1e7, wall_poisson=0.3,
                wall_restitution=0.9, wall_friction=0.3, wall_rolling_friction=0.01,
                g=(0.0, 0.0, -9.81), lo=tuple(lo), hi=tuple(hi),
                max_radius=float(w["r"].max()), capacity=24)
    with torch.cuda.stream(s):
        x0, r, up, un, pn = (env.t(w[k]) for k in ("x", "r", "u_p", "u_nodal", "p_nodal"))
        x, v, om = x0.clone(), up.clone(), torch.zeros_like(up)
        nn = un.shape[0]
        E = int(np.prod(w["n_el"]))
        eps = torch.zeros(nn, dtype=torch.float64, device=dev)
        f = torch.zeros((n, 3), dtype=torch.float64, device=dev)
        fd, Fe = torch.zeros_like(f), torch.zeros((E, 3), dtype=torch.float64, device=dev)
    prm = dict(w["params"], precision=1, max_radius=float(w["r"].max()), cg_rtol=1e-12)
    bh = cf.cfdem_batch_create(1, env.local, s.cuda_stream)
    bed = cf.cfdem_batch_bed(bh, 0)
    cf.cfdem_set_mesh(bed, w["origin"], w["extent"], w["n_el"], w["k"])
    cf.cfdem_set_params(bed, cf.make_params(**prm))
    dem = cf.Dem(dprm, device=env.local, stream=s.cuda_stream)

    def coupling():
        eps.zero_()
        io = cf.bed_io(n, x, r, v, un, pn, eps, f, fd, Fe)
        assert cf.cfdem_batch_coupling_step(bh, [io]) == cf.OK

    with torch.cuda.stream(s):
        coupling()                                  # forces of the packed bed
        cf.cfdem_batch_synchronize(bh)
    per = {}
    for prec in (0, 1):                              # FP64, then mixed (kept for the coupled run)
        dem.set_params(dict(dprm, precision=prec))
        dem.reset()
        with torch.cuda.stream(s):
            x.copy_(x0)
            v.copy_(up)
            om.zero_()
            for _ in range(warmup):
                dem.step(x, v, om, r, f, dt, nsub)
        ms_p, clk_p = env.timed(lambda: dem.step(x, v, om, r, f, dt, nsub), steps)
        m = float(np.mean(ms_p))
        per[prec] = {"ms_per_step": m, "value": n * nsub / (m * 1e-3),
                     "status": int(dem.synchronize()), "clocks": clk_p}

    def coupled():
        coupling()
        dem.step(x, v, om, r, f, dt, nsub)

    with torch.cuda.stream(s):
        for _ in range(warmup):
            coupled()
    ms_cpl, clocks_cpl = env.timed(coupled, steps)
    st_b = cf.cfdem_batch_synchronize(bh)
    st_dem2 = dem.synchronize()
    drift = float(torch.linalg.norm(x - x0, dim=1).max().item())
    dem.close()
    cf.cfdem_batch_destroy(bh)
    m_cpl = float(np.mean(ms_cpl))
    return {"metric": "DEM particle sub-steps/s (visco-elastic contacts, Velocity Verlet)",
            "value": per[1]["value"], "unit": "particle sub-steps/s", "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": per[1]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "dem_" + WORKLOAD, "particles": n, "substeps_per_step": nsub,
                       "dt_dem": dt, "contact_capacity": 24,
                       "l2": "256 MiB buffer written between timed steps"},
            "status": {"dem": per[1]["status"], "dem_coupled": int(st_dem2),
                       "batch": list(st_b)},
            "precision": "mixed (FP32 contact forces, FP64 state)", "fp64": per[0],
            "coupled_step": {"ms_per_step": m_cpl, "value": n / (m_cpl * 1e-3),
                             "unit": "particle CFD steps/s (coupling + 10 DEM sub-steps)",
                             "clocks": clocks_cpl},
            "max_displacement_m": drift, "clocks": per[1]["clocks"]}


def run_profile(args):
    """Eager coupling steps of one bed for ncu captures: the autotuner off and
    the bin edge given (the one the tuned bench run reports), so that a
    capture filtered by kernel name sees the step's own launches only."""
    import torch
    from paper_2211_01185_gb300 import build as B
    from paper_2211_01185_gb300 import cfdem as cf
    from paper_2211_01185_gb300 import synth
    B.build()
    w = synth.make_workload(args.workload)
    n = w["x"].shape[0]
    dev = torch.device("cuda", 0)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64).to(dev).contiguous()  # noqa: E731
    x, r, up, un, pn = (t(w[k]) for k in ("x", "r", "u_p", "u_nodal", "p_nodal"))
    prec = 0 if args.precision == "fp64" else 1
    prm = dict(w["params"], precision=prec, max_radius=float(w["r"].max()),
               cg_rtol=1e-13 if prec == 0 else 1e-12, autotune=0, bin_edge=args.bin_edge)
    with cf.Context(w["origin"], w["extent"], w["n_el"], w["k"], prm) as ctx:
        st = ctx.stats()
        eps = torch.zeros(st.n_nodes, dtype=torch.float64, device=dev)
        f = torch.empty((n, 3), dtype=torch.float64, device=dev)
        fd = torch.empty_like(f)
        Fe = torch.empty((st.n_elem, 3), dtype=torch.float64, device=dev)
        for _ in range(args.steps):
            eps.zero_()
            cf.cfdem_coupling_step(ctx.h, n, x, r, up, un, pn, eps, f, fd, Fe)
        cf.cfdem_synchronize(ctx.h)
        st = ctx.stats()
    print(json.dumps({"profile": args.workload, "precision": args.precision,
                      "bins": list(st.nb), "bin_edge_m": list(st.bin_edge),
                      "tile_shape": st.tile_shape, "cg_iterations": st.cg_iterations}))
    return 0


def _summary(r):
    """The keys of a secondary workload that the bench line carries."""
    keep = ("workload", "mesh", "particles", "nodes", "value", "ms_per_step", "steps",
            "mixed", "fp64", "mixed_speedup_over_fp64", "err_mixed_vs_fp64", "roofline",
            "step_hbm", "cpu_baseline", "solo_sequential", "solo_graphs", "graph_replayed",
            "batch_status", "cg_iterations", "coupled_step", "status", "config", "clocks", "metric", "unit")
    return {k: v for k, v in r.items() if k in keep}


# ------------------------------------------------------------------ main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="the headline bed only (no secondary workloads)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=list(SINGLE_BEDS) + ["batch64", "adjoint5", "dem"],
                    help="a single bed (the default is the headline Q2 bed plus every other "
                         "workload in brief); batch64: the 64-bed ensemble; adjoint5: forward "
                         "step + adjoint; dem: 10 DEM sub-steps per step on the Q2 bed")
    ap.add_argument("--profile", action="store_true",
                    help="eager steps of one bed only (for ncu): --steps steps, autotuner "
                         "off, bins of edge --bin-edge (0: R + largest radius)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="precision of the --profile run")
    ap.add_argument("--bin-edge", type=float, default=0.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)

    env = Env(use_dist=True)
    if args.workload == "batch64":
        print(json.dumps(run_batch(env, args.steps, args.warmup)), flush=True)
        return 0
    if args.workload == "adjoint5":
        print(json.dumps(run_adjoint(env, args.steps, args.warmup)), flush=True)
        return 0
    if args.workload == "dem":
        print(json.dumps(run_dem(env, args.steps, args.warmup)), flush=True)
        return 0

    alu = alu_peaks()
    name = args.workload
    main_bed = run_bed(env, name, args.steps, args.warmup, alu, headline=True,
                       e2e=not args.no_e2e, cpu=not args.no_cpu_baseline)
    ms_all = main_bed.pop("_ms")
    clocks = main_bed.pop("_clocks")
    launches = main_bed.pop("_launches")
    ms_g = _max_over_ranks(float(np.mean(ms_all)), env.dist, env.dev)
    ms_g_median = _max_over_ranks(float(np.median(ms_all)), env.dist, env.dev)
    n = main_bed["particles"]
    res = {"metric": METRIC, "value": _job_value(n, env.world, ms_g),
           "unit": "particle updates/s", "n_gpus": env.world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_g, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": main_bed.pop("_config"),
           "run": {"precision": "mixed", "cg_rtol": 1e-12,
                   "launch": "one CUDA-graph replay per step (cfdem_batch_coupling_step)",
                   "parallelism": "replicas" if env.world > 1 else "single GPU"},
           "ms_per_step_median": ms_g_median}
    for key in ("mixed", "fp64", "mixed_speedup_over_fp64", "err_mixed_vs_fp64", "roofline",
                "step_hbm", "e2e", "cpu_baseline"):
        if key in main_bed:
            res[key] = main_bed[key]
    res["alu_peaks_tflops"] = alu
    res["gpu_launches"] = int(round(launches * args.steps))
    res["gpu_launches_note"] = ("library kernels per eager step x K; the graph replays the "
                                "same kernels less the CG iterations after convergence")
    res["clocks"] = clocks
    if env.world == 1 and name == WORKLOAD and not args.quick:
        k2 = max(3, min(args.steps, 50))
        wl = {}
        t0 = time.time()
        for other in ("q1_8x8x32_2k", "q3_24x24x96_1m"):
            wl[other] = _summary(run_bed(env, other, k2, args.warmup, alu, e2e=False,
                                         cpu=not args.no_cpu_baseline,
                                         cpu_steps=None if other == "q1_8x8x32_2k" else 2))
        kb = max(3, min(args.steps, 10))
        wl["batch64"] = _summary(run_batch(env, kb, args.warmup))
        wl["adjoint5"] = _summary(run_adjoint(env, kb, args.warmup))
        wl["dem"] = _summary(run_dem(env, kb, args.warmup))
        res["workloads"] = wl
        res["workloads_seconds"] = time.time() - t0
    if env.dist is not None:
        env.dist.barrier()
    if env.rank == 0:
        print(json.dumps(res), flush=True)
    if env.dist is not None:
        env.dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

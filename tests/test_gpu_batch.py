"""Batched ensemble of independent beds (cfdem_batch_*), replayed as one
CUDA graph whose CG loops iterate on the device.

Every bed of a batch step must give what cfdem_coupling_step gives on that
bed alone (bit for bit for the void fraction and the forces; the fluid
source up to the order of its atomic additions), on the eager first step and
on graph replays; a
replay must read the current contents of the captured buffers; a bed that
cannot be captured keeps the batch eager; and a replayed FP64 bed must match
the oracle within the FP64 bound."""
import numpy as np
import pytest

from _parity import dev, host, rel_err
from oracle import oracle as O
from paper_2211_01185_gb300 import cfdem as cf
from paper_2211_01185_gb300 import synth

pytestmark = pytest.mark.gpu

SAME = 1e-12  # fluid source: sums of the same FP64 terms in another order


def _beds():
    beds = synth.make_batch_workload(6, seed=77, n_range=(400, 2500), nxy=(4, 8), nz=(4, 10))
    for i, b in enumerate(beds):
        b["params"] = dict(b["params"], precision=i % 2, cg_rtol=1e-12)
    # one FP64 bed with the Jacobi preconditioner (a longer device-driven loop)
    beds[2]["params"] = dict(beds[2]["params"], precision=0, cg_precond=0)
    return beds


def _buffers(b):
    import torch
    n = b["x"].shape[0]
    ne = int(np.prod(b["n_el"]))
    nn = int(np.prod([b["n_el"][a] * b["k"] + 1 for a in range(3)]))
    z = lambda *s: torch.zeros(s, dtype=torch.float64, device="cuda:0")
    return dict(x=dev(b["x"]), r=dev(b["r"]), u_p=dev(b["u_p"]), u=dev(b["u_nodal"]),
                p=dev(b["p_nodal"]), eps=z(nn), f=z(n, 3), fd=z(n, 3), Fe=z(ne, 3), n=n)


def _io(t):
    return cf.bed_io(t["n"], t["x"], t["r"], t["u_p"], t["u"], t["p"], t["eps"], t["f"],
                     t["fd"], t["Fe"])


def _solo(b, t):
    """cfdem_coupling_step on the bed alone, cold start; host copies."""
    import torch
    out = {k: torch.zeros_like(t[k]) for k in ("eps", "f", "fd", "Fe")}
    with cf.Context(b["origin"], b["extent"], b["n_el"], b["k"], b["params"]) as ctx:
        cf.cfdem_coupling_step(ctx.h, t["n"], t["x"], t["r"], t["u_p"], t["u"], t["p"],
                               out["eps"], out["f"], out["fd"], out["Fe"])
        cf.cfdem_synchronize(ctx.h)
    return {k: host(v) for k, v in out.items()}


def _make_batch(beds):
    import torch
    bh = cf.cfdem_batch_create(len(beds), 0, torch.cuda.current_stream().cuda_stream)
    for i, b in enumerate(beds):
        h = cf.cfdem_batch_bed(bh, i)
        cf.cfdem_set_mesh(h, b["origin"], b["extent"], b["n_el"], b["k"])
        cf.cfdem_set_params(h, cf.make_params(**b["params"]))
    return bh


def _step(bh, bufs):
    for t in bufs:
        t["eps"].zero_()  # cold start, as the solo reference
    st = cf.cfdem_batch_coupling_step(bh, [_io(t) for t in bufs])
    assert st == cf.OK, cf.cfdem_batch_last_error(bh)
    st, bad = cf.cfdem_batch_synchronize(bh)
    assert st == cf.OK and bad == -1
    return cf.cfdem_batch_last_replayed(bh)


def _check(bufs, refs):
    for t, ref in zip(bufs, refs):
        for k in ("eps", "f", "fd"):
            assert np.array_equal(host(t[k]), ref[k]), k
        assert rel_err(host(t["Fe"]), ref["Fe"]) <= SAME


def test_batch_matches_solo_eager_and_replayed():
    beds = _beds()
    bufs = [_buffers(b) for b in beds]
    refs = [_solo(b, t) for b, t in zip(beds, bufs)]
    bh = _make_batch(beds)
    try:
        replayed = []
        for _ in range(3):
            replayed.append(_step(bh, bufs))
            _check(bufs, refs)
        assert replayed == [0, 1, 1]
        for i, b in enumerate(beds):
            s = cf.cfdem_get_stats(cf.cfdem_batch_bed(bh, i))
            assert s.converged == 1 and s.cg_iterations >= 1
            if b["params"].get("cg_precond", 1) == 1:
                assert s.cg_iterations <= 8
    finally:
        cf.cfdem_batch_destroy(bh)


def test_replay_reads_current_buffer_contents():
    beds = _beds()[:3]
    bufs = [_buffers(b) for b in beds]
    bh = _make_batch(beds)
    try:
        assert _step(bh, bufs) == 0
        rng = np.random.default_rng(5)
        for b, t in zip(beds, bufs):  # move the particles and change the flow in place
            ext = np.asarray(b["extent"])
            x = np.clip(b["x"] + 0.05 * b["r"][:, None] * rng.standard_normal(b["x"].shape),
                        0.0, ext)
            b["x"] = x
            b["u_nodal"] = b["u_nodal"] * 1.3
            t["x"].copy_(dev(x))
            t["u"].copy_(dev(b["u_nodal"]))
        refs = [_solo(b, t) for b, t in zip(beds, bufs)]
        assert _step(bh, bufs) == 1
        _check(bufs, refs)
    finally:
        cf.cfdem_batch_destroy(bh)


def test_uncapturable_bed_keeps_the_batch_eager():
    beds = _beds()[:2]
    beds[1]["params"] = dict(beds[1]["params"], precision=1, cg_precond=0)
    bufs = [_buffers(b) for b in beds]
    refs = [_solo(b, t) for b, t in zip(beds, bufs)]
    bh = _make_batch(beds)
    try:
        assert [_step(bh, bufs) for _ in range(2)] == [0, 0]
        _check(bufs, refs)
    finally:
        cf.cfdem_batch_destroy(bh)


def test_replayed_fp64_bed_matches_oracle():
    case = synth.make_random_case(321, n_el=(5, 4, 6), k=2, n=300, extent=(0.05, 0.04, 0.06))
    prm = dict(case["params"], precision=0)
    bed = dict(origin=case["origin"], extent=case["extent"], n_el=case["n_el"], k=case["k"],
               x=case["x"], r=case["r"], u_p=case["u_p"], u_nodal=case["u_nodal"],
               p_nodal=case["p_nodal"], params=prm)
    bufs = [_buffers(bed)]
    bh = _make_batch([bed])
    try:
        _step(bh, bufs)
        assert _step(bh, bufs) == 1
    finally:
        cf.cfdem_batch_destroy(bh)
    m = O.Mesh(case["origin"], case["extent"], case["n_el"], case["k"])
    ref = O.coupling_step(m, prm, case["x"], case["r"], case["u_p"], case["u_nodal"],
                          case["p_nodal"])
    t = bufs[0]
    assert rel_err(host(t["eps"]), ref["eps_h"]) <= 1e-10
    assert rel_err(host(t["f"]), ref["f"]) <= 1e-10
    assert rel_err(host(t["fd"]), ref["f_drag"]) <= 1e-10
    assert rel_err(host(t["Fe"]), ref["F_e"]) <= 1e-10


def test_replayed_loop_stops_at_the_iteration_cap():
    """A bed whose CG is capped at 3 iterations: the device-driven loop of the
    replayed graph must end there and the batch must report the bed as not
    converged, with the other bed unaffected."""
    beds = _beds()[:2]
    beds[1]["params"] = dict(beds[1]["params"], precision=0, cg_precond=0, cg_maxit=3)
    bufs = [_buffers(b) for b in beds]
    bh = _make_batch(beds)
    try:
        for replay in (0, 1, 1):
            for t in bufs:
                t["eps"].zero_()
            assert cf.cfdem_batch_coupling_step(bh, [_io(t) for t in bufs]) == cf.OK
            st, bad = cf.cfdem_batch_synchronize(bh)
            assert cf.cfdem_batch_last_replayed(bh) == replay
            assert st == cf.NOT_CONVERGED and bad == 1
            s1 = cf.cfdem_get_stats(cf.cfdem_batch_bed(bh, 1))
            assert s1.converged == 0 and s1.cg_iterations == 3
            s0 = cf.cfdem_get_stats(cf.cfdem_batch_bed(bh, 0))
            assert s0.converged == 1
    finally:
        cf.cfdem_batch_destroy(bh)


def test_empty_bed_in_a_batch():
    """A bed with no particles steps (eps = 1, no forces) inside a replayed graph."""
    import torch
    beds = _beds()[:2]
    b = beds[1]
    b["x"] = b["x"][:0]
    b["r"] = b["r"][:0]
    b["u_p"] = b["u_p"][:0]
    bufs = [_buffers(bb) for bb in beds]
    bh = _make_batch(beds)
    try:
        assert [_step(bh, bufs) for _ in range(2)] == [0, 1]
        eps = host(bufs[1]["eps"])
        # mixed path: the right-hand side is summed in FP32 (the mixed bound
        # is 1e-5); FP64 path: to the CG tolerance
        tol = 1e-6 if b["params"].get("precision", 0) == 1 else 1e-10
        assert np.abs(eps - 1.0).max() <= tol
        assert torch.count_nonzero(bufs[1]["Fe"]).item() == 0
    finally:
        cf.cfdem_batch_destroy(bh)


def _host_copies(b, pinned):
    import torch
    n = b["x"].shape[0]
    ne = int(np.prod(b["n_el"]))
    src = {"x": b["x"], "r": b["r"], "u_p": b["u_p"], "u_nodal": b["u_nodal"],
           "p_nodal": b["p_nodal"]}
    h = {k: torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64)) for k, v in src.items()}
    h["f"] = torch.zeros((n, 3), dtype=torch.float64)
    h["F_elem"] = torch.zeros((ne, 3), dtype=torch.float64)
    if pinned:
        h = {k: v.pin_memory() for k, v in h.items()}
    return h


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffers_staged_inside_the_step(pinned):
    """A batch step that starts and ends in host memory: x and r uploaded
    first, u_p, u_nodal and p_nodal on a second stream beside the void
    fraction and the projection, f and F_elem downloaded at the end.  The
    results are those of device inputs; with page-locked buffers the copies
    are captured and replayed with the step, with pageable ones the batch
    stays eager."""
    import torch
    beds = _beds()[:3]
    bufs = [_buffers(b) for b in beds]
    refs = [_solo(b, t) for b, t in zip(beds, bufs)]
    hosts = [_host_copies(b, pinned) for b in beds]
    bh = _make_batch(beds)
    try:
        replayed = []
        for it in range(3):
            for t in bufs:  # the step itself must bring the inputs in
                for k in ("x", "r", "u_p", "u", "p", "eps"):
                    t[k].zero_()
            for h in hosts:
                h["f"].zero_()
                h["F_elem"].zero_()
            ios = [cf.bed_io(t["n"], t["x"], t["r"], t["u_p"], t["u"], t["p"], t["eps"],
                             t["f"], t["fd"], t["Fe"], host=h) for t, h in zip(bufs, hosts)]
            st = cf.cfdem_batch_coupling_step(bh, ios)
            assert st == cf.OK, cf.cfdem_batch_last_error(bh)
            st, bad = cf.cfdem_batch_synchronize(bh)
            assert st == cf.OK and bad == -1
            torch.cuda.synchronize()
            replayed.append(cf.cfdem_batch_last_replayed(bh))
            for h, ref in zip(hosts, refs):
                assert np.array_equal(h["f"].numpy(), ref["f"])
                assert rel_err(h["F_elem"].numpy(), ref["Fe"]) <= SAME
            _check(bufs, refs)
        assert replayed == ([0, 1, 1] if pinned else [0, 0, 0])
    finally:
        cf.cfdem_batch_destroy(bh)

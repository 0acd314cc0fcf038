"""The autotuner (autotune = 1): the first eager step of a signature times
candidate bin edges of the QCM and the operator's tile shapes and keeps the
fastest.  The choice must not change what is computed: neighbour counts and
id sums are the same bits for every bin edge, the floats agree to the
rounding of their sums, and the tuned step matches the oracle."""
import numpy as np
import pytest

from _parity import dev, host, rel_err
from oracle import oracle as O
from paper_2211_01185_gb300 import cfdem as cf
from paper_2211_01185_gb300 import synth

pytestmark = pytest.mark.gpu


def _zeros(*shape, dtype=None):
    import torch
    return torch.zeros(shape, dtype=dtype or torch.float64, device="cuda:0")


def _step(w, **prm):
    import torch
    p = dict(w["params"], max_radius=float(w["r"].max()), **prm)
    m = O.Mesh(w["origin"], w["extent"], w["n_el"], w["k"])
    n = w["x"].shape[0]
    with cf.Context(w["origin"], w["extent"], w["n_el"], w["k"], p) as ctx:
        x, r = dev(w["x"]), dev(w["r"])
        eps = _zeros(m.n_elem, m.Q)
        cnt = _zeros(m.n_elem, m.Q, dtype=torch.int32)
        ids = _zeros(m.n_elem, m.Q, dtype=torch.int64)
        eps_h, f, Fe = _zeros(m.n_nodes()), _zeros(n, 3), _zeros(m.n_elem, 3)
        cf.cfdem_coupling_step(ctx.h, n, x, r, dev(w["u_p"]), dev(w["u_nodal"]),
                               dev(w["p_nodal"]), eps_h, f, None, Fe)
        cf.cfdem_void_fraction(ctx.h, n, x, r, eps, cnt, ids)
        cf.cfdem_synchronize(ctx.h)
        st = ctx.stats()
        return dict(eps=host(eps), cnt=host(cnt), ids=host(ids), eps_h=host(eps_h), f=host(f),
                    Fe=host(Fe), tuned=st.tuned, nb=tuple(st.nb), shape=st.tile_shape,
                    R=st.qcm_radius, fdm_tile=st.fdm_tile, precond=st.precond)


@pytest.fixture(scope="module")
def bed():
    # the Q3 bed of this size keeps the test short; the Q1 bed is the small config
    return synth.make_random_case(77, n_el=(6, 7, 9), k=3, n=3000,
                                  extent=(0.06, 0.07, 0.09), overlap_ok=False)


@pytest.mark.parametrize("precision", [0, 1])
def test_tuned_step_matches_untuned_and_oracle(bed, precision):
    tol = 1e-10 if precision == 0 else 1e-5
    a = _step(bed, precision=precision, autotune=0)
    b = _step(bed, precision=precision, autotune=1)
    assert a["tuned"] == 0 and b["tuned"] == 3
    assert np.array_equal(a["cnt"], b["cnt"]) and np.array_equal(a["ids"], b["ids"])
    for key in ("eps", "eps_h", "f", "Fe"):
        assert rel_err(b[key], a[key]) <= (1e-12 if precision == 0 else 2e-6), key
    m = O.Mesh(bed["origin"], bed["extent"], bed["n_el"], bed["k"])
    e_ref, c_ref, _ = O.qcm(m, b["R"], bed["x"], bed["r"])
    assert np.array_equal(b["cnt"], c_ref)
    assert rel_err(b["eps"], e_ref) <= tol


def test_every_bin_edge_gives_the_same_neighbours(bed):
    """Each candidate the tuner may pick, forced through bin_edge."""
    m = O.Mesh(bed["origin"], bed["extent"], bed["n_el"], bed["k"])
    R = O.default_qcm_radius(m)
    cut = R + float(bed["r"].max())
    h = min(m.h)
    ref = None
    grids = set()
    for edge in (cut, cut / 1.5, cut / 2, cut / 3, h, h / 2, h / 3):
        out = _step(bed, precision=0, bin_edge=edge, autotune=1)
        assert out["tuned"] == 2             # a fixed bin edge is not tuned
        grids.add(out["nb"])
        if ref is None:
            ref = out
            continue
        assert np.array_equal(out["cnt"], ref["cnt"]) and np.array_equal(out["ids"], ref["ids"])
        assert rel_err(out["eps"], ref["eps"]) <= 1e-12
        assert rel_err(out["f"], ref["f"]) <= 1e-12
    assert len(grids) >= 4


def test_full_q3_bed_tunes_and_keeps_the_neighbours():
    """The Q3 24x24x96 bed of 1,000,000 spheres (about 360 neighbours per
    Gauss point in the bed): the tuned mixed step reports its choice and
    gives the FP64 neighbour counts of the untuned grid."""
    w = synth.make_workload("q3_24x24x96_1m")
    a = _step(w, precision=0, autotune=0)
    b = _step(w, precision=1, autotune=1)
    assert b["tuned"] == 3 and b["shape"] in (0, 1, 2)
    # the FDM slab form's register tile, timed when the plan was built
    assert b["precond"] == 1 and b["fdm_tile"] in (44, 48, 84, 88)
    assert rel_err(b["eps"], a["eps"]) <= 1e-5
    assert rel_err(b["f"], a["f"]) <= 1e-5
    c = _step(w, precision=0, autotune=1)
    assert np.array_equal(c["cnt"], a["cnt"]) and np.array_equal(c["ids"], a["ids"])

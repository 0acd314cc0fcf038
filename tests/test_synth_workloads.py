"""The seeded synthetic workloads have the structure of the beds they stand
in for: mesh, particle count and size distribution, where the bed sits, its
solid fraction, and no (or bounded) overlap between spheres.  The parity
tests and the benchmark run on exactly these arrays, so a change to a
generator that drifted from the recipe would change what is measured."""
import math

import numpy as np
import pytest

from paper_2211_01185_gb300 import synth

scipy_spatial = pytest.importorskip("scipy.spatial")


def _nearest(x):
    """Distance from each centre to its nearest other centre, and that index."""
    tree = scipy_spatial.cKDTree(x)
    d, j = tree.query(x, k=2)
    return d[:, 1], j[:, 1]


def _inside(w, whole=True):
    """Centres inside the box; with whole, the spheres too (the lattice beds
    let a jittered sphere at a wall cross it by part of its radius: only its
    centre, which locates it, must lie in the mesh)."""
    lo = np.asarray(w["origin"])
    hi = lo + np.asarray(w["extent"])
    r = w["r"][:, None] if whole else 0.0
    return bool(np.all(w["x"] - r >= lo - 1e-12) and np.all(w["x"] + r <= hi + 1e-12))


def _solid_fraction(w, z_top):
    ext = w["extent"]
    return float(np.sum(4.0 / 3.0 * math.pi * w["r"] ** 3) / (ext[0] * ext[1] * z_top))


def test_q1_bed():
    w = synth.make_workload("q1_8x8x32_2k")
    assert w["n_el"] == (8, 8, 32) and w["k"] == 1 and w["x"].shape == (2000, 3)
    assert np.all(w["r"] == 0.5e-3) and _inside(w)
    assert np.all(w["x"][:, 2] <= 0.5 * w["extent"][2])          # the lower half
    d, _ = _nearest(w["x"])
    assert d.min() >= 1e-3 * (1 - 1e-12)                          # no overlap
    assert w["u_nodal"].shape == (9 * 9 * 33, 3) and w["p_nodal"].shape == (9 * 9 * 33,)


@pytest.fixture(scope="module")
def q2():
    return synth.make_workload("q2_32x32x128_100k")


def test_q2_bed(q2):
    w = q2
    assert w["n_el"] == (32, 32, 128) and w["k"] == 2 and w["x"].shape == (100_000, 3)
    d = 2 * w["r"]
    assert d.min() >= 2e-3 and d.max() <= 3e-3 and _inside(w)
    assert abs(np.mean(d) - 2.5e-3) < 0.02e-3                     # U[2, 3] mm
    z_top = float(np.max(w["x"][:, 2] + w["r"]))
    assert z_top <= 0.4 * w["extent"][2] * 1.02                    # the lower 40 %
    assert 0.50 <= _solid_fraction(w, z_top) <= 0.56
    dist, j = _nearest(w["x"])
    gap = dist - (w["r"] + w["r"][j])
    assert gap.min() > -0.01 * d.min()                            # overlap < 1 % of d_min
    n_nodes = (64 + 1) * (64 + 1) * (256 + 1)
    assert w["u_nodal"].shape == (n_nodes, 3)
    u = w["u_nodal"]
    assert abs(np.mean(u[:, 2]) - 1.0) < 0.01                     # 1 m/s upward
    assert 0.01 < np.std(u[:, 2]) < 0.05                          # + 5 % noise


def test_q3_bed():
    w = synth.make_workload("q3_24x24x96_1m")
    assert w["n_el"] == (24, 24, 96) and w["k"] == 3 and w["x"].shape == (1_000_000, 3)
    assert np.all(w["r"] == 0.5e-3) and _inside(w, whole=False)
    z_top = float(np.max(w["x"][:, 2] + w["r"]))
    assert z_top <= 0.5 * w["extent"][2]
    assert abs(_solid_fraction(w, z_top) - 0.6) < 0.03
    dist, _ = _nearest(w["x"])
    assert dist.min() >= 1e-3 * (1 - 1e-9)                        # no overlap
    h = w["extent"][0] / w["n_el"][0]
    assert abs(h / 1e-3 - 6.0) < 1e-9                             # elements of ~6 diameters


def test_batch_of_64_beds():
    beds = synth.make_batch_workload(64)
    assert len(beds) == 64
    n = np.array([b["x"].shape[0] for b in beds])
    assert n.min() >= 5_000 and n.max() <= 200_000
    assert {b["k"] for b in beds} == {1, 2, 3}
    for b in beds:
        ne = b["n_el"]
        assert 8 <= ne[0] <= 32 and 8 <= ne[1] <= 32 and 8 <= ne[2] <= 64
        d = 2 * b["r"][0]
        assert np.all(b["r"] == b["r"][0]) and 1e-3 <= d <= 3e-3
        assert _inside(b, whole=False)
    # log-uniform counts: the median sits near the geometric mean of the range
    assert 0.4 < np.median(n) / math.sqrt(5_000 * 200_000) < 2.5


def test_adjoint_bed():
    w = synth.make_adjoint_workload()
    assert w["n_el"] == (24, 24, 96) and w["k"] == 2 and w["x"].shape == (200_000, 3)
    assert np.all(w["r"] == 1e-3) and _inside(w, whole=False)
    dist, _ = _nearest(w["x"])
    assert dist.min() >= 2e-3 * (1 - 1e-9)
    L = w["extent"][0]
    rho = np.hypot(w["x"][:, 0] - L / 2, w["x"][:, 1] - L / 2)
    column = rho < 0.15 * L
    assert 0 < column.sum() < 0.1 * len(rho)                      # a sparse central column

"""Pins of the oracle's element location and binning (Sec. 2.3: particles are
located directly on the shared mesh).

Location is checked against the definition of the element by its bounds,
hand-placed particles on faces, edges and corners, and the out-of-domain
report; binning against an independent stable sort in numpy."""
import numpy as np
import pytest

from oracle import oracle as O


def _mesh():
    return O.Mesh([0.1, -0.2, 0.05], [0.03, 0.04, 0.05], [3, 4, 5], 2)


def test_locate_bounds_random():
    m = _mesh()
    rng = np.random.default_rng(1)
    x = m.origin + m.extent * rng.random((500, 3))
    elem, xi, bad = O.locate(m, x)
    assert bad == -1
    ex = elem % 3
    ey = (elem // 3) % 4
    ez = elem // 12
    ie = np.stack([ex, ey, ez], axis=1)
    lo = m.origin + m.h * ie
    assert np.all(x >= lo - 1e-15) and np.all(x < lo + m.h + 1e-15)
    assert np.all(xi >= -1e-12) and np.all(xi <= 1 + 1e-12)
    assert np.allclose(lo + m.h * xi, x, atol=1e-15, rtol=0)


def test_locate_faces_edges_corners():
    m = O.Mesh([0.0, 0.0, 0.0], [3.0, 4.0, 5.0], [3, 4, 5], 1)    # h = 1 exactly
    pts = np.array([[1.0, 0.5, 0.5],     # interior face -> upper element (ex = 1)
                    [1.0, 2.0, 3.0],     # edge/corner of interior elements
                    [0.0, 0.0, 0.0],     # lower corner
                    [3.0, 4.0, 5.0],     # upper corner -> last element, xi = 1
                    [2.5, 4.0, 0.0]])
    elem, xi, bad = O.locate(m, pts)
    assert bad == -1
    assert list(elem) == [1 + 3 * (0 + 4 * 0), 1 + 3 * (2 + 4 * 3), 0, 2 + 3 * (3 + 4 * 4),
                          2 + 3 * (3 + 4 * 0)]
    assert np.array_equal(xi[0], [0.0, 0.5, 0.5])
    assert np.array_equal(xi[3], [1.0, 1.0, 1.0])


def test_locate_out_of_domain():
    m = _mesh()
    x = m.origin + 0.5 * m.extent + np.zeros((6, 3))
    x[3, 1] = m.origin[1] - 1e-6
    x[5, 2] = np.nan
    elem, xi, bad = O.locate(m, x)
    assert bad == 3 and elem[3] == -1 and elem[5] == -1
    # within the 1e-12 L slack: accepted and clamped
    x2 = m.origin + np.zeros((1, 3))
    x2[0, 0] -= 1e-14
    e2, xi2, bad2 = O.locate(m, x2)
    assert bad2 == -1 and e2[0] == 0


@pytest.mark.parametrize("nb", [(1, 1, 1), (2, 3, 4), (7, 5, 3)])
def test_bin_stable_counting_sort(nb):
    m = _mesh()
    rng = np.random.default_rng(2)
    x = m.origin + m.extent * rng.random((400, 3))
    x[:5] = m.origin                       # corner particles
    x[5:8] = m.origin + m.extent           # top wall -> last bins
    bin_of, start, perm = O.bin_particles(m, nb, x)
    be = m.extent / np.asarray(nb)
    ib = np.clip(np.floor((x - m.origin) / be), 0, np.asarray(nb) - 1).astype(int)
    want = ib[:, 0] + nb[0] * (ib[:, 1] + nb[1] * ib[:, 2])
    assert np.array_equal(bin_of, want)
    order = np.argsort(want, kind="stable")
    assert np.array_equal(perm, order)
    counts = np.bincount(want, minlength=int(np.prod(nb)))
    assert np.array_equal(start, np.concatenate([[0], np.cumsum(counts)]))

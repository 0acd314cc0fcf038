"""Pins of the oracle's void fraction.

* lens volume: its two tangency limits, symmetry in (R, r), continuity of V
  and dV/dd, and an independent 1D integral of the cross-section area;
* QCM: a particle wholly inside an averaging sphere contributes exactly its
  volume; cell-list neighbour sets equal brute force (C and numpy); no
  particles gives eps = 1; the integral of the solid fraction tends to the
  total particle volume as the quadrature is refined (exact in the continuum
  for particles away from the walls);
* PCM (Eq. void_fraction): sum_e V_e (1 - eps_e) equals the total particle
  volume."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2211_01185_gb300 import synth


def _lens_by_area(R, r, d):
    # cross-section at abscissa t along the line of centres: a disc of radius
    # min(sqrt(R^2 - t^2), sqrt(r^2 - (t - d)^2)) where both exist
    def area(t):
        a = R * R - t * t
        b = r * r - (t - d) ** 2
        m = min(a, b)
        return math.pi * m if m > 0 else 0.0
    lo = max(-R, d - r)
    hi = min(R, d + r)
    if hi <= lo:
        return 0.0
    pts = [p for p in [(R * R - r * r + d * d) / (2 * d) if d > 0 else None] if p is not None
           and lo < p < hi]
    v, _ = integrate.quad(area, lo, hi, points=pts or None, epsabs=0, epsrel=1e-13, limit=200)
    return v


@pytest.mark.parametrize("R,r", [(1.0, 0.3), (1.0, 1.0), (0.4, 1.3), (2.0, 0.05)])
def test_lens_limits_symmetry_integral(R, r):
    full = 4.0 / 3.0 * math.pi * min(R, r) ** 3
    assert O.lens_volume(R, r, R + r) == 0.0
    assert O.lens_volume(R, r, R + r + 1e-9) == 0.0
    assert abs(O.lens_volume(R, r, abs(R - r)) - full) <= 1e-14 * full
    assert O.lens_volume(R, r, 0.0) == full
    for d in np.linspace(abs(R - r) + 1e-6, R + r - 1e-6, 9):
        v = O.lens_volume(R, r, d)
        assert abs(v - O.lens_volume(r, R, d)) <= 1e-14 * full
        w = _lens_by_area(R, r, d)
        assert abs(v - w) <= 1e-11 * full, (d, v, w)
    # continuity of V and dV/dd at both tangencies: the gap between the
    # one-sided difference quotients closes linearly with the step
    for d0 in [abs(R - r), R + r]:
        if d0 == 0:
            continue

        def gap(e):
            dm = (O.lens_volume(R, r, d0 - e) - O.lens_volume(R, r, d0 - 2 * e)) / e
            dp = (O.lens_volume(R, r, d0 + 2 * e) - O.lens_volume(R, r, d0 + e)) / e
            return abs(dm - dp)
        e = 1e-4 * min(R, r)
        vm, vp = O.lens_volume(R, r, d0 - e), O.lens_volume(R, r, d0 + e)
        assert abs(vm - vp) < 1e-6 * full
        g1, g2 = gap(e), gap(e / 10)
        assert g2 < 0.2 * g1 or g2 < 1e-12 * full / min(R, r)


def test_qcm_particle_inside_sphere_contributes_its_volume():
    m = O.Mesh([0, 0, 0], [0.04, 0.04, 0.04], [1, 1, 1], 1)
    R = 0.01
    qp = O.quadrature_points(m)[0, 0]
    r = np.array([0.002])
    x = (qp + np.array([0.003, -0.004, 0.002]))[None, :]   # |dx| + r < R
    eps, cnt, ids = O.qcm(m, R, x, r)
    want = 1.0 - (4.0 / 3.0 * math.pi * r[0] ** 3) / (4.0 / 3.0 * math.pi * R ** 3)
    assert abs(eps[0, 0] - want) < 1e-15
    assert cnt[0, 0] == 1 and ids[0, 0] == 0


def test_qcm_empty_is_one():
    m = O.Mesh([0, 0, 0], [1, 1, 1], [2, 2, 2], 2)
    eps, cnt, _ = O.qcm(m, 0.3, np.zeros((0, 3)), np.zeros(0))
    assert np.all(eps == 1.0) and np.all(cnt == 0)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_qcm_cell_list_equals_brute_force(k):
    case = synth.make_random_case(10 + k, n_el=(3, 2, 4), k=k, n=90)
    m = O.Mesh(case["origin"], case["extent"], case["n_el"], k)
    R = O.default_qcm_radius(m)
    a = O.qcm(m, R, case["x"], case["r"], brute=False)
    b = O.qcm(m, R, case["x"], case["r"], brute=True)
    c = O.qcm_bruteforce(m, R, case["x"], case["r"])
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert np.array_equal(a[0], b[0])                      # same ascending-id sums
    assert np.array_equal(a[1], c[1]) and np.array_equal(a[2], c[2])
    assert np.max(np.abs(a[0] - c[0])) < 1e-14
    assert a[1].sum() > 0


def test_qcm_volume_conservation_under_refinement():
    rng = np.random.default_rng(5)
    L = 0.04
    R = 0.004
    n = 40
    x = 0.012 + 0.016 * rng.random((n, 3))                 # far from the walls
    r = 0.0005 + 0.001 * rng.random(n)
    vp = np.sum(4.0 / 3.0 * math.pi * r ** 3)
    errs = []
    for ne in (4, 8, 16):
        m = O.Mesh([0, 0, 0], [L, L, L], [ne, ne, ne], 2)
        eps, _, _ = O.qcm(m, R, x, r)
        g, w = O.gauss_rule(3)
        wq = np.einsum("i,j,k->kji", w, w, w).reshape(-1) * m.elem_volume
        solid = np.sum((1.0 - eps) * wq[None, :])
        errs.append(abs(solid - vp) / vp)
    assert errs[-1] < 5e-3 and errs[2] < errs[0]


def test_pcm_conservation_exact():
    case = synth.make_random_case(3, n_el=(4, 3, 5), k=2, n=300)
    m = O.Mesh(case["origin"], case["extent"], case["n_el"], 2)
    eps, bad = O.pcm(m, case["x"], case["r"])
    assert bad == -1
    assert np.all(eps == eps[:, :1])                    # constant per element
    solid = np.sum(m.elem_volume * (1.0 - eps[:, 0]))
    vp = np.sum(4.0 / 3.0 * math.pi * case["r"] ** 3)
    assert abs(solid - vp) <= 1e-13 * vp

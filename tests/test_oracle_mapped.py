"""Pins of the oracle's location on mapped (curved) Q_k hex meshes
(or_locate_mapped: Newton inversion of the element maps).

* On a box written as a mapped mesh it gives the box location's element
  and reference coordinates.
* On a subdivided cylinder (curved ring elements) it inverts the element
  map: points made as X_e(xi*) from random interior reference coordinates,
  with the map evaluated here by numpy's own polynomial tools, come back as
  (e, xi*).
* Points outside the cylinder are in no element.
The mesh generator itself is checked for positive Jacobians and the
cylinder's volume."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2211_01185_gb300 import synth


def _gll(k):
    """GLL nodes on [0,1] from numpy: the ends and the roots of P_k'."""
    if k == 1:
        inner = np.array([])
    else:
        inner = np.real(np.polynomial.legendre.Legendre.basis(k).deriv().roots())
    return np.sort(np.concatenate([[-1.0], inner, [1.0]])) * 0.5 + 0.5


def _basis(k, t):
    """Lagrange basis values and derivatives at t (numpy polynomials)."""
    z = _gll(k)
    vals, ders = [], []
    for a in range(k + 1):
        others = np.delete(z, a)
        p = np.polynomial.Polynomial.fromroots(others) / np.prod(z[a] - others)
        vals.append(p(t))
        ders.append(p.deriv()(t))
    return np.array(vals), np.array(ders)


def _map(mesh, e, xi):
    k = mesh["k"]
    P = mesh["nodes"][mesh["conn"][e]].reshape(k + 1, k + 1, k + 1, 3)   # [c][b][a]
    la, da = _basis(k, xi[0])
    lb, db = _basis(k, xi[1])
    lc, dc = _basis(k, xi[2])
    X = np.einsum("cbai,a,b,c->i", P, la, lb, lc)
    J = np.stack([np.einsum("cbai,a,b,c->i", P, da, lb, lc),
                  np.einsum("cbai,a,b,c->i", P, la, db, lc),
                  np.einsum("cbai,a,b,c->i", P, la, lb, dc)], axis=1)
    return X, J


@pytest.mark.parametrize("k", [1, 2, 3])
def test_box_as_mapped_mesh_matches_box_location(k):
    origin, extent, n_el = (0.01, -0.02, 0.0), (0.03, 0.04, 0.05), (3, 4, 5)
    mesh = synth.make_box_mapped_mesh(origin, extent, n_el, k)
    rng = np.random.default_rng(k)
    h = np.asarray(extent) / np.asarray(n_el)
    cell = rng.integers(0, n_el, size=(300, 3))
    frac = 0.02 + 0.96 * rng.random((300, 3))          # off the element faces
    x = np.asarray(origin) + (cell + frac) * h
    e_box, xi_box, bad = O.locate(O.Mesh(origin, extent, n_el, k), x)
    assert bad == -1
    e, xi, miss = O.locate_mapped(k, mesh["conn"], mesh["nodes"], x)
    assert miss == 0
    assert np.array_equal(e, e_box)
    assert np.allclose(xi, xi_box, rtol=0, atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_cylinder_round_trip(k):
    mesh = synth.make_cylinder_mesh(0.05, 0.08, 3, 2, 3, k)
    E = mesh["conn"].shape[0]
    rng = np.random.default_rng(10 + k)
    es = rng.integers(0, E, 200)
    xis = 0.03 + 0.94 * rng.random((200, 3))
    x = np.array([_map(mesh, e, xi)[0] for e, xi in zip(es, xis)])
    e, xi, miss = O.locate_mapped(k, mesh["conn"], mesh["nodes"], x)
    assert miss == 0
    assert np.array_equal(e, es)
    assert np.allclose(xi, xis, rtol=0, atol=1e-11)


def test_points_outside_the_cylinder_are_in_no_element():
    mesh = synth.make_cylinder_mesh(0.05, 0.08, 3, 2, 3, 2)
    rng = np.random.default_rng(3)
    th = rng.random(100) * 2 * math.pi
    r = 0.05 * (1.03 + 0.2 * rng.random(100))
    z = 0.08 * rng.random(100)
    out = np.stack([r * np.cos(th), r * np.sin(th), z], axis=1)
    above = np.stack([0.01 * np.cos(th), 0.01 * np.sin(th), 0.08 + 0.002 + 0.01 * rng.random(100)],
                     axis=1)
    e, xi, miss = O.locate_mapped(2, mesh["conn"], mesh["nodes"], np.vstack([out, above]))
    assert miss == 200 and np.all(e == -1) and np.all(xi == 0.0)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_cylinder_mesh_is_valid(k):
    """Positive Jacobians at the Gauss points; volume pi R^2 H up to the
    polygonal (k = 1) or polynomial (k > 1) approximation of the circle."""
    R, H = 0.05, 0.08
    mesh = synth.make_cylinder_mesh(R, H, 3, 2, 1, k)
    g, w = np.polynomial.legendre.leggauss(k + 2)
    g, w = 0.5 * (g + 1), 0.5 * w
    vol = 0.0
    for e in range(mesh["conn"].shape[0]):
        for a in range(len(g)):
            for b in range(len(g)):
                for c in range(len(g)):
                    _, J = _map(mesh, e, (g[a], g[b], g[c]))
                    d = np.linalg.det(J)
                    assert d > 0
                    vol += w[a] * w[b] * w[c] * d
    exact = math.pi * R * R * H
    # 12 segments on the circle: the chord polygon's area deficit for k = 1
    tol = 0.05 if k == 1 else 2e-3
    assert abs(vol - exact) <= tol * exact

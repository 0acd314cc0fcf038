"""Pins of the oracle's fluid-side drag (Sec. 2.3.2: the single-particle drag
written with the fluid velocity at the quadrature point and the mean
particle velocity of the cell), F_pf(x_q) = -beta_e (u_f(x_q) - u_p,avg,e).

It must equal the explicit per-element source when the fluid velocity is
uniform and the particles share one velocity; with one particle per element
and a linear fluid velocity it must give, at every Gauss point, the closed
form -beta_i / V_e (u_f(x_q) - u_p,i) with u_f(x_q) evaluated analytically
at the Gauss point coordinates, and the element mean must be that at the
element centre; model B adds the per-element pressure and shear terms."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2211_01185_gb300 import synth


def _case(k, seed=11, n=60):
    c = synth.make_random_case(seed, n_el=(3, 4, 3), k=k, n=n, extent=(0.03, 0.04, 0.03),
                               overlap_ok=False)
    return c, O.Mesh(c["origin"], c["extent"], c["n_el"], c["k"])


def _forces(m, c, u, eps, **over):
    prm = dict(c["params"], **over)
    return O.forces(m, prm, c["x"], c["r"], c["u_p"], u, c["p_nodal"], eps)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_uniform_flow_equals_explicit_source(k):
    c, m = _case(k)
    c["u_p"][:] = np.array([0.01, -0.02, 0.05])
    u = np.tile(np.array([0.1, 0.2, 1.3]), (m.n_nodes(), 1))
    eps = np.full(m.n_nodes(), 0.7)
    fo = _forces(m, c, u, eps)
    F_exp, _ = O.fluid_source(m, 0, c["x"], fo["f_drag"], fo["f_gradp"])
    Fq, Fe, bad = O.fluid_source_semi(m, 0, c["x"], c["u_p"], u, fo["f_drag"], fo["f_gradp"])
    assert bad == -1
    scale = np.abs(F_exp).max()
    assert np.abs(Fq - F_exp[:, None, :]).max() <= 1e-12 * scale
    assert np.abs(Fe - F_exp).max() <= 1e-12 * scale


@pytest.mark.parametrize("k", [1, 2, 3])
def test_linear_flow_one_particle_per_element(k):
    c, m = _case(k, seed=12, n=1)
    rng = np.random.default_rng(5)
    E = m.n_elem
    idx = np.arange(E)
    ie = np.stack([idx % m.n_el[0], (idx // m.n_el[0]) % m.n_el[1],
                   idx // (m.n_el[0] * m.n_el[1])], axis=1)
    h = np.asarray(m.h)
    origin = np.asarray(m.origin)
    x = origin + h * (ie + 0.2 + 0.6 * rng.random((E, 3)))   # one particle inside each element
    r = np.full(E, 0.1 * h.min())
    u_p = 0.05 * rng.standard_normal((E, 3))
    Bm = rng.standard_normal((3, 3)) * 20.0
    u0 = np.array([0.2, -0.1, 1.0])
    lin = lambda pts: pts @ Bm.T + u0                        # noqa: E731
    u = lin(O.node_coords(m))
    eps = np.full(m.n_nodes(), 0.8)
    fo = O.forces(m, dict(c["params"]), x, r, u_p, u, c["p_nodal"], eps)
    Fq, Fe, _ = O.fluid_source_semi(m, 0, x, u_p, u, fo["f_drag"], fo["f_gradp"])
    slip = lin(x) - u_p
    beta = np.sum(fo["f_drag"] * slip, axis=1) / np.sum(slip * slip, axis=1)
    Ve = np.prod(h)
    g, _ = O.gauss_rule(m.nq)
    nq = m.nq
    for e in range(E):
        for qz in range(nq):
            for qy in range(nq):
                for qx in range(nq):
                    xq = origin + h * (ie[e] + np.array([g[qx], g[qy], g[qz]]))
                    want = -beta[e] / Ve * (lin(xq) - u_p[e])
                    got = Fq[e, qx + nq * (qy + nq * qz)]
                    assert np.allclose(got, want, rtol=1e-11, atol=1e-11 * np.abs(want).max())
        centre = origin + h * (ie[e] + 0.5)
        want = -beta[e] / Ve * (lin(centre) - u_p[e])
        assert np.allclose(Fe[e], want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


def test_empty_elements_and_model_b_terms():
    c, m = _case(2, seed=13, n=8)
    rng = np.random.default_rng(6)
    u = c["u_nodal"] * (1.0 + 0.2 * rng.standard_normal(c["u_nodal"].shape))
    eps = np.full(m.n_nodes(), 0.6)
    fo = _forces(m, c, u, eps, mu_f=1e-3, shear_force=1)
    FqA, FeA, _ = O.fluid_source_semi(m, 0, c["x"], c["u_p"], u, fo["f_drag"], fo["f_gradp"],
                                      fo["f_shear"])
    FqB, FeB, _ = O.fluid_source_semi(m, 1, c["x"], c["u_p"], u, fo["f_drag"], fo["f_gradp"],
                                      fo["f_shear"])
    elem, _, _ = O.locate(m, c["x"])
    occupied = np.zeros(m.n_elem, bool)
    occupied[elem] = True
    assert not occupied.all()
    assert np.array_equal(FqA[~occupied], np.zeros_like(FqA[~occupied]))
    T = np.zeros((m.n_elem, 3))
    np.add.at(T, elem, fo["f_gradp"] + fo["f_shear"])
    Ve = np.prod(m.h)
    extra = FqB - FqA
    assert np.allclose(extra, -(T / Ve)[:, None, :], rtol=1e-12,
                       atol=1e-12 * np.abs(T / Ve).max())

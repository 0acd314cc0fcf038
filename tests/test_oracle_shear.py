"""Pins of the oracle's shear force -V_p div tau (Sec. 2.3.2, undisturbed
flow forces) with the deviatoric stress of Eq. (stress).

Second derivatives of the Lagrange basis must reproduce p'' for every
polynomial of the element's degree; the force must vanish for a linear
velocity and equal the closed form -V_p mu (lap u + grad div u / 3) for
polynomial fields the element reproduces exactly (quadratic for Q2 and Q3,
bilinear for Q1); model B adds it to the fluid source, keeping Newton's
third law."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2211_01185_gb300 import synth

MU = 1e-3


@pytest.mark.parametrize("k", [1, 2, 3])
def test_second_derivatives_reproduce_polynomials(k):
    z = O.gll_nodes(k)
    rng = np.random.default_rng(k)
    for _ in range(5):
        coef = rng.standard_normal(k + 1)           # p(t) = sum c_n t^n, degree k
        p = np.polynomial.Polynomial(coef)
        for t in rng.uniform(-0.2, 1.2, 7):
            got = float(np.dot(O.lagrange_dd(k, t), p(z)))
            assert got == pytest.approx(p.deriv(2)(t), rel=1e-11, abs=1e-11 * np.abs(coef).sum())


def _case(k, seed=3, n=40):
    c = synth.make_random_case(seed, n_el=(3, 4, 3), k=k, n=n, extent=(0.03, 0.04, 0.03),
                               overlap_ok=False)
    return c, O.Mesh(c["origin"], c["extent"], c["n_el"], c["k"])


def _closed_form(H, r):
    """-V_p mu (tr H_a + (1/3) sum_b H_b[a][b]) for the Hessians H[a] of u_a."""
    Vp = 4.0 / 3.0 * math.pi * r ** 3
    out = np.zeros((len(r), 3))
    for a in range(3):
        lap = H[a][0][0] + H[a][1][1] + H[a][2][2]
        gd = H[0][a][0] + H[1][a][1] + H[2][a][2]
        out[:, a] = -Vp * MU * (lap + gd / 3.0)
    return out


@pytest.mark.parametrize("k", [1, 2, 3])
def test_linear_velocity_has_no_shear_force(k):
    c, m = _case(k)
    X = O.node_coords(m)
    B = np.random.default_rng(1).standard_normal((3, 3))
    u = X @ B.T + np.array([0.3, -0.1, 1.0])
    f, bad = O.shear_force(m, MU, c["x"], c["r"], u)
    assert bad == -1
    scale = 4.0 / 3.0 * math.pi * c["r"].max() ** 3 * MU * np.abs(B).max() / min(m.h)
    assert np.abs(f).max() <= 1e-9 * scale


@pytest.mark.parametrize("k", [2, 3])
def test_quadratic_velocity_closed_form(k):
    c, m = _case(k, seed=4)
    X = O.node_coords(m) - np.asarray(c["origin"])
    rng = np.random.default_rng(2)
    C2 = rng.standard_normal((3, 3, 3)) * 50.0      # u_a = x^T C2[a] x + linear
    u = np.einsum("np,apq,nq->na", X, C2, X) + X @ rng.standard_normal((3, 3)).T
    H = C2 + np.transpose(C2, (0, 2, 1))            # constant Hessians
    f, _ = O.shear_force(m, MU, c["x"], c["r"], u)
    want = _closed_form(H, c["r"])
    assert np.abs(f - want).max() <= 1e-9 * np.abs(want).max()


def test_bilinear_velocity_on_q1():
    """u = (x y, 0, 0): lap u = 0, div u = y, so div tau = (0, mu/3, 0)."""
    c, m = _case(1, seed=5)
    X = O.node_coords(m)
    u = np.zeros_like(X)
    u[:, 0] = X[:, 0] * X[:, 1] * 1e3
    f, _ = O.shear_force(m, MU, c["x"], c["r"], u)
    Vp = 4.0 / 3.0 * math.pi * c["r"] ** 3
    assert np.allclose(f[:, 0], 0.0, atol=1e-12 * Vp.max() * MU * 1e3)
    assert np.allclose(f[:, 1], -Vp * MU * 1e3 / 3.0, rtol=1e-10, atol=0)
    assert np.allclose(f[:, 2], 0.0, atol=1e-12 * Vp.max() * MU * 1e3)


@pytest.mark.parametrize("vans", [0, 1])
def test_shear_in_forces_and_model_b_source(vans):
    c, m = _case(2, seed=6)
    rng = np.random.default_rng(3)
    u = c["u_nodal"] * (1.0 + 0.3 * rng.standard_normal(c["u_nodal"].shape))
    prm = dict(c["params"], mu_f=MU, vans_model=vans)
    eps = np.full(m.n_nodes(), 0.6)
    off = O.forces(m, prm, c["x"], c["r"], c["u_p"], u, c["p_nodal"], eps)
    on = O.forces(m, dict(prm, shear_force=1), c["x"], c["r"], c["u_p"], u, c["p_nodal"], eps)
    fs, _ = O.shear_force(m, MU, c["x"], c["r"], u)
    assert np.abs(fs).max() > 0
    assert np.allclose(on["f"], off["f"] + fs, rtol=1e-15, atol=1e-300)
    assert np.array_equal(on["f_drag"], off["f_drag"])
    F, _ = O.fluid_source(m, vans, c["x"], on["f_drag"], on["f_gradp"], on["f_shear"])
    S = on["f_drag"] + (on["f_gradp"] + fs if vans == 1 else 0.0)
    lhs = F.sum(axis=0) * m.h[0] * m.h[1] * m.h[2]
    assert np.allclose(lhs, -S.sum(axis=0), rtol=1e-12, atol=1e-12 * np.abs(S).sum())

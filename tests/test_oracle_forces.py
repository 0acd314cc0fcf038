"""Pins of the oracle's particle-fluid forces (Sec. 2.3.2) and fluid source.

* the paper's worked number: the settling velocity 0.2328 m/s of Sec. 3.1
  (tests/golden/terminal_velocity.json) from the oracle's drag closure;
* limits of the Dallavalle correlation: C_D -> 0.63^2 at high Re and
  F_D -> (23.04/24) 3 pi mu d U (0.96 x Stokes) as Re -> 0;
* Di Felice reduces to Dallavalle at eps = 1; its exponent chi is largest
  (3.7 - 0.65) at log10 Re = 1.5;
* linear u and p are interpolated exactly, so the pressure-gradient force is
  -V_p grad p for every particle; buoyancy is -rho_f V_p g;
* Newton's third law: sum_e V_e F_pf,e = -sum_i S_i."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2211_01185_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_terminal_velocity_matches_paper():
    g = json.load(open(os.path.join(GOLD, "terminal_velocity.json")))
    rp = 0.5 * g["d_p"]
    mu = g["nu"] * g["rho_f"]
    Vp = 4.0 / 3.0 * math.pi * rp ** 3
    weight = Vp * (g["rho_p"] - g["rho_f"]) * g["g"]

    def excess(v):
        f = O.drag_force(0, 0, g["rho_f"], mu, 1.0, np.array([0.0, 0.0, v]), rp)
        return f[2] - weight
    lo, hi = 1e-4, 5.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if excess(mid) > 0:
            hi = mid
        else:
            lo = mid
    v = 0.5 * (lo + hi)
    assert abs(v - g["value"]) < g["tol"], v


def test_dallavalle_limits():
    rho, mu, d = 1.2, 1.8e-5, 1e-3
    U = 1e3                                   # Re = 6.7e4
    Re = O.reynolds(rho, mu, 1.0, U, d)
    cd = O.cd_times_speed_dallavalle(rho, mu, 1.0, U, d) / U
    assert abs(cd - (0.63 + 4.8 / math.sqrt(Re)) ** 2) < 1e-14
    assert abs(cd / 0.63 ** 2 - 1.0) < 0.2
    # the low-Re error of the limit shrinks like sqrt(Re)
    for U, tol in ((1e-10, 1e-4), (1e-14, 1e-6)):
        f = O.drag_force(1, 0, rho, mu, 1.0, np.array([U, 0.0, 0.0]), 0.5 * d)
        stokes = 3.0 * math.pi * mu * d * U
        assert abs(f[0] / stokes - 23.04 / 24.0) < tol
    assert np.array_equal(O.drag_force(0, 0, rho, mu, 0.7, np.zeros(3), 1e-3), np.zeros(3))


def test_difelice_reduces_to_dallavalle_at_eps_one_and_chi_peak():
    rng = np.random.default_rng(0)
    for _ in range(10):
        U = rng.standard_normal(3)
        a = O.drag_force(0, 0, 1.2, 1.8e-5, 1.0, U, 1e-3)
        b = O.drag_force(1, 0, 1.2, 1.8e-5, 1.0, U, 1e-3)
        assert np.allclose(a, b, rtol=1e-15, atol=0)
    assert abs(O.difelice_chi(10 ** 1.5) - 3.05) < 1e-14
    assert O.difelice_chi(10 ** 1.5) < O.difelice_chi(10.0) < 3.7
    # eps^(2 - chi) with chi < 3.7: a denser bed (lower eps) raises the drag
    lo = O.drag_force(0, 0, 1.2, 1.8e-5, 0.5, np.array([0, 0, 1.0]), 1e-3)[2]
    hi = O.drag_force(0, 0, 1.2, 1.8e-5, 1.0, np.array([0, 0, 1.0]), 1e-3)[2]
    assert lo > hi
    # beta_B = beta_A / eps
    c = O.drag_force(0, 1, 1.2, 1.8e-5, 0.5, np.array([0, 0, 1.0]), 1e-3)[2]
    assert abs(c - lo / 0.5) < 1e-15 * abs(c)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_linear_fields_and_closed_form_forces(k):
    case = synth.make_random_case(20 + k, n_el=(3, 3, 4), k=k, n=60)
    m = O.Mesh(case["origin"], case["extent"], case["n_el"], k)
    prm = dict(case["params"])
    kp = max(1, k - 1)
    A = np.array([[0.1, -0.2, 0.3], [0.0, 0.5, -0.1], [0.2, 0.1, 0.4]])
    c = np.array([0.01, -0.02, 1.0])
    nodes = O.node_coords(m)
    u = nodes @ A.T + c
    gp = np.array([3.0, -7.0, -1.2e4])
    p = O.node_coords(m, kp) @ gp + 11.0
    eps_n = np.full(m.n_nodes(), 0.6)
    out = O.forces(m, prm, case["x"], case["r"], case["u_p"], u, p, eps_n)
    assert out["bad"] == -1
    Vp = 4.0 / 3.0 * math.pi * case["r"] ** 3
    # rounding of the nodal differences: ~eps_mach * max|p| / h per component
    tol = 1e-13 * np.max(np.abs(p)) / np.min(m.h) * Vp[:, None]
    assert np.all(np.abs(out["f_gradp"] + Vp[:, None] * gp[None, :]) <= tol)
    assert np.allclose(out["eps_p"], 0.6, rtol=0, atol=1e-14)
    uf = case["x"] @ A.T + c
    for i in range(0, 60, 7):
        fd = O.drag_force(prm["drag_model"], 0, prm["rho_f"], prm["mu_f"], 0.6,
                          uf[i] - case["u_p"][i], case["r"][i])
        assert np.allclose(out["f_drag"][i], fd, rtol=1e-12, atol=0)
    fb = -prm["rho_f"] * Vp[:, None] * np.asarray(prm["g"])[None, :]
    assert np.allclose(out["f"], out["f_drag"] + fb + out["f_gradp"], rtol=1e-13, atol=1e-22)


def test_eps_clamped_in_closures_only():
    m = O.Mesh([0, 0, 0], [1, 1, 1], [1, 1, 1], 1)
    x = np.array([[0.5, 0.5, 0.5]])
    r = np.array([1e-3])
    u = np.tile([0.0, 0.0, 1.0], (8, 1))
    p = np.zeros(8)
    prm = dict(rho_f=1.2, mu_f=1.8e-5, g=(0, 0, -9.81), drag_model=0, eps_floor=0.05)
    lo = O.forces(m, prm, x, r, np.zeros((1, 3)), u, p, np.full(8, 0.01))
    at = O.forces(m, prm, x, r, np.zeros((1, 3)), u, p, np.full(8, 0.05))
    hi = O.forces(m, prm, x, r, np.zeros((1, 3)), u, p, np.full(8, 1.3))
    one = O.forces(m, prm, x, r, np.zeros((1, 3)), u, p, np.full(8, 1.0))
    assert np.array_equal(lo["f_drag"], at["f_drag"])
    assert np.array_equal(hi["f_drag"], one["f_drag"])
    assert abs(lo["eps_p"][0] - 0.01) < 1e-15


@pytest.mark.parametrize("model", [0, 1])
def test_newtons_third_law(model):
    case = synth.make_random_case(31, n_el=(3, 4, 2), k=2, n=200)
    m = O.Mesh(case["origin"], case["extent"], case["n_el"], 2)
    rng = np.random.default_rng(1)
    fd = rng.standard_normal((200, 3))
    fg = rng.standard_normal((200, 3))
    F, bad = O.fluid_source(m, model, case["x"], fd, fg)
    S = fd + (fg if model == 1 else 0.0)
    assert np.allclose(m.elem_volume * F.sum(axis=0), -S.sum(axis=0), rtol=1e-12, atol=1e-12)
    elem, _, _ = O.locate(m, case["x"])
    for e in np.unique(elem)[:5]:
        assert np.allclose(m.elem_volume * F[e], -S[elem == e].sum(axis=0), rtol=1e-12)

"""Pins of the closure branches that limits alone leave open (Sec. 2.3.2):
the Rong exponent below eps = 1, Koch-Hill's F_0 on both sides of the
eps_p = 0.4 switch and its F_3 at eps_p > 0, Beetstra's inertial bracket, and
Gidaspow's Wen-Yu branch below eps = 1.

Two kinds of pin: textbook results the closures are built to reproduce
(Carman-Kozeny for the dense Koch-Hill branch, Brinkman's square-root
correction for its dilute branch, the Wen-Yu voidage factor eps^-3.65 at
equal particle Reynolds number, Newton's-regime drag), and worked values of
the printed formulas at points where they simplify by hand
(tests/golden/closure_worked_values.json).  Every force comes from the
oracle's drag_force, the function the coupling step uses."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

RHO, MU = 1.2, 1.8e-5
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "closure_worked_values.json")))
DIR = np.array([0.3, -0.2, 0.9]) / np.linalg.norm([0.3, -0.2, 0.9])


def _force(model, eps, speed, rp):
    return O.drag_force(model, 0, RHO, MU, eps, DIR * speed, rp)


def _speed_for(Re, eps, d):
    """Slip speed at which Re_p = rho eps |U| d / mu equals Re."""
    return Re * MU / (RHO * eps * d)


def test_worked_values_match_their_expressions():
    for group in ("rong_ratio", "koch_hill_f3", "koch_hill_f0_dilute", "beetstra_f"):
        for row in GOLD[group]:
            assert eval(row["expr"], {"math": math}) == pytest.approx(row["value"], rel=1e-15)


@pytest.mark.parametrize("row", GOLD["rong_ratio"])
def test_rong_exponent_below_the_fluid_limit(row):
    """Rong = Dallavalle x eps^(2 - chi_R): the force ratio at a Reynolds
    number where the Gaussian factor is 1 (log10 Re = 1.5) or exp(-1/2)."""
    rp = 1e-3
    eps = row["eps"]
    s = _speed_for(10.0 ** row["log10_re"], eps, 2 * rp)
    ratio = np.linalg.norm(_force(2, eps, s, rp)) / np.linalg.norm(_force(1, eps, s, rp))
    assert ratio == pytest.approx(row["value"], rel=1e-13)


def _koch_hill_F(eps, Re, rp):
    """F_0 + F_3 Re / 2 recovered from the force: coef = 18 mu eps^2 V_p / d^2 x F."""
    d = 2 * rp
    vp = 4.0 / 3.0 * math.pi * rp ** 3
    s = _speed_for(Re, eps, d)
    coef = np.linalg.norm(_force(3, eps, s, rp)) / s
    return coef * d * d / (18.0 * MU * eps * eps * vp)


@pytest.mark.parametrize("phi", [0.4, 0.45, 0.5, 0.6])
def test_koch_hill_dense_branch_is_carman_kozeny(phi):
    """eps_p >= 0.4 and Re -> 0: the drag of the eps_p / V_p particles in a
    unit volume, divided by eps (the fluid feels eps grad p), is the
    Carman-Kozeny pressure gradient 180 mu eps_p^2 U_s / (eps^3 d^2) at
    superficial velocity U_s = eps |U|."""
    rp = 1e-3
    d = 2 * rp
    eps = 1.0 - phi
    s = _speed_for(1e-12, eps, d)
    vp = 4.0 / 3.0 * math.pi * rp ** 3
    per_volume = phi / vp * np.linalg.norm(_force(3, eps, s, rp)) / eps
    ck = 180.0 * MU * phi * phi * (eps * s) / (eps ** 3 * d * d)
    assert per_volume == pytest.approx(ck, rel=1e-10)


def test_koch_hill_dilute_branch_has_brinkmans_square_root():
    """eps_p -> 0: F_0 = 1 + (3/sqrt 2) eps_p^(1/2) + O(eps_p ln eps_p), the
    screened-Stokeslet correction of a dilute random array (Brinkman)."""
    # powers of two, so that eps = 1 - eps_p is exact; the tolerance covers
    # the next term, (135/64) eps_p^(1/2) ln eps_p relative to 3/sqrt 2
    for phi, tol in ((2.0 ** -30, 1e-3), (2.0 ** -44, 1e-5)):
        F0 = _koch_hill_F(1.0 - phi, 1e-14, 1e-3)
        assert (F0 - 1.0) / math.sqrt(phi) == pytest.approx(3.0 / math.sqrt(2.0), rel=tol)


@pytest.mark.parametrize("row", GOLD["koch_hill_f0_dilute"])
def test_koch_hill_f0_worked_value(row):
    F = _koch_hill_F(1.0 - row["eps_p"], 1e-13, 1e-3)
    assert F == pytest.approx(row["value"], rel=1e-12)


def test_koch_hill_f0_dense_worked_value():
    """eps_p = 0.5: F_0 = 10 x 0.5 / 0.5^3 = 40."""
    assert _koch_hill_F(0.5, 1e-13, 1e-3) == pytest.approx(40.0, rel=1e-12)


@pytest.mark.parametrize("row", GOLD["koch_hill_f3"])
def test_koch_hill_f3_from_the_reynolds_slope(row):
    """F grows linearly in Re with slope F_3 / 2 at fixed eps_p."""
    eps = 1.0 - row["eps_p"]
    slope = (_koch_hill_F(eps, 1001.0, 1e-3) - _koch_hill_F(eps, 1.0, 1e-3)) / 1000.0
    assert 2.0 * slope == pytest.approx(row["value"], rel=1e-11)


@pytest.mark.parametrize("eps", [0.8, 0.85, 0.9, 0.95])
def test_gidaspow_wen_yu_newton_regime(eps):
    """Re >= 1000 (C_D = 0.44): the force on one particle is the Newton-regime
    drag 1/2 rho 0.44 (pi d^2 / 4) |U| U of a lone sphere times eps^-1.65."""
    rp = 1e-3
    d = 2 * rp
    s = _speed_for(5000.0, eps, d)
    newton = 0.5 * RHO * 0.44 * math.pi * d * d / 4.0 * s * s
    assert np.linalg.norm(_force(4, eps, s, rp)) == pytest.approx(newton * eps ** -1.65,
                                                                  rel=1e-13)


@pytest.mark.parametrize("Re", [0.5, 20.0, 400.0])
@pytest.mark.parametrize("eps", [0.8, 0.9, 0.97])
def test_gidaspow_wen_yu_voidage_factor(eps, Re):
    """At equal particle Reynolds number the Wen-Yu drag is the lone-sphere
    drag (the same model at eps = 1) times eps^-3.65, written with the
    superficial velocity: f(eps, U/eps) = f(1, U) eps^-3.65."""
    rp = 1e-3
    d = 2 * rp
    f_bed = np.linalg.norm(_force(4, eps, _speed_for(Re, eps, d), rp))
    f_one = np.linalg.norm(_force(4, 1.0, _speed_for(Re, 1.0, d), rp))
    assert f_bed == pytest.approx(f_one * eps ** -3.65, rel=1e-12)


def _beetstra_F(eps, Re, rp=1e-3):
    d = 2 * rp
    s = _speed_for(Re, eps, d)
    return np.linalg.norm(_force(5, eps, s, rp)) / (3.0 * math.pi * MU * d * eps * s)


@pytest.mark.parametrize("row", GOLD["beetstra_f"])
def test_beetstra_worked_values(row):
    assert _beetstra_F(1.0 - row["eps_p"], row["re"]) == pytest.approx(row["value"], rel=1e-12)


@pytest.mark.parametrize("phi", [0.1, 0.3, 0.5])
def test_beetstra_inertial_asymptote(phi):
    """Re -> infinity: with the bracket read as one fraction, F_i / Re tends
    to 0.413 (1/eps + 3 eps_p eps) / (24 eps^2) (the Re^-0.343 term and the
    denominator's correction vanish)."""
    eps = 1.0 - phi
    Re = 1e16
    want = 0.413 * (1.0 / eps + 3.0 * phi * eps) / (24.0 * eps * eps)
    assert _beetstra_F(eps, Re) / Re == pytest.approx(want, rel=3e-5)

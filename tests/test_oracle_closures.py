"""Pins of the oracle's drag closures (Sec. 2.3.2) other than Dallavalle and
Di Felice: Rong, Koch-Hill, Gidaspow and Beetstra.

Each is pinned to something outside its own formula: the reduction of Rong
to Dallavalle in the fluid limit (1^x = 1), the Stokes drag 3 pi mu d U of a
lone sphere at vanishing Reynolds number, the textbook single-sphere drag
with the Schiller-Naumann coefficient, the Ergun pressure gradient of a
packed bed, the low-Reynolds correlation of van der Hoef et al. that
Beetstra's extends, and the factor 1/eps of beta_B (Eq. beta)."""
import math

import numpy as np
import pytest

from oracle import oracle as O

RHO, MU = 1.2, 1.8e-5
ROUGH = (0.3, -0.2, 0.9)   # direction of the slip


def _force(model, eps, speed, rp, boe=0):
    u = np.asarray(ROUGH) / np.linalg.norm(ROUGH) * speed
    return O.drag_force(model, boe, RHO, MU, eps, u, rp), u


@pytest.mark.parametrize("speed", [1e-5, 0.03, 0.7, 12.0])
def test_rong_is_dallavalle_in_the_fluid_limit(speed):
    f_rong, _ = _force(2, 1.0, speed, 1.2e-3)
    f_dall, _ = _force(1, 1.0, speed, 1.2e-3)
    assert np.array_equal(f_rong, f_dall)
    # below eps = 1 the Rong exponent differs from Di Felice's
    assert not np.allclose(_force(2, 0.6, speed, 1.2e-3)[0], _force(0, 0.6, speed, 1.2e-3)[0],
                           rtol=1e-3, atol=0)


@pytest.mark.parametrize("model", [3, 4, 5])
def test_stokes_drag_of_a_lone_sphere(model):
    rp = 1e-3
    d = 2 * rp
    speed = 1e-12         # Re ~ 1e-10
    f, u = _force(model, 1.0, speed, rp)
    stokes = 3 * math.pi * MU * d * u
    assert np.allclose(f, stokes, rtol=2e-6, atol=0)


@pytest.mark.parametrize("speed", [1e-4, 0.05, 0.4, 3.0])
def test_koch_hill_fluid_limit_closed_form(speed):
    """eps_p = 0: F_0 = 1, F_3 = 0.0673 + 0.0232, so the force is the Stokes
    drag times 1 + F_3 Re / 2 at every Reynolds number."""
    rp = 1.5e-3
    d = 2 * rp
    f, u = _force(3, 1.0, speed, rp)
    Re = RHO * speed * d / MU
    want = 3 * math.pi * MU * d * (1 + 0.5 * (0.0673 + 0.0232) * Re) * u
    assert np.allclose(f, want, rtol=1e-13, atol=0)


@pytest.mark.parametrize("speed", [1e-3, 0.1, 2.0, 20.0])
def test_gidaspow_lone_sphere_is_schiller_naumann(speed):
    """eps = 1 (Wen-Yu branch): 1/2 rho C_D (pi d^2 / 4) |U| U with the
    Schiller-Naumann C_D (0.44 beyond Re = 1000)."""
    rp = 1e-3
    d = 2 * rp
    f, u = _force(4, 1.0, speed, rp)
    Re = RHO * speed * d / MU
    cd = 24 / Re * (1 + 0.15 * Re ** 0.687) if Re < 1000 else 0.44
    want = 0.5 * RHO * cd * math.pi * d * d / 4 * speed * u
    assert np.allclose(f, want, rtol=1e-13, atol=0)


@pytest.mark.parametrize("eps", [0.38, 0.45, 0.6, 0.79])
@pytest.mark.parametrize("speed", [0.01, 0.3, 2.5])
def test_gidaspow_dense_bed_reproduces_ergun(eps, speed):
    """Below eps = 0.8 the drag of the (1 - eps) / V_p particles in a unit
    volume, divided by eps (model A: the fluid feels eps grad p), is the
    Ergun pressure gradient 150 mu (1-eps)^2 U_s / (eps^3 d^2) + 1.75 rho
    (1-eps) U_s^2 / (eps^3 d) at superficial velocity U_s = eps |U|."""
    rp = 1.25e-3
    d = 2 * rp
    f, u = _force(4, eps, speed, rp)
    Vp = 4 / 3 * math.pi * rp ** 3
    per_volume = (1 - eps) / Vp * np.linalg.norm(f) / eps
    Us = eps * speed
    ergun = 150 * MU * (1 - eps) ** 2 * Us / (eps ** 3 * d * d) + \
        1.75 * RHO * (1 - eps) * Us * Us / (eps ** 3 * d)
    assert per_volume == pytest.approx(ergun, rel=1e-12)
    assert np.allclose(np.cross(f, u), 0.0, atol=1e-12 * np.linalg.norm(f) * speed)


def test_gidaspow_switches_branch_at_eps_08():
    """The model is piecewise: the value just below 0.8 is Ergun's and at
    0.8 Wen-Yu's (the two differ; the oracle does not smooth the jump)."""
    rp, speed = 1e-3, 0.5
    lo, _ = _force(4, 0.8 * (1 - 1e-12), speed, rp)
    hi, _ = _force(4, 0.8, speed, rp)
    d = 2 * rp
    Vp = 4 / 3 * math.pi * rp ** 3
    e = 0.8
    ergun_coef = Vp * (150 * (1 - e) * MU / (e * d * d) + 1.75 * RHO * speed / d)
    Re = RHO * e * speed * d / MU
    cd = 24 / Re * (1 + 0.15 * Re ** 0.687)
    wen_yu_coef = Vp * 0.75 * cd * e * speed * RHO / d * e ** -2.65
    assert np.linalg.norm(lo) / speed == pytest.approx(ergun_coef, rel=1e-9)
    assert np.linalg.norm(hi) / speed == pytest.approx(wen_yu_coef, rel=1e-12)


@pytest.mark.parametrize("phi", [0.0, 0.1, 0.3, 0.5])
def test_beetstra_low_reynolds_limit(phi):
    """Re -> 0: F_i -> 10 phi / (1-phi)^2 + (1-phi)^2 (1 + 1.5 sqrt(phi)),
    the Stokes-flow correlation of van der Hoef et al. (2005), phi = eps_p."""
    rp = 1e-3
    d = 2 * rp
    eps = 1 - phi
    f, u = _force(5, eps, 1e-10, rp)
    Fi = 10 * phi / eps ** 2 + eps ** 2 * (1 + 1.5 * math.sqrt(phi))
    want = 3 * math.pi * MU * d * eps * Fi * u
    assert np.allclose(f, want, rtol=1e-6, atol=0)


def test_beetstra_inertial_part_grows_with_reynolds():
    rp = 1e-3
    g = [np.linalg.norm(_force(5, 0.7, s, rp)[0]) / s for s in (0.01, 0.1, 1.0, 10.0)]
    assert all(b > a for a, b in zip(g, g[1:]))


@pytest.mark.parametrize("model", [0, 1, 2, 3, 4, 5])
def test_model_b_divides_by_eps(model):
    for eps in (0.42, 0.81, 1.0):
        fa, _ = _force(model, eps, 0.37, 1.1e-3, boe=0)
        fb, _ = _force(model, eps, 0.37, 1.1e-3, boe=1)
        assert np.allclose(fb, fa / eps, rtol=1e-15, atol=0)


@pytest.mark.parametrize("model", [0, 1, 2, 3, 4, 5])
def test_no_slip_no_drag(model):
    f = O.drag_force(model, 0, RHO, MU, 0.5, np.zeros(3), 1e-3)
    assert np.array_equal(f, np.zeros(3))

"""Pins of the oracle's DEM step (Sec. 2.2: Newton's laws, the visco-elastic
contact model of Table (viscoelastic), Velocity Verlet).

Each is pinned to something outside the code's own formulas: the exact
Velocity Verlet trajectory of free fall; the Hertz law of a static contact
(force 4/3 Y_e sqrt(R_e) d_n^(3/2) after the particle settles on a wall, so
d_n = (3 m g / (4 Y_e sqrt(R_e)))^(2/3)); the coefficient of restitution
of a head-on collision, which the damping of the table is built to give;
energy conservation without damping; conservation of linear and angular
momentum in particle-particle collisions; and the Coulomb limit of a
particle sliding on a wall."""
import math

import numpy as np
import pytest

from oracle import dem as D

LO, HI = (0.0, 0.0, 0.0), (0.02, 0.02, 0.02)


def _one(x, v, r=1e-3, w=(0.0, 0.0, 0.0)):
    return D.State(np.array([x]), np.array([v]), np.array([w]), np.array([r]))


def test_free_fall_is_exact():
    p = D.glass_params(LO, HI)
    s = _one((0.01, 0.01, 0.015), (0.01, -0.02, 0.3))
    dt, k = 1e-5, 200
    s.step(p, dt, k)
    t = dt * k
    want = np.array([0.01 + 0.01 * t, 0.01 - 0.02 * t, 0.015 + 0.3 * t - 0.5 * 9.81 * t * t])
    assert np.allclose(s.x[0], want, rtol=0, atol=1e-15)
    assert np.allclose(s.v[0], [0.01, -0.02, 0.3 - 9.81 * t], rtol=0, atol=1e-14)


def test_resting_particle_obeys_hertz():
    p = D.glass_params(LO, HI, restitution=0.3, wall_restitution=0.3)
    r = 1e-3
    s = _one((0.01, 0.01, r * 0.999), (0.0, 0.0, 0.0), r=r)
    for _ in range(40):
        s.step(p, 2e-6, 500)
    m = 2500.0 * 4.0 / 3.0 * math.pi * r ** 3
    nu = 0.3
    Ye = 1.0 / (2 * (1 - nu * nu) / 1e7)
    dn = (3 * m * 9.81 / (4 * Ye * math.sqrt(r))) ** (2.0 / 3.0)
    assert r - s.x[0, 2] == pytest.approx(dn, rel=1e-6)
    assert abs(s.v[0, 2]) < 1e-9


@pytest.mark.parametrize("e", [0.3, 0.6, 0.9])
def test_head_on_restitution(e):
    p = D.glass_params(LO, HI, restitution=e, friction=0.0, g=(0.0, 0.0, 0.0))
    r = 1e-3
    v0 = 0.2
    s = D.State(np.array([[0.008, 0.01, 0.01], [0.01 + 1e-5, 0.01, 0.01]]),
                np.array([[v0, 0.0, 0.0], [-v0, 0.0, 0.0]]), np.zeros((2, 3)),
                np.array([r, r]))
    s.step(p, 1e-7, 40000)
    vrel_after = s.v[1, 0] - s.v[0, 0]
    assert vrel_after / (2 * v0) == pytest.approx(e, rel=0.02)


@pytest.mark.parametrize("friction", [0.0, 0.3])
def test_energy_and_momentum_without_damping(friction):
    """Oblique, spinning pair: linear momentum is conserved exactly; angular
    momentum too without friction (central forces); with friction the two
    contact points lie d_n apart, so it is conserved only to d_n |f_t| dt;
    the kinetic energy never grows."""
    p = D.glass_params((-1, -1, -1), (1, 1, 1), restitution=1.0, friction=friction,
                       g=(0.0, 0.0, 0.0))
    r = np.array([1.0e-3, 1.5e-3])
    x = np.array([[0.0, 0.0, 0.0], [2.7e-3, 0.6e-3, -0.2e-3]])   # apart, closing in
    v = np.array([[0.1, 0.02, 0.0], [-0.1, 0.0, 0.01]])
    w = np.array([[0.0, 0.0, 30.0], [5.0, 0.0, 0.0]])
    s = D.State(x, v, w, r)
    m = 2500.0 * 4.0 / 3.0 * math.pi * r ** 3
    I = 0.4 * m * r * r

    def momentum(st):
        return (m[:, None] * st.v).sum(axis=0)

    def angular(st):
        return (np.cross(st.x, m[:, None] * st.v) + I[:, None] * st.w).sum(axis=0)

    p0, L0 = momentum(s), angular(s)
    E0 = 0.5 * (m * (s.v ** 2).sum(1)).sum() + 0.5 * (I * (s.w ** 2).sum(1)).sum()
    s.step(p, 1e-7, 30000)
    assert np.allclose(momentum(s), p0, rtol=0, atol=1e-12 * np.abs(p0).max())
    tol = 1e-10 if friction == 0.0 else 1e-2
    assert np.allclose(angular(s), L0, rtol=0, atol=tol * np.abs(L0).max())
    E1 = 0.5 * (m * (s.v ** 2).sum(1)).sum() + 0.5 * (I * (s.w ** 2).sum(1)).sum()
    # elastic normal contact; the tangential spring stores energy while in
    # contact and friction can dissipate it, so only the normal-only case is exact
    assert E1 <= E0 * (1 + 1e-6)


def test_elastic_normal_collision_conserves_energy():
    p = D.glass_params((-1, -1, -1), (1, 1, 1), restitution=1.0, friction=0.0,
                       g=(0.0, 0.0, 0.0))
    r = np.array([1.0e-3, 1.0e-3])
    s = D.State(np.array([[0.0, 0.0, 0.0], [2.05e-3, 0.0, 0.0]]),
                np.array([[0.3, 0.0, 0.0], [0.0, 0.0, 0.0]]), np.zeros((2, 3)), r)
    s.step(p, 1e-8, 60000)
    assert s.v[0, 0] == pytest.approx(0.0, abs=1e-4)
    assert s.v[1, 0] == pytest.approx(0.3, rel=1e-4)


def test_sliding_on_a_wall_decelerates_at_mu_g():
    mu = 0.4
    p = D.glass_params(LO, HI, restitution=0.2, wall_restitution=0.2, wall_friction=mu)
    r = 1e-3
    s = _one((0.005, 0.01, r * 0.99988), (0.0, 0.0, 0.0), r=r)
    for _ in range(10):                      # settle on the floor
        s.step(p, 2e-6, 500)
    s.v[0, 0] = 0.05                         # start sliding, no spin
    v_before = s.v[0, 0]
    s.step(p, 2e-6, 200)
    t = 2e-6 * 200
    # while sliding the floor's friction is mu m g, but it also spins the
    # sphere up (alpha = 5 mu g / (2 r)): the centre decelerates at mu g
    assert (v_before - s.v[0, 0]) / t == pytest.approx(mu * 9.81, rel=2e-2)
    assert s.w[0, 1] / t == pytest.approx(5 * mu * 9.81 / (2 * r), rel=2e-2)

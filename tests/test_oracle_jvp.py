"""Pins of the oracle's forward-mode derivatives (oracle/jvp.py).

The adjoint's reference is the derivative of the oracle's own FP64 coupling
step along an input direction, computed with dual numbers.  It is pinned to
things outside itself: elementary calculus, the geometry of the sphere-sphere
lens (its volume decreases at the rate of the area of the intersection disc),
the C oracle's values, and central finite differences of the C oracle's
coupling step."""
import math

import numpy as np
import pytest

from oracle import jvp as J
from oracle import oracle as O
from paper_2211_01185_gb300 import synth


def test_dual_elementary_rules():
    rng = np.random.default_rng(1)
    a = rng.uniform(0.5, 2.0, 7)
    da = rng.standard_normal(7)
    x = J.Dual(a, da)
    checks = [
        (J.sqrt(x), np.sqrt(a), da / (2 * np.sqrt(a))),
        (J.exp(x), np.exp(a), np.exp(a) * da),
        (J.log10(x), np.log10(a), da / (a * math.log(10.0))),
        (J.power(x, 2.5), a ** 2.5, 2.5 * a ** 1.5 * da),
        (1.0 / x, 1.0 / a, -da / a ** 2),
        (x * x * x, a ** 3, 3 * a ** 2 * da),
        (J.power(x, J.Dual(a, da)), a ** a, a ** a * (np.log(a) + 1.0) * da),
    ]
    for got, v, t in checks:
        assert np.allclose(got.v, v, rtol=1e-14, atol=0)
        assert np.allclose(got.t, t, rtol=1e-13, atol=0)
    c = J.clamp(J.Dual(np.array([0.01, 0.5, 1.2]), np.ones(3)), 0.05, 1.0)
    assert np.array_equal(c.v, [0.05, 0.5, 1.0]) and np.array_equal(c.t, [0.0, 1.0, 0.0])


def _lens_rate_closed_form(R, r, d):
    """-pi a^2, a the radius of the circle where the two spheres meet."""
    a2 = (4 * d * d * R * R - (d * d - r * r + R * R) ** 2) / (4 * d * d)
    return -math.pi * a2


@pytest.mark.parametrize("R,r", [(2e-3, 1e-3), (1e-3, 2.5e-3), (1.5e-3, 1.5e-3)])
def test_lens_derivative_is_minus_the_disc_area(R, r):
    lo, hi = abs(R - r), R + r
    for d in np.linspace(lo, hi, 41)[1:-1]:
        v = J.lens_volume(R, np.array([r]), J.Dual(np.array([d]), np.array([1.0])))
        assert v.v[0] == pytest.approx(O.lens_volume(R, r, d), rel=1e-13)
        assert v.t[0] == pytest.approx(_lens_rate_closed_form(R, r, d), rel=1e-9, abs=1e-18)
        h = 1e-7 * hi
        fd = (O.lens_volume(R, r, d + h) - O.lens_volume(R, r, d - h)) / (2 * h)
        assert v.t[0] == pytest.approx(fd, rel=1e-6, abs=1e-14 * hi * hi)
    # both tangencies: the rate goes to zero (continuity of dV/dd); with equal
    # radii the inner one is d = 0, where the spheres coincide (a cone point
    # of V(|x_i - x_q|), not a tangency)
    for d in ((lo * (1 + 1e-9),) if lo > 0 else ()) + (hi * (1 - 1e-9),):
        assert abs(_lens_rate_closed_form(R, r, d)) < 1e-6 * math.pi * min(R, r) ** 2
    inside = J.lens_volume(R, np.array([r]), J.Dual(np.array([0.5 * lo]), np.array([1.0])))
    assert inside.t[0] == 0.0


def _case(seed, k=2, n=60, n_el=(3, 4, 3), extent=(0.03, 0.04, 0.03), rough_p=False):
    c = synth.make_random_case(seed, n_el=n_el, k=k, n=n, extent=extent, overlap_ok=False)
    if rough_p:  # a pressure whose gradient varies inside the elements
        rng = np.random.default_rng(seed + 1000)
        c["p_nodal"] = c["p_nodal"] * (1.0 + 0.3 * rng.standard_normal(c["p_nodal"].shape))
    return c


def _mesh(c):
    return O.Mesh(c["origin"], c["extent"], c["n_el"], c["k"])


@pytest.mark.parametrize("k,drag", [(1, 0), (2, 0), (3, 1)])
def test_dual_primal_equals_the_c_oracle(k, drag):
    c = _case(10 + k, k=k)
    m = _mesh(c)
    prm = dict(c["params"], drag_model=drag)
    ref = O.coupling_step(m, prm, c["x"], c["r"], c["u_p"], c["u_nodal"], c["p_nodal"])
    out = J.coupling_jvp(m, prm, c["x"], c["r"], c["u_p"], c["u_nodal"], c["p_nodal"])
    assert np.allclose(out["eps_q"].v, ref["eps_q"].reshape(-1), rtol=0, atol=1e-14)
    assert np.allclose(out["eps_h"].v, ref["eps_h"], rtol=1e-11, atol=1e-13)
    for key in ("f", "f_drag", "f_gradp"):
        scale = np.abs(ref[key]).max()
        assert np.abs(out[key].v - ref[key]).max() <= 1e-11 * scale, key
    assert not np.any(out["eps_h"].t) and not np.any(out["f"].t)


def _fd(m, prm, c, dx, du, t):
    def run(s):
        x = c["x"] + s * dx
        u = c["u_nodal"] + s * du
        o = O.coupling_step(m, dict(prm, oracle_rtol=1e-15), x, c["r"], c["u_p"], u,
                            c["p_nodal"])
        return o
    p, q = run(t), run(-t)
    return {k: (p[k] - q[k]) / (2 * t) for k in ("eps_h", "f", "f_drag", "f_gradp")}


def _rel(a, b):
    b = np.asarray(b).ravel()
    a = np.asarray(a).ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("k,which", [(1, "x"), (2, "x"), (2, "u"), (3, "xu")])
def test_tangents_match_central_differences(k, which):
    c = _case(20 + k, k=k, rough_p=True)
    m = _mesh(c)
    prm = dict(c["params"])
    rng = np.random.default_rng(3)
    dx = rng.standard_normal(c["x"].shape) * c["r"][:, None] if "x" in which else \
        np.zeros_like(c["x"])
    du = rng.standard_normal(c["u_nodal"].shape) if "u" in which else \
        np.zeros_like(c["u_nodal"])
    out = J.coupling_jvp(m, prm, c["x"], c["r"], c["u_p"], c["u_nodal"], c["p_nodal"], dx, du)
    fd = _fd(m, prm, c, dx, du, 1e-6)
    for key in ("eps_h", "f", "f_drag", "f_gradp"):
        if not np.any(fd[key]) and not np.any(out[key].t):
            continue
        assert _rel(out[key].t, fd[key]) <= 2e-6, key


def test_loss_derivative_matches_central_difference():
    """J = sum_i e_z . f_D,i + ||eps_h||_M, the loss of the adjoint workload."""
    c = _case(31, k=2, n=80, rough_p=True)
    m = _mesh(c)
    prm = dict(c["params"])
    rng = np.random.default_rng(4)
    dx = rng.standard_normal(c["x"].shape) * c["r"][:, None]
    du = rng.standard_normal(c["u_nodal"].shape)

    def loss(s):
        o = O.coupling_step(m, dict(prm, oracle_rtol=1e-15), c["x"] + s * dx, c["r"],
                            c["u_p"], c["u_nodal"] + s * du, c["p_nodal"])
        e = o["eps_h"]
        return o["f_drag"][:, 2].sum() + math.sqrt(e @ O.kron_apply(m, 0.0, e))

    out = J.coupling_jvp(m, prm, c["x"], c["r"], c["u_p"], c["u_nodal"], c["p_nodal"], dx, du)
    dJ = out["f_drag"].t[:, 2].sum() + J.mass_norm(m, out["eps_h"]).t
    t = 1e-6
    fd = (loss(t) - loss(-t)) / (2 * t)
    assert dJ == pytest.approx(fd, rel=1e-6)


@pytest.mark.parametrize("drag", [2, 3, 4, 5])
def test_other_closures_primal_and_tangents(drag):
    """Rong, Koch-Hill, Gidaspow, Beetstra: the dual primal is the C oracle's
    step and the tangents its central differences (the seeded void
    fractions stay clear of the Gidaspow and Koch-Hill branch points)."""
    c = _case(40 + drag, k=2, rough_p=True)
    m = _mesh(c)
    prm = dict(c["params"], drag_model=drag, beta_over_eps=drag % 2)
    ref = O.coupling_step(m, prm, c["x"], c["r"], c["u_p"], c["u_nodal"], c["p_nodal"])
    rng = np.random.default_rng(5)
    dx = rng.standard_normal(c["x"].shape) * c["r"][:, None]
    du = rng.standard_normal(c["u_nodal"].shape)
    out = J.coupling_jvp(m, prm, c["x"], c["r"], c["u_p"], c["u_nodal"], c["p_nodal"], dx, du)
    for key in ("f", "f_drag"):
        scale = np.abs(ref[key]).max()
        assert np.abs(out[key].v - ref[key]).max() <= 1e-11 * scale, key
    fd = _fd(m, prm, c, dx, du, 1e-6)
    for key in ("f", "f_drag"):
        assert _rel(out[key].t, fd[key]) <= 2e-6, key


@pytest.mark.parametrize("k", [1, 2, 3])
def test_shear_force_primal_and_tangents(k):
    """The shear force (second derivatives of the Q_k velocity at the
    particle): dual primal = C oracle, tangents = central differences."""
    c = _case(50 + k, k=k, rough_p=True)
    m = _mesh(c)
    rng = np.random.default_rng(6)
    c["u_nodal"] = c["u_nodal"] * (1.0 + 0.3 * rng.standard_normal(c["u_nodal"].shape))
    prm = dict(c["params"], shear_force=1, mu_f=1e-3)
    ref = O.coupling_step(m, prm, c["x"], c["r"], c["u_p"], c["u_nodal"], c["p_nodal"])
    dx = rng.standard_normal(c["x"].shape) * c["r"][:, None]
    du = rng.standard_normal(c["u_nodal"].shape)
    out = J.coupling_jvp(m, prm, c["x"], c["r"], c["u_p"], c["u_nodal"], c["p_nodal"], dx, du)
    assert np.abs(out["f_shear"].v - ref["f_shear"]).max() <= 1e-11 * np.abs(ref["f_shear"]).max()
    fd = _fd(m, prm, c, dx, du, 1e-6)
    sh = lambda o: o["f_shear"]  # noqa: E731
    p, q = (O.coupling_step(m, dict(prm, oracle_rtol=1e-15), c["x"] + s * dx, c["r"], c["u_p"],
                            c["u_nodal"] + s * du, c["p_nodal"]) for s in (1e-6, -1e-6))
    assert _rel(out["f_shear"].t, (sh(p) - sh(q)) / 2e-6) <= 2e-6
    assert _rel(out["f"].t, fd["f"]) <= 2e-6


def test_sparse_qcm_tangent_equals_all_pairs():
    """qcm_dual_rows (value from the C oracle, tangent from the moved
    particles only) gives the all-pairs dual void fraction along a direction
    that moves a few particles, and so the same step derivative."""
    c = synth.make_random_case(41, n_el=(3, 4, 3), k=2, n=60, extent=(0.03, 0.04, 0.03),
                               overlap_ok=False)
    m = O.Mesh(c["origin"], c["extent"], c["n_el"], c["k"])
    rng = np.random.default_rng(5)
    dx = np.zeros_like(c["x"])
    rows = rng.choice(c["x"].shape[0], 5, replace=False)
    dx[rows] = rng.standard_normal((5, 3))
    du = rng.standard_normal(c["u_nodal"].shape)
    R = O.default_qcm_radius(m)
    a = J.qcm_dual(m, R, J.Dual(c["x"], dx), c["r"])
    b = J.qcm_dual_rows(m, R, c["x"], c["r"], dx)
    assert np.allclose(b.v, a.v, rtol=0, atol=1e-14)
    assert np.allclose(b.t, a.t, rtol=0, atol=1e-12 * np.abs(a.t).max())
    assert np.abs(a.t).max() > 0
    full = J.coupling_jvp(m, c["params"], c["x"], c["r"], c["u_p"], c["u_nodal"], c["p_nodal"],
                          dx, du)
    sp = J.coupling_jvp(m, c["params"], c["x"], c["r"], c["u_p"], c["u_nodal"], c["p_nodal"],
                        dx, du, sparse_qcm=True)
    for key in ("eps_h", "f", "f_drag"):
        assert np.allclose(sp[key].t, full[key].t, rtol=0, atol=1e-11 * np.abs(full[key].t).max())

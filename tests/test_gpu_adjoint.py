"""Adjoint of the coupling step (cfdem_adjoint) against the oracle's
forward-mode derivatives.

For a loss J with gradients g_f, g_fD, g_eps with respect to the outputs
(f, f_D, eps_h), the GPU returns dJ/dx and dJ/du.  The oracle gives, for any
input direction (dx, du), the derivative of the outputs along it (dual
numbers through its own FP64 step), hence dJ/dv = g_f . f' + g_fD . f_D' +
g_eps . eps_h'.  Every component of dJ/dx is checked (one direction per
coordinate) and dJ/du along random directions; then the loss of the adjoint
workload, J = sum_i e_z . f_D,i + ||eps_h||_M, end to end."""
import math

import numpy as np
import pytest

from _parity import dev, host, rel_err
from oracle import jvp as JV
from oracle import oracle as O
from paper_2211_01185_gb300 import cfdem as cf
from paper_2211_01185_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-8, 1: 2e-5}


def _case(seed, k, n=40, n_el=(3, 4, 3), extent=(0.03, 0.04, 0.03)):
    c = synth.make_random_case(seed, n_el=n_el, k=k, n=n, extent=extent, overlap_ok=False)
    rng = np.random.default_rng(seed + 1000)   # a pressure whose gradient varies in the elements
    c["p_nodal"] = c["p_nodal"] * (1.0 + 0.3 * rng.standard_normal(c["p_nodal"].shape))
    return c


def _gpu(c, prm, g_f, g_fd, g_eps):
    """forward step on the GPU, then its adjoint; host arrays"""
    import torch
    n = c["x"].shape[0]
    m = O.Mesh(c["origin"], c["extent"], c["n_el"], c["k"])
    z = lambda *s: torch.zeros(s, dtype=torch.float64, device="cuda:0")  # noqa: E731
    x, r, up = dev(c["x"]), dev(c["r"]), dev(c["u_p"])
    un, pn = dev(c["u_nodal"]), dev(c["p_nodal"])
    eps, f, fd, Fe = z(m.n_nodes()), z(n, 3), z(n, 3), z(m.n_elem, 3)
    dJdx, dJdu = z(n, 3), z(m.n_nodes(), 3)
    with cf.Context(c["origin"], c["extent"], c["n_el"], c["k"], prm) as ctx:
        cf.cfdem_coupling_step(ctx.h, n, x, r, up, un, pn, eps, f, fd, Fe)
        g_eps_d = g_eps(ctx, eps) if callable(g_eps) else (None if g_eps is None else dev(g_eps))
        cf.cfdem_adjoint(ctx.h, n, x, r, up, un, pn, eps,
                         None if g_f is None else dev(g_f), None if g_fd is None else dev(g_fd),
                         g_eps_d, dJdx, dJdu)
        cf.cfdem_synchronize(ctx.h)
        assert ctx.stats().converged == 1
    return host(dJdx), host(dJdu), host(eps)


def _directional(m, prm, c, dx, du, g_f, g_fd, g_eps):
    o = JV.coupling_jvp(m, prm, c["x"], c["r"], c["u_p"], c["u_nodal"], c["p_nodal"], dx, du)
    s = 0.0
    if g_f is not None:
        s += float(np.sum(g_f * o["f"].t))
    if g_fd is not None:
        s += float(np.sum(g_fd * o["f_drag"].t))
    if g_eps is not None:
        s += float(np.sum(g_eps * o["eps_h"].t))
    return s


@pytest.mark.parametrize("k,precision,drag", [(1, 0, 0), (2, 0, 0), (3, 0, 1), (2, 1, 0),
                                               (2, 0, 2), (1, 0, 3), (2, 0, 4), (2, 1, 5)])
def test_adjoint_matches_oracle_directional_derivatives(k, precision, drag):
    c = _case(600 + k, k)
    m = O.Mesh(c["origin"], c["extent"], c["n_el"], c["k"])
    prm = dict(c["params"], precision=precision, drag_model=drag, cg_rtol=1e-13 if
               precision == 0 else 1e-12)
    rng = np.random.default_rng(7 + k)
    n = c["x"].shape[0]
    g_f = rng.standard_normal((n, 3))
    g_fd = rng.standard_normal((n, 3))
    g_eps = rng.standard_normal(m.n_nodes()) * 1e-3
    dJdx, dJdu, _ = _gpu(c, prm, g_f, g_fd, g_eps)
    # every component of dJ/dx
    ref = np.zeros((n, 3))
    for i in range(n):
        for a in range(3):
            dx = np.zeros((n, 3))
            dx[i, a] = 1.0
            ref[i, a] = _directional(m, prm, c, dx, None, g_f, g_fd, g_eps)
    assert rel_err(dJdx, ref) <= TOL[precision]
    # dJ/du along random directions
    for t in range(4):
        du = rng.standard_normal(c["u_nodal"].shape)
        want = _directional(m, prm, c, None, du, g_f, g_fd, g_eps)
        got = float(np.sum(dJdu * du))
        scale = np.linalg.norm(dJdu) * np.linalg.norm(du)
        assert abs(got - want) <= TOL[precision] * scale


@pytest.mark.parametrize("k,precision", [(1, 0), (2, 0), (3, 0), (2, 1)])
def test_adjoint_with_shear_force(k, precision):
    """The shear force in a viscous liquid with a rough velocity field: its
    weights reach dJ/du, its third derivatives dJ/dx."""
    c = _case(700 + k, k)
    rng = np.random.default_rng(3 + k)
    c["u_nodal"] = c["u_nodal"] * (1.0 + 0.3 * rng.standard_normal(c["u_nodal"].shape))
    m = O.Mesh(c["origin"], c["extent"], c["n_el"], c["k"])
    prm = dict(c["params"], precision=precision, shear_force=1, mu_f=1e-3,
               cg_rtol=1e-13 if precision == 0 else 1e-12)
    n = c["x"].shape[0]
    g_f = rng.standard_normal((n, 3))
    dJdx, dJdu, _ = _gpu(c, prm, g_f, None, None)
    ref = np.zeros((n, 3))
    for i in range(n):
        for a in range(3):
            dx = np.zeros((n, 3))
            dx[i, a] = 1.0
            ref[i, a] = _directional(m, prm, c, dx, None, g_f, None, None)
    assert rel_err(dJdx, ref) <= TOL[precision]
    for t in range(3):
        du = rng.standard_normal(c["u_nodal"].shape)
        want = _directional(m, prm, c, None, du, g_f, None, None)
        got = float(np.sum(dJdu * du))
        assert abs(got - want) <= TOL[precision] * np.linalg.norm(dJdu) * np.linalg.norm(du)


def test_mass_apply_matches_oracle():
    import torch
    c = _case(650, 2)
    m = O.Mesh(c["origin"], c["extent"], c["n_el"], c["k"])
    v = np.random.default_rng(1).standard_normal(m.n_nodes())
    y = torch.zeros(m.n_nodes(), dtype=torch.float64, device="cuda:0")
    with cf.Context(c["origin"], c["extent"], c["n_el"], c["k"], c["params"]) as ctx:
        cf.cfdem_mass_apply(ctx.h, dev(v), y)
        cf.cfdem_synchronize(ctx.h)
    assert rel_err(host(y), O.kron_apply(m, 0.0, v)) <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_workload_loss_gradient(precision):
    """J = sum_i e_z . f_D,i + ||eps_h||_M (the loss of the adjoint workload)."""
    import torch
    c = _case(660, 2, n=50)
    m = O.Mesh(c["origin"], c["extent"], c["n_el"], c["k"])
    prm = dict(c["params"], precision=precision,
               cg_rtol=1e-13 if precision == 0 else 1e-12)
    n = c["x"].shape[0]
    g_fd = np.zeros((n, 3))
    g_fd[:, 2] = 1.0

    def g_eps(ctx, eps):
        Me = torch.zeros_like(eps)
        cf.cfdem_mass_apply(ctx.h, eps, Me)
        return Me / torch.sqrt(torch.dot(eps, Me))

    dJdx, dJdu, _ = _gpu(c, prm, None, g_fd, g_eps)
    rng = np.random.default_rng(11)
    for _ in range(3):
        dx = rng.standard_normal(c["x"].shape) * c["r"][:, None]
        du = rng.standard_normal(c["u_nodal"].shape)
        o = JV.coupling_jvp(m, prm, c["x"], c["r"], c["u_p"], c["u_nodal"], c["p_nodal"], dx, du)
        want = float(o["f_drag"].t[:, 2].sum()) + float(JV.mass_norm(m, o["eps_h"]).t)
        got = float(np.sum(dJdx * dx) + np.sum(dJdu * du))
        scale = (np.linalg.norm(dJdx) * np.linalg.norm(dx) +
                 np.linalg.norm(dJdu) * np.linalg.norm(du))
        assert abs(got - want) <= TOL[precision] * scale
    assert math.isfinite(float(np.abs(dJdx).max()))

"""The torch.autograd front end of the coupling step and its adjoint
(paper_2211_01185_gb300.autograd) on the sensitivity workload: a dense
annulus of 2 mm spheres around a sparse central column under a 2 m/s jet,
Q2 elements of 4 mm, loss J = sum_i e_z . f_D,i + ||eps_h||_M.

torch.autograd.grad of J with respect to the particle positions and the
nodal fluid velocities is compared with the derivative of the oracle's own
FP64 step along input directions (forward-mode dual numbers, oracle/jvp.py):
on a reduced bed (8 x 8 x 16 elements, 3,704 spheres, same layout) along
directions that move many particles, and on the full 24 x 24 x 96 bed of
200,000 spheres along directions that move a few particles in the annulus
and in the column.  The FP64 gradient is also checked against central
differences of the GPU's own forward step."""
import numpy as np
import pytest

from _parity import dev
from oracle import jvp as JV
from oracle import oracle as O
from paper_2211_01185_gb300 import autograd as AG
from paper_2211_01185_gb300 import cfdem as cf
from paper_2211_01185_gb300 import synth

pytestmark = pytest.mark.gpu

# |dJ(dx, du) - (g_x . dx + g_u . du)| <= TOL (|g_x| |dx| + |g_u| |du|)
TOL = {0: 1e-10, 1: 1e-5}

_BEDS = {}


def _bed(full):
    key = "full" if full else "small"
    if key not in _BEDS:
        _BEDS[key] = synth.make_adjoint_workload(n_el=(24, 24, 96) if full else (8, 8, 16))
    return _BEDS[key]


def _params(w, precision):
    return dict(w["params"], precision=precision, max_radius=float(w["r"].max()),
                cg_rtol=1e-13 if precision == 0 else 1e-12)


def _grads(w, precision):
    import torch
    with cf.Context(w["origin"], w["extent"], w["n_el"], w["k"], _params(w, precision)) as ctx:
        x = dev(w["x"]).requires_grad_()
        u = dev(w["u_nodal"]).requires_grad_()
        f, fd, eps, Fe = AG.coupling_step(ctx, x, dev(w["r"]), dev(w["u_p"]), u,
                                          dev(w["p_nodal"]))
        J = fd[:, 2].sum() + AG.mass_norm(ctx, eps)
        gx, gu = torch.autograd.grad(J, (x, u))
        assert not Fe.requires_grad
    return float(J.item()), gx.cpu().numpy(), gu.cpu().numpy()


def _oracle_dJ(w, prm, dx, du, sparse):
    m = O.Mesh(w["origin"], w["extent"], w["n_el"], w["k"])
    o = JV.coupling_jvp(m, prm, w["x"], w["r"], w["u_p"], w["u_nodal"], w["p_nodal"], dx, du,
                        sparse_qcm=sparse)
    J = float(o["f_drag"].v[:, 2].sum()) + float(JV.mass_norm(m, o["eps_h"]).v)
    dJ = float(o["f_drag"].t[:, 2].sum()) + float(JV.mass_norm(m, o["eps_h"]).t)
    return J, dJ


def _directions(w, rng, rows):
    dx = np.zeros_like(w["x"])
    dx[rows] = rng.standard_normal((len(rows), 3)) * w["r"][rows, None]
    du = rng.standard_normal(w["u_nodal"].shape) * 0.05
    return dx, du


def _check(w, precision, rows_list, sparse):
    J, gx, gu = _grads(w, precision)
    prm = _params(w, precision)
    rng = np.random.default_rng(17)
    for rows in rows_list:
        dx, du = _directions(w, rng, rows)
        J_ref, want = _oracle_dJ(w, prm, dx, du, sparse)
        got = float(np.sum(gx * dx) + np.sum(gu * du))
        scale = np.linalg.norm(gx) * np.linalg.norm(dx) + np.linalg.norm(gu) * np.linalg.norm(du)
        assert abs(got - want) <= TOL[precision] * scale, (got, want, scale)
        assert J == pytest.approx(J_ref, rel=TOL[precision])


@pytest.mark.parametrize("precision", [0, 1])
def test_autograd_reduced_bed(precision):
    w = _bed(False)
    n = w["x"].shape[0]
    rng = np.random.default_rng(3)
    rows = [rng.choice(n, 40, replace=False) for _ in range(3)]
    rows.append(np.array([0, 1, n - 1]))     # the floor of the annulus and the column's last
    _check(w, precision, rows, sparse=False)


@pytest.mark.parametrize("precision", [0, 1])
def test_autograd_full_bed(precision):
    """The 200,000-sphere bed: directions moving 8 spheres of the annulus and
    8 of the column (the column's spheres are the last ones)."""
    w = _bed(True)
    n = w["x"].shape[0]
    rng = np.random.default_rng(4)
    ann = rng.choice(n - 2000, 8, replace=False)
    col = n - 1 - rng.choice(500, 8, replace=False)
    _check(w, precision, [np.concatenate([ann, col]), ann[:2]], sparse=True)


def test_autograd_fp64_against_central_differences():
    """The FP64 gradient along one direction against (J(+h) - J(-h)) / 2h of
    the GPU's own forward step (h = 1e-6 of the sphere radius)."""
    import torch
    w = _bed(False)
    J0, gx, gu = _grads(w, 0)
    rng = np.random.default_rng(9)
    dx, du = _directions(w, rng, rng.choice(w["x"].shape[0], 25, replace=False))
    prm = _params(w, 0)

    def J_at(t):
        with cf.Context(w["origin"], w["extent"], w["n_el"], w["k"], prm) as ctx:
            f, fd, eps, _ = AG.coupling_step(ctx, dev(w["x"] + t * dx), dev(w["r"]),
                                             dev(w["u_p"]), dev(w["u_nodal"] + t * du),
                                             dev(w["p_nodal"]))
            with torch.no_grad():
                return float((fd[:, 2].sum() + AG.mass_norm(ctx, eps)).item())

    h = 1e-6
    fd_dJ = (J_at(h) - J_at(-h)) / (2 * h)
    got = float(np.sum(gx * dx) + np.sum(gu * du))
    assert got == pytest.approx(fd_dJ, rel=1e-6)


def test_autograd_refuses_gradients_it_does_not_give():
    import torch
    w = _bed(False)
    with cf.Context(w["origin"], w["extent"], w["n_el"], w["k"], _params(w, 0)) as ctx:
        x = dev(w["x"]).requires_grad_()
        r = dev(w["r"]).requires_grad_()
        f, fd, eps, _ = AG.coupling_step(ctx, x, r, dev(w["u_p"]), dev(w["u_nodal"]),
                                         dev(w["p_nodal"]))
        with pytest.raises(RuntimeError):
            torch.autograd.grad(fd.sum(), (x, r))

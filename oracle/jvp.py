"""Forward-mode derivatives of the coupling step for the oracle (test
infrastructure only: the tests may import it, nothing in the product does).

The adjoint of the coupling step -- gradients of a loss of the outputs
(forces f, drag forces f_D, projected void fraction eps_h) with respect to
the particle positions x and the nodal fluid velocities u -- has no
counterpart in the paper.  Its reference here is the directional derivative
of the same FP64 computation the oracle performs, taken in forward mode with
dual numbers: every quantity carries its value and its derivative along one
fixed direction (dx, du) of the inputs, and every elementary operation
propagates both by the chain rule.  Nothing here uses a closed-form
derivative of a model formula: the lens volume, the Lagrange basis, the
drag closures and the norms are differentiated by running
their defining expressions on dual numbers.

The pipeline follows the oracle step by step (oracle.py):
  1. quadrature-centred void fraction by brute force over all (Gauss point,
     particle) pairs with the piecewise lens volume -- neighbour sets are
     decided on values, so they are those of the primal;
  2. right-hand side b(eps_q) and the smoothed projection eps_h = A^-1 b are
     linear: value and derivative go through the oracle's rhs and its exact
     fast-diagonalisation solve separately;
  3. per-particle interpolation of u, eps_h and grad p at xi(x) with the
     tensor Lagrange basis built from its product formula, the void-fraction
     clamp of the closures, the drag closure, buoyancy and pressure force.
A one-sided point of a piecewise definition (clamp, lens branches) takes the
derivative of the branch its value selects.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

PI = O.PI


class Dual:
    """Value v and derivative t (same shape) along one input direction."""

    __array_priority__ = 100.0

    def __init__(self, v, t=None):
        self.v = np.asarray(v, dtype=np.float64)
        self.t = np.zeros_like(self.v) if t is None else np.broadcast_to(
            np.asarray(t, dtype=np.float64), self.v.shape).copy()

    # ---- structure
    def __getitem__(self, idx):
        return Dual(self.v[idx], self.t[idx])

    @property
    def shape(self):
        return self.v.shape

    def sum(self, axis=None):
        return Dual(self.v.sum(axis=axis), self.t.sum(axis=axis))

    # ---- arithmetic
    @staticmethod
    def lift(a):
        return a if isinstance(a, Dual) else Dual(a)

    def __add__(self, o):
        o = Dual.lift(o)
        return Dual(self.v + o.v, self.t + o.t)

    __radd__ = __add__

    def __sub__(self, o):
        o = Dual.lift(o)
        return Dual(self.v - o.v, self.t - o.t)

    def __rsub__(self, o):
        return Dual.lift(o) - self

    def __neg__(self):
        return Dual(-self.v, -self.t)

    def __mul__(self, o):
        o = Dual.lift(o)
        return Dual(self.v * o.v, self.t * o.v + self.v * o.t)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = Dual.lift(o)
        q = self.v / o.v
        return Dual(q, (self.t - q * o.t) / o.v)

    def __rtruediv__(self, o):
        return Dual.lift(o) / self


def sqrt(a):
    s = np.sqrt(a.v)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(s > 0, a.t / (2.0 * np.where(s > 0, s, 1.0)), 0.0)
    return Dual(s, t)


def exp(a):
    e = np.exp(a.v)
    return Dual(e, e * a.t)


def log(a):
    return Dual(np.log(a.v), a.t / a.v)


def log10(a):
    return Dual(np.log10(a.v), a.t / (a.v * np.log(10.0)))


def power(a, b):
    """a ** b for a > 0 (b may be a dual number)."""
    return exp(Dual.lift(b) * log(a))


def where(cond, a, b):
    a, b = Dual.lift(a), Dual.lift(b)
    return Dual(np.where(cond, a.v, b.v), np.where(cond, a.t, b.t))


def clamp(a, lo, hi):
    """min(max(a, lo), hi): outside [lo, hi] the value is a constant."""
    inside = (a.v >= lo) & (a.v <= hi)
    return Dual(np.clip(a.v, lo, hi), np.where(inside, a.t, 0.0))


# ------------------------------------------------------------------ pieces

def lens_volume(R, r, d):
    """Intersection volume of spheres of radii R, r at centre distance d
    (dual), d < R + r: the full smaller sphere for d <= |R - r|, else
    pi (R + r - d)^2 (d^2 + 2 d (R + r) - 3 (R - r)^2) / (12 d)."""
    s = (R + r) - d
    dm = R - r
    part = PI * s * s * (d * d + 2.0 * d * (R + r) - 3.0 * dm * dm) / (12.0 * d)
    mn = np.minimum(R, r)
    full = 4.0 / 3.0 * PI * mn ** 3
    return where(d.v <= np.abs(dm), full * np.ones_like(d.v), part)


def lagrange_basis(z, xi):
    """phi_a(xi) = prod_{b != a} (xi - z_b) / (z_a - z_b) and its derivative
    d phi_a / d xi, both dual, for the nodes z of one axis."""
    k = len(z) - 1
    phi, dphi = [], []
    for a in range(k + 1):
        p = Dual(np.ones_like(xi.v))
        for b in range(k + 1):
            if b != a:
                p = p * ((xi - z[b]) / (z[a] - z[b]))
        phi.append(p)
        dp = Dual(np.zeros_like(xi.v))
        for c in range(k + 1):
            if c == a:
                continue
            term = Dual(np.full_like(xi.v, 1.0 / (z[a] - z[c])))
            for b in range(k + 1):
                if b != a and b != c:
                    term = term * ((xi - z[b]) / (z[a] - z[b]))
            dp = dp + term
        dphi.append(dp)
    return phi, dphi


def lagrange_dd(z, xi):
    """d^2 phi_a / d xi^2 (dual) from the product formula differentiated
    twice: a sum over ordered pairs b != c of the other nodes."""
    k = len(z) - 1
    out = []
    for a in range(k + 1):
        s = Dual(np.zeros_like(xi.v))
        for b in range(k + 1):
            for c in range(k + 1):
                if b == a or c == a or b == c:
                    continue
                term = Dual(np.full_like(xi.v, 1.0 / ((z[a] - z[b]) * (z[a] - z[c]))))
                for m in range(k + 1):
                    if m not in (a, b, c):
                        term = term * ((xi - z[m]) / (z[a] - z[m]))
                s = s + term
        out.append(s)
    return out


def qcm_dual(mesh: O.Mesh, R, x: Dual, r):
    """eps_q[E*Q] (dual) by brute force over all pairs."""
    qp = O.quadrature_points(mesh).reshape(-1, 3)
    d2 = Dual(np.zeros((qp.shape[0], x.shape[0])))
    for a in range(3):
        da = Dual(x.v[None, :, a] - qp[:, None, a], np.broadcast_to(x.t[None, :, a], d2.shape))
        d2 = d2 + da * da
    c = R + np.asarray(r)[None, :]
    inside = d2.v < c * c
    d = sqrt(d2)
    V = lens_volume(R, np.asarray(r)[None, :] * np.ones_like(d.v), d)
    V = where(inside, V, 0.0)
    return 1.0 - V.sum(axis=1) / (4.0 / 3.0 * PI * R ** 3)


def qcm_dual_rows(mesh: O.Mesh, R, x, r, dx):
    """eps_q[E*Q] (dual) along a direction dx that moves few particles: the
    value from the C oracle's cell-list QCM, the tangent from the moved
    particles alone (the distances of every other pair do not change along
    dx), each by brute force over every Gauss point.  Equal to qcm_dual up
    to the order of the sums; usable on beds too large for all pairs."""
    x = np.asarray(x, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    e, _, _ = O.qcm(mesh, R, x, r)
    qp = O.quadrature_points(mesh).reshape(-1, 3)
    t = np.zeros(qp.shape[0])
    VR = 4.0 / 3.0 * PI * R ** 3
    for i in np.nonzero(np.any(np.asarray(dx) != 0.0, axis=1))[0]:
        d2 = Dual(np.zeros(qp.shape[0]))
        for a in range(3):
            da = Dual(x[i, a] - qp[:, a], np.full(qp.shape[0], dx[i, a]))
            d2 = d2 + da * da
        c = R + r[i]
        inside = d2.v < c * c
        d = sqrt(d2)
        V = where(inside, lens_volume(R, np.full(qp.shape[0], r[i]), d), 0.0)
        t -= V.t / VR
    return Dual(e.reshape(-1), t)


def _axis_locate(mesh, x, a):
    """element index (by value) and dual local coordinate along axis a"""
    h = mesh.h[a]
    s = (x.v[:, a] - mesh.origin[a]) / h
    ie = np.clip(np.floor(s).astype(np.int64), 0, int(mesh.n_el[a]) - 1)
    xi = Dual(s - ie, x.t[:, a] / h)
    return ie, xi


def _gnode(mesh, deg, ie, a, b, c):
    nx = int(mesh.n_el[0]) * deg + 1
    ny = int(mesh.n_el[1]) * deg + 1
    return (ie[0] * deg + a) + nx * ((ie[1] * deg + b) + ny * (ie[2] * deg + c))


def drag_coef(model, rho, mu, epsc: Dual, speed: Dual, r):
    """f_D = coef U for the closures of Sec. 2.3.2 (model numbers as in the
    C oracle's or_drag_force), with Re = rho eps |U| d / mu.  Written from
    the printed formulas (C_D = 24/Re (...), 10^(3 eps_p) Re^-s, ...);
    branches are chosen on values, both sides evaluated on safe inputs."""
    dp = 2.0 * r
    Re = rho * epsc * speed * dp / mu
    Vp = 4.0 / 3.0 * PI * r ** 3
    ep = 1.0 - epsc
    if model <= 2:
        a_ = 0.63 * sqrt(speed) + 4.8 * sqrt(mu / (rho * epsc * dp))
        cds = a_ * a_
        re = where(Re.v > 1e-300, Re, 1e-300)
        t = 1.5 - log10(re)
        g = exp(-(t * t) / 2.0)
        if model == 0:
            cds = cds * power(epsc, 2.0 - (3.7 - 0.65 * g))
        elif model == 2:
            cds = cds * power(epsc, 2.0 - (2.65 * (epsc + 1.0) - (5.3 - 3.5 * epsc) * epsc * epsc * g))
        return 0.5 * rho * cds * PI * r * r
    if model == 3:  # Koch-Hill, eps_p cancelled between beta and V_p / eps_p
        eps_s = where(ep.v > 0, ep, 1.0)
        plogp = where(ep.v > 0, eps_s * log(eps_s), 0.0)
        f0_dilute = (1.0 + 3.0 * sqrt(ep / 2.0) + 135.0 / 64.0 * plogp + 16.14 * ep) / \
            (1.0 + 0.681 * ep - 8.48 * ep * ep + 8.14 * ep * ep * ep)
        f0_dense = 10.0 * ep / (epsc * epsc * epsc)
        F0 = where(ep.v >= 0.4, f0_dense, f0_dilute)
        F3 = 0.0673 + 0.212 * ep + 0.0232 / power(epsc, 5.0)
        return 18.0 * mu * epsc * epsc / (dp * dp) * (F0 + 0.5 * F3 * Re) * Vp
    if model == 4:  # Gidaspow: beta V_p / eps_p with eps_p cancelled
        dense = 150.0 * ep * mu / (epsc * dp * dp) + 1.75 * rho * speed / dp
        re = where(Re.v > 0, Re, 1.0)
        cd = where(Re.v < 1000.0, 24.0 / re * (1.0 + 0.15 * power(re, 0.687)), 0.44)
        dilute = 0.75 * cd * epsc * speed * rho / dp * power(epsc, -2.65)
        return where(epsc.v < 0.8, dense, dilute) * Vp
    # Beetstra, the slip velocity for the printed u_f
    a_ = 10.0 * ep / (epsc * epsc) + epsc * epsc * (1.0 + 1.5 * sqrt(ep))
    re = where(Re.v > 0, Re, 1.0)
    num = 1.0 / epsc + 3.0 * ep * epsc + 8.4 * power(re, -0.343)
    den = 1.0 + power(Dual(10.0), 3.0 * ep) * power(re, -(1.0 + 4.0 * ep) / 2.0)
    F = a_ + where(Re.v > 0, 0.413 * Re / (24.0 * epsc * epsc) * num / den, 0.0)
    return 3.0 * PI * mu * dp * epsc * F


def forces_dual(mesh: O.Mesh, params: dict, x: Dual, r, u_p, u_nodal: Dual, p_nodal,
                eps_nodal: Dual):
    k = mesh.k
    kp = params.get("pressure_degree", 0) or max(1, k - 1)
    rho, mu = float(params["rho_f"]), float(params["mu_f"])
    grav = np.asarray(params.get("g", (0.0, 0.0, -9.81)), dtype=np.float64)
    floor = float(params.get("eps_floor", 0.05))
    model = int(params.get("drag_model", 0))
    boe = int(params.get("beta_over_eps", 0))
    r = np.asarray(r, dtype=np.float64)
    u_p = np.asarray(u_p, dtype=np.float64)
    p_nodal = np.asarray(p_nodal, dtype=np.float64)
    n = x.shape[0]
    ie, xi = [], []
    for a in range(3):
        e, s = _axis_locate(mesh, x, a)
        ie.append(e)
        xi.append(s)
    z = O.gll_nodes(k)
    zp = O.gll_nodes(kp)
    L = [lagrange_basis(z, xi[a])[0] for a in range(3)]
    P = [lagrange_basis(zp, xi[a]) for a in range(3)]
    uf = [Dual(np.zeros(n)) for _ in range(3)]
    eps = Dual(np.zeros(n))
    for c in range(k + 1):
        for b in range(k + 1):
            for a in range(k + 1):
                phi = L[0][a] * L[1][b] * L[2][c]
                nd = _gnode(mesh, k, ie, a, b, c)
                for comp in range(3):
                    uf[comp] = uf[comp] + phi * u_nodal[nd, comp]
                eps = eps + phi * eps_nodal[nd]
    gp = [Dual(np.zeros(n)) for _ in range(3)]
    for c in range(kp + 1):
        for b in range(kp + 1):
            for a in range(kp + 1):
                # the derivative along an axis from the nodal differences
                # along it (as the C oracle)
                pv = p_nodal[_gnode(mesh, kp, ie, a, b, c)]
                dx = pv - p_nodal[_gnode(mesh, kp, ie, 0, b, c)]
                dy = pv - p_nodal[_gnode(mesh, kp, ie, a, 0, c)]
                dz = pv - p_nodal[_gnode(mesh, kp, ie, a, b, 0)]
                gp[0] = gp[0] + P[0][1][a] / mesh.h[0] * P[1][0][b] * P[2][0][c] * dx
                gp[1] = gp[1] + P[0][0][a] * P[1][1][b] / mesh.h[1] * P[2][0][c] * dy
                gp[2] = gp[2] + P[0][0][a] * P[1][0][b] * P[2][1][c] / mesh.h[2] * dz
    epsc = clamp(eps, floor, 1.0)
    U = [uf[c] - u_p[:, c] for c in range(3)]
    speed = sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2])
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        coef = drag_coef(model, rho, mu, epsc, speed, r)
    if boe:
        coef = coef / epsc
    moving = speed.v > 0
    Vp = 4.0 / 3.0 * PI * r ** 3
    fd = [where(moving, coef * U[c], 0.0) for c in range(3)]
    fg = [-Vp * gp[c] for c in range(3)]
    f = [fd[c] + (-rho * Vp * grav[c]) + fg[c] for c in range(3)]
    stack = lambda parts: Dual(np.stack([p.v for p in parts], axis=1),  # noqa: E731
                               np.stack([p.t for p in parts], axis=1))
    out = {"f_drag": stack(fd), "f_gradp": stack(fg), "eps_p": eps}
    if params.get("shear_force", 0):
        # -V_p div tau, tau = mu (grad u + grad u^T) - 2/3 mu (div u) I:
        # (div tau)_a = mu lap u_a + mu/3 d_a div u, second derivatives of the
        # Q_k interpolant (chain rule 1/h per axis)
        D1 = [lagrange_basis(z, xi[a])[1] for a in range(3)]
        D2 = [lagrange_dd(z, xi[a]) for a in range(3)]
        H = [[[Dual(np.zeros(n)) for _ in range(3)] for _ in range(3)] for _ in range(3)]
        for c in range(k + 1):
            for b in range(k + 1):
                for a in range(k + 1):
                    nd = _gnode(mesh, k, ie, a, b, c)
                    idx = (a, b, c)
                    for p in range(3):
                        for q in range(p, 3):
                            w = 1.0
                            for ax in range(3):
                                order = (ax == p) + (ax == q)
                                basis = (L, D1, D2)[order][ax][idx[ax]]
                                w = basis * w if order == 0 else basis / mesh.h[ax] ** order * w
                            for comp in range(3):
                                H[comp][p][q] = H[comp][p][q] + w * u_nodal[nd, comp]
        for comp in range(3):
            for p in range(3):
                for q in range(p):
                    H[comp][p][q] = H[comp][q][p]
        fs = []
        for a in range(3):
            lap = H[a][0][0] + H[a][1][1] + H[a][2][2]
            graddiv = H[0][a][0] + H[1][a][1] + H[2][a][2]
            fs.append(-Vp * (mu * lap + (mu / 3.0) * graddiv))
        f = [f[c] + fs[c] for c in range(3)]
        out["f_shear"] = stack(fs)
    out["f"] = stack(f)
    return out


def coupling_jvp(mesh: O.Mesh, params: dict, x, r, u_p, u_nodal, p_nodal, dx=None, du=None,
                 sparse_qcm=False):
    """Outputs of the coupling step (eps_h, f, f_drag, f_gradp) as dual
    numbers: values and derivatives along the input direction (dx on the
    particle positions, du on the nodal fluid velocities).  sparse_qcm: the
    void fraction by qcm_dual_rows (for a dx that moves few particles of a
    large bed) instead of all pairs."""
    x = np.asarray(x, dtype=np.float64)
    u_nodal = np.asarray(u_nodal, dtype=np.float64)
    X = Dual(x, np.zeros_like(x) if dx is None else dx)
    Un = Dual(u_nodal, np.zeros_like(u_nodal) if du is None else du)
    L2 = float(params.get("l2_smoothing", 0.0))
    if params.get("scheme", 0) == 0:
        R = params.get("qcm_radius", 0.0) or O.default_qcm_radius(mesh)
        if sparse_qcm:
            eps_q = qcm_dual_rows(mesh, R, x, r, X.t)
        else:
            eps_q = qcm_dual(mesh, R, X, r)
    else:
        # the particle-centroid void fraction is piecewise constant in x
        e, _ = O.pcm(mesh, x, r)
        eps_q = Dual(e.reshape(-1))
    b = Dual(O.rhs(mesh, eps_q.v), O.rhs(mesh, eps_q.t))
    eps_h = Dual(O.fdm_solve(mesh, L2, b.v), O.fdm_solve(mesh, L2, b.t))
    out = forces_dual(mesh, params, X, r, u_p, Un, p_nodal, eps_h)
    out["eps_h"] = eps_h
    out["eps_q"] = eps_q
    return out


def mass_norm(mesh: O.Mesh, eps_h: Dual):
    """||eps_h||_M = sqrt(eps_h^T M eps_h) (M the consistent mass matrix)."""
    Mv = Dual(O.kron_apply(mesh, 0.0, eps_h.v), O.kron_apply(mesh, 0.0, eps_h.t))
    s = (eps_h * Mv).sum()
    return sqrt(s)

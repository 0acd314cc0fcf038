"""Python face of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It loads ``cfdem_oracle.c`` (compiled
with gcc, ``-O2 -ffp-contract=off``) through ctypes and adds two pieces that
are easier to state in numpy:

* ``fdm_solve`` -- the exact direct solve of the smoothed L2 projection by
  fast diagonalisation (Lynch, Rice & Thomas 1964): on an axis-aligned box of
  equal elements the operator is a Kronecker sum of assembled 1D mass and
  stiffness matrices, so the generalised 1D eigenproblems K v = lam M v
  diagonalise it.  Its 1D matrices are built here from numpy's polynomial
  tools, independently of the C element matrices, so CG (C) against FDM
  (numpy) checks both.
* ``qcm_bruteforce`` -- the quadrature-centred void fraction by brute force
  over all (quadrature point, particle) pairs for tiny inputs.

Readings of the paper that these functions fix (QCM averaging radius, the
L^2 smoothing operator, closures' void-fraction clamp, the sign of F_pf) are
stated at each function.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cfdem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PI = 3.14159265358979323846


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
            "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stdout=subprocess.DEVNULL,
                              stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp, ip, lp = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
            i64, dbl, cint = C.c_int64, C.c_double, C.c_int
            L.or_gauss_rule.argtypes = [cint, dp, dp]
            L.or_gll_nodes.argtypes = [cint, dp]
            L.or_lagrange.argtypes = [cint, dbl, dp, dp]
            L.or_lagrange_dd.argtypes = [cint, dbl, dp]
            L.or_shear_force.argtypes = [dp, dp, ip, cint, dbl, i64, dp, dp, dp, dp]
            L.or_shear_force.restype = i64
            L.or_locate.argtypes = [dp, dp, ip, cint, i64, dp, ip, dp]
            L.or_locate.restype = i64
            L.or_bin.argtypes = [dp, dp, ip, i64, dp, ip, ip, ip]
            L.or_lens_volume.argtypes = [dbl, dbl, dbl]
            L.or_lens_volume.restype = dbl
            L.or_qcm.argtypes = [dp, dp, ip, cint, dbl, i64, dp, dp, dp, cint, dp, ip, lp]
            L.or_qcm_weights.argtypes = [dp, dp, ip, cint, dbl, i64, dp, dp, dp]
            L.or_pcm.argtypes = [dp, dp, ip, cint, i64, dp, dp, dp]
            L.or_pcm.restype = i64
            L.or_element_matrix.argtypes = [cint, dp, dp, dp]
            L.or_rhs.argtypes = [dp, dp, ip, cint, dp, dp]
            L.or_apply.argtypes = [dp, dp, ip, cint, dbl, dp, dp]
            L.or_diag.argtypes = [dp, dp, ip, cint, dbl, dp]
            L.or_cg.argtypes = [dp, dp, ip, cint, dbl, dp, dp, dbl, cint, dp]
            L.or_cg.restype = cint
            L.or_cd_times_speed_dallavalle.argtypes = [dbl] * 5
            L.or_cd_times_speed_dallavalle.restype = dbl
            L.or_reynolds.argtypes = [dbl] * 5
            L.or_reynolds.restype = dbl
            L.or_difelice_chi.argtypes = [dbl]
            L.or_difelice_chi.restype = dbl
            L.or_drag_force.argtypes = [cint, cint, dbl, dbl, dbl, dp, dbl, dp]
            L.or_forces.argtypes = [dp, dp, ip, cint, cint, dbl, dbl, dp, cint, cint, dbl, i64,
                                    dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
            L.or_forces.restype = i64
            L.or_fluid_source.argtypes = [dp, dp, ip, cint, cint, i64, dp, dp, dp, dp, dp]
            L.or_fluid_source_semi.argtypes = [dp, dp, ip, cint, cint, i64, dp, dp, dp, dp, dp,
                                               dp, dp, dp]
            L.or_fluid_source_semi.restype = i64
            L.or_fluid_source.restype = i64
            L.or_locate_mapped.argtypes = [cint, i64, ip, dp, dbl, i64, dp, ip, dp]
            L.or_locate_mapped.restype = i64
            L.or_num_threads.restype = cint
            L.or_set_num_threads.argtypes = [cint]
            _lib = L
    return _lib


# ---------------------------------------------------------------- helpers

def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def _nullable(a, fn):
    if a is None:
        return None, None
    return fn(a)


class Mesh:
    """Axis-aligned box of equal hexahedra carrying a Q_k Lagrange space."""

    def __init__(self, origin, extent, n_el, k):
        self.origin = np.asarray(origin, dtype=np.float64)
        self.extent = np.asarray(extent, dtype=np.float64)
        self.n_el = np.asarray(n_el, dtype=np.int32)
        self.k = int(k)
        self.h = self.extent / self.n_el

    @property
    def n_elem(self):
        return int(np.prod(self.n_el))

    @property
    def nq(self):
        return self.k + 1

    @property
    def Q(self):
        return self.nq ** 3

    def n_nodes(self, deg=None):
        deg = self.k if deg is None else deg
        return int(np.prod(self.n_el * deg + 1))

    @property
    def elem_volume(self):
        return float(self.h[0] * self.h[1] * self.h[2])

    def args(self):
        o, po = _d(self.origin)
        e, pe = _d(self.extent)
        n, pn = _i(self.n_el)
        self._keep = (o, e, n)
        return po, pe, pn, self.k


# ---------------------------------------------------------------- 1D tables

def gauss_rule(n):
    p = np.zeros(n)
    w = np.zeros(n)
    _, pp = _d(p)
    lib().or_gauss_rule(n, p.ctypes.data_as(C.POINTER(C.c_double)),
                        w.ctypes.data_as(C.POINTER(C.c_double)))
    return p, w


def gll_nodes(k):
    z = np.zeros(k + 1)
    lib().or_gll_nodes(k, z.ctypes.data_as(C.POINTER(C.c_double)))
    return z


def lagrange(k, t):
    l = np.zeros(k + 1)
    dl = np.zeros(k + 1)
    lib().or_lagrange(k, float(t), l.ctypes.data_as(C.POINTER(C.c_double)),
                      dl.ctypes.data_as(C.POINTER(C.c_double)))
    return l, dl


def lagrange_dd(k, t):
    ddl = np.zeros(k + 1)
    lib().or_lagrange_dd(k, float(t), ddl.ctypes.data_as(C.POINTER(C.c_double)))
    return ddl


# ---------------------------------------------------------------- locate / bin

def locate(mesh: Mesh, x):
    x, px = _d(x)
    n = x.shape[0]
    elem = np.zeros(n, dtype=np.int32)
    xi = np.zeros((n, 3))
    bad = lib().or_locate(*mesh.args(), n, px, elem.ctypes.data_as(C.POINTER(C.c_int32)),
                          xi.ctypes.data_as(C.POINTER(C.c_double)))
    return elem, xi, int(bad)


def bin_particles(mesh: Mesh, nb, x):
    """Stable counting sort into nb[0] x nb[1] x nb[2] equal bins over the box."""
    x, px = _d(x)
    n = x.shape[0]
    nb_a, pnb = _i(np.asarray(nb))
    nbins = int(np.prod(nb_a))
    bin_of = np.zeros(n, dtype=np.int32)
    start = np.zeros(nbins + 1, dtype=np.int32)
    perm = np.zeros(n, dtype=np.int32)
    o, po = _d(mesh.origin)
    e, pe = _d(mesh.extent)
    ipt = C.POINTER(C.c_int32)
    lib().or_bin(po, pe, pnb, n, px, bin_of.ctypes.data_as(ipt), start.ctypes.data_as(ipt),
                 perm.ctypes.data_as(ipt))
    return bin_of, start, perm


# ---------------------------------------------------------------- void fraction

def lens_volume(R, r, d):
    return lib().or_lens_volume(float(R), float(r), float(d))


def default_qcm_radius(mesh: Mesh):
    """Averaging-sphere radius whose volume equals the element volume
    (reading of the quadrature-centred scheme: R = (3 V_e / 4 pi)^(1/3))."""
    return (3.0 * mesh.elem_volume / (4.0 * PI)) ** (1.0 / 3.0)


def qcm_weights(mesh: Mesh, R, x, r):
    """Per-particle scaling c_i = V_p,i / S_i of the volume-conserving QCM."""
    x, px = _d(x)
    r, pr = _d(r)
    c = np.zeros(x.shape[0])
    lib().or_qcm_weights(*mesh.args(), float(R), x.shape[0], px, pr,
                         c.ctypes.data_as(C.POINTER(C.c_double)))
    return c


def qcm(mesh: Mesh, R, x, r, brute=False, want_lists=False, conserve=False):
    """Quadrature-centred void fraction eps_q[E][Q]; also neighbour counts
    and id sums per quadrature point.  conserve: lens volumes scaled per
    particle by qcm_weights."""
    x, px = _d(x)
    r, pr = _d(r)
    n = x.shape[0]
    E, Q = mesh.n_elem, mesh.Q
    eps = np.zeros(E * Q)
    cnt = np.zeros(E * Q, dtype=np.int32)
    ids = np.zeros(E * Q, dtype=np.int64)
    cw = qcm_weights(mesh, R, x, r) if conserve else None
    pcw = None if cw is None else cw.ctypes.data_as(C.POINTER(C.c_double))
    lib().or_qcm(*mesh.args(), float(R), n, px, pr, pcw, int(bool(brute)),
                 eps.ctypes.data_as(C.POINTER(C.c_double)),
                 cnt.ctypes.data_as(C.POINTER(C.c_int32)),
                 ids.ctypes.data_as(C.POINTER(C.c_int64)))
    return eps.reshape(E, Q), cnt.reshape(E, Q), ids.reshape(E, Q)


def pcm(mesh: Mesh, x, r):
    x, px = _d(x)
    r, pr = _d(r)
    n = x.shape[0]
    eps = np.zeros(mesh.n_elem * mesh.Q)
    bad = lib().or_pcm(*mesh.args(), n, px, pr, eps.ctypes.data_as(C.POINTER(C.c_double)))
    return eps.reshape(mesh.n_elem, mesh.Q), int(bad)


def quadrature_points(mesh: Mesh):
    """Physical coordinates of the Gauss points, [E][Q][3], in the same
    arithmetic order as the oracle's predicate (x0 + h (e + g))."""
    g, _ = gauss_rule(mesh.nq)
    nx, ny, nz = (int(v) for v in mesh.n_el)
    ex = np.arange(nx)
    coords = []
    for a, ne in enumerate((nx, ny, nz)):
        t = (np.arange(ne)[:, None].astype(np.float64) + g[None, :])
        coords.append(mesh.origin[a] + mesh.h[a] * t)      # [ne][nq]
    X, Y, Z = coords
    E, nq = mesh.n_elem, mesh.nq
    out = np.zeros((nz, ny, nx, nq, nq, nq, 3))
    out[..., 0] = X[None, None, :, None, None, :]
    out[..., 1] = Y[None, :, None, None, :, None]
    out[..., 2] = Z[:, None, None, :, None, None]
    del ex
    return out.reshape(E, nq ** 3, 3)


def qcm_bruteforce(mesh: Mesh, R, x, r):
    """Vectorised brute force for tiny inputs: every (quadrature point,
    particle) pair, lens volume evaluated by the piecewise formula in numpy."""
    x = np.asarray(x, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    qp = quadrature_points(mesh).reshape(-1, 3)
    dx = x[None, :, 0] - qp[:, None, 0]
    dy = x[None, :, 1] - qp[:, None, 1]
    dz = x[None, :, 2] - qp[:, None, 2]
    d2 = dx * dx + dy * dy + dz * dz
    c = R + r[None, :]
    inside = d2 < c * c
    d = np.sqrt(d2)
    mn = np.minimum(R, r)[None, :] * np.ones_like(d)
    s = R + r[None, :] - d
    dm = R - r[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        part = PI * s * s * (d * d + 2.0 * d * (R + r[None, :]) - 3.0 * dm * dm) / (12.0 * d)
    full = 4.0 / 3.0 * PI * mn ** 3
    v = np.where(d <= np.abs(dm), full, part)
    v = np.where(inside, v, 0.0)
    eps = 1.0 - v.sum(axis=1) / (4.0 / 3.0 * PI * R ** 3)
    cnt = inside.sum(axis=1).astype(np.int32)
    ids = (inside * np.arange(x.shape[0])[None, :]).sum(axis=1).astype(np.int64)
    E, Q = mesh.n_elem, mesh.Q
    return eps.reshape(E, Q), cnt.reshape(E, Q), ids.reshape(E, Q)


# ---------------------------------------------------------------- projection

def element_matrices(k, h):
    nloc = (k + 1) ** 3
    hh, ph = _d(np.asarray(h))
    Me = np.zeros(nloc * nloc)
    Ke = np.zeros(nloc * nloc)
    lib().or_element_matrix(k, ph, Me.ctypes.data_as(C.POINTER(C.c_double)),
                            Ke.ctypes.data_as(C.POINTER(C.c_double)))
    return Me.reshape(nloc, nloc), Ke.reshape(nloc, nloc)


def rhs(mesh: Mesh, eps_q):
    e, pe = _d(np.asarray(eps_q).reshape(-1))
    b = np.zeros(mesh.n_nodes())
    lib().or_rhs(*mesh.args(), pe, b.ctypes.data_as(C.POINTER(C.c_double)))
    return b


def apply(mesh: Mesh, L2, xv):
    xv, px = _d(xv)
    y = np.zeros(mesh.n_nodes())
    lib().or_apply(*mesh.args(), float(L2), px, y.ctypes.data_as(C.POINTER(C.c_double)))
    return y


def diag(mesh: Mesh, L2):
    dg = np.zeros(mesh.n_nodes())
    lib().or_diag(*mesh.args(), float(L2), dg.ctypes.data_as(C.POINTER(C.c_double)))
    return dg


def cg(mesh: Mesh, L2, b, x0=None, rtol=1e-14, maxit=20000):
    b, pb = _d(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    res = C.c_double(0.0)
    it = lib().or_cg(*mesh.args(), float(L2), pb, x.ctypes.data_as(C.POINTER(C.c_double)),
                     float(rtol), int(maxit), C.byref(res))
    return x, int(it), float(res.value)


def _ref_1d(k):
    """1D reference mass and stiffness on [0,1] built with numpy: Lagrange
    basis on the GLL nodes (roots of P_k' plus the end points) integrated by
    numpy's Gauss-Legendre rule with k+1 points."""
    from numpy.polynomial import legendre as Lg
    if k == 1:
        s = np.array([-1.0, 1.0])
    else:
        inner = Lg.Legendre.basis(k).deriv().roots()
        s = np.concatenate([[-1.0], np.sort(inner.real), [1.0]])
    z = 0.5 * (s + 1.0)
    V = np.vander(z, k + 1, increasing=True)
    coef = np.linalg.inv(V)                  # column a: monomial coefficients of l_a
    gs, gw = Lg.leggauss(k + 1)
    g = 0.5 * (gs + 1.0)
    w = 0.5 * gw
    P = np.vander(g, k + 1, increasing=True) @ coef          # [q][a] l_a(g_q)
    dV = np.zeros_like(P)
    for j in range(1, k + 1):
        dV += j * np.outer(g ** (j - 1), coef[j, :])
    Mh = (P * w[:, None]).T @ P
    Kh = (dV * w[:, None]).T @ dV
    return Mh, Kh


def _assemble_1d(Mh, n_el, k):
    n = n_el * k + 1
    A = np.zeros((n, n))
    for e in range(n_el):
        A[e * k:e * k + k + 1, e * k:e * k + k + 1] += Mh
    return A


def fdm_solve(mesh: Mesh, L2, b):
    """Exact solve of (M + L2 K) x = b by fast diagonalisation.

    With assembled 1D reference matrices M_a, K_a (unit element length) the
    operator is hx hy hz Mz(x)My(x)Mx + L2 [ (hy hz/hx) Mz(x)My(x)Kx + ... ]
    in the node order ix fastest.  Generalised eigenvectors V_a with
    V_a^T M_a V_a = I, V_a^T K_a V_a = diag(lam_a) give
    A^{-1} = (V (x) V (x) V) D^{-1} (V (x) V (x) V)^T."""
    import scipy.linalg as sl
    k = mesh.k
    Mh, Kh = _ref_1d(k)
    lam, Vs = [], []
    for a in range(3):
        Ma = _assemble_1d(Mh, int(mesh.n_el[a]), k)
        Ka = _assemble_1d(Kh, int(mesh.n_el[a]), k)
        w, V = sl.eigh(Ka, Ma)
        lam.append(w)
        Vs.append(V)
    hx, hy, hz = (float(v) for v in mesh.h)
    nx, ny, nz = (int(v) * k + 1 for v in mesh.n_el)
    B = np.asarray(b, dtype=np.float64).reshape(nz, ny, nx)
    T = np.einsum("zyx,xi->zyi", B, Vs[0])
    T = np.einsum("zyi,yj->zji", T, Vs[1])
    T = np.einsum("zji,zk->kji", T, Vs[2])
    D = (hx * hy * hz
         + L2 * ((hy * hz / hx) * lam[0][None, None, :]
                 + (hx * hz / hy) * lam[1][None, :, None]
                 + (hx * hy / hz) * lam[2][:, None, None]))
    T = T / D
    T = np.einsum("kji,zk->zji", T, Vs[2])
    T = np.einsum("zji,yj->zyi", T, Vs[1])
    T = np.einsum("zyi,xi->zyx", T, Vs[0])
    return T.reshape(-1)


def kron_apply(mesh: Mesh, L2, xv):
    """y = A x with A the Kronecker-sum form used by fdm_solve (numpy)."""
    k = mesh.k
    Mh, Kh = _ref_1d(k)
    Ms = [_assemble_1d(Mh, int(mesh.n_el[a]), k) for a in range(3)]
    Ks = [_assemble_1d(Kh, int(mesh.n_el[a]), k) for a in range(3)]
    hx, hy, hz = (float(v) for v in mesh.h)
    nx, ny, nz = (int(v) * k + 1 for v in mesh.n_el)
    X = np.asarray(xv, dtype=np.float64).reshape(nz, ny, nx)

    def ap(Az, Ay, Ax):
        T = np.einsum("zyx,ix->zyi", X, Ax)
        T = np.einsum("zyi,jy->zji", T, Ay)
        return np.einsum("zji,kz->kji", T, Az)
    y = hx * hy * hz * ap(Ms[2], Ms[1], Ms[0])
    y = y + L2 * ((hy * hz / hx) * ap(Ms[2], Ms[1], Ks[0])
                  + (hx * hz / hy) * ap(Ms[2], Ks[1], Ms[0])
                  + (hx * hy / hz) * ap(Ks[2], Ms[1], Ms[0]))
    return y.reshape(-1)


def node_coords(mesh: Mesh, deg=None):
    """Coordinates of the Q_deg nodes [n_nodes][3], ix fastest."""
    deg = mesh.k if deg is None else deg
    z = gll_nodes(deg)
    axes = []
    for a in range(3):
        ne = int(mesh.n_el[a])
        t = (np.arange(ne)[:, None] + z[None, :-1]).reshape(-1)
        t = np.concatenate([t, [float(ne)]])
        axes.append(mesh.origin[a] + mesh.h[a] * t)
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)


# ---------------------------------------------------------------- forces

def cd_times_speed_dallavalle(rho, mu, eps, speed, dp):
    return lib().or_cd_times_speed_dallavalle(rho, mu, eps, speed, dp)


def reynolds(rho, mu, eps, speed, dp):
    return lib().or_reynolds(rho, mu, eps, speed, dp)


def difelice_chi(Re):
    return lib().or_difelice_chi(Re)


def drag_force(model, beta_over_eps, rho, mu, eps, U, rp):
    U, pU = _d(U)
    f = np.zeros(3)
    lib().or_drag_force(int(model), int(beta_over_eps), rho, mu, eps, pU, rp,
                        f.ctypes.data_as(C.POINTER(C.c_double)))
    return f


def forces(mesh: Mesh, params: dict, x, r, u_p, u_nodal, p_nodal, eps_nodal):
    """Per-particle forces; returns dict with f, f_drag, f_gradp, eps_p and
    the first out-of-domain index (or -1)."""
    kp = params.get("pressure_degree", 0) or max(1, mesh.k - 1)
    x, px = _d(x)
    r, pr = _d(r)
    up, pup = _d(u_p)
    un, pun = _d(u_nodal)
    pn, ppn = _d(p_nodal)
    en, pen = _d(eps_nodal)
    g, pg = _d(np.asarray(params.get("g", (0.0, 0.0, -9.81))))
    n = x.shape[0]
    f = np.zeros((n, 3))
    fd = np.zeros((n, 3))
    fg = np.zeros((n, 3))
    ep = np.zeros(n)
    dp = C.POINTER(C.c_double)
    bad = lib().or_forces(*mesh.args(), int(kp), float(params["rho_f"]), float(params["mu_f"]),
                          pg, int(params.get("drag_model", 0)),
                          int(params.get("beta_over_eps", 0)),
                          float(params.get("eps_floor", 0.05)), n, px, pr, pup, pun, ppn, pen,
                          f.ctypes.data_as(dp), fd.ctypes.data_as(dp), fg.ctypes.data_as(dp),
                          ep.ctypes.data_as(dp))
    out = {"f": f, "f_drag": fd, "f_gradp": fg, "eps_p": ep, "bad": int(bad)}
    if params.get("shear_force", 0):
        fs, _ = shear_force(mesh, float(params["mu_f"]), x, r, u_nodal)
        out["f"] = f + fs
        out["f_shear"] = fs
    return out


def shear_force(mesh: Mesh, mu, x, r, u_nodal):
    """-V_p div tau per particle (deviatoric stress of Eq. (stress))."""
    x, px = _d(x)
    r, pr = _d(r)
    un, pun = _d(u_nodal)
    f = np.zeros((x.shape[0], 3))
    bad = lib().or_shear_force(*mesh.args(), float(mu), x.shape[0], px, pr, pun,
                               f.ctypes.data_as(C.POINTER(C.c_double)))
    return f, int(bad)


def fluid_source(mesh: Mesh, vans_model, x, f_drag, f_gradp, f_shear=None):
    x, px = _d(x)
    fd, pfd = _d(f_drag)
    fg, pfg = _d(f_gradp)
    if f_shear is not None:
        fs, pfs = _d(f_shear)
    else:
        pfs = None
    F = np.zeros((mesh.n_elem, 3))
    bad = lib().or_fluid_source(*mesh.args(), int(vans_model), x.shape[0], px, pfd, pfg, pfs,
                                F.ctypes.data_as(C.POINTER(C.c_double)))
    return F, int(bad)


def fluid_source_semi(mesh: Mesh, vans_model, x, u_p, u_nodal, f_drag, f_gradp, f_shear=None):
    """Fluid source with the fluid-side drag -beta_e (u_f(x_q) - u_p,avg,e):
    (F_q [E][Q][3], F_e [E][3] the element mean, first out-of-domain index)."""
    x, px = _d(x)
    up, pup = _d(u_p)
    un, pun = _d(u_nodal)
    fd, pfd = _d(f_drag)
    fg, pfg = _d(f_gradp)
    if f_shear is not None:
        fs, pfs = _d(f_shear)
    else:
        pfs = None
    Fq = np.zeros((mesh.n_elem, mesh.Q, 3))
    Fe = np.zeros((mesh.n_elem, 3))
    dp = C.POINTER(C.c_double)
    bad = lib().or_fluid_source_semi(*mesh.args(), int(vans_model), x.shape[0], px, pup, pun,
                                     pfd, pfg, pfs, Fq.ctypes.data_as(dp), Fe.ctypes.data_as(dp))
    return Fq, Fe, int(bad)


def coupling_step(mesh: Mesh, params: dict, x, r, u_p, u_nodal, p_nodal, eps0=None):
    """The whole coupling step in FP64: void fraction (QCM or PCM), smoothed
    projection (Jacobi-PCG), forces and fluid source."""
    R = params.get("qcm_radius", 0.0) or default_qcm_radius(mesh)
    if params.get("scheme", 0) == 0:
        eps_q, _, _ = qcm(mesh, R, x, r, conserve=bool(params.get("qcm_conserve", 0)))
    else:
        eps_q, _ = pcm(mesh, x, r)
    b = rhs(mesh, eps_q)
    L2 = float(params.get("l2_smoothing", 0.0))
    eps_h, it, res = cg(mesh, L2, b, x0=eps0, rtol=float(params.get("oracle_rtol", 1e-14)))
    fo = forces(mesh, params, x, r, u_p, u_nodal, p_nodal, eps_h)
    vans = int(params.get("vans_model", 0))
    out = {"eps_q": eps_q, "b": b, "eps_h": eps_h, "cg_iters": it, "cg_relres": res, **fo}
    if params.get("fluid_drag", 0):
        out["F_q"], out["F_e"], _ = fluid_source_semi(mesh, vans, x, u_p, u_nodal, fo["f_drag"],
                                                       fo["f_gradp"], fo.get("f_shear"))
    else:
        out["F_e"], _ = fluid_source(mesh, vans, x, fo["f_drag"], fo["f_gradp"], fo.get("f_shear"))
    return out


def locate_mapped(k, conn, nodes, x, margin=0.1):
    """Element and reference coordinates of each point on a mapped Q_k hex
    mesh (conn[E][(k+1)^3] node indices, a fastest; nodes[N][3]) by Newton
    inversion of the element maps (see or_locate_mapped); returns (elem,
    xi, number of points in no element)."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    nodes, pn = _d(nodes)
    x, px = _d(x)
    n = x.shape[0]
    elem = np.zeros(n, dtype=np.int32)
    xi = np.zeros((n, 3))
    miss = lib().or_locate_mapped(int(k), conn.shape[0], conn.ctypes.data_as(C.POINTER(C.c_int32)),
                                  pn, float(margin), n, px,
                                  elem.ctypes.data_as(C.POINTER(C.c_int32)),
                                  xi.ctypes.data_as(C.POINTER(C.c_double)))
    return elem, xi, int(miss)


def num_threads():
    return lib().or_num_threads()


def set_num_threads(t):
    lib().or_set_num_threads(int(t))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))

"""Thin ctypes binding of the C ABI in ``include/cfdem.h``.

Argument marshalling only: every step of the coupling path runs in the CUDA
library ``_lib/libcfdem.so``.  Functions keep the C names; device buffers are
passed as integer addresses (``tensor.data_ptr()``), so PyTorch serves only
as the device allocator and stream provider.  There is no CPU fallback: if
the library is missing the import of any entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcfdem.so")
HEADER = os.path.join(_HERE, "..", "include", "cfdem.h")

OK = 0
EINVAL = -1
OUT_OF_DOMAIN = -2
NOT_CONVERGED = -3
ENOMEM = -4
ECUDA = -5
ESTATE = -6
ECAPACITY = -7
STATUS_NAMES = {0: "CFDEM_OK", -1: "CFDEM_EINVAL", -2: "CFDEM_OUT_OF_DOMAIN",
                -3: "CFDEM_NOT_CONVERGED", -4: "CFDEM_ENOMEM", -5: "CFDEM_ECUDA",
                -6: "CFDEM_ESTATE", -7: "CFDEM_ECAPACITY"}


class cfdem_dem_params(C.Structure):
    _fields_ = [("rho_p", C.c_double), ("youngs", C.c_double), ("poisson", C.c_double),
                ("restitution", C.c_double), ("friction", C.c_double),
                ("rolling_friction", C.c_double), ("wall_youngs", C.c_double),
                ("wall_poisson", C.c_double), ("wall_restitution", C.c_double),
                ("wall_friction", C.c_double), ("wall_rolling_friction", C.c_double),
                ("g", C.c_double * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("max_radius", C.c_double), ("capacity", C.c_int), ("precision", C.c_int)]


class cfdem_params(C.Structure):
    _fields_ = [("rho_f", C.c_double), ("mu_f", C.c_double), ("g", C.c_double * 3),
                ("scheme", C.c_int), ("qcm_radius", C.c_double), ("l2_smoothing", C.c_double),
                ("drag_model", C.c_int), ("vans_model", C.c_int), ("beta_over_eps", C.c_int),
                ("precision", C.c_int), ("cg_rtol", C.c_double), ("cg_maxit", C.c_int),
                ("eps_floor", C.c_double), ("pressure_degree", C.c_int),
                ("max_radius", C.c_double), ("bin_edge", C.c_double),
                ("cg_precond", C.c_int), ("shear_force", C.c_int), ("fluid_drag", C.c_int),
                ("qcm_conserve", C.c_int), ("autotune", C.c_int)]


class cfdem_stats(C.Structure):
    _fields_ = [("first_bad_particle", C.c_int64), ("cg_iterations", C.c_int32),
                ("cg_outer", C.c_int32), ("cg_relres", C.c_double), ("converged", C.c_int32),
                ("nb", C.c_int32 * 3), ("bin_edge", C.c_double * 3), ("qcm_radius", C.c_double),
                ("n_elem", C.c_int64), ("n_qp", C.c_int64), ("n_nodes", C.c_int64),
                ("n_pnodes", C.c_int64), ("stage_ms", C.c_double * 8),
                ("stage_calls", C.c_int64 * 8), ("timer_overflow", C.c_int32),
                ("kernel_launches", C.c_int64), ("precond", C.c_int32),
                ("tile_shape", C.c_int32), ("tuned", C.c_int32), ("tune_ms", C.c_double),
                ("fdm_tile", C.c_int32)]

class cfdem_bed_io(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("r", C.c_void_p), ("u_p", C.c_void_p),
                ("u_nodal", C.c_void_p), ("p_nodal", C.c_void_p), ("eps_nodal", C.c_void_p),
                ("f", C.c_void_p), ("f_drag", C.c_void_p), ("F_elem", C.c_void_p),
                ("F_q", C.c_void_p), ("host_x", C.c_void_p), ("host_r", C.c_void_p),
                ("host_u_p", C.c_void_p), ("host_u_nodal", C.c_void_p),
                ("host_p_nodal", C.c_void_p), ("host_f", C.c_void_p),
                ("host_F_elem", C.c_void_p)]


STAGES = ("bin", "void_fraction", "rhs", "solve", "forces", "fluid_source", "op32", "op64")


_lib = None


def header_functions():
    """Names of the functions that include/cfdem.h declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(cfdem_\w+)\s*\(", txt, re.M)))


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libcfdem.so is not built (run __graft_entry__.build() or "
                           "python -m paper_2211_01185_gb300.build)")
    try:  # share PyTorch's CUDA runtime when it is loaded
        import torch  # noqa: F401
    except Exception:  # pragma: no cover
        pass
    L = C.CDLL(LIB_PATH)
    vp, i64, dbl, cint = C.c_void_p, C.c_int64, C.c_double, C.c_int
    d3 = C.POINTER(C.c_double)
    L.cfdem_version.restype = C.c_char_p
    L.cfdem_create.argtypes = [C.POINTER(vp), cint, vp]
    L.cfdem_destroy.argtypes = [vp]
    L.cfdem_params_default.argtypes = [C.POINTER(cfdem_params)]
    L.cfdem_params_default.restype = None
    L.cfdem_set_mesh.argtypes = [vp, d3, d3, C.POINTER(cint), cint]
    L.cfdem_set_params.argtypes = [vp, C.POINTER(cfdem_params)]
    L.cfdem_get_params.argtypes = [vp, C.POINTER(cfdem_params)]
    L.cfdem_locate.argtypes = [vp, i64, vp, vp, vp]
    L.cfdem_bin.argtypes = [vp, i64, vp, vp, vp]
    L.cfdem_void_fraction.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    L.cfdem_project_rhs.argtypes = [vp, vp, vp]
    L.cfdem_apply.argtypes = [vp, vp, vp]
    L.cfdem_project.argtypes = [vp, vp, vp]
    L.cfdem_forces.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.cfdem_fluid_drag_coefficients.argtypes = [vp, vp, vp]
    L.cfdem_dem_params_default.argtypes = [C.POINTER(cfdem_dem_params)]
    L.cfdem_dem_params_default.restype = None
    L.cfdem_dem_create.argtypes = [C.POINTER(vp), C.c_int, vp]
    L.cfdem_dem_destroy.argtypes = [vp]
    L.cfdem_dem_set_params.argtypes = [vp, C.POINTER(cfdem_dem_params)]
    L.cfdem_dem_reset.argtypes = [vp]
    L.cfdem_dem_step.argtypes = [vp, i64, vp, vp, vp, vp, vp, C.c_double, C.c_int]
    L.cfdem_dem_synchronize.argtypes = [vp]
    L.cfdem_dem_last_error.argtypes = [vp]
    L.cfdem_dem_last_error.restype = C.c_char_p
    L.cfdem_coupling_step.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.cfdem_synchronize.argtypes = [vp]
    L.cfdem_get_stats.argtypes = [vp, C.POINTER(cfdem_stats)]
    L.cfdem_set_timing.argtypes = [vp, cint]
    L.cfdem_pcm_void_fraction_static.argtypes = [d3, d3, C.POINTER(cint), cint, i64, vp, vp, vp,
                                                 vp]
    L.cfdem_adjoint.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.cfdem_mass_apply.argtypes = [vp, vp, vp]
    L.cfdem_batch_create.argtypes = [C.POINTER(vp), cint, vp, cint]
    L.cfdem_batch_destroy.argtypes = [vp]
    L.cfdem_batch_bed.argtypes = [vp, cint]
    L.cfdem_batch_bed.restype = vp
    L.cfdem_batch_set_graph.argtypes = [vp, cint]
    L.cfdem_batch_coupling_step.argtypes = [vp, C.POINTER(cfdem_bed_io)]
    L.cfdem_batch_synchronize.argtypes = [vp, C.POINTER(cint)]
    L.cfdem_batch_last_replayed.argtypes = [vp]
    L.cfdem_batch_last_error.argtypes = [vp]
    L.cfdem_batch_last_error.restype = C.c_char_p
    L.cfdem_mapped_create.argtypes = [C.POINTER(vp), cint, cint, i64, vp, i64, vp, dbl]
    L.cfdem_mapped_destroy.argtypes = [vp]
    L.cfdem_mapped_locate.argtypes = [vp, i64, vp, vp, vp, vp]
    L.cfdem_mapped_interpolate.argtypes = [vp, i64, vp, vp, cint, vp, vp, vp]
    L.cfdem_last_error.argtypes = [vp]
    L.cfdem_last_error.restype = C.c_char_p
    _lib = L
    return L


class CfdemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(int(t.data_ptr()) if hasattr(t, "data_ptr") else int(t))


def _check(h, st):
    if st != OK:
        raise CfdemError(st, lib().cfdem_last_error(h).decode())
    return st


# ------------------------------------------------------------------ C names

def cfdem_version():
    return lib().cfdem_version().decode()


def cfdem_params_default():
    p = cfdem_params()
    lib().cfdem_params_default(C.byref(p))
    return p


def cfdem_create(device=0, stream=None):
    h = C.c_void_p()
    st = lib().cfdem_create(C.byref(h), int(device), C.c_void_p(stream or 0))
    if st != OK:
        raise CfdemError(st, "cfdem_create failed")
    return h


def cfdem_destroy(h):
    return lib().cfdem_destroy(h)


def cfdem_set_mesh(h, origin, extent, n_el, degree):
    o = (C.c_double * 3)(*[float(v) for v in origin])
    e = (C.c_double * 3)(*[float(v) for v in extent])
    n = (C.c_int * 3)(*[int(v) for v in n_el])
    return _check(h, lib().cfdem_set_mesh(h, o, e, n, int(degree)))


def cfdem_set_params(h, p):
    return _check(h, lib().cfdem_set_params(h, C.byref(p)))


def cfdem_get_params(h):
    p = cfdem_params()
    _check(h, lib().cfdem_get_params(h, C.byref(p)))
    return p


def cfdem_locate(h, n, x, elem, xi):
    return _check(h, lib().cfdem_locate(h, int(n), _ptr(x), _ptr(elem), _ptr(xi)))


def cfdem_bin(h, n, x, bin_start, perm):
    return _check(h, lib().cfdem_bin(h, int(n), _ptr(x), _ptr(bin_start), _ptr(perm)))


def cfdem_void_fraction(h, n, x, r, eps_q=None, nb_count=None, nb_idsum=None):
    return _check(h, lib().cfdem_void_fraction(h, int(n), _ptr(x), _ptr(r), _ptr(eps_q),
                                               _ptr(nb_count), _ptr(nb_idsum)))


def cfdem_project_rhs(h, eps_q, b):
    return _check(h, lib().cfdem_project_rhs(h, _ptr(eps_q), _ptr(b)))


def cfdem_apply(h, x, y):
    return _check(h, lib().cfdem_apply(h, _ptr(x), _ptr(y)))


def cfdem_project(h, eps_q, eps_nodal):
    return _check(h, lib().cfdem_project(h, _ptr(eps_q), _ptr(eps_nodal)))


def cfdem_forces(h, n, x, r, u_p, u_nodal, p_nodal, eps_nodal, f, f_drag=None, F_elem=None,
                 F_q=None):
    return _check(h, lib().cfdem_forces(h, int(n), _ptr(x), _ptr(r), _ptr(u_p), _ptr(u_nodal),
                                        _ptr(p_nodal), _ptr(eps_nodal), _ptr(f), _ptr(f_drag),
                                        _ptr(F_elem), _ptr(F_q)))


def cfdem_fluid_drag_coefficients(h, beta_e=None, up_avg=None):
    return _check(h, lib().cfdem_fluid_drag_coefficients(h, _ptr(beta_e), _ptr(up_avg)))


def cfdem_coupling_step(h, n, x, r, u_p, u_nodal, p_nodal, eps_nodal, f, f_drag=None,
                        F_elem=None, F_q=None):
    return _check(h, lib().cfdem_coupling_step(h, int(n), _ptr(x), _ptr(r), _ptr(u_p),
                                               _ptr(u_nodal), _ptr(p_nodal), _ptr(eps_nodal),
                                               _ptr(f), _ptr(f_drag), _ptr(F_elem), _ptr(F_q)))


def cfdem_synchronize(h, raise_on_error=True):
    st = lib().cfdem_synchronize(h)
    if raise_on_error:
        _check(h, st)
    return st


def cfdem_get_stats(h):
    s = cfdem_stats()
    _check(h, lib().cfdem_get_stats(h, C.byref(s)))
    return s


PCM_STATIC_MAX_ELEMS = 524288


def cfdem_pcm_void_fraction_static(origin, extent, n_el, degree, n, x, r, eps_q, stream=None):
    """Particle-centroid void fraction without any device allocation (see
    include/cfdem.h); returns the status code."""
    o = (C.c_double * 3)(*[float(v) for v in origin])
    e = (C.c_double * 3)(*[float(v) for v in extent])
    ne = (C.c_int * 3)(*[int(v) for v in n_el])
    return lib().cfdem_pcm_void_fraction_static(o, e, ne, int(degree), int(n), _ptr(x), _ptr(r),
                                                _ptr(eps_q), C.c_void_p(stream or 0))


def cfdem_adjoint(h, n, x, r, u_p, u_nodal, p_nodal, eps_nodal, g_f, g_fdrag, g_eps, dJdx,
                  dJdu=None):
    return _check(h, lib().cfdem_adjoint(h, int(n), _ptr(x), _ptr(r), _ptr(u_p), _ptr(u_nodal),
                                         _ptr(p_nodal), _ptr(eps_nodal), _ptr(g_f),
                                         _ptr(g_fdrag), _ptr(g_eps), _ptr(dJdx), _ptr(dJdu)))


def cfdem_mass_apply(h, x, y):
    return _check(h, lib().cfdem_mass_apply(h, _ptr(x), _ptr(y)))


def cfdem_batch_create(n_beds, device=0, stream=None):
    h = C.c_void_p()
    st = lib().cfdem_batch_create(C.byref(h), int(device), C.c_void_p(stream or 0), int(n_beds))
    if st != OK:
        raise CfdemError(st, "cfdem_batch_create failed")
    return h


def cfdem_batch_destroy(b):
    return lib().cfdem_batch_destroy(b)


def cfdem_batch_bed(b, i):
    """The context handle of bed i (owned by the batch)."""
    v = lib().cfdem_batch_bed(b, int(i))
    if not v:
        raise CfdemError(EINVAL, "bed index out of range")
    return C.c_void_p(v)


def cfdem_batch_set_graph(b, enable):
    return lib().cfdem_batch_set_graph(b, int(bool(enable)))


def bed_io(n, x, r, u_p, u_nodal, p_nodal, eps_nodal, f, f_drag=None, F_elem=None, F_q=None,
           host=None):
    """One cfdem_bed_io record (device tensors or addresses).  host: optional
    dict of page-locked host tensors or addresses, keys x, r, u_p, u_nodal,
    p_nodal (uploaded into the device buffers by the step) and f, F_elem
    (downloaded into at its end)."""
    h = host or {}
    return cfdem_bed_io(int(n), _ptr(x), _ptr(r), _ptr(u_p), _ptr(u_nodal), _ptr(p_nodal),
                        _ptr(eps_nodal), _ptr(f), _ptr(f_drag), _ptr(F_elem), _ptr(F_q),
                        _ptr(h.get("x")), _ptr(h.get("r")), _ptr(h.get("u_p")),
                        _ptr(h.get("u_nodal")), _ptr(h.get("p_nodal")), _ptr(h.get("f")),
                        _ptr(h.get("F_elem")))


def cfdem_batch_coupling_step(b, ios):
    """One coupling step of every bed; ios: sequence of cfdem_bed_io (one per
    bed).  Returns the status code."""
    arr = (cfdem_bed_io * len(ios))(*ios)
    return lib().cfdem_batch_coupling_step(b, arr)


def cfdem_batch_synchronize(b):
    """Returns (status, first failing bed or -1)."""
    bad = C.c_int(-1)
    st = lib().cfdem_batch_synchronize(b, C.byref(bad))
    return st, bad.value


def cfdem_batch_last_replayed(b):
    return lib().cfdem_batch_last_replayed(b)


def cfdem_batch_last_error(b):
    return lib().cfdem_batch_last_error(b).decode()


def cfdem_set_timing(h, enable):
    return _check(h, lib().cfdem_set_timing(h, int(bool(enable))))


def cfdem_last_error(h):
    return lib().cfdem_last_error(h).decode()


# ------------------------------------------------------------------ helpers

def make_params(**kw):
    """cfdem_params from keyword arguments on top of the library defaults."""
    p = cfdem_params_default()
    for k, v in kw.items():
        if k == "g":
            for a in range(3):
                p.g[a] = float(v[a])
        elif k == "oracle_rtol":
            continue
        else:
            setattr(p, k, v)
    return p


class Context:
    """Owns one library context; tensors are torch CUDA tensors."""

    def __init__(self, origin, extent, n_el, degree, params=None, device=0, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self.h = cfdem_create(device, stream)
        cfdem_set_mesh(self.h, origin, extent, n_el, degree)
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        p = params if isinstance(params, cfdem_params) else make_params(**params)
        cfdem_set_params(self.h, p)

    def stats(self):
        return cfdem_get_stats(self.h)

    def close(self):
        if self.h is not None:
            cfdem_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ mapped meshes

class MappedMesh:
    """A mapped (curved) Q_k hex mesh on the device (cfdem_mapped_*):
    conn[E][(k+1)^3] and nodes[N][3] as numpy arrays."""

    def __init__(self, k, conn, nodes, margin=0.1, device=0):
        import numpy as np
        conn = np.ascontiguousarray(conn, dtype=np.int32)
        nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        h = C.c_void_p()
        st = lib().cfdem_mapped_create(C.byref(h), int(device), int(k), conn.shape[0],
                                       conn.ctypes.data, nodes.shape[0], nodes.ctypes.data,
                                       float(margin))
        if st != OK:
            raise CfdemError(st, "cfdem_mapped_create failed")
        self.h = h

    def locate(self, n, x, elem, xi=None, stream=None):
        return lib().cfdem_mapped_locate(self.h, int(n), _ptr(x), _ptr(elem), _ptr(xi),
                                         C.c_void_p(stream or 0))

    def interpolate(self, n, elem, xi, ncomp, field, out, stream=None):
        return lib().cfdem_mapped_interpolate(self.h, int(n), _ptr(elem), _ptr(xi), int(ncomp),
                                              _ptr(field), _ptr(out), C.c_void_p(stream or 0))

    def close(self):
        if self.h:
            lib().cfdem_mapped_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------------ DEM

def _dcheck(h, st):
    if st != OK:
        raise CfdemError(st, lib().cfdem_dem_last_error(h).decode())
    return st


def dem_params(**kw):
    """cfdem_dem_params from keyword arguments on top of the library defaults."""
    p = cfdem_dem_params()
    lib().cfdem_dem_params_default(C.byref(p))
    for k, v in kw.items():
        if k in ("g", "lo", "hi"):
            arr = getattr(p, k)
            for a in range(3):
                arr[a] = float(v[a])
        else:
            setattr(p, k, v)
    return p


class Dem:
    """Owns one DEM state; tensors are torch CUDA tensors (FP64)."""

    def __init__(self, params=None, device=0, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        h = C.c_void_p()
        st = lib().cfdem_dem_create(C.byref(h), int(device), C.c_void_p(stream))
        if st != OK:
            raise CfdemError(st, "cfdem_dem_create failed")
        self.h = h
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        p = params if isinstance(params, cfdem_dem_params) else dem_params(**params)
        _dcheck(self.h, lib().cfdem_dem_set_params(self.h, C.byref(p)))

    def reset(self):
        _dcheck(self.h, lib().cfdem_dem_reset(self.h))

    def step(self, x, v, w, r, f_ext, dt, nsub):
        n = x.shape[0]
        return _dcheck(self.h, lib().cfdem_dem_step(self.h, int(n), _ptr(x), _ptr(v), _ptr(w),
                                                    _ptr(r), _ptr(f_ext), float(dt), int(nsub)))

    def synchronize(self):
        return lib().cfdem_dem_synchronize(self.h)

    def last_error(self):
        return lib().cfdem_dem_last_error(self.h).decode()

    def close(self):
        if self.h:
            lib().cfdem_dem_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

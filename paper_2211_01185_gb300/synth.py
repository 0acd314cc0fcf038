"""Seeded synthetic inputs shaped like the paper's beds.

This module only draws inputs: particle positions and radii, particle
velocities and nodal fluid fields.  It holds none of the coupling method's
arithmetic (no void fraction, projection, interpolation or closure), and both
the CUDA path and the CPU oracle receive exactly the arrays it returns.

Workloads (seed = 2211011850 + workload index):

* ``q1_8x8x32_2k``   box 0.02 x 0.02 x 0.08 m, 8x8x32 Q1, 2,000 spheres of
  d = 1 mm by random sequential addition (no overlap) in the lower half;
  u = (0, 0, 0.5 + 0.05 sin(2 pi x / L_x)), p linear in z.
* ``q2_32x32x128_100k`` box 0.1 x 0.1 x 0.4 m, 32x32x128 Q2, 100,000 spheres
  with d ~ U[2, 3] mm on a jittered FCC lattice in the lower 40 % (solid
  fraction ~0.53), pushed apart until the worst overlap is below 1 % of the
  smallest diameter; u = (0, 0, 1) + 5 % seeded noise per nodal component.
* ``q3_24x24x96_1m`` box 0.144 x 0.144 x 0.576 m, 24x24x96 Q3, 1,000,000
  spheres of d = 1 mm on a jittered FCC lattice at solid fraction 0.6 (the
  bottom ~43 mm), no overlap by construction.

Fluid properties are those of a gas (rho_f = 1.2 kg/m^3, mu_f = 1.8e-5 Pa s),
g = (0, 0, -9.81); particle velocities are uniform in [-0.05, 0.05]^3 m/s;
the pressure is p = G (L_z - z) with G = phi (rho_p - rho_f) |g|, rho_p =
2500 kg/m^3 (glass); the smoothing length is L^2 = 4 mean(d)^2.
"""
from __future__ import annotations

import math

import numpy as np

SEED0 = 2211011850
RHO_P = 2500.0

WORKLOADS = {
    "q1_8x8x32_2k": dict(index=1, origin=(0.0, 0.0, 0.0), extent=(0.02, 0.02, 0.08),
                          n_el=(8, 8, 32), k=1, n=2000, d=(1e-3, 1e-3), phi=0.065,
                          packing="rsa", bed_frac=0.5, field="sine", u_mean=0.5),
    "q2_32x32x128_100k": dict(index=2, origin=(0.0, 0.0, 0.0), extent=(0.1, 0.1, 0.4),
                               n_el=(32, 32, 128), k=2, n=100_000, d=(2e-3, 3e-3), phi=0.53,
                               packing="fcc_relax", bed_frac=0.4, field="noise", u_mean=1.0),
    "q3_24x24x96_1m": dict(index=3, origin=(0.0, 0.0, 0.0), extent=(0.144, 0.144, 0.576),
                            n_el=(24, 24, 96), k=3, n=1_000_000, d=(1e-3, 1e-3), phi=0.6,
                            packing="fcc", bed_frac=0.5, field="noise", u_mean=1.0),
}


def gas_params(mean_d: float, k: int) -> dict:
    """Physical and numerical parameters shared by the workloads."""
    return dict(rho_f=1.2, mu_f=1.8e-5, g=(0.0, 0.0, -9.81), scheme=0, qcm_radius=0.0,
                l2_smoothing=4.0 * mean_d * mean_d, drag_model=0, vans_model=0,
                beta_over_eps=0, eps_floor=0.05, pressure_degree=max(1, k - 1))


# --------------------------------------------------------------- particles

def rsa(rng, n, d, lo, hi, max_tries=200, radii=None):
    """Random sequential addition of n spheres with centres in the box
    [lo, hi] and no overlap: equal diameter d, or the given radii."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    pts = np.zeros((0, 3))
    tries = 0
    while pts.shape[0] < n:
        tries += 1
        if tries > max_tries * n:
            raise RuntimeError("random sequential addition jammed")
        c = lo + (hi - lo) * rng.random(3)
        if pts.shape[0]:
            dd = np.sum((pts - c) ** 2, axis=1)
            if radii is None:
                lim = d * d
            else:
                lim = (radii[:pts.shape[0]] + radii[pts.shape[0]]) ** 2
            if np.any(dd < lim):
                continue
        pts = np.vstack([pts, c])
    return pts


def fcc_sites(a_nn, lo, hi, n):
    """The n lowest sites (by z, then y, then x) of an FCC lattice of
    nearest-neighbour distance a_nn filling the box [lo, hi]."""
    a = a_nn * math.sqrt(2.0)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    nc = np.floor((hi - lo) / a + 1e-9).astype(int)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) + 0.25
    per_layer = 4 * nc[0] * nc[1]
    nz = int(math.ceil(n / per_layer)) + 1
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(nc[1]), np.arange(nc[0]), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a + lo
    order = np.lexsort((sites[:, 0], sites[:, 1], sites[:, 2]))
    sites = sites[order]
    if sites.shape[0] < n:
        raise RuntimeError("lattice too small")
    return sites[:n]


def push_apart(rng, x, r, lo, hi, tol, iters=400):
    """Soft relaxation: move every overlapping pair apart along the line of
    centres and keep centres at least a radius inside the side walls and the
    floor, until the largest overlap is below tol."""
    from scipy.spatial import cKDTree
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    rmax = float(r.max())
    for _ in range(iters):
        tree = cKDTree(x)
        pairs = tree.query_pairs(2.0 * rmax, output_type="ndarray")
        if pairs.shape[0] == 0:
            break
        i, j = pairs[:, 0], pairs[:, 1]
        dv = x[j] - x[i]
        dist = np.sqrt(np.sum(dv * dv, axis=1))
        ov = r[i] + r[j] - dist
        m = ov > 0
        worst = float(ov[m].max()) if np.any(m) else 0.0
        if worst <= tol:
            break
        i, j, dv, dist, ov = i[m], j[m], dv[m], dist[m], ov[m]
        nrm = dv / np.maximum(dist, 1e-12)[:, None]
        step = 0.55 * ov[:, None] * nrm
        disp = np.zeros_like(x)
        np.add.at(disp, i, -step)
        np.add.at(disp, j, step)
        x = x + disp
        x[:, 0] = np.clip(x[:, 0], lo[0] + r, hi[0] - r)
        x[:, 1] = np.clip(x[:, 1], lo[1] + r, hi[1] - r)
        x[:, 2] = np.clip(x[:, 2], lo[2] + r, hi[2] - r)
    return x


def make_particles(spec: dict, rng):
    n = int(spec["n"])
    dlo, dhi = spec["d"]
    origin = np.asarray(spec["origin"], dtype=np.float64)
    extent = np.asarray(spec["extent"], dtype=np.float64)
    if dlo == dhi:
        d = np.full(n, dlo)
    else:
        d = dlo + (dhi - dlo) * rng.random(n)
    r = 0.5 * d
    top = origin[2] + spec["bed_frac"] * extent[2]
    if spec["packing"] == "rsa":
        rr = 0.5 * dlo
        x = rsa(rng, n, dlo, origin + rr, np.array([origin[0] + extent[0] - rr,
                                                   origin[1] + extent[1] - rr, top - rr]))
    elif spec["packing"] == "fcc":
        a_nn = dhi * (0.74048 / spec["phi"]) ** (1.0 / 3.0)
        x = fcc_sites(a_nn, origin, origin + extent, n)
        jit = 0.5 * (a_nn - dhi)
        u = rng.normal(size=(n, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        x = x + u * (jit * rng.random(n) ** (1.0 / 3.0))[:, None]
    elif spec["packing"] == "fcc_relax":
        vol = extent[0] * extent[1] * spec["bed_frac"] * extent[2]
        density = n / vol
        a_nn = (math.sqrt(2.0) / density) ** (1.0 / 3.0)
        x = fcc_sites(a_nn, origin, origin + extent, n)
        x = x + (0.05 * a_nn) * (rng.random((n, 3)) - 0.5)
        x = push_apart(rng, x, r, origin, origin + extent, tol=0.01 * dlo)
    else:
        raise ValueError(spec["packing"])
    return np.ascontiguousarray(x), np.ascontiguousarray(r)


# --------------------------------------------------------------- fields

_GLL = {1: [0.0, 1.0], 2: [0.0, 0.5, 1.0],
        3: [0.0, 0.5 - 0.5 / math.sqrt(5.0), 0.5 + 0.5 / math.sqrt(5.0), 1.0]}


def node_axes(origin, extent, n_el, deg):
    """1D node coordinates of the Q_deg grid per axis (GLL points in each
    element), used only to sample the analytic input fields."""
    z = np.asarray(_GLL[deg])
    out = []
    for a in range(3):
        h = extent[a] / n_el[a]
        t = (np.arange(n_el[a])[:, None] + z[None, :-1]).reshape(-1)
        t = np.concatenate([t, [float(n_el[a])]])
        out.append(origin[a] + h * t)
    return out


def make_fields(spec: dict, rng, n_particles: int):
    k = spec["k"]
    kp = max(1, k - 1)
    origin = np.asarray(spec["origin"], dtype=np.float64)
    extent = np.asarray(spec["extent"], dtype=np.float64)
    n_el = spec["n_el"]
    ax, ay, az = node_axes(origin, extent, n_el, k)
    Z, Y, X = np.meshgrid(az, ay, ax, indexing="ij")
    nn = X.size
    u = np.zeros((nn, 3))
    if spec["field"] == "sine":
        u[:, 2] = spec["u_mean"] + 0.05 * np.sin(2.0 * math.pi * (X.ravel() - origin[0]) / extent[0])
    else:
        u[:, 2] = spec["u_mean"]
        u += 0.05 * spec["u_mean"] * (2.0 * rng.random((nn, 3)) - 1.0)
    px, py, pz = node_axes(origin, extent, n_el, kp)
    PZ, PY, PX = np.meshgrid(pz, py, px, indexing="ij")
    G = spec["phi"] * (RHO_P - 1.2) * 9.81
    p = G * (origin[2] + extent[2] - PZ.ravel())
    u_p = 0.1 * rng.random((n_particles, 3)) - 0.05
    return np.ascontiguousarray(u), np.ascontiguousarray(p), np.ascontiguousarray(u_p)


def make_workload(name: str, seed: int | None = None) -> dict:
    """All inputs of one coupling step of the named workload."""
    spec = dict(WORKLOADS[name])
    rng = np.random.default_rng(SEED0 + spec["index"] if seed is None else seed)
    x, r = make_particles(spec, rng)
    u, p, u_p = make_fields(spec, rng, x.shape[0])
    params = gas_params(float(np.mean(spec["d"])), spec["k"])
    return dict(name=name, origin=tuple(spec["origin"]), extent=tuple(spec["extent"]),
                n_el=tuple(spec["n_el"]), k=spec["k"], x=x, r=r, u_p=u_p, u_nodal=u,
                p_nodal=p, params=params)


def make_batch_workload(n_beds: int = 64, seed: int | None = None, n_range=(5_000, 200_000),
                        nxy=(8, 32), nz=(8, 64)) -> list:
    """The ensemble of independent beds: per bed, elements per axis drawn from
    nxy (x, y) and nz (z), degree k uniform in {1, 2, 3}, N log-uniform in
    n_range, one diameter d ~ U[1, 3] mm, cubic elements of edge h chosen so
    that N V_p = 0.3 of the box volume, particles on a jittered FCC lattice
    at solid fraction 0.55 from the floor up, averaging radius at least the
    particle radius, inflow u_z ~ U[0.5, 2] m/s with 5 % noise."""
    rng = np.random.default_rng(SEED0 + 4 if seed is None else seed)
    beds = []
    for b in range(n_beds):
        ne = (int(rng.integers(nxy[0], nxy[1] + 1)), int(rng.integers(nxy[0], nxy[1] + 1)),
              int(rng.integers(nz[0], nz[1] + 1)))
        k = int(rng.integers(1, 4))
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        d = float(rng.uniform(1e-3, 3e-3))
        vp = math.pi * d ** 3 / 6.0
        h = (n * vp / (0.3 * ne[0] * ne[1] * ne[2])) ** (1.0 / 3.0)
        spec = dict(index=4, origin=(0.0, 0.0, 0.0),
                    extent=(ne[0] * h, ne[1] * h, ne[2] * h), n_el=ne, k=k, n=n, d=(d, d),
                    phi=0.55, packing="fcc", bed_frac=0.55, field="noise",
                    u_mean=float(rng.uniform(0.5, 2.0)))
        x, r = make_particles(spec, rng)
        u, p, u_p = make_fields(spec, rng, n)
        params = gas_params(d, k)
        r_default = (3.0 * h ** 3 / (4.0 * math.pi)) ** (1.0 / 3.0)
        if r_default < 0.5 * d:
            params["qcm_radius"] = 0.5 * d
        beds.append(dict(name="bed%02d" % b, origin=spec["origin"], extent=spec["extent"],
                         n_el=ne, k=k, x=x, r=r, u_p=u_p, u_nodal=u, p_nodal=p, params=params))
    return beds


def make_adjoint_workload(seed: int | None = None, n_el=(24, 24, 96)) -> dict:
    """The sensitivity workload: a 0.096 x 0.096 x 0.384 m box of 24 x 24 x 96
    Q2 elements (h = 4 mm, averaging radius 2.481 mm), 200,000 spheres of
    d = 2 mm from the floor up -- an annulus at solid fraction 0.5 on a
    jittered FCC lattice (its top a little above half height) and a central
    column of radius 0.15 L_x, lower half, at 0.05 by random sequential
    addition -- under a jet u_z = 0.2 + 1.8 (1 - tanh((rho - 0.15
    L_x) / (0.02 L_x))) / 2 m/s (rho the distance from the axis).  The loss
    of this workload is J = sum_i e_z . f_D,i + ||eps_h||_M.
    A smaller n_el keeps h = 4 mm and the layout relative to the box and
    scales the particle count with the element count."""
    rng = np.random.default_rng(SEED0 + 5 if seed is None else seed)
    n_el, k, d = tuple(int(v) for v in n_el), 2, 2e-3
    n_total = int(round(200_000 * (n_el[0] * n_el[1] * n_el[2]) / (24 * 24 * 96)))
    h = 4e-3
    extent = (n_el[0] * h, n_el[1] * h, n_el[2] * h)
    Lx = extent[0]
    rc = 0.15 * Lx
    cx = cy = 0.5 * Lx
    top = 0.5 * extent[2]
    r0 = 0.5 * d
    # annulus: FCC at 0.5, sites whose sphere stays outside the column
    a_nn = d * (0.74048 / 0.5) ** (1.0 / 3.0)
    a = a_nn * math.sqrt(2.0)
    ncx = int(math.floor(extent[0] / a))
    ncz = int(math.floor(extent[2] / a))
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) + 0.25
    iz, iy, ix = np.meshgrid(np.arange(ncz), np.arange(ncx), np.arange(ncx), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    rad = np.hypot(sites[:, 0] - cx, sites[:, 1] - cy)
    sites = sites[rad >= rc + r0]
    vcol = math.pi * rc * rc * top
    ncol = int(round(0.05 * vcol / (math.pi * d ** 3 / 6.0)))
    # the lowest annulus sites up to N = 200,000 in all (the lattice, cut by
    # the walls, holds a little less than that below half height)
    sites = sites[np.lexsort((sites[:, 0], sites[:, 1], sites[:, 2]))][:n_total - ncol]
    jit = 0.5 * (a_nn - d)
    u = rng.normal(size=sites.shape)
    u /= np.linalg.norm(u, axis=1)[:, None]
    xa = sites + u * (jit * rng.random(sites.shape[0]) ** (1.0 / 3.0))[:, None]
    # column: random sequential addition at 0.05
    cand = []
    lo = np.array([cx - rc + r0, cy - rc + r0, r0])
    hi = np.array([cx + rc - r0, cy + rc - r0, top - r0])
    pts = np.zeros((0, 3))
    while pts.shape[0] < ncol:
        c = lo + (hi - lo) * rng.random((4 * ncol, 3))
        c = c[np.hypot(c[:, 0] - cx, c[:, 1] - cy) <= rc - r0]
        for q in c:
            if pts.shape[0] >= ncol:
                break
            if pts.shape[0] == 0 or np.min(np.sum((pts - q) ** 2, axis=1)) >= d * d:
                pts = np.vstack([pts, q])
        cand.append(c.shape[0])
    x = np.ascontiguousarray(np.vstack([xa, pts]))
    n = x.shape[0]
    r = np.full(n, r0)
    spec = dict(index=5, origin=(0.0, 0.0, 0.0), extent=extent, n_el=n_el, k=k, n=n, d=(d, d),
                phi=0.5, packing="fcc", bed_frac=0.5, field="noise", u_mean=0.0)
    ax, ay, az = node_axes(np.zeros(3), np.asarray(extent), n_el, k)
    Z, Y, X = np.meshgrid(az, ay, ax, indexing="ij")
    rho = np.hypot(X.ravel() - cx, Y.ravel() - cy)
    un = np.zeros((X.size, 3))
    un[:, 2] = 0.2 + 1.8 * 0.5 * (1.0 - np.tanh((rho - rc) / (0.02 * Lx)))
    kp = max(1, k - 1)
    px, py, pz = node_axes(np.zeros(3), np.asarray(extent), n_el, kp)
    PZ, PY, PX = np.meshgrid(pz, py, px, indexing="ij")
    p = 0.5 * (RHO_P - 1.2) * 9.81 * (extent[2] - PZ.ravel())
    u_p = 0.1 * rng.random((n, 3)) - 0.05
    params = gas_params(d, k)
    del spec, cand
    name = "adjoint_%dx%dx%d_%d" % (n_el + (n,))
    if n_el == (24, 24, 96):
        name = "adjoint_24x24x96_200k"
    return dict(name=name, origin=(0.0, 0.0, 0.0), extent=extent, n_el=n_el,
                k=k, x=x, r=r, u_p=u_p, u_nodal=np.ascontiguousarray(un), p_nodal=p,
                params=params)


def make_random_case(seed: int, n_el=(3, 4, 5), k=2, n=150, extent=(0.03, 0.04, 0.05),
                     d=(2e-3, 6e-3), origin=(0.0, 0.0, 0.0), overlap_ok=True) -> dict:
    """Small uneven case for parity tests: uniform random centres over the
    whole box with overlaps allowed (overlap_ok), or placed by random
    sequential addition without overlap; diameters uniform in d."""
    rng = np.random.default_rng(seed)
    origin = np.asarray(origin, dtype=np.float64)
    extent = np.asarray(extent, dtype=np.float64)
    r = 0.5 * (d[0] + (d[1] - d[0]) * rng.random(n))
    if overlap_ok:
        x = origin + extent * rng.random((n, 3))
    else:
        x = rsa(rng, n, 0.0, origin, origin + extent, radii=r)
    spec = dict(origin=origin, extent=extent, n_el=n_el, k=k, field="noise", u_mean=1.0,
                phi=0.3)
    u, p, u_p = make_fields(spec, rng, n)
    params = gas_params(float(np.mean(d)), k)
    return dict(name="random%d" % seed, origin=tuple(origin), extent=tuple(extent),
                n_el=tuple(n_el), k=k, x=np.ascontiguousarray(x), r=np.ascontiguousarray(r),
                u_p=u_p, u_nodal=u, p_nodal=p, params=params)


# --------------------------------------------------------------- mapped meshes

def _merge_nodes(pts, scale):
    """Global node numbering of element-local node coordinates: points that
    coincide (to 1e-9 of the mesh size) share a node."""
    key = np.round(pts / (1e-9 * scale)).astype(np.int64)
    uniq, inv = np.unique(key, axis=0, return_inverse=True)
    nodes = np.zeros((uniq.shape[0], 3))
    nodes[inv.ravel()] = pts
    return nodes, inv.ravel().astype(np.int32)


def make_box_mapped_mesh(origin, extent, n_el, k):
    """An axis-aligned box of equal Q_k hex elements written as a mapped mesh
    (conn[E][(k+1)^3] with the local index a + (k+1)(b + (k+1)c), element
    index ex + nx (ey + ny ez), and node coordinates), for the location on
    mapped meshes to be compared with the box's own location."""
    z = np.asarray(_GLL[k])
    o = np.asarray(origin, dtype=np.float64)
    h = np.asarray(extent, dtype=np.float64) / np.asarray(n_el)
    pts = []
    for ez in range(n_el[2]):
        for ey in range(n_el[1]):
            for ex in range(n_el[0]):
                C, B, A = np.meshgrid(z, z, z, indexing="ij")
                loc = np.stack([o[0] + h[0] * (ex + A.ravel()), o[1] + h[1] * (ey + B.ravel()),
                                o[2] + h[2] * (ez + C.ravel())], axis=1)
                pts.append(loc)
    pts = np.concatenate(pts)
    nodes, inv = _merge_nodes(pts, float(np.max(extent)))
    return dict(k=k, conn=inv.reshape(-1, (k + 1) ** 3), nodes=nodes)


def make_cylinder_mesh(radius, height, n_core, n_ring, n_z, k, origin=(0.0, 0.0, 0.0)):
    """A subdivided cylinder (the mesh type of the paper's sedimentation and
    fluidised-bed cases) of Q_k hex elements: in the cross-section a square
    core of side radius/sqrt(2) (n_core x n_core elements) and four blocks
    between the square's sides and the circle (n_core tangential x n_ring
    radial elements), each point of a block on the straight line from the
    square's side to the arc at the same tangential fraction; n_z layers
    along z.  Nodes at the GLL points of each element's reference
    coordinates, so the ring elements are curved.  Returns conn[E][(k+1)^3]
    (a fastest, right-handed reference axes) and nodes[N][3]."""
    z = np.asarray(_GLL[k])
    R = float(radius)
    a = R / math.sqrt(2.0) * 0.5
    o = np.asarray(origin, dtype=np.float64)
    C, B, A = np.meshgrid(z, z, z, indexing="ij")
    s, t, w = A.ravel(), B.ravel(), C.ravel()
    pts = []

    def rot(xy, q):
        c, sn = math.cos(q * math.pi / 2), math.sin(q * math.pi / 2)
        return np.stack([c * xy[:, 0] - sn * xy[:, 1], sn * xy[:, 0] + c * xy[:, 1]], axis=1)

    for lz in range(n_z):
        zz = o[2] + height * (lz + w) / n_z
        for j in range(n_core):          # core
            for i in range(n_core):
                x = -a + 2 * a * (i + s) / n_core
                y = -a + 2 * a * (j + t) / n_core
                pts.append(np.stack([o[0] + x, o[1] + y, zz], axis=1))
        for q in range(4):               # ring blocks, the first one on the +x side
            for j in range(n_core):      # tangential
                for i in range(n_ring):  # radial
                    v = (i + s) / n_ring
                    u = (j + t) / n_core
                    side = np.stack([np.full_like(u, a), -a + 2 * a * u], axis=1)
                    th = -math.pi / 4 + math.pi / 2 * u
                    arc = np.stack([R * np.cos(th), R * np.sin(th)], axis=1)
                    xy = rot((1.0 - v)[:, None] * side + v[:, None] * arc, q)
                    pts.append(np.stack([o[0] + xy[:, 0], o[1] + xy[:, 1], zz], axis=1))
    pts = np.concatenate(pts)
    nodes, inv = _merge_nodes(pts, max(R, height))
    return dict(k=k, conn=inv.reshape(-1, (k + 1) ** 3), nodes=nodes, radius=R, height=height)

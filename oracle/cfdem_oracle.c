/*
 * cfdem_oracle.c -- plain FP64 CPU oracle of the CFD-DEM coupling step of
 * "Towards High-Order CFD-DEM: Development and Validation" (arXiv 2211.01185).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the package's smoke() check and the CPU
 * baseline leg of bench.py use it.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * It is written for a reader checking it against the paper by eye: every
 * quantity is computed from its definition, loops follow the order of the
 * sums, nothing is blocked or fused.  Built with -O2 -ffp-contract=off so that
 * no multiply-add is contracted (the neighbour predicate and the element
 * location must be decided exactly as written).
 *
 * What each function follows:
 *   or_locate          Sec. 2.3 (particle and fluid share one mesh: the element
 *                      containing a particle is found directly from its position)
 *   or_bin             the same localisation on a coarser grid of bins, stable
 *   or_lens_volume     sphere-sphere intersection volume (textbook geometry)
 *   or_qcm             Eq. (void_fraction) evaluated with averaging spheres
 *                      centred at the quadrature points (quadrature-centred
 *                      reading of the deferred void-fraction scheme)
 *   or_qcm_weights     per-particle scaling of the QCM sum that conserves
 *                      the particle volume on the mesh (walls included)
 *   or_pcm             Eq. (void_fraction), particle-centroid method
 *   or_rhs / or_apply  smoothed L2 projection (M + L^2 K) eps_h = b, the
 *   or_cg              reading of the "void fraction smoothing factor L^2"
 *                      (Tables setup1, setup2, setup4)
 *   or_drag_*          Eq. (drag) and the closures of Sec. 2.3.2: Di Felice,
 *                      Dallavalle, Rong, Koch-Hill, Gidaspow, Beetstra, Re_p
 *   or_forces          drag + buoyancy + pressure gradient per particle,
 *                      f_fp,i of Eqs. (fb)/(fa) without the shear term
 *   or_shear_force     the shear term -V_p div tau, Eq. (stress)
 *   or_fluid_source    F_pf of Eqs. (fb)/(fa), with the minus sign that
 *                      Newton's third law requires (Sec. 2.3.2)
 *   or_fluid_source_semi  the same with the fluid-side drag of Sec. 2.3.2
 *                      (fluid velocity at the quadrature point, cell-mean
 *                      particle velocity)
 * Parity is pinned by the tests: closed forms, limits, brute force,
 * conservation laws and the worked numbers the paper prints.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* 1D tables                                                          */
/* ------------------------------------------------------------------ */

/* Legendre polynomial P_n(s) and its derivative, three-term recurrence. */
static void legendre(int n, double s, double *p, double *dp)
{
    double p0 = 1.0, p1 = s;
    if (n == 0) { *p = 1.0; *dp = 0.0; return; }
    for (int m = 2; m <= n; ++m) {
        double p2 = ((2.0 * m - 1.0) * s * p1 - (m - 1.0) * p0) / m;
        p0 = p1;
        p1 = p2;
    }
    *p = p1;
    /* (1 - s^2) P_n' = n (P_{n-1} - s P_n) */
    *dp = n * (p0 - s * p1) / (1.0 - s * s);
}

/* n-point Gauss-Legendre rule mapped to [0,1]: Newton on the roots of P_n,
 * weights 2/((1-s^2) P_n'(s)^2) halved for the unit interval. */
void or_gauss_rule(int n, double *pts, double *wts)
{
    for (int i = 0; i < n; ++i) {
        double s = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double p, dp;
        for (int it = 0; it < 100; ++it) {
            legendre(n, s, &p, &dp);
            double ds = p / dp;
            s -= ds;
            if (fabs(ds) < 1e-17) break;
        }
        legendre(n, s, &p, &dp);
        /* s descends with i, so 0.5 (1 - s) ascends on [0,1]; the weight
         * 2 / ((1 - s^2) P_n'(s)^2) of [-1,1] is halved on [0,1] */
        pts[i] = 0.5 * (1.0 - s);
        wts[i] = 1.0 / ((1.0 - s * s) * dp * dp);
    }
}

/* Gauss-Lobatto-Legendre nodes of degree k on [0,1]: the end points and the
 * roots of P_k'. */
void or_gll_nodes(int k, double *z)
{
    z[0] = 0.0;
    z[k] = 1.0;
    for (int i = 1; i < k; ++i) {
        /* Chebyshev-Gauss-Lobatto start, Newton on P_k' using
         * (1-s^2) P_k'' = 2 s P_k' - k(k+1) P_k */
        double s = -cos(OR_PI * i / k);
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre(k, s, &p, &dp);
            double d2p = (2.0 * s * dp - k * (k + 1.0) * p) / (1.0 - s * s);
            double ds = dp / d2p;
            s -= ds;
            if (fabs(ds) < 1e-17) break;
        }
        z[i] = 0.5 * (1.0 + s);
    }
}

/* Lagrange basis on the nodes z[0..k] and its derivative at t. */
static void lagrange(int k, const double *z, double t, double *l, double *dl)
{
    for (int a = 0; a <= k; ++a) {
        double v = 1.0, dv = 0.0;
        for (int b = 0; b <= k; ++b) {
            if (b == a) continue;
            double den = z[a] - z[b];
            /* product rule: d/dt prod (t - z_b)/den */
            dv = dv * (t - z[b]) / den + v / den;
            v = v * (t - z[b]) / den;
        }
        l[a] = v;
        if (dl) dl[a] = dv;
    }
}

/* Second derivatives of the Lagrange basis from the definition
 *   l_a(t) = prod_{m != a} (t - z_m) / (z_a - z_m),
 * differentiated twice: l_a''(t) = sum over ordered pairs b != c (both != a)
 * of 1/((z_a - z_b)(z_a - z_c)) prod_{m != a, b, c} (t - z_m)/(z_a - z_m). */
static void lagrange_dd(int k, const double *z, double t, double *ddl)
{
    for (int a = 0; a <= k; ++a) {
        double s = 0.0;
        for (int b = 0; b <= k; ++b) {
            if (b == a) continue;
            for (int c = 0; c <= k; ++c) {
                if (c == a || c == b) continue;
                double p = 1.0 / ((z[a] - z[b]) * (z[a] - z[c]));
                for (int m = 0; m <= k; ++m) {
                    if (m == a || m == b || m == c) continue;
                    p *= (t - z[m]) / (z[a] - z[m]);
                }
                s += p;
            }
        }
        ddl[a] = s;
    }
}

void or_lagrange_dd(int k, double t, double *ddl)
{
    double z[8];
    or_gll_nodes(k, z);
    lagrange_dd(k, z, t, ddl);
}

void or_lagrange(int k, double t, double *l, double *dl)
{
    double z[8];
    or_gll_nodes(k, z);
    lagrange(k, z, t, l, dl);
}

/* ------------------------------------------------------------------ */
/* Mesh                                                               */
/* ------------------------------------------------------------------ */

typedef struct {
    double x0[3], L[3], h[3];
    int ne[3];
    int k;
} omesh;

static omesh make_mesh(const double *origin, const double *extent, const int *n_el, int k)
{
    omesh m;
    for (int a = 0; a < 3; ++a) {
        m.x0[a] = origin[a];
        m.L[a] = extent[a];
        m.ne[a] = n_el[a];
        m.h[a] = extent[a] / n_el[a];
    }
    m.k = k;
    return m;
}

static int64_t n_elem(const omesh *m) { return (int64_t)m->ne[0] * m->ne[1] * m->ne[2]; }

/* number of nodes per axis of the Q_deg grid */
static int nn_axis(const omesh *m, int a, int deg) { return m->ne[a] * deg + 1; }

/* ------------------------------------------------------------------ */
/* Locate                                                             */
/* ------------------------------------------------------------------ */

/* Element index along one axis: floor of (x - x0)/h with IEEE division,
 * clamped to [0, N-1]; a particle on an interior face belongs to the upper
 * element, one on the top wall to the last element.  Returns 0 when x lies
 * outside [x0, x0+L] by more than 1e-12 L (NaN included). */
static int locate_axis(double x, double x0, double L, double h, int N, int *ie, double *xi)
{
    double lo = x0 - 1e-12 * L;
    double hi = (x0 + L) + 1e-12 * L;
    if (!(x >= lo && x <= hi)) return 0;
    double t = (x - x0) / h;
    double f = floor(t);
    int i = (int)f;
    if (i < 0) i = 0;
    if (i > N - 1) i = N - 1;
    *ie = i;
    *xi = t - (double)i;
    return 1;
}

/* elem[n] = ex + Nx (ey + Ny ez); xi[n][3] reference coordinates in [0,1].
 * Returns -1 if every particle is inside, else the first bad index. */
int64_t or_locate(const double *origin, const double *extent, const int *n_el, int k,
                  int64_t n, const double *x, int32_t *elem, double *xi)
{
    omesh m = make_mesh(origin, extent, n_el, k);
    int64_t bad = -1;
    for (int64_t i = 0; i < n; ++i) {
        int ie[3];
        double t[3];
        int ok = 1;
        for (int a = 0; a < 3; ++a)
            ok &= locate_axis(x[3 * i + a], m.x0[a], m.L[a], m.h[a], m.ne[a], &ie[a], &t[a]);
        if (!ok) {
            if (bad < 0) bad = i;
            elem[i] = -1;
            if (xi) xi[3 * i] = xi[3 * i + 1] = xi[3 * i + 2] = 0.0;
            continue;
        }
        elem[i] = ie[0] + m.ne[0] * (ie[1] + m.ne[1] * ie[2]);
        if (xi) for (int a = 0; a < 3; ++a) xi[3 * i + a] = t[a];
    }
    return bad;
}

/* ------------------------------------------------------------------ */
/* Bins                                                               */
/* ------------------------------------------------------------------ */

/* Bin of a particle on a grid of nb[a] equal bins per axis over the box:
 * floor((x - x0)/(L/nb)), clamped. */
static int bin_axis(double x, double x0, double L, int nb)
{
    double be = L / nb;
    double t = (x - x0) / be;
    double f = floor(t);
    int i;
    if (!(f >= 0.0)) i = 0;            /* also catches NaN */
    else if (f > (double)(nb - 1)) i = nb - 1;
    else i = (int)f;
    return i;
}

/* Stable counting sort of the particles into bins (bx fastest):
 * bin_start[nbins+1] exclusive prefix of the counts, perm[n] the particle
 * ids in bin order, ascending id inside a bin. */
void or_bin(const double *origin, const double *extent, const int *nb,
            int64_t n, const double *x, int32_t *bin_of, int32_t *bin_start, int32_t *perm)
{
    int64_t nbins = (int64_t)nb[0] * nb[1] * nb[2];
    memset(bin_start, 0, sizeof(int32_t) * (nbins + 1));
    for (int64_t i = 0; i < n; ++i) {
        int b[3];
        for (int a = 0; a < 3; ++a) b[a] = bin_axis(x[3 * i + a], origin[a], extent[a], nb[a]);
        int32_t id = b[0] + nb[0] * (b[1] + nb[1] * b[2]);
        bin_of[i] = id;
        bin_start[id + 1] += 1;
    }
    for (int64_t j = 0; j < nbins; ++j) bin_start[j + 1] += bin_start[j];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (nbins > 0 ? nbins : 1));
    for (int64_t j = 0; j < nbins; ++j) fill[j] = bin_start[j];
    for (int64_t i = 0; i < n; ++i) perm[fill[bin_of[i]]++] = (int32_t)i; /* ascending i */
    free(fill);
}

/* ------------------------------------------------------------------ */
/* Void fraction                                                      */
/* ------------------------------------------------------------------ */

/* Volume of the intersection of two spheres of radii R and r whose centres
 * are d apart. */
double or_lens_volume(double R, double r, double d)
{
    if (d >= R + r) return 0.0;
    double mn = R < r ? R : r;
    if (d <= fabs(R - r)) return 4.0 / 3.0 * OR_PI * mn * mn * mn;
    double s = R + r - d;
    double dm = R - r;
    return OR_PI * s * s * (d * d + 2.0 * d * (R + r) - 3.0 * dm * dm) / (12.0 * d);
}

/* physical coordinate of Gauss point g of element index ie along an axis */
static double qp_coord(double x0, double h, int ie, double g)
{
    double t1 = (double)ie + g;
    double t2 = h * t1;
    return x0 + t2;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Quadrature-centred void fraction: for every Gauss point x_q of every
 * element, eps_q = 1 - sum_i V_lens(R, r_i, |x_q - x_i|) / (4/3 pi R^3) over
 * the particles with |x_q - x_i|^2 < (R + r_i)^2, summed in ascending id.
 * Neighbour sets come from a cell list of edge >= R + max r (or from brute
 * force when brute != 0).  Optional outputs: neighbour count and id sum per
 * quadrature point. */
void or_qcm(const double *origin, const double *extent, const int *n_el, int k, double R,
            int64_t n, const double *x, const double *r, const double *cw, int brute,
            double *eps_q, int32_t *nb_count, int64_t *nb_idsum)
{
    omesh m = make_mesh(origin, extent, n_el, k);
    int nq = k + 1;
    double g[8], w[8];
    or_gauss_rule(nq, g, w);
    double VR = 4.0 / 3.0 * OR_PI * R * R * R;
    double rmax = 0.0;
    for (int64_t i = 0; i < n; ++i) if (r[i] > rmax) rmax = r[i];
    double cut = R + rmax;

    int nc[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)floor(m.L[a] / cut);
        if (nc[a] < 1) nc[a] = 1;
    }
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int32_t *cstart = (int32_t *)malloc(sizeof(int32_t) * (ncell + 1));
    int32_t *cperm = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    or_bin(m.x0, m.L, nc, n, x, cell_of, cstart, cperm);

    int64_t E = n_elem(&m);
    int Q = nq * nq * nq;
#pragma omp parallel
    {
        int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 64)
        for (int64_t e = 0; e < E; ++e) {
            int ex = (int)(e % m.ne[0]);
            int ey = (int)((e / m.ne[0]) % m.ne[1]);
            int ez = (int)(e / ((int64_t)m.ne[0] * m.ne[1]));
            for (int qz = 0; qz < nq; ++qz)
            for (int qy = 0; qy < nq; ++qy)
            for (int qx = 0; qx < nq; ++qx) {
                int q = qx + nq * (qy + nq * qz);
                double xq = qp_coord(m.x0[0], m.h[0], ex, g[qx]);
                double yq = qp_coord(m.x0[1], m.h[1], ey, g[qy]);
                double zq = qp_coord(m.x0[2], m.h[2], ez, g[qz]);
                int cnt = 0;
                if (brute) {
                    for (int64_t i = 0; i < n; ++i) {
                        double dx = x[3 * i] - xq, dy = x[3 * i + 1] - yq, dz = x[3 * i + 2] - zq;
                        double d2 = dx * dx + dy * dy + dz * dz;
                        double c = R + r[i];
                        if (d2 < c * c) list[cnt++] = (int32_t)i;
                    }
                } else {
                    int cq[3];
                    cq[0] = bin_axis(xq, m.x0[0], m.L[0], nc[0]);
                    cq[1] = bin_axis(yq, m.x0[1], m.L[1], nc[1]);
                    cq[2] = bin_axis(zq, m.x0[2], m.L[2], nc[2]);
                    for (int cz = cq[2] - 1; cz <= cq[2] + 1; ++cz) {
                        if (cz < 0 || cz >= nc[2]) continue;
                        for (int cy = cq[1] - 1; cy <= cq[1] + 1; ++cy) {
                            if (cy < 0 || cy >= nc[1]) continue;
                            for (int cx = cq[0] - 1; cx <= cq[0] + 1; ++cx) {
                                if (cx < 0 || cx >= nc[0]) continue;
                                int64_t c = cx + (int64_t)nc[0] * (cy + (int64_t)nc[1] * cz);
                                for (int32_t s = cstart[c]; s < cstart[c + 1]; ++s) {
                                    int32_t i = cperm[s];
                                    double dx = x[3 * i] - xq, dy = x[3 * i + 1] - yq,
                                           dz = x[3 * i + 2] - zq;
                                    double d2 = dx * dx + dy * dy + dz * dz;
                                    double cc = R + r[i];
                                    if (d2 < cc * cc) list[cnt++] = i;
                                }
                            }
                        }
                    }
                    qsort(list, cnt, sizeof(int32_t), cmp_i32);
                }
                double vs = 0.0;
                int64_t ids = 0;
                for (int j = 0; j < cnt; ++j) {
                    int32_t i = list[j];
                    double dx = x[3 * i] - xq, dy = x[3 * i + 1] - yq, dz = x[3 * i + 2] - zq;
                    double d = sqrt(dx * dx + dy * dy + dz * dz);
                    double v = or_lens_volume(R, r[i], d);
                    vs += cw ? cw[i] * v : v;
                    ids += i;
                }
                eps_q[e * Q + q] = 1.0 - vs / VR;
                if (nb_count) nb_count[e * Q + q] = cnt;
                if (nb_idsum) nb_idsum[e * Q + q] = ids;
            }
        }
        free(list);
    }
    free(cell_of);
    free(cstart);
    free(cperm);
}

/* Weights of the volume-conserving quadrature-centred void fraction: the
 * volume a particle deposits on the mesh through the QCM sum is
 *   S_i = sum_e sum_q w_q |J_e| V(R, r_i, |x_i - x_q|) / V_R
 * (every Gauss point of every element, w_q the unit-cube Gauss weights, |J_e|
 * = V_e), which differs from V_p,i by the quadrature error and, near a wall,
 * by the part of the averaging spheres outside the mesh.  Scaling the
 * particle's lens volumes by c_i = V_p,i / S_i makes sum_q w_q |J| (1 - eps_q)
 * equal sum_i V_p,i.  A particle that reaches no Gauss point keeps c_i = 1.
 * Elements are visited when their box meets the cube of half-width R + r_i
 * around x_i; the Gauss points of the others are farther than R + r_i. */
void or_qcm_weights(const double *origin, const double *extent, const int *n_el, int k,
                    double R, int64_t n, const double *x, const double *r, double *cw)
{
    omesh m = make_mesh(origin, extent, n_el, k);
    int nq = k + 1;
    double g[8], w[8];
    or_gauss_rule(nq, g, w);
    double VR = 4.0 / 3.0 * OR_PI * R * R * R;
    double Ve = m.h[0] * m.h[1] * m.h[2];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double cut = R + r[i];
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = (int)floor((x[3 * i + a] - cut - m.x0[a]) / m.h[a]);
            hi[a] = (int)floor((x[3 * i + a] + cut - m.x0[a]) / m.h[a]);
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > m.ne[a] - 1) hi[a] = m.ne[a] - 1;
        }
        double S = 0.0;
        for (int ez = lo[2]; ez <= hi[2]; ++ez)
        for (int ey = lo[1]; ey <= hi[1]; ++ey)
        for (int ex = lo[0]; ex <= hi[0]; ++ex)
            for (int qz = 0; qz < nq; ++qz)
            for (int qy = 0; qy < nq; ++qy)
            for (int qx = 0; qx < nq; ++qx) {
                double dx = x[3 * i] - qp_coord(m.x0[0], m.h[0], ex, g[qx]);
                double dy = x[3 * i + 1] - qp_coord(m.x0[1], m.h[1], ey, g[qy]);
                double dz = x[3 * i + 2] - qp_coord(m.x0[2], m.h[2], ez, g[qz]);
                double d2 = dx * dx + dy * dy + dz * dz;
                if (!(d2 < cut * cut)) continue;
                S += w[qx] * w[qy] * w[qz] * Ve * or_lens_volume(R, r[i], sqrt(d2)) / VR;
            }
        double Vp = 4.0 / 3.0 * OR_PI * r[i] * r[i] * r[i];
        cw[i] = S > 0.0 ? Vp / S : 1.0;
    }
}

/* Particle-centroid void fraction, Eq. (void_fraction): eps_e = (V_e -
 * sum_{i in e} V_p,i) / V_e with the particle assigned to the element holding
 * its centre; copied to all quadrature points of e. */
int64_t or_pcm(const double *origin, const double *extent, const int *n_el, int k,
               int64_t n, const double *x, const double *r, double *eps_q)
{
    omesh m = make_mesh(origin, extent, n_el, k);
    int64_t E = n_elem(&m);
    int nq = k + 1, Q = nq * nq * nq;
    double Ve = m.h[0] * m.h[1] * m.h[2];
    int32_t *elem = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int64_t bad = or_locate(origin, extent, n_el, k, n, x, elem, NULL);
    double *vs = (double *)calloc(E, sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        if (elem[i] < 0) continue;
        vs[elem[i]] += 4.0 / 3.0 * OR_PI * r[i] * r[i] * r[i];
    }
    for (int64_t e = 0; e < E; ++e) {
        double eps = (Ve - vs[e]) / Ve;
        for (int q = 0; q < Q; ++q) eps_q[e * Q + q] = eps;
    }
    free(vs);
    free(elem);
    return bad;
}

/* ------------------------------------------------------------------ */
/* Smoothed L2 projection                                             */
/* ------------------------------------------------------------------ */

/* global node of local node (a,b,c) of element (ex,ey,ez) on the Q_deg grid */
static int64_t gnode(const omesh *m, int deg, int ex, int ey, int ez, int a, int b, int c)
{
    int64_t nx = nn_axis(m, 0, deg), ny = nn_axis(m, 1, deg);
    return (int64_t)(ex * deg + a) + nx * ((int64_t)(ey * deg + b) + ny * (int64_t)(ez * deg + c));
}

/* Element matrix A_e = M_e + L2 K_e of an axis-aligned box element, by 3D
 * Gauss quadrature of the basis products:
 *   M_e[i][j] = sum_q phi_i phi_j w_q |J|,
 *   K_e[i][j] = sum_q grad phi_i . grad phi_j w_q |J|,
 * local node i = a + (k+1)(b + (k+1) c). */
void or_element_matrix(int k, const double *h, double *Me, double *Ke)
{
    int np = k + 1, nq = k + 1;
    int nloc = np * np * np;
    double g[8], w[8], z[8];
    or_gauss_rule(nq, g, w);
    or_gll_nodes(k, z);
    double l[8][8], dl[8][8];
    for (int q = 0; q < nq; ++q) lagrange(k, z, g[q], l[q], dl[q]);
    double detJ = h[0] * h[1] * h[2];
    for (int i = 0; i < nloc * nloc; ++i) { Me[i] = 0.0; Ke[i] = 0.0; }
    for (int qz = 0; qz < nq; ++qz)
    for (int qy = 0; qy < nq; ++qy)
    for (int qx = 0; qx < nq; ++qx) {
        double wq = w[qx] * w[qy] * w[qz] * detJ;
        for (int i = 0; i < nloc; ++i) {
            int ia = i % np, ib = (i / np) % np, ic = i / (np * np);
            double pi = l[qx][ia] * l[qy][ib] * l[qz][ic];
            double gi0 = dl[qx][ia] / h[0] * l[qy][ib] * l[qz][ic];
            double gi1 = l[qx][ia] * dl[qy][ib] / h[1] * l[qz][ic];
            double gi2 = l[qx][ia] * l[qy][ib] * dl[qz][ic] / h[2];
            for (int j = 0; j < nloc; ++j) {
                int ja = j % np, jb = (j / np) % np, jc = j / (np * np);
                double pj = l[qx][ja] * l[qy][jb] * l[qz][jc];
                double gj0 = dl[qx][ja] / h[0] * l[qy][jb] * l[qz][jc];
                double gj1 = l[qx][ja] * dl[qy][jb] / h[1] * l[qz][jc];
                double gj2 = l[qx][ja] * l[qy][jb] * dl[qz][jc] / h[2];
                Me[i * nloc + j] += pi * pj * wq;
                Ke[i * nloc + j] += (gi0 * gj0 + gi1 * gj1 + gi2 * gj2) * wq;
            }
        }
    }
}

/* b_j = sum_e sum_q phi_j(x_q) w_q |J_e| eps_q */
void or_rhs(const double *origin, const double *extent, const int *n_el, int k,
            const double *eps_q, double *b)
{
    omesh m = make_mesh(origin, extent, n_el, k);
    int np = k + 1, nq = k + 1, Q = nq * nq * nq;
    double g[8], w[8], z[8], l[8][8];
    or_gauss_rule(nq, g, w);
    or_gll_nodes(k, z);
    for (int q = 0; q < nq; ++q) lagrange(k, z, g[q], l[q], NULL);
    int64_t nnodes = (int64_t)nn_axis(&m, 0, k) * nn_axis(&m, 1, k) * nn_axis(&m, 2, k);
    for (int64_t j = 0; j < nnodes; ++j) b[j] = 0.0;
    double detJ = m.h[0] * m.h[1] * m.h[2];
    for (int color = 0; color < 2; ++color) {
#pragma omp parallel for schedule(static)
        for (int ez = color; ez < m.ne[2]; ez += 2)
        for (int ey = 0; ey < m.ne[1]; ++ey)
        for (int ex = 0; ex < m.ne[0]; ++ex) {
            int64_t e = ex + (int64_t)m.ne[0] * (ey + (int64_t)m.ne[1] * ez);
            for (int qz = 0; qz < nq; ++qz)
            for (int qy = 0; qy < nq; ++qy)
            for (int qx = 0; qx < nq; ++qx) {
                int q = qx + nq * (qy + nq * qz);
                double wq = w[qx] * w[qy] * w[qz] * detJ;
                double val = eps_q[e * Q + q];
                for (int c = 0; c < np; ++c)
                for (int bb = 0; bb < np; ++bb)
                for (int a = 0; a < np; ++a) {
                    double phi = l[qx][a] * l[qy][bb] * l[qz][c];
                    b[gnode(&m, k, ex, ey, ez, a, bb, c)] += phi * wq * val;
                }
            }
        }
    }
}

/* y = (M + L2 K) x, assembled element by element from the element matrix.
 * Elements are visited in slabs of even then odd ez so that no two threads
 * add into the same node. */
void or_apply(const double *origin, const double *extent, const int *n_el, int k, double L2,
              const double *xv, double *y)
{
    omesh m = make_mesh(origin, extent, n_el, k);
    int np = k + 1, nloc = np * np * np;
    double *Me = (double *)malloc(sizeof(double) * nloc * nloc);
    double *Ke = (double *)malloc(sizeof(double) * nloc * nloc);
    or_element_matrix(k, m.h, Me, Ke);
    double *Ae = (double *)malloc(sizeof(double) * nloc * nloc);
    for (int i = 0; i < nloc * nloc; ++i) Ae[i] = Me[i] + L2 * Ke[i];
    int64_t nnodes = (int64_t)nn_axis(&m, 0, k) * nn_axis(&m, 1, k) * nn_axis(&m, 2, k);
    for (int64_t j = 0; j < nnodes; ++j) y[j] = 0.0;
    for (int color = 0; color < 2; ++color) {
#pragma omp parallel for schedule(static)
        for (int ez = color; ez < m.ne[2]; ez += 2) {
            int64_t idx[64];
            double xl[64];
            for (int ey = 0; ey < m.ne[1]; ++ey)
            for (int ex = 0; ex < m.ne[0]; ++ex) {
                for (int i = 0; i < nloc; ++i) {
                    int a = i % np, b = (i / np) % np, c = i / (np * np);
                    idx[i] = gnode(&m, k, ex, ey, ez, a, b, c);
                    xl[i] = xv[idx[i]];
                }
                for (int i = 0; i < nloc; ++i) {
                    double s = 0.0;
                    for (int j = 0; j < nloc; ++j) s += Ae[i * nloc + j] * xl[j];
                    y[idx[i]] += s;
                }
            }
        }
    }
    free(Me);
    free(Ke);
    free(Ae);
}

/* diagonal of the assembled (M + L2 K) */
void or_diag(const double *origin, const double *extent, const int *n_el, int k, double L2,
             double *dg)
{
    omesh m = make_mesh(origin, extent, n_el, k);
    int np = k + 1, nloc = np * np * np;
    double *Me = (double *)malloc(sizeof(double) * nloc * nloc);
    double *Ke = (double *)malloc(sizeof(double) * nloc * nloc);
    or_element_matrix(k, m.h, Me, Ke);
    int64_t nnodes = (int64_t)nn_axis(&m, 0, k) * nn_axis(&m, 1, k) * nn_axis(&m, 2, k);
    for (int64_t j = 0; j < nnodes; ++j) dg[j] = 0.0;
    for (int ez = 0; ez < m.ne[2]; ++ez)
    for (int ey = 0; ey < m.ne[1]; ++ey)
    for (int ex = 0; ex < m.ne[0]; ++ex)
    for (int i = 0; i < nloc; ++i) {
        int a = i % np, b = (i / np) % np, c = i / (np * np);
        dg[gnode(&m, k, ex, ey, ez, a, b, c)] += Me[i * nloc + i] + L2 * Ke[i * nloc + i];
    }
    free(Me);
    free(Ke);
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Jacobi-preconditioned conjugate gradients on (M + L2 K) x = b; x holds the
 * start vector on entry.  Stops when ||r||_2 <= rtol ||b||_2.  Returns the
 * number of iterations, or -1 if maxit was reached first. */
int or_cg(const double *origin, const double *extent, const int *n_el, int k, double L2,
          const double *b, double *xv, double rtol, int maxit, double *relres)
{
    omesh m = make_mesh(origin, extent, n_el, k);
    int64_t nn = (int64_t)nn_axis(&m, 0, k) * nn_axis(&m, 1, k) * nn_axis(&m, 2, k);
    double *dg = (double *)malloc(sizeof(double) * nn);
    double *rv = (double *)malloc(sizeof(double) * nn);
    double *zv = (double *)malloc(sizeof(double) * nn);
    double *pv = (double *)malloc(sizeof(double) * nn);
    double *Ap = (double *)malloc(sizeof(double) * nn);
    or_diag(origin, extent, n_el, k, L2, dg);
    or_apply(origin, extent, n_el, k, L2, xv, Ap);
    for (int64_t i = 0; i < nn; ++i) rv[i] = b[i] - Ap[i];
    double bn = sqrt(dot(nn, b, b));
    if (bn == 0.0) bn = 1.0;
    for (int64_t i = 0; i < nn; ++i) zv[i] = rv[i] / dg[i];
    for (int64_t i = 0; i < nn; ++i) pv[i] = zv[i];
    double rz = dot(nn, rv, zv);
    double res = sqrt(dot(nn, rv, rv)) / bn;
    int it = 0;
    while (res > rtol && it < maxit) {
        or_apply(origin, extent, n_el, k, L2, pv, Ap);
        double alpha = rz / dot(nn, pv, Ap);
        for (int64_t i = 0; i < nn; ++i) xv[i] += alpha * pv[i];
        for (int64_t i = 0; i < nn; ++i) rv[i] -= alpha * Ap[i];
        for (int64_t i = 0; i < nn; ++i) zv[i] = rv[i] / dg[i];
        double rz_new = dot(nn, rv, zv);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < nn; ++i) pv[i] = zv[i] + beta * pv[i];
        res = sqrt(dot(nn, rv, rv)) / bn;
        ++it;
    }
    if (relres) *relres = res;
    free(dg);
    free(rv);
    free(zv);
    free(pv);
    free(Ap);
    return res <= rtol ? it : -1;
}

/* ------------------------------------------------------------------ */
/* Particle-fluid forces                                              */
/* ------------------------------------------------------------------ */

/* C_D |U| of the Dallavalle correlation, C_D = (0.63 + 4.8/sqrt(Re_p))^2
 * with Re_p = rho eps |U| d / mu, written as
 * (0.63 sqrt|U| + 4.8 sqrt(mu / (rho eps d)))^2 so that |U| -> 0 is finite. */
double or_cd_times_speed_dallavalle(double rho, double mu, double eps, double speed, double dp)
{
    double a = 0.63 * sqrt(speed) + 4.8 * sqrt(mu / (rho * eps * dp));
    return a * a;
}

double or_reynolds(double rho, double mu, double eps, double speed, double dp)
{
    return rho * eps * speed * dp / mu;
}

/* Di Felice exponent chi = 3.7 - 0.65 exp(-(1.5 - log10 Re)^2 / 2) */
double or_difelice_chi(double Re)
{
    double re = Re > 1e-300 ? Re : 1e-300;
    double t = 1.5 - log10(re);
    return 3.7 - 0.65 * exp(-(t * t) / 2.0);
}

/* Rong et al. exponent 2.65 (eps + 1) - (5.3 - 3.5 eps) eps^2
 * exp(-(1.5 - log10 Re)^2 / 2); C_D is Dallavalle times eps^(2 - it). */
double or_rong_exponent(double eps, double Re)
{
    double re = Re > 1e-300 ? Re : 1e-300;
    double t = 1.5 - log10(re);
    return 2.65 * (eps + 1.0) - (5.3 - 3.5 * eps) * eps * eps * exp(-(t * t) / 2.0);
}

/* Koch-Hill F_0(eps_p): the dilute rational form below eps_p = 0.4, with
 * eps_p ln eps_p taken as its limit 0 at eps_p = 0; 10 eps_p / eps_f^3 from
 * 0.4 up. */
double or_koch_hill_f0(double eps_p)
{
    double eps_f = 1.0 - eps_p;
    if (eps_p >= 0.4) return 10.0 * eps_p / (eps_f * eps_f * eps_f);
    double plogp = eps_p > 0.0 ? eps_p * log(eps_p) : 0.0;
    double num = 1.0 + 3.0 * sqrt(eps_p / 2.0) + 135.0 / 64.0 * plogp + 16.14 * eps_p;
    double den = 1.0 + 0.681 * eps_p - 8.48 * eps_p * eps_p + 8.14 * eps_p * eps_p * eps_p;
    return num / den;
}

/* Koch-Hill F_3(eps_p) = 0.0673 + 0.212 eps_p + 0.0232 / eps_f^5 */
double or_koch_hill_f3(double eps_p)
{
    double eps_f = 1.0 - eps_p;
    return 0.0673 + 0.212 * eps_p + 0.0232 / pow(eps_f, 5.0);
}

/* Beetstra normalised drag F_i(eps_f, Re) with the bracket read as one
 * fraction:
 *   10 eps_p / eps_f^2 + eps_f^2 (1 + 1.5 sqrt(eps_p))
 *   + 0.413 Re / (24 eps_f^2) (1/eps_f + 3 eps_p eps_f + 8.4 Re^-0.343)
 *                            / (1 + 10^(3 eps_p) Re^(-(1 + 4 eps_p)/2)). */
double or_beetstra_f(double eps_f, double Re)
{
    double eps_p = 1.0 - eps_f;
    double a = 10.0 * eps_p / (eps_f * eps_f) + eps_f * eps_f * (1.0 + 1.5 * sqrt(eps_p));
    if (Re <= 0.0) return a;
    double num = 1.0 / eps_f + 3.0 * eps_p * eps_f + 8.4 * pow(Re, -0.343);
    double den = 1.0 + pow(10.0, 3.0 * eps_p) * pow(Re, -(1.0 + 4.0 * eps_p) / 2.0);
    return a + 0.413 * Re / (24.0 * eps_f * eps_f) * num / den;
}

/* Drag coefficient of the Schiller-Naumann law used by Gidaspow above
 * eps_f = 0.8: 24/Re (1 + 0.15 Re^0.687) below Re = 1000, 0.44 above. */
double or_schiller_naumann_cd(double Re)
{
    return Re < 1000.0 ? 24.0 / Re * (1.0 + 0.15 * pow(Re, 0.687)) : 0.44;
}

/* Drag force on one particle of radius rp with slip U = u_f - u_p, eps the
 * (clamped) fluid fraction, Re = rho eps |U| d / mu (Sec. 2.3.2):
 *   0 Di Felice  1/2 rho C_D pi rp^2 |U| U, C_D Dallavalle x eps^(2 - chi)
 *   1 Dallavalle 1/2 rho C_D pi rp^2 |U| U, C_D = (0.63 + 4.8/sqrt(Re))^2
 *   2 Rong       as Di Felice with the Rong exponent
 *   3 Koch-Hill  beta U, beta = 18 mu eps^2 eps_p / d^2 (F_0 + F_3 Re / 2) V_p / eps_p,
 *                evaluated with eps_p cancelled (finite at eps_p = 0)
 *   4 Gidaspow   the printed beta is per unit volume of the mixture; one
 *                particle takes the share V_p / eps_p of it, so the force
 *                is beta V_p / eps_p U, again with eps_p cancelled: Ergun
 *                below eps = 0.8 (|U| for the printed vector), Wen-Yu with
 *                the Schiller-Naumann C_D from 0.8 up
 *   5 Beetstra   3 pi mu d eps F_i U (the slip U for the printed u_f)
 * divided by eps when beta_over_eps (beta_B = beta_A / eps). */
void or_drag_force(int model, int beta_over_eps, double rho, double mu, double eps,
                   const double *U, double rp, double *fd)
{
    double speed = sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
    if (speed == 0.0) { fd[0] = fd[1] = fd[2] = 0.0; return; }
    double dp = 2.0 * rp;
    double Re = or_reynolds(rho, mu, eps, speed, dp);
    double Vp = 4.0 / 3.0 * OR_PI * rp * rp * rp;
    double eps_p = 1.0 - eps;
    double coef;
    if (model <= 2) {
        double cds = or_cd_times_speed_dallavalle(rho, mu, eps, speed, dp);
        if (model == 0) cds = cds * pow(eps, 2.0 - or_difelice_chi(Re));
        if (model == 2) cds = cds * pow(eps, 2.0 - or_rong_exponent(eps, Re));
        coef = 0.5 * rho * cds * OR_PI * rp * rp;
    } else if (model == 3) {
        coef = 18.0 * mu * eps * eps / (dp * dp) *
               (or_koch_hill_f0(eps_p) + 0.5 * or_koch_hill_f3(eps_p) * Re) * Vp;
    } else if (model == 4) {
        double beta_over_epsp;   /* beta / eps_p */
        if (eps < 0.8) {
            beta_over_epsp = 150.0 * eps_p * mu / (eps * dp * dp) + 1.75 * rho * speed / dp;
        } else {
            double cd = or_schiller_naumann_cd(Re);
            beta_over_epsp = 0.75 * cd * eps * speed * rho / dp * pow(eps, -2.65);
        }
        coef = beta_over_epsp * Vp;
    } else {
        coef = 3.0 * OR_PI * mu * dp * eps * or_beetstra_f(eps, Re);
    }
    if (beta_over_eps) coef = coef / eps;
    for (int a = 0; a < 3; ++a) fd[a] = coef * U[a];
}

/* Per-particle forces (Sec. 2.3.2):
 *   u_f, eps at x_i by Q_k interpolation, grad p by Q_kp interpolation;
 *   eps_c = min(max(eps, eps_floor), 1) used in the closures only;
 *   f_D (drag), f_B = -rho V_p g, f_gradp = -V_p grad p,
 *   f = f_D + f_B + f_gradp.
 * Outputs may be NULL except f.  Returns the first particle outside the
 * mesh, or -1. */
int64_t or_forces(const double *origin, const double *extent, const int *n_el, int k, int kp,
                  double rho, double mu, const double *grav, int drag_model, int beta_over_eps,
                  double eps_floor, int64_t n, const double *x, const double *r,
                  const double *u_p, const double *u_nodal, const double *p_nodal,
                  const double *eps_nodal, double *f, double *f_drag, double *f_gradp,
                  double *eps_at_p)
{
    omesh m = make_mesh(origin, extent, n_el, k);
    double z[8], zp[8];
    or_gll_nodes(k, z);
    or_gll_nodes(kp, zp);
    int64_t bad = -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int ie[3];
        double xi[3];
        int ok = 1;
        for (int a = 0; a < 3; ++a)
            ok &= locate_axis(x[3 * i + a], m.x0[a], m.L[a], m.h[a], m.ne[a], &ie[a], &xi[a]);
        if (!ok) {
#pragma omp critical
            { if (bad < 0 || i < bad) bad = i; }
            for (int a = 0; a < 3; ++a) f[3 * i + a] = 0.0;
            continue;
        }
        double lx[8], ly[8], lz[8];
        lagrange(k, z, xi[0], lx, NULL);
        lagrange(k, z, xi[1], ly, NULL);
        lagrange(k, z, xi[2], lz, NULL);
        double uf[3] = {0.0, 0.0, 0.0}, eps = 0.0;
        for (int c = 0; c <= k; ++c)
        for (int b = 0; b <= k; ++b)
        for (int a = 0; a <= k; ++a) {
            double phi = lx[a] * ly[b] * lz[c];
            int64_t nd = gnode(&m, k, ie[0], ie[1], ie[2], a, b, c);
            uf[0] += phi * u_nodal[3 * nd];
            uf[1] += phi * u_nodal[3 * nd + 1];
            uf[2] += phi * u_nodal[3 * nd + 2];
            eps += phi * eps_nodal[nd];
        }
        double px[8], py[8], pz[8], dpx[8], dpy[8], dpz[8];
        lagrange(kp, zp, xi[0], px, dpx);
        lagrange(kp, zp, xi[1], py, dpy);
        lagrange(kp, zp, xi[2], pz, dpz);
        /* grad p of the Q_kp interpolant.  Its derivative along an axis
         * sees the nodal values only through their differences along that
         * axis (the derivative of a constant is zero, so each dl sums to
         * zero): d/dx = sum dl_a l_b l_c (p_abc - p_0bc) / h_x, and so on.
         * Written with the differences, a pressure that varies along one
         * axis only leaves the other two components exactly zero instead of
         * the rounding of sum_a dl_a p. */
        double gp[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c <= kp; ++c)
        for (int b = 0; b <= kp; ++b)
        for (int a = 0; a <= kp; ++a) {
            double pv = p_nodal[gnode(&m, kp, ie[0], ie[1], ie[2], a, b, c)];
            double p0x = p_nodal[gnode(&m, kp, ie[0], ie[1], ie[2], 0, b, c)];
            double p0y = p_nodal[gnode(&m, kp, ie[0], ie[1], ie[2], a, 0, c)];
            double p0z = p_nodal[gnode(&m, kp, ie[0], ie[1], ie[2], a, b, 0)];
            gp[0] += dpx[a] / m.h[0] * py[b] * pz[c] * (pv - p0x);
            gp[1] += px[a] * dpy[b] / m.h[1] * pz[c] * (pv - p0y);
            gp[2] += px[a] * py[b] * dpz[c] / m.h[2] * (pv - p0z);
        }
        double epsc = eps;
        if (epsc < eps_floor) epsc = eps_floor;
        if (epsc > 1.0) epsc = 1.0;
        double U[3] = {uf[0] - u_p[3 * i], uf[1] - u_p[3 * i + 1], uf[2] - u_p[3 * i + 2]};
        double fd[3];
        or_drag_force(drag_model, beta_over_eps, rho, mu, epsc, U, r[i], fd);
        double Vp = 4.0 / 3.0 * OR_PI * r[i] * r[i] * r[i];
        for (int a = 0; a < 3; ++a) {
            double fb = -rho * Vp * grav[a];
            double fg = -Vp * gp[a];
            f[3 * i + a] = fd[a] + fb + fg;
            if (f_drag) f_drag[3 * i + a] = fd[a];
            if (f_gradp) f_gradp[3 * i + a] = fg;
        }
        if (eps_at_p) eps_at_p[i] = eps;
    }
    return bad;
}

/* Shear force on each particle, F_div_tau = -V_p div tau (Sec. 2.3.2,
 * undisturbed-flow forces), with the deviatoric stress of Eq. (stress),
 * tau = mu (grad u + grad u^T) - 2/3 mu (div u) I, whose divergence is
 *   (div tau)_a = mu sum_b d_b d_b u_a + mu/3 d_a (sum_b d_b u_b),
 * all second derivatives taken of the Q_k interpolant of u at x_i (the
 * element's tensor Lagrange basis, chain rule 1/h per axis).  f_shear[n][3].
 * Returns the first particle outside the mesh, or -1 (its force is 0). */
int64_t or_shear_force(const double *origin, const double *extent, const int *n_el, int k,
                       double mu, int64_t n, const double *x, const double *r,
                       const double *u_nodal, double *f_shear)
{
    omesh m = make_mesh(origin, extent, n_el, k);
    double z[8];
    or_gll_nodes(k, z);
    int64_t bad = -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int ie[3];
        double xi[3];
        int ok = 1;
        for (int a = 0; a < 3; ++a)
            ok &= locate_axis(x[3 * i + a], m.x0[a], m.L[a], m.h[a], m.ne[a], &ie[a], &xi[a]);
        if (!ok) {
#pragma omp critical
            { if (bad < 0 || i < bad) bad = i; }
            for (int a = 0; a < 3; ++a) f_shear[3 * i + a] = 0.0;
            continue;
        }
        double l[3][8], dl[3][8], ddl[3][8];
        for (int a = 0; a < 3; ++a) {
            lagrange(k, z, xi[a], l[a], dl[a]);
            lagrange_dd(k, z, xi[a], ddl[a]);
        }
        /* H[c][p][q] = d_p d_q u_c at x_i */
        double H[3][3][3];
        memset(H, 0, sizeof(H));
        for (int cz = 0; cz <= k; ++cz)
        for (int cy = 0; cy <= k; ++cy)
        for (int cx = 0; cx <= k; ++cx) {
            int64_t nd = gnode(&m, k, ie[0], ie[1], ie[2], cx, cy, cz);
            int idx[3] = {cx, cy, cz};
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) {
                    /* d_p d_q of phi = prod_axis (derivative order along axis) */
                    double w = 1.0;
                    for (int a = 0; a < 3; ++a) {
                        int order = (a == p) + (a == q);
                        double v = order == 0 ? l[a][idx[a]]
                                 : order == 1 ? dl[a][idx[a]] : ddl[a][idx[a]];
                        for (int o = 0; o < order; ++o) v /= m.h[a];
                        w *= v;
                    }
                    for (int c = 0; c < 3; ++c) H[c][p][q] += w * u_nodal[3 * nd + c];
                }
        }
        double Vp = 4.0 / 3.0 * OR_PI * r[i] * r[i] * r[i];
        for (int a = 0; a < 3; ++a) {
            double lap = H[a][0][0] + H[a][1][1] + H[a][2][2];
            double graddiv = H[0][a][0] + H[1][a][1] + H[2][a][2];
            f_shear[3 * i + a] = -Vp * (mu * lap + mu / 3.0 * graddiv);
        }
    }
    return bad;
}

/* Fluid source per element, Eqs. (fa)/(fb): F_pf,e = -(1/V_e) sum_{i in e} S_i
 * with S_i = f_D,i (model A, vans_model 0) or f_D,i + f_gradp,i (+ f_shear,i
 * when given) (model B).
 * F_e[E][3]; the same value holds at every quadrature point of e. */
int64_t or_fluid_source(const double *origin, const double *extent, const int *n_el, int k,
                        int vans_model, int64_t n, const double *x, const double *f_drag,
                        const double *f_gradp, const double *f_shear, double *F_e)
{
    omesh m = make_mesh(origin, extent, n_el, k);
    int64_t E = n_elem(&m);
    double Ve = m.h[0] * m.h[1] * m.h[2];
    int32_t *elem = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int64_t bad = or_locate(origin, extent, n_el, k, n, x, elem, NULL);
    double *S = (double *)calloc(3 * E, sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        if (elem[i] < 0) continue;
        for (int a = 0; a < 3; ++a) {
            double s = f_drag[3 * i + a];
            if (vans_model == 1) s += f_gradp[3 * i + a];
            if (vans_model == 1 && f_shear) s += f_shear[3 * i + a];
            S[3 * (int64_t)elem[i] + a] += s;
        }
    }
    for (int64_t e = 0; e < 3 * E; ++e) F_e[e] = -S[e] / Ve;
    free(S);
    free(elem);
    return bad;
}

/* Fluid source with the fluid-side drag of Sec. 2.3.2 (the single-particle
 * drag written with the fluid velocity at the quadrature point and the mean
 * particle velocity of the cell):
 *   F_pf(x_q) = -beta_e (u_f(x_q) - u_p,avg,e) - (1/V_e) sum_{i in e} T_i,
 * beta_e = (1/V_e) sum_{i in e} beta_i, beta_i the particle's drag
 * coefficient (f_D,i = beta_i (u_f(x_i) - u_p,i)), u_p,avg,e the plain mean
 * of the particle velocities in e, T_i = 0 (model A) or f_gradp,i (+
 * f_shear,i when given) (model B).  beta_i is recovered from f_D,i and the
 * slip at the particle (Q_k interpolation of u at x_i).  An element without
 * particles has beta_e = 0.  F_q[E][Q][3] with q = qx + nq (qy + nq qz);
 * F_e[E][3] is the Gauss average of F_q (the element mean of F_pf). */
int64_t or_fluid_source_semi(const double *origin, const double *extent, const int *n_el,
                             int k, int vans_model, int64_t n, const double *x,
                             const double *u_p, const double *u_nodal, const double *f_drag,
                             const double *f_gradp, const double *f_shear, double *F_q,
                             double *F_e)
{
    omesh m = make_mesh(origin, extent, n_el, k);
    int64_t E = n_elem(&m);
    int nq = k + 1, Q = nq * nq * nq;
    double Ve = m.h[0] * m.h[1] * m.h[2];
    double z[8], g[8], w[8];
    or_gll_nodes(k, z);
    or_gauss_rule(nq, g, w);
    int32_t *elem = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    double *xi = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    int64_t bad = or_locate(origin, extent, n_el, k, n, x, elem, xi);
    double *B = (double *)calloc(E, sizeof(double));
    double *U = (double *)calloc(3 * E, sizeof(double));
    double *T = (double *)calloc(3 * E, sizeof(double));
    double *cnt = (double *)calloc(E, sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        if (elem[i] < 0) continue;
        int64_t e = elem[i];
        int ie[3] = {(int)(e % m.ne[0]), (int)((e / m.ne[0]) % m.ne[1]),
                     (int)(e / ((int64_t)m.ne[0] * m.ne[1]))};
        double lx[8], ly[8], lz[8];
        lagrange(k, z, xi[3 * i], lx, NULL);
        lagrange(k, z, xi[3 * i + 1], ly, NULL);
        lagrange(k, z, xi[3 * i + 2], lz, NULL);
        double uf[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c <= k; ++c)
        for (int b = 0; b <= k; ++b)
        for (int a = 0; a <= k; ++a) {
            int64_t nd = gnode(&m, k, ie[0], ie[1], ie[2], a, b, c);
            for (int d = 0; d < 3; ++d) uf[d] += lx[a] * ly[b] * lz[c] * u_nodal[3 * nd + d];
        }
        double slip[3], num = 0.0, den = 0.0;
        for (int d = 0; d < 3; ++d) {
            slip[d] = uf[d] - u_p[3 * i + d];
            num += f_drag[3 * i + d] * slip[d];
            den += slip[d] * slip[d];
        }
        B[e] += den > 0.0 ? num / den : 0.0;
        cnt[e] += 1.0;
        for (int d = 0; d < 3; ++d) {
            U[3 * e + d] += u_p[3 * i + d];
            double t = 0.0;
            if (vans_model == 1) t += f_gradp[3 * i + d];
            if (vans_model == 1 && f_shear) t += f_shear[3 * i + d];
            T[3 * e + d] += t;
        }
    }
    for (int64_t e = 0; e < E; ++e) {
        int ie[3] = {(int)(e % m.ne[0]), (int)((e / m.ne[0]) % m.ne[1]),
                     (int)(e / ((int64_t)m.ne[0] * m.ne[1]))};
        double beta = B[e] / Ve, upa[3] = {0.0, 0.0, 0.0};
        if (cnt[e] > 0.0)
            for (int d = 0; d < 3; ++d) upa[d] = U[3 * e + d] / cnt[e];
        double mean[3] = {0.0, 0.0, 0.0};
        for (int qz = 0; qz < nq; ++qz)
        for (int qy = 0; qy < nq; ++qy)
        for (int qx = 0; qx < nq; ++qx) {
            double lx[8], ly[8], lz[8];
            lagrange(k, z, g[qx], lx, NULL);
            lagrange(k, z, g[qy], ly, NULL);
            lagrange(k, z, g[qz], lz, NULL);
            double uf[3] = {0.0, 0.0, 0.0};
            for (int c = 0; c <= k; ++c)
            for (int b = 0; b <= k; ++b)
            for (int a = 0; a <= k; ++a) {
                int64_t nd = gnode(&m, k, ie[0], ie[1], ie[2], a, b, c);
                for (int d = 0; d < 3; ++d) uf[d] += lx[a] * ly[b] * lz[c] * u_nodal[3 * nd + d];
            }
            int q = qx + nq * (qy + nq * qz);
            for (int d = 0; d < 3; ++d) {
                double F = -beta * (uf[d] - upa[d]) - T[3 * e + d] / Ve;
                F_q[(e * Q + q) * 3 + d] = F;
                mean[d] += w[qx] * w[qy] * w[qz] * F;
            }
        }
        for (int d = 0; d < 3; ++d) F_e[3 * e + d] = mean[d];
    }
    free(cnt);
    free(T);
    free(U);
    free(B);
    free(xi);
    free(elem);
    return bad;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------ */
/* Location on a mapped (isoparametric) Q_k hex mesh                   */
/* ------------------------------------------------------------------ */

/* The paper's beds sit in curved meshes (a subdivided cylinder, Secs. 3.1 and
 * 3.2; a gmsh mesh of the spouted bed, Sec. 3.4), and particles are located
 * on the fluid mesh itself (Sec. 2.3).  Element e maps the reference cube
 * [0,1]^3 onto space by its Q_k nodes:
 *   X_e(xi) = sum_{a,b,c} P[conn[e][a + (k+1)(b + (k+1) c)]] l_a(xi_0) l_b(xi_1) l_c(xi_2)
 * with the GLL Lagrange basis l.  A point x lies in e when X_e(xi) = x for a
 * xi in the cube.  The oracle tries the candidate elements -- those whose
 * node box, widened on every side by `margin` times its largest edge,
 * contains x -- in ascending index, each by Newton's method
 *   xi <- xi - J(xi)^-1 (X_e(xi) - x),   J = dX_e / dxi,
 * from the cube's centre: at most 50 steps, converged once the largest step
 * component is at most 1e-13, abandoned once xi leaves [-3, 4]^3 or J is
 * singular.  The first candidate whose converged xi lies in [-1e-10,
 * 1 + 1e-10]^3 is the element, and xi is clamped to [0,1]^3; a point in no
 * element gets elem = -1, xi = 0.  Returns the number of such points. */

static void mapped_box(int k, const int32_t *conn, const double *nodes, int64_t e,
                       double margin, double *lo, double *hi)
{
    int nloc = (k + 1) * (k + 1) * (k + 1);
    for (int a = 0; a < 3; ++a) { lo[a] = INFINITY; hi[a] = -INFINITY; }
    for (int j = 0; j < nloc; ++j) {
        const double *P = nodes + 3 * (int64_t)conn[e * nloc + j];
        for (int a = 0; a < 3; ++a) {
            if (P[a] < lo[a]) lo[a] = P[a];
            if (P[a] > hi[a]) hi[a] = P[a];
        }
    }
    double side = 0.0;
    for (int a = 0; a < 3; ++a) if (hi[a] - lo[a] > side) side = hi[a] - lo[a];
    double w = margin * side;
    for (int a = 0; a < 3; ++a) { lo[a] -= w; hi[a] += w; }
}

/* Newton inversion of X_e at x; returns 1 and xi in the widened cube, else 0 */
static int mapped_newton(int k, const double *z, const int32_t *conn, const double *nodes,
                         int64_t e, const double *x, double *xi_out)
{
    int nq = k + 1, nloc = nq * nq * nq;
    double xi[3] = {0.5, 0.5, 0.5};
    for (int it = 0; it < 50; ++it) {
        double l[3][4], dl[3][4];
        for (int a = 0; a < 3; ++a) lagrange(k, z, xi[a], l[a], dl[a]);
        double X[3] = {0.0, 0.0, 0.0}, J[3][3] = {{0.0}};   /* J[i][a] = dX_i/dxi_a */
        for (int c = 0; c < nq; ++c)
        for (int b = 0; b < nq; ++b)
        for (int a = 0; a < nq; ++a) {
            const double *P = nodes + 3 * (int64_t)conn[e * nloc + a + nq * (b + nq * c)];
            double w = l[0][a] * l[1][b] * l[2][c];
            double w0 = dl[0][a] * l[1][b] * l[2][c];
            double w1 = l[0][a] * dl[1][b] * l[2][c];
            double w2 = l[0][a] * l[1][b] * dl[2][c];
            for (int i = 0; i < 3; ++i) {
                X[i] += w * P[i];
                J[i][0] += w0 * P[i];
                J[i][1] += w1 * P[i];
                J[i][2] += w2 * P[i];
            }
        }
        double r[3] = {X[0] - x[0], X[1] - x[1], X[2] - x[2]};
        /* J d = r by Cramer's rule */
        double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
                   - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
                   + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!(fabs(det) > 0.0)) return 0;
        double d[3];
        for (int col = 0; col < 3; ++col) {
            double M[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) M[i][j] = (j == col) ? r[i] : J[i][j];
            double dm = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
                      - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
                      + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
            d[col] = dm / det;
        }
        double big = 0.0;
        for (int a = 0; a < 3; ++a) {
            xi[a] -= d[a];
            if (fabs(d[a]) > big) big = fabs(d[a]);
            if (!(xi[a] >= -3.0 && xi[a] <= 4.0)) return 0;
        }
        if (big <= 1e-13) {
            for (int a = 0; a < 3; ++a)
                if (!(xi[a] >= -1e-10 && xi[a] <= 1.0 + 1e-10)) return 0;
            for (int a = 0; a < 3; ++a)
                xi_out[a] = xi[a] < 0.0 ? 0.0 : (xi[a] > 1.0 ? 1.0 : xi[a]);
            return 1;
        }
    }
    return 0;
}

int64_t or_locate_mapped(int k, int64_t E, const int32_t *conn, const double *nodes,
                         double margin, int64_t n, const double *x, int32_t *elem, double *xi)
{
    double z[8];
    or_gll_nodes(k, z);
    double *box = (double *)malloc(sizeof(double) * 6 * (E > 0 ? E : 1));
    for (int64_t e = 0; e < E; ++e) mapped_box(k, conn, nodes, e, margin, box + 6 * e, box + 6 * e + 3);
    int64_t missing = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : missing)
    for (int64_t i = 0; i < n; ++i) {
        const double *p = x + 3 * i;
        elem[i] = -1;
        xi[3 * i] = xi[3 * i + 1] = xi[3 * i + 2] = 0.0;
        for (int64_t e = 0; e < E; ++e) {
            const double *lo = box + 6 * e, *hi = lo + 3;
            if (!(p[0] >= lo[0] && p[0] <= hi[0] && p[1] >= lo[1] && p[1] <= hi[1] &&
                  p[2] >= lo[2] && p[2] <= hi[2]))
                continue;
            if (mapped_newton(k, z, conn, nodes, e, p, xi + 3 * i)) {
                elem[i] = (int32_t)e;
                break;
            }
        }
        if (elem[i] < 0) ++missing;
    }
    free(box);
    return missing;
}

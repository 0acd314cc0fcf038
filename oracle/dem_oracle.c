/*
 * dem_oracle.c -- plain FP64 CPU oracle of the DEM step of "Towards
 * High-Order CFD-DEM: Development and Validation" (arXiv 2211.01185).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests use it.  It shares no code, header or
 * constant with the CUDA library.
 *
 * What it computes (Sec. 2.2):
 *   Newton's laws for translation and rotation, Eqs. (newton_law) and
 *   (angular_momentum): m dv/dt = sum_j f_ij + sum_w f_wi + m g + f_fp,
 *   I dw/dt = sum_j (M^t_ij + M^r_ij), I = 2/5 m r^2.
 *   Soft-sphere contacts with the non-linear visco-elastic model of Table
 *   (viscoelastic): k_n = 4/3 Y_e sqrt(R_e d_n), eta_n = -2 sqrt(5/6) beta
 *   sqrt(S_n m_e), k_t = 8 G_e sqrt(R_e d_n), eta_t = -2 sqrt(5/6) beta
 *   sqrt(S_t m_e), S_n = 2 Y_e sqrt(R_e d_n), S_t = 8 G_e sqrt(R_e d_n),
 *   beta = ln e / sqrt(ln^2 e + pi^2), and the effective mass, radius,
 *   Young's and shear moduli of the table; f^n = -k_n d_n n - eta_n v_rn,
 *   f^t = -k_t d_t - eta_t v_rt (Eq. for f_ij).
 *   Velocity Verlet time integration (Sec. 2.2, after Delacroix et al.).
 *
 * Readings (the paper defers details to the Lethe-DEM paper):
 *   - n points from particle i to its partner (or to the wall); the overlap
 *     is d_n = r_i + r_j - |x_j - x_i| (walls: r_i minus the distance to the
 *     wall plane); the contact point lies at r_i n from the centre of i.
 *   - relative velocity of the contact point of i with respect to j:
 *     v_rel = v_i - v_j + (r_i w_i + r_j w_j) x n; v_rn = (v_rel . n) n,
 *     v_rt = v_rel - v_rn (walls: v_rel = v_i + r_i w_i x n).
 *   - tangential displacement d_t: carried per contact from step to step,
 *     rotated onto the current tangent plane (its normal component removed)
 *     and incremented by v_rt dt; a new contact starts from 0; a contact that
 *     opens is forgotten.
 *   - Coulomb limit (the sliding friction coefficient mu_s of Lethe): when
 *     |f^t| > mu_s |f^n|, f^t is scaled to mu_s |f^n| and d_t is reset to
 *     -(f^t + eta_t v_rt) / k_t, consistent with the limited force.
 *   - tangential torque M^t = (r_i n) x f^t; rolling resistance, constant
 *     model: M^r = -mu_r R_e |f^n| w_rel / |w_rel|, w_rel = w_i - w_j (walls:
 *     w_i), zero when w_rel = 0.
 *   - walls: the six faces of the box [lo, hi], infinitely heavy and large
 *     (m_e = m_i, R_e = r_i), with their own Young's modulus, Poisson
 *     ratio, restitution and friction coefficients.
 *   - Velocity Verlet with velocity-dependent forces: v(n+1/2) = v(n) + a(n)
 *     dt/2, x(n+1) = x(n) + v(n+1/2) dt, a(n+1) from x(n+1) and v(n+1/2),
 *     v(n+1) = v(n+1/2) + a(n+1) dt/2 (the same for w with the torques).
 *     The fluid force f_fp is held over the sub-steps of one call.
 *   - each particle sums its contacts in ascending partner index, then the
 *     walls (x-, x+, y-, y+, z-, z+), then gravity and the fluid force.
 *
 * Parameter array prm[20]: rho_p, Y, nu, e, mu_s, mu_r (particles);
 * Y_w, nu_w, e_w, mu_s_w, mu_r_w (walls); g[3]; lo[3]; hi[3].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DEM_PI 3.14159265358979323846

static void cross(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* One contact: given the unit normal n (from i towards the partner), the
 * overlap dn > 0, the contact-point relative velocity vrel, the relative
 * angular velocity wrel, the effective quantities and the carried tangential
 * displacement dt_hist (updated in place), add the force on i to F and the
 * torque on i to T. */
static void contact(const double *n, double dn, const double *vrel, const double *wrel,
                    double ri, double me, double Re, double Ye, double Ge, double e,
                    double mus, double mur, double dt, double *dt_hist, double *F, double *T)
{
    double vn = dot(vrel, n);
    double vrn[3], vrt[3];
    for (int a = 0; a < 3; ++a) {
        vrn[a] = vn * n[a];
        vrt[a] = vrel[a] - vrn[a];
    }
    double sq = sqrt(Re * dn);
    double kn = 4.0 / 3.0 * Ye * sq;
    double kt = 8.0 * Ge * sq;
    double Sn = 2.0 * Ye * sq;
    double St = 8.0 * Ge * sq;
    double le = log(e);
    double beta = le / sqrt(le * le + DEM_PI * DEM_PI);
    double etan = -2.0 * sqrt(5.0 / 6.0) * beta * sqrt(Sn * me);
    double etat = -2.0 * sqrt(5.0 / 6.0) * beta * sqrt(St * me);
    /* tangential displacement: onto the current tangent plane, then advanced */
    double hn = dot(dt_hist, n);
    for (int a = 0; a < 3; ++a) dt_hist[a] = dt_hist[a] - hn * n[a] + vrt[a] * dt;
    double fn[3], ft[3];
    for (int a = 0; a < 3; ++a) {
        fn[a] = -(kn * dn) * n[a] - etan * vrn[a];
        ft[a] = -kt * dt_hist[a] - etat * vrt[a];
    }
    double fnm = sqrt(dot(fn, fn));
    double ftm = sqrt(dot(ft, ft));
    if (ftm > mus * fnm) {
        double s = mus * fnm / ftm;
        for (int a = 0; a < 3; ++a) {
            ft[a] = ft[a] * s;
            dt_hist[a] = -(ft[a] + etat * vrt[a]) / kt;
        }
    }
    double arm[3] = {ri * n[0], ri * n[1], ri * n[2]};
    double mt[3];
    cross(arm, ft, mt);
    double wm = sqrt(dot(wrel, wrel));
    for (int a = 0; a < 3; ++a) {
        F[a] += fn[a] + ft[a];
        T[a] += mt[a];
        if (wm > 0.0) T[a] += -mur * Re * fnm * wrel[a] / wm;
    }
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* Forces and torques on every particle at the current state; the carried
 * tangential displacements advance by dt (0 for the very first evaluation).
 * hist_j[i*C + s] (partner index, -1 empty, ascending) and hist_t[...][3]
 * hold up to C contacts per particle; whist[i][6][3] the walls'.
 * Returns 0, or -1 if a particle had more than C contacts. */
int dem_forces(int64_t n, const double *prm, double dt, const double *x, const double *v,
               const double *w, const double *r, const double *f_ext, double *acc,
               double *alpha, int C, int32_t *hist_j, double *hist_t, double *whist)
{
    const double rho = prm[0], Y = prm[1], nu = prm[2], e = prm[3], mus = prm[4], mur = prm[5];
    const double Yw = prm[6], nuw = prm[7], ew = prm[8], musw = prm[9], murw = prm[10];
    const double *g = prm + 11, *lo = prm + 14, *hi = prm + 17;
    int status = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        int *cand = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
        int nc = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1],
                           x[3 * j + 2] - x[3 * i + 2]};
            double dist = sqrt(dot(d, d));
            if (dist < r[i] + r[j] && dist > 0.0) cand[nc++] = (int)j;
        }
        qsort(cand, nc, sizeof(int), cmp_int);
        double mi = rho * 4.0 / 3.0 * DEM_PI * r[i] * r[i] * r[i];
        double Ii = 0.4 * mi * r[i] * r[i];
        double F[3] = {0.0, 0.0, 0.0}, T[3] = {0.0, 0.0, 0.0};
        int32_t oj[256];
        double ot[256 * 3];
        int no = 0;
        for (int s = 0; s < C && s < 256; ++s) {
            if (hist_j[i * C + s] < 0) break;
            oj[no] = hist_j[i * C + s];
            for (int a = 0; a < 3; ++a) ot[3 * no + a] = hist_t[(i * C + s) * 3 + a];
            ++no;
        }
        if (nc > C) {
#pragma omp critical
            status = -1;
            nc = C;
        }
        for (int s = 0; s < C; ++s) hist_j[i * C + s] = -1;
        for (int c = 0; c < nc; ++c) {
            int j = cand[c];
            double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1],
                           x[3 * j + 2] - x[3 * i + 2]};
            double dist = sqrt(dot(d, d));
            double nrm[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
            double dn = r[i] + r[j] - dist;
            double mj = rho * 4.0 / 3.0 * DEM_PI * r[j] * r[j] * r[j];
            double me = 1.0 / (1.0 / mi + 1.0 / mj);
            double Re = 1.0 / (1.0 / r[i] + 1.0 / r[j]);
            double Ye = 1.0 / ((1.0 - nu * nu) / Y + (1.0 - nu * nu) / Y);
            double Ge = 1.0 / (2.0 * (2.0 - nu) * (1.0 + nu) / Y + 2.0 * (2.0 - nu) * (1.0 + nu) / Y);
            double wsum[3] = {r[i] * w[3 * i] + r[j] * w[3 * j],
                              r[i] * w[3 * i + 1] + r[j] * w[3 * j + 1],
                              r[i] * w[3 * i + 2] + r[j] * w[3 * j + 2]};
            double wxn[3];
            cross(wsum, nrm, wxn);
            double vrel[3], wrel[3];
            for (int a = 0; a < 3; ++a) {
                vrel[a] = v[3 * i + a] - v[3 * j + a] + wxn[a];
                wrel[a] = w[3 * i + a] - w[3 * j + a];
            }
            double th[3] = {0.0, 0.0, 0.0};
            for (int o = 0; o < no; ++o)
                if (oj[o] == j) {
                    for (int a = 0; a < 3; ++a) th[a] = ot[3 * o + a];
                    break;
                }
            contact(nrm, dn, vrel, wrel, r[i], me, Re, Ye, Ge, e, mus, mur, dt, th, F, T);
            hist_j[i * C + c] = j;
            for (int a = 0; a < 3; ++a) hist_t[(i * C + c) * 3 + a] = th[a];
        }
        /* walls x-, x+, y-, y+, z-, z+ */
        for (int wl = 0; wl < 6; ++wl) {
            int ax = wl / 2;
            double nrm[3] = {0.0, 0.0, 0.0};
            double dn;
            if (wl % 2 == 0) {
                nrm[ax] = -1.0;
                dn = r[i] - (x[3 * i + ax] - lo[ax]);
            } else {
                nrm[ax] = 1.0;
                dn = r[i] - (hi[ax] - x[3 * i + ax]);
            }
            double *th = whist + (i * 6 + wl) * 3;
            if (!(dn > 0.0)) {
                th[0] = th[1] = th[2] = 0.0;
                continue;
            }
            double Ye = 1.0 / ((1.0 - nu * nu) / Y + (1.0 - nuw * nuw) / Yw);
            double Ge = 1.0 / (2.0 * (2.0 - nu) * (1.0 + nu) / Y + 2.0 * (2.0 - nuw) * (1.0 + nuw) / Yw);
            double rw[3] = {r[i] * w[3 * i], r[i] * w[3 * i + 1], r[i] * w[3 * i + 2]};
            double wxn[3];
            cross(rw, nrm, wxn);
            double vrel[3] = {v[3 * i] + wxn[0], v[3 * i + 1] + wxn[1], v[3 * i + 2] + wxn[2]};
            double wrel[3] = {w[3 * i], w[3 * i + 1], w[3 * i + 2]};
            contact(nrm, dn, vrel, wrel, r[i], mi, r[i], Ye, Ge, ew, musw, murw, dt, th, F, T);
        }
        for (int a = 0; a < 3; ++a) {
            double fa = F[a] + mi * g[a] + f_ext[3 * i + a];
            acc[3 * i + a] = fa / mi;
            alpha[3 * i + a] = T[a] / Ii;
        }
        free(cand);
    }
    return status;
}

/* nsub Velocity Verlet sub-steps of length dt.  acc/alpha carry the last
 * accelerations between calls; *have_acc = 0 makes the first evaluation at
 * the current state (without advancing the tangential displacements). */
int or_dem_step(int64_t n, const double *prm, double dt, int nsub, double *x, double *v,
                double *w, const double *r, const double *f_ext, double *acc, double *alpha,
                int C, int32_t *hist_j, double *hist_t, double *whist, int *have_acc)
{
    int st = 0;
    if (!*have_acc) {
        st |= dem_forces(n, prm, 0.0, x, v, w, r, f_ext, acc, alpha, C, hist_j, hist_t, whist);
        *have_acc = 1;
    }
    for (int s = 0; s < nsub; ++s) {
        for (int64_t i = 0; i < 3 * n; ++i) {
            v[i] += 0.5 * dt * acc[i];
            w[i] += 0.5 * dt * alpha[i];
            x[i] += dt * v[i];
        }
        st |= dem_forces(n, prm, dt, x, v, w, r, f_ext, acc, alpha, C, hist_j, hist_t, whist);
        for (int64_t i = 0; i < 3 * n; ++i) {
            v[i] += 0.5 * dt * acc[i];
            w[i] += 0.5 * dt * alpha[i];
        }
    }
    return st;
}

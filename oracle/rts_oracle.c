/*
 * rts_oracle.c -- FP64 CPU oracle of the short-characteristics radiation
 * transport solve. TEST INFRASTRUCTURE ONLY: it is what the CUDA library is
 * checked against, and it shares no code with it.
 *
 * Each function follows one step of the method (paper Sect. 5.1 and the
 * "core computational loop" figure: interpol -> iterate {integrate, exchange,
 * error} -> flux), written as plain loops in the order the method states:
 *   orc_a4_quadrature      3 rays per octant, 24 directions (Sect. 2, 5.1)
 *   orc_direction_geometry upwind point of a short characteristic
 *   orc_segment_weights    linear-in-tau source integral over one segment
 *   orc_sweep_direction    integrate() in dependency order; the horizontally
 *                          periodic wrap is iterated to a tolerance, as the
 *                          paper iterates boundary intensities (Sect. 2, 5.1)
 *   orc_solve              flux(): J and F over directions, then Q_rad
 *   orc_adjoint            reverse-mode derivative of orc_solve
 * Where the paper gives no formula, the reading taken is stated at the
 * function that takes it (quadrature values, dominant axis and ties, set
 * boundary layers, linear chi interpolation, trapezoidal dtau, the periodic
 * wrap's seed and tolerance, the one-sided divergence at the bottom and top,
 * the thin/thick blend).
 */
#include "rts_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FOUR_PI (4.0 * 3.14159265358979323846)
/* Below this optical depth the segment weights use their Taylor series. */
#define SERIES_SWITCH 0.01

/* ------------------------------------------------------------------------ */
/* Quadrature                                                                */
/* ------------------------------------------------------------------------ */

void orc_a4_quadrature(double *n, double *w)
{
    /* Level-symmetric set with 3 directions per octant: every direction has
     * two components of size mu1 and one of size mu2 = sqrt(1 - 2 mu1^2).
     * mu1 is fixed by requiring the 4th moment <n_z^4> = 1/5 to be exact:
     * (1 - 2x)^2 + 2x^2 = 3/5 with x = mu1^2, i.e. x = (1 - sqrt(2/5)) / 3. */
    const double mu1 = sqrt((1.0 - sqrt(0.4)) / 3.0);
    const double mu2 = sqrt(1.0 - 2.0 * mu1 * mu1);
    int d = 0;
    /* groups: +z, -z, +x, -x, +y, -y; within a group the two minor-axis
     * signs (+,+), (-,+), (+,-), (-,-). */
    for (int grp = 0; grp < 6; ++grp) {
        int axis = grp == 0 || grp == 1 ? 2 : (grp == 2 || grp == 3 ? 0 : 1);
        double sa = (grp % 2 == 0) ? 1.0 : -1.0;
        int b1 = axis == 0 ? 1 : 0;
        int b2 = axis == 2 ? 1 : 2;
        for (int m = 0; m < 4; ++m) {
            double s1 = (m & 1) ? -1.0 : 1.0;
            double s2 = (m & 2) ? -1.0 : 1.0;
            double v[3];
            v[axis] = sa * mu2;
            v[b1] = s1 * mu1;
            v[b2] = s2 * mu1;
            n[3 * d + 0] = v[0];
            n[3 * d + 1] = v[1];
            n[3 * d + 2] = v[2];
            w[d] = 1.0 / 24.0;
            ++d;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Geometry of a short characteristic                                        */
/* ------------------------------------------------------------------------ */

int orc_direction_geometry(const orc_problem *p, int d, orc_dirgeom *g)
{
    const double h[3] = {p->dx, p->dy, p->dz};
    const double *n = p->n + 3 * d;
    /* The dominant axis is the one whose neighbouring grid plane the ray
     * reaches first going upwind: argmin h_a / |n_a|; ties go to z, then y,
     * then x. */
    int order[3] = {2, 1, 0};
    int a = -1;
    double best = 0.0;
    for (int t = 0; t < 3; ++t) {
        int ax = order[t];
        if (fabs(n[ax]) <= 0.0) continue;
        double s = h[ax] / fabs(n[ax]);
        if (a < 0 || s < best) {
            a = ax;
            best = s;
        }
    }
    if (a < 0) return ORC_EINVAL;
    if (n[2] == 0.0) return ORC_EINVAL; /* every ray must go up or down */
    g->axis = a;
    g->sa = n[a] > 0 ? 1 : -1;
    g->b1 = a == 0 ? 1 : 0;
    g->b2 = a == 2 ? 1 : 2;
    g->ds = best;
    g->s1 = n[g->b1] < 0 ? -1 : 1;
    g->s2 = n[g->b2] < 0 ? -1 : 1;
    /* the upwind point r_p - ds*n sits a fraction d of a cell towards -sign */
    g->d1 = best * fabs(n[g->b1]) / h[g->b1];
    g->d2 = best * fabs(n[g->b2]) / h[g->b2];
    if (g->d1 > 1.0) g->d1 = 1.0;
    if (g->d2 > 1.0) g->d2 = 1.0;
    g->beta[0] = (1.0 - g->d1) * (1.0 - g->d2);
    g->beta[1] = g->d1 * (1.0 - g->d2);
    g->beta[2] = (1.0 - g->d1) * g->d2;
    g->beta[3] = g->d1 * g->d2;
    g->up = n[2] > 0;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Formal solution over one segment                                          */
/* ------------------------------------------------------------------------ */

void orc_segment_weights(double x, double *e, double *w_up, double *w_p)
{
    /* S linear in optical depth t along the segment, t = 0 at the upwind end:
     * I_p = e^{-x} I_up + int_0^x S(t) e^{-(x-t)} dt
     *     = e I_up + w_up S_up + w_p S_p with
     * w_up = (1-e)/x - e and w_p = 1 - (1-e)/x. */
    *e = exp(-x);
    if (x < SERIES_SWITCH) {
        /* Taylor series of the two weights in x (from the series of e^{-x}):
         * w_p  = sum_{n>=1} (-1)^{n+1} x^n / (n+1)!
         * w_up = sum_{n>=1} (-1)^{n+1} n x^n / (n+1)!              */
        double wp = 0.0, wu = 0.0, xn = 1.0, fact = 1.0, sgn = 1.0;
        for (int k = 1; k <= 6; ++k) {
            xn *= x;
            fact *= (double)(k + 1);
            wp += sgn * xn / fact;
            wu += sgn * (double)k * xn / fact;
            sgn = -sgn;
        }
        *w_p = wp;
        *w_up = wu;
    } else {
        double one_minus_e = -expm1(-x);
        *w_up = one_minus_e / x - *e;
        *w_p = 1.0 - one_minus_e / x;
    }
}

/* d w_up / dx and d w_p / dx (used by the adjoint). */
static void segment_weight_derivs(double x, double *dwu, double *dwp)
{
    if (x < SERIES_SWITCH) {
        double wp = 0.0, wu = 0.0, xn1 = 1.0, fact = 1.0, sgn = 1.0;
        for (int k = 1; k <= 6; ++k) {
            fact *= (double)(k + 1);
            wp += sgn * (double)k * xn1 / fact;
            wu += sgn * (double)(k * k) * xn1 / fact;
            xn1 *= x;
            sgn = -sgn;
        }
        *dwp = wp;
        *dwu = wu;
    } else {
        double e = exp(-x);
        double ome = -expm1(-x);
        *dwu = e / x - ome / (x * x) + e;
        *dwp = ome / (x * x) - e / x;
    }
}

/* ------------------------------------------------------------------------ */
/* Grid helpers                                                              */
/* ------------------------------------------------------------------------ */

static inline int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

static inline size_t lin(const orc_problem *p, const int c[3])
{
    int i = wrapi(c[0], p->nx), j = wrapi(c[1], p->ny);
    return ((size_t)c[2] * (size_t)p->ny + (size_t)j) * (size_t)p->nx + (size_t)i;
}

static inline int extent(const orc_problem *p, int axis)
{
    return axis == 0 ? p->nx : (axis == 1 ? p->ny : p->nz);
}

/* index of direction d among the up (or down) directions */
static int updown_index(const orc_problem *p, int d)
{
    int up = p->n[3 * d + 2] > 0, c = 0;
    for (int e = 0; e < d; ++e)
        if ((p->n[3 * e + 2] > 0) == up) ++c;
    return c;
}

static int count_up(const orc_problem *p)
{
    int c = 0;
    for (int d = 0; d < p->ndir; ++d) c += p->n[3 * d + 2] > 0;
    return c;
}

/* Boundary value of direction d at the layer where it enters (k = 0 for up
 * rays, k = Nz-1 for down rays): the value is set, not integrated. */
static double boundary_value(const orc_problem *p, int band, int d, int i, int j, const double *S_b)
{
    int up = p->n[3 * d + 2] > 0;
    int kind = up ? p->bottom_kind : p->top_kind;
    int k = up ? 0 : p->nz - 1;
    size_t plane = (size_t)p->nx * p->ny;
    if (kind == ORC_BC_ZERO) return 0.0;
    if (kind == ORC_BC_EQUAL_S) return S_b[(size_t)k * plane + (size_t)j * p->nx + i];
    int nsel = up ? count_up(p) : p->ndir - count_up(p);
    const double *arr = up ? p->bottom_I : p->top_I;
    int u = updown_index(p, d);
    return arr[(((size_t)band * nsel + u) * p->ny + j) * p->nx + i];
}

/* Is the point at level k a boundary point (value set) for this direction? */
static inline int is_boundary_level(const orc_problem *p, const orc_dirgeom *g, int k)
{
    return g->up ? (k == 0) : (k == p->nz - 1);
}

/* The four upwind corners of point c: linear indices and weights. */
static void upwind_corners(const orc_problem *p, const orc_dirgeom *g, const int c[3],
                           size_t idx[4])
{
    for (int q = 0; q < 4; ++q) {
        int u[3] = {c[0], c[1], c[2]};
        u[g->axis] -= g->sa;
        if (q & 1) u[g->b1] -= g->s1;
        if (q & 2) u[g->b2] -= g->s2;
        idx[q] = lin(p, u);
    }
}

/* Formal solution at one point: returns I_p and, optionally, the pieces the
 * adjoint needs. */
static double solve_point(const orc_problem *p, const orc_dirgeom *g, const int c[3],
                          const double *chi_b, const double *S_b, const double *I,
                          double *Iup_o, double *Sup_o, double *dtau_o)
{
    size_t idx[4];
    upwind_corners(p, g, c, idx);
    size_t ip = lin(p, c);
    double Iup = 0.0, chiup = 0.0, Sup = 0.0;
    for (int q = 0; q < 4; ++q) {
        Iup += g->beta[q] * I[idx[q]];
        chiup += g->beta[q] * chi_b[idx[q]];
        Sup += g->beta[q] * S_b[idx[q]];
    }
    double dtau = g->ds * 0.5 * (chiup + chi_b[ip]);
    double e, wu, wp;
    orc_segment_weights(dtau, &e, &wu, &wp);
    if (Iup_o) *Iup_o = Iup;
    if (Sup_o) *Sup_o = Sup;
    if (dtau_o) *dtau_o = dtau;
    return e * Iup + wu * Sup + wp * S_b[ip];
}

/* Loop over the integrated points of plane `v` along the dominant axis
 * (points of the boundary layer of this direction are skipped). The body
 * sees the point coordinates in c[3]; `continue` skips to the next point. */
#define PLANE_LOOP(p, g, v, c)                                          \
    for (int x2_ = 0; x2_ < extent(p, (g)->b2); ++x2_)                  \
        for (int y1_ = 0; y1_ < extent(p, (g)->b1); ++y1_) {            \
            int c[3];                                                   \
            c[(g)->axis] = (v);                                         \
            c[(g)->b1] = y1_;                                           \
            c[(g)->b2] = x2_;                                           \
            if (is_boundary_level(p, g, c[2])) continue;
#define PLANE_END }

/* ------------------------------------------------------------------------ */
/* integrate(): one direction of one band                                    */
/* ------------------------------------------------------------------------ */

int orc_sweep_direction(const orc_problem *p, int band, int d,
                        const double *chi_b, const double *S_b, double *I, int *iters)
{
    orc_dirgeom g;
    int rc = orc_direction_geometry(p, d, &g);
    if (rc) return rc;
    const size_t plane = (size_t)p->nx * p->ny;

    /* boundary layer of this direction: set, not integrated */
    {
        int kb = g.up ? 0 : p->nz - 1;
        for (int j = 0; j < p->ny; ++j)
            for (int i = 0; i < p->nx; ++i)
                I[(size_t)kb * plane + (size_t)j * p->nx + i] = boundary_value(p, band, d, i, j, S_b);
    }

    const int na = extent(p, g.axis);
    if (g.axis == 2) {
        /* z-dominant: planes in order away from the boundary layer; each plane
         * depends only on the previous one, so there is no cycle. */
        int kb = g.up ? 0 : p->nz - 1;
        for (int t = 1; t < p->nz; ++t) {
            int k = kb + g.sa * t;
            PLANE_LOOP(p, &g, k, c) I[lin(p, c)] = solve_point(p, &g, c, chi_b, S_b, I, 0, 0, 0); PLANE_END
        }
        if (iters) *iters = 1;
        return ORC_OK;
    }

    /* x- or y-dominant: the horizontal period closes the dependency chain.
     * Seed the plane upwind of the first swept plane with I = S, sweep the
     * whole period, and repeat with the last plane as the new seed until it
     * no longer changes (the paper's iteration of boundary intensities). */
    const int start = g.sa > 0 ? 0 : na - 1;
    const int last = wrapi(start - g.sa, na);
    PLANE_LOOP(p, &g, last, c) I[lin(p, c)] = S_b[lin(p, c)]; PLANE_END

    size_t nlast = 0;
    PLANE_LOOP(p, &g, last, c) ++nlast; PLANE_END
    double *old = (double *)malloc((nlast ? nlast : 1) * sizeof(double));
    if (!old) return ORC_ENOMEM;
    int it = 0;
    for (;;) {
        size_t m = 0;
        PLANE_LOOP(p, &g, last, c) old[m++] = I[lin(p, c)]; PLANE_END
        for (int t = 0; t < na; ++t) {
            int v = wrapi(start + g.sa * t, na);
            PLANE_LOOP(p, &g, v, c) I[lin(p, c)] = solve_point(p, &g, c, chi_b, S_b, I, 0, 0, 0); PLANE_END
        }
        ++it;
        double res = 0.0, mx = 0.0;
        m = 0;
        PLANE_LOOP(p, &g, last, c)
            double nv = I[lin(p, c)];
            double dv = fabs(nv - old[m++]);
            if (dv > res) res = dv;
            if (fabs(nv) > mx) mx = fabs(nv);
        PLANE_END
        if (res <= p->wrap_tol * mx) break;
        if (it >= p->max_wrap_iters) {
            free(old);
            if (iters) *iters = it;
            return ORC_ENOCONV;
        }
    }
    free(old);
    if (iters) *iters = it;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* flux(): divergence stencil and Q_rad                                       */
/* ------------------------------------------------------------------------ */

/* The terms of (D_a F_a)(i,j,k) = sum coef * F_a[idx]: central differences,
 * periodic in x and y; first-order one-sided at the bottom and top layers. */
static int div_terms(int nx, int ny, int nz, double h, int axis, int i, int j, int k,
                     size_t idx[2], double coef[2])
{
    size_t plane = (size_t)nx * ny;
#define L3(I, J, K) ((size_t)(K) * plane + (size_t)(J) * nx + (size_t)(I))
    if (axis == 0) {
        idx[0] = L3(wrapi(i + 1, nx), j, k);
        idx[1] = L3(wrapi(i - 1, nx), j, k);
        coef[0] = 0.5 / h;
        coef[1] = -0.5 / h;
        return 2;
    }
    if (axis == 1) {
        idx[0] = L3(i, wrapi(j + 1, ny), k);
        idx[1] = L3(i, wrapi(j - 1, ny), k);
        coef[0] = 0.5 / h;
        coef[1] = -0.5 / h;
        return 2;
    }
    if (nz == 1) return 0;
    if (k == 0) {
        idx[0] = L3(i, j, 1);
        idx[1] = L3(i, j, 0);
        coef[0] = 1.0 / h;
        coef[1] = -1.0 / h;
    } else if (k == nz - 1) {
        idx[0] = L3(i, j, nz - 1);
        idx[1] = L3(i, j, nz - 2);
        coef[0] = 1.0 / h;
        coef[1] = -1.0 / h;
    } else {
        idx[0] = L3(i, j, k + 1);
        idx[1] = L3(i, j, k - 1);
        coef[0] = 0.5 / h;
        coef[1] = -0.5 / h;
    }
    return 2;
#undef L3
}

void orc_divergence(int nx, int ny, int nz, double dx, double dy, double dz,
                    const double *F, double *neg_div)
{
    const double h[3] = {dx, dy, dz};
    const size_t N = (size_t)nx * ny * nz;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double s = 0.0;
                for (int a = 0; a < 3; ++a) {
                    size_t idx[2];
                    double cf[2];
                    int nt = div_terms(nx, ny, nz, h[a], a, i, j, k, idx, cf);
                    for (int t = 0; t < nt; ++t) s += cf[t] * F[(size_t)a * N + idx[t]];
                }
                neg_div[((size_t)k * ny + j) * nx + i] = -s;
            }
}

static double hmin3(const orc_problem *p)
{
    double h = p->dx;
    if (p->dy < h) h = p->dy;
    if (p->dz < h) h = p->dz;
    return h;
}

/* thin/thick blend weight: 1 where a cell is optically thin, 0 where thick */
static inline double blend_omega(const orc_problem *p, double chi)
{
    return exp(-chi * hmin3(p) / p->tau_switch);
}

static int validate(const orc_problem *p)
{
    if (!p || p->nx < 1 || p->ny < 1 || p->nz < 2 || p->nbands < 1 || p->ndir < 1) return ORC_EINVAL;
    if (!(p->dx > 0 && p->dy > 0 && p->dz > 0 && p->tau_switch > 0)) return ORC_EINVAL;
    if (!p->n || !p->w) return ORC_EINVAL;
    if (p->bottom_kind == ORC_BC_EXPLICIT && !p->bottom_I) return ORC_EINVAL;
    if (p->top_kind == ORC_BC_EXPLICIT && !p->top_I) return ORC_EINVAL;
    for (int d = 0; d < p->ndir; ++d) {
        orc_dirgeom g;
        if (orc_direction_geometry(p, d, &g)) return ORC_EINVAL;
    }
    return ORC_OK;
}

/* Per-band intensities for a set of (band, direction) tasks, computed in
 * parallel chunks and accumulated in a fixed order afterwards, so that the
 * sums do not depend on the thread count. */
int orc_solve(const orc_problem *p, const double *chi, const double *S,
              double *I_top, double *J, double *F, double *Q,
              double *Jb, double *Fb, double *QJb, double *QFb,
              int *wrap_iters, int nthreads)
{
    int rc = validate(p);
    if (rc) return rc;
    const size_t plane = (size_t)p->nx * p->ny;
    const size_t N = plane * p->nz;
    const int B = p->nbands, D = p->ndir;
    const int nup = count_up(p);
    if (nthreads < 1) nthreads = 1;
    int chunk = nthreads;
    if (chunk > B * D) chunk = B * D;
    if (chunk > 256) chunk = 256;

    double *Iw = (double *)malloc((size_t)chunk * N * sizeof(double));
    double *jb = (double *)calloc(N, sizeof(double));
    double *fb = (double *)calloc(3 * N, sizeof(double));
    double *qf = (double *)malloc(N * sizeof(double));
    if (!Iw || !jb || !fb || !qf) {
        free(Iw); free(jb); free(fb); free(qf);
        return ORC_ENOMEM;
    }
    if (J) memset(J, 0, N * sizeof(double));
    if (F) memset(F, 0, 3 * N * sizeof(double));
    if (Q) memset(Q, 0, N * sizeof(double));

    int status = ORC_OK;
    for (int b = 0; b < B && status == ORC_OK; ++b) {
        const double *chi_b = chi + (size_t)b * N;
        const double *S_b = S + (size_t)b * N;
        memset(jb, 0, N * sizeof(double));
        memset(fb, 0, 3 * N * sizeof(double));
        for (int d0 = 0; d0 < D && status == ORC_OK; d0 += chunk) {
            int nd = D - d0 < chunk ? D - d0 : chunk;
            int rcs[512];
            int its[512];
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
            for (int t = 0; t < nd; ++t)
                rcs[t] = orc_sweep_direction(p, b, d0 + t, chi_b, S_b, Iw + (size_t)t * N, &its[t]);
            for (int t = 0; t < nd; ++t) {
                int d = d0 + t;
                if (rcs[t]) status = rcs[t];
                if (wrap_iters) wrap_iters[b * D + d] = its[t];
                const double *Id = Iw + (size_t)t * N;
                const double wd = p->w[d];
                const double *nd3 = p->n + 3 * d;
                /* mean intensity and flux: J = sum w I, F = 4 pi sum w n I */
                for (size_t q = 0; q < N; ++q) {
                    jb[q] += wd * Id[q];
                    fb[q] += FOUR_PI * wd * nd3[0] * Id[q];
                    fb[N + q] += FOUR_PI * wd * nd3[1] * Id[q];
                    fb[2 * N + q] += FOUR_PI * wd * nd3[2] * Id[q];
                }
                if (I_top && nd3[2] > 0) {
                    int u = updown_index(p, d);
                    double *dst = I_top + ((size_t)b * nup + u) * plane;
                    memcpy(dst, Id + (size_t)(p->nz - 1) * plane, plane * sizeof(double));
                }
            }
        }
        if (status) break;
        /* Q step: 4 pi chi (J - S) where thin, -div F where thick */
        orc_divergence(p->nx, p->ny, p->nz, p->dx, p->dy, p->dz, fb, qf);
        for (size_t q = 0; q < N; ++q) {
            double qj = FOUR_PI * chi_b[q] * (jb[q] - S_b[q]);
            double om = blend_omega(p, chi_b[q]);
            double qb = om * qj + (1.0 - om) * qf[q];
            if (J) J[q] += jb[q];
            if (F) {
                F[q] += fb[q];
                F[N + q] += fb[N + q];
                F[2 * N + q] += fb[2 * N + q];
            }
            if (Q) Q[q] += qb;
            if (QJb) QJb[(size_t)b * N + q] = qj;
            if (QFb) QFb[(size_t)b * N + q] = qf[q];
        }
        if (Jb) memcpy(Jb + (size_t)b * N, jb, N * sizeof(double));
        if (Fb) memcpy(Fb + (size_t)b * 3 * N, fb, 3 * N * sizeof(double));
    }
    free(Iw); free(jb); free(fb); free(qf);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Adjoint                                                                   */
/* ------------------------------------------------------------------------ */

/* Reverse sweep of one direction. lam enters holding the direct cotangent
 * lam0 of every point and leaves holding the total cotangent dL/dI. The
 * gradient contributions of this direction are added to gchi and gS. */
static int reverse_direction(const orc_problem *p, int d, const double *chi_b,
                             const double *S_b, const double *I, const double *lam0,
                             double *lam, double *gchi, double *gS)
{
    orc_dirgeom g;
    int rc = orc_direction_geometry(p, d, &g);
    if (rc) return rc;
    const size_t plane = (size_t)p->nx * p->ny;
    const size_t N = plane * p->nz;
    const int na = extent(p, g.axis);

    /* Adjoint recurrence: lam(u) = lam0(u) + sum over the points r that use
     * u as an upwind corner of beta * e_r * lam(r). Points are visited in the
     * reverse of the forward order, so lam(r) is complete when r scatters. */
    if (g.axis == 2) {
        memcpy(lam, lam0, N * sizeof(double));
        int kb = g.up ? 0 : p->nz - 1;
        for (int t = p->nz - 1; t >= 1; --t) {
            int k = kb + g.sa * t;
            PLANE_LOOP(p, &g, k, c)
                double dtau, e, wu, wp;
                size_t idx[4];
                solve_point(p, &g, c, chi_b, S_b, I, 0, 0, &dtau);
                orc_segment_weights(dtau, &e, &wu, &wp);
                upwind_corners(p, &g, c, idx);
                double lr = lam[lin(p, c)];
                for (int q = 0; q < 4; ++q) lam[idx[q]] += g.beta[q] * e * lr;
            PLANE_END
        }
    } else {
        const int start = g.sa > 0 ? 0 : na - 1;
        const int last = wrapi(start - g.sa, na);
        /* carry[q]: contributions that the first swept plane sends, through
         * the periodic wrap, into the last plane (a whole plane, boundary
         * level included). */
        const int n1 = extent(p, g.b1), n2 = extent(p, g.b2);
        size_t np = (size_t)n1 * n2;
        double *carry = (double *)calloc(np, sizeof(double));
        double *ncarry = (double *)calloc(np, sizeof(double));
        if (!carry || !ncarry) {
            free(carry); free(ncarry);
            return ORC_ENOMEM;
        }
        int it = 0;
        for (;;) {
            memcpy(lam, lam0, N * sizeof(double));
            for (int x = 0; x < n2; ++x)
                for (int y = 0; y < n1; ++y) {
                    int c[3];
                    c[g.axis] = last; c[g.b1] = y; c[g.b2] = x;
                    lam[lin(p, c)] += carry[(size_t)x * n1 + y];
                }
            memset(ncarry, 0, np * sizeof(double));
            for (int t = na - 1; t >= 0; --t) {
                int v = wrapi(start + g.sa * t, na);
                PLANE_LOOP(p, &g, v, c)
                    double dtau, e, wu, wp;
                    size_t idx[4];
                    solve_point(p, &g, c, chi_b, S_b, I, 0, 0, &dtau);
                    orc_segment_weights(dtau, &e, &wu, &wp);
                    upwind_corners(p, &g, c, idx);
                    double lr = lam[lin(p, c)];
                    for (int q = 0; q < 4; ++q) {
                        if (t == 0) {
                            /* corner lies in the last plane: goes to the carry */
                            int u[3] = {c[0], c[1], c[2]};
                            u[g.axis] = last;
                            if (q & 1) u[g.b1] -= g.s1;
                            if (q & 2) u[g.b2] -= g.s2;
                            int y = g.b1 == 2 ? u[2] : wrapi(u[g.b1], n1);
                            int x = g.b2 == 2 ? u[2] : wrapi(u[g.b2], n2);
                            ncarry[(size_t)x * n1 + y] += g.beta[q] * e * lr;
                        } else {
                            lam[idx[q]] += g.beta[q] * e * lr;
                        }
                    }
                PLANE_END
            }
            ++it;
            double res = 0.0, mx = 0.0;
            for (size_t q = 0; q < np; ++q) {
                double dv = fabs(ncarry[q] - carry[q]);
                if (dv > res) res = dv;
            }
            for (int x = 0; x < n2; ++x)
                for (int y = 0; y < n1; ++y) {
                    int c[3];
                    c[g.axis] = last; c[g.b1] = y; c[g.b2] = x;
                    double v = fabs(lam[lin(p, c)]);
                    if (v > mx) mx = v;
                }
            memcpy(carry, ncarry, np * sizeof(double));
            if (res <= p->wrap_tol * mx) break;
            if (it >= p->max_wrap_iters) {
                free(carry); free(ncarry);
                return ORC_ENOCONV;
            }
        }
        free(carry); free(ncarry);
    }

    /* Parameter gradients from the converged cotangents. */
    for (int v = 0; v < na; ++v) {
        PLANE_LOOP(p, &g, v, c)
            double Iup, Sup, dtau, e, wu, wp, dwu, dwp;
            size_t idx[4];
            size_t ip = lin(p, c);
            solve_point(p, &g, c, chi_b, S_b, I, &Iup, &Sup, &dtau);
            orc_segment_weights(dtau, &e, &wu, &wp);
            segment_weight_derivs(dtau, &dwu, &dwp);
            upwind_corners(p, &g, c, idx);
            double lr = lam[ip];
            /* dI_p/d(dtau) = -e I_up + w_up' S_up + w_p' S_p */
            double gdt = lr * (-e * Iup + dwu * Sup + dwp * S_b[ip]);
            double gc = gdt * 0.5 * g.ds; /* dtau = ds (chi_up + chi_p) / 2 */
            gchi[ip] += gc;
            gS[ip] += lr * wp;
            for (int q = 0; q < 4; ++q) {
                gchi[idx[q]] += g.beta[q] * gc;
                gS[idx[q]] += g.beta[q] * lr * wu;
            }
        PLANE_END
    }
    /* boundary layer with I = S passes its cotangent to S */
    int kind = g.up ? p->bottom_kind : p->top_kind;
    if (kind == ORC_BC_EQUAL_S) {
        int kb = g.up ? 0 : p->nz - 1;
        for (size_t q = 0; q < plane; ++q) gS[(size_t)kb * plane + q] += lam[(size_t)kb * plane + q];
    }
    return ORC_OK;
}

int orc_adjoint(const orc_problem *p, const double *chi, const double *S,
                const double *gI_top, const double *gJ, const double *gF, const double *gQ,
                double *g_logchi, double *g_S, int nthreads)
{
    int rc = validate(p);
    if (rc) return rc;
    const size_t plane = (size_t)p->nx * p->ny;
    const size_t N = plane * p->nz;
    const int B = p->nbands, D = p->ndir;
    const int nup = count_up(p);
    const double h[3] = {p->dx, p->dy, p->dz};
    if (nthreads < 1) nthreads = 1;
    int chunk = nthreads < D ? nthreads : D;
    if (chunk > 256) chunk = 256;

    double *Jb = (double *)malloc((size_t)B * N * sizeof(double));
    double *Fb = (double *)malloc((size_t)B * 3 * N * sizeof(double));
    double *QJb = (double *)malloc((size_t)B * N * sizeof(double));
    double *QFb = (double *)malloc((size_t)B * N * sizeof(double));
    double *gJb = (double *)malloc(N * sizeof(double));
    double *gFb = (double *)malloc(3 * N * sizeof(double));
    double *gchi = (double *)malloc(N * sizeof(double));
    double *gchid = (double *)malloc((size_t)chunk * N * sizeof(double));
    double *gSd = (double *)malloc((size_t)chunk * N * sizeof(double));
    double *Iw = (double *)malloc((size_t)chunk * N * sizeof(double));
    double *l0 = (double *)malloc((size_t)chunk * N * sizeof(double));
    double *lw = (double *)malloc((size_t)chunk * N * sizeof(double));
    if (!Jb || !Fb || !QJb || !QFb || !gJb || !gFb || !gchi || !gchid || !gSd || !Iw || !l0 || !lw) {
        free(Jb); free(Fb); free(QJb); free(QFb); free(gJb); free(gFb); free(gchi);
        free(gchid); free(gSd); free(Iw); free(l0); free(lw);
        return ORC_ENOMEM;
    }
    int status = orc_solve(p, chi, S, 0, 0, 0, 0, Jb, Fb, QJb, QFb, 0, nthreads);
    const double hm = hmin3(p);

    for (int b = 0; b < B && status == ORC_OK; ++b) {
        const double *chi_b = chi + (size_t)b * N;
        const double *S_b = S + (size_t)b * N;
        double *gS_b = g_S + (size_t)b * N;
        memset(gchi, 0, N * sizeof(double));
        memset(gS_b, 0, N * sizeof(double));
        /* Backward through the Q step and the band sums:
         * Q_b = om (4 pi chi (J_b - S)) + (1 - om) (-div F_b), om = om(chi). */
        for (size_t q = 0; q < N; ++q) {
            gJb[q] = gJ ? gJ[q] : 0.0;
            gFb[q] = gF ? gF[q] : 0.0;
            gFb[N + q] = gF ? gF[N + q] : 0.0;
            gFb[2 * N + q] = gF ? gF[2 * N + q] : 0.0;
        }
        if (gQ) {
            for (size_t q = 0; q < N; ++q) {
                double om = blend_omega(p, chi_b[q]);
                double dom = -hm / p->tau_switch * om;
                double qj = QJb[(size_t)b * N + q], qf = QFb[(size_t)b * N + q];
                gJb[q] += gQ[q] * om * FOUR_PI * chi_b[q];
                gS_b[q] += -gQ[q] * om * FOUR_PI * chi_b[q];
                gchi[q] += gQ[q] * (om * FOUR_PI * (Jb[(size_t)b * N + q] - S_b[q]) + dom * (qj - qf));
            }
            /* -div is linear in F: scatter the transpose of its stencil */
            for (int k = 0; k < p->nz; ++k)
                for (int j = 0; j < p->ny; ++j)
                    for (int i = 0; i < p->nx; ++i) {
                        size_t q = ((size_t)k * p->ny + j) * p->nx + i;
                        double u = gQ[q] * (1.0 - blend_omega(p, chi_b[q]));
                        for (int a = 0; a < 3; ++a) {
                            size_t idx[2];
                            double cf[2];
                            int nt = div_terms(p->nx, p->ny, p->nz, h[a], a, i, j, k, idx, cf);
                            for (int t = 0; t < nt; ++t) gFb[(size_t)a * N + idx[t]] += -u * cf[t];
                        }
                    }
        }
        /* per direction: seed cotangent, reverse sweep, gradient pieces */
        for (int d0 = 0; d0 < D && status == ORC_OK; d0 += chunk) {
            int nd = D - d0 < chunk ? D - d0 : chunk;
            int rcs[512];
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
            for (int t = 0; t < nd; ++t) {
                int d = d0 + t;
                double *Id = Iw + (size_t)t * N, *lam0 = l0 + (size_t)t * N, *lam = lw + (size_t)t * N;
                double *gc = gchid + (size_t)t * N, *gs = gSd + (size_t)t * N;
                int its;
                rcs[t] = orc_sweep_direction(p, b, d, chi_b, S_b, Id, &its);
                if (rcs[t]) continue;
                const double *nd3 = p->n + 3 * d;
                const double wd = p->w[d];
                for (size_t q = 0; q < N; ++q)
                    lam0[q] = wd * gJb[q] + FOUR_PI * wd *
                              (nd3[0] * gFb[q] + nd3[1] * gFb[N + q] + nd3[2] * gFb[2 * N + q]);
                if (gI_top && nd3[2] > 0) {
                    int u = updown_index(p, d);
                    const double *src = gI_top + ((size_t)b * nup + u) * plane;
                    for (size_t q = 0; q < plane; ++q) lam0[(size_t)(p->nz - 1) * plane + q] += src[q];
                }
                memset(gc, 0, N * sizeof(double));
                memset(gs, 0, N * sizeof(double));
                rcs[t] = reverse_direction(p, d, chi_b, S_b, Id, lam0, lam, gc, gs);
            }
            for (int t = 0; t < nd; ++t) {
                if (rcs[t]) { status = rcs[t]; break; }
                const double *gc = gchid + (size_t)t * N, *gs = gSd + (size_t)t * N;
                for (size_t q = 0; q < N; ++q) {
                    gchi[q] += gc[q];
                    gS_b[q] += gs[q];
                }
            }
        }
        /* d/d log chi = chi d/d chi */
        for (size_t q = 0; q < N; ++q) g_logchi[(size_t)b * N + q] = chi_b[q] * gchi[q];
    }
    free(Jb); free(Fb); free(QJb); free(QFb); free(gJb); free(gFb); free(gchi);
    free(gchid); free(gSd); free(Iw); free(l0); free(lw);
    return status;
}

/*
 * rts_oracle.h -- plain, slow, FP64 CPU oracle of the short-characteristics
 * radiation transport solve (test infrastructure only).
 *
 * This is the reference the CUDA library is checked against. It shares no
 * code, header, table or helper with the CUDA path. Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Method (paper Sect. 5.1, "Summary of the Radiation Transport Solver"):
 * short characteristics (Kunasz & Auer) on a 3-D Cartesian grid, 3 rays per
 * octant (24 directions, Carlson quadrature), one solve per opacity band,
 * boundary intensities iterated to a tolerance, then mean intensity J, flux F
 * and radiative heating Q_rad. The paper gives no formulas: the formal
 * solution, the interpolation, the boundary handling and the Q_rad blend
 * below are readings of it, each stated where it is used.
 *
 * Layouts (C order, x fastest): grid arrays [B][Nz][Ny][Nx]; F [3][Nz][Ny][Nx];
 * I_top [B][n_up][Ny][Nx] (up directions in direction-table order);
 * bottom_I [B][n_up][Ny][Nx]; top_I [B][n_down][Ny][Nx].
 */
#ifndef RTS_ORACLE_H
#define RTS_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENOCONV = 5 };
enum { ORC_BC_ZERO = 0, ORC_BC_EQUAL_S = 1, ORC_BC_EXPLICIT = 2 };

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    int nbands;
    int ndir;
    const double *n;      /* [ndir][3] unit vectors */
    const double *w;      /* [ndir] weights (sum 1) */
    double tau_switch;    /* thin/thick blend constant */
    double wrap_tol;      /* relative tolerance of the periodic-wrap iteration */
    int max_wrap_iters;   /* cap on wrap iterations (ORC_ENOCONV beyond) */
    int bottom_kind;      /* boundary for up rays at k = 0 */
    int top_kind;         /* boundary for down rays at k = Nz-1 */
    const double *bottom_I;
    const double *top_I;
} orc_problem;

/* The default angular set: level-symmetric 4th-order (3 directions per
 * octant), ordered as 6 sweep groups of 4. Writes n[72], w[24]. */
void orc_a4_quadrature(double *n, double *w);

/* Geometry of one direction (exposed for tests). */
typedef struct {
    int axis, sa;         /* dominant axis (0 x, 1 y, 2 z) and sign of n along it */
    int b1, b2;           /* minor axes, b1 < b2 */
    int s1, s2;           /* signs of n along b1, b2 (+1 when the component is 0) */
    double ds;            /* path length to the upwind plane */
    double d1, d2;        /* fractional offsets along b1, b2, in [0,1] */
    double beta[4];       /* bilinear weights of corners (0,0),(1,0),(0,1),(1,1) */
    int up;               /* n_z > 0 */
} orc_dirgeom;
int orc_direction_geometry(const orc_problem *p, int d, orc_dirgeom *g);

/* Linear-in-tau formal-solution weights of one segment of optical depth x. */
void orc_segment_weights(double x, double *e, double *w_up, double *w_p);

/* Intensity of one direction of one band on the whole grid (I[N]).
 * iters receives the number of periodic-wrap sweeps (1 for z-dominant). */
int orc_sweep_direction(const orc_problem *p, int band, int d,
                        const double *chi_b, const double *S_b, double *I, int *iters);

/* -(dFx/dx + dFy/dy + dFz/dz), central differences, periodic in x and y,
 * one-sided first order at k = 0 and k = Nz-1. F [3][N], out [N]. */
void orc_divergence(int nx, int ny, int nz, double dx, double dy, double dz,
                    const double *F, double *neg_div);

/* Full forward solve. Any output pointer may be NULL. Jb/Fb/QJb/QFb are the
 * per-band debug outputs [B][N], [B][3][N], [B][N], [B][N]. wrap_iters is
 * [B][ndir]. nthreads <= 1 runs single-threaded; the result does not depend
 * on nthreads. */
int orc_solve(const orc_problem *p, const double *chi, const double *S,
              double *I_top, double *J, double *F, double *Q,
              double *Jb, double *Fb, double *QJb, double *QFb,
              int *wrap_iters, int nthreads);

/* Gradient of L = <gI_top,I_top> + <gJ,J> + <gF,F> + <gQ,Q> with respect to
 * log chi and S ([B][N] each). NULL cotangents count as zero. */
int orc_adjoint(const orc_problem *p, const double *chi, const double *S,
                const double *gI_top, const double *gJ, const double *gF, const double *gQ,
                double *g_logchi, double *g_S, int nthreads);

#ifdef __cplusplus
}
#endif
#endif

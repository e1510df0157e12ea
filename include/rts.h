/*
 * rts.h -- C ABI of the B300-native short-characteristics radiation transport
 * solver (RTS).
 *
 * The operation (paper Sect. 2 "MURaM Routines" and Sect. 5.1 "Summary of the
 * Radiation Transport Solver"): for every opacity band and every ray of a
 * 3-rays-per-octant (24-ray) Carlson quadrature, integrate the transfer
 * equation along short characteristics on a 3-D Cartesian grid that is
 * periodic in x and y, iterating the periodic boundary intensities to a
 * tolerance; then form the mean intensity J, the radiative flux F and the
 * radiative heating/cooling Q_rad that is fed back to the MHD solver. The
 * multi-band scheme (Sect. 1, Nordlund's opacity binning) runs the transfer
 * once per band and sums over bands.
 *
 * Per point p, direction d and band b (one short characteristic):
 *   I_up, chi_up, S_up = bilinear interpolation on the face the ray crosses
 *   dtau = ds_d (chi_up + chi_p) / 2,  e = exp(-dtau)
 *   I_p  = e I_up + w_up S_up + w_p S_p,
 *   w_up = (1-e)/dtau - e,  w_p = 1 - (1-e)/dtau   (S linear in tau)
 * Accumulation: J = sum_b sum_d w_d I,  F = 4 pi sum_b sum_d w_d n_d I,
 * Q_rad = sum_b [om_b 4 pi chi_b (J_b - S_b) + (1 - om_b)(-div F_b)],
 * om_b = exp(-chi_b min(dx,dy,dz) / tau_switch) (thin/thick blend).
 * I_top[b][u] is the intensity of the u-th upward direction at k = Nz-1.
 *
 * Conventions
 *  - Grid arrays are C-contiguous [B][Nz][Ny][Nx] (x fastest, k = 0 bottom);
 *    F is [3][Nz][Ny][Nx]; J and Q_rad are [Nz][Ny][Nx].
 *  - I_top and explicit bottom intensities are [B][n_up][Ny][Nx]; explicit
 *    top intensities are [B][n_down][Ny][Nx]; up/down directions are counted
 *    in quadrature-table order.
 *  - Precision: chi, S, I_top and explicit boundary arrays are float64 for
 *    RTS_FP64 and float32 for the FP32 modes. J, F and Q_rad are float64.
 *  - Ownership: every array argument is a caller-owned DEVICE pointer
 *    (unless stated otherwise), valid on the handle's stream. Inputs are
 *    read-only. The handle owns all scratch, allocated in rts_create;
 *    rts_solve and rts_adjoint allocate nothing and do not synchronise.
 *  - Errors: every call returns an rts_status. Argument errors are returned
 *    at once. Errors found on the device (a wait that timed out, a periodic
 *    wrap that did not converge) are recorded in a device status word and
 *    returned by the next rts_check or rts_get_stats. rts_last_error gives a
 *    text. No C++ exception crosses the ABI.
 */
#ifndef RTS_H
#define RTS_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RTS_OK = 0,
    RTS_EINVAL = 1,      /* bad argument (NULL, size, band count, spacing) */
    RTS_ENOMEM = 2,      /* device allocation failed in rts_create */
    RTS_ECUDA = 3,       /* a CUDA runtime call failed */
    RTS_ETIMEOUT = 4,    /* a device-side wait gave up (no hang) */
    RTS_ENOCONV = 5,     /* the periodic wrap did not converge within the cap */
    RTS_ENONFINITE = 6   /* a NaN or an infinity in chi or S (found on the device
                            while the solve runs; reported by rts_check) */
} rts_status;

typedef enum {
    RTS_FP64 = 0,             /* FP64 sweep, FP64 accumulation and Q step */
    RTS_FP32_MIXED = 1,       /* FP32 sweep; band/group accumulation and Q step in FP64 */
    RTS_FP32_COMPENSATED = 2  /* FP32 sweep; accumulation and Q step in compensated
                                 (double-float, two-FP32) arithmetic */
} rts_precision;

typedef enum { RTS_BC_ZERO = 0, RTS_BC_EQUAL_S = 1, RTS_BC_EXPLICIT = 2 } rts_bc_kind;

typedef struct {
    int nx, ny, nz;       /* nx, ny >= 1 (periodic), nz >= 2 */
    double dx, dy, dz;    /* > 0 */
} rts_grid;

/* Angular quadrature (host pointers, copied in rts_create). NULL selects the
 * default 24-direction level-symmetric S4 (Carlson) set. Every direction must
 * have n_z != 0. */
typedef struct {
    int ndir;
    const double *n;      /* [ndir][3] unit vectors */
    const double *w;      /* [ndir] weights, sum 1 */
} rts_quadrature;

enum {
    RTS_FLAG_HOST_IO = 1, /* allocate staging buffers for rts_solve_host */
    RTS_FLAG_TIMING = 2,  /* record CUDA events around each phase of every
                             solve (on the handle's stream); rts_get_stats
                             reports their mean over the solves since the
                             previous rts_get_stats call */
    RTS_FLAG_ADJOINT = 4, /* allocate the scratch of rts_adjoint */
    RTS_FLAG_HOST_IO_ASYNC = 8, /* two staging sets and two copy streams for
                             rts_solve_host_async */
    RTS_FLAG_SCATTER = 32, /* the scratch of rts_scatter_solve */
    RTS_FLAG_LOG_CHI = 16 /* the chi argument of rts_solve, rts_adjoint and
                             rts_graph_create is log chi: the library forms
                             chi = exp(log chi) in a scratch array of B x N
                             elements first (one more kernel); the gradient
                             rts_adjoint returns is the one w.r.t. log chi as
                             always. Not accepted by batched handles. */
};

typedef struct {
    rts_precision prec;
    double tau_switch;    /* thin/thick blend constant (default 0.1) */
    double wrap_tol;      /* bound on the remaining seed error of the periodic
                             wrap, relative to the seed error (default 1e-15
                             for FP64, 2^-24 for FP32) */
    int max_wrap_iters;   /* cap on the wrap warm-up, in periods (default 64) */
    int tile_rows;        /* rows of a sweep tile (0 = automatic) */
    int threads;          /* threads per CTA of the sweep (0 = automatic) */
    int flags;            /* RTS_FLAG_* */
    double timeout_s;     /* device-side wait limit in seconds (default 2) */
    void *stream;         /* cudaStream_t to run on (NULL = legacy default stream) */
    int adjoint_chunk_bands; /* bands whose intensities rts_adjoint recomputes
                             and keeps at a time (the checkpoint unit);
                             larger chunks run more sweep units at once and
                             need proportionally more scratch. 0 = automatic:
                             equal chunks, as large as fit in 85 % of the
                             device memory free at rts_create next to the
                             handle's other arrays (at least 1 band) */
    int sweep_kernel;     /* forward sweep of the FP32 modes: RTS_SWEEP_AUTO (0),
                             RTS_SWEEP_SHARED (1) or RTS_SWEEP_REGISTER (2) */
} rts_options;

enum {
    RTS_SWEEP_AUTO = 0,     /* the register-resident sweep where it applies, else the shared one */
    RTS_SWEEP_SHARED = 1,   /* tile rows and chi/S in shared memory, any grid and quadrature */
    RTS_SWEEP_REGISTER = 2  /* two columns per thread in registers, packed FP32 arithmetic;
                               needs FP32, even nx and ny, and one bilinear stencil
                               per direction group (any 3-rays-per-octant set);
                               rts_create fails with RTS_EINVAL otherwise */
};

typedef struct {
    int n_units;          /* sweep units of the last solve (band x direction group) */
    int n_tiles;          /* tiles of the last solve */
    int max_warmup_steps; /* longest periodic-wrap warm-up of the last solve (planes) */
    double mean_warmup_steps;
    int device_status;    /* rts_status recorded on the device */
    int grid;             /* CTAs of the persistent sweep launch */
    int tile_rows;        /* rows per sweep tile */
    int kernels_per_solve;/* kernels one rts_solve launches */
    /* with RTS_FLAG_TIMING: mean milliseconds per solve of each phase over the
     * timed_solves solves since the previous call (else 0) */
    int timed_solves;
    float ms_transpose, ms_sweep, ms_reduce, ms_qstep;
    /* with RTS_FLAG_TIMING: mean milliseconds per rts_adjoint call of its
     * phases since the previous call: [0] transposes and Q-step adjoints,
     * [1] forward re-sweeps (checkpoints) and their band reductions,
     * [2] reverse sweeps, [3] gradient passes and reduction; over
     * timed_adjoints calls */
    int timed_adjoints;
    float ms_adjoint[4];
    int sweep_kernel;     /* forward sweep rts_solve runs: RTS_SWEEP_SHARED or RTS_SWEEP_REGISTER */
    int adjoint_chunk_bands; /* bands per checkpoint of rts_adjoint (0 without RTS_FLAG_ADJOINT) */
} rts_stats;

/* Boundary conditions of a solve, and the optional warm start of the
 * horizontally periodic wrap (paper Sect. 2: the solver starts from the
 * intensities of a previous time step or iteration and iterates the boundary
 * intensities until they converge).
 * wrap_seed (device, float, rts_wrap_seed_elems(h) elements; FP32 register
 * sweep only, else RTS_EINVAL): for every x- and y-dominant direction group
 * the intensities of its wrap plane (the plane upwind of the first swept
 * one, [Nq][Np][4 sign slots] per group). Written with the converged values
 * by every solve that is given it. With seed_in != 0 it is also read as the
 * starting values: the sweep accumulates from the first period, carrying in
 * that period the seed-error bound from 1 on the wrap plane. With r_p the
 * wrap plane's change over period p (relative to its largest intensity,
 * per tile) and gam the bound after one period (its contraction of a wrap
 * error), the seed error is at most r_0 / (1 - gam): the solve stops when
 * one whole period of planes is shown to carry at most seed_tol (default
 * 1e-6) relative error -- planes of the first period once their bound times
 * r_0 / (1 - gam) is below it, later planes once r_p / (1 - gam) is (the
 * paper's test on boundary intensities, made rigorous by gam; with gam >= 1
 * the plain test r_p <= seed_tol). Without seed_in the wrap converges from
 * I = S with the seed-error bound alone. */
typedef struct {
    rts_bc_kind bottom, top;
    const void *bottom_I;  /* [B][n_up][Ny][Nx] when bottom == RTS_BC_EXPLICIT */
    const void *top_I;     /* [B][n_down][Ny][Nx] when top == RTS_BC_EXPLICIT */
    void *wrap_seed;       /* optional warm start, in/out (see above); NULL = none */
    int seed_in;           /* read wrap_seed as the starting values */
    double seed_tol;       /* relative error that ends a warm-started wrap (0 = 1e-6) */
} rts_boundary;


typedef struct rts_handle rts_handle;

/* Default options: RTS_FP64, tau_switch 0.1, automatic tiling, 2 s timeout. */
void rts_default_options(rts_options *opt);

/* Create a solver for one grid and band count (the paper's RTS setup,
 * Sect. 5.1: the grid, its spacing, the band count of the multi-band scheme
 * and the 24-ray quadrature of Sect. 2; q may be NULL for that set, or give
 * 1..24 directions with n_z != 0 and weights). Plans the direction groups and
 * tiles, allocates all device scratch (nothing is allocated by solves) and
 * owns it until rts_destroy. opt may be NULL (defaults). On failure *h may
 * still be set (read rts_last_error, then rts_destroy). Errors: RTS_EINVAL
 * (grid, band count, quadrature or options out of range; nz * nbands >
 * 65535), RTS_ENOMEM, RTS_ECUDA. */
rts_status rts_create(rts_handle **h, const rts_grid *g, int nbands,
                      const rts_quadrature *q, const rts_options *opt);

/* Forward solve (paper Sect. 5.1: integrate over all rays and bands, then
 * flux). chi, S: [B][Nz][Ny][Nx]; bc may be NULL (bottom I = S, top I = 0).
 * Any output may be NULL. Enqueued on the handle's stream; no sync. */
rts_status rts_solve(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc,
                     void *I_top, double *J, double *F, double *Q_rad);

/* Same as rts_solve with HOST pointers: copies the inputs to the device,
 * solves, copies the outputs back and synchronises the stream. Needs
 * RTS_FLAG_HOST_IO at create time; explicit boundary arrays are not
 * accepted here (bc kinds ZERO / EQUAL_S only). */
rts_status rts_solve_host(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc,
                          void *I_top, double *J, double *F, double *Q_rad);

/* Pipelined form of rts_solve_host for a stream of solves: enqueues the
 * copy of the inputs (a copy stream), the solve (the handle's stream) and the
 * copy of the outputs back (a second copy stream) and returns at once.
 * Consecutive calls alternate between two device staging sets, so the input
 * copy of one call, the solve of the previous one and the output copy of the
 * one before run at the same time (both copy engines and the SMs). Host
 * buffers should be pinned (page-locked) for the copies to overlap; inputs
 * must stay unchanged and outputs unread until rts_host_wait returns (or
 * two later calls have been made and waited for). Needs
 * RTS_FLAG_HOST_IO_ASYNC; bc kinds ZERO / EQUAL_S only. */
rts_status rts_solve_host_async(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc,
                                void *I_top, double *J, double *F, double *Q_rad);

/* Scattering solve (paper Sect. 5.3.2: in strongly scattering media the
 * source function depends on the intensity, S_b = (1 - eps_b) J_b + eps_b B_b,
 * J_b the band's mean intensity): iterates
 *   S <- S + [(1 - eps) J[S] + eps B - S] / [1 - (1 - eps) L*]
 * until the largest relative change of S over all bands and points is
 * <= tol, each iteration a forward solve of all bands with the current S
 * (sweep and band reduction; J[S] is the formal solution) followed by the
 * update. L* is a local approximation of the operator's diagonal,
 * sum_d w_d (1 - (1 - e^-x_d)/x_d) with x_d = ds_d chi / 2 at the point (a
 * lower bound of each segment's optical depth, so L* stays below the true
 * diagonal and the iteration stable): it only preconditions the iteration
 * (an accelerated Lambda iteration); the converged S solves the equation
 * above. The paper's alternative, a Gauss-Seidel update along each ray, does
 * not fit the direction-group sweep (the x/y groups advance their rays
 * plane by plane across the horizontal), so every point is updated at once.
 * In the FP32 modes L* and the update are taken in float, the residual
 * (1 - eps) J + eps B - S in double.
 * Arguments: chi, B_src (the thermal source) and eps (photon destruction
 * probability, 0 < eps <= 1) are [B][Nz][Ny][Nx] device arrays of the sweep
 * precision; S (same layout) is the initial guess on entry and the converged
 * source function on return (bottom boundary kind EQUAL_S uses it). After
 * convergence a last solve with that S writes I_top, J, F, Q_rad (any may be
 * NULL). *iters (may be NULL) receives the number of iterations. Returns
 * RTS_ENOCONV after max_iter iterations without convergence. Needs
 * RTS_FLAG_SCATTER at create time. Synchronises once per iteration (it reads
 * the change back), so not for stream capture. The problem's conditioning
 * grows like 1/eps: in the FP32 modes the attainable tol and accuracy are
 * about 3e-7 / min(eps); use RTS_FP64 for small eps. */
rts_status rts_scatter_solve(rts_handle *h, const void *chi, const void *B_src, const void *eps, void *S,
                             const rts_boundary *bc, int max_iter, double tol, int *iters,
                             void *I_top, double *J, double *F, double *Q_rad);

/* Wait for every rts_solve_host_async call of the handle and return the
 * device status (as rts_check). */
rts_status rts_host_wait(rts_handle *h);

/* Wait for the handle's stream and return the device status of the last
 * solve (RTS_OK, RTS_ETIMEOUT, RTS_ENOCONV, RTS_ENONFINITE). */
rts_status rts_check(rts_handle *h);

/* The compute capability the library's device code was built for, as
 * major * 10 + minor (103 for sm_103a), read from the loaded kernel image on
 * the current device; -1 if it cannot be read (no device). */
int rts_device_code_version(void);

/* Statistics of the last solve and, with RTS_FLAG_TIMING, mean phase times
 * of the solves since the previous call (synchronises the stream): the
 * tiling, the kernels per solve, the periodic wrap's warm-up planes (the
 * paper's iterations of boundary intensities, Sect. 5.1) and the transpose /
 * sweep / reduction / Q-step times (the phases of Sect. 5.3). */
rts_status rts_get_stats(rts_handle *h, rts_stats *out);

/* Text of the last error on this handle (never NULL). */
const char *rts_last_error(rts_handle *h);

/* Number of upward directions of the handle's quadrature. */
int rts_num_up(rts_handle *h);

/* Elements (floats) of the warm-start buffer of rts_boundary.wrap_seed for
 * this handle (0 when the handle has no register sweep). */
long long rts_wrap_seed_elems(rts_handle *h);

/* Release a handle of rts_create or rts_create_batched: its device scratch
 * (cudaFree, which waits for the device's outstanding work), its events and
 * copy streams (graphs of rts_graph_create are released by
 * rts_graph_destroy). NULL is ignored. */
void rts_destroy(rts_handle *h);

/* Gradient of the scalar
 *   L = <gI_top, I_top> + <gJ, J> + <gF, F> + <gQ, Q_rad>
 * (the outputs of rts_solve on the same chi, S, bc) with respect to log chi
 * and S of every band: reverse-mode differentiation of the discrete solve.
 * The paper has no adjoint; this is the transpose of its forward operator.
 * Per chunk of adjoint_chunk_bands bands (the checkpoint):
 *   1. the forward sweep of the chunk, keeping the derivative dI/d(dtau) of
 *      every ray's converged segment (4 values per point and sweep unit);
 *      the intensities it produces give the chunk's J_b, F_b (on FP32
 *      handles that run the register sweep, the register sweep's own
 *      checkpoint form with the double-float reduction and a double-float
 *      Q-step transpose, in both FP32 modes);
 *   2. the Q step transposed for those bands (cotangents of J_b and F_b, and
 *      the direct chi and S terms of Q_rad), then the reverse sweep: the
 *      cotangent of I along each ray, lam_p = lam0_p + sum over the downwind
 *      points r that interpolate from p of beta e_r lam_r, swept in the
 *      reverse plane order with tiles, ready flags and a periodic-wrap
 *      bound like the forward sweep; then the derivative of each segment's
 *      formal solution with respect to the opacity and source it used,
 *      gathered onto the grid points it was interpolated from;
 *   3. g_logchi = chi * dL/dchi.
 * Boundary layers with I = S pass their cotangent to g_S; explicit boundary
 * intensities are treated as constants.
 * Arguments: chi, S, bc as for rts_solve. gI_top is [B][n_up][Ny][Nx] in the
 * sweep precision; gJ [Nz][Ny][Nx], gF [3][Nz][Ny][Nx] and gQ [Nz][Ny][Nx]
 * are float64; any cotangent may be NULL (zero). g_logchi and g_S are
 * [B][Nz][Ny][Nx] in the sweep precision (written, not accumulated). All
 * device pointers; outputs must not alias inputs. When gQ is NULL the band
 * reductions are skipped (J, F enter L linearly). Needs RTS_FLAG_ADJOINT
 * at create time; allocates nothing and does not synchronise. Device errors
 * as for rts_solve (rts_check). */
rts_status rts_adjoint(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc,
                       const void *gI_top, const double *gJ, const double *gF, const double *gQ,
                       void *g_logchi, void *g_S);

/* ---------------------------------------------------------------------------
 * Batched solves: many independent grids ("subdomains") of uneven size, each
 * with the same band count, solved in ONE persistent sweep launch (the paper
 * pays one kernel launch per plane and direction per grid, Sect. 5.2; here
 * all grids, bands and direction groups share one work list of tiles, longest
 * units first), plus one launch each of the transpose, the unit reduction and
 * the Q step over all grids. Results are identical to rts_solve on each grid.
 *
 * Packed layout: the arrays of subdomain s follow those of s-1 in one buffer:
 *   chi, S:  [B][Nz_s][Ny_s][Nx_s] at element grid_offset(s)
 *   I_top:   [B][n_up][Ny_s][Nx_s] at element top_offset(s)
 *   J, Q:    [Nz_s][Ny_s][Nx_s] at element point_offset(s); F: [3][...] at 3 * point_offset(s)
 * rts_batched_layout returns these offsets and the totals
 * (totals[0] = chi elements, totals[1] = I_top elements, totals[2] = points).
 * Boundary kinds ZERO and EQUAL_S only. RTS_FLAG_ADJOINT and RTS_FLAG_HOST_IO
 * are not accepted. Errors as for rts_solve. */
rts_status rts_create_batched(rts_handle **h, int nsub, const rts_grid *grids, int nbands,
                              const rts_quadrature *q, const rts_options *opt);
rts_status rts_solve_batched(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc,
                             void *I_top, double *J, double *F, double *Q_rad);
rts_status rts_batched_layout(rts_handle *h, int sub, long long *grid_offset, long long *top_offset,
                              long long *point_offset, long long totals[3]);

/* CUDA graph of one solve (rts_solve or rts_solve_batched, by handle kind)
 * with fixed arguments, captured on the handle's stream, which must not be
 * the legacy default stream. rts_graph_launch replays it on that stream (the
 * pointers captured must stay valid); device errors are read with rts_check
 * on the handle. */
typedef struct rts_graph rts_graph;
rts_status rts_graph_create(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc,
                            void *I_top, double *J, double *F, double *Q_rad, rts_graph **g);
rts_status rts_graph_launch(rts_graph *g);
void rts_graph_destroy(rts_graph *g);

/* Tile-size autotuner: for every tile height the library instantiates for
 * these plane extents (1, 2, 4, 6, 7, 8, 12, 16 rows, where the tile fits) builds a
 * batched handle for the given grids (nsub = 1 for a single grid; packed chi,
 * S as above, device pointers), times `repeats` solves with CUDA events on
 * opt->stream after one warm-up, and returns the fastest in *best_tile_rows;
 * the *ncand candidates timed and their mean milliseconds go to rows[] and
 * ms[] (up to 8). Allocates and frees device memory and synchronises: a
 * set-up step, not for the hot path. */
rts_status rts_autotune(int nsub, const rts_grid *grids, int nbands, const rts_quadrature *q,
                        const rts_options *opt, const void *chi, const void *S, int repeats,
                        int *best_tile_rows, int *ncand, int rows[8], float ms[8]);

/* ---------------------------------------------------------------------------
 * Forward solve without any memory allocation. The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory --
 * an embedding code (for example an MHD code that owns the GPU's memory and
 * hands the solver a fixed budget) that does not allow cudaMalloc outside its
 * own pool, or a process whose allocator is already at its limit. It runs
 * the same kernels as rts_solve on the same inputs and outputs (caller-owned
 * device pointers, layouts as above), with the default quadrature, bottom
 * I = S, top I = 0 and default options, and takes all its scratch from one
 * static device array of RTS_NOALLOC_SCRATCH_BYTES that the CUDA runtime sets
 * up when the library is loaded on a GPU (every GPU that loads the library
 * keeps it until exit).
 *  - It calls no cudaMalloc/cudaFree and allocates no host memory.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and keeps it for the
 *    process. After a cudaDeviceReset that address is stale: do not call this
 *    function again in a process that reset its device.
 *  - The call waits for its stream (it reads back the device status), so it
 *    cannot run inside a stream capture: on a capturing stream it returns
 *    RTS_EINVAL without touching the capture.
 *  - Problems whose scratch would not fit are rejected with RTS_EINVAL and a
 *    message in err. The scratch of one FP32 band is about 36 bytes per
 *    grid point (its 6 sweep units' partial sums, the band's J and F and the
 *    transposed copies), so 64^3 x 1 band fits and 64^3 x 2 bands do not.
 *  - All calls share the one array and it keeps the previous call's contents;
 *    the control words are cleared on every call. Calls that overlap on the
 *    GPU (other streams, other host threads) race: serialise them.
 *  - Returns the device status (RTS_OK, RTS_ETIMEOUT, RTS_ENOCONV,
 *    RTS_ENONFINITE). err (may be NULL) receives a text.
 *  - nbands <= 16; nx, ny <= 1024. */
#define RTS_NOALLOC_SCRATCH_BYTES (64u << 20)
rts_status rts_solve_noalloc(const rts_grid *g, int nbands, rts_precision prec,
                             const void *chi, const void *S,
                             void *I_top, double *J, double *F, double *Q_rad,
                             void *stream, char *err, size_t errlen);

/* ---------------------------------------------------------------------------
 * The solver's input step (paper Sect. 2, RTS "Interpolate": trilinear
 * interpolation of the MHD variables from the MHD grid to the staggered RTS
 * grid, then the source function and the opacities used by the integration).
 * The MHD fields T and rho are given at the MHD cell centres of a grid of
 * the same extents as the RTS grid; RTS point (i, j, k) lies at MHD cell
 * coordinates (i, j, k) + shift (shift = -0.5 each: the RTS points on the
 * cell corners). Per point: ln T and ln rho interpolated trilinearly from the
 * 8 surrounding cells (periodic in x and y, clamped to the first and last
 * layer in z); then for every band b
 *   ln kappa_b = bilinear in the table ln_kappa[b][ir][it] at
 *                (ln T - lnT0)/dlnT, (ln rho - lnR0)/dlnR (clamped to the table),
 *   chi_b      = exp(ln kappa_b) rho,
 *   S_b        = exp(ln B_b), ln B_b linear in ln_B[b][it] along ln T.
 * The table is a band-integrated opacity (opacity binning, paper Sect. 1)
 * and a band source function; the paper's tables are not available, so the
 * library only defines the lookup. Arrays are device pointers: T_mhd, rho_mhd
 * [Nz][Ny][Nx] and the tables in the precision's type (FP64 for RTS_FP64,
 * FP32 otherwise), chi and S out, [B][Nz][Ny][Nx], the layout rts_solve
 * reads. Enqueued on `stream`; no synchronisation, no allocation. err (may
 * be NULL) receives a text. */
typedef struct {
    int nbands, nT, nR;
    double lnT0, dlnT;     /* ln T of table column 0, step (> 0) */
    double lnR0, dlnR;     /* ln rho of table row 0, step (> 0) */
    const void *ln_kappa;  /* [nbands][nR][nT] ln of the opacity per unit density */
    const void *ln_B;      /* [nbands][nT] ln of the band source function */
    double shift[3];       /* RTS point (0,0,0) on the MHD grid, in cells;
                              finite, |shift| <= 2^20, else RTS_EINVAL */
} rts_front_table;
rts_status rts_front_end(const rts_grid *g, const rts_front_table *tab, rts_precision prec,
                         const void *T_mhd, const void *rho_mhd, void *chi, void *S, void *stream,
                         char *err, size_t errlen);

/* ---------------------------------------------------------------------------
 * Spatial decomposition (paper Sect. 2 and 5.1: the domain is split into
 * sub-domains; each integrates its rays from the boundary intensities of the
 * previous iteration, and the boundary intensities are iterated until a
 * global error is below a tolerance -- 3 to 4 iterations in the paper). A
 * one-GPU form of that scheme: the grid is cut into nblocks slabs of levels
 * (the periodic x, y wrap stays inside every slab's solve). Slab k owns
 * levels [a_k, b_k) (a_k = k nz / nblocks) and is solved on [a_k - 1, b_k + 1)
 * (a ghost level towards each neighbour) with explicit boundary intensities:
 * its bottom layer takes the upward intensities slab k-1 computed at level
 * a_k - 1 in the previous iteration, its top layer the downward intensities
 * slab k+1 computed at level b_k (the first iteration starts from I = S).
 * Iterations end when the largest change of J over the grid is <= tol times
 * max J (the global J criterion). The slabs then hold the undecomposed
 * solution: J, F and Q_rad of every owned level are those of rts_solve, and
 * I_top is the top slab's. FP32 modes only (the interface intensities are
 * read from the register sweep's slot partials); options as rts_create
 * (only RTS_FLAG_TIMING among the flags). rts_solve_decomposed synchronises
 * once per iteration (the convergence test); J must be given. */
typedef struct rts_decomp rts_decomp;
rts_status rts_create_decomposed(rts_decomp **d, const rts_grid *g, int nbands, int nblocks,
                                 const rts_quadrature *q, const rts_options *opt);
rts_status rts_solve_decomposed(rts_decomp *d, const void *chi, const void *S, const rts_boundary *bc,
                                double tol, int max_iter, int *iters,
                                void *I_top, double *J, double *F, double *Q_rad);
const char *rts_decomposed_last_error(rts_decomp *d);
void rts_destroy_decomposed(rts_decomp *d);

#ifdef __cplusplus
}
#endif
#endif

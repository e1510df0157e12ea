// sweep.cuh -- persistent short-characteristics sweep (the paper's
// integrate(), Sect. 5.1, restructured for one launch).
//
// Work decomposition
//  * A sweep unit is (band, direction group): up to 4 directions that share
//    the dominant axis and its sign (the paper's "6 groups of 4 rays with a
//    similar dependency pattern", Sect. 5.3.3). Along the dominant axis (M)
//    the planes are sequential; each plane (P x Q) is 2-D parallel
//    (the wavefront of Sect. 5.1).
//  * A unit's plane is cut into tiles of TQ rows along Q spanning the whole
//    (periodic) P extent; thread p of the CTA owns column p of the tile. A
//    CTA owns one tile for the whole sweep and keeps the previous plane (I
//    and the seed-error bound g, by plane parity) and three planes of chi
//    and S (the next one prefetched a whole plane ahead with cp.async) in
//    shared memory. Each plane: integrate the interior rows; one thread
//    acquires the neighbours' flags (one 8-byte load: each tile keeps the
//    pair its two neighbours write) and every thread loads its column of their edge rows
//    into the halo rows; barrier; integrate the edge rows and write them to
//    the ring; barrier; release the tile's flag; only then store the
//    plane's partial sums, so the release never waits for those stores. Only the
//    first and last row of a tile cross CTAs: they are published to a small
//    global ring with a release flag per tile, and the neighbouring tiles
//    wait on that flag (bounded) before their next plane.
//    This is the tile-level DAG: node (tile, plane) depends on
//    (tile +-1, plane - 1). Tiles are handed out by an atomic ticket in
//    unit-major order, so every tile a CTA waits for is owned by a CTA that
//    is already running; one launch covers all bands and groups.
//  * P is always the unit-stride axis of the layout the unit reads (x for the
//    z and y groups; y for the x groups, which read a transposed copy made
//    once per solve -- the paper's "RTS Transpose", Sect. 5.3.1).
//
// Periodic wrap (x/y-dominant groups). The horizontal period closes the
// dependency chain. The paper iterates boundary intensities to a tolerance
// (Sect. 2, 5.1). Here the sweep simply keeps going around the period from a
// seed plane (I = S) and carries, per point and direction, a bound g on the
// remaining seed error: g = 1 on the seed plane, 0 on boundary-layer points,
// and g_p = e_p * sum_c beta_c g(corner c). The error of I at p is at most
// g_p times the seed error, and the plane maximum of g never grows. One bound
// is kept per point for the upward and one for the downward rays of a group
// (the maximum over the rays of each set, still a valid bound). Once the
// plane maximum, reduced over all tiles of the unit through a per-unit
// counter and a tagged atomic maximum, is below the tolerance L planes
// later, every later plane is converged; from then on one more full period
// is swept and accumulated. Unlike a residual test this needs no second pass
// to confirm convergence.
#pragma once
#include <climits>
#include <type_traits>

#include "common.cuh"

namespace rts {

constexpr int MAXD = 4;     // directions per sweep unit
constexpr int STORE_CH = 1; // values per slot kept by the checkpoint sweep
constexpr int HALO_CH = MAXD + 2;  // ring channels: I of each ray, g of up / down rays

// Rays of a unit sit in "sign slots": slot s holds the ray whose components
// along P and Q have signs sP = (s & 1 ? -1 : +1), sQ = (s & 2 ? -1 : +1), so
// its upwind corners are the compile-time offsets (0,0), (-sP,0), (0,-sQ),
// (-sP,-sQ). A slot without a ray is inactive (zero weights, not exported).
// In the x and y groups Q is z, so slots 0 and 1 hold rising rays and slots
// 2 and 3 descending ones.
struct SweepUnit {
    void *partial;              // [N][4] J, Fx, Fy, Fz of this unit, unit layout
    long long sQ, sM, N;        // strides of Q and M (elements), points
    long long halo_off;         // element offset of tile 0's halo block
    long long in_off;           // offset of this unit's band in chi, S (and their x-transposed copies)
    long long top_off;          // offset of this unit's band in I_top and the explicit bottom intensities
    long long dn_off;           // offset of this unit's band in the explicit top intensities
    int band, transposed;       // band index; reads the x-transposed copy
    int NP, NQ, NM;
    int axis, sa, wrap, qper;
    int TQ, ntiles, tile0;
    int nx, ny;
    int active[MAXD];           // slot holds a ray
    int up[MAXD], udx[MAXD];    // upward?; index among up (or down) rays
    double beta[MAXD][4];       // bilinear weights of corners (0,0),(1,0),(0,1),(1,1)
    double ds[MAXD];            // path length to the upwind plane
    double cJ[MAXD];            // w_d
    double cF[3][MAXD];         // 4 pi w_d n_d
    long long seed_off;         // x/y groups: element offset of the unit's wrap plane [NQ][NP][4] in the
                                // warm-start buffer (SweepArgs::seed)
};

template <typename T>
struct SweepArgs {
    const SweepUnit *units;
    const int *unit_of_tile;
    // register sweep: the tile that ticket k takes, tile_order[k] (every
    // unit's tiles consecutive); null: tile k
    const int *tile_order;
    int total_tiles;            // tiles of this launch: tile_base .. tile_base+total_tiles-1
    int tile_base, unit_base;   // first tile and first unit of this launch
    // optional (forward: checkpoint for the adjoint): per accumulated point
    // (offset off in the unit's layout) and slot d of unit u, at
    // store + (u-unit_base)*STORE_CH*MAXD*N + off*MAXD + d (the 4 slots of a
    // point together), the segment's D = dI/d(dtau) (0 at set points).
    // Reverse sweep: the gradient terms, see adjoint.cuh.
    T *store;
    // reverse (adjoint) sweep only
    const T *lam0, *lam0T;      // [B][N][4] cotangents of J_b, F_b (natural / x-transposed layout)
    const T *gitop;             // [B][n_up][ny][nx] cotangent of I_top, or null
    const T *ckpt;              // the checkpoint sweep's store (layout of `store`, forward)
    // per-call data
    const T *chi, *S;           // [B][N] natural layout
    const T *chiT, *ST;         // [B][N] x-transposed layout ([i][k][j])
    T *itop;                    // [B][n_up][ny][nx] or null
    const T *bc_up, *bc_dn;     // explicit boundary arrays or null
    int bc_bottom, bc_top;      // rts_bc_kind of the up / down rays
    int n_up, n_dn;
    // scratch
    int *ticket;
    // [total_tiles][2]: per tile the planes (+1) its lower and its upper
    // neighbour have published, read together
    int *flags;
    T *halo;                    // per tile: [2 slots][2 sides][HALO_CH][NP]
    unsigned int *gcnt;         // [units][R] tiles that posted a plane (cumulative per slot)
    unsigned long long *gmax;   // [units][R] (plane+1)<<32 | bits(max g), atomic max
    unsigned int *pcnt;         // [units][4] tiles that posted a period's wrap residual (warm start)
    unsigned long long *pmax;   // [units][4] (period+1)<<32 | bits(residual), atomic max
    int R, L;
    int *status;
    int *unit_tacc;             // per unit: first accumulated step
    float tol;
    int max_periods;
    // warm start of the periodic wrap (register sweep, x/y groups): per unit the
    // intensities of its wrap plane (the plane upwind of the first swept one),
    // written with the converged values; with seed_in they are also the
    // starting values, and periods are swept until that plane changes by at
    // most seed_tol (relative) over a period
    T *seed;
    int seed_in;
    float seed_tol;
    unsigned long long timeout_ns;
};

// ---------------------------------------------------------------------------
// Linear-in-tau weights of one segment (S linear in optical depth):
//   e = exp(-x), w_up = (1-e)/x - e, w_p = 1 - (1-e)/x
// For small x both weights lose digits to cancellation, so below a switch
// point they are evaluated from polynomials in x: in FP64 their Taylor series
// (obtained from the series of exp), in FP32 Chebyshev interpolants.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void seg_weights(float x, float &e, float &wu, float &wp)
{
    // FP32: below the switch point x times the degree-4 polynomials that
    // interpolate w_up / x and w_p / x at the Chebyshev nodes of [0, 1/4]
    // (relative error below 5e-9 there); both forms are evaluated and one
    // selected, so the lanes of a warp never diverge here
    e = __expf(-x);
    const float q = __fdividef(1.f - e, x);
    const float pu =
        x * (0.49999999793f + x * (-0.33333291823f + x * (0.12498666530f + x * (-0.03318270431f + x * 0.00624265650f))));
    const float pp =
        x * (0.49999999965f + x * (-0.16666659659f + x * (0.04166441676f + x * (-0.00830794980f + x * 0.00127094972f))));
    const bool small = x < 0.25f;
    wu = small ? pu : q - e;
    wp = small ? pp : 1.f - q;
}

__device__ __forceinline__ void seg_weights(double x, double &e, double &wu, double &wp)
{
    e = exp(-x);
    if (x < 0.01) {
        wp = x * (0.5 - x * (1.0 / 6.0 - x * (1.0 / 24.0 - x * (1.0 / 120.0 - x * (1.0 / 720.0 - x * (1.0 / 5040.0))))));
        wu = x * (0.5 - x * (2.0 / 6.0 - x * (3.0 / 24.0 - x * (4.0 / 120.0 - x * (5.0 / 720.0 - x * (6.0 / 5040.0))))));
    } else {
        double ome = -expm1(-x);
        double q = ome / x;
        wu = q - e;
        wp = 1.0 - q;
    }
}

// The same segment in the form the sweep evaluates. With q = (1 - e)/x the
// weights are w_up = q - e and w_p = 1 - q, so
//   I = I_up + w_up (S_up - I_up) + w_p (S_p - I_up) = S_p + e (I_up - S_up) + q (S_up - S_p),
// which needs e and q only. Below the switch point, where 1 - e cancels, q
// is a polynomial: in FP64 its Taylor series (sum over n of (-x)^n / (n+1)!),
// in FP32 the degree-4 polynomial interpolating q at the 5 Chebyshev nodes of
// [0, 1/4] (relative error below 3e-9 there, under the FP32 rounding of its
// evaluation); FP32 evaluates both forms and selects, without a branch.
__device__ __forceinline__ void seg_eq(float x, float &e, float &q)
{
    e = __expf(-x);
    const float qd = __fdividef(1.f - e, x);
    const float qs =
        0.99999999758f + x * (-0.49999951482f + x * (0.16665108207f + x * (-0.04149065410f + x * 0.00751360622f)));
    q = x < 0.25f ? qs : qd;
}
__device__ __forceinline__ void seg_eq(double x, double &e, double &q)
{
    e = exp(-x);
    if (x < 0.01)
        q = 1.0 - x * (0.5 - x * (1.0 / 6.0 - x * (1.0 / 24.0 - x * (1.0 / 120.0 - x * (1.0 / 720.0 - x * (1.0 / 5040.0))))));
    else
        q = -expm1(-x) / x;
}

// Derivative of the new intensity with respect to x for the adjoint's
// checkpoint. With d w_p / dx = w_up / x and d w_up / dx = e - d w_p / dx,
//   dI/dx = -e I_up + w_up' S_up + w_p' S_p = e (S_up - I_up) + w_p' (S_p - S_up),
// so only w_p' = (q - e) / x is needed. It cancels for small x: below the
// switch point FP64 takes its Taylor series, FP32 the degree-4 polynomial
// interpolating w_up / x at the Chebyshev nodes of [0, 1/4] (relative error
// below 5e-9), selected without a branch.
__device__ __forceinline__ double seg_dwp(double x, double e, double q)
{
    if (x < 0.01)
        return 0.5 - x * (2.0 / 6.0 - x * (3.0 / 24.0 - x * (4.0 / 120.0 - x * (5.0 / 720.0 - x * (6.0 / 5040.0)))));
    return (q - e) / x;
}
__device__ __forceinline__ float seg_dwp(float x, float e, float q)
{
    const float small =
        0.49999999793f + x * (-0.33333291823f + x * (0.12498666530f + x * (-0.03318270431f + x * 0.00624265650f)));
    return x < 0.25f ? small : __fdividef(q - e, x);
}

__device__ __forceinline__ int plane_of(int t, int NM, int sa)
{
    int r = t % NM;
    if (r < 0) r += NM;
    return sa > 0 ? r : NM - 1 - r;
}

// natural (i, j) of a point given its (p, q, m) in a unit's layout
__device__ __forceinline__ void natural_ij(int axis, int p, int q, int m, int &i, int &j)
{
    if (axis == 2) { i = p; j = q; }
    else if (axis == 1) { i = p; j = m; }
    else { i = m; j = p; }
}

// Ray constants of the unit's slots in shared memory.
template <typename T>
struct __align__(16) DirConst {
    T beta[MAXD][4];
    T hds[MAXD];           // ds / 2
    T cJ[MAXD], cF[3][MAXD];
    int up[MAXD], bck[MAXD], udx[MAXD], active[MAXD];
};

// four consecutive values of a 16-byte aligned shared array in one or two loads
__device__ __forceinline__ void ld4(const float *p, float &a, float &b, float &c, float &d)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double &a, double &b, double &c, double &d)
{
    const double2 u = *reinterpret_cast<const double2 *>(p), v = *reinterpret_cast<const double2 *>(p + 2);
    a = u.x; b = u.y; c = v.x; d = v.y;
}

template <typename T>
__device__ __noinline__ T bc_value(const SweepArgs<T> &a, const SweepUnit &U, const DirConst<T> &D, int d,
                                     int p, int q, int m, T Sp)
{
    const int kind = D.bck[d];
    if (kind == 0) return T(0);
    if (kind == 1) return Sp;
    int i, j;
    natural_ij(U.axis, p, q, m, i, j);
    const long long plane = (long long)U.ny * U.nx;
    const T *arr = D.up[d] ? a.bc_up + U.top_off : a.bc_dn + U.dn_off;
    return arr[(long long)D.udx[d] * plane + (long long)j * U.nx + i];
}

// Shared memory of a tile, NPP = NP + 2 columns per row: column c = p + 1,
// columns 0 and NP+1 repeat p = NP-1 and p = 0 (periodic padding), so a P
// neighbour is always the next column. Each field has RW = TQ+2 rows (halo
// row, TQ own rows, halo row) and stores the values of a point together, so
// one vector load brings all of them:
//   sI  [RW][NPP][4]      the previous plane's intensities of the 4 slots
//   sXS [2][RW][NPP][2]   chi and S of plane t at parity t & 1
//   sG  [RW][NPP][2]      seed-error bounds of the up and down rays, bf16
//                         rounded up (still bounds; half the bytes, which
//                         leaves the SM more L1 cache)
// The previous plane's intensities and bounds are kept once: a plane's new
// values stay in registers until every thread has read the previous plane.
// chi and S are kept for two planes: the previous plane for the upwind
// interpolation, the current one for the own points; the slot of the plane
// before is refilled with cp.async a whole plane ahead.
template <typename T>
__host__ __device__ constexpr size_t tile_smem_bytes(int tq, int np)
{
    return (size_t)(tq + 2) * (np + 2) * (8 * sizeof(T) + 2 * sizeof(unsigned short));
}

// bf16 of a non-negative bound, rounded up, and back
__device__ __forceinline__ unsigned bound16(float g)
{
    unsigned b = __float_as_uint(g);
    if (b & 0xffffu) b += 0x10000u;
    return b >> 16;
}
__device__ __forceinline__ float bound32(unsigned short h) { return __uint_as_float((unsigned)h << 16); }

// vector accesses to 2 or 4 consecutive values (8 / 16 / 32-byte aligned)
__device__ __forceinline__ void ld2(const float *p, float &a, float &b)
{
    const float2 v = *reinterpret_cast<const float2 *>(p);
    a = v.x; b = v.y;
}
__device__ __forceinline__ void ld2(const double *p, double &a, double &b)
{
    const double2 v = *reinterpret_cast<const double2 *>(p);
    a = v.x; b = v.y;
}
__device__ __forceinline__ void st2(float *p, float a, float b) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }
__device__ __forceinline__ void st2(double *p, double a, double b)
{
    *reinterpret_cast<double2 *>(p) = make_double2(a, b);
}
__device__ __forceinline__ void st4(float *p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double *p, double a, double b, double c, double d)
{
    *reinterpret_cast<double2 *>(p) = make_double2(a, b);
    *reinterpret_cast<double2 *>(p + 2) = make_double2(c, d);
}

// New values of one point of a plane: the 4 slots' intensities and, during
// the periodic warm-up, the seed-error bounds of the up / down rays.
template <typename T, bool ACC>
struct RowVals {
    T v[MAXD];
    float g[2];
};
template <typename T>
struct RowVals<T, true> {
    T v[MAXD];
};

template <bool B>
using Flag = std::integral_constant<bool, B>;

// One tile of one sweep unit, from its first plane to the last. Thread p
// owns column p (p < NP) of rows q0 .. q0+nrows-1.
// CKPT: this launch keeps the adjoint's checkpoint (SweepArgs::store); the
// code for it is compiled only into the instantiations the adjoint uses.
template <typename T, int TQ, bool CKPT>
__device__ void run_tile(const SweepArgs<T> &a, const SweepUnit *__restrict__ Ug, int uidx, int r, int gt,
                         unsigned char *smem)
{
    constexpr int RW = TQ + 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NT = blockDim.x;
    // unit description in registers (the struct lives in global memory)
    const int NP = Ug->NP, NQ = Ug->NQ, NM = Ug->NM;
    const int axis = Ug->axis, sa = Ug->sa, ntl = Ug->ntiles, tile0 = Ug->tile0;
    const bool wrap = Ug->wrap != 0, qper = Ug->qper != 0;
    const int unx = Ug->nx, uny = Ug->ny;
    const long long sQ = Ug->sQ, sM = Ug->sM, N = Ug->N;
    const T *__restrict__ chi = (Ug->transposed ? a.chiT : a.chi) + Ug->in_off;
    const T *__restrict__ Sg = (Ug->transposed ? a.ST : a.S) + Ug->in_off;
    T *const itop = a.itop ? a.itop + Ug->top_off : nullptr;
    T *const part = (T *)Ug->partial;
    const long long tile_stride = (long long)2 * 2 * HALO_CH * NP;
    T *const halo_base = a.halo + Ug->halo_off;
    T *const myhalo = halo_base + (long long)r * tile_stride;

    const int q0 = r * TQ;
    const int nrows = min(TQ, NQ - q0);
    const int p = tid;
    const bool act = p < NP;
    const int c = p + 1;                        // smem column
    const int npp = NP + 2;
    const int FL = RW * npp;                    // points of one field
    T *const sI = (T *)smem;                    // [FL][4]
    T *const sXS = sI + 4 * FL;                 // [2][FL][2]
    unsigned short *const sG = (unsigned short *)(sXS + 4 * FL);  // [FL][2]
    auto fXS = [&](int t) -> T * { return sXS + (t & 1) * 2 * FL; };

    __shared__ DirConst<T> D;
    __shared__ float s_wmax[32];
    __shared__ int s_ctl[4];                    // 0 abort, 1 decision for the next plane
    __shared__ int s_q[RW];                     // global row of smem row k, -1 outside

    if (tid < MAXD) {
        const int d = tid;
        for (int cc = 0; cc < 4; ++cc) D.beta[d][cc] = (T)Ug->beta[d][cc];
        D.hds[d] = (T)(0.5 * Ug->ds[d]);
        D.cJ[d] = (T)Ug->cJ[d];
        for (int cc = 0; cc < 3; ++cc) D.cF[cc][d] = (T)Ug->cF[cc][d];
        D.up[d] = Ug->up[d];
        D.bck[d] = Ug->up[d] ? a.bc_bottom : a.bc_top;
        D.udx[d] = Ug->udx[d];
        D.active[d] = Ug->active[d];
    }
    if (tid < RW) {
        int q = q0 - 1 + tid;
        if (qper) q = (q % NQ + NQ) % NQ;
        else if (q < 0 || q >= NQ) q = -1;
        s_q[tid] = tid <= nrows + 1 ? q : -1;
    }
    if (tid == 0) { s_ctl[0] = 0; s_ctl[1] = 0; }

    const int t_first = wrap ? 0 : 1;
    const int lower = qper ? (r + ntl - 1) % ntl : r - 1;
    const int upper = qper ? (r + 1) % ntl : r + 1;
    const bool has_lower = qper || r > 0;
    const bool has_upper = qper || r < ntl - 1;

    // periodic padding: thread p = 0 also writes column NP + 1 and thread
    // p = NP - 1 column 0 (with NP == 1 the one thread writes both)
    const bool padA = act && (p == 0 || p == NP - 1), padB = act && NP == 1;
    const int pc = p == 0 ? NP + 1 : 0;
    auto put4 = [&](int k, T v0, T v1, T v2, T v3) {
        st4(sI + (k * npp + c) * 4, v0, v1, v2, v3);
        if (padA) st4(sI + (k * npp + pc) * 4, v0, v1, v2, v3);
        if (padB) st4(sI + (k * npp) * 4, v0, v1, v2, v3);
    };
    auto putG = [&](int k, float gu, float gd) {
        const unsigned w = bound16(gu) | bound16(gd) << 16;
        unsigned *const g32 = (unsigned *)sG;
        g32[k * npp + c] = w;
        if (padA) g32[k * npp + pc] = w;
        if (padB) g32[k * npp] = w;
    };
    auto putXS = [&](T *f, int k, T x, T s) {
        st2(f + (k * npp + c) * 2, x, s);
        if (padA) st2(f + (k * npp + pc) * 2, x, s);
        if (padB) st2(f + (k * npp) * 2, x, s);
    };
    // asynchronous copy of this thread's column of the chi/S rows of plane t
    // into slot t & 1
    auto prefetch_row = [&](T *f, long long mo, int k) __attribute__((always_inline)) {
        const int q = s_q[k];
        if (q < 0) {
            putXS(f, k, T(0), T(0));
            return;
        }
        const T *gx = chi + mo + (long long)q * sQ, *gs = Sg + mo + (long long)q * sQ;
        T *d0 = f + (k * npp + c) * 2;
        cp_async(d0, gx);
        cp_async(d0 + 1, gs);
        if (padA) { T *d1 = f + (k * npp + pc) * 2; cp_async(d1, gx); cp_async(d1 + 1, gs); }
        if (padB) { T *d1 = f + (k * npp) * 2; cp_async(d1, gx); cp_async(d1 + 1, gs); }
    };
    auto prefetch = [&](int t) {
        if (act) {
            const long long mo = (long long)plane_of(t, NM, sa) * sM + p;
            T *f = fXS(t);
            if (nrows == TQ) {  // full tile: the TQ + 2 rows unrolled
#pragma unroll
                for (int k = 0; k < TQ + 2; ++k) prefetch_row(f, mo, k);
            } else {
                for (int k = 0; k < nrows + 2; ++k) prefetch_row(f, mo, k);
            }
        }
        cp_async_commit();
    };

    __syncthreads();
    int actm = 0;  // slot bit mask: slot holds a ray
    for (int d = 0; d < MAXD; ++d) actm |= D.active[d] ? 1 << d : 0;

    // ---------------- prologue: the plane before the first integrated one ----
    const int tp = t_first - 1;
    prefetch(t_first);
    if (act) {
        const int m = plane_of(tp, NM, sa);
        const long long mo = (long long)m * sM + p;
        for (int k = 0; k < nrows + 2; ++k) {
            const int q = s_q[k];
            const bool ok = q >= 0;
            const long long off = mo + (long long)(ok ? q : 0) * sQ;
            const T x = ok ? chi[off] : T(0);
            const T s = ok ? Sg[off] : T(0);
            putXS(fXS(tp), k, x, s);
            float gu = 0.f, gd = 0.f;
            T v[MAXD];
            for (int d = 0; d < MAXD; ++d) {
                v[d] = T(0);
                const bool bcrow = wrap ? ((D.up[d] && q == 0) || (!D.up[d] && q == NQ - 1)) : true;
                if (ok && D.active[d]) {
                    if (bcrow) v[d] = bc_value(a, *Ug, D, d, p, q, m, s);
                    else {  // seed: I = S, unit seed-error bound
                        v[d] = s;
                        if (D.up[d]) gu = 1.f; else gd = 1.f;
                    }
                }
            }
            put4(k, v[0], v[1], v[2], v[3]);
            putG(k, gu, gd);
        }
        // z groups: the boundary plane is the first of the NM accumulated planes
        if (!wrap) {
            for (int k = 1; k <= nrows; ++k) {
                T v[MAXD];
                ld4(sI + (k * npp + c) * 4, v[0], v[1], v[2], v[3]);
                T aJ = 0, aX = 0, aY = 0, aZ = 0;
                for (int d = 0; d < MAXD; ++d) {
                    aJ += D.cJ[d] * v[d]; aX += D.cF[0][d] * v[d]; aY += D.cF[1][d] * v[d]; aZ += D.cF[2][d] * v[d];
                }
                const long long off = (long long)m * sM + (long long)s_q[k] * sQ + p;
                st4(part + off * 4, aJ, aX, aY, aZ);
                if (CKPT) {  // boundary plane: set points, no segment
                    st4(a.store + (long long)(uidx - a.unit_base) * STORE_CH * MAXD * N + off * MAXD, T(0), T(0), T(0),
                        T(0));
                }
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();

    int t_acc = wrap ? -1 : 0;
    // warm-up cap in planes whose bound was examined (the decision lags by L)
    const int warm_cap = a.max_periods * NM + a.L;
    const int dec_thread = NT > 32 ? 32 : 0;

    // One plane t (m its index along M). ACC: the plane is accumulated (the
    // periodic warm-up is over, or the unit has none). Returns 0 to go on,
    // 1 after the last plane, 2 to abandon the tile (a wait failed).
    auto plane_step = [&](auto ACC, int t, int m) __attribute__((always_inline)) -> int {
        constexpr bool acc = decltype(ACC)::value;
        using Row = RowVals<T, acc>;
        const bool last = acc && (t - t_acc == NM - 1);
        cp_async_wait_all();  // this thread's chi/S of plane t (read only by this thread in this step)

        const T *XSp = fXS(t + 1), *XSc = fXS(t);  // (t+1) & 1 == (t-1) & 1
        const bool top_plane = axis == 2 && t == NM - 1 && sa > 0;
        float gmax = 0.f;

        // new values of row k (1..nrows) from the previous plane in shared
        // memory; EDGE: a first or last row, the only ones that can lie on
        // the boundary layer of the x/y groups
        auto do_row = [&](int k, auto EDGE) __attribute__((always_inline)) -> Row {
            constexpr bool edge = decltype(EDGE)::value;
            Row out;
            T *v = out.v;
            const int q = q0 + k - 1;
            const int o = k * npp + c;
            // previous plane's chi and S on the 3 x 3 neighbourhood, shared by the rays
            T xs[3][3], ss[3][3];
#pragma unroll
            for (int dq = 0; dq < 3; ++dq)
#pragma unroll
                for (int dp = 0; dp < 3; ++dp) ld2(XSp + (o + (dq - 1) * npp + dp - 1) * 2, xs[dq][dp], ss[dq][dp]);
            T xp, sp;
            ld2(XSc + o * 2, xp, sp);
            // previous plane's I and bounds: slot d (signs sP = d & 1 ? -1 : 1,
            // sQ = d & 2 ? -1 : 1) interpolates at (q, p), (q, p - sP), (q - sQ, p),
            // (q - sQ, p - sP); the bounds of the x/y groups' rising rays (slots
            // 0, 1) are the first value of a point's pair, the descending ones'
            // (slots 2, 3) the second
            const T *Ib = sI + o * 4;
            const int ir = npp * 4;
            [[maybe_unused]] const unsigned short *Gb = sG + o * 2;
            [[maybe_unused]] const int gr = npp * 2;
            T hd[MAXD];
            ld4(D.hds, hd[0], hd[1], hd[2], hd[3]);
            [[maybe_unused]] float g[MAXD];
            [[maybe_unused]] T ck[STORE_CH][MAXD];
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                const int SP = (d & 1) ? -1 : 1, SQ = (d & 2) ? -1 : 1;  // compile time after unrolling
                T b0, b1, b2, b3;
                ld4(D.beta[d], b0, b1, b2, b3);
                const T *Id = Ib + d;
                const int oq = -SQ * ir;
                const T Iup = b0 * Id[0] + b1 * Id[-4 * SP] + b2 * Id[oq] + b3 * Id[oq - 4 * SP];
                const T xup = b0 * xs[1][1] + b1 * xs[1][1 - SP] + b2 * xs[1 - SQ][1] + b3 * xs[1 - SQ][1 - SP];
                const T sup = b0 * ss[1][1] + b1 * ss[1][1 - SP] + b2 * ss[1 - SQ][1] + b3 * ss[1 - SQ][1 - SP];
                T e, qw;
                const T x = hd[d] * (xup + xp);
                seg_eq(x, e, qw);
                v[d] = sp + e * (Iup - sup) + qw * (sup - sp);
                if constexpr (CKPT && acc)  // checkpoint for the adjoint: dI/dx of the segment
                    ck[0][d] = e * (sup - Iup) + seg_dwp(x, e, qw) * (sp - sup);
                if constexpr (!acc) {
                    const unsigned short *Gd = Gb + (d >> 1);
                    const int gq = -SQ * gr;
                    g[d] = (float)e * ((float)b0 * bound32(Gd[0]) + (float)b1 * bound32(Gd[-2 * SP]) +
                                       (float)b2 * bound32(Gd[gq]) + (float)b3 * bound32(Gd[gq - 2 * SP]));
                }
            }
            float gu = 0.f, gd = 0.f;
            if constexpr (!acc) {
                gu = fmaxf(g[0], g[1]);
                gd = fmaxf(g[2], g[3]);
            }
            // boundary layer of the x/y groups: set, not integrated
            bool bnd = false;
            if constexpr (edge) {
                bnd = wrap && (q == 0 || q == NQ - 1);
                if (bnd) {
                    for (int d = 0; d < MAXD; ++d)
                        if (d < 2 ? q == 0 : q == NQ - 1) v[d] = (actm >> d) & 1 ? bc_value(a, *Ug, D, d, p, q, m, sp) : T(0);
                    if (q == 0) gu = 0.f;
                    if (q == NQ - 1) gd = 0.f;
                }
            }
            // an empty slot has zero weights and path length (e = q = 1, I_up =
            // S_up = 0), so its intensity stays exactly 0 without a mask
            if constexpr (CKPT && acc) {
                T *st = a.store + (long long)(uidx - a.unit_base) * STORE_CH * MAXD * N +
                        ((long long)m * sM + (long long)q * sQ + p) * MAXD;
                T cv[MAXD];
#pragma unroll
                for (int d = 0; d < MAXD; ++d) {
                    const bool set = bnd && (d < 2 ? q == 0 : q == NQ - 1);
                    const bool live = ((actm >> d) & 1) && !set;
                    cv[d] = live ? ck[0][d] : T(0);
                }
                st4(st, cv[0], cv[1], cv[2], cv[3]);
            }
            if constexpr (!acc) {
                out.g[0] = gu;
                out.g[1] = gd;
                gmax = fmaxf(gmax, fmaxf(gu, gd));
            }
            return out;
        };

        // first and last rows go to the neighbours through the global ring
        auto to_ring = [&](int sd, const Row &rw) __attribute__((always_inline)) {
            T *dst = myhalo + ((long long)((t & 1) * 2 + sd) * HALO_CH) * NP + p;
#pragma unroll
            for (int d = 0; d < MAXD; ++d) dst[(long long)d * NP] = rw.v[d];
            if constexpr (!acc) {
                dst[(long long)MAXD * NP] = (T)rw.g[0];
                dst[(long long)(MAXD + 1) * NP] = (T)rw.g[1];
            }
        };

        // the plane's new rows, kept in registers until the previous plane is no
        // longer read: rows 1 .. nrows-1 in nR (constant indices only), the last in rl
        Row nR[TQ], rl;
        // a full tile (every tile but a short last one) takes the rows
        // without per-row guards, so their code can interleave
        const bool full = nrows == TQ;
        // ---- interior rows need only this tile's own rows of the previous
        //      plane; meanwhile the neighbours finish their edge rows ----
        if (act) {
            if (full) {
#pragma unroll
                for (int k = 2; k < TQ; ++k) nR[k - 1] = do_row(k, Flag<false>{});
            } else {
#pragma unroll
                for (int k = 2; k < TQ; ++k)
                    if (k < nrows) nR[k - 1] = do_row(k, Flag<false>{});
            }
        }
        // ---- one thread waits for the neighbours' plane t-1 (acquire); after
        //      the barrier every thread loads its column of their edge rows
        //      into the halo rows ----
        if (t > t_first) {
            if (tid == 0) {
                bool ok = true;
                ok = wait_pair_geq(a.flags + 2 * gt, has_lower ? t : INT_MIN, has_upper ? t : INT_MIN, a.status,
                                   a.timeout_ns);
                if (!ok) s_ctl[0] = 1;
            }
            __syncthreads();  // B0: the neighbours' rows of plane t-1 are published (or the wait failed)
            if (act && !s_ctl[0]) {
                const int hslot = (t - 1) & 1;
                for (int side = 0; side < 2; ++side) {
                    if (side == 0 ? !has_lower : !has_upper) continue;
                    const int nb = side == 0 ? lower : upper;
                    const int row = side == 0 ? 0 : nrows + 1;
                    // the neighbour below sends its last row (sd 1), the one above its first (sd 0)
                    const T *src = halo_base + (long long)nb * tile_stride +
                                   ((long long)(hslot * 2 + (side == 0 ? 1 : 0)) * HALO_CH) * NP + p;
                    T hv[HALO_CH];
#pragma unroll
                    for (int ch = 0; ch < HALO_CH; ++ch)
                        hv[ch] = (ch < MAXD || !acc) ? ld_cg(src + (long long)ch * NP) : T(0);
                    put4(row, hv[0], hv[1], hv[2], hv[3]);
                    if constexpr (!acc) putG(row, (float)hv[MAXD], (float)hv[MAXD + 1]);
                }
            }
        }
        __syncthreads();  // B1: halo rows of plane t-1 are in place
        if (s_ctl[0]) {
            cp_async_wait_all();
            return 2;
        }
        if (act) {
            nR[0] = do_row(1, Flag<true>{});
            to_ring(0, nR[0]);
            if (full) rl = TQ == 1 ? nR[0] : do_row(TQ, Flag<true>{});
            else rl = nrows == 1 ? nR[0] : do_row(nrows, Flag<true>{});
            to_ring(1, rl);
        }
        if constexpr (!acc) {
            for (int o = 16; o; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
            if (lane == 0) s_wmax[warp] = gmax;
            // decision for plane t+1 (its bound is L planes old: normally already complete)
            if (tid == dec_thread && t + 1 - a.L >= 0) {
                const int ts = t + 1 - a.L;
                const int slot = ts % a.R;
                const unsigned want = (unsigned)ntl * (unsigned)(ts / a.R + 1);
                bool ok = wait_count_geq(a.gcnt + (long long)uidx * a.R + slot, want, a.status, a.timeout_ns);
                if (ok) {
                    const unsigned long long v = ld_acquire64(a.gmax + (long long)uidx * a.R + slot);
                    if ((unsigned)(v >> 32) != (unsigned)(ts + 1)) {
                        atomicOr(a.status, ST_BADARG);  // ring overrun: never expected
                        ok = false;
                    } else {
                        s_ctl[1] = __uint_as_float((unsigned)(v & 0xffffffffu)) <= a.tol ? 1 : 0;
                    }
                }
                if (!ok) s_ctl[0] = 1;
            }
        }
        __syncthreads();  // B2: plane t's edge rows are in the ring; the previous plane is no longer read
        if (tid == 0) {
            // release the edge rows (the barrier orders the CTA's ring writes
            // before the fence) to the tile above, as its lower neighbour's,
            // and to the tile below, as its upper neighbour's
            fence_acq_rel_gpu();
            if (has_upper) st_relaxed(a.flags + 2 * (tile0 + upper), t + 1);
            if (has_lower) st_relaxed(a.flags + 2 * (tile0 + lower) + 1, t + 1);
            if constexpr (!acc) {
                float g = 0.f;
                for (int w = 0; w < (NT + 31) / 32; ++w) g = fmaxf(g, s_wmax[w]);
                const int slot = t % a.R;
                const unsigned long long pv = ((unsigned long long)(unsigned)(t + 1) << 32) | __float_as_uint(g);
                atomicMax(a.gmax + (long long)uidx * a.R + slot, pv);
                red_release_add(a.gcnt + (long long)uidx * a.R + slot, 1u);
            }
        }
        if (s_ctl[0]) return 2;
        // ---- plane t becomes the previous plane: own rows into shared memory;
        //      accumulated planes also go out as partial sums ----
        auto write_row = [&](int kk, const Row &rw) __attribute__((always_inline)) {
            put4(kk + 1, rw.v[0], rw.v[1], rw.v[2], rw.v[3]);
            if constexpr (!acc) {
                putG(kk + 1, rw.g[0], rw.g[1]);
            } else {
                const int q = q0 + kk;
                const long long off = (long long)m * sM + (long long)q * sQ + p;
                T cw[4][MAXD];
                ld4(D.cJ, cw[0][0], cw[0][1], cw[0][2], cw[0][3]);
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) ld4(D.cF[cc], cw[cc + 1][0], cw[cc + 1][1], cw[cc + 1][2], cw[cc + 1][3]);
                T aJ = 0, aX = 0, aY = 0, aZ = 0;
#pragma unroll
                for (int d = 0; d < MAXD; ++d) {
                    const T v = rw.v[d];
                    aJ += cw[0][d] * v; aX += cw[1][d] * v; aY += cw[2][d] * v; aZ += cw[3][d] * v;
                }
                st4(part + off * 4, aJ, aX, aY, aZ);
            }
        };
        // upward intensities leaving the top: the whole top plane of a z
        // group, the last row of an x/y group
        auto write_top = [&](int kk, const Row &rw) {
            const int q = q0 + kk;
            int i, j;
            natural_ij(axis, p, q, m, i, j);
            for (int d = 0; d < MAXD; ++d)
                if (D.up[d] && D.active[d]) itop[((long long)D.udx[d] * uny + j) * unx + i] = rw.v[d];
        };
        if (act) {
            if (full) {
#pragma unroll
                for (int kk = 0; kk < TQ - 1; ++kk) write_row(kk, nR[kk]);
                write_row(TQ - 1, rl);
            } else {
#pragma unroll
                for (int kk = 0; kk < TQ - 1; ++kk)
                    if (kk < nrows - 1) write_row(kk, nR[kk]);
                write_row(nrows - 1, rl);
            }
            if constexpr (acc) {
                if (itop) {
                    if (axis == 2 && top_plane) {
#pragma unroll
                        for (int kk = 0; kk < TQ - 1; ++kk)
                            if (kk < nrows - 1) write_top(kk, nR[kk]);
                        write_top(nrows - 1, rl);
                    } else if (axis != 2 && q0 + nrows == NQ) {
                        write_top(nrows - 1, rl);
                    }
                }
            }
        }
        if (last) return 1;
        prefetch(t + 1);  // into the slot of plane t-1 (no longer read)
        __syncthreads();  // B3: plane t is the previous plane for every thread
        return 0;
    };

    // the periodic warm-up and the accumulated planes run as two loops, each
    // compiled for its own phase
    int t = t_first;
    if (wrap) {
        for (;; ++t) {
            if (s_ctl[1]) {  // decision taken during the previous plane
                t_acc = t;
                if (r == 0 && tid == 0) a.unit_tacc[uidx] = t;
                break;
            }
            if (t >= warm_cap) {
                if (tid == 0) atomicOr(a.status, ST_NOCONV);
                cp_async_wait_all();
                return;  // every tile of the unit stops at the same plane; nothing in flight
            }
            if (plane_step(Flag<false>{}, t, plane_of(t, NM, sa)) == 2) return;
        }
    }
    for (;; ++t) {
        const int rc = plane_step(Flag<true>{}, t, plane_of(t, NM, sa));
        if (rc == 2) return;
        if (rc == 1) break;
    }
    cp_async_wait_all();
}

// MAXR caps the registers per thread so that two to four CTAs share an SM
template <typename T, int TQ, int MAXR, bool CKPT = false>
__global__ void __maxnreg__(MAXR) sweep_kernel(SweepArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_tile;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int tk = -1;
            if (ld_relaxed(a.status) == 0) tk = atomicAdd(a.ticket, 1);
            s_tile = tk;
        }
        __syncthreads();
        if (s_tile < 0 || s_tile >= a.total_tiles) return;
        const int tile = a.tile_base + s_tile;
        const int u = a.unit_of_tile[tile];
        run_tile<T, TQ, CKPT>(a, a.units + u, u, tile - a.units[u].tile0, tile, smem);
    }
}

}  // namespace rts

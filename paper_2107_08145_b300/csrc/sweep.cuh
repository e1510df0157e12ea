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
//    CTA owns one tile for the whole sweep and keeps the previous plane
//    (I, chi, S and the seed-error bound g) in shared memory; chi and S of the
//    next plane are prefetched with cp.async into a two-slot ring. Only the
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
#include "common.cuh"

namespace rts {

constexpr int MAXD = 4;     // directions per sweep unit
constexpr int HALO_CH = MAXD + 2;  // ring channels: I of each ray, g of up / down rays

struct SweepUnit {
    void *partial;              // [4][N] J, Fx, Fy, Fz of this unit, unit layout
    long long sQ, sM, N;        // strides of Q and M (elements), points
    long long halo_off;         // element offset of tile 0's halo block
    int band, transposed;       // band index; reads the x-transposed copy
    int NP, NQ, NM;
    int axis, sa, wrap, qper, nd;
    int TQ, ntiles, tile0;
    int nx, ny;
    double beta[MAXD][4];       // bilinear weights of corners (0,0),(1,0),(0,1),(1,1)
    double ds[MAXD];            // path length to the upwind plane
    double cJ[MAXD];            // w_d
    double cF[3][MAXD];         // 4 pi w_d n_d
    int sP[MAXD], sQd[MAXD];    // corner step along P and Q is -sP, -sQ
    int up[MAXD], udx[MAXD];    // upward?; index among up (or down) directions
};

template <typename T>
struct SweepArgs {
    const SweepUnit *units;
    const int *unit_of_tile;
    int total_tiles;
    // per-call data
    const T *chi, *S;           // [B][N] natural layout
    const T *chiT, *ST;         // [B][N] x-transposed layout ([i][k][j])
    T *itop;                    // [B][n_up][ny][nx] or null
    const T *bc_up, *bc_dn;     // explicit boundary arrays or null
    int bc_bottom, bc_top;      // rts_bc_kind of the up / down rays
    int n_up, n_dn;
    // scratch
    int *ticket;
    int *flags;                 // [total_tiles] published plane + 1
    T *halo;                    // per tile: [2 slots][2 sides][HALO_CH][NP]
    unsigned int *gcnt;         // [units][R] tiles that posted a plane (cumulative per slot)
    unsigned long long *gmax;   // [units][R] (plane+1)<<32 | bits(max g), atomic max
    int R, L;
    int *status;
    int *unit_tacc;             // per unit: first accumulated step
    float tol;
    int max_periods;
    unsigned long long timeout_ns;
};

// ---------------------------------------------------------------------------
// Linear-in-tau weights of one segment (S linear in optical depth):
//   e = exp(-x), w_up = (1-e)/x - e, w_p = 1 - (1-e)/x
// For small x both weights lose digits to cancellation, so below a switch
// point they are evaluated from their Taylor series in x (obtained from the
// series of exp).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void seg_weights(float x, float &e, float &wu, float &wp)
{
    e = __expf(-x);
    if (x < 0.25f) {
        wp = x * (0.5f - x * (1.f / 6.f - x * (1.f / 24.f - x * (1.f / 120.f - x * (1.f / 720.f - x * (1.f / 5040.f - x * (1.f / 40320.f)))))));
        wu = x * (0.5f - x * (2.f / 6.f - x * (3.f / 24.f - x * (4.f / 120.f - x * (5.f / 720.f - x * (6.f / 5040.f - x * (7.f / 40320.f)))))));
    } else {
        float q = __fdividef(1.f - e, x);
        wu = q - e;
        wp = 1.f - q;
    }
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

// Direction constants of the unit in shared memory.
template <typename T>
struct DirConst {
    T beta[MAXD][4];
    T hds[MAXD];           // ds / 2
    T cJ[MAXD], cF[3][MAXD];
    int sP[MAXD], sQ[MAXD], up[MAXD], bck[MAXD], udx[MAXD];
};

template <typename T>
__device__ __forceinline__ T bc_value(const SweepArgs<T> &a, const SweepUnit &U, const DirConst<T> &D, int d,
                                     int p, int q, int m, T Sp)
{
    const int kind = D.bck[d];
    if (kind == 0) return T(0);
    if (kind == 1) return Sp;
    int i, j;
    natural_ij(U.axis, p, q, m, i, j);
    const long long plane = (long long)U.ny * U.nx;
    const T *arr = D.up[d] ? a.bc_up + (long long)U.band * a.n_up * plane
                           : a.bc_dn + (long long)U.band * a.n_dn * plane;
    return arr[(long long)D.udx[d] * plane + (long long)j * U.nx + i];
}

// One tile of one sweep unit, from its first plane to the last. Thread p
// owns column p (p < NP) of rows q0 .. q0+nrows-1.
template <typename T, int TQ>
__device__ void run_tile(const SweepArgs<T> &a, const SweepUnit &U, int uidx, int r, int gt,
                         unsigned char *smem)
{
    constexpr int RW = TQ + 2;                  // rows in shared memory incl. halo rows
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NT = blockDim.x;
    const int NP = U.NP, NQ = U.NQ, NM = U.NM, nd = U.nd;
    const int q0 = r * TQ;
    const int nrows = min(TQ, NQ - q0);
    const int p = tid;
    const bool act = p < NP;
    const int pm = p == 0 ? NP - 1 : p - 1;
    const int pn = p >= NP - 1 ? 0 : p + 1;
    const T *__restrict__ chi = (U.transposed ? a.chiT : a.chi) + (long long)U.band * U.N;
    const T *__restrict__ Sg = (U.transposed ? a.ST : a.S) + (long long)U.band * U.N;
    T *const itop = a.itop ? a.itop + (long long)U.band * a.n_up * U.ny * U.nx : nullptr;
    T *const part = (T *)U.partial;

    const int PL = RW * NP;                     // one smem plane
    T *sI = (T *)smem;                          // [MAXD][RW][NP] previous plane
    T *sX = sI + MAXD * PL;                     // [2][RW][NP] chi ring (slot = plane & 1)
    T *sS = sX + 2 * PL;                        // [2][RW][NP] S ring
    float *sG = (float *)(sS + 2 * PL);         // [2][RW][NP] seed-error bound (up, down)
    __shared__ DirConst<T> D;
    __shared__ float s_wmax[32];
    __shared__ int s_ctl[4];                    // 0 abort, 2 decision

    if (tid < MAXD) {
        const int d = tid;
        for (int c = 0; c < 4; ++c) D.beta[d][c] = (T)U.beta[d][c];
        D.hds[d] = (T)(0.5 * U.ds[d]);
        D.cJ[d] = (T)U.cJ[d];
        for (int c = 0; c < 3; ++c) D.cF[c][d] = (T)U.cF[c][d];
        D.sP[d] = U.sP[d];
        D.sQ[d] = U.sQd[d];
        D.up[d] = U.up[d];
        D.bck[d] = U.up[d] ? a.bc_bottom : a.bc_top;
        D.udx[d] = U.udx[d];
    }
    if (tid == 0) { s_ctl[0] = 0; s_ctl[2] = 0; }

    // global row of smem row k (0 .. nrows+1), or -1 outside a non-periodic Q
    auto grow = [&](int k) -> int {
        int q = q0 - 1 + k;
        if (U.qper) return (q % NQ + NQ) % NQ;
        return (q >= 0 && q < NQ) ? q : -1;
    };
    const int t_first = U.wrap ? 0 : 1;
    const int ntl = U.ntiles;
    const int lower = U.qper ? (r + ntl - 1) % ntl : r - 1;
    const int upper = U.qper ? (r + 1) % ntl : r + 1;
    const bool has_lower = U.qper || r > 0;
    const bool has_upper = U.qper || r < ntl - 1;
    const long long tile_stride = (long long)2 * 2 * HALO_CH * NP;
    T *__restrict__ myhalo = a.halo + U.halo_off + (long long)r * tile_stride;

    // asynchronous copy of the chi/S rows of plane t into ring slot t & 1
    auto prefetch = [&](int t) {
        const int m = plane_of(t, NM, U.sa);
        const long long mo = (long long)m * U.sM;
        const int slot = t & 1;
        if (act) {
            for (int k = 0; k < nrows + 2; ++k) {
                const int q = grow(k);
                T *dx = sX + slot * PL + k * NP + p;
                T *ds = sS + slot * PL + k * NP + p;
                if (q < 0) { *dx = T(0); *ds = T(0); continue; }
                const long long off = mo + (long long)q * U.sQ + p;
                cp_async(dx, chi + off);
                cp_async(ds, Sg + off);
            }
        }
        cp_async_commit();
    };

    __syncthreads();

    // ---------------- prologue: the plane before the first integrated one ----
    {
        const int tp = t_first - 1;
        const int m = plane_of(tp, NM, U.sa);
        const long long mo = (long long)m * U.sM;
        const int slot = tp & 1;
        if (act) {
            for (int k = 0; k < nrows + 2; ++k) {
                const int q = grow(k);
                const bool ok = q >= 0;
                const long long off = mo + (long long)(ok ? q : 0) * U.sQ + p;
                const T x = ok ? chi[off] : T(0);
                const T s = ok ? Sg[off] : T(0);
                sX[slot * PL + k * NP + p] = x;
                sS[slot * PL + k * NP + p] = s;
                float gu = 0.f, gd = 0.f;
                for (int d = 0; d < nd; ++d) {
                    T v;
                    const bool bcrow = U.wrap ? ((D.up[d] && q == 0) || (!D.up[d] && q == NQ - 1)) : true;
                    if (!ok) v = T(0);
                    else if (bcrow) v = bc_value(a, U, D, d, p, q, m, s);
                    else {  // seed: I = S, unit seed-error bound
                        v = s;
                        if (D.up[d]) gu = 1.f; else gd = 1.f;
                    }
                    sI[d * PL + k * NP + p] = v;
                }
                sG[k * NP + p] = gu;
                sG[PL + k * NP + p] = gd;
            }
        }
        __syncthreads();
        // z groups: the boundary plane is the first of the NM accumulated planes
        if (!U.wrap && act) {
            for (int k = 1; k <= nrows; ++k) {
                const int q = q0 + k - 1;
                T aJ = 0, aX = 0, aY = 0, aZ = 0;
                for (int d = 0; d < nd; ++d) {
                    const T v = sI[d * PL + k * NP + p];
                    aJ += D.cJ[d] * v; aX += D.cF[0][d] * v; aY += D.cF[1][d] * v; aZ += D.cF[2][d] * v;
                }
                const long long off = (long long)m * U.sM + (long long)q * U.sQ + p;
                part[off] = aJ; part[U.N + off] = aX; part[2 * U.N + off] = aY; part[3 * U.N + off] = aZ;
            }
        }
    }
    prefetch(t_first);

    int t_acc = U.wrap ? -1 : 0;
    const int warm_cap = a.max_periods * NM;
    const int dec_thread = NT > 32 ? 32 : 0;

    for (int t = t_first;; ++t) {
        const int m = plane_of(t, NM, U.sa);
        const bool acc_before = t_acc >= 0;  // same in every thread
        const bool need_decision = !acc_before && t - a.L >= 0;
        // ---- (A) plane t's chi/S landed; neighbours published plane t-1; wrap decision ----
        if (tid == 0 && t > t_first) {
            bool ok = true;
            if (has_lower) ok = wait_flag_geq(a.flags + U.tile0 + lower, t, a.status, a.timeout_ns);
            if (ok && has_upper) ok = wait_flag_geq(a.flags + U.tile0 + upper, t, a.status, a.timeout_ns);
            if (!ok) s_ctl[0] = 1;
        }
        if (tid == dec_thread && need_decision) {
            const int ts = t - a.L;
            const int slot = ts % a.R;
            const unsigned want = (unsigned)ntl * (unsigned)(ts / a.R + 1);
            const unsigned int *cnt = a.gcnt + (long long)uidx * a.R + slot;
            bool ok = wait_count_geq(cnt, want, a.status, a.timeout_ns);
            if (ok) {
                const unsigned long long v = ld_acquire64(a.gmax + (long long)uidx * a.R + slot);
                if ((unsigned)(v >> 32) != (unsigned)(ts + 1)) {
                    atomicOr(a.status, ST_BADARG);  // ring overrun: never expected
                    ok = false;
                } else {
                    s_ctl[2] = __uint_as_float((unsigned)(v & 0xffffffffu)) <= a.tol ? 1 : 0;
                }
            }
            if (!ok) s_ctl[0] = 1;
        }
        cp_async_wait_all();
        __syncthreads();
        if (s_ctl[0]) return;
        if (need_decision && s_ctl[2]) {
            t_acc = t;
            if (r == 0 && tid == 0) a.unit_tacc[uidx] = t;
        }
        if (U.wrap && t_acc < 0 && t >= warm_cap) {
            if (tid == 0) atomicOr(a.status, ST_NOCONV);
            return;  // every tile of the unit stops at the same plane
        }
        const bool acc = t_acc >= 0;

        // ---- (B) neighbours' edge rows of plane t-1 -> smem rows 0 and nrows+1 ----
        if (t > t_first && act) {
            const int slot = (t - 1) & 1;
            for (int side = 0; side < 2; ++side) {
                if (side == 0 ? !has_lower : !has_upper) continue;
                const int nb = side == 0 ? lower : upper;
                const int row = side == 0 ? 0 : nrows + 1;
                // the neighbour below sends its last row (sd 1), the one above its first (sd 0)
                const T *src = a.halo + U.halo_off + (long long)nb * tile_stride +
                               ((long long)(slot * 2 + (side == 0 ? 1 : 0)) * HALO_CH) * NP + p;
                for (int d = 0; d < nd; ++d) sI[d * PL + row * NP + p] = ld_cg(src + (long long)d * NP);
                if (!acc) {
                    sG[row * NP + p] = (float)ld_cg(src + (long long)MAXD * NP);
                    sG[PL + row * NP + p] = (float)ld_cg(src + (long long)(MAXD + 1) * NP);
                }
            }
        }
        __syncthreads();

        // ---- (C) integrate the own points of plane t ----
        const T *Xp = sX + ((t - 1) & 1) * PL, *Sp = sS + ((t - 1) & 1) * PL;
        const T *Xc = sX + (t & 1) * PL, *Sc = sS + (t & 1) * PL;
        T nI[TQ][MAXD];
        float nG[TQ][2];
        float gmax = 0.f;
#pragma unroll
        for (int k = 0; k < TQ; ++k) {
            const int row = k + 1;
            nG[k][0] = 0.f;
            nG[k][1] = 0.f;
            if (!act || row > nrows) continue;
            const int q = q0 + k;
            const T xp = Xc[row * NP + p], sp = Sc[row * NP + p];
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                if (d >= nd) break;
                const bool bcrow = U.wrap && ((D.up[d] && q == 0) || (!D.up[d] && q == NQ - 1));
                if (bcrow) {
                    nI[k][d] = bc_value(a, U, D, d, p, q, m, sp);
                    continue;
                }
                const int pc = D.sP[d] > 0 ? pm : pn;
                const int rc = row - D.sQ[d];
                const int i0 = row * NP + p, i1 = row * NP + pc, i2 = rc * NP + p, i3 = rc * NP + pc;
                const T b0 = D.beta[d][0], b1 = D.beta[d][1], b2 = D.beta[d][2], b3 = D.beta[d][3];
                const T *Id = sI + d * PL;
                const T Iup = b0 * Id[i0] + b1 * Id[i1] + b2 * Id[i2] + b3 * Id[i3];
                const T xup = b0 * Xp[i0] + b1 * Xp[i1] + b2 * Xp[i2] + b3 * Xp[i3];
                const T sup = b0 * Sp[i0] + b1 * Sp[i1] + b2 * Sp[i2] + b3 * Sp[i3];
                const T x = D.hds[d] * (xup + xp);
                T e, wu, wp;
                seg_weights(x, e, wu, wp);
                nI[k][d] = Iup + wu * (sup - Iup) + wp * (sp - Iup);
                if (!acc) {
                    const int grp = D.up[d] ? 0 : 1;
                    const float *Gd = sG + grp * PL;
                    const float g = (float)e * ((float)b0 * Gd[i0] + (float)b1 * Gd[i1] + (float)b2 * Gd[i2] +
                                                (float)b3 * Gd[i3]);
                    nG[k][grp] = fmaxf(nG[k][grp], g);
                }
            }
            gmax = fmaxf(gmax, fmaxf(nG[k][0], nG[k][1]));
        }
        if (!acc) {
            for (int o = 16; o; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
            if (lane == 0) s_wmax[warp] = gmax;
        }
        __syncthreads();

        // ---- (D) plane t becomes the previous plane; publish edge rows ----
        const int oslot = t & 1;
        const bool last = acc && (t - t_acc == NM - 1);
        if (!last) prefetch(t + 1);  // into the slot of plane t-1, no longer read
#pragma unroll
        for (int k = 0; k < TQ; ++k) {
            const int row = k + 1;
            if (!act || row > nrows) continue;
            const int q = q0 + k;
            T aJ = 0, aX = 0, aY = 0, aZ = 0;
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                if (d >= nd) break;
                const T v = nI[k][d];
                sI[d * PL + row * NP + p] = v;
                aJ += D.cJ[d] * v; aX += D.cF[0][d] * v; aY += D.cF[1][d] * v; aZ += D.cF[2][d] * v;
            }
            if (!acc) {
                sG[row * NP + p] = nG[k][0];
                sG[PL + row * NP + p] = nG[k][1];
            }
            for (int sd = 0; sd < 2; ++sd) {
                if (!((sd == 0 && row == 1) || (sd == 1 && row == nrows))) continue;
                T *dst = myhalo + ((long long)(oslot * 2 + sd) * HALO_CH) * NP + p;
                for (int d = 0; d < nd; ++d) dst[(long long)d * NP] = nI[k][d];
                if (!acc) {
                    dst[(long long)MAXD * NP] = (T)nG[k][0];
                    dst[(long long)(MAXD + 1) * NP] = (T)nG[k][1];
                }
            }
            if (acc) {
                const long long off = (long long)m * U.sM + (long long)q * U.sQ + p;
                part[off] = aJ; part[U.N + off] = aX; part[2 * U.N + off] = aY; part[3 * U.N + off] = aZ;
                if (itop) {
                    const bool top = U.axis == 2 ? (t == NM - 1 && U.sa > 0) : (q == NQ - 1);
                    if (top) {
                        int i, j;
                        natural_ij(U.axis, p, q, m, i, j);
                        for (int d = 0; d < nd; ++d)
                            if (D.up[d]) itop[((long long)D.udx[d] * U.ny + j) * U.nx + i] = nI[k][d];
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            if (!acc) {
                float g = 0.f;
                for (int w = 0; w < (NT + 31) / 32; ++w) g = fmaxf(g, s_wmax[w]);
                const int slot = t % a.R;
                const unsigned long long v = ((unsigned long long)(unsigned)(t + 1) << 32) | __float_as_uint(g);
                atomicMax(a.gmax + (long long)uidx * a.R + slot, v);
                __threadfence();
                atomicAdd(a.gcnt + (long long)uidx * a.R + slot, 1u);
            }
            __threadfence();
            st_release(a.flags + gt, t + 1);
        }
        if (last) break;
    }
}

template <typename T, int TQ>
__global__ void __launch_bounds__(1024) sweep_kernel(SweepArgs<T> a)
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
        const int tile = s_tile;
        if (tile < 0 || tile >= a.total_tiles) return;
        const int u = a.unit_of_tile[tile];
        const SweepUnit &U = a.units[u];
        run_tile<T, TQ>(a, U, u, tile - U.tile0, tile, smem);
    }
}

}  // namespace rts

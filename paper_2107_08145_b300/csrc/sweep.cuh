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
//    (periodic) P extent. A CTA owns one tile for the whole sweep and keeps
//    the previous plane (I, chi, S and the seed-error bound g) in shared
//    memory. Only the first and last row of a tile cross CTAs: they are
//    published to a small global ring with a release flag per tile, and the
//    neighbouring tiles wait on that flag (bounded) before their next plane.
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
// g_p times the seed error, and the plane maximum of g never grows. Once the
// plane maximum (reduced over all tiles of the unit, L planes later) is below
// the tolerance, every later plane is converged; from then on one more full
// period is swept and accumulated. Unlike a residual test this needs no
// second pass to confirm convergence.
#pragma once
#include "common.cuh"

namespace rts {

constexpr int MAXD = 4;     // directions per sweep unit
constexpr int SWEEP_NT = 256;

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
    T *halo;                    // per tile: [2 slots][2 sides][2*MAXD channels][NP]
    unsigned long long *gsync;  // [total_tiles][R] (step+1)<<32 | bits(g)
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

// One tile of one sweep unit, from its first plane to the last.
template <typename T, int PPT>
__device__ void run_tile(const SweepArgs<T> &a, const SweepUnit &U, int uidx, int r, int gt,
                         unsigned char *smem)
{
    constexpr int NT = SWEEP_NT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int NP = U.NP, NQ = U.NQ, NM = U.NM, nd = U.nd;
    const int q0 = r * U.TQ;
    const int nrows = min(U.TQ, NQ - q0);
    const int RW = U.TQ + 2;                 // smem row stride (rows incl. halo)
    const int npts = nrows * NP;
    const T *__restrict__ chi = (U.transposed ? a.chiT : a.chi) + (long long)U.band * U.N;
    const T *__restrict__ Sg = (U.transposed ? a.ST : a.S) + (long long)U.band * U.N;
    T *const itop = a.itop ? a.itop + (long long)U.band * a.n_up * U.ny * U.nx : nullptr;

    // shared memory carve-up
    T *sI = (T *)smem;                        // [MAXD][RW][NP]
    T *sX = sI + MAXD * RW * NP;              // [RW][NP] chi of previous plane
    T *sS = sX + RW * NP;                     // [RW][NP] S of previous plane
    float *sG = (float *)(sS + RW * NP);      // [MAXD][RW][NP] seed-error bound
    __shared__ DirConst<T> D;
    __shared__ float s_wmax[NT / 32];
    __shared__ int s_ctl[4];                  // 0: abort, 1: accumulate, 2: decision

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
    if (tid == 0) { s_ctl[0] = 0; s_ctl[1] = U.wrap ? 0 : 1; s_ctl[2] = 0; }

    // own points: (p, row) with row 1..nrows in smem coordinates
    int pp_[PPT], row_[PPT], pm_[PPT], pn_[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        int l = tid + k * NT;
        if (l >= npts) l = 0;
        pp_[k] = l % NP;
        row_[k] = l / NP + 1;
        pm_[k] = pp_[k] == 0 ? NP - 1 : pp_[k] - 1;
        pn_[k] = pp_[k] == NP - 1 ? 0 : pp_[k] + 1;
    }
    // halo rows of chi/S are loaded by the "halo mapping": h in [0, 2 NP)
    const int nh = 2 * NP;
    auto halo_q = [&](int side) -> int {  // global row of halo side 0 (below) / 1 (above)
        int q = side == 0 ? q0 - 1 : q0 + nrows;
        if (U.qper) q = (q % NQ + NQ) % NQ;
        return q;
    };
    const int qlo = halo_q(0), qhi = halo_q(1);
    const bool lo_ok = U.qper || qlo >= 0;
    const bool hi_ok = U.qper || qhi < NQ;

    const int t_first = U.wrap ? 0 : 1;
    const int ntl = U.ntiles;
    const int lower = U.qper ? (r + ntl - 1) % ntl : r - 1;
    const int upper = U.qper ? (r + 1) % ntl : r + 1;
    const bool has_lower = U.qper || r > 0;
    const bool has_upper = U.qper || r < ntl - 1;
    T *__restrict__ myhalo = a.halo + U.halo_off + (long long)r * (8 * MAXD * NP);

    __syncthreads();

    // ---------------- prologue: the plane before the first integrated one --------------
    {
        const int m = plane_of(t_first - 1, NM, U.sa);
        const long long mo = (long long)m * U.sM;
        for (int l = tid; l < (nrows + 2) * NP; l += NT) {
            const int row = l / NP, p = l % NP;
            int q = q0 - 1 + row;
            bool ok = true;
            if (U.qper) q = (q % NQ + NQ) % NQ;
            else ok = q >= 0 && q < NQ;
            const T x = ok ? chi[mo + (long long)q * U.sQ + p] : T(0);
            const T s = ok ? Sg[mo + (long long)q * U.sQ + p] : T(0);
            sX[row * NP + p] = x;
            sS[row * NP + p] = s;
            for (int d = 0; d < nd; ++d) {
                T v;
                float g;
                const bool bcrow = U.wrap ? ((D.up[d] && q == 0) || (!D.up[d] && q == NQ - 1)) : true;
                if (!ok) { v = T(0); g = 0.f; }
                else if (bcrow) { v = bc_value(a, U, D, d, p, q, m, s); g = 0.f; }
                else { v = s; g = 1.f; }          // seed: I = S
                sI[(d * RW + row) * NP + p] = v;
                sG[(d * RW + row) * NP + p] = g;
            }
        }
    }
    __syncthreads();
    // z groups: the boundary plane is the first of the NM accumulated planes
    if (!U.wrap) {
        const int m = plane_of(0, NM, U.sa);
        T *part = (T *)U.partial;
        for (int l = tid; l < npts; l += NT) {
            const int row = l / NP + 1, p = l % NP;
            const int q = q0 + row - 1;
            T aJ = 0, aX = 0, aY = 0, aZ = 0;
            for (int d = 0; d < nd; ++d) {
                const T v = sI[(d * RW + row) * NP + p];
                aJ += D.cJ[d] * v; aX += D.cF[0][d] * v; aY += D.cF[1][d] * v; aZ += D.cF[2][d] * v;
            }
            const long long off = (long long)m * U.sM + (long long)q * U.sQ + p;
            part[off] = aJ; part[U.N + off] = aX; part[2 * U.N + off] = aY; part[3 * U.N + off] = aZ;
        }
    }

    // current-plane registers: own chi/S and halo-row chi/S of plane t
    T cx[PPT], cs[PPT];
    constexpr int HPT = 8;
    T hx[HPT], hs[HPT];
    auto load_plane = [&](int t) {
        const int m = plane_of(t, NM, U.sa);
        const long long mo = (long long)m * U.sM;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int l = tid + k * NT;
            if (l < npts) {
                const long long off = mo + (long long)(q0 + row_[k] - 1) * U.sQ + pp_[k];
                cx[k] = __ldg(chi + off);
                cs[k] = __ldg(Sg + off);
            }
        }
#pragma unroll
        for (int k = 0; k < HPT; ++k) {
            const int h = tid + k * NT;
            if (h < nh) {
                const int side = h >= NP, p = h - side * NP;
                const int q = side ? qhi : qlo;
                const bool ok = side ? hi_ok : lo_ok;
                const long long off = mo + (long long)q * U.sQ + p;
                hx[k] = ok ? __ldg(chi + off) : T(0);
                hs[k] = ok ? __ldg(Sg + off) : T(0);
            }
        }
    };
    load_plane(t_first);

    int t_acc = U.wrap ? -1 : 0;
    const int warm_cap = a.max_periods * NM;
    T *part = (T *)U.partial;

    for (int t = t_first;; ++t) {
        const int m = plane_of(t, NM, U.sa);
        const bool acc_now = s_ctl[1] != 0;
        // ---- (1) periodic-wrap decision for this step, (2) halo of plane t-1 ----
        const bool need_decision = !acc_now && t - a.L >= 0;
        if (warp == 1 && need_decision) {
            const int ts = t - a.L;
            float gm = 0.f;
            bool ok = true;
            for (int i = lane; i < ntl; i += 32) {
                const unsigned long long *slot = a.gsync + (long long)(U.tile0 + i) * a.R + (ts % a.R);
                unsigned long long v = ld_acquire64(slot);
                if ((unsigned)(v >> 32) != (unsigned)(ts + 1)) {
                    const uint64_t t0 = global_ns();
                    for (;;) {
                        __nanosleep(64);
                        v = ld_acquire64(slot);
                        if ((unsigned)(v >> 32) == (unsigned)(ts + 1)) break;
                        if (ld_relaxed(a.status) != 0) { ok = false; break; }
                        if (global_ns() - t0 > a.timeout_ns) { atomicOr(a.status, ST_TIMEOUT); ok = false; break; }
                    }
                }
                if (!ok) break;
                gm = fmaxf(gm, __uint_as_float((unsigned)(v & 0xffffffffu)));
            }
            for (int o = 16; o; o >>= 1) {
                gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
                ok = __all_sync(0xffffffffu, ok);
            }
            if (lane == 0) {
                if (!ok) s_ctl[0] = 1;
                else s_ctl[2] = gm <= a.tol ? 1 : 0;
            }
        }
        if (tid == 0 && t > t_first) {
            bool ok = true;
            if (has_lower) ok = wait_flag_geq(a.flags + U.tile0 + lower, t, a.status, a.timeout_ns);
            if (ok && has_upper) ok = wait_flag_geq(a.flags + U.tile0 + upper, t, a.status, a.timeout_ns);
            if (!ok) s_ctl[0] = 1;
        }
        __syncthreads();
        if (s_ctl[0]) return;
        if (need_decision && s_ctl[2]) {
            if (tid == 0) s_ctl[1] = 1;
            t_acc = t;
            if (r == 0 && tid == 0) a.unit_tacc[uidx] = t;
        }
        if (!U.wrap || (t_acc >= 0)) {
            // accumulate this step
        } else if (t >= warm_cap) {
            if (tid == 0) atomicOr(a.status, ST_NOCONV);
            return;  // every tile of the unit stops at the same step
        }
        const bool acc = t_acc >= 0;
        if (t > t_first) {
            // neighbours' edge rows of plane t-1 -> halo rows 0 and nrows+1
            const int slot = (t - 1) & 1;
            const int nch = acc ? nd : 2 * nd;
            for (int h = tid; h < 2 * nch * NP; h += NT) {
                const int side = h / (nch * NP);
                const int rem = h - side * nch * NP;
                const int ch = rem / NP, p = rem - ch * NP;
                const int nb = side == 0 ? lower : upper;
                if (side == 0 ? !has_lower : !has_upper) continue;
                const T *src = a.halo + U.halo_off + (long long)nb * (8 * MAXD * NP) +
                               ((long long)(slot * 2 + (side == 0 ? 1 : 0)) * (2 * MAXD) + (ch < nd ? ch : MAXD + ch - nd)) * NP + p;
                const T v = ld_cg(src);
                const int row = side == 0 ? 0 : nrows + 1;
                if (ch < nd) sI[(ch * RW + row) * NP + p] = v;
                else sG[((ch - nd) * RW + row) * NP + p] = (float)v;
            }
            __syncthreads();
        }

        // ---- (3) integrate the own points of plane t ----
        T nI[PPT][MAXD];
        float nG[PPT][MAXD];
        float gmax = 0.f;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int l = tid + k * NT;
            if (l >= npts) continue;
            const int p = pp_[k], row = row_[k], q = q0 + row - 1;
            const T xp = cx[k], sp = cs[k];
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                if (d >= nd) break;
                const bool bcrow = U.wrap && ((D.up[d] && q == 0) || (!D.up[d] && q == NQ - 1));
                if (bcrow) {
                    nI[k][d] = bc_value(a, U, D, d, p, q, m, sp);
                    nG[k][d] = 0.f;
                    continue;
                }
                const int pc = D.sP[d] > 0 ? pm_[k] : pn_[k];
                const int rc = row - D.sQ[d];
                const int i0 = row * NP + p, i1 = row * NP + pc, i2 = rc * NP + p, i3 = rc * NP + pc;
                const T b0 = D.beta[d][0], b1 = D.beta[d][1], b2 = D.beta[d][2], b3 = D.beta[d][3];
                const T *Id = sI + d * RW * NP;
                const T Iup = b0 * Id[i0] + b1 * Id[i1] + b2 * Id[i2] + b3 * Id[i3];
                const T xup = b0 * sX[i0] + b1 * sX[i1] + b2 * sX[i2] + b3 * sX[i3];
                const T sup = b0 * sS[i0] + b1 * sS[i1] + b2 * sS[i2] + b3 * sS[i3];
                const T x = D.hds[d] * (xup + xp);
                T e, wu, wp;
                seg_weights(x, e, wu, wp);
                nI[k][d] = Iup + wu * (sup - Iup) + wp * (sp - Iup);
                if (!acc) {
                    const float *Gd = sG + d * RW * NP;
                    const float g = (float)e * ((float)b0 * Gd[i0] + (float)b1 * Gd[i1] + (float)b2 * Gd[i2] + (float)b3 * Gd[i3]);
                    nG[k][d] = g;
                    gmax = fmaxf(gmax, g);
                }
            }
        }
        if (!acc) {
            for (int o = 16; o; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
            if (lane == 0) s_wmax[warp] = gmax;
        }
        __syncthreads();

        // ---- (4) plane t becomes the previous plane; publish edge rows ----
        const int slot = t & 1;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int l = tid + k * NT;
            if (l >= npts) continue;
            const int p = pp_[k], row = row_[k], q = q0 + row - 1;
            const int i0 = row * NP + p;
            sX[i0] = cx[k];
            sS[i0] = cs[k];
            T aJ = 0, aX = 0, aY = 0, aZ = 0;
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                if (d >= nd) break;
                const T v = nI[k][d];
                sI[d * RW * NP + i0] = v;
                if (!acc) sG[d * RW * NP + i0] = nG[k][d];
                aJ += D.cJ[d] * v; aX += D.cF[0][d] * v; aY += D.cF[1][d] * v; aZ += D.cF[2][d] * v;
            }
            // edge rows to the neighbours
            const int side = (row == 1) ? 0 : ((row == nrows) ? 1 : -1);
            if (side >= 0 || (nrows == 1)) {
                for (int sd = 0; sd < 2; ++sd) {
                    if (!(nrows == 1 || sd == side)) continue;
                    T *dst = myhalo + ((long long)(slot * 2 + sd) * (2 * MAXD)) * NP + p;
                    for (int d = 0; d < nd; ++d) {
                        dst[(long long)d * NP] = nI[k][d];
                        if (!acc) dst[(long long)(MAXD + d) * NP] = (T)nG[k][d];
                    }
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
        // halo rows of chi/S for plane t
#pragma unroll
        for (int k = 0; k < HPT; ++k) {
            const int h = tid + k * NT;
            if (h < nh) {
                const int side = h >= NP, p = h - side * NP;
                const int row = side ? nrows + 1 : 0;
                sX[row * NP + p] = hx[k];
                sS[row * NP + p] = hs[k];
            }
        }
        const bool last = acc && (t - t_acc == NM - 1);
        if (!last) load_plane(t + 1);
        __syncthreads();
        if (tid == 0) {
            if (!acc) {
                float g = 0.f;
                for (int w = 0; w < NT / 32; ++w) g = fmaxf(g, s_wmax[w]);
                const unsigned long long v = ((unsigned long long)(unsigned)(t + 1) << 32) | __float_as_uint(g);
                __threadfence();
                st_release64(a.gsync + (long long)gt * a.R + (t % a.R), v);
            }
            __threadfence();
            st_release(a.flags + gt, t + 1);
        }
        if (last) break;
    }
}

template <typename T, int PPT>
__global__ void __launch_bounds__(SWEEP_NT) sweep_kernel(SweepArgs<T> a)
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
        run_tile<T, PPT>(a, U, u, tile - U.tile0, tile, smem);
    }
}

}  // namespace rts

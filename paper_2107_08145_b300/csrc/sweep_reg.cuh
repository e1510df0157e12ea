// sweep_reg.cuh -- FP32 forward sweep with the tile's intensities in
// registers (the paper's integrate(), Sect. 5.1, one persistent launch for
// all bands and direction groups like sweep.cuh, laid out for fewer
// instructions per update).
//
// What differs from sweep_kernel (sweep.cuh), which it replaces for the FP32
// forward solve when a unit's rays share one bilinear stencil:
//  * Thread c owns columns c and c + P/2 of the tile's TQ rows and keeps
//    their intensities (4 sign slots) and, during the periodic warm-up, their
//    seed-error bounds in registers. Every value of the two columns is a
//    float2, so the segment arithmetic runs on Blackwell's packed FP32
//    instructions (two columns per FFMA2).
//  * A column pair's P neighbours are the adjacent threads' pairs, passed by
//    warp shuffles; a warp's first and last lanes take theirs from small
//    per-warp records in shared memory (every lane loads the record and the
//    edge lanes select it, so no branch diverges); c = 0 and c = P/2 - 1 take
//    the periodic neighbour pair swapped.
//  * chi and S of the next plane are copied into a triple-buffered shared
//    tile with cp.async while the current plane is computed; a record holds
//    {chi(c), chi(c+P/2), S(c), S(c+P/2)}, so a column pair's neighbourhood
//    is three 16-byte loads per row.
//  * One CTA barrier per plane. The rows the neighbour tiles need are
//    computed first and written to a global ring; after the barrier one
//    thread releases them with a counter add per neighbour. The rows that
//    need the neighbours come last, after one bounded acquire wait; every
//    lane reads its own and its adjacent pairs of the neighbours' rows.
//  * The kernel stores the four slot intensities of every point (raw, one
//    16-byte store per point); the per-band reduction forms J and F from them
//    (with exact differences for the cancelling flux components).
//
// Requirements (checked on the host): FP32, every active slot of a unit has
// the same path length and bilinear weights (true for every 3-rays-per-octant
// set), the plane extent P is even, and the tile height divides the extent of
// the periodic z-group rows.
#pragma once
#include "df32.cuh"
#include "sweep.cuh"

namespace rts {

// q(x) = (1 - e^-x)/x below x = 1/4: the degree-4 polynomial interpolating q
// at the Chebyshev nodes of [0, 1/4] (the same literals as seg_eq), evaluated
// in y = -x log2(e), the argument the kernel keeps
constexpr double kQPolyX[5] = {0.99999999758, -0.49999951482, 0.16665108207, -0.04149065410, 0.00751360622};
constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLog2e = 1.44269504088896340736;
constexpr float kQPolyY[5] = {(float)kQPolyX[0], (float)(kQPolyX[1] * -kLn2), (float)(kQPolyX[2] * kLn2 * kLn2),
                              (float)(kQPolyX[3] * -kLn2 * kLn2 * kLn2),
                              (float)(kQPolyX[4] * kLn2 * kLn2 * kLn2 * kLn2)};
constexpr float kYSwitch = (float)(-0.25 * kLog2e);  // x < 1/4  <=>  y > kYSwitch

__device__ __forceinline__ float2 max2(float2 a, float2 b) { return f2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
// hardware approximations (PTX ex2.approx / rcp.approx)
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src)
{
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(gmem_src) : "memory");
}

template <int M>
using Mode = std::integral_constant<int, M>;

// Constants of a unit's stencil, packed for both columns.
struct RegStencil {
    float2 b0, b1, b2, b3;  // bilinear weights of corners (0,0), (-sP,0), (0,-sQ), (-sP,-sQ)
    float2 hdn;             // -(ds/2) log2(e): y = hdn (chi_up + chi_p) = -dtau log2(e)
};

// dw_p/dx = (q - e)/x below x = 1/4: the degree-4 polynomial interpolating
// it at the Chebyshev nodes of [0, 1/4] (the same literals as seg_dwp),
// evaluated in y = -x log2(e) and negated, as the checkpoint uses it
constexpr double kDwpX[5] = {0.49999999793, -0.33333291823, 0.12498666530, -0.03318270431, 0.00624265650};
constexpr float kNDwpY[5] = {(float)-kDwpX[0], (float)(-kDwpX[1] * -kLn2), (float)(-kDwpX[2] * kLn2 * kLn2),
                             (float)(-kDwpX[3] * -kLn2 * kLn2 * kLn2),
                             (float)(-kDwpX[4] * kLn2 * kLn2 * kLn2 * kLn2)};

// One segment for two columns: the upwind intensity, opacity and source
// interpolated with the shared weights, dtau, e = exp(-dtau) and
// q = (1 - e)/dtau, and the new intensity
//   I = S_p + e (I_up - S_up) + q (S_up - S_p)
// (the linear-in-tau formal solution, same form as seg_eq). Returns I; e
// goes to the seed-error bound. WD (the adjoint's checkpoint): also the
// segment's derivative D = dI/d(dtau) = e (S_up - I_up) + dw_p (S_p - S_up),
// with dw_p = (q - e)/dtau the derivative of the own-point weight 1 - q.
template <bool WD = false>
__device__ __forceinline__ float2 seg2(const RegStencil &K, float2 i0, float2 i1, float2 i2, float2 i3, float2 x0,
                                       float2 x1, float2 x2, float2 x3, float2 s0, float2 s1, float2 s2, float2 s3,
                                       float2 xp, float2 sp, float2 &e, float2 *D = nullptr)
{
    const float2 iup = fma2(K.b3, i3, fma2(K.b2, i2, fma2(K.b1, i1, mul2(K.b0, i0))));
    const float2 xup = fma2(K.b3, x3, fma2(K.b2, x2, fma2(K.b1, x1, mul2(K.b0, x0))));
    const float2 sup = fma2(K.b3, s3, fma2(K.b2, s2, fma2(K.b1, s1, mul2(K.b0, s0))));
    const float2 y = mul2(K.hdn, add2(xup, xp));
    e = f2(ex2_approx(y.x), ex2_approx(y.y));
    if constexpr (!WD) {
        // (1 - e)/x = (e - 1) log2(e) / y
        const float2 qd = mul2(fma2(f2((float)kLog2e), e, f2(-(float)kLog2e)), f2(rcp_approx(y.x), rcp_approx(y.y)));
        const float2 qs = fma2(fma2(fma2(fma2(f2(kQPolyY[4]), y, f2(kQPolyY[3])), y, f2(kQPolyY[2])), y,
                                    f2(kQPolyY[1])),
                               y, f2(kQPolyY[0]));
        const float2 q = f2(y.x > kYSwitch ? qs.x : qd.x, y.y > kYSwitch ? qs.y : qd.y);
        return fma2(q, sub2(sup, sp), fma2(e, sub2(iup, sup), sp));
    } else {
        const float2 ry = f2(rcp_approx(y.x), rcp_approx(y.y));
        const float2 qd = mul2(fma2(f2((float)kLog2e), e, f2(-(float)kLog2e)), ry);
        const float2 qs = fma2(fma2(fma2(fma2(f2(kQPolyY[4]), y, f2(kQPolyY[3])), y, f2(kQPolyY[2])), y,
                                    f2(kQPolyY[1])),
                               y, f2(kQPolyY[0]));
        const bool smx = y.x > kYSwitch, smy = y.y > kYSwitch;
        const float2 q = f2(smx ? qs.x : qd.x, smy ? qs.y : qd.y);
        const float2 bv = sub2(sup, sp);
        // dw_p: (q - e)/x = (e - q) log2(e) / y above x = 1/4, else the polynomial
        const float2 dd = mul2(mul2(sub2(e, q), f2((float)kLog2e)), ry);
        const float2 ds = fma2(
            fma2(fma2(fma2(f2(kNDwpY[4]), y, f2(kNDwpY[3])), y, f2(kNDwpY[2])), y, f2(kNDwpY[1])), y, f2(kNDwpY[0]));
        const float2 ndwp = f2(smx ? ds.x : -dd.x, smy ? ds.y : -dd.y);
        *D = fma2(ndwp, bv, mul2(e, sub2(sup, iup)));
        return fma2(q, bv, fma2(e, sub2(iup, sup), sp));
    }
}

// bound of the remaining seed error: g = e * sum_c beta_c g(corner c)
__device__ __forceinline__ float2 bound2(const RegStencil &K, float2 g0, float2 g1, float2 g2, float2 g3, float2 e)
{
    return mul2(e, fma2(K.b3, g3, fma2(K.b2, g2, fma2(K.b1, g1, mul2(K.b0, g0)))));
}

// smem bytes of a tile: chi/S records [3][TQ+2][NP/2+2] x 16 B and the
// per-warp edge-column records [2][warps][2][TQ][3] x 16 B
__host__ __device__ constexpr size_t reg_tile_smem_bytes(int tq, int np)
{
    return (size_t)3 * (tq + 2) * (np / 2 + 2) * 16 + (size_t)2 * ((np / 2 + 31) / 32) * 2 * tq * 3 * 16;
}

// ring of one tile: [4 slots][6 channels][NP/2 pairs][2], in floats
__host__ __device__ constexpr long long reg_ring_elems(int np) { return 24LL * np; }

// boundary intensity of a set point (kind as rts_bc_kind), natural (i, j)
__device__ __forceinline__ float reg_bc(int kind, const float *arr, int udx, int nx, int ny, int i, int j, float sp)
{
    if (kind == 0) return 0.f;
    if (kind == 1) return sp;
    return arr[((long long)udx * ny + j) * nx + i];
}

// SEED: the instantiation for warm-started solves (rts_boundary.wrap_seed
// with seed_in); the plain one carries none of that code. CK: the adjoint's
// checkpoint sweep, which also stores every accumulated segment's
// D = dI/d(dtau) (0 at set points and in empty slots) at
// a.store + (unit - a.unit_base) * 4 N + 4 off + slot, off the point's offset
// in the unit's layout (the layout the reverse sweep reads).
template <int TQ, bool SEED, bool CK>
__device__ void run_tile_reg(const SweepArgs<float> &a, const SweepUnit *__restrict__ Ug, int uidx, int r, int gt,
                             unsigned char *smem)
{
    static_assert(TQ >= 2, "the rows published to the neighbours must not depend on them");
    constexpr int RWS = TQ + 2;  // rows of a plane in shared memory (halo, TQ own, halo)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NT = blockDim.x;
    const int NP = Ug->NP, NQ = Ug->NQ, NM = Ug->NM;
    const int axis = Ug->axis, sa = Ug->sa, ntl = Ug->ntiles, tile0 = Ug->tile0;
    const bool wrap = Ug->wrap != 0, qper = Ug->qper != 0;
    const int unx = Ug->nx, uny = Ug->ny;
    const long long sQ = Ug->sQ, sM = Ug->sM;
    const float *__restrict__ chi = (Ug->transposed ? a.chiT : a.chi) + Ug->in_off;
    const float *__restrict__ Sg = (Ug->transposed ? a.ST : a.S) + Ug->in_off;
    float *const itop = a.itop ? a.itop + Ug->top_off : nullptr;
    float *const part = (float *)Ug->partial;
    // the adjoint's checkpoint of this unit (CK only)
    float *const ckb = CK ? a.store + (long long)(uidx - a.unit_base) * MAXD * Ug->N : nullptr;
    // thread c owns columns c (.x of every pair) and c + H (.y)
    const int H = NP >> 1;
    const int RR = H + 2;                        // records per shared row: record c + 1 holds pair c
    const long long tstride = reg_ring_elems(NP);
    float *const halo_base = a.halo + Ug->halo_off;
    float *const myhalo = halo_base + (long long)r * tstride;

    const int q0 = r * TQ;
    const int nrows = min(TQ, NQ - q0);          // rows beyond are padding (x/y groups only)
    const bool act = tid < H;
    const int c = act ? tid : H - 1;             // column pair read (clamped for idle lanes)
    const int lastw = (H - 1) >> 5;
    const int Lw = warp < lastw ? 31 : ((H - 1) & 31);
    // warps past the last column pair (a unit narrower than the CTA) only
    // take part in the barriers and shuffles: no edge-column role
    const bool wact = warp <= lastw;
    const bool isF = wact && lane == 0, isL = wact && lane == Lw;
    const int NW = lastw + 1;
    const int wprev = warp == 0 ? lastw : warp - 1, wnext = warp == lastw ? 0 : warp + 1;
    // the pair left of c = 0 is (NP-1, H-1), that of H-1's right (H, 0): the
    // neighbouring thread's pair with its halves swapped
    const bool swapL = c == 0, swapR = c == H - 1;

    float4 *const XS = (float4 *)smem;                                        // [3][RWS][RR]
    float4 *const EDG = XS + 3 * RWS * RR;                                    // [2][NW][2][TQ][3]
    auto edg = [&](int slot, int w, int side, int k) -> float4 * {            // k = 1..TQ
        return EDG + ((((slot * NW + w) * 2 + side) * TQ) + (k - 1)) * 3;
    };

    __shared__ float s_wmax[32], s_imax[32], s_dmax[32];
    __shared__ float s_glog[SEED ? 1024 : 1];    // warm start: the unit's bound of every plane of period 0
    __shared__ int s_ctl[4];                     // 0 abort, 1 wrap decision for the next plane, 2 warm start: last plane
    __shared__ int s_q[RWS];                     // grid row of shared row k, -1 outside

    // unit constants (every active slot has the same stencil)
    int s_first = 0;
    while (s_first < MAXD - 1 && !Ug->active[s_first]) ++s_first;
    RegStencil K;
    K.b0 = f2((float)Ug->beta[s_first][0]);
    K.b1 = f2((float)Ug->beta[s_first][1]);
    K.b2 = f2((float)Ug->beta[s_first][2]);
    K.b3 = f2((float)Ug->beta[s_first][3]);
    K.hdn = f2((float)(-0.5 * Ug->ds[s_first] * kLog2e));
    int actm = 0, upm = 0;
    for (int d = 0; d < MAXD; ++d) {
        actm |= Ug->active[d] ? 1 << d : 0;
        upm |= Ug->up[d] ? 1 << d : 0;
    }
    const int kind_up = a.bc_bottom, kind_dn = a.bc_top;

    if (tid < RWS) {
        int q = q0 - 1 + tid;
        if (qper) q = (q % NQ + NQ) % NQ;
        else if (q < 0 || q >= NQ) q = -1;
        s_q[tid] = q;
    }
    if (tid == 0) { s_ctl[0] = 0; s_ctl[1] = 0; s_ctl[2] = INT_MAX; }
    __syncthreads();

    const int t_first = wrap ? 0 : 1;
    const int tp = t_first - 1;
    const int lower = qper ? (r + ntl - 1) % ntl : r - 1;
    const int upper = qper ? (r + 1) % ntl : r + 1;
    const bool has_lower = qper || r > 0;
    const bool has_upper = qper || r < ntl - 1;
    // the last grid row (q = NQ - 1) of an x/y group: shared row kb of this tile, else 0
    const int kb = (wrap && q0 + nrows == NQ) ? nrows : 0;
    // warm start (x/y groups): the unit's wrap plane in the caller's buffer
    float *const sbuf = (wrap && a.seed) ? a.seed + Ug->seed_off : nullptr;
    const bool seeded = SEED && sbuf != nullptr && a.seed_in != 0;
    const int m_seed = plane_of(-1, NM, sa);

    // chi and S of plane t into shared slot `slot`: record c + 1 of row k holds
    // {chi(c), chi(c+H), S(c), S(c+H)}; record 0 is pair H-1 swapped and record
    // H+1 pair 0 swapped (the periodic neighbours of the first and last pair)
    const bool padR = act && tid == 0, padL = act && tid == H - 1;
    // the plane after plane mm in sweep order (periodic)
    auto next_m = [&](int mm) { return sa > 0 ? (mm + 1 == NM ? 0 : mm + 1) : (mm == 0 ? NM - 1 : mm - 1); };
    // (offsets within a band's array: below 2^31 points, checked on the host)
    const int sQi = (int)sQ, sMi = (int)sM;
    auto prefetch = [&](int mpl, int slot) {
        if (act) {
            const int mo = mpl * sMi + c;
            float4 *row0 = XS + slot * RWS * RR;
#pragma unroll
            for (int k = 0; k < RWS; ++k) {
                const int q = s_q[k];
                float *dst = reinterpret_cast<float *>(row0 + k * RR + c + 1);
                if (q >= 0) {
                    const int off = mo + q * sQi;
                    const float *gx = chi + off, *gs = Sg + off;
                    cp_async(dst, gx);
                    cp_async(dst + 1, gx + H);
                    cp_async(dst + 2, gs);
                    cp_async(dst + 3, gs + H);
                    if (padR) {
                        float *d2 = reinterpret_cast<float *>(row0 + k * RR + H + 1);
                        cp_async(d2, gx + H); cp_async(d2 + 1, gx); cp_async(d2 + 2, gs + H); cp_async(d2 + 3, gs);
                    }
                    if (padL) {
                        float *d2 = reinterpret_cast<float *>(row0 + k * RR);
                        cp_async(d2, gx + H); cp_async(d2 + 1, gx); cp_async(d2 + 2, gs + H); cp_async(d2 + 3, gs);
                    }
                } else {
                    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                    *reinterpret_cast<float4 *>(dst) = z;
                    if (padR) row0[k * RR + H + 1] = z;
                    if (padL) row0[k * RR] = z;
                }
            }
        }
        cp_async_commit();
    };

    // intensities {I(c), I(c+H)} of the previous plane per shared row and slot,
    // and seed-error bounds [row][0 = rising slots 0,1 / 1 = descending 2,3]
    float2 Ip[RWS][MAXD], Gp[RWS][2];
#pragma unroll
    for (int k = 0; k < RWS; ++k) {
#pragma unroll
        for (int d = 0; d < MAXD; ++d) Ip[k][d] = f2(0.f);
        Gp[k][0] = Gp[k][1] = f2(0.f);
    }

    // What a neighbour tile needs of plane t: the lower one the descending
    // slots (2, 3) of this tile's first row, the upper one the rising slots
    // (0, 1) of its last row, with their bounds. Those depend only on this
    // tile's own rows of plane t-1 (a descending ray at row 1 reads rows 1 and
    // 2, a rising ray at row TQ rows TQ-1 and TQ), so they are computed and
    // written first in every plane, before this tile waits for anything.
    // Ring [slot t & 3][channel][pair c] (four slots: a tile can be two planes
    // ahead of a neighbour still reading); after the plane's barrier one
    // counter add per neighbour releases them, and a neighbour needs plane t
    // only at the end of its plane t+1.
    auto ring_at = [&](const float *tile, int slot, int ch) -> const float2 * {
        return reinterpret_cast<const float2 *>(tile + (long long)slot * 6 * NP + (long long)ch * NP);
    };
    auto publish_ring = [&](int t, float2 d2, float2 d3, float2 gd, float2 r0, float2 r1, float2 gu) {
        if (!wact) return;
        if (act) {
            float2 *h = reinterpret_cast<float2 *>(myhalo + (long long)(t & 3) * 6 * NP) + c;
            h[0 * H] = d2;  // side 0: first row, descending slots
            h[1 * H] = d3;
            h[2 * H] = gd;
            h[3 * H] = r0;  // side 1: last row, rising slots
            h[4 * H] = r1;
            h[5 * H] = gu;
        }
    };
    // one release per tile and plane, after the CTA barrier: every warp's ring
    // writes of the plane happen before it (the barrier orders them, the
    // release makes them visible with the count), so only one thread pays the
    // fence
    auto release_plane = [&]() {
        if (tid == 0) {
            if (has_upper) red_release_add((unsigned *)(a.flags + 2 * (tile0 + upper)), 1u);
            if (has_lower) red_release_add((unsigned *)(a.flags + 2 * (tile0 + lower) + 1), 1u);
        }
    };
    // the warp's first and last thread's pairs of the own rows of plane t
    // (shared slot t & 1): {I0, I2}, {I1, I3}, {gu, gd} pairs
    auto publish_edges = [&](int t) {
        if (isF || isL) {
            float4 *const eo = edg(t & 1, warp, 0, 1);  // this warp's records of plane t (side 1 follows side 0)
#pragma unroll
            for (int k = 1; k <= TQ; ++k) {
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    if (side == 0 ? !isF : !isL) continue;
                    float4 *e = eo + (side * TQ + (k - 1)) * 3;
                    e[0] = make_float4(Ip[k][0].x, Ip[k][0].y, Ip[k][2].x, Ip[k][2].y);
                    e[1] = make_float4(Ip[k][1].x, Ip[k][1].y, Ip[k][3].x, Ip[k][3].y);
                    e[2] = make_float4(Gp[k][0].x, Gp[k][0].y, Gp[k][1].x, Gp[k][1].y);
                }
            }
        }
    };
    // checkpoint: D of slots 2h, 2h+1 of own row k of plane m ({D(2h),
    // D(2h+1)} of column c in lo, of column c + H in hi)
    auto store_ck = [&](int m, int k, int h, float2 lo, float2 hi) {
        if constexpr (CK) {
            if (!act || k > nrows) return;
            float4 *pp = reinterpret_cast<float4 *>(ckb) + (m * sMi + (q0 + k - 1) * sQi + c);
            reinterpret_cast<float2 *>(pp)[h] = lo;
            reinterpret_cast<float2 *>(pp + H)[h] = hi;
        }
    };
    // raw slot intensities and I_top of the own rows of an accumulated plane m
    // (held in Ip)
    auto store_rows = [&](int m) {
        if (!act) return;
#pragma unroll
        for (int k = 1; k <= TQ; ++k) {
            if (k > nrows) break;
            float4 *pp = reinterpret_cast<float4 *>(part) + (m * sMi + (q0 + k - 1) * sQi + c);
            pp[0] = make_float4(Ip[k][0].x, Ip[k][1].x, Ip[k][2].x, Ip[k][3].x);
            pp[H] = make_float4(Ip[k][0].y, Ip[k][1].y, Ip[k][2].y, Ip[k][3].y);
        }
        if (!itop) return;
        if (axis == 2 && sa > 0 && m == NM - 1) {  // top plane of a rising z group
#pragma unroll
            for (int k = 1; k <= TQ; ++k) {
                float *row = itop + (long long)(q0 + k - 1) * unx;
#pragma unroll
                for (int d = 0; d < MAXD; ++d) {
                    if (!((actm >> d) & 1)) continue;
                    const float2 v = Ip[k][d];
                    float *b = row + (long long)Ug->udx[d] * uny * unx;
                    b[c] = v.x;
                    b[c + H] = v.y;
                }
            }
        } else if (axis != 2 && kb > 0) {  // top row of an x/y group, rising slots 0, 1
#pragma unroll
            for (int k = 1; k <= TQ; ++k) {
                if (k != kb) continue;
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    if (!((actm >> d) & 1)) continue;
                    const float2 v = Ip[k][d];
                    float *b = itop + (long long)Ug->udx[d] * uny * unx;
                    if (axis == 1) {  // natural (i, j) = (p, m)
                        b[(long long)m * unx + c] = v.x;
                        b[(long long)m * unx + c + H] = v.y;
                    } else {          // natural (i, j) = (m, p)
                        b[(long long)c * unx + m] = v.x;
                        b[(long long)(c + H) * unx + m] = v.y;
                    }
                }
            }
        }
    };

    // ---------------- prologue: plane tp = t_first - 1 (seed or boundary plane) ----
    int s_prev = (tp + 3) % 3, s_cur = (t_first + 3) % 3, s_next = (t_first + 4) % 3;
    prefetch(plane_of(tp, NM, sa), s_prev);
    prefetch(plane_of(t_first, NM, sa), s_cur);
    cp_async_wait_all();
    __syncthreads();
    {
        const int m = plane_of(tp, NM, sa);
        const float4 *row0 = XS + s_prev * RWS * RR;
#pragma unroll
        for (int k = 1; k <= TQ; ++k) {
            const int q = s_q[k];
            const float4 xs = row0[k * RR + c + 1];
            const float sv[2] = {xs.z, xs.w};
            float v[MAXD][2], g[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                const bool up = (upm >> d) & 1;
                for (int hh = 0; hh < 2; ++hh) {
                    float val = 0.f;
                    if (q >= 0 && ((actm >> d) & 1)) {
                        // x/y groups: set only on the bottom (rising) / top (descending)
                        // boundary rows; z groups: the whole plane is the boundary layer
                        const bool set = wrap ? (up ? q == 0 : q == NQ - 1) : true;
                        if (set) {
                            int i, j;
                            natural_ij(axis, c + hh * H, q, m, i, j);
                            val = reg_bc(up ? kind_up : kind_dn, up ? a.bc_up + Ug->top_off : a.bc_dn + Ug->dn_off,
                                         Ug->udx[d], unx, uny, i, j, sv[hh]);
                        } else {  // seed of the periodic wrap: I = S or the caller's warm start; unit bound
                            val = seeded ? sbuf[((long long)q * NP + c + hh * H) * 4 + d] : sv[hh];
                            g[d >> 1][hh] = 1.f;
                        }
                    }
                    v[d][hh] = val;
                }
                Ip[k][d] = f2(v[d][0], v[d][1]);
            }
            Gp[k][0] = f2(g[0][0], g[0][1]);
            Gp[k][1] = f2(g[1][0], g[1][1]);
        }
        publish_ring(tp, Ip[1][2], Ip[1][3], Gp[1][1], Ip[TQ][0], Ip[TQ][1], Gp[TQ][0]);
        publish_edges(tp);
        if (!wrap) {  // z groups: the boundary plane is the first accumulated plane
            store_rows(m);
            if constexpr (CK) {  // set points: D = 0
#pragma unroll
                for (int k = 1; k <= TQ; ++k) {
                    store_ck(m, k, 0, f2(0.f), f2(0.f));
                    store_ck(m, k, 1, f2(0.f), f2(0.f));
                }
            }
        }
    }
    __syncthreads();
    release_plane();

    // z groups: the boundary plane tp is the first accumulated plane
    int t_acc = (wrap && !seeded) ? -1 : 0;
    const int warm_cap = a.max_periods * NM + a.L;
    const int dec_thread = NT > 32 ? 32 : 0;

    auto shfl_up2 = [](float2 v) {
        return f2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
    };
    auto shfl_dn2 = [](float2 v) {
        return f2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
    };
    auto swp = [](float2 v) { return f2(v.y, v.x); };

    // One plane t. ACC: accumulated (outputs written, no bounds). Returns 0 to
    // go on, 1 after the last plane, 2 to abandon the tile (a wait failed).
    //
    // The rising slots (0, 1) of row k read rows k and k-1 of the previous
    // plane, the descending slots (2, 3) rows k and k+1, and the two sets never
    // mix. So each set is updated in place: the rising rows from the top row
    // down (row k's old values are last read by row k+1, done before), the
    // descending rows from the first row up. The rows a neighbour tile needs
    // (rising TQ, descending 1) come first and are published at once; the rows
    // that need a neighbour (rising 1, descending TQ) come last.
    auto plane_step = [&](auto ACCF, int t, int m) __attribute__((always_inline)) -> int {
        // 0: warm-up (bounds), 1: accumulated, 2: accumulated with bounds (the first
        // period of a warm-started x/y group)
        constexpr int MD = decltype(ACCF)::value;
        constexpr bool ACC = MD != 0;
        constexpr bool BND = MD != 1;
        const bool last = ACC && !seeded && (t - t_acc == NM - 1);
        const int es = (t - 1) & 1;  // shared edge records of the previous plane
        // (warps past the last column pair read warp 0's records: in bounds, and discarded)
        const float4 *const eprev = edg(es, wact ? wprev : 0, 1, 1), *const enext = edg(es, wact ? wnext : 0, 0, 1);

        const float4 *XP = XS + s_prev * RWS * RR + c + 1;   // previous plane, own record
        const float4 *XC = XS + s_cur * RWS * RR + c + 1;    // current plane

        // chi/S pairs of a previous-plane row: own {c, c+H}, left {c-1, c-1+H}, right
        struct XRow {
            float2 x0, xl, xr, s0, sl, sr;
        };
        auto xs_row = [&](int j) -> XRow {
            const float4 m_ = XP[j * RR - 1], c_ = XP[j * RR], p_ = XP[j * RR + 1];
            return XRow{f2(c_.x, c_.y), f2(m_.x, m_.y), f2(p_.x, p_.y), f2(c_.z, c_.w), f2(m_.z, m_.w), f2(p_.z, p_.w)};
        };
        // neighbour pairs of an own row of the previous plane for one slot set:
        // the left pair of the sP = +1 slot, the right pair of the sP = -1 slot
        // and the same for the set's bound
        struct NRow {
            float2 il, ir, gl, gr;
        };
        auto nb_row = [&](int k, auto HF) __attribute__((always_inline)) -> NRow {
            constexpr int h = decltype(HF)::value;  // 0: rising slots 0, 1; 1: descending 2, 3
            NRow n;
            n.il = shfl_up2(Ip[k][2 * h]);
            n.ir = shfl_dn2(Ip[k][2 * h + 1]);
            if constexpr (BND) {
                n.gl = shfl_up2(Gp[k][h]);
                n.gr = shfl_dn2(Gp[k][h]);
            }
            // the warp-edge lanes take their outer neighbour from the records of
            // the adjacent warps: every lane loads them (one broadcast load per
            // record) and selects, so the warp does not diverge
            {  // the previous warp's last thread (for c = 0: the last pair, swapped)
                const float4 *e = eprev + (k - 1) * 3;
                const float4 iv = e[0];
                float2 v = h ? f2(iv.z, iv.w) : f2(iv.x, iv.y);
                v = swapL ? swp(v) : v;
                n.il = f2(isF ? v.x : n.il.x, isF ? v.y : n.il.y);
                if constexpr (BND) {
                    const float4 gg = e[2];
                    float2 g = h ? f2(gg.z, gg.w) : f2(gg.x, gg.y);
                    g = swapL ? swp(g) : g;
                    n.gl = f2(isF ? g.x : n.gl.x, isF ? g.y : n.gl.y);
                }
            }
            {  // the next warp's first thread (for c = H-1: pair 0, swapped)
                const float4 *e = enext + (k - 1) * 3;
                const float4 iv = e[1];
                float2 v = h ? f2(iv.z, iv.w) : f2(iv.x, iv.y);
                v = swapR ? swp(v) : v;
                n.ir = f2(isL ? v.x : n.ir.x, isL ? v.y : n.ir.y);
                if constexpr (BND) {
                    const float4 gg = e[2];
                    float2 g = h ? f2(gg.z, gg.w) : f2(gg.x, gg.y);
                    g = swapR ? swp(g) : g;
                    n.gr = f2(isL ? g.x : n.gr.x, isL ? g.y : n.gr.y);
                }
            }
            return n;
        };
        // slot set h of row k from row k (A, NA) and row k2 = k -+ 1 (B, NB),
        // written in place
        auto do_set = [&](int k, auto HF, const XRow &A, const NRow &NA, int k2, const XRow &B, const NRow &NB)
            __attribute__((always_inline)) {
            constexpr int h = decltype(HF)::value;
            const float4 cc = XC[k * RR];
            const float2 xp = f2(cc.x, cc.y), sp = f2(cc.z, cc.w);
            float2 e0, e1;
            constexpr bool WD = CK && ACC;
            [[maybe_unused]] float2 d0, d1;
            // sP = +1 slot: corners (k, c), (k, c-1), (k2, c), (k2, c-1)
            const float2 v0 = seg2<WD>(K, Ip[k][2 * h], NA.il, Ip[k2][2 * h], NB.il, A.x0, A.xl, B.x0, B.xl, A.s0,
                                       A.sl, B.s0, B.sl, xp, sp, e0, &d0);
            // sP = -1 slot: corners (k, c), (k, c+1), (k2, c), (k2, c+1)
            const float2 v1 = seg2<WD>(K, Ip[k][2 * h + 1], NA.ir, Ip[k2][2 * h + 1], NB.ir, A.x0, A.xr, B.x0, B.xr,
                                       A.s0, A.sr, B.s0, B.sr, xp, sp, e1, &d1);
            if constexpr (WD) {
                // empty slots carry D = 0; a set row overwrites its slots' D later
                const bool a0 = (actm >> (2 * h)) & 1, a1 = (actm >> (2 * h + 1)) & 1;
                store_ck(m, k, h, f2(a0 ? d0.x : 0.f, a1 ? d1.x : 0.f), f2(a0 ? d0.y : 0.f, a1 ? d1.y : 0.f));
            }
            if constexpr (BND) {
                const float2 g0 = bound2(K, Gp[k][h], NA.gl, Gp[k2][h], NB.gl, e0);
                const float2 g1 = bound2(K, Gp[k][h], NA.gr, Gp[k2][h], NB.gr, e1);
                Gp[k][h] = max2(g0, g1);
            }
            Ip[k][2 * h] = v0;
            Ip[k][2 * h + 1] = v1;
        };
        using H0 = std::integral_constant<int, 0>;
        using H1 = std::integral_constant<int, 1>;
        // set boundary values (x/y groups): rising slots of the bottom row,
        // descending slots of the top row
        auto set_bc = [&](int k, int h) {
            const int q = q0 + k - 1;
            const float4 cc = XC[k * RR];
#pragma unroll
            for (int dd = 0; dd < 2; ++dd) {
                const int d = 2 * h + dd;
                float v[2] = {0.f, 0.f};
                if ((actm >> d) & 1) {
                    for (int hh = 0; hh < 2; ++hh) {
                        int i, j;
                        natural_ij(axis, c + hh * H, q, m, i, j);
                        v[hh] = reg_bc(h ? kind_dn : kind_up, h ? a.bc_dn + Ug->dn_off : a.bc_up + Ug->top_off,
                                       Ug->udx[d], unx, uny, i, j, hh ? cc.w : cc.z);
                    }
                }
                Ip[k][d] = f2(v[0], v[1]);
            }
            if constexpr (BND) Gp[k][h] = f2(0.f);
            if constexpr (CK && ACC) store_ck(m, k, h, f2(0.f), f2(0.f));
        };

        // ---- rising row TQ and descending row 1 (own rows only), published at once ----
        XRow Xr = xs_row(TQ), Xr2 = xs_row(TQ - 1);
        NRow Nr = nb_row(TQ, H0{}), Nr2 = nb_row(TQ - 1, H0{});
        do_set(TQ, H0{}, Xr, Nr, TQ - 1, Xr2, Nr2);
        XRow Xf = xs_row(1), Xf2 = xs_row(2);
        NRow Nf = nb_row(1, H1{}), Nf2 = nb_row(2, H1{});
        do_set(1, H1{}, Xf, Nf, 2, Xf2, Nf2);
        if (wrap && kb == 1) set_bc(1, 1);  // the first row is the top boundary row
        {
            float2 gd1 = f2(0.f), guq = f2(0.f);
            if constexpr (BND) {
                gd1 = Gp[1][1];
                guq = Gp[TQ][0];
            }
            publish_ring(t, Ip[1][2], Ip[1][3], gd1, Ip[TQ][0], Ip[TQ][1], guq);
        }
        prefetch(next_m(m), s_next);  // after the release, so that its fence does not wait for the copies
        // ---- the other rows that need no neighbour tile ----
#pragma unroll
        for (int k = TQ - 1; k >= 2; --k) {  // rising, downwards: row k from rows k and k-1
            Xr = Xr2;
            Nr = Nr2;
            Xr2 = xs_row(k - 1);
            Nr2 = nb_row(k - 1, H0{});
            do_set(k, H0{}, Xr, Nr, k - 1, Xr2, Nr2);
        }
#pragma unroll
        for (int k = 2; k <= TQ - 1; ++k) {  // descending, upwards: row k from rows k and k+1
            Xf = Xf2;
            Nf = Nf2;
            Xf2 = xs_row(k + 1);
            Nf2 = nb_row(k + 1, H1{});
            do_set(k, H1{}, Xf, Nf, k + 1, Xf2, Nf2);
        }

        // ---- the neighbours' rows of plane t-1: ring slot (t-1) & 3 ----
        NRow Nlo, Nup;
        Nlo.il = Nlo.ir = Nlo.gl = Nlo.gr = f2(0.f);
        Nup.il = Nup.ir = Nup.gl = Nup.gr = f2(0.f);
        bool ok = true;
        if (lane == 0) {
            const int want = t - tp;  // the neighbour released planes tp .. t-1
            ok = wait_pair_geq(a.flags + 2 * gt, has_lower ? want : INT_MIN, has_upper ? want : INT_MIN, a.status,
                               a.timeout_ns);
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (ok) {
            const int hs = (t - 1) & 3;
            const int cm = swapL ? H - 1 : c - 1, cpp = swapR ? 0 : c + 1;
            // every lane loads its own pair and its left and right neighbours' pairs
            // (the same ring lines, shifted by one; no shuffle, no divergent edge
            // lanes); c = 0 and c = H-1 take the periodic pair swapped
            if (has_lower) {  // its last row: rising slots and bound (side 1, channels 3..5)
                const float *tl = halo_base + (long long)lower * tstride;
                Ip[0][0] = __ldcg(ring_at(tl, hs, 3) + c);
                Ip[0][1] = __ldcg(ring_at(tl, hs, 4) + c);
                const float2 vl = __ldcg(ring_at(tl, hs, 3) + cm), vr = __ldcg(ring_at(tl, hs, 4) + cpp);
                Nlo.il = swapL ? swp(vl) : vl;
                Nlo.ir = swapR ? swp(vr) : vr;
                if constexpr (BND) {
                    Gp[0][0] = __ldcg(ring_at(tl, hs, 5) + c);
                    const float2 gl = __ldcg(ring_at(tl, hs, 5) + cm), gr = __ldcg(ring_at(tl, hs, 5) + cpp);
                    Nlo.gl = swapL ? swp(gl) : gl;
                    Nlo.gr = swapR ? swp(gr) : gr;
                }
            }
            if (has_upper) {  // its first row: descending slots and bound (side 0, channels 0..2)
                const float *tu = halo_base + (long long)upper * tstride;
                Ip[TQ + 1][2] = __ldcg(ring_at(tu, hs, 0) + c);
                Ip[TQ + 1][3] = __ldcg(ring_at(tu, hs, 1) + c);
                const float2 vl = __ldcg(ring_at(tu, hs, 0) + cm), vr = __ldcg(ring_at(tu, hs, 1) + cpp);
                Nup.il = swapL ? swp(vl) : vl;
                Nup.ir = swapR ? swp(vr) : vr;
                if constexpr (BND) {
                    Gp[TQ + 1][1] = __ldcg(ring_at(tu, hs, 2) + c);
                    const float2 gl = __ldcg(ring_at(tu, hs, 2) + cm), gr = __ldcg(ring_at(tu, hs, 2) + cpp);
                    Nup.gl = swapL ? swp(gl) : gl;
                    Nup.gr = swapR ? swp(gr) : gr;
                }
            }
        }
        if (ok) {
            // ---- the rows next to the neighbours ----
            {
                const XRow Xh = xs_row(0);
                do_set(1, H0{}, Xr2, Nr2, 0, Xh, Nlo);
            }
            {
                const XRow Xh = xs_row(TQ + 1);
                do_set(TQ, H1{}, Xf2, Nf2, TQ + 1, Xh, Nup);
            }
            // boundary rows of the x/y groups: set, not integrated
            if (wrap) {
                if (q0 == 0) set_bc(1, 0);
                if (kb > 0) {
#pragma unroll
                    for (int k = 1; k <= TQ; ++k)
                        if (k == kb) set_bc(k, 1);
                }
            }
            publish_edges(t);
            if constexpr (ACC) store_rows(m);
        } else if (lane == 0) {
            s_ctl[0] = 1;
        }
        // the wrap plane of an accumulated period: kept for the next solve and,
        // when seeded, compared with the previous period's (the paper's
        // iteration of boundary intensities to a tolerance)
        if constexpr (ACC) {
            if (sbuf && m == m_seed) {
                float dmax = 0.f, imax = 0.f;
                if (act && ok) {
#pragma unroll
                    for (int k = 1; k <= TQ; ++k) {
                        if (k > nrows) break;
                        const long long o = ((long long)(q0 + k - 1) * NP + c) * 4;
#pragma unroll
                        for (int d = 0; d < MAXD; ++d) {
                            if (!((actm >> d) & 1)) continue;
                            const float v0 = Ip[k][d].x, v1 = Ip[k][d].y;
                            if (seeded) {
                                dmax = fmaxf(dmax, fmaxf(fabsf(v0 - sbuf[o + d]), fabsf(v1 - sbuf[o + 4 * H + d])));
                                imax = fmaxf(imax, fmaxf(fabsf(v0), fabsf(v1)));
                            }
                            sbuf[o + d] = v0;
                            sbuf[o + 4 * H + d] = v1;
                        }
                    }
                }
                if (seeded) {
                    for (int o = 16; o; o >>= 1) {
                        dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
                        imax = fmaxf(imax, __shfl_xor_sync(0xffffffffu, imax, o));
                    }
                    if (lane == 0) {
                        s_dmax[warp] = dmax;
                        s_imax[warp] = imax;
                    }
                }
            }
            // warm start: the unit's bound of each plane of period 0 (swept from
            // the seed with unit bound) and, L planes after each period's wrap
            // plane, the decision. With gam = the bound after one period (a
            // contraction of the wrap error per period) and r_p the period's
            // relative change of the wrap plane, the seed error is at most
            // r_0 / (1 - gam), a plane u of period 0 carries at most G_u times
            // that, and every plane after period p-1 at most r_p / (1 - gam).
            // The stop plane closes a window of one period whose planes all
            // meet seed_tol.
            if (seeded && tid == dec_thread) {
                const int ts = t + 1 - a.L;
                if (ts >= 0 && ts < NM && ts < 1024) {
                    const int slot = ts % a.R;
                    const unsigned want = (unsigned)ntl * (unsigned)(ts / a.R + 1);
                    bool okd = wait_count_geq(a.gcnt + (long long)uidx * a.R + slot, want, a.status, a.timeout_ns);
                    if (okd) {
                        const unsigned long long v = ld_acquire64(a.gmax + (long long)uidx * a.R + slot);
                        if ((unsigned)(v >> 32) != (unsigned)(ts + 1)) {
                            atomicOr(a.status, ST_BADARG);  // ring overrun: never expected
                            okd = false;
                        } else {
                            s_glog[ts] = __uint_as_float((unsigned)(v & 0xffffffffu));
                        }
                    }
                    if (!okd) s_ctl[0] = 1;
                }
                const int tp_end = t - a.L - (NM - 1);
                if (tp_end >= 0 && tp_end % NM == 0) {
                    const int p = tp_end / NM, slot = p & 3;
                    const unsigned want = (unsigned)ntl * (unsigned)(p / 4 + 1);
                    bool okd = wait_count_geq(a.pcnt + (long long)uidx * 4 + slot, want, a.status, a.timeout_ns);
                    if (okd) {
                        const unsigned long long v = ld_acquire64(a.pmax + (long long)uidx * 4 + slot);
                        if ((unsigned)(v >> 32) != (unsigned)(p + 1)) {
                            atomicOr(a.status, ST_BADARG);
                            okd = false;
                        } else {
                            const float rp = __uint_as_float((unsigned)(v & 0xffffffffu));
                            const float gam = NM <= 1024 ? s_glog[NM - 1] : 2.f;
                            int stop = INT_MAX;
                            if (!(gam < 1.f)) {
                                if (rp <= a.seed_tol) stop = t;  // no contraction shown: the plain residual test
                            } else if (p == 0) {
                                const float th = a.seed_tol * (1.f - gam);
                                for (int u = 0; u < NM; ++u) {
                                    if (s_glog[u] * rp <= th) {
                                        stop = max(t, u + NM - 1);
                                        break;
                                    }
                                }
                            } else if (rp <= a.seed_tol * (1.f - gam)) {
                                stop = t;
                            }
                            if (stop != INT_MAX) s_ctl[2] = stop;
                        }
                    }
                    if (!okd) s_ctl[0] = 1;
                }
            }
        }
        if constexpr (BND) {
            float gmax = 0.f;
            if (act) {
#pragma unroll
                for (int k = 1; k <= TQ; ++k)
                    if (k <= nrows) gmax = fmaxf(gmax, fmaxf(fmaxf(Gp[k][0].x, Gp[k][0].y), fmaxf(Gp[k][1].x, Gp[k][1].y)));
            }
            for (int o = 16; o; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
            if (lane == 0) s_wmax[warp] = gmax;
            // decision for plane t+1 (its bound is L planes old: normally complete)
            if (MD == 0 && tid == dec_thread && t + 1 - a.L >= 0) {
                const int ts = t + 1 - a.L;
                const int slot = ts % a.R;
                const unsigned want = (unsigned)ntl * (unsigned)(ts / a.R + 1);
                bool okd = wait_count_geq(a.gcnt + (long long)uidx * a.R + slot, want, a.status, a.timeout_ns);
                if (okd) {
                    const unsigned long long v = ld_acquire64(a.gmax + (long long)uidx * a.R + slot);
                    if ((unsigned)(v >> 32) != (unsigned)(ts + 1)) {
                        atomicOr(a.status, ST_BADARG);  // ring overrun: never expected
                        okd = false;
                    } else {
                        s_ctl[1] = __uint_as_float((unsigned)(v & 0xffffffffu)) <= a.tol ? 1 : 0;
                    }
                }
                if (!okd) s_ctl[0] = 1;
            }
        }
        cp_async_wait_all();  // this thread's chi/S of plane t+1
        __syncthreads();      // plane t complete in the CTA; plane t+1's chi/S visible
        if (s_ctl[0]) return 2;
        release_plane();
        if constexpr (BND) {
            if (tid == 0) {
                float g = 0.f;
                for (int w = 0; w < NW; ++w) g = fmaxf(g, s_wmax[w]);
                const int slot = t % a.R;
                const unsigned long long pv = ((unsigned long long)(unsigned)(t + 1) << 32) | __float_as_uint(g);
                atomicMax(a.gmax + (long long)uidx * a.R + slot, pv);
                red_release_add(a.gcnt + (long long)uidx * a.R + slot, 1u);
            }
        }
        if constexpr (ACC) {
            if (seeded && m == m_seed && tid == 0) {  // this tile's relative change over period p
                float dm = 0.f, im = 0.f;
                for (int w = 0; w < NW; ++w) {
                    dm = fmaxf(dm, s_dmax[w]);
                    im = fmaxf(im, s_imax[w]);
                }
                const float rel = im > 0.f ? dm / im : (dm > 0.f ? 1.f : 0.f);
                const int p = (t - (NM - 1)) / NM;
                const int slot = p & 3;
                const unsigned long long pv = ((unsigned long long)(unsigned)(p + 1) << 32) | __float_as_uint(rel);
                atomicMax(a.pmax + (long long)uidx * 4 + slot, pv);
                red_release_add(a.pcnt + (long long)uidx * 4 + slot, 1u);
            }
        }
        const int sp_old = s_prev;
        s_prev = s_cur;
        s_cur = s_next;
        s_next = sp_old;
        if (seeded && ACC && t >= s_ctl[2]) {  // warm start decided (before the barrier): last plane
            if (r == 0 && tid == 0) a.unit_tacc[uidx] = t + 1 - NM;
            return 1;
        }
        return last ? 1 : 0;
    };

    int t = t_first;
    int mc = plane_of(t_first, NM, sa);  // plane of step t, advanced without a division
    if (wrap && !seeded) {
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
            if (plane_step(Mode<0>{}, t, mc) == 2) {
                cp_async_wait_all();
                return;
            }
            mc = next_m(mc);
        }
    }
    for (;; ++t) {
        if (seeded && t >= warm_cap) {  // the warm start did not converge within max_periods
            if (tid == 0) atomicOr(a.status, ST_NOCONV);
            break;
        }
        int rc;
        if constexpr (SEED)
            rc = (seeded && t < NM) ? plane_step(Mode<2>{}, t, mc) : plane_step(Mode<1>{}, t, mc);
        else
            rc = plane_step(Mode<1>{}, t, mc);
        if (rc == 2) {
            cp_async_wait_all();
            return;
        }
        if (rc == 1) break;
        mc = next_m(mc);
    }
    cp_async_wait_all();
}

template <int TQ, int MAXR, bool SEED, bool CK = false>
__global__ void __maxnreg__(MAXR) sweep_reg_kernel(SweepArgs<float> a)
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
        const int tile = a.tile_base + (a.tile_order ? a.tile_order[s_tile] : s_tile);
        const int u = a.unit_of_tile[tile];
        run_tile_reg<TQ, SEED, CK>(a, a.units + u, u, tile - a.units[u].tile0, tile, smem);
    }
}

}  // namespace rts

// adjoint.cuh -- reverse-mode derivative of the solve: gradients of
// L = <gI_top, I_top> + <gJ, J> + <gF, F> + <gQ, Q_rad> with respect to
// log chi and S of every band.
//
// The solve is a chain  (chi, S) -> I (per ray, by the sweep recurrence)
// -> (J_b, F_b) -> Q_rad. Its adjoint, written for this GPU layout, runs per
// checkpoint chunk of bands:
//  1. the forward sweep of the chunk again (sweep.cuh), storing per point and
//     ray of the converged period the segment's dI/d(dtau); its partial sums
//     give the chunk's J_b and F_b;
//  2. qstep_adjoint_kernel: cotangents of J_b and F_b (through the Q step
//     and the band sums) and the direct chi/S terms of the Q step;
//  3. sweep_adj_kernel: the reverse sweep. For ray d the cotangent of I obeys
//     lam(p) = lam0(p) + sum_c beta_c e(r_c) lam(r_c), summed over the
//     downwind points r_c whose upwind corner c is p: the transpose of the
//     forward interpolation, run over the planes in reverse order with tiles,
//     ready flags and a periodic-wrap bound like the forward sweep. With lam
//     known it writes each segment's gradient terms: B = lam dI/d(dtau) ds/2
//     (opacity, own point and upwind corners), C = lam w_up (source at the
//     corners) and the own-point chi and S terms; it recomputes the segment's
//     dtau, e and weights from the same chi as the forward sweep;
//  4. adj_gather_kernel: adds to every point the B and C of the downwind
//     points that interpolated from it;
//  5. adj_reduce_kernel: sum over the band's sweep units, times chi for
//     d/d log chi.
#pragma once
#include "df32.cuh"
#include "qstep.cuh"
#include "sweep.cuh"

namespace rts {

// ---------------------------------------------------------------------------
// 1. Q step adjoint (natural layout, one thread per point, loop over bands)
// ---------------------------------------------------------------------------
struct QAdjParams {
    int nx, ny, nz, nbands;
    double inv2dx, inv2dy, inv2dz, invdz;  // stencil coefficients
    double thin;                           // min(dx, dy, dz) / tau_switch
};

// coefficient of F_z(level k) in the z part of div F at level q: central
// differences inside, first-order one-sided at the bottom and top levels,
// nothing when there is a single level
__device__ __forceinline__ double coef_z(int q, int k, const QAdjParams &P)
{
    const int nz = P.nz;
    if (nz == 1) return 0.0;
    if (q == 0) return k == 1 ? P.invdz : (k == 0 ? -P.invdz : 0.0);
    if (q == nz - 1) return k == nz - 1 ? P.invdz : (k == nz - 2 ? -P.invdz : 0.0);
    return k == q + 1 ? P.inv2dz : (k == q - 1 ? -P.inv2dz : 0.0);
}

// Per band b and point p, with u = gQ (1 - om_b):
//   lam0 = (gJ_b, gF_b) = (gJ + gQ om_b 4 pi chi_b,  gF - D^T u)
//   direct d/dchi_b = gQ (om_b 4 pi (J_b - S_b) + dom_b/dchi_b (QJ_b - QF_b)),
//   direct d/dS_b   = -gQ om_b 4 pi chi_b,
// QJ_b = 4 pi chi_b (J_b - S_b), QF_b = -div F_b, D the divergence stencil.
// The blend weights are evaluated exactly as the forward Q step does (in the
// sweep precision, blend_weights), so this is the derivative of the computed
// function. Bands b0 .. b1-1; JF, lam0, direct are indexed by band; u
// ([b1-b0][N], from qstep_adjoint_u_kernel) only when gQ is given.
template <typename T>
__global__ void __launch_bounds__(256) qstep_adjoint_u_kernel(const T *__restrict__ chi,
                                                               const double *__restrict__ gQ, QAdjParams P, int b0,
                                                               int b1, T *__restrict__ u)
{
    const long long N = (long long)P.nx * P.ny * P.nz, total = (long long)(b1 - b0) * N;
    const T thin = (T)P.thin;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long bb = idx / N, p = idx - bb * N;
        T om, omc;
        blend_weights(chi[(b0 + bb) * N + p], thin, om, omc);
        u[idx] = (T)gQ[p] * omc;
    }
}

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) qstep_adjoint_kernel(const Acc *__restrict__ JF, const T *__restrict__ chi,
                                                             const T *__restrict__ S, const double *__restrict__ gJ,
                                                             const double *__restrict__ gF,
                                                             const double *__restrict__ gQ, const T *__restrict__ u,
                                                             QAdjParams P, int b0, int b1, T *__restrict__ lam0,
                                                             T *__restrict__ direct)
{
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= P.nx || j >= P.ny) return;
    const long long nx = P.nx, ny = P.ny, nz = P.nz, N = nx * ny * nz, pl = nx * ny;
    const long long p = (long long)k * pl + (long long)j * nx + i;
    const int im = i == 0 ? P.nx - 1 : i - 1, ip = i + 1 == P.nx ? 0 : i + 1;
    const int jm = j == 0 ? P.ny - 1 : j - 1, jp = j + 1 == P.ny ? 0 : j + 1;
    const long long pxp = p - i + ip, pxm = p - i + im;
    const long long pyp = p + (long long)(jp - j) * nx, pym = p + (long long)(jm - j) * nx;
    const double four_pi = 12.566370614359172953850573533118;
    const T thin = (T)P.thin;
    const double gq = gQ ? gQ[p] : 0.0;
    for (int b = b0; b < b1; ++b) {
        const T *cb = chi + (long long)b * N;
        const Acc *jf = JF + (long long)b * 4 * N;
        // cancelling differences in FP64, the rest in the sweep precision T
        const T *ub = gQ ? u + (long long)(b - b0) * N : nullptr;
        auto u_at = [&](long long q) -> T { return ub ? ub[q] : T(0); };  // gQ (1 - om_b) at point q
        T om, omc;
        blend_weights(cb[p], thin, om, omc);
        const T c = cb[p];
        const T fpc = (T)four_pi * c;
        double gJb = gJ ? gJ[p] : 0.0;
        T gchi = 0, gs = 0;
        if (gQ) {  // J_b and F_b of the forward solve are read only when Q_rad enters L
            double divz = 0.0;
            for (int q = k - 1; q <= k + 1; ++q) {
                if (q < 0 || q >= P.nz) continue;
                const double cf = coef_z(k, q, P);
                if (cf != 0.0) divz += cf * acc_to_double(jf[3 * N + (long long)q * pl + (long long)j * nx + i]);
            }
            const T qf = (T)(-((acc_to_double(jf[N + pxp]) - acc_to_double(jf[N + pxm])) * P.inv2dx +
                               (acc_to_double(jf[2 * N + pyp]) - acc_to_double(jf[2 * N + pym])) * P.inv2dy + divz));
            const T dJ = (T)(acc_to_double(jf[p]) - (double)S[(long long)b * N + p]);  // J_b - S_b
            const T gqT = (T)gq;
            const T qj = fpc * dJ;
            gJb += gq * (double)(om * fpc);
            gchi = gqT * (om * (T)four_pi * dJ - thin * om * (qj - qf));
            gs = -gqT * om * fpc;
        }
        const double gFx = (gF ? gF[p] : 0.0) + (double)((u_at(pxp) - u_at(pxm)) * (T)P.inv2dx);
        const double gFy = (gF ? gF[N + p] : 0.0) + (double)((u_at(pyp) - u_at(pym)) * (T)P.inv2dy);
        T dTz = 0;  // (D_z^T u)(k) = sum_q u(q) coef_z(q, k)
        for (int q = k - 1; q <= k + 1; ++q) {
            if (q < 0 || q >= P.nz) continue;
            const T cf = (T)coef_z(q, k, P);
            if (cf != T(0)) dTz += u_at((long long)q * pl + (long long)j * nx + i) * cf;
        }
        const double gFz = (gF ? gF[2 * N + p] : 0.0) - (double)dTz;
        // lam0 of a point together ([b][N][4]), one vector store
        st4(lam0 + ((long long)b * N + p) * 4, (T)gJb, (T)gFx, (T)gFy, (T)gFz);
        T *dr = direct + (long long)b * 2 * N;
        dr[p] = (T)gchi;
        dr[N + p] = (T)gs;
    }
}

// The same Q-step adjoint for double-float J_b, F_b (the register sweep's
// reduction) in FP32 arithmetic: each cancelling difference is formed from
// the two double-float values as (hi - hi) + (lo - lo) -- the high parts of
// neighbouring values differ by less than a factor 2 where the difference is
// small, so their difference is exact there -- and everything else in FP32.
// The cotangent inputs (FP64) are converted once per point, outside the band
// loop, so the kernel does no FP64 arithmetic per band.
__device__ __forceinline__ float df_diff(df32 a, df32 b) { return (a.hi - b.hi) + (a.lo - b.lo); }

template <int = 0>  // a template, so that every translation unit including this header may define it
__global__ void __launch_bounds__(256) qstep_adjoint_df_kernel(const df32 *__restrict__ JF,
                                                                const float *__restrict__ chi,
                                                                const float *__restrict__ S,
                                                                const double *__restrict__ gJ,
                                                                const double *__restrict__ gF,
                                                                const double *__restrict__ gQ,
                                                                const float *__restrict__ u, QAdjParams P, int b0,
                                                                int b1, float *__restrict__ lam0,
                                                                float *__restrict__ direct)
{
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= P.nx || j >= P.ny) return;
    const long long nx = P.nx, ny = P.ny, nz = P.nz, N = nx * ny * nz, pl = nx * ny;
    const long long p = (long long)k * pl + (long long)j * nx + i;
    const int im = i == 0 ? P.nx - 1 : i - 1, ip = i + 1 == P.nx ? 0 : i + 1;
    const int jm = j == 0 ? P.ny - 1 : j - 1, jp = j + 1 == P.ny ? 0 : j + 1;
    const long long pxp = p - i + ip, pxm = p - i + im;
    const long long pyp = p + (long long)(jp - j) * nx, pym = p + (long long)(jm - j) * nx;
    const float four_pi = 12.566370614359172954f;
    const float thin = (float)P.thin, i2x = (float)P.inv2dx, i2y = (float)P.inv2dy;
    // z part of div F at level k: the two levels it differences and their coefficient
    int zq1 = k + 1, zq0 = k - 1;
    float zc = (float)P.inv2dz;
    if (nz == 1) zc = 0.f, zq1 = zq0 = k;
    else if (k == 0) zq1 = 1, zq0 = 0, zc = (float)P.invdz;
    else if (k == nz - 1) zq1 = k, zq0 = k - 1, zc = (float)P.invdz;
    const float gq = gQ ? (float)gQ[p] : 0.f;
    const float gJp = gJ ? (float)gJ[p] : 0.f;
    const float gFxp = gF ? (float)gF[p] : 0.f, gFyp = gF ? (float)gF[N + p] : 0.f;
    const float gFzp = gF ? (float)gF[2 * N + p] : 0.f;
    for (int b = b0; b < b1; ++b) {
        const float *cb = chi + (long long)b * N;
        const df32 *jf = JF + (long long)b * 4 * N;
        const float *ub = gQ ? u + (long long)(b - b0) * N : nullptr;
        auto u_at = [&](long long q) -> float { return ub ? ub[q] : 0.f; };  // gQ (1 - om_b) at point q
        float om, omc;
        blend_weights(cb[p], thin, om, omc);
        const float fpc = four_pi * cb[p];
        float gJb = gJp, gchi = 0.f, gs = 0.f;
        if (gQ) {  // J_b and F_b of the forward solve are read only when Q_rad enters L
            const long long col = (long long)j * nx + i;
            const float divz = zc == 0.f ? 0.f : df_diff(jf[3 * N + zq1 * pl + col], jf[3 * N + zq0 * pl + col]) * zc;
            const float qf = -(df_diff(jf[N + pxp], jf[N + pxm]) * i2x + df_diff(jf[2 * N + pyp], jf[2 * N + pym]) * i2y +
                               divz);
            const df32 Jb = jf[p];
            const float dJ = (Jb.hi - S[(long long)b * N + p]) + Jb.lo;  // J_b - S_b
            const float qj = fpc * dJ;
            gJb += gq * (om * fpc);
            gchi = gq * (om * four_pi * dJ - thin * om * (qj - qf));
            gs = -gq * om * fpc;
        }
        const float gFx = gFxp + (u_at(pxp) - u_at(pxm)) * i2x;
        const float gFy = gFyp + (u_at(pyp) - u_at(pym)) * i2y;
        float dTz = 0.f;  // (D_z^T u)(k) = sum_q u(q) coef_z(q, k)
        for (int q = k - 1; q <= k + 1; ++q) {
            if (q < 0 || q >= P.nz) continue;
            const float cf = (float)coef_z(q, k, P);
            if (cf != 0.f) dTz += u_at((long long)q * pl + (long long)j * nx + i) * cf;
        }
        st4(lam0 + ((long long)b * N + p) * 4, gJb, gFx, gFy, gFzp - dTz);
        float *dr = direct + (long long)b * 2 * N;
        dr[p] = gchi;
        dr[N + p] = gs;
    }
}

// ---------------------------------------------------------------------------
// 3. Reverse sweep of one tile (cotangent lam of the rays of one unit)
// ---------------------------------------------------------------------------
// Shared memory of a reverse tile, (TQ+2) rows x (NP+2) columns per field like
// the forward tile: A = e lam of the 4 slots of a point stored together
// ([row][col][4]; the downwind plane, kept once: new rows stay in registers
// until every thread has read it), chi of three planes (the own plane, its
// forward-upwind plane and the next one in flight), and the two seed-error
// bounds of a point as bf16 rounded up.
enum { AF_A = 4, AF_X = 3 };
// gradient terms written by the reverse sweep per point of a unit: B of the 4
// slots, C of the 4 slots, the own chi and S terms
constexpr int GRAD_CH = 2 * MAXD + 2;

template <typename T>
__host__ __device__ constexpr size_t adj_tile_smem_bytes(int tq, int np)
{
    return (size_t)(tq + 2) * (np + 2) * ((AF_A + AF_X) * sizeof(T) + 2 * sizeof(unsigned short));
}

__device__ __forceinline__ void cp_async_wait_newest_pending() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// new values of one point of the reverse plane: e lam of the 4 slots and,
// during the periodic warm-up, the carried bounds of the up / down rays
template <typename T, bool ACC>
struct AdjRow {
    T A[MAXD];
    float g[2];
};
template <typename T>
struct AdjRow<T, true> {
    T A[MAXD];
};

// cotangent of the upward intensity of slot d leaving the top at (p, q) of
// plane m (out of line: only the top row or plane takes it)
template <typename T>
__device__ __noinline__ T top_cotangent(const T *gitop, const DirConst<T> &D, int d, int axis, int p, int q, int m,
                                        int unx, int uny)
{
    int i, j;
    natural_ij(axis, p, q, m, i, j);
    return gitop[((long long)D.udx[d] * uny + j) * unx + i];
}

template <typename T, int TQ>
__device__ void run_tile_adj(const SweepArgs<T> &a, const SweepUnit *__restrict__ Ug, int uidx, int r, int gt,
                             unsigned char *smem)
{
    constexpr int RW = TQ + 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NT = blockDim.x;
    const int NP = Ug->NP, NQ = Ug->NQ, NM = Ug->NM;
    const int axis = Ug->axis, sa = Ug->sa, ntl = Ug->ntiles, tile0 = Ug->tile0;
    const bool wrap = Ug->wrap != 0, qper = Ug->qper != 0;
    const int band = Ug->band, unx = Ug->nx, uny = Ug->ny;
    const long long sQ = Ug->sQ, sM = Ug->sM, N = Ug->N;
    const T *__restrict__ chi = (Ug->transposed ? a.chiT : a.chi) + Ug->in_off;
    const T *__restrict__ l0 = (Ug->transposed ? a.lam0T : a.lam0) + (long long)band * 4 * N;
    const T *const gitop = a.gitop ? a.gitop + Ug->top_off : nullptr;
    // gradient terms of this unit: B [4][N], C [4][N], own chi / S terms [2][N]
    T *const gout = a.store + (long long)(uidx - a.unit_base) * GRAD_CH * N;
    const T *const ck = a.ckpt + (long long)(uidx - a.unit_base) * STORE_CH * MAXD * N;
    const long long tile_stride = (long long)2 * 2 * HALO_CH * NP;
    T *const halo_base = a.halo + Ug->halo_off;
    T *const myhalo = halo_base + (long long)r * tile_stride;
    const int msa = -sa;  // planes are visited in reverse order

    const int q0 = r * TQ;
    const int nrows = min(TQ, NQ - q0);
    const int p = tid;
    const bool act = p < NP;
    const int c = p + 1;
    const int npp = NP + 2;
    const int FL = RW * npp;
    T *const sA = (T *)smem;                                   // [FL][4]
    T *const sX = sA + AF_A * FL;                              // chi of reverse step t: sX + (t % 3) * FL
    unsigned short *const sG = (unsigned short *)(sX + AF_X * FL);  // [FL][2]
    auto fX = [&](int t) -> T * { return sX + (t % 3) * FL; };

    __shared__ DirConst<T> D;
    __shared__ float s_wmax[32];
    __shared__ int s_ctl[4];
    __shared__ int s_q[RW];

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

    const int lower = qper ? (r + ntl - 1) % ntl : r - 1;
    const int upper = qper ? (r + 1) % ntl : r + 1;
    const bool has_lower = qper || r > 0;
    const bool has_upper = qper || r < ntl - 1;

    // periodic padding: thread p = 0 also writes column NP + 1 and thread
    // p = NP - 1 column 0 (with NP == 1 the one thread writes both)
    const bool padA = act && (p == 0 || p == NP - 1), padB = act && NP == 1;
    const int pc = p == 0 ? NP + 1 : 0;
    auto putA = [&](int k, T v0, T v1, T v2, T v3) {
        st4(sA + (k * npp + c) * 4, v0, v1, v2, v3);
        if (padA) st4(sA + (k * npp + pc) * 4, v0, v1, v2, v3);
        if (padB) st4(sA + (k * npp) * 4, v0, v1, v2, v3);
    };
    auto putG = [&](int k, float gu, float gd) {
        const unsigned w = bound16(gu) | bound16(gd) << 16;
        unsigned *const g32 = (unsigned *)sG;
        g32[k * npp + c] = w;
        if (padA) g32[k * npp + pc] = w;
        if (padB) g32[k * npp] = w;
    };
    auto putX = [&](T *f, int k, T v) {
        f[k * npp + c] = v;
        if (padA) f[k * npp + pc] = v;
        if (padB) f[k * npp] = v;
    };
    // chi rows of reverse step t into slot t % 3
    auto prefetch = [&](int t) {
        if (act) {
            const long long mo = (long long)plane_of(t, NM, msa) * sM + p;
            T *dx = fX(t);
            for (int k = 0; k < nrows + 2; ++k) {
                const int q = s_q[k];
                if (q < 0) { putX(dx, k, T(0)); continue; }
                const T *gx = chi + mo + (long long)q * sQ;
                cp_async(dx + k * npp + c, gx);
                if (padA) cp_async(dx + k * npp + pc, gx);
                if (padB) cp_async(dx + k * npp, gx);
            }
        }
        cp_async_commit();
    };

    __syncthreads();
    int upm = 0, actm = 0;
    for (int d = 0; d < MAXD; ++d) {
        upm |= D.up[d] ? 1 << d : 0;
        actm |= D.active[d] ? 1 << d : 0;
    }
    // prologue: the (downwind) plane before the first reverse step carries
    // A = 0; for the periodic groups that is the seed, with a unit bound on
    // the points that are not set. Rows outside a non-periodic Q range stay
    // zero for the whole sweep.
    if (act) {
        for (int k = 0; k < nrows + 2; ++k) {
            const int q = s_q[k];
            putA(k, T(0), T(0), T(0), T(0));
            float gu = 0.f, gd = 0.f;
            if (wrap && q >= 0) {
                if (q != 0) gu = 1.f;
                if (q != NQ - 1) gd = 1.f;
            }
            putG(k, gu, gd);
        }
    }
    prefetch(0);
    prefetch(1);
    cp_async_wait_all();
    prefetch(2);
    __syncthreads();

    int t_acc = wrap ? -1 : 0;
    const int warm_cap = a.max_periods * NM + a.L;
    const int dec_thread = NT > 32 ? 32 : 0;

    // One reverse step t. ACC: the plane is in the converged period (its
    // gradient terms are written). Returns 0 to go on, 1 after the last
    // plane, 2 to abandon the tile (a wait failed).
    auto plane_step = [&](auto ACC, int t) __attribute__((always_inline)) -> int {
        constexpr bool acc = decltype(ACC)::value;
        using Row = AdjRow<T, acc>;
        const int m = plane_of(t, NM, msa);
        const bool last = acc && (t - t_acc == NM - 1);
        const T *Xc = fX(t), *Xn = fX(t + 1);  // chi of this plane and of its forward-upwind plane
        // a z group's last reverse plane is its boundary layer (set points)
        const bool bnd_plane = !wrap && t == NM - 1;
        const bool top_plane = axis == 2 && t == 0 && sa > 0;
        float gmax = 0.f;

        // row k (1..nrows): lam from the downwind plane in shared memory, the
        // point's own cotangents, then A = e lam for the upwind plane
        auto do_row = [&](int k) __attribute__((always_inline)) -> Row {
            Row out;
            const int q = q0 + k - 1;
            const int o = k * npp + c;
            const long long goff = (long long)m * sM + (long long)q * sQ + p;
            T lv[4];
            ld_part(l0 + goff * 4, lv);
            const T gJ = lv[0], gFx = lv[1], gFy = lv[2], gFz = lv[3];
            const bool top = axis == 2 ? top_plane : q == NQ - 1;
            // forward-upwind plane's chi on the 3 x 3 neighbourhood, shared by the rays
            T xs[3][3];
#pragma unroll
            for (int dq = 0; dq < 3; ++dq)
#pragma unroll
                for (int dp = 0; dp < 3; ++dp) xs[dq][dp] = Xn[o + (dq - 1) * npp + dp - 1];
            const T xp = Xc[o];
            T hd[MAXD], cw[4][MAXD];
            ld4(D.hds, hd[0], hd[1], hd[2], hd[3]);
            ld4(D.cJ, cw[0][0], cw[0][1], cw[0][2], cw[0][3]);
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) ld4(D.cF[cc], cw[cc + 1][0], cw[cc + 1][1], cw[cc + 1][2], cw[cc + 1][3]);
            const T *Ab = sA + o * 4;
            const int ar = npp * 4;
            [[maybe_unused]] const unsigned short *Gb = sG + o * 2;
            [[maybe_unused]] const int gr = npp * 2;
            float gu = 0.f, gd = 0.f, egu = 0.f, egd = 0.f;
            [[maybe_unused]] T own_chi = 0, own_S = 0;
            // the checkpoint's D of the 4 slots of this point (converged period only)
            [[maybe_unused]] T ckv[MAXD];
            if constexpr (acc) ld_part(ck + goff * MAXD, ckv);
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                const int SP = (d & 1) ? -1 : 1, SQ = (d & 2) ? -1 : 1;  // compile time after unrolling
                T b0, b1, b2, b3;
                ld4(D.beta[d], b0, b1, b2, b3);
                // downwind points r_c whose corner c is this point: offsets (+SP, +SQ)
                const T *Ap = Ab + d;
                const int oq = SQ * ar;
                T lam = b0 * Ap[0] + b1 * Ap[4 * SP] + b2 * Ap[oq] + b3 * Ap[oq + 4 * SP];
                lam += cw[0][d] * gJ + cw[1][d] * gFx + cw[2][d] * gFy + cw[3][d] * gFz;
                const bool isup = (upm >> d) & 1;
                if (gitop && top && isup && ((actm >> d) & 1)) lam += top_cotangent(gitop, D, d, axis, p, q, m, unx, uny);
                if (!((actm >> d) & 1)) lam = T(0);
                const bool set = wrap ? (isup ? q == 0 : q == NQ - 1) : bnd_plane;
                T e = T(0), wu = T(0), wp = T(0);
                if (!set) {
                    const T xup = b0 * xs[1][1] + b1 * xs[1][1 - SP] + b2 * xs[1 - SQ][1] + b3 * xs[1 - SQ][1 - SP];
                    seg_weights(hd[d] * (xup + xp), e, wu, wp);
                }
                out.A[d] = e * lam;
                if constexpr (acc) {
                    // gradient terms of this point's segment (lam known now):
                    // B = lam dI/dx ds/2 (to chi here and at the corners), C = lam w_up
                    // (to S at the corners), lam w_p (to S here); set points with
                    // I = S pass lam to S
                    T Bv = 0, Cv = 0;
                    if (((actm >> d) & 1) && !set) {
                        const T dI = ckv[d];
                        Bv = lam * dI * hd[d];
                        Cv = lam * wu;
                        own_chi += Bv;
                        own_S += lam * wp;
                    } else if (((actm >> d) & 1) && D.bck[d] == 1) {
                        own_S += lam;
                    }
                    gout[(long long)d * N + goff] = Bv;
                    gout[(long long)(MAXD + d) * N + goff] = Cv;
                } else {
                    // bounds of the downwind points this point's ray d feeds (the
                    // x/y groups' rising rays are the first value of a pair)
                    const unsigned short *Gd = Gb + (isup ? 0 : 1);
                    const int gq = SQ * gr;
                    const float gg = (float)b0 * bound32(Gd[0]) + (float)b1 * bound32(Gd[2 * SP]) +
                                     (float)b2 * bound32(Gd[gq]) + (float)b3 * bound32(Gd[gq + 2 * SP]);
                    if (isup) { gu = fmaxf(gu, gg); egu = fmaxf(egu, (float)e); }
                    else { gd = fmaxf(gd, gg); egd = fmaxf(egd, (float)e); }
                }
            }
            if constexpr (acc) {
                gout[(long long)(2 * MAXD) * N + goff] = own_chi;
                gout[(long long)(2 * MAXD + 1) * N + goff] = own_S;
            } else {
                // the bound carried to the upwind plane: e * g (max over the rays of each set)
                gu *= egu;
                gd *= egd;
                if (wrap && q == 0) gu = 0.f;
                if (wrap && q == NQ - 1) gd = 0.f;
                out.g[0] = gu;
                out.g[1] = gd;
                gmax = fmaxf(gmax, fmaxf(gu, gd));
            }
            return out;
        };
        auto to_ring = [&](int sd, const Row &rw) __attribute__((always_inline)) {
            T *dst = myhalo + ((long long)((t & 1) * 2 + sd) * HALO_CH) * NP + p;
#pragma unroll
            for (int d = 0; d < MAXD; ++d) dst[(long long)d * NP] = rw.A[d];
            if constexpr (!acc) {
                dst[(long long)MAXD * NP] = (T)rw.g[0];
                dst[(long long)(MAXD + 1) * NP] = (T)rw.g[1];
            }
        };

        Row nR[TQ], rl;
        if (act) {
#pragma unroll
            for (int k = 2; k < TQ; ++k)
                if (k < nrows) nR[k - 1] = do_row(k);
        }
        if (t > 0) {
            if (tid == 0) {
                bool ok = true;
                ok = wait_pair_geq(a.flags + 2 * gt, has_lower ? t : INT_MIN, has_upper ? t : INT_MIN, a.status,
                                   a.timeout_ns);
                if (!ok) s_ctl[0] = 1;
            }
            __syncthreads();  // B0: the neighbours' rows of step t-1 are published (or the wait failed)
            if (act && !s_ctl[0]) {
                const int hslot = (t - 1) & 1;
                for (int side = 0; side < 2; ++side) {
                    if (side == 0 ? !has_lower : !has_upper) continue;
                    const int nb = side == 0 ? lower : upper;
                    const int row = side == 0 ? 0 : nrows + 1;
                    const T *src = halo_base + (long long)nb * tile_stride +
                                   ((long long)(hslot * 2 + (side == 0 ? 1 : 0)) * HALO_CH) * NP + p;
                    T hv[HALO_CH];
#pragma unroll
                    for (int ch = 0; ch < HALO_CH; ++ch)
                        hv[ch] = (ch < MAXD || !acc) ? ld_cg(src + (long long)ch * NP) : T(0);
                    putA(row, hv[0], hv[1], hv[2], hv[3]);
                    if constexpr (!acc) putG(row, (float)hv[MAXD], (float)hv[MAXD + 1]);
                }
            }
        }
        __syncthreads();  // B1
        if (s_ctl[0]) {
            cp_async_wait_all();
            return 2;
        }
        if (act) {
            nR[0] = do_row(1);
            to_ring(0, nR[0]);
            rl = nrows == 1 ? nR[0] : do_row(nrows);
            to_ring(1, rl);
        }
        if constexpr (!acc) {
            for (int o = 16; o; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
            if (lane == 0) s_wmax[warp] = gmax;
            if (tid == dec_thread && t + 1 - a.L >= 0) {
                const int ts = t + 1 - a.L;
                const int slot = ts % a.R;
                const unsigned want = (unsigned)ntl * (unsigned)(ts / a.R + 1);
                bool ok = wait_count_geq(a.gcnt + (long long)uidx * a.R + slot, want, a.status, a.timeout_ns);
                if (ok) {
                    const unsigned long long v = ld_acquire64(a.gmax + (long long)uidx * a.R + slot);
                    if ((unsigned)(v >> 32) != (unsigned)(ts + 1)) {
                        atomicOr(a.status, ST_BADARG);
                        ok = false;
                    } else {
                        s_ctl[1] = __uint_as_float((unsigned)(v & 0xffffffffu)) <= a.tol ? 1 : 0;
                    }
                }
                if (!ok) s_ctl[0] = 1;
            }
        }
        __syncthreads();  // B2: step t's edge rows are in the ring; the downwind plane is no longer read
        if (tid == 0) {
            // to the tile above (as its lower neighbour) and the tile below (as its upper)
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
        if (s_ctl[0]) {
            cp_async_wait_all();
            return 2;
        }
        auto write_row = [&](int kk, const Row &rw) __attribute__((always_inline)) {
            putA(kk + 1, rw.A[0], rw.A[1], rw.A[2], rw.A[3]);
            if constexpr (!acc) putG(kk + 1, rw.g[0], rw.g[1]);
        };
        if (act) {
#pragma unroll
            for (int kk = 0; kk < TQ - 1; ++kk)
                if (kk < nrows - 1) write_row(kk, nR[kk]);
            write_row(nrows - 1, rl);
        }
        if (last) return 1;
        // chi of step t+3 into the slot of step t; step t+2's copy (issued a
        // step ago) must be complete before the barrier
        prefetch(t + 3);
        cp_async_wait_newest_pending();
        __syncthreads();  // B3
        return 0;
    };

    // the periodic warm-up and the converged period run as two loops, each
    // compiled for its own phase
    int t = 0;
    if (wrap) {
        for (;; ++t) {
            if (s_ctl[1]) {  // decision taken during the previous step
                t_acc = t;
                if (r == 0 && tid == 0) a.unit_tacc[uidx] = t;
                break;
            }
            if (t >= warm_cap) {
                if (tid == 0) atomicOr(a.status, ST_NOCONV);
                cp_async_wait_all();
                return;
            }
            if (plane_step(Flag<false>{}, t) == 2) return;
        }
    }
    for (;; ++t) {
        const int rc = plane_step(Flag<true>{}, t);
        if (rc == 2) return;
        if (rc == 1) break;
    }
    cp_async_wait_all();
}

template <typename T, int TQ, int MAXR>
__global__ void __maxnreg__(MAXR) sweep_adj_kernel(SweepArgs<T> a)
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
        run_tile_adj<T, TQ>(a, a.units + u, u, tile - a.units[u].tile0, tile, smem);
    }
}

// ---------------------------------------------------------------------------
// 4. Segment gradient terms gathered onto the corners they interpolated from
// ---------------------------------------------------------------------------
template <typename T>
struct GradArgs {
    const SweepUnit *units;
    int unit_base;
    T *grad;          // [units][GRAD_CH][N]: B, C (read), own terms (updated in place)
};

// a unit's ray constants in the sweep precision, converted once per block
template <typename T>
struct PassConst {
    T beta[MAXD][4], hds[MAXD];
    int active, up;
};
template <typename T>
__device__ __forceinline__ void load_pass_const(const SweepUnit &U, PassConst<T> &K)
{
    if (threadIdx.x < MAXD * 4) K.beta[threadIdx.x >> 2][threadIdx.x & 3] = (T)U.beta[threadIdx.x >> 2][threadIdx.x & 3];
    if (threadIdx.x < MAXD) K.hds[threadIdx.x] = (T)(0.5 * U.ds[threadIdx.x]);
    if (threadIdx.x == 0) {
        int a = 0, u = 0;
        for (int d = 0; d < MAXD; ++d) {
            a |= U.active[d] ? 1 << d : 0;
            u |= U.up[d] ? 1 << d : 0;
        }
        K.active = a;
        K.up = u;
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(512) adj_gather_kernel(GradArgs<T> g, int maxNM)
{
    const int uu = blockIdx.z / maxNM, m = blockIdx.z % maxNM;
    const SweepUnit &U = g.units[g.unit_base + uu];
    __shared__ PassConst<T> K;
    load_pass_const(U, K);
    const int NP = U.NP, NQ = U.NQ, NM = U.NM;
    const int p = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
    if (m >= NM || q >= NQ || p >= NP) return;
    const long long N = U.N, sQ = U.sQ, sM = U.sM;
    const T *B = g.grad + (long long)uu * GRAD_CH * N;
    const T *C = B + MAXD * N;
    T *G = g.grad + (long long)uu * GRAD_CH * N + 2 * MAXD * N;
    const long long off = (long long)m * sM + (long long)q * sQ + p;
    int md = m + U.sa;  // forward-downwind plane
    if (U.wrap) md = md < 0 ? md + NM : (md >= NM ? md - NM : md);
    T gx = G[off], gs = G[N + off];
    if (md >= 0 && md < NM) {
        // the 3 x 3 neighbourhood of (p, q) in the downwind plane: columns
        // periodic in P, rows periodic or cut off in Q
        const int col[3] = {p == 0 ? NP - 1 : p - 1, p, p + 1 == NP ? 0 : p + 1};
        long long row[3];
        bool rok[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int qr = q + k - 1;
            rok[k] = true;
            if (U.qper) qr = qr < 0 ? qr + NQ : (qr >= NQ ? qr - NQ : qr);
            else rok[k] = qr >= 0 && qr < NQ;
            row[k] = (long long)md * sM + (long long)qr * sQ;
        }
#pragma unroll
        for (int d = 0; d < MAXD; ++d) {
            if (!((K.active >> d) & 1)) continue;
            const int sP = (d & 1) ? -1 : 1, sQd = (d & 2) ? -1 : 1;  // compile time after unrolling
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                // the downwind point whose corner cc is this point
                const int kp = 1 + ((cc & 1) ? sP : 0), kq = 1 + ((cc & 2) ? sQd : 0);
                if (!rok[kq]) continue;
                const long long orr = row[kq] + col[kp];
                const T bt = K.beta[d][cc];
                gx += bt * B[(long long)d * N + orr];
                gs += bt * C[(long long)d * N + orr];
            }
        }
    }
    G[off] = gx;
    G[N + off] = gs;
}

// ---------------------------------------------------------------------------
// 5. Sum over the band's units (x groups transposed), add the direct Q-step
//    terms, d/d log chi = chi d/d chi. Natural layout, one band per blockIdx.z / nz.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) adj_reduce_kernel(const SweepUnit *__restrict__ units, int u0, int u1,
                                                          int b0, const T *__restrict__ G, const T *__restrict__ direct,
                                                          const T *__restrict__ chi, T *__restrict__ g_logchi,
                                                          T *__restrict__ g_S, int nx, int ny, int nz)
{
    __shared__ T tile[2][32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int b = b0 + blockIdx.z / nz, k = blockIdx.z % nz;
    const long long N = (long long)nx * ny * nz;
    for (int c = 0; c < 2; ++c)
        for (int jj = ty; jj < 32; jj += 8) tile[c][jj][tx] = T(0);
    __syncthreads();
    for (int u = u0; u < u1; ++u) {
        if (units[u].band != b || !units[u].transposed) continue;
        const T *pg = G + (long long)(u - u0) * GRAD_CH * N + 2 * MAXD * N;
        for (int ii = ty; ii < 32; ii += 8) {
            const int i = i0 + ii, j = j0 + tx;
            if (i >= nx || j >= ny) continue;
            const long long off = ((long long)i * nz + k) * ny + j;
            tile[0][ii][tx] += pg[off];
            tile[1][ii][tx] += pg[N + off];
        }
    }
    __syncthreads();
    for (int jj = ty; jj < 32; jj += 8) {
        const int i = i0 + tx, j = j0 + jj;
        if (i >= nx || j >= ny) continue;
        const long long noff = ((long long)k * ny + j) * nx + i;
        T gx = tile[0][tx][jj], gs = tile[1][tx][jj];
        for (int u = u0; u < u1; ++u) {
            if (units[u].band != b || units[u].transposed) continue;
            const T *pg = G + (long long)(u - u0) * GRAD_CH * N + 2 * MAXD * N;
            gx += pg[noff];
            gs += pg[N + noff];
        }
        const long long bo = (long long)b * N + noff;
        gx += direct[(long long)b * 2 * N + noff];
        gs += direct[(long long)b * 2 * N + N + noff];
        g_logchi[bo] = chi[bo] * gx;
        g_S[bo] = gs;
    }
}

}  // namespace rts

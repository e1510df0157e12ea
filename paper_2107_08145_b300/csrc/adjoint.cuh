// adjoint.cuh -- reverse-mode derivative of the solve: gradients of
// L = <gI_top, I_top> + <gJ, J> + <gF, F> + <gQ, Q_rad> with respect to
// log chi and S of every band.
//
// The solve is a chain  (chi, S) -> I (per ray, by the sweep recurrence)
// -> (J_b, F_b) -> Q_rad. Its adjoint, written for this GPU layout:
//  1. qstep_adjoint_kernel: cotangents of J_b and F_b (through the Q step
//     and the band sums) and the direct chi/S terms of the Q step;
//  2. the forward sweep again, storing the converged I of every ray of a
//     band chunk (the checkpoint);
//  3. sweep_adj_kernel: the reverse sweep. For ray d the cotangent of I obeys
//     lam(p) = lam0(p) + sum_c beta_c e(r_c) lam(r_c), summed over the
//     downwind points r_c whose upwind corner c is p: the transpose of the
//     forward interpolation, run over the planes in reverse order with the
//     same tiles, ready flags and periodic-wrap bound as the forward sweep;
//  4. adj_pass1/adj_pass2: parallel over points, the derivative of each
//     segment's formal solution with respect to its opacity and source,
//     gathered onto the grid points they were interpolated from;
//  5. adj_reduce_kernel: sum over the band's sweep units, times chi for
//     d/d log chi.
#pragma once
#include "df32.cuh"
#include "sweep.cuh"

namespace rts {

// d w_up / dx and d w_p / dx of the linear-in-tau weights
__device__ __forceinline__ void seg_derivs(double x, double e, double &dwu, double &dwp)
{
    if (x < 0.01) {
        // derivatives of the Taylor series of w_up and w_p
        dwp = 0.5 - x * (2.0 / 6.0 - x * (3.0 / 24.0 - x * (4.0 / 120.0 - x * (5.0 / 720.0 - x * (6.0 / 5040.0)))));
        dwu = 0.5 - x * (4.0 / 6.0 - x * (9.0 / 24.0 - x * (16.0 / 120.0 - x * (25.0 / 720.0 - x * (36.0 / 5040.0)))));
    } else {
        const double ome = -expm1(-x);
        dwu = e / x - ome / (x * x) + e;
        dwp = ome / (x * x) - e / x;
    }
}
__device__ __forceinline__ void seg_derivs(float x, float e, float &dwu, float &dwp)
{
    if (x < 0.25f) {
        dwp = 0.5f - x * (2.f / 6.f - x * (3.f / 24.f - x * (4.f / 120.f - x * (5.f / 720.f - x * (6.f / 5040.f - x * (7.f / 40320.f))))));
        dwu = 0.5f - x * (4.f / 6.f - x * (9.f / 24.f - x * (16.f / 120.f - x * (25.f / 720.f - x * (36.f / 5040.f - x * (49.f / 40320.f))))));
    } else {
        const float r = 1.f / x;
        const float ome = 1.f - e;
        dwu = e * r - ome * r * r + e;
        dwp = ome * r * r - e * r;
    }
}

// ---------------------------------------------------------------------------
// 1. Q step adjoint (natural layout, one thread per point, loop over bands)
// ---------------------------------------------------------------------------
struct QAdjParams {
    int nx, ny, nz, nbands;
    double dx, dy, dz;
    double thin;  // min(dx, dy, dz) / tau_switch
};

// coefficient of F_z(level k) in the z part of div F at level q: central
// differences inside, first-order one-sided at the bottom and top levels,
// nothing when there is a single level
__device__ __forceinline__ double coef_z(int q, int k, int nz, double dz)
{
    if (nz == 1) return 0.0;
    if (q == 0) return k == 1 ? 1.0 / dz : (k == 0 ? -1.0 / dz : 0.0);
    if (q == nz - 1) return k == nz - 1 ? 1.0 / dz : (k == nz - 2 ? -1.0 / dz : 0.0);
    return k == q + 1 ? 0.5 / dz : (k == q - 1 ? -0.5 / dz : 0.0);
}

// Per band b and point p, with u = gQ (1 - om_b):
//   lam0 = (gJ_b, gF_b) = (gJ + gQ om_b 4 pi chi_b,  gF - D^T u)
//   direct d/dchi_b = gQ (om_b 4 pi (J_b - S_b) + dom_b/dchi_b (QJ_b - QF_b)),
//   direct d/dS_b   = -gQ om_b 4 pi chi_b,
// QJ_b = 4 pi chi_b (J_b - S_b), QF_b = -div F_b, D the divergence stencil.
template <typename T, typename Acc>
__global__ void __launch_bounds__(256) qstep_adjoint_kernel(const Acc *__restrict__ JF, const T *__restrict__ chi,
                                                             const T *__restrict__ S, const double *__restrict__ gJ,
                                                             const double *__restrict__ gF,
                                                             const double *__restrict__ gQ, QAdjParams P,
                                                             T *__restrict__ lam0, T *__restrict__ direct)
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
    const double gq = gQ ? gQ[p] : 0.0;
    for (int b = 0; b < P.nbands; ++b) {
        const T *cb = chi + (long long)b * N;
        const Acc *jf = JF + (long long)b * 4 * N;
        auto u_at = [&](long long q) -> double {
            if (!gQ) return 0.0;
            return gQ[q] * -expm1(-(double)cb[q] * P.thin);
        };
        const double c = (double)cb[p];
        const double om = exp(-c * P.thin);
        double gJb = gJ ? gJ[p] : 0.0, gchi = 0.0, gs = 0.0;
        if (gQ) {  // J_b and F_b of the forward solve are read only when Q_rad enters L
            double divz = 0.0;
            for (int q = k - 1; q <= k + 1; ++q) {
                if (q < 0 || q >= P.nz) continue;
                const double cf = coef_z(k, q, P.nz, P.dz);
                if (cf != 0.0) divz += cf * acc_to_double(jf[3 * N + (long long)q * pl + (long long)j * nx + i]);
            }
            const double qf = -((acc_to_double(jf[N + pxp]) - acc_to_double(jf[N + pxm])) * 0.5 / P.dx +
                                (acc_to_double(jf[2 * N + pyp]) - acc_to_double(jf[2 * N + pym])) * 0.5 / P.dy + divz);
            const double s = (double)S[(long long)b * N + p];
            const double Jb = acc_to_double(jf[p]);
            const double qj = four_pi * c * (Jb - s);
            gJb += gq * om * four_pi * c;
            gchi = gq * (om * four_pi * (Jb - s) - P.thin * om * (qj - qf));
            gs = -gq * om * four_pi * c;
        }
        const double gFx = (gF ? gF[p] : 0.0) + (u_at(pxp) - u_at(pxm)) * 0.5 / P.dx;
        const double gFy = (gF ? gF[N + p] : 0.0) + (u_at(pyp) - u_at(pym)) * 0.5 / P.dy;
        double dTz = 0.0;  // (D_z^T u)(k) = sum_q u(q) coef_z(q, k)
        for (int q = k - 1; q <= k + 1; ++q) {
            if (q < 0 || q >= P.nz) continue;
            const double cf = coef_z(q, k, P.nz, P.dz);
            if (cf != 0.0) dTz += u_at((long long)q * pl + (long long)j * nx + i) * cf;
        }
        const double gFz = (gF ? gF[2 * N + p] : 0.0) - dTz;
        T *l0 = lam0 + (long long)b * 4 * N;
        l0[p] = (T)gJb;
        l0[N + p] = (T)gFx;
        l0[2 * N + p] = (T)gFy;
        l0[3 * N + p] = (T)gFz;
        T *dr = direct + (long long)b * 2 * N;
        dr[p] = (T)gchi;
        dr[N + p] = (T)gs;
    }
}

// ---------------------------------------------------------------------------
// 3. Reverse sweep of one tile (cotangent lam of the rays of one unit)
// ---------------------------------------------------------------------------
// sum_c beta_c A(r_c): r_c are the downwind points whose corner c is this one
template <typename T, int SP, int SQ>
__device__ __forceinline__ T gather_down(const T *__restrict__ A, int npp, T b0, T b1, T b2, T b3)
{
    const int oq = SQ * npp;
    return b0 * A[0] + b1 * A[SP] + b2 * A[oq] + b3 * A[oq + SP];
}
// forward-upwind interpolation (corners at -SP, -SQ)
template <typename T, int SP, int SQ>
__device__ __forceinline__ T interp_up(const T *__restrict__ X, int npp, T b0, T b1, T b2, T b3)
{
    const int oq = -SQ * npp;
    return b0 * X[0] + b1 * X[-SP] + b2 * X[oq] + b3 * X[oq - SP];
}

enum { FA_A0 = 0, FA_GU = 4, FA_GD = 5, NPARF_A = 6, NFIELD_A = 2 * NPARF_A + 2 };

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
    T *const lstore = a.store + (long long)(uidx - a.unit_base) * 4 * N;
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
    T *const sm = (T *)smem;
    auto fA = [&](int par, int f) -> T * { return sm + (par * NPARF_A + f) * FL; };
    auto fX = [&](int t) -> T * { return sm + (2 * NPARF_A + (t & 1)) * FL; };

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
        D.bck[d] = 0;
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

    auto put = [&](T *f, int k, T v) {
        f[k * npp + c] = v;
        if (p == 0) f[k * npp + NP + 1] = v;
        if (p == NP - 1) f[k * npp] = v;
    };
    // chi rows of reverse step t into slot t & 1
    auto prefetch = [&](int t) {
        if (act) {
            const long long mo = (long long)plane_of(t, NM, msa) * sM + p;
            T *dx = fX(t);
            for (int k = 0; k < nrows + 2; ++k) {
                const int q = s_q[k];
                if (q < 0) { put(dx, k, T(0)); continue; }
                const T *gx = chi + mo + (long long)q * sQ;
                cp_async(dx + k * npp + c, gx);
                if (p == 0) cp_async(dx + k * npp + NP + 1, gx);
                if (p == NP - 1) cp_async(dx + k * npp, gx);
            }
        }
        cp_async_commit();
    };

    __syncthreads();
    // prologue: the (downwind) plane before the first reverse step carries
    // A = 0; for the periodic groups that is the seed, with a unit bound on
    // the points that are not set. Rows outside a non-periodic Q range stay
    // zero in both parities for the whole sweep.
    if (act) {
        for (int par = 0; par < 2; ++par)
            for (int k = 0; k < nrows + 2; ++k) {
                const int q = s_q[k];
                for (int d = 0; d < MAXD; ++d) put(fA(par, FA_A0 + d), k, T(0));
                T gu = 0, gd = 0;
                if (par == 1 && wrap && q >= 0) {
                    if (q != 0) gu = 1;
                    if (q != NQ - 1) gd = 1;
                }
                put(fA(par, FA_GU), k, gu);
                put(fA(par, FA_GD), k, gd);
            }
    }
    prefetch(0);
    prefetch(1);
    cp_async_wait_all();
    __syncthreads();

    int t_acc = wrap ? -1 : 0;
    const int warm_cap = a.max_periods * NM + a.L;
    const int dec_thread = NT > 32 ? 32 : 0;

    for (int t = 0;; ++t) {
        const int m = plane_of(t, NM, msa);
        const int cur = t & 1, prv = cur ^ 1;
        if (t_acc < 0 && s_ctl[1]) {
            t_acc = t;
            if (r == 0 && tid == 0) a.unit_tacc[uidx] = t;
        }
        if (wrap && t_acc < 0 && t >= warm_cap) {
            if (tid == 0) atomicOr(a.status, ST_NOCONV);
            return;
        }
        const bool acc = t_acc >= 0;
        const bool last = acc && (t - t_acc == NM - 1);
        T b[MAXD][4], hds[MAXD];
#pragma unroll
        for (int d = 0; d < MAXD; ++d) {
            hds[d] = D.hds[d];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) b[d][cc] = D.beta[d][cc];
        }
        const T *Xc = fX(t), *Xn = fX(t + 1);  // chi of this plane and of its forward-upwind plane
        // a z group's last reverse plane is its boundary layer (set points)
        const bool bnd_plane = !wrap && t == NM - 1;
        const bool top_plane = axis == 2 && t == 0 && sa > 0;
        float gmax = 0.f;

        auto do_row = [&](int k) {
            const int q = q0 + k - 1;
            const int o = k * npp + c;
            const long long goff = (long long)m * sM + (long long)q * sQ + p;
            const T gJ = l0[goff], gFx = l0[N + goff], gFy = l0[2 * N + goff], gFz = l0[3 * N + goff];
            const bool top = axis == 2 ? top_plane : q == NQ - 1;
            T lam[MAXD];
            lam[0] = gather_down<T, 1, 1>(fA(prv, FA_A0 + 0) + o, npp, b[0][0], b[0][1], b[0][2], b[0][3]);
            lam[1] = gather_down<T, -1, 1>(fA(prv, FA_A0 + 1) + o, npp, b[1][0], b[1][1], b[1][2], b[1][3]);
            lam[2] = gather_down<T, 1, -1>(fA(prv, FA_A0 + 2) + o, npp, b[2][0], b[2][1], b[2][2], b[2][3]);
            lam[3] = gather_down<T, -1, -1>(fA(prv, FA_A0 + 3) + o, npp, b[3][0], b[3][1], b[3][2], b[3][3]);
            float gu = 0.f, gd = 0.f;
            if (!acc) {
                const float g0 = (float)gather_down<T, 1, 1>(fA(prv, D.up[0] ? FA_GU : FA_GD) + o, npp, b[0][0], b[0][1], b[0][2], b[0][3]);
                const float g1 = (float)gather_down<T, -1, 1>(fA(prv, D.up[1] ? FA_GU : FA_GD) + o, npp, b[1][0], b[1][1], b[1][2], b[1][3]);
                const float g2 = (float)gather_down<T, 1, -1>(fA(prv, D.up[2] ? FA_GU : FA_GD) + o, npp, b[2][0], b[2][1], b[2][2], b[2][3]);
                const float g3 = (float)gather_down<T, -1, -1>(fA(prv, D.up[3] ? FA_GU : FA_GD) + o, npp, b[3][0], b[3][1], b[3][2], b[3][3]);
                gu = fmaxf(fmaxf(D.up[0] ? g0 : 0.f, D.up[1] ? g1 : 0.f), fmaxf(D.up[2] ? g2 : 0.f, D.up[3] ? g3 : 0.f));
                gd = fmaxf(fmaxf(D.up[0] ? 0.f : g0, D.up[1] ? 0.f : g1), fmaxf(D.up[2] ? 0.f : g2, D.up[3] ? 0.f : g3));
            }
            const T xp = Xc[o];
            T Aout[MAXD];
            float egu = 0.f, egd = 0.f;
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                // direct cotangent of this ray's intensity at this point
                lam[d] += D.cJ[d] * gJ + D.cF[0][d] * gFx + D.cF[1][d] * gFy + D.cF[2][d] * gFz;
                if (gitop && top && D.up[d] && D.active[d]) {
                    int i, j;
                    natural_ij(axis, p, q, m, i, j);
                    lam[d] += gitop[((long long)D.udx[d] * uny + j) * unx + i];
                }
                if (!D.active[d]) lam[d] = T(0);
                const bool set = wrap ? (D.up[d] ? q == 0 : q == NQ - 1) : bnd_plane;
                T e = T(0);
                if (!set) {
                    T xup;
                    if (d == 0) xup = interp_up<T, 1, 1>(Xn + o, npp, b[0][0], b[0][1], b[0][2], b[0][3]);
                    else if (d == 1) xup = interp_up<T, -1, 1>(Xn + o, npp, b[1][0], b[1][1], b[1][2], b[1][3]);
                    else if (d == 2) xup = interp_up<T, 1, -1>(Xn + o, npp, b[2][0], b[2][1], b[2][2], b[2][3]);
                    else xup = interp_up<T, -1, -1>(Xn + o, npp, b[3][0], b[3][1], b[3][2], b[3][3]);
                    T wu, wp;
                    seg_weights(hds[d] * (xup + xp), e, wu, wp);
                }
                Aout[d] = e * lam[d];
                if (!acc) {
                    if (D.up[d]) egu = fmaxf(egu, (float)e); else egd = fmaxf(egd, (float)e);
                }
            }
            // the bound carried to the upwind plane: e * g (max over the rays of each set)
            gu *= egu;
            gd *= egd;
            if (wrap && q == 0) gu = 0.f;
            if (wrap && q == NQ - 1) gd = 0.f;
#pragma unroll
            for (int d = 0; d < MAXD; ++d) put(fA(cur, FA_A0 + d), k, Aout[d]);
            if (!acc) {
                put(fA(cur, FA_GU), k, (T)gu);
                put(fA(cur, FA_GD), k, (T)gd);
                gmax = fmaxf(gmax, fmaxf(gu, gd));
            } else {
#pragma unroll
                for (int d = 0; d < MAXD; ++d) lstore[(long long)d * N + goff] = lam[d];
            }
            if (k == 1 || k == nrows) {
                for (int sd = 0; sd < 2; ++sd) {
                    if (!((sd == 0 && k == 1) || (sd == 1 && k == nrows))) continue;
                    T *dst = myhalo + ((long long)(cur * 2 + sd) * HALO_CH) * NP + p;
                    for (int d = 0; d < MAXD; ++d) dst[(long long)d * NP] = Aout[d];
                    if (!acc) {
                        dst[(long long)MAXD * NP] = (T)gu;
                        dst[(long long)(MAXD + 1) * NP] = (T)gd;
                    }
                }
            }
        };

        if (act) {
#pragma unroll 1
            for (int k = 2; k < nrows; ++k) do_row(k);
        }
        if (t > 0 && act) {
            bool ok = true;
            if (has_lower) ok = wait_flag_geq(a.flags + tile0 + lower, t, a.status, a.timeout_ns);
            if (ok && has_upper) ok = wait_flag_geq(a.flags + tile0 + upper, t, a.status, a.timeout_ns);
            if (!ok) {
                s_ctl[0] = 1;
            } else {
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
#pragma unroll
                    for (int d = 0; d < MAXD; ++d) put(fA(prv, FA_A0 + d), row, hv[d]);
                    if (!acc) {
                        put(fA(prv, FA_GU), row, hv[MAXD]);
                        put(fA(prv, FA_GD), row, hv[MAXD + 1]);
                    }
                }
            }
        }
        __syncthreads();  // B1
        if (s_ctl[0]) {
            cp_async_wait_all();
            return;
        }
        if (act) {
            do_row(1);
            if (nrows > 1) do_row(nrows);
        }
        if (!acc) {
            for (int o = 16; o; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
            if (lane == 0) s_wmax[warp] = gmax;
        }
        if (tid == dec_thread && t_acc < 0 && t + 1 - a.L >= 0) {
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
        __syncthreads();  // B2: plane t complete; chi of plane t no longer read
        if (tid == 0) {
            st_release(a.flags + gt, t + 1);
            if (!acc) {
                float g = 0.f;
                for (int w = 0; w < (NT + 31) / 32; ++w) g = fmaxf(g, s_wmax[w]);
                const int slot = t % a.R;
                const unsigned long long pv = ((unsigned long long)(unsigned)(t + 1) << 32) | __float_as_uint(g);
                atomicMax(a.gmax + (long long)uidx * a.R + slot, pv);
                red_release_add(a.gcnt + (long long)uidx * a.R + slot, 1u);
            }
        }
        if (s_ctl[0]) return;
        if (last) break;
        // chi of plane t+2 into the slot of plane t; needed across columns at
        // step t+1, so wait and synchronise before it is read
        prefetch(t + 2);
        cp_async_wait_all();
        __syncthreads();
    }
}

template <typename T, int TQ>
__global__ void __launch_bounds__(1024) sweep_adj_kernel(SweepArgs<T> a)
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
        run_tile_adj<T, TQ>(a, a.units + u, u, tile - a.units[u].tile0, tile, smem);
    }
}

// ---------------------------------------------------------------------------
// 4. Gradient of each segment, gathered to the grid (parallel over points)
// ---------------------------------------------------------------------------
template <typename T>
struct GradArgs {
    const SweepUnit *units;
    int unit_base;
    const T *chi, *S, *chiT, *ST;
    const T *I;       // stored forward I, [units][4][N]
    T *LB;            // in: lam [units][4][N]; pass 1 turns it into B = dL/d dtau * ds/2
    T *C;             // [units][4][N]: lam * w_up
    T *G;             // [units][2][N]: own terms (pass 1), then the gradients (pass 2)
    int bc_bottom, bc_top;
};

// point (p, q, m) of a unit, one thread per p; blockIdx.y = q, blockIdx.z = m + NM * (u - unit_base)
template <typename T>
__global__ void __launch_bounds__(128) adj_pass1_kernel(GradArgs<T> g, int maxNM)
{
    const int uu = blockIdx.z / maxNM, m = blockIdx.z % maxNM;
    const SweepUnit &U = g.units[g.unit_base + uu];
    const int NP = U.NP, NQ = U.NQ, NM = U.NM;
    const int p = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
    if (m >= NM || q >= NQ || p >= NP) return;
    const long long N = U.N, sQ = U.sQ, sM = U.sM;
    const T *chi = (U.transposed ? g.chiT : g.chi) + U.in_off;
    const T *S = (U.transposed ? g.ST : g.S) + U.in_off;
    const T *I = g.I + (long long)uu * 4 * N;
    T *LB = g.LB + (long long)uu * 4 * N;
    T *C = g.C + (long long)uu * 4 * N;
    T *G = g.G + (long long)uu * 2 * N;
    const long long off = (long long)m * sM + (long long)q * sQ + p;
    const int mu = U.wrap ? (m - U.sa + NM) % NM : m - U.sa;  // forward-upwind plane
    const bool zbnd = !U.wrap && (mu < 0 || mu >= NM);
    T own_chi = 0, own_S = 0;
    for (int d = 0; d < MAXD; ++d) {
        const T lam = LB[(long long)d * N + off];
        T Bv = 0, Cv = 0;
        const int sP = (d & 1) ? -1 : 1, sQd = (d & 2) ? -1 : 1;
        const bool set = U.wrap ? (U.up[d] ? q == 0 : q == NQ - 1) : zbnd;
        if (!U.active[d]) {
        } else if (set) {
            const int kind = U.up[d] ? g.bc_bottom : g.bc_top;
            if (kind == 1) own_S += lam;  // I = S on the boundary layer
        } else {
            T Iup = 0, Sup = 0, Xup = 0;
            for (int cc = 0; cc < 4; ++cc) {
                int pc = p - ((cc & 1) ? sP : 0);
                pc = (pc + NP) % NP;
                int qc = q - ((cc & 2) ? sQd : 0);
                if (U.qper) qc = (qc + NQ) % NQ;
                const long long oc = (long long)mu * sM + (long long)qc * sQ + pc;
                const T bt = (T)U.beta[d][cc];
                Iup += bt * I[(long long)d * N + oc];
                Sup += bt * S[oc];
                Xup += bt * chi[oc];
            }
            const T hds = (T)(0.5 * U.ds[d]);
            const T x = hds * (Xup + chi[off]);
            T e, wu, wp, dwu, dwp;
            seg_weights(x, e, wu, wp);
            seg_derivs(x, e, dwu, dwp);
            const T gdt = lam * (-e * Iup + dwu * Sup + dwp * S[off]);
            Bv = gdt * hds;
            Cv = lam * wu;
            own_chi += Bv;
            own_S += lam * wp;
        }
        LB[(long long)d * N + off] = Bv;
        C[(long long)d * N + off] = Cv;
    }
    G[off] = own_chi;
    G[N + off] = own_S;
}

template <typename T>
__global__ void __launch_bounds__(128) adj_pass2_kernel(GradArgs<T> g, int maxNM)
{
    const int uu = blockIdx.z / maxNM, m = blockIdx.z % maxNM;
    const SweepUnit &U = g.units[g.unit_base + uu];
    const int NP = U.NP, NQ = U.NQ, NM = U.NM;
    const int p = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
    if (m >= NM || q >= NQ || p >= NP) return;
    const long long N = U.N, sQ = U.sQ, sM = U.sM;
    const T *B = g.LB + (long long)uu * 4 * N;
    const T *C = g.C + (long long)uu * 4 * N;
    T *G = g.G + (long long)uu * 2 * N;
    const long long off = (long long)m * sM + (long long)q * sQ + p;
    const int md = U.wrap ? (m + U.sa + NM) % NM : m + U.sa;  // forward-downwind plane
    T gx = G[off], gs = G[N + off];
    if (md >= 0 && md < NM) {
        for (int d = 0; d < MAXD; ++d) {
            if (!U.active[d]) continue;
            const int sP = (d & 1) ? -1 : 1, sQd = (d & 2) ? -1 : 1;
            for (int cc = 0; cc < 4; ++cc) {
                // the downwind point whose corner cc is this point
                int pr = p + ((cc & 1) ? sP : 0);
                pr = (pr + NP) % NP;
                int qr = q + ((cc & 2) ? sQd : 0);
                if (U.qper) qr = (qr + NQ) % NQ;
                else if (qr < 0 || qr >= NQ) continue;
                const long long orr = (long long)md * sM + (long long)qr * sQ + pr;
                const T bt = (T)U.beta[d][cc];
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
        const T *pg = G + (long long)(u - u0) * 2 * N;
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
            const T *pg = G + (long long)(u - u0) * 2 * N;
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

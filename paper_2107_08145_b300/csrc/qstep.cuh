// qstep.cuh -- the paper's flux() step (Sect. 5.1: "from the specific
// intensity calculate the average intensity and radiative fluxes", and the
// radiative heating/cooling fed back to the MHD), plus the transpose that
// lets x-dominant sweeps read unit-stride planes (Sect. 5.3.1).
//
//   J_b  = sum over the band's sweep units of their partial sums (w_d I_d)
//   F_b  = same for the 4 pi w_d n_d I_d partials
//   Q_b  = om_b 4 pi chi_b (J_b - S_b) + (1 - om_b)(-div F_b)
//   om_b = exp(-chi_b min(dx,dy,dz) / tau_switch)
//   J = sum_b J_b, F = sum_b F_b, Q_rad = sum_b Q_b
// The divergence uses central differences, periodic in x and y, first-order
// one-sided at k = 0 and k = Nz-1. The arithmetic type Acc is double (FP64)
// or df32 (compensated two-FP32); outputs are written as double.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "df32.cuh"

namespace rts {

// out[b][i][k][j] = in[b][k][j][i] for the 32 x 32 (i, j) tile at (i0, j0)
// of level k of band b
template <typename T>
__device__ __forceinline__ void transpose_tile(const T *__restrict__ in, T *__restrict__ out, int nx, int ny, int nz,
                                               int i0, int j0, long long b, long long k)
{
    __shared__ T tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const T *src = in + (b * nz + k) * (long long)ny * nx;
    for (int jj = ty; jj < 32; jj += 8) {
        const int i = i0 + tx, j = j0 + jj;
        if (i < nx && j < ny) tile[jj][tx] = src[(long long)j * nx + i];
    }
    __syncthreads();
    for (int ii = ty; ii < 32; ii += 8) {
        const int i = i0 + ii, j = j0 + tx;
        if (i < nx && j < ny) out[((b * nx + i) * nz + k) * (long long)ny + j] = tile[tx][ii];
    }
}

// the same tile of two arrays at once (chi and S: all 8 loads of a thread
// in flight together, one launch for both). Every input value passes here
// once per solve, so this is also where non-finite chi or S is detected:
// ST_NONFINITE in *status (the solve still runs; rts_check reports it).
template <typename T>
__device__ __forceinline__ void transpose_tile2(const T *__restrict__ in0, const T *__restrict__ in1,
                                                T *__restrict__ out0, T *__restrict__ out1, int nx, int ny, int nz,
                                                int i0, int j0, long long b, long long k, int *status)
{
    __shared__ T tile[2][32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const long long so = (b * nz + k) * (long long)ny * nx;
    bool bad = false;
#pragma unroll
    for (int jj = ty; jj < 32; jj += 8) {
        const int i = i0 + tx, j = j0 + jj;
        if (i < nx && j < ny) {
            const T c = in0[so + (long long)j * nx + i], s = in1[so + (long long)j * nx + i];
            tile[0][jj][tx] = c;
            tile[1][jj][tx] = s;
            bad = bad || !isfinite(c) || !isfinite(s);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
    __syncthreads();
#pragma unroll
    for (int ii = ty; ii < 32; ii += 8) {
        const int i = i0 + ii, j = j0 + tx;
        if (i < nx && j < ny) {
            const long long o = ((b * nx + i) * nz + k) * (long long)ny + j;
            out0[o] = tile[0][tx][ii];
            out1[o] = tile[1][tx][ii];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) transpose_x2_kernel(const T *__restrict__ in0, const T *__restrict__ in1,
                                                             T *__restrict__ out0, T *__restrict__ out1, int nx,
                                                             int ny, int nz, int *status)
{
    const long long bk = blockIdx.z;
    transpose_tile2(in0, in1, out0, out1, nx, ny, nz, blockIdx.x * 32, blockIdx.y * 32, bk / nz, bk % nz, status);
}

// The non-finite check alone, for grids whose solve needs no transposed
// copy: every value of chi and S once, a grid-stride loop.
template <typename T>
__global__ void __launch_bounds__(256) check_finite_kernel(const T *__restrict__ a, const T *__restrict__ b,
                                                             long long n, int *status)
{
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        bad = bad || !isfinite(a[i]) || !isfinite(b[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

// four values moved as one element (the adjoint's lam0 of a point)
template <typename T>
struct __align__(16) Vec4 {
    T v[4];
};

template <typename T>
__global__ void __launch_bounds__(256) transpose_x_kernel(const T *__restrict__ in, T *__restrict__ out,
                                                            int nx, int ny, int nz)
{
    const long long bk = blockIdx.z;
    transpose_tile(in, out, nx, ny, nz, blockIdx.x * 32, blockIdx.y * 32, bk / nz, bk % nz);
}

struct RedUnit {
    const void *partial;  // [N][4] in the unit's layout
    int axis;             // 0: transposed layout [i][k][j]; else natural
    // raw partials (the slot intensities I_0..I_3 of a point, from
    // sweep_reg_kernel): J = sum_d c[0][d] I_d and F_x, F_y, F_z with
    // c[1..3][d] = 4 pi w_d n_d; qpair[c] selects the slot pairing of the
    // exact differences (0: (0,1)+(2,3), 1: (0,2)+(1,3))
    float c[4][4];
    int qpair[4];
};

// a x + b y with one rounding relative to the result, however much the two
// products cancel: p = b y rounded, b y - p exactly (FMA), a x + p rounded
__device__ __forceinline__ float pair_sum(float a, float x, float b, float y)
{
    const float p = b * y;
    return fmaf(a, x, p) + fmaf(b, y, -p);
}

// J, F_x, F_y, F_z of one point of one unit from its 4 slot intensities. The
// flux components across the unit's dominant axis cancel between slots of
// opposite sign; they are summed as two exact pair differences (the pairs of
// slots that differ only in that component's sign), so their error is
// relative to the component itself.
__device__ __forceinline__ void unit_moments(const RedUnit &u, const float (&I)[4], float (&v)[4])
{
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float *k = u.c[c];
        v[c] = u.qpair[c] ? pair_sum(k[0], I[0], k[2], I[2]) + pair_sum(k[1], I[1], k[3], I[3])
                          : pair_sum(k[0], I[0], k[1], I[1]) + pair_sum(k[2], I[2], k[3], I[3]);
    }
}
__device__ __forceinline__ void unit_moments(const RedUnit &, const double (&I)[4], double (&v)[4])
{
    for (int c = 0; c < 4; ++c) v[c] = I[c];  // FP64 partials are never raw
}

// Sums of sweep-unit partials. FP32 partials are summed in double-float
// arithmetic (error-free TwoSum), which for a handful of terms is exact to
// ~2^-48 relative; the FP64 form of that sum is then taken once. This keeps
// the FP64 pipe (a small fraction of the FP32 rate on B300) out of the loop.
template <typename T>
struct PartSum;
template <>
struct PartSum<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ double as_double() const { return v; }
    __device__ __forceinline__ df32 as_df32() const { return {(float)v, (float)(v - (double)(float)v)}; }
};
template <>
struct PartSum<float> {
    df32 v = {0.f, 0.f};
    __device__ __forceinline__ void add(float x) { v = df_add(v, x); }
    __device__ __forceinline__ void add(df32 x) { v = df_add(v, x); }
    __device__ __forceinline__ double as_double() const { return df_to_double(v); }
    __device__ __forceinline__ df32 as_df32() const { return v; }
};
__device__ __forceinline__ double part_out(const PartSum<double> &s, double *) { return s.as_double(); }
__device__ __forceinline__ double part_out(const PartSum<float> &s, double *) { return s.as_double(); }
__device__ __forceinline__ df32 part_out(const PartSum<float> &s, df32 *) { return s.as_df32(); }

// the 4 partial sums of one point (16 / 32 bytes, aligned)
__device__ __forceinline__ void ld_part(const float *p, float (&v)[4])
{
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld_part(const double *p, double (&v)[4])
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p + 2));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// JF[b][c][N] (c = J, Fx, Fy, Fz) from the band's sweep-unit partials. A CTA
// covers a 32 x 32 (i, j) tile of one level k of one band. Units in natural
// layout are read along i; units of the x groups, stored [i][k][j], are read
// along j into a shared tile and summed transposed, so every global read is
// coalesced.
// sums for the 32 x 32 (i, j) tile at (i0, j0) of level k, units u0..u1-1 of
// one band, into JFb = JF of that band ([4][N])
template <typename T, typename Acc>
__device__ __forceinline__ void reduce_tile(const RedUnit *__restrict__ ru, int u0, int u1, Acc *__restrict__ JFb,
                                            int nx, int ny, int nz, int i0, int j0, int k, bool raw)
{
    __shared__ PartSum<T> tile[4][32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const long long N = (long long)nx * ny * nz;
    // transposed units: tile[c][i - i0][j - j0]
    for (int c = 0; c < 4; ++c)
        for (int jj = ty; jj < 32; jj += 8) tile[c][jj][tx] = PartSum<T>();
    __syncthreads();
    for (int u = u0; u < u1; ++u) {
        if (ru[u].axis != 0) continue;
        const T *pt = (const T *)ru[u].partial;
        for (int ii = ty; ii < 32; ii += 8) {
            const int i = i0 + ii, j = j0 + tx;
            if (i >= nx || j >= ny) continue;
            const long long off = ((long long)i * nz + k) * ny + j;
            T v[4];
            ld_part(pt + off * 4, v);
            if (raw) {
                T I[4] = {v[0], v[1], v[2], v[3]};
                unit_moments(ru[u], I, v);
            }
            for (int c = 0; c < 4; ++c) tile[c][ii][tx].add(v[c]);
        }
    }
    __syncthreads();
    for (int jj = ty; jj < 32; jj += 8) {
        const int i = i0 + tx, j = j0 + jj;
        if (i >= nx || j >= ny) continue;
        const long long noff = ((long long)k * ny + j) * nx + i;
        PartSum<T> s[4];
        for (int c = 0; c < 4; ++c) s[c] = tile[c][tx][jj];
        for (int u = u0; u < u1; ++u) {
            if (ru[u].axis == 0) continue;
            const T *pn = (const T *)ru[u].partial;
            T v[4];
            ld_part(pn + noff * 4, v);
            if (raw) {
                T I[4] = {v[0], v[1], v[2], v[3]};
                unit_moments(ru[u], I, v);
            }
            for (int c = 0; c < 4; ++c) s[c].add(v[c]);
        }
        for (int c = 0; c < 4; ++c) JFb[c * N + noff] = part_out(s[c], (Acc *)nullptr);
    }
}

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) reduce_units_kernel(const RedUnit *__restrict__ ru,
                                                            const int *__restrict__ ru_begin,
                                                            Acc *__restrict__ JF, int nx, int ny, int nz, int raw)
{
    const int b = blockIdx.z / nz, k = blockIdx.z % nz;
    const long long N = (long long)nx * ny * nz;
    reduce_tile<T, Acc>(ru, ru_begin[b], ru_begin[b + 1], JF + (long long)b * 4 * N, nx, ny, nz, blockIdx.x * 32,
                        blockIdx.y * 32, k, raw != 0);
}

struct QParams {
    int nx, ny, nz, nbands;
    double inv2dx, inv2dy, inv2dz, invdz;   // stencil coefficients
    double thin;                            // min(dx,dy,dz) / tau_switch
};

__device__ __forceinline__ void blend_weights(double chi, double thin, double &om, double &omc)
{
    const double x = chi * thin;
    om = exp(-x);
    omc = -expm1(-x);
}
__device__ __forceinline__ void blend_weights(float chi, float thin, float &om, float &omc)
{
    const float x = chi * thin;
    om = expf(-x);
    omc = -expm1f(-x);
}

__device__ __forceinline__ double accT(double *, double v) { return v; }
__device__ __forceinline__ double accT(double *, float v) { return (double)v; }
__device__ __forceinline__ df32 accT(df32 *, float v) { return df_make(v); }

// Accumulator of the Q step at one point over the bands, in band order: the
// band sums J, F and Q_rad = sum_b [om_b 4 pi chi_b (J_b - S_b) +
// (1 - om_b)(-div F_b)]. add() takes band b's J_b, its own F_b and the six
// neighbour values of the divergence (x+-1, y+-1, z+ / z-, with cz the z
// coefficient: central, one-sided at the bottom and top levels).
template <typename T, typename Acc>
struct QAccum {
    Acc Jt, Fx, Fy, Fz, Qt, cx, cy, cz, four_pi;
    T thin;
    __device__ __forceinline__ QAccum(const QParams &P, Acc czv)
    {
        Acc *tag = nullptr;
        Jt = Fx = Fy = Fz = Qt = acc_zero(tag);
        cx = acc_from(tag, P.inv2dx);
        cy = acc_from(tag, P.inv2dy);
        cz = czv;
        four_pi = acc_from(tag, 12.566370614359172953850573533118);
        thin = (T)P.thin;
    }
    __device__ __forceinline__ void add(Acc Jb, Acc fx, Acc fy, Acc fz, Acc fxp, Acc fxm, Acc fyp, Acc fym, Acc fzp,
                                        Acc fzm, T c, T s)
    {
        Acc *tag = nullptr;
        const Acc dvx = acc_mul(acc_sub(fxp, fxm), cx);
        const Acc dvy = acc_mul(acc_sub(fyp, fym), cy);
        const Acc dvz = acc_mul(acc_sub(fzp, fzm), cz);
        const Acc negdiv = acc_sub(acc_zero(tag), acc_add(acc_add(dvx, dvy), dvz));
        const Acc qj = acc_mul(acc_mul(four_pi, accT(tag, c)), acc_sub(Jb, accT(tag, s)));
        T om, omc;
        blend_weights(c, thin, om, omc);
        const Acc qb = acc_add(acc_mul(accT(tag, om), qj), acc_mul(accT(tag, omc), negdiv));
        Jt = acc_add(Jt, Jb);
        Fx = acc_add(Fx, fx);
        Fy = acc_add(Fy, fy);
        Fz = acc_add(Fz, fz);
        Qt = acc_add(Qt, qb);
    }
    __device__ __forceinline__ void store(double *J, double *F, double *Q, long long p, long long N) const
    {
        if (J) J[p] = acc_to_double(Jt);
        if (F) {
            F[p] = acc_to_double(Fx);
            F[N + p] = acc_to_double(Fy);
            F[2 * N + p] = acc_to_double(Fz);
        }
        if (Q) Q[p] = acc_to_double(Qt);
    }
};

// FP32 sweep with the FP64 Q step: FP64 for the cancelling parts -- the band
// and direction sums, J_b - S_b, the flux differences and their sum, and the
// sum of Q over bands; the products with chi and the blend weights (no
// cancellation) in FP32, which B300 runs at many times its FP64 rate.
template <>
struct QAccum<float, double> {
    double Jd, Fxd, Fyd, Fzd, Qd, dcx, dcy, dcz;
    float thin_f;
    __device__ __forceinline__ QAccum(const QParams &P, double czv)
    {
        Jd = Fxd = Fyd = Fzd = Qd = 0.0;
        dcx = P.inv2dx;
        dcy = P.inv2dy;
        dcz = czv;
        thin_f = (float)P.thin;
    }
    __device__ __forceinline__ void add(double Jb, double fx, double fy, double fz, double fxp, double fxm,
                                        double fyp, double fym, double fzp, double fzm, float c, float sv)
    {
        const float four_pi_f = 12.566370614359172953850573533118f;
        Jd += Jb;
        Fxd += fx;
        Fyd += fy;
        Fzd += fz;
        const double div = (fxp - fxm) * dcx + (fyp - fym) * dcy + (fzp - fzm) * dcz;
        const float dJ = (float)(Jb - (double)sv);
        float om, omc;
        blend_weights(c, thin_f, om, omc);
        Qd += (double)(om * (four_pi_f * c * dJ) + omc * (float)(-div));
    }
    __device__ __forceinline__ void store(double *J, double *F, double *Q, long long p, long long N) const
    {
        if (J) J[p] = Jd;
        if (F) {
            F[p] = Fxd;
            F[N + p] = Fyd;
            F[2 * N + p] = Fzd;
        }
        if (Q) Q[p] = Qd;
    }
};

// z coefficient of the divergence at level k
template <typename Acc>
__device__ __forceinline__ Acc z_coef(const QParams &P, int k)
{
    Acc *tag = nullptr;
    if (P.nz == 1) return acc_zero(tag);
    if (k == 0 || k == P.nz - 1) return acc_from(tag, P.invdz);
    return acc_from(tag, P.inv2dz);
}

// Q step at point (i, j, k) of one grid (pointers at that grid's data)
template <typename T, typename Acc>
__device__ __forceinline__ void qstep_point(const Acc *__restrict__ JF, const T *__restrict__ chi,
                                            const T *__restrict__ S, const QParams &P, double *__restrict__ J,
                                            double *__restrict__ F, double *__restrict__ Q, int i, int j, int k)
{
    if (i >= P.nx || j >= P.ny) return;
    const long long nx = P.nx, ny = P.ny, nz = P.nz;
    const long long N = nx * ny * nz;
    const long long p = ((long long)k * ny + j) * nx + i;
    const long long xp = p - i + (i + 1 == nx ? 0 : i + 1), xm = p - i + (i == 0 ? nx - 1 : i - 1);
    const long long yp = p + ((j + 1 == ny ? 0 : j + 1) - j) * nx, ym = p + ((j == 0 ? ny - 1 : j - 1) - j) * nx;
    long long zp, zm;
    if (nz == 1) { zp = zm = p; }
    else if (k == 0) { zp = p + nx * ny; zm = p; }
    else if (k == nz - 1) { zp = p; zm = p - nx * ny; }
    else { zp = p + nx * ny; zm = p - nx * ny; }
    QAccum<T, Acc> qa(P, z_coef<Acc>(P, k));
    for (int b = 0; b < P.nbands; ++b) {
        const Acc *jf = JF + (long long)b * 4 * N;
        qa.add(jf[p], jf[N + p], jf[2 * N + p], jf[3 * N + p], jf[N + xp], jf[N + xm], jf[2 * N + yp],
               jf[2 * N + ym], jf[3 * N + zp], jf[3 * N + zm], chi[(long long)b * N + p], S[(long long)b * N + p]);
    }
    qa.store(J, F, Q, p, N);
}

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) qstep_kernel(const Acc *__restrict__ JF, const T *__restrict__ chi,
                                                     const T *__restrict__ S, QParams P,
                                                     double *__restrict__ J, double *__restrict__ F,
                                                     double *__restrict__ Q)
{
    qstep_point<T, Acc>(JF, chi, S, P, J, F, Q, blockIdx.x * 32 + threadIdx.x, blockIdx.y * 8 + threadIdx.y,
                        blockIdx.z);
}

}  // namespace rts

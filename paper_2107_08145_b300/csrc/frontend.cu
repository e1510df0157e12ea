// frontend.cu -- the RTS input step (the paper's "Interpolate", Sect. 2:
// trilinear interpolation of the MHD variables from the MHD grid to the
// staggered RTS grid, then the source function and opacities of every band).
//
// For every RTS point (i, j, k) and band b:
//   position on the MHD grid      u = (i + sx, j + sy, k + sz)  (cell units)
//   trilinear in ln T and ln rho  from the 8 MHD cells around u (periodic in
//                                 x, y; clamped to the first / last layer in z)
//   ln kappa_b                    bilinear in the (ln T, ln rho) table
//   chi_b = exp(ln kappa_b) rho,  S_b = exp(ln B_b(ln T)), ln B_b linear in ln T
// Table coordinates outside the table are clamped to its edge. One thread per
// RTS point; the tables are read through the read-only cache.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "rts.h"

namespace {

struct FrontArgs {
    int nx, ny, nz, nb, nT, nR;
    double sx, sy, sz;         // RTS point (0,0,0) on the MHD grid, in cells
    double lnT0, dlnT, lnR0, dlnR;
};

// clamped cell and weight of coordinate x on a grid of n nodes (0 .. n-1)
__device__ __forceinline__ void node_weight(double x, int n, int &i0, double &w)
{
    if (!(x > 0.0)) { i0 = 0; w = 0.0; return; }
    if (x >= (double)(n - 1)) { i0 = n > 1 ? n - 2 : 0; w = n > 1 ? 1.0 : 0.0; return; }
    i0 = (int)floor(x);
    w = x - i0;
}

template <typename T>
__global__ void __launch_bounds__(256) front_end_kernel(FrontArgs A, const T *__restrict__ Tm,
                                                          const T *__restrict__ rho, const T *__restrict__ lnk,
                                                          const T *__restrict__ lnB, T *__restrict__ chi,
                                                          T *__restrict__ S)
{
    const long long nxy = (long long)A.nx * A.ny, N = nxy * A.nz;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int i = (int)(p % A.nx), j = (int)((p / A.nx) % A.ny), k = (int)(p / nxy);
    // the 8 MHD cells around the point
    const double ux = i + A.sx, uy = j + A.sy, uz = k + A.sz;
    const double fx = floor(ux), fy = floor(uy);
    const double wx = ux - fx, wy = uy - fy;
    int x0 = (int)fx % A.nx, y0 = (int)fy % A.ny;
    if (x0 < 0) x0 += A.nx;
    if (y0 < 0) y0 += A.ny;
    const int x1 = x0 + 1 == A.nx ? 0 : x0 + 1, y1 = y0 + 1 == A.ny ? 0 : y0 + 1;
    int z0;
    double wz;
    node_weight(uz, A.nz, z0, wz);
    const int z1 = A.nz > 1 ? z0 + 1 : z0;
    const int xs[2] = {x0, x1}, ys[2] = {y0, y1}, zs[2] = {z0, z1};
    const double wxs[2] = {1.0 - wx, wx}, wys[2] = {1.0 - wy, wy}, wzs[2] = {1.0 - wz, wz};
    double lt = 0.0, lr = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long q = (long long)zs[c >> 2] * nxy + (long long)ys[(c >> 1) & 1] * A.nx + xs[c & 1];
        const double w = wzs[c >> 2] * wys[(c >> 1) & 1] * wxs[c & 1];
        lt += w * log((double)Tm[q]);
        lr += w * log((double)rho[q]);
    }
    const double rh = exp(lr);
    // table position
    int it, ir;
    double at, ar;
    node_weight((lt - A.lnT0) / A.dlnT, A.nT, it, at);
    node_weight((lr - A.lnR0) / A.dlnR, A.nR, ir, ar);
    const int it1 = A.nT > 1 ? it + 1 : it, ir1 = A.nR > 1 ? ir + 1 : ir;
    for (int b = 0; b < A.nb; ++b) {
        const T *kb = lnk + (long long)b * A.nR * A.nT;
        const double lk = (1.0 - ar) * ((1.0 - at) * (double)__ldg(kb + (long long)ir * A.nT + it) +
                                        at * (double)__ldg(kb + (long long)ir * A.nT + it1)) +
                          ar * ((1.0 - at) * (double)__ldg(kb + (long long)ir1 * A.nT + it) +
                                at * (double)__ldg(kb + (long long)ir1 * A.nT + it1));
        const T *bb = lnB + (long long)b * A.nT;
        const double lb = (1.0 - at) * (double)__ldg(bb + it) + at * (double)__ldg(bb + it1);
        chi[(long long)b * N + p] = (T)(exp(lk) * rh);
        S[(long long)b * N + p] = (T)exp(lb);
    }
}

// FP32: the same steps in float (logs and exps of the FP32 library)
__global__ void __launch_bounds__(256) front_end_f32_kernel(FrontArgs A, const float *__restrict__ Tm,
                                                              const float *__restrict__ rho,
                                                              const float *__restrict__ lnk,
                                                              const float *__restrict__ lnB, float *__restrict__ chi,
                                                              float *__restrict__ S)
{
    const long long nxy = (long long)A.nx * A.ny, N = nxy * A.nz;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int i = (int)(p % A.nx), j = (int)((p / A.nx) % A.ny), k = (int)(p / nxy);
    const float ux = (float)(i + A.sx), uy = (float)(j + A.sy);
    const double uz = k + A.sz;
    const float fx = floorf(ux), fy = floorf(uy);
    const float wx = ux - fx, wy = uy - fy;
    int x0 = (int)fx % A.nx, y0 = (int)fy % A.ny;
    if (x0 < 0) x0 += A.nx;
    if (y0 < 0) y0 += A.ny;
    const int x1 = x0 + 1 == A.nx ? 0 : x0 + 1, y1 = y0 + 1 == A.ny ? 0 : y0 + 1;
    int z0;
    double wzd;
    node_weight(uz, A.nz, z0, wzd);
    const float wz = (float)wzd;
    const int z1 = A.nz > 1 ? z0 + 1 : z0;
    const int xs[2] = {x0, x1}, ys[2] = {y0, y1}, zs[2] = {z0, z1};
    const float wxs[2] = {1.f - wx, wx}, wys[2] = {1.f - wy, wy}, wzs[2] = {1.f - wz, wz};
    float lt = 0.f, lr = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long q = (long long)zs[c >> 2] * nxy + (long long)ys[(c >> 1) & 1] * A.nx + xs[c & 1];
        const float w = wzs[c >> 2] * wys[(c >> 1) & 1] * wxs[c & 1];
        lt = fmaf(w, logf(Tm[q]), lt);
        lr = fmaf(w, logf(rho[q]), lr);
    }
    const float rh = expf(lr);
    int it, ir;
    double atd, ard;
    node_weight(((double)lt - A.lnT0) / A.dlnT, A.nT, it, atd);
    node_weight(((double)lr - A.lnR0) / A.dlnR, A.nR, ir, ard);
    const float at = (float)atd, ar = (float)ard;
    const int it1 = A.nT > 1 ? it + 1 : it, ir1 = A.nR > 1 ? ir + 1 : ir;
    for (int b = 0; b < A.nb; ++b) {
        const float *kb = lnk + (long long)b * A.nR * A.nT;
        const float lk = (1.f - ar) * ((1.f - at) * __ldg(kb + (long long)ir * A.nT + it) +
                                       at * __ldg(kb + (long long)ir * A.nT + it1)) +
                         ar * ((1.f - at) * __ldg(kb + (long long)ir1 * A.nT + it) +
                               at * __ldg(kb + (long long)ir1 * A.nT + it1));
        const float *bb = lnB + (long long)b * A.nT;
        const float lb = (1.f - at) * __ldg(bb + it) + at * __ldg(bb + it1);
        chi[(long long)b * N + p] = expf(lk) * rh;
        S[(long long)b * N + p] = expf(lb);
    }
}

}  // namespace

extern "C" rts_status rts_front_end(const rts_grid *g, const rts_front_table *tab, rts_precision prec,
                                    const void *T_mhd, const void *rho_mhd, void *chi, void *S, void *stream,
                                    char *err, size_t errlen)
{
    auto msg = [&](const char *m) {
        if (err && errlen) snprintf(err, errlen, "%s", m);
    };
    if (!g || !tab || g->nx < 1 || g->ny < 1 || g->nz < 1) return msg("bad grid or table"), RTS_EINVAL;
    if (tab->nbands < 1 || tab->nT < 1 || tab->nR < 1 || !(tab->dlnT > 0) || !(tab->dlnR > 0))
        return msg("table needs nbands, nT, nR >= 1 and positive steps"), RTS_EINVAL;
    if (!T_mhd || !rho_mhd || !chi || !S || !tab->ln_kappa || !tab->ln_B)
        return msg("NULL array"), RTS_EINVAL;
    if (prec != RTS_FP64 && prec != RTS_FP32_MIXED && prec != RTS_FP32_COMPENSATED)
        return msg("unknown precision"), RTS_EINVAL;
    FrontArgs A;
    A.nx = g->nx; A.ny = g->ny; A.nz = g->nz; A.nb = tab->nbands; A.nT = tab->nT; A.nR = tab->nR;
    A.sx = tab->shift[0]; A.sy = tab->shift[1]; A.sz = tab->shift[2];
    A.lnT0 = tab->lnT0; A.dlnT = tab->dlnT; A.lnR0 = tab->lnR0; A.dlnR = tab->dlnR;
    const long long N = (long long)g->nx * g->ny * g->nz;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == RTS_FP64)
        front_end_kernel<double><<<blocks, 256, 0, st>>>(A, (const double *)T_mhd, (const double *)rho_mhd,
                                                         (const double *)tab->ln_kappa, (const double *)tab->ln_B,
                                                         (double *)chi, (double *)S);
    else
        front_end_f32_kernel<<<blocks, 256, 0, st>>>(A, (const float *)T_mhd, (const float *)rho_mhd,
                                                            (const float *)tab->ln_kappa, (const float *)tab->ln_B,
                                                            (float *)chi, (float *)S);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return msg(cudaGetErrorString(e)), RTS_ECUDA;
    msg("ok");
    return RTS_OK;
}

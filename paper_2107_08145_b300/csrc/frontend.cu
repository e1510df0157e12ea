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
// Table coordinates outside the table are clamped to its edge. FP64: one
// thread per RTS point. FP32: tiled, the logarithms of T and rho taken once
// per MHD cell in shared memory, in base 2. The tables are read through the
// read-only cache.
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

// FP32: the same steps in float, tiled. A CTA covers kFX x kFY points of one
// RTS level. The stagger is the same for every point, so the 8 MHD cells of
// a point are (i, j, z0) + (fx, fy, 0) + {0, 1}^3 with fixed weights (wx, wy)
// and the level's clamped (z0, wz): the CTA takes log2 T and log2 rho once
// per MHD cell of its (kFX + 1) x (kFY + 1) x 2 footprint into shared memory
// (4.3 logarithms per point instead of 16) and interpolates from there.
// Base-2 logarithms: interpolating log2 x is interpolating ln x scaled by
// 1 / ln 2, the table position takes the scale into its step, and
// chi_b = 2^(ln kappa_b / ln 2 + log2 rho), S_b = 2^(ln B_b / ln 2).
constexpr int kFX = 96, kFY = 16, kFThreads = 2 * kFX;
constexpr float kLog2e = 1.44269504088896340736f;  // 1 / ln 2

struct FrontArgsF {
    int nx, ny, nz, nb, nT, nR;
    int fx, fy, fz;                  // floor of the shift
    float wx, wy, wz;                // shift - floor(shift)
    float pT, oT, pR, oR;            // table position = log2(x) p - o (ln 2 / step, origin / step)
};

// node_weight in float; x > 0 makes the truncation a floor
__device__ __forceinline__ void node_weight_f(float x, int n, int &i0, float &w)
{
    if (!(x > 0.f)) { i0 = 0; w = 0.f; return; }
    if (x >= (float)(n - 1)) { i0 = n > 1 ? n - 2 : 0; w = n > 1 ? 1.f : 0.f; return; }
    i0 = (int)x;
    w = x - (float)i0;
}

__global__ void __launch_bounds__(kFThreads) front_end_f32_kernel(FrontArgsF A, const float *__restrict__ Tm,
                                                                  const float *__restrict__ rho,
                                                                  const float *__restrict__ lnk,
                                                                  const float *__restrict__ lnB,
                                                                  float *__restrict__ chi, float *__restrict__ S)
{
    __shared__ float sT[2][kFY + 1][kFX + 1], sR[2][kFY + 1][kFX + 1];
    const int ntx = (A.nx + kFX - 1) / kFX, nty = (A.ny + kFY - 1) / kFY;
    const int k = blockIdx.x / (ntx * nty), t = blockIdx.x - k * (ntx * nty);
    const int i0 = (t % ntx) * kFX, j0 = (t / ntx) * kFY;
    // the level's two MHD layers (the clamp of node_weight on z = k + shift_z)
    int z0 = k + A.fz;
    float wz = A.wz;
    if (z0 < 0) {
        z0 = 0;
        wz = 0.f;
    } else if (z0 >= A.nz - 1) {
        z0 = A.nz > 1 ? A.nz - 2 : 0;
        wz = A.nz > 1 ? 1.f : 0.f;
    }
    const int z1 = A.nz > 1 ? z0 + 1 : z0;
    const long long nxy = (long long)A.nx * A.ny, N = nxy * A.nz;
    int xb = (i0 + A.fx) % A.nx, yb = (j0 + A.fy) % A.ny;
    if (xb < 0) xb += A.nx;
    if (yb < 0) yb += A.ny;
    // footprint: thread (c, h) loads column c of rows h, h + 2, ..; the last
    // column (kFX) goes to threads 0 .. 2 (kFY + 1) - 1
    const int c = threadIdx.x % kFX, h = threadIdx.x / kFX;
    const int gx = (xb + c) % A.nx;
#pragma unroll
    for (int zz = 0; zz < 2; ++zz) {
        const float *tz = Tm + (long long)(zz ? z1 : z0) * nxy, *rz = rho + (long long)(zz ? z1 : z0) * nxy;
        int gy = (yb + h) % A.ny;
#pragma unroll
        for (int rr = h; rr <= kFY; rr += kFThreads / kFX) {
            const long long q = (long long)gy * A.nx + gx;
            sT[zz][rr][c] = log2f(__ldg(tz + q));
            sR[zz][rr][c] = log2f(__ldg(rz + q));
            gy += kFThreads / kFX;
            if (gy >= A.ny) gy -= A.ny;
            if (gy >= A.ny) gy -= A.ny;
        }
    }
    if (threadIdx.x < 2 * (kFY + 1)) {
        const int zz = threadIdx.x / (kFY + 1), rr = threadIdx.x - zz * (kFY + 1);
        const long long q = (long long)(zz ? z1 : z0) * nxy + (long long)((yb + rr) % A.ny) * A.nx + (xb + kFX) % A.nx;
        sT[zz][rr][kFX] = log2f(__ldg(Tm + q));
        sR[zz][rr][kFX] = log2f(__ldg(rho + q));
    }
    __syncthreads();
    const int i = i0 + c;
    if (i >= A.nx) return;
    const float wx1 = A.wx, wx0 = 1.f - A.wx, wy1 = A.wy, wy0 = 1.f - A.wy, wz0 = 1.f - wz;
    for (int r = threadIdx.x / kFX; r < kFY && j0 + r < A.ny; r += kFThreads / kFX) {
        float lt = 0.f, lr = 0.f;
#pragma unroll
        for (int zz = 0; zz < 2; ++zz) {
            const float w = zz ? wz : wz0;
            const float t0 = fmaf(wx1, sT[zz][r][c + 1], wx0 * sT[zz][r][c]);
            const float t1 = fmaf(wx1, sT[zz][r + 1][c + 1], wx0 * sT[zz][r + 1][c]);
            const float r0 = fmaf(wx1, sR[zz][r][c + 1], wx0 * sR[zz][r][c]);
            const float r1 = fmaf(wx1, sR[zz][r + 1][c + 1], wx0 * sR[zz][r + 1][c]);
            lt = fmaf(w, fmaf(wy1, t1, wy0 * t0), lt);
            lr = fmaf(w, fmaf(wy1, r1, wy0 * r0), lr);
        }
        int it, ir;
        float at, ar;
        node_weight_f(fmaf(lt, A.pT, -A.oT), A.nT, it, at);
        node_weight_f(fmaf(lr, A.pR, -A.oR), A.nR, ir, ar);
        const int dt = A.nT > 1 ? 1 : 0, dr = A.nR > 1 ? A.nT : 0;
        const float *kb = lnk + ir * A.nT + it, *bb = lnB + it;
        float *cp = chi + (long long)k * nxy + (long long)(j0 + r) * A.nx + i, *sp = S + (cp - chi);
        for (int b = 0; b < A.nb; ++b) {
            const float lk = (1.f - ar) * ((1.f - at) * __ldg(kb) + at * __ldg(kb + dt)) +
                             ar * ((1.f - at) * __ldg(kb + dr) + at * __ldg(kb + dr + dt));
            const float lb = (1.f - at) * __ldg(bb) + at * __ldg(bb + dt);
            *cp = exp2f(fmaf(lk, kLog2e, lr));  // kappa rho = 2^(log2 kappa + log2 rho)
            *sp = exp2f(lb * kLog2e);
            kb += A.nR * A.nT;
            bb += A.nT;
            cp += N;
            sp += N;
        }
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
    for (int d = 0; d < 3; ++d)
        if (!(fabs(tab->shift[d]) <= 1048576.0)) return msg("shift must be finite, |shift| <= 2^20"), RTS_EINVAL;
    if (prec != RTS_FP64 && prec != RTS_FP32_MIXED && prec != RTS_FP32_COMPENSATED)
        return msg("unknown precision"), RTS_EINVAL;
    FrontArgs A;
    A.nx = g->nx; A.ny = g->ny; A.nz = g->nz; A.nb = tab->nbands; A.nT = tab->nT; A.nR = tab->nR;
    A.sx = tab->shift[0]; A.sy = tab->shift[1]; A.sz = tab->shift[2];
    A.lnT0 = tab->lnT0; A.dlnT = tab->dlnT; A.lnR0 = tab->lnR0; A.dlnR = tab->dlnR;
    const long long N = (long long)g->nx * g->ny * g->nz;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == RTS_FP64) {
        const unsigned blocks = (unsigned)((N + 255) / 256);
        front_end_kernel<double><<<blocks, 256, 0, st>>>(A, (const double *)T_mhd, (const double *)rho_mhd,
                                                         (const double *)tab->ln_kappa, (const double *)tab->ln_B,
                                                         (double *)chi, (double *)S);
    } else {
        FrontArgsF F;
        F.nx = A.nx; F.ny = A.ny; F.nz = A.nz; F.nb = A.nb; F.nT = A.nT; F.nR = A.nR;
        const double *sh = tab->shift;
        F.fx = (int)floor(sh[0]); F.fy = (int)floor(sh[1]); F.fz = (int)floor(sh[2]);
        F.wx = (float)(sh[0] - floor(sh[0])); F.wy = (float)(sh[1] - floor(sh[1])); F.wz = (float)(sh[2] - floor(sh[2]));
        F.pT = (float)(M_LN2 / tab->dlnT); F.oT = (float)(tab->lnT0 / tab->dlnT);
        F.pR = (float)(M_LN2 / tab->dlnR); F.oR = (float)(tab->lnR0 / tab->dlnR);
        const long long tiles = (long long)((g->nx + kFX - 1) / kFX) * ((g->ny + kFY - 1) / kFY) * g->nz;
        if (tiles > 0x7fffffffLL) return msg("grid too large for the FP32 input step"), RTS_EINVAL;
        front_end_f32_kernel<<<(unsigned)tiles, kFThreads, 0, st>>>(F, (const float *)T_mhd, (const float *)rho_mhd,
                                                                    (const float *)tab->ln_kappa,
                                                                    (const float *)tab->ln_B, (float *)chi, (float *)S);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return msg(cudaGetErrorString(e)), RTS_ECUDA;
    msg("ok");
    return RTS_OK;
}

// batched.cuh -- the per-grid kernels of a solve (transpose, unit reduction,
// Q step) for many independent grids ("subdomains") of uneven size in one
// launch each. Subdomain arrays are packed one after another in caller
// buffers; a descriptor table gives each one's sizes and offsets. A launch is
// a flat 1-D grid of CTAs; each subdomain owns a contiguous range of CTA
// indices (prefix sums in the table) and a CTA finds its subdomain by binary
// search. The sweep itself needs no batched variant: its units already carry
// their own extents and offsets.
#pragma once
#include "qstep.cuh"

namespace rts {

struct SubDesc {
    int nx, ny, nz;
    long long N;
    long long in_off;    // chi, S (and their x-transposed copies) of band 0
    long long top_off;   // I_top of band 0
    long long out_off;   // J and Q; F starts at 3 * out_off
    long long jf_off;    // JF of band 0 ([B][4][N] from here)
    int ru0;             // RedUnit range of band b: ru_begin[ru0 + b] .. ru_begin[ru0 + b + 1]
    int blk[3];          // first CTA of this subdomain in the transpose, reduce and Q-step launches
    QParams P;
};

// subdomain owning CTA `blk` of launch kind `which` (blk[] ascending, every
// subdomain owns at least one CTA)
__device__ __forceinline__ int find_sub(const SubDesc *__restrict__ d, int nsub, int which, int blk)
{
    int lo = 0, hi = nsub - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].blk[which] <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// CTAs of one subdomain: (32 x 32 tiles of a level) x levels x bands for the
// transpose and the reduction; (32 x 8 tiles of a level) x levels for the Q step
__host__ __device__ inline long long sub_blocks(int which, int nx, int ny, int nz, int B)
{
    if (which < 2) return (long long)((nx + 31) / 32) * ((ny + 31) / 32) * nz * B;
    return (long long)((nx + 31) / 32) * ((ny + 7) / 8) * nz;
}

template <typename T>
__global__ void __launch_bounds__(256) transpose_x2_batched(const SubDesc *__restrict__ d, int nsub, int B,
                                                              const T *__restrict__ in0, const T *__restrict__ in1,
                                                              T *__restrict__ out0, T *__restrict__ out1,
                                                              int *status)
{
    const int s = find_sub(d, nsub, 0, blockIdx.x);
    const SubDesc &sd = d[s];
    const int r = blockIdx.x - sd.blk[0];
    const int tx = (sd.nx + 31) / 32, ty = (sd.ny + 31) / 32;
    const int bx = r % tx, by = (r / tx) % ty;
    const long long bk = r / (tx * ty);
    transpose_tile2(in0 + sd.in_off, in1 + sd.in_off, out0 + sd.in_off, out1 + sd.in_off, sd.nx, sd.ny, sd.nz, bx * 32,
                    by * 32, bk / sd.nz, bk % sd.nz, status);
}

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) reduce_units_batched(const SubDesc *__restrict__ d, int nsub,
                                                            const RedUnit *__restrict__ ru,
                                                            const int *__restrict__ ru_begin, Acc *__restrict__ JF,
                                                            int raw)
{
    const int s = find_sub(d, nsub, 1, blockIdx.x);
    const SubDesc &sd = d[s];
    const int r = blockIdx.x - sd.blk[1];
    const int tx = (sd.nx + 31) / 32, ty = (sd.ny + 31) / 32;
    const int bx = r % tx, by = (r / tx) % ty;
    const int bk = r / (tx * ty);
    const int b = bk / sd.nz, k = bk % sd.nz;
    reduce_tile<T, Acc>(ru, ru_begin[sd.ru0 + b], ru_begin[sd.ru0 + b + 1], JF + sd.jf_off + (long long)b * 4 * sd.N,
                        sd.nx, sd.ny, sd.nz, bx * 32, by * 32, k, raw != 0);
}

template <typename T, typename Acc>
__global__ void __launch_bounds__(256) qstep_batched(const SubDesc *__restrict__ d, int nsub,
                                                     const Acc *__restrict__ JF, const T *__restrict__ chi,
                                                     const T *__restrict__ S, double *__restrict__ J,
                                                     double *__restrict__ F, double *__restrict__ Q)
{
    const int s = find_sub(d, nsub, 2, blockIdx.x);
    const SubDesc &sd = d[s];
    const int r = blockIdx.x - sd.blk[2];
    const int tx = (sd.nx + 31) / 32, ty = (sd.ny + 7) / 8;
    const int bx = r % tx, by = (r / tx) % ty, k = r / (tx * ty);
    qstep_point<T, Acc>(JF + sd.jf_off, chi + sd.in_off, S + sd.in_off, sd.P, J ? J + sd.out_off : nullptr,
                        F ? F + 3 * sd.out_off : nullptr, Q ? Q + sd.out_off : nullptr, bx * 32 + threadIdx.x,
                        by * 8 + threadIdx.y, k);
}

}  // namespace rts

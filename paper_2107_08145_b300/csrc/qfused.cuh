// qfused.cuh -- the band reduction of the FP32 forward solve (the paper's
// flux() step, Sect. 5.1: J_b and F_b of every band from the ray
// intensities) over the raw slot intensities of the register sweep.
//
// A persistent kernel: each CTA walks tiles of 32 x 16 (i, j) points of one
// level of one band, and while it sums tile n the 16-byte cp.async copies of
// tile n+1 (every unit's four slot intensities of every point, in the
// unit's own layout) are in flight into the other half of a double buffer,
// so memory latency is not paid per tile. Units in natural layout ([k][j][i])
// are copied along i; the x groups ([i][k][j]) along j, into rows padded to
// 17 points so that the owner's transposed reads are free of bank
// conflicts. The moments are formed with the exact pair differences of
// unit_moments and summed with the rounding error of every addition kept
// exactly (TwoSum) and added back at the end (the compensated sum of Ogita,
// Rump and Oishi, as accurate as summing in twice the precision), written as
// double-float J_b, F_b ([b][c][N], the layout qstep_kernel<float, df32>
// reads). No FP64 arithmetic: B300's FP64 rate would bound this step.
#pragma once
#include "qstep.cuh"

namespace rts {

constexpr int QR_TI = 32;  // tile extent in i (threads in x)
constexpr int QR_TJ = 16;  // tile extent in j
constexpr int QR_RY = 8;   // threads in y: each owns QR_TJ / QR_RY points
constexpr int QR_NT = QR_TI * QR_RY;
constexpr int QR_NAT = QR_TJ * QR_TI;         // float4 of a natural unit's tile
constexpr int QR_XR = QR_TJ + 1;              // padded row of an x group's tile
constexpr int QR_XU = QR_TI * QR_XR;          // float4 of an x group's tile

// shared memory: two buffers of the largest band's units, then the units
__host__ __device__ constexpr size_t qr_smem_bytes(int max_nat, int max_x, int nunits)
{
    return (size_t)2 * (max_nat * QR_NAT + max_x * QR_XU) * sizeof(float4) + sizeof(RedUnit) * (size_t)nunits;
}

// 16-byte copy global -> shared; src_bytes 0 fills zeros (the source is not read)
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src, int src_bytes)
{
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(gmem_src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// qb: [0 .. B] first unit of each band, [B+1 .. 2B] end of the band's x
// groups (each band's units are ordered x groups first)
__global__ void __launch_bounds__(QR_NT, 2) qf_reduce_kernel(const RedUnit *__restrict__ ru,
                                                               const int *__restrict__ qb, int nx, int ny, int nz,
                                                               int nbands, int nunits, int max_nat, int max_x,
                                                               df32 *__restrict__ JF)
{
    constexpr int RP = QR_TJ / QR_RY;
    extern __shared__ __align__(16) float4 qr_sm[];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * QR_TI + tx;
    // the units' coefficients, read by every thread of the CTA (broadcast loads)
    RedUnit *su = reinterpret_cast<RedUnit *>(qr_sm + 2 * (max_nat * QR_NAT + max_x * QR_XU));
    {
        const int words = (int)(sizeof(RedUnit) / 4) * nunits;
        const int *src = reinterpret_cast<const int *>(ru);
        int *dst = reinterpret_cast<int *>(su);
        for (int w = tid; w < words; w += QR_NT) dst[w] = src[w];
    }
    const long long N = (long long)nx * ny * nz;
    const int nti = (nx + QR_TI - 1) / QR_TI, ntj = (ny + QR_TJ - 1) / QR_TJ;
    const int ntiles = nti * ntj * nz * nbands;  // < 2^31: checked on the host
    const int buf = max_nat * QR_NAT + max_x * QR_XU;
    // x groups are copied along j: point (xi + 16 r, xj) of the tile
    const int xj = tid % QR_TJ, xi = tid / QR_TJ;
    constexpr int XR = QR_NT / QR_TJ;

    // tile t: i tile fastest, then j tile, level, band
    auto decode = [&](int t, int &ti, int &tj, int &k, int &b) {
        ti = t % nti;
        t /= nti;
        tj = t % ntj;
        t /= ntj;
        k = t % nz;
        b = t / nz;
    };
    auto issue = [&](int t, int half) {
        if (t < ntiles) {
            int ti, tj, k, b;
            decode(t, ti, tj, k, b);
            const int i0 = ti * QR_TI, j0 = tj * QR_TJ;
            const int ub = qb[b], ux = qb[nbands + 1 + b], ue = qb[b + 1];
            float4 *sb = qr_sm + (long long)half * buf;
            for (int u = ux; u < ue; ++u) {  // natural: [j][i]
                const float4 *part = reinterpret_cast<const float4 *>(ru[u].partial);
                float4 *dst = sb + (u - ux) * QR_NAT;
#pragma unroll
                for (int r = 0; r < RP; ++r) {
                    const int i = i0 + tx, j = j0 + ty + QR_RY * r;
                    const bool in = i < nx && j < ny;
                    cp_async16(dst + (ty + QR_RY * r) * QR_TI + tx,
                               part + (in ? ((long long)k * ny + j) * nx + i : 0), in ? 16 : 0);
                }
            }
            for (int u = ub; u < ux; ++u) {  // x groups: [i][j], rows padded
                const float4 *part = reinterpret_cast<const float4 *>(ru[u].partial);
                float4 *dst = sb + max_nat * QR_NAT + (u - ub) * QR_XU;
#pragma unroll
                for (int r = 0; r < RP; ++r) {
                    const int i = i0 + xi + XR * r, j = j0 + xj;
                    const bool in = i < nx && j < ny;
                    cp_async16(dst + (xi + XR * r) * QR_XR + xj,
                               part + (in ? ((long long)i * nz + k) * ny + j : 0), in ? 16 : 0);
                }
            }
        }
        cp_async_commit_group();
    };

    int t = blockIdx.x;
    issue(t, 0);
    for (int n = 0; t < ntiles; ++n, t += gridDim.x) {
        issue(t + (int)gridDim.x, (n + 1) & 1);
        cp_async_wait_prev();
        __syncthreads();  // tile t in shared memory
        int ti, tj, k, b;
        decode(t, ti, tj, k, b);
        const int ub = qb[b], ux = qb[nbands + 1 + b], ue = qb[b + 1];
        const float4 *sb = qr_sm + (long long)(n & 1) * buf;
        // per point and moment: the running sum s and the sum e of the rounding
        // errors of its additions (each exact by TwoSum), s + e at the end
        float sm[RP][4], se[RP][4];
#pragma unroll
        for (int r = 0; r < RP; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) sm[r][c] = se[r][c] = 0.f;
        for (int u = ub; u < ue; ++u) {
            const RedUnit &U = su[u];
            const bool xg = u < ux;
            const float4 *src = xg ? sb + max_nat * QR_NAT + (u - ub) * QR_XU : sb + (u - ux) * QR_NAT;
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                const int jj = ty + QR_RY * r;
                const float4 I = xg ? src[tx * QR_XR + jj] : src[jj * QR_TI + tx];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    // the moment with the unit's pairing (a unit-wide branch)
                    const float *kc = U.c[c];
                    float m;
                    if (U.qpair[c])
                        m = pair_sum(kc[0], I.x, kc[2], I.z) + pair_sum(kc[1], I.y, kc[3], I.w);
                    else
                        m = pair_sum(kc[0], I.x, kc[1], I.y) + pair_sum(kc[2], I.z, kc[3], I.w);
                    float s2, e2;
                    two_sum(sm[r][c], m, s2, e2);
                    sm[r][c] = s2;
                    se[r][c] += e2;
                }
            }
        }
        const int i = ti * QR_TI + tx;
        df32 *jf = JF + (long long)b * 4 * N;
#pragma unroll
        for (int r = 0; r < RP; ++r) {
            const int j = tj * QR_TJ + ty + QR_RY * r;
            if (i >= nx || j >= ny) continue;
            const long long p = ((long long)k * ny + j) * nx + i;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                df32 v;
                two_sum(sm[r][c], se[r][c], v.hi, v.lo);
                jf[c * N + p] = v;
            }
        }
        __syncthreads();  // buffer n & 1 is refilled by the next iteration's copies
    }
}

}  // namespace rts

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
//
// The kernel is issue-bound unless its instruction count per point is small,
// so: each thread owns two points of a tile and runs every operation on the
// pair as one packed FP32x2 instruction (lane-wise the same roundings as
// the scalar form, so the result is the scalar kernel's to the bit); the
// slot pairing of each moment is fixed at compile time per group of units
// (a unit's own flux component across its sweep axis pairs slots (0,2) and
// (1,3): F_z for x and y units, F_y for z units; the host checks that
// every unit's table agrees), so the unit loop has no branch; the
// coefficients sit in shared memory already duplicated for both lanes and
// with the negated ones the exact product errors need; a tile's index is
// decoded once and its copy offsets computed once for all its units.
#pragma once
#include "qstep.cuh"

namespace rts {

constexpr int QR_TI = 32;  // tile extent in i (threads in x)
constexpr int QR_TJ = 16;  // tile extent in j
constexpr int QR_RY = 8;   // threads in y: each owns QR_TJ / QR_RY = 2 points
constexpr int QR_NT = QR_TI * QR_RY;
constexpr int QR_NAT = QR_TJ * QR_TI;         // float4 of a natural unit's tile
constexpr int QR_XR = QR_TJ + 1;              // padded row of an x group's tile
constexpr int QR_XU = QR_TI * QR_XR;          // float4 of an x group's tile
constexpr int QR_KU = 13;                     // float4 of a unit's shared record
static_assert(QR_TJ == 2 * QR_RY, "each thread owns two points of a tile");

// the moment whose slot pairing is (0,2)+(1,3) for units sweeping along
// axis a (the component along the unit's second transverse axis)
__host__ __device__ constexpr int qr_cross_moment(int axis) { return axis == 2 ? 2 : 3; }

// shared memory: two buffers of the largest band's units, the unit records
// (partial pointer, then per moment three float4 of duplicated
// coefficients) and the band table (3 B + 1 ints)
__host__ __device__ constexpr size_t qr_smem_bytes(int max_nat, int max_x, int nunits, int nbands)
{
    return (size_t)2 * (max_nat * QR_NAT + max_x * QR_XU) * sizeof(float4) +
           sizeof(float4) * QR_KU * (size_t)nunits + ((size_t)(3 * nbands + 1) * sizeof(int) + 15) / 16 * 16;
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

// a x + b y on both lanes, as pair_sum: p = b y rounded, the exact error
// b y - p recovered as -(p - b y) = -fma(-b, y, p), added to fma(a, x, p)
__device__ __forceinline__ float2 pair_sum2(float2 a, float2 x, float2 b, float2 nb, float2 y)
{
    const float2 p = mul2(b, y);
    return sub2(fma2(a, x, p), fma2(nb, y, p));
}

// one unit's four moments at the thread's two points, added to (s, e). K:
// the unit's record; per moment c three float4 (a1 a1 b1 b1), (-b1 -b1 a2
// a2), (b2 b2 -b2 -b2) for the pairs (a1, b1) + (a2, b2) of its pairing.
template <int QC>
__device__ __forceinline__ void qr_unit(const float4 *__restrict__ K, float4 A, float4 B, float2 (&s)[4],
                                        float2 (&e)[4])
{
    const float2 I0 = f2(A.x, B.x), I1 = f2(A.y, B.y), I2 = f2(A.z, B.z), I3 = f2(A.w, B.w);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float4 q0 = K[1 + 3 * c], q1 = K[2 + 3 * c], q2 = K[3 + 3 * c];
        const float2 m = add2(pair_sum2(f2(q0.x, q0.y), I0, f2(q0.z, q0.w), f2(q1.x, q1.y), c == QC ? I2 : I1),
                              pair_sum2(f2(q1.z, q1.w), c == QC ? I1 : I2, f2(q2.x, q2.y), f2(q2.z, q2.w), I3));
        float2 s2, e2;
        two_sum2(s[c], m, s2, e2);
        s[c] = s2;
        e[c] = add2(e[c], e2);
    }
}

// qb: [0 .. B] first unit of each band, [B+1 .. 2B] end of the band's x
// groups, [2B+1 .. 3B] end of its y units (each band's units are ordered
// x groups, y units, z units)
__global__ void __launch_bounds__(QR_NT, 2) qf_reduce_kernel(const RedUnit *__restrict__ ru,
                                                               const int *__restrict__ qb, int nx, int ny, int nz,
                                                               int nbands, int nunits, int max_nat, int max_x,
                                                               df32 *__restrict__ JF)
{
    extern __shared__ __align__(16) float4 qr_sm[];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * QR_TI + tx;
    const int buf = max_nat * QR_NAT + max_x * QR_XU;
    float4 *sk = qr_sm + 2 * buf;  // unit records, read by every thread (broadcast loads)
    int *sq = reinterpret_cast<int *>(sk + QR_KU * nunits);
    for (int w = tid; w < QR_KU * nunits; w += QR_NT) {
        const int u = w / QR_KU, q = w % QR_KU;
        const RedUnit &U = ru[u];
        float4 v;
        if (q == 0) {
            v = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<const void **>(&v) = U.partial;
        } else {
            const int c = (q - 1) / 3, f = (q - 1) % 3;
            const float *k = U.c[c];
            const int a1 = 0, b1 = U.qpair[c] ? 2 : 1, a2 = U.qpair[c] ? 1 : 2, b2 = 3;
            if (f == 0) v = make_float4(k[a1], k[a1], k[b1], k[b1]);
            else if (f == 1) v = make_float4(-k[b1], -k[b1], k[a2], k[a2]);
            else v = make_float4(k[b2], k[b2], -k[b2], -k[b2]);
        }
        sk[w] = v;
    }
    for (int w = tid; w < 3 * nbands + 1; w += QR_NT) sq[w] = qb[w];
    __syncthreads();

    const long long N = (long long)nx * ny * nz;
    const int nti = (nx + QR_TI - 1) / QR_TI, ntj = (ny + QR_TJ - 1) / QR_TJ;
    const int ntiles = nti * ntj * nz * nbands;  // < 2^31: checked on the host
    // x groups are copied along j: point (xi + 16 r, xj) of the tile
    const int xj = tid % QR_TJ, xi = tid / QR_TJ;
    constexpr int XR = QR_NT / QR_TJ;
    // the thread's shared offsets of its two points: natural, x group
    const int on0 = ty * QR_TI + tx, on1 = on0 + QR_RY * QR_TI;
    const int ox0 = tx * QR_XR + ty, ox1 = ox0 + QR_RY;
    const int cn0 = ty * QR_TI + tx, cx0 = xi * QR_XR + xj;  // its copy destinations

    // tile t: i tile fastest, then j tile, level, band
    auto decode = [&](int t) {
        int4 d;
        d.x = t % nti;
        t /= nti;
        d.y = t % ntj;
        t /= ntj;
        d.z = t % nz;
        d.w = t / nz;
        return d;
    };
    auto issue = [&](bool live, int4 d, int half) {
        if (live) {
            const int i0 = d.x * QR_TI, j0 = d.y * QR_TJ, k = d.z, b = d.w;
            const int ub = sq[b], ux = sq[nbands + 1 + b], ue = sq[b + 1];
            float4 *sb = qr_sm + half * buf;
            // the point offsets (float4) and source sizes of this tile, for all units
            long long gn[2], gx[2];
            int zn[2], zx[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int i = i0 + tx, j = j0 + ty + QR_RY * r;
                const bool in = i < nx && j < ny;
                gn[r] = in ? ((long long)k * ny + j) * nx + i : 0;
                zn[r] = in ? 16 : 0;
                const int ii = i0 + xi + XR * r, jj = j0 + xj;
                const bool inx = ii < nx && jj < ny;
                gx[r] = inx ? ((long long)ii * nz + k) * ny + jj : 0;
                zx[r] = inx ? 16 : 0;
            }
            for (int u = ux; u < ue; ++u) {  // natural: [j][i]
                const float4 *part = *reinterpret_cast<const float4 *const *>(sk + QR_KU * u);
                float4 *dst = sb + (u - ux) * QR_NAT + cn0;
                cp_async16(dst, part + gn[0], zn[0]);
                cp_async16(dst + QR_RY * QR_TI, part + gn[1], zn[1]);
            }
            for (int u = ub; u < ux; ++u) {  // x groups: [i][j], rows padded
                const float4 *part = *reinterpret_cast<const float4 *const *>(sk + QR_KU * u);
                float4 *dst = sb + max_nat * QR_NAT + (u - ub) * QR_XU + cx0;
                cp_async16(dst, part + gx[0], zx[0]);
                cp_async16(dst + XR * QR_XR, part + gx[1], zx[1]);
            }
        }
        cp_async_commit_group();
    };

    int t = blockIdx.x;
    int4 cur = decode(t < ntiles ? t : 0);
    issue(t < ntiles, cur, 0);
    for (int n = 0; t < ntiles; ++n, t += gridDim.x) {
        const int tn = t + (int)gridDim.x;
        const int4 nxt = decode(tn < ntiles ? tn : 0);
        issue(tn < ntiles, nxt, (n + 1) & 1);
        cp_async_wait_prev();
        __syncthreads();  // tile t in shared memory
        const int b = cur.w;
        const int ub = sq[b], ux = sq[nbands + 1 + b], uy = sq[2 * nbands + 1 + b], ue = sq[b + 1];
        const float4 *sb = qr_sm + (n & 1) * buf;
        // per point pair and moment: the running sum s and the sum e of the
        // rounding errors of its additions (each exact by TwoSum), s + e at the end
        float2 s[4], e[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) s[c] = e[c] = f2(0.f);
        {
            const float4 *src = sb + max_nat * QR_NAT;
            for (int u = ub; u < ux; ++u, src += QR_XU)
                qr_unit<qr_cross_moment(0)>(sk + QR_KU * u, src[ox0], src[ox1], s, e);
        }
        const float4 *src = sb;
        for (int u = ux; u < uy; ++u, src += QR_NAT)
            qr_unit<qr_cross_moment(1)>(sk + QR_KU * u, src[on0], src[on1], s, e);
        for (int u = uy; u < ue; ++u, src += QR_NAT)
            qr_unit<qr_cross_moment(2)>(sk + QR_KU * u, src[on0], src[on1], s, e);
        const int i = cur.x * QR_TI + tx, j = cur.y * QR_TJ + ty;
        df32 *jf = JF + (long long)b * 4 * N + ((long long)cur.z * ny + j) * nx + i;
        const bool in0 = i < nx && j < ny, in1 = i < nx && j + QR_RY < ny;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float2 hi, lo;
            two_sum2(s[c], e[c], hi, lo);
            if (in0) jf[c * N] = df32{hi.x, lo.x};
            if (in1) jf[c * N + QR_RY * nx] = df32{hi.y, lo.y};
        }
        cur = nxt;
        __syncthreads();  // buffer n & 1 is refilled by the next iteration's copies
    }
}

// The Q step over double-float J_b, F_b (qstep_kernel<float, df32>'s
// arithmetic, Sect. 5.1's Q_rad = sum_b [om_b 4 pi chi_b (J_b - S_b) +
// (1 - om_b)(-div F_b)] with the band sums of J and F), two points per
// thread -- (i, j) and (i, j + 8) of a 32 x 16 tile of one level -- so that
// the double-float operations run packed and each thread has both points'
// loads in flight. Up to the sign of a zero, the results are those of the
// one-point kernel.
constexpr int QS_TJ = 16;
// the double-float stencil and 4 pi constants of qstep_kernel<float, df32>
// (acc_from of the FP64 values), splatted on both lanes with their negations
struct Acc2Const {
    df2 cx, ncx, cy, ncy, cz, ncz, four_pi, nfour_pi;
    float thin;
    __device__ __forceinline__ Acc2Const(const QParams &P, int k)
    {
        df32 *tag = nullptr;
        cx = df2_splat(acc_from(tag, P.inv2dx));
        cy = df2_splat(acc_from(tag, P.inv2dy));
        cz = df2_splat(z_coef<df32>(P, k));
        four_pi = df2_splat(acc_from(tag, 12.566370614359172953850573533118));
        ncx = df2_neg(cx);
        ncy = df2_neg(cy);
        ncz = df2_neg(cz);
        nfour_pi = df2_neg(four_pi);
        thin = (float)P.thin;
    }
};
__global__ void __launch_bounds__(256, 4) qstep_df2_kernel(const df32 *__restrict__ JF, const float *__restrict__ chi,
                                                        const float *__restrict__ S, QParams P,
                                                        double *__restrict__ J, double *__restrict__ F,
                                                        double *__restrict__ Q)
{
    const int i = blockIdx.x * 32 + threadIdx.x, j0 = blockIdx.y * QS_TJ + threadIdx.y, k = blockIdx.z;
    if (i >= P.nx || j0 >= P.ny) return;
    const bool two = j0 + QS_TJ / 2 < P.ny;
    const int j1 = two ? j0 + QS_TJ / 2 : j0;  // outside the grid: the first point again, not stored
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const long long N = (long long)nx * ny * nz;
    // the two points and their neighbours (periodic in x and y; one-sided
    // differences at the bottom and top levels); in-band offsets are below
    // N < 2^31 (the register sweep serves no larger band)
    int p[2], xp[2], xm[2], yp[2], ym[2];
    const int jj[2] = {j0, j1};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int j = jj[r];
        p[r] = (k * ny + j) * nx + i;
        xp[r] = p[r] - i + (i + 1 == nx ? 0 : i + 1);
        xm[r] = p[r] - i + (i == 0 ? nx - 1 : i - 1);
        yp[r] = p[r] + ((j + 1 == ny ? 0 : j + 1) - j) * nx;
        ym[r] = p[r] + ((j == 0 ? ny - 1 : j - 1) - j) * nx;
    }
    int dzp, dzm;  // z neighbours as offsets from the point
    if (nz == 1) { dzp = dzm = 0; }
    else if (k == 0) { dzp = nx * ny; dzm = 0; }
    else if (k == nz - 1) { dzp = 0; dzm = -nx * ny; }
    else { dzp = nx * ny; dzm = -nx * ny; }
    Acc2Const K(P, k);
    auto ld2 = [&](const df32 *a, int o0, int o1) { return df2_pair(a[o0], a[o1]); };
    const df2 z2 = {f2(0.f), f2(0.f)};
    df2 Jt = z2, Fx = z2, Fy = z2, Fz = z2, Qt = z2;
    for (int b = 0; b < P.nbands; ++b) {
        const df32 *jf = JF + (long long)b * 4 * N;
        const df2 Jb = ld2(jf, p[0], p[1]);
        const df2 fx = ld2(jf + N, p[0], p[1]), fy = ld2(jf + 2 * N, p[0], p[1]), fz = ld2(jf + 3 * N, p[0], p[1]);
        const df2 dvx = df2_mul(df2_sub(ld2(jf + N, xp[0], xp[1]), ld2(jf + N, xm[0], xm[1])), K.cx, K.ncx);
        const df2 dvy = df2_mul(df2_sub(ld2(jf + 2 * N, yp[0], yp[1]), ld2(jf + 2 * N, ym[0], ym[1])), K.cy, K.ncy);
        const df2 dvz = df2_mul(df2_sub(ld2(jf + 3 * N, p[0] + dzp, p[1] + dzp), ld2(jf + 3 * N, p[0] + dzm, p[1] + dzm)),
                                K.cz, K.ncz);
        const df2 D = df2_add(df2_add(dvx, dvy), dvz);  // div F_b; the Q step uses -D
        const float *cb = chi + (long long)b * N, *sb = S + (long long)b * N;
        const float2 c = f2(cb[p[0]], cb[p[1]]), sv = f2(sb[p[0]], sb[p[1]]);
        const df2 dJ = df2_sub(Jb, sv);
        const df2 qj = df2_mul(df2_mul(K.four_pi, K.nfour_pi, c), dJ, df2_neg(dJ));
        // om = e^-x, omc = 1 - om = -expm1(-x), x = chi thin (blend_weights)
        float2 om, m1;  // m1 = expm1(-x) = -omc
        {
            const float x0 = c.x * K.thin, x1 = c.y * K.thin;
            om = f2(expf(-x0), expf(-x1));
            m1 = f2(expm1f(-x0), expm1f(-x1));
        }
        // om qj + omc (-D), with omc (-D) = (-omc) D = m1 D
        const df2 qb = df2_add(df2_mul(om, neg2(om), qj), df2_mul(m1, neg2(m1), D));
        if (b == 0) {
            Jt = Jb; Fx = fx; Fy = fy; Fz = fz; Qt = qb;  // 0 + v is v for a normalised v
        } else {
            Jt = df2_add(Jt, Jb);
            Fx = df2_add(Fx, fx);
            Fy = df2_add(Fy, fy);
            Fz = df2_add(Fz, fz);
            Qt = df2_add(Qt, qb);
        }
    }
    const int p1 = p[1];
    auto st = [&](double *o, df2 v) {
        o[p[0]] = (double)v.hi.x + (double)v.lo.x;
        if (two) o[p1] = (double)v.hi.y + (double)v.lo.y;
    };
    if (J) st(J, Jt);
    if (F) {
        st(F, Fx);
        st(F + N, Fy);
        st(F + 2 * N, Fz);
    }
    if (Q) st(Q, Qt);
}

}  // namespace rts

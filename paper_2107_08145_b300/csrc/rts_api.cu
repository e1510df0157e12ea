// rts_api.cu -- C ABI of the B300 radiation transport solver (include/rts.h).
//
// rts_create plans the solve once per grid: the angular set, the geometry of
// every short characteristic, the sweep units (band x direction group, up to
// 4 directions each), their tiling, and all device scratch. rts_solve then
// only enqueues kernels on the handle's stream:
//   1. transpose of chi and S for the x-dominant groups (paper Sect. 5.3.1)
//   2. one persistent sweep launch over every band and group (Sect. 5.1
//      integrate(); Sect. 5.2 launch overhead removed by construction)
//   3. per-band reduction of the sweep-unit partial sums, and
//   4. the Q step (flux(): J, F and the thin/thick Q_rad blend).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <type_traits>
#include <vector>

#include "rts.h"
#include "adjoint.cuh"
#include "batched.cuh"
#include "qstep.cuh"
#include "sweep.cuh"
#include "kernels.h"
#include "sweep_reg.cuh"
#include "qfused.cuh"

namespace {

// chi = exp(log chi) for RTS_FLAG_LOG_CHI (accurate exp of the precision)
template <typename T>
__global__ void __launch_bounds__(256) exp_kernel(const T *__restrict__ in, T *__restrict__ out, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = exp(in[i]);
}

// Local operator of the scattering iteration: the weight of S at a point in
// its own mean intensity is sum_d w_d (1 - q(dtau_d)), q(x) = (1 - e^-x)/x,
// with dtau_d = ds_d (chi_up + chi_p)/2 the segment's optical depth. It is
// taken here with dtau_d = ds_d chi_p / 2, a lower bound (chi_up >= 0), so
// that L* never exceeds the true diagonal (1 - q grows with dtau): a larger
// L* over-corrects and the iteration can diverge. Only the preconditioner:
// the fixed point does not depend on it. dirw lists each distinct segment
// length once with the summed weight of its directions.
template <typename T>
__global__ void __launch_bounds__(256) lambda_star_kernel(const T *__restrict__ chi, const double *__restrict__ dirw,
                                                           int ndir, long long n, T *__restrict__ lstar)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if constexpr (sizeof(T) == 4) {  // FP32 inputs: the preconditioner in float
            const float cf = chi[i];
            float lf = 0.f;
            for (int d = 0; d < ndir; ++d) {
                const float x = 0.5f * (float)dirw[2 * d] * cf;  // 1 - q: its series below x = 0.03
                const float om = x < 0.03f ? x * (0.5f - x * (1.f / 6.f - x * (1.f / 24.f))) : 1.f + expm1f(-x) / x;
                lf = fmaf((float)dirw[2 * d + 1], om, lf);
            }
            lstar[i] = lf;
        } else {
            const double c = (double)chi[i];
            double l = 0.0;
            for (int d = 0; d < ndir; ++d) {
                const double x = 0.5 * dirw[2 * d] * c;
                const double q = x < 1e-4 ? 1.0 - 0.5 * x + x * x / 6.0 : -expm1(-x) / x;
                l += dirw[2 * d + 1] * (1.0 - q);
            }
            lstar[i] = (T)l;
        }
    }
}

template <typename A>
__device__ __forceinline__ double acc_val(const A &v)
{
    return rts::acc_to_double(v);
}

// One step of the scattering iteration per band and point:
//   S <- S + [(1 - eps) J_b + eps B - S] / [1 - (1 - eps) L*]
// (J_b of the solve with the current S, from the handle's JF array), and the
// largest |change| / |S| over all points into *dsmax (float bits, atomic max).
template <typename T, typename Acc>
__global__ void __launch_bounds__(256) scatter_update_kernel(const Acc *__restrict__ JF, const T *__restrict__ eps,
                                                              const T *__restrict__ Bp, const T *__restrict__ lstar,
                                                              T *__restrict__ S, long long N, int nb,
                                                              unsigned *dsmax)
{
    float m = 0.f;
    const long long n = N * nb;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / N, p = i - b * N;
        const double J = acc_val(JF[b * 4 * N + p]);
        const double e = (double)eps[i], s = (double)S[i];
        const double num = (1.0 - e) * J + e * (double)Bp[i] - s;
        if constexpr (sizeof(T) == 4) {
            // FP32 S: the residual in double (it cancels), the rest in float
            const float ds = (float)num / (1.f - (1.f - eps[i]) * lstar[i]);
            const float sn = S[i] + ds, den = fabsf(sn);
            S[i] = sn;
            m = fmaxf(m, den > 0.f ? fabsf(ds) / den : (ds != 0.f ? 1.f : 0.f));
        } else {
            const double ds = num / (1.0 - (1.0 - e) * (double)lstar[i]);
            const T sn = (T)(s + ds);
            S[i] = sn;
            const double den = fabs((double)sn);
            m = fmaxf(m, (float)(den > 0.0 ? fabs(ds) / den : (ds != 0.0 ? 1.0 : 0.0)));
        }
    }
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dsmax, __float_as_uint(m));
}

constexpr double kPi = 3.14159265358979323846;
constexpr int kLag = 8;  // planes between posting the seed-error bound and using it

struct DirGeo {
    int axis, sa, b1, b2, s1, s2, up;
    double ds, d1, d2, beta[4];
};

// Geometry of the short characteristic of direction n on spacing h: the
// upwind point r - ds n lies on the nearest grid plane perpendicular to the
// dominant axis; its position on that plane gives bilinear corner weights.
bool direction_geometry(const double h[3], const double n[3], DirGeo &g)
{
    const int order[3] = {2, 1, 0};  // ties resolved towards z, then y
    int a = -1;
    double best = 0;
    for (int t = 0; t < 3; ++t) {
        const int ax = order[t];
        if (n[ax] == 0.0) continue;
        const double s = h[ax] / std::fabs(n[ax]);
        if (a < 0 || s < best) { a = ax; best = s; }
    }
    if (a < 0 || n[2] == 0.0) return false;
    g.axis = a;
    g.sa = n[a] > 0 ? 1 : -1;
    g.b1 = a == 0 ? 1 : 0;
    g.b2 = a == 2 ? 1 : 2;
    g.s1 = n[g.b1] < 0 ? -1 : 1;
    g.s2 = n[g.b2] < 0 ? -1 : 1;
    g.ds = best;
    g.d1 = std::min(1.0, best * std::fabs(n[g.b1]) / h[g.b1]);
    g.d2 = std::min(1.0, best * std::fabs(n[g.b2]) / h[g.b2]);
    g.beta[0] = (1 - g.d1) * (1 - g.d2);
    g.beta[1] = g.d1 * (1 - g.d2);
    g.beta[2] = (1 - g.d1) * g.d2;
    g.beta[3] = g.d1 * g.d2;
    g.up = n[2] > 0;
    return true;
}

// Default angular set: 3 directions per octant, each with two components
// mu1 and one component mu2 = sqrt(1 - 2 mu1^2); mu1^2 = (1 - sqrt(2/5))/3
// makes the set integrate the 4th moment of each axis exactly (S4 level
// symmetric). Order: groups +z, -z, +x, -x, +y, -y, minor signs (+,+),(-,+),(+,-),(-,-).
void default_quadrature(std::vector<double> &n, std::vector<double> &w)
{
    const double m1 = std::sqrt((1.0 - std::sqrt(0.4)) / 3.0);
    const double m2 = std::sqrt(1.0 - 2.0 * m1 * m1);
    const int axis_of[6] = {2, 2, 0, 0, 1, 1};
    n.clear();
    w.clear();
    for (int grp = 0; grp < 6; ++grp) {
        const int ax = axis_of[grp];
        const double sa = grp % 2 == 0 ? 1.0 : -1.0;
        const int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;
        for (int m = 0; m < 4; ++m) {
            double v[3];
            v[ax] = sa * m2;
            v[b1] = (m & 1) ? -m1 : m1;
            v[b2] = (m & 2) ? -m1 : m1;
            n.insert(n.end(), v, v + 3);
            w.push_back(1.0 / 24.0);
        }
    }
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// extents of a group's plane (P, Q) and sweep axis (M)
void unit_extents(int axis, long long nx, long long ny, long long nz, int &NP, int &NQ, int &NM)
{
    if (axis == 2) { NP = (int)nx; NQ = (int)ny; NM = (int)nz; }
    else if (axis == 1) { NP = (int)nx; NQ = (int)nz; NM = (int)ny; }
    else { NP = (int)ny; NQ = (int)nz; NM = (int)nx; }
}

struct PlanOut {
    int nunits = 0, ntiles = 0, max_ntiles = 0;
    long long halo_elems = 0, seed_elems = 0;
    bool has_x = false;
};

// Sweep units of B bands. Per band and per (dominant axis, sign) group --
// the x and y groups first, as their periodic warm-up makes them run longer --
// the group's rays are bucketed by sign slot (sign along P, sign along Q);
// unit u of the group takes the u-th ray of every slot. Writes at most
// max_units units and max_tiles tile -> unit entries (fixed arrays, no
// allocation); returns false if either would overflow.
bool plan_units(const DirGeo *geo, const int *udx, const double *n, const double *w, int ndir, long long nx,
                long long ny, long long nz, int B, int tq, rts::SweepUnit *units, int max_units, int *unit_of_tile,
                int max_tiles, PlanOut &po)
{
    int n_up = 0, n_dn = 0;
    for (int d = 0; d < ndir; ++d) (geo[d].up ? n_up : n_dn)++;
    const int keys[6][2] = {{0, 1}, {0, -1}, {1, 1}, {1, -1}, {2, 1}, {2, -1}};
    const long long N = nx * ny * nz;
    po = PlanOut();
    for (int b = 0; b < B; ++b) {
        for (const auto &k : keys) {
            // rays of this group by slot, in table order
            int cnt[rts::MAXD] = {0, 0, 0, 0}, nunit = 0;
            for (int d = 0; d < ndir; ++d) {
                if (geo[d].axis != k[0] || geo[d].sa != k[1]) continue;
                const int sl = (geo[d].s1 < 0 ? 1 : 0) + (geo[d].s2 < 0 ? 2 : 0);
                nunit = std::max(nunit, ++cnt[sl]);
            }
            for (int u = 0; u < nunit; ++u) {
                if (po.nunits >= max_units) return false;
                rts::SweepUnit &U = units[po.nunits];
                std::memset(&U, 0, sizeof(U));
                U.N = N;
                U.band = b;
                U.in_off = (long long)b * N;
                U.top_off = (long long)b * n_up * nx * ny;
                U.dn_off = (long long)b * n_dn * nx * ny;
                U.axis = k[0];
                U.sa = k[1];
                unit_extents(U.axis, nx, ny, nz, U.NP, U.NQ, U.NM);
                if (U.axis == 2) { U.sQ = nx; U.sM = nx * ny; U.qper = 1; }
                else if (U.axis == 1) { U.sQ = nx * ny; U.sM = nx; U.wrap = 1; }
                else { U.sQ = ny; U.sM = nz * ny; U.wrap = 1; U.transposed = 1; po.has_x = true; }
                U.TQ = tq;
                U.ntiles = (U.NQ + tq - 1) / tq;
                U.tile0 = po.ntiles;
                U.nx = (int)nx;
                U.ny = (int)ny;
                U.halo_off = po.halo_elems;
                int seen[rts::MAXD] = {0, 0, 0, 0};
                for (int sl = 0; sl < rts::MAXD; ++sl) U.up[sl] = U.axis == 2 ? (U.sa > 0) : (sl < 2);
                for (int d = 0; d < ndir; ++d) {
                    if (geo[d].axis != k[0] || geo[d].sa != k[1]) continue;
                    const int sl = (geo[d].s1 < 0 ? 1 : 0) + (geo[d].s2 < 0 ? 2 : 0);
                    if (seen[sl]++ != u) continue;
                    U.active[sl] = 1;
                    for (int cc = 0; cc < 4; ++cc) U.beta[sl][cc] = geo[d].beta[cc];
                    U.ds[sl] = geo[d].ds;
                    U.cJ[sl] = w[d];
                    for (int cc = 0; cc < 3; ++cc) U.cF[cc][sl] = 4.0 * kPi * w[d] * n[3 * d + cc];
                    U.up[sl] = geo[d].up;
                    U.udx[sl] = udx[d];
                }
                U.seed_off = -1;
                if (U.wrap) {  // the unit's wrap plane in the warm-start buffer
                    U.seed_off = po.seed_elems;
                    po.seed_elems += (long long)U.NP * U.NQ * rts::MAXD;
                }
                if (po.ntiles + U.ntiles > max_tiles) return false;
                for (int t = 0; t < U.ntiles; ++t) unit_of_tile[po.ntiles + t] = po.nunits;
                po.ntiles += U.ntiles;
                po.max_ntiles = std::max(po.max_ntiles, U.ntiles);
                // per tile: the shared-memory sweep's ring (4 x HALO_CH x NP) or the
                // register sweep's tagged ring, whichever is larger
                po.halo_elems += (long long)U.ntiles * std::max<long long>(4 * rts::HALO_CH * U.NP, rts::reg_ring_elems(U.NP));
                ++po.nunits;
            }
        }
    }
    return true;
}

}  // namespace

struct rts_handle {
    rts_grid g{};
    int B = 0, ndir = 0, n_up = 0, n_dn = 0;
    std::vector<double> n, w;
    rts_options opt{};
    cudaStream_t stream = nullptr;
    int esize = 8;  // bytes of the sweep precision

    std::vector<rts::SweepUnit> units;
    std::vector<int> unit_of_tile;
    int total_tiles = 0, max_ntiles = 0, R = 0, grid = 0, nt = 32, tq = 0, maxt = 0;  // maxt: register cap
    unsigned carveout = 100;      // forward sweep's shared-memory carveout (percent)
    // batched: one forward launch per CTA-width class (units of plane
    // extents that round up to the same number of warps), tiles contiguous
    struct SweepClass {
        int tile_base = 0, ntiles = 0, nt = 0, grid = 0;
        size_t smem = 0;
        unsigned carveout = 100;
    };
    std::vector<SweepClass> classes;
    unsigned adj_carveout = 100;  // reverse sweep's
    size_t smem = 0;
    // reverse sweep: the same units tiled for the adjoint kernel
    std::vector<rts::SweepUnit> adj_units;
    std::vector<int> adj_unit_of_tile;
    rts::SweepUnit *d_adj_units = nullptr;
    int *d_adj_uot = nullptr;
    int *d_adj_order = nullptr;  // tickets -> tiles of the reverse sweep over all units
    int adj_tq = 0, adj_maxr = 0, adj_total_tiles = 0, adj_max_ntiles = 0;
    // register-resident FP32 forward sweep (sweep_reg.cuh): its own tiling of the same units
    bool use_reg = false;
    long long seed_elems = 0;     // warm-start buffer of the register sweep
    std::vector<rts::SweepUnit> reg_units;
    std::vector<int> reg_unit_of_tile;
    rts::SweepUnit *d_reg_units = nullptr;
    int *d_reg_uot = nullptr;
    int *d_reg_order = nullptr;  // tickets -> tiles of the single-grid register sweep (null: identity)
    int reg_tq = 0, reg_maxr = 0, reg_total_tiles = 0, reg_grid = 0, reg_nt = 32;
    size_t reg_smem = 0;
    unsigned reg_carveout = 100;
    int flag_tiles = 0;           // ready flags allocated (a pair per tile, max over all tilings)
    size_t adj_smem = 0;
    bool has_x = false;
    long long N = 0;

    // device memory (one allocation, carved)
    void *dmem = nullptr;
    void *d_chi_exp = nullptr;    // RTS_FLAG_LOG_CHI: exp(log chi) of the current call
    // RTS_FLAG_SCATTER: the local operator of every band and point, the
    // per-direction path lengths and weights it is formed from, the iteration's
    // largest relative change of S
    void *d_lstar = nullptr;
    double *d_dirw = nullptr;     // [n_lsd][2]: a segment length ds and the summed weight of its directions
    int n_lsd = 0;
    unsigned *d_dsmax = nullptr;
    rts::SweepUnit *d_units = nullptr;
    int *d_unit_of_tile = nullptr;
    void *d_partial = nullptr, *d_chiT = nullptr, *d_ST = nullptr, *d_JF = nullptr, *d_halo = nullptr;
    int *d_flags = nullptr, *d_ticket = nullptr, *d_status = nullptr, *d_unit_tacc = nullptr;
    unsigned int *d_gcnt = nullptr;
    unsigned long long *d_gmax = nullptr;
    rts::RedUnit *d_ru = nullptr;
    int *d_ru_begin = nullptr;
    bool qf_ok = false;  // the register sweep's reduction (qfused.cuh) is used
    int reg_grid_seed = 0;       // grid and carveout of the warm-start instantiation (0: none fits)
    unsigned reg_carveout_seed = 100;
    int reg_grid_ck = 0;         // grid and carveout of the adjoint's checkpoint instantiation (0: none fits)
    unsigned reg_carveout_ck = 100;
    size_t qr_smem = 0;
    int qr_grid = 0, qr_max_nat = 0, qr_max_x = 0;
    rts::RedUnit *d_qfu = nullptr;  // its units: per band the x groups first
    int *d_qfb = nullptr;           // band begins [B+1], the ends of each band's x groups [B], of its y units [B]
    // adjoint scratch (RTS_FLAG_ADJOINT): lam0 [B][N][4] natural and
    // x-transposed, direct Q-step terms [B][2][N], and per checkpoint chunk of
    // at most chunk_units units: the checkpoint [u][N][STORE_CH*4] and the
    // gradient terms [u][GRAD_CH][N]
    void *d_lam0 = nullptr, *d_lam0T = nullptr, *d_direct = nullptr;
    void *d_ckpt = nullptr, *d_grad = nullptr;
    int chunk_bands = 1, chunk_units = 0, grid_adj = 0;
    std::vector<int> band_unit;   // first unit of band b (b = 0..B)
    // batched handles (rts_create_batched): subdomain table and packed sizes
    bool batched = false;
    int nsub = 1;
    std::vector<rts::SubDesc> subs;
    rts::SubDesc *d_subs = nullptr;
    long long in_total = 0, top_total = 0, out_total = 0, nblk[3] = {0, 0, 0};
    bool capturing = false;
    // host-IO staging
    void *d_in_chi = nullptr, *d_in_S = nullptr, *d_out_itop = nullptr;
    double *d_out_J = nullptr, *d_out_F = nullptr, *d_out_Q = nullptr;
    // RTS_FLAG_HOST_IO_ASYNC: two staging sets (inputs chi, S; outputs I_top,
    // J, F, Q), an input and an output copy stream, and per set the events
    // "inputs copied", "solve done" and "outputs copied"
    void *a_in[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    void *a_out[2][4] = {{nullptr, nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr, nullptr}};
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_h2d[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_d2h[2] = {nullptr, nullptr};
    bool a_used[2] = {false, false};
    int a_next = 0;

    // RTS_FLAG_TIMING: one set of phase events per solve since the last stats call
    bool timing = false;
    std::vector<std::array<cudaEvent_t, 5>> evs;
    size_t nrec = 0;
    // adjoint phases: events in recording order and the phase each interval ends
    std::vector<cudaEvent_t> adj_evs;
    std::vector<int> adj_phase;
    size_t adj_nev = 0;
    int adj_calls = 0;
    int kernels_last = 0;

    char err[512] = {0};
};

static rts_status fail(rts_handle *h, rts_status s, const char *fmt, ...)
{
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define CUDA_TRY(h, call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fail(h, RTS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
using SweepFn = rts::SweepFn<T>;

// Forward sweep kernels instantiated: (rows per tile, register cap per thread).
// The caps let 2 to 4 CTAs of up to 288 threads share an SM; the last three
// serve CTAs of up to 1024 threads (plane extents above 384). The kernels are
// compiled in their own translation units (sweep_f32.cu, sweep_f64.cu,
// adj_f32.cu, adj_f64.cu) and looked up here by configuration.
struct FwdCfg {
    int tq, maxr;
};
static const FwdCfg kFwdCfg[] = {{16, 168}, {12, 168}, {8, 112}, {7, 112}, {6, 104}, {4, 72}, {2, 56}, {1, 56},
                                 {4, 64}, {2, 64}, {1, 64}};
static const int kNumFwdCfg = sizeof(kFwdCfg) / sizeof(kFwdCfg[0]);
template <typename T>
static SweepFn<T> fwd_kernel(int tq, int maxr, bool ckpt = false);
template <>
SweepFn<float> fwd_kernel<float>(int tq, int maxr, bool ckpt)
{
    return rts::fwd_kernel_f32(tq, maxr, ckpt);
}
template <>
SweepFn<double> fwd_kernel<double>(int tq, int maxr, bool ckpt)
{
    return rts::fwd_kernel_f64(tq, maxr, ckpt);
}

template <typename T>
static SweepFn<T> adj_kernel(int tq, int maxr);
template <>
SweepFn<float> adj_kernel<float>(int tq, int maxr)
{
    return rts::adj_kernel_f32(tq, maxr);
}
template <>
SweepFn<double> adj_kernel<double>(int tq, int maxr)
{
    return rts::adj_kernel_f64(tq, maxr);
}

static size_t fwd_smem(int tq, int np, int esize)
{
    return esize == 8 ? rts::tile_smem_bytes<double>(tq, np) : rts::tile_smem_bytes<float>(tq, np);
}

static size_t adj_smem(int tq, int np, int esize)
{
    return esize == 8 ? rts::adj_tile_smem_bytes<double>(tq, np) : rts::adj_tile_smem_bytes<float>(tq, np);
}

struct Tiling {
    int tq = 0, nt = 32, maxt = 0, blocks = 0;  // maxt: register cap of the forward kernel
    size_t smem = 0;
};

// Shared-memory carveout (percent of the SM's maximum) that holds `blocks`
// CTAs of `smem` dynamic bytes each, with room for the kernel's static shared
// memory and the per-CTA reservation. The rest of the SM's L1/shared storage
// stays L1 cache, where register spills and the cp.async lines live.
// Shared-memory carveout (percent) that holds `blocks` CTAs of kernel `kern`
// with `smem` dynamic bytes: per CTA the dynamic and the kernel's static
// shared memory and the 1 KB the hardware reserves, plus 1 KB of margin. A
// cooperative launch sized for `blocks` CTAs per SM needs every one of them
// resident, so the carveout must not be smaller.
static unsigned carveout_percent(int blocks, size_t smem, const void *kern)
{
    int dev = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        per_sm <= 0)
        return 100;
    cudaFuncAttributes fa;
    size_t st = 8192;  // when the attributes cannot be read: more than any of the sweeps' static arrays
    if (kern && cudaFuncGetAttributes(&fa, kern) == cudaSuccess) st = fa.sharedSizeBytes;
    cudaGetLastError();
    const double need = (double)blocks * ((double)smem + (double)st + 2048.0);
    const int pct = (int)std::ceil(100.0 * need / per_sm);
    return (unsigned)std::min(100, std::max(1, pct));
}

template <typename T>
static cudaError_t kernel_occupancy(SweepFn<T> kern, int nt, size_t smem, int *blocks)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, nt, smem);
}

// Forward tiling for plane extents up to npmax and units of up to
// ceil(nqmax / tq) tiles. Candidates are the instantiated (rows, register cap)
// pairs whose cap fits the CTA size. With `requested` > 0: the tallest tile
// not above it that fits. Otherwise the score is the plane rows resident per
// SM, halved when only one CTA fits (one CTA cannot hide its own barrier and
// neighbour waits) and quartered for tiles taller than 4 rows. Every unit's tiles must fit on the GPU at once (the
// persistent launch waits on neighbours).
template <typename T>
static Tiling choose_fwd(int requested, int npmax, int nqmax, int nsm, bool ckpt = false)
{
    Tiling best;
    best.nt = 32 * ((npmax + 31) / 32);
    double best_score = -1;
    for (int i = 0; i < kNumFwdCfg; ++i) {
        const int tq = kFwdCfg[i].tq, maxr = kFwdCfg[i].maxr;
        if ((long long)maxr * best.nt > 65536) continue;
        if (requested > 0 && tq > requested) continue;
        if (ckpt && !fwd_kernel<T>(tq, maxr, true)) continue;  // the adjoint re-sweeps with this tiling
        const size_t smem = fwd_smem(tq, npmax, (int)sizeof(T));
        if (smem > 227 * 1024) continue;
        int blocks = 0;
        if (kernel_occupancy<T>(fwd_kernel<T>(tq, maxr), best.nt, smem, &blocks) != cudaSuccess || blocks < 1)
            continue;
        if ((long long)blocks * nsm < (nqmax + tq - 1) / tq) continue;
        // Measured on B300 (rts288x4 and the batched workload): tiles taller than
        // 4 rows lose more to instruction fetch (their unrolled row code) than
        // they gain in resident rows, so they are only taken on request.
        double score = (double)tq * blocks * (blocks > 1 ? 1.0 : 0.5) * (tq <= 4 ? 1.0 : 0.25);
        if (requested > 0) score = tq;  // tallest fitting tile
        if (score > best_score) {
            best_score = score;
            best.tq = tq;
            best.maxt = maxr;
            best.blocks = blocks;
            best.smem = smem;
        }
    }
    return best;
}

// reverse-sweep tiling: among the instantiated (rows, register cap) pairs
// (4,72), (2,56), (1,56) for CTAs up to 384 threads and (4,64), (2,64),
// (1,64) above, the one that keeps the most plane rows resident per SM
template <typename T>
static Tiling choose_adj(int npmax, int nqmax, int nsm)
{
    static const int cfg[6][2] = {{4, 72}, {2, 56}, {1, 56}, {4, 64}, {2, 64}, {1, 64}};
    Tiling best;
    best.nt = 32 * ((npmax + 31) / 32);
    long long best_rows = -1;
    for (const auto &cf : cfg) {
        const int tq = cf[0], maxr = cf[1];
        if ((long long)maxr * best.nt > 65536) continue;
        const size_t smem = adj_smem(tq, npmax, (int)sizeof(T));
        if (smem > 227 * 1024) continue;
        int blocks = 0;
        if (kernel_occupancy<T>(adj_kernel<T>(tq, maxr), best.nt, smem, &blocks) != cudaSuccess || blocks < 1) continue;
        if ((long long)blocks * nsm < (nqmax + tq - 1) / tq) continue;
        const long long rows = (long long)tq * blocks;
        if (rows > best_rows) {
            best_rows = rows;
            best.tq = tq;
            best.maxt = maxr;
            best.blocks = blocks;
            best.smem = smem;
        }
    }
    return best;
}

// reduction table entry of a unit: its partial array, layout and the per-slot
// coefficients of J and F (used when the partials are raw slot intensities)
static rts::RedUnit red_unit(const rts::SweepUnit &U)
{
    rts::RedUnit r;
    std::memset(&r, 0, sizeof(r));
    r.partial = U.partial;
    r.axis = U.axis;
    for (int d = 0; d < rts::MAXD; ++d) {
        if (!U.active[d]) continue;
        r.c[0][d] = (float)U.cJ[d];
        for (int c = 0; c < 3; ++c) r.c[1 + c][d] = (float)U.cF[c][d];
    }
    // the flux component along the unit's Q axis pairs the slots that differ in sQ
    const int b2 = U.axis == 2 ? 1 : 2;
    r.qpair[1 + b2] = 1;
    return r;
}

// The register-resident sweep serves a grid when every unit's active slots
// share one stencil (path length and bilinear weights), every plane extent is
// even and at most 2048, and (for the row tiles of the periodic z groups) the
// tile height divides ny.
static bool reg_eligible(const std::vector<rts::SweepUnit> &units)
{
    for (const rts::SweepUnit &U : units) {
        if (U.NP % 2 != 0 || U.NP > 2048 || U.NM < 2) return false;
        if (U.N >= (1LL << 31)) return false;  // the kernel's in-band offsets are 32-bit
        int f = -1;
        for (int d = 0; d < rts::MAXD; ++d) {
            if (!U.active[d]) continue;
            if (f < 0) { f = d; continue; }
            if (U.ds[d] != U.ds[f]) return false;
            for (int c = 0; c < 4; ++c)
                if (U.beta[d][c] != U.beta[f][c]) return false;
        }
    }
    return true;
}

// Ticket order of a persistent sweep launch: units by decreasing planes
// per tile (a periodic x/y unit counted twice for its warm-up), each unit's
// tiles together -- the long tiles start first and the short ones fill the
// end of the launch.
static std::vector<int> ticket_order(const std::vector<rts::SweepUnit> &units)
{
    std::vector<int> idx(units.size());
    std::iota(idx.begin(), idx.end(), 0);
    auto key = [&](int u) { return (long long)units[u].NM * (units[u].wrap ? 2 : 1); };
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return key(a) > key(b); });
    std::vector<int> order;
    for (int u : idx)
        for (int t = 0; t < units[u].ntiles; ++t) order.push_back(units[u].tile0 + t);
    return order;
}

struct RegCfg {
    int tq, maxr;
};
// (rows, register cap): measured at 288^3 x 4 bands, 4 rows at 128 registers
// (3 CTAs of 160 threads per SM) is the fastest; 2 rows at 96 registers (4
// CTAs per SM) serve grids whose periodic rows are not a multiple of 4
// (13.7 against 13.5 ms at 288^3 x 4, the same outputs).
static const RegCfg kRegCfg[] = {{8, 255}, {4, 168}, {4, 128}, {2, 96}};

// Tiling of the register-resident sweep: among the instantiated (rows,
// register cap) pairs whose tile height divides the periodic rows (nq_per),
// whose CTA fits and whose units' tiles all fit on the GPU at once, the one
// with the most plane rows resident per SM (requested > 0: the tallest not
// above it, at least 2 rows).
static Tiling choose_reg(int requested, int npmax, int nqmax, int nq_per, int nsm)
{
    Tiling best;
    best.nt = 32 * ((npmax / 2 + 31) / 32);
    double best_score = -1;
    for (const RegCfg &c : kRegCfg) {
        if (requested > 0 && c.tq > std::max(requested, 2)) continue;  // 2 rows is the smallest tile
        if (nq_per % c.tq != 0) continue;
        if ((long long)c.maxr * best.nt > 65536) continue;
        const size_t smem = rts::reg_tile_smem_bytes(c.tq, npmax);
        if (smem > 200 * 1024) continue;
        rts::SweepFn<float> k = rts::reg_kernel_f32(c.tq, c.maxr);
        int blocks = 0;
        if (!k || kernel_occupancy<float>(k, best.nt, smem, &blocks) != cudaSuccess || blocks < 1) continue;
        if ((long long)blocks * nsm < (nqmax + c.tq - 1) / c.tq) continue;
        double score = (double)c.tq * blocks;
        if (requested > 0) score = c.tq + 1e-3 * blocks;
        if (score > best_score) {
            best_score = score;
            best.tq = c.tq;
            best.maxt = c.maxr;
            best.blocks = blocks;
            best.smem = smem;
        }
    }
    return best;
}

template <typename T>
static cudaError_t launch_sweep(rts_handle *h, const rts::SweepArgs<T> &a, bool reverse = false)
{
    SweepFn<T> kern = reverse ? adj_kernel<T>(h->adj_tq, h->adj_maxr) : fwd_kernel<T>(h->tq, h->maxt, a.store != nullptr);
    const size_t smem = reverse ? h->adj_smem : h->smem;
    if (!kern) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::min(reverse ? h->grid_adj : h->grid, a.total_tiles));
    cfg.blockDim = dim3(h->nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs co-resident
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    attr[1].val.sharedMemCarveout = reverse ? h->adj_carveout : h->carveout;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

// the register-resident FP32 forward sweep over all units (its own tiling)
static cudaError_t launch_reg_sweep(rts_handle *h, rts::SweepArgs<float> a)
{
    const bool sd = a.seed != nullptr && a.seed_in != 0;  // warm start: its own instantiation
    rts::SweepFn<float> kern = rts::reg_kernel_f32(h->reg_tq, h->reg_maxr, sd);
    if (!kern || (sd && h->reg_grid_seed < 1)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->reg_smem);
    if (e != cudaSuccess) return e;
    a.units = h->d_reg_units;
    a.unit_of_tile = h->d_reg_uot;
    a.tile_order = h->d_reg_order;
    a.tile_base = 0;
    a.total_tiles = h->reg_total_tiles;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::min(sd ? h->reg_grid_seed : h->reg_grid, a.total_tiles));
    cfg.blockDim = dim3(h->reg_nt);
    cfg.dynamicSmemBytes = h->reg_smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs co-resident
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    attr[1].val.sharedMemCarveout = sd ? h->reg_carveout_seed : h->reg_carveout;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

// the register sweep's checkpoint instantiation over units u0 .. u1-1 (one
// chunk of bands of rts_adjoint): raw slot intensities and D = dI/d(dtau)
static cudaError_t launch_reg_ckpt(rts_handle *h, rts::SweepArgs<float> a, int u0, int u1)
{
    rts::SweepFn<float> kern = rts::reg_kernel_f32(h->reg_tq, h->reg_maxr, false, true);
    if (!kern || h->reg_grid_ck < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->reg_smem);
    if (e != cudaSuccess) return e;
    const rts::SweepUnit &U0 = h->reg_units[u0], &U1 = h->reg_units[u1 - 1];
    a.units = h->d_reg_units;
    a.unit_of_tile = h->d_reg_uot;
    a.tile_order = (u0 == 0 && u1 == (int)h->reg_units.size()) ? h->d_reg_order : nullptr;
    a.unit_base = u0;
    a.tile_base = U0.tile0;
    a.total_tiles = U1.tile0 + U1.ntiles - U0.tile0;
    a.seed = nullptr;
    a.seed_in = 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::min(h->reg_grid_ck, a.total_tiles));
    cfg.blockDim = dim3(h->reg_nt);
    cfg.dynamicSmemBytes = h->reg_smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs co-resident
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    attr[1].val.sharedMemCarveout = h->reg_carveout_ck;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

// Batched forward sweep: one cooperative launch per CTA-width class (a single
// class is the plain launch). Each class's CTA has as many threads as its
// widest plane needs, so narrow subdomains leave no idle warps; the ticket is
// cleared between the launches, flags and counters are per tile and unit.
template <typename T>
static cudaError_t launch_sweep_classes(rts_handle *h, const rts::SweepArgs<T> &a, int *launches)
{
    if (h->classes.size() <= 1) {
        *launches = 1;
        return launch_sweep<T>(h, a);
    }
    SweepFn<T> kern = fwd_kernel<T>(h->tq, h->maxt, false);
    if (!kern) return cudaErrorInvalidValue;
    *launches = 0;
    for (size_t c = 0; c < h->classes.size(); ++c) {
        const rts_handle::SweepClass &C = h->classes[c];
        cudaError_t e;
        if (c > 0 && (e = cudaMemsetAsync(h->d_ticket, 0, sizeof(int), h->stream)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C.smem)) != cudaSuccess)
            return e;
        rts::SweepArgs<T> ac = a;
        ac.tile_base = C.tile_base;
        ac.total_tiles = C.ntiles;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(std::min(C.grid, C.ntiles));
        cfg.blockDim = dim3(C.nt);
        cfg.dynamicSmemBytes = C.smem;
        cfg.stream = h->stream;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        attr[1].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
        attr[1].val.sharedMemCarveout = C.carveout;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        if ((e = cudaLaunchKernelEx(&cfg, kern, ac)) != cudaSuccess) return e;
        ++*launches;
    }
    return cudaSuccess;
}

// occupancy of the forward kernel (tq, register cap) with nt threads and smem bytes
static cudaError_t class_blocks(int esize, int tq, int maxt, int nt, size_t smem, int *blocks)
{
    return esize == 8 ? kernel_occupancy<double>(fwd_kernel<double>(tq, maxt, false), nt, smem, blocks)
                      : kernel_occupancy<float>(fwd_kernel<float>(tq, maxt, false), nt, smem, blocks);
}

extern "C" {

void rts_default_options(rts_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->prec = RTS_FP64;
    o->tau_switch = 0.1;
    o->wrap_tol = 0.0;  // 0 = precision default
    o->max_wrap_iters = 64;
    o->timeout_s = 2.0;
}

const char *rts_last_error(rts_handle *h) { return h ? h->err : "null handle"; }

int rts_num_up(rts_handle *h) { return h ? h->n_up : 0; }

static void free_all(rts_handle *h)
{
    if (h->s_h2d) cudaStreamSynchronize(h->s_h2d);
    if (h->s_d2h) cudaStreamSynchronize(h->s_d2h);
    for (int i = 0; i < 2; ++i) {
        if (h->ev_h2d[i]) cudaEventDestroy(h->ev_h2d[i]);
        if (h->ev_comp[i]) cudaEventDestroy(h->ev_comp[i]);
        if (h->ev_d2h[i]) cudaEventDestroy(h->ev_d2h[i]);
        h->ev_h2d[i] = h->ev_comp[i] = h->ev_d2h[i] = nullptr;
    }
    if (h->s_h2d) cudaStreamDestroy(h->s_h2d);
    if (h->s_d2h) cudaStreamDestroy(h->s_d2h);
    h->s_h2d = h->s_d2h = nullptr;
    if (h->dmem) cudaFree(h->dmem);
    h->dmem = nullptr;
    for (cudaEvent_t e : h->adj_evs)
        if (e) cudaEventDestroy(e);
    h->adj_evs.clear();
    for (auto &set : h->evs)
        for (cudaEvent_t e : set)
            if (e) cudaEventDestroy(e);
    h->evs.clear();
}

void rts_destroy(rts_handle *h)
{
    if (!h) return;
    free_all(h);
    delete h;
}

rts_status rts_create(rts_handle **out, const rts_grid *g, int nbands, const rts_quadrature *q,
                      const rts_options *opt)
{
    if (!out) return RTS_EINVAL;
    *out = nullptr;
    rts_handle *h = new (std::nothrow) rts_handle();
    if (!h) return RTS_ENOMEM;
    if (opt) h->opt = *opt;
    else rts_default_options(&h->opt);
    rts_options &o = h->opt;
    auto bail = [&](rts_status s) {
        // keep the handle so the caller can read the error text
        *out = h;
        return s;
    };
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 2 || nbands < 1)
        return bail(fail(h, RTS_EINVAL, "grid must have nx, ny >= 1, nz >= 2 and nbands >= 1"));
    if (!(g->dx > 0 && g->dy > 0 && g->dz > 0) || !std::isfinite(g->dx) || !std::isfinite(g->dy) ||
        !std::isfinite(g->dz))
        return bail(fail(h, RTS_EINVAL, "grid spacing must be finite and positive"));
    if (o.prec != RTS_FP64 && o.prec != RTS_FP32_MIXED && o.prec != RTS_FP32_COMPENSATED)
        return bail(fail(h, RTS_EINVAL, "unknown precision %d", (int)o.prec));
    if (!(o.tau_switch > 0)) return bail(fail(h, RTS_EINVAL, "tau_switch must be > 0"));
    if (o.max_wrap_iters < 1) o.max_wrap_iters = 64;
    if (!(o.timeout_s > 0)) o.timeout_s = 2.0;
    if (!(o.wrap_tol > 0)) o.wrap_tol = o.prec == RTS_FP64 ? 1e-15 : 0x1p-24;
    h->g = *g;
    h->B = nbands;
    h->stream = (cudaStream_t)o.stream;
    h->esize = o.prec == RTS_FP64 ? 8 : 4;

    if (q && q->ndir > 0) {
        if (!q->n || !q->w) return bail(fail(h, RTS_EINVAL, "quadrature arrays are NULL"));
        h->n.assign(q->n, q->n + 3 * q->ndir);
        h->w.assign(q->w, q->w + q->ndir);
    } else {
        default_quadrature(h->n, h->w);
    }
    h->ndir = (int)h->w.size();
    const double hsp[3] = {g->dx, g->dy, g->dz};
    std::vector<DirGeo> geo(h->ndir);
    std::vector<int> udx(h->ndir);
    for (int d = 0; d < h->ndir; ++d) {
        if (!direction_geometry(hsp, &h->n[3 * d], geo[d]))
            return bail(fail(h, RTS_EINVAL, "direction %d has n_z == 0 or is zero", d));
        udx[d] = geo[d].up ? h->n_up++ : h->n_dn++;
    }

    const long long nx = g->nx, ny = g->ny, nz = g->nz;
    h->N = nx * ny * nz;
    if (nz * nbands > 65535)  // the transposes and reductions launch one CTA layer per (band, level)
        return bail(fail(h, RTS_EINVAL, "nz * nbands = %lld exceeds 65535", nz * (long long)nbands));

    // ---- sweep units and tiling ----
    int npmax = 0;
    for (int d = 0; d < h->ndir; ++d) {
        int NP, NQ, NM;
        unit_extents(geo[d].axis, nx, ny, nz, NP, NQ, NM);
        npmax = std::max(npmax, NP);
    }
    if (npmax > 1024) return bail(fail(h, RTS_EINVAL, "plane extent %d > 1024 is not supported", npmax));
    const int nqmax = (int)std::max(ny, nz);
    int dev = 0, nsm = 0;
    CUDA_TRY(h, cudaGetDevice(&dev));
    CUDA_TRY(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const bool want_adj = (o.flags & RTS_FLAG_ADJOINT) != 0;
    const Tiling tl = o.prec == RTS_FP64 ? choose_fwd<double>(o.tile_rows, npmax, nqmax, nsm, want_adj)
                                         : choose_fwd<float>(o.tile_rows, npmax, nqmax, nsm, want_adj);
    if (tl.tq < 1) return bail(fail(h, RTS_EINVAL, "no sweep tile fits plane extent %d with %d-row units", npmax, nqmax));
    const int tq = tl.tq;
    h->tq = tq;
    h->nt = tl.nt;
    h->maxt = tl.maxt;
    h->smem = tl.smem;
    h->carveout = carveout_percent(tl.blocks, tl.smem,
                                   o.prec == RTS_FP64 ? (const void *)fwd_kernel<double>(tq, tl.maxt)
                                                      : (const void *)fwd_kernel<float>(tq, tl.maxt));
    const int max_units = nbands * 6 * h->ndir;
    const long long max_tiles = (long long)max_units * std::max(nx, std::max(ny, nz));  // tiles of >= 1 row
    h->units.resize(max_units);
    h->unit_of_tile.resize(max_tiles);
    PlanOut po;
    if (!plan_units(geo.data(), udx.data(), h->n.data(), h->w.data(), h->ndir, nx, ny, nz, nbands, tq,
                    h->units.data(), max_units, h->unit_of_tile.data(), (int)max_tiles, po))
        return bail(fail(h, RTS_EINVAL, "too many sweep units or tiles"));
    h->units.resize(po.nunits);
    h->unit_of_tile.resize(po.ntiles);
    h->has_x = po.has_x;
    h->max_ntiles = po.max_ntiles;
    long long halo_elems = po.halo_elems;
    h->total_tiles = po.ntiles;
    h->grid = std::min(h->total_tiles, tl.blocks * nsm);

    const bool adjoint = (o.flags & RTS_FLAG_ADJOINT) != 0;
    h->band_unit.assign(nbands + 1, 0);
    for (size_t u = 0; u < h->units.size(); ++u) h->band_unit[h->units[u].band + 1]++;
    for (int b = 0; b < nbands; ++b) h->band_unit[b + 1] += h->band_unit[b];
    int flag_tiles = 2 * h->total_tiles, max_nt = h->max_ntiles;  // forward: a pair per tile
    if (adjoint) {
        if (o.adjoint_chunk_bands > 0) {
            h->chunk_bands = std::min(nbands, o.adjoint_chunk_bands);
        } else {
            // automatic: as many bands per checkpoint as fit in 85 % of the free
            // device memory next to the handle's other arrays (more bands at once
            // keep more sweep units resident; measured on B300, 4-band chunks run
            // the 288^3 x 4 adjoint in 0.88 and the 96^3 x 4 one in 0.56 of the
            // 1-band time), split into equal chunks
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = 0;
            cudaGetLastError();
            int upb = 0;
            for (int b = 0; b < nbands; ++b) upb = std::max(upb, h->band_unit[b + 1] - h->band_unit[b]);
            const double es_ = (double)h->esize, Nd = (double)h->N, Bd = (double)nbands;
            const double per_band = (double)upb * (rts::STORE_CH * rts::MAXD + rts::GRAD_CH) * Nd * es_;
            // partials, transposed inputs, J_b/F_b, lam0 (and its transpose), direct terms, exp(log chi)
            const double others = (double)h->units.size() * 4 * Nd * es_ + (h->has_x ? 2 * Bd * Nd * es_ : 0.0) +
                                  Bd * 4 * Nd * 8 + Bd * 4 * Nd * es_ * (h->has_x ? 2 : 1) + Bd * 2 * Nd * es_ +
                                  ((o.flags & RTS_FLAG_LOG_CHI) ? Bd * Nd * es_ : 0.0);
            const double room = 0.85 * (double)fr - others;
            const int fit = per_band > 0 ? (int)std::max(1.0, std::min<double>(nbands, room / per_band)) : nbands;
            const int nchunks = (nbands + std::max(1, fit) - 1) / std::max(1, fit);
            h->chunk_bands = (nbands + nchunks - 1) / nchunks;
        }
        for (int b = 0; b < nbands; b += h->chunk_bands) {
            const int b1 = std::min(nbands, b + h->chunk_bands);
            h->chunk_units = std::max(h->chunk_units, h->band_unit[b1] - h->band_unit[b]);
        }
        const Tiling ta = o.prec == RTS_FP64 ? choose_adj<double>(npmax, nqmax, nsm) : choose_adj<float>(npmax, nqmax, nsm);
        if (ta.tq < 1) return bail(fail(h, RTS_EINVAL, "no reverse-sweep tile fits plane extent %d", npmax));
        h->adj_tq = ta.tq;
        h->adj_maxr = ta.maxt;
        h->adj_smem = ta.smem;
        h->adj_carveout = carveout_percent(ta.blocks, ta.smem,
                                           o.prec == RTS_FP64 ? (const void *)adj_kernel<double>(ta.tq, ta.maxt)
                                                              : (const void *)adj_kernel<float>(ta.tq, ta.maxt));
        h->adj_units.resize(max_units);
        h->adj_unit_of_tile.resize(max_tiles);
        PlanOut pa;
        if (!plan_units(geo.data(), udx.data(), h->n.data(), h->w.data(), h->ndir, nx, ny, nz, nbands, ta.tq,
                        h->adj_units.data(), max_units, h->adj_unit_of_tile.data(), (int)max_tiles, pa) ||
            pa.nunits != po.nunits)
            return bail(fail(h, RTS_EINVAL, "too many reverse-sweep tiles"));
        h->adj_units.resize(pa.nunits);
        h->adj_unit_of_tile.resize(pa.ntiles);
        h->adj_total_tiles = pa.ntiles;
        h->adj_max_ntiles = pa.max_ntiles;
        h->grid_adj = std::min(pa.ntiles, ta.blocks * nsm);
        halo_elems = std::max(halo_elems, pa.halo_elems);
        flag_tiles = std::max(flag_tiles, 2 * pa.ntiles);
        max_nt = std::max(max_nt, pa.max_ntiles);
    }
    // register-resident forward sweep (FP32): its own tiling of the same units
    if (o.sweep_kernel < RTS_SWEEP_AUTO || o.sweep_kernel > RTS_SWEEP_REGISTER)
        return bail(fail(h, RTS_EINVAL, "unknown sweep_kernel %d", o.sweep_kernel));
    if (o.prec == RTS_FP64 && o.sweep_kernel == RTS_SWEEP_REGISTER)
        return bail(fail(h, RTS_EINVAL, "the register sweep is FP32 only"));
    if (o.prec != RTS_FP64 && o.sweep_kernel != RTS_SWEEP_SHARED) {
        const bool elig = reg_eligible(h->units);
        Tiling tr;
        if (elig) tr = choose_reg(o.tile_rows, npmax, nqmax, (int)ny, nsm);
        if (tr.tq >= 1) {
            h->reg_units.resize(max_units);
            h->reg_unit_of_tile.resize(max_tiles);
            PlanOut pr;
            if (!plan_units(geo.data(), udx.data(), h->n.data(), h->w.data(), h->ndir, nx, ny, nz, nbands, tr.tq,
                            h->reg_units.data(), max_units, h->reg_unit_of_tile.data(), (int)max_tiles, pr) ||
                pr.nunits != po.nunits)
                return bail(fail(h, RTS_EINVAL, "too many register-sweep tiles"));
            h->reg_units.resize(pr.nunits);
            h->reg_unit_of_tile.resize(pr.ntiles);
            h->reg_total_tiles = pr.ntiles;
            h->reg_tq = tr.tq;
            h->reg_maxr = tr.maxt;
            h->reg_nt = tr.nt;
            h->reg_smem = tr.smem;
            h->reg_carveout = carveout_percent(tr.blocks, tr.smem, (const void *)rts::reg_kernel_f32(tr.tq, tr.maxt));
            h->reg_grid = std::min(pr.ntiles, tr.blocks * nsm);
            {  // the warm-start instantiation (more static shared memory): its own residency
                rts::SweepFn<float> ks = rts::reg_kernel_f32(tr.tq, tr.maxt, true);
                int bs = 0;
                if (ks && kernel_occupancy<float>(ks, tr.nt, tr.smem, &bs) == cudaSuccess && bs > 0 &&
                    (long long)bs * nsm >= pr.max_ntiles) {
                    h->reg_grid_seed = std::min(pr.ntiles, bs * nsm);
                    h->reg_carveout_seed = carveout_percent(bs, tr.smem, (const void *)ks);
                }
                cudaGetLastError();
            }
            if (want_adj) {  // the adjoint's checkpoint instantiation: its own residency
                rts::SweepFn<float> kc = rts::reg_kernel_f32(tr.tq, tr.maxt, false, true);
                int bc = 0;
                if (kc && kernel_occupancy<float>(kc, tr.nt, tr.smem, &bc) == cudaSuccess && bc > 0 &&
                    (long long)bc * nsm >= pr.max_ntiles) {
                    h->reg_grid_ck = std::min(pr.ntiles, bc * nsm);
                    h->reg_carveout_ck = carveout_percent(bc, tr.smem, (const void *)kc);
                }
                cudaGetLastError();
            }
            h->seed_elems = pr.seed_elems;
            halo_elems = std::max(halo_elems, pr.halo_elems);
            flag_tiles = std::max(flag_tiles, 2 * pr.ntiles);
            max_nt = std::max(max_nt, pr.max_ntiles);
            h->use_reg = true;
        } else if (o.sweep_kernel == RTS_SWEEP_REGISTER) {
            return bail(fail(h, RTS_EINVAL,
                             elig ? "no register-sweep tile fits this grid (the tile height must divide ny)"
                                  : "the register sweep needs even nx, ny and one stencil per direction group"));
        }
    }
    h->flag_tiles = flag_tiles;
    int R = 8;
    while (R < 2 * (max_nt + kLag + 2)) R *= 2;
    h->R = R;

    // ---- device memory ----
    const size_t es = h->esize;
    const size_t accsz = 8;  // double or df32
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = round_up(off + bytes, 256); return at; };
    const size_t o_units = take(sizeof(rts::SweepUnit) * h->units.size());
    const size_t o_uot = take(sizeof(int) * h->unit_of_tile.size());
    const size_t o_part = take((size_t)h->units.size() * 4 * h->N * es);
    const size_t o_chiT = h->has_x ? take((size_t)nbands * h->N * es) : 0;
    const size_t o_ST = h->has_x ? take((size_t)nbands * h->N * es) : 0;
    const size_t o_JF = take((size_t)nbands * 4 * h->N * accsz);
    const size_t o_halo = take((size_t)halo_elems * es);
    const size_t o_flags = take(sizeof(int) * flag_tiles);
    // per unit: R plane slots, then 4 period slots (the warm start's residual)
    const size_t o_gcnt = take(sizeof(unsigned int) * h->units.size() * (R + 4));
    const size_t o_gmax = take(sizeof(unsigned long long) * h->units.size() * (R + 4));
    const size_t o_ticket = take(sizeof(int) * 4);
    const size_t o_status = take(sizeof(int) * 4);
    const size_t o_tacc = take(sizeof(int) * h->units.size());
    const size_t o_ru = take(sizeof(rts::RedUnit) * h->units.size());
    const size_t o_rub = take(sizeof(int) * (nbands + 1));
    const size_t o_qfu = take(sizeof(rts::RedUnit) * h->units.size());
    const size_t o_qfb = take(sizeof(int) * (3 * nbands + 1));
    const bool log_chi = (o.flags & RTS_FLAG_LOG_CHI) != 0;
    const size_t o_cexp = log_chi ? take((size_t)nbands * h->N * es) : 0;
    const bool scatter = (o.flags & RTS_FLAG_SCATTER) != 0;
    const size_t o_lstar = scatter ? take((size_t)nbands * h->N * es) : 0;
    const size_t o_dirw = scatter ? take(sizeof(double) * 2 * h->ndir) : 0;
    const size_t o_dsmax = scatter ? take(sizeof(unsigned) * 4) : 0;
    const size_t o_regu = h->use_reg ? take(sizeof(rts::SweepUnit) * h->reg_units.size()) : 0;
    // the register tiles' unit table and ticket order
    const size_t o_reguot = h->use_reg ? take(2 * sizeof(int) * h->reg_unit_of_tile.size()) : 0;
    size_t o_adj[9] = {0};
    if (adjoint) {
        o_adj[7] = take(sizeof(rts::SweepUnit) * h->adj_units.size());
        o_adj[8] = take(2 * sizeof(int) * h->adj_unit_of_tile.size());  // unit table and ticket order
        const size_t cu = (size_t)h->chunk_units;
        o_adj[0] = take((size_t)nbands * 4 * h->N * es);
        o_adj[1] = h->has_x ? take((size_t)nbands * 4 * h->N * es) : 0;
        o_adj[2] = take((size_t)nbands * 2 * h->N * es);
        o_adj[3] = take(cu * rts::STORE_CH * rts::MAXD * h->N * es);
        o_adj[4] = take(cu * rts::GRAD_CH * h->N * es);
    }
    size_t o_as[2][6] = {{0}};
    const bool hostio_async = (o.flags & RTS_FLAG_HOST_IO_ASYNC) != 0;
    if (hostio_async) {
        for (int st_ = 0; st_ < 2; ++st_) {
            o_as[st_][0] = take((size_t)nbands * h->N * es);
            o_as[st_][1] = take((size_t)nbands * h->N * es);
            o_as[st_][2] = take((size_t)nbands * h->n_up * nx * ny * es);
            o_as[st_][3] = take((size_t)h->N * 8);
            o_as[st_][4] = take((size_t)3 * h->N * 8);
            o_as[st_][5] = take((size_t)h->N * 8);
        }
    }
    size_t o_io[6] = {0};
    const bool hostio = (o.flags & RTS_FLAG_HOST_IO) != 0;
    if (hostio) {
        o_io[0] = take((size_t)nbands * h->N * es);
        o_io[1] = take((size_t)nbands * h->N * es);
        o_io[2] = take((size_t)nbands * h->n_up * nx * ny * es);
        o_io[3] = take((size_t)h->N * 8);
        o_io[4] = take((size_t)3 * h->N * 8);
        o_io[5] = take((size_t)h->N * 8);
    }
    cudaError_t ae = cudaMalloc(&h->dmem, off);
    if (ae != cudaSuccess) {
        h->dmem = nullptr;
        return bail(fail(h, RTS_ENOMEM, "cudaMalloc of %zu bytes: %s", off, cudaGetErrorString(ae)));
    }
    char *base = (char *)h->dmem;
    h->d_units = (rts::SweepUnit *)(base + o_units);
    h->d_unit_of_tile = (int *)(base + o_uot);
    h->d_partial = base + o_part;
    h->d_chiT = h->has_x ? base + o_chiT : nullptr;
    h->d_ST = h->has_x ? base + o_ST : nullptr;
    h->d_JF = base + o_JF;
    h->d_halo = base + o_halo;
    h->d_flags = (int *)(base + o_flags);
    h->d_gcnt = (unsigned int *)(base + o_gcnt);
    h->d_gmax = (unsigned long long *)(base + o_gmax);
    h->d_ticket = (int *)(base + o_ticket);
    h->d_status = (int *)(base + o_status);
    h->d_unit_tacc = (int *)(base + o_tacc);
    h->d_ru = (rts::RedUnit *)(base + o_ru);
    h->d_ru_begin = (int *)(base + o_rub);
    h->d_qfu = (rts::RedUnit *)(base + o_qfu);
    h->d_qfb = (int *)(base + o_qfb);
    if (log_chi) h->d_chi_exp = base + o_cexp;
    if (scatter) {
        h->d_lstar = base + o_lstar;
        h->d_dirw = (double *)(base + o_dirw);
        h->d_dsmax = (unsigned *)(base + o_dsmax);
        // (ds_d, w_d) with the weights of directions of equal segment length
        // summed (the 24 S4 directions share their dominant cosine: one
        // length per axis, one in all on a grid of cubic cells)
        std::vector<double> dw;
        for (int d = 0; d < h->ndir; ++d) {
            size_t e = 0;
            while (e < dw.size() && dw[e] != geo[d].ds) e += 2;
            if (e == dw.size()) dw.insert(dw.end(), {geo[d].ds, 0.0});
            dw[e + 1] += h->w[d];
        }
        h->n_lsd = (int)(dw.size() / 2);
        CUDA_TRY(h, cudaMemcpy(h->d_dirw, dw.data(), sizeof(double) * dw.size(), cudaMemcpyHostToDevice));
    }
    if (h->use_reg) {
        h->d_reg_units = (rts::SweepUnit *)(base + o_regu);
        h->d_reg_uot = (int *)(base + o_reguot);
        h->d_reg_order = h->d_reg_uot + h->reg_unit_of_tile.size();
    }
    if (adjoint) {
        h->d_adj_units = (rts::SweepUnit *)(base + o_adj[7]);
        h->d_adj_uot = (int *)(base + o_adj[8]);
        h->d_adj_order = h->d_adj_uot + h->adj_unit_of_tile.size();
        h->d_lam0 = base + o_adj[0];
        h->d_lam0T = h->has_x ? base + o_adj[1] : nullptr;
        h->d_direct = base + o_adj[2];
        h->d_ckpt = base + o_adj[3];
        h->d_grad = base + o_adj[4];
    }
    if (hostio_async) {
        for (int st_ = 0; st_ < 2; ++st_) {
            h->a_in[st_][0] = base + o_as[st_][0];
            h->a_in[st_][1] = base + o_as[st_][1];
            for (int i = 0; i < 4; ++i) h->a_out[st_][i] = base + o_as[st_][2 + i];
            CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_h2d[st_], cudaEventDisableTiming));
            CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_comp[st_], cudaEventDisableTiming));
            CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_d2h[st_], cudaEventDisableTiming));
        }
        CUDA_TRY(h, cudaStreamCreateWithFlags(&h->s_h2d, cudaStreamNonBlocking));
        CUDA_TRY(h, cudaStreamCreateWithFlags(&h->s_d2h, cudaStreamNonBlocking));
    }
    if (hostio) {
        h->d_in_chi = base + o_io[0];
        h->d_in_S = base + o_io[1];
        h->d_out_itop = base + o_io[2];
        h->d_out_J = (double *)(base + o_io[3]);
        h->d_out_F = (double *)(base + o_io[4]);
        h->d_out_Q = (double *)(base + o_io[5]);
    }
    // partial pointers and the reduction table (units are band-major)
    std::vector<rts::RedUnit> ru(h->units.size());
    std::vector<int> rub(nbands + 1, 0);
    for (size_t u = 0; u < h->units.size(); ++u) {
        h->units[u].partial = (char *)h->d_partial + u * 4 * h->N * es;
        ru[u] = red_unit(h->units[u]);
        rub[h->units[u].band + 1]++;
    }
    for (int b = 0; b < nbands; ++b) rub[b + 1] += rub[b];
    CUDA_TRY(h, cudaMemcpy(h->d_units, h->units.data(), sizeof(rts::SweepUnit) * h->units.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(h->d_unit_of_tile, h->unit_of_tile.data(), sizeof(int) * h->unit_of_tile.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(h->d_ru, ru.data(), sizeof(rts::RedUnit) * ru.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(h->d_ru_begin, rub.data(), sizeof(int) * rub.size(), cudaMemcpyHostToDevice));
    if (h->use_reg) {
        // the streaming reduction of the register sweep's raw partials: per
        // band the x groups, then the y units, then the z units
        {
            std::vector<rts::RedUnit> qfu;
            std::vector<int> qfb(3 * nbands + 1, 0);
            bool pairing_ok = true;  // each unit pairs slots as its group's code assumes
            for (int b = 0; b < nbands; ++b) {
                qfb[b] = (int)qfu.size();
                for (int axis = 0; axis < 3; ++axis) {
                    for (int u = rub[b]; u < rub[b + 1]; ++u) {
                        if (ru[u].axis != axis) continue;
                        qfu.push_back(ru[u]);
                        for (int c = 0; c < 4; ++c)
                            pairing_ok &= (ru[u].qpair[c] != 0) == (c == rts::qr_cross_moment(axis));
                    }
                    if (axis == 0) qfb[nbands + 1 + b] = (int)qfu.size();
                    if (axis == 1) qfb[2 * nbands + 1 + b] = (int)qfu.size();
                }
            }
            qfb[nbands] = (int)qfu.size();
            CUDA_TRY(h, cudaMemcpy(h->d_qfu, qfu.data(), sizeof(rts::RedUnit) * qfu.size(), cudaMemcpyHostToDevice));
            CUDA_TRY(h, cudaMemcpy(h->d_qfb, qfb.data(), sizeof(int) * qfb.size(), cudaMemcpyHostToDevice));
            for (int b = 0; b < nbands; ++b) {
                h->qr_max_x = std::max(h->qr_max_x, qfb[nbands + 1 + b] - qfb[b]);
                h->qr_max_nat = std::max(h->qr_max_nat, qfb[b + 1] - qfb[nbands + 1 + b]);
            }
            h->qr_smem = rts::qr_smem_bytes(h->qr_max_nat, h->qr_max_x, (int)qfu.size(), nbands);
            int per_sm = 0;
            const long long qr_tiles = (long long)((nx + rts::QR_TI - 1) / rts::QR_TI) *
                                       ((ny + rts::QR_TJ - 1) / rts::QR_TJ) * nz * nbands;
            if (pairing_ok && qfu.size() == h->units.size() && h->qr_smem <= 113 * 1024 &&
                qr_tiles < (1LL << 31) - (1LL << 20) &&
                cudaFuncSetAttribute(rts::qf_reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)h->qr_smem) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rts::qf_reduce_kernel, rts::QR_NT,
                                                              h->qr_smem) == cudaSuccess &&
                per_sm > 0) {
                h->qr_grid = per_sm * nsm;
                h->qf_ok = true;
            }
            cudaGetLastError();
        }
        for (size_t u = 0; u < h->reg_units.size(); ++u) h->reg_units[u].partial = h->units[u].partial;
        CUDA_TRY(h, cudaMemcpy(h->d_reg_units, h->reg_units.data(), sizeof(rts::SweepUnit) * h->reg_units.size(),
                               cudaMemcpyHostToDevice));
        CUDA_TRY(h, cudaMemcpy(h->d_reg_uot, h->reg_unit_of_tile.data(), sizeof(int) * h->reg_unit_of_tile.size(),
                               cudaMemcpyHostToDevice));
        const std::vector<int> order = ticket_order(h->reg_units);
        CUDA_TRY(h, cudaMemcpy(h->d_reg_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice));
    }
    if (adjoint) {
        for (size_t u = 0; u < h->adj_units.size(); ++u) h->adj_units[u].partial = h->units[u].partial;
        CUDA_TRY(h, cudaMemcpy(h->d_adj_units, h->adj_units.data(), sizeof(rts::SweepUnit) * h->adj_units.size(),
                               cudaMemcpyHostToDevice));
        CUDA_TRY(h, cudaMemcpy(h->d_adj_uot, h->adj_unit_of_tile.data(), sizeof(int) * h->adj_unit_of_tile.size(),
                               cudaMemcpyHostToDevice));
        // as the forward's (used when a chunk covers every unit)
        const std::vector<int> order = ticket_order(h->adj_units);
        CUDA_TRY(h, cudaMemcpy(h->d_adj_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice));
    }
    // a status word and warm-up record that read as "nothing ran yet"
    CUDA_TRY(h, cudaMemset(h->d_status, 0, sizeof(int) * 4));
    CUDA_TRY(h, cudaMemset(h->d_unit_tacc, 0, sizeof(int) * h->units.size()));
    h->timing = (o.flags & RTS_FLAG_TIMING) != 0;
    *out = h;
    return RTS_OK;
}

}  // extern "C"

// launch arguments of a sweep over all units; callers narrow the tile range
template <typename T>
static rts::SweepArgs<T> sweep_args(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc)
{
    rts::SweepArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.units = h->d_units;
    a.unit_of_tile = h->d_unit_of_tile;
    a.total_tiles = h->total_tiles;
    a.chi = (const T *)chi;
    a.S = (const T *)S;
    a.chiT = (const T *)h->d_chiT;
    a.ST = (const T *)h->d_ST;
    a.bc_bottom = bc ? bc->bottom : RTS_BC_EQUAL_S;
    a.bc_top = bc ? bc->top : RTS_BC_ZERO;
    a.bc_up = bc ? (const T *)bc->bottom_I : nullptr;
    a.bc_dn = bc ? (const T *)bc->top_I : nullptr;
    a.n_up = h->n_up;
    a.n_dn = h->n_dn;
    a.ticket = h->d_ticket;
    a.flags = h->d_flags;
    a.halo = (T *)h->d_halo;
    a.gcnt = h->d_gcnt;
    a.gmax = h->d_gmax;
    a.pcnt = h->d_gcnt + h->units.size() * h->R;
    a.pmax = h->d_gmax + h->units.size() * h->R;
    a.R = h->R;
    a.L = kLag;
    a.status = h->d_status;
    a.unit_tacc = h->d_unit_tacc;
    a.tol = (float)h->opt.wrap_tol;
    a.max_periods = h->opt.max_wrap_iters;
    if (bc && bc->wrap_seed) {
        a.seed = (T *)bc->wrap_seed;
        a.seed_in = bc->seed_in;
        a.seed_tol = bc->seed_tol > 0 ? (float)bc->seed_tol : 1e-6f;
    }
    a.timeout_ns = (unsigned long long)(h->opt.timeout_s * 1e9);
    return a;
}

// clear the ticket, ready flags and wrap-decision counters before a sweep launch
static rts_status reset_sweep_state(rts_handle *h, cudaStream_t st)
{
    CUDA_TRY(h, cudaMemsetAsync(h->d_ticket, 0, sizeof(int) * 4, st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_flags, 0, sizeof(int) * std::max(h->flag_tiles, 2 * h->total_tiles), st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_gcnt, 0, sizeof(unsigned int) * h->units.size() * (h->R + 4), st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_gmax, 0, sizeof(unsigned long long) * h->units.size() * (h->R + 4), st));
    return RTS_OK;
}

// RTS_FLAG_LOG_CHI: the caller passed log chi; chi = exp(log chi) goes to the
// handle's scratch array, which the solve then reads
template <typename T>
static rts_status form_chi(rts_handle *h, const void *&chi, int &kernels)
{
    if (!h->d_chi_exp) return RTS_OK;
    const long long n = (long long)h->B * h->N;
    const int cb = (int)std::min<long long>((n + 255) / 256, 148LL * 8);
    exp_kernel<T><<<cb, 256, 0, h->stream>>>((const T *)chi, (T *)h->d_chi_exp, n);
    CUDA_TRY(h, cudaGetLastError());
    chi = h->d_chi_exp;
    kernels += 1;
    return RTS_OK;
}

template <typename T, typename Acc>
static rts_status solve_impl(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc, void *I_top,
                             double *J, double *F, double *Q, bool reduce_only = false)
{
    const rts_grid &g = h->g;
    const int B = h->B;
    cudaStream_t st = h->stream;
    CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int) * 4, st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_ticket, 0, sizeof(int) * 4, st));
    const bool reg = h->use_reg && sizeof(T) == 4;
    CUDA_TRY(h, cudaMemsetAsync(h->d_flags, 0, sizeof(int) * 2 * (reg ? h->reg_total_tiles : h->total_tiles), st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_gcnt, 0, sizeof(unsigned int) * h->units.size() * (h->R + 4), st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_gmax, 0, sizeof(unsigned long long) * h->units.size() * (h->R + 4), st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_unit_tacc, 0, sizeof(int) * h->units.size(), st));
    cudaEvent_t *ev = nullptr;
    if (h->timing && !h->capturing) {
        if (h->nrec == h->evs.size()) {
            std::array<cudaEvent_t, 5> set{};
            for (cudaEvent_t &e : set) CUDA_TRY(h, cudaEventCreate(&e));
            h->evs.push_back(set);
        }
        ev = h->evs[h->nrec++].data();
        CUDA_TRY(h, cudaEventRecord(ev[0], st));
    }
    int kernels = 0;
    if (rts_status fs = form_chi<T>(h, chi, kernels)) return fs;
    if (h->has_x) {
        dim3 tb(32, 8), tg((g.nx + 31) / 32, (g.ny + 31) / 32, (unsigned)(g.nz * B));
        rts::transpose_x2_kernel<T><<<tg, tb, 0, st>>>((const T *)chi, (const T *)S, (T *)h->d_chiT, (T *)h->d_ST,
                                                      g.nx, g.ny, g.nz, h->d_status);
        CUDA_TRY(h, cudaGetLastError());
        kernels += 1;
    } else {  // no transposed copy to make: the non-finite check alone
        const long long n = (long long)B * h->N;
        const int cb = (int)std::min<long long>((n + 255) / 256, 148LL * 8);
        rts::check_finite_kernel<T><<<cb, 256, 0, st>>>((const T *)chi, (const T *)S, n, h->d_status);
        CUDA_TRY(h, cudaGetLastError());
        kernels += 1;
    }
    if (ev) CUDA_TRY(h, cudaEventRecord(ev[1], st));
    rts::SweepArgs<T> a = sweep_args<T>(h, chi, S, bc);
    a.itop = (T *)I_top;
    cudaError_t e = reg ? launch_reg_sweep(h, *reinterpret_cast<const rts::SweepArgs<float> *>(&a))
                        : launch_sweep<T>(h, a);
    if (e != cudaSuccess) return fail(h, RTS_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
    kernels += 1;
    if (ev) CUDA_TRY(h, cudaEventRecord(ev[2], st));
    if (reg && h->qf_ok && (reduce_only || J || F || Q)) {
        // the register sweep's raw partials: the streaming reduction into
        // double-float J_b, F_b, then the double-float Q step (both FP32 modes)
        rts::QParams P;
        P.nx = g.nx; P.ny = g.ny; P.nz = g.nz; P.nbands = B;
        P.inv2dx = 0.5 / g.dx; P.inv2dy = 0.5 / g.dy; P.inv2dz = 0.5 / g.dz; P.invdz = 1.0 / g.dz;
        P.thin = std::min(g.dx, std::min(g.dy, g.dz)) / h->opt.tau_switch;
        rts::df32 *jf = (rts::df32 *)h->d_JF;
        rts::qf_reduce_kernel<<<h->qr_grid, dim3(rts::QR_TI, rts::QR_RY), h->qr_smem, st>>>(
            h->d_qfu, h->d_qfb, g.nx, g.ny, g.nz, B, (int)h->units.size(), h->qr_max_nat, h->qr_max_x, jf);
        CUDA_TRY(h, cudaGetLastError());
        if (ev) CUDA_TRY(h, cudaEventRecord(ev[3], st));
        kernels += 1;
        if (!reduce_only) {  // else the per-band J_b, F_b (double-float) stay in the handle's JF array
            dim3 rb(32, 8), qg((g.nx + 31) / 32, (g.ny + rts::QS_TJ - 1) / rts::QS_TJ, (unsigned)g.nz);
            rts::qstep_df2_kernel<<<qg, rb, 0, st>>>(jf, (const float *)chi, (const float *)S, P, J, F, Q);
            CUDA_TRY(h, cudaGetLastError());
            kernels += 1;
        }
    } else if (J || F || Q || reduce_only) {
        dim3 rb(32, 8);
        rts::QParams P;
        P.nx = g.nx; P.ny = g.ny; P.nz = g.nz; P.nbands = B;
        P.inv2dx = 0.5 / g.dx; P.inv2dy = 0.5 / g.dy; P.inv2dz = 0.5 / g.dz; P.invdz = 1.0 / g.dz;
        P.thin = std::min(g.dx, std::min(g.dy, g.dz)) / h->opt.tau_switch;
        dim3 rg((g.nx + 31) / 32, (g.ny + 31) / 32, (unsigned)(g.nz * B));
        rts::reduce_units_kernel<T, Acc><<<rg, rb, 0, st>>>(h->d_ru, h->d_ru_begin, (Acc *)h->d_JF, g.nx, g.ny, g.nz,
                                                           reg ? 1 : 0);
        if (ev) CUDA_TRY(h, cudaEventRecord(ev[3], st));
        kernels += 1;
        if (!reduce_only) {  // the per-band J_b, F_b stay in the handle's JF array
            dim3 qg((g.nx + 31) / 32, (g.ny + 7) / 8, (unsigned)g.nz);
            rts::qstep_kernel<T, Acc><<<qg, rb, 0, st>>>((const Acc *)h->d_JF, (const T *)chi, (const T *)S, P, J, F,
                                                        Q);
            kernels += 1;
        }
        CUDA_TRY(h, cudaGetLastError());
    } else if (ev) {
        CUDA_TRY(h, cudaEventRecord(ev[3], st));
    }
    if (ev) CUDA_TRY(h, cudaEventRecord(ev[4], st));
    h->kernels_last = kernels;
    return RTS_OK;
}

static rts_status check_bc(rts_handle *h, const rts_boundary *bc)
{
    if (!bc) return RTS_OK;
    if (bc->wrap_seed && (!h->use_reg || h->batched))
        return fail(h, RTS_EINVAL, "the warm start (wrap_seed) needs the FP32 register sweep of a single-grid handle");
    if (bc->wrap_seed && bc->seed_in && h->reg_grid_seed < 1)
        return fail(h, RTS_EINVAL, "the warm-started sweep's tiles do not all fit on the GPU at once");
    if (bc->wrap_seed && !(bc->seed_tol >= 0)) return fail(h, RTS_EINVAL, "seed_tol must be >= 0");
    if (bc->bottom < RTS_BC_ZERO || bc->bottom > RTS_BC_EXPLICIT || bc->top < RTS_BC_ZERO || bc->top > RTS_BC_EXPLICIT)
        return fail(h, RTS_EINVAL, "unknown boundary kind");
    if (bc->bottom == RTS_BC_EXPLICIT && !bc->bottom_I) return fail(h, RTS_EINVAL, "bottom_I is NULL");
    if (bc->top == RTS_BC_EXPLICIT && !bc->top_I) return fail(h, RTS_EINVAL, "top_I is NULL");
    return RTS_OK;
}

// Reverse-mode gradient (declared in rts.h). Enqueues, on the handle's stream:
// [transpose of chi, S], then per checkpoint chunk of bands: forward sweep
// that keeps every ray's I (and whose partial sums give the chunk's J_b, F_b:
// reduction only when Q_rad enters L) -> Q-step adjoint of the chunk's bands
// -> [transpose of lam0] -> reverse sweep -> two gradient passes -> reduce
// into g_logchi, g_S.
template <typename T, typename Acc>
static rts_status adjoint_impl(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc,
                               const void *gI_top, const double *gJ, const double *gF, const double *gQ,
                               void *g_logchi, void *g_S)
{
    const rts_grid &g = h->g;
    const int B = h->B;
    const long long N = h->N;
    cudaStream_t st = h->stream;
    CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int) * 4, st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_unit_tacc, 0, sizeof(int) * h->units.size(), st));
    int kernels = 0;
    const dim3 tb(32, 8), tg((g.nx + 31) / 32, (g.ny + 31) / 32, (unsigned)(g.nz * B));
    // RTS_FLAG_TIMING: an event at each phase boundary (phase ids as in rts_stats.ms_adjoint)
    const bool tim = h->timing && !h->capturing;
    auto mark = [&](int phase) -> rts_status {
        if (!tim) return RTS_OK;
        if (h->adj_nev == h->adj_evs.size()) {
            cudaEvent_t e = nullptr;
            CUDA_TRY(h, cudaEventCreate(&e));
            h->adj_evs.push_back(e);
            h->adj_phase.push_back(0);
        }
        h->adj_phase[h->adj_nev] = phase;
        CUDA_TRY(h, cudaEventRecord(h->adj_evs[h->adj_nev++], st));
        return RTS_OK;
    };
    if (tim) {
        if (h->adj_calls == 0) h->adj_nev = 0;
        if (rts_status ms = mark(-1)) return ms;
        ++h->adj_calls;
    }
    if (rts_status fs = form_chi<T>(h, chi, kernels)) return fs;
    if (h->has_x) {
        rts::transpose_x2_kernel<T><<<tg, tb, 0, st>>>((const T *)chi, (const T *)S, (T *)h->d_chiT, (T *)h->d_ST,
                                                      g.nx, g.ny, g.nz, h->d_status);
        CUDA_TRY(h, cudaGetLastError());
        kernels += 1;
    } else {
        const long long n = (long long)B * N;
        const int cb = (int)std::min<long long>((n + 255) / 256, 148LL * 8);
        rts::check_finite_kernel<T><<<cb, 256, 0, st>>>((const T *)chi, (const T *)S, n, h->d_status);
        CUDA_TRY(h, cudaGetLastError());
        kernels += 1;
    }
    if (rts_status ms = mark(0)) return ms;
    rts::QAdjParams QP;
    QP.nx = g.nx; QP.ny = g.ny; QP.nz = g.nz; QP.nbands = B;
    QP.inv2dx = 0.5 / g.dx; QP.inv2dy = 0.5 / g.dy; QP.inv2dz = 0.5 / g.dz; QP.invdz = 1.0 / g.dz;
    QP.thin = std::min(g.dx, std::min(g.dy, g.dz)) / h->opt.tau_switch;
    for (int b0 = 0; b0 < B; b0 += h->chunk_bands) {
        const int b1 = std::min(B, b0 + h->chunk_bands), nbc = b1 - b0;
        const int u0 = h->band_unit[b0], u1 = h->band_unit[b1];
        const rts::SweepUnit &U0 = h->units[u0], &U1 = h->units[u1 - 1];
        rts::SweepArgs<T> a = sweep_args<T>(h, chi, S, bc);
        a.tile_base = U0.tile0;
        a.total_tiles = U1.tile0 + U1.ntiles - U0.tile0;
        a.unit_base = u0;
        // forward sweep of the chunk (the checkpoint): every ray's converged I,
        // and the partial sums that give J_b, F_b of the chunk's bands
        rts_status rs = reset_sweep_state(h, st);
        if (rs) return rs;
        a.store = (T *)h->d_ckpt;
        // FP32 on a register-sweep handle: the register sweep's checkpoint
        // instantiation (raw slot intensities and D), then the forward solve's
        // double-float reduction and a double-float Q-step adjoint, in both
        // FP32 modes (as the forward solve's register path)
        bool regck = false;
        if constexpr (std::is_same<T, float>::value) regck = h->use_reg && !h->batched && h->reg_grid_ck > 0;
        cudaError_t e;
        if constexpr (std::is_same<T, float>::value) {
            if (regck) e = launch_reg_ckpt(h, a, u0, u1);
            else e = launch_sweep<T>(h, a);
        } else {
            e = launch_sweep<T>(h, a);
        }
        if (e != cudaSuccess) return fail(h, RTS_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
        kernels += 1;
        if (gQ) {
            const dim3 rg((g.nx + 31) / 32, (g.ny + 31) / 32, (unsigned)(g.nz * nbc));
            if (regck && b0 == 0 && b1 == B && h->qf_ok) {
                rts::qf_reduce_kernel<<<h->qr_grid, dim3(rts::QR_TI, rts::QR_RY), h->qr_smem, st>>>(
                    h->d_qfu, h->d_qfb, g.nx, g.ny, g.nz, B, (int)h->units.size(), h->qr_max_nat, h->qr_max_x,
                    (rts::df32 *)h->d_JF);
            } else if (regck) {  // raw slot intensities of the chunk's units
                rts::reduce_units_kernel<float, rts::df32><<<rg, tb, 0, st>>>(
                    h->d_ru, h->d_ru_begin + b0, (rts::df32 *)h->d_JF + (long long)b0 * 4 * N, g.nx, g.ny, g.nz, 1);
            } else {
                rts::reduce_units_kernel<T, Acc><<<rg, tb, 0, st>>>(h->d_ru, h->d_ru_begin + b0,
                                                                   (Acc *)h->d_JF + (long long)b0 * 4 * N, g.nx,
                                                                   g.ny, g.nz, 0);
            }
            CUDA_TRY(h, cudaGetLastError());
            kernels += 1;
        }
        if (rts_status ms = mark(1)) return ms;
        {  // Q step transposed for the chunk's bands
            const dim3 qg((g.nx + 31) / 32, (g.ny + 7) / 8, (unsigned)g.nz);
            // gQ (1 - om_b) of the chunk's bands, read by the divergence
            // transpose at the neighbours; the gradient scratch is free here
            T *u = nullptr;
            if (gQ) {
                u = (T *)h->d_grad;
                const long long total = (long long)(b1 - b0) * N;
                const int ub = (int)std::min<long long>((total + 255) / 256, 148LL * 16);
                rts::qstep_adjoint_u_kernel<T><<<ub, 256, 0, st>>>((const T *)chi, gQ, QP, b0, b1, u);
                CUDA_TRY(h, cudaGetLastError());
                kernels += 1;
            }
            if constexpr (std::is_same<T, float>::value) {
                if (regck)
                    rts::qstep_adjoint_df_kernel<><<<qg, tb, 0, st>>>(
                        (const rts::df32 *)h->d_JF, (const float *)chi, (const float *)S, gJ, gF, gQ, u, QP, b0, b1,
                        (float *)h->d_lam0, (float *)h->d_direct);
                else
                    rts::qstep_adjoint_kernel<T, Acc><<<qg, tb, 0, st>>>((const Acc *)h->d_JF, (const T *)chi,
                                                                        (const T *)S, gJ, gF, gQ, u, QP, b0, b1,
                                                                        (T *)h->d_lam0, (T *)h->d_direct);
            } else {
                rts::qstep_adjoint_kernel<T, Acc><<<qg, tb, 0, st>>>((const Acc *)h->d_JF, (const T *)chi,
                                                                    (const T *)S, gJ, gF, gQ, u, QP, b0, b1,
                                                                    (T *)h->d_lam0, (T *)h->d_direct);
            }
            CUDA_TRY(h, cudaGetLastError());
            kernels += 1;
            if (h->has_x) {
                // lam0 [b][N][4]: the 4 values of a point move as one element
                const dim3 lg((g.nx + 31) / 32, (g.ny + 31) / 32, (unsigned)(g.nz * nbc));
                rts::transpose_x_kernel<rts::Vec4<T>><<<lg, tb, 0, st>>>(
                    (const rts::Vec4<T> *)((const T *)h->d_lam0 + (long long)b0 * 4 * N),
                    (rts::Vec4<T> *)((T *)h->d_lam0T + (long long)b0 * 4 * N), g.nx, g.ny, g.nz);
                CUDA_TRY(h, cudaGetLastError());
                kernels += 1;
            }
        }
        if (rts_status ms = mark(0)) return ms;
        // reverse sweep: cotangent of I of every ray (the adjoint kernel's tiling)
        rs = reset_sweep_state(h, st);
        if (rs) return rs;
        const rts::SweepUnit &A0 = h->adj_units[u0], &A1 = h->adj_units[u1 - 1];
        a.units = h->d_adj_units;
        a.unit_of_tile = h->d_adj_uot;
        a.tile_order = (u0 == 0 && u1 == (int)h->units.size()) ? h->d_adj_order : nullptr;
        a.tile_base = A0.tile0;
        a.total_tiles = A1.tile0 + A1.ntiles - A0.tile0;
        a.store = (T *)h->d_grad;
        a.ckpt = (const T *)h->d_ckpt;
        a.lam0 = (const T *)h->d_lam0;
        a.lam0T = (const T *)h->d_lam0T;
        a.gitop = (const T *)gI_top;
        e = launch_sweep<T>(h, a, true);
        if (e != cudaSuccess) return fail(h, RTS_ECUDA, "reverse sweep launch: %s", cudaGetErrorString(e));
        kernels += 1;
        if (rts_status ms = mark(2)) return ms;
        // each point gathers the gradient terms of the downwind points that
        // interpolated from it (every unit of the chunk)
        rts::GradArgs<T> ga;
        ga.units = h->d_units;
        ga.unit_base = u0;
        ga.grad = (T *)h->d_grad;
        int np = 0, nq = 0, nm = 0;
        for (int u = u0; u < u1; ++u) {
            np = std::max(np, h->units[u].NP);
            nq = std::max(nq, h->units[u].NQ);
            nm = std::max(nm, h->units[u].NM);
        }
        // blockIdx.z = m + nm * (unit - first unit of the launch); at most 65535
        const int per = std::max(1, 65535 / nm);
        for (int us = u0; us < u1; us += per) {
            const int ue = std::min(u1, us + per);
            rts::GradArgs<T> gs = ga;
            gs.unit_base = us;
            gs.grad = ga.grad + (long long)(us - u0) * rts::GRAD_CH * N;
            // a row of the plane per block (up to 512 columns)
            const int gt = std::min(512, 32 * ((np + 31) / 32));
            const dim3 gg((np + gt - 1) / gt, nq, (unsigned)(nm * (ue - us)));
            rts::adj_gather_kernel<T><<<gg, gt, 0, st>>>(gs, nm);
            CUDA_TRY(h, cudaGetLastError());
            kernels += 1;
        }
        const dim3 rg((g.nx + 31) / 32, (g.ny + 31) / 32, (unsigned)(g.nz * (b1 - b0)));
        rts::adj_reduce_kernel<T><<<rg, tb, 0, st>>>(h->d_units, u0, u1, b0, (const T *)h->d_grad,
                                                    (const T *)h->d_direct, (const T *)chi, (T *)g_logchi, (T *)g_S,
                                                    g.nx, g.ny, g.nz);
        CUDA_TRY(h, cudaGetLastError());
        kernels += 1;
        if (rts_status ms = mark(3)) return ms;
    }
    h->kernels_last = kernels;
    return RTS_OK;
}

extern "C" {

rts_status rts_solve(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc, void *I_top, double *J,
                     double *F, double *Q)
{
    if (!h || !h->dmem) return h ? fail(h, RTS_EINVAL, "handle was not created successfully") : RTS_EINVAL;
    if (!chi || !S) return fail(h, RTS_EINVAL, "chi and S must not be NULL");
    rts_status s = check_bc(h, bc);
    if (s) return s;
    switch (h->opt.prec) {
    case RTS_FP64: return solve_impl<double, double>(h, chi, S, bc, I_top, J, F, Q);
    case RTS_FP32_MIXED: return solve_impl<float, double>(h, chi, S, bc, I_top, J, F, Q);
    default: return solve_impl<float, rts::df32>(h, chi, S, bc, I_top, J, F, Q);
    }
}

rts_status rts_adjoint(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc, const void *gI_top,
                       const double *gJ, const double *gF, const double *gQ, void *g_logchi, void *g_S)
{
    if (!h || !h->dmem) return h ? fail(h, RTS_EINVAL, "handle was not created successfully") : RTS_EINVAL;
    if (!h->d_lam0) return fail(h, RTS_EINVAL, "rts_adjoint needs RTS_FLAG_ADJOINT at create time");
    if (!chi || !S || !g_logchi || !g_S) return fail(h, RTS_EINVAL, "chi, S, g_logchi and g_S must not be NULL");
    if (g_logchi == g_S || g_logchi == chi || g_logchi == S || g_S == chi || g_S == S)
        return fail(h, RTS_EINVAL, "gradient outputs must not alias the inputs or each other");
    if (bc && bc->wrap_seed) return fail(h, RTS_EINVAL, "rts_adjoint takes no warm start");
    rts_status s = check_bc(h, bc);
    if (s) return s;
    switch (h->opt.prec) {
    case RTS_FP64: return adjoint_impl<double, double>(h, chi, S, bc, gI_top, gJ, gF, gQ, g_logchi, g_S);
    case RTS_FP32_MIXED: return adjoint_impl<float, double>(h, chi, S, bc, gI_top, gJ, gF, gQ, g_logchi, g_S);
    default: return adjoint_impl<float, rts::df32>(h, chi, S, bc, gI_top, gJ, gF, gQ, g_logchi, g_S);
    }
}

rts_status rts_solve_host(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc, void *I_top,
                          double *J, double *F, double *Q)
{
    if (!h || !h->dmem) return h ? fail(h, RTS_EINVAL, "handle was not created successfully") : RTS_EINVAL;
    if (!h->d_in_chi) return fail(h, RTS_EINVAL, "rts_solve_host needs RTS_FLAG_HOST_IO at create time");
    if (!chi || !S) return fail(h, RTS_EINVAL, "chi and S must not be NULL");
    if (bc && (bc->bottom == RTS_BC_EXPLICIT || bc->top == RTS_BC_EXPLICIT))
        return fail(h, RTS_EINVAL, "rts_solve_host does not take explicit boundary arrays");
    rts_status s = check_bc(h, bc);
    if (s) return s;
    cudaStream_t st = h->stream;
    const size_t in_bytes = (size_t)h->B * h->N * h->esize;
    CUDA_TRY(h, cudaMemcpyAsync(h->d_in_chi, chi, in_bytes, cudaMemcpyHostToDevice, st));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_in_S, S, in_bytes, cudaMemcpyHostToDevice, st));
    s = rts_solve(h, h->d_in_chi, h->d_in_S, bc, I_top ? h->d_out_itop : nullptr, J ? h->d_out_J : nullptr,
                  F ? h->d_out_F : nullptr, Q ? h->d_out_Q : nullptr);
    if (s) return s;
    const size_t plane = (size_t)h->g.nx * h->g.ny;
    if (I_top)
        CUDA_TRY(h, cudaMemcpyAsync(I_top, h->d_out_itop, (size_t)h->B * h->n_up * plane * h->esize, cudaMemcpyDeviceToHost, st));
    if (J) CUDA_TRY(h, cudaMemcpyAsync(J, h->d_out_J, h->N * 8, cudaMemcpyDeviceToHost, st));
    if (F) CUDA_TRY(h, cudaMemcpyAsync(F, h->d_out_F, 3 * h->N * 8, cudaMemcpyDeviceToHost, st));
    if (Q) CUDA_TRY(h, cudaMemcpyAsync(Q, h->d_out_Q, h->N * 8, cudaMemcpyDeviceToHost, st));
    return rts_check(h);
}

rts_status rts_solve_host_async(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc, void *I_top,
                                double *J, double *F, double *Q)
{
    if (!h || !h->dmem) return h ? fail(h, RTS_EINVAL, "handle was not created successfully") : RTS_EINVAL;
    if (!h->s_h2d) return fail(h, RTS_EINVAL, "rts_solve_host_async needs RTS_FLAG_HOST_IO_ASYNC at create time");
    if (!chi || !S) return fail(h, RTS_EINVAL, "chi and S must not be NULL");
    if (bc && (bc->bottom == RTS_BC_EXPLICIT || bc->top == RTS_BC_EXPLICIT))
        return fail(h, RTS_EINVAL, "rts_solve_host_async does not take explicit boundary arrays");
    rts_status s = check_bc(h, bc);
    if (s) return s;
    const int k = h->a_next;
    h->a_next ^= 1;
    void *const *in = h->a_in[k];
    void *const *out = h->a_out[k];
    const size_t in_bytes = (size_t)h->B * h->N * h->esize;
    const size_t plane = (size_t)h->g.nx * h->g.ny;
    const size_t out_bytes[4] = {(size_t)h->B * h->n_up * plane * h->esize, (size_t)h->N * 8, (size_t)3 * h->N * 8,
                                 (size_t)h->N * 8};
    void *const host_out[4] = {I_top, J, F, Q};
    // inputs: wait until the solve that last read this set has finished
    if (h->a_used[k]) CUDA_TRY(h, cudaStreamWaitEvent(h->s_h2d, h->ev_comp[k], 0));
    CUDA_TRY(h, cudaMemcpyAsync(in[0], chi, in_bytes, cudaMemcpyHostToDevice, h->s_h2d));
    CUDA_TRY(h, cudaMemcpyAsync(in[1], S, in_bytes, cudaMemcpyHostToDevice, h->s_h2d));
    CUDA_TRY(h, cudaEventRecord(h->ev_h2d[k], h->s_h2d));
    // solve: after the inputs arrived and the outputs of this set were copied out
    CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_h2d[k], 0));
    if (h->a_used[k]) CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_d2h[k], 0));
    s = rts_solve(h, in[0], in[1], bc, I_top ? out[0] : nullptr, J ? (double *)out[1] : nullptr,
                  F ? (double *)out[2] : nullptr, Q ? (double *)out[3] : nullptr);
    if (s) return s;
    CUDA_TRY(h, cudaEventRecord(h->ev_comp[k], h->stream));
    // outputs
    CUDA_TRY(h, cudaStreamWaitEvent(h->s_d2h, h->ev_comp[k], 0));
    for (int i = 0; i < 4; ++i)
        if (host_out[i]) CUDA_TRY(h, cudaMemcpyAsync(host_out[i], out[i], out_bytes[i], cudaMemcpyDeviceToHost, h->s_d2h));
    CUDA_TRY(h, cudaEventRecord(h->ev_d2h[k], h->s_d2h));
    h->a_used[k] = true;
    return RTS_OK;
}

rts_status rts_host_wait(rts_handle *h)
{
    if (!h || !h->dmem) return RTS_EINVAL;
    if (h->s_h2d) CUDA_TRY(h, cudaStreamSynchronize(h->s_h2d));
    if (h->s_d2h) CUDA_TRY(h, cudaStreamSynchronize(h->s_d2h));
    return rts_check(h);
}

}  // extern "C"

// The scattering solve (declared in rts.h): the iteration of the band source
// functions S = (1 - eps) J + eps B, each iteration a forward solve (sweep and
// band reduction) and the preconditioned update; the outputs of the last
// solve with the converged S.
template <typename T, typename Acc>
static rts_status scatter_impl(rts_handle *h, const void *chi, const void *Bp, const void *eps, void *S,
                               const rts_boundary *bc, int max_iter, double tol, int *iters, void *I_top, double *J,
                               double *F, double *Q)
{
    cudaStream_t st = h->stream;
    const long long n = (long long)h->B * h->N;
    const int cb = (int)std::min<long long>((n + 255) / 256, 148LL * 8);
    int dummy = 0;
    const void *c = chi;
    if (rts_status fs = form_chi<T>(h, c, dummy)) return fs;
    lambda_star_kernel<T><<<cb, 256, 0, st>>>((const T *)c, h->d_dirw, h->n_lsd, n, (T *)h->d_lstar);
    CUDA_TRY(h, cudaGetLastError());
    int it = 0;
    bool conv = false;
    for (; it < max_iter && !conv; ++it) {
        rts_status rs = solve_impl<T, Acc>(h, chi, S, bc, nullptr, nullptr, nullptr, nullptr, true);
        if (rs) return rs;
        CUDA_TRY(h, cudaMemsetAsync(h->d_dsmax, 0, sizeof(unsigned), st));
        if (h->use_reg && h->qf_ok && sizeof(T) == 4)  // the register sweep's reduction left double-float J_b
            scatter_update_kernel<T, rts::df32><<<cb, 256, 0, st>>>((const rts::df32 *)h->d_JF, (const T *)eps,
                                                                    (const T *)Bp, (const T *)h->d_lstar, (T *)S,
                                                                    h->N, h->B, h->d_dsmax);
        else
            scatter_update_kernel<T, Acc><<<cb, 256, 0, st>>>((const Acc *)h->d_JF, (const T *)eps, (const T *)Bp,
                                                              (const T *)h->d_lstar, (T *)S, h->N, h->B, h->d_dsmax);
        CUDA_TRY(h, cudaGetLastError());
        unsigned bits = 0;
        CUDA_TRY(h, cudaMemcpyAsync(&bits, h->d_dsmax, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        rs = rts_check(h);  // waits for the stream; device errors end the iteration
        if (rs) return rs;
        float m;
        std::memcpy(&m, &bits, sizeof(m));
        conv = m <= tol;
    }
    if (iters) *iters = it;
    if (!conv) return fail(h, RTS_ENOCONV, "scattering iteration not converged in %d iterations", max_iter);
    return solve_impl<T, Acc>(h, chi, S, bc, I_top, J, F, Q);
}

extern "C" {

rts_status rts_scatter_solve(rts_handle *h, const void *chi, const void *B_src, const void *eps, void *S,
                             const rts_boundary *bc, int max_iter, double tol, int *iters, void *I_top, double *J,
                             double *F, double *Q_rad)
{
    if (!h || !h->dmem) return h ? fail(h, RTS_EINVAL, "handle was not created successfully") : RTS_EINVAL;
    if (!h->d_lstar) return fail(h, RTS_EINVAL, "rts_scatter_solve needs RTS_FLAG_SCATTER at create time");
    if (!chi || !B_src || !eps || !S) return fail(h, RTS_EINVAL, "chi, B, eps and S must not be NULL");
    if (S == chi || S == B_src || S == eps) return fail(h, RTS_EINVAL, "S must not alias the other inputs");
    if (max_iter < 1 || !(tol > 0)) return fail(h, RTS_EINVAL, "max_iter >= 1 and tol > 0 are needed");
    if (h->capturing) return fail(h, RTS_EINVAL, "the scattering iteration synchronises: not inside a capture");
    rts_status s = check_bc(h, bc);
    if (s) return s;
    switch (h->opt.prec) {
    case RTS_FP64: return scatter_impl<double, double>(h, chi, B_src, eps, S, bc, max_iter, tol, iters, I_top, J, F, Q_rad);
    case RTS_FP32_MIXED:
        return scatter_impl<float, double>(h, chi, B_src, eps, S, bc, max_iter, tol, iters, I_top, J, F, Q_rad);
    default:
        return scatter_impl<float, rts::df32>(h, chi, B_src, eps, S, bc, max_iter, tol, iters, I_top, J, F, Q_rad);
    }
}

rts_status rts_check(rts_handle *h)
{
    if (!h || !h->dmem) return RTS_EINVAL;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    int st = 0;
    CUDA_TRY(h, cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & rts::ST_NONFINITE) return fail(h, RTS_ENONFINITE, "non-finite value in chi or S (a NaN or an infinity)");
    if (st & rts::ST_TIMEOUT) return fail(h, RTS_ETIMEOUT, "a device-side wait exceeded %.3g s", h->opt.timeout_s);
    if (st & rts::ST_NOCONV)
        return fail(h, RTS_ENOCONV, "periodic wrap not converged within %d periods", h->opt.max_wrap_iters);
    return RTS_OK;
}

long long rts_wrap_seed_elems(rts_handle *h) { return h && h->use_reg ? h->seed_elems : 0; }

int rts_device_code_version(void)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, rts::check_finite_kernel<float>) != cudaSuccess) return -1;
    return fa.binaryVersion;
}

rts_status rts_get_stats(rts_handle *h, rts_stats *out)
{
    if (!h || !h->dmem || !out) return RTS_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->n_units = (int)h->units.size();
    out->n_tiles = h->use_reg ? h->reg_total_tiles : h->total_tiles;
    rts_status s = rts_check(h);
    out->device_status = s;
    std::vector<int> tacc(h->units.size());
    CUDA_TRY(h, cudaMemcpy(tacc.data(), h->d_unit_tacc, sizeof(int) * tacc.size(), cudaMemcpyDeviceToHost));
    int nw = 0;
    double sum = 0;
    for (size_t u = 0; u < tacc.size(); ++u) {
        if (!h->units[u].wrap) continue;
        out->max_warmup_steps = std::max(out->max_warmup_steps, tacc[u]);
        sum += tacc[u];
        ++nw;
    }
    out->mean_warmup_steps = nw ? sum / nw : 0.0;
    out->sweep_kernel = h->use_reg ? RTS_SWEEP_REGISTER : RTS_SWEEP_SHARED;
    out->adjoint_chunk_bands = h->d_adj_units ? h->chunk_bands : 0;
    out->grid = h->use_reg ? h->reg_grid : h->grid;
    out->tile_rows = h->use_reg ? h->reg_tq : h->tq;
    out->kernels_per_solve = h->kernels_last;
    if (h->timing && h->nrec > 0) {
        double acc[4] = {0, 0, 0, 0};
        for (size_t r = 0; r < h->nrec; ++r)
            for (int i = 0; i < 4; ++i) {
                float ms = 0.f;
                CUDA_TRY(h, cudaEventElapsedTime(&ms, h->evs[r][i], h->evs[r][i + 1]));
                acc[i] += ms;
            }
        out->timed_solves = (int)h->nrec;
        out->ms_transpose = (float)(acc[0] / h->nrec);
        out->ms_sweep = (float)(acc[1] / h->nrec);
        out->ms_reduce = (float)(acc[2] / h->nrec);
        out->ms_qstep = (float)(acc[3] / h->nrec);
        h->nrec = 0;
    }
    if (h->timing && h->adj_calls > 0) {
        double acc[4] = {0, 0, 0, 0};
        for (size_t i = 1; i < h->adj_nev; ++i) {
            const int ph = h->adj_phase[i];
            if (ph < 0) continue;  // start of the next call
            float ms = 0.f;
            CUDA_TRY(h, cudaEventElapsedTime(&ms, h->adj_evs[i - 1], h->adj_evs[i]));
            acc[ph] += ms;
        }
        out->timed_adjoints = h->adj_calls;
        for (int i = 0; i < 4; ++i) out->ms_adjoint[i] = (float)(acc[i] / h->adj_calls);
        h->adj_calls = 0;
        h->adj_nev = 0;
    }
    return s;
}

}  // extern "C"

// ===========================================================================
// rts_solve_noalloc: a forward solve for callers that cannot allocate device
// memory (for example code running inside a caller's CUDA graph capture, or
// an embedding application that owns a fixed device-memory budget and forbids
// cudaMalloc outside its own pool). It runs the same kernels as rts_solve, but
// every piece of scratch comes from one file-scope device array of fixed size
// that the CUDA runtime creates when the library's module is loaded on a GPU
// (every GPU that loads the library keeps it until the process exits).
// ===========================================================================

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[RTS_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
constexpr int kNoallocMaxUnits = 6 * 16;  // 6 direction groups x 16 bands
constexpr int kNoallocMaxTiles = 4096;

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

void noalloc_msg(char *err, size_t n, const char *fmt, ...)
{
    if (!err || n == 0) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, n, fmt, ap);
    va_end(ap);
}

template <typename T, typename Acc>
rts_status noalloc_solve(const rts_grid *g, int B, const void *chi, const void *S, void *I_top, double *J,
                         double *F, double *Q, cudaStream_t st, char *err, size_t errlen)
{
    // device address of the scratch array on the current device, looked up once
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
        noalloc_msg(err, errlen, "no usable current CUDA device");
        return RTS_ECUDA;
    }
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                noalloc_msg(err, errlen, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
                return RTS_ECUDA;
            }
            g_noalloc_ptr[dev] = p;
        }
        base = (unsigned char *)g_noalloc_ptr[dev];
    }

    // plan: default quadrature, bottom I = S, top I = 0, default options
    // (fixed-size host arrays: nothing is allocated, on the host or the device)
    double n[72], w[24];
    {
        const double m1 = std::sqrt((1.0 - std::sqrt(0.4)) / 3.0);
        const double m2 = std::sqrt(1.0 - 2.0 * m1 * m1);
        const int axis_of[6] = {2, 2, 0, 0, 1, 1};
        for (int grp = 0, d = 0; grp < 6; ++grp) {
            const int ax = axis_of[grp];
            const int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;
            for (int m = 0; m < 4; ++m, ++d) {
                n[3 * d + ax] = (grp % 2 == 0 ? 1.0 : -1.0) * m2;
                n[3 * d + b1] = (m & 1) ? -m1 : m1;
                n[3 * d + b2] = (m & 2) ? -m1 : m1;
                w[d] = 1.0 / 24.0;
            }
        }
    }
    const double hsp[3] = {g->dx, g->dy, g->dz};
    DirGeo geo[24];
    int udx[24], nup = 0, ndn = 0;
    for (int d = 0; d < 24; ++d) {
        if (!direction_geometry(hsp, &n[3 * d], geo[d])) {
            noalloc_msg(err, errlen, "direction %d has no valid geometry", d);
            return RTS_EINVAL;
        }
        udx[d] = geo[d].up ? nup++ : ndn++;
    }
    const long long nx = g->nx, ny = g->ny, nz = g->nz, N = nx * ny * nz;
    const int npmax = (int)std::max(nx, ny);
    if (npmax > 1024) {
        noalloc_msg(err, errlen, "plane extent %d > 1024 is not supported", npmax);
        return RTS_EINVAL;
    }
    const size_t es = sizeof(T);
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        noalloc_msg(err, errlen, "cannot query the device");
        return RTS_ECUDA;
    }
    const Tiling tl = choose_fwd<T>(0, npmax, (int)std::max(ny, nz), nsm);
    if (tl.tq < 1) {
        noalloc_msg(err, errlen, "no sweep tile fits plane extent %d", npmax);
        return RTS_EINVAL;
    }
    const int tq = tl.tq;
    const int nt = tl.nt;
    const size_t smem = tl.smem;

    rts::SweepUnit units[kNoallocMaxUnits];
    int unit_of_tile[kNoallocMaxTiles];
    rts::RedUnit ru[kNoallocMaxUnits];
    int rub[17] = {0};
    PlanOut po;
    if (!plan_units(geo, udx, n, w, 24, nx, ny, nz, B, tq, units, kNoallocMaxUnits, unit_of_tile, kNoallocMaxTiles,
                    po)) {
        noalloc_msg(err, errlen, "more than %d sweep units or %d tiles", kNoallocMaxUnits, kNoallocMaxTiles);
        return RTS_EINVAL;
    }
    const int nunits = po.nunits, ntile = po.ntiles, maxnt = po.max_ntiles;
    const long long halo_elems = po.halo_elems;
    const bool has_x = po.has_x;
    for (int u = 0; u < nunits; ++u) rub[units[u].band + 1]++;
    for (int b = 0; b < B; ++b) rub[b + 1] += rub[b];
    int R = 8;
    while (R < 2 * (maxnt + kLag + 2)) R *= 2;

    // carve the scratch array
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = round_up(off + bytes, 256); return at; };
    const size_t o_units = take(sizeof(rts::SweepUnit) * nunits);
    const size_t o_uot = take(sizeof(int) * ntile);
    const size_t o_ru = take(sizeof(rts::RedUnit) * nunits);
    const size_t o_rub = take(sizeof(int) * (B + 1));
    const size_t o_flags = take(sizeof(int) * 2 * ntile);  // a pair per tile
    const size_t o_gcnt = take(sizeof(unsigned int) * nunits * (R + 4));
    const size_t o_gmax = take(sizeof(unsigned long long) * nunits * (R + 4));
    const size_t o_ctl = take(sizeof(int) * 8);  // ticket, status
    const size_t o_tacc = take(sizeof(int) * nunits);
    const size_t o_halo = take((size_t)halo_elems * es);
    const size_t o_part = take((size_t)nunits * 4 * N * es);
    const size_t o_chiT = has_x ? take((size_t)B * N * es) : 0;
    const size_t o_ST = has_x ? take((size_t)B * N * es) : 0;
    const size_t o_JF = take((size_t)B * 4 * N * sizeof(Acc));
    if (off > (size_t)RTS_NOALLOC_SCRATCH_BYTES) {
        noalloc_msg(err, errlen, "grid %lldx%lldx%lld with %d bands needs %zu bytes of scratch; the fixed array has %zu",
                    nx, ny, nz, B, off, (size_t)RTS_NOALLOC_SCRATCH_BYTES);
        return RTS_EINVAL;
    }
    for (int u = 0; u < nunits; ++u) {
        units[u].partial = base + o_part + (size_t)u * 4 * N * es;
        ru[u] = red_unit(units[u]);
    }

    // residency of the persistent launch
    SweepFn<T> kern = fwd_kernel<T>(tq, tl.maxt);
    int blocks = 0;
#define NA_TRY(call)                                                                              \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            noalloc_msg(err, errlen, "%s: %s", #call, cudaGetErrorString(e_));                    \
            return RTS_ECUDA;                                                                     \
        }                                                                                         \
    } while (0)
    NA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    NA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, nt, smem));
    const int grid = std::min(ntile, blocks * nsm);
    if (blocks < 1 || grid < maxnt) {
        noalloc_msg(err, errlen, "a sweep unit has %d tiles but only %d CTAs fit", maxnt, blocks * nsm);
        return RTS_EINVAL;
    }

    // tables in, control words cleared (the array keeps the previous call's contents)
    NA_TRY(cudaMemcpyAsync(base + o_units, units, sizeof(rts::SweepUnit) * nunits, cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(base + o_uot, unit_of_tile, sizeof(int) * ntile, cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(base + o_ru, ru, sizeof(rts::RedUnit) * nunits, cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(base + o_rub, rub, sizeof(int) * (B + 1), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemsetAsync(base + o_flags, 0, sizeof(int) * 2 * ntile, st));
    NA_TRY(cudaMemsetAsync(base + o_gcnt, 0, sizeof(unsigned int) * nunits * (R + 4), st));
    NA_TRY(cudaMemsetAsync(base + o_gmax, 0, sizeof(unsigned long long) * nunits * (R + 4), st));
    NA_TRY(cudaMemsetAsync(base + o_ctl, 0, sizeof(int) * 8, st));
    NA_TRY(cudaMemsetAsync(base + o_tacc, 0, sizeof(int) * nunits, st));

    if (has_x) {
        dim3 tb(32, 8), tg((g->nx + 31) / 32, (g->ny + 31) / 32, (unsigned)(g->nz * B));
        rts::transpose_x2_kernel<T><<<tg, tb, 0, st>>>((const T *)chi, (const T *)S, (T *)(base + o_chiT),
                                                      (T *)(base + o_ST), g->nx, g->ny, g->nz,
                                                      (int *)(base + o_ctl) + 4);
        NA_TRY(cudaGetLastError());
    }
    rts::SweepArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.units = (const rts::SweepUnit *)(base + o_units);
    a.unit_of_tile = (const int *)(base + o_uot);
    a.total_tiles = ntile;
    a.chi = (const T *)chi;
    a.S = (const T *)S;
    a.chiT = has_x ? (const T *)(base + o_chiT) : nullptr;
    a.ST = has_x ? (const T *)(base + o_ST) : nullptr;
    a.itop = (T *)I_top;
    a.bc_bottom = RTS_BC_EQUAL_S;
    a.bc_top = RTS_BC_ZERO;
    a.n_up = nup;
    a.n_dn = ndn;
    a.ticket = (int *)(base + o_ctl);
    a.status = (int *)(base + o_ctl) + 4;
    a.flags = (int *)(base + o_flags);
    a.halo = (T *)(base + o_halo);
    a.gcnt = (unsigned int *)(base + o_gcnt);
    a.gmax = (unsigned long long *)(base + o_gmax);
    a.pcnt = a.gcnt + (long long)nunits * R;
    a.pmax = a.gmax + (long long)nunits * R;
    a.R = R;
    a.L = kLag;
    a.unit_tacc = (int *)(base + o_tacc);
    a.tol = sizeof(T) == 8 ? 1e-15f : 0x1p-24f;
    a.max_periods = 64;
    a.timeout_ns = 2000000000ull;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    attr[1].val.sharedMemCarveout = carveout_percent(blocks, smem, (const void *)kern);
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    NA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
    if (J || F || Q) {
        dim3 rb(32, 8), rg((g->nx + 31) / 32, (g->ny + 31) / 32, (unsigned)(g->nz * B));
        rts::reduce_units_kernel<T, Acc><<<rg, rb, 0, st>>>((const rts::RedUnit *)(base + o_ru),
                                                             (const int *)(base + o_rub), (Acc *)(base + o_JF),
                                                             g->nx, g->ny, g->nz, 0);
        rts::QParams P;
        P.nx = g->nx; P.ny = g->ny; P.nz = g->nz; P.nbands = B;
        P.inv2dx = 0.5 / g->dx; P.inv2dy = 0.5 / g->dy; P.inv2dz = 0.5 / g->dz; P.invdz = 1.0 / g->dz;
        P.thin = std::min(g->dx, std::min(g->dy, g->dz)) / 0.1;
        dim3 qg((g->nx + 31) / 32, (g->ny + 7) / 8, (unsigned)g->nz);
        rts::qstep_kernel<T, Acc><<<qg, rb, 0, st>>>((const Acc *)(base + o_JF), (const T *)chi, (const T *)S, P,
                                                      J, F, Q);
        NA_TRY(cudaGetLastError());
    }
    // wait for the solve and report what the device recorded
    NA_TRY(cudaStreamSynchronize(st));
    int status = 0;
    NA_TRY(cudaMemcpy(&status, base + o_ctl + 4 * sizeof(int), sizeof(int), cudaMemcpyDeviceToHost));
#undef NA_TRY
    if (status & rts::ST_NONFINITE) {
        noalloc_msg(err, errlen, "non-finite value in chi or S");
        return RTS_ENONFINITE;
    }
    if (status & rts::ST_TIMEOUT) {
        noalloc_msg(err, errlen, "a device-side wait exceeded 2 s");
        return RTS_ETIMEOUT;
    }
    if (status & rts::ST_NOCONV) {
        noalloc_msg(err, errlen, "periodic wrap not converged within 64 periods");
        return RTS_ENOCONV;
    }
    noalloc_msg(err, errlen, "ok");
    return RTS_OK;
}

}  // namespace

extern "C" rts_status rts_solve_noalloc(const rts_grid *g, int nbands, rts_precision prec, const void *chi,
                                        const void *S, void *I_top, double *J, double *F, double *Q_rad,
                                        void *stream, char *err, size_t errlen)
{
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 2 || nbands < 1 || nbands > 16) {
        noalloc_msg(err, errlen, "grid must have nx, ny >= 1, nz >= 2 and 1 <= nbands <= 16");
        return RTS_EINVAL;
    }
    if (!(g->dx > 0 && g->dy > 0 && g->dz > 0) || !std::isfinite(g->dx) || !std::isfinite(g->dy) ||
        !std::isfinite(g->dz)) {
        noalloc_msg(err, errlen, "grid spacing must be finite and positive");
        return RTS_EINVAL;
    }
    if (!chi || !S) {
        noalloc_msg(err, errlen, "chi and S must not be NULL");
        return RTS_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        noalloc_msg(err, errlen, "rts_solve_noalloc waits for its stream and cannot run inside a stream capture");
        return RTS_EINVAL;
    }
    switch (prec) {
    case RTS_FP64: return noalloc_solve<double, double>(g, nbands, chi, S, I_top, J, F, Q_rad, st, err, errlen);
    case RTS_FP32_MIXED: return noalloc_solve<float, double>(g, nbands, chi, S, I_top, J, F, Q_rad, st, err, errlen);
    case RTS_FP32_COMPENSATED:
        return noalloc_solve<float, rts::df32>(g, nbands, chi, S, I_top, J, F, Q_rad, st, err, errlen);
    default: noalloc_msg(err, errlen, "unknown precision %d", (int)prec); return RTS_EINVAL;
    }
}

// ===========================================================================
// Batched solves: many independent grids of uneven size x bands in one
// persistent sweep launch (plus one transpose, reduction and Q-step launch
// each), CUDA-graph capture of a solve, and the tile-size autotuner.
// ===========================================================================

namespace {

// expected length of a unit in planes: the periodic groups sweep about one
// extra period of warm-up
long long unit_weight(const rts::SweepUnit &U) { return (long long)U.NM * (U.wrap ? 2 : 1); }

}  // namespace

extern "C" rts_status rts_create_batched(rts_handle **out, int nsub, const rts_grid *grids, int nbands,
                                         const rts_quadrature *q, const rts_options *opt)
{
    if (!out) return RTS_EINVAL;
    *out = nullptr;
    rts_handle *h = new (std::nothrow) rts_handle();
    if (!h) return RTS_ENOMEM;
    if (opt) h->opt = *opt;
    else rts_default_options(&h->opt);
    rts_options &o = h->opt;
    auto bail = [&](rts_status s) {
        *out = h;
        return s;
    };
    if (nsub < 1 || !grids || nbands < 1) return bail(fail(h, RTS_EINVAL, "need nsub >= 1, grids and nbands >= 1"));
    for (int s = 0; s < nsub; ++s) {
        const rts_grid &g = grids[s];
        if (g.nx < 1 || g.ny < 1 || g.nz < 2)
            return bail(fail(h, RTS_EINVAL, "subdomain %d: need nx, ny >= 1 and nz >= 2", s));
        if (!(g.dx > 0 && g.dy > 0 && g.dz > 0) || !std::isfinite(g.dx) || !std::isfinite(g.dy) || !std::isfinite(g.dz))
            return bail(fail(h, RTS_EINVAL, "subdomain %d: spacing must be finite and positive", s));
    }
    if (o.prec != RTS_FP64 && o.prec != RTS_FP32_MIXED && o.prec != RTS_FP32_COMPENSATED)
        return bail(fail(h, RTS_EINVAL, "unknown precision %d", (int)o.prec));
    if (!(o.tau_switch > 0)) return bail(fail(h, RTS_EINVAL, "tau_switch must be > 0"));
    if (o.flags & (RTS_FLAG_ADJOINT | RTS_FLAG_HOST_IO | RTS_FLAG_HOST_IO_ASYNC | RTS_FLAG_LOG_CHI))
        return bail(fail(h, RTS_EINVAL,
                         "batched handles take none of RTS_FLAG_ADJOINT, RTS_FLAG_HOST_IO(_ASYNC), RTS_FLAG_LOG_CHI"));
    if (o.max_wrap_iters < 1) o.max_wrap_iters = 64;
    if (!(o.timeout_s > 0)) o.timeout_s = 2.0;
    if (!(o.wrap_tol > 0)) o.wrap_tol = o.prec == RTS_FP64 ? 1e-15 : 0x1p-24;
    h->batched = true;
    h->nsub = nsub;
    h->g = grids[0];
    h->B = nbands;
    h->stream = (cudaStream_t)o.stream;
    h->esize = o.prec == RTS_FP64 ? 8 : 4;
    if (q && q->ndir > 0) {
        if (!q->n || !q->w) return bail(fail(h, RTS_EINVAL, "quadrature arrays are NULL"));
        h->n.assign(q->n, q->n + 3 * q->ndir);
        h->w.assign(q->w, q->w + q->ndir);
    } else {
        default_quadrature(h->n, h->w);
    }
    h->ndir = (int)h->w.size();

    // ---- units of every subdomain (per subdomain in band-major plan order) ----
    int npmax = 0;
    long long maxext = 0;
    for (int s = 0; s < nsub; ++s) {
        npmax = std::max(npmax, std::max(grids[s].nx, grids[s].ny));
        maxext = std::max<long long>(maxext, std::max(grids[s].nx, std::max(grids[s].ny, grids[s].nz)));
    }
    if (npmax > 1024) return bail(fail(h, RTS_EINVAL, "plane extent %d > 1024 is not supported", npmax));
    int nqmax = 0;
    for (int s = 0; s < nsub; ++s) nqmax = std::max(nqmax, std::max(grids[s].ny, grids[s].nz));
    int dev = 0, nsm = 0;
    CUDA_TRY(h, cudaGetDevice(&dev));
    CUDA_TRY(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const Tiling tl = o.prec == RTS_FP64 ? choose_fwd<double>(o.tile_rows, npmax, nqmax, nsm)
                                         : choose_fwd<float>(o.tile_rows, npmax, nqmax, nsm);
    if (tl.tq < 1) return bail(fail(h, RTS_EINVAL, "no sweep tile fits plane extent %d", npmax));
    const int tq = tl.tq;
    h->tq = tq;
    h->nt = tl.nt;
    h->maxt = tl.maxt;
    h->smem = tl.smem;
    h->carveout = carveout_percent(tl.blocks, tl.smem,
                                   o.prec == RTS_FP64 ? (const void *)fwd_kernel<double>(tq, tl.maxt)
                                                      : (const void *)fwd_kernel<float>(tq, tl.maxt));

    std::vector<rts::SweepUnit> plan;       // plan order
    std::vector<int> plan_sub;              // subdomain of each planned unit
    std::vector<int> ru_begin(1, 0);        // per (subdomain, band)
    h->subs.resize(nsub);
    const int max_units = nbands * 6 * h->ndir;
    std::vector<rts::SweepUnit> tmp(max_units);
    std::vector<int> tmp_uot((size_t)max_units * ((maxext + tq - 1) / tq));
    long long in_off = 0, top_off = 0, out_off = 0, jf_off = 0, blk[3] = {0, 0, 0};
    for (int s = 0; s < nsub; ++s) {
        const rts_grid &g = grids[s];
        const double hsp[3] = {g.dx, g.dy, g.dz};
        std::vector<DirGeo> geo(h->ndir);
        std::vector<int> udx(h->ndir);
        int nup = 0, ndn = 0;
        for (int d = 0; d < h->ndir; ++d) {
            if (!direction_geometry(hsp, &h->n[3 * d], geo[d]))
                return bail(fail(h, RTS_EINVAL, "direction %d has n_z == 0 or is zero", d));
            udx[d] = geo[d].up ? nup++ : ndn++;
        }
        h->n_up = nup;
        h->n_dn = ndn;
        PlanOut po;
        if (!plan_units(geo.data(), udx.data(), h->n.data(), h->w.data(), h->ndir, g.nx, g.ny, g.nz, nbands, tq,
                        tmp.data(), max_units, tmp_uot.data(), (int)tmp_uot.size(), po))
            return bail(fail(h, RTS_EINVAL, "subdomain %d: too many sweep units or tiles", s));
        const long long N = (long long)g.nx * g.ny * g.nz;
        rts::SubDesc &sd = h->subs[s];
        std::memset(&sd, 0, sizeof(sd));
        sd.nx = g.nx; sd.ny = g.ny; sd.nz = g.nz; sd.N = N;
        sd.in_off = in_off; sd.top_off = top_off; sd.out_off = out_off; sd.jf_off = jf_off;
        sd.ru0 = s * nbands;
        for (int w = 0; w < 3; ++w) {
            sd.blk[w] = (int)blk[w];
            blk[w] += rts::sub_blocks(w, g.nx, g.ny, g.nz, nbands);
        }
        sd.P.nx = g.nx; sd.P.ny = g.ny; sd.P.nz = g.nz; sd.P.nbands = nbands;
        sd.P.inv2dx = 0.5 / g.dx; sd.P.inv2dy = 0.5 / g.dy; sd.P.inv2dz = 0.5 / g.dz; sd.P.invdz = 1.0 / g.dz;
        sd.P.thin = std::min(g.dx, std::min(g.dy, g.dz)) / o.tau_switch;
        for (int u = 0; u < po.nunits; ++u) {
            rts::SweepUnit U = tmp[u];
            U.in_off += in_off;
            U.top_off += top_off;
            U.dn_off = 0;  // explicit boundary arrays are not taken by batched solves
            plan.push_back(U);
            plan_sub.push_back(s);
        }
        // units of (s, b) in plan order
        std::vector<int> cnt(nbands, 0);
        for (int u = 0; u < po.nunits; ++u) cnt[tmp[u].band]++;
        for (int b = 0; b < nbands; ++b) ru_begin.push_back(ru_begin.back() + cnt[b]);
        in_off += (long long)nbands * N;
        top_off += (long long)nbands * nup * g.nx * g.ny;
        out_off += N;
        jf_off += (long long)nbands * 4 * N;
        h->has_x = h->has_x || po.has_x;
    }
    if (blk[0] > 0x7fffffffLL || blk[1] > 0x7fffffffLL || blk[2] > 0x7fffffffLL)
        return bail(fail(h, RTS_EINVAL, "batch too large for one launch of the per-grid kernels"));
    h->in_total = in_off;
    h->top_total = top_off;
    h->out_total = out_off;
    for (int w = 0; w < 3; ++w) h->nblk[w] = blk[w];

    // ---- sweep order: longest units first (tickets are handed out in this order) ----
    const int nunits = (int)plan.size();
    std::vector<int> order(nunits);
    for (int u = 0; u < nunits; ++u) order[u] = u;
    auto warps_of = [&](int u) { return (plan[u].NP + 31) / 32; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (warps_of(a) != warps_of(b)) return warps_of(a) > warps_of(b);
        return unit_weight(plan[a]) > unit_weight(plan[b]);
    });
    std::vector<int> pos(nunits);
    h->units.resize(nunits);
    h->unit_of_tile.clear();
    long long halo = 0, part_elems = 0;
    std::vector<long long> part_off(nunits);
    for (int k = 0; k < nunits; ++k) {
        rts::SweepUnit U = plan[order[k]];
        pos[order[k]] = k;
        U.tile0 = (int)h->unit_of_tile.size();
        for (int t = 0; t < U.ntiles; ++t) h->unit_of_tile.push_back(k);
        U.halo_off = halo;
        halo += (long long)U.ntiles * 4 * rts::HALO_CH * U.NP;
        part_off[k] = part_elems;
        part_elems += 4 * U.N;
        h->max_ntiles = std::max(h->max_ntiles, U.ntiles);
        h->units[k] = U;
    }
    h->total_tiles = (int)h->unit_of_tile.size();
    int R = 8;
    while (R < 2 * (h->max_ntiles + kLag + 2)) R *= 2;
    h->R = R;

    h->grid = std::min(h->total_tiles, tl.blocks * nsm);
    h->flag_tiles = 2 * h->total_tiles;  // a pair per tile
    // CTA-width classes (units are ordered by class): each class gets a CTA of
    // its own width, shared memory for its widest plane and its occupancy;
    // every unit's tiles must still fit on the GPU at once within its class
    for (int k = 0; k < nunits;) {
        const int w = (h->units[k].NP + 31) / 32;
        rts_handle::SweepClass C;
        C.tile_base = h->units[k].tile0;
        int npc = 0, maxnt = 0;
        int k1 = k;
        for (; k1 < nunits && (h->units[k1].NP + 31) / 32 == w; ++k1) {
            npc = std::max(npc, h->units[k1].NP);
            maxnt = std::max(maxnt, h->units[k1].ntiles);
            C.ntiles += h->units[k1].ntiles;
        }
        C.nt = 32 * w;
        C.smem = fwd_smem(tq, npc, (int)h->esize);
        int blocks = 0;
        if (class_blocks((int)h->esize, tq, h->maxt, C.nt, C.smem, &blocks) != cudaSuccess || blocks < 1 ||
            (long long)blocks * nsm < maxnt)
            return bail(fail(h, RTS_EINVAL, "no co-resident launch for the subdomains of plane width %d", npc));
        C.grid = std::min(C.ntiles, blocks * nsm);
        C.carveout = carveout_percent(blocks, C.smem,
                                      h->esize == 8 ? (const void *)fwd_kernel<double>(tq, h->maxt)
                                                    : (const void *)fwd_kernel<float>(tq, h->maxt));
        h->classes.push_back(C);
        k = k1;
    }

    // ---- FP32: the register-resident sweep, one persistent launch for every
    // subdomain (units narrower than the CTA leave their extra threads idle) ----
    long long reg_halo = 0;
    if (o.prec != RTS_FP64 && o.sweep_kernel != RTS_SWEEP_SHARED && reg_eligible(h->units)) {
        int nq_per = 0;  // the tile height must divide every subdomain's periodic z-group rows (ny)
        for (int s = 0; s < nsub; ++s) nq_per = std::gcd(nq_per, grids[s].ny);
        const Tiling tr = choose_reg(o.tile_rows, npmax, nqmax, nq_per, nsm);
        if (tr.tq >= 1) {
            std::vector<rts::SweepUnit> rplan;
            std::vector<int> rtmp_uot((size_t)max_units * ((maxext + tr.tq - 1) / tr.tq));
            bool ok = true;
            for (int s = 0; s < nsub && ok; ++s) {
                const rts_grid &g = grids[s];
                const double hsp[3] = {g.dx, g.dy, g.dz};
                std::vector<DirGeo> geo(h->ndir);
                std::vector<int> udx(h->ndir);
                int nup = 0, ndn = 0;
                for (int d = 0; d < h->ndir; ++d) {
                    direction_geometry(hsp, &h->n[3 * d], geo[d]);
                    udx[d] = geo[d].up ? nup++ : ndn++;
                }
                PlanOut pr;
                ok = plan_units(geo.data(), udx.data(), h->n.data(), h->w.data(), h->ndir, g.nx, g.ny, g.nz, nbands,
                                tr.tq, tmp.data(), max_units, rtmp_uot.data(), (int)rtmp_uot.size(), pr);
                for (int u = 0; ok && u < pr.nunits; ++u) {
                    rts::SweepUnit U = tmp[u];
                    U.in_off += h->subs[s].in_off;
                    U.top_off += h->subs[s].top_off;
                    U.dn_off = 0;
                    rplan.push_back(U);
                }
            }
            if (ok && (int)rplan.size() == nunits) {
                h->reg_units.resize(nunits);
                h->reg_unit_of_tile.clear();
                for (int k = 0; k < nunits; ++k) {  // the shared-sweep order, so that unit k is the same in both
                    rts::SweepUnit U = rplan[order[k]];
                    U.tile0 = (int)h->reg_unit_of_tile.size();
                    for (int t = 0; t < U.ntiles; ++t) h->reg_unit_of_tile.push_back(k);
                    U.halo_off = reg_halo;
                    reg_halo += (long long)U.ntiles * rts::reg_ring_elems(U.NP);
                    h->reg_units[k] = U;
                }
                h->reg_total_tiles = (int)h->reg_unit_of_tile.size();
                h->reg_tq = tr.tq;
                h->reg_maxr = tr.maxt;
                h->reg_nt = tr.nt;
                h->reg_smem = tr.smem;
                h->reg_carveout = carveout_percent(tr.blocks, tr.smem,
                                                   (const void *)rts::reg_kernel_f32(tr.tq, tr.maxt));
                h->reg_grid = std::min(h->reg_total_tiles, tr.blocks * nsm);
                h->flag_tiles = std::max(h->flag_tiles, 2 * h->reg_total_tiles);
                h->use_reg = true;
            } else {
                h->reg_units.clear();
                h->reg_unit_of_tile.clear();
                reg_halo = 0;
            }
        }
    }

    // ---- device memory ----
    const size_t es = h->esize;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = round_up(off + bytes, 256); return at; };
    const size_t o_units = take(sizeof(rts::SweepUnit) * nunits);
    const size_t o_uot = take(sizeof(int) * h->unit_of_tile.size());
    const size_t o_regu = h->use_reg ? take(sizeof(rts::SweepUnit) * nunits) : 0;
    const size_t o_reguot = h->use_reg ? take(2 * sizeof(int) * h->reg_unit_of_tile.size()) : 0;  // and the ticket order
    const size_t o_part = take((size_t)part_elems * es);
    const size_t o_chiT = h->has_x ? take((size_t)h->in_total * es) : 0;
    const size_t o_ST = h->has_x ? take((size_t)h->in_total * es) : 0;
    const size_t o_JF = take((size_t)jf_off * 8);
    const size_t o_halo = take((size_t)std::max(halo, reg_halo) * es);
    const size_t o_flags = take(sizeof(int) * h->flag_tiles);
    const size_t o_gcnt = take(sizeof(unsigned int) * nunits * (R + 4));
    const size_t o_gmax = take(sizeof(unsigned long long) * nunits * (R + 4));
    const size_t o_ticket = take(sizeof(int) * 4);
    const size_t o_status = take(sizeof(int) * 4);
    const size_t o_tacc = take(sizeof(int) * nunits);
    const size_t o_ru = take(sizeof(rts::RedUnit) * nunits);
    const size_t o_rub = take(sizeof(int) * ru_begin.size());
    const size_t o_subs = take(sizeof(rts::SubDesc) * nsub);
    cudaError_t ae = cudaMalloc(&h->dmem, off);
    if (ae != cudaSuccess) {
        h->dmem = nullptr;
        return bail(fail(h, RTS_ENOMEM, "cudaMalloc of %zu bytes: %s", off, cudaGetErrorString(ae)));
    }
    char *base = (char *)h->dmem;
    h->d_units = (rts::SweepUnit *)(base + o_units);
    h->d_unit_of_tile = (int *)(base + o_uot);
    h->d_partial = base + o_part;
    h->d_chiT = h->has_x ? base + o_chiT : nullptr;
    h->d_ST = h->has_x ? base + o_ST : nullptr;
    h->d_JF = base + o_JF;
    h->d_halo = base + o_halo;
    h->d_flags = (int *)(base + o_flags);
    h->d_gcnt = (unsigned int *)(base + o_gcnt);
    h->d_gmax = (unsigned long long *)(base + o_gmax);
    h->d_ticket = (int *)(base + o_ticket);
    h->d_status = (int *)(base + o_status);
    h->d_unit_tacc = (int *)(base + o_tacc);
    h->d_ru = (rts::RedUnit *)(base + o_ru);
    h->d_ru_begin = (int *)(base + o_rub);
    h->d_subs = (rts::SubDesc *)(base + o_subs);
    std::vector<rts::RedUnit> ru(nunits);
    for (int k = 0; k < nunits; ++k) h->units[k].partial = (char *)h->d_partial + part_off[k] * es;
    for (int u = 0; u < nunits; ++u) {  // reduction table in plan order: (subdomain, band), then group
        ru[u] = red_unit(h->units[pos[u]]);
    }
    CUDA_TRY(h, cudaMemcpy(h->d_units, h->units.data(), sizeof(rts::SweepUnit) * nunits, cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(h->d_unit_of_tile, h->unit_of_tile.data(), sizeof(int) * h->unit_of_tile.size(),
                           cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(h->d_ru, ru.data(), sizeof(rts::RedUnit) * nunits, cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(h->d_ru_begin, ru_begin.data(), sizeof(int) * ru_begin.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(h->d_subs, h->subs.data(), sizeof(rts::SubDesc) * nsub, cudaMemcpyHostToDevice));
    if (h->use_reg) {
        h->d_reg_units = (rts::SweepUnit *)(base + o_regu);
        h->d_reg_uot = (int *)(base + o_reguot);
        h->d_reg_order = h->d_reg_uot + h->reg_unit_of_tile.size();
        for (int k = 0; k < nunits; ++k) h->reg_units[k].partial = h->units[k].partial;
        CUDA_TRY(h, cudaMemcpy(h->d_reg_units, h->reg_units.data(), sizeof(rts::SweepUnit) * nunits,
                               cudaMemcpyHostToDevice));
        CUDA_TRY(h, cudaMemcpy(h->d_reg_uot, h->reg_unit_of_tile.data(), sizeof(int) * h->reg_unit_of_tile.size(),
                               cudaMemcpyHostToDevice));
        const std::vector<int> order = ticket_order(h->reg_units);
        CUDA_TRY(h, cudaMemcpy(h->d_reg_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice));
    }
    h->band_unit.assign(1, 0);
    CUDA_TRY(h, cudaMemset(h->d_status, 0, sizeof(int) * 4));
    CUDA_TRY(h, cudaMemset(h->d_unit_tacc, 0, sizeof(int) * nunits));
    h->timing = (o.flags & RTS_FLAG_TIMING) != 0;
    *out = h;
    return RTS_OK;
}

template <typename T, typename Acc>
static rts_status solve_batched_impl(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc,
                                     void *I_top, double *J, double *F, double *Q)
{
    cudaStream_t st = h->stream;
    const int ns = h->nsub;
    CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int) * 4, st));
    CUDA_TRY(h, cudaMemsetAsync(h->d_unit_tacc, 0, sizeof(int) * h->units.size(), st));
    rts_status rs = reset_sweep_state(h, st);
    if (rs) return rs;
    cudaEvent_t *ev = nullptr;
    if (h->timing && !h->capturing) {
        if (h->nrec == h->evs.size()) {
            std::array<cudaEvent_t, 5> set{};
            for (cudaEvent_t &e : set) CUDA_TRY(h, cudaEventCreate(&e));
            h->evs.push_back(set);
        }
        ev = h->evs[h->nrec++].data();
        CUDA_TRY(h, cudaEventRecord(ev[0], st));
    }
    int kernels = 0;
    if (h->has_x) {
        rts::transpose_x2_batched<T><<<(unsigned)h->nblk[0], dim3(32, 8), 0, st>>>(h->d_subs, ns, h->B, (const T *)chi,
                                                                                  (const T *)S, (T *)h->d_chiT,
                                                                                  (T *)h->d_ST, h->d_status);
        CUDA_TRY(h, cudaGetLastError());
        kernels += 1;
    }
    if (ev) CUDA_TRY(h, cudaEventRecord(ev[1], st));
    rts::SweepArgs<T> a = sweep_args<T>(h, chi, S, bc);
    a.itop = (T *)I_top;
    int launches = 0;
    const bool reg = h->use_reg && sizeof(T) == 4;
    cudaError_t e = reg ? launch_reg_sweep(h, *reinterpret_cast<const rts::SweepArgs<float> *>(&a))
                        : launch_sweep_classes<T>(h, a, &launches);
    if (e != cudaSuccess) return fail(h, RTS_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
    kernels += reg ? 1 : launches;
    if (ev) CUDA_TRY(h, cudaEventRecord(ev[2], st));
    if (J || F || Q) {
        rts::reduce_units_batched<T, Acc><<<(unsigned)h->nblk[1], dim3(32, 8), 0, st>>>(
            h->d_subs, ns, h->d_ru, h->d_ru_begin, (Acc *)h->d_JF, reg ? 1 : 0);
        if (ev) CUDA_TRY(h, cudaEventRecord(ev[3], st));
        rts::qstep_batched<T, Acc><<<(unsigned)h->nblk[2], dim3(32, 8), 0, st>>>(
            h->d_subs, ns, (const Acc *)h->d_JF, (const T *)chi, (const T *)S, J, F, Q);
        CUDA_TRY(h, cudaGetLastError());
        kernels += 2;
    } else if (ev) {
        CUDA_TRY(h, cudaEventRecord(ev[3], st));
    }
    if (ev) CUDA_TRY(h, cudaEventRecord(ev[4], st));
    h->kernels_last = kernels;
    return RTS_OK;
}

extern "C" rts_status rts_solve_batched(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc,
                                        void *I_top, double *J, double *F, double *Q)
{
    if (!h || !h->dmem) return h ? fail(h, RTS_EINVAL, "handle was not created successfully") : RTS_EINVAL;
    if (!h->batched) return fail(h, RTS_EINVAL, "rts_solve_batched needs a handle from rts_create_batched");
    if (!chi || !S) return fail(h, RTS_EINVAL, "chi and S must not be NULL");
    if (bc && (bc->bottom == RTS_BC_EXPLICIT || bc->top == RTS_BC_EXPLICIT))
        return fail(h, RTS_EINVAL, "batched solves take boundary kinds ZERO and EQUAL_S only");
    rts_status s = check_bc(h, bc);
    if (s) return s;
    switch (h->opt.prec) {
    case RTS_FP64: return solve_batched_impl<double, double>(h, chi, S, bc, I_top, J, F, Q);
    case RTS_FP32_MIXED: return solve_batched_impl<float, double>(h, chi, S, bc, I_top, J, F, Q);
    default: return solve_batched_impl<float, rts::df32>(h, chi, S, bc, I_top, J, F, Q);
    }
}

extern "C" rts_status rts_batched_layout(rts_handle *h, int sub, long long *grid_offset, long long *top_offset,
                                         long long *point_offset, long long totals[3])
{
    if (!h || !h->dmem || !h->batched) return h ? fail(h, RTS_EINVAL, "not a batched handle") : RTS_EINVAL;
    if (sub < 0 || sub >= h->nsub) return fail(h, RTS_EINVAL, "subdomain %d out of range", sub);
    const rts::SubDesc &sd = h->subs[sub];
    if (grid_offset) *grid_offset = sd.in_off;
    if (top_offset) *top_offset = sd.top_off;
    if (point_offset) *point_offset = sd.out_off;
    if (totals) {
        totals[0] = h->in_total;
        totals[1] = h->top_total;
        totals[2] = h->out_total;
    }
    return RTS_OK;
}

// ---- CUDA graph of one solve ----------------------------------------------
struct rts_graph {
    rts_handle *h = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" rts_status rts_graph_create(rts_handle *h, const void *chi, const void *S, const rts_boundary *bc,
                                       void *I_top, double *J, double *F, double *Q, rts_graph **out)
{
    if (!h || !h->dmem || !out) return h ? fail(h, RTS_EINVAL, "bad arguments") : RTS_EINVAL;
    *out = nullptr;
    if (!h->stream) return fail(h, RTS_EINVAL, "graph capture needs a handle created with a non-default stream");
    rts_graph *g = new (std::nothrow) rts_graph();
    if (!g) return RTS_ENOMEM;
    g->h = h;
    CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    rts_status s = h->batched ? rts_solve_batched(h, chi, S, bc, I_top, J, F, Q) : rts_solve(h, chi, S, bc, I_top, J, F, Q);
    h->capturing = false;
    cudaError_t ce = cudaStreamEndCapture(h->stream, &g->graph);
    if (s != RTS_OK || ce != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return s != RTS_OK ? s : fail(h, RTS_ECUDA, "stream capture: %s", cudaGetErrorString(ce));
    }
    ce = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (ce != cudaSuccess) {
        cudaGraphDestroy(g->graph);
        delete g;
        return fail(h, RTS_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    }
    *out = g;
    return RTS_OK;
}

extern "C" rts_status rts_graph_launch(rts_graph *g)
{
    if (!g || !g->exec) return RTS_EINVAL;
    CUDA_TRY(g->h, cudaGraphLaunch(g->exec, g->h->stream));
    return RTS_OK;
}

extern "C" void rts_graph_destroy(rts_graph *g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

// ---- tile-size autotuner --------------------------------------------------
extern "C" rts_status rts_autotune(int nsub, const rts_grid *grids, int nbands, const rts_quadrature *q,
                                   const rts_options *opt, const void *chi, const void *S, int repeats,
                                   int *best_tile_rows, int *ncand, int rows[8], float ms[8])
{
    if (nsub < 1 || !grids || !chi || !S || !best_tile_rows) return RTS_EINVAL;
    rts_options o;
    if (opt) o = *opt;
    else rts_default_options(&o);
    o.flags &= ~(RTS_FLAG_TIMING | RTS_FLAG_ADJOINT | RTS_FLAG_HOST_IO);
    const int reps = std::max(1, repeats);
    const int cand[8] = {1, 2, 4, 6, 7, 8, 12, 16};
    float best = 0.f;
    int n = 0;
    *best_tile_rows = 0;
    for (int c = 0; c < 8; ++c) {
        const int tq = cand[c];
        o.tile_rows = tq;
        rts_handle *h = nullptr;
        rts_status s = rts_create_batched(&h, nsub, grids, nbands, q, &o);
        if (s != RTS_OK || !h || h->tq != tq) {  // not instantiated for this extent, or does not fit
            rts_destroy(h);
            continue;
        }
        cudaStream_t st = h->stream;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        bool ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
        ok = ok && rts_solve_batched(h, chi, S, nullptr, nullptr, nullptr, nullptr, nullptr) == RTS_OK;
        ok = ok && cudaEventRecord(e0, st) == cudaSuccess;
        for (int r = 0; ok && r < reps; ++r)
            ok = rts_solve_batched(h, chi, S, nullptr, nullptr, nullptr, nullptr, nullptr) == RTS_OK;
        ok = ok && cudaEventRecord(e1, st) == cudaSuccess && rts_check(h) == RTS_OK;
        float t = 0.f;
        ok = ok && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        rts_destroy(h);
        if (!ok) continue;
        t /= reps;
        if (rows && ms && n < 8) {
            rows[n] = tq;
            ms[n] = t;
        }
        ++n;
        if (*best_tile_rows == 0 || t < best) {
            best = t;
            *best_tile_rows = tq;
        }
    }
    if (ncand) *ncand = std::min(n, 8);
    return *best_tile_rows ? RTS_OK : RTS_ECUDA;
}

// ===========================================================================
// Spatial decomposition (the paper's scheme, Sect. 2 and 5.1: the domain is
// split into sub-domains, each integrates its rays from the boundary
// intensities of the previous iteration, and the boundary intensities are
// iterated until a global error is below a tolerance). Here the sub-domains
// are slabs of levels on one GPU (the horizontal periodic wrap stays inside
// every slab's solve). Slab k owns levels [a_k, b_k) and is solved on
// [a_k - 1, b_k + 1) (one ghost level each side where it has a neighbour):
// its bottom layer takes the upward intensities that slab k-1 computed at
// level a_k - 1, its top layer the downward intensities that slab k+1
// computed at level b_k, both from the previous iteration (block Jacobi).
// Those intensities are gathered from the neighbours' raw slot partials (the
// register sweep stores every ray's intensity at every point), and with a
// ghost level on each side every owned level sees the same neighbours as in
// the undecomposed solve, so J, F and Q_rad of the owned levels converge to
// the undecomposed values. Convergence: the largest change of J between two
// iterations, relative to max J (the paper's global J criterion).
// ===========================================================================

namespace {

struct GatherEnt {
    const float *part;   // the unit's raw partials [N][4] in its layout
    long long sQ, sM;
    int axis, slot, band, dir;
};

// intensity of every gathered (unit, slot) at grid level `level` of a slab,
// into out[band][dir][j][i] (the layout of the explicit boundary arrays)
__global__ void __launch_bounds__(256) gather_level_kernel(const GatherEnt *__restrict__ ents, int nx, int ny,
                                                            int level, int ndir_sel, float *__restrict__ out)
{
    const GatherEnt e = ents[blockIdx.y];
    const long long ij = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ij >= (long long)nx * ny) return;
    const int i = (int)(ij % nx), j = (int)(ij / nx);
    int p, q, m;
    if (e.axis == 2) { p = i; q = j; m = level; }
    else if (e.axis == 1) { p = i; q = level; m = j; }
    else { p = j; q = level; m = i; }
    const float v = e.part[((long long)m * e.sM + (long long)q * e.sQ + p) * 4 + e.slot];
    out[(((long long)e.band * ndir_sel + e.dir) * ny + j) * nx + i] = v;
}

// largest |a - b| and |a| over n values (atomic maxima of their float bits)
__global__ void __launch_bounds__(256) change_kernel(const double *__restrict__ a, const double *__restrict__ b,
                                                      long long n, unsigned *out)
{
    float d = 0.f, m = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        d = fmaxf(d, (float)fabs(a[i] - b[i]));
        m = fmaxf(m, (float)fabs(a[i]));
    }
    for (int o = 16; o; o >>= 1) {
        d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, __float_as_uint(d));
        atomicMax(out + 1, __float_as_uint(m));
    }
}

}  // namespace

struct rts_decomp {
    rts_grid g{};
    int B = 0, n_up = 0, n_dn = 0, nblk = 0;
    std::vector<rts_handle *> blk;
    std::vector<int> lo, hi, a, b;   // slab grid [lo, hi) and owned levels [a, b)
    void *mem = nullptr;
    std::vector<float *> chi, S;       // per slab inputs [B][hi-lo][N2]
    std::vector<double *> J, F, Q;     // per slab outputs
    std::vector<float *> up[2], dn[2]; // per interface k (between slab k and k+1), double-buffered
    std::vector<GatherEnt *> ents_up, ents_dn;  // per slab: its rising / descending (unit, slot) entries
    std::vector<int> nent_up, nent_dn;
    double *Jprev = nullptr;
    unsigned *dmax = nullptr;
    cudaStream_t stream = nullptr;
    char err[512] = {0};
};

extern "C" {

rts_status rts_create_decomposed(rts_decomp **out, const rts_grid *g, int nbands, int nblocks,
                                 const rts_quadrature *q, const rts_options *opt)
{
    if (!out) return RTS_EINVAL;
    *out = nullptr;
    rts_decomp *d = new (std::nothrow) rts_decomp();
    if (!d) return RTS_ENOMEM;
    *out = d;
    auto bad = [&](rts_status s, const char *m) {
        snprintf(d->err, sizeof(d->err), "%s", m);
        return s;
    };
    rts_options o;
    if (opt) o = *opt;
    else rts_default_options(&o);
    if (!g || nbands < 1 || nblocks < 1) return bad(RTS_EINVAL, "grid, nbands >= 1 and nblocks >= 1 are needed");
    if (o.prec == RTS_FP64) return bad(RTS_EINVAL, "the decomposed solve needs an FP32 mode (raw slot partials)");
    if (g->nz < 2 * nblocks) return bad(RTS_EINVAL, "every slab needs at least 2 levels of its own");
    if (o.flags & ~RTS_FLAG_TIMING) return bad(RTS_EINVAL, "the decomposed solve takes only RTS_FLAG_TIMING");
    o.sweep_kernel = RTS_SWEEP_REGISTER;
    d->g = *g;
    d->B = nbands;
    d->nblk = nblocks;
    d->stream = (cudaStream_t)o.stream;
    const long long N2 = (long long)g->nx * g->ny;
    for (int k = 0; k < nblocks; ++k) {
        d->a.push_back((int)((long long)g->nz * k / nblocks));
        d->b.push_back((int)((long long)g->nz * (k + 1) / nblocks));
        d->lo.push_back(std::max(d->a[k] - 1, 0));
        d->hi.push_back(std::min(d->b[k] + 1, g->nz));
        rts_grid gk = *g;
        gk.nz = d->hi[k] - d->lo[k];
        rts_handle *h = nullptr;
        rts_status s = rts_create(&h, &gk, nbands, q, &o);
        d->blk.push_back(h);
        if (s) return bad(s, h ? h->err : "slab handle");
    }
    d->n_up = d->blk[0]->n_up;
    d->n_dn = d->blk[0]->n_dn;
    // device memory: slab inputs and outputs, interface arrays, the change check
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = round_up(off + bytes, 256); return at; };
    std::vector<size_t> oc, os, oj, of, oq, oeu, oed;
    for (int k = 0; k < nblocks; ++k) {
        const long long nk = (long long)(d->hi[k] - d->lo[k]) * N2;
        oc.push_back(take(sizeof(float) * nbands * nk));
        os.push_back(take(sizeof(float) * nbands * nk));
        oj.push_back(take(sizeof(double) * nk));
        of.push_back(take(sizeof(double) * 3 * nk));
        oq.push_back(take(sizeof(double) * nk));
        oeu.push_back(take(sizeof(GatherEnt) * nbands * d->n_up));
        oed.push_back(take(sizeof(GatherEnt) * nbands * d->n_dn));
    }
    std::vector<size_t> ou[2], odn[2];
    for (int k = 0; k + 1 < nblocks; ++k)
        for (int t = 0; t < 2; ++t) {
            ou[t].push_back(take(sizeof(float) * nbands * d->n_up * N2));
            odn[t].push_back(take(sizeof(float) * nbands * d->n_dn * N2));
        }
    const size_t oJp = take(sizeof(double) * N2 * g->nz);
    const size_t omax = take(sizeof(unsigned) * 4);
    if (cudaMalloc(&d->mem, off) != cudaSuccess) {
        d->mem = nullptr;
        return bad(RTS_ENOMEM, "cudaMalloc of the decomposition's buffers failed");
    }
    char *base = (char *)d->mem;
    for (int k = 0; k < nblocks; ++k) {
        d->chi.push_back((float *)(base + oc[k]));
        d->S.push_back((float *)(base + os[k]));
        d->J.push_back((double *)(base + oj[k]));
        d->F.push_back((double *)(base + of[k]));
        d->Q.push_back((double *)(base + oq[k]));
        // the slab's (unit, slot) entries, rising and descending
        rts_handle *h = d->blk[k];
        std::vector<GatherEnt> eu, ed;
        for (const rts::SweepUnit &U : h->units)
            for (int sl = 0; sl < rts::MAXD; ++sl) {
                if (!U.active[sl]) continue;
                GatherEnt e;
                e.part = (const float *)U.partial;
                e.sQ = U.sQ;
                e.sM = U.sM;
                e.axis = U.axis;
                e.slot = sl;
                e.band = U.band;
                e.dir = U.udx[sl];
                (U.up[sl] ? eu : ed).push_back(e);
            }
        d->ents_up.push_back((GatherEnt *)(base + oeu[k]));
        d->ents_dn.push_back((GatherEnt *)(base + oed[k]));
        d->nent_up.push_back((int)eu.size());
        d->nent_dn.push_back((int)ed.size());
        if (eu.size() > (size_t)nbands * d->n_up || ed.size() > (size_t)nbands * d->n_dn)
            return bad(RTS_EINVAL, "gather table overflow");
        if (cudaMemcpy(d->ents_up[k], eu.data(), sizeof(GatherEnt) * eu.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d->ents_dn[k], ed.data(), sizeof(GatherEnt) * ed.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return bad(RTS_ECUDA, "copy of the gather tables failed");
    }
    for (int t = 0; t < 2; ++t)
        for (int k = 0; k + 1 < nblocks; ++k) {
            d->up[t].push_back((float *)(base + ou[t][k]));
            d->dn[t].push_back((float *)(base + odn[t][k]));
        }
    d->Jprev = (double *)(base + oJp);
    d->dmax = (unsigned *)(base + omax);
    return RTS_OK;
}

const char *rts_decomposed_last_error(rts_decomp *d) { return d ? d->err : "null handle"; }

void rts_destroy_decomposed(rts_decomp *d)
{
    if (!d) return;
    for (rts_handle *h : d->blk) rts_destroy(h);
    if (d->mem) cudaFree(d->mem);
    delete d;
}

rts_status rts_solve_decomposed(rts_decomp *d, const void *chi, const void *S, const rts_boundary *bc, double tol,
                                int max_iter, int *iters, void *I_top, double *J, double *F, double *Q_rad)
{
    if (!d || !d->mem) return RTS_EINVAL;
    auto bad = [&](rts_status s, const char *m) {
        snprintf(d->err, sizeof(d->err), "%s", m);
        return s;
    };
    if (!chi || !S || !J) return bad(RTS_EINVAL, "chi, S and J must not be NULL (J carries the convergence test)");
    if (max_iter < 1 || !(tol > 0)) return bad(RTS_EINVAL, "max_iter >= 1 and tol > 0 are needed");
    if (bc && bc->wrap_seed) return bad(RTS_EINVAL, "the decomposed solve takes no warm start");
    const rts_grid &g = d->g;
    const long long N2 = (long long)g.nx * g.ny, N = N2 * g.nz;
    cudaStream_t st = d->stream;
#define DC_TRY(call)                                                                                         \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess) return bad(RTS_ECUDA, cudaGetErrorString(e_));                                \
    } while (0)
    // the slabs' inputs: levels [lo, hi) of every band
    for (int k = 0; k < d->nblk; ++k) {
        const size_t w = sizeof(float) * (size_t)(d->hi[k] - d->lo[k]) * N2;
        const size_t sp = sizeof(float) * (size_t)N;
        DC_TRY(cudaMemcpy2DAsync(d->chi[k], w, (const float *)chi + d->lo[k] * N2, sp, w, d->B, cudaMemcpyDeviceToDevice, st));
        DC_TRY(cudaMemcpy2DAsync(d->S[k], w, (const float *)S + d->lo[k] * N2, sp, w, d->B, cudaMemcpyDeviceToDevice, st));
    }
    int it = 0, cur = 0;
    bool conv = false;
    for (; it < max_iter && !conv; ++it) {
        const int nxt = cur ^ 1;
        for (int k = 0; k < d->nblk; ++k) {
            rts_boundary b;
            std::memset(&b, 0, sizeof(b));
            b.bottom = bc ? bc->bottom : RTS_BC_EQUAL_S;
            b.top = bc ? bc->top : RTS_BC_ZERO;
            b.bottom_I = bc ? bc->bottom_I : nullptr;
            b.top_I = bc ? bc->top_I : nullptr;
            if (k > 0) {  // from slab k-1; the first iteration starts from I = S
                b.bottom = it == 0 ? RTS_BC_EQUAL_S : RTS_BC_EXPLICIT;
                b.bottom_I = d->up[cur][k - 1];
            }
            if (k + 1 < d->nblk) {
                b.top = it == 0 ? RTS_BC_EQUAL_S : RTS_BC_EXPLICIT;
                b.top_I = d->dn[cur][k];
            }
            rts_status s = rts_solve(d->blk[k], d->chi[k], d->S[k], &b, k + 1 == d->nblk ? I_top : nullptr, d->J[k],
                                     d->F[k], d->Q[k]);
            if (s) return bad(s, d->blk[k]->err);
            // the intensities the neighbours take next iteration
            const unsigned gx = (unsigned)((N2 + 255) / 256);
            if (k + 1 < d->nblk && d->nent_up[k] > 0)  // rising, at level b_k - 1 (slab k+1's bottom layer)
                gather_level_kernel<<<dim3(gx, (unsigned)d->nent_up[k]), 256, 0, st>>>(
                    d->ents_up[k], g.nx, g.ny, d->b[k] - 1 - d->lo[k], d->n_up, d->up[nxt][k]);
            if (k > 0 && d->nent_dn[k] > 0)  // descending, at level a_k (slab k-1's top layer)
                gather_level_kernel<<<dim3(gx, (unsigned)d->nent_dn[k]), 256, 0, st>>>(
                    d->ents_dn[k], g.nx, g.ny, d->a[k] - d->lo[k], d->n_dn, d->dn[nxt][k - 1]);
            DC_TRY(cudaGetLastError());
            // the owned levels of J
            DC_TRY(cudaMemcpyAsync(J + d->a[k] * N2, d->J[k] + (d->a[k] - d->lo[k]) * N2,
                                   sizeof(double) * (size_t)(d->b[k] - d->a[k]) * N2, cudaMemcpyDeviceToDevice, st));
        }
        // the global J criterion: max |J - J_prev| <= tol max |J|
        DC_TRY(cudaMemsetAsync(d->dmax, 0, sizeof(unsigned) * 2, st));
        change_kernel<<<(unsigned)std::min<long long>((N + 255) / 256, 148LL * 8), 256, 0, st>>>(J, d->Jprev, N,
                                                                                                 d->dmax);
        DC_TRY(cudaGetLastError());
        unsigned mx[2] = {0, 0};
        DC_TRY(cudaMemcpyAsync(mx, d->dmax, sizeof(mx), cudaMemcpyDeviceToHost, st));
        DC_TRY(cudaMemcpyAsync(d->Jprev, J, sizeof(double) * (size_t)N, cudaMemcpyDeviceToDevice, st));
        DC_TRY(cudaStreamSynchronize(st));
        for (rts_handle *h : d->blk) {
            rts_status s = rts_check(h);
            if (s) return bad(s, h->err);
        }
        float dj, jm;
        std::memcpy(&dj, &mx[0], sizeof(float));
        std::memcpy(&jm, &mx[1], sizeof(float));
        conv = it > 0 && dj <= tol * jm;
        cur = nxt;
    }
    if (iters) *iters = it;
    if (!conv) return bad(RTS_ENOCONV, "the slab iteration did not converge");
    // the owned levels of F and Q_rad from the last iteration
    for (int k = 0; k < d->nblk; ++k) {
        const size_t nb = sizeof(double) * (size_t)(d->b[k] - d->a[k]) * N2;
        const long long nk = (long long)(d->hi[k] - d->lo[k]) * N2;
        if (Q_rad) DC_TRY(cudaMemcpyAsync(Q_rad + d->a[k] * N2, d->Q[k] + (d->a[k] - d->lo[k]) * N2, nb,
                                          cudaMemcpyDeviceToDevice, st));
        if (F)
            for (int c = 0; c < 3; ++c)
                DC_TRY(cudaMemcpyAsync(F + c * N + d->a[k] * N2, d->F[k] + c * nk + (d->a[k] - d->lo[k]) * N2, nb,
                                       cudaMemcpyDeviceToDevice, st));
    }
#undef DC_TRY
    return RTS_OK;
}

}  // extern "C"

// common.cuh -- device helpers shared by the RTS kernels: memory-order
// primitives for the tile ready flags, bounded waits and the device status
// word. Every wait has a time limit; on expiry it records RTS_ETIMEOUT in the
// status word and returns false so the kernel can unwind (no trap, no hang).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rts {

// Device status bits (mapped to rts_status on the host).
enum : int { ST_TIMEOUT = 1, ST_NOCONV = 2, ST_BADARG = 4, ST_NONFINITE = 8 };

__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void st_relaxed(int *p, int v)
{
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until pair[0] >= w0 and pair[1] >= w1 (8-byte aligned pair), both
// read by one 8-byte acquire load per poll. Returns false (and records why)
// if the device status already carries an error or the time limit expires.
__device__ __forceinline__ bool wait_pair_geq(const int *pair, int w0, int w1, int *status, uint64_t limit_ns)
{
    const unsigned long long *p64 = reinterpret_cast<const unsigned long long *>(pair);
    auto ready = [&](unsigned long long v) { return (int)(unsigned)(v & 0xffffffffu) >= w0 && (int)(unsigned)(v >> 32) >= w1; };
    if (ready(ld_acquire64(p64))) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        __nanosleep(64);
        if (ready(ld_acquire64(p64))) return true;
        if (ld_relaxed(status) != 0) return false;
        if (global_ns() - t0 > limit_ns) {
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until *cnt >= want (same limits as wait_pair_geq).
__device__ __forceinline__ bool wait_count_geq(const unsigned *cnt, unsigned want, int *status, uint64_t limit_ns)
{
    if (ld_acquire_u32(cnt) >= want) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        __nanosleep(64);
        if (ld_acquire_u32(cnt) >= want) return true;
        if (ld_relaxed(status) != 0) return false;
        if (global_ns() - t0 > limit_ns) {
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
}

// Asynchronous global -> shared copies of one element (4 or 8 bytes).
template <typename T>
__device__ __forceinline__ void cp_async(T *smem_dst, const T *gmem_src)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element size");
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(gmem_src), "n"(sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Loads that bypass L1 (data written by other CTAs during this kernel).
template <typename T>
__device__ __forceinline__ T ld_cg(const T *p)
{
    return __ldcg(p);
}

}  // namespace rts

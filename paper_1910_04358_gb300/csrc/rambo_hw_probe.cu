// rambo_hw_probe.cu -- two hardware-rate microbenchmarks behind design
// choices (measurement support, not part of the method).
//
//   l2 atomics  64-bit atomicOr (no return value) at hashed addresses of a
//               buffer: with the buffer inside L2 this is the rate the
//               region-binned insert's apply pass can reach, with it far
//               larger the rate the direct insert meets.
//   tmem read   tcgen05.ld 32x32b.x32 from all 512 tensor-memory columns,
//               one CTA per SM, W warps each with L loads in flight before a
//               wait, every register folded: the rate at which an epilogue
//               can drain accumulators.
#include "rambo.h"
#include "rambo_internal.cuh"

namespace rgpu {
namespace {

constexpr int HW_THREADS = 256;

__device__ __forceinline__ uint64_t hw_mix(uint64_t x) {
    // SplitMix64's finaliser (a published 64-bit mixer)
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

__global__ void __launch_bounds__(HW_THREADS) k_l2_atomics(unsigned long long *buf, uint64_t mask, uint32_t ops) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t i = 0; i < ops; ++i) {
        const uint64_t h = hw_mix(t * 0x9E3779B97F4A7C15ull + i);
        atomicOr(buf + (h & mask), 1ull << (h >> 58));
    }
}

__device__ __forceinline__ void hw_tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// Warp w reads lane quadrant w % 4 (the quadrant its warp may access) and
// columns cycling through the 512 it allocated; cycles[blockIdx.x] gets the
// clock64 span of thread 0's loop.
template <int L>
__global__ void k_tmem_read(uint32_t iters, uint32_t *sink, long long *cycles) {
    __shared__ uint32_t tm;
    const uint32_t warp = threadIdx.x >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&tm))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t base = tm + (((warp & 3) * 32) << 16);
    uint32_t acc = 0;
    const long long t0 = clock64();
    for (uint32_t it = 0; it < iters; ++it) {
        uint32_t v[L][32];
#pragma unroll
        for (int l = 0; l < L; ++l) hw_tmem_ld32(base + (((it * L + l) * 32 + (warp >> 2) * 64) & 511), v[l]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int l = 0; l < L; ++l)
#pragma unroll
            for (int k = 0; k < 32; ++k) acc ^= v[l][k];
    }
    const long long t1 = clock64();
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tm) : "memory");
}

constexpr int TMEM_SMEM = 120 * 1024;  // one CTA per SM, so each may take all 512 columns

template <int L>
cudaError_t launch_tmem(uint32_t warps, uint32_t iters, uint32_t *sink, long long *cycles, int sms, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_tmem_read<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, TMEM_SMEM);
    if (e != cudaSuccess) return e;
    k_tmem_read<L><<<sms, warps * 32, TMEM_SMEM, s>>>(iters, sink, cycles);
    return cudaGetLastError();
}

}  // namespace
}  // namespace rgpu

using namespace rgpu;

extern "C" {

int rambo_probe_l2_atomics(void *buf, uint64_t words, uint32_t ops_per_thread, uint32_t blocks, void *stream) {
    if (!buf || words == 0 || (words & (words - 1)) || ops_per_thread == 0 || ops_per_thread > (1u << 16) ||
        blocks == 0 || blocks > (1u << 20) || (reinterpret_cast<uintptr_t>(buf) & 7))
        return RAMBO_EINVAL;
    k_l2_atomics<<<blocks, HW_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<unsigned long long *>(buf), words - 1, ops_per_thread);
    return cudaGetLastError() == cudaSuccess ? RAMBO_OK : RAMBO_ECUDA;
}

int rambo_probe_tmem_read(uint32_t warps, uint32_t loads_in_flight, uint32_t iters, uint32_t *sink,
                          long long *cycles, void *stream) {
    if ((warps != 4 && warps != 8 && warps != 16) || iters == 0 || iters > (1u << 24) || !sink || !cycles)
        return RAMBO_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RAMBO_ECUDA;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (loads_in_flight) {
        case 1: e = launch_tmem<1>(warps, iters, sink, cycles, sms, s); break;
        case 2: e = launch_tmem<2>(warps, iters, sink, cycles, sms, s); break;
        case 4: e = launch_tmem<4>(warps, iters, sink, cycles, sms, s); break;
        default: return RAMBO_EINVAL;
    }
    return e == cudaSuccess ? RAMBO_OK : RAMBO_ECUDA;
}

}  // extern "C"

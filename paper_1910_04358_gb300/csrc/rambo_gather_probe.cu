// rambo_gather_probe.cu -- random-record gather microbenchmark (measurement
// support, not part of the method).
//
// Reads n_probes records of record_bytes bytes at pseudo-random record
// indices of a device buffer, the access pattern of one index probe with no
// hashing or bit logic around it.  Its throughput is the practical ceiling
// for the probe kernels at a given record size, load instruction and L2
// fetch granularity.  The XOR of everything read goes to *sink so no load is
// dead.
#include "rambo.h"
#include "rambo_internal.cuh"

namespace rgpu {
namespace {

constexpr int GATHER_THREADS = 256;

template <int V>
__device__ __forceinline__ uint4 ld16(const uint4 *p) {
    uint4 v;
    if constexpr (V == 0) {
        asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
            : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    } else if constexpr (V == 1) {
        asm("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];"
            : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    } else if constexpr (V == 2) {
        asm("ld.global.v4.u32 {%0,%1,%2,%3}, [%4];"
            : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    } else if constexpr (V == 3) {
        asm("ld.global.nc.L2::64B.v4.u32 {%0,%1,%2,%3}, [%4];"
            : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    } else if constexpr (V == 4) {
        asm("ld.global.cs.v4.u32 {%0,%1,%2,%3}, [%4];"
            : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    } else {
        asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
            : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    }
    return v;
}

// LPR lanes read one record of 16*LPR bytes; U independent 16-byte loads per
// lane are in flight per iteration.
template <int LPR, int V, int U>
__global__ void __launch_bounds__(GATHER_THREADS) k_gather(const uint4 *buf, uint64_t n_records,
                                                           uint64_t n_probes, uint64_t seed,
                                                           unsigned long long *sink) {
    constexpr int RPW = 32 / LPR;  // records per warp instruction
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (uint64_t)blockIdx.x * (GATHER_THREADS / 32) + threadIdx.x / 32;
    const uint64_t nwarps = (uint64_t)gridDim.x * (GATHER_THREADS / 32);
    uint4 acc = make_uint4(0, 0, 0, 0);
    for (uint64_t base = warp * RPW * U; base < n_probes; base += nwarps * RPW * U) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t i = base + (uint64_t)u * RPW + lane / LPR;
            const uint64_t rec = fmix64(i ^ seed) % n_records;
            if (i < n_probes) v[u] = ld16<V>(buf + rec * LPR + (lane % LPR));
            else v[u] = make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            acc.x ^= v[u].x; acc.y ^= v[u].y; acc.z ^= v[u].z; acc.w ^= v[u].w;
        }
    }
    const unsigned long long x = ((unsigned long long)(acc.x ^ acc.z) << 32) | (acc.y ^ acc.w);
    if (x == 0x9e3779b97f4a7c15ULL) atomicXor(sink, x);  // practically never taken
}

template <int LPR, int U>
cudaError_t launch_gather_v(const void *buf, uint64_t n_records, uint64_t n_probes, uint32_t variant,
                            uint64_t seed, unsigned long long *sink, int blocks, cudaStream_t s) {
    const uint4 *b = static_cast<const uint4 *>(buf);
    switch (variant) {
        case 0: k_gather<LPR, 0, U><<<blocks, GATHER_THREADS, 0, s>>>(b, n_records, n_probes, seed, sink); break;
        case 1: k_gather<LPR, 1, U><<<blocks, GATHER_THREADS, 0, s>>>(b, n_records, n_probes, seed, sink); break;
        case 2: k_gather<LPR, 2, U><<<blocks, GATHER_THREADS, 0, s>>>(b, n_records, n_probes, seed, sink); break;
        case 3: k_gather<LPR, 3, U><<<blocks, GATHER_THREADS, 0, s>>>(b, n_records, n_probes, seed, sink); break;
        case 4: k_gather<LPR, 4, U><<<blocks, GATHER_THREADS, 0, s>>>(b, n_records, n_probes, seed, sink); break;
        default: k_gather<LPR, 5, U><<<blocks, GATHER_THREADS, 0, s>>>(b, n_records, n_probes, seed, sink); break;
    }
    return cudaGetLastError();
}

template <int LPR>
cudaError_t launch_gather_u(const void *buf, uint64_t n_records, uint64_t n_probes, uint32_t variant,
                            uint32_t unroll, uint64_t seed, unsigned long long *sink, int blocks,
                            cudaStream_t s) {
    if (unroll >= 32) return launch_gather_v<LPR, 32>(buf, n_records, n_probes, variant, seed, sink, blocks, s);
    if (unroll >= 16) return launch_gather_v<LPR, 16>(buf, n_records, n_probes, variant, seed, sink, blocks, s);
    if (unroll >= 8) return launch_gather_v<LPR, 8>(buf, n_records, n_probes, variant, seed, sink, blocks, s);
    return launch_gather_v<LPR, 4>(buf, n_records, n_probes, variant, seed, sink, blocks, s);
}

}  // namespace
}  // namespace rgpu

extern "C" int rambo_probe_gather(const void *buf, uint64_t buf_bytes, uint32_t record_bytes,
                                  uint64_t n_probes, uint32_t load_variant, uint32_t unroll,
                                  uint64_t seed, void *sink, void *stream) {
    using namespace rgpu;
    if (!buf || !sink || load_variant > 5) return RAMBO_EINVAL;
    if (record_bytes != 16 && record_bytes != 32 && record_bytes != 64 && record_bytes != 128 &&
        record_bytes != 256 && record_bytes != 512)
        return RAMBO_EINVAL;
    if ((reinterpret_cast<uintptr_t>(buf) & 15) || buf_bytes < record_bytes) return RAMBO_EINVAL;
    const uint64_t n_records = buf_bytes / record_bytes;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RAMBO_ECUDA;
    const int blocks = sms * 8;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto *sk = static_cast<unsigned long long *>(sink);
    cudaError_t e;
    switch (record_bytes) {
        case 16: e = launch_gather_u<1>(buf, n_records, n_probes, load_variant, unroll, seed, sk, blocks, s); break;
        case 32: e = launch_gather_u<2>(buf, n_records, n_probes, load_variant, unroll, seed, sk, blocks, s); break;
        case 64: e = launch_gather_u<4>(buf, n_records, n_probes, load_variant, unroll, seed, sk, blocks, s); break;
        case 128: e = launch_gather_u<8>(buf, n_records, n_probes, load_variant, unroll, seed, sk, blocks, s); break;
        case 256: e = launch_gather_u<16>(buf, n_records, n_probes, load_variant, unroll, seed, sk, blocks, s); break;
        default: e = launch_gather_u<32>(buf, n_records, n_probes, load_variant, unroll, seed, sk, blocks, s); break;
    }
    return e == cudaSuccess ? RAMBO_OK : RAMBO_ECUDA;
}

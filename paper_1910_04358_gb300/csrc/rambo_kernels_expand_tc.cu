// rambo_kernels_expand_tc.cu -- expansion of bucket masks on the tensor cores
// (Algorithm 2's union over the passing buckets of each repetition and the
// intersection over repetitions).
//
// Document d lies in exactly one bucket per repetition, bucket phi_r(d), so
// the number of repetitions whose union holds d is
//     count[q][d] = sum_i mask[q][i] * E[i][d],   i = r*B + b,
// with E[i][d] = 1 iff d was inserted and phi_r(d) = b (the bucket->document
// bitmaps, transposed), and d answers q iff count[q][d] = R.  That is a
// 0/1 matrix product: queries x (R*B) times (R*B) x documents.  Two more
// columns, A = 1 against E = -R and A = 1 against E = 1/2, make the result
// count - R + 1/2, whose sign bit is clear exactly for the answers.  It runs
// as tcgen05.mma kind::f8f6f4 (E4M3 operands: 0, 1, 1/2 and -R for R <= 15
// are exact; f32 accumulators in tensor memory, so every sum is exact),
// M = 128 queries by N = 256 documents by K = 32 columns per instruction.
//
// One CTA per SM (persistent over 128-query tiles, 8 warps, so that a CTA
// of the fused sequence query still fits beside it):
//   - E (all documents; R*B + 2 columns rounded up to 32) is staged once in
//     shared memory, K-major, in the canonical no-swizzle layout: core
//     matrices of 8 rows x 16 bytes, 8-row groups SBO bytes apart, 16-byte
//     column chunks LBO = 128 bytes apart;
//   - each tile's A (its 128 bucket masks, one byte per bit) is built by the
//     threads in the same layout, double-buffered: the next tile's masks are
//     loaded while the current tile drains;
//   - thread 0 issues the MMAs of 256-document chunks into two tensor-memory
//     buffers of 256 columns, two chunks ahead of the epilogue and across
//     tile boundaries; tcgen05.commit arrives on the buffer's mbarrier;
//   - the epilogue: warp w reads tensor-memory lanes 32*(w%4).. (its queries)
//     and 128 columns (half w/4 of the chunk), two tcgen05.ld in flight at a
//     time; each sign bit is shifted into the answer word with one funnel
//     shift per document, and the word is complemented.
// Every wait on an mbarrier is bounded: on expiry the kernel latches
// ERR_WAIT, waits (bounded) for its MMAs once more, frees its tensor memory
// and returns.
#include "rambo_query_common.cuh"

namespace rgpu {
namespace {

constexpr int TC_THREADS = 256;
constexpr uint32_t TC_M = 128;              // queries per tile (MMA M)
constexpr uint32_t TC_N = 256;              // documents per chunk (MMA N)
constexpr uint32_t TC_LBO = 128;            // bytes between 16-byte column chunks
constexpr uint32_t TC_TMEM_COLS = 512;      // two accumulator buffers of TC_N columns
constexpr size_t TC_SMEM_MIN = 120 * 1024;  // keeps one CTA (one TMEM owner) per SM
constexpr size_t TC_SMEM_MAX = 216 * 1024;  // leaves room for a fused-query CTA
constexpr uint64_t TC_WAIT_SPINS = 1ull << 22;  // try_wait rounds before giving up

constexpr uint32_t E4M3_ONE = 0x38u, E4M3_HALF = 0x30u;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start, leading and stride byte offsets
// (16-byte units), descriptor version 1, no swizzle, base offset 0.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3, both K-major,
// dense, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc_e4m3(uint32_t M, uint32_t N) {
    return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// E4M3 byte of -v for an integer 1 <= v <= 15 (exact: at most four
// significant bits; exponent bias 7, three mantissa bits).
__host__ __device__ constexpr uint32_t e4m3_neg_int(uint32_t v) {
    uint32_t e = 0;
    while ((v >> (e + 1)) != 0) ++e;
    return 0x80u | ((e + 7u) << 3) | ((((v - (1u << e)) << 3) >> e) & 7u);
}

// Four bits -> four bytes, each E4M3 1.0 or 0.
__device__ __forceinline__ uint32_t nib_to_e4m3(uint32_t v) {
    return ((v * 0x00204081u) & 0x01010101u) * E4M3_ONE;
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the given phase parity; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t spins = TC_WAIT_SPINS) {
    for (uint64_t i = 0; i < spins; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// A wait that nothing completes: one thread waits on a fresh mbarrier (no
// arrivals are ever made) with the kernels' bounded wait and latches ERR_WAIT
// when it gives up.  It exercises the timeout path of the tensor-core
// expansion without any fault or hang.
__global__ void k_wait_expiry(uint32_t *err, uint64_t spins) {
    __shared__ unsigned long long bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    if (!mbar_wait(b, 0, spins)) atomicOr(err, ERR_WAIT);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
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

struct TcShared {
    unsigned long long bar[2];
    uint32_t tmem;
    uint32_t abort;
};

// Mask chunk of A: 16 bucket bits of query q starting at column `bit`, the
// constant columns RB and RB + 1 set, everything past them clear.
__device__ __forceinline__ uint32_t a_bits(const ExpandArgs &a, uint32_t RB, uint64_t q, uint32_t bit) {
    uint32_t v = 0;
    if (q < a.n && bit < RB) v = (__ldg(a.acc + q * a.Gw + (bit >> 5)) >> (bit & 31)) & 0xFFFFu;
    if (bit + 16 > RB) {
        const uint32_t keep = RB > bit ? RB - bit : 0u;
        v &= keep >= 16 ? 0xFFFFu : ((1u << keep) - 1u);
        if (RB >= bit && RB < bit + 16) v |= 1u << (RB - bit);
        if (RB + 1 >= bit && RB + 1 < bit + 16) v |= 1u << (RB + 1 - bit);
    }
    return v;
}

__device__ __forceinline__ void a_store(uint8_t *sA, uint32_t sbo, uint32_t r, uint32_t c, uint32_t v) {
    *reinterpret_cast<uint4 *>(sA + (r >> 3) * sbo + c * TC_LBO + (r & 7) * 16) =
        make_uint4(nib_to_e4m3(v & 15u), nib_to_e4m3((v >> 4) & 15u), nib_to_e4m3((v >> 8) & 15u),
                   nib_to_e4m3(v >> 12));
}

// Work of one CTA: its tiles are blockIdx.x + i * gridDim.x, i < ntile; the
// MMA stream is the sequence of chunks g = i * nch + j, issued two ahead of
// the epilogue (across tile boundaries), TMEM buffer g & 1, A buffer i & 1.
// A(i + 1) is loaded into registers while chunk (i, 0) is waited for and
// drained, and written to its buffer before chunk (i + 1, 0) is issued.
__global__ void __launch_bounds__(TC_THREADS, 1) k_expand_tc(ExpandArgs a, uint32_t kdim, uint32_t nch) {
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    const uint32_t sbo = (kdim / 16) * 128;  // bytes between 8-row groups
    const uint32_t chunks = kdim / 16;       // 16-byte column chunks per row
    const size_t a_bytes = (size_t)TC_M * kdim;
    uint8_t *sA0 = tc_smem;                   // two A buffers of TC_M x kdim
    uint8_t *sE = tc_smem + 2 * a_bytes;      // nch*TC_N x kdim
    TcShared *sh = reinterpret_cast<TcShared *>(sE + (size_t)nch * TC_N * kdim);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t RB = a.R * a.B;
    const uint64_t tiles = (a.n + TC_M - 1) / TC_M;
    const uint64_t ntile = blockIdx.x < tiles ? (tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const uint64_t total = ntile * nch;
    constexpr uint32_t A_PER_THREAD = (TC_M * 256 / 16 + TC_THREADS - 1) / TC_THREADS;  // kdim <= 256

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sh->tmem)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh->bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh->bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh->abort = 0;
    }
    // E: row d (a document) holds bytes E[i][d]: 1 for its inserted buckets
    // (i < RB), -R at column RB and 1/2 at column RB + 1, else 0
    const uint32_t neg_r = e4m3_neg_int(a.R);
    for (uint32_t idx = tid; idx < nch * TC_N * chunks; idx += TC_THREADS) {
        const uint32_t d = idx / chunks, c = idx - d * chunks;
        const bool doc = d < a.K;
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t word = 0;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint32_t i = c * 16 + k * 4 + t;
                uint32_t byte = 0;
                if (i < RB) {
                    if (doc && ((__ldg(a.docbits + (uint64_t)i * a.W + (d >> 5)) >> (d & 31)) & 1u))
                        byte = E4M3_ONE;
                } else if (i == RB) {
                    byte = neg_r;
                } else if (i == RB + 1) {
                    byte = E4M3_HALF;
                }
                word |= byte << (8 * t);
            }
            w[k] = word;
        }
        *reinterpret_cast<uint4 *>(sE + (d >> 3) * sbo + c * TC_LBO + (d & 7) * 16) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
    // A of this CTA's first tile
    if (ntile > 0) {
        const uint64_t q0 = (uint64_t)blockIdx.x * TC_M;
        for (uint32_t idx = tid; idx < TC_M * chunks; idx += TC_THREADS) {
            const uint32_t r = idx / chunks, c = idx - r * chunks;
            a_store(sA0, sbo, r, c, a_bits(a, RB, q0 + r, c * 16));
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sh->tmem;
    const uint32_t sA_u = smem_u32(sA0), sE_u = smem_u32(sE);
    const uint32_t bar0 = smem_u32(&sh->bar[0]), bar1 = smem_u32(&sh->bar[1]);
    constexpr uint32_t IDESC = idesc_e4m3(TC_M, TC_N);
    const uint32_t ksteps = kdim / 32;
    uint32_t par0 = 0, par1 = 0;  // thread 0: phase parity each buffer's mbarrier completes next
    bool aborted = false;

    auto issue = [&](uint64_t g) {  // chunk g of this CTA's stream (thread 0)
        const uint64_t i = g / nch;
        const uint32_t j = (uint32_t)(g - i * nch);
        const uint32_t dcol = tmem + (uint32_t)(g & 1) * TC_N;
        const uint32_t ab = sA_u + (uint32_t)(i & 1) * (uint32_t)a_bytes;
        const uint32_t eb = sE_u + j * (TC_N / 8) * sbo;
        for (uint32_t s = 0; s < ksteps; ++s)
            tc_mma(dcol, umma_desc(ab + s * 2 * TC_LBO, TC_LBO, sbo), umma_desc(eb + s * 2 * TC_LBO, TC_LBO, sbo),
                   IDESC, s > 0);
        tc_commit((g & 1) ? bar1 : bar0);
    };
    if (tid == 0) {
        if (total > 0) issue(0);
        if (total > 1) issue(1);
    }

    for (uint64_t g = 0; g < total; ++g) {
        const uint64_t i = g / nch;
        const uint32_t j = (uint32_t)(g - i * nch);
        const uint64_t q0 = ((uint64_t)blockIdx.x + i * gridDim.x) * TC_M;
        const uint64_t q1 = q0 + (uint64_t)gridDim.x * TC_M;  // the next tile's first query
        const bool next_tile = i + 1 < ntile;
        // the next tile's mask chunks, loaded now so their latency overlaps this chunk's drain
        uint32_t pre[A_PER_THREAD];
        if (j == 0 && next_tile) {
#pragma unroll
            for (uint32_t u = 0; u < A_PER_THREAD; ++u) {
                const uint32_t idx = tid + u * TC_THREADS;
                pre[u] = 0;
                if (idx < TC_M * chunks) {
                    const uint32_t r = idx / chunks, c = idx - r * chunks;
                    pre[u] = a_bits(a, RB, q1 + r, c * 16);
                }
            }
        }
        const uint32_t b = (uint32_t)(g & 1);
        if (tid == 0) {  // only thread 0 waits and tracks the parities
            if (mbar_wait(b ? bar1 : bar0, b ? par1 : par0)) {
                if (b) par1 ^= 1u;
                else par0 ^= 1u;
            } else {
                sh->abort = 1;
                atomicOr(a.err, ERR_WAIT);
            }
        }
        __syncthreads();
        if (sh->abort) {
            aborted = true;
            break;
        }
        fence_after();
        // epilogue: warp w reads its 32 lanes (queries) and 128 columns (half
        // w/4) of the chunk, 64 at a time; a clear sign bit is an answer
        {
            const uint32_t quad = warp & 3, half = warp >> 2;
            const uint64_t q = q0 + quad * 32 + lane;
#pragma unroll 1
            for (uint32_t p = 0; p < 2; ++p) {
                const uint32_t col = tmem + ((quad * 32) << 16) + b * TC_N + half * 128 + p * 64;
                uint32_t v0[32], v1[32];
                tmem_ld32(col, v0);
                tmem_ld32(col + 32, v1);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                uint32_t w0 = 0, w1 = 0;
#pragma unroll
                for (int k = 31; k >= 0; --k) {
                    w0 = __funnelshift_l(v0[k], w0, 1);
                    w1 = __funnelshift_l(v1[k], w1, 1);
                }
                const uint32_t word = j * (TC_N / 32) + half * 4 + p * 2;
                if (q < a.n) {
                    uint32_t *o = a.out + q * a.W + word;
                    if (word < a.W) o[0] = ~w0;
                    if (word + 1 < a.W) o[1] = ~w1;
                }
            }
        }
        if (j == 0 && next_tile) {
            // A(i + 1) into the other buffer: its last reader, tile i - 1, is done
            uint8_t *dst = sA0 + ((i + 1) & 1) * a_bytes;
#pragma unroll
            for (uint32_t u = 0; u < A_PER_THREAD; ++u) {
                const uint32_t idx = tid + u * TC_THREADS;
                if (idx < TC_M * chunks) {
                    const uint32_t r = idx / chunks, c = idx - r * chunks;
                    a_store(dst, sbo, r, c, pre[u]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        fence_before();
        __syncthreads();
        if (tid == 0 && g + 2 < total) {
            fence_after();
            issue(g + 2);
        }
    }
    if (aborted && tid == 0) {
        // MMAs may still be in flight: give each buffer one more bounded wait
        // for the phase it was last committed to
        mbar_wait(bar0, par0);
        mbar_wait(bar1, par1);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
}

uint32_t tc_kdim(const ExpandArgs &a) { return (a.R * a.B + 2 + 31) / 32 * 32; }
// Document chunks, at least two (the MMA stream runs two chunks ahead and
// must not reach past the next tile).
uint32_t tc_chunks(const ExpandArgs &a) {
    const uint32_t c = (a.K + TC_N - 1) / TC_N;
    return c < 2 ? 2 : c;
}

}  // namespace

// Shared memory of the tensor-core expansion, 0 when it does not apply.
size_t expand_tc_smem(const ExpandArgs &a) {
    const uint32_t rb = a.R * a.B;
    if (rb == 0 || rb + 2 > 256 || a.K == 0 || a.R > 15) return 0;
    const uint32_t kdim = tc_kdim(a);
    const uint32_t nch = tc_chunks(a);
    const size_t bytes = 2 * (size_t)TC_M * kdim + (size_t)nch * TC_N * kdim + sizeof(TcShared);
    if (bytes > TC_SMEM_MAX) return 0;
    return bytes < TC_SMEM_MIN ? TC_SMEM_MIN : bytes;
}

cudaError_t launch_wait_expiry(uint32_t *err, uint64_t spins, cudaStream_t s) {
    k_wait_expiry<<<1, 32, 0, s>>>(err, spins);
    return cudaGetLastError();
}

cudaError_t launch_expand_tc(const ExpandArgs &a, int sm_count, cudaStream_t s) {
    const size_t smem = expand_tc_smem(a);
    if (!smem || !a.err) return cudaErrorInvalidValue;
    const uint32_t kdim = tc_kdim(a);
    const uint32_t nch = tc_chunks(a);
    cudaError_t e = cudaFuncSetAttribute(k_expand_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uint64_t tiles = (a.n + TC_M - 1) / TC_M;
    const int grid = tiles < (uint64_t)sm_count ? (int)tiles : sm_count;
    k_expand_tc<<<grid, TC_THREADS, smem, s>>>(a, kdim, nch);
    return cudaGetLastError();
}

}  // namespace rgpu

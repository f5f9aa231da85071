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
// One persistent CTA per SM over 128-query tiles, warp-specialised:
//   - E (all documents; R*B + 2 columns rounded up to 32) is staged once in
//     shared memory by every thread, K-major, in the canonical no-swizzle
//     layout: core matrices of 8 rows x 16 bytes, 8-row groups SBO bytes
//     apart, 16-byte column chunks LBO = 128 bytes apart;
//   - 4 producer warps (one thread per query row) build each tile's A (its
//     128 bucket masks, one byte per bit, same layout) into one of two
//     buffers, loading the next tile's masks while they wait for a buffer;
//   - one thread of the MMA warp issues, per 256-document chunk, the K/32
//     MMAs into one of two tensor-memory buffers of 256 columns and commits
//     them to that buffer's "full" mbarrier; after a tile's last chunk it
//     commits the A buffer's "empty" mbarrier;
//   - 8 epilogue warps drain a full buffer: warp w reads tensor-memory
//     lanes 32*(w%4).. (its queries) and 128 columns (part w/4 of the chunk),
//     releases the buffer as soon as its loads have landed, shifts each sign
//     bit into the answer word (one funnel shift per document) and stores the
//     complemented words.
// The roles meet only on mbarriers (full/empty pairs for A and for tensor
// memory).  Every wait is bounded: on expiry the waiter latches ERR_WAIT and
// raises a shared abort flag that every other wait polls, all roles leave
// their loops, the MMA thread waits (bounded) for its MMAs to finish, and
// the tensor memory is freed before the kernel returns.
#include "rambo_query_common.cuh"

namespace rgpu {
namespace {

constexpr uint32_t TC_EPI_WARPS = 8;                       // tensor memory -> answers
constexpr uint32_t TC_PROD_WARPS = 4;                      // bucket masks -> A tiles
constexpr uint32_t TC_MMA_WARP = TC_EPI_WARPS + TC_PROD_WARPS;
constexpr int TC_THREADS = 32 * (TC_MMA_WARP + 1);         // 416
constexpr uint32_t TC_PROD_THREADS = 32 * TC_PROD_WARPS;
constexpr uint32_t TC_EPI_THREADS = 32 * TC_EPI_WARPS;
constexpr uint32_t TC_M = 128;              // queries per tile (MMA M)
constexpr uint32_t TC_N = 256;              // documents per chunk (MMA N)
constexpr uint32_t TC_NBUF = 2;             // tensor-memory accumulator buffers of TC_N columns
constexpr uint32_t TC_LBO = 128;            // bytes between 16-byte column chunks
constexpr uint32_t TC_TMEM_COLS = TC_NBUF * TC_N;  // all 512 columns
constexpr size_t TC_SMEM_MIN = 120 * 1024;  // keeps one CTA (one TMEM owner) per SM
constexpr size_t TC_SMEM_MAX = 216 * 1024;  // leaves room for a fused-query CTA
constexpr uint64_t TC_WAIT_SPINS = 1ull << 22;  // suspending try_wait rounds before giving up
constexpr uint64_t TC_POLL_SPINS = 1ull << 26;  // non-suspending polls before giving up (about a second)

constexpr uint32_t TC_EPI_PARTS = TC_EPI_WARPS / 4;         // column parts of a chunk (per lane quadrant)
constexpr uint32_t TC_EPI_COLS = TC_N / TC_EPI_PARTS;         // columns per epilogue warp and chunk
static_assert(TC_PROD_THREADS == TC_M, "one producer thread per row of an A tile");
static_assert(TC_EPI_WARPS % 4 == 0 && TC_EPI_COLS % 64 == 0, "whole lane quadrants, 64-column passes");

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
    unsigned long long a_full[2];   // producers -> MMA: A buffer written (TC_PROD_THREADS arrivals)
    unsigned long long a_empty[2];  // MMA -> producers: the tile's MMAs read it (commit)
    unsigned long long t_full[TC_NBUF];   // MMA -> epilogue: chunk accumulated (commit)
    unsigned long long t_empty[TC_NBUF];  // epilogue -> MMA: chunk read out (TC_EPI_THREADS arrivals)
    unsigned long long done;        // MMA thread: every MMA it issued has finished (commit)
    uint32_t tmem;
    uint32_t abort;
};

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Non-suspending test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait of one role, polling without suspending the warp (each
// hand-off is on the critical path of a two-deep pipeline): false when the
// abort flag is raised (polled every 64 rounds) or when this wait runs out
// after `spins` polls, which raises the flag and latches ERR_WAIT.
__device__ __forceinline__ bool role_wait(uint32_t bar, uint32_t parity, volatile uint32_t *abort,
                                          uint32_t *err, uint64_t spins = TC_POLL_SPINS) {
    for (uint64_t i = 0;; ++i) {
        if (mbar_test_wait(bar, parity)) return true;
        if ((i & 63) == 63 && *abort) return false;
        if (i >= spins) {
            *abort = 1;
            atomicOr(err, ERR_WAIT);
            return false;
        }
    }
}

// A wait that nothing completes: one thread waits on a fresh mbarrier (no
// arrivals are ever made) with the roles' bounded polling wait, which runs
// out after `spins` polls and latches ERR_WAIT.  It exercises the timeout
// path of the tensor-core expansion without any fault or hang.
__global__ void k_wait_expiry(uint32_t *err, uint64_t spins) {
    __shared__ unsigned long long bar;
    __shared__ uint32_t abort;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    abort = 0;
    mbar_init(b, 1);
    role_wait(b, 0, &abort, err, spins);
}

// Chunk of A at column `bit` (a multiple of 16) from the 16 mask bits v found
// there: the constant columns RB and RB + 1 set, everything past them clear.
__device__ __forceinline__ uint32_t a_chunk(uint32_t v, uint32_t RB, uint32_t bit) {
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

// Four bytes of E for one document: byte t is 1 iff bit `d` of w[t] is set.
__device__ __forceinline__ uint32_t e_word(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t d) {
    const uint32_t v = ((w0 >> d) & 1u) | (((w1 >> d) & 1u) << 8) | (((w2 >> d) & 1u) << 16) |
                       (((w3 >> d) & 1u) << 24);
    return v * E4M3_ONE;
}

// n consecutive answer words of one query at word `word` of W: one vector
// store when they fit and are aligned, else word by word.
template <uint32_t N>
__device__ __forceinline__ void store_words(uint32_t *o, const uint32_t (&w)[N], uint32_t word, uint32_t W) {
    static_assert(N == 2 || N == 4, "two or four words");
    if (word + N <= W && (reinterpret_cast<uintptr_t>(o) & (4 * N - 1)) == 0) {
        if constexpr (N == 4) *reinterpret_cast<uint4 *>(o) = make_uint4(w[0], w[1], w[2], w[3]);
        else *reinterpret_cast<uint2 *>(o) = make_uint2(w[0], w[1]);
    } else {
#pragma unroll
        for (uint32_t k = 0; k < N; ++k)
            if (word + k < W) o[k] = w[k];
    }
}

// Work of one CTA: its tiles are blockIdx.x + i * gridDim.x, i < ntile;
// chunk g = i * nch + j of its stream uses A buffer i & 1 and tensor-memory
// buffer g % 2.  A buffer b is filled for the (i >> 1)-th time by tile i, so
// its "full" phase is (i >> 1) & 1 and the producers wait for the "empty"
// phase before it (a fresh mbarrier has completed the phase of parity 1);
// the same holds for the tensor-memory buffers with g / 2.
__global__ void __launch_bounds__(TC_THREADS, 1) k_expand_tc(ExpandArgs a, uint32_t kdim, uint32_t nch) {
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    const uint32_t sbo = (kdim / 16) * 128;  // bytes between 8-row groups
    const uint32_t chunks = kdim / 16;       // 16-byte column chunks per row
    const size_t a_bytes = (size_t)TC_M * kdim;
    uint8_t *sA0 = tc_smem;                   // two A buffers of TC_M x kdim
    uint8_t *sE = tc_smem + 2 * a_bytes;      // nch*TC_N x kdim
    TcShared *sh = reinterpret_cast<TcShared *>(sE + (size_t)nch * TC_N * kdim);
    volatile uint32_t *abort = &sh->abort;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t RB = a.R * a.B;
    const uint64_t tiles = (a.n + TC_M - 1) / TC_M;
    const uint64_t ntile = blockIdx.x < tiles ? (tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const uint64_t total = ntile * nch;

    if (warp == TC_MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sh->tmem)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&sh->a_full[b]), TC_PROD_THREADS);
            mbar_init(smem_u32(&sh->a_empty[b]), 1);
        }
        for (uint32_t b = 0; b < TC_NBUF; ++b) {
            mbar_init(smem_u32(&sh->t_full[b]), 1);
            mbar_init(smem_u32(&sh->t_empty[b]), TC_EPI_THREADS);
        }
        mbar_init(smem_u32(&sh->done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh->abort = 0;
    }
    // E: row d (a document) holds bytes E[i][d]: 1 for its inserted buckets
    // (i < RB), -R at column RB and 1/2 at column RB + 1, else 0.  One item is
    // (16-column chunk c, 32-document word dw, half h): 16 bitmap words read
    // once, 16 document rows written.
    {
        const uint32_t neg_r = e4m3_neg_int(a.R);
        const uint32_t dwords = nch * TC_N / 32;
        for (uint32_t it = tid; it < chunks * dwords * 2; it += TC_THREADS) {
            const uint32_t c = it / (dwords * 2), rem = it - c * dwords * 2, dw = rem >> 1, h = rem & 1;
            uint32_t w[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const uint32_t i = c * 16 + t;
                w[t] = (i < RB && dw < a.W) ? __ldg(a.docbits + (uint64_t)i * a.W + dw) : 0u;
            }
            uint32_t bias[4];  // the constant columns, where they fall in this chunk
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                const uint32_t lo = c * 16 + 4 * k;
                bias[k] = (RB >= lo && RB < lo + 4 ? neg_r << (8 * (RB - lo)) : 0u) |
                          (RB + 1 >= lo && RB + 1 < lo + 4 ? E4M3_HALF << (8 * (RB + 1 - lo)) : 0u);
            }
#pragma unroll 4
            for (uint32_t dd = h * 16; dd < h * 16 + 16; ++dd) {
                const uint32_t d = dw * 32 + dd;
                uint4 v = make_uint4(bias[0], bias[1], bias[2], bias[3]);
                if (d < a.K) {
                    v.x |= e_word(w[0], w[1], w[2], w[3], dd);
                    v.y |= e_word(w[4], w[5], w[6], w[7], dd);
                    v.z |= e_word(w[8], w[9], w[10], w[11], dd);
                    v.w |= e_word(w[12], w[13], w[14], w[15], dd);
                }
                *reinterpret_cast<uint4 *>(sE + (d >> 3) * sbo + c * TC_LBO + (d & 7) * 16) = v;
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = sh->tmem;

    if (warp < TC_EPI_WARPS) {
        // epilogue: warp w reads its 32 lanes (queries) and TC_EPI_COLS
        // columns (part w/4) of each chunk, 64 at a time (two loads in
        // flight), releases the buffer once the last loads have landed, and
        // turns the sign bits into TC_EPI_COLS/32 answer words
        constexpr uint32_t PASSES = TC_EPI_COLS / 64;
        const uint32_t quad = warp & 3, part = warp >> 2;
        for (uint64_t g = 0; g < total; ++g) {
            const uint64_t i = g / nch;
            const uint32_t j = (uint32_t)(g - i * nch), b = (uint32_t)(g % TC_NBUF);
            const bool ok =
                role_wait(smem_u32(&sh->t_full[b]), (uint32_t)(g / TC_NBUF) & 1u, abort, a.err);
            if (!__all_sync(0xFFFFFFFFu, ok)) break;
            fence_after();
            const uint32_t col = tmem + ((quad * 32) << 16) + b * TC_N + part * TC_EPI_COLS;
            uint32_t out[2 * PASSES];
#pragma unroll
            for (uint32_t p = 0; p < PASSES; ++p) {
                uint32_t v0[32], v1[32];
                tmem_ld32(col + p * 64, v0);
                tmem_ld32(col + p * 64 + 32, v1);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (p == PASSES - 1) {  // every column of this buffer is in registers
                    fence_before();
                    mbar_arrive(smem_u32(&sh->t_empty[b]));
                }
                uint32_t w0 = 0, w1 = 0;
#pragma unroll
                for (int k = 31; k >= 0; --k) {
                    w0 = __funnelshift_l(v0[k], w0, 1);
                    w1 = __funnelshift_l(v1[k], w1, 1);
                }
                out[2 * p] = ~w0;
                out[2 * p + 1] = ~w1;
            }
            const uint64_t q = ((uint64_t)blockIdx.x + i * gridDim.x) * TC_M + quad * 32 + lane;
            const uint32_t word = j * (TC_N / 32) + part * (2 * PASSES);
            if (q < a.n) store_words<2 * PASSES>(a.out + q * a.W + word, out, word, a.W);
        }
    } else if (warp < TC_MMA_WARP) {
        // producers: thread t builds row t of every A tile from its query's
        // mask words (Gw <= 8 since R*B + 2 <= 256), the next tile's words
        // loaded while the buffer they go to is still being read; a warp's
        // stores cover whole core matrices (no bank conflicts)
        const uint32_t r = tid - TC_EPI_THREADS;
        uint32_t wv[8];
        auto load = [&](uint64_t i) {
            const uint64_t q = ((uint64_t)blockIdx.x + i * gridDim.x) * TC_M + r;
#pragma unroll
            for (uint32_t k = 0; k < 8; ++k)
                wv[k] = (q < a.n && k < a.Gw) ? __ldg(a.acc + q * a.Gw + k) : 0u;
        };
        if (ntile > 0) load(0);
        for (uint64_t i = 0; i < ntile; ++i) {
            const uint32_t b = (uint32_t)(i & 1);
            const bool ok = role_wait(smem_u32(&sh->a_empty[b]), ((uint32_t)(i >> 1) & 1u) ^ 1u, abort, a.err);
            if (!__all_sync(0xFFFFFFFFu, ok)) break;
            uint8_t *dst = sA0 + b * a_bytes;
#pragma unroll
            for (uint32_t c = 0; c < 16; ++c)
                if (c < chunks)
                    a_store(dst, sbo, r, c, a_chunk((wv[c >> 1] >> ((c & 1) * 16)) & 0xFFFFu, RB, c * 16));
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&sh->a_full[b]));
            if (i + 1 < ntile) load(i + 1);
        }
    } else if (lane == 0) {
        // MMA issuer
        const uint32_t sA_u = smem_u32(sA0), sE_u = smem_u32(sE);
        constexpr uint32_t IDESC = idesc_e4m3(TC_M, TC_N);
        const uint32_t ksteps = kdim / 32;
        uint64_t g = 0;
        bool stop = false;
        for (uint64_t i = 0; i < ntile && !stop; ++i) {
            const uint32_t ab = (uint32_t)(i & 1);
            if (!role_wait(smem_u32(&sh->a_full[ab]), (uint32_t)(i >> 1) & 1u, abort, a.err)) break;
            fence_after();
            const uint64_t adesc = umma_desc(sA_u + ab * (uint32_t)a_bytes, TC_LBO, sbo);
            for (uint32_t j = 0; j < nch; ++j, ++g) {
                const uint32_t b = (uint32_t)(g % TC_NBUF);
                if (!role_wait(smem_u32(&sh->t_empty[b]), ((uint32_t)(g / TC_NBUF) & 1u) ^ 1u, abort, a.err)) {
                    stop = true;
                    break;
                }
                fence_after();
                const uint32_t dcol = tmem + b * TC_N;
                const uint64_t edesc = umma_desc(sE_u + j * (TC_N / 8) * sbo, TC_LBO, sbo);
                // consecutive K steps are 2 * TC_LBO bytes apart: 16 in the
                // descriptor's start-address field (16-byte units)
                for (uint32_t s = 0; s < ksteps; ++s)
                    tc_mma(dcol, adesc + s * (2 * TC_LBO / 16), edesc + s * (2 * TC_LBO / 16), IDESC, s > 0);
                tc_commit(smem_u32(&sh->t_full[b]));
            }
            if (!stop) tc_commit(smem_u32(&sh->a_empty[ab]));
        }
        // every MMA issued above has finished before the tensor memory is freed
        tc_commit(smem_u32(&sh->done));
        if (!mbar_wait(smem_u32(&sh->done), 0)) {
            *abort = 1;
            atomicOr(a.err, ERR_WAIT);
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == TC_MMA_WARP)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
}

uint32_t tc_kdim(const ExpandArgs &a) { return (a.R * a.B + 2 + 31) / 32 * 32; }
// 256-document chunks covering every document.
uint32_t tc_chunks(const ExpandArgs &a) { return (a.K + TC_N - 1) / TC_N; }

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

// rambo_query_common.cuh -- device helpers shared by the query kernels
// (probe, expansion, persistent fused path); included by each of their
// translation units, never by host-only code.
#pragma once

#include "rambo_internal.cuh"

namespace rgpu {
namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr uint32_t NONE = 0xffffffffu;
constexpr int PROBE_THREADS = 256;

__device__ __forceinline__ uint32_t reduce_pos(uint64_t h, uint64_t m, uint32_t m_pow2) {
    return (uint32_t)(m_pow2 ? (h & (m - 1)) : (h % m));
}

// 16-byte copy from global to shared memory that does not pass through
// registers (caching in L2 only), and the wait for this thread's copies.
__device__ __forceinline__ void cp_async16(uint4 *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Largest q in [0, n) with kcum[q] <= g, given kcum[0] <= g < kcum[n].
__device__ __forceinline__ uint64_t find_query(const uint64_t *kcum, uint64_t n, uint64_t g) {
    uint64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        uint64_t mid = (lo + hi) >> 1;
        if (kcum[mid] <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int SW>
__device__ __forceinline__ void slice_ones(Slice<SW> &s) {
#pragma unroll
    for (int w = 0; w < SW; ++w) s.w[w] = FULL;
}

template <int SW>
__device__ __forceinline__ void slice_and(Slice<SW> &a, const Slice<SW> &b) {
#pragma unroll
    for (int w = 0; w < SW; ++w) a.w[w] &= b.w[w];
}

// atomicAnd of one lane's slice into a query's bucket mask (all-ones words
// change nothing and are skipped).
template <int SW>
__device__ __forceinline__ void flush_slice(uint32_t *acc, uint64_t q, uint32_t Gw, uint32_t word0,
                                            const Slice<SW> &v) {
    uint32_t *p = acc + q * Gw + word0;
#pragma unroll
    for (int w = 0; w < SW; ++w)
        if (v.w[w] != FULL) atomicAnd(p + w, v.w[w]);
}

// Per-warp contiguous range of the flattened k-mer index space [0, T).
template <int STEP>
__device__ __forceinline__ void warp_range(uint64_t T, uint32_t min_chunk, uint64_t &c0, uint64_t &c1) {
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    uint64_t per = (T + nwarps - 1) / nwarps;
    if (per < min_chunk) per = min_chunk;
    per = (per + STEP - 1) / STEP * STEP;
    if (per < 2 * STEP) per = 2 * STEP;
    c0 = warp * per;
    c1 = c0 + per < T ? c0 + per : T;
}

// ---------------------------------------------------------------------------
// expand.  Work unit = (query, chunk of 32*C output words); one warp per unit
// (grid-stride), no block barriers.  For repetition r the bucket row is bits
// [r*B, r*B+B) of the query's bucket mask, read as ceil(B/8) bytes.  The
// union of the passing buckets' document bitmaps is built byte by byte:
//  - with the byte table (the precomputed OR of DocBits over every 8-bucket
//    pattern), every nonzero byte costs exactly one table row; the lanes
//    first extract the bytes of 16/C (repetition, byte) pairs in parallel,
//    then every lane issues all of those row loads before consuming any, so
//    a query's loads are in flight together instead of one L2 round trip each;
//  - without the table, each set bit costs one DocBits row.
// The answer is the AND of the R unions; a repetition with no passing bucket,
// or an all-zero running AND, ends the unit early.
constexpr int EXPAND_THREADS = 256;
constexpr size_t SMEM_DOCBITS_MAX = 96 * 1024;

// Byte j of repetition r's bucket row (buckets 8j .. 8j+7), masked to B.
// (bm may point to global or shared memory.)
__device__ __forceinline__ uint32_t row_byte(const uint32_t *bm, uint32_t Gw, uint32_t B, uint32_t r,
                                             uint32_t j) {
    const uint32_t bit = r * B + 8 * j;
    uint64_t two = bm[bit >> 5];
    if ((bit & 31) > 24 && (bit >> 5) + 1 < Gw) two |= (uint64_t)bm[(bit >> 5) + 1] << 32;
    const uint32_t nb = B - 8 * j < 8 ? B - 8 * j : 8;
    return (uint32_t)(two >> (bit & 31)) & ((1u << nb) - 1u);
}

template <int C>
__device__ __forceinline__ void expand_unit_table(const ExpandArgs &a, const uint32_t *bm, uint64_t q,
                                                  uint32_t w0, int lane) {
    constexpr int PB = 16 / C;  // (repetition, byte) pairs per batch
    const uint32_t NJ = (a.B + 7) / 8;
    const uint32_t NP = a.R * NJ;
    uint32_t res[C], o[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        res[c] = FULL;
        o[c] = 0;
    }
    bool row_any = false, dead = false;
    uint32_t j0 = 0;  // byte index (within its repetition) of pair p0
    for (uint32_t p0 = 0; p0 < NP && !dead; p0 += PB) {
        uint32_t mine = 0;
        if (lane < PB && p0 + lane < NP) {
            const uint32_t p = p0 + lane;
            const uint32_t r = p / NJ;
            mine = row_byte(bm, a.Gw, a.B, r, p - r * NJ);
        }
        uint32_t v[PB];
        uint32_t val[PB][C];
#pragma unroll
        for (int t = 0; t < PB; ++t) {
            v[t] = __shfl_sync(FULL, mine, t);
            const uint32_t p = p0 + t;
            const uint32_t *row = a.tab + ((uint64_t)p * 256 + v[t]) * a.W;  // p = r*NJ + j
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const uint32_t w = w0 + 32 * c;
                val[t][c] = (v[t] && w < a.W) ? __ldg(row + w) : 0u;
            }
        }
#pragma unroll
        for (int t = 0; t < PB; ++t) {
            const uint32_t p = p0 + t;
            if (p >= NP) break;
#pragma unroll
            for (int c = 0; c < C; ++c) o[c] |= val[t][c];
            row_any |= v[t] != 0;
            if (j0 == NJ - 1) {  // repetition complete
                if (!row_any) dead = true;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    res[c] &= o[c];
                    o[c] = 0;
                }
                row_any = false;
                j0 = 0;
            } else {
                ++j0;
            }
        }
        uint32_t nz = 0;
#pragma unroll
        for (int c = 0; c < C; ++c) nz |= res[c];
        if (!__any_sync(FULL, nz)) dead = true;
    }
    uint32_t *out = a.out + q * a.W;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const uint32_t w = w0 + 32 * c;
        if (w < a.W) out[w] = dead ? 0u : res[c];
    }
}

template <int C>
__device__ __forceinline__ void expand_unit_sparse(const ExpandArgs &a, const uint32_t *bm, uint64_t q,
                                                   uint32_t w0) {
    const uint32_t NJ = (a.B + 7) / 8;
    uint32_t res[C];
#pragma unroll
    for (int c = 0; c < C; ++c) res[c] = FULL;
    bool dead = false;
    for (uint32_t r = 0; r < a.R && !dead; ++r) {
        uint32_t o[C];
#pragma unroll
        for (int c = 0; c < C; ++c) o[c] = 0;
        bool any = false;
        for (uint32_t j = 0; j < NJ; ++j) {
            const uint32_t v = row_byte(bm, a.Gw, a.B, r, j);
            if (!v) continue;
            any = true;
            // the rows of the byte's set bits, all loads issued before any is used
            const uint32_t *row0 = a.docbits + (uint64_t)(r * a.B + 8 * j) * a.W;
            uint32_t val[8][C];
#pragma unroll
            for (int t = 0; t < 8; ++t)
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t w = w0 + 32 * c;
                    val[t][c] = ((v >> t) & 1u) && w < a.W ? __ldg(row0 + (uint64_t)t * a.W + w) : 0u;
                }
#pragma unroll
            for (int t = 0; t < 8; ++t)
#pragma unroll
                for (int c = 0; c < C; ++c) o[c] |= val[t][c];
        }
        uint32_t nz = 0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            res[c] &= o[c];
            nz |= res[c];
        }
        if (!any || !__any_sync(FULL, nz)) dead = true;
    }
    uint32_t *out = a.out + q * a.W;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const uint32_t w = w0 + 32 * c;
        if (w < a.W) out[w] = dead ? 0u : res[c];
    }
}

// Union per repetition from DocBits staged in shared memory (sdb): each set
// bit of the bucket row, taken 32 buckets at a time, ORs one row of W words
// (consecutive words per lane: no bank conflicts).
template <int C>
__device__ __forceinline__ void expand_unit_smem(const ExpandArgs &a, const uint32_t *sdb,
                                                 const uint32_t *bm, uint64_t q, uint32_t w0) {
    uint32_t res[C];
#pragma unroll
    for (int c = 0; c < C; ++c) res[c] = FULL;
    bool dead = false;
    for (uint32_t r = 0; r < a.R && !dead; ++r) {
        uint32_t o[C];
#pragma unroll
        for (int c = 0; c < C; ++c) o[c] = 0;
        bool any = false;
        const uint32_t lo = r * a.B;
        for (uint32_t i = 0; i < a.B; i += 32) {
            const uint32_t bit = lo + i;
            const uint32_t wi = bit >> 5, sh = bit & 31;
            uint32_t x = bm[wi];
            if (sh) x = __funnelshift_r(x, wi + 1 < a.Gw ? bm[wi + 1] : 0u, sh);
            const uint32_t nb = a.B - i < 32 ? a.B - i : 32;
            if (nb < 32) x &= (1u << nb) - 1u;
            any |= x != 0;
            while (x) {
                const uint32_t b = i + __ffs(x) - 1;
                x &= x - 1;
                const uint32_t *row = sdb + (lo + b) * a.W;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t w = w0 + 32 * c;
                    if (w < a.W) o[c] |= row[w];
                }
            }
        }
        uint32_t nz = 0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            res[c] &= o[c];
            nz |= res[c];
        }
        if (!any || !__any_sync(FULL, nz)) dead = true;
    }
    uint32_t *out = a.out + q * a.W;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const uint32_t w = w0 + 32 * c;
        if (w < a.W) out[w] = dead ? 0u : res[c];
    }
}

// One expansion unit: query q's answer words w0, w0+32, .. w0+32*(C-1) from
// its bucket mask bm.
template <int C>
__device__ __forceinline__ void expand_one(const ExpandArgs &a, const uint32_t *bm, uint64_t q,
                                           uint32_t w0, int lane) {
    if (a.tab) expand_unit_table<C>(a, bm, q, w0, lane);
    else expand_unit_sparse<C>(a, bm, q, w0);
}

// Passing buckets of one query, decoded once for all of its answer chunks
// (Algorithm 2's union needs only the buckets whose bit survived): the warp
// writes the indices i = r*B + b of the set bits of bm (bits past R*B
// ignored) in increasing order into `list` (EXPAND_LIST_MAX words of the
// warp's shared memory) and returns how many there are, or
// EXPAND_LIST_MAX + 1 when more pass (the caller then scans the mask per
// chunk).  *dead is set when some repetition has no passing bucket: the
// answer is then empty.
constexpr uint32_t EXPAND_LIST_MAX = 32;

__device__ __forceinline__ uint32_t bucket_list(const uint32_t *bm, uint32_t R, uint32_t B, uint32_t *list,
                                                int lane, bool *dead) {
    const uint32_t RB = R * B;
    const uint32_t nw = (RB + 31) / 32;
    uint32_t total = 0;
    for (uint32_t base = 0; base < nw; base += 32) {
        const uint32_t w = base + lane;
        uint32_t v = w < nw ? bm[w] : 0u;
        if (w == nw - 1 && (RB & 31)) v &= (1u << (RB & 31)) - 1u;
        const uint32_t cnt = __popc(v);
        uint32_t incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += o;
        }
        const uint32_t block = __shfl_sync(FULL, incl, 31);
        if (total + block > EXPAND_LIST_MAX) {
            __syncwarp();
            return EXPAND_LIST_MAX + 1;
        }
        uint32_t at = total + incl - cnt;
        while (v) {
            list[at++] = 32 * w + __ffs(v) - 1;
            v &= v - 1;
        }
        total += block;
    }
    __syncwarp();
    // every repetition present?  the entries are sorted, so count the
    // repetition changes along the list
    bool first = false;
    if ((uint32_t)lane < total) {
        const uint32_t r = list[lane] / B;
        first = lane == 0 || list[lane - 1] / B != r;
    }
    *dead = (uint32_t)__popc(__ballot_sync(FULL, first)) < R;
    return total;
}

// One chunk of a query's answer (lane words w0 + 32c, c < C) from its
// decoded bucket list: rows of the same repetition ORed, repetitions ANDed.
// Every repetition has an entry unless `dead`, so a repetition boundary is
// crossed exactly when an entry reaches the next repetition's first bucket.
template <int C>
__device__ __forceinline__ void expand_unit_list(const ExpandArgs &a, const uint32_t *list, uint32_t n,
                                                 bool dead, uint64_t q, uint32_t w0) {
    uint32_t res[C], o[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        res[c] = dead ? 0u : FULL;
        o[c] = 0;
    }
    if (!dead) {
        uint32_t next = (list[0] / a.B + 1) * a.B;  // first bucket index of the next repetition
        for (uint32_t t = 0; t < n; ++t) {
            const uint32_t i = list[t];
            if (i >= next) {
                uint32_t nz = 0;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    res[c] &= o[c];
                    o[c] = 0;
                    nz |= res[c];
                }
                next += a.B;
                if (!__any_sync(FULL, nz)) break;  // the intersection is already empty
            }
            const uint32_t *row = a.docbits + (uint64_t)i * a.W;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const uint32_t w = w0 + 32 * c;
                if (w < a.W) o[c] |= __ldg(row + w);
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) res[c] &= o[c];
    }
    uint32_t *out = a.out + q * a.W;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const uint32_t w = w0 + 32 * c;
        if (w < a.W) out[w] = res[c];
    }
}

// The whole answer of one query (chunks of 32*C words), by one warp: with
// several chunks and no byte table, the passing buckets are decoded once
// into `list` (EXPAND_LIST_MAX words of the warp's shared memory) and each
// chunk walks them; otherwise, or when more buckets pass, each chunk scans
// the mask itself.
//
// With a heavy list (the persistent fused query), a query with more passing
// buckets than the list holds is not expanded here: its mask is stored at
// acc_out[q] and q is appended to heavy_list, and a later launch spreads its
// chunks over all warps (one such query costs R*B/8 byte scans and a row per
// passing bucket for every chunk, which one warp would take alone).
template <int C>
__device__ __forceinline__ void expand_query(const ExpandArgs &a, const uint32_t *bm, uint64_t q,
                                             uint32_t chunks, int lane, uint32_t *list,
                                             uint32_t *heavy_list = nullptr, uint32_t *heavy_count = nullptr,
                                             uint32_t *acc_out = nullptr) {
    if (chunks > 1 && !a.tab) {
        bool dead = false;
        const uint32_t n = bucket_list(bm, a.R, a.B, list, lane, &dead);
        if (n <= EXPAND_LIST_MAX) {
            for (uint32_t c = 0; c < chunks; ++c) expand_unit_list<C>(a, list, n, dead, q, c * 32 * C + lane);
            __syncwarp();  // the list is the next query's
            return;
        }
        if (heavy_list) {
            for (uint32_t w = lane; w < a.Gw; w += 32) acc_out[q * a.Gw + w] = bm[w];
            if (lane == 0) heavy_list[atomicAdd(heavy_count, 1u)] = (uint32_t)q;
            __syncwarp();
            return;
        }
    }
    for (uint32_t c = 0; c < chunks; ++c) expand_one<C>(a, bm, q, c * 32 * C + lane, lane);
}

template <typename KernelT>
int blocks_per_sm(KernelT kernel, int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

}  // namespace
}  // namespace rgpu

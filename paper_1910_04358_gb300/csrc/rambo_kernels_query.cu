// rambo_kernels_query.cu -- the batched query path.
//
//   probe  (Algorithm 2's BFU membership tests, Section 3.3 / 3.3.1): every
//          k-mer of every query is canonicalised and hashed eta times; each
//          probe reads ONE position group -- the bits of all R*B BFUs at that
//          position -- so the per-BFU AND over eta probes and over all k-mers
//          of a query is a plain bitwise AND of groups.  The result per query
//          is its bucket mask: bit r*B+b set iff "Q in BFU(M[b,r])".
//   expand (Algorithm 2's union and intersection): per repetition, the OR of
//          the document bitmaps of the passing buckets; then the AND over the
//          R repetitions, written as a K-bit mask.
#include "rambo_internal.cuh"

namespace rgpu {
namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr uint32_t NONE = 0xffffffffu;
constexpr int PROBE_THREADS = 256;

__device__ __forceinline__ uint32_t reduce_pos(uint64_t h, uint64_t m, uint32_t m_pow2) {
    return (uint32_t)(m_pow2 ? (h & (m - 1)) : (h % m));
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
// probe: sequences.
//
// Lane roles.  A position group is read by LPG lanes, each loading an SW-word
// slice (16 bytes when the group is >= 16 bytes), so one warp instruction
// reads 32/LPG whole groups as runs of full 32-byte sectors.  Each warp walks
// a contiguous range of the batch's flattened k-mer index in batches of
// NT tiles of 32 k-mers: first every lane extracts and hashes one k-mer per
// tile (phase 1), then the lanes load the groups of those k-mers four rounds
// at a time, 4*ETA independent loads per lane in flight (phase 2).  Each lane
// keeps a running AND of its slice for the query it is on and flushes it with
// atomicAnd when its query changes; at the end the warp combines lanes that
// share a query before flushing.
template <int SW, int LPG, int ETA>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_seqs(ProbeArgs a) {
    constexpr int NT = LPG >= 4 ? 1 : 4 / LPG;
    constexpr int KPR = 32 / LPG;
    constexpr int ROUNDS = NT * LPG;
    constexpr int STEP = 32 * NT;
    const int lane = threadIdx.x & 31;
    const int sub = lane / LPG;
    const uint32_t word0 = blockIdx.y * (LPG * SW) + (lane % LPG) * SW;

    const uint64_t T = a.kcum[a.n];
    uint64_t c0, c1;
    warp_range<STEP>(T, a.min_chunk, c0, c1);
    if (c0 >= T) return;
    const uint64_t q_first = find_query(a.kcum, a.n, c0);

    uint32_t cur_q = NONE;
    Slice<SW> accv;
    slice_ones(accv);

    for (uint32_t jb = 0; jb < a.eta; jb += ETA) {
        uint64_t qlane = q_first;
        for (uint64_t base = c0; base < c1; base += STEP) {
            // phase 1: k-mer, canonical form, probe positions
            uint32_t qid[NT];
            uint32_t pos[NT][ETA];
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const uint64_t g = base + (uint64_t)t * 32 + lane;
                uint64_t c = 0;
                qid[t] = NONE;
                if (g < c1) {
                    while (a.kcum[qlane + 1] <= g) ++qlane;
                    const uint64_t start = a.offsets[qlane] + a.base_shift + (g - a.kcum[qlane]);
                    c = canonical_from_window(base_window(a.packed, a.packed_bytes, start), a.k);
                    qid[t] = (uint32_t)qlane;
                }
                const uint64_t km = mh_mix_key(c);
#pragma unroll
                for (int e = 0; e < ETA; ++e) {
                    const uint32_t j = jb + e < a.eta ? jb + e : a.eta - 1;
                    pos[t][e] = reduce_pos(mh_first_word(km, a.seed32 + j), a.m, a.m_pow2);
                }
            }
            // phase 2: group loads, four rounds in flight, then accumulate
#pragma unroll
            for (int rg = 0; rg < ROUNDS; rg += 4) {
                Slice<SW> v[4][ETA];
                uint32_t qk[4];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    const int rho = rg + rr;
                    const int t = rho / LPG;
                    const int src = (rho % LPG) * KPR + sub;
                    qk[rr] = __shfl_sync(FULL, qid[t], src);
#pragma unroll
                    for (int e = 0; e < ETA; ++e) {
                        const uint32_t p = __shfl_sync(FULL, pos[t][e], src);
                        if (qk[rr] != NONE) v[rr][e] = ld_slice<SW>(a.index + (uint64_t)p * a.Gw + word0);
                        else slice_ones(v[rr][e]);
                    }
                }
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    if (qk[rr] == NONE) continue;
                    Slice<SW> x = v[rr][0];
#pragma unroll
                    for (int e = 1; e < ETA; ++e) slice_and(x, v[rr][e]);
                    if (qk[rr] != cur_q) {
                        if (cur_q != NONE) flush_slice<SW>(a.acc, cur_q, a.Gw, word0, accv);
                        cur_q = qk[rr];
                        accv = x;
                    } else {
                        slice_and(accv, x);
                    }
                }
            }
        }
    }
    // final flush: if the whole warp is on one query, AND the lanes that hold
    // the same slice first so only one lane per slice issues atomics
    int same = 0;
    __match_all_sync(FULL, cur_q, &same);
    if (same) {
        if (cur_q == NONE) return;
#pragma unroll
        for (int w = 0; w < SW; ++w)
#pragma unroll
            for (int off = LPG; off < 32; off <<= 1) accv.w[w] &= __shfl_xor_sync(FULL, accv.w[w], off);
        if (sub == 0) flush_slice<SW>(a.acc, cur_q, a.Gw, word0, accv);
    } else if (cur_q != NONE) {
        flush_slice<SW>(a.acc, cur_q, a.Gw, word0, accv);
    }
}

// ---------------------------------------------------------------------------
// probe: single k-mers (each k-mer is its own query; no cross-k-mer AND, so
// the bucket mask is stored directly).
template <int SW, int LPG, int ETA>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_kmers(ProbeArgs a) {
    constexpr int NT = LPG >= 4 ? 1 : 4 / LPG;
    constexpr int KPR = 32 / LPG;
    constexpr int ROUNDS = NT * LPG;
    constexpr int STEP = 32 * NT;
    const int lane = threadIdx.x & 31;
    const int sub = lane / LPG;
    const uint32_t word0 = blockIdx.y * (LPG * SW) + (lane % LPG) * SW;

    const uint64_t T = a.n;
    uint64_t c0, c1;
    warp_range<STEP>(T, a.min_chunk, c0, c1);
    if (c0 >= T) return;
    const uint64_t kbits = kmask(a.k);

    for (uint32_t jb = 0; jb < a.eta; jb += ETA) {
        for (uint64_t base = c0; base < c1; base += STEP) {
            uint32_t pos[NT][ETA];
            bool val[NT];
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const uint64_t g = base + (uint64_t)t * 32 + lane;
                val[t] = g < c1;
                uint64_t c = 0;
                if (val[t]) {
                    uint64_t code = a.kmers[g];
                    if (code & ~kbits) {
                        if (jb == 0) atomicOr(a.err, ERR_KMER_CODE);
                        code &= kbits;
                    }
                    c = canonical_from_forward(code, a.k);
                }
                const uint64_t km = mh_mix_key(c);
#pragma unroll
                for (int e = 0; e < ETA; ++e) {
                    const uint32_t j = jb + e < a.eta ? jb + e : a.eta - 1;
                    pos[t][e] = reduce_pos(mh_first_word(km, a.seed32 + j), a.m, a.m_pow2);
                }
            }
#pragma unroll
            for (int rg = 0; rg < ROUNDS; rg += 4) {
                Slice<SW> v[4][ETA];
                bool vs[4];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    const int rho = rg + rr;
                    const int t = rho / LPG;
                    const int src = (rho % LPG) * KPR + sub;
                    vs[rr] = __shfl_sync(FULL, (int)val[t], src) != 0;
#pragma unroll
                    for (int e = 0; e < ETA; ++e) {
                        const uint32_t p = __shfl_sync(FULL, pos[t][e], src);
                        if (vs[rr]) v[rr][e] = ld_slice<SW>(a.index + (uint64_t)p * a.Gw + word0);
                        else slice_ones(v[rr][e]);
                    }
                }
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    if (!vs[rr]) continue;
                    const int rho = rg + rr;
                    const uint64_t g = base + (uint64_t)(rho / LPG) * 32 + (rho % LPG) * KPR + sub;
                    Slice<SW> x = v[rr][0];
#pragma unroll
                    for (int e = 1; e < ETA; ++e) slice_and(x, v[rr][e]);
                    uint32_t *p = a.acc + g * a.Gw + word0;
                    if (jb == 0) {
#pragma unroll
                        for (int w = 0; w < SW; ++w) p[w] = x.w[w];
                    } else {
#pragma unroll
                        for (int w = 0; w < SW; ++w) atomicAnd(p + w, x.w[w]);
                    }
                }
            }
        }
    }
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
            uint32_t v = row_byte(bm, a.Gw, a.B, r, j);
            any |= v != 0;
            while (v) {
                const uint32_t b = 8 * j + __ffs(v) - 1;
                v &= v - 1;
                const uint32_t *row = a.docbits + (uint64_t)(r * a.B + b) * a.W;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t w = w0 + 32 * c;
                    if (w < a.W) o[c] |= __ldg(row + w);
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

// SMEM: DocBits is first copied into shared memory by the whole block.
template <int C, bool SMEM>
__global__ void __launch_bounds__(EXPAND_THREADS) k_expand(ExpandArgs a) {
    extern __shared__ uint32_t sdb[];
    if (SMEM) {
        const uint32_t words = a.R * a.B * a.W;
        for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) sdb[i] = __ldg(a.docbits + i);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (uint64_t)blockIdx.x * (EXPAND_THREADS / 32) + threadIdx.x / 32;
    const uint64_t nwarps = (uint64_t)gridDim.x * (EXPAND_THREADS / 32);
    const uint32_t chunks = (a.W + 32 * C - 1) / (32 * C);
    const uint64_t units = a.n * chunks;
    for (uint64_t u = warp; u < units; u += nwarps) {
        const uint64_t q = chunks == 1 ? u : u / chunks;
        const uint32_t w0 = (uint32_t)(u - q * chunks) * 32 * C + lane;
        if (SMEM) expand_unit_smem<C>(a, sdb, a.acc + q * a.Gw, q, w0);
        else expand_one<C>(a, a.acc + q * a.Gw, q, w0, lane);
    }
}

// Expansion through the nibble table in shared memory (small K): one query
// per warp, every lane holding up to 32*C answer words.  The query's bucket
// mask (Gw <= 32 words) sits in lane registers, one word per lane, and rows
// are fetched 32 bits at a time with shuffles; every nonzero 4-bucket nibble
// of a row costs one conflict-free shared-memory row read.
constexpr size_t SMEM_NIBTAB_MAX = 96 * 1024;

template <int C>
__global__ void __launch_bounds__(EXPAND_THREADS) k_expand_nib(ExpandArgs a) {
    extern __shared__ uint32_t stab[];
    const uint32_t NQ = (a.B + 3) / 4;
    const uint32_t words = a.R * NQ * 16 * a.W;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) stab[i] = __ldg(a.ntab + i);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t stride = 16 * a.W;  // words from one nibble position to the next
    const uint64_t warp = (uint64_t)blockIdx.x * (EXPAND_THREADS / 32) + threadIdx.x / 32;
    const uint64_t nwarps = (uint64_t)gridDim.x * (EXPAND_THREADS / 32);
    for (uint64_t q = warp; q < a.n; q += nwarps) {
        const uint32_t bmw = (uint32_t)lane < a.Gw ? __ldg(a.acc + q * a.Gw + lane) : 0u;
        uint32_t res[C];
#pragma unroll
        for (int c = 0; c < C; ++c) res[c] = FULL;
        bool dead = false;
        const uint32_t *tj = stab + lane;  // table row of (r, nibble position), this lane's word
        for (uint32_t r = 0; r < a.R; ++r) {
            uint32_t o[C];
#pragma unroll
            for (int c = 0; c < C; ++c) o[c] = 0;
            uint32_t any = 0;
            for (uint32_t i = 0; i < a.B; i += 32) {
                const uint32_t bit = r * a.B + i, wi = bit >> 5, sh = bit & 31;
                const uint32_t w0v = __shfl_sync(FULL, bmw, wi & 31);
                const uint32_t w1v = __shfl_sync(FULL, bmw, (wi + 1) & 31);
                uint32_t chunk = sh ? __funnelshift_r(w0v, wi + 1 < a.Gw ? w1v : 0u, sh) : w0v;
                const uint32_t nb = a.B - i < 32 ? a.B - i : 32;
                if (nb < 32) chunk &= (1u << nb) - 1u;
                any |= chunk;
                // every nibble is looked up: value 0 selects the all-zero row
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    if (i + 4 * t < a.B) {
                        const uint32_t *row = tj + ((chunk >> (4 * t)) & 15u) * a.W;
#pragma unroll
                        for (int c = 0; c < C; ++c)
                            if (lane + 32 * c < (int)a.W) o[c] |= row[32 * c];
                        tj += stride;
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c) res[c] &= o[c];
            if (!any) dead = true;
        }
        uint32_t *out = a.out + q * a.W;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const uint32_t w = lane + 32 * c;
            if (w < a.W) out[w] = dead ? 0u : res[c];
        }
    }
}

// Expansion by candidate filtering (the paper's sparse evaluation, Section
// 5.1 "Query time speedup", applied per document): the union of repetition 0
// is formed from the nibble table (its repetition-0 rows staged in shared
// memory); for every later repetition r only the documents still set are
// tested -- document d survives iff bit phi_r(d) of row r is set -- with phi
// staged in shared memory as bytes (B <= 256) and the query's bucket mask in
// a per-warp shared slot.  The surviving set after the last repetition is
// exactly AND_r of the unions.  One query per warp, each lane owning answer
// words lane + 32c (W <= 32*C); Gw <= 32.
template <int C>
__global__ void __launch_bounds__(EXPAND_THREADS) k_expand_filter(ExpandArgs a) {
    extern __shared__ uint32_t smem_f[];
    const uint32_t NQ = (a.B + 3) / 4;
    const uint32_t tab0 = NQ * 16 * a.W;  // nibble-table words of repetition 0
    uint32_t *stab = smem_f;
    uint32_t *sbm = smem_f + tab0;        // EXPAND_THREADS/32 slots of 32 words
    uint8_t *sphi = reinterpret_cast<uint8_t *>(sbm + EXPAND_THREADS);  // K*R bytes
    for (uint32_t i = threadIdx.x; i < tab0; i += blockDim.x) stab[i] = __ldg(a.ntab + i);
    for (uint32_t i = threadIdx.x; i < a.K * a.R; i += blockDim.x) sphi[i] = (uint8_t)__ldg(a.phi + i);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint32_t *bm = sbm + (threadIdx.x / 32) * 32;
    const uint64_t warp = (uint64_t)blockIdx.x * (EXPAND_THREADS / 32) + threadIdx.x / 32;
    const uint64_t nwarps = (uint64_t)gridDim.x * (EXPAND_THREADS / 32);
    for (uint64_t q = warp; q < a.n; q += nwarps) {
        bm[lane] = (uint32_t)lane < a.Gw ? __ldg(a.acc + q * a.Gw + lane) : 0u;
        __syncwarp();
        // repetition 0: union of the passing buckets via the nibble table
        uint32_t res[C];
#pragma unroll
        for (int c = 0; c < C; ++c) res[c] = 0;
        for (uint32_t i = 0; i < a.B; i += 32) {
            uint32_t chunk = bm[i >> 5];
            const uint32_t nb = a.B - i < 32 ? a.B - i : 32;
            if (nb < 32) chunk &= (1u << nb) - 1u;
            const uint32_t j0 = i / 4;
            while (chunk) {
                const uint32_t t = (__ffs(chunk) - 1) & ~3u;
                const uint32_t v = (chunk >> t) & 15u;
                chunk &= ~(15u << t);
                const uint32_t *row = stab + (((j0 + t / 4) * 16 + v) * a.W);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t w = lane + 32 * c;
                    if (w < a.W) res[c] |= row[w];
                }
            }
        }
        // repetitions 1..R-1: keep the candidates whose bucket passes
        for (uint32_t r = 1; r < a.R; ++r) {
            uint32_t nz = 0;
            const uint32_t lo = r * a.B;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                uint32_t x = res[c], keep = 0;
                const uint32_t d0 = 32 * (lane + 32 * c);
                while (x) {
                    const uint32_t j = __ffs(x) - 1;
                    x &= x - 1;
                    const uint32_t bit = lo + sphi[(d0 + j) * a.R + r];
                    keep |= ((bm[bit >> 5] >> (bit & 31)) & 1u) << j;
                }
                res[c] = keep;
                nz |= keep;
            }
            if (!__any_sync(FULL, nz)) break;
        }
        uint32_t *out = a.out + q * a.W;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const uint32_t w = lane + 32 * c;
            if (w < a.W) out[w] = res[c];
        }
        __syncwarp();
    }
}

// Nibble table: ntab[((r*NQ + j)*16 + v)*W + w] = OR over set bits t of v
// (4j+t < B) of DocBits[r][4j+t][w].
__global__ void k_build_nibtab(const uint32_t *docbits, uint32_t B, uint32_t R, uint32_t W,
                               uint32_t *ntab) {
    const uint32_t NQ = (B + 3) / 4;
    const uint64_t total = (uint64_t)R * NQ * 16 * W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t w = (uint32_t)(i % W);
        const uint64_t rest = i / W;
        const uint32_t v = (uint32_t)(rest % 16);
        const uint64_t rj = rest / 16;
        const uint32_t j = (uint32_t)(rj % NQ), r = (uint32_t)(rj / NQ);
        uint32_t o = 0;
        for (uint32_t t = 0; t < 4; ++t) {
            const uint32_t b = 4 * j + t;
            if (((v >> t) & 1u) && b < B) o |= docbits[((uint64_t)r * B + b) * W + w];
        }
        ntab[i] = o;
    }
}

// Byte table: tab[((r*NJ + j)*256 + v)*W + w] = OR over set bits i of v
// (8j+i < B) of DocBits[r][8j+i][w].
__global__ void k_build_bytetab(const uint32_t *docbits, uint32_t B, uint32_t R, uint32_t W,
                                uint32_t *tab) {
    const uint32_t NJ = (B + 7) / 8;
    const uint64_t total = (uint64_t)R * NJ * 256 * W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t w = (uint32_t)(i % W);
        const uint64_t rest = i / W;
        const uint32_t v = (uint32_t)(rest % 256);
        const uint64_t rj = rest / 256;
        const uint32_t j = (uint32_t)(rj % NJ), r = (uint32_t)(rj / NJ);
        uint32_t o = 0;
        for (uint32_t t = 0; t < 8; ++t) {
            const uint32_t b = 8 * j + t;
            if (((v >> t) & 1u) && b < B) o |= docbits[((uint64_t)r * B + b) * W + w];
        }
        tab[i] = o;
    }
}

// ---------------------------------------------------------------------------
// persistent fused query: length-bucketed work queues in one launch.
//
// Before the launch, a prefix scan numbers the tiles of the long queries
// (more than short_max k-mers; ceil(k-mers / tile) tiles each) into one
// global range, and a prep kernel (one thread per query) appends each short
// query to the short queue and sets each long query's bucket mask to all
// ones and its completion counter to zero.  The persistent kernel's warps
// then
//   1. claim long-query tiles with one atomicAdd on a global tile counter
//      (tile -> query by binary search in the tile prefix); a tile's AND is
//      flushed with atomicAnd, and the warp that completes a query's last
//      tile expands its answer;
//   2. then take whole short queries from the short queue: the warp probes
//      all k-mers, combines the lanes' slices into the bucket mask in shared
//      memory and expands the answer itself, with no global round trip.
// No warp ever waits on another.  Every k-mer of every query is probed; the
// answers are the plain path's.
constexpr int FUSED_THREADS = 256;

struct FusedArgs {
    ProbeArgs p;                 // index, geometry, batch (kcum unused)
    uint32_t *counters;          // [0] short count [1] short head [2..3] 64-bit tile head
    uint32_t *short_list;        // n
    const uint64_t *tile_prefix; // n+1
    uint32_t *done;              // n (long queries)
    uint32_t tile;               // k-mers per long tile
    uint32_t short_max;          // k-mers of the longest short query
    uint64_t user_bases;         // bases addressable from the caller's pointer
    ExpandArgs e;                // acc = bucket masks of long queries
    uint32_t early_exit;         // 1: stop probing a query once a repetition row is empty
    uint32_t segment;            // early exit: k-mers between checks of a short query
    unsigned long long *probed;  // early exit: k-mers actually probed (or null)
};

// True when some repetition's row of the bucket mask bm (shared memory) has
// no bit set: the answer is then empty whatever the remaining k-mers give.
__device__ __forceinline__ bool mask_dead(const uint32_t *bm, uint32_t Gw, uint32_t B, uint32_t R,
                                          int lane) {
    bool dead = false;
    for (uint32_t r0 = 0; r0 < R; r0 += 32) {
        const uint32_t r = r0 + lane;
        bool empty = false;
        if (r < R) {
            empty = true;
            for (uint32_t i = 0; i < B && empty; i += 32) {
                const uint32_t bit = r * B + i, wi = bit >> 5, sh = bit & 31;
                uint32_t chunk = bm[wi];
                if (sh) chunk = __funnelshift_r(chunk, wi + 1 < Gw ? bm[wi + 1] : 0u, sh);
                const uint32_t nb = B - i < 32 ? B - i : 32;
                if (nb < 32) chunk &= (1u << nb) - 1u;
                if (chunk) empty = false;
            }
        }
        if (__any_sync(FULL, empty)) dead = true;
    }
    return dead;
}

__device__ __forceinline__ uint64_t fused_kmers(const FusedArgs &f, uint64_t q, uint64_t *start) {
    const uint64_t b0 = f.p.offsets[q], b1 = f.p.ends[q];
    *start = b0;
    if (b1 < b0 || b1 > f.user_bases) return 0;
    const uint64_t L = b1 - b0;
    return L >= f.p.k ? L - f.p.k + 1 : 0;
}

__global__ void k_fused_prep(FusedArgs f) {
    const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= f.p.n) return;
    if (f.tile_prefix[q + 1] == f.tile_prefix[q]) {
        f.short_list[atomicAdd(&f.counters[0], 1u)] = (uint32_t)q;
    } else {
        uint32_t *acc = const_cast<uint32_t *>(f.e.acc);  // the masks this launch owns
        for (uint32_t w = 0; w < f.p.Gw; ++w) acc[q * f.p.Gw + w] = FULL;
        f.done[q] = 0;
    }
}

// AND of the groups of k-mers [k0, k1) of one query, per lane slice (every
// lane of the warp works on the same query).
template <int SW, int LPG, int ETA>
__device__ __forceinline__ Slice<SW> fused_probe_range(const ProbeArgs &a, uint64_t start,
                                                        uint64_t k0, uint64_t k1, int lane,
                                                        uint32_t word0) {
    constexpr int NT = LPG >= 4 ? 1 : 4 / LPG;
    constexpr int KPR = 32 / LPG;
    constexpr int ROUNDS = NT * LPG;
    constexpr int STEP = 32 * NT;
    const int sub = lane / LPG;
    Slice<SW> accv;
    slice_ones(accv);
    for (uint32_t jb = 0; jb < a.eta; jb += ETA) {
        for (uint64_t base = k0; base < k1; base += STEP) {
            uint32_t pos[NT][ETA];
            bool val[NT];
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const uint64_t g = base + (uint64_t)t * 32 + lane;
                val[t] = g < k1;
                uint64_t c = 0;
                if (val[t])
                    c = canonical_from_window(base_window(a.packed, a.packed_bytes, start + a.base_shift + g), a.k);
                const uint64_t km = mh_mix_key(c);
#pragma unroll
                for (int e = 0; e < ETA; ++e) {
                    const uint32_t j = jb + e < a.eta ? jb + e : a.eta - 1;
                    pos[t][e] = reduce_pos(mh_first_word(km, a.seed32 + j), a.m, a.m_pow2);
                }
            }
#pragma unroll
            for (int rg = 0; rg < ROUNDS; rg += 4) {
                Slice<SW> v[4][ETA];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    const int rho = rg + rr;
                    const int t = rho / LPG;
                    const int src = (rho % LPG) * KPR + sub;
                    const bool vs = __shfl_sync(FULL, (int)val[t], src) != 0;
#pragma unroll
                    for (int e = 0; e < ETA; ++e) {
                        const uint32_t p = __shfl_sync(FULL, pos[t][e], src);
                        if (vs) v[rr][e] = ld_slice<SW>(a.index + (uint64_t)p * a.Gw + word0);
                        else slice_ones(v[rr][e]);
                    }
                }
#pragma unroll
                for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                    for (int e = 0; e < ETA; ++e) slice_and(accv, v[rr][e]);
            }
        }
    }
    // combine the lanes that hold the same slice
#pragma unroll
    for (int w = 0; w < SW; ++w)
#pragma unroll
        for (int off = LPG; off < 32; off <<= 1) accv.w[w] &= __shfl_xor_sync(FULL, accv.w[w], off);
    return accv;
}

template <int SW, int LPG, int ETA, int C>
__global__ void __launch_bounds__(FUSED_THREADS) k_fused(FusedArgs f) {
    __shared__ uint32_t bm_smem[FUSED_THREADS / 32][128];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t *bm = bm_smem[wib];
    const int sub = lane / LPG;
    const uint32_t word0 = (lane % LPG) * SW;
    const uint32_t n_short = f.counters[0];
    const uint64_t n_tiles = f.tile_prefix[f.p.n];
    const uint32_t chunks = (f.e.W + 32 * C - 1) / (32 * C);

    // 1. long queries, tile by tile
    while (true) {
        uint64_t t = 0;
        if (lane == 0) t = atomicAdd(reinterpret_cast<unsigned long long *>(f.counters + 2), 1ULL);
        t = __shfl_sync(FULL, t, 0);
        if (t >= n_tiles) break;
        // the query whose tile range holds t: largest q with tile_prefix[q] <= t
        uint64_t lo = 0, hi = f.p.n;
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) >> 1;
            if (f.tile_prefix[mid] <= t) lo = mid;
            else hi = mid;
        }
        const uint64_t q = lo;
        const uint64_t tiles = f.tile_prefix[q + 1] - f.tile_prefix[q];
        uint64_t start;
        const uint64_t nk = fused_kmers(f, q, &start);
        const uint64_t k0 = (t - f.tile_prefix[q]) * f.tile;
        const uint64_t k1 = k0 + f.tile < nk ? k0 + f.tile : nk;
        bool skip = false;
        if (f.early_exit) {  // a tile of an already-empty query changes nothing
            for (uint32_t w = lane; w < f.p.Gw; w += 32) bm[w] = __ldcg(f.e.acc + q * f.p.Gw + w);
            __syncwarp();
            skip = mask_dead(bm, f.p.Gw, f.e.B, f.e.R, lane);
            __syncwarp();
            if (!skip && lane == 0 && f.probed) atomicAdd(f.probed, (unsigned long long)(k1 - k0));
        }
        if (!skip) {
            const Slice<SW> s = fused_probe_range<SW, LPG, ETA>(f.p, start, k0, k1, lane, word0);
            if (sub == 0) flush_slice<SW>(const_cast<uint32_t *>(f.e.acc), q, f.p.Gw, word0, s);
        }
        __threadfence();
        __syncwarp();
        uint32_t last = 0;
        if (lane == 0) last = atomicAdd(&f.done[q], 1u) == tiles - 1;
        last = __shfl_sync(FULL, last, 0);
        if (last) {
            __threadfence();
            for (uint32_t w = lane; w < f.p.Gw; w += 32) bm[w] = __ldcg(f.e.acc + q * f.p.Gw + w);
            __syncwarp();
            for (uint32_t c = 0; c < chunks; ++c) expand_one<C>(f.e, bm, q, c * 32 * C + lane, lane);
            __syncwarp();
        }
    }
    // 2. short queries, one warp each, probe and expand fused
    while (true) {
        uint32_t s = 0;
        if (lane == 0) s = atomicAdd(&f.counters[1], 1u);
        s = __shfl_sync(FULL, s, 0);
        if (s >= n_short) break;
        const uint32_t q = f.short_list[s];
        uint64_t start;
        const uint64_t nk = fused_kmers(f, q, &start);
        Slice<SW> sl;
        slice_ones(sl);
        const uint64_t seg = f.early_exit ? f.segment : (nk ? nk : 1);
        for (uint64_t k0 = 0; k0 < nk; k0 += seg) {
            const uint64_t k1 = k0 + seg < nk ? k0 + seg : nk;
            slice_and(sl, fused_probe_range<SW, LPG, ETA>(f.p, start, k0, k1, lane, word0));
            if (!f.early_exit) continue;
            if (lane == 0 && f.probed) atomicAdd(f.probed, (unsigned long long)(k1 - k0));
            if (k1 >= nk) break;
            if (sub == 0)
#pragma unroll
                for (int w = 0; w < SW; ++w) bm[word0 + w] = sl.w[w];
            __syncwarp();
            const bool dead = mask_dead(bm, f.p.Gw, f.e.B, f.e.R, lane);
            __syncwarp();
            if (dead) break;
        }
        if (sub == 0)
#pragma unroll
            for (int w = 0; w < SW; ++w) bm[word0 + w] = sl.w[w];
        __syncwarp();
        for (uint32_t c = 0; c < chunks; ++c) expand_one<C>(f.e, bm, q, c * 32 * C + lane, lane);
        __syncwarp();
    }
}

template <typename KernelT>
int blocks_per_sm(KernelT kernel, int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

template <int SW, int LPG, int ETA>
cudaError_t launch_probe_t(const ProbeArgs &a, const Geometry &g, int sm_count, cudaStream_t s,
                           bool kmers) {
    // sm_count > 0: SMs x occupancy maximum; sm_count < 0: -sm_count CTAs
    dim3 grid, block(PROBE_THREADS);
    if (kmers) {
        static int occ = blocks_per_sm(k_probe_kmers<SW, LPG, ETA>, PROBE_THREADS, 0);
        grid = dim3(sm_count > 0 ? sm_count * occ : -sm_count, g.chunks);
        k_probe_kmers<SW, LPG, ETA><<<grid, block, 0, s>>>(a);
    } else {
        static int occ = blocks_per_sm(k_probe_seqs<SW, LPG, ETA>, PROBE_THREADS, 0);
        grid = dim3(sm_count > 0 ? sm_count * occ : -sm_count, g.chunks);
        k_probe_seqs<SW, LPG, ETA><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int SW, int LPG>
cudaError_t launch_probe_eta(const ProbeArgs &a, const Geometry &g, int sm, cudaStream_t s, bool km) {
    switch (g.eta) {
        case 1: return launch_probe_t<SW, LPG, 1>(a, g, sm, s, km);
        case 2: return launch_probe_t<SW, LPG, 2>(a, g, sm, s, km);
        case 3: return launch_probe_t<SW, LPG, 3>(a, g, sm, s, km);
        default: return launch_probe_t<SW, LPG, 4>(a, g, sm, s, km);
    }
}

cudaError_t launch_probe(const ProbeArgs &a, const Geometry &g, int sm, cudaStream_t s, bool km) {
    if (g.SW == 1) return launch_probe_eta<1, 1>(a, g, sm, s, km);
    if (g.SW == 2) return launch_probe_eta<2, 1>(a, g, sm, s, km);
    switch (g.LPG) {
        case 1: return launch_probe_eta<4, 1>(a, g, sm, s, km);
        case 2: return launch_probe_eta<4, 2>(a, g, sm, s, km);
        case 4: return launch_probe_eta<4, 4>(a, g, sm, s, km);
        case 8: return launch_probe_eta<4, 8>(a, g, sm, s, km);
        case 16: return launch_probe_eta<4, 16>(a, g, sm, s, km);
        case 32: return launch_probe_eta<4, 32>(a, g, sm, s, km);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_probe_seqs(const ProbeArgs &a, const Geometry &g, int sm_count, cudaStream_t s) {
    return launch_probe(a, g, sm_count, s, false);
}

cudaError_t launch_probe_kmers(const ProbeArgs &a, const Geometry &g, int sm_count, cudaStream_t s) {
    return launch_probe(a, g, sm_count, s, true);
}

cudaError_t launch_expand(const ExpandArgs &a, int max_blocks, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    const uint32_t wc = (a.W + 31) / 32;
    const int C = wc >= 8 ? 8 : wc >= 4 ? 4 : wc >= 2 ? 2 : 1;
    const uint64_t units = a.n * ((a.W + 32 * C - 1) / (32 * C));
    uint64_t blocks = (units + EXPAND_THREADS / 32 - 1) / (EXPAND_THREADS / 32);
    const uint64_t cap = (uint64_t)max_blocks;
    if (blocks > cap) blocks = cap;
    // candidate filtering: repetition-0 nibble rows, the per-warp mask slots
    // and phi as bytes in shared memory
    const size_t filt_bytes = (size_t)((a.B + 3) / 4) * 16 * a.W * 4 + EXPAND_THREADS * 4 +
                              ((size_t)a.K * a.R + 3) / 4 * 4;
    if (a.filter && a.ntab && a.phi && a.Gw <= 32 && a.W <= 64 && a.B <= 256 &&
        filt_bytes <= SMEM_NIBTAB_MAX && a.n >= (uint64_t)max_blocks * 64) {
        cudaError_t e2 = cudaSuccess;
        if (filt_bytes > 48 * 1024)
            e2 = a.W > 32 ? cudaFuncSetAttribute(k_expand_filter<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filt_bytes)
                          : cudaFuncSetAttribute(k_expand_filter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filt_bytes);
        if (e2 != cudaSuccess) return e2;
        if (a.W > 32) k_expand_filter<2><<<(unsigned)max_blocks, EXPAND_THREADS, filt_bytes, s>>>(a);
        else k_expand_filter<1><<<(unsigned)max_blocks, EXPAND_THREADS, filt_bytes, s>>>(a);
        return cudaGetLastError();
    }
    // nibble table in shared memory (small K): one query per warp
    const size_t nib_bytes = nibtab_words(a.B, a.R, a.W) * 4;
    if (a.ntab && a.Gw <= 32 && a.W <= 64 && nib_bytes <= SMEM_NIBTAB_MAX &&
        a.n >= (uint64_t)max_blocks * 64) {
        cudaError_t e2 = cudaSuccess;
        if (nib_bytes > 48 * 1024)
            e2 = a.W > 32 ? cudaFuncSetAttribute(k_expand_nib<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nib_bytes)
                          : cudaFuncSetAttribute(k_expand_nib<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nib_bytes);
        if (e2 != cudaSuccess) return e2;
        if (a.W > 32) k_expand_nib<2><<<(unsigned)max_blocks, EXPAND_THREADS, nib_bytes, s>>>(a);
        else k_expand_nib<1><<<(unsigned)max_blocks, EXPAND_THREADS, nib_bytes, s>>>(a);
        return cudaGetLastError();
    }
    // DocBits in shared memory when it fits and every block gets enough
    // queries to pay for staging it
    const size_t db_bytes = (size_t)a.R * a.B * a.W * 4;
    const bool smem = a.smem_docbits && db_bytes <= SMEM_DOCBITS_MAX && units >= blocks * 64;
    const size_t dyn = smem ? db_bytes : 0;
    cudaError_t e = cudaSuccess;
#define RGPU_EXPAND(CC)                                                                            \
    if (smem) {                                                                                    \
        if (dyn > 48 * 1024)                                                                       \
            e = cudaFuncSetAttribute(k_expand<CC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)dyn);                                                    \
        if (e == cudaSuccess) k_expand<CC, true><<<(unsigned)blocks, EXPAND_THREADS, dyn, s>>>(a); \
    } else {                                                                                       \
        k_expand<CC, false><<<(unsigned)blocks, EXPAND_THREADS, 0, s>>>(a);                       \
    }
    switch (C) {
        case 1: RGPU_EXPAND(1) break;
        case 2: RGPU_EXPAND(2) break;
        case 4: RGPU_EXPAND(4) break;
        default: RGPU_EXPAND(8) break;
    }
#undef RGPU_EXPAND
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int SW, int LPG, int ETA, int C>
cudaError_t launch_fused_t(const FusedArgs &f, int grid_override, int sm_count, cudaStream_t s) {
    static int occ = blocks_per_sm(k_fused<SW, LPG, ETA, C>, FUSED_THREADS, 0);
    const int grid = grid_override > 0 ? grid_override : sm_count * occ;
    k_fused<SW, LPG, ETA, C><<<grid, FUSED_THREADS, 0, s>>>(f);
    return cudaGetLastError();
}

template <int SW, int LPG, int ETA>
cudaError_t launch_fused_c(const FusedArgs &f, int go, int sm, cudaStream_t s) {
    if (f.e.W > 64) return launch_fused_t<SW, LPG, ETA, 4>(f, go, sm, s);
    return launch_fused_t<SW, LPG, ETA, 1>(f, go, sm, s);
}

template <int SW, int LPG>
cudaError_t launch_fused_e(const FusedArgs &f, int go, int sm, cudaStream_t s) {
    switch (f.p.eta) {
        case 1: return launch_fused_c<SW, LPG, 1>(f, go, sm, s);
        case 2: return launch_fused_c<SW, LPG, 2>(f, go, sm, s);
        default: return launch_fused_c<SW, LPG, 4>(f, go, sm, s);
    }
}

bool fused_supported(const Geometry &g) { return g.chunks == 1 && g.Gw <= 128; }

uint64_t nibtab_words(uint32_t B, uint32_t R, uint32_t W) {
    return (uint64_t)R * ((B + 3) / 4) * 16 * W;
}

cudaError_t launch_build_nibtab(const uint32_t *docbits, uint32_t B, uint32_t R, uint32_t W,
                                uint32_t *ntab, int sm_count, cudaStream_t s) {
    k_build_nibtab<<<sm_count * 4, 256, 0, s>>>(docbits, B, R, W, ntab);
    return cudaGetLastError();
}

uint64_t bytetab_words(uint32_t B, uint32_t R, uint32_t W) {
    return (uint64_t)R * ((B + 7) / 8) * 256 * W;
}

cudaError_t launch_build_bytetab(const uint32_t *docbits, uint32_t B, uint32_t R, uint32_t W,
                                 uint32_t *tab, int sm_count, cudaStream_t s) {
    k_build_bytetab<<<sm_count * 8, 256, 0, s>>>(docbits, B, R, W, tab);
    return cudaGetLastError();
}

cudaError_t launch_fused(const ProbeArgs &p, const ExpandArgs &e, const Geometry &g,
                         const FusedQueues &qs, int grid_override, int sm_count, cudaStream_t s) {
    if (!fused_supported(g)) return cudaErrorInvalidValue;
    FusedArgs f{};
    f.p = p;
    f.counters = qs.counters;
    f.short_list = qs.short_list;
    f.tile_prefix = qs.tile_prefix;
    f.done = qs.done;
    f.tile = qs.tile;
    f.short_max = qs.short_max;
    f.user_bases = qs.user_bases;
    f.e = e;
    f.early_exit = qs.early_exit;
    f.segment = qs.segment;
    f.probed = qs.probed;
    cudaError_t err = cudaMemsetAsync(qs.counters, 0, 4 * sizeof(uint32_t), s);
    if (err != cudaSuccess) return err;
    if (p.n == 0) return cudaSuccess;
    k_fused_prep<<<(unsigned)((p.n + 255) / 256), 256, 0, s>>>(f);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (g.SW == 1) return launch_fused_e<1, 1>(f, grid_override, sm_count, s);
    if (g.SW == 2) return launch_fused_e<2, 1>(f, grid_override, sm_count, s);
    switch (g.LPG) {
        case 1: return launch_fused_e<4, 1>(f, grid_override, sm_count, s);
        case 2: return launch_fused_e<4, 2>(f, grid_override, sm_count, s);
        case 4: return launch_fused_e<4, 4>(f, grid_override, sm_count, s);
        case 8: return launch_fused_e<4, 8>(f, grid_override, sm_count, s);
        case 16: return launch_fused_e<4, 16>(f, grid_override, sm_count, s);
        case 32: return launch_fused_e<4, 32>(f, grid_override, sm_count, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rgpu

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
// [r*B, r*B+B) of the query's bucket mask; the union of the passing buckets'
// document bitmaps is built byte by byte: a zero byte costs nothing, a byte
// with one set bit costs one DocBits row, a byte with several set bits costs
// one row of the byte table (the precomputed OR of DocBits over that 8-bucket
// pattern) when the table exists, else one row per set bit.  The answer is
// the AND of the R unions; a repetition with no passing bucket, or an
// all-zero running AND, ends the unit early.
constexpr int EXPAND_THREADS = 256;

template <int C>
__global__ void __launch_bounds__(EXPAND_THREADS) k_expand(ExpandArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (uint64_t)blockIdx.x * (EXPAND_THREADS / 32) + threadIdx.x / 32;
    const uint64_t nwarps = (uint64_t)gridDim.x * (EXPAND_THREADS / 32);
    const uint32_t chunks = (a.W + 32 * C - 1) / (32 * C);
    const uint64_t units = a.n * chunks;
    const uint32_t NJ = (a.B + 7) / 8;
    for (uint64_t u = warp; u < units; u += nwarps) {
        const uint64_t q = u / chunks;
        const uint32_t w0 = (uint32_t)(u % chunks) * 32 * C + lane;
        const uint32_t *bm = a.acc + q * a.Gw;
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
            for (uint32_t j = 0; j < NJ; ++j) {
                // byte j of the row: buckets 8j .. 8j+7 at bits lo+8j ..
                const uint32_t bit = lo + 8 * j;
                uint64_t two = __ldg(bm + (bit >> 5));
                if ((bit & 31) > 24 && (bit >> 5) + 1 < a.Gw)
                    two |= (uint64_t)__ldg(bm + (bit >> 5) + 1) << 32;
                uint32_t v = (uint32_t)(two >> (bit & 31)) & 0xffu;
                const uint32_t nb = a.B - 8 * j < 8 ? a.B - 8 * j : 8;
                v &= (1u << nb) - 1u;
                if (!v) continue;
                any = true;
                if (a.tab && (v & (v - 1))) {
                    const uint32_t *row = a.tab + ((uint64_t)(r * NJ + j) * 256 + v) * a.W;
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const uint32_t w = w0 + 32 * c;
                        if (w < a.W) o[c] |= __ldg(row + w);
                    }
                } else {
                    while (v) {
                        const uint32_t b = 8 * j + __ffs(v) - 1;
                        v &= v - 1;
                        const uint32_t *row = a.docbits + (uint64_t)(lo + b) * a.W;
#pragma unroll
                        for (int c = 0; c < C; ++c) {
                            const uint32_t w = w0 + 32 * c;
                            if (w < a.W) o[c] |= __ldg(row + w);
                        }
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

cudaError_t launch_expand(const ExpandArgs &a, int sm_count, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    const uint32_t wc = (a.W + 31) / 32;
    const int C = wc >= 8 ? 8 : wc >= 4 ? 4 : wc >= 2 ? 2 : 1;
    const uint64_t units = a.n * ((a.W + 32 * C - 1) / (32 * C));
    uint64_t blocks = (units + EXPAND_THREADS / 32 - 1) / (EXPAND_THREADS / 32);
    const uint64_t cap = (uint64_t)sm_count * 8;
    if (blocks > cap) blocks = cap;
    switch (C) {
        case 1: k_expand<1><<<(unsigned)blocks, EXPAND_THREADS, 0, s>>>(a); break;
        case 2: k_expand<2><<<(unsigned)blocks, EXPAND_THREADS, 0, s>>>(a); break;
        case 4: k_expand<4><<<(unsigned)blocks, EXPAND_THREADS, 0, s>>>(a); break;
        default: k_expand<8><<<(unsigned)blocks, EXPAND_THREADS, 0, s>>>(a); break;
    }
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

}  // namespace rgpu

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
__device__ __forceinline__ void warp_range(uint64_t T, uint64_t &c0, uint64_t &c1) {
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    uint64_t per = (T + nwarps - 1) / nwarps;
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
    warp_range<STEP>(T, c0, c1);
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
    warp_range<STEP>(T, c0, c1);
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
// expand: one CTA per query (grid-stride).  The passing buckets of each
// repetition are listed in shared memory; output word w of the K-bit mask is
// AND over r of (OR over listed b of DocBits[r][b][w]).  A repetition with no
// passing bucket makes the answer empty.
constexpr int EXPAND_THREADS = 128;

template <bool USE_LIST>
__global__ void __launch_bounds__(EXPAND_THREADS) k_expand(ExpandArgs a) {
    extern __shared__ uint32_t smem[];
    uint32_t *bm = smem;                // Gw words: the query's bucket mask
    uint32_t *cnt = bm + a.Gw;          // R counters
    uint32_t *lst = cnt + a.R;          // R*B bucket lists (USE_LIST)
    const uint32_t RB = a.R * a.B;
    for (uint64_t q = blockIdx.x; q < a.n; q += gridDim.x) {
        for (uint32_t i = threadIdx.x; i < a.Gw; i += blockDim.x) bm[i] = a.acc[q * a.Gw + i];
        for (uint32_t r = threadIdx.x; r < a.R; r += blockDim.x) cnt[r] = 0;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < RB; i += blockDim.x) {
            if ((bm[i >> 5] >> (i & 31)) & 1u) {
                const uint32_t r = i / a.B;
                const uint32_t slot = atomicAdd(&cnt[r], 1u);
                if (USE_LIST) lst[r * a.B + slot] = i - r * a.B;
            }
        }
        __syncthreads();
        bool empty = false;
        for (uint32_t r = 0; r < a.R; ++r) empty |= (cnt[r] == 0);
        uint32_t *out = a.out + q * a.W;
        for (uint32_t w = threadIdx.x; w < a.W; w += blockDim.x) {
            uint32_t res = 0;
            if (!empty) {
                res = FULL;
                for (uint32_t r = 0; r < a.R && res; ++r) {
                    const uint32_t *db = a.docbits + (uint64_t)r * a.B * a.W + w;
                    uint32_t o = 0;
                    if (USE_LIST) {
                        const uint32_t c = cnt[r];
                        for (uint32_t i = 0; i < c; ++i) o |= __ldg(db + (uint64_t)lst[r * a.B + i] * a.W);
                    } else {
                        for (uint32_t b = 0; b < a.B; ++b) {
                            const uint32_t i = r * a.B + b;
                            if ((bm[i >> 5] >> (i & 31)) & 1u) o |= __ldg(db + (uint64_t)b * a.W);
                        }
                    }
                    res &= o;
                }
            }
            out[w] = res;
        }
        __syncthreads();
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
    dim3 grid, block(PROBE_THREADS);
    if (kmers) {
        static int occ = blocks_per_sm(k_probe_kmers<SW, LPG, ETA>, PROBE_THREADS, 0);
        grid = dim3(sm_count * occ, g.chunks);
        k_probe_kmers<SW, LPG, ETA><<<grid, block, 0, s>>>(a);
    } else {
        static int occ = blocks_per_sm(k_probe_seqs<SW, LPG, ETA>, PROBE_THREADS, 0);
        grid = dim3(sm_count * occ, g.chunks);
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
    const size_t list_smem = (size_t)(a.Gw + a.R + (size_t)a.R * a.B) * 4;
    const size_t flat_smem = (size_t)(a.Gw + a.R) * 4;
    const bool use_list = list_smem <= 96 * 1024;
    const size_t smem = use_list ? list_smem : flat_smem;
    if (smem > 48 * 1024) {
        cudaError_t e = use_list ? cudaFuncSetAttribute(k_expand<true>,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)smem)
                                 : cudaFuncSetAttribute(k_expand<false>,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)smem);
        if (e != cudaSuccess) return e;
    }
    uint64_t blocks = (uint64_t)sm_count * 16;
    if (blocks > a.n) blocks = a.n;
    if (use_list) k_expand<true><<<(unsigned)blocks, EXPAND_THREADS, smem, s>>>(a);
    else k_expand<false><<<(unsigned)blocks, EXPAND_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rgpu

// rambo_kernels_probe.cu -- probe kernels of the batched query.
//
//   probe  (Algorithm 2's BFU membership tests, Section 3.3 / 3.3.1): every
//          k-mer of every query is canonicalised and hashed eta times; each
//          probe reads ONE position group -- the bits of all R*B BFUs at that
//          position -- so the per-BFU AND over eta probes and over all k-mers
//          of a query is a plain bitwise AND of groups.  The result per query
//          is its bucket mask: bit r*B+b set iff "Q in BFU(M[b,r])".
#include "rambo_query_common.cuh"

namespace rgpu {
namespace {

// ---------------------------------------------------------------------------
// probe: sequences.
//
// Lane roles.  A position group is read by LPG lanes, each loading an SW-word
// slice (16 bytes when the group is >= 16 bytes), so one warp instruction
// reads 32/LPG whole groups as runs of full 32-byte sectors.  Each warp walks
// a contiguous range of the batch's flattened k-mer index in batches of
// NT tiles of 32 k-mers: first every lane extracts and hashes one k-mer per
// tile (phase 1), then the lanes load the groups of those k-mers four rounds
// at a time (eight for one-lane groups), RIF*ETA independent loads per lane
// in flight (phase 2).  Each lane
// keeps a running AND of its slice for the query it is on and flushes it with
// atomicAnd when its query changes; at the end the warp combines lanes that
// share a query before flushing.
template <int SW, int LPG, int ETA>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_seqs(ProbeArgs a) {
    constexpr int RIF = LPG == 1 ? 8 : 4;  // rounds whose loads are in flight together
    constexpr int NT = LPG >= RIF ? 1 : RIF / LPG;
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
            // phase 2: group loads, RIF rounds in flight, then accumulate
#pragma unroll
            for (int rg = 0; rg < ROUNDS; rg += RIF) {
                Slice<SW> v[RIF][ETA];
                uint32_t qk[RIF];
#pragma unroll
                for (int rr = 0; rr < RIF; ++rr) {
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
                for (int rr = 0; rr < RIF; ++rr) {
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
// the bucket mask is stored directly).  STAGED (one lane per 16-byte group):
// the gathers land in the warp's shared-memory stage through cp.async, so a
// lane holds no load data in flight and the kernel fits beside other work.
constexpr int KMER_RIF1 = 8;  // rounds in flight for one-lane groups
template <int ETA>
constexpr size_t kmer_stage_bytes() { return (size_t)(PROBE_THREADS / 32) * KMER_RIF1 * ETA * 32 * 16; }

template <int SW, int LPG, int ETA, bool STAGED = false>
__global__ void __launch_bounds__(PROBE_THREADS, STAGED ? 3 : 1) k_probe_kmers(ProbeArgs a) {
    static_assert(!STAGED || (LPG == 1 && SW == 4), "staged gathers: one lane per 16-byte group");
    extern __shared__ uint4 kmer_stage[];
    constexpr int RIF = LPG == 1 ? KMER_RIF1 : 4;  // rounds whose loads are in flight together
    constexpr int NT = LPG >= RIF ? 1 : RIF / LPG;
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
            for (int rg = 0; rg < ROUNDS; rg += RIF) {
                if constexpr (STAGED) {
                    // each lane gathers its own k-mers' groups (LPG == 1)
                    uint4 *stage = kmer_stage + (size_t)(threadIdx.x >> 5) * RIF * ETA * 32;
#pragma unroll
                    for (int rr = 0; rr < RIF; ++rr)
                        if (val[rg + rr])
#pragma unroll
                            for (int e = 0; e < ETA; ++e)
                                cp_async16(stage + (rr * ETA + e) * 32 + lane,
                                           a.index + (uint64_t)pos[rg + rr][e] * a.Gw + word0);
                    cp_async_wait_all();
#pragma unroll
                    for (int rr = 0; rr < RIF; ++rr) {
                        if (!val[rg + rr]) continue;
                        const uint64_t g = base + (uint64_t)(rg + rr) * 32 + lane;
                        uint4 x = stage[(rr * ETA) * 32 + lane];
#pragma unroll
                        for (int e = 1; e < ETA; ++e) {
                            const uint4 y = stage[(rr * ETA + e) * 32 + lane];
                            x.x &= y.x;
                            x.y &= y.y;
                            x.z &= y.z;
                            x.w &= y.w;
                        }
                        uint32_t *p = a.acc + g * a.Gw + word0;
                        if (jb == 0) {
                            *reinterpret_cast<uint4 *>(p) = x;
                        } else {
                            atomicAnd(p, x.x);
                            atomicAnd(p + 1, x.y);
                            atomicAnd(p + 2, x.z);
                            atomicAnd(p + 3, x.w);
                        }
                    }
                    continue;
                }
                Slice<SW> v[RIF][ETA];
                bool vs[RIF];
#pragma unroll
                for (int rr = 0; rr < RIF; ++rr) {
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
                for (int rr = 0; rr < RIF; ++rr) {
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

template <int ETA>
cudaError_t launch_kmers_staged(const ProbeArgs &a, const Geometry &g, int sm_count, cudaStream_t s) {
    const size_t smem = kmer_stage_bytes<ETA>();
    cudaError_t e = cudaFuncSetAttribute(k_probe_kmers<4, 1, ETA, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    static int occ = blocks_per_sm(k_probe_kmers<4, 1, ETA, true>, PROBE_THREADS, smem);
    const dim3 grid(sm_count > 0 ? sm_count * occ : -sm_count, g.chunks);
    k_probe_kmers<4, 1, ETA, true><<<grid, PROBE_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int SW, int LPG, int ETA>
cudaError_t launch_probe_t(const ProbeArgs &a, const Geometry &g, int sm_count, cudaStream_t s,
                           bool kmers, bool staged) {
    // sm_count > 0: SMs x occupancy maximum; sm_count < 0: -sm_count CTAs
    if constexpr (SW == 4 && LPG == 1 && ETA <= 2)
        if (kmers && staged) return launch_kmers_staged<ETA>(a, g, sm_count, s);
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
cudaError_t launch_probe_eta(const ProbeArgs &a, const Geometry &g, int sm, cudaStream_t s, bool km,
                             bool st) {
    switch (g.eta) {
        case 1: return launch_probe_t<SW, LPG, 1>(a, g, sm, s, km, st);
        case 2: return launch_probe_t<SW, LPG, 2>(a, g, sm, s, km, st);
        case 3: return launch_probe_t<SW, LPG, 3>(a, g, sm, s, km, st);
        default: return launch_probe_t<SW, LPG, 4>(a, g, sm, s, km, st);
    }
}

cudaError_t launch_probe(const ProbeArgs &a, const Geometry &g, int sm, cudaStream_t s, bool km, bool st) {
    if (g.SW == 1) return launch_probe_eta<1, 1>(a, g, sm, s, km, st);
    if (g.SW == 2) return launch_probe_eta<2, 1>(a, g, sm, s, km, st);
    switch (g.LPG) {
        case 1: return launch_probe_eta<4, 1>(a, g, sm, s, km, st);
        case 2: return launch_probe_eta<4, 2>(a, g, sm, s, km, st);
        case 4: return launch_probe_eta<4, 4>(a, g, sm, s, km, st);
        case 8: return launch_probe_eta<4, 8>(a, g, sm, s, km, st);
        case 16: return launch_probe_eta<4, 16>(a, g, sm, s, km, st);
        case 32: return launch_probe_eta<4, 32>(a, g, sm, s, km, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_probe_seqs(const ProbeArgs &a, const Geometry &g, int sm_count, cudaStream_t s) {
    return launch_probe(a, g, sm_count, s, false, false);
}

cudaError_t launch_probe_kmers(const ProbeArgs &a, const Geometry &g, int sm_count, cudaStream_t s,
                               bool staged) {
    return launch_probe(a, g, sm_count, s, true, staged);
}

}  // namespace rgpu

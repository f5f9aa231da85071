// rambo_kernels_fused.cu -- the persistent fused query (probe and
// expansion in one launch with length-bucketed work queues).
#include "rambo_query_common.cuh"

namespace rgpu {
namespace {

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
// No warp ever waits on another.  With early exit off (the default) every
// k-mer of every query is probed; the answers are the plain path's either way.
constexpr int FUSED_THREADS = 256;

struct FusedArgs {
    ProbeArgs p;                 // index, geometry, batch (kcum unused)
    uint32_t *counters;          // [0] short count [1] short head [2..3] 64-bit tile head
                                 // [4] heavy count
    uint32_t *short_list;        // n
    const uint64_t *tile_prefix; // n+1
    uint32_t *done;              // n (long queries)
    uint32_t *heavy;             // n: queries whose expansion is left to k_fused_heavy
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

// Rounds of loads a lane keeps in flight, and (ASYNC) the shared-memory
// staging a warp needs for them: one 16-byte slot per lane, round and probe.
template <int LPG>
__host__ __device__ constexpr int fused_rif() { return LPG == 1 ? 8 : 4; }
template <int ETA>
__host__ __device__ constexpr size_t fused_stage_bytes() { return (size_t)(FUSED_THREADS / 32) * fused_rif<1>() * ETA * 32 * 16; }

// AND of the groups of k-mers [k0, k1) of one query, per lane slice (every
// lane of the warp works on the same query).  ASYNC (one lane per 16-byte
// group): the gathers land in the warp's shared-memory `stage` through
// cp.async instead of registers, so a lane holds no load data in flight.
template <int SW, int LPG, int ETA, bool ASYNC>
__device__ __forceinline__ Slice<SW> fused_probe_range(const ProbeArgs &a, uint64_t start,
                                                        uint64_t k0, uint64_t k1, int lane,
                                                        uint32_t word0, uint4 *stage) {
    static_assert(!ASYNC || (LPG == 1 && SW == 4), "staged gathers: one lane per 16-byte group");
    constexpr int RIF = fused_rif<LPG>();  // rounds whose loads are in flight together
    constexpr int NT = LPG >= RIF ? 1 : RIF / LPG;
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
            for (int rg = 0; rg < ROUNDS; rg += RIF) {
                if constexpr (ASYNC) {
                    // each lane gathers its own k-mers' groups (LPG == 1)
                    uint32_t live = 0;
#pragma unroll
                    for (int rr = 0; rr < RIF; ++rr) {
                        const int t = rg + rr;
#pragma unroll
                        for (int e = 0; e < ETA; ++e)
                            if (val[t]) {
                                cp_async16(stage + (rr * ETA + e) * 32 + lane,
                                           a.index + (uint64_t)pos[t][e] * a.Gw + word0);
                                live |= 1u << (rr * ETA + e);
                            }
                    }
                    cp_async_wait_all();
#pragma unroll
                    for (int i = 0; i < RIF * ETA; ++i)
                        if (live & (1u << i)) {
                            const uint4 v = stage[i * 32 + lane];
                            accv.w[0] &= v.x;
                            accv.w[1] &= v.y;
                            accv.w[2] &= v.z;
                            accv.w[3] &= v.w;
                        }
                    continue;
                }
                Slice<SW> v[RIF][ETA];
#pragma unroll
                for (int rr = 0; rr < RIF; ++rr) {
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
                for (int rr = 0; rr < RIF; ++rr)
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

template <int SW, int LPG, int ETA, int C, bool ASYNC>
// three resident blocks per SM fit without spills for groups read by 4+
// lanes; one-lane groups keep 16 loads per lane in flight at two (in
// registers) or at three (staged in shared memory)
__global__ void __launch_bounds__(FUSED_THREADS, (LPG >= 4 || ASYNC) ? 3 : 2) k_fused(FusedArgs f) {
    __shared__ uint32_t bm_smem[FUSED_THREADS / 32][128];
    __shared__ uint32_t list_smem[FUSED_THREADS / 32][EXPAND_LIST_MAX];
    extern __shared__ uint4 fused_stage[];  // ASYNC: fused_stage_bytes<ETA>()
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t *bm = bm_smem[wib];
    uint32_t *list = list_smem[wib];
    uint4 *stage = fused_stage + (size_t)wib * fused_rif<1>() * ETA * 32;
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
        }
        if (!skip) {
            // early exit: probe the tile segment by segment; after each, the
            // query's mask so far is this tile's part ANDed with what other
            // tiles have flushed, and an empty repetition row ends the tile
            Slice<SW> s;
            slice_ones(s);
            const uint64_t seg = f.early_exit ? f.segment : (k1 > k0 ? k1 - k0 : 1);
            for (uint64_t a0 = k0; a0 < k1; a0 += seg) {
                const uint64_t a1 = a0 + seg < k1 ? a0 + seg : k1;
                slice_and(s, fused_probe_range<SW, LPG, ETA, ASYNC>(f.p, start, a0, a1, lane, word0, stage));
                if (!f.early_exit) continue;
                if (lane == 0 && f.probed) atomicAdd(f.probed, (unsigned long long)(a1 - a0));
                if (a1 >= k1) break;
                if (sub == 0)
#pragma unroll
                    for (int w = 0; w < SW; ++w)
                        bm[word0 + w] = s.w[w] & __ldcg(f.e.acc + q * f.p.Gw + word0 + w);
                __syncwarp();
                const bool dead = mask_dead(bm, f.p.Gw, f.e.B, f.e.R, lane);
                __syncwarp();
                if (dead) break;
            }
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
            expand_query<C>(f.e, bm, q, chunks, lane, list, f.heavy, f.counters + 4,
                            const_cast<uint32_t *>(f.e.acc));
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
            slice_and(sl, fused_probe_range<SW, LPG, ETA, ASYNC>(f.p, start, k0, k1, lane, word0, stage));
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
        expand_query<C>(f.e, bm, q, chunks, lane, list, f.heavy, f.counters + 4,
                        const_cast<uint32_t *>(f.e.acc));
        __syncwarp();
    }
}

// The heavy queries' answers (more passing buckets than a warp's list
// holds): one warp per (query, chunk of 32*C answer words), grid-stride.
// The warp decodes the query's passing buckets (bucket-space mask in acc)
// into a sorted list of bucket indices r*B + b in its shared memory, then
// ORs the rows of each repetition, several rows in flight, and ANDs the
// repetitions (Algorithm 2's union per repetition and intersection over R).
constexpr int HEAVY_WARPS = 8;

// Indices i = r*B + b of the set bits of bm (bits below R*B), increasing,
// into list; returns how many.  *dead: some repetition has none.
__device__ __forceinline__ uint32_t bucket_list_all(const uint32_t *bm, uint32_t R, uint32_t B, uint16_t *list,
                                                    int lane, bool *dead) {
    const uint32_t RB = R * B;
    const uint32_t nw = (RB + 31) / 32;
    uint32_t total = 0;
    for (uint32_t base = 0; base < nw; base += 32) {
        const uint32_t w = base + lane;
        uint32_t v = w < nw ? __ldg(bm + w) : 0u;
        if (w == nw - 1 && (RB & 31)) v &= (1u << (RB & 31)) - 1u;
        const uint32_t cnt = __popc(v);
        uint32_t incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += o;
        }
        uint32_t at = total + incl - cnt;
        while (v) {
            list[at++] = (uint16_t)(32 * w + __ffs(v) - 1);
            v &= v - 1;
        }
        total += __shfl_sync(FULL, incl, 31);
    }
    __syncwarp();
    // every repetition present?  count the repetition changes along the list
    uint32_t reps = 0;
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
        const uint32_t t = t0 + lane;
        bool first = false;
        if (t < total) first = t == 0 || list[t - 1] / B != list[t] / B;
        reps += __popc(__ballot_sync(FULL, first));
    }
    *dead = reps < R;
    return total;
}

template <int C>
__device__ __forceinline__ void expand_heavy_unit(const ExpandArgs &a, const uint16_t *list, uint32_t n,
                                                  bool dead, uint64_t q, uint32_t w0) {
    constexpr int U = 4;  // rows in flight
    uint32_t res[C], o[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        res[c] = dead ? 0u : FULL;
        o[c] = 0;
    }
    if (!dead && n) {
        uint32_t rep = list[0] / a.B;
        bool empty = false;
        for (uint32_t t0 = 0; t0 < n && !empty; t0 += U) {
            uint32_t idx[U], val[U][C];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                idx[u] = t0 + u < n ? list[t0 + u] : NONE;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t w = w0 + 32 * c;
                    val[u][c] = idx[u] != NONE && w < a.W ? __ldg(a.docbits + (uint64_t)idx[u] * a.W + w) : 0u;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (idx[u] == NONE) break;
                const uint32_t r = idx[u] / a.B;
                if (r != rep) {  // a repetition is complete
                    uint32_t nz = 0;
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        res[c] &= o[c];
                        o[c] = 0;
                        nz |= res[c];
                    }
                    rep = r;
                    if (!__any_sync(FULL, nz)) empty = true;
                }
#pragma unroll
                for (int c = 0; c < C; ++c) o[c] |= val[u][c];
            }
        }
        if (!empty)
#pragma unroll
            for (int c = 0; c < C; ++c) res[c] &= o[c];
        else
#pragma unroll
            for (int c = 0; c < C; ++c) res[c] = 0;
    }
    uint32_t *out = a.out + q * a.W;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const uint32_t w = w0 + 32 * c;
        if (w < a.W) out[w] = res[c];
    }
}

template <int C>
__global__ void __launch_bounds__(HEAVY_WARPS * 32) k_fused_heavy(FusedArgs f) {
    extern __shared__ uint16_t heavy_lists[];  // HEAVY_WARPS x R*B
    const uint32_t count = f.counters[4];
    const uint32_t chunks = (f.e.W + 32 * C - 1) / (32 * C);
    const uint64_t units = (uint64_t)count * chunks;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint16_t *list = heavy_lists + (size_t)wib * f.e.R * f.e.B;
    const uint64_t warp = (uint64_t)blockIdx.x * HEAVY_WARPS + wib;
    const uint64_t nwarps = (uint64_t)gridDim.x * HEAVY_WARPS;
    for (uint64_t u = warp; u < units; u += nwarps) {
        const uint64_t q = f.heavy[u / chunks];
        const uint32_t c = (uint32_t)(u % chunks);
        bool dead = false;
        const uint32_t n = bucket_list_all(f.e.acc + q * f.p.Gw, f.e.R, f.e.B, list, lane, &dead);
        expand_heavy_unit<C>(f.e, list, n, dead, q, c * 32 * C + lane);
        __syncwarp();  // the list is the next unit's
    }
}

}  // namespace

template <int SW, int LPG, int ETA, int C, bool ASYNC>
cudaError_t launch_fused_t(const FusedArgs &f, int grid_override, int sm_count, cudaStream_t s) {
    const size_t smem = ASYNC ? fused_stage_bytes<ETA>() : 0;
    if (ASYNC) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<SW, LPG, ETA, C, ASYNC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    static int occ = blocks_per_sm(k_fused<SW, LPG, ETA, C, ASYNC>, FUSED_THREADS, smem);
    const int grid = grid_override > 0 ? grid_override : sm_count * occ;
    k_fused<SW, LPG, ETA, C, ASYNC><<<grid, FUSED_THREADS, smem, s>>>(f);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t hsmem = (size_t)HEAVY_WARPS * f.e.R * f.e.B * sizeof(uint16_t);
    if (hsmem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_fused_heavy<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem);
        if (e != cudaSuccess) return e;
    }
    k_fused_heavy<C><<<sm_count * 4, HEAVY_WARPS * 32, hsmem, s>>>(f);
    return cudaGetLastError();
}

template <int SW, int LPG, int ETA, bool ASYNC>
cudaError_t launch_fused_c(const FusedArgs &f, int go, int sm, cudaStream_t s) {
    if (f.e.W > 64) return launch_fused_t<SW, LPG, ETA, 4, ASYNC>(f, go, sm, s);
    return launch_fused_t<SW, LPG, ETA, 1, ASYNC>(f, go, sm, s);
}

template <int SW, int LPG>
cudaError_t launch_fused_e(const FusedArgs &f, int go, int sm, cudaStream_t s, bool async) {
    // staged gathers for one lane per 16-byte group and at most two probes a
    // round (the staging of four would take 128 KB per block)
    if constexpr (SW == 4 && LPG == 1) {
        if (async && f.p.eta <= 2) {
            if (f.p.eta == 1) return launch_fused_c<SW, LPG, 1, true>(f, go, sm, s);
            return launch_fused_c<SW, LPG, 2, true>(f, go, sm, s);
        }
    }
    switch (f.p.eta) {
        case 1: return launch_fused_c<SW, LPG, 1, false>(f, go, sm, s);
        case 2: return launch_fused_c<SW, LPG, 2, false>(f, go, sm, s);
        default: return launch_fused_c<SW, LPG, 4, false>(f, go, sm, s);
    }
}

bool fused_supported(const Geometry &g) { return g.chunks == 1 && g.Gw <= 128; }

cudaError_t launch_fused(const ProbeArgs &p, const ExpandArgs &e, const Geometry &g,
                         const FusedQueues &qs, int grid_override, int sm_count, cudaStream_t s) {
    if (!fused_supported(g)) return cudaErrorInvalidValue;
    FusedArgs f{};
    f.p = p;
    f.counters = qs.counters;
    f.short_list = qs.short_list;
    f.tile_prefix = qs.tile_prefix;
    f.done = qs.done;
    f.heavy = qs.heavy;
    f.tile = qs.tile;
    f.short_max = qs.short_max;
    f.user_bases = qs.user_bases;
    f.e = e;
    f.early_exit = qs.early_exit;
    f.segment = qs.segment;
    f.probed = qs.probed;
    cudaError_t err = cudaMemsetAsync(qs.counters, 0, 8 * sizeof(uint32_t), s);
    if (err != cudaSuccess) return err;
    if (p.n == 0) return cudaSuccess;
    k_fused_prep<<<(unsigned)((p.n + 255) / 256), 256, 0, s>>>(f);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const bool as = qs.async != 0;
    if (g.SW == 1) return launch_fused_e<1, 1>(f, grid_override, sm_count, s, as);
    if (g.SW == 2) return launch_fused_e<2, 1>(f, grid_override, sm_count, s, as);
    switch (g.LPG) {
        case 1: return launch_fused_e<4, 1>(f, grid_override, sm_count, s, as);
        case 2: return launch_fused_e<4, 2>(f, grid_override, sm_count, s, as);
        case 4: return launch_fused_e<4, 4>(f, grid_override, sm_count, s, as);
        case 8: return launch_fused_e<4, 8>(f, grid_override, sm_count, s, as);
        case 16: return launch_fused_e<4, 16>(f, grid_override, sm_count, s, as);
        case 32: return launch_fused_e<4, 32>(f, grid_override, sm_count, s, as);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rgpu

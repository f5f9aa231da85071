// rambo_kernels_binned.cu -- region-binned probing of a sequence batch
// (query path 2; the membership tests of Algorithm 2, Section 3.3.1).
//
// The flat and fused probes read one random position group per probe.  With
// groups of at most 16 bytes every probe costs a whole 128-byte DRAM line, and
// over a batch the same line is fetched again and again, because the index is
// far larger than L2.  Here the probes of a batch are first binned by index
// region (a power-of-two number of groups spanning about 32 MiB):
//   scatter  every k-mer is extracted and hashed once; each probe becomes a
//            record (group, query) in its region's bin.  A block stages a
//            tile of records with their ranks in a shared-memory histogram,
//            reserves each bin's run with one atomicAdd on the bin's counter
//            and writes every record to its slot.  A record that finds its
//            bin's share of the workspace full is probed on the spot.
//   chunks   one block turns the bin counts into a prefix of work items.
//   probe    warps take the work items in region order, so at any moment the
//            grid probes inside one or two regions that fit in L2 and each
//            line comes from DRAM about once per batch.
// The per-query result does not depend on the order of the probes (a BFU
// passes a query iff every probe of every k-mer finds its bit, so the bucket
// mask is the AND of all probed groups); records of the same query are ANDed
// within a warp and folded into the query's mask with atomicAnd.
#include "rambo_query_common.cuh"

namespace rgpu {
namespace {

constexpr int BIN_THREADS = 256;
constexpr uint32_t BIN_TILE_RECS = 2048;  // probe records staged per block tile
constexpr uint64_t BIN_MAX = 4096;        // most bins (index regions) per batch

__device__ __forceinline__ uint64_t make_rec(uint32_t pos, uint32_t q) {
    return ((uint64_t)pos << 32) | q;
}

// Exclusive prefix (64-bit) of n values by one block; in place allowed when
// in and out are the same 64-bit array (each thread reads its own segment
// before writing it).  Returns the total to every thread.
template <typename TI>
__device__ uint64_t block_excl_scan(const TI *in, uint64_t *out, uint32_t n) {
    __shared__ uint64_t warp_tot[BIN_THREADS / 32];
    const uint32_t per = (n + BIN_THREADS - 1) / BIN_THREADS;
    const uint32_t b0 = threadIdx.x * per;
    uint64_t sum = 0;
    for (uint32_t i = 0; i < per; ++i)
        if (b0 + i < n) sum += in[b0 + i];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t y = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint64_t v = lane < BIN_THREADS / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint64_t y = __shfl_up_sync(FULL, v, off);
            if (lane >= off) v += y;
        }
        if (lane < BIN_THREADS / 32) warp_tot[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    uint64_t run = (wid ? warp_tot[wid - 1] : 0) + incl - sum;
    const uint64_t total = warp_tot[BIN_THREADS / 32 - 1];
    for (uint32_t i = 0; i < per; ++i) {
        if (b0 + i < n) {
            const uint64_t v = (uint64_t)in[b0 + i];
            out[b0 + i] = run;
            run += v;
        }
    }
    __syncthreads();
    return total;
}

template <int SW>
__global__ void __launch_bounds__(BIN_THREADS) k_bin_scatter(BinnedArgs a) {
    extern __shared__ uint64_t smem64[];
    uint64_t *s_rec = smem64;                                        // BIN_TILE_RECS, tile order
    uint64_t *s_base = s_rec + BIN_TILE_RECS;                        // nb: first slot of the tile's run
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_base + a.nb);  // nb: records per bin
    uint16_t *s_rank = reinterpret_cast<uint16_t *>(s_hist + a.nb);  // BIN_TILE_RECS
    __shared__ uint64_t s_qa[BIN_THREADS], s_qb[BIN_THREADS];

    const ProbeArgs &p = a.p;
    const uint64_t T = p.kcum[p.n];
    const uint32_t kpt = BIN_TILE_RECS / p.eta;  // k-mers per tile
    const uint64_t tiles = (T + kpt - 1) / kpt;
    for (uint32_t b = threadIdx.x; b < a.nb; b += BIN_THREADS) s_hist[b] = 0;
    // this block's tiles are blockIdx.x + i * gridDim.x; their query ranges
    // are looked up BIN_THREADS tiles at a time, one tile per thread
    for (uint64_t i0 = 0; blockIdx.x + i0 * gridDim.x < tiles; i0 += BIN_THREADS) {
        {
            const uint64_t tile = blockIdx.x + (i0 + threadIdx.x) * gridDim.x;
            if (tile < tiles) {
                const uint64_t t0 = tile * kpt, t1 = t0 + kpt < T ? t0 + kpt : T;
                s_qa[threadIdx.x] = find_query(p.kcum, p.n, t0);
                s_qb[threadIdx.x] = find_query(p.kcum, p.n, t1 - 1);
            }
        }
        __syncthreads();
        for (uint32_t i = 0; i < BIN_THREADS; ++i) {
            const uint64_t tile = blockIdx.x + (i0 + i) * gridDim.x;
            if (tile >= tiles) break;
            const uint64_t t0 = tile * kpt;
            const uint64_t t1 = t0 + kpt < T ? t0 + kpt : T;
            const uint64_t qa = s_qa[i], qb = s_qb[i];
            // phase 1: k-mers of the tile -> records; rank within the bin's run
            for (uint64_t g = t0 + threadIdx.x; g < t1; g += BIN_THREADS) {
                uint64_t lo = qa, hi = qb + 1;
                while (hi - lo > 1) {
                    const uint64_t mid = (lo + hi) >> 1;
                    if (p.kcum[mid] <= g) lo = mid;
                    else hi = mid;
                }
                const uint64_t start = p.offsets[lo] + p.base_shift + (g - p.kcum[lo]);
                const uint64_t c = canonical_from_window(base_window(p.packed, p.packed_bytes, start), p.k);
                const uint64_t km = mh_mix_key(c);
                const uint32_t r0 = (uint32_t)(g - t0) * p.eta;
                for (uint32_t j = 0; j < p.eta; ++j) {
                    const uint32_t pos = reduce_pos(mh_first_word(km, p.seed32 + j), p.m, p.m_pow2);
                    s_rec[r0 + j] = make_rec(pos, (uint32_t)lo);
                    s_rank[r0 + j] = (uint16_t)atomicAdd(&s_hist[pos >> a.shift], 1u);
                }
            }
            __syncthreads();
            // phase 2: reserve every bin's run once
            for (uint32_t b = threadIdx.x; b < a.nb; b += BIN_THREADS) {
                const uint32_t cnt = s_hist[b];
                s_base[b] = cnt ? atomicAdd(a.bin_count + b, (unsigned long long)cnt) : 0ull;
            }
            __syncthreads();
            // phase 3: every record to its slot (the bin's share full: probe it now)
            const uint32_t nrec = (uint32_t)(t1 - t0) * p.eta;
            for (uint32_t r = threadIdx.x; r < nrec; r += BIN_THREADS) {
                const uint64_t rec = s_rec[r];
                const uint32_t pos = (uint32_t)(rec >> 32), q = (uint32_t)rec;
                const uint32_t b = pos >> a.shift;
                const uint64_t slot = s_base[b] + s_rank[r];
                if (slot < a.cap) {
                    __stcs(reinterpret_cast<unsigned long long *>(a.records) + (uint64_t)b * a.cap + slot,
                           (unsigned long long)rec);
                } else {
                    const Slice<SW> v = ld_slice<SW>(p.index + (uint64_t)pos * p.Gw);
                    flush_slice<SW>(p.acc, q, p.Gw, 0, v);
                }
            }
            for (uint32_t b = threadIdx.x; b < a.nb; b += BIN_THREADS) s_hist[b] = 0;
            __syncthreads();
        }
    }
}

// One block: chunk_pre[b] = exclusive prefix over bins of their work items,
// chunk_pre[nb] = total.
__global__ void __launch_bounds__(BIN_THREADS) k_bin_chunks(BinnedArgs a) {
    const uint32_t chunk = 32u * a.rows;
    for (uint32_t b = threadIdx.x; b < a.nb; b += BIN_THREADS) {
        const uint64_t cnt = a.bin_count[b] < a.cap ? a.bin_count[b] : a.cap;
        a.chunk_pre[b] = (cnt + chunk - 1) / chunk;
    }
    __syncthreads();
    const uint64_t total = block_excl_scan(a.chunk_pre, a.chunk_pre, a.nb);
    if (threadIdx.x == 0) a.chunk_pre[a.nb] = total;
}

// U rows of 32 records per warp work item; the grid's work items in flight
// span U * 32 * (warps) records, which should stay within about one region.
template <int SW, int BIN_U>
__global__ void __launch_bounds__(BIN_THREADS) k_bin_probe(BinnedArgs a) {
    constexpr uint32_t BIN_CHUNK = 32u * BIN_U;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (uint64_t)blockIdx.x * (BIN_THREADS / 32) + (threadIdx.x >> 5);
    const uint64_t nwarps = (uint64_t)gridDim.x * (BIN_THREADS / 32);
    const uint64_t total = a.chunk_pre[a.nb];
    const uint32_t Gw = a.p.Gw;
    for (uint64_t c = warp; c < total; c += nwarps) {
        // bin holding work item c: largest b with chunk_pre[b] <= c
        uint32_t lo = 0, hi = a.nb;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.chunk_pre[mid] <= c) lo = mid;
            else hi = mid;
        }
        const uint64_t cnt = a.bin_count[lo] < a.cap ? a.bin_count[lo] : a.cap;
        const uint64_t off = (c - a.chunk_pre[lo]) * BIN_CHUNK;
        const unsigned long long *rec =
            reinterpret_cast<const unsigned long long *>(a.records) + (uint64_t)lo * a.cap;
        uint64_t r[BIN_U];
#pragma unroll
        for (int u = 0; u < BIN_U; ++u) {
            const uint64_t i = off + (uint64_t)u * 32 + lane;
            r[u] = i < cnt ? __ldcs(rec + i) : ~0ull;
        }
        Slice<SW> v[BIN_U];
#pragma unroll
        for (int u = 0; u < BIN_U; ++u) {
            if (r[u] != ~0ull) v[u] = ld_slice<SW>(a.p.index + (r[u] >> 32) * Gw);
            else slice_ones(v[u]);
        }
        // AND the records of each query present in a row, one atomic per word
#pragma unroll
        for (int u = 0; u < BIN_U; ++u) {
            const uint32_t q = r[u] != ~0ull ? (uint32_t)r[u] : NONE;
            uint32_t todo = __ballot_sync(FULL, q != NONE);
            while (todo) {
                const int l = __ffs(todo) - 1;
                const uint32_t qq = __shfl_sync(FULL, q, l);
                const bool mine = q == qq;
                todo &= ~__ballot_sync(FULL, mine);
#pragma unroll
                for (int w = 0; w < SW; ++w) {
                    const uint32_t x = __reduce_and_sync(FULL, mine ? v[u].w[w] : FULL);
                    if (lane == l && x != FULL) atomicAnd(a.p.acc + (uint64_t)qq * Gw + w, x);
                }
            }
        }
    }
}

size_t scatter_smem(uint32_t nb) {
    return (size_t)BIN_TILE_RECS * 8 + (size_t)nb * (8 + 4) + (size_t)BIN_TILE_RECS * 2;
}

template <int SW>
cudaError_t launch_binned_t(const BinnedArgs &a, int sm_count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.bin_count, 0, (size_t)a.nb * 8, s);
    if (e != cudaSuccess) return e;
    const size_t smem = scatter_smem(a.nb);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_bin_scatter<SW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int occ = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bin_scatter<SW>, BIN_THREADS, smem);
    if (e != cudaSuccess) return e;
    k_bin_scatter<SW><<<(occ > 0 ? occ : 1) * sm_count, BIN_THREADS, smem, s>>>(a);
    k_bin_chunks<<<1, BIN_THREADS, 0, s>>>(a);
    int occ_p = 1;
#define RGPU_BIN_PROBE(U)                                                                          \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, k_bin_probe<SW, U>, BIN_THREADS, 0); \
    if (e != cudaSuccess) return e;                                                                \
    k_bin_probe<SW, U><<<(occ_p > 0 ? occ_p : 1) * sm_count, BIN_THREADS, 0, s>>>(a);
    switch (a.rows) {
        case 1: RGPU_BIN_PROBE(1) break;
        case 2: RGPU_BIN_PROBE(2) break;
        case 4: RGPU_BIN_PROBE(4) break;
        default: RGPU_BIN_PROBE(8) break;
    }
#undef RGPU_BIN_PROBE
    return cudaGetLastError();
}

}  // namespace

bool binned_supported(const Geometry &g) { return g.LPG == 1 && (g.Gw == 1 || g.Gw == 2 || g.Gw == 4); }

uint32_t binned_bins(const Geometry &g, uint64_t region_bytes, uint32_t *shift) {
    uint64_t region_groups = region_bytes / ((uint64_t)g.Gw * 4);
    if (region_groups == 0) region_groups = 1;
    uint32_t sh = 0;
    while ((1ull << (sh + 1)) <= region_groups) ++sh;
    // at most BIN_MAX bins (the scatter's shared-memory histogram)
    while (((g.m + (1ull << sh) - 1) >> sh) > BIN_MAX) ++sh;
    *shift = sh;
    return (uint32_t)((g.m + (1ull << sh) - 1) >> sh);
}

int binned_launches() { return 3; }

cudaError_t launch_binned(const BinnedArgs &a, const Geometry &g, int sm_count, cudaStream_t s) {
    switch (g.Gw) {
        case 1: return launch_binned_t<1>(a, sm_count, s);
        case 2: return launch_binned_t<2>(a, sm_count, s);
        default: return launch_binned_t<4>(a, sm_count, s);
    }
}

}  // namespace rgpu

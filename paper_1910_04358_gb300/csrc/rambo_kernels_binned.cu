// rambo_kernels_binned.cu -- region-binned probing of a sequence batch
// (query path 2; the membership tests of Algorithm 2, Section 3.3.1).
//
// The flat and fused probes read one random position group per probe.  A
// random read of at most 128 bytes costs a whole 128-byte DRAM line, and over
// a batch the same line is fetched again and again, because the index is far
// larger than L2: with 16-byte groups a probe uses an eighth of the line it
// pays for, with 64-byte groups half of it.  Here the probes of a batch are
// first binned by index region (a power-of-two number of groups spanning a
// few tens of MiB), then probed region by region:
//   scatter  a block takes one tile at a time: up to `tile` consecutive
//            k-mers of ONE query (the tile prefix numbers every query's
//            tiles).  Its threads extract and hash the k-mers and append
//            every probe as a record (group, query) to the block's own
//            sub-bin of the probe's region, the slot taken from a per-block
//            cursor in shared memory: no global atomics, and the records a
//            tile adds to a sub-bin are one run of one query.  A record that
//            finds its sub-bin full is probed on the spot.
//   probe    work items are fixed chunks of sub-bins, claimed in
//            region-major order from a counter, so at any moment the grid
//            probes inside about one region that fits in L2, and each line
//            comes from DRAM about once per batch.  The lanes that read one
//            group walk a run of consecutive records, ANDing the groups of a
//            query's run in registers with the next gathers in flight; a
//            closed run is folded into its query's mask by one coalesced
//            atomicAnd per mask row.
// The per-query result does not depend on the order of the probes (a BFU
// passes a query iff every probe of every k-mer finds its bit, so the bucket
// mask is the AND of all probed groups), and neither does the sub-bin layout.
#include "rambo_query_common.cuh"

namespace rgpu {
namespace {

constexpr int SCATTER_THREADS = 512;
constexpr uint64_t BIN_MAX = 4096;   // most bins (index regions) per batch

__device__ __forceinline__ uint64_t make_rec(uint32_t pos, uint32_t q) {
    return ((uint64_t)pos << 32) | q;
}

// A probe whose sub-bin is full: its group ANDed into the query's mask directly.
template <int SW>
__device__ __forceinline__ void probe_direct(const ProbeArgs &p, uint32_t pos, uint32_t q) {
    for (uint32_t w = 0; w < p.Gw; w += SW) {
        const Slice<SW> v = ld_slice<SW>(p.index + (uint64_t)pos * p.Gw + w);
        flush_slice<SW>(p.acc, q, p.Gw, w, v);
    }
}

// tile_q[t] = the query whose k-mers tile t covers (one thread per query),
// for the first max_tiles tiles (ranges may overlap, so a batch can have
// more tiles than its packed bytes suggest; those are looked up by search).
// Also zeroes the probe pass's work-item counter (the pass launches after).
__global__ void k_bin_tiles(BinnedArgs a) {
    const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0 && a.item_ctr) *a.item_ctr = 0ull;
    if (q >= a.p.n) return;
    const uint64_t t1 = a.p.kcum[q + 1] < a.max_tiles ? a.p.kcum[q + 1] : a.max_tiles;
    for (uint64_t t = a.p.kcum[q]; t < t1; ++t) a.tile_q[t] = (uint32_t)q;
}

// First k-mer, end and start base of tile t.
struct TileHead {
    uint64_t k0, k1, start;
    uint32_t q;
};
__device__ __forceinline__ TileHead tile_head(const BinnedArgs &a, uint64_t t) {
    const ProbeArgs &p = a.p;
    TileHead h;
    h.q = t < a.max_tiles ? a.tile_q[t] : (uint32_t)find_query(p.kcum, p.n, t);
    const uint64_t b0 = p.offsets[h.q], b1 = p.ends[h.q];
    const uint64_t nk = b1 - b0 - p.k + 1;  // the prefix counted only items with k-mers
    h.k0 = (t - p.kcum[h.q]) * a.tile;
    h.k1 = h.k0 + a.tile < nk ? h.k0 + a.tile : nk;
    h.start = b0 + p.base_shift;
    return h;
}

// Exclusive prefix of n 32-bit counts in shared memory, in place, by the
// whole block (n up to a few thousand); every thread returns after the
// prefix is written.
__device__ void block_scan_counts(uint32_t *v, uint32_t n) {
    __shared__ uint32_t warp_tot[SCATTER_THREADS / 32];
    const uint32_t per = (n + SCATTER_THREADS - 1) / SCATTER_THREADS;
    const uint32_t b0 = threadIdx.x * per;
    uint32_t sum = 0;
    for (uint32_t i = 0; i < per; ++i)
        if (b0 + i < n) sum += v[b0 + i];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t x = lane < SCATTER_THREADS / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, off);
            if (lane >= off) x += y;
        }
        if (lane < SCATTER_THREADS / 32) warp_tot[lane] = x;
    }
    __syncthreads();
    uint32_t run = (wid ? warp_tot[wid - 1] : 0) + incl - sum;
    for (uint32_t i = 0; i < per; ++i) {
        if (b0 + i < n) {
            const uint32_t x = v[b0 + i];
            v[b0 + i] = run;
            run += x;
        }
    }
}

__host__ __device__ inline size_t scatter_smem(uint32_t nb, uint32_t tile_recs) {
    // per bin: two count / offset arrays (alternate tiles), sub-bin cursor,
    // cursor before the tile; per record: group, group in bin order, rank
    return (size_t)nb * 16 + (size_t)tile_recs * 10;
}

// Scatter.  Sub-bin (b, blk) of the records is b * G + blk.  Per tile:
//   1  extract and hash the k-mers; count the tile's probes per bin (rank)
//   2  prefix of the counts = the tile's records in bin order; the block's
//      sub-bin cursors advance by the counts
//   3  the records in bin order in shared memory
//   4  written out in that order, so the lanes of a warp store a few whole
//      runs (consecutive slots of one sub-bin) instead of 32 scattered
//      records; the other count array is cleared for the next tile
template <int SW>
__global__ void __launch_bounds__(SCATTER_THREADS) k_bin_scatter(BinnedArgs a) {
    extern __shared__ uint32_t smem32[];
    uint32_t *s_cnt2 = smem32;                       // 2 x nb: tile counts, then tile offsets
    uint32_t *s_cursor = s_cnt2 + 2 * a.nb;          // nb: the block's records per sub-bin
    uint32_t *s_gbase = s_cursor + a.nb;             // nb: cursor before this tile
    const uint32_t TR = a.tile * a.p.eta;
    uint32_t *s_pos = s_gbase + a.nb;                // TR
    uint32_t *s_sorted = s_pos + TR;                 // TR
    uint16_t *s_rank = reinterpret_cast<uint16_t *>(s_sorted + TR);  // TR
    __shared__ TileHead s_head[2];
    const ProbeArgs &p = a.p;
    const uint64_t tiles = p.kcum[p.n];  // the tile prefix
    for (uint32_t b = threadIdx.x; b < 2 * a.nb; b += SCATTER_THREADS) s_cnt2[b] = 0;
    for (uint32_t b = threadIdx.x; b < a.nb; b += SCATTER_THREADS) s_cursor[b] = 0;
    if (threadIdx.x == 0 && blockIdx.x < tiles) s_head[0] = tile_head(a, blockIdx.x);
    __syncthreads();
    unsigned long long *rec = reinterpret_cast<unsigned long long *>(a.records);
    uint32_t parity = 0;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x, parity ^= 1u) {
        uint32_t *s_cnt = s_cnt2 + parity * a.nb;
        uint32_t *s_other = s_cnt2 + (parity ^ 1u) * a.nb;
        const TileHead h = s_head[parity];
        TileHead nxt{};
        const bool has_next = t + gridDim.x < tiles;
        if (threadIdx.x == 0 && has_next) nxt = tile_head(a, t + gridDim.x);  // in flight during 1
        // 1
        for (uint64_t g = h.k0 + threadIdx.x; g < h.k1; g += SCATTER_THREADS) {
            const uint64_t c = canonical_from_window(base_window(p.packed, p.packed_bytes, h.start + g), p.k);
            const uint64_t km = mh_mix_key(c);
            const uint32_t r0 = (uint32_t)(g - h.k0) * p.eta;
            for (uint32_t j = 0; j < p.eta; ++j) {
                const uint32_t pos = reduce_pos(mh_first_word(km, p.seed32 + j), p.m, p.m_pow2);
                s_pos[r0 + j] = pos;
                s_rank[r0 + j] = (uint16_t)atomicAdd(&s_cnt[pos >> a.shift], 1u);
            }
        }
        if (threadIdx.x == 0 && has_next) s_head[parity ^ 1u] = nxt;
        __syncthreads();
        // 2
        for (uint32_t b = threadIdx.x; b < a.nb; b += SCATTER_THREADS) {
            s_gbase[b] = s_cursor[b];
            s_cursor[b] += s_cnt[b];
        }
        block_scan_counts(s_cnt, a.nb);
        __syncthreads();
        // 3
        const uint32_t nrec = (uint32_t)(h.k1 - h.k0) * p.eta;
        for (uint32_t r = threadIdx.x; r < nrec; r += SCATTER_THREADS) {
            const uint32_t pos = s_pos[r];
            s_sorted[s_cnt[pos >> a.shift] + s_rank[r]] = pos;
        }
        __syncthreads();
        // 4
        for (uint32_t i = threadIdx.x; i < nrec; i += SCATTER_THREADS) {
            const uint32_t pos = s_sorted[i];
            const uint32_t b = pos >> a.shift;
            const uint32_t slot = s_gbase[b] + (i - s_cnt[b]);
            if (slot < a.cap)
                __stcs(rec + ((uint64_t)b * gridDim.x + blockIdx.x) * a.cap + slot,
                       (unsigned long long)make_rec(pos, h.q));
            else
                probe_direct<SW>(p, pos, h.q);
        }
        for (uint32_t b = threadIdx.x; b < a.nb; b += SCATTER_THREADS) s_other[b] = 0;
        __syncthreads();
    }
    for (uint32_t b = threadIdx.x; b < a.nb; b += SCATTER_THREADS)
        a.sub_count[(uint64_t)b * gridDim.x + blockIdx.x] = s_cursor[b] < a.cap ? s_cursor[b] : (uint32_t)a.cap;
}

// ANDs a run's slice into the query's bucket mask: 64-bit atomics for
// 16-byte slices (the mask rows are 8-byte aligned), all-ones words skipped.
// The L lanes of a group flush its L slices in one instruction: a coalesced
// reduction over the query's whole mask row.
template <int SW>
__device__ __forceinline__ void flush_run(uint32_t *acc, uint32_t q, uint32_t Gw, uint32_t word0,
                                          const Slice<SW> &v) {
    if constexpr (SW == 4) {
        unsigned long long *p = reinterpret_cast<unsigned long long *>(acc + (uint64_t)q * Gw + word0);
        const unsigned long long lo = ((unsigned long long)v.w[1] << 32) | v.w[0];
        const unsigned long long hi = ((unsigned long long)v.w[3] << 32) | v.w[2];
        if (lo != ~0ull) atomicAnd(p, lo);
        if (hi != ~0ull) atomicAnd(p + 1, hi);
    } else {
        flush_slice<SW>(acc, q, Gw, word0, v);
    }
}

// Probe pass.  A group of GW words is
// read by SL lanes, one 16-byte slice each (one lane holding the whole group
// under 16 bytes), so a warp runs NS = 32 / SL streams side by side.  A work
// item (BINNED_ITEM_RECS consecutive records of one sub-bin) is handed out in
// parts of NS runs of PS consecutive records, one per stream; a stream walks its records
// in order with the gathers of the next D records in flight in registers,
// keeps the AND of the current run (records of one query) in registers, and
// folds a closed run into its query's mask with one coalesced atomicAnd per
// mask row.  One warp load instruction therefore reads NS whole groups (NS
// lines), not 32 scattered slices.  The item's records are copied into the
// warp's shared memory by coalesced cp.async (evict-first in L2: they are
// read once), one part ahead; parts are claimed from a counter in
// region-major order, so the warps in flight stay within about one region
// and the lines a region's probes share come from L2.
constexpr int STREAM_WARPS = 8;
// Records a lane group walks per part.  Parts of 16 records (8 x 16 per warp
// for 64-byte groups) keep the records in flight to about a quarter of what
// whole 512-record items held, so more of a region's reuse stays within L2:
// 12.9 ms against 15.8 ms for the 32 GiB batch.
constexpr int BIN_PART_RECS = 16;

template <int GW>
struct StreamShape {
    static constexpr int SL = GW >= 4 ? GW / 4 : 1;     // lanes per group
    static constexpr int SW = GW >= 4 ? 4 : GW;         // words per lane
    static constexpr int NS = 32 / SL;                  // streams per warp
    static constexpr int PS0 = (int)BINNED_ITEM_RECS / NS;
    static constexpr int PS = PS0 < BIN_PART_RECS ? PS0 : BIN_PART_RECS;  // records per stream and part
    static constexpr int SUB = NS * PS;                 // records per part
    static constexpr int SPLIT = (int)BINNED_ITEM_RECS / SUB;  // parts per work item
    static constexpr int STRIDE = PS * 8 + 16;          // bytes per stream row (bank offset)
    static constexpr int BUF = NS * STRIDE;             // bytes per part buffer
};

template <int GW>
__host__ __device__ constexpr size_t stream_smem() {
    return (size_t)STREAM_WARPS * 2 * StreamShape<GW>::BUF;
}

// Copies the valid records of item (sb, chunk0) into buf (stream-major rows),
// 16 bytes (two records) per copy; commits one cp.async group either way.
template <int GW>
__device__ __forceinline__ void stage_item(unsigned char *buf, const unsigned long long *rec,
                                           uint32_t valid, int lane, uint64_t policy) {
    using S = StreamShape<GW>;
    const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(buf);
#pragma unroll
    for (int j = 0; j < S::SUB / 64; ++j) {
        const uint32_t t = (uint32_t)(j * 32 + lane);  // record pair
        if (2 * t < valid) {
            const uint32_t g = t / (S::PS / 2), i = 2 * (t % (S::PS / 2));
            asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(
                             d0 + g * S::STRIDE + i * 8),
                         "l"(rec + 2 * t), "l"(policy)
                         : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int GW, int D>
__global__ void __launch_bounds__(STREAM_WARPS * 32) k_bin_probe(BinnedArgs a) {
    using S = StreamShape<GW>;
    constexpr int SW = S::SW;
    extern __shared__ __align__(16) unsigned char stream_smem_u8[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int grp = lane / S::SL;
    const uint32_t word0 = (uint32_t)(lane % S::SL) * SW;
    unsigned char *bufs = stream_smem_u8 + (size_t)wib * 2 * S::BUF;
    // the counter hands out parts (SPLIT per work item), in region-major order
    const uint64_t items = (uint64_t)a.nb * a.G * a.cps * S::SPLIT;
    uint32_t *acc = a.p.acc;
    const uint32_t *index = a.p.index;
    const unsigned long long *records = reinterpret_cast<const unsigned long long *>(a.records);
    uint64_t policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    // part c: sub-bin sb, records [chunk0, chunk0 + SUB) of it, `valid` of them present
    auto item_at = [&](uint64_t c, uint64_t &sb, uint32_t &chunk0, uint32_t &valid) {
        const uint64_t it = c / S::SPLIT;
        sb = it / a.cps;
        chunk0 = (uint32_t)(it - sb * a.cps) * BINNED_ITEM_RECS + (uint32_t)(c % S::SPLIT) * S::SUB;
        const uint32_t cnt = a.sub_count[sb];
        valid = chunk0 < cnt ? (cnt - chunk0 < (uint32_t)S::SUB ? cnt - chunk0 : (uint32_t)S::SUB) : 0u;
    };
    uint64_t cur = 0;
    if (lane == 0) cur = atomicAdd(a.item_ctr, 1ull);
    cur = __shfl_sync(FULL, cur, 0);
    uint64_t sb;
    uint32_t chunk0, valid;
    if (cur < items) {
        item_at(cur, sb, chunk0, valid);
        stage_item<GW>(bufs, records + sb * a.cap + chunk0, valid, lane, policy);
    }
    int p = 0;
    while (cur < items) {
        uint64_t nxt = 0;
        if (lane == 0) nxt = atomicAdd(a.item_ctr, 1ull);
        nxt = __shfl_sync(FULL, nxt, 0);
        uint64_t nsb = 0;
        uint32_t nchunk0 = 0, nvalid = 0;
        if (nxt < items) {
            item_at(nxt, nsb, nchunk0, nvalid);
            stage_item<GW>(bufs + (p ^ 1) * S::BUF, records + nsb * a.cap + nchunk0, nvalid, lane, policy);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncwarp();
        // this stream's records of the item: ng of them, in row grp of the buffer
        const int first = grp * S::PS;
        const int ng = (int)valid > first ? ((int)valid - first < S::PS ? (int)valid - first : S::PS) : 0;
        const unsigned long long *row =
            reinterpret_cast<const unsigned long long *>(bufs + p * S::BUF + grp * S::STRIDE);
        Slice<SW> buf[D];
        uint32_t qq[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if (d < ng) {
                const unsigned long long x = row[d];
                qq[d] = (uint32_t)x;
                buf[d] = ld_slice<SW>(index + (x >> 32) * GW + word0);
            }
        }
        uint32_t cq = NONE;
        Slice<SW> run;
        slice_ones(run);
#pragma unroll 1
        for (int i0 = 0; i0 < ng; i0 += D) {
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int i = i0 + d;
                if (i < ng) {
                    const uint32_t q = qq[d];
                    if (q != cq) {
                        if (cq != NONE) flush_run<SW>(acc, cq, GW, word0, run);
                        cq = q;
                        slice_ones(run);
                    }
                    slice_and(run, buf[d]);
                    if (i + D < ng) {
                        const unsigned long long y = row[i + D];
                        qq[d] = (uint32_t)y;
                        buf[d] = ld_slice<SW>(index + (y >> 32) * GW + word0);
                    }
                }
            }
        }
        if (cq != NONE) flush_run<SW>(acc, cq, GW, word0, run);
        __syncwarp();  // every lane is done with this buffer before it is refilled
        cur = nxt;
        sb = nsb;
        chunk0 = nchunk0;
        valid = nvalid;
        p ^= 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <int GW, int D>
cudaError_t launch_streams_d(const BinnedArgs &a, int sm_count, cudaStream_t s) {
    constexpr size_t smem = stream_smem<GW>();
    cudaError_t e = cudaFuncSetAttribute(k_bin_probe<GW, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bin_probe<GW, D>, STREAM_WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    k_bin_probe<GW, D><<<(occ > 0 ? occ : 1) * sm_count, STREAM_WARPS * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int GW>
cudaError_t launch_probe_pass(const BinnedArgs &a, int sm_count, cudaStream_t s) {
    switch (a.depth) {
        case 2: return launch_streams_d<GW, 4>(a, sm_count, s);
        case 4: return launch_streams_d<GW, 8>(a, sm_count, s);
        default: return launch_streams_d<GW, 12>(a, sm_count, s);
    }
}

template <int SW>
int scatter_blocks_per_sm(size_t smem) {
    // (always set: the kernel's static shared memory counts against the
    // default 48 KB too)
    if (cudaFuncSetAttribute(k_bin_scatter<SW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 1;
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bin_scatter<SW>, SCATTER_THREADS, smem) !=
            cudaSuccess || occ < 1)
        occ = 1;
    return occ;
}

}  // namespace

bool binned_supported(const Geometry &g) { return g.Gw == 1 || g.Gw == 2 || g.Gw == 4 || g.Gw == 8 || g.Gw == 16; }

uint32_t binned_records_per_item() { return BINNED_ITEM_RECS; }

uint32_t binned_depth(uint32_t rows) { return rows == 1 ? 2u : (rows == 0 || rows == 2) ? 4u : 8u; }

uint32_t binned_tile_kmers(const Geometry &g) {
    const uint32_t t = BINNED_TILE_RECS / (g.eta ? g.eta : 1);
    return t ? t : 1;
}

uint64_t binned_max_tiles(const Geometry &g, uint64_t n, uint64_t packed_bytes) {
    // every query with k-mers has ceil(k-mers / tile) tiles, and its k-mers
    // are at most its bases (queries' ranges may overlap: see k_bin_tiles)
    return n + 4 * packed_bytes / binned_tile_kmers(g) + 1;
}

uint32_t binned_scatter_grid(const Geometry &g, uint32_t nb, int sm_count) {
    const size_t smem = scatter_smem(nb, binned_tile_kmers(g) * g.eta);
    const int occ = g.SW == 1 ? scatter_blocks_per_sm<1>(smem)
                              : g.SW == 2 ? scatter_blocks_per_sm<2>(smem) : scatter_blocks_per_sm<4>(smem);
    return (uint32_t)(occ * sm_count);
}

uint32_t binned_bins(const Geometry &g, uint64_t region_bytes, uint32_t *shift) {
    uint64_t region_groups = region_bytes / ((uint64_t)g.Gw * 4);
    if (region_groups == 0) region_groups = 1;
    uint32_t sh = 0;
    while ((1ull << (sh + 1)) <= region_groups) ++sh;
    // at most BIN_MAX bins (the scatter's shared-memory cursors)
    while (((g.m + (1ull << sh) - 1) >> sh) > BIN_MAX) ++sh;
    *shift = sh;
    return (uint32_t)((g.m + (1ull << sh) - 1) >> sh);
}

int binned_launches() { return 3; }

cudaError_t launch_binned(const BinnedArgs &a, const Geometry &g, int sm_count, cudaStream_t s) {
    if (!binned_supported(g) || a.tile == 0 || (uint64_t)a.tile * a.p.eta > BINNED_TILE_RECS ||
        a.nb == 0 || a.nb > BIN_MAX || a.G == 0 || (a.cap & 1) ||
        (a.depth != 2 && a.depth != 4 && a.depth != 8) ||
        a.cps != (uint32_t)((a.cap + BINNED_ITEM_RECS - 1) / BINNED_ITEM_RECS) || a.item_ctr == nullptr)
        return cudaErrorInvalidValue;
    if (a.p.n == 0) return cudaSuccess;
    k_bin_tiles<<<(unsigned)((a.p.n + 255) / 256), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = scatter_smem(a.nb, a.tile * a.p.eta);
    switch (g.SW) {
        case 1: scatter_blocks_per_sm<1>(smem); k_bin_scatter<1><<<a.G, SCATTER_THREADS, smem, s>>>(a); break;
        case 2: scatter_blocks_per_sm<2>(smem); k_bin_scatter<2><<<a.G, SCATTER_THREADS, smem, s>>>(a); break;
        default: scatter_blocks_per_sm<4>(smem); k_bin_scatter<4><<<a.G, SCATTER_THREADS, smem, s>>>(a); break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    switch (g.Gw) {
        case 1: return launch_probe_pass<1>(a, sm_count, s);
        case 2: return launch_probe_pass<2>(a, sm_count, s);
        case 4: return launch_probe_pass<4>(a, sm_count, s);
        case 8: return launch_probe_pass<8>(a, sm_count, s);
        default: return launch_probe_pass<16>(a, sm_count, s);
    }
}

}  // namespace rgpu

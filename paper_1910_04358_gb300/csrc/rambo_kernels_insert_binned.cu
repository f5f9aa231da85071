// rambo_kernels_insert_binned.cu -- Algorithm 1's bit setting, binned by
// index region so that its atomics hit L2.
//
// The direct insert ORs every probe's bits into a random line of the index:
// once the index outgrows L2, nearly every atomic misses and costs a DRAM
// read and write of the line.  Here a chunk of the batch's k-mers goes
// through two passes:
//   scatter  every probe (k-mer x, document d, position h_j(x)) becomes one
//            8-byte record (h_j(x), d) appended to the bin of its index
//            region; a CTA stages a tile of 4096 records in shared memory,
//            counts them per bin, reserves each bin's share with one global
//            atomicAdd and writes them out;
//   apply    a persistent grid claims units of records in bin order, so all
//            CTAs work inside one or two regions at a time and the regions
//            stay in L2 while their records set bit r*B + phi_r(d) of group
//            h_j(x) for every r (repetitions sharing a 64-bit word merged
//            into one atomicOr, as the direct insert does).
// Records past a bin's capacity set their bits during the scatter pass.  OR
// is commutative and idempotent, so the index is bit-identical to the
// direct insert's whatever the order.
#include "rambo_insert_binned.cuh"

namespace rgpu {
namespace {

constexpr int IB_THREADS = 256;
constexpr uint32_t IB_UNIT = 2048;  // records per unit of the apply pass
constexpr uint32_t NO_RANK = 0xffffffffu;

// Sets the bits of one record: bit r*B + phi_r(d) of position group p for
// every repetition r; `wide` merges repetitions that share a 64-bit word.
__device__ __forceinline__ void or_record(const InsertArgs &a, uint64_t p, uint32_t d, bool wide) {
    const uint64_t gbit = p * a.Gw * 32;  // first bit of the group
    if (wide) {
        unsigned long long *idx64 = reinterpret_cast<unsigned long long *>(a.index);
        uint64_t cur = ~0ULL, bits = 0;
        for (uint32_t r = 0; r < a.R; ++r) {
            const uint64_t bb = gbit + r * a.B + __ldg(a.phi + (uint64_t)d * a.R + r);
            if ((bb >> 6) != cur) {
                if (bits) atomicOr(idx64 + cur, (unsigned long long)bits);
                cur = bb >> 6;
                bits = 0;
            }
            bits |= 1ull << (bb & 63);
        }
        if (bits) atomicOr(idx64 + cur, (unsigned long long)bits);
    } else {
        for (uint32_t r = 0; r < a.R; ++r) {
            const uint64_t bb = gbit + r * a.B + __ldg(a.phi + (uint64_t)d * a.R + r);
            atomicOr(a.index + (bb >> 5), 1u << (bb & 31));
        }
    }
}

// Scatter pass over [f0, f1) of the flat k-mer index: each CTA takes a
// contiguous range in tiles of IB_TILE_RECORDS / ETA k-mers (every thread a
// strided share), up to ETA probes of each per pass over the hash seeds.  A
// tile's records are staged in shared memory with their bins and ranks, so
// that a bin's share is reserved with one global atomic per tile even when
// there are many bins.  The records are then written in bin order (a
// counting sort of the tile in shared memory), so that a warp's store covers
// a few runs of consecutive slots instead of 32 scattered records.
constexpr uint32_t IB_TILE_RECORDS = 4096;

// Bins from which a tile is written in bin order: with few bins a warp's
// slot-order stores already fall in few runs, and the sorted copy's shared
// memory would cost the scatter a CTA per SM (medium build, 16 bins: 42.2
// against 36.7 ms; large, 512 bins: 346 against 489 ms).
constexpr uint32_t IB_SORT_MIN_BINS = 64;

// s_rec (8 bytes a record), s_bin, s_rank (4 each), s_sorted (8, SORTED
// only); s_cnt, s_base (4 a bin), s_pre (4, SORTED only)
template <bool SORTED>
constexpr size_t scatter_smem() {
    return (size_t)IB_TILE_RECORDS * (8 + 4 + 4 + (SORTED ? 8 : 0)) + (size_t)IB_MAX_BINS * (4 + 4 + (SORTED ? 4 : 0));
}

// Exclusive prefix of n <= IB_MAX_BINS counts, in place, by the whole CTA;
// returns the total to every thread.
__device__ uint32_t ib_block_scan(uint32_t *v, uint32_t n) {
    __shared__ uint32_t warp_tot[IB_THREADS / 32];
    constexpr uint32_t PER = IB_MAX_BINS / IB_THREADS;
    const uint32_t b0 = threadIdx.x * PER;
    uint32_t sum = 0;
#pragma unroll
    for (uint32_t i = 0; i < PER; ++i) sum += b0 + i < n ? v[b0 + i] : 0u;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t x = lane < IB_THREADS / 32 ? warp_tot[lane] : 0u;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane < IB_THREADS / 32) warp_tot[lane] = x;
    }
    __syncthreads();
    uint32_t run = (wid ? warp_tot[wid - 1] : 0u) + incl - sum;
    const uint32_t total = warp_tot[IB_THREADS / 32 - 1];
#pragma unroll
    for (uint32_t i = 0; i < PER; ++i) {
        if (b0 + i < n) {
            const uint32_t x = v[b0 + i];
            v[b0 + i] = run;
            run += x;
        }
    }
    __syncthreads();
    return total;
}

template <int ETA, bool SORTED>
__global__ void __launch_bounds__(IB_THREADS) k_insert_bin_scatter(InsertArgs a, BinnedInsert b, uint64_t f0,
                                                                   uint64_t f1, bool wide) {
    constexpr uint32_t TK = IB_TILE_RECORDS / ETA;  // k-mers per tile
    constexpr uint32_t KPT = TK / IB_THREADS;       // k-mers per thread per tile
    static_assert(KPT * IB_THREADS * ETA == IB_TILE_RECORDS, "tile of whole k-mer rounds");
    extern __shared__ unsigned long long ib_smem[];
    unsigned long long *s_rec = ib_smem;                                         // IB_TILE_RECORDS
    uint32_t *s_bin = reinterpret_cast<uint32_t *>(s_rec + IB_TILE_RECORDS);     // bin, or NO_RANK
    uint32_t *s_rank = s_bin + IB_TILE_RECORDS;                                  // rank within the bin
    uint32_t *s_cnt = s_rank + IB_TILE_RECORDS;                                  // IB_MAX_BINS
    uint32_t *s_base = s_cnt + IB_MAX_BINS;                                      // IB_MAX_BINS
    // SORTED only (past the end of the unsorted variant's shared memory):
    uint32_t *s_pre = s_base + IB_MAX_BINS;      // IB_MAX_BINS: the tile's records before bin i
    unsigned long long *s_sorted = reinterpret_cast<unsigned long long *>(s_pre + IB_MAX_BINS);  // tile, bin order
    const uint64_t T = a.kcum[a.n];
    const uint64_t e1 = f1 < T ? f1 : T;
    if (f0 >= e1) return;  // the whole CTA
    uint64_t per = (e1 - f0 + gridDim.x - 1) / gridDim.x;
    per = (per + TK - 1) / TK * TK;
    const uint64_t c0 = f0 + (uint64_t)blockIdx.x * per;
    if (c0 >= e1) return;  // the whole CTA
    const uint64_t c1 = c0 + per < e1 ? c0 + per : e1;
    for (uint32_t i = threadIdx.x; i < b.nbins; i += IB_THREADS) s_cnt[i] = 0;
    __syncthreads();

    // document of this thread's first k-mer (largest i with kcum[i] <= g)
    const uint64_t g_first = c0 + threadIdx.x < c1 ? c0 + threadIdx.x : c1 - 1;
    uint64_t lo = 0, hi = a.n;
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a.kcum[mid] <= g_first) lo = mid;
        else hi = mid;
    }
    const uint64_t item_first = lo;

    for (uint32_t jb = 0; jb < a.eta; jb += ETA) {
        uint64_t item = item_first;
        for (uint64_t base = c0; base < c1; base += TK) {
            // 1. the tile's records, ranked within their bins (the k-mers a
            //    thread takes increase, so its document walk only goes forward)
            for (uint32_t kk = 0; kk < KPT; ++kk) {
                const uint32_t j = kk * IB_THREADS + threadIdx.x;
                const uint64_t g = base + j;
                bool val = g < c1;
                uint32_t d = 0;
                uint64_t c = 0;
                if (val) {
                    while (a.kcum[item + 1] <= g) ++item;
                    d = a.doc_ids[item];
                    if (d >= a.K) {
                        val = false;
                    } else {
                        const uint64_t start = a.offsets[item] + a.base_shift + (g - a.kcum[item]);
                        c = canonical_from_window(base_window(a.packed, a.packed_bytes, start), a.k);
                    }
                }
                const uint64_t km = mh_mix_key(c);
#pragma unroll
                for (int e = 0; e < ETA; ++e) {
                    const uint32_t slot = j * ETA + e;
                    if (val && jb + e < a.eta) {
                        const uint64_t h = mh_first_word(km, a.seed32 + jb + e);
                        const uint64_t p = a.m_pow2 ? (h & (a.m - 1)) : (h % a.m);
                        const uint32_t bin = (uint32_t)(p >> b.rshift);
                        s_rec[slot] = (p << IB_DOC_BITS) | d;
                        s_bin[slot] = bin;
                        s_rank[slot] = atomicAdd(&s_cnt[bin], 1u);
                    } else {
                        s_bin[slot] = NO_RANK;
                    }
                }
            }
            __syncthreads();
            // 2. each bin's share of the global bin, one atomic per bin, and
            //    the tile's bin offsets
            for (uint32_t i = threadIdx.x; i < b.nbins; i += IB_THREADS) {
                const uint32_t n = s_cnt[i];
                s_base[i] = n ? atomicAdd(b.count + i, n) : 0u;
                if constexpr (SORTED) s_pre[i] = n;
                s_cnt[i] = 0;
            }
            __syncthreads();
            if constexpr (SORTED) {
                const uint32_t total = ib_block_scan(s_pre, b.nbins);
                // 3. the tile in bin order
                for (uint32_t slot = threadIdx.x; slot < IB_TILE_RECORDS; slot += IB_THREADS) {
                    const uint32_t bin = s_bin[slot];
                    if (bin != NO_RANK) s_sorted[s_pre[bin] + s_rank[slot]] = s_rec[slot];
                }
                __syncthreads();
                // 4. the records, or their bits when the bin is full
                for (uint32_t i = threadIdx.x; i < total; i += IB_THREADS) {
                    const unsigned long long rec = s_sorted[i];
                    const uint32_t bin = (uint32_t)((rec >> IB_DOC_BITS) >> b.rshift);
                    const uint64_t at = (uint64_t)s_base[bin] + (i - s_pre[bin]);
                    if (at < b.cap) b.buf[(uint64_t)bin * b.cap + at] = rec;
                    else or_record(a, rec >> IB_DOC_BITS, (uint32_t)(rec & ((1u << IB_DOC_BITS) - 1)), wide);
                }
            } else {
                // 3. the records in slot order, or their bits when the bin is full
                for (uint32_t slot = threadIdx.x; slot < IB_TILE_RECORDS; slot += IB_THREADS) {
                    const uint32_t bin = s_bin[slot];
                    if (bin == NO_RANK) continue;
                    const unsigned long long rec = s_rec[slot];
                    const uint64_t at = (uint64_t)s_base[bin] + s_rank[slot];
                    if (at < b.cap) b.buf[(uint64_t)bin * b.cap + at] = rec;
                    else or_record(a, rec >> IB_DOC_BITS, (uint32_t)(rec & ((1u << IB_DOC_BITS) - 1)), wide);
                }
            }
            __syncthreads();  // the staging is the next tile's
        }
    }
}

// Apply pass: units of IB_UNIT records, claimed in bin order.
__global__ void __launch_bounds__(IB_THREADS) k_insert_bin_apply(InsertArgs a, BinnedInsert b, bool wide) {
    __shared__ uint32_t s_pre[IB_MAX_BINS + 1];  // units before bin i
    __shared__ uint32_t s_unit;
    // units per bin, then their exclusive prefix (warp 0: lane l sums bins
    // l*PER .. l*PER + PER - 1, a warp scan, then each lane writes its run)
    for (uint32_t i = threadIdx.x; i < b.nbins; i += IB_THREADS) {
        const uint64_t n = b.count[i] < b.cap ? b.count[i] : b.cap;
        s_pre[i] = (uint32_t)((n + IB_UNIT - 1) / IB_UNIT);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        constexpr uint32_t PER = IB_MAX_BINS / 32;
        const uint32_t lane = threadIdx.x, i0 = lane * PER;
        uint32_t sum = 0;
        for (uint32_t i = i0; i < i0 + PER; ++i) sum += i < b.nbins ? s_pre[i] : 0u;
        uint32_t incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= (uint32_t)off) incl += o;
        }
        uint32_t run = incl - sum;
        for (uint32_t i = i0; i < i0 + PER && i < b.nbins; ++i) {
            const uint32_t u = s_pre[i];
            s_pre[i] = run;
            run += u;
        }
        if (lane == 31) s_pre[b.nbins] = incl;
    }
    __syncthreads();
    const uint32_t units = s_pre[b.nbins];
    uint32_t *claim = b.count + IB_MAX_BINS;
    while (true) {
        if (threadIdx.x == 0) s_unit = atomicAdd(claim, 1u);
        __syncthreads();
        const uint32_t u = s_unit;
        __syncthreads();
        if (u >= units) break;
        // the bin holding unit u: s_pre[lo] <= u < s_pre[lo + 1]
        uint32_t lo = 0, hi = b.nbins;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_pre[mid] <= u) lo = mid;
            else hi = mid;
        }
        const uint64_t n = b.count[lo] < b.cap ? b.count[lo] : b.cap;
        const uint64_t r0 = (uint64_t)(u - s_pre[lo]) * IB_UNIT;
        const unsigned long long *src = b.buf + (uint64_t)lo * b.cap;
        for (uint32_t k = threadIdx.x; k < IB_UNIT; k += IB_THREADS) {
            const uint64_t r = r0 + k;
            if (r < n) {
                const unsigned long long rec = __ldcs(src + r);  // read once: do not keep in L2
                or_record(a, rec >> IB_DOC_BITS, (uint32_t)(rec & ((1u << IB_DOC_BITS) - 1)), wide);
            }
        }
    }
}

template <typename KernelT>
int ib_blocks_per_sm(KernelT kernel) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, IB_THREADS, 0) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

template <int ETA, bool SORTED>
cudaError_t launch_scatter_t(const InsertArgs &a, const BinnedInsert &b, uint64_t f0, uint64_t f1, bool wide,
                             int sm_count, cudaStream_t s) {
    constexpr size_t smem = scatter_smem<SORTED>();
    static int occ = [] {
        int n = 0;
        if (cudaFuncSetAttribute(k_insert_bin_scatter<ETA, SORTED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_insert_bin_scatter<ETA, SORTED>, IB_THREADS,
                                                          smem) != cudaSuccess ||
            n < 1)
            n = 1;
        return n;
    }();
    cudaError_t e = cudaFuncSetAttribute(k_insert_bin_scatter<ETA, SORTED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_insert_bin_scatter<ETA, SORTED><<<sm_count * occ, IB_THREADS, smem, s>>>(a, b, f0, f1, wide);
    return cudaGetLastError();
}

template <int ETA>
cudaError_t launch_scatter(const InsertArgs &a, const BinnedInsert &b, uint64_t f0, uint64_t f1, bool wide,
                           int sm_count, cudaStream_t s) {
    return b.nbins >= IB_SORT_MIN_BINS ? launch_scatter_t<ETA, true>(a, b, f0, f1, wide, sm_count, s)
                                       : launch_scatter_t<ETA, false>(a, b, f0, f1, wide, sm_count, s);
}

}  // namespace

uint32_t binned_insert_bins(uint64_t m, uint32_t group_bytes, uint32_t K, uint64_t region_bytes,
                            uint32_t *rshift) {
    if (m == 0 || group_bytes == 0 || m > (1ull << (64 - IB_DOC_BITS)) || K > (1u << IB_DOC_BITS)) return 0;
    uint32_t sh = 0;
    while (sh < 40 && ((uint64_t)group_bytes << (sh + 1)) <= region_bytes) ++sh;
    const uint64_t bins = (m + (1ull << sh) - 1) >> sh;
    if (bins > IB_MAX_BINS) return 0;
    *rshift = sh;
    return (uint32_t)bins;
}

cudaError_t launch_insert_binned(const InsertArgs &a, const BinnedInsert &b, uint64_t f0, uint64_t f1,
                                 int sm_count, cudaStream_t s) {
    // 64-bit words need the index (m * Gw words) to end on a 64-bit boundary
    const bool wide = (a.m * a.Gw) % 2 == 0;
    cudaError_t e;
    if (a.eta == 1) e = launch_scatter<1>(a, b, f0, f1, wide, sm_count, s);
    else if (a.eta == 2) e = launch_scatter<2>(a, b, f0, f1, wide, sm_count, s);
    else e = launch_scatter<4>(a, b, f0, f1, wide, sm_count, s);
    if (e != cudaSuccess) return e;
    static int occ = ib_blocks_per_sm(k_insert_bin_apply);
    k_insert_bin_apply<<<sm_count * occ, IB_THREADS, 0, s>>>(a, b, wide);
    return cudaGetLastError();
}

}  // namespace rgpu

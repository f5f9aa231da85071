// rambo_kernels_build.cu -- index construction and batch bookkeeping.
//
//   partition  phi_r(d) for every document and repetition (Section 3.2).
//   prefix     exclusive prefix of the k-mer counts of a batch, so that the
//              k-mers of all items form one flat index space [0, T).
//   register   DocIDs(M[phi_r(d), r]) += d, as bits of the bucket->document
//              bitmaps (Algorithm 2's DocIDs, the "inverted index mapping B
//              buckets to K documents" of Section 5.2).
//   insert     Algorithm 1: every k-mer x of document d sets bits
//              h_1(x)..h_eta(x) of BFU (phi_r(d), r) for every r.  In the
//              bit-sliced layout that is bit r*B+phi_r(d) of position group
//              h_j(x); lanes of a warp that hit the same word are combined
//              (warp-aggregated atomicOr) before one atomic is issued.
#include "rambo_internal.cuh"

namespace rgpu {
namespace {

constexpr uint32_t FULL = 0xffffffffu;

__global__ void k_partition(uint32_t *phi, uint32_t K, uint32_t R, uint32_t B, uint64_t seed) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (uint64_t)K * R) return;
    const uint32_t d = (uint32_t)(i / R), r = (uint32_t)(i % R);
    const uint64_t h = mh_first_word(mh_mix_key((uint64_t)d), (uint32_t)(seed + 1000 + r));
    phi[i] = (uint32_t)(h % B);
}

// -------------------------------------------------------------- prefix scan
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr uint64_t SCAN_TILE = (uint64_t)SCAN_THREADS * SCAN_ITEMS;

// Count of item i: its k-mers, or (tile > 0) the tiles of `tile` k-mers of
// an item with more than short_max k-mers (0 for shorter items).
struct CountMode {
    uint32_t tile;
    uint32_t short_max;
};

__device__ __forceinline__ uint64_t kmer_count(const uint64_t *begins, const uint64_t *ends,
                                               uint64_t i, uint32_t k, uint64_t limit,
                                               uint32_t *err, CountMode cm) {
    const uint64_t b0 = begins[i], b1 = ends[i];
    if (b1 < b0 || b1 > limit) {
        if (err) atomicOr(err, ERR_OFFSETS);
        return 0;
    }
    const uint64_t L = b1 - b0;
    const uint64_t nk = L >= k ? L - k + 1 : 0;
    if (cm.tile == 0) return nk;
    if (nk <= cm.short_max) return 0;
    if (nk < (1ull << 31)) return ((uint32_t)nk + cm.tile - 1u) / cm.tile;  // tile < 2^25
    return (nk + cm.tile - 1) / cm.tile;
}

// Block-wide exclusive scan of one value per thread (THREADS a multiple of
// 32, at most 1024); returns the prefix and writes the block total to *total.
template <int THREADS = SCAN_THREADS>
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *total) {
    __shared__ uint64_t warp_sums[THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t y = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint64_t s = lane < THREADS / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint64_t y = __shfl_up_sync(FULL, s, off);
            if (lane >= off) s += y;
        }
        if (lane < THREADS / 32) warp_sums[lane] = s;  // inclusive warp prefix
    }
    __syncthreads();
    const uint64_t before = wid ? warp_sums[wid - 1] : 0;
    *total = warp_sums[THREADS / 32 - 1];
    __syncthreads();
    return before + incl - v;
}

__global__ void __launch_bounds__(SCAN_THREADS)
k_prefix_partial(const uint64_t *begins, const uint64_t *ends, uint64_t n, uint32_t k,
                 uint64_t limit, uint64_t *bsum, uint32_t *err, CountMode cm) {
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    uint64_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * SCAN_THREADS + threadIdx.x;
        if (i < n) s += kmer_count(begins, ends, i, k, limit, err, cm);
    }
    uint64_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// One block: exclusive scan of the block sums in place; kcum[n] = grand total.
__global__ void __launch_bounds__(SCAN_THREADS)
k_prefix_blocks(uint64_t *bsum, uint64_t nblk, uint64_t *kcum, uint64_t n) {
    uint64_t carry = 0;
    for (uint64_t b0 = 0; b0 < nblk; b0 += SCAN_THREADS) {
        const uint64_t i = b0 + threadIdx.x;
        const uint64_t v = i < nblk ? bsum[i] : 0;
        uint64_t total;
        const uint64_t ex = block_exclusive_scan(v, &total);
        if (i < nblk) bsum[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) kcum[n] = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS)
k_prefix_final(const uint64_t *begins, const uint64_t *ends, uint64_t n, uint32_t k, uint64_t limit,
               const uint64_t *bsum, uint64_t *kcum, CountMode cm) {
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    uint64_t carry = bsum[blockIdx.x];
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * SCAN_THREADS + threadIdx.x;
        const uint64_t c = i < n ? kmer_count(begins, ends, i, k, limit, nullptr, cm) : 0;
        uint64_t total;
        const uint64_t ex = block_exclusive_scan(c, &total);
        if (i < n) kcum[i] = carry + ex;
        carry += total;
    }
}

// Small batches: the whole scan in one block of 1024 threads (one launch
// instead of three).  Each pass counts a tile of items with coalesced loads
// into shared memory, then every thread scans four consecutive counts;
// kcum[n] = grand total.
constexpr uint64_t SCAN_SINGLE_MAX = 16 * SCAN_TILE;
constexpr int SCAN1_THREADS = 1024;
constexpr int SCAN1_ITEMS = 4;
constexpr uint32_t SCAN1_TILE = SCAN1_THREADS * SCAN1_ITEMS;

__global__ void __launch_bounds__(SCAN1_THREADS)
k_prefix_single(const uint64_t *begins, const uint64_t *ends, uint64_t n, uint32_t k,
                uint64_t limit, uint64_t *kcum, uint32_t *err, CountMode cm) {
    __shared__ uint64_t s_cnt[SCAN1_TILE];
    uint64_t carry = 0;
    for (uint64_t base = 0; base < n; base += SCAN1_TILE) {
#pragma unroll
        for (int j = 0; j < SCAN1_ITEMS; ++j) {
            const uint32_t t = threadIdx.x + j * SCAN1_THREADS;
            s_cnt[t] = base + t < n ? kmer_count(begins, ends, base + t, k, limit, err, cm) : 0;
        }
        __syncthreads();
        uint64_t c[SCAN1_ITEMS];
        uint64_t sum = 0;
#pragma unroll
        for (int j = 0; j < SCAN1_ITEMS; ++j) {
            c[j] = s_cnt[threadIdx.x * SCAN1_ITEMS + j];
            sum += c[j];
        }
        uint64_t total;
        uint64_t run = carry + block_exclusive_scan<SCAN1_THREADS>(sum, &total);
        const uint64_t i0 = base + (uint64_t)threadIdx.x * SCAN1_ITEMS;
#pragma unroll
        for (int j = 0; j < SCAN1_ITEMS; ++j) {
            if (i0 + j < n) kcum[i0 + j] = run;
            run += c[j];
        }
        carry += total;  // the scan ends with a barrier: s_cnt may be refilled
    }
    if (threadIdx.x == 0) kcum[n] = carry;
}

// ------------------------------------------------------------- registration
__global__ void k_register(const uint32_t *doc_ids, uint64_t n, const uint32_t *phi, uint32_t K,
                           uint32_t R, uint32_t B, uint32_t W, uint32_t *docbits, uint32_t *err) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * R) return;
    const uint64_t item = i / R;
    const uint32_t r = (uint32_t)(i % R);
    const uint32_t d = doc_ids[item];
    if (d >= K) {
        if (r == 0) atomicOr(err, ERR_DOC_RANGE);
        return;
    }
    const uint32_t b = phi[(uint64_t)d * R + r];
    atomicOr(&docbits[((uint64_t)r * B + b) * W + (d >> 5)], 1u << (d & 31));
}

// ------------------------------------------------------------------- insert
constexpr int INSERT_THREADS = 256;

// MODE 0: lanes that hit the same index word combine their bits first
// (match + OR-reduce) and one of them issues the atomic; MODE 1: every
// (k-mer, probe, repetition) issues its own atomicOr; MODE 2: as 1, but the
// bits of consecutive repetitions that fall into one 64-bit word go in one
// 64-bit atomicOr (the repetitions' bits r*B + phi_r(d) ascend with r).
template <int ETA, int MODE>
__global__ void __launch_bounds__(INSERT_THREADS, 1) k_insert(InsertArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t T = a.kcum[a.n];
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    uint64_t per = (T + nwarps - 1) / nwarps;
    per = (per + 31) / 32 * 32;
    if (per < 64) per = 64;
    const uint64_t c0 = warp * per;
    if (c0 >= T) return;
    const uint64_t c1 = c0 + per < T ? c0 + per : T;

    // document of the warp's first k-mer (largest i with kcum[i] <= c0)
    uint64_t lo = 0, hi = a.n;
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a.kcum[mid] <= c0) lo = mid;
        else hi = mid;
    }
    const uint64_t i_first = lo;

    for (uint32_t jb = 0; jb < a.eta; jb += ETA) {
        uint64_t item = i_first;
        for (uint64_t base = c0; base < c1; base += 32) {
            const uint64_t g = base + lane;
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
                if (jb + e >= a.eta) break;  // warp-uniform
                const uint64_t h = mh_first_word(km, a.seed32 + jb + e);
                const uint64_t p = a.m_pow2 ? (h & (a.m - 1)) : (h % a.m);
                if (MODE == 0) {
                    for (uint32_t r = 0; r < a.R; ++r) {
                        uint64_t addr = ~0ULL;
                        uint32_t bit = 0;
                        if (val) {
                            const uint32_t bb = r * a.B + a.phi[(uint64_t)d * a.R + r];
                            addr = p * a.Gw + (bb >> 5);
                            bit = 1u << (bb & 31);
                        }
                        const uint32_t peers = __match_any_sync(FULL, addr);
                        const uint32_t v = __reduce_or_sync(peers, bit);
                        if (val && lane == __ffs(peers) - 1) atomicOr(a.index + addr, v);
                    }
                } else if (val) {
                    const uint64_t gbit = p * a.Gw * 32;  // first bit of the group
                    if (MODE == 1) {
                        for (uint32_t r = 0; r < a.R; ++r) {
                            const uint64_t bb = gbit + r * a.B + a.phi[(uint64_t)d * a.R + r];
                            atomicOr(a.index + (bb >> 5), 1u << (bb & 31));
                        }
                    } else {
                        unsigned long long *idx64 = reinterpret_cast<unsigned long long *>(a.index);
                        uint64_t cur = ~0ULL, bits = 0;
                        for (uint32_t r = 0; r < a.R; ++r) {
                            const uint64_t bb = gbit + r * a.B + a.phi[(uint64_t)d * a.R + r];
                            if ((bb >> 6) != cur) {
                                if (bits) atomicOr(idx64 + cur, (unsigned long long)bits);
                                cur = bb >> 6;
                                bits = 0;
                            }
                            bits |= 1ull << (bb & 63);
                        }
                        if (bits) atomicOr(idx64 + cur, (unsigned long long)bits);
                    }
                }
            }
        }
    }
}

// --------------------------------------------------------------------- fold
// Folding over (Section 5.3, Fig. 5): B -> Bh = B/2.  In position group p,
// repetition r's row of B bits (bits r*B ..) becomes the OR of its two halves,
// stored as the Bh-bit row at bits r*Bh of the new group.  One warp per group:
// the old group is staged in shared memory, lane r builds row r 32 bits at a
// time, and the new words are assembled with shared-memory atomicOr.
constexpr int FOLD_THREADS = 256;
constexpr int FOLD_MAX_WORDS = 128;  // groups up to 512 bytes

__device__ __forceinline__ uint32_t bits_at(const uint32_t *w, uint32_t nwords, uint32_t bit) {
    const uint32_t i = bit >> 5, sh = bit & 31;
    const uint32_t lo = w[i];
    const uint32_t hi = i + 1 < nwords ? w[i + 1] : 0u;
    return sh ? __funnelshift_r(lo, hi, sh) : lo;
}

__global__ void __launch_bounds__(FOLD_THREADS)
k_fold(const uint32_t *old_index, uint32_t old_gw, uint32_t *new_index, uint32_t new_gw, uint64_t m,
       uint32_t B, uint32_t R) {
    __shared__ uint32_t s_old[FOLD_THREADS / 32][FOLD_MAX_WORDS];
    __shared__ uint32_t s_new[FOLD_THREADS / 32][FOLD_MAX_WORDS];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t Bh = B / 2;
    const uint64_t warp = (uint64_t)blockIdx.x * (FOLD_THREADS / 32) + wib;
    const uint64_t nwarps = (uint64_t)gridDim.x * (FOLD_THREADS / 32);
    for (uint64_t p = warp; p < m; p += nwarps) {
        for (uint32_t i = lane; i < old_gw; i += 32) s_old[wib][i] = old_index[p * old_gw + i];
        for (uint32_t i = lane; i < new_gw; i += 32) s_new[wib][i] = 0;
        __syncwarp();
        for (uint32_t r = lane; r < R; r += 32) {
            for (uint32_t c = 0; c < Bh; c += 32) {
                const uint32_t len = Bh - c < 32 ? Bh - c : 32;
                const uint32_t mask = len == 32 ? FULL : ((1u << len) - 1u);
                const uint32_t x = (bits_at(s_old[wib], old_gw, r * B + c) |
                                    bits_at(s_old[wib], old_gw, r * B + Bh + c)) & mask;
                const uint32_t dst = r * Bh + c;
                const uint32_t wi = dst >> 5, sh = dst & 31;
                atomicOr(&s_new[wib][wi], x << sh);
                if (sh && len > 32 - sh) atomicOr(&s_new[wib][wi + 1], x >> (32 - sh));
            }
        }
        __syncwarp();
        for (uint32_t i = lane; i < new_gw; i += 32) new_index[p * new_gw + i] = s_new[wib][i];
        __syncwarp();
    }
}

// new DocBits[r][b] = old[r][b] | old[r][b + Bh]
__global__ void k_fold_docbits(const uint32_t *old_db, uint32_t *new_db, uint32_t B, uint32_t R,
                               uint32_t W) {
    const uint32_t Bh = B / 2;
    const uint64_t total = (uint64_t)R * Bh * W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t w = (uint32_t)(i % W);
        const uint64_t rb = i / W;
        const uint32_t b = (uint32_t)(rb % Bh), r = (uint32_t)(rb / Bh);
        new_db[i] = old_db[((uint64_t)r * B + b) * W + w] | old_db[((uint64_t)r * B + b + Bh) * W + w];
    }
}

template <typename KernelT>
int blocks_per_sm(KernelT kernel, int threads) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

template <int ETA>
cudaError_t launch_insert_t(const InsertArgs &a, int sm_count, cudaStream_t s) {
    // 64-bit words need the index (m * Gw words) to end on a 64-bit boundary
    const int mode = a.mode == 2 && (a.m * a.Gw) % 2 != 0 ? 1 : (int)a.mode;
    if (mode == 1) {
        static int occ = blocks_per_sm(k_insert<ETA, 1>, INSERT_THREADS);
        k_insert<ETA, 1><<<sm_count * occ, INSERT_THREADS, 0, s>>>(a);
    } else if (mode == 2) {
        static int occ = blocks_per_sm(k_insert<ETA, 2>, INSERT_THREADS);
        k_insert<ETA, 2><<<sm_count * occ, INSERT_THREADS, 0, s>>>(a);
    } else {
        static int occ = blocks_per_sm(k_insert<ETA, 0>, INSERT_THREADS);
        k_insert<ETA, 0><<<sm_count * occ, INSERT_THREADS, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_partition(uint32_t *phi, uint32_t K, uint32_t R, uint32_t B, uint64_t seed,
                             cudaStream_t s) {
    const uint64_t n = (uint64_t)K * R;
    k_partition<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(phi, K, R, B, seed);
    return cudaGetLastError();
}

size_t kmer_prefix_block_sums(uint64_t n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE); }

int kmer_prefix_launches(uint64_t n) { return n == 0 ? 0 : n <= SCAN_SINGLE_MAX ? 1 : 3; }

cudaError_t launch_kmer_prefix(const uint64_t *begins, const uint64_t *ends, uint64_t n, uint32_t k,
                               uint64_t packed_bytes, uint64_t *kcum, uint64_t *block_sums,
                               uint32_t *err, cudaStream_t s, uint32_t tile, uint32_t short_max) {
    const uint64_t limit = packed_bytes * 4;  // bases addressable from the caller's pointer
    const uint64_t nblk = kmer_prefix_block_sums(n);
    if (nblk == 0) return cudaSuccess;
    const CountMode cm{tile, short_max};
    if (n <= SCAN_SINGLE_MAX) {
        k_prefix_single<<<1, SCAN1_THREADS, 0, s>>>(begins, ends, n, k, limit, kcum, err, cm);
        return cudaGetLastError();
    }
    k_prefix_partial<<<(unsigned)nblk, SCAN_THREADS, 0, s>>>(begins, ends, n, k, limit, block_sums, err, cm);
    k_prefix_blocks<<<1, SCAN_THREADS, 0, s>>>(block_sums, nblk, kcum, n);
    k_prefix_final<<<(unsigned)nblk, SCAN_THREADS, 0, s>>>(begins, ends, n, k, limit, block_sums, kcum, cm);
    return cudaGetLastError();
}

cudaError_t launch_register_docs(const uint32_t *doc_ids, uint64_t n, const uint32_t *phi,
                                 uint32_t K, uint32_t R, uint32_t B, uint32_t W, uint32_t *docbits,
                                 uint32_t *err, cudaStream_t s) {
    const uint64_t total = n * R;
    if (total == 0) return cudaSuccess;
    k_register<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(doc_ids, n, phi, K, R, B, W, docbits,
                                                               err);
    return cudaGetLastError();
}

cudaError_t launch_fold(const uint32_t *old_index, uint32_t old_gw, uint32_t *new_index,
                        uint32_t new_gw, uint64_t m, uint32_t B, uint32_t R,
                        const uint32_t *old_db, uint32_t *new_db, uint32_t W, int sm_count,
                        cudaStream_t s) {
    if (old_gw > FOLD_MAX_WORDS || new_gw > FOLD_MAX_WORDS || (B & 1)) return cudaErrorInvalidValue;
    k_fold<<<sm_count * 8, FOLD_THREADS, 0, s>>>(old_index, old_gw, new_index, new_gw, m, B, R);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_fold_docbits<<<sm_count * 4, 256, 0, s>>>(old_db, new_db, B, R, W);
    return cudaGetLastError();
}

cudaError_t launch_insert(const InsertArgs &a, int sm_count, cudaStream_t s) {
    switch (a.eta) {
        case 1: return launch_insert_t<1>(a, sm_count, s);
        case 2: return launch_insert_t<2>(a, sm_count, s);
        case 3: return launch_insert_t<3>(a, sm_count, s);
        default: return launch_insert_t<4>(a, sm_count, s);
    }
}

// ---------------------------------------------------------------------------
// Document-sharded answers (Section 5.3): shard s holds the documents that
// the routing hash sends to it, as local documents 0..K_s-1; the global
// answer of a query is the union over shards of their answers placed at the
// documents' global ids (the shards' documents are disjoint, so this is a
// concatenation in global document order).  One thread per (query, shard
// word): each set bit is ORed into the global row.
namespace {
__global__ void k_merge_shard(uint64_t n, const uint32_t *masks, uint32_t sw, uint32_t sd,
                              const uint32_t *gid, uint32_t *out, uint32_t ow) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * sw) return;
    const uint64_t q = i / sw;
    const uint32_t w = (uint32_t)(i - q * sw);
    uint32_t v = masks[i];
    while (v) {
        const uint32_t j = 32 * w + (uint32_t)(__ffs(v) - 1);
        v &= v - 1;
        if (j >= sd) break;
        const uint32_t d = gid[j];
        if (d / 32 < ow) atomicOr(out + q * ow + d / 32, 1u << (d & 31));
    }
}
}  // namespace

cudaError_t launch_merge_shard(uint64_t n, const uint32_t *shard_masks, uint32_t shard_words,
                               uint32_t shard_docs, const uint32_t *global_ids, uint32_t *out,
                               uint32_t out_words, cudaStream_t s) {
    const uint64_t items = n * shard_words;
    k_merge_shard<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(n, shard_masks, shard_words, shard_docs,
                                                                   global_ids, out, out_words);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Failure-detection check of a bounded device wait: one thread polls an
// mbarrier that nothing ever completes (no arrivals are made), without
// suspending, and gives up after `spins` polls by latching ERR_WAIT.  Nothing
// faults or hangs; the host reads the latched word as RAMBO_ETIMEOUT.
namespace {
__global__ void k_wait_expiry(uint32_t *err, uint64_t spins) {
    __shared__ unsigned long long bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(1u) : "memory");
    for (uint64_t i = 0;; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(b), "r"(0u)
            : "memory");
        if (ok) return;
        if (i >= spins) {
            atomicOr(err, ERR_WAIT);
            return;
        }
    }
}
}  // namespace

cudaError_t launch_wait_expiry(uint32_t *err, uint64_t spins, cudaStream_t s) {
    k_wait_expiry<<<1, 32, 0, s>>>(err, spins);
    return cudaGetLastError();
}

}  // namespace rgpu

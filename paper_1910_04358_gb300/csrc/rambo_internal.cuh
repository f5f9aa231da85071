// rambo_internal.cuh -- device helpers and kernel launchers shared by the
// library's translation units (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace rgpu {

// ---------------------------------------------------------------------------
// Device error word bits (latched by kernels, read by rambo_sync).
enum : uint32_t {
    ERR_DOC_RANGE = 1u,     // document id >= K
    ERR_KMER_CODE = 2u,     // k-mer code with a bit at or above 2k
    ERR_OFFSETS = 4u,       // decreasing offsets or offsets past the buffer
    ERR_QUEUE = 8u,         // a work-queue claim loop exceeded its bound
    ERR_WAIT = 16u,         // a bounded device wait ran out
};

// ---------------------------------------------------------------------------
// MurmurHash3_x64_128 restricted to one 8-byte key (the only key length the
// index hashes).  The key block is mixed once (independent of the seed);
// each seed then costs the two finalisers.  First output word only.

__device__ __forceinline__ uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

// Mixed key block k1 of an 8-byte key (the key is the whole "tail").
__device__ __forceinline__ uint64_t mh_mix_key(uint64_t key) {
    uint64_t k1 = key * 0x87c37b91114253d5ULL;
    k1 = rotl64(k1, 31);
    return k1 * 0x4cf5ad432745937fULL;
}

// First output word for a mixed key and a 32-bit seed (length 8).
__device__ __forceinline__ uint64_t mh_first_word(uint64_t k1mix, uint32_t seed) {
    uint64_t h1 = (uint64_t)seed ^ k1mix ^ 8ULL;
    uint64_t h2 = (uint64_t)seed ^ 8ULL;
    h1 += h2;
    h2 += h1;
    return fmix64(h1) + fmix64(h2);
}

// ---------------------------------------------------------------------------
// k-mers from the 2-bit packed stream.

// 64-bit little-endian word wi of a byte buffer of nbytes bytes whose start
// is 8-byte aligned; bytes at or past nbytes read as zero and are not touched.
__device__ __forceinline__ uint64_t ld_stream_word(const uint8_t *p, uint64_t nbytes, uint64_t wi) {
    uint64_t b = wi * 8;
    if (b + 8 <= nbytes) return __ldg(reinterpret_cast<const unsigned long long *>(p) + wi);
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i)
        if (b + i < nbytes) v |= (uint64_t)__ldg(p + b + i) << (8 * i);
    return v;
}

// The 32 bases starting at base t, base t+i in bits 2i..2i+1.
__device__ __forceinline__ uint64_t base_window(const uint8_t *p, uint64_t nbytes, uint64_t t) {
    uint64_t bit = t * 2;
    uint64_t wi = bit >> 6;
    int sh = (int)(bit & 63);
    uint64_t lo = ld_stream_word(p, nbytes, wi);
    if (sh == 0) return lo;
    uint64_t hi = ld_stream_word(p, nbytes, wi + 1);
    return (lo >> sh) | (hi << (64 - sh));
}

// Reverses the order of the 32 two-bit digits of a 64-bit word.
__device__ __forceinline__ uint64_t reverse_digits(uint64_t x) {
    uint64_t y = __brevll(x);
    return ((y >> 1) & 0x5555555555555555ULL) | ((y & 0x5555555555555555ULL) << 1);
}

__device__ __forceinline__ uint64_t kmask(uint32_t k) {
    return k >= 32 ? ~0ULL : ((1ULL << (2 * k)) - 1);
}

// Canonical code of the k-mer whose bases sit least-significant-first in x:
// the reverse complement is the digit-wise complement of x read as is, the
// forward code is x with its digits reversed.
__device__ __forceinline__ uint64_t canonical_from_window(uint64_t x, uint32_t k) {
    uint64_t mask = kmask(k);
    uint64_t rc = ~x & mask;
    uint64_t fwd = reverse_digits(x) >> (64 - 2 * k);
    return fwd < rc ? fwd : rc;
}

// Canonical code of a forward code (first base most significant).
__device__ __forceinline__ uint64_t canonical_from_forward(uint64_t fwd, uint32_t k) {
    uint64_t x = reverse_digits(fwd) >> (64 - 2 * k);  // bases least significant first
    uint64_t rc = ~x & kmask(k);
    return fwd < rc ? fwd : rc;
}

// ---------------------------------------------------------------------------
// Streaming loads of index slices (read once: no L1 allocation).

template <int SW>
struct Slice;
template <>
struct Slice<1> {
    uint32_t w[1];
};
template <>
struct Slice<2> {
    uint32_t w[2];
};
template <>
struct Slice<4> {
    uint32_t w[4];
};

template <int SW>
__device__ __forceinline__ Slice<SW> ld_slice(const uint32_t *p);

template <>
__device__ __forceinline__ Slice<1> ld_slice<1>(const uint32_t *p) {
    Slice<1> s;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(s.w[0]) : "l"(p));
    return s;
}
template <>
__device__ __forceinline__ Slice<2> ld_slice<2>(const uint32_t *p) {
    Slice<2> s;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(s.w[0]), "=r"(s.w[1]) : "l"(p));
    return s;
}
template <>
__device__ __forceinline__ Slice<4> ld_slice<4>(const uint32_t *p) {
    Slice<4> s;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(s.w[0]), "=r"(s.w[1]), "=r"(s.w[2]), "=r"(s.w[3])
        : "l"(p));
    return s;
}

// ---------------------------------------------------------------------------
// Geometry of the bit-sliced index: m position groups, group p holding bit p
// of every BFU; BFU (b, r) is bit r*B+b of the group.

struct Geometry {
    uint32_t K, B, R, eta, k;
    uint64_t m;
    uint64_t seed;
    uint32_t W;        // mask words
    uint32_t gbits;    // R*B
    uint32_t Gw;       // words per group
    uint32_t SW;       // words per lane slice (1, 2 or 4)
    uint32_t LPG;      // lanes per group chunk (1..32)
    uint32_t chunks;   // group chunks of LPG*SW words (G > 512 bytes)
};

Geometry make_geometry(uint32_t K, uint32_t B, uint32_t R, uint64_t m, uint32_t eta, uint32_t k,
                       uint64_t seed);

// Arguments of the probe kernels.
struct ProbeArgs {
    const uint32_t *index;
    uint64_t m;
    uint32_t m_pow2;      // m is a power of two: reduce with a mask
    uint32_t Gw;
    uint32_t eta;
    uint32_t k;
    uint32_t seed32;      // (uint32) seed
    // sequence batch
    const uint8_t *packed;   // 8-byte aligned base of the packed stream
    uint64_t packed_bytes;   // readable bytes from `packed`
    uint64_t base_shift;     // bases to add to every offset (alignment fix-up)
    const uint64_t *offsets; // n item begins (base index)
    const uint64_t *ends;    // n item ends (CSR batches: offsets + 1)
    const uint64_t *kcum;    // n+1 exclusive prefix of k-mer counts
    uint64_t n;
    // single k-mers
    const uint64_t *kmers;
    // output: per query Gw words (bucket-space AND over its k-mers)
    uint32_t *acc;
    uint32_t *err;
    uint32_t min_chunk;      // minimum k-mers per warp (0 = default)
};

struct ExpandArgs {
    const uint32_t *acc;     // n x Gw
    uint64_t n;
    uint32_t Gw, B, R, W;
    const uint32_t *docbits; // R*B*W
    uint32_t *out;           // n x W
    const uint32_t *tab;     // byte table (R*ceil(B/8)*256*W) or null
    uint32_t smem_docbits;   // 1: stage DocBits in shared memory when it fits
    const uint32_t *ntab;    // nibble table (R*ceil(B/4)*16*W) or null
    const uint32_t *phi;     // K x R partition (candidate filtering)
    uint32_t K;
    uint32_t filter;         // 1: expand by candidate filtering when it fits
};

struct InsertArgs {
    uint32_t *index;
    uint64_t m;
    uint32_t m_pow2;
    uint32_t Gw, B, R, K, eta, k, seed32;
    const uint32_t *phi;       // K x R
    const uint32_t *doc_ids;   // n
    const uint8_t *packed;
    uint64_t packed_bytes;
    uint64_t base_shift;
    const uint64_t *offsets;   // n+1
    const uint64_t *kcum;      // n+1
    uint64_t n;
    uint32_t *err;
    uint32_t mode;             // 0: warp-aggregated 32-bit atomics; 1: plain 32-bit;
                               // 2: plain, repetitions sharing a 64-bit word merged
};

// Word documents (Section 5.4): term t is bytes [term_offs[t], term_offs[t+1])
// of `bytes`; item i (a document or a query) is terms [item_terms[i],
// item_terms[i+1]).
struct WordArgs {
    uint32_t *index;           // insert: written with atomicOr
    const uint32_t *index_ro;  // probe: read only
    uint64_t m;
    uint32_t m_pow2;
    uint32_t Gw, B, R, K, eta, seed32;
    const uint32_t *phi;       // K x R
    const uint32_t *doc_ids;   // insert: n
    const uint8_t *bytes;
    uint64_t bytes_len;
    const uint64_t *term_offs;
    const uint64_t *item_terms;  // n+1
    uint64_t n;
    uint32_t *acc;             // probe: n x Gw, preset to all ones
    uint32_t *err;
};
cudaError_t launch_insert_words(const WordArgs &a, int sm_count, cudaStream_t s);
cudaError_t launch_probe_words(const WordArgs &a, int sm_count, cudaStream_t s);

// Launchers (rambo_kernels_*.cu).  All enqueue on `s` and return the launch
// status.
cudaError_t launch_partition(uint32_t *phi, uint32_t K, uint32_t R, uint32_t B, uint64_t seed,
                             cudaStream_t s);
// Exclusive prefix (n+1 values) of the k-mer counts of items
// [begins[i], ends[i]); with tile > 0, of the tile counts of the items with
// more than short_max k-mers (ceil(k-mers / tile); shorter items count 0).
// Device address of the host range [p, p + bytes) when both its ends lie in
// page-locked host memory that the current device can address (allocated
// with cudaHostAlloc / cudaMallocHost or registered, mapped under unified
// addressing) at consistent device addresses; null otherwise (pageable
// memory, device memory, or a range that does not look like one buffer).
void *mapped_host_range(const void *p, uint64_t bytes);

// Kernels one launch_kmer_prefix of n items enqueues.
int kmer_prefix_launches(uint64_t n);
cudaError_t launch_kmer_prefix(const uint64_t *begins, const uint64_t *ends, uint64_t n, uint32_t k,
                               uint64_t packed_bytes, uint64_t *kcum, uint64_t *block_sums,
                               uint32_t *err, cudaStream_t s, uint32_t tile = 0,
                               uint32_t short_max = 0);
size_t kmer_prefix_block_sums(uint64_t n);
cudaError_t launch_register_docs(const uint32_t *doc_ids, uint64_t n, const uint32_t *phi,
                                 uint32_t K, uint32_t R, uint32_t B, uint32_t W, uint32_t *docbits,
                                 uint32_t *err, cudaStream_t s);
cudaError_t launch_insert(const InsertArgs &a, int sm_count, cudaStream_t s);
// ORs the answers of one document shard (n rows of shard_words words, bit j
// = the shard's local document j) into global answer rows of out_words
// words at bit global_ids[j] (device array of shard_docs ids).
cudaError_t launch_merge_shard(uint64_t n, const uint32_t *shard_masks, uint32_t shard_words,
                               uint32_t shard_docs, const uint32_t *global_ids, uint32_t *out,
                               uint32_t out_words, cudaStream_t s);
// Folding over B -> B/2 of the index (groups up to 512 bytes) and DocBits.
cudaError_t launch_fold(const uint32_t *old_index, uint32_t old_gw, uint32_t *new_index,
                        uint32_t new_gw, uint64_t m, uint32_t B, uint32_t R,
                        const uint32_t *old_db, uint32_t *new_db, uint32_t W, int sm_count,
                        cudaStream_t s);
cudaError_t launch_probe_seqs(const ProbeArgs &a, const Geometry &g, int sm_count, cudaStream_t s);
// staged: one-lane 16-byte groups and eta <= 2 gather into shared memory (cp.async)
cudaError_t launch_probe_kmers(const ProbeArgs &a, const Geometry &g, int sm_count, cudaStream_t s,
                               bool staged);
// Work queues of the persistent fused query (workspace arrays).
struct FusedQueues {
    uint32_t *counters;      // 8 words, zeroed by the launcher
    uint32_t *short_list;    // n
    const uint64_t *tile_prefix;  // n+1: exclusive prefix of long-query tile counts
    uint32_t *done;          // n
    uint32_t *heavy;         // n: queries expanded by the second launch
    uint32_t tile;           // k-mers per long tile
    uint32_t short_max;      // longest short query (k-mers)
    uint64_t user_bases;     // bases addressable from the caller's packed pointer
    uint32_t early_exit;     // 1: skip the rest of a query once a repetition row is empty
    uint32_t segment;        // early exit: k-mers between checks (multiple of 128)
    unsigned long long *probed;  // early exit: k-mers actually probed (or null)
    uint32_t async;          // 1: one-lane 16-byte groups gathered into shared memory (cp.async)
};
bool fused_supported(const Geometry &g);
// Region-binned probing of a sequence batch (query path 2; groups of up to
// 64 bytes): records in nb x G sub-bins of cap records each (bin = region
// pos >> shift, G = the scatter's grid: one sub-bin per bin and block).
constexpr uint32_t BINNED_TILE_RECS = 4096;  // probe records per scatter tile
constexpr uint32_t BINNED_ITEM_RECS = 512;   // records per probe-pass work item
struct BinnedArgs {
    ProbeArgs p;                    // index, hashing, batch; kcum = the tile prefix
                                    // (tiles of `tile` k-mers, every query with k-mers);
                                    // acc preset to all ones
    uint64_t *records;              // nb * G * cap records (group << 32 | query)
    uint32_t *sub_count;            // nb * G: records in each sub-bin (at most cap)
    uint32_t *tile_q;               // query of each of the first max_tiles scatter tiles
    uint64_t max_tiles;             // binned_max_tiles
    uint64_t cap;                   // record slots per sub-bin (even)
    uint32_t nb, shift;
    uint32_t G;                     // scatter grid (binned_scatter_grid)
    uint32_t tile;                  // k-mers per scatter tile (binned_tile_kmers)
    uint32_t depth;                 // probe pass: 2, 4 or 8 for 4, 8 or 12 gathers a lane keeps in flight
    uint32_t cps;                   // work items per sub-bin: ceil(cap / BINNED_ITEM_RECS)
    unsigned long long *item_ctr;   // probe pass: next work item, zeroed by k_bin_tiles
};
bool binned_supported(const Geometry &g);
uint32_t binned_tile_kmers(const Geometry &g);
uint32_t binned_depth(uint32_t rows);  // from the bin_rows knob
uint64_t binned_max_tiles(const Geometry &g, uint64_t n, uint64_t packed_bytes);
uint32_t binned_scatter_grid(const Geometry &g, uint32_t nb, int sm_count);
// Regions of (at most) region_bytes, a power-of-two number of groups, and at
// most 4096 of them: returns the bin count, *shift = log2(groups per region).
uint32_t binned_bins(const Geometry &g, uint64_t region_bytes, uint32_t *shift);
int binned_launches();
cudaError_t launch_binned(const BinnedArgs &a, const Geometry &g, int sm_count, cudaStream_t s);

// Content-ordered segments (query path 3; groups of up to 64 bytes, eta <=
// 4): the batch's k-mers cut at content-defined points into segments, the
// segments ordered by the bucket of their key, then probed in that order.
struct SegArgs {
    ProbeArgs p;                  // index, hashing, the query batch (kcum over the
                                  // queries), acc preset to all ones
    uint32_t cut_bits;            // a k-mer starts a segment when the low cut_bits
    uint32_t min_len;             //   bits of its order hash are zero and the last
                                  //   start is min_len k-mers back (or it is forced)
    uint32_t bucket_shift;        // bucket = key >> bucket_shift
    uint32_t nbuckets;
    uint64_t cap;                 // segment slots of every array below
    unsigned long long *ctr;      // [0] segments recorded, [1] probe items claimed (zeroed)
    uint32_t *bucket;             // nbuckets counts (zeroed) -> offsets -> cursors
    uint64_t *raw_begin;          // recorded segments: first base (caller's base index)
    uint32_t *raw_len, *raw_q, *raw_key;  //   k-mers, query, key
    uint64_t *sbeg, *send;        // ordered segments as base ranges [sbeg, send)
    uint32_t *sq;                 //   and their queries
    uint64_t *scum;               // cap + 1: k-mer prefix of the ordered segments
    uint32_t *chunk_seg;          // max_chunks: segment of every PSK-th ordered k-mer
    uint64_t max_chunks;
};
bool segments_supported(const Geometry &g);
uint32_t seg_cut_grid(int sm_count);
// Segment slots a batch of n items with at most max_kmers k-mers can need.
uint64_t seg_capacity(uint64_t max_kmers, uint64_t n, uint32_t min_len, uint32_t cut_grid);
uint64_t seg_max_chunks(uint64_t max_kmers);
int seg_launches_before_prefix();
int seg_launches_after_prefix();
// cut + bucket offsets + placement (after the query prefix; ctr and bucket zeroed)
cudaError_t launch_seg_order(const SegArgs &a, uint32_t cut_grid, int sm_count, cudaStream_t s);
// chunk map + probe (after the prefix of the ordered segments into scum)
cudaError_t launch_seg_probe(const SegArgs &a, const Geometry &g, int sm_count, cudaStream_t s);

// p.acc is unused (the bucket masks of long queries, and of queries with too
// many passing buckets to expand in place, are e.acc).  Two launches after
// the prep: the persistent query and the heavy queries' expansion.
cudaError_t launch_fused(const ProbeArgs &p, const ExpandArgs &e, const Geometry &g,
                         const FusedQueues &qs, int grid_override, int sm_count, cudaStream_t s);

// max_blocks caps the expansion grid
cudaError_t launch_expand(const ExpandArgs &a, int max_blocks, int sm_count, cudaStream_t s);
// A bounded mbarrier wait that nothing completes; latches ERR_WAIT on expiry.
cudaError_t launch_wait_expiry(uint32_t *err, uint64_t spins, cudaStream_t s);
uint64_t bytetab_words(uint32_t B, uint32_t R, uint32_t W);
uint64_t nibtab_words(uint32_t B, uint32_t R, uint32_t W);
cudaError_t launch_build_nibtab(const uint32_t *docbits, uint32_t B, uint32_t R, uint32_t W,
                                uint32_t *ntab, int sm_count, cudaStream_t s);
cudaError_t launch_build_bytetab(const uint32_t *docbits, uint32_t B, uint32_t R, uint32_t W,
                                 uint32_t *tab, int sm_count, cudaStream_t s);

}  // namespace rgpu

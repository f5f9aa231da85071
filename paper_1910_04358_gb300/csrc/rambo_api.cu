// rambo_api.cu -- the C ABI declared in include/rambo.h: handle lifetime,
// argument checks, workspace layout, host staging and kernel sequencing.
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "rambo.h"
#include "rambo_insert_binned.cuh"
#include "rambo_internal.cuh"

using namespace rgpu;

struct rambo {
    Geometry g;
    int device;
    int sm_count;
    cudaStream_t stream;     // used by the host-buffer calls
    cudaStream_t kstream[RAMBO_MAX_HOST_SLOTS];  // k-mer branch of mixed batches (host calls
                                                 // rotate chunks over them)
    cudaStream_t pstream[RAMBO_MAX_HOST_SLOTS];  // the same at the device's greatest priority
    cudaEvent_t ev_fork, ev_join, ev_join2;
    uint64_t *h_offs;        // page-locked staging of rebased host offsets
    size_t h_offs_bytes;
    uint32_t *h_err;         // page-locked copy of the latched error word
    uint32_t *d_index;       // m * Gw words
    uint32_t *d_docbits;     // R * B * W words
    uint32_t *d_phi;         // K * R
    uint32_t *d_err;         // latched device error bits
    unsigned long long *d_probed;  // k-mers probed under early exit
    void *d_stage;           // host-call staging + workspace
    size_t stage_bytes;
    bool any_inserted;       // set by the first insert call
    uint32_t *d_tab;         // byte table for the expansion (or null)
    uint32_t *d_ntab;        // nibble table for the expansion (or null)
    unsigned long long *d_bins;  // binned insert: records (insert_mode 3), or null
    uint32_t *d_bin_count;       // binned insert: per-bin counts and the unit counter
    uint64_t bins_records;       // records d_bins holds
    rambo_tuning_t tune;
    // profiling
    uint32_t prof_mask;
    uint64_t launches[RAMBO_NUM_STAGES];
    uint64_t timed[RAMBO_NUM_STAGES];
    double ms[RAMBO_NUM_STAGES];
    struct Pending {
        int stage;
        cudaEvent_t start, stop;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
};

namespace rgpu {

void *mapped_host_range(const void *p, uint64_t bytes) {
    if (!p || !bytes) return nullptr;
    const char *first = static_cast<const char *>(p);
    const char *last = first + (bytes - 1);
    cudaPointerAttributes a0{}, a1{};
    if (cudaPointerGetAttributes(&a0, first) != cudaSuccess ||
        cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
        cudaGetLastError();  // an unknown pointer leaves a (non-sticky) error behind
        return nullptr;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer ||
        !a1.devicePointer)
        return nullptr;
    if (static_cast<const char *>(a1.devicePointer) - static_cast<const char *>(a0.devicePointer) !=
        static_cast<ptrdiff_t>(bytes - 1))
        return nullptr;
    return a0.devicePointer;
}

Geometry make_geometry(uint32_t K, uint32_t B, uint32_t R, uint64_t m, uint32_t eta, uint32_t k,
                       uint64_t seed) {
    Geometry g{};
    g.K = K; g.B = B; g.R = R; g.m = m; g.eta = eta; g.k = k; g.seed = seed;
    g.W = (K + 31) / 32;
    g.gbits = R * B;
    const uint64_t raw = ((uint64_t)g.gbits + 31) / 32 * 4;  // bytes
    uint64_t G;
    if (raw <= 512) {
        G = 4;
        while (G < raw) G <<= 1;
    } else {
        G = (raw + 511) / 512 * 512;
    }
    g.Gw = (uint32_t)(G / 4);
    if (G <= 16) {
        g.SW = (uint32_t)(G / 4);
        g.LPG = 1;
        g.chunks = 1;
    } else {
        g.SW = 4;
        g.LPG = (uint32_t)(G >= 512 ? 32 : G / 16);
        g.chunks = (uint32_t)(G >= 512 ? G / 512 : 1);
    }
    return g;
}

}  // namespace rgpu

namespace {

constexpr size_t ALIGN = 256;

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return RAMBO_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return RAMBO_ENOMEM;
    }
    return RAMBO_ECUDA;
}

#define RAMBO_TRY(expr)                         \
    do {                                        \
        const int rc_ = cuda_rc(expr);          \
        if (rc_ != RAMBO_OK) return rc_;        \
    } while (0)

// Brackets the launches of one stage: counts them and, if the stage is
// selected for timing, records events on the launching stream.
class StageScope {
  public:
    StageScope(rambo_t *h, int stage, cudaStream_t s, int kernels) : h_(h), stage_(stage), s_(s) {
        h_->launches[stage] += kernels;
        if (!(h_->prof_mask & (1u << stage))) return;
        start_ = take();
        stop_ = take();
        if (start_ && stop_ && cudaEventRecord(start_, s_) == cudaSuccess) armed_ = true;
    }
    ~StageScope() {
        if (armed_ && cudaEventRecord(stop_, s_) == cudaSuccess) {
            h_->pending.push_back({stage_, start_, stop_});
        } else {
            give(start_);
            give(stop_);
        }
    }

  private:
    cudaEvent_t take() {
        if (!h_->event_pool.empty()) {
            cudaEvent_t e = h_->event_pool.back();
            h_->event_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    void give(cudaEvent_t e) {
        if (e) h_->event_pool.push_back(e);
    }
    rambo_t *h_;
    int stage_;
    cudaStream_t s_;
    cudaEvent_t start_ = nullptr, stop_ = nullptr;
    bool armed_ = false;
};

// Probe grid: CTAs per SM from the tuning (0 = occupancy maximum).
int probe_grid(const rambo_t *h) {
    return h->tune.probe_ctas_per_sm ? -(int)(h->sm_count * h->tune.probe_ctas_per_sm) : h->sm_count;
}

// Grid of the single-k-mer probe: its own knob, else the sequence probe's.
int kmer_probe_grid(const rambo_t *h) {
    const uint32_t c = h->tune.kmer_probe_ctas_per_sm;
    return c ? -(int)(h->sm_count * c) : probe_grid(h);
}

// (Re)allocates or frees the byte table to match the tuning; the table is
// rebuilt from the current bitmaps on the handle's stream.  The nibble table
// (small enough for shared memory) is kept whenever it fits 96 KiB.
int apply_bytetab(rambo_t *h) {
    const Geometry &g = h->g;
    const uint64_t nbytes = nibtab_words(g.B, g.R, g.W) * 4;
    if (nbytes <= 96 * 1024 && g.W <= 128) {
        if (!h->d_ntab) RAMBO_TRY(cudaMalloc(&h->d_ntab, nbytes));
        RAMBO_TRY(launch_build_nibtab(h->d_docbits, g.B, g.R, g.W, h->d_ntab, h->sm_count, h->stream));
    } else if (h->d_ntab) {
        RAMBO_TRY(cudaStreamSynchronize(h->stream));
        cudaFree(h->d_ntab);
        h->d_ntab = nullptr;
    }
    const uint64_t bytes = bytetab_words(g.B, g.R, g.W) * 4;
    const bool want = h->tune.use_byte_table &&
                      bytes <= (uint64_t)h->tune.byte_table_max_mb * (1ull << 20);
    if (!want) {
        if (h->d_tab) {
            RAMBO_TRY(cudaStreamSynchronize(h->stream));
            cudaDeviceSynchronize();
            cudaFree(h->d_tab);
            h->d_tab = nullptr;
        }
        return RAMBO_OK;
    }
    if (!h->d_tab) {
        cudaDeviceSynchronize();
        RAMBO_TRY(cudaMalloc(&h->d_tab, bytes));
    }
    RAMBO_TRY(launch_build_bytetab(h->d_docbits, g.B, g.R, g.W, h->d_tab, h->sm_count, h->stream));
    RAMBO_TRY(cudaStreamSynchronize(h->stream));
    return RAMBO_OK;
}

// Workspace layouts (offsets are 256-byte aligned).
struct SeqWs {
    size_t kcum, bsum, acc, qcnt, slist, done, heavy, total;
};
SeqWs seq_ws(const Geometry &g, uint64_t n) {
    SeqWs w;
    w.kcum = 0;
    w.bsum = align_up((n + 1) * 8);
    w.acc = w.bsum + align_up((kmer_prefix_block_sums(n) + 1) * 8);
    w.qcnt = w.acc + align_up(n * (uint64_t)g.Gw * 4);
    w.slist = w.qcnt + ALIGN;
    w.done = w.slist + align_up(n * 4);
    w.heavy = w.done + align_up(n * 4);
    w.total = w.heavy + align_up(n * 4);
    return w;
}

size_t kmers_ws(const Geometry &g, uint64_t n) { return align_up(n * (uint64_t)g.Gw * 4); }

// Extra workspace of the region-binned path (after the sequence layout):
// the sub-bin counts, the tile -> query map and nb x G sub-bins of cap
// records (G = the scatter's grid).  A sub-bin holds 1/8 more than its
// expected share of a batch whose k-mers are at most the bases of
// packed_bytes (plus 64), so with hashed positions records almost never
// spill into the direct-probe path.
struct BinLayout {
    uint32_t nb, shift, G;
    uint64_t cap;
    size_t ctr_off, count_off, tile_off, rec_off, bytes;
};
BinLayout bin_layout(const rambo_t *h, uint64_t n, uint64_t packed_bytes) {
    const Geometry &g = h->g;
    BinLayout L{};
    const uint64_t region = (uint64_t)(h->tune.bin_region_kib ? h->tune.bin_region_kib : 32768) << 10;
    L.nb = binned_bins(g, region, &L.shift);
    L.G = binned_scatter_grid(g, L.nb, h->sm_count);
    const uint64_t subs = (uint64_t)L.nb * L.G;
    const uint64_t expect = (4 * packed_bytes * g.eta + subs - 1) / subs;
    L.cap = (expect + expect / 8 + 64 + 1) / 2 * 2;  // even: 16-byte aligned record pairs
    L.ctr_off = 0;  // the probe pass's work-item counter
    L.count_off = 256;
    L.tile_off = L.count_off + align_up((size_t)subs * 4);
    L.rec_off = L.tile_off + align_up((size_t)binned_max_tiles(g, n, packed_bytes) * 4);
    L.bytes = L.rec_off + (size_t)subs * L.cap * 8;
    return L;
}
bool use_binned(const rambo_t *h) { return h->tune.query_path == 2 && binned_supported(h->g); }

// Extra workspace of the content-ordered path (after the sequence layout):
// counters and bucket counts (zeroed per call), the recorded segments, the
// ordered segments with their k-mer prefix, and the chunk map, for a CSR
// batch of n items over packed_bytes (at most 4 * packed_bytes k-mers).
constexpr uint32_t SEG_BUCKET_BITS = 16;
struct SegLayout {
    uint64_t cap, max_chunks;
    uint32_t cut_grid, cut_bits, min_len;
    size_t hdr_off, hdr_bytes, rbeg_off, rlen_off, rq_off, rkey_off, sbeg_off, send_off, sq_off, scum_off,
        sbsum_off, chunk_off, bytes;
};
SegLayout seg_layout(const rambo_t *h, uint64_t n, uint64_t packed_bytes) {
    SegLayout S{};
    S.cut_bits = h->tune.seg_cut_bits ? h->tune.seg_cut_bits : 6;
    S.min_len = 1u << (S.cut_bits - 1);
    S.cut_grid = seg_cut_grid(h->sm_count);
    const uint64_t max_kmers = 4 * packed_bytes;
    S.cap = seg_capacity(max_kmers, n, S.min_len, S.cut_grid);
    S.max_chunks = seg_max_chunks(max_kmers);
    S.hdr_off = 0;
    S.hdr_bytes = ALIGN + ((size_t)1 << SEG_BUCKET_BITS) * 4;
    S.rbeg_off = align_up(S.hdr_bytes);
    S.rlen_off = S.rbeg_off + align_up(S.cap * 8);
    S.rq_off = S.rlen_off + align_up(S.cap * 4);
    S.rkey_off = S.rq_off + align_up(S.cap * 4);
    S.sbeg_off = S.rkey_off + align_up(S.cap * 4);
    S.send_off = S.sbeg_off + align_up(S.cap * 8);
    S.sq_off = S.send_off + align_up(S.cap * 8);
    S.scum_off = S.sq_off + align_up(S.cap * 4);
    S.sbsum_off = S.scum_off + align_up((S.cap + 1) * 8);
    S.chunk_off = S.sbsum_off + align_up((kmer_prefix_block_sums(S.cap) + 1) * 8);
    S.bytes = S.chunk_off + align_up(S.max_chunks * 4);
    return S;
}
bool use_segments(const rambo_t *h) { return h->tune.query_path == 3 && segments_supported(h->g); }
// Sequence workspace that lets the tuned path run on a batch over packed_bytes.
size_t seq_ws_for(const rambo_t *h, uint64_t n, uint64_t packed_bytes) {
    size_t t = seq_ws(h->g, n).total;
    if (use_binned(h)) t += bin_layout(h, n, packed_bytes).bytes;
    if (use_segments(h)) t += seg_layout(h, n, packed_bytes).bytes;
    return t;
}

struct InsWs {
    size_t kcum, bsum, total;
};
InsWs ins_ws(uint64_t n) {
    InsWs w;
    w.kcum = 0;
    w.bsum = align_up((n + 1) * 8);
    w.total = w.bsum + align_up((kmer_prefix_block_sums(n) + 1) * 8);
    return w;
}

// Waits for the handle's own streams; returns the first error seen.
cudaError_t sync_own_streams(rambo_t *h) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    for (cudaStream_t ks : h->kstream) {
        const cudaError_t e2 = cudaStreamSynchronize(ks);
        if (e == cudaSuccess) e = e2;
    }
    for (cudaStream_t ps : h->pstream) {
        const cudaError_t e2 = cudaStreamSynchronize(ps);
        if (e == cudaSuccess) e = e2;
    }
    return e;
}

int reserve_stage(rambo_t *h, size_t bytes) {
    if (bytes <= h->stage_bytes) return RAMBO_OK;
    RAMBO_TRY(sync_own_streams(h));
    if (h->d_stage) cudaFree(h->d_stage);
    h->d_stage = nullptr;
    h->stage_bytes = 0;
    size_t want = bytes + bytes / 4;
    RAMBO_TRY(cudaMalloc(&h->d_stage, want));
    h->stage_bytes = want;
    return RAMBO_OK;
}

// Packed pointers of any alignment: read from the 8-byte aligned address
// below and shift every base offset by the bytes in between.
struct Aligned {
    const uint8_t *p;
    uint64_t bytes;
    uint64_t base_shift;
};
Aligned align_packed(const uint8_t *packed, uint64_t packed_bytes) {
    const uintptr_t mis = reinterpret_cast<uintptr_t>(packed) & 7;
    return Aligned{packed - mis, packed_bytes + mis, (uint64_t)mis * 4};
}

// Items are [begins[i], ends[i]); a CSR batch passes (offsets, offsets + 1).
// fused_ctas_cap > 0 caps the persistent fused launch at that many CTAs per
// SM (so that other kernels of the same batch can run beside it).
int query_seqs_enqueue(rambo_t *h, uint64_t n, const uint8_t *packed, uint64_t packed_bytes,
                       const uint64_t *offsets, const uint64_t *ends, uint32_t *out, void *ws,
                       size_t ws_bytes, cudaStream_t s, uint32_t fused_ctas_cap = 0) {
    const Geometry &g = h->g;
    const SeqWs L = seq_ws(g, n);
    char *w = static_cast<char *>(ws);
    uint64_t *kcum = reinterpret_cast<uint64_t *>(w + L.kcum);
    uint64_t *bsum = reinterpret_cast<uint64_t *>(w + L.bsum);
    uint32_t *acc = reinterpret_cast<uint32_t *>(w + L.acc);
    const Aligned al = align_packed(packed, packed_bytes);
    if (use_binned(h)) {
        const BinLayout B = bin_layout(h, n, packed_bytes);
        if (ws_bytes >= L.total + B.bytes) {
            // region-binned probing: records binned by index region, probed
            // region by region (L2 holds a region), then the expansion
            BinnedArgs ba{};
            ba.tile = binned_tile_kmers(g);
            {
                // tile prefix: every query's k-mers in tiles of ba.tile
                StageScope sc(h, RAMBO_STAGE_PREFIX, s, kmer_prefix_launches(n));
                RAMBO_TRY(launch_kmer_prefix(offsets, ends, n, g.k, packed_bytes, kcum, bsum, h->d_err, s,
                                             ba.tile, 0));
            }
            RAMBO_TRY(cudaMemsetAsync(acc, 0xFF, n * (uint64_t)g.Gw * 4, s));
            ProbeArgs &a = ba.p;
            a.index = h->d_index;
            a.m = g.m;
            a.m_pow2 = (g.m & (g.m - 1)) == 0;
            a.Gw = g.Gw;
            a.eta = g.eta;
            a.k = g.k;
            a.seed32 = (uint32_t)g.seed;
            a.packed = al.p;
            a.packed_bytes = al.bytes;
            a.base_shift = al.base_shift;
            a.offsets = offsets;
            a.ends = ends;
            a.kcum = kcum;
            a.n = n;
            a.acc = acc;
            a.err = h->d_err;
            char *bw = w + L.total;
            ba.sub_count = reinterpret_cast<uint32_t *>(bw + B.count_off);
            ba.records = reinterpret_cast<uint64_t *>(bw + B.rec_off);
            ba.tile_q = reinterpret_cast<uint32_t *>(bw + B.tile_off);
            ba.max_tiles = binned_max_tiles(g, n, packed_bytes);
            ba.cap = B.cap;
            ba.nb = B.nb;
            ba.shift = B.shift;
            ba.G = B.G;
            ba.depth = binned_depth(h->tune.bin_rows);
            ba.cps = (uint32_t)((B.cap + BINNED_ITEM_RECS - 1) / BINNED_ITEM_RECS);
            ba.item_ctr = reinterpret_cast<unsigned long long *>(bw + B.ctr_off);
            {
                StageScope sc(h, RAMBO_STAGE_PROBE_SEQS, s, binned_launches());
                RAMBO_TRY(launch_binned(ba, g, h->sm_count, s));
            }
            ExpandArgs e{acc, n, g.Gw, g.B, g.R, g.W, h->d_docbits, out, h->d_tab, h->tune.smem_docbits,
                         h->tune.use_nibble_table ? h->d_ntab : nullptr, h->d_phi, g.K,
                         h->tune.expand_filter};
            StageScope sc(h, RAMBO_STAGE_EXPAND, s, 1);
            RAMBO_TRY(launch_expand(e, h->sm_count * (int)h->tune.expand_ctas_per_sm, h->sm_count, s));
            return RAMBO_OK;
        }
    }
    if (use_segments(h) && ends == offsets + 1) {
        // content-ordered segments (CSR batches: at most 4 * packed_bytes k-mers)
        const SegLayout S = seg_layout(h, n, packed_bytes);
        // (segment and query indexes are 32-bit: larger batches take path 1)
        if (ws_bytes >= L.total + S.bytes && S.cap <= 0xffffffffull) {
            {
                StageScope sc(h, RAMBO_STAGE_PREFIX, s, kmer_prefix_launches(n));
                RAMBO_TRY(launch_kmer_prefix(offsets, ends, n, g.k, packed_bytes, kcum, bsum, h->d_err, s));
            }
            char *sw = w + L.total;
            RAMBO_TRY(cudaMemsetAsync(acc, 0xFF, n * (uint64_t)g.Gw * 4, s));
            RAMBO_TRY(cudaMemsetAsync(sw + S.hdr_off, 0, S.hdr_bytes, s));
            SegArgs sa{};
            ProbeArgs &a = sa.p;
            a.index = h->d_index;
            a.m = g.m;
            a.m_pow2 = (g.m & (g.m - 1)) == 0;
            a.Gw = g.Gw;
            a.eta = g.eta;
            a.k = g.k;
            a.seed32 = (uint32_t)g.seed;
            a.packed = al.p;
            a.packed_bytes = al.bytes;
            a.base_shift = al.base_shift;
            a.offsets = offsets;
            a.ends = ends;
            a.kcum = kcum;
            a.n = n;
            a.acc = acc;
            a.err = h->d_err;
            sa.cut_bits = S.cut_bits;
            sa.min_len = S.min_len;
            sa.bucket_shift = 32 - SEG_BUCKET_BITS;
            sa.nbuckets = 1u << SEG_BUCKET_BITS;
            sa.cap = S.cap;
            sa.ctr = reinterpret_cast<unsigned long long *>(sw + S.hdr_off);
            sa.bucket = reinterpret_cast<uint32_t *>(sw + S.hdr_off + ALIGN);
            sa.raw_begin = reinterpret_cast<uint64_t *>(sw + S.rbeg_off);
            sa.raw_len = reinterpret_cast<uint32_t *>(sw + S.rlen_off);
            sa.raw_q = reinterpret_cast<uint32_t *>(sw + S.rq_off);
            sa.raw_key = reinterpret_cast<uint32_t *>(sw + S.rkey_off);
            sa.sbeg = reinterpret_cast<uint64_t *>(sw + S.sbeg_off);
            sa.send = reinterpret_cast<uint64_t *>(sw + S.send_off);
            sa.sq = reinterpret_cast<uint32_t *>(sw + S.sq_off);
            sa.scum = reinterpret_cast<uint64_t *>(sw + S.scum_off);
            sa.chunk_seg = reinterpret_cast<uint32_t *>(sw + S.chunk_off);
            sa.max_chunks = S.max_chunks;
            {
                StageScope sc(h, RAMBO_STAGE_PROBE_SEQS, s,
                              seg_launches_before_prefix() + kmer_prefix_launches(S.cap) +
                                  seg_launches_after_prefix());
                RAMBO_TRY(launch_seg_order(sa, S.cut_grid, h->sm_count, s));
                RAMBO_TRY(launch_kmer_prefix(sa.sbeg, sa.send, S.cap, g.k, packed_bytes, sa.scum,
                                             reinterpret_cast<uint64_t *>(sw + S.sbsum_off), h->d_err, s));
                RAMBO_TRY(launch_seg_probe(sa, g, h->sm_count, s));
            }
            ExpandArgs e{acc, n, g.Gw, g.B, g.R, g.W, h->d_docbits, out, h->d_tab, h->tune.smem_docbits,
                         h->tune.use_nibble_table ? h->d_ntab : nullptr, h->d_phi, g.K,
                         h->tune.expand_filter};
            StageScope sc(h, RAMBO_STAGE_EXPAND, s, 1);
            RAMBO_TRY(launch_expand(e, h->sm_count * (int)h->tune.expand_ctas_per_sm, h->sm_count, s));
            return RAMBO_OK;
        }
    }
    if (h->tune.query_path >= 1 && fused_supported(g)) {
        // persistent fused query: length-bucketed queues, probe + expand in one launch
        ProbeArgs a{};
        a.index = h->d_index;
        a.m = g.m;
        a.m_pow2 = (g.m & (g.m - 1)) == 0;
        a.Gw = g.Gw;
        a.eta = g.eta;
        a.k = g.k;
        a.seed32 = (uint32_t)g.seed;
        a.packed = al.p;
        a.packed_bytes = al.bytes;
        a.base_shift = al.base_shift;
        a.offsets = offsets;
        a.ends = ends;
        a.n = n;
        a.err = h->d_err;
        ExpandArgs e{acc, n, g.Gw, g.B, g.R, g.W, h->d_docbits, out, h->d_tab, h->tune.smem_docbits,
                     h->tune.use_nibble_table ? h->d_ntab : nullptr, h->d_phi, g.K,
                     h->tune.expand_filter};
        FusedQueues qs{};
        qs.counters = reinterpret_cast<uint32_t *>(w + L.qcnt);
        qs.short_list = reinterpret_cast<uint32_t *>(w + L.slist);
        qs.tile_prefix = kcum;
        qs.done = reinterpret_cast<uint32_t *>(w + L.done);
        qs.heavy = reinterpret_cast<uint32_t *>(w + L.heavy);
        qs.tile = h->tune.fused_tile_kmers;
        qs.short_max = h->tune.fused_short_max;
        qs.user_bases = packed_bytes * 4;
        qs.early_exit = h->tune.early_exit;
        qs.segment = h->tune.early_exit_segment;
        qs.async = h->tune.fused_async;
        qs.probed = h->d_probed;
        {
            StageScope sc(h, RAMBO_STAGE_PREFIX, s, kmer_prefix_launches(n));
            RAMBO_TRY(launch_kmer_prefix(offsets, ends, n, g.k, packed_bytes, kcum, bsum, h->d_err, s,
                                         qs.tile, qs.short_max));
        }
        StageScope sc(h, RAMBO_STAGE_PROBE_SEQS, s, 3);
        uint32_t ctas = h->tune.probe_ctas_per_sm;
        if (fused_ctas_cap && (ctas == 0 || ctas > fused_ctas_cap)) ctas = fused_ctas_cap;
        const int go = ctas ? (int)(h->sm_count * ctas) : 0;
        RAMBO_TRY(launch_fused(a, e, g, qs, go, h->sm_count, s));
        return RAMBO_OK;
    }
    {
        StageScope sc(h, RAMBO_STAGE_PREFIX, s, kmer_prefix_launches(n));
        RAMBO_TRY(launch_kmer_prefix(offsets, ends, n, g.k, packed_bytes, kcum, bsum, h->d_err, s));
    }
    RAMBO_TRY(cudaMemsetAsync(acc, 0xFF, n * (uint64_t)g.Gw * 4, s));
    ProbeArgs a{};
    a.index = h->d_index;
    a.m = g.m;
    a.m_pow2 = (g.m & (g.m - 1)) == 0;
    a.Gw = g.Gw;
    a.eta = g.eta;
    a.k = g.k;
    a.seed32 = (uint32_t)g.seed;
    a.packed = al.p;
    a.packed_bytes = al.bytes;
    a.base_shift = al.base_shift;
    a.offsets = offsets;
    a.ends = ends;
    a.kcum = kcum;
    a.n = n;
    a.acc = acc;
    a.err = h->d_err;
    a.min_chunk = h->tune.probe_min_kmers_per_warp;
    {
        StageScope sc(h, RAMBO_STAGE_PROBE_SEQS, s, 1);
        RAMBO_TRY(launch_probe_seqs(a, g, probe_grid(h), s));
    }
    ExpandArgs e{acc, n, g.Gw, g.B, g.R, g.W, h->d_docbits, out, h->d_tab, h->tune.smem_docbits,
                     h->tune.use_nibble_table ? h->d_ntab : nullptr, h->d_phi, g.K,
                     h->tune.expand_filter};
    {
        StageScope sc(h, RAMBO_STAGE_EXPAND, s, 1);
        RAMBO_TRY(launch_expand(e, h->sm_count * (int)h->tune.expand_ctas_per_sm, h->sm_count, s));
    }
    return RAMBO_OK;
}

int query_kmers_enqueue(rambo_t *h, uint64_t n, const uint64_t *kmers, uint32_t *out, void *ws,
                        cudaStream_t s) {
    const Geometry &g = h->g;
    uint32_t *acc = static_cast<uint32_t *>(ws);
    if (g.eta > 4) RAMBO_TRY(cudaMemsetAsync(acc, 0xFF, n * (uint64_t)g.Gw * 4, s));
    ProbeArgs a{};
    a.index = h->d_index;
    a.m = g.m;
    a.m_pow2 = (g.m & (g.m - 1)) == 0;
    a.Gw = g.Gw;
    a.eta = g.eta;
    a.k = g.k;
    a.seed32 = (uint32_t)g.seed;
    a.kmers = kmers;
    a.n = n;
    a.acc = acc;
    a.err = h->d_err;
    a.min_chunk = h->tune.probe_min_kmers_per_warp;
    {
        StageScope sc(h, RAMBO_STAGE_PROBE_KMERS, s, 1);
        RAMBO_TRY(launch_probe_kmers(a, g, kmer_probe_grid(h), s, h->tune.kmer_async != 0));
    }
    ExpandArgs e{acc, n, g.Gw, g.B, g.R, g.W, h->d_docbits, out, h->d_tab, h->tune.smem_docbits,
                     h->tune.use_nibble_table ? h->d_ntab : nullptr, h->d_phi, g.K,
                     h->tune.expand_filter};
    {
        StageScope sc(h, RAMBO_STAGE_EXPAND, s, 1);
        RAMBO_TRY(launch_expand(e, h->sm_count * (int)h->tune.expand_ctas_per_sm, h->sm_count, s));
    }
    return RAMBO_OK;
}

// Documents are [begins[i], ends[i]); a CSR batch passes (offsets, offsets +
// 1).  Ranges that are not a CSR batch may overlap, so the region-binned
// insert (whose chunks assume at most one k-mer per packed base) is not used
// for them.
int insert_enqueue(rambo_t *h, uint64_t n, const uint32_t *doc_ids, const uint8_t *packed,
                   uint64_t packed_bytes, const uint64_t *offsets, const uint64_t *ends, void *ws,
                   cudaStream_t s) {
    const Geometry &g = h->g;
    h->any_inserted = true;
    const InsWs L = ins_ws(n);
    char *w = static_cast<char *>(ws);
    uint64_t *kcum = reinterpret_cast<uint64_t *>(w + L.kcum);
    uint64_t *bsum = reinterpret_cast<uint64_t *>(w + L.bsum);
    const Aligned al = align_packed(packed, packed_bytes);
    {
        StageScope sc(h, RAMBO_STAGE_REGISTER, s, 1);
        RAMBO_TRY(launch_register_docs(doc_ids, n, h->d_phi, g.K, g.R, g.B, g.W, h->d_docbits, h->d_err, s));
    }
    {
        StageScope sc(h, RAMBO_STAGE_PREFIX, s, kmer_prefix_launches(n));
        RAMBO_TRY(launch_kmer_prefix(offsets, ends, n, g.k, packed_bytes, kcum, bsum, h->d_err, s));
    }
    InsertArgs a{};
    a.index = h->d_index;
    a.m = g.m;
    a.m_pow2 = (g.m & (g.m - 1)) == 0;
    a.Gw = g.Gw;
    a.B = g.B;
    a.R = g.R;
    a.K = g.K;
    a.eta = g.eta;
    a.k = g.k;
    a.seed32 = (uint32_t)g.seed;
    a.phi = h->d_phi;
    a.doc_ids = doc_ids;
    a.packed = al.p;
    a.packed_bytes = al.bytes;
    a.base_shift = al.base_shift;
    a.offsets = offsets;
    a.kcum = kcum;
    a.n = n;
    a.err = h->d_err;
    a.mode = h->tune.insert_mode;
    uint32_t rshift = 0;
    uint32_t nbins =
        a.mode == 3 && h->d_bins && ends == offsets + 1
            ? binned_insert_bins(g.m, g.Gw * 4, g.K,
                                 (uint64_t)(h->tune.bin_region_kib ? h->tune.bin_region_kib : 32768) * 1024,
                                 &rshift)
            : 0;
    // chunks of the flat k-mer index sized to fill the record buffer (k-mers
    // <= bases; chunks past the batch's k-mers do nothing); a buffer far too
    // small for the batch takes the direct insert instead of a launch storm
    const uint64_t per = h->bins_records / g.eta > 0 ? h->bins_records / g.eta : 1;
    const uint64_t bound = packed_bytes * 4;
    const uint64_t chunks = (bound + per - 1) / per;
    if (chunks > IB_MAX_CHUNKS) nbins = 0;
    if (nbins) {
        BinnedInsert b{h->d_bins, h->d_bin_count, h->bins_records / nbins, nbins, rshift};
        StageScope sc(h, RAMBO_STAGE_INSERT, s, (int)(2 * chunks));
        for (uint64_t f0 = 0; f0 < bound; f0 += per) {
            RAMBO_TRY(cudaMemsetAsync(h->d_bin_count, 0, (IB_MAX_BINS + 1) * 4, s));
            RAMBO_TRY(launch_insert_binned(a, b, f0, f0 + per, h->sm_count, s));
        }
    } else {
        if (a.mode == 3) a.mode = 2;  // too many regions, or too many chunks
        StageScope sc(h, RAMBO_STAGE_INSERT, s, 1);
        RAMBO_TRY(launch_insert(a, h->sm_count, s));
    }
    if (h->d_tab) {
        StageScope sc(h, RAMBO_STAGE_REGISTER, s, 1);
        RAMBO_TRY(launch_build_bytetab(h->d_docbits, g.B, g.R, g.W, h->d_tab, h->sm_count, s));
    }
    if (h->d_ntab) {
        StageScope sc(h, RAMBO_STAGE_REGISTER, s, 1);
        RAMBO_TRY(launch_build_nibtab(h->d_docbits, g.B, g.R, g.W, h->d_ntab, h->sm_count, s));
    }
    return RAMBO_OK;
}

// Reads and clears the latched error word on the handle's own stream (the
// caller has already waited for the stream the kernels ran on).
// Return code of a latched error word.
int err_code(uint32_t e) {
    if (e & (ERR_QUEUE | ERR_WAIT)) return RAMBO_ETIMEOUT;
    if (e & ERR_DOC_RANGE) return RAMBO_ERANGE;
    if (e & (ERR_KMER_CODE | ERR_OFFSETS)) return RAMBO_EINVAL;
    return RAMBO_OK;
}

int read_and_clear_err(rambo_t *h) {
    uint32_t e = 0;
    RAMBO_TRY(cudaMemcpyAsync(&e, h->d_err, 4, cudaMemcpyDeviceToHost, h->stream));
    RAMBO_TRY(cudaStreamSynchronize(h->stream));
    if (e) {
        RAMBO_TRY(cudaMemsetAsync(h->d_err, 0, 4, h->stream));
        RAMBO_TRY(cudaStreamSynchronize(h->stream));
    }
    return err_code(e);
}

bool offsets_ok(uint64_t n, const uint64_t *offs) {
    for (uint64_t i = 0; i < n; ++i)
        if (offs[i + 1] < offs[i]) return false;
    return true;
}

// Copies the bytes holding bases [offs[0], offs[n]) of a host batch into the
// staging buffer (plus 16 zero bytes) and rebased offsets after it.
struct Staged {
    uint8_t *packed;
    uint64_t packed_bytes;
    uint64_t *offsets;
    char *rest;
};
int stage_batch(rambo_t *h, uint64_t n, const uint8_t *packed, const uint64_t *offs, size_t extra,
                Staged *st) {
    const uint64_t b_lo = offs[0] >> 2;
    const uint64_t b_hi = (offs[n] + 3) >> 2;
    const uint64_t nbytes = b_hi - b_lo;
    const size_t p_sz = align_up(nbytes + 16);
    const size_t o_sz = align_up((n + 1) * 8);
    int rc = reserve_stage(h, p_sz + o_sz + extra);
    if (rc) return rc;
    char *base = static_cast<char *>(h->d_stage);
    st->packed = reinterpret_cast<uint8_t *>(base);
    st->packed_bytes = nbytes;
    st->offsets = reinterpret_cast<uint64_t *>(base + p_sz);
    st->rest = base + p_sz + o_sz;
    uint64_t *reb = static_cast<uint64_t *>(std::malloc((n + 1) * 8));
    if (!reb) return RAMBO_ENOMEM;
    for (uint64_t i = 0; i <= n; ++i) reb[i] = offs[i] - 4 * b_lo;
    cudaError_t e = cudaMemcpyAsync(st->packed, packed + b_lo, nbytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(st->packed + nbytes, 0, 16, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st->offsets, reb, (n + 1) * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // reb is freed next
    std::free(reb);
    return cuda_rc(e);
}

int reserve_host_offsets(rambo_t *h, size_t bytes) {
    if (bytes <= h->h_offs_bytes) return RAMBO_OK;
    if (h->h_offs) cudaFreeHost(h->h_offs);
    h->h_offs = nullptr;
    h->h_offs_bytes = 0;
    const size_t want = bytes + bytes / 4;
    void *p = nullptr;
    RAMBO_TRY(cudaMallocHost(&p, want));
    h->h_offs = static_cast<uint64_t *>(p);
    h->h_offs_bytes = want;
    return RAMBO_OK;
}

// K-mers per chunk of a host-buffer k-mer batch: about 32 MiB of answers.
// K-mers per chunk of a host-buffer k-mer batch: about 16 MiB of answers
// unless the knob says otherwise.  The first chunk is an eighth of that, so
// the copy-out engine starts early.
uint64_t host_chunk(const rambo_t *h, uint64_t n) {
    uint64_t c = h->tune.host_chunk_kmers;
    if (!c) {
        c = (16ull << 20) / ((uint64_t)h->g.W * 4 + 8);
        if (c < (1u << 14)) c = 1u << 14;
    }
    return c < n ? c : n;
}
uint64_t host_chunk_begin(uint64_t c, uint64_t ck, uint64_t n) {
    if (c == 0) return 0;
    const uint64_t first = ck >= 8 ? ck / 8 : ck;
    const uint64_t b = first + (c - 1) * ck;
    return b < n ? b : n;
}

// Host-buffer mixed batch.  The sequence branch (copy in, query, copy out)
// runs on the handle's stream; the k-mer branch is cut into chunks that
// alternate over two more streams, so that one chunk's copies overlap the
// next chunk's kernels and both branches overlap each other.  Page-locked
// host buffers make every copy asynchronous; pageable ones still work (the
// runtime then copies synchronously).  Waits for all of it before returning.
int query_batch_host(rambo_t *h, uint64_t nk, const uint64_t *kmers, uint32_t *out_k, uint64_t ns,
                     const uint8_t *packed, const uint64_t *offs, uint32_t *out_s) {
    const Geometry &g = h->g;
    const uint64_t row = (uint64_t)g.W * 4;
    const uint64_t ck = nk ? host_chunk(h, nk) : 0;
    uint64_t nchunks = 0;
    while (nk && host_chunk_begin(nchunks, ck, nk) < nk) ++nchunks;
    const uint32_t want_slots = h->tune.host_slots ? h->tune.host_slots : 3;
    const int slots = (int)(nchunks < want_slots ? nchunks : want_slots);
    const size_t kin = align_up(ck * 8), kout = align_up(ck * row);
    const size_t kslot = kin + kout + kmers_ws(g, ck);
    uint64_t b_lo = 0, nbytes = 0;
    size_t p_sz = 0, o_sz = 0, s_out = 0, s_ws = 0;
    if (ns) {
        b_lo = offs[0] >> 2;
        nbytes = ((offs[ns] + 3) >> 2) - b_lo;
        p_sz = align_up(nbytes + 16);
        o_sz = align_up((ns + 1) * 8);
        s_out = align_up(ns * row);
        s_ws = seq_ws_for(h, ns, nbytes + 16);
    }
    const size_t seq_bytes = p_sz + o_sz + s_out + s_ws;
    int rc = reserve_stage(h, seq_bytes + (size_t)slots * kslot);
    if (rc) return rc;
    if (ns) {
        if ((rc = reserve_host_offsets(h, (ns + 1) * 8))) return rc;
        for (uint64_t i = 0; i <= ns; ++i) h->h_offs[i] = offs[i] - 4 * b_lo;
    }
    char *base = static_cast<char *>(h->d_stage);
    // on any failure: wait for what was enqueued, then report
    auto bail = [&](int code) {
        sync_own_streams(h);
        return code;
    };
    // branch_priority 1: sequences on a high-priority stream; 2: k-mer chunks
    // (chunk c uses slot c mod slots: its stream and its staging)
    cudaStream_t ss = h->tune.branch_priority == 1 ? h->pstream[0] : h->stream;
    cudaStream_t *ks = h->tune.branch_priority == 2 ? h->pstream : h->kstream;
    // host_direct: answers written by the kernels straight into page-locked
    // output buffers (device-addressable), instead of staged and copied
    uint32_t *direct_k = nullptr, *direct_s = nullptr;
    if (h->tune.host_direct) {
        if (nk) direct_k = static_cast<uint32_t *>(mapped_host_range(out_k, nk * row));
        if (ns) direct_s = static_cast<uint32_t *>(mapped_host_range(out_s, ns * row));
    }
    cudaError_t e = cudaEventRecord(h->ev_fork, h->stream);
    if (e != cudaSuccess) return bail(cuda_rc(e));
    if (ns && ss != h->stream && (e = cudaStreamWaitEvent(ss, h->ev_fork, 0)) != cudaSuccess)
        return bail(cuda_rc(e));
    if (ns) {
        uint8_t *d_p = reinterpret_cast<uint8_t *>(base);
        uint64_t *d_o = reinterpret_cast<uint64_t *>(base + p_sz);
        uint32_t *d_out = direct_s ? direct_s : reinterpret_cast<uint32_t *>(base + p_sz + o_sz);
        e = cudaMemcpyAsync(d_p, packed + b_lo, nbytes, cudaMemcpyHostToDevice, ss);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_p + nbytes, 0, 16, ss);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_o, h->h_offs, (ns + 1) * 8, cudaMemcpyHostToDevice, ss);
        if (e != cudaSuccess) return bail(cuda_rc(e));
        // with k-mer chunks beside it, the fused launch leaves room for them:
        // their copies out are what bounds a host call
        rc = query_seqs_enqueue(h, ns, d_p, nbytes + 16, d_o, d_o + 1, d_out,
                                base + p_sz + o_sz + s_out, s_ws, ss, nk ? h->tune.host_fused_ctas_per_sm : 0u);
        if (rc) return bail(rc);
        if (!direct_s) {
            e = cudaMemcpyAsync(out_s, d_out, ns * row, cudaMemcpyDeviceToHost, ss);
            if (e != cudaSuccess) return bail(cuda_rc(e));
        }
    }
    for (uint64_t c = 0; c < nchunks; ++c) {
        const int sl = (int)(c % (uint64_t)slots);
        cudaStream_t s = ks[sl];
        if (c < (uint64_t)slots && (e = cudaStreamWaitEvent(s, h->ev_fork, 0)) != cudaSuccess)
            return bail(cuda_rc(e));
        char *slot = base + seq_bytes + (size_t)sl * kslot;
        const uint64_t i0 = host_chunk_begin(c, ck, nk), cn = host_chunk_begin(c + 1, ck, nk) - i0;
        uint64_t *d_k = reinterpret_cast<uint64_t *>(slot);
        uint32_t *d_out = direct_k ? direct_k + i0 * g.W : reinterpret_cast<uint32_t *>(slot + kin);
        e = cudaMemcpyAsync(d_k, kmers + i0, cn * 8, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return bail(cuda_rc(e));
        rc = query_kmers_enqueue(h, cn, d_k, d_out, slot + kin + kout, s);
        if (rc) return bail(rc);
        if (!direct_k) {
            e = cudaMemcpyAsync(out_k + i0 * g.W, d_out, cn * row, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return bail(cuda_rc(e));
        }
    }
    // join every stream of the call into the handle's stream and read the
    // error word there: one wait for the whole call
    for (int sl = 0; sl < slots; ++sl) {
        if ((e = cudaEventRecord(h->ev_join, ks[sl])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(h->stream, h->ev_join, 0)) != cudaSuccess)
            return bail(cuda_rc(e));
    }
    if (ns && ss != h->stream &&
        ((e = cudaEventRecord(h->ev_join, ss)) != cudaSuccess ||
         (e = cudaStreamWaitEvent(h->stream, h->ev_join, 0)) != cudaSuccess))
        return bail(cuda_rc(e));
    e = cudaMemcpyAsync(h->h_err, h->d_err, 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return bail(cuda_rc(e));
    const uint32_t bits = *h->h_err;
    if (bits) {
        RAMBO_TRY(cudaMemsetAsync(h->d_err, 0, 4, h->stream));
        RAMBO_TRY(cudaStreamSynchronize(h->stream));
    }
    return err_code(bits);
}

}  // namespace

extern "C" {

const char *rambo_strerror(int code) {
    switch (code) {
        case RAMBO_OK: return "ok";
        case RAMBO_EINVAL: return "invalid argument";
        case RAMBO_ENOMEM: return "out of memory";
        case RAMBO_ECUDA: return "CUDA runtime error";
        case RAMBO_ERANGE: return "document id out of range";
        case RAMBO_ETIMEOUT: return "device wait timed out";
        case RAMBO_ESTATE: return "invalid state";
        default: return "unknown error";
    }
}

int rambo_create(uint32_t K, uint32_t B, uint32_t R, uint64_t m, uint32_t eta, uint32_t k,
                 uint64_t seed, int device, rambo_t **out) {
    if (!out || K == 0 || B == 0 || R == 0 || m == 0 || m > (1ULL << 32) || eta == 0 || eta > 64 ||
        k == 0 || k > 32)
        return RAMBO_EINVAL;
    if ((uint64_t)R * B > (1ULL << 24)) return RAMBO_EINVAL;
    if (device < 0 && cudaGetDevice(&device) != cudaSuccess) return RAMBO_ECUDA;
    DeviceGuard guard(device);
    if (!guard.ok) return RAMBO_ECUDA;
    rambo_t *h = new (std::nothrow) rambo();
    if (!h) return RAMBO_ENOMEM;
    h->g = make_geometry(K, B, R, m, eta, k, seed);
    h->device = device;
    int rc = RAMBO_OK;
    auto fail = [&](int code) {
        rambo_destroy(h);
        return code;
    };
    if ((rc = cuda_rc(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device))))
        return fail(rc);
    if ((rc = cuda_rc(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)))) return fail(rc);
    for (cudaStream_t &ks : h->kstream)
        if ((rc = cuda_rc(cudaStreamCreateWithFlags(&ks, cudaStreamNonBlocking)))) return fail(rc);
    {
        int least = 0, greatest = 0;
        if ((rc = cuda_rc(cudaDeviceGetStreamPriorityRange(&least, &greatest)))) return fail(rc);
        for (cudaStream_t &ps : h->pstream)
            if ((rc = cuda_rc(cudaStreamCreateWithPriority(&ps, cudaStreamNonBlocking, greatest))))
                return fail(rc);
    }
    if ((rc = cuda_rc(cudaMallocHost(reinterpret_cast<void **>(&h->h_err), sizeof(uint32_t))))) return fail(rc);
    if ((rc = cuda_rc(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming)))) return fail(rc);
    if ((rc = cuda_rc(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming)))) return fail(rc);
    if ((rc = cuda_rc(cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming)))) return fail(rc);
    const uint64_t index_bytes = m * (uint64_t)h->g.Gw * 4;
    const uint64_t docbits_bytes = (uint64_t)R * B * h->g.W * 4;
    if ((rc = cuda_rc(cudaMalloc(&h->d_index, index_bytes)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&h->d_docbits, docbits_bytes)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&h->d_phi, (uint64_t)K * R * 4)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&h->d_err, 4)))) return fail(rc);
    if ((rc = cuda_rc(cudaMalloc(&h->d_probed, 8)))) return fail(rc);
    if ((rc = cuda_rc(cudaMemsetAsync(h->d_probed, 0, 8, h->stream)))) return fail(rc);
    if ((rc = cuda_rc(cudaMemsetAsync(h->d_index, 0, index_bytes, h->stream)))) return fail(rc);
    if ((rc = cuda_rc(cudaMemsetAsync(h->d_docbits, 0, docbits_bytes, h->stream)))) return fail(rc);
    if ((rc = cuda_rc(cudaMemsetAsync(h->d_err, 0, 4, h->stream)))) return fail(rc);
    if ((rc = cuda_rc(launch_partition(h->d_phi, K, R, B, seed, h->stream)))) return fail(rc);
    if ((rc = cuda_rc(cudaStreamSynchronize(h->stream)))) return fail(rc);
    h->tune.probe_ctas_per_sm = 0;
    h->tune.probe_min_kmers_per_warp = 0;
    h->tune.expand_ctas_per_sm = 8;
    h->tune.use_byte_table = 1;
    h->tune.byte_table_max_mb = 64;
    h->tune.query_path = 0;
    h->tune.smem_docbits = 1;
    h->tune.use_nibble_table = 1;
    h->tune.expand_filter = 0;
    h->tune.early_exit = 0;
    h->tune.early_exit_segment = 256;
    h->tune.fused_tile_kmers = 1024;
    h->tune.fused_short_max = 1024;
    h->tune.kmer_probe_ctas_per_sm = 0;
    h->tune.host_chunk_kmers = 0;
    h->tune.branch_priority = 0;
    h->tune.host_slots = 3;
    h->tune.bin_region_kib = 32768;
    h->tune.bin_rows = 2;
    h->tune.seg_cut_bits = 6;
    h->tune.host_direct = 0;
    h->tune.host_fused_ctas_per_sm = 1;
    h->tune.insert_mode = 2;
    h->tune.insert_bin_records = 0;
    h->tune.fused_async = 0;
    h->tune.kmer_async = 0;
    if ((rc = apply_bytetab(h))) return fail(rc);
    *out = h;
    return RAMBO_OK;
}

int rambo_destroy(rambo_t *h) {
    if (!h) return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (cudaStream_t ks : h->kstream)
        if (ks) cudaStreamSynchronize(ks);
    for (cudaStream_t ps : h->pstream)
        if (ps) cudaStreamSynchronize(ps);
    cudaFree(h->d_index);
    cudaFree(h->d_docbits);
    cudaFree(h->d_phi);
    cudaFree(h->d_err);
    cudaFree(h->d_probed);
    cudaFree(h->d_stage);
    cudaFree(h->d_tab);
    cudaFree(h->d_ntab);
    cudaFree(h->d_bins);
    cudaFree(h->d_bin_count);
    for (auto &p : h->pending) {
        cudaEventDestroy(p.start);
        cudaEventDestroy(p.stop);
    }
    for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
    if (h->h_offs) cudaFreeHost(h->h_offs);
    if (h->h_err) cudaFreeHost(h->h_err);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_join2) cudaEventDestroy(h->ev_join2);
    for (cudaStream_t ks : h->kstream)
        if (ks) cudaStreamDestroy(ks);
    for (cudaStream_t ps : h->pstream)
        if (ps) cudaStreamDestroy(ps);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return RAMBO_OK;
}

uint32_t rambo_mask_words(const rambo_t *h) { return h ? h->g.W : 0; }

int rambo_get_info(const rambo_t *h, rambo_info_t *info) {
    if (!h || !info) return RAMBO_EINVAL;
    const Geometry &g = h->g;
    info->K = g.K; info->B = g.B; info->R = g.R; info->eta = g.eta; info->k = g.k;
    info->m = g.m; info->seed = g.seed;
    info->mask_words = g.W;
    info->group_bytes = g.Gw * 4;
    info->index_bytes = g.m * (uint64_t)g.Gw * 4;
    info->docbits_bytes = (uint64_t)g.R * g.B * g.W * 4;
    info->device = h->device;
    return RAMBO_OK;
}

size_t rambo_insert_workspace(const rambo_t *h, uint64_t n_docs) {
    return h ? ins_ws(n_docs).total : 0;
}
size_t rambo_query_kmers_workspace(const rambo_t *h, uint64_t n) {
    return h ? kmers_ws(h->g, n) : 0;
}
size_t rambo_query_seqs_workspace(const rambo_t *h, uint64_t n) {
    return h ? seq_ws(h->g, n).total : 0;
}
size_t rambo_query_seqs_workspace_for(const rambo_t *h, uint64_t n, uint64_t packed_bytes) {
    return h ? seq_ws_for(h, n, packed_bytes) : 0;
}

// ----------------------------------------------------------------- device

int rambo_insert_batch_dev(rambo_t *h, uint32_t n_docs, const uint32_t *doc_ids,
                           const uint8_t *packed, uint64_t packed_bytes,
                           const uint64_t *base_offsets, void *workspace, size_t workspace_bytes,
                           void *stream) {
    if (!h) return RAMBO_EINVAL;
    if (n_docs == 0) return RAMBO_OK;
    if (!doc_ids || !base_offsets || !workspace || (!packed && packed_bytes) ||
        workspace_bytes < ins_ws(n_docs).total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    return insert_enqueue(h, n_docs, doc_ids, packed, packed_bytes, base_offsets, base_offsets + 1, workspace,
                          static_cast<cudaStream_t>(stream));
}

int rambo_insert_ranges_dev(rambo_t *h, uint32_t n_docs, const uint32_t *doc_ids,
                            const uint8_t *packed, uint64_t packed_bytes, const uint64_t *begins,
                            const uint64_t *ends, void *workspace, size_t workspace_bytes,
                            void *stream) {
    if (!h) return RAMBO_EINVAL;
    if (n_docs == 0) return RAMBO_OK;
    if (!doc_ids || !begins || !ends || !workspace || (!packed && packed_bytes) ||
        workspace_bytes < ins_ws(n_docs).total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    return insert_enqueue(h, n_docs, doc_ids, packed, packed_bytes, begins, ends, workspace,
                          static_cast<cudaStream_t>(stream));
}

int rambo_merge_shard_answers(uint64_t n, const uint32_t *shard_masks, uint32_t shard_words,
                              uint32_t shard_docs, const uint32_t *global_ids, uint32_t *out,
                              uint32_t out_words, void *stream) {
    if (n == 0 || shard_docs == 0) return RAMBO_OK;
    if (!shard_masks || !global_ids || !out || shard_words < (shard_docs + 31) / 32 || out_words == 0)
        return RAMBO_EINVAL;
    return cuda_rc(launch_merge_shard(n, shard_masks, shard_words, shard_docs, global_ids, out, out_words,
                                      static_cast<cudaStream_t>(stream)));
}

int rambo_query_kmers_dev(rambo_t *h, uint64_t n, const uint64_t *kmers, uint32_t *out,
                          void *workspace, size_t workspace_bytes, void *stream) {
    if (!h) return RAMBO_EINVAL;
    if (n == 0) return RAMBO_OK;
    if (!kmers || !out || !workspace || workspace_bytes < kmers_ws(h->g, n) ||
        (reinterpret_cast<uintptr_t>(workspace) & 255))
        return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    return query_kmers_enqueue(h, n, kmers, out, workspace, static_cast<cudaStream_t>(stream));
}

int rambo_query_seqs_dev(rambo_t *h, uint64_t n, const uint8_t *packed, uint64_t packed_bytes,
                         const uint64_t *base_offsets, uint32_t *out, void *workspace,
                         size_t workspace_bytes, void *stream) {
    if (!h) return RAMBO_EINVAL;
    if (n == 0) return RAMBO_OK;
    if (n >= 0xffffffffULL || !base_offsets || !out || !workspace || (!packed && packed_bytes) ||
        workspace_bytes < seq_ws(h->g, n).total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    return query_seqs_enqueue(h, n, packed, packed_bytes, base_offsets, base_offsets + 1, out,
                              workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
}

int rambo_query_ranges_dev(rambo_t *h, uint64_t n, const uint8_t *packed, uint64_t packed_bytes,
                           const uint64_t *begins, const uint64_t *ends, uint32_t *out,
                           void *workspace, size_t workspace_bytes, void *stream) {
    if (!h) return RAMBO_EINVAL;
    if (n == 0) return RAMBO_OK;
    if (n >= 0xffffffffULL || !begins || !ends || !out || !workspace || (!packed && packed_bytes) ||
        workspace_bytes < seq_ws(h->g, n).total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    return query_seqs_enqueue(h, n, packed, packed_bytes, begins, ends, out, workspace,
                              workspace_bytes, static_cast<cudaStream_t>(stream));
}

size_t rambo_query_batch_workspace(const rambo_t *h, uint64_t n_kmers, uint64_t n_seqs,
                                   uint64_t packed_bytes) {
    if (!h) return 0;
    return (n_kmers ? kmers_ws(h->g, n_kmers) : 0) +
           (n_seqs ? seq_ws_for(h, n_seqs, packed_bytes + 8) : 0);
}

int rambo_query_batch_dev(rambo_t *h, uint64_t n_kmers, const uint64_t *kmers, uint32_t *out_kmers,
                          uint64_t n_seqs, const uint8_t *packed, uint64_t packed_bytes,
                          const uint64_t *base_offsets, uint32_t *out_seqs, void *workspace,
                          size_t workspace_bytes, void *stream) {
    if (!h) return RAMBO_EINVAL;
    if (n_kmers == 0 && n_seqs == 0) return RAMBO_OK;
    if ((n_kmers && (!kmers || !out_kmers)) ||
        (n_seqs && (n_seqs >= 0xffffffffULL || !base_offsets || !out_seqs || (!packed && packed_bytes))) ||
        !workspace || workspace_bytes < (n_kmers ? kmers_ws(h->g, n_kmers) : 0) +
                                            (n_seqs ? seq_ws(h->g, n_seqs).total : 0) ||
        (reinterpret_cast<uintptr_t>(workspace) & 255))
        return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(workspace);
    if (!n_seqs) return query_kmers_enqueue(h, n_kmers, kmers, out_kmers, w, s);
    char *wseq = w + (n_kmers ? kmers_ws(h->g, n_kmers) : 0);
    if (!n_kmers)
        return query_seqs_enqueue(h, n_seqs, packed, packed_bytes, base_offsets, base_offsets + 1,
                                  out_seqs, wseq, workspace_bytes - (size_t)(wseq - w), s);
    // fork the k-mer branch onto a stream of the handle and join it back, so
    // that both branches run at once (also inside a stream capture);
    // branch_priority 1 moves the sequence branch to a high-priority stream
    // of the handle, 2 puts the k-mer branch on one
    const uint32_t prio = h->tune.branch_priority;
    cudaStream_t sk = prio == 2 ? h->pstream[0] : h->kstream[0];
    cudaStream_t ss = prio == 1 ? h->pstream[1] : s;
    RAMBO_TRY(cudaEventRecord(h->ev_fork, s));
    RAMBO_TRY(cudaStreamWaitEvent(sk, h->ev_fork, 0));
    if (ss != s) RAMBO_TRY(cudaStreamWaitEvent(ss, h->ev_fork, 0));
    const int rk = query_kmers_enqueue(h, n_kmers, kmers, out_kmers, w, sk);
    const int rs = query_seqs_enqueue(h, n_seqs, packed, packed_bytes, base_offsets, base_offsets + 1,
                                      out_seqs, wseq, workspace_bytes - (size_t)(wseq - w), ss);
    RAMBO_TRY(cudaEventRecord(h->ev_join, sk));
    RAMBO_TRY(cudaStreamWaitEvent(s, h->ev_join, 0));
    if (ss != s) {
        RAMBO_TRY(cudaEventRecord(h->ev_join2, ss));
        RAMBO_TRY(cudaStreamWaitEvent(s, h->ev_join2, 0));
    }
    return rk ? rk : rs;
}

int rambo_probe_wait_expiry(rambo_t *h, uint64_t spins, void *stream) {
    if (!h || spins == 0 || spins > (1ull << 22)) return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    return cuda_rc(launch_wait_expiry(h->d_err, spins, static_cast<cudaStream_t>(stream)));
}

int rambo_sync(rambo_t *h, void *stream) {
    if (!h) return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    RAMBO_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return read_and_clear_err(h);
}

// ------------------------------------------------------------------- host

int rambo_insert_batch(rambo_t *h, uint32_t n_docs, const uint32_t *doc_ids,
                       const uint8_t *packed, const uint64_t *base_offsets) {
    if (!h) return RAMBO_EINVAL;
    if (n_docs == 0) return RAMBO_OK;
    if (!doc_ids || !base_offsets || !offsets_ok(n_docs, base_offsets)) return RAMBO_EINVAL;
    if (!packed && base_offsets[n_docs] > base_offsets[0]) return RAMBO_EINVAL;
    for (uint32_t i = 0; i < n_docs; ++i)
        if (doc_ids[i] >= h->g.K) return RAMBO_ERANGE;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    const size_t ids_sz = align_up((size_t)n_docs * 4);
    Staged st;
    int rc = stage_batch(h, n_docs, packed, base_offsets, ids_sz + ins_ws(n_docs).total, &st);
    if (rc) return rc;
    uint32_t *d_ids = reinterpret_cast<uint32_t *>(st.rest);
    RAMBO_TRY(cudaMemcpyAsync(d_ids, doc_ids, (size_t)n_docs * 4, cudaMemcpyHostToDevice, h->stream));
    rc = insert_enqueue(h, n_docs, d_ids, st.packed, st.packed_bytes + 16, st.offsets, st.offsets + 1,
                        st.rest + ids_sz, h->stream);
    if (rc) return rc;
    RAMBO_TRY(cudaStreamSynchronize(h->stream));
    return read_and_clear_err(h);
}

int rambo_insert(rambo_t *h, uint32_t doc_id, const uint8_t *packed, uint64_t n_bases) {
    const uint64_t offs[2] = {0, n_bases};
    return rambo_insert_batch(h, 1, &doc_id, packed, offs);
}

int rambo_query_kmers(rambo_t *h, uint64_t n, const uint64_t *kmers, uint32_t *out) {
    return rambo_query_batch(h, n, kmers, out, 0, nullptr, nullptr, nullptr);
}

int rambo_query_seqs(rambo_t *h, uint64_t n, const uint8_t *packed, const uint64_t *base_offsets,
                     uint32_t *out) {
    return rambo_query_batch(h, 0, nullptr, nullptr, n, packed, base_offsets, out);
}

int rambo_query_batch(rambo_t *h, uint64_t n_kmers, const uint64_t *kmers, uint32_t *out_kmers,
                      uint64_t n_seqs, const uint8_t *packed, const uint64_t *base_offsets,
                      uint32_t *out_seqs) {
    if (!h) return RAMBO_EINVAL;
    if (n_kmers && (!kmers || !out_kmers)) return RAMBO_EINVAL;
    if (n_seqs) {
        if (n_seqs >= 0xffffffffULL || !base_offsets || !out_seqs || !offsets_ok(n_seqs, base_offsets))
            return RAMBO_EINVAL;
        if (!packed && base_offsets[n_seqs] > base_offsets[0]) return RAMBO_EINVAL;
    }
    if (n_kmers == 0 && n_seqs == 0) return RAMBO_OK;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    return query_batch_host(h, n_kmers, kmers, out_kmers, n_seqs, packed, base_offsets, out_seqs);
}

// ---------------------------------------------------- documents of words

int rambo_insert_words_dev(rambo_t *h, uint32_t n_docs, const uint32_t *doc_ids,
                           const uint8_t *bytes, uint64_t bytes_len, const uint64_t *term_offs,
                           const uint64_t *doc_terms, void *stream) {
    if (!h) return RAMBO_EINVAL;
    if (n_docs == 0) return RAMBO_OK;
    if (!doc_ids || !term_offs || !doc_terms || (!bytes && bytes_len)) return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Geometry &g = h->g;
    h->any_inserted = true;
    {
        StageScope sc(h, RAMBO_STAGE_REGISTER, s, 1);
        RAMBO_TRY(launch_register_docs(doc_ids, n_docs, h->d_phi, g.K, g.R, g.B, g.W, h->d_docbits,
                                       h->d_err, s));
    }
    WordArgs a{};
    a.index = h->d_index;
    a.m = g.m;
    a.m_pow2 = (g.m & (g.m - 1)) == 0;
    a.Gw = g.Gw; a.B = g.B; a.R = g.R; a.K = g.K; a.eta = g.eta;
    a.seed32 = (uint32_t)g.seed;
    a.phi = h->d_phi;
    a.doc_ids = doc_ids;
    a.bytes = bytes;
    a.bytes_len = bytes_len;
    a.term_offs = term_offs;
    a.item_terms = doc_terms;
    a.n = n_docs;
    a.err = h->d_err;
    {
        StageScope sc(h, RAMBO_STAGE_INSERT, s, 1);
        RAMBO_TRY(launch_insert_words(a, h->sm_count, s));
    }
    if (h->d_tab) RAMBO_TRY(launch_build_bytetab(h->d_docbits, g.B, g.R, g.W, h->d_tab, h->sm_count, s));
    if (h->d_ntab) RAMBO_TRY(launch_build_nibtab(h->d_docbits, g.B, g.R, g.W, h->d_ntab, h->sm_count, s));
    return RAMBO_OK;
}

size_t rambo_query_words_workspace(const rambo_t *h, uint64_t n) {
    return h ? align_up(n * (uint64_t)h->g.Gw * 4) : 0;
}

int rambo_query_words_dev(rambo_t *h, uint64_t n, const uint8_t *bytes, uint64_t bytes_len,
                          const uint64_t *term_offs, const uint64_t *query_terms, uint32_t *out,
                          void *workspace, size_t workspace_bytes, void *stream) {
    if (!h) return RAMBO_EINVAL;
    if (n == 0) return RAMBO_OK;
    if (!term_offs || !query_terms || !out || !workspace || (!bytes && bytes_len) ||
        workspace_bytes < align_up(n * (uint64_t)h->g.Gw * 4) ||
        (reinterpret_cast<uintptr_t>(workspace) & 255))
        return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Geometry &g = h->g;
    uint32_t *acc = static_cast<uint32_t *>(workspace);
    RAMBO_TRY(cudaMemsetAsync(acc, 0xFF, n * (uint64_t)g.Gw * 4, s));
    WordArgs a{};
    a.index_ro = h->d_index;
    a.m = g.m;
    a.m_pow2 = (g.m & (g.m - 1)) == 0;
    a.Gw = g.Gw; a.B = g.B; a.R = g.R; a.K = g.K; a.eta = g.eta;
    a.seed32 = (uint32_t)g.seed;
    a.bytes = bytes;
    a.bytes_len = bytes_len;
    a.term_offs = term_offs;
    a.item_terms = query_terms;
    a.n = n;
    a.acc = acc;
    a.err = h->d_err;
    {
        StageScope sc(h, RAMBO_STAGE_PROBE_SEQS, s, 1);
        RAMBO_TRY(launch_probe_words(a, h->sm_count, s));
    }
    ExpandArgs e{acc, n, g.Gw, g.B, g.R, g.W, h->d_docbits, out, h->d_tab, h->tune.smem_docbits,
                 h->tune.use_nibble_table ? h->d_ntab : nullptr, h->d_phi, g.K, h->tune.expand_filter};
    {
        StageScope sc(h, RAMBO_STAGE_EXPAND, s, 1);
        RAMBO_TRY(launch_expand(e, h->sm_count * (int)h->tune.expand_ctas_per_sm, h->sm_count, s));
    }
    return RAMBO_OK;
}

// -------------------------------------------------------- explicit partition

int rambo_set_partition(rambo_t *h, const uint32_t *phi) {
    if (!h || !phi) return RAMBO_EINVAL;
    if (h->any_inserted) return RAMBO_ESTATE;
    const uint64_t n = (uint64_t)h->g.K * h->g.R;
    for (uint64_t i = 0; i < n; ++i)
        if (phi[i] >= h->g.B) return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    RAMBO_TRY(cudaStreamSynchronize(h->stream));
    RAMBO_TRY(cudaMemcpy(h->d_phi, phi, n * 4, cudaMemcpyHostToDevice));
    return RAMBO_OK;
}

// ---------------------------------------------------------------- folding

int rambo_fold(rambo_t *h) {
    if (!h) return RAMBO_EINVAL;
    const Geometry old = h->g;
    if (old.B < 2 || (old.B & 1) || old.Gw > 128) return RAMBO_EINVAL;
    const Geometry ng = make_geometry(old.K, old.B / 2, old.R, old.m, old.eta, old.k, old.seed);
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    RAMBO_TRY(cudaStreamSynchronize(h->stream));
    uint32_t *ni = nullptr, *nd = nullptr, *np = nullptr;
    const uint64_t ni_bytes = ng.m * (uint64_t)ng.Gw * 4;
    const uint64_t nd_bytes = (uint64_t)ng.R * ng.B * ng.W * 4;
    int rc = cuda_rc(cudaMalloc(&ni, ni_bytes));
    if (!rc) rc = cuda_rc(cudaMalloc(&nd, nd_bytes));
    if (!rc) rc = cuda_rc(cudaMalloc(&np, (uint64_t)ng.K * ng.R * 4));
    if (!rc) rc = cuda_rc(launch_fold(h->d_index, old.Gw, ni, ng.Gw, old.m, old.B, old.R, h->d_docbits,
                                      nd, old.W, h->sm_count, h->stream));
    // the folded partition is phi_r(d) mod B/2 = hash mod B/2, since B/2 divides B
    if (!rc) rc = cuda_rc(launch_partition(np, ng.K, ng.R, ng.B, ng.seed, h->stream));
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(h->stream));
    if (rc) {
        cudaFree(ni);
        cudaFree(nd);
        cudaFree(np);
        return rc;  // the index is unchanged
    }
    cudaFree(h->d_index);
    cudaFree(h->d_docbits);
    cudaFree(h->d_phi);
    h->d_index = ni;
    h->d_docbits = nd;
    h->d_phi = np;
    h->g = ng;
    if (h->d_tab) {
        cudaFree(h->d_tab);
        h->d_tab = nullptr;
    }
    if (h->d_ntab) {
        cudaFree(h->d_ntab);
        h->d_ntab = nullptr;
    }
    return apply_bytetab(h);
}

// --------------------------------------------------------- introspection

int rambo_copy_index(const rambo_t *h, uint64_t offset, uint64_t nbytes, void *dst) {
    if (!h || (!dst && nbytes)) return RAMBO_EINVAL;
    const uint64_t total = h->g.m * (uint64_t)h->g.Gw * 4;
    if (offset > total || nbytes > total - offset) return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    RAMBO_TRY(cudaStreamSynchronize(h->stream));
    RAMBO_TRY(cudaMemcpy(dst, reinterpret_cast<const char *>(h->d_index) + offset, nbytes,
                         cudaMemcpyDeviceToHost));
    return RAMBO_OK;
}

int rambo_copy_docbits(const rambo_t *h, uint32_t *dst) {
    if (!h || !dst) return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    RAMBO_TRY(cudaStreamSynchronize(h->stream));
    RAMBO_TRY(cudaMemcpy(dst, h->d_docbits, (uint64_t)h->g.R * h->g.B * h->g.W * 4,
                         cudaMemcpyDeviceToHost));
    return RAMBO_OK;
}

int rambo_copy_partition(const rambo_t *h, uint32_t *dst) {
    if (!h || !dst) return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    RAMBO_TRY(cudaMemcpy(dst, h->d_phi, (uint64_t)h->g.K * h->g.R * 4, cudaMemcpyDeviceToHost));
    return RAMBO_OK;
}

int rambo_get_tuning(const rambo_t *h, rambo_tuning_t *out) {
    if (!h || !out) return RAMBO_EINVAL;
    *out = h->tune;
    return RAMBO_OK;
}

// The binned insert's record buffer, reserved when insert_mode 3 is chosen
// (never during an insert, so that a captured insert allocates nothing) and
// released when another mode is chosen.  The handle keeps its old buffer if
// the new one cannot be had.
static int reserve_bins(rambo_t *h, const rambo_tuning_t *t) {
    if (t->insert_mode != 3) {
        cudaFree(h->d_bins);
        cudaFree(h->d_bin_count);
        h->d_bins = nullptr;
        h->d_bin_count = nullptr;
        h->bins_records = 0;
        return RAMBO_OK;
    }
    const uint64_t want = t->insert_bin_records ? t->insert_bin_records : (1ull << 28);
    if (h->d_bins && h->bins_records == want) return RAMBO_OK;
    unsigned long long *buf = nullptr;
    uint32_t *cnt = nullptr;
    if (cudaMalloc(&buf, want * 8) != cudaSuccess || cudaMalloc(&cnt, (IB_MAX_BINS + 1) * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(buf);
        return RAMBO_ENOMEM;
    }
    cudaFree(h->d_bins);
    cudaFree(h->d_bin_count);
    h->d_bins = buf;
    h->d_bin_count = cnt;
    h->bins_records = want;
    return RAMBO_OK;
}

int rambo_set_tuning(rambo_t *h, const rambo_tuning_t *t) {
    if (!h || !t) return RAMBO_EINVAL;
    if (t->probe_ctas_per_sm > 32 || t->expand_ctas_per_sm == 0 || t->expand_ctas_per_sm > 64 ||
        t->probe_min_kmers_per_warp > (1u << 24) || t->query_path > 3 || t->fused_tile_kmers == 0 ||
        t->fused_tile_kmers > (1u << 24) || t->fused_short_max > (1u << 24) || t->smem_docbits > 1 ||
        t->use_nibble_table > 1 || t->expand_filter > 1 || t->early_exit > 1 ||
        t->early_exit_segment == 0 || (t->early_exit_segment & 127) || t->early_exit_segment > (1u << 24) ||
        t->kmer_probe_ctas_per_sm > 32 || t->host_chunk_kmers > (1u << 30) || t->branch_priority > 2 ||
        t->host_slots == 0 || t->host_slots > RAMBO_MAX_HOST_SLOTS || t->bin_region_kib > (1u << 22) ||
        (t->bin_rows != 0 && t->bin_rows != 1 && t->bin_rows != 2 && t->bin_rows != 4 && t->bin_rows != 8) ||
        t->seg_cut_bits > 10 ||
        t->host_direct > 1 || t->host_fused_ctas_per_sm > 32 ||
        t->insert_mode > 3 || (t->insert_bin_records != 0 && t->insert_bin_records < 4096) ||
        t->fused_async > 1 || t->kmer_async > 1)
        return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    RAMBO_TRY(sync_own_streams(h));
    const int rc = reserve_bins(h, t);
    if (rc) return rc;
    h->tune = *t;
    return apply_bytetab(h);
}

int rambo_probed_kmers(rambo_t *h, uint64_t *out, int reset) {
    if (!h || !out) return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    unsigned long long v = 0;
    RAMBO_TRY(cudaDeviceSynchronize());
    RAMBO_TRY(cudaMemcpy(&v, h->d_probed, 8, cudaMemcpyDeviceToHost));
    if (reset) RAMBO_TRY(cudaMemset(h->d_probed, 0, 8));
    RAMBO_TRY(cudaDeviceSynchronize());
    *out = v;
    return RAMBO_OK;
}

int rambo_profile_reset(rambo_t *h, uint32_t stage_mask) {
    if (!h) return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    for (auto &p : h->pending) {
        cudaEventSynchronize(p.stop);
        h->event_pool.push_back(p.start);
        h->event_pool.push_back(p.stop);
    }
    h->pending.clear();
    h->prof_mask = stage_mask;
    for (int i = 0; i < RAMBO_NUM_STAGES; ++i) {
        h->launches[i] = 0;
        h->timed[i] = 0;
        h->ms[i] = 0.0;
    }
    return RAMBO_OK;
}

int rambo_profile_read(rambo_t *h, rambo_profile_t *out) {
    if (!h || !out) return RAMBO_EINVAL;
    DeviceGuard guard(h->device);
    if (!guard.ok) return RAMBO_ECUDA;
    for (auto &p : h->pending) {
        RAMBO_TRY(cudaEventSynchronize(p.stop));
        float ms = 0.f;
        RAMBO_TRY(cudaEventElapsedTime(&ms, p.start, p.stop));
        h->ms[p.stage] += ms;
        h->timed[p.stage] += 1;
        h->event_pool.push_back(p.start);
        h->event_pool.push_back(p.stop);
    }
    h->pending.clear();
    for (int i = 0; i < RAMBO_NUM_STAGES; ++i) {
        out->launches[i] = h->launches[i];
        out->timed[i] = h->timed[i];
        out->ms[i] = h->ms[i];
    }
    return RAMBO_OK;
}

}  // extern "C"

// rambo_kernels_segments.cu -- query path 3: the membership tests of
// Algorithm 2 (Section 3.3.1) over a batch reordered by content.
//
// A probe of a large index reads a random 128-byte DRAM line; the fused path
// moves its lines at the copy bandwidth, so it can only go faster by reading
// fewer of them.  Query batches repeat k-mers: reads of one genome overlap,
// and a k-mer probed twice reads the same groups twice.  Here each query's
// k-mers are cut into segments at content-defined points, the segments of
// the whole batch are ordered by a hash of their first k-mer, and the probes
// run in that order: the same stretch of sequence in two queries gives the
// same segment with the same key, so its second copy is probed right after
// the first and finds its lines in L2.
//   cut     every k-mer gets a 32-bit order hash of its canonical code; a
//           k-mer starts a segment when the low cut_bits bits of its hash are
//           zero and the previous start is at least min_len k-mers back, or
//           when it is the first k-mer of a query or of the warp's range.
//           Segments never span two queries.  Each is recorded as (first
//           base, k-mers, query, key = hash of its first k-mer), and counted
//           in bucket key >> bucket_shift.
//   place   the bucket counts become offsets (one block), and every segment
//           moves to a slot of its bucket; unused slots become empty ranges.
//   prefix  the k-mer prefix of the ordered segments (the shared prefix
//           kernels), and the segment holding every PSK-th k-mer of it.
//   probe   work items of NS x PSK consecutive k-mers of the ordered batch
//           are claimed in order from a counter, so the warps in flight stay
//           within a narrow window of the order.  A group of LPG lanes walks
//           PSK k-mers: its lanes hash the next k-mers, exchange the probe
//           positions, gather their slices of all eta groups of each, and
//           AND them per segment; a segment's AND goes to its query's bucket
//           mask with one coalesced atomicAnd per mask row when the segment
//           (or the lane group's PSK k-mers) ends.
// The bucket mask of a query is the AND over all its probed groups, so the
// result does not depend on how the k-mers are cut or ordered: the cut rule
// and the hash only decide the speed.
#include "rambo_query_common.cuh"

namespace rgpu {
namespace {

constexpr int SEG_THREADS = 256;
constexpr uint32_t SEG_MIN_RANGE = 2048;  // k-mers per warp in the cut pass, at least
constexpr int SEG_PSK = 16;               // k-mers per lane group and work item
constexpr uint64_t SEG_MAX_LEN = 1ull << 30;  // a start is forced this far after the last one

// Order hash of a canonical code: the high word of one multiply-xorshift round
// (only the order of the probes depends on it).
__device__ __forceinline__ uint32_t order_hash(uint64_t c) {
    uint64_t x = (c ^ (c >> 31)) * 0xbf58476d1ce4e5b9ULL;
    x ^= x >> 29;
    return (uint32_t)(x >> 32);
}

// Cut pass.  Each warp walks a contiguous range of the batch's flattened
// k-mer index 32 k-mers at a time; the start decisions of a step are settled
// in index order from the ballot of candidates (the minimum length makes
// each depend on the previous one).  A start closes the segment before it;
// the warp collects closed segments in shared memory and appends them in
// runs (one atomicAdd on the shared counter per run, coalesced stores).
constexpr int SEG_CUT_BUF = 128;  // closed segments a warp buffers before appending them

__global__ void __launch_bounds__(SEG_THREADS) k_seg_cut(SegArgs a) {
    // per warp: closed segments collected in shared memory and appended to
    // the recorded list with one atomicAdd per SEG_CUT_BUF of them
    __shared__ uint64_t s_beg[SEG_THREADS / 32][SEG_CUT_BUF];
    __shared__ uint32_t s_len[SEG_THREADS / 32][SEG_CUT_BUF];
    __shared__ uint32_t s_q[SEG_THREADS / 32][SEG_CUT_BUF];
    __shared__ uint32_t s_key[SEG_THREADS / 32][SEG_CUT_BUF];
    const ProbeArgs &p = a.p;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint64_t T = p.kcum[p.n];
    uint64_t c0, c1;
    warp_range<32>(T, SEG_MIN_RANGE, c0, c1);
    if (c0 >= T) return;
    uint64_t qlane = find_query(p.kcum, p.n, c0);
    const uint32_t cut_mask = (1u << a.cut_bits) - 1u;
    // the open segment (warp-uniform): first k-mer index, first base, key, query
    uint64_t o_start = ~0ull, o_beg = 0, last_kept = c0;  // (c0 is a forced start)
    uint32_t o_key = 0, o_q = 0;
    uint32_t buffered = 0;  // warp-uniform
    auto flush = [&]() {
        __syncwarp();
        unsigned long long slot0 = 0;
        if (lane == 0) slot0 = atomicAdd(a.ctr, (unsigned long long)buffered);
        slot0 = __shfl_sync(FULL, slot0, 0);
        for (uint32_t i = lane; i < buffered; i += 32) {
            const uint64_t slot = slot0 + i;
            if (slot < a.cap) {
                a.raw_begin[slot] = s_beg[wib][i];
                a.raw_len[slot] = s_len[wib][i];
                a.raw_q[slot] = s_q[wib][i];
                a.raw_key[slot] = s_key[wib][i];
                atomicAdd(a.bucket + (s_key[wib][i] >> a.bucket_shift), 1u);
            } else {
                atomicOr(p.err, ERR_QUEUE);  // cannot happen: cap bounds the segments
            }
        }
        __syncwarp();
        buffered = 0;
    };
    auto emit = [&](bool e, uint64_t start, uint64_t beg, uint64_t end_idx, uint32_t key, uint32_t q) {
        const uint32_t em = __ballot_sync(FULL, e);
        if (!em) return;
        if (buffered + 32 > SEG_CUT_BUF) flush();
        if (e) {
            const uint32_t i = buffered + __popc(em & ((1u << lane) - 1u));
            s_beg[wib][i] = beg;
            s_len[wib][i] = (uint32_t)(end_idx - start);
            s_q[wib][i] = q;
            s_key[wib][i] = key;
        }
        buffered += __popc(em);
    };
    for (uint64_t base = c0; base < c1; base += 32) {
        const uint64_t g = base + lane;
        const bool valid = g < c1;
        uint32_t key = 0;
        uint64_t beg = 0;
        bool forced = false;
        if (valid) {
            while (p.kcum[qlane + 1] <= g) ++qlane;
            const uint64_t qk = g - p.kcum[qlane];
            beg = p.offsets[qlane] + qk;
            key = order_hash(canonical_from_window(base_window(p.packed, p.packed_bytes, beg + p.base_shift), p.k));
            forced = qk == 0 || g == c0 || g - last_kept >= SEG_MAX_LEN;  // (lengths fit 32 bits)
        }
        const uint32_t cm = __ballot_sync(FULL, valid && (forced || (key & cut_mask) == 0));
        const uint32_t fm = __ballot_sync(FULL, valid && forced);
        uint32_t kept = 0;
        for (uint32_t rem = cm; rem; rem &= rem - 1) {
            const int b = __ffs(rem) - 1;
            const uint64_t gi = base + (uint64_t)b;
            if (((fm >> b) & 1u) || gi - last_kept >= a.min_len) {
                kept |= 1u << b;
                last_kept = gi;
            }
        }
        if (!kept) continue;
        // a kept start closes the segment opened by the kept start below it
        // (or the open one carried in)
        const uint32_t below = kept & ((1u << lane) - 1u);
        const int src = below ? 31 - __clz(below) : 0;
        uint64_t ps = __shfl_sync(FULL, g, src), pb = __shfl_sync(FULL, beg, src);
        uint32_t pk = __shfl_sync(FULL, key, src), pq = __shfl_sync(FULL, (uint32_t)qlane, src);
        if (!below) {
            ps = o_start;
            pb = o_beg;
            pk = o_key;
            pq = o_q;
        }
        emit(((kept >> lane) & 1u) && ps != ~0ull, ps, pb, g, pk, pq);
        const int top = 31 - __clz(kept);
        o_start = __shfl_sync(FULL, g, top);
        o_beg = __shfl_sync(FULL, beg, top);
        o_key = __shfl_sync(FULL, key, top);
        o_q = __shfl_sync(FULL, (uint32_t)qlane, top);
    }
    emit(lane == 0 && o_start != ~0ull, o_start, o_beg, c1, o_key, o_q);
    if (buffered) flush();
}

// Bucket counts -> exclusive offsets, in place (one block).
constexpr int SEG_SCAN_THREADS = 1024;
__global__ void __launch_bounds__(SEG_SCAN_THREADS) k_seg_scan(uint32_t *bucket, uint32_t nb) {
    __shared__ uint32_t warp_tot[SEG_SCAN_THREADS / 32];
    const uint32_t per = (nb + SEG_SCAN_THREADS - 1) / SEG_SCAN_THREADS;
    const uint32_t b0 = threadIdx.x * per;
    uint32_t sum = 0;
    for (uint32_t i = 0; i < per; ++i)
        if (b0 + i < nb) sum += bucket[b0 + i];
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
        uint32_t x = warp_tot[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, off);
            if (lane >= off) x += y;
        }
        warp_tot[lane] = x;
    }
    __syncthreads();
    uint32_t run = (wid ? warp_tot[wid - 1] : 0) + incl - sum;
    for (uint32_t i = 0; i < per; ++i) {
        if (b0 + i < nb) {
            const uint32_t x = bucket[b0 + i];
            bucket[b0 + i] = run;
            run += x;
        }
    }
}

// Every recorded segment to a slot of its bucket (as the item range
// [first base, first base + k-mers + k - 1)); the slots past the segment
// count become empty ranges.
__global__ void __launch_bounds__(SEG_THREADS) k_seg_place(SegArgs a) {
    const unsigned long long emitted = *a.ctr;
    const uint64_t nseg = emitted < a.cap ? emitted : a.cap;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.cap;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (i < nseg) {
            const uint32_t slot = atomicAdd(a.bucket + (a.raw_key[i] >> a.bucket_shift), 1u);
            const uint64_t b = a.raw_begin[i];
            a.sbeg[slot] = b;
            a.send[slot] = b + a.raw_len[i] + a.p.k - 1;
            a.sq[slot] = a.raw_q[i];
        } else {
            a.sbeg[i] = 0;
            a.send[i] = 0;
            a.sq[i] = NONE;
        }
    }
}

// chunk_seg[j] = the ordered segment holding k-mer j * PSK.
__global__ void __launch_bounds__(SEG_THREADS) k_seg_chunks(SegArgs a) {
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.cap;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k0 = a.scum[s], k1 = a.scum[s + 1];
        for (uint64_t j = (k0 + SEG_PSK - 1) / SEG_PSK; j * SEG_PSK < k1; ++j)
            if (j < a.max_chunks) a.chunk_seg[j] = (uint32_t)s;
    }
}

// ANDs a lane's slice of a segment into its query's mask.
template <int SW>
__device__ __forceinline__ void seg_flush(const SegArgs &a, uint32_t seg, uint32_t word0, const Slice<SW> &v) {
    const uint32_t q = a.sq[seg];
    uint32_t *acc = a.p.acc;
    if constexpr (SW == 4) {
        unsigned long long *p = reinterpret_cast<unsigned long long *>(acc + (uint64_t)q * a.p.Gw + word0);
        const unsigned long long lo = ((unsigned long long)v.w[1] << 32) | v.w[0];
        const unsigned long long hi = ((unsigned long long)v.w[3] << 32) | v.w[2];
        if (lo != ~0ull) atomicAnd(p, lo);
        if (hi != ~0ull) atomicAnd(p + 1, hi);
    } else {
        flush_slice<SW>(acc, q, a.p.Gw, word0, v);
    }
}

// Probe pass.  LPG lanes per group (SW words each), NS = 32 / LPG lane groups
// per warp; a round covers RK consecutive k-mers of a lane group, HPL of them
// hashed by each of its lanes; the next round is hashed while the current
// round's RK * ETA gathers are in flight.
template <int SW, int LPG, int ETA>
__global__ void __launch_bounds__(SEG_THREADS) k_seg_probe(SegArgs a) {
    constexpr int NS = 32 / LPG;
    constexpr int RK = LPG >= 4 ? LPG : 4;
    constexpr int HPL = RK / LPG;
    static_assert(SEG_PSK % RK == 0, "a lane group's k-mers are whole rounds");
    const ProbeArgs &p = a.p;
    const int lane = threadIdx.x & 31;
    const int grp = lane / LPG, sub = lane % LPG;
    const uint32_t word0 = (uint32_t)sub * SW;
    const uint64_t T = a.scum[a.cap];
    const uint64_t IK = (uint64_t)NS * SEG_PSK;
    const uint64_t items = (T + IK - 1) / IK;
    unsigned long long *claim = a.ctr + 1;

    uint64_t item = 0;
    if (lane == 0) item = atomicAdd(claim, 1ull);
    item = __shfl_sync(FULL, item, 0);
    while (item < items) {
        uint64_t nxt = 0;
        if (lane == 0) nxt = atomicAdd(claim, 1ull);  // in flight during this item
        const uint64_t s0 = item * IK + (uint64_t)grp * SEG_PSK;
        const uint64_t s1 = s0 + SEG_PSK < T ? s0 + SEG_PSK : T;
        uint32_t lseg = s0 < T ? a.chunk_seg[s0 / SEG_PSK] : 0u;
        // hash the k-mers of the round starting at r: this lane's HPL of them
        uint32_t pos[HPL][ETA], sid[HPL];
        auto hash_round = [&](uint64_t r) {
#pragma unroll
            for (int h = 0; h < HPL; ++h) {
                const uint64_t idx = r + (uint64_t)(sub + h * LPG);
                uint64_t c = 0;
                sid[h] = NONE;
                if (idx < s1) {
                    while (a.scum[lseg + 1] <= idx) ++lseg;
                    const uint64_t start = a.sbeg[lseg] + p.base_shift + (idx - a.scum[lseg]);
                    c = canonical_from_window(base_window(p.packed, p.packed_bytes, start), p.k);
                    sid[h] = lseg;
                }
                const uint64_t km = mh_mix_key(c);
#pragma unroll
                for (int e = 0; e < ETA; ++e)
                    pos[h][e] = reduce_pos(mh_first_word(km, p.seed32 + (uint32_t)e), p.m, p.m_pow2);
            }
        };
        uint32_t cur = NONE;
        Slice<SW> run;
        slice_ones(run);
        // rounds are warp-uniform (the shuffles need every lane); k-mers past
        // a lane group's end are skipped inside
        hash_round(s0);
#pragma unroll 1
        for (int rr = 0; rr < SEG_PSK; rr += RK) {
            Slice<SW> v[RK][ETA];
            uint32_t ks[RK];
#pragma unroll
            for (int kk = 0; kk < RK; ++kk) {
                const int src = grp * LPG + kk % LPG;
                ks[kk] = __shfl_sync(FULL, sid[kk / LPG], src, 32);
#pragma unroll
                for (int e = 0; e < ETA; ++e) {
                    const uint32_t pe = __shfl_sync(FULL, pos[kk / LPG][e], src, 32);
                    if (ks[kk] != NONE) v[kk][e] = ld_slice<SW>(p.index + (uint64_t)pe * p.Gw + word0);
                    else slice_ones(v[kk][e]);
                }
            }
            if (rr + RK < SEG_PSK) hash_round(s0 + (uint64_t)(rr + RK));  // overlaps the gathers above
#pragma unroll
            for (int kk = 0; kk < RK; ++kk) {
                if (ks[kk] == NONE) continue;
                Slice<SW> x = v[kk][0];
#pragma unroll
                for (int e = 1; e < ETA; ++e) slice_and(x, v[kk][e]);
                if (ks[kk] != cur) {
                    if (cur != NONE) seg_flush<SW>(a, cur, word0, run);
                    cur = ks[kk];
                    run = x;
                } else {
                    slice_and(run, x);
                }
            }
        }
        if (cur != NONE) seg_flush<SW>(a, cur, word0, run);
        item = __shfl_sync(FULL, nxt, 0);
    }
}

template <int SW, int LPG, int ETA>
cudaError_t launch_seg_probe_t(const SegArgs &a, int sm_count, cudaStream_t s) {
    static int occ = [] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_seg_probe<SW, LPG, ETA>, SEG_THREADS, 0) !=
                cudaSuccess || n < 1)
            n = 1;
        return n;
    }();
    k_seg_probe<SW, LPG, ETA><<<occ * sm_count, SEG_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

template <int ETA>
cudaError_t launch_seg_probe_eta(const SegArgs &a, const Geometry &g, int sm_count, cudaStream_t s) {
    switch (g.Gw) {
        case 1: return launch_seg_probe_t<1, 1, ETA>(a, sm_count, s);
        case 2: return launch_seg_probe_t<2, 1, ETA>(a, sm_count, s);
        case 4: return launch_seg_probe_t<4, 1, ETA>(a, sm_count, s);
        case 8: return launch_seg_probe_t<4, 2, ETA>(a, sm_count, s);
        default: return launch_seg_probe_t<4, 4, ETA>(a, sm_count, s);
    }
}

}  // namespace

bool segments_supported(const Geometry &g) {
    return (g.Gw == 1 || g.Gw == 2 || g.Gw == 4 || g.Gw == 8 || g.Gw == 16) && g.eta >= 1 && g.eta <= 4;
}

uint32_t seg_cut_grid(int sm_count) {
    static int occ = [] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_seg_cut, SEG_THREADS, 0) != cudaSuccess || n < 1)
            n = 1;
        return n;
    }();
    return (uint32_t)(occ * sm_count);
}

uint64_t seg_capacity(uint64_t max_kmers, uint64_t n, uint32_t min_len, uint32_t cut_grid) {
    // starts that are not forced are min_len apart; forced ones are query
    // starts, warp-range starts, and at most one step's 32 k-mers per
    // SEG_MAX_LEN k-mers without a start
    const uint64_t ml = min_len ? min_len : 1;
    return (max_kmers + ml - 1) / ml + n + (uint64_t)cut_grid * (SEG_THREADS / 32) +
           32 * (max_kmers / SEG_MAX_LEN) + 1;
}

uint64_t seg_max_chunks(uint64_t max_kmers) { return (max_kmers + SEG_PSK - 1) / SEG_PSK + 1; }

int seg_launches_before_prefix() { return 3; }
int seg_launches_after_prefix() { return 2; }

cudaError_t launch_seg_order(const SegArgs &a, uint32_t cut_grid, int sm_count, cudaStream_t s) {
    if (a.cut_bits > 16 || a.nbuckets == 0 || a.nbuckets > (1u << 20) || a.cap == 0 || a.cap > 0xffffffffull)
        return cudaErrorInvalidValue;
    k_seg_cut<<<cut_grid, SEG_THREADS, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_seg_scan<<<1, SEG_SCAN_THREADS, 0, s>>>(a.bucket, a.nbuckets);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_seg_place<<<4 * sm_count, SEG_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_seg_probe(const SegArgs &a, const Geometry &g, int sm_count, cudaStream_t s) {
    if (!segments_supported(g)) return cudaErrorInvalidValue;
    k_seg_chunks<<<4 * sm_count, SEG_THREADS, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (g.eta) {
        case 1: return launch_seg_probe_eta<1>(a, g, sm_count, s);
        case 2: return launch_seg_probe_eta<2>(a, g, sm_count, s);
        case 3: return launch_seg_probe_eta<3>(a, g, sm_count, s);
        default: return launch_seg_probe_eta<4>(a, g, sm_count, s);
    }
}

}  // namespace rgpu

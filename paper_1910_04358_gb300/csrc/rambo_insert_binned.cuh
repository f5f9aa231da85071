// rambo_insert_binned.cuh -- region-binned index construction (Algorithm 1's
// bit setting in two passes whose atomics land in L2).
#pragma once

#include "rambo_internal.cuh"

namespace rgpu {

// Index regions the records are binned by: at most IB_MAX_BINS of them, each
// 2^rshift position groups (about bin_region_kib of index bytes, a region
// that stays in L2 while its records are applied).
constexpr uint32_t IB_MAX_BINS = 1024;

// Chunks one insert call may take (record buffer / eta k-mers each); a
// batch needing more is inserted directly.
constexpr uint64_t IB_MAX_CHUNKS = 65536;

// A record is (position << IB_DOC_BITS) | document: positions below 2^40,
// documents below 2^24.
constexpr uint32_t IB_DOC_BITS = 24;

struct BinnedInsert {
    unsigned long long *buf;  // nbins x cap records
    uint32_t *count;          // IB_MAX_BINS record counts, then the apply pass's unit counter
    uint64_t cap;             // records per bin
    uint32_t nbins;
    uint32_t rshift;          // position >> rshift = bin
};

// Region shift for groups of `group_bytes` and regions of about
// `region_bytes`, and the bin count for m positions; 0 bins when the binned
// construction does not apply (too many regions, or positions or documents
// beyond the record encoding).
uint32_t binned_insert_bins(uint64_t m, uint32_t group_bytes, uint32_t K, uint64_t region_bytes,
                            uint32_t *rshift);

// One chunk [f0, f1) of the batch's flat k-mer index (clamped to the batch's
// k-mer count on the device): a scatter pass appends every probe's record to
// the bin of its region (records past a bin's capacity set their bits on the
// spot), then an apply pass walks the bins in region order and sets the
// bits.  b.count must be zero on entry (the caller clears it per chunk).
// Two kernel launches on `s`.
cudaError_t launch_insert_binned(const InsertArgs &a, const BinnedInsert &b, uint64_t f0, uint64_t f1,
                                 int sm_count, cudaStream_t s);

}  // namespace rgpu

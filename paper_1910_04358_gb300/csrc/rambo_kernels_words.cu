// rambo_kernels_words.cu -- documents of words (Section 5.4 "Document
// indexing": every document is a set of word unigrams).
//
// A term is an arbitrary byte string; probe j of a term is the first output
// word of MurmurHash3_x64_128(term bytes, seed + j) reduced mod m, so the same
// index layout, partition and expansion serve word documents.  Batches are
// CSR twice over: term t is bytes [term_offs[t], term_offs[t+1]) and item i
// (a document to insert or a query) is terms [item_terms[i], item_terms[i+1]).
#include "rambo_query_common.cuh"

namespace rgpu {
namespace {

// MurmurHash3_x64_128 of a byte string, first output word (the general
// form: 16-byte blocks, then the 0..15-byte tail, then the finalisation).
__device__ uint64_t mh_bytes_first_word(const uint8_t *p, uint64_t len, uint32_t seed) {
    const uint64_t c1 = 0x87c37b91114253d5ULL, c2 = 0x4cf5ad432745937fULL;
    uint64_t h1 = seed, h2 = seed;
    const uint64_t nblocks = len / 16;
    auto le = [&](const uint8_t *q, int n) {
        uint64_t v = 0;
        for (int i = n - 1; i >= 0; --i) v = (v << 8) | q[i];
        return v;
    };
    for (uint64_t b = 0; b < nblocks; ++b) {
        uint64_t k1 = le(p + 16 * b, 8), k2 = le(p + 16 * b + 8, 8);
        k1 *= c1; k1 = rotl64(k1, 31); k1 *= c2; h1 ^= k1;
        h1 = rotl64(h1, 27); h1 += h2; h1 = h1 * 5 + 0x52dce729;
        k2 *= c2; k2 = rotl64(k2, 33); k2 *= c1; h2 ^= k2;
        h2 = rotl64(h2, 31); h2 += h1; h2 = h2 * 5 + 0x38495ab5;
    }
    const uint8_t *tail = p + 16 * nblocks;
    const int rem = (int)(len & 15);
    if (rem > 8) {
        uint64_t k2 = le(tail + 8, rem - 8);
        k2 *= c2; k2 = rotl64(k2, 33); k2 *= c1; h2 ^= k2;
    }
    if (rem > 0) {
        uint64_t k1 = le(tail, rem > 8 ? 8 : rem);
        k1 *= c1; k1 = rotl64(k1, 31); k1 *= c2; h1 ^= k1;
    }
    h1 ^= len; h2 ^= len;
    h1 += h2; h2 += h1;
    h1 = fmix64(h1); h2 = fmix64(h2);
    return h1 + h2;
}

// Item of flattened term t: largest i with item_terms[i] <= t.
__device__ __forceinline__ uint64_t item_of(const uint64_t *item_terms, uint64_t n, uint64_t t) {
    uint64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (item_terms[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool term_bytes(const WordArgs &a, uint64_t t, const uint8_t **p,
                                           uint64_t *len) {
    const uint64_t b0 = a.term_offs[t], b1 = a.term_offs[t + 1];
    if (b1 < b0 || b1 > a.bytes_len) {
        atomicOr(a.err, ERR_OFFSETS);
        return false;
    }
    *p = a.bytes + b0;
    *len = b1 - b0;
    return true;
}

// Algorithm 1 for word documents: one thread per (document, term).
__global__ void k_insert_words(WordArgs a) {
    const uint64_t t0 = a.item_terms[0], t1 = a.item_terms[a.n];
    for (uint64_t t = t0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < t1;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = item_of(a.item_terms, a.n, t);
        const uint32_t d = a.doc_ids[i];
        if (d >= a.K) continue;  // latched by the registration kernel
        const uint8_t *w;
        uint64_t len;
        if (!term_bytes(a, t, &w, &len)) continue;
        for (uint32_t j = 0; j < a.eta; ++j) {
            const uint64_t h = mh_bytes_first_word(w, len, a.seed32 + j);
            const uint64_t p = a.m_pow2 ? (h & (a.m - 1)) : (h % a.m);
            for (uint32_t r = 0; r < a.R; ++r) {
                const uint32_t bb = r * a.B + a.phi[(uint64_t)d * a.R + r];
                atomicOr(a.index + p * a.Gw + (bb >> 5), 1u << (bb & 31));
            }
        }
    }
}

// Probe of word queries: one thread per (query, term); the AND of the eta
// groups of the term is folded into the query's bucket mask with atomicAnd
// (all-ones words skipped).
__global__ void k_probe_words(WordArgs a) {
    const uint64_t t0 = a.item_terms[0], t1 = a.item_terms[a.n];
    for (uint64_t t = t0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < t1;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q = item_of(a.item_terms, a.n, t);
        const uint8_t *w;
        uint64_t len;
        if (!term_bytes(a, t, &w, &len)) continue;
        uint32_t pos[64];
        for (uint32_t j = 0; j < a.eta; ++j) {
            const uint64_t h = mh_bytes_first_word(w, len, a.seed32 + j);
            pos[j] = (uint32_t)(a.m_pow2 ? (h & (a.m - 1)) : (h % a.m));
        }
        uint32_t *acc = a.acc + q * a.Gw;
        for (uint32_t word = 0; word < a.Gw; ++word) {
            uint32_t v = FULL;
            for (uint32_t j = 0; j < a.eta && v; ++j) v &= __ldg(a.index_ro + (uint64_t)pos[j] * a.Gw + word);
            if (v != FULL) atomicAnd(acc + word, v);
        }
    }
}

}  // namespace

cudaError_t launch_insert_words(const WordArgs &a, int sm_count, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_insert_words<<<sm_count * 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_probe_words(const WordArgs &a, int sm_count, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_probe_words<<<sm_count * 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace rgpu

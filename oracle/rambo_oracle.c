/*
 * rambo_oracle.c -- plain, slow, single-threaded CPU RAMBO used as TEST
 * INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the product path (the CUDA
 * library) never does, and the two share no code.
 *
 * What it computes (Gupta et al., "Fast Processing and Querying of 170TB of
 * Genomics Data via a Repeated And Merged BloOm Filter (RAMBO)", SIGMOD'21):
 *
 *   - A Bloom filter ("BFU") is an array of m bits; a term x is inserted by
 *     setting the bits h_1(x)..h_eta(x) and is a member iff all eta bits are
 *     set (Section 2.1).
 *   - RAMBO is an R x B table of BFUs.  In repetition r the documents are
 *     partitioned into B buckets by a partition hash phi_r applied to the
 *     document identity (Section 3, Section 3.2).  Inserting document S_i adds
 *     every term of S_i to the BFU of bucket phi_r(i) in every repetition r
 *     (Algorithm 1).
 *   - A query q with term set Q = Terms(q): in each repetition r the union G_r
 *     of the document sets of all BFUs that contain every term of Q, then the
 *     intersection of G_1..G_R (Algorithm 2, Section 3.3, Section 3.3.1).
 *   - Terms of a sequence are its length-k windows (k = 31 in the paper),
 *     2-bit encoded into a 64-bit integer (Section 3.3.1, Section 5.1).
 *
 * Readings taken where the paper is silent (each one is also listed in the
 * design notes of the repository):
 *   - Algorithm 1 prints phi applied to the term; Section 3.2 applies phi to
 *     the document.  The document reading is used: bucket = phi_r(doc id).
 *   - Repetitions are numbered r = 0..R-1.
 *   - Hash family: MurmurHash3_x64_128 (Appleby's public algorithm, written
 *     here from its published description).  Keys are 8-byte little-endian
 *     integers.  Probe j of a term uses seed (uint32)(seed + j) and takes the
 *     first 64-bit output word modulo m; document d goes to bucket
 *     first-word(MurmurHash3(d, seed (uint32)(seed + 1000 + r))) modulo B.
 *     The same probe positions serve every BFU (Section 5.3 requires all
 *     machines to share h).
 *   - Bases are coded A=0, C=1, G=2, T=3; the complement of b is 3-b; the
 *     first base of a window is the most significant digit; a term is the
 *     canonical k-mer min(forward code, reverse-complement code).
 *   - Packed input: base t of a buffer sits in byte t>>2 at bits
 *     2*(t&3)..2*(t&3)+1 (least significant pair first).
 *   - A query with no term (length < k) satisfies "for all x in Q" vacuously,
 *     so every inserted document is returned.
 *   - DocIDs(M[b,r]) holds only documents that were inserted.
 *
 * Everything here is deliberately unoptimised: each BFU is its own m-bit
 * array, terms are built base by base from the decoded sequence, the reverse
 * complement is built by reversing and complementing the bases, and the query
 * walks Algorithm 2's loops over r and b literally.
 *
 * "Restricted" mode keeps, for every BFU, only the bits at a caller-given
 * sorted list of positions.  It computes exactly the same answers for
 * queries whose probe positions all lie in that list, and lets the tests
 * check sampled queries on indices too large to hold as R*B full filters.
 *
 * Multi-threading is only a way to spend host cores on independent work:
 * insert_batch splits documents over threads that OR bits into the shared
 * filters (OR is order-independent), and query_seqs splits queries.  The
 * answers do not depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------ */
/* Error codes (the oracle's own; unrelated to the CUDA library's).    */
#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ERANGE (-4)
#define ORC_EUNTRACKED (-7)

/* ------------------------------------------------------------------ */
/* MurmurHash3_x64_128, general byte-string form.                       */

static uint64_t orc_rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

static uint64_t orc_fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

/* Little-endian read of n (<= 8) bytes. */
static uint64_t orc_load_le(const uint8_t *p, int n) {
    uint64_t v = 0;
    for (int i = n - 1; i >= 0; --i) v = (v << 8) | p[i];
    return v;
}

void orc_mmh3_x64_128(const void *key, uint64_t len, uint32_t seed, uint64_t out[2]) {
    const uint8_t *data = (const uint8_t *)key;
    const uint64_t c1 = 0x87c37b91114253d5ULL;
    const uint64_t c2 = 0x4cf5ad432745937fULL;
    uint64_t h1 = seed, h2 = seed;
    uint64_t nblocks = len / 16;
    for (uint64_t i = 0; i < nblocks; ++i) {
        uint64_t k1 = orc_load_le(data + 16 * i, 8);
        uint64_t k2 = orc_load_le(data + 16 * i + 8, 8);
        k1 *= c1; k1 = orc_rotl64(k1, 31); k1 *= c2; h1 ^= k1;
        h1 = orc_rotl64(h1, 27); h1 += h2; h1 = h1 * 5 + 0x52dce729;
        k2 *= c2; k2 = orc_rotl64(k2, 33); k2 *= c1; h2 ^= k2;
        h2 = orc_rotl64(h2, 31); h2 += h1; h2 = h2 * 5 + 0x38495ab5;
    }
    const uint8_t *tail = data + 16 * nblocks;
    int rem = (int)(len & 15);
    if (rem > 8) {
        uint64_t k2 = orc_load_le(tail + 8, rem - 8);
        k2 *= c2; k2 = orc_rotl64(k2, 33); k2 *= c1; h2 ^= k2;
    }
    if (rem > 0) {
        uint64_t k1 = orc_load_le(tail, rem > 8 ? 8 : rem);
        k1 *= c1; k1 = orc_rotl64(k1, 31); k1 *= c2; h1 ^= k1;
    }
    h1 ^= len; h2 ^= len;
    h1 += h2; h2 += h1;
    h1 = orc_fmix64(h1); h2 = orc_fmix64(h2);
    h1 += h2; h2 += h1;
    out[0] = h1;
    out[1] = h2;
}

/* First output word of MurmurHash3_x64_128 over an integer as 8 LE bytes. */
static uint64_t orc_hash_u64(uint64_t v, uint32_t seed) {
    uint8_t b[8];
    for (int i = 0; i < 8; ++i) b[i] = (uint8_t)(v >> (8 * i));
    uint64_t o[2];
    orc_mmh3_x64_128(b, 8, seed, o);
    return o[0];
}

/* ------------------------------------------------------------------ */
/* Sequences and terms.                                                 */

/* Base t of a packed buffer (2 bits per base, least significant first). */
static int orc_base_at(const uint8_t *packed, uint64_t t) {
    return (packed[t >> 2] >> (2 * (t & 3))) & 3;
}

void orc_unpack(const uint8_t *packed, uint64_t begin, uint64_t n, uint8_t *bases) {
    for (uint64_t i = 0; i < n; ++i) bases[i] = (uint8_t)orc_base_at(packed, begin + i);
}

/* Forward code of the window bases[0..k-1]: first base most significant. */
static uint64_t orc_forward_code(const uint8_t *bases, uint32_t k) {
    uint64_t f = 0;
    for (uint32_t i = 0; i < k; ++i) f = f * 4 + bases[i];
    return f;
}

/* Reverse complement, built the way it is defined: reverse the window, then
 * complement every base, then read it off like a forward window. */
static uint64_t orc_revcomp_code(const uint8_t *bases, uint32_t k) {
    uint8_t rc[64];
    for (uint32_t i = 0; i < k; ++i) rc[i] = (uint8_t)(3 - bases[k - 1 - i]);
    return orc_forward_code(rc, k);
}

static uint64_t orc_canonical_of_window(const uint8_t *bases, uint32_t k) {
    uint64_t f = orc_forward_code(bases, k);
    uint64_t r = orc_revcomp_code(bases, k);
    return f < r ? f : r;
}

/* Exported helpers for the pins. */
uint64_t orc_kmer_forward(const uint8_t *packed, uint64_t begin, uint32_t k) {
    uint8_t b[64];
    orc_unpack(packed, begin, k, b);
    return orc_forward_code(b, k);
}
uint64_t orc_kmer_canonical(const uint8_t *packed, uint64_t begin, uint32_t k) {
    uint8_t b[64];
    orc_unpack(packed, begin, k, b);
    return orc_canonical_of_window(b, k);
}
/* Canonical form of a k-mer given by its forward code. */
uint64_t orc_canonical_of_code(uint64_t fwd, uint32_t k) {
    uint8_t b[64];
    for (uint32_t i = 0; i < k; ++i) b[k - 1 - i] = (uint8_t)((fwd >> (2 * i)) & 3);
    return orc_canonical_of_window(b, k);
}

/* ------------------------------------------------------------------ */
/* The RAMBO table.                                                     */

typedef struct {
    uint32_t K, B, R, eta, k;
    uint64_t m, seed;
    /* R*B Bloom filters, filter (r,b) at index r*B+b, each nbits bits. */
    uint64_t **filter;
    uint64_t nbits;
    /* Restricted mode: sorted distinct tracked positions (NULL = full),
     * plus an m-bit membership bitmap of them. */
    uint64_t *tracked;
    uint64_t n_tracked;
    uint64_t *tracked_bits;
    /* DocIDs(M[b,r]) as growable lists; bucket[d*R + r] = phi_r(d). */
    uint32_t **docs;
    uint32_t *ndocs, *capdocs;
    uint32_t *bucket;
    uint8_t *inserted;
} orc_rambo;

uint32_t orc_partition(const orc_rambo *o, uint32_t d, uint32_t r) {
    return (uint32_t)(orc_hash_u64((uint64_t)d, (uint32_t)(o->seed + 1000 + r)) % o->B);
}

uint64_t orc_probe_position(const orc_rambo *o, uint64_t term, uint32_t j) {
    return orc_hash_u64(term, (uint32_t)(o->seed + j)) % o->m;
}

/* Position -> bit index inside a filter; -1 when restricted and untracked. */
static int64_t orc_slot(const orc_rambo *o, uint64_t pos) {
    if (!o->tracked) return (int64_t)pos;
    if (!((o->tracked_bits[pos >> 6] >> (pos & 63)) & 1)) return -1;
    uint64_t lo = 0, hi = o->n_tracked;
    while (lo < hi) {
        uint64_t mid = (lo + hi) / 2;
        if (o->tracked[mid] < pos) lo = mid + 1; else hi = mid;
    }
    if (lo < o->n_tracked && o->tracked[lo] == pos) return (int64_t)lo;
    return -1;
}

void orc_destroy(orc_rambo *o) {
    if (!o) return;
    if (o->filter)
        for (uint64_t i = 0; i < (uint64_t)o->R * o->B; ++i) free(o->filter[i]);
    if (o->docs)
        for (uint64_t i = 0; i < (uint64_t)o->R * o->B; ++i) free(o->docs[i]);
    free(o->filter); free(o->docs); free(o->ndocs); free(o->capdocs);
    free(o->bucket); free(o->inserted); free(o->tracked); free(o->tracked_bits);
    free(o);
}

static orc_rambo *orc_create_impl(uint32_t K, uint32_t B, uint32_t R, uint64_t m, uint32_t eta,
                                  uint32_t k, uint64_t seed, const uint64_t *tracked,
                                  uint64_t n_tracked) {
    if (K == 0 || B == 0 || R == 0 || m == 0 || eta == 0 || eta > 64 || k == 0 || k > 32)
        return NULL;
    orc_rambo *o = (orc_rambo *)calloc(1, sizeof(orc_rambo));
    if (!o) return NULL;
    o->K = K; o->B = B; o->R = R; o->m = m; o->eta = eta; o->k = k; o->seed = seed;
    if (tracked) {
        o->tracked = (uint64_t *)malloc(sizeof(uint64_t) * (n_tracked ? n_tracked : 1));
        if (!o->tracked) { orc_destroy(o); return NULL; }
        memcpy(o->tracked, tracked, sizeof(uint64_t) * n_tracked);
        o->n_tracked = n_tracked;
        for (uint64_t i = 1; i < n_tracked; ++i)
            if (tracked[i] <= tracked[i - 1]) { orc_destroy(o); return NULL; }
        if (n_tracked && tracked[n_tracked - 1] >= m) { orc_destroy(o); return NULL; }
        o->tracked_bits = (uint64_t *)calloc((m + 63) / 64, sizeof(uint64_t));
        if (!o->tracked_bits) { orc_destroy(o); return NULL; }
        for (uint64_t i = 0; i < n_tracked; ++i)
            o->tracked_bits[tracked[i] >> 6] |= (uint64_t)1 << (tracked[i] & 63);
        o->nbits = n_tracked;
    } else {
        o->nbits = m;
    }
    uint64_t nf = (uint64_t)R * B;
    uint64_t words = (o->nbits + 63) / 64;
    o->filter = (uint64_t **)calloc(nf, sizeof(uint64_t *));
    o->docs = (uint32_t **)calloc(nf, sizeof(uint32_t *));
    o->ndocs = (uint32_t *)calloc(nf, sizeof(uint32_t));
    o->capdocs = (uint32_t *)calloc(nf, sizeof(uint32_t));
    o->bucket = (uint32_t *)malloc(sizeof(uint32_t) * (uint64_t)K * R);
    o->inserted = (uint8_t *)calloc(K, 1);
    if (!o->filter || !o->docs || !o->ndocs || !o->capdocs || !o->bucket || !o->inserted) {
        orc_destroy(o);
        return NULL;
    }
    for (uint64_t i = 0; i < nf; ++i) {
        o->filter[i] = (uint64_t *)calloc(words ? words : 1, sizeof(uint64_t));
        if (!o->filter[i]) { orc_destroy(o); return NULL; }
    }
    for (uint32_t d = 0; d < K; ++d)
        for (uint32_t r = 0; r < R; ++r) o->bucket[(uint64_t)d * R + r] = orc_partition(o, d, r);
    return o;
}

orc_rambo *orc_create(uint32_t K, uint32_t B, uint32_t R, uint64_t m, uint32_t eta, uint32_t k,
                      uint64_t seed) {
    return orc_create_impl(K, B, R, m, eta, k, seed, NULL, 0);
}

orc_rambo *orc_create_restricted(uint32_t K, uint32_t B, uint32_t R, uint64_t m, uint32_t eta,
                                 uint32_t k, uint64_t seed, const uint64_t *tracked,
                                 uint64_t n_tracked) {
    return orc_create_impl(K, B, R, m, eta, k, seed, tracked, n_tracked);
}

uint64_t orc_num_filters_bits(const orc_rambo *o) { return o->nbits; }

/* Adds d to DocIDs(M[phi_r(d), r]) for every r, once (set semantics). */
static int orc_register_doc(orc_rambo *o, uint32_t d) {
    if (o->inserted[d]) return ORC_OK;
    for (uint32_t r = 0; r < o->R; ++r) {
        uint64_t f = (uint64_t)r * o->B + o->bucket[(uint64_t)d * o->R + r];
        if (o->ndocs[f] == o->capdocs[f]) {
            uint32_t cap = o->capdocs[f] ? 2 * o->capdocs[f] : 4;
            uint32_t *p = (uint32_t *)realloc(o->docs[f], sizeof(uint32_t) * cap);
            if (!p) return ORC_ENOMEM;
            o->docs[f] = p;
            o->capdocs[f] = cap;
        }
        o->docs[f][o->ndocs[f]++] = d;
    }
    o->inserted[d] = 1;
    return ORC_OK;
}

static void orc_set_bit(uint64_t *bits, uint64_t i, int atomic) {
    uint64_t w = (uint64_t)1 << (i & 63);
    if (atomic) __atomic_fetch_or(&bits[i >> 6], w, __ATOMIC_RELAXED);
    else bits[i >> 6] |= w;
}

static int orc_get_bit(const uint64_t *bits, uint64_t i) {
    return (int)((bits[i >> 6] >> (i & 63)) & 1);
}

/* Algorithm 1 for one document: every term x of the document goes into
 * BFU (phi_r(d), r) for every r; Insert(x) sets bits h_1(x)..h_eta(x).
 * Untracked positions (restricted mode) are skipped. */
static void orc_insert_terms(orc_rambo *o, uint32_t d, const uint8_t *packed, uint64_t begin,
                             uint64_t n_bases, int atomic) {
    if (n_bases < o->k) return;
    uint8_t *bases = (uint8_t *)malloc(n_bases);
    if (!bases) return;
    orc_unpack(packed, begin, n_bases, bases);
    int64_t slot[64];
    for (uint64_t s = 0; s + o->k <= n_bases; ++s) {
        uint64_t x = orc_canonical_of_window(bases + s, o->k);
        /* Insert(x): the eta bit positions h_1(x)..h_eta(x) of a BFU */
        for (uint32_t j = 0; j < o->eta; ++j) slot[j] = orc_slot(o, orc_probe_position(o, x, j));
        /* ... set in BFU (phi_r(d), r) of every repetition r */
        for (uint32_t r = 0; r < o->R; ++r) {
            uint64_t f = (uint64_t)r * o->B + o->bucket[(uint64_t)d * o->R + r];
            for (uint32_t j = 0; j < o->eta; ++j)
                if (slot[j] >= 0) orc_set_bit(o->filter[f], (uint64_t)slot[j], atomic);
        }
    }
    free(bases);
}

int orc_insert(orc_rambo *o, uint32_t d, const uint8_t *packed, uint64_t begin, uint64_t n_bases) {
    if (d >= o->K) return ORC_ERANGE;
    int rc = orc_register_doc(o, d);
    if (rc) return rc;
    orc_insert_terms(o, d, packed, begin, n_bases, 0);
    return ORC_OK;
}

typedef struct {
    orc_rambo *o;
    uint32_t n, t, T;
    const uint32_t *ids;
    const uint8_t *packed;
    const uint64_t *offs;
} orc_ins_job;

static void *orc_insert_worker(void *arg) {
    orc_ins_job *j = (orc_ins_job *)arg;
    for (uint32_t i = j->t; i < j->n; i += j->T)
        orc_insert_terms(j->o, j->ids[i], j->packed, j->offs[i], j->offs[i + 1] - j->offs[i], 1);
    return NULL;
}

int orc_insert_batch(orc_rambo *o, uint32_t n, const uint32_t *ids, const uint8_t *packed,
                     const uint64_t *offs, uint32_t n_threads) {
    for (uint32_t i = 0; i < n; ++i) {
        if (ids[i] >= o->K) return ORC_ERANGE;
        if (offs[i + 1] < offs[i]) return ORC_EINVAL;
    }
    for (uint32_t i = 0; i < n; ++i) {
        int rc = orc_register_doc(o, ids[i]);
        if (rc) return rc;
    }
    if (n_threads <= 1) {
        for (uint32_t i = 0; i < n; ++i)
            orc_insert_terms(o, ids[i], packed, offs[i], offs[i + 1] - offs[i], 0);
        return ORC_OK;
    }
    pthread_t th[256];
    orc_ins_job jobs[256];
    if (n_threads > 256) n_threads = 256;
    for (uint32_t t = 0; t < n_threads; ++t) {
        jobs[t] = (orc_ins_job){o, n, t, n_threads, ids, packed, offs};
        pthread_create(&th[t], NULL, orc_insert_worker, &jobs[t]);
    }
    for (uint32_t t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    return ORC_OK;
}

/* Algorithm 2 given the eta probe slots of every term of Q (pos[i*eta + j]).
 * Writes the K-bit answer as ceil(K/32) uint32 words: document d is word
 * d>>5, bit d&31. */
static int orc_query_slots(const orc_rambo *o, const uint64_t *pos, uint64_t nq, uint32_t *out) {
    uint32_t W = (o->K + 31) / 32;
    uint8_t *G = (uint8_t *)calloc(o->K, 1);   /* G_r for the current r */
    uint8_t *A = (uint8_t *)malloc(o->K);      /* running intersection  */
    if (!G || !A) { free(G); free(A); return ORC_ENOMEM; }
    memset(A, 1, o->K);
    for (uint32_t r = 0; r < o->R; ++r) {
        memset(G, 0, o->K);
        for (uint32_t b = 0; b < o->B; ++b) {
            uint64_t f = (uint64_t)r * o->B + b;
            /* Q in BFU(M[b,r]) iff every term passes; the first miss decides */
            int pass = 1;
            for (uint64_t i = 0; i < nq && pass; ++i)
                for (uint32_t j = 0; j < o->eta && pass; ++j)
                    if (!orc_get_bit(o->filter[f], pos[i * o->eta + j])) pass = 0;
            if (pass)
                for (uint32_t t = 0; t < o->ndocs[f]; ++t) G[o->docs[f][t]] = 1;
        }
        for (uint32_t d = 0; d < o->K; ++d) A[d] = (uint8_t)(A[d] & G[d]);
    }
    memset(out, 0, sizeof(uint32_t) * W);
    for (uint32_t d = 0; d < o->K; ++d)
        if (A[d]) out[d >> 5] |= (uint32_t)1 << (d & 31);
    free(G); free(A);
    return ORC_OK;
}

/* Algorithm 2 for a term set Q given as canonical k-mer codes. */
static int orc_query_terms(const orc_rambo *o, const uint64_t *Q, uint64_t nq, uint32_t *out) {
    uint64_t *pos = (uint64_t *)malloc(sizeof(uint64_t) * (nq ? nq : 1) * o->eta);
    if (!pos) return ORC_ENOMEM;
    int rc = ORC_OK;
    /* the eta probe positions of every term, one slot per (term, j) */
    for (uint64_t i = 0; i < nq; ++i)
        for (uint32_t j = 0; j < o->eta; ++j) {
            int64_t s = orc_slot(o, orc_probe_position(o, Q[i], j));
            if (s < 0) rc = ORC_EUNTRACKED;
            pos[i * o->eta + j] = (uint64_t)s;
        }
    if (!rc) rc = orc_query_slots(o, pos, nq, out);
    free(pos);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Documents of words (Section 5.4: each document is a set of word       */
/* unigrams).  A term is an arbitrary byte string; probe j of a term is   */
/* the first word of MurmurHash3_x64_128(term bytes, seed + j) mod m.     */

uint64_t orc_word_position(const orc_rambo *o, const uint8_t *bytes, uint64_t len, uint32_t j) {
    uint64_t h[2];
    orc_mmh3_x64_128(bytes, len, (uint32_t)(o->seed + j), h);
    return h[0] % o->m;
}

/* Algorithm 1 for document d given as n_terms byte strings: term t is bytes
 * [term_offs[t], term_offs[t+1]). */
int orc_insert_words(orc_rambo *o, uint32_t d, const uint8_t *bytes, const uint64_t *term_offs,
                     uint64_t n_terms) {
    if (d >= o->K) return ORC_ERANGE;
    int rc = orc_register_doc(o, d);
    if (rc) return rc;
    for (uint64_t t = 0; t < n_terms; ++t) {
        const uint8_t *w = bytes + term_offs[t];
        const uint64_t len = term_offs[t + 1] - term_offs[t];
        for (uint32_t r = 0; r < o->R; ++r) {
            uint64_t f = (uint64_t)r * o->B + o->bucket[(uint64_t)d * o->R + r];
            for (uint32_t j = 0; j < o->eta; ++j) {
                int64_t slot = orc_slot(o, orc_word_position(o, w, len, j));
                if (slot >= 0) orc_set_bit(o->filter[f], (uint64_t)slot, 0);
            }
        }
    }
    return ORC_OK;
}

/* Algorithm 2 for a query given as a set of words (every word must pass). */
int orc_query_words(const orc_rambo *o, const uint8_t *bytes, const uint64_t *term_offs,
                    uint64_t n_terms, uint32_t *out) {
    uint64_t *pos = (uint64_t *)malloc(sizeof(uint64_t) * (n_terms ? n_terms : 1) * o->eta);
    if (!pos) return ORC_ENOMEM;
    int rc = ORC_OK;
    for (uint64_t t = 0; t < n_terms; ++t)
        for (uint32_t j = 0; j < o->eta; ++j) {
            int64_t s = orc_slot(o, orc_word_position(o, bytes + term_offs[t],
                                                      term_offs[t + 1] - term_offs[t], j));
            if (s < 0) rc = ORC_EUNTRACKED;
            pos[t * o->eta + j] = (uint64_t)s;
        }
    if (!rc) rc = orc_query_slots(o, pos, n_terms, out);
    free(pos);
    return rc;
}

/* Terms(q) for the sequence of n_bases bases starting at base `begin`. */
int orc_query_seq(const orc_rambo *o, const uint8_t *packed, uint64_t begin, uint64_t n_bases,
                  uint32_t *out) {
    uint64_t nq = n_bases >= o->k ? n_bases - o->k + 1 : 0;
    uint8_t *bases = (uint8_t *)malloc(n_bases ? n_bases : 1);
    uint64_t *Q = (uint64_t *)malloc(sizeof(uint64_t) * (nq ? nq : 1));
    if (!bases || !Q) { free(bases); free(Q); return ORC_ENOMEM; }
    orc_unpack(packed, begin, n_bases, bases);
    for (uint64_t s = 0; s < nq; ++s) Q[s] = orc_canonical_of_window(bases + s, o->k);
    int rc = orc_query_terms(o, Q, nq, out);
    free(bases); free(Q);
    return rc;
}

/* A single k-mer given by its forward code (bits at or above 2k must be 0). */
int orc_query_kmer(const orc_rambo *o, uint64_t fwd, uint32_t *out) {
    if (o->k < 32 && (fwd >> (2 * o->k)) != 0) return ORC_EINVAL;
    uint64_t x = orc_canonical_of_code(fwd, o->k);
    return orc_query_terms(o, &x, 1, out);
}

typedef struct {
    const orc_rambo *o;
    uint64_t n, t, T;
    const uint8_t *packed;
    const uint64_t *offs;
    const uint64_t *kmers;
    uint32_t *out;
    int rc;
} orc_q_job;

static void *orc_query_worker(void *arg) {
    orc_q_job *j = (orc_q_job *)arg;
    uint32_t W = (j->o->K + 31) / 32;
    for (uint64_t i = j->t; i < j->n; i += j->T) {
        int rc = j->kmers
                     ? orc_query_kmer(j->o, j->kmers[i], j->out + i * W)
                     : orc_query_seq(j->o, j->packed, j->offs[i], j->offs[i + 1] - j->offs[i],
                                     j->out + i * W);
        if (rc) j->rc = rc;
    }
    return NULL;
}

static int orc_query_many(const orc_rambo *o, uint64_t n, const uint8_t *packed,
                          const uint64_t *offs, const uint64_t *kmers, uint32_t *out,
                          uint32_t n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    orc_q_job jobs[256];
    for (uint32_t t = 0; t < n_threads; ++t) {
        jobs[t] = (orc_q_job){o, n, t, n_threads, packed, offs, kmers, out, ORC_OK};
        if (n_threads == 1) orc_query_worker(&jobs[0]);
        else pthread_create(&th[t], NULL, orc_query_worker, &jobs[t]);
    }
    int rc = ORC_OK;
    for (uint32_t t = 0; t < n_threads; ++t) {
        if (n_threads > 1) pthread_join(th[t], NULL);
        if (jobs[t].rc) rc = jobs[t].rc;
    }
    return rc;
}

int orc_query_seqs(const orc_rambo *o, uint64_t n, const uint8_t *packed, const uint64_t *offs,
                   uint32_t *out, uint32_t n_threads) {
    for (uint64_t i = 0; i < n; ++i)
        if (offs[i + 1] < offs[i]) return ORC_EINVAL;
    return orc_query_many(o, n, packed, offs, NULL, out, n_threads);
}

int orc_query_kmers(const orc_rambo *o, uint64_t n, const uint64_t *kmers, uint32_t *out,
                    uint32_t n_threads) {
    return orc_query_many(o, n, NULL, NULL, kmers, out, n_threads);
}

/* The eta probe positions h_1(x)..h_eta(x) (Section 2.1) of every term x of
 * every sequence i, Terms in window order (Section 3.3.1), written to
 * pos[(first term of i + s) * eta + j].  `pos` holds eta * (total terms).
 * Used to list the positions a restricted-mode oracle must track. */
int orc_seq_positions(const orc_rambo *o, uint64_t n, const uint8_t *packed, const uint64_t *offs,
                      uint64_t *pos) {
    uint64_t at = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (offs[i + 1] < offs[i]) return ORC_EINVAL;
        uint64_t n_bases = offs[i + 1] - offs[i];
        if (n_bases < o->k) continue;
        uint8_t *bases = (uint8_t *)malloc(n_bases);
        if (!bases) return ORC_ENOMEM;
        orc_unpack(packed, offs[i], n_bases, bases);
        for (uint64_t s = 0; s + o->k <= n_bases; ++s) {
            uint64_t x = orc_canonical_of_window(bases + s, o->k);
            for (uint32_t j = 0; j < o->eta; ++j) pos[at++] = orc_probe_position(o, x, j);
        }
        free(bases);
    }
    return ORC_OK;
}

/* Explicit partition (Section 5.3 two-level routing: a stacked RAMBO uses
 * bucket b*tau(D) + phi(D)).  phi[d*R + r] < B; only before any insert. */
int orc_set_partition(orc_rambo *o, const uint32_t *phi) {
    for (uint32_t d = 0; d < o->K; ++d)
        if (o->inserted[d]) return ORC_EINVAL;
    for (uint64_t i = 0; i < (uint64_t)o->K * o->R; ++i)
        if (phi[i] >= o->B) return ORC_EINVAL;
    memcpy(o->bucket, phi, sizeof(uint32_t) * (uint64_t)o->K * o->R);
    return ORC_OK;
}

/* Folding over (Section 5.3, Fig. 5): the BFUs of the second half of every
 * repetition are ORed onto the first half, B -> B/2, R unchanged.  Bucket
 * b + B/2 merges into bucket b, so DocIDs(M[b,r]) gains DocIDs(M[b+B/2,r])
 * and every document's bucket becomes phi_r(d) mod B/2.  Needs B even. */
int orc_fold(orc_rambo *o) {
    if (o->B < 2 || (o->B & 1)) return ORC_EINVAL;
    const uint32_t Bh = o->B / 2;
    const uint64_t words = (o->nbits + 63) / 64;
    uint64_t **filter = (uint64_t **)calloc((uint64_t)o->R * Bh, sizeof(uint64_t *));
    uint32_t **docs = (uint32_t **)calloc((uint64_t)o->R * Bh, sizeof(uint32_t *));
    uint32_t *ndocs = (uint32_t *)calloc((uint64_t)o->R * Bh, sizeof(uint32_t));
    uint32_t *capdocs = (uint32_t *)calloc((uint64_t)o->R * Bh, sizeof(uint32_t));
    if (!filter || !docs || !ndocs || !capdocs) {
        free(filter); free(docs); free(ndocs); free(capdocs);
        return ORC_ENOMEM;
    }
    for (uint32_t r = 0; r < o->R; ++r) {
        for (uint32_t b = 0; b < Bh; ++b) {
            const uint64_t lo = (uint64_t)r * o->B + b, hi = lo + Bh, nf = (uint64_t)r * Bh + b;
            /* bitwise OR of the two filters */
            for (uint64_t w = 0; w < words; ++w) o->filter[lo][w] |= o->filter[hi][w];
            filter[nf] = o->filter[lo];
            free(o->filter[hi]);
            /* union of the two document lists (disjoint: a document has one bucket) */
            const uint32_t n = o->ndocs[lo] + o->ndocs[hi];
            uint32_t *d = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
            if (!d) return ORC_ENOMEM;
            memcpy(d, o->docs[lo], sizeof(uint32_t) * o->ndocs[lo]);
            memcpy(d + o->ndocs[lo], o->docs[hi], sizeof(uint32_t) * o->ndocs[hi]);
            free(o->docs[lo]);
            free(o->docs[hi]);
            docs[nf] = d;
            ndocs[nf] = n;
            capdocs[nf] = n ? n : 1;
        }
    }
    free(o->filter); free(o->docs); free(o->ndocs); free(o->capdocs);
    o->filter = filter; o->docs = docs; o->ndocs = ndocs; o->capdocs = capdocs;
    for (uint64_t i = 0; i < (uint64_t)o->K * o->R; ++i) o->bucket[i] %= Bh;
    o->B = Bh;
    return ORC_OK;
}

/* Introspection for the tests. */
uint32_t orc_bucket_of(const orc_rambo *o, uint32_t d, uint32_t r) {
    return o->bucket[(uint64_t)d * o->R + r];
}
int orc_filter_bit(const orc_rambo *o, uint32_t r, uint32_t b, uint64_t pos) {
    int64_t s = orc_slot(o, pos);
    if (s < 0) return -1;
    return orc_get_bit(o->filter[(uint64_t)r * o->B + b], (uint64_t)s);
}
/* Copies filter (r,b) as raw 64-bit words (nbits bits, LSB-first). */
void orc_filter_words(const orc_rambo *o, uint32_t r, uint32_t b, uint64_t *dst) {
    memcpy(dst, o->filter[(uint64_t)r * o->B + b], sizeof(uint64_t) * ((o->nbits + 63) / 64));
}
/* Number of set bits of filter (r,b); the fill fraction is this / nbits. */
uint64_t orc_filter_popcount(const orc_rambo *o, uint32_t r, uint32_t b) {
    const uint64_t *f = o->filter[(uint64_t)r * o->B + b];
    uint64_t c = 0;
    for (uint64_t w = 0; w < (o->nbits + 63) / 64; ++w) c += (uint64_t)__builtin_popcountll(f[w]);
    return c;
}
int orc_is_inserted(const orc_rambo *o, uint32_t d) { return o->inserted[d]; }
/* The bits of every BFU at each of n positions: for position i, bit
 * r*B + b of the R*B-bit string at out + i * ceil(R*B/8) (LSB-first within
 * a byte) is bit pos[i] of filter (r,b).  ORC_EUNTRACKED if a position is
 * not kept (restricted mode). */
int orc_position_bits(const orc_rambo *o, uint64_t n, const uint64_t *pos, uint8_t *out) {
    const uint64_t nbf = (uint64_t)o->R * o->B, row = (nbf + 7) / 8;
    memset(out, 0, n * row);
    for (uint64_t i = 0; i < n; ++i) {
        const int64_t s = orc_slot(o, pos[i]);
        if (s < 0) return ORC_EUNTRACKED;
        for (uint64_t f = 0; f < nbf; ++f)
            if (orc_get_bit(o->filter[f], (uint64_t)s)) out[i * row + f / 8] |= (uint8_t)(1u << (f % 8));
    }
    return ORC_OK;
}

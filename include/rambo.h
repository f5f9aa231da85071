/*
 * rambo.h -- C ABI of the GB300 RAMBO library (librambo_gpu.so).
 *
 * RAMBO (Repeated And Merged BloOm filter; Gupta et al., SIGMOD'21) answers
 * "which of K documents contain every k-mer of this sequence?".  It keeps an
 * R x B table of Bloom filters ("BFUs", Section 2.1): in repetition r the K
 * documents are partitioned into B buckets by a hash phi_r of the document id,
 * and each bucket's documents are merged into one BFU of m bits probed by eta
 * hash functions (Section 3, Algorithm 1).  A query ANDs, per BFU, the
 * membership of all its k-mers, takes per repetition the union of the
 * documents of the passing BFUs, and intersects the R unions (Algorithm 2,
 * Section 3.3, Section 3.3.1).
 *
 * The library owns the index in GPU memory (HBM).  Every step of insertion
 * and query runs in the library's CUDA kernels; there is no CPU fallback.
 *
 * Conventions shared by every call
 * --------------------------------
 *  Sequences   2-bit packed: base t of a buffer is in byte t>>2 at bits
 *              2*(t&3)..2*(t&3)+1; A=0, C=1, G=2, T=3.  A batch is one packed
 *              buffer plus CSR base offsets (n+1 uint64): item i is bases
 *              [offsets[i], offsets[i+1]).  Offsets may start at any base;
 *              host calls read every byte holding bases [offsets[0],
 *              offsets[n]), device calls read at most `packed_bytes` bytes.
 *  Terms       canonical k-mers: min(forward code, reverse-complement code),
 *              forward code = first base most significant (Section 3.3.1,
 *              Section 5.1 "2-bit encoding"; canonical form is this library's
 *              strand-independent reading).
 *  Hashes      MurmurHash3_x64_128 over the 8-byte little-endian key, first
 *              64-bit output word.  Probe j uses seed (uint32)(seed + j) and
 *              is reduced mod m; document d goes to bucket
 *              hash(d, (uint32)(seed + 1000 + r)) mod B.  All BFUs share the
 *              probe positions (Section 5.3: every node uses the same h).
 *  Masks       a query answer is a K-bit document mask of W = ceil(K/32)
 *              uint32 words: document d is word d>>5, bit d&31; bits >= K are
 *              zero.  Only inserted documents can appear.  A query with no
 *              k-mer (length < k) returns every inserted document (Algorithm
 *              2's "for all x in Q" holds vacuously).
 *  Ownership   the caller owns every buffer it passes; the library keeps no
 *              pointer after a call returns (device calls: after the work
 *              enqueued on `stream` completes).  The library owns the index.
 *  Errors      every int-returning call returns RAMBO_OK (0) or a negative
 *              RAMBO_E* code; no exception crosses the ABI.  On error the
 *              outputs are unspecified.  Argument errors are detected before
 *              anything is enqueued, so the index is unchanged.  Device-side
 *              checks of device-resident data (doc id >= K, bad k-mer code,
 *              decreasing offsets) skip the offending item and latch an error
 *              that rambo_sync() reports.
 *  Threads     a handle is not thread-safe; serialise calls on one handle.
 *              Inserts and queries are ordered by the stream they are enqueued
 *              on (an insert is visible to every later query on that stream).
 */
#ifndef RAMBO_H
#define RAMBO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RAMBO_OK 0
#define RAMBO_EINVAL (-1)   /* bad argument (size, pointer, parameter, k-mer code) */
#define RAMBO_ENOMEM (-2)   /* device or host allocation failed                  */
#define RAMBO_ECUDA (-3)    /* a CUDA runtime call failed                        */
#define RAMBO_ERANGE (-4)   /* document id >= K                                  */
#define RAMBO_ETIMEOUT (-5) /* a bounded device wait gave up                     */
#define RAMBO_ESTATE (-6)   /* call not valid in the handle's current state      */

typedef struct rambo rambo_t;

/* Layout facts of a handle (all sizes in bytes unless noted). */
typedef struct {
    uint32_t K, B, R, eta, k;
    uint64_t m, seed;
    uint32_t mask_words;     /* W = ceil(K/32)                                    */
    uint32_t group_bytes;    /* bytes of one position group (all R*B bits of one */
                             /* probe position; power of two up to 512, then     */
                             /* multiples of 512)                                 */
    uint64_t index_bytes;    /* m * group_bytes                                    */
    uint64_t docbits_bytes;  /* R * B * W * 4: bucket -> document bitmaps         */
    int device;              /* CUDA device ordinal the index lives on            */
} rambo_info_t;

/* Creates an empty index (Section 3.2, "RAMBO <- B x R array of Bloom
 * Filters"; partition functions phi_r generated from `seed`).
 *   K   number of documents (ids 0..K-1), >= 1
 *   B   buckets (BFUs) per repetition, >= 1
 *   R   repetitions, >= 1
 *   m   bits per BFU, 1 <= m <= 2^32
 *   eta Bloom hash functions, 1..64
 *   k   k-mer length, 1..32
 *   seed base seed of the hash functions
 *   device CUDA device ordinal (-1 = the current device)
 * Allocates m*group_bytes of index plus R*B*W*4 of bitmaps on the device and
 * zeroes them.  Returns RAMBO_EINVAL on bad parameters, RAMBO_ENOMEM if the
 * index does not fit.  *out is set only on success. */
int rambo_create(uint32_t K, uint32_t B, uint32_t R, uint64_t m, uint32_t eta, uint32_t k,
                 uint64_t seed, int device, rambo_t **out);

/* Frees the index and every buffer the handle owns (waits for its work). */
int rambo_destroy(rambo_t *h);

/* W = ceil(K/32), the uint32 words of one answer mask (0 if h is NULL). */
uint32_t rambo_mask_words(const rambo_t *h);

int rambo_get_info(const rambo_t *h, rambo_info_t *info);

/* Human-readable name of an error code (static string). */
const char *rambo_strerror(int code);

/* ---------------------------------------------------------------------- */
/* Host-buffer calls: synchronous; inputs and outputs are host memory.     */
/* The library stages the data through its own device workspace.          */

/* Algorithm 1 for one document: every canonical k-mer of the n_bases bases
 * starting at base 0 of `packed` is inserted into BFU (phi_r(doc_id), r) for
 * every r.  Re-inserting a document or a k-mer is idempotent.  A document
 * shorter than k is still registered (it has no terms).
 * RAMBO_ERANGE if doc_id >= K. */
int rambo_insert(rambo_t *h, uint32_t doc_id, const uint8_t *packed, uint64_t n_bases);

/* Algorithm 1 for n_docs documents: document i has id doc_ids[i] and bases
 * [base_offsets[i], base_offsets[i+1]) of `packed`.  base_offsets has
 * n_docs+1 non-decreasing entries.  RAMBO_ERANGE if any id >= K (nothing is
 * inserted then). */
int rambo_insert_batch(rambo_t *h, uint32_t n_docs, const uint32_t *doc_ids,
                       const uint8_t *packed, const uint64_t *base_offsets);

/* Algorithm 2 for n single k-mers.  kmers[i] is a forward code (first base
 * most significant, 2 bits per base); it is canonicalised inside.  A code
 * with a bit set at or above 2k is found on the device: the call still runs
 * to the end, returns RAMBO_EINVAL and leaves `out` unspecified.  out
 * receives n*W words (query i at out + i*W).  Same as rambo_query_batch with
 * no sequences. */
int rambo_query_kmers(rambo_t *h, uint64_t n, const uint64_t *kmers, uint32_t *out);

/* Section 3.3.1 sequence queries: the answer for sequence i (bases
 * [base_offsets[i], base_offsets[i+1]) of `packed`) is the set of documents
 * whose BFUs pass every k-mer of the sequence in every repetition.  out
 * receives n*W words. */
int rambo_query_seqs(rambo_t *h, uint64_t n, const uint8_t *packed, const uint64_t *base_offsets,
                     uint32_t *out);

/* One batch of both query kinds (either count may be 0): n_kmers single
 * k-mers as in rambo_query_kmers (answers to out_kmers, n_kmers*W words) and
 * n_seqs sequences as in rambo_query_seqs (answers to out_seqs, n_seqs*W
 * words).  The two kinds run concurrently on the GPU, and the k-mers are
 * pipelined in chunks (tuning knob host_chunk_kmers) so that copies to and
 * from the host overlap the kernels.  Page-locked host buffers (e.g. from
 * cudaMallocHost) make every copy asynchronous; pageable buffers work but
 * serialise the copies.  Synchronous; errors as in the two calls above. */
int rambo_query_batch(rambo_t *h, uint64_t n_kmers, const uint64_t *kmers, uint32_t *out_kmers,
                      uint64_t n_seqs, const uint8_t *packed, const uint64_t *base_offsets,
                      uint32_t *out_seqs);

/* ---------------------------------------------------------------------- */
/* Device-buffer calls: asynchronous on `stream` (a cudaStream_t, NULL =    */
/* the legacy default stream).  Pointers are device memory.  Each call     */
/* needs a caller-provided device workspace of at least the size returned  */
/* by the matching *_workspace() call, 256-byte aligned; a workspace must   */
/* not be shared by calls that may run at the same time.  `packed_bytes`   */
/* bounds every read of `packed` (any alignment is accepted).  Errors       */
/* found on the device are latched and reported by rambo_sync().            */

size_t rambo_insert_workspace(const rambo_t *h, uint64_t n_docs);
size_t rambo_query_kmers_workspace(const rambo_t *h, uint64_t n);
size_t rambo_query_seqs_workspace(const rambo_t *h, uint64_t n);
/* Workspace with which a batch of n sequences over packed_bytes bytes can
 * take the tuned query path: query_path 2 (region-binned probing) needs room
 * for its probe records, query_path 3 (content-ordered segments) for its
 * segment lists, and each runs only when the workspace passed to the call
 * is at least this large; with less (down to rambo_query_seqs_workspace) the
 * call takes path 1.  Same answers either way. */
size_t rambo_query_seqs_workspace_for(const rambo_t *h, uint64_t n, uint64_t packed_bytes);

int rambo_insert_batch_dev(rambo_t *h, uint32_t n_docs, const uint32_t *doc_ids,
                           const uint8_t *packed, uint64_t packed_bytes,
                           const uint64_t *base_offsets, void *workspace, size_t workspace_bytes,
                           void *stream);

/* rambo_insert_batch_dev with documents given as separate ranges: document
 * doc_ids[i] is bases [begins[i], ends[i]) of `packed` (n_docs entries each,
 * device memory), so a subset of a packed corpus -- e.g. the documents one
 * shard of a document-sharded index holds (Section 5.3) -- is inserted
 * without repacking.  Ranges may overlap.  Workspace:
 * rambo_insert_workspace(h, n_docs).  Same errors as rambo_insert_batch_dev;
 * insert_mode 3 takes the direct insert here. */
int rambo_insert_ranges_dev(rambo_t *h, uint32_t n_docs, const uint32_t *doc_ids,
                            const uint8_t *packed, uint64_t packed_bytes, const uint64_t *begins,
                            const uint64_t *ends, void *workspace, size_t workspace_bytes,
                            void *stream);

/* Answers of a document-sharded deployment (Section 5.3: a routing hash
 * sends each document to one shard, whose RAMBO holds it as a local
 * document; the stacked structure answers a query with the union of the
 * shards' answers, each placed at its documents' global ids).  ORs the n
 * answer rows of one shard (shard_masks: n x shard_words uint32, bit j =
 * local document j, j < shard_docs) into `out` (n x out_words uint32, bit d =
 * global document d) at bits global_ids[j] (shard_docs uint32).  All
 * pointers are device memory; `out` starts zeroed and is ORed into, so
 * merging every shard yields the global answers.  Ids at or past
 * 32*out_words are skipped.  Asynchronous on `stream`; RAMBO_EINVAL for
 * missing pointers or shard_words < ceil(shard_docs/32). */
int rambo_merge_shard_answers(uint64_t n, const uint32_t *shard_masks, uint32_t shard_words,
                              uint32_t shard_docs, const uint32_t *global_ids, uint32_t *out,
                              uint32_t out_words, void *stream);

int rambo_query_kmers_dev(rambo_t *h, uint64_t n, const uint64_t *kmers, uint32_t *out,
                          void *workspace, size_t workspace_bytes, void *stream);

int rambo_query_seqs_dev(rambo_t *h, uint64_t n, const uint8_t *packed, uint64_t packed_bytes,
                         const uint64_t *base_offsets, uint32_t *out, void *workspace,
                         size_t workspace_bytes, void *stream);

/* Device-buffer form of rambo_query_batch: the k-mer part and the sequence
 * part of one batch, each as in rambo_query_kmers_dev / rambo_query_seqs_dev,
 * in one workspace of rambo_query_batch_workspace(h, n_kmers, n_seqs,
 * packed_bytes) bytes (the k-mer part first; a smaller one down to the two
 * parts' minimum sizes is accepted, as for rambo_query_seqs_workspace_for).
 * With both parts present the k-mer part is forked onto a stream the handle
 * owns (an event recorded on `stream`) and joined back (`stream` waits for
 * it), so the parts run concurrently and the call may be captured into a
 * CUDA graph from `stream`.  Because that side stream belongs to the handle,
 * two such calls on one handle do not overlap their k-mer parts. */
size_t rambo_query_batch_workspace(const rambo_t *h, uint64_t n_kmers, uint64_t n_seqs,
                                   uint64_t packed_bytes);
int rambo_query_batch_dev(rambo_t *h, uint64_t n_kmers, const uint64_t *kmers, uint32_t *out_kmers,
                          uint64_t n_seqs, const uint8_t *packed, uint64_t packed_bytes,
                          const uint64_t *base_offsets, uint32_t *out_seqs, void *workspace,
                          size_t workspace_bytes, void *stream);

/* Sequence query that allocates nothing.  The paper has no counterpart: this
 * exists for callers that cannot allocate device memory -- hosts that own
 * every device byte and forbid library allocations, and latency-critical
 * threads that must never reach cudaMalloc/cudaFree (which can block on or
 * synchronise the device).  Same arguments, results and errors as
 * rambo_query_seqs_dev, but the workspace is one static device array of
 * RAMBO_STATIC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  A batch whose rambo_query_seqs_workspace(h, n) exceeds
 * RAMBO_STATIC_SCRATCH_BYTES is rejected with RAMBO_EINVAL before anything is
 * enqueued.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device); make that first call before any
 * stream capture.  The address is kept for the rest of the process, so
 * after a cudaDeviceReset of that device (which ends every handle on it as
 * well) this entry point must not be called again in the same process.
 * Every call on a device shares the one array, so calls whose work can
 * overlap on the GPU (different streams, or handles on the same device)
 * race: serialise them.  With query_path 2 or 3 the region-binned or the
 * content-ordered path runs when its records or segment lists fit the array
 * as well, else path 1. */
#define RAMBO_STATIC_SCRATCH_BYTES (8u << 20)
int rambo_query_seqs_noalloc(rambo_t *h, uint64_t n, const uint8_t *packed, uint64_t packed_bytes,
                             const uint64_t *base_offsets, uint32_t *out, void *stream);

/* rambo_query_seqs_dev with items given as separate ranges: item i is bases
 * [begins[i], ends[i]) of `packed` (n entries each, device memory), so items
 * may be placed anywhere -- e.g. each at a byte boundary of a buffer that
 * concatenates independently packed requests.  Same workspace size as
 * rambo_query_seqs_workspace(h, n). */
int rambo_query_ranges_dev(rambo_t *h, uint64_t n, const uint8_t *packed, uint64_t packed_bytes,
                           const uint64_t *begins, const uint64_t *ends, uint32_t *out,
                           void *workspace, size_t workspace_bytes, void *stream);

/* ---------------------------------------------------------------------- */
/* Documents of words (Section 5.4 "Document indexing": a document is a    */
/* set of word unigrams).  A term is an arbitrary byte string; probe j of a */
/* term is MurmurHash3_x64_128(term bytes, (uint32)(seed + j)) first word   */
/* mod m, so index, partition and expansion are the k-mer ones.  Device     */
/* buffers, asynchronous on `stream`.  Term t is bytes [term_offs[t],       */
/* term_offs[t+1]) of `bytes` (bytes_len readable bytes); item i is terms   */
/* [item_terms[i], item_terms[i+1]) (n+1 entries), and term_offs must have  */
/* item_terms[n]+1 entries.  Terms past bytes_len are skipped and latched   */
/* (rambo_sync).                                                            */

/* Algorithm 1 for word documents: document i (id doc_ids[i]) is the terms
 * [doc_terms[i], doc_terms[i+1]).  Needs no workspace. */
int rambo_insert_words_dev(rambo_t *h, uint32_t n_docs, const uint32_t *doc_ids,
                           const uint8_t *bytes, uint64_t bytes_len, const uint64_t *term_offs,
                           const uint64_t *doc_terms, void *stream);

size_t rambo_query_words_workspace(const rambo_t *h, uint64_t n);

/* Algorithm 2 for n word queries: query i passes a BFU iff every one of its
 * terms [query_terms[i], query_terms[i+1]) does.  out receives n*W words. */
int rambo_query_words_dev(rambo_t *h, uint64_t n, const uint8_t *bytes, uint64_t bytes_len,
                          const uint64_t *term_offs, const uint64_t *query_terms, uint32_t *out,
                          void *workspace, size_t workspace_bytes, void *stream);

/* Waits for `stream` and returns the first device-side error latched since
 * the last rambo_sync (then clears it), or RAMBO_OK. */
int rambo_sync(rambo_t *h, void *stream);

/* Replaces the partition functions by an explicit map: phi[d*R + r] (host,
 * K*R values < B) is document d's bucket in repetition r.  This is how a
 * stacked, document-sharded deployment is expressed as one index (Section
 * 5.3: bucket b*tau(D) + phi_i(D) over S shards of b buckets each).  Allowed
 * only before the first insert (RAMBO_ESTATE afterwards); RAMBO_EINVAL if a
 * bucket is out of range.  Folding afterwards recomputes the default
 * partition. */
int rambo_set_partition(rambo_t *h, const uint32_t *phi);

/* ---------------------------------------------------------------------- */
/* Folding over (Section 5.3, Fig. 5): every repetition's BFUs of buckets   */
/* B/2..B-1 are ORed onto buckets 0..B/2-1, halving B and the index while R */
/* stays; bucket b+B/2's documents join bucket b.  Because phi_r(d) = h mod */
/* B and B/2 divides B, the result equals an index built with B/2 buckets   */
/* from the same documents.  Synchronous; B must be even and the groups at  */
/* most 512 bytes (RAMBO_EINVAL otherwise).  On failure (RAMBO_ENOMEM when  */
/* the folded index cannot be allocated next to the current one) the index  */
/* is unchanged.  Answers can only gain false positives.                    */
int rambo_fold(rambo_t *h);

/* ---------------------------------------------------------------------- */
/* Introspection (host copies; synchronous).                               */

/* Copies `nbytes` of the index starting at byte `offset` to host `dst`.
 * The index is m position groups of group_bytes; in group p, bit r*B+b (word
 * (r*B+b)>>5, bit (r*B+b)&31) is bit p of BFU (b, r). */
int rambo_copy_index(const rambo_t *h, uint64_t offset, uint64_t nbytes, void *dst);

/* Copies the R*B*W-word bucket->document bitmaps: bucket b of repetition r
 * at words (r*B+b)*W .. +W; bit d set iff document d was inserted and
 * phi_r(d) = b (DocIDs(M[b,r]) of Algorithm 2). */
int rambo_copy_docbits(const rambo_t *h, uint32_t *dst);

/* Copies phi: dst[d*R + r] = bucket of document d in repetition r. */
int rambo_copy_partition(const rambo_t *h, uint32_t *dst);

/* ---------------------------------------------------------------------- */
/* Tuning knobs (launch shapes; none changes any result).                  */

typedef struct {
    uint32_t probe_ctas_per_sm;        /* probe grid = SMs x this; 0 = occupancy max */
    uint32_t probe_min_kmers_per_warp; /* smallest k-mer range a warp takes; 0 = 64  */
    uint32_t expand_ctas_per_sm;       /* expansion grid cap = SMs x this (1..64)    */
    uint32_t use_byte_table;           /* 1: expand through a per-8-bucket OR table  */
    uint32_t byte_table_max_mb;        /* ... only if it fits this many MiB          */
    uint32_t query_path;               /* sequence queries: 0 = prefix scan + probe +  */
                                       /* expand launches; 1 = persistent fused launch */
                                       /* with length-bucketed work queues (groups up  */
                                       /* to 512 B; otherwise path 0 is used); 2 =     */
                                       /* region-binned probing (groups up to 64 B    */
                                       /* and a workspace from                         */
                                       /* rambo_query_seqs_workspace_for; otherwise    */
                                       /* path 1); 3 = content-ordered segments: the   */
                                       /* batch's k-mers cut at content-defined points */
                                       /* and probed in the order of the segments'     */
                                       /* keys, so k-mers repeated across queries find */
                                       /* their groups in L2 (groups up to 64 B, eta   */
                                       /* <= 4, CSR batches, a workspace from          */
                                       /* rambo_query_seqs_workspace_for; otherwise    */
                                       /* path 1)                                      */
    uint32_t fused_tile_kmers;         /* path 1: k-mers per tile of a long query      */
    uint32_t fused_short_max;          /* path 1: queries with at most this many       */
                                       /* k-mers are probed and expanded by one warp   */
    uint32_t smem_docbits;             /* 1: expansion stages the bucket->document     */
                                       /* bitmaps in shared memory when they fit       */
    uint32_t use_nibble_table;         /* 1: expansion through a per-4-bucket OR table */
                                       /* staged in shared memory, when it fits 96 KiB */
    uint32_t expand_filter;            /* 1: expansion forms repetition 0's union and  */
                                       /* then tests only surviving documents against  */
                                       /* the later repetitions (needs the nibble      */
                                       /* table, B <= 256 and a small K)               */
    uint32_t early_exit;               /* path 1: stop probing a query once one of its */
                                       /* repetition rows is empty (its answer is then */
                                       /* empty; Section 3.3.1 "the first FALSE is     */
                                       /* conclusive", Section 5.1 RAMBO+).  Off by    */
                                       /* default: every k-mer is probed               */
    uint32_t early_exit_segment;       /* k-mers between checks (multiple of 128)      */
    uint32_t kmer_probe_ctas_per_sm;   /* single-k-mer probe grid = SMs x this;        */
                                       /* 0 = as probe_ctas_per_sm                     */
    uint32_t host_chunk_kmers;         /* host-buffer calls: k-mers per pipelined      */
                                       /* chunk (copy in, query, copy out); 0 = about  */
                                       /* 16 MiB of answers per chunk; the first chunk */
                                       /* is an eighth of it                           */
    uint32_t branch_priority;          /* mixed batches: 0 = both kinds at the caller's */
                                       /* stream priority; 1 = sequences, 2 = k-mers  */
                                       /* on a stream of the greatest priority        */
    uint32_t host_slots;               /* host-buffer calls: k-mer chunks in flight    */
                                       /* (1..RAMBO_MAX_HOST_SLOTS; default 3)         */
    uint32_t bin_region_kib;           /* path 2: index bytes per region (KiB; 0 =     */
                                       /* 32768); regions hold a power-of-two number   */
                                       /* of groups and are at most 4096              */
    uint32_t bin_rows;                 /* path 2: group gathers a lane keeps in flight */
                                       /* in the probe pass: 4, 8, 12 for 1, 2 (or 0), */
                                       /* 4 and 8                                      */
    uint32_t host_direct;              /* host-buffer calls: 1 = kernels write answers */
                                       /* straight into output buffers that are        */
                                       /* page-locked and device-addressable (each     */
                                       /* must be one such allocation); others are     */
                                       /* staged and copied as with 0 (the default)    */
    uint32_t host_fused_ctas_per_sm;   /* host-buffer batches with both kinds: the     */
                                       /* persistent fused launch takes at most this   */
                                       /* many CTAs per SM (0 = as probe_ctas_per_sm;  */
                                       /* default 1), leaving room for the k-mer       */
                                       /* chunks whose copies out bound the call       */
    uint32_t insert_mode;              /* Algorithm 1's bit setting: 0 = lanes hitting */
                                       /* one word combine first (match + OR-reduce);  */
                                       /* 1 = one 32-bit atomicOr per repetition; 2    */
                                       /* (default) = as 1 with repetitions that share */
                                       /* a 64-bit word merged into one 64-bit         */
                                       /* atomicOr (32-bit when m * Gw is odd); 3 =    */
                                       /* binned by index region (bin_region_kib):     */
                                       /* probes are first written as 8-byte records   */
                                       /* per region, then applied region by region so */
                                       /* the atomics hit L2 -- for indexes of at most */
                                       /* 1024 regions, K <= 2^24 and m <= 2^40, else  */
                                       /* as 2.  Choosing 3 reserves the record buffer */
                                       /* (RAMBO_ENOMEM if it cannot be had)           */
    uint32_t insert_bin_records;       /* insert_mode 3: records the buffer holds      */
                                       /* (8 bytes each; 0 = 2^28, else >= 4096); a    */
                                       /* batch is applied in chunks that fill it (a   */
                                       /* batch needing over 65536 chunks is inserted  */
                                       /* directly)                                    */
    uint32_t fused_async;              /* query_path 1, 16-byte groups, eta <= 2: 1 =  */
                                       /* the probes' gathers land in shared memory    */
                                       /* (cp.async) instead of registers, so the      */
                                       /* launch needs fewer registers (default 0)     */
    uint32_t kmer_async;               /* the same for the single k-mer probe (16-byte */
                                       /* groups, eta <= 2; default 0)                 */
    uint32_t seg_cut_bits;             /* query_path 3: a k-mer whose order hash has   */
                                       /* this many low zero bits starts a segment     */
                                       /* (segments of about 2^bits k-mers, at least   */
                                       /* 2^(bits-1)); 0 = 6 (the default), <= 10      */
} rambo_tuning_t;
#define RAMBO_MAX_HOST_SLOTS 4

int rambo_get_tuning(const rambo_t *h, rambo_tuning_t *out);
/* Applies new knobs after waiting for the handle's stream; RAMBO_EINVAL if a
 * knob is out of range.  Results are bit-identical for every setting. */
int rambo_set_tuning(rambo_t *h, const rambo_tuning_t *t);

/* ---------------------------------------------------------------------- */
/* Measurement support (not part of the paper).                            */

/* Random-record gather on the current device: n_probes reads of
 * record_bytes (16..512, power of two) at pseudo-random record indices of
 * `buf` (device, 16-byte aligned, buf_bytes long), with load instruction
 * variant 0..5 (0 = the probe kernels' streaming load) and `unroll` (4, 8, 16
 * or 32) 16-byte loads in flight per lane.  XOR of the data goes
 * to the 8-byte device word `sink`.  Asynchronous on `stream`. */
int rambo_probe_gather(const void *buf, uint64_t buf_bytes, uint32_t record_bytes,
                       uint64_t n_probes, uint32_t load_variant, uint32_t unroll, uint64_t seed,
                       void *sink, void *stream);

/* Failure-detection check: enqueues on `stream` one kernel whose thread
 * polls, without suspending, an mbarrier that nothing ever completes, and
 * gives up after `spins` polls (1..2^22).  The wait runs out and latches the
 * error that the next rambo_sync on that stream reports as RAMBO_ETIMEOUT;
 * nothing faults or hangs, and the handle stays usable.  RAMBO_EINVAL for
 * spins out of range. */
int rambo_probe_wait_expiry(rambo_t *h, uint64_t spins, void *stream);

/* ---------------------------------------------------------------------- */
/* Profiling.  The library counts every kernel it launches, per stage, and */
/* can bracket the launches of selected stages with CUDA events recorded on */
/* the launching stream.  (Not part of the paper: measurement support.)    */

#define RAMBO_STAGE_PREFIX 0      /* k-mer count prefix scan (3 kernels)      */
#define RAMBO_STAGE_REGISTER 1    /* bucket->document bitmap registration     */
#define RAMBO_STAGE_INSERT 2      /* Algorithm 1 bit setting                  */
#define RAMBO_STAGE_PROBE_SEQS 3  /* sequence probe + bucket-space AND        */
#define RAMBO_STAGE_PROBE_KMERS 4 /* single k-mer probe                        */
#define RAMBO_STAGE_EXPAND 5      /* union per repetition, AND over R          */
#define RAMBO_NUM_STAGES 6

typedef struct {
    uint64_t launches[RAMBO_NUM_STAGES]; /* kernels launched since the last reset      */
    uint64_t timed[RAMBO_NUM_STAGES];    /* launches bracketed by events                */
    double ms[RAMBO_NUM_STAGES];         /* summed event time of the bracketed launches */
} rambo_profile_t;

/* Resets the counters and selects the stages whose launches are bracketed
 * by events (bit s of stage_mask = stage s; 0 = counting only). */
int rambo_profile_reset(rambo_t *h, uint32_t stage_mask);

/* Waits for every recorded event, then copies the counters to *out. */
int rambo_profile_read(rambo_t *h, rambo_profile_t *out);

/* k-mers the fused path actually probed while early_exit was on (waits for
 * the device); reset != 0 zeroes the counter afterwards. */
int rambo_probed_kmers(rambo_t *h, uint64_t *out, int reset);

#ifdef __cplusplus
}
#endif

#endif /* RAMBO_H */

// rambo_kernels_expand.cu -- expansion kernels of the batched query
// (Algorithm 2's union and intersection): per repetition, the OR of the
// document bitmaps of the passing buckets; then the AND over the R
// repetitions, written as a K-bit mask.  Also the OR tables they use.
#include "rambo_query_common.cuh"

namespace rgpu {
namespace {

// SMEM: DocBits is first copied into shared memory by the whole block.
template <int C, bool SMEM>
__global__ void __launch_bounds__(EXPAND_THREADS) k_expand(ExpandArgs a) {
    extern __shared__ uint32_t sdb[];
    if (SMEM) {
        const uint32_t words = a.R * a.B * a.W;
        for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) sdb[i] = __ldg(a.docbits + i);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (uint64_t)blockIdx.x * (EXPAND_THREADS / 32) + threadIdx.x / 32;
    const uint64_t nwarps = (uint64_t)gridDim.x * (EXPAND_THREADS / 32);
    const uint32_t chunks = (a.W + 32 * C - 1) / (32 * C);
    const uint64_t units = a.n * chunks;
    for (uint64_t u = warp; u < units; u += nwarps) {
        const uint64_t q = chunks == 1 ? u : u / chunks;
        const uint32_t w0 = (uint32_t)(u - q * chunks) * 32 * C + lane;
        if (SMEM) expand_unit_smem<C>(a, sdb, a.acc + q * a.Gw, q, w0);
        else expand_one<C>(a, a.acc + q * a.Gw, q, w0, lane);
    }
}

// Expansion through the nibble table in shared memory (small K): one query
// per warp, every lane holding up to 32*C answer words.  The query's bucket
// mask (Gw <= 32 words) sits in lane registers, one word per lane, and rows
// are fetched 32 bits at a time with shuffles; every nonzero 4-bucket nibble
// of a row costs one conflict-free shared-memory row read.
constexpr size_t SMEM_NIBTAB_MAX = 96 * 1024;

// Several queries per warp: LPQ lanes per query, each lane owning a 16-byte
// slice (4 answer words) of its query, so the per-nibble extract and address
// work is shared by 32/LPQ queries per warp instruction.  Table rows are
// staged in shared memory padded to W4 = 4*ceil(W/4) words; an empty row (a
// nibble of value 0) is all zero, so no lookup needs a branch and an empty
// repetition makes the answer zero by itself.
template <int LPQ, int VPL>
__global__ void __launch_bounds__(EXPAND_THREADS) k_expand_nib(ExpandArgs a) {
    extern __shared__ uint4 stab4[];
    const uint32_t NQ = (a.B + 3) / 4;
    const uint32_t RW = (a.W + 3) / 4;  // uint4 per padded row
    const uint32_t rows = a.R * NQ * 16;
    uint32_t *stab = reinterpret_cast<uint32_t *>(stab4);
    for (uint32_t i = threadIdx.x; i < rows * RW * 4; i += blockDim.x) {
        const uint32_t row = i / (RW * 4), w = i - row * (RW * 4);
        stab[i] = w < a.W ? __ldg(a.ntab + (uint64_t)row * a.W + w) : 0u;
    }
    __syncthreads();
    constexpr int QPW = 32 / LPQ;
    const int lane = threadIdx.x & 31;
    const int sub = lane / LPQ, ch = lane % LPQ;  // lane owns uint4 slices ch*VPL .. +VPL-1
    const uint64_t warp = (uint64_t)blockIdx.x * (EXPAND_THREADS / 32) + threadIdx.x / 32;
    const uint64_t nwarps = (uint64_t)gridDim.x * (EXPAND_THREADS / 32);
    const uint32_t c0 = (uint32_t)ch * VPL;
    for (uint64_t q0 = warp * QPW; q0 < a.n; q0 += nwarps * QPW) {
        const uint64_t q = q0 + sub;
        const bool valid = q < a.n && c0 < RW;
        const uint32_t *bm = a.acc + q * a.Gw;
        uint4 res[VPL];
#pragma unroll
        for (int v = 0; v < VPL; ++v) res[v] = make_uint4(FULL, FULL, FULL, FULL);
        const uint4 *tj = stab4 + (c0 < RW ? c0 : 0);
        for (uint32_t r = 0; r < a.R; ++r) {
            uint4 o[VPL];
#pragma unroll
            for (int v = 0; v < VPL; ++v) o[v] = make_uint4(0, 0, 0, 0);
            for (uint32_t i = 0; i < a.B; i += 32) {
                uint32_t chunk = 0;
                if (valid) {
                    const uint32_t bit = r * a.B + i, wi = bit >> 5, sh = bit & 31;
                    chunk = __ldg(bm + wi);
                    if (sh) chunk = __funnelshift_r(chunk, wi + 1 < a.Gw ? __ldg(bm + wi + 1) : 0u, sh);
                    const uint32_t nb = a.B - i < 32 ? a.B - i : 32;
                    if (nb < 32) chunk &= (1u << nb) - 1u;
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    if (i + 4 * t < a.B) {
                        const uint4 *row = tj + ((chunk >> (4 * t)) & 15u) * RW;
#pragma unroll
                        for (int v = 0; v < VPL; ++v) {
                            const uint4 x = row[v];
                            o[v].x |= x.x; o[v].y |= x.y; o[v].z |= x.z; o[v].w |= x.w;
                        }
                        tj += 16 * RW;
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                res[v].x &= o[v].x; res[v].y &= o[v].y; res[v].z &= o[v].z; res[v].w &= o[v].w;
            }
        }
        if (valid) {
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const uint32_t w0 = 4 * (c0 + v);
                if (w0 >= a.W) break;
                uint32_t *out = a.out + q * a.W + w0;
                const uint32_t left = a.W - w0;
                out[0] = res[v].x;
                if (left > 1) out[1] = res[v].y;
                if (left > 2) out[2] = res[v].z;
                if (left > 3) out[3] = res[v].w;
            }
        }
    }
}

// Nibble-table expansion for B a multiple of 32 (each repetition's row of
// the bucket mask is B/32 whole words).  Rows are staged at a power-of-two
// stride of RWP 16-byte slices (RWP >= ceil(W/4)), every lane owns one slice
// of one query (RWP lanes per query, 32/RWP queries per warp), and a lookup
// is a shift, a mask, an add and one 16-byte shared-memory read at an offset
// known at compile time up to the nibble: no per-lookup branches or
// multiplies.  The RWP lanes of a query read one contiguous row, so a warp's
// read takes the minimum 32*16/128 = 4 shared-memory wavefronts.
template <int RWP>
__global__ void __launch_bounds__(EXPAND_THREADS) k_expand_nib32(ExpandArgs a) {
    extern __shared__ uint4 stab4[];
    constexpr int QPW = 32 / RWP;
    constexpr uint32_t RS = RWP * 16;  // bytes per staged row
    constexpr uint32_t SEC = 16 * RS;  // bytes per (repetition, nibble) section
    const uint32_t rows = a.R * (a.B / 4) * 16;
    uint32_t *stab = reinterpret_cast<uint32_t *>(stab4);
    for (uint32_t i = threadIdx.x; i < rows * RWP * 4; i += blockDim.x) {
        const uint32_t row = i / (RWP * 4), w = i % (RWP * 4);
        stab[i] = w < a.W ? __ldg(a.ntab + (uint64_t)row * a.W + w) : 0u;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane / RWP, ch = lane % RWP;
    const char *tb = reinterpret_cast<const char *>(stab4) + ch * 16;
    const uint32_t BW = a.B / 32;  // mask words per repetition
    const uint32_t w0 = 4u * (uint32_t)ch;
    const bool vec_store = (a.W & 3u) == 0 && (reinterpret_cast<uintptr_t>(a.out) & 15u) == 0;
    const uint64_t warp = (uint64_t)blockIdx.x * (EXPAND_THREADS / 32) + threadIdx.x / 32;
    const uint64_t nwarps = (uint64_t)gridDim.x * (EXPAND_THREADS / 32);
    for (uint64_t q0 = warp * QPW; q0 < a.n; q0 += nwarps * QPW) {
        const uint64_t q = q0 + sub;
        const bool valid = q < a.n;
        const uint32_t *bm = a.acc + (valid ? q : 0) * a.Gw;
        uint4 res = make_uint4(FULL, FULL, FULL, FULL);
        uint32_t off = 0;
        for (uint32_t r = 0; r < a.R; ++r) {
            uint4 o = make_uint4(0, 0, 0, 0);
            for (uint32_t wd = 0; wd < BW; ++wd) {
                const uint32_t chunk = valid ? __ldg(bm + r * BW + wd) : 0u;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const uint4 x = *reinterpret_cast<const uint4 *>(
                        tb + off + t * SEC + ((chunk >> (4 * t)) & 15u) * RS);
                    o.x |= x.x; o.y |= x.y; o.z |= x.z; o.w |= x.w;
                }
                off += 8 * SEC;
            }
            res.x &= o.x; res.y &= o.y; res.z &= o.z; res.w &= o.w;
        }
        if (valid && w0 < a.W) {
            uint32_t *out = a.out + q * a.W + w0;
            if (vec_store) {
                *reinterpret_cast<uint4 *>(out) = res;
            } else {
                const uint32_t left = a.W - w0;
                out[0] = res.x;
                if (left > 1) out[1] = res.y;
                if (left > 2) out[2] = res.z;
                if (left > 3) out[3] = res.w;
            }
        }
    }
}

// Expansion by candidate filtering (the paper's sparse evaluation, Section
// 5.1 "Query time speedup", applied per document): the union of repetition 0
// is formed from the nibble table (its repetition-0 rows staged in shared
// memory); for every later repetition r only the documents still set are
// tested -- document d survives iff bit phi_r(d) of row r is set -- with phi
// staged in shared memory as bytes (B <= 256) and the query's bucket mask in
// a per-warp shared slot.  The surviving set after the last repetition is
// exactly AND_r of the unions.  One query per warp, each lane owning answer
// words lane + 32c (W <= 32*C); Gw <= 32.
template <int C>
__global__ void __launch_bounds__(EXPAND_THREADS) k_expand_filter(ExpandArgs a) {
    extern __shared__ uint32_t smem_f[];
    const uint32_t NQ = (a.B + 3) / 4;
    const uint32_t tab0 = NQ * 16 * a.W;  // nibble-table words of repetition 0
    uint32_t *stab = smem_f;
    uint32_t *sbm = smem_f + tab0;        // EXPAND_THREADS/32 slots of 32 words
    uint8_t *sphi = reinterpret_cast<uint8_t *>(sbm + EXPAND_THREADS);  // K*R bytes
    for (uint32_t i = threadIdx.x; i < tab0; i += blockDim.x) stab[i] = __ldg(a.ntab + i);
    for (uint32_t i = threadIdx.x; i < a.K * a.R; i += blockDim.x) sphi[i] = (uint8_t)__ldg(a.phi + i);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint32_t *bm = sbm + (threadIdx.x / 32) * 32;
    const uint64_t warp = (uint64_t)blockIdx.x * (EXPAND_THREADS / 32) + threadIdx.x / 32;
    const uint64_t nwarps = (uint64_t)gridDim.x * (EXPAND_THREADS / 32);
    for (uint64_t q = warp; q < a.n; q += nwarps) {
        bm[lane] = (uint32_t)lane < a.Gw ? __ldg(a.acc + q * a.Gw + lane) : 0u;
        __syncwarp();
        // repetition 0: union of the passing buckets via the nibble table
        uint32_t res[C];
#pragma unroll
        for (int c = 0; c < C; ++c) res[c] = 0;
        for (uint32_t i = 0; i < a.B; i += 32) {
            uint32_t chunk = bm[i >> 5];
            const uint32_t nb = a.B - i < 32 ? a.B - i : 32;
            if (nb < 32) chunk &= (1u << nb) - 1u;
            const uint32_t j0 = i / 4;
            while (chunk) {
                const uint32_t t = (__ffs(chunk) - 1) & ~3u;
                const uint32_t v = (chunk >> t) & 15u;
                chunk &= ~(15u << t);
                const uint32_t *row = stab + (((j0 + t / 4) * 16 + v) * a.W);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t w = lane + 32 * c;
                    if (w < a.W) res[c] |= row[w];
                }
            }
        }
        // repetitions 1..R-1: keep the candidates whose bucket passes
        for (uint32_t r = 1; r < a.R; ++r) {
            uint32_t nz = 0;
            const uint32_t lo = r * a.B;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                uint32_t x = res[c], keep = 0;
                const uint32_t d0 = 32 * (lane + 32 * c);
                while (x) {
                    const uint32_t j = __ffs(x) - 1;
                    x &= x - 1;
                    const uint32_t bit = lo + sphi[(d0 + j) * a.R + r];
                    keep |= ((bm[bit >> 5] >> (bit & 31)) & 1u) << j;
                }
                res[c] = keep;
                nz |= keep;
            }
            if (!__any_sync(FULL, nz)) break;
        }
        uint32_t *out = a.out + q * a.W;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const uint32_t w = lane + 32 * c;
            if (w < a.W) out[w] = res[c];
        }
        __syncwarp();
    }
}

// Nibble table: ntab[((r*NQ + j)*16 + v)*W + w] = OR over set bits t of v
// (4j+t < B) of DocBits[r][4j+t][w].
__global__ void k_build_nibtab(const uint32_t *docbits, uint32_t B, uint32_t R, uint32_t W,
                               uint32_t *ntab) {
    const uint32_t NQ = (B + 3) / 4;
    const uint64_t total = (uint64_t)R * NQ * 16 * W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t w = (uint32_t)(i % W);
        const uint64_t rest = i / W;
        const uint32_t v = (uint32_t)(rest % 16);
        const uint64_t rj = rest / 16;
        const uint32_t j = (uint32_t)(rj % NQ), r = (uint32_t)(rj / NQ);
        uint32_t o = 0;
        for (uint32_t t = 0; t < 4; ++t) {
            const uint32_t b = 4 * j + t;
            if (((v >> t) & 1u) && b < B) o |= docbits[((uint64_t)r * B + b) * W + w];
        }
        ntab[i] = o;
    }
}

// Byte table: tab[((r*NJ + j)*256 + v)*W + w] = OR over set bits i of v
// (8j+i < B) of DocBits[r][8j+i][w].
__global__ void k_build_bytetab(const uint32_t *docbits, uint32_t B, uint32_t R, uint32_t W,
                                uint32_t *tab) {
    const uint32_t NJ = (B + 7) / 8;
    const uint64_t total = (uint64_t)R * NJ * 256 * W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t w = (uint32_t)(i % W);
        const uint64_t rest = i / W;
        const uint32_t v = (uint32_t)(rest % 256);
        const uint64_t rj = rest / 256;
        const uint32_t j = (uint32_t)(rj % NJ), r = (uint32_t)(rj / NJ);
        uint32_t o = 0;
        for (uint32_t t = 0; t < 8; ++t) {
            const uint32_t b = 8 * j + t;
            if (((v >> t) & 1u) && b < B) o |= docbits[((uint64_t)r * B + b) * W + w];
        }
        tab[i] = o;
    }
}

// Grid of the table-staging expansions: one resident wave at most, and no
// more blocks than give each about 512 queries (every block stages the whole
// table, so small batches would otherwise spend their time staging).
int nib_grid(int occ, int sm_count, int max_blocks, uint64_t n) {
    uint64_t g = (uint64_t)(occ > 0 ? occ : 1) * (uint64_t)sm_count;
    if (g > (uint64_t)max_blocks) g = (uint64_t)max_blocks;
    const uint64_t by_n = (n + 511) / 512;
    if (g > by_n) g = by_n;
    return g > 0 ? (int)g : 1;
}

}  // namespace

cudaError_t launch_expand(const ExpandArgs &a, int max_blocks, int sm_count, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    const uint32_t wc = (a.W + 31) / 32;
    const int C = wc >= 8 ? 8 : wc >= 4 ? 4 : wc >= 2 ? 2 : 1;
    const uint64_t units = a.n * ((a.W + 32 * C - 1) / (32 * C));
    uint64_t blocks = (units + EXPAND_THREADS / 32 - 1) / (EXPAND_THREADS / 32);
    const uint64_t cap = (uint64_t)max_blocks;
    if (blocks > cap) blocks = cap;
    // candidate filtering: repetition-0 nibble rows, the per-warp mask slots
    // and phi as bytes in shared memory
    const size_t filt_bytes = (size_t)((a.B + 3) / 4) * 16 * a.W * 4 + EXPAND_THREADS * 4 +
                              ((size_t)a.K * a.R + 3) / 4 * 4;
    if (a.filter && a.ntab && a.phi && a.Gw <= 32 && a.W <= 64 && a.B <= 256 &&
        filt_bytes <= SMEM_NIBTAB_MAX && a.n >= (uint64_t)max_blocks * 64) {
        cudaError_t e2 = cudaSuccess;
        if (filt_bytes > 48 * 1024)
            e2 = a.W > 32 ? cudaFuncSetAttribute(k_expand_filter<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filt_bytes)
                          : cudaFuncSetAttribute(k_expand_filter<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filt_bytes);
        if (e2 != cudaSuccess) return e2;
        if (a.W > 32) k_expand_filter<2><<<(unsigned)max_blocks, EXPAND_THREADS, filt_bytes, s>>>(a);
        else k_expand_filter<1><<<(unsigned)max_blocks, EXPAND_THREADS, filt_bytes, s>>>(a);
        return cudaGetLastError();
    }
    // nibble table in shared memory (small K), B a multiple of 32: rows at a
    // power-of-two stride, one 16-byte slice per lane
    const uint32_t rw = (a.W + 3) / 4;
    uint32_t rwp = 1;
    while (rwp < rw) rwp <<= 1;
    const size_t nib32_bytes = (size_t)a.R * (a.B / 4) * 16 * rwp * 16;
    if (a.ntab && a.B % 32 == 0 && rwp <= 32 && nib32_bytes <= SMEM_NIBTAB_MAX &&
        a.n >= (uint64_t)sm_count * 64) {
        cudaError_t e2 = cudaSuccess;
#define RGPU_NIB32(P)                                                                              \
    if (rwp == P) {                                                                                \
        if (nib32_bytes > 48 * 1024)                                                               \
            e2 = cudaFuncSetAttribute(k_expand_nib32<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      (int)nib32_bytes);                                           \
        int occ = 1;                                                                               \
        if (e2 == cudaSuccess)                                                                     \
            e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_expand_nib32<P>,            \
                                                               EXPAND_THREADS, nib32_bytes);       \
        const int grid = nib_grid(occ, sm_count, max_blocks, a.n);                                  \
        if (e2 == cudaSuccess)                                                                     \
            k_expand_nib32<P><<<grid, EXPAND_THREADS, nib32_bytes, s>>>(a);                         \
    }
        RGPU_NIB32(1)
        RGPU_NIB32(2)
        RGPU_NIB32(4)
        RGPU_NIB32(8)
        RGPU_NIB32(16)
        RGPU_NIB32(32)
#undef RGPU_NIB32
        if (e2 != cudaSuccess) return e2;
        return cudaGetLastError();
    }
    // nibble table in shared memory (small K): several queries per warp
    const size_t nib_bytes = (size_t)a.R * ((a.B + 3) / 4) * 16 * rw * 16;
    if (a.ntab && rw <= 32 && nib_bytes <= SMEM_NIBTAB_MAX && a.n >= (uint64_t)sm_count * 64) {
        // rw <= 32 slices -> at most 32 lanes of one slice
        // one 16-byte slice per lane when a row spans 8+ slices: an 8-lane
        // shared-memory phase then reads 128 contiguous bytes of one query's
        // row (no bank conflicts); narrower rows pack two slices per lane
        const int vpl = (rw >= 8 || rw < 2) ? 1 : 2;
        const uint32_t slices = (rw + vpl - 1) / vpl;
        const int lpq = slices <= 1 ? 1 : slices <= 2 ? 2 : slices <= 4 ? 4 : slices <= 8 ? 8 : slices <= 16 ? 16 : 32;
        cudaError_t e2 = cudaSuccess;
        // one resident wave (every block stages the table once)
#define RGPU_NIB(L, V)                                                                             \
    if (lpq == L && vpl == V) {                                                                    \
        if (nib_bytes > 48 * 1024)                                                                 \
            e2 = cudaFuncSetAttribute(k_expand_nib<L, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      (int)nib_bytes);                                             \
        int occ = 1;                                                                               \
        if (e2 == cudaSuccess)                                                                     \
            e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_expand_nib<L, V>,           \
                                                               EXPAND_THREADS, nib_bytes);         \
        const int grid = nib_grid(occ, sm_count, max_blocks, a.n);                                  \
        if (e2 == cudaSuccess) k_expand_nib<L, V><<<grid, EXPAND_THREADS, nib_bytes, s>>>(a);       \
    }
        RGPU_NIB(1, 1)
        RGPU_NIB(1, 2)
        RGPU_NIB(2, 2)
        RGPU_NIB(4, 2)
        RGPU_NIB(8, 1)
        RGPU_NIB(16, 1)
        RGPU_NIB(32, 1)
#undef RGPU_NIB
        if (e2 != cudaSuccess) return e2;
        return cudaGetLastError();
    }
    // DocBits in shared memory when it fits and every block gets enough
    // queries to pay for staging it
    const size_t db_bytes = (size_t)a.R * a.B * a.W * 4;
    const bool smem = a.smem_docbits && db_bytes <= SMEM_DOCBITS_MAX && units >= blocks * 64;
    const size_t dyn = smem ? db_bytes : 0;
    cudaError_t e = cudaSuccess;
#define RGPU_EXPAND(CC)                                                                            \
    if (smem) {                                                                                    \
        if (dyn > 48 * 1024)                                                                       \
            e = cudaFuncSetAttribute(k_expand<CC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)dyn);                                                    \
        if (e == cudaSuccess) k_expand<CC, true><<<(unsigned)blocks, EXPAND_THREADS, dyn, s>>>(a); \
    } else {                                                                                       \
        k_expand<CC, false><<<(unsigned)blocks, EXPAND_THREADS, 0, s>>>(a);                       \
    }
    switch (C) {
        case 1: RGPU_EXPAND(1) break;
        case 2: RGPU_EXPAND(2) break;
        case 4: RGPU_EXPAND(4) break;
        default: RGPU_EXPAND(8) break;
    }
#undef RGPU_EXPAND
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

uint64_t nibtab_words(uint32_t B, uint32_t R, uint32_t W) {
    return (uint64_t)R * ((B + 3) / 4) * 16 * W;
}

cudaError_t launch_build_nibtab(const uint32_t *docbits, uint32_t B, uint32_t R, uint32_t W,
                                uint32_t *ntab, int sm_count, cudaStream_t s) {
    k_build_nibtab<<<sm_count * 4, 256, 0, s>>>(docbits, B, R, W, ntab);
    return cudaGetLastError();
}

uint64_t bytetab_words(uint32_t B, uint32_t R, uint32_t W) {
    return (uint64_t)R * ((B + 7) / 8) * 256 * W;
}

cudaError_t launch_build_bytetab(const uint32_t *docbits, uint32_t B, uint32_t R, uint32_t W,
                                 uint32_t *tab, int sm_count, cudaStream_t s) {
    k_build_bytetab<<<sm_count * 8, 256, 0, s>>>(docbits, B, R, W, tab);
    return cudaGetLastError();
}

}  // namespace rgpu

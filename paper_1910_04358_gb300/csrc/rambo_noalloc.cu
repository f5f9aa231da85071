// rambo_noalloc.cu -- the sequence query for callers that cannot allocate
// device memory.
//
// rambo_query_seqs_dev needs a caller-provided workspace, and the host-buffer
// calls grow one inside the library with cudaMalloc.  Some callers can do
// neither: hosts that own every device byte themselves and forbid libraries
// to allocate (plugin and embedded runtimes with a fixed memory budget), and
// latency-critical threads that must never reach cudaMalloc/cudaFree, which
// can block on or synchronise the whole device.  For them this file keeps the
// query's scratch in one file-scope device array of a fixed size that the
// CUDA runtime places on every GPU that loads the library and keeps there
// until the process exits.  The caller still passes the inputs and the
// output; nothing is allocated per call.
#include <cuda_runtime.h>

#include <mutex>

#include "rambo.h"

namespace {

// The scratch itself.  In host code `g_scratch` only names a host-side
// stand-in: handing that address to a kernel would fault or, where the GPU
// can reach host memory, silently use the wrong memory.  The device address
// is looked up with cudaGetSymbolAddress once per device (below).
static __device__ __align__(256) unsigned char g_scratch[RAMBO_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_on_device[kMaxDevices];  // device address of g_scratch, per device

// Looks up (once per device, with that device current) the device address of
// the scratch array.  The address is kept until the process exits; a
// cudaDeviceReset of the device would make it stale, which is why the entry
// point must not be used after one (the header says so).
int scratch_address(int device, void **out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_on_device[device]) {
        int prev = -1;
        if (cudaGetDevice(&prev) != cudaSuccess) return RAMBO_ECUDA;
        if (prev != device && cudaSetDevice(device) != cudaSuccess) return RAMBO_ECUDA;
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (prev != device) cudaSetDevice(prev);
        if (e != cudaSuccess || p == nullptr) return RAMBO_ECUDA;
        g_scratch_on_device[device] = p;
    }
    *out = g_scratch_on_device[device];
    return RAMBO_OK;
}

}  // namespace

extern "C" int rambo_query_seqs_noalloc(rambo_t *h, uint64_t n, const uint8_t *packed,
                                        uint64_t packed_bytes, const uint64_t *base_offsets,
                                        uint32_t *out, void *stream) {
    if (!h) return RAMBO_EINVAL;
    if (n == 0) return RAMBO_OK;
    // the batch must fit the fixed scratch: k-mer prefix, scan block sums and
    // one bucket mask per query
    const size_t need = rambo_query_seqs_workspace(h, n);
    if (need == 0 || need > (size_t)RAMBO_STATIC_SCRATCH_BYTES) return RAMBO_EINVAL;
    rambo_info_t info;
    const int rc = rambo_get_info(h, &info);
    if (rc != RAMBO_OK) return rc;
    if (info.device < 0 || info.device >= kMaxDevices) return RAMBO_EINVAL;
    void *scratch = nullptr;
    const int rs = scratch_address(info.device, &scratch);
    if (rs != RAMBO_OK) return rs;
    // the query clears what must start fresh (it sets every bucket mask to
    // all ones and rewrites the whole prefix) before using the scratch
    return rambo_query_seqs_dev(h, n, packed, packed_bytes, base_offsets, out, scratch,
                                (size_t)RAMBO_STATIC_SCRATCH_BYTES, stream);
}

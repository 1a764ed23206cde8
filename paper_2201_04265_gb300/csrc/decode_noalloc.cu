// ldpc_decode_noalloc: decoding for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc (or any allocator) at
// decode time: a real-time receive thread of a software radio that must not
// block on an allocation that may synchronise the device, or a host framework
// that owns every device buffer and gives the decoder none to spare.  For
// them this entry point runs the plain decoding schedule (the same kernels as
// ldpc_decode with LDPC_SCHED_PLAIN) with its scratch taken from one static
// device array defined in this file, of LDPC_NOALLOC_SCRATCH_BYTES.  Every
// GPU that loads the library holds that array until the process exits.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress and keeps it; make that
// first call before any stream capture.  All calls share the one array and it
// keeps the previous call's contents; the decoder rewrites or clears every
// part it reads (the iteration flags are cleared on the stream at the start
// of each call), so nothing carries over between calls.  Calls whose work
// overlaps on the GPU (other streams, other host threads) race on the array:
// serialise them.
#include <mutex>

#include "ldpc_internal.h"

namespace ldpc {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[LDPC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the static array on the current device (set up once).
int scratch_address(void **out) {
    int dev = -1;
    LDPC_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(LDPC_ENOTSUP, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess) return cuda_fail(err, "cudaGetSymbolAddress(static decode scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LDPC_OK;
}

}  // namespace
}  // namespace ldpc

using namespace ldpc;

extern "C" int ldpc_decode_noalloc(const ldpc_code *c, const float *d_llr, int32_t F,
                                   const ldpc_decode_opts *o, float *d_post, uint32_t *d_hard,
                                   int32_t *d_iters, uint8_t *d_ok, ldpc_stream_t stream) {
    TraceRange trace_("ldpc_decode_noalloc");
    if (!c) return fail(LDPC_EINVAL, "code is NULL");
    if (!c->on_device) return fail(LDPC_EINVAL, "code was created host-only");
    if (!o) return fail(LDPC_EINVAL, "opts is NULL");
    if (o->schedule != LDPC_SCHED_AUTO && o->schedule != LDPC_SCHED_PLAIN)
        return fail(LDPC_EINVAL, "ldpc_decode_noalloc runs the plain schedule only");
    ldpc_decode_opts plain = *o;
    plain.schedule = LDPC_SCHED_PLAIN;
    size_t need = 0;
    LDPC_TRY(ldpc_decode_workspace_size(c, F, &plain, &need));
    if (need > (size_t)LDPC_NOALLOC_SCRATCH_BYTES)
        return fail(LDPC_EINVAL,
                    "ldpc_decode_noalloc: %d frames of this code need %zu bytes of scratch, more than "
                    "the static array's %u bytes; decode fewer frames per call",
                    F, need, (unsigned)LDPC_NOALLOC_SCRATCH_BYTES);
    void *scratch = nullptr;
    LDPC_TRY(scratch_address(&scratch));
    return ldpc_decode(c, d_llr, F, &plain, d_post, d_hard, d_iters, d_ok, scratch,
                       (size_t)LDPC_NOALLOC_SCRATCH_BYTES, stream);
}

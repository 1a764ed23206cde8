// Entry points of the C ABI that launch work: argument checks and dispatch.
#include "ldpc_internal.h"

#include <map>
#include <mutex>
#include <tuple>

namespace ldpc {

int kernel_setup(const void *fn, int threads, size_t smem, int *per_sm) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int, size_t>, int> cache;  // (fn, dev, threads, smem)
    static std::map<std::pair<const void *, int>, size_t> smem_set;          // (fn, dev) -> limit
    int dev = -1;
    LDPC_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(fn, dev, threads, smem);
    auto it = cache.find(key);
    if (it != cache.end()) {
        if (per_sm) *per_sm = it->second;
        return LDPC_OK;
    }
    size_t &lim = smem_set[std::make_pair(fn, dev)];
    if (smem > lim) {  // (static shared memory counts against the default 48 KB too)
        LDPC_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        lim = smem;
    }
    int n = 0;
    LDPC_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem));
    cache[key] = n;
    if (per_sm) *per_sm = n;
    return LDPC_OK;
}

int sm_count(int *sms) {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = -1;
    LDPC_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(dev);
    if (it == cache.end()) {
        int n = 0;
        LDPC_TRY_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        it = cache.emplace(dev, n).first;
    }
    *sms = it->second;
    return LDPC_OK;
}

int decode_resident(const ldpc_code *c, const float *d_llr, int32_t F, const ldpc_decode_opts *o,
                    float *d_post, uint32_t *d_hard, int32_t *d_iters, uint8_t *d_ok, void *d_work,
                    size_t work_bytes, cudaStream_t s);
size_t resident_workspace(const ldpc_code *c, int32_t F, const ldpc_decode_opts *o);
bool resident_fits(const ldpc_code *c, const ldpc_decode_opts *o);

namespace {

int check_code(const ldpc_code *c) {
    if (!c) return fail(LDPC_EINVAL, "code is NULL");
    if (!c->on_device) return fail(LDPC_EINVAL, "code was created host-only");
    int dev = -1;
    LDPC_TRY_CUDA(cudaGetDevice(&dev));
    if (dev != c->device)
        return fail(LDPC_EINVAL, "code lives on device %d but device %d is current", c->device, dev);
    return LDPC_OK;
}

int check_opts(const ldpc_decode_opts *o) {
    if (!o) return fail(LDPC_EINVAL, "opts is NULL");
    if (o->max_iters < 0) return fail(LDPC_EINVAL, "max_iters < 0");
    if (!(o->clip > 0.f) || o->clip > 1e30f) return fail(LDPC_EINVAL, "clip must be positive and finite");
    if (o->early_stop != 0 && o->early_stop != 1) return fail(LDPC_EINVAL, "early_stop must be 0 or 1");
    if (o->msg_fp16 != 0 && o->msg_fp16 != 1) return fail(LDPC_EINVAL, "msg_fp16 must be 0 or 1");
    if (o->schedule < LDPC_SCHED_AUTO || o->schedule > LDPC_SCHED_CLUSTER)
        return fail(LDPC_EINVAL, "unknown schedule %d", o->schedule);
    return LDPC_OK;
}

int pick_schedule(const ldpc_code *c, const ldpc_decode_opts *o) {
    if (o->schedule != LDPC_SCHED_AUTO) return o->schedule;
    if (resident_fits(c, o)) return LDPC_SCHED_RESIDENT;
    return cluster_fits(c, o) ? LDPC_SCHED_CLUSTER : LDPC_SCHED_PLAIN;
}

}  // namespace
}  // namespace ldpc

using namespace ldpc;

extern "C" {

int ldpc_encode(const ldpc_code *c, const uint32_t *d_info, uint32_t *d_code, int32_t F,
                ldpc_stream_t stream) {
    TraceRange trace_("ldpc_encode");
    LDPC_TRY(check_code(c));
    if (F < 0) return fail(LDPC_EINVAL, "F < 0");
    if (F == 0) return LDPC_OK;
    if (!d_info || !d_code) return fail(LDPC_EINVAL, "d_info/d_code is NULL");
    return launch_encode(c, d_info, d_code, F, (cudaStream_t)stream);
}

int ldpc_encode_tables_build(ldpc_code *c, size_t *bytes) {
    LDPC_TRY(check_code(c));
    return build_encode_tables(c, bytes);
}

int ldpc_encode_tables_free(ldpc_code *c) {
    LDPC_TRY(check_code(c));
    free_encode_tables(c);
    return LDPC_OK;
}

int ldpc_syndrome(const ldpc_code *c, const uint32_t *d_bits, int32_t F, uint32_t *d_syn,
                  uint8_t *d_ok, ldpc_stream_t stream) {
    TraceRange trace_("ldpc_syndrome");
    LDPC_TRY(check_code(c));
    if (F < 0) return fail(LDPC_EINVAL, "F < 0");
    if (F == 0 || (!d_syn && !d_ok)) return LDPC_OK;
    if (!d_bits) return fail(LDPC_EINVAL, "d_bits is NULL");
    return launch_syndrome(c, d_bits, F, d_syn, d_ok, (cudaStream_t)stream);
}

int ldpc_decode_workspace_size(const ldpc_code *c, int32_t F, const ldpc_decode_opts *o,
                               size_t *bytes) {
    if (!c || !bytes) return fail(LDPC_EINVAL, "code or bytes is NULL");
    LDPC_TRY(check_opts(o));
    if (F < 0) return fail(LDPC_EINVAL, "F < 0");
    const int sched = pick_schedule(c, o);
    *bytes = sched == LDPC_SCHED_RESIDENT  ? resident_workspace(c, F, o)
             : sched == LDPC_SCHED_CLUSTER ? (size_t)256
                                           : plain_workspace(c, F, o);
    return LDPC_OK;
}

int ldpc_decode(const ldpc_code *c, const float *d_llr, int32_t F, const ldpc_decode_opts *o,
                float *d_post, uint32_t *d_hard, int32_t *d_iters, uint8_t *d_ok, void *d_work,
                size_t work_bytes, ldpc_stream_t stream) {
    TraceRange trace_("ldpc_decode");
    LDPC_TRY(check_code(c));
    LDPC_TRY(check_opts(o));
    if (F < 0) return fail(LDPC_EINVAL, "F < 0");
    if (F == 0) return LDPC_OK;
    if (!d_llr) return fail(LDPC_EINVAL, "d_llr is NULL");
    if (d_work && (reinterpret_cast<uintptr_t>(d_work) & 255u))
        return fail(LDPC_EINVAL, "d_work must be 256-byte aligned");
    const int sched = pick_schedule(c, o);
    if (sched == LDPC_SCHED_RESIDENT) {
        if (!resident_fits(c, o))
            return fail(LDPC_ENOTSUP, "this code does not fit the resident decoder");
        return decode_resident(c, d_llr, F, o, d_post, d_hard, d_iters, d_ok, d_work, work_bytes,
                               (cudaStream_t)stream);
    }
    if (sched == LDPC_SCHED_CLUSTER) {
        if (!cluster_fits(c, o))
            return fail(LDPC_ENOTSUP, "this code has no cluster layout (quasi-cyclic codes created from "
                                      "their base matrix only)");
        return decode_cluster(c, d_llr, F, o, d_post, d_hard, d_iters, d_ok, d_work, work_bytes,
                              (cudaStream_t)stream);
    }
    return decode_plain(c, d_llr, F, o, d_post, d_hard, d_iters, d_ok, d_work, work_bytes,
                        (cudaStream_t)stream);
}

}  // extern "C"

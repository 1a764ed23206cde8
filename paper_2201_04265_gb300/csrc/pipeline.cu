// Decoding from host memory with copies overlapped with decoding.
//
// The batch is cut into chunks; chunk i's channel LLRs are copied to the
// device on an upload stream while chunk i-1 is decoded on the caller's
// stream, and each chunk's results are copied back on a download stream as
// soon as it is decoded.  Three device staging buffers rotate, so an upload
// may run up to two chunks ahead of the decoder and a copy slowed down by
// other traffic on the host link is absorbed; events order every reuse, and
// uploads and downloads use separate streams so that an upload never queues
// behind the previous chunk's download.  This is the host
// side of the paper's batch processing (Sec. III-C) on one GPU: frames are
// independent, so chunks are too.
#include <map>
#include <mutex>
#include <vector>

#include "ldpc_internal.h"

namespace ldpc {
namespace {

constexpr int kStage = 3;  // staging buffers

struct CopyRes {
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t h2d[kStage] = {}, dec[kStage] = {}, d2h[kStage] = {};
};

// Two copy streams and 3 kStage events per device, created on first use.
int copy_resources(CopyRes **out) {
    static std::mutex mu;
    static std::map<int, CopyRes> res;
    int dev = -1;
    LDPC_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto it = res.find(dev);
    if (it == res.end()) {
        CopyRes r;
        LDPC_TRY_CUDA(cudaStreamCreateWithFlags(&r.up, cudaStreamNonBlocking));
        LDPC_TRY_CUDA(cudaStreamCreateWithFlags(&r.down, cudaStreamNonBlocking));
        for (int b = 0; b < kStage; ++b) {
            LDPC_TRY_CUDA(cudaEventCreateWithFlags(&r.h2d[b], cudaEventDisableTiming));
            LDPC_TRY_CUDA(cudaEventCreateWithFlags(&r.dec[b], cudaEventDisableTiming));
            LDPC_TRY_CUDA(cudaEventCreateWithFlags(&r.d2h[b], cudaEventDisableTiming));
        }
        it = res.emplace(dev, r).first;
    }
    *out = &it->second;
    return LDPC_OK;
}

struct PipeWs {
    float *llr[kStage];
    float *post[kStage];
    uint32_t *hard[kStage];
    int32_t *iters[kStage];
    uint8_t *ok[kStage];
    void *dec;
    size_t dec_bytes;
};

size_t pipe_layout(const ldpc_code *c, int32_t chunk, const ldpc_decode_opts *o, PipeWs *w, void *base) {
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t at = off;
        off += align256(b);
        return at;
    };
    size_t oL[kStage], oP[kStage], oH[kStage], oI[kStage], oK[kStage];
    for (int b = 0; b < kStage; ++b) {
        oL[b] = take(sizeof(float) * (size_t)chunk * c->n);
        oP[b] = take(sizeof(float) * (size_t)chunk * c->n);
        oH[b] = take(sizeof(uint32_t) * (size_t)chunk * c->NW);
        oI[b] = take(sizeof(int32_t) * (size_t)chunk);
        oK[b] = take((size_t)chunk);
    }
    size_t dec = 0;
    ldpc_decode_workspace_size(c, chunk, o, &dec);
    const size_t oD = take(dec);
    if (w && base) {
        char *p = static_cast<char *>(base);
        for (int b = 0; b < kStage; ++b) {
            w->llr[b] = reinterpret_cast<float *>(p + oL[b]);
            w->post[b] = reinterpret_cast<float *>(p + oP[b]);
            w->hard[b] = reinterpret_cast<uint32_t *>(p + oH[b]);
            w->iters[b] = reinterpret_cast<int32_t *>(p + oI[b]);
            w->ok[b] = reinterpret_cast<uint8_t *>(p + oK[b]);
        }
        w->dec = p + oD;
        w->dec_bytes = dec;
    }
    return off;
}

}  // namespace
}  // namespace ldpc

using namespace ldpc;

extern "C" {

int ldpc_decode_host_workspace_size(const ldpc_code *c, int32_t chunk, const ldpc_decode_opts *o,
                                    size_t *bytes) {
    if (!c || !o || !bytes || chunk < 1) return fail(LDPC_EINVAL, "bad arguments");
    *bytes = pipe_layout(c, chunk, o, nullptr, nullptr);
    return LDPC_OK;
}

}  // extern "C"

namespace ldpc {
namespace {

// Timing events of one chunk (timeline mode): upload, decode and download,
// each bracketed on the stream that runs it.
struct ChunkMarks {
    cudaEvent_t ev[6] = {};
};

// The pipeline; with `marks` (one entry per chunk, events created by the
// caller), each chunk's upload, decode and download are bracketed by events.
int host_pipeline(const ldpc_code *c, const float *h_llr, int32_t F, const ldpc_decode_opts *o,
                  float *h_post, uint32_t *h_hard, int32_t *h_iters, uint8_t *h_ok, int32_t chunk,
                  void *d_work, size_t work_bytes, ldpc_stream_t stream, ChunkMarks *marks) {
    if (!c || !o) return fail(LDPC_EINVAL, "code or opts is NULL");
    if (F < 0 || chunk < 1) return fail(LDPC_EINVAL, "F < 0 or chunk < 1");
    if (F == 0) return LDPC_OK;
    if (!h_llr) return fail(LDPC_EINVAL, "h_llr is NULL");
    PipeWs w{};
    const size_t need = pipe_layout(c, chunk, o, &w, d_work);
    if (!d_work || work_bytes < need) return fail(LDPC_EINVAL, "workspace too small (%zu < %zu)", work_bytes, need);
    CopyRes *r = nullptr;
    LDPC_TRY(copy_resources(&r));
    cudaStream_t s = (cudaStream_t)stream;
    // the copy streams start after everything already queued on the caller's stream
    LDPC_TRY_CUDA(cudaEventRecord(r->dec[0], s));
    LDPC_TRY_CUDA(cudaStreamWaitEvent(r->up, r->dec[0], 0));
    LDPC_TRY_CUDA(cudaStreamWaitEvent(r->down, r->dec[0], 0));
    const int64_t nchunks = ceil_div(F, chunk);
    bool used[kStage] = {};
    for (int64_t ci = 0; ci < nchunks; ++ci) {
        const int b = (int)(ci % kStage);
        const int64_t f0 = ci * chunk;
        const int32_t fc = (int32_t)std::min<int64_t>(chunk, F - f0);
        // staging buffer b is free once chunk ci - kStage's results are copied out
        if (used[b]) LDPC_TRY_CUDA(cudaStreamWaitEvent(r->up, r->d2h[b], 0));
        if (marks) LDPC_TRY_CUDA(cudaEventRecord(marks[ci].ev[0], r->up));
        LDPC_TRY_CUDA(cudaMemcpyAsync(w.llr[b], h_llr + f0 * c->n, sizeof(float) * (size_t)fc * c->n,
                                      cudaMemcpyHostToDevice, r->up));
        if (marks) LDPC_TRY_CUDA(cudaEventRecord(marks[ci].ev[1], r->up));
        LDPC_TRY_CUDA(cudaEventRecord(r->h2d[b], r->up));
        LDPC_TRY_CUDA(cudaStreamWaitEvent(s, r->h2d[b], 0));
        if (marks) LDPC_TRY_CUDA(cudaEventRecord(marks[ci].ev[2], s));
        LDPC_TRY(ldpc_decode(c, w.llr[b], fc, o, h_post ? w.post[b] : nullptr, w.hard[b], w.iters[b], w.ok[b],
                             w.dec, w.dec_bytes, stream));
        if (marks) LDPC_TRY_CUDA(cudaEventRecord(marks[ci].ev[3], s));
        LDPC_TRY_CUDA(cudaEventRecord(r->dec[b], s));
        LDPC_TRY_CUDA(cudaStreamWaitEvent(r->down, r->dec[b], 0));
        if (marks) LDPC_TRY_CUDA(cudaEventRecord(marks[ci].ev[4], r->down));
        if (h_post)
            LDPC_TRY_CUDA(cudaMemcpyAsync(h_post + f0 * c->n, w.post[b], sizeof(float) * (size_t)fc * c->n,
                                          cudaMemcpyDeviceToHost, r->down));
        if (h_hard)
            LDPC_TRY_CUDA(cudaMemcpyAsync(h_hard + f0 * c->NW, w.hard[b], sizeof(uint32_t) * (size_t)fc * c->NW,
                                          cudaMemcpyDeviceToHost, r->down));
        if (h_iters)
            LDPC_TRY_CUDA(cudaMemcpyAsync(h_iters + f0, w.iters[b], sizeof(int32_t) * (size_t)fc,
                                          cudaMemcpyDeviceToHost, r->down));
        if (h_ok)
            LDPC_TRY_CUDA(cudaMemcpyAsync(h_ok + f0, w.ok[b], (size_t)fc, cudaMemcpyDeviceToHost, r->down));
        if (marks) LDPC_TRY_CUDA(cudaEventRecord(marks[ci].ev[5], r->down));
        LDPC_TRY_CUDA(cudaEventRecord(r->d2h[b], r->down));
        used[b] = true;
    }
    // the caller's stream completes only after the last results reach the host
    LDPC_TRY_CUDA(cudaStreamWaitEvent(s, r->d2h[(nchunks - 1) % kStage], 0));
    return LDPC_OK;
}

}  // namespace
}  // namespace ldpc

extern "C" {

int ldpc_decode_host(const ldpc_code *c, const float *h_llr, int32_t F, const ldpc_decode_opts *o,
                     float *h_post, uint32_t *h_hard, int32_t *h_iters, uint8_t *h_ok, int32_t chunk,
                     void *d_work, size_t work_bytes, ldpc_stream_t stream) {
    TraceRange trace_("ldpc_decode_host");
    return host_pipeline(c, h_llr, F, o, h_post, h_hard, h_iters, h_ok, chunk, d_work, work_bytes, stream,
                         nullptr);
}

int ldpc_decode_host_timeline(const ldpc_code *c, const float *h_llr, int32_t F, const ldpc_decode_opts *o,
                              float *h_post, uint32_t *h_hard, int32_t *h_iters, uint8_t *h_ok, int32_t chunk,
                              void *d_work, size_t work_bytes, ldpc_stream_t stream, float *h_ms) {
    TraceRange trace_("ldpc_decode_host_timeline");
    if (!h_ms) return fail(LDPC_EINVAL, "h_ms is NULL");
    if (F <= 0 || chunk < 1) return fail(LDPC_EINVAL, "need F >= 1 and chunk >= 1");
    const int64_t nchunks = ceil_div(F, chunk);
    std::vector<ChunkMarks> marks((size_t)nchunks);
    cudaEvent_t t0 = nullptr;
    int st = LDPC_OK;
    cudaError_t e = cudaEventCreate(&t0);
    for (int64_t i = 0; i < nchunks && e == cudaSuccess; ++i)
        for (int k = 0; k < 6 && e == cudaSuccess; ++k) e = cudaEventCreate(&marks[i].ev[k]);
    if (e == cudaSuccess) e = cudaEventRecord(t0, (cudaStream_t)stream);
    if (e != cudaSuccess) st = cuda_fail(e, "timeline events");
    if (st == LDPC_OK)
        st = host_pipeline(c, h_llr, F, o, h_post, h_hard, h_iters, h_ok, chunk, d_work, work_bytes, stream,
                           marks.data());
    if (st == LDPC_OK) {
        e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize(timeline)");
    }
    for (int64_t i = 0; i < nchunks && st == LDPC_OK; ++i)
        for (int k = 0; k < 6 && st == LDPC_OK; ++k) {
            e = cudaEventElapsedTime(&h_ms[i * 6 + k], t0, marks[i].ev[k]);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaEventElapsedTime(timeline)");
        }
    for (auto &m : marks)
        for (cudaEvent_t ev : m.ev)
            if (ev) cudaEventDestroy(ev);
    if (t0) cudaEventDestroy(t0);
    return st;
}

}  // extern "C"

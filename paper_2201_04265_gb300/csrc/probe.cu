// Measured throughput of the three transcendental instructions the decoders
// issue per edge (ex2.approx, rcp.approx, lg2.approx), in results per SM per
// clock.  Not part of the method: it gives the ALU roofline of the resident
// decoder a measured denominator on the GPU it runs on.
//
// One CTA of 1024 threads per SM; every thread runs 8 independent chains of
// the instruction for N rounds (the rcp chain adds a constant between steps,
// so that no pair of reciprocals cancels).  Each CTA times its loop with the
// SM clock; the rate is taken from the fastest CTA, so a CTA that shared its
// SM can only lower the reported rate's denominator, never raise it.
#include "ldpc_internal.h"

namespace ldpc {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeChains = 8;
constexpr int kProbeRounds = 2048;

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) xu_probe(float *sink, long long *cycles) {
    float x[kProbeChains];
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) x[j] = 0.5f + 0.01f * j + 1e-6f * threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < kProbeRounds; ++it) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) {
            float y;
            if (OP == 0) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x[j]));
            if (OP == 1) {
                asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[j]));
                y += 0.75f;
            }
            if (OP == 2) asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[j]));
            x[j] = y;
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) s += x[j];
    sink[blockIdx.x * kProbeThreads + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace ldpc

using namespace ldpc;

extern "C" int ldpc_probe_xu_rates(float *rates) {
    if (!rates) return fail(LDPC_EINVAL, "rates is NULL");
    int sms = 0;
    LDPC_TRY(sm_count(&sms));
    float *sink = nullptr;
    long long *cyc = nullptr;
    int st = LDPC_OK;
    cudaError_t e = cudaMalloc((void **)&sink, sizeof(float) * (size_t)sms * kProbeThreads);
    if (e == cudaSuccess) e = cudaMalloc((void **)&cyc, sizeof(long long) * (size_t)sms);
    std::vector<long long> h((size_t)sms);
    for (int op = 0; op < 3 && e == cudaSuccess; ++op) {
        if (op == 0) xu_probe<0><<<sms, kProbeThreads>>>(sink, cyc);
        if (op == 1) xu_probe<1><<<sms, kProbeThreads>>>(sink, cyc);
        if (op == 2) xu_probe<2><<<sms, kProbeThreads>>>(sink, cyc);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        long long best = h[0];
        for (long long c : h) best = c < best ? c : best;
        rates[op] = best > 0 ? (float)((double)kProbeThreads * kProbeChains * kProbeRounds / (double)best) : 0.f;
    }
    if (e != cudaSuccess) st = cuda_fail(e, "ldpc_probe_xu_rates");
    if (sink) cudaFree(sink);
    if (cyc) cudaFree(cyc);
    return st;
}

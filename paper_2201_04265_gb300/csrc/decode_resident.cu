// K5: persistent decoder with whole frames resident in shared memory.
//
// The same flooding sum-product iteration as the plain decoder (Sec. II-B,
// Eqs. 5-8, Algorithm 1's schedule) and the same arithmetic (check_math.cuh),
// but every message of a frame stays on chip for all iterations: HBM is read
// once (the channel LLRs) and written once (outputs) per frame.  This is the
// paper's batch processing (Sec. III-C) mapped onto the GPU: each CTA takes
// frames from a global work counter and decodes them one group at a time.
//
// Per CTA, for a group of G frames (G = 2 with binary16 messages, 1 with FP32
// messages), shared memory holds
//   Ls[n]        total LLRs L_v of the G frames      (float2 / float)
//   Es[n * DV]   check messages E_cv, bit-major: the DV slots of bit v are
//                Es[v*DV .. v*DV+DV)                 (half2 / float)
// The G frames of a group share every index computation and every shared
// memory access (a 4- or 8-byte vector covers both frames).
//
// Thread t owns checks t, t+T, ..., and bits t, t+T, ... for the whole
// kernel: its checks' edge slots (16-bit positions in Es; bit index = slot /
// DV) are loaded once into registers from a table built at code creation, and
// its bits' channel LLRs R_v stay in registers while a group is decoded.
//
// Per iteration: check pass (each thread updates its checks' messages in
// place and, for early stop, evaluates the syndrome of the previous hard
// decisions), barrier, bit pass (L_v = R_v + sum of the bit's DV slots, in
// ascending edge order), barrier.
#include <algorithm>

#include "check_math.cuh"
#include "ldpc_internal.h"

namespace ldpc {
namespace {

constexpr int kResVPT = 16;       // bits per thread
constexpr int kResMaxThreads = 512;
constexpr int kResDV = 3;         // padded column degree (slots per bit)
constexpr uint32_t kNoSlot = 0xFFFFu;

// Row shapes: padded row degree and checks per thread (about 48 edges/thread).
struct Shape {
    int dc, cpt;
};
constexpr Shape kShapes[] = {{6, 8}, {9, 5}, {12, 4}, {16, 3}};

template <int G>
struct LVec;
template <>
struct LVec<1> {
    using T = float;
    __device__ static void get(T v, float *x) { x[0] = v; }
    __device__ static T make(const float *x) { return x[0]; }
};
template <>
struct LVec<2> {
    using T = float2;
    __device__ static void get(T v, float *x) {
        x[0] = v.x;
        x[1] = v.y;
    }
    __device__ static T make(const float *x) { return make_float2(x[0], x[1]); }
};

template <class MsgT, int G>
struct EVec;
template <>
struct EVec<__half, 2> {
    using T = __half2;
    __device__ static void get(T v, float *x) {
        const float2 f = __half22float2(v);
        x[0] = f.x;
        x[1] = f.y;
    }
    __device__ static T make(const float *x) { return __floats2half2_rn(x[0], x[1]); }
    __device__ static T zero() { return __floats2half2_rn(0.f, 0.f); }
};
template <>
struct EVec<float, 1> {
    using T = float;
    __device__ static void get(T v, float *x) { x[0] = v; }
    __device__ static T make(const float *x) { return x[0]; }
    __device__ static T zero() { return 0.f; }
};

struct ResArgs {
    const float *llr;
    int32_t F, n, m, NW, T_iters, early_stop, pad_slots;
    float clip2;
    const uint32_t *edges;  // [CPT * DCW][T]
    float *post;
    uint32_t *hard;
    int32_t *iters;
    uint8_t *ok;
    unsigned *counter;
};

// One check pass over the thread's checks.  COMPUTE = false evaluates only the
// syndrome.  Returns bit i set when a check of frame i is unsatisfied by the
// hard decisions z = [L >= 0] read in this pass.
template <class MsgT, int G, int DC, int CPT, bool COMPUTE>
__device__ __forceinline__ uint32_t check_pass(const uint32_t (&idx)[CPT][(DC + 1) / 2],
                                               typename LVec<G>::T *Ls,
                                               typename EVec<MsgT, G>::T *Es, bool first,
                                               float clip2) {
    using LV = LVec<G>;
    using EV = EVec<MsgT, G>;
    uint32_t bad = 0;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        if ((idx[k][0] & 0xFFFFu) == kNoSlot) continue;  // no check in this slot
        uint32_t slot[DC];
#pragma unroll
        for (int j = 0; j < DC; ++j) slot[j] = (idx[k][j >> 1] >> ((j & 1) * 16)) & 0xFFFFu;
        float u[DC][G];
        uint32_t smask[G], zpar[G];
        int d = 0;
#pragma unroll
        for (int i = 0; i < G; ++i) smask[i] = zpar[i] = 0;
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (slot[j] != kNoSlot) {
                ++d;
                float L[G], Eo[G];
                LV::get(Ls[slot[j] / kResDV], L);
                if (COMPUTE) {
                    if (first) {
#pragma unroll
                        for (int i = 0; i < G; ++i) Eo[i] = 0.f;
                    } else {
                        EV::get(Es[slot[j]], Eo);
                    }
                }
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    zpar[i] ^= (uint32_t)(L[i] >= 0.f);
                    if (COMPUTE) {
                        const float x = check_input(L[i], Eo[i], clip2);
                        smask[i] |= (__float_as_uint(x) >> 31) << j;
                        u[j][i] = check_u(x);
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < G; ++i) u[j][i] = 0.f;  // identity for the pair products
            }
        }
#pragma unroll
        for (int i = 0; i < G; ++i) bad |= zpar[i] << i;
        if (!COMPUTE) continue;
        EvOd pre[DC][G];
        uint32_t sall[G];
#pragma unroll
        for (int i = 0; i < G; ++i) {
            pre[0][i] = {1.f, 0.f};
            sall[i] = (__popc(smask[i]) + d) & 1u;
        }
#pragma unroll
        for (int j = 1; j < DC; ++j)
#pragma unroll
            for (int i = 0; i < G; ++i) pre[j][i] = evod_add(pre[j - 1][i], u[j - 1][i]);
        EvOd suf[G];
#pragma unroll
        for (int i = 0; i < G; ++i) suf[i] = {1.f, 0.f};
#pragma unroll
        for (int j = DC - 1; j >= 0; --j) {
            if (slot[j] != kNoSlot) {
                float out[G];
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    const float mag = evod_magnitude(evod_join(pre[j][i], suf[i]), clip2);
                    const uint32_t sgn = sall[i] ^ ((smask[i] >> j) & 1u);
                    out[i] = sgn ? -mag : mag;
                    suf[i] = evod_add(suf[i], u[j][i]);
                }
                Es[slot[j]] = EV::make(out);
            }
        }
    }
    return bad;
}

template <class MsgT, int G, int DC, int CPT>
__global__ void __launch_bounds__(kResMaxThreads)
resident_kernel(ResArgs a) {
    using LV = LVec<G>;
    using EV = EVec<MsgT, G>;
    constexpr int DCW = (DC + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename LV::T *Ls = reinterpret_cast<typename LV::T *>(smem_raw);
    const size_t lbytes = ((size_t)a.n * sizeof(typename LV::T) + 15) & ~size_t(15);
    typename EV::T *Es = reinterpret_cast<typename EV::T *>(smem_raw + lbytes);
    __shared__ int s_group;

    const int T = blockDim.x, tid = threadIdx.x;
    const int lane = tid & 31;
    uint32_t idx[CPT][DCW];
#pragma unroll
    for (int k = 0; k < CPT; ++k)
#pragma unroll
        for (int w = 0; w < DCW; ++w) idx[k][w] = __ldg(&a.edges[(size_t)(k * DCW + w) * T + tid]);

    const int groups = (a.F + G - 1) / G;
    for (;;) {
        if (tid == 0) s_group = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int grp = s_group;
        __syncthreads();
        if (grp >= groups) break;
        const int64_t f0 = (int64_t)grp * G;
        uint32_t exists = 0;
#pragma unroll
        for (int i = 0; i < G; ++i) exists |= (uint32_t)(f0 + i < a.F) << i;

        // channel LLRs (log2 units) into registers and L_v = R_v into Ls
        float R[kResVPT][G];
#pragma unroll
        for (int k = 0; k < kResVPT; ++k) {
            const int v = tid + k * T;
#pragma unroll
            for (int i = 0; i < G; ++i)
                R[k][i] = (v < a.n && ((exists >> i) & 1u)) ? a.llr[(f0 + i) * a.n + v] * kLog2e : 0.f;
            if (v < a.n) Ls[v] = LV::make(R[k]);
        }
        if (a.pad_slots)
            for (int s = tid; s < a.n * kResDV; s += T) Es[s] = EV::zero();
        __syncthreads();

        uint32_t active = exists, okm = 0;
        int it_done[G];
#pragma unroll
        for (int i = 0; i < G; ++i) it_done[i] = 0;
        for (int t = 1; t <= a.T_iters; ++t) {
            const uint32_t bad = check_pass<MsgT, G, DC, CPT, true>(idx, Ls, Es, t == 1, a.clip2);
            if (a.early_stop && t >= 2) {
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    const int any_bad = __syncthreads_or((int)((bad >> i) & 1u));
                    if (((active >> i) & 1u) && !any_bad) {  // z^(t-1) satisfies H z = 0
                        active &= ~(1u << i);
                        it_done[i] = t - 1;
                        okm |= 1u << i;
                    }
                }
                if (!active) break;
            } else {
                __syncthreads();
            }
            // bit pass (Eq. 7), frozen frames keep their L_v
#pragma unroll
            for (int k = 0; k < kResVPT; ++k) {
                const int v = tid + k * T;
                if (v < a.n) {
                    float L[G];
#pragma unroll
                    for (int i = 0; i < G; ++i) L[i] = R[k][i];
#pragma unroll
                    for (int q = 0; q < kResDV; ++q) {
                        float e[G];
                        EV::get(Es[v * kResDV + q], e);
#pragma unroll
                        for (int i = 0; i < G; ++i) L[i] += e[i];
                    }
                    if (active != exists) {
                        float old[G];
                        LV::get(Ls[v], old);
#pragma unroll
                        for (int i = 0; i < G; ++i)
                            if (!((active >> i) & 1u)) L[i] = old[i];
                    }
                    Ls[v] = LV::make(L);
                }
            }
            __syncthreads();
        }
        if (active) {  // frames that ran every iteration: syndrome of the final z
            const uint32_t bad = check_pass<MsgT, G, DC, CPT, false>(idx, Ls, Es, false, a.clip2);
#pragma unroll
            for (int i = 0; i < G; ++i) {
                const int any_bad = __syncthreads_or((int)((bad >> i) & 1u));
                if ((active >> i) & 1u) {
                    it_done[i] = a.T_iters;
                    if (!any_bad) okm |= 1u << i;
                }
            }
        }
        // outputs: total LLRs (natural units), packed hard decisions, counts
#pragma unroll
        for (int k = 0; k < kResVPT; ++k) {
            const int v = tid + k * T;
            const int v0 = v - lane;
            float L[G];
            if (v < a.n) {
                LV::get(Ls[v], L);
            } else {
#pragma unroll
                for (int i = 0; i < G; ++i) L[i] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < G; ++i) {
                const uint32_t word = __ballot_sync(0xffffffffu, v < a.n && L[i] >= 0.f);
                if ((exists >> i) & 1u) {
                    const int64_t f = f0 + i;
                    if (a.post && v < a.n)
                        a.post[f * a.n + v] = a.T_iters == 0 ? a.llr[f * a.n + v] : L[i] * kLn2;
                    if (a.hard && lane == 0 && v0 < a.n) a.hard[f * a.NW + (v0 >> 5)] = word;
                }
            }
        }
        if (tid == 0)
#pragma unroll
            for (int i = 0; i < G; ++i)
                if ((exists >> i) & 1u) {
                    if (a.iters) a.iters[f0 + i] = it_done[i];
                    if (a.ok) a.ok[f0 + i] = (uint8_t)((okm >> i) & 1u);
                }
        __syncthreads();
    }
}

using KernelFn = void (*)(ResArgs);

template <class MsgT, int G>
KernelFn pick_kernel(int dc) {
    switch (dc) {
        case 6: return resident_kernel<MsgT, G, 6, 8>;
        case 9: return resident_kernel<MsgT, G, 9, 5>;
        case 12: return resident_kernel<MsgT, G, 12, 4>;
        case 16: return resident_kernel<MsgT, G, 16, 3>;
        default: return nullptr;
    }
}

size_t res_smem(const ldpc_code *c, bool fp16) {
    const int G = fp16 ? 2 : 1;
    const size_t lbytes = ((size_t)c->n * 4 * G + 15) & ~size_t(15);
    return lbytes + (size_t)c->n * kResDV * (fp16 ? 2 : 4) * G;
}

}  // namespace

// Host-side plan: pick the row shape, the thread count, and lay out each
// thread's edge slots as [CPT * DCW][T] 32-bit words (two 16-bit slots each).
int build_resident_plan(ldpc_code *c) {
    ResidentPlan &p = c->res;
    p = ResidentPlan{};
    if (c->dv_max > kResDV || (int64_t)c->n * kResDV > 0xFFFE) return LDPC_OK;
    const Shape *shape = nullptr;
    for (const Shape &s : kShapes)
        if (s.dc >= c->dc_max) {
            shape = &s;
            break;
        }
    if (!shape) return LDPC_OK;
    const int64_t need = std::max(ceil_div(c->m, shape->cpt), ceil_div(c->n, kResVPT));
    const int T = (int)ceil_div(need, 32) * 32;
    if (T > kResMaxThreads) return LDPC_OK;
    const int DCW = (shape->dc + 1) / 2;
    // slot of each edge: bit * DV + rank of the edge within its bit's column
    std::vector<uint32_t> slot_of((size_t)c->nnz);
    for (int32_t v = 0; v < c->n; ++v)
        for (int32_t q = c->col_ptr[v]; q < c->col_ptr[v + 1]; ++q)
            slot_of[c->col_edge[q]] = (uint32_t)(v * kResDV + (q - c->col_ptr[v]));
    p.edges.assign((size_t)shape->cpt * DCW * T, 0xFFFFFFFFu);
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < shape->cpt; ++k) {
            const int64_t cidx = t + (int64_t)k * T;
            if (cidx >= c->m) continue;
            const int32_t e0 = c->row_ptr[cidx], d = c->row_ptr[cidx + 1] - e0;
            for (int j = 0; j < d; ++j) {
                uint32_t &w = p.edges[(size_t)(k * DCW + j / 2) * T + t];
                const int sh = (j & 1) * 16;
                w = (w & ~(0xFFFFu << sh)) | (slot_of[e0 + j] << sh);
            }
        }
    p.dc_pad = shape->dc;
    p.dv_pad = kResDV;
    p.rows_pad = T;  // thread count of the launch
    p.pad_slots = c->dv_min < kResDV;
    p.ok = true;
    return LDPC_OK;
}

bool resident_fits(const ldpc_code *c, const ldpc_decode_opts *o) {
    if (!c->res.ok) return false;
    return res_smem(c, o->msg_fp16 != 0) <= 220 * 1024;
}

size_t resident_workspace(const ldpc_code *, int32_t, const ldpc_decode_opts *) { return 256; }

int decode_resident(const ldpc_code *c, const float *d_llr, int32_t F, const ldpc_decode_opts *o,
                    float *d_post, uint32_t *d_hard, int32_t *d_iters, uint8_t *d_ok, void *d_work,
                    size_t work_bytes, cudaStream_t s) {
    if (!d_work || work_bytes < 256) return fail(LDPC_EINVAL, "workspace too small (need 256 bytes)");
    const bool fp16 = o->msg_fp16 != 0;
    KernelFn fn = fp16 ? pick_kernel<__half, 2>(c->res.dc_pad) : pick_kernel<float, 1>(c->res.dc_pad);
    if (!fn) return fail(LDPC_ENOTSUP, "no resident kernel for row degree %d", c->res.dc_pad);
    const int T = c->res.rows_pad;
    const size_t smem = res_smem(c, fp16);
    LDPC_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    LDPC_TRY_CUDA(cudaGetDevice(&dev));
    LDPC_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LDPC_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, T, smem));
    if (per_sm < 1) return fail(LDPC_ENOTSUP, "resident kernel cannot be resident (smem %zu B)", smem);
    const int G = fp16 ? 2 : 1;
    const int64_t groups = ceil_div(F, G);
    const int grid = (int)std::min<int64_t>(groups, (int64_t)sms * per_sm);
    ResArgs a;
    a.llr = d_llr;
    a.F = F;
    a.n = c->n;
    a.m = c->m;
    a.NW = c->NW;
    a.T_iters = o->max_iters;
    a.early_stop = o->early_stop;
    a.pad_slots = c->res.pad_slots ? 1 : 0;
    a.clip2 = clip_log2(o->clip);
    a.edges = c->d.res_edges;
    a.post = d_post;
    a.hard = d_hard;
    a.iters = d_iters;
    a.ok = d_ok;
    a.counter = static_cast<unsigned *>(d_work);
    LDPC_TRY_CUDA(cudaMemsetAsync(d_work, 0, sizeof(unsigned), s));
    fn<<<grid, T, smem, s>>>(a);
    LDPC_TRY_CUDA(cudaGetLastError());
    return LDPC_OK;
}

}  // namespace ldpc

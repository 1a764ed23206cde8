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
constexpr int kResSlots = 4;      // message slots per bit (column degree <= 4)
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

// One message slot holding G frames, and the 16-byte record of a bit's slots.
template <class MsgT, int G>
struct EVec;
template <>
struct EVec<__half, 2> {
    using T = __half2;
    using Rec = uint4;  // 4 x half2
    __device__ static void get(T v, float *x) {
        const float2 f = __half22float2(v);
        x[0] = f.x;
        x[1] = f.y;
    }
    __device__ static T make(const float *x) { return __floats2half2_rn(x[0], x[1]); }
    __device__ static void slot(const Rec &r, int q, float *x) {
        const uint32_t w = q == 0 ? r.x : q == 1 ? r.y : q == 2 ? r.z : r.w;
        get(*reinterpret_cast<const __half2 *>(&w), x);
    }
};
template <>
struct EVec<float, 1> {
    using T = float;
    using Rec = float4;
    __device__ static void get(T v, float *x) { x[0] = v; }
    __device__ static T make(const float *x) { return x[0]; }
    __device__ static void slot(const Rec &r, int q, float *x) {
        x[0] = q == 0 ? r.x : q == 1 ? r.y : q == 2 ? r.z : r.w;
    }
};

struct ResArgs {
    const float *llr;
    int32_t F, n, m, NW, T_iters, early_stop;
    float clip2;
    const uint32_t *edges;  // [CPT * DCW][T]
    float *post;
    uint32_t *hard;
    int32_t *iters;
    uint8_t *ok;
    unsigned *counter;
};

// Shared-memory layout of a group: Ls[n] (LV::T) then Es[n][4] (EV::T), so
// that the 16-bit slot s = 4 v + r of an edge gives both addresses:
// message at byte 4 s * sizeof(slot) / 4, total LLR of bit v = s >> 2.
template <class MsgT, int G>
struct Smem {
    unsigned char *L;  // Ls base
    unsigned char *E;  // Es base
    __device__ typename LVec<G>::T &Lv(uint32_t s) const {
        return *reinterpret_cast<typename LVec<G>::T *>(L + (s >> 2) * sizeof(typename LVec<G>::T));
    }
    __device__ typename EVec<MsgT, G>::T &Ev(uint32_t s) const {
        return *reinterpret_cast<typename EVec<MsgT, G>::T *>(E + s * sizeof(typename EVec<MsgT, G>::T));
    }
};

__device__ __forceinline__ uint32_t slot_of(const uint32_t *w, int j) {
    return (j & 1) ? (w[j >> 1] >> 16) : (w[j >> 1] & 0xFFFFu);
}

// Check pass over the thread's checks, rows of exactly DC edges (REG) or of
// at most DC edges with unused slots marked kNoSlot.  Updates the messages in
// place.  With SYN, also returns bit i set when frame i has a check that the
// hard decisions z = [L >= 0] (L as left by the last bit pass) do not satisfy.
template <class MsgT, int G, int DC, int CPT, bool REG, bool SYN>
__device__ __forceinline__ uint32_t check_pass(const uint32_t (&idx)[CPT][(DC + 1) / 2],
                                               const Smem<MsgT, G> &sm, float clip2) {
    using LV = LVec<G>;
    using EV = EVec<MsgT, G>;
    uint32_t zacc[G];
#pragma unroll
    for (int i = 0; i < G; ++i) zacc[i] = 0;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        if ((idx[k][0] & 0xFFFFu) == kNoSlot) continue;  // no check in this slot
        uint32_t slot[DC];
#pragma unroll
        for (int j = 0; j < DC; ++j) slot[j] = slot_of(idx[k], j);
        float u[DC][G];
        uint32_t xbits[DC][G], sacc[G], zsgn[G];
        int d = 0;
#pragma unroll
        for (int i = 0; i < G; ++i) sacc[i] = zsgn[i] = 0;
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (REG || slot[j] != kNoSlot) {
                ++d;
                float L[G], Eo[G];
                LV::get(sm.Lv(slot[j]), L);
                EV::get(sm.Ev(slot[j]), Eo);
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    if (SYN) zsgn[i] ^= __float_as_uint(L[i]);  // bit 31: parity of [L < 0]
                    const float x = L[i] - Eo[i];  // Eq. 6 rearranged
                    xbits[j][i] = __float_as_uint(x);
                    sacc[i] ^= xbits[j][i];
                    u[j][i] = ex2_approx(-fminf(fabsf(x), clip2));
                }
            } else {
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    u[j][i] = 0.f;  // identity for the pair products
                    xbits[j][i] = 0u;
                }
            }
        }
        // parity of z = [L >= 0] over the row = d + parity of [L < 0] (the bit
        // pass leaves no -0, so the sign bit is exactly [L < 0])
        if (SYN)
#pragma unroll
            for (int i = 0; i < G; ++i) zacc[i] |= (zsgn[i] >> 31) ^ (uint32_t)(d & 1);
        // (-1)^d folded into the accumulated sign bit
#pragma unroll
        for (int i = 0; i < G; ++i) sacc[i] ^= (uint32_t)(d & 1) << 31;
        EvOd pre[DC][G];
#pragma unroll
        for (int i = 0; i < G; ++i) pre[0][i] = {1.f, 0.f};
#pragma unroll
        for (int j = 1; j < DC; ++j)
#pragma unroll
            for (int i = 0; i < G; ++i) pre[j][i] = evod_add(pre[j - 1][i], u[j - 1][i]);
        EvOd suf[G];
#pragma unroll
        for (int i = 0; i < G; ++i) suf[i] = {1.f, 0.f};
#pragma unroll
        for (int j = DC - 1; j >= 0; --j) {
            if (REG || slot[j] != kNoSlot) {
                float out[G];
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    const float mag = evod_magnitude(evod_join(pre[j][i], suf[i]), clip2);
                    out[i] = __uint_as_float(__float_as_uint(mag) |
                                             ((sacc[i] ^ xbits[j][i]) & 0x80000000u));
                    suf[i] = evod_add(suf[i], u[j][i]);
                }
                sm.Ev(slot[j]) = EV::make(out);
            }
        }
    }
    uint32_t bad = 0;
    if (SYN)
#pragma unroll
        for (int i = 0; i < G; ++i) bad |= (zacc[i] & 1u) << i;
    return bad;
}

// Syndrome of z = [L >= 0] over the thread's checks (no message update).
template <class MsgT, int G, int DC, int CPT>
__device__ __forceinline__ uint32_t syndrome_pass(const uint32_t (&idx)[CPT][(DC + 1) / 2],
                                                  const Smem<MsgT, G> &sm) {
    uint32_t bad = 0;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        uint32_t par = 0;
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            const uint32_t s = slot_of(idx[k], j);
            if (s == kNoSlot) continue;
            float L[G];
            LVec<G>::get(sm.Lv(s), L);
#pragma unroll
            for (int i = 0; i < G; ++i) par ^= (uint32_t)(L[i] >= 0.f) << i;
        }
        bad |= par;  // a check with odd parity is unsatisfied
    }
    return bad;
}

// Bit pass (Eq. 7): L_v = R_v + the bit's message slots in ascending edge
// order; frames not in `active` keep their L_v.  REG codes have exactly three
// edges per bit; otherwise all four slots are summed (unused ones hold 0).
template <class MsgT, int G, bool REG, bool SYN>
__device__ __forceinline__ void bit_pass(const float (&R)[kResVPT][G], const Smem<MsgT, G> &sm,
                                         int n, int T, uint32_t active, uint32_t exists) {
    using LV = LVec<G>;
    using EV = EVec<MsgT, G>;
    constexpr int NS = REG ? 3 : kResSlots;
#pragma unroll
    for (int k = 0; k < kResVPT; ++k) {
        const int v = threadIdx.x + k * T;
        if (v < n) {
            const typename EV::Rec rec =
                *reinterpret_cast<const typename EV::Rec *>(sm.E + (size_t)v * kResSlots * sizeof(typename EV::T));
            float L[G];
#pragma unroll
            for (int i = 0; i < G; ++i) L[i] = R[k][i];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                float e[G];
                EV::slot(rec, q, e);
#pragma unroll
                for (int i = 0; i < G; ++i) L[i] += e[i];
            }
            if (SYN)
#pragma unroll
                for (int i = 0; i < G; ++i) L[i] += 0.f;  // no -0: z = [L >= 0] by sign
            typename LV::T *dst = reinterpret_cast<typename LV::T *>(sm.L) + v;
            if (active != exists) {
                float old[G];
                LV::get(*dst, old);
#pragma unroll
                for (int i = 0; i < G; ++i)
                    if (!((active >> i) & 1u)) L[i] = old[i];
            }
            *dst = LV::make(L);
        }
    }
}

template <class MsgT, int G, int DC, int CPT, bool REG, bool SYN>
__global__ void __launch_bounds__(kResMaxThreads)
resident_kernel(ResArgs a) {
    using LV = LVec<G>;
    using EV = EVec<MsgT, G>;
    constexpr int DCW = (DC + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<MsgT, G> sm;
    sm.L = smem_raw;
    sm.E = smem_raw + (((size_t)a.n * sizeof(typename LV::T) + 15) & ~size_t(15));
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

        // channel LLRs (log2 units) into registers and L_v = R_v; messages 0
        float R[kResVPT][G];
#pragma unroll
        for (int k = 0; k < kResVPT; ++k) {
            const int v = tid + k * T;
#pragma unroll
            for (int i = 0; i < G; ++i)
                R[k][i] = (v < a.n && ((exists >> i) & 1u)) ? a.llr[(f0 + i) * a.n + v] * kLog2e : 0.f;
            if (v < a.n) {
                reinterpret_cast<typename LV::T *>(sm.L)[v] = LV::make(R[k]);
                *reinterpret_cast<uint4 *>(sm.E + (size_t)v * kResSlots * sizeof(typename EV::T)) =
                    make_uint4(0u, 0u, 0u, 0u);
                if (sizeof(typename EV::T) == 8)
                    *reinterpret_cast<uint4 *>(sm.E + (size_t)v * kResSlots * 8 + 16) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        __syncthreads();

        uint32_t active = exists, okm = 0;
        int it_done[G];
#pragma unroll
        for (int i = 0; i < G; ++i) it_done[i] = 0;
        for (int t = 1; t <= a.T_iters; ++t) {
            if (SYN && t >= 2) {
                const uint32_t bad = check_pass<MsgT, G, DC, CPT, REG, true>(idx, sm, a.clip2);
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
                check_pass<MsgT, G, DC, CPT, REG, false>(idx, sm, a.clip2);
                __syncthreads();
            }
            bit_pass<MsgT, G, REG, SYN>(R, sm, a.n, T, active, exists);
            __syncthreads();
        }
        if (active) {  // frames that ran every iteration: syndrome of the final z
            const uint32_t bad = syndrome_pass<MsgT, G, DC, CPT>(idx, sm);
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
                LV::get(reinterpret_cast<typename LV::T *>(sm.L)[v], L);
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

template <class MsgT, int G, int DC, int CPT>
KernelFn pick_flags(bool reg, bool syn) {
    if (reg) return syn ? resident_kernel<MsgT, G, DC, CPT, true, true> : resident_kernel<MsgT, G, DC, CPT, true, false>;
    return syn ? resident_kernel<MsgT, G, DC, CPT, false, true> : resident_kernel<MsgT, G, DC, CPT, false, false>;
}

template <class MsgT, int G>
KernelFn pick_kernel(int dc, bool reg, bool syn) {
    switch (dc) {
        case 6: return pick_flags<MsgT, G, 6, 8>(reg, syn);
        case 9: return pick_flags<MsgT, G, 9, 5>(reg, syn);
        case 12: return pick_flags<MsgT, G, 12, 4>(reg, syn);
        case 16: return pick_flags<MsgT, G, 16, 3>(reg, syn);
        default: return nullptr;
    }
}

size_t res_smem(const ldpc_code *c, bool fp16) {
    const int G = fp16 ? 2 : 1;
    const size_t lbytes = ((size_t)c->n * 4 * G + 15) & ~size_t(15);
    return lbytes + (size_t)c->n * kResSlots * (fp16 ? 2 : 4) * G;
}

}  // namespace

// Host-side plan: pick the row shape and the thread count, and lay out each
// thread's edge slots as [CPT * DCW][T] 32-bit words (two 16-bit slots each).
// The slot of an edge is 4 v + r, v its bit and r its rank in v's column.
int build_resident_plan(ldpc_code *c) {
    ResidentPlan &p = c->res;
    p = ResidentPlan{};
    if (c->dv_max > kResSlots || (int64_t)c->n * kResSlots > 0xFFFE) return LDPC_OK;
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
    std::vector<uint32_t> slot_of((size_t)c->nnz);
    for (int32_t v = 0; v < c->n; ++v)
        for (int32_t q = c->col_ptr[v]; q < c->col_ptr[v + 1]; ++q)
            slot_of[c->col_edge[q]] = (uint32_t)(v * kResSlots + (q - c->col_ptr[v]));
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
    p.dv_pad = kResSlots;
    p.rows_pad = T;  // thread count of the launch
    // exactly dc edges per check and three per bit: the specialised kernels
    p.regular = c->dc_min == shape->dc && c->dc_max == shape->dc && c->dv_min == 3 && c->dv_max == 3;
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
    const bool syn = o->early_stop != 0 && o->max_iters >= 2;
    KernelFn fn = fp16 ? pick_kernel<__half, 2>(c->res.dc_pad, c->res.regular, syn)
                       : pick_kernel<float, 1>(c->res.dc_pad, c->res.regular, syn);
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

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
constexpr Shape kShapes[] = {{6, 8}, {9, 6}, {12, 4}, {16, 3}};

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
                                         int n, int tid, int T, uint32_t active, uint32_t exists) {
    using LV = LVec<G>;
    using EV = EVec<MsgT, G>;
    constexpr int NS = REG ? 3 : kResSlots;
#pragma unroll
    for (int k = 0; k < kResVPT; ++k) {
        const int v = tid + k * T;
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

// A group of threads decoding one frame group: the whole CTA ...
struct BlockTeam {
    __device__ int tid() const { return threadIdx.x; }
    __device__ int size() const { return blockDim.x; }
    __device__ void sync() const { __syncthreads(); }
    __device__ int any(int p) const { return __syncthreads_or(p); }
};

// ... or a warp-aligned slice of it with its own named barrier (id >= 1);
// a one-warp team synchronises with warp primitives.
struct SubTeam {
    int base, count, bar_id;
    __device__ int tid() const { return (int)threadIdx.x - base; }
    __device__ int size() const { return count; }
    __device__ void sync() const {
        if (count == 32)
            __syncwarp();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(count) : "memory");
    }
    __device__ int any(int p) const {
        if (count == 32) return __any_sync(0xffffffffu, p);
        int r;
        asm volatile(
            "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\t"
            "bar.red.or.pred q, %2, %3, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
            : "=r"(r)
            : "r"(p), "r"(bar_id), "r"(count)
            : "memory");
        return r;
    }
};

// Where the G frames of a group come from and go to (NULL llr = no frame).
template <int G>
struct FrameIO {
    const float *llr[G];
    float *post[G];
    uint32_t *hard[G];
    int32_t *iters[G];
    uint8_t *ok[G];
};

// Decodes one group of G frames with the team's threads: load R, iterate
// (check pass, bit pass), final syndrome, outputs.  Ends with a team barrier.
template <class MsgT, int G, int DC, int CPT, bool REG, bool SYN, class Team>
__device__ __forceinline__ void decode_group(const Team &tm, const uint32_t (&idx)[CPT][(DC + 1) / 2],
                                             const Smem<MsgT, G> &sm, int n, const FrameIO<G> &io,
                                             int T_iters, float clip2) {
    using LV = LVec<G>;
    using EV = EVec<MsgT, G>;
    const int tid = tm.tid(), T = tm.size();
    const int lane = threadIdx.x & 31;
    uint32_t exists = 0;
#pragma unroll
    for (int i = 0; i < G; ++i) exists |= (uint32_t)(io.llr[i] != nullptr) << i;

    // channel LLRs (log2 units) into registers and L_v = R_v; messages 0
    float R[kResVPT][G];
#pragma unroll
    for (int k = 0; k < kResVPT; ++k) {
        const int v = tid + k * T;
#pragma unroll
        for (int i = 0; i < G; ++i) R[k][i] = (v < n && io.llr[i]) ? io.llr[i][v] * kLog2e : 0.f;
        if (v < n) {
            reinterpret_cast<typename LV::T *>(sm.L)[v] = LV::make(R[k]);
            *reinterpret_cast<uint4 *>(sm.E + (size_t)v * kResSlots * sizeof(typename EV::T)) =
                make_uint4(0u, 0u, 0u, 0u);
            if (sizeof(typename EV::T) == 8)
                *reinterpret_cast<uint4 *>(sm.E + (size_t)v * kResSlots * 8 + 16) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    tm.sync();

    uint32_t active = exists, okm = 0;
    int it_done[G];
#pragma unroll
    for (int i = 0; i < G; ++i) it_done[i] = 0;
    for (int t = 1; t <= T_iters; ++t) {
        if (SYN && t >= 2) {
            const uint32_t bad = check_pass<MsgT, G, DC, CPT, REG, true>(idx, sm, clip2);
#pragma unroll
            for (int i = 0; i < G; ++i) {
                const int any_bad = tm.any((int)((bad >> i) & 1u));
                if (((active >> i) & 1u) && !any_bad) {  // z^(t-1) satisfies H z = 0
                    active &= ~(1u << i);
                    it_done[i] = t - 1;
                    okm |= 1u << i;
                }
            }
            if (!active) break;
        } else {
            check_pass<MsgT, G, DC, CPT, REG, false>(idx, sm, clip2);
            tm.sync();
        }
        bit_pass<MsgT, G, REG, SYN>(R, sm, n, tid, T, active, exists);
        tm.sync();
    }
    if (active) {  // frames that ran every iteration: syndrome of the final z
        const uint32_t bad = syndrome_pass<MsgT, G, DC, CPT>(idx, sm);
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const int any_bad = tm.any((int)((bad >> i) & 1u));
            if ((active >> i) & 1u) {
                it_done[i] = T_iters;
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
        if (v < n) {
            LV::get(reinterpret_cast<typename LV::T *>(sm.L)[v], L);
        } else {
#pragma unroll
            for (int i = 0; i < G; ++i) L[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const uint32_t word = __ballot_sync(0xffffffffu, v < n && L[i] >= 0.f);
            if (io.llr[i]) {
                if (io.post[i] && v < n) io.post[i][v] = T_iters == 0 ? io.llr[i][v] : L[i] * kLn2;
                if (io.hard[i] && lane == 0 && v0 < n) io.hard[i][v0 >> 5] = word;
            }
        }
    }
    if (tid == 0)
#pragma unroll
        for (int i = 0; i < G; ++i)
            if (io.llr[i]) {
                if (io.iters[i]) *io.iters[i] = it_done[i];
                if (io.ok[i]) *io.ok[i] = (uint8_t)((okm >> i) & 1u);
            }
    tm.sync();
}

template <class MsgT, int G>
__device__ __forceinline__ Smem<MsgT, G> smem_at(unsigned char *base, int n) {
    Smem<MsgT, G> sm;
    sm.L = base;
    sm.E = base + (((size_t)n * sizeof(typename LVec<G>::T) + 15) & ~size_t(15));
    return sm;
}

template <class MsgT, int G, int DC, int CPT, bool REG, bool SYN>
__global__ void __launch_bounds__(kResMaxThreads)
resident_kernel(ResArgs a) {
    constexpr int DCW = (DC + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem<MsgT, G> sm = smem_at<MsgT, G>(smem_raw, a.n);
    __shared__ int s_group;
    const int T = blockDim.x, tid = threadIdx.x;
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
        FrameIO<G> io;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const int64_t f = (int64_t)grp * G + i;
            const bool ex = f < a.F;
            io.llr[i] = ex ? a.llr + f * a.n : nullptr;
            io.post[i] = ex && a.post ? a.post + f * a.n : nullptr;
            io.hard[i] = ex && a.hard ? a.hard + f * a.NW : nullptr;
            io.iters[i] = ex && a.iters ? a.iters + f : nullptr;
            io.ok[i] = ex && a.ok ? a.ok + f : nullptr;
        }
        decode_group<MsgT, G, DC, CPT, REG, SYN>(BlockTeam{}, idx, sm, a.n, io, a.T_iters, a.clip2);
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
        case 9: return pick_flags<MsgT, G, 9, 6>(reg, syn);
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

// Edge-slot table for threads of a team of T: [CPT * DCW][T] 32-bit words,
// two 16-bit slots each; check t + k T goes to thread t, slot k.  The slot of
// an edge is 4 v + r, v its bit and r its rank in v's column.
std::vector<uint32_t> build_slot_table(const ldpc_code *c, int dc, int cpt, int T) {
    const int DCW = (dc + 1) / 2;
    std::vector<uint32_t> slot_of((size_t)c->nnz);
    for (int32_t v = 0; v < c->n; ++v)
        for (int32_t q = c->col_ptr[v]; q < c->col_ptr[v + 1]; ++q)
            slot_of[c->col_edge[q]] = (uint32_t)(v * kResSlots + (q - c->col_ptr[v]));
    std::vector<uint32_t> tab((size_t)cpt * DCW * T, 0xFFFFFFFFu);
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < cpt; ++k) {
            const int64_t cidx = t + (int64_t)k * T;
            if (cidx >= c->m) continue;
            const int32_t e0 = c->row_ptr[cidx], d = c->row_ptr[cidx + 1] - e0;
            for (int j = 0; j < d; ++j) {
                uint32_t &w = tab[(size_t)(k * DCW + j / 2) * T + t];
                const int sh = (j & 1) * 16;
                w = (w & ~(0xFFFFu << sh)) | (slot_of[e0 + j] << sh);
            }
        }
    return tab;
}

const Shape *pick_shape(const ldpc_code *c) {
    if (c->dv_max > kResSlots || (int64_t)c->n * kResSlots > 0xFFFE) return nullptr;
    for (const Shape &s : kShapes)
        if (s.dc >= c->dc_max) return &s;
    return nullptr;
}

int team_threads(const ldpc_code *c, const Shape &s) {
    const int64_t need = std::max(ceil_div(c->m, s.cpt), ceil_div(c->n, kResVPT));
    return (int)ceil_div(need, 32) * 32;
}

}  // namespace

// Host-side plan of the single-code resident launch: row shape, thread count
// and slot table.
int build_resident_plan(ldpc_code *c) {
    ResidentPlan &p = c->res;
    p = ResidentPlan{};
    const Shape *shape = pick_shape(c);
    if (!shape) return LDPC_OK;
    const int T = team_threads(c, *shape);
    if (T > kResMaxThreads) return LDPC_OK;
    p.edges = build_slot_table(c, shape->dc, shape->cpt, T);
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
    int sms = 0, per_sm = 0;
    LDPC_TRY(sm_count(&sms));
    LDPC_TRY(kernel_setup((const void *)fn, T, smem, &per_sm));
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

// ---------------------------------------------------------------------------
// Mixed-code batches: frames of several codes in one persistent launch.
//
// Each code of the plan is decoded by teams of T_c threads (T_c a power of two
// <= 512, from the code's resident shape); a 512-thread CTA holds 512 / T_c
// teams (as many as its shared memory allows), each decoding its own group of
// G frames with its own named barrier, so a CTA works on many frames of a
// small code or on one group of the largest.  Frames are bucketed by code on
// the device (count, offsets, scatter), and CTAs take work items -- a CTA-full
// of groups of one code -- from a counter, codes with the most edges first by
// default.  Every step is a kernel or a memset on the caller's stream, so the
// call can be captured in a CUDA graph.  Results per frame do not depend on
// the bucketing or the configuration: each frame's arithmetic is that of the
// single-code decoder.
namespace ldpc {
namespace {

constexpr int kMixThreads = 512;

struct MixedDesc {
    int32_t n, dc, team, teams, code;
    const uint32_t *edges;  // [cpt * DCW][team]
};

struct MixedArgs {
    const MixedDesc *desc;      // by work-order position
    int32_t ncodes;
    const unsigned *item_off;   // [ncodes + 1], by position
    const unsigned *start;      // [ncodes], by code: first slot in `sorted`
    const unsigned *count;      // [ncodes], by code
    const int32_t *sorted;      // frame indices grouped by code
    const int64_t *llr_off, *hard_off;
    const float *llr;
    float *post;
    uint32_t *hard;
    int32_t *iters;
    uint8_t *ok;
    unsigned *counter;
    int32_t T_iters, gpi;
    float clip2;
};

template <class MsgT, int G>
__host__ __device__ __forceinline__ size_t team_bytes(int n) {
    return (((size_t)n * sizeof(float) * G + 15) & ~size_t(15)) + (size_t)n * kResSlots * sizeof(MsgT) * G;
}

__global__ void mixed_count(const int32_t *__restrict__ frame_code, int32_t F, int32_t ncodes,
                            unsigned *__restrict__ count, int32_t *__restrict__ iters,
                            uint8_t *__restrict__ ok) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int c = frame_code[f];
    if (c < 0 || c >= ncodes) {  // not decoded: marked with iters = -1, ok = 0
        if (iters) iters[f] = -1;
        if (ok) ok[f] = 0;
        return;
    }
    atomicAdd(&count[c], 1u);
}

__global__ void mixed_offsets(const unsigned *__restrict__ count, const MixedDesc *__restrict__ desc,
                              int32_t ncodes, int32_t G, int32_t gpi, unsigned *__restrict__ start,
                              unsigned *__restrict__ item_off, unsigned *__restrict__ fill) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned fo = 0, io = 0;
    for (int p = 0; p < ncodes; ++p) {
        const int c = desc[p].code;
        start[c] = fo;
        fill[c] = 0;
        item_off[p] = io;
        const unsigned groups = (count[c] + G - 1) / G;
        const unsigned per_item = (unsigned)(desc[p].teams * gpi);
        io += (groups + per_item - 1) / per_item;
        fo += count[c];
    }
    item_off[ncodes] = io;
}

__global__ void mixed_scatter(const int32_t *__restrict__ frame_code, int32_t F, int32_t ncodes,
                              const unsigned *__restrict__ start, unsigned *__restrict__ fill,
                              int32_t *__restrict__ sorted) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int c = frame_code[f];
    if (c < 0 || c >= ncodes) return;
    sorted[start[c] + atomicAdd(&fill[c], 1u)] = (int32_t)f;
}

template <class MsgT, int G, int DC, int CPT, bool SYN>
__device__ __forceinline__ void mixed_run(const SubTeam &tm, const MixedDesc &d, const MixedArgs &a,
                                          unsigned char *base, unsigned local) {
    constexpr int DCW = (DC + 1) / 2;
    uint32_t idx[CPT][DCW];
#pragma unroll
    for (int k = 0; k < CPT; ++k)
#pragma unroll
        for (int w = 0; w < DCW; ++w) idx[k][w] = __ldg(&d.edges[(size_t)(k * DCW + w) * d.team + tm.tid()]);
    const Smem<MsgT, G> sm = smem_at<MsgT, G>(base, d.n);
    const unsigned cnt = a.count[d.code], st = a.start[d.code];
    const int team = tm.base / d.team;
    for (int gi = 0; gi < a.gpi; ++gi) {
        const unsigned grp = (local * a.gpi + gi) * d.teams + team;
        if ((size_t)grp * G >= cnt) break;
        FrameIO<G> io;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const unsigned j = grp * G + i;
            if (j < cnt) {
                const int f = a.sorted[st + j];
                io.llr[i] = a.llr + a.llr_off[f];
                io.post[i] = a.post ? a.post + a.llr_off[f] : nullptr;
                io.hard[i] = a.hard ? a.hard + a.hard_off[f] : nullptr;
                io.iters[i] = a.iters ? a.iters + f : nullptr;
                io.ok[i] = a.ok ? a.ok + f : nullptr;
            } else {
                io.llr[i] = nullptr;
                io.post[i] = nullptr;
                io.hard[i] = nullptr;
                io.iters[i] = nullptr;
                io.ok[i] = nullptr;
            }
        }
        decode_group<MsgT, G, DC, CPT, true, SYN>(tm, idx, sm, d.n, io, a.T_iters, a.clip2);
    }
}

template <class MsgT, int G, bool SYN>
__global__ void __launch_bounds__(kMixThreads)
mixed_kernel(MixedArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned s_item;
    const unsigned total = a.item_off[a.ncodes];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u);
        __syncthreads();
        const unsigned item = s_item;
        __syncthreads();
        if (item >= total) break;
        int p = 0;
        while (item >= a.item_off[p + 1]) ++p;
        const MixedDesc d = a.desc[p];
        const int team = threadIdx.x / d.team;
        if (team < d.teams) {
            const SubTeam tm{team * d.team, d.team, 1 + team};
            unsigned char *base = smem_raw + (size_t)team * team_bytes<MsgT, G>(d.n);
            const unsigned local = item - a.item_off[p];
            switch (d.dc) {
                case 6: mixed_run<MsgT, G, 6, 8, SYN>(tm, d, a, base, local); break;
                case 9: mixed_run<MsgT, G, 9, 6, SYN>(tm, d, a, base, local); break;
                case 12: mixed_run<MsgT, G, 12, 4, SYN>(tm, d, a, base, local); break;
                default: break;
            }
        }
        __syncthreads();
    }
}

using MixedFn = void (*)(MixedArgs);

MixedFn pick_mixed(bool fp16, bool syn) {
    if (fp16) return syn ? mixed_kernel<__half, 2, true> : mixed_kernel<__half, 2, false>;
    return syn ? mixed_kernel<float, 1, true> : mixed_kernel<float, 1, false>;
}

}  // namespace
}  // namespace ldpc

struct ldpc_mixed {
    int32_t ncodes = 0;
    bool fp16 = true;
    int device = -1;
    std::vector<const ldpc_code *> codes;
    std::vector<ldpc::MixedDesc> host_desc;   // in code order
    std::vector<uint32_t *> tables;           // device slot tables, per code
    ldpc::MixedDesc *d_desc = nullptr;        // device, in work order
    size_t smem = 0;
    ldpc_mixed_config cfg{0, 1, 1};
    int32_t desc_order = -1;                  // cfg.order the device array holds
};

namespace ldpc {
namespace {

int upload_order(ldpc_mixed *p, int32_t order) {
    std::vector<MixedDesc> d(p->host_desc);
    if (order == LDPC_MIXED_ORDER_LARGEST_FIRST)
        std::stable_sort(d.begin(), d.end(), [&](const MixedDesc &a, const MixedDesc &b) {
            return p->codes[a.code]->nnz > p->codes[b.code]->nnz;
        });
    LDPC_TRY_CUDA(cudaMemcpy(p->d_desc, d.data(), sizeof(MixedDesc) * d.size(), cudaMemcpyHostToDevice));
    p->desc_order = order;
    return LDPC_OK;
}

struct MixedWs {
    unsigned *count, *fill, *start, *item_off, *counter;
    int32_t *sorted;
};

size_t mixed_layout(int32_t ncodes, int32_t F, MixedWs *w, void *base) {
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += align256(b);
        return o;
    };
    const size_t oC = take(sizeof(unsigned) * ncodes);
    const size_t oF = take(sizeof(unsigned) * ncodes);
    const size_t oS = take(sizeof(unsigned) * ncodes);
    const size_t oI = take(sizeof(unsigned) * (ncodes + 1));
    const size_t oK = take(sizeof(unsigned));
    const size_t oX = take(sizeof(int32_t) * std::max(F, 1));
    if (w && base) {
        char *b = static_cast<char *>(base);
        w->count = reinterpret_cast<unsigned *>(b + oC);
        w->fill = reinterpret_cast<unsigned *>(b + oF);
        w->start = reinterpret_cast<unsigned *>(b + oS);
        w->item_off = reinterpret_cast<unsigned *>(b + oI);
        w->counter = reinterpret_cast<unsigned *>(b + oK);
        w->sorted = reinterpret_cast<int32_t *>(b + oX);
    }
    return off;
}

}  // namespace
}  // namespace ldpc

using namespace ldpc;

extern "C" {

int ldpc_mixed_create(const ldpc_code *const *codes, int32_t ncodes, int32_t msg_fp16,
                      ldpc_mixed **out) {
    if (!out) return fail(LDPC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!codes || ncodes < 1 || ncodes > 4096) return fail(LDPC_EINVAL, "need 1..4096 codes");
    if (msg_fp16 != 0 && msg_fp16 != 1) return fail(LDPC_EINVAL, "msg_fp16 must be 0 or 1");
    int dev = -1;
    LDPC_TRY_CUDA(cudaGetDevice(&dev));
    ldpc_mixed *p = new (std::nothrow) ldpc_mixed();
    if (!p) return fail(LDPC_ENOMEM, "host allocation failed");
    p->ncodes = ncodes;
    p->fp16 = msg_fp16 != 0;
    p->device = dev;
    const int G = p->fp16 ? 2 : 1;
    auto cleanup = [&](int st) {
        ldpc_mixed_destroy(p);
        return st;
    };
    for (int32_t i = 0; i < ncodes; ++i) {
        const ldpc_code *c = codes[i];
        if (!c || !c->on_device || c->device != dev) return cleanup(fail(LDPC_EINVAL, "code %d is missing or not on this device", i));
        const Shape *sh = pick_shape(c);
        if (!sh || !c->res.ok || !c->res.regular || sh->dc > 12)
            return cleanup(fail(LDPC_ENOTSUP, "code %d is not a regular column-weight-3 code with row weight 6, 9 or 12", i));
        int team = 32;
        while (team < team_threads(c, *sh)) team *= 2;
        if (team > kMixThreads) return cleanup(fail(LDPC_ENOTSUP, "code %d is too long for a mixed batch", i));
        const size_t tb = G == 2 ? team_bytes<__half, 2>(c->n) : team_bytes<float, 1>(c->n);
        const int teams = std::min<int>(kMixThreads / team, (int)((220 * 1024) / tb));
        if (teams < 1) return cleanup(fail(LDPC_ENOTSUP, "code %d does not fit in shared memory", i));
        std::vector<uint32_t> tab = build_slot_table(c, sh->dc, sh->cpt, team);
        uint32_t *dt = nullptr;
        cudaError_t err = cudaMalloc(&dt, sizeof(uint32_t) * tab.size());
        if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaMalloc(mixed slot table)"));
        p->tables.push_back(dt);
        err = cudaMemcpy(dt, tab.data(), sizeof(uint32_t) * tab.size(), cudaMemcpyHostToDevice);
        if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaMemcpy(mixed slot table)"));
        p->codes.push_back(c);
        p->host_desc.push_back(MixedDesc{c->n, sh->dc, team, teams, i, dt});
        p->smem = std::max(p->smem, (size_t)teams * tb);
    }
    cudaError_t err = cudaMalloc(&p->d_desc, sizeof(MixedDesc) * ncodes);
    if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaMalloc(mixed descriptors)"));
    int st = upload_order(p, p->cfg.order);
    if (st != LDPC_OK) return cleanup(st);
    *out = p;
    return LDPC_OK;
}

void ldpc_mixed_destroy(ldpc_mixed *p) {
    if (!p) return;
    for (uint32_t *t : p->tables) cudaFree(t);
    if (p->d_desc) cudaFree(p->d_desc);
    delete p;
}

int ldpc_mixed_workspace_size(const ldpc_mixed *p, int32_t F, size_t *bytes) {
    if (!p || !bytes || F < 0) return fail(LDPC_EINVAL, "bad arguments");
    *bytes = mixed_layout(p->ncodes, F, nullptr, nullptr);
    return LDPC_OK;
}

int ldpc_mixed_get_config(const ldpc_mixed *p, ldpc_mixed_config *cfg) {
    if (!p || !cfg) return fail(LDPC_EINVAL, "bad arguments");
    *cfg = p->cfg;
    return LDPC_OK;
}

int ldpc_mixed_set_config(ldpc_mixed *p, const ldpc_mixed_config *cfg) {
    if (!p || !cfg) return fail(LDPC_EINVAL, "bad arguments");
    if (cfg->order < 0 || cfg->order > 1 || cfg->groups_per_item < 1 || cfg->groups_per_item > 64 ||
        cfg->ctas_per_sm < 1 || cfg->ctas_per_sm > 4)
        return fail(LDPC_EINVAL, "configuration out of range");
    if (cfg->order != p->desc_order) LDPC_TRY(upload_order(p, cfg->order));
    p->cfg = *cfg;
    return LDPC_OK;
}

int ldpc_decode_mixed(const ldpc_mixed *p, const int32_t *d_frame_code, const int64_t *d_llr_off,
                      const int64_t *d_hard_off, const float *d_llr, int32_t F, int32_t max_iters,
                      int32_t early_stop, float clip, float *d_post, uint32_t *d_hard,
                      int32_t *d_iters, uint8_t *d_ok, void *d_work, size_t work_bytes,
                      ldpc_stream_t stream) {
    if (!p) return fail(LDPC_EINVAL, "plan is NULL");
    if (F < 0 || max_iters < 0 || !(clip > 0.f)) return fail(LDPC_EINVAL, "bad F, max_iters or clip");
    if (early_stop != 0 && early_stop != 1) return fail(LDPC_EINVAL, "early_stop must be 0 or 1");
    if (F == 0) return LDPC_OK;
    if (!d_frame_code || !d_llr_off || !d_llr || (d_hard && !d_hard_off))
        return fail(LDPC_EINVAL, "NULL pointer");
    int dev = -1;
    LDPC_TRY_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return fail(LDPC_EINVAL, "plan lives on device %d", p->device);
    MixedWs w{};
    const size_t need = mixed_layout(p->ncodes, F, &w, d_work);
    if (!d_work || work_bytes < need) return fail(LDPC_EINVAL, "workspace too small (%zu < %zu)", work_bytes, need);
    cudaStream_t s = (cudaStream_t)stream;
    const int G = p->fp16 ? 2 : 1;
    LDPC_TRY_CUDA(cudaMemsetAsync(w.count, 0, sizeof(unsigned) * p->ncodes, s));
    LDPC_TRY_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned), s));
    const unsigned fb = (unsigned)ceil_div(F, 256);
    mixed_count<<<fb, 256, 0, s>>>(d_frame_code, F, p->ncodes, w.count, d_iters, d_ok);
    mixed_offsets<<<1, 32, 0, s>>>(w.count, p->d_desc, p->ncodes, G, p->cfg.groups_per_item, w.start,
                                   w.item_off, w.fill);
    mixed_scatter<<<fb, 256, 0, s>>>(d_frame_code, F, p->ncodes, w.start, w.fill, w.sorted);
    const bool syn = early_stop && max_iters >= 2;
    MixedFn fn = pick_mixed(p->fp16, syn);
    int sms = 0, per_sm = 0;
    LDPC_TRY(sm_count(&sms));
    LDPC_TRY(kernel_setup((const void *)fn, kMixThreads, p->smem, &per_sm));
    if (per_sm < 1) return fail(LDPC_ENOTSUP, "mixed kernel cannot be resident");
    MixedArgs a;
    a.desc = p->d_desc;
    a.ncodes = p->ncodes;
    a.item_off = w.item_off;
    a.start = w.start;
    a.count = w.count;
    a.sorted = w.sorted;
    a.llr_off = d_llr_off;
    a.hard_off = d_hard_off;
    a.llr = d_llr;
    a.post = d_post;
    a.hard = d_hard;
    a.iters = d_iters;
    a.ok = d_ok;
    a.counter = w.counter;
    a.T_iters = max_iters;
    a.gpi = p->cfg.groups_per_item;
    a.clip2 = clip_log2(clip);
    const int grid = sms * std::min(per_sm, p->cfg.ctas_per_sm);
    fn<<<grid, kMixThreads, p->smem, s>>>(a);
    LDPC_TRY_CUDA(cudaGetLastError());
    return LDPC_OK;
}

int ldpc_mixed_autotune(ldpc_mixed *p, const int32_t *d_frame_code, const int64_t *d_llr_off,
                        const int64_t *d_hard_off, const float *d_llr, int32_t F, int32_t max_iters,
                        int32_t early_stop, float clip, float *d_post, uint32_t *d_hard,
                        int32_t *d_iters, uint8_t *d_ok, void *d_work, size_t work_bytes,
                        int32_t reps, ldpc_stream_t stream, ldpc_mixed_config *chosen) {
    if (!p || reps < 1) return fail(LDPC_EINVAL, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const ldpc_mixed_config start = p->cfg;
    std::vector<ldpc_mixed_config> cands;
    for (int order = 0; order <= 1; ++order)
        for (int gpi : {1, 2, 4})
            for (int cps : {1, 2}) cands.push_back({order, gpi, cps});
    cudaEvent_t e0, e1;
    LDPC_TRY_CUDA(cudaEventCreate(&e0));
    LDPC_TRY_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    ldpc_mixed_config best_cfg = start;
    int st = LDPC_OK;
    for (const ldpc_mixed_config &cand : cands) {
        if ((st = ldpc_mixed_set_config(p, &cand)) != LDPC_OK) break;
        // one untimed run, then `reps` timed runs
        if ((st = ldpc_decode_mixed(p, d_frame_code, d_llr_off, d_hard_off, d_llr, F, max_iters, early_stop, clip,
                                    d_post, d_hard, d_iters, d_ok, d_work, work_bytes, stream)) != LDPC_OK)
            break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == LDPC_OK; ++r)
            st = ldpc_decode_mixed(p, d_frame_code, d_llr_off, d_hard_off, d_llr, F, max_iters, early_stop, clip,
                                   d_post, d_hard, d_iters, d_ok, d_work, work_bytes, stream);
        cudaEventRecord(e1, s);
        if (st != LDPC_OK) break;
        const cudaError_t err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) {
            st = cuda_fail(err, "cudaEventSynchronize(autotune)");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_cfg = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LDPC_OK) {
        ldpc_mixed_set_config(p, &start);
        return st;
    }
    LDPC_TRY(ldpc_mixed_set_config(p, &best_cfg));
    if (chosen) *chosen = best_cfg;
    return LDPC_OK;
}

}  // extern "C"

// Core of the on-chip decoders (K5 resident, K6 mixed): the shared-memory
// layout of one frame group, the check, bit and syndrome passes, the team
// abstractions and decode_group, which decodes one group of G frames.  The
// file comment of decode_resident.cu describes the layout and the schedule.
#pragma once

#include <algorithm>

#include "check_math.cuh"
#include "ldpc_internal.h"

namespace ldpc {

struct ResArgs {
    const float *llr;
    int32_t F, n, npad, m, NW, T_iters, early_stop;
    float clip2;
    const uint32_t *edges;  // [CPT * DCW][T]
    float *post;
    uint32_t *hard;
    int32_t *iters;
    uint8_t *ok;
    unsigned *counter;
};

using KernelFn = void (*)(ResArgs);

// Resident kernels with planes of 2^pl words fixed at compile time (pl =
// 10..13) for regular codes (three edges per bit) with binary16 messages and
// rows of 6, 9 or 12 edges; null for other pl.  Instantiated per row weight
// in rows6.cu, rows9.cu and rows12.cu.
KernelFn resident_fixed_rows6(int pl, bool syn);
KernelFn resident_fixed_rows9(int pl, bool syn);
KernelFn resident_fixed_rows12(int pl, bool syn);

namespace {

constexpr int kResVPT = 16;       // bits per thread
constexpr int kResMaxThreads = 512;
constexpr size_t kSmemLimit = 226 * 1024;  // dynamic shared memory per CTA we allow ourselves
constexpr int kResSlots = 4;      // message slots per bit (column degree <= 4)
constexpr int kResSlotsWide = 9;  // ... for the wide-column instances (degree <= 9)
constexpr uint32_t kNoSlot = 0xFFFFu;

// Row shapes: padded row degree and checks per thread (about 48 edges/thread).
struct Shape {
    int dc, cpt;
};
constexpr Shape kShapes[] = {{6, 8}, {9, 6}, {12, 4}, {16, 3}};


// 32-bit shared-memory accesses (addresses in the shared window).  Stores
// are volatile and clobber memory, so they keep their order with each other
// and with the barriers.  Loads are plain (not volatile) asm: the compiler may
// schedule them early, which the passes allow because within a pass no
// location is both written and read by different accesses (each message
// belongs to one check, and L or R are only read).  A load may not move
// across a barrier: its address is derived from the plane bases, which are
// redefined after every barrier (Smem::fence).
__device__ __forceinline__ float lds_f(uint32_t a) {
    float v;
    asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u(uint32_t a) {
    uint32_t v;
    asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_f(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void sts_u(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
// The two frames' values of one bit (8-byte aligned), in one access.
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
    float2 v;
    asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_f2(uint32_t a, float x, float y) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x), "f"(y) : "memory");
}

// Planar shared-memory layout of one frame group (see the file comment):
// NE message planes, then the totals L, then (regular codes) the channel LLRs
// R, each a plane of P entries of G floats (the G frames of a bit adjacent,
// so a two-frame group reads or writes a bit's pair in one 8-byte access).  Regular codes (three edges per bit) need three message
// planes and keep R on chip, which frees the registers that would hold it.
// Regular codes keep a row of 32 spare words right after the message planes:
// a thread's unused check slots point there (slot NE P + lane), so every
// thread runs all its check slots without a branch; such a dummy check reads
// real totals (bits 0..31), writes only its spare word, and is left out of
// every syndrome.
constexpr uint32_t kDummyBytes = 128;

template <bool REG, int NSL = kResSlots>
struct Planes {
    static constexpr int NE = REG ? 3 : NSL;
    static constexpr bool RSM = REG;
};

// PL > 0: planes of 2^PL words known at compile time, so that every plane
// offset is an immediate of the shared-memory instruction and one base
// register serves all planes of a bit; PL = 0: the plane size is a run-time
// value.
template <class MsgT, int G, bool REG, int PL = 0, int NSL = kResSlots>
struct Smem {
    static constexpr int NE = Planes<REG, NSL>::NE;  // message planes
    uint32_t e0;      // shared address of message plane 0
    uint32_t l0_;     // shared address of the first total plane (PL = 0)
    uint32_t plane_;  // bytes per plane, 4 P (PL = 0)
    uint32_t pmask_;  // P - 1 (PL = 0)
    __device__ uint32_t plane() const {
        if constexpr (PL > 0) return 4u << PL;
        else return plane_;
    }
    __device__ uint32_t pmask() const {
        if constexpr (PL > 0) return (1u << PL) - 1u;
        else return pmask_;
    }
    __device__ uint32_t l0() const {
        if constexpr (PL > 0) return e0 + NE * (4u << PL) + (REG ? kDummyBytes : 0);
        else return l0_;
    }
    __device__ uint32_t eaddr(uint32_t s) const { return e0 + 4u * s; }
    __device__ uint32_t dummy_slot() const { return NE * (pmask() + 1u); }
    __device__ uint32_t laddr(uint32_t s, int i) const { return l0() + 4u * (G * (s & pmask()) + i); }
    __device__ uint32_t eb(int v, int r) const { return e0 + r * plane() + 4u * v; }
    __device__ uint32_t lb(int v, int i) const { return l0() + 4u * (G * v + i); }
    __device__ uint32_t rb(int v, int i) const { return l0() + G * plane() + 4u * (G * v + i); }
    // after a barrier: the bases become new values to the compiler, so no
    // shared load of the next pass can be placed before the barrier
    __device__ void fence() { asm volatile("" : "+r"(e0), "+r"(l0_)); }
};

template <class MsgT, int G, bool REG, int NSL = kResSlots>
__host__ __device__ __forceinline__ size_t group_bytes(int npad) {
    return (size_t)(Planes<REG, NSL>::NE + G + (Planes<REG, NSL>::RSM ? G : 0)) * 4u * npad + (REG ? kDummyBytes : 0);
}

__device__ __forceinline__ uint32_t slot_of(const uint32_t *w, int j) {
    return (j & 1) ? (w[j >> 1] >> 16) : (w[j >> 1] & 0xFFFFu);
}

// Check pass over the thread's checks, rows of exactly DC edges (REG) or of
// at most DC edges with unused slots marked kNoSlot.  Updates the messages in
// place.  With SYN, also returns bit i set when frame i has a check that the
// hard decisions z = [L >= 0] (L as left by the last bit pass) do not satisfy.
template <class MsgT, int G, int DC, int CPT, bool REG, bool SYN, class SM>
__device__ __forceinline__ uint32_t check_pass(const uint32_t (&idx)[CPT][(DC + 1) / 2],
                                               const SM &sm, float clip2) {
    using EV = EVec<MsgT, G>;
    using LV = Lanes<G>;
    using V = typename LV::T;
    const V zero = LV::splat(0.f);
    uint32_t zacc[G];
#pragma unroll
    for (int i = 0; i < G; ++i) zacc[i] = 0;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        if (!REG && (idx[k][0] & 0xFFFFu) == kNoSlot) continue;  // no check in this slot
        uint32_t slot[DC];
#pragma unroll
        for (int j = 0; j < DC; ++j) slot[j] = slot_of(idx[k], j);
        V u[DC];
        uint32_t xbits[DC][G], sacc[G], zsgn[G];
        int d = 0;
#pragma unroll
        for (int i = 0; i < G; ++i) sacc[i] = zsgn[i] = 0;
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (REG || slot[j] != kNoSlot) {
                ++d;
                float Lf[G], uf[G];
#pragma unroll
                if constexpr (G == 2) {
                    const float2 t = lds_f2(sm.laddr(slot[j], 0));
                    Lf[0] = t.x;
                    Lf[G - 1] = t.y;
                } else {
                    for (int i = 0; i < G; ++i) Lf[i] = lds_f(sm.laddr(slot[j], i));
                }
                const V x = EV::sub_from(LV::make(Lf), lds_u(sm.eaddr(slot[j])));  // Eq. 6 rearranged
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    if (SYN) zsgn[i] ^= __float_as_uint(Lf[i]);  // bit 31: parity of [L < 0]
                    xbits[j][i] = __float_as_uint(LV::get(x, i));
                    sacc[i] ^= xbits[j][i];
                    uf[i] = ex2_approx(-fminf(fabsf(LV::get(x, i)), clip2));
                }
                u[j] = LV::make(uf);
            } else {
                u[j] = zero;  // identity for the pair products
#pragma unroll
                for (int i = 0; i < G; ++i) xbits[j][i] = 0u;
            }
        }
        // parity of z = [L >= 0] over the row = d + parity of [L < 0] (the bit
        // pass leaves no -0, so the sign bit is exactly [L < 0])
        const bool real = !REG || slot[0] < sm.dummy_slot();
        if (SYN && real)
#pragma unroll
            for (int i = 0; i < G; ++i) zacc[i] |= (zsgn[i] >> 31) ^ (uint32_t)(d & 1);
        // (-1)^d folded into the accumulated sign bit
#pragma unroll
        for (int i = 0; i < G; ++i) sacc[i] ^= (uint32_t)(d & 1) << 31;
        EvOdV<G> loo[DC];  // leave-one-out pairs
        evod_leave_one_out<G, DC>(u, loo);
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (REG || slot[j] != kNoSlot) {
                float rc[G], mag[G];
                uint32_t sgn[G];
#pragma unroll
                for (int i = 0; i < G; ++i) rc[i] = rcp_approx(LV::get(loo[j].o, i));
                const V ratio = LV::mul(loo[j].e, LV::make(rc));
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    mag[i] = fminf(lg2_approx(LV::get(ratio, i)), clip2);
                    sgn[i] = sacc[i] ^ xbits[j][i];
                }
                sts_u(sm.eaddr(slot[j]), EV::signed_word(mag, sgn));
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
template <class MsgT, int G, int DC, int CPT, bool REG, class SM>
__device__ __forceinline__ uint32_t syndrome_pass(const uint32_t (&idx)[CPT][(DC + 1) / 2],
                                                  const SM &sm) {
    uint32_t bad = 0;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        uint32_t par = 0;
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            const uint32_t s = slot_of(idx[k], j);
            if (s == kNoSlot || (REG && s >= sm.dummy_slot())) continue;
#pragma unroll
            if constexpr (G == 2) {
                const float2 t = lds_f2(sm.laddr(s, 0));
                par ^= (uint32_t)(t.x >= 0.f) | ((uint32_t)(t.y >= 0.f) << 1);
            } else {
                for (int i = 0; i < G; ++i) par ^= (uint32_t)(lds_f(sm.laddr(s, i)) >= 0.f) << i;
            }
        }
        bad |= par;  // a check with odd parity is unsatisfied
    }
    return bad;
}

// Bit pass (Eq. 7): L_v = R_v + the bit's messages in ascending edge order;
// frames not in `active` keep their L_v.  REG codes have exactly three edges
// per bit and R on chip; otherwise all four planes are summed (unused slots
// hold 0) and R comes from registers.
template <class MsgT, int G, bool REG, bool SYN, int NR, class SM>
__device__ __forceinline__ void bit_pass(const float (&R)[NR][G], const SM &sm, int n,
                                         int tid, int T, uint32_t active) {
    using EV = EVec<MsgT, G>;
    using LV = Lanes<G>;
    constexpr int NS = SM::NE;
#pragma unroll
    for (int k = 0; k < kResVPT; ++k) {
        const int v = tid + k * T;
        if (v < n) {
            float r[G];
            if constexpr (REG && G == 2) {
                const float2 t = lds_f2(sm.rb(v, 0));
                r[0] = t.x;
                r[G - 1] = t.y;
            } else {
#pragma unroll
                for (int i = 0; i < G; ++i) r[i] = REG ? lds_f(sm.rb(v, i)) : R[REG ? 0 : k][i];
            }
            typename LV::T L = LV::make(r);
#pragma unroll
            for (int q = 0; q < NS; ++q) L = EV::add_to(L, lds_u(sm.eb(v, q)));
            if (SYN) L = LV::add(L, LV::splat(0.f));  // no -0: z = [L >= 0] by sign
            if (G == 2 && active == 3u) {  // both frames still running: one store
                sts_f2(sm.lb(v, 0), LV::get(L, 0), LV::get(L, G - 1));
            } else {
#pragma unroll
                for (int i = 0; i < G; ++i)
                    if ((active >> i) & 1u) sts_f(sm.lb(v, i), LV::get(L, i));
            }
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

// Where the G frames of a group come from and go to (null llr = no frame).
template <int G>
struct ResIO {
    const float *llr_[G];
    float *post_[G];
    uint32_t *hard_[G];
    int32_t *iters_[G];
    uint8_t *ok_[G];
    __device__ bool exists(int i) const { return llr_[i] != nullptr; }
    __device__ const float *llr(int i) const { return llr_[i]; }
    __device__ float *post(int i) const { return post_[i]; }
    __device__ uint32_t *hard(int i) const { return hard_[i]; }
    __device__ int32_t *iters(int i) const { return iters_[i]; }
    __device__ uint8_t *ok(int i) const { return ok_[i]; }
};

// Decodes one group of G frames with the team's threads: load R, iterate
// (check pass, bit pass), final syndrome, outputs.  Ends with a team barrier.
template <class MsgT, int G, int DC, int CPT, bool REG, bool SYN, class Team, class IO, class SM>
__device__ __forceinline__ void decode_group(const Team &tm, const uint32_t (&idx)[CPT][(DC + 1) / 2],
                                             const SM &sm_in, int n, int npad,
                                             const IO &io, int T_iters, float clip2) {
    SM sm = sm_in;  // local copy: its bases are fenced at every barrier
    const int tid = tm.tid(), T = tm.size();
    const int lane = threadIdx.x & 31;
    uint32_t exists = 0;
#pragma unroll
    for (int i = 0; i < G; ++i) exists |= (uint32_t)io.exists(i) << i;

    // channel LLRs (log2 units) into shared memory (REG) or registers, and
    // L_v = R_v; messages 0.  All of a thread's loads are issued before its
    // first shared store (a store is ordered with every memory access).
    const float *src[G];
#pragma unroll
    for (int i = 0; i < G; ++i) src[i] = ((exists >> i) & 1u) ? io.llr(i) : nullptr;
    constexpr int NR = REG ? 1 : kResVPT;
    float R[NR][G], Rv[kResVPT][G];
#pragma unroll
    for (int k = 0; k < kResVPT; ++k) {
        const int v = tid + k * T;
#pragma unroll
        for (int i = 0; i < G; ++i) Rv[k][i] = (v < n && src[i]) ? src[i][v] * kLog2e : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kResVPT; ++k) {
        const int v = tid + k * T;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            if (!REG) R[REG ? 0 : k][i] = Rv[k][i];
            if (G == 1 && v < n) {
                sts_f(sm.lb(v, i), Rv[k][i]);
                if (REG) sts_f(sm.rb(v, i), Rv[k][i]);
            }
        }
        if (G == 2 && v < n) {
            sts_f2(sm.lb(v, 0), Rv[k][0], Rv[k][G - 1]);
            if (REG) sts_f2(sm.rb(v, 0), Rv[k][0], Rv[k][G - 1]);
        }
    }
    for (int w = tid; w < SM::NE * npad; w += T) sts_u(sm.e0 + 4u * w, 0u);
    { tm.sync(); sm.fence(); }

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
            sm.fence();
            if (!active) break;
        } else {
            check_pass<MsgT, G, DC, CPT, REG, false>(idx, sm, clip2);
            { tm.sync(); sm.fence(); }
        }
        bit_pass<MsgT, G, REG, SYN>(R, sm, n, tid, T, active);
        { tm.sync(); sm.fence(); }
    }
    if (active) {  // frames that ran every iteration: syndrome of the final z
        const uint32_t bad = syndrome_pass<MsgT, G, DC, CPT, REG>(idx, sm);
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const int any_bad = tm.any((int)((bad >> i) & 1u));
            if ((active >> i) & 1u) {
                it_done[i] = T_iters;
                if (!any_bad) okm |= 1u << i;
            }
        }
        sm.fence();
    }
    // outputs: total LLRs (natural units), packed hard decisions, counts
    float *post[G];
    uint32_t *hard[G];
    const float *in0[G];  // with no iterations the posterior is the input itself
#pragma unroll
    for (int i = 0; i < G; ++i) {
        post[i] = ((exists >> i) & 1u) ? io.post(i) : nullptr;
        hard[i] = ((exists >> i) & 1u) ? io.hard(i) : nullptr;
        in0[i] = post[i] && T_iters == 0 ? io.llr(i) : nullptr;
    }
#pragma unroll
    for (int k = 0; k < kResVPT; ++k) {
        const int v = tid + k * T;
        const int v0 = v - lane;
        float Lo[G];
        if constexpr (G == 2) {
            const float2 t = v < n ? lds_f2(sm.lb(v, 0)) : make_float2(0.f, 0.f);
            Lo[0] = t.x;
            Lo[G - 1] = t.y;
        } else {
#pragma unroll
            for (int i = 0; i < G; ++i) Lo[i] = v < n ? lds_f(sm.lb(v, i)) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const float L = Lo[i];
            const uint32_t word = __ballot_sync(0xffffffffu, v < n && L >= 0.f);
            if (post[i] && v < n) post[i][v] = in0[i] ? in0[i][v] : L * kLn2;
            if (hard[i] && lane == 0 && v0 < n) hard[i][v0 >> 5] = word;
        }
    }
    if (tid == 0)
#pragma unroll
        for (int i = 0; i < G; ++i)
            if ((exists >> i) & 1u) {
                if (int32_t *it = io.iters(i)) *it = it_done[i];
                if (uint8_t *okp = io.ok(i)) *okp = (uint8_t)((okm >> i) & 1u);
            }
    { tm.sync(); sm.fence(); }
}

template <class MsgT, int G, bool REG, int PL = 0, int NSL = kResSlots>
__device__ __forceinline__ Smem<MsgT, G, REG, PL, NSL> smem_at(unsigned char *base, int npad) {
    Smem<MsgT, G, REG, PL, NSL> sm;
    sm.e0 = (uint32_t)__cvta_generic_to_shared(base);
    sm.plane_ = 4u * (uint32_t)npad;
    sm.pmask_ = (uint32_t)npad - 1u;
    sm.l0_ = sm.e0 + Planes<REG, NSL>::NE * sm.plane_ + (REG ? kDummyBytes : 0);
    return sm;
}

template <class MsgT, int G, int DC, int CPT, bool REG, bool SYN, int PL = 0, int NSL = kResSlots>
__global__ void __launch_bounds__(kResMaxThreads)
resident_kernel(ResArgs a) {
    constexpr int DCW = (DC + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem<MsgT, G, REG, PL, NSL> sm = smem_at<MsgT, G, REG, PL, NSL>(smem_raw, a.npad);
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
        ResIO<G> io;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const int64_t f = (int64_t)grp * G + i;
            const bool ex = f < a.F;
            io.llr_[i] = ex ? a.llr + f * a.n : nullptr;
            io.post_[i] = ex && a.post ? a.post + f * a.n : nullptr;
            io.hard_[i] = ex && a.hard ? a.hard + f * a.NW : nullptr;
            io.iters_[i] = ex && a.iters ? a.iters + f : nullptr;
            io.ok_[i] = ex && a.ok ? a.ok + f : nullptr;
        }
        decode_group<MsgT, G, DC, CPT, REG, SYN>(BlockTeam{}, idx, sm, a.n, a.npad, io, a.T_iters, a.clip2);
    }
}

template <int DC, int CPT>
KernelFn resident_fixed_pick(int pl, bool syn) {
    switch (pl) {
        case 10: return syn ? resident_kernel<__half, 2, DC, CPT, true, true, 10> : resident_kernel<__half, 2, DC, CPT, true, false, 10>;
        case 11: return syn ? resident_kernel<__half, 2, DC, CPT, true, true, 11> : resident_kernel<__half, 2, DC, CPT, true, false, 11>;
        case 12: return syn ? resident_kernel<__half, 2, DC, CPT, true, true, 12> : resident_kernel<__half, 2, DC, CPT, true, false, 12>;
        case 13: return syn ? resident_kernel<__half, 2, DC, CPT, true, true, 13> : resident_kernel<__half, 2, DC, CPT, true, false, 13>;
        default: return nullptr;
    }
}

}  // namespace
}  // namespace ldpc

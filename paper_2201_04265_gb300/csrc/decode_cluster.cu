// K9: cluster-resident decoder for quasi-cyclic codes whose frames do not fit
// one SM.
//
// The same flooding sum-product iteration as the plain decoder (Sec. II-B,
// Eqs. 5-8, Algorithm 1's schedule) and the same arithmetic (check_math.cuh)
// in the same order, so the results are the plain decoder's bits.  A thread
// block cluster of C CTAs (C = 2, 4 or 8, one per SM) keeps a group of G
// frames on chip for all iterations: HBM is read for the channel LLRs and
// written for the outputs only.  This is the on-chip form of the paper's node
// split (Algorithm 1: each process owns part of the check and bit nodes and
// exchanges messages every half iteration): the CTAs own the nodes, and the
// exchange is a read of a peer CTA's shared memory.
//
// Quasi-cyclic structure.  H is an mb x nb array of z x z circulants; base
// entry b = (i, j, s) connects check i z + r to bit j z + (r + s) mod z.  CTA k
// owns whole base rows (their z checks each and the messages of their
// entries) and whole base columns (their z bits each), chosen on the host to
// keep as many entries as possible inside one CTA (partition_base below):
//   E[e][z]  one message plane per entry of its rows, binary16 pairs of two
//            frames (G = 2) or FP32 (G = 1), rows in ascending order
//   L[w][z]  one plane of total LLRs per column, float (G = 1) or float2
// The 32 lanes of a warp update 32 consecutive checks of one base row (or
// bits of one base column).  At every step they read 32 consecutive words of
// one plane of one CTA (the circulant shift only rotates the run within the
// plane).  Measured on GB300, reads from a peer CTA's shared memory run at
// about 14 bytes per clock per SM and local ones at about 100, so the bytes
// that cross CTAs bound this kernel: the partition keeps about 60 % of the
// entries of the 46 x 68 workload code inside one CTA of four.
//
// Per iteration: check pass (each warp's check items: gather L from the
// columns' owners, E from local planes, Eq. 5, store E), cluster barrier, bit
// pass (each warp's bit items: R_v plus the bit's messages in ascending base
// row order, read from the rows' owners, Eq. 7, store L), cluster barrier.
// The channel LLRs R are re-read from global memory (L2) in every bit pass;
// the group's LLR rows stay in L2 while it is decoded.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <random>
#include <tuple>

#include "check_math.cuh"
#include "ldpc_internal.h"

namespace ldpc {
namespace {

constexpr int kClThreads = 512;
constexpr int kClWarps = kClThreads / 32;
constexpr int kClMaxRow = 16;               // widest base row of the instances
constexpr int kBitChunk = 4;                // message loads of a bit issued together
constexpr size_t kClSmemLimit = 227 * 1024;  // dynamic shared memory per CTA

// Table blob (int32 words), copied into every CTA's shared memory.
//   header [16]: z, C, words, -, then the word offset of each CTA's section
//                and of the end of the last one
//   section of CTA k [16 header words, then arrays at the offsets given,
//   counted from the section's start; each CTA copies only its own section]:
//     crow   rows x 2: first local message plane, row weight (base rows of
//            CTA k ascending; the row's entries occupy consecutive planes)
//     cent   entries of those rows x 4, ascending column within a row (the
//            code's evaluation order): owner CTA of the column, its total
//            plane in the owner, shift s, 0
//     bcol   columns x 4: base column j, total plane, first and end index in
//            bent (base columns of CTA k ascending)
//     bent   entries of those columns x 4, ascending row (ascending edge
//            index): owner CTA of the row, the entry's message plane in the
//            owner, shift s, 0
//     cptr   kClWarps + 1, citems: check items (row ordinal << 16 | q)
//     bptr   kClWarps + 1, bitems: bit items (column ordinal << 16 | q)
enum { kHZ, kHC, kHWords, kHSec = 4, kHeader = 16 };
enum { kSRows, kSCols, kSNentC, kSNentB, kSCRow, kSCEnt, kSBCol, kSBEnt, kSCPtr, kSCItems, kSBPtr, kSBItems,
       kSecHeader = 16 };

// ------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Cluster barrier: every thread of every CTA of the cluster arrives; release
// / acquire order the shared-memory writes before it with the reads after it.
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The shared::cluster address of the same word in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cl_map(uint32_t a, uint32_t rank) {
    uint32_t d;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(rank));
    return d;
}
// The generic address of the same shared-memory byte in CTA `rank`: remote
// reads through generic addresses need no shared-window conversion per load.
__device__ __forceinline__ uint64_t cl_map64(const void *p, uint32_t rank) {
    uint64_t d;
    asm("mapa.u64 %0, %1, %2;" : "=l"(d) : "l"(p), "r"(rank));
    return d;
}
// Loads (plain asm: schedulable within a pass, never across a barrier: their
// addresses come from shared tables or bases read after it) and stores
// (volatile, ordered with the barriers).
__device__ __forceinline__ float ldg_f(uint64_t a) {
    float v;
    asm("ld.f32 %0, [%1];" : "=f"(v) : "l"(a));
    return v;
}
__device__ __forceinline__ float2 ldg_f2(uint64_t a) {
    float2 v;
    asm("ld.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(a));
    return v;
}
__device__ __forceinline__ uint32_t ldg_u32(uint64_t a) {
    uint32_t v;
    asm("ld.u32 %0, [%1];" : "=r"(v) : "l"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
    uint32_t v;
    asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
    float2 v;
    asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ float lds_f(uint32_t a) {
    float v;
    asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sts_f(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void sts_f2(uint32_t a, float2 v) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void atom_or_cluster(uint32_t a, uint32_t v) {
    asm volatile("atom.shared::cluster.or.b32 _, [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ldc_u32_volatile(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

// Message planes: 4 bytes per (entry, lane) -- a binary16 pair of two frames
// or one FP32 message.
template <class MsgT, int G>
struct ClMsg {
    static constexpr uint32_t B = 4;
    __device__ static uint32_t ld(uint32_t a) { return lds_u32(a); }
    __device__ static uint32_t ldg(uint64_t a) { return ldg_u32(a); }
    __device__ static void st(uint32_t a, uint32_t w) { sts_u32(a, w); }
};

// Total LLRs of G frames at one bit: float (G = 1) or float2.
template <int G>
struct ClL;
template <>
struct ClL<1> {
    __device__ static float ldg(uint64_t a) { return ldg_f(a); }
    __device__ static float ld(uint32_t a) { return lds_f(a); }
    __device__ static void st(uint32_t a, float v) { sts_f(a, v); }
};
template <>
struct ClL<2> {
    __device__ static float2 ldg(uint64_t a) { return ldg_f2(a); }
    __device__ static float2 ld(uint32_t a) { return lds_f2(a); }
    __device__ static void st(uint32_t a, float2 v) { sts_f2(a, v); }
};

// This CTA's plane bases (shared addresses) and its place in the cluster.
struct ClCtx {
    uint32_t e;      // message plane 0
    uint32_t l;      // total plane 0
    uint32_t rank;   // CTA rank in the cluster
    uint32_t z;      // lifting size
    // after a barrier: the bases become new values to the compiler, so no
    // shared load of the next pass is hoisted above the barrier
    __device__ void fence() { asm volatile("" : "+r"(e), "+r"(l)); }
};

// A 64-bit generic address held in an int4 table entry (x, y).
__device__ __forceinline__ uint64_t tab_addr(const int4 &en) {
    return ((uint64_t)(uint32_t)en.y << 32) | (uint32_t)en.x;
}

// Per-CTA address tables, built in shared memory when the kernel starts from
// the section of the blob (the peers' planes mapped once, generic 64-bit
// addresses in x, y): entry c of the check table holds the address of bit
// (j, s) in its column's plane in the owner CTA, and z - s in z, so that lane
// r reads bit (j, (r + s) mod z) at addr + 4 G r, less one plane width when
// r >= z - s.  Entry k of the bit table holds the address of the message
// plane of check row i in the owner CTA, less s words, and s in z, so that
// lane t reads the message of check (i, (t - s) mod z) at addr + 4 t, plus one
// plane width when t < s.

// Check-node update (Eq. 5) of the 32 checks (i, r) of one warp item, rows of
// d <= D inputs taken in ascending base column order (the code's evaluation
// order; check table entries c0 .. c0+d-1, local message planes likewise):
// gather, leave-one-out pairs, new messages stored in place.  With SYN,
// returns bit i set when the hard decisions z = [L >= 0] of frame i (L as
// left by the last bit pass) violate this check.
template <class MsgT, int G, int D, int DLO, bool SYN>
__device__ __forceinline__ uint32_t cl_check_item(const ClCtx &cx, const int4 *ctab, int c0, int d, uint32_t r,
                                                  float clip2) {
    using EV = EVec<MsgT, G>;
    using LV = Lanes<G>;
    using V = typename LV::T;
    using M = ClMsg<MsgT, G>;
    const uint32_t ea = cx.e + ((uint32_t)c0 * cx.z + r) * M::B;  // position 0's message
    const uint32_t estep = cx.z * M::B;
    const int32_t roff = (int32_t)(r * (4u * G)), wrap = (int32_t)(cx.z * (4u * G));
    V u[D];
    uint32_t smask[G], zpar[G];
#pragma unroll
    for (int i = 0; i < G; ++i) smask[i] = zpar[i] = 0;
#pragma unroll
    for (int p = 0; p < D; ++p) {
        float uf[G];
#pragma unroll
        for (int i = 0; i < G; ++i) uf[i] = 0.f;  // positions beyond d: the identity
        if (p < DLO || p < d) {  // the instance serves DLO < d <= D
            const int4 en = ctab[c0 + p];
            const int32_t off = r >= (uint32_t)en.z ? roff - wrap : roff;
            const V Lv = ClL<G>::ldg(tab_addr(en) + (int64_t)off);
            const V x = EV::sub_from(Lv, M::ld(ea + (uint32_t)p * estep));  // Eq. 6 rearranged
#pragma unroll
            for (int i = 0; i < G; ++i) {
                if (SYN) zpar[i] ^= (uint32_t)(LV::get(Lv, i) >= 0.f);
                const float xi = LV::get(x, i);
                smask[i] |= (__float_as_uint(xi) >> 31) << p;
                uf[i] = ex2_approx(-fminf(fabsf(xi), clip2));
            }
        }
        u[p] = LV::make(uf);
    }
    uint32_t sall[G];
#pragma unroll
    for (int i = 0; i < G; ++i) sall[i] = (uint32_t)(__popc(smask[i]) + d) & 1u;
    EvOdV<G> loo[D];
    evod_leave_one_out<G, D>(u, loo);
#pragma unroll
    for (int p = 0; p < D; ++p) {
        if (p < DLO || p < d) {
            float rc[G], mag[G];
            uint32_t sg[G];
#pragma unroll
            for (int i = 0; i < G; ++i) rc[i] = rcp_approx(LV::get(loo[p].o, i));
            const V ratio = LV::mul(loo[p].e, LV::make(rc));
#pragma unroll
            for (int i = 0; i < G; ++i) {
                mag[i] = fminf(lg2_approx(LV::get(ratio, i)), clip2);
                sg[i] = (sall[i] ^ (smask[i] >> p)) << 31;
            }
            M::st(ea + (uint32_t)p * estep, EV::signed_word(mag, sg));
        }
    }
    uint32_t bad = 0;
    if (SYN)
#pragma unroll
        for (int i = 0; i < G; ++i) bad |= (zpar[i] & 1u) << i;
    return bad;
}

// Syndrome of z = [L >= 0] over one check item (no message update).
template <int G>
__device__ __forceinline__ uint32_t cl_syndrome_item(const ClCtx &cx, const int4 *ctab, int c0, int d,
                                                     uint32_t r) {
    using LV = Lanes<G>;
    const int32_t roff = (int32_t)(r * (4u * G)), wrap = (int32_t)(cx.z * (4u * G));
    uint32_t par = 0;
    for (int p = 0; p < d; ++p) {
        const int4 en = ctab[c0 + p];
        const int32_t off = r >= (uint32_t)en.z ? roff - wrap : roff;
        const typename LV::T Lv = ClL<G>::ldg(tab_addr(en) + (int64_t)off);
#pragma unroll
        for (int i = 0; i < G; ++i) par ^= (uint32_t)(LV::get(Lv, i) >= 0.f) << i;
    }
    return par;
}

// One check item through the instance sized for its row (any D >= d gives
// the same bits: padded positions hold the identity pair).
template <class MsgT, int G, bool SYN>
__device__ __forceinline__ uint32_t cl_check_dispatch(const ClCtx &cx, const int4 *ctab, int c0, int d,
                                                      uint32_t r, float clip2) {
    if (d <= 4) return cl_check_item<MsgT, G, 4, 1, SYN>(cx, ctab, c0, d, r, clip2);
    if (d <= 6) return cl_check_item<MsgT, G, 6, 4, SYN>(cx, ctab, c0, d, r, clip2);
    if (d <= 8) return cl_check_item<MsgT, G, 8, 6, SYN>(cx, ctab, c0, d, r, clip2);
    if (d <= 10) return cl_check_item<MsgT, G, 10, 8, SYN>(cx, ctab, c0, d, r, clip2);
    if (d <= 12) return cl_check_item<MsgT, G, 12, 10, SYN>(cx, ctab, c0, d, r, clip2);
    if (d <= 14) return cl_check_item<MsgT, G, 14, 12, SYN>(cx, ctab, c0, d, r, clip2);
    return cl_check_item<MsgT, G, kClMaxRow, 14, SYN>(cx, ctab, c0, d, r, clip2);
}

// Channel LLRs R_v of G frames in log2 units (0 for a frame that does not
// exist), the same product the plain decoder stores once.
template <int G>
__device__ __forceinline__ typename Lanes<G>::T cl_channel(const float *const (&llr)[G], int64_t v) {
    float r[G];
#pragma unroll
    for (int i = 0; i < G; ++i) r[i] = llr[i] ? __ldg(llr[i] + v) * kLog2e : 0.f;
    return Lanes<G>::make(r);
}

// Bit-node update (Eq. 7) of the 32 bits (j, t) of one warp item: L = R + the
// bit's messages in ascending base row order (ascending edge index, the plain
// decoder's order), each read from the CTA that owns its row; bit table
// entries k0 .. k1-1.  Up to kBitChunk messages are requested together, then
// added in order.  Frames not in `active` keep their L.
template <class MsgT, int G>
__device__ __forceinline__ void cl_bit_item(const ClCtx &cx, const int4 *btab, int k0, int k1, uint32_t la,
                                            uint32_t t, typename Lanes<G>::T L, uint32_t active) {
    using EV = EVec<MsgT, G>;
    using M = ClMsg<MsgT, G>;
    const int32_t toff = (int32_t)(t * M::B), wrap = (int32_t)(cx.z * M::B);
    for (int k = k0; k < k1; k += kBitChunk) {
        uint32_t w[kBitChunk];
#pragma unroll
        for (int u = 0; u < kBitChunk; ++u) {
            if (k + u < k1) {
                const int4 en = btab[k + u];
                const int32_t off = t < (uint32_t)en.z ? toff + wrap : toff;
                w[u] = M::ldg(tab_addr(en) + (int64_t)off);
            }
        }
#pragma unroll
        for (int u = 0; u < kBitChunk; ++u)
            if (k + u < k1) L = EV::add_to(L, w[u]);
    }
    if (active == (1u << G) - 1u) {
        ClL<G>::st(la, L);
    } else {
#pragma unroll
        for (int i = 0; i < G; ++i)
            if ((active >> i) & 1u) sts_f(la + 4u * i, Lanes<G>::get(L, i));
    }
}

struct ClArgs {
    const float *llr;
    int32_t F, n, NW, z, T_iters, C;
    float clip2;
    float *post;
    uint32_t *hard;
    int32_t *iters;
    uint8_t *ok;
    unsigned *counter;
    const int32_t *tab;         // table blob (global memory)
    int32_t sec_words;          // words of the largest section (a multiple of 4)
    uint32_t e_bytes, l_bytes;  // multiples of 16
};

// Every CTA of a cluster runs the same control flow (the same group, the
// same iteration count, the same early-stop decisions from the same flags),
// so all reach every cluster barrier.
template <class MsgT, int G, bool SYN>
__global__ void __launch_bounds__(kClThreads, 1) cluster_kernel(ClArgs a) {
    using LV = Lanes<G>;
    using V = typename LV::T;
    using M = ClMsg<MsgT, G>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // layout: E planes | L planes | control words (flags by iteration parity,
    // group slot) | table blob | check and bit address tables
    ClCtx cx;
    cx.rank = cl_rank();
    int32_t *sec = reinterpret_cast<int32_t *>(smem + a.e_bytes + a.l_bytes + 16);
    {
        const int32_t s0 = __ldg(&a.tab[kHSec + cx.rank]), s1 = __ldg(&a.tab[kHSec + cx.rank + 1]);
        for (int w = tid; w < s1 - s0; w += kClThreads) sec[w] = __ldg(&a.tab[s0 + w]);
        __syncthreads();
    }
    cx.e = (uint32_t)__cvta_generic_to_shared(smem);
    cx.l = cx.e + a.e_bytes;
    cx.z = (uint32_t)a.z;
    const uint32_t ctl = cx.l + a.l_bytes;  // [0], [1]: flags, [2]: group slot
    const int32_t *crow = sec + sec[kSCRow];
    const int4 *cent = reinterpret_cast<const int4 *>(sec + sec[kSCEnt]);
    const int4 *bcol = reinterpret_cast<const int4 *>(sec + sec[kSBCol]);
    const int4 *bent = reinterpret_cast<const int4 *>(sec + sec[kSBEnt]);
    const int c0w = sec[sec[kSCPtr] + warp], c1w = sec[sec[kSCPtr] + warp + 1];
    const int32_t *citems = sec + sec[kSCItems];
    const int g0 = sec[sec[kSBPtr] + warp], g1 = sec[sec[kSBPtr] + warp + 1];
    const int32_t *bitems = sec + sec[kSBItems];
    const int nentc = sec[kSNentC], nentb = sec[kSNentB];
    int4 *ctab = reinterpret_cast<int4 *>(sec + a.sec_words);  // check table, then bit table
    int4 *btab = ctab + nentc;
    for (int c = tid; c < nentc; c += kClThreads) {
        const int4 en = cent[c];  // {owner, plane, s, 0}
        const uint64_t x = cl_map64(smem + a.e_bytes + ((size_t)en.y * cx.z + (uint32_t)en.z) * (4u * G),
                                    (uint32_t)en.x);
        ctab[c] = make_int4((int)(uint32_t)x, (int)(uint32_t)(x >> 32), (int)(cx.z - (uint32_t)en.z), 0);
    }
    for (int k = tid; k < nentb; k += kClThreads) {
        const int4 en = bent[k];  // {owner, plane, s, 0}
        const uint64_t x = cl_map64(smem + (size_t)en.y * cx.z * M::B, (uint32_t)en.x) - (uint64_t)en.z * M::B;
        btab[k] = make_int4((int)(uint32_t)x, (int)(uint32_t)(x >> 32), en.z, 0);
    }
    __syncthreads();
    const int groups = (a.F + G - 1) / G;
    for (;;) {
        if (cx.rank == 0 && tid == 0) sts_u32(ctl + 8, atomicAdd(a.counter, 1u));
        cl_sync();
        cx.fence();
        const int grp = (int)ldc_u32_volatile(cl_map(ctl + 8, 0));
        if (grp >= groups) {
            cl_sync();  // no CTA leaves while a peer may still read its memory
            break;
        }
        const float *llr[G];
        uint32_t exists = 0;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const int64_t f = (int64_t)grp * G + i;
            llr[i] = f < a.F ? a.llr + f * a.n : nullptr;
            exists |= (uint32_t)(f < a.F) << i;
        }
        // messages 0, flags 0, L = R
        for (uint32_t w = tid; w < a.e_bytes / 16; w += kClThreads)
            asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(cx.e + 16u * w), "r"(0u) : "memory");
        if (tid == 0) {
            sts_u32(ctl, 0u);
            sts_u32(ctl + 4, 0u);
        }
        for (int k = g0; k < g1; ++k) {
            const int4 bc = bcol[bitems[k] >> 16];  // {j, plane, k0, k1}
            const uint32_t t = 32u * (bitems[k] & 0xFFFF) + lane;
            const V R = cl_channel<G>(llr, (int64_t)bc.x * cx.z + t);
            ClL<G>::st(cx.l + ((uint32_t)bc.y * cx.z + t) * (4u * G), R);
        }
        cl_sync();
        cx.fence();

        uint32_t active = exists, okm = 0;
        int it_done[G];
#pragma unroll
        for (int i = 0; i < G; ++i) it_done[i] = 0;
        int t = 1;
        for (; t <= a.T_iters; ++t) {
            uint32_t bad = 0;
            for (int k = c0w; k < c1w; ++k) {
                const int rho = citems[k] >> 16;
                bad |= cl_check_dispatch<MsgT, G, SYN>(cx, ctab, crow[2 * rho], crow[2 * rho + 1],
                                                       32u * (citems[k] & 0xFFFF) + lane, a.clip2);
            }
            const bool syn = SYN && t >= 2;  // syndrome of z^(t-1)
            if (syn) {
                const uint32_t wb = __reduce_or_sync(0xffffffffu, bad);
                if (lane == 0 && wb)
                    for (int r = 0; r < a.C; ++r) atom_or_cluster(cl_map(ctl + 4u * (t & 1), (uint32_t)r), wb);
            }
            cl_sync();
            cx.fence();
            if (syn) {
                const uint32_t flags = ldc_u32_volatile(ctl + 4u * (t & 1));
#pragma unroll
                for (int i = 0; i < G; ++i)
                    if (((active >> i) & 1u) && !((flags >> i) & 1u)) {  // z^(t-1) satisfies H z = 0
                        active &= ~(1u << i);
                        it_done[i] = t - 1;
                        okm |= 1u << i;
                    }
                if (!active) break;
            }
            if (SYN && tid == 0) sts_u32(ctl + 4u * ((t + 1) & 1), 0u);  // next iteration's flags
            V Rn{};
            if (g0 < g1) {
                const int4 bc = bcol[bitems[g0] >> 16];
                Rn = cl_channel<G>(llr, (int64_t)bc.x * cx.z + 32u * (bitems[g0] & 0xFFFF) + lane);
            }
            for (int k = g0; k < g1; ++k) {
                const int4 bc = bcol[bitems[k] >> 16];
                const uint32_t tt = 32u * (bitems[k] & 0xFFFF) + lane;
                const V R = Rn;
                if (k + 1 < g1) {
                    const int4 bn = bcol[bitems[k + 1] >> 16];
                    Rn = cl_channel<G>(llr, (int64_t)bn.x * cx.z + 32u * (bitems[k + 1] & 0xFFFF) + lane);
                }
                cl_bit_item<MsgT, G>(cx, btab, bc.z, bc.w, cx.l + ((uint32_t)bc.y * cx.z + tt) * (4u * G), tt, R,
                                     active);
            }
            cl_sync();
            cx.fence();
        }
        if (active) {  // frames that ran every iteration: syndrome of the final z
            uint32_t bad = 0;
            for (int k = c0w; k < c1w; ++k) {
                const int rho = citems[k] >> 16;
                bad |= cl_syndrome_item<G>(cx, ctab, crow[2 * rho], crow[2 * rho + 1],
                                           32u * (citems[k] & 0xFFFF) + lane);
            }
            // slot t & 1 is clear: zeroed at the start of the group or in the
            // last bit pass
            const uint32_t wb = __reduce_or_sync(0xffffffffu, bad);
            if (lane == 0 && wb)
                for (int r = 0; r < a.C; ++r) atom_or_cluster(cl_map(ctl + 4u * (t & 1), (uint32_t)r), wb);
            cl_sync();
            cx.fence();
            const uint32_t flags = ldc_u32_volatile(ctl + 4u * (t & 1));
#pragma unroll
            for (int i = 0; i < G; ++i)
                if ((active >> i) & 1u) {
                    it_done[i] = a.T_iters;
                    if (!((flags >> i) & 1u)) okm |= 1u << i;
                }
        }
        // outputs of this CTA's bits: total LLRs (natural units), packed hard
        // decisions (Eq. 8), and, from rank 0, iteration counts and flags
        for (int k = g0; k < g1; ++k) {
            const int4 bc = bcol[bitems[k] >> 16];
            const uint32_t tt = 32u * (bitems[k] & 0xFFFF) + lane;
            const int64_t v = (int64_t)bc.x * cx.z + tt;
            const V Lv = ClL<G>::ld(cx.l + ((uint32_t)bc.y * cx.z + tt) * (4u * G));
#pragma unroll
            for (int i = 0; i < G; ++i) {
                const float L = LV::get(Lv, i);
                const uint32_t word = __ballot_sync(0xffffffffu, L >= 0.f);
                if ((exists >> i) & 1u) {
                    const int64_t f = (int64_t)grp * G + i;
                    if (a.post) a.post[f * a.n + v] = a.T_iters == 0 ? llr[i][v] : L * kLn2;
                    if (a.hard && lane == 0) a.hard[f * a.NW + ((v - lane) >> 5)] = word;
                }
            }
        }
        if (cx.rank == 0 && tid == 0)
#pragma unroll
            for (int i = 0; i < G; ++i)
                if ((exists >> i) & 1u) {
                    const int64_t f = (int64_t)grp * G + i;
                    if (a.iters) a.iters[f] = it_done[i];
                    if (a.ok) a.ok[f] = (uint8_t)((okm >> i) & 1u);
                }
    }
}

using ClFn = void (*)(ClArgs);

// Binary16 messages: two frames per group (one binary16 pair per message
// word); FP32 messages: one frame per group.
ClFn pick_cluster(bool fp16, bool syn) {
    if (fp16) return syn ? cluster_kernel<__half, 2, true> : cluster_kernel<__half, 2, false>;
    return syn ? cluster_kernel<float, 1, true> : cluster_kernel<float, 1, false>;
}

// ---------------------------------------------------------------- host side --
//
// Partition of the base graph.  CTA k of the cluster owns the base rows R_k
// (their checks, for every lifting index, and the messages of their entries)
// and the base columns C_k (their bits and totals).  An entry (i, j) is read
// within one CTA when i and j have the same owner; otherwise its check reads
// the bit's totals from a peer in the check pass, and its bit reads the
// message from a peer in the bit pass.  Remote reads cost about 14 bytes per
// clock per SM on GB300 against about 100 for local ones, so the partition
// maximises the entries with both ends in one CTA, within the shared memory
// of a CTA (at most ecap entries and lcap columns) and with balanced check
// and bit work.  Simulated annealing over single row or column moves,
// deterministic seed.
struct Partition {
    std::vector<int32_t> row_of, col_of;  // owner CTA of each base row / column
    int32_t internal = -1;                // entries with both ends in one CTA
};

Partition partition_base(const QcInfo &qc, int C, int ecap, int lcap) {
    const int mb = qc.mb, nb = qc.nb;
    std::vector<std::vector<int32_t>> rcols(mb), crows(nb);
    for (int i = 0; i < mb; ++i)
        for (int j = 0; j < nb; ++j)
            if (qc.shift[(size_t)i * nb + j] >= 0) {
                rcols[i].push_back(j);
                crows[j].push_back(i);
            }
    int64_t nnzb = 0;
    for (auto &r : rcols) nnzb += (int64_t)r.size();
    std::mt19937 rng(12345);
    Partition best;
    for (int restart = 0; restart < 4; ++restart) {
        Partition p;
        p.row_of.assign(mb, 0);
        p.col_of.assign(nb, 0);
        std::vector<int64_t> ecount(C, 0), lcount(C, 0), bload(C, 0);
        // start: rows and columns dealt round robin in a random order
        std::vector<int32_t> order(mb);
        for (int i = 0; i < mb; ++i) order[i] = i;
        std::shuffle(order.begin(), order.end(), rng);
        for (int x = 0; x < mb; ++x) {
            const int i = order[x], k = (int)(std::min_element(ecount.begin(), ecount.end()) - ecount.begin());
            p.row_of[i] = k;
            ecount[k] += (int64_t)rcols[i].size();
        }
        order.resize(nb);
        for (int j = 0; j < nb; ++j) order[j] = j;
        std::shuffle(order.begin(), order.end(), rng);
        for (int x = 0; x < nb; ++x) {
            const int j = order[x], k = (int)(std::min_element(lcount.begin(), lcount.end()) - lcount.begin());
            p.col_of[j] = k;
            lcount[k] += 1;
            bload[k] += (int64_t)crows[j].size();
        }
        if (*std::max_element(ecount.begin(), ecount.end()) > ecap ||
            *std::max_element(lcount.begin(), lcount.end()) > lcap)
            continue;
        int64_t internal = 0;
        for (int i = 0; i < mb; ++i)
            for (int j : rcols[i]) internal += p.row_of[i] == p.col_of[j];
        // score: internal entries, minus the excess of the busiest CTA's check
        // and bit work over the mean (half an entry per entry of excess)
        auto score = [&](int64_t in) {
            const double me = (double)nnzb / C;
            return (double)in - 0.5 * (*std::max_element(ecount.begin(), ecount.end()) - me) -
                   0.5 * (*std::max_element(bload.begin(), bload.end()) - me);
        };
        double cur = score(internal);
        const int steps = 40000;
        std::uniform_real_distribution<double> unif(0.0, 1.0);
        for (int s = 0; s < steps; ++s) {
            const double temp = 2.0 * (1.0 - (double)s / steps) + 0.01;
            const bool row = (rng() % (unsigned)(mb + nb)) < (unsigned)mb;
            const int x = row ? (int)(rng() % (unsigned)mb) : (int)(rng() % (unsigned)nb);
            const int from = row ? p.row_of[x] : p.col_of[x];
            const int to = (from + 1 + (int)(rng() % (unsigned)(C - 1))) % C;
            int64_t d = 0;
            if (row) {
                const int64_t deg = (int64_t)rcols[x].size();
                if (ecount[to] + deg > ecap) continue;
                for (int j : rcols[x]) d += (p.col_of[j] == to) - (p.col_of[j] == from);
                ecount[from] -= deg;
                ecount[to] += deg;
                const double nxt = score(internal + d);
                if (nxt >= cur || unif(rng) < std::exp((nxt - cur) / temp)) {
                    p.row_of[x] = to;
                    internal += d;
                    cur = nxt;
                } else {
                    ecount[from] += deg;
                    ecount[to] -= deg;
                }
            } else {
                if (lcount[to] + 1 > lcap) continue;
                const int64_t deg = (int64_t)crows[x].size();
                for (int i : crows[x]) d += (p.row_of[i] == to) - (p.row_of[i] == from);
                lcount[from] -= 1;
                lcount[to] += 1;
                bload[from] -= deg;
                bload[to] += deg;
                const double nxt = score(internal + d);
                if (nxt >= cur || unif(rng) < std::exp((nxt - cur) / temp)) {
                    p.col_of[x] = to;
                    internal += d;
                    cur = nxt;
                } else {
                    lcount[from] += 1;
                    lcount[to] -= 1;
                    bload[from] += deg;
                    bload[to] -= deg;
                }
            }
        }
        p.internal = (int32_t)internal;
        if (p.internal > best.internal) best = p;
    }
    return best;
}

// Table blob of a partition (layout at the top of the file).  Work items are
// dealt to the warps longest first, each to the warp with the least work so
// far (check items cost their row weight, bit items their column weight + 1).
std::vector<int32_t> build_cluster_table(const ldpc_code *c, const Partition &pt, int C, int32_t *max_ent,
                                         int32_t *max_col) {
    const QcInfo &qc = c->qc;
    const int32_t z = qc.z, nq = z / 32;
    // per base entry: row, column, shift, CSR (row-major) order
    std::vector<std::vector<std::pair<int32_t, int32_t>>> rent(qc.mb), cent_(qc.nb);  // (col or row, shift)
    for (int32_t i = 0; i < qc.mb; ++i)
        for (int32_t j = 0; j < qc.nb; ++j) {
            const int16_t s = qc.shift[(size_t)i * qc.nb + j];
            if (s < 0) continue;
            rent[i].emplace_back(j, s);
            cent_[j].emplace_back(i, s);  // ascending i
        }
    // local slots: rows of CTA k in ascending order hold consecutive message
    // planes; columns of CTA k in ascending order hold consecutive total planes
    std::vector<int32_t> lslot(qc.nb), eslot0(qc.mb);
    std::vector<int32_t> nent(C, 0), ncol(C, 0);
    for (int32_t i = 0; i < qc.mb; ++i) {
        const int k = pt.row_of[i];
        eslot0[i] = nent[k];
        nent[k] += (int32_t)rent[i].size();
    }
    for (int32_t j = 0; j < qc.nb; ++j) lslot[j] = ncol[pt.col_of[j]]++;
    *max_ent = *std::max_element(nent.begin(), nent.end());
    *max_col = *std::max_element(ncol.begin(), ncol.end());
    auto deal = [](std::vector<std::pair<int32_t, int32_t>> items) {  // (cost, item)
        std::stable_sort(items.begin(), items.end(), [](auto &x, auto &y) { return x.first > y.first; });
        std::vector<std::vector<int32_t>> per(kClWarps);
        std::vector<int64_t> load(kClWarps, 0);
        for (auto &it : items) {
            const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            per[w].push_back(it.second);
            load[w] += it.first;
        }
        std::vector<int32_t> ptr(1, 0), flat;
        for (auto &p : per) {
            std::sort(p.begin(), p.end());
            flat.insert(flat.end(), p.begin(), p.end());
            ptr.push_back((int32_t)flat.size());
        }
        return std::make_pair(ptr, flat);
    };
    std::vector<int32_t> tab(kHeader, 0);
    int32_t sec_start = 0;
    auto put = [&](const std::vector<int32_t> &v) {  // offset from the section's start
        while (tab.size() % 4) tab.push_back(0);      // 16-byte aligned arrays
        const int32_t at = (int32_t)tab.size() - sec_start;
        tab.insert(tab.end(), v.begin(), v.end());
        return at;
    };
    tab[kHZ] = z;
    tab[kHC] = C;
    for (int k = 0; k < C; ++k) {
        std::vector<int32_t> sec(kSecHeader, 0), crow, cent, bcol, bent;
        std::vector<std::pair<int32_t, int32_t>> ci, bi;
        int32_t rho = 0;
        for (int32_t i = 0; i < qc.mb; ++i) {
            if (pt.row_of[i] != k) continue;
            crow.push_back((int32_t)cent.size() / 4);  // first entry = its local message plane
            crow.push_back((int32_t)rent[i].size());
            for (auto &e : rent[i]) {  // ascending j: the code's evaluation order
                cent.push_back(pt.col_of[e.first]);
                cent.push_back(lslot[e.first]);
                cent.push_back(e.second);
                cent.push_back(0);
            }
            for (int32_t q = 0; q < nq; ++q) ci.emplace_back((int32_t)rent[i].size(), (rho << 16) | q);
            ++rho;
        }
        int32_t omega = 0;
        for (int32_t j = 0; j < qc.nb; ++j) {
            if (pt.col_of[j] != k) continue;
            bcol.push_back(j);
            bcol.push_back(lslot[j]);
            bcol.push_back((int32_t)bent.size() / 4);
            for (auto &e : cent_[j]) {  // ascending i: ascending edge index, the bit sum's order
                const int32_t i = e.first;
                int32_t p = 0;
                while (rent[i][p].first != j) ++p;
                bent.push_back(pt.row_of[i]);
                bent.push_back(eslot0[i] + p);
                bent.push_back(e.second);
                bent.push_back(0);
            }
            bcol.push_back((int32_t)bent.size() / 4);
            for (int32_t q = 0; q < nq; ++q) bi.emplace_back((int32_t)cent_[j].size() + 1, (omega << 16) | q);
            ++omega;
        }
        const auto cd = deal(ci), bd = deal(bi);
        while (tab.size() % 4) tab.push_back(0);
        sec_start = (int32_t)tab.size();
        tab[kHSec + k] = sec_start;
        put(sec);
        const int32_t s0 = sec_start;
        tab[s0 + kSRows] = rho;
        tab[s0 + kSCols] = omega;
        tab[s0 + kSNentC] = (int32_t)cent.size() / 4;
        tab[s0 + kSNentB] = (int32_t)bent.size() / 4;
        tab[s0 + kSCRow] = put(crow);
        tab[s0 + kSCEnt] = put(cent);
        tab[s0 + kSBCol] = put(bcol);
        tab[s0 + kSBEnt] = put(bent);
        tab[s0 + kSCPtr] = put(cd.first);
        tab[s0 + kSCItems] = put(cd.second);
        tab[s0 + kSBPtr] = put(bd.first);
        tab[s0 + kSBItems] = put(bd.second);
    }
    while (tab.size() % 4) tab.push_back(0);
    tab[kHSec + C] = (int32_t)tab.size();
    tab[kHWords] = (int32_t)tab.size();
    return tab;
}

// Checks every index of a table blob against the planes and items it refers
// to (the kernel trusts them): owners below C, total planes below the
// owner's column count, message planes below the owner's entry count, items
// within the rank's rows and columns and within z / 32 lanes groups.
bool cluster_table_valid(const std::vector<int32_t> &tab, int C, int32_t z, int32_t max_ent, int32_t max_col) {
    std::vector<int32_t> ncol(C), nent(C);
    for (int k = 0; k < C; ++k) {
        const int32_t s0 = tab[kHSec + k];
        ncol[k] = tab[s0 + kSCols];
        nent[k] = tab[s0 + kSNentC];
        if (ncol[k] > max_col || nent[k] > max_ent) return false;
    }
    for (int k = 0; k < C; ++k) {
        const int32_t s0 = tab[kHSec + k];
        const int32_t rows = tab[s0 + kSRows], cols = tab[s0 + kSCols];
        const int32_t *crow = &tab[s0 + tab[s0 + kSCRow]], *cent = &tab[s0 + tab[s0 + kSCEnt]];
        const int32_t *bcol = &tab[s0 + tab[s0 + kSBCol]], *bent = &tab[s0 + tab[s0 + kSBEnt]];
        for (int32_t r = 0; r < rows; ++r) {
            if (crow[2 * r] < 0 || crow[2 * r + 1] < 1 || crow[2 * r + 1] > kClMaxRow ||
                crow[2 * r] + crow[2 * r + 1] > nent[k])
                return false;
            for (int32_t p = 0; p < crow[2 * r + 1]; ++p) {
                const int32_t *e = &cent[4 * (crow[2 * r] + p)];
                if (e[0] < 0 || e[0] >= C || e[1] < 0 || e[1] >= ncol[e[0]] || e[2] < 0 || e[2] >= z) return false;
            }
        }
        for (int32_t w = 0; w < cols; ++w) {
            const int32_t *b = &bcol[4 * w];
            if (b[1] != w || b[2] < 0 || b[3] < b[2] || b[3] > tab[s0 + kSNentB]) return false;
            for (int32_t q = b[2]; q < b[3]; ++q) {
                const int32_t *e = &bent[4 * q];
                if (e[0] < 0 || e[0] >= C || e[1] < 0 || e[1] >= nent[e[0]] || e[2] < 0 || e[2] >= z) return false;
            }
        }
        for (int pass = 0; pass < 2; ++pass) {
            const int32_t *ptr = &tab[s0 + tab[s0 + (pass ? kSBPtr : kSCPtr)]];
            const int32_t *it = &tab[s0 + tab[s0 + (pass ? kSBItems : kSCItems)]];
            if (ptr[0] != 0) return false;
            for (int w = 0; w < kClWarps; ++w) {
                if (ptr[w + 1] < ptr[w]) return false;
                for (int32_t x = ptr[w]; x < ptr[w + 1]; ++x)
                    if ((it[x] >> 16) >= (pass ? cols : rows) || (it[x] & 0xFFFF) >= z / 32) return false;
            }
        }
    }
    return true;
}

// The launch shape for one message type: the smallest cluster whose
// partition fits one SM's shared memory per CTA.
ClusterCfg choose_cluster(const ldpc_code *c, bool fp16) {
    ClusterCfg best;
    const int G = fp16 ? 2 : 1;
    const uint32_t mbytes = fp16 ? 4u : 4u;  // a binary16 pair or one FP32 per (entry, lane)
    const int64_t z = c->qc.z;
    int64_t nnzb = 0;
    for (int16_t s : c->qc.shift) nnzb += s >= 0;
    for (int C : {2, 4, 8}) {
        if (c->qc.mb < C || c->qc.nb < C) break;
        // room for the tables (blob + two address tables, about 64 B per
        // entry and 16 per item), then columns first, then entries
        // a CTA's share of the table blob (16 words per entry, 2 per row, 4
        // per column, 1 per item) and of the two address tables (16 B per
        // entry of its rows and of its columns), with slack for imbalance
        const int64_t items = (int64_t)(c->qc.mb + c->qc.nb) * (z / 32);
        const int64_t fixed = 16 + (2 * (64 * nnzb + 8 * c->qc.mb + 16 * c->qc.nb + 4 * items)) / C + 1024;
        const int64_t lcap = ceil_div(c->qc.nb, C) + 2;
        const int64_t lbytes = align256((size_t)(lcap * z * 4 * G));
        const int64_t room = (int64_t)kClSmemLimit - fixed - lbytes;
        if (room <= 0) continue;
        const int64_t ecap = room / (z * mbytes);
        if (ecap * C < nnzb + nnzb / 20) continue;  // needs some slack to partition
        const Partition pt = partition_base(c->qc, C, (int)ecap, (int)lcap);
        if (pt.internal < 0) continue;
        int32_t max_ent = 0, max_col = 0;
        std::vector<int32_t> tab = build_cluster_table(c, pt, C, &max_ent, &max_col);
        if (!cluster_table_valid(tab, C, c->qc.z, max_ent, max_col)) continue;
        ClusterCfg cfg;
        cfg.C = C;
        cfg.G = G;
        cfg.e_bytes = (uint32_t)align256((size_t)max_ent * z * mbytes);
        cfg.l_bytes = (uint32_t)align256((size_t)max_col * z * 4 * G);
        cfg.internal = pt.internal;
        cfg.entries = (int32_t)nnzb;
        int32_t tab_ent = 0, sec_words = 0;
        for (int k = 0; k < C; ++k) {
            const int32_t s0 = tab[kHSec + k];
            tab_ent = std::max(tab_ent, tab[s0 + kSNentC] + tab[s0 + kSNentB]);
            sec_words = std::max(sec_words, tab[kHSec + k + 1] - s0);
        }
        cfg.sec_words = sec_words;
        cfg.smem = cfg.e_bytes + cfg.l_bytes + 16 + (size_t)sec_words * 4 + (size_t)tab_ent * 16;
        if (cfg.smem > kClSmemLimit) continue;
        cfg.tab = std::move(tab);
        return cfg;
    }
    return best;
}

// Co-resident clusters of a launch shape (cached per kernel, device, size).
int cluster_capacity(ClFn fn, int C, size_t smem, int *nclusters) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int, size_t>, int> cache;
    int dev = -1;
    LDPC_TRY_CUDA(cudaGetDevice(&dev));
    LDPC_TRY(kernel_setup((const void *)fn, kClThreads, smem, nullptr));
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple((const void *)fn, dev, C, smem);
    auto it = cache.find(key);
    if (it == cache.end()) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3(kClThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        LDPC_TRY_CUDA(cudaOccupancyMaxActiveClusters(&n, (const void *)fn, &cfg));
        it = cache.emplace(key, n).first;
    }
    *nclusters = it->second;
    return LDPC_OK;
}

}  // namespace

// Host-side plans of a quasi-cyclic code created from its base matrix (none
// otherwise): z a multiple of 32, rows of at most 16 ones, and a partition
// whose part fits one SM.
int build_cluster_plan(ldpc_code *c) {
    c->cl_half = ClusterCfg{};
    c->cl_single = ClusterCfg{};
    if (c->qc.z <= 0 || c->qc.z % 32 || c->qc.z > 32 * 65535) return LDPC_OK;
    for (int32_t i = 0; i < c->qc.mb; ++i) {
        int d = 0;
        for (int32_t j = 0; j < c->qc.nb; ++j) d += c->qc.shift[(size_t)i * c->qc.nb + j] >= 0;
        if (d > kClMaxRow || d < 1) return LDPC_OK;
    }
    c->cl_half = choose_cluster(c, true);
    c->cl_single = choose_cluster(c, false);
    return LDPC_OK;
}

bool cluster_fits(const ldpc_code *c, const ldpc_decode_opts *o) {
    return (o->msg_fp16 ? c->cl_half.C : c->cl_single.C) > 0;
}

int decode_cluster(const ldpc_code *c, const float *d_llr, int32_t F, const ldpc_decode_opts *o,
                   float *d_post, uint32_t *d_hard, int32_t *d_iters, uint8_t *d_ok, void *d_work,
                   size_t work_bytes, cudaStream_t s) {
    if (!d_work || work_bytes < 256) return fail(LDPC_EINVAL, "workspace too small (need 256 bytes)");
    const bool fp16 = o->msg_fp16 != 0;
    const ClusterCfg &cfg = fp16 ? c->cl_half : c->cl_single;
    if (!cfg.C) return fail(LDPC_ENOTSUP, "no cluster layout for this code");
    const bool syn = o->early_stop != 0 && o->max_iters >= 2;
    ClFn fn = pick_cluster(fp16, syn);
    int nclusters = 0;
    LDPC_TRY(cluster_capacity(fn, cfg.C, cfg.smem, &nclusters));
    if (nclusters < 1) return fail(LDPC_ENOTSUP, "cluster of %d CTAs with %zu B each cannot be resident", cfg.C, cfg.smem);
    const int64_t groups = ceil_div(F, cfg.G);
    const int grid_clusters = (int)std::min<int64_t>(groups, nclusters);
    ClArgs a;
    a.llr = d_llr;
    a.F = F;
    a.n = c->n;
    a.NW = c->NW;
    a.z = c->qc.z;
    a.T_iters = o->max_iters;
    a.C = cfg.C;
    a.clip2 = clip_log2(o->clip);
    a.post = d_post;
    a.hard = d_hard;
    a.iters = d_iters;
    a.ok = d_ok;
    a.counter = static_cast<unsigned *>(d_work);
    a.tab = fp16 ? c->d.cl_tab_half : c->d.cl_tab_single;
    a.sec_words = cfg.sec_words;
    a.e_bytes = cfg.e_bytes;
    a.l_bytes = cfg.l_bytes;
    LDPC_TRY_CUDA(cudaMemsetAsync(d_work, 0, sizeof(unsigned), s));
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)(grid_clusters * cfg.C));
    lc.blockDim = dim3(kClThreads);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cfg.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    LDPC_TRY_CUDA(cudaLaunchKernelEx(&lc, fn, a));
    return LDPC_OK;
}

}  // namespace ldpc

using namespace ldpc;

extern "C" int ldpc_code_cluster_shape(const ldpc_code *c, int32_t msg_fp16, int32_t *ctas,
                                       int32_t *frames_per_group, float *local_fraction) {
    if (!c) return fail(LDPC_EINVAL, "code is NULL");
    const ClusterCfg &cfg = msg_fp16 ? c->cl_half : c->cl_single;
    if (ctas) *ctas = cfg.C;
    if (frames_per_group) *frames_per_group = cfg.G;
    if (local_fraction) *local_fraction = cfg.entries ? (float)cfg.internal / (float)cfg.entries : 0.f;
    return LDPC_OK;
}

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
// entry b = (i, j, s) connects check i z + r to bit j z + (r + s) mod z.
// CTA k of the cluster owns the lifting indices [k zc, (k+1) zc), zc = z / C,
// of every base row and column:
//   E[b][zc]  the messages of its checks (i, r), one plane per base entry,
//             binary16 pairs of two frames (G = 2) or FP32 (G = 1)
//   L[j][zc]  the total LLRs of its bits (j, t), float (G = 1) or float2
// The 32 lanes of a warp update 32 consecutive checks of one base row (or
// bits of one base column).  At every step they read 32 consecutive words of
// one plane, which lie in at most two CTAs (the circulant shift moves the run
// across the slice boundary), so the remote reads are contiguous: measured on
// GB300, contiguous remote 4-byte loads run at about 60 B per clock per SM,
// scattered ones at about 1.3.
//
// Per iteration: check pass (each warp's check items: gather L from the bits'
// owners, E from local planes, Eq. 5, store E), cluster barrier, bit pass
// (each warp's bit items: R_v plus the messages of the bit in ascending base
// row order, read from their owners, Eq. 7, store L), cluster barrier.  The
// channel LLRs R are re-read from global memory (L2) in every bit pass; the
// group's LLR rows stay in L2 while it is decoded.
#include <algorithm>
#include <map>
#include <mutex>
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

// Table blob (int32 words), copied into every CTA's shared memory:
//   [0..15]  header: nnzb, mb, nb, zc, then the word offsets below
//   ent      nnzb x 4: {j zc + s_lo, zc - s_lo, s_hi, b zc - s_lo}, s = s_hi zc + s_lo
//   rowptr   mb + 1 (base entries of row i: rowptr[i] .. rowptr[i+1]-1, ascending j)
//   colptr   nb + 1, colent nnzb (base entries of column j, ascending i)
//   cptr     kClWarps + 1, citems: check items (i << 16 | q) of each warp
//   bptr     kClWarps + 1, bitems: bit items (j << 16 | q) of each warp
enum { kHNnzb, kHMb, kHNb, kHZc, kHEnt, kHRow, kHColPtr, kHColEnt, kHCPtr, kHCItems, kHBPtr, kHBItems,
       kHWords, kHeader = 16 };

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
// The address of the same shared-memory word in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cl_map(uint32_t a, uint32_t rank) {
    uint32_t d;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(rank));
    return d;
}
// Loads (plain asm: schedulable within a pass, never across a barrier, whose
// base addresses are redefined after every barrier) and stores (volatile).
__device__ __forceinline__ float ldc_f(uint32_t a) {
    float v;
    asm("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float2 ldc_f2(uint32_t a) {
    float2 v;
    asm("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t ldc_u32(uint32_t a) {
    uint32_t v;
    asm("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a));
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

// Message planes: bytes per (entry, lane) and the word access of G frames.
template <class MsgT, int G>
struct ClMsg;
template <>
struct ClMsg<__half, 2> {  // binary16 pair (both frames) in one word
    static constexpr uint32_t B = 4;
    __device__ static uint32_t ld(uint32_t a) { return lds_u32(a); }
    __device__ static uint32_t ldc(uint32_t a) { return ldc_u32(a); }
    __device__ static void st(uint32_t a, uint32_t w) { sts_u32(a, w); }
};
template <>
struct ClMsg<float, 1> {
    static constexpr uint32_t B = 4;
    __device__ static uint32_t ld(uint32_t a) { return lds_u32(a); }
    __device__ static uint32_t ldc(uint32_t a) { return ldc_u32(a); }
    __device__ static void st(uint32_t a, uint32_t w) { sts_u32(a, w); }
};

// Total LLRs of G frames at one bit: float (G = 1) or float2.
template <int G>
struct ClL;
template <>
struct ClL<1> {
    __device__ static float ldc(uint32_t a) { return ldc_f(a); }
    __device__ static float ld(uint32_t a) { return lds_f(a); }
    __device__ static void st(uint32_t a, float v) { sts_f(a, v); }
};
template <>
struct ClL<2> {
    __device__ static float2 ldc(uint32_t a) { return ldc_f2(a); }
    __device__ static float2 ld(uint32_t a) { return lds_f2(a); }
    __device__ static void st(uint32_t a, float2 v) { sts_f2(a, v); }
};

// This CTA's plane bases and its place in the cluster.  The bases are
// redefined after every barrier (fence), so that no shared load of a pass is
// placed before the barrier that opens it.
struct ClCtx {
    uint32_t e;      // shared address of message plane 0
    uint32_t l;      // shared address of total plane 0
    uint32_t rank;   // CTA rank in the cluster
    uint32_t cmask;  // C - 1
    uint32_t zc;     // lifting indices per CTA
    __device__ void fence() { asm volatile("" : "+r"(e), "+r"(l)); }
};

// Per-CTA address tables, built in shared memory when the kernel starts (the
// peers' plane bases, mapped once): entry b of the check table (base rows in
// order) holds the cluster address of bit (j, s_lo) in the CTA that owns it
// when rloc + s_lo < zc (x), the address for the carry into the next CTA
// minus the slice width (y), and the carry threshold zc - s_lo (z), so that
// lane rloc reads bit (j, (r + s) mod z) at (rloc >= z ? y : x) + 4 G rloc.
// Entry k of the bit table (base columns in order, ascending rows) holds the
// same for the message of check (i, (t - s) mod z): x when tloc >= s_lo,
// y (the previous CTA's plane, plus the slice width) otherwise, z = s_lo.

// Check-node update (Eq. 5) of the 32 checks (i, rloc) of one warp item, rows
// of d <= D inputs taken in ascending base column order (the code's
// evaluation order): gather, leave-one-out pairs, new messages stored in
// place.  With SYN, returns bit i set when the hard decisions z = [L >= 0] of
// frame i (L as left by the last bit pass) violate this check.
template <class MsgT, int G, int D, bool SYN>
__device__ __forceinline__ uint32_t cl_check_item(const ClCtx &cx, const int4 *ctab, int b0, int d,
                                                  uint32_t rloc, float clip2) {
    using EV = EVec<MsgT, G>;
    using LV = Lanes<G>;
    using V = typename LV::T;
    using M = ClMsg<MsgT, G>;
    const uint32_t ea = cx.e + ((uint32_t)b0 * cx.zc + rloc) * M::B;  // position 0's message
    const uint32_t estep = cx.zc * M::B;
    const uint32_t roff = rloc * (4u * G);
    V u[D];
    uint32_t smask[G], zpar[G];
#pragma unroll
    for (int i = 0; i < G; ++i) smask[i] = zpar[i] = 0;
#pragma unroll
    for (int p = 0; p < D; ++p) {
        float uf[G];
#pragma unroll
        for (int i = 0; i < G; ++i) uf[i] = 0.f;  // positions beyond d: the identity
        if (p < d) {
            const int4 en = ctab[b0 + p];
            const uint32_t la = (rloc >= (uint32_t)en.z ? (uint32_t)en.y : (uint32_t)en.x) + roff;
            const V Lv = ClL<G>::ldc(la);
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
        if (p < d) {
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
__device__ __forceinline__ uint32_t cl_syndrome_item(const int4 *ctab, int b0, int d, uint32_t rloc) {
    using LV = Lanes<G>;
    const uint32_t roff = rloc * (4u * G);
    uint32_t par = 0;
    for (int p = 0; p < d; ++p) {
        const int4 en = ctab[b0 + p];
        const uint32_t la = (rloc >= (uint32_t)en.z ? (uint32_t)en.y : (uint32_t)en.x) + roff;
        const typename LV::T Lv = ClL<G>::ldc(la);
#pragma unroll
        for (int i = 0; i < G; ++i) par ^= (uint32_t)(LV::get(Lv, i) >= 0.f) << i;
    }
    return par;
}

// One check item through the instance sized for its row (any D >= d gives
// the same bits: padded positions hold the identity pair).
template <class MsgT, int G, bool SYN>
__device__ __forceinline__ uint32_t cl_check_dispatch(const ClCtx &cx, const int4 *ctab, int b0, int d,
                                                      uint32_t rloc, float clip2) {
    if (d <= 4) return cl_check_item<MsgT, G, 4, SYN>(cx, ctab, b0, d, rloc, clip2);
    if (d <= 6) return cl_check_item<MsgT, G, 6, SYN>(cx, ctab, b0, d, rloc, clip2);
    if (d <= 8) return cl_check_item<MsgT, G, 8, SYN>(cx, ctab, b0, d, rloc, clip2);
    if (d <= 10) return cl_check_item<MsgT, G, 10, SYN>(cx, ctab, b0, d, rloc, clip2);
    if (d <= 12) return cl_check_item<MsgT, G, 12, SYN>(cx, ctab, b0, d, rloc, clip2);
    if (d <= 14) return cl_check_item<MsgT, G, 14, SYN>(cx, ctab, b0, d, rloc, clip2);
    return cl_check_item<MsgT, G, kClMaxRow, SYN>(cx, ctab, b0, d, rloc, clip2);
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

// Bit-node update (Eq. 7) of the 32 bits (j, tloc) of one warp item:
// L = R + the bit's messages in ascending base row order (ascending edge
// index, the plain decoder's order), each read from the CTA that owns its
// check; bit table entries btab[k0 .. k1-1].  Frames not in `active` keep
// their L.
template <class MsgT, int G>
__device__ __forceinline__ void cl_bit_item(const ClCtx &cx, const int4 *btab, int k0, int k1, int j,
                                            uint32_t tloc, typename Lanes<G>::T L, uint32_t active) {
    using EV = EVec<MsgT, G>;
    using M = ClMsg<MsgT, G>;
    const uint32_t toff = tloc * M::B;
    // the messages of up to kBitChunk edges are requested together, then
    // added in order (the sum's order is fixed, the loads' is not)
    for (int k = k0; k < k1; k += kBitChunk) {
        uint32_t w[kBitChunk];
#pragma unroll
        for (int u = 0; u < kBitChunk; ++u) {
            if (k + u < k1) {
                const int4 en = btab[k + u];
                w[u] = M::ldc((tloc < (uint32_t)en.z ? (uint32_t)en.y : (uint32_t)en.x) + toff);
            }
        }
#pragma unroll
        for (int u = 0; u < kBitChunk; ++u)
            if (k + u < k1) L = EV::add_to(L, w[u]);
    }
    const uint32_t la = cx.l + ((uint32_t)j * cx.zc + tloc) * (4u * G);
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
    const int32_t *tab;
    int32_t tab_words;
    uint32_t e_bytes, l_bytes;  // multiples of 16
};

// Every CTA of a cluster runs the same control flow (the same group, the
// same iteration count, the same early-stop decisions from the same flags),
// so all reach every cluster barrier.
template <class MsgT, int G, bool SYN>
__global__ void __launch_bounds__(kClThreads, 1) cluster_kernel(ClArgs a) {
    using LV = Lanes<G>;
    using V = typename LV::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // layout: E planes | L planes | control words (flags by iteration parity,
    // group slot) | table blob | check and bit address tables
    int32_t *tab = reinterpret_cast<int32_t *>(smem + a.e_bytes + a.l_bytes + 16);
    for (int w = tid; w < a.tab_words; w += kClThreads) tab[w] = __ldg(&a.tab[w]);
    __syncthreads();
    ClCtx cx;
    cx.e = (uint32_t)__cvta_generic_to_shared(smem);
    cx.l = cx.e + a.e_bytes;
    cx.rank = cl_rank();
    cx.cmask = (uint32_t)a.C - 1u;
    cx.zc = (uint32_t)tab[kHZc];
    const uint32_t ctl = cx.l + a.l_bytes;  // [0], [1]: flags, [2]: group slot
    const int4 *ent = reinterpret_cast<const int4 *>(tab + tab[kHEnt]);
    const int32_t *rowptr = tab + tab[kHRow];
    const int32_t *colptr = tab + tab[kHColPtr];
    const int32_t *colent = tab + tab[kHColEnt];
    const int nnzb = tab[kHNnzb];
    int4 *ctab = reinterpret_cast<int4 *>(tab + a.tab_words);  // check table, then bit table
    int4 *btab = ctab + nnzb;
    {
        const uint32_t zc = cx.zc, lw = 4u * G, mb = ClMsg<MsgT, G>::B;
        for (int b = tid; b < nnzb; b += kClThreads) {
            const int4 en = ent[b];  // {j zc + s_lo, zc - s_lo, s_hi, b zc - s_lo}
            const uint32_t slo = zc - (uint32_t)en.y, shi = (uint32_t)en.z;
            const uint32_t lp = cx.l + ((uint32_t)en.x - slo) * lw;  // plane j
            const uint32_t o0 = (cx.rank + shi) & cx.cmask, o1 = (o0 + 1u) & cx.cmask;
            ctab[b] = make_int4((int)(cl_map(lp, o0) + slo * lw), (int)(cl_map(lp, o1) + slo * lw - zc * lw),
                                en.y, 0);
        }
        for (int k = tid; k < nnzb; k += kClThreads) {
            const int b = colent[k];
            const int4 en = ent[b];
            const uint32_t slo = zc - (uint32_t)en.y, shi = (uint32_t)en.z;
            const uint32_t ep = cx.e + (uint32_t)b * zc * mb;  // plane b
            const uint32_t q0 = (cx.rank - shi) & cx.cmask, q1 = (cx.rank - shi - 1u) & cx.cmask;
            btab[k] = make_int4((int)(cl_map(ep, q0) - slo * mb), (int)(cl_map(ep, q1) + (zc - slo) * mb),
                                (int)slo, 0);
        }
    }
    __syncthreads();
    const int c0 = tab[tab[kHCPtr] + warp], c1 = tab[tab[kHCPtr] + warp + 1];
    const int32_t *citems = tab + tab[kHCItems];
    const int g0 = tab[tab[kHBPtr] + warp], g1 = tab[tab[kHBPtr] + warp + 1];
    const int32_t *bitems = tab + tab[kHBItems];
    const int64_t vbase = (int64_t)cx.rank * cx.zc + lane;  // bit (j, 32q + lane) is j z + 32q + vbase
    const int groups = (a.F + G - 1) / G;
    for (;;) {
        if (cx.rank == 0 && tid == 0) sts_u32(ctl + 8, atomicAdd(a.counter, 1u));
        cl_sync();
        cx.fence();
        const int grp = (int)ldc_u32_volatile(cl_map(ctl + 8, 0));
        if (grp >= groups) {
            cl_sync();  // no CTA leaves while a peer may still read its slot
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
            const int j = bitems[k] >> 16, q = bitems[k] & 0xFFFF;
            const V R = cl_channel<G>(llr, (int64_t)j * a.z + 32 * q + vbase);
            ClL<G>::st(cx.l + ((uint32_t)j * cx.zc + 32u * q + lane) * (4u * G), R);
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
            for (int k = c0; k < c1; ++k) {
                const int i = citems[k] >> 16, q = citems[k] & 0xFFFF;
                const int b0 = rowptr[i], d = rowptr[i + 1] - b0;
                bad |= cl_check_dispatch<MsgT, G, SYN>(cx, ctab, b0, d, 32u * q + lane, a.clip2);
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
            if (g0 < g1) Rn = cl_channel<G>(llr, (int64_t)(bitems[g0] >> 16) * a.z + 32 * (bitems[g0] & 0xFFFF) + vbase);
            for (int k = g0; k < g1; ++k) {
                const int j = bitems[k] >> 16, q = bitems[k] & 0xFFFF;
                const V R = Rn;
                if (k + 1 < g1)
                    Rn = cl_channel<G>(llr, (int64_t)(bitems[k + 1] >> 16) * a.z + 32 * (bitems[k + 1] & 0xFFFF) + vbase);
                cl_bit_item<MsgT, G>(cx, btab, colptr[j], colptr[j + 1], j, 32u * q + lane, R, active);
            }
            cl_sync();
            cx.fence();
        }
        if (active) {  // frames that ran every iteration: syndrome of the final z
            uint32_t bad = 0;
            for (int k = c0; k < c1; ++k) {
                const int i = citems[k] >> 16, q = citems[k] & 0xFFFF;
                const int b0 = rowptr[i];
                bad |= cl_syndrome_item<G>(ctab, b0, rowptr[i + 1] - b0, 32u * q + lane);
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
            const int j = bitems[k] >> 16, q = bitems[k] & 0xFFFF;
            const int64_t v = (int64_t)j * a.z + 32 * q + vbase;
            const V Lv = ClL<G>::ld(cx.l + ((uint32_t)j * cx.zc + 32u * q + lane) * (4u * G));
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

// Table blob for one slice width zc (see the layout above).  Work items are
// dealt to the warps longest first, each to the warp with the least work so
// far (check items cost their row weight, bit items their column weight + 1).
std::vector<int32_t> build_cluster_table(const ldpc_code *c, int32_t zc) {
    const QcInfo &qc = c->qc;
    std::vector<int32_t> ej, es, rowptr(1, 0);
    for (int32_t i = 0; i < qc.mb; ++i) {
        for (int32_t j = 0; j < qc.nb; ++j) {
            const int16_t s = qc.shift[(size_t)i * qc.nb + j];
            if (s < 0) continue;
            ej.push_back(j);
            es.push_back(s);
        }
        rowptr.push_back((int32_t)ej.size());
    }
    const int32_t nnzb = (int32_t)ej.size();
    std::vector<int32_t> colptr(qc.nb + 1, 0), colent(nnzb);
    for (int32_t b = 0; b < nnzb; ++b) ++colptr[ej[b] + 1];
    for (int32_t j = 0; j < qc.nb; ++j) colptr[j + 1] += colptr[j];
    {
        std::vector<int32_t> fill(colptr.begin(), colptr.end() - 1);
        for (int32_t b = 0; b < nnzb; ++b) colent[fill[ej[b]]++] = b;  // b ascending = i ascending
    }
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
    const int32_t nq = zc / 32;
    std::vector<std::pair<int32_t, int32_t>> ci, bi;
    for (int32_t i = 0; i < qc.mb; ++i)
        for (int32_t q = 0; q < nq; ++q) ci.emplace_back(rowptr[i + 1] - rowptr[i], (i << 16) | q);
    for (int32_t j = 0; j < qc.nb; ++j)
        for (int32_t q = 0; q < nq; ++q) bi.emplace_back(colptr[j + 1] - colptr[j] + 1, (j << 16) | q);
    const auto cd = deal(ci), bd = deal(bi);
    std::vector<int32_t> tab(kHeader, 0);
    auto put = [&](int slot, const std::vector<int32_t> &v) {
        while (tab.size() % 4) tab.push_back(0);  // 16-byte aligned arrays
        tab[slot] = (int32_t)tab.size();
        tab.insert(tab.end(), v.begin(), v.end());
    };
    std::vector<int32_t> ent((size_t)nnzb * 4);
    for (int32_t b = 0; b < nnzb; ++b) {
        const int32_t slo = es[b] % zc, shi = es[b] / zc;
        ent[4 * b + 0] = ej[b] * zc + slo;
        ent[4 * b + 1] = zc - slo;
        ent[4 * b + 2] = shi;
        ent[4 * b + 3] = b * zc - slo;
    }
    tab[kHNnzb] = nnzb;
    tab[kHMb] = qc.mb;
    tab[kHNb] = qc.nb;
    tab[kHZc] = zc;
    put(kHEnt, ent);
    put(kHRow, rowptr);
    put(kHColPtr, colptr);
    put(kHColEnt, colent);
    put(kHCPtr, cd.first);
    put(kHCItems, cd.second);
    put(kHBPtr, bd.first);
    put(kHBItems, bd.second);
    while (tab.size() % 4) tab.push_back(0);
    tab[kHWords] = (int32_t)tab.size();
    return tab;
}

size_t cluster_smem(const ldpc_code *c, int32_t nnzb, int32_t zc, int G, int msg_bytes, size_t tab_words) {
    const size_t e = align256((size_t)nnzb * zc * G * msg_bytes);
    const size_t l = align256((size_t)c->qc.nb * zc * G * 4);
    return e + l + 16 + tab_words * 4 + (size_t)nnzb * 32;  // + the two address tables
}

// Region sizes of the layout (the kernel's e_bytes, l_bytes).
void cluster_regions(const ldpc_code *c, const ClusterCfg &cfg, bool fp16, uint32_t *e_bytes, uint32_t *l_bytes) {
    const int msg_bytes = fp16 ? 2 : 4;
    *e_bytes = (uint32_t)align256((size_t)cfg.tab[kHNnzb] * cfg.zc * cfg.G * msg_bytes);
    *l_bytes = (uint32_t)align256((size_t)c->qc.nb * cfg.zc * cfg.G * 4);
}

// The launch shape for one message type: the smallest cluster that divides
// z into slices of whole warps and whose slice fits one SM's shared memory.
ClusterCfg choose_cluster(const ldpc_code *c, bool fp16) {
    ClusterCfg best;
    const int msg_bytes = fp16 ? 2 : 4;
    const int G = fp16 ? 2 : 1;
    for (int C : {2, 4, 8}) {
            if (c->qc.z % (32 * C)) continue;
            const int32_t zc = c->qc.z / C;
            std::vector<int32_t> tab = build_cluster_table(c, zc);
            const size_t smem = cluster_smem(c, tab[kHNnzb], zc, G, msg_bytes, tab.size());
            if (smem > kClSmemLimit) continue;
            best.C = C;
            best.G = G;
            best.zc = zc;
            best.smem = smem;
            best.tab = std::move(tab);
            return best;
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
// otherwise): rows of at most 16 ones, and a slice that fits one SM.
int build_cluster_plan(ldpc_code *c) {
    c->cl_half = ClusterCfg{};
    c->cl_single = ClusterCfg{};
    if (c->qc.z <= 0) return LDPC_OK;
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
    a.tab_words = (int32_t)cfg.tab.size();
    cluster_regions(c, cfg, fp16, &a.e_bytes, &a.l_bytes);
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
                                       int32_t *frames_per_group) {
    if (!c) return fail(LDPC_EINVAL, "code is NULL");
    const ClusterCfg &cfg = msg_fp16 ? c->cl_half : c->cl_single;
    if (ctas) *ctas = cfg.C;
    if (frames_per_group) *frames_per_group = cfg.G;
    return LDPC_OK;
}

// Check-node arithmetic shared by every decoder kernel (FP32).
//
// Eq. 5 (sign-corrected for the LLR sign of Eq. 4) for edge j of a check of
// degree d with clipped inputs x_i:
//
//   E_j = (-1)^d * prod_{i != j} sgn(x_i) * 2 atanh( prod_{i != j} tanh(|x_i|/2) ).
//
// With u_i = exp(-|x_i|), tanh(|x_i|/2) = (1 - u_i) / (1 + u_i).  Expanding
// prod_{i in S} (1 + u_i) and prod_{i in S} (1 - u_i) over a set S gives
// ev + od and ev - od, where ev (od) is the sum of the products of u over the
// even-sized (odd-sized) subsets of S.  Hence
//
//   2 atanh( prod_{i in S} tanh(|x_i|/2) ) = ln( ev_S / od_S ).
//
// The pair (ev, od) of a union of disjoint sets is (e1 e2 + o1 o2,
// e1 o2 + o1 e2), and a single input contributes (1, u_i).  Every term is
// non-negative, so the pairs are formed without cancellation in FP32 even
// when the magnitudes saturate (u_i ~ e^-20) or vanish (u_i ~ 1), where the
// direct tanh / atanh form loses all precision in single precision.  The
// leave-one-out pairs come from a tree of partial products (LooTree below),
// so no division by an input is ever needed.
//
// Units: inside the kernels every LLR is held in log2 units (L / ln 2), so
// that u = 2^-|x| and |E| = log2(ev / od) map onto the hardware's base-2
// exponential and logarithm with no extra scaling; inputs are scaled by
// log2(e) when loaded and outputs by ln(2) when stored.  Per edge this costs
// one ex2, one reciprocal and one lg2.  All decoder schedules share these
// functions and the same operand order, so they produce identical bits.
#pragma once

#include <cuda_fp16.h>

#include <cstdint>

namespace ldpc {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct EvOd {
    float e, o;
};

__device__ __forceinline__ EvOd evod_join(EvOd a, EvOd b) {
    return {fmaf(a.e, b.e, __fmul_rn(a.o, b.o)), fmaf(a.e, b.o, __fmul_rn(a.o, b.e))};
}

// Adds one input u to a pair: (e, o) (+) (1, u).  u = 0 is the identity.
__device__ __forceinline__ EvOd evod_add(EvOd a, float u) {
    return {fmaf(u, a.o, a.e), fmaf(u, a.e, a.o)};
}

// (1, 0) (+) (1, u) = (1, u) and p (+) (1, 0) = p hold exactly in FP32 for
// the non-negative pairs formed here, so a combination with the identity may
// be skipped.  A 1 that such a skipped step would have produced at run time
// must then be opaque_one(): with a literal 1 the compiler rewrites
// fma(a, 1, b * c) as a + b * c and fuses that into fma(b, c, a), which rounds
// once where the written form rounds twice, and the decoders would no longer
// agree bit for bit.
__device__ __forceinline__ float opaque_one() {
    uint32_t b;
    asm("mov.b32 %0, 0x3f800000;" : "=r"(b));
    return __uint_as_float(b);
}

// Clipped check input x (log2 units) from the total LLR and the old message:
// L_vc = L_v - E_cv (Eq. 6 rearranged), clipped to +-clip2.
__device__ __forceinline__ float check_input(float L, float Eold, float clip2) {
    return fminf(fmaxf(L - Eold, -clip2), clip2);
}

// u = 2^-|x| for a clipped input.
__device__ __forceinline__ float check_u(float x) { return ex2_approx(-fabsf(x)); }

// |E| = min(log2(ev / od), clip2); od = 0 (a degree-1 check) gives clip2.
__device__ __forceinline__ float evod_magnitude(EvOd p, float clip2) {
    return fminf(lg2_approx(__fmul_rn(p.e, rcp_approx(p.o))), clip2);
}

// The same FP32 value of G frames (G = 1 or 2).  With two frames, one packed
// instruction (add/mul/fma .rn.f32x2 of sm_100 and later) does both; every
// lane rounds exactly as the scalar instruction does (round to nearest, no
// flush to zero), so the results are bit-identical to two scalar operations.
// Every add and multiply carries an explicit rounding (__fadd_rn / __fmul_rn,
// or inline PTX with .rn), so that the compiler evaluates scalar expressions
// exactly as written.  Packed products are used only where no sum consumes
// them (see evod_join<2>).
template <int G>
struct Lanes;
template <>
struct Lanes<1> {
    using T = float;
    __device__ static T make(const float *x) { return x[0]; }
    __device__ static T splat(float a) { return a; }
    __device__ static float get(T v, int) { return v; }
    __device__ static T add(T a, T b) { return __fadd_rn(a, b); }
    __device__ static T mul(T a, T b) { return __fmul_rn(a, b); }
    __device__ static T fma(T a, T b, T c) { return fmaf(a, b, c); }
};
template <>
struct Lanes<2> {
    using T = float2;
    __device__ static T make(const float *x) { return make_float2(x[0], x[1]); }
    __device__ static T splat(float a) { return make_float2(a, a); }
    __device__ static float get(T v, int i) { return i ? v.y : v.x; }
    __device__ static T add(T a, T b) {
        T r;
        asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
            "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
            : "=f"(r.x), "=f"(r.y)
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
        return r;
    }
    __device__ static T mul(T a, T b) {
        T r;
        asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
            "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
            : "=f"(r.x), "=f"(r.y)
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
        return r;
    }
    __device__ static T fma(T a, T b, T c) {
        T r;
        asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
            "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
            : "=f"(r.x), "=f"(r.y)
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
        return r;
    }
};

// The (ev, od) pair of G frames, with the operations of EvOd lane by lane.
template <int G>
struct EvOdV {
    typename Lanes<G>::T e, o;
};
template <int G>
__device__ __forceinline__ EvOdV<G> evod_join(EvOdV<G> a, EvOdV<G> b) {
    using LV = Lanes<G>;
    return {LV::fma(a.e, b.e, LV::mul(a.o, b.o)), LV::fma(a.e, b.o, LV::mul(a.o, b.e))};
}
// Two frames: the join is done lane by lane in scalar instructions.  In
// packed form ptxas contracted a packed product with the packed sum that
// consumes it (it treats mul.rn.f32x2 + add.rn.f32x2 as one fma, measured), and
// joins came out rounded differently from the scalar decoders; the packed
// pair additions below have no product feeding a sum and stay exact.
template <>
__device__ __forceinline__ EvOdV<2> evod_join<2>(EvOdV<2> a, EvOdV<2> b) {
    return {make_float2(fmaf(a.e.x, b.e.x, __fmul_rn(a.o.x, b.o.x)), fmaf(a.e.y, b.e.y, __fmul_rn(a.o.y, b.o.y))),
            make_float2(fmaf(a.e.x, b.o.x, __fmul_rn(a.o.x, b.e.x)), fmaf(a.e.y, b.o.y, __fmul_rn(a.o.y, b.e.y)))};
}
template <int G>
__device__ __forceinline__ EvOdV<G> evod_add(EvOdV<G> a, typename Lanes<G>::T u) {
    using LV = Lanes<G>;
    return {LV::fma(u, a.o, a.e), LV::fma(u, a.e, a.o)};
}
// Two inputs: (1, a) (+) (1, b) = (1 + a b, a + b), each part rounded once.
template <int G>
__device__ __forceinline__ EvOdV<G> evod_pair(typename Lanes<G>::T a, typename Lanes<G>::T b) {
    using LV = Lanes<G>;
    return {LV::fma(a, b, LV::splat(opaque_one())), LV::add(a, b)};
}

// Leave-one-out pairs of a row: out[j] = (+) of the pairs (1, u_i) of all its
// inputs i != j, for the D input positions of a kernel (D fixed at compile
// time; positions beyond the row's degree hold u = 0, the pair (1, 0), which
// is the identity of (+)).
//
// The pairs are formed on a segment tree over positions [0, W), W the power
// of two >= D: each node's total is the (+) of its two halves (leaves (1, u);
// two leaves combine by evod_pair), and each node passes down to each half the
// pair of everything outside that half -- the pair it received joined with the
// other half's total (at the leaves, with the sibling's u by evod_add).  This
// takes about 5 pair operations per input where prefix and suffix products
// take 8.  Every operation with an identity operand reproduces the other
// operand exactly (all values are non-negative), so nodes made only of
// positions >= D are left out, and a kernel with a larger D, whose extra
// positions hold u = 0 at run time, produces the same bits for every real
// input.  Wherever a left-out part would have supplied a 1, opaque_one() does,
// so that the compiler performs the same roundings either way.
template <int G, int D, int LO = 0, int HI = 1>
struct LooTree {
    using LV = Lanes<G>;
    using V = typename LV::T;
    using P = EvOdV<G>;
    static constexpr int MID = (LO + HI) / 2;
    __device__ static P leaf(V u) { return {LV::splat(opaque_one()), u}; }
    __device__ static P total(const V (&u)[D]) {
        if constexpr (HI - LO == 1) {
            return leaf(u[LO]);
        } else if constexpr (MID >= D) {
            return LooTree<G, D, LO, MID>::total(u);
        } else if constexpr (HI - LO == 2) {
            return evod_pair<G>(u[LO], u[MID]);
        } else {
            return evod_join<G>(LooTree<G, D, LO, MID>::total(u), LooTree<G, D, MID, HI>::total(u));
        }
    }
    // C: the pair of all inputs outside [LO, HI) (none at the root: HAS_C false)
    template <bool HAS_C>
    __device__ static void down(const V (&u)[D], P C, P (&out)[D]) {
        if constexpr (HI - LO == 1) {
            if constexpr (HAS_C) out[LO] = C;
            else out[LO] = P{LV::splat(opaque_one()), LV::splat(0.f)};
        } else if constexpr (MID >= D) {
            LooTree<G, D, LO, MID>::template down<HAS_C>(u, C, out);
        } else if constexpr (HI - LO == 2) {
            if constexpr (HAS_C) {
                out[LO] = evod_add<G>(C, u[MID]);
                out[MID] = evod_add<G>(C, u[LO]);
            } else {
                out[LO] = leaf(u[MID]);
                out[MID] = leaf(u[LO]);
            }
        } else {
            const P tl = LooTree<G, D, LO, MID>::total(u);
            const P tr = LooTree<G, D, MID, HI>::total(u);
            if constexpr (HAS_C) {
                LooTree<G, D, LO, MID>::template down<true>(u, evod_join<G>(C, tr), out);
                LooTree<G, D, MID, HI>::template down<true>(u, evod_join<G>(C, tl), out);
            } else {
                LooTree<G, D, LO, MID>::template down<true>(u, tr, out);
                LooTree<G, D, MID, HI>::template down<true>(u, tl, out);
            }
        }
    }
};
__host__ __device__ constexpr int loo_width(int d) { return d <= 1 ? 1 : 2 * loo_width((d + 1) / 2); }
template <int G, int D>
__device__ __forceinline__ void evod_leave_one_out(const typename Lanes<G>::T (&u)[D], EvOdV<G> (&out)[D]) {
    LooTree<G, D, 0, loo_width(D)>::template down<false>(u, EvOdV<G>{}, out);
}

// Loads and stores of V consecutive frames' messages (V = 1 or 2), widened
// to / narrowed from FP32.
template <class T, int V>
struct MsgVec;
template <>
struct MsgVec<float, 1> {
    __device__ static void load(const float *p, float *x) { x[0] = *p; }
    __device__ static void store(float *p, const float *x) { *p = x[0]; }
};
template <>
struct MsgVec<float, 2> {
    __device__ static void load(const float *p, float *x) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        x[0] = v.x;
        x[1] = v.y;
    }
    __device__ static void store(float *p, const float *x) {
        *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
    }
};
template <>
struct MsgVec<__half, 1> {
    __device__ static void load(const __half *p, float *x) { x[0] = __half2float(*p); }
    __device__ static void store(__half *p, const float *x) { *p = __float2half_rn(x[0]); }
};
template <>
struct MsgVec<__half, 2> {
    __device__ static void load(const __half *p, float *x) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(p));
        x[0] = v.x;
        x[1] = v.y;
    }
    __device__ static void store(__half *p, const float *x) {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(x[0], x[1]);
    }
};

// Raw (unconverted) message vectors, for loads issued well before use: the
// widening to FP32 happens when the values are consumed.
template <class T, int V>
struct MsgRaw;
template <>
struct MsgRaw<float, 1> {
    using R = float;
    __device__ static R load(const float *p) { return *p; }
    __device__ static void widen(R r, float *x) { x[0] = r; }
};
template <>
struct MsgRaw<float, 2> {
    using R = float2;
    __device__ static R load(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    __device__ static void widen(R r, float *x) {
        x[0] = r.x;
        x[1] = r.y;
    }
};
template <>
struct MsgRaw<__half, 1> {
    using R = __half;
    __device__ static R load(const __half *p) { return *p; }
    __device__ static void widen(R r, float *x) { x[0] = __half2float(r); }
};
template <>
struct MsgRaw<__half, 2> {
    using R = __half2;
    __device__ static R load(const __half *p) { return *reinterpret_cast<const __half2 *>(p); }
    __device__ static void widen(R r, float *x) {
        const float2 v = __half22float2(r);
        x[0] = v.x;
        x[1] = v.y;
    }
};

template <class T>
__device__ __forceinline__ float msg_load(const T *p);
template <>
__device__ __forceinline__ float msg_load<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float msg_load<__half>(const __half *p) { return __half2float(*p); }

template <class T>
__device__ __forceinline__ T msg_cvt(float x);
template <>
__device__ __forceinline__ float msg_cvt<float>(float x) { return x; }
template <>
__device__ __forceinline__ __half msg_cvt<__half>(float x) { return __float2half_rn(x); }

// Message words of G frames as the decoders store them (binary16 pairs or
// FP32), with three fused forms used by every resident-style kernel.
template <class T>
__device__ __forceinline__ uint32_t as_u32(T x) {
    return *reinterpret_cast<uint32_t *>(&x);
}
template <class T>
__device__ __forceinline__ T from_u32(uint32_t x) {
    return *reinterpret_cast<T *>(&x);
}

template <class MsgT, int G>
struct EVec;
// Besides widening and narrowing, each message word has three fused forms:
//   add_to(L, w)   = L + E    (the bit sum, Eq. 7)
//   sub_from(L, w) = L - E    (Eq. 6 rearranged)
//   signed_word(m, s) = the word of E_i = (bit 31 of s_i ? -m_i : m_i)
// each rounding exactly like the widened FP32 operation (binary16 widens
// exactly; the mixed-precision add and fma round once, like FADD; negation
// commutes with round-to-nearest).
template <>
struct EVec<__half, 2> {
    using T = __half2;
    __device__ static void get(T v, float *x) {
        const float2 f = __half22float2(v);
        x[0] = f.x;
        x[1] = f.y;
    }
    __device__ static T make(const float *x) { return __floats2half2_rn(x[0], x[1]); }
    __device__ static float2 add_to(float2 L, uint32_t w) {
        float2 r;
        asm("{\n\t.reg .f16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
            "add.rn.f32.f16 %0, lo, %3;\n\tadd.rn.f32.f16 %1, hi, %4;\n\t}"
            : "=f"(r.x), "=f"(r.y)
            : "r"(w), "f"(L.x), "f"(L.y));
        return r;
    }
    __device__ static float2 sub_from(float2 L, uint32_t w) {
        float2 r;  // (-1) E + L: the product is exact, one rounding
        asm("{\n\t.reg .f16 lo, hi, m;\n\tmov.b32 {lo, hi}, %2;\n\tmov.b16 m, 0xBC00;\n\t"
            "fma.rn.f32.f16 %0, lo, m, %3;\n\tfma.rn.f32.f16 %1, hi, m, %4;\n\t}"
            : "=f"(r.x), "=f"(r.y)
            : "r"(w), "f"(L.x), "f"(L.y));
        return r;
    }
    __device__ static uint32_t signed_word(const float *m, const uint32_t *s) {
        const uint32_t h = as_u32(__floats2half2_rn(m[0], m[1]));
        return h ^ (__byte_perm(s[0], s[1], 0x7030) & 0x80008000u);  // sign bytes -> bits 15, 31
    }
};
template <>
struct EVec<float, 1> {
    using T = float;
    __device__ static void get(T v, float *x) { x[0] = v; }
    __device__ static T make(const float *x) { return x[0]; }
    __device__ static float add_to(float L, uint32_t w) { return L + __uint_as_float(w); }
    __device__ static float sub_from(float L, uint32_t w) { return L - __uint_as_float(w); }
    __device__ static uint32_t signed_word(const float *m, const uint32_t *s) {
        return __float_as_uint(m[0]) ^ (s[0] & 0x80000000u);
    }
};


}  // namespace ldpc

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
// leave-one-out pairs come from prefix and suffix products, so no division
// by an input is ever needed.
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
    return {fmaf(a.e, b.e, a.o * b.o), fmaf(a.e, b.o, a.o * b.e)};
}

// Adds one input u to a pair: (e, o) (+) (1, u).  u = 0 is the identity.
__device__ __forceinline__ EvOd evod_add(EvOd a, float u) {
    return {fmaf(u, a.o, a.e), fmaf(u, a.e, a.o)};
}

// (1, 0) (+) (1, u) = (1, u) and p (+) (1, 0) = p hold exactly in FP32 for
// the non-negative pairs formed here, so the first prefix pair and the joins
// with an empty prefix or suffix may be taken as they are, not computed.  The
// 1 of such a pair must then be opaque_one(): with a literal 1 the compiler
// rewrites fma(a, 1, b * c) as a + b * c and fuses that into fma(b, c, a),
// which rounds once where the written form rounds twice, and the decoders
// would no longer agree bit for bit.
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
    return fminf(lg2_approx(p.e * rcp_approx(p.o)), clip2);
}

// The same FP32 value of G frames (G = 1 or 2).  With two frames, one packed
// instruction (FADD2 / FMUL2 / FFMA2 of sm_100 and later) does both; every
// lane rounds exactly as the scalar instruction does (round to nearest, no
// flush to zero), so the results are bit-identical to two scalar operations.
template <int G>
struct Lanes;
template <>
struct Lanes<1> {
    using T = float;
    __device__ static T make(const float *x) { return x[0]; }
    __device__ static T splat(float a) { return a; }
    __device__ static float get(T v, int) { return v; }
    __device__ static T add(T a, T b) { return a + b; }
    __device__ static T mul(T a, T b) { return a * b; }
    __device__ static T fma(T a, T b, T c) { return fmaf(a, b, c); }
};
template <>
struct Lanes<2> {
    using T = float2;
    __device__ static T make(const float *x) { return make_float2(x[0], x[1]); }
    __device__ static T splat(float a) { return make_float2(a, a); }
    __device__ static float get(T v, int i) { return i ? v.y : v.x; }
    __device__ static T add(T a, T b) { return __fadd2_rn(a, b); }
    __device__ static T mul(T a, T b) { return __fmul2_rn(a, b); }
    __device__ static T fma(T a, T b, T c) { return __ffma2_rn(a, b, c); }
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
template <int G>
__device__ __forceinline__ EvOdV<G> evod_add(EvOdV<G> a, typename Lanes<G>::T u) {
    using LV = Lanes<G>;
    return {LV::fma(u, a.o, a.e), LV::fma(u, a.e, a.o)};
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

}  // namespace ldpc

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

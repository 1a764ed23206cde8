// K7/K8: weighted belief propagation, forward with per-iteration checkpoints
// and its hand-written adjoint.
//
// Forward (T unrolled flooding iterations, Sec. II-B with one weight per edge
// and iteration multiplying E_cv in Eqs. 6 and 7):
//   x^t_e = L^{t-1}_v - w_{t-1,e} E^{t-1}_e      (x^1_e = R_v; Eq. 6)
//   E^t_e = check update of clip(x^t) over the row (Eq. 5)
//   L^t_v = R_v + sum_e w_{t,e} E^t_e             (Eq. 7)
// Every E^t and L^t is kept in the checkpoint buffer.  With all weights 1 the
// arithmetic is that of the plain decoder, operation for operation.
//
// Backward, for t = T..1, given g(L^T) = dloss/dL^T:
//   gL^t_v = g(L^T)_v (t = T) or sum_e gx^{t+1}_e
//   gR_v  += gL^t_v
//   gE^t_e = w_{t,e} (gL^t_v - gx^{t+1}_e)
//   gw_{t,e} = sum over frames of E^t_e (gL^t_v - gx^{t+1}_e)
//   gx^t_i = [|x_i| <= clip] sum_{j != i} gE_j [|E_j raw| <= clip] dE_j/dM_i
// and finally gR_v += sum_e gx^1_e.  The check Jacobian uses the even/odd
// subset-product form of check_math.cuh: with u = e^-|M|, (ev_j, od_j) the
// pair of the row without j and Q_ij = prod_{k not i,j} (1 - u_k^2),
//   dE_j/dM_i = (-1)^d prod_{k not i,j} sgn(M_k) * u_i Q_ij / (ev_j od_j).
// 1 - u is formed by a Taylor series for small |M| to avoid cancellation.
// Units: as in the decoders, LLRs are held in log2 units; this Jacobian is
// unit-free and the weight gradient equals that in natural units.
//
// Layout: frame-interleaved [index][Fs] as in the plain decoder; messages at
// the code's evaluation positions, weights and weight gradients by CSR edge.
// A thread takes 1, 2 or 4 adjacent frames through one vector access per
// row, so the index arithmetic of a row serves all of them.  The weight
// gradient is reduced over frames deterministically (a thread's frames in
// order, warp shuffles, then the warps of a block in order, then the frame
// blocks in order).
#include <algorithm>

#include "check_math.cuh"
#include "ldpc_internal.h"

namespace ldpc {
namespace {

constexpr int kWFB = 128;  // frames (threads) per block
constexpr int kWMaxDeg = 16;  // widest row: instances for rows of <= 8, <= 12 and <= 16 edges
constexpr int kWMaxCol = 32;  // column weight bound of the backward bit kernel

struct WbpCkpt {
    float *Rt;  // [n][Fs]
    float *L;   // [T][n][Fs]   L^1..L^T
    float *E;   // [T][E][Fs]   E^1..E^T
    int64_t Fs;
};

size_t ckpt_layout(const ldpc_code *c, int32_t F, int32_t T, WbpCkpt *ck, void *base) {
    const int64_t Fs = ceil_div(std::max(F, 1), 32) * 32;
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += align256(b);
        return o;
    };
    const size_t oR = take((size_t)c->n * Fs * 4);
    const size_t oL = take((size_t)T * c->n * Fs * 4);
    const size_t oE = take((size_t)T * c->nnz * Fs * 4);
    if (ck && base) {
        char *b = static_cast<char *>(base);
        ck->Rt = reinterpret_cast<float *>(b + oR);
        ck->L = reinterpret_cast<float *>(b + oL);
        ck->E = reinterpret_cast<float *>(b + oE);
        ck->Fs = Fs;
    }
    return off;
}

struct WbpWork {
    float *gR;      // [n][Fs]
    float *gOut;    // [n][Fs]  dloss/dL^T in log2 units
    float *gX;      // [E][Fs]
    float *gE;      // [E][Fs]
    float *gwpart;  // [nfb][E] partial weight gradients of one iteration
    int64_t nfb;
};

size_t work_layout(const ldpc_code *c, int32_t F, WbpWork *wk, void *base) {
    const int64_t Fs = ceil_div(std::max(F, 1), 32) * 32;
    const int64_t nfb = ceil_div(std::max(F, 1), kWFB);
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += align256(b);
        return o;
    };
    const size_t oR = take((size_t)c->n * Fs * 4);
    const size_t oO = take((size_t)c->n * Fs * 4);
    const size_t oX = take((size_t)c->nnz * Fs * 4);
    const size_t oE = take((size_t)c->nnz * Fs * 4);
    const size_t oP = take((size_t)nfb * c->nnz * 4);
    if (wk && base) {
        char *b = static_cast<char *>(base);
        wk->gR = reinterpret_cast<float *>(b + oR);
        wk->gOut = reinterpret_cast<float *>(b + oO);
        wk->gX = reinterpret_cast<float *>(b + oX);
        wk->gE = reinterpret_cast<float *>(b + oE);
        wk->gwpart = reinterpret_cast<float *>(b + oP);
        wk->nfb = nfb;
    }
    return off;
}

// V adjacent frames of one row are one aligned 4V-byte word of the
// frame-interleaved layout (Fs is a multiple of 32 and every buffer starts on
// a 16-byte boundary), read and written with one vector access.
template <int V>
struct FV;
template <>
struct FV<1> {
    __device__ static void ld(const float *p, float (&x)[1]) { x[0] = *p; }
    __device__ static void st(float *p, const float (&x)[1]) { *p = x[0]; }
};
template <>
struct FV<2> {
    __device__ static void ld(const float *p, float (&x)[2]) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        x[0] = t.x;
        x[1] = t.y;
    }
    __device__ static void st(float *p, const float (&x)[2]) {
        *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
    }
};
template <>
struct FV<4> {
    __device__ static void ld(const float *p, float (&x)[4]) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        x[0] = t.x;
        x[1] = t.y;
        x[2] = t.z;
        x[3] = t.w;
    }
    __device__ static void st(float *p, const float (&x)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
    }
};

// Frames each thread of a kernel takes (bounded by registers): forward
// checks 4 for rows of up to 8 edges, else 2; backward checks 2 and 1; bit
// kernels 4 for columns of up to 8 edges, else 1.
constexpr int check_frames(int dmax) { return dmax <= 8 ? 4 : 2; }
constexpr int back_check_frames(int dmax) { return dmax <= 8 ? 2 : 1; }
constexpr int bit_frames(int dv) { return dv <= 8 ? 4 : 1; }
constexpr int kBackBitFrames = 4;

// First frame of this thread, V frames per thread; every kernel covers all Fs
// frames (the padding frames hold zeros from the transposes below and stay
// finite), so each frame read was written by the kernel before.
template <int V>
__device__ __forceinline__ int64_t first_frame() {
    return ((int64_t)blockIdx.y * kWFB + threadIdx.x) * V;
}
inline unsigned frame_blocks(int64_t Fs, int V) { return (unsigned)ceil_div(Fs, (int64_t)kWFB * V); }

// llr[F][n] (natural units) -> dst[n][Fs] scaled by `scale`; the padding
// frames F..Fs-1 are set to 0.
__global__ void to_interleaved(const float *__restrict__ src, float *__restrict__ dst, int32_t n,
                               int32_t F, int64_t Fs, float scale) {
    __shared__ float tile[32][33];
    const int64_t v0 = (int64_t)blockIdx.x * 32, f0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t f = f0 + i, v = v0 + threadIdx.x;
        tile[i][threadIdx.x] = (f < F && v < n) ? src[f * n + v] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t v = v0 + i, f = f0 + threadIdx.x;
        if (v < n && f < Fs) dst[v * Fs + f] = tile[threadIdx.x][i] * scale;
    }
}

// src[n][Fs] -> dst[F][n] scaled by `scale`.
__global__ void from_interleaved(const float *__restrict__ src, float *__restrict__ dst, int32_t n,
                                 int32_t F, int64_t Fs, float scale) {
    __shared__ float tile[32][33];
    const int64_t v0 = (int64_t)blockIdx.x * 32, f0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t v = v0 + i, f = f0 + threadIdx.x;
        tile[i][threadIdx.x] = (v < n && f < F) ? src[v * Fs + f] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t f = f0 + i, v = v0 + threadIdx.x;
        if (f < F && v < n) dst[f * n + v] = tile[threadIdx.x][i] * scale;
    }
}

// Forward check update of iteration t (inputs from the previous checkpoint),
// V frames per thread, each with the scalar arithmetic of the plain decoder.
// EXACT: the row has DMAX edges, so no position needs a guard.
template <int DMAX, int V, bool EXACT>
__device__ __forceinline__ void check_row(const float *__restrict__ Lprev, const float *__restrict__ Eprev,
                                          const float *__restrict__ wprev, float *__restrict__ Ecur,
                                          const int32_t *__restrict__ eval_col,
                                          const int32_t *__restrict__ eval_edge, int64_t Fs, float clip2,
                                          int64_t f, int e0, int d_row) {
    const int d = EXACT ? DMAX : d_row;
    // every load of the row first, then the arithmetic
    float x[DMAX][V], wp[DMAX];
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        if (j < d) {
            const int e = e0 + j;  // evaluation position
            FV<V>::ld(Lprev + (int64_t)__ldg(&eval_col[e]) * Fs + f, x[j]);
            if (Eprev) wp[j] = __ldg(&wprev[__ldg(&eval_edge[e])]);
        }
    }
    if (Eprev) {
        float Ev[DMAX][V];
#pragma unroll
        for (int j = 0; j < DMAX; ++j)
            if (j < d) FV<V>::ld(Eprev + (int64_t)(e0 + j) * Fs + f, Ev[j]);
#pragma unroll
        for (int j = 0; j < DMAX; ++j)
            if (j < d) {
#pragma unroll
                for (int a = 0; a < V; ++a) x[j][a] = fmaf(-wp[j], Ev[j][a], x[j][a]);
            }
    }
    float u[V][DMAX];  // positions beyond the degree: u = 0 (identity)
    uint32_t xb[V][DMAX], sacc[V];
#pragma unroll
    for (int a = 0; a < V; ++a) sacc[a] = (uint32_t)(d & 1) << 31;
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
#pragma unroll
        for (int a = 0; a < V; ++a) {
            u[a][j] = 0.f;
            xb[a][j] = 0u;
            if (j < d) {
                xb[a][j] = __float_as_uint(x[j][a]);
                sacc[a] ^= xb[a][j];
                u[a][j] = check_u(fminf(fmaxf(x[j][a], -clip2), clip2));
            }
        }
    }
    EvOdV<1> loo[V][DMAX];  // leave-one-out pairs
#pragma unroll
    for (int a = 0; a < V; ++a) evod_leave_one_out<1, DMAX>(u[a], loo[a]);
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        if (j < d) {
            float out[V];
#pragma unroll
            for (int a = 0; a < V; ++a) {
                const float mag = fminf(lg2_approx(__fmul_rn(loo[a][j].e, rcp_approx(loo[a][j].o))), clip2);
                // sign flip = negation, as in every decoder
                out[a] = __uint_as_float(__float_as_uint(mag) ^ ((sacc[a] ^ xb[a][j]) & 0x80000000u));
            }
            FV<V>::st(Ecur + (int64_t)(e0 + j) * Fs + f, out);
        }
    }
}

template <int DMAX, int V>
__global__ void __launch_bounds__(kWFB)
wbp_check(const float *__restrict__ Lprev, const float *__restrict__ Eprev,
          const float *__restrict__ wprev, float *__restrict__ Ecur,
          const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ eval_col,
          const int32_t *__restrict__ eval_edge, int32_t m, int64_t Fs, float clip2) {
    const int64_t f = first_frame<V>();
    const int c = blockIdx.x;
    if (f >= Fs || c >= m) return;
    const int e0 = __ldg(&row_ptr[c]);
    const int d = __ldg(&row_ptr[c + 1]) - e0;
    if (d == DMAX)  // the same for the whole block
        check_row<DMAX, V, true>(Lprev, Eprev, wprev, Ecur, eval_col, eval_edge, Fs, clip2, f, e0, d);
    else
        check_row<DMAX, V, false>(Lprev, Eprev, wprev, Ecur, eval_col, eval_edge, Fs, clip2, f, e0, d);
}

// Forward bit update of iteration t: L^t_v = R_v + sum_e w_{t,e} E^t_e, the
// terms in ascending edge order.  Columns of up to DV edges: every load of a
// bit is issued before the first addition (the sum's order is fixed, the
// loads' is not).
template <int DV, int V>
__global__ void __launch_bounds__(kWFB)
wbp_bit(const float *__restrict__ Rt, const float *__restrict__ Ecur, const float *__restrict__ wcur,
        float *__restrict__ Lcur, const int32_t *__restrict__ col_ptr,
        const int32_t *__restrict__ col_edge, const int32_t *__restrict__ col_pos, int32_t n, int64_t Fs) {
    const int64_t f = first_frame<V>();
    const int v = blockIdx.x;
    if (f >= Fs || v >= n) return;
    const int q0 = __ldg(&col_ptr[v]), dv = __ldg(&col_ptr[v + 1]) - q0;
    float wq[DV], eq[DV][V];
#pragma unroll
    for (int k = 0; k < DV; ++k)
        if (k < dv) {
            wq[k] = __ldg(&wcur[__ldg(&col_edge[q0 + k])]);
            FV<V>::ld(Ecur + (int64_t)__ldg(&col_pos[q0 + k]) * Fs + f, eq[k]);
        }
    float L[V];
    FV<V>::ld(Rt + (int64_t)v * Fs + f, L);
#pragma unroll
    for (int k = 0; k < DV; ++k)
        if (k < dv) {
#pragma unroll
            for (int a = 0; a < V; ++a) L[a] = fmaf(wq[k], eq[k][a], L[a]);
        }
    FV<V>::st(Lcur + (int64_t)v * Fs + f, L);
}

// 1 - 2^-y for y >= 0 without cancellation near y = 0.
__device__ __forceinline__ float one_minus_exp2neg(float y, float u) {
    if (y >= 0.25f) return 1.f - u;
    const float z = y * kLn2;  // 1 - e^-z = z - z^2/2 + z^3/6 - z^4/24 + z^5/120 - ...
    return z * (1.f + z * (-0.5f + z * (1.f / 6.f + z * (-1.f / 24.f + z * (1.f / 120.f)))));
}

// Backward bit side of iteration t, V frames per thread.  Accumulates gR,
// forms gE^t and the weight-gradient contributions of the frames below F,
// reduced over the block's frames into gwpart[blockIdx.y][e].
template <int V>
__global__ void __launch_bounds__(kWFB)
wbp_bit_back(const float *__restrict__ gout2, const float *__restrict__ gX,
             const float *__restrict__ Ecur, const float *__restrict__ wcur, float *__restrict__ gE,
             float *__restrict__ gR, float *__restrict__ gwpart, const int32_t *__restrict__ col_ptr,
             const int32_t *__restrict__ col_edge, const int32_t *__restrict__ col_pos, int32_t n,
             int32_t F, int64_t Fs, int last, int first_acc, int32_t nnz) {
    __shared__ float red[kWMaxCol * (kWFB / 32)];
    const int64_t f = first_frame<V>();
    const int v = blockIdx.x;
    const bool live = f < Fs;
    const int q0 = __ldg(&col_ptr[v]), q1 = __ldg(&col_ptr[v + 1]);
    float gL[V];
#pragma unroll
    for (int a = 0; a < V; ++a) gL[a] = 0.f;
    if (live) {
        if (last) {
            FV<V>::ld(gout2 + (int64_t)v * Fs + f, gL);
        } else {
            for (int q = q0; q < q1; ++q) {
                float x[V];
                FV<V>::ld(gX + (int64_t)__ldg(&col_pos[q]) * Fs + f, x);
#pragma unroll
                for (int a = 0; a < V; ++a) gL[a] += x[a];
            }
        }
        float *pr = gR + (int64_t)v * Fs + f;
        float r[V];
        if (first_acc) {
#pragma unroll
            for (int a = 0; a < V; ++a) r[a] = gL[a];
        } else {
            FV<V>::ld(pr, r);
#pragma unroll
            for (int a = 0; a < V; ++a) r[a] += gL[a];
        }
        FV<V>::st(pr, r);
    }
    // weight-gradient partials: each thread sums its frames in order, each
    // warp reduces every edge of the bit by shuffles, then one barrier, then
    // thread q sums edge q over the warps in order (the same order of
    // additions as one reduction per edge)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = q0; q < q1; ++q) {
        float contrib = 0.f;
        if (live) {
            const int64_t ie = (int64_t)__ldg(&col_pos[q]) * Fs + f;
            const float w = __ldg(&wcur[__ldg(&col_edge[q])]);
            float g[V], ev[V], ge[V];
            if (last) {
#pragma unroll
                for (int a = 0; a < V; ++a) g[a] = gL[a];
            } else {
                FV<V>::ld(gX + ie, g);
#pragma unroll
                for (int a = 0; a < V; ++a) g[a] = gL[a] - g[a];
            }
            FV<V>::ld(Ecur + ie, ev);
#pragma unroll
            for (int a = 0; a < V; ++a) {
                ge[a] = w * g[a];
                if (f + a < F) contrib += ev[a] * g[a];
            }
            FV<V>::st(gE + ie, ge);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, off);
        if (lane == 0) red[(q - q0) * (kWFB / 32) + warp] = contrib;
    }
    __syncthreads();
    const int q = q0 + (int)threadIdx.x;
    if (q < q1) {
        float sum = 0.f;
        for (int w = 0; w < kWFB / 32; ++w) sum += red[(q - q0) * (kWFB / 32) + w];
        gwpart[(int64_t)blockIdx.y * nnz + __ldg(&col_edge[q])] = sum;
    }
}

// Backward check side of iteration t: gx^t from gE^t through the check
// Jacobian, with the clip masks; V frames per thread.
//
// With b_k the sign bit of x_k and pi the parity of all of them,
//   gx_i = u_i (-1)^(pi + d + b_i) sum_{j != i} Q_ij h'_j,
//   h'_j = (-1)^b_j gE_j [|E_j raw| <= clip] / (ev_j od_j),
// and Q_ij = P_i M_ij S_j for i < j (P_i the product of q_k below i, S_j that
// above j, M_ij that strictly between).  So the sum is P_i R_i + S_i W_i with
//   R_i = S_{i+1} h'_{i+1} + q_{i+1} R_{i+1}  (R_{d-1} = 0, terms j > i)
//   W_i = P_{i-1} h'_{i-1} + q_{i-1} W_{i-1}  (W_0 = 0,     terms j < i),
// O(d) operations per row.  Positions beyond the degree hold q = 1, h' = 0.
template <int DMAX, int V, bool EXACT>
__device__ __forceinline__ void check_back_row(const float *__restrict__ Lprev, const float *__restrict__ Eprev,
                                               const float *__restrict__ wprev, const float *__restrict__ gE,
                                               float *__restrict__ gX, const int32_t *__restrict__ eval_col,
                                               const int32_t *__restrict__ eval_edge, int64_t Fs, float clip2,
                                               int64_t f, int e0, int d_row) {
    const int d = EXACT ? DMAX : d_row;
    // every load of the row first, then the arithmetic
    float x[DMAX][V], g[DMAX][V], wp[DMAX];
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        if (j < d) {
            const int e = e0 + j;  // evaluation position
            FV<V>::ld(Lprev + (int64_t)__ldg(&eval_col[e]) * Fs + f, x[j]);
            FV<V>::ld(gE + (int64_t)e * Fs + f, g[j]);
            if (Eprev) wp[j] = __ldg(&wprev[__ldg(&eval_edge[e])]);
        }
    }
    if (Eprev) {
        float Ev[DMAX][V];
#pragma unroll
        for (int j = 0; j < DMAX; ++j)
            if (j < d) FV<V>::ld(Eprev + (int64_t)(e0 + j) * Fs + f, Ev[j]);
#pragma unroll
        for (int j = 0; j < DMAX; ++j)
            if (j < d) {
#pragma unroll
                for (int a = 0; a < V; ++a) x[j][a] = fmaf(-wp[j], Ev[j][a], x[j][a]);
            }
    }
    float out[DMAX][V];
#pragma unroll
    for (int a = 0; a < V; ++a) {
        float u[DMAX], q[DMAX], h[DMAX];
        uint32_t sb[DMAX], par = (uint32_t)(d & 1) << 31;
        bool in[DMAX];
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            u[j] = 0.f;
            q[j] = 1.f;
            sb[j] = 0u;
            in[j] = false;
            if (j < d) {
                const float xv = x[j][a];
                sb[j] = __float_as_uint(xv) & 0x80000000u;
                par ^= sb[j];
                in[j] = fabsf(xv) <= clip2;
                const float y = fminf(fabsf(xv), clip2);
                u[j] = check_u(y);
                q[j] = one_minus_exp2neg(y, u[j]) * (1.f + u[j]);
            }
        }
        // leave-one-out pairs as in the forward, for ev_j od_j and the output
        // mask; 1 / (ev_j od_j) by one reciprocal (its 1-ulp error is far below
        // the tolerance of a gradient)
        EvOdV<1> loo[DMAX];
        evod_leave_one_out<1, DMAX>(u, loo);
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            const EvOdV<1> p = loo[j];
            const float raw = lg2_approx(__fmul_rn(p.e, rcp_approx(p.o)));
            const float hj = (j < d && raw <= clip2 && p.o > 0.f) ? g[j][a] * rcp_approx(p.e * p.o) : 0.f;
            h[j] = __uint_as_float(__float_as_uint(hj) ^ sb[j]);
        }
        float P[DMAX], S[DMAX], R[DMAX], W[DMAX];
        P[0] = 1.f;
#pragma unroll
        for (int k = 1; k < DMAX; ++k) P[k] = P[k - 1] * q[k - 1];
        S[DMAX - 1] = 1.f;
#pragma unroll
        for (int k = DMAX - 2; k >= 0; --k) S[k] = S[k + 1] * q[k + 1];
        R[DMAX - 1] = 0.f;
#pragma unroll
        for (int k = DMAX - 2; k >= 0; --k) R[k] = fmaf(q[k + 1], R[k + 1], S[k + 1] * h[k + 1]);
        W[0] = 0.f;
#pragma unroll
        for (int k = 1; k < DMAX; ++k) W[k] = fmaf(q[k - 1], W[k - 1], P[k - 1] * h[k - 1]);
#pragma unroll
        for (int i = 0; i < DMAX; ++i) {
            const float acc = fmaf(P[i], R[i], S[i] * W[i]);
            const float gx = __uint_as_float(__float_as_uint(u[i] * acc) ^ par ^ sb[i]);
            out[i][a] = in[i] ? gx : 0.f;
        }
    }
#pragma unroll
    for (int i = 0; i < DMAX; ++i)
        if (i < d) FV<V>::st(gX + (int64_t)(e0 + i) * Fs + f, out[i]);
}

template <int DMAX, int V>
__global__ void __launch_bounds__(kWFB)
wbp_check_back(const float *__restrict__ Lprev, const float *__restrict__ Eprev,
               const float *__restrict__ wprev, const float *__restrict__ gE,
               float *__restrict__ gX, const int32_t *__restrict__ row_ptr,
               const int32_t *__restrict__ eval_col, const int32_t *__restrict__ eval_edge, int32_t m,
               int64_t Fs, float clip2) {
    const int64_t f = first_frame<V>();
    const int c = blockIdx.x;
    if (f >= Fs || c >= m) return;
    const int e0 = __ldg(&row_ptr[c]);
    const int d = __ldg(&row_ptr[c + 1]) - e0;
    if (d == DMAX)
        check_back_row<DMAX, V, true>(Lprev, Eprev, wprev, gE, gX, eval_col, eval_edge, Fs, clip2, f, e0, d);
    else
        check_back_row<DMAX, V, false>(Lprev, Eprev, wprev, gE, gX, eval_col, eval_edge, Fs, clip2, f, e0, d);
}

// gR_v += sum_e gx^1_e (x^1 = R).
template <int V>
__global__ void __launch_bounds__(kWFB)
wbp_final_r(const float *__restrict__ gX, float *__restrict__ gR, const int32_t *__restrict__ col_ptr,
            const int32_t *__restrict__ col_pos, int32_t n, int64_t Fs) {
    const int64_t f = first_frame<V>();
    const int v = blockIdx.x;
    if (f >= Fs || v >= n) return;
    float s[V];
    FV<V>::ld(gR + (int64_t)v * Fs + f, s);
    for (int q = __ldg(&col_ptr[v]), q1 = __ldg(&col_ptr[v + 1]); q < q1; ++q) {
        float x[V];
        FV<V>::ld(gX + (int64_t)__ldg(&col_pos[q]) * Fs + f, x);
#pragma unroll
        for (int a = 0; a < V; ++a) s[a] += x[a];
    }
    FV<V>::st(gR + (int64_t)v * Fs + f, s);
}

// grad_w[t][e] = sum over frame blocks (in order) of the partials.
__global__ void wbp_reduce_w(const float *__restrict__ gwpart, float *__restrict__ gw, int64_t nfb,
                             int32_t nnz) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    float s = 0.f;
    for (int64_t b = 0; b < nfb; ++b) s += gwpart[b * nnz + e];
    gw[e] = s;
}

int check_wbp_args(const ldpc_code *c, int32_t F, int32_t T, float clip) {
    if (!c) return fail(LDPC_EINVAL, "code is NULL");
    if (!c->on_device) return fail(LDPC_EINVAL, "code was created host-only");
    if (F < 0 || T < 0) return fail(LDPC_EINVAL, "F and T must be >= 0");
    if (!(clip > 0.f)) return fail(LDPC_EINVAL, "clip must be positive");
    if (c->dc_max > kWMaxDeg) return fail(LDPC_ENOTSUP, "weighted BP supports row degree <= %d", kWMaxDeg);
    if (c->dv_max > kWMaxCol) return fail(LDPC_ENOTSUP, "weighted BP supports column degree <= %d", kWMaxCol);
    if (ceil_div(F, kWFB) > 65535) return fail(LDPC_ENOTSUP, "too many frames (F=%d)", F);
    return LDPC_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

template <int DMAX>
void launch_check(const ldpc_code *c, const float *Lprev, const float *Eprev, const float *wprev, float *Ecur,
                  int64_t Fs, float clip2, cudaStream_t s) {
    constexpr int V = check_frames(DMAX);
    const dim3 g((unsigned)c->m, frame_blocks(Fs, V));
    wbp_check<DMAX, V><<<g, kWFB, 0, s>>>(Lprev, Eprev, wprev, Ecur, c->d.row_ptr, c->d.eval_col, c->d.eval_edge,
                                          c->m, Fs, clip2);
}

template <int DV>
void launch_bit(const ldpc_code *c, const float *Rt, const float *Ecur, const float *wcur, float *Lcur,
                int64_t Fs, cudaStream_t s) {
    constexpr int V = bit_frames(DV);
    const dim3 g((unsigned)c->n, frame_blocks(Fs, V));
    wbp_bit<DV, V><<<g, kWFB, 0, s>>>(Rt, Ecur, wcur, Lcur, c->d.col_ptr, c->d.col_edge, c->d.col_pos, c->n, Fs);
}

template <int DMAX>
void launch_check_back(const ldpc_code *c, const float *Lprev, const float *Eprev, const float *wprev,
                       const float *gE, float *gX, int64_t Fs, float clip2, cudaStream_t s) {
    constexpr int V = back_check_frames(DMAX);
    const dim3 g((unsigned)c->m, frame_blocks(Fs, V));
    wbp_check_back<DMAX, V><<<g, kWFB, 0, s>>>(Lprev, Eprev, wprev, gE, gX, c->d.row_ptr, c->d.eval_col,
                                               c->d.eval_edge, c->m, Fs, clip2);
}

}  // namespace
}  // namespace ldpc

using namespace ldpc;

extern "C" {

int ldpc_wbp_checkpoint_size(const ldpc_code *c, int32_t F, int32_t T, size_t *bytes) {
    if (!c || !bytes || F < 0 || T < 0) return fail(LDPC_EINVAL, "bad arguments");
    *bytes = ckpt_layout(c, F, T, nullptr, nullptr);
    return LDPC_OK;
}

int ldpc_wbp_forward(const ldpc_code *c, const float *d_llr, int32_t F, int32_t T, const float *d_w,
                     float clip, float *d_post, void *d_ckpt, size_t ckpt_bytes,
                     ldpc_stream_t stream) {
    TraceRange trace_("ldpc_wbp_forward");
    LDPC_TRY(check_wbp_args(c, F, T, clip));
    if (F == 0) return LDPC_OK;
    if (!d_llr || !d_post || !d_ckpt || (T > 0 && !d_w)) return fail(LDPC_EINVAL, "NULL pointer");
    if (!aligned16(d_ckpt)) return fail(LDPC_EINVAL, "checkpoint buffer not 16-byte aligned");
    WbpCkpt ck{};
    const size_t need = ckpt_layout(c, F, T, &ck, d_ckpt);
    if (ckpt_bytes < need) return fail(LDPC_EINVAL, "checkpoint buffer too small (%zu < %zu)", ckpt_bytes, need);
    cudaStream_t s = (cudaStream_t)stream;
    const float clip2 = clip_log2(clip);
    const dim3 tgrid((unsigned)ceil_div(c->n, 32), (unsigned)ceil_div(F, 32));
    to_interleaved<<<tgrid, dim3(32, 8), 0, s>>>(d_llr, ck.Rt, c->n, F, ck.Fs, kLog2e);
    const size_t nF = (size_t)c->n * ck.Fs, eF = (size_t)c->nnz * ck.Fs;
    for (int t = 1; t <= T; ++t) {
        const float *Lprev = t == 1 ? ck.Rt : ck.L + (t - 2) * nF;
        const float *Eprev = t == 1 ? nullptr : ck.E + (t - 2) * eF;
        const float *wprev = t == 1 ? nullptr : d_w + (size_t)(t - 2) * c->nnz;
        float *Ecur = ck.E + (t - 1) * eF;
        float *Lcur = ck.L + (t - 1) * nF;
        if (c->dc_max <= 6)
            launch_check<6>(c, Lprev, Eprev, wprev, Ecur, ck.Fs, clip2, s);
        else if (c->dc_max <= 8)
            launch_check<8>(c, Lprev, Eprev, wprev, Ecur, ck.Fs, clip2, s);
        else if (c->dc_max <= 12)
            launch_check<12>(c, Lprev, Eprev, wprev, Ecur, ck.Fs, clip2, s);
        else
            launch_check<kWMaxDeg>(c, Lprev, Eprev, wprev, Ecur, ck.Fs, clip2, s);
        const float *wcur = d_w + (size_t)(t - 1) * c->nnz;
        if (c->dv_max <= 4)
            launch_bit<4>(c, ck.Rt, Ecur, wcur, Lcur, ck.Fs, s);
        else if (c->dv_max <= 8)
            launch_bit<8>(c, ck.Rt, Ecur, wcur, Lcur, ck.Fs, s);
        else
            launch_bit<kWMaxCol>(c, ck.Rt, Ecur, wcur, Lcur, ck.Fs, s);
    }
    if (T == 0) {
        LDPC_TRY_CUDA(cudaMemcpyAsync(d_post, d_llr, sizeof(float) * (size_t)F * c->n,
                                      cudaMemcpyDeviceToDevice, s));
    } else {
        from_interleaved<<<tgrid, dim3(32, 8), 0, s>>>(ck.L + (T - 1) * nF, d_post, c->n, F, ck.Fs, kLn2);
    }
    LDPC_TRY_CUDA(cudaGetLastError());
    return LDPC_OK;
}

int ldpc_decode_backward_workspace_size(const ldpc_code *c, int32_t F, int32_t T, size_t *bytes) {
    if (!c || !bytes || F < 0 || T < 0) return fail(LDPC_EINVAL, "bad arguments");
    *bytes = work_layout(c, F, nullptr, nullptr);
    return LDPC_OK;
}

int ldpc_decode_backward(const ldpc_code *c, int32_t F, int32_t T, const float *d_w, float clip,
                         const void *d_ckpt, size_t ckpt_bytes,
                         const float *d_grad_post, float *d_grad_w, float *d_grad_llr, void *d_work,
                         size_t work_bytes, ldpc_stream_t stream) {
    TraceRange trace_("ldpc_decode_backward");
    LDPC_TRY(check_wbp_args(c, F, T, clip));
    cudaStream_t s = (cudaStream_t)stream;
    if (T > 0 && d_grad_w && F == 0)
        LDPC_TRY_CUDA(cudaMemsetAsync(d_grad_w, 0, sizeof(float) * (size_t)T * c->nnz, s));
    if (F == 0) return LDPC_OK;
    if (!d_ckpt || !d_grad_post || (T > 0 && !d_w)) return fail(LDPC_EINVAL, "NULL pointer");
    WbpCkpt ck{};
    if (ckpt_bytes < ckpt_layout(c, F, T, &ck, const_cast<void *>(d_ckpt)))
        return fail(LDPC_EINVAL, "checkpoint buffer too small");
    WbpWork wk{};
    const size_t need = work_layout(c, F, &wk, d_work);
    if (!d_work || work_bytes < need) return fail(LDPC_EINVAL, "workspace too small (%zu < %zu)", work_bytes, need);
    if (!aligned16(d_ckpt) || !aligned16(d_work))
        return fail(LDPC_EINVAL, "checkpoint and workspace must be 16-byte aligned");
    const float clip2 = clip_log2(clip);
    const dim3 tgrid((unsigned)ceil_div(c->n, 32), (unsigned)ceil_div(F, 32));
    if (T == 0) {  // post = llr: the gradient passes straight through
        if (d_grad_llr)
            LDPC_TRY_CUDA(cudaMemcpyAsync(d_grad_llr, d_grad_post, sizeof(float) * (size_t)F * c->n,
                                          cudaMemcpyDeviceToDevice, s));
        return LDPC_OK;
    }
    // dloss/dL2 = dloss/dpost * ln 2 (post = L2 ln 2)
    to_interleaved<<<tgrid, dim3(32, 8), 0, s>>>(d_grad_post, wk.gOut, c->n, F, ck.Fs, kLn2);
    float *gX = wk.gX;
    const size_t nF = (size_t)c->n * ck.Fs, eF = (size_t)c->nnz * ck.Fs;
    const dim3 bg((unsigned)c->n, frame_blocks(ck.Fs, kBackBitFrames));
    for (int t = T; t >= 1; --t) {
        const float *Ecur = ck.E + (t - 1) * eF;
        const float *wcur = d_w + (size_t)(t - 1) * c->nnz;
        wbp_bit_back<kBackBitFrames><<<bg, kWFB, 0, s>>>(wk.gOut, gX, Ecur, wcur, wk.gE, wk.gR, wk.gwpart,
                                                         c->d.col_ptr, c->d.col_edge, c->d.col_pos, c->n, F,
                                                         ck.Fs, t == T, t == T, (int32_t)c->nnz);
        if (d_grad_w)
            wbp_reduce_w<<<(unsigned)ceil_div(c->nnz, 256), 256, 0, s>>>(
                wk.gwpart, d_grad_w + (size_t)(t - 1) * c->nnz, (int64_t)bg.y, (int32_t)c->nnz);
        const float *Lprev = t == 1 ? ck.Rt : ck.L + (t - 2) * nF;
        const float *Eprev = t == 1 ? nullptr : ck.E + (t - 2) * eF;
        const float *wprev = t == 1 ? nullptr : d_w + (size_t)(t - 2) * c->nnz;
        if (c->dc_max <= 6)
            launch_check_back<6>(c, Lprev, Eprev, wprev, wk.gE, gX, ck.Fs, clip2, s);
        else if (c->dc_max <= 8)
            launch_check_back<8>(c, Lprev, Eprev, wprev, wk.gE, gX, ck.Fs, clip2, s);
        else if (c->dc_max <= 12)
            launch_check_back<12>(c, Lprev, Eprev, wprev, wk.gE, gX, ck.Fs, clip2, s);
        else
            launch_check_back<kWMaxDeg>(c, Lprev, Eprev, wprev, wk.gE, gX, ck.Fs, clip2, s);
    }
    wbp_final_r<kBackBitFrames><<<bg, kWFB, 0, s>>>(gX, wk.gR, c->d.col_ptr, c->d.col_pos, c->n, ck.Fs);
    if (d_grad_llr)
        from_interleaved<<<tgrid, dim3(32, 8), 0, s>>>(wk.gR, d_grad_llr, c->n, F, ck.Fs, kLog2e);
    LDPC_TRY_CUDA(cudaGetLastError());
    return LDPC_OK;
}

}  // extern "C"

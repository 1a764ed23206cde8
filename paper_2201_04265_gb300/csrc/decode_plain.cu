// K3/K4: the plain flooding sum-product decoder with messages in HBM.
//
// One check kernel (Eq. 5) and one bit kernel (Eqs. 6-8) per iteration, the
// schedule of Algorithm 1 without its MPI exchange: the whole batch of frames
// is the parallel axis (the paper's batch processing, Sec. III-C).
//
// Layout (workspace, frame-interleaved): every per-bit and per-edge array is
// stored [index][frame] with the frame index fastest, Fs = F rounded up to
// 32.  A thread owns V (1 or 2) consecutive frames; the lanes of a warp work
// on the same check (or bit) of 32 V consecutive frames, so graph indices are
// warp-uniform (broadcast loads) and every message load or store is one
// coalesced row segment of 32 V values.
//
//   Rt[n][Fs]  channel LLRs R_v          (float)
//   Lt[n][Fs]  total LLRs L_v (Eq. 7)    (float)
//   Et[E][Fs]  check messages E_cv       (float or binary16), check-major
//
// Only E_cv is stored per edge; the bit-to-check message of Eq. 6 is formed
// on the fly as L_vc = L_v - E_cv, which is Eq. 6 rearranged.  Edges are
// stored and combined in the code's evaluation order (the order every
// decoder shares, from the check schedule), and each bit sums its messages
// in ascending CSR edge order.
//
// Early stop: the check kernel of iteration t also evaluates the syndrome of
// the hard decisions z^(t-1) = [L^(t-1) >= 0] (it reads every L_v of its
// checks anyway) and flags frames with an unsatisfied check; the bit kernel of
// iteration t then freezes frames with no flag at iteration t-1, before
// touching their L_v.  Flags are double-buffered by iteration parity.
#include <algorithm>

#include "check_math.cuh"
#include "ldpc_internal.h"

namespace ldpc {
namespace {

constexpr int kFB = 128;   // frames (threads) per block
constexpr int kCPB = 4;    // checks per block in the check kernel
constexpr int kVPB = 8;    // bits per block in the bit kernel

struct PlainWs {
    float *Rt, *Lt;
    void *Et;
    uint32_t *unsat;   // [2][Fs]
    int32_t *stop_it;  // [Fs], -1 while active
    uint32_t *hard;    // [F][NW] scratch when the caller wants no hard bits
    uint8_t *ok;       // [F] scratch
    int64_t Fs;
};

size_t carve(const ldpc_code *c, int32_t F, bool fp16, PlainWs *ws, void *base) {
    const int64_t Fs = ceil_div(std::max(F, 1), 32) * 32;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t oR = take((size_t)c->n * Fs * 4);
    const size_t oL = take((size_t)c->n * Fs * 4);
    const size_t oE = take((size_t)c->nnz * Fs * (fp16 ? 2 : 4));
    const size_t oU = take((size_t)2 * Fs * 4);
    const size_t oS = take((size_t)Fs * 4);
    const size_t oH = take((size_t)F * c->NW * 4);
    const size_t oK = take((size_t)F);
    if (ws && base) {
        char *b = static_cast<char *>(base);
        ws->Rt = reinterpret_cast<float *>(b + oR);
        ws->Lt = reinterpret_cast<float *>(b + oL);
        ws->Et = b + oE;
        ws->unsat = reinterpret_cast<uint32_t *>(b + oU);
        ws->stop_it = reinterpret_cast<int32_t *>(b + oS);
        ws->hard = reinterpret_cast<uint32_t *>(b + oH);
        ws->ok = reinterpret_cast<uint8_t *>(b + oK);
        ws->Fs = Fs;
    }
    return off;
}

// llr[F][n] -> Rt[n][Fs] and Lt = Rt (L_v = R_v before the first iteration),
// scaled to log2 units.
__global__ void plain_init(const float *__restrict__ llr, float *__restrict__ Rt,
                           float *__restrict__ Lt, int32_t n, int32_t F, int64_t Fs) {
    __shared__ float tile[32][33];
    const int64_t v0 = (int64_t)blockIdx.x * 32, f0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t f = f0 + i, v = v0 + threadIdx.x;
        tile[i][threadIdx.x] = (f < F && v < n) ? llr[f * n + v] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t v = v0 + i, f = f0 + threadIdx.x;
        if (v < n && f < F) {
            const float r = tile[threadIdx.x][i] * kLog2e;
            Rt[v * Fs + f] = r;
            Lt[v * Fs + f] = r;
        }
    }
}

// Check-node update (Eq. 5) for kCPB checks x (kFB * V) frames; each thread
// owns V consecutive frames (vector loads of V floats / halves).  DMAX bounds
// the row degree so that the per-edge values stay in registers.  The inputs of
// the next check are loaded before the current one is computed, so that its
// memory latency overlaps the arithmetic.
template <class MsgT, int DMAX, int V>
__device__ __forceinline__ void plain_check_load(const float *__restrict__ Lt,
                                                 const MsgT *__restrict__ Et,
                                                 const int32_t *__restrict__ col_idx, int e0, int d,
                                                 int64_t Fs, int64_t f, int first,
                                                 typename MsgRaw<float, V>::R (&L)[DMAX],
                                                 typename MsgRaw<MsgT, V>::R (&Eo)[DMAX]) {
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        if (j < d) {
            const int v = __ldg(&col_idx[e0 + j]);
            L[j] = MsgRaw<float, V>::load(Lt + (int64_t)v * Fs + f);
            if (!first) Eo[j] = MsgRaw<MsgT, V>::load(Et + (int64_t)(e0 + j) * Fs + f);
        }
    }
}

// Blocks per SM a check instance is compiled for (a register budget of
// 65536 / (128 x blocks) per thread): the 16-wide one fits 4 blocks in 128
// registers without spilling (3 blocks at its natural 133).
template <int DMAX, int V>
constexpr int check_min_blocks() { return DMAX == 16 && V == 1 ? 4 : 0; }  // 0: no minimum

template <class MsgT, int DMAX, int V>
__global__ void __launch_bounds__(kFB, check_min_blocks<DMAX, V>())
plain_check(const float *__restrict__ Lt, MsgT *__restrict__ Et,
            const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
            const int32_t *__restrict__ rows, const int32_t *__restrict__ stop_it,
            uint32_t *__restrict__ unsat, int32_t mc, int32_t F, int64_t Fs, float clip2, int first,
            int check_syndrome) {
    const int64_t f = ((int64_t)blockIdx.y * kFB + threadIdx.x) * V;
    if (f >= F) return;
    bool any = false;
#pragma unroll
    for (int i = 0; i < V; ++i) any |= (f + i < F) && stop_it[f + i] < 0;
    if (!any) return;
    uint32_t bad[V];
#pragma unroll
    for (int i = 0; i < V; ++i) bad[i] = 0;
    const int c0 = blockIdx.x * kCPB;
    const int ncheck = min(kCPB, mc - c0);
    // raw prefetch buffers: widened to FP32 only when the check is computed, so
    // the next check's loads stay in flight during this check's arithmetic
    typename MsgRaw<float, V>::R Ln[DMAX];
    typename MsgRaw<MsgT, V>::R En[DMAX];
    int rn = __ldg(&rows[c0]);
    int e0n = __ldg(&row_ptr[rn]);
    int dn = __ldg(&row_ptr[rn + 1]) - e0n;
    plain_check_load<MsgT, DMAX, V>(Lt, Et, col_idx, e0n, dn, Fs, f, first, Ln, En);
    for (int cc = 0; cc < ncheck; ++cc) {
        const int e0 = e0n, d = dn;
        float L[DMAX][V], Eo[DMAX][V];
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            if (j < d) {
                MsgRaw<float, V>::widen(Ln[j], L[j]);
                if (first) {
#pragma unroll
                    for (int i = 0; i < V; ++i) Eo[j][i] = 0.f;
                } else {
                    MsgRaw<MsgT, V>::widen(En[j], Eo[j]);
                }
            }
        }
        if (cc + 1 < ncheck) {
            rn = __ldg(&rows[c0 + cc + 1]);
            e0n = __ldg(&row_ptr[rn]);
            dn = __ldg(&row_ptr[rn + 1]) - e0n;
            plain_check_load<MsgT, DMAX, V>(Lt, Et, col_idx, e0n, dn, Fs, f, first, Ln, En);
        }
        using LV = Lanes<V>;
        typename LV::T u[DMAX];  // positions beyond the degree: u = 0 (identity)
        uint32_t smask[V], zpar[V];
#pragma unroll
        for (int i = 0; i < V; ++i) smask[i] = zpar[i] = 0;
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            float uj[V];
#pragma unroll
            for (int i = 0; i < V; ++i) uj[i] = 0.f;
            if (j < d) {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    zpar[i] ^= (uint32_t)(L[j][i] >= 0.f);
                    const float x = check_input(L[j][i], Eo[j][i], clip2);
                    smask[i] |= (__float_as_uint(x) >> 31) << j;
                    uj[i] = check_u(x);
                }
            }
            u[j] = LV::make(uj);
        }
        uint32_t sall[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            bad[i] |= zpar[i];
            sall[i] = (__popc(smask[i]) + d) & 1u;
        }
        EvOdV<V> loo[DMAX];  // leave-one-out pairs
        evod_leave_one_out<V, DMAX>(u, loo);
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            if (j < d) {
                float out[V], rc[V];
#pragma unroll
                for (int i = 0; i < V; ++i) rc[i] = rcp_approx(LV::get(loo[j].o, i));
                const typename LV::T ratio = LV::mul(loo[j].e, LV::make(rc));
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const float mag = fminf(lg2_approx(LV::get(ratio, i)), clip2);
                    const uint32_t sgn = sall[i] ^ ((smask[i] >> j) & 1u);
                    out[i] = sgn ? -mag : mag;
                }
                MsgVec<MsgT, V>::store(Et + (int64_t)(e0 + j) * Fs + f, out);
            }
        }
    }
    if (check_syndrome)
#pragma unroll
        for (int i = 0; i < V; ++i)
            if (bad[i] && f + i < F) unsat[f + i] = 1u;
}

// Check-node update for rows wider than 32 (one frame per thread): inputs are
// combined in chunks of 8; a first pass forms each chunk's pair, a second pass
// reloads each chunk's inputs and combines the within-chunk leave-one-out pair
// with the pairs of all other chunks.  Rows up to 8 * kMaxChunks wide.  The
// chunk pairs and their prefixes are kept in shared memory ([4][chunk][thread]
// floats, so a warp's accesses hit 32 banks), not in registers.
constexpr int kMaxChunks = 32;
constexpr size_t kWideSmem = sizeof(float) * 4 * kMaxChunks * kFB;

template <class MsgT>
__global__ void __launch_bounds__(kFB)
plain_check_wide(const float *__restrict__ Lt, MsgT *__restrict__ Et,
                 const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                 const int32_t *__restrict__ rows, const int32_t *__restrict__ stop_it,
                 uint32_t *__restrict__ unsat, int32_t mc, int32_t F, int64_t Fs, float clip2,
                 int first, int check_syndrome) {
    extern __shared__ float wide_pairs[];  // [4][kMaxChunks][kFB]: ch.e, ch.o, preC.e, preC.o
    const int64_t f = (int64_t)blockIdx.y * kFB + threadIdx.x;
    if (f >= F || stop_it[f] >= 0) return;
    float *ch_e = wide_pairs + threadIdx.x, *ch_o = ch_e + kMaxChunks * kFB;
    float *pre_e = ch_o + kMaxChunks * kFB, *pre_o = pre_e + kMaxChunks * kFB;
    uint32_t bad = 0;
    for (int cc = 0; cc < kCPB; ++cc) {
        const int ci = blockIdx.x * kCPB + cc;
        if (ci >= mc) break;
        const int c = __ldg(&rows[ci]);
        const int e0 = __ldg(&row_ptr[c]);
        const int d = __ldg(&row_ptr[c + 1]) - e0;
        const int nch = (d + 7) >> 3;
        uint32_t sall = (uint32_t)d & 1u, zpar = 0;
        EvOd run = {1.f, 0.f};
        for (int k = 0; k < kMaxChunks; ++k) {
            if (k < nch) {
                EvOd p = {1.f, 0.f};
                for (int jj = 0; jj < 8; ++jj) {
                    const int j = 8 * k + jj;
                    if (j >= d) break;
                    const int v = __ldg(&col_idx[e0 + j]);
                    float Eo = 0.f;
                    if (!first) Eo = msg_load(&Et[(int64_t)(e0 + j) * Fs + f]);
                    const float L = Lt[(int64_t)v * Fs + f];
                    zpar ^= (uint32_t)(L >= 0.f);
                    const float x = check_input(L, Eo, clip2);
                    sall ^= __float_as_uint(x) >> 31;
                    p = evod_add(p, check_u(x));
                }
                ch_e[k * kFB] = p.e;
                ch_o[k * kFB] = p.o;
                pre_e[k * kFB] = run.e;
                pre_o[k * kFB] = run.o;
                run = evod_join(run, p);
            }
        }
        bad |= zpar;
        EvOd sufC = {1.f, 0.f};
        for (int k = kMaxChunks - 1; k >= 0; --k) {
            if (k < nch) {
                const EvOd other = evod_join(EvOd{pre_e[k * kFB], pre_o[k * kFB]}, sufC);
                const int jn = min(8, d - 8 * k);
                float u[8];
                uint32_t sm = 0;
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    if (jj < jn) {
                        const int j = 8 * k + jj;
                        const int v = __ldg(&col_idx[e0 + j]);
                        const float Eo = first ? 0.f : msg_load(&Et[(int64_t)(e0 + j) * Fs + f]);
                        const float x = check_input(Lt[(int64_t)v * Fs + f], Eo, clip2);
                        sm |= (__float_as_uint(x) >> 31) << jj;
                        u[jj] = check_u(x);
                    }
                }
                EvOd pre[8];
                pre[0] = other;
#pragma unroll
                for (int jj = 1; jj < 8; ++jj)
                    if (jj < jn) pre[jj] = evod_add(pre[jj - 1], u[jj - 1]);
                EvOd suf = {1.f, 0.f};
#pragma unroll
                for (int jj = 7; jj >= 0; --jj) {
                    if (jj < jn) {
                        const float mag = evod_magnitude(evod_join(pre[jj], suf), clip2);
                        const uint32_t sgn = sall ^ ((sm >> jj) & 1u);
                        Et[(int64_t)(e0 + 8 * k + jj) * Fs + f] = msg_cvt<MsgT>(sgn ? -mag : mag);
                        suf = evod_add(suf, u[jj]);
                    }
                }
                sufC = evod_join(EvOd{ch_e[k * kFB], ch_o[k * kFB]}, sufC);
            }
        }
    }
    if (check_syndrome && bad) unsat[f] = 1u;
}

// Bit-node update (Eq. 7) for kVPB bits x (kFB * V) frames.  Frames whose
// previous hard decisions satisfied every check stop here (early stop).  All
// loads of one bit are issued before the ordered summation R_v + E_1 + ...
// (ascending edge index), so the result does not depend on the launch shape.
template <class MsgT, int DVMAX, int V>
__global__ void __launch_bounds__(kFB)
plain_bit(const float *__restrict__ Rt, float *__restrict__ Lt, const MsgT *__restrict__ Et,
          const int32_t *__restrict__ col_ptr, const int32_t *__restrict__ col_edge,
          const int32_t *__restrict__ cols, int32_t *__restrict__ stop_it,
          const uint32_t *__restrict__ unsat_cur, uint32_t *__restrict__ unsat_next, int32_t nc,
          int32_t F, int64_t Fs, int t, int early_stop, int lead) {
    const int64_t f = ((int64_t)blockIdx.y * kFB + threadIdx.x) * V;
    if (f >= F) return;
    bool act[V];
    bool all = true, any = false;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        act[i] = (f + i < F) && stop_it[f + i] < 0;
        if (act[i] && early_stop) {
            if (lead && blockIdx.x == 0) unsat_next[f + i] = 0u;
            if (t >= 2 && unsat_cur[f + i] == 0u) {
                if (lead && blockIdx.x == 0) stop_it[f + i] = t - 1;
                act[i] = false;
            }
        }
        all &= act[i];
        any |= act[i];
    }
    if (!any) return;
    for (int vv = 0; vv < kVPB; ++vv) {
        const int vi = blockIdx.x * kVPB + vv;
        if (vi >= nc) break;
        const int v = __ldg(&cols[vi]);
        const int q0 = __ldg(&col_ptr[v]);
        const int dv = __ldg(&col_ptr[v + 1]) - q0;
        float L[V], Ev[DVMAX][V];
        MsgVec<float, V>::load(Rt + (int64_t)v * Fs + f, L);
#pragma unroll
        for (int q = 0; q < DVMAX; ++q)
            if (q < dv) MsgVec<MsgT, V>::load(Et + (int64_t)__ldg(&col_edge[q0 + q]) * Fs + f, Ev[q]);
#pragma unroll
        for (int q = 0; q < DVMAX; ++q)
            if (q < dv)
#pragma unroll
                for (int i = 0; i < V; ++i) L[i] += Ev[q][i];
        float *dst = Lt + (int64_t)v * Fs + f;
        if (all) {
            MsgVec<float, V>::store(dst, L);
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i)
                if (act[i]) dst[i] = L[i];
        }
    }
}

// Bit-node update for columns wider than 32 (one frame per thread).
template <class MsgT>
__global__ void __launch_bounds__(kFB)
plain_bit_wide(const float *__restrict__ Rt, float *__restrict__ Lt, const MsgT *__restrict__ Et,
               const int32_t *__restrict__ col_ptr, const int32_t *__restrict__ col_edge,
               const int32_t *__restrict__ cols, int32_t *__restrict__ stop_it,
               const uint32_t *__restrict__ unsat_cur, uint32_t *__restrict__ unsat_next, int32_t nc,
               int32_t F, int64_t Fs, int t, int early_stop, int lead) {
    const int64_t f = (int64_t)blockIdx.y * kFB + threadIdx.x;
    if (f >= F || stop_it[f] >= 0) return;
    if (early_stop) {
        if (lead && blockIdx.x == 0) unsat_next[f] = 0u;
        if (t >= 2 && unsat_cur[f] == 0u) {
            if (lead && blockIdx.x == 0) stop_it[f] = t - 1;
            return;
        }
    }
    for (int vv = 0; vv < kVPB; ++vv) {
        const int vi = blockIdx.x * kVPB + vv;
        if (vi >= nc) break;
        const int v = __ldg(&cols[vi]);
        float L = Rt[(int64_t)v * Fs + f];
        for (int q = __ldg(&col_ptr[v]), q1 = __ldg(&col_ptr[v + 1]); q < q1; ++q)
            L += msg_load(&Et[(int64_t)__ldg(&col_edge[q]) * Fs + f]);
        Lt[(int64_t)v * Fs + f] = L;
    }
}

// Lt[n][Fs] -> post[F][n] (optional, back to natural units) and packed hard
// decisions (Eq. 8).
__global__ void plain_output(const float *__restrict__ Lt, float *__restrict__ post,
                             uint32_t *__restrict__ hard, int32_t n, int32_t NW, int32_t F,
                             int64_t Fs) {
    __shared__ float tile[32][33];
    const int64_t v0 = (int64_t)blockIdx.x * 32, f0 = (int64_t)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t v = v0 + i, f = f0 + threadIdx.x;
        tile[i][threadIdx.x] = (v < n && f < F) ? Lt[v * Fs + f] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t f = f0 + i, v = v0 + threadIdx.x;
        const float L = tile[threadIdx.x][i];
        const uint32_t word = __ballot_sync(0xffffffffu, v < n && L >= 0.f);
        if (f < F) {
            if (post && v < n) post[f * n + v] = L * kLn2;
            if (threadIdx.x == 0) hard[f * NW + (v0 >> 5)] = word;
        }
    }
}

__global__ void plain_iters(const int32_t *__restrict__ stop_it, int32_t *__restrict__ iters,
                            int32_t F, int32_t T) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f < F) iters[f] = stop_it[f] >= 0 ? stop_it[f] : T;
}

// One launch per non-empty degree class; the instance is sized for the
// class's largest degree.  Check order does not matter (each check writes
// only its own messages), so the classes give the same bits as one launch.
template <class MsgT, int DMAX, int V>
void launch_check(const ldpc_code *c, const PlainWs &ws, int q, int32_t F, float clip2, int first,
                  int check_syn, uint32_t *unsat, cudaStream_t s) {
    const int32_t r0 = c->row_class[q], mc = c->row_class[q + 1] - r0;
    dim3 grid((unsigned)ceil_div(mc, kCPB), (unsigned)ceil_div(F, kFB * V));
    plain_check<MsgT, DMAX, V><<<grid, kFB, 0, s>>>(ws.Lt, static_cast<MsgT *>(ws.Et), c->d.row_ptr,
                                                    c->d.eval_col, c->d.row_order + r0, ws.stop_it,
                                                    unsat, mc, F, ws.Fs, clip2, first, check_syn);
}

template <class MsgT, int DVMAX, int V>
void launch_bit(const ldpc_code *c, const PlainWs &ws, int q, int lead, int32_t F, int t, int es,
                const uint32_t *u_cur, uint32_t *u_next, cudaStream_t s) {
    const int32_t v0 = c->col_class[q], nc = c->col_class[q + 1] - v0;
    dim3 grid((unsigned)ceil_div(nc, kVPB), (unsigned)ceil_div(F, kFB * V));
    plain_bit<MsgT, DVMAX, V><<<grid, kFB, 0, s>>>(ws.Rt, ws.Lt, static_cast<const MsgT *>(ws.Et),
                                                   c->d.col_ptr, c->d.col_pos, c->d.col_order + v0,
                                                   ws.stop_it, u_cur, u_next, nc, F, ws.Fs, t, es, lead);
}

template <class MsgT>
int run_plain(const ldpc_code *c, const float *d_llr, int32_t F, const ldpc_decode_opts *o,
              float *d_post, uint32_t *d_hard, int32_t *d_iters, uint8_t *d_ok, const PlainWs &ws,
              cudaStream_t s) {
    const int T = o->max_iters;
    const bool es = o->early_stop != 0;
    const float clip2 = clip_log2(o->clip);
    {
        dim3 grid((unsigned)ceil_div(c->n, 32), (unsigned)ceil_div(F, 32));
        plain_init<<<grid, dim3(32, 8), 0, s>>>(d_llr, ws.Rt, ws.Lt, c->n, F, ws.Fs);
    }
    LDPC_TRY_CUDA(cudaMemsetAsync(ws.unsat, 0, sizeof(uint32_t) * 2 * ws.Fs, s));
    LDPC_TRY_CUDA(cudaMemsetAsync(ws.stop_it, 0xff, sizeof(int32_t) * ws.Fs, s));
    for (int t = 1; t <= T; ++t) {
        uint32_t *u_cur = ws.unsat + (t & 1) * ws.Fs;
        uint32_t *u_next = ws.unsat + ((t + 1) & 1) * ws.Fs;
        const int first = t == 1;
        const int check_syn = es && t >= 2;
        for (int q = 0; q < kRowClasses; ++q) {
            if (c->row_class[q + 1] == c->row_class[q]) continue;
            switch (q) {
            case 0: launch_check<MsgT, 6, 2>(c, ws, q, F, clip2, first, check_syn, u_cur, s); break;
            case 1: launch_check<MsgT, 8, 2>(c, ws, q, F, clip2, first, check_syn, u_cur, s); break;
            case 2: launch_check<MsgT, 12, 1>(c, ws, q, F, clip2, first, check_syn, u_cur, s); break;
            case 3: launch_check<MsgT, 16, 1>(c, ws, q, F, clip2, first, check_syn, u_cur, s); break;
            case 4: launch_check<MsgT, 32, 1>(c, ws, q, F, clip2, first, check_syn, u_cur, s); break;
            default: {
                const int32_t r0 = c->row_class[q], mc = c->row_class[q + 1] - r0;
                dim3 grid((unsigned)ceil_div(mc, kCPB), (unsigned)ceil_div(F, kFB));
                LDPC_TRY(kernel_setup((const void *)plain_check_wide<MsgT>, kFB, kWideSmem, nullptr));
                plain_check_wide<MsgT><<<grid, kFB, kWideSmem, s>>>(
                    ws.Lt, static_cast<MsgT *>(ws.Et), c->d.row_ptr, c->d.eval_col, c->d.row_order + r0,
                    ws.stop_it, u_cur, mc, F, ws.Fs, clip2, first, check_syn);
            }
            }
        }
        // the first launched bit class also resets the next flags and records
        // stopped frames; later classes see those frames as stopped
        const int e = es ? 1 : 0;
        int lead = 1;
        for (int q = 0; q < kColClasses; ++q) {
            if (c->col_class[q + 1] == c->col_class[q]) continue;
            switch (q) {
            case 0: launch_bit<MsgT, 4, 2>(c, ws, q, lead, F, t, e, u_cur, u_next, s); break;
            case 1: launch_bit<MsgT, 8, 2>(c, ws, q, lead, F, t, e, u_cur, u_next, s); break;
            case 2: launch_bit<MsgT, 16, 1>(c, ws, q, lead, F, t, e, u_cur, u_next, s); break;
            default: {
                const int32_t v0 = c->col_class[q], nc = c->col_class[q + 1] - v0;
                dim3 grid((unsigned)ceil_div(nc, kVPB), (unsigned)ceil_div(F, kFB));
                plain_bit_wide<MsgT><<<grid, kFB, 0, s>>>(
                    ws.Rt, ws.Lt, static_cast<const MsgT *>(ws.Et), c->d.col_ptr, c->d.col_pos,
                    c->d.col_order + v0, ws.stop_it, u_cur, u_next, nc, F, ws.Fs, t, e, lead);
            }
            }
            lead = 0;
        }
    }
    LDPC_TRY_CUDA(cudaGetLastError());
    uint32_t *hard = d_hard ? d_hard : ws.hard;
    {
        dim3 grid((unsigned)ceil_div(c->n, 32), (unsigned)ceil_div(F, 32));
        plain_output<<<grid, dim3(32, 8), 0, s>>>(ws.Lt, d_post, hard, c->n, c->NW, F, ws.Fs);
    }
    if (T == 0 && d_post)  // no iteration: L_v = R_v exactly (Eq. 4), not a scaled round trip
        LDPC_TRY_CUDA(cudaMemcpyAsync(d_post, d_llr, sizeof(float) * (size_t)F * c->n,
                                      cudaMemcpyDeviceToDevice, s));
    LDPC_TRY(launch_syndrome(c, hard, F, nullptr, d_ok ? d_ok : ws.ok, s));
    if (d_iters) plain_iters<<<(unsigned)ceil_div(F, 256), 256, 0, s>>>(ws.stop_it, d_iters, F, T);
    LDPC_TRY_CUDA(cudaGetLastError());
    return LDPC_OK;
}

}  // namespace

size_t plain_workspace(const ldpc_code *c, int32_t F, const ldpc_decode_opts *o) {
    return carve(c, F, o->msg_fp16 != 0, nullptr, nullptr);
}

int decode_plain(const ldpc_code *c, const float *d_llr, int32_t F, const ldpc_decode_opts *o,
                 float *d_post, uint32_t *d_hard, int32_t *d_iters, uint8_t *d_ok, void *d_work,
                 size_t work_bytes, cudaStream_t s) {
    if (c->dc_max > 8 * kMaxChunks)
        return fail(LDPC_ENOTSUP, "plain decoder supports row degree <= %d (got %d)", 8 * kMaxChunks,
                    c->dc_max);
    if (ceil_div(F, kFB) > 65535 || ceil_div(F, 32) > 65535)
        return fail(LDPC_ENOTSUP, "too many frames for one plain decode call (F=%d)", F);
    PlainWs ws{};
    const size_t need = carve(c, F, o->msg_fp16 != 0, &ws, d_work);
    if (!d_work || work_bytes < need)
        return fail(LDPC_EINVAL, "workspace too small (%zu < %zu bytes)", work_bytes, need);
    if (o->msg_fp16) return run_plain<__half>(c, d_llr, F, o, d_post, d_hard, d_iters, d_ok, ws, s);
    return run_plain<float>(c, d_llr, F, o, d_post, d_hard, d_iters, d_ok, ws, s);
}

}  // namespace ldpc

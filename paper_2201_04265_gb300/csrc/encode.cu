// K1 (systematic encoding, Eq. 3) and K2 (syndrome, Eq. 1) kernels.
//
// Encoding computes p^T = m^T G with G = [I_k : P] up to H's column order
// (Sec. III-B): the k information bits are copied to their positions and
// parity bit j is the GF(2) inner product of row j of A = P^T with m.  Bits
// are packed 32 per word, so one inner product is an AND/XOR reduction over
// KW words followed by one population-count parity; the AND+XOR pair is a
// single LOP3 per word.  The GF(2) products are dense, so this is ALU work on
// packed words, not a tensor-core contraction.
#include <algorithm>

#include "ldpc_internal.h"

namespace ldpc {
namespace {

constexpr int kEncThreads = 256;
constexpr int kEncRows = 2;  // parity rows per thread per pass

// One block encodes FT frames.  Shared memory: the FT information words
// transposed to [KW][FT] (so one 128-bit load gives 4 frames' word w) and
// the FT output codewords [FT][NW] assembled with shared-memory atomics.
template <int FT>
__global__ void __launch_bounds__(kEncThreads)
encode_kernel(const uint32_t *__restrict__ info, uint32_t *__restrict__ code,
              const uint32_t *__restrict__ AT, const int32_t *__restrict__ info_pos,
              const int32_t *__restrict__ parity_pos, int32_t F, int32_t k, int32_t rank,
              int32_t KW, int32_t NW) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *msg = smem;                  // [KW][FT]
    uint32_t *cw = smem + (size_t)KW * FT; // [FT][NW]
    const int64_t f0 = (int64_t)blockIdx.x * FT;
    const int nf = (int)((int64_t)F - f0 < FT ? (int64_t)F - f0 : FT);
    for (int idx = threadIdx.x; idx < KW * FT; idx += blockDim.x) {
        const int f = idx / KW, w = idx - f * KW;
        msg[w * FT + f] = f < nf ? info[(f0 + f) * KW + w] : 0u;
    }
    for (int idx = threadIdx.x; idx < FT * NW; idx += blockDim.x) cw[idx] = 0u;
    __syncthreads();
    // information bits -> their codeword positions
    for (int idx = threadIdx.x; idx < KW * nf; idx += blockDim.x) {
        const int w = idx / nf, f = idx - w * nf;
        uint32_t word = msg[w * FT + f];
        if (w == KW - 1 && (k & 31)) word &= (1u << (k & 31)) - 1u;
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1u;
            const int p = info_pos[w * 32 + b];
            atomicOr(&cw[f * NW + (p >> 5)], 1u << (p & 31));
        }
    }
    // parity bits: parity(popc(XOR_w (A_jw & m_w)))
    for (int j0 = 0; j0 < rank; j0 += kEncThreads * kEncRows) {
        uint32_t acc[kEncRows][FT];
#pragma unroll
        for (int r = 0; r < kEncRows; ++r)
#pragma unroll
            for (int f = 0; f < FT; ++f) acc[r][f] = 0u;
        int j[kEncRows];
#pragma unroll
        for (int r = 0; r < kEncRows; ++r) j[r] = j0 + r * kEncThreads + threadIdx.x;
        for (int w = 0; w < KW; ++w) {
            uint32_t a[kEncRows];
#pragma unroll
            for (int r = 0; r < kEncRows; ++r) a[r] = j[r] < rank ? __ldg(&AT[(size_t)w * rank + j[r]]) : 0u;
            const uint4 *mrow = reinterpret_cast<const uint4 *>(msg + w * FT);
#pragma unroll
            for (int q = 0; q < FT / 4; ++q) {
                const uint4 mm = mrow[q];
#pragma unroll
                for (int r = 0; r < kEncRows; ++r) {
                    acc[r][4 * q + 0] ^= a[r] & mm.x;
                    acc[r][4 * q + 1] ^= a[r] & mm.y;
                    acc[r][4 * q + 2] ^= a[r] & mm.z;
                    acc[r][4 * q + 3] ^= a[r] & mm.w;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kEncRows; ++r) {
            if (j[r] >= rank) continue;
            const int p = parity_pos[j[r]];
#pragma unroll
            for (int f = 0; f < FT; ++f)
                if (f < nf && (__popc(acc[r][f]) & 1)) atomicOr(&cw[f * NW + (p >> 5)], 1u << (p & 31));
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nf * NW; idx += blockDim.x) code[f0 * NW + idx] = cw[idx];
}

// One block per frame (grid-stride): the frame's packed bits are staged in
// shared memory, each thread XORs the bits of one check row at a time, and a
// warp ballot packs 32 check results into one syndrome word.
__global__ void __launch_bounds__(256)
syndrome_kernel(const uint32_t *__restrict__ bits, int32_t F, int32_t m, int32_t NW, int32_t MW,
                const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                uint32_t *__restrict__ syn, uint8_t *__restrict__ ok) {
    extern __shared__ uint32_t z[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t f = blockIdx.x; f < F; f += gridDim.x) {
        for (int w = threadIdx.x; w < NW; w += blockDim.x) z[w] = bits[f * NW + w];
        __syncthreads();
        int unsat = 0;
        for (int c0 = 0; c0 < m; c0 += blockDim.x) {
            const int c = c0 + threadIdx.x;
            uint32_t s = 0;
            if (c < m)
                for (int e = __ldg(&row_ptr[c]), e1 = __ldg(&row_ptr[c + 1]); e < e1; ++e) {
                    const int v = __ldg(&col_idx[e]);
                    s ^= (z[v >> 5] >> (v & 31)) & 1u;
                }
            unsat |= (int)s;
            const uint32_t word = __ballot_sync(0xffffffffu, s);
            const int wc = c0 + warp * 32;
            if (syn && lane == 0 && wc < m) syn[f * MW + (wc >> 5)] = word;
        }
        const int any = __syncthreads_or(unsat);
        if (ok && threadIdx.x == 0) ok[f] = (uint8_t)(any == 0);
        __syncthreads();
    }
}

template <int FT>
size_t enc_smem(const ldpc_code *c) {
    return ((size_t)c->KW * FT + (size_t)FT * c->NW) * sizeof(uint32_t);
}

template <int FT>
int launch_enc(const ldpc_code *c, const uint32_t *d_info, uint32_t *d_code, int32_t F,
               cudaStream_t s) {
    const size_t sm = enc_smem<FT>(c);
    LDPC_TRY(kernel_setup((const void *)encode_kernel<FT>, kEncThreads, sm, nullptr));
    const unsigned grid = (unsigned)ceil_div(F, FT);
    encode_kernel<FT><<<grid, kEncThreads, sm, s>>>(d_info, d_code, c->d.AT, c->d.info_pos,
                                                   c->d.parity_pos, F, c->k, c->rank, c->KW, c->NW);
    LDPC_TRY_CUDA(cudaGetLastError());
    return LDPC_OK;
}

}  // namespace

int launch_encode(const ldpc_code *c, const uint32_t *d_info, uint32_t *d_code, int32_t F,
                  cudaStream_t s) {
    // The widest frame tile that fits in shared memory and still gives every
    // SM at least two blocks (fewer frames per block re-read A more often from
    // L2, but a small batch of a long code would otherwise leave SMs idle);
    // the result does not depend on the tile.
    constexpr size_t kMaxSmem = 200 * 1024;
    int sms = 0;
    LDPC_TRY(sm_count(&sms));
    const int64_t want = 2 * (int64_t)sms;
    const bool f32 = enc_smem<32>(c) <= kMaxSmem, f16 = enc_smem<16>(c) <= kMaxSmem,
               f8 = enc_smem<8>(c) <= kMaxSmem;
    if (f32 && ceil_div(F, 32) >= want) return launch_enc<32>(c, d_info, d_code, F, s);
    if (f16 && ceil_div(F, 16) >= want) return launch_enc<16>(c, d_info, d_code, F, s);
    if (f8) return launch_enc<8>(c, d_info, d_code, F, s);
    if (f16) return launch_enc<16>(c, d_info, d_code, F, s);
    if (f32) return launch_enc<32>(c, d_info, d_code, F, s);
    return fail(LDPC_ENOTSUP, "code too long for the encoder's shared-memory tile (n=%d)", c->n);
}

int launch_syndrome(const ldpc_code *c, const uint32_t *d_bits, int32_t F, uint32_t *d_syn,
                    uint8_t *d_ok, cudaStream_t s) {
    const size_t sm = (size_t)c->NW * sizeof(uint32_t);
    if (sm > 200 * 1024) return fail(LDPC_ENOTSUP, "code too long for the syndrome kernel");
    LDPC_TRY(kernel_setup((const void *)syndrome_kernel, 256, sm, nullptr));
    int sms = 0;
    LDPC_TRY(sm_count(&sms));
    const unsigned grid = (unsigned)std::min<int64_t>(F, (int64_t)sms * 8);
    syndrome_kernel<<<grid, 256, sm, s>>>(d_bits, F, c->m, c->NW, c->MW, c->d.row_ptr, c->d.col_idx,
                                          d_syn, d_ok);
    LDPC_TRY_CUDA(cudaGetLastError());
    return LDPC_OK;
}

}  // namespace ldpc

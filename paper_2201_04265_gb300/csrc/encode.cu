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

// ---------------------------------------------------------------------------
// Four-Russians encoding (no counterpart in the paper, which states only the
// product of Eq. 3).  The information bits are cut into groups of 8; for
// group g and every byte value b, a table holds the XOR of the columns of A
// selected by b (columns 8g + i for the set bits i of b).  The parity vector of
// a frame is then the XOR over groups of one table row each, instead of
// rank / 32 AND/XOR word steps per information word.  Parity is handled in
// slices of 128 bits (4 words): table block (s, g) holds the 256 rows of
// slice s, 4 KB, contiguous.  Result bits are those of the AND/XOR form:
// XOR is associative and every table row is an exact XOR of columns of A.
constexpr int kM4Slice = 4;       // parity words per slice
constexpr int kM4Threads = 256;   // frames per block of the lookup kernel

// AC[i][q] = word q of column i of A (bit l = A[32 q + l][i]), i < 8 NG,
// q < 4 NS; zero for i >= k or 32 q + l >= rank.
__global__ void m4_columns_kernel(const uint32_t *__restrict__ AT, int32_t k, int32_t rank,
                                  int32_t I8, int32_t RWp, uint32_t *__restrict__ AC) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)I8 * RWp) return;
    const int i = (int)(idx % I8), q = (int)(idx / I8);
    uint32_t col = 0;
    if (i < k)
        for (int l = 0; l < 32; ++l) {
            const int j = 32 * q + l;
            if (j < rank) col |= ((__ldg(&AT[(size_t)(i >> 5) * rank + j]) >> (i & 31)) & 1u) << l;
        }
    AC[(size_t)i * RWp + q] = col;
}

// tab[((s NG + g) 256 + b) 4 + c] = XOR over set bits i of b of AC[8 g + i][4 s + c].
__global__ void m4_tables_kernel(const uint32_t *__restrict__ AC, int32_t RWp, int32_t NG,
                                 int64_t total, uint32_t *__restrict__ tab) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int b = (int)(idx & 255);
    const int64_t sg = idx >> 8;
    const int g = (int)(sg % NG), s = (int)(sg / NG);
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
    for (int i = 0; i < 8; ++i)
        if ((b >> i) & 1) {
            const uint4 a = *reinterpret_cast<const uint4 *>(AC + (size_t)(8 * g + i) * RWp + kM4Slice * s);
            acc.x ^= a.x;
            acc.y ^= a.y;
            acc.z ^= a.z;
            acc.w ^= a.w;
        }
    reinterpret_cast<uint4 *>(tab)[idx] = acc;
}

// Parity slice blockIdx.y of frames blockIdx.x * 256 + t (one per thread):
// the table block of each group is staged in shared memory (double-buffered,
// one 16-byte load per thread, one barrier per group) and the frame's
// information byte picks its row.  The 128 parity bits go to words
// 4 s .. 4 s + 3 of the frame's codeword row, used as scratch until the
// assembly kernel places every bit.
__global__ void __launch_bounds__(kM4Threads)
m4_lookup_kernel(const uint32_t *__restrict__ info, int32_t F, int32_t KW, int32_t NG,
                 const uint32_t *__restrict__ tab, uint32_t *__restrict__ code, int32_t NW) {
    __shared__ uint4 rows[2][256];
    const int tid = threadIdx.x, s = blockIdx.y;
    const int64_t f = (int64_t)blockIdx.x * kM4Threads + tid;
    const bool live = f < F;
    const uint4 *tb = reinterpret_cast<const uint4 *>(tab) + (size_t)s * NG * 256;
    uint4 next = NG > 0 ? __ldg(tb + tid) : make_uint4(0u, 0u, 0u, 0u);
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
    uint32_t word = 0;
    for (int g = 0; g < NG; ++g) {
        uint4 *buf = rows[g & 1];
        buf[tid] = next;
        __syncthreads();
        if (g + 1 < NG) next = __ldg(tb + (size_t)(g + 1) * 256 + tid);
        if ((g & 3) == 0) word = live ? __ldg(&info[f * KW + (g >> 2)]) : 0u;
        const uint4 t = buf[(word >> (8 * (g & 3))) & 0xFFu];
        acc.x ^= t.x;
        acc.y ^= t.y;
        acc.z ^= t.z;
        acc.w ^= t.w;
    }
    if (live) {
        uint32_t *out = code + f * NW + kM4Slice * s;
        out[0] = acc.x;
        out[1] = acc.y;
        out[2] = acc.z;
        out[3] = acc.w;
    }
}

// Places the information bits and the parity bits (from the scratch words at
// the start of each codeword row) at their positions, FT frames per block.
// All scratch reads of the block's rows precede the barrier; the rows are
// written after it.
template <int FT>
__global__ void __launch_bounds__(kEncThreads)
m4_assemble_kernel(const uint32_t *__restrict__ info, uint32_t *__restrict__ code,
                   const int32_t *__restrict__ info_pos, const int32_t *__restrict__ parity_pos,
                   int32_t F, int32_t k, int32_t rank, int32_t KW, int32_t NW) {
    extern __shared__ __align__(16) uint32_t cw[];  // [FT][NW]
    const int64_t f0 = (int64_t)blockIdx.x * FT;
    const int nf = (int)((int64_t)F - f0 < FT ? (int64_t)F - f0 : FT);
    const int RW = (rank + 31) >> 5;
    for (int idx = threadIdx.x; idx < FT * NW; idx += blockDim.x) cw[idx] = 0u;
    __syncthreads();
    for (int idx = threadIdx.x; idx < nf * KW; idx += blockDim.x) {
        const int f = idx / KW, w = idx - f * KW;
        uint32_t word = info[(f0 + f) * KW + w];
        if (w == KW - 1 && (k & 31)) word &= (1u << (k & 31)) - 1u;
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1u;
            const int p = info_pos[w * 32 + b];
            atomicOr(&cw[f * NW + (p >> 5)], 1u << (p & 31));
        }
    }
    for (int idx = threadIdx.x; idx < nf * RW; idx += blockDim.x) {
        const int f = idx / RW, q = idx - f * RW;
        uint32_t word = code[(f0 + f) * NW + q];
        if (q == RW - 1 && (rank & 31)) word &= (1u << (rank & 31)) - 1u;
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1u;
            const int p = parity_pos[q * 32 + b];
            atomicOr(&cw[f * NW + (p >> 5)], 1u << (p & 31));
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nf * NW; idx += blockDim.x) code[f0 * NW + idx] = cw[idx];
}

constexpr int kM4AsmFrames = 8;

// The table path applies when the tables exist and the scratch words fit in a
// codeword row.
bool m4_usable(const ldpc_code *c) {
    return c->d.enc_tab && kM4Slice * c->d.enc_ns <= c->NW &&
           (size_t)kM4AsmFrames * c->NW * sizeof(uint32_t) <= 200 * 1024;
}

int launch_m4(const ldpc_code *c, const uint32_t *d_info, uint32_t *d_code, int32_t F,
              cudaStream_t s) {
    const dim3 grid((unsigned)ceil_div(F, kM4Threads), (unsigned)c->d.enc_ns);
    m4_lookup_kernel<<<grid, kM4Threads, 0, s>>>(d_info, F, c->KW, c->d.enc_ng, c->d.enc_tab, d_code, c->NW);
    LDPC_TRY_CUDA(cudaGetLastError());
    const size_t sm = (size_t)kM4AsmFrames * c->NW * sizeof(uint32_t);
    LDPC_TRY(kernel_setup((const void *)m4_assemble_kernel<kM4AsmFrames>, kEncThreads, sm, nullptr));
    m4_assemble_kernel<kM4AsmFrames><<<(unsigned)ceil_div(F, kM4AsmFrames), kEncThreads, sm, s>>>(
        d_info, d_code, c->d.info_pos, c->d.parity_pos, F, c->k, c->rank, c->KW, c->NW);
    LDPC_TRY_CUDA(cudaGetLastError());
    return LDPC_OK;
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
    if (m4_usable(c)) return launch_m4(c, d_info, d_code, F, s);
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

void free_encode_tables(ldpc_code *c) {
    if (c->d.enc_tab) cudaFree(c->d.enc_tab);
    c->d.enc_tab = nullptr;
    c->d.enc_ns = c->d.enc_ng = 0;
    c->d.enc_tab_bytes = 0;
}

int build_encode_tables(ldpc_code *c, size_t *bytes) {
    free_encode_tables(c);
    if (bytes) *bytes = 0;
    if (c->k <= 0 || c->rank <= 0) return LDPC_OK;  // nothing to look up
    const int64_t NS = ceil_div(ceil_div(c->rank, 32), kM4Slice);
    const int64_t NG = ceil_div(c->k, 8);
    if (NS > 65535) return fail(LDPC_ENOTSUP, "rank %d too large for the table encoder", c->rank);
    if (kM4Slice * NS > c->NW)  // the lookup kernel's scratch must fit in a codeword row
        return fail(LDPC_ENOTSUP, "the table encoder needs 4 ceil(rank/128) <= ceil(n/32) (rank %d, n %d)",
                    c->rank, c->n);
    const int32_t RWp = (int32_t)(kM4Slice * NS), I8 = (int32_t)(8 * NG);
    const int64_t total = NS * NG * 256;  // table rows of 4 words
    const size_t tab_bytes = (size_t)total * kM4Slice * sizeof(uint32_t);
    uint32_t *AC = nullptr, *tab = nullptr;
    cudaError_t e = dev_malloc((void **)&AC, (size_t)I8 * RWp * sizeof(uint32_t));
    if (e != cudaSuccess) return fail(LDPC_ENOMEM, "column table allocation: %s", cudaGetErrorString(e));
    e = dev_malloc((void **)&tab, tab_bytes);
    if (e != cudaSuccess) {
        cudaFree(AC);
        return fail(LDPC_ENOMEM, "table allocation (%zu bytes): %s", tab_bytes, cudaGetErrorString(e));
    }
    const int64_t ncol = (int64_t)I8 * RWp;
    m4_columns_kernel<<<(unsigned)ceil_div(ncol, 256), 256>>>(c->d.AT, c->k, c->rank, I8, RWp, AC);
    m4_tables_kernel<<<(unsigned)ceil_div(total, 256), 256>>>(AC, RWp, (int32_t)NG, total, tab);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(AC);
    if (e != cudaSuccess) {
        cudaFree(tab);
        return fail(LDPC_ECUDA, "table build: %s", cudaGetErrorString(e));
    }
    c->d.enc_tab = tab;
    c->d.enc_ns = (int32_t)NS;
    c->d.enc_ng = (int32_t)NG;
    c->d.enc_tab_bytes = tab_bytes;
    if (bytes) *bytes = tab_bytes;
    return LDPC_OK;
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

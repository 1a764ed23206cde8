// K5: persistent decoder with whole frames resident in shared memory.
//
// The same flooding sum-product iteration as the plain decoder (Sec. II-B,
// Eqs. 5-8, Algorithm 1's schedule) and the same arithmetic (check_math.cuh),
// but every message of a frame stays on chip for all iterations: HBM is read
// once (the channel LLRs) and written once (outputs) per frame.  This is the
// paper's batch processing (Sec. III-C) mapped onto the GPU: each CTA takes
// frames from a global work counter and decodes them one group at a time.
//
// Per CTA (or per team of a CTA, see the mixed-code launch), for a group of
// G frames (G = 2 with binary16 messages, 1 with FP32 messages), shared
// memory holds, with P = n rounded up to a power of two:
//   E[r][P]  check messages, plane r = the r-th edge of each bit (in
//            ascending CSR edge order); half2 (both frames) or float
//   L[P][G]  total LLRs L_v of the G frames (float), a bit's G values
//            adjacent (one 8-byte access for a two-frame group)
//   R[P][G]  channel LLRs of regular codes, laid out like L
// All planes have a stride that is a multiple of 32 words, so an access to
// bit v falls in bank v mod 32 (bank pair v mod 16 for the 8-byte pairs).
// The check schedule (schedule.cpp) groups the checks of each warp and orders
// each check's edges so that at every step the 32 lanes touch 32 distinct
// banks.  An edge is a 16-bit slot s = r P + v: its message is at byte 4 s,
// its bit's totals at 4 G (s mod P) + the base of L.
//
// Thread t owns the checks of its (warp, slot) schedule groups and the bits
// t, t+T, ...: its checks' slots are loaded once into registers from a table
// built at code creation, and its bits' channel LLRs stay in registers while
// a group is decoded.
//
// Per iteration: check pass (each thread updates its checks' messages in
// place and, for early stop, evaluates the syndrome of the previous hard
// decisions), barrier, bit pass (L_v = R_v + the bit's messages in ascending
// edge order), barrier.
#include "mixed_core.cuh"
#include "resident_core.cuh"

namespace ldpc {
namespace {


template <class MsgT, int G, int DC, int CPT>
KernelFn pick_flags(bool reg, bool syn) {
    if (reg) return syn ? resident_kernel<MsgT, G, DC, CPT, true, true> : resident_kernel<MsgT, G, DC, CPT, true, false>;
    return syn ? resident_kernel<MsgT, G, DC, CPT, false, true> : resident_kernel<MsgT, G, DC, CPT, false, false>;
}

// Regular codes with binary16 messages -- the common long-code case -- also
// have instances with the plane size fixed at compile time (2^10 .. 2^13
// words); the results are the same bits.
KernelFn pick_fixed(int dc, int npad, bool syn) {
    int pl = 0;
    for (int k = 10; k <= 13; ++k)
        if (npad == (1 << k)) pl = k;
    switch (dc) {
        case 6: return resident_fixed_rows6(pl, syn);
        case 9: return resident_fixed_rows9(pl, syn);
        case 12: return resident_fixed_rows12(pl, syn);
        default: return nullptr;
    }
}

template <class MsgT, int G>
KernelFn pick_kernel(int dc, bool reg, bool syn) {
    switch (dc) {
        case 6: return pick_flags<MsgT, G, 6, 8>(reg, syn);
        case 9: return pick_flags<MsgT, G, 9, 6>(reg, syn);
        case 12: return pick_flags<MsgT, G, 12, 4>(reg, syn);
        case 16: return pick_flags<MsgT, G, 16, 3>(reg, syn);
        default: return nullptr;
    }
}

int pad_bits(const ldpc_code *c) {
    int p = 32;
    while (p < c->n) p *= 2;
    return p;
}

size_t res_smem(const ldpc_code *c, bool fp16, bool reg, int slots = kResSlots) {
    const int P = pad_bits(c);
    if (reg) return fp16 ? group_bytes<__half, 2, true>(P) : group_bytes<float, 1, true>(P);
    if (slots == kResSlotsWide)
        return fp16 ? group_bytes<__half, 2, false, kResSlotsWide>(P) : group_bytes<float, 1, false, kResSlotsWide>(P);
    return fp16 ? group_bytes<__half, 2, false>(P) : group_bytes<float, 1, false>(P);
}

// Message slots per bit of a code's resident layout: 4, or 9 for the
// wide-column instances (instantiated for rows of up to 12 edges, the paper's
// Table I codes with 6 or 9 ones per column); 0 if neither fits.
int res_slots(const ldpc_code *c) {
    if (c->dv_max <= kResSlots) return kResSlots;
    if (c->dv_max <= kResSlotsWide && c->dc_max > 9 && c->dc_max <= 12) return kResSlotsWide;
    return 0;
}

// Edge-slot table for a team of T threads: [CPT * DCW][T] 32-bit words, two
// 16-bit slots each.  Warp group g of the check schedule goes to warp
// g mod (T/32), check slot g / (T/32); lane u takes the group's u-th check,
// whose slots are listed in evaluation order.  The slot of an edge is r P + v,
// v its bit and r the edge's rank in v's column (ascending CSR edge order).
// Returns an empty table if the schedule needs more slots than CPT.  With
// `dummies` (the regular-code kernels), unused check slots of a regular code
// get dummy checks; otherwise they stay empty (kNoSlot), for the general
// kernels.
std::vector<uint32_t> build_slot_table(const ldpc_code *c, int dc, int cpt, int T, bool dummies = true) {
    const int DCW = (dc + 1) / 2;
    const int npad = pad_bits(c);
    const int warps = T / 32;
    std::vector<uint32_t> rank((size_t)c->nnz);
    for (int32_t v = 0; v < c->n; ++v)
        for (int32_t q = c->col_ptr[v]; q < c->col_ptr[v + 1]; ++q)
            rank[c->col_edge[q]] = (uint32_t)(q - c->col_ptr[v]);
    const bool reg = dummies && c->dc_min == dc && c->dc_max == dc && c->dv_min == 3 && c->dv_max == 3;
    std::vector<uint32_t> tab((size_t)cpt * DCW * T, 0xFFFFFFFFu);
    if (reg)
        for (size_t w = 0; w < (size_t)cpt * DCW; ++w)
            for (int t = 0; t < T; ++t) {
                const uint32_t d = 3u * (uint32_t)npad + (uint32_t)(t % 32);
                tab[w * T + t] = d | (d << 16);
            }
    const int ngroups = (int)(c->sched_groups.size() / 32);
    for (int g = 0; g < ngroups; ++g) {
        const int w = g % warps, k = g / warps;
        if (k >= cpt) return {};
        for (int u = 0; u < 32; ++u) {
            const int32_t chk = c->sched_groups[(size_t)g * 32 + u];
            if (chk < 0) continue;
            const int t = 32 * w + u;
            const int32_t e0 = c->row_ptr[chk], d = c->row_ptr[chk + 1] - e0;
            for (int j = 0; j < d; ++j) {
                const int32_t e = c->eval_edge[e0 + j];
                const uint32_t slot = rank[e] * (uint32_t)npad + (uint32_t)c->col_idx[e];
                uint32_t &word = tab[(size_t)(k * DCW + j / 2) * T + t];
                const int sh = (j & 1) * 16;
                word = (word & ~(0xFFFFu << sh)) | (slot << sh);
            }
        }
    }
    // dummy checks of regular codes: at every step, on the spare word whose
    // bank no real check of the warp touches at that step (spare word b sits in
    // bank b, like bit b), so they add no bank conflict
    if (reg)
        for (int k = 0; k < cpt; ++k)
            for (int w = 0; w < warps; ++w) {
                const int g = k * warps + w;
                for (int j = 0; j < dc; ++j) {
                    uint32_t used = 0;
                    for (int u = 0; u < 32; ++u) {
                        const int32_t chk = g < ngroups ? c->sched_groups[(size_t)g * 32 + u] : -1;
                        if (chk >= 0) used |= 1u << (c->col_idx[c->eval_edge[c->row_ptr[chk] + j]] & 31);
                    }
                    uint32_t b = 0;
                    for (int u = 0; u < 32; ++u) {
                        const int32_t chk = g < ngroups ? c->sched_groups[(size_t)g * 32 + u] : -1;
                        if (chk >= 0) continue;
                        while ((used >> b) & 1u) ++b;  // a free bank remains: at most 32 lanes
                        const uint32_t slot = 3u * (uint32_t)npad + b;
                        used |= 1u << b;
                        uint32_t &word = tab[(size_t)(k * DCW + j / 2) * T + 32 * w + u];
                        const int sh = (j & 1) * 16;
                        word = (word & ~(0xFFFFu << sh)) | (slot << sh);
                    }
                }
            }
    return tab;
}

const Shape *pick_shape(const ldpc_code *c) {
    // slots up to (slots - 1) P + n - 1 must stay below the 16-bit empty mark
    const int slots = res_slots(c);
    if (!slots || (int64_t)(slots - 1) * pad_bits(c) + c->n > 0xFFFE) return nullptr;
    for (const Shape &s : kShapes)
        if (s.dc >= c->dc_max) return &s;
    return nullptr;
}

// Threads per frame group: enough for the bits (kResVPT each) and for the
// checks with about 5 % spare check slots, which the check schedule uses to
// balance banks.
int team_threads(const ldpc_code *c, const Shape &s) {
    const int64_t need = std::max(ceil_div(c->m + c->m / 20 + 1, s.cpt), ceil_div(c->n, kResVPT));
    return (int)std::min<int64_t>(ceil_div(need, 32) * 32,
                                  std::max<int64_t>(kResMaxThreads, ceil_div(ceil_div(c->m, s.cpt), 32) * 32));
}

}  // namespace

// Warp groups the single-code resident launch offers (0 without a resident
// layout): the check schedule spreads the checks over all of them.
int resident_group_slots(const ldpc_code *c) {
    const Shape *shape = pick_shape(c);
    if (!shape) return 0;
    const int T = team_threads(c, *shape);
    if (T > kResMaxThreads) return 0;
    return (T / 32) * shape->cpt;
}

// Host-side plan of the single-code resident launch: row shape, thread count
// and slot table.
int build_resident_plan(ldpc_code *c) {
    ResidentPlan &p = c->res;
    p = ResidentPlan{};
    const Shape *shape = pick_shape(c);
    if (!shape) return LDPC_OK;
    const int T = team_threads(c, *shape);
    if (T > kResMaxThreads) return LDPC_OK;
    p.edges = build_slot_table(c, shape->dc, shape->cpt, T);
    if (p.edges.empty()) return LDPC_OK;
    p.dc_pad = shape->dc;
    p.dv_pad = res_slots(c);
    p.rows_pad = T;  // thread count of the launch
    // exactly dc edges per check and three per bit: the specialised kernels
    p.regular = c->dc_min == shape->dc && c->dc_max == shape->dc && c->dv_min == 3 && c->dv_max == 3;
    p.ok = true;
    // Small-batch plan: when there are fewer frames than SMs, each CTA has the
    // SM to itself, so the same schedule groups are spread over as many warps
    // as a CTA holds (at most 16), cutting the checks each thread runs in
    // sequence -- the critical path of an iteration -- from cpt to
    // ceil(groups / 16).  It runs the general (non-regular) kernel with empty
    // check slots skipped.  Every check keeps its evaluation order and every
    // bit its summation order, so the results are the same bits.
    const int ngroups = (int)(c->sched_groups.size() / 32);
    const int warps_max = kResMaxThreads / 32;
    const int per_thread = (int)ceil_div(ngroups, warps_max);
    const int warps = (int)ceil_div(ngroups, std::max(per_thread, 1));
    const int Tl = 32 * warps;
    if (ngroups > 0 && per_thread < shape->cpt && (int64_t)Tl * kResVPT >= c->n) {
        p.lat_edges = build_slot_table(c, shape->dc, shape->cpt, Tl, false);
        if (!p.lat_edges.empty()) p.lat_threads = Tl;
    }
    return LDPC_OK;
}

bool resident_fits(const ldpc_code *c, const ldpc_decode_opts *o) {
    if (!c->res.ok) return false;
    return res_smem(c, o->msg_fp16 != 0, c->res.regular, c->res.dv_pad) <= kSmemLimit;
}

size_t resident_workspace(const ldpc_code *, int32_t, const ldpc_decode_opts *) { return 256; }

int decode_resident(const ldpc_code *c, const float *d_llr, int32_t F, const ldpc_decode_opts *o,
                    float *d_post, uint32_t *d_hard, int32_t *d_iters, uint8_t *d_ok, void *d_work,
                    size_t work_bytes, cudaStream_t s) {
    if (!d_work || work_bytes < 256) return fail(LDPC_EINVAL, "workspace too small (need 256 bytes)");
    const bool fp16 = o->msg_fp16 != 0;
    const bool syn = o->early_stop != 0 && o->max_iters >= 2;
    KernelFn fn = nullptr;
    if (fp16 && c->res.regular) fn = pick_fixed(c->res.dc_pad, pad_bits(c), syn);
    if (c->res.dv_pad == kResSlotsWide) {
        if (c->res.dc_pad != 12) return fail(LDPC_ENOTSUP, "no wide-column resident kernel for rows of %d", c->res.dc_pad);
        fn = fp16 ? (syn ? resident_kernel<__half, 2, 12, 4, false, true, 0, kResSlotsWide>
                         : resident_kernel<__half, 2, 12, 4, false, false, 0, kResSlotsWide>)
                  : (syn ? resident_kernel<float, 1, 12, 4, false, true, 0, kResSlotsWide>
                         : resident_kernel<float, 1, 12, 4, false, false, 0, kResSlotsWide>);
    }
    if (!fn)
        fn = fp16 ? pick_kernel<__half, 2>(c->res.dc_pad, c->res.regular, syn)
                  : pick_kernel<float, 1>(c->res.dc_pad, c->res.regular, syn);
    if (!fn) return fail(LDPC_ENOTSUP, "no resident kernel for row degree %d", c->res.dc_pad);
    int sms = 0, per_sm = 0;
    LDPC_TRY(sm_count(&sms));
    int T = c->res.rows_pad;
    bool reg = c->res.regular;
    const uint32_t *edges = c->d.res_edges;
    if (!fp16 && c->res.lat_threads > 0 && F <= sms) {  // the small-batch plan
        reg = false;
        T = c->res.lat_threads;
        edges = c->d.lat_edges;
        fn = c->res.dv_pad == kResSlotsWide
                 ? (syn ? resident_kernel<float, 1, 12, 4, false, true, 0, kResSlotsWide>
                        : resident_kernel<float, 1, 12, 4, false, false, 0, kResSlotsWide>)
                 : pick_kernel<float, 1>(c->res.dc_pad, false, syn);
        if (!fn) return fail(LDPC_ENOTSUP, "no resident kernel for row degree %d", c->res.dc_pad);
    }
    const size_t smem = res_smem(c, fp16, reg, c->res.dv_pad);
    LDPC_TRY(kernel_setup((const void *)fn, T, smem, &per_sm));
    if (per_sm < 1) return fail(LDPC_ENOTSUP, "resident kernel cannot be resident (smem %zu B)", smem);
    const int G = fp16 ? 2 : 1;
    const int64_t groups = ceil_div(F, G);
    const int grid = (int)std::min<int64_t>(groups, (int64_t)sms * per_sm);
    ResArgs a;
    a.llr = d_llr;
    a.F = F;
    a.n = c->n;
    a.npad = pad_bits(c);
    a.m = c->m;
    a.NW = c->NW;
    a.T_iters = o->max_iters;
    a.early_stop = o->early_stop;
    a.clip2 = clip_log2(o->clip);
    a.edges = edges;
    a.post = d_post;
    a.hard = d_hard;
    a.iters = d_iters;
    a.ok = d_ok;
    a.counter = static_cast<unsigned *>(d_work);
    LDPC_TRY_CUDA(cudaMemsetAsync(d_work, 0, sizeof(unsigned), s));
    fn<<<grid, T, smem, s>>>(a);
    LDPC_TRY_CUDA(cudaGetLastError());
    return LDPC_OK;
}

}  // namespace ldpc

// ---------------------------------------------------------------------------
// Mixed-code batches: frames of several codes in one persistent launch.
//
// Each code of the plan is decoded by teams of T_c threads (T_c a power of two
// <= 512, from the code's resident shape); a 512-thread CTA holds 512 / T_c
// teams (as many as its shared memory allows), each decoding its own group of
// G frames with its own named barrier, so a CTA works on many frames of a
// small code or on one group of the largest.  Frames are bucketed by code on
// the device (count, offsets, scatter), and CTAs take work items -- a CTA-full
// of groups of one code -- from a counter, codes with the most edges first by
// default.  Every step is a kernel or a memset on the caller's stream, so the
// call can be captured in a CUDA graph.  Results per frame do not depend on
// the bucketing or the configuration: each frame's arithmetic is that of the
// single-code decoder.
namespace ldpc {
namespace {

__global__ void mixed_count(const int32_t *__restrict__ frame_code, int32_t F, int32_t ncodes,
                            unsigned *__restrict__ count, int32_t *__restrict__ iters,
                            uint8_t *__restrict__ ok) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int c = frame_code[f];
    if (c < 0 || c >= ncodes) {  // not decoded: marked with iters = -1, ok = 0
        if (iters) iters[f] = -1;
        if (ok) ok[f] = 0;
        return;
    }
    atomicAdd(&count[c], 1u);
}

__global__ void mixed_offsets(const unsigned *__restrict__ count, const MixedDesc *__restrict__ desc,
                              int32_t ncodes, int32_t G, int32_t gpi, unsigned *__restrict__ start,
                              unsigned *__restrict__ item_off, unsigned *__restrict__ fill) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned fo = 0, io = 0;
    for (int p = 0; p < ncodes; ++p) {
        const int c = desc[p].code;
        start[c] = fo;
        fill[c] = 0;
        item_off[p] = io;
        const unsigned groups = (count[c] + G - 1) / G;
        const unsigned per_item = (unsigned)(desc[p].teams * gpi);
        io += (groups + per_item - 1) / per_item;
        fo += count[c];
    }
    item_off[ncodes] = io;
}

__global__ void mixed_scatter(const int32_t *__restrict__ frame_code, int32_t F, int32_t ncodes,
                              const unsigned *__restrict__ start, unsigned *__restrict__ fill,
                              int32_t *__restrict__ sorted) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int c = frame_code[f];
    if (c < 0 || c >= ncodes) return;
    sorted[start[c] + atomicAdd(&fill[c], 1u)] = (int32_t)f;
}

// Channel quality of each frame: the mean |R_v| of its first (up to) 1024
// bits (for BPSK over AWGN it grows with Eb/N0), one warp per frame.  Frames of
// poor quality are the ones likely to run every iteration.
__global__ void mixed_score(const int32_t *__restrict__ frame_code, const int64_t *__restrict__ llr_off,
                            const float *__restrict__ llr, const int32_t *__restrict__ nbits, int32_t F,
                            int32_t ncodes, float *__restrict__ score) {
    const int64_t f = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (f >= F) return;
    const int c = frame_code[f];
    if (c < 0 || c >= ncodes) return;
    const int n = min(nbits[c], 1024);
    const float *x = llr + llr_off[f];
    float sum = 0.f;
#pragma unroll 8
    for (int v = lane; v < n; v += 32) sum += fabsf(x[v]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) score[f] = sum / (float)n;
}

// Orders each code's bucket by channel quality, poorest first (ties by frame
// index), one CTA per code: a frame's rank is the number of frames before it.
// The work items then start with the frame groups most likely to run every
// iteration, and the two frames of a binary16 group have similar quality, so a
// group rarely waits for one slow frame.  The order changes no result.
constexpr int kSortCap = 4096;  // larger buckets keep their arrival order

// Orders one code's bucket of frames by (score, frame index) ascending: a
// bitonic sort of 64-bit keys (the score's bits above the frame index; scores
// are non-negative, so their bit patterns order like the values) in shared
// memory, the bucket padded to a power of two with keys above every real one.
__global__ void __launch_bounds__(512) mixed_sort(const unsigned *__restrict__ start,
                                                  const unsigned *__restrict__ count,
                                                  const float *__restrict__ score, int32_t *__restrict__ sorted) {
    __shared__ unsigned long long key[kSortCap];
    const int c = blockIdx.x;
    const unsigned n = count[c], st = start[c];
    if (n < 2 || n > kSortCap) return;
    unsigned P = 2;
    while (P < n) P <<= 1;
    for (unsigned i = threadIdx.x; i < P; i += blockDim.x) {
        if (i < n) {
            const int32_t f = sorted[st + i];
            key[i] = ((unsigned long long)__float_as_uint(score[f]) << 32) | (uint32_t)f;
        } else {
            key[i] = ~0ull;
        }
    }
    __syncthreads();
    for (unsigned k = 2; k <= P; k <<= 1)
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            for (unsigned i = threadIdx.x; i < P; i += blockDim.x) {
                const unsigned l = i ^ j;
                if (l > i) {
                    const unsigned long long x = key[i], y = key[l];
                    if ((x > y) == ((i & k) == 0)) {  // ascending where bit k of i is 0
                        key[i] = y;
                        key[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) sorted[st + i] = (int32_t)(uint32_t)key[i];
}


}  // namespace
}  // namespace ldpc

// A shape class of a plan: the codes with one row weight and (binary16
// messages, planes of 2^10..2^13 words) one plane size, decoded by one kernel
// instance; in work order they hold the positions [pb, pe).
struct MixedClass {
    int dc = 0, pl = 0, pb = 0, pe = 0;
    size_t smem = 0;
};

struct ldpc_mixed {
    int32_t ncodes = 0;
    bool fp16 = true;
    int device = -1;
    std::vector<const ldpc_code *> codes;
    std::vector<ldpc::MixedDesc> host_desc;   // in code order
    std::vector<uint32_t *> tables;           // device slot tables, per code
    ldpc::MixedDesc *d_desc = nullptr;        // device, in work order
    int32_t *d_nbits = nullptr;               // device, n of each code (by code index)
    ldpc_mixed_config cfg{0, 1, 1};
    int32_t desc_order = -1;                  // cfg.order the device array holds
    std::vector<MixedClass> classes;          // in work order (for desc_order)
    // classes after the first run on these streams, forked from and joined
    // to the caller's stream by events
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
};

namespace ldpc {
namespace {

// Plane-size exponent of a code's kernel instance (0: size at run time).
int mixed_plane_log(const MixedDesc &d, bool fp16) {
    if (!fp16) return 0;
    for (int pl = 10; pl <= 13; ++pl)
        if (d.npad == (1 << pl)) return pl;
    return 0;
}

// Work order: the codes (largest first, or as given), then grouped by shape
// class with the classes in the order of their first code, so that each
// class is one run of positions.
int upload_order(ldpc_mixed *p, int32_t order) {
    std::vector<MixedDesc> d(p->host_desc);
    if (order == LDPC_MIXED_ORDER_LARGEST_FIRST)
        std::stable_sort(d.begin(), d.end(), [&](const MixedDesc &a, const MixedDesc &b) {
            return p->codes[a.code]->nnz > p->codes[b.code]->nnz;
        });
    std::vector<std::pair<int, int>> keys;  // (dc, pl) in order of first appearance
    auto key_of = [&](const MixedDesc &x) { return std::make_pair(x.dc, mixed_plane_log(x, p->fp16)); };
    for (const MixedDesc &x : d)
        if (std::find(keys.begin(), keys.end(), key_of(x)) == keys.end()) keys.push_back(key_of(x));
    auto rank = [&](const MixedDesc &x) { return std::find(keys.begin(), keys.end(), key_of(x)) - keys.begin(); };
    std::stable_sort(d.begin(), d.end(), [&](const MixedDesc &a, const MixedDesc &b) { return rank(a) < rank(b); });
    std::vector<MixedClass> cls(keys.size());
    for (size_t k = 0; k < keys.size(); ++k) {
        cls[k].dc = keys[k].first;
        cls[k].pl = keys[k].second;
        cls[k].pb = (int)d.size();
    }
    for (int pos = 0; pos < (int)d.size(); ++pos) {
        MixedClass &c = cls[rank(d[pos])];
        c.pb = std::min(c.pb, pos);
        c.pe = pos + 1;
        c.smem = std::max(c.smem, (size_t)d[pos].teams * res_smem(p->codes[d[pos].code], p->fp16, true));
    }
    LDPC_TRY_CUDA(cudaMemcpy(p->d_desc, d.data(), sizeof(MixedDesc) * d.size(), cudaMemcpyHostToDevice));
    p->classes = cls;
    p->desc_order = order;
    return LDPC_OK;
}

MixedFn mixed_fn(int dc, bool fp16, bool syn, int pl) {
    switch (dc) {
        case 6: return mixed_fn_rows6(fp16, syn, pl);
        case 9: return mixed_fn_rows9(fp16, syn, pl);
        case 12: return mixed_fn_rows12(fp16, syn, pl);
        default: return nullptr;
    }
}

struct MixedWs {
    unsigned *count, *fill, *start, *item_off, *counter;  // counter: one per shape class
    int32_t *sorted;
    float *score;
};

size_t mixed_layout(int32_t ncodes, int32_t F, MixedWs *w, void *base) {
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += align256(b);
        return o;
    };
    const size_t oC = take(sizeof(unsigned) * ncodes);
    const size_t oF = take(sizeof(unsigned) * ncodes);
    const size_t oS = take(sizeof(unsigned) * ncodes);
    const size_t oI = take(sizeof(unsigned) * (ncodes + 1));
    const size_t oK = take(sizeof(unsigned) * kMixMaxClasses);
    const size_t oX = take(sizeof(int32_t) * std::max(F, 1));
    const size_t oQ = take(sizeof(float) * std::max(F, 1));
    if (w && base) {
        char *b = static_cast<char *>(base);
        w->count = reinterpret_cast<unsigned *>(b + oC);
        w->fill = reinterpret_cast<unsigned *>(b + oF);
        w->start = reinterpret_cast<unsigned *>(b + oS);
        w->item_off = reinterpret_cast<unsigned *>(b + oI);
        w->counter = reinterpret_cast<unsigned *>(b + oK);
        w->sorted = reinterpret_cast<int32_t *>(b + oX);
        w->score = reinterpret_cast<float *>(b + oQ);
    }
    return off;
}

}  // namespace
}  // namespace ldpc

using namespace ldpc;

extern "C" {

int ldpc_mixed_create(const ldpc_code *const *codes, int32_t ncodes, int32_t msg_fp16,
                      ldpc_mixed **out) {
    if (!out) return fail(LDPC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!codes || ncodes < 1 || ncodes > 4096) return fail(LDPC_EINVAL, "need 1..4096 codes");
    if (msg_fp16 != 0 && msg_fp16 != 1) return fail(LDPC_EINVAL, "msg_fp16 must be 0 or 1");
    int dev = -1;
    LDPC_TRY_CUDA(cudaGetDevice(&dev));
    ldpc_mixed *p = new (std::nothrow) ldpc_mixed();
    if (!p) return fail(LDPC_ENOMEM, "host allocation failed");
    p->ncodes = ncodes;
    p->fp16 = msg_fp16 != 0;
    p->device = dev;
    const int G = p->fp16 ? 2 : 1;
    auto cleanup = [&](int st) {
        ldpc_mixed_destroy(p);
        return st;
    };
    for (int32_t i = 0; i < ncodes; ++i) {
        const ldpc_code *c = codes[i];
        if (!c || !c->on_device || c->device != dev) return cleanup(fail(LDPC_EINVAL, "code %d is missing or not on this device", i));
        const Shape *sh = pick_shape(c);
        if (!sh || !c->res.ok || !c->res.regular || sh->dc > 12)
            return cleanup(fail(LDPC_ENOTSUP, "code %d is not a regular column-weight-3 code with row weight 6, 9 or 12", i));
        int team = 32;
        while (team < team_threads(c, *sh)) team *= 2;
        if (team > kMixThreads) return cleanup(fail(LDPC_ENOTSUP, "code %d is too long for a mixed batch", i));
        const size_t tb = res_smem(c, G == 2, true);
        const int teams = std::min<int>(kMixThreads / team, (int)(kSmemLimit / tb));
        if (teams < 1) return cleanup(fail(LDPC_ENOTSUP, "code %d does not fit in shared memory", i));
        std::vector<uint32_t> tab = build_slot_table(c, sh->dc, sh->cpt, team);
        if (tab.empty()) return cleanup(fail(LDPC_ENOTSUP, "code %d: no slot table for team %d", i, team));
        uint32_t *dt = nullptr;
        cudaError_t err = dev_malloc((void **)&dt, sizeof(uint32_t) * tab.size());
        if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaMalloc(mixed slot table)"));
        p->tables.push_back(dt);
        err = cudaMemcpy(dt, tab.data(), sizeof(uint32_t) * tab.size(), cudaMemcpyHostToDevice);
        if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaMemcpy(mixed slot table)"));
        p->codes.push_back(c);
        p->host_desc.push_back(MixedDesc{c->n, pad_bits(c), sh->dc, team, teams, i, dt});
    }
    cudaError_t err = dev_malloc((void **)&p->d_desc, sizeof(MixedDesc) * ncodes);
    if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaMalloc(mixed descriptors)"));
    err = dev_malloc((void **)&p->d_nbits, sizeof(int32_t) * ncodes);
    if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaMalloc(mixed code sizes)"));
    {
        std::vector<int32_t> nb(ncodes);
        for (int32_t i = 0; i < ncodes; ++i) nb[i] = codes[i]->n;
        err = cudaMemcpy(p->d_nbits, nb.data(), sizeof(int32_t) * ncodes, cudaMemcpyHostToDevice);
        if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaMemcpy(mixed code sizes)"));
    }
    int st = upload_order(p, p->cfg.order);
    if (st != LDPC_OK) return cleanup(st);
    if (p->classes.size() > (size_t)kMixMaxClasses) return cleanup(fail(LDPC_ENOTSUP, "too many shape classes"));
    if (p->classes.size() > 1) {
        err = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
        if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaEventCreate(mixed fork)"));
        for (size_t k = 1; k < p->classes.size(); ++k) {
            cudaStream_t cs = nullptr;
            err = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaStreamCreate(mixed class)"));
            p->streams.push_back(cs);
            cudaEvent_t ev = nullptr;
            err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaEventCreate(mixed join)"));
            p->joins.push_back(ev);
        }
    }
    *out = p;
    return LDPC_OK;
}

void ldpc_mixed_destroy(ldpc_mixed *p) {
    if (!p) return;
    for (uint32_t *t : p->tables) cudaFree(t);
    if (p->d_desc) cudaFree(p->d_desc);
    if (p->d_nbits) cudaFree(p->d_nbits);
    for (cudaStream_t cs : p->streams) cudaStreamDestroy(cs);
    for (cudaEvent_t ev : p->joins) cudaEventDestroy(ev);
    if (p->fork) cudaEventDestroy(p->fork);
    delete p;
}

int ldpc_mixed_workspace_size(const ldpc_mixed *p, int32_t F, size_t *bytes) {
    if (!p || !bytes || F < 0) return fail(LDPC_EINVAL, "bad arguments");
    *bytes = mixed_layout(p->ncodes, F, nullptr, nullptr);
    return LDPC_OK;
}

int ldpc_mixed_get_config(const ldpc_mixed *p, ldpc_mixed_config *cfg) {
    if (!p || !cfg) return fail(LDPC_EINVAL, "bad arguments");
    *cfg = p->cfg;
    return LDPC_OK;
}

int ldpc_mixed_set_config(ldpc_mixed *p, const ldpc_mixed_config *cfg) {
    if (!p || !cfg) return fail(LDPC_EINVAL, "bad arguments");
    if (cfg->order < 0 || cfg->order > 1 || cfg->groups_per_item < 1 || cfg->groups_per_item > 64 ||
        cfg->ctas_per_sm < 1 || cfg->ctas_per_sm > 4)
        return fail(LDPC_EINVAL, "configuration out of range");
    if (cfg->order != p->desc_order) LDPC_TRY(upload_order(p, cfg->order));
    p->cfg = *cfg;
    return LDPC_OK;
}

int ldpc_decode_mixed(const ldpc_mixed *p, const int32_t *d_frame_code, const int64_t *d_llr_off,
                      const int64_t *d_hard_off, const float *d_llr, int32_t F, int32_t max_iters,
                      int32_t early_stop, float clip, float *d_post, uint32_t *d_hard,
                      int32_t *d_iters, uint8_t *d_ok, void *d_work, size_t work_bytes,
                      ldpc_stream_t stream) {
    TraceRange trace_("ldpc_decode_mixed");
    if (!p) return fail(LDPC_EINVAL, "plan is NULL");
    if (F < 0 || max_iters < 0 || !(clip > 0.f)) return fail(LDPC_EINVAL, "bad F, max_iters or clip");
    if (early_stop != 0 && early_stop != 1) return fail(LDPC_EINVAL, "early_stop must be 0 or 1");
    if (F == 0) return LDPC_OK;
    if (!d_frame_code || !d_llr_off || !d_llr || (d_hard && !d_hard_off))
        return fail(LDPC_EINVAL, "NULL pointer");
    int dev = -1;
    LDPC_TRY_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return fail(LDPC_EINVAL, "plan lives on device %d", p->device);
    MixedWs w{};
    const size_t need = mixed_layout(p->ncodes, F, &w, d_work);
    if (!d_work || work_bytes < need) return fail(LDPC_EINVAL, "workspace too small (%zu < %zu)", work_bytes, need);
    cudaStream_t s = (cudaStream_t)stream;
    const int G = p->fp16 ? 2 : 1;
    LDPC_TRY_CUDA(cudaMemsetAsync(w.count, 0, sizeof(unsigned) * p->ncodes, s));
    LDPC_TRY_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(unsigned) * kMixMaxClasses, s));
    const unsigned fb = (unsigned)ceil_div(F, 256);
    mixed_count<<<fb, 256, 0, s>>>(d_frame_code, F, p->ncodes, w.count, d_iters, d_ok);
    mixed_offsets<<<1, 32, 0, s>>>(w.count, p->d_desc, p->ncodes, G, p->cfg.groups_per_item, w.start,
                                   w.item_off, w.fill);
    mixed_scatter<<<fb, 256, 0, s>>>(d_frame_code, F, p->ncodes, w.start, w.fill, w.sorted);
    mixed_score<<<(unsigned)ceil_div(F, 8), 256, 0, s>>>(d_frame_code, d_llr_off, d_llr, p->d_nbits, F, p->ncodes,
                                                          w.score);
    mixed_sort<<<(unsigned)p->ncodes, 512, 0, s>>>(w.start, w.count, w.score, w.sorted);
    const bool syn = early_stop && max_iters >= 2;
    int sms = 0;
    LDPC_TRY(sm_count(&sms));
    MixedArgs a;
    a.desc = p->d_desc;
    a.ncodes = p->ncodes;
    a.item_off = w.item_off;
    a.start = w.start;
    a.count = w.count;
    a.sorted = w.sorted;
    a.llr_off = d_llr_off;
    a.hard_off = d_hard_off;
    a.llr = d_llr;
    a.post = d_post;
    a.hard = d_hard;
    a.iters = d_iters;
    a.ok = d_ok;
    a.T_iters = max_iters;
    a.gpi = p->cfg.groups_per_item;
    a.clip2 = clip_log2(clip);
    // one persistent kernel per shape class, in work order: the first on the
    // caller's stream, the others on the plan's streams, which wait for the
    // steps above and are joined back; a later class's CTAs take the SMs that
    // an earlier class's CTAs leave
    if (p->classes.size() > 1) LDPC_TRY_CUDA(cudaEventRecord(p->fork, s));
    for (size_t k = 0; k < p->classes.size(); ++k) {
        const MixedClass &cl = p->classes[k];
        MixedFn fn = mixed_fn(cl.dc, p->fp16, syn, cl.pl);
        if (!fn) return fail(LDPC_ENOTSUP, "no mixed kernel for rows of %d", cl.dc);
        int per_sm = 0;
        LDPC_TRY(kernel_setup((const void *)fn, kMixThreads, cl.smem, &per_sm));
        if (per_sm < 1) return fail(LDPC_ENOTSUP, "mixed kernel cannot be resident");
        MixedArgs ak = a;
        ak.pb = cl.pb;
        ak.pe = cl.pe;
        ak.counter = w.counter + k;
        const int grid = sms * std::min(per_sm, p->cfg.ctas_per_sm);
        cudaStream_t ks = s;
        if (k > 0) {
            ks = p->streams[k - 1];
            LDPC_TRY_CUDA(cudaStreamWaitEvent(ks, p->fork, 0));
        }
        fn<<<grid, kMixThreads, cl.smem, ks>>>(ak);
        LDPC_TRY_CUDA(cudaGetLastError());
        if (k > 0) {
            LDPC_TRY_CUDA(cudaEventRecord(p->joins[k - 1], ks));
            LDPC_TRY_CUDA(cudaStreamWaitEvent(s, p->joins[k - 1], 0));
        }
    }
    LDPC_TRY_CUDA(cudaGetLastError());
    return LDPC_OK;
}

int ldpc_mixed_autotune(ldpc_mixed *p, const int32_t *d_frame_code, const int64_t *d_llr_off,
                        const int64_t *d_hard_off, const float *d_llr, int32_t F, int32_t max_iters,
                        int32_t early_stop, float clip, float *d_post, uint32_t *d_hard,
                        int32_t *d_iters, uint8_t *d_ok, void *d_work, size_t work_bytes,
                        int32_t reps, ldpc_stream_t stream, ldpc_mixed_config *chosen) {
    TraceRange trace_("ldpc_mixed_autotune");
    if (!p || reps < 1) return fail(LDPC_EINVAL, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const ldpc_mixed_config start = p->cfg;
    std::vector<ldpc_mixed_config> cands;
    for (int order = 0; order <= 1; ++order)
        for (int gpi : {1, 2, 4})
            for (int cps : {1, 2}) cands.push_back({order, gpi, cps});
    // Each candidate's call is captured in a CUDA graph on a private stream,
    // the way a serving loop replays it (eager launches of the shape classes
    // are scheduled differently), and timed replay by replay: `reps` replays
    // after an untimed one, in two passes over the candidates (the second in
    // reverse order, so that no candidate always runs first, on a GPU still
    // raising its clocks).  The lowest median of a candidate's 2 x reps times
    // wins.  One eager call first does the per-kernel set-up outside capture;
    // the private stream starts after the work queued on `stream`.
    cudaStream_t cs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LDPC_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t cerr = cudaEventCreate(&e0);
    if (cerr == cudaSuccess) cerr = cudaEventCreate(&e1);
    if (cerr == cudaSuccess) cerr = cudaEventRecord(e0, s);
    if (cerr == cudaSuccess) cerr = cudaStreamWaitEvent(cs, e0, 0);
    int st = cerr == cudaSuccess ? LDPC_OK : cuda_fail(cerr, "autotune stream set-up");
    if (st == LDPC_OK)
        st = ldpc_decode_mixed(p, d_frame_code, d_llr_off, d_hard_off, d_llr, F, max_iters, early_stop, clip, d_post,
                               d_hard, d_iters, d_ok, d_work, work_bytes, (ldpc_stream_t)cs);
    std::vector<std::vector<float>> times(cands.size());
    for (int pass = 0; pass < 2 && st == LDPC_OK; ++pass)
        for (size_t ci = 0; ci < cands.size() && st == LDPC_OK; ++ci) {
            const size_t c = pass == 0 ? ci : cands.size() - 1 - ci;
            if ((st = ldpc_mixed_set_config(p, &cands[c])) != LDPC_OK) break;
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            cudaError_t err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (err != cudaSuccess) {
                st = cuda_fail(err, "cudaStreamBeginCapture(autotune)");
                break;
            }
            const int dst = ldpc_decode_mixed(p, d_frame_code, d_llr_off, d_hard_off, d_llr, F, max_iters,
                                              early_stop, clip, d_post, d_hard, d_iters, d_ok, d_work, work_bytes,
                                              (ldpc_stream_t)cs);
            err = cudaStreamEndCapture(cs, &graph);
            if (dst != LDPC_OK)
                st = dst;
            else if (err != cudaSuccess)
                st = cuda_fail(err, "cudaStreamEndCapture(autotune)");
            else if ((err = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess)
                st = cuda_fail(err, "cudaGraphInstantiate(autotune)");
            for (int r = -1; r < reps && st == LDPC_OK; ++r) {
                cudaEventRecord(e0, cs);
                err = cudaGraphLaunch(exec, cs);
                cudaEventRecord(e1, cs);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                if (err != cudaSuccess) {
                    st = cuda_fail(err, "graph replay (autotune)");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r >= 0) times[c].push_back(ms);
            }
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
        }
    float best = 1e30f;
    ldpc_mixed_config best_cfg = start;
    for (size_t c = 0; c < cands.size() && st == LDPC_OK; ++c) {
        std::vector<float> &t = times[c];
        std::sort(t.begin(), t.end());
        const float med = t.empty() ? 1e30f : t[t.size() / 2];
        if (med < best) {
            best = med;
            best_cfg = cands[c];
        }
    }
    if (st == LDPC_OK) {
        const cudaError_t err = cudaStreamSynchronize(cs);
        if (err != cudaSuccess) st = cuda_fail(err, "cudaStreamSynchronize(autotune)");
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(cs);
    if (st != LDPC_OK) {
        ldpc_mixed_set_config(p, &start);
        return st;
    }
    LDPC_TRY(ldpc_mixed_set_config(p, &best_cfg));
    if (chosen) *chosen = best_cfg;
    return LDPC_OK;
}

}  // extern "C"

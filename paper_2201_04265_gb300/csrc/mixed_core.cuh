// K6 mixed-code batches: the argument block shared by the host side
// (decode_resident.cu) and the kernels, and the kernel of one row shape.
//
// A plan's codes are grouped into shape classes -- row weight and, for
// binary16 messages with planes of 2^10..2^13 words, the plane size -- and
// each class has its own persistent kernel, instantiated in its own
// translation unit (rows6.cu, rows9.cu, rows12.cu).  With
// the decode of a group inlined into a kernel of one shape, the register
// allocation is that of the single-code resident kernel; a kernel holding all
// shapes (inlined, or as called functions) spilled inside the check pass.
#pragma once

#include "resident_core.cuh"

namespace ldpc {

constexpr int kMixThreads = 512;
constexpr int kMixMaxClasses = 16;  // 3 row weights x (4 fixed plane sizes + run-time size), rounded up

struct MixedDesc {
    int32_t n, npad, dc, team, teams, code;
    const uint32_t *edges;  // [cpt * DCW][team]
};

struct MixedArgs {
    const MixedDesc *desc;      // by work-order position
    int32_t ncodes;
    int32_t pb, pe;             // positions of this launch's shape class: [pb, pe)
    const unsigned *item_off;   // [ncodes + 1], by position
    const unsigned *start;      // [ncodes], by code: first slot in `sorted`
    const unsigned *count;      // [ncodes], by code
    const int32_t *sorted;      // frame indices grouped by code
    const int64_t *llr_off, *hard_off;
    const float *llr;
    float *post;
    uint32_t *hard;
    int32_t *iters;
    uint8_t *ok;
    unsigned *counter;          // this class's work counter
    int32_t T_iters, gpi;
    float clip2;
};

using MixedFn = void (*)(MixedArgs);

// The kernel of one shape class: rows of dc (6, 9 or 12) edges, binary16
// (two-frame groups) or FP32 messages, planes of 2^pl words (pl = 10..13,
// binary16 only) or of a size given at run time (pl = 0).
MixedFn mixed_fn_rows6(bool fp16, bool syn, int pl);
MixedFn mixed_fn_rows9(bool fp16, bool syn, int pl);
MixedFn mixed_fn_rows12(bool fp16, bool syn, int pl);

namespace {

// Where a mixed group's frames come from and go to (by the sorted bucket).
template <int G>
struct MixIO {
    const MixedArgs &a;
    unsigned first, cnt, st;  // group's first index in the code's bucket
    __device__ bool exists(int i) const { return first + i < cnt; }
    __device__ int f(int i) const { return a.sorted[st + first + i]; }
    __device__ const float *llr(int i) const { return a.llr + a.llr_off[f(i)]; }
    __device__ float *post(int i) const { return a.post ? a.post + a.llr_off[f(i)] : nullptr; }
    __device__ uint32_t *hard(int i) const { return a.hard ? a.hard + a.hard_off[f(i)] : nullptr; }
    __device__ int32_t *iters(int i) const { return a.iters ? a.iters + f(i) : nullptr; }
    __device__ uint8_t *ok(int i) const { return a.ok ? a.ok + f(i) : nullptr; }
};

// One work item of a team: gpi groups of G frames of the item's code.
template <class MsgT, int G, int DC, int CPT, bool SYN, int PL>
__device__ __forceinline__ void mixed_run(const SubTeam &tm, const MixedDesc &d, const MixedArgs &a,
                                          unsigned char *base, unsigned local) {
    constexpr int DCW = (DC + 1) / 2;
    uint32_t idx[CPT][DCW];
#pragma unroll
    for (int k = 0; k < CPT; ++k)
#pragma unroll
        for (int w = 0; w < DCW; ++w) idx[k][w] = __ldg(&d.edges[(size_t)(k * DCW + w) * d.team + tm.tid()]);
    const Smem<MsgT, G, true, PL> sm = smem_at<MsgT, G, true, PL>(base, d.npad);
    const unsigned cnt = a.count[d.code], st = a.start[d.code];
    const int team = tm.base / d.team;
    for (int gi = 0; gi < a.gpi; ++gi) {
        const unsigned grp = (local * a.gpi + gi) * d.teams + team;
        if ((size_t)grp * G >= cnt) break;
        const MixIO<G> io{a, grp * G, cnt, st};
        decode_group<MsgT, G, DC, CPT, true, SYN>(tm, idx, sm, d.n, d.npad, io, a.T_iters, a.clip2);
    }
}

// Persistent kernel of one shape class: CTAs take work items (a CTA-full of
// groups of one code) of the positions [a.pb, a.pe) from the class counter.
template <class MsgT, int G, int DC, int CPT, bool SYN, int PL>
__global__ void __launch_bounds__(kMixThreads)
mixed_kernel(MixedArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned s_item;
    const unsigned ib = a.item_off[a.pb], ie = a.item_off[a.pe];
    for (;;) {
        if (threadIdx.x == 0) s_item = ib + atomicAdd(a.counter, 1u);
        __syncthreads();
        const unsigned item = s_item;
        __syncthreads();
        if (item >= ie) break;
        int p = a.pb;
        while (item >= a.item_off[p + 1]) ++p;
        const MixedDesc d = a.desc[p];
        const int team = threadIdx.x / d.team;
        if (team < d.teams) {
            const SubTeam tm{team * d.team, d.team, 1 + team};
            unsigned char *base = smem_raw + (size_t)team * group_bytes<MsgT, G, true>(d.npad);
            mixed_run<MsgT, G, DC, CPT, SYN, PL>(tm, d, a, base, item - a.item_off[p]);
        }
        __syncthreads();
    }
}

template <int DC, int CPT, int PL>
MixedFn mixed_pick_half(bool syn) {
    return syn ? mixed_kernel<__half, 2, DC, CPT, true, PL> : mixed_kernel<__half, 2, DC, CPT, false, PL>;
}

template <int DC, int CPT>
MixedFn mixed_pick(bool fp16, bool syn, int pl) {
    if (!fp16) return syn ? mixed_kernel<float, 1, DC, CPT, true, 0> : mixed_kernel<float, 1, DC, CPT, false, 0>;
    switch (pl) {
        case 10: return mixed_pick_half<DC, CPT, 10>(syn);
        case 11: return mixed_pick_half<DC, CPT, 11>(syn);
        case 12: return mixed_pick_half<DC, CPT, 12>(syn);
        case 13: return mixed_pick_half<DC, CPT, 13>(syn);
        default: return mixed_pick_half<DC, CPT, 0>(syn);
    }
}

}  // namespace
}  // namespace ldpc

// Internal declarations shared by the translation units of libldpc.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <climits>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ldpc.h"

namespace ldpc {

// Sets the calling thread's error message and returns `status`.
int fail(int status, const char *fmt, ...);
// Converts a CUDA error into LDPC_ECUDA with a message naming `what`.
int cuda_fail(cudaError_t err, const char *what);

#define LDPC_TRY_CUDA(expr)                                      \
    do {                                                         \
        cudaError_t _e = (expr);                                 \
        if (_e != cudaSuccess) return ::ldpc::cuda_fail(_e, #expr); \
    } while (0)

#define LDPC_TRY(expr)              \
    do {                            \
        int _s = (expr);            \
        if (_s != LDPC_OK) return _s; \
    } while (0)

// Every device allocation of the library goes through here, so that a test
// can make one fail on the host (ldpc_test_fail_allocation) and check that the
// caller returns LDPC_ENOMEM and frees what it took.
cudaError_t dev_malloc(void **p, size_t bytes);

// A named range on the host timeline for profilers (NVTX, domain "ldpc"):
// each entry point that queues work marks its span, so a timeline shows
// which call issued which kernels.  Costs nothing when no tool is attached.
class TraceRange {
   public:
    explicit TraceRange(const char *name) {
        nvtxEventAttributes_t a = {};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(domain(), &a);
    }
    ~TraceRange() { nvtxDomainRangePop(domain()); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;

   private:
    static nvtxDomainHandle_t domain() {
        static nvtxDomainHandle_t d = nvtxDomainCreateA("ldpc");
        return d;
    }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
// The message clip in the kernels' log2 units.
inline float clip_log2(float clip) { return (float)((double)clip * 1.4426950408889634); }

// Degree classes of the plain decoder: each class of checks (bits) is
// updated by a kernel instance sized for its largest degree.
constexpr int kRowClasses = 6;
constexpr int kRowClassMax[kRowClasses] = {6, 8, 12, 16, 32, INT32_MAX};
constexpr int kColClasses = 4;
constexpr int kColClassMax[kColClasses] = {4, 8, 16, INT32_MAX};
inline int row_class_of(int d) {
    int q = 0;
    while (d > kRowClassMax[q]) ++q;
    return q;
}
inline int col_class_of(int d) {
    int q = 0;
    while (d > kColClassMax[q]) ++q;
    return q;
}

// Device-side tables of a code (all owned by the code object).
struct DeviceCode {
    int32_t *row_ptr = nullptr;    // [m+1]
    int32_t *col_idx = nullptr;    // [E]  check-major edge -> bit
    int32_t *col_ptr = nullptr;    // [n+1]
    int32_t *col_edge = nullptr;   // [E]  bit-major list of edge ids (ascending)
    int32_t *info_pos = nullptr;   // [k]
    int32_t *parity_pos = nullptr; // [rank]
    int32_t *eval_col = nullptr;  // [E]  column at each evaluation position
    int32_t *eval_edge = nullptr; // [E]  CSR edge id at each evaluation position
    int32_t *col_pos = nullptr;   // [E]  evaluation position of col_edge[q]
    uint32_t *AT = nullptr;       // [KW][rank] parity map, word-major
    int32_t *row_order = nullptr; // [m] checks grouped by degree class (plain decoder)
    int32_t *col_order = nullptr; // [n] bits grouped by degree class (plain decoder)
    // resident decoder tables (see decode_resident.cu)
    uint32_t *res_edges = nullptr; // resident slot table of the single-code launch
    int32_t res_edges_len = 0;
    uint32_t *lat_edges = nullptr; // slot table of the small-batch (latency) launch
    int32_t *cl_tab_half = nullptr;    // cluster-decoder tables (binary16 / FP32 messages)
    int32_t *cl_tab_single = nullptr;
    // Four-Russians encoding tables (encode.cu), built on request:
    // [enc_ns][enc_ng][256][4] words, 0 = not built
    uint32_t *enc_tab = nullptr;
    int32_t enc_ns = 0, enc_ng = 0;
    size_t enc_tab_bytes = 0;
};

// Resident-decoder plan: how one frame's checks and bits are laid out in
// shared memory (built on the host at create time).
struct ResidentPlan {
    bool ok = false;          // the code has a resident layout
    bool regular = false;     // every row has dc_pad edges and every column 3
    int32_t dc_pad = 0;       // row degree padded to an instantiated shape
    int32_t dv_pad = 0;       // message slots per bit (16-byte records)
    int32_t rows_pad = 0;     // threads per CTA of the resident launch
    int32_t lat_threads = 0;  // threads per CTA of the small-batch launch, 0 = none
    std::vector<uint32_t> lat_edges;  // its slot table, same form as `edges`
    std::vector<uint32_t> edges; // [cpt * ceil(dc_pad/2)][threads] 16-bit slot pairs
};

// Quasi-cyclic description kept from creation (z = 0 when H came as CSR).
struct QcInfo {
    int32_t mb = 0, nb = 0, z = 0;
    std::vector<int16_t> shift;  // [mb][nb], -1 = zero block
};

// Cluster-decoder launch shape for one message type (decode_cluster.cu).
struct ClusterCfg {
    int32_t C = 0;              // CTAs per cluster, 0 = no plan
    int32_t G = 0;              // frames per group
    uint32_t e_bytes = 0;       // message planes per CTA
    uint32_t l_bytes = 0;       // total planes per CTA
    int32_t internal = 0;       // base entries whose row and column share a CTA
    int32_t entries = 0;        // base entries
    int32_t sec_words = 0;      // words of the largest per-CTA table section
    size_t smem = 0;            // dynamic shared memory per CTA
    std::vector<int32_t> tab;   // table blob every CTA copies into shared memory
};

}  // namespace ldpc

struct ldpc_code {
    int32_t n = 0, m = 0, k = 0, rank = 0;
    int64_t nnz = 0;
    int32_t KW = 0, NW = 0, MW = 0;  // words per info word, codeword, syndrome
    int32_t dc_max = 0, dv_max = 0, dc_min = 0, dv_min = 0;
    std::vector<int32_t> row_ptr, col_idx, col_ptr, col_edge, info_pos, parity_pos;
    std::vector<uint32_t> A;  // [rank][KW]
    // check evaluation order (shared by every decoder; see schedule.cpp):
    // positions row_ptr[c]..row_ptr[c+1]-1 hold check c's edges in the order
    // its inputs are combined
    std::vector<int32_t> eval_edge, eval_col, col_pos, pos_of_edge;
    std::vector<int32_t> sched_groups;  // [ceil(m/32)][32] checks per warp group, -1 = none
    int64_t sched_excess = 0;           // edges above d_c per (group, bank): 0 = conflict-free
    // checks (bits) grouped by degree class, ascending index within a class;
    // class q holds row_order[row_class[q] .. row_class[q+1]-1]
    std::vector<int32_t> row_order, col_order;
    int32_t row_class[ldpc::kRowClasses + 1] = {}, col_class[ldpc::kColClasses + 1] = {};
    bool on_device = false;
    int device = -1;
    ldpc::DeviceCode d;
    ldpc::ResidentPlan res;
    ldpc::QcInfo qc;
    ldpc::ClusterCfg cl_half, cl_single;  // binary16 / FP32 messages
};

namespace ldpc {
int build_check_schedule(ldpc_code *c, int ngroups);  // schedule.cpp
int resident_group_slots(const ldpc_code *c);       // decode_resident.cu
// Sets a kernel's dynamic shared-memory limit (once per kernel and device)
// and returns its resident CTAs per SM for the launch shape (cached), so that
// launchers make no attribute calls on the repeat calls a CUDA graph captures.
int kernel_setup(const void *fn, int threads, size_t smem, int *per_sm);
int sm_count(int *sms);
// Kernel launchers (defined in the .cu files).
int build_encode_tables(ldpc_code *c, size_t *bytes);
void free_encode_tables(ldpc_code *c);
int launch_encode(const ldpc_code *c, const uint32_t *d_info, uint32_t *d_code, int32_t F,
                  cudaStream_t s);
int launch_syndrome(const ldpc_code *c, const uint32_t *d_bits, int32_t F, uint32_t *d_syn,
                    uint8_t *d_ok, cudaStream_t s);
int build_cluster_plan(ldpc_code *c);                                 // decode_cluster.cu
bool cluster_fits(const ldpc_code *c, const ldpc_decode_opts *o);
int decode_cluster(const ldpc_code *c, const float *d_llr, int32_t F, const ldpc_decode_opts *o,
                   float *d_post, uint32_t *d_hard, int32_t *d_iters, uint8_t *d_ok, void *d_work,
                   size_t work_bytes, cudaStream_t s);
size_t plain_workspace(const ldpc_code *c, int32_t F, const ldpc_decode_opts *o);
int decode_plain(const ldpc_code *c, const float *d_llr, int32_t F, const ldpc_decode_opts *o,
                 float *d_post, uint32_t *d_hard, int32_t *d_iters, uint8_t *d_ok, void *d_work,
                 size_t work_bytes, cudaStream_t s);
}  // namespace ldpc

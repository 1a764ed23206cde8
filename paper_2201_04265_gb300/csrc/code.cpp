// Code objects: validation of H, Tanner-graph edge layouts (Sec. II-B,
// Fig. 1) and the systematic generator (Eq. 2, Sec. III-B) by bit-packed
// GF(2) Gauss-Jordan elimination.  Host code, run once per code.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <thread>

#include "ldpc_internal.h"

namespace ldpc {

static thread_local std::string g_last_error;

// Allocations left before the injected failure; < 0: no failure pending.
static std::atomic<int64_t> g_fail_after{-1};

cudaError_t dev_malloc(void **p, size_t bytes) {
    int64_t left = g_fail_after.load();
    while (left >= 0) {
        if (g_fail_after.compare_exchange_weak(left, left - 1)) {
            if (left == 0) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;  // the injected failure; the hook is spent
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

int fail(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

int cuda_fail(cudaError_t err, const char *what) {
    return fail(err == cudaErrorMemoryAllocation ? LDPC_ENOMEM : LDPC_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorName(err), cudaGetErrorString(err));
}

namespace {

// Spin barrier for the elimination worker threads (one use per pivot).
class SpinBarrier {
   public:
    explicit SpinBarrier(int n) : n_(n) {}
    void wait() {
        int gen = gen_.load(std::memory_order_acquire);
        if (count_.fetch_add(1, std::memory_order_acq_rel) + 1 == n_) {
            count_.store(0, std::memory_order_relaxed);
            gen_.fetch_add(1, std::memory_order_acq_rel);
        } else {
            while (gen_.load(std::memory_order_acquire) == gen) std::this_thread::yield();
        }
    }

   private:
    const int n_;
    std::atomic<int> count_{0};
    std::atomic<int> gen_{0};
};

// Reduced row echelon form of H over GF(2), pivot columns taken from the
// right.  Rows are packed 64 bits per word.  On return rows[0..rank) are the
// pivot rows in the order found (pivot columns descending) and piv[] their
// pivot columns.  Work is split over threads by rows for large matrices.
int32_t rref_right_to_left(int32_t m, int32_t n, std::vector<uint64_t> &rows,
                           std::vector<int32_t> &piv) {
    const int32_t W = (n + 63) / 64;
    piv.clear();
    int nthreads = 1;
    if ((int64_t)m * W > (int64_t)1 << 18) {
        unsigned hc = std::thread::hardware_concurrency();
        nthreads = (int)std::min<unsigned>(hc ? hc : 1, 32);
    }
    int32_t rank = 0;
    auto bit = [&](int32_t r, int32_t col) -> bool {
        return (rows[(size_t)r * W + (col >> 6)] >> (col & 63)) & 1u;
    };
    // shared state for the workers of one pivot step
    std::atomic<bool> stop{false};
    int32_t cur_col = -1, cur_row = -1;
    SpinBarrier start(nthreads), done(nthreads);
    auto eliminate = [&](int tid) {
        // zero column cur_col in every row except the pivot row
        const int32_t wc = cur_col >> 6;
        const uint64_t mask = (uint64_t)1 << (cur_col & 63);
        const uint64_t *p = &rows[(size_t)cur_row * W];
        for (int32_t r = tid; r < m; r += nthreads) {
            if (r == cur_row) continue;
            uint64_t *q = &rows[(size_t)r * W];
            if (!(q[wc] & mask)) continue;
            for (int32_t w = 0; w < W; ++w) q[w] ^= p[w];
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nthreads; ++t)
        pool.emplace_back([&, t] {
            for (;;) {
                start.wait();
                if (stop.load()) return;
                eliminate(t);
                done.wait();
            }
        });
    for (int32_t col = n - 1; col >= 0 && rank < m; --col) {
        int32_t r = -1;
        for (int32_t i = rank; i < m; ++i)
            if (bit(i, col)) {
                r = i;
                break;
            }
        if (r < 0) continue;
        if (r != rank)
            std::swap_ranges(rows.begin() + (size_t)r * W, rows.begin() + (size_t)(r + 1) * W,
                             rows.begin() + (size_t)rank * W);
        cur_col = col;
        cur_row = rank;
        if (nthreads > 1) start.wait();
        eliminate(0);
        if (nthreads > 1) done.wait();
        piv.push_back(col);
        ++rank;
    }
    if (nthreads > 1) {
        stop.store(true);
        start.wait();
        for (auto &t : pool) t.join();
    }
    return rank;
}

int build_host(ldpc_code *c) {
    const int32_t n = c->n, m = c->m;
    const int64_t E = c->nnz;
    // bit-major edge lists
    c->col_ptr.assign((size_t)n + 1, 0);
    for (int64_t e = 0; e < E; ++e) c->col_ptr[c->col_idx[e] + 1]++;
    for (int32_t v = 0; v < n; ++v) c->col_ptr[v + 1] += c->col_ptr[v];
    c->col_edge.resize((size_t)E);
    {
        std::vector<int32_t> fill(c->col_ptr.begin(), c->col_ptr.end() - 1);
        for (int64_t e = 0; e < E; ++e) c->col_edge[fill[c->col_idx[e]]++] = (int32_t)e;
    }
    c->dc_max = 0;
    c->dc_min = INT32_MAX;
    for (int32_t r = 0; r < m; ++r) {
        int32_t d = c->row_ptr[r + 1] - c->row_ptr[r];
        c->dc_max = std::max(c->dc_max, d);
        c->dc_min = std::min(c->dc_min, d);
    }
    c->dv_max = 0;
    c->dv_min = INT32_MAX;
    for (int32_t v = 0; v < n; ++v) {
        int32_t d = c->col_ptr[v + 1] - c->col_ptr[v];
        c->dv_max = std::max(c->dv_max, d);
        c->dv_min = std::min(c->dv_min, d);
    }
    // degree classes of the plain decoder
    {
        auto group = [](int32_t count, const std::vector<int32_t> &ptr, int nclass, int (*cls)(int),
                        std::vector<int32_t> &order, int32_t *off) {
            std::vector<int32_t> cnt((size_t)nclass + 1, 0);
            for (int32_t i = 0; i < count; ++i) cnt[cls(ptr[i + 1] - ptr[i]) + 1]++;
            for (int q = 0; q < nclass; ++q) cnt[q + 1] += cnt[q];
            for (int q = 0; q <= nclass; ++q) off[q] = cnt[q];
            order.resize((size_t)count);
            for (int32_t i = 0; i < count; ++i) order[cnt[cls(ptr[i + 1] - ptr[i])]++] = i;
        };
        group(m, c->row_ptr, kRowClasses, row_class_of, c->row_order, c->row_class);
        group(n, c->col_ptr, kColClasses, col_class_of, c->col_order, c->col_class);
    }
    // systematic generator
    const int32_t W = (n + 63) / 64;
    std::vector<uint64_t> rows((size_t)m * W, 0);
    for (int32_t r = 0; r < m; ++r)
        for (int32_t e = c->row_ptr[r]; e < c->row_ptr[r + 1]; ++e) {
            int32_t v = c->col_idx[e];
            rows[(size_t)r * W + (v >> 6)] |= (uint64_t)1 << (v & 63);
        }
    std::vector<int32_t> piv;
    const int32_t rank = rref_right_to_left(m, n, rows, piv);
    if (rank >= n) return fail(LDPC_EINVAL, "rank(H) = n: the code has no information bits");
    c->rank = rank;
    c->k = n - rank;
    c->KW = (int32_t)ceil_div(c->k, 32);
    c->NW = (int32_t)ceil_div(n, 32);
    c->MW = (int32_t)ceil_div(m, 32);
    std::vector<char> is_piv((size_t)n, 0);
    for (int32_t p : piv) is_piv[p] = 1;
    c->info_pos.clear();
    for (int32_t v = 0; v < n; ++v)
        if (!is_piv[v]) c->info_pos.push_back(v);
    c->parity_pos.resize((size_t)rank);
    c->A.assign((size_t)rank * c->KW, 0u);
    for (int32_t j = 0; j < rank; ++j) {
        // pivots were found with descending columns: ascending order reverses them
        const int32_t src = rank - 1 - j;
        c->parity_pos[j] = piv[src];
        const uint64_t *row = &rows[(size_t)src * W];
        uint32_t *a = &c->A[(size_t)j * c->KW];
        for (int32_t i = 0; i < c->k; ++i) {
            int32_t v = c->info_pos[i];
            if ((row[v >> 6] >> (v & 63)) & 1u) a[i >> 5] |= 1u << (i & 31);
        }
    }
    return LDPC_OK;
}

template <class T>
int upload(T **dst, const T *src, size_t count) {
    if (count == 0) count = 1;  // keep a valid, non-null allocation
    LDPC_TRY_CUDA(dev_malloc((void **)dst, count * sizeof(T)));
    if (src) LDPC_TRY_CUDA(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
    return LDPC_OK;
}

void free_device(ldpc_code *c) {
    void *ptrs[] = {c->d.row_ptr,   c->d.col_idx,    c->d.col_ptr,  c->d.col_edge,
                    c->d.info_pos,  c->d.parity_pos, c->d.AT,       c->d.res_edges,  c->d.lat_edges,
                    c->d.eval_col,  c->d.eval_edge,  c->d.col_pos,  c->d.row_order,
                    c->d.col_order, c->d.enc_tab,    c->d.cl_tab_half, c->d.cl_tab_single};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    c->d = DeviceCode{};
}

}  // namespace

int build_resident_plan(ldpc_code *c);  // decode_resident.cu

namespace {

// A quasi-cyclic code created from its base matrix combines each check's
// inputs in ascending column order: the z checks of a base row then visit
// their circulants in the same order, so the lanes of a warp that update z
// consecutive checks read consecutive bits at every step (the cluster
// decoder's access pattern).  The count of edges outside a bank-conflict-free
// step of the resident schedule groups is recomputed for this order.
void lifted_check_order(ldpc_code *c) {
    for (int64_t e = 0; e < c->nnz; ++e) c->eval_edge[e] = (int32_t)e;
    int64_t excess = 0;
    const int ngroups = (int)(c->sched_groups.size() / 32);
    for (int g = 0; g < ngroups; ++g)
        for (int j = 0; j < c->dc_max; ++j) {
            uint32_t seen = 0;
            for (int u = 0; u < 32; ++u) {
                const int32_t chk = c->sched_groups[(size_t)g * 32 + u];
                if (chk < 0 || c->row_ptr[chk] + j >= c->row_ptr[chk + 1]) continue;
                const uint32_t bit = 1u << (c->col_idx[c->row_ptr[chk] + j] & 31);
                if (seen & bit) ++excess;
                seen |= bit;
            }
        }
    c->sched_excess = excess;
}

}  // namespace

int upload_code(ldpc_code *c) {
    LDPC_TRY_CUDA(cudaGetDevice(&c->device));
    LDPC_TRY(upload(&c->d.row_ptr, c->row_ptr.data(), c->row_ptr.size()));
    LDPC_TRY(upload(&c->d.col_idx, c->col_idx.data(), c->col_idx.size()));
    LDPC_TRY(upload(&c->d.col_ptr, c->col_ptr.data(), c->col_ptr.size()));
    LDPC_TRY(upload(&c->d.col_edge, c->col_edge.data(), c->col_edge.size()));
    LDPC_TRY(upload(&c->d.info_pos, c->info_pos.data(), c->info_pos.size()));
    LDPC_TRY(upload(&c->d.parity_pos, c->parity_pos.data(), c->parity_pos.size()));
    LDPC_TRY(upload(&c->d.eval_col, c->eval_col.data(), c->eval_col.size()));
    LDPC_TRY(upload(&c->d.eval_edge, c->eval_edge.data(), c->eval_edge.size()));
    LDPC_TRY(upload(&c->d.col_pos, c->col_pos.data(), c->col_pos.size()));
    LDPC_TRY(upload(&c->d.row_order, c->row_order.data(), c->row_order.size()));
    LDPC_TRY(upload(&c->d.col_order, c->col_order.data(), c->col_order.size()));
    std::vector<uint32_t> AT((size_t)c->KW * c->rank);
    for (int32_t j = 0; j < c->rank; ++j)
        for (int32_t w = 0; w < c->KW; ++w) AT[(size_t)w * c->rank + j] = c->A[(size_t)j * c->KW + w];
    LDPC_TRY(upload(&c->d.AT, AT.data(), AT.size()));
    if (c->res.ok) {
        LDPC_TRY(upload(&c->d.res_edges, c->res.edges.data(), c->res.edges.size()));
        c->d.res_edges_len = (int32_t)c->res.edges.size();
        if (c->res.lat_threads > 0)
            LDPC_TRY(upload(&c->d.lat_edges, c->res.lat_edges.data(), c->res.lat_edges.size()));
    }
    if (c->cl_half.C) LDPC_TRY(upload(&c->d.cl_tab_half, c->cl_half.tab.data(), c->cl_half.tab.size()));
    if (c->cl_single.C) LDPC_TRY(upload(&c->d.cl_tab_single, c->cl_single.tab.data(), c->cl_single.tab.size()));
    c->on_device = true;
    return LDPC_OK;
}

}  // namespace ldpc

using namespace ldpc;

extern "C" {

const char *ldpc_status_string(int s) {
    switch (s) {
        case LDPC_OK: return "LDPC_OK";
        case LDPC_EINVAL: return "LDPC_EINVAL: invalid argument";
        case LDPC_ENOMEM: return "LDPC_ENOMEM: out of memory";
        case LDPC_ECUDA: return "LDPC_ECUDA: CUDA error";
        case LDPC_ETIMEOUT: return "LDPC_ETIMEOUT: bounded wait expired";
        case LDPC_ENOTSUP: return "LDPC_ENOTSUP: not supported";
        default: return "LDPC: unknown status";
    }
}

const char *ldpc_last_error(void) { return g_last_error.c_str(); }

int ldpc_test_fail_allocation(int32_t after) {
    g_fail_after.store(after < 0 ? -1 : (int64_t)after);
    return LDPC_OK;
}

int ldpc_code_create(int32_t n, int32_t m, const int32_t *row_ptr, const int32_t *col_idx,
                     const ldpc_qc_desc *qc, uint32_t flags, ldpc_code **out) {
    if (!out) return fail(LDPC_EINVAL, "out is NULL");
    *out = nullptr;
    if (flags & ~LDPC_CREATE_HOST_ONLY) return fail(LDPC_EINVAL, "unknown flags 0x%x", flags);
    std::vector<int32_t> rp, ci;
    if (qc) {
        if (row_ptr || col_idx) return fail(LDPC_EINVAL, "give either CSR arrays or a QC description");
        if (qc->mb < 1 || qc->nb < 1 || qc->z < 1 || !qc->shift)
            return fail(LDPC_EINVAL, "bad QC description");
        if ((int64_t)qc->nb * qc->z != n || (int64_t)qc->mb * qc->z != m)
            return fail(LDPC_EINVAL, "QC sizes disagree with n, m");
        rp.reserve((size_t)m + 1);
        rp.push_back(0);
        for (int32_t i = 0; i < qc->mb; ++i) {
            for (int32_t r = 0; r < qc->z; ++r) {
                std::vector<int32_t> cols;
                for (int32_t j = 0; j < qc->nb; ++j) {
                    int16_t s = qc->shift[(size_t)i * qc->nb + j];
                    if (s < -1 || s >= qc->z) return fail(LDPC_EINVAL, "QC shift out of range");
                    if (s >= 0) cols.push_back(j * qc->z + (r + s) % qc->z);
                }
                std::sort(cols.begin(), cols.end());
                ci.insert(ci.end(), cols.begin(), cols.end());
                rp.push_back((int32_t)ci.size());
            }
        }
    } else {
        if (!row_ptr || !col_idx) return fail(LDPC_EINVAL, "row_ptr/col_idx is NULL");
        if (n < 1 || m < 1) return fail(LDPC_EINVAL, "need n >= 1 and m >= 1 (n=%d, m=%d)", n, m);
        if (row_ptr[0] != 0) return fail(LDPC_EINVAL, "row_ptr[0] must be 0");
        for (int32_t r = 0; r < m; ++r) {
            if (row_ptr[r + 1] < row_ptr[r]) return fail(LDPC_EINVAL, "row_ptr not monotone at row %d", r);
            for (int32_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
                if (col_idx[e] < 0 || col_idx[e] >= n)
                    return fail(LDPC_EINVAL, "column %d out of range in row %d", col_idx[e], r);
                if (e > row_ptr[r] && col_idx[e] <= col_idx[e - 1])
                    return fail(LDPC_EINVAL, "columns of row %d not strictly increasing", r);
            }
        }
        rp.assign(row_ptr, row_ptr + m + 1);
        ci.assign(col_idx, col_idx + row_ptr[m]);
    }
    ldpc_code *c = new (std::nothrow) ldpc_code();
    if (!c) return fail(LDPC_ENOMEM, "host allocation failed");
    c->n = n;
    c->m = m;
    c->nnz = (int64_t)ci.size();
    c->row_ptr = std::move(rp);
    c->col_idx = std::move(ci);
    if (qc) {
        c->qc.mb = qc->mb;
        c->qc.nb = qc->nb;
        c->qc.z = qc->z;
        c->qc.shift.assign(qc->shift, qc->shift + (size_t)qc->mb * qc->nb);
    }
    int st = build_host(c);
    if (st == LDPC_OK) st = build_check_schedule(c, resident_group_slots(c));
    if (st == LDPC_OK && qc) lifted_check_order(c);
    if (st == LDPC_OK) {
        // derived evaluation-order arrays
        c->eval_col.resize((size_t)c->nnz);
        c->pos_of_edge.resize((size_t)c->nnz);
        for (int64_t p = 0; p < c->nnz; ++p) {
            c->eval_col[p] = c->col_idx[c->eval_edge[p]];
            c->pos_of_edge[c->eval_edge[p]] = (int32_t)p;
        }
        c->col_pos.resize((size_t)c->nnz);
        for (int64_t q = 0; q < c->nnz; ++q) c->col_pos[q] = c->pos_of_edge[c->col_edge[q]];
        st = build_resident_plan(c);
    }
    if (st == LDPC_OK) st = build_cluster_plan(c);
    if (st == LDPC_OK && !(flags & LDPC_CREATE_HOST_ONLY)) {
        st = upload_code(c);
        if (st != LDPC_OK) free_device(c);
    }
    if (st != LDPC_OK) {
        delete c;
        return st;
    }
    *out = c;
    return LDPC_OK;
}

int ldpc_code_info(const ldpc_code *c, int32_t *n, int32_t *m, int32_t *k, int32_t *rank,
                   int64_t *nnz) {
    if (!c) return fail(LDPC_EINVAL, "code is NULL");
    if (n) *n = c->n;
    if (m) *m = c->m;
    if (k) *k = c->k;
    if (rank) *rank = c->rank;
    if (nnz) *nnz = c->nnz;
    return LDPC_OK;
}

int ldpc_code_positions(const ldpc_code *c, int32_t *info_pos, int32_t *parity_pos) {
    if (!c) return fail(LDPC_EINVAL, "code is NULL");
    if (info_pos) std::copy(c->info_pos.begin(), c->info_pos.end(), info_pos);
    if (parity_pos) std::copy(c->parity_pos.begin(), c->parity_pos.end(), parity_pos);
    return LDPC_OK;
}

int ldpc_code_schedule(const ldpc_code *c, int32_t *eval_edge, int64_t *unplaced) {
    if (!c) return fail(LDPC_EINVAL, "code is NULL");
    if (eval_edge) std::copy(c->eval_edge.begin(), c->eval_edge.end(), eval_edge);
    if (unplaced) *unplaced = c->sched_excess;
    return LDPC_OK;
}

int ldpc_code_parity_map(const ldpc_code *c, uint32_t *A) {
    if (!c || !A) return fail(LDPC_EINVAL, "code or A is NULL");
    std::copy(c->A.begin(), c->A.end(), A);
    return LDPC_OK;
}

void ldpc_code_destroy(ldpc_code *c) {
    if (!c) return;
    if (c->on_device) {
        int prev = -1;
        cudaGetDevice(&prev);
        if (prev != c->device) cudaSetDevice(c->device);
        free_device(c);
        if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    }
    delete c;
}

}  // extern "C"

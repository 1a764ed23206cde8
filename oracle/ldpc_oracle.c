/*
 * ldpc_oracle.c -- plain FP64 CPU restatement of the paper's method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU
 * baseline leg of bench.py load this code; the CUDA library never does, and
 * it shares no code, header or table with the library.  It is written to be
 * checked against the paper by eye, not to be fast.
 *
 * What it computes (arXiv 2201.04265):
 *   - oracle_systematic: the generator in standard form [I_k : P] (Eq. 2 and
 *     Sec. III-B "Encoding"): GF(2) Gauss-Jordan elimination of H scanning
 *     pivot columns from right to left, so that H = [X | I] gives the
 *     information positions 0..k-1 as in Fig. 2.
 *   - oracle_encode: m^T G = p^T (Eq. 3) in systematic form: information bits
 *     copied to their positions, parity bit j = XOR of the information bits
 *     selected by row j of A = P^T.
 *   - oracle_syndrome: H z^T over GF(2) (Eq. 1).
 *   - oracle_decode: flooding sum-product decoding (Sec. II-B, Algorithm 1's
 *     schedule without the MPI split): check-node update Eq. 5, read as
 *     E_cv = -2 atanh( prod_{v' != v} tanh(-L_v'c / 2) ), which carries the
 *     (-1)^{d_c} factor that the paper's LLR sign (Eq. 4, ln p(1)/p(0))
 *     needs; variable-node update Eq. 6; total LLR Eq. 7; hard decision Eq. 8
 *     (tie L_v = 0 decides 1).  Additions not in the paper: |message| clipping
 *     (inputs to and outputs of the check update), an optional syndrome
 *     early stop checked after every iteration, and an optional weight per
 *     edge and iteration multiplying E_cv in Eqs. 6 and 7 (weighted BP).
 *
 * Parity status: every function here is pinned by the not-gpu tests
 * (worked examples of Figs. 1-2, closed-form rational LLRs, brute-force
 * bitwise MAP on cycle-free codes, invariants).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- GF(2) -- */

static int get_bit(const uint64_t *row, int32_t j) { return (int)((row[j >> 6] >> (j & 63)) & 1u); }

/* Returns 0 on success, -1 on bad input or allocation failure, -2 if the A
 * buffer is too small.  A is written rank x k, row-major, one byte per bit:
 * A[j*k + i] = coefficient of information bit i in parity bit j. */
int oracle_systematic(int32_t m, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                      int32_t *rank_out, int32_t *info_pos, int32_t *parity_pos, uint8_t *A,
                      int64_t A_capacity) {
    if (m < 0 || n <= 0) return -1;
    int32_t W = (n + 63) / 64;
    uint64_t *rows = (uint64_t *)calloc((size_t)(m > 0 ? m : 1) * W, sizeof(uint64_t));
    int32_t *pivcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    uint8_t *is_pivot = (uint8_t *)calloc((size_t)n, 1);
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
    if (!rows || !pivcol || !is_pivot || !tmp) { free(rows); free(pivcol); free(is_pivot); free(tmp); return -1; }
    for (int32_t c = 0; c < m; ++c)
        for (int32_t e = row_ptr[c]; e < row_ptr[c + 1]; ++e) {
            int32_t v = col_idx[e];
            if (v < 0 || v >= n) { free(rows); free(pivcol); free(is_pivot); free(tmp); return -1; }
            rows[(size_t)c * W + (v >> 6)] ^= (uint64_t)1 << (v & 63);
        }
    int32_t rank = 0;
    for (int32_t col = n - 1; col >= 0 && rank < m; --col) {
        int32_t r = -1;
        for (int32_t i = rank; i < m; ++i)
            if (get_bit(rows + (size_t)i * W, col)) { r = i; break; }
        if (r < 0) continue;
        if (r != rank) {
            memcpy(tmp, rows + (size_t)r * W, sizeof(uint64_t) * W);
            memcpy(rows + (size_t)r * W, rows + (size_t)rank * W, sizeof(uint64_t) * W);
            memcpy(rows + (size_t)rank * W, tmp, sizeof(uint64_t) * W);
        }
        const uint64_t *prow = rows + (size_t)rank * W;
        for (int32_t i = 0; i < m; ++i) {
            if (i == rank) continue;
            uint64_t *ri = rows + (size_t)i * W;
            if (get_bit(ri, col))
                for (int32_t w = 0; w < W; ++w) ri[w] ^= prow[w];
        }
        pivcol[rank] = col;
        is_pivot[col] = 1;
        ++rank;
    }
    int32_t k = n - rank;
    if ((int64_t)rank * k > A_capacity) { free(rows); free(pivcol); free(is_pivot); free(tmp); return -2; }
    int32_t ni = 0;
    for (int32_t v = 0; v < n; ++v)
        if (!is_pivot[v]) info_pos[ni++] = v;
    /* pivots were found right to left, so ascending parity positions are the
     * pivot rows taken in reverse order */
    for (int32_t j = 0; j < rank; ++j) {
        const uint64_t *prow = rows + (size_t)(rank - 1 - j) * W;
        parity_pos[j] = pivcol[rank - 1 - j];
        for (int32_t i = 0; i < k; ++i) A[(size_t)j * k + i] = (uint8_t)get_bit(prow, info_pos[i]);
    }
    *rank_out = rank;
    free(rows); free(pivcol); free(is_pivot); free(tmp);
    return 0;
}

void oracle_encode(int32_t n, int32_t k, const int32_t *info_pos, const int32_t *parity_pos,
                   const uint8_t *A, const uint8_t *msg, int32_t F, uint8_t *cw) {
    int32_t r = n - k;
    for (int32_t f = 0; f < F; ++f) {
        const uint8_t *mf = msg + (size_t)f * k;
        uint8_t *cf = cw + (size_t)f * n;
        for (int32_t i = 0; i < k; ++i) cf[info_pos[i]] = mf[i] & 1;
        for (int32_t j = 0; j < r; ++j) {
            uint8_t p = 0;
            for (int32_t i = 0; i < k; ++i) p ^= (uint8_t)(A[(size_t)j * k + i] & mf[i] & 1);
            cf[parity_pos[j]] = p;
        }
    }
}

void oracle_syndrome(int32_t m, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                     const uint8_t *bits, int32_t F, uint8_t *syn) {
    for (int32_t f = 0; f < F; ++f)
        for (int32_t c = 0; c < m; ++c) {
            uint8_t s = 0;
            for (int32_t e = row_ptr[c]; e < row_ptr[c + 1]; ++e) s ^= bits[(size_t)f * n + col_idx[e]] & 1;
            syn[(size_t)f * m + c] = s;
        }
}

/* ----------------------------------------------------- sum-product (BP) -- */

typedef struct {
    int32_t m, n, E;
    const int32_t *row_ptr, *col_idx;
    int32_t *col_ptr, *col_edge; /* edges of each bit, ascending edge index */
    const double *R;
    int32_t F, T, early_stop;
    double clip;
    const double *w; /* T x E or NULL */
    double *post;
    uint8_t *hard;
    int32_t *iters;
    uint8_t *ok;
    int32_t next_frame;
    pthread_mutex_t lock;
} dec_job;

static double clipd(double x, double c) { return x > c ? c : (x < -c ? -c : x); }

static int syndrome_zero(const dec_job *J, const uint8_t *z) {
    for (int32_t c = 0; c < J->m; ++c) {
        uint8_t s = 0;
        for (int32_t e = J->row_ptr[c]; e < J->row_ptr[c + 1]; ++e) s ^= z[J->col_idx[e]];
        if (s) return 0;
    }
    return 1;
}

static void decode_frame(const dec_job *J, int32_t f, double *Lvc, double *Ecv, double *Lv) {
    const int32_t m = J->m, n = J->n;
    const double *R = J->R + (size_t)f * n;
    uint8_t *z = J->hard + (size_t)f * n;
    /* Eq. 4 / Algorithm 1 initialisation: L_v = R_v, and every bit sends R_v
     * to each of its checks */
    for (int32_t v = 0; v < n; ++v) {
        Lv[v] = R[v];
        z[v] = (uint8_t)(Lv[v] >= 0.0);
        for (int32_t q = J->col_ptr[v]; q < J->col_ptr[v + 1]; ++q) Lvc[J->col_edge[q]] = R[v];
    }
    int32_t t_done = 0, stopped = 0;
    for (int32_t t = 1; t <= J->T; ++t) {
        const double *wt = J->w ? J->w + (size_t)(t - 1) * J->E : NULL;
        /* check-node update, Eq. 5 (sign-corrected reading) */
        for (int32_t c = 0; c < m; ++c) {
            for (int32_t e = J->row_ptr[c]; e < J->row_ptr[c + 1]; ++e) {
                double prod = 1.0;
                for (int32_t e2 = J->row_ptr[c]; e2 < J->row_ptr[c + 1]; ++e2) {
                    if (e2 == e) continue;
                    double M = clipd(Lvc[e2], J->clip);
                    prod *= tanh(-M / 2.0);
                }
                Ecv[e] = clipd(-2.0 * atanh(prod), J->clip);
            }
        }
        /* variable-node update, Eq. 6, and total LLR, Eq. 7 */
        for (int32_t v = 0; v < n; ++v) {
            double tot = R[v];
            for (int32_t q = J->col_ptr[v]; q < J->col_ptr[v + 1]; ++q) {
                int32_t e = J->col_edge[q];
                tot += (wt ? wt[e] : 1.0) * Ecv[e];
            }
            Lv[v] = tot;
            for (int32_t q = J->col_ptr[v]; q < J->col_ptr[v + 1]; ++q) {
                double ext = R[v];
                for (int32_t q2 = J->col_ptr[v]; q2 < J->col_ptr[v + 1]; ++q2) {
                    if (q2 == q) continue;
                    int32_t e2 = J->col_edge[q2];
                    ext += (wt ? wt[e2] : 1.0) * Ecv[e2];
                }
                Lvc[J->col_edge[q]] = ext;
            }
            /* hard decision, Eq. 8 */
            z[v] = (uint8_t)(Lv[v] >= 0.0);
        }
        t_done = t;
        if (J->early_stop && syndrome_zero(J, z)) { stopped = 1; break; }
    }
    memcpy(J->post + (size_t)f * n, Lv, sizeof(double) * (size_t)n);
    J->iters[f] = t_done;
    J->ok[f] = (uint8_t)(stopped ? 1 : syndrome_zero(J, z));
}

static void *decode_worker(void *arg) {
    dec_job *J = (dec_job *)arg;
    double *Lvc = (double *)malloc(sizeof(double) * (size_t)(J->E > 0 ? J->E : 1));
    double *Ecv = (double *)malloc(sizeof(double) * (size_t)(J->E > 0 ? J->E : 1));
    double *Lv = (double *)malloc(sizeof(double) * (size_t)J->n);
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int32_t f = J->next_frame++;
        pthread_mutex_unlock(&J->lock);
        if (f >= J->F) break;
        decode_frame(J, f, Lvc, Ecv, Lv);
    }
    free(Lvc); free(Ecv); free(Lv);
    return NULL;
}

/* Decodes F frames of n FP64 channel LLRs (frame-major).  Outputs the total
 * LLR of the last iteration performed (post, F x n), hard decisions (F x n
 * bytes), iterations performed and the final syndrome flag.  Returns 0, or -1
 * on bad input. */
int oracle_decode(int32_t m, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                  const double *R, int32_t F, int32_t T, int32_t early_stop, double clip,
                  const double *w, double *post, uint8_t *hard, int32_t *iters, uint8_t *ok,
                  int32_t nthreads) {
    if (m < 0 || n <= 0 || F < 0 || T < 0 || !(clip > 0.0)) return -1;
    int32_t E = row_ptr[m];
    int32_t *col_ptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *col_edge = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
    int32_t *fill = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    for (int32_t e = 0; e < E; ++e) {
        if (col_idx[e] < 0 || col_idx[e] >= n) { free(col_ptr); free(col_edge); free(fill); return -1; }
        col_ptr[col_idx[e] + 1]++;
    }
    for (int32_t v = 0; v < n; ++v) col_ptr[v + 1] += col_ptr[v];
    for (int32_t e = 0; e < E; ++e) {
        int32_t v = col_idx[e];
        col_edge[col_ptr[v] + fill[v]++] = e;
    }
    dec_job J = {m, n, E, row_ptr, col_idx, col_ptr, col_edge, R, F, T, early_stop, clip, w,
                 post, hard, iters, ok, 0, PTHREAD_MUTEX_INITIALIZER};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads == 1) {
        decode_worker(&J);
    } else {
        pthread_t th[256];
        for (int32_t i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, decode_worker, &J);
        for (int32_t i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    }
    free(col_ptr); free(col_edge); free(fill);
    return 0;
}

/*
 * Assembly of the synthetic "proton x neutron" Kronecker test matrices
 *
 *     H = Hp (x) I_nN  +  I_nP (x) Hn  +  sum_k Cp_k (x) Cn_k
 *
 * into CSR (int64 row pointers, int32 column indices, values rounded to FP32,
 * or kept as the FP64 sums of the factor products: the "exact" Kronecker sum
 * that an operator applying the factors directly, without storing H, applies).
 * The factor matrices are small sparse symmetric CSR matrices drawn by
 * synth/kron.py; this file only expands the Kronecker sum row by row.
 *
 * Index convention: row r = p * nN + q for p < nP, q < nN, i.e.
 * (A (x) B)[p*nN + q, p'*nN + q'] = A[p,p'] * B[q,q'].
 *
 * This is input generation only: it holds none of the eigensolver's
 * arithmetic and is shared by the oracle and the GPU path.
 *
 * Determinism: every row is built independently in a fixed term order
 * (Hp term, Hn term, then k = 0..K-1), duplicate columns are summed in that
 * order in FP64 and the sum is rounded once to FP32.  The result does not
 * depend on the thread count.  Compile with -ffp-contract=off so that the
 * compiler does not fuse the coupling products into FMAs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    const int64_t* ptr;   /* n + 1 */
    const int32_t* idx;
    const double* val;
} fcsr;

typedef struct {
    int64_t col;
    int32_t seq;
    double v;
} entry;

static int cmp_entry(const void* a, const void* b) {
    const entry* x = (const entry*)a;
    const entry* y = (const entry*)b;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    return x->seq < y->seq ? -1 : (x->seq > y->seq);
}

/* Builds the (unmerged) list of contributions of row r in term order.
 * Returns the number of contributions written to buf. */
static int64_t row_terms(int64_t p, int64_t q, int64_t nN, fcsr Hp, fcsr Hn, int K,
                         const fcsr* Cp, const fcsr* Cn, entry* buf) {
    int64_t t = 0;
    for (int64_t e = Hp.ptr[p]; e < Hp.ptr[p + 1]; ++e) {
        buf[t].col = (int64_t)Hp.idx[e] * nN + q;
        buf[t].v = Hp.val[e];
        buf[t].seq = (int32_t)t;
        ++t;
    }
    for (int64_t e = Hn.ptr[q]; e < Hn.ptr[q + 1]; ++e) {
        buf[t].col = p * nN + Hn.idx[e];
        buf[t].v = Hn.val[e];
        buf[t].seq = (int32_t)t;
        ++t;
    }
    for (int k = 0; k < K; ++k) {
        for (int64_t e = Cp[k].ptr[p]; e < Cp[k].ptr[p + 1]; ++e) {
            const int64_t pc = Cp[k].idx[e];
            const double a = Cp[k].val[e];
            for (int64_t f = Cn[k].ptr[q]; f < Cn[k].ptr[q + 1]; ++f) {
                buf[t].col = pc * nN + Cn[k].idx[f];
                buf[t].v = a * Cn[k].val[f];
                buf[t].seq = (int32_t)t;
                ++t;
            }
        }
    }
    return t;
}

/* Sorts and merges the contributions; returns the merged count.  Merged
 * values are the FP64 sums in term order, rounded to FP32 when round32. */
static int64_t merge_terms(entry* buf, int64_t t, int round32) {
    qsort(buf, (size_t)t, sizeof(entry), cmp_entry);
    int64_t out = 0;
    for (int64_t i = 0; i < t;) {
        int64_t j = i;
        double s = 0.0;
        while (j < t && buf[j].col == buf[i].col) { s += buf[j].v; ++j; }
        buf[out].col = buf[i].col;
        buf[out].v = round32 ? (double)(float)s : s;
        ++out;
        i = j;
    }
    return out;
}

static int64_t max_row_len(const int64_t* ptr, int64_t n) {
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) if (ptr[i + 1] - ptr[i] > m) m = ptr[i + 1] - ptr[i];
    return m;
}

static void unpack(const int64_t* ptrs, const int32_t* idxs, const double* vals,
                   const int64_t* offs_ptr, const int64_t* offs_nz, int i, fcsr* out) {
    out->ptr = ptrs + offs_ptr[i];
    out->idx = idxs + offs_nz[i];
    out->val = vals + offs_nz[i];
}

/*
 * Factor storage: all 2 + 2K factor matrices are packed into three arrays
 * (ptrs, idxs, vals) in the order Hp, Hn, Cp_0, Cn_0, Cp_1, Cn_1, ...;
 * offs_ptr[i] / offs_nz[i] give the start of factor i in ptrs / (idxs, vals).
 *
 * Pass 1 (row_ptr != NULL, col == NULL): writes the CSR row pointer (n+1).
 * Pass 2 (col != NULL): fills col / val (val64 or val32, whichever is non-NULL)
 *                       using the row pointer from pass 1.
 * round32: 1 rounds every merged entry to FP32 once (both solvers then see
 * the same FP32-exact matrix); 0 keeps the FP64 sums (requires val64).
 * Returns the number of nonzeros, or -1 on allocation failure.
 */
int64_t kron_assemble(int64_t nP, int64_t nN, int K,
                      const int64_t* ptrs, const int32_t* idxs, const double* vals,
                      const int64_t* offs_ptr, const int64_t* offs_nz,
                      int64_t* row_ptr, int32_t* col, double* val64, float* val32, int round32) {
    fcsr Hp, Hn;
    fcsr* Cp = (fcsr*)malloc(sizeof(fcsr) * (K > 0 ? K : 1));
    fcsr* Cn = (fcsr*)malloc(sizeof(fcsr) * (K > 0 ? K : 1));
    if (!Cp || !Cn) { free(Cp); free(Cn); return -1; }
    unpack(ptrs, idxs, vals, offs_ptr, offs_nz, 0, &Hp);
    unpack(ptrs, idxs, vals, offs_ptr, offs_nz, 1, &Hn);
    int64_t cap = max_row_len(Hp.ptr, nP) + max_row_len(Hn.ptr, nN);
    for (int k = 0; k < K; ++k) {
        unpack(ptrs, idxs, vals, offs_ptr, offs_nz, 2 + 2 * k, &Cp[k]);
        unpack(ptrs, idxs, vals, offs_ptr, offs_nz, 3 + 2 * k, &Cn[k]);
        cap += max_row_len(Cp[k].ptr, nP) * max_row_len(Cn[k].ptr, nN);
    }
    const int64_t n = nP * nN;
    int failed = 0;
    if (col == NULL) {
        row_ptr[0] = 0;
#pragma omp parallel
        {
            entry* buf = (entry*)malloc(sizeof(entry) * (size_t)(cap > 0 ? cap : 1));
            if (!buf) {
#pragma omp atomic write
                failed = 1;
            } else {
#pragma omp for schedule(dynamic, 16)
                for (int64_t p = 0; p < nP; ++p) {
                    for (int64_t q = 0; q < nN; ++q) {
                        int64_t t = row_terms(p, q, nN, Hp, Hn, K, Cp, Cn, buf);
                        row_ptr[p * nN + q + 1] = merge_terms(buf, t, round32);
                    }
                }
            }
            free(buf);
        }
        if (!failed)
            for (int64_t r = 0; r < n; ++r) row_ptr[r + 1] += row_ptr[r];
    } else {
#pragma omp parallel
        {
            entry* buf = (entry*)malloc(sizeof(entry) * (size_t)(cap > 0 ? cap : 1));
            if (!buf) {
#pragma omp atomic write
                failed = 1;
            } else {
#pragma omp for schedule(dynamic, 16)
                for (int64_t p = 0; p < nP; ++p) {
                    for (int64_t q = 0; q < nN; ++q) {
                        const int64_t r = p * nN + q;
                        int64_t t = merge_terms(buf, row_terms(p, q, nN, Hp, Hn, K, Cp, Cn, buf), round32);
                        int64_t base = row_ptr[r];
                        for (int64_t e = 0; e < t; ++e) {
                            col[base + e] = (int32_t)buf[e].col;
                            if (val64) val64[base + e] = buf[e].v;
                            if (val32) val32[base + e] = (float)buf[e].v;
                        }
                    }
                }
            }
            free(buf);
        }
    }
    free(Cp);
    free(Cn);
    return failed ? -1 : row_ptr[n];
}

/*
 * Plain, slow, FP64 CPU oracle for the SPAI preconditioner, its cheap update and the
 * sparse products used by the block Krylov solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header or table with the
 * CUDA path; both only consume the same seeded inputs.
 *
 * Every function states the passage of the paper (arXiv 1809.06574, "Preconditioned
 * Linear Solves for Parametric Model Order Reduction") that it writes out:
 *   - Sec. 1.1, Eqs. (4)-(9): the affine form A = A0 + sum_j s~_j A_j and A(l).
 *   - Sec. 2.2: SPAI, min_P ||I - A P||_F^2 = sum_i min ||e_i - A p_i||_2^2, one
 *     least-squares problem per column.
 *   - Sec. 2.3 / Table 1 (first approach) and Sec. 2.4: the update
 *     min_Q ||A(1) - A(l) Q||_F^2 = sum_i min ||a1_i - A(l) q_i||_2^2, P_l = Q_l P_1.
 *   - Sec. 2.2 (footnote): right preconditioning A P X~ = B, X = P X~.
 *
 * Conventions: int32 indices, CSR with strictly increasing columns per row, dense
 * blocks column-major with a leading dimension.  Compiled with -ffp-contract=off so
 * that every product and sum is rounded separately, in the order written here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* sort + unique in place; returns the new length */
static int64_t sort_unique(int32_t *buf, int64_t len)
{
    if (len <= 0) return 0;
    qsort(buf, (size_t)len, sizeof(int32_t), cmp_i32);
    int64_t w = 1;
    for (int64_t r = 1; r < len; ++r)
        if (buf[r] != buf[w - 1]) buf[w++] = buf[r];
    return w;
}

/* ------------------------------------------------------------------------------------
 * Assembly of A = sum_t c_t A_t on the union of the terms' patterns (Sec. 1.1, Eq. (4)
 * and Eqs. (7)-(9): every A(l) is the same affine combination with other coefficients).
 * The pattern is structural: an entry exists if any term has it, whatever its value.
 *
 * Terms are passed concatenated: term t has row pointer rowptr_all + t*(n+1) and its
 * column / value arrays start at offset coff[t] of colind_all / val_all.
 * ------------------------------------------------------------------------------------ */
int64_t oracle_union_pattern(int32_t n, int32_t T, const int32_t *rowptr_all,
                             const int32_t *colind_all, const int64_t *coff,
                             int32_t *out_rowptr, int32_t *out_colind)
{
    int64_t maxrow = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t len = 0;
        for (int32_t t = 0; t < T; ++t) {
            const int32_t *rp = rowptr_all + (int64_t)t * (n + 1);
            len += rp[i + 1] - rp[i];
        }
        if (len > maxrow) maxrow = len;
    }
    int32_t *buf = (int32_t *)malloc((size_t)(maxrow > 0 ? maxrow : 1) * sizeof(int32_t));
    int64_t nnz = 0;
    if (out_rowptr) out_rowptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t len = 0;
        for (int32_t t = 0; t < T; ++t) {
            const int32_t *rp = rowptr_all + (int64_t)t * (n + 1);
            const int32_t *ci = colind_all + coff[t];
            for (int32_t q = rp[i]; q < rp[i + 1]; ++q) buf[len++] = ci[q];
        }
        len = sort_unique(buf, len);
        if (out_colind) memcpy(out_colind + nnz, buf, (size_t)len * sizeof(int32_t));
        nnz += len;
        if (out_rowptr) out_rowptr[i + 1] = (int32_t)nnz;
    }
    free(buf);
    return nnz;
}

/* Values of sum_t c_t A_t on the union pattern, terms added in the order t = 0..T-1,
 * each as (acc + c_t * a_t(i,j)) with the product and the sum rounded separately. */
void oracle_assemble_values(int32_t n, int32_t T, const int32_t *rowptr_all,
                            const int32_t *colind_all, const double *val_all,
                            const int64_t *coff, const double *coef,
                            const int32_t *u_rowptr, const int32_t *u_colind, double *out_val)
{
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t q = u_rowptr[i]; q < u_rowptr[i + 1]; ++q) {
            int32_t j = u_colind[q];
            double acc = 0.0;
            for (int32_t t = 0; t < T; ++t) {
                const int32_t *rp = rowptr_all + (int64_t)t * (n + 1);
                const int32_t *ci = colind_all + coff[t];
                const double *va = val_all + coff[t];
                for (int32_t r = rp[i]; r < rp[i + 1]; ++r) {
                    if (ci[r] == j) {
                        double prod = coef[t] * va[r];
                        acc = acc + prod;
                        break;
                    }
                }
            }
            out_val[q] = acc;
        }
    }
}

/* ------------------------------------------------------------------------------------
 * Column access to A (Sec. 2.2 works on columns of A): CSR -> CSC by counting.
 * Rows inside each column come out ascending because rows are visited in order.
 * ------------------------------------------------------------------------------------ */
void oracle_csr_to_csc(int32_t n, const int32_t *rowptr, const int32_t *colind,
                       const double *val, int32_t *colptr, int32_t *rowind, double *cval)
{
    int32_t *next = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t j = 0; j <= n; ++j) colptr[j] = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t q = rowptr[i]; q < rowptr[i + 1]; ++q) colptr[colind[q] + 1]++;
    for (int32_t j = 0; j < n; ++j) colptr[j + 1] += colptr[j];
    for (int32_t j = 0; j < n; ++j) next[j] = colptr[j];
    for (int32_t i = 0; i < n; ++i)
        for (int32_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            int32_t j = colind[q];
            int32_t d = next[j]++;
            rowind[d] = i;
            if (cval) cval[d] = val[q];
        }
    free(next);
}

/* ------------------------------------------------------------------------------------
 * Sparsity pattern of the columns of P.  The paper's MSPAI run grows it adaptively;
 * here it is fixed: the pattern of A (J_k = rows of column k of A, i.e. the CSC
 * column itself, no routine needed) or the structural pattern of A^2:
 *   J_k = union over j in rows(A(:,k)) of rows(A(:,j)), ascending.
 * ------------------------------------------------------------------------------------ */
int64_t oracle_pattern_a2(int32_t n, const int32_t *colptr, const int32_t *rowind,
                          int32_t *Jptr, int32_t *Jind)
{
    int64_t maxlen = 0;
    for (int32_t k = 0; k < n; ++k) {
        int64_t len = 0;
        for (int32_t q = colptr[k]; q < colptr[k + 1]; ++q) {
            int32_t j = rowind[q];
            len += colptr[j + 1] - colptr[j];
        }
        if (len > maxlen) maxlen = len;
    }
    int32_t *buf = (int32_t *)malloc((size_t)(maxlen > 0 ? maxlen : 1) * sizeof(int32_t));
    int64_t tot = 0;
    if (Jptr) Jptr[0] = 0;
    for (int32_t k = 0; k < n; ++k) {
        int64_t len = 0;
        for (int32_t q = colptr[k]; q < colptr[k + 1]; ++q) {
            int32_t j = rowind[q];
            for (int32_t r = colptr[j]; r < colptr[j + 1]; ++r) buf[len++] = rowind[r];
        }
        len = sort_unique(buf, len);
        if (Jind) memcpy(Jind + tot, buf, (size_t)len * sizeof(int32_t));
        tot += len;
        if (Jptr) Jptr[k + 1] = (int32_t)tot;
    }
    free(buf);
    return tot;
}

/* Row index sets of the column least-squares problems (Sec. 2.2): for column k only
 * the columns A(:, J_k) enter, so only the rows
 *   I_k = union over j in J_k of rows(A(:,j))   (ascending)
 * can hold nonzeros of A m_k; every other row of e_k - A m_k is constant in m_k. */
int64_t oracle_index_sets(int32_t n, const int32_t *colptr, const int32_t *rowind,
                          const int32_t *Jptr, const int32_t *Jind,
                          int32_t *Iptr, int32_t *Ilist)
{
    int64_t maxlen = 0;
    for (int32_t k = 0; k < n; ++k) {
        int64_t len = 0;
        for (int32_t q = Jptr[k]; q < Jptr[k + 1]; ++q) {
            int32_t j = Jind[q];
            len += colptr[j + 1] - colptr[j];
        }
        if (len > maxlen) maxlen = len;
    }
    int32_t *buf = (int32_t *)malloc((size_t)(maxlen > 0 ? maxlen : 1) * sizeof(int32_t));
    int64_t tot = 0;
    if (Iptr) Iptr[0] = 0;
    for (int32_t k = 0; k < n; ++k) {
        int64_t len = 0;
        for (int32_t q = Jptr[k]; q < Jptr[k + 1]; ++q) {
            int32_t j = Jind[q];
            for (int32_t r = colptr[j]; r < colptr[j + 1]; ++r) buf[len++] = rowind[r];
        }
        len = sort_unique(buf, len);
        if (Ilist) memcpy(Ilist + tot, buf, (size_t)len * sizeof(int32_t));
        tot += len;
        if (Iptr) Iptr[k + 1] = (int32_t)tot;
    }
    free(buf);
    return tot;
}

/* position of key in the ascending list a[0..len), or -1 */
static int32_t find_pos(const int32_t *a, int32_t len, int32_t key)
{
    int32_t lo = 0, hi = len - 1;
    while (lo <= hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (a[mid] == key) return mid;
        if (a[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------------------------------------
 * Column least-squares problems of SPAI (Sec. 2.2) and of the update (Sec. 2.3, Table 1
 * first approach; Sec. 2.4):
 *   mode 0 (build):  m_k = argmin_{supp m subset J_k} || e_k - A m ||_2
 *   mode 1 (update): q_k = argmin_{supp q subset J_k} || a1_k - A(l) q ||_2,
 *                    a1_k = column k of A(1), given in CSC (r_colptr, r_rowind, r_val).
 * Restricting the rows to I_k is exact (rows outside I_k do not depend on m).
 *
 * Solved by Householder QR of Ahat = A(I_k, J_k): for each column c the reflector
 * v = x + sign(x_1)||x|| e_1 (sign(0) = +1) is applied to the remaining columns and to
 * the right-hand side, then R m = (Q^T rhs)(0:|J|) is solved by back substitution.
 * A column is singular (status 1, values 0) if |I_k| < |J_k| or some
 * |R_cc| <= 1e-14 * max_t |R_tt|.
 *
 * Columns k0 <= k < k1 are processed; results go to out_val[Jptr[k] + c] (column k of
 * the result stored column-wise on pattern J).  Returns the number of singular columns.
 * ------------------------------------------------------------------------------------ */
int64_t oracle_spai_columns(int32_t n, const int32_t *colptr, const int32_t *rowind,
                            const double *cval, const int32_t *Jptr, const int32_t *Jind,
                            const int32_t *Iptr, const int32_t *Ilist, int32_t mode,
                            const int32_t *r_colptr, const int32_t *r_rowind,
                            const double *r_val, int32_t k0, int32_t k1, double *out_val,
                            int32_t *status)
{
    (void)n;
    int32_t maxI = 0, maxJ = 0;
    for (int32_t k = k0; k < k1; ++k) {
        int32_t ni = Iptr[k + 1] - Iptr[k], nj = Jptr[k + 1] - Jptr[k];
        if (ni > maxI) maxI = ni;
        if (nj > maxJ) maxJ = nj;
    }
    double *Ah = (double *)malloc((size_t)(maxI > 0 ? maxI : 1) * (size_t)(maxJ > 0 ? maxJ : 1) * sizeof(double));
    double *rhs = (double *)malloc((size_t)(maxI > 0 ? maxI : 1) * sizeof(double));
    double *v = (double *)malloc((size_t)(maxI > 0 ? maxI : 1) * sizeof(double));
    double *m = (double *)malloc((size_t)(maxJ > 0 ? maxJ : 1) * sizeof(double));
    int64_t nsing = 0;
    for (int32_t k = k0; k < k1; ++k) {
        const int32_t *I = Ilist + Iptr[k];
        const int32_t *J = Jind + Jptr[k];
        int32_t ni = Iptr[k + 1] - Iptr[k], nj = Jptr[k + 1] - Jptr[k];
        int singular = (ni < nj);
        /* gather Ahat = A(I, J), column-major with leading dimension ni */
        for (int64_t e = 0; e < (int64_t)ni * nj; ++e) Ah[e] = 0.0;
        for (int32_t c = 0; c < nj; ++c) {
            int32_t j = J[c];
            for (int32_t q = colptr[j]; q < colptr[j + 1]; ++q) {
                int32_t r = find_pos(I, ni, rowind[q]);
                if (r >= 0) Ah[(int64_t)c * ni + r] = cval[q];
            }
        }
        /* right-hand side restricted to I */
        for (int32_t r = 0; r < ni; ++r) rhs[r] = 0.0;
        if (mode == 0) {
            int32_t r = find_pos(I, ni, k);
            if (r >= 0) rhs[r] = 1.0;
        } else {
            for (int32_t q = r_colptr[k]; q < r_colptr[k + 1]; ++q) {
                int32_t r = find_pos(I, ni, r_rowind[q]);
                if (r >= 0) rhs[r] = r_val[q];
            }
        }
        /* Householder QR, applied to the right-hand side as it goes */
        int32_t steps = nj < ni ? nj : ni;
        for (int32_t c = 0; c < steps && !singular; ++c) {
            double *x = Ah + (int64_t)c * ni;
            double ss = 0.0;
            for (int32_t r = c; r < ni; ++r) ss = ss + x[r] * x[r];
            double alpha = sqrt(ss);
            if (alpha == 0.0) { singular = 1; break; }
            double sgn = (x[c] >= 0.0) ? 1.0 : -1.0;
            for (int32_t r = c; r < ni; ++r) v[r] = x[r];
            v[c] = v[c] + sgn * alpha;
            double vtv = 0.0;
            for (int32_t r = c; r < ni; ++r) vtv = vtv + v[r] * v[r];
            x[c] = -sgn * alpha;
            for (int32_t r = c + 1; r < ni; ++r) x[r] = 0.0;
            for (int32_t t = c + 1; t < nj; ++t) {
                double *y = Ah + (int64_t)t * ni;
                double d = 0.0;
                for (int32_t r = c; r < ni; ++r) d = d + v[r] * y[r];
                double g = 2.0 * d / vtv;
                for (int32_t r = c; r < ni; ++r) y[r] = y[r] - g * v[r];
            }
            double d = 0.0;
            for (int32_t r = c; r < ni; ++r) d = d + v[r] * rhs[r];
            double g = 2.0 * d / vtv;
            for (int32_t r = c; r < ni; ++r) rhs[r] = rhs[r] - g * v[r];
        }
        if (!singular) {
            double rmax = 0.0;
            for (int32_t c = 0; c < nj; ++c) {
                double a = fabs(Ah[(int64_t)c * ni + c]);
                if (a > rmax) rmax = a;
            }
            for (int32_t c = 0; c < nj; ++c)
                if (fabs(Ah[(int64_t)c * ni + c]) <= 1e-14 * rmax) singular = 1;
        }
        if (singular) {
            for (int32_t c = 0; c < nj; ++c) out_val[Jptr[k] + c] = 0.0;
            if (status) status[k - k0] = 1;
            ++nsing;
            continue;
        }
        /* back substitution R m = rhs(0:nj) */
        for (int32_t c = nj - 1; c >= 0; --c) {
            double acc = rhs[c];
            for (int32_t t = c + 1; t < nj; ++t) acc = acc - Ah[(int64_t)t * ni + c] * m[t];
            m[c] = acc / Ah[(int64_t)c * ni + c];
        }
        for (int32_t c = 0; c < nj; ++c) out_val[Jptr[k] + c] = m[c];
        if (status) status[k - k0] = 0;
    }
    free(Ah);
    free(rhs);
    free(v);
    free(m);
    return nsing;
}

/* ------------------------------------------------------------------------------------
 * Sparse times dense block, Y = A X (the products A P V and P V of the right-
 * preconditioned block Krylov method, Sec. 2.1-2.2).  X, Y column-major.
 * ------------------------------------------------------------------------------------ */
void oracle_spmm_csr(int32_t n, const int32_t *rowptr, const int32_t *colind,
                     const double *val, int32_t s, const double *X, int64_t ldx,
                     double *Y, int64_t ldy)
{
    for (int32_t c = 0; c < s; ++c)
        for (int32_t i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int32_t q = rowptr[i]; q < rowptr[i + 1]; ++q)
                acc = acc + val[q] * X[(int64_t)c * ldx + colind[q]];
            Y[(int64_t)c * ldy + i] = acc;
        }
}

/* Same with A given column-wise (CSC): Y = sum_k A(:,k) X(k,:). */
void oracle_spmm_csc(int32_t n, const int32_t *colptr, const int32_t *rowind,
                     const double *val, int32_t s, const double *X, int64_t ldx,
                     double *Y, int64_t ldy)
{
    for (int32_t c = 0; c < s; ++c) {
        double *y = Y + (int64_t)c * ldy;
        const double *x = X + (int64_t)c * ldx;
        for (int32_t i = 0; i < n; ++i) y[i] = 0.0;
        for (int32_t k = 0; k < n; ++k)
            for (int32_t q = colptr[k]; q < colptr[k + 1]; ++q)
                y[rowind[q]] = y[rowind[q]] + val[q] * x[k];
    }
}

/* ------------------------------------------------------------------------------------
 * Dense LU with partial pivoting (test solves on tiny systems; Sec. 2.1 contrasts the
 * direct approach with the iterative one).  A (n x n, column-major, lda) is overwritten
 * by its factors, B (n x nrhs, ldb) by the solution.  Returns 0, or 1 if a pivot is 0.
 * ------------------------------------------------------------------------------------ */
int32_t oracle_dense_lu_solve(int32_t n, double *A, int64_t lda, int32_t nrhs, double *B,
                              int64_t ldb)
{
#define AE(i, j) A[(int64_t)(j) * lda + (i)]
#define BE(i, j) B[(int64_t)(j) * ldb + (i)]
    for (int32_t k = 0; k < n; ++k) {
        int32_t p = k;
        double best = fabs(AE(k, k));
        for (int32_t i = k + 1; i < n; ++i)
            if (fabs(AE(i, k)) > best) { best = fabs(AE(i, k)); p = i; }
        if (best == 0.0) return 1;
        if (p != k) {
            for (int32_t j = 0; j < n; ++j) { double t = AE(k, j); AE(k, j) = AE(p, j); AE(p, j) = t; }
            for (int32_t j = 0; j < nrhs; ++j) { double t = BE(k, j); BE(k, j) = BE(p, j); BE(p, j) = t; }
        }
        for (int32_t i = k + 1; i < n; ++i) {
            double l = AE(i, k) / AE(k, k);
            AE(i, k) = l;
            for (int32_t j = k + 1; j < n; ++j) AE(i, j) = AE(i, j) - l * AE(k, j);
            for (int32_t j = 0; j < nrhs; ++j) BE(i, j) = BE(i, j) - l * BE(k, j);
        }
    }
    for (int32_t j = 0; j < nrhs; ++j)
        for (int32_t i = n - 1; i >= 0; --i) {
            double acc = BE(i, j);
            for (int32_t t = i + 1; t < n; ++t) acc = acc - AE(i, t) * BE(t, j);
            BE(i, j) = acc / AE(i, i);
        }
    return 0;
#undef AE
#undef BE
}

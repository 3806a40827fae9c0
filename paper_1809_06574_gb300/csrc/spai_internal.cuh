// Internal declarations shared by the CUDA translation units of libspai_gb300.
// Kernels live in k_sparse.cu (assembly, transposition, index sets, SpMM), k_spai.cu
// (per-column gather + Householder least squares) and k_krylov.cu (block GMRES pieces);
// spai_api.cu implements the C ABI declared in include/spai_gb300.h on top of them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "spai_gb300.h"

namespace spai {

constexpr int kMaxTerms = 16;

// Device-side error word bits (written with atomicOr, read by the host after a sync).
enum : int {
    ERR_ROWPTR = 1 << 0,      // rowptr not monotone / wrong ends
    ERR_COLIND = 1 << 1,      // column index out of range or not strictly increasing
    ERR_OVERFLOW = 1 << 2,    // a prefix sum exceeds int32
    ERR_TOO_WIDE = 1 << 3,    // a column problem exceeds the kernel's tile
    ERR_PATTERN = 1 << 4,     // values do not fit the expected pattern
    ERR_TIMEOUT = 1 << 5,     // a bounded device-side wait gave up
    ERR_RANGE = 1 << 6,       // a value outside the fixed-point range of the digit Gram product
};

struct TermPtrs {
    const int32_t *rowptr[kMaxTerms];
    const int32_t *colind[kMaxTerms];
    const double *val[kMaxTerms];
    double coef[kMaxTerms];
};

// process-wide count of kernels launched by the library
void note_launches(int k);
long long launches_total();

// ---------------------------------------------------------------------- k_sparse.cu
int launch_validate_csr(cudaStream_t st, int32_t n, int32_t nnz, const int32_t *rowptr,
                        const int32_t *colind, int *d_err);
int launch_union_count(cudaStream_t st, int32_t n, int32_t T, const TermPtrs &tp, int32_t *counts);
int launch_union_fill(cudaStream_t st, int32_t n, int32_t T, const TermPtrs &tp,
                      const int32_t *u_rowptr, int32_t *u_colind, double *aligned,
                      int64_t nnzU);
int launch_assemble(cudaStream_t st, int64_t nnz, int32_t T, const double *aligned,
                    const double *coef_host, double *out);
// ptr[0] = 0, ptr[i+1] = ptr[i] + counts[i]; temp must hold scan_temp_bytes(n)
size_t scan_temp_bytes(int64_t n);
int launch_exclusive_scan(cudaStream_t st, const int32_t *counts, int32_t *ptr, int64_t n,
                          void *temp, int *d_err);
// CSR (n x n) -> CSC pattern: colptr[n+1], rowind[nnz] ascending per column, perm[csc] = csr
size_t transpose_temp_bytes(int32_t n, int32_t nnz);
int launch_transpose(cudaStream_t st, int32_t n, int32_t nnz, const int32_t *rowptr,
                     const int32_t *colind, int32_t *colptr, int32_t *rowind, int32_t *perm,
                     void *temp, int *d_err);
// out_k = sorted union over j in L_k of rows(colptr/rowind column j); two passes
// (at most colunion_max_lists() columns in any L_k, else ERR_TOO_WIDE)
int colunion_max_lists();
// maxL: an upper bound of every |L_k| (picks the team width; a longer list sets ERR_TOO_WIDE
// when it exceeds the widest team's capacity, colunion_max_lists())
int launch_colunion_count(cudaStream_t st, int32_t n, int32_t maxL, const int32_t *Lptr, const int32_t *Lind,
                          const int32_t *colptr, const int32_t *rowind, int32_t *counts, int *d_err);
int launch_colunion_fill(cudaStream_t st, int32_t n, int32_t maxL, const int32_t *Lptr, const int32_t *Lind,
                         const int32_t *colptr, const int32_t *rowind, const int32_t *out_ptr,
                         int32_t *out_list, int *d_err);
int launch_gather_f64(cudaStream_t st, int64_t count, const int32_t *idx, const double *src,
                      double *dst);
int launch_gather_f32_f64(cudaStream_t st, int64_t count, const int32_t *idx, const float *src, double *dst);
int launch_invert_perm(cudaStream_t st, int64_t count, const int32_t *perm, int32_t *inv);
int launch_max_i32_diff(cudaStream_t st, int32_t n, const int32_t *ptr, int32_t *d_max);
int launch_fill_i32(cudaStream_t st, int64_t count, int32_t v, int32_t *dst);
// *d_out = smallest i with a[i] != 0, or INT_MAX
int launch_first_nonzero(cudaStream_t st, int32_t n, const int32_t *a, int32_t *d_out);
// sets ERR_PATTERN in *d_err if a[i] != b[i] for some i < count
int launch_compare_i32(cudaStream_t st, int64_t count, const int32_t *a, const int32_t *b, int *d_err);
// row-major blocks: X[r * s + c]
int launch_spmm(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr,
                const int32_t *colind, const double *val, const double *X, double *Y);
// same with BF16 values (bit patterns; products and sums in FP64)
int launch_spmm_bf16v(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind,
                      const uint16_t *val, const double *X, double *Y);
int launch_gather_bf16_f64(cudaStream_t st, int64_t count, const int32_t *idx, const uint16_t *src, double *dst);
// ---- batches of matrices stacked into one block-diagonal matrix (device tables; systems
// laid end to end: off / nzoff hold nsys + 1 row / nonzero offsets, start nseg + 1)
// rp[ntot + 1], ci[nnz] of the stacked CSR; checks each system's rows (ERR_ROWPTR) and
// column indices (ERR_COLIND)
int launch_stack_csr(cudaStream_t st, int32_t nsys, int64_t ntot, int64_t nnz, const int64_t *off, const int64_t *nzoff,
                     const int32_t *const *rowptr, const int32_t *const *colind, int32_t *rp, int32_t *ci, int *d_err);
// union lists L_k: {k} (kind 0) or the rows of column k (kind 1): counts (Lptr NULL) or fill
int launch_union_lists(cudaStream_t st, int32_t nsys, int64_t ntot, const int64_t *off, const int32_t *kind,
                       const int32_t *colptr, const int32_t *rowind, int32_t *counts, const int32_t *Lptr, int32_t *Lind);
// per system: total entries of a pointer array over its rows and its longest row
int launch_seg_ptr_stats(cudaStream_t st, int32_t nsys, int64_t ntot, const int64_t *off, const int32_t *ptr,
                         int64_t *tot, int32_t *mx);
// dst_g[j] = src_g[j] - sub_g; val gather dst_g[j] = val_g[perm_g[j]]; first nonzero per segment
int launch_unstack(cudaStream_t st, int32_t nseg, int64_t total, const int64_t *start, const int32_t *const *src,
                   int32_t *const *dst, const int32_t *sub);
int launch_gather_seg(cudaStream_t st, int32_t nseg, int64_t total, const int64_t *start, const double *const *val,
                      const int32_t *const *perm, double *const *dst);
int launch_first_nonzero_seg(cudaStream_t st, int32_t nseg, int64_t total, const int64_t *start,
                             const int32_t *const *a, int32_t *out);
// dst[i] = src[i] + add
int launch_add_i32(cudaStream_t st, int64_t count, const int32_t *src, int32_t add, int32_t *dst);
// dst[i] = i; the FP32 / BF16 gathers take idx = NULL for the identity
int launch_iota_i32(cudaStream_t st, int64_t count, int32_t *dst);
// same with FP32 values (products and sums in FP64)
int launch_spmm_f32v(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind,
                     const float *val, const double *X, double *Y);
// ---- the FP32 operator of the mixed-precision solve: values (one of the three pointers)
// and X rounded to FP32, products and sums in FP32 in each row's order; X and Y FP64 or FP32
struct F32Vals {
    const float *f32 = nullptr;
    const uint16_t *bf16 = nullptr;
    const double *f64 = nullptr;
};
int launch_spmm32(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind,
                  const F32Vals &v, const double *X, float *Y);
int launch_spmm32(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind,
                  const F32Vals &v, const float *X, float *Y);
int launch_spmm32(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind,
                  const F32Vals &v, const double *X, double *Y);
int launch_spmm32(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind,
                  const F32Vals &v, const float *X, double *Y);
// Y[r][c] = q[r] X[r][c] in FP32
int launch_scale_rows32(cudaStream_t st, int32_t s, int32_t n, const F32Vals &q, const double *X, float *Y);
int launch_scale_rows32(cudaStream_t st, int32_t s, int32_t n, const F32Vals &q, const float *X, float *Y);
int launch_scale_rows32(cudaStream_t st, int32_t s, int32_t n, const F32Vals &q, const double *X, double *Y);
int launch_scale_rows32(cudaStream_t st, int32_t s, int32_t n, const F32Vals &q, const float *X, double *Y);
// dst[i] = src[i] rounded to FP32
int launch_round_f32(cudaStream_t st, int64_t count, const double *src, float *dst);
// dst[start[g] + j] = (float)src[g][j] for the nseg segments laid end to end (total = start[nseg];
// start and src device arrays)
int launch_round_seg(cudaStream_t st, int32_t nseg, int64_t total, const int64_t *start, const double *const *src,
                     float *dst);
int launch_pack(cudaStream_t st, int32_t s, int32_t n, const double *src, int64_t ld, double *dst);
// Y[r][c] = q[r] X[r][c] (a diagonal factor; q FP64, FP32 or BF16 bits, one of them given)
// Y = A X and Y = diag(q) X on the rows of a list of nchunks row chunks [r0[c], r1[c]) of at
// most max_rows rows each (one value array given: FP64, FP32 or BF16 bits; FP64 arithmetic)
int launch_spmm_seg(cudaStream_t st, int32_t s, int32_t nchunks, int64_t max_rows, const int64_t *r0,
                    const int64_t *r1, const int32_t *rowptr, const int32_t *colind, const double *val,
                    const float *val32, const uint16_t *val16, const double *X, double *Y);
int launch_scale_rows_seg(cudaStream_t st, int32_t s, int32_t nchunks, int64_t max_rows, const int64_t *r0,
                          const int64_t *r1, const double *q, const float *q32, const uint16_t *q16, const double *X,
                          double *Y);
int launch_scale_rows(cudaStream_t st, int32_t s, int32_t n, const double *q, const float *q32, const uint16_t *q16,
                      const double *X, double *Y);
int launch_unpack(cudaStream_t st, int32_t s, int32_t n, const double *src, double *dst,
                  int64_t ld);

// ---------------------------------------------------------------------- k_spai.cu
struct ColumnProblem {
    int32_t n;
    const int32_t *colptr, *rowind;  // CSC pattern of A (matrix of the least squares)
    const double *cval;              // A values in CSC order
    const int32_t *Jptr, *Jind;      // column pattern of the result
    const int32_t *Iptr, *Ilist;     // row sets
    int32_t mode;                    // 0 build (rhs e_k), 1 update (rhs column k of R)
    const int32_t *r_colptr, *r_rowind;
    const double *r_val;             // rhs matrix (CSC values) in update mode
    const float *cval32, *r_val32;   // non-null: the same values rounded to FP32 once (FP32 solves read these)
    const int32_t *out_map;          // J position -> position in the output array
    double *out_val;
    float *out_val32;                // non-null: solve in FP32 and write here instead
    uint16_t *out_val16;             // non-null: solve in FP32 and write BF16 bits here instead
    int32_t *col_status;             // 0 ok, 1 singular
    int *d_err;
};
// Adaptive SPAI pattern search (k_adaptive.cu): one warp per column grows J_k from {k};
// the final lists go to out_J[k * adaptive_max_cols() ...], their sizes to out_count[k].
struct AdaptiveProblem {
    int32_t n;
    const int32_t *colptr, *rowind;  // CSC of A
    const double *cval;
    const int32_t *rowptr, *colind;  // CSR pattern of A
    const double *colnorm2;          // ||A(:,j)||^2
    double eps;
    int32_t max_steps, max_new, max_rows;
    int32_t *out_J, *out_count;
    int *d_err;
};
int adaptive_max_cols();
int adaptive_max_rows();
int launch_adaptive_pattern(cudaStream_t st, const AdaptiveProblem &ap);
int launch_colnorm2_csc(cudaStream_t st, int32_t n, const int32_t *colptr, const double *cval, double *out);
// out[ptr[k] + c] = lists[k * stride + c] for c < ptr[k + 1] - ptr[k]
int launch_compact_lists(cudaStream_t st, int32_t n, const int32_t *lists, int32_t stride, const int32_t *ptr,
                         int32_t *out);
// Column problems of several systems: column g (0 <= g < total) is local column
// g - start[i] of system i, start[i] <= g < start[i + 1]; tab[i] is its problem (device).
struct ColumnBatch {
    const ColumnProblem *tab;
    const int64_t *start;  // nsys + 1 entries, device
    int32_t nsys;
    int64_t total;
};
// diagonal update: out[k] = <cval(:,k), rval(:,k)> / ||cval(:,k)||^2 on the CSC pattern
// colptr (FP32 working precision when out32 or out16 is given, else FP64)
int launch_diag_update(cudaStream_t st, int32_t n, const int32_t *colptr, const double *cval, const double *rval,
                       double *out, float *out32, uint16_t *out16, int32_t *status);
// true if one column problem of maxI x maxJ fits the kernel's shared-memory tile
bool spai_columns_fit(int32_t maxI, int32_t maxJ);
// Picks the team size by the largest |I_k|, |J_k|; returns 0 or -1 if no tile fits.
int launch_spai_columns(cudaStream_t st, const ColumnProblem &cp, int32_t maxI, int32_t maxJ);
// One problem's columns with team size (or register-tiled shape code) `team`.
int launch_spai_columns_team(cudaStream_t st, const ColumnProblem &cp, bool low_precision, int32_t maxI,
                             int32_t maxJ, int team);
// Team sizes that fit a maxI x maxJ problem (the default choice first), then the codes
// (64 + i) of the register-tiled shapes and (96 + i) of the one-lane shapes that fit;
// returns how many (at most 15; teams needs room for 32).
int spai_columns_teams(int32_t maxI, int32_t maxJ, bool low_precision, int *teams);
// Codes (112 + i) of the normal-equations shapes (SPAI_LS_NORMAL) that fit; 0 when the tile
// is too large for them (such problems are solved by Householder QR).
int spai_columns_ne_teams(int32_t maxI, int32_t maxJ, bool low_precision, int *teams);
// All columns of a batch in one persistent launch with team size `team` (FP32 working
// precision if low_precision); every problem must fit maxI x maxJ.
int launch_spai_columns_batch(cudaStream_t st, const ColumnBatch &bt, bool low_precision, int32_t maxI,
                              int32_t maxJ, int team);

// ---------------------------------------------------------------------- shared device code
#ifdef __CUDACC__
// Conversions between FP32 and FP64 written from the IEEE 754 binary32 / binary64 layouts
// with integer operations: GB300 runs the conversion instructions on its FP64 pipe, whose
// throughput is a small fraction of the integer pipes', and the mixed-precision operator
// converts every entry it reads or writes.  Numbers whose result is normal take the integer
// path; zeros, subnormals, infinities and NaN (rare here) take the conversion instruction.
//
// binary32 -> binary64 (exact): the sign moves from bit 31 to bit 63, the biased exponent
// gains 1023 - 127 = 896, the 23 fraction bits gain 29 low zero bits.
__device__ __forceinline__ double f32_to_f64(float x)
{
    const uint32_t u = __float_as_uint(x), e = (u >> 23) & 0xFFu;
    if (e - 1u < 254u)  // normal
        return __hiloint2double((int)((u & 0x80000000u) | (((u >> 3) & 0x0FFFFFFFu) + (896u << 20))),
                                (int)(u << 29));
    if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);  // +-0
    return (double)x;
}

// binary64 -> binary32, rounded to nearest, ties to even: the biased exponent loses 896 and
// the fraction its 29 low bits, rounded up when they exceed half a unit of the last kept
// place or equal it with an odd last kept bit (a carry out of the fraction moves to the next
// binade, and past the largest finite value to infinity, as the rounding rule asks).
__device__ __forceinline__ float f64_to_f32(double x)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t e = (hi >> 20) & 0x7FFu;
    if (e - 897u < 254u) {  // the result's biased exponent e - 896 is in 1 .. 254: normal
        uint32_t f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
        const uint32_t rem = lo & 0x1FFFFFFFu;
        f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
        return __uint_as_float(f);
    }
    return (float)x;
}

// x := x R^{-1} for one row (R upper triangular S x S, row-major; rinv[b] = 1 / R_bb, or 0
// for a deflated column).  Every row-wise triangular solve of the block orthogonalisation
// uses this one sequence, so a row solved in different kernels gets the same bits.
template <int S>
__device__ __forceinline__ void trsm_row(double (&x)[S], const double *Rs, const double *rinv)
{
#pragma unroll
    for (int b = 0; b < S; ++b) {
        double acc = x[b];
#pragma unroll
        for (int a = 0; a < b; ++a) acc = fma(-x[a], Rs[a * S + b], acc);
        x[b] = acc * rinv[b];
    }
}

// one row of an n x S row-major block, 16-byte loads / stores when S is even (plain
// loads: the in-place kernels read a row and then overwrite it)
template <int S>
__device__ __forceinline__ void row_load(const double *W, int64_t r, double (&x)[S])
{
    if constexpr (S % 2 == 0) {
        const double2 *p = reinterpret_cast<const double2 *>(W + r * S);
#pragma unroll
        for (int k = 0; k < S / 2; ++k) {
            const double2 v = p[k];
            x[2 * k] = v.x;
            x[2 * k + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < S; ++k) x[k] = W[r * S + k];
    }
}

template <int S>
__device__ __forceinline__ void row_store(double *W, int64_t r, const double (&x)[S])
{
    if constexpr (S % 2 == 0) {
        double2 *p = reinterpret_cast<double2 *>(W + r * S);
#pragma unroll
        for (int k = 0; k < S / 2; ++k) p[k] = make_double2(x[2 * k], x[2 * k + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < S; ++k) W[r * S + k] = x[k];
    }
}
#endif

// ---------------------------------------------------------------------- k_krylov.cu
struct KrylovWs;
// Row chunks of a batch of systems stacked row-wise (device arrays): chunk c covers rows
// [r0[c], r1[c]) of system sys[c]; system b's chunks are c0[b] .. c0[b + 1] - 1.
struct SegChunks {
    const int32_t *sys;
    const int64_t *r0, *r1;
    const int32_t *c0;
    int32_t nchunks, nsys;
};
// per-system versions of the block-GMRES pieces (outputs of system b at b * stride)
int launch_colnorm2_seg(cudaStream_t st, int32_t s, const double *W, const SegChunks &sc, double *partial,
                        double *out);
// partial: nchunks * nblk * s * s doubles
int launch_block_dot_seg(cudaStream_t st, int32_t s, int64_t ntot, int32_t nblk, const double *V, const double *W,
                         const SegChunks &sc, double *partial, double *out, int64_t ostride);
// jlim (may be NULL): system b uses its first min(nblk, jlim[b]) blocks only
int launch_block_update_seg(cudaStream_t st, int32_t s, int64_t ntot, int32_t nblk, const double *V, const double *H,
                            int64_t hstride, const double *base, double *out, double sign, const SegChunks &sc,
                            const int32_t *jlim = nullptr);
int launch_gram_seg(cudaStream_t st, int32_t s, const double *W, const SegChunks &sc, double *partial, double *G);
int launch_trsm_gram_seg(cudaStream_t st, int32_t s, const double *W, const double *R, const int32_t *deflated,
                         double *Q1, const SegChunks &sc, double *partial, double *G2);
int launch_trsm_rows_seg(cudaStream_t st, int32_t s, const double *W, const double *R, const int32_t *deflated,
                         double *out, const SegChunks &sc);
int launch_chol_small_b(cudaStream_t st, int32_t s, int32_t nsys, const double *G, const double *ref2, double tau2,
                        double *R, int32_t *deflated);
int launch_triu_mul_b(cudaStream_t st, int32_t s, int32_t nsys, const double *R2, const double *R1, double *out);
// jlim (may be NULL): system b takes step j only when j < jlim[b] (its state is kept otherwise)
int launch_arnoldi_ls_b(cudaStream_t st, int32_t s, int32_t nsys, int32_t j, int32_t m, const double *H1,
                        const double *H2, const double *Rsub, double *Qs, double *Rtri, double *G, const double *thresh,
                        double *est, int32_t *flag, const int32_t *jlim = nullptr);
int launch_set_rhs_b(cudaStream_t st, int32_t s, int32_t nsys, int32_t m, const double *S0, double *G);
// jlim (may be NULL): system b solves for its first min(J, jlim[b]) block rows, the rest of Y zero
int launch_backsolve_b(cudaStream_t st, int32_t s, int32_t nsys, int32_t J, int32_t m, const double *Rtri,
                       const double *G, double *Y, const int32_t *jlim = nullptr);
int krylov_chunks(int32_t n);
// doubles needed for the partial sums of launch_block_dot with up to nblk_max blocks
size_t dot_partial_elems(int32_t s, int32_t nblk_max);
int launch_colnorm2(cudaStream_t st, int32_t s, int32_t n, const double *W, double *partial,
                    double *out, int chunks);
int launch_block_dot(cudaStream_t st, int32_t s, int32_t n, int32_t nblk, const double *V,
                     const double *W, double *partial, double *out, int chunks);
int launch_block_update(cudaStream_t st, int32_t s, int32_t n, int32_t nblk, const double *V,
                        const double *H, const double *base, double *out, double sign);
int launch_chol_small(cudaStream_t st, int32_t s, const double *G, const double *ref2,
                      double tau2, double *R, int32_t *deflated);
int launch_trsm_rows(cudaStream_t st, int32_t s, int32_t n, const double *W, const double *R,
                     const int32_t *deflated, double *out);
// 16-column blocks on the 8-column tensor-core kernels: W (n x 16) <-> halves Wl, Wr = Wl +
// 8 n (n x 8 each); H (nb blocks of 16 x 16) <-> 8 x 8 pieces HL / HR of the 2 nb half-blocks
int launch_halves16(cudaStream_t st, int32_t n, double *W, double *Wl, bool merge);
int launch_pieces16(cudaStream_t st, int32_t nb, double *H, double *HL, double *HR, bool merge);
// Cholesky-QR pieces with rows held in registers (s <= 8): G = W^T W; and Q1 = W R^{-1}
// written to Q1 together with G2 = Q1^T Q1.  partial needs 1216 * s * s doubles.
bool gram_rows_supported(int32_t s);
int launch_gram_rows(cudaStream_t st, int32_t s, int32_t n, const double *W, double *partial, double *out);
int launch_trsm_gram(cudaStream_t st, int32_t s, int32_t n, const double *W, const double *R,
                     const int32_t *deflated, double *Q1, double *partial, double *G2);
int launch_triu_mul(cudaStream_t st, int32_t s, const double *R2, const double *R1, double *out);
// Cholesky-QR W = Q R (s <= 8) in three launches whose last CTA (ticket, zero before the
// first launch and left zero) finishes each pass: R1 = chol(W^T W) with deflation against
// ref2 (tau2); Q1 = W R1^{-1} stored in Q (Q must not overlap W), R2 = chol of its Gram,
// Rout = R2 R1; Q := Q1 R2^{-1} in place.  partial: cqr_chunks(n) * s * s doubles.  Column
// norms^2 the same way (out: s doubles).  With H1 non-null, W is what two block CGS passes
// with coefficients H1, H2 (hrows x s each, against an orthonormal basis) left of a block
// W0, and the deflation scale is W0's column norms^2, ||(H1 + H2)(:, c)||^2 + (W^T W)_cc;
// ref2 is then not read.
bool cqr_supported(int32_t s);
int cqr_chunks(int32_t n);
int launch_cqr_gram(cudaStream_t st, int32_t s, int32_t n, const double *W, const double *ref2, double tau2,
                    const double *H1, const double *H2, int32_t hrows, double *partial, unsigned *ticket,
                    double *R1, int32_t *defl1);
int launch_cqr_gram2(cudaStream_t st, int32_t s, int32_t n, const double *W, const double *R1, const int32_t *defl1,
                     double *Q1, double *partial, unsigned *ticket, double *R2, int32_t *defl2, double *Rout);
// (Q32: non-null for an FP32 copy of Q as well)
int launch_cqr_apply(cudaStream_t st, int32_t s, int32_t n, double *Q, const double *R2, const int32_t *defl2,
                     float *Q32);
int launch_colnorm2_t(cudaStream_t st, int32_t s, int32_t n, const double *W, double *partial, unsigned *ticket,
                      double *out);
// projected least squares of block column j (Hessenberg column = H1 + H2 over Rsub)
int launch_arnoldi_ls(cudaStream_t st, int32_t s, int32_t j, int32_t m, const double *H1, const double *H2,
                      const double *Rsub, double *Qs, double *Rtri, double *G, const double *thresh, double *est,
                      int32_t *flag);
int launch_set_rhs(cudaStream_t st, int32_t s, int32_t m, const double *S0, double *G);
// least-squares state with kb identity block columns first (recycled space), S0 at block kb
int launch_ls_prefix(cudaStream_t st, int32_t s, int32_t kb, int32_t m, const double *S0, double *Qs, double *Rtri,
                     double *G);
int launch_backsolve(cudaStream_t st, int32_t s, int32_t J, int32_t ldr, const double *Rtri,
                     const double *G, double *Y);
int launch_axpy(cudaStream_t st, int64_t count, double alpha, const double *x, double *y);
int launch_residual(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr,
                    const int32_t *colind, const double *val, const double *X, const double *B,
                    double *R);
int launch_zero(cudaStream_t st, int64_t count, double *dst);
// G = W^T W (s x s) summing only the pairs a <= b; partial needs 1216 * s * s doubles
int launch_gram_sym(cudaStream_t st, int32_t s, int32_t n, const double *W, double *partial, double *out);
// out[p] = sum over chunks of partial[chunk * count + p] (deterministic)
int launch_reduce_chunks(cudaStream_t st, int32_t count, int chunks, const double *partial, double *out);

// ---------------------------------------------------------------------- k_ozaki.cu
// Bounded waits of the tensor-core kernels: pipeline waits give up after ns nanoseconds
// (the drain of a CTA's own copies and MMAs keeps 1 s); stall != 0 adds, at the start of
// the MMA issuer, a bounded wait on a barrier that nothing completes (a test of the
// give-up path).
struct TcWait {
    uint64_t ns = 1000000000ull;
    int stall = 0;
};
// FP64-accurate products on the tensor cores (s == 8): basis blocks as fixed point (Vf,
// from launch_to_fixed, |v| < 2), W as FP64; BF16 digits are cut in shared memory.
bool block_dot_tc_supported(int32_t s);
size_t tc_partial_elems(int32_t n, int32_t nblk);
// fixed point of nblocks blocks in the row layout (F_row, like X) and/or the sub-tile
// layout (F_sub: block slots iblk0.. of an array of ipad slots, tc_fixed_sub_bytes(n, ipad))
size_t tc_fixed_sub_bytes(int32_t n, int32_t nblocks);
int launch_to_fixed(cudaStream_t st, int32_t n, int32_t nblocks, const double *X, uint64_t *F_row, uint64_t *F_sub,
                    int32_t ipad, int32_t iblk0, int *d_err);
// H = V_{0..nblk-1}^T W (H[i][a][b]) from the sub-tile layout of ipad slots; partial needs
// tc_partial_elems(n, nblk) doubles
int launch_block_dot_tc(cudaStream_t st, int32_t n, int32_t nblk, const uint64_t *Vfs, int32_t ipad, const double *W,
                        double *partial, double *out, int *d_err, TcWait wt);
// out = base + sign * V_{0..nblk-1} H (base may be null, may equal out): H is nblk*8 x 8
// ([i][a][b]); hdig needs tc_hdig_bytes(nblk) bytes, hexp 8 ints
int block_update_tc_max_blocks();
size_t tc_hdig_bytes(int32_t nblk);
int launch_block_update_tc(cudaStream_t st, int32_t n, int32_t nblk, const uint64_t *Vf, const double *H, void *hdig,
                           int32_t *hexp, const double *base, double *out, double sign, int *d_err, TcWait wt);
// Q := Q1 R2^{-1} in place, Q holding Q1 = W R1^{-1} from launch_cqr_gram2 (s == 8,
// deflated columns -> 0, the last pass of the fused Cholesky-QR) with the new basis block's
// fixed point, laid out as launch_trsm_fixed does
int launch_cqr_apply_fixed(cudaStream_t st, int32_t n, double *Q, const double *R2, const int32_t *defl2,
                           uint64_t *F_row, uint64_t *F_sub, int32_t ipad, int32_t blk, int *d_err, float *Q32);
// Q := Q R^{-1} in place (s == 8, deflated columns -> 0) and the new basis block's fixed
// point: row layout at F_row (n x 8), sub-tile layout at slot blk of ipad slots of F_sub
int launch_trsm_fixed(cudaStream_t st, int32_t n, double *Q, const double *R, const int32_t *deflated, uint64_t *F_row,
                      uint64_t *F_sub, int32_t ipad, int32_t blk, int *d_err);
// FP64 FMA throughput probe: blocks x threads x 8 chains x iters FMAs
int launch_fp64_probe(cudaStream_t st, int blocks, int threads, int iters, double *sink);
// FP32 FMA throughput probe: blocks x threads x 8 chains x iters FMAs
int launch_fp32_probe(cudaStream_t st, int blocks, int threads, int iters, float *sink);

}  // namespace spai

/*
 * spai_gb300 -- C ABI of the GB300 (sm_103a) library for SPAI preconditioning of
 * parametric shifted second-order systems, its cheap parameter update, and the
 * right-preconditioned block GMRES solve that applies it.
 *
 * Method: arXiv 1809.06574 (Singh & Ahuja, "Preconditioned Linear Solves for Parametric
 * Model Order Reduction").  Each entry point below cites the passage that defines the
 * operation it performs.
 *
 * General rules
 *  - Plain C types only.  Indices are int32 (nnz < 2^31, checked).  Values are FP64.
 *  - Matrices are CSR with strictly increasing column indices in every row (checked:
 *    SPAI_EINVAL).  Only square matrices are accepted.
 *  - Dense blocks (B, X, Y) are column-major n x s arrays with a leading dimension >= n.
 *  - Unless stated otherwise, pointers are DEVICE pointers to memory the caller owns and
 *    keeps alive for the duration of the call.  Entry points that also accept HOST
 *    pointers say so; they detect the memory kind with cudaPointerGetAttributes.
 *  - Handles (spai_ctx, spai_affine, spai_pc) are owned by the library and released
 *    with their destroy call.  A handle must not outlive the context that made it.
 *  - Work is enqueued on the context's CUDA stream.  Calls return after enqueueing
 *    except where a call must read a result on the host (noted per call).
 *  - No call aborts, traps or exits: every failure is a status code, with a message
 *    readable through spai_last_error(ctx).  Device-side checks report through an error
 *    word, never through a trap.
 */
#ifndef SPAI_GB300_H
#define SPAI_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SPAI_API __attribute__((visibility("default")))
#else
#define SPAI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPAI_OK = 0,
    SPAI_EINVAL = 1,     /* malformed argument or matrix */
    SPAI_ENOMEM = 2,     /* device allocation failed or the context's budget is exceeded */
    SPAI_ECUDA = 3,      /* a CUDA runtime call failed */
    SPAI_ESINGULAR = 4,  /* a column least-squares problem is rank deficient */
    SPAI_ENOTCONV = 5,   /* block_solve reached max_cycles before every column converged */
    SPAI_ETIMEOUT = 6    /* a bounded device-side wait gave up */
} spai_status;

/* Square CSR matrix: rowptr[n+1], colind[nnz] (ascending within each row), val[nnz]. */
typedef struct {
    int32_t n;
    int32_t nnz;
    const int32_t *rowptr;
    const int32_t *colind;
    const double *val;
} spai_csr;

typedef struct spai_ctx_s *spai_ctx;
typedef struct spai_affine_s *spai_affine;
typedef struct spai_pc_s *spai_pc;

/* Column patterns of the preconditioner (the paper's MSPAI run grows the pattern
 * adaptively, Sec. 3; here it is fixed). */
#define SPAI_PATTERN_A 0   /* J_k = rows of column k of A */
#define SPAI_PATTERN_A2 1  /* J_k = rows of column k of A^2 (structural) */

/* Working precision of a factor, OR-ed into spai_build's pattern_kind or spai_update's
 * approach.  Default FP64.  SPAI_PREC_FP32: the column least-squares problems are solved
 * in FP32 (A's values rounded once) and the factor is stored in FP32; every apply reads
 * the FP32 values and forms products and sums in FP64, so the preconditioner stays an
 * exactly linear operator and block_solve's FP64 residuals and tolerance are unchanged.
 * No counterpart in the paper: the mixed-precision form of its preconditioner. */
#define SPAI_PREC_FP32 0x100
/* SPAI_PREC_BF16: the least-squares problems are solved in FP32 as for SPAI_PREC_FP32 and
 * each factor entry is rounded to nearest-even BF16 for storage (2 bytes per entry); the
 * apply converts exactly to FP64 and forms products and sums in FP64.  Exclusive with
 * SPAI_PREC_FP32 (SPAI_EINVAL if both are set). */
#define SPAI_PREC_BF16 0x200
/* SPAI_LS_NORMAL, OR-ed into spai_build's pattern_kind, spai_update's approach or
 * spai_build_batch's kinds: each column least-squares problem (Sec. 2.2; the update's,
 * Sec. 2.4) is solved by its normal equations instead of Householder QR -- G = Ahat^T Ahat
 * and h = Ahat^T rhs summed over the nonzero entries of Ahat's columns, G = R^T R by
 * Cholesky, two triangular solves, one GPU lane per column.  The same minimiser in exact
 * arithmetic, at a fraction of the work for sparse tiles, with a rounding error that grows
 * with cond(Ahat)^2 instead of cond(Ahat); a column is rank deficient (status 1, entries 0)
 * when a Cholesky pivot R_cc^2 is at most rel^2 times the largest diagonal entry of G, rel
 * = 1e-7 in FP64 and 1e-3 in FP32 (QR's test is |R_cc| <= 1e-14 / 1e-5 times max |R_tt|).
 * Tiles larger than 32 rows x 8 columns are solved by QR as without the flag.  Not the
 * paper's solver for these problems: an opt-in for well-conditioned sparse tiles. */
#define SPAI_LS_NORMAL 0x400

/* Update approaches of Table 1 (Sec. 2.3). */
#define SPAI_UPDATE_FIRST 1    /* min ||A(1) - A(l) Q||_F, P_l = Q_l P_1 (proposed, Sec. 2.4) */
#define SPAI_UPDATE_CHAINED 2  /* min ||A(l-1) - A(l) Q||_F, P_l = Q_l P_{l-1} */
/* OR-ed into either approach: Q_l diagonal (Sec. 2.4 states no pattern for Q_l; this is
 * the diagonal reading): the column least squares over J_k = {k}, whose rows are
 * I_k = rows(A(l)(:,k)), q_kk = <A(l)(:,k), a_k> / ||A(l)(:,k)||^2 with a_k the base
 * column; a zero column of A(l) is rank deficient (q_kk = 0, SPAI_ESINGULAR).  One dot
 * product per column instead of a QR; applied as a row scaling. */
#define SPAI_UPDATE_DIAGONAL 4

/* ----------------------------------------------------------------------------------
 * Context
 * ---------------------------------------------------------------------------------- */

/* Create a context bound to the current CUDA device and to `stream` (a cudaStream_t;
 * NULL = the legacy default stream).  `mem_budget` caps the device bytes the library
 * holds at once (0 = no cap); exceeding it returns SPAI_ENOMEM.  The stream is not
 * owned.  *out is NULL on failure.
 *
 * Threads: one context serves one host thread at a time.  Several contexts (each with its
 * own stream, used from its own thread) may share read-only handles: an spai_affine, or
 * an spai_pc once the call that made it has returned, can be passed to spai_assemble,
 * spai_update, spai_pc_apply and block_solve on another context concurrently.  A handle
 * must not be destroyed while another call uses it; an update made on context B from a
 * base made on context A belongs to B and is destroyed by B's thread. */
SPAI_API spai_status spai_ctx_create(spai_ctx *out, void *stream, size_t mem_budget);

/* Release the context's workspace.  Every spai_affine / spai_pc made with it must have
 * been destroyed first. */
SPAI_API spai_status spai_ctx_destroy(spai_ctx ctx);

/* Message of the last failed call on this context (never NULL; "" if none). */
SPAI_API const char *spai_last_error(spai_ctx ctx);

/* Block the host until the context's stream has finished its work. */
SPAI_API spai_status spai_ctx_sync(spai_ctx ctx);

/* Time limit of the bounded device-side waits of this context's tensor-core products (the
 * block Gram-Schmidt kernels of block_solve, spai_block_gram and spai_block_update), in
 * seconds, 0 < seconds <= 10 (default 1).  A pipeline wait that runs out makes its kernel
 * stop, wait for its own copies and tensor-core operations in flight (those waits keep a 1 s
 * limit), free its tensor memory and return; the call then returns SPAI_ETIMEOUT (block_solve
 * at the end of that Arnoldi step) and the context stays usable. */
SPAI_API spai_status spai_ctx_set_wait_limit(spai_ctx ctx, double seconds);

/* Test of the give-up path above: each of the next `count` tensor-core product launches on
 * this context also waits, within the limit, on a barrier that nothing completes, so its
 * wait runs out.  count 0 cancels.  No counterpart in the paper (failure detection). */
SPAI_API spai_status spai_ctx_inject_stall(spai_ctx ctx, int32_t count);

/* Device bytes currently held by the library for this context (handles + workspace). */
SPAI_API size_t spai_ctx_mem_in_use(spai_ctx ctx);

/* Release the context's grow-only workspace (the Krylov basis and blocks of block_solve,
 * staging blocks of the product calls); the next call that needs it allocates it again.
 * The memory is returned in stream order on the context's stream. */
SPAI_API spai_status spai_ctx_trim(spai_ctx ctx);

/* Number of kernels the library has launched in this process (all contexts). */
SPAI_API int64_t spai_launch_count(void);

/* Diagnostics: measured FP64 fused-multiply-add throughput of the current device in
 * TFLOP/s (a short kernel of independent FMA chains on every SM; synchronises).  Most of
 * this library's FP64 kernels are bound by this rate rather than by HBM bandwidth. */
SPAI_API spai_status spai_measure_fp64_rate(spai_ctx ctx, double *tflops);

/* Diagnostics: measured FP32 (non-tensor) fused-multiply-add throughput of the current
 * device in TFLOP/s, measured the same way (synchronises).  It is what the FP32 kernels
 * could reach: the FP32 column problems of FP32 builds, and the FP32 operator products of
 * the mixed-precision solve.  Like the FP64 probe, it has no counterpart in the paper. */
SPAI_API spai_status spai_measure_fp32_rate(spai_ctx ctx, double *tflops);

/* Optional timing of the library's kernels by family ("spmm_A", "block_dot", ...): while
 * enabled, each launch is bracketed by CUDA events recorded on the context's stream and
 * credited with the algorithmic flops and bytes of that launch.  spai_ctx_profile
 * enables / disables and clears the totals. */
SPAI_API spai_status spai_ctx_profile(spai_ctx ctx, int32_t enable);
/* Number of kernel families recorded so far (synchronises the stream). */
SPAI_API int32_t spai_ctx_profile_count(spai_ctx ctx);
/* Totals of family i: launches, summed event time (ms), algorithmic flops and bytes.
 * A family named "idle:<family>" is not a kernel: it sums the stream time between the
 * previous profiled launch and each launch of <family> (other work on the stream, or the
 * device waiting for the host), with zero flops and bytes.
 * *name stays valid until the next spai_ctx_profile call. */
SPAI_API spai_status spai_ctx_profile_entry(spai_ctx ctx, int32_t i, const char **name,
                                            int64_t *launches, double *ms, double *flops,
                                            double *bytes);

/* ----------------------------------------------------------------------------------
 * Affine assembly, Sec. 1.1 Eqs. (4)-(9): A = A_0 + s~_1 A_1 + ... + s~_{w+1} A_{w+1},
 * every A(l) being the same combination with other coefficients.  The terms are
 * merged once onto the union of their patterns (structural zeros kept); afterwards
 * every A(l) costs one value-only pass.
 * ---------------------------------------------------------------------------------- */

/* Copy `nterms` (1..16) CSR terms of equal size n into library memory and build the
 * union pattern.  terms[t] pointers may be HOST or DEVICE memory.  Validates every term
 * (SPAI_EINVAL).  Synchronises the stream once (it reads the union size). */
SPAI_API spai_status spai_affine_create(spai_ctx ctx, int32_t nterms, const spai_csr *terms,
                               spai_affine *out);

/* Union pattern (device pointers owned by the handle, valid until it is destroyed). */
SPAI_API spai_status spai_affine_pattern(spai_affine aff, int32_t *n, int32_t *nnz,
                                const int32_t **rowptr, const int32_t **colind);

/* val_out[q] = sum_t coef[t] * term_t(q) on the union pattern, t in order, each product
 * and sum rounded separately.  coef: HOST array of nterms doubles.  val_out: device,
 * nnz doubles.  Asynchronous. */
SPAI_API spai_status spai_assemble(spai_ctx ctx, spai_affine aff, const double *coef, double *val_out);

/* Coefficients of the shifted parametric second-order system, Sec. 1.1 Eqs. (3)-(9), with
 * the Rayleigh damping of the experiments (Sec. 3: D = alpha M + beta K):
 *   A(p, s) = s^2 M + s D(p) + K(p),  K(p) = K_0 + sum_i p_i K_i,  D(p) = alpha M + beta K(p)
 * collected over the terms (M, K_0, K_1, ..., K_np):
 *   coef[0] = s*s + alpha*s,  coef[1] = 1 + beta*s,  coef[1 + i] = (1 + beta*s) * p_i,
 * each product and sum rounded separately (no fused multiply-add).  p: HOST array of np
 * parameters (may be NULL when np = 0); coef: HOST array of np + 2 doubles.  0 <= np <= 14.
 * Host arithmetic only (no context, no device work).  SPAI_EINVAL on bad sizes, NULL
 * pointers or non-finite inputs. */
SPAI_API spai_status spai_shifted_coefficients(int32_t np, const double *p, double s, double alpha, double beta,
                                               double *coef);

/* val_out = A(p, s) on the union pattern of `aff`, whose terms must be (M, K_0, ..., K_np)
 * (nterms = np + 2, else SPAI_EINVAL): the coefficients of spai_shifted_coefficients, then
 * spai_assemble.  p: HOST, np doubles.  val_out: device, nnz doubles.  Asynchronous. */
SPAI_API spai_status spai_assemble_shifted(spai_ctx ctx, spai_affine aff, double s, int32_t np, const double *p,
                                           double alpha, double beta, double *val_out);

/* Copy the union pattern into caller memory (HOST or DEVICE): rowptr[n+1], colind[nnz].
 * Synchronises the stream. */
SPAI_API spai_status spai_affine_export(spai_ctx ctx, spai_affine aff, int32_t *rowptr,
                                        int32_t *colind);

/* Releases the assembly handle and its device arrays (the pattern arrays returned by
 * spai_affine_pattern become invalid).  The release is stream-ordered on the creating
 * context's stream: work queued there before the call still sees the arrays; work on
 * other streams that reads them must be complete first.  SPAI_EINVAL on NULL. */
SPAI_API spai_status spai_affine_destroy(spai_affine aff);

/* ----------------------------------------------------------------------------------
 * SPAI build, Sec. 2.2: min_P ||I - A P||_F^2 = sum_k min ||e_k - A p_k||_2^2, one
 * small least-squares problem per column over the fixed pattern J_k, restricted to
 * the rows I_k = union of rows(A(:,j)), j in J_k.  Solved on the device by Householder
 * QR of A(I_k, J_k) and back substitution.
 * ---------------------------------------------------------------------------------- */

/* Build P for A (device CSR, values read during the call).  pattern_kind is
 * SPAI_PATTERN_A or SPAI_PATTERN_A2, optionally OR SPAI_PREC_FP32 (FP32 least squares
 * and factor, rank-deficiency test |R_cc| <= 1e-5 max|R_tt|) or SPAI_PREC_BF16 (the same,
 * factor stored in BF16).  The handle keeps the
 * pattern analysis (I_k, J_k),
 * A's values in column order (for later updates) and P in row order (for the apply).
 * Column kernel: the first build or update of the process that meets a tile shape
 * (working precision, max |I_k| rounded up to 8, max |J_k|) times every fitting kernel
 * variant -- shared-memory tiles with teams of 1 ... 32 lanes per column, and
 * register-tiled variants for tiles up to 32 x 13 -- on up to 262,144 of its columns and
 * keeps the fastest for the rest of the process (one thread tunes at a time; variants
 * differ only in the rounding order of the reductions, within the FP64 bar).
 * Synchronises once (reads index-set sizes and the column status).  Returns
 * SPAI_ESINGULAR if some column problem is rank deficient (|I_k| < |J_k| or
 * |R_cc| <= 1e-14 max|R_tt|): the handle is still returned, those columns are zero,
 * and spai_pc_export reports them. */
SPAI_API spai_status spai_build(spai_ctx ctx, const spai_csr *A, int32_t pattern_kind, spai_pc *out);

/* Build the SPAI preconditioners of nsys independent systems at once (Sec. 2.2: every
 * column of every system is an independent least-squares problem).  A[i] and
 * pattern_kind[i] are as for spai_build (the pattern and the precision may differ between
 * systems); out[i] receives system i's handle, the same kind of handle spai_build returns
 * (update, apply, solve and destroy it on its own).  With two or more systems, none of
 * them empty, the systems are stacked into one block-diagonal matrix and each phase of the
 * pattern analysis (transposition, the unions J_k and I_k, the row pattern of P) is one
 * launch over all of them; the per-system arrays of the analyses and the factors are carved
 * from ONE device allocation shared by the batch's handles, which is freed when the last
 * of them (and of the updates that share their analyses) is destroyed -- so destroying
 * some handles of a batch returns no memory until the rest go too.  Otherwise (one system,
 * or an empty one) the analyses run phase by phase per system with one host read-back per
 * phase.  The column problems of all systems run in one persistent launch per tile shape --
 * systems are grouped by working precision, max |J_k| and max |I_k| rounded up to 8.
 * Kernel variant per shape: chosen and cached as for spai_build (the same process-wide
 * choice serves both; variants change the rounding of the reductions only, results stay
 * within the FP64 bar of spai_build).  1 <= nsys <= 65536.  Synchronises.
 * Returns SPAI_ESINGULAR (handles still returned) if some column of some system is rank
 * deficient; on any other error no handle is returned. */
SPAI_API spai_status spai_build_batch(spai_ctx ctx, int32_t nsys, const spai_csr *A, const int32_t *pattern_kind,
                                      spai_pc *out);

/* Cheap update, Table 1 and Sec. 2.4: for A_new = A(l) on the SAME pattern as the base
 * matrix, column k of Q_l = argmin_{supp q in J_k} ||a1_k - A(l) q||_2 with a1_k column
 * k of A(1) (approach SPAI_UPDATE_FIRST: A(1) is the root build's matrix; approach
 * SPAI_UPDATE_CHAINED: A(1) is `base`'s own matrix).  The preconditioner of A(l) is
 * P_l = Q_l P_base, applied factored as Q_l (P_base X).  No pattern analysis is redone.
 * `base` must stay alive while the result is used.  Synchronises once (column status).
 * approach may be OR-ed with SPAI_PREC_FP32 (this factor in FP32; the chain may mix
 * precisions).  Returns SPAI_ESINGULAR like spai_build. */
SPAI_API spai_status spai_update(spai_ctx ctx, spai_pc base, const spai_csr *A_new, int32_t approach,
                        spai_pc *out);

/* ----------------------------------------------------------------------------------
 * Adaptive SPAI (the pattern growth of the MSPAI code the paper's experiments run, Sec. 3,
 * "tolerance 1e-4", around the column least squares of Sec. 2.2).  For each column k,
 * J_k starts as {k}; each step solves the column least squares on J_k (rows I_k = {k} and
 * the rows of the columns in J_k), forms the residual r = e_k - A m_k, takes as
 * candidates the columns j not in J_k with a nonzero in a row of I_k, scores each by the
 * squared residual after the best one-column correction, rho_j = ||r||^2 - (r . A(:,j))^2
 * / ||A(:,j)||^2, and adds the max_new best among those not above the candidates' mean
 * (scores compared as floor(rho / ||r||^2 * 2^30), ties by the lower column index).  It
 * stops when ||r||_2 <= eps, after max_steps steps, on a rank-deficient column problem,
 * when no candidate is left, or when |I_k| would exceed max_rows (that step is undone).
 * Every candidate of a step is scored, however many there are (the kernel scores them in
 * windows of 1024).  The search runs in FP64; the factor on the final pattern is then computed by
 * the column kernel of spai_build in the precision that `flags` selects.  The handle is an
 * ordinary one: spai_update keeps its pattern (the update skips the search, Sec. 2.3-2.4),
 * and apply, solve, export and destroy work as for spai_build.
 * ---------------------------------------------------------------------------------- */
typedef struct {
    double eps;         /* target ||e_k - A m_k||_2 of every column (the paper's 1e-4) */
    int32_t max_steps;  /* pattern-growth steps per column, >= 0 */
    int32_t max_new;    /* columns added per step, >= 1; 1 + max_steps * max_new <= 32 */
    int32_t max_rows;   /* largest |I_k|, 1 ... 128 */
    int32_t reserved;   /* 0 */
} spai_adaptive_opts;

/* Build an adaptive SPAI of A (device CSR).  opts NULL: eps 1e-4, max_steps 5, max_new 5,
 * max_rows 128.  flags: 0 (FP64 factor), SPAI_PREC_FP32 or SPAI_PREC_BF16.  Columns whose
 * growth stopped at a size limit keep the pattern they had.  Synchronises a few times.
 * Returns SPAI_ESINGULAR as spai_build does (handle still returned). */
SPAI_API spai_status spai_build_adaptive(spai_ctx ctx, const spai_csr *A, const spai_adaptive_opts *opts,
                                         int32_t flags, spai_pc *out);

/* Kernel variants of the column least squares (process-wide; no device work).  A tile
 * shape is (low_precision: 0 FP64 / 1 FP32 working precision, max |I_k|, max |J_k|); its
 * variants are shared-memory tiles with teams of T = 1 ... 32 lanes per column (code T)
 * and register-tiled kernels (codes >= 64).  Every variant solves the same column
 * problems and differs only in the rounding order of the reductions.
 *   spai_column_variants: writes the codes that fit the shape to codes[0 .. cap-1] and
 *     returns how many fit (the first one is the untuned default).
 *   spai_column_variant_get: the code the process uses for the shape (the tuned or pinned
 *     one; max |I_k| counts rounded up to a multiple of 8), or 0 before the first build or
 *     update of that shape.
 *   spai_column_variant_set: pins the shape to `code` for the rest of the process (code 0
 *     clears it: the next build or update of the shape tunes again) -- for results that
 *     are bitwise reproducible across processes, or to test one variant.  SPAI_EINVAL if
 *     the code does not fit the shape. */
SPAI_API int32_t spai_column_variants(int32_t low_precision, int32_t maxI, int32_t maxJ, int32_t *codes, int32_t cap);
SPAI_API int32_t spai_column_variant_get(int32_t low_precision, int32_t maxI, int32_t maxJ);
SPAI_API spai_status spai_column_variant_set(int32_t low_precision, int32_t maxI, int32_t maxJ, int32_t code);

/* Sizes: n, nnz of this handle's own factor (P or Q_l; n for a diagonal update), total
 * length of the I_k lists, and depth (0 = built, 1 = updated from a build, ...).  Host outputs, any may be NULL. */
SPAI_API spai_status spai_pc_info(spai_pc pc, int32_t *n, int32_t *nnz, int64_t *nI, int32_t *depth);

/* Copy out this handle's own factor in column order on its pattern -- Jptr[n+1],
 * Jind[nnz], val[nnz] -- the row sets Iptr[n+1], Ilist[nI], and col_status[n] (0 ok, 1
 * singular).  A diagonal update exports J_k = {k}, its values, and I_k = rows(A(:,k))
 * (Ilist then holds nnz(A) entries).  DEVICE pointers; any may be NULL.  Asynchronous. */
SPAI_API spai_status spai_pc_export(spai_ctx ctx, spai_pc pc, int32_t *Jptr, int32_t *Jind, double *val,
                           int32_t *Iptr, int32_t *Ilist, int32_t *col_status);

/* Device bytes held by this handle's own factor and matrix values; with_analysis != 0
 * adds its pattern analysis (I_k, J_k, transposed pattern), which a build shares with
 * every update made from it and which is released with the last of them. */
SPAI_API size_t spai_pc_mem_size(spai_pc pc, int32_t with_analysis);

/* Releases the handle: its factor and matrix values, and its pattern analysis once the
 * last handle sharing it is gone (for spai_build_batch, the batch's one allocation once
 * all of its handles and their updates are gone).  Stream-ordered on the creating
 * context's stream, as spai_affine_destroy.  An update must not be used after its base
 * is destroyed.  SPAI_EINVAL on NULL. */
SPAI_API spai_status spai_pc_destroy(spai_pc pc);

/* ----------------------------------------------------------------------------------
 * Products of the right-preconditioned Krylov method (Sec. 2.2 footnote: A P X~ = B,
 * X = P X~).  s in {1, 2, 4, 8, 16}.  Column-major device blocks.  Asynchronous.
 * ---------------------------------------------------------------------------------- */

/* Y = A X. */
SPAI_API spai_status spai_spmm(spai_ctx ctx, const spai_csr *A, int32_t s, const double *X, int64_t ldx,
                      double *Y, int64_t ldy);

/* Y = P X for a handle (factored for updated handles: Q_l (P_base X)). */
SPAI_API spai_status spai_pc_apply(spai_ctx ctx, spai_pc pc, int32_t s, const double *X, int64_t ldx,
                          double *Y, int64_t ldy);

/* The FP32 operator of SPAI_SOLVE_MIXED (see block_solve) on its own: Y = A X and Y = P X
 * with the matrix's or factors' values and X rounded to FP32 (X once, before the product,
 * as the solve keeps its newest basis block in FP32), products and sums in FP32 in each
 * row's order (a factored chain keeps its intermediate blocks in FP32), Y written as FP64
 * (exact).  Arguments as spai_spmm / spai_pc_apply.  Asynchronous. */
SPAI_API spai_status spai_spmm_fp32(spai_ctx ctx, const spai_csr *A, int32_t s, const double *X, int64_t ldx,
                                    double *Y, int64_t ldy);
SPAI_API spai_status spai_pc_apply_fp32(spai_ctx ctx, spai_pc pc, int32_t s, const double *X, int64_t ldx,
                                        double *Y, int64_t ldy);

/* Y = P X like spai_pc_apply, but without allocating any device memory.  The paper has
 * no counterpart: this entry point serves callers that cannot allocate at the point of
 * the apply -- an outside Krylov solver whose inner loop must not stall the device (a
 * cudaMalloc or cudaFree can synchronise it), or a process whose device memory is
 * already reserved by another allocator so that a new allocation would fail.
 * The staging blocks live in one fixed device array of 64 MiB built into the library,
 * which every device that loads the library holds until the process exits; n * s must
 * be <= 2,097,152, else SPAI_EINVAL.  X and Y must be DEVICE memory of the context's
 * device, which must be the current device (else SPAI_EINVAL).  The first call on each
 * device looks up the array's address and caches it for the rest of the process, so make
 * that call before any stream capture; a device reset (cudaDeviceReset) while the library
 * is loaded is not supported by this call.  All calls share the array: calls that overlap
 * on the GPU (other streams, other host threads) race.  Asynchronous on the context's
 * stream. */
SPAI_API spai_status spai_pc_apply_noalloc(spai_ctx ctx, spai_pc pc, int32_t s, const double *X,
                                           int64_t ldx, double *Y, int64_t ldy);

/* ----------------------------------------------------------------------------------
 * Block Krylov solve, Sec. 2.1 (block methods solve all right-hand sides at once in
 * span{R0, A R0, A^2 R0, ...}) with right preconditioning (Sec. 2.2 footnote): block
 * GMRES(m) on A P X~ = B, X = X0 + P X~.
 * ---------------------------------------------------------------------------------- */

/* How the block Gram products V^T W of the orthogonalisation are computed. */
#define SPAI_ORTH_AUTO 0    /* tensor-core digits when s == 8 and the product has >= 2 blocks, else FP64 */
#define SPAI_ORTH_FP64 1    /* FP64 fused multiply-adds on the CUDA cores */
#define SPAI_ORTH_TENSOR 2  /* tensor-core digits whenever s == 8 */

/* Arithmetic of the solve's operator products (no counterpart in the paper: the mixed-
 * precision form of its solve, with the accuracy won back by iterative refinement).
 * SPAI_SOLVE_FP64: every product in FP64 (FP32 / BF16 factors converted exactly).
 * SPAI_SOLVE_MIXED: inside each restart cycle the operator A P is applied in FP32 -- A's
 * values (rounded once per solve), the factors' values and each input block rounded to
 * FP32, products and sums in FP32 -- while the Krylov basis, the block Gram-Schmidt / QR,
 * the projected least squares and the true residual b - A x stay FP64.  Every cycle starts
 * from the FP64 true residual r (iterative refinement) and ends once each column's
 * estimate is below max(tol ||b_i||, 2^-20 ||r_i||) or the restart length is reached; the
 * solve stops when every column's FP64 true residual meets tol, as in SPAI_SOLVE_FP64.
 * The workspace grows by 4 nnz(A) bytes. */
#define SPAI_SOLVE_FP64 0
#define SPAI_SOLVE_MIXED 1

typedef struct {
    int32_t restart;     /* m: block Arnoldi steps per cycle, >= 1 */
    int32_t max_cycles;  /* restart cycles before SPAI_ENOTCONV, >= 1 */
    double tol;          /* stop when ||b_i - A x_i||_2 <= tol * ||b_i||_2 for every column */
    int32_t orth;        /* SPAI_ORTH_* */
    int32_t precision;   /* SPAI_SOLVE_FP64 (0) or SPAI_SOLVE_MIXED */
} spai_solve_opts;

/* Block Gram product H_i = V_i^T W, i < nblk, of the block orthogonalisation (Sec. 2.1).
 * V: nblk blocks of n x s, each row-major (s consecutive doubles per row) and back to
 * back; W: n x s row-major; H: nblk x s x s, H[i][a][b] = sum_r V_i[r][a] W[r][b].  All
 * DEVICE memory.  method SPAI_ORTH_FP64: FP64 on the CUDA cores; SPAI_ORTH_TENSOR (s == 8
 * only): every value is cut into nine 6-bit fixed-point digits (V's entries must satisfy
 * |v| < 2; W's columns are scaled by powers of two), digit products are summed exactly in
 * FP32 on the tensor cores and combined in FP64 -- as accurate as FP64 arithmetic.
 * Returns SPAI_EINVAL if a V entry is out of range, SPAI_ETIMEOUT if a bounded device
 * wait gave up.  Synchronises. */
SPAI_API spai_status spai_block_gram(spai_ctx ctx, int32_t s, int32_t n, int32_t nblk, const double *V,
                                     const double *W, double *H, int32_t method);

/* Block update of the orthogonalisation (Sec. 2.1): W := W + sign * sum_i V_i H_i, with V
 * and W laid out as for spai_block_gram and H as its output (nblk x s x s).  DEVICE
 * memory, in place.  method SPAI_ORTH_TENSOR (s == 8) uses the same digit scheme with the
 * basis rows as the MMA's M dimension.  Synchronises. */
SPAI_API spai_status spai_block_update(spai_ctx ctx, int32_t s, int32_t n, int32_t nblk, const double *V,
                                       const double *H, double *W, double sign, int32_t method);

typedef struct {
    int32_t iterations;        /* block Arnoldi steps over all cycles */
    int32_t cycles;            /* restart cycles run */
    int32_t converged;         /* 1 if every column met tol (true residual) */
    int32_t worst_column;      /* column with the largest relative true residual */
    double max_rel_residual;   /* that residual, ||b_i - A x_i|| / ||b_i|| (FP64) */
} spai_solve_info;

/* Device bytes of the workspace block_solve uses for n unknowns, s right-hand sides and
 * restart length m = restart (the context keeps it between calls; 0 for invalid sizes). */
SPAI_API size_t spai_solve_workspace_size(int32_t n, int32_t s, int32_t restart);

/* Solve nsys independent systems A_i X_i = B_i (s right-hand sides each) at once, each by
 * the right-preconditioned block GMRES(m) of block_solve, all of them in lockstep: the
 * matrix and preconditioner products run on the block-diagonal union of the systems, the
 * Gram-Schmidt products, Cholesky-QR and projected least squares per system (segmented
 * reductions, one CTA per system for the small blocks), and one read-back per Arnoldi step
 * covers every system's convergence test -- so the launches and synchronisations of a
 * step do not grow with nsys.  A system leaves the lockstep when its residual estimate
 * meets tol: its steps of the cycle are over (the per-step kernels run on the row chunks of
 * the systems still stepping), its X is updated at the cycle's end from its own steps, and
 * it takes part in later cycles only while its true residual is above tol -- so each
 * system takes the steps block_solve would take on it alone.  A[i]: DEVICE CSR (n_i >= 1, sum of n_i and of nnz below 2^31); P: NULL (no
 * preconditioner) or nsys handles whose chains have the same depth, each level of the
 * same kind (full or diagonal) and precision in every system; B[i], X[i]: DEVICE arrays
 * (host array of device pointers), n_i x s column-major, leading dimension n_i; X[i]
 * holds the initial guess on entry.  info: nsys entries (iterations = the Arnoldi steps the
 * system took over all cycles; cycles = the cycle after which its true residual met tol).
 * Orthogonalisation in FP64 (opts->orth ignored).  1 <= nsys <= 65536.  Synchronises.
 * Returns SPAI_ENOTCONV if some system did not converge. */
SPAI_API spai_status block_solve_batch(spai_ctx ctx, int32_t nsys, const spai_csr *A, const spai_pc *P, int32_t s,
                                       const double *const *B, double *const *X, const spai_solve_opts *opts,
                                       spai_solve_info *info);

/* Solve A X = B for s right-hand sides at once.  P may be NULL (no preconditioner).
 * B (n x s, ldb) and X (n x s, ldx) may be HOST or DEVICE memory; X holds the initial
 * guess on entry and the solution on return.  rel_residual: HOST array of s doubles
 * (or NULL) receiving every column's final relative true residual.  Synchronises: it
 * returns after the final true-residual check.  Returns SPAI_ENOTCONV (X still holds
 * the last iterate) if max_cycles ran out. */
SPAI_API spai_status block_solve(spai_ctx ctx, const spai_csr *A, spai_pc P, int32_t s, const double *B,
                        int64_t ldb, double *X, int64_t ldx, const spai_solve_opts *opts,
                        spai_solve_info *info, double *rel_residual);

/* ----------------------------------------------------------------------------------
 * Block GCRO, the solver of the paper's experiments (Sec. 3: GCRO and block GCRO), with its
 * outer space carried along a sequence of systems A(p_1) X = B, A(p_2) X = B, ... (Sec. 1.3).
 * A recycle space holds up to kmax columns U (in the preconditioned space of the right-
 * preconditioned solve).  For each solve, with AP = A P:
 *  - C T = AP U (block Gram-Schmidt and Cholesky-QR by s-column blocks; columns that AP U
 *    leaves dependent are dropped as the Krylov blocks' are), U <- U T^{-1}, so AP U = C;
 *  - every restart cycle starts from the residual projected off C (X~ += U C^T R,
 *    R -= C C^T R), runs block Arnoldi on (I - C C^T) AP with two passes of block classical
 *    Gram-Schmidt against [C, V], and minimises every column's residual over span([U, V]):
 *    AP [U, V_j] = [C, V_{j+1}] [[I, C^T AP V_j], [0, Hbar_j]];
 *  - the solve's iterate X~ (X = P X~) then joins U, the oldest s columns leaving a full
 *    space: the span of the sequence's latest solutions is the next system's start.
 * With an empty recycle space the solve is block_solve's block GMRES.
 * ---------------------------------------------------------------------------------- */
typedef struct spai_recycle_s *spai_recycle;

/* Recycle space for n unknowns and s right-hand sides: kmax columns at most (a multiple of s,
 * kmax / s <= 16), empty at first.  Device memory of the context (8 n kmax bytes). */
SPAI_API spai_status spai_recycle_create(spai_ctx ctx, int32_t n, int32_t s, int32_t kmax, spai_recycle *out);
/* Columns currently held (a multiple of s). */
SPAI_API spai_status spai_recycle_info(spai_recycle r, int32_t *k);
/* Copy the k columns to U (DEVICE, n x k column-major, leading dimension ldu >= n).  Asynchronous. */
SPAI_API spai_status spai_recycle_export(spai_ctx ctx, spai_recycle r, double *U, int64_t ldu);
/* Empty the space (the next solve starts without a recycled space). */
SPAI_API spai_status spai_recycle_clear(spai_recycle r);
SPAI_API spai_status spai_recycle_destroy(spai_recycle r);

/* Solve A X = B by block GCRO with the recycle space rc (arguments as block_solve; X holds
 * the initial guess on entry).  The workspace is that of block_solve with restart + kmax/s
 * basis blocks.  On success the iterate joins rc; rc is left as it was on a failure except
 * that its columns are rescaled (U <- U T^{-1}, the same span).  The recycle space may serve
 * one solve at a time.  Synchronises; SPAI_ENOTCONV as block_solve. */
SPAI_API spai_status block_solve_gcro(spai_ctx ctx, const spai_csr *A, spai_pc P, int32_t s, const double *B,
                                      int64_t ldb, double *X, int64_t ldx, const spai_solve_opts *opts,
                                      spai_recycle rc, spai_solve_info *info, double *rel_residual);

/* ----------------------------------------------------------------------------------
 * Serving.  The paper's setting is a sequence of linear systems A(p_j) X_j = B_j that
 * differ only in the parameter (Sec. 1.3), whose SPAI preconditioner is updated cheaply
 * from an earlier build instead of being rebuilt (Sec. 2.3, Table 1; Sec. 2.4).  A server
 * takes such solves as requests, as they arrive, for several registered systems:
 *  - it keeps every system (its affine terms), its cached SPAI builds and the Krylov
 *    workspaces resident on the device;
 *  - it runs up to `slots` requests at once, each on its own CUDA stream and context, so
 *    the kernels of different requests overlap on the GPU; a request is admitted when a
 *    slot is free and its device memory fits the budget (idle slots' workspaces are
 *    released first, then least recently used cached builds evicted, else it waits for
 *    running requests);
 *  - with `reuse`, a request whose parameter p lies within `radius` of a cached build's
 *    parameter, for the same system and the same shift s, is served by spai_update
 *    (SPAI_UPDATE_FIRST from that build) instead of a new build; at p equal to the
 *    build's it reuses the build itself; otherwise it builds and caches a new base.
 *    Without `reuse` every request builds its own factor (the plain method);
 *  - each request is solved by block_solve from X0 = 0 to the server's tolerance.
 * Results do not depend on what else runs: every kernel reduces in a fixed order, so a
 * request gives the same bits as the same route (build at the same base p, update,
 * solve) run alone through the calls above.
 * ---------------------------------------------------------------------------------- */
typedef struct spai_server_s *spai_server;

typedef struct {
    int32_t slots;         /* requests on the GPU at once, 1..64 */
    int32_t pattern_kind;  /* SPAI_PATTERN_A or SPAI_PATTERN_A2, optionally | SPAI_PREC_FP32 or SPAI_PREC_BF16,
                              | SPAI_LS_NORMAL (builds and updates alike) */
    int32_t reuse;         /* 1: cache builds and route nearby requests to spai_update; 0: build per request */
    int32_t restart;       /* block GMRES(m) restart length m */
    int32_t max_cycles;    /* restart cycles before a request fails with SPAI_ENOTCONV */
    int32_t orth;          /* SPAI_ORTH_* of the solves */
    double radius;         /* route to an update when |p - p_build| <= radius (same system and shift) */
    double tol;            /* every column's true relative residual <= tol */
    size_t mem_budget;     /* device bytes for systems, cached builds and in-flight requests (0: no cap);
                              a request counts its slot's workspace and buffers, its factor and,
                              for a build, 16 nnz + 16 (n + 1) + 1 MiB of pattern-analysis buffers */
    int32_t precision;     /* SPAI_SOLVE_FP64 or SPAI_SOLVE_MIXED: the solves' operator arithmetic */
    int32_t reserved;      /* 0 */
} spai_server_opts;

typedef struct {
    int32_t system;        /* id from spai_server_add_system */
    int32_t nrhs;          /* right-hand sides: 1, 2, 4, 8 or 16 */
    double p;              /* parameter value (routing distance) */
    double s;              /* shift (routing key: only builds at exactly this shift are reused) */
    const double *coef;    /* HOST, nterms doubles: A = sum_t coef[t] * term_t; copied at submit.
                              Requests with equal (system, s, p) must pass equal coefficients.
                              NULL for a system from spai_server_add_shifted_system: A(p, s) */
    const double *B;       /* HOST or DEVICE, n x nrhs column-major, leading dimension n; read
                              while the request runs, so it must stay valid until it completes */
    double *X;             /* HOST or DEVICE, n x nrhs, leading dimension n: the solution, written
                              when the request completes; NULL: the solution is not returned */
    double t_arrival;      /* arrival time on the server clock (spai_server_clock); < 0: now */
} spai_request;

#define SPAI_ROUTE_BUILD 0   /* a new SPAI build (cached when reuse is on) */
#define SPAI_ROUTE_UPDATE 1  /* spai_update from a cached build */
#define SPAI_ROUTE_REUSE 2   /* a cached build at the same p, used as it is */

typedef struct {
    int32_t status;            /* spai_status of the request */
    int32_t route;             /* SPAI_ROUTE_* */
    int32_t slot;              /* slot that ran it */
    int32_t iterations;        /* block Arnoldi steps */
    double base_p;             /* p of the build it used */
    double max_rel_residual;   /* largest true relative residual over its columns */
    double t_arrival, t_start, t_done;  /* server clock, seconds */
} spai_result;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t builds, updates, reuses, evictions, waits_for_memory;
    size_t mem_in_use;        /* bytes accounted now (systems, cache, slots, reservations) */
    size_t mem_peak;          /* the largest such figure so far */
    int32_t cached_builds;    /* cache entries now */
    int32_t reserved;
} spai_server_stats;

/* Create a server on the current device with `opts` (copied).  It starts `slots` host
 * worker threads, each with its own non-blocking stream and context.  Device inputs of a
 * request must be complete (synchronised) before it is submitted. */
SPAI_API spai_status spai_server_create(const spai_server_opts *opts, spai_server *out);

/* Register a system A = sum_t coef[t] term_t (spai_affine_create's rules: 1..16 CSR terms
 * of equal n, HOST or DEVICE arrays, copied); at most 1024 systems per server (SPAI_EINVAL
 * beyond).  *id receives its id (0, 1, ...).  Counts
 * against the memory budget (SPAI_ENOMEM if it does not fit).  Synchronises. */
SPAI_API spai_status spai_server_add_system(spai_server srv, int32_t nterms, const spai_csr *terms, int32_t *id);

/* Register a shifted parametric second-order system (Sec. 1.1 Eqs. (3)-(9), Rayleigh damping
 * D = alpha M + beta K(p) as in Sec. 3): terms = (M, K_0, K_1), so that a request's p and s
 * define A(p, s) = (s^2 + alpha s) M + (1 + beta s) (K_0 + p K_1) (spai_shifted_coefficients).
 * Requests to such a system may pass coef = NULL: the server forms these coefficients from
 * the request's p and s.  Otherwise as spai_server_add_system. */
SPAI_API spai_status spai_server_add_shifted_system(spai_server srv, const spai_csr *terms, double alpha, double beta,
                                                    int32_t *id);

/* Queue a request; *ticket identifies it for spai_server_wait.  Never blocks on the GPU. */
SPAI_API spai_status spai_server_submit(spai_server srv, const spai_request *req, int64_t *ticket);

/* Block until request `ticket` has completed, copy its result to *out (may be NULL) and
 * forget the ticket.  Returns SPAI_EINVAL for an unknown ticket, else SPAI_OK (the
 * request's own status is out->status). */
SPAI_API spai_status spai_server_wait(spai_server srv, int64_t ticket, spai_result *out);

/* Seconds since the server was created (steady clock): the time base of the results. */
SPAI_API double spai_server_clock(spai_server srv);

SPAI_API spai_status spai_server_stats_get(spai_server srv, spai_server_stats *out);

/* Message of the last failed server call or request ("" if none). */
SPAI_API const char *spai_server_last_error(spai_server srv);

/* Finish every queued request, stop the workers and release all device memory.  Results
 * not collected with spai_server_wait are dropped. */
SPAI_API spai_status spai_server_destroy(spai_server srv);

#ifdef __cplusplus
}
#endif

#endif /* SPAI_GB300_H */

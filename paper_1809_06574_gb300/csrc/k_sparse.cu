// Sparse-structure and streaming kernels of the SPAI path:
//  * CSR validation, union of the affine terms' patterns and value assembly
//    (Sec. 1.1, Eqs. (4)-(9): every A(l) is one affine combination of fixed matrices);
//  * CSR -> CSC transposition (column access for the column least-squares problems of
//    Sec. 2.2) and the row sets I_k = union of rows(A(:,j)), j in J_k;
//  * the CSR sparse-times-block product used for A P V in the block Krylov method
//    (Sec. 2.1) and for the preconditioner apply (Sec. 2.2 footnote).
#include <cuda_bf16.h>

#include <atomic>
#include <climits>

#include "spai_internal.cuh"

namespace spai {

static std::atomic<long long> g_launches{0};

void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t work, int threads = kThreads)
{
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > (1LL << 30)) g = 1 << 30;
    return (int)g;
}

inline int check_launch(int kernels = 1)
{
    note_launches(kernels);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------------
__global__ void k_validate_csr(int32_t n, int32_t nnz, const int32_t *__restrict__ rowptr,
                               const int32_t *__restrict__ colind, int *err)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0 && (rowptr[0] != 0 || rowptr[n] != nnz)) atomicOr(err, ERR_ROWPTR);
    if (i >= n) return;
    int32_t a = rowptr[i], b = rowptr[i + 1];
    if (a < 0 || b < a || b > nnz) {
        atomicOr(err, ERR_ROWPTR);
        return;
    }
    int32_t prev = -1;
    for (int32_t q = a; q < b; ++q) {
        int32_t c = colind[q];
        if (c < 0 || c >= n || c <= prev) {
            atomicOr(err, ERR_COLIND);
            return;
        }
        prev = c;
    }
}

// ---------------------------------------------------------------------------------
// union pattern of T terms (thread per row, T-way merge of sorted rows)
// ---------------------------------------------------------------------------------
template <bool FILL>
__global__ void k_union(int32_t n, int32_t T, TermPtrs tp, int32_t *counts,
                        const int32_t *__restrict__ u_rowptr, int32_t *__restrict__ u_colind,
                        double *__restrict__ aligned, int64_t nnzU)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t pos[kMaxTerms], end[kMaxTerms];
    for (int t = 0; t < T; ++t) {
        pos[t] = tp.rowptr[t][i];
        end[t] = tp.rowptr[t][i + 1];
    }
    int64_t out = FILL ? (int64_t)u_rowptr[i] : 0;
    int32_t cnt = 0;
    while (true) {
        int32_t m = INT_MAX;
        for (int t = 0; t < T; ++t)
            if (pos[t] < end[t]) m = min(m, tp.colind[t][pos[t]]);
        if (m == INT_MAX) break;
        if (FILL) u_colind[out + cnt] = m;
        for (int t = 0; t < T; ++t) {
            double v = 0.0;
            if (pos[t] < end[t] && tp.colind[t][pos[t]] == m) {
                v = tp.val[t][pos[t]];
                ++pos[t];
            }
            if (FILL) aligned[(int64_t)t * nnzU + out + cnt] = v;
        }
        ++cnt;
    }
    if (!FILL) counts[i] = cnt;
}

// val[q] = sum_t c_t * aligned_t[q], t in order, product and sum rounded separately
__global__ void k_assemble(int64_t nnz, int32_t T, const double *__restrict__ aligned,
                           TermPtrs tp, double *__restrict__ out)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int t = 0; t < T; ++t)
            acc = __dadd_rn(acc, __dmul_rn(tp.coef[t], __ldg(aligned + (int64_t)t * nnz + q)));
        out[q] = acc;
    }
}

// ---------------------------------------------------------------------------------
// exclusive scan of int32 counts into an int32 pointer array (3 phases, int64 carries)
// ---------------------------------------------------------------------------------
constexpr int kScanItems = 4;
constexpr int kScanTile = kThreads * kScanItems;

__device__ long long block_exclusive_scan(long long v, long long *total)
{
    __shared__ long long warp_sums[kThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long w = (lane < kThreads / 32) ? warp_sums[lane] : 0;
        long long wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kThreads / 32) warp_sums[lane] = wi - w;
        if (lane == kThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    long long r = incl - v + warp_sums[wid];
    __syncthreads();
    return r;
}

__global__ void k_scan_tile_sums(const int32_t *__restrict__ counts, int64_t n,
                                 long long *__restrict__ sums)
{
    __shared__ long long tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long s = 0;
    for (int u = 0; u < kScanItems; ++u)
        if (base + u < n) s += counts[base + u];
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(long long *sums, int64_t ntiles, int32_t *ptr, int64_t n, int *err)
{
    __shared__ long long tot;
    long long carry = 0;
    for (int64_t base = 0; base < ntiles; base += kThreads) {
        int64_t i = base + threadIdx.x;
        long long v = (i < ntiles) ? sums[i] : 0;
        long long ex = block_exclusive_scan(v, &tot);
        if (i < ntiles) sums[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (carry > INT_MAX) atomicOr(err, ERR_OVERFLOW);
        ptr[n] = (int32_t)carry;
    }
}

__global__ void k_scan_apply(const int32_t *__restrict__ counts, int64_t n,
                             const long long *__restrict__ sums, int32_t *__restrict__ ptr)
{
    __shared__ long long tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long v[kScanItems];
    long long s = 0;
    for (int u = 0; u < kScanItems; ++u) {
        v[u] = (base + u < n) ? counts[base + u] : 0;
        s += v[u];
    }
    long long ex = block_exclusive_scan(s, &tot) + sums[blockIdx.x];
    for (int u = 0; u < kScanItems; ++u) {
        if (base + u < n) ptr[base + u] = (int32_t)ex;
        ex += v[u];
    }
}

// ---------------------------------------------------------------------------------
// transposition
// ---------------------------------------------------------------------------------
__global__ void k_count_cols(int32_t nnz, const int32_t *__restrict__ colind, int32_t *cnt)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + colind[q], 1);
}

__global__ void k_fill_cols(int32_t n, const int32_t *__restrict__ rowptr,
                            const int32_t *__restrict__ colind, int32_t *next,
                            int32_t *__restrict__ rowind_tmp, int32_t *__restrict__ perm_tmp)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        int32_t d = atomicAdd(next + colind[q], 1);
        rowind_tmp[d] = (int32_t)i;
        perm_tmp[d] = q;
    }
}

// warp per column: place every entry at its rank (rows are distinct inside a column)
__global__ void k_rank_sort_cols(int32_t n, const int32_t *__restrict__ colptr,
                                 const int32_t *__restrict__ rowind_tmp,
                                 const int32_t *__restrict__ perm_tmp,
                                 int32_t *__restrict__ rowind, int32_t *__restrict__ perm)
{
    int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= n) return;
    int32_t a = colptr[w], L = colptr[w + 1] - a;
    for (int32_t e = lane; e < L; e += 32) {
        int32_t r = rowind_tmp[a + e];
        int32_t rank = 0;
        for (int32_t f = 0; f < L; ++f) rank += (rowind_tmp[a + f] < r);
        rowind[a + rank] = r;
        if (perm) perm[a + rank] = perm_tmp[a + e];
    }
}

// ---------------------------------------------------------------------------------
// column unions (row sets): a team of T lanes per output column (T = 4, 8 or 32: the
// narrowest that holds L_k at 4 lists per lane, so that short lists put several columns
// in one warp), team-wide minimum merge of the sorted row lists of the columns in L_k
// ---------------------------------------------------------------------------------
constexpr int kListsPerLane = 4;

template <int T>
__device__ __forceinline__ int32_t team_min(int32_t v)
{
    if constexpr (T == 32) {
        return __reduce_min_sync(0xffffffffu, v);
    } else {
#pragma unroll
        for (int o = T / 2; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));  // stays in the team
        return v;
    }
}

template <bool FILL, int T>
__global__ void k_colunion(int32_t n, const int32_t *__restrict__ Lptr,
                           const int32_t *__restrict__ Lind, const int32_t *__restrict__ colptr,
                           const int32_t *__restrict__ rowind, const int32_t *__restrict__ out_ptr,
                           int32_t *__restrict__ out, int *err)
{
    // every lane of the warp takes part in every step (full-mask shuffles); lanes past the
    // last column merge nothing
    const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / T;
    const int sub = threadIdx.x % T;
    if ((blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31)) / T >= n) return;  // the whole warp is past the end
    int32_t a = 0, L = 0;
    if (k < n) {
        a = Lptr[k];
        L = Lptr[k + 1] - a;
        if (L > T * kListsPerLane) {
            if (sub == 0 && err) atomicOr(err, ERR_TOO_WIDE);
            L = 0;
        }
    }
    int32_t pos[kListsPerLane], end[kListsPerLane], head[kListsPerLane];
#pragma unroll
    for (int u = 0; u < kListsPerLane; ++u) {
        const int32_t c = sub + T * u;
        pos[u] = end[u] = 0;
        head[u] = INT_MAX;
        if (c < L) {
            const int32_t j = Lind[a + c];
            pos[u] = colptr[j];
            end[u] = colptr[j + 1];
            if (pos[u] < end[u]) head[u] = rowind[pos[u]];
        }
    }
    const int64_t ob = (FILL && k < n) ? (int64_t)out_ptr[k] : 0;
    int32_t cnt = 0;
    while (true) {
        int32_t cand = head[0];
#pragma unroll
        for (int u = 1; u < kListsPerLane; ++u) cand = min(cand, head[u]);
        const int32_t m = team_min<T>(cand);
        if (!__any_sync(0xffffffffu, m != INT_MAX)) break;  // every team of the warp is done
        if (m == INT_MAX) continue;                           // this team is done, others are not
        if (FILL && sub == 0) out[ob + cnt] = m;
#pragma unroll
        for (int u = 0; u < kListsPerLane; ++u) {
            if (head[u] == m) {
                ++pos[u];
                head[u] = (pos[u] < end[u]) ? rowind[pos[u]] : INT_MAX;
            }
        }
        ++cnt;
    }
    if (!FILL && sub == 0 && k < n) out[k] = cnt;
}

__global__ void k_gather_f64(int64_t count, const int32_t *__restrict__ idx,
                             const double *__restrict__ src, double *__restrict__ dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}

__global__ void k_gather_f32_f64(int64_t count, const int32_t *__restrict__ idx, const float *__restrict__ src,
                                 double *__restrict__ dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[idx ? idx[i] : i];
}

__global__ void k_gather_bf16_f64(int64_t count, const int32_t *__restrict__ idx, const uint16_t *__restrict__ src,
                                  double *__restrict__ dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)__bfloat162float(__ushort_as_bfloat16(src[idx ? idx[i] : i]));
}

// ---------------------------------------------------------------------------------
// Batches of matrices stacked into one block-diagonal matrix: segment g of a list laid end
// to end covers elements start[g] <= e < start[g + 1] (empty segments allowed)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ int seg_of(const int64_t *__restrict__ start, int nseg, int64_t e)
{
    int lo = 0, hi = nseg - 1;  // the last g with start[g] <= e
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// rp[r] = rowptr_sys[r - off_sys] + nzoff_sys for the stacked rows (and rp[ntot] = nnz_tot),
// checking every system's row pointer (starts at 0, monotone, ends at its nnz)
__global__ void k_stack_rows(int32_t nsys, const int64_t *__restrict__ off, const int64_t *__restrict__ nzoff,
                             const int32_t *const *__restrict__ rowptr, int32_t *__restrict__ rp, int *err)
{
    const int64_t ntot = off[nsys];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= ntot;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (r == ntot) {
            rp[r] = (int32_t)nzoff[nsys];
            continue;
        }
        const int g = seg_of(off, nsys, r);
        const int64_t lr = r - off[g], ng = off[g + 1] - off[g], nz = nzoff[g + 1] - nzoff[g];
        const int32_t *p = rowptr[g];
        const int32_t a = p[lr], b = p[lr + 1];
        if ((lr == 0 && a != 0) || b < a || (lr == ng - 1 && b != nz)) atomicOr(err, ERR_ROWPTR);
        rp[r] = (int32_t)(a + nzoff[g]);
    }
}

// ci[q] = colind_sys[q - nzoff_sys] + off_sys, checking 0 <= colind < n_sys
__global__ void k_stack_cols(int32_t nsys, const int64_t *__restrict__ off, const int64_t *__restrict__ nzoff,
                             const int32_t *const *__restrict__ colind, int32_t *__restrict__ ci, int *err)
{
    const int64_t nnz = nzoff[nsys];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
        const int g = seg_of(nzoff, nsys, q);
        const int32_t c = colind[g][q - nzoff[g]];
        if (c < 0 || c >= off[g + 1] - off[g]) atomicOr(err, ERR_COLIND);
        ci[q] = (int32_t)(c + off[g]);
    }
}

// lists L_k of the column unions: {k} for a system of kind 0 (pattern of A), the rows of
// column k for kind 1 (pattern of A^2); counts, then the lists
__global__ void k_list_counts(int32_t nsys, const int64_t *__restrict__ off, const int32_t *__restrict__ kind,
                              const int32_t *__restrict__ colptr, int32_t *__restrict__ counts)
{
    const int64_t ntot = off[nsys];
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ntot; k += (int64_t)gridDim.x * blockDim.x)
        counts[k] = kind[seg_of(off, nsys, k)] ? colptr[k + 1] - colptr[k] : 1;
}

__global__ void k_list_fill(int32_t nsys, const int64_t *__restrict__ off, const int32_t *__restrict__ kind,
                            const int32_t *__restrict__ colptr, const int32_t *__restrict__ rowind,
                            const int32_t *__restrict__ Lptr, int32_t *__restrict__ Lind)
{
    const int64_t ntot = off[nsys];
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ntot; k += (int64_t)gridDim.x * blockDim.x) {
        if (!kind[seg_of(off, nsys, k)]) {
            Lind[Lptr[k]] = (int32_t)k;
        } else {
            for (int32_t q = colptr[k]; q < colptr[k + 1]; ++q) Lind[Lptr[k] + (q - colptr[k])] = rowind[q];
        }
    }
}

// per system: tot[g] = ptr[off[g+1]] - ptr[off[g]], mx[g] = max over its columns of
// ptr[k+1] - ptr[k] (mx zeroed first)
__global__ void k_seg_ptr_stats(int32_t nsys, const int64_t *__restrict__ off, const int32_t *__restrict__ ptr,
                                int64_t *__restrict__ tot, int32_t *__restrict__ mx)
{
    const int64_t ntot = off[nsys];
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ntot; k += (int64_t)gridDim.x * blockDim.x) {
        const int g = seg_of(off, nsys, k);
        atomicMax(mx + g, ptr[k + 1] - ptr[k]);
        if (k == off[g]) tot[g] = (int64_t)ptr[off[g + 1]] - ptr[k];
    }
}

// Segmented element-wise passes walk a tile of kSegTile consecutive elements per block: the
// segment of the tile's first element is found once (binary search), and each thread,
// whose elements increase, steps its segment forward from there -- coalesced accesses and
// no search per element.
constexpr int kSegTile = 16 * 256;

// dst_g[j] = src_g[j] - sub_g over segments laid end to end
__global__ void k_unstack(int32_t nseg, const int64_t *__restrict__ start, const int32_t *const *__restrict__ src,
                          int32_t *const *__restrict__ dst, const int32_t *__restrict__ sub)
{
    const int64_t total = start[nseg];
    for (int64_t t0 = (int64_t)blockIdx.x * kSegTile; t0 < total; t0 += (int64_t)gridDim.x * kSegTile) {
        int g = seg_of(start, nseg, t0);
        const int64_t t1 = min(t0 + (int64_t)kSegTile, total);
        for (int64_t e = t0 + threadIdx.x; e < t1; e += blockDim.x) {
            while (e >= __ldg(start + g + 1)) ++g;
            const int64_t j = e - start[g];
            dst[g][j] = src[g][j] - sub[g];
        }
    }
}

// dst_g[j] = val_g[perm_g[j]] over segments laid end to end
__global__ void k_gather_seg(int32_t nseg, const int64_t *__restrict__ start, const double *const *__restrict__ val,
                             const int32_t *const *__restrict__ perm, double *const *__restrict__ dst)
{
    const int64_t total = start[nseg];
    for (int64_t t0 = (int64_t)blockIdx.x * kSegTile; t0 < total; t0 += (int64_t)gridDim.x * kSegTile) {
        int g = seg_of(start, nseg, t0);
        const int64_t t1 = min(t0 + (int64_t)kSegTile, total);
        for (int64_t e = t0 + threadIdx.x; e < t1; e += blockDim.x) {
            while (e >= __ldg(start + g + 1)) ++g;
            const int64_t j = e - start[g];
            dst[g][j] = val[g][perm[g][j]];
        }
    }
}

// dst[start[g] + j] = (float)src_g[j]: segments rounded to FP32 into one stacked array
__global__ void k_round_seg(int32_t nseg, const int64_t *__restrict__ start, const double *const *__restrict__ src,
                            float *__restrict__ dst)
{
    const int64_t total = start[nseg];
    for (int64_t t0 = (int64_t)blockIdx.x * kSegTile; t0 < total; t0 += (int64_t)gridDim.x * kSegTile) {
        int g = seg_of(start, nseg, t0);
        const int64_t t1 = min(t0 + (int64_t)kSegTile, total);
        for (int64_t e = t0 + threadIdx.x; e < t1; e += blockDim.x) {
            while (e >= __ldg(start + g + 1)) ++g;
            dst[e] = (float)src[g][e - start[g]];
        }
    }
}

// out[g] = smallest j with a_g[j] != 0 (INT_MAX if none; out filled with INT_MAX first)
__global__ void k_first_nonzero_seg(int32_t nseg, const int64_t *__restrict__ start, const int32_t *const *__restrict__ a,
                                    int32_t *__restrict__ out)
{
    const int64_t total = start[nseg];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int g = seg_of(start, nseg, e);
        const int64_t j = e - start[g];
        if (a[g][j] != 0) atomicMin(out + g, (int32_t)j);
    }
}

__global__ void k_add_i32(int64_t count, const int32_t *__restrict__ src, int32_t add, int32_t *__restrict__ dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] + add;
}

__global__ void k_iota_i32(int64_t count, int32_t *__restrict__ dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (int32_t)i;
}

__global__ void k_invert_perm(int64_t count, const int32_t *__restrict__ perm,
                              int32_t *__restrict__ inv)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        inv[perm[i]] = (int32_t)i;
}

__global__ void k_max_diff(int32_t n, const int32_t *__restrict__ ptr, int32_t *out)
{
    int32_t m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, ptr[i + 1] - ptr[i]);
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void k_first_nonzero(int32_t n, const int32_t *__restrict__ a, int32_t *out)
{
    int32_t best = INT_MAX;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (a[i] != 0) { best = (int32_t)i; break; }
    best = __reduce_min_sync(0xffffffffu, best);
    if ((threadIdx.x & 31) == 0 && best != INT_MAX) atomicMin(out, best);
}

__global__ void k_compare_i32(int64_t count, const int32_t *__restrict__ a,
                              const int32_t *__restrict__ b, int *err)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        if (a[i] != b[i]) { atomicOr(err, ERR_PATTERN); return; }
}

__global__ void k_fill_i32(int64_t count, int32_t v, int32_t *dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = v;
}

// ---------------------------------------------------------------------------------
// CSR times row-major block: S consecutive lanes per row, lane c owns column c
// ---------------------------------------------------------------------------------
// a stored factor value as FP64 (FP64, FP32 or BF16 bits): conversions are exact
__device__ __forceinline__ double as_f64(double v) { return v; }
__device__ __forceinline__ double as_f64(float v) { return (double)v; }
__device__ __forceinline__ double as_f64(uint16_t b) { return (double)__bfloat162float(__ushort_as_bfloat16(b)); }

template <int S, typename V>
__global__ void __launch_bounds__(kThreads) k_spmm(int32_t n, const int32_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ colind,
                                                   const V *__restrict__ val,
                                                   const double *__restrict__ X,
                                                   double *__restrict__ Y)
{
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t row = g / S;
    int c = (int)(g % S);
    if (row >= n) return;
    int32_t a = __ldg(rowptr + row), b = __ldg(rowptr + row + 1);
    double acc = 0.0;
    for (int32_t q = a; q < b; ++q)
        acc = fma(as_f64(__ldg(val + q)), __ldg(X + (int64_t)__ldg(colind + q) * S + c), acc);
    Y[row * S + c] = acc;
}

// The same product restricted to a list of row chunks: chunk c (grid column blockIdx.x)
// covers rows [r0[c], r1[c]), at most kThreads / S * gridDim.y of them.  Rows outside the
// listed chunks are neither read as outputs nor written.
template <int S, typename V>
__global__ void __launch_bounds__(kThreads) k_spmm_seg(const int64_t *__restrict__ r0s,
                                                       const int64_t *__restrict__ r1s,
                                                       const int32_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ colind,
                                                       const V *__restrict__ val,
                                                       const double *__restrict__ X, double *__restrict__ Y)
{
    const int64_t g = blockIdx.y * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = __ldg(r0s + blockIdx.x) + g / S;
    const int c = (int)(g % S);
    if (row >= __ldg(r1s + blockIdx.x)) return;
    const int32_t a = __ldg(rowptr + row), b = __ldg(rowptr + row + 1);
    double acc = 0.0;
    for (int32_t q = a; q < b; ++q)
        acc = fma(as_f64(__ldg(val + q)), __ldg(X + (int64_t)__ldg(colind + q) * S + c), acc);
    Y[row * S + c] = acc;
}

template <int S, typename V>
__global__ void k_scale_rows_seg(const int64_t *__restrict__ r0s, const int64_t *__restrict__ r1s,
                                 const V *__restrict__ q, const double *__restrict__ X, double *__restrict__ Y)
{
    const int64_t g = blockIdx.y * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = __ldg(r0s + blockIdx.x) + g / S;
    if (row >= __ldg(r1s + blockIdx.x)) return;
    const int64_t e = row * S + g % S;
    Y[e] = as_f64(__ldg(q + row)) * X[e];
}

// ---------------------------------------------------------------------------------
// FP32 CSR times row-major block: the operator of the mixed-precision solve.  The matrix
// values (FP32, BF16 bits, or FP64 rounded once) and the X entries (FP64 rounded once, or
// FP32) are multiplied and summed in FP32 in the row's order; Y is written as FP32 or as
// FP64 (exact conversion).  T = S / C lanes per row, each owning C = min(S, 4) consecutive
// columns (vector loads of X and Y); the nonzeros are taken eight at a time, their index,
// value and X loads issued together before the multiply-adds.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float as_f32(float v) { return v; }
__device__ __forceinline__ float as_f32(double v) { return f64_to_f32(v); }
__device__ __forceinline__ float as_f32(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

template <int C>
__device__ __forceinline__ void load_x(const float *p, float (&x)[C])
{
    if constexpr (C == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else if constexpr (C == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        x[0] = v.x; x[1] = v.y;
    } else {
        x[0] = __ldg(p);
    }
}

template <int C>
__device__ __forceinline__ void load_x(const double *p, float (&x)[C])
{
    if constexpr (C >= 2) {
#pragma unroll
        for (int h = 0; h < C / 2; ++h) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(p) + h);
            x[2 * h] = f64_to_f32(v.x);
            x[2 * h + 1] = f64_to_f32(v.y);
        }
    } else {
        x[0] = f64_to_f32(__ldg(p));
    }
}

template <int C>
__device__ __forceinline__ void store_y(float *p, const float (&y)[C])
{
    if constexpr (C == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(y[0], y[1], y[2], y[3]);
    } else if constexpr (C == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(y[0], y[1]);
    } else {
        p[0] = y[0];
    }
}

template <int C>
__device__ __forceinline__ void store_y(double *p, const float (&y)[C])
{
    if constexpr (C >= 2) {
#pragma unroll
        for (int h = 0; h < C / 2; ++h)
            reinterpret_cast<double2 *>(p)[h] = make_double2(f32_to_f64(y[2 * h]), f32_to_f64(y[2 * h + 1]));
    } else {
        p[0] = f32_to_f64(y[0]);
    }
}

template <int S, typename V, typename XT, typename YT>
__global__ void __launch_bounds__(kThreads) k_spmm32(int32_t n, const int32_t *__restrict__ rowptr,
                                                     const int32_t *__restrict__ colind, const V *__restrict__ val,
                                                     const XT *__restrict__ X, YT *__restrict__ Y)
{
    constexpr int C = S < 4 ? S : 4, T = S / C, U = 8;
    const int64_t lanes = (int64_t)n * T;
    // one wave of blocks walks all (row, part) lanes; a lane's nonzeros go eight at a time,
    // every index, value and X load of the eight issued before the multiply-adds (a row of
    // a 7- or 27-point stencil takes one or four such rounds); the sums stay in row order
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < lanes; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = g / T;
        const int part = (int)(g % T);
        const int32_t a = __ldg(rowptr + row), b = __ldg(rowptr + row + 1);
        const XT *xb = X + part * C;
        float acc[C];
#pragma unroll
        for (int k = 0; k < C; ++k) acc[k] = 0.0f;
        for (int32_t q = a; q < b; q += U) {
            int32_t c[U];
            float v[U], x[U][C];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool in = q + u < b;
                c[u] = in ? __ldg(colind + q + u) : -1;
                v[u] = in ? as_f32(__ldg(val + q + u)) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (c[u] >= 0) load_x<C>(xb + (int64_t)c[u] * S, x[u]);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (c[u] >= 0)
#pragma unroll
                    for (int k = 0; k < C; ++k) acc[k] = fmaf(v[u], x[u][k], acc[k]);
        }
        store_y<C>(Y + row * S + part * C, acc);
    }
}

// Y[r][c] = q[r] X[r][c] in FP32 (a diagonal factor of the FP32 operator)
template <int S, typename V, typename XT, typename YT>
__global__ void k_scale_rows32(int32_t n, const V *__restrict__ q, const XT *__restrict__ X, YT *__restrict__ Y)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)n * S) return;
    const float y = as_f32(__ldg(q + g / S)) * as_f32(X[g]);
    if constexpr (sizeof(YT) == 8) Y[g] = f32_to_f64(y);
    else Y[g] = y;
}

__global__ void k_round_f32(int64_t count, const double *__restrict__ src, float *__restrict__ dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = f64_to_f32(src[i]);
}

template <int S, typename V>
__global__ void k_scale_rows(int32_t n, const V *__restrict__ q, const double *__restrict__ X,
                             double *__restrict__ Y)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)n * S) return;
    Y[g] = as_f64(__ldg(q + g / S)) * X[g];
}

template <int S>
__global__ void k_pack(int32_t n, const double *__restrict__ src, int64_t ld,
                       double *__restrict__ dst)
{
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)n * S) return;
    int64_t r = g % n;
    int c = (int)(g / n);
    dst[r * S + c] = src[(int64_t)c * ld + r];
}

template <int S>
__global__ void k_unpack(int32_t n, const double *__restrict__ src, double *__restrict__ dst,
                         int64_t ld)
{
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)n * S) return;
    int64_t r = g % n;
    int c = (int)(g / n);
    dst[(int64_t)c * ld + r] = src[r * S + c];
}

}  // namespace

// ===================================================================================
// launchers
// ===================================================================================
int launch_validate_csr(cudaStream_t st, int32_t n, int32_t nnz, const int32_t *rowptr,
                        const int32_t *colind, int *d_err)
{
    k_validate_csr<<<grid_for((int64_t)n + 1), kThreads, 0, st>>>(n, nnz, rowptr, colind, d_err);
    return check_launch();
}

int launch_union_count(cudaStream_t st, int32_t n, int32_t T, const TermPtrs &tp, int32_t *counts)
{
    k_union<false><<<grid_for(n), kThreads, 0, st>>>(n, T, tp, counts, nullptr, nullptr, nullptr, 0);
    return check_launch();
}

int launch_union_fill(cudaStream_t st, int32_t n, int32_t T, const TermPtrs &tp,
                      const int32_t *u_rowptr, int32_t *u_colind, double *aligned, int64_t nnzU)
{
    k_union<true><<<grid_for(n), kThreads, 0, st>>>(n, T, tp, nullptr, u_rowptr, u_colind,
                                                     aligned, nnzU);
    return check_launch();
}

int launch_assemble(cudaStream_t st, int64_t nnz, int32_t T, const double *aligned,
                    const double *coef_host, double *out)
{
    TermPtrs tp{};
    for (int t = 0; t < T; ++t) tp.coef[t] = coef_host[t];
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (nnz + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)sms * 8;
    int grid = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    k_assemble<<<grid, kThreads, 0, st>>>(nnz, T, aligned, tp, out);
    return check_launch();
}

size_t scan_temp_bytes(int64_t n)
{
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    return (size_t)(tiles + 1) * sizeof(long long);
}

int launch_exclusive_scan(cudaStream_t st, const int32_t *counts, int32_t *ptr, int64_t n,
                          void *temp, int *d_err)
{
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles < 1) tiles = 1;
    long long *sums = (long long *)temp;
    k_scan_tile_sums<<<(unsigned)tiles, kThreads, 0, st>>>(counts, n, sums);
    k_scan_sums<<<1, kThreads, 0, st>>>(sums, tiles, ptr, n, d_err);
    k_scan_apply<<<(unsigned)tiles, kThreads, 0, st>>>(counts, n, sums, ptr);
    return check_launch(3);
}

static size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// must match the carving in launch_transpose: every piece is rounded up to 256 bytes
size_t transpose_temp_bytes(int32_t n, int32_t nnz)
{
    return 2 * round256(((size_t)n + 1) * sizeof(int32_t)) +
           2 * round256(((size_t)nnz + 1) * sizeof(int32_t)) + round256(scan_temp_bytes(n));
}

int launch_transpose(cudaStream_t st, int32_t n, int32_t nnz, const int32_t *rowptr,
                     const int32_t *colind, int32_t *colptr, int32_t *rowind, int32_t *perm,
                     void *temp, int *d_err)
{
    char *p = (char *)temp;
    auto take = [&](size_t bytes) {
        void *r = p;
        p += (bytes + 255) / 256 * 256;
        return r;
    };
    int32_t *cnt = (int32_t *)take(((size_t)n + 1) * sizeof(int32_t));
    int32_t *next = (int32_t *)take(((size_t)n + 1) * sizeof(int32_t));
    int32_t *rtmp = (int32_t *)take(((size_t)nnz + 1) * sizeof(int32_t));
    int32_t *ptmp = (int32_t *)take(((size_t)nnz + 1) * sizeof(int32_t));
    void *stemp = take(scan_temp_bytes(n));
    if (cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int32_t), st) != cudaSuccess) return -1;
    k_count_cols<<<grid_for(nnz), kThreads, 0, st>>>(nnz, colind, cnt);
    if (launch_exclusive_scan(st, cnt, colptr, n, stemp, d_err)) return -1;
    if (cudaMemcpyAsync(next, colptr, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
        return -1;
    k_fill_cols<<<grid_for(n), kThreads, 0, st>>>(n, rowptr, colind, next, rtmp, ptmp);
    k_rank_sort_cols<<<grid_for((int64_t)n * 32), kThreads, 0, st>>>(n, colptr, rtmp, ptmp, rowind,
                                                                      perm);
    return check_launch(3);
}

int colunion_max_lists() { return 32 * kListsPerLane; }

namespace {
template <bool FILL>
int colunion_launch(cudaStream_t st, int32_t n, int32_t maxL, const int32_t *Lptr, const int32_t *Lind,
                    const int32_t *colptr, const int32_t *rowind, const int32_t *out_ptr, int32_t *out, int *d_err)
{
    if (n <= 0) return 0;
    if (maxL <= 4 * kListsPerLane)
        k_colunion<FILL, 4><<<grid_for((int64_t)n * 4), kThreads, 0, st>>>(n, Lptr, Lind, colptr, rowind, out_ptr,
                                                                             out, d_err);
    else if (maxL <= 8 * kListsPerLane)
        k_colunion<FILL, 8><<<grid_for((int64_t)n * 8), kThreads, 0, st>>>(n, Lptr, Lind, colptr, rowind, out_ptr,
                                                                             out, d_err);
    else
        k_colunion<FILL, 32><<<grid_for((int64_t)n * 32), kThreads, 0, st>>>(n, Lptr, Lind, colptr, rowind, out_ptr,
                                                                               out, d_err);
    return check_launch();
}
}  // namespace

int launch_colunion_count(cudaStream_t st, int32_t n, int32_t maxL, const int32_t *Lptr, const int32_t *Lind,
                          const int32_t *colptr, const int32_t *rowind, int32_t *counts, int *d_err)
{
    return colunion_launch<false>(st, n, maxL, Lptr, Lind, colptr, rowind, nullptr, counts, d_err);
}

int launch_colunion_fill(cudaStream_t st, int32_t n, int32_t maxL, const int32_t *Lptr, const int32_t *Lind,
                         const int32_t *colptr, const int32_t *rowind, const int32_t *out_ptr,
                         int32_t *out_list, int *d_err)
{
    return colunion_launch<true>(st, n, maxL, Lptr, Lind, colptr, rowind, out_ptr, out_list, d_err);
}

int launch_gather_f64(cudaStream_t st, int64_t count, const int32_t *idx, const double *src,
                      double *dst)
{
    if (count <= 0) return 0;
    k_gather_f64<<<grid_for(count), kThreads, 0, st>>>(count, idx, src, dst);
    return check_launch();
}

int launch_gather_f32_f64(cudaStream_t st, int64_t count, const int32_t *idx, const float *src, double *dst)
{
    if (count <= 0) return 0;
    k_gather_f32_f64<<<grid_for(count), kThreads, 0, st>>>(count, idx, src, dst);
    return check_launch();
}

namespace {
inline int grid_cap(int64_t work) { int g = grid_for(work); return g > 8 * 1216 ? 8 * 1216 : g; }
}  // namespace

int launch_stack_csr(cudaStream_t st, int32_t nsys, int64_t ntot, int64_t nnz, const int64_t *off, const int64_t *nzoff,
                     const int32_t *const *rowptr, const int32_t *const *colind, int32_t *rp, int32_t *ci, int *d_err)
{
    k_stack_rows<<<grid_cap(ntot + 1), kThreads, 0, st>>>(nsys, off, nzoff, rowptr, rp, d_err);
    if (nnz > 0) k_stack_cols<<<grid_cap(nnz), kThreads, 0, st>>>(nsys, off, nzoff, colind, ci, d_err);
    return check_launch(2);
}

int launch_union_lists(cudaStream_t st, int32_t nsys, int64_t ntot, const int64_t *off, const int32_t *kind,
                       const int32_t *colptr, const int32_t *rowind, int32_t *counts, const int32_t *Lptr, int32_t *Lind)
{
    if (!Lptr) k_list_counts<<<grid_cap(ntot), kThreads, 0, st>>>(nsys, off, kind, colptr, counts);
    else k_list_fill<<<grid_cap(ntot), kThreads, 0, st>>>(nsys, off, kind, colptr, rowind, Lptr, Lind);
    return check_launch();
}

int launch_seg_ptr_stats(cudaStream_t st, int32_t nsys, int64_t ntot, const int64_t *off, const int32_t *ptr,
                         int64_t *tot, int32_t *mx)
{
    if (cudaMemsetAsync(mx, 0, (size_t)nsys * sizeof(int32_t), st) != cudaSuccess) return -1;
    k_seg_ptr_stats<<<grid_cap(ntot), kThreads, 0, st>>>(nsys, off, ptr, tot, mx);
    return check_launch();
}

int launch_unstack(cudaStream_t st, int32_t nseg, int64_t total, const int64_t *start, const int32_t *const *src,
                   int32_t *const *dst, const int32_t *sub)
{
    if (total <= 0) return 0;
    k_unstack<<<grid_cap((total + kSegTile - 1) / kSegTile * kThreads), kThreads, 0, st>>>(nseg, start, src, dst, sub);
    return check_launch();
}

int launch_gather_seg(cudaStream_t st, int32_t nseg, int64_t total, const int64_t *start, const double *const *val,
                      const int32_t *const *perm, double *const *dst)
{
    if (total <= 0) return 0;
    k_gather_seg<<<grid_cap((total + kSegTile - 1) / kSegTile * kThreads), kThreads, 0, st>>>(nseg, start, val, perm,
                                                                                               dst);
    return check_launch();
}

int launch_round_seg(cudaStream_t st, int32_t nseg, int64_t total, const int64_t *start, const double *const *src,
                     float *dst)
{
    if (total <= 0) return 0;
    k_round_seg<<<grid_cap((total + kSegTile - 1) / kSegTile * kThreads), kThreads, 0, st>>>(nseg, start, src, dst);
    return check_launch();
}

int launch_first_nonzero_seg(cudaStream_t st, int32_t nseg, int64_t total, const int64_t *start,
                             const int32_t *const *a, int32_t *out)
{
    k_fill_i32<<<grid_for(nseg), kThreads, 0, st>>>(nseg, INT_MAX, out);
    if (total > 0) k_first_nonzero_seg<<<grid_cap(total), kThreads, 0, st>>>(nseg, start, a, out);
    return check_launch(2);
}

int launch_add_i32(cudaStream_t st, int64_t count, const int32_t *src, int32_t add, int32_t *dst)
{
    if (count <= 0) return 0;
    int g = grid_for(count);
    if (g > 8192) g = 8192;
    k_add_i32<<<g, kThreads, 0, st>>>(count, src, add, dst);
    return check_launch();
}

int launch_iota_i32(cudaStream_t st, int64_t count, int32_t *dst)
{
    if (count <= 0) return 0;
    k_iota_i32<<<grid_for(count), kThreads, 0, st>>>(count, dst);
    return check_launch();
}

int launch_gather_bf16_f64(cudaStream_t st, int64_t count, const int32_t *idx, const uint16_t *src, double *dst)
{
    if (count <= 0) return 0;
    k_gather_bf16_f64<<<grid_for(count), kThreads, 0, st>>>(count, idx, src, dst);
    return check_launch();
}

int launch_invert_perm(cudaStream_t st, int64_t count, const int32_t *perm, int32_t *inv)
{
    if (count <= 0) return 0;
    k_invert_perm<<<grid_for(count), kThreads, 0, st>>>(count, perm, inv);
    return check_launch();
}

int launch_max_i32_diff(cudaStream_t st, int32_t n, const int32_t *ptr, int32_t *d_max)
{
    if (cudaMemsetAsync(d_max, 0, sizeof(int32_t), st) != cudaSuccess) return -1;
    if (n <= 0) return 0;
    int g = grid_for(n);
    if (g > 4096) g = 4096;
    k_max_diff<<<g, kThreads, 0, st>>>(n, ptr, d_max);
    return check_launch();
}

int launch_fill_i32(cudaStream_t st, int64_t count, int32_t v, int32_t *dst)
{
    if (count <= 0) return 0;
    k_fill_i32<<<grid_for(count), kThreads, 0, st>>>(count, v, dst);
    return check_launch();
}

int launch_first_nonzero(cudaStream_t st, int32_t n, const int32_t *a, int32_t *d_out)
{
    k_fill_i32<<<1, 32, 0, st>>>(1, INT_MAX, d_out);
    if (n <= 0) return check_launch();
    int g = grid_for(n);
    if (g > 4096) g = 4096;
    k_first_nonzero<<<g, kThreads, 0, st>>>(n, a, d_out);
    return check_launch(2);
}

int launch_compare_i32(cudaStream_t st, int64_t count, const int32_t *a, const int32_t *b, int *d_err)
{
    if (count <= 0) return 0;
    int g = grid_for(count);
    if (g > 8192) g = 8192;
    k_compare_i32<<<g, kThreads, 0, st>>>(count, a, b, d_err);
    return check_launch();
}

namespace {

template <typename V>
int spmm_any(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind, const V *val,
             const double *X, double *Y)
{
    if (n <= 0) return 0;
    int g = grid_for((int64_t)n * s);
    switch (s) {
    case 1: k_spmm<1, V><<<g, kThreads, 0, st>>>(n, rowptr, colind, val, X, Y); break;
    case 2: k_spmm<2, V><<<g, kThreads, 0, st>>>(n, rowptr, colind, val, X, Y); break;
    case 4: k_spmm<4, V><<<g, kThreads, 0, st>>>(n, rowptr, colind, val, X, Y); break;
    case 8: k_spmm<8, V><<<g, kThreads, 0, st>>>(n, rowptr, colind, val, X, Y); break;
    case 16: k_spmm<16, V><<<g, kThreads, 0, st>>>(n, rowptr, colind, val, X, Y); break;
    default: return -1;
    }
    return check_launch();
}

}  // namespace

int launch_spmm(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr,
                const int32_t *colind, const double *val, const double *X, double *Y)
{
    return spmm_any<double>(st, s, n, rowptr, colind, val, X, Y);
}

int launch_spmm_f32v(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind,
                     const float *val, const double *X, double *Y)
{
    return spmm_any<float>(st, s, n, rowptr, colind, val, X, Y);
}

int launch_spmm_bf16v(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind,
                      const uint16_t *val, const double *X, double *Y)
{
    return spmm_any<uint16_t>(st, s, n, rowptr, colind, val, X, Y);
}

namespace {

template <typename V, typename XT, typename YT>
int spmm32_any(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind, const V *val,
               const XT *X, YT *Y)
{
    if (n <= 0) return 0;
    const int T = s < 4 ? 1 : s / 4;
    // one wave: every SM's resident blocks, fewer for small n
    int dev = 0, sms = 152, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    cudaError_t oe = cudaErrorInvalidValue;
    switch (s) {
    case 1: oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm32<1, V, XT, YT>, kThreads, 0); break;
    case 2: oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm32<2, V, XT, YT>, kThreads, 0); break;
    case 4: oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm32<4, V, XT, YT>, kThreads, 0); break;
    case 8: oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm32<8, V, XT, YT>, kThreads, 0); break;
    case 16: oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm32<16, V, XT, YT>, kThreads, 0); break;
    default: return -1;
    }
    if (oe != cudaSuccess) return -1;
    const int64_t want = ((int64_t)n * T + kThreads - 1) / kThreads, wave = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int g = (int)(want < wave ? want : wave);
    switch (s) {
    case 1: k_spmm32<1, V, XT, YT><<<g, kThreads, 0, st>>>(n, rowptr, colind, val, X, Y); break;
    case 2: k_spmm32<2, V, XT, YT><<<g, kThreads, 0, st>>>(n, rowptr, colind, val, X, Y); break;
    case 4: k_spmm32<4, V, XT, YT><<<g, kThreads, 0, st>>>(n, rowptr, colind, val, X, Y); break;
    case 8: k_spmm32<8, V, XT, YT><<<g, kThreads, 0, st>>>(n, rowptr, colind, val, X, Y); break;
    case 16: k_spmm32<16, V, XT, YT><<<g, kThreads, 0, st>>>(n, rowptr, colind, val, X, Y); break;
    default: return -1;
    }
    return check_launch();
}

template <typename V, typename XT, typename YT>
int scale_rows32_any(cudaStream_t st, int32_t s, int32_t n, const V *q, const XT *X, YT *Y)
{
    if (n <= 0) return 0;
    const int g = grid_for((int64_t)n * s);
    switch (s) {
    case 1: k_scale_rows32<1, V, XT, YT><<<g, kThreads, 0, st>>>(n, q, X, Y); break;
    case 2: k_scale_rows32<2, V, XT, YT><<<g, kThreads, 0, st>>>(n, q, X, Y); break;
    case 4: k_scale_rows32<4, V, XT, YT><<<g, kThreads, 0, st>>>(n, q, X, Y); break;
    case 8: k_scale_rows32<8, V, XT, YT><<<g, kThreads, 0, st>>>(n, q, X, Y); break;
    case 16: k_scale_rows32<16, V, XT, YT><<<g, kThreads, 0, st>>>(n, q, X, Y); break;
    default: return -1;
    }
    return check_launch();
}

template <typename XT, typename YT>
int spmm32_vals(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind, const F32Vals &v,
                const XT *X, YT *Y)
{
    if (v.f32) return spmm32_any<float, XT, YT>(st, s, n, rowptr, colind, v.f32, X, Y);
    if (v.bf16) return spmm32_any<uint16_t, XT, YT>(st, s, n, rowptr, colind, v.bf16, X, Y);
    if (v.f64) return spmm32_any<double, XT, YT>(st, s, n, rowptr, colind, v.f64, X, Y);
    return -1;
}

template <typename XT, typename YT>
int scale32_vals(cudaStream_t st, int32_t s, int32_t n, const F32Vals &v, const XT *X, YT *Y)
{
    if (v.f32) return scale_rows32_any<float, XT, YT>(st, s, n, v.f32, X, Y);
    if (v.bf16) return scale_rows32_any<uint16_t, XT, YT>(st, s, n, v.bf16, X, Y);
    if (v.f64) return scale_rows32_any<double, XT, YT>(st, s, n, v.f64, X, Y);
    return -1;
}

}  // namespace

int launch_spmm32(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind,
                  const F32Vals &v, const double *X, float *Y)
{
    return spmm32_vals(st, s, n, rowptr, colind, v, X, Y);
}
int launch_spmm32(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind,
                  const F32Vals &v, const float *X, float *Y)
{
    return spmm32_vals(st, s, n, rowptr, colind, v, X, Y);
}
int launch_spmm32(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind,
                  const F32Vals &v, const double *X, double *Y)
{
    return spmm32_vals(st, s, n, rowptr, colind, v, X, Y);
}
int launch_spmm32(cudaStream_t st, int32_t s, int32_t n, const int32_t *rowptr, const int32_t *colind,
                  const F32Vals &v, const float *X, double *Y)
{
    return spmm32_vals(st, s, n, rowptr, colind, v, X, Y);
}
int launch_scale_rows32(cudaStream_t st, int32_t s, int32_t n, const F32Vals &q, const double *X, float *Y)
{
    return scale32_vals(st, s, n, q, X, Y);
}
int launch_scale_rows32(cudaStream_t st, int32_t s, int32_t n, const F32Vals &q, const float *X, float *Y)
{
    return scale32_vals(st, s, n, q, X, Y);
}
int launch_scale_rows32(cudaStream_t st, int32_t s, int32_t n, const F32Vals &q, const double *X, double *Y)
{
    return scale32_vals(st, s, n, q, X, Y);
}
int launch_scale_rows32(cudaStream_t st, int32_t s, int32_t n, const F32Vals &q, const float *X, double *Y)
{
    return scale32_vals(st, s, n, q, X, Y);
}

int launch_round_f32(cudaStream_t st, int64_t count, const double *src, float *dst)
{
    if (count <= 0) return 0;
    int g = grid_for(count);
    if (g > 8 * 152) g = 8 * 152;
    k_round_f32<<<g, kThreads, 0, st>>>(count, src, dst);
    return check_launch();
}

namespace {
template <typename V>
int scale_rows_any(cudaStream_t st, int32_t s, int32_t n, const V *q, const double *X, double *Y)
{
    if (n <= 0) return 0;
    const int g = grid_for((int64_t)n * s);
    switch (s) {
    case 1: k_scale_rows<1, V><<<g, kThreads, 0, st>>>(n, q, X, Y); break;
    case 2: k_scale_rows<2, V><<<g, kThreads, 0, st>>>(n, q, X, Y); break;
    case 4: k_scale_rows<4, V><<<g, kThreads, 0, st>>>(n, q, X, Y); break;
    case 8: k_scale_rows<8, V><<<g, kThreads, 0, st>>>(n, q, X, Y); break;
    case 16: k_scale_rows<16, V><<<g, kThreads, 0, st>>>(n, q, X, Y); break;
    default: return -1;
    }
    return check_launch();
}
}  // namespace

int launch_scale_rows(cudaStream_t st, int32_t s, int32_t n, const double *q, const float *q32, const uint16_t *q16,
                      const double *X, double *Y)
{
    if (q16) return scale_rows_any<uint16_t>(st, s, n, q16, X, Y);
    if (q32) return scale_rows_any<float>(st, s, n, q32, X, Y);
    return scale_rows_any<double>(st, s, n, q, X, Y);
}

namespace {

template <typename V>
int spmm_seg_any(cudaStream_t st, int32_t s, int32_t nchunks, int64_t max_rows, const int64_t *r0, const int64_t *r1,
                 const int32_t *rowptr, const int32_t *colind, const V *val, const double *X, double *Y)
{
    if (nchunks <= 0) return 0;
    const int64_t sub = (max_rows * s + kThreads - 1) / kThreads;
    if (sub < 1 || sub > 65535) return -1;
    const dim3 grid((unsigned)nchunks, (unsigned)sub);
    switch (s) {
    case 1: k_spmm_seg<1, V><<<grid, kThreads, 0, st>>>(r0, r1, rowptr, colind, val, X, Y); break;
    case 2: k_spmm_seg<2, V><<<grid, kThreads, 0, st>>>(r0, r1, rowptr, colind, val, X, Y); break;
    case 4: k_spmm_seg<4, V><<<grid, kThreads, 0, st>>>(r0, r1, rowptr, colind, val, X, Y); break;
    case 8: k_spmm_seg<8, V><<<grid, kThreads, 0, st>>>(r0, r1, rowptr, colind, val, X, Y); break;
    case 16: k_spmm_seg<16, V><<<grid, kThreads, 0, st>>>(r0, r1, rowptr, colind, val, X, Y); break;
    default: return -1;
    }
    return check_launch();
}

template <typename V>
int scale_rows_seg_any(cudaStream_t st, int32_t s, int32_t nchunks, int64_t max_rows, const int64_t *r0,
                       const int64_t *r1, const V *q, const double *X, double *Y)
{
    if (nchunks <= 0) return 0;
    const int64_t sub = (max_rows * s + kThreads - 1) / kThreads;
    if (sub < 1 || sub > 65535) return -1;
    const dim3 grid((unsigned)nchunks, (unsigned)sub);
    switch (s) {
    case 1: k_scale_rows_seg<1, V><<<grid, kThreads, 0, st>>>(r0, r1, q, X, Y); break;
    case 2: k_scale_rows_seg<2, V><<<grid, kThreads, 0, st>>>(r0, r1, q, X, Y); break;
    case 4: k_scale_rows_seg<4, V><<<grid, kThreads, 0, st>>>(r0, r1, q, X, Y); break;
    case 8: k_scale_rows_seg<8, V><<<grid, kThreads, 0, st>>>(r0, r1, q, X, Y); break;
    case 16: k_scale_rows_seg<16, V><<<grid, kThreads, 0, st>>>(r0, r1, q, X, Y); break;
    default: return -1;
    }
    return check_launch();
}

}  // namespace

int launch_spmm_seg(cudaStream_t st, int32_t s, int32_t nchunks, int64_t max_rows, const int64_t *r0,
                    const int64_t *r1, const int32_t *rowptr, const int32_t *colind, const double *val,
                    const float *val32, const uint16_t *val16, const double *X, double *Y)
{
    if (val16) return spmm_seg_any<uint16_t>(st, s, nchunks, max_rows, r0, r1, rowptr, colind, val16, X, Y);
    if (val32) return spmm_seg_any<float>(st, s, nchunks, max_rows, r0, r1, rowptr, colind, val32, X, Y);
    return spmm_seg_any<double>(st, s, nchunks, max_rows, r0, r1, rowptr, colind, val, X, Y);
}

int launch_scale_rows_seg(cudaStream_t st, int32_t s, int32_t nchunks, int64_t max_rows, const int64_t *r0,
                          const int64_t *r1, const double *q, const float *q32, const uint16_t *q16, const double *X,
                          double *Y)
{
    if (q16) return scale_rows_seg_any<uint16_t>(st, s, nchunks, max_rows, r0, r1, q16, X, Y);
    if (q32) return scale_rows_seg_any<float>(st, s, nchunks, max_rows, r0, r1, q32, X, Y);
    return scale_rows_seg_any<double>(st, s, nchunks, max_rows, r0, r1, q, X, Y);
}

int launch_pack(cudaStream_t st, int32_t s, int32_t n, const double *src, int64_t ld, double *dst)
{
    if (n <= 0) return 0;
    int g = grid_for((int64_t)n * s);
    switch (s) {
    case 1: k_pack<1><<<g, kThreads, 0, st>>>(n, src, ld, dst); break;
    case 2: k_pack<2><<<g, kThreads, 0, st>>>(n, src, ld, dst); break;
    case 4: k_pack<4><<<g, kThreads, 0, st>>>(n, src, ld, dst); break;
    case 8: k_pack<8><<<g, kThreads, 0, st>>>(n, src, ld, dst); break;
    case 16: k_pack<16><<<g, kThreads, 0, st>>>(n, src, ld, dst); break;
    default: return -1;
    }
    return check_launch();
}

int launch_unpack(cudaStream_t st, int32_t s, int32_t n, const double *src, double *dst, int64_t ld)
{
    if (n <= 0) return 0;
    int g = grid_for((int64_t)n * s);
    switch (s) {
    case 1: k_unpack<1><<<g, kThreads, 0, st>>>(n, src, dst, ld); break;
    case 2: k_unpack<2><<<g, kThreads, 0, st>>>(n, src, dst, ld); break;
    case 4: k_unpack<4><<<g, kThreads, 0, st>>>(n, src, dst, ld); break;
    case 8: k_unpack<8><<<g, kThreads, 0, st>>>(n, src, dst, ld); break;
    case 16: k_unpack<16><<<g, kThreads, 0, st>>>(n, src, dst, ld); break;
    default: return -1;
    }
    return check_launch();
}

}  // namespace spai

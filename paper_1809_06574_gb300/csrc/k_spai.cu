// Column least-squares problems of SPAI and of its update.
//
//   build  (Sec. 2.2):            m_k = argmin_{supp m in J_k} || e_k  - A    m ||_2
//   update (Table 1, Sec. 2.4):   q_k = argmin_{supp q in J_k} || a1_k - A(l) q ||_2
//
// Only the rows I_k = union of rows(A(:,j)), j in J_k, can be nonzero in A m, so each
// problem is the dense |I_k| x |J_k| least-squares problem on Ahat = A(I_k, J_k).
//
// A team of T lanes (T = 1, 2, 4, ..., 32, chosen from the tile size) owns one column.
// The team stages Ahat (column-major, leading dimension maxI) and the right-hand side in
// shared memory straight from A's column-ordered (CSC) arrays, locating every row in I_k
// by binary search, then runs Householder QR -- rows split over the team's lanes, norms
// and reflector dot products reduced with shuffles inside the team -- applying each
// reflector to the right-hand side as it goes, and back-substitutes R m = (Q^T rhs)(0:|J_k|).
// Results go straight to the row-ordered (CSR) value array of the factor via out_map.
//
// FP64 throughput is the limit on GB300 (about 1.1 TFLOP/s), so small tiles use small
// teams: a shuffle reduction spends log2(T) FP64 adds per dot product, and lanes beyond
// |I_k| idle.  Large tiles (the 27-point stencil's 125 x 27) use whole warps.
#include <cuda_bf16.h>

#include <cmath>

#include "spai_internal.cuh"

namespace spai {

namespace {

__device__ __forceinline__ int bsearch_i32(const int32_t *__restrict__ a, int32_t len, int32_t key)
{
    int32_t lo = 0, hi = len - 1;
    while (lo <= hi) {
        int32_t mid = (lo + hi) >> 1;
        int32_t v = __ldg(a + mid);
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

template <int T, typename R>
__device__ __forceinline__ R team_sum(R v, unsigned mask)
{
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// rank-deficiency threshold on |R_cc| / max |R_tt| for the working precision
template <typename R> __device__ __forceinline__ R singular_rel();
template <> __device__ __forceinline__ double singular_rel<double>() { return 1e-14; }
template <> __device__ __forceinline__ float singular_rel<float>() { return 1e-5f; }

constexpr int kBlock = 128;

// A's value q (or the right-hand side's) in the working precision: an FP32 solve reads the
// values rounded to FP32 beforehand when they are given (the same rounding, no FP64
// conversion per lane), else it rounds the FP64 value itself
template <typename R, typename P>
__device__ __forceinline__ R a_value(const P &cp, int32_t q)
{
    if constexpr (sizeof(R) == 4) {
        if (cp.cval32) return __ldg(cp.cval32 + q);
    }
    return (R)__ldg(cp.cval + q);
}
template <typename R, typename P>
__device__ __forceinline__ R r_value(const P &cp, int32_t q)
{
    if constexpr (sizeof(R) == 4) {
        if (cp.r_val32) return __ldg(cp.r_val32 + q);
    }
    return (R)__ldg(cp.r_val + q);
}

// per-column shared-memory region: Ahat (maxJ x ld, column-major) | rhs (ld) | rdiag (maxJ)
// R: working precision (double, or float for SPAI_PREC_FP32 / SPAI_PREC_BF16); A's values
// are read in FP64 and rounded once to R; the result is written to out_val (R = double),
// out_val32, or rounded to nearest-even BF16 into out_val16.
template <int T, typename R, typename P>
__device__ __forceinline__ void column_ls(const P &cp, int64_t k, R *Ah, int ld, int maxJ, int tl, unsigned mask)
{
    R *rhs = Ah + (size_t)maxJ * ld;
    R *rdiag = rhs + ld;

    const int32_t ia = __ldg(cp.Iptr + k), ni = __ldg(cp.Iptr + k + 1) - ia;
    const int32_t ja = __ldg(cp.Jptr + k), nj = __ldg(cp.Jptr + k + 1) - ja;
    const int32_t *Ik = cp.Ilist + ia;
    if (ni > ld || nj > maxJ) {
        if (tl == 0) {
            atomicOr(cp.d_err, ERR_TOO_WIDE);
            cp.col_status[k] = 1;
        }
        return;
    }
    for (int e = tl; e < nj * ld; e += T) Ah[e] = R(0);
    for (int r = tl; r < ni; r += T) rhs[r] = R(0);
    __syncwarp(mask);

    // ---- gather Ahat = A(I_k, J_k) and the right-hand side
    for (int c = 0; c < nj; ++c) {
        const int32_t j = __ldg(cp.Jind + ja + c);
        const int32_t a = __ldg(cp.colptr + j), b = __ldg(cp.colptr + j + 1);
        for (int32_t q = a + tl; q < b; q += T) {
            const int pos = bsearch_i32(Ik, ni, __ldg(cp.rowind + q));
            if (pos >= 0) Ah[c * ld + pos] = a_value<R>(cp, q);
        }
    }
    if (cp.mode == 0) {
        if (tl == 0) {
            const int pos = bsearch_i32(Ik, ni, (int32_t)k);
            if (pos >= 0) rhs[pos] = R(1);
        }
    } else {
        const int32_t a = __ldg(cp.r_colptr + k), b = __ldg(cp.r_colptr + k + 1);
        for (int32_t q = a + tl; q < b; q += T) {
            const int pos = bsearch_i32(Ik, ni, __ldg(cp.r_rowind + q));
            if (pos >= 0) rhs[pos] = r_value<R>(cp, q);
        }
    }
    __syncwarp(mask);

    // ---- Householder QR; column c keeps its reflector v below (and on) the diagonal
    bool singular = ni < nj;
    for (int c = 0; c < nj && !singular; ++c) {
        const R *vc = Ah + c * ld;
        R ss = R(0);
        for (int r = c + tl; r < ni; r += T) ss = fma(vc[r], vc[r], ss);
        ss = team_sum<T, R>(ss, mask);
        const R alpha = sqrt(ss);
        if (!(alpha > R(0))) {
            singular = true;
            break;
        }
        const R xc = vc[c];
        const R sgn = (xc >= R(0)) ? R(1) : R(-1);
        const R inv = R(1) / (alpha * (alpha + fabs(xc)));  // 2 / v^T v
        __syncwarp(mask);
        if (tl == (c % T)) Ah[c * ld + c] = xc + sgn * alpha;
        if (tl == 0) rdiag[c] = -sgn * alpha;
        __syncwarp(mask);
        for (int t = c + 1; t <= nj; ++t) {  // t == nj is the right-hand side
            R *col = (t < nj) ? (Ah + t * ld) : rhs;
            R d = R(0);
            for (int r = c + tl; r < ni; r += T) d = fma(vc[r], col[r], d);
            const R g = team_sum<T, R>(d, mask) * inv;
            for (int r = c + tl; r < ni; r += T) col[r] = fma(-g, vc[r], col[r]);
        }
        __syncwarp(mask);
    }
    if (!singular) {
        R rmax = R(0);
        for (int c = 0; c < nj; ++c) rmax = fmax(rmax, fabs(rdiag[c]));
        for (int c = 0; c < nj; ++c)
            if (fabs(rdiag[c]) <= singular_rel<R>() * rmax) singular = true;
    }
    if (singular) {
        for (int c = tl; c < nj; c += T) {
            if (cp.out_val16) cp.out_val16[cp.out_map[ja + c]] = 0;
            else if (cp.out_val32) cp.out_val32[cp.out_map[ja + c]] = 0.0f;
            else cp.out_val[cp.out_map[ja + c]] = 0.0;
        }
        if (tl == 0) cp.col_status[k] = 1;
        return;
    }

    // ---- back substitution R m = (Q^T rhs)(0:nj); m overwrites rhs(0:nj)
    for (int c = nj - 1; c >= 0; --c) {
        R acc = R(0);
        for (int t = c + 1 + tl; t < nj; t += T) acc = fma(Ah[t * ld + c], rhs[t], acc);
        acc = team_sum<T, R>(acc, mask);
        if (tl == 0) rhs[c] = (rhs[c] - acc) / rdiag[c];
        __syncwarp(mask);
    }
    for (int c = tl; c < nj; c += T) {
        if (cp.out_val16) cp.out_val16[cp.out_map[ja + c]] = __bfloat16_as_ushort(__float2bfloat16_rn((float)rhs[c]));
        else if (cp.out_val32) cp.out_val32[cp.out_map[ja + c]] = (float)rhs[c];
        else cp.out_val[cp.out_map[ja + c]] = (double)rhs[c];
    }
    if (tl == 0) cp.col_status[k] = 0;
}


// One team per column problem, persistent over the columns: column g of a batch belongs to
// the system i with start[i] <= g < start[i + 1] (its local column g - start[i]); without
// a batch table the columns are those of cp0.
template <int T, typename R>
__global__ void __launch_bounds__(kBlock) k_spai_columns(ColumnProblem cp0, ColumnBatch bt, int ld, int maxJ, int L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *smem = reinterpret_cast<R *>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int team = threadIdx.x / T, tl = threadIdx.x % T;
    const int teams = blockDim.x / T;
    const unsigned mask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << ((lane / T) * T));
    R *Ah = smem + (size_t)team * L;
    const int64_t total = bt.tab ? bt.total : (int64_t)cp0.n;
    // the whole team takes the same columns and leaves together
    for (int64_t g = (int64_t)blockIdx.x * teams + team; g < total; g += (int64_t)gridDim.x * teams) {
        if (bt.tab) {
            int lo = 0, hi = bt.nsys - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(bt.start + mid) <= g) lo = mid; else hi = mid - 1;
            }
            column_ls<T, R>(bt.tab[lo], g - __ldg(bt.start + lo), Ah, ld, maxJ, tl, mask);
        } else {
            column_ls<T, R>(cp0, g, Ah, ld, maxJ, tl, mask);
        }
        __syncwarp(mask);
    }
}

// ---- register-tiled variant for small tiles: no shared memory, everything unrolled.
// Lane tl of a team of T owns rows tl, tl + T, ..., tl + (RPL-1) T of the tile (RPL rows
// per lane, up to T * RPL rows) for all MJ (>= |J_k|) columns and the right-hand side, in
// registers.  The gather compares each lane's rows with the (sorted) row lists of the
// columns of J_k, so it needs no search; the Householder sweep is the one of column_ls with
// every loop bound a compile-time constant (columns past |J_k| are skipped by a team-uniform
// predicate); the back substitution runs on the lane that owns each row of R and broadcasts
// the solved value.  Same arithmetic as column_ls, in another order of the reductions.
template <int T, int RPL, int MJ, typename R, typename P>
__device__ __forceinline__ void column_ls_reg(const P &cp, int64_t k, int tl, unsigned mask)
{
    const int32_t ia = __ldg(cp.Iptr + k), ni = __ldg(cp.Iptr + k + 1) - ia;
    const int32_t ja = __ldg(cp.Jptr + k), nj = __ldg(cp.Jptr + k + 1) - ja;
    if (ni > T * RPL || nj > MJ) {
        if (tl == 0) {
            atomicOr(cp.d_err, ERR_TOO_WIDE);
            cp.col_status[k] = 1;
        }
        return;
    }
    int32_t row[RPL];
#pragma unroll
    for (int i = 0; i < RPL; ++i) row[i] = (tl + T * i < ni) ? __ldg(cp.Ilist + ia + tl + T * i) : -1;
    R a[MJ][RPL], b[RPL];
#pragma unroll
    for (int c = 0; c < MJ; ++c) {
#pragma unroll
        for (int i = 0; i < RPL; ++i) a[c][i] = R(0);
        if (c < nj) {
            const int32_t j = __ldg(cp.Jind + ja + c);
            const int32_t q1 = __ldg(cp.colptr + j + 1);
            for (int32_t q = __ldg(cp.colptr + j); q < q1; ++q) {
                const int32_t r = __ldg(cp.rowind + q);
                const R v = a_value<R>(cp, q);
#pragma unroll
                for (int i = 0; i < RPL; ++i)
                    if (row[i] == r) a[c][i] = v;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < RPL; ++i) b[i] = (cp.mode == 0 && row[i] == (int32_t)k) ? R(1) : R(0);
    if (cp.mode != 0) {
        const int32_t q1 = __ldg(cp.r_colptr + k + 1);
        for (int32_t q = __ldg(cp.r_colptr + k); q < q1; ++q) {
            const int32_t r = __ldg(cp.r_rowind + q);
            const R v = r_value<R>(cp, q);
#pragma unroll
            for (int i = 0; i < RPL; ++i)
                if (row[i] == r) b[i] = v;
        }
    }

    // ---- Householder QR, reflectors applied to the columns right of c and to b
    R rd[MJ];
    bool singular = ni < nj;
#pragma unroll
    for (int c = 0; c < MJ; ++c) {
        rd[c] = R(1);
        if (c < nj && !singular) {
            // slot i holds rows T*i .. T*i + T-1: slots wholly above row c (known at compile
            // time) and slots wholly past the last row (team-uniform) take no part
            R v[RPL];
            R ss = R(0);
#pragma unroll
            for (int i = 0; i < RPL; ++i) {
                v[i] = (tl + T * i >= c) ? a[c][i] : R(0);
                if (T * i + T - 1 >= c && T * i < ni) ss = fma(v[i], v[i], ss);
            }
            ss = team_sum<T, R>(ss, mask);
            const R alpha = sqrt(ss);
            if (!(alpha > R(0))) {
                singular = true;
            } else {
                const R xc = __shfl_sync(mask, a[c][c / T], c % T, T);
                const R sgn = (xc >= R(0)) ? R(1) : R(-1);
                const R inv = R(1) / (alpha * (alpha + fabs(xc)));  // 2 / v^T v
                if (tl == c % T) v[c / T] = xc + sgn * alpha;
                rd[c] = -sgn * alpha;
#pragma unroll
                for (int t = 1; t < MJ; ++t) {  // (a fixed range keeps the nest fully unrolled)
                    if (t > c && t < nj) {
                        R d = R(0);
#pragma unroll
                        for (int i = 0; i < RPL; ++i)
                            if (T * i + T - 1 >= c && T * i < ni) d = fma(v[i], a[t][i], d);
                        const R g = team_sum<T, R>(d, mask) * inv;
#pragma unroll
                        for (int i = 0; i < RPL; ++i)
                            if (T * i + T - 1 >= c && T * i < ni) a[t][i] = fma(-g, v[i], a[t][i]);
                    }
                }
                R d = R(0);
#pragma unroll
                for (int i = 0; i < RPL; ++i)
                    if (T * i + T - 1 >= c && T * i < ni) d = fma(v[i], b[i], d);
                const R g = team_sum<T, R>(d, mask) * inv;
#pragma unroll
                for (int i = 0; i < RPL; ++i)
                    if (T * i + T - 1 >= c && T * i < ni) b[i] = fma(-g, v[i], b[i]);
            }
        }
    }
    if (!singular) {
        R rmax = R(0);
#pragma unroll
        for (int c = 0; c < MJ; ++c)
            if (c < nj) rmax = fmax(rmax, fabs(rd[c]));
#pragma unroll
        for (int c = 0; c < MJ; ++c)
            if (c < nj && fabs(rd[c]) <= singular_rel<R>() * rmax) singular = true;
    }
    if (singular) {
        for (int c = tl; c < nj; c += T) {
            if (cp.out_val16) cp.out_val16[cp.out_map[ja + c]] = 0;
            else if (cp.out_val32) cp.out_val32[cp.out_map[ja + c]] = 0.0f;
            else cp.out_val[cp.out_map[ja + c]] = 0.0;
        }
        if (tl == 0) cp.col_status[k] = 1;
        return;
    }

    // ---- back substitution: row c of R and of Q^T b live on lane c % T, slot c / T
    R m[MJ];
#pragma unroll
    for (int c = MJ - 1; c >= 0; --c) {
        m[c] = R(0);
        if (c < nj) {
            R acc = R(0);
#pragma unroll
            for (int t = 1; t < MJ; ++t)
                if (t > c && t < nj) acc = fma(a[t][c / T], m[t], acc);
            m[c] = __shfl_sync(mask, (b[c / T] - acc) / rd[c], c % T, T);
        }
    }
#pragma unroll
    for (int c = 0; c < MJ; ++c) {
        if (c < nj && c % T == tl) {
            if (cp.out_val16) cp.out_val16[cp.out_map[ja + c]] = __bfloat16_as_ushort(__float2bfloat16_rn((float)m[c]));
            else if (cp.out_val32) cp.out_val32[cp.out_map[ja + c]] = (float)m[c];
            else cp.out_val[cp.out_map[ja + c]] = (double)m[c];
        }
    }
    if (tl == 0) cp.col_status[k] = 0;
}

template <int T, int RPL, int MJ, typename R>
__global__ void __launch_bounds__(kBlock) k_spai_columns_reg(ColumnProblem cp0, ColumnBatch bt)
{
    const int lane = threadIdx.x & 31;
    const int team = threadIdx.x / T, tl = threadIdx.x % T;
    const int teams = blockDim.x / T;
    const unsigned mask = (T == 32) ? 0xffffffffu : (((1u << T) - 1u) << ((lane / T) * T));
    const int64_t total = bt.tab ? bt.total : (int64_t)cp0.n;
    for (int64_t g = (int64_t)blockIdx.x * teams + team; g < total; g += (int64_t)gridDim.x * teams) {
        if (bt.tab) {
            int lo = 0, hi = bt.nsys - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(bt.start + mid) <= g) lo = mid; else hi = mid - 1;
            }
            column_ls_reg<T, RPL, MJ, R>(bt.tab[lo], g - __ldg(bt.start + lo), tl, mask);
        } else {
            column_ls_reg<T, RPL, MJ, R>(cp0, g, tl, mask);
        }
        __syncwarp(mask);
    }
}

// ---- one lane per column problem for small tiles.  The lane stages its own problem in
// its own shared-memory region -- the row list I_k padded with INT_MAX to MI entries, Ahat
// column-major with leading dimension ld, the right-hand side -- placing every entry of
// A(:, J_k) by a fixed-step binary search over the staged rows, then runs the Householder
// sweep of column_ls with T = 1: the reflector of column c and the column it is applied
// to sit in registers (each tile entry is loaded and stored once per reflector, nothing is
// reduced across lanes), R stays in the tile (its diagonal in registers) for the back
// substitution.  MI (a power of two >= ld) and MJ (>= |J_k|) are compile-time bounds:
// every row loop is unrolled over MI, rows past |I_k| skipped by predicates, rows above
// the reflector's row skipped at compile time.  Same arithmetic as column_ls, the dot
// products summed in four interleaved partial sums.
constexpr int kLaneBlock = 32;

// index of the first staged row >= r (rows sorted, INT_MAX beyond |I_k|, MI a power of two)
template <int MI>
__device__ __forceinline__ int lane_pos(const int32_t *rows, int32_t r)
{
    int p = 0;
#pragma unroll
    for (int s = MI / 2; s > 0; s >>= 1)
        if (rows[p + s - 1] < r) p += s;
    return p;
}

// stage the lane's problem: rows of I_k, Ahat = A(I_k, J_k) and the right-hand side;
// false (status 1, ERR_TOO_WIDE) when the tile exceeds the lane's region
// With rhs NULL (a build by the normal equations) the right-hand side e_k is not staged: *pk
// is the position of row k in I_k (or -1).
template <int MI, int MJ, typename R, typename P>
__device__ __forceinline__ bool gather_lane(const P &cp, int64_t k, int32_t *rows, R *Ah, R *rhs, int ld, int mj,
                                            int32_t ni, int32_t ja, int32_t nj, int32_t ia, int *pk = nullptr)
{
    if (ni > ld || nj > mj || ni > MI || nj > MJ) {
        atomicOr(cp.d_err, ERR_TOO_WIDE);
        cp.col_status[k] = 1;
        return false;
    }
    // the column pointers of all of J_k first (two rounds of independent loads), then each
    // column's entries four at a time with their four searches interleaved
    int32_t q0[MJ], q1[MJ];
#pragma unroll
    for (int c = 0; c < MJ; ++c) q0[c] = (c < nj) ? __ldg(cp.Jind + ja + c) : 0;
#pragma unroll
    for (int c = 0; c < MJ; ++c) {
        const int32_t j = q0[c];
        q0[c] = (c < nj) ? __ldg(cp.colptr + j) : 0;
        q1[c] = (c < nj) ? __ldg(cp.colptr + j + 1) : 0;
    }
#pragma unroll
    for (int i = 0; i < MI; ++i) rows[i] = (i < ni) ? __ldg(cp.Ilist + ia + i) : INT_MAX;
    for (int e = 0; e < nj * ld; ++e) Ah[e] = R(0);
    if (rhs)
        for (int i = 0; i < ni; ++i) rhs[i] = R(0);
#pragma unroll
    for (int c = 0; c < MJ; ++c) {
#pragma unroll 2
        for (int32_t q = q0[c]; q < q1[c]; q += 4) {
            int32_t r[4];
            R v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool in = q + u < q1[c];
                r[u] = in ? __ldg(cp.rowind + q + u) : INT_MAX;
                v[u] = in ? a_value<R>(cp, q + u) : R(0);
            }
            int p[4] = {0, 0, 0, 0};
#pragma unroll
            for (int s = MI / 2; s > 0; s >>= 1)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (rows[p[u] + s - 1] < r[u]) p[u] += s;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (r[u] != INT_MAX && rows[p[u]] == r[u]) Ah[c * ld + p[u]] = v[u];
        }
    }
    if (!rhs) {
        const int p = lane_pos<MI>(rows, (int32_t)k);
        *pk = (rows[p] == (int32_t)k) ? p : -1;
    } else if (cp.mode == 0) {
        const int p = lane_pos<MI>(rows, (int32_t)k);
        if (rows[p] == (int32_t)k) rhs[p] = R(1);
    } else {
        const int32_t a = __ldg(cp.r_colptr + k), b = __ldg(cp.r_colptr + k + 1);
        for (int32_t q = a; q < b; ++q) {
            const int32_t r = __ldg(cp.r_rowind + q);
            const int p = lane_pos<MI>(rows, r);
            if (rows[p] == r) rhs[p] = r_value<R>(cp, q);
        }
    }
    return true;
}

// the solution m (or zeros for a rank-deficient column) to the factor, and the status;
// om: the output positions out_map[ja + c], loaded early by the caller
template <int MJ, typename R, typename P>
__device__ __forceinline__ void store_lane(const P &cp, int64_t k, int32_t nj, const int32_t (&om)[MJ],
                                           const R (&m)[MJ], bool singular)
{
#pragma unroll
    for (int c = 0; c < MJ; ++c) {
        if (c < nj) {
            const R v = singular ? R(0) : m[c];
            if (cp.out_val16) cp.out_val16[om[c]] = __bfloat16_as_ushort(__float2bfloat16_rn((float)v));
            else if (cp.out_val32) cp.out_val32[om[c]] = (float)v;
            else cp.out_val[om[c]] = (double)v;
        }
    }
    cp.col_status[k] = singular ? 1 : 0;
}

template <int MJ, typename P>
__device__ __forceinline__ void load_out_map(const P &cp, int32_t ja, int32_t nj, int32_t (&om)[MJ])
{
#pragma unroll
    for (int c = 0; c < MJ; ++c) om[c] = (c < nj) ? __ldg(cp.out_map + ja + c) : 0;
}

template <int MI, int MJ, typename R, typename P>
__device__ __forceinline__ void column_ls_lane(const P &cp, int64_t k, int32_t *rows, R *Ah, int ld, int mj)
{
    R *rhs = Ah + (size_t)mj * ld;
    const int32_t ia = __ldg(cp.Iptr + k), ni = __ldg(cp.Iptr + k + 1) - ia;
    const int32_t ja = __ldg(cp.Jptr + k), nj = __ldg(cp.Jptr + k + 1) - ja;
    if (!gather_lane<MI, MJ, R>(cp, k, rows, Ah, rhs, ld, mj, ni, ja, nj, ia)) return;
    int32_t om[MJ];
    load_out_map<MJ>(cp, ja, nj, om);

    // ---- Householder QR; R above the diagonal stays in the tile, its diagonal in rd
    bool singular = ni < nj;
    R rd[MJ];
#pragma unroll
    for (int c = 0; c < MJ; ++c) {
        rd[c] = R(1);
        if (c < nj && !singular) {
            R v[MI];
            R s4[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
            for (int i = c; i < MI; ++i) {
                v[i] = (i < ni) ? Ah[c * ld + i] : R(0);
                s4[i & 3] = fma(v[i], v[i], s4[i & 3]);
            }
            const R alpha = sqrt((s4[0] + s4[1]) + (s4[2] + s4[3]));
            if (!(alpha > R(0))) {
                singular = true;
            } else {
                const R xc = v[c];
                const R sgn = (xc >= R(0)) ? R(1) : R(-1);
                const R inv = R(1) / (alpha * (alpha + fabs(xc)));  // 2 / v^T v
                v[c] = xc + sgn * alpha;
                rd[c] = -sgn * alpha;
                for (int t = c + 1; t <= nj; ++t) {  // t == nj is the right-hand side
                    R *col = (t < nj) ? (Ah + t * ld) : rhs;
                    R x[MI];
                    R d4[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
                    for (int i = c; i < MI; ++i) {
                        if (i < ni) {
                            x[i] = col[i];
                            d4[i & 3] = fma(v[i], x[i], d4[i & 3]);
                        }
                    }
                    const R g = ((d4[0] + d4[1]) + (d4[2] + d4[3])) * inv;
#pragma unroll
                    for (int i = c; i < MI; ++i)
                        if (i < ni) col[i] = fma(-g, v[i], x[i]);
                }
            }
        }
    }
    if (!singular) {
        R rmax = R(0);
#pragma unroll
        for (int c = 0; c < MJ; ++c)
            if (c < nj) rmax = fmax(rmax, fabs(rd[c]));
#pragma unroll
        for (int c = 0; c < MJ; ++c)
            if (c < nj && fabs(rd[c]) <= singular_rel<R>() * rmax) singular = true;
    }
    // ---- back substitution R m = (Q^T rhs)(0:nj)
    R m[MJ];
#pragma unroll
    for (int c = MJ - 1; c >= 0; --c) {
        m[c] = R(0);
        if (c < nj && !singular) {
            R acc = R(0);
#pragma unroll
            for (int t = c + 1; t < MJ; ++t)
                if (t < nj) acc = fma(Ah[t * ld + c], m[t], acc);
            m[c] = (rhs[c] - acc) / rd[c];
        }
    }
    store_lane<MJ, R>(cp, k, nj, om, m, singular);
}

// rank-deficiency threshold of the normal equations: a Cholesky pivot (R_cc^2) at most
// rel^2 times the largest diagonal entry of G; the normal equations resolve R's diagonal
// only to about the square root of the working precision
template <typename R> __device__ __forceinline__ R singular_rel_ne();
template <> __device__ __forceinline__ double singular_rel_ne<double>() { return 1e-7; }
template <> __device__ __forceinline__ float singular_rel_ne<float>() { return 1e-3f; }

// The same column problem by its normal equations (SPAI_LS_NORMAL): G = Ahat^T Ahat and
// h = Ahat^T rhs (in FP64 summed over the nonzero entries of each column of Ahat only --
// a column of A has few, so the work is the nonzeros' products, not the dense tile's; in
// FP32 row by row over the dense tile), then G = R^T R by Cholesky and R^T R m = h by two
// triangular solves, all in registers.  Exact arithmetic gives the least-squares
// solution of column_ls; in floating point the error grows with cond(Ahat)^2 instead of
// cond(Ahat).
template <int MI, int MJ, typename R, typename P>
__device__ __forceinline__ void column_ne_lane(const P &cp, int64_t k, int32_t *rows, R *Ah, int ld, int mj,
                                               bool with_rhs)
{
    // a build (rhs e_k) stages no right-hand side: h_c = Ahat(k, c)
    R *rhs = with_rhs ? Ah + (size_t)mj * ld : nullptr;
    const int32_t ia = __ldg(cp.Iptr + k), ni = __ldg(cp.Iptr + k + 1) - ia;
    const int32_t ja = __ldg(cp.Jptr + k), nj = __ldg(cp.Jptr + k + 1) - ja;
    int pk = -1;
    if (!gather_lane<MI, MJ, R>(cp, k, rows, Ah, rhs, ld, mj, ni, ja, nj, ia, &pk)) return;
    int32_t om[MJ];
    load_out_map<MJ>(cp, ja, nj, om);

    // ---- G (upper triangle) and h
    R G[MJ][MJ], h[MJ];
#pragma unroll
    for (int c = 0; c < MJ; ++c) {
        h[c] = R(0);
#pragma unroll
        for (int t = c; t < MJ; ++t) G[c][t] = R(0);
    }
    if constexpr (sizeof(R) == 4) {
        // FP32: row by row over the dense tile, every product of a row at once (no branches;
        // the FP32 pipe has the throughput to spare)
        for (int i = 0; i < ni; ++i) {
            R a[MJ];
#pragma unroll
            for (int c = 0; c < MJ; ++c) a[c] = (c < nj) ? Ah[c * ld + i] : R(0);
#pragma unroll
            for (int c = 0; c < MJ; ++c)
#pragma unroll
                for (int t = c; t < MJ; ++t) G[c][t] = fma(a[c], a[t], G[c][t]);
            if (rhs) {
                const R b = rhs[i];
#pragma unroll
                for (int c = 0; c < MJ; ++c) h[c] = fma(a[c], b, h[c]);
            }
        }
    } else {
        // FP64: the products of each column's nonzero entries only (the FP64 pipe is the
        // bound: a column of A has few nonzeros in its tile column)
#pragma unroll
        for (int c = 0; c < MJ; ++c) {
            if (c < nj) {
                for (int i = 0; i < ni; ++i) {
                    const R a = Ah[c * ld + i];
                    if (a != R(0)) {
#pragma unroll
                        for (int t = c; t < MJ; ++t)
                            if (t < nj) G[c][t] = fma(a, Ah[t * ld + i], G[c][t]);
                        if (rhs) h[c] = fma(a, rhs[i], h[c]);
                    }
                }
            }
        }
    }
    if (!rhs) {
#pragma unroll
        for (int c = 0; c < MJ; ++c) h[c] = (c < nj && pk >= 0) ? Ah[c * ld + pk] : R(0);
    }
    // ---- G = R^T R (R upper, over G's upper triangle), R^T y = h, R m = y
    bool singular = ni < nj;
    R gmax = R(0);
#pragma unroll
    for (int c = 0; c < MJ; ++c)
        if (c < nj) gmax = fmax(gmax, G[c][c]);
    const R rel = singular_rel_ne<R>();
    const R tiny = rel * rel * gmax;
    R rinv[MJ];
#pragma unroll
    for (int c = 0; c < MJ; ++c) {
        rinv[c] = R(0);
        if (c < nj && !singular) {
            R d = G[c][c];
#pragma unroll
            for (int p = 0; p < c; ++p) d = fma(-G[p][c], G[p][c], d);
            if (!(d > tiny)) {
                singular = true;
            } else {
                const R rcc = sqrt(d);
                rinv[c] = R(1) / rcc;
                G[c][c] = rcc;
#pragma unroll
                for (int t = c + 1; t < MJ; ++t) {
                    if (t < nj) {
                        R e = G[c][t];
#pragma unroll
                        for (int p = 0; p < c; ++p) e = fma(-G[p][c], G[p][t], e);
                        G[c][t] = e * rinv[c];
                    }
                }
            }
        }
    }
    R m[MJ];
#pragma unroll
    for (int c = 0; c < MJ; ++c) {  // R^T y = h
        m[c] = R(0);
        if (c < nj && !singular) {
            R e = h[c];
#pragma unroll
            for (int p = 0; p < c; ++p) e = fma(-G[p][c], m[p], e);
            m[c] = e * rinv[c];
        }
    }
#pragma unroll
    for (int c = MJ - 1; c >= 0; --c) {  // R m = y
        if (c < nj && !singular) {
            R e = m[c];
#pragma unroll
            for (int t = c + 1; t < MJ; ++t)
                if (t < nj) e = fma(-G[c][t], m[t], e);
            m[c] = e * rinv[c];
        }
    }
    store_lane<MJ, R>(cp, k, nj, om, m, singular);
}

// words of one lane's region: MI row slots, then (mj + 1) x ld values of R; odd in units of
// R, so that the lanes of a warp reading the same offset of their regions hit distinct banks
__host__ __device__ inline int lane_words(int mi, int ld, int mj, bool low, bool with_rhs = true)
{
    const int vals = (mj + (with_rhs ? 1 : 0)) * ld;
    return low ? ((mi + vals) | 1) : 2 * ((mi / 2 + vals) | 1);
}
template <int MI, typename R>
__host__ __device__ inline int lane_stride_words(int ld, int mj, bool with_rhs)
{
    return lane_words(MI, ld, mj, sizeof(R) == 4, with_rhs);
}

template <int MI, int MJ, typename R, bool NE>
__global__ void __launch_bounds__(kLaneBlock) k_spai_columns_lane(ColumnProblem cp0, ColumnBatch bt, int ld, int mj,
                                                                  bool with_rhs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *base =
        reinterpret_cast<uint32_t *>(smem_raw) + (size_t)threadIdx.x * lane_stride_words<MI, R>(ld, mj, with_rhs);
    int32_t *rows = reinterpret_cast<int32_t *>(base);
    R *Ah = reinterpret_cast<R *>(base + MI);
    const int64_t total = bt.tab ? bt.total : (int64_t)cp0.n;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        if (bt.tab) {
            int lo = 0, hi = bt.nsys - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(bt.start + mid) <= g) lo = mid; else hi = mid - 1;
            }
            if constexpr (NE) column_ne_lane<MI, MJ, R>(bt.tab[lo], g - __ldg(bt.start + lo), rows, Ah, ld, mj, with_rhs);
            else column_ls_lane<MI, MJ, R>(bt.tab[lo], g - __ldg(bt.start + lo), rows, Ah, ld, mj);
        } else {
            if constexpr (NE) column_ne_lane<MI, MJ, R>(cp0, g, rows, Ah, ld, mj, with_rhs);
            else column_ls_lane<MI, MJ, R>(cp0, g, rows, Ah, ld, mj);
        }
    }
}

// the one-lane shapes: rows MI (a power of two), columns MJ
struct LaneShape {
    int MI, MJ;
};
constexpr LaneShape kLaneShapes[] = {{16, 5}, {32, 7}, {32, 8}, {32, 13}};
constexpr int kNumLaneShapes = 4;
constexpr int kLaneTeamBase = 96;  // team codes kLaneTeamBase + i select kLaneShapes[i]

bool lane_fits(int i, int32_t maxI, int32_t maxJ, bool low)
{
    if (maxI > kLaneShapes[i].MI || maxJ > kLaneShapes[i].MJ) return false;
    const int ld = maxI < 1 ? 1 : maxI, mj = maxJ < 1 ? 1 : maxJ;
    return (size_t)kLaneBlock * lane_words(kLaneShapes[i].MI, ld, mj, low) * 4 <= 200 * 1024;
}

template <int MI, int MJ, typename R, bool NE = false>
int launch_lane(cudaStream_t st, const ColumnProblem &cp, const ColumnBatch &bt, int32_t maxI, int32_t maxJ)
{
    const int ld = maxI < 1 ? 1 : maxI, mj = maxJ < 1 ? 1 : maxJ;
    if (ld > MI || mj > MJ) return -1;
    // the normal equations of a build stage no right-hand side (batches are builds)
    const bool with_rhs = !(NE && (bt.tab || cp.mode == 0));
    const size_t smem = (size_t)kLaneBlock * lane_stride_words<MI, R>(ld, mj, with_rhs) * 4;
    if (smem > 227 * 1024) return -1;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_spai_columns_lane<MI, MJ, R, NE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return -1;
    const int64_t total = bt.tab ? bt.total : (int64_t)cp.n;
    int64_t blocks = (total + kLaneBlock - 1) / kLaneBlock;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spai_columns_lane<MI, MJ, R, NE>, kLaneBlock, smem) !=
            cudaSuccess)
        return -1;
    const int64_t resident = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > resident) blocks = resident;
    if (blocks < 1) blocks = 1;
    k_spai_columns_lane<MI, MJ, R, NE><<<(unsigned)blocks, kLaneBlock, smem, st>>>(cp, bt, ld, mj, with_rhs);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// normal-equations shapes (SPAI_LS_NORMAL): G's upper triangle stays in registers, so MJ <= 8
constexpr LaneShape kNeShapes[] = {{16, 5}, {32, 7}, {32, 8}};
constexpr int kNumNeShapes = 3;
constexpr int kNeTeamBase = 112;  // team codes kNeTeamBase + i select kNeShapes[i]

bool ne_fits(int i, int32_t maxI, int32_t maxJ, bool low)
{
    if (maxI > kNeShapes[i].MI || maxJ > kNeShapes[i].MJ) return false;
    const int ld = maxI < 1 ? 1 : maxI, mj = maxJ < 1 ? 1 : maxJ;
    return (size_t)kLaneBlock * lane_words(kNeShapes[i].MI, ld, mj, low) * 4 <= 200 * 1024;
}

template <typename R>
int launch_ne_shape(cudaStream_t st, const ColumnProblem &cp, const ColumnBatch &bt, int i, int32_t maxI,
                    int32_t maxJ)
{
    switch (i) {
    case 0: return launch_lane<16, 5, R, true>(st, cp, bt, maxI, maxJ);
    case 1: return launch_lane<32, 7, R, true>(st, cp, bt, maxI, maxJ);
    case 2: return launch_lane<32, 8, R, true>(st, cp, bt, maxI, maxJ);
    default: return -1;
    }
}

template <typename R>
int launch_lane_shape(cudaStream_t st, const ColumnProblem &cp, const ColumnBatch &bt, int i, int32_t maxI,
                      int32_t maxJ)
{
    switch (i) {
    case 0: return launch_lane<16, 5, R>(st, cp, bt, maxI, maxJ);
    case 1: return launch_lane<32, 7, R>(st, cp, bt, maxI, maxJ);
    case 2: return launch_lane<32, 8, R>(st, cp, bt, maxI, maxJ);
    case 3: return launch_lane<32, 13, R>(st, cp, bt, maxI, maxJ);
    default: return -1;
    }
}

// the register-tiled shapes: team T, rows per lane RPL (tile rows <= T * RPL), columns MJ
struct RegShape {
    int T, RPL, MJ;
};
constexpr RegShape kRegShapes[] = {{4, 4, 5}, {8, 4, 8}, {4, 8, 8}, {8, 4, 13}, {4, 8, 7}};
constexpr int kNumRegShapes = 5;
constexpr int kRegTeamBase = 64;  // team codes kRegTeamBase + i select kRegShapes[i]

template <int T, int RPL, int MJ, typename R>
int launch_reg(cudaStream_t st, const ColumnProblem &cp, const ColumnBatch &bt)
{
    const int teams = kBlock / T;
    const int64_t total = bt.tab ? bt.total : (int64_t)cp.n;
    int64_t blocks = (total + teams - 1) / teams;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spai_columns_reg<T, RPL, MJ, R>, kBlock, 0) !=
            cudaSuccess)
        return -1;
    const int64_t resident = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > resident) blocks = resident;
    if (blocks < 1) blocks = 1;
    k_spai_columns_reg<T, RPL, MJ, R><<<(unsigned)blocks, kBlock, 0, st>>>(cp, bt);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

bool reg_fits(int i, int32_t maxI, int32_t maxJ)
{
    return maxI <= kRegShapes[i].T * kRegShapes[i].RPL && maxJ <= kRegShapes[i].MJ;
}

template <typename R>
int launch_reg_shape(cudaStream_t st, const ColumnProblem &cp, const ColumnBatch &bt, int i)
{
    switch (i) {
    case 0: return launch_reg<4, 4, 5, R>(st, cp, bt);
    case 1: return launch_reg<8, 4, 8, R>(st, cp, bt);
    case 2: return launch_reg<4, 8, 8, R>(st, cp, bt);
    case 3: return launch_reg<8, 4, 13, R>(st, cp, bt);
    case 4: return launch_reg<4, 8, 7, R>(st, cp, bt);  // the 3D 7-point tiles (25 x 7): no padded column
    default: return -1;
    }
}

template <int T, typename R>
int launch_team(cudaStream_t st, const ColumnProblem &cp, const ColumnBatch &bt, int ld, int maxJ, int L,
                int threads)
{
    const int teams = threads / T;
    const size_t smem = (size_t)teams * L * sizeof(R);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_spai_columns<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return -1;
    const int64_t total = bt.tab ? bt.total : (int64_t)cp.n;
    int64_t blocks = (total + teams - 1) / teams;
    if (bt.tab) {
        // persistent: as many blocks as are resident at once
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spai_columns<T, R>, threads, smem) != cudaSuccess)
            return -1;
        const int64_t resident = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
        if (blocks > resident) blocks = resident;
    }
    if (blocks < 1) blocks = 1;
    k_spai_columns<T, R><<<(unsigned)blocks, threads, smem, st>>>(cp, bt, ld, maxJ, L);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Diagonal update (J_k = {k}): the column least squares over one unknown,
// q_kk = <A(l)(:,k), a1_k> / ||A(l)(:,k)||^2 in the working precision R, both columns on
// A's CSC pattern (cval: A(l), rval: A(1)); a zero column is rank deficient (q = 0,
// status 1).  One thread per column.
template <typename R>
__global__ void k_diag_update(int32_t n, const int32_t *__restrict__ colptr, const double *__restrict__ cval,
                              const double *__restrict__ rval, double *__restrict__ out, float *__restrict__ out32,
                              uint16_t *__restrict__ out16, int32_t *__restrict__ status)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    R dot = R(0), nrm = R(0);
    for (int32_t q = __ldg(colptr + k); q < __ldg(colptr + k + 1); ++q) {
        const R a = (R)__ldg(cval + q);
        dot = fma(a, (R)__ldg(rval + q), dot);
        nrm = fma(a, a, nrm);
    }
    const bool sing = !(nrm > R(0));
    const R v = sing ? R(0) : dot / nrm;
    if (out16) out16[k] = __bfloat16_as_ushort(__float2bfloat16_rn((float)v));
    else if (out32) out32[k] = (float)v;
    else out[k] = (double)v;
    status[k] = sing ? 1 : 0;
}

}  // namespace

int launch_diag_update(cudaStream_t st, int32_t n, const int32_t *colptr, const double *cval, const double *rval,
                       double *out, float *out32, uint16_t *out16, int32_t *status)
{
    if (n <= 0) return 0;
    const unsigned g = (unsigned)(((int64_t)n + 255) / 256);
    if (out32 || out16)
        k_diag_update<float><<<g, 256, 0, st>>>(n, colptr, cval, rval, out, out32, out16, status);
    else
        k_diag_update<double><<<g, 256, 0, st>>>(n, colptr, cval, rval, out, out32, out16, status);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

bool spai_columns_fit(int32_t maxI, int32_t maxJ)
{
    const size_t L = ((size_t)(maxJ < 1 ? 1 : maxJ) * (maxI < 1 ? 1 : maxI) + maxI + maxJ) | 1;
    return L * sizeof(double) <= 220 * 1024;
}

namespace {

// Shared-memory stride of one problem (odd: spreads the teams over the banks).
int tile_stride(int32_t maxI, int32_t maxJ)
{
    const int ld = maxI < 1 ? 1 : maxI, mj = maxJ < 1 ? 1 : maxJ;
    return (mj * ld + ld + mj) | 1;
}

// Threads per block for team size T, or 0 if one block of that team size does not fit.
int threads_for(int T, size_t per)
{
    int threads = kBlock;
    while (threads > T && (size_t)(threads / T) * per > 200 * 1024) threads /= 2;
    return (threads >= 32 && (size_t)(threads / T) * per <= 220 * 1024) ? threads : 0;
}

// Default team size: the smallest team whose 128-thread block fits in ~110 KB (two blocks
// per SM).
int default_team(size_t per)
{
    int T = 1;
    while (T < 32 && (size_t)(kBlock / T) * per > 110 * 1024) T *= 2;
    return T;
}

template <typename R>
int launch_columns(cudaStream_t st, const ColumnProblem &cp, const ColumnBatch &bt, int32_t maxI, int32_t maxJ,
                   int T)
{
    if (T >= kNeTeamBase) {
        const int i = T - kNeTeamBase;
        if (i >= kNumNeShapes || !ne_fits(i, maxI, maxJ, sizeof(R) == 4)) return -1;
        return launch_ne_shape<R>(st, cp, bt, i, maxI, maxJ);
    }
    if (T >= kLaneTeamBase) {
        const int i = T - kLaneTeamBase;
        if (i >= kNumLaneShapes || !lane_fits(i, maxI, maxJ, sizeof(R) == 4)) return -1;
        return launch_lane_shape<R>(st, cp, bt, i, maxI, maxJ);
    }
    if (T >= kRegTeamBase) {
        const int i = T - kRegTeamBase;
        if (i >= kNumRegShapes || !reg_fits(i, maxI, maxJ)) return -1;
        return launch_reg_shape<R>(st, cp, bt, i);
    }
    const int ld = maxI < 1 ? 1 : maxI;
    const int mj = maxJ < 1 ? 1 : maxJ;
    const int L = tile_stride(maxI, maxJ);
    const size_t per = (size_t)L * sizeof(R);
    if (T == 0) T = default_team(per);
    const int threads = threads_for(T, per);
    if (!threads) return -1;
    switch (T) {
    case 1: return launch_team<1, R>(st, cp, bt, ld, mj, L, threads);
    case 2: return launch_team<2, R>(st, cp, bt, ld, mj, L, threads);
    case 4: return launch_team<4, R>(st, cp, bt, ld, mj, L, threads);
    case 8: return launch_team<8, R>(st, cp, bt, ld, mj, L, threads);
    case 16: return launch_team<16, R>(st, cp, bt, ld, mj, L, threads);
    case 32: return launch_team<32, R>(st, cp, bt, ld, mj, L, threads);
    default: return -1;
    }
}

}  // namespace

int launch_spai_columns(cudaStream_t st, const ColumnProblem &cp, int32_t maxI, int32_t maxJ)
{
    if (cp.n <= 0) return 0;
    const ColumnBatch none{};
    return (cp.out_val32 || cp.out_val16) ? launch_columns<float>(st, cp, none, maxI, maxJ, 0)
                                          : launch_columns<double>(st, cp, none, maxI, maxJ, 0);
}

int launch_spai_columns_team(cudaStream_t st, const ColumnProblem &cp, bool low_precision, int32_t maxI,
                             int32_t maxJ, int team)
{
    if (cp.n <= 0) return 0;
    const ColumnBatch none{};
    return low_precision ? launch_columns<float>(st, cp, none, maxI, maxJ, team)
                         : launch_columns<double>(st, cp, none, maxI, maxJ, team);
}

int spai_columns_teams(int32_t maxI, int32_t maxJ, bool low_precision, int *teams)
{
    const size_t per = (size_t)tile_stride(maxI, maxJ) * (low_precision ? sizeof(float) : sizeof(double));
    int k = 0;
    const int def = default_team(per);
    teams[k++] = def;  // the default first
    for (int T = 1; T <= 32; T *= 2)
        if (T != def && threads_for(T, per)) teams[k++] = T;
    for (int i = 0; i < kNumRegShapes; ++i)
        if (reg_fits(i, maxI, maxJ)) teams[k++] = kRegTeamBase + i;
    for (int i = 0; i < kNumLaneShapes; ++i)
        if (lane_fits(i, maxI, maxJ, low_precision)) teams[k++] = kLaneTeamBase + i;
    return k;
}

int spai_columns_ne_teams(int32_t maxI, int32_t maxJ, bool low_precision, int *teams)
{
    int k = 0;
    for (int i = 0; i < kNumNeShapes; ++i)
        if (ne_fits(i, maxI, maxJ, low_precision)) teams[k++] = kNeTeamBase + i;
    return k;
}

int launch_spai_columns_batch(cudaStream_t st, const ColumnBatch &bt, bool low_precision, int32_t maxI,
                              int32_t maxJ, int team)
{
    if (bt.total <= 0) return 0;
    const ColumnProblem none{};
    return low_precision ? launch_columns<float>(st, none, bt, maxI, maxJ, team)
                         : launch_columns<double>(st, none, bt, maxI, maxJ, team);
}

}  // namespace spai

// Column least-squares problems of SPAI and of its update.
//
//   build  (Sec. 2.2):            m_k = argmin_{supp m in J_k} || e_k  - A    m ||_2
//   update (Table 1, Sec. 2.4):   q_k = argmin_{supp q in J_k} || a1_k - A(l) q ||_2
//
// Only the rows I_k = union of rows(A(:,j)), j in J_k, can be nonzero in A m, so each
// problem is the dense |I_k| x |J_k| least-squares problem on Ahat = A(I_k, J_k).
//
// One warp per column.  The warp stages Ahat (column-major, |I_k| rows spread over the
// lanes, row r on lane r % 32) and the right-hand side in shared memory straight from
// A's column-ordered (CSC) arrays, locating every row in I_k by binary search, then runs
// Householder QR with warp-shuffle reductions for the norms and reflector dot products,
// applies each reflector to the right-hand side as it goes, and back-substitutes
// R m = (Q^T rhs)(0:|J_k|) with one unknown per lane.  Results are written straight to
// the row-ordered (CSR) value array of the factor through out_map.
#include <cmath>

#include "spai_internal.cuh"

namespace spai {

namespace {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int bsearch_i32(const int32_t *a, int32_t len, int32_t key)
{
    int32_t lo = 0, hi = len - 1;
    while (lo <= hi) {
        int32_t mid = (lo + hi) >> 1;
        int32_t v = a[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

template <int RPL, int JMAX>
struct Tile {
    static constexpr int IMAX = 32 * RPL;
    static constexpr int kDoubles = JMAX * IMAX + IMAX;  // Ahat + rhs
    static constexpr int kInts = IMAX + JMAX;            // I_k, J_k
    static constexpr size_t bytes_per_warp = kDoubles * sizeof(double) + kInts * sizeof(int32_t);
};

template <int RPL, int JMAX>
__global__ void __launch_bounds__(256) k_spai_columns(ColumnProblem cp)
{
    using T = Tile<RPL, JMAX>;
    constexpr int IMAX = T::IMAX;
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    double *Ah = smem + (size_t)wib * T::kDoubles;
    double *rhs = Ah + JMAX * IMAX;
    int32_t *Iset = reinterpret_cast<int32_t *>(smem + (size_t)wpb * T::kDoubles) + wib * T::kInts;
    int32_t *Jset = Iset + IMAX;

    const int64_t k = (int64_t)blockIdx.x * wpb + wib;
    if (k >= cp.n) return;

    const int32_t ia = cp.Iptr[k], ni = cp.Iptr[k + 1] - ia;
    const int32_t ja = cp.Jptr[k], nj = cp.Jptr[k + 1] - ja;
    if (ni > IMAX || nj > JMAX) {
        if (lane == 0) {
            atomicOr(cp.d_err, ERR_TOO_WIDE);
            cp.col_status[k] = 1;
        }
        return;
    }
    for (int r = lane; r < ni; r += 32) Iset[r] = cp.Ilist[ia + r];
    if (lane < nj) Jset[lane] = cp.Jind[ja + lane];
    for (int e = lane; e < nj * IMAX; e += 32) Ah[e] = 0.0;
#pragma unroll
    for (int u = 0; u < RPL; ++u) rhs[lane + 32 * u] = 0.0;
    __syncwarp();

    // ---- gather Ahat = A(I_k, J_k) and the right-hand side
    for (int c = 0; c < nj; ++c) {
        const int32_t j = Jset[c];
        const int32_t a = __ldg(cp.colptr + j), L = __ldg(cp.colptr + j + 1) - a;
        for (int e = lane; e < L; e += 32) {
            int pos = bsearch_i32(Iset, ni, __ldg(cp.rowind + a + e));
            if (pos >= 0) Ah[c * IMAX + pos] = __ldg(cp.cval + a + e);
        }
    }
    if (cp.mode == 0) {
        if (lane == 0) {
            int pos = bsearch_i32(Iset, ni, (int32_t)k);
            if (pos >= 0) rhs[pos] = 1.0;
        }
    } else {
        const int32_t a = __ldg(cp.r_colptr + k), L = __ldg(cp.r_colptr + k + 1) - a;
        for (int e = lane; e < L; e += 32) {
            int pos = bsearch_i32(Iset, ni, __ldg(cp.r_rowind + a + e));
            if (pos >= 0) rhs[pos] = __ldg(cp.r_val + a + e);
        }
    }
    __syncwarp();

    // ---- Householder QR, reflectors applied to the right-hand side as they are made
    bool singular = ni < nj;
    for (int c = 0; c < nj && !singular; ++c) {
        double v[RPL];
        double ss = 0.0;
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
            const int r = lane + 32 * u;
            v[u] = (r >= c && r < ni) ? Ah[c * IMAX + r] : 0.0;
            ss = fma(v[u], v[u], ss);
        }
        ss = warp_sum(ss);
        const double alpha = sqrt(ss);
        if (alpha == 0.0) {
            singular = true;
            break;
        }
        const double xc = Ah[c * IMAX + c];
        const double sgn = (xc >= 0.0) ? 1.0 : -1.0;
#pragma unroll
        for (int u = 0; u < RPL; ++u)
            if (lane + 32 * u == c) v[u] += sgn * alpha;
        const double vtv = 2.0 * alpha * (alpha + fabs(xc));
        for (int t = c + 1; t <= nj; ++t) {  // t == nj is the right-hand side
            double *col = (t < nj) ? (Ah + t * IMAX) : rhs;
            double d = 0.0;
#pragma unroll
            for (int u = 0; u < RPL; ++u) d = fma(v[u], col[lane + 32 * u], d);
            d = warp_sum(d);
            const double g = 2.0 * d / vtv;
#pragma unroll
            for (int u = 0; u < RPL; ++u) {
                const int r = lane + 32 * u;
                if (r >= c && r < ni) col[r] = fma(-g, v[u], col[r]);
            }
        }
        __syncwarp();
        if (lane == (c & 31)) Ah[c * IMAX + c] = -sgn * alpha;
        __syncwarp();
    }
    if (!singular) {
        double rmax = 0.0;
        for (int c = 0; c < nj; ++c) rmax = fmax(rmax, fabs(Ah[c * IMAX + c]));
        for (int c = 0; c < nj; ++c)
            if (fabs(Ah[c * IMAX + c]) <= 1e-14 * rmax) singular = true;
    }
    if (singular) {
        if (lane < nj) cp.out_val[cp.out_map[ja + lane]] = 0.0;
        if (lane == 0) cp.col_status[k] = 1;
        return;
    }

    // ---- back substitution R m = rhs(0:nj), unknown t on lane t
    double y = (lane < nj) ? rhs[lane] : 0.0;
    for (int c = nj - 1; c >= 0; --c) {
        const double mc = __shfl_sync(0xffffffffu, y, c) / Ah[c * IMAX + c];
        if (lane < c) y = fma(-Ah[c * IMAX + lane], mc, y);
        if (lane == c) y = mc;
    }
    if (lane < nj) cp.out_val[cp.out_map[ja + lane]] = y;
    if (lane == 0) cp.col_status[k] = 0;
}

template <int RPL, int JMAX>
int launch_tile(cudaStream_t st, const ColumnProblem &cp)
{
    using T = Tile<RPL, JMAX>;
    int wpb = (T::bytes_per_warp * 8 <= 200 * 1024) ? 8 : 4;
    size_t smem = T::bytes_per_warp * wpb;
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(k_spai_columns<RPL, JMAX>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return -1;
    }
    int64_t blocks = ((int64_t)cp.n + wpb - 1) / wpb;
    if (blocks < 1) return 0;
    k_spai_columns<RPL, JMAX><<<(unsigned)blocks, wpb * 32, smem, st>>>(cp);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

int launch_spai_columns(cudaStream_t st, const ColumnProblem &cp, int32_t maxI, int32_t maxJ)
{
    if (cp.n <= 0) return 0;
    if (maxJ > 32 || maxI > 128) return -1;
    const int rpl = maxI <= 32 ? 1 : (maxI <= 64 ? 2 : 4);
    const int jm = maxJ <= 8 ? 8 : (maxJ <= 16 ? 16 : 32);
    switch (rpl * 100 + jm) {
    case 108: return launch_tile<1, 8>(st, cp);
    case 116: return launch_tile<1, 16>(st, cp);
    case 132: return launch_tile<1, 32>(st, cp);
    case 208: return launch_tile<2, 8>(st, cp);
    case 216: return launch_tile<2, 16>(st, cp);
    case 232: return launch_tile<2, 32>(st, cp);
    case 408: return launch_tile<4, 8>(st, cp);
    case 416: return launch_tile<4, 16>(st, cp);
    case 432: return launch_tile<4, 32>(st, cp);
    default: return -1;
    }
}

}  // namespace spai

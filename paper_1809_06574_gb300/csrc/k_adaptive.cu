// Adaptive SPAI pattern (the pattern growth of the MSPAI code the paper's experiments use,
// Sec. 3, around the column least squares of Sec. 2.2).
//
// One warp per column k, persistent over the columns.  Starting from J_k = {k}:
//   1. I_k = {k} and the rows of the columns in J_k (a warp-wide merge of the sorted
//      column lists, one list per lane); m = argmin ||e_k - A(I_k, J_k) m||_2 by Householder
//      QR of the tile in shared memory (lanes own rows), back substitution;
//   2. r = e_k - sum_c A(:, J_c) m_c (column by column) on I_k and ||r||^2; stop when
//      ||r||_2 <= eps, after max_steps additions, or on a rank-deficient tile;
//   3. candidates: columns j not in J_k with a nonzero in a row of I_k -- the sorted union
//      of A's CSR rows of I_k (a warp-wide merge, 4 rows per lane), at most 1024;
//      rho_j = ||r||^2 - (r . A(:,j))^2 / ||A(:,j)||^2 for each (A's column in CSC order);
//   4. the <= max_new candidates of smallest rho_j among those not above the candidates'
//      mean, both compared as floor(rho / ||r||^2 * 2^30) (ties: lower column index), join
//      J_k; if |I_k| would then exceed max_rows the step is undone and the growth stops.
// The final J_k (at most kAMJ = 32 columns) goes to out_J[k * 32 ...], its size to
// out_count[k].  The factor values are computed afterwards by the ordinary column kernel
// on the final pattern.  Every loop is bounded by the list sizes; nothing waits.
#include <climits>
#include <cmath>

#include "spai_internal.cuh"

namespace spai {

namespace {

constexpr int kAMJ = 32;     // columns of J_k
constexpr int kAMI = 128;    // rows of I_k
constexpr int kAMC = 1024;   // distinct candidates of one step
constexpr int kKeyBits = 30;

// per-warp shared memory
constexpr int kOffAh = 0;                                  // kAMI x kAMJ doubles; reused for keys
constexpr int kOffRhs = kOffAh + kAMI * kAMJ * 8;          // kAMI doubles
constexpr int kOffR = kOffRhs + kAMI * 8;                  // kAMI doubles
constexpr int kOffM = kOffR + kAMI * 8;                    // kAMJ doubles
constexpr int kOffRd = kOffM + kAMJ * 8;                   // kAMJ doubles
constexpr int kOffJ = kOffRd + kAMJ * 8;                   // kAMJ ints
constexpr int kOffI = kOffJ + kAMJ * 4;                    // kAMI ints
constexpr int kOffNJ = kOffI + kAMI * 4;                   // kAMJ ints (next J)
constexpr int kOffC = kOffNJ + kAMJ * 4;                   // kAMC ints (candidates; next I)
constexpr int kOffCnt = kOffC + kAMC * 4;                  // (spare)
constexpr int kAdaptiveSmem = kOffCnt + 16;
static_assert(kAMI * kAMJ * 8 >= kAMC * 8, "keys fit the tile");

__device__ __forceinline__ int bsearch_list(const int32_t *a, int len, int32_t key)
{
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int32_t v = a[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long warp_min_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long y = __shfl_xor_sync(0xffffffffu, v, o);
        v = y < v ? y : v;
    }
    return v;
}

__device__ __forceinline__ long long adaptive_key(double x, double rr)
{
    double q = floor((x / rr) * (double)(1ll << kKeyBits));
    q = q < 0.0 ? 0.0 : q;
    q = q > (double)(1ll << kKeyBits) ? (double)(1ll << kKeyBits) : q;
    return (long long)q;
}

// rows of the columns J[0..nj) (one sorted CSC list per lane) and {k}, merged into out
// (at most cap entries written); returns the size of the union
__device__ int union_rows(const AdaptiveProblem &ap, const int32_t *J, int nj, int32_t k, int32_t *out, int cap,
                          int lane)
{
    int32_t pos = 0, end = 0, head = INT_MAX;
    if (lane < nj) {
        const int32_t j = J[lane];
        pos = __ldg(ap.colptr + j);
        end = __ldg(ap.colptr + j + 1);
        if (pos < end) head = __ldg(ap.rowind + pos);
    }
    int32_t kx = lane == 0 ? k : INT_MAX;
    int cnt = 0;
    while (true) {
        const int32_t m = __reduce_min_sync(0xffffffffu, min(head, kx));
        if (m == INT_MAX) break;
        if (lane == 0 && cnt < cap) out[cnt] = m;
        ++cnt;
        if (head == m) {
            ++pos;
            head = pos < end ? __ldg(ap.rowind + pos) : INT_MAX;
        }
        if (kx == m) kx = INT_MAX;
    }
    __syncwarp();
    return cnt;
}

__global__ void __launch_bounds__(32) k_adaptive_pattern(AdaptiveProblem ap)
{
    extern __shared__ __align__(16) char sm[];
    double *Ah = reinterpret_cast<double *>(sm + kOffAh);
    long long *keys = reinterpret_cast<long long *>(sm + kOffAh);
    double *rhs = reinterpret_cast<double *>(sm + kOffRhs);
    double *r = reinterpret_cast<double *>(sm + kOffR);
    double *m = reinterpret_cast<double *>(sm + kOffM);
    double *rd = reinterpret_cast<double *>(sm + kOffRd);
    int32_t *Jl = reinterpret_cast<int32_t *>(sm + kOffJ);
    int32_t *Il = reinterpret_cast<int32_t *>(sm + kOffI);
    int32_t *nJl = reinterpret_cast<int32_t *>(sm + kOffNJ);
    int32_t *cand = reinterpret_cast<int32_t *>(sm + kOffC);
    const int lane = threadIdx.x;
    const int max_cols = 1 + ap.max_steps * ap.max_new;

    for (int64_t kk = blockIdx.x; kk < ap.n; kk += gridDim.x) {
        const int32_t k = (int32_t)kk;
        int nj = 1;
        if (lane == 0) Jl[0] = k;
        __syncwarp();
        int ni = union_rows(ap, Jl, nj, k, Il, kAMI, lane);
        if (ni > ap.max_rows) {  // even {k} is too tall: keep it
            if (lane == 0) atomicOr(ap.d_err, ERR_TOO_WIDE);
        }
        for (int step = 0; step <= ap.max_steps && ni <= ap.max_rows; ++step) {
            // ---- tile A(I, J) and e_k
            for (int e = lane; e < nj * kAMI; e += 32) Ah[e] = 0.0;
            for (int i = lane; i < ni; i += 32) rhs[i] = (Il[i] == k) ? 1.0 : 0.0;
            __syncwarp();
            for (int c = 0; c < nj; ++c) {
                const int32_t j = Jl[c];
                const int32_t q1 = __ldg(ap.colptr + j + 1);
                for (int32_t q = __ldg(ap.colptr + j) + lane; q < q1; q += 32) {
                    const int i = bsearch_list(Il, ni, __ldg(ap.rowind + q));
                    if (i >= 0) Ah[c * kAMI + i] = __ldg(ap.cval + q);
                }
            }
            __syncwarp();
            // ---- Householder QR (rows over lanes) applied to e_k as it goes
            bool singular = ni < nj;
            for (int c = 0; c < nj && !singular; ++c) {
                double *vc = Ah + c * kAMI;
                double ss = 0.0;
                for (int i = c + lane; i < ni; i += 32) ss = fma(vc[i], vc[i], ss);
                ss = warp_sum(ss);
                const double alpha = sqrt(ss);
                if (!(alpha > 0.0)) {
                    singular = true;
                    break;
                }
                const double xc = vc[c];
                const double sgn = xc >= 0.0 ? 1.0 : -1.0;
                const double inv = 1.0 / (alpha * (alpha + fabs(xc)));
                __syncwarp();
                if (lane == 0) {
                    vc[c] = xc + sgn * alpha;
                    rd[c] = -sgn * alpha;
                }
                __syncwarp();
                for (int t = c + 1; t <= nj; ++t) {
                    double *col = t < nj ? Ah + t * kAMI : rhs;
                    double d = 0.0;
                    for (int i = c + lane; i < ni; i += 32) d = fma(vc[i], col[i], d);
                    const double g = warp_sum(d) * inv;
                    for (int i = c + lane; i < ni; i += 32) col[i] = fma(-g, vc[i], col[i]);
                }
                __syncwarp();
            }
            if (!singular) {
                double rmax = 0.0;
                for (int c = 0; c < nj; ++c) rmax = fmax(rmax, fabs(rd[c]));
                for (int c = 0; c < nj; ++c)
                    if (fabs(rd[c]) <= 1e-14 * rmax) singular = true;
            }
            if (singular) break;  // J_k stays as it is; the final build reports the column
            for (int c = nj - 1; c >= 0; --c) {  // R m = (Q^T e_k)(0:nj)
                double acc = 0.0;
                for (int t = c + 1 + lane; t < nj; t += 32) acc = fma(Ah[t * kAMI + c], m[t], acc);
                acc = warp_sum(acc);
                if (lane == 0) m[c] = (rhs[c] - acc) / rd[c];
                __syncwarp();
            }
            // ---- residual on I_k, column by column
            for (int i = lane; i < ni; i += 32) r[i] = (Il[i] == k) ? 1.0 : 0.0;
            __syncwarp();
            for (int c = 0; c < nj; ++c) {
                const int32_t j = Jl[c];
                const double mc = m[c];
                const int32_t q1 = __ldg(ap.colptr + j + 1);
                for (int32_t q = __ldg(ap.colptr + j) + lane; q < q1; q += 32) {
                    const int i = bsearch_list(Il, ni, __ldg(ap.rowind + q));
                    if (i >= 0) r[i] = r[i] - __ldg(ap.cval + q) * mc;
                }
                __syncwarp();
            }
            double rr = 0.0;
            for (int i = lane; i < ni; i += 32) rr = fma(r[i], r[i], rr);
            rr = warp_sum(rr);
            if (sqrt(rr) <= ap.eps || step == ap.max_steps || nj >= max_cols || !(rr > 0.0)) break;

            // ---- candidates: the sorted union of A's CSR rows of I_k without J_k (a warp-wide
            // merge of the row lists, 4 rows per lane; each distinct column comes out once)
            int32_t cpos[4], cend[4], chead[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = lane + 32 * u;
                cpos[u] = cend[u] = 0;
                chead[u] = INT_MAX;
                if (i < ni) {
                    const int32_t l = Il[i];
                    cpos[u] = __ldg(ap.rowptr + l);
                    cend[u] = __ldg(ap.rowptr + l + 1);
                    if (cpos[u] < cend[u]) chead[u] = __ldg(ap.colind + cpos[u]);
                }
            }
            int nc = 0;
            while (true) {
                int32_t lo = chead[0];
#pragma unroll
                for (int u = 1; u < 4; ++u) lo = min(lo, chead[u]);
                const int32_t mcol = __reduce_min_sync(0xffffffffu, lo);
                if (mcol == INT_MAX) break;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (chead[u] == mcol) {
                        ++cpos[u];
                        chead[u] = cpos[u] < cend[u] ? __ldg(ap.colind + cpos[u]) : INT_MAX;
                    }
                if (bsearch_list(Jl, nj, mcol) < 0) {
                    if (lane == 0 && nc < kAMC) cand[nc] = mcol;
                    ++nc;
                }
            }
            __syncwarp();
            if (nc > kAMC) {  // more candidates than the buffer holds: stop growing
                if (lane == 0) atomicOr(ap.d_err, ERR_TOO_WIDE);
                break;
            }
            if (nc == 0) break;
            // ---- improvements rho_j, their mean, and the keys (in the tile's space)
            double psum = 0.0;
            for (int e = lane; e < nc; e += 32) {
                const int32_t j = cand[e];
                double dot = 0.0;
                const int32_t q1 = __ldg(ap.colptr + j + 1);
                for (int32_t q = __ldg(ap.colptr + j); q < q1; ++q) {
                    const int i = bsearch_list(Il, ni, __ldg(ap.rowind + q));
                    if (i >= 0) dot = dot + r[i] * __ldg(ap.cval + q);
                }
                const double cn = __ldg(ap.colnorm2 + j);
                const double rho = cn == 0.0 ? rr : rr - dot * dot / cn;
                keys[e] = adaptive_key(rho, rr);
                psum += rho;
            }
            const double mean = warp_sum(psum) / (double)nc;
            const long long kmean = adaptive_key(mean, rr);
            __syncwarp();
            for (int e = lane; e < nc; e += 32)
                keys[e] = keys[e] <= kmean ? ((keys[e] << 32) | (long long)cand[e]) : LLONG_MAX;
            __syncwarp();
            // ---- the max_new smallest (key, column)
            int nsel = 0;
            for (int t = 0; t < ap.max_new && nj + nsel < max_cols; ++t) {
                long long best = LLONG_MAX;
                for (int e = lane; e < nc; e += 32) best = keys[e] < best ? keys[e] : best;
                best = warp_min_ll(best);
                if (best == LLONG_MAX) break;
                const int32_t j = (int32_t)(best & 0xffffffffll);
                for (int e = lane; e < nc; e += 32)
                    if (keys[e] == best) keys[e] = LLONG_MAX;
                if (lane == 0) nJl[kAMJ - 1 - nsel] = j;  // chosen columns, kept at the end
                ++nsel;
                __syncwarp();
            }
            if (nsel == 0) break;
            if (lane == 0) {  // merge J and the chosen columns into nJl[0 .. nj + nsel)
                int32_t ch[kAMJ];
                for (int t = 0; t < nsel; ++t) ch[t] = nJl[kAMJ - 1 - t];
                for (int a = 1; a < nsel; ++a)  // insertion sort of <= 5 values
                    for (int b = a; b > 0 && ch[b - 1] > ch[b]; --b) {
                        const int32_t x = ch[b];
                        ch[b] = ch[b - 1];
                        ch[b - 1] = x;
                    }
                int a = 0, b = 0, o = 0;
                while (a < nj || b < nsel) nJl[o++] = (b >= nsel || (a < nj && Jl[a] < ch[b])) ? Jl[a++] : ch[b++];
            }
            __syncwarp();
            const int nnj = nj + nsel;
            const int nni = union_rows(ap, nJl, nnj, k, cand, kAMI, lane);
            if (nni > ap.max_rows) break;  // the step is undone: J_k, I_k stay
            for (int c = lane; c < nnj; c += 32) Jl[c] = nJl[c];
            for (int i = lane; i < nni; i += 32) Il[i] = cand[i];
            __syncwarp();
            nj = nnj;
            ni = nni;
        }
        for (int c = lane; c < nj; c += 32) ap.out_J[kk * kAMJ + c] = Jl[c];
        if (lane == 0) ap.out_count[kk] = nj;
        __syncwarp();
    }
}

__global__ void k_colnorm2_csc(int32_t n, const int32_t *__restrict__ colptr, const double *__restrict__ cval,
                               double *__restrict__ out)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    double acc = 0.0;
    for (int32_t q = colptr[j]; q < colptr[j + 1]; ++q) acc = acc + cval[q] * cval[q];
    out[j] = acc;
}

__global__ void k_compact_lists(int32_t n, const int32_t *__restrict__ lists, int32_t stride,
                                const int32_t *__restrict__ ptr, int32_t *__restrict__ out)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t a = ptr[k], len = ptr[k + 1] - a;
    for (int32_t c = 0; c < len; ++c) out[a + c] = lists[k * (int64_t)stride + c];
}

}  // namespace

int adaptive_max_cols() { return kAMJ; }
int adaptive_max_rows() { return kAMI; }

int launch_adaptive_pattern(cudaStream_t st, const AdaptiveProblem &ap)
{
    if (ap.n <= 0) return 0;
    if (cudaFuncSetAttribute(k_adaptive_pattern, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdaptiveSmem) !=
        cudaSuccess)
        return -1;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adaptive_pattern, 32, kAdaptiveSmem) != cudaSuccess)
        return -1;
    int64_t blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > ap.n) blocks = ap.n;
    k_adaptive_pattern<<<(unsigned)blocks, 32, kAdaptiveSmem, st>>>(ap);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_colnorm2_csc(cudaStream_t st, int32_t n, const int32_t *colptr, const double *cval, double *out)
{
    if (n <= 0) return 0;
    k_colnorm2_csc<<<(unsigned)(((int64_t)n + 255) / 256), 256, 0, st>>>(n, colptr, cval, out);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_compact_lists(cudaStream_t st, int32_t n, const int32_t *lists, int32_t stride, const int32_t *ptr,
                         int32_t *out)
{
    if (n <= 0) return 0;
    k_compact_lists<<<(unsigned)(((int64_t)n + 255) / 256), 256, 0, st>>>(n, lists, stride, ptr, out);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace spai

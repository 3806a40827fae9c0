// Adaptive SPAI pattern (the pattern growth of the MSPAI code the paper's experiments use,
// Sec. 3, around the column least squares of Sec. 2.2).
//
// One warp per column k, persistent over the columns.  Starting from J_k = {k}:
//   1. I_k = {k} and the rows of the columns in J_k; m = argmin ||e_k - A(I_k, J_k) m||_2
//      by Householder QR of the tile in shared memory (lanes own rows), back substitution.
//      The QR is incremental: tile rows and columns are kept in the order they joined, the
//      columns of earlier steps are zero in the rows added later, so their reflectors stay
//      valid and a step only applies them to the new columns and factors those;
//   2. r = e_k - sum_c A(:, J_c) m_c (column by column) on I_k and ||r||^2; stop when
//      ||r||_2 <= eps, after max_steps additions, or on a rank-deficient tile;
//   3. candidates: columns j not in J_k with a nonzero in a row of I_k -- the sorted union
//      of A's CSR rows of I_k (a warp-wide merge, 4 rows per lane), scored in windows of
//      1024 however many there are; rho_j = ||r||^2 - (r . A(:,j))^2 / ||A(:,j)||^2 for
//      each (A's column in CSC order);
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
constexpr int kAMC = 1024;   // candidates per scoring window
constexpr int kKeyBits = 30;

// per-warp shared memory, sized from the options: ld = max_rows, mc = 1 + max_steps * max_new
//   Ah[ld * mc] tile (tile rows and columns in insertion order), rhs[ld] (Q^T e_k so far),
//   r[ld], m[32], rd[32], invv[32], ck[kAMC + 32] (a window of candidates, then (key << 32) |
//   column, and room for the running list), sel[32] (the smallest (key, column) so far),
//   Jl[32] (J sorted), Jt[32] (tile column -> column), nJl[32] (scratch),
//   It[128] (tile row -> row), Is[128] (rows sorted), Ip[128] (sorted -> tile row), newR[128]
__host__ __device__ constexpr int adaptive_smem(int ld, int mc)
{
    return 8 * (ld * mc + 2 * ld + 3 * kAMJ) + 8 * (kAMC + 2 * kAMJ) + 4 * (3 * kAMJ + 4 * kAMI);
}

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

// tile row of row `row`, or -1
__device__ __forceinline__ int tile_row(const int32_t *Is, const int32_t *Ip, int ni, int32_t row)
{
    const int i = bsearch_list(Is, ni, row);
    return i < 0 ? -1 : Ip[i];
}

// Householder reflector of tile column c over tile rows c .. ni-1 (the QR is incremental:
// columns factored in earlier steps keep their reflectors, stored below the diagonal with
// v's first entry on it, 2 / v^T v in invv[c] and R's diagonal in rd[c]); false if the
// column is zero there.  The caller applies it.
__device__ __forceinline__ bool make_reflector(double *vc, int c, int ni, double *invv, double *rd, int lane)
{
    __syncwarp();  // the column's entries were last written by other lanes
    double ss = 0.0;
    for (int i = c + lane; i < ni; i += 32) ss = fma(vc[i], vc[i], ss);
    ss = warp_sum(ss);
    const double alpha = sqrt(ss);
    if (!(alpha > 0.0)) return false;
    const double xc = vc[c];
    const double sgn = xc >= 0.0 ? 1.0 : -1.0;
    __syncwarp();
    if (lane == 0) {
        vc[c] = xc + sgn * alpha;
        rd[c] = -sgn * alpha;
        invv[c] = 1.0 / (alpha * (alpha + fabs(xc)));
    }
    __syncwarp();
    return true;
}

// col -= (2 v v^T / v^T v) col over tile rows c .. ni-1
__device__ __forceinline__ void apply_reflector(const double *vc, double inv, int c, int ni, double *col, int lane)
{
    double d = 0.0;
    for (int i = c + lane; i < ni; i += 32) d = fma(vc[i], col[i], d);
    const double g = warp_sum(d) * inv;
    for (int i = c + lane; i < ni; i += 32) col[i] = fma(-g, vc[i], col[i]);
}

// gathers column j of A into tile column `col` (rows already zero)
__device__ __forceinline__ void gather_column(const AdaptiveProblem &ap, int32_t j, double *col, const int32_t *Is,
                                              const int32_t *Ip, int ni, int lane)
{
    const int32_t q1 = __ldg(ap.colptr + j + 1);
    for (int32_t q = __ldg(ap.colptr + j) + lane; q < q1; q += 32) {
        const int t = tile_row(Is, Ip, ni, __ldg(ap.rowind + q));
        if (t >= 0) col[t] = __ldg(ap.cval + q);
    }
}

__global__ void __launch_bounds__(32) k_adaptive_pattern(AdaptiveProblem ap)
{
    extern __shared__ __align__(16) char sm[];
    const int ld = ap.max_rows, mc = 1 + ap.max_steps * ap.max_new;
    double *Ah = reinterpret_cast<double *>(sm);
    double *rhs = Ah + ld * mc;
    double *r = rhs + ld;
    double *m = r + ld;
    double *rd = m + kAMJ;
    double *invv = rd + kAMJ;
    long long *ck = reinterpret_cast<long long *>(invv + kAMJ);
    long long *sel = ck + kAMC + kAMJ;
    int32_t *Jl = reinterpret_cast<int32_t *>(sel + kAMJ);
    int32_t *Jt = Jl + kAMJ;
    int32_t *nJl = Jt + kAMJ;
    int32_t *It = nJl + kAMJ;
    int32_t *Is = It + kAMI;
    int32_t *Ip = Is + kAMI;
    int32_t *newR = Ip + kAMI;
    const int lane = threadIdx.x;

    for (int64_t kk = blockIdx.x; kk < ap.n; kk += gridDim.x) {
        const int32_t k = (int32_t)kk;
        int nj = 1, ndone = 0;
        if (lane == 0) Jl[0] = Jt[0] = k;
        __syncwarp();
        int ni = union_rows(ap, Jl, 1, k, Is, kAMI, lane);
        if (ni > ld) {
            // even {k} is taller than max_rows: J_k = {k} (the row limit's rule, not an error)
        } else {
            for (int i = lane; i < ni; i += 32) {
                It[i] = Is[i];
                Ip[i] = i;
                Ah[i] = 0.0;
                rhs[i] = Is[i] == k ? 1.0 : 0.0;
            }
            __syncwarp();
            gather_column(ap, k, Ah, Is, Ip, ni, lane);
            __syncwarp();
        }
        for (int step = 0; step <= ap.max_steps && ni <= ld; ++step) {
            // ---- factor the columns added since the last step: earlier reflectors first
            bool singular = ni < nj;
            for (int c = 0; c < ndone && !singular; ++c)
                for (int t = ndone; t < nj; ++t) apply_reflector(Ah + c * ld, invv[c], c, ni, Ah + t * ld, lane);
            __syncwarp();
            for (int c = ndone; c < nj && !singular; ++c) {
                double *vc = Ah + c * ld;
                if (!make_reflector(vc, c, ni, invv, rd, lane)) {
                    singular = true;
                    break;
                }
                const double inv = invv[c];
                for (int t = c + 1; t < nj; ++t) apply_reflector(vc, inv, c, ni, Ah + t * ld, lane);
                apply_reflector(vc, inv, c, ni, rhs, lane);
                __syncwarp();
            }
            ndone = nj;
            if (!singular) {
                double rmax = 0.0;
                for (int c = 0; c < nj; ++c) rmax = fmax(rmax, fabs(rd[c]));
                for (int c = 0; c < nj; ++c)
                    if (fabs(rd[c]) <= 1e-14 * rmax) singular = true;
            }
            if (singular) break;  // J_k stays as it is; the final build reports the column
            for (int c = nj - 1; c >= 0; --c) {  // R m = (Q^T e_k)(0:nj), tile column order
                double acc = 0.0;
                for (int t = c + 1 + lane; t < nj; t += 32) acc = fma(Ah[t * ld + c], m[t], acc);
                acc = warp_sum(acc);
                if (lane == 0) m[c] = (rhs[c] - acc) / rd[c];
                __syncwarp();
            }
            // ---- residual on I_k (tile rows), column by column
            for (int i = lane; i < ni; i += 32) r[i] = It[i] == k ? 1.0 : 0.0;
            __syncwarp();
            for (int c = 0; c < nj; ++c) {
                const int32_t j = Jt[c];
                const double mcv = m[c];
                const int32_t q1 = __ldg(ap.colptr + j + 1);
                for (int32_t q = __ldg(ap.colptr + j) + lane; q < q1; q += 32) {
                    const int t = tile_row(Is, Ip, ni, __ldg(ap.rowind + q));
                    if (t >= 0) r[t] = r[t] - __ldg(ap.cval + q) * mcv;
                }
                __syncwarp();
            }
            double rr = 0.0;
            for (int i = lane; i < ni; i += 32) rr = fma(r[i], r[i], rr);
            rr = warp_sum(rr);
            if (sqrt(rr) <= ap.eps || step == ap.max_steps || nj >= mc || !(rr > 0.0)) break;

            // ---- candidates: the sorted union of A's CSR rows of I_k without J_k (a warp-wide
            // merge of the row lists, 4 rows per lane; each distinct column comes out once),
            // taken in windows of kAMC.  Each window is scored -- its improvements rho_j summed
            // for the mean, its (key << 32 | column) merged with the running list `sel` of the
            // lim smallest so far.  Taking the lim smallest and then dropping those above the
            // mean's key chooses what filtering by the mean first would: however many
            // candidates there are, all of them are scored, with a buffer of kAMC.
            int32_t cpos[4], cend[4], chead[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = lane + 32 * u;
                cpos[u] = cend[u] = 0;
                chead[u] = INT_MAX;
                if (i < ni) {
                    const int32_t l = It[i];
                    cpos[u] = __ldg(ap.rowptr + l);
                    cend[u] = __ldg(ap.rowptr + l + 1);
                    if (cpos[u] < cend[u]) chead[u] = __ldg(ap.colind + cpos[u]);
                }
            }
            const int lim = min(ap.max_new, mc - nj);
            int jp = 0;       // jp walks the sorted J_k alongside the ascending output
            int nbest = 0;    // sel[0 .. nbest): the smallest (key, column) so far, ascending
            int64_t ncand = 0;
            double psum = 0.0;
            bool more = true;
            while (more) {
                int nw = 0;
                while (true) {
                    int32_t lo = chead[0];
#pragma unroll
                    for (int u = 1; u < 4; ++u) lo = min(lo, chead[u]);
                    const int32_t mcol = __reduce_min_sync(0xffffffffu, lo);
                    if (mcol == INT_MAX) {
                        more = false;
                        break;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (chead[u] == mcol) {
                            ++cpos[u];
                            chead[u] = cpos[u] < cend[u] ? __ldg(ap.colind + cpos[u]) : INT_MAX;
                        }
                    while (jp < nj && Jl[jp] < mcol) ++jp;
                    if (!(jp < nj && Jl[jp] == mcol)) {
                        if (lane == 0) ck[nw] = mcol;
                        if (++nw == kAMC) break;  // window full: score it, then merge on
                    }
                }
                __syncwarp();
                // ---- improvements rho_j of the window and their keys (key << 32 | column)
                for (int e = lane; e < nw; e += 32) {
                    const int32_t j = (int32_t)ck[e];
                    double dot = 0.0;
                    const int32_t q1 = __ldg(ap.colptr + j + 1);
                    for (int32_t q = __ldg(ap.colptr + j); q < q1; ++q) {
                        const int t = tile_row(Is, Ip, ni, __ldg(ap.rowind + q));
                        if (t >= 0) dot = dot + r[t] * __ldg(ap.cval + q);
                    }
                    const double cn = __ldg(ap.colnorm2 + j);
                    const double rho = cn == 0.0 ? rr : rr - dot * dot / cn;
                    ck[e] = (adaptive_key(rho, rr) << 32) | (long long)j;
                    psum += rho;
                }
                ncand += nw;
                // ---- the lim smallest of the window and the running list
                for (int e = lane; e < nbest; e += 32) ck[nw + e] = sel[e];
                __syncwarp();
                const int tot = nw + nbest;
                int ns = 0;
                for (int t = 0; t < lim; ++t) {
                    long long best = LLONG_MAX;
                    for (int e = lane; e < tot; e += 32) best = ck[e] < best ? ck[e] : best;
                    best = warp_min_ll(best);
                    if (best == LLONG_MAX) break;
                    for (int e = lane; e < tot; e += 32)
                        if (ck[e] == best) ck[e] = LLONG_MAX;
                    if (lane == 0) sel[ns] = best;
                    ++ns;
                    __syncwarp();
                }
                nbest = ns;
                __syncwarp();
            }
            if (ncand == 0) break;
            const double mean = warp_sum(psum) / (double)ncand;
            const long long kmean = adaptive_key(mean, rr);
            // ---- the chosen columns: the running list's entries whose key is not above the mean's
            int nsel = 0;
            while (nsel < nbest && (sel[nsel] >> 32) <= kmean) ++nsel;
            if (lane == 0)
                for (int t = 0; t < nsel; ++t) nJl[t] = (int32_t)(sel[t] & 0xffffffffll);
            __syncwarp();
            if (nsel == 0) break;
            // chosen columns ascending (insertion sort of <= 31 values)
            if (lane == 0)
                for (int a = 1; a < nsel; ++a)
                    for (int b = a; b > 0 && nJl[b - 1] > nJl[b]; --b) {
                        const int32_t x = nJl[b];
                        nJl[b] = nJl[b - 1];
                        nJl[b - 1] = x;
                    }
            __syncwarp();
            // ---- rows the chosen columns add (sorted union of their lists, minus I_k)
            int nnew = 0;
            {
                int32_t pos = 0, end = 0, head = INT_MAX;
                if (lane < nsel) {
                    const int32_t j = nJl[lane];
                    pos = __ldg(ap.colptr + j);
                    end = __ldg(ap.colptr + j + 1);
                    if (pos < end) head = __ldg(ap.rowind + pos);
                }
                while (true) {
                    const int32_t mrow = __reduce_min_sync(0xffffffffu, head);
                    if (mrow == INT_MAX) break;
                    if (head == mrow) {
                        ++pos;
                        head = pos < end ? __ldg(ap.rowind + pos) : INT_MAX;
                    }
                    if (bsearch_list(Is, ni, mrow) < 0) {
                        if (lane == 0 && nnew < kAMI) newR[nnew] = mrow;
                        ++nnew;
                    }
                }
                __syncwarp();
            }
            if (ni + nnew > ld) break;  // the step is undone: J_k, I_k stay
            // ---- commit: new rows (appended), new columns (appended), sorted views
            const int nni = ni + nnew;
            for (int i = lane; i < nnew; i += 32) {
                It[ni + i] = newR[i];
                rhs[ni + i] = 0.0;
            }
            for (int c = 0; c < nj; ++c)
                for (int i = ni + lane; i < nni; i += 32) Ah[c * ld + i] = 0.0;
            if (lane == 0) {
                // merge the sorted rows with the sorted new rows, from the end (in place)
                int a = ni - 1, b = nnew - 1, o = nni - 1;
                while (b >= 0) {
                    if (a >= 0 && Is[a] > newR[b]) {
                        Is[o] = Is[a];
                        Ip[o] = Ip[a];
                        --a;
                    } else {
                        Is[o] = newR[b];
                        Ip[o] = ni + b;
                        --b;
                    }
                    --o;
                }
                // J sorted: merge with the chosen columns (from the end); tile columns appended
                a = nj - 1;
                b = nsel - 1;
                o = nj + nsel - 1;
                while (b >= 0) {
                    if (a >= 0 && Jl[a] > nJl[b]) {
                        Jl[o--] = Jl[a--];
                    } else {
                        Jl[o--] = nJl[b--];
                    }
                }
                for (int t = 0; t < nsel; ++t) Jt[nj + t] = nJl[t];
            }
            __syncwarp();
            for (int t = 0; t < nsel; ++t) {
                double *col = Ah + (nj + t) * ld;
                for (int i = lane; i < nni; i += 32) col[i] = 0.0;
                __syncwarp();
                gather_column(ap, nJl[t], col, Is, Ip, nni, lane);
            }
            __syncwarp();
            nj += nsel;
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
    const int mc = 1 + ap.max_steps * ap.max_new;
    if (ap.max_rows < 1 || ap.max_rows > kAMI || mc > kAMJ || ap.max_new < 1 || ap.max_steps < 0) return -1;
    const int smem = adaptive_smem(ap.max_rows, mc);
    if (cudaFuncSetAttribute(k_adaptive_pattern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return -1;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adaptive_pattern, 32, smem) != cudaSuccess)
        return -1;
    int64_t blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > ap.n) blocks = ap.n;
    k_adaptive_pattern<<<(unsigned)blocks, 32, smem, st>>>(ap);
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

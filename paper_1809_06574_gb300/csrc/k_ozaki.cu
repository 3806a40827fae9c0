// FP64-accurate block Gram product H = V_{0..j}^T W on the tensor cores (tcgen05).
//
// The block orthogonalisation of the Krylov basis (block classical Gram-Schmidt inside
// block GMRES, Sec. 2.1) is the one dense contraction of the path: K = n rows, M = (j+1) s
// basis columns, N = s right-hand sides.  GB300's FP64 pipe gives ~1.2 TFLOP/s, so it is
// done here with integer digits on the BF16 tensor cores and FP64 only for the final sum:
//
//  * every value is written in fixed point with 54 bits below 2^1 (V's columns are unit
//    vectors, so |v| <= 1; W's columns are scaled by a power of two 2^-e_b so that
//    |w| < 1) and rounded to nearest: x = sign * sum_p d_p 2^(6(8-p)-53), d_p in [0, 63];
//  * each digit is exact in BF16; a digit product is < 2^12 and a sum of at most 4096 of
//    them is < 2^24, so FP32 accumulation in tensor memory stays exact over a CTA's rows;
//  * digit pairs with p + q <= 9 are kept (53 products); the dropped pairs weigh < 2^-58
//    relative, below FP64 rounding of the same dot products;
//  * the exact FP32 sums are combined in FP64 with their powers of two.
//
// Digits are made once per basis block (when the block is created; it is reused by every
// later Gram product) and once per W, by k_to_digits, and stored in global memory already
// in the MMA's shared-memory layout: for 16-row sub-tile t, digit plane p and block i, one
// 256-byte piece holding the block's 8 columns as 8 rows of two K-major core matrices
// (8 rows x 16 bytes each).  In the Gram kernel one thread streams the pieces of up to 16
// blocks into shared memory with cp.async.bulk (completion counted on an mbarrier), five
// stages deep, while another thread issues, for every V digit plane p, one K=16 MMA
// against all W digit planes q at once (N = 8 * #q, padded to 16) into tensor memory;
// tcgen05.commit frees a stage for the next copy.  Every wait is bounded: on time-out the
// kernel raises an error bit, waits (bounded) for its copies in flight, frees its tensor
// memory and returns.
#include <cstdint>

#include "spai_internal.cuh"

namespace spai {

namespace {

constexpr int kS = 8;              // right-hand-side block width handled here
constexpr int kBlocksPerTile = 16; // basis blocks per CTA: MMA M = 128 columns
constexpr int kM = kS * kBlocksPerTile;
constexpr int kKT = 16;            // rows per sub-tile / digit piece (= MMA K)
constexpr int kDig = 9;            // 6-bit digits per value
constexpr int kPiece = kS * kKT * 2;             // 256 bytes: 8 columns x 16 rows of BF16
constexpr int kLBO = 128;                        // next core matrix along K
constexpr int kSBO = kPiece;                     // next 8-row group (next block / digit)
constexpr int kThreads = 128;
constexpr int kAPlane = kBlocksPerTile * kPiece;            // 4 KB
constexpr int kABytes = kDig * kAPlane;                      // 36 KB
constexpr int kBBytes = (kDig + 1) * kPiece;                 // 9 W digits + a zero row group
constexpr int kStage = kABytes + kBBytes;                    // 39424
constexpr int kStages = 5;
constexpr int kSmemBar = kStages * kStage;                   // full[5], empty[5]
constexpr int kSmemFlag = kSmemBar + 2 * kStages * 8;
constexpr int kSmemTmem = kSmemFlag + 8;
constexpr int kSmemTotal = kSmemTmem + 16;
constexpr int kTmemCols = 512;
constexpr unsigned kWaitLimit = 1u << 22;
constexpr int kMaxRows = 4096;     // exactness bound of the FP32 sums
static_assert(kSmemTotal <= 227 * 1024, "shared memory");

// number of W digits q used with V digit p (q <= min(8, 9 - p)), MMA N (padded to 16)
__host__ __device__ constexpr int nq(int p) { return (9 - p < 8 ? 9 - p : 8) + 1; }
__host__ __device__ constexpr int nmma(int p) { return ((8 * nq(p) + 15) / 16) * 16; }
__host__ __device__ constexpr int tcol(int p)
{
    int c = 0;
    for (int i = 0; i < p; ++i) c += nmma(i);
    return c;
}
static_assert(tcol(8) + nmma(8) <= kTmemCols, "tensor memory columns");
static_assert(nmma(0) <= 8 * (kDig + 1), "B row groups");

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, no swizzle
}

// kind::f16, BF16 x BF16 -> FP32, both operands K-major
__host__ __device__ constexpr uint32_t make_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    unsigned it = 0;
    while (!mbar_try_wait(bar, parity))
        if (++it >= kWaitLimit) return false;
    return true;
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// fixed-point magnitude round(|x| * 2^(53 - e)) from the IEEE bits (integer ops only);
// returns false if |x| * 2^-e >= 2
__device__ __forceinline__ bool fixed_mag(double x, int e, uint64_t &mag, uint32_t &neg)
{
    const uint64_t bits = (uint64_t)__double_as_longlong(x);
    neg = (uint32_t)(bits >> 63);
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0) {  // zero or subnormal: below the fixed-point resolution
        mag = 0;
        return true;
    }
    const uint64_t mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int shift = ex - 1022 - e;  // mag = mant * 2^shift
    if (shift > 1) {
        mag = 0;
        return false;
    }
    if (shift >= 0) {
        mag = mant << shift;
    } else if (shift > -64) {
        const int rs = -shift;
        mag = (mant >> rs) + ((mant >> (rs - 1)) & 1ull);
    } else {
        mag = 0;
    }
    return true;
}

// BF16 bits of the signed digit (sign, d in [0, 63])
__device__ __forceinline__ uint32_t digit_bf16(uint32_t d, uint32_t neg)
{
    const float f = __uint_as_float(0x4B000000u | d) - 8388608.0f;  // exact
    return (__float_as_uint(f) >> 16) | (neg << 15);
}

// Digit pieces of one n x 8 row-major block X (scaled by 2^-exps[a] if exps != null):
// piece (t, p) at dig + ((t * 9 + p) * ipad + iblk) * 256 bytes; rows >= n are zero.
// Thread = (sub-tile t, column a, 8-row group ko).
// If udig != null the same pieces are also written row-tile-major for the update kernel:
// piece (t, p) at udig + ((p * nt8 + t / 8) * ipad + iblk) * 2048 + (t % 8) * 256.
__global__ void k_to_digits(int32_t n, const double *__restrict__ X, const int32_t *__restrict__ exps,
                            char *__restrict__ dig, int32_t ipad, int32_t iblk, int *err,
                            char *__restrict__ udig, int64_t nt8)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    if (g >= nt * kS * (kKT / 8)) return;
    const int a = (int)(g % kS), ko = (int)((g / kS) % (kKT / 8));
    const int64_t t = g / (kS * (kKT / 8));
    const int e = exps ? exps[a] : 0;
    uint64_t mag[8];
    uint32_t neg[8];
    bool bad = false;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int64_t r = t * kKT + ko * 8 + u;
        const double x = (r < n) ? X[r * kS + a] : 0.0;
        if (!fixed_mag(x, e, mag[u], neg[u])) bad = true;
    }
    if (bad) atomicOr(err, ERR_RANGE);
#pragma unroll
    for (int p = 0; p < kDig; ++p) {
        const int sh = 6 * (8 - p);
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t lo = digit_bf16((uint32_t)(mag[2 * u] >> sh) & 63u, neg[2 * u]);
            const uint32_t hi = digit_bf16((uint32_t)(mag[2 * u + 1] >> sh) & 63u, neg[2 * u + 1]);
            w[u] = lo | (hi << 16);
        }
        const uint4 val = make_uint4(w[0], w[1], w[2], w[3]);
        char *dst = dig + ((t * kDig + p) * (int64_t)ipad + iblk) * kPiece + ko * kLBO + a * 16;
        *reinterpret_cast<uint4 *>(dst) = val;
        if (udig) {
            char *u = udig + ((p * nt8 + t / 8) * (int64_t)ipad + iblk) * (8 * kPiece) + (t % 8) * kPiece + ko * kLBO +
                      a * 16;
            *reinterpret_cast<uint4 *>(u) = val;
        }
    }
}

__device__ __forceinline__ void drain_row(uint32_t tmem, int warp, int S[10][kS]);
__device__ __forceinline__ double combine_scaled(const int S[10][kS], int b, int e);

// Gram product from digit pieces.  grid = (row chunks, M tiles of 16 blocks); a chunk is
// a whole number of 16-row sub-tiles, at most 4096 rows.  Thread 0 copies, thread 32
// issues MMAs, warps 0..3 drain tensor memory.
__global__ void __launch_bounds__(kThreads, 1)
    k_block_dot_tc(int32_t n, int32_t nblk, int32_t subs_per_chunk, const char *__restrict__ vdig, int32_t ipad,
                   const char *__restrict__ wdig, const int32_t *__restrict__ wexp, double *__restrict__ partial,
                   int *err)
{
    extern __shared__ __align__(128) char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chunk = blockIdx.x, mt = blockIdx.y;
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    const int64_t t0 = (int64_t)chunk * subs_per_chunk;
    const int nsub = (int)min((int64_t)subs_per_chunk, nt - t0);
    const int blk0 = mt * kBlocksPerTile;
    const int nvb = min(kBlocksPerTile, nblk - blk0);  // valid blocks in this tile
    const uint32_t full0 = smem_u32(smem + kSmemBar), empty0 = full0 + kStages * 8;
    volatile int *flag = reinterpret_cast<volatile int *>(smem + kSmemFlag);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kSmemTmem);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * s));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * s));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        *flag = 0;
    }
    // zero row group 9 of every B stage (MMAs with N = 80 read it; copies never write it)
    for (int e = tid; e < kStages * (kPiece / 16); e += kThreads) {
        const int s = e / (kPiece / 16), o = e % (kPiece / 16);
        *reinterpret_cast<uint4 *>(smem + s * kStage + kABytes + kDig * kPiece + o * 16) = make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const bool work = nvb > 0 && nsub > 0;

    if (tid == 0 && work) {  // ---- producer: bulk copies of sub-tile u into stage u % kStages
        const uint32_t abytes = (uint32_t)nvb * kPiece;
        const uint32_t stage_bytes = kDig * abytes + kDig * kPiece;
        int issued = 0;
        for (int u = 0; u < nsub; ++u) {
            const int s = u % kStages;
            if (u >= kStages && !mbar_wait_bounded(empty0 + 8 * s, (uint32_t)(((u - kStages) / kStages) & 1))) {
                *flag = 1;
                break;
            }
            if (*flag) break;
            const uint32_t fb = full0 + 8 * s;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(stage_bytes)
                         : "memory");
            const int64_t t = t0 + u;
            char *st = smem + s * kStage;
#pragma unroll 1
            for (int p = 0; p < kDig; ++p)
                bulk_copy(smem_u32(st + p * kAPlane), vdig + ((t * kDig + p) * (int64_t)ipad + blk0) * kPiece,
                          abytes, fb);
            bulk_copy(smem_u32(st + kABytes), wdig + t * kDig * kPiece, kDig * kPiece, fb);
            issued = u + 1;
        }
        // every copy issued must have landed before shared memory is released
        for (int u = issued - kStages < 0 ? 0 : issued - kStages; u < issued; ++u)
            if (!mbar_wait_bounded(full0 + 8 * (u % kStages), (uint32_t)((u / kStages) & 1))) *flag = 1;
    } else if (tid == 32 && work) {  // ---- MMA issuer
        int done = 0;
        for (int u = 0; u < nsub; ++u) {
            const int s = u % kStages;
            if (!mbar_wait_bounded(full0 + 8 * s, (uint32_t)((u / kStages) & 1))) {
                *flag = 1;
                break;
            }
            if (*flag) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const char *st = smem + s * kStage;
#pragma unroll
            for (int p = 0; p < kDig; ++p) {
                const uint64_t da = make_desc(smem_u32(st + p * kAPlane));
                const uint64_t db = make_desc(smem_u32(st + kABytes));
                mma_bf16(tmem + tcol(p), da, db, make_idesc(kM, nmma(p)), u > 0 ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             empty0 + 8 * s)
                         : "memory");
            done = u + 1;
        }
        // the last commit: all MMAs done before tensor memory is read
        if (done > 0) {
            const int u = done - 1;
            if (!mbar_wait_bounded(empty0 + 8 * (u % kStages), (uint32_t)((u / kStages) & 1))) *flag = 1;
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const bool failed = *flag != 0;
    if (failed && tid == 0) atomicOr(err, ERR_TIMEOUT);

    // ---- drain: warp w owns tensor-memory lanes 32w..32w+31 = basis columns
    if (!failed && work) {
        const int m = warp * 32 + lane;
        int S[10][kS];
        drain_row(tmem, warp, S);
        if (m < nvb * kS) {
            const int gm = blk0 * kS + m;
            double *dst = partial + ((int64_t)chunk * nblk + (gm >> 3)) * (kS * kS) + (gm & 7) * kS;
#pragma unroll
            for (int b = 0; b < kS; ++b) dst[b] = combine_scaled(S, b, wexp[b]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// per-column max |W| (bit patterns of non-negative doubles order like the values):
// warp and block reductions, then one atomicMax per column per block
__global__ void k_col_maxabs(int32_t n, const double *__restrict__ W, unsigned long long *scratch)
{
    __shared__ unsigned long long red[kS][32];
    unsigned long long m[kS];
#pragma unroll
    for (int b = 0; b < kS; ++b) m[b] = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const double2 *row = reinterpret_cast<const double2 *>(W + r * kS);
#pragma unroll
        for (int h = 0; h < kS / 2; ++h) {
            const double2 x = row[h];
            const unsigned long long b0 = (unsigned long long)__double_as_longlong(fabs(x.x));
            const unsigned long long b1 = (unsigned long long)__double_as_longlong(fabs(x.y));
            m[2 * h] = b0 > m[2 * h] ? b0 : m[2 * h];
            m[2 * h + 1] = b1 > m[2 * h + 1] ? b1 : m[2 * h + 1];
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int b = 0; b < kS; ++b) {
        unsigned long long v = m[b];
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, v, o);
            v = y > v ? y : v;
        }
        if (lane == 0) red[b][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kS) {
        unsigned long long v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = red[threadIdx.x][w] > v ? red[threadIdx.x][w] : v;
        if (v) atomicMax(scratch + threadIdx.x, v);
    }
}

__global__ void k_maxexp_finish(unsigned long long *scratch, int32_t *exps)
{
    const int b = threadIdx.x;
    if (b >= kS) return;
    const unsigned long long bits = scratch[b];
    const int ex = (int)((bits >> 52) & 0x7FF);
    exps[b] = ex == 0 ? 0 : ex - 1022;  // |w| < 2^(ex - 1022) for a normal number
    scratch[b] = 0;                      // ready for the next use
}

// ---------------------------------------------------------------------------------
// Block update out = base - sign' * V_{0..nblk-1} H on the tensor cores (W -= V H of the
// Gram-Schmidt passes, U = V Y of the solution update), same digit scheme.  The MMA's M
// dimension is 128 rows of V, K runs over basis columns (16 = two blocks per MMA), N over
// H's digit planes x 8 columns.  V's pieces are read MN-major (8 basis columns x 8
// contiguous rows per core matrix) from their row-tile-major copy; H's digits are built
// per call by k_h_digits as K-major pieces, one 2304-byte group per 16 basis columns.
// ---------------------------------------------------------------------------------
constexpr int kUStageA = kDig * 2 * (8 * kPiece);          // 9 planes x 2 blocks x 2 KB
constexpr int kUStage = kUStageA + kBBytes;                  // + 9 H digit pieces + zero group
constexpr int kUSmemBar = kStages * kUStage;
constexpr int kUSmemFlag = kUSmemBar + 2 * kStages * 8;
constexpr int kUSmemTmem = kUSmemFlag + 8;
constexpr int kUSmemTotal = kUSmemTmem + 16;
static_assert(kUSmemTotal <= 227 * 1024, "shared memory");
constexpr int kULBO = 8 * kPiece;  // MN-major: next 8 basis columns (next block)
constexpr int kUSBO = 128;         // MN-major: next 8 rows

__device__ __forceinline__ uint64_t make_desc_mn(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((kULBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((kUSBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// A (V) MN-major, B (H digits) K-major
__host__ __device__ constexpr uint32_t make_idesc_amn(int M, int N) { return make_idesc(M, N) | (1u << 15); }

// exact FP32 integer (|x| < 2^24) to int
__device__ __forceinline__ int f2i_exact(uint32_t bits) { return __float2int_rz(__uint_as_float(bits)); }

// Digits of H (nblk*8 basis columns x 8, H[c * 8 + b]) scaled per column b: piece (kappa, q)
// at hdig + (kappa * 9 + q) * 256 holds columns 16 kappa .. 16 kappa + 15 (zero beyond
// nblk * 8); hexp[b] = column exponent.  One CTA.
__global__ void k_h_digits(int32_t nblk, const double *__restrict__ H, char *__restrict__ hdig,
                           int32_t *__restrict__ hexp, int *err)
{
    __shared__ int32_t ex_s[kS];
    const int ncol = nblk * kS;
    if (threadIdx.x < kS) {
        unsigned long long m = 0;
        for (int c = 0; c < ncol; ++c) {
            const unsigned long long bits = (unsigned long long)__double_as_longlong(fabs(H[c * kS + threadIdx.x]));
            m = bits > m ? bits : m;
        }
        const int ex = (int)((m >> 52) & 0x7FF);
        ex_s[threadIdx.x] = ex == 0 ? 0 : ex - 1022;
        hexp[threadIdx.x] = ex_s[threadIdx.x];
    }
    __syncthreads();
    const int nk = (nblk + 1) / 2;
    for (int item = threadIdx.x; item < nk * kS * 2; item += blockDim.x) {
        const int b = item % kS, ko = (item / kS) % 2, kappa = item / (2 * kS);
        uint64_t mag[8];
        uint32_t neg[8];
        bool bad = false;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = kappa * 16 + ko * 8 + u;
            const double x = c < ncol ? H[c * kS + b] : 0.0;
            if (!fixed_mag(x, ex_s[b], mag[u], neg[u])) bad = true;
        }
        if (bad) atomicOr(err, ERR_RANGE);
#pragma unroll
        for (int q = 0; q < kDig; ++q) {
            const int sh = 6 * (8 - q);
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t lo = digit_bf16((uint32_t)(mag[2 * u] >> sh) & 63u, neg[2 * u]);
                const uint32_t hi = digit_bf16((uint32_t)(mag[2 * u + 1] >> sh) & 63u, neg[2 * u + 1]);
                w[u] = lo | (hi << 16);
            }
            *reinterpret_cast<uint4 *>(hdig + (kappa * kDig + q) * kPiece + ko * kLBO + b * 16) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Sum of the digit products of tensor-memory row `lane` for output column b:
// sum_{p,q} D_p[q*8+b] 2^(-10-6(p+q)).  Products of equal weight are added as integers
// (|D| < 2^24), three weights are merged in 64-bit integers, four FP64 terms remain.
__device__ __forceinline__ void combine_row(const int S[10][kS], double out[kS])
{
#pragma unroll
    for (int b = 0; b < kS; ++b) {
        const long long g0 = ((long long)S[0][b] << 12) + ((long long)S[1][b] << 6) + S[2][b];
        const long long g1 = ((long long)S[3][b] << 12) + ((long long)S[4][b] << 6) + S[5][b];
        const long long g2 = ((long long)S[6][b] << 12) + ((long long)S[7][b] << 6) + S[8][b];
        const long long g3 = S[9][b];
        double v = (double)g3 * 0x1p-64;
        v = fma((double)g2, 0x1p-58, v);
        v = fma((double)g1, 0x1p-40, v);
        v = fma((double)g0, 0x1p-22, v);
        out[b] = v;
    }
}

// read all digit-product columns of this thread's tensor-memory row, grouped by p + q
__device__ __forceinline__ void drain_row(uint32_t tmem, int warp, int S[10][kS])
{
#pragma unroll
    for (int s = 0; s < 10; ++s)
#pragma unroll
        for (int b = 0; b < kS; ++b) S[s][b] = 0;
#pragma unroll
    for (int p = 0; p < kDig; ++p) {
#pragma unroll
        for (int c0 = 0; c0 < nmma(p); c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(tcol(p) + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int q = (c0 + c) >> 3, b = (c0 + c) & 7;
                if (q < nq(p)) S[p + q][b] += f2i_exact(v[c]);
            }
        }
    }
}


// Value of row `lane`'s digit products for output column b times 2^e_b, from the
// equal-weight integer sums S[p+q][b] (|S| < 2^28): two 64-bit integers carry
// S_0..S_4 (weights 2^-10..2^-34 -> hi * 2^-34) and S_5..S_9 (2^-40..2^-64 -> lo * 2^-64),
// each converted once; the power-of-two scale is added to the exponent fields.
__device__ __forceinline__ double combine_scaled(const int S[10][kS], int b, int e)
{
    long long hi = S[0][b];
#pragma unroll
    for (int s = 1; s < 5; ++s) hi = (hi << 6) + S[s][b];
    long long lo = S[5][b];
#pragma unroll
    for (int s = 6; s < 10; ++s) lo = (lo << 6) + S[s][b];
    // |hi|, |lo| < 2^53: exact conversions; 2^e is a normal double for the exponents of
    // finite nonzero columns (e >= -1021), and a zero column has e = 0
    const double v = fma((double)hi, 0x1p-34, (double)lo * 0x1p-64);
    return v * __longlong_as_double((long long)(1023 + e) << 52);
}

// Update drain: |D| < 2^22 here (K <= 1024 columns), so a D value's integer is read by
// adding 1.5 * 2^23 in FP32 (exact) instead of a conversion instruction.
__device__ __forceinline__ void drain_row_small(uint32_t tmem, int quarter, int S[10][kS])
{
#pragma unroll
    for (int s = 0; s < 10; ++s)
#pragma unroll
        for (int b = 0; b < kS; ++b) S[s][b] = 0;
#pragma unroll
    for (int p = 0; p < kDig; ++p) {
#pragma unroll
        for (int c0 = 0; c0 < nmma(p); c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tcol(p) + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int q = (c0 + c) >> 3, b = (c0 + c) & 7;
                if (q < nq(p))
                    S[p + q][b] += __float_as_int(__uint_as_float(v[c]) + 12582912.0f) - 0x4B400000;
            }
        }
    }
}

constexpr int kUThreads = 192;  // warp 0 copies, warp 1 issues MMAs, warps 2..5 drain

// Persistent block update: out[r][b] = base[r][b] + sign * (V H)[r][b] (base == null:
// sign * V H).  One CTA per SM walks 128-row tiles; the copy warp streams stages ahead
// across tiles, the MMA warp waits for the drain warps to hand tensor memory back before
// starting the next tile.
__global__ void __launch_bounds__(kUThreads, 1)
    k_block_update_tc(int32_t n, int32_t nblk, const char *__restrict__ udig, int32_t ipad, int64_t nt8,
                      const char *__restrict__ hdig, const int32_t *__restrict__ hexp, const char *__restrict__ zeros,
                      const double *base, double *out, double sign, int *err)
{
    extern __shared__ __align__(128) char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nk = (nblk + 1) / 2;  // K steps of 16 basis columns
    const int64_t ntiles = nt8;
    const uint32_t full0 = smem_u32(smem + kUSmemBar), empty0 = full0 + kStages * 8;
    const uint32_t tdone = smem_u32(smem + kUSmemFlag + 16), tfree = tdone + 8;
    volatile int *flag = reinterpret_cast<volatile int *>(smem + kUSmemFlag);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kUSmemTmem);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * s));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * s));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tdone));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(tfree));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *flag = 0;
    }
    for (int e = tid; e < kStages * (kPiece / 16); e += kUThreads) {
        const int s = e / (kPiece / 16), o = e % (kPiece / 16);
        *reinterpret_cast<uint4 *>(smem + s * kUStage + kUStageA + kDig * kPiece + o * 16) = make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // ---- copy thread
            int64_t g = 0, issued = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && !*flag; tile += gridDim.x) {
                for (int kk = 0; kk < nk; ++kk, ++g) {
                    const int s = (int)(g % kStages);
                    if (g >= kStages &&
                        !mbar_wait_bounded(empty0 + 8 * s, (uint32_t)(((g - kStages) / kStages) & 1))) {
                        *flag = 1;
                        break;
                    }
                    const int nbk = min(2, nblk - 2 * kk);
                    const uint32_t fb = full0 + 8 * s;
                    const uint32_t bytes = kDig * 2 * (8 * kPiece) + kDig * kPiece;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(bytes)
                                 : "memory");
                    char *st = smem + s * kUStage;
#pragma unroll 1
                    for (int p = 0; p < kDig; ++p) {
                        const char *src = udig + ((p * nt8 + tile) * (int64_t)ipad + 2 * kk) * (8 * kPiece);
                        bulk_copy(smem_u32(st + p * 2 * (8 * kPiece)), src, (uint32_t)nbk * 8 * kPiece, fb);
                        if (nbk == 1)  // second block slot of an odd tail: zeros (its H digits are zero)
                            bulk_copy(smem_u32(st + p * 2 * (8 * kPiece) + 8 * kPiece), zeros, 8 * kPiece, fb);
                    }
                    bulk_copy(smem_u32(st + kUStageA), hdig + (int64_t)kk * kDig * kPiece, kDig * kPiece, fb);
                    issued = g + 1;
                }
            }
            // copies in flight must land before shared memory is released
            for (int64_t u = issued - kStages < 0 ? 0 : issued - kStages; u < issued; ++u)
                if (!mbar_wait_bounded(full0 + 8 * (int)(u % kStages), (uint32_t)((u / kStages) & 1))) *flag = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA thread
            int64_t g = 0, t = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && !*flag; tile += gridDim.x, ++t) {
                if (t > 0 && !mbar_wait_bounded(tfree, (uint32_t)((t - 1) & 1))) {
                    *flag = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                bool ok = true;
                for (int kk = 0; kk < nk; ++kk, ++g) {
                    const int s = (int)(g % kStages);
                    if (!mbar_wait_bounded(full0 + 8 * s, (uint32_t)((g / kStages) & 1))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const char *st = smem + s * kUStage;
#pragma unroll
                    for (int p = 0; p < kDig; ++p) {
                        const uint64_t da = make_desc_mn(smem_u32(st + p * 2 * (8 * kPiece)));
                        const uint64_t db = make_desc(smem_u32(st + kUStageA));
                        mma_bf16(tmem + tcol(p), da, db, make_idesc_amn(kM, nmma(p)), kk > 0 ? 1u : 0u);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     empty0 + 8 * s)
                                 : "memory");
                }
                if (!ok) {
                    *flag = 1;
                    break;
                }
                // tile finished: the drain warps may read tensor memory
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 tdone)
                             : "memory");
            }
        }
    } else {  // ---- drain warps 2..5: tensor-memory lane quarter = warp % 4
        const int quarter = warp & 3;
        int64_t t = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++t) {
            if (!mbar_wait_bounded(tdone, (uint32_t)(t & 1)) || *flag) {
                *flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            int S[10][kS];
            drain_row_small(tmem, quarter, S);
            asm volatile("tcgen05.fence::before_thread_sync;");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tfree) : "memory");
            const int64_t r = tile * 128 + quarter * 32 + lane;
            if (r < n) {
#pragma unroll
                for (int b = 0; b < kS; ++b) {
                    const double vh = combine_scaled(S, b, hexp[b]);
                    out[r * kS + b] = base ? fma(sign, vh, base[r * kS + b]) : sign * vh;
                }
            }
        }
    }
    __syncthreads();
    if (*flag && tid == 0) atomicOr(err, ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

}  // namespace

bool block_dot_tc_supported(int32_t s) { return s == kS; }

size_t tc_digit_bytes(int32_t n, int32_t nblocks)
{
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    return (size_t)nt * kDig * (size_t)nblocks * kPiece;
}

size_t tc_scratch_bytes() { return 256; }

int launch_to_digits(cudaStream_t st, int32_t n, const double *X, const int32_t *exps, void *dig, int32_t ipad,
                     int32_t iblk, int *d_err, void *udig)
{
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    const int64_t work = nt * kS * (kKT / 8);
    k_to_digits<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(n, X, exps, (char *)dig, ipad, iblk, d_err,
                                                                  (char *)udig, (nt + 7) / 8);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_w_digits(cudaStream_t st, int32_t n, const double *W, void *wdig, void *scratch, int *d_err)
{
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(scratch);
    int32_t *exps = reinterpret_cast<int32_t *>(mx + kS);
    int g = (int)(((int64_t)n + 255) / 256);
    if (g > 2 * 152) g = 2 * 152;
    k_col_maxabs<<<g, 256, 0, st>>>(n, W, mx);
    k_maxexp_finish<<<1, 32, 0, st>>>(mx, exps);
    note_launches(2);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return launch_to_digits(st, n, W, exps, wdig, 1, 0, d_err, nullptr);
}

int tc_subs_per_chunk(int32_t n, int32_t nblk)
{
    const int mtiles = (nblk + kBlocksPerTile - 1) / kBlocksPerTile;
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    int64_t want = (nt * mtiles + 152 - 1) / 152;  // ~1 CTA per SM in total
    if (want < 8) want = 8;
    if (want > kMaxRows / kKT) want = kMaxRows / kKT;
    return (int)want;
}

size_t tc_udig_bytes(int32_t n, int32_t nblocks)
{
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    return (size_t)((nt + 7) / 8) * kDig * (size_t)nblocks * (8 * kPiece);
}

size_t tc_hdig_bytes(int32_t nblk) { return (size_t)((nblk + 1) / 2) * kDig * kPiece; }

int block_update_tc_max_blocks() { return 1024 / kS; }

// the whole shared memory of an SM: every descriptor reading stays inside the allocation
constexpr int kUSmemAlloc = 227 * 1024;
static_assert(kUSmemAlloc >= kUSmemTotal, "update kernel shared memory");

int launch_block_update_tc(cudaStream_t st, int32_t n, int32_t nblk, const void *udig, int32_t ipad,
                           const double *H, void *hdig, int32_t *hexp, const void *zeros, const double *base,
                           double *out, double sign, int *d_err)
{
    // the drain reads the FP32 sums as integers below 2^22: at most 1024 basis columns
    if (n <= 0 || nblk <= 0 || nblk > block_update_tc_max_blocks()) return -1;
    k_h_digits<<<1, 256, 0, st>>>(nblk, H, (char *)hdig, hexp, d_err);
    note_launches(1);
    if (cudaFuncSetAttribute(k_block_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kUSmemAlloc) !=
        cudaSuccess)
        return -1;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    const int64_t tiles = (nt + 7) / 8;
    const int grid = (int)(tiles < sms ? tiles : sms);
    k_block_update_tc<<<grid, kUThreads, kUSmemAlloc, st>>>(n, nblk, (const char *)udig, ipad, (nt + 7) / 8,
                                                             (const char *)hdig, hexp, (const char *)zeros, base, out,
                                                             sign, d_err);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

size_t tc_partial_elems(int32_t n, int32_t nblk)
{
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    return (size_t)((nt + 7) / 8) * nblk * kS * kS;  // chunks hold at least 8 sub-tiles
}

int launch_block_dot_tc(cudaStream_t st, int32_t n, int32_t nblk, const void *vdig, int32_t ipad, const void *wdig,
                        const void *scratch, double *partial, double *out, int *d_err)
{
    if (n <= 0 || nblk <= 0) return -1;
    if (cudaFuncSetAttribute(k_block_dot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal) != cudaSuccess)
        return -1;
    const int32_t *exps = reinterpret_cast<const int32_t *>(reinterpret_cast<const unsigned long long *>(scratch) + kS);
    const int spc = tc_subs_per_chunk(n, nblk);
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    const int chunks = (int)((nt + spc - 1) / spc);
    const int mtiles = (nblk + kBlocksPerTile - 1) / kBlocksPerTile;
    dim3 grid(chunks, mtiles);
    k_block_dot_tc<<<grid, kThreads, kSmemTotal, st>>>(n, nblk, spc, (const char *)vdig, ipad, (const char *)wdig,
                                                         exps, partial, d_err);
    note_launches(1);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return launch_reduce_chunks(st, nblk * kS * kS, chunks, partial, out);
}

}  // namespace spai

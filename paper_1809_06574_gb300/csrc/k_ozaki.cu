// FP64-accurate block Gram product H = V_{0..j}^T W and block update W -= V H on the
// tensor cores (tcgen05).
//
// The block orthogonalisation of the Krylov basis (block classical Gram-Schmidt inside
// block GMRES, Sec. 2.1) is the one dense contraction of the path: K = n rows, M = (j+1) s
// basis columns, N = s right-hand sides.  GB300's FP64 pipe gives ~1.2 TFLOP/s, so it is
// done here with integer digits on the BF16 tensor cores and FP64 only for the final sum:
//
//  * every value is written in fixed point with resolution 2^-54 (V's columns are unit
//    vectors, so |v| <= 1; W's columns are scaled by a power of two 2^-e_b so that
//    |w| < 1): m = round(x 2^54), and m in balanced base 128, m = sum_p d_p 128^(7-p) with
//    eight digits d_p in [-64, 63] (p = 0 the most significant);
//  * each digit is exact in BF16; the products of digits p and q are accumulated in FP32
//    in tensor memory by weight class c = p + q (the MMA for digit p writes its products
//    with W digit q into the columns of class p + q); a class collects at most 8 products
//    of at most 64^2 per row, so sums over at most 512 rows stay within 2^24 and exact;
//  * digit pairs with p + q <= 8 are kept (43 products); the dropped pairs weigh < 2^-61
//    relative to the largest entries per row, below FP64 rounding of the same dot products;
//  * every <= 512 rows (a segment) four drain warps read the exact class sums out of tensor
//    memory into two exact 64-bit integers per output, hi = sum_{c<=4} S_c 128^(4-c) and
//    lo = sum_{5<=c<=8} S_c 128^(8-c), and at the end combine them in FP64 with the scale.
//    Four accumulator buffers of 128 columns let the MMAs of the next segment run while a
//    segment is drained.
//
// Every basis block is kept, besides its FP64 copy, as its eight digit bytes (byte i holds
// d + 64 of the digit of weight 128^i: 8 bytes per value, the same traffic as FP64, made
// once by the kernel that creates the block); W is read as FP64 and scaled per CTA.  Both
// kernels stream these 8-byte values and cut the digits in shared memory with byte
// permutes: one thread issues cp.async.bulk copies of raw row tiles into a ring of stages
// (completion counted on mbarriers), eight converter warps turn each raw stage into eight
// BF16 digit planes laid out as the MMA's shared-memory operand (a second ring), one
// thread issues the tcgen05.mma of every stage and frees the digit stage with
// tcgen05.commit.  Every wait is bounded in time (1 s): on time-out the kernel raises an
// error bit, waits (bounded) for its copies in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include "spai_internal.cuh"

namespace spai {

namespace {

constexpr int kS = 8;              // right-hand-side block width handled here
constexpr int kBlocksPerTile = 16; // basis blocks per Gram CTA: MMA M = 128 columns
constexpr int kM = kS * kBlocksPerTile;
constexpr int kKT = 16;            // rows per sub-tile / digit piece (= MMA K)
constexpr int kDig = 8;            // balanced base-128 digits per value
constexpr int kPiece = kS * kKT * 2;             // 256 bytes: 8 columns x 16 rows of BF16
constexpr int kLBO = 128;                        // next core matrix along K
constexpr int kSBO = kPiece;                     // next 8-row group (next block / digit)
constexpr int kTmemCols = 512;
constexpr int kBufCols = 128;      // one class accumulator: classes 0..10 x 8 columns
constexpr int kBufs = kTmemCols / kBufCols;
constexpr int kClsCols = 80;       // classes 0..9 are read (class 9 only collects padding products)
constexpr int kSegK = 512;         // rows (Gram) / basis columns (update) per accumulation
constexpr int kMaxRows = 4096;     // rows per Gram CTA: hi, lo stay below 2^53
constexpr int kCW = 8;             // converter warps
constexpr int kCT = 32 * kCW;      // converter threads
constexpr int kCG = 2;             // Gram kernel: converter groups taking alternate stages
constexpr int kCTG = kCT / kCG;    // threads of one converter group
constexpr int kThreadsTC = 64 + 128 + kCT;  // copy warp, MMA warp, 4 drain warps, converters
constexpr int kRawRow = kS * 8;    // 64 bytes: one row of an n x 8 block
constexpr unsigned long long kWaitNs = 1000000000ull;  // drain waits give up after 1 s
#ifndef SPAI_TC_SUSPEND_NS
#define SPAI_TC_SUSPEND_NS 20000
#endif
constexpr unsigned kSuspendNs = SPAI_TC_SUSPEND_NS;     // suspend hint of one try_wait
static_assert(8 * 64 * 64 * kSegK <= (1 << 24), "exact FP32 class sums");
static_assert(kClsCols == 5 * 16, "drain_classes reads five 16-column groups");

// number of W digits q used with V digit p (p + q <= 8, q <= 7), MMA N (padded to 16: the
// padding products land in class 9, which is never read).  The MMA of digit 0 opens each
// segment (accumulate off), so it spans all 80 class columns: the W digit planes are
// followed by two zero groups, and its products with them clear classes 8 and 9.
__host__ __device__ constexpr int nq(int p) { return 9 - p < 8 ? 9 - p : 8; }
__host__ __device__ constexpr int nmma(int p) { return p == 0 ? kClsCols : ((8 * nq(p) + 15) / 16) * 16; }
constexpr int kBGroups = kDig + 2;  // B operand row groups: the digit planes and two zero groups
__host__ __device__ constexpr bool classes_fit()
{
    for (int p = 0; p < kDig; ++p)
        if (8 * p + nmma(p) > kClsCols || nmma(p) > 8 * kBGroups) return false;
    return true;
}
static_assert(classes_fit(), "class columns and B row groups");

// ---- Gram kernel shared memory: raw ring | digit ring | slack | ... | barriers, flag, tmem, exps,
// maxima at the end of the allocation.  The ring depths follow the tile's block count: a
// stage carries S sub-tiles (<= kDDigStage / kDRawStage bytes), three digit stages, and as
// many raw stages (up to 8) as the rest holds, so that the copies run well ahead.
constexpr int kDRawStage = 24 * 1024;   // cap of one raw stage: S sub-tiles x (blocks + W)
constexpr int kDRawMax = 8;
constexpr int kDDigStage = 42 * 1024;   // cap of one digit stage
constexpr int kDDigStages = 3;
constexpr int kDSmem = 227 * 1024;
constexpr int kDOffBar = kDSmem - 1024;
constexpr int kDBars = 2 * (kDRawMax + kDDigStages + kBufs) + 1;  // + one that nothing completes (stall test)
constexpr int kDOffFlag = kDOffBar + kDBars * 8;
constexpr int kDOffTmem = kDOffFlag + 8;
constexpr int kDOffExp = kDOffTmem + 8;
constexpr int kDOffMax = kDOffExp + kS * 4;
static_assert(kDOffMax + kCW * kS * 8 <= kDSmem, "Gram kernel shared memory");
static_assert(2 * kDRawStage + kDDigStages * kDDigStage + 4096 <= kDOffBar, "two raw stages at least");

// bytes of one sub-tile's digit pieces for nvb blocks: A planes + W digit planes + 2 zero groups
__host__ __device__ constexpr int dsub_bytes(int nvb) { return kDig * nvb * kPiece + kBGroups * kPiece; }
// sub-tiles per stage: the stage carries >= ~240 digit groups of 8 values when it can
__host__ __device__ inline int dsubs_per_stage(int nvb)
{
    const int a = kDDigStage / dsub_bytes(nvb), b = kDRawStage / ((nvb + 1) * kKT * kRawRow);
    const int s = a < b ? a : b;
    return s < 1 ? 1 : s;
}
static_assert(kDDigStage >= dsub_bytes(kBlocksPerTile) && kDRawStage >= (kBlocksPerTile + 1) * kKT * kRawRow,
              "one full sub-tile per stage");

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


// The same MMA (and the commit below) issued by one lane of a converged warp: the whole warp
// runs the issuing loop, so the descriptors and addresses it computes are warp-uniform, and
// an elect.sync predicate lets exactly one lane issue.
__device__ __forceinline__ void mma_bf16_warp(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                              uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__host__ __device__ constexpr uint32_t make_idesc_amn(int M, int N) { return make_idesc(M, N) | (1u << 15); }

// MN-major descriptor of the update kernel's A operand (basis rows): next 8 basis columns
// (next block) 2 KB on, next 8 rows 128 bytes on
__device__ __forceinline__ uint64_t make_desc_mn(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(((8 * kPiece) >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((128 >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2, %3;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase of the given parity; false after `limit` ns without it.  The pipeline
// waits take the caller's limit; the waits that drain a CTA's own copies and MMAs before
// its shared and tensor memory are released always take kWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, unsigned long long limit = kWaitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit) return false;
    return true;
}

// a warp's bounded wait on one mbarrier phase; the outcome is the same in every lane
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, unsigned long long limit)
{
    return __all_sync(0xffffffffu, mbar_wait_bounded(bar, parity, limit)) != 0;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mma_commit_warp(uint32_t bar)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}\n" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t v[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

// Add the class sums of one accumulator buffer (this thread's tensor-memory row) into the
// exact integers hi, lo of its 8 output columns.  |S_c| <= 2^24: exact FP32 integers.
__device__ __forceinline__ void drain_classes(uint32_t tbuf, long long hi[kS], long long lo[kS])
{
    uint32_t v[3][16];
#pragma unroll
    for (int k = 0; k < 3; ++k) tmem_ld16(tbuf + 16 * k, v[k]);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int col = 16 * k + c, cls = col >> 3, b = col & 7;
            const long long d = (long long)__float2int_rz(__uint_as_float(v[k][c]));
            if (cls <= 4) hi[b] += d << (7 * (4 - cls));
            else lo[b] += d << (7 * (8 - cls));
        }
#pragma unroll
    for (int k = 0; k < 2; ++k) tmem_ld16(tbuf + 48 + 16 * k, v[k]);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int col = 48 + 16 * k + c, cls = col >> 3, b = col & 7;
            if (cls > 8) continue;  // class 9: padding products only
            const long long d = (long long)__float2int_rz(__uint_as_float(v[k][c]));
            if (cls <= 4) hi[b] += d << (7 * (4 - cls));
            else lo[b] += d << (7 * (8 - cls));
        }
}

// The same sums for one V digit p when the digit planes are stacked in M (the Gram kernel
// with at most two blocks, one MMA per sub-tile): this thread's tensor-memory row is (p,
// block, column) and its 64 columns are (W digit q, output column b); the products of
// class c = p + q <= 8 are added with the weights of drain_classes, higher classes dropped.
// Every cell sums at most 512 products of at most 64^2: exact FP32 integers.
__device__ __forceinline__ void drain_stacked(uint32_t tbuf, int p, long long hi[kS], long long lo[kS])
{
    uint32_t v[4][16];
#pragma unroll
    for (int k = 0; k < 4; ++k) tmem_ld16(tbuf + 16 * k, v[k]);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int col = 16 * k + c, q = col >> 3, b = col & 7, cls = p + q;
            if (cls > 8) continue;
            const long long d = (long long)__float2int_rz(__uint_as_float(v[k][c]));
            if (cls <= 4) hi[b] += d << (7 * (4 - cls));
            else lo[b] += d << (7 * (8 - cls));
        }
}

// value of the digit products times 2^e: a product of digits p, q weighs 2^(e - 10 - 7(p+q)),
// so hi carries class 4's weight 2^(e-38) and lo class 8's 2^(e-66); |hi|, |lo| < 2^53
// convert exactly, and 2^e is a normal double for the exponents of finite nonzero columns
// (a zero column has e = 0)
__device__ __forceinline__ double combine_hilo(long long hi, long long lo, int e)
{
    const double v = fma((double)hi, 0x1p-38, (double)lo * 0x1p-66);
    return v * __longlong_as_double((long long)(1023 + e) << 52);
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// sum over i < 8 of 64 * 128^i: m + kBdOffset has the base-128 digits d_i + 64 of the
// balanced digits d_i of m
constexpr uint64_t kBdOffset = 0x81020408102040ull;
constexpr uint64_t kBdZero = 0x4040404040404040ull;  // the byte digits of 0

// the eight 7-bit fields of a 28-bit value, one per byte of a 32-bit word
__device__ __forceinline__ uint32_t spread28(uint32_t x)
{
    return (x & 0x7Fu) | ((x << 1) & 0x7F00u) | ((x << 2) & 0x7F0000u) | ((x << 3) & 0x7F000000u);
}

// fixed-point magnitude round(|x| * 2^(54 - e)) (half away from zero) from the IEEE bits
// (integer operations only: the FP64 conversions are slow on this GPU); false if
// |x| * 2^-e >= 2 or x is not finite
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
    const int shift = ex - 1021 - e;  // mag = mant * 2^shift
    if (shift > 2) {
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

// Byte digits of x at scale 2^e: byte i = d_i + 64, m = round(x 2^(54-e)) = sum_i d_i 128^i,
// d_i in [-64, 63]: the bytes are the base-128 digits of m + kBdOffset.  False if
// |x| 2^-e >= 2, m is outside the eight digits' range, or x is not finite.
__device__ __forceinline__ bool to_bdigits(double x, int e, uint64_t &word)
{
    uint64_t mag;
    uint32_t neg;
    const bool ok = fixed_mag(x, e, mag, neg);
    const long long m = neg ? -(long long)mag : (long long)mag;
    const uint64_t u = (uint64_t)(m + (long long)kBdOffset);
    if (!ok || (u >> 56)) {  // outside [-kBdOffset, 2^56 - kBdOffset)
        word = kBdZero;
        return false;
    }
    word = (uint64_t)spread28((uint32_t)u & 0x0FFFFFFFu) | ((uint64_t)spread28((uint32_t)(u >> 28)) << 32);
    return true;
}

// Eight BF16 digit planes of 8 values in byte-digit form (8 consecutive rows of one
// column), one 16-byte chunk per plane at dst + p * pstride, plane p = digit of weight
// 128^(7-p).  For two rows and two digits one byte permute gathers the four digit bytes; a
// second puts each beside the byte 0x43, so that each half is the BF16 number 128 + x
// (x = d + 64 < 128, exact), and a BF16x2 add of -192 leaves d, exactly.
__device__ __forceinline__ void bexpand8(const uint64_t f[8], char *dst, int pstride)
{
    const __nv_bfloat162 off = __floats2bfloat162_rn(-192.0f, -192.0f);
#pragma unroll
    for (int pp = 0; pp < kDig; pp += 2) {
        // planes pp, pp + 1: bytes 7 - pp and 6 - pp, in the high word for pp < 4
        const int b0 = (7 - pp) & 3, b1 = (6 - pp) & 3;
        const uint32_t sel = (uint32_t)(b0 | ((4 + b0) << 4) | (b1 << 8) | ((4 + b1) << 12));
        uint32_t w0[4], w1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t a = pp < 4 ? (uint32_t)(f[2 * q] >> 32) : (uint32_t)f[2 * q];
            const uint32_t b = pp < 4 ? (uint32_t)(f[2 * q + 1] >> 32) : (uint32_t)f[2 * q + 1];
            const uint32_t g = __byte_perm(a, b, sel);  // [x_pp(r0), x_pp(r1), x_pp+1(r0), x_pp+1(r1)]
            uint32_t t0 = __byte_perm(g, 0x43434343u, 0x4140);
            uint32_t t1 = __byte_perm(g, 0x43434343u, 0x4342);
            const __nv_bfloat162 r0 = __hadd2(*reinterpret_cast<const __nv_bfloat162 *>(&t0), off);
            const __nv_bfloat162 r1 = __hadd2(*reinterpret_cast<const __nv_bfloat162 *>(&t1), off);
            w0[q] = *reinterpret_cast<const uint32_t *>(&r0);
            w1[q] = *reinterpret_cast<const uint32_t *>(&r1);
        }
        *reinterpret_cast<uint4 *>(dst + pp * pstride) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        *reinterpret_cast<uint4 *>(dst + (pp + 1) * pstride) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    }
}

// Byte-digit copies of nblocks n x 8 row-major blocks X (|x| < 2, else ERR_RANGE), in
// one or both layouts: F_row like X (the update kernel's rows), F_sub sub-tile-major
// across blocks -- block iblk0 + b, 16-row sub-tile t at ((t * ipad + iblk0 + b) * 16) * 8,
// 1 KB per (sub-tile, block), rows past n the digits of 0 -- so that the Gram kernel
// fetches a sub-tile of all its blocks in one copy.
__global__ void k_to_fixed(int32_t n, int32_t nblocks, const double *__restrict__ X, uint64_t *__restrict__ F_row,
                           uint64_t *__restrict__ F_sub, int32_t ipad, int32_t iblk0, int *err)
{
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    const int64_t per = nt * kKT * kS;  // padded entries per block
    bool bad = false;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < per * nblocks;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = g / per, e = g - b * per;
        const int64_t r = e / kS;
        const int a = (int)(e - r * kS);
        uint64_t f = kBdZero;
        if (r < n) {
            if (!to_bdigits(X[(b * n + r) * kS + a], 0, f)) bad = true;
            if (F_row) F_row[(b * n + r) * kS + a] = f;
        }
        if (F_sub) F_sub[(((r / kKT) * ipad + iblk0 + b) * kKT + (r % kKT)) * kS + a] = f;
    }
    if (bad) atomicOr(err, ERR_RANGE);
}

// Last step of Cholesky-QR for an 8-column basis block: Q := Q R^{-1} in place (the row
// solve every orthogonalisation kernel shares; deflated columns -> 0), and the block's
// byte digits written as k_to_fixed writes them (row layout; sub-tile layout at slot blk,
// padding rows of the last sub-tile the digits of 0), saving a pass over the new block.
__global__ void __launch_bounds__(256) k_trsm_fixed(int32_t n, double *__restrict__ Q, const double *__restrict__ R,
                                                    const int32_t *__restrict__ deflated, uint64_t *__restrict__ F_row,
                                                    uint64_t *__restrict__ F_sub, int32_t ipad, int32_t blk, int *err)
{
    __shared__ double Rs[kS * kS];
    __shared__ double rinv[kS];
    for (int e = threadIdx.x; e < kS * kS; e += blockDim.x) Rs[e] = R[e];
    if (threadIdx.x < kS) rinv[threadIdx.x] = deflated[threadIdx.x] ? 0.0 : 1.0 / R[threadIdx.x * kS + threadIdx.x];
    __syncthreads();
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT * kKT;
    bool bad = false;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nt; r += (int64_t)gridDim.x * blockDim.x) {
        uint64_t f[kS];
#pragma unroll
        for (int a = 0; a < kS; ++a) f[a] = kBdZero;
        if (r < n) {
            double x[kS];
            row_load<kS>(Q, r, x);
            trsm_row<kS>(x, Rs, rinv);
            row_store<kS>(Q, r, x);
#pragma unroll
            for (int a = 0; a < kS; ++a)
                if (!to_bdigits(x[a], 0, f[a])) bad = true;
            ulonglong2 *fr = reinterpret_cast<ulonglong2 *>(F_row + r * kS);
#pragma unroll
            for (int k = 0; k < kS / 2; ++k) fr[k] = make_ulonglong2(f[2 * k], f[2 * k + 1]);
        }
        ulonglong2 *fs = reinterpret_cast<ulonglong2 *>(F_sub + (((r / kKT) * ipad + blk) * kKT + (r % kKT)) * kS);
#pragma unroll
        for (int k = 0; k < kS / 2; ++k) fs[k] = make_ulonglong2(f[2 * k], f[2 * k + 1]);
    }
    if (bad) atomicOr(err, ERR_RANGE);
}

// Last pass of the fused Cholesky-QR for an 8-column basis block: Q := Q1 R2^{-1} in place,
// Q holding Q1 = W R1^{-1} from the second pass (the row solve every orthogonalisation
// kernel shares), and the block's fixed point as k_trsm_fixed writes it.  Four CTAs per
// SM, each thread over rows r, r + grid, ... with its next row loaded before the current
// one is solved (the row solve keeps the FP64 pipe busy meanwhile); the register cap keeps
// the factor in shared memory rather than in registers.
__global__ void __launch_bounds__(256, 4) k_cqr_apply_fixed(int32_t n, double *Q, const double *__restrict__ R2,
                                                            const int32_t *__restrict__ defl2,
                                                            uint64_t *__restrict__ F_row, uint64_t *__restrict__ F_sub,
                                                            int32_t ipad, int32_t blk, int *err, float *__restrict__ Q32)
{
    __shared__ double Rs2[kS * kS];
    __shared__ double rinv2[kS];
    for (int e = threadIdx.x; e < kS * kS; e += blockDim.x) Rs2[e] = R2[e];
    if (threadIdx.x < kS) rinv2[threadIdx.x] = defl2[threadIdx.x] ? 0.0 : 1.0 / R2[threadIdx.x * kS + threadIdx.x];
    __syncthreads();
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT * kKT;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double xn[kS];
    if (r < n) row_load<kS>(Q, r, xn);
    for (; r < nt; r += step) {
        asm volatile("" ::: "memory");  // the factors are read from shared memory in every row
        uint64_t f[kS];
#pragma unroll
        for (int a = 0; a < kS; ++a) f[a] = kBdZero;
        if (r < n) {
            double x[kS];
#pragma unroll
            for (int a = 0; a < kS; ++a) x[a] = xn[a];
            if (r + step < n) row_load<kS>(Q, r + step, xn);
            trsm_row<kS>(x, Rs2, rinv2);
            row_store<kS>(Q, r, x);
            if (Q32) {  // the block in FP32: the input of the mixed solve's FP32 operator
                float4 *q = reinterpret_cast<float4 *>(Q32 + r * kS);
                q[0] = make_float4(f64_to_f32(x[0]), f64_to_f32(x[1]), f64_to_f32(x[2]), f64_to_f32(x[3]));
                q[1] = make_float4(f64_to_f32(x[4]), f64_to_f32(x[5]), f64_to_f32(x[6]), f64_to_f32(x[7]));
            }
#pragma unroll
            for (int a = 0; a < kS; ++a)
                if (!to_bdigits(x[a], 0, f[a])) bad = true;
            ulonglong2 *fr = reinterpret_cast<ulonglong2 *>(F_row + r * kS);
#pragma unroll
            for (int k = 0; k < kS / 2; ++k) fr[k] = make_ulonglong2(f[2 * k], f[2 * k + 1]);
        }
        ulonglong2 *fs = reinterpret_cast<ulonglong2 *>(F_sub + (((r / kKT) * ipad + blk) * kKT + (r % kKT)) * kS);
#pragma unroll
        for (int k = 0; k < kS / 2; ++k) fs[k] = make_ulonglong2(f[2 * k], f[2 * k + 1]);
    }
    if (bad) atomicOr(err, ERR_RANGE);
}

// Gram product H_i = V_i^T W.  grid = (row chunks, M tiles of 16 blocks); a chunk is a
// whole number of 16-row sub-tiles, at most 4096 rows.  A stage carries S sub-tiles (S
// from the tile's block count, so that small products still fill the converters); a
// segment of whole stages covers at most 512 rows and owns one accumulator buffer.
// Warp 0 copies, warp 1 issues MMAs, warps 2..5 drain, warps 6..13 convert.  W's columns
// are scaled by powers of two from this chunk's own column maxima, so the chunk's partial
// sums carry their own scale.
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_block_dot_tc(int32_t n, int32_t nblk, int32_t subs_per_chunk, const uint64_t *__restrict__ Vfs, int32_t ipad,
                   const double *__restrict__ W, double *__restrict__ partial, int *err, unsigned long long wl,
                   int stall)
{
    extern __shared__ __align__(128) char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chunk = blockIdx.x, mt = blockIdx.y;
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    const int64_t t0 = (int64_t)chunk * subs_per_chunk;
    const int nsub = (int)min((int64_t)subs_per_chunk, nt - t0);
    const int blk0 = mt * kBlocksPerTile;
    const int nvb = min(kBlocksPerTile, nblk - blk0);  // valid blocks in this tile
    const int S = dsubs_per_stage(nvb);
    const int sub_bytes = dsub_bytes(nvb), plane = nvb * kPiece;
    const int nst = (nsub + S - 1) / S;                // stages
    const int sps = (kSegK / kKT) / S;                 // stages per segment (>= 2: S <= 12)
    const int nseg = (nst + sps - 1) / sps;
    const int rsb = S * (nvb + 1) * kKT * kRawRow, dsb = S * sub_bytes;  // stage bytes
    const int dig_off = ((kDOffBar - 4096 - kDDigStages * dsb) / rsb < kDRawMax
                             ? (kDOffBar - 4096 - kDDigStages * dsb) / rsb
                             : kDRawMax) * rsb;
    const int R = dig_off / rsb;  // raw stages
    const uint32_t bar0 = smem_u32(smem + kDOffBar);
    const uint32_t rfull0 = bar0, rempty0 = rfull0 + kDRawMax * 8;
    const uint32_t dfull0 = rempty0 + kDRawMax * 8, dempty0 = dfull0 + kDDigStages * 8;
    const uint32_t bfull0 = dempty0 + kDDigStages * 8, bfree0 = bfull0 + kBufs * 8;
    const uint32_t never = bfree0 + kBufs * 8;  // initialised, never arrived at
    volatile int *flag = reinterpret_cast<volatile int *>(smem + kDOffFlag);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kDOffTmem);
    int32_t *wexp = reinterpret_cast<int32_t *>(smem + kDOffExp);
    unsigned long long *wmax = reinterpret_cast<unsigned long long *>(smem + kDOffMax);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < R; ++s) {
            mbar_init(rfull0 + 8 * s, 1);
            mbar_init(rempty0 + 8 * s, kCW / kCG);
        }
        for (int s = 0; s < kDDigStages; ++s) {
            mbar_init(dfull0 + 8 * s, kCW / kCG);
            mbar_init(dempty0 + 8 * s, 1);
        }
        for (int b = 0; b < kBufs; ++b) {
            mbar_init(bfull0 + 8 * b, 1);
            mbar_init(bfree0 + 8 * b, 128);
        }
        mbar_init(never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        *flag = 0;
    }
    // zero groups 8 and 9 of every sub-tile's B operand (the digit-0 MMA reads them; the
    // converters never write them)
    for (int e = tid; e < kDDigStages * S * 2 * (kPiece / 16); e += kThreadsTC) {
        const int o = e % (2 * (kPiece / 16)), sd = e / (2 * (kPiece / 16));
        const int d = sd / S, sg = sd % S;
        *reinterpret_cast<uint4 *>(smem + dig_off + d * dsb + sg * sub_bytes + kDig * plane + kDig * kPiece +
                                   o * 16) = make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const bool work = nvb > 0 && nsub > 0;
    // at most two blocks: the eight V digit planes stacked in M (rows (p, block, column),
    // 64 nvb of the MMA's 128) against the eight W digit planes in N, one MMA per sub-tile;
    // classes are formed when the sums are drained
    const bool stacked = nvb <= 2;

    if (warp == 0) {
        if (lane == 0 && work) {  // ---- copies of stage k into raw stage k % R
            int issued = 0;
            for (int k = 0; k < nst; ++k) {
                const int s = k % R;
                if (k >= R && !mbar_wait_bounded(rempty0 + 8 * s, (uint32_t)(((k - R) / R) & 1), wl)) {
                    *flag = 1;
                    break;
                }
                if (*flag) break;
                const int ns = min(S, nsub - k * S);
                const int64_t tf = t0 + (int64_t)k * S;  // first sub-tile of the stage
                const uint32_t wbytes = (uint32_t)min((int64_t)ns * kKT, (int64_t)n - tf * kKT) * kRawRow;
                const uint32_t fb = rfull0 + 8 * s;
                mbar_expect_tx(fb, (uint32_t)(ns * nvb * kKT * kRawRow) + wbytes);
                char *st = smem + s * rsb;
#pragma unroll 1
                for (int sg = 0; sg < ns; ++sg)  // all nvb blocks of sub-tile tf + sg: one copy
                    bulk_copy(smem_u32(st + sg * nvb * (kKT * kRawRow)),
                              Vfs + (((tf + sg) * ipad + blk0) * kKT) * kS, (uint32_t)(nvb * kKT * kRawRow), fb);
                bulk_copy(smem_u32(st + S * nvb * (kKT * kRawRow)), W + tf * kKT * kS, wbytes, fb);
                issued = k + 1;
            }
            // every copy issued must have landed before shared memory is released
            for (int k = issued - R < 0 ? 0 : issued - R; k < issued; ++k)
                if (!mbar_wait_bounded(rfull0 + 8 * (k % R), (uint32_t)((k / R) & 1))) *flag = 1;
        }
    } else if (warp == 1) {
        if (work) {  // ---- MMA issuer: the whole warp runs the loop, one elected lane issues
            // test of the give-up path: a bounded wait on a barrier that nothing completes
            if (stall && !warp_wait(never, 0, wl) && lane == 0) *flag = 1;
            int done = 0;
            for (int k = 0; k < nst; ++k) {
                const int d = k % kDDigStages, seg = k / sps, buf = seg % kBufs;
                const bool first = k % sps == 0;
                bool ok = !(first && seg >= kBufs) ||
                          warp_wait(bfree0 + 8 * buf, (uint32_t)((seg / kBufs - 1) & 1), wl);
                if (ok) ok = warp_wait(dfull0 + 8 * d, (uint32_t)((k / kDDigStages) & 1), wl);
                if (!ok || __any_sync(0xffffffffu, *flag != 0)) {
                    if (lane == 0) *flag = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const char *st = smem + dig_off + d * dsb;
                const int ns = min(S, nsub - k * S);
                for (int sg = 0; sg < ns; ++sg) {
                    const char *sb = st + sg * sub_bytes;
                    const uint64_t db = make_desc(smem_u32(sb + kDig * plane));
                    if (stacked) {
                        mma_bf16_warp(tmem + buf * kBufCols, make_desc(smem_u32(sb)), db, make_idesc(kM, 8 * kDig),
                                      (first && sg == 0) ? 0u : 1u);
                        continue;
                    }
#pragma unroll
                    for (int p = 0; p < kDig; ++p) {
                        const uint64_t da = make_desc(smem_u32(sb + p * plane));
                        mma_bf16_warp(tmem + buf * kBufCols + 8 * p, da, db, make_idesc(kM, nmma(p)),
                                      (first && sg == 0 && p == 0) ? 0u : 1u);
                    }
                }
                mma_commit_warp(dempty0 + 8 * d);
                if (k % sps == sps - 1 || k == nst - 1) mma_commit_warp(bfull0 + 8 * buf);
                done = k + 1;
            }
            // the last commit: all MMAs done before shared memory is released
            if (done > 0) {
                const int k = done - 1;
                if (!warp_wait(dempty0 + 8 * (k % kDDigStages), (uint32_t)((k / kDDigStages) & 1), kWaitNs) &&
                    lane == 0)
                    *flag = 1;
            }
        }
    } else if (warp < 6) {  // ---- drain warps: tensor-memory lanes 32 (warp % 4) .. + 31 = basis columns
        if (work) {
            const int quarter = warp & 3;
            const int m = quarter * 32 + lane;
            const int pd = m / (8 * nvb);  // stacked: this row's V digit
            long long hi[kS], lo[kS];
#pragma unroll
            for (int b = 0; b < kS; ++b) hi[b] = lo[b] = 0;
            bool ok = true;
            for (int seg = 0; seg < nseg; ++seg) {
                const int buf = seg % kBufs;
                if (!mbar_wait_bounded(bfull0 + 8 * buf, (uint32_t)((seg / kBufs) & 1), wl) || *flag) {
                    *flag = 1;
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + buf * kBufCols;
                if (stacked) drain_stacked(tb, pd < kDig ? pd : kDig, hi, lo);  // rows past 64 nvb: unused
                else drain_classes(tb, hi, lo);
                asm volatile("tcgen05.fence::before_thread_sync;");
                mbar_arrive(bfree0 + 8 * buf);
            }
            // the chunk's W scale is known once the converters have started (named barrier 1)
            asm volatile("bar.sync 2, %0;" ::"r"(128 + kCT) : "memory");
            if (stacked) {
                // sum the eight digit rows of every (block, column): through the raw ring, idle
                // once the last accumulator is drained (all copies landed, all converted)
                long long *stg = reinterpret_cast<long long *>(smem);
                if (ok && m < 64 * nvb)
#pragma unroll
                    for (int b = 0; b < kS; ++b) {
                        stg[(2 * m) * kS + b] = hi[b];
                        stg[(2 * m + 1) * kS + b] = lo[b];
                    }
                asm volatile("bar.sync 3, 128;" ::: "memory");
                if (ok && m < 8 * nvb) {
#pragma unroll
                    for (int b = 0; b < kS; ++b) {
                        long long h = 0, l = 0;
                        for (int p = 0; p < kDig; ++p) {
                            h += stg[(2 * (p * 8 * nvb + m)) * kS + b];
                            l += stg[(2 * (p * 8 * nvb + m) + 1) * kS + b];
                        }
                        hi[b] = h;
                        lo[b] = l;
                    }
                }
            }
            if (ok && m < nvb * kS) {
                const int gm = blk0 * kS + m;
                double *dst = partial + ((int64_t)chunk * nblk + (gm >> 3)) * (kS * kS) + (gm & 7) * kS;
#pragma unroll
                for (int b = 0; b < kS; ++b) dst[b] = combine_hilo(hi[b], lo[b], wexp[b]);
            }
        }
    } else if (work) {  // ---- converters
        const int ct = tid - 192, cw = warp - 6;
        // W column maxima over this chunk's rows -> exponents e_b with |w| < 2^e_b
        {
            unsigned long long mx[kS];
#pragma unroll
            for (int b = 0; b < kS; ++b) mx[b] = 0;
            const int64_t r1 = min((int64_t)n, (t0 + nsub) * kKT);
#pragma unroll 4
            for (int64_t r = t0 * kKT + ct; r < r1; r += kCT) {
                const double2 *row = reinterpret_cast<const double2 *>(W + r * kS);
#pragma unroll
                for (int h = 0; h < kS / 2; ++h) {
                    const double2 x = row[h];
                    const unsigned long long b0 = (unsigned long long)__double_as_longlong(fabs(x.x));
                    const unsigned long long b1 = (unsigned long long)__double_as_longlong(fabs(x.y));
                    mx[2 * h] = b0 > mx[2 * h] ? b0 : mx[2 * h];
                    mx[2 * h + 1] = b1 > mx[2 * h + 1] ? b1 : mx[2 * h + 1];
                }
            }
#pragma unroll
            for (int b = 0; b < kS; ++b) {
                unsigned long long v = mx[b];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(0xffffffffu, v, o);
                    v = y > v ? y : v;
                }
                if (lane == 0) wmax[cw * kS + b] = v;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(kCT) : "memory");
            if (ct < kS) {
                unsigned long long v = 0;
                for (int w = 0; w < kCW; ++w) v = wmax[w * kS + ct] > v ? wmax[w * kS + ct] : v;
                const int ex = (int)((v >> 52) & 0x7FF);
                if (ex == 0x7FF) atomicOr(err, ERR_RANGE);  // not finite
                wexp[ct] = (ex == 0 || ex == 0x7FF) ? 0 : ex - 1022;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(kCT) : "memory");
            asm volatile("bar.arrive 2, %0;" ::"r"(128 + kCT) : "memory");  // exps ready for the drain warps
        }
        // two groups of four warps take alternate stages, so that two stages are converted at
        // once (a stage's conversion is a chain of dependent shared-memory steps)
        const int cg = cw / (kCW / kCG), ctg = ct % kCTG;
        bool bad = false;
        for (int k = cg; k < nst; k += kCG) {
            const int s = k % R, d = k % kDDigStages;
            bool ok = warp_wait(rfull0 + 8 * s, (uint32_t)((k / R) & 1), wl);
            if (ok && k >= kDDigStages)
                ok = warp_wait(dempty0 + 8 * d, (uint32_t)(((k - kDDigStages) / kDDigStages) & 1), wl);
            if (!ok || *flag) {
                if (lane == 0) *flag = 1;
                break;
            }
            const int ns = min(S, nsub - k * S);
            const char *raw = smem + s * rsb;
            char *dig = smem + dig_off + d * dsb;
            // W groups (FP64 -> digits, about four times a V group's work) on threads 0, 1, ...;
            // V groups first to the threads without a W group, four each, then to all in turn,
            // so that the stage's slowest warp carries about the mean work
            const int nwg = 16 * ns, nvg = 16 * nvb * ns;
            // the roles rotate by a warp from stage to stage: a warp does not wait for the
            // others between its stages, so each carries the mean over stages
            const int cr = (ctg + (k / kCG) * 32) & (kCTG - 1);
            for (int w = cr; w < nwg; w += kCTG) {
                const int sg = w >> 4, ko = (w >> 3) & 1, a = w & 7;
                const int64_t tt = t0 + (int64_t)k * S + sg;
                const int rv = (int)min((int64_t)kKT, (int64_t)n - tt * kKT);
                const double *src =
                    reinterpret_cast<const double *>(raw + (S * nvb + sg) * (kKT * kRawRow)) + ko * 8 * kS + a;
                const int e = wexp[a];
                uint64_t f[8];
#pragma unroll
                for (int v = 0; v < 8; ++v)
                    if (!to_bdigits((ko * 8 + v < rv) ? src[v * kS] : 0.0, e, f[v])) bad = true;
                bexpand8(f, dig + sg * sub_bytes + kDig * plane + ko * kLBO + a * 16, kPiece);
            }
            auto v_group = [&](int j) {  // V group j of the stage: (sub-tile, block, 8-row half, column)
                const int sg = j / (16 * nvb), r = j - sg * 16 * nvb;
                const int i = r >> 4, ko = (r >> 3) & 1, a = r & 7;
                const uint64_t *src =
                    reinterpret_cast<const uint64_t *>(raw + (sg * nvb + i) * (kKT * kRawRow)) + ko * 8 * kS + a;
                uint64_t f[8];
#pragma unroll
                for (int v = 0; v < 8; ++v) f[v] = src[v * kS];  // rows past n are zero in the sub-tile layout
                bexpand8(f, dig + sg * sub_bytes + i * kPiece + ko * kLBO + a * 16, plane);
            };
            // (a warp pays for every path its lanes take, so the first deal goes to whole warps
            // without a W group)
            const int ww = (nwg + 31) & ~31;             // threads of the warps with W groups
            const int tf = ww < kCTG ? kCTG - ww : 0;    // threads of the other warps
            const int first = min(4 * tf, nvg);          // V groups dealt to those threads alone
            if (cr >= ww)
                for (int j = cr - ww; j < first; j += tf) v_group(j);
            for (int j = first + cr; j < nvg; j += kCTG) v_group(j);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(rempty0 + 8 * s);
                mbar_arrive(dfull0 + 8 * d);
            }
        }
        if (bad) atomicOr(err, ERR_RANGE);
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (*flag && tid == 0) atomicOr(err, ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// Digits of H (nblk*8 basis columns x 8, H[c * 8 + b]) scaled per column b: piece (kappa, q)
// at hdig + (kappa * 8 + q) * 256 holds columns 16 kappa .. 16 kappa + 15 (zero beyond
// nblk * 8); hexp[b] = column exponent.  One CTA.
__global__ void k_h_digits(int32_t nblk, const double *__restrict__ H, char *__restrict__ hdig,
                           int32_t *__restrict__ hexp, int *err)
{
    __shared__ int32_t ex_s[kS];
    __shared__ unsigned long long mx_s[256];
    const int ncol = nblk * kS;
    {
        // column maxima: thread t scans column t % 8 at rows t / 8, t / 8 + 32, ... (the
        // block has 256 threads), then one thread per column combines the 32 partial maxima
        unsigned long long m = 0;
        for (int c = threadIdx.x / kS; c < ncol; c += 256 / kS) {
            const unsigned long long bits =
                (unsigned long long)__double_as_longlong(fabs(H[c * kS + threadIdx.x % kS]));
            m = bits > m ? bits : m;
        }
        mx_s[threadIdx.x] = m;
    }
    __syncthreads();
    if (threadIdx.x < kS) {
        unsigned long long m = 0;
        for (int g = 0; g < 256 / kS; ++g) m = mx_s[g * kS + threadIdx.x] > m ? mx_s[g * kS + threadIdx.x] : m;
        const int ex = (int)((m >> 52) & 0x7FF);
        ex_s[threadIdx.x] = ex == 0 ? 0 : ex - 1022;
        hexp[threadIdx.x] = ex_s[threadIdx.x];
    }
    __syncthreads();
    const int nk = (nblk + 1) / 2;
    for (int item = threadIdx.x; item < nk * kS * 2; item += blockDim.x) {
        const int b = item % kS, ko = (item / kS) % 2, kappa = item / (2 * kS);
        uint64_t f[8];
        bool bad = false;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = kappa * 16 + ko * 8 + u;
            const double x = c < ncol ? H[c * kS + b] : 0.0;
            if (!to_bdigits(x, ex_s[b], f[u])) bad = true;
        }
        if (bad) atomicOr(err, ERR_RANGE);
        bexpand8(f, hdig + kappa * kDig * kPiece + ko * kLBO + b * 16, kPiece);
    }
}


// ---------------------------------------------------------------------------------
// Block update out = base + sign * V_{0..nblk-1} H on the tensor cores (W -= V H of the
// Gram-Schmidt passes, U = V Y of the solution update), same digit scheme.  The MMA's M
// dimension is 128 rows of V, K runs over basis columns (16 = two blocks per MMA), N over
// H's digit planes x 8 columns.  V's digits are cut per stage from its byte-digit rows
// and laid out MN-major (8 basis columns x 8 contiguous rows per core matrix); H's digits
// are built once per call by k_h_digits as K-major pieces, one 2048-byte group per 16
// basis columns.  A segment of at most 32 K steps (512 basis columns) owns one accumulator
// buffer; a 128-row tile has at most two segments.
// ---------------------------------------------------------------------------------
constexpr int kURawBlk = 128 * kRawRow;       // 8 KB: 128 rows of one block
constexpr int kURawStage = 2 * kURawBlk;      // two blocks = one K step
constexpr int kURawStages = 6;
constexpr int kUPlane = 2 * (8 * kPiece);     // one digit plane of a stage: 2 blocks x 2 KB
constexpr int kUStageA = kDig * kUPlane;      // 32 KB
constexpr int kUDigStage = kUStageA + kBGroups * kPiece;  // + the 8 H digit pieces and 2 zero groups
constexpr int kUDigStages = 3;
constexpr int kUSegSteps = kSegK / 16;        // K steps per segment
constexpr int kUOffDig = kURawStages * kURawStage;
constexpr int kUOffBar = kUOffDig + kUDigStages * kUDigStage;
constexpr int kUBars = 2 * (kURawStages + kUDigStages + kBufs) + 1;  // + one that nothing completes (stall test)
constexpr int kUOffFlag = kUOffBar + kUBars * 8;
constexpr int kUOffTmem = kUOffFlag + 8;
constexpr int kUSmem = kUOffTmem + 16;
static_assert(kUSmem <= 227 * 1024, "update kernel shared memory");
static_assert(kUOffDig % 16 == 0 && kUDigStage % 16 == 0 && kUOffBar % 8 == 0, "alignment");

// Persistent block update: out[r][b] = base[r][b] + sign * (V H)[r][b] (base == null:
// sign * V H).  One CTA per SM walks 128-row tiles, one stage per K step of two basis
// blocks.  Warp 0 copies raw rows, warps 6..13 cut digits (and copy H's digit pieces of
// the step), warp 1 issues the MMAs, warps 2..5 drain the accumulator buffers and write
// the tile's rows.
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_block_update_tc(int32_t n, int32_t nblk, const uint64_t *__restrict__ Vf, const char *__restrict__ hdig,
                      const int32_t *__restrict__ hexp, const double *base, double *out, double sign, int *err,
                      unsigned long long wl, int stall)
{
    extern __shared__ __align__(128) char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nk = (nblk + 1) / 2;  // K steps of 16 basis columns
    const int nsegt = (nk + kUSegSteps - 1) / kUSegSteps;  // segments per tile
    const int64_t ntiles = ((int64_t)n + 127) / 128;
    const uint32_t bar0 = smem_u32(smem + kUOffBar);
    const uint32_t rfull0 = bar0, rempty0 = rfull0 + kURawStages * 8;
    const uint32_t dfull0 = rempty0 + kURawStages * 8, dempty0 = dfull0 + kUDigStages * 8;
    const uint32_t bfull0 = dempty0 + kUDigStages * 8, bfree0 = bfull0 + kBufs * 8;
    const uint32_t never = bfree0 + kBufs * 8;  // initialised, never arrived at
    volatile int *flag = reinterpret_cast<volatile int *>(smem + kUOffFlag);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kUOffTmem);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kURawStages; ++s) {
            mbar_init(rfull0 + 8 * s, 1);
            mbar_init(rempty0 + 8 * s, kCW);
        }
        for (int s = 0; s < kUDigStages; ++s) {
            mbar_init(dfull0 + 8 * s, kCW);
            mbar_init(dempty0 + 8 * s, 1);
        }
        for (int b = 0; b < kBufs; ++b) {
            mbar_init(bfull0 + 8 * b, 1);
            mbar_init(bfree0 + 8 * b, 128);
        }
        mbar_init(never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        *flag = 0;
    }
    // the two zero groups after each stage's H digit pieces (read by the digit-0 MMA)
    for (int e = tid; e < kUDigStages * 2 * (kPiece / 16); e += kThreadsTC) {
        const int s = e / (2 * (kPiece / 16)), o = e % (2 * (kPiece / 16));
        *reinterpret_cast<uint4 *>(smem + kUOffDig + s * kUDigStage + kUStageA + kDig * kPiece + o * 16) =
            make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // ---- copy thread: raw rows of the two blocks of every K step
            int64_t g = 0, issued = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && !*flag; tile += gridDim.x) {
                const uint32_t bytes = (uint32_t)min((int64_t)128, (int64_t)n - tile * 128) * kRawRow;
                for (int kk = 0; kk < nk; ++kk, ++g) {
                    const int s = (int)(g % kURawStages);
                    if (g >= kURawStages &&
                        !mbar_wait_bounded(rempty0 + 8 * s, (uint32_t)(((g - kURawStages) / kURawStages) & 1), wl)) {
                        *flag = 1;
                        break;
                    }
                    const int nbk = min(2, nblk - 2 * kk);
                    const uint32_t fb = rfull0 + 8 * s;
                    mbar_expect_tx(fb, (uint32_t)nbk * bytes);
                    char *st = smem + s * kURawStage;
#pragma unroll 1
                    for (int i = 0; i < nbk; ++i)
                        bulk_copy(smem_u32(st + i * kURawBlk), Vf + ((int64_t)(2 * kk + i) * n + tile * 128) * kS,
                                  bytes, fb);
                    issued = g + 1;
                }
            }
            // copies in flight must land before shared memory is released
            for (int64_t u = issued - kURawStages < 0 ? 0 : issued - kURawStages; u < issued; ++u)
                if (!mbar_wait_bounded(rfull0 + 8 * (int)(u % kURawStages), (uint32_t)((u / kURawStages) & 1)))
                    *flag = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA thread
            // test of the give-up path: a bounded wait on a barrier that nothing completes
            if (stall && !mbar_wait_bounded(never, 0, wl)) *flag = 1;
            int64_t g = 0, gs = 0;
            int64_t last = -1;  // last digit stage consumed
            for (int64_t tile = blockIdx.x; tile < ntiles && !*flag; tile += gridDim.x) {
                bool ok = true;
                for (int sgm = 0; sgm < nsegt && ok; ++sgm, ++gs) {
                    const int buf = (int)(gs % kBufs);
                    if (gs >= kBufs && !mbar_wait_bounded(bfree0 + 8 * buf, (uint32_t)((gs / kBufs - 1) & 1), wl)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const int k0 = sgm * kUSegSteps, k1 = min(nk, k0 + kUSegSteps);
                    for (int kk = k0; kk < k1; ++kk, ++g) {
                        const int d = (int)(g % kUDigStages);
                        if (!mbar_wait_bounded(dfull0 + 8 * d, (uint32_t)((g / kUDigStages) & 1), wl)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const char *st = smem + kUOffDig + d * kUDigStage;
                        const uint64_t db = make_desc(smem_u32(st + kUStageA));
#pragma unroll
                        for (int p = 0; p < kDig; ++p) {
                            const uint64_t da = make_desc_mn(smem_u32(st + p * kUPlane));
                            mma_bf16(tmem + buf * kBufCols + 8 * p, da, db, make_idesc_amn(kM, nmma(p)),
                                     (kk == k0 && p == 0) ? 0u : 1u);
                        }
                        mma_commit(dempty0 + 8 * d);
                        last = g;
                    }
                    if (ok) mma_commit(bfull0 + 8 * buf);  // segment finished: the drain may read it
                }
                if (!ok) {
                    *flag = 1;
                    break;
                }
            }
            // all MMAs done before shared memory is released
            if (last >= 0 &&
                !mbar_wait_bounded(dempty0 + 8 * (int)(last % kUDigStages), (uint32_t)((last / kUDigStages) & 1)))
                *flag = 1;
        }
    } else if (warp < 6) {  // ---- drain warps 2..5: tensor-memory lane quarter = warp % 4
        const int quarter = warp & 3;
        int64_t gs = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            long long hi[kS], lo[kS];
#pragma unroll
            for (int b = 0; b < kS; ++b) hi[b] = lo[b] = 0;
            // this row of the base, loaded before the tile's sums are waited for
            const int64_t r = tile * 128 + quarter * 32 + lane;
            double bv[kS];
#pragma unroll
            for (int b = 0; b < kS; ++b) bv[b] = 0.0;
            if (base && r < n)
#pragma unroll
                for (int h = 0; h < kS / 2; ++h) {
                    const double2 x = reinterpret_cast<const double2 *>(base + r * kS)[h];
                    bv[2 * h] = x.x;
                    bv[2 * h + 1] = x.y;
                }
            for (int sgm = 0; sgm < nsegt; ++sgm, ++gs) {
                const int buf = (int)(gs % kBufs);
                if (!mbar_wait_bounded(bfull0 + 8 * buf, (uint32_t)((gs / kBufs) & 1), wl) || *flag) {
                    *flag = 1;
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                drain_classes(tmem + ((uint32_t)(quarter * 32) << 16) + buf * kBufCols, hi, lo);
                asm volatile("tcgen05.fence::before_thread_sync;");
                mbar_arrive(bfree0 + 8 * buf);
            }
            if (ok && r < n) {
#pragma unroll
                for (int b = 0; b < kS; ++b) {
                    // hi 2^28 + lo in one exact 64-bit integer when hi is small (it is unless the
                    // basis entries reach 2^-8): one conversion and one scaling instead of
                    // combine_hilo's two and three, the same single rounding of the same exact sum
                    double vh;
                    const long long ah = hi[b] < 0 ? -hi[b] : hi[b];
                    if (ah < (1ll << 34) && hexp[b] > -900)
                        vh = (double)((hi[b] << 28) + lo[b]) * __longlong_as_double((long long)(1023 + hexp[b] - 66) << 52);
                    else
                        vh = combine_hilo(hi[b], lo[b], hexp[b]);
                    out[r * kS + b] = base ? fma(sign, vh, bv[b]) : sign * vh;
                }
            }
        }
    } else {  // ---- converters: group = (block slot, 16-row sub-tile, 8-row half, column)
        const int ct = tid - 192;
        const int i = ct >> 7, t8 = (ct >> 4) & 7, ko = (ct >> 3) & 1, a = ct & 7;
        const int rloc = t8 * kKT + ko * 8;
        int64_t g = 0;
        bool stop = false;
        for (int64_t tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x) {
            const int rv = (int)min((int64_t)128, (int64_t)n - tile * 128);
            for (int kk = 0; kk < nk; ++kk, ++g) {
                const int s = (int)(g % kURawStages), d = (int)(g % kUDigStages);
                bool ok = warp_wait(rfull0 + 8 * s, (uint32_t)((g / kURawStages) & 1), wl);
                if (ok && g >= kUDigStages)
                    ok = warp_wait(dempty0 + 8 * d, (uint32_t)(((g - kUDigStages) / kUDigStages) & 1), wl);
                if (!ok || *flag) {
                    if (lane == 0) *flag = 1;
                    stop = true;
                    break;
                }
                const int nbk = min(2, nblk - 2 * kk);
                const uint64_t *src =
                    reinterpret_cast<const uint64_t *>(smem + s * kURawStage + i * kURawBlk) + rloc * kS + a;
                char *dig = smem + kUOffDig + d * kUDigStage;
                uint64_t f[8];
#pragma unroll
                for (int v = 0; v < 8; ++v) f[v] = (i < nbk && rloc + v < rv) ? src[v * kS] : kBdZero;
                bexpand8(f, dig + i * (8 * kPiece) + t8 * kPiece + ko * kLBO + a * 16, kUPlane);
                if (ct < kDig * kPiece / 16)  // H's digit pieces of this K step
                    reinterpret_cast<uint4 *>(dig + kUStageA)[ct] =
                        reinterpret_cast<const uint4 *>(hdig + (int64_t)kk * kDig * kPiece)[ct];
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(rempty0 + 8 * s);
                    mbar_arrive(dfull0 + 8 * d);
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

size_t tc_hdig_bytes(int32_t nblk) { return (size_t)((nblk + 1) / 2) * kDig * kPiece; }

int block_update_tc_max_blocks() { return 128; }

int tc_subs_per_chunk(int32_t n, int32_t nblk)
{
    const int mtiles = (nblk + kBlocksPerTile - 1) / kBlocksPerTile;
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    int64_t want = (nt * mtiles + 152 - 1) / 152;  // ~1 CTA per SM in total
    if (want < 8) want = 8;
    if (want > kMaxRows / kKT) want = kMaxRows / kKT;
    return (int)want;
}

size_t tc_partial_elems(int32_t n, int32_t nblk)
{
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    return (size_t)((nt + 7) / 8) * nblk * kS * kS;  // chunks hold at least 8 sub-tiles
}

size_t tc_fixed_sub_bytes(int32_t n, int32_t nblocks)
{
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    return (size_t)nt * nblocks * kKT * kS * 8;
}

int launch_to_fixed(cudaStream_t st, int32_t n, int32_t nblocks, const double *X, uint64_t *F_row, uint64_t *F_sub,
                    int32_t ipad, int32_t iblk0, int *d_err)
{
    if (n <= 0 || nblocks <= 0) return 0;
    const int64_t count = (((int64_t)n + kKT - 1) / kKT) * kKT * kS * nblocks;
    int64_t g = (count + 255) / 256;
    if (g > 4 * 152) g = 4 * 152;
    k_to_fixed<<<(unsigned)g, 256, 0, st>>>(n, nblocks, X, F_row, F_sub, ipad, iblk0, d_err);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_trsm_fixed(cudaStream_t st, int32_t n, double *Q, const double *R, const int32_t *deflated, uint64_t *F_row,
                      uint64_t *F_sub, int32_t ipad, int32_t blk, int *d_err)
{
    if (n <= 0) return 0;
    const int64_t rows = ((int64_t)n + kKT - 1) / kKT * kKT;
    int64_t g = (rows + 255) / 256;
    if (g > 8 * 152) g = 8 * 152;
    k_trsm_fixed<<<(unsigned)g, 256, 0, st>>>(n, Q, R, deflated, F_row, F_sub, ipad, blk, d_err);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_cqr_apply_fixed(cudaStream_t st, int32_t n, double *Q, const double *R2, const int32_t *defl2,
                           uint64_t *F_row, uint64_t *F_sub, int32_t ipad, int32_t blk, int *d_err, float *Q32)
{
    if (n <= 0) return 0;
    const int64_t rows = ((int64_t)n + kKT - 1) / kKT * kKT;
    int64_t g = (rows + 255) / 256;
    if (g > 4 * 152) g = 4 * 152;
    k_cqr_apply_fixed<<<(unsigned)g, 256, 0, st>>>(n, Q, R2, defl2, F_row, F_sub, ipad, blk, d_err, Q32);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_block_update_tc(cudaStream_t st, int32_t n, int32_t nblk, const uint64_t *Vf, const double *H, void *hdig,
                           int32_t *hexp, const double *base, double *out, double sign, int *d_err, TcWait wt)
{
    if (n <= 0 || nblk <= 0 || nblk > block_update_tc_max_blocks()) return -1;
    k_h_digits<<<1, 256, 0, st>>>(nblk, H, (char *)hdig, hexp, d_err);
    note_launches(1);
    if (cudaFuncSetAttribute(k_block_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kUSmem) != cudaSuccess)
        return -1;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = ((int64_t)n + 127) / 128;
    const int grid = (int)(tiles < sms ? tiles : sms);
    k_block_update_tc<<<grid, kThreadsTC, kUSmem, st>>>(n, nblk, Vf, (const char *)hdig, hexp, base, out, sign,
                                                         d_err, (unsigned long long)wt.ns, wt.stall);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_block_dot_tc(cudaStream_t st, int32_t n, int32_t nblk, const uint64_t *Vfs, int32_t ipad, const double *W,
                        double *partial, double *out, int *d_err, TcWait wt)
{
    if (n <= 0 || nblk <= 0) return -1;
    if (cudaFuncSetAttribute(k_block_dot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kDSmem) != cudaSuccess)
        return -1;
    const int spc = tc_subs_per_chunk(n, nblk);
    const int64_t nt = ((int64_t)n + kKT - 1) / kKT;
    const int chunks = (int)((nt + spc - 1) / spc);
    const int mtiles = (nblk + kBlocksPerTile - 1) / kBlocksPerTile;
    dim3 grid(chunks, mtiles);
    k_block_dot_tc<<<grid, kThreadsTC, kDSmem, st>>>(n, nblk, spc, Vfs, ipad, W, partial, d_err,
                                                      (unsigned long long)wt.ns, wt.stall);
    note_launches(1);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return launch_reduce_chunks(st, nblk * kS * kS, chunks, partial, out);
}

}  // namespace spai

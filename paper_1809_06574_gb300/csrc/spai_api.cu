// C ABI of libspai_gb300 (declared in include/spai_gb300.h): context and handle
// management, the build / update pipelines of the SPAI preconditioner (Sec. 2.2,
// Sec. 2.3 Table 1, Sec. 2.4) and the host loop of right-preconditioned block GMRES(m)
// (Sec. 2.1, Sec. 2.2 footnote).  Every arithmetic step runs in the kernels of
// k_sparse.cu, k_spai.cu and k_krylov.cu; this file only sequences them, owns device
// memory and turns failures into status codes.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <tuple>
#include <atomic>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "spai_internal.cuh"

using namespace spai;

struct spai_ctx_s {
    cudaStream_t stream = nullptr;
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0;
    std::unordered_map<void *, size_t> sizes;
    std::mutex mu;  // guards budget and sizes: a pattern analysis may be released from another context's thread
    std::string err;
    int *d_err = nullptr;      // device error word
    int32_t *d_scalar = nullptr;  // small device scratch for host read-backs
    void *ws = nullptr;        // grow-only solve workspace
    size_t ws_bytes = 0;
    double *h_pinned = nullptr;  // pinned host scratch for per-iteration read-backs
    uint64_t wait_ns = 1000000000ull;  // limit of the tensor-core kernels' pipeline waits
    int32_t stall_left = 0;            // tensor-core launches still to run the stall test
    // optional per-kernel-family timing with CUDA events on the context's stream
    struct ProfRec {
        int family;
        cudaEvent_t a, b;
        double flops, bytes;
    };
    struct ProfFamily {
        std::string name;
        int64_t launches = 0;
        double ms = 0.0, flops = 0.0, bytes = 0.0;
    };
    bool prof_on = false;
    cudaEvent_t prof_last = nullptr;  // end event of the latest resolved launch
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
    std::vector<ProfFamily> prof_fam;
};

namespace {

// One device allocation holding the arrays of many handles (a batched build): released
// when the last handle that points into it is.
struct Arena {
    std::atomic<int> refs{0};
    spai_ctx ctx = nullptr;
    void *mem = nullptr;
};

void arena_release(Arena *a);

struct Sym {
    std::atomic<int> refs{1};  // handles on other contexts (host threads) may share it
    Arena *arena = nullptr;    // non-null: the arrays live in this arena, not in own allocations
    spai_ctx ctx = nullptr;
    int32_t n = 0, nnzA = 0, kind = 0;
    int32_t *a_rowptr = nullptr, *a_colind = nullptr;            // copy of A's CSR pattern
    int32_t *a_colptr = nullptr, *a_rowind = nullptr, *a_perm = nullptr;  // CSC + csc->csr
    int32_t *Jptr = nullptr, *Jind = nullptr;                     // pattern of P (columns)
    int32_t nnzP = 0;
    int32_t *p_rowptr = nullptr, *p_colind = nullptr;             // pattern of P (rows)
    int32_t *p_map = nullptr;                                     // J position -> P CSR position
    bool alias = true;                                            // P pattern == A pattern
    int32_t nI = 0;
    int32_t *Iptr = nullptr, *Ilist = nullptr;
    int32_t maxI = 0, maxJ = 0;
};

}  // namespace

struct spai_pc_s {
    spai_ctx ctx = nullptr;
    Sym *sym = nullptr;
    spai_pc parent = nullptr;
    spai_pc root = nullptr;
    int depth = 0;
    double *fval = nullptr;    // own factor, P's CSR order (FP64 factors)
    float *fval32 = nullptr;   // the same for SPAI_PREC_FP32 factors
    uint16_t *fval16 = nullptr;  // the same for SPAI_PREC_BF16 factors (BF16 bit patterns)
    double *a_cval = nullptr;  // this matrix's values in CSC order
    int32_t *status = nullptr;
    bool diag = false;         // diagonal factor (n values, SPAI_UPDATE_DIAGONAL)
    bool normal = false;       // column problems by their normal equations (SPAI_LS_NORMAL)
    Arena *arena = nullptr;    // non-null: fval*, a_cval and status live in this arena
};

// recycled outer space of block GCRO: k of kmax columns as k / s row-major n x s blocks
struct spai_recycle_s {
    spai_ctx ctx = nullptr;
    int32_t n = 0, s = 0, kmax = 0, k = 0;
    double *U = nullptr;
};

struct spai_affine_s {
    spai_ctx ctx = nullptr;
    int32_t n = 0, T = 0;
    int64_t nnz = 0;
    int32_t *rowptr = nullptr, *colind = nullptr;
    double *aligned = nullptr;  // T x nnz
};

namespace {

spai_status fail(spai_ctx ctx, spai_status st, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

spai_status cuda_fail(spai_ctx ctx, cudaError_t e, const char *what)
{
    return fail(ctx, SPAI_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

#define KL(call, what)                                                     \
    do {                                                                   \
        if ((call) != 0) {                                                 \
            cudaError_t e_ = cudaGetLastError();                           \
            return fail(ctx, SPAI_ECUDA, "%s: kernel launch failed (%s)", what, \
                        cudaGetErrorString(e_));                           \
        }                                                                  \
    } while (0)

cudaEvent_t prof_event(spai_ctx ctx)
{
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int prof_family(spai_ctx ctx, const char *name)
{
    for (size_t i = 0; i < ctx->prof_fam.size(); ++i)
        if (ctx->prof_fam[i].name == name) return (int)i;
    ctx->prof_fam.push_back({name});
    return (int)ctx->prof_fam.size() - 1;
}

// Resolve recorded event pairs into the per-family totals.  wait: synchronise the stream
// and resolve all; otherwise resolve the completed prefix only (never blocks).
void prof_flush(spai_ctx ctx, bool wait = true)
{
    if (ctx->prof_recs.empty()) return;
    size_t done = ctx->prof_recs.size();
    if (wait) {
        cudaStreamSynchronize(ctx->stream);
    } else {
        done = 0;
        while (done < ctx->prof_recs.size() && cudaEventQuery(ctx->prof_recs[done].b) == cudaSuccess) ++done;
        cudaGetLastError();  // cudaErrorNotReady is not an error here
        if (done == 0) return;
    }
    for (size_t k = 0; k < done; ++k) {
        auto &r = ctx->prof_recs[k];
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto &f = ctx->prof_fam[r.family];
        f.launches += 1;
        f.ms += ms;
        f.flops += r.flops;
        f.bytes += r.bytes;
        if (ctx->prof_last) {
            // stream time between the previous profiled launch and this one: other work on
            // the stream (copies, memsets, foreign kernels) or the device waiting for the host
            float gap = 0.f;
            cudaEventElapsedTime(&gap, ctx->prof_last, r.a);
            const int gi = prof_family(ctx, ("idle:" + ctx->prof_fam[r.family].name).c_str());
            ctx->prof_fam[gi].launches += 1;
            ctx->prof_fam[gi].ms += gap > 0.f ? gap : 0.f;
            ctx->prof_pool.push_back(ctx->prof_last);
        }
        ctx->prof_last = r.b;
        ctx->prof_pool.push_back(r.a);
    }
    ctx->prof_recs.erase(ctx->prof_recs.begin(), ctx->prof_recs.begin() + (ptrdiff_t)done);
}

// RAII timing of the launches issued inside its scope (no-op unless profiling is on).
struct ProfScope {
    spai_ctx ctx;
    int fam = -1;
    cudaEvent_t a = nullptr;
    double flops, bytes;
    ProfScope(spai_ctx c, const char *name, double fl, double by) : ctx(c), flops(fl), bytes(by)
    {
        if (!ctx->prof_on) return;
        fam = prof_family(ctx, name);
        a = prof_event(ctx);
        cudaEventRecord(a, ctx->stream);
    }
    ~ProfScope()
    {
        if (fam < 0) return;
        cudaEvent_t b = prof_event(ctx);
        cudaEventRecord(b, ctx->stream);
        ctx->prof_recs.push_back({fam, a, b, flops, bytes});
        if (ctx->prof_recs.size() > 4096) prof_flush(ctx, false);
    }
};

#define PKL(name, fl, by, call, what)          \
    do {                                       \
        ProfScope ps_(ctx, name, (fl), (by));  \
        KL(call, what);                        \
    } while (0)

spai_status dalloc(spai_ctx ctx, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) / 256 * 256;
    std::unique_lock<std::mutex> lock(ctx->mu);
    if (ctx->budget && ctx->in_use + bytes > ctx->budget) {
        const size_t used = ctx->in_use;
        lock.unlock();
        return fail(ctx, SPAI_ENOMEM, "memory budget exceeded: %zu in use + %zu requested > %zu", used, bytes,
                    ctx->budget);
    }
    cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        lock.unlock();
        return fail(ctx, SPAI_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    }
    ctx->in_use += bytes;
    ctx->sizes[*p] = bytes;
    return SPAI_OK;
}

template <class Tp>
spai_status dalloc_n(spai_ctx ctx, Tp **p, int64_t count)
{
    void *q = nullptr;
    spai_status st = dalloc(ctx, &q, (size_t)(count < 1 ? 1 : count) * sizeof(Tp));
    *p = (Tp *)q;
    return st;
}

void dfree(spai_ctx ctx, void *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(ctx->mu);
    auto it = ctx->sizes.find(p);
    if (it != ctx->sizes.end()) {
        ctx->in_use -= it->second;
        ctx->sizes.erase(it);
    }
    cudaFreeAsync(p, ctx->stream);
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

spai_status read_err(spai_ctx ctx, int *h)
{
    CU(cudaMemcpyAsync(h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "read error word");
    CU(cudaStreamSynchronize(ctx->stream), "stream sync");
    CU(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream), "clear error word");
    return SPAI_OK;
}

spai_status read_i32(spai_ctx ctx, const int32_t *d, int32_t *h)
{
    CU(cudaMemcpyAsync(h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream), "read back");
    CU(cudaStreamSynchronize(ctx->stream), "stream sync");
    return SPAI_OK;
}

spai_status check_csr_args(spai_ctx ctx, const spai_csr *A, const char *name)
{
    if (!A) return fail(ctx, SPAI_EINVAL, "%s is NULL", name);
    if (A->n < 0 || A->nnz < 0) return fail(ctx, SPAI_EINVAL, "%s: negative size", name);
    if (A->n > 0 && (!A->rowptr || (A->nnz > 0 && (!A->colind || !A->val))))
        return fail(ctx, SPAI_EINVAL, "%s: NULL array", name);
    return SPAI_OK;
}

spai_status validate_device_csr(spai_ctx ctx, const spai_csr *A, const char *name)
{
    spai_status st = check_csr_args(ctx, A, name);
    if (st) return st;
    if (A->n == 0) return SPAI_OK;
    if (!is_device_ptr(A->rowptr) || (A->nnz > 0 && (!is_device_ptr(A->colind) || !is_device_ptr(A->val))))
        return fail(ctx, SPAI_EINVAL, "%s: arrays must be device memory", name);
    KL(launch_validate_csr(ctx->stream, A->n, A->nnz, A->rowptr, A->colind, ctx->d_err), "validate");
    int h = 0;
    st = read_err(ctx, &h);
    if (st) return st;
    if (h & ERR_ROWPTR) return fail(ctx, SPAI_EINVAL, "%s: row pointer array is not a valid CSR row pointer", name);
    if (h & ERR_COLIND)
        return fail(ctx, SPAI_EINVAL, "%s: column indices out of range or not strictly increasing in a row", name);
    return SPAI_OK;
}

void arena_release(Arena *a)
{
    if (!a || a->refs.fetch_sub(1) > 1) return;
    dfree(a->ctx, a->mem);
    delete a;
}

void sym_release(Sym *s)
{
    if (!s || s->refs.fetch_sub(1) > 1) return;
    if (s->arena) {
        arena_release(s->arena);
        delete s;
        return;
    }
    spai_ctx ctx = s->ctx;
    dfree(ctx, s->a_rowptr);
    dfree(ctx, s->a_colind);
    dfree(ctx, s->a_colptr);
    dfree(ctx, s->a_rowind);
    dfree(ctx, s->a_perm);
    if (!s->alias) {
        dfree(ctx, s->Jptr);
        dfree(ctx, s->Jind);
        dfree(ctx, s->p_rowptr);
        dfree(ctx, s->p_colind);
        dfree(ctx, s->p_map);
    }
    dfree(ctx, s->Iptr);
    dfree(ctx, s->Ilist);
    delete s;
}

// Pattern analyses of nsys matrices (Sec. 2.2: the column patterns J_k and the row sets
// I_k = union of rows(A(:,j)), j in J_k), run phase by phase over all systems so that each
// host read-back of sizes covers every system at once: at most five synchronisations
// whatever nsys is.  kinds[i] is SPAI_PATTERN_A or SPAI_PATTERN_A2.
spai_status sym_create_batch(spai_ctx ctx, int32_t nsys, const spai_csr *A, const int32_t *kinds, Sym **out)
{
    std::vector<Sym *> S((size_t)nsys, nullptr);
    int32_t *d_vals = nullptr;  // [4][nsys]: max column length / max |J|, total |J|, total |I|, max |I|
    void *temp = nullptr, *temp2 = nullptr;
    spai_status st = SPAI_OK;
    auto cleanup = [&](spai_status rc) {
        dfree(ctx, d_vals);
        dfree(ctx, temp);
        dfree(ctx, temp2);
        if (rc) {
            for (Sym *s : S) sym_release(s);
        }
        return rc;
    };
#define TRY(x)                              \
    do {                                    \
        if ((st = (x)) != SPAI_OK) return cleanup(st); \
    } while (0)
#define TRYK(call, what)                                                                  \
    do {                                                                                  \
        if ((call) != 0) return cleanup(fail(ctx, SPAI_ECUDA, "%s: kernel launch failed (%s)", what, \
                                             cudaGetErrorString(cudaGetLastError())));   \
    } while (0)
    std::vector<int32_t> h((size_t)4 * nsys, 0);
    auto readback = [&](int field) -> spai_status {
        CU(cudaMemcpyAsync(h.data() + (size_t)field * nsys, d_vals + (size_t)field * nsys, (size_t)nsys * 4,
                           cudaMemcpyDeviceToHost, ctx->stream), "read back");
        CU(cudaStreamSynchronize(ctx->stream), "stream sync");
        return SPAI_OK;
    };
    TRY(dalloc_n(ctx, &d_vals, (int64_t)4 * nsys));
    CU(cudaMemsetAsync(d_vals, 0, (size_t)16 * nsys, ctx->stream), "memset");
    // scratch shared by the systems (stream order serialises its reuse)
    size_t tbytes = 0, cbytes = 0;
    for (int i = 0; i < nsys; ++i) {
        tbytes = std::max(tbytes, transpose_temp_bytes(A[i].n, A[i].nnz));
        cbytes = std::max(cbytes, ((size_t)A[i].n + 1) * 4 + 256 + scan_temp_bytes(A[i].n));
    }
    TRY(dalloc(ctx, &temp, std::max(tbytes, cbytes)));
    int32_t *counts = (int32_t *)temp;
    auto scan_temp = [&](int32_t n) { return (void *)((char *)temp + ((((size_t)n + 1) * 4 + 255) / 256 * 256)); };

    // ---- phase A: copy A's pattern, transpose it (CSC + position map), longest column
    for (int i = 0; i < nsys; ++i) {
        Sym *s = new Sym();
        S[i] = s;
        s->ctx = ctx;
        s->n = A[i].n;
        s->nnzA = A[i].nnz;
        s->kind = kinds[i];
        const int32_t n = A[i].n, nnz = A[i].nnz;
        TRY(dalloc_n(ctx, &s->a_rowptr, (int64_t)n + 1));
        TRY(dalloc_n(ctx, &s->a_colind, nnz));
        TRY(dalloc_n(ctx, &s->a_colptr, (int64_t)n + 1));
        TRY(dalloc_n(ctx, &s->a_rowind, nnz));
        TRY(dalloc_n(ctx, &s->a_perm, nnz));
        CU(cudaMemcpyAsync(s->a_rowptr, A[i].rowptr, ((size_t)n + 1) * 4, cudaMemcpyDeviceToDevice, ctx->stream), "copy");
        if (nnz)
            CU(cudaMemcpyAsync(s->a_colind, A[i].colind, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, ctx->stream), "copy");
        TRYK(launch_transpose(ctx->stream, n, nnz, s->a_rowptr, s->a_colind, s->a_colptr, s->a_rowind, s->a_perm,
                              temp, ctx->d_err), "transpose");
        TRYK(launch_max_i32_diff(ctx->stream, n, s->a_colptr, d_vals + i), "longest column");
        if (kinds[i] == SPAI_PATTERN_A) {
            s->alias = true;
            s->Jptr = s->a_colptr;
            s->Jind = s->a_rowind;
            s->nnzP = nnz;
            s->p_rowptr = s->a_rowptr;
            s->p_colind = s->a_colind;
            s->p_map = s->a_perm;
        } else {
            s->alias = false;
        }
    }
    TRY(readback(0));
    bool any_a2 = false;
    for (int i = 0; i < nsys; ++i) {
        if (h[i] > colunion_max_lists())
            return cleanup(fail(ctx, SPAI_EINVAL, "system %d: a column has %d entries; at most %d are supported", i,
                                h[i], colunion_max_lists()));
        if (kinds[i] == SPAI_PATTERN_A) S[i]->maxJ = h[i];
        else any_a2 = true;
    }
    // ---- phase B (pattern of A^2): J_k = union over j in rows(A(:,k)) of rows(A(:,j))
    if (any_a2) {
        for (int i = 0; i < nsys; ++i) {
            Sym *s = S[i];
            if (s->alias) continue;
            const int32_t n = s->n;
            TRY(dalloc_n(ctx, &s->Jptr, (int64_t)n + 1));
            TRYK(launch_colunion_count(ctx->stream, n, h[i], s->a_colptr, s->a_rowind, s->a_colptr, s->a_rowind, counts,
                                       ctx->d_err), "pattern count");
            TRYK(launch_exclusive_scan(ctx->stream, counts, s->Jptr, n, scan_temp(n), ctx->d_err), "scan");
            CU(cudaMemcpyAsync(d_vals + nsys + i, s->Jptr + n, 4, cudaMemcpyDeviceToDevice, ctx->stream), "total");
        }
        TRY(readback(1));
        size_t t2 = 0;
        for (int i = 0; i < nsys; ++i)
            if (!S[i]->alias) t2 = std::max(t2, transpose_temp_bytes(S[i]->n, h[nsys + i]));
        TRY(dalloc(ctx, &temp2, t2));
        for (int i = 0; i < nsys; ++i) {
            Sym *s = S[i];
            if (s->alias) continue;
            const int32_t n = s->n;
            s->nnzP = h[nsys + i];
            int32_t *perm_rows = nullptr;
            TRY(dalloc_n(ctx, &s->Jind, s->nnzP));
            TRYK(launch_colunion_fill(ctx->stream, n, h[i], s->a_colptr, s->a_rowind, s->a_colptr, s->a_rowind, s->Jptr,
                                      s->Jind, ctx->d_err), "pattern fill");
            TRYK(launch_max_i32_diff(ctx->stream, n, s->Jptr, d_vals + i), "max |J|");
            // row-wise pattern of P and the map from column positions to row positions
            TRY(dalloc_n(ctx, &s->p_rowptr, (int64_t)n + 1));
            TRY(dalloc_n(ctx, &s->p_colind, s->nnzP));
            TRY(dalloc_n(ctx, &s->p_map, s->nnzP));
            TRY(dalloc_n(ctx, &perm_rows, s->nnzP));
            TRYK(launch_transpose(ctx->stream, n, s->nnzP, s->Jptr, s->Jind, s->p_rowptr, s->p_colind, perm_rows, temp2,
                                  ctx->d_err), "transpose pattern");
            TRYK(launch_invert_perm(ctx->stream, s->nnzP, perm_rows, s->p_map), "invert");
            dfree(ctx, perm_rows);
        }
        TRY(readback(0));
        for (int i = 0; i < nsys; ++i) {
            if (S[i]->alias) continue;
            S[i]->maxJ = h[i];
            if (h[i] > colunion_max_lists())
                return cleanup(fail(ctx, SPAI_EINVAL, "system %d: a column pattern has %d entries; at most %d are "
                                    "supported", i, h[i], colunion_max_lists()));
        }
    }
    // ---- phase C: I_k = union over j in J_k of rows(A(:,j))
    for (int i = 0; i < nsys; ++i) {
        Sym *s = S[i];
        const int32_t n = s->n;
        TRY(dalloc_n(ctx, &s->Iptr, (int64_t)n + 1));
        TRYK(launch_colunion_count(ctx->stream, n, s->maxJ, s->Jptr, s->Jind, s->a_colptr, s->a_rowind, counts, ctx->d_err),
             "index set count");
        TRYK(launch_exclusive_scan(ctx->stream, counts, s->Iptr, n, scan_temp(n), ctx->d_err), "scan");
        CU(cudaMemcpyAsync(d_vals + 2 * nsys + i, s->Iptr + n, 4, cudaMemcpyDeviceToDevice, ctx->stream), "total");
    }
    CU(cudaMemcpyAsync(h.data() + 2 * nsys, d_vals + 2 * nsys, (size_t)nsys * 4, cudaMemcpyDeviceToHost, ctx->stream),
       "read back");
    int herr = 0;
    TRY(read_err(ctx, &herr));  // synchronises
    if (herr & ERR_OVERFLOW) return cleanup(fail(ctx, SPAI_EINVAL, "index sets exceed 2^31 entries"));
    if (herr) return cleanup(fail(ctx, SPAI_EINVAL, "pattern analysis failed (device error 0x%x)", herr));
    for (int i = 0; i < nsys; ++i) {
        Sym *s = S[i];
        s->nI = h[2 * nsys + i];
        TRY(dalloc_n(ctx, &s->Ilist, s->nI));
        TRYK(launch_colunion_fill(ctx->stream, s->n, s->maxJ, s->Jptr, s->Jind, s->a_colptr, s->a_rowind, s->Iptr, s->Ilist,
                                  ctx->d_err), "index set fill");
        TRYK(launch_max_i32_diff(ctx->stream, s->n, s->Iptr, d_vals + 3 * nsys + i), "max |I|");
    }
    CU(cudaMemcpyAsync(h.data() + 3 * nsys, d_vals + 3 * nsys, (size_t)nsys * 4, cudaMemcpyDeviceToHost, ctx->stream),
       "read back");
    TRY(read_err(ctx, &herr));
    if (herr) return cleanup(fail(ctx, SPAI_EINVAL, "pattern analysis failed (device error 0x%x)", herr));
    for (int i = 0; i < nsys; ++i) {
        Sym *s = S[i];
        s->maxI = h[3 * nsys + i];
        if (!spai_columns_fit(s->maxI, s->maxJ))
            return cleanup(fail(ctx, SPAI_EINVAL, "system %d: column problem of %d x %d exceeds the shared-memory tile",
                                i, s->maxI, s->maxJ));
    }
#undef TRY
#undef TRYK
    for (int i = 0; i < nsys; ++i) out[i] = S[i];
    return cleanup(SPAI_OK);
}

spai_status sym_create(spai_ctx ctx, const spai_csr *A, int32_t kind, Sym **out)
{
    *out = nullptr;
    return sym_create_batch(ctx, 1, A, &kind, out);
}

// Team size (or register-tiled shape) of the column kernel, chosen per (working precision,
// tile rows rounded up to 8, tile columns) process-wide: the first call that meets a shape
// -- a batch or a single build or update -- times every fitting candidate on its own
// columns with CUDA events and keeps the fastest; later calls reuse it.  One thread tunes
// at a time (others that meet the same shape wait and reuse its choice), so every call
// after the first uses one team per shape.  Candidates change the rounding of the
// reductions only.  Candidates are timed on the first kTuneColumns columns when there are
// more (a bounded one-time cost: the 27-point 128^3 FP64 build would otherwise pay a dozen
// full launches; smaller samples misjudged variants whose blocks hold different numbers
// of columns by a few per cent); when all columns were timed, each candidate wrote the
// complete result and *done on return says the chosen candidate's result is in place.
std::mutex g_tune_mu;      // guards g_tune
std::mutex g_tune_run_mu;  // one tuning run at a time
std::map<std::tuple<int, int, int>, int> g_tune;

constexpr int64_t kTuneColumns = 262144;

spai_status tuned_team(spai_ctx ctx, bool low, int32_t maxI, int32_t maxJ, int64_t total,
                       const std::function<int(int, int64_t)> &launch, int *team, bool *done, bool normal = false)
{
    const int64_t sample = std::min(total, kTuneColumns);
    // normal-equations shapes are tuned apart (keys 2, 3): they are another arithmetic
    const auto key = std::make_tuple((low ? 1 : 0) + (normal ? 2 : 0), (maxI + 7) / 8 * 8, maxJ);
    auto lookup = [&]() {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        return it == g_tune.end() ? 0 : it->second;
    };
    *done = false;
    if ((*team = lookup())) return SPAI_OK;
    std::lock_guard<std::mutex> run(g_tune_run_mu);
    if ((*team = lookup())) return SPAI_OK;  // tuned by another thread meanwhile
    int cand[32];
    const int nc = normal ? spai_columns_ne_teams(maxI, maxJ, low, cand) : spai_columns_teams(maxI, maxJ, low, cand);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(cudaEventCreate(&e0), "event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, SPAI_ECUDA, "event");
    }
    // two timed runs per candidate, the faster one counts (the first launch of a kernel in
    // the process, and the first candidate's cold caches, would otherwise bias the choice)
    float best_ms = 0.f;
    int best = 0, last = 0;
    for (int c = 0; c < nc; ++c) {
        float ms = -1.f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, ctx->stream);
            if (launch(cand[c], sample)) {
                cudaGetLastError();
                break;
            }
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            last = cand[c];
            if (ms < 0.f || t < ms) ms = t;
        }
        if (ms >= 0.f && (!best || ms < best_ms)) {
            best = cand[c];
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!best) return fail(ctx, SPAI_EINVAL, "no team size fits column problems of %d x %d", maxI, maxJ);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune.emplace(key, best);
    }
    *team = best;
    *done = last == best && sample == total;
    return SPAI_OK;
}

// device scratch released (stream-ordered) when the scope ends
struct DevScratch {
    spai_ctx ctx;
    void *p = nullptr;
    ~DevScratch() { dfree(ctx, p); }
};

spai_status run_columns(spai_ctx ctx, spai_pc pc, int mode, const double *rhs_cval)
{
    Sym *s = pc->sym;
    ColumnProblem cp{};
    cp.n = s->n;
    cp.colptr = s->a_colptr;
    cp.rowind = s->a_rowind;
    cp.cval = pc->a_cval;
    cp.Jptr = s->Jptr;
    cp.Jind = s->Jind;
    cp.Iptr = s->Iptr;
    cp.Ilist = s->Ilist;
    cp.mode = mode;
    cp.r_colptr = s->a_colptr;
    cp.r_rowind = s->a_rowind;
    cp.r_val = rhs_cval;
    cp.out_map = s->p_map;
    cp.out_val = pc->fval;
    cp.out_val32 = pc->fval32;
    cp.out_val16 = pc->fval16;
    cp.col_status = pc->status;
    cp.d_err = ctx->d_err;
    if (s->n == 0) return SPAI_OK;
    {
        const double aI = (double)s->nI / s->n, aJ = (double)s->nnzP / s->n;
        double fl = (double)s->n * (2 * aJ * aJ * (aI - aJ / 3) + 4 * aI * aJ + aJ * aJ);
        const double by = 12.0 * s->nnzA * (mode ? 2 : 1) + 8.0 * (s->n + 1) + 4.0 * s->nI + 16.0 * s->nnzP;
        const bool low = cp.out_val32 || cp.out_val16;
        // an FP32 solve reads A's values (and the right-hand side's) rounded to FP32 once here
        DevScratch scratch{ctx};
        float *v32 = nullptr;
        if (low && s->nnzA > 0) {
            spai_status st = dalloc_n(ctx, &v32, (int64_t)s->nnzA * (mode ? 2 : 1));
            if (st) return st;
            scratch.p = v32;
            KL(launch_round_f32(ctx->stream, s->nnzA, cp.cval, v32), "values in FP32");
            cp.cval32 = v32;
            if (mode) {
                KL(launch_round_f32(ctx->stream, s->nnzA, cp.r_val, v32 + s->nnzA), "values in FP32");
                cp.r_val32 = v32 + s->nnzA;
            }
        }
        auto launch = [&](int t, int64_t limit) {
            ColumnProblem part = cp;
            part.n = (int32_t)std::min<int64_t>(cp.n, limit);
            return launch_spai_columns_team(ctx->stream, part, low, s->maxI, s->maxJ, t);
        };
        int team = 0, ne[32];
        bool done = false;
        // SPAI_LS_NORMAL: the normal-equations kernels where the tile fits them, else QR
        const bool normal = pc->normal && spai_columns_ne_teams(s->maxI, s->maxJ, low, ne) > 0;
        if (normal) {  // G from the nonzeros (nnz(A) / n per column), Cholesky, two solves
            const double az = (double)s->nnzA / s->n;
            fl = (double)s->n * (az * aJ * (aJ + 1) + (mode ? 2 * az * aJ : 0) + aJ * aJ * aJ / 3 + 2 * aJ * aJ);
        }
        spai_status st = tuned_team(ctx, low, s->maxI, s->maxJ, cp.n, launch, &team, &done, normal);
        if (st) return st;
        if (!done) PKL("spai_columns", fl, by, launch(team, cp.n), "column least squares");
    }
    // first singular column (or INT_MAX)
    KL(launch_first_nonzero(ctx->stream, s->n, pc->status, ctx->d_scalar), "status scan");
    int32_t first = INT_MAX;
    spai_status st = read_i32(ctx, ctx->d_scalar, &first);
    if (st) return st;
    int h = 0;
    if ((st = read_err(ctx, &h))) return st;
    if (h) return fail(ctx, SPAI_EINVAL, "column least squares failed (device error 0x%x)", h);
    if (first != INT_MAX)
        return fail(ctx, SPAI_ESINGULAR, "column %d: rank-deficient least-squares problem (column set to 0)", first);
    return SPAI_OK;
}

// factor storage precision from the SPAI_PREC_* bits: 0 FP64, 1 FP32, 2 BF16, -1 invalid
int prec_of(int32_t flags)
{
    const int32_t p = flags & (SPAI_PREC_FP32 | SPAI_PREC_BF16);
    if (p == 0) return 0;
    if (p == SPAI_PREC_FP32) return 1;
    if (p == SPAI_PREC_BF16) return 2;
    return -1;
}

// a factor on P's pattern, or (diag) a diagonal factor of n values
spai_status pc_alloc(spai_ctx ctx, Sym *s, int prec, spai_pc *out, bool diag = false)
{
    spai_pc pc = new spai_pc_s();
    pc->ctx = ctx;
    pc->sym = s;
    pc->diag = diag;
    const int64_t nf = diag ? (int64_t)s->n : (int64_t)s->nnzP;
    spai_status st;
    if ((prec == 1   ? (st = dalloc_n(ctx, &pc->fval32, nf))
         : prec == 2 ? (st = dalloc_n(ctx, &pc->fval16, nf))
                     : (st = dalloc_n(ctx, &pc->fval, nf))) ||
        (st = dalloc_n(ctx, &pc->a_cval, s->nnzA)) || (st = dalloc_n(ctx, &pc->status, s->n))) {
        dfree(ctx, pc->fval);
        dfree(ctx, pc->fval32);
        dfree(ctx, pc->fval16);
        dfree(ctx, pc->a_cval);
        dfree(ctx, pc->status);
        delete pc;
        return st;
    }
    if (nf && pc->fval) CU(cudaMemsetAsync(pc->fval, 0, (size_t)nf * 8, ctx->stream), "memset");
    if (nf && pc->fval32) CU(cudaMemsetAsync(pc->fval32, 0, (size_t)nf * 4, ctx->stream), "memset");
    if (nf && pc->fval16) CU(cudaMemsetAsync(pc->fval16, 0, (size_t)nf * 2, ctx->stream), "memset");
    *out = pc;
    return SPAI_OK;
}

// Y = (chain of factors) X on row-major blocks; t0/t1 are n*s scratch blocks
spai_status apply_rm(spai_ctx ctx, spai_pc pc, int32_t s, const double *X, double *Y, double *t0, double *t1)
{
    std::vector<spai_pc> chain;
    for (spai_pc p = pc; p; p = p->parent) chain.push_back(p);
    const double *cur = X;
    double *bufs[2] = {t0, t1};
    for (size_t i = chain.size(); i-- > 0;) {
        spai_pc h = chain[i];
        double *dst = (i == 0) ? Y : bufs[(chain.size() - 1 - i) & 1];
        const double nz = h->sym->nnzP, nn = h->sym->n;
        if (h->diag) {
            PKL("scale_rows", nn * s, (h->fval16 ? 2.0 : h->fval32 ? 4.0 : 8.0) * nn + 16.0 * nn * s,
                launch_scale_rows(ctx->stream, s, h->sym->n, h->fval, h->fval32, h->fval16, cur, dst),
                "diagonal factor apply");
        } else if (h->fval16) {
            PKL("spmm_P", 2.0 * nz * s, 6.0 * nz + 4.0 * (nn + 1) + 16.0 * nn * s,
                launch_spmm_bf16v(ctx->stream, s, h->sym->n, h->sym->p_rowptr, h->sym->p_colind, h->fval16, cur, dst),
                "preconditioner apply");
        } else if (h->fval32) {
            PKL("spmm_P", 2.0 * nz * s, 8.0 * nz + 4.0 * (nn + 1) + 16.0 * nn * s,
                launch_spmm_f32v(ctx->stream, s, h->sym->n, h->sym->p_rowptr, h->sym->p_colind, h->fval32, cur, dst),
                "preconditioner apply");
        } else {
            PKL("spmm_P", 2.0 * nz * s, 12.0 * nz + 4.0 * (nn + 1) + 16.0 * nn * s,
                launch_spmm(ctx->stream, s, h->sym->n, h->sym->p_rowptr, h->sym->p_colind, h->fval, cur, dst),
                "preconditioner apply");
        }
        cur = dst;
    }
    return SPAI_OK;
}

// Y = P X with the FP32 operator of the mixed-precision solve: every factor's values and
// its input rounded to FP32, products and sums in FP32; the intermediate blocks of a
// factored chain are FP32 (t0 / t1), the last factor writes Y (FP32 or FP64).
template <typename YT, typename XT>
spai_status apply32(spai_ctx ctx, spai_pc pc, int32_t s, const XT *X, YT *Y, float *t0, float *t1)
{
    std::vector<spai_pc> chain;
    for (spai_pc p = pc; p; p = p->parent) chain.push_back(p);
    const void *cur = X;
    bool cur_f64 = sizeof(XT) == 8;
    float *bufs[2] = {t0, t1};
    for (size_t i = chain.size(); i-- > 0;) {
        spai_pc h = chain[i];
        F32Vals v;
        v.f32 = h->fval32;
        v.bf16 = h->fval16;
        v.f64 = (h->fval32 || h->fval16) ? nullptr : h->fval;
        const int32_t n = h->sym->n;
        const double nz = h->diag ? n : h->sym->nnzP, nn = n;
        const double vb = h->fval16 ? 2.0 : h->fval32 ? 4.0 : 8.0;
        const double xin = cur_f64 ? 8.0 : 4.0, yout = (i == 0) ? (double)sizeof(YT) : 4.0;
        const double flops = (h->diag ? 1.0 : 2.0) * nz * s;
        const double bytes = h->diag ? vb * nn + (xin + yout) * nn * s
                                     : (vb + 4.0) * nz + 4.0 * (nn + 1) + (xin + yout) * nn * s;
        int rc;
        void *dst = (i == 0) ? (void *)Y : (void *)bufs[(chain.size() - 1 - i) & 1];
        {
            ProfScope ps(ctx, h->diag ? "scale_rows32" : "spmm32_P", flops, bytes);
            if (i == 0) {
                if (h->diag)
                    rc = cur_f64 ? launch_scale_rows32(ctx->stream, s, n, v, (const double *)cur, (YT *)dst)
                                 : launch_scale_rows32(ctx->stream, s, n, v, (const float *)cur, (YT *)dst);
                else
                    rc = cur_f64 ? launch_spmm32(ctx->stream, s, n, h->sym->p_rowptr, h->sym->p_colind, v,
                                                 (const double *)cur, (YT *)dst)
                                 : launch_spmm32(ctx->stream, s, n, h->sym->p_rowptr, h->sym->p_colind, v,
                                                 (const float *)cur, (YT *)dst);
            } else {
                if (h->diag)
                    rc = cur_f64 ? launch_scale_rows32(ctx->stream, s, n, v, (const double *)cur, (float *)dst)
                                 : launch_scale_rows32(ctx->stream, s, n, v, (const float *)cur, (float *)dst);
                else
                    rc = cur_f64 ? launch_spmm32(ctx->stream, s, n, h->sym->p_rowptr, h->sym->p_colind, v,
                                                 (const double *)cur, (float *)dst)
                                 : launch_spmm32(ctx->stream, s, n, h->sym->p_rowptr, h->sym->p_colind, v,
                                                 (const float *)cur, (float *)dst);
            }
        }
        if (rc) return fail(ctx, SPAI_ECUDA, "FP32 preconditioner apply: kernel launch failed");
        cur = dst;
        cur_f64 = false;
    }
    return SPAI_OK;
}

bool valid_s(int32_t s) { return s == 1 || s == 2 || s == 4 || s == 8 || s == 16; }

// Reduction of the residual one cycle of the mixed-precision solve aims for (2^-20, sixteen
// FP32 unit roundoffs): below it the FP32 operator's rounding, not the Krylov space, limits
// what the cycle can resolve.
constexpr double kMixedCycleReduction = 0x1p-20;

// largest recycled space of block GCRO, in blocks of s columns
constexpr int kMaxRecycleBlocks = 16;

// wait settings of the next tensor-core launch on this context
TcWait tc_wait(spai_ctx ctx)
{
    TcWait w;
    w.ns = ctx->wait_ns;
    if (ctx->stall_left > 0) {
        --ctx->stall_left;
        w.stall = 1;
    }
    return w;
}

}  // namespace

// ===================================================================================
// context
// ===================================================================================
extern "C" spai_status spai_ctx_create(spai_ctx *out, void *stream, size_t mem_budget)
{
    if (!out) return SPAI_EINVAL;
    *out = nullptr;
    spai_ctx ctx = new spai_ctx_s();
    ctx->stream = (cudaStream_t)stream;
    ctx->budget = mem_budget;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, 256);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, 256);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_pinned, 4096);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_err) cudaFree(ctx->d_err);
        delete ctx;
        return SPAI_ECUDA;
    }
    ctx->d_scalar = (int32_t *)(ctx->d_err + 16);
    *out = ctx;
    return SPAI_OK;
}

extern "C" spai_status spai_ctx_destroy(spai_ctx ctx)
{
    if (!ctx) return SPAI_EINVAL;
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ws) dfree(ctx, ctx->ws);
    cudaStreamSynchronize(ctx->stream);
    prof_flush(ctx);
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    if (ctx->prof_last) cudaEventDestroy(ctx->prof_last);
    cudaFree(ctx->d_err);
    cudaFreeHost(ctx->h_pinned);
    delete ctx;
    return SPAI_OK;
}

extern "C" const char *spai_last_error(spai_ctx ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

extern "C" spai_status spai_ctx_sync(spai_ctx ctx)
{
    if (!ctx) return SPAI_EINVAL;
    CU(cudaStreamSynchronize(ctx->stream), "stream sync");
    return SPAI_OK;
}

extern "C" spai_status spai_ctx_set_wait_limit(spai_ctx ctx, double seconds)
{
    if (!ctx) return SPAI_EINVAL;
    if (!(seconds > 0.0 && seconds <= 10.0))
        return fail(ctx, SPAI_EINVAL, "wait limit must be in (0, 10] seconds");
    const double ns = seconds * 1e9;
    ctx->wait_ns = ns < 1.0 ? 1ull : (uint64_t)ns;
    return SPAI_OK;
}

extern "C" spai_status spai_ctx_inject_stall(spai_ctx ctx, int32_t count)
{
    if (!ctx) return SPAI_EINVAL;
    if (count < 0) return fail(ctx, SPAI_EINVAL, "count must be >= 0");
    ctx->stall_left = count;
    return SPAI_OK;
}

extern "C" size_t spai_ctx_mem_in_use(spai_ctx ctx)
{
    if (!ctx) return 0;
    std::lock_guard<std::mutex> lock(ctx->mu);
    return ctx->in_use;
}

extern "C" int64_t spai_launch_count(void) { return spai::launches_total(); }

namespace {
// FMA throughput of one probe kernel in TFLOP/s: a warm-up launch, then one timed launch of
// 8 blocks per SM x 256 threads x 8 chains x iters FMAs on the context's stream
template <class Launch>
spai_status measure_fma_rate(spai_ctx ctx, int iters, Launch launch, double *tflops)
{
    int sms = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "attribute");
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t a = nullptr, b = nullptr;
    CU(cudaEventCreate(&a), "event");
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return fail(ctx, SPAI_ECUDA, "event");
    }
    spai_status st = SPAI_OK;
    if (launch(blocks, threads, iters / 16) != 0 || cudaEventRecord(a, ctx->stream) != cudaSuccess ||
        launch(blocks, threads, iters) != 0 || cudaEventRecord(b, ctx->stream) != cudaSuccess ||
        cudaEventSynchronize(b) != cudaSuccess)
        st = fail(ctx, SPAI_ECUDA, "FMA probe: %s", cudaGetErrorString(cudaGetLastError()));
    float ms = 0.f;
    if (st == SPAI_OK && cudaEventElapsedTime(&ms, a, b) != cudaSuccess) st = fail(ctx, SPAI_ECUDA, "event time");
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st == SPAI_OK) *tflops = 2.0 * 8.0 * (double)blocks * threads * iters / (ms * 1e-3) / 1e12;
    return st;
}
}  // namespace

extern "C" spai_status spai_measure_fp64_rate(spai_ctx ctx, double *tflops)
{
    if (!ctx || !tflops) return fail(ctx, SPAI_EINVAL, "NULL argument");
    double *sink = (double *)ctx->d_scalar + 8;
    return measure_fma_rate(
        ctx, 4096, [&](int blocks, int threads, int it) { return launch_fp64_probe(ctx->stream, blocks, threads, it, sink); },
        tflops);
}

extern "C" spai_status spai_measure_fp32_rate(spai_ctx ctx, double *tflops)
{
    if (!ctx || !tflops) return fail(ctx, SPAI_EINVAL, "NULL argument");
    float *sink = (float *)((double *)ctx->d_scalar + 8);
    return measure_fma_rate(
        ctx, 65536, [&](int blocks, int threads, int it) { return launch_fp32_probe(ctx->stream, blocks, threads, it, sink); },
        tflops);
}

extern "C" spai_status spai_ctx_profile(spai_ctx ctx, int32_t enable)
{
    if (!ctx) return SPAI_EINVAL;
    prof_flush(ctx);
    ctx->prof_fam.clear();
    if (ctx->prof_last) ctx->prof_pool.push_back(ctx->prof_last);
    ctx->prof_last = nullptr;
    ctx->prof_on = enable != 0;
    return SPAI_OK;
}

extern "C" int32_t spai_ctx_profile_count(spai_ctx ctx)
{
    if (!ctx) return 0;
    prof_flush(ctx);
    return (int32_t)ctx->prof_fam.size();
}

extern "C" spai_status spai_ctx_profile_entry(spai_ctx ctx, int32_t i, const char **name, int64_t *launches,
                                              double *ms, double *flops, double *bytes)
{
    if (!ctx) return SPAI_EINVAL;
    prof_flush(ctx);
    if (i < 0 || i >= (int32_t)ctx->prof_fam.size()) return fail(ctx, SPAI_EINVAL, "profile index out of range");
    const auto &f = ctx->prof_fam[i];
    if (name) *name = f.name.c_str();
    if (launches) *launches = f.launches;
    if (ms) *ms = f.ms;
    if (flops) *flops = f.flops;
    if (bytes) *bytes = f.bytes;
    return SPAI_OK;
}

// ===================================================================================
// affine assembly
// ===================================================================================
extern "C" spai_status spai_affine_create(spai_ctx ctx, int32_t nterms, const spai_csr *terms, spai_affine *out)
{
    if (!ctx || !out || !terms) return fail(ctx, SPAI_EINVAL, "NULL argument");
    *out = nullptr;
    if (nterms < 1 || nterms > kMaxTerms) return fail(ctx, SPAI_EINVAL, "nterms must be in 1..%d", kMaxTerms);
    const int32_t n = terms[0].n;
    for (int t = 0; t < nterms; ++t) {
        spai_status st = check_csr_args(ctx, &terms[t], "term");
        if (st) return st;
        if (terms[t].n != n) return fail(ctx, SPAI_EINVAL, "term %d has n=%d, expected %d", t, terms[t].n, n);
    }
    // copy every term to library memory (host or device source)
    std::vector<int32_t *> rp(nterms, nullptr), ci(nterms, nullptr);
    std::vector<double *> va(nterms, nullptr);
    auto cleanup = [&]() {
        for (int t = 0; t < nterms; ++t) { dfree(ctx, rp[t]); dfree(ctx, ci[t]); dfree(ctx, va[t]); }
    };
    spai_status st = SPAI_OK;
    for (int t = 0; t < nterms && !st; ++t) {
        const spai_csr &A = terms[t];
        if ((st = dalloc_n(ctx, &rp[t], (int64_t)n + 1)) || (st = dalloc_n(ctx, &ci[t], A.nnz)) ||
            (st = dalloc_n(ctx, &va[t], A.nnz)))
            break;
        cudaError_t e = cudaMemcpyAsync(rp[t], A.rowptr, ((size_t)n + 1) * 4, cudaMemcpyDefault, ctx->stream);
        if (e == cudaSuccess && A.nnz)
            e = cudaMemcpyAsync(ci[t], A.colind, (size_t)A.nnz * 4, cudaMemcpyDefault, ctx->stream);
        if (e == cudaSuccess && A.nnz)
            e = cudaMemcpyAsync(va[t], A.val, (size_t)A.nnz * 8, cudaMemcpyDefault, ctx->stream);
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "copy term");
        if (!st && n > 0) {
            if (launch_validate_csr(ctx->stream, n, A.nnz, rp[t], ci[t], ctx->d_err)) st = fail(ctx, SPAI_ECUDA, "validate");
        }
    }
    int h = 0;
    if (!st) st = read_err(ctx, &h);
    if (!st && h) st = fail(ctx, SPAI_EINVAL, "a term is not a valid CSR matrix (device error 0x%x)", h);
    if (st) { cleanup(); return st; }
    TermPtrs tp{};
    for (int t = 0; t < nterms; ++t) { tp.rowptr[t] = rp[t]; tp.colind[t] = ci[t]; tp.val[t] = va[t]; }
    spai_affine aff = new spai_affine_s();
    aff->ctx = ctx;
    aff->n = n;
    aff->T = nterms;
    int32_t *counts = nullptr;
    void *stemp = nullptr;
    st = dalloc_n(ctx, &aff->rowptr, (int64_t)n + 1);
    if (!st) st = dalloc_n(ctx, &counts, (int64_t)n + 1);
    if (!st) st = dalloc(ctx, &stemp, scan_temp_bytes(n));
    if (!st && n > 0) {
        if (launch_union_count(ctx->stream, n, nterms, tp, counts) ||
            launch_exclusive_scan(ctx->stream, counts, aff->rowptr, n, stemp, ctx->d_err))
            st = fail(ctx, SPAI_ECUDA, "union pattern");
    } else if (!st) {
        cudaMemsetAsync(aff->rowptr, 0, 4, ctx->stream);
    }
    int32_t nnzU = 0;
    if (!st) st = read_i32(ctx, aff->rowptr + n, &nnzU);
    if (!st) st = read_err(ctx, &h);
    if (!st && h) st = fail(ctx, SPAI_EINVAL, "union pattern exceeds 2^31 entries");
    if (!st) { aff->nnz = nnzU; st = dalloc_n(ctx, &aff->colind, nnzU); }
    if (!st) st = dalloc_n(ctx, &aff->aligned, (int64_t)nterms * nnzU);
    if (!st && n > 0 && launch_union_fill(ctx->stream, n, nterms, tp, aff->rowptr, aff->colind, aff->aligned, nnzU))
        st = fail(ctx, SPAI_ECUDA, "union fill");
    if (!st) { cudaError_t e = cudaStreamSynchronize(ctx->stream); if (e) st = cuda_fail(ctx, e, "sync"); }
    dfree(ctx, counts);
    dfree(ctx, stemp);
    cleanup();
    if (st) { spai_affine_destroy(aff); return st; }
    *out = aff;
    return SPAI_OK;
}

extern "C" spai_status spai_affine_pattern(spai_affine aff, int32_t *n, int32_t *nnz, const int32_t **rowptr,
                                           const int32_t **colind)
{
    if (!aff) return SPAI_EINVAL;
    if (n) *n = aff->n;
    if (nnz) *nnz = (int32_t)aff->nnz;
    if (rowptr) *rowptr = aff->rowptr;
    if (colind) *colind = aff->colind;
    return SPAI_OK;
}

extern "C" spai_status spai_assemble(spai_ctx ctx, spai_affine aff, const double *coef, double *val_out)
{
    if (!ctx || !aff || !coef || (!val_out && aff->nnz)) return fail(ctx, SPAI_EINVAL, "NULL argument");
    if (aff->nnz == 0) return SPAI_OK;
    if (!is_device_ptr(val_out)) return fail(ctx, SPAI_EINVAL, "val_out must be device memory");
    PKL("assemble", 2.0 * aff->T * aff->nnz, 8.0 * (aff->T + 1) * aff->nnz,
        launch_assemble(ctx->stream, aff->nnz, aff->T, aff->aligned, coef, val_out), "assemble");
    return SPAI_OK;
}

// Sec. 1.1 Eqs. (3)-(9) with Rayleigh damping (Sec. 3).  Host code is compiled with
// -ffp-contract=off, so every product and sum below is rounded on its own on every host.
extern "C" spai_status spai_shifted_coefficients(int32_t np, const double *p, double s, double alpha, double beta,
                                                 double *coef)
{
    if (np < 0 || np > kMaxTerms - 2 || (np > 0 && !p) || !coef) return SPAI_EINVAL;
    if (!std::isfinite(s) || !std::isfinite(alpha) || !std::isfinite(beta)) return SPAI_EINVAL;
    for (int i = 0; i < np; ++i)
        if (!std::isfinite(p[i])) return SPAI_EINVAL;
    const double ss = s * s, as = alpha * s, bs = beta * s;
    const double cK = 1.0 + bs;
    coef[0] = ss + as;
    coef[1] = cK;
    for (int i = 0; i < np; ++i) coef[2 + i] = cK * p[i];
    return SPAI_OK;
}

extern "C" spai_status spai_assemble_shifted(spai_ctx ctx, spai_affine aff, double s, int32_t np, const double *p,
                                             double alpha, double beta, double *val_out)
{
    if (!ctx || !aff) return fail(ctx, SPAI_EINVAL, "NULL argument");
    if (np + 2 != aff->T)
        return fail(ctx, SPAI_EINVAL, "the affine handle has %d terms; (M, K_0, ..., K_np) needs np + 2 = %d", aff->T,
                    np + 2);
    double coef[kMaxTerms];
    if (spai_shifted_coefficients(np, p, s, alpha, beta, coef))
        return fail(ctx, SPAI_EINVAL, "shifted coefficients: bad parameters (NULL or non-finite)");
    return spai_assemble(ctx, aff, coef, val_out);
}

extern "C" spai_status spai_affine_export(spai_ctx ctx, spai_affine aff, int32_t *rowptr, int32_t *colind)
{
    if (!ctx || !aff) return fail(ctx, SPAI_EINVAL, "NULL argument");
    if (rowptr)
        CU(cudaMemcpyAsync(rowptr, aff->rowptr, ((size_t)aff->n + 1) * 4, cudaMemcpyDefault, ctx->stream), "export");
    if (colind && aff->nnz)
        CU(cudaMemcpyAsync(colind, aff->colind, (size_t)aff->nnz * 4, cudaMemcpyDefault, ctx->stream), "export");
    CU(cudaStreamSynchronize(ctx->stream), "sync");
    return SPAI_OK;
}

extern "C" spai_status spai_affine_destroy(spai_affine aff)
{
    if (!aff) return SPAI_EINVAL;
    spai_ctx ctx = aff->ctx;
    dfree(ctx, aff->rowptr);
    dfree(ctx, aff->colind);
    dfree(ctx, aff->aligned);
    delete aff;
    return SPAI_OK;
}

// ===================================================================================
// SPAI build / update
// ===================================================================================
extern "C" spai_status spai_build(spai_ctx ctx, const spai_csr *A, int32_t pattern_kind, spai_pc *out)
{
    if (!ctx || !out) return fail(ctx, SPAI_EINVAL, "NULL argument");
    *out = nullptr;
    const int prec = prec_of(pattern_kind);
    if (prec < 0) return fail(ctx, SPAI_EINVAL, "SPAI_PREC_FP32 and SPAI_PREC_BF16 are exclusive");
    const bool normal = (pattern_kind & SPAI_LS_NORMAL) != 0;
    pattern_kind &= ~(SPAI_PREC_FP32 | SPAI_PREC_BF16 | SPAI_LS_NORMAL);
    if (pattern_kind != SPAI_PATTERN_A && pattern_kind != SPAI_PATTERN_A2)
        return fail(ctx, SPAI_EINVAL, "unknown pattern kind %d", pattern_kind);
    spai_status st = validate_device_csr(ctx, A, "A");
    if (st) return st;
    Sym *s = nullptr;
    if ((st = sym_create(ctx, A, pattern_kind, &s))) return st;
    spai_pc pc = nullptr;
    if ((st = pc_alloc(ctx, s, prec, &pc))) { sym_release(s); return st; }
    pc->root = pc;
    pc->normal = normal;
    if (s->nnzA)
        PKL("gather_csc", 0.0, 20.0 * s->nnzA, launch_gather_f64(ctx->stream, s->nnzA, s->a_perm, A->val, pc->a_cval),
            "gather values");
    st = run_columns(ctx, pc, 0, nullptr);
    if (st && st != SPAI_ESINGULAR) { spai_pc_destroy(pc); return st; }
    *out = pc;
    return st;
}

namespace {

// Gives s (an analysis of pattern kind A) the column pattern (Jptr, Jind) instead, taking
// ownership of both arrays on success: the row pattern of P and its position map
// (transposition of J), I_k = union of rows(A(:,j)) over J_k, and the sizes.
spai_status sym_set_pattern(spai_ctx ctx, Sym *s, int32_t *Jptr, int32_t *Jind, int32_t nnzP)
{
    cudaStream_t cs = ctx->stream;
    const int32_t n = s->n;
    spai_status st = SPAI_OK;
    int32_t *p_rowptr = nullptr, *p_colind = nullptr, *p_map = nullptr, *perm = nullptr, *Iptr = nullptr,
            *Ilist = nullptr, *counts = nullptr, *d_max = nullptr;
    void *temp = nullptr;
    auto done = [&](spai_status rc) {
        dfree(ctx, perm);
        dfree(ctx, temp);
        dfree(ctx, counts);
        dfree(ctx, d_max);
        if (rc) {
            dfree(ctx, p_rowptr);
            dfree(ctx, p_colind);
            dfree(ctx, p_map);
            dfree(ctx, Iptr);
            dfree(ctx, Ilist);
        }
        return rc;
    };
#define TRY(x)                                         \
    do {                                               \
        if ((st = (x)) != SPAI_OK) return done(st);    \
    } while (0)
#define TRYK(call, what)                                                                                     \
    do {                                                                                                     \
        if ((call) != 0)                                                                                     \
            return done(fail(ctx, SPAI_ECUDA, "%s: kernel launch failed (%s)", what,                         \
                             cudaGetErrorString(cudaGetLastError())));                                       \
    } while (0)
    const size_t tb = std::max(transpose_temp_bytes(n, std::max(nnzP, 1)), scan_temp_bytes(n));
    TRY(dalloc(ctx, &temp, tb));
    TRY(dalloc_n(ctx, &p_rowptr, (int64_t)n + 1));
    TRY(dalloc_n(ctx, &p_colind, nnzP));
    TRY(dalloc_n(ctx, &p_map, nnzP));
    TRY(dalloc_n(ctx, &perm, nnzP));
    TRY(dalloc_n(ctx, &counts, (int64_t)n + 1));
    TRY(dalloc_n(ctx, &d_max, 2));
    TRYK(launch_transpose(cs, n, nnzP, Jptr, Jind, p_rowptr, p_colind, perm, temp, ctx->d_err), "transpose pattern");
    TRYK(launch_invert_perm(cs, nnzP, perm, p_map), "invert");
    TRYK(launch_max_i32_diff(cs, n, Jptr, d_max), "max |J|");
    int32_t maxJ = 0;
    TRY(read_i32(ctx, d_max, &maxJ));
    if (maxJ > colunion_max_lists())
        return done(fail(ctx, SPAI_EINVAL, "a column pattern has %d entries; at most %d are supported", maxJ,
                         colunion_max_lists()));
    TRY(dalloc_n(ctx, &Iptr, (int64_t)n + 1));
    TRYK(launch_colunion_count(cs, n, maxJ, Jptr, Jind, s->a_colptr, s->a_rowind, counts, ctx->d_err), "I count");
    TRYK(launch_exclusive_scan(cs, counts, Iptr, n, temp, ctx->d_err), "scan");
    int32_t nI = 0;
    TRY(read_i32(ctx, Iptr + n, &nI));
    TRY(dalloc_n(ctx, &Ilist, nI));
    TRYK(launch_colunion_fill(cs, n, maxJ, Jptr, Jind, s->a_colptr, s->a_rowind, Iptr, Ilist, ctx->d_err), "I fill");
    TRYK(launch_max_i32_diff(cs, n, Iptr, d_max + 1), "max |I|");
    int32_t maxI = 0;
    TRY(read_i32(ctx, d_max + 1, &maxI));
    int herr = 0;
    TRY(read_err(ctx, &herr));
    if (herr) return done(fail(ctx, SPAI_EINVAL, "pattern analysis failed (device error 0x%x)", herr));
    if (!spai_columns_fit(maxI, maxJ))
        return done(fail(ctx, SPAI_EINVAL, "column problem of %d x %d exceeds the shared-memory tile", maxI, maxJ));
#undef TRY
#undef TRYK
    // adopt the new pattern (pattern kind A aliases J and the row pattern to A's arrays)
    if (!s->alias) {
        dfree(ctx, s->Jptr);
        dfree(ctx, s->Jind);
        dfree(ctx, s->p_rowptr);
        dfree(ctx, s->p_colind);
        dfree(ctx, s->p_map);
    }
    dfree(ctx, s->Iptr);
    dfree(ctx, s->Ilist);
    s->alias = false;
    s->Jptr = Jptr;
    s->Jind = Jind;
    s->nnzP = nnzP;
    s->p_rowptr = p_rowptr;
    s->p_colind = p_colind;
    s->p_map = p_map;
    s->Iptr = Iptr;
    s->Ilist = Ilist;
    s->nI = nI;
    s->maxI = maxI;
    s->maxJ = maxJ;
    return done(SPAI_OK);
}

}  // namespace

extern "C" spai_status spai_build_adaptive(spai_ctx ctx, const spai_csr *A, const spai_adaptive_opts *opts,
                                           int32_t flags, spai_pc *out)
{
    if (!ctx || !out) return fail(ctx, SPAI_EINVAL, "NULL argument");
    *out = nullptr;
    spai_adaptive_opts o{1e-4, 5, 5, 128, 0};
    if (opts) o = *opts;
    const int prec = prec_of(flags);
    if (prec < 0 || (flags & ~(SPAI_PREC_FP32 | SPAI_PREC_BF16)))
        return fail(ctx, SPAI_EINVAL, "flags: SPAI_PREC_FP32 or SPAI_PREC_BF16 (exclusive) or 0");
    if (!(o.eps >= 0.0) || o.max_steps < 0 || o.max_new < 1 || o.max_rows < 1 ||
        o.max_rows > adaptive_max_rows() || 1 + (int64_t)o.max_steps * o.max_new > adaptive_max_cols())
        return fail(ctx, SPAI_EINVAL, "adaptive options: eps >= 0, max_new >= 1, 1 <= max_rows <= %d, "
                    "1 + max_steps * max_new <= %d", adaptive_max_rows(), adaptive_max_cols());
    spai_status st = validate_device_csr(ctx, A, "A");
    if (st) return st;
    Sym *s = nullptr;
    if ((st = sym_create(ctx, A, SPAI_PATTERN_A, &s))) return st;
    const int32_t n = s->n;
    double *cval = nullptr, *cn = nullptr;
    int32_t *outJ = nullptr, *cnt = nullptr, *Jptr = nullptr, *Jind = nullptr;
    void *temp = nullptr;
    auto bail = [&](spai_status rc) {
        dfree(ctx, cval);
        dfree(ctx, cn);
        dfree(ctx, outJ);
        dfree(ctx, cnt);
        dfree(ctx, temp);
        dfree(ctx, Jptr);
        dfree(ctx, Jind);
        sym_release(s);
        return rc;
    };
    if (n > 0) {
        const int mc = adaptive_max_cols();
        if ((st = dalloc_n(ctx, &cval, std::max(s->nnzA, 1))) || (st = dalloc_n(ctx, &cn, n)) ||
            (st = dalloc_n(ctx, &outJ, (int64_t)n * mc)) || (st = dalloc_n(ctx, &cnt, (int64_t)n + 1)) ||
            (st = dalloc(ctx, &temp, scan_temp_bytes(n))) || (st = dalloc_n(ctx, &Jptr, (int64_t)n + 1)))
            return bail(st);
        if (s->nnzA && launch_gather_f64(ctx->stream, s->nnzA, s->a_perm, A->val, cval))
            return bail(fail(ctx, SPAI_ECUDA, "gather values: kernel launch failed"));
        if (launch_colnorm2_csc(ctx->stream, n, s->a_colptr, cval, cn))
            return bail(fail(ctx, SPAI_ECUDA, "column norms: kernel launch failed"));
        AdaptiveProblem ap{};
        ap.n = n;
        ap.colptr = s->a_colptr;
        ap.rowind = s->a_rowind;
        ap.cval = cval;
        ap.rowptr = s->a_rowptr;
        ap.colind = s->a_colind;
        ap.colnorm2 = cn;
        ap.eps = o.eps;
        ap.max_steps = o.max_steps;
        ap.max_new = o.max_new;
        ap.max_rows = o.max_rows;
        ap.out_J = outJ;
        ap.out_count = cnt;
        ap.d_err = ctx->d_err;
        {
            ProfScope ps_(ctx, "adaptive_pattern", 0.0, 0.0);
            if (launch_adaptive_pattern(ctx->stream, ap))
                return bail(fail(ctx, SPAI_ECUDA, "adaptive pattern: kernel launch failed (%s)",
                                 cudaGetErrorString(cudaGetLastError())));
        }
        if (launch_exclusive_scan(ctx->stream, cnt, Jptr, n, temp, ctx->d_err))
            return bail(fail(ctx, SPAI_ECUDA, "scan: kernel launch failed"));
        int32_t nnzP = 0;
        if ((st = read_i32(ctx, Jptr + n, &nnzP))) return bail(st);
        int herr = 0;
        if ((st = read_err(ctx, &herr))) return bail(st);
        if (herr) return bail(fail(ctx, SPAI_EINVAL, "adaptive pattern failed (device error 0x%x)", herr));
        if ((st = dalloc_n(ctx, &Jind, std::max(nnzP, 1)))) return bail(st);
        if (launch_compact_lists(ctx->stream, n, outJ, mc, Jptr, Jind))
            return bail(fail(ctx, SPAI_ECUDA, "compaction: kernel launch failed"));
        if ((st = sym_set_pattern(ctx, s, Jptr, Jind, nnzP))) return bail(st);
        Jptr = Jind = nullptr;  // owned by s now
        dfree(ctx, cval);
        dfree(ctx, cn);
        dfree(ctx, outJ);
        dfree(ctx, cnt);
        dfree(ctx, temp);
        cval = cn = nullptr;
        outJ = cnt = nullptr;
        temp = nullptr;
    }
    spai_pc pc = nullptr;
    if ((st = pc_alloc(ctx, s, prec, &pc))) return bail(st);
    pc->root = pc;
    if (s->nnzA)
        PKL("gather_csc", 0.0, 20.0 * s->nnzA, launch_gather_f64(ctx->stream, s->nnzA, s->a_perm, A->val, pc->a_cval),
            "gather values");
    st = run_columns(ctx, pc, 0, nullptr);
    if (st && st != SPAI_ESINGULAR) {
        spai_pc_destroy(pc);
        return st;
    }
    *out = pc;
    return st;
}

extern "C" spai_status spai_update(spai_ctx ctx, spai_pc base, const spai_csr *A_new, int32_t approach, spai_pc *out)
{
    if (!ctx || !out || !base) return fail(ctx, SPAI_EINVAL, "NULL argument");
    *out = nullptr;
    const int prec = prec_of(approach);
    if (prec < 0) return fail(ctx, SPAI_EINVAL, "SPAI_PREC_FP32 and SPAI_PREC_BF16 are exclusive");
    const bool diag = (approach & SPAI_UPDATE_DIAGONAL) != 0;
    const bool normal = (approach & SPAI_LS_NORMAL) != 0;
    approach &= ~(SPAI_PREC_FP32 | SPAI_PREC_BF16 | SPAI_UPDATE_DIAGONAL | SPAI_LS_NORMAL);
    if (approach != SPAI_UPDATE_FIRST && approach != SPAI_UPDATE_CHAINED)
        return fail(ctx, SPAI_EINVAL, "unknown update approach %d", approach);
    spai_status st = check_csr_args(ctx, A_new, "A_new");
    if (st) return st;
    Sym *s = base->sym;
    if (A_new->n != s->n || A_new->nnz != s->nnzA)
        return fail(ctx, SPAI_EINVAL, "A_new (n=%d, nnz=%d) does not have the base pattern (n=%d, nnz=%d)",
                    A_new->n, A_new->nnz, s->n, s->nnzA);
    if (s->n && (!is_device_ptr(A_new->rowptr) || (s->nnzA && (!is_device_ptr(A_new->colind) || !is_device_ptr(A_new->val)))))
        return fail(ctx, SPAI_EINVAL, "A_new: arrays must be device memory");
    if (s->n) {
        KL(launch_compare_i32(ctx->stream, (int64_t)s->n + 1, A_new->rowptr, s->a_rowptr, ctx->d_err), "compare");
        KL(launch_compare_i32(ctx->stream, s->nnzA, A_new->colind, s->a_colind, ctx->d_err), "compare");
        int h = 0;
        if ((st = read_err(ctx, &h))) return st;
        if (h) return fail(ctx, SPAI_EINVAL, "A_new does not have the base matrix's sparsity pattern");
    }
    spai_pc pc = nullptr;
    if ((st = pc_alloc(ctx, s, prec, &pc, diag))) return st;
    pc->normal = normal;
    s->refs++;
    spai_pc from = (approach == SPAI_UPDATE_FIRST) ? base->root : base;
    pc->parent = from;
    pc->root = base->root;
    pc->depth = from->depth + 1;
    if (s->nnzA)
        PKL("gather_csc", 0.0, 20.0 * s->nnzA,
            launch_gather_f64(ctx->stream, s->nnzA, s->a_perm, A_new->val, pc->a_cval), "gather values");
    if (diag) {
        // one unknown per column: rows I_k = rows(A(l)(:,k)), A(1)'s column on the same pattern
        if (s->n)
            PKL("spai_columns", 4.0 * s->nnzA + s->n, 16.0 * s->nnzA + 4.0 * (s->n + 1) + 12.0 * s->n,
                launch_diag_update(ctx->stream, s->n, s->a_colptr, pc->a_cval, from->a_cval, pc->fval, pc->fval32,
                                   pc->fval16, pc->status),
                "diagonal update");
        st = SPAI_OK;
        if (s->n) {
            KL(launch_first_nonzero(ctx->stream, s->n, pc->status, ctx->d_scalar), "status scan");
            int32_t first = INT_MAX;
            if ((st = read_i32(ctx, ctx->d_scalar, &first))) { spai_pc_destroy(pc); return st; }
            if (first != INT_MAX)
                st = fail(ctx, SPAI_ESINGULAR, "column %d: zero column, diagonal update entry set to 0", first);
        }
    } else {
        st = run_columns(ctx, pc, 1, from->a_cval);
    }
    if (st && st != SPAI_ESINGULAR) { spai_pc_destroy(pc); return st; }
    *out = pc;
    return st;
}

// ===================================================================================
// Batched build: many independent systems at once
// ===================================================================================
namespace {

spai_status run_columns_batch(spai_ctx ctx, int32_t nsys, spai_pc *pcs)
{
    // buckets of systems whose problems share a tile: (low precision + 2 for the normal
    // equations, max |J|, max |I| rounded up to 8)
    std::map<std::tuple<int, int, int>, std::vector<int>> buckets;
    for (int i = 0; i < nsys; ++i) {
        const Sym *s = pcs[i]->sym;
        if (s->n == 0) continue;
        buckets[std::make_tuple((pcs[i]->fval ? 0 : 1) + (pcs[i]->normal ? 2 : 0), s->maxJ, (s->maxI + 7) / 8 * 8)]
            .push_back(i);
    }
    spai_status st = SPAI_OK;
    for (auto &b : buckets) {
        const int low = std::get<0>(b.first) & 1, maxJ = std::get<1>(b.first);
        const bool want_normal = std::get<0>(b.first) >= 2;
        const std::vector<int> &mem = b.second;
        const int m = (int)mem.size();
        int maxI = 0;  // tile rows: the bucket's largest |I_k| (its class, a multiple of 8, keys the tuning)
        std::vector<ColumnProblem> tab((size_t)m);
        std::vector<int64_t> start((size_t)m + 1, 0);
        double fl = 0.0, by = 0.0;
        for (int t = 0; t < m; ++t) {
            spai_pc pc = pcs[mem[t]];
            const Sym *s = pc->sym;
            maxI = std::max(maxI, s->maxI);
            ColumnProblem &cp = tab[t];
            cp = ColumnProblem{};
            cp.n = s->n;
            cp.colptr = s->a_colptr;
            cp.rowind = s->a_rowind;
            cp.cval = pc->a_cval;
            cp.Jptr = s->Jptr;
            cp.Jind = s->Jind;
            cp.Iptr = s->Iptr;
            cp.Ilist = s->Ilist;
            cp.mode = 0;
            cp.r_colptr = s->a_colptr;
            cp.r_rowind = s->a_rowind;
            cp.out_map = s->p_map;
            cp.out_val = pc->fval;
            cp.out_val32 = pc->fval32;
            cp.out_val16 = pc->fval16;
            cp.col_status = pc->status;
            cp.d_err = ctx->d_err;
            start[t + 1] = start[t] + s->n;
            const double aI = (double)s->nI / s->n, aJ = (double)s->nnzP / s->n;
            fl += (double)s->n * (2 * aJ * aJ * (aI - aJ / 3) + 4 * aI * aJ + aJ * aJ);
            by += 12.0 * s->nnzA + 8.0 * (s->n + 1) + 4.0 * s->nI + 16.0 * s->nnzP;
        }
        // FP32 solves read A's values rounded to FP32 once here (all systems of the bucket)
        DevScratch scratch{ctx};
        if (low) {
            std::vector<int64_t> vstart((size_t)m + 1, 0);
            std::vector<const double *> vsrc((size_t)m);
            for (int t = 0; t < m; ++t) {
                vstart[t + 1] = vstart[t] + pcs[mem[t]]->sym->nnzA;
                vsrc[t] = tab[t].cval;
            }
            const int64_t tot = vstart[m];
            const size_t o_start = ((size_t)tot * 4 + 255) / 256 * 256, o_src = o_start + ((size_t)m + 1) * 8;
            char *sc = nullptr;
            if ((st = dalloc(ctx, (void **)&sc, o_src + (size_t)m * 8))) return st;
            scratch.p = sc;
            float *v32 = (float *)sc;
            CU(cudaMemcpyAsync(sc + o_start, vstart.data(), ((size_t)m + 1) * 8, cudaMemcpyHostToDevice, ctx->stream),
               "segments");
            CU(cudaMemcpyAsync(sc + o_src, vsrc.data(), (size_t)m * 8, cudaMemcpyHostToDevice, ctx->stream), "segments");
            KL(launch_round_seg(ctx->stream, m, tot, (const int64_t *)(sc + o_start), (const double *const *)(sc + o_src),
                                v32),
               "values in FP32");
            for (int t = 0; t < m; ++t) tab[t].cval32 = v32 + vstart[t];
        }
        ColumnProblem *d_tab = nullptr;
        int64_t *d_start = nullptr;
        if ((st = dalloc_n(ctx, &d_tab, m)) || (st = dalloc_n(ctx, &d_start, (int64_t)m + 1))) {
            dfree(ctx, d_tab);
            return st;
        }
        CU(cudaMemcpyAsync(d_tab, tab.data(), sizeof(ColumnProblem) * m, cudaMemcpyHostToDevice, ctx->stream), "table");
        CU(cudaMemcpyAsync(d_start, start.data(), sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, ctx->stream),
           "table");
        const ColumnBatch bt{d_tab, d_start, m, start[m]};
        auto launch = [&](int t, int64_t limit) {
            ColumnBatch part = bt;
            part.total = std::min(bt.total, limit);
            return launch_spai_columns_batch(ctx->stream, part, low != 0, maxI, maxJ, t);
        };
        int team = 0, ne[32];
        bool done = false;
        const bool normal = want_normal && spai_columns_ne_teams(maxI, maxJ, low != 0, ne) > 0;
        if ((st = tuned_team(ctx, low != 0, maxI, maxJ, bt.total, launch, &team, &done, normal))) {
            dfree(ctx, d_tab);
            dfree(ctx, d_start);
            return st;
        }
        if (done) {  // the result of the chosen candidate is already in place
            dfree(ctx, d_tab);
            dfree(ctx, d_start);
            continue;
        }
        PKL("spai_columns", fl, by, launch_spai_columns_batch(ctx->stream, bt, low != 0, maxI, maxJ, team),
            "batched column least squares");
        dfree(ctx, d_tab);
        dfree(ctx, d_start);
    }
    // first singular column of every system (INT_MAX if none), one read-back for all
    // (a segmented scan over the systems' status arrays: two launches for the whole batch)
    std::vector<int64_t> sstart((size_t)nsys + 1, 0);
    std::vector<const int32_t *> sptr((size_t)nsys);
    for (int i = 0; i < nsys; ++i) {
        sstart[i + 1] = sstart[i] + pcs[i]->sym->n;
        sptr[i] = pcs[i]->status;
    }
    const size_t o_ptr = ((size_t)nsys + 1) * 8, o_first = o_ptr + (size_t)nsys * 8;
    char *d_scan = nullptr;
    if ((st = dalloc(ctx, (void **)&d_scan, o_first + (size_t)nsys * 4))) return st;
    int32_t *d_first = (int32_t *)(d_scan + o_first);
    std::vector<int32_t> first((size_t)nsys);
    cudaError_t ce = cudaMemcpyAsync(d_scan, sstart.data(), o_ptr, cudaMemcpyHostToDevice, ctx->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(d_scan + o_ptr, sptr.data(), (size_t)nsys * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (ce == cudaSuccess &&
        launch_first_nonzero_seg(ctx->stream, nsys, sstart[nsys], (const int64_t *)d_scan,
                                 (const int32_t *const *)(d_scan + o_ptr), d_first))
        ce = cudaGetLastError();
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(first.data(), d_first, (size_t)nsys * 4, cudaMemcpyDeviceToHost, ctx->stream);
    int h = 0;
    st = ce == cudaSuccess ? read_err(ctx, &h) : cuda_fail(ctx, ce, "status scan");
    dfree(ctx, d_scan);
    if (st) return st;
    if (h) return fail(ctx, SPAI_EINVAL, "batched column least squares failed (device error 0x%x)", h);
    for (int i = 0; i < nsys; ++i)
        if (pcs[i]->sym->n && first[i] != INT_MAX)
            return fail(ctx, SPAI_ESINGULAR, "system %d, column %d: rank-deficient least-squares problem (column set "
                        "to 0)", i, first[i]);
    return SPAI_OK;
}

// Pattern analyses and factor storage of a batch of systems at once: the systems are
// stacked into one block-diagonal matrix (global indices), each phase of the analysis --
// transposition, the column lists of the unions, the unions J_k and I_k, the row pattern of
// P -- runs once over the stacked matrix (its unions never leave a diagonal block), and the
// per-system arrays (local indices, as spai_build makes them) are carved from one arena by
// a single unstacking launch.  The CUDA calls do not grow with nsys except for a few small
// host-to-device tables.  Every system must have n >= 1.
spai_status build_batch_stacked(spai_ctx ctx, int32_t nsys, const spai_csr *A, const int32_t *kinds,
                                const int32_t *precs, std::vector<spai_pc> &pcs)
{
    cudaStream_t cs = ctx->stream;
    spai_status st = SPAI_OK;
    std::vector<int64_t> off((size_t)nsys + 1, 0), nzoff((size_t)nsys + 1, 0);
    for (int i = 0; i < nsys; ++i) {
        off[i + 1] = off[i] + A[i].n;
        nzoff[i + 1] = nzoff[i] + A[i].nnz;
    }
    const int64_t ntot = off[nsys], nnz = nzoff[nsys];
    if (ntot >= INT32_MAX || nnz >= INT32_MAX)
        return fail(ctx, SPAI_EINVAL, "the stacked batch exceeds 2^31 rows or nonzeros");
    std::vector<void *> tmp;  // stacked temporaries, freed at the end
    auto cleanup = [&](spai_status rc) {  // on failure the handles made so far go too
        for (void *p : tmp) dfree(ctx, p);
        if (rc != SPAI_OK) {
            for (spai_pc pc : pcs)
                if (pc) spai_pc_destroy(pc);
            pcs.clear();
        }
        return rc;
    };
    auto talloc = [&](auto **p, int64_t count) -> spai_status {
        spai_status s2 = dalloc_n(ctx, p, count);
        if (!s2) tmp.push_back((void *)*p);
        return s2;
    };
#define TRY(x)                                          \
    do {                                                \
        if ((st = (x)) != SPAI_OK) return cleanup(st);  \
    } while (0)
#define TRYC(call, what)                                            \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cleanup(cuda_fail(ctx, e_, what)); \
    } while (0)
#define TRYK(call, what)                                                                                    \
    do {                                                                                                    \
        if ((call) != 0)                                                                                    \
            return cleanup(fail(ctx, SPAI_ECUDA, "%s: kernel launch failed (%s)", what,                     \
                                cudaGetErrorString(cudaGetLastError())));                                   \
    } while (0)
    // ---- system table: offsets, kinds, the callers' pattern arrays
    int64_t *d_off = nullptr, *d_nzoff = nullptr;
    int32_t *d_kind = nullptr;
    const int32_t **d_rp = nullptr, **d_ci = nullptr;
    TRY(talloc(&d_off, nsys + 1));
    TRY(talloc(&d_nzoff, nsys + 1));
    TRY(talloc(&d_kind, nsys));
    TRY(talloc(&d_rp, nsys));
    TRY(talloc(&d_ci, nsys));
    {
        std::vector<const int32_t *> hrp((size_t)nsys), hci((size_t)nsys);
        for (int i = 0; i < nsys; ++i) {
            hrp[i] = A[i].rowptr;
            hci[i] = A[i].colind;
        }
        TRYC(cudaMemcpyAsync(d_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice, cs), "table");
        TRYC(cudaMemcpyAsync(d_nzoff, nzoff.data(), nzoff.size() * 8, cudaMemcpyHostToDevice, cs), "table");
        TRYC(cudaMemcpyAsync(d_kind, kinds, (size_t)nsys * 4, cudaMemcpyHostToDevice, cs), "table");
        TRYC(cudaMemcpyAsync(d_rp, hrp.data(), (size_t)nsys * 8, cudaMemcpyHostToDevice, cs), "table");
        TRYC(cudaMemcpyAsync(d_ci, hci.data(), (size_t)nsys * 8, cudaMemcpyHostToDevice, cs), "table");
        TRYC(cudaStreamSynchronize(cs), "sync");  // the host tables are read by the copies above
    }
    // ---- stacked CSR (checked per system), its transpose
    int32_t *rp = nullptr, *ci = nullptr, *colptr = nullptr, *rowind = nullptr, *perm = nullptr;
    void *ttemp = nullptr;
    TRY(talloc(&rp, ntot + 1));
    TRY(talloc(&ci, nnz));
    TRY(talloc(&colptr, ntot + 1));
    TRY(talloc(&rowind, nnz));
    TRY(talloc(&perm, nnz));
    {
        ProfScope ps_(ctx, "analysis:stack", 0.0, 0.0);
        TRYK(launch_stack_csr(cs, nsys, ntot, nnz, d_off, d_nzoff, d_rp, d_ci, rp, ci, ctx->d_err), "stack");
        TRYK(launch_validate_csr(cs, (int32_t)ntot, (int32_t)nnz, rp, ci, ctx->d_err), "validate");
    }
    int herr = 0;
    TRY(read_err(ctx, &herr));
    if (herr & ERR_ROWPTR) return cleanup(fail(ctx, SPAI_EINVAL, "a matrix of the batch has an invalid row pointer array"));
    if (herr) return cleanup(fail(ctx, SPAI_EINVAL, "a matrix of the batch has column indices out of range or not "
                                  "strictly increasing in a row (device error 0x%x)", herr));
    {
        char *t = nullptr;
        TRY(talloc(&t, (int64_t)transpose_temp_bytes((int32_t)ntot, (int32_t)std::max<int64_t>(nnz, 1))));
        ttemp = t;
    }
    {
        ProfScope ps_(ctx, "analysis:transpose", 0.0, 0.0);
        TRYK(launch_transpose(cs, (int32_t)ntot, (int32_t)nnz, rp, ci, colptr, rowind, perm, ttemp, ctx->d_err), "transpose");
    }
    // ---- union lists L_k ({k} or the rows of column k) and their longest
    int32_t *counts = nullptr, *Lptr = nullptr, *Lind = nullptr, *Jptr = nullptr, *Jind = nullptr, *Iptr = nullptr,
            *Ilist = nullptr, *d_scal = nullptr;
    char *stemp = nullptr;
    TRY(talloc(&counts, ntot + 1));
    TRY(talloc(&Lptr, ntot + 1));
    TRY(talloc(&stemp, (int64_t)scan_temp_bytes(ntot)));
    TRY(talloc(&d_scal, 4));
    {
        ProfScope ps_(ctx, "analysis:lists", 0.0, 0.0);
        TRYK(launch_union_lists(cs, nsys, ntot, d_off, d_kind, colptr, rowind, counts, nullptr, nullptr), "list counts");
        TRYK(launch_exclusive_scan(cs, counts, Lptr, ntot, stemp, ctx->d_err), "scan");
        TRYK(launch_max_i32_diff(cs, (int32_t)ntot, Lptr, d_scal), "longest list");
    }
    int32_t h2[2] = {0, 0};
    TRYC(cudaMemcpyAsync(&h2[0], Lptr + ntot, 4, cudaMemcpyDeviceToHost, cs), "read back");
    TRYC(cudaMemcpyAsync(&h2[1], d_scal, 4, cudaMemcpyDeviceToHost, cs), "read back");
    TRY(read_err(ctx, &herr));
    if (herr) return cleanup(fail(ctx, SPAI_EINVAL, "pattern analysis failed (device error 0x%x)", herr));
    if (h2[1] > colunion_max_lists())
        return cleanup(fail(ctx, SPAI_EINVAL, "a column has %d entries; at most %d are supported", h2[1],
                            colunion_max_lists()));
    TRY(talloc(&Lind, h2[0]));
    TRYK(launch_union_lists(cs, nsys, ntot, d_off, d_kind, colptr, rowind, nullptr, Lptr, Lind), "list fill");
    // ---- J_k = union over L_k of rows(A(:,j)); per system its total and longest column
    int64_t *d_tot = nullptr;
    int32_t *d_mx = nullptr;
    TRY(talloc(&d_tot, 2 * (int64_t)nsys));
    TRY(talloc(&d_mx, 2 * (int64_t)nsys));
    TRY(talloc(&Jptr, ntot + 1));
    {
        ProfScope ps_(ctx, "analysis:J", 0.0, 0.0);
        TRYK(launch_colunion_count(cs, (int32_t)ntot, h2[1], Lptr, Lind, colptr, rowind, counts, ctx->d_err), "J count");
        TRYK(launch_exclusive_scan(cs, counts, Jptr, ntot, stemp, ctx->d_err), "scan");
        TRYK(launch_seg_ptr_stats(cs, nsys, ntot, d_off, Jptr, d_tot, d_mx), "J sizes");
    }
    std::vector<int64_t> totJ((size_t)nsys), totI((size_t)nsys);
    std::vector<int32_t> mxJ((size_t)nsys), mxI((size_t)nsys);
    TRYC(cudaMemcpyAsync(totJ.data(), d_tot, (size_t)nsys * 8, cudaMemcpyDeviceToHost, cs), "read back");
    TRYC(cudaMemcpyAsync(mxJ.data(), d_mx, (size_t)nsys * 4, cudaMemcpyDeviceToHost, cs), "read back");
    TRY(read_err(ctx, &herr));
    if (herr & ERR_OVERFLOW) return cleanup(fail(ctx, SPAI_EINVAL, "index sets exceed 2^31 entries"));
    if (herr) return cleanup(fail(ctx, SPAI_EINVAL, "pattern analysis failed (device error 0x%x)", herr));
    int64_t nJ = 0;
    int32_t mxJall = 0;
    for (int i = 0; i < nsys; ++i) {
        nJ += totJ[i];
        mxJall = std::max(mxJall, mxJ[i]);
        if (mxJ[i] > colunion_max_lists())
            return cleanup(fail(ctx, SPAI_EINVAL, "system %d: a column pattern has %d entries; at most %d are supported",
                                i, mxJ[i], colunion_max_lists()));
    }
    if (nJ >= INT32_MAX) return cleanup(fail(ctx, SPAI_EINVAL, "the stacked pattern of P exceeds 2^31 entries"));
    TRY(talloc(&Jind, nJ));
    {
        ProfScope ps_(ctx, "analysis:J", 0.0, 0.0);
        TRYK(launch_colunion_fill(cs, (int32_t)ntot, h2[1], Lptr, Lind, colptr, rowind, Jptr, Jind, ctx->d_err), "J fill");
    }
    // ---- rows of P (the transpose of the J pattern) and the map J position -> P row position
    int32_t *prp = nullptr, *pci = nullptr, *pperm = nullptr, *pmap = nullptr;
    TRY(talloc(&prp, ntot + 1));
    TRY(talloc(&pci, nJ));
    TRY(talloc(&pperm, nJ));
    TRY(talloc(&pmap, nJ));
    {
        char *t = nullptr;
        TRY(talloc(&t, (int64_t)transpose_temp_bytes((int32_t)ntot, (int32_t)std::max<int64_t>(nJ, 1))));
        {
            ProfScope ps_(ctx, "analysis:P_rows", 0.0, 0.0);
            TRYK(launch_transpose(cs, (int32_t)ntot, (int32_t)nJ, Jptr, Jind, prp, pci, pperm, t, ctx->d_err),
                 "transpose pattern");
        }
    }
    {
        ProfScope ps_(ctx, "analysis:P_rows", 0.0, 0.0);
        TRYK(launch_invert_perm(cs, nJ, pperm, pmap), "invert");
    }
    // ---- I_k = union over J_k of rows(A(:,j))
    TRY(talloc(&Iptr, ntot + 1));
    {
        ProfScope ps_(ctx, "analysis:I", 0.0, 0.0);
        TRYK(launch_colunion_count(cs, (int32_t)ntot, mxJall, Jptr, Jind, colptr, rowind, counts, ctx->d_err), "I count");
        TRYK(launch_exclusive_scan(cs, counts, Iptr, ntot, stemp, ctx->d_err), "scan");
        TRYK(launch_seg_ptr_stats(cs, nsys, ntot, d_off, Iptr, d_tot + nsys, d_mx + nsys), "I sizes");
    }
    TRYC(cudaMemcpyAsync(totI.data(), d_tot + nsys, (size_t)nsys * 8, cudaMemcpyDeviceToHost, cs), "read back");
    TRYC(cudaMemcpyAsync(mxI.data(), d_mx + nsys, (size_t)nsys * 4, cudaMemcpyDeviceToHost, cs), "read back");
    TRY(read_err(ctx, &herr));
    if (herr & ERR_OVERFLOW) return cleanup(fail(ctx, SPAI_EINVAL, "index sets exceed 2^31 entries"));
    if (herr) return cleanup(fail(ctx, SPAI_EINVAL, "pattern analysis failed (device error 0x%x)", herr));
    int64_t nIt = 0;
    for (int i = 0; i < nsys; ++i) {
        nIt += totI[i];
        if (!spai_columns_fit(mxI[i], mxJ[i]))
            return cleanup(fail(ctx, SPAI_EINVAL, "system %d: column problem of %d x %d exceeds the shared-memory tile",
                                i, mxI[i], mxJ[i]));
    }
    if (nIt >= INT32_MAX) return cleanup(fail(ctx, SPAI_EINVAL, "the stacked index sets exceed 2^31 entries"));
    TRY(talloc(&Ilist, nIt));
    {
        ProfScope ps_(ctx, "analysis:I", 0.0, 0.0);
        TRYK(launch_colunion_fill(cs, (int32_t)ntot, mxJall, Jptr, Jind, colptr, rowind, Iptr, Ilist, ctx->d_err), "I fill");
    }

    // ---- the arena: every system's analysis (local indices) and factor storage
    auto r256 = [](size_t b) { return ((b ? b : 16) + 255) / 256 * 256; };
    std::vector<size_t> base((size_t)nsys);
    size_t abytes = 0;
    std::vector<int64_t> jb((size_t)nsys + 1, 0), ib((size_t)nsys + 1, 0);
    for (int i = 0; i < nsys; ++i) {
        jb[i + 1] = jb[i] + totJ[i];
        ib[i + 1] = ib[i] + totI[i];
        const size_t n1 = (size_t)A[i].n + 1, nz = (size_t)A[i].nnz, nzP = (size_t)totJ[i];
        const size_t vb = precs[i] == 2 ? 2 : precs[i] == 1 ? 4 : 8;
        base[i] = abytes;
        abytes += 2 * r256(n1 * 4) + 3 * r256(nz * 4);  // a_rowptr, a_colptr; a_colind, a_rowind, a_perm
        if (kinds[i]) abytes += 2 * r256(n1 * 4) + 3 * r256(nzP * 4);  // Jptr, p_rowptr; Jind, p_colind, p_map
        abytes += r256(n1 * 4) + r256((size_t)totI[i] * 4);          // Iptr, Ilist
        abytes += r256(nzP * vb) + r256(nz * 8) + r256((size_t)A[i].n * 4);  // factor, a_cval, status
    }
    Arena *arena = new Arena();
    arena->ctx = ctx;
    if ((st = dalloc(ctx, &arena->mem, abytes))) {
        delete arena;
        return cleanup(st);
    }
    char *am = (char *)arena->mem;
    TRYC(cudaMemsetAsync(am, 0, abytes, cs), "zero arena");  // factors and status start at zero
    // segments of the unstacking: (source, destination, count, subtracted offset)
    std::vector<const int32_t *> usrc;
    std::vector<int32_t *> udst;
    std::vector<int32_t> usub;
    std::vector<int64_t> ustart(1, 0);
    auto seg = [&](const int32_t *src, int32_t *dst, int64_t count, int64_t sub) {
        usrc.push_back(src);
        udst.push_back(dst);
        usub.push_back((int32_t)sub);
        ustart.push_back(ustart.back() + count);
    };
    std::vector<const double *> gval;
    std::vector<const int32_t *> gperm;
    std::vector<double *> gdst;
    std::vector<int64_t> gstart(1, 0);
    std::vector<const int32_t *> sstat;
    std::vector<int64_t> sstart(1, 0);
    pcs.assign((size_t)nsys, nullptr);
    for (int i = 0; i < nsys; ++i) {
        const int32_t n = A[i].n;
        const size_t n1 = (size_t)n + 1, nz = (size_t)A[i].nnz, nzP = (size_t)totJ[i];
        char *p = am + base[i];
        auto take = [&](size_t bytes) {
            char *r = p;
            p += r256(bytes);
            return r;
        };
        Sym *s = new Sym();
        s->ctx = ctx;
        s->arena = arena;
        arena->refs++;
        s->n = n;
        s->nnzA = (int32_t)nz;
        s->kind = kinds[i];
        s->a_rowptr = (int32_t *)take(n1 * 4);
        s->a_colptr = (int32_t *)take(n1 * 4);
        s->a_colind = (int32_t *)take(nz * 4);
        s->a_rowind = (int32_t *)take(nz * 4);
        s->a_perm = (int32_t *)take(nz * 4);
        seg(rp + off[i], s->a_rowptr, (int64_t)n1, nzoff[i]);
        seg(ci + nzoff[i], s->a_colind, (int64_t)nz, off[i]);
        seg(colptr + off[i], s->a_colptr, (int64_t)n1, nzoff[i]);
        seg(rowind + nzoff[i], s->a_rowind, (int64_t)nz, off[i]);
        seg(perm + nzoff[i], s->a_perm, (int64_t)nz, nzoff[i]);
        s->nnzP = (int32_t)nzP;
        if (kinds[i]) {
            s->alias = false;
            s->Jptr = (int32_t *)take(n1 * 4);
            s->p_rowptr = (int32_t *)take(n1 * 4);
            s->Jind = (int32_t *)take(nzP * 4);
            s->p_colind = (int32_t *)take(nzP * 4);
            s->p_map = (int32_t *)take(nzP * 4);
            seg(Jptr + off[i], s->Jptr, (int64_t)n1, jb[i]);
            seg(Jind + jb[i], s->Jind, (int64_t)nzP, off[i]);
            seg(prp + off[i], s->p_rowptr, (int64_t)n1, jb[i]);
            seg(pci + jb[i], s->p_colind, (int64_t)nzP, off[i]);
            seg(pmap + jb[i], s->p_map, (int64_t)nzP, jb[i]);
        } else {
            s->alias = true;  // P's pattern is A's: the same arrays as spai_build uses
            s->Jptr = s->a_colptr;
            s->Jind = s->a_rowind;
            s->p_rowptr = s->a_rowptr;
            s->p_colind = s->a_colind;
            s->p_map = s->a_perm;
        }
        s->Iptr = (int32_t *)take(n1 * 4);
        s->Ilist = (int32_t *)take((size_t)totI[i] * 4);
        s->nI = (int32_t)totI[i];
        seg(Iptr + off[i], s->Iptr, (int64_t)n1, ib[i]);
        seg(Ilist + ib[i], s->Ilist, totI[i], off[i]);
        s->maxI = mxI[i];
        s->maxJ = mxJ[i];
        spai_pc pc = new spai_pc_s();
        pc->ctx = ctx;
        pc->sym = s;
        pc->root = pc;
        pc->arena = arena;
        arena->refs++;
        const size_t vb = precs[i] == 2 ? 2 : precs[i] == 1 ? 4 : 8;
        char *fv = take(nzP * vb);
        if (precs[i] == 2) pc->fval16 = (uint16_t *)fv;
        else if (precs[i] == 1) pc->fval32 = (float *)fv;
        else pc->fval = (double *)fv;
        pc->a_cval = (double *)take(nz * 8);
        pc->status = (int32_t *)take((size_t)n * 4);
        pcs[i] = pc;
        gval.push_back(A[i].val);
        gperm.push_back(s->a_perm);
        gdst.push_back(pc->a_cval);
        gstart.push_back(gstart.back() + (int64_t)nz);
    }
    // device copies of the segment tables (one buffer), the unstacking and the value gathers
    const int nu = (int)usrc.size();
    const size_t tbytes = (size_t)(nu + 1) * 8 + (size_t)nu * 8 * 2 + r256((size_t)nu * 4) + (size_t)(nsys + 1) * 8 +
                          (size_t)nsys * 8 * 3 + 256;
    char *d_tab = nullptr;
    TRY(talloc(&d_tab, (int64_t)tbytes));
    {
        std::vector<char> h(tbytes, 0);
        size_t o = 0;
        auto put = [&](const void *src, size_t bytes) {
            memcpy(h.data() + o, src, bytes);
            const size_t at = o;
            o += (bytes + 15) / 16 * 16;
            return at;
        };
        const size_t o_us = put(ustart.data(), ustart.size() * 8), o_src = put(usrc.data(), usrc.size() * 8),
                     o_dst = put(udst.data(), udst.size() * 8), o_sub = put(usub.data(), usub.size() * 4),
                     o_gs = put(gstart.data(), gstart.size() * 8), o_gv = put(gval.data(), gval.size() * 8),
                     o_gp = put(gperm.data(), gperm.size() * 8), o_gd = put(gdst.data(), gdst.size() * 8);
        TRYC(cudaMemcpyAsync(d_tab, h.data(), o, cudaMemcpyHostToDevice, cs), "tables");
        TRYC(cudaStreamSynchronize(cs), "sync");  // h is read by the copy above
        {
            ProfScope ps_(ctx, "analysis:unstack", 0.0, 0.0);
            TRYK(launch_unstack(cs, nu, ustart.back(), (const int64_t *)(d_tab + o_us), (const int32_t *const *)(d_tab + o_src),
                                (int32_t *const *)(d_tab + o_dst), (const int32_t *)(d_tab + o_sub)),
                 "unstack");
        }
        {
            ProfScope ps_(ctx, "gather_csc", 0.0, 20.0 * (double)nnz);
            TRYK(launch_gather_seg(cs, nsys, gstart.back(), (const int64_t *)(d_tab + o_gs),
                                   (const double *const *)(d_tab + o_gv), (const int32_t *const *)(d_tab + o_gp),
                                   (double *const *)(d_tab + o_gd)),
                 "gather values");
        }
    }
    TRYC(cudaStreamSynchronize(cs), "sync");  // the stacked temporaries are released after their last use
#undef TRY
#undef TRYC
#undef TRYK
    return cleanup(SPAI_OK);
}

}  // namespace

extern "C" spai_status spai_build_batch(spai_ctx ctx, int32_t nsys, const spai_csr *A, const int32_t *pattern_kind,
                                        spai_pc *out)
{
    if (!ctx || !A || !pattern_kind || !out) return fail(ctx, SPAI_EINVAL, "NULL argument");
    if (nsys < 1 || nsys > 65536) return fail(ctx, SPAI_EINVAL, "nsys must be in 1..65536");
    for (int i = 0; i < nsys; ++i) out[i] = nullptr;
    std::vector<int32_t> kinds((size_t)nsys), precs((size_t)nsys);
    spai_status st;
    for (int i = 0; i < nsys; ++i) {
        precs[i] = prec_of(pattern_kind[i]);
        if (precs[i] < 0) return fail(ctx, SPAI_EINVAL, "system %d: SPAI_PREC_FP32 and SPAI_PREC_BF16 are exclusive", i);
        kinds[i] = pattern_kind[i] & ~(SPAI_PREC_FP32 | SPAI_PREC_BF16 | SPAI_LS_NORMAL);
        if (kinds[i] != SPAI_PATTERN_A && kinds[i] != SPAI_PATTERN_A2)
            return fail(ctx, SPAI_EINVAL, "system %d: unknown pattern kind %d", i, kinds[i]);
        if ((st = check_csr_args(ctx, &A[i], "A"))) return st;
        if (A[i].n == 0) continue;
        if (!is_device_ptr(A[i].rowptr) ||
            (A[i].nnz > 0 && (!is_device_ptr(A[i].colind) || !is_device_ptr(A[i].val))))
            return fail(ctx, SPAI_EINVAL, "system %d: arrays must be device memory", i);
    }
    // two or more systems, none empty: the stacked analysis (its CUDA calls do not grow with
    // the number of systems); otherwise one analysis per system
    bool stacked = nsys >= 2;
    int64_t ntot = 0, nnztot = 0;
    for (int i = 0; i < nsys; ++i) {
        stacked = stacked && A[i].n >= 1;
        ntot += A[i].n;
        nnztot += A[i].nnz;
    }
    stacked = stacked && ntot < INT32_MAX && nnztot < INT32_MAX;
    if (stacked) {
        std::vector<spai_pc> pcs;
        if ((st = build_batch_stacked(ctx, nsys, A, kinds.data(), precs.data(), pcs))) return st;
        for (int i = 0; i < nsys; ++i) pcs[i]->normal = (pattern_kind[i] & SPAI_LS_NORMAL) != 0;
        st = run_columns_batch(ctx, nsys, pcs.data());
        if (st && st != SPAI_ESINGULAR) {
            for (spai_pc pc : pcs) spai_pc_destroy(pc);
            return st;
        }
        for (int i = 0; i < nsys; ++i) out[i] = pcs[i];
        return st;
    }
    for (int i = 0; i < nsys; ++i)
        if (A[i].n)
            KL(launch_validate_csr(ctx->stream, A[i].n, A[i].nnz, A[i].rowptr, A[i].colind, ctx->d_err), "validate");
    int h = 0;
    if ((st = read_err(ctx, &h))) return st;
    if (h) return fail(ctx, SPAI_EINVAL, "a matrix of the batch is not a valid CSR matrix (device error 0x%x)", h);
    std::vector<Sym *> syms((size_t)nsys, nullptr);
    if ((st = sym_create_batch(ctx, nsys, A, kinds.data(), syms.data()))) return st;
    std::vector<spai_pc> pcs((size_t)nsys, nullptr);
    for (int i = 0; i < nsys; ++i) {
        if ((st = pc_alloc(ctx, syms[i], precs[i], &pcs[i]))) {
            for (int k = 0; k < nsys; ++k) {
                if (pcs[k]) spai_pc_destroy(pcs[k]);  // releases its analysis too
                else sym_release(syms[k]);
            }
            return st;
        }
        pcs[i]->root = pcs[i];
        pcs[i]->normal = (pattern_kind[i] & SPAI_LS_NORMAL) != 0;
        if (syms[i]->nnzA)
            PKL("gather_csc", 0.0, 20.0 * syms[i]->nnzA,
                launch_gather_f64(ctx->stream, syms[i]->nnzA, syms[i]->a_perm, A[i].val, pcs[i]->a_cval),
                "gather values");
    }
    st = run_columns_batch(ctx, nsys, pcs.data());
    if (st && st != SPAI_ESINGULAR) {
        for (spai_pc pc : pcs) spai_pc_destroy(pc);
        return st;
    }
    for (int i = 0; i < nsys; ++i) out[i] = pcs[i];
    return st;
}

extern "C" int32_t spai_column_variants(int32_t low_precision, int32_t maxI, int32_t maxJ, int32_t *codes, int32_t cap)
{
    if (maxI < 1 || maxJ < 1 || !spai_columns_fit(maxI, maxJ)) return 0;
    int cand[32];
    const int nc = spai_columns_teams(maxI, maxJ, low_precision != 0, cand);
    for (int i = 0; i < nc && i < cap && codes; ++i) codes[i] = cand[i];
    return nc;
}

extern "C" int32_t spai_column_variant_get(int32_t low_precision, int32_t maxI, int32_t maxJ)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(low_precision ? 1 : 0, (maxI + 7) / 8 * 8, maxJ));
    return it == g_tune.end() ? 0 : it->second;
}

extern "C" spai_status spai_column_variant_set(int32_t low_precision, int32_t maxI, int32_t maxJ, int32_t code)
{
    if (maxI < 1 || maxJ < 1) return SPAI_EINVAL;
    const auto key = std::make_tuple(low_precision ? 1 : 0, (maxI + 7) / 8 * 8, maxJ);
    if (code == 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune.erase(key);
        return SPAI_OK;
    }
    // the code must fit every shape of the class: the largest max |I_k| it holds
    int cand[32];
    const int nc = spai_columns_fit(std::get<1>(key), maxJ)
                       ? spai_columns_teams(std::get<1>(key), maxJ, low_precision != 0, cand)
                       : 0;
    bool ok = false;
    for (int i = 0; i < nc; ++i) ok = ok || cand[i] == code;
    if (!ok) return SPAI_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = code;
    return SPAI_OK;
}

extern "C" spai_status spai_pc_info(spai_pc pc, int32_t *n, int32_t *nnz, int64_t *nI, int32_t *depth)
{
    if (!pc) return SPAI_EINVAL;
    if (n) *n = pc->sym->n;
    if (nnz) *nnz = pc->diag ? pc->sym->n : pc->sym->nnzP;
    if (nI) *nI = pc->diag ? (int64_t)pc->sym->nnzA : pc->sym->nI;
    if (depth) *depth = pc->depth;
    return SPAI_OK;
}

extern "C" size_t spai_pc_mem_size(spai_pc pc, int32_t with_analysis)
{
    if (!pc) return 0;
    auto r = [](size_t b) { return ((b ? b : 16) + 255) / 256 * 256; };  // as dalloc rounds
    const Sym *s = pc->sym;
    const size_t n1 = (size_t)s->n + 1;
    const size_t nf = pc->diag ? (size_t)s->n : (size_t)s->nnzP;
    size_t b = r(nf * (pc->fval16 ? 2 : pc->fval32 ? 4 : 8)) + r((size_t)s->nnzA * 8) + r((size_t)s->n * 4);
    if (with_analysis) {
        b += 2 * r(n1 * 4) + 3 * r((size_t)s->nnzA * 4) + r(n1 * 4) + r((size_t)s->nI * 4);
        if (!s->alias) b += 2 * r(n1 * 4) + 3 * r((size_t)s->nnzP * 4);
    }
    return b;
}

extern "C" spai_status spai_pc_export(spai_ctx ctx, spai_pc pc, int32_t *Jptr, int32_t *Jind, double *val,
                                      int32_t *Iptr, int32_t *Ilist, int32_t *col_status)
{
    if (!ctx || !pc) return fail(ctx, SPAI_EINVAL, "NULL argument");
    Sym *s = pc->sym;
    const int32_t n = s->n;
    if (pc->diag) {
        // J_k = {k}, I_k = rows(A(:,k)), values in column order already
        if (Jptr) KL(launch_iota_i32(ctx->stream, (int64_t)n + 1, Jptr), "export");
        if (Jind && n) KL(launch_iota_i32(ctx->stream, n, Jind), "export");
        if (val && n) {
            if (pc->fval16) KL(launch_gather_bf16_f64(ctx->stream, n, nullptr, pc->fval16, val), "export values");
            else if (pc->fval32) KL(launch_gather_f32_f64(ctx->stream, n, nullptr, pc->fval32, val), "export values");
            else CU(cudaMemcpyAsync(val, pc->fval, (size_t)n * 8, cudaMemcpyDeviceToDevice, ctx->stream), "export");
        }
        if (Iptr) CU(cudaMemcpyAsync(Iptr, s->a_colptr, ((size_t)n + 1) * 4, cudaMemcpyDeviceToDevice, ctx->stream), "export");
        if (Ilist && s->nnzA)
            CU(cudaMemcpyAsync(Ilist, s->a_rowind, (size_t)s->nnzA * 4, cudaMemcpyDeviceToDevice, ctx->stream), "export");
        if (col_status && n) CU(cudaMemcpyAsync(col_status, pc->status, (size_t)n * 4, cudaMemcpyDeviceToDevice, ctx->stream), "export");
        return SPAI_OK;
    }
    if (Jptr) CU(cudaMemcpyAsync(Jptr, s->Jptr, ((size_t)n + 1) * 4, cudaMemcpyDeviceToDevice, ctx->stream), "export");
    if (Jind && s->nnzP) CU(cudaMemcpyAsync(Jind, s->Jind, (size_t)s->nnzP * 4, cudaMemcpyDeviceToDevice, ctx->stream), "export");
    if (val && s->nnzP) {
        if (pc->fval16)
            KL(launch_gather_bf16_f64(ctx->stream, s->nnzP, s->p_map, pc->fval16, val), "export values");
        else if (pc->fval32)
            KL(launch_gather_f32_f64(ctx->stream, s->nnzP, s->p_map, pc->fval32, val), "export values");
        else
            KL(launch_gather_f64(ctx->stream, s->nnzP, s->p_map, pc->fval, val), "export values");
    }
    if (Iptr) CU(cudaMemcpyAsync(Iptr, s->Iptr, ((size_t)n + 1) * 4, cudaMemcpyDeviceToDevice, ctx->stream), "export");
    if (Ilist && s->nI) CU(cudaMemcpyAsync(Ilist, s->Ilist, (size_t)s->nI * 4, cudaMemcpyDeviceToDevice, ctx->stream), "export");
    if (col_status && n) CU(cudaMemcpyAsync(col_status, pc->status, (size_t)n * 4, cudaMemcpyDeviceToDevice, ctx->stream), "export");
    return SPAI_OK;
}

extern "C" spai_status spai_pc_destroy(spai_pc pc)
{
    if (!pc) return SPAI_EINVAL;
    spai_ctx ctx = pc->ctx;
    if (pc->arena) {
        arena_release(pc->arena);
    } else {
        dfree(ctx, pc->fval);
        dfree(ctx, pc->fval32);
        dfree(ctx, pc->fval16);
        dfree(ctx, pc->a_cval);
        dfree(ctx, pc->status);
    }
    sym_release(pc->sym);
    delete pc;
    return SPAI_OK;
}

// ===================================================================================
// products
// ===================================================================================
namespace {

struct Block {
    double *p = nullptr;
};

spai_status temp_blocks(spai_ctx ctx, size_t bytes, void **p)
{
    if (ctx->ws_bytes >= bytes) { *p = ctx->ws; return SPAI_OK; }
    if (ctx->ws) { dfree(ctx, ctx->ws); ctx->ws = nullptr; ctx->ws_bytes = 0; }
    spai_status st = dalloc(ctx, &ctx->ws, bytes);
    if (st) return st;
    ctx->ws_bytes = bytes;
    *p = ctx->ws;
    return SPAI_OK;
}

}  // namespace

extern "C" spai_status spai_spmm(spai_ctx ctx, const spai_csr *A, int32_t s, const double *X, int64_t ldx,
                                 double *Y, int64_t ldy)
{
    if (!ctx) return SPAI_EINVAL;
    spai_status st = check_csr_args(ctx, A, "A");
    if (st) return st;
    if (!valid_s(s)) return fail(ctx, SPAI_EINVAL, "s must be 1, 2, 4, 8 or 16");
    const int32_t n = A->n;
    if (n == 0) return SPAI_OK;
    if (ldx < n || ldy < n || !X || !Y) return fail(ctx, SPAI_EINVAL, "bad block arguments");
    void *w = nullptr;
    const size_t blk = (size_t)n * s * 8;
    if ((st = temp_blocks(ctx, 2 * blk, &w))) return st;
    double *xr = (double *)w, *yr = (double *)((char *)w + blk);
    KL(launch_pack(ctx->stream, s, n, X, ldx, xr), "pack");
    PKL("spmm_A", 2.0 * A->nnz * s, 12.0 * A->nnz + 4.0 * (n + 1) + 16.0 * n * s,
        launch_spmm(ctx->stream, s, n, A->rowptr, A->colind, A->val, xr, yr), "spmm");
    KL(launch_unpack(ctx->stream, s, n, yr, Y, ldy), "unpack");
    return SPAI_OK;
}

extern "C" spai_status spai_pc_apply(spai_ctx ctx, spai_pc pc, int32_t s, const double *X, int64_t ldx, double *Y,
                                     int64_t ldy)
{
    if (!ctx || !pc) return fail(ctx, SPAI_EINVAL, "NULL argument");
    if (!valid_s(s)) return fail(ctx, SPAI_EINVAL, "s must be 1, 2, 4, 8 or 16");
    const int32_t n = pc->sym->n;
    if (n == 0) return SPAI_OK;
    if (ldx < n || ldy < n || !X || !Y) return fail(ctx, SPAI_EINVAL, "bad block arguments");
    void *w = nullptr;
    const size_t blk = (size_t)n * s * 8;
    spai_status st = temp_blocks(ctx, 4 * blk, &w);
    if (st) return st;
    double *xr = (double *)w, *yr = xr + (size_t)n * s, *t0 = yr + (size_t)n * s, *t1 = t0 + (size_t)n * s;
    KL(launch_pack(ctx->stream, s, n, X, ldx, xr), "pack");
    if ((st = apply_rm(ctx, pc, s, xr, yr, t0, t1))) return st;
    KL(launch_unpack(ctx->stream, s, n, yr, Y, ldy), "unpack");
    return SPAI_OK;
}

extern "C" spai_status spai_spmm_fp32(spai_ctx ctx, const spai_csr *A, int32_t s, const double *X, int64_t ldx,
                                      double *Y, int64_t ldy)
{
    if (!ctx) return SPAI_EINVAL;
    spai_status st = check_csr_args(ctx, A, "A");
    if (st) return st;
    if (!valid_s(s)) return fail(ctx, SPAI_EINVAL, "s must be 1, 2, 4, 8 or 16");
    const int32_t n = A->n;
    if (n == 0) return SPAI_OK;
    if (ldx < n || ldy < n || !X || !Y) return fail(ctx, SPAI_EINVAL, "bad block arguments");
    void *w = nullptr;
    const size_t blk = (size_t)n * s * 8, a32 = ((size_t)A->nnz * 4 + 255) / 256 * 256;
    if ((st = temp_blocks(ctx, 2 * blk + a32 + blk / 2, &w))) return st;
    double *xr = (double *)w, *yr = (double *)((char *)w + blk);
    float *av = (float *)((char *)w + 2 * blk);
    float *x32 = (float *)((char *)w + 2 * blk + a32);
    F32Vals v;
    v.f32 = av;
    KL(launch_round_f32(ctx->stream, A->nnz, A->val, av), "A in FP32");
    KL(launch_pack(ctx->stream, s, n, X, ldx, xr), "pack");
    KL(launch_round_f32(ctx->stream, (int64_t)n * s, xr, x32), "X in FP32");  // once, as the solve's basis
    PKL("spmm32_A", 2.0 * A->nnz * s, 8.0 * A->nnz + 4.0 * (n + 1) + 12.0 * n * s,
        launch_spmm32(ctx->stream, s, n, A->rowptr, A->colind, v, (const float *)x32, yr), "spmm fp32");
    KL(launch_unpack(ctx->stream, s, n, yr, Y, ldy), "unpack");
    return SPAI_OK;
}

extern "C" spai_status spai_pc_apply_fp32(spai_ctx ctx, spai_pc pc, int32_t s, const double *X, int64_t ldx,
                                          double *Y, int64_t ldy)
{
    if (!ctx || !pc) return fail(ctx, SPAI_EINVAL, "NULL argument");
    if (!valid_s(s)) return fail(ctx, SPAI_EINVAL, "s must be 1, 2, 4, 8 or 16");
    const int32_t n = pc->sym->n;
    if (n == 0) return SPAI_OK;
    if (ldx < n || ldy < n || !X || !Y) return fail(ctx, SPAI_EINVAL, "bad block arguments");
    void *w = nullptr;
    const size_t blk = (size_t)n * s * 8;
    spai_status st = temp_blocks(ctx, 4 * blk, &w);
    if (st) return st;
    double *xr = (double *)w, *yr = xr + (size_t)n * s;
    float *t0 = (float *)(yr + (size_t)n * s), *t1 = t0 + (size_t)n * s;
    KL(launch_pack(ctx->stream, s, n, X, ldx, xr), "pack");
    if ((st = apply32<double>(ctx, pc, s, xr, yr, t0, t1))) return st;
    KL(launch_unpack(ctx->stream, s, n, yr, Y, ldy), "unpack");
    return SPAI_OK;
}

// ===================================================================================
// block GMRES(m)
// ===================================================================================
namespace {

struct SolveWs {
    double *Bw, *Xw, *W, *Z, *T0, *T1, *V;
    double *Xh, *D;     // block GCRO: the preconditioned-space iterate and a correction block
    float *V32;         // mixed precision: the newest basis block in FP32 (the FP32 operator's input)
    double *partial, *H1, *H2, *G1, *R1, *R2, *Rn, *ref2, *nrm2, *thresh, *Qs, *Rtri, *G, *Y, *est;
    int32_t *defl1, *defl2, *flag;
    unsigned *ticket;   // last-CTA tickets of the fused Cholesky-QR and norm kernels (zero between launches)
    uint64_t *vfix;     // fixed-point copies of the basis blocks, row layout (block update)
    uint64_t *vfix_sub; // the same, sub-tile layout across blocks (Gram product)
    void *hdig;     // digit pieces of H (tensor-core block update)
    int32_t *hexp;  // column exponents of H
    double *Wh;     // s == 16: column halves of a block (n x 8 each, back to back)
    double *HL, *HR;  // s == 16: 8 x 8 pieces of the small blocks, per half-block
};

// Block widths whose Gram-Schmidt products can run on the tensor-core digit kernels: 8
// directly, 16 as two 8-column halves (2 (m + 1) half-blocks within the update kernel's limit)
bool digits_for(int32_t s, int32_t m)
{
    return block_dot_tc_supported(s) || (s == 16 && 2 * (m + 1) <= block_update_tc_max_blocks());
}

size_t carve(SolveWs &w, void *base, int32_t n, int32_t s, int32_t m, int chunks)
{
    char *p = (char *)base;
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        void *r = base ? (void *)(p + off) : nullptr;
        off += (bytes + 255) / 256 * 256;
        return r;
    };
    const size_t blk = (size_t)n * s * 8;
    const size_t ss = (size_t)s * s * 8;
    w.Bw = (double *)take(blk);
    w.Xw = (double *)take(blk);
    w.W = (double *)take(blk);
    w.Z = (double *)take(blk);
    w.T0 = (double *)take(blk);
    w.T1 = (double *)take(blk);
    w.V = (double *)take(blk * (m + 1));
    w.Xh = (double *)take(blk);
    w.D = (double *)take(blk);
    w.V32 = (float *)take(blk / 2);
    const bool digits = digits_for(s, m);
    const int32_t nh = (s == 16 ? 2 : 1) * (m + 1);  // basis (half-)blocks of the digit kernels
    {
        const size_t a = (size_t)chunks * s * 8, b = dot_partial_elems(s, m + 1) * 8;
        const size_t c = tc_partial_elems(n, nh) * 8;  // tensor-core row chunks
        size_t mx = a > b ? a : b;
        w.partial = (double *)take(mx > c ? mx : c);
    }
    w.H1 = (double *)take((m + 1) * ss);
    w.H2 = (double *)take((m + 1) * ss);
    w.G1 = (double *)take(ss);
    w.R1 = (double *)take(ss);
    w.R2 = (double *)take(ss);
    w.Rn = (double *)take(ss);
    w.ref2 = (double *)take(s * 8);
    w.nrm2 = (double *)take(s * 8);
    w.thresh = (double *)take(s * 8);
    w.Qs = (double *)take((size_t)m * 4 * ss);
    w.Rtri = (double *)take((size_t)(m + 1) * s * m * s * 8);
    w.G = (double *)take((m + 1) * ss);
    w.Y = (double *)take(m * ss);
    w.est = (double *)take(s * 8);
    w.defl1 = (int32_t *)take(s * 4);
    w.defl2 = (int32_t *)take(s * 4);
    w.flag = (int32_t *)take(64);
    w.ticket = (unsigned *)take(64);
    w.vfix = (uint64_t *)take(digits ? blk * (m + 1) : 16);
    w.vfix_sub = (uint64_t *)take(digits ? tc_fixed_sub_bytes(n, nh) : 16);
    w.hdig = take(digits ? tc_hdig_bytes(nh) : 16);
    w.hexp = (int32_t *)take(64);
    const bool halves = digits && s == 16;
    w.Wh = (double *)take(halves ? blk : 16);
    w.HL = (double *)take(halves ? (size_t)nh * 64 * 8 : 16);
    w.HR = (double *)take(halves ? (size_t)nh * 64 * 8 : 16);
    return off;
}

// W = Q R with Q orthonormal (deflated columns zero), two passes of Cholesky QR:
//   G1 = W^T W, R1 = chol(G1); Q1 = W R1^{-1}; G2 = Q1^T Q1, R2 = chol(G2); Q = Q1 R2^{-1};
//   R = R2 R1.
// For s <= 8, Q1 (written to Qout) and G2 come from one pass over W, the last pass solves
// Qout in place, and with fix_blk >= 0 (s == 8) it also writes Q's fixed-point copies
// (basis slot fix_blk of ipad) for the tensor-core products.  Qout must not overlap Win.
// Deflation is judged against ref2 (squared column norms before orthogonalisation), or for
// s <= 8 with H1 non-null against the norms the first pass forms from the block CGS
// coefficients H1, H2 (hrows rows).
spai_status cholqr2(spai_ctx ctx, SolveWs &w, int32_t n, int32_t s, const double *Win, double *Qout, double *Rout,
                    const double *ref2, int fix_blk, int32_t ipad, float *Q32 = nullptr, const double *H1 = nullptr,
                    const double *H2 = nullptr, int32_t hrows = 0)
{
    cudaStream_t st = ctx->stream;
    const double nsd = (double)n * s;
    if (cqr_supported(s)) {
        // three launches; each pass's last CTA does its Cholesky (and R = R2 R1)
        PKL("cqr_gram", nsd * (s + 1), 8.0 * nsd,
            launch_cqr_gram(st, s, n, Win, ref2, 1e-24, H1, H2, hrows, w.partial, w.ticket, w.R1, w.defl1),
            "Cholesky-QR pass 1");
        PKL("cqr_gram2", nsd * s + nsd * (s + 1), 16.0 * nsd,
            launch_cqr_gram2(st, s, n, Win, w.R1, w.defl1, Qout, w.partial, w.ticket, w.R2, w.defl2, Rout),
            "Cholesky-QR pass 2");
        if (fix_blk >= 0) {
            PKL("cqr_apply_fixed", nsd * s, 32.0 * nsd,
                launch_cqr_apply_fixed(st, n, Qout, w.R2, w.defl2, w.vfix + (size_t)fix_blk * n * s, w.vfix_sub, ipad,
                                       fix_blk, ctx->d_err, Q32),
                "Cholesky-QR pass 3 with fixed point");
        } else {
            PKL("cqr_apply", nsd * s, 16.0 * nsd, launch_cqr_apply(st, s, n, Qout, w.R2, w.defl2, Q32),
                "Cholesky-QR pass 3");
        }
        return SPAI_OK;
    } else {
        PKL("gram", nsd * (s + 1), 8.0 * nsd, launch_gram_sym(st, s, n, Win, w.partial, w.G1), "gram");
        PKL("small_dense", 0.0, 0.0, launch_chol_small(st, s, w.G1, ref2, 1e-24, w.R1, w.defl1), "chol");
        PKL("trsm_rows", nsd * s, 16.0 * nsd, launch_trsm_rows(st, s, n, Win, w.R1, w.defl1, Qout), "trsm");
        PKL("gram", nsd * (s + 1), 8.0 * nsd, launch_gram_sym(st, s, n, Qout, w.partial, w.G1), "gram");
        PKL("small_dense", 0.0, 0.0, launch_chol_small(st, s, w.G1, nullptr, 0.0, w.R2, w.defl2), "chol");
        PKL("trsm_rows", nsd * s, 16.0 * nsd, launch_trsm_rows(st, s, n, Qout, w.R2, w.defl2, Qout), "trsm");
        if (fix_blk >= 0)
            PKL("to_fixed", 0.0, 24.0 * nsd,
                launch_to_fixed(st, n, 1, Qout, w.vfix + (size_t)fix_blk * n * s, w.vfix_sub, ipad, fix_blk,
                                ctx->d_err),
                "fixed point");
    }
    PKL("small_dense", 0.0, 0.0, launch_triu_mul(st, s, w.R2, w.R1, Rout), "triu");
    if (Q32) KL(launch_round_f32(st, (int64_t)n * s, Qout, Q32), "basis block in FP32");
    return SPAI_OK;
}

}  // namespace

extern "C" size_t spai_solve_workspace_size(int32_t n, int32_t s, int32_t restart)
{
    if (n < 1 || !valid_s(s) || restart < 1) return 0;
    SolveWs w{};
    return carve(w, nullptr, n, s, restart, krylov_chunks(n));
}

extern "C" spai_status spai_ctx_trim(spai_ctx ctx)
{
    if (!ctx) return SPAI_EINVAL;
    if (ctx->ws) {
        dfree(ctx, ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    return SPAI_OK;
}

namespace {

// Right-preconditioned block GMRES(m) (rc == nullptr) and block GCRO with a recycled outer
// space rc (its columns U, with C = AP U orthonormal, come first in the basis: every cycle
// starts from the residual projected off C, orthogonalises against [C, V], and minimises
// over span([U, V]); the solve's iterate joins rc for the next system).  With rc empty the
// two are the same computation.
spai_status solve_impl(spai_ctx ctx, const spai_csr *A, spai_pc P, int32_t s, const double *B, int64_t ldb,
                       double *X, int64_t ldx, const spai_solve_opts *opts, spai_solve_info *info,
                       double *rel_residual, spai_recycle rc)
{
    if (!ctx) return SPAI_EINVAL;
    spai_status st = check_csr_args(ctx, A, "A");
    if (st) return st;
    if (!opts || !B || !X) return fail(ctx, SPAI_EINVAL, "NULL argument");
    if (!valid_s(s)) return fail(ctx, SPAI_EINVAL, "s must be 1, 2, 4, 8 or 16");
    const int32_t n = A->n, m = opts->restart;
    if (m < 1 || opts->max_cycles < 1 || !(opts->tol >= 0.0))
        return fail(ctx, SPAI_EINVAL, "restart and max_cycles must be >= 1 and tol >= 0");
    if (ldb < n || ldx < n) return fail(ctx, SPAI_EINVAL, "leading dimension smaller than n");
    if (P && P->sym->n != n) return fail(ctx, SPAI_EINVAL, "preconditioner size %d != n %d", P->sym->n, n);
    if (n > 0 && (!is_device_ptr(A->rowptr) || !is_device_ptr(A->colind) || !is_device_ptr(A->val)))
        return fail(ctx, SPAI_EINVAL, "A: arrays must be device memory");
    if (info) memset(info, 0, sizeof *info);
    if (n == 0) {
        if (info) info->converged = 1;
        return SPAI_OK;
    }
    if (opts->precision != SPAI_SOLVE_FP64 && opts->precision != SPAI_SOLVE_MIXED)
        return fail(ctx, SPAI_EINVAL, "unknown solve precision %d", opts->precision);
    if (rc && (rc->n != n || rc->s != s))
        return fail(ctx, SPAI_EINVAL, "recycle space made for n=%d, s=%d; the solve has n=%d, s=%d", rc->n, rc->s, n, s);
    const bool mixed = opts->precision == SPAI_SOLVE_MIXED;
    const int32_t kbmax = rc ? rc->kmax / s : 0;  // recycled blocks: basis slots 0 .. kb-1 hold C
    int32_t kb = rc ? rc->k / s : 0;
    const int32_t mt = m + kbmax;                 // the workspace's restart length
    const int chunks = krylov_chunks(n);
    SolveWs w{};
    const size_t need = carve(w, nullptr, n, s, mt, chunks);
    const size_t need32 = mixed ? ((size_t)A->nnz * 4 + 255) / 256 * 256 : 0;  // A's values in FP32
    void *base = nullptr;
    if ((st = temp_blocks(ctx, need + need32, &base))) return st;
    carve(w, base, n, s, mt, chunks);
    float *a32 = mixed ? (float *)((char *)base + need) : nullptr;
    cudaStream_t cs = ctx->stream;
    const bool b_dev = is_device_ptr(B), x_dev = is_device_ptr(X);
    if (opts->orth < SPAI_ORTH_AUTO || opts->orth > SPAI_ORTH_TENSOR)
        return fail(ctx, SPAI_EINVAL, "unknown orthogonalisation method %d", opts->orth);
    const bool use_digits = digits_for(s, mt) && opts->orth != SPAI_ORTH_FP64;
    const bool halves = use_digits && s == 16;  // 16 columns as two 8-column halves
    const int32_t ipad = (halves ? 2 : 1) * (mt + 1);
    const size_t half_elems = (size_t)n * 8;
    // H = V_{0..nb-1}^T Wsrc on the tensor cores: a 16-column block as two halves against
    // all 2 nb half-blocks of the basis, the two 8-column results merged into 16 x 16 blocks
    auto gram_tc = [&](int nb, double *Wsrc, double *H) -> spai_status {
        const double f = 2.0 * n * s * s * nb, by = 8.0 * n * s * (nb + 1);
        if (!halves) {
            PKL("block_dot_tc", f, by, launch_block_dot_tc(cs, n, nb, w.vfix_sub, ipad, Wsrc, w.partial, H, ctx->d_err, tc_wait(ctx)),
                "block Gram product");
            return SPAI_OK;
        }
        ProfScope ps(ctx, "block_dot_tc", f, by);
        KL(launch_halves16(cs, n, Wsrc, w.Wh, false), "column halves");
        KL(launch_block_dot_tc(cs, n, 2 * nb, w.vfix_sub, ipad, w.Wh, w.partial, w.HL, ctx->d_err, tc_wait(ctx)), "block Gram product");
        KL(launch_block_dot_tc(cs, n, 2 * nb, w.vfix_sub, ipad, w.Wh + half_elems, w.partial, w.HR, ctx->d_err,
                               tc_wait(ctx)),
           "block Gram product");
        KL(launch_pieces16(cs, nb, H, w.HL, w.HR, true), "merge pieces");
        return SPAI_OK;
    };
    // fixed point of basis block blk of a 16-column basis: its two halves as half-blocks
    // 2 blk and 2 blk + 1 (8-column blocks get theirs from the Cholesky-QR pass)
    auto fixed16 = [&](int blk) -> spai_status {
        if (!halves) return SPAI_OK;
        ProfScope ps(ctx, "to_fixed", 0.0, 24.0 * n * s);
        KL(launch_halves16(cs, n, w.V + (size_t)blk * n * s, w.Wh, false), "column halves");
        KL(launch_to_fixed(cs, n, 2, w.Wh, w.vfix + (size_t)2 * blk * half_elems, w.vfix_sub, ipad, 2 * blk, ctx->d_err),
           "fixed point");
        return SPAI_OK;
    };
    // out = base + sign * V_{first..first+nb-1} H: tensor-core digits when available, else FP64
    auto vupdate_at = [&](int first, int nb, const double *H, const double *basep, double *out,
                          double sign) -> spai_status {
        const double f = 2.0 * n * s * s * nb;
        const uint64_t *vf = w.vfix + (size_t)first * n * s;  // 8-column blocks or pairs of half-blocks
        if (use_digits && (halves ? 2 : 1) * nb <= block_update_tc_max_blocks() &&
            (opts->orth == SPAI_ORTH_TENSOR || nb >= 2)) {
            if (!halves) {
                PKL("block_update_tc", f, 8.0 * n * s * (nb + 2),
                    launch_block_update_tc(cs, n, nb, vf, H, w.hdig, w.hexp, basep, out, sign, ctx->d_err, tc_wait(ctx)),
                    "block update");
                return SPAI_OK;
            }
            // each output half: base half + sign * sum over half-blocks of V_hb times its piece of H
            ProfScope ps(ctx, "block_update_tc", f, 8.0 * n * s * (nb + 2));
            KL(launch_pieces16(cs, nb, const_cast<double *>(H), w.HL, w.HR, false), "split pieces");
            if (basep) KL(launch_halves16(cs, n, const_cast<double *>(basep), w.Wh, false), "column halves");
            for (int h = 0; h < 2; ++h) {
                double *wh = w.Wh + h * half_elems;
                KL(launch_block_update_tc(cs, n, 2 * nb, vf, h ? w.HR : w.HL, w.hdig, w.hexp, basep ? wh : nullptr, wh,
                                          sign, ctx->d_err, tc_wait(ctx)),
                   "block update");
            }
            KL(launch_halves16(cs, n, out, w.Wh, true), "merge halves");
        } else {
            PKL("block_update", f, 8.0 * n * s * (nb + 2),
                launch_block_update(cs, s, n, nb, w.V + (size_t)first * n * s, H, basep, out, sign), "block update");
        }
        return SPAI_OK;
    };
    auto vupdate = [&](int nb, const double *H, const double *basep, double *out, double sign) -> spai_status {
        return vupdate_at(0, nb, H, basep, out, sign);
    };

    // inputs -> row-major device blocks (T0 stages host data column-major)
    if (b_dev) {
        KL(launch_pack(cs, s, n, B, ldb, w.Bw), "pack B");
    } else {
        CU(cudaMemcpy2DAsync(w.T0, (size_t)n * 8, B, (size_t)ldb * 8, (size_t)n * 8, s, cudaMemcpyHostToDevice, cs), "copy B");
        KL(launch_pack(cs, s, n, w.T0, n, w.Bw), "pack B");
    }
    if (x_dev) {
        KL(launch_pack(cs, s, n, X, ldx, w.Xw), "pack X");
    } else {
        CU(cudaMemcpy2DAsync(w.T0, (size_t)n * 8, X, (size_t)ldx * 8, (size_t)n * 8, s, cudaMemcpyHostToDevice, cs), "copy X");
        KL(launch_pack(cs, s, n, w.T0, n, w.Xw), "pack X");
    }
    const size_t blk_elems = (size_t)n * s;
    const double nsd = (double)n * s;
    CU(cudaMemsetAsync(w.ticket, 0, 64, cs), "clear tickets");
    // column norms^2 of a block (one launch with the last-CTA sum for s <= 8)
    auto colnorms = [&](const double *Wb, double *out) -> spai_status {
        if (cqr_supported(s)) {
            PKL("colnorm2", 2.0 * nsd, 8.0 * nsd, launch_colnorm2_t(cs, s, n, Wb, w.partial, w.ticket, out), "norms");
        } else {
            PKL("colnorm2", 2.0 * nsd, 8.0 * nsd, launch_colnorm2(cs, s, n, Wb, w.partial, out, chunks), "norms");
        }
        return SPAI_OK;
    };
    double *h = ctx->h_pinned;  // [0,16) bnorm2, [16,32) rn2, [32,48) est, [48] flag, [49] error word
    KL(launch_colnorm2(cs, s, n, w.Bw, w.partial, w.nrm2, chunks), "norm B");
    CU(cudaMemcpyAsync(h, w.nrm2, s * 8, cudaMemcpyDeviceToHost, cs), "read norms");
    CU(cudaStreamSynchronize(cs), "sync");
    double thresh[16], bnorm[16];
    for (int i = 0; i < s; ++i) {
        bnorm[i] = sqrt(h[i]);
        thresh[i] = opts->tol * bnorm[i];
    }
    CU(cudaMemcpyAsync(w.thresh, thresh, s * 8, cudaMemcpyHostToDevice, cs), "write thresholds");

    auto residual = [&]() -> spai_status {
        PKL("residual", 2.0 * A->nnz * s + nsd, 12.0 * A->nnz + 4.0 * (n + 1) + 24.0 * nsd,
            launch_residual(cs, s, n, A->rowptr, A->colind, A->val, w.Xw, w.Bw, w.W), "residual");
        if ((st = colnorms(w.W, w.ref2))) return st;
        CU(cudaMemcpyAsync(h + 16, w.ref2, s * 8, cudaMemcpyDeviceToHost, cs), "read norms");
        CU(cudaStreamSynchronize(cs), "sync");
        return SPAI_OK;
    };
    auto converged = [&]() {
        for (int i = 0; i < s; ++i)
            if (!(sqrt(h[16 + i]) <= thresh[i])) return false;
        return true;
    };
    F32Vals a32v;
    if (mixed) {
        a32v.f32 = a32;
        PKL("round_f32", 0.0, 12.0 * A->nnz, launch_round_f32(cs, A->nnz, A->val, a32), "A in FP32");
    }
    // the FP32 operator's (A P) W = A (P V_j), intermediates FP32 in the Z / T blocks
    float *z32 = (float *)w.Z, *t032 = (float *)w.T0, *t132 = (float *)w.T1;
    const double nnzA = A->nnz;
    // Wout = A P Vin (FP64 products, or the FP32 operator of the mixed solve; Vin32, when
    // given, is Vin in FP32 and the FP32 operator reads it instead)
    auto apply_op = [&](const double *Vin, double *Wout, const float *Vin32 = nullptr) -> spai_status {
        if (mixed && Vin32) {
            if (P) {
                if ((st = apply32<float>(ctx, P, s, Vin32, z32, t032, t132))) return st;
                PKL("spmm32_A", 2.0 * nnzA * s, 8.0 * nnzA + 4.0 * (n + 1) + 12.0 * nsd,
                    launch_spmm32(cs, s, n, A->rowptr, A->colind, a32v, (const float *)z32, Wout), "A Z (FP32)");
            } else {
                PKL("spmm32_A", 2.0 * nnzA * s, 8.0 * nnzA + 4.0 * (n + 1) + 12.0 * nsd,
                    launch_spmm32(cs, s, n, A->rowptr, A->colind, a32v, Vin32, Wout), "A V (FP32)");
            }
        } else if (mixed) {
            if (P) {
                if ((st = apply32<float>(ctx, P, s, Vin, z32, t032, t132))) return st;
                PKL("spmm32_A", 2.0 * nnzA * s, 8.0 * nnzA + 4.0 * (n + 1) + 12.0 * nsd,
                    launch_spmm32(cs, s, n, A->rowptr, A->colind, a32v, (const float *)z32, Wout), "A Z (FP32)");
            } else {
                PKL("spmm32_A", 2.0 * nnzA * s, 8.0 * nnzA + 4.0 * (n + 1) + 16.0 * nsd,
                    launch_spmm32(cs, s, n, A->rowptr, A->colind, a32v, Vin, Wout), "A V (FP32)");
            }
        } else {
            const double *Zj = Vin;
            if (P) {
                if ((st = apply_rm(ctx, P, s, Vin, w.Z, w.T0, w.T1))) return st;
                Zj = w.Z;
            }
            PKL("spmm_A", 2.0 * A->nnz * s, 12.0 * A->nnz + 4.0 * (n + 1) + 16.0 * nsd,
                launch_spmm(cs, s, n, A->rowptr, A->colind, A->val, Zj, Wout), "A Z");
        }
        return SPAI_OK;
    };
    // Out += P Din (the preconditioner in the solve's arithmetic); Din is left as it is
    auto add_precond = [&](const double *Din, double *Out) -> spai_status {
        const double *U = Din;
        if (P && mixed) {
            if ((st = apply32<double>(ctx, P, s, Din, w.Z, t032, t132))) return st;
            U = w.Z;
        } else if (P) {
            if ((st = apply_rm(ctx, P, s, Din, w.Z, w.T0, w.T1))) return st;
            U = w.Z;
        }
        PKL("axpy", 2.0 * nsd, 24.0 * nsd, launch_axpy(cs, (int64_t)blk_elems, 1.0, U, Out), "X update");
        return SPAI_OK;
    };
    // H = V_{0..nb-1}^T Wsrc over the first nb basis slots
    auto gram_any = [&](int nb, double *Wsrc, double *H) -> spai_status {
        if (use_digits && (opts->orth == SPAI_ORTH_TENSOR || nb >= 2)) return gram_tc(nb, Wsrc, H);
        PKL("block_dot", 2.0 * nsd * s * nb, 8.0 * nsd * (nb + 1),
            launch_block_dot(cs, s, n, nb, w.V, Wsrc, w.partial, H, chunks), "block Gram product");
        return SPAI_OK;
    };
    if (rc) KL(launch_zero(cs, (int64_t)blk_elems, w.Xh), "zero the GCRO iterate");
    // the recycled space's image: C T = A P U block by block (two passes of block CGS against
    // the C blocks before it, Cholesky-QR), C_i in basis slot i, U <- U T^{-1} in place
    for (int i = 0; i < kb; ++i) {
        double *Ui = rc->U + (size_t)i * blk_elems;
        if ((st = apply_op(Ui, w.W))) return st;
        if ((st = colnorms(w.W, w.ref2))) return st;
        if (i > 0) {
            if ((st = gram_any(i, w.W, w.H1))) return st;
            if ((st = vupdate(i, w.H1, w.W, w.W, -1.0))) return st;
            if ((st = gram_any(i, w.W, w.H2))) return st;
            if ((st = vupdate(i, w.H2, w.W, w.W, -1.0))) return st;
            KL(launch_axpy(cs, (int64_t)i * s * s, 1.0, w.H2, w.H1), "T column");
        }
        if ((st = cholqr2(ctx, w, n, s, w.W, w.V + (size_t)i * blk_elems, w.Rn, w.ref2,
                          (use_digits && !halves) ? i : -1, ipad)))
            return st;
        if ((st = fixed16(i))) return st;
        // U_i <- (U_i - U_{<i} T_{<i,i}) T_ii^{-1}; columns deflated in the Cholesky-QR -> 0
        if (i > 0) KL(launch_block_update(cs, s, n, i, rc->U, w.H1, Ui, w.D, -1.0), "recycled space");
        KL(launch_trsm_rows(cs, s, n, i > 0 ? w.D : Ui, w.Rn, w.defl2, Ui), "recycled space");
    }
    if ((st = residual())) return st;
    int cycles = 0, iters = 0;
    while (!converged() && cycles < opts->max_cycles) {
        ++cycles;
        if (kb > 0) {
            // start from the residual projected off C: X~ += U C^T R, R -= C C^T R
            if ((st = gram_any(kb, w.W, w.H1))) return st;
            KL(launch_block_update(cs, s, n, kb, rc->U, w.H1, nullptr, w.D, 1.0), "U C^T R");
            if ((st = vupdate(kb, w.H1, w.W, w.W, -1.0))) return st;
            KL(launch_axpy(cs, (int64_t)blk_elems, 1.0, w.D, w.Xh), "GCRO iterate");
            if ((st = add_precond(w.D, w.Xw))) return st;
            if ((st = colnorms(w.W, w.ref2))) return st;
            CU(cudaMemcpyAsync(h + 16, w.ref2, s * 8, cudaMemcpyDeviceToHost, cs), "read norms");
            CU(cudaStreamSynchronize(cs), "sync");
            if (converged()) {  // the recycled space held the solution: confirm with the true residual
                if ((st = residual())) return st;
                continue;
            }
        }
        if (mixed) {
            // iterative refinement: this cycle solves the correction equation from the FP64 true
            // residual r; its FP32 operator resolves r only to ~FP32 rounding, so the cycle stops
            // once every column's estimate is below max(tol ||b_i||, eta ||r_i||), and the next
            // cycle starts from the new FP64 true residual
            double cthr[16];
            for (int i = 0; i < s; ++i) cthr[i] = std::max(thresh[i], kMixedCycleReduction * sqrt(h[16 + i]));
            CU(cudaMemcpyAsync(w.thresh, cthr, s * 8, cudaMemcpyHostToDevice, cs), "write thresholds");
        }
        // V_0 S_0 = R (ref2 holds the residual norms^2), in basis slot kb (and in FP32 for the
        // mixed solve's operator)
        float *v32 = mixed ? w.V32 : nullptr;
        if ((st = cholqr2(ctx, w, n, s, w.W, w.V + (size_t)kb * blk_elems, w.Rn, w.ref2,
                          (use_digits && !halves) ? kb : -1, ipad, v32)))
            return st;
        if ((st = fixed16(kb))) return st;
        PKL("small_dense", 0.0, 0.0, launch_ls_prefix(cs, s, kb, mt, w.Rn, w.Qs, w.Rtri, w.G), "rhs");
        int J = 0;
        for (int j = 0; j < m; ++j) {
            const double *Vj = w.V + (size_t)(kb + j) * blk_elems;
            if ((st = apply_op(Vj, w.W, v32))) return st;
            // the deflation scale, W's column norms before the projections: for s <= 8 the
            // first Cholesky-QR pass forms them from the projections' coefficients
            if (!cqr_supported(s) && (st = colnorms(w.W, w.ref2))) return st;
            // two passes of block classical Gram-Schmidt against C_0..C_{kb-1}, V_0..V_j
            const int nb = kb + j + 1;
            if ((st = gram_any(nb, w.W, w.H1))) return st;
            if ((st = vupdate(nb, w.H1, w.W, w.W, -1.0))) return st;
            if ((st = gram_any(nb, w.W, w.H2))) return st;
            if ((st = vupdate(nb, w.H2, w.W, w.W, -1.0))) return st;
            double *Vn = w.V + (size_t)(kb + j + 1) * blk_elems;
            // the new block's fixed point (for the products of the next steps) comes with it
            if ((st = cholqr2(ctx, w, n, s, w.W, Vn, w.Rn, w.ref2,
                              (use_digits && !halves && j + 1 < m) ? kb + j + 1 : -1, ipad, j + 1 < m ? v32 : nullptr,
                              w.H1, w.H2, nb * s)))
                return st;
            if (j + 1 < m && (st = fixed16(kb + j + 1))) return st;
            PKL("arnoldi_ls", 16.0 * s * s * s * (nb), 0.0,
                launch_arnoldi_ls(cs, s, kb + j, mt, w.H1, w.H2, w.Rn, w.Qs, w.Rtri, w.G, w.thresh, w.est, w.flag),
                "least squares");
            CU(cudaMemcpyAsync(h + 32, w.est, s * 8, cudaMemcpyDeviceToHost, cs), "read estimates");
            CU(cudaMemcpyAsync(h + 48, w.flag, 4, cudaMemcpyDeviceToHost, cs), "read flag");
            CU(cudaMemcpyAsync(h + 49, ctx->d_err, 4, cudaMemcpyDeviceToHost, cs), "read error word");
            CU(cudaStreamSynchronize(cs), "sync");
            ++iters;
            J = j + 1;
            if (*(int32_t *)(h + 49) & ERR_TIMEOUT) {  // a bounded wait gave up: stop at once
                int h_err = 0;
                if ((st = read_err(ctx, &h_err))) return st;
                return fail(ctx, SPAI_ETIMEOUT, "a bounded wait in a tensor-core product gave up (Arnoldi step %d)",
                            iters);
            }
            if (*(int32_t *)(h + 48)) break;
        }
        // X += P ([U, V] Y)
        PKL("backsolve", (double)(kb + J) * s * (kb + J) * s * s, 0.0,
            launch_backsolve(cs, s, kb + J, (mt + 1) * s, w.Rtri, w.G, w.Y), "back substitution");
        if (kb > 0) {
            KL(launch_block_update(cs, s, n, kb, rc->U, w.Y, nullptr, w.D, 1.0), "U Y_U");
            if ((st = vupdate_at(kb, J, w.Y + (size_t)kb * s * s, w.D, w.W, 1.0))) return st;
        } else {
            if ((st = vupdate(J, w.Y, nullptr, w.W, 1.0))) return st;
        }
        if (rc) KL(launch_axpy(cs, (int64_t)blk_elems, 1.0, w.W, w.Xh), "GCRO iterate");
        if ((st = add_precond(w.W, w.Xw))) return st;
        if ((st = residual())) return st;
    }
    // solution out
    if (x_dev) {
        KL(launch_unpack(cs, s, n, w.Xw, X, ldx), "unpack X");
    } else {
        KL(launch_unpack(cs, s, n, w.Xw, w.T0, n), "unpack X");
        CU(cudaMemcpy2DAsync(X, (size_t)ldx * 8, w.T0, (size_t)n * 8, (size_t)n * 8, s, cudaMemcpyDeviceToHost, cs), "copy X");
    }
    CU(cudaStreamSynchronize(cs), "sync");
    {
        int h_err = 0;
        if ((st = read_err(ctx, &h_err))) return st;
        if (h_err & ERR_TIMEOUT) return fail(ctx, SPAI_ETIMEOUT, "a bounded wait in the tensor-core Gram product gave up");
        if (h_err & ERR_RANGE) return fail(ctx, SPAI_EINVAL, "basis entry out of the digit range (|v| >= 2) or a non-finite block");
    }
    int worst = 0;
    double worst_rel = -1.0;
    bool conv = true;
    for (int i = 0; i < s; ++i) {
        const double rn = sqrt(h[16 + i]);
        const double rel = bnorm[i] > 0 ? rn / bnorm[i] : rn;
        if (rel > worst_rel) { worst_rel = rel; worst = i; }
        if (!(rn <= thresh[i])) conv = false;
        if (rel_residual) rel_residual[i] = rel;
    }
    if (info) {
        info->iterations = iters;
        info->cycles = cycles;
        info->converged = conv ? 1 : 0;
        info->worst_column = worst;
        info->max_rel_residual = worst_rel;
    }
    if (!conv) return fail(ctx, SPAI_ENOTCONV, "not converged after %d cycles: column %d relative residual %.3e",
                           cycles, worst, worst_rel);
    if (rc && kbmax > 0) {
        // the solve's iterate joins the recycled space (the oldest block leaves a full one)
        if (kb == kbmax) {
            for (int i = 0; i + 1 < kbmax; ++i)
                CU(cudaMemcpyAsync(rc->U + (size_t)i * blk_elems, rc->U + (size_t)(i + 1) * blk_elems, blk_elems * 8,
                                   cudaMemcpyDeviceToDevice, cs),
                   "recycled space");
            kb = kbmax - 1;
        }
        CU(cudaMemcpyAsync(rc->U + (size_t)kb * blk_elems, w.Xh, blk_elems * 8, cudaMemcpyDeviceToDevice, cs),
           "recycled space");
        rc->k = (kb + 1) * s;
        CU(cudaStreamSynchronize(cs), "sync");
    }
    return SPAI_OK;
}

}  // namespace

extern "C" spai_status block_solve(spai_ctx ctx, const spai_csr *A, spai_pc P, int32_t s, const double *B,
                                   int64_t ldb, double *X, int64_t ldx, const spai_solve_opts *opts,
                                   spai_solve_info *info, double *rel_residual)
{
    return solve_impl(ctx, A, P, s, B, ldb, X, ldx, opts, info, rel_residual, nullptr);
}

extern "C" spai_status block_solve_gcro(spai_ctx ctx, const spai_csr *A, spai_pc P, int32_t s, const double *B,
                                        int64_t ldb, double *X, int64_t ldx, const spai_solve_opts *opts,
                                        spai_recycle rc, spai_solve_info *info, double *rel_residual)
{
    if (!ctx) return SPAI_EINVAL;
    if (!rc) return fail(ctx, SPAI_EINVAL, "NULL recycle space");
    return solve_impl(ctx, A, P, s, B, ldb, X, ldx, opts, info, rel_residual, rc);
}

extern "C" spai_status spai_recycle_create(spai_ctx ctx, int32_t n, int32_t s, int32_t kmax, spai_recycle *out)
{
    if (!ctx || !out) return fail(ctx, SPAI_EINVAL, "NULL argument");
    *out = nullptr;
    if (n < 1 || !valid_s(s) || kmax < 0 || kmax % s != 0 || kmax / s > kMaxRecycleBlocks)
        return fail(ctx, SPAI_EINVAL, "recycle space: n >= 1, s in {1,2,4,8,16}, kmax a multiple of s, kmax / s <= %d",
                    kMaxRecycleBlocks);
    spai_recycle r = new spai_recycle_s();
    r->ctx = ctx;
    r->n = n;
    r->s = s;
    r->kmax = kmax;
    if (kmax > 0) {
        spai_status st = dalloc_n(ctx, &r->U, (int64_t)n * kmax);
        if (st) {
            delete r;
            return st;
        }
    }
    *out = r;
    return SPAI_OK;
}

extern "C" spai_status spai_recycle_info(spai_recycle r, int32_t *k)
{
    if (!r) return SPAI_EINVAL;
    if (k) *k = r->k;
    return SPAI_OK;
}

extern "C" spai_status spai_recycle_export(spai_ctx ctx, spai_recycle r, double *U, int64_t ldu)
{
    if (!ctx || !r) return fail(ctx, SPAI_EINVAL, "NULL argument");
    if (r->k == 0) return SPAI_OK;
    if (!U || ldu < r->n) return fail(ctx, SPAI_EINVAL, "bad export arguments");
    const int32_t s = r->s, n = r->n;
    for (int i = 0; i < r->k / s; ++i)
        KL(launch_unpack(ctx->stream, s, n, r->U + (size_t)i * n * s, U + (size_t)i * s * ldu, ldu), "unpack");
    return SPAI_OK;
}

extern "C" spai_status spai_recycle_clear(spai_recycle r)
{
    if (!r) return SPAI_EINVAL;
    r->k = 0;
    return SPAI_OK;
}

extern "C" spai_status spai_recycle_destroy(spai_recycle r)
{
    if (!r) return SPAI_EINVAL;
    dfree(r->ctx, r->U);
    delete r;
    return SPAI_OK;
}

// ===================================================================================
// Batched block GMRES: many independent systems in lockstep
// ===================================================================================
namespace {

// Device memory of one batched solve, released together.
struct Allocs {
    spai_ctx ctx;
    std::vector<void *> ptrs;
    explicit Allocs(spai_ctx c) : ctx(c) {}
    ~Allocs()
    {
        for (void *p : ptrs) dfree(ctx, p);
    }
    template <class Tp>
    spai_status get(Tp **p, int64_t count)
    {
        spai_status st = dalloc_n(ctx, p, count);
        if (!st) ptrs.push_back((void *)*p);
        return st;
    }
};

// one level of the stacked preconditioner chain: the factors of every system at that depth
struct StackedFactor {
    bool diag = false;
    int prec = 0;  // 0 FP64, 1 FP32, 2 BF16
    int32_t *rowptr = nullptr, *colind = nullptr;
    void *val = nullptr;
    int64_t nnz = 0;
};

}  // namespace

extern "C" spai_status block_solve_batch(spai_ctx ctx, int32_t nsys, const spai_csr *A, const spai_pc *P, int32_t s,
                                         const double *const *B, double *const *X, const spai_solve_opts *opts,
                                         spai_solve_info *info)
{
    if (!ctx) return SPAI_EINVAL;
    if (!A || !B || !X || !opts || !info) return fail(ctx, SPAI_EINVAL, "NULL argument");
    if (nsys < 1 || nsys > 65536) return fail(ctx, SPAI_EINVAL, "nsys must be in 1..65536");
    if (!valid_s(s)) return fail(ctx, SPAI_EINVAL, "s must be 1, 2, 4, 8 or 16");
    const int32_t m = opts->restart;
    if (m < 1 || opts->max_cycles < 1 || !(opts->tol >= 0.0))
        return fail(ctx, SPAI_EINVAL, "restart and max_cycles must be >= 1 and tol >= 0");
    spai_status st;
    std::vector<int64_t> off((size_t)nsys + 1, 0), nzoff((size_t)nsys + 1, 0);
    int depth = -1;
    for (int i = 0; i < nsys; ++i) {
        if ((st = check_csr_args(ctx, &A[i], "A"))) return st;
        if (A[i].n < 1) return fail(ctx, SPAI_EINVAL, "system %d is empty", i);
        if (!is_device_ptr(A[i].rowptr) || !is_device_ptr(A[i].colind) || !is_device_ptr(A[i].val))
            return fail(ctx, SPAI_EINVAL, "system %d: A arrays must be device memory", i);
        if (!B[i] || !X[i] || !is_device_ptr(B[i]) || !is_device_ptr(X[i]))
            return fail(ctx, SPAI_EINVAL, "system %d: B and X must be device memory", i);
        off[i + 1] = off[i] + A[i].n;
        nzoff[i + 1] = nzoff[i] + A[i].nnz;
        const int d = P ? (P[i] ? P[i]->depth : -2) : -1;
        if (P && (!P[i] || P[i]->sym->n != A[i].n))
            return fail(ctx, SPAI_EINVAL, "system %d: preconditioner missing or of another size", i);
        if (i == 0) depth = d;
        else if (d != depth) return fail(ctx, SPAI_EINVAL, "all preconditioners must have the same depth");
    }
    if (off[nsys] >= INT32_MAX || nzoff[nsys] >= INT32_MAX)
        return fail(ctx, SPAI_EINVAL, "the stacked batch exceeds 2^31 rows or nonzeros");
    const int32_t ntot = (int32_t)off[nsys];
    const int64_t nnz = nzoff[nsys];
    memset(info, 0, sizeof(spai_solve_info) * (size_t)nsys);
    cudaStream_t cs = ctx->stream;
    Allocs al(ctx);

    // ---- the block-diagonal union of the systems (CSR, global row and column indices)
    int32_t *rp = nullptr, *ci = nullptr;
    double *va = nullptr;
    if ((st = al.get(&rp, (int64_t)ntot + 1)) || (st = al.get(&ci, nnz)) || (st = al.get(&va, nnz))) return st;
    for (int i = 0; i < nsys; ++i) {
        KL(launch_add_i32(cs, (int64_t)A[i].n + 1, A[i].rowptr, (int32_t)nzoff[i], rp + off[i]), "stack rows");
        KL(launch_add_i32(cs, A[i].nnz, A[i].colind, (int32_t)off[i], ci + nzoff[i]), "stack columns");
        if (A[i].nnz)
            CU(cudaMemcpyAsync(va + nzoff[i], A[i].val, (size_t)A[i].nnz * 8, cudaMemcpyDeviceToDevice, cs), "stack");
    }
    // ---- the preconditioner chains, level by level from the root (P_l X = Q_l (P_1 X))
    std::vector<StackedFactor> levels;
    if (P) {
        std::vector<std::vector<spai_pc>> chains((size_t)nsys);
        for (int i = 0; i < nsys; ++i)
            for (spai_pc p = P[i]; p; p = p->parent) chains[i].insert(chains[i].begin(), p);
        const int L = (int)chains[0].size();
        for (int l = 0; l < L; ++l) {
            StackedFactor f;
            const spai_pc h0 = chains[0][l];
            f.diag = h0->diag;
            f.prec = h0->fval16 ? 2 : h0->fval32 ? 1 : 0;
            int64_t tot = 0;
            std::vector<int64_t> foff((size_t)nsys + 1, 0);
            for (int i = 0; i < nsys; ++i) {
                const spai_pc h = chains[i][l];
                if ((int)chains[i].size() != L || h->diag != f.diag || (h->fval16 ? 2 : h->fval32 ? 1 : 0) != f.prec)
                    return fail(ctx, SPAI_EINVAL, "preconditioner level %d differs between systems (kind or precision)", l);
                foff[i + 1] = foff[i] + (f.diag ? h->sym->n : h->sym->nnzP);
            }
            tot = foff[nsys];
            if (tot >= INT32_MAX) return fail(ctx, SPAI_EINVAL, "the stacked preconditioner exceeds 2^31 entries");
            f.nnz = tot;
            const size_t vb = f.prec == 2 ? 2 : f.prec == 1 ? 4 : 8;
            char *v = nullptr;
            if ((st = al.get(&v, tot * (int64_t)vb))) return st;
            f.val = v;
            if (!f.diag && ((st = al.get(&f.rowptr, (int64_t)ntot + 1)) || (st = al.get(&f.colind, tot)))) return st;
            for (int i = 0; i < nsys; ++i) {
                const spai_pc h = chains[i][l];
                const Sym *sy = h->sym;
                const int64_t cnt = foff[i + 1] - foff[i];
                const void *src = f.prec == 2 ? (const void *)h->fval16 : f.prec == 1 ? (const void *)h->fval32
                                                                                      : (const void *)h->fval;
                if (cnt) CU(cudaMemcpyAsync(v + foff[i] * vb, src, (size_t)cnt * vb, cudaMemcpyDeviceToDevice, cs), "stack");
                if (!f.diag) {
                    KL(launch_add_i32(cs, (int64_t)sy->n + 1, sy->p_rowptr, (int32_t)foff[i], f.rowptr + off[i]), "stack rows");
                    KL(launch_add_i32(cs, sy->nnzP, sy->p_colind, (int32_t)off[i], f.colind + foff[i]), "stack columns");
                }
            }
            levels.push_back(f);
        }
    }
    // ---- row chunks that never straddle two systems
    constexpr int64_t kChunkRows = 1024;
    std::vector<int32_t> csys, c0((size_t)nsys + 1, 0);
    std::vector<int64_t> cr0, cr1;
    for (int i = 0; i < nsys; ++i) {
        c0[i] = (int32_t)csys.size();
        for (int64_t r = off[i]; r < off[i + 1]; r += kChunkRows) {
            csys.push_back(i);
            cr0.push_back(r);
            cr1.push_back(std::min(r + kChunkRows, off[i + 1]));
        }
    }
    c0[nsys] = (int32_t)csys.size();
    const int32_t nch = (int32_t)csys.size();
    int32_t *d_csys = nullptr, *d_c0 = nullptr;
    int64_t *d_r0 = nullptr, *d_r1 = nullptr;
    if ((st = al.get(&d_csys, nch)) || (st = al.get(&d_c0, (int64_t)nsys + 1)) || (st = al.get(&d_r0, nch)) ||
        (st = al.get(&d_r1, nch)))
        return st;
    CU(cudaMemcpyAsync(d_csys, csys.data(), (size_t)nch * 4, cudaMemcpyHostToDevice, cs), "chunks");
    CU(cudaMemcpyAsync(d_c0, c0.data(), ((size_t)nsys + 1) * 4, cudaMemcpyHostToDevice, cs), "chunks");
    CU(cudaMemcpyAsync(d_r0, cr0.data(), (size_t)nch * 8, cudaMemcpyHostToDevice, cs), "chunks");
    CU(cudaMemcpyAsync(d_r1, cr1.data(), (size_t)nch * 8, cudaMemcpyHostToDevice, cs), "chunks");
    const SegChunks sc{d_csys, d_r0, d_r1, d_c0, nch, nsys};
    // Systems leave the lockstep as they finish: jlim[b] is system b's step limit in the
    // current cycle (m while it takes Arnoldi steps, the steps it took once its residual
    // estimate met tol, 0 once its true residual did), and sca lists the row chunks of the
    // systems still stepping (a compacted copy of sc, rebuilt when one stops), so that the
    // per-step kernels run over those rows only.
    int32_t *d_csys_a = nullptr, *d_c0_a = nullptr, *d_jlim = nullptr;
    int64_t *d_r0_a = nullptr, *d_r1_a = nullptr;
    if ((st = al.get(&d_csys_a, nch)) || (st = al.get(&d_c0_a, (int64_t)nsys + 1)) || (st = al.get(&d_r0_a, nch)) ||
        (st = al.get(&d_r1_a, nch)) || (st = al.get(&d_jlim, nsys)))
        return st;
    SegChunks sca{d_csys_a, d_r0_a, d_r1_a, d_c0_a, 0, nsys};
    std::vector<int32_t> jlim((size_t)nsys, m), csys_a, c0_a((size_t)nsys + 1, 0);
    std::vector<int64_t> r0_a, r1_a;
    csys_a.reserve((size_t)nch);
    r0_a.reserve((size_t)nch);
    r1_a.reserve((size_t)nch);
    double rows_a = 0.0, nnz_a = 0.0;  // rows and nonzeros of A in the listed chunks
    auto set_active = [&]() -> spai_status {
        csys_a.clear();
        r0_a.clear();
        r1_a.clear();
        rows_a = nnz_a = 0.0;
        for (int i = 0; i < nsys; ++i) {
            c0_a[i] = (int32_t)csys_a.size();
            if (jlim[i] != m) continue;
            rows_a += (double)A[i].n;
            nnz_a += (double)A[i].nnz;
            for (int32_t c = c0[i]; c < c0[i + 1]; ++c) {
                csys_a.push_back(i);
                r0_a.push_back(cr0[c]);
                r1_a.push_back(cr1[c]);
            }
        }
        c0_a[nsys] = (int32_t)csys_a.size();
        sca.nchunks = c0_a[nsys];
        if (sca.nchunks) {
            CU(cudaMemcpyAsync(d_csys_a, csys_a.data(), (size_t)sca.nchunks * 4, cudaMemcpyHostToDevice, cs), "chunks");
            CU(cudaMemcpyAsync(d_r0_a, r0_a.data(), (size_t)sca.nchunks * 8, cudaMemcpyHostToDevice, cs), "chunks");
            CU(cudaMemcpyAsync(d_r1_a, r1_a.data(), (size_t)sca.nchunks * 8, cudaMemcpyHostToDevice, cs), "chunks");
        }
        CU(cudaMemcpyAsync(d_c0_a, c0_a.data(), ((size_t)nsys + 1) * 4, cudaMemcpyHostToDevice, cs), "chunks");
        CU(cudaMemcpyAsync(d_jlim, jlim.data(), (size_t)nsys * 4, cudaMemcpyHostToDevice, cs), "step limits");
        return SPAI_OK;
    };

    // ---- workspace: n_tot x s blocks, the basis, and every system's small blocks
    const int64_t blk = (int64_t)ntot * s, ss = (int64_t)s * s;
    double *Bw, *Xw, *W, *Z, *T0, *T1, *V, *partial;
    double *H1, *H2, *G1, *R1, *R2, *Rn, *ref2, *thresh, *Qs, *Rtri, *Gv, *Y, *est;
    int32_t *defl1, *defl2, *flag;
    if ((st = al.get(&Bw, blk)) || (st = al.get(&Xw, blk)) || (st = al.get(&W, blk)) || (st = al.get(&Z, blk)) ||
        (st = al.get(&T0, blk)) || (st = al.get(&T1, blk)) || (st = al.get(&V, blk * (m + 1))) ||
        (st = al.get(&partial, (int64_t)nch * std::max<int64_t>((int64_t)(m + 1) * ss, s))) ||
        (st = al.get(&H1, nsys * (m + 1) * ss)) || (st = al.get(&H2, nsys * (m + 1) * ss)) ||
        (st = al.get(&G1, nsys * ss)) || (st = al.get(&R1, nsys * ss)) || (st = al.get(&R2, nsys * ss)) ||
        (st = al.get(&Rn, nsys * ss)) || (st = al.get(&ref2, (int64_t)nsys * s)) ||
        (st = al.get(&thresh, (int64_t)nsys * s)) || (st = al.get(&Qs, nsys * (int64_t)m * 4 * ss)) ||
        (st = al.get(&Rtri, nsys * (int64_t)(m + 1) * s * m * s)) || (st = al.get(&Gv, nsys * (m + 1) * ss)) ||
        (st = al.get(&Y, nsys * (int64_t)m * ss)) || (st = al.get(&est, (int64_t)nsys * s)) ||
        (st = al.get(&defl1, (int64_t)nsys * s)) || (st = al.get(&defl2, (int64_t)nsys * s)) ||
        (st = al.get(&flag, nsys)))
        return st;

    // Y = P X through the stacked chain (T0 / T1 between levels); on the rows of the systems
    // still stepping when `active` (the factors' nonzeros counted in proportion to the rows)
    auto apply_P = [&](const double *Xin, double *Yout, bool active) -> spai_status {
        const double *cur = Xin;
        for (size_t l = 0; l < levels.size(); ++l) {
            const StackedFactor &f = levels[l];
            double *dst = (l + 1 == levels.size()) ? Yout : ((l & 1) ? T1 : T0);
            if (active) {
                const double share = rows_a / (double)ntot, fnz = (double)f.nnz * share, ab = rows_a * s;
                if (f.diag) {
                    PKL("scale_rows", ab, 8.0 * rows_a + 16.0 * ab,
                        launch_scale_rows_seg(cs, s, sca.nchunks, kChunkRows, d_r0_a, d_r1_a,
                                              f.prec == 0 ? (const double *)f.val : nullptr,
                                              f.prec == 1 ? (const float *)f.val : nullptr,
                                              f.prec == 2 ? (const uint16_t *)f.val : nullptr, cur, dst),
                        "diagonal factor apply");
                } else {
                    const double vb = f.prec == 2 ? 6.0 : f.prec == 1 ? 8.0 : 12.0;
                    PKL("spmm_P", 2.0 * fnz * s, vb * fnz + 4.0 * rows_a + 16.0 * ab,
                        launch_spmm_seg(cs, s, sca.nchunks, kChunkRows, d_r0_a, d_r1_a, f.rowptr, f.colind,
                                        f.prec == 0 ? (const double *)f.val : nullptr,
                                        f.prec == 1 ? (const float *)f.val : nullptr,
                                        f.prec == 2 ? (const uint16_t *)f.val : nullptr, cur, dst),
                        "apply");
                }
                cur = dst;
                continue;
            }
            const double fl = 2.0 * (double)f.nnz * s;
            if (f.diag) {
                PKL("scale_rows", (double)ntot * s, 8.0 * ntot + 16.0 * blk,
                    launch_scale_rows(cs, s, ntot, f.prec == 0 ? (const double *)f.val : nullptr,
                                      f.prec == 1 ? (const float *)f.val : nullptr,
                                      f.prec == 2 ? (const uint16_t *)f.val : nullptr, cur, dst),
                    "diagonal factor apply");
            } else if (f.prec == 2) {
                PKL("spmm_P", fl, 6.0 * f.nnz + 4.0 * (ntot + 1) + 16.0 * blk,
                    launch_spmm_bf16v(cs, s, ntot, f.rowptr, f.colind, (const uint16_t *)f.val, cur, dst), "apply");
            } else if (f.prec == 1) {
                PKL("spmm_P", fl, 8.0 * f.nnz + 4.0 * (ntot + 1) + 16.0 * blk,
                    launch_spmm_f32v(cs, s, ntot, f.rowptr, f.colind, (const float *)f.val, cur, dst), "apply");
            } else {
                PKL("spmm_P", fl, 12.0 * f.nnz + 4.0 * (ntot + 1) + 16.0 * blk,
                    launch_spmm(cs, s, ntot, f.rowptr, f.colind, (const double *)f.val, cur, dst), "apply");
            }
            cur = dst;
        }
        return SPAI_OK;
    };
    // W = Q R per system still stepping, two passes of Cholesky QR (the block_solve sequence,
    // per system)
    auto cholqr2_b = [&](const double *Win, double *Qout) -> spai_status {
        const double nsd = rows_a * s;
        PKL("gram", nsd * (s + 1), 8.0 * nsd, launch_gram_seg(cs, s, Win, sca, partial, G1), "gram");
        PKL("small_dense", 0.0, 0.0, launch_chol_small_b(cs, s, nsys, G1, ref2, 1e-24, R1, defl1), "chol");
        PKL("trsm_gram", nsd * s + nsd * (s + 1), 16.0 * nsd,
            launch_trsm_gram_seg(cs, s, Win, R1, defl1, Qout, sca, partial, G1), "trsm gram");
        PKL("small_dense", 0.0, 0.0, launch_chol_small_b(cs, s, nsys, G1, nullptr, 0.0, R2, defl2), "chol");
        PKL("trsm_rows", nsd * s, 16.0 * nsd, launch_trsm_rows_seg(cs, s, Qout, R2, defl2, Qout, sca), "trsm");
        PKL("small_dense", 0.0, 0.0, launch_triu_mul_b(cs, s, nsys, R2, R1, Rn), "triu");
        return SPAI_OK;
    };

    // inputs -> stacked row-major blocks
    for (int i = 0; i < nsys; ++i) {
        KL(launch_pack(cs, s, A[i].n, B[i], A[i].n, Bw + off[i] * s), "pack B");
        KL(launch_pack(cs, s, A[i].n, X[i], A[i].n, Xw + off[i] * s), "pack X");
    }
    std::vector<double> hb((size_t)nsys * s), hr((size_t)nsys * s), bnorm((size_t)nsys * s), th((size_t)nsys * s);
    std::vector<int32_t> hflag((size_t)nsys);
    KL(launch_colnorm2_seg(cs, s, Bw, sc, partial, ref2), "norm B");
    CU(cudaMemcpyAsync(hb.data(), ref2, hb.size() * 8, cudaMemcpyDeviceToHost, cs), "read norms");
    CU(cudaStreamSynchronize(cs), "sync");
    for (size_t k = 0; k < hb.size(); ++k) {
        bnorm[k] = sqrt(hb[k]);
        th[k] = opts->tol * bnorm[k];
    }
    CU(cudaMemcpyAsync(thresh, th.data(), th.size() * 8, cudaMemcpyHostToDevice, cs), "thresholds");
    CU(cudaStreamSynchronize(cs), "sync");  // th is read by the copy above
    auto residual = [&]() -> spai_status {
        PKL("residual", 2.0 * nnz * s + blk, 12.0 * nnz + 4.0 * (ntot + 1) + 24.0 * blk,
            launch_residual(cs, s, ntot, rp, ci, va, Xw, Bw, W), "residual");
        PKL("colnorm2", 2.0 * blk, 8.0 * blk, launch_colnorm2_seg(cs, s, W, sc, partial, ref2), "residual norms");
        CU(cudaMemcpyAsync(hr.data(), ref2, hr.size() * 8, cudaMemcpyDeviceToHost, cs), "read norms");
        CU(cudaStreamSynchronize(cs), "sync");
        return SPAI_OK;
    };
    auto sys_converged = [&](int i) {
        for (int c = 0; c < s; ++c)
            if (!(sqrt(hr[(size_t)i * s + c]) <= th[(size_t)i * s + c])) return false;
        return true;
    };
    auto all_converged = [&]() {
        for (int i = 0; i < nsys; ++i)
            if (!sys_converged(i)) return false;
        return true;
    };
    if ((st = residual())) return st;
    // per system: the cycle after which its true residual met tol (0: at the start), and
    // the Arnoldi steps it took (it takes none once its steps of a cycle are over)
    std::vector<int> conv_cycle((size_t)nsys, -1), own_it((size_t)nsys, 0);
    int cycles = 0;
    for (int i = 0; i < nsys; ++i)
        if (sys_converged(i)) conv_cycle[i] = 0;
    while (!all_converged() && cycles < opts->max_cycles) {
        ++cycles;
        int nact = 0;
        for (int i = 0; i < nsys; ++i) {
            jlim[i] = conv_cycle[i] >= 0 ? 0 : m;
            nact += jlim[i] == m;
        }
        if ((st = set_active())) return st;
        if ((st = cholqr2_b(W, V))) return st;
        PKL("small_dense", 0.0, 0.0, launch_set_rhs_b(cs, s, nsys, m, Rn, Gv), "rhs");
        int J = 0;
        for (int j = 0; j < m && nact > 0; ++j) {
            const double *Vj = V + (int64_t)j * blk;
            const double *Zj = Vj;
            if (!levels.empty()) {
                if ((st = apply_P(Vj, Z, true))) return st;
                Zj = Z;
            }
            const double ab = rows_a * s;
            PKL("spmm_A", 2.0 * nnz_a * s, 12.0 * nnz_a + 4.0 * rows_a + 16.0 * ab,
                launch_spmm_seg(cs, s, sca.nchunks, kChunkRows, d_r0_a, d_r1_a, rp, ci, va, nullptr, nullptr, Zj, W),
                "A Z");
            PKL("colnorm2", 2.0 * ab, 8.0 * ab, launch_colnorm2_seg(cs, s, W, sca, partial, ref2), "norms");
            const double nb = j + 1, f = 2.0 * ab * s * nb, by = 8.0 * ab * (nb + 1);
            const int64_t hs = (int64_t)(m + 1) * ss;
            PKL("block_dot", f, by, launch_block_dot_seg(cs, s, ntot, j + 1, V, W, sca, partial, H1, hs), "H1");
            PKL("block_update", f, 8.0 * ab * (nb + 2),
                launch_block_update_seg(cs, s, ntot, j + 1, V, H1, hs, W, W, -1.0, sca), "update");
            PKL("block_dot", f, by, launch_block_dot_seg(cs, s, ntot, j + 1, V, W, sca, partial, H2, hs), "H2");
            PKL("block_update", f, 8.0 * ab * (nb + 2),
                launch_block_update_seg(cs, s, ntot, j + 1, V, H2, hs, W, W, -1.0, sca), "update");
            if ((st = cholqr2_b(W, V + (int64_t)(j + 1) * blk))) return st;
            PKL("arnoldi_ls", 16.0 * ss * s * (j + 1) * nact, 0.0,
                launch_arnoldi_ls_b(cs, s, nsys, j, m, H1, H2, Rn, Qs, Rtri, Gv, thresh, est, flag, d_jlim),
                "least squares");
            CU(cudaMemcpyAsync(hflag.data(), flag, (size_t)nsys * 4, cudaMemcpyDeviceToHost, cs), "read flags");
            CU(cudaStreamSynchronize(cs), "sync");
            J = j + 1;
            int stopped = 0;
            for (int i = 0; i < nsys; ++i) {
                if (jlim[i] != m) continue;
                ++own_it[i];
                if (!hflag[i]) continue;
                jlim[i] = j + 1;  // its estimate met tol: its steps of this cycle are over
                ++stopped;
            }
            nact -= stopped;
            if (stopped && nact > 0 && (st = set_active())) return st;
        }
        // X += P (V Y), every system with its own Y over its own steps (none for a system
        // that had converged before the cycle, whose X is left as it was)
        CU(cudaMemcpyAsync(d_jlim, jlim.data(), (size_t)nsys * 4, cudaMemcpyHostToDevice, cs), "step limits");
        PKL("backsolve", (double)J * s * J * s * s * nsys, 0.0,
            launch_backsolve_b(cs, s, nsys, J, m, Rtri, Gv, Y, d_jlim), "back substitution");
        PKL("block_update", 2.0 * blk * s * J, 8.0 * blk * (J + 2),
            launch_block_update_seg(cs, s, ntot, J, V, Y, (int64_t)m * ss, nullptr, W, 1.0, sc, d_jlim), "V Y");
        const double *U = W;
        if (!levels.empty()) {
            if ((st = apply_P(W, Z, false))) return st;
            U = Z;
        }
        PKL("axpy", 2.0 * blk, 24.0 * blk, launch_axpy(cs, blk, 1.0, U, Xw), "X update");
        if ((st = residual())) return st;
        for (int i = 0; i < nsys; ++i) {
            if (conv_cycle[i] >= 0) continue;
            if (sys_converged(i)) conv_cycle[i] = cycles;
        }
    }
    for (int i = 0; i < nsys; ++i) KL(launch_unpack(cs, s, A[i].n, Xw + off[i] * s, X[i], A[i].n), "unpack X");
    CU(cudaStreamSynchronize(cs), "sync");
    int h_err = 0;
    if ((st = read_err(ctx, &h_err))) return st;
    bool all = true;
    for (int i = 0; i < nsys; ++i) {
        int worst = 0;
        double wr = -1.0;
        bool conv = true;
        for (int c = 0; c < s; ++c) {
            const size_t k = (size_t)i * s + c;
            const double rn = sqrt(hr[k]);
            const double rel = bnorm[k] > 0 ? rn / bnorm[k] : rn;
            if (rel > wr) { wr = rel; worst = c; }
            if (!(rn <= th[k])) conv = false;
        }
        info[i].iterations = own_it[i];
        info[i].cycles = conv_cycle[i] >= 0 ? conv_cycle[i] : cycles;
        info[i].converged = conv ? 1 : 0;
        info[i].worst_column = worst;
        info[i].max_rel_residual = wr;
        all = all && conv;
    }
    if (!all) return fail(ctx, SPAI_ENOTCONV, "not every system of the batch converged after %d cycles", cycles);
    return SPAI_OK;
}

extern "C" spai_status spai_block_gram(spai_ctx ctx, int32_t s, int32_t n, int32_t nblk, const double *V,
                                       const double *W, double *H, int32_t method)
{
    if (!ctx) return SPAI_EINVAL;
    if (!valid_s(s) || n < 1 || nblk < 1 || !V || !W || !H) return fail(ctx, SPAI_EINVAL, "bad arguments");
    if (!is_device_ptr(V) || !is_device_ptr(W) || !is_device_ptr(H))
        return fail(ctx, SPAI_EINVAL, "V, W and H must be device memory");
    if (method != SPAI_ORTH_FP64 && method != SPAI_ORTH_TENSOR) return fail(ctx, SPAI_EINVAL, "unknown method");
    if (method == SPAI_ORTH_TENSOR && !block_dot_tc_supported(s))
        return fail(ctx, SPAI_EINVAL, "the tensor-core Gram product needs s == 8");
    if (((uintptr_t)V | (uintptr_t)W | (uintptr_t)H) & 15)
        return fail(ctx, SPAI_EINVAL, "V, W and H must be 16-byte aligned");
    const size_t a = (dot_partial_elems(s, nblk) * 8 + 255) / 256 * 256;
    const bool tcm = method == SPAI_ORTH_TENSOR;
    const size_t c = tcm ? (tc_partial_elems(n, nblk) * 8 + 255) / 256 * 256 : 0;
    const size_t fx = tcm ? tc_fixed_sub_bytes(n, nblk) : 0;
    void *ws = nullptr;
    spai_status st = temp_blocks(ctx, (a > c ? a : c) + fx, &ws);
    if (st) return st;
    double *partial = (double *)ws;
    uint64_t *vfix = (uint64_t *)((char *)ws + (a > c ? a : c));
    const double nsd = (double)n * s;
    if (!tcm) {
        PKL("block_dot", 2.0 * nsd * s * nblk, 8.0 * nsd * (nblk + 1),
            launch_block_dot(ctx->stream, s, n, nblk, V, W, partial, H, krylov_chunks(n)), "gram");
    } else {
        PKL("to_fixed", 0.0, 16.0 * nsd * nblk,
            launch_to_fixed(ctx->stream, n, nblk, V, nullptr, vfix, nblk, 0, ctx->d_err), "fixed point");
        PKL("block_dot_tc", 2.0 * nsd * s * nblk, 8.0 * nsd * (nblk + 1),
            launch_block_dot_tc(ctx->stream, n, nblk, vfix, nblk, W, partial, H, ctx->d_err, tc_wait(ctx)), "tensor gram");
    }
    int h = 0;
    if ((st = read_err(ctx, &h))) return st;
    if (h & ERR_TIMEOUT) return fail(ctx, SPAI_ETIMEOUT, "a bounded wait in the tensor-core Gram product gave up");
    if (h & ERR_RANGE) return fail(ctx, SPAI_EINVAL, "a V entry is out of the digit range (|v| >= 2) or W is not finite");
    return SPAI_OK;
}

extern "C" spai_status spai_block_update(spai_ctx ctx, int32_t s, int32_t n, int32_t nblk, const double *V,
                                         const double *H, double *W, double sign, int32_t method)
{
    if (!ctx) return SPAI_EINVAL;
    if (!valid_s(s) || n < 1 || nblk < 1 || !V || !W || !H) return fail(ctx, SPAI_EINVAL, "bad arguments");
    if (!is_device_ptr(V) || !is_device_ptr(W) || !is_device_ptr(H))
        return fail(ctx, SPAI_EINVAL, "V, W and H must be device memory");
    if (method != SPAI_ORTH_FP64 && method != SPAI_ORTH_TENSOR) return fail(ctx, SPAI_EINVAL, "unknown method");
    if (method == SPAI_ORTH_TENSOR && (!block_dot_tc_supported(s) || nblk > block_update_tc_max_blocks()))
        return fail(ctx, SPAI_EINVAL, "the tensor-core block update needs s == 8 and at most %d blocks",
                    block_update_tc_max_blocks());
    if (((uintptr_t)V | (uintptr_t)W | (uintptr_t)H) & 15)
        return fail(ctx, SPAI_EINVAL, "V, W and H must be 16-byte aligned");
    if (method == SPAI_ORTH_FP64) {
        const double nsd = (double)n * s;
        PKL("block_update", 2.0 * nsd * s * nblk, 8.0 * nsd * (nblk + 2),
            launch_block_update(ctx->stream, s, n, nblk, V, H, W, W, sign), "block update");
    } else {
        const size_t hd = (tc_hdig_bytes(nblk) + 255) / 256 * 256;
        void *ws = nullptr;
        spai_status st = temp_blocks(ctx, hd + 256 + (size_t)nblk * n * s * 8, &ws);
        if (st) return st;
        void *hdig = ws;
        int32_t *hexp = (int32_t *)((char *)ws + hd);
        uint64_t *vfix = (uint64_t *)((char *)ws + hd + 256);
        const double nsd = (double)n * s;
        PKL("to_fixed", 0.0, 16.0 * nsd * nblk,
            launch_to_fixed(ctx->stream, n, nblk, V, vfix, nullptr, 0, 0, ctx->d_err), "fixed point");
        PKL("block_update_tc", 2.0 * nsd * s * nblk, 8.0 * nsd * (nblk + 2),
            launch_block_update_tc(ctx->stream, n, nblk, vfix, H, hdig, hexp, W, W, sign, ctx->d_err, tc_wait(ctx)),
            "tensor block update");
    }
    int h = 0;
    spai_status st = read_err(ctx, &h);
    if (st) return st;
    if (h & ERR_TIMEOUT) return fail(ctx, SPAI_ETIMEOUT, "a bounded wait in the tensor-core block update gave up");
    if (h & ERR_RANGE) return fail(ctx, SPAI_EINVAL, "a V entry is out of the digit range (|v| >= 2)");
    return SPAI_OK;
}

// ===================================================================================
// Preconditioner apply that allocates nothing.
//
// For callers that cannot allocate device memory at the point where they apply the
// preconditioner: an outside Krylov solver whose inner loop must not stall the device
// (cudaMalloc / cudaFree may synchronise), or a process whose device memory is already
// reserved by another allocator, so that a new allocation would fail.  The row-major
// staging blocks live in one file-scope device array of fixed size, allocated when the
// library's module is loaded on a device and held by every device that loads it until
// the process exits.  The first call on each device looks the array's address up (with
// that device current) and caches it; make that first call before any stream capture.
// Every call shares the array, so calls that overlap on the GPU (two streams, two host
// threads) race; the staging blocks are fully overwritten by each call, nothing in them
// needs to start at zero.
// ===================================================================================
namespace {

constexpr size_t kNoAllocDoubles = (size_t)1 << 23;  // 64 MiB: four n x s blocks, n * s <= 2^21
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

double *g_noalloc_addr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mutex;

}  // namespace

extern "C" spai_status spai_pc_apply_noalloc(spai_ctx ctx, spai_pc pc, int32_t s, const double *X, int64_t ldx,
                                             double *Y, int64_t ldy)
{
    if (!ctx || !pc) return fail(ctx, SPAI_EINVAL, "NULL argument");
    if (!valid_s(s)) return fail(ctx, SPAI_EINVAL, "s must be 1, 2, 4, 8 or 16");
    const int32_t n = pc->sym->n;
    if (n == 0) return SPAI_OK;
    if (ldx < n || ldy < n || !X || !Y) return fail(ctx, SPAI_EINVAL, "bad block arguments");
    if (!is_device_ptr(X) || !is_device_ptr(Y)) return fail(ctx, SPAI_EINVAL, "X and Y must be device memory");
    {
        // on the context's own device: a peer pointer would reach the kernels unchecked
        cudaPointerAttributes ax, ay;
        if (cudaPointerGetAttributes(&ax, X) != cudaSuccess || cudaPointerGetAttributes(&ay, Y) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, SPAI_EINVAL, "X, Y: pointer attributes unavailable");
        }
        if (ax.device != ctx->device || ay.device != ctx->device)
            return fail(ctx, SPAI_EINVAL, "X and Y must be memory of the context's device %d (got %d, %d)", ctx->device,
                        ax.device, ay.device);
    }
    const size_t blk = (size_t)n * s;
    if (4 * blk > kNoAllocDoubles)
        return fail(ctx, SPAI_EINVAL, "n * s = %zu exceeds the no-allocation apply limit of %zu", blk,
                    kNoAllocDoubles / 4);
    int dev = -1;
    CU(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != ctx->device || dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(ctx, SPAI_EINVAL, "current device %d is not the context's device %d", dev, ctx->device);
    double *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return cuda_fail(ctx, e, "cudaGetSymbolAddress(no-allocation scratch)");
            g_noalloc_addr[dev] = (double *)p;
        }
        base = g_noalloc_addr[dev];
    }
    double *xr = base, *yr = base + blk, *t0 = yr + blk, *t1 = t0 + blk;
    KL(launch_pack(ctx->stream, s, n, X, ldx, xr), "pack");
    // factors from the root build to pc, as in the allocating apply, on the fixed staging
    // blocks; the chain is walked through parent pointers (no container)
    int len = 0;
    for (spai_pc p = pc; p; p = p->parent) ++len;
    const double *cur = xr;
    double *bufs[2] = {t0, t1};
    for (int i = len - 1; i >= 0; --i) {
        spai_pc h = pc;
        for (int hop = 0; hop < i; ++hop) h = h->parent;
        double *dst = (i == 0) ? yr : bufs[(len - 1 - i) & 1];
        if (h->diag)
            KL(launch_scale_rows(ctx->stream, s, n, h->fval, h->fval32, h->fval16, cur, dst), "diagonal factor apply");
        else if (h->fval16)
            KL(launch_spmm_bf16v(ctx->stream, s, n, h->sym->p_rowptr, h->sym->p_colind, h->fval16, cur, dst),
               "preconditioner apply");
        else if (h->fval32)
            KL(launch_spmm_f32v(ctx->stream, s, n, h->sym->p_rowptr, h->sym->p_colind, h->fval32, cur, dst),
               "preconditioner apply");
        else
            KL(launch_spmm(ctx->stream, s, n, h->sym->p_rowptr, h->sym->p_colind, h->fval, cur, dst),
               "preconditioner apply");
        cur = dst;
    }
    KL(launch_unpack(ctx->stream, s, n, yr, Y, ldy), "unpack");
    return SPAI_OK;
}

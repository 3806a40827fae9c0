// Request server of libspai_gb300 (the "Serving" part of include/spai_gb300.h).
//
// The paper's sequences of systems A(p_j) X_j = B_j (Sec. 1.3) are served as requests:
// the SPAI preconditioner of a request is a cached build, an update of a cached build
// (first approach of Table 1, Sec. 2.3-2.4) or a new build, and the request is solved
// by block GMRES (Sec. 2.1).  This file is host code only: it schedules requests onto
// slots (host threads, each with its own stream and library context) and calls the
// library's own entry points; every arithmetic step runs in their kernels.
//
// Scheduling.  An idle slot takes the first queued request whose route is ready (a
// request routed to a build still in progress on another slot is passed over until the
// build is cached).  Its device memory -- growth of the slot's workspace and buffers
// plus the factor it will create -- must fit the budget next to the systems, the cached
// builds and the other slots; if it does not, idle slots' workspaces are released
// (largest first; they are cheap to allocate again), then least recently used idle
// builds evicted (each costs a build to get back); if it still does not fit the slot
// waits for a running request to finish (a request that cannot fit even on an empty
// server fails with SPAI_ENOMEM).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "spai_gb300.h"

namespace {

using Clock = std::chrono::steady_clock;

size_t round256(size_t b) { return ((b ? b : 16) + 255) / 256 * 256; }

// systems per server: their pointer array is reserved once, so workers can read it
// without the lock while add_system appends
constexpr size_t kMaxSystems = 1024;

constexpr int32_t kPrecBits = SPAI_PREC_FP32 | SPAI_PREC_BF16;
constexpr int32_t kKindFlags = kPrecBits | SPAI_LS_NORMAL;  // bits of pattern_kind beside the pattern

struct System {
    spai_affine aff = nullptr;
    int32_t n = 0, nnz = 0, nterms = 0, max_row = 0;
    const int32_t *rowptr = nullptr, *colind = nullptr;
    size_t bytes = 0;        // device bytes of the affine handle
    size_t build_bytes = 0;  // measured bytes of one build with its analysis (0: none yet)
    bool shifted = false;    // terms (M, K_0, K_1): requests may leave the coefficients to the server
    double alpha = 0.0, beta = 0.0;  // its Rayleigh damping D = alpha M + beta K(p)
};

struct Entry {  // a cached SPAI build
    int32_t system = 0;
    double s = 0.0, p = 0.0;
    spai_pc pc = nullptr;
    bool ready = false;
    int refs = 0;       // in-flight requests using it (the building one included)
    size_t bytes = 0;   // estimate while building, measured once cached
    uint64_t last_use = 0;
};

struct Req {
    spai_request r{};
    std::vector<double> coef;
    int64_t ticket = 0;
    bool done = false;
    bool waited = false;  // counted once in waits_for_memory
    spai_result res{};
};

struct Slot {
    std::thread th;
    cudaStream_t stream = nullptr;
    spai_ctx ctx = nullptr;
    double *A = nullptr, *X = nullptr;  // assembled values, solution block
    size_t A_alloc = 0, X_alloc = 0;    // their allocated bytes
    size_t A_cap = 0, X_cap = 0;        // their accounted bytes (raised at admission)
    size_t ws_cap = 0;                  // bytes of the context's solve workspace (tracked)
    bool busy = false;
};

struct Job {
    Req *q = nullptr;
    int route = SPAI_ROUTE_BUILD;
    Entry *e = nullptr;       // cache entry used (or being built), null for an uncached build
    size_t reserve = 0;       // transient factor bytes reserved for the request
};

}  // namespace

struct spai_server_s {
    spai_server_opts o{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;   // queue, completion and cache changes
    bool stop = false;
    spai_ctx main_ctx = nullptr;  // owns the systems' affine handles
    cudaStream_t main_stream = nullptr;
    std::vector<System *> systems;  // stable addresses: workers read them without the lock
    std::vector<Entry *> cache;
    std::vector<Slot> slots;
    std::deque<Req *> queue;
    std::unordered_map<int64_t, Req *> reqs;
    int64_t next_ticket = 1;
    uint64_t use_clock = 0;
    size_t reserved = 0;  // transient reservations of in-flight requests
    spai_server_stats st{};
    std::string err;
};

namespace {

double now_s(const spai_server_s *S)
{
    return std::chrono::duration<double>(Clock::now() - S->t0).count();
}

void set_err(spai_server_s *S, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    S->err = buf;
}

// bytes accounted now: systems, cached builds, slot buffers and workspaces, reservations
size_t mem_now(const spai_server_s *S)
{
    size_t m = S->reserved;
    for (const System *y : S->systems) m += y->bytes;
    for (const Entry *e : S->cache) m += e->bytes;
    for (const auto &sl : S->slots) m += sl.ws_cap + sl.A_cap + sl.X_cap;
    return m;
}

void note_mem(spai_server_s *S)
{
    const size_t m = mem_now(S);
    S->st.mem_in_use = m;
    if (m > S->st.mem_peak) S->st.mem_peak = m;
}

// Device bytes of a build of system y with its analysis (pattern of A or of A^2), before
// one has been measured: index sets bounded through the longest row.
size_t build_estimate(const spai_server_s *S, const System &y)
{
    if (y.build_bytes) return y.build_bytes;
    const size_t n1 = (size_t)y.n + 1, nz = (size_t)y.nnz, mr = (size_t)(y.max_row > 0 ? y.max_row : 1);
    const bool a2 = (S->o.pattern_kind & ~kKindFlags) == SPAI_PATTERN_A2;
    const size_t nzP = a2 ? nz * mr : nz;
    size_t b = 3 * round256(n1 * 4) + 3 * round256(nz * 4) + round256(nzP * mr * 4);
    if (a2) b += 2 * round256(n1 * 4) + 3 * round256(nzP * 4);
    b += round256(nzP * 8) + round256(nz * 8) + round256((size_t)y.n * 4);
    return b;
}

// transient allocations of one pattern analysis (transposition and scan buffers)
size_t analysis_transient(const System &y) { return 16 * (size_t)y.nnz + 16 * ((size_t)y.n + 1) + (1u << 20); }

size_t update_estimate(const spai_server_s *S, const System &y)
{
    const bool a2 = (S->o.pattern_kind & ~kKindFlags) == SPAI_PATTERN_A2;
    const int32_t prec = S->o.pattern_kind & kPrecBits;
    const size_t nzP = a2 ? (size_t)y.nnz * (size_t)(y.max_row > 0 ? y.max_row : 1) : (size_t)y.nnz;
    const size_t vb = prec == SPAI_PREC_BF16 ? 2 : prec == SPAI_PREC_FP32 ? 4 : 8;
    return round256(nzP * vb) + round256((size_t)y.nnz * 8) + round256((size_t)y.n * 4);
}

// nearest cached build for (system, s) within the radius (ready or in progress)
Entry *find_entry(spai_server_s *S, const spai_request &r)
{
    if (!S->o.reuse) return nullptr;
    Entry *best = nullptr;
    double bd = 0.0;
    for (Entry *e : S->cache) {
        if (e->system != r.system || e->s != r.s) continue;
        const double d = std::fabs(e->p - r.p);
        if (d > S->o.radius) continue;
        if (!best || d < bd) { best = e; bd = d; }
    }
    return best;
}

void destroy_entry(spai_server_s *S, Entry *e)
{
    if (e->pc) spai_pc_destroy(e->pc);
    for (size_t i = 0; i < S->cache.size(); ++i)
        if (S->cache[i] == e) { S->cache.erase(S->cache.begin() + (ptrdiff_t)i); break; }
    delete e;
}

// evict least recently used idle builds (never `keep`) until `need` more bytes fit
bool make_room(spai_server_s *S, size_t need, const Entry *keep, int slot)
{
    const size_t budget = S->o.mem_budget;
    if (!budget) return true;
    // first the idle slots' workspaces and buffers (not this slot's: it is about to use
    // them), largest first -- they are allocated again on demand -- then cached builds,
    // least recently used first, which cost a build to get back
    while (mem_now(S) + need > budget) {
        int big = -1;
        size_t big_b = 0;
        for (int k = 0; k < (int)S->slots.size(); ++k) {
            const Slot &sl = S->slots[k];
            const size_t b = sl.ws_cap + sl.A_cap + sl.X_cap;
            if (k != slot && !sl.busy && b > big_b) { big = k; big_b = b; }
        }
        if (big < 0) break;
        Slot &sl = S->slots[big];
        if (sl.ws_cap) { spai_ctx_trim(sl.ctx); sl.ws_cap = 0; }
        if (sl.A) { cudaFreeAsync(sl.A, sl.stream); sl.A = nullptr; }
        if (sl.X) { cudaFreeAsync(sl.X, sl.stream); sl.X = nullptr; }
        sl.A_alloc = sl.A_cap = sl.X_alloc = sl.X_cap = 0;
    }
    while (mem_now(S) + need > budget) {
        Entry *lru = nullptr;
        for (Entry *e : S->cache)
            if (e != keep && e->ready && e->refs == 0 && (!lru || e->last_use < lru->last_use)) lru = e;
        if (!lru) break;
        destroy_entry(S, lru);
        S->st.evictions++;
    }
    return mem_now(S) + need <= budget;
}

bool any_busy(const spai_server_s *S)
{
    for (const auto &sl : S->slots)
        if (sl.busy) return true;
    return false;
}

void complete(spai_server_s *S, Req *q, int status)
{
    q->res.status = status;
    q->res.t_done = now_s(S);
    q->done = true;
    S->st.completed++;
    if (status != SPAI_OK) S->st.failed++;
}

enum Take { TOOK, NOTHING, RETRY };

// Pick work for slot k (mutex held).  NOTHING: nothing can start now; RETRY: the queue
// changed (a request failed at admission), look again.
Take take(spai_server_s *S, int k, Job *job)
{
    Slot &sl = S->slots[k];
    for (size_t qi = 0; qi < S->queue.size(); ++qi) {
        Req *q = S->queue[qi];
        const System &y = *S->systems[q->r.system];
        Entry *e = find_entry(S, q->r);
        if (e && !e->ready) continue;  // its base is being built on another slot
        int route = SPAI_ROUTE_BUILD;
        size_t factor = 0;
        if (e) {
            route = (e->p == q->r.p) ? SPAI_ROUTE_REUSE : SPAI_ROUTE_UPDATE;
            factor = route == SPAI_ROUTE_UPDATE ? update_estimate(S, y) : 0;
        } else {
            factor = build_estimate(S, y) + analysis_transient(y);
        }
        // the mixed-precision solve adds A's values in FP32 to the workspace
        const size_t ws = spai_solve_workspace_size(y.n, q->r.nrhs, S->o.restart) +
                          (S->o.precision == SPAI_SOLVE_MIXED ? ((size_t)y.nnz * 4 + 255) / 256 * 256 : 0);
        const size_t a_need = round256((size_t)y.nnz * 8), x_need = round256((size_t)y.n * q->r.nrhs * 8);
        // a growing buffer is freed before it is allocated again: only the difference counts
        auto grow = [](size_t want, size_t cap) { return want > cap ? want - cap : 0; };
        const size_t need = grow(ws, sl.ws_cap) + grow(a_need, sl.A_cap) + grow(x_need, sl.X_cap) + factor;
        if (!make_room(S, need, e, k)) {
            if (!any_busy(S) && mem_now(S) + need > S->o.mem_budget) {
                // cannot fit even with every other slot idle and the cache emptied
                S->queue.erase(S->queue.begin() + (ptrdiff_t)qi);
                set_err(S, "request %lld needs %zu more device bytes than the budget allows",
                        (long long)q->ticket, need);
                complete(S, q, SPAI_ENOMEM);
                S->cv.notify_all();
                return RETRY;
            }
            if (!q->waited) {
                q->waited = true;
                S->st.waits_for_memory++;
            }
            return NOTHING;  // the first routable request waits for memory (FIFO among routable requests)
        }
        S->queue.erase(S->queue.begin() + (ptrdiff_t)qi);
        if (route == SPAI_ROUTE_BUILD && S->o.reuse) {
            e = new Entry();
            e->system = q->r.system;
            e->s = q->r.s;
            e->p = q->r.p;
            e->bytes = build_estimate(S, y);
            S->cache.push_back(e);
            factor -= e->bytes;  // the entry itself accounts for the build
        }
        if (e) {
            e->refs++;
            e->last_use = ++S->use_clock;
        }
        // the slot's buffers at their new sizes (reallocated by the worker)
        if (ws > sl.ws_cap) sl.ws_cap = ws;
        if (a_need > sl.A_cap) sl.A_cap = a_need;
        if (x_need > sl.X_cap) sl.X_cap = x_need;
        S->reserved += factor;
        sl.busy = true;
        job->q = q;
        job->route = route;
        job->e = e;
        job->reserve = factor;
        note_mem(S);
        return TOOK;
    }
    return NOTHING;
}

// grow-only device buffer on the slot's stream
int ensure(Slot &sl, double **buf, size_t *have, size_t need)
{
    if (*buf && *have >= need) return 0;
    if (*buf) cudaFreeAsync(*buf, sl.stream);
    *buf = nullptr;
    void *p = nullptr;
    if (cudaMallocAsync(&p, need, sl.stream) != cudaSuccess) {
        cudaGetLastError();
        *have = 0;
        return -1;
    }
    *buf = (double *)p;
    *have = need;
    return 0;
}

// Run one admitted request on slot k (mutex not held).  Returns its status; *built is
// the new build (route BUILD) to be cached or destroyed by the caller.
int run(spai_server_s *S, int k, const Job &job, spai_pc *built, std::string *msg)
{
    Slot &sl = S->slots[k];
    Req *q = job.q;
    const System &y = *S->systems[q->r.system];
    const int32_t n = y.n, s = q->r.nrhs;
    *built = nullptr;
    // the buffers at the sizes accounted at admission
    if (ensure(sl, &sl.A, &sl.A_alloc, sl.A_cap) || ensure(sl, &sl.X, &sl.X_alloc, sl.X_cap)) {
        *msg = "device allocation of the slot's buffers failed";
        return SPAI_ENOMEM;
    }
    spai_ctx ctx = sl.ctx;
    int st = spai_assemble(ctx, y.aff, q->coef.data(), sl.A);
    if (st) { *msg = spai_last_error(ctx); return st; }
    spai_csr A{n, y.nnz, y.rowptr, y.colind, sl.A};
    spai_pc pc = nullptr, own = nullptr;
    const int32_t prec = S->o.pattern_kind & kPrecBits;
    if (job.route == SPAI_ROUTE_BUILD) {
        st = spai_build(ctx, &A, S->o.pattern_kind, &own);
        if (st) {
            *msg = spai_last_error(ctx);
            if (own) spai_pc_destroy(own);
            return st;
        }
        pc = own;
        *built = own;  // the caller caches or destroys it, whatever happens to the solve
    } else if (job.route == SPAI_ROUTE_UPDATE) {
        st = spai_update(ctx, job.e->pc, &A, SPAI_UPDATE_FIRST | prec | (S->o.pattern_kind & SPAI_LS_NORMAL), &own);
        if (st) {
            *msg = spai_last_error(ctx);
            if (own) spai_pc_destroy(own);
            return st;
        }
        pc = own;
    } else {
        pc = job.e->pc;
    }
    q->res.base_p = job.e ? job.e->p : q->r.p;
    cudaError_t ce = cudaMemsetAsync(sl.X, 0, (size_t)n * s * 8, sl.stream);
    if (ce != cudaSuccess) {
        *msg = cudaGetErrorString(ce);
        st = SPAI_ECUDA;
    }
    spai_solve_opts so{S->o.restart, S->o.max_cycles, S->o.tol, S->o.orth, S->o.precision};
    spai_solve_info info{};
    if (!st) {
        st = block_solve(ctx, &A, pc, s, q->r.B, n, sl.X, n, &so, &info, nullptr);
        if (st) *msg = spai_last_error(ctx);
    }
    q->res.iterations = info.iterations;
    q->res.max_rel_residual = info.max_rel_residual;
    if (!st && q->r.X) {
        ce = cudaMemcpyAsync(q->r.X, sl.X, (size_t)n * s * 8, cudaMemcpyDefault, sl.stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(sl.stream);
        if (ce != cudaSuccess) {
            *msg = cudaGetErrorString(ce);
            st = SPAI_ECUDA;
        }
    }
    if (job.route == SPAI_ROUTE_UPDATE) spai_pc_destroy(own);
    return st;
}

void worker(spai_server_s *S, int k)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        Job job;
        Take t;
        while ((t = take(S, k, &job)) != TOOK) {
            if (t == RETRY) continue;
            if (S->stop && S->queue.empty()) return;
            S->cv.wait(lk);
        }
        Slot &sl = S->slots[k];
        job.q->res.t_start = now_s(S);
        job.q->res.slot = k;
        job.q->res.route = job.route;
        lk.unlock();
        spai_pc built = nullptr;
        std::string msg;
        const int st = run(S, k, job, &built, &msg);
        lk.lock();
        S->reserved -= job.reserve;
        if (job.route == SPAI_ROUTE_BUILD) {
            S->st.builds++;
            System &y = *S->systems[job.q->r.system];
            if (built) {
                const size_t measured = spai_pc_mem_size(built, 1);
                y.build_bytes = measured;
                if (job.e) {
                    job.e->pc = built;
                    job.e->bytes = measured;
                    job.e->ready = true;
                } else {
                    spai_pc_destroy(built);
                }
            }
            if (job.e && !job.e->ready) {
                job.e->refs--;
                destroy_entry(S, job.e);  // failed build: requests routed to it build their own
                job.e = nullptr;
            }
        } else if (job.route == SPAI_ROUTE_UPDATE) {
            S->st.updates++;
        } else {
            S->st.reuses++;
        }
        if (job.e) {
            job.e->refs--;
            job.e->last_use = ++S->use_clock;
        }
        if (st) set_err(S, "request %lld: %s", (long long)job.q->ticket, msg.c_str());
        sl.busy = false;
        complete(S, job.q, st);
        note_mem(S);
        S->cv.notify_all();
    }
}

}  // namespace

extern "C" spai_status spai_server_create(const spai_server_opts *opts, spai_server *out)
{
    if (!opts || !out) return SPAI_EINVAL;
    *out = nullptr;
    const int32_t kind = opts->pattern_kind & ~kKindFlags;
    if (opts->slots < 1 || opts->slots > 64 || opts->restart < 1 || opts->max_cycles < 1 || !(opts->tol >= 0.0) ||
        !(opts->radius >= 0.0) || (kind != SPAI_PATTERN_A && kind != SPAI_PATTERN_A2) ||
        (opts->pattern_kind & ~(kKindFlags | 1)) || (opts->pattern_kind & kPrecBits) == kPrecBits ||
        opts->orth < SPAI_ORTH_AUTO || opts->orth > SPAI_ORTH_TENSOR ||
        (opts->precision != SPAI_SOLVE_FP64 && opts->precision != SPAI_SOLVE_MIXED) || opts->reserved != 0)
        return SPAI_EINVAL;
    spai_server_s *S = new spai_server_s();
    S->o = *opts;
    S->t0 = Clock::now();
    S->systems.reserve(kMaxSystems);
    if (cudaGetDevice(&S->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->main_stream, cudaStreamNonBlocking) != cudaSuccess ||
        spai_ctx_create(&S->main_ctx, S->main_stream, 0) != SPAI_OK) {
        cudaGetLastError();
        if (S->main_stream) cudaStreamDestroy(S->main_stream);
        delete S;
        return SPAI_ECUDA;
    }
    S->slots.resize(opts->slots);
    for (auto &sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            spai_ctx_create(&sl.ctx, sl.stream, 0) != SPAI_OK) {
            cudaGetLastError();
            for (auto &t : S->slots) {
                if (t.ctx) spai_ctx_destroy(t.ctx);
                if (t.stream) cudaStreamDestroy(t.stream);
            }
            spai_ctx_destroy(S->main_ctx);
            cudaStreamDestroy(S->main_stream);
            delete S;
            return SPAI_ECUDA;
        }
    }
    for (int k = 0; k < opts->slots; ++k) S->slots[k].th = std::thread(worker, S, k);
    *out = S;
    return SPAI_OK;
}

namespace {

spai_status add_system(spai_server S, int32_t nterms, const spai_csr *terms, int32_t *id, const System &proto)
{
    if (!S || !terms || !id) return SPAI_EINVAL;
    System y = proto;
    spai_status st = spai_affine_create(S->main_ctx, nterms, terms, &y.aff);
    if (st) {
        std::lock_guard<std::mutex> lk(S->mu);
        set_err(S, "add_system: %s", spai_last_error(S->main_ctx));
        return st;
    }
    int32_t n = 0, nnz = 0;
    spai_affine_pattern(y.aff, &n, &nnz, &y.rowptr, &y.colind);
    y.n = n;
    y.nnz = nnz;
    y.nterms = nterms;
    // longest row of the union pattern (for the first memory estimate of a build)
    std::vector<int32_t> rp((size_t)n + 1);
    if (cudaMemcpy(rp.data(), y.rowptr, rp.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        spai_affine_destroy(y.aff);
        return SPAI_ECUDA;
    }
    for (int32_t i = 0; i < n; ++i) y.max_row = std::max(y.max_row, rp[i + 1] - rp[i]);
    y.bytes = round256(((size_t)n + 1) * 4) + round256((size_t)nnz * 4) + round256((size_t)nterms * nnz * 8);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->systems.size() >= kMaxSystems) {
        spai_affine_destroy(y.aff);
        set_err(S, "add_system: at most %zu systems per server", kMaxSystems);
        return SPAI_EINVAL;
    }
    if (S->o.mem_budget && mem_now(S) + y.bytes > S->o.mem_budget && !make_room(S, y.bytes, nullptr, -1)) {
        spai_affine_destroy(y.aff);
        set_err(S, "add_system: %zu bytes exceed the memory budget", y.bytes);
        return SPAI_ENOMEM;
    }
    *id = (int32_t)S->systems.size();
    S->systems.push_back(new System(y));
    note_mem(S);
    return SPAI_OK;
}

}  // namespace

extern "C" spai_status spai_server_add_system(spai_server S, int32_t nterms, const spai_csr *terms, int32_t *id)
{
    return add_system(S, nterms, terms, id, System{});
}

extern "C" spai_status spai_server_add_shifted_system(spai_server S, const spai_csr *terms, double alpha, double beta,
                                                      int32_t *id)
{
    if (!S) return SPAI_EINVAL;
    if (!std::isfinite(alpha) || !std::isfinite(beta)) {
        std::lock_guard<std::mutex> lk(S->mu);
        set_err(S, "add_shifted_system: damping coefficients must be finite");
        return SPAI_EINVAL;
    }
    System proto;
    proto.shifted = true;
    proto.alpha = alpha;
    proto.beta = beta;
    return add_system(S, 3, terms, id, proto);
}

extern "C" spai_status spai_server_submit(spai_server S, const spai_request *req, int64_t *ticket)
{
    if (!S || !req || !ticket) return SPAI_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (req->system < 0 || req->system >= (int32_t)S->systems.size()) {
        set_err(S, "submit: unknown system %d", req->system);
        return SPAI_EINVAL;
    }
    const int32_t s = req->nrhs;
    const System &ys = *S->systems[req->system];
    if (!(s == 1 || s == 2 || s == 4 || s == 8 || s == 16) || (!req->coef && !ys.shifted) || !req->B ||
        !std::isfinite(req->p) || !std::isfinite(req->s)) {
        set_err(S, "submit: bad request (nrhs must be 1, 2, 4, 8 or 16; B non-NULL, and coef too unless the "
                   "system is a shifted one; p, s finite)");
        return SPAI_EINVAL;
    }
    if (S->stop) {
        set_err(S, "submit: server is shutting down");
        return SPAI_EINVAL;
    }
    Req *q = new Req();
    q->r = *req;
    const System &y = ys;
    if (req->coef) {
        q->coef.assign(req->coef, req->coef + y.nterms);
    } else {  // A(p, s) of the shifted second-order system
        q->coef.assign(3, 0.0);
        spai_shifted_coefficients(1, &req->p, req->s, y.alpha, y.beta, q->coef.data());
    }
    q->r.coef = q->coef.data();
    q->ticket = S->next_ticket++;
    q->res.t_arrival = req->t_arrival >= 0.0 ? req->t_arrival : now_s(S);
    S->reqs[q->ticket] = q;
    S->queue.push_back(q);
    S->st.submitted++;
    *ticket = q->ticket;
    S->cv.notify_all();
    return SPAI_OK;
}

extern "C" spai_status spai_server_wait(spai_server S, int64_t ticket, spai_result *out)
{
    if (!S) return SPAI_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
        set_err(S, "wait: unknown ticket %lld", (long long)ticket);
        return SPAI_EINVAL;
    }
    Req *q = it->second;
    S->cv.wait(lk, [&] { return q->done; });
    if (out) *out = q->res;
    S->reqs.erase(ticket);
    delete q;
    return SPAI_OK;
}

extern "C" double spai_server_clock(spai_server S) { return S ? now_s(S) : 0.0; }

extern "C" spai_status spai_server_stats_get(spai_server S, spai_server_stats *out)
{
    if (!S || !out) return SPAI_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    note_mem(S);
    *out = S->st;
    out->cached_builds = (int32_t)S->cache.size();
    return SPAI_OK;
}

extern "C" const char *spai_server_last_error(spai_server S) { return S ? S->err.c_str() : "NULL server"; }

extern "C" spai_status spai_server_destroy(spai_server S)
{
    if (!S) return SPAI_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    for (auto &sl : S->slots)
        if (sl.th.joinable()) sl.th.join();
    cudaSetDevice(S->device);
    while (!S->cache.empty()) destroy_entry(S, S->cache.back());
    for (auto &sl : S->slots) {
        if (sl.A) cudaFreeAsync(sl.A, sl.stream);
        if (sl.X) cudaFreeAsync(sl.X, sl.stream);
        cudaStreamSynchronize(sl.stream);
        spai_ctx_destroy(sl.ctx);
        cudaStreamDestroy(sl.stream);
    }
    for (System *y : S->systems) {
        spai_affine_destroy(y->aff);
        delete y;
    }
    spai_ctx_destroy(S->main_ctx);
    cudaStreamDestroy(S->main_stream);
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
    return SPAI_OK;
}

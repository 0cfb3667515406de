// Request server: many ChASE solves of different sizes in flight on one GPU.
//
// The paper's BSE workflow solves sequences of related eigenproblems (the
// convergence tests over k-point meshes and energy cutoffs, Sec. 2 and
// Sec. 4; ChASE targets such sequences, Sec. 3).  The server runs such a
// stream of requests:
//   - a FIFO queue with admission by an HBM budget: a request starts when a
//     slot is free and its memory estimate (H, the tensor-core slices of H,
//     the search-space blocks, the eigenvectors it keeps) fits beside what
//     the running requests and the resident eigenvectors hold; requests
//     behind a head that does not fit may start first (no slot idles while
//     memory is available); an estimate above the whole budget is refused;
//   - continuous batching: every slot is a host worker with its own CUDA
//     stream and solver context, so requests admitted while others run
//     execute concurrently on the device; the tensor-core products that the
//     running solves submit at about the same time run in one launch of the
//     persistent product kernel (the product batcher of ozaki.cu), each with
//     the same units and arithmetic as alone, so results are identical alone
//     and in a mix;
//   - resident results: a finished request keeps its eigenvectors on the
//     device (counted in the budget, evicted least-recently-used) so that a
//     later request can warm-start from them (chase_request.warm_ticket);
//   - latency stamps: submit, start and end times on a steady clock.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "context.h"

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Req {
    uint64_t ticket = 0;
    chase_request rq{};
    int64_t N = 0;
    size_t run_bytes = 0;      // admission estimate while running
    size_t keep_bytes = 0;     // eigenvectors kept after the solve
    int state = 0;             // 0 queued, 1 running, 2 done
    int status = BSE_EBUSY;
    double t_submit = 0, t_start = 0, t_end = 0;
    std::vector<double> evals, resid;
    chase_stats stats{};
    void *d_evecs = nullptr;   // resident N x nev eigenvectors (ld = N)
    int pins = 0;              // queued/running warm starts that read d_evecs
    uint64_t pinned = 0;       // ticket this request pinned for its warm start
    bool cancelled = false;
    std::string err;
};

}  // namespace

struct BseServer {
    bsechase_ctx *owner = nullptr;
    size_t budget = 0, held = 0;    // bytes admitted (running + resident)
    std::vector<bsechase_ctx *> slots;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> queue;
    std::map<uint64_t, std::shared_ptr<Req>> reqs;
    std::list<uint64_t> lru;        // finished requests holding eigenvectors, oldest first
    uint64_t next_ticket = 1;
    bool stop = false;
    OzBatcher *batcher = nullptr;   // products of the slots' solves in shared launches
    int running = 0;                // solves in progress
};

namespace {

size_t estimate_run_bytes(int64_t N, int m, int nev, int precision, bool own_h, bool half) {
    const size_t Np = (size_t)ozaki_padded(N);
    const size_t mp = (size_t)((std::max(m, 32) + 31) / 32 * 32);
    size_t b = own_h ? 16 * (size_t)N * N : 0;              // H, unless the caller's
    b += 4 * 16 * (size_t)N * m;                            // V and three scratch blocks
    b += 16 * (size_t)N * nev;                              // eigenvectors
    b += (size_t)N * 8 * 3 * 16 + ((size_t)20 << 20);       // Lanczos blocks, small matrices
    if (precision != CHASE_FP64_DFMA) {
        b += half ? ozaki_a_bytes_tri(N) + 16 * Np          // slices of H (half storage:
                  : 24 * Np * Np;                           // the lower triangle, scales)
        b += 36 * mp * Np;                                  // slices of the operand
        b += ozaki_partial_bytes(N, std::max(m, 32));       // split-K partials
        b += std::max(ozaki_gen_a_bytes(std::max(m, 32), N),  // slices of op(A) in the
                      ozaki_gen_a_bytes(N, std::max(m, 32))); // QR / Rayleigh-Ritz products
    }
    return b;
}

// Free least-recently-used resident eigenvectors until `need` more bytes fit.
// Nothing is freed when even evicting every unpinned block would not make
// room (the request waits, and the warm-start data stays).  Caller holds the
// lock.  Frees go on `st` after the data is no longer read (nothing reads an
// unpinned resident block).
void evict_for(BseServer *S, size_t need, cudaStream_t st) {
    size_t evictable = 0;
    for (uint64_t t : S->lru) {
        auto r = S->reqs.find(t);
        if (r != S->reqs.end() && r->second->d_evecs && r->second->pins == 0)
            evictable += r->second->keep_bytes;
    }
    if (S->held - std::min(evictable, S->held) + need > S->budget) return;
    for (auto it = S->lru.begin(); it != S->lru.end() && S->held + need > S->budget;) {
        auto r = S->reqs.find(*it);
        if (r == S->reqs.end() || !r->second->d_evecs) {
            it = S->lru.erase(it);
            continue;
        }
        Req &q = *r->second;
        if (q.pins > 0) {
            ++it;
            continue;
        }
        cudaFreeAsync(q.d_evecs, st);
        q.d_evecs = nullptr;
        S->held -= q.keep_bytes;
        q.keep_bytes = 0;
        it = S->lru.erase(it);
    }
}

void worker(BseServer *S, int slot) {
    bsechase_ctx *ctx = S->slots[slot];
    cudaSetDevice(ctx->device);
    for (;;) {
        std::shared_ptr<Req> job;
        std::shared_ptr<Req> warm;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop) return;
                for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
                    Req &q = **it;
                    if (S->held + q.run_bytes > S->budget) evict_for(S, q.run_bytes, ctx->st);
                    if (S->held + q.run_bytes <= S->budget) {
                        job = *it;
                        S->queue.erase(it);
                        break;
                    }
                }
                if (job) break;
                S->cv_work.wait(lk);
            }
            S->held += job->run_bytes;
            job->state = 1;
            job->t_start = now_s();
            if (S->batcher) ozb_set_active(S->batcher, ++S->running);
            if (job->rq.warm_ticket) {
                auto w = S->reqs.find(job->rq.warm_ticket);
                if (w != S->reqs.end() && w->second->d_evecs && w->second->N == job->N) warm = w->second;
            }
        }
        // ---- run the request on this slot's stream
        const chase_request &rq = job->rq;
        const int64_t N = job->N;
        void *dH = nullptr, *dZ = nullptr;
        int rc = BSE_OK;
        const bool store_h = !rq.d_H && !rq.h_free;
        if ((store_h && cudaMallocAsync(&dH, 16 * (size_t)N * N, ctx->st) != cudaSuccess) ||
            cudaMallocAsync(&dZ, 16 * (size_t)N * rq.nev, ctx->st) != cudaSuccess) {
            cudaGetLastError();
            rc = BSE_ENOMEM;
        }
        if (rc == BSE_OK && store_h)
            rc = bse_build_hamiltonian(ctx, rq.seed, rq.Nk, rq.Nv, rq.Nc,
                                       rq.use_model ? &rq.model : nullptr, dH, N);
        // h_free: the generator's tables, its elements go straight into the slices
        BseSource src{};
        if (rc == BSE_OK && rq.h_free)
            rc = bse_source(ctx, rq.seed, rq.Nk, rq.Nv, rq.Nc,
                            bse_model_of(rq.use_model ? &rq.model : nullptr), &src);
        const z_t *Hs = rq.d_H ? (const z_t *)rq.d_H : (const z_t *)dH;
        const int64_t lds = rq.d_H ? rq.ldh : N;
        chase_opts o{};
        o.seed = rq.seed;
        o.degree_group = rq.degree_group;
        o.nex_damping = rq.nex_damping;
        o.half_storage = rq.half_storage;
        if (warm) {
            o.d_V0 = warm->d_evecs;
            o.ldv0 = N;
            o.n_v0 = std::min(warm->rq.nev, rq.nev + rq.nex);
        }
        std::vector<double> ev(rq.nev), rs(rq.nev);
        chase_stats st{};
        if (rc == BSE_OK)
            rc = solve_device(ctx, rq.h_free ? nullptr : Hs, N, rq.h_free ? N : lds, rq.nev,
                              rq.nex, rq.tol, rq.deg_max, rq.precision, &o, ev.data(), (z_t *)dZ,
                              N, rs.data(), &st, rq.h_free ? &src : nullptr);
        if (dH) cudaFreeAsync(dH, ctx->st);
        release_workspace(ctx);
        cudaStreamSynchronize(ctx->st);
        const double t_end = now_s();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (job->pinned) {
                auto w = S->reqs.find(job->pinned);
                if (w != S->reqs.end()) w->second->pins--;
            }
            S->held -= job->run_bytes;
            if (S->batcher) ozb_set_active(S->batcher, --S->running);
            job->t_end = t_end;
            job->status = rc;
            job->err = (rc == BSE_OK) ? std::string() : ctx->err;
            job->evals = ev;
            job->resid = rs;
            job->stats = st;
            if ((rc == BSE_OK || rc == BSE_ENOCONV) && dZ && !job->cancelled) {
                job->d_evecs = dZ;
                job->keep_bytes = 16 * (size_t)N * rq.nev;
                S->held += job->keep_bytes;
                S->lru.push_back(job->ticket);
            } else if (dZ) {
                cudaFreeAsync(dZ, ctx->st);
            }
            job->state = 2;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

void fill_result(const Req &q, chase_result *out) {
    memset(out, 0, sizeof *out);
    out->status = q.status;
    out->N = q.N;
    out->nev = q.rq.nev;
    out->evals = q.evals.empty() ? nullptr : q.evals.data();
    out->resid = q.resid.empty() ? nullptr : q.resid.data();
    out->stats = q.stats;
    out->t_submit = q.t_submit;
    out->t_start = q.t_start;
    out->t_end = q.t_end;
    out->has_evecs = q.d_evecs != nullptr;
}

}  // namespace

void bse_server_shutdown(bsechase_ctx *ctx) {
    BseServer *S = ctx ? ctx->server : nullptr;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers)
        if (t.joinable()) t.join();
    ozb_destroy(S->batcher);
    for (auto &kv : S->reqs)
        if (kv.second->d_evecs) cudaFree(kv.second->d_evecs);
    for (bsechase_ctx *c : S->slots) bsechase_destroy(c);
    delete S;
    ctx->server = nullptr;
}

extern "C" {

int chase_server_create(bsechase_ctx *ctx, size_t hbm_budget_bytes, int max_slots) {
    if (!ctx) return BSE_EINVAL;
    if (ctx->server) return fail(ctx, BSE_EINVAL, "a server already runs on this context%s");
    if (max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0)
        return fail(ctx, BSE_EINVAL, "need 1 <= max_slots <= 64 and a positive budget%s");
    BseServer *S = new BseServer();
    S->owner = ctx;
    S->budget = hbm_budget_bytes;
    for (int i = 0; i < max_slots; i++) {
        bsechase_ctx *c = nullptr;
        int rc = bsechase_create(&c, ctx->device, nullptr);
        if (rc != BSE_OK) {
            for (bsechase_ctx *d : S->slots) bsechase_destroy(d);
            delete S;
            return fail(ctx, rc, "cannot create server slot contexts%s");
        }
        S->slots.push_back(c);
    }
    ctx->server = S;
    for (int i = 0; i < max_slots; i++) S->workers.emplace_back(worker, S, i);
    return BSE_OK;
}

int chase_server_submit(bsechase_ctx *ctx, const chase_request *req, uint64_t *ticket) {
    if (!ctx || !req || !ticket) return BSE_EINVAL;
    BseServer *S = ctx->server;
    if (!S) return fail(ctx, BSE_EINVAL, "no server on this context%s");
    const int64_t N = bse_dim(req->Nk, req->Nv, req->Nc);
    const int m = req->nev + req->nex;
    if (N < 1 || req->nev < 1 || req->nex < 0 || m > N || m > 512 || !(req->tol > 0) ||
        req->deg_max < 2 || req->degree_group < 0 || !precision_valid(req->precision) ||
        (req->half_storage != 0 && req->half_storage != 1) || (req->h_free != 0 && req->h_free != 1))
        return fail(ctx, BSE_EINVAL, "invalid request%s");
    if ((req->half_storage || req->h_free) && !precision_uses_tc(precision_mode(req->precision)))
        return fail(ctx, BSE_EINVAL, "half_storage and h_free need a tensor-core precision%s");
    if (req->h_free && req->d_H) return fail(ctx, BSE_EINVAL, "h_free with a caller's H%s");
    if (req->use_model && (req->model.rank_x < 0 || req->model.rank_x > 64))
        return fail(ctx, BSE_EINVAL, "rank_x outside 0..64%s");
    auto q = std::make_shared<Req>();
    q->rq = *req;
    q->rq.precision = precision_mode(req->precision);
    q->N = N;
    if (req->d_H && req->ldh < N) return fail(ctx, BSE_EINVAL, "request H: ldh < N%s");
    q->run_bytes = estimate_run_bytes(N, m, req->nev, q->rq.precision,
                                      req->d_H == nullptr && !req->h_free, req->half_storage == 1);
    if (q->run_bytes > S->budget)
        return fail(ctx, BSE_ENOMEM, "request needs more than the whole HBM budget%s");
    q->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        q->ticket = S->next_ticket++;
        if (req->warm_ticket) {
            auto w = S->reqs.find(req->warm_ticket);
            if (w != S->reqs.end()) {
                w->second->pins++;                        // keep its eigenvectors resident
                q->pinned = req->warm_ticket;
            } else {
                q->rq.warm_ticket = 0;
            }
        }
        S->reqs[q->ticket] = q;
        S->queue.push_back(q);
        *ticket = q->ticket;
    }
    S->cv_work.notify_all();
    return BSE_OK;
}

int chase_server_poll(bsechase_ctx *ctx, uint64_t ticket, chase_result *out) {
    if (!ctx || !out || !ctx->server) return BSE_EINVAL;
    BseServer *S = ctx->server;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(ctx, BSE_EINVAL, "unknown ticket%s");
    if (it->second->state != 2) return BSE_EBUSY;
    fill_result(*it->second, out);
    return BSE_OK;
}

int chase_server_wait(bsechase_ctx *ctx, uint64_t ticket, double timeout_s, chase_result *out) {
    if (!ctx || !out || !ctx->server) return BSE_EINVAL;
    BseServer *S = ctx->server;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(ctx, BSE_EINVAL, "unknown ticket%s");
    std::shared_ptr<Req> q = it->second;
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                              std::chrono::duration<double>(timeout_s < 0 ? 0 : timeout_s));
    while (q->state != 2) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && q->state != 2)
            return BSE_ETIMEOUT;
    }
    fill_result(*q, out);
    return BSE_OK;
}

int chase_server_evecs(bsechase_ctx *ctx, uint64_t ticket, void *d_out, int64_t ld) {
    if (!ctx || !d_out || !ctx->server) return BSE_EINVAL;
    BseServer *S = ctx->server;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(ctx, BSE_EINVAL, "unknown ticket%s");
    Req &q = *it->second;
    if (q.state != 2) return BSE_EBUSY;
    if (!q.d_evecs) return fail(ctx, BSE_EINVAL, "eigenvectors were not kept (evicted or failed)%s");
    if (ld < q.N) return fail(ctx, BSE_EINVAL, "ld < N%s");
    if (cudaMemcpy2DAsync(d_out, ld * 16, q.d_evecs, q.N * 16, q.N * 16, q.rq.nev,
                          cudaMemcpyDefault, ctx->st) != cudaSuccess ||
        cudaStreamSynchronize(ctx->st) != cudaSuccess)
        return fail(ctx, BSE_ECUDA, "copy failed%s");
    // touch: most recently used
    S->lru.remove(ticket);
    S->lru.push_back(ticket);
    return BSE_OK;
}

int chase_server_release(bsechase_ctx *ctx, uint64_t ticket) {
    if (!ctx || !ctx->server) return BSE_EINVAL;
    BseServer *S = ctx->server;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return fail(ctx, BSE_EINVAL, "unknown ticket%s");
        Req &q = *it->second;
        if (q.state == 0) {            // still queued: cancel it
            q.cancelled = true;
            S->queue.erase(std::remove(S->queue.begin(), S->queue.end(), it->second), S->queue.end());
            if (q.pinned) {
                auto w = S->reqs.find(q.pinned);
                if (w != S->reqs.end()) w->second->pins--;
            }
            q.state = 2;
            q.status = BSE_EINVAL;
            q.err = "cancelled";
            S->cv_done.notify_all();
        } else if (q.state == 1) {
            return BSE_EBUSY;
        } else {
            if (q.pins > 0) return BSE_EBUSY;
            if (q.d_evecs) {
                cudaFreeAsync(q.d_evecs, S->owner->st);
                S->held -= q.keep_bytes;
            }
            S->lru.remove(ticket);
            S->reqs.erase(it);
        }
    }
    S->cv_work.notify_all();
    return BSE_OK;
}

int chase_server_destroy(bsechase_ctx *ctx) {
    if (!ctx) return BSE_EINVAL;
    bse_server_shutdown(ctx);
    return BSE_OK;
}

int chase_server_batching(bsechase_ctx *ctx, int enabled, double window_s) {
    if (!ctx || !ctx->server) return BSE_EINVAL;
    BseServer *S = ctx->server;
    if (!(window_s >= 0.0 && window_s <= 1.0))
        return fail(ctx, BSE_EINVAL, "batching window must be in [0, 1] s%s");
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto &kv : S->reqs)
        if (kv.second->state != 2 && !kv.second->cancelled)
            return fail(ctx, BSE_EBUSY, "requests are queued or running%s");
    if (!enabled) {
        for (bsechase_ctx *c : S->slots) c->batcher = nullptr;
        ozb_destroy(S->batcher);
        S->batcher = nullptr;
        return BSE_OK;
    }
    if (!S->batcher) S->batcher = ozb_create(ctx->device, ctx->sms, window_s);
    if (!S->batcher) return fail(ctx, BSE_ECUDA, "cannot create the product batcher%s");
    ozb_set_window(S->batcher, window_s);
    for (bsechase_ctx *c : S->slots) c->batcher = S->batcher;
    return BSE_OK;
}

int chase_server_batch_stats(bsechase_ctx *ctx, int64_t *launches, int64_t *products,
                             int *max_products) {
    if (!ctx || !ctx->server || !launches || !products || !max_products) return BSE_EINVAL;
    BseServer *S = ctx->server;
    std::lock_guard<std::mutex> lk(S->mu);
    *launches = *products = 0;
    *max_products = 0;
    if (S->batcher) ozb_counts(S->batcher, launches, products, max_products);
    return BSE_OK;
}

int chase_server_info(bsechase_ctx *ctx, size_t *held_bytes, int *queued, int *running) {
    if (!ctx || !ctx->server) return BSE_EINVAL;
    BseServer *S = ctx->server;
    std::lock_guard<std::mutex> lk(S->mu);
    int nq = 0, nr = 0;
    for (auto &kv : S->reqs) {
        nq += kv.second->state == 0 && !kv.second->cancelled;
        nr += kv.second->state == 1;
    }
    if (held_bytes) *held_bytes = S->held;
    if (queued) *queued = nq;
    if (running) *running = nr;
    return BSE_OK;
}

}  // extern "C"

// Request loop with continuous batching (helm_serve_start / helm_submit /
// helm_poll / helm_serve_stop).
//
// One worker thread owns the context's stream.  Per factor set (a cached
// grid + ORAS handle keyed by model id, grid, decomposition and solver
// settings) it keeps one batched Krylov engine with a fixed number of column
// slots.  Each right-hand side of a request occupies one slot.  The worker
// repeats: take over factor sets the builder has finished; admit queued
// requests whose factors are ready and whose columns fit the free slots,
// and for a request whose factors are neither ready nor being built reserve
// their estimated bytes within the HBM budget (evicting idle factor sets
// least-recently-used) and hand the build to the builder; run one restart
// cycle of every batch that has active columns; hand back the columns that
// finished (copying their solutions out) and free their slots.  New requests
// therefore join running batches at cycle boundaries and share every kernel
// launch with them.
//
// The builder is a second host thread with a context of its own (its own
// non-blocking stream on the same device): it sets up the grid and factors a
// new set while the worker keeps cycling the running batches, so admission
// of a new model or frequency never stalls the others.  A finished set is
// handed over to the serving context (its grid is re-parented and its bytes
// move from the builder's account to the serving context's) before its
// engine is made and its first request admitted.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include <cstdarg>
#include <cstdio>
#include <cstdlib>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// HELM_SERVE_TRACE=1 in the environment: the worker and the builder log their events on stderr.
bool trace_on() {
    static const bool on = [] {
        const char* v = std::getenv("HELM_SERVE_TRACE");
        return v && v[0] == '1';
    }();
    return on;
}
void trace(const char* fmt, ...) {
    if (!trace_on()) return;
    static const Clock::time_point t0 = Clock::now();
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    fprintf(stderr, "[serve %9.3f] %s\n", std::chrono::duration<double>(Clock::now() - t0).count(), buf);
    fflush(stderr);
}

double ms_since(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct FactorSet;

struct SRequest {
    uint64_t ticket = 0;
    helm_request req{};
    int state = 0;   // 0 queued, 1 running, 2 done
    helm_status status = HELM_OK;
    Clock::time_point t_submit, t_admit, t_done;
    std::vector<int> slots;
    int cols_left = 0;
    int iters_max = 0;
    double rel_max = 0.0;
    bool reused = false;
    bool built_for = false;   // its factor set was built for it (not found in the cache)
    bool notconv = false;
    FactorSet* fs = nullptr;
};

bool same_grid(const helm_grid_desc& a, const helm_grid_desc& b) {
    if (a.nx != b.nx || a.ny != b.ny || a.nz != b.nz || a.h != b.h || a.freq_hz != b.freq_hz || a.npml != b.npml ||
        a.pml_R != b.pml_R || a.top_bc != b.top_bc || a.weight_bins != b.weight_bins)
        return false;
    for (int i = 0; i < 7; ++i)
        if (a.weights[i] != b.weights[i]) return false;
    return true;
}
bool same_oras(const helm_oras_desc& a, const helm_oras_desc& b) {
    return a.px == b.px && a.py == b.py && a.pz == b.pz && a.overlap == b.overlap && a.coarse_ratio == b.coarse_ratio &&
           a.interface_bc == b.interface_bc && a.factor_prec == b.factor_prec && a.coarse_iters == b.coarse_iters &&
           (a.coarse_iters == 0 || a.coarse_overlap == b.coarse_overlap);
}

struct FactorSet {
    int building = 0;               // 1 while the builder owns it (queued or being built)
    const void* c = nullptr;        // wave speed of the request that asked for it (read by the build)
    size_t reserved = 0;            // budget bytes reserved from the request to the handover
    size_t reserved_at_queue = 0;   // the same estimate (factors, solver workspace, apply scratch)
    bool cycled = false;            // its first restart cycle has run (the apply scratch is allocated by then)
    size_t built_bytes = 0;         // device bytes the build left allocated
    helm_status build_status = HELM_OK;
    std::string build_msg;
    uint64_t model_id = 0;
    helm_grid_desc gd{};
    helm_oras_desc od{};
    int restart = 0, flexible = 0, basis_prec = 0;
    int width = 0;                  // column slots of its engine (a power of two >= 16, at most the server's)
    helm_grid g = nullptr;
    helm_oras o = nullptr;
    std::unique_ptr<KrylovEngine> K;
    std::vector<SRequest*> owner;   // per slot
    std::vector<int> col;           // per slot: column index within its request
    int active = 0;
    Clock::time_point last_used;

    bool matches(const helm_request& r) const {
        return model_id == r.model_id && same_grid(gd, r.grid) && same_oras(od, r.oras) &&
               restart == r.gmres.restart && flexible == r.gmres.flexible && basis_prec == r.gmres.basis_prec;
    }
    int free_slots() const {
        int n = 0;
        for (auto* p : owner) n += p == nullptr;
        return n;
    }
};

// dst[p * S + slot[c]] = src[p * ns + c]   (request columns into batch slots)
__global__ void pack_columns(const c128* __restrict__ src, c128* __restrict__ dst, const int* __restrict__ slot,
                             long long N, int ns, int S) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N * ns; e += (long long)gridDim.x * blockDim.x) {
        const long long p = e / ns;
        const int c = (int)(e % ns);
        dst[p * S + slot[c]] = src[e];
    }
}

// dst[p * ns + c] = src[p * S + slot[c]]   (batch slots back into a request's layout)
__global__ void unpack_columns(const c128* __restrict__ src, c128* __restrict__ dst, const int* __restrict__ slot,
                               long long N, int ns, int S) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N * ns; e += (long long)gridDim.x * blockDim.x) {
        const long long p = e / ns;
        const int c = (int)(e % ns);
        dst[e] = src[p * S + slot[c]];
    }
}

}  // namespace

struct Server {
    helm_ctx ctx = nullptr;
    int slots = 0;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::deque<SRequest*> incoming;                 // submitted, not yet seen by the worker
    std::unordered_map<uint64_t, SRequest*> reqs;   // every live ticket
    uint64_t next_ticket = 1;
    // worker-only state
    std::deque<SRequest*> waiting;
    std::vector<FactorSet*> sets;
    int* dslot = nullptr;                           // device slot map for (un)packing
    size_t reserved = 0;                            // worker: bytes reserved for sets being built
    // builders: NBUILD host threads, each with its own context and stream; queues guarded by mu.  Two builders
    // (two sets factored at once) measured no gain on the request stream (0.86 vs 0.87 requests/s saturated:
    // the solves, not the builds, bound it), so one is used
    static constexpr int NBUILD = 1;
    helm_ctx bctxs[NBUILD] = {};
    cudaStream_t bstreams[NBUILD] = {};
    std::thread bths[NBUILD];
    std::condition_variable bcv;
    bool bstop = false;
    std::deque<FactorSet*> to_build, built;

    void build_loop(int bi) {
        helm_ctx bctx = bctxs[bi];
        cudaSetDevice(ctx->device);
        for (;;) {
            FactorSet* fs = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                bcv.wait(lk, [&] { return bstop || !to_build.empty(); });
                if (to_build.empty()) break;
                fs = to_build.front();
                to_build.pop_front();
            }
            const size_t before = bctx->in_use;
            trace("build start: model %llu, grid %dx%dx%d, f %.2f", (unsigned long long)fs->model_id, fs->gd.nx,
                  fs->gd.ny, fs->gd.nz, fs->gd.freq_hz);
            helm_status st = helm_setup_grid(bctx, &fs->gd, fs->c, &fs->g);
            if (!st) st = oras_factor(fs->g, &fs->od, &fs->o);
            if (!st) st = cuda_check(bctx, cudaStreamSynchronize(bctx->stream), "factor set build");
            if (st) {
                fs->build_msg = bctx->last_error;
                if (fs->o) oras_destroy(fs->o);
                fs->o = nullptr;
                if (fs->g) helm_destroy_grid(fs->g);
                fs->g = nullptr;
            } else {
                // the set's bytes leave the builder's account; the worker adds them to the serving context
                fs->built_bytes = bctx->in_use - before;
                bctx->in_use = before;
                bctx->children--;
            }
            fs->build_status = st;
            trace("build done: model %llu, status %d, %.2f GB", (unsigned long long)fs->model_id, st,
                  fs->built_bytes / 1e9);
            {
                std::lock_guard<std::mutex> lk(mu);
                built.push_back(fs);
            }
            cv.notify_one();
        }
    }

    // Worker: take over the sets the builder has finished.
    void take_built() {
        std::deque<FactorSet*> done;
        {
            std::lock_guard<std::mutex> lk(mu);
            done.swap(built);
        }
        for (FactorSet* fs : done) {
            reserved -= fs->reserved;
            fs->reserved = 0;
            helm_status st = fs->build_status;
            if (!st) {
                fs->g->ctx = ctx;   // re-parent: every later call on the set runs on the serving stream
                ctx->children++;
                ctx->in_use += fs->built_bytes;
                trace("take over model %llu: %.2f GB built against %.2f GB reserved", (unsigned long long)fs->model_id,
                      fs->built_bytes / 1e9, fs->reserved_at_queue / 1e9);
                const size_t in0 = ctx->in_use;
                fs->K.reset(make_krylov_engine(fs->o, fs->width, fs->restart, fs->flexible != 0, fs->basis_prec,
                                               nullptr, nullptr, &st));
                if (!st) hold_residual(fs, fs->built_bytes + (ctx->in_use - in0));
                if (st == HELM_ENOMEM) {
                    // the budget has no room for the engine now (the factors took more than their estimate, or
                    // other sets grew meanwhile): the set stays without one, and try_admit makes it once idle
                    // sets can be evicted or running ones have finished
                    trace("engine for model %llu deferred: no room in the budget", (unsigned long long)fs->model_id);
                    fs->K.reset();
                    st = HELM_OK;
                } else if (st) {
                    fs->build_msg = ctx->last_error;
                }
            }
            fs->building = 0;
            if (st) {
                // every waiting request for this set fails with the build's error
                set_error(ctx, st, "%s", fs->build_msg.c_str());
                for (auto it = waiting.begin(); it != waiting.end();) {
                    if (fs->matches((*it)->req)) {
                        finish(*it, st);
                        it = waiting.erase(it);
                    } else {
                        ++it;
                    }
                }
                sets.erase(std::find(sets.begin(), sets.end(), fs));
                destroy_set(fs);
                continue;
            }
            fs->owner.assign(fs->width, nullptr);
            fs->col.assign(fs->width, -1);
            fs->last_used = Clock::now();
        }
    }

    // engine width for a request of nrhs columns: a power of two from 16 up, at most the server's slot count
    int width_for(int nrhs) const {
        int w = 16;
        while (w < nrhs) w *= 2;
        return std::min(w, slots);
    }

    void finish(SRequest* r, helm_status st) {
        trace("finish ticket %llu: status %d", (unsigned long long)r->ticket, st);
        std::lock_guard<std::mutex> lk(mu);
        r->status = st;
        r->state = 2;
        r->t_done = Clock::now();
    }

    void destroy_set(FactorSet* fs) {
        reserved -= fs->reserved;   // a residual still held for its first cycle
        fs->reserved = 0;
        fs->K.reset();
        if (fs->o) oras_destroy(fs->o);
        if (fs->g) helm_destroy_grid(fs->g);
        delete fs;
    }

    size_t engine_estimate(const helm_request& r, int width) const {
        const size_t N = (size_t)r.grid.nx * r.grid.ny * r.grid.nz;
        const size_t e = r.gmres.basis_prec == HELM_PREC_FP64 ? sizeof(c128) : sizeof(c64);
        const size_t m = (size_t)r.gmres.restart;
        return N * width * ((2 * m + 3) * e + 3 * sizeof(c128)) + N * 48;
    }

    // Evict idle factor sets other than keep (least recently used first) until `bytes` more fit the budget;
    // returns whether they fit.
    bool make_room(size_t bytes, FactorSet* keep) {
        auto room = [&]() { return ctx->budget == 0 || ctx->in_use + reserved + bytes <= ctx->budget; };
        while (!room()) {
            FactorSet* lru = nullptr;
            for (auto* s2 : sets)
                if (s2 != keep && !s2->building && s2->active == 0 && !wanted(s2) &&
                    (!lru || s2->last_used < lru->last_used))
                    lru = s2;
            if (!lru) break;
            sets.erase(std::find(sets.begin(), sets.end(), lru));
            trace("evict model %llu (grid %d^3)", (unsigned long long)lru->model_id, lru->gd.nx);
            destroy_set(lru);
        }
        return room();
    }

    // Whether a queued request asks for this set (a set built for a request that is not admitted yet is not
    // evicted for another's room: that would throw the build away and queue it again).
    bool wanted(const FactorSet* fs) const {
        for (const SRequest* w : waiting)
            if (fs->matches(w->req)) return true;
        return false;
    }

    // After a set's solver workspace is made: keep reserved what its estimate still expects (the apply scratch,
    // allocated by its first restart cycle), so that other admissions do not spend it meanwhile.
    void hold_residual(FactorSet* fs, size_t used) {
        reserved -= fs->reserved;
        fs->reserved = fs->reserved_at_queue > used ? fs->reserved_at_queue - used : 0;
        reserved += fs->reserved;
    }

    // Whether a set other than fs is being built or has running columns (so that budget room will come back).
    bool others_busy(const FactorSet* fs) const {
        for (auto* s2 : sets)
            if (s2 != fs && (s2->building || s2->active > 0)) return true;
        return false;
    }

    // Try to place r: returns true if admitted (or failed), false if it must keep waiting (its factors are
    // being built, or its columns or its factors do not fit yet).
    bool try_admit(SRequest* r, bool idle) {
        FactorSet* fs = nullptr;
        for (auto* s : sets)
            if (s->matches(r->req)) fs = s;
        if (!fs) {
            const int width = width_for(r->req.nrhs);
            const size_t need = oras_estimate_bytes(r->req.grid, r->req.oras, width) + engine_estimate(r->req, width);
            if (!make_room(need, nullptr)) {
                if (idle && sets.empty()) {
                    set_error(ctx, HELM_ENOMEM, "request needs about %zu bytes, more than the HBM budget", need);
                    finish(r, HELM_ENOMEM);
                    return true;
                }
                return false;
            }
            fs = new FactorSet();
            fs->model_id = r->req.model_id;
            fs->gd = r->req.grid;
            fs->od = r->req.oras;
            fs->restart = r->req.gmres.restart;
            fs->flexible = r->req.gmres.flexible;
            fs->basis_prec = r->req.gmres.basis_prec;
            fs->c = r->req.c;
            fs->width = width;
            fs->building = 1;
            trace("queue build for ticket %llu (need %.2f GB, in use %.2f, reserved %.2f)",
                  (unsigned long long)r->ticket, need / 1e9, ctx->in_use / 1e9, reserved / 1e9);
            r->built_for = true;
            fs->reserved = need;
            fs->reserved_at_queue = need;
            reserved += need;
            sets.push_back(fs);
            {
                std::lock_guard<std::mutex> lk(mu);
                to_build.push_back(fs);
            }
            bcv.notify_one();
            return false;
        }
        if (fs->building) return false;
        if (!fs->K) {
            // the engine deferred at the handover: make it once the budget has room, evicting idle sets
            const size_t eb = engine_estimate(r->req, fs->width);
            if (!make_room(eb, fs)) {
                if (others_busy(fs)) return false;   // room comes back when the others finish
                set_error(ctx, HELM_ENOMEM, "request's solver workspace (about %zu bytes) does not fit the HBM budget",
                          eb);
                finish(r, HELM_ENOMEM);
                return true;
            }
            helm_status st = HELM_OK;
            const size_t in0 = ctx->in_use;
            fs->K.reset(make_krylov_engine(fs->o, fs->width, fs->restart, fs->flexible != 0, fs->basis_prec, nullptr,
                                           nullptr, &st));
            if (st) {
                fs->K.reset();
                if (st == HELM_ENOMEM && others_busy(fs)) return false;
                finish(r, st);
                return true;
            }
            hold_residual(fs, fs->built_bytes + (ctx->in_use - in0));
            trace("engine for model %llu made (%d columns)", (unsigned long long)fs->model_id, fs->width);
        }
        if (fs->width < r->req.nrhs) {
            // a wider engine for this set, made once its running columns have finished, with room made by
            // evicting other idle sets if needed
            if (fs->active > 0) return false;
            const int width = width_for(r->req.nrhs);
            // the solver workspace grows now, the apply scratch at the set's next cycle (reserved until then)
            const size_t s_new = oras_estimate_bytes(r->req.grid, r->req.oras, width);
            const size_t s_old = oras_estimate_bytes(r->req.grid, r->req.oras, fs->width);
            const size_t scratch = s_new > s_old ? s_new - s_old : 0;
            const size_t more = engine_estimate(r->req, width) - engine_estimate(r->req, fs->width) + scratch;
            if (!make_room(more, fs)) {
                if (others_busy(fs)) return false;   // room comes back when the others finish
                set_error(ctx, HELM_ENOMEM, "request needs about %zu more bytes than the HBM budget leaves", more);
                finish(r, HELM_ENOMEM);
                return true;
            }
            trace("widen model %llu to %d columns", (unsigned long long)fs->model_id, width);
            helm_status st = HELM_OK;
            fs->K.reset();
            fs->K.reset(make_krylov_engine(fs->o, width, fs->restart, fs->flexible != 0, fs->basis_prec, nullptr,
                                           nullptr, &st));
            if (st) {
                // no room for the wider engine after all: drop the (idle) set; a later request rebuilds it
                sets.erase(std::find(sets.begin(), sets.end(), fs));
                destroy_set(fs);
                finish(r, st);
                return true;
            }
            fs->width = width;
            fs->owner.assign(width, nullptr);
            fs->col.assign(width, -1);
            reserved -= fs->reserved;
            fs->reserved = scratch;
            reserved += scratch;
            fs->cycled = false;
        }
        if (fs->free_slots() < r->req.nrhs) return false;
        r->reused = !r->built_for;
        // take slots, copy the request's columns into them and start them
        const long long N = fs->g->n;
        std::vector<int> sl;
        for (int s = 0; s < fs->width && (int)sl.size() < r->req.nrhs; ++s)
            if (!fs->owner[s]) sl.push_back(s);
        cudaStream_t st = ctx->stream;
        const size_t bytes = (size_t)N * r->req.nrhs * sizeof(c128);
        void* stage = nullptr;
        const c128* src = (const c128*)r->req.b;
        helm_status rc = HELM_OK;
        if (!is_device_pointer(r->req.b)) {
            rc = dev_alloc(ctx, &stage, bytes, "request b staging");
            if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(stage, r->req.b, bytes, cudaMemcpyHostToDevice, st), "b H2D");
            src = (const c128*)stage;
        }
        if (!rc) rc = cuda_check(ctx, cudaMemcpyAsync(dslot, sl.data(), sl.size() * sizeof(int), cudaMemcpyHostToDevice, st),
                                 "slot map");
        if (!rc) {
            pack_columns<<<(unsigned)std::min<long long>((N * r->req.nrhs + 255) / 256, 4096), 256, 0, st>>>(
                src, fs->K->B(), dslot, N, r->req.nrhs, fs->width);
            ctx->launches++;
            std::vector<double> tol(sl.size(), r->req.gmres.tol);
            std::vector<int> maxit(sl.size(), r->req.gmres.maxit);
            rc = fs->K->begin_columns(sl.data(), (int)sl.size(), tol.data(), maxit.data());
        }
        cudaStreamSynchronize(st);
        if (stage) dev_free(ctx, stage, bytes);
        if (rc) {
            for (int s : sl) fs->K->retire(s);
            fs->K->push_state();
            finish(r, rc);
            return true;
        }
        for (size_t i = 0; i < sl.size(); ++i) {
            fs->owner[sl[i]] = r;
            fs->col[sl[i]] = (int)i;
        }
        fs->active += (int)sl.size();
        fs->last_used = Clock::now();
        trace("admit ticket %llu: %d columns into a set of width %d (%d active)", (unsigned long long)r->ticket,
              (int)sl.size(), fs->width, fs->active);
        r->fs = fs;
        r->slots = sl;
        r->cols_left = (int)sl.size();
        {
            std::lock_guard<std::mutex> lk(mu);
            r->state = 1;
            r->t_admit = Clock::now();
        }
        return true;
    }

    // Copy a finished request's columns out and release its slots.
    void complete(FactorSet* fs, SRequest* r) {
        const long long N = fs->g->n;
        cudaStream_t st = ctx->stream;
        const size_t bytes = (size_t)N * r->req.nrhs * sizeof(c128);
        helm_status rc = cuda_check(
            ctx, cudaMemcpyAsync(dslot, r->slots.data(), r->slots.size() * sizeof(int), cudaMemcpyHostToDevice, st),
            "slot map");
        void* stage = nullptr;
        c128* dst = (c128*)r->req.x;
        const bool xdev = is_device_pointer(r->req.x);
        if (!rc && !xdev) {
            rc = dev_alloc(ctx, &stage, bytes, "request x staging");
            dst = (c128*)stage;
        }
        if (!rc) {
            unpack_columns<<<(unsigned)std::min<long long>((N * r->req.nrhs + 255) / 256, 4096), 256, 0, st>>>(
                fs->K->X(), dst, dslot, N, r->req.nrhs, fs->width);
            ctx->launches++;
            if (!xdev) rc = cuda_check(ctx, cudaMemcpyAsync(r->req.x, stage, bytes, cudaMemcpyDeviceToHost, st), "x D2H");
        }
        if (!rc) rc = cuda_check(ctx, cudaStreamSynchronize(st), "request completion");
        if (stage) dev_free(ctx, stage, bytes);
        for (int s : r->slots) {
            fs->K->retire(s);
            fs->owner[s] = nullptr;
            fs->col[s] = -1;
        }
        fs->K->push_state();
        fs->active -= (int)r->slots.size();
        fs->last_used = Clock::now();
        finish(r, rc ? rc : (r->notconv ? HELM_ENOTCONV : HELM_OK));
    }

    void loop() {
        cudaSetDevice(ctx->device);
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu);
                bool running = false, building = false;
                for (auto* s : sets) {
                    running = running || s->active > 0;
                    building = building || s->building;
                }
                if (!running && incoming.empty() && built.empty()) {
                    if (stop && waiting.empty() && !building) break;
                    // nothing to cycle: sleep until a submission or a finished build (or 20 ms)
                    cv.wait_for(lk, std::chrono::milliseconds(20));
                }
                while (!incoming.empty()) {
                    waiting.push_back(incoming.front());
                    incoming.pop_front();
                }
            }
            take_built();
            bool idle = true;
            for (auto* s : sets) idle = idle && s->active == 0 && !s->building;
            for (auto it = waiting.begin(); it != waiting.end();) {
                if (try_admit(*it, idle)) {
                    it = waiting.erase(it);
                    idle = false;
                } else {
                    ++it;
                }
            }
            for (auto* fs : sets) {
                if (fs->active == 0) continue;
                bool any = false;
                const auto tc0 = Clock::now();
                helm_status rc = fs->K->cycle(&any);
                if (!fs->cycled) {
                    // the apply scratch exists now and is counted in use: the residual reservation is not needed
                    fs->cycled = true;
                    reserved -= fs->reserved;
                    fs->reserved = 0;
                }
                trace("cycle model %llu (grid %d^3, width %d, %d active): status %d, %.1f ms",
                      (unsigned long long)fs->model_id, fs->gd.nx, fs->width, fs->active, rc,
                      ms_since(tc0, Clock::now()));
                std::vector<SRequest*> done_reqs;
                for (int s = 0; s < fs->width; ++s) {
                    SRequest* r = fs->owner[s];
                    if (!r) continue;
                    const RhsState& cs = fs->K->state(s);
                    if (rc || cs.done) {
                        if (std::find(done_reqs.begin(), done_reqs.end(), r) == done_reqs.end()) done_reqs.push_back(r);
                    }
                }
                for (auto* r : done_reqs) {
                    bool all = true;
                    for (int s : r->slots) all = all && (rc || fs->K->state(s).done);
                    if (!all) continue;
                    for (int s : r->slots) {
                        const RhsState& cs = fs->K->state(s);
                        const double tr = fs->K->true_rel(s);
                        r->iters_max = std::max(r->iters_max, cs.iters);
                        r->rel_max = std::max(r->rel_max, tr);
                        if (!(tr <= cs.tol)) r->notconv = true;
                    }
                    if (rc) {
                        for (int s : r->slots) {
                            fs->K->retire(s);
                            fs->owner[s] = nullptr;
                        }
                        fs->K->push_state();
                        fs->active -= (int)r->slots.size();
                        finish(r, rc);
                    } else {
                        complete(fs, r);
                    }
                }
            }
        }
        for (auto* s : sets) destroy_set(s);
        sets.clear();
    }
};

extern "C" helm_status helm_serve_start(helm_ctx ctx, int slots) {
    if (!ctx) return HELM_EINVAL;
    if (ctx->server) return set_error(ctx, HELM_EBUSY, "helm_serve_start: already serving");
    if (slots < 1 || slots > 256) return set_error(ctx, HELM_EINVAL, "helm_serve_start: slots must be 1..256");
    HELM_CUDA(ctx, cudaSetDevice(ctx->device));
    Server* sv = new Server();
    sv->ctx = ctx;
    sv->slots = slots;
    helm_status rc = dev_alloc(ctx, (void**)&sv->dslot, 256 * sizeof(int), "slot map");
    if (rc) {
        delete sv;
        return rc;
    }
    // the builders' contexts: same device, each its own non-blocking stream, no budget of their own (the worker
    // reserves every build's bytes within the serving context's budget), the serving context's tuning
    for (int i = 0; i < Server::NBUILD && !rc; ++i) {
        rc = cuda_check(ctx, cudaStreamCreateWithFlags(&sv->bstreams[i], cudaStreamNonBlocking), "builder stream");
        if (!rc) rc = helm_create(&sv->bctxs[i], ctx->device, sv->bstreams[i], 0);
    }
    if (rc) {
        for (int i = 0; i < Server::NBUILD; ++i) {
            if (sv->bctxs[i]) helm_destroy(sv->bctxs[i]);
            if (sv->bstreams[i]) cudaStreamDestroy(sv->bstreams[i]);
        }
        dev_free(ctx, sv->dslot, 256 * sizeof(int));
        delete sv;
        return set_error(ctx, rc, "helm_serve_start: builder context");
    }
    for (helm_ctx b : sv->bctxs) {
        b->tc_stages = ctx->tc_stages;
        b->coarse_coop = ctx->coarse_coop;
        b->use_graphs = ctx->use_graphs;
        b->tc_flow = ctx->tc_flow;
        b->stencil_march = ctx->stencil_march;
        b->stencil_planes = ctx->stencil_planes;
        b->tc_factor = ctx->tc_factor;
        b->block_gj = ctx->block_gj;
    }
    ctx->server = sv;
    for (int i = 0; i < Server::NBUILD; ++i) sv->bths[i] = std::thread([sv, i]() { sv->build_loop(i); });
    sv->th = std::thread([sv]() { sv->loop(); });
    return HELM_OK;
}

extern "C" helm_status helm_submit(helm_ctx ctx, const helm_request* req, uint64_t* ticket) {
    if (!ctx || !req || !ticket) return HELM_EINVAL;
    Server* sv = ctx->server;
    if (!sv) return set_error(ctx, HELM_EINVAL, "helm_submit: serving not started");
    if (req->nrhs < 1 || req->nrhs > sv->slots || !req->b || !req->x || !req->c || !(req->gmres.tol > 0) ||
        req->gmres.restart < 1 || req->gmres.restart > 200 || req->gmres.maxit < 1 ||
        (req->gmres.basis_prec != HELM_PREC_FP64 && req->gmres.basis_prec != HELM_PREC_FP32))
        return set_error(ctx, HELM_EINVAL, "helm_submit: malformed request");
    if (req->gmres.use_x0) return set_error(ctx, HELM_EINVAL, "helm_submit: warm starts are for gmres_solve only");
    SRequest* r = new SRequest();
    r->req = *req;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            delete r;
            return set_error(ctx, HELM_EBUSY, "helm_submit: serving is stopping");
        }
        r->ticket = sv->next_ticket++;
        sv->reqs[r->ticket] = r;
        sv->incoming.push_back(r);
    }
    sv->cv.notify_one();
    *ticket = r->ticket;
    return HELM_OK;
}

extern "C" helm_status helm_poll(helm_ctx ctx, uint64_t ticket, int* done, helm_request_stats* stats) {
    if (!ctx || !done) return HELM_EINVAL;
    Server* sv = ctx->server;
    if (!sv) return set_error(ctx, HELM_EINVAL, "helm_poll: serving not started");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return HELM_ENOTFOUND;
    SRequest* r = it->second;
    *done = r->state == 2;
    if (stats) {
        const auto now = Clock::now();
        stats->done = *done;
        stats->status = r->status;
        stats->iterations_max = r->iters_max;
        stats->true_relres_max = r->rel_max;
        stats->queue_ms = r->state >= 1 ? ms_since(r->t_submit, r->t_admit) : ms_since(r->t_submit, now);
        stats->latency_ms = r->state == 2 ? ms_since(r->t_submit, r->t_done) : ms_since(r->t_submit, now);
        stats->factors_reused = r->reused ? 1 : 0;
    }
    if (*done) {
        sv->reqs.erase(it);
        delete r;
    }
    return HELM_OK;
}

extern "C" helm_status helm_serve_stop(helm_ctx ctx) {
    if (!ctx) return HELM_EINVAL;
    Server* sv = ctx->server;
    if (!sv) return HELM_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_one();
    sv->th.join();   // the worker waits for every build it started before it ends
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->bstop = true;
    }
    sv->bcv.notify_all();
    for (auto& t : sv->bths) t.join();
    for (int i = 0; i < Server::NBUILD; ++i) {
        helm_destroy(sv->bctxs[i]);
        cudaStreamDestroy(sv->bstreams[i]);
    }
    for (auto& kv : sv->reqs) delete kv.second;
    dev_free(ctx, sv->dslot, 256 * sizeof(int));
    delete sv;
    ctx->server = nullptr;
    return HELM_OK;
}

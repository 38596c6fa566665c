// Frequency sweeps over one model (helm_frequency_sweep): grid set-up, ORAS factorisation and
// (F)GMRES per frequency, with optional warm starts from the previous frequency's solution and
// optional overlap of the next frequency's factorisation with the current solve.
//
// Overlap: a second host thread builds the handles of frequency i + 1 while the caller's thread
// solves frequency i.  Frequencies alternate between two contexts (the caller's and one made for the
// call, on a stream of its own), and a context is used by one thread at a time: the builder starts
// frequency i only after the solver has released frequency i - 2, the last user of that context.
// Each handle is built, used and freed on its own context, so a solve runs on exactly the kernels and
// stream order it would have without the overlap (bit-identical results).
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

struct FreqSlot {
    helm_grid g = nullptr;
    helm_oras o = nullptr;
    helm_status st = HELM_OK;
    std::string msg;
    double setup_s = 0.0;
    bool built = false;      // handles (or the error) are ready
    bool released = false;   // the solver is done with this frequency's context
};

struct Shared {
    std::mutex mu;
    std::condition_variable cv;
    std::vector<FreqSlot> slot;
    bool abort = false;
};

helm_status build_one(helm_ctx ctx, const helm_sweep_desc& d, const void* c, int i, FreqSlot& s) {
    const auto t0 = std::chrono::steady_clock::now();
    helm_grid_desc gd = d.grid;
    gd.freq_hz = d.freqs[i];
    helm_status st = helm_setup_grid(ctx, &gd, c, &s.g);
    if (st == HELM_OK) st = oras_factor(s.g, &d.oras, &s.o);
    if (st != HELM_OK) s.msg = ctx->last_error;
    s.setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

void free_one(FreqSlot& s) {
    if (s.o) oras_destroy(s.o);
    if (s.g) helm_destroy_grid(s.g);
    s.o = nullptr;
    s.g = nullptr;
}

bool is_device(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" helm_status helm_frequency_sweep(helm_ctx ctx, const helm_sweep_desc* d, const void* c, const void* b,
                                            void* x, int nrhs, helm_rhs_stats* stats, double* setup_s) {
    if (!ctx) return HELM_EINVAL;
    if (!d || !c || !b || !x || nrhs < 1 || d->nfreq < 1 || d->nfreq > 64 || !d->freqs ||
        (d->warm != 0 && d->warm != 1) || (d->overlap != 0 && d->overlap != 1))
        return set_error(ctx, HELM_EINVAL, "helm_frequency_sweep: invalid argument");
    for (int i = 0; i < d->nfreq; ++i)
        if (!(d->freqs[i] > 0.0)) return set_error(ctx, HELM_EINVAL, "helm_frequency_sweep: frequencies must be > 0");
    if (ctx->server) return set_error(ctx, HELM_EBUSY, "helm_frequency_sweep: the serving loop is active");
    const bool dev = is_device(x);
    if (dev != is_device(b)) return set_error(ctx, HELM_EINVAL, "helm_frequency_sweep: b and x must be on the same side");
    const long long n = (long long)d->grid.nx * d->grid.ny * d->grid.nz;
    if (n <= 0) return set_error(ctx, HELM_EINVAL, "helm_frequency_sweep: empty grid");
    const size_t bytes = (size_t)n * nrhs * sizeof(c128);
    helm_gmres_desc gm = d->gmres;
    const int nf = d->nfreq;

    // the second context (overlap): same device and budget, its own non-blocking stream, the caller's tuning
    helm_ctx ctx2 = nullptr;
    cudaStream_t st2 = nullptr;
    if (d->overlap) {
        HELM_CUDA(ctx, cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
        helm_status rc = helm_create(&ctx2, ctx->device, st2, ctx->budget);
        if (rc != HELM_OK) {
            cudaStreamDestroy(st2);
            return set_error(ctx, rc, "helm_frequency_sweep: second context: %s", helm_last_error(nullptr));
        }
        ctx2->tc_stages = ctx->tc_stages;
        ctx2->coarse_coop = ctx->coarse_coop;
        ctx2->use_graphs = ctx->use_graphs;
        ctx2->tc_flow = ctx->tc_flow;
        ctx2->stencil_march = ctx->stencil_march;
        ctx2->stencil_planes = ctx->stencil_planes;
    }
    auto ctx_of = [&](int i) { return (d->overlap && (i & 1)) ? ctx2 : ctx; };

    Shared sh;
    sh.slot.resize(nf);
    std::thread builder;
    if (d->overlap) {
        builder = std::thread([&]() {
            cudaSetDevice(ctx->device);
            for (int i = 0; i < nf; ++i) {
                {
                    // frequency i reuses the context of frequency i - 2: wait until the solver released it
                    std::unique_lock<std::mutex> lk(sh.mu);
                    sh.cv.wait(lk, [&] { return sh.abort || i < 2 || sh.slot[i - 2].released; });
                    if (sh.abort) return;
                }
                FreqSlot tmp;
                tmp.st = build_one(ctx_of(i), *d, c, i, tmp);
                {
                    std::lock_guard<std::mutex> lk(sh.mu);
                    sh.slot[i].g = tmp.g;
                    sh.slot[i].o = tmp.o;
                    sh.slot[i].st = tmp.st;
                    sh.slot[i].msg = tmp.msg;
                    sh.slot[i].setup_s = tmp.setup_s;
                    sh.slot[i].built = true;
                }
                sh.cv.notify_all();
                if (tmp.st != HELM_OK) return;
            }
        });
    }

    // errors are recorded here and set on ctx after the builder has stopped (it may be using ctx)
    helm_status result = HELM_OK;
    std::string why;
    bool notconv = false;
    for (int i = 0; i < nf; ++i) {
        FreqSlot* s = &sh.slot[i];
        if (d->overlap) {
            std::unique_lock<std::mutex> lk(sh.mu);
            sh.cv.wait(lk, [&] { return s->built; });
        } else {
            s->st = build_one(ctx, *d, c, i, *s);
            s->built = true;
        }
        if (setup_s) setup_s[i] = s->setup_s;
        helm_ctx ci = ctx_of(i);
        if (s->st != HELM_OK) {
            result = s->st;
            why = "frequency " + std::to_string(i) + ": " + s->msg;
        } else {
            char* xi = (char*)x + (size_t)i * bytes;
            gm.use_x0 = 0;
            if (d->warm && i > 0) {
                const char* xp = (const char*)x + (size_t)(i - 1) * bytes;
                if (dev) {
                    helm_status rc = cuda_check(ci, cudaMemcpyAsync(xi, xp, bytes, cudaMemcpyDeviceToDevice, ci->stream),
                                                "warm-start copy");
                    if (rc == HELM_OK) rc = cuda_check(ci, cudaStreamSynchronize(ci->stream), "warm-start copy");
                    if (rc != HELM_OK) {
                        result = rc;
                        why = ci->last_error;
                    }
                } else {
                    memcpy(xi, xp, bytes);
                }
                gm.use_x0 = 1;
            }
            if (result == HELM_OK) {
                helm_status rc = gmres_solve(s->o, b, xi, nrhs, &gm, stats ? stats + (size_t)i * nrhs : nullptr);
                if (rc == HELM_ENOTCONV) {
                    notconv = true;
                } else if (rc != HELM_OK) {
                    result = rc;
                    why = "frequency " + std::to_string(i) + ": " + ci->last_error;
                }
            }
        }
        {
            std::lock_guard<std::mutex> lk(sh.mu);
            free_one(*s);
            s->released = true;
            if (result != HELM_OK) sh.abort = true;
        }
        sh.cv.notify_all();
        if (result != HELM_OK) break;
    }
    if (builder.joinable()) builder.join();
    for (auto& s : sh.slot) free_one(s);   // built ahead of an error
    if (ctx2) helm_destroy(ctx2);
    if (st2) cudaStreamDestroy(st2);
    if (result != HELM_OK) return set_error(ctx, result, "helm_frequency_sweep: %s", why.c_str());
    if (notconv) return set_error(ctx, HELM_ENOTCONV, "helm_frequency_sweep: some columns did not reach tol");
    return HELM_OK;
}

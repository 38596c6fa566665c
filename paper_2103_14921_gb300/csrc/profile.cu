// helm_profile_*: CUDA-event timing of instrumented kernel families on the
// context's stream, with the algorithmic bytes each launch declares.
#include <string.h>

#include "internal.h"

static int family_index(Profiler& P, const char* name) {
    for (size_t i = 0; i < P.names.size(); ++i)
        if (P.names[i] == name) return (int)i;
    P.names.push_back(name);
    P.launches.push_back(0);
    P.ms.push_back(0.0);
    P.bytes.push_back(0.0);
    return (int)P.names.size() - 1;
}

static cudaEvent_t take_event(Profiler& P) {
    if (!P.pool.empty()) {
        cudaEvent_t e = P.pool.back();
        P.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void prof_drain(helm_ctx ctx) {
    Profiler& P = ctx->prof;
    if (P.pending.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& r : P.pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            P.launches[r.family] += 1;
            P.ms[r.family] += ms;
            P.bytes[r.family] += r.bytes;
        }
        P.pool.push_back(r.a);
        P.pool.push_back(r.b);
    }
    P.pending.clear();
}

constexpr int CAPTURED = 1 << 30;   // token flag: the record lives in P.capture

int prof_begin(helm_ctx ctx, const char* family) {
    Profiler& P = ctx->prof;
    if (!P.on) return -1;
    if (!P.only.empty() && std::find(P.only.begin(), P.only.end(), family) == P.only.end()) return -1;
    if (P.capture) {
        ProfRecord r;
        r.family = family_index(P, family);
        r.a = take_event(P);
        r.b = take_event(P);
        r.bytes = 0;
        cudaEventRecordWithFlags(r.a, ctx->stream, cudaEventRecordExternal);
        P.capture->push_back(r);
        return CAPTURED | (int)(P.capture->size() - 1);
    }
    if (P.pending.size() > 4096) prof_drain(ctx);
    ProfRecord r;
    r.family = family_index(P, family);
    r.a = take_event(P);
    r.b = take_event(P);
    r.bytes = 0;
    cudaEventRecord(r.a, ctx->stream);
    P.pending.push_back(r);
    return (int)P.pending.size() - 1;
}

void prof_end(helm_ctx ctx, int token, double bytes) {
    if (token < 0) return;
    Profiler& P = ctx->prof;
    if (token & CAPTURED) {
        ProfRecord& r = (*P.capture)[token & ~CAPTURED];
        r.bytes = bytes;
        cudaEventRecordWithFlags(r.b, ctx->stream, cudaEventRecordExternal);
        return;
    }
    P.pending[token].bytes = bytes;
    cudaEventRecord(P.pending[token].b, ctx->stream);
}

void prof_reserve(helm_ctx ctx, size_t n) {
    Profiler& P = ctx->prof;
    while (P.pool.size() < n) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) break;
        P.pool.push_back(e);
    }
}

void prof_harvest(helm_ctx ctx, const std::vector<ProfRecord>& recs) {
    Profiler& P = ctx->prof;
    for (const auto& r : recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            P.launches[r.family] += 1;
            P.ms[r.family] += ms;
            P.bytes[r.family] += r.bytes;
        }
    }
}

void prof_release(helm_ctx ctx, std::vector<ProfRecord>& recs) {
    Profiler& P = ctx->prof;
    for (auto& r : recs) {
        P.pool.push_back(r.a);
        P.pool.push_back(r.b);
    }
    recs.clear();
}

extern "C" helm_status helm_profile_enable(helm_ctx ctx, int on) {
    if (!ctx) return HELM_EINVAL;
    prof_drain(ctx);
    Profiler& P = ctx->prof;
    // graphs captured while profiling was off lack the event nodes; graphs that have them keep
    // recording while profiling is off, harmlessly (nothing harvests them)
    if (on && !P.on) ctx->graph_gen++;
    P.on = on != 0;
    if (P.on)
        for (size_t i = 0; i < P.names.size(); ++i) {
            P.launches[i] = 0;
            P.ms[i] = 0;
            P.bytes[i] = 0;
        }
    return HELM_OK;
}

extern "C" helm_status helm_profile_query(helm_ctx ctx, const char* name, uint64_t* launches, double* ms,
                                          double* bytes) {
    if (!ctx || !name) return HELM_EINVAL;
    prof_drain(ctx);
    Profiler& P = ctx->prof;
    for (size_t i = 0; i < P.names.size(); ++i)
        if (P.names[i] == name && P.launches[i] > 0) {
            if (launches) *launches = P.launches[i];
            if (ms) *ms = P.ms[i];
            if (bytes) *bytes = P.bytes[i];
            return HELM_OK;
        }
    return set_error(ctx, HELM_ENOTFOUND, "helm_profile_query: no launches recorded for %s", name);
}

extern "C" helm_status helm_profile_select(helm_ctx ctx, const char* families) {
    if (!ctx) return HELM_EINVAL;
    Profiler& P = ctx->prof;
    std::vector<std::string> only;
    std::string cur;
    for (const char* c = families ? families : "";; ++c) {
        if (*c == ',' || *c == 0) {
            if (!cur.empty()) only.push_back(cur);
            cur.clear();
            if (!*c) break;
        } else if (*c != ' ') {
            cur.push_back(*c);
        }
    }
    if (only != P.only) ctx->graph_gen++;   // captured graphs hold event nodes for the old selection
    P.only = only;
    return HELM_OK;
}

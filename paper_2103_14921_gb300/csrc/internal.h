// Internal declarations of the Helmholtz ORAS-GMRES library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/helm.h"

// ----------------------------------------------------------------- complex

template <typename T> struct cplx;
template <> struct __align__(8) cplx<float> { float x, y; };
template <> struct __align__(16) cplx<double> { double x, y; };

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T a, T b) { cplx<T> c; c.x = a; c.y = b; return c; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return mk<T>(s * a.x, s * a.y); }
// acc += a * b
template <typename T> __host__ __device__ __forceinline__ void cmac(cplx<T>& acc, cplx<T> a, cplx<T> b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += conj(a) * b
template <typename T> __host__ __device__ __forceinline__ void cmac_conj(cplx<T>& acc, cplx<T> a, cplx<T> b) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}

typedef cplx<double> c128;
typedef cplx<float> c64;

// ----------------------------------------------------------------- objects

struct helm_ctx_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;         // 0 = unlimited
    size_t in_use = 0;
    uint64_t launches = 0;
    std::string last_error;
    int sm_count = 0;
    int children = 0;          // live grids; helm_destroy defers the delete until they are gone
    bool destroy_pending = false;
};

// Stencil weights in product form (see stencil.cu).
struct StencilW {
    double a2, a3, m0, m1, m2, m3, inv_h2;
};

struct helm_grid_s {
    helm_ctx ctx = nullptr;
    helm_grid_desc d{};
    long long n = 0;           // nx*ny*nz
    double omega = 0, c_ref = 0;
    StencilW w{};
    // device arrays
    c128* c = nullptr;         // wave speed [N]
    c128* k2 = nullptr;        // (omega/c)^2 [N]
    c64* k2f = nullptr;
    c128* tab = nullptr;       // stretched 1-D tables, [nx+ny+nz][3] (cm, c0, cp): x, then y, then z
    c64* tabf = nullptr;
    std::vector<c128> htab;    // host copy of the tables
    int refs = 0;              // ORAS handles built on this grid
};

// ----------------------------------------------------------------- helpers

helm_status set_error(helm_ctx ctx, helm_status st, const char* fmt, ...);
helm_status cuda_check(helm_ctx ctx, cudaError_t e, const char* what);
helm_status dev_alloc(helm_ctx ctx, void** p, size_t bytes, const char* what);
void dev_free(helm_ctx ctx, void* p, size_t bytes);

#define HELM_TRY(expr)                                   \
    do {                                                 \
        helm_status _st = (expr);                        \
        if (_st != HELM_OK) return _st;                  \
    } while (0)

#define HELM_CUDA(ctx, expr) HELM_TRY(cuda_check((ctx), (expr), #expr))

// Launch helper: counts launches and checks the launch status.
#define HELM_LAUNCH_CHECK(ctx, name)                                   \
    do {                                                               \
        (ctx)->launches++;                                             \
        cudaError_t _e = cudaGetLastError();                           \
        if (_e != cudaSuccess) return cuda_check((ctx), _e, name);     \
    } while (0)

// ----------------------------------------------------------------- kernels (launchers)

helm_status launch_stencil(helm_grid g, int prec, const void* u, void* y, int nrhs, cudaStream_t s);
helm_status launch_k2(helm_grid g);
helm_status launch_max_real(helm_ctx ctx, const c128* v, long long n, double* host_out);

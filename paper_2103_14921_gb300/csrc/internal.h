// Internal declarations of the Helmholtz ORAS-GMRES library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <algorithm>
#include <memory>
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

// Event-pair timing of instrumented kernel families (helm_profile_*).
struct ProfRecord {
    cudaEvent_t a, b;
    double bytes;
    int family;
};
struct Profiler {
    bool on = false;
    std::vector<ProfRecord>* capture = nullptr;   // set while a CUDA graph is captured: records go here
    std::vector<std::string> only;   // when non-empty, only these families are recorded
    std::vector<std::string> names;
    std::vector<ProfRecord> pending;
    std::vector<cudaEvent_t> pool;
    std::vector<uint64_t> launches;
    std::vector<double> ms, bytes;
};

struct Server;   // serve.cu

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
    Profiler prof;
    Server* server = nullptr;
    int tc_stages = 0;         // tuning: pipeline stages of the tensor-core sweep (0 = automatic)
    int coarse_coop = 1;       // tuning: one cooperative launch for the complex64 coarse sweeps
    int use_graphs = 1;        // tuning: Krylov iterations replayed from captured CUDA graphs
    int tc_flow = 1;           // tuning: tensor-core sweeps as one persistent launch with a work queue
    int stencil_march = 1;     // tuning: complex64 stencils (16-column chunks) walk z-planes (in-plane terms reused)
    int stencil_planes = 0;    // tuning: output planes per z-march block (0 = chosen per grid)
    long long flow_wait_us = 2000000;   // tuning: bound of the persistent sweep's queue-slot wait (microseconds)
    int tc_factor = 1;         // tuning: tensor-core blocked Gauss-Jordan for complex64 tensor-core factor sets
    int block_gj = 1;          // tuning: block-pivot Gauss-Jordan on the CUDA cores for the other factor sets
    uint64_t factor_fallbacks = 0;   // sets refactored with full pivoting after a tiny block pivot
    uint64_t graph_gen = 1;    // bumped when a setting that captured graphs depend on changes
    cudaStream_t cap_stream = nullptr;   // private stream graphs are captured on (the context's may be
                                         // the legacy default stream, which cannot be captured)
    ~helm_ctx_s() {
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

// Bracket one launch of an instrumented family with events on the context's stream.
int prof_begin(helm_ctx ctx, const char* family);   // returns a token (-1 when profiling is off)
void prof_end(helm_ctx ctx, int token, double bytes);
void prof_drain(helm_ctx ctx);                       // fold completed records into the totals
// Records captured into a CUDA graph (external event nodes): after each replay has completed,
// prof_harvest adds their times to the totals; prof_release returns their events.
void prof_harvest(helm_ctx ctx, const std::vector<ProfRecord>& recs);
void prof_reserve(helm_ctx ctx, size_t n);   // pool at least n events (none are created during a capture)
void prof_release(helm_ctx ctx, std::vector<ProfRecord>& recs);

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
    bool k2_real = false;      // wave speed real everywhere (no attenuation)
    // adaptive weights (weight_bins > 0): per-bin product-form weights and each node's bin
    int nbins = 0;
    StencilW* wtab = nullptr;  // device [nbins]
    unsigned char* wbin = nullptr;   // device [N]
    std::vector<double> hedges, hweights;   // host copies: edges [nbins + 1], weights [nbins][7]
    int refs = 0;              // ORAS handles built on this grid
    bool destroy_pending = false;   // helm_destroy_grid called while ORAS handles were alive
};

// One box of a plane-by-plane block LU (a fine subdomain, or the whole coarse grid).
struct BoxInfo {
    int lo[3], dims[3];        // origin and extent in (x, y, z)
    int core_lo[3], core_hi[3];
    int m;                     // dims[0] * dims[1]: unknowns per z-plane
    int ld;                    // row pitch of the stored S_k^{-1} (complex entries)
    int plane0;                // global index of plane 0 in the factor storage
    int pad;
    long long loc_off;         // index of the box's first node in the concatenated local vectors
    long long fac_off;         // index of the first entry of S_0^{-1} in the factor storage
    long long pstride;         // entries between consecutive planes of the box
};

// Plane-by-plane block LU of a set of boxes: the local operators as 27
// coefficients per node and the dense inverses S_k^{-1}, all resident.
struct PlaneSet {
    int prec = HELM_PREC_FP64;  // FP64 -> complex128 storage, otherwise complex64
    bool padded = false;        // every plane stored as ld x ld with ld = m_max rounded up (tensor-core layout)
    int ld = 0;                 // padded row pitch
    // tensor-core tile layout (planeset_pack_tc): plane = [row tile t][chunk c][row i < 128][128 bytes],
    // the bytes [128 c, 128 c + 128) of row 128 t + i, so each 128-row x 128-byte operand tile is
    // one contiguous 16 KB block
    bool packed = false;
    int pk_tiles = 0, pk_chunks = 0;
    bool coef_only = false;     // local operator coefficients without factor storage (the coarse E of the
                                // inexact coarse solve, which is applied, not factorised)
    int nplanes = 0;            // total planes over all boxes
    int nbox = 0, m_max = 0, bz_max = 0;
    long long nloc = 0;         // total local nodes
    size_t fac_entries = 0;     // total factor entries
    std::vector<BoxInfo> hbox;
    BoxInfo* dbox = nullptr;
    void* coef = nullptr;       // [nloc][27] in the set's precision
    void* G = nullptr;          // factors, per box: bz planes of m x m row-major
    // bytes of one stored factor entry, and of one coefficient / local-vector entry
    size_t esize() const { return prec == HELM_PREC_FP64 ? sizeof(c128) : (prec == HELM_PREC_BF16 ? 4 : sizeof(c64)); }
    size_t cesize() const { return prec == HELM_PREC_FP64 ? sizeof(c128) : sizeof(c64); }
};

struct KrylovEngine;

// Work queue of the persistent tensor-core sweep (sweep_tc.cu), sized by the box geometry alone.
// One allocation: ctl (head, tail, one counter per box) and flag (one per pushed slot: the slot's packed
// item once published, 0 before) first, reset before every launch, then the initial items (packed).
struct TcFlow {
    void* mem = nullptr;
    size_t bytes = 0;
    size_t reset_bytes = 0;
    int* ctl = nullptr;
    int* flag = nullptr;
    int* init = nullptr;
    int ninit = 0, total = 0;
    int tpn = 128;   // plane nodes per operand-preparation item
};

struct helm_oras_s {
    helm_grid g = nullptr;
    helm_oras_desc d{};
    PlaneSet fine, coarse;
    PlaneSet coarse32;          // complex64 copy of the FP64 coarse factors (mixed-precision apply)
    int cdims[3] = {0, 0, 0};
    long long nc = 0;
    int* owner = nullptr;       // device: per axis owner part index, [nx + ny + nz]
    int* cuts = nullptr;        // device: per axis cut positions, [px+1 + py+1 + pz+1]
    double setup_s = 0;
    // apply scratch (grown on demand)
    int cap_nrhs = 0;
    void* loc = nullptr;        // local vectors, fine factor precision
    void* rbuf = nullptr;       // sweep right-hand sides, nbox * m_max * nrhs
    c128* cvec = nullptr;       // coarse vector
    c128* crbuf = nullptr;
    void* qf = nullptr;         // fine coarse-correction vector (work precision)
    void* tf = nullptr;         // fine residual v - A q (work precision)
    int cap_wp = -1;
    size_t scratch_bytes = 0;
    void* tcb = nullptr;        // tensor-core sweep operand B^T, [nbox][tc_npad][2 ld] fp32
    void* lb = nullptr;         // restricted right-hand sides of the tensor-core sweeps (same layout as loc)
    int tc_npad = 0;
    TcFlow flow;                // persistent tensor-core sweep queue (fine set with the tile layout)
    int* dev_err = nullptr;     // device error code of bounded waits (0 = none)
    uint64_t scratch_gen = 0;   // bumped whenever the apply scratch is reallocated
    // inexact coarse solve (coarse_iters > 0): one-level ORAS on the coarse grid and inner GMRES
    PlaneSet cdd, cdd32;        // coarse local factors over the coarse boxes (FP64; complex64 copy when mixed)
    int* cowner = nullptr;      // device: coarse owner part per axis, [cx + cy + cz]
    void* Ecoef32 = nullptr;    // complex64 copy of E's 27 coefficients per coarse node (mixed precision)
    void* cy = nullptr;         // inner solution, coarse vector (work precision)
    void* cloc = nullptr;       // coarse local vectors (coarse factor precision)
    void* crb = nullptr;        // coarse sweep buffer
    struct InnerKrylov* inner = nullptr;   // inner GMRES workspace (krylov.cu)
    // Krylov workspace of the last gmres_solve, kept with its captured iteration graphs
    KrylovEngine* kcache = nullptr;
    int kc_slots = 0, kc_restart = 0, kc_flex = 0, kc_prec = -1;
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
// y = b - A u (same precisions as launch_stencil)
helm_status launch_stencil_sub(helm_grid g, int prec, const void* u, const void* b, void* y, int nrhs, cudaStream_t s);
// out = M^{-1} v on vectors of precision wp (HELM_PREC_FP64: complex128, HELM_PREC_FP32: complex64), device pointers.
helm_status oras_apply_wp(helm_oras o, int wp, const void* v, void* out, int nrhs);
bool is_device_pointer(const void* p);
helm_status launch_k2(helm_grid g);
helm_status launch_max_real(helm_ctx ctx, const c128* v, long long n, double* host_out);

// plane-by-plane block LU (planelu.cu)
helm_status planeset_alloc(helm_ctx ctx, PlaneSet& P);
void planeset_free(helm_ctx ctx, PlaneSet& P);
helm_status planeset_factor(helm_ctx ctx, PlaneSet& P, int* singular);
// tensor-core blocked Gauss-Jordan of a padded complex64 set (planelu_tc.cu); *weak: a block pivot was tiny
helm_status planeset_factor_tc(helm_ctx ctx, PlaneSet& P, int* singular, int* weak);
helm_status planeset_to_bf16(helm_ctx ctx, PlaneSet& P);
helm_status planeset_pack_tc(helm_ctx ctx, PlaneSet& P);   // row-major padded planes -> tile layout
// plane slot of a padded set, in stored entries: room for ld x ld row-major or the tile layout
inline long long padded_pstride(int ld) { return (long long)((ld + 127) / 128) * 128 * ((ld + 31) / 32 * 32); }
// err: device error flag of bounded waits; with it a one-box complex64 set may use the
// cooperative single-launch sweeps (sweep_coop.cu), whose rbuf needs m * nrhs + 1 entries
helm_status planeset_solve(helm_ctx ctx, const PlaneSet& P, void* loc, void* rbuf, int nrhs, cudaStream_t st,
                           int* err = nullptr);
helm_status planeset_solve_coop(helm_ctx ctx, const PlaneSet& P, c64* loc, c64* rbuf, int nrhs, cudaStream_t st,
                                int* err, bool* done);
// tensor-core sweeps (sweep_tc.cu), complex64 local vectors, padded factor layout
int tc_npad(int nrhs);
// lb: the restricted right-hand sides b (read by the forward sweep); loc receives y, then x.
// flow (may be null): the queue of the persistent single-launch sweep, used when the context allows it.
helm_status planeset_solve_tc(helm_ctx ctx, const PlaneSet& P, const void* lb, void* loc, void* bt, int npad, int nrhs,
                              cudaStream_t st, int* err, const TcFlow* flow = nullptr);
// tpn: plane nodes per preparation item (tc_flow_tpn(nrhs) for the column count the queue is made for)
helm_status tc_flow_alloc(helm_ctx ctx, const PlaneSet& P, TcFlow& F, int tpn);
int tc_flow_tpn(int nrhs);
void tc_flow_free(helm_ctx ctx, TcFlow& F);
// Device bytes an ORAS handle with this description will hold (factors, local operators,
// coarse level) plus its apply scratch for nrhs columns; an estimate for admission control.
size_t oras_estimate_bytes(const helm_grid_desc& g, const helm_oras_desc& d, int nrhs);
// HELM_ETIMEOUT if a bounded device wait of this handle's kernels gave up
helm_status oras_check_device_error(helm_oras o);

// Per-column state of a batched (F)GMRES (FP64 quantities).
struct RhsState {
    double bnorm;
    int active;       // column still iterating this cycle
    int steps;        // Krylov steps taken in this cycle
    int iters;        // total iterations
    int done;         // finished (converged, out of iterations, or an empty slot)
    double est;       // last residual estimate (relative)
    double tol;
    int maxit;
};

// Batched (F)GMRES over a fixed number of columns (krylov.cu).  Columns are started with
// begin_columns, advanced one restart cycle at a time, and retired; a column's arithmetic
// does not depend on which other columns are active.
struct KrylovEngine {
    virtual ~KrylovEngine() {}
    virtual c128* B() = 0;   // [N][S] right-hand sides
    virtual c128* X() = 0;   // [N][S] solutions
    virtual int slots() const = 0;
    virtual const RhsState& state(int c) const = 0;
    virtual double true_rel(int c) const = 0;
    virtual size_t bytes() const = 0;
    // warm: X() holds the initial guess of every column (all S columns must be listed): r = b - A x
    virtual helm_status begin_columns(const int* cols, int n, const double* tol, const int* maxit,
                                      bool warm = false) = 0;
    virtual void retire(int c) = 0;
    virtual helm_status push_state() = 0;
    virtual helm_status cycle(bool* any_left) = 0;
    // point the engine at other caller-owned b / x buffers (engines made with external buffers)
    virtual void rebind(c128* B_ext, c128* X_ext) = 0;
    // replay each iteration j from a CUDA graph captured on its second use
    virtual void enable_graphs(bool on) = 0;
};
KrylovEngine* make_krylov_engine(helm_oras o, int S, int restart, bool flexible, int basis_prec, c128* B_ext,
                                 c128* X_ext, helm_status* rc);

// Inexact coarse solve (oras.cu, krylov.cu): y ~ E^{-1} c by o->d.coarse_iters right-preconditioned GMRES
// iterations with one-level ORAS on the coarse grid, all on the device (no host synchronisation), vectors
// [nc][nrhs] in the work precision wp.
helm_status coarse_dd_apply(helm_oras o, int wp, const void* v, void* out, int nrhs);   // M_c^{-1} v
helm_status coarse_E_apply(helm_oras o, int wp, const void* x, void* y, int nrhs);      // y = E x
helm_status inner_alloc(helm_oras o, int wp, int nrhs);
void inner_free(helm_oras o);
helm_status inner_solve(helm_oras o, int wp, const void* c, void* y, int nrhs);

/*
 * helm.h -- C ABI of the GB300 ORAS-GMRES solver for the 27-point
 * finite-difference Helmholtz problem.
 *
 * The method (Dolean, Jolivet, Tournier, Combe, Operto, Riffo, EAGE 2021,
 * arXiv 2103.14921):
 *   - Eq. (eqh)/(eq1): (Delta + k^2(x)) u = b, k = omega / c(x), c complex in
 *     viscous media, discretised as A u = b with absorbing layers on the
 *     vertical and bottom faces and a homogeneous Dirichlet top.
 *   - The 27-point mixed-grid stencil (rotated-coordinate Laplacians plus a
 *     consistent mass term, weights fitted on numerical dispersion).
 *   - Eq. (2lvl): M^{-1} = M1^{-1}(I - A Q) + Q, Q = Z E^{-1} Z^T, E = Z^T A Z.
 *   - Eq. (oras): M1^{-1} = sum_i R_i^T D_i A_i^{-1} R_i with absorbing
 *     conditions on the subdomain interfaces.
 *   - GMRES, flexible when the preconditioner varies.
 *
 * Conventions shared by every call:
 *   - Grid vectors are complex, interleaved (re, im), point-major and
 *     right-hand-side-minor: element (i, j, k, r) of an nrhs-column vector is
 *     at offset ((k * ny + j) * nx + i) * nrhs + r.  Node (i, j, k) sits at
 *     x = i h, y = j h, depth z = (k + 1) h; the Dirichlet plane is the ghost
 *     k = -1.
 *   - "complex128" = two doubles, "complex64" = two floats.
 *   - Unless stated otherwise a pointer argument may point to device memory
 *     or to host memory (pinned or pageable); host buffers are staged through
 *     device memory inside the call.  Caller-owned buffers are never retained
 *     after a call returns.
 *   - All work is ordered on the CUDA stream given to helm_create.  Calls are
 *     synchronous with respect to the host unless stated otherwise.
 *   - Errors are returned as status codes; nothing aborts, throws or traps.
 *     helm_last_error() gives the message of the last failure on a context.
 *   - Handles are owned by the library until the matching destroy call.  A
 *     grid must outlive the ORAS handles built on it; a context must outlive
 *     its grids.
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int helm_status;
#define HELM_OK          0
#define HELM_EINVAL      1  /* invalid argument or unsupported combination            */
#define HELM_ENOMEM      2  /* device allocation failed or HBM budget exceeded        */
#define HELM_ENOTCONV    3  /* maxit reached; best iterate and residual still written */
#define HELM_ESINGULAR   4  /* zero pivot in a plane Schur-complement inverse         */
#define HELM_ENONFINITE  5  /* NaN/Inf in a right-hand side or a residual             */
#define HELM_ETIMEOUT    6  /* a bounded device wait expired                          */
#define HELM_EBUSY       7  /* resource in use (request queue full)                   */
#define HELM_ECUDA       8  /* CUDA runtime error                                     */
#define HELM_ENOTFOUND   9  /* unknown ticket or index out of range                  */

typedef struct helm_ctx_s*  helm_ctx;
typedef struct helm_grid_s* helm_grid;
typedef struct helm_oras_s* helm_oras;

/* Top boundary: the paper's homogeneous Dirichlet condition, or an absorbing
 * layer (used to compare against whole-space closed-form solutions). */
#define HELM_TOP_DIRICHLET 0
#define HELM_TOP_PML       1

/* Arithmetic of a kernel family.  FP64: complex128 throughout.  FP32:
 * complex64 storage and arithmetic.  TF32: complex64 storage, plane products
 * on the tensor cores in TF32 with FP32 accumulation.  TF32X3: the same with
 * the three-product split (hi*hi + hi*lo + lo*hi) for near-FP32 accuracy. */
#define HELM_PREC_FP64   0
#define HELM_PREC_FP32   1
#define HELM_PREC_TF32   2
#define HELM_PREC_TF32X3 3
#define HELM_PREC_BF16   4   /* local factors stored as bfloat16 pairs, sweeps on the tensor cores (kind::f16)
                                with FP32 accumulation; factorised in FP32 first */

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, ordering all work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * `hbm_budget_bytes` caps the device memory the context may allocate
 * (0 = no cap).  Returns HELM_ECUDA if the device cannot be used. */
helm_status helm_create(helm_ctx* out, int device, void* cuda_stream, size_t hbm_budget_bytes);
void        helm_destroy(helm_ctx ctx);
/* Message of the last failure on this context ("" if none).  Valid until the
 * next call on the context.  ctx may be NULL (then: last failure of helm_create). */
const char* helm_last_error(helm_ctx ctx);
/* Bytes of device memory currently held by the context. */
size_t      helm_bytes_in_use(helm_ctx ctx);
/* Number of CUDA kernel launches the library has issued on this context. */
uint64_t    helm_launch_count(helm_ctx ctx);

/* Per-kernel-family timing with CUDA events recorded on the context's stream
 * around every launch of the instrumented families ("stencil", "stencil64", "sweep_flow" (the persistent
 * tensor-core sweep), "sweep_gemm_tc", "sweep_prep", "sweep_gemv", "coarse_sweep", "coarse_prep",
 * "coarse_restrict", "coarse_prolong", "coarse_inner", "oras_transfer", "gj_panel", "gj_update",
 * "gj_diag", "gj_panel_tc", "gj_update_tc" (the panel steps and the tensor-core rank-128 update of the plane
 * factorisation), "arnoldi",
 * "arnoldi_reorth", "krylov_misc").  on = 1 enables (and
 * clears the counters), 0 disables.  helm_profile_query synchronizes the
 * stream and returns, for family `name`, the launches recorded, their summed
 * device time in milliseconds and their summed algorithmic bytes (the data a
 * launch must move at least once, as stated in each kernel's description).
 * Returns HELM_ENOTFOUND for a family with no recorded launch. */
helm_status helm_profile_enable(helm_ctx ctx, int on);
/* Restrict recording to a comma-separated list of families (NULL or "" = all), so that
 * the events bracket only the kernels of interest inside a timed region. */
helm_status helm_profile_select(helm_ctx ctx, const char* families);
helm_status helm_profile_query(helm_ctx ctx, const char* name, uint64_t* launches, double* ms, double* bytes);

/* Tuning knobs (read by the autotuner).  HELM_TUNE_TC_STAGES: pipeline depth of the
 * tensor-core plane sweep, 2..5 (0 = automatic: 4, or 3 above 64 right-hand sides).
 * HELM_TUNE_COARSE_COOP: 1 (default) runs both sweeps of a complex64 coarse problem in one
 * cooperative launch when the device supports it and a coarse plane fits in shared memory;
 * 0 uses three launches per plane.  HELM_TUNE_GRAPHS: 1 (default) keeps the Krylov workspace
 * of the last gmres_solve on its ORAS handle (freed by oras_destroy, by a gmres_solve with
 * another slot count, restart, method or basis precision, or by setting this knob to 0) and
 * replays each Krylov iteration from a CUDA graph captured on its second use; 0 launches every
 * kernel from the host and frees the workspace after each call.  HELM_TUNE_TC_FLOW: 1 (default)
 * runs both tensor-core sweeps of every box as one persistent launch that takes its work (row
 * tiles of the products, tiles of the operand preparation) from a device queue, each box's next
 * step queued as soon as its current one completes (an even number of right-hand sides and
 * 16-byte aligned vectors; otherwise, and with 0, two launches per plane step).  Both give
 * bit-identical results.  HELM_TUNE_STENCIL_MARCH: 1 (default) applies complex64 stencils whose column
 * count is a multiple of 16, with constant weights, by walking z-planes (the in-plane terms of a plane are
 * formed once and reused by the three output planes it touches; blocks wholly inside the interior take the
 * class-sum form, the others the product form); 2 the same with the blocks of one absorbing layer (one
 * stretched axis) in product forms specialised to that axis; 0 uses the per-node kernel.  All agree to
 * FP32 rounding.  Returns HELM_EINVAL for an unknown key or value out of range. */
#define HELM_TUNE_TC_STAGES 1
#define HELM_TUNE_COARSE_COOP 2
#define HELM_TUNE_GRAPHS 3
#define HELM_TUNE_TC_FLOW 4
#define HELM_TUNE_STENCIL_MARCH 5
/* HELM_TUNE_FLOW_WAIT_US: how long (microseconds) a CTA of the persistent tensor-core sweep waits for its
 * queue slot to be published before it gives up and the call returns HELM_ETIMEOUT (default 2,000,000).
 * 0 makes any wait give up at once: a test uses it to exercise the HELM_ETIMEOUT path (the launch then
 * drains, frees its TMEM and returns; the handle stays usable once the knob is restored).  Not captured
 * into CUDA graphs: it only affects launches made after it is set. */
#define HELM_TUNE_FLOW_WAIT_US 6
/* HELM_TUNE_TC_FACTOR: 1 (default) factors the complex64 local planes of HELM_PREC_TF32 / HELM_PREC_BF16
 * sets by blocked Gauss-Jordan on the tensor cores (128-column panels; block pivots with partial pivoting
 * inside each 128 x 128 diagonal block; rank-128 updates as tcgen05 products with the three-product TF32
 * split hi*hi + hi*lo + lo*hi and FP32 accumulation); a block pivot below 1e-6 of its block's largest entry
 * makes oras_factor factor the set again with full partial pivoting.  0 always uses the fully pivoted
 * Gauss-Jordan on the CUDA cores.  Read by oras_factor. */
#define HELM_TUNE_TC_FACTOR 7
/* HELM_TUNE_BLOCK_GJ: 1 (default) factors the other plane sets (FP64 and FP32 local factors, the FP64
 * coarse problem) by the same blocked Gauss-Jordan with block pivots on the CUDA cores (64-column panels for
 * complex64, 32 for complex128; the rank-NB updates spread over every SM), falling back to full partial pivoting after a tiny block
 * pivot; 0 always uses the fully pivoted elimination.  Read by oras_factor. */
#define HELM_TUNE_BLOCK_GJ 8
/* HELM_TUNE_STENCIL_PLANES: output planes per block of the z-marching stencil (HELM_TUNE_STENCIL_MARCH);
 * 0 (default) picks, per grid, the longest walks (at most 64 planes, at least 8) that still give every
 * resident block slot two blocks or more; else 4..128.  The split decides which blocks
 * lie wholly inside the interior (and take the cheaper class-sum form), so results differ with it by FP32
 * rounding only.  Captured graphs are re-captured after a change. */
#define HELM_TUNE_STENCIL_PLANES 9
helm_status helm_set_tuning(helm_ctx ctx, int key, int value);

/* ------------------------------------------------------------ grid / model */

typedef struct {
    int    nx, ny, nz;    /* unknown nodes per axis (each >= 2)                              */
    double h;             /* grid spacing, metres                                             */
    double freq_hz;       /* frequency; omega = 2 pi freq_hz                                  */
    int    npml;          /* absorbing-layer thickness in nodes (0 = none)                    */
    double pml_R;         /* nominal layer reflection; gamma0 = 3 c_ref/(2 L) ln(1/R)         */
    int    top_bc;        /* HELM_TOP_DIRICHLET or HELM_TOP_PML                               */
    double weights[7];    /* w1, w2, w3, wm1, wm2, wm3, wm4 of the mixed-grid stencil;
                             w1+w2+w3 = 1 and wm1+6wm2+12wm3+8wm4 = 1 (checked, 1e-9)       */
    int    weight_bins;   /* 0: every row uses weights[] (zero-initialise to keep this);
                             1..64: adaptive weights matched to the local wave speed (the paper's
                             adaptive coefficients): the points-per-wavelength range of the model,
                             G = Re c / (f h) from its minimum to its maximum, is cut into this many
                             geometric bins, each fitted as helm_fit_weights does over its own G
                             interval, and each row uses the bin holding its own G (needs G >= 2) */
} helm_grid_desc;

/* Fit the stencil weights by least squares on the normalised phase-velocity
 * error 1 - sqrt(-L(kappa)/M(kappa))/|kappa| of plane waves over G_min..G_max
 * grid points per wavelength and directions in one octant, all weights kept
 * non-negative (the paper fits the weights by least squares against the
 * stencil's phase and direction errors, section 2).  Host-only; writes weights_out[7]. */
helm_status helm_fit_weights(double G_min, double G_max, double weights_out[7]);

/* Set up one problem: copies the wave speed c (complex128 [nz][ny][nx],
 * device or host) and builds k^2 = (omega/c)^2 and the stretched 1-D
 * difference tables of the absorbing layers (separable PML, xi = 1 + i
 * gamma(d)/omega, gamma = gamma0 (d/L)^2, c_ref = max Re c).  Eq. (eqh). */
helm_status helm_setup_grid(helm_ctx ctx, const helm_grid_desc* desc, const void* c, helm_grid* out);
void        helm_destroy_grid(helm_grid g);

/* The adaptive weights of a grid built with weight_bins > 0: *nbins, and when the arrays are not
 * NULL the bin edges in points per wavelength (edges[nbins + 1]: edge b = G_min ratio^b) and each
 * bin's weights (table[nbins * 7], w1..wm4).  *nbins = 0 for constant weights.  Host memory. */
helm_status helm_grid_row_weights(helm_grid g, int* nbins, double* edges, double* table);

/* y = A u (Eq. eq1), matrix-free 27-point stencil, nrhs columns.
 * prec = HELM_PREC_FP64: u, y complex128; prec = HELM_PREC_FP32: complex64.
 * u and y must not overlap.  Device pointers only. */
helm_status helm_apply(helm_grid g, int prec, const void* u, void* y, int nrhs);

/* ----------------------------------------------------------- ORAS factors */

typedef struct {
    int px, py, pz;       /* boxes per axis; axis a is cut at floor(t n_a / p_a)            */
    int overlap;          /* nodes added on every interior side of each core (>= 1)         */
    int coarse_ratio;     /* 0 = one level (Eq. oras); r >= 2 = trilinear coarse grid (Eq. 2lvl) */
    int interface_bc;     /* 0 = absorbing (ORAS, rho = exp(i k_p h) folding); 1 = Dirichlet (RAS) */
    int factor_prec;      /* HELM_PREC_FP64, _FP32, _TF32 or _BF16 for the fine local factors
                             (_TF32X3 is rejected: not available).  The coarse factors are always computed
                             in FP64; with non-FP64 fine factors they are applied from a complex64
                             copy, with FP64 fine factors in FP64                                   */
    int coarse_iters;     /* 0 = the coarse problem E solved exactly (plane LU of the whole coarse grid);
                             k >= 1 = solved as in the paper by k GMRES iterations (x0 = 0, no restart)
                             preconditioned by one-level ORAS on the coarse grid over the same
                             spatial partition (the paper uses 10).  The preconditioner then depends
                             on its input nonlinearly: solve with flexible GMRES.  Zero-initialise
                             the struct to keep the exact coarse solve                              */
    int coarse_overlap;   /* coarse layers added on every interior side of each coarse core
                             (coarse_iters >= 1 only)                                              */
} helm_oras_desc;

/* Build the ORAS preconditioner: box decomposition, local operators A_i with
 * absorbing interface folding, and for every box the plane-by-plane block LU
 * S_0 = D_0, S_k = D_k - L_k S_{k-1}^{-1} U_{k-1} with the dense complex
 * inverses S_k^{-1} kept resident; with coarse_ratio > 0 also Z, E = Z^T A Z
 * and E's plane factors in FP64.  Eq. (2lvl), Eq. (oras).
 * Returns HELM_ESINGULAR if a pivot vanishes, HELM_ENOMEM past the budget. */
helm_status oras_factor(helm_grid g, const helm_oras_desc* desc, helm_oras* out);
void        oras_destroy(helm_oras o);

/* Estimated device bytes an ORAS handle with this description holds (factors, local
 * operators, coarse level, set-up probes) plus its apply scratch for nrhs columns -- the
 * figure the serving loop admits against.  Host-only, no device work. */
helm_status oras_estimate_bytes_c(const helm_grid_desc* grid, const helm_oras_desc* desc, int nrhs, size_t* bytes);

/* out = M^{-1} v (Eq. 2lvl, or Eq. oras without a coarse level).
 * v, out: complex128, nrhs columns, device pointers. */
helm_status oras_apply(helm_oras o, const void* v, void* out, int nrhs);

/* out = M^{-1} v exactly as oras_apply computes it, but without allocating
 * any device memory inside the call.  No counterpart in the paper: it is
 * there for callers that cannot let a library call cudaMalloc/cudaFree --
 * an application that has reserved the GPU's memory in its own pool, or a
 * serving loop that must not pay the device-wide synchronisation those calls
 * imply.  The working vectors live in one fixed 8 MiB device array inside the
 * library (held by every GPU that loads it until the process exits); a
 * problem whose working vectors do not fit is rejected with HELM_EINVAL and a
 * message giving the size it would need.  The array's device address is
 * looked up on the first call on each device, so make that first call before
 * any stream capture.  All calls share the array: calls whose GPU work
 * overlaps (other streams or threads) race on it.  While the call runs the
 * handle's working vectors point into the array, so no other call may use
 * the same handle (from another thread) until it returns.  A bounded device
 * wait that gives up returns HELM_ETIMEOUT, as oras_apply does.  v, out:
 * complex128, nrhs columns, device pointers. */
helm_status oras_apply_noalloc(helm_oras o, const void* v, void* out, int nrhs);

/* Sizes of the decomposition: number of boxes, and for box `box` its origin
 * lo[3] and extent dims[3] in (x, y, z) order.  box < 0 fills only nboxes. */
helm_status oras_box_info(helm_oras o, int box, int* nboxes, int lo[3], int dims[3]);

/* Copy S_k^{-1} of box `box`, plane `plane` to `out` as a complex128 m x m
 * row-major matrix (m = dims[0]*dims[1], in-plane index j*dims[0]+i).
 * Device or host pointer. */
helm_status oras_plane_inverse(helm_oras o, int box, int plane, void* out);

/* Seconds spent in oras_factor (device time of the setup kernels). */
double      oras_setup_seconds(helm_oras o);

/* ---------------------------------------------------------------- Krylov */

typedef struct {
    double tol;           /* stop when ||b - A x||_2 / ||b||_2 <= tol (per column)           */
    int    restart;       /* Krylov dimension per cycle (1..200)                              */
    int    maxit;         /* total iteration cap per column                                   */
    int    flexible;      /* 1 = FGMRES (keeps Z_j = M^{-1} v_j), 0 = right-preconditioned GMRES */
    int    basis_prec;    /* HELM_PREC_FP64 (complex128 basis) or HELM_PREC_FP32 (complex64)  */
    int    use_x0;        /* 0: x0 = 0; 1: x holds the initial guess on entry (a warm start, e.g.
                             the solution at a neighbouring frequency of a sweep); columns whose
                             b is zero still return x = 0, and a column whose guess already has an
                             FP64 relative residual <= tol returns it unchanged with 0 iterations.
                             A NaN/Inf in x gives HELM_ENONFINITE.  gmres_solve only (helm_submit
                             rejects it with HELM_EINVAL)                                        */
} helm_gmres_desc;

typedef struct {
    int    iterations;    /* Krylov iterations taken                                          */
    int    converged;     /* 1 if the true relative residual <= tol                          */
    double true_relres;   /* FP64 ||b - A x|| / ||b|| at exit                                 */
    double est_relres;    /* last Givens residual estimate                                    */
} helm_rhs_stats;

/* Solve A x = b for nrhs columns with right-preconditioned (F)GMRES(m),
 * x0 = 0 (or the caller's x with use_x0), independent Krylov spaces per column, CGS2 Arnoldi with FP64
 * accumulation, complex Givens rotations, FP64 true residual at every cycle
 * end (restart if above tol).  b, x complex128 [N][nrhs]; device or host.
 * stats (host array of nrhs, may be NULL) receives per-column results.
 * Returns HELM_ENOTCONV (x still written) if some column missed tol. */
helm_status gmres_solve(helm_oras o, const void* b, void* x, int nrhs, const helm_gmres_desc* desc,
                        helm_rhs_stats* stats);

/* -------------------------------------------------------------- frequency sweeps
 *
 * Several frequencies of one model and one set of sources (the paper's forward problem is solved for many
 * frequencies and sources per model, section 1).  For each frequency f_i the driver builds the grid
 * (helm_setup_grid with desc.grid and freq_hz = freqs[i]) and the ORAS factors (oras_factor), solves
 * (gmres_solve) and frees the factors again, so that at most two factor sets are resident.
 *   warm = 1: frequency i > 0 starts from the solution at frequency i - 1 (use_x0; the solution of a
 *             neighbouring frequency is close when the frequencies are close);
 *   overlap = 1: the factors of frequency i + 1 are built on a second stream by a second host thread
 *             (with a context of its own, created and destroyed by the call) while frequency i is
 *             solved; 0 runs everything in order on ctx's stream.  Both give bit-identical x.
 * c: wave speed complex128 [nz][ny][nx] (device or host), read once per frequency.  b: complex128
 * [N][nrhs], the same right-hand sides at every frequency; x: complex128 [nfreq][N][nrhs]; b and x both
 * device or both host.  stats (host, may be NULL): [nfreq][nrhs].  setup_s (host, may be NULL): [nfreq],
 * the wall time of each frequency's grid set-up and factorisation.  desc.gmres.use_x0 is ignored.
 * Returns the first error (later frequencies are then not solved), else HELM_ENOTCONV if some column of
 * some frequency missed tol (every frequency is still solved), else HELM_OK.  The serving loop must not
 * be active on ctx. */
typedef struct {
    helm_grid_desc  grid;     /* freq_hz is ignored: each frequency comes from freqs */
    helm_oras_desc  oras;
    helm_gmres_desc gmres;
    int             nfreq;    /* 1 .. 64 */
    const double*   freqs;    /* host array of nfreq frequencies in Hz (> 0) */
    int             warm;     /* 0 or 1 */
    int             overlap;  /* 0 or 1 */
} helm_sweep_desc;

helm_status helm_frequency_sweep(helm_ctx ctx, const helm_sweep_desc* desc, const void* c, const void* b, void* x,
                                 int nrhs, helm_rhs_stats* stats, double* setup_s);

/* -------------------------------------------------------------- serving
 *
 * A request loop on one context (the serving pattern: the paper's
 * forward problem with many right-hand sides per frequency arriving over
 * time).  A worker thread owns the context's stream: factors are built on
 * first use -- by a second host thread on a stream (and context) of its own,
 * so that the batches already running keep cycling meanwhile; the finished
 * set joins the context -- and kept resident in a cache keyed by (model_id, grid
 * description, ORAS description, restart, flexible, basis precision), and
 * evicted least-recently-used when idle and the HBM budget needs the room.
 * Requests that share factors are batched: each right-hand side takes one
 * column slot of the factor set's batch, new requests join at the next
 * restart-cycle boundary while others are running, and every column keeps
 * its own Krylov space, tolerance and iteration count, so a result does not
 * depend on which other requests share the batch.  A request is admitted
 * when its columns fit the free slots and its factors (if not cached) fit
 * the budget; one that cannot fit even on an idle server fails with
 * HELM_ENOMEM.  While serving is active no other call may use the context.
 */
typedef struct {
    uint64_t        model_id;  /* caller's identifier of the wave-speed model (part of the cache key) */
    helm_grid_desc  grid;
    const void*     c;         /* complex128 [nz][ny][nx], host or device; read when the factors are built */
    helm_oras_desc  oras;
    helm_gmres_desc gmres;     /* tol and maxit per request; restart, flexible, basis_prec key the batch */
    int             nrhs;      /* 1 .. slots_per_batch */
    const void*     b;         /* complex128 [N][nrhs], host or device; read when the request is admitted */
    void*           x;         /* complex128 [N][nrhs], host or device; written before poll reports done */
} helm_request;

typedef struct {
    int    done;               /* 1 once x is written (or the request failed)                  */
    int    status;             /* HELM_OK, HELM_ENOTCONV, or the error that ended the request   */
    int    iterations_max;     /* largest iteration count over the request's columns            */
    double true_relres_max;    /* largest FP64 true relative residual over its columns          */
    double queue_ms;           /* submit -> admitted into a batch                               */
    double latency_ms;         /* submit -> done                                                */
    int    factors_reused;     /* 1 if the factors came from the cache                          */
} helm_request_stats;

/* Start the worker with `slots_per_batch` columns per factor set (1..256). */
helm_status helm_serve_start(helm_ctx ctx, int slots_per_batch);
/* Queue a request (non-blocking).  The buffers c, b and x must stay valid
 * until helm_poll reports done.  Returns HELM_EINVAL for a malformed request. */
helm_status helm_submit(helm_ctx ctx, const helm_request* req, uint64_t* ticket);
/* Non-blocking status of a ticket; HELM_ENOTFOUND for an unknown ticket.
 * Once done is reported the ticket is forgotten. */
helm_status helm_poll(helm_ctx ctx, uint64_t ticket, int* done, helm_request_stats* stats);
/* Finish every queued and running request, then stop the worker and free
 * the cached factors. */
helm_status helm_serve_stop(helm_ctx ctx);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */

// Context, device memory accounting and problem setup (Eq. eqh: k = omega / c;
// absorbing layers on the vertical and bottom faces, Dirichlet or absorbing top).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <complex>

#include "internal.h"

static thread_local std::string g_create_error;

helm_status set_error(helm_ctx ctx, helm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->last_error = buf;
    else g_create_error = buf;
    return st;
}

helm_status cuda_check(helm_ctx ctx, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return HELM_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(ctx, HELM_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_error(ctx, HELM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

helm_status dev_alloc(helm_ctx ctx, void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) return HELM_OK;
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        return set_error(ctx, HELM_ENOMEM, "%s: %zu bytes exceed the HBM budget (%zu of %zu in use)", what, bytes,
                         ctx->in_use, ctx->budget);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(ctx, HELM_ENOMEM, "%s: cudaMalloc(%zu) failed: %s", what, bytes, cudaGetErrorString(e));
    }
    ctx->in_use += bytes;
    return HELM_OK;
}

// Stream-ordered free on the context's stream: unlike cudaFree it does not wait for the whole device, so a
// context that frees memory (the serving worker evicting a factor set, a factorisation releasing its work
// buffers) does not stall behind the kernels of another context sharing the GPU.
void dev_free(helm_ctx ctx, void* p, size_t bytes) {
    if (!p) return;
    if (cudaFreeAsync(p, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
    }
    ctx->in_use -= bytes;
}

extern "C" helm_status helm_create(helm_ctx* out, int device, void* stream, size_t budget) {
    if (!out) return set_error(nullptr, HELM_EINVAL, "helm_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return set_error(nullptr, HELM_ECUDA, "helm_create: no CUDA device (%s)", cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return set_error(nullptr, HELM_EINVAL, "helm_create: bad device %d", device);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return set_error(nullptr, HELM_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    helm_ctx c = new helm_ctx_s();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    c->budget = budget;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    *out = c;
    return HELM_OK;
}

extern "C" void helm_destroy(helm_ctx ctx) {
    if (!ctx) return;
    if (ctx->server) helm_serve_stop(ctx);
    if (ctx->children > 0) {
        ctx->destroy_pending = true;   // freed when its last grid is destroyed
        return;
    }
    delete ctx;
}

extern "C" const char* helm_last_error(helm_ctx ctx) {
    return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

extern "C" size_t helm_bytes_in_use(helm_ctx ctx) { return ctx ? ctx->in_use : 0; }

extern "C" helm_status helm_set_tuning(helm_ctx ctx, int key, int value) {
    if (!ctx) return HELM_EINVAL;
    if (key == HELM_TUNE_TC_STAGES) {
        if (value != 0 && (value < 2 || value > 5))
            return set_error(ctx, HELM_EINVAL, "helm_set_tuning: tensor-core stages must be 0 or 2..5");
        ctx->tc_stages = value;
        ctx->graph_gen++;
        return HELM_OK;
    }
    if (key == HELM_TUNE_COARSE_COOP) {
        if (value != 0 && value != 1) return set_error(ctx, HELM_EINVAL, "helm_set_tuning: coarse_coop must be 0 or 1");
        ctx->coarse_coop = value;
        ctx->graph_gen++;
        return HELM_OK;
    }
    if (key == HELM_TUNE_GRAPHS) {
        if (value != 0 && value != 1) return set_error(ctx, HELM_EINVAL, "helm_set_tuning: graphs must be 0 or 1");
        ctx->use_graphs = value;
        ctx->graph_gen++;
        return HELM_OK;
    }
    if (key == HELM_TUNE_TC_FLOW) {
        if (value != 0 && value != 1) return set_error(ctx, HELM_EINVAL, "helm_set_tuning: tc_flow must be 0 or 1");
        ctx->tc_flow = value;
        ctx->graph_gen++;
        return HELM_OK;
    }
    if (key == HELM_TUNE_STENCIL_MARCH) {
        if (value < 0 || value > 2) return set_error(ctx, HELM_EINVAL, "helm_set_tuning: stencil_march must be 0..2");
        ctx->stencil_march = value;
        ctx->graph_gen++;
        return HELM_OK;
    }
    if (key == HELM_TUNE_TC_FACTOR) {
        if (value < 0 || value > 2) return set_error(ctx, HELM_EINVAL, "helm_set_tuning: tc_factor must be 0..2");
        ctx->tc_factor = value;
        return HELM_OK;
    }
    if (key == HELM_TUNE_STENCIL_PLANES) {
        if (value != 0 && (value < 4 || value > 128))
            return set_error(ctx, HELM_EINVAL, "helm_set_tuning: stencil_planes must be 0 or 4..128");
        ctx->stencil_planes = value;
        ctx->graph_gen++;
        return HELM_OK;
    }
    if (key == HELM_TUNE_BLOCK_GJ) {
        if (value != 0 && value != 1) return set_error(ctx, HELM_EINVAL, "helm_set_tuning: block_gj must be 0 or 1");
        ctx->block_gj = value;
        return HELM_OK;
    }
    if (key == HELM_TUNE_FLOW_WAIT_US) {
        if (value < 0) return set_error(ctx, HELM_EINVAL, "helm_set_tuning: flow_wait_us must be >= 0");
        ctx->flow_wait_us = value == 0 ? 0 : value;
        return HELM_OK;
    }
    return set_error(ctx, HELM_EINVAL, "helm_set_tuning: unknown key %d", key);
}
extern "C" uint64_t helm_launch_count(helm_ctx ctx) { return ctx ? ctx->launches : 0; }

// ------------------------------------------------------------------ setup kernels

namespace {

__global__ void k2_kernel(const c128* __restrict__ c, c128* __restrict__ k2, c64* __restrict__ k2f, long long n,
                          double omega) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // (omega / c)^2 = omega^2 conj(c)^2 / |c|^4
    const c128 v = c[i];
    const double den = v.x * v.x + v.y * v.y;
    const double re = omega * v.x / den, im = -omega * v.y / den;
    const c128 r = mk<double>(re * re - im * im, 2.0 * re * im);
    k2[i] = r;
    k2f[i] = mk<float>((float)r.x, (float)r.y);
}

__global__ void max_real_kernel(const c128* __restrict__ v, long long n, double* out) {
    __shared__ double s[256];
    double m = -1e300;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, v[i].x);
    s[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

__global__ void min_real_kernel(const c128* __restrict__ v, long long n, double* out) {
    __shared__ double s[256];
    double m = 1e300;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmin(m, v[i].x);
    s[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] = fmin(s[threadIdx.x], s[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

// Bin of every node for the adaptive weights: the number of interior edges at or below G = Re c / (f h).
__global__ void weight_bin_kernel(const c128* __restrict__ c, long long n, double fh, const double* __restrict__ edges,
                                  int nbins, unsigned char* __restrict__ bin) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double G = c[i].x / fh;
        int b = 0;
        for (int e = 1; e < nbins; ++e) b += G >= edges[e];
        bin[i] = (unsigned char)b;
    }
}

// bad |= 1: NaN/Inf or Re c <= 0;  bad |= 2: some Im c != 0 (attenuation, complex k^2)
__global__ void finite_check_kernel(const c128* __restrict__ v, long long n, int* bad) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const c128 a = v[i];
    if (!isfinite(a.x) || !isfinite(a.y) || a.x <= 0.0) atomicOr(bad, 1);
    if (a.y != 0.0) atomicOr(bad, 2);
}

}  // namespace

helm_status launch_max_real(helm_ctx ctx, const c128* v, long long n, double* host_out) {
    const int blocks = 256;
    double* part = nullptr;
    HELM_TRY(dev_alloc(ctx, (void**)&part, blocks * sizeof(double), "max_real partials"));
    max_real_kernel<<<blocks, 256, 0, ctx->stream>>>(v, n, part);
    ctx->launches++;
    double h[blocks];
    cudaError_t e = cudaMemcpyAsync(h, part, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, part, blocks * sizeof(double));
    HELM_CUDA(ctx, e);
    double m = -1e300;
    for (int i = 0; i < blocks; ++i) m = fmax(m, h[i]);
    *host_out = m;
    return HELM_OK;
}

static helm_status launch_min_real(helm_ctx ctx, const c128* v, long long n, double* host_out) {
    const int blocks = 256;
    double* part = nullptr;
    HELM_TRY(dev_alloc(ctx, (void**)&part, blocks * sizeof(double), "min_real partials"));
    min_real_kernel<<<blocks, 256, 0, ctx->stream>>>(v, n, part);
    ctx->launches++;
    double h[blocks];
    cudaError_t e = cudaMemcpyAsync(h, part, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, part, blocks * sizeof(double));
    HELM_CUDA(ctx, e);
    double m = 1e300;
    for (int i = 0; i < blocks; ++i) m = fmin(m, h[i]);
    *host_out = m;
    return HELM_OK;
}

static StencilW product_form(const double* w, double h) {
    StencilW s;
    s.a2 = w[1] / 6.0 + w[2] / 2.0;
    s.a3 = w[2] / 4.0;
    s.m0 = w[3] + 6 * w[4] + 12 * w[5] + 8 * w[6];
    s.m1 = w[4] + 4 * w[5] + 4 * w[6];
    s.m2 = w[5] + 2 * w[6];
    s.m3 = w[6];
    s.inv_h2 = 1.0 / (h * h);
    return s;
}

// Adaptive weights: geometric bins over the model's points-per-wavelength range, one least-squares fit per
// bin over its own interval, and each node's bin.
static helm_status setup_row_weights(helm_grid g) {
    helm_ctx ctx = g->ctx;
    const int nb = g->d.weight_bins;
    const double fh = g->d.freq_hz * g->d.h;
    double cmin = 0;
    HELM_TRY(launch_min_real(ctx, g->c, g->n, &cmin));
    const double G_lo = cmin / fh, G_hi = g->c_ref / fh;
    if (!(G_lo >= 2.0))
        return set_error(ctx, HELM_EINVAL, "helm_setup_grid: adaptive weights need >= 2 points per wavelength "
                                           "(minimum here %.3g)", G_lo);
    const double ratio = pow(G_hi / G_lo, 1.0 / nb);
    g->hedges.resize(nb + 1);
    for (int b = 0; b <= nb; ++b) g->hedges[b] = G_lo * pow(ratio, (double)b);
    g->hweights.resize((size_t)nb * 7);
    std::vector<StencilW> tab(nb);
    for (int b = 0; b < nb; ++b) {
        double lo = g->hedges[b], hi = g->hedges[b + 1];
        if (!(hi > lo)) hi = lo * (1.0 + 1e-6);   // a homogeneous model: one G, fitted on a sliver around it
        if (helm_fit_weights(lo, hi, &g->hweights[(size_t)b * 7]) != HELM_OK)
            return set_error(ctx, HELM_EINVAL, "helm_setup_grid: weight fit failed for bin %d", b);
        tab[b] = product_form(&g->hweights[(size_t)b * 7], g->d.h);
    }
    g->nbins = nb;
    double* dedges = nullptr;
    HELM_TRY(dev_alloc(ctx, (void**)&g->wtab, nb * sizeof(StencilW), "adaptive weight table"));
    HELM_TRY(dev_alloc(ctx, (void**)&g->wbin, (size_t)g->n, "adaptive weight bins"));
    HELM_TRY(dev_alloc(ctx, (void**)&dedges, (nb + 1) * sizeof(double), "bin edges"));
    HELM_CUDA(ctx, cudaMemcpyAsync(g->wtab, tab.data(), nb * sizeof(StencilW), cudaMemcpyHostToDevice, ctx->stream));
    HELM_CUDA(ctx, cudaMemcpyAsync(dedges, g->hedges.data(), (nb + 1) * sizeof(double), cudaMemcpyHostToDevice,
                                   ctx->stream));
    HELM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    weight_bin_kernel<<<(unsigned)std::min<long long>((g->n + 255) / 256, 4096), 256, 0, ctx->stream>>>(
        g->c, g->n, fh, dedges, nb, g->wbin);
    ctx->launches++;
    helm_status st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "weight bins");
    dev_free(ctx, dedges, (nb + 1) * sizeof(double));
    return st;
}

extern "C" helm_status helm_grid_row_weights(helm_grid g, int* nbins, double* edges, double* table) {
    if (!g || !nbins) return HELM_EINVAL;
    *nbins = g->nbins;
    if (g->nbins && edges) memcpy(edges, g->hedges.data(), (g->nbins + 1) * sizeof(double));
    if (g->nbins && table) memcpy(table, g->hweights.data(), (size_t)g->nbins * 7 * sizeof(double));
    return HELM_OK;
}

// Stretched 1-D second-difference coefficients (cm, c0, cp) of one axis:
// xi(s) = 1 + i gamma(d(s))/omega, gamma = gamma0 (d/L)^2, d = (npml - s) h on
// the low side, (s - (n-1-npml)) h on the high side; cm = 1/(xi_i xi_{i-1/2}),
// cp = 1/(xi_i xi_{i+1/2}), c0 = -(cm + cp).
static void axis_table(int n, double h, int npml, bool low, bool high, double omega, double c_ref, double R,
                       c128* out) {
    typedef std::complex<double> C;
    const double L = npml * h;
    const double gamma0 = npml > 0 ? 1.5 * c_ref / L * log(1.0 / R) : 0.0;
    auto xi = [&](double s) {
        double d = 0.0;
        if (low && npml > 0 && s < npml) d = (npml - s) * h;
        if (high && npml > 0 && s > n - 1 - npml) d = (s - (n - 1 - npml)) * h;
        const double g = npml > 0 ? gamma0 * (d / L) * (d / L) : 0.0;
        return C(1.0, g / omega);
    };
    for (int i = 0; i < n; ++i) {
        const C xn = xi(i), xm = xi(i - 0.5), xp = xi(i + 0.5);
        const C cm = 1.0 / (xn * xm), cp = 1.0 / (xn * xp), c0 = -(cm + cp);
        out[3 * i + 0] = mk<double>(cm.real(), cm.imag());
        out[3 * i + 1] = mk<double>(c0.real(), c0.imag());
        out[3 * i + 2] = mk<double>(cp.real(), cp.imag());
    }
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

extern "C" helm_status helm_setup_grid(helm_ctx ctx, const helm_grid_desc* d, const void* c, helm_grid* out) {
    if (!ctx || !d || !c || !out) return set_error(ctx, HELM_EINVAL, "helm_setup_grid: NULL argument");
    *out = nullptr;
    if (d->nx < 2 || d->ny < 2 || d->nz < 2 || !(d->h > 0) || !(d->freq_hz > 0) || d->npml < 0 ||
        !(d->pml_R > 0 && d->pml_R < 1) || (d->top_bc != HELM_TOP_DIRICHLET && d->top_bc != HELM_TOP_PML))
        return set_error(ctx, HELM_EINVAL, "helm_setup_grid: invalid grid description");
    if (2 * d->npml >= d->nx || 2 * d->npml >= d->ny || d->npml * (d->top_bc == HELM_TOP_PML ? 2 : 1) >= d->nz)
        return set_error(ctx, HELM_EINVAL, "helm_setup_grid: absorbing layers leave no interior");
    const double* w = d->weights;
    if (fabs(w[0] + w[1] + w[2] - 1.0) > 1e-9 || fabs(w[3] + 6 * w[4] + 12 * w[5] + 8 * w[6] - 1.0) > 1e-9)
        return set_error(ctx, HELM_EINVAL, "helm_setup_grid: stencil weights do not sum to one");
    if (d->weight_bins < 0 || d->weight_bins > 64)
        return set_error(ctx, HELM_EINVAL, "helm_setup_grid: weight_bins must be 0..64");
    HELM_CUDA(ctx, cudaSetDevice(ctx->device));

    helm_grid g = new helm_grid_s();
    g->ctx = ctx;
    ctx->children++;
    g->d = *d;
    g->n = (long long)d->nx * d->ny * d->nz;
    g->omega = 2.0 * M_PI * d->freq_hz;
    g->w = product_form(w, d->h);
    const long long n = g->n;
    const int ntab = d->nx + d->ny + d->nz;
    helm_status st = HELM_OK;
    auto fail = [&](helm_status s) { helm_destroy_grid(g); return s; };
    if ((st = dev_alloc(ctx, (void**)&g->c, n * sizeof(c128), "wave speed"))) return fail(st);
    if ((st = dev_alloc(ctx, (void**)&g->k2, n * sizeof(c128), "k^2"))) return fail(st);
    if ((st = dev_alloc(ctx, (void**)&g->k2f, n * sizeof(c64), "k^2 (fp32)"))) return fail(st);
    if ((st = dev_alloc(ctx, (void**)&g->tab, 3 * ntab * sizeof(c128), "pml tables"))) return fail(st);
    if ((st = dev_alloc(ctx, (void**)&g->tabf, 3 * ntab * sizeof(c64), "pml tables (fp32)"))) return fail(st);
    cudaMemcpyKind kind = is_device_pointer(c) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if ((st = cuda_check(ctx, cudaMemcpyAsync(g->c, c, n * sizeof(c128), kind, ctx->stream), "copy c")))
        return fail(st);
    {
        int* bad = nullptr;
        if ((st = dev_alloc(ctx, (void**)&bad, sizeof(int), "flag"))) return fail(st);
        cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream);
        finite_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(g->c, n, bad);
        ctx->launches++;
        int hbad = 0;
        cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
        st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "finite check");
        dev_free(ctx, bad, sizeof(int));
        if (st) return fail(st);
        if (hbad & 1)
            return fail(set_error(ctx, HELM_ENONFINITE, "helm_setup_grid: wave speed has NaN/Inf or Re c <= 0"));
        g->k2_real = (hbad & 2) == 0;
    }
    k2_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(g->c, g->k2, g->k2f, n, g->omega);
    ctx->launches++;
    if ((st = cuda_check(ctx, cudaGetLastError(), "k2_kernel"))) return fail(st);
    if ((st = launch_max_real(ctx, g->c, n, &g->c_ref))) return fail(st);
    if (d->weight_bins > 0 && (st = setup_row_weights(g))) return fail(st);

    g->htab.resize(3 * ntab);
    const bool top = d->top_bc == HELM_TOP_PML;
    axis_table(d->nx, d->h, d->npml, true, true, g->omega, g->c_ref, d->pml_R, &g->htab[0]);
    axis_table(d->ny, d->h, d->npml, true, true, g->omega, g->c_ref, d->pml_R, &g->htab[3 * d->nx]);
    axis_table(d->nz, d->h, d->npml, top, true, g->omega, g->c_ref, d->pml_R, &g->htab[3 * (d->nx + d->ny)]);
    std::vector<c64> hf(3 * ntab);
    for (int i = 0; i < 3 * ntab; ++i) hf[i] = mk<float>((float)g->htab[i].x, (float)g->htab[i].y);
    if ((st = cuda_check(ctx, cudaMemcpyAsync(g->tab, g->htab.data(), 3 * ntab * sizeof(c128), cudaMemcpyHostToDevice,
                                              g->ctx->stream),
                         "copy tables")))
        return fail(st);
    if ((st = cuda_check(ctx, cudaMemcpyAsync(g->tabf, hf.data(), 3 * ntab * sizeof(c64), cudaMemcpyHostToDevice,
                                              g->ctx->stream),
                         "copy tables")))
        return fail(st);
    if ((st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "grid setup"))) return fail(st);
    *out = g;
    return HELM_OK;
}

extern "C" void helm_destroy_grid(helm_grid g) {
    if (!g) return;
    if (g->refs > 0) {
        g->destroy_pending = true;   // freed when its last ORAS handle is destroyed
        return;
    }
    helm_ctx ctx = g->ctx;
    cudaStreamSynchronize(ctx->stream);
    const long long n = g->n;
    const int ntab = g->d.nx + g->d.ny + g->d.nz;
    dev_free(ctx, g->c, n * sizeof(c128));
    dev_free(ctx, g->k2, n * sizeof(c128));
    dev_free(ctx, g->k2f, n * sizeof(c64));
    dev_free(ctx, g->tab, 3 * ntab * sizeof(c128));
    dev_free(ctx, g->tabf, 3 * ntab * sizeof(c64));
    dev_free(ctx, g->wtab, g->nbins * sizeof(StencilW));
    dev_free(ctx, g->wbin, g->nbins ? (size_t)n : 0);
    delete g;
    if (--ctx->children == 0 && ctx->destroy_pending) delete ctx;
}

extern "C" helm_status helm_apply(helm_grid g, int prec, const void* u, void* y, int nrhs) {
    if (!g) return HELM_EINVAL;
    helm_ctx ctx = g->ctx;
    if (!u || !y || nrhs < 0) return set_error(ctx, HELM_EINVAL, "helm_apply: invalid argument");
    if (prec != HELM_PREC_FP64 && prec != HELM_PREC_FP32)
        return set_error(ctx, HELM_EINVAL, "helm_apply: prec must be FP64 or FP32");
    if (nrhs == 0) return HELM_OK;
    const size_t bytes = (size_t)g->n * nrhs * (prec == HELM_PREC_FP64 ? sizeof(c128) : sizeof(c64));
    const char* a = (const char*)u;
    const char* b = (const char*)y;
    if (a < b + bytes && b < a + bytes) return set_error(ctx, HELM_EINVAL, "helm_apply: u and y overlap");
    HELM_CUDA(ctx, cudaSetDevice(ctx->device));
    HELM_TRY(launch_stencil(g, prec, u, y, nrhs, ctx->stream));
    HELM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HELM_OK;
}

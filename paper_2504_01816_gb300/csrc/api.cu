// C entry points of librpa (declared in include/rpa.h) and the subspace-iteration driver of
// Algorithm 1 (arXiv 2504.01816) with Rayleigh-Ritz energies.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace rpa {

constexpr size_t kReadBackBytes = 16384;   // pinned read-back block of a context

static thread_local std::string g_last_error;
thread_local long long g_launches = 0;

void fail(rpa_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    throw Error{st, buf};
}

void check_cuda(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    const rpa_status st = (e == cudaErrorMemoryAllocation) ? RPA_ERR_OOM : RPA_ERR_CUDA;
    fail(st, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

void allow_dynamic_smem(const void *kernel, size_t need) {
    int dev = 0, optin = 0;
    RPA_CUDA(cudaGetDevice(&dev));
    RPA_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    RPA_CUDA(cudaFuncGetAttributes(&fa, kernel));
    const long long avail = (long long)optin - (long long)fa.sharedSizeBytes;
    if ((long long)need > avail)
        fail(RPA_ERR_INVALID, "a kernel needs %zu bytes of shared memory, more than the %lld available", need, avail);
    if (fa.maxDynamicSharedSizeBytes < avail)
        RPA_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)avail));
}

void *DevBuf::ensure(size_t need) {
    if (need <= bytes && ptr) return ptr;
    release();
    size_t want = std::max(need, (size_t)256);
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        (void)cudaGetLastError();
        fail(RPA_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", want, cudaGetErrorString(e));
    }
    bytes = want;
    return ptr;
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

Ctx::~Ctx() {
    cudaFree(vloc64);
    cudaFree(vloc32);
    cudaFree(vloc_lo);
    cudaFree(psi64);
    cudaFree(psi32);
    cudaFree(eps_dev);
    for (double *q : Q) cudaFree(q);
    cudaFree(lam);
    for (int a = 0; a < 3; ++a) {
        cudaFree(mu[a]);
        cudaFree(Qf[a]);
        cudaFree(muf[a]);
    }
    for (DevBuf *b : {&cocg_state, &cocg_partials, &sys_state, &rhs, &pc_coef, &coul_tmp, &blockA, &blockB,
                      &blockC, &blockD, &small, &slot_idx, &dense_scratch, &proj_buf, &coef_buf, &blockE})
        b->release();
    if (h_state) cudaFreeHost(h_state);
    if (h_count) cudaFreeHost(h_count);
    cudaFree(d_tc_err);
    cudaFree(d_qstats);
    cudaFree(d_loop);
    if (h_rb) cudaFreeHost(h_rb);
    for (cudaEvent_t e : ev_apply)
        if (e) cudaEventDestroy(e);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cudaFree(d_prof_points);
}

int prof_slot(Ctx &c, const char *name) {
    for (int i = 0; i < c.stats.prof_count; ++i)
        if (std::strncmp(c.stats.prof_name[i], name, 31) == 0) return i;
    if (c.stats.prof_count >= RPA_PROF_SLOTS) return RPA_PROF_SLOTS - 1;
    const int i = c.stats.prof_count++;
    std::strncpy(c.stats.prof_name[i], name, 31);
    c.stats.prof_name[i][31] = 0;
    return i;
}

void sync_stream(Ctx &c, cudaStream_t s) {
    RPA_CUDA(cudaStreamSynchronize(s));
    c.host_syncs += 1;
}

int add_queue_stats(Ctx &c, const QueueStats &h) {
    c.stats.sternheimer_solves += h.solves;
    c.stats.cocg_iterations += h.iters;
    c.stats.refinement_steps += h.refines;
    c.stats.stencil_points += (h.iters + h.refines) * c.nd;
    c.stats.near_breakdowns += h.nearb;
    g_launches += h.launches;
    int worst = h.worst;
    if (h.unfinished) worst = std::max(worst, (int)RPA_ERR_NOT_CONVERGED);
    c.stats.worst_status = std::max(c.stats.worst_status, worst);
    return worst;
}

void check_tensor_core_status(Ctx &c, cudaStream_t s) {
    int h = 0;
    RPA_CUDA(cudaMemcpyAsync(&h, c.d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    RPA_CUDA(cudaStreamSynchronize(s));
    if (h) {
        RPA_CUDA(cudaMemsetAsync(c.d_tc_err, 0, sizeof(int), s));
        fail(RPA_ERR_CUDA, "a tensor-core contraction timed out waiting for its MMAs");
    }
}

namespace {

__global__ void k_to_float(const double *in, float *out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

// lo = x - (float)x in FP32: x = hi + lo to ~2^-48 |x|
__global__ void k_low_part(const double *in, float *out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)(in[i] - (double)(float)in[i]);
}

void validate_options(const rpa_options &o) {
    if (o.prec != RPA_FP64 && o.prec != RPA_MIXED) fail(RPA_ERR_INVALID, "prec must be RPA_FP64 or RPA_MIXED");
    if (!(o.tol > 0.0) || !(o.tol < 1.0)) fail(RPA_ERR_INVALID, "tol must be in (0, 1)");
    if (o.maxit < 1) fail(RPA_ERR_INVALID, "maxit must be >= 1");
    if (o.max_refine < 1) fail(RPA_ERR_INVALID, "max_refine must be >= 1");
    if (!(o.inner_tol > 0.0) || !(o.inner_tol < 1.0)) fail(RPA_ERR_INVALID, "inner_tol must be in (0, 1)");
    if (!(o.eps_c >= 0.0)) fail(RPA_ERR_INVALID, "eps_c must be >= 0");
    if (o.n_omega < 1 || o.n_omega > kMaxOmega) fail(RPA_ERR_INVALID, "n_omega must be in [1, %d]", kMaxOmega);
    if (!(o.omega0 > 0.0)) fail(RPA_ERR_INVALID, "omega0 must be > 0");
    if (o.max_subspace_iters < 1) fail(RPA_ERR_INVALID, "max_subspace_iters must be >= 1");
    if (o.fixed_subspace_iters < 0) fail(RPA_ERR_INVALID, "fixed_subspace_iters must be >= 0");
    if (o.n_atoms < 1) fail(RPA_ERR_INVALID, "n_atoms must be >= 1");
    if (o.batch_systems < 0) fail(RPA_ERR_INVALID, "batch_systems must be >= 0");
    if (o.z_chunks < 0 || o.z_chunks > 64) fail(RPA_ERR_INVALID, "z_chunks must be in [0, 64]");
    if (o.stencil_shape < 0 || o.stencil_shape > 6) fail(RPA_ERR_INVALID, "stencil_shape must be in [0, 6]");
    if (o.sq_order < 0 || o.sq_order > kMaxSqOrder) fail(RPA_ERR_INVALID, "sq_order must be in [0, %d]", kMaxSqOrder);
    if (o.contractions < 0 || o.contractions > 3) fail(RPA_ERR_INVALID, "contractions must be in [0, 3]");
    if (o.periodic != 0 && o.periodic != 1) fail(RPA_ERR_INVALID, "periodic must be 0 or 1");
    if (o.precondition != 0 && o.precondition != 1) fail(RPA_ERR_INVALID, "precondition must be 0 or 1");
    if (o.block_cocg < 0 || o.block_cocg > kMaxBlock) fail(RPA_ERR_INVALID, "block_cocg must be in [0, %d]", kMaxBlock);
    if (o.block_cocg > 0 && (o.precondition || o.project_solution))
        fail(RPA_ERR_INVALID, "block_cocg runs without precondition and project_solution");
    if (o.omega_count < 0 || o.omega_first < 0 || (o.omega_count > 0 && o.omega_first + o.omega_count > o.n_omega) ||
        (o.omega_count == 0 && o.omega_first != 0))
        fail(RPA_ERR_INVALID, "omega_first/omega_count must select a range of the n_omega frequencies");
}

// Gauss-Legendre nodes and weights on (-1, 1) by Newton iteration on P_n, then the map
// omega = w0 (1+x)/(1-x), weight = 2 w0 w / (1-x)^2.  Ascending omega.
void frequency_rule(int n, double w0, double *om, double *wt) {
    std::vector<double> x(n), w(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute the derivative at the converged root
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    // roots come out descending in x; emit ascending
    for (int i = 0; i < n; ++i) {
        const double xi = x[n - 1 - i], wi = w[n - 1 - i];
        om[i] = w0 * (1.0 + xi) / (1.0 - xi);
        wt[i] = 2.0 * w0 * wi / ((1.0 - xi) * (1.0 - xi));
    }
}

template <typename F>
rpa_status guarded(F &&f) {
    try {
        f();
        g_last_error.clear();
        return RPA_OK;
    } catch (const Error &e) {
        g_last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return RPA_ERR_OOM;
    } catch (...) {
        g_last_error = "unexpected internal error";
        return RPA_ERR_INVALID;
    }
}

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

float ms_between(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

// R = nu^1/2 chi0 nu^1/2 V (symmetric) or nu chi0 V.  tmp1, tmp2: ncols x nd scratch.  Enqueues
// the work without waiting for it: the phase times (events) and the per-system statuses (device
// statistics) are collected by finish_call after the caller's next synchronisation.
// Returns the worst per-system status known on the host (queues run without graphs or with
// profiling); device-driven queues report theirs through finish_call.
int apply_nuchi0_impl(Ctx &c, double omega, const double *V, double *R, int ncols, int symmetric, double *tmp1,
                      double *tmp2, cudaStream_t s) {
    cudaEvent_t *e = c.ev_apply;
    RPA_CUDA(cudaEventRecord(e[0], s));
    const double *dv = V;
    const bool tc = use_tensor_cores_kronecker(c);
    if (symmetric) {
        coulomb_apply(c, 0.5, V, tmp1, ncols, s, tc);
        dv = tmp1;
    }
    RPA_CUDA(cudaEventRecord(e[1], s));
    const int worst = chi0_apply(c, omega, dv, tmp2, ncols, s);
    RPA_CUDA(cudaEventRecord(e[2], s));
    coulomb_apply(c, symmetric ? 0.5 : 1.0, tmp2, R, ncols, s, tc);
    RPA_CUDA(cudaEventRecord(e[3], s));
    c.apply_timed = true;
    return worst;
}

// Bytes of the pinned read-back block: Ritz values (up to 1024), two energies, two pivot flags, the
// tensor-core flag and the queue statistics.
constexpr size_t kReadBackLam = 1024 * sizeof(double);
// offsets in the read-back block
constexpr size_t kRbScal = kReadBackLam, kRbInfo = kRbScal + 2 * sizeof(double), kRbTc = kRbInfo + 2 * sizeof(int),
                 kRbStats = (kRbTc + sizeof(int) + 15) / 16 * 16;

// Enqueue the read-back of the device flags and statistics into the pinned block (the caller
// synchronises once, then calls finish_call).
void enqueue_status_readback(Ctx &c, cudaStream_t s) {
    RPA_CUDA(cudaMemcpyAsync(c.h_rb + kRbTc, c.d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    RPA_CUDA(cudaMemcpyAsync(c.h_rb + kRbStats, c.d_qstats, sizeof(QueueStats), cudaMemcpyDeviceToHost, s));
    RPA_CUDA(cudaMemsetAsync(c.d_qstats, 0, sizeof(QueueStats), s));
}

// After the synchronisation that completed enqueue_status_readback: phase times, tensor-core flag
// and queue statistics; returns the worst per-system status.
int finish_call(Ctx &c, cudaStream_t s) {
    if (c.apply_timed) {
        c.stats.ms_coulomb += ms_between(c.ev_apply[0], c.ev_apply[1]) + ms_between(c.ev_apply[2], c.ev_apply[3]);
        c.stats.ms_cocg += ms_between(c.ev_apply[1], c.ev_apply[2]);
        c.apply_timed = false;
    }
    int tcerr = 0;
    std::memcpy(&tcerr, c.h_rb + kRbTc, sizeof(int));
    if (tcerr) {
        RPA_CUDA(cudaMemsetAsync(c.d_tc_err, 0, sizeof(int), s));
        fail(RPA_ERR_CUDA, "a tensor-core contraction timed out waiting for its MMAs");
    }
    QueueStats q;
    std::memcpy(&q, c.h_rb + kRbStats, sizeof q);
    return add_queue_stats(c, q);
}

}  // namespace
}  // namespace rpa

using namespace rpa;

extern "C" {

void rpa_default_options(rpa_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->prec = RPA_FP64;
    o->tol = 1e-8;
    o->maxit = 20000;
    o->max_refine = 20;
    o->inner_tol = 1e-4;
    o->eps_c = 1e-5;
    o->n_omega = 8;
    o->omega0 = 1.0;
    o->max_subspace_iters = 100;
    o->fixed_subspace_iters = 0;
    o->n_atoms = 1;
    o->batch_systems = 0;
    o->profile = 0;
    o->project_solution = 0;
    o->z_chunks = 0;
    o->stencil_shape = 0;
    o->independent_frequencies = 0;
    o->sq_order = 0;
    o->contractions = 0;
    o->omega_first = 0;
    o->omega_count = 0;
    o->periodic = 0;
    o->precondition = 0;
    o->block_cocg = 0;
}

const char *rpa_last_error(void) { return g_last_error.c_str(); }

const char *rpa_version(void) { return "librpa 0.1 (sm_103a)"; }

rpa_status rpa_setup(rpa_ctx **out, int nx, int ny, int nz, double h, int fd_order, const double *vloc_dev,
                     const double *psi_dev, const double *eps_host, int n_s, const rpa_options *opt, void *stream) {
    return guarded([&] {
        if (!out) fail(RPA_ERR_INVALID, "out is NULL");
        *out = nullptr;
        if (nx < 1 || ny < 1 || nz < 1) fail(RPA_ERR_INVALID, "grid dimensions must be >= 1");
        if (!(h > 0.0)) fail(RPA_ERR_INVALID, "h must be > 0");
        if (fd_order != 2 * kRadius) fail(RPA_ERR_INVALID, "fd_order must be %d", 2 * kRadius);
        if (n_s < 1) fail(RPA_ERR_INVALID, "n_s must be >= 1");
        if (!vloc_dev || !psi_dev || !eps_host) fail(RPA_ERR_INVALID, "NULL input pointer");
        const long long nd = (long long)nx * ny * nz;
        if (n_s >= nd) fail(RPA_ERR_INVALID, "n_s must be smaller than the number of grid points");
        if (nd >= (1LL << 31)) fail(RPA_ERR_INVALID, "grids of 2^31 points or more are not supported");
        rpa_options o;
        rpa_default_options(&o);
        if (opt) o = *opt;
        validate_options(o);
        cudaStream_t s = as_stream(stream);
        auto *ctx = new rpa_ctx();
        Ctx &c = ctx->impl;
        try {
            RPA_CUDA(cudaGetDevice(&c.device));
            c.nx = nx; c.ny = ny; c.nz = nz; c.nd = nd; c.h = h; c.ns = n_s; c.opt = o;
            // centred weights of order 12: w_k = 2(-1)^{k+1}(p!)^2/(k^2 (p-k)!(p+k)!), w_0 = -2 sum 1/k^2
            double fact[2 * kRadius + 1];
            fact[0] = 1.0;
            for (int i = 1; i <= 2 * kRadius; ++i) fact[i] = fact[i - 1] * i;
            double w0 = 0.0;
            for (int k = 1; k <= kRadius; ++k) {
                const double wk = 2.0 * ((k & 1) ? 1.0 : -1.0) * fact[kRadius] * fact[kRadius] /
                                  ((double)k * k * fact[kRadius - k] * fact[kRadius + k]);
                c.coef.a[k] = -wk / (2.0 * h * h);
                w0 -= 2.0 / ((double)k * k);
            }
            c.coef.a[0] = -w0 / (2.0 * h * h);
            c.eps.assign(eps_host, eps_host + n_s);
            RPA_CUDA(cudaMalloc(&c.vloc64, sizeof(double) * nd));
            RPA_CUDA(cudaMalloc(&c.vloc32, sizeof(float) * nd));
            RPA_CUDA(cudaMalloc(&c.vloc_lo, sizeof(float) * nd));
            RPA_CUDA(cudaMalloc(&c.psi64, sizeof(double) * nd * n_s));
            RPA_CUDA(cudaMalloc(&c.psi32, sizeof(float) * nd * n_s));
            RPA_CUDA(cudaMalloc(&c.eps_dev, sizeof(double) * n_s));
            RPA_CUDA(cudaMemcpyAsync(c.vloc64, vloc_dev, sizeof(double) * nd, cudaMemcpyDeviceToDevice, s));
            RPA_CUDA(cudaMemcpyAsync(c.psi64, psi_dev, sizeof(double) * nd * n_s, cudaMemcpyDeviceToDevice, s));
            RPA_CUDA(cudaMemcpyAsync(c.eps_dev, eps_host, sizeof(double) * n_s, cudaMemcpyHostToDevice, s));
            k_to_float<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(c.vloc64, c.vloc32, nd);
            k_low_part<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(c.vloc64, c.vloc_lo, nd);
            k_to_float<<<(unsigned)((nd * n_s + 255) / 256), 256, 0, s>>>(c.psi64, c.psi32, nd * n_s);
            RPA_LAUNCH("setup");
            RPA_CUDA(cudaMallocHost((void **)&c.h_count, 8 * sizeof(int)));
            RPA_CUDA(cudaMalloc(&c.d_tc_err, sizeof(int)));
            RPA_CUDA(cudaMemsetAsync(c.d_tc_err, 0, sizeof(int), s));
            RPA_CUDA(cudaMalloc(&c.d_qstats, sizeof(QueueStats)));
            RPA_CUDA(cudaMemsetAsync(c.d_qstats, 0, sizeof(QueueStats), s));
            RPA_CUDA(cudaMalloc(&c.d_loop, sizeof(int)));
            RPA_CUDA(cudaMallocHost((void **)&c.h_rb, kReadBackBytes));
            for (auto &e : c.ev_apply) RPA_CUDA(cudaEventCreate(&e));
            RPA_CUDA(cudaMalloc(&c.d_prof_points, sizeof(unsigned long long) * RPA_PROF_SLOTS));
            RPA_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
            {
                const char *g = std::getenv("RPA_GRAPHS");
                c.use_graphs = !(g && g[0] == '0');
            }
            RPA_CUDA(cudaStreamSynchronize(s));
            {   // mean V_loc: the constant potential of the Laplacian preconditioner
                std::vector<double> v((size_t)nd);
                RPA_CUDA(cudaMemcpy(v.data(), c.vloc64, sizeof(double) * nd, cudaMemcpyDeviceToHost));
                double sum = 0.0;
                for (double x : v) sum += x;
                c.vbar = sum / (double)nd;
            }
            coulomb_setup(c);
        } catch (...) {
            delete ctx;
            throw;
        }
        *out = ctx;
    });
}

rpa_status rpa_set_options(rpa_ctx *ctx, const rpa_options *opt) {
    return guarded([&] {
        if (!ctx || !opt) fail(RPA_ERR_INVALID, "NULL argument");
        validate_options(*opt);
        if (opt->periodic != ctx->impl.opt.periodic)
            fail(RPA_ERR_INVALID, "periodic is fixed at rpa_setup (the Coulomb operator is built for it)");
        ctx->impl.opt = *opt;
    });
}

void rpa_destroy(rpa_ctx *ctx) { delete ctx; }

rpa_status rpa_coulomb_apply(rpa_ctx *ctx, double power, const double *in_dev, double *out_dev, int ncols,
                             void *stream) {
    return guarded([&] {
        if (!ctx || !in_dev || !out_dev) fail(RPA_ERR_INVALID, "NULL argument");
        if (ncols < 0) fail(RPA_ERR_INVALID, "ncols must be >= 0");
        if (!std::isfinite(power)) fail(RPA_ERR_INVALID, "power must be finite");
        coulomb_apply(ctx->impl, power, in_dev, out_dev, ncols, as_stream(stream));
        RPA_CUDA(cudaStreamSynchronize(as_stream(stream)));
    });
}

rpa_status rpa_coulomb_apply_noalloc(rpa_ctx *ctx, double power, const double *in_dev, double *out_dev, int ncols,
                                     void *stream) {
    return guarded([&] {
        if (!ctx || !in_dev || !out_dev) fail(RPA_ERR_INVALID, "NULL argument");
        if (ncols < 0) fail(RPA_ERR_INVALID, "ncols must be >= 0");
        if (!std::isfinite(power)) fail(RPA_ERR_INVALID, "power must be finite");
        coulomb_apply_noalloc(ctx->impl, power, in_dev, out_dev, ncols, as_stream(stream));
        RPA_CUDA(cudaStreamSynchronize(as_stream(stream)));
    });
}

rpa_status rpa_sternheimer_solve(rpa_ctx *ctx, double omega, const int *orbital_idx_host, int nsys,
                                 const double *rhs_dev, int project, double *x_dev, int *iters_dev,
                                 int *status_dev, void *stream) {
    int worst = 0;
    rpa_status st = guarded([&] {
        if (!ctx || !orbital_idx_host || !rhs_dev || !x_dev) fail(RPA_ERR_INVALID, "NULL argument");
        if (nsys < 0) fail(RPA_ERR_INVALID, "nsys must be >= 0");
        if (!std::isfinite(omega)) fail(RPA_ERR_INVALID, "omega must be finite");
        if (nsys == 0) return;
        Ctx &c = ctx->impl;
        cudaStream_t s = as_stream(stream);
        std::vector<int> it(nsys), stv(nsys);
        worst = project ? sternheimer_batch_projected(c, omega, orbital_idx_host, nsys, rhs_dev, x_dev, &it, &stv, s)
                        : sternheimer_batch(c, omega, orbital_idx_host, nsys, rhs_dev, x_dev, &it, &stv, s);
        if (iters_dev) RPA_CUDA(cudaMemcpyAsync(iters_dev, it.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s));
        if (status_dev) RPA_CUDA(cudaMemcpyAsync(status_dev, stv.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s));
        RPA_CUDA(cudaStreamSynchronize(s));
    });
    if (st != RPA_OK) return st;
    if (worst != RPA_OK) g_last_error = "a Sternheimer system did not converge";
    return (rpa_status)worst;
}

rpa_status rpa_autotune(rpa_ctx *ctx, double omega, const double *V_dev, int n_r, int *chosen_host,
                        double *times_ms_host, void *stream) {
    return guarded([&] {
        if (!ctx || !V_dev) fail(RPA_ERR_INVALID, "NULL argument");
        if (n_r < 1) fail(RPA_ERR_INVALID, "n_r must be >= 1");
        if (!std::isfinite(omega)) fail(RPA_ERR_INVALID, "omega must be finite");
        Ctx &c = ctx->impl;
        cudaStream_t s = as_stream(stream);
        const size_t blk = sizeof(double) * (size_t)n_r * c.nd;
        double *t1 = (double *)c.blockA.ensure(blk);
        double *t2 = (double *)c.blockB.ensure(blk);
        double *R = (double *)c.blockC.ensure(blk);
        // candidates 0..5: split kernel variant v (stencil_shape v + 1) with z chunks z + 1, index
        // 2 v + z; candidate 6: the fused single-pass kernel (stencil_shape 4), candidate 7 its
        // warp-specialised form (stencil_shape 5), where a plane fits; candidate 8 its cluster form
        // with two blocks per SM (stencil_shape 6), where the plane's bands fit
        const bool mixed = c.opt.prec == RPA_MIXED;
        const bool fused_ok = mixed && fused_kernel_applies(c);
        const bool ws_ok = mixed && fused_kernel_applies(c, true);
        const bool cl_ok = mixed && fused_kernel_applies(c, false, true);
        double best = 1e300;
        int best_i = 0;
        cudaEvent_t a, b;
        RPA_CUDA(cudaEventCreate(&a));
        RPA_CUDA(cudaEventCreate(&b));
        for (int i = 0; i < RPA_AUTOTUNE_CANDIDATES; ++i) {
            const bool run = i == 8 ? cl_ok : i == 7 ? ws_ok : i == 6 ? fused_ok : (mixed || i == 0);
            double ms = -1.0;
            if (run) {
                c.opt.stencil_shape = i >= 6 ? i - 2 : i / 2 + 1;
                c.opt.z_chunks = i >= 6 ? 1 : i % 2 + 1;
                RPA_CUDA(cudaEventRecord(a, s));
                apply_nuchi0_impl(c, omega, V_dev, R, n_r, 1, t1, t2, s);
                RPA_CUDA(cudaEventRecord(b, s));
                RPA_CUDA(cudaEventSynchronize(b));
                ms = ms_between(a, b);
                if (ms < best) {
                    best = ms;
                    best_i = i;
                }
            }
            if (times_ms_host) times_ms_host[i] = ms;
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        enqueue_status_readback(c, s);
        sync_stream(c, s);
        finish_call(c, s);
        c.opt.stencil_shape = best_i >= 6 ? best_i - 2 : best_i / 2 + 1;
        c.opt.z_chunks = best_i >= 6 ? 1 : best_i % 2 + 1;
        if (chosen_host) *chosen_host = best_i;
    });
}

rpa_status rpa_apply_nuchi0(rpa_ctx *ctx, double omega, const double *V_dev, double *R_dev, int n_r, int symmetric,
                            void *stream) {
    int worst = 0;
    rpa_status st = guarded([&] {
        if (!ctx || !V_dev || !R_dev) fail(RPA_ERR_INVALID, "NULL argument");
        if (n_r < 0) fail(RPA_ERR_INVALID, "n_r must be >= 0");
        if (!std::isfinite(omega)) fail(RPA_ERR_INVALID, "omega must be finite");
        if (V_dev == R_dev && n_r > 0) fail(RPA_ERR_INVALID, "V and R must not alias");
        if (n_r == 0) return;
        Ctx &c = ctx->impl;
        cudaStream_t s = as_stream(stream);
        const size_t blk = sizeof(double) * (size_t)n_r * c.nd;
        double *t1 = (double *)c.blockA.ensure(blk);
        double *t2 = (double *)c.blockB.ensure(blk);
        worst = apply_nuchi0_impl(c, omega, V_dev, R_dev, n_r, symmetric, t1, t2, s);
        enqueue_status_readback(c, s);
        sync_stream(c, s);
        worst = std::max(worst, finish_call(c, s));
    });
    if (st != RPA_OK) return st;
    if (worst != RPA_OK) g_last_error = "a Sternheimer system did not converge";
    return (rpa_status)worst;
}

}  // extern "C"

namespace rpa {
namespace {

// Algorithm 1 with Rayleigh-Ritz; with grad != nullptr also dE_c/dV_loc (see rpa_ec_gradient).
//
// A subspace iteration is enqueued without waiting: the chi0 application (its COCG queue replayed
// by a device-side graph loop), the projection and eigenvalues, the orthonormalisation (the
// Cholesky pivot check stays on the device) and the read-back of the Ritz values, energies, pivot
// flags and statistics into pinned memory; the host then synchronises once per iteration to take
// the stopping decision.
int ec_impl(Ctx &c, int n_r, const double *V0_dev, double *lambdas_host, double *ec_host, double *ec_per_omega_host,
            rpa_stats *stats, cudaStream_t s, double *grad, double *V_out) {
    int worst = 0;
    if (n_r < 1 || n_r > c.nd) fail(RPA_ERR_INVALID, "n_r must be in [1, N_d]");
    if (n_r > 1024) fail(RPA_ERR_INVALID, "n_r above 1024 is not supported");
    std::memset(&c.stats, 0, sizeof c.stats);
    g_launches = 0;
    c.host_syncs = 0;
    const rpa_options &o = c.opt;
    const int nw = o.n_omega;
    double om[kMaxOmega], wt[kMaxOmega];
    frequency_rule(nw, o.omega0, om, wt);
    for (int m = 0; m < nw; ++m) {
        c.stats.omegas[m] = om[m];
        c.stats.weights[m] = wt[m];
    }
    const size_t blk = sizeof(double) * (size_t)n_r * c.nd;
    double *V = (double *)c.blockA.ensure(blk);
    double *R = (double *)c.blockB.ensure(blk);
    double *T1 = (double *)c.blockC.ensure(blk);
    double *T2 = (double *)c.blockD.ensure(blk);
    double *Vprev = grad ? (double *)c.blockE.ensure(blk) : nullptr;
    const size_t nn = (size_t)n_r * n_r;
    char *sm = (char *)c.small.ensure(sizeof(double) * (5 * nn + 4 * (size_t)n_r + 8) + 64);
    double *Cm = (double *)sm;            // projection / overlap
    double *Lm = Cm + nn;                 // inverse factor
    double *Wm = Lm + nn;                 // copy for the eigen solve
    double *Cprev = Wm + nn;              // projected matrix of the last iteration (gradient)
    double *Sm = Cprev + nn;              // rotation to Ritz vectors (gradient)
    double *lam = Sm + nn;
    double *work = lam + n_r;             // 3 n_r
    double *ecm_dev = work + 3 * (size_t)n_r;
    int *info = (int *)(ecm_dev + 2);     // [0]: starting block, [1]: the block A V
    const double *h_lam = (const double *)c.h_rb;
    const double *h_scal = (const double *)(c.h_rb + kRbScal);
    const int *h_info = (const int *)(c.h_rb + kRbInfo);
    if (grad) RPA_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * c.nd, s));
    RPA_CUDA(cudaMemsetAsync(info, 0, 2 * sizeof(int), s));

    cudaEvent_t t0, t1, a, b;
    RPA_CUDA(cudaEventCreate(&t0));
    RPA_CUDA(cudaEventCreate(&t1));
    RPA_CUDA(cudaEventCreate(&a));
    RPA_CUDA(cudaEventCreate(&b));
    RPA_CUDA(cudaEventRecord(t0, s));

    // Y = X L^{-T}, L L^T = X^T X (rows: Y = L^{-1} X); a failed pivot is recorded in *flag (the
    // first failure is kept) and read with the iteration's other results.
    auto orthonormalize = [&](const double *X, double *Y, int *flag) {
        gram(X, n_r, X, n_r, c.nd, Cm, s, c.dense_scratch);
        symmetrize(Cm, n_r, s);
        cholesky(Cm, n_r, flag, s);
        tri_inverse(Cm, n_r, Lm, s);
        combine_rows(Lm, n_r, n_r, X, c.nd, Y, s);
    };
    // the overlap again, for the message of a failed orthonormalisation: its diagonal holds the
    // squared row norms
    auto fail_not_spd = [&](const double *X, int pivot, const char *what, int m, int it) {
        gram(X, n_r, X, n_r, c.nd, Wm, s, c.dense_scratch);
        std::vector<double> M(nn);
        RPA_CUDA(cudaMemcpyAsync(M.data(), Wm, sizeof(double) * nn, cudaMemcpyDeviceToHost, s));
        sync_stream(c, s);
        double dmin = 1e300, dmax = 0.0;
        int bad = 0;
        for (int i = 0; i < n_r; ++i) {
            const double d = M[(size_t)i * n_r + i];
            if (!std::isfinite(d)) ++bad;
            else {
                dmin = std::min(dmin, d);
                dmax = std::max(dmax, d);
            }
        }
        fail(RPA_ERR_NOT_SPD,
             "overlap matrix not positive definite (pivot %d) of %s (frequency %d, subspace iteration %d); "
             "recomputed overlap: diagonal in [%.3e, %.3e], %d non-finite, pivot entry %.3e",
             pivot, what, m, it, dmin, dmax, bad, M[(size_t)pivot * n_r + pivot]);
    };
    orthonormalize(V0_dev, V, info);

    double ec = 0.0;
    std::vector<double> ecm_all(nw, 0.0);
    if (lambdas_host) std::memset(lambdas_host, 0, sizeof(double) * (size_t)nw * n_r);
    const double thr = o.eps_c * o.n_atoms / nw;
    // frequencies of this call (all, or the range omega_first .. +omega_count), highest first
    const int m_lo = o.omega_count > 0 ? o.omega_first : 0;
    const int m_hi = o.omega_count > 0 ? o.omega_first + o.omega_count - 1 : nw - 1;
    for (int m = m_hi; m >= m_lo; --m) {
        if (o.independent_frequencies && m != m_hi) orthonormalize(V0_dev, V, info);
        double ecm = 0.0;
        int it = 0;
        for (;;) {
            const double ecm_old = ecm;
            worst = std::max(worst, apply_nuchi0_impl(c, om[m], V, R, n_r, 1, T1, T2, s));
            RPA_CUDA(cudaEventRecord(a, s));
            // Rayleigh-Ritz: C = V^T R, eigenvalues, E_cm = (w_m / 2 pi) sum g(lambda)
            if (use_tensor_cores(c))
                tc_gemm(V, c.nd, 1, R, c.nd, 1, n_r, n_r, c.nd, Wm, s, c.dense_scratch, c.d_tc_err);
            else
                gram(V, n_r, R, n_r, c.nd, Wm, s, c.dense_scratch);
            symmetrize(Wm, n_r, s);
            if (grad) {
                RPA_CUDA(cudaMemcpyAsync(Cprev, Wm, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
                RPA_CUDA(cudaMemcpyAsync(Vprev, V, blk, cudaMemcpyDeviceToDevice, s));
            }
            // Gauss spectral quadrature reads C before the eigensolver may overwrite it
            if (o.sq_order > 0) sq_trace(Wm, n_r, o.sq_order, work, wt[m] / (2.0 * M_PI), ecm_dev + 1, s);
            sym_eigvals(Wm, n_r, lam, work, wt[m] / (2.0 * M_PI), ecm_dev, s);
            // orthonormalisation: M = R^T R = L L^T, V = R L^{-T}
            orthonormalize(R, V, info + 1);
            RPA_CUDA(cudaEventRecord(b, s));
            // the iteration's one read-back
            RPA_CUDA(cudaMemcpyAsync(c.h_rb, lam, sizeof(double) * n_r, cudaMemcpyDeviceToHost, s));
            RPA_CUDA(cudaMemcpyAsync(c.h_rb + kRbScal, ecm_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
            RPA_CUDA(cudaMemcpyAsync(c.h_rb + kRbInfo, info, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
            enqueue_status_readback(c, s);
            sync_stream(c, s);
            worst = std::max(worst, finish_call(c, s));
            if (h_info[0] != 0) fail_not_spd(V0_dev, h_info[0] - 1, "the starting block", -1, 0);
            if (h_info[1] != 0) fail_not_spd(R, h_info[1] - 1, "the block A V", m, it);
            c.stats.ms_subspace += ms_between(a, b);
            ecm = o.sq_order > 0 ? h_scal[1] : h_scal[0];
            ++it;
            if (o.fixed_subspace_iters > 0) {
                if (it >= o.fixed_subspace_iters) break;
            } else if (std::fabs(ecm - ecm_old) <= thr || it >= o.max_subspace_iters) {
                break;
            }
        }
        c.stats.subspace_iterations[m] = it;
        ecm_all[m] = ecm;
        ec += ecm;
        if (lambdas_host) std::memcpy(lambdas_host + (size_t)m * n_r, h_lam, sizeof(double) * n_r);
        if (grad) {
            // Ritz pairs of the last iteration on the device: C = Q diag(lambda) Q^T (parallel Jacobi,
            // C destroyed), y_i = sum_k Q[k][i] v_k, coef_i = (w_m / 2pi) g'(lambda_i)
            double *coef = (double *)c.coef_buf.ensure(sizeof(double) * (4 * (size_t)n_r + 8));
            jacobi_eigh_device(Cprev, n_r, Lm, work, coef + n_r, s);   // Q -> Lm, lambda -> work
            ritz_rotation(Lm, work, n_r, wt[m] / (2.0 * M_PI), Sm, coef, s);
            combine_rows(Sm, n_r, n_r, Vprev, c.nd, T1, s);           // Ritz vectors
            coulomb_apply(c, 0.5, T1, T2, n_r, s);                    // nu^1/2 y_i
            worst = std::max(worst, response_square(c, om[m], T2, coef, grad, n_r, s));
            enqueue_status_readback(c, s);
            sync_stream(c, s);
            worst = std::max(worst, finish_call(c, s));
        }
    }
    if (V_out) RPA_CUDA(cudaMemcpyAsync(V_out, V, blk, cudaMemcpyDeviceToDevice, s));
    RPA_CUDA(cudaEventRecord(t1, s));
    RPA_CUDA(cudaEventSynchronize(t1));
    c.stats.ms_total = ms_between(t0, t1);
    c.stats.launches = g_launches;
    c.stats.host_syncs = c.host_syncs;
    for (cudaEvent_t e : {t0, t1, a, b}) cudaEventDestroy(e);
    if (ec_host) {
        ec_host[0] = ec;
        ec_host[1] = ec / o.n_atoms;
    }
    if (ec_per_omega_host) std::memcpy(ec_per_omega_host, ecm_all.data(), sizeof(double) * nw);
    if (stats) *stats = c.stats;
    return worst;
}

}  // namespace
}  // namespace rpa

extern "C" {

rpa_status rpa_ec(rpa_ctx *ctx, int n_r, const double *V0_dev, double *lambdas_host, double *ec_host,
                  double *ec_per_omega_host, rpa_stats *stats, void *stream) {
    int worst = 0;
    rpa_status st = guarded([&] {
        if (!ctx || !V0_dev) fail(RPA_ERR_INVALID, "NULL argument");
        worst = ec_impl(ctx->impl, n_r, V0_dev, lambdas_host, ec_host, ec_per_omega_host, stats, as_stream(stream),
                        nullptr, nullptr);
    });
    if (st != RPA_OK) return st;
    if (worst != RPA_OK) g_last_error = "a Sternheimer system did not converge";
    return (rpa_status)worst;
}

rpa_status rpa_ec_gradient(rpa_ctx *ctx, int n_r, const double *V0_dev, double *grad_dev, double *V_out_dev,
                           double *lambdas_host, double *ec_host, double *ec_per_omega_host, rpa_stats *stats,
                           void *stream) {
    int worst = 0;
    rpa_status st = guarded([&] {
        if (!ctx || !V0_dev || !grad_dev) fail(RPA_ERR_INVALID, "NULL argument");
        Ctx &c = ctx->impl;
        if (c.opt.sq_order != 0)
            fail(RPA_ERR_INVALID, "rpa_ec_gradient differentiates the Rayleigh-Ritz energy: set sq_order = 0");
        const int saved = c.opt.project_solution;
        c.opt.project_solution = 1;
        try {
            worst = ec_impl(c, n_r, V0_dev, lambdas_host, ec_host, ec_per_omega_host, stats, as_stream(stream),
                            grad_dev, V_out_dev);
        } catch (...) {
            c.opt.project_solution = saved;
            throw;
        }
        c.opt.project_solution = saved;
    });
    if (st != RPA_OK) return st;
    if (worst != RPA_OK) g_last_error = "a Sternheimer system did not converge";
    return (rpa_status)worst;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Several contexts at once (an uneven batch of independent systems)
// ------------------------------------------------------------------------------------------
namespace rpa {

// Rendezvous of rpa_ec_batch's threads, one per context: a thread's chi0 application waits until
// every thread still running has posted one, and the last to arrive runs them all as one batch
// on its own stream; every thread's stream then waits for the batch before going on.  A thread
// that finishes (or fails) leaves, and the others no longer wait for it.
struct BatchCoord {
    struct Pending {
        Chi0Request r;
        cudaEvent_t ready;   // the request's inputs are ready on its thread's stream
        int *status;
    };
    std::mutex m;
    std::condition_variable cv;
    int active = 0;
    long long batches = 0;         // batches run so far
    std::vector<Pending> pending;
    cudaEvent_t done = nullptr;    // recorded after each batch
    bool failed = false;
    rpa_status fail_status = RPA_OK;
    std::string fail_msg;

    void run(cudaStream_t s, const Ctx *runner) {   // m held
        try {
            // the runner's own request first: its context lends the workspaces and counts the syncs
            std::stable_partition(pending.begin(), pending.end(), [&](const Pending &p) { return p.r.c == runner; });
            std::vector<Chi0Request> reqs;
            for (const Pending &p : pending) {
                RPA_CUDA(cudaStreamWaitEvent(s, p.ready, 0));
                reqs.push_back(p.r);
            }
            std::vector<int> st;
            chi0_apply_batch(reqs, s, &st);
            RPA_CUDA(cudaEventRecord(done, s));
            for (size_t k = 0; k < pending.size(); ++k) *pending[k].status = st[k];
            pending.clear();
            ++batches;
        } catch (const Error &e) {
            failed = true;
            fail_status = e.status;
            fail_msg = e.msg;
        } catch (const std::bad_alloc &) {
            failed = true;
            fail_status = RPA_ERR_OOM;
            fail_msg = "host allocation failed";
        } catch (...) {
            failed = true;
            fail_status = RPA_ERR_INVALID;
            fail_msg = "unexpected internal error";
        }
        cv.notify_all();   // the waiting threads wake either way
    }

    int apply(Ctx &c, double omega, const double *dv, double *drho, int ncols, cudaStream_t s) {
        cudaEvent_t ready;
        RPA_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        RPA_CUDA(cudaEventRecord(ready, s));
        int st = RPA_OK;
        std::unique_lock<std::mutex> lk(m);
        if (!failed) {
            pending.push_back({Chi0Request{&c, omega, dv, drho, ncols}, ready, &st});
            const long long my = batches;
            if ((int)pending.size() == active) run(s, &c);
            else cv.wait(lk, [&] { return batches > my || failed; });
        }
        cudaEventDestroy(ready);
        if (failed) fail(fail_status, "%s", fail_msg.c_str());
        RPA_CUDA(cudaStreamWaitEvent(s, done, 0));
        return st;
    }

    void leave(cudaStream_t s, const Ctx *c) {
        std::unique_lock<std::mutex> lk(m);
        --active;
        if (active > 0 && !failed && !pending.empty() && (int)pending.size() == active) run(s, c);
        cv.notify_all();
    }
};

int batch_chi0(Ctx &c, double omega, const double *dv, double *drho, int ncols, cudaStream_t s) {
    return c.coord->apply(c, omega, dv, drho, ncols, s);
}

namespace {

// The contexts of a batch: distinct, on one device, with the same precision and COCG settings
// (the batch runs them with the first one's), and without the options the batch does not run.
void check_batch(rpa_ctx *const *ctxs, int n) {
    if (!ctxs || n < 1) fail(RPA_ERR_INVALID, "a batch needs n >= 1 contexts");
    for (int k = 0; k < n; ++k)
        if (!ctxs[k]) fail(RPA_ERR_INVALID, "NULL context %d", k);
    const Ctx &c0 = ctxs[0]->impl;
    for (int k = 0; k < n; ++k) {
        const Ctx &c = ctxs[k]->impl;
        for (int q = 0; q < k; ++q)
            if (ctxs[q] == ctxs[k]) fail(RPA_ERR_INVALID, "context %d appears twice in the batch", k);
        if (c.device != c0.device) fail(RPA_ERR_INVALID, "the contexts of a batch must be on one device");
        if (c.opt.prec != c0.opt.prec || c.opt.tol != c0.opt.tol || c.opt.inner_tol != c0.opt.inner_tol ||
            c.opt.maxit != c0.opt.maxit || c.opt.max_refine != c0.opt.max_refine ||
            c.opt.block_cocg != c0.opt.block_cocg)
            fail(RPA_ERR_INVALID,
                 "the contexts of a batch need equal prec, tol, inner_tol, maxit, max_refine and block_cocg");
        if (c.opt.precondition || c.opt.project_solution)
            fail(RPA_ERR_INVALID, "a batch runs without precondition and project_solution");
        if (c.coord) fail(RPA_ERR_INVALID, "context %d is already in a running batch", k);
    }
}

}  // namespace
}  // namespace rpa

extern "C" {

rpa_status rpa_apply_nuchi0_batch(rpa_ctx *const *ctxs, int n, double omega, const double *const *V_dev,
                                  double *const *R_dev, const int *ncols, int symmetric, void *stream) {
    int worst = 0;
    rpa_status st = guarded([&] {
        check_batch(ctxs, n);
        if (!V_dev || !R_dev || !ncols) fail(RPA_ERR_INVALID, "NULL argument");
        if (!std::isfinite(omega)) fail(RPA_ERR_INVALID, "omega must be finite");
        cudaStream_t s = as_stream(stream);
        std::vector<Chi0Request> reqs;
        std::vector<int> who;
        for (int k = 0; k < n; ++k) {
            Ctx &c = ctxs[k]->impl;
            if (ncols[k] < 0 || ncols[k] > 1024) fail(RPA_ERR_INVALID, "ncols[%d] must be in [0, 1024]", k);
            if (ncols[k] == 0) continue;
            if (!V_dev[k] || !R_dev[k]) fail(RPA_ERR_INVALID, "NULL argument (context %d)", k);
            if (V_dev[k] == R_dev[k]) fail(RPA_ERR_INVALID, "V and R must not alias (context %d)", k);
            const size_t blk = sizeof(double) * (size_t)ncols[k] * c.nd;
            double *t1 = (double *)c.blockA.ensure(blk);
            double *t2 = (double *)c.blockB.ensure(blk);
            const double *dv = V_dev[k];
            if (symmetric) {
                coulomb_apply(c, 0.5, V_dev[k], t1, ncols[k], s, use_tensor_cores_kronecker(c));
                dv = t1;
            }
            reqs.push_back(Chi0Request{&c, omega, dv, t2, ncols[k]});
            who.push_back(k);
        }
        worst = chi0_apply_batch(reqs, s);
        for (size_t q = 0; q < reqs.size(); ++q) {
            const int k = who[q];
            Ctx &c = ctxs[k]->impl;
            coulomb_apply(c, symmetric ? 0.5 : 1.0, reqs[q].drho, R_dev[k], ncols[k], s, use_tensor_cores_kronecker(c));
        }
        RPA_CUDA(cudaStreamSynchronize(s));
    });
    if (st != RPA_OK) return st;
    if (worst != RPA_OK) g_last_error = "a Sternheimer system did not converge";
    return (rpa_status)worst;
}

rpa_status rpa_ec_batch(rpa_ctx *const *ctxs, int n, const int *n_r, const double *const *V0_dev,
                        double *const *lambdas_host, double *ec_host, double *const *ec_per_omega_host,
                        rpa_stats *stats, void *stream) {
    std::vector<int> worst(n > 0 ? n : 0, 0);
    rpa_status st = guarded([&] {
        check_batch(ctxs, n);
        if (!n_r || !V0_dev) fail(RPA_ERR_INVALID, "NULL argument");
        for (int k = 0; k < n; ++k)
            if (!V0_dev[k]) fail(RPA_ERR_INVALID, "NULL argument (context %d)", k);
        BatchCoord coord;
        coord.active = n;
        cudaEvent_t start;
        RPA_CUDA(cudaEventCreateWithFlags(&coord.done, cudaEventDisableTiming));
        RPA_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
        RPA_CUDA(cudaEventRecord(start, as_stream(stream)));   // V0 is ready on the caller's stream
        std::vector<rpa_status> sts(n, RPA_OK);
        std::vector<std::string> msgs(n);
        for (int k = 0; k < n; ++k) ctxs[k]->impl.coord = &coord;
        const int dev = ctxs[0]->impl.device;
        std::vector<std::thread> threads;
        auto finish = [&] {
            for (std::thread &t : threads) t.join();
            for (int k = 0; k < n; ++k) ctxs[k]->impl.coord = nullptr;
            cudaEventDestroy(coord.done);
            cudaEventDestroy(start);
        };
        int spawned = 0;
        try {
            for (int k = 0; k < n; ++k, ++spawned)
                threads.emplace_back([&, k] {
                    Ctx &c = ctxs[k]->impl;
                    cudaStream_t s = nullptr;
                    try {
                        RPA_CUDA(cudaSetDevice(dev));
                        RPA_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
                        RPA_CUDA(cudaStreamWaitEvent(s, start, 0));
                        double e2[2] = {0.0, 0.0};
                        worst[k] = ec_impl(c, n_r[k], V0_dev[k], lambdas_host ? lambdas_host[k] : nullptr, e2,
                                           ec_per_omega_host ? ec_per_omega_host[k] : nullptr,
                                           stats ? stats + k : nullptr, s, nullptr, nullptr);
                        if (ec_host) {
                            ec_host[2 * k] = e2[0];
                            ec_host[2 * k + 1] = e2[1];
                        }
                    } catch (const Error &e) {
                        sts[k] = e.status;
                        msgs[k] = e.msg;
                    } catch (...) {
                        sts[k] = RPA_ERR_INVALID;
                        msgs[k] = "unexpected internal error";
                    }
                    coord.leave(s, &c);
                    if (s) {
                        cudaStreamSynchronize(s);
                        cudaStreamDestroy(s);
                    }
                });
        } catch (...) {
            // a thread could not be started: the ones that run must not wait for it
            for (int k = spawned; k < n; ++k) coord.leave(nullptr, nullptr);
            finish();
            throw;
        }
        finish();
        for (int k = 0; k < n; ++k)
            if (sts[k] != RPA_OK) fail(sts[k], "context %d: %s", k, msgs[k].c_str());
    });
    if (st != RPA_OK) return st;
    int w = 0;
    for (int v : worst) w = std::max(w, v);
    if (w != RPA_OK) g_last_error = "a Sternheimer system did not converge";
    return (rpa_status)w;
}

}  // extern "C"

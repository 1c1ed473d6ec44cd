// Coulomb operator nu^p = (4 pi)^p (-L_h)^{-p} by the Kronecker-product formalism
// (arXiv 2504.01816, Section "Implementation"; Poisson equation, Eq. 5).
//
// With zero values outside the box, -L_h = K_x (+) K_y (+) K_z (Kronecker sum) where K_a is
// the n_a x n_a matrix of the 1D centred second difference (symmetric Toeplitz, SPD).  With
// K_a = Q_a diag(mu_a) Q_a^T:
//     nu^p f = (Q_z x Q_y x Q_x) diag((4 pi)^p (mu_x + mu_y + mu_z)^{-p}) (Q_z x Q_y x Q_x)^T f
// i.e. three per-axis transforms with Q^T, a pointwise scale, three transforms with Q.
// The 1D eigendecompositions are computed once per context on the host (cyclic Jacobi in
// FP64; n_a is at most a few hundred).
#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace rpa {

// Symmetric eigendecomposition A = Q diag(w) Q^T (row-major n x n, Q[i*n+a] = component i of
// eigenvector a) by cyclic Jacobi rotations.
void jacobi_eigh(std::vector<double> A, int n, std::vector<double> &w, std::vector<double> &Q) {
    Q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double a = A[(size_t)i * n + j];
                tot += a * a;
                if (i != j) off += a * a;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {   // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {   // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
                    Q[(size_t)k * n + p] = c * qkp - s * qkq;
                    Q[(size_t)k * n + q] = s * qkp + c * qkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

namespace {

// out[o][a][i] = sum_b M[a][b] in[o][b][i]; M = Q^T (forward) or Q (back).  The data are viewed
// as [outer][n][inner].  Each block takes one outer index and 32 consecutive inner indices
// (inner > 1), or 32 consecutive outer indices (inner == 1); lines are staged in shared memory.
__global__ void __launch_bounds__(256) k_axis(const double *__restrict__ in, double *__restrict__ out,
                                              const double *__restrict__ Q, int n, long long inner,
                                              long long outer, int forward, const double *__restrict__ scale,
                                              long long nd) {
    extern __shared__ double sh[];
    double *Ms = sh;                 // n x n, Ms[a*n+b] = M[a][b]
    double *X = sh + (size_t)n * n;  // n x 32, X[b*33 + w]
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int a = e / n, b = e % n;
        Ms[e] = forward ? Q[(size_t)b * n + a] : Q[(size_t)a * n + b];
    }
    long long o0, i0;
    int wcount;
    if (inner > 1) {
        const long long tiles = (inner + 31) / 32;
        o0 = blockIdx.x / tiles;
        i0 = (blockIdx.x % tiles) * 32;
        wcount = (int)min(32LL, inner - i0);
    } else {
        o0 = (long long)blockIdx.x * 32;
        i0 = 0;
        wcount = (int)min(32LL, outer - o0);
    }
    // load
    for (int e = threadIdx.x; e < n * 32; e += blockDim.x) {
        int b, w;
        if (inner > 1) { b = e / 32; w = e % 32; }
        else { w = e / n; b = e % n; }
        double v = 0.0;
        if (w < wcount) {
            const long long addr = inner > 1 ? (o0 * n + b) * inner + i0 + w : (o0 + w) * n + b;
            v = in[addr];
        }
        X[b * 33 + w] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * 32; e += blockDim.x) {
        int a, w;
        if (inner > 1) { a = e / 32; w = e % 32; }
        else { w = e / n; a = e % n; }
        if (w >= wcount) continue;
        double acc = 0.0;
        for (int b = 0; b < n; ++b) acc += Ms[a * n + b] * X[b * 33 + w];
        const long long addr = inner > 1 ? (o0 * n + a) * inner + i0 + w : (o0 + w) * n + a;
        if (scale) acc *= scale[addr % nd];
        out[addr] = acc;
    }
}

// Pointwise factor (4 pi / lam)^power of nu^power in the eigenbasis; lam = 0 only for the G = 0
// mode of a periodic grid, which nu^power maps to zero.
__global__ void k_scale_grid(const double *__restrict__ lam, double *__restrict__ sc, long long nd, double power) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nd) sc[i] = lam[i] > 0.0 ? pow(4.0 * 3.14159265358979323846, power) * pow(lam[i], -power) : 0.0;
}

}  // namespace

void coulomb_setup(Ctx &c) {
    const int dims[3] = {c.nx, c.ny, c.nz};
    std::vector<double> mu[3];
    for (int a = 0; a < 3; ++a) {
        const int n = dims[a];
        std::vector<double> K((size_t)n * n, 0.0), Q;
        // K = -D, D the 1D second difference with weights w_k / h^2;  c.coef.a = -w/(2h^2).
        // Dirichlet: taps past the ends are dropped (Toeplitz); periodic: taps wrap, and taps
        // that land on the same point add up (circulant).
        for (int i = 0; i < n; ++i)
            for (int d = -kRadius; d <= kRadius; ++d) {
                int j = i + d;
                if (c.opt.periodic) j = ((j % n) + n) % n;
                else if (j < 0 || j >= n) continue;
                K[(size_t)i * n + j] += 2.0 * c.coef.a[std::abs(d)];
            }
        jacobi_eigh(K, n, mu[a], Q);
        if (c.opt.periodic) {
            // one zero eigenvalue (the constant mode), returned to rounding: made exactly zero so
            // that the G = 0 mode of the 3D operator is the one point where lam = 0
            double top = 0.0;
            for (double m : mu[a]) top = std::max(top, std::fabs(m));
            int zi = 0;
            for (int i = 1; i < n; ++i)
                if (std::fabs(mu[a][i]) < std::fabs(mu[a][zi])) zi = i;
            if (!(std::fabs(mu[a][zi]) <= 1e-10 * top)) fail(RPA_ERR_INVALID, "periodic 1D Laplacian: no zero mode (n=%d)", n);
            mu[a][zi] = 0.0;
            for (int i = 0; i < n; ++i)
                if (i != zi && !(mu[a][i] > 0.0)) fail(RPA_ERR_INVALID, "periodic 1D Laplacian not semidefinite (n=%d)", n);
        } else {
            for (double m : mu[a])
                if (!(m > 0.0)) fail(RPA_ERR_INVALID, "1D Laplacian not positive definite (n=%d)", n);
        }
        RPA_CUDA(cudaMalloc(&c.Q[a], sizeof(double) * n * n));
        RPA_CUDA(cudaMemcpy(c.Q[a], Q.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice));
        // the same factors for the Laplacian preconditioner of COCG, in FP64 and FP32
        std::vector<float> qf(Q.begin(), Q.end()), mf(mu[a].begin(), mu[a].end());
        RPA_CUDA(cudaMalloc(&c.mu[a], sizeof(double) * n));
        RPA_CUDA(cudaMemcpy(c.mu[a], mu[a].data(), sizeof(double) * n, cudaMemcpyHostToDevice));
        RPA_CUDA(cudaMalloc(&c.Qf[a], sizeof(float) * n * n));
        RPA_CUDA(cudaMemcpy(c.Qf[a], qf.data(), sizeof(float) * n * n, cudaMemcpyHostToDevice));
        RPA_CUDA(cudaMalloc(&c.muf[a], sizeof(float) * n));
        RPA_CUDA(cudaMemcpy(c.muf[a], mf.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    }
    std::vector<double> lam((size_t)c.nd);
    for (int k = 0; k < c.nz; ++k)
        for (int j = 0; j < c.ny; ++j)
            for (int i = 0; i < c.nx; ++i)
                lam[(size_t)i + (size_t)c.nx * (j + (size_t)c.ny * k)] = mu[0][i] + mu[1][j] + mu[2][k];
    RPA_CUDA(cudaMalloc(&c.lam, sizeof(double) * c.nd));
    RPA_CUDA(cudaMemcpy(c.lam, lam.data(), sizeof(double) * c.nd, cudaMemcpyHostToDevice));
}

static void axis_pass(Ctx &c, int axis, const double *in, double *out, int ncols, int forward, const double *scale,
                      cudaStream_t s) {
    const int n = axis == 0 ? c.nx : axis == 1 ? c.ny : c.nz;
    const long long inner = axis == 0 ? 1 : axis == 1 ? c.nx : (long long)c.nx * c.ny;
    const long long outer = (long long)ncols * c.nd / ((long long)n * inner);
    const size_t sh = sizeof(double) * ((size_t)n * n + (size_t)n * 33);
    allow_dynamic_smem((const void *)k_axis, sh);   // rejects grid dimensions above ~150
    const long long blocks = inner > 1 ? outer * ((inner + 31) / 32) : (outer + 31) / 32;
    k_axis<<<(unsigned)blocks, 256, sh, s>>>(in, out, c.Q[axis], n, inner, outer, forward, scale, c.nd);
    RPA_LAUNCH("coulomb axis transform");
}

// Fixed scratch for rpa_coulomb_apply_noalloc.  Every device that loads the library holds
// RPA_STATIC_SCRATCH_BYTES of it until the process exits.  In host code the symbol is only a
// stand-in: the device address is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[RPA_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (looked up on first use).
void *static_scratch(int dev) {
    if (dev < 0 || dev >= kMaxDevices) fail(RPA_ERR_INVALID, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        RPA_CUDA(cudaGetSymbolAddress(&ptr, g_static_scratch));
        g_scratch_addr[dev] = ptr;
    }
    return g_scratch_addr[dev];
}
}  // namespace

// The same per-axis transform as a batch of tensor-core contractions (tc_gemm_batched):
//   axis x: one contraction, rows (o) of length n_x times M^T;
//   axis y: one contraction per (column, z) slab, M (n_y x n_y) times the slab (n_y x n_x);
//   axis z: one contraction per column, M (n_z x n_z) times the column (n_z x n_x n_y),
// with M = Q^T (forward) or Q (back), Q[i*n+a] row-major.
static void axis_pass_tc(Ctx &c, int axis, const double *in, double *out, int ncols, int forward,
                         const double *scale, cudaStream_t s) {
    const int n = axis == 0 ? c.nx : axis == 1 ? c.ny : c.nz;
    const double *Q = c.Q[axis];
    // M(a, b) = Q[b][a] (forward) or Q[a][b] (back): element strides of (a, b)
    const long long ma = forward ? 1 : n, mb = forward ? n : 1;
    if (axis == 0) {
        const long long rows = (long long)ncols * c.nd / n;
        if (rows > (long long)INT32_MAX) fail(RPA_ERR_INVALID, "too many rows for the tensor-core transform");
        // D[o][a] = sum_b in[o][b] M(a, b): A = in (rows o, k = b), B(a, b) = M(a, b)
        tc_gemm_batched(in, n, 1, 0, Q, ma, mb, 0, (int)rows, n, n, out, n, 1, 1, 1, scale, c.nd, s, c.d_tc_err);
    } else if (axis == 1) {
        const long long slab = (long long)n * c.nx;
        const long long batch = (long long)ncols * c.nz;
        // D_o[a][i] = sum_b M(a, b) in_o[b][i]: A(a, b) = M(a, b), B(i, b) = in_o[b][i]
        for (long long z0 = 0; z0 < batch; z0 += 65535) {
            const int nb = (int)std::min<long long>(65535, batch - z0);
            tc_gemm_batched(Q, ma, mb, 0, in + z0 * slab, 1, c.nx, slab, n, c.nx, n, out + z0 * slab, c.nx, 1, slab,
                            nb, scale, c.nd, s, c.d_tc_err);
        }
    } else {
        const long long plane = (long long)c.nx * c.ny;
        if (plane > (long long)INT32_MAX) fail(RPA_ERR_INVALID, "plane too large for the tensor-core transform");
        if (ncols > 65535) fail(RPA_ERR_INVALID, "too many columns for the tensor-core transform");
        tc_gemm_batched(Q, ma, mb, 0, in, 1, plane, c.nd, n, (int)plane, n, out, plane, 1, c.nd, ncols, scale, c.nd, s,
                        c.d_tc_err);
    }
}

static void coulomb_passes_tc(Ctx &c, double power, const double *in, double *out, int ncols, double *t1, double *t2,
                              double *sc, cudaStream_t s) {
    k_scale_grid<<<(unsigned)((c.nd + 255) / 256), 256, 0, s>>>(c.lam, sc, c.nd, power);
    RPA_LAUNCH("coulomb scale");
    count_launches(1);
    axis_pass_tc(c, 0, in, t1, ncols, 1, nullptr, s);
    axis_pass_tc(c, 1, t1, t2, ncols, 1, nullptr, s);
    axis_pass_tc(c, 2, t2, t1, ncols, 1, sc, s);
    axis_pass_tc(c, 2, t1, t2, ncols, 0, nullptr, s);
    axis_pass_tc(c, 1, t2, t1, ncols, 0, nullptr, s);
    axis_pass_tc(c, 0, t1, out, ncols, 0, nullptr, s);
}

static void coulomb_passes(Ctx &c, double power, const double *in, double *out, int ncols, double *t1, double *t2,
                           double *sc, cudaStream_t s) {
    k_scale_grid<<<(unsigned)((c.nd + 255) / 256), 256, 0, s>>>(c.lam, sc, c.nd, power);
    RPA_LAUNCH("coulomb scale");
    count_launches(7);   // scale + six axis passes
    axis_pass(c, 0, in, t1, ncols, 1, nullptr, s);
    axis_pass(c, 1, t1, t2, ncols, 1, nullptr, s);
    axis_pass(c, 2, t2, t1, ncols, 1, sc, s);
    axis_pass(c, 2, t1, t2, ncols, 0, nullptr, s);
    axis_pass(c, 1, t2, t1, ncols, 0, nullptr, s);
    axis_pass(c, 0, t1, out, ncols, 0, nullptr, s);
}

void coulomb_apply_noalloc(Ctx &c, double power, const double *in, double *out, int ncols, cudaStream_t s) {
    if (ncols <= 0) return;
    const size_t blk = (sizeof(double) * (size_t)ncols * c.nd + 255) / 256 * 256;
    const size_t need = 2 * blk + sizeof(double) * (size_t)c.nd;
    if (need > (size_t)RPA_STATIC_SCRATCH_BYTES)
        fail(RPA_ERR_INVALID, "rpa_coulomb_apply_noalloc: %d columns of %lld points need %zu bytes of scratch, "
                              "more than the fixed %zu", ncols, c.nd, need, (size_t)RPA_STATIC_SCRATCH_BYTES);
    int dev = 0;
    RPA_CUDA(cudaGetDevice(&dev));
    if (dev != c.device) fail(RPA_ERR_INVALID, "the current device is not the context's device");
    char *base = (char *)static_scratch(dev);
    double *t1 = (double *)base, *t2 = (double *)(base + blk), *sc = (double *)(base + 2 * blk);
    // every scratch word is written before it is read: nothing needs clearing
    coulomb_passes(c, power, in, out, ncols, t1, t2, sc, s);
}

void coulomb_apply(Ctx &c, double power, const double *in, double *out, int ncols, cudaStream_t s, bool tensor) {
    if (ncols <= 0) return;
    const size_t blk = sizeof(double) * (size_t)ncols * c.nd;
    char *base = (char *)c.coul_tmp.ensure(2 * blk + sizeof(double) * c.nd);
    double *t1 = (double *)base, *t2 = (double *)(base + blk), *sc = (double *)(base + 2 * blk);
    if (tensor)
        coulomb_passes_tc(c, power, in, out, ncols, t1, t2, sc, s);
    else
        coulomb_passes(c, power, in, out, ncols, t1, t2, sc, s);
}

}  // namespace rpa

// Dense FP64 kernels of the subspace step (Algorithm 1 of arXiv 2504.01816): projection
// C = V^T R, overlap M = R^T R, Cholesky L L^T = M, the inverse L^{-1} used for
// V = R L^{-T}, and the Rayleigh-Ritz eigenvalues of the symmetric N_r x N_r matrix C with
// the energy sum E = w sum_i [log(1 - lambda_i) + lambda_i] (Eq. 10).
//
// Blocks of grid functions are stored as rows (row c = column c of the N_d x K matrix), so
// V^T R becomes G = V R^T over rows.  Long contractions are split over the grid and the
// partial sums are added in a fixed order (deterministic).
#include <cmath>

#include "internal.cuh"

namespace rpa {

namespace {

constexpr int kTile = 32;     // output tile of the Gram kernel
constexpr int kKc = 32;       // contraction chunk staged in shared memory
constexpr int kEigThreads = 256;   // one block for the small Rayleigh-Ritz eigenproblem

// partial[z][a][b] = sum_{r in chunk z} A[a][r] B[b][r]
__global__ void __launch_bounds__(256) k_gram(const double *__restrict__ A, int na, const double *__restrict__ B,
                                              int nb, long long len, long long chunk, double *__restrict__ part) {
    __shared__ double sa[kKc][kTile + 1];
    __shared__ double sb[kKc][kTile + 1];
    const int a0 = blockIdx.x * kTile, b0 = blockIdx.y * kTile;
    const long long r0 = (long long)blockIdx.z * chunk;
    const long long r1 = min(len, r0 + chunk);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, 2 x 2 outputs each
    double acc[2][2] = {{0, 0}, {0, 0}};
    for (long long rb = r0; rb < r1; rb += kKc) {
        for (int e = threadIdx.x; e < kTile * kKc; e += 256) {
            const int row = e / kKc, kk = e % kKc;
            const long long r = rb + kk;
            sa[kk][row] = (a0 + row < na && r < r1) ? A[(long long)(a0 + row) * len + r] : 0.0;
            sb[kk][row] = (b0 + row < nb && r < r1) ? B[(long long)(b0 + row) * len + r] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kKc; ++kk) {
            const double x0 = sa[kk][ty], x1 = sa[kk][ty + 16];
            const double y0 = sb[kk][tx], y1 = sb[kk][tx + 16];
            acc[0][0] += x0 * y0;
            acc[0][1] += x0 * y1;
            acc[1][0] += x1 * y0;
            acc[1][1] += x1 * y1;
        }
        __syncthreads();
    }
    double *out = part + (long long)blockIdx.z * na * nb;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int a = a0 + ty + 16 * u, b = b0 + tx + 16 * v;
            if (a < na && b < nb) out[(long long)a * nb + b] = acc[u][v];
        }
}

__global__ void k_sum_splits(const double *__restrict__ part, int splits, long long n, double *__restrict__ G) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < splits; ++z) s += part[(long long)z * n + e];
        G[e] = s;
    }
}

// Y[c][r] = sum_k S[c][k] X[k][r]; blockIdx.y picks 16 output rows.
__global__ void __launch_bounds__(256) k_combine(const double *__restrict__ S, int nc, int nk,
                                                 const double *__restrict__ X, long long len, double *__restrict__ Y) {
    extern __shared__ double ssh[];    // 16 x nk
    const int c0 = blockIdx.y * 16;
    for (int e = threadIdx.x; e < 16 * nk; e += blockDim.x) {
        const int c = e / nk, k = e % nk;
        ssh[e] = (c0 + c < nc) ? S[(long long)(c0 + c) * nk + k] : 0.0;
    }
    __syncthreads();
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < len; r += (long long)gridDim.x * blockDim.x) {
        double acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = 0.0;
        for (int k = 0; k < nk; ++k) {
            const double x = X[(long long)k * len + r];
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] += ssh[c * nk + k] * x;
        }
#pragma unroll
        for (int c = 0; c < 16; ++c)
            if (c0 + c < nc) Y[(long long)(c0 + c) * len + r] = acc[c];
    }
}

// In-place Cholesky (lower) of an n x n row-major SPD matrix by one block.
__global__ void __launch_bounds__(1024) k_cholesky(double *__restrict__ M, int n, int *__restrict__ info) {
    __shared__ int bad;
    __shared__ double floor_;
    if (threadIdx.x == 0) {
        // a pivot at or below n * eps * max diagonal means the columns are linearly dependent
        double mx = 0.0;
        for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(M[(long long)i * n + i]));
        floor_ = (double)n * 2.220446049250313e-16 * mx;
        bad = 0;
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            const double d = M[(long long)j * n + j];
            if (!(d > floor_) || !isfinite(d)) bad = j + 1;
            else M[(long long)j * n + j] = sqrt(d);
        }
        __syncthreads();
        if (bad) break;
        const double piv = M[(long long)j * n + j];
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) M[(long long)i * n + j] /= piv;
        __syncthreads();
        const int m = n - j - 1;                       // trailing block (j+1..n-1)^2, lower part
        for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
            const int i = j + 1 + (int)(e / m), k = j + 1 + (int)(e % m);
            if (k <= i) M[(long long)i * n + k] -= M[(long long)i * n + j] * M[(long long)k * n + j];
        }
        __syncthreads();
    }
    if (!bad)
        for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
            const int i = (int)(e / n), k = (int)(e % n);
            if (k > i) M[e] = 0.0;
        }
    if (threadIdx.x == 0) *info = bad;
}

// Linv = L^{-1} for lower-triangular L; one thread per column (forward substitution).
__global__ void k_tri_inverse(const double *__restrict__ L, int n, double *__restrict__ X) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    for (int i = 0; i < n; ++i) {
        if (i < c) {
            X[(long long)i * n + c] = 0.0;
            continue;
        }
        double s = (i == c) ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) s -= L[(long long)i * n + k] * X[(long long)k * n + c];
        X[(long long)i * n + c] = s / L[(long long)i * n + i];
    }
}

__global__ void k_symmetrize(double *C, int n) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    const int i = (int)(e / n), k = (int)(e % n);
    if (k > i) {
        const double v = 0.5 * (C[(long long)i * n + k] + C[(long long)k * n + i]);
        C[(long long)i * n + k] = v;
        C[(long long)k * n + i] = v;
    }
}

// Householder reduction of the symmetric matrix A (n x n, row-major, destroyed) to tridiagonal
// form, written to work[0..2n) (diagonal, off-diagonal) for k_sturm_bisect; k_eig_energy then sums
// the energy in ascending order.  One block.  work: 3n doubles.
// With use_smem the matrix and the work vectors are copied to shared memory first (n^2 + 3n
// doubles); A is then left unchanged.  (The eigenvalues by bisection in this block, one thread
// each, took ~2.3 ms for n = 64 on the FP64 pipe of one SM; one warp per eigenvalue over n SMs, by
// multisection, takes a few tens of microseconds.)
__global__ void __launch_bounds__(kEigThreads) k_sym_eigvals(double *__restrict__ Ag, int n, double *__restrict__ lam,
                                                             double *__restrict__ workg, double weight,
                                                             double *__restrict__ e_out, int use_smem) {
    __shared__ double red[32];
    __shared__ double sh_scalar[2];
    extern __shared__ double dyn[];
    const int tid = threadIdx.x, nt = blockDim.x;
    double *A = Ag, *work = workg;
    if (use_smem) {
        A = dyn;
        work = dyn + (size_t)n * n;
        for (long long e = tid; e < (long long)n * n; e += nt) A[e] = Ag[e];
        __syncthreads();
    }
    double *v = work;           // Householder vector (length n, entries k+1..n-1 used)
    double *p = work + n;       // A v
    auto block_sum = [&](double x) -> double {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((tid & 31) == 0) red[tid >> 5] = x;
        __syncthreads();
        double t = 0.0;
        if (tid == 0) {
            for (int w = 0; w < (nt + 31) / 32; ++w) t += red[w];
            sh_scalar[0] = t;
        }
        __syncthreads();
        t = sh_scalar[0];
        __syncthreads();
        return t;
    };
    for (int k = 0; k + 2 < n; ++k) {
        // x = A[k+1..n-1][k]
        double part = 0.0;
        for (int i = k + 1 + tid; i < n; i += nt) {
            const double x = A[(long long)i * n + k];
            part += x * x;
        }
        const double xnorm = sqrt(block_sum(part));
        const double x0 = A[(long long)(k + 1) * n + k];
        if (xnorm == 0.0) continue;
        const double alpha = x0 > 0 ? -xnorm : xnorm;
        for (int i = k + 1 + tid; i < n; i += nt) v[i] = A[(long long)i * n + k] - (i == k + 1 ? alpha : 0.0);
        __syncthreads();
        part = 0.0;
        for (int i = k + 1 + tid; i < n; i += nt) part += v[i] * v[i];
        const double vv = block_sum(part);
        if (vv == 0.0) continue;
        // p = (2/vv) A22 v
        for (int i = k + 1 + tid; i < n; i += nt) {
            double s = 0.0;
            for (int j = k + 1; j < n; ++j) s += A[(long long)i * n + j] * v[j];
            p[i] = 2.0 * s / vv;
        }
        __syncthreads();
        part = 0.0;
        for (int i = k + 1 + tid; i < n; i += nt) part += v[i] * p[i];
        const double K = block_sum(part) / vv;
        for (int i = k + 1 + tid; i < n; i += nt) p[i] -= K * v[i];     // q
        __syncthreads();
        const int m = n - k - 1;
        for (long long e = tid; e < (long long)m * m; e += nt) {
            const int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
            A[(long long)i * n + j] -= v[i] * p[j] + p[i] * v[j];
        }
        __syncthreads();
        if (tid == 0) {
            A[(long long)(k + 1) * n + k] = alpha;
            A[(long long)k * n + k + 1] = alpha;
        }
        __syncthreads();
    }
    // the tridiagonal matrix to global memory for the bisection kernel: diagonal, then off-diagonal
    for (int i = tid; i < n; i += nt) {
        workg[i] = A[(long long)i * n + i];
        workg[n + i] = (i + 1 < n) ? A[(long long)(i + 1) * n + i] : 0.0;
    }
}

// Eigenvalue t = blockIdx.x of the symmetric tridiagonal matrix (diagonal tri[0..n), off-diagonal
// tri[n..2n)), ascending, by multisection on Sturm counts: the warp's 32 lanes count the eigenvalues
// below 32 points splitting the interval into 33 parts, the interval shrinks to the part where the
// count passes t (5 bits per step), until it reaches machine precision.  One warp per eigenvalue,
// so the eigenvalues run on different SMs.
__global__ void __launch_bounds__(32) k_sturm_bisect(const double *__restrict__ tri, int n, double *__restrict__ lam) {
    const int t = blockIdx.x, lane = threadIdx.x;
    const double *d = tri, *e = tri + n;
    // Gershgorin bounds
    double lo = 1e300, hi = -1e300;
    for (int i = lane; i < n; i += 32) {
        const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const double pad = 1e-12 * fmax(1.0, fmax(fabs(lo), fabs(hi)));
    lo -= pad;
    hi += pad;
    for (int it = 0; it < 40; ++it) {
        const double w = (hi - lo) / 33.0;
        if (!(lo + w > lo) || !(hi - w < hi)) break;   // the interval is at machine precision
        const double x = lane == 31 ? hi - w : lo + (lane + 1) * w;
        int cnt = 0;                                     // eigenvalues below x
        double q = d[0] - x;
        if (q < 0) ++cnt;
        for (int i = 1; i < n; ++i) {
            if (q == 0.0) q = 1e-300;
            q = d[i] - x - e[i - 1] * e[i - 1] / q;
            if (q < 0) ++cnt;
        }
        const unsigned above = __ballot_sync(0xffffffffu, cnt > t);   // points past eigenvalue t
        const double xprev = __shfl_up_sync(0xffffffffu, x, 1);
        if (above == 0u) {
            lo = __shfl_sync(0xffffffffu, x, 31);
        } else {
            const int f = __ffs(above) - 1;
            const double xf = __shfl_sync(0xffffffffu, x, f);
            const double xl = __shfl_sync(0xffffffffu, xprev, f);
            if (f > 0) lo = xl;
            hi = xf;
        }
    }
    if (lane == 0) lam[t] = 0.5 * (lo + hi);
}

// E = weight * sum_i [log(1 - lambda_i) + lambda_i], in index order (one thread).
__global__ void k_eig_energy(const double *__restrict__ lam, int n, double weight, double *__restrict__ e_out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += log1p(-lam[i]) + lam[i];
        *e_out = weight * s;
    }
}

// Gauss spectral quadrature of Tr g(C), g(x) = log(1 - x) + x (Section "Implementation",
// Algorithm 1).  Block r runs n_o Lanczos steps with C from the basis vector e_r; the resulting
// tridiagonal J (alpha, beta) is the Jacobi matrix of a Gauss rule whose nodes are its
// eigenvalues (bisection on Sturm counts) and whose weights are the squared first components
// of its eigenvectors, here 1 / sum_k p_k(theta)^2 with the orthonormal polynomials
// p_0 = 1, beta_k p_{k+1} = (theta - alpha_k) p_k - beta_{k-1} p_{k-1} (Golub-Welsch).  A run
// whose Krylov space is exhausted (beta <= 1e-13 max|C|) stops early; its rule is then exact.
// part[r] = e_r^T g(C) e_r as the rule gives it.
constexpr int kSqThreads = 128;
__global__ void __launch_bounds__(kSqThreads) k_sq_trace(const double *__restrict__ C, int n, int n_o,
                                                         double *__restrict__ part) {
    extern __shared__ double sq_sh[];
    double *qp = sq_sh, *q = sq_sh + n, *w = sq_sh + 2 * n;
    __shared__ double al[kMaxSqOrder], be[kMaxSqOrder], red[kSqThreads / 32];
    __shared__ int m_sh;
    const int r = blockIdx.x, tid = threadIdx.x;
    auto bsum = [&](double x) -> double {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = x;
        __syncthreads();
        double s = 0.0;
        for (int i = 0; i < kSqThreads / 32; ++i) s += red[i];
        return s;
    };
    double mx = 0.0;
    for (long long e = tid; e < (long long)n * n; e += kSqThreads) mx = fmax(mx, fabs(C[e]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    double scale = 0.0;
    for (int i = 0; i < kSqThreads / 32; ++i) scale = fmax(scale, red[i]);
    for (int i = tid; i < n; i += kSqThreads) {
        qp[i] = 0.0;
        q[i] = (i == r) ? 1.0 : 0.0;
    }
    __syncthreads();
    int m = 0;
    double b = 0.0;
    for (int k = 0; k < n_o; ++k) {
        double part_a = 0.0;
        for (int i = tid; i < n; i += kSqThreads) {
            double s = -b * qp[i];
            for (int j = 0; j < n; ++j) s += C[(long long)i * n + j] * q[j];
            w[i] = s;
            part_a += q[i] * s;
        }
        const double a = bsum(part_a);
        m = k + 1;
        if (tid == 0) al[k] = a;
        if (k == n_o - 1) break;
        double part_b = 0.0;
        for (int i = tid; i < n; i += kSqThreads) {
            w[i] -= a * q[i];
            part_b += w[i] * w[i];
        }
        b = sqrt(bsum(part_b));
        if (!(b > 1e-13 * scale)) break;
        if (tid == 0) be[k] = b;
        for (int i = tid; i < n; i += kSqThreads) {
            qp[i] = q[i];
            q[i] = w[i] / b;
        }
        __syncthreads();
    }
    if (tid == 0) m_sh = m;
    __syncthreads();
    m = m_sh;
    double contrib = 0.0;
    if (tid < m) {
        // Gershgorin interval of J, then bisection for its (tid)-th smallest eigenvalue
        double lo = 1e300, hi = -1e300;
        for (int i = 0; i < m; ++i) {
            const double rad = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < m ? fabs(be[i]) : 0.0);
            lo = fmin(lo, al[i] - rad);
            hi = fmax(hi, al[i] + rad);
        }
        const double pad = 1e-12 * fmax(1.0, fmax(fabs(lo), fabs(hi)));
        lo -= pad;
        hi += pad;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            int cnt = 0;
            double d = al[0] - mid;
            if (d < 0) ++cnt;
            for (int i = 1; i < m; ++i) {
                if (d == 0.0) d = 1e-300;
                d = al[i] - mid - be[i - 1] * be[i - 1] / d;
                if (d < 0) ++cnt;
            }
            if (cnt > tid) hi = mid;
            else lo = mid;
        }
        const double th = 0.5 * (lo + hi);
        // weight 1 / sum_k p_k(theta)^2
        double p0 = 1.0, p1 = 0.0, ssq = 1.0;
        for (int k = 0; k + 1 < m; ++k) {
            const double pn = ((th - al[k]) * p0 - (k > 0 ? be[k - 1] * p1 : 0.0)) / be[k];
            p1 = p0;
            p0 = pn;
            ssq += pn * pn;
        }
        contrib = (log1p(-th) + th) / ssq;
    }
    const double s = bsum(contrib);
    if (tid == 0) part[r] = s;
}

// e_out = weight * sum_r part[r], in order.
__global__ void k_sq_sum(const double *__restrict__ part, int n, double weight, double *__restrict__ e_out) {
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += part[r];
    *e_out = weight * s;
}

// Symmetric eigendecomposition A = Q diag(w) Q^T of an n x n matrix (row-major, destroyed) by the
// cyclic Jacobi method in parallel (round-robin) order, one block: in each of the n' - 1 rounds of a
// sweep (n' = n rounded up to even) the n'/2 disjoint index pairs of a round-robin tournament are
// rotated together -- rotation angles from the current 2 x 2 blocks, then all column updates
// A <- A J, Q <- Q J, then all row updates A <- J^T A.  Sweeps stop when the off-diagonal part falls
// below 1e-30 of the whole (squared) or after 100 sweeps.  Q[i*n+a] = component i of eigenvector a;
// w[a] = A[a][a].  work: 2 n' doubles (cosines, sines) and n' ints (the tournament).
__global__ void __launch_bounds__(1024) k_jacobi_eigh(double *__restrict__ A, int n, double *__restrict__ Q,
                                                      double *__restrict__ w, double *__restrict__ cs,
                                                      int *__restrict__ perm) {
    __shared__ double red[32];
    __shared__ double tot_sh, off_sh;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int m = n + (n & 1);                 // an odd n gets a dummy index n (no rotation)
    const int half = m / 2;
    double *sn = cs + half;
    for (long long e = tid; e < (long long)n * n; e += nt) Q[e] = (e / n == e % n) ? 1.0 : 0.0;
    for (int i = tid; i < m; i += nt) perm[i] = i;
    __syncthreads();
    auto block_sum2 = [&](double a, double b) {
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if ((tid & 31) == 0) {
            red[tid >> 5] = a;
        }
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int k = 0; k < (nt + 31) / 32; ++k) t += red[k];
            tot_sh = t;
        }
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = b;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int k = 0; k < (nt + 31) / 32; ++k) t += red[k];
            off_sh = t;
        }
        __syncthreads();
    };
    for (int sweep = 0; sweep < 100; ++sweep) {
        double ta = 0.0, oa = 0.0;
        for (long long e = tid; e < (long long)n * n; e += nt) {
            const double a = A[e];
            ta += a * a;
            if (e / n != e % n) oa += a * a;
        }
        block_sum2(ta, oa);
        if (!(off_sh > 1e-30 * tot_sh)) break;
        for (int round = 0; round < m - 1; ++round) {
            // pair k: (perm[k], perm[m - 1 - k])
            for (int k = tid; k < half; k += nt) {
                int p = perm[k], q = perm[m - 1 - k];
                double c = 1.0, sg = 0.0;
                if (p < n && q < n) {
                    if (p > q) { const int t = p; p = q; q = t; }
                    const double apq = A[(long long)p * n + q];
                    if (apq != 0.0) {
                        const double theta = (A[(long long)q * n + q] - A[(long long)p * n + p]) / (2.0 * apq);
                        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        sg = t * c;
                    }
                }
                cs[k] = c;
                sn[k] = sg;
            }
            __syncthreads();
            // columns p, q of A and Q
            for (long long e = tid; e < (long long)n * half; e += nt) {
                const int row = (int)(e / half), k = (int)(e % half);
                int p = perm[k], q = perm[m - 1 - k];
                if (p >= n || q >= n) continue;
                if (p > q) { const int t = p; p = q; q = t; }
                const double c = cs[k], sg = sn[k];
                const double akp = A[(long long)row * n + p], akq = A[(long long)row * n + q];
                A[(long long)row * n + p] = c * akp - sg * akq;
                A[(long long)row * n + q] = sg * akp + c * akq;
                const double qkp = Q[(long long)row * n + p], qkq = Q[(long long)row * n + q];
                Q[(long long)row * n + p] = c * qkp - sg * qkq;
                Q[(long long)row * n + q] = sg * qkp + c * qkq;
            }
            __syncthreads();
            // rows p, q of A
            for (long long e = tid; e < (long long)n * half; e += nt) {
                const int col = (int)(e / half), k = (int)(e % half);
                int p = perm[k], q = perm[m - 1 - k];
                if (p >= n || q >= n) continue;
                if (p > q) { const int t = p; p = q; q = t; }
                const double c = cs[k], sg = sn[k];
                const double apk = A[(long long)p * n + col], aqk = A[(long long)q * n + col];
                A[(long long)p * n + col] = c * apk - sg * aqk;
                A[(long long)q * n + col] = sg * apk + c * aqk;
            }
            __syncthreads();
            // next round of the tournament: index 0 stays, the others rotate by one place
            if (tid == 0) {
                const int last = perm[m - 1];
                for (int i = m - 1; i > 1; --i) perm[i] = perm[i - 1];
                perm[1] = last;
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < n; i += nt) w[i] = A[(long long)i * n + i];
}

// The adjoint's rotation to Ritz vectors and weights: S[i][k] = Q[k][i] (row i of S combines the
// basis into Ritz vector i) and coef[i] = weight * g'(lambda_i), g'(x) = -x / (1 - x).
__global__ void k_ritz_rotation(const double *__restrict__ Q, const double *__restrict__ w, int n, double weight,
                                double *__restrict__ S, double *__restrict__ coef) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), k = (int)(e % n);
        S[e] = Q[(long long)k * n + i];
        if (k == 0) coef[i] = weight * (-w[i] / (1.0 - w[i]));
    }
}

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

void jacobi_eigh_device(double *A, int n, double *Q, double *w, double *work, cudaStream_t s) {
    const int m = n + (n & 1);
    k_jacobi_eigh<<<1, 1024, 0, s>>>(A, n, Q, w, work, (int *)(work + m));
    RPA_LAUNCH("jacobi eigensolver");
    count_launches(1);
}

void ritz_rotation(const double *Q, const double *w, int n, double weight, double *S, double *coef, cudaStream_t s) {
    k_ritz_rotation<<<std::min<unsigned>(cdiv((long long)n * n, 256), 1024u), 256, 0, s>>>(Q, w, n, weight, S, coef);
    RPA_LAUNCH("ritz rotation");
    count_launches(1);
}

void gram(const double *A, int na, const double *B, int nb, long long len, double *G, cudaStream_t s,
          DevBuf &scratch) {
    const int ta = cdiv(na, kTile), tb = cdiv(nb, kTile);
    long long splits = std::max(1LL, std::min<long long>(len / 512, 1200 / std::max(1, ta * tb)));
    const long long chunk = ((len + splits - 1) / splits + kKc - 1) / kKc * kKc;
    splits = (len + chunk - 1) / chunk;
    double *part = (double *)scratch.ensure(sizeof(double) * (size_t)splits * na * nb);
    k_gram<<<dim3(ta, tb, (unsigned)splits), 256, 0, s>>>(A, na, B, nb, len, chunk, part);
    const long long n = (long long)na * nb;
    k_sum_splits<<<std::min<unsigned>(cdiv(n, 256), 4096u), 256, 0, s>>>(part, (int)splits, n, G);
    RPA_LAUNCH("gram");
    count_launches(2);
}

void combine_rows(const double *S, int nc, int nk, const double *X, long long len, double *Y, cudaStream_t s) {
    const size_t sh = sizeof(double) * 16 * nk;
    allow_dynamic_smem((const void *)k_combine, sh);
    k_combine<<<dim3(std::min<unsigned>(cdiv(len, 256), 2048u), cdiv(nc, 16)), 256, sh, s>>>(S, nc, nk, X, len, Y);
    RPA_LAUNCH("combine_rows");
    count_launches(1);
}

void cholesky(double *M, int n, int *dev_info, cudaStream_t s) {
    k_cholesky<<<1, 1024, 0, s>>>(M, n, dev_info);
    RPA_LAUNCH("cholesky");
    count_launches(1);
}

void tri_inverse(const double *L, int n, double *Linv, cudaStream_t s) {
    k_tri_inverse<<<cdiv(n, 64), 64, 0, s>>>(L, n, Linv);
    RPA_LAUNCH("tri_inverse");
    count_launches(1);
}

void symmetrize(double *C, int n, cudaStream_t s) {
    k_symmetrize<<<cdiv((long long)n * n, 256), 256, 0, s>>>(C, n);
    RPA_LAUNCH("symmetrize");
    count_launches(1);
}

void sq_trace(const double *C, int n, int n_o, double *part, double weight, double *e_out, cudaStream_t s) {
    const size_t sh = sizeof(double) * 3 * (size_t)n;
    allow_dynamic_smem((const void *)k_sq_trace, sh);
    k_sq_trace<<<n, kSqThreads, sh, s>>>(C, n, n_o, part);
    k_sq_sum<<<1, 1, 0, s>>>(part, n, weight, e_out);
    RPA_LAUNCH("sq_trace");
    count_launches(2);
}

void sym_eigvals(double *C, int n, double *lam, double *work, double weight, double *e_out, cudaStream_t s) {
    const size_t sh = sizeof(double) * ((size_t)n * n + 3 * (size_t)n);
    const bool use_smem = sh <= 200 * 1024;
    if (use_smem) allow_dynamic_smem((const void *)k_sym_eigvals, sh);
    k_sym_eigvals<<<1, kEigThreads, use_smem ? sh : 0, s>>>(C, n, lam, work, weight, e_out, use_smem ? 1 : 0);
    k_sturm_bisect<<<n, 32, 0, s>>>(work, n, lam);
    k_eig_energy<<<1, 32, 0, s>>>(lam, n, weight, e_out);
    RPA_LAUNCH("sym_eigvals");
    count_launches(3);
}

}  // namespace rpa

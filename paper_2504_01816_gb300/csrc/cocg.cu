// Batched COCG for the Sternheimer systems (H - eps_n + i omega) x = b of the real-space RPA
// method (arXiv 2504.01816: Sternheimer equation, Eq. 9; COCG, Section "Implementation").
//
// Persistent slot queue.  A fixed set of S slots holds the systems in flight; each slot owns
// its Krylov vectors and a small state record.  All systems of a call wait in a queue; when
// a slot's system is solved its contribution is retired (drho or the gradient accumulated, or
// x copied out) and the slot takes the next system.
//
// One COCG iteration over the slots of the active list is four launches:
//   k_beta:     one warp per slot: rho = r^T r and ||r|| from the partial sums of the last
//               update (fixed order), stopping test, beta = rho / rho_old, active list
//   k_cocg_pa:  p = r + beta p_old and q = (H - eps_n + i omega) p (12th-order stencil, z-marching
//               register window), partial sums of p^T q
//   k_alpha:    one warp per slot: alpha = rho / p^T q
//   k_cocg_b:   x += alpha p, r -= alpha q, partial sums of r^T r and ||r||^2
// Reductions are deterministic: every block writes its own partial sums; consumers add them in
// block order.  Groups of iterations ("epochs") are replayed as CUDA graphs; between epochs
// maintenance kernels refine, retire, refill and load slots.  The mixed form's fused kernel
// (k_cocg_ring, where a plane fits its shared-memory ring) replaces the four launches: one block
// owns one system, so one launch per epoch runs every active inner solve to its end.
//
// Plain form:  complex FP64 COCG to ||r|| <= tol ||b||.
// Mixed form:  FP64 iterative refinement around complex FP32 COCG: r64 = b - A x64 in FP64,
//              FP32 COCG for A d = r64 to a relative reduction inner_tol, x64 += d, repeat until
//              ||r64|| <= tol ||b||.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include <cooperative_groups.h>

#include "internal.cuh"

namespace rpa {

namespace {

constexpr int kThreads = 256;
constexpr int kPPT = 8;
constexpr int kChunk = kThreads * kPPT;   // grid points per work item
constexpr int kEpoch = 8;                 // COCG iterations between maintenance passes (even)
constexpr int kWarpsPerBlock = kThreads / 32;
// Near-breakdown of the FP32 inner solve (mixed form).  COCG divides by r^T r, an unconjugated
// form that can vanish for a nonzero complex r.  FP32 sums carry errors of ~1e-7..1e-6 of
// ||r||^2, so when |r^T r| falls below kNearBreak ||r||^2 the next beta = r_new^T r_new / r^T r
// is mostly rounding: the inner solve ends there and the FP64 refinement restarts it from the
// true residual.  For unrelated complex vectors of N_d >= 10^4 points the ratio is
// ~N_d^-1/2 >= 1e-3, so this is rare in a healthy solve.
constexpr double kNearBreak = 1e-5;

enum Phase : int { kEmpty = 0, kInner = 1, kInnerDone = 2, kFinished = 3, kLoading = 4 };

struct Slot {
    double rho_re[2], rho_im[2];    // r^T r of the last two iterations (by parity of the iteration)
    double alpha_re, alpha_im, beta_re, beta_im;
    double shift_re, shift_im;
    double bnorm, ref_norm, rnorm;  // ||b||; inner solve: norms of the scaled FP32 residual
    double scale;                   // mixed: the FP32 inner solve works on scale * (b - A x64)
    int phase, sys, n, j;
    int iters, total_iters, refines, status;
    int discard;                    // mixed: the inner solve went non-finite; its correction is dropped
    int nearbreak;                  // mixed: inner solves ended at a near-breakdown
};

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

struct Grid3 {
    int nx, ny, nz;
    long long nd;
    int periodic;                  // 1: periodic continuation outside the box, 0: zero values
};

// Grid index a (any integer) along an axis of n points, taken into [0, n) (periodic grids).
__device__ __forceinline__ int wrap_index(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

template <typename T> struct Coef {
    T a[kRadius + 1];
};

template <typename T> Coef<T> cast_coef(const StencilCoef &c) {
    Coef<T> r;
    for (int k = 0; k <= kRadius; ++k) r.a[k] = (T)c.a[k];
    return r;
}

// Everything the kernels need, passed by value.
struct Params {
    Slot *slots;
    int S, nblk;       // items per slot of the streaming kernels
    int nparta;        // partial sums per slot written by the stencil kernel (its tiles)
    Grid3 g;
    double *partA;     // [S][nparta][2] p^T q
    double *partB;     // [S][nblk][3]   r^T r (re, im), ||r||^2
    int *list;         // [2][S] active slots of the current iteration (by parity)
    int *cnt;          // [2]    their number
    int mixed;
    double tol, inner_tol;
    int maxit, max_refine;
    int *head;         // next system of the queue
    int nsys;
    int *count;        // slots busy + systems waiting (for the host)
    int *sys_out;      // [4][nsys] per system: iterations, status, refinements, near-breakdowns
    int *fin_list;     // [S] the finished slots of this maintenance pass, in slot order
    int *fin_cnt;      // their number
    unsigned long long *prof;   // grid points processed by k_cocg_p/_a/_b (nullptr = off)
    // occupied-space projection of finished solutions (x <- x - sum_k (u_k . x) u_k)
    int project, ns;
    const double *psi;          // ns x nd orbitals
    double *partP;              // [S][nblk][ns][2] partial u_k . x
    double *Tp;                 // [S][ns][2]       u_k . x
    // mixed form with projected right-hand sides: P_c on every FP32 correction and residual
    int cproject;
    int proj_re_only;           // only Re(u_k . x) is needed (the solutions retire into drho)
    float *Tp32;                // [S][ns][2]       Tp in FP32 (for FP32 updates)
    const float *psi32;         // ns x nd orbitals in FP32
    // Laplacian-preconditioned COCG: rho = r^T z from the per-plane partial sums of z = M r
    int precond;
    double *partZ;              // [S][nz][3] r^T z (re, im), ||z||^2
};

// The fields of Params that the two streaming kernels of the iteration read, passed on their
// own: with the whole Params struct their kernel parameter blocks reached 256 bytes, and
// k_cocg_b measured 18% slower from that size on (same code, same registers).
struct IterArgs {
    Slot *slots;
    const int *list;               // active slots of the iteration's parity
    const int *cnt;                // their number
    double *part;                  // per-item partial sums: [S][nper][k_cocg_pa: 2, k_cocg_b: 3]
    unsigned long long *prof;      // grid points processed (nullptr = off)
    long long nd;
    int nx, ny, nz;
    int nper;                      // work items per slot (stencil tiles, or chunks)
    int periodic;                  // 1: periodic continuation outside the box, 0: zero values
};

// Sum N doubles over the block; the result is valid in thread 0.  Fixed order.
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N]) {
    __shared__ double sh[N][kWarpsPerBlock];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    __syncthreads();   // sh may still be read from the previous item
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < N; ++c) sh[c][warp] = v[c];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < N; ++c) {
            v[c] = lane < kWarpsPerBlock ? sh[c][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
        }
    }
}

// Block sum in the working precision T (256 threads), converted to double once at the end;
// result valid in thread 0.  Fixed order.
template <typename T, int N>
__device__ __forceinline__ void block_sum_t(const T (&in)[N], double (&out)[N]) {
    __shared__ T sh[N][kWarpsPerBlock];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T v[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        v[c] = in[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < N; ++c) sh[c][warp] = v[c];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < N; ++c) out[c] = 0.0;
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < N; ++c) {
            T t = lane < kWarpsPerBlock ? sh[c][lane] : (T)0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            out[c] = (double)t;
        }
    }
}

// Sum one slot's per-item partials with one warp (fixed order); result in every lane.
template <int N, int STRIDE>
__device__ __forceinline__ void warp_slot_sum(const double *part, int nblk, double (&out)[N]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < N; ++c) out[c] = 0.0;
    for (int b = lane; b < nblk; b += 32)
#pragma unroll
        for (int c = 0; c < N; ++c) out[c] += part[(long long)b * STRIDE + c];
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) out[c] += __shfl_xor_sync(0xffffffffu, out[c], o);
}

// Grid coordinates of a point index (grid functions have < 2^31 points: 32-bit divisions).
__device__ __forceinline__ void coords(long long idx, const Grid3 &g, int &i, int &j, int &k) {
    const int id = (int)idx, pl = g.nx * g.ny;
    k = id / pl;
    const int rem = id - k * pl;
    j = rem / g.nx;
    i = rem - j * g.nx;
}

// ---------------------------------------------------------------------------------------------
// Laplacian preconditioner (rpa_options.precondition; paper, Section "Implementation": Laplacian-
// based preconditioning through the Kronecker product formalism).  z = M r with
//   M = (-1/2 L_h + s)^(-1) = Q diag(1 / (lam / 2 + s)) Q^T,  s = mean(V_loc) - eps_n + i omega,
// Q = Q_z x Q_y x Q_x and lam = mu_x + mu_y + mu_z the eigendecompositions of the 1D -D (those of
// the Coulomb operator), for every slot in its inner solve, in three passes over the slot's vector:
// the x and y transforms of every plane (k_pc_xy, forward), the z transform, the diagonal and the
// inverse z transform of every column (k_pc_z), the inverse x and y transforms (k_pc_xy, back, which
// also forms the partial sums of r^T z and ||z||^2 per plane).  Each transform is a small matrix
// product in shared memory with 2 x 4 outputs per thread.
// ---------------------------------------------------------------------------------------------
constexpr int kPcThreads = 256;

template <typename T> struct PcArgs {
    Slot *slots;
    int S, nx, ny, nz;
    long long nd;
    const T *Qx, *Qy, *Qz;         // n x n, Q[i n + a] = component i of eigenvector a
    const T *mux, *muy, *muz;      // their eigenvalues (of -D, the 1D factors of -L_h)
    double vbar;                   // mean V_loc, the constant potential of the preconditioner
    double *partZ;                 // [S][nz][3] per plane: r^T z (re, im), ||z||^2
};

// Bytes of the real 1D matrices at the start of the preconditioner kernels' shared memory, rounded
// up to 16 so that the complex arrays after them are aligned for their element type.
__host__ __device__ inline size_t pc_mat_bytes(size_t elems, size_t tsz) { return (elems * tsz + 15) / 16 * 16; }
constexpr int kPcTiles = 4;        // 2 x 4 output tiles per thread in k_pc_xy (planes of <= 4 x 256 tiles)
// Shared-memory bytes of k_pc_xy: the two 1D matrices and one complex plane (rows padded by one).
template <typename T> size_t pc_xy_bytes(int nx, int ny) {
    return pc_mat_bytes((size_t)nx * nx + (size_t)ny * ny, sizeof(T)) + sizeof(typename Cx<T>::t) * (size_t)ny * (nx + 1);
}
// acc += m x for a real m and a complex x (packed FP32x2 for float)
__device__ __forceinline__ void cmac(float2 &acc, float m, float2 x) { acc = __ffma2_rn(make_float2(m, m), x, acc); }
__device__ __forceinline__ void cmac(double2 &acc, double m, double2 x) {
    acc.x = fma(m, x.x, acc.x);
    acc.y = fma(m, x.y, acc.y);
}

// out(plane) = (M_y (x) M_x) in(plane) for every plane of every slot in its inner solve, with
// M = Q^T (FWD) or Q (back); back also sums r^T out and ||out||^2 per plane.  The x pass keeps its
// tiles in registers and writes them over the plane after a barrier (one plane buffer).
template <typename T, bool FWD>
__global__ void __launch_bounds__(kPcThreads) k_pc_xy(PcArgs<T> A, const typename Cx<T>::t *__restrict__ in,
                                                      typename Cx<T>::t *__restrict__ out,
                                                      const typename Cx<T>::t *__restrict__ r) {
    using C = typename Cx<T>::t;
    extern __shared__ double pc_sh[];
    const int nx = A.nx, ny = A.ny, W = nx + 1;
    T *const Mx = reinterpret_cast<T *>(pc_sh);          // Mx[i nx + a]: x pass Y[j][a] = sum_i X[j][i] Mx[i][a]
    T *const My = Mx + (size_t)nx * nx;                   // My[b ny + j]: y pass Z[b][a] = sum_j My[b][j] Y[j][a]
    C *const X = reinterpret_cast<C *>(reinterpret_cast<char *>(pc_sh) +
                                       pc_mat_bytes((size_t)nx * nx + (size_t)ny * ny, sizeof(T)));
    for (int e = threadIdx.x; e < nx * nx; e += blockDim.x) {
        const int i = e / nx, a = e - i * nx;
        Mx[e] = FWD ? A.Qx[(size_t)i * nx + a] : A.Qx[(size_t)a * nx + i];
    }
    for (int e = threadIdx.x; e < ny * ny; e += blockDim.x) {
        const int b = e / ny, j = e - b * ny;
        My[e] = FWD ? A.Qy[(size_t)j * ny + b] : A.Qy[(size_t)b * ny + j];
    }
    const int plane = nx * ny;
    const int tx = (nx + 3) / 4, ty = (ny + 1) / 2;      // 2 x 4 output tiles
    const C zc = C{0, 0};
    const long long items = (long long)A.S * A.nz;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = (int)(it / A.nz), k = (int)(it - (long long)s * A.nz);
        if (A.slots[s].phase != kInner) continue;         // uniform per block
        const long long base = (long long)s * A.nd + (long long)k * plane;
        __syncthreads();                                  // the previous item's readers are done
        for (int e = threadIdx.x; e < plane; e += blockDim.x) {
            const int j = e / nx, i = e - j * nx;
            X[j * W + i] = in[base + e];
        }
        __syncthreads();
        // x pass: Y = X Mx, tiles in registers
        C acc[kPcTiles][2][4];
#pragma unroll
        for (int u = 0; u < kPcTiles; ++u) {
            const int t = threadIdx.x + u * kPcThreads;
#pragma unroll
            for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[u][rr][q] = zc;
            if (t < tx * ty) {
                const int j0 = 2 * (t / tx), a0 = 4 * (t % tx);
                const int j1 = min(j0 + 1, ny - 1);          // a row past the plane repeats the last (discarded)
                for (int i = 0; i < nx; ++i) {
                    const C x0 = X[j0 * W + i], x1 = X[j1 * W + i];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const T m = a0 + q < nx ? Mx[i * nx + a0 + q] : (T)0;
                        cmac(acc[u][0][q], m, x0);
                        cmac(acc[u][1][q], m, x1);
                    }
                }
            }
        }
        __syncthreads();                                  // every thread has read X
#pragma unroll
        for (int u = 0; u < kPcTiles; ++u) {
            const int t = threadIdx.x + u * kPcThreads;
            if (t < tx * ty) {
                const int j0 = 2 * (t / tx), a0 = 4 * (t % tx);
#pragma unroll
                for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (j0 + rr < ny && a0 + q < nx) X[(j0 + rr) * W + a0 + q] = acc[u][rr][q];
            }
        }
        __syncthreads();
        // y pass: Z = My Y, written out; back: partial sums with r
        T d0 = 0, d1 = 0, d2 = 0;
#pragma unroll
        for (int u = 0; u < kPcTiles; ++u) {
            const int t = threadIdx.x + u * kPcThreads;
            if (t >= tx * ty) continue;
            const int b0 = 2 * (t / tx), a0 = 4 * (t % tx);
            C z[2][4];
#pragma unroll
            for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                for (int q = 0; q < 4; ++q) z[rr][q] = zc;
            for (int j = 0; j < ny; ++j) {
                const T m0 = My[b0 * ny + j], m1 = b0 + 1 < ny ? My[(b0 + 1) * ny + j] : (T)0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const C y = a0 + q < nx ? X[j * W + a0 + q] : zc;
                    cmac(z[0][q], m0, y);
                    cmac(z[1][q], m1, y);
                }
            }
#pragma unroll
            for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (b0 + rr < ny && a0 + q < nx) {
                        const long long g = base + (long long)(b0 + rr) * nx + a0 + q;
                        out[g] = z[rr][q];
                        if (!FWD) {
                            const C rv = r[g];
                            d0 += rv.x * z[rr][q].x - rv.y * z[rr][q].y;
                            d1 += rv.x * z[rr][q].y + rv.y * z[rr][q].x;
                            d2 += z[rr][q].x * z[rr][q].x + z[rr][q].y * z[rr][q].y;
                        }
                    }
        }
        if (!FWD) {
            const T dv[3] = {d0, d1, d2};
            double v[3];
            block_sum_t<T, 3>(dv, v);
            if (threadIdx.x == 0) {
                double *o = A.partZ + ((long long)s * A.nz + k) * 3;
                o[0] = v[0];
                o[1] = v[1];
                o[2] = v[2];
            }
        }
    }
}

// In place, for every column of every slot in its inner solve: the z transform (Q_z^T), the
// diagonal 1 / (lam / 2 + s), the inverse z transform (Q_z).  A block takes 32 consecutive
// columns; warp w forms the outputs c = w, w + 8, ... of its lane's column.
template <typename T>
__global__ void __launch_bounds__(kPcThreads) k_pc_z(PcArgs<T> A, typename Cx<T>::t *__restrict__ buf) {
    using C = typename Cx<T>::t;
    constexpr int kMaxPer = 12;                           // outputs per thread: nz <= 8 kMaxPer
    extern __shared__ double pc_sh[];
    const int nz = A.nz, plane = A.nx * A.ny;
    T *const Qz = reinterpret_cast<T *>(pc_sh);           // Qz[k nz + c]
    C *const X = reinterpret_cast<C *>(reinterpret_cast<char *>(pc_sh) + pc_mat_bytes((size_t)nz * nz, sizeof(T)));   // X[k * 33 + lane]
    for (int e = threadIdx.x; e < nz * nz; e += blockDim.x) Qz[e] = A.Qz[e];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tiles = (plane + 31) / 32;
    const long long items = (long long)A.S * tiles;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = (int)(it / tiles), p0 = (int)(it - (long long)s * tiles) * 32;
        const Slot &sl = A.slots[s];
        if (sl.phase != kInner) continue;                 // uniform per block
        const long long base = (long long)s * A.nd;
        const int p = p0 + lane;
        const bool own = p < plane;
        __syncthreads();
        for (int e = threadIdx.x; e < nz * 32; e += blockDim.x) {
            const int k = e >> 5, l = e & 31;
            X[k * 33 + l] = p0 + l < plane ? buf[base + (long long)k * plane + p0 + l] : C{0, 0};
        }
        __syncthreads();
        // forward and diagonal: W[c] = d_c sum_k Qz[k][c] X[k]
        T wr[kMaxPer], wi[kMaxPer];
#pragma unroll
        for (int m = 0; m < kMaxPer; ++m) wr[m] = wi[m] = 0;
        for (int k = 0; k < nz; ++k) {
            const C x = X[k * 33 + lane];
#pragma unroll
            for (int m = 0; m < kMaxPer; ++m) {
                const int c = warp + 8 * m;
                if (c < nz) {
                    const T q = Qz[k * nz + c];
                    wr[m] += q * x.x;
                    wi[m] += q * x.y;
                }
            }
        }
        const int iy = own ? p / A.nx : 0, ix = own ? p - iy * A.nx : 0;
        const T sr = (T)(A.vbar + sl.shift_re), si = (T)sl.shift_im;
        const T mxy = own ? A.mux[ix] + A.muy[iy] : (T)0;
#pragma unroll
        for (int m = 0; m < kMaxPer; ++m) {
            const int c = warp + 8 * m;
            if (c < nz) {
                const T dr = (T)0.5 * (mxy + A.muz[c]) + sr;
                const T inv = (T)1 / (dr * dr + si * si);
                const T fr = dr * inv, fi = -si * inv;                // 1 / (dr + i si)
                const T a = wr[m], b = wi[m];
                wr[m] = a * fr - b * fi;
                wi[m] = a * fi + b * fr;
            }
        }
        __syncthreads();                                  // every warp has read X
#pragma unroll
        for (int m = 0; m < kMaxPer; ++m) {
            const int c = warp + 8 * m;
            if (c < nz) X[c * 33 + lane] = C{wr[m], wi[m]};
        }
        __syncthreads();
        // inverse: Z[k] = sum_c Qz[k][c] W[c]
#pragma unroll
        for (int m = 0; m < kMaxPer; ++m) wr[m] = wi[m] = 0;
        for (int c = 0; c < nz; ++c) {
            const C w = X[c * 33 + lane];
#pragma unroll
            for (int m = 0; m < kMaxPer; ++m) {
                const int k = warp + 8 * m;
                if (k < nz) {
                    const T q = Qz[k * nz + c];
                    wr[m] += q * w.x;
                    wi[m] += q * w.y;
                }
            }
        }
        if (own)
#pragma unroll
            for (int m = 0; m < kMaxPer; ++m) {
                const int k = warp + 8 * m;
                if (k < nz) buf[base + (long long)k * plane + p] = C{wr[m], wi[m]};
            }
    }
}

// ---------------------------------------------------------------------------------------------
// COCG iteration: two per-slot scalar kernels (one warp per slot, the only writers of the slot
// state during the iteration) and three kernels over the active (slot, chunk) items.
// ---------------------------------------------------------------------------------------------
// rho = r^T r and ||r|| from the partial sums of the last update; convergence test; beta;
// append the slot to the active list of this iteration.
__global__ void k_beta(Params P, int par) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= P.S) return;
    Slot &sl = P.slots[w];
    if (sl.phase != kInner) return;
    double v[3];
    warp_slot_sum<3, 3>(P.partB + (long long)w * P.nblk * 3, P.nblk, v);
    double zz = v[2];                   // ||z||^2 (preconditioned), else ||r||^2
    if (P.precond) {                    // rho = r^T z, the stopping test on ||r||
        double vz[3];
        warp_slot_sum<3, 3>(P.partZ + (long long)w * P.g.nz * 3, P.g.nz, vz);
        v[0] = vz[0];
        v[1] = vz[1];
        zz = vz[2];
    }
    if (lane != 0) return;
    const int k = sl.iters;
    const double rn = sqrt(v[2]);
    const double thr =
        P.mixed ? fmax(P.inner_tol * sl.ref_norm, 0.3 * P.tol * sl.bnorm * sl.scale) : P.tol * sl.bnorm;
    const bool conv = rn <= thr;
    const double rr2 = v[0] * v[0] + v[1] * v[1];
    const bool nonfinite = !isfinite(rn) || !isfinite(rr2);
    const bool zero = !(rr2 > 0.0);
    const bool nearb = P.mixed && k > 0 && !(rr2 > kNearBreak * kNearBreak * v[2] * zz);
    sl.rnorm = rn;
    if (conv || k >= P.maxit || nonfinite || zero || nearb) {
        if (P.mixed) {
            // the inner solve ends; the refinement restarts it from the true residual unless it
            // went non-finite (its correction is dropped) or r^T r vanished at its start
            if (nonfinite) sl.discard = 1;
            if (!conv && (nonfinite || (zero && k == 0))) sl.status = RPA_ERR_BREAKDOWN;
            if (!conv && !nonfinite && nearb) sl.nearbreak += 1;
            sl.phase = kInnerDone;
        } else {
            sl.status = conv ? RPA_OK : ((nonfinite || zero) ? RPA_ERR_BREAKDOWN : RPA_ERR_NOT_CONVERGED);
            sl.phase = kFinished;
        }
        return;
    }
    double br = 0.0, bi = 0.0;
    if (k > 0) {
        const double orr = sl.rho_re[(k - 1) & 1], ori = sl.rho_im[(k - 1) & 1];
        const double den = orr * orr + ori * ori;
        br = (v[0] * orr + v[1] * ori) / den;
        bi = (v[1] * orr - v[0] * ori) / den;
    }
    sl.rho_re[k & 1] = v[0];
    sl.rho_im[k & 1] = v[1];
    sl.beta_re = br;
    sl.beta_im = bi;
    const int pos = atomicAdd(P.cnt + par, 1);
    P.list[par * P.S + pos] = w;
}

// alpha = rho / p^T q for the active slots; breakdown retires the slot; the iteration is
// counted.  Also clears the other parity's list counter for the next iteration.
__global__ void k_alpha(Params P, int par) {
    if (blockIdx.x == 0 && threadIdx.x == 0) P.cnt[par ^ 1] = 0;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= P.cnt[par]) return;
    const int s = P.list[par * P.S + w];
    Slot &sl = P.slots[s];
    double mu[2];
    warp_slot_sum<2, 2>(P.partA + (long long)s * P.nparta * 2, P.nparta, mu);
    if (lane != 0) return;
    const int k = sl.iters;
    const double den = mu[0] * mu[0] + mu[1] * mu[1];
    if (!(den > 0.0) || !isfinite(den)) {
        sl.status = RPA_ERR_BREAKDOWN;
        if (P.mixed && !isfinite(den)) sl.discard = 1;
        sl.phase = P.mixed ? kInnerDone : kFinished;
        return;
    }
    const double rr = sl.rho_re[k & 1], ri = sl.rho_im[k & 1];
    sl.alpha_re = (rr * mu[0] + ri * mu[1]) / den;
    sl.alpha_im = (ri * mu[0] - rr * mu[1]) / den;
    // the iteration is counted here, by the slot's single writer, before k_cocg_b reads it
    sl.iters = k + 1;
    sl.total_iters += 1;
}

// x += alpha p ; r -= alpha q ; partial sums of r^T r and ||r||^2
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cocg_b(IterArgs A, typename Cx<T>::t *__restrict__ x,
                                                     typename Cx<T>::t *__restrict__ r,
                                                     const typename Cx<T>::t *__restrict__ pbuf, long long pstride,
                                                     const typename Cx<T>::t *__restrict__ q) {
    using C = typename Cx<T>::t;
    const long long items = (long long)*A.cnt * A.nper;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = A.list[(int)(it / A.nper)], chunk = (int)(it % A.nper);
        Slot &sl = A.slots[s];
        if (sl.phase != kInner) continue;      // breakdown in k_alpha (stable during this kernel)
        const T ar = (T)sl.alpha_re, ai = (T)sl.alpha_im;
        const long long off = (long long)s * A.nd;
        const C *p = pbuf + (long long)(sl.iters & 1) * pstride;   // the new direction (iters counted in k_alpha)
        T a0 = 0, a1 = 0, a2 = 0;          // per-thread sums in the working precision (FP64 is slow)
#pragma unroll 4
        for (int t = 0; t < kPPT; ++t) {
            const long long idx = (long long)chunk * kChunk + t * kThreads + threadIdx.x;
            if (idx < A.nd) {
                const C pv = p[off + idx], qv = q[off + idx];
                C xv = x[off + idx], rv = r[off + idx];
                xv.x += ar * pv.x - ai * pv.y;
                xv.y += ar * pv.y + ai * pv.x;
                rv.x -= ar * qv.x - ai * qv.y;
                rv.y -= ar * qv.y + ai * qv.x;
                x[off + idx] = xv;
                r[off + idx] = rv;
                a0 += rv.x * rv.x - rv.y * rv.y;
                a1 += 2 * rv.x * rv.y;
                a2 += rv.x * rv.x + rv.y * rv.y;
            }
        }
        const T a[3] = {a0, a1, a2};
        double v[3];
        block_sum_t<T, 3>(a, v);
        if (threadIdx.x == 0) {
            double *o = A.part + ((long long)s * A.nper + chunk) * 3;
            o[0] = v[0];
            o[1] = v[1];
            o[2] = v[2];
        }
        if (A.prof && threadIdx.x == 0) {
            const long long left = A.nd - (long long)chunk * kChunk;
            atomicAdd(A.prof + 2, (unsigned long long)(left < kChunk ? left : kChunk));
        }
    }
}

// Block-wide sum for any block size (<= 1024 threads); result valid in thread 0.  Fixed order.
template <int N>
__device__ __forceinline__ void block_sum_any(double (&v)[N]) {
    __shared__ double sh[N][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < N; ++c) sh[c][warp] = v[c];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < N; ++c) {
            v[c] = lane < nw ? sh[c][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
        }
    }
}

// Tiling of the fused stencil kernel: xy tiles of tx x ty grid columns (one thread per column)
// and nzc chunks of zlen planes along z.
struct Tiles {
    int tx, ty, ntx, nty;
    int nzc, zlen;
};

// Fused direction update and stencil (one COCG half-step), for the slots of the active list:
//   p_new = r + beta p_old          (p is double-buffered per slot by iteration parity)
//   q     = (H - eps_n + i omega) p_new ,  partial sums of p_new^T q
// Work item = (slot, xy tile).  The block marches along z.  Each thread keeps the 13 values of
// p_new on its own column (z-6 .. z+6) in registers; the centre plane of the tile and its
// 6-point halo (computed from r and p_old, never read back from p_new) go to one of two shared
// frames, so one barrier per plane suffices.  Loads are issued ahead of use: the halo of plane
// z+1 and the column front two planes ahead are in flight while plane z is computed.  Values
// outside the box are zero.
// Variants of the FP32 stencil kernel the autotuner (rpa_autotune) chooses from, by
// rpa_options.stencil_shape: 0 = one column per thread, up to 640 threads per block; 1 = one
// column per thread, up to 320 threads and two blocks per SM (one block computes while the
// other waits at its per-plane barrier; same 96 registers); 2 = two columns per thread, up to 384
// threads.  The FP64 form has one shape.
struct PaShape {
    int max_threads, blocks_per_sm, pairs;   // blocks_per_sm: the kernel's launch-bounds minimum
};
constexpr PaShape kPaShapes32[3] = {{640, 1, 0}, {320, 2, 0}, {384, 1, 1}};
constexpr PaShape kPaShape64 = {448, 1, 0};
// MAXH: halo elements per thread that are prefetched into registers; any rest loads in place.
template <typename T, int MAXH, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
    k_cocg_pa(IterArgs A, Tiles tl, const typename Cx<T>::t *__restrict__ r, typename Cx<T>::t *__restrict__ pbuf,
              long long pstride, typename Cx<T>::t *__restrict__ q, const T *__restrict__ vloc, Coef<T> cf) {
    using C = typename Cx<T>::t;
    extern __shared__ unsigned char smraw[];
    constexpr int R = kRadius;
    const int W = tl.tx + 2 * R, H = tl.ty + 2 * R, frame = W * H;
    C *const fr0 = reinterpret_cast<C *>(smraw);
    C *const fr1 = fr0 + frame;
    // the block is rounded up to whole warps; threads past tx * ty only help with the halo
    const bool in_tile = threadIdx.x < tl.tx * tl.ty;
    const int lx = threadIdx.x % tl.tx, ly = in_tile ? threadIdx.x / tl.tx : 0;
    const int ntiles = tl.ntx * tl.nty * tl.nzc;
    const long long items = (long long)*A.cnt * ntiles;
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const int plane = nx * ny;                    // grid functions have < 2^31 points
    // with one tile across x the left/right strips lie outside the box: zero, never loaded (on a
    // periodic grid they hold the wrapped columns)
    const bool per = A.periodic != 0;
    const bool sides = tl.ntx > 1 || per;
    const int nhalo = sides ? 2 * R * (tl.tx + tl.ty) : 2 * R * tl.tx;
    const C zero = {(T)0, (T)0};
    // plane z of the column window: itself, its periodic image, or -1 (outside: zero)
    auto zplane = [&](int z) -> int { return (z >= 0 && z < nz) ? z : (per ? wrap_index(z, nz) : -1); };
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = A.list[(int)(it / ntiles)], tile = (int)(it % ntiles);
        const Slot &sl = A.slots[s];
        const int k = sl.iters;
        const T br = (T)sl.beta_re, bi = (T)sl.beta_im;
        const T sre = (T)sl.shift_re, sim = (T)sl.shift_im;
        const long long off = (long long)s * A.nd;
        const C *__restrict__ rs = r + off;
        const C *__restrict__ po = pbuf + (long long)(k & 1) * pstride + off;
        C *__restrict__ pn = pbuf + (long long)((k + 1) & 1) * pstride + off;
        C *__restrict__ qs = q + off;
        const int xyt = tile / tl.nzc, zc = tile % tl.nzc;
        const int x0 = (xyt % tl.ntx) * tl.tx, y0 = (xyt / tl.ntx) * tl.ty;
        const int zb = zc * tl.zlen, ze = min(nz, zb + tl.zlen);   // planes computed by this item
        const int gx = x0 + lx, gy = y0 + ly;
        const bool own = in_tile && gx < nx && gy < ny;
        const int col = gy * nx + gx;
        auto pnew = [&](const C a, const C b) -> C {
            C o;
            o.x = a.x + br * b.x - bi * b.y;
            o.y = a.y + br * b.y + bi * b.x;
            return o;
        };
        // halo element e -> frame offset and in-plane grid offset (-1: outside the box)
        auto halo_of = [&](int e, int &foff, int &goff) {
            int hx, hy;
            if (e < 2 * R * tl.tx) {                  // top / bottom strips
                const int rr = e / tl.tx;
                hx = e - rr * tl.tx + R;
                hy = rr < R ? rr : tl.ty + rr;
            } else {                                  // left / right strips
                const int e2 = e - 2 * R * tl.tx;
                const int cc = e2 / tl.ty;
                hy = e2 - cc * tl.ty + R;
                hx = cc < R ? cc : tl.tx + cc;
            }
            int ax = x0 + hx - R, ay = y0 + hy - R;
            if (per) {
                ax = wrap_index(ax, nx);
                ay = wrap_index(ay, ny);
            }
            foff = hy * W + hx;
            goff = (ax >= 0 && ax < nx && ay >= 0 && ay < ny) ? ay * nx + ax : -1;
        };
        __syncthreads();                              // the previous item's readers are done
        if (!sides) {                                 // zero the side strips of both frames
            for (int e = threadIdx.x; e < 2 * R * tl.ty; e += blockDim.x) {
                const int cc = e / tl.ty, hy = e - cc * tl.ty + R;
                const int hx = cc < R ? cc : tl.tx + cc;
                fr0[hy * W + hx] = zero;
                fr1[hy * W + hx] = zero;
            }
        }
        int hf[MAXH], hg[MAXH];
        C hr[MAXH], hp[MAXH];
#pragma unroll
        for (int h = 0; h < MAXH; ++h) {
            const int e = threadIdx.x + h * blockDim.x;
            hf[h] = -1;
            hg[h] = -1;
            if (e < nhalo) halo_of(e, hf[h], hg[h]);
            hr[h] = zero;
            hp[h] = zero;
            if (hg[h] >= 0) {                         // plane zb
                hr[h] = rs[zb * plane + hg[h]];
                hp[h] = po[zb * plane + hg[h]];
            }
        }
        // column window z = zb-6 .. zb+6 and the front plane zb+7 (raw r, p_old)
        C qv[2 * R + 1];
#pragma unroll
        for (int m = 0; m < 2 * R + 1; ++m) {
            const int z = zplane(zb + m - R);
            qv[m] = (own && z >= 0) ? pnew(rs[col + z * plane], po[col + z * plane]) : zero;
        }
        C f1r = zero, f1p = zero;          // raw front of plane z+R+1, consumed at the end of step z
        if (own && zplane(zb + R + 1) >= 0) {
            f1r = rs[col + zplane(zb + R + 1) * plane];
            f1p = po[col + zplane(zb + R + 1) * plane];
        }
        T vnext = own ? vloc[col + zb * plane] : (T)0;  // potential of the next plane
        T acc0 = 0, acc1 = 0;              // per-thread sums in the working precision (FP64 is slow)
        // The z loop is unrolled by the window length: slot (u + m) % 13 of qv holds plane z-6+m,
        // so the window turns without moving registers.
        for (int z0 = zb; z0 < ze; z0 += 2 * R + 1) {
#pragma unroll
            for (int u = 0; u < 2 * R + 1; ++u) {
                const int z = z0 + u;
                if (z >= ze) break;
                C *const fb = (z & 1) ? fr1 : fr0;
                if (in_tile) fb[(ly + R) * W + lx + R] = qv[(u + R) % (2 * R + 1)];
#pragma unroll
                for (int h = 0; h < MAXH; ++h)
                    if (hf[h] >= 0) fb[hf[h]] = hg[h] >= 0 ? pnew(hr[h], hp[h]) : zero;
                for (int e = threadIdx.x + MAXH * blockDim.x; e < nhalo; e += blockDim.x) {   // rare: small blocks
                    int foff, goff;
                    halo_of(e, foff, goff);
                    fb[foff] = goff >= 0 ? pnew(rs[z * plane + goff], po[z * plane + goff]) : zero;
                }
                // loads for later planes: halo of z+1, column front z+R+2
                if (z + 1 < ze) {
#pragma unroll
                    for (int h = 0; h < MAXH; ++h)
                        if (hg[h] >= 0) {
                            hr[h] = rs[(z + 1) * plane + hg[h]];
                            hp[h] = po[(z + 1) * plane + hg[h]];
                        }
                }
                C f2r = zero, f2p = zero;
                if (own && zplane(z + R + 2) >= 0) {
                    f2r = rs[col + zplane(z + R + 2) * plane];
                    f2p = po[col + zplane(z + R + 2) * plane];
                }
                const T vz = vnext;                          // potential of plane z (loaded one plane ago)
                if (own && z + 1 < ze) vnext = vloc[col + (z + 1) * plane];
                __syncthreads();
                if (own) {
                    const int idx = col + z * plane;
                    const C c = qv[(u + R) % (2 * R + 1)];
                    const T dre = (T)3 * cf.a[0] + vz + sre;
                    T re = dre * c.x - sim * c.y;
                    T im = dre * c.y + sim * c.x;
                    const C *cs = fb + (ly + R) * W + lx + R;
#pragma unroll
                    for (int d = 1; d <= R; ++d) {
                        const C a1 = cs[-d], a2 = cs[d], a3 = cs[-d * W], a4 = cs[d * W];
                        const C a5 = qv[(u + R - d) % (2 * R + 1)], a6 = qv[(u + R + d) % (2 * R + 1)];
                        re += cf.a[d] * (((a1.x + a2.x) + (a3.x + a4.x)) + (a5.x + a6.x));
                        im += cf.a[d] * (((a1.y + a2.y) + (a3.y + a4.y)) + (a5.y + a6.y));
                    }
                    C y;
                    y.x = re;
                    y.y = im;
                    qs[idx] = y;
                    pn[idx] = c;
                    acc0 += c.x * y.x - c.y * y.y;
                    acc1 += c.x * y.y + c.y * y.x;

                }
                // the front loaded one plane ago takes the slot of plane z-6
                qv[u] = (own && zplane(z + R + 1) >= 0) ? pnew(f1r, f1p) : zero;
                f1r = f2r;
                f1p = f2p;
            }
        }
        double acc[2] = {(double)acc0, (double)acc1};
        block_sum_any<2>(acc);
        if (threadIdx.x == 0) {
            double *o = A.part + ((long long)s * A.nper + tile) * 2;
            o[0] = acc[0];
            o[1] = acc[1];
            if (A.prof) {
                const long long w = (long long)min(tl.tx, nx - x0) * min(tl.ty, ny - y0) * (ze - zb);
                atomicAdd(A.prof + 1, (unsigned long long)w);
            }
        }
    }
}

// The FP32 stencil kernel with two grid columns per thread (x and x+1).  Same algorithm as
// k_cocg_pa; the pair shares its x-neighbours, so the shared-memory frame is read with 16-byte
// loads: 7 for the 14 x-neighbours of the pair and 12 for the y-neighbours of both points (19
// per two points instead of 48 8-byte loads), and the per-plane overhead (halo, barrier, index
// arithmetic, window turn) is paid once per two points.  Tiles are an even number of columns
// wide; a column past nx (odd nx) is held at zero.
template <int MAXH, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
    k_cocg_pa2(IterArgs A, Tiles tl, const float2 *__restrict__ r, float2 *__restrict__ pbuf, long long pstride,
               float2 *__restrict__ q, const float *__restrict__ vloc, Coef<float> cf) {
    extern __shared__ float4 smv[];
    constexpr int R = kRadius;
    constexpr int NW = 2 * R + 1;
    const int W = tl.tx + 2 * R, H = tl.ty + 2 * R, frame = W * H;   // in float2 units (W even)
    float2 *const fr0 = reinterpret_cast<float2 *>(smv);
    float2 *const fr1 = fr0 + frame;
    const int txp = tl.tx / 2;                            // column pairs per tile row
    const bool in_tile = threadIdx.x < txp * tl.ty;
    const int lp = threadIdx.x % txp, ly = in_tile ? threadIdx.x / txp : 0;
    const int ntiles = tl.ntx * tl.nty * tl.nzc;
    const long long items = (long long)*A.cnt * ntiles;
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const int plane = nx * ny;
    const bool sides = tl.ntx > 1;
    const int nhalo = sides ? R * (tl.tx + tl.ty) : R * tl.tx;      // halo pairs per plane
    const float2 zero = make_float2(0.f, 0.f);
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = A.list[(int)(it / ntiles)], tile = (int)(it % ntiles);
        const Slot &sl = A.slots[s];
        const int k = sl.iters;
        const float br = (float)sl.beta_re, bi = (float)sl.beta_im;
        const float sre = (float)sl.shift_re, sim = (float)sl.shift_im;
        const long long off = (long long)s * A.nd;
        const float2 *__restrict__ rs = r + off;
        const float2 *__restrict__ po = pbuf + (long long)(k & 1) * pstride + off;
        float2 *__restrict__ pn = pbuf + (long long)((k + 1) & 1) * pstride + off;
        float2 *__restrict__ qs = q + off;
        const int xyt = tile / tl.nzc, zc = tile % tl.nzc;
        const int x0 = (xyt % tl.ntx) * tl.tx, y0 = (xyt / tl.ntx) * tl.ty;
        const int zb = zc * tl.zlen, ze = min(nz, zb + tl.zlen);
        const int gx = x0 + 2 * lp, gy = y0 + ly;
        const bool own0 = in_tile && gx < nx && gy < ny;
        const bool own1 = in_tile && gx + 1 < nx && gy < ny;
        const int col = gy * nx + gx;
        auto pnew = [&](const float2 a, const float2 b) -> float2 {
            return make_float2(a.x + br * b.x - bi * b.y, a.y + br * b.y + bi * b.x);
        };
        // halo pair e -> frame offset of its first point, grid offsets of its two points
        auto halo_of = [&](int e, int &foff, int &g0, int &g1) {
            int hx, hy;
            if (e < R * tl.tx) {                          // top / bottom strips: tx/2 pairs per row
                const int rr = e / txp;
                hx = 2 * (e - rr * txp) + R;
                hy = rr < R ? rr : tl.ty + rr;
            } else {                                      // left / right strips: R/2 pairs per row
                const int e2 = e - R * tl.tx;
                const int cc = e2 / tl.ty;                // 0 .. R-1 (pair column)
                hy = e2 - cc * tl.ty + R;
                hx = cc < R / 2 ? 2 * cc : tl.tx + R + 2 * (cc - R / 2);
            }
            const int ax = x0 + hx - R, ay = y0 + hy - R;
            foff = hy * W + hx;
            const bool iy = ay >= 0 && ay < ny;
            g0 = (iy && ax >= 0 && ax < nx) ? ay * nx + ax : -1;
            g1 = (iy && ax + 1 >= 0 && ax + 1 < nx) ? ay * nx + ax + 1 : -1;
        };
        __syncthreads();                                  // the previous item's readers are done
        if (!sides) {                                     // zero the side strips of both frames
            for (int e = threadIdx.x; e < 2 * R * tl.ty; e += blockDim.x) {
                const int cc = e / tl.ty, hy = e - cc * tl.ty + R;
                const int hx = cc < R ? cc : tl.tx + cc;
                fr0[hy * W + hx] = zero;
                fr1[hy * W + hx] = zero;
            }
        }
        int hf[MAXH], hg0[MAXH], hg1[MAXH];
        float2 hr0[MAXH], hp0[MAXH], hr1[MAXH], hp1[MAXH];
#pragma unroll
        for (int h = 0; h < MAXH; ++h) {
            const int e = threadIdx.x + h * blockDim.x;
            hf[h] = -1;
            hg0[h] = -1;
            hg1[h] = -1;
            if (e < nhalo) halo_of(e, hf[h], hg0[h], hg1[h]);
            hr0[h] = hp0[h] = hr1[h] = hp1[h] = zero;
            if (hg0[h] >= 0) {
                hr0[h] = rs[zb * plane + hg0[h]];
                hp0[h] = po[zb * plane + hg0[h]];
            }
            if (hg1[h] >= 0) {
                hr1[h] = rs[zb * plane + hg1[h]];
                hp1[h] = po[zb * plane + hg1[h]];
            }
        }
        float2 qa[NW], qb[NW];                            // column windows z-6 .. z+6 (p_new)
#pragma unroll
        for (int m = 0; m < NW; ++m) {
            const int z = zb + m - R;
            const bool iz = z >= 0 && z < nz;
            qa[m] = (own0 && iz) ? pnew(rs[col + z * plane], po[col + z * plane]) : zero;
            qb[m] = (own1 && iz) ? pnew(rs[col + 1 + z * plane], po[col + 1 + z * plane]) : zero;
        }
        float2 f1ra = zero, f1pa = zero, f1rb = zero, f1pb = zero;   // raw fronts of plane z+R+1
        if (zb + R + 1 < nz) {
            if (own0) {
                f1ra = rs[col + (zb + R + 1) * plane];
                f1pa = po[col + (zb + R + 1) * plane];
            }
            if (own1) {
                f1rb = rs[col + 1 + (zb + R + 1) * plane];
                f1pb = po[col + 1 + (zb + R + 1) * plane];
            }
        }
        float va = own0 ? vloc[col + zb * plane] : 0.f, vb = own1 ? vloc[col + 1 + zb * plane] : 0.f;
        float acc0 = 0.f, acc1 = 0.f;
        for (int z0 = zb; z0 < ze; z0 += NW) {
#pragma unroll
            for (int u = 0; u < NW; ++u) {
                const int z = z0 + u;
                if (z >= ze) break;
                float2 *const fb = (z & 1) ? fr1 : fr0;
                const int ci = (ly + R) * W + 2 * lp + R;     // even: 16-byte aligned pair
                const float2 ca = qa[(u + R) % NW], cb = qb[(u + R) % NW];
                if (in_tile) reinterpret_cast<float4 *>(fb)[ci >> 1] = make_float4(ca.x, ca.y, cb.x, cb.y);
#pragma unroll
                for (int h = 0; h < MAXH; ++h)
                    if (hf[h] >= 0) {
                        const float2 e0 = hg0[h] >= 0 ? pnew(hr0[h], hp0[h]) : zero;
                        const float2 e1 = hg1[h] >= 0 ? pnew(hr1[h], hp1[h]) : zero;
                        reinterpret_cast<float4 *>(fb)[hf[h] >> 1] = make_float4(e0.x, e0.y, e1.x, e1.y);
                    }
                for (int e = threadIdx.x + MAXH * blockDim.x; e < nhalo; e += blockDim.x) {   // small blocks
                    int foff, g0, g1;
                    halo_of(e, foff, g0, g1);
                    const float2 e0 = g0 >= 0 ? pnew(rs[z * plane + g0], po[z * plane + g0]) : zero;
                    const float2 e1 = g1 >= 0 ? pnew(rs[z * plane + g1], po[z * plane + g1]) : zero;
                    reinterpret_cast<float4 *>(fb)[foff >> 1] = make_float4(e0.x, e0.y, e1.x, e1.y);
                }
                if (z + 1 < ze) {                         // halo of the next plane
#pragma unroll
                    for (int h = 0; h < MAXH; ++h) {
                        if (hg0[h] >= 0) {
                            hr0[h] = rs[(z + 1) * plane + hg0[h]];
                            hp0[h] = po[(z + 1) * plane + hg0[h]];
                        }
                        if (hg1[h] >= 0) {
                            hr1[h] = rs[(z + 1) * plane + hg1[h]];
                            hp1[h] = po[(z + 1) * plane + hg1[h]];
                        }
                    }
                }
                float2 f2ra = zero, f2pa = zero, f2rb = zero, f2pb = zero;   // column fronts z+R+2
                if (z + R + 2 < nz) {
                    if (own0) {
                        f2ra = rs[col + (z + R + 2) * plane];
                        f2pa = po[col + (z + R + 2) * plane];
                    }
                    if (own1) {
                        f2rb = rs[col + 1 + (z + R + 2) * plane];
                        f2pb = po[col + 1 + (z + R + 2) * plane];
                    }
                }
                const float vza = va, vzb = vb;
                if (z + 1 < ze) {
                    if (own0) va = vloc[col + (z + 1) * plane];
                    if (own1) vb = vloc[col + 1 + (z + 1) * plane];
                }
                __syncthreads();
                if (own0) {
                    const float4 *cv = reinterpret_cast<const float4 *>(fb) + (ci >> 1);
                    float4 X[7];                          // frame positions ci-6 .. ci+7
#pragma unroll
                    for (int m = 0; m < 7; ++m) X[m] = cv[m - 3];
                    // position ci + o of the x row, o in [-6, 7]
                    auto xat = [&](int o) -> float2 {
                        const float4 v = X[(o + 6) >> 1];
                        return ((o + 6) & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
                    };
                    const float dra = 3.f * cf.a[0] + vza + sre, drb = 3.f * cf.a[0] + vzb + sre;
                    float rea = dra * ca.x - sim * ca.y, ima = dra * ca.y + sim * ca.x;
                    float reb = drb * cb.x - sim * cb.y, imb = drb * cb.y + sim * cb.x;
#pragma unroll
                    for (int d = 1; d <= R; ++d) {
                        const float4 ym = cv[-(d * W) / 2], yp = cv[(d * W) / 2];
                        const float2 a1 = xat(-d), a2 = xat(d), b1 = xat(1 - d), b2 = xat(1 + d);
                        const float2 za = qa[(u + R - d) % NW], zp = qa[(u + R + d) % NW];
                        const float2 zbm = qb[(u + R - d) % NW], zbp = qb[(u + R + d) % NW];
                        rea += cf.a[d] * (((a1.x + a2.x) + (ym.x + yp.x)) + (za.x + zp.x));
                        ima += cf.a[d] * (((a1.y + a2.y) + (ym.y + yp.y)) + (za.y + zp.y));
                        reb += cf.a[d] * (((b1.x + b2.x) + (ym.z + yp.z)) + (zbm.x + zbp.x));
                        imb += cf.a[d] * (((b1.y + b2.y) + (ym.w + yp.w)) + (zbm.y + zbp.y));
                    }
                    const int idx = col + z * plane;
                    qs[idx] = make_float2(rea, ima);
                    pn[idx] = ca;
                    acc0 += ca.x * rea - ca.y * ima;
                    acc1 += ca.x * ima + ca.y * rea;
                    if (own1) {
                        qs[idx + 1] = make_float2(reb, imb);
                        pn[idx + 1] = cb;
                        acc0 += cb.x * reb - cb.y * imb;
                        acc1 += cb.x * imb + cb.y * reb;
                    }
                }
                // the fronts loaded one plane ago take the window slot of plane z-6
                const bool inz = z + R + 1 < nz;
                qa[u] = (own0 && inz) ? pnew(f1ra, f1pa) : zero;
                qb[u] = (own1 && inz) ? pnew(f1rb, f1pb) : zero;
                f1ra = f2ra;
                f1pa = f2pa;
                f1rb = f2rb;
                f1pb = f2pb;
            }
        }
        double acc[2] = {(double)acc0, (double)acc1};
        block_sum_any<2>(acc);
        if (threadIdx.x == 0) {
            double *o = A.part + ((long long)s * A.nper + tile) * 2;
            o[0] = acc[0];
            o[1] = acc[1];
            if (A.prof) {
                const long long w = (long long)min(tl.tx, nx - x0) * min(tl.ty, ny - y0) * (ze - zb);
                atomicAdd(A.prof + 1, (unsigned long long)w);
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Fused single-pass COCG iteration (mixed form; whole xy planes held in a shared-memory ring).
// ---------------------------------------------------------------------------------------------
// The recurrences of COCG rearranged so that one sweep over the state finishes iteration k-1
// and starts iteration k.  With alpha = alpha_{k-1} and beta = beta_k known at the start
// (both absent at k = 0), at every grid point:
//   x_k = x_{k-1} + alpha p_{k-1},  r_k = r_{k-1} - alpha q_{k-1},  p_k = r_k + beta p_{k-1},
//   q_k = (H - eps_n + i omega) p_k,
// with the sums rho_k = r_k^T r_k, ||r_k||^2, pi_k = p_k^T q_k, tau_k = r_k^T q_k and
// theta_k = q_k^T q_k (unconjugated products except the norm).  The block that owns the
// system then takes the scalar step itself: stop on ||r_k||, else alpha_k = rho_k / pi_k and
//   rho_{k+1} = (r_k - alpha_k q_k)^T (r_k - alpha_k q_k) = rho_k - 2 alpha_k tau_k + alpha_k^2 theta_k,
//   beta_{k+1} = rho_{k+1} / rho_k.
// x, r, p and q are each read and written once per iteration (64 bytes per grid point in
// complex FP32) instead of the 84 of the two-kernel form, and one launch replaces four.  The
// true rho_k of every sweep still sets alpha_k; only beta uses the expanded rho.
//
// One block owns one system and marches along z.  At step f it forms x, r, p of plane f
// ("front", loaded one plane ahead into registers), writes them back, and stores p_k of the
// plane into a ring of kRingPlanes planes in shared memory; after one barrier it applies the
// 12th-order stencil to plane f-6, whose 6 planes on either side are in the ring.  A thread owns
// 2 x 2 points (x, x+1; y, y+1), so a ring access is one 16-byte load for both x points, and rows
// y and y+1 share their y neighbours.  Ring layout (complex elements): a 16-byte zero
// word at the start of every plane, then its rows of 2 hw elements, each followed by a few unused
// elements so that two rows span hw 16-byte words modulo 8 (for even hw): the 16-byte words of
// consecutive units then fall in consecutive bank groups across row pairs, and a quarter warp's
// 16-byte loads are free of bank conflicts.  Neighbours past the box in x or y are read from the
// zero word (x: per-unit masks; y: predicated addresses); ring planes outside [0, nz) hold zeros.
// With 14 ring planes the plane written at step f+1 is the one read last at step f-1, so one
// barrier per step suffices.  Each block handles whole systems, so the state is single-buffered:
// a thread reads q at plane f six steps before it writes q there, and reads back r_k of plane f-6
// that it wrote itself.
//
// Periodic grids (PER; nx even, so that the point pairs wrap onto point pairs): x and y neighbours
// are read at their periodic images in the ring; at the start of a sweep the ring slots of planes
// -6 .. -1 receive p_k of planes nz-6 .. nz-1, formed from their old values as the front would form
// them (not written back: the front forms them again at their own steps), and at steps f >= nz the
// ring receives p_k of plane f - nz, read back from the direction this thread wrote at step f - nz.
//
// Because a block holds every sum of its system, it takes the scalar step itself and goes on
// with the next sweep: one launch runs each system of the active list through its whole inner
// solve.  Blocks take systems from a shared counter as they finish the previous one, so solves of
// different lengths balance over the SMs and no launch waits on a partly filled last wave; the
// list is taken from its end (it is in slot order, i.e. by orbital, and the highest orbitals,
// nearest the unoccupied spectrum, need the most iterations: the longest solves start first).
constexpr int kRingPlanes = 14;
constexpr int kRingMaxThreads = 512;
constexpr int kRingWsMaxThreads = 672;     // consumers + producers (planes of up to 416 units)

struct RingArgs {
    Slot *slots;
    const int *list_in;            // slots whose inner solve runs
    const int *cnt_in;
    int *grab;                     // systems taken so far (zero at the launch)
    unsigned long long *prof;      // [1] grid points processed, [2] those of first sweeps (nullptr = off)
    long long nd;
    double tol, inner_tol;
    int maxit;
    int nx, ny, nz;
    int hw;                        // point pairs per row: ceil(nx / 2)
    int hh;                        // row pairs: ceil(ny / 2)
    int rs;                        // ring row stride (complex elements): 2 hw + ring_row_pad(hw)
    int ps;                        // ring plane stride: 2 + ny rs (the zero word, then the rows);
                                   // cluster form: 2 + 2 bp rs (the block's band)
    int bp;                        // cluster form: row pairs per band (the last band may hold fewer)
};

// Unused elements after each ring row: even, and for even hw the smallest that makes two rows span
// hw 16-byte words modulo 8.
inline int ring_row_pad(int hw) {
    const int p = (8 - hw % 8) % 8;
    return p + (p & 1);
}
// Shared-memory bytes of the ring for an nx x ny plane.
inline size_t ring_bytes(int nx, int ny) {
    const int hw = (nx + 1) / 2;
    return (size_t)kRingPlanes * (2 + (size_t)ny * (2 * hw + ring_row_pad(hw))) * sizeof(float2);
}

__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }
// a + s b for a complex scalar s = (sr, si) given as S1 = (sr, sr), S2 = (-si, si)
__device__ __forceinline__ float2 cax(float2 a, float2 S1, float2 S2, float2 b) {
    return __ffma2_rn(S2, swp(b), __ffma2_rn(S1, b, a));
}
// unconjugated product u^T v accumulated into (re, im)
__device__ __forceinline__ void cdot(float &re, float &im, float2 u, float2 v) {
    re = fmaf(u.x, v.x, fmaf(-u.y, v.y, re));
    im = fmaf(u.x, v.y, fmaf(u.y, v.x, im));
}

template <bool EVEN>
__device__ __forceinline__ void ld_pair(const float2 *base, int idx, bool hasb, float2 &a, float2 &b) {
    if (EVEN) {
        const float4 v = *reinterpret_cast<const float4 *>(base + idx);
        a = make_float2(v.x, v.y);
        b = make_float2(v.z, v.w);
    } else {
        a = base[idx];
        b = hasb ? base[idx + 1] : make_float2(0.f, 0.f);
    }
}
template <bool EVEN>
__device__ __forceinline__ void st_pair(float2 *base, int idx, bool hasb, float2 a, float2 b) {
    if (EVEN) {
        *reinterpret_cast<float4 *>(base + idx) = make_float4(a.x, a.y, b.x, b.y);
    } else {
        base[idx] = a;
        if (hasb) base[idx + 1] = b;
    }
}

// Scalar step of the fused iteration for one slot (thread 0 of its block).  v: rho (re, im),
// ||r||^2, pi (re, im), tau (re, im), theta (re, im).  Same stopping rules as k_beta/k_alpha.
// Returns whether the inner solve goes on.
__device__ bool ring_scalar_step(const RingArgs &A, Slot &sl, const double (&v)[9]) {
    const int k = sl.iters;
    const double rn = sqrt(v[2]);
    const double thr = fmax(A.inner_tol * sl.ref_norm, 0.3 * A.tol * sl.bnorm * sl.scale);
    const bool conv = rn <= thr;
    const double rr2 = v[0] * v[0] + v[1] * v[1];
    const bool nonfinite = !isfinite(rn) || !isfinite(rr2);
    const bool zero = !(rr2 > 0.0);
    const bool nearb = k > 0 && !(rr2 > kNearBreak * kNearBreak * v[2] * v[2]);
    sl.rnorm = rn;
    sl.iters = k + 1;
    sl.total_iters += 1;
    if (conv || k >= A.maxit || nonfinite || zero || nearb) {
        // x_k is consistent with r_k: the inner solve ends here and the refinement takes over
        if (nonfinite) sl.discard = 1;
        if (!conv && (nonfinite || (zero && k == 0))) sl.status = RPA_ERR_BREAKDOWN;
        if (!conv && !nonfinite && nearb) sl.nearbreak += 1;
        sl.phase = kInnerDone;
        return false;
    }
    const double den = v[3] * v[3] + v[4] * v[4];
    if (!(den > 0.0) || !isfinite(den)) {
        sl.status = RPA_ERR_BREAKDOWN;
        if (!isfinite(den)) sl.discard = 1;
        sl.phase = kInnerDone;
        return false;
    }
    const double ar = (v[0] * v[3] + v[1] * v[4]) / den;   // alpha_k = rho / pi
    const double ai = (v[1] * v[3] - v[0] * v[4]) / den;
    const double atr = ar * v[5] - ai * v[6], ati = ar * v[6] + ai * v[5];        // alpha tau
    const double a2r = ar * ar - ai * ai, a2i = 2.0 * ar * ai;                    // alpha^2
    const double a2tr = a2r * v[7] - a2i * v[8], a2ti = a2r * v[8] + a2i * v[7];  // alpha^2 theta
    const double nr_ = v[0] - 2.0 * atr + a2tr, ni_ = v[1] - 2.0 * ati + a2ti;    // rho_{k+1}
    sl.alpha_re = ar;
    sl.alpha_im = ai;
    sl.beta_re = (nr_ * v[0] + ni_ * v[1]) / rr2;
    sl.beta_im = (ni_ * v[0] - nr_ * v[1]) / rr2;
    return true;
}

// Two x-adjacent points (x, x+1) of row y from a ring plane: one 16-byte shared load.
__device__ __forceinline__ void ring_pair(const unsigned char *addr, float2 &a, float2 &b) {
    const float4 t = *reinterpret_cast<const float4 *>(addr);
    a = make_float2(t.x, t.y);
    b = make_float2(t.z, t.w);
}

// A unit of the fused kernels: the 2 x 2 points (x, x+1; y, y+1) of a plane, x and y even.
struct RingUnit {
    bool own, hasb, row1;          // a unit of the plane; point x+1 and row y+1 inside the box
    int gy, col0, col1;            // row; in-plane indices of (x, y) and (x, y+1)
    int rb0, rb1, rb1z;            // ring byte offsets of rows y and y+1 (rb1z: 0 if row y+1 is outside)
    int xm;                        // bit m: x load m (point pair x/2 - 3 + m) lies inside the row
    int bx;                        // point pair of the unit in its row: x / 2
};

// Unit u of a ring that holds the npairs row pairs from row y0 on (a whole plane: y0 = 0, npairs = hh).
__device__ __forceinline__ RingUnit ring_unit(int u, const RingArgs &A, int y0 = 0, int npairs = -1) {
    RingUnit r;
    r.own = u >= 0 && u < A.hw * (npairs < 0 ? A.hh : npairs);
    const int by = r.own ? u / A.hw : 0;
    const int gx = r.own ? 2 * (u - by * A.hw) : 0;
    r.gy = y0 + 2 * by;
    r.hasb = r.own && gx + 1 < A.nx;
    r.row1 = r.own && r.gy + 1 < A.ny;
    r.col0 = r.gy * A.nx + gx;
    r.col1 = r.col0 + A.nx;
    r.rb0 = (2 + (r.gy - y0) * A.rs + gx) * 8;
    r.rb1 = r.rb0 + A.rs * 8;
    r.rb1z = r.row1 ? r.rb1 : 0;
    const int xlo = max(0, 3 - gx / 2), xhi = min(6, A.hw + 2 - gx / 2);
    r.xm = ((1 << (xhi + 1)) - 1) & ~((1 << xlo) - 1);
    r.bx = gx / 2;
    return r;
}

// Raw values of a unit at a front plane: x, r, p, q of its four points (points outside the box
// stay zero; x, p, q are not needed at the first pass).
struct RingFront {
    float2 x[4], r[4], p[4], q[4];
};

template <bool EVEN>
__device__ __forceinline__ void ring_load_front(const RingUnit &U, int g0, bool first, const float2 *xs,
                                                const float2 *rsv, const float2 *psv, const float2 *qs,
                                                RingFront &F) {
    const float2 zero = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 4; ++i) F.x[i] = F.r[i] = F.p[i] = F.q[i] = zero;
    const int g1 = g0 + (U.col1 - U.col0);
    ld_pair<EVEN>(rsv, g0, U.hasb, F.r[0], F.r[1]);
    if (U.row1) ld_pair<EVEN>(rsv, g1, U.hasb, F.r[2], F.r[3]);
    if (!first) {
        ld_pair<EVEN>(xs, g0, U.hasb, F.x[0], F.x[1]);
        ld_pair<EVEN>(psv, g0, U.hasb, F.p[0], F.p[1]);
        ld_pair<EVEN>(qs, g0, U.hasb, F.q[0], F.q[1]);
        if (U.row1) {
            ld_pair<EVEN>(xs, g1, U.hasb, F.x[2], F.x[3]);
            ld_pair<EVEN>(psv, g1, U.hasb, F.p[2], F.p[3]);
            ld_pair<EVEN>(qs, g1, U.hasb, F.q[2], F.q[3]);
        }
    }
}

// Front plane f of a unit: x_k, r_k, p_k from the raw values, written back, and p_k into the ring
// slot at `slot` (zeros for planes past the box); sums rho = r_k^T r_k and ||r_k||^2 (acc[0..2]).
template <bool EVEN>
__device__ __forceinline__ void ring_front(const RingUnit &U, int f, int nz, int plane, bool first, float alr,
                                           float ali, float ber, float bei, const RingFront &F, float2 *xs,
                                           float2 *rsv, float2 *psv, unsigned char *slot, float (&acc)[3]) {
    const float2 zero = make_float2(0.f, 0.f);
    float2 pk[4] = {zero, zero, zero, zero};
    if (f < nz) {
        const int g0 = f * plane + U.col0, g1 = f * plane + U.col1;
        float2 rr[4];
        if (first) {
#pragma unroll
            for (int i = 0; i < 4; ++i) rr[i] = pk[i] = F.r[i];
        } else {
            const float2 A1 = make_float2(alr, alr), A2 = make_float2(-ali, ali);
            const float2 N1 = make_float2(-alr, -alr), N2 = make_float2(ali, -ali);
            const float2 B1 = make_float2(ber, ber), B2 = make_float2(-bei, bei);
            float2 xx[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                xx[i] = cax(F.x[i], A1, A2, F.p[i]);
                rr[i] = cax(F.r[i], N1, N2, F.q[i]);
                pk[i] = cax(rr[i], B1, B2, F.p[i]);
            }
            st_pair<EVEN>(xs, g0, U.hasb, xx[0], xx[1]);
            st_pair<EVEN>(rsv, g0, U.hasb, rr[0], rr[1]);
            if (U.row1) {
                st_pair<EVEN>(xs, g1, U.hasb, xx[2], xx[3]);
                st_pair<EVEN>(rsv, g1, U.hasb, rr[2], rr[3]);
            }
        }
        if (!U.hasb) pk[1] = pk[3] = zero;
        if (!U.row1) pk[2] = pk[3] = zero;
        st_pair<EVEN>(psv, g0, U.hasb, pk[0], pk[1]);
        if (U.row1) st_pair<EVEN>(psv, g1, U.hasb, pk[2], pk[3]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool in = (i & 1 ? U.hasb : true) && (i & 2 ? U.row1 : true);
            if (in) {
                cdot(acc[0], acc[1], rr[i], rr[i]);
                acc[2] = fmaf(rr[i].x, rr[i].x, fmaf(rr[i].y, rr[i].y, acc[2]));
            }
        }
    }
    *reinterpret_cast<float4 *>(slot + U.rb0) = make_float4(pk[0].x, pk[0].y, pk[1].x, pk[1].y);
    if (U.row1) *reinterpret_cast<float4 *>(slot + U.rb1) = make_float4(pk[2].x, pk[2].y, pk[3].x, pk[3].y);
}

// Periodic grids: p_k of a unit at a plane from its raw values (as ring_front forms it), into a ring
// slot only: nothing is written back and nothing summed.
template <bool EVEN>
__device__ __forceinline__ void ring_halo_plane(const RingUnit &U, bool first, float alr, float ali, float ber,
                                                float bei, const RingFront &F, unsigned char *slot) {
    const float2 zero = make_float2(0.f, 0.f);
    float2 pk[4];
    const float2 N1 = make_float2(-alr, -alr), N2 = make_float2(ali, -ali);
    const float2 B1 = make_float2(ber, ber), B2 = make_float2(-bei, bei);
#pragma unroll
    for (int i = 0; i < 4; ++i) pk[i] = first ? F.r[i] : cax(cax(F.r[i], N1, N2, F.q[i]), B1, B2, F.p[i]);
    if (!U.hasb) pk[1] = pk[3] = zero;
    if (!U.row1) pk[2] = pk[3] = zero;
    *reinterpret_cast<float4 *>(slot + U.rb0) = make_float4(pk[0].x, pk[0].y, pk[1].x, pk[1].y);
    if (U.row1) *reinterpret_cast<float4 *>(slot + U.rb1) = make_float4(pk[2].x, pk[2].y, pk[3].x, pk[3].y);
}

// Periodic grids: p_k of a unit at plane z (< the step's plane, so formed and written by this
// thread earlier in the sweep) from global memory into a ring slot.
template <bool EVEN>
__device__ __forceinline__ void ring_wrap_front(const RingUnit &U, int g0, const float2 *psv, unsigned char *slot) {
    float2 a, b, c = make_float2(0.f, 0.f), d = c;
    ld_pair<EVEN>(psv, g0, U.hasb, a, b);
    if (U.row1) ld_pair<EVEN>(psv, g0 + (U.col1 - U.col0), U.hasb, c, d);
    *reinterpret_cast<float4 *>(slot + U.rb0) = make_float4(a.x, a.y, b.x, b.y);
    if (U.row1) *reinterpret_cast<float4 *>(slot + U.rb1) = make_float4(c.x, c.y, d.x, d.y);
}

// r_k and V of a unit at plane z (r_k written at the step that formed plane z).
template <bool EVEN>
__device__ __forceinline__ void ring_load_rv(const RingUnit &U, int g0, const float2 *rsv, const float *vloc,
                                             float2 (&rk)[4], float (&vv)[4]) {
    const int g1 = g0 + (U.col1 - U.col0);
    ld_pair<EVEN>(rsv, g0, U.hasb, rk[0], rk[1]);
    vv[0] = vloc[g0];
    vv[1] = U.hasb ? vloc[g0 + 1] : 0.f;
    if (U.row1) {
        ld_pair<EVEN>(rsv, g1, U.hasb, rk[2], rk[3]);
        vv[2] = vloc[g1];
        vv[3] = U.hasb ? vloc[g1 + 1] : 0.f;
    }
}

// Cluster form: the rows of a block's band, [y0, y1), and the block's copy of the plane's 6 rows
// above and 6 rows below its band (the halo, rows y0-6 .. y0-1 then y1 .. y1+5, laid out as ring rows
// after a zero word), taken from the neighbouring blocks' rings.
struct Band {
    int y0, y1;
    const unsigned char *halo;
};

// Two x-adjacent points from a ring slot of any block of the cluster: one 16-byte load.
__device__ __forceinline__ void ring_pair_cl(unsigned addr, float2 &a, float2 &b) {
    float4 t;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(t.x), "=f"(t.y), "=f"(t.z), "=f"(t.w)
                 : "r"(addr)
                 : "memory");
    a = make_float2(t.x, t.y);
    b = make_float2(t.z, t.w);
}

// q_k = (H + sigma) p_k on plane z for a unit, from the ring (cz: the ring slot of plane z), stored;
// sums pi = p_k^T q_k, tau = r_k^T q_k, theta = q_k^T q_k (acc[0..5]); rk, vv: r_k and V of the
// unit's points (V's term of the diagonal is added last).  A variant that loaded each row of y
// neighbours once for both rows (12 loads instead of 22) and one that loaded r_k and V inside this
// function both measured slower: the values they keep live spill registers.
template <bool EVEN, bool PER, bool BAND = false>
__device__ __forceinline__ void ring_stencil(const RingUnit &U, const unsigned char *ring, int psb, int rsb, int hw,
                                             int ny, int cz, int gq0, const float2 (&rk)[4], const float (&vv)[4],
                                             float shr, float shi, const Coef<float> &cf, float2 *qs,
                                             float (&acc)[6], const Band &B = Band{}) {
    const float2 zero = make_float2(0.f, 0.f);
    const unsigned char *const pz = ring + cz * psb;
    // row r of the plane (periodic: its image; cluster form: in this block's band or a neighbour's;
    // else the zero word outside the box)
    auto row = [&](int r) -> const unsigned char * {
        if (PER) return pz + U.rb0 + (wrap_index(r, ny) - U.gy) * rsb;
        return (r >= 0 && r < ny) ? pz + U.rb0 + (r - U.gy) * rsb : pz;
    };
    // cluster form: row r in this block's band, in its halo copy of the neighbouring bands' rows, or
    // the zero word outside the box
    auto yrow = [&](int r, float2 &a, float2 &b) {
        if (BAND) {
            const int xoff = U.rb0 - (U.gy - B.y0) * rsb;      // the unit's column within a row
            const unsigned char *ad = pz;
            if (r >= 0 && r < ny) {
                if (r < B.y0) ad = B.halo + xoff + (r - B.y0 + kRadius) * rsb;
                else if (r >= B.y1) ad = B.halo + xoff + (r - B.y1 + kRadius) * rsb;
                else ad = pz + xoff + (r - B.y0) * rsb;
            }
            ring_pair(ad, a, b);
        } else {
            ring_pair(row(r), a, b);
        }
    };
    const float2 c0 = make_float2(3.f * cf.a[0], 3.f * cf.a[0]);
    const float2 SH = make_float2(shr, shr), SI = make_float2(-shi, shi);
    // centre and x neighbours of one row: 7 16-byte loads (positions x-6 .. x+7; those past the row
    // read the plane's zero word)
    auto xrow = [&](const unsigned char *pr, float2 &ca, float2 &cb, float2 &qa, float2 &qb) {
        float4 X[7];
#pragma unroll
        for (int m = 0; m < 7; ++m)
            X[m] = *reinterpret_cast<const float4 *>(
                PER ? pr + 16 * (wrap_index(U.bx - 3 + m, hw) - U.bx) : ((U.xm >> m) & 1 ? pr - 48 + 16 * m : pz));
        auto xat = [&](int o) -> float2 {
            const float4 t = X[(o + 6) >> 1];
            return ((o + 6) & 1) ? make_float2(t.z, t.w) : make_float2(t.x, t.y);
        };
        ca = xat(0);
        cb = xat(1);
        qa = __ffma2_rn(SI, swp(ca), __fmul2_rn(__fadd2_rn(c0, SH), ca));
        qb = __ffma2_rn(SI, swp(cb), __fmul2_rn(__fadd2_rn(c0, SH), cb));
#pragma unroll
        for (int d = 1; d <= kRadius; ++d) {
            const float2 cd = make_float2(cf.a[d], cf.a[d]);
            qa = __ffma2_rn(cd, __fadd2_rn(xat(-d), xat(d)), qa);
            qb = __ffma2_rn(cd, __fadd2_rn(xat(1 - d), xat(1 + d)), qb);
        }
    };
    float2 c0_, c1_, c2_, c3_, q0, q1, q2, q3;
    xrow(pz + U.rb0, c0_, c1_, q0, q1);
    // row y+1 outside the box (odd ny): its values are zero neighbours of row y, and its own q is
    // discarded (the loads repeat row y, an address inside the plane)
    xrow(pz + (U.row1 ? U.rb1 : U.rb0), c2_, c3_, q2, q3);
    if (!U.row1) c2_ = c3_ = zero;
    const bool row1_centre = U.row1 || !PER;   // row y+1 is a centre, or outside the box (zero)
    // y neighbours: rows y-d and y+1+d, and for d > 1 rows y+d and y+1-d (rows outside the box read
    // the zero word); rows y and y+1 are the centres
#pragma unroll
    for (int d = 1; d <= kRadius; ++d) {
        float2 u0, u1, l0, l1;              // rows y-d and y+1+d
        if (PER || BAND) {
            yrow(U.gy - d, u0, u1);
            yrow(U.gy + 1 + d, l0, l1);
        } else {
            ring_pair(pz + (U.gy - d >= 0 ? U.rb0 - d * rsb : 0), u0, u1);
            ring_pair(pz + (U.gy + 1 + d < ny ? U.rb1 + d * rsb : 0), l0, l1);
        }
        float2 dn0, dn1, up0, up1;          // row y+d (for row y), row y+1-d (for row y+1)
        if (d == 1) {
            if (row1_centre) {
                dn0 = c2_;
                dn1 = c3_;
            } else {                        // periodic, row y+1 past the box: its image
                yrow(U.gy + 1, dn0, dn1);
            }
            up0 = c0_;
            up1 = c1_;
        } else if (PER || BAND) {
            yrow(U.gy + d, dn0, dn1);
            yrow(U.gy + 1 - d, up0, up1);
        } else {
            ring_pair(pz + (U.gy + d < ny ? U.rb0 + d * rsb : 0), dn0, dn1);
            ring_pair(pz + (U.gy + 1 - d >= 0 ? U.rb1 - d * rsb : 0), up0, up1);
        }
        const int sm = cz >= d ? cz - d : cz + kRingPlanes - d;
        const int sp = cz + d < kRingPlanes ? cz + d : cz + d - kRingPlanes;
        float2 zm0, zm1, zm2, zm3, zp0, zp1, zp2, zp3;
        ring_pair(ring + sm * psb + U.rb0, zm0, zm1);
        ring_pair(ring + sp * psb + U.rb0, zp0, zp1);
        ring_pair(ring + sm * psb + U.rb1z, zm2, zm3);   // row y+1 outside the box: the zero word
        ring_pair(ring + sp * psb + U.rb1z, zp2, zp3);
        const float2 cd = make_float2(cf.a[d], cf.a[d]);
        q0 = __ffma2_rn(cd, __fadd2_rn(__fadd2_rn(u0, dn0), __fadd2_rn(zm0, zp0)), q0);
        q1 = __ffma2_rn(cd, __fadd2_rn(__fadd2_rn(u1, dn1), __fadd2_rn(zm1, zp1)), q1);
        q2 = __ffma2_rn(cd, __fadd2_rn(__fadd2_rn(up0, l0), __fadd2_rn(zm2, zp2)), q2);
        q3 = __ffma2_rn(cd, __fadd2_rn(__fadd2_rn(up1, l1), __fadd2_rn(zm3, zp3)), q3);
    }
    q0 = __ffma2_rn(make_float2(vv[0], vv[0]), c0_, q0);
    q1 = __ffma2_rn(make_float2(vv[1], vv[1]), c1_, q1);
    q2 = __ffma2_rn(make_float2(vv[2], vv[2]), c2_, q2);
    q3 = __ffma2_rn(make_float2(vv[3], vv[3]), c3_, q3);
    st_pair<EVEN>(qs, gq0, U.hasb, q0, q1);
    if (U.row1) st_pair<EVEN>(qs, gq0 + (U.col1 - U.col0), U.hasb, q2, q3);
    cdot(acc[0], acc[1], c0_, q0);
    cdot(acc[2], acc[3], rk[0], q0);
    cdot(acc[4], acc[5], q0, q0);
    if (U.hasb) {
        cdot(acc[0], acc[1], c1_, q1);
        cdot(acc[2], acc[3], rk[1], q1);
        cdot(acc[4], acc[5], q1, q1);
    }
    if (U.row1) {
        cdot(acc[0], acc[1], c2_, q2);
        cdot(acc[2], acc[3], rk[2], q2);
        cdot(acc[4], acc[5], q2, q2);
        if (U.hasb) {
            cdot(acc[0], acc[1], c3_, q3);
            cdot(acc[2], acc[3], rk[3], q3);
            cdot(acc[4], acc[5], q3, q3);
        }
    }
}

// Next system of a fused-kernel block from the shared counter (index into the active list, taken
// from its end), or -1 when the list is exhausted.  All threads of the block call it.
__device__ __forceinline__ int ring_next_item(const RingArgs &A, int n_items) {
    __shared__ int item;
    if (threadIdx.x == 0) item = atomicAdd(A.grab, 1);
    __syncthreads();
    const int it = item;
    return it < n_items ? A.list_in[n_items - 1 - it] : -1;
}

// End of a sweep of a fused-kernel block: block sums, scalar step by thread 0; returns (in every
// thread) whether the system's inner solve goes on.
__device__ __forceinline__ bool ring_end_sweep(const RingArgs &A, Slot &sl, bool first, const float (&fa)[3],
                                               const float (&sa)[6]) {
    __shared__ int more;
    double v[9] = {fa[0], fa[1], fa[2], sa[0], sa[1], sa[2], sa[3], sa[4], sa[5]};
    block_sum_any<9>(v);
    if (threadIdx.x == 0) {
        more = ring_scalar_step(A, sl, v) ? 1 : 0;
        if (A.prof) {
            atomicAdd(A.prof + 1, (unsigned long long)A.nd);
            if (first) atomicAdd(A.prof + 2, (unsigned long long)A.nd);
        }
    }
    __syncthreads();
    return more != 0;
}

// The fused kernel: every thread takes one unit through both phases of a step (front, then the
// stencil six planes behind), the front's loads for the next plane in flight during the stencil.
template <bool EVEN, bool PER>
__global__ void __launch_bounds__(kRingMaxThreads, 1)
    k_cocg_ring(RingArgs A, float2 *__restrict__ xg, float2 *__restrict__ rg, float2 *__restrict__ pg,
                float2 *__restrict__ qg, const float *__restrict__ vloc, Coef<float> cf) {
    extern __shared__ float4 ring4[];
    unsigned char *const ring = reinterpret_cast<unsigned char *>(ring4);
    const int tid = threadIdx.x;
    const int nz = A.nz, plane = A.nx * A.ny;      // grid functions have < 2^31 points
    const int rsb = A.rs * 8, psb = A.ps * 8;      // ring row / plane strides in bytes
    const RingUnit U = ring_unit(tid, A);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = tid; e < kRingPlanes * A.ps / 2; e += blockDim.x) ring4[e] = zero4;   // padding stays zero
    const int n_items = *A.cnt_in;
    for (int s; (s = ring_next_item(A, n_items)) >= 0;) {
        Slot &sl = A.slots[s];
        const float shr = (float)sl.shift_re, shi = (float)sl.shift_im;
        const long long off = (long long)s * A.nd;
        float2 *const xs = xg + off;
        float2 *const rsv = rg + off;
        float2 *const psv = pg + off;
        float2 *const qs = qg + off;
        bool more = true;
        while (more) {                             // sweeps of this system (iterations of COCG)
            const bool first = sl.iters == 0;
            const float alr = (float)sl.alpha_re, ali = (float)sl.alpha_im;
            const float ber = (float)sl.beta_re, bei = (float)sl.beta_im;
            __syncthreads();                       // the previous sweep's ring readers are done
            if (U.own) {                           // planes -6 .. -1 (ring slots 8 .. 13)
                if (PER) {                         // p_k of their images nz-6 .. nz-1
                    for (int m = kRingPlanes - kRadius; m < kRingPlanes; ++m) {
                        RingFront H;
                        ring_load_front<EVEN>(U, wrap_index(m - kRingPlanes, nz) * plane + U.col0, first, xs, rsv,
                                              psv, qs, H);
                        ring_halo_plane<EVEN>(U, first, alr, ali, ber, bei, H, ring + m * psb);
                    }
                } else {                           // zero
#pragma unroll
                    for (int m = kRingPlanes - kRadius; m < kRingPlanes; ++m) {
                        *reinterpret_cast<float4 *>(ring + m * psb + U.rb0) = zero4;
                        if (U.row1) *reinterpret_cast<float4 *>(ring + m * psb + U.rb1) = zero4;
                    }
                }
            }
            RingFront F;
            if (U.own) ring_load_front<EVEN>(U, U.col0, first, xs, rsv, psv, qs, F);   // front plane 0
            float fa[3] = {0.f, 0.f, 0.f}, sa[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const int nsteps = nz + kRadius;
            // rolled loop: unrolled over the ring (compile-time slots) it needs far more registers
            for (int f = 0, u = 0; f < nsteps; ++f, u = (u + 1 == kRingPlanes) ? 0 : u + 1) {
                // r_k and V of the stencil's plane z = f - 6, in flight during the front and the barrier
                const int z = f - kRadius;
                float2 rk[4] = {};
                float vv[4] = {0.f, 0.f, 0.f, 0.f};
                if (U.own && z >= 0) ring_load_rv<EVEN>(U, z * plane + U.col0, rsv, vloc, rk, vv);
                // 1. front plane f, p_k into ring slot u (periodic, f >= nz: p_k of plane f - nz)
                if (U.own) {
                    if (PER && f >= nz)
                        ring_wrap_front<EVEN>(U, wrap_index(f, nz) * plane + U.col0, psv, ring + u * psb);
                    else
                        ring_front<EVEN>(U, f, nz, plane, first, alr, ali, ber, bei, F, xs, rsv, psv, ring + u * psb,
                                         fa);
                }
                // 2. the next front plane, in flight during the stencil below
                if (U.own && f + 1 < nz)
                    ring_load_front<EVEN>(U, (f + 1) * plane + U.col0, first, xs, rsv, psv, qs, F);
                __syncthreads();
                // 3. q_k on plane z, its 6 neighbour planes from the ring
                if (U.own && z >= 0) {
                    const int cz = u >= kRadius ? u - kRadius : u + kRingPlanes - kRadius;   // ring slot of z
                    ring_stencil<EVEN, PER>(U, ring, psb, rsb, A.hw, A.ny, cz, z * plane + U.col0, rk, vv, shr, shi, cf,
                                            qs, sa);
                }
            }
            more = ring_end_sweep(A, sl, first, fa, sa);
        }
    }
}

// Cluster form of the fused kernel, for planes whose ring does not fit one block's shared memory
// (72 x 72: 580 KB), and for smaller planes as two blocks per SM: the C blocks of a thread-block
// cluster split every plane into bands of bp row pairs (the last band may hold fewer; bp >= 3, so
// that the y neighbours of a band lie in the bands next to it) and each block keeps the ring of its
// band.  The stencil reads the y neighbours past its band from the neighbouring blocks' rings
// (distributed shared memory); x and z neighbours are in its own ring.  Only the centre plane's rows
// are read across blocks, and that plane was written six steps before, so the cluster barrier (a
// release / acquire fence across the cluster) is needed only every kClusterEvery steps and runs one
// step behind: a block arrives after writing its front plane at steps f = 0 mod kClusterEvery and
// waits for that phase at step f+1, a step of work after the others arrived; the block barrier of
// every step orders the block's own ring.  Remote rows of plane z, read at step z+6, were written at
// step z and released by the first arrival at or after it (at most kClusterEvery-1 steps later,
// waited on one step after that, so by step z+kClusterEvery <= z+5); the ring slot a block overwrites
// at step f was last read by any block at step f-8, before that block's next arrival (one falls in
// every window of kClusterEvery steps) and so before the writer's wait.  The neighbours' rows are
// not read in the stencil: at step f a block copies the 6 rows next to its band of plane f-5 from
// the neighbouring blocks' rings into a local halo (double-buffered by plane parity; the copy's
// distributed shared-memory loads overlap the stencil), and the stencil of step f+1 reads them
// there.  Units whose y neighbours all lie in their own band run the single-block stencil.  The
// scalar step is taken by rank 0 from the bands' sums, added in rank order; the next system, the
// stopping decision and the bands' sums pass through shared memory of the cluster.  Dirichlet
// grids.
namespace cg = cooperative_groups;

constexpr int kClusterEvery = 4;           // steps per cluster barrier phase (at most 5, see above)
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

template <bool EVEN>
__global__ void __launch_bounds__(kRingMaxThreads, 1)
    k_cocg_ring_cl(RingArgs A, float2 *__restrict__ xg, float2 *__restrict__ rg, float2 *__restrict__ pg,
                   float2 *__restrict__ qg, const float *__restrict__ vloc, Coef<float> cf) {
    extern __shared__ float4 ring4[];
    __shared__ int cl_item, cl_more;
    __shared__ double cl_part[9];
    unsigned char *const ring = reinterpret_cast<unsigned char *>(ring4);
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), ncl = (int)cl.num_blocks();
    const int tid = threadIdx.x;
    const int nz = A.nz, plane = A.nx * A.ny;
    const int rsb = A.rs * 8, psb = A.ps * 8;
    const int hsb = (2 + 2 * kRadius * A.rs) * 8;  // halo buffer: zero word and 12 rows
    unsigned char *const halo = ring + kRingPlanes * psb;
    const int rows = 2 * A.bp;                     // every band but the last
    Band B;
    B.y0 = rank * rows;
    B.y1 = min(A.ny, B.y0 + rows);
    const int npairs = max(0, (B.y1 - B.y0 + 1) / 2);
    const RingUnit U = ring_unit(tid, A, B.y0, npairs);
    // a unit whose y neighbours (rows y-6 .. y+7) reach into another block's band
    const bool remote = (U.gy - kRadius < B.y0 && B.y0 > 0) || (U.gy + 1 + kRadius >= B.y1 && B.y1 < A.ny);
    // the rings' shared::cluster addresses: this block's, and those of the neighbouring bands' blocks
    const unsigned ring_self = (unsigned)__cvta_generic_to_shared(ring);
    unsigned ring_up = 0, ring_dn = 0;
    if (rank > 0) asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ring_up) : "r"(ring_self), "r"(rank - 1));
    if (rank + 1 < ncl) asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ring_dn) : "r"(ring_self), "r"(rank + 1));
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = tid; e < (kRingPlanes * psb + 2 * hsb) / 16; e += blockDim.x) ring4[e] = zero4;   // padding stays zero
    const int nhalo = 2 * kRadius * A.hw;          // 16-byte words copied into the halo per plane
    const int n_items = *A.cnt_in;
    for (;;) {
        cl.sync();                                 // every block is done with the previous system
        if (rank == 0 && tid == 0) {
            const int it = atomicAdd(A.grab, 1);
            for (int t = 0; t < ncl; ++t) *cl.map_shared_rank(&cl_item, t) = it;
        }
        cl.sync();
        const int it = cl_item;
        if (it >= n_items) break;
        const int s = A.list_in[n_items - 1 - it];
        Slot &sl = A.slots[s];
        const float shr = (float)sl.shift_re, shi = (float)sl.shift_im;
        const long long off = (long long)s * A.nd;
        float2 *const xs = xg + off;
        float2 *const rsv = rg + off;
        float2 *const psv = pg + off;
        float2 *const qs = qg + off;
        bool more = true;
        while (more) {                             // sweeps of this system (iterations of COCG)
            const bool first = sl.iters == 0;
            const float alr = (float)sl.alpha_re, ali = (float)sl.alpha_im;
            const float ber = (float)sl.beta_re, bei = (float)sl.beta_im;
            if (U.own) {                           // planes -6 .. -1 (ring slots 8 .. 13) are zero
#pragma unroll
                for (int m = kRingPlanes - kRadius; m < kRingPlanes; ++m) {
                    *reinterpret_cast<float4 *>(ring + m * psb + U.rb0) = zero4;
                    if (U.row1) *reinterpret_cast<float4 *>(ring + m * psb + U.rb1) = zero4;
                }
            }
            RingFront F;
            if (U.own) ring_load_front<EVEN>(U, U.col0, first, xs, rsv, psv, qs, F);   // front plane 0
            float fa[3] = {0.f, 0.f, 0.f}, sa[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const int nsteps = nz + kRadius;
            for (int f = 0, u = 0; f < nsteps; ++f, u = (u + 1 == kRingPlanes) ? 0 : u + 1) {
                // r_k and V of the stencil's plane z = f - 6, in flight during the front and the barrier
                const int z = f - kRadius;
                float2 rk[4] = {};
                float vv[4] = {0.f, 0.f, 0.f, 0.f};
                if (U.own && z >= 0) ring_load_rv<EVEN>(U, z * plane + U.col0, rsv, vloc, rk, vv);
                if (f % kClusterEvery == 1) cluster_wait();   // the phase this block arrived at last step
                // 1. front plane f, p_k into ring slot u
                if (U.own)
                    ring_front<EVEN>(U, f, nz, plane, first, alr, ali, ber, bei, F, xs, rsv, psv, ring + u * psb, fa);
                if (f % kClusterEvery == 0) cluster_arrive();
                // 2. the next front plane, in flight during the stencil
                if (U.own && f + 1 < nz)
                    ring_load_front<EVEN>(U, (f + 1) * plane + U.col0, first, xs, rsv, psv, qs, F);
                __syncthreads();
                // 3. the halo of plane f-5 (used at the next step) from the neighbouring blocks' rings
                const int zc = f - kRadius + 1;
                if (zc >= 0 && zc < nz) {
                    const int cs = u >= kRadius - 1 ? u - (kRadius - 1) : u + kRingPlanes - (kRadius - 1);   // slot of zc
                    unsigned char *const hb = halo + (zc & 1) * hsb;
                    for (int e = tid; e < nhalo; e += blockDim.x) {
                        const int h = e / A.hw, bx = e - h * A.hw;          // halo row, point pair
                        const int r = h < kRadius ? B.y0 - kRadius + h : B.y1 + h - kRadius;
                        if (r < 0 || r >= A.ny) continue;                   // outside the box: read as zeros
                        const unsigned src = (h < kRadius ? ring_up : ring_dn) + cs * psb +
                                             (2 + (h < kRadius ? r - (B.y0 - rows) : r - B.y1) * A.rs + 2 * bx) * 8;
                        float2 a, b;
                        ring_pair_cl(src, a, b);
                        *reinterpret_cast<float4 *>(hb + (2 + h * A.rs + 2 * bx) * 8) = make_float4(a.x, a.y, b.x, b.y);
                    }
                }
                // 4. q_k on plane z, its 6 neighbour planes from the ring, rows past the band from the halo
                if (U.own && z >= 0) {
                    const int cz = u >= kRadius ? u - kRadius : u + kRingPlanes - kRadius;   // ring slot of z
                    if (remote) {
                        B.halo = halo + (z & 1) * hsb;
                        ring_stencil<EVEN, false, true>(U, ring, psb, rsb, A.hw, A.ny, cz, z * plane + U.col0, rk, vv,
                                                        shr, shi, cf, qs, sa, B);
                    } else {
                        ring_stencil<EVEN, false>(U, ring, psb, rsb, A.hw, A.ny, cz, z * plane + U.col0, rk, vv, shr,
                                                  shi, cf, qs, sa);
                    }
                }
            }
            if ((nsteps - 1) % kClusterEvery == 0) cluster_wait();   // the last arrival's phase
            // the sweep's sums: the band's, then the cluster's in rank order (rank 0)
            double v[9] = {fa[0], fa[1], fa[2], sa[0], sa[1], sa[2], sa[3], sa[4], sa[5]};
            block_sum_any<9>(v);
            if (tid == 0)
                for (int c = 0; c < 9; ++c) cl_part[c] = v[c];
            cl.sync();
            if (rank == 0 && tid == 0) {
                double tot[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                for (int t = 0; t < ncl; ++t) {
                    const double *pt = cl.map_shared_rank(cl_part, t);
                    for (int c = 0; c < 9; ++c) tot[c] += pt[c];
                }
                const int m = ring_scalar_step(A, sl, tot) ? 1 : 0;
                if (A.prof) {
                    atomicAdd(A.prof + 1, (unsigned long long)A.nd);
                    if (first) atomicAdd(A.prof + 2, (unsigned long long)A.nd);
                }
                for (int t = 0; t < ncl; ++t) *cl.map_shared_rank(&cl_more, t) = m;
            }
            cl.sync();                             // also: every block's ring readers of the sweep are done
            more = cl_more != 0;
        }
    }
    cl.sync();                                     // no block leaves while another may read its ring
}

// Warp-specialised form of the fused kernel: the first threads (consumers, one unit each) apply
// the stencil to plane f-6 while the threads after them (producers, two units each, one after the
// other) form plane f+1, so the front's global-memory latency and the stencil's shared-memory work
// overlap.  The producers
// write the ring slot of plane f-13 during step f, which no consumer reads at that step (they
// read f-12 .. f), and one barrier per step hands the planes over.
template <bool EVEN>
__global__ void __maxnreg__(96)
    k_cocg_ring_ws(RingArgs A, float2 *__restrict__ xg, float2 *__restrict__ rg, float2 *__restrict__ pg,
                   float2 *__restrict__ qg, const float *__restrict__ vloc, Coef<float> cf) {
    extern __shared__ float4 ring4[];
    unsigned char *const ring = reinterpret_cast<unsigned char *>(ring4);
    const int tid = threadIdx.x;
    const int nz = A.nz, plane = A.nx * A.ny;
    const int rsb = A.rs * 8, psb = A.ps * 8;
    const int nunits = A.hw * A.hh;
    const int ncons = (nunits + 31) / 32 * 32;     // consumer threads; the rest produce
    const int nprod = ((nunits + 1) / 2 + 31) / 32 * 32;
    const bool producer = tid >= ncons;
    const int pt = tid - ncons;                    // producer index: units pt and pt + nprod
    const RingUnit U = ring_unit(producer ? -1 : tid, A);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = tid; e < kRingPlanes * A.ps / 2; e += blockDim.x) ring4[e] = zero4;   // padding stays zero
    const int n_items = *A.cnt_in;
    for (int s; (s = ring_next_item(A, n_items)) >= 0;) {
        Slot &sl = A.slots[s];
        const float shr = (float)sl.shift_re, shi = (float)sl.shift_im;
        const long long off = (long long)s * A.nd;
        float2 *const xs = xg + off;
        float2 *const rsv = rg + off;
        float2 *const psv = pg + off;
        float2 *const qs = qg + off;
        bool more = true;
        while (more) {                             // sweeps of this system (iterations of COCG)
            const bool first = sl.iters == 0;
            const float alr = (float)sl.alpha_re, ali = (float)sl.alpha_im;
            const float ber = (float)sl.beta_re, bei = (float)sl.beta_im;
            float fa[3] = {0.f, 0.f, 0.f}, sa[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            __syncthreads();                       // the previous sweep's ring readers are done
            if (producer)                          // planes -6 .. -1 (ring slots 8 .. 13) are zero; plane 0
                for (int pu = pt; pu < nunits; pu += nprod) {
                    const RingUnit P = ring_unit(pu, A);
#pragma unroll
                    for (int m = kRingPlanes - kRadius; m < kRingPlanes; ++m) {
                        *reinterpret_cast<float4 *>(ring + m * psb + P.rb0) = zero4;
                        if (P.row1) *reinterpret_cast<float4 *>(ring + m * psb + P.rb1) = zero4;
                    }
                    RingFront F;
                    ring_load_front<EVEN>(P, P.col0, first, xs, rsv, psv, qs, F);
                    ring_front<EVEN>(P, 0, nz, plane, first, alr, ali, ber, bei, F, xs, rsv, psv, ring, fa);
                }
            __syncthreads();
            const int nsteps = nz + kRadius;
            for (int f = 0, u = 0; f < nsteps; ++f, u = (u + 1 == kRingPlanes) ? 0 : u + 1) {
                if (producer) {
                    // plane f + 1 into ring slot u + 1
                    if (f + 1 < nsteps) {
                        const int un = u + 1 == kRingPlanes ? 0 : u + 1;
                        for (int pu = pt; pu < nunits; pu += nprod) {
                            const RingUnit P = ring_unit(pu, A);
                            RingFront F;
                            if (f + 1 < nz)
                                ring_load_front<EVEN>(P, (f + 1) * plane + P.col0, first, xs, rsv, psv, qs, F);
                            ring_front<EVEN>(P, f + 1, nz, plane, first, alr, ali, ber, bei, F, xs, rsv, psv,
                                             ring + un * psb, fa);
                        }
                    }
                } else {
                    const int z = f - kRadius;
                    if (U.own && z >= 0) {
                        float2 rk[4] = {};
                        float vv[4] = {0.f, 0.f, 0.f, 0.f};
                        ring_load_rv<EVEN>(U, z * plane + U.col0, rsv, vloc, rk, vv);
                        const int cz = u >= kRadius ? u - kRadius : u + kRingPlanes - kRadius;
                        ring_stencil<EVEN, false>(U, ring, psb, rsb, A.hw, A.ny, cz, z * plane + U.col0, rk, vv, shr,
                                                  shi, cf, qs, sa);
                    }
                }
                __syncthreads();
            }
            more = ring_end_sweep(A, sl, first, fa, sa);
        }
    }
}

// Active list of the fused kernel's launch: the slots whose inner solve runs, in slot order
// (block scan); clears the other list counters.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) k_ring_list(Params P) {
    __shared__ int wsum[32];
    __shared__ int base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) base = 0;
    if (tid < 3) P.cnt[1 + tid] = 0;
    __syncthreads();
    for (int s0 = 0; s0 < P.S; s0 += blockDim.x) {
        const int s = s0 + tid;
        const int f = (s < P.S && P.slots[s].phase == kInner) ? 1 : 0;
        int x = f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int t = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            wsum[lane] = t;
        }
        __syncthreads();
        const int excl = x - f + (warp > 0 ? wsum[warp - 1] : 0);
        if (f) P.list[base + excl] = s;
        __syncthreads();
        if (tid == 0) base += wsum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (tid == 0) P.cnt[0] = base;
}

using RingFn = void (*)(RingArgs, float2 *, float2 *, float2 *, float2 *, const float *, Coef<float>);

// The fused kernel applies when a plane's ring fits in a block's shared memory (beside the
// kernel's static shared memory) and a plane has at most kRingMaxThreads blocks of 2 x 2 points.
bool ring_fits(int nx, int ny, RingFn fn, int smem_optin, bool ws = false) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    const long long units = (long long)((nx + 1) / 2) * ((ny + 1) / 2);
    const long long threads = ws ? (units + 31) / 32 * 32 + ((units + 1) / 2 + 31) / 32 * 32 : units;
    return threads <= (ws ? kRingWsMaxThreads : kRingMaxThreads) &&
           ring_bytes(nx, ny) + fa.sharedSizeBytes <= (size_t)smem_optin;
}

// Cluster form of the fused kernel: the smallest cluster of C <= 8 blocks whose bands of bp row pairs
// (bp >= 3, every band non-empty) fit a block's shared memory and kRingMaxThreads units.  With
// `two_per_sm` it asks for rings small enough for two blocks per SM.  False where none fits.
bool cluster_plan(int nx, int ny, int smem_optin, bool two_per_sm, int &ncl, int &bp) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k_cocg_ring_cl<true>) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    const int hw = (nx + 1) / 2, hh = (ny + 1) / 2, rs = 2 * hw + ring_row_pad(hw);
    const size_t limit = two_per_sm ? (size_t)smem_optin / 2 - 1024 : (size_t)smem_optin;
    for (int c = 2; c <= 8; ++c) {
        const int b = (hh + c - 1) / c;
        if (b < 3 || (long long)(c - 1) * b >= hh) continue;
        const size_t bytes = ((size_t)kRingPlanes * (2 + (size_t)2 * b * rs) + 2 * (2 + (size_t)2 * kRadius * rs)) *
                                 sizeof(float2) + fa.sharedSizeBytes;
        if ((long long)hw * b <= kRingMaxThreads && bytes <= limit) {
            ncl = c;
            bp = b;
            return true;
        }
    }
    return false;
}

// ---------------------------------------------------------------------------------------------
// Maintenance kernels (between epochs).  Slot phases do not change while these item kernels
// run, so every thread of a block reads the same phase.
// ---------------------------------------------------------------------------------------------
// Mixed form: the FP32 inner solve works on the residual times a per-slot scale chosen so that
// its norm starts near 1.  Late refinements (tol 1e-12 of a small ||b||) would otherwise run
// FP32 COCG on values whose squares fall into FP32's subnormal range.  The scale of the next
// inner solve comes from the norm the last one ended at (its recursive residual, which tracks
// the true one to within the FP32 accuracy), limited to 1e12 per step.
__device__ __forceinline__ double next_scale(const Slot &sl) {
    const double rn = sl.rnorm;
    if (sl.discard || !isfinite(rn) || !(rn > 0.0)) return sl.scale;
    return sl.scale / fmax(rn, 1e-12 * sl.ref_norm);
}

// Mixed form, slots whose inner solve ended: the correction d' = d (projected first when
// P.cproject) goes into x64 += d' / scale and, for the residual update, into dq (the idle q
// buffer); d is cleared for the next inner solve.  A correction that went non-finite is dropped:
// only d is cleared.
__global__ void __launch_bounds__(kThreads) k_refine_x(Params P, double2 *__restrict__ x64, float2 *__restrict__ d,
                                                       float2 *__restrict__ dq) {
    const long long items = (long long)P.S * P.nblk;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = (int)(it / P.nblk), chunk = (int)(it % P.nblk);
        const Slot &sl = P.slots[s];
        if (sl.phase != kInnerDone) continue;
        const bool keep = !sl.discard;
        const double inv = 1.0 / sl.scale;
        const long long off = (long long)s * P.g.nd;
        const float *tp = P.Tp32 + (long long)s * P.ns * 2;
        for (int t = 0; t < kPPT; ++t) {
            const long long idx = (long long)chunk * kChunk + t * kThreads + threadIdx.x;
            if (idx < P.g.nd) {
                if (keep) {
                    double2 xv = x64[off + idx];
                    float2 dv = d[off + idx];
                    if (P.cproject)
                        for (int k = 0; k < P.ns; ++k) {
                            const float u = P.psi32[(long long)k * P.g.nd + idx];
                            dv.x -= tp[2 * k] * u;
                            dv.y -= tp[2 * k + 1] * u;
                        }
                    xv.x += (double)dv.x * inv;
                    xv.y += (double)dv.y * inv;
                    x64[off + idx] = xv;
                    dq[off + idx] = dv;
                }
                d[off + idx] = make_float2(0.f, 0.f);
            }
        }
    }
}

// Error-free transformations on FP32 (Knuth's TwoSum; the product error from one fma), the
// building blocks of double-float ("float-float") arithmetic: a value is an unevaluated sum
// hi + lo of two FP32 numbers, ~48 significant bits (Ogita, Rump and Oishi, "Accurate sum and dot
// product", 2005, use the same transformations).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (S, E) += (hi, lo) * x for an FP32 x: the product's rounding error is exact through fma.
__device__ __forceinline__ void df_mad(float hi, float lo, float x, float &S, float &E) {
    const float p = __fmul_rn(hi, x);
    const float pe = __fmaf_rn(hi, x, -p);
    float t;
    two_sum(S, p, S, t);
    E += t + pe + lo * x;
}

// (H + sigma) v at one point in double-float arithmetic for an FP32 complex v: the six
// neighbours at each distance are summed exactly (TwoSum), multiplied by the split coefficient
// (hi + lo) and accumulated with their rounding errors.  Zero outside the box.
__device__ __forceinline__ void df_stencil(const float2 *__restrict__ v, long long idx, int i, int j, int k,
                                           const Grid3 &g, const Coef<float> &ch, const Coef<float> &cl, float dh,
                                           float dl, float oh, float ol, float (&re)[2], float (&im)[2]) {
    const float2 c = v[idx];
    float Sr = 0.f, Er = 0.f, Si = 0.f, Ei = 0.f;
    df_mad(dh, dl, c.x, Sr, Er);          // (3 a0 + V + sigma_re) c
    df_mad(dh, dl, c.y, Si, Ei);
    df_mad(-oh, -ol, c.y, Sr, Er);        // i sigma_im c
    df_mad(oh, ol, c.x, Si, Ei);
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
#pragma unroll
    for (int s = 1; s <= kRadius; ++s) {
        float ar = 0.f, er = 0.f, ai = 0.f, ei = 0.f, t;
        auto add = [&](float2 u) {
            two_sum(ar, u.x, ar, t);
            er += t;
            two_sum(ai, u.y, ai, t);
            ei += t;
        };
        if (g.periodic) {
            add(v[idx + (wrap_index(i - s, g.nx) - i)]);
            add(v[idx + (wrap_index(i + s, g.nx) - i)]);
            add(v[idx + (wrap_index(j - s, g.ny) - j) * sy]);
            add(v[idx + (wrap_index(j + s, g.ny) - j) * sy]);
            add(v[idx + (wrap_index(k - s, g.nz) - k) * sz]);
            add(v[idx + (wrap_index(k + s, g.nz) - k) * sz]);
        } else {
            if (i - s >= 0) add(v[idx - s]);
            if (i + s < g.nx) add(v[idx + s]);
            if (j - s >= 0) add(v[idx - s * sy]);
            if (j + s < g.ny) add(v[idx + s * sy]);
            if (k - s >= 0) add(v[idx - s * sz]);
            if (k + s < g.nz) add(v[idx + s * sz]);
        }
        // a_s (ar + er): the sum's low part times the coefficient's high part joins the error term
        df_mad(ch.a[s], cl.a[s], ar, Sr, Er);
        Er += ch.a[s] * er;
        df_mad(ch.a[s], cl.a[s], ai, Si, Ei);
        Ei += ch.a[s] * ei;
    }
    re[0] = Sr;
    re[1] = Er;
    im[0] = Si;
    im[1] = Ei;
}

// Mixed form: the FP64 residual of the slots whose inner solve ended, updated with their
// correction, r64 -= (H + sigma) d' / scale, where (H + sigma) d' is evaluated in double-float
// arithmetic on the FP32 pipes from the FP32 correction d' (the coefficients and V_loc split into
// FP32 pairs).  It agrees with recomputing b - (H + sigma) x64 in FP64 to ~2^-48 of the update,
// without the ~90 FP64 operations per point that GB300's FP64 rate makes the bottleneck.  The next
// inner solve starts from r32 = scale * r64 (scale = next_scale) with p = 0 (d was cleared by
// k_refine_x).  Partials (into partB): r32^T r32 and ||scale * r64||^2, summed in FP32 per thread.
// (Continuing the FP32 recurrence with the replaced residual instead of restarting was measured
// to lose convergence: the FP32 recursive residual can be far below the true one.)
__global__ void __launch_bounds__(kThreads) k_residual_df(Params P, double2 *__restrict__ r64,
                                                          const float2 *__restrict__ dq, float2 *__restrict__ r32,
                                                          float2 *__restrict__ p32, const float *__restrict__ vhi,
                                                          const float *__restrict__ vlo, Coef<float> ch,
                                                          Coef<float> cl, double a0x3) {
    const long long items = (long long)P.S * P.nblk;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = (int)(it / P.nblk), chunk = (int)(it % P.nblk);
        const Slot &sl = P.slots[s];
        if (sl.phase != kInnerDone) continue;
        const bool upd = !sl.discard;
        const double sc = next_scale(sl), inv = 1.0 / sl.scale;
        // 3 a0 + sigma_re and sigma_im as FP32 pairs
        const double d0 = a0x3 + sl.shift_re;
        const float d0h = (float)d0, d0l = (float)(d0 - (double)d0h);
        const float oh = (float)sl.shift_im, ol = (float)(sl.shift_im - (double)oh);
        const long long off = (long long)s * P.g.nd;
        float v0 = 0.f, v1 = 0.f, v2 = 0.f;
        for (int t = 0; t < kPPT; ++t) {
            const long long idx = (long long)chunk * kChunk + t * kThreads + threadIdx.x;
            if (idx < P.g.nd) {
                double2 rv = r64[off + idx];
                if (upd) {
                    int i, j, k;
                    coords(idx, P.g, i, j, k);
                    float dh, dl, e;                      // 3 a0 + V + sigma_re as a pair
                    two_sum(d0h, vhi[idx], dh, e);
                    dl = e + d0l + vlo[idx];
                    float re[2], im[2];
                    df_stencil(dq + off, idx, i, j, k, P.g, ch, cl, dh, dl, oh, ol, re, im);
                    rv.x = fma(-((double)re[0] + (double)re[1]), inv, rv.x);
                    rv.y = fma(-((double)im[0] + (double)im[1]), inv, rv.y);
                    r64[off + idx] = rv;
                }
                const float2 rf = make_float2((float)(rv.x * sc), (float)(rv.y * sc));
                r32[off + idx] = rf;
                p32[off + idx] = make_float2(0.f, 0.f);         // direction buffer of iteration 0
                v0 += rf.x * rf.x - rf.y * rf.y;
                v1 += 2.f * rf.x * rf.y;
                v2 += rf.x * rf.x + rf.y * rf.y;
            }
        }
        const float vf[3] = {v0, v1, v2};
        double v[3];
        block_sum_t<float, 3>(vf, v);
        if (threadIdx.x == 0) {
            double *o = P.partB + ((long long)s * P.nblk + chunk) * 3;
            o[0] = v[0];
            o[1] = v[1];
            o[2] = v[2];
        }
    }
}

// Mixed form with projected right-hand sides (P.cproject): the refinement works in the
// unoccupied space, where the solution lies.  Each FP32 solve leaves occupied components of
// ~1e-7 ||d|| in its correction d; accumulated in x64 they put occupied components into the
// residual, and the next inner solves would have to solve for them, where (H - eps_n + i omega)
// is indefinite (eigenvalues eps_k - eps_n + i omega, k <= n) and COCG stagnates.  So both the
// correction (before x64 absorbs it) and the FP32 residual (before the inner solve) are
// projected, v <- v - sum_k (u_k . v) u_k, and convergence is tested on ||P_c r||.  FP32 dots
// against FP32 orbitals resolve the occupied components to ~1e-9 of the vector's norm, which
// keeps those of x64 far below the residuals the refinement reaches.
// Partial sums of u_k . v over each item of the slots whose inner solve ended, for k < ns.
// (Projecting the residual only in late refinements was measured to cost more than it saves:
// the occupied components of the first refinement's residual raise the next inner solve's
// iterations by 15% at 40^3.)
// A work item is one chunk of grid points of kSlotGroup consecutive slots: each orbital value
// loaded (from L2) serves all of them.  A thread sums its kPPT points in FP32 for kDotK orbitals
// at a time (32 sums: kDotK orbitals x kSlotGroup slots x re/im), its warp adds them over the
// lanes with a transposing butterfly (each level exchanges half of the remaining sums, so 31
// shuffles give lane l the warp's total of sum l, instead of 5 shuffles per sum), and the warps'
// totals are added in FP64 in warp order: one barrier per kDotBatch orbitals instead of a block
// reduction per orbital.  Fixed order throughout.
constexpr int kSlotGroup = 4;
constexpr int kDotK = 4;                          // orbitals per butterfly (kDotK * 2 * kSlotGroup = 32)
constexpr int kDotBatch = 32;                     // orbitals per shared-memory batch
static_assert(kDotK * 2 * kSlotGroup == 32, "one butterfly reduces 32 sums");

// In-warp transposing reduction: on return lane l holds the sum over the warp's lanes of a[l].
__device__ __forceinline__ float warp_transpose_sum(float (&a)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;          // this lane keeps the upper half of the h-blocks
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float keep = up ? a[i + h] : a[i];
            const float send = up ? a[i] : a[i + h];
            a[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    return a[0];
}

__global__ void __launch_bounds__(kThreads) k_cproj_dots(Params P, const float2 *__restrict__ v) {
    __shared__ float red[kWarpsPerBlock][kDotBatch * 2 * kSlotGroup];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ngroups = (P.S + kSlotGroup - 1) / kSlotGroup;
    const long long items = (long long)ngroups * P.nblk;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int g = (int)(it / P.nblk), chunk = (int)(it % P.nblk);
        bool act[kSlotGroup];
        bool any = false;
#pragma unroll
        for (int q = 0; q < kSlotGroup; ++q) {
            const int s = g * kSlotGroup + q;
            act[q] = s < P.S && P.slots[s].phase == kInnerDone;
            any = any || act[q];
        }
        if (!any) continue;                              // uniform per block
        float2 vv[kSlotGroup][kPPT];
#pragma unroll
        for (int q = 0; q < kSlotGroup; ++q)
#pragma unroll
            for (int t = 0; t < kPPT; ++t) {
                const long long idx = (long long)chunk * kChunk + t * kThreads + threadIdx.x;
                vv[q][t] = (act[q] && idx < P.g.nd) ? v[(long long)(g * kSlotGroup + q) * P.g.nd + idx]
                                                    : make_float2(0.f, 0.f);
            }
        for (int k0 = 0; k0 < P.ns; k0 += kDotBatch) {
            const int kn = min(kDotBatch, P.ns - k0);
            for (int kk = 0; kk < kn; kk += kDotK) {
                float a[32];
#pragma unroll
                for (int j = 0; j < kDotK; ++j) {
                    const int k = k0 + kk + j;
                    float2 acc[kSlotGroup];
#pragma unroll
                    for (int q = 0; q < kSlotGroup; ++q) acc[q] = make_float2(0.f, 0.f);
                    if (k < P.ns) {
#pragma unroll
                        for (int t = 0; t < kPPT; ++t) {
                            const long long idx = (long long)chunk * kChunk + t * kThreads + threadIdx.x;
                            const float u = idx < P.g.nd ? P.psi32[(long long)k * P.g.nd + idx] : 0.f;
                            const float2 uu = make_float2(u, u);
#pragma unroll
                            for (int q = 0; q < kSlotGroup; ++q) acc[q] = __ffma2_rn(uu, vv[q][t], acc[q]);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < kSlotGroup; ++q) {
                        a[j * 2 * kSlotGroup + 2 * q] = acc[q].x;
                        a[j * 2 * kSlotGroup + 2 * q + 1] = acc[q].y;
                    }
                }
                red[warp][kk * 2 * kSlotGroup + lane] = warp_transpose_sum(a);
            }
            __syncthreads();
            // thread e: orbital k0 + e / (2 kSlotGroup), slot e / 2 % kSlotGroup, part e % 2
            for (int e = threadIdx.x; e < kn * 2 * kSlotGroup; e += blockDim.x) {
                const int q = (e >> 1) % kSlotGroup;
                if (act[q]) {
                    double sum = 0.0;
#pragma unroll
                    for (int w = 0; w < kWarpsPerBlock; ++w) sum += (double)red[w][e];
                    const int s = g * kSlotGroup + q, k = k0 + e / (2 * kSlotGroup);
                    P.partP[(((long long)s * P.nblk + chunk) * P.ns + k) * 2 + (e & 1)] = sum;
                }
            }
            __syncthreads();
        }
    }
}

// P.cproject: r32 -= sum_k Tp[s][k] u_k for the slots whose inner solve ended; partials (into
// partB): r32^T r32 and ||r32||^2 of the projected residual.
__global__ void __launch_bounds__(kThreads) k_cproj_residual(Params P, float2 *__restrict__ r32) {
    const long long items = (long long)P.S * P.nblk;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = (int)(it / P.nblk), chunk = (int)(it % P.nblk);
        if (P.slots[s].phase != kInnerDone) continue;
        const long long off = (long long)s * P.g.nd;
        const float *tp = P.Tp32 + (long long)s * P.ns * 2;
        double v[3] = {0.0, 0.0, 0.0};
        for (int t = 0; t < kPPT; ++t) {
            const long long idx = (long long)chunk * kChunk + t * kThreads + threadIdx.x;
            if (idx < P.g.nd) {
                float2 rv = r32[off + idx];
                for (int k = 0; k < P.ns; ++k) {
                    const float u = P.psi32[(long long)k * P.g.nd + idx];
                    rv.x -= tp[2 * k] * u;
                    rv.y -= tp[2 * k + 1] * u;
                }
                r32[off + idx] = rv;
                v[0] += (double)rv.x * rv.x - (double)rv.y * rv.y;
                v[1] += 2.0 * (double)rv.x * rv.y;
                v[2] += (double)rv.x * rv.x + (double)rv.y * rv.y;
            }
        }
        block_sum<3>(v);
        if (threadIdx.x == 0) {
            double *o = P.partB + ((long long)s * P.nblk + chunk) * 3;
            o[0] = v[0];
            o[1] = v[1];
            o[2] = v[2];
        }
    }
}

// Per-slot transitions after a refinement or a load (one warp per slot).
__global__ void k_state(Params P) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= P.S) return;
    Slot &sl = P.slots[w];
    const int ph = sl.phase;
    if (ph != kInnerDone && ph != kLoading) return;
    double v[3];
    warp_slot_sum<3, 3>(P.partB + (long long)w * P.nblk * 3, P.nblk, v);
    if (lane != 0) return;
    const double rn = sqrt(v[2]);
    if (ph == kLoading) {
        sl.bnorm = rn;
        sl.ref_norm = rn;
        sl.rnorm = rn;
        sl.iters = 0;
        sl.total_iters = 0;
        sl.refines = 0;
        sl.status = RPA_OK;
        sl.discard = 0;
        sl.nearbreak = 0;
        sl.scale = 1.0;
        sl.phase = (rn > 0.0) ? kInner : kFinished;
        return;
    }
    // kInnerDone (mixed form): rn = ||scale * (b - A x64)|| with the scale of the next inner solve
    const double sc = next_scale(sl);
    sl.refines += 1;
    sl.scale = sc;
    sl.discard = 0;
    sl.rnorm = rn;
    if (rn <= P.tol * sl.bnorm * sc) {
        sl.status = RPA_OK;
        sl.phase = kFinished;
    } else if (sl.status == RPA_ERR_BREAKDOWN) {
        sl.phase = kFinished;
    } else if (sl.refines >= P.max_refine || !isfinite(rn)) {
        sl.status = RPA_ERR_NOT_CONVERGED;
        sl.phase = kFinished;
    } else {
        sl.ref_norm = rn;
        sl.iters = 0;
        sl.phase = kInner;
    }
}

// Partial sums of u_k . x64 (complex) over each item of the finished slots, for k < ns.
constexpr int kProjGroup = 8;   // orbitals reduced together (one block reduction per group)
__global__ void __launch_bounds__(kThreads) k_proj_dots(Params P, const double2 *__restrict__ x64) {
    const long long items = (long long)P.S * P.nblk;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = (int)(it / P.nblk), chunk = (int)(it % P.nblk);
        if (P.slots[s].phase != kFinished) continue;
        const long long off = (long long)s * P.g.nd;
        double2 xv[kPPT];
#pragma unroll
        for (int t = 0; t < kPPT; ++t) {
            const long long idx = (long long)chunk * kChunk + t * kThreads + threadIdx.x;
            xv[t] = idx < P.g.nd ? x64[off + idx] : make_double2(0.0, 0.0);
        }
        for (int k0 = 0; k0 < P.ns; k0 += kProjGroup) {
            double v[2 * kProjGroup];
#pragma unroll
            for (int g = 0; g < kProjGroup; ++g) {
                double a0 = 0.0, a1 = 0.0;
                if (k0 + g < P.ns) {
#pragma unroll
                    for (int t = 0; t < kPPT; ++t) {
                        const long long idx = (long long)chunk * kChunk + t * kThreads + threadIdx.x;
                        if (idx < P.g.nd) {
                            const double u = P.psi[(long long)(k0 + g) * P.g.nd + idx];
                            a0 += u * xv[t].x;
                            if (!P.proj_re_only) a1 += u * xv[t].y;
                        }
                    }
                }
                v[2 * g] = a0;
                v[2 * g + 1] = a1;
            }
            block_sum<2 * kProjGroup>(v);
            if (threadIdx.x == 0)
                for (int g = 0; g < kProjGroup && k0 + g < P.ns; ++g) {
                    double *o = P.partP + (((long long)s * P.nblk + chunk) * P.ns + k0 + g) * 2;
                    o[0] = v[2 * g];
                    o[1] = v[2 * g + 1];
                }
        }
    }
}

// Tp[s][k] = sum over items of the partial dots (fixed order); one warp per slot in phase ph.
__global__ void k_proj_sum(Params P, int ph) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= P.S || P.slots[w].phase != ph) return;
    for (int k = 0; k < P.ns; ++k) {
        double v[2];
        const double *base = P.partP + ((long long)w * P.nblk * P.ns + k) * 2;
        v[0] = v[1] = 0.0;
        for (int b = lane; b < P.nblk; b += 32) {
            v[0] += base[(long long)b * P.ns * 2 + 0];
            v[1] += base[(long long)b * P.ns * 2 + 1];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
            v[1] += __shfl_xor_sync(0xffffffffu, v[1], o);
        }
        if (lane == 0) {
            P.Tp[((long long)w * P.ns + k) * 2 + 0] = v[0];
            P.Tp[((long long)w * P.ns + k) * 2 + 1] = v[1];
            P.Tp32[((long long)w * P.ns + k) * 2 + 0] = (float)v[0];
            P.Tp32[((long long)w * P.ns + k) * 2 + 1] = (float)v[1];
        }
    }
}

// The finished solution of slot s at one point, with its occupied components removed when
// P.project is set.
__device__ __forceinline__ double2 solution_at(const Params &P, const double2 *__restrict__ x64, int s, long long idx) {
    double2 x = x64[(long long)s * P.g.nd + idx];
    if (P.project) {
        const double *t = P.Tp + (long long)s * P.ns * 2;
        for (int k = 0; k < P.ns; ++k) {
            const double u = P.psi[(long long)k * P.g.nd + idx];
            x.x -= t[2 * k] * u;
            x.y -= t[2 * k + 1] * u;
        }
    }
    return x;
}

// fin_list = the finished slots in slot order (block scan), so that the retiring kernels visit
// only those, in the same order as a scan over all slots.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) k_finished_list(Params P) {
    __shared__ int wsum[32];
    __shared__ int base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) base = 0;
    __syncthreads();
    for (int s0 = 0; s0 < P.S; s0 += blockDim.x) {
        const int s = s0 + tid;
        const int f = (s < P.S && P.slots[s].phase == kFinished) ? 1 : 0;
        int x = f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            wsum[lane] = v;
        }
        __syncthreads();
        const int excl = x - f + (warp > 0 ? wsum[warp - 1] : 0);
        if (f) P.fin_list[base + excl] = s;
        __syncthreads();
        if (tid == 0) base += wsum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (tid == 0) *P.fin_cnt = base;
}

// grad += scale * coef[j] * Re(x^2) for every finished slot, slots added in slot order.
__global__ void k_retire_grad(Params P, const double2 *__restrict__ x64, const double *__restrict__ coef,
                              double *__restrict__ grad, double scale) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < P.g.nd;
         idx += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        const int nf = *P.fin_cnt;
        for (int i = 0; i < nf; ++i) {
            const int s = P.fin_list[i];
            const Slot &sl = P.slots[s];
            const double2 x = solution_at(P, x64, s, idx);
            acc += coef[sl.j] * (x.x * x.x - x.y * x.y);
        }
        grad[idx] += scale * acc;
    }
}

// drho_j += (4/h^3) u_n (.) Re x64 for every finished slot, slots added in slot order.
__global__ void k_retire_drho(Params P, const double2 *__restrict__ x64, const double *__restrict__ psi,
                              double *__restrict__ drho, double scale) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < P.g.nd;
         idx += (long long)gridDim.x * blockDim.x) {
        const int nf = *P.fin_cnt;
        for (int i = 0; i < nf; ++i) {
            const int s = P.fin_list[i];
            const Slot &sl = P.slots[s];
            drho[(long long)sl.j * P.g.nd + idx] +=
                scale * psi[(long long)sl.n * P.g.nd + idx] * solution_at(P, x64, s, idx).x;
        }
    }
}

// x_out[sys] = x64 for every finished slot.
__global__ void k_retire_copy(Params P, const double2 *__restrict__ x64, double2 *__restrict__ xout) {
    const long long items = (long long)P.S * P.nblk;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = (int)(it / P.nblk), chunk = (int)(it % P.nblk);
        const Slot &sl = P.slots[s];
        if (sl.phase != kFinished) continue;
        for (int t = 0; t < kPPT; ++t) {
            const long long idx = (long long)chunk * kChunk + t * kThreads + threadIdx.x;
            if (idx < P.g.nd) xout[(long long)sl.sys * P.g.nd + idx] = solution_at(P, x64, s, idx);
        }
    }
}

// Finished slots report and empty; empty slots take the next systems in slot order (a block
// scan keeps the assignment deterministic); count what is left.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) k_refill(Params P, const int *__restrict__ sys_n,
                                                 const int *__restrict__ sys_j, const double *__restrict__ eps,
                                                 double omega) {
    __shared__ int wsum[32];
    __shared__ int base_head, busy_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        base_head = *P.head;
        busy_total = 0;
        P.cnt[0] = 0;
    }
    __syncthreads();
    for (int s0 = 0; s0 < P.S; s0 += blockDim.x) {
        const int s = s0 + tid;
        int want = 0;
        Slot *sl = s < P.S ? P.slots + s : nullptr;
        if (sl) {
            if (sl->phase == kFinished) {
                if (sl->sys >= 0) {
                    P.sys_out[sl->sys] = sl->total_iters;
                    P.sys_out[P.nsys + sl->sys] = sl->status;
                    P.sys_out[2 * P.nsys + sl->sys] = sl->refines;
                    P.sys_out[3 * P.nsys + sl->sys] = sl->nearbreak;
                }
                sl->phase = kEmpty;
                sl->sys = -1;
            }
            want = sl->phase == kEmpty;
        }
        // exclusive scan of want over the block
        int x = want;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int t = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            wsum[lane] = t;    // inclusive prefix over warps
        }
        __syncthreads();
        const int excl = x - want + (warp > 0 ? wsum[warp - 1] : 0);
        const int total = wsum[(blockDim.x >> 5) - 1];
        if (sl && want) {
            const int q = base_head + excl;
            if (q < P.nsys) {
                sl->sys = q;
                sl->n = sys_n[q];
                sl->j = sys_j[q];
                sl->shift_re = -eps[sl->n];
                sl->shift_im = omega;
                sl->status = RPA_OK;
                sl->phase = kLoading;
            }
        }
        const int busy = (sl && sl->phase != kEmpty) ? 1 : 0;
        if (busy) atomicAdd(&busy_total, 1);
        __syncthreads();
        if (tid == 0) base_head = min(P.nsys, base_head + total);
        __syncthreads();
    }
    if (tid == 0) {
        *P.head = base_head;
        *P.count = busy_total + (P.nsys - base_head);
    }
}

// Load the right-hand side of every loading slot:
//   b = sign * (base - sum_k T[sys][k] u_k),  base = u_n (.) vt_j (pair) or rhs[sys]
// then x64 = 0, the FP64 residual r64 = b (mixed form), and the inner vectors start from r = b,
// x = 0, p = 0.  Partials: r^T r, ||b||^2.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_load(Params P, const double *__restrict__ psi, int ns,
                                                   const double *__restrict__ vt, const double *__restrict__ rhs,
                                                   const double *__restrict__ Tc, double sign, double2 *__restrict__ b,
                                                   double2 *__restrict__ x64, typename Cx<T>::t *__restrict__ xin,
                                                   typename Cx<T>::t *__restrict__ r, typename Cx<T>::t *__restrict__ p,
                                                   long long pstride) {
    using C = typename Cx<T>::t;
    const long long items = (long long)P.S * P.nblk;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = (int)(it / P.nblk), chunk = (int)(it % P.nblk);
        const Slot &sl = P.slots[s];
        if (sl.phase != kLoading) continue;
        const long long off = (long long)s * P.g.nd;
        const double *tc = Tc ? Tc + (long long)sl.sys * ns : nullptr;
        double v[3] = {0.0, 0.0, 0.0};
        for (int t = 0; t < kPPT; ++t) {
            const long long idx = (long long)chunk * kChunk + t * kThreads + threadIdx.x;
            if (idx < P.g.nd) {
                double base = vt ? psi[(long long)sl.n * P.g.nd + idx] * vt[(long long)sl.j * P.g.nd + idx]
                                 : rhs[(long long)sl.sys * P.g.nd + idx];
                if (tc)
                    for (int k = 0; k < ns; ++k) base -= tc[k] * psi[(long long)k * P.g.nd + idx];
                const double bv = sign * base;
                b[off + idx] = make_double2(bv, 0.0);     // the FP64 residual of x64 = 0
                x64[off + idx] = make_double2(0.0, 0.0);
                C z;
                z.x = (T)0;
                z.y = (T)0;
                C rv;
                rv.x = (T)bv;
                rv.y = (T)0;
                if ((const void *)xin != (const void *)x64) xin[off + idx] = z;
                r[off + idx] = rv;
                p[off + idx] = z;
                p[pstride + off + idx] = z;
                v[0] += (double)rv.x * rv.x;
                v[2] += bv * bv;
            }
        }
        block_sum<3>(v);
        if (threadIdx.x == 0) {
            double *o = P.partB + ((long long)s * P.nblk + chunk) * 3;
            o[0] = v[0];
            o[1] = v[1];
            o[2] = v[2];
        }
    }
}

__global__ void k_init_slots(Slot *slots, int S) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    Slot z = {};
    z.phase = kEmpty;
    z.sys = -1;
    slots[s] = z;
}

// rows[j] = u_n (.) dv_j for j < ncols (right-hand sides before projection, for one orbital).
__global__ void k_pair_rows(const double *__restrict__ psi, const double *__restrict__ dv, int n, long long nd,
                            double *__restrict__ rows) {
    const int j = blockIdx.y;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nd;
         idx += (long long)gridDim.x * blockDim.x)
        rows[(long long)j * nd + idx] = psi[(long long)n * nd + idx] * dv[(long long)j * nd + idx];
}

// (n, j) of the pair systems q = n * ncols + j (chi0 and the adjoint's response).
__global__ void k_pair_index(int *__restrict__ sys_n, int *__restrict__ sys_j, int nsys, int ncols) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nsys) {
        sys_n[q] = q / ncols;
        sys_j[q] = q % ncols;
    }
}

// Add a finished queue's per-system outputs to the device statistics (one block; integer sums).
__global__ void k_queue_stats(const int *__restrict__ sys_out, int nsys, const int *__restrict__ count,
                              QueueStats *__restrict__ qs, long long launches) {
    __shared__ long long red[3][8];
    __shared__ int wred[8];
    long long it = 0, rf = 0, nb = 0;
    int worst = 0;
    for (int i = threadIdx.x; i < nsys; i += blockDim.x) {
        it += sys_out[i];
        worst = max(worst, sys_out[nsys + i]);
        rf += sys_out[2 * nsys + i];
        nb += sys_out[3 * nsys + i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        it += __shfl_down_sync(0xffffffffu, it, o);
        rf += __shfl_down_sync(0xffffffffu, rf, o);
        nb += __shfl_down_sync(0xffffffffu, nb, o);
        worst = max(worst, __shfl_down_sync(0xffffffffu, worst, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = it;
        red[1][w] = rf;
        red[2][w] = nb;
        wred[w] = worst;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            it += red[0][k];
            rf += red[1][k];
            nb += red[2][k];
            worst = max(worst, wred[k]);
        }
        qs->solves += nsys;
        qs->iters += it;
        qs->refines += rf;
        qs->nearb += nb;
        qs->launches += launches;
        qs->worst = max(qs->worst, worst);
        if (*count > 0) qs->unfinished = 1;
    }
}

// End of an epoch of a device-driven queue: continue while systems are busy or waiting and the
// epoch bound is not reached (the bound guarantees that the loop ends).
__global__ void k_continue(cudaGraphConditionalHandle h, const int *__restrict__ count, int *__restrict__ epochs,
                           long long max_epochs, QueueStats *__restrict__ qs, long long per_epoch) {
    const int e = ++(*epochs);
    qs->launches += per_epoch;
    cudaGraphSetConditional(h, (*count > 0 && e < max_epochs) ? 1u : 0u);
}

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------------------------
namespace {

struct SolveSpec {
    const double *vt = nullptr;     // chi0 mode: dV block (ncols x nd); drho accumulated
    double *drho = nullptr;
    const double *rhs = nullptr;    // solve mode: right-hand side per system; x copied out
    double2 *xout = nullptr;
    const double *Tc = nullptr;     // P_c coefficients per system (nullptr = no projection)
    double *grad = nullptr;         // response-square mode: gradient accumulated with coef[j]
    const double *coef = nullptr;   // device, one per column j
    double sign = 1.0;
    double omega = 0.0;
    std::vector<int> n, j;          // systems given on the host, or:
    int pairs = 0;                  // > 0: the pair systems q = n * pairs + j (n < N_s, j < pairs)
    int nsys = 0;
};

// xy tiles of the stencil kernel: at most 64 columns wide and at most max_threads grid columns
// (one thread each) per block.
// With pairs, tiles are an even number of columns wide and a thread takes two of them.
Tiles pick_tiles(int nx, int ny, int max_threads, bool pairs = false) {
    Tiles t;
    t.ntx = (nx + 63) / 64;
    t.tx = (nx + t.ntx - 1) / t.ntx;
    if (pairs) {
        t.tx += t.tx & 1;
        t.ntx = (nx + t.tx - 1) / t.tx;
    }
    const int per_row = pairs ? t.tx / 2 : t.tx;
    const int ty_max = std::max(1, (pairs ? max_threads : max_threads - 31) / per_row);
    const int nty = (ny + ty_max - 1) / ty_max;
    t.ty = (ny + nty - 1) / nty;
    t.nty = (ny + t.ty - 1) / t.ty;
    t.nzc = 1;
    t.zlen = 1 << 30;
    return t;
}

int choose_slots(const Ctx &c, int nsys) {
    if (c.opt.batch_systems > 0) return std::max(1, std::min(nsys, c.opt.batch_systems));
    // All systems of a call in flight when they fit in 8 GB of slot storage; otherwise as many
    // as fit (the queue refills the slots).
    const double slot_bytes = (double)c.nd * (c.opt.prec == RPA_MIXED ? 72.0 : 96.0);
    long long S = std::max(1LL, (long long)(8.0e9 / slot_bytes));
    return (int)std::min<long long>(S, nsys);
}

// Carve aligned pieces out of one allocation.
struct Carver {
    char *base;
    size_t off = 0;
    template <typename T> T *take(size_t count) {
        off = (off + 255) / 256 * 256;
        T *p = (T *)(base + off);
        off += sizeof(T) * count;
        return p;
    }
};

size_t slot_storage_bytes(bool mixed, long long nd, int S, bool precond) {
    const size_t n = (size_t)nd * S;
    return 16 * n + 16 * n + (mixed ? 5 * 8 * n : 4 * 16 * n) + (precond ? 2 * (mixed ? 8 : 16) * n : 0) + 8 * 256;
}

int run_queue(Ctx &c, SolveSpec &sp, cudaStream_t st, std::vector<int> *iters_out, std::vector<int> *status_out) {
    const int nsys = sp.pairs > 0 ? sp.nsys : (int)sp.n.size();
    if (nsys == 0) return RPA_OK;
    const int S = choose_slots(c, nsys);
    const bool mixed = c.opt.prec == RPA_MIXED;
    const long long nd = c.nd;
    const int nblk = (int)cdiv(nd, kChunk);
    const size_t n = (size_t)nd * S;

    // slot storage: x64, b, then the inner vectors x, r, p, q (FP32 complex, or FP64 sharing x64),
    // and with the preconditioner z = M r and the transforms' work vector
    const bool precond = c.opt.precondition != 0;
    Carver cv{(char *)c.cocg_state.ensure(slot_storage_bytes(mixed, nd, S, precond))};
    double2 *x64 = cv.take<double2>(n);
    double2 *b = cv.take<double2>(n);      // right-hand side; the mixed form's FP64 residual r64
    void *xin, *r, *p, *q;           // p: two direction buffers, pstride elements apart
    if (mixed) {
        xin = cv.take<float2>(n);
        r = cv.take<float2>(n);
        p = cv.take<float2>(2 * n);
        q = cv.take<float2>(n);
    } else {
        xin = x64;
        r = cv.take<double2>(n);
        p = cv.take<double2>(2 * n);
        q = cv.take<double2>(n);
    }
    void *zv = nullptr, *wv = nullptr;
    if (precond) {
        zv = mixed ? (void *)cv.take<float2>(n) : (void *)cv.take<double2>(n);
        wv = mixed ? (void *)cv.take<float2>(n) : (void *)cv.take<double2>(n);
    }
    const long long pstride = (long long)n;
    int dev_sms = 0, smem_optin = 0;
    RPA_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c.device));
    RPA_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device));
    // rpa_options.stencil_shape: 0 = automatic (the fused kernel where a plane fits its ring, its
    // cluster form where a band of the plane does, else split variant 1), 1..3 = the split kernels'
    // variants, 4 = the fused kernel (as 0), 5 = its warp-specialised form, 6 = its cluster form
    // with two blocks per SM where the bands fit (else as 0).  The plain FP64 form always runs the
    // split kernels.  Periodic grids: the fused kernel needs even nx (point pairs wrap onto point
    // pairs); the warp-specialised and cluster forms and the two-column split variant are Dirichlet
    // only (the fused kernel or the first split variant stands in for them).
    const int want = std::max(0, std::min(6, c.opt.stencil_shape));
    const bool per = c.opt.periodic != 0;
    const bool even_nx = (c.nx % 2) == 0;
    const bool ws = want == 5 && !per &&
                    ring_fits(c.nx, c.ny, even_nx ? k_cocg_ring_ws<true> : k_cocg_ring_ws<false>, smem_optin, true);
    const RingFn ring1_fn = per ? k_cocg_ring<true, true> : even_nx ? k_cocg_ring<true, false> : k_cocg_ring<false, false>;
    const bool ring1 = (!per || even_nx) && ring_fits(c.nx, c.ny, ring1_fn, smem_optin);
    int ncl = 1, band_pairs = 0;
    const bool clus = mixed && !per && !ws && !precond && (want == 0 || want >= 4) &&
                      ((want == 6 && (cluster_plan(c.nx, c.ny, smem_optin, true, ncl, band_pairs) ||
                                      cluster_plan(c.nx, c.ny, smem_optin, false, ncl, band_pairs))) ||
                       (!ring1 && cluster_plan(c.nx, c.ny, smem_optin, false, ncl, band_pairs)));
    const RingFn ring_fn = ws ? (even_nx ? k_cocg_ring_ws<true> : k_cocg_ring_ws<false>)
                              : clus ? (even_nx ? k_cocg_ring_cl<true> : k_cocg_ring_cl<false>) : ring1_fn;
    const bool use_ring = mixed && !precond && (want == 0 || want >= 4) && (ws || clus || ring1);
    const int variant = (want >= 1 && want <= 3 && !(per && want == 3)) ? want - 1 : 0;
    const PaShape shape = mixed ? kPaShapes32[variant] : kPaShape64;
    Tiles tl = pick_tiles(c.nx, c.ny, shape.max_threads, shape.pairs != 0);
    if (c.opt.z_chunks > 1) {
        tl.zlen = (c.nz + c.opt.z_chunks - 1) / c.opt.z_chunks;
        tl.nzc = (c.nz + tl.zlen - 1) / tl.zlen;
    } else {
        tl.zlen = c.nz;
    }
    const int ntiles = tl.ntx * tl.nty * tl.nzc;
    double *partA =
        (double *)c.cocg_partials.ensure(sizeof(double) * (size_t)S * (2 * ntiles + 3 * nblk + 3 * c.nz));
    double *partB = partA + (size_t)S * ntiles * 2;
    double *partZ = partB + (size_t)S * nblk * 3;
    Slot *slots = (Slot *)c.sys_state.ensure(sizeof(Slot) * S);
    // ints: head, count, cnt[4], list[4][S], then per system: n, j, iters, status, refines,
    // near-breakdowns; then the finished-slot count and list [S].  The split kernels use lists 0
    // and 1 (by iteration parity); the fused kernel list 0, with counter 1 as its work counter.
    const size_t nint = 6 + 4 * (size_t)S + 6 * (size_t)nsys + 1 + (size_t)S;
    int *qi = (int *)c.slot_idx.ensure(sizeof(int) * nint);
    int *head = qi, *count = qi + 1, *cnt = qi + 2, *list = qi + 6;
    int *sys_n = list + 4 * S, *sys_j = sys_n + nsys, *sys_out = sys_j + nsys;
    int *fin_cnt = sys_out + 4 * (size_t)nsys, *fin_list = fin_cnt + 1;
    RPA_CUDA(cudaMemsetAsync(qi, 0, sizeof(int) * nint, st));
    if (sp.pairs > 0) {                 // generated on the device: no host copy, no synchronisation
        k_pair_index<<<cdiv(nsys, 256), 256, 0, st>>>(sys_n, sys_j, nsys, sp.pairs);
        RPA_LAUNCH("pair index");
    } else {
        RPA_CUDA(cudaMemcpyAsync(sys_n, sp.n.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
        RPA_CUDA(cudaMemcpyAsync(sys_j, sp.j.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
    }
    k_init_slots<<<cdiv(S, 128), 128, 0, st>>>(slots, S);
    RPA_LAUNCH("init slots");

    Params P{};
    P.slots = slots;
    P.S = S;
    P.nblk = nblk;
    P.nparta = ntiles;
    P.g = Grid3{c.nx, c.ny, c.nz, nd, c.opt.periodic};
    P.partA = partA;
    P.partB = partB;
    P.list = list;
    P.cnt = cnt;
    P.mixed = mixed;
    P.tol = c.opt.tol;
    P.inner_tol = c.opt.inner_tol;
    P.maxit = c.opt.maxit;
    P.max_refine = c.opt.max_refine;
    P.head = head;
    P.nsys = nsys;
    P.count = count;
    P.sys_out = sys_out;
    P.fin_list = fin_list;
    P.fin_cnt = fin_cnt;
    // mixed form with P_c applied to the right-hand sides: the refinement works in the
    // unoccupied space.  The FP32 projections leave occupied components of ~1e-9 of the
    // solution's norm; below that tolerance the finished solution is also projected in FP64.
    P.precond = precond ? 1 : 0;
    P.partZ = partZ;
    P.cproject = mixed && sp.Tc != nullptr;
    P.project = c.opt.project_solution != 0 || sp.grad != nullptr || (P.cproject && c.opt.tol < 1e-9);
    P.proj_re_only = sp.drho != nullptr && sp.grad == nullptr;
    P.ns = c.ns;
    P.psi = c.psi64;
    P.psi32 = c.psi32;
    if (P.project || P.cproject) {
        // Tp, partP, then Tp32
        double *pp = (double *)c.proj_buf.ensure(sizeof(double) * 2 * (size_t)S * c.ns * (nblk + 2));
        P.Tp = pp;
        P.partP = pp + (size_t)S * c.ns * 2;
        P.Tp32 = (float *)(P.partP + (size_t)S * c.ns * 2 * nblk);
    }

    // per parity: the stencil kernel's and the update kernel's views of P
    IterArgs ia_pa[2], ia_b[2];
    for (int par = 0; par < 2; ++par) {
        const IterArgs base{slots, list + par * S, cnt + par, nullptr, nullptr, nd, c.nx, c.ny, c.nz, 0,
                            c.opt.periodic};
        ia_pa[par] = base;
        ia_pa[par].part = partA;
        ia_pa[par].nper = ntiles;
        ia_b[par] = base;
        ia_b[par].part = partB;
        ia_b[par].nper = nblk;
    }

    const long long items = (long long)S * nblk;
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(items, (long long)dev_sms * 8));
    const unsigned wgrid = cdiv(S, kWarpsPerBlock);      // one warp per slot
    const int per_row = shape.pairs ? tl.tx / 2 : tl.tx;
    const int pa_threads = (per_row * tl.ty + 31) / 32 * 32;
    // halo elements (pairs of elements for the two-column kernel) per plane
    const int pa_halo = shape.pairs ? (tl.ntx > 1 ? kRadius * (tl.tx + tl.ty) : kRadius * tl.tx)
                                    : (tl.ntx > 1 ? 2 * kRadius * (tl.tx + tl.ty) : 2 * kRadius * tl.tx);
    const bool pa_h1 = pa_halo <= pa_threads;
    using Pa32 = void (*)(IterArgs, Tiles, const float2 *, float2 *, long long, float2 *, const float *, Coef<float>);
    static const Pa32 pa32_table[3][2] = {
        {k_cocg_pa<float, 1, 640, 1>, k_cocg_pa<float, 2, 640, 1>},
        {k_cocg_pa<float, 1, 320, 2>, k_cocg_pa<float, 2, 320, 2>},
        {k_cocg_pa2<1, 384>, k_cocg_pa2<2, 384>}};
    const Pa32 pa32 = pa32_table[variant][pa_h1 ? 0 : 1];
    auto pa64 = pa_h1 ? k_cocg_pa<double, 1, 448, 1> : k_cocg_pa<double, 2, 448, 1>;
    const size_t pa_smem = 2 * (size_t)(tl.tx + 2 * kRadius) * (tl.ty + 2 * kRadius) * (mixed ? 8 : 16);
    if (mixed) allow_dynamic_smem((const void *)pa32, pa_smem);
    else allow_dynamic_smem((const void *)pa64, pa_smem);
    int pa_per_sm = 1;
    if (mixed)
        RPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pa_per_sm, pa32, pa_threads, pa_smem));
    else
        RPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pa_per_sm, pa64, pa_threads, pa_smem));
    const unsigned pa_grid = (unsigned)std::max<long long>(
        1, std::min<long long>((long long)S * ntiles, (long long)dev_sms * std::max(1, pa_per_sm)));
    const Coef<float> cf32 = cast_coef<float>(c.coef);
    const Coef<double> cf64 = cast_coef<double>(c.coef);
    Coef<float> cf_hi, cf_lo;              // the coefficients as FP32 pairs (double-float residual)
    for (int k = 0; k <= kRadius; ++k) {
        cf_hi.a[k] = (float)c.coef.a[k];
        cf_lo.a[k] = (float)(c.coef.a[k] - (double)cf_hi.a[k]);
    }
    const double scale = 4.0 / (c.h * c.h * c.h);

    // the fused kernel: one block per system at a time, each run through its inner solve
    RingArgs ra{};
    unsigned ring_grid = 1, ring_threads = 32;
    size_t ring_smem = 0;
    if (use_ring) {
        const int hw = (c.nx + 1) / 2;
        ra.slots = slots;
        ra.list_in = list;             // built by k_ring_list, which also clears the counter
        ra.cnt_in = cnt;
        ra.grab = cnt + 1;
        ra.nd = nd;
        ra.tol = c.opt.tol;
        ra.inner_tol = c.opt.inner_tol;
        ra.maxit = c.opt.maxit;
        ra.nx = c.nx;
        ra.ny = c.ny;
        ra.nz = c.nz;
        ra.hw = hw;
        ra.hh = (c.ny + 1) / 2;
        ra.rs = 2 * hw + ring_row_pad(hw);
        ra.ps = clus ? 2 + 2 * band_pairs * ra.rs : 2 + c.ny * ra.rs;
        ra.bp = band_pairs;
        ring_smem = (size_t)kRingPlanes * ra.ps * sizeof(float2);
        if (clus) ring_smem += 2 * (2 + (size_t)2 * kRadius * ra.rs) * sizeof(float2);   // the halo buffers
        {
            const int units = hw * (clus ? band_pairs : (c.ny + 1) / 2);
            ring_threads = (unsigned)((units + 31) / 32 * 32);
            if (ws) ring_threads += (unsigned)(((units + 1) / 2 + 31) / 32 * 32);   // consumers + producers
        }
        allow_dynamic_smem((const void *)ring_fn, ring_smem);
        if (clus) {
            // one cluster of ncl blocks per system at a time, as many clusters as are resident
            cudaLaunchConfig_t lc{};
            cudaLaunchAttribute at{};
            at.id = cudaLaunchAttributeClusterDimension;
            at.val.clusterDim.x = (unsigned)ncl;
            at.val.clusterDim.y = 1;
            at.val.clusterDim.z = 1;
            lc.gridDim = dim3((unsigned)ncl * (unsigned)dev_sms, 1, 1);
            lc.blockDim = dim3(ring_threads, 1, 1);
            lc.dynamicSmemBytes = ring_smem;
            lc.attrs = &at;
            lc.numAttrs = 1;
            int nclusters = 0;
            RPA_CUDA(cudaOccupancyMaxActiveClusters(&nclusters, (const void *)ring_fn, &lc));
            if (nclusters < 1) fail(RPA_ERR_CUDA, "cluster form of the fused kernel: no cluster of %d blocks fits", ncl);
            ring_grid = (unsigned)ncl * (unsigned)std::min<long long>(S, nclusters);
        } else {
            int per_sm = 1;
            RPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ring_fn, (int)ring_threads, ring_smem));
            ring_grid = (unsigned)std::max<long long>(1, std::min<long long>(S, (long long)dev_sms * std::max(1, per_sm)));
        }
    }

    // the Laplacian preconditioner: z = M r in three passes (see k_pc_xy, k_pc_z)
    PcArgs<float> pc32{};
    PcArgs<double> pc64{};
    size_t pcxy_smem = 0, pcz_smem = 0;
    unsigned pcxy_grid = 1, pcz_grid = 1;
    if (precond) {
        auto fill = [&](auto &a, auto Qs, auto mus) {
            a.slots = slots;
            a.S = S;
            a.nx = c.nx;
            a.ny = c.ny;
            a.nz = c.nz;
            a.nd = nd;
            a.Qx = Qs[0];
            a.Qy = Qs[1];
            a.Qz = Qs[2];
            a.mux = mus[0];
            a.muy = mus[1];
            a.muz = mus[2];
            a.vbar = c.vbar;
            a.partZ = partZ;
        };
        const size_t tsz = mixed ? sizeof(float) : sizeof(double);
        pcxy_smem = mixed ? pc_xy_bytes<float>(c.nx, c.ny) : pc_xy_bytes<double>(c.nx, c.ny);
        pcz_smem = pc_mat_bytes((size_t)c.nz * c.nz, tsz) + 2 * tsz * (size_t)c.nz * 33;
        if (pcxy_smem > (size_t)smem_optin || pcz_smem > (size_t)smem_optin || c.nz > 8 * 12 ||
            (long long)((c.nx + 3) / 4) * ((c.ny + 1) / 2) > (long long)kPcTiles * kPcThreads)
            fail(RPA_ERR_INVALID, "precondition: a %d x %d plane or %d planes exceed the preconditioner's limits",
                 c.nx, c.ny, c.nz);
        if (mixed) {
            fill(pc32, c.Qf, c.muf);
            allow_dynamic_smem((const void *)k_pc_xy<float, true>, pcxy_smem);
            allow_dynamic_smem((const void *)k_pc_xy<float, false>, pcxy_smem);
            allow_dynamic_smem((const void *)k_pc_z<float>, pcz_smem);
        } else {
            const double *Qd[3] = {c.Q[0], c.Q[1], c.Q[2]};
            const double *md[3] = {c.mu[0], c.mu[1], c.mu[2]};
            fill(pc64, Qd, md);
            allow_dynamic_smem((const void *)k_pc_xy<double, true>, pcxy_smem);
            allow_dynamic_smem((const void *)k_pc_xy<double, false>, pcxy_smem);
            allow_dynamic_smem((const void *)k_pc_z<double>, pcz_smem);
        }
        const int per_sm_xy = std::max<int>(1, (int)(smem_optin / std::max<size_t>(pcxy_smem, 1)));
        pcxy_grid = (unsigned)std::max<long long>(
            1, std::min<long long>((long long)S * c.nz, (long long)dev_sms * std::min(per_sm_xy, 4)));
        pcz_grid = (unsigned)std::max<long long>(
            1, std::min<long long>((long long)S * cdiv((long long)c.nx * c.ny, 32), (long long)dev_sms * 4));
    }
    auto precondition = [&](cudaStream_t ss) {   // z = M r for the slots in their inner solve
        if (mixed) {
            k_pc_xy<float, true><<<pcxy_grid, kPcThreads, pcxy_smem, ss>>>(pc32, (const float2 *)r, (float2 *)wv,
                                                                           nullptr);
            k_pc_z<float><<<pcz_grid, kPcThreads, pcz_smem, ss>>>(pc32, (float2 *)wv);
            k_pc_xy<float, false><<<pcxy_grid, kPcThreads, pcxy_smem, ss>>>(pc32, (const float2 *)wv, (float2 *)zv,
                                                                            (const float2 *)r);
        } else {
            k_pc_xy<double, true><<<pcxy_grid, kPcThreads, pcxy_smem, ss>>>(pc64, (const double2 *)r,
                                                                            (double2 *)wv, nullptr);
            k_pc_z<double><<<pcz_grid, kPcThreads, pcz_smem, ss>>>(pc64, (double2 *)wv);
            k_pc_xy<double, false><<<pcxy_grid, kPcThreads, pcxy_smem, ss>>>(pc64, (const double2 *)wv,
                                                                             (double2 *)zv, (const double2 *)r);
        }
    };

    // profiling: events around every launch of the item kernels of the iteration
    const bool prof = c.opt.profile != 0;
    const char *tn = mixed ? "c64" : "c128";
    char names[3][32];
    std::snprintf(names[0], 32, "-");
    if (use_ring) {
        std::snprintf(names[1], 32, ws ? "k_cocg_ring_ws<%s>" : clus ? "k_cocg_ring_cl<%s>" : "k_cocg_ring<%s>", tn);
        std::snprintf(names[2], 32, "-");
    } else {
        std::snprintf(names[1], 32, "k_cocg_pa<%s>", tn);
        std::snprintf(names[2], 32, "k_cocg_b<%s>", tn);
    }
    const double csz = mixed ? 8.0 : 16.0, rsz = mixed ? 4.0 : 8.0;
    // algorithmic bytes per grid point: pa reads r, p_old, V and writes p_new, q; b reads x, r, p, q
    // and writes x, r; the fused kernel reads and writes x, r, p, q, except in the first sweep of an
    // inner solve, which reads r and writes p, q (V is read once per plane and block, not per system,
    // and is not counted)
    const double bytes_per_point[3] = {0.0, use_ring ? 8 * csz : 4 * csz + rsz, use_ring ? 0.0 : 6 * csz};
    if (prof) {
        RPA_CUDA(cudaMemsetAsync(c.d_prof_points, 0, sizeof(unsigned long long) * 3, st));
        P.prof = c.d_prof_points;
        for (int par = 0; par < 2; ++par) ia_pa[par].prof = ia_b[par].prof = c.d_prof_points;
        ra.prof = c.d_prof_points;
    }
    // Two graph instances of one epoch (alternating, so that the events of one can be read while
    // the other runs); without graphs the same launches go straight to the stream.
    const bool use_graph = c.use_graphs;
    constexpr int kTimed = 2 * kEpoch;
    std::vector<cudaEvent_t> evs;      // [2][kTimed][2]
    if (prof) {
        evs.resize(2 * kTimed * 2);
        for (auto &e : evs) {
            RPA_CUDA(cudaEventCreate(&e));
        }
    }
    long long launches = 0;
    double prof_ms[3] = {0, 0, 0};
    long long prof_n[3] = {0, 0, 0};

    auto maintenance = [&](cudaStream_t ss) {
        if (mixed) {
            if (P.cproject) {
                k_cproj_dots<<<grid, kThreads, 0, ss>>>(P, (const float2 *)xin);
                k_proj_sum<<<wgrid, kThreads, 0, ss>>>(P, kInnerDone);
            }
            k_refine_x<<<grid, kThreads, 0, ss>>>(P, x64, (float2 *)xin, (float2 *)q);
            k_residual_df<<<grid, kThreads, 0, ss>>>(P, b, (const float2 *)q, (float2 *)r, (float2 *)p, c.vloc32,
                                                     c.vloc_lo, cf_hi, cf_lo, 3.0 * c.coef.a[0]);   // p = direction buffer 0
            if (P.cproject) {
                k_cproj_dots<<<grid, kThreads, 0, ss>>>(P, (const float2 *)r);
                k_proj_sum<<<wgrid, kThreads, 0, ss>>>(P, kInnerDone);
                k_cproj_residual<<<grid, kThreads, 0, ss>>>(P, (float2 *)r);
            }
            k_state<<<wgrid, kThreads, 0, ss>>>(P);
        }
        k_finished_list<<<1, 1024, 0, ss>>>(P);
        if (P.project) {
            k_proj_dots<<<grid, kThreads, 0, ss>>>(P, x64);
            k_proj_sum<<<wgrid, kThreads, 0, ss>>>(P, kFinished);
        }
        if (sp.grad)
            k_retire_grad<<<std::min<unsigned>(cdiv(nd, 256), 2048u), 256, 0, ss>>>(P, x64, sp.coef, sp.grad, scale);
        else if (sp.drho)
            k_retire_drho<<<std::min<unsigned>(cdiv(nd, 256), 2048u), 256, 0, ss>>>(P, x64, c.psi64, sp.drho, scale);
        else
            k_retire_copy<<<grid, kThreads, 0, ss>>>(P, x64, sp.xout);
        k_refill<<<1, 1024, 0, ss>>>(P, sys_n, sys_j, c.eps_dev, sp.omega);
        if (mixed)
            k_load<float><<<grid, kThreads, 0, ss>>>(P, c.psi64, c.ns, sp.vt, sp.rhs, sp.Tc, sp.sign, b, x64,
                                                     (float2 *)xin, (float2 *)r, (float2 *)p, pstride);
        else
            k_load<double><<<grid, kThreads, 0, ss>>>(P, c.psi64, c.ns, sp.vt, sp.rhs, sp.Tc, sp.sign, b, x64,
                                                      (double2 *)xin, (double2 *)r, (double2 *)p, pstride);
        k_state<<<wgrid, kThreads, 0, ss>>>(P);
        RPA_LAUNCH("cocg maintenance");
    };
    auto epoch = [&](cudaStream_t ss, int evset) {
        const bool capturing = use_graph && ss == c.cap_stream;
        auto rec = [&](int slot) {
            if (!prof) return;
            cudaEvent_t e = evs[(size_t)evset * kTimed * 2 + slot];
            if (capturing) RPA_CUDA(cudaEventRecordWithFlags(e, ss, cudaEventRecordExternal));
            else RPA_CUDA(cudaEventRecord(e, ss));
        };
        if (use_ring) {
            k_ring_list<<<1, 1024, 0, ss>>>(P);
            rec(0);
            if (clus) {
                cudaLaunchConfig_t lc{};
                cudaLaunchAttribute at{};
                at.id = cudaLaunchAttributeClusterDimension;
                at.val.clusterDim.x = (unsigned)ncl;
                at.val.clusterDim.y = 1;
                at.val.clusterDim.z = 1;
                lc.gridDim = dim3(ring_grid, 1, 1);
                lc.blockDim = dim3(ring_threads, 1, 1);
                lc.dynamicSmemBytes = ring_smem;
                lc.stream = ss;
                lc.attrs = &at;
                lc.numAttrs = 1;
                RPA_CUDA(cudaLaunchKernelEx(&lc, ring_fn, ra, (float2 *)xin, (float2 *)r, (float2 *)p, (float2 *)q,
                                            (const float *)c.vloc32, cf32));
            } else {
                ring_fn<<<ring_grid, ring_threads, ring_smem, ss>>>(ra, (float2 *)xin, (float2 *)r, (float2 *)p,
                                                                    (float2 *)q, c.vloc32, cf32);
            }
            rec(1);
            RPA_LAUNCH("cocg inner solves (fused)");
            maintenance(ss);
            return;
        }
        for (int e = 0; e < kEpoch; ++e) {
            const int par = e & 1;
            const int t0 = 2 * e * 2;
            if (precond) precondition(ss);
            k_beta<<<wgrid, kThreads, 0, ss>>>(P, par);
            // the direction update takes z = M r in place of r when preconditioned
            if (mixed) {
                rec(t0 + 0);
                pa32<<<pa_grid, pa_threads, pa_smem, ss>>>(ia_pa[par], tl, (const float2 *)(precond ? zv : r), (float2 *)p,
                                                                      pstride, (float2 *)q, c.vloc32, cf32);
                rec(t0 + 1);
                k_alpha<<<wgrid, kThreads, 0, ss>>>(P, par);
                rec(t0 + 2);
                k_cocg_b<float><<<grid, kThreads, 0, ss>>>(ia_b[par], (float2 *)xin, (float2 *)r, (const float2 *)p,
                                                           pstride, (const float2 *)q);
                rec(t0 + 3);
            } else {
                rec(t0 + 0);
                pa64<<<pa_grid, pa_threads, pa_smem, ss>>>(ia_pa[par], tl, (const double2 *)(precond ? zv : r), (double2 *)p,
                                                                        pstride, (double2 *)q, c.vloc64, cf64);
                rec(t0 + 1);
                k_alpha<<<wgrid, kThreads, 0, ss>>>(P, par);
                rec(t0 + 2);
                k_cocg_b<double><<<grid, kThreads, 0, ss>>>(ia_b[par], (double2 *)xin, (double2 *)r, (const double2 *)p,
                                                            pstride, (const double2 *)q);
                rec(t0 + 3);
            }
        }
        RPA_LAUNCH("cocg iterations");
        maintenance(ss);
    };
    const int per_maint = (mixed ? 8 : 5) + (P.project ? 2 : 0) + (P.cproject ? 5 : 0);
    const int per_epoch = (use_ring ? 2 : (precond ? 7 : 4) * kEpoch) + per_maint;

    // device-driven queue: CUDA graphs, no profiling, no per-system outputs wanted
    const bool device_loop = use_graph && !prof && !iters_out && !status_out;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    if (use_graph && !device_loop) {
        for (int g = 0; g < (prof ? 2 : 1); ++g) {
            cudaGraph_t graph;
            RPA_CUDA(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
            epoch(c.cap_stream, g);
            RPA_CUDA(cudaStreamEndCapture(c.cap_stream, &graph));
            RPA_CUDA(cudaGraphInstantiate(&gexec[g], graph, 0));
            cudaGraphDestroy(graph);
        }
        if (!prof) gexec[1] = gexec[0];
    }
    auto run_epoch = [&](long long k) {
        if (use_graph) RPA_CUDA(cudaGraphLaunch(gexec[k & 1], st));
        else epoch(st, (int)(k & 1));
        launches += per_epoch;
    };
    auto collect_epoch = [&](long long k) {
        if (!prof) return;
        const int set = (int)(k & 1);
        for (int t = 0; t < (use_ring ? 1 : kTimed); ++t) {   // the fused kernel: one timed launch
            float ms = 0.f;
            RPA_CUDA(cudaEventElapsedTime(&ms, evs[((size_t)set * kTimed + t) * 2], evs[((size_t)set * kTimed + t) * 2 + 1]));
            prof_ms[1 + t % 2] += ms;
            prof_n[1 + t % 2] += 1;
        }
    };

    maintenance(st);   // first fill of the slots
    launches += per_maint;
    const long long per_sys = (long long)c.opt.maxit * (mixed ? c.opt.max_refine : 1) / kEpoch + 3;
    const long long max_epochs = ((long long)nsys + S - 1) / S * per_sys + 4;

    // Device-driven queue (CUDA graphs, no profiling, no per-system outputs wanted): one graph whose
    // conditional while node replays the epoch until no system is busy or waiting, so the host never
    // waits on the queue; its statistics accumulate on the device for the caller's next read-back.
    if (device_loop) {
        cudaGraph_t parent = nullptr, body_end = nullptr;
        cudaGraphExec_t loop = nullptr;
        RPA_CUDA(cudaGraphCreate(&parent, 0));
        try {
            cudaGraphConditionalHandle h;
            RPA_CUDA(cudaGraphConditionalHandleCreate(&h, parent, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams np{};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t cnode;
            RPA_CUDA(cudaGraphAddNode(&cnode, parent, nullptr, nullptr, 0, &np));
            cudaGraph_t body = np.conditional.phGraph_out[0];
            RPA_CUDA(cudaStreamBeginCaptureToGraph(c.cap_stream, body, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeThreadLocal));
            epoch(c.cap_stream, 0);
            k_continue<<<1, 1, 0, c.cap_stream>>>(h, count, c.d_loop, max_epochs, c.d_qstats, per_epoch + 1);
            RPA_LAUNCH("queue loop condition");
            RPA_CUDA(cudaStreamEndCapture(c.cap_stream, &body_end));
            RPA_CUDA(cudaGraphInstantiate(&loop, parent, 0));
        } catch (...) {
            cudaGraph_t dummy;
            if (cudaStreamEndCapture(c.cap_stream, &dummy) == cudaSuccess && dummy) cudaGraphDestroy(dummy);
            (void)cudaGetLastError();
            cudaGraphDestroy(parent);
            throw;
        }
        RPA_CUDA(cudaMemsetAsync(c.d_loop, 0, sizeof(int), st));
        RPA_CUDA(cudaGraphLaunch(loop, st));
        k_queue_stats<<<1, 256, 0, st>>>(sys_out, nsys, count, c.d_qstats, launches + 3);
        RPA_LAUNCH("queue statistics");
        cudaGraphExecDestroy(loop);     // freed once the launch completes
        cudaGraphDestroy(parent);
        for (auto &e : evs) cudaEventDestroy(e);
        count_launches(2);
        return RPA_OK;                  // per-system statuses arrive with the statistics
    }

    // Epochs are enqueued up to two ahead of the host's check of the busy count.
    constexpr int kRing = 4;
    int *hc = c.h_count;
    cudaEvent_t ev[kRing];
    for (auto &e : ev) RPA_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    long long issued = 0, checked = 0;
    bool done = false;
    while (!done) {
        while (issued - checked < 2 && issued < max_epochs) {
            run_epoch(issued);
            RPA_CUDA(cudaMemcpyAsync(hc + (issued % kRing), count, sizeof(int), cudaMemcpyDeviceToHost, st));
            RPA_CUDA(cudaEventRecord(ev[issued % kRing], st));
            ++issued;
        }
        if (checked >= issued) break;
        RPA_CUDA(cudaEventSynchronize(ev[checked % kRing]));
        c.host_syncs += 1;
        collect_epoch(checked);
        if (hc[checked % kRing] == 0) done = true;
        ++checked;
    }
    sync_stream(c, st);
    while (checked < issued) collect_epoch(checked++);
    for (auto &e : ev) cudaEventDestroy(e);
    for (int g = 0; g < 2; ++g)
        if (gexec[g] && (g == 0 || gexec[1] != gexec[0])) cudaGraphExecDestroy(gexec[g]);
    for (auto &e : evs) cudaEventDestroy(e);
    count_launches(launches + 1);
    if (prof) {
        unsigned long long pts[3];
        RPA_CUDA(cudaMemcpy(pts, c.d_prof_points, sizeof pts, cudaMemcpyDeviceToHost));
        for (int k = 1; k < (use_ring ? 2 : 3); ++k) {
            const int sl = prof_slot(c, names[k]);
            c.stats.prof_ms[sl] += prof_ms[k];
            c.stats.prof_launches[sl] += prof_n[k];
            c.stats.prof_points[sl] += (double)pts[k];
            c.stats.prof_bytes[sl] += (double)pts[k] * bytes_per_point[k];
            if (use_ring) c.stats.prof_bytes[sl] -= (double)pts[2] * 5 * csz;   // first sweeps: 3 streams
        }
    }

    std::vector<int> h(4 * (size_t)nsys);
    RPA_CUDA(cudaMemcpy(h.data(), sys_out, sizeof(int) * 4 * nsys, cudaMemcpyDeviceToHost));
    int worst = 0;
    for (int i = 0; i < nsys; ++i) {
        const int it = h[i], stt = h[nsys + i], rf = h[2 * nsys + i];
        c.stats.near_breakdowns += h[3 * (size_t)nsys + i];
        worst = std::max(worst, stt);
        c.stats.sternheimer_solves += 1;
        c.stats.cocg_iterations += it;
        c.stats.refinement_steps += rf;
        c.stats.stencil_points += (long long)(it + rf) * nd;
        c.stats.worst_status = std::max(c.stats.worst_status, stt);
        if (iters_out) (*iters_out)[i] = it;
        if (status_out) (*status_out)[i] = stt;
    }
    if (!done) {
        worst = std::max(worst, (int)RPA_ERR_NOT_CONVERGED);
        c.stats.worst_status = std::max(c.stats.worst_status, (int)RPA_ERR_NOT_CONVERGED);
    }
    return worst;
}

// T[s][k] = u_k . rows[s] for nrows rows.
void pc_coefficients(Ctx &c, const double *rows, int nrows, double *T, cudaStream_t st) {
    if (use_tensor_cores(c))
        tc_gemm(rows, c.nd, 1, c.psi64, c.nd, 1, nrows, c.ns, c.nd, T, st, c.dense_scratch, c.d_tc_err);
    else
        gram(rows, nrows, c.psi64, c.ns, c.nd, T, st, c.dense_scratch);
}

void check_orbitals(const Ctx &c, const int *orb, int nsys) {
    for (int i = 0; i < nsys; ++i)
        if (orb[i] < 0 || orb[i] >= c.ns) fail(RPA_ERR_INVALID, "orbital index %d out of range", orb[i]);
}

}  // namespace

bool fused_kernel_applies(const Ctx &c, bool warp_specialised, bool cluster) {
    if (c.opt.precondition) return false;   // the preconditioned COCG runs the split kernels
    int smem_optin = 0;
    RPA_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device));
    const bool even = (c.nx % 2) == 0;
    if (cluster) {
        int ncl = 0, bp = 0;
        return !c.opt.periodic && cluster_plan(c.nx, c.ny, smem_optin, true, ncl, bp);
    }
    if (c.opt.periodic)
        return !warp_specialised && even && ring_fits(c.nx, c.ny, k_cocg_ring<true, true>, smem_optin);
    if (warp_specialised)
        return ring_fits(c.nx, c.ny, even ? k_cocg_ring_ws<true> : k_cocg_ring_ws<false>, smem_optin, true);
    return ring_fits(c.nx, c.ny, even ? k_cocg_ring<true, false> : k_cocg_ring<false, false>, smem_optin);
}

int sternheimer_batch(Ctx &c, double omega, const int *orb, int nsys, const double *b, double *x,
                      std::vector<int> *iters, std::vector<int> *status, cudaStream_t s) {
    check_orbitals(c, orb, nsys);
    if (c.opt.block_cocg > 0) return sternheimer_block(c, omega, orb, nsys, b, nullptr, x, iters, status, s);
    SolveSpec sp;
    sp.rhs = b;
    sp.xout = (double2 *)x;
    sp.omega = omega;
    sp.n.assign(orb, orb + nsys);
    sp.j.resize(nsys);
    for (int i = 0; i < nsys; ++i) sp.j[i] = i;
    return run_queue(c, sp, s, iters, status);
}

int sternheimer_batch_projected(Ctx &c, double omega, const int *orb, int nsys, const double *b, double *x,
                                std::vector<int> *iters, std::vector<int> *status, cudaStream_t s) {
    check_orbitals(c, orb, nsys);
    double *T = (double *)c.pc_coef.ensure(sizeof(double) * (size_t)nsys * c.ns);
    if (c.opt.block_cocg > 0) {
        // FP64 coefficients: the block iteration does not project its residuals again
        gram(b, nsys, c.psi64, c.ns, c.nd, T, s, c.dense_scratch);
        return sternheimer_block(c, omega, orb, nsys, b, T, x, iters, status, s);
    }
    pc_coefficients(c, b, nsys, T, s);
    SolveSpec sp;
    sp.rhs = b;
    sp.xout = (double2 *)x;
    sp.Tc = T;
    sp.omega = omega;
    sp.n.assign(orb, orb + nsys);
    sp.j.resize(nsys);
    for (int i = 0; i < nsys; ++i) sp.j[i] = i;
    return run_queue(c, sp, s, iters, status);
}

// P_c coefficients of the pair right-hand sides u_n (.) dv_j for all (n, j), system n*ncols + j.
static double *pair_coefficients(Ctx &c, const double *dv, int ncols, cudaStream_t s) {
    const int nsys = c.ns * ncols;
    double *T = (double *)c.pc_coef.ensure(sizeof(double) * (size_t)nsys * c.ns);
    double *rows = (double *)c.rhs.ensure(sizeof(double) * (size_t)ncols * c.nd);
    for (int n = 0; n < c.ns; ++n) {
        k_pair_rows<<<dim3(std::min<unsigned>(cdiv(c.nd, 256), 1024u), ncols), 256, 0, s>>>(c.psi64, dv, n, c.nd,
                                                                                             rows);
        RPA_LAUNCH("pair rows");
        count_launches(1);
        pc_coefficients(c, rows, ncols, T + (size_t)n * ncols * c.ns, s);
    }
    return T;
}

int response_square(Ctx &c, double omega, const double *dv, const double *coef, double *grad, int ncols,
                    cudaStream_t s) {
    const int nsys = c.ns * ncols;
    SolveSpec sp;
    sp.vt = dv;
    sp.grad = grad;
    sp.coef = coef;
    sp.Tc = pair_coefficients(c, dv, ncols, s);
    sp.sign = -1.0;
    sp.omega = omega;
    sp.pairs = ncols;
    sp.nsys = nsys;
    return run_queue(c, sp, s, nullptr, nullptr);
}

int chi0_apply(Ctx &c, double omega, const double *dv, double *drho, int ncols, cudaStream_t s) {
    if (c.coord) return batch_chi0(c, omega, dv, drho, ncols, s);
    if (c.opt.block_cocg > 0) return chi0_apply_block(c, omega, dv, drho, ncols, s);
    RPA_CUDA(cudaMemsetAsync(drho, 0, sizeof(double) * (size_t)ncols * c.nd, s));
    const int nsys = c.ns * ncols;
    SolveSpec sp;
    sp.vt = dv;
    sp.drho = drho;
    sp.Tc = pair_coefficients(c, dv, ncols, s);   // T[(n, j)][k] = u_k . (u_n (.) dv_j)
    sp.sign = -1.0;
    sp.omega = omega;
    sp.pairs = ncols;
    sp.nsys = nsys;
    return run_queue(c, sp, s, nullptr, nullptr);
}

}  // namespace rpa

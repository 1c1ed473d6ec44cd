// Block COCG for the Sternheimer systems that share an orbital: the block variant of COCG that the
// paper names beside Laplacian preconditioning as its preliminary alternative (arXiv 2504.01816,
// Section "Implementation").  The systems (H - eps_n + i omega) x = b of Eq. 9 for the columns of
// one orbital n share their operator, so s of them (a group) are solved together.
//
// Block conjugate gradients with the unconjugated bilinear form x^T y (as COCG is to CG), with the
// group's right-hand sides as the columns of B:
//   X = 0, R = B, P = R, rho = R^T R                                    (s x s)
//   repeat: Q = A P, alpha = (P^T Q)^-1 rho, X += P alpha, R -= Q alpha,
//           rho' = R^T R, beta = rho^-1 rho', P = R + P beta, rho = rho'
// until every column meets its stopping threshold.
//
// The inner solves sit in the same FP64 iterative refinement as the single-system queue: r64 =
// b - A x64 in FP64, block COCG for A D = r64 (complex FP32 for the mixed form, FP64 for the plain
// form) on the columns not yet converged, each scaled to unit norm, x64 += D, repeat until every
// column has ||r64|| <= tol ||b||.  Where alpha or beta needs an s x s matrix that is singular to
// working precision (the block form of COCG's breakdown: the residuals of the block have become
// nearly dependent, as they do once the FP32 solves reach their rounding floor and every column's
// residual is dominated by the same few directions) the inner solve ends, and the refinement
// restarts it from the true residual with at most half as many columns, those with the largest
// relative residuals; a group can so shrink to single-column COCG.  Converged columns are left out
// of every inner solve, and max_refine bounds the inner solves each column takes part in.
//
// One inner iteration is seven launches over the groups whose inner solve runs: the stencil, a
// Gram kernel (P^T Q), a per-group kernel (alpha by Gaussian elimination with partial pivoting on
// the equilibrated s x s system), the X/R update, a Gram kernel (R^T R and the column norms), a
// per-group kernel (stopping test, beta) and the direction update.  Every 8 iterations a
// maintenance pass refines, tests and restarts the groups whose inner solve ended.  The Gram
// partial sums are written per block and added in block order, so results do not depend on
// scheduling.
//
// The kernels read each group's grid, operator and orbitals from a table of systems, so one set of
// launches can serve several contexts at once (an uneven batch of independent systems, with
// single-column groups when block COCG is off); a group's arithmetic is the same whichever other
// groups are in flight.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace rpa {
namespace {

constexpr int kBT = 256;               // threads of the streaming kernels
constexpr int kBChunk = 2048;          // grid points per norm work item (8 per thread)
constexpr int kBCheckEvery = 8;        // inner iterations between maintenance passes
constexpr int kBGramSlots = 32;        // blocks per group of a Gram launch (each sums every 32nd tile)
constexpr double kBBudget = 8.0e9;     // bytes of vectors of the groups in flight

// A group's phase: its inner solve starting (kBStart) or running (kBInner), ended and awaiting the
// FP64 residual (kBInnerDone), loaded and awaiting the first check (kBCheck), or done.
enum BPhase : int { kBDone = 0, kBInner = 1, kBInnerDone = 2, kBCheck = 3, kBStart = 4 };

template <typename T> struct BCx;
template <> struct BCx<float> { using t = float2; };
template <> struct BCx<double> { using t = double2; };

// grid points per Gram tile (two tiles of s rows in shared memory)
template <typename T> struct BTile { static constexpr int v = 256; };
template <> struct BTile<double> { static constexpr int v = 128; };

// One system (context) of a call: its grid, operator, orbitals and where its right-hand sides come
// from and its solutions go.  A call may hold several (the uneven batch), one table entry each.
struct BSys {
    long long nd;
    int nx, ny, nz, periodic;
    int ntile, nslot;              // Gram tiles, and Gram blocks per group (each sums every nslot-th tile)
    int ns;
    double a[kRadius + 1];         // stencil coefficients
    const double *V64;
    const float *V32;
    const double *psi;             // ns x nd orbitals
    const double *vt, *rhs, *Tc;   // right-hand sides: u_n (.) vt_row or rhs_row, P_c coefficients
    double sign;
    double *drho;                  // retire: drho_row += scale u_n (.) Re x (or nullptr) ...
    double scale;
    double2 *xout;                 // ... or x_out[sys] = x
};

// One group: the columns row0 .. row0 + ncol - 1 of orbital n (systems sys0 ..) of system ctx;
// column c of its vectors starts at element off + c nd.
struct BGroup {
    int n, ncol, sys0, row0, ctx;
    long long off;
    int phase, status, iters, refines, nearb, discard, nin, inner_iters;
    int nonfinite;
    int cap;                       // most columns an inner solve takes (halved at a near-breakdown)
    double sre, sim;               // shift -eps_n + i omega
    int refc[kMaxBlock];           // inner solves column c took part in
    int itc[kMaxBlock];            // inner iterations of column c
    int cmap[kMaxBlock];           // inner column -> column of the group
    double bn[kMaxBlock];          // ||b_c||
    double thr[kMaxBlock];         // stopping threshold of inner column ci (its residual starts at 1)
    double scl[kMaxBlock];         // ||r64|| of inner column ci at the start of the inner solve
};

struct BArgs {
    BGroup *g;
    const BSys *sys;
    int ngroups, sb;               // groups in flight, columns per group
    int nchunk;                    // norm work items per column (of the largest system)
    int mixed, maxit, max_refine;
    double tol, inner_tol, piv_tol;
    double2 *gpart;                // [group][kBGramSlots][sb*sb + sb] Gram partial sums; norms in .x of the tail
    double2 *rho;                  // [group][nin*nin]
    void *coef;                    // [group][nin*nin] alpha, then beta (complex T)
    double *npart;                 // [group*sb + c][nchunk][2] ||r64_c||^2, ||b_c||^2
    int *count;                    // [0] groups not done, [1] groups with an inner solve running
    const int *alist;              // the inner iterations' launches: grid index -> group (else identity)
};

__device__ __forceinline__ int group_of(const BArgs &A, int y) { return A.alist ? A.alist[y] : y; }

__device__ __forceinline__ int bwrap(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

// (H + sigma) v at point idx of one grid function: (3 a_0 + V + sigma) v + sum_k a_k (the six
// neighbours at distance k), zero outside the box or the periodic continuation.
template <typename T, typename C>
__device__ __forceinline__ C bstencil_at(const C *__restrict__ v, const T *__restrict__ V, int idx, int nx, int ny,
                                         int nz, int per, const T (&a)[kRadius + 1], T sre, T sim) {
    const int ix = idx % nx, t = idx / nx, iy = t % ny, iz = t / ny;
    const int sxy = nx * ny;
    const C c0 = v[idx];
    const T d = (T)3 * a[0] + V[idx] + sre;
    T re = d * c0.x - sim * c0.y, im = d * c0.y + sim * c0.x;
#pragma unroll
    for (int k = 1; k <= kRadius; ++k) {
        T sr = 0, si = 0;
        auto add = [&](int j) {
            const C w = v[j];
            sr += w.x;
            si += w.y;
        };
        if (per) {
            const int row = idx - ix, plane = idx - iy * nx, col = idx - iz * sxy;
            add(row + bwrap(ix - k, nx));
            add(row + bwrap(ix + k, nx));
            add(plane + bwrap(iy - k, ny) * nx);
            add(plane + bwrap(iy + k, ny) * nx);
            add(col + bwrap(iz - k, nz) * sxy);
            add(col + bwrap(iz + k, nz) * sxy);
        } else {
            if (ix - k >= 0) add(idx - k);
            if (ix + k < nx) add(idx + k);
            if (iy - k >= 0) add(idx - k * nx);
            if (iy + k < ny) add(idx + k * nx);
            if (iz - k >= 0) add(idx - k * sxy);
            if (iz + k < nz) add(idx + k * sxy);
        }
        re += a[k] * sr;
        im += a[k] * si;
    }
    C out;
    out.x = re;
    out.y = im;
    return out;
}

// Sum two doubles over the block (256 threads); valid in thread 0.  Fixed order.
__device__ __forceinline__ void bblock_sum2(double &a, double &b) {
    __shared__ double sh[2][kBT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        sh[0][warp] = a;
        sh[1][warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = b = 0.0;
        for (int w = 0; w < kBT / 32; ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
    }
}

// b = sign * (base - sum_k Tc[sys][k] u_k), base = u_n (.) vt_row (pairs) or rhs_row; x64 = 0,
// r64 = b.  Grid: (points / 256, groups * sb).
__global__ void __launch_bounds__(kBT) k_bload(BArgs A, double *__restrict__ b, double2 *__restrict__ x64,
                                               double2 *__restrict__ r64) {
    const int gi = blockIdx.y / A.sb, c = blockIdx.y % A.sb;
    const BGroup &G = A.g[gi];
    const BSys &S = A.sys[G.ctx];
    const long long idx = (long long)blockIdx.x * kBT + threadIdx.x;
    if (c >= G.ncol || idx >= S.nd) return;
    const int row = G.row0 + c, sys = G.sys0 + c;
    double base = S.vt ? S.psi[(long long)G.n * S.nd + idx] * S.vt[(long long)row * S.nd + idx]
                       : S.rhs[(long long)row * S.nd + idx];
    if (S.Tc)
        for (int k = 0; k < S.ns; ++k) base -= S.Tc[(long long)sys * S.ns + k] * S.psi[(long long)k * S.nd + idx];
    const double bv = S.sign * base;
    const long long o = G.off + (long long)c * S.nd + idx;
    b[o] = bv;
    x64[o] = make_double2(0.0, 0.0);
    r64[o] = make_double2(bv, 0.0);
}

// Partial sums of ||r64_c||^2 and ||b_c||^2 for the groups awaiting a check.
// Grid: (nchunk, groups * sb).
__global__ void __launch_bounds__(kBT) k_bnorm(BArgs A, const double *__restrict__ b,
                                               const double2 *__restrict__ r64) {
    const int gi = blockIdx.y / A.sb, c = blockIdx.y % A.sb;
    const BGroup &G = A.g[gi];
    if (c >= G.ncol || (G.phase != kBInnerDone && G.phase != kBCheck)) return;
    const long long nd = A.sys[G.ctx].nd;
    const long long o = G.off + (long long)c * nd;
    double rr = 0.0, bb = 0.0;
    for (int t = 0; t < kBChunk / kBT; ++t) {
        const long long idx = (long long)blockIdx.x * kBChunk + t * kBT + threadIdx.x;
        if (idx < nd) {
            const double2 r = r64[o + idx];
            const double bv = b[o + idx];
            rr += r.x * r.x + r.y * r.y;
            bb += bv * bv;
        }
    }
    bblock_sum2(rr, bb);
    if (threadIdx.x == 0) {
        double *q = A.npart + ((long long)blockIdx.y * A.nchunk + blockIdx.x) * 2;
        q[0] = rr;
        q[1] = bb;
    }
}

// Per group (one warp): the stopping test on the FP64 residual, then either the group is done or
// its next inner solve is set up on at most cap of the columns not yet converged (those with the
// largest relative residuals, ties by column; columns that have had max_refine inner solves are
// not taken again).
__global__ void k_bcheck(BArgs A) {
    const int gi = blockIdx.x, c = threadIdx.x;
    BGroup &G = A.g[gi];
    const int ph = G.phase;
    if (ph != kBInnerDone && ph != kBCheck) return;
    bool unconv = false, bad = false, elig = false;
    double rn = 0.0, bn = 0.0, key = -1.0;
    if (c < G.ncol) {
        const double *q = A.npart + ((long long)gi * A.sb + c) * A.nchunk * 2;
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < A.nchunk; ++k) {
            s0 += q[2 * k];
            s1 += q[2 * k + 1];
        }
        rn = sqrt(s0);
        if (ph == kBCheck) G.bn[c] = sqrt(s1);
        bn = G.bn[c];
        unconv = !(rn <= A.tol * bn);
        bad = !isfinite(rn);
        elig = unconv && G.refc[c] < A.max_refine;
        if (elig) key = bad ? 0.0 : rn / bn;
    }
    int rank = 0;
    for (int o = 0; o < 32; ++o) {
        const double ko = __shfl_sync(0xffffffffu, key, o);
        const int eo = __shfl_sync(0xffffffffu, (int)elig, o);
        if (eo && (ko > key || (ko == key && o < c))) ++rank;
    }
    const bool take = elig && rank < G.cap;
    const unsigned m = __ballot_sync(0xffffffffu, take);
    const unsigned mu = __ballot_sync(0xffffffffu, unconv);
    const unsigned mb = __ballot_sync(0xffffffffu, bad);
    const int nin = __popc(m);
    if (take) {
        const int ci = __popc(m & ((1u << c) - 1u));
        G.cmap[ci] = c;
        G.scl[ci] = rn;
        G.thr[ci] = A.mixed ? fmax(A.inner_tol, 0.3 * A.tol * bn / rn) : A.tol * bn / rn;
        G.refc[c] += 1;
    }
    __syncwarp();
    if (c == 0) {
        if (mu == 0) {
            G.phase = kBDone;
            G.status = RPA_OK;
        } else if (nin == 0) {
            G.phase = kBDone;
            G.status = (mb || G.nonfinite) ? RPA_ERR_BREAKDOWN : RPA_ERR_NOT_CONVERGED;
        } else {
            G.phase = kBStart;
            G.nin = nin;
            G.refines += 1;
            G.inner_iters = 0;
            G.discard = 0;
        }
    }
}

// Inner solve start: R = r64 / ||r64|| on the inner columns, X = 0, P = R.
template <typename T>
__global__ void __launch_bounds__(kBT) k_bstart(BArgs A, const double2 *__restrict__ r64,
                                                typename BCx<T>::t *__restrict__ x, typename BCx<T>::t *__restrict__ r,
                                                typename BCx<T>::t *__restrict__ p) {
    using C = typename BCx<T>::t;
    const int gi = blockIdx.y / A.sb, ci = blockIdx.y % A.sb;
    const BGroup &G = A.g[gi];
    const long long nd = A.sys[G.ctx].nd;
    const long long idx = (long long)blockIdx.x * kBT + threadIdx.x;
    if (G.phase != kBStart || ci >= G.nin || idx >= nd) return;
    const double inv = 1.0 / G.scl[ci];
    const double2 v = r64[G.off + (long long)G.cmap[ci] * nd + idx];
    const long long o = G.off + (long long)ci * nd + idx;
    C rv, z;
    rv.x = (T)(v.x * inv);
    rv.y = (T)(v.y * inv);
    z.x = (T)0;
    z.y = (T)0;
    x[o] = z;
    r[o] = rv;
    p[o] = rv;
}

template <typename T> __device__ __forceinline__ const T *bsys_v(const BSys &S);
template <> __device__ __forceinline__ const float *bsys_v<float>(const BSys &S) { return S.V32; }
template <> __device__ __forceinline__ const double *bsys_v<double>(const BSys &S) { return S.V64; }

// out = (H + sigma) in on the inner columns (T = the inner precision).
template <typename T>
__global__ void __launch_bounds__(kBT) k_bstencil(BArgs A, const typename BCx<T>::t *__restrict__ in,
                                                  typename BCx<T>::t *__restrict__ out) {
    const int gi = group_of(A, blockIdx.y / A.sb), ci = blockIdx.y % A.sb;
    const BGroup &G = A.g[gi];
    const BSys &S = A.sys[G.ctx];
    const long long idx = (long long)blockIdx.x * kBT + threadIdx.x;
    if (G.phase != kBInner || ci >= G.nin || idx >= S.nd) return;
    T a[kRadius + 1];
#pragma unroll
    for (int k = 0; k <= kRadius; ++k) a[k] = (T)S.a[k];
    const long long o = G.off + (long long)ci * S.nd;
    out[o + idx] = bstencil_at<T>(in + o, bsys_v<T>(S), (int)idx, S.nx, S.ny, S.nz, S.periodic, a, (T)G.sre,
                                  (T)G.sim);
}

// Gram partial sums: G_ij = sum_t X_i(t) Y_j(t) (unconjugated), and with norms != 0 also ||X_i||^2,
// over the tiles blockIdx.x, blockIdx.x + nslot, ... of the group's points (blocks past the
// system's nslot have nothing to do).  A tile of TP
// points of the n rows is staged in shared memory (once when X and Y are the same block), and the
// next tile's values are loaded into registers while the current one is summed.  Thread (e, sub)
// adds every nsub-th point of a tile for entry e = (i, j), in T within a tile and in FP64 across
// tiles; the nsub sums of an entry are added in order.  Grid: (kBGramSlots or fewer, groups); the
// partial sums of slot blockIdx.x go to gpart[group][blockIdx.x].
template <typename T, int NB>
__global__ void __launch_bounds__(kBT) k_bgram(BArgs A, const typename BCx<T>::t *__restrict__ X,
                                               const typename BCx<T>::t *__restrict__ Y, int norms, int ph) {
    using C = typename BCx<T>::t;
    constexpr int TP = BTile<T>::v;
    constexpr int LPT = NB * TP / kBT;            // staged values per thread and row block, at most
    extern __shared__ __align__(16) unsigned char bsm[];
    C *sx = reinterpret_cast<C *>(bsm);
    C *sy = sx + (size_t)A.sb * (TP + 1);
    __shared__ double2 red[kBT];
    __shared__ double redn[kBT];
    const int gi = group_of(A, blockIdx.y);
    const BGroup &G = A.g[gi];
    const BSys &S = A.sys[G.ctx];
    if (G.phase != ph || (int)blockIdx.x >= S.nslot) return;
    const bool same = X == Y;
    const int n = G.nin, E = n * n, tid = threadIdx.x;
    const long long gbase = G.off, nd = S.nd;
    C xr[LPT], yr[LPT];
    auto fetch = [&](int tile) {
        const long long p0 = (long long)tile * TP;
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            const int e = tid + l * kBT;
            xr[l].x = xr[l].y = (T)0;
            yr[l] = xr[l];
            if (e < n * TP) {
                const int c = e / TP, t = e % TP;
                if (p0 + t < nd) {
                    const long long o = gbase + (long long)c * nd + p0 + t;
                    xr[l] = X[o];
                    if (!same) yr[l] = Y[o];
                }
            }
        }
    };
    const int nsub = kBT / E;
    const bool active = tid < E * nsub;
    const int e0 = tid % E, sub = tid / E, i = e0 / n, j = e0 % n;
    const C *ys = same ? sx : sy;
    double sr = 0.0, si = 0.0, sn = 0.0;
    int tile = blockIdx.x;
    if (tile < S.ntile) fetch(tile);
    for (; tile < S.ntile; tile += S.nslot) {
        __syncthreads();                          // the previous tile has been summed
#pragma unroll
        for (int l = 0; l < LPT; ++l) {
            const int e = tid + l * kBT;
            if (e < n * TP) {
                const int c = e / TP, t = e % TP;
                sx[c * (TP + 1) + t] = xr[l];
                if (!same) sy[c * (TP + 1) + t] = yr[l];
            }
        }
        __syncthreads();
        const int len = (int)min((long long)TP, nd - (long long)tile * TP);
        if (tile + S.nslot < S.ntile) fetch(tile + S.nslot);
        if (active) {
            T ar = 0, ai = 0, an = 0;
            for (int t = sub; t < len; t += nsub) {
                const C u = sx[i * (TP + 1) + t], w = ys[j * (TP + 1) + t];
                ar += u.x * w.x - u.y * w.y;
                ai += u.x * w.y + u.y * w.x;
                an += u.x * u.x + u.y * u.y;
            }
            sr += (double)ar;
            si += (double)ai;
            sn += (double)an;
        }
    }
    red[tid] = make_double2(sr, si);
    redn[tid] = sn;
    __syncthreads();
    if (tid < E) {
        double tr = 0.0, ti = 0.0, tn = 0.0;
        for (int q = 0; q < nsub; ++q) {
            tr += red[q * E + tid].x;
            ti += red[q * E + tid].y;
            tn += redn[q * E + tid];
        }
        const int ii = tid / n, jj = tid % n;
        const int ld = A.sb * A.sb + A.sb;
        double2 *o = A.gpart + ((long long)gi * kBGramSlots + blockIdx.x) * ld;
        o[ii * A.sb + jj] = make_double2(tr, ti);
        if (norms && ii == jj) o[A.sb * A.sb + ii] = make_double2(tn, 0.0);
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdivd(double2 a, double2 b) {
    const double den = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

// Per group (one block): add the Gram partial sums in tile order, then
//   mode 0 (inner start): rho = R^T R; stopping test; the inner solve runs from here on;
//   mode 1: alpha = (P^T Q)^-1 rho;
//   mode 2: stopping test on the column norms, iteration limit; beta = rho^-1 rho', rho = rho'.
// The s x s solves run in FP64 by Gaussian elimination with partial pivoting on the system
// equilibrated by the rows' largest entries (D M D) y = D rhs, x = D y, D_i = max_j |M_ij|^-1/2; a
// pivot below piv_tol (entries of D M D are at most 1) ends the inner solve.
template <typename T>
__global__ void __launch_bounds__(256) k_bsmall(BArgs A, int mode) {
    using C = typename BCx<T>::t;
    __shared__ double2 M[kMaxBlock * kMaxBlock];
    __shared__ double2 Bm[kMaxBlock * kMaxBlock];
    __shared__ double2 S[kMaxBlock * kMaxBlock];
    __shared__ double nrm[kMaxBlock], sc[kMaxBlock];
    __shared__ double2 fct[kMaxBlock];
    __shared__ int flag, piv;     // flag: 1 converged, 2 singular, 3 non-finite, 4 iteration limit
    const int gi = group_of(A, blockIdx.x), tid = threadIdx.x;
    BGroup &G = A.g[gi];
    if (G.phase != (mode == 0 ? kBStart : kBInner)) return;
    const int n = G.nin, E = n * n, ld = A.sb * A.sb + A.sb, nslot = A.sys[G.ctx].nslot;
    for (int e = tid; e < E + n; e += blockDim.x) {
        const int off = e < E ? (e / n) * A.sb + e % n : A.sb * A.sb + (e - E);
        const double2 *q = A.gpart + (long long)gi * kBGramSlots * ld + off;
        double sr = 0.0, si = 0.0;
        for (int t = 0; t < nslot; ++t) {
            const double2 v = q[(long long)t * ld];
            sr += v.x;
            si += v.y;
        }
        if (e < E) S[e] = make_double2(sr, si);
        else nrm[e - E] = sr;
    }
    if (tid == 0) flag = 0;
    __syncthreads();
    double2 *rho = A.rho + (long long)gi * A.sb * A.sb;
    if (tid == 0) {
        bool fin = true, all = true;
        for (int e = 0; e < E; ++e)
            if (!isfinite(S[e].x) || !isfinite(S[e].y)) fin = false;
        if (mode != 1)
            for (int i = 0; i < n; ++i) {
                const double r = sqrt(nrm[i]);
                if (!isfinite(r)) fin = false;
                if (!(r <= G.thr[i])) all = false;
            }
        if (!fin) flag = 3;
        else if (mode != 1 && all) flag = 1;
        else if (mode == 2 && G.inner_iters >= A.maxit) flag = 4;
    }
    __syncthreads();
    if (flag) {
        if (tid == 0) {
            if (flag == 3) {
                G.discard = 1;
                G.nonfinite = 1;
            }
            G.phase = kBInnerDone;
        }
        return;
    }
    if (mode == 0) {
        for (int e = tid; e < E; e += blockDim.x) rho[e] = S[e];
        if (tid == 0) G.phase = kBInner;
        return;
    }
    for (int e = tid; e < E; e += blockDim.x) {
        M[e] = mode == 1 ? S[e] : rho[e];
        Bm[e] = mode == 1 ? rho[e] : S[e];
    }
    __syncthreads();
    if (tid < n) {
        double mx = 0.0;
        for (int j = 0; j < n; ++j) mx = fmax(mx, hypot(M[tid * n + j].x, M[tid * n + j].y));
        sc[tid] = (mx > 0.0 && isfinite(mx)) ? 1.0 / sqrt(mx) : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < E; e += blockDim.x) {
        const int i = e / n, j = e % n;
        const double f = sc[i] * sc[j];
        M[e] = make_double2(M[e].x * f, M[e].y * f);
        Bm[e] = make_double2(Bm[e].x * sc[i], Bm[e].y * sc[i]);
    }
    if (tid == 0)
        for (int i = 0; i < n; ++i)
            if (sc[i] == 0.0) flag = 2;
    __syncthreads();
    // flag is written by thread 0 only before a barrier and read by all only after one
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            int r = k;
            double best = hypot(M[k * n + k].x, M[k * n + k].y);
            for (int i = k + 1; i < n; ++i) {
                const double v = hypot(M[i * n + k].x, M[i * n + k].y);
                if (v > best) {
                    best = v;
                    r = i;
                }
            }
            if (!(best > A.piv_tol)) flag = 2;
            piv = r;
        }
        __syncthreads();
        if (flag) break;
        const int r = piv;
        if (r != k)
            for (int t = tid; t < 2 * n; t += blockDim.x) {
                double2 *a = t < n ? &M[k * n + t] : &Bm[k * n + t - n];
                double2 *b = t < n ? &M[r * n + t] : &Bm[r * n + t - n];
                const double2 tmp = *a;
                *a = *b;
                *b = tmp;
            }
        __syncthreads();
        if (tid > k && tid < n) fct[tid] = cdivd(M[tid * n + k], M[k * n + k]);
        __syncthreads();
        for (int t = tid; t < (n - k - 1) * 2 * n; t += blockDim.x) {
            const int i = k + 1 + t / (2 * n), col = t % (2 * n);
            if (col < n) {
                if (col > k) {
                    const double2 d = cmul(fct[i], M[k * n + col]);
                    M[i * n + col].x -= d.x;
                    M[i * n + col].y -= d.y;
                }
            } else {
                const double2 d = cmul(fct[i], Bm[k * n + col - n]);
                Bm[i * n + col - n].x -= d.x;
                Bm[i * n + col - n].y -= d.y;
            }
        }
        __syncthreads();
    }
    if (flag) {
        if (tid == 0) {
            G.nearb += 1;
            G.cap = max(1, n / 2);
            G.phase = kBInnerDone;
        }
        return;
    }
    if (tid < n) {
        const int j = tid;
        for (int k = n - 1; k >= 0; --k) {
            double2 s = Bm[k * n + j];
            for (int m = k + 1; m < n; ++m) {
                const double2 d = cmul(M[k * n + m], Bm[m * n + j]);
                s.x -= d.x;
                s.y -= d.y;
            }
            Bm[k * n + j] = cdivd(s, M[k * n + k]);
        }
    }
    __syncthreads();
    C *cf = reinterpret_cast<C *>(A.coef) + (long long)gi * A.sb * A.sb;
    for (int e = tid; e < E; e += blockDim.x) {
        const double f = sc[e / n];
        C v;
        v.x = (T)(Bm[e].x * f);
        v.y = (T)(Bm[e].y * f);
        cf[e] = v;
    }
    if (mode == 1) {
        if (tid == 0) {
            G.inner_iters += 1;
            G.iters += 1;
            for (int i = 0; i < n; ++i) G.itc[G.cmap[i]] += 1;
        }
    } else {
        for (int e = tid; e < E; e += blockDim.x) rho[e] = S[e];
    }
}

// X += P alpha, R -= Q alpha (UPDATE), or P = R + P beta, per grid point over the group's inner
// columns held in registers.  Grid: (points / 256, groups).
template <typename T, int NB, bool UPDATE>
__global__ void __launch_bounds__(kBT) k_bmix(BArgs A, typename BCx<T>::t *__restrict__ x,
                                              typename BCx<T>::t *__restrict__ r, typename BCx<T>::t *__restrict__ p,
                                              const typename BCx<T>::t *__restrict__ q) {
    using C = typename BCx<T>::t;
    __shared__ C cf[NB * NB];
    const int gi = group_of(A, blockIdx.y);
    const BGroup &G = A.g[gi];
    if (G.phase != kBInner) return;
    const int n = G.nin;
    const C *src = reinterpret_cast<const C *>(A.coef) + (long long)gi * A.sb * A.sb;
    for (int e = threadIdx.x; e < NB * NB; e += kBT) {
        const int i = e / NB, j = e % NB;
        C v;
        v.x = v.y = (T)0;
        if (i < n && j < n) v = src[i * n + j];
        cf[e] = v;
    }
    __syncthreads();
    const long long nd = A.sys[G.ctx].nd;
    const long long idx = (long long)blockIdx.x * kBT + threadIdx.x;
    if (idx >= nd) return;
    const long long base = G.off + idx;
    C pk[NB], qk[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        pk[k].x = pk[k].y = (T)0;
        qk[k] = pk[k];
        if (k < n) {
            pk[k] = p[base + (long long)k * nd];
            if (UPDATE) qk[k] = q[base + (long long)k * nd];
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (j < n) {
            T ur = 0, ui = 0, vr = 0, vi = 0;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const C a = cf[k * NB + j];
                ur += pk[k].x * a.x - pk[k].y * a.y;
                ui += pk[k].x * a.y + pk[k].y * a.x;
                if (UPDATE) {
                    vr += qk[k].x * a.x - qk[k].y * a.y;
                    vi += qk[k].x * a.y + qk[k].y * a.x;
                }
            }
            const long long o = base + (long long)j * nd;
            C rv = r[o];
            if (UPDATE) {
                C xv = x[o];
                xv.x += ur;
                xv.y += ui;
                rv.x -= vr;
                rv.y -= vi;
                x[o] = xv;
                r[o] = rv;
            } else {
                rv.x += ur;
                rv.y += ui;
                p[o] = rv;
            }
        }
    }
}

// x64 += ||r64|| X on the inner columns of the groups whose inner solve ended (unless it went
// non-finite).  Grid: (points / 256, groups * sb).
template <typename T>
__global__ void __launch_bounds__(kBT) k_bacc(BArgs A, const typename BCx<T>::t *__restrict__ x,
                                              double2 *__restrict__ x64) {
    const int gi = blockIdx.y / A.sb, ci = blockIdx.y % A.sb;
    const BGroup &G = A.g[gi];
    const long long nd = A.sys[G.ctx].nd;
    const long long idx = (long long)blockIdx.x * kBT + threadIdx.x;
    if (G.phase != kBInnerDone || G.discard || ci >= G.nin || idx >= nd) return;
    const double s = G.scl[ci];
    const typename BCx<T>::t d = x[G.off + (long long)ci * nd + idx];
    double2 &o = x64[G.off + (long long)G.cmap[ci] * nd + idx];
    o.x += s * (double)d.x;
    o.y += s * (double)d.y;
}

// r64 = b - (H + sigma) x64 in FP64 on every column of the groups whose inner solve ended.
__global__ void __launch_bounds__(kBT) k_bresid(BArgs A, const double *__restrict__ b,
                                                const double2 *__restrict__ x64, double2 *__restrict__ r64) {
    const int gi = blockIdx.y / A.sb, c = blockIdx.y % A.sb;
    const BGroup &G = A.g[gi];
    const BSys &S = A.sys[G.ctx];
    const long long idx = (long long)blockIdx.x * kBT + threadIdx.x;
    if (G.phase != kBInnerDone || c >= G.ncol || idx >= S.nd) return;
    double a[kRadius + 1];
#pragma unroll
    for (int k = 0; k <= kRadius; ++k) a[k] = S.a[k];
    const long long o = G.off + (long long)c * S.nd;
    const double2 ax = bstencil_at<double>(x64 + o, S.V64, (int)idx, S.nx, S.ny, S.nz, S.periodic, a, G.sre, G.sim);
    r64[o + idx] = make_double2(b[o + idx] - ax.x, -ax.y);
}

// The groups with an inner solve running, in group order (each thread takes a contiguous range;
// the ranges' counts are scanned in order), and the number of groups not done.  One block of 1024.
__global__ void __launch_bounds__(1024) k_blist(BArgs A, int *__restrict__ list) {
    __shared__ int cnt[1024];
    __shared__ int notdone;
    const int t = threadIdx.x;
    const int per = (A.ngroups + 1023) / 1024;
    const int g0 = min(A.ngroups, t * per), g1 = min(A.ngroups, g0 + per);
    int m = 0, nd = 0;
    for (int g = g0; g < g1; ++g) {
        const int ph = A.g[g].phase;
        m += ph == kBInner;
        nd += ph != kBDone;
    }
    cnt[t] = m;
    if (t == 0) notdone = 0;
    __syncthreads();
    atomicAdd(&notdone, nd);
    if (t == 0) {
        int sum = 0;
        for (int i = 0; i < 1024; ++i) {
            const int v = cnt[i];
            cnt[i] = sum;
            sum += v;
        }
        A.count[1] = sum;
    }
    __syncthreads();
    int w = cnt[t];
    for (int g = g0; g < g1; ++g)
        if (A.g[g].phase == kBInner) list[w++] = g;
    if (t == 0) A.count[0] = notdone;
}

// drho_j += (4/h^3) u_n (.) Re x64 for every row (system ctx, column j) of rows, the groups of
// that system's orbitals added in group order.  Grid: (points / 256, rows).
__global__ void __launch_bounds__(kBT) k_bretire_drho(BArgs A, const int2 *__restrict__ rows,
                                                      const double2 *__restrict__ x64) {
    const int2 rj = rows[blockIdx.y];
    const BSys &S = A.sys[rj.x];
    const int j = rj.y;
    const long long idx = (long long)blockIdx.x * kBT + threadIdx.x;
    if (idx >= S.nd) return;
    double acc = S.drho[(long long)j * S.nd + idx];
    for (int gi = 0; gi < A.ngroups; ++gi) {
        const BGroup &G = A.g[gi];
        const int c = j - G.row0;
        if (G.ctx != rj.x || c < 0 || c >= G.ncol) continue;
        acc += S.scale * S.psi[(long long)G.n * S.nd + idx] * x64[G.off + (long long)c * S.nd + idx].x;
    }
    S.drho[(long long)j * S.nd + idx] = acc;
}

// x_out[sys] = x64 for every column of the systems that copy their solutions out.
// Grid: (points / 256, groups * sb).
__global__ void __launch_bounds__(kBT) k_bretire_copy(BArgs A, const double2 *__restrict__ x64) {
    const int gi = blockIdx.y / A.sb, c = blockIdx.y % A.sb;
    const BGroup &G = A.g[gi];
    const BSys &S = A.sys[G.ctx];
    const long long idx = (long long)blockIdx.x * kBT + threadIdx.x;
    if (!S.xout || c >= G.ncol || idx >= S.nd) return;
    S.xout[(long long)(G.sys0 + c) * S.nd + idx] = x64[G.off + (long long)c * S.nd + idx];
}

// rows[j] = u_n (.) dv_j for j < ncols (right-hand sides of orbital n before the projection).
__global__ void k_bpair_rows(const double *__restrict__ psi, const double *__restrict__ dv, int n, long long nd,
                             double *__restrict__ rows) {
    const int j = blockIdx.y;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += (long long)gridDim.x * blockDim.x)
        rows[(long long)j * nd + i] = psi[(long long)n * nd + i] * dv[(long long)j * nd + i];
}

// One system's share of a call: its context, where its right-hand sides come from, where its
// solutions go, and its groups.
struct BSpec {
    Ctx *c = nullptr;
    const double *vt = nullptr;     // pair right-hand sides u_n (.) vt_row ...
    const double *rhs = nullptr;    // ... or rows of rhs
    const double *Tc = nullptr;     // P_c coefficients per system (or nullptr)
    double sign = 1.0;
    double omega = 0.0;
    double *drho = nullptr;         // retire into drho (ncols rows) ...
    int ncols = 0;
    double2 *xout = nullptr;        // ... or copy the solutions out
    std::vector<BGroup> groups;     // in retire order
};

template <typename T, int NB>
void launch_mix(const BArgs &A, void *x, void *r, void *p, const void *q, bool update, dim3 grid, cudaStream_t s) {
    using C = typename BCx<T>::t;
    if (update)
        k_bmix<T, NB, true><<<grid, kBT, 0, s>>>(A, (C *)x, (C *)r, (C *)p, (const C *)q);
    else
        k_bmix<T, NB, false><<<grid, kBT, 0, s>>>(A, (C *)x, (C *)r, (C *)p, (const C *)q);
    RPA_LAUNCH("block COCG mix");
}

template <typename T>
void mix(const BArgs &A, void *x, void *r, void *p, const void *q, bool update, dim3 grid, cudaStream_t s) {
    if (A.sb <= 4) launch_mix<T, 4>(A, x, r, p, q, update, grid, s);
    else if (A.sb <= 8) launch_mix<T, 8>(A, x, r, p, q, update, grid, s);
    else launch_mix<T, 16>(A, x, r, p, q, update, grid, s);
}

// With rpa_options.profile: CUDA events around every launch of the block path by kind, added up at
// each synchronisation and reported in rpa_stats.prof_* (times and launches; no point counts).
struct BTimer {
    enum { kStencil, kGram, kSmall, kMix, kMaint, kLoadRetire, kKinds };
    Ctx &c;
    cudaStream_t st;
    bool on;
    std::vector<std::pair<int, size_t>> rec;
    double ms[kKinds] = {};
    long long n[kKinds] = {};
    cudaEvent_t ev(size_t i) {
        while (c.ev_pool.size() <= i) {
            cudaEvent_t e;
            RPA_CUDA(cudaEventCreate(&e));
            c.ev_pool.push_back(e);
        }
        return c.ev_pool[i];
    }
    void begin(int kind) {
        if (!on) return;
        const size_t i = 2 * rec.size();
        RPA_CUDA(cudaEventRecord(ev(i), st));
        rec.push_back({kind, i});
    }
    void end() {
        if (on) RPA_CUDA(cudaEventRecord(ev(rec.back().second + 1), st));
    }
    void collect() {   // after a synchronisation of st
        for (const auto &r : rec) {
            float t = 0.f;
            RPA_CUDA(cudaEventElapsedTime(&t, c.ev_pool[r.second], c.ev_pool[r.second + 1]));
            ms[r.first] += t;
            n[r.first] += 1;
        }
        rec.clear();
    }
    void report() {
        if (!on) return;
        static const char *names[kKinds] = {"block_stencil", "block_gram", "block_small", "block_mix",
                                            "block_maintenance", "block_load_retire"};
        for (int k = 0; k < kKinds; ++k) {
            if (!n[k]) continue;
            const int sl = prof_slot(c, names[k]);
            c.stats.prof_ms[sl] += ms[k];
            c.stats.prof_launches[sl] += n[k];
        }
    }
};

// Gram launch for groups of up to NB >= sb columns; gx blocks per group (the largest nslot).
template <typename T>
void gram_launch(const BArgs &A, const void *X, const void *Y, int norms, int ph, int gx, unsigned groups,
                 size_t smem, cudaStream_t s) {
    using C = typename BCx<T>::t;
    const dim3 grid(gx, groups);
    if (A.sb <= 4) k_bgram<T, 4><<<grid, kBT, smem, s>>>(A, (const C *)X, (const C *)Y, norms, ph);
    else if (A.sb <= 8) k_bgram<T, 8><<<grid, kBT, smem, s>>>(A, (const C *)X, (const C *)Y, norms, ph);
    else k_bgram<T, 16><<<grid, kBT, smem, s>>>(A, (const C *)X, (const C *)Y, norms, ph);
    RPA_LAUNCH("block COCG gram");
}

// The block solves of every group of every system in specs, with the iteration settings and the
// workspaces of `lead` (all systems share its precision, tolerances and block size).  Groups are
// taken in waves (in spec order, then group order) as far as the vector budget allows.
template <typename T>
int run_block_t(Ctx &lead, std::vector<BSpec *> &specs, cudaStream_t st, std::vector<int> *iters_out,
                std::vector<int> *status_out, std::vector<int> *spec_worst) {
    using C = typename BCx<T>::t;
    constexpr int TP = BTile<T>::v;
    const bool mixed = lead.opt.prec == RPA_MIXED;
    const int sb = lead.opt.block_cocg > 0 ? lead.opt.block_cocg : 1;
    const int nspec = (int)specs.size();

    // the system table (host copy)
    std::vector<BSys> sys(nspec);
    long long nd_max = 0;
    for (int k = 0; k < nspec; ++k) {
        const BSpec &sp = *specs[k];
        const Ctx &c = *sp.c;
        BSys &S = sys[k];
        S = BSys{};
        S.nd = c.nd;
        S.nx = c.nx;
        S.ny = c.ny;
        S.nz = c.nz;
        S.periodic = c.opt.periodic;
        S.ntile = (int)((c.nd + TP - 1) / TP);
        S.nslot = std::min(S.ntile, kBGramSlots);
        S.ns = c.ns;
        for (int q = 0; q <= kRadius; ++q) S.a[q] = c.coef.a[q];
        S.V64 = c.vloc64;
        S.V32 = c.vloc32;
        S.psi = c.psi64;
        S.vt = sp.vt;
        S.rhs = sp.rhs;
        S.Tc = sp.Tc;
        S.sign = sp.sign;
        S.drho = sp.drho;
        S.scale = 4.0 / (c.h * c.h * c.h);
        S.xout = sp.xout;
        nd_max = std::max(nd_max, c.nd);
    }
    // all groups, and the waves: consecutive groups whose vectors fit the budget
    std::vector<BGroup> all;
    for (int k = 0; k < nspec; ++k)
        for (BGroup g : specs[k]->groups) {
            g.ctx = k;
            g.cap = g.ncol;
            g.phase = kBCheck;
            g.status = RPA_OK;
            g.sre = -specs[k]->c->eps[g.n];
            g.sim = specs[k]->omega;
            all.push_back(g);
        }
    const int total = (int)all.size();
    if (total == 0) return RPA_OK;
    const double per_point = 8.0 + 16.0 + 16.0 + 4.0 * sizeof(C);
    int wmax = 65535 / sb;
    if (lead.opt.batch_systems > 0) wmax = std::min(wmax, std::max(1, lead.opt.batch_systems / sb));
    std::vector<int> wave_start{0};
    std::vector<long long> wave_elems;
    {
        long long elems = 0;
        int count = 0;
        for (int i = 0; i < total; ++i) {
            const long long e = (long long)sb * sys[all[i].ctx].nd;
            if (count > 0 && (count >= wmax || (elems + e) * per_point > kBBudget)) {
                wave_start.push_back(i);
                wave_elems.push_back(elems);
                elems = 0;
                count = 0;
            }
            all[i].off = elems;
            elems += e;
            ++count;
        }
        wave_start.push_back(total);
        wave_elems.push_back(elems);
    }
    int W = 0;
    long long n = 0;
    for (size_t w = 0; w + 1 < wave_start.size(); ++w) {
        W = std::max(W, wave_start[w + 1] - wave_start[w]);
        n = std::max(n, wave_elems[w]);
    }
    // drho rows (system, column) of the systems that retire into drho
    std::vector<int2> rows;
    for (int k = 0; k < nspec; ++k)
        if (specs[k]->drho)
            for (int j = 0; j < specs[k]->ncols; ++j) rows.push_back(make_int2(k, j));
    if (rows.size() > 65535) fail(RPA_ERR_INVALID, "block COCG: more than 65535 columns in one call");

    BArgs A{};
    A.sb = sb;
    A.nchunk = (int)((nd_max + kBChunk - 1) / kBChunk);
    A.mixed = mixed;
    A.maxit = lead.opt.maxit;
    A.max_refine = lead.opt.max_refine;
    A.tol = lead.opt.tol;
    A.inner_tol = lead.opt.inner_tol;
    A.piv_tol = mixed ? 1e-5 : 1e-12;
    int gx = 1;
    for (const BSys &S : sys) gx = std::max(gx, S.nslot);

    // storage: b, x64, r64 (FP64), then X, R, P, Q (inner precision), then the small arrays
    const size_t ld = (size_t)sb * sb + sb;
    const size_t bytes = (size_t)n * (8 + 16 + 16 + 4 * sizeof(C)) + sizeof(BGroup) * W + sizeof(BSys) * nspec +
                         sizeof(int2) * rows.size() +
                         sizeof(double2) * ((size_t)W * kBGramSlots * ld + 2 * (size_t)W * sb * sb) +
                         sizeof(double) * (size_t)W * sb * A.nchunk * 2 + sizeof(int) * (W + 4) + 16 * 256;
    char *base = (char *)lead.cocg_state.ensure(bytes);
    size_t off = 0;
    auto take = [&](size_t nb) {
        off = (off + 255) / 256 * 256;
        char *q = base + off;
        off += nb;
        return (void *)q;
    };
    double *b = (double *)take(sizeof(double) * n);
    double2 *x64 = (double2 *)take(sizeof(double2) * n);
    double2 *r64 = (double2 *)take(sizeof(double2) * n);
    C *xv = (C *)take(sizeof(C) * n);
    C *rv = (C *)take(sizeof(C) * n);
    C *pv = (C *)take(sizeof(C) * n);
    C *qv = (C *)take(sizeof(C) * n);
    A.g = (BGroup *)take(sizeof(BGroup) * W);
    BSys *sys_dev = (BSys *)take(sizeof(BSys) * nspec);
    A.sys = sys_dev;
    int2 *rows_dev = (int2 *)take(sizeof(int2) * std::max<size_t>(rows.size(), 1));
    A.gpart = (double2 *)take(sizeof(double2) * (size_t)W * kBGramSlots * ld);
    A.rho = (double2 *)take(sizeof(double2) * (size_t)W * sb * sb);
    A.coef = take(sizeof(double2) * (size_t)W * sb * sb);
    A.npart = (double *)take(sizeof(double) * (size_t)W * sb * A.nchunk * 2);
    A.count = (int *)take(sizeof(int) * 4);
    int *alist = (int *)take(sizeof(int) * W);
    RPA_CUDA(cudaMemcpyAsync(sys_dev, sys.data(), sizeof(BSys) * nspec, cudaMemcpyHostToDevice, st));
    if (!rows.empty())
        RPA_CUDA(cudaMemcpyAsync(rows_dev, rows.data(), sizeof(int2) * rows.size(), cudaMemcpyHostToDevice, st));

    const size_t gram_smem = 2 * (size_t)sb * (TP + 1) * sizeof(C);
    allow_dynamic_smem((const void *)k_bgram<T, 4>, gram_smem);
    allow_dynamic_smem((const void *)k_bgram<T, 8>, gram_smem);
    allow_dynamic_smem((const void *)k_bgram<T, 16>, gram_smem);
    const unsigned pblk = (unsigned)((nd_max + kBT - 1) / kBT);

    std::vector<QueueStats> qs(nspec, QueueStats{});
    std::vector<int> worst(nspec, RPA_OK);
    std::vector<BGroup> h(W);
    BTimer tm{lead, st, lead.opt.profile != 0};
    auto read_counts = [&]() {
        RPA_CUDA(cudaMemcpyAsync(lead.h_count, A.count, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        sync_stream(lead, st);
        tm.collect();
    };
    for (size_t w = 0; w + 1 < wave_start.size(); ++w) {
        const int w0 = wave_start[w], nw = wave_start[w + 1] - w0;
        A.ngroups = nw;
        std::copy(all.begin() + w0, all.begin() + w0 + nw, h.begin());
        RPA_CUDA(cudaMemcpyAsync(A.g, h.data(), sizeof(BGroup) * nw, cudaMemcpyHostToDevice, st));
        const dim3 gcols(pblk, nw * sb);
        tm.begin(BTimer::kLoadRetire);
        k_bload<<<gcols, kBT, 0, st>>>(A, b, x64, r64);
        RPA_LAUNCH("block COCG load");
        tm.end();
        count_launches(1);
        // Maintenance, then kBCheckEvery inner iterations over the groups whose inner solve runs,
        // until every group is done: a group whose inner solve ended takes its FP64 residual,
        // stopping test and next inner start at the next maintenance pass while the others keep
        // iterating.  The inner iterations launch over the list of running groups only.
        BArgs Ai = A;
        Ai.alist = alist;
        for (;;) {
            tm.begin(BTimer::kMaint);
            k_bacc<T><<<gcols, kBT, 0, st>>>(A, xv, x64);
            RPA_LAUNCH("block COCG accumulate");
            k_bresid<<<gcols, kBT, 0, st>>>(A, b, x64, r64);
            RPA_LAUNCH("block COCG residual");
            k_bnorm<<<dim3(A.nchunk, nw * sb), kBT, 0, st>>>(A, b, r64);
            RPA_LAUNCH("block COCG norms");
            k_bcheck<<<nw, 32, 0, st>>>(A);
            RPA_LAUNCH("block COCG check");
            k_bstart<T><<<gcols, kBT, 0, st>>>(A, r64, xv, rv, pv);
            RPA_LAUNCH("block COCG start");
            gram_launch<T>(A, rv, rv, 1, kBStart, gx, nw, gram_smem, st);
            k_bsmall<T><<<nw, 256, 0, st>>>(A, 0);
            RPA_LAUNCH("block COCG small");
            k_blist<<<1, 1024, 0, st>>>(A, alist);
            RPA_LAUNCH("block COCG list");
            tm.end();
            count_launches(8);
            read_counts();
            const int notdone = lead.h_count[0], running = lead.h_count[1];
            if (notdone == 0) break;
            if (running == 0) continue;
            const dim3 icols(pblk, running * sb), igrp(pblk, running);
            for (int it = 0; it < kBCheckEvery; ++it) {
                tm.begin(BTimer::kStencil);
                k_bstencil<T><<<icols, kBT, 0, st>>>(Ai, pv, qv);
                RPA_LAUNCH("block COCG stencil");
                tm.end();
                tm.begin(BTimer::kGram);
                gram_launch<T>(Ai, pv, qv, 0, kBInner, gx, running, gram_smem, st);
                tm.end();
                tm.begin(BTimer::kSmall);
                k_bsmall<T><<<running, 256, 0, st>>>(Ai, 1);
                RPA_LAUNCH("block COCG small");
                tm.end();
                tm.begin(BTimer::kMix);
                mix<T>(Ai, xv, rv, pv, qv, true, igrp, st);
                tm.end();
                tm.begin(BTimer::kGram);
                gram_launch<T>(Ai, rv, rv, 1, kBInner, gx, running, gram_smem, st);
                tm.end();
                tm.begin(BTimer::kSmall);
                k_bsmall<T><<<running, 256, 0, st>>>(Ai, 2);
                RPA_LAUNCH("block COCG small");
                tm.end();
                tm.begin(BTimer::kMix);
                mix<T>(Ai, xv, rv, pv, qv, false, igrp, st);
                tm.end();
                count_launches(7);
            }
        }
        tm.begin(BTimer::kLoadRetire);
        if (!rows.empty()) {
            k_bretire_drho<<<dim3(pblk, (unsigned)rows.size()), kBT, 0, st>>>(A, rows_dev, x64);
            RPA_LAUNCH("block COCG retire");
            count_launches(1);
        }
        bool copies = false;
        for (const BSpec *sp : specs) copies = copies || sp->xout;
        if (copies) {
            k_bretire_copy<<<gcols, kBT, 0, st>>>(A, x64);
            RPA_LAUNCH("block COCG copy");
            count_launches(1);
        }
        tm.end();
        RPA_CUDA(cudaMemcpyAsync(h.data(), A.g, sizeof(BGroup) * nw, cudaMemcpyDeviceToHost, st));
        sync_stream(lead, st);
        tm.collect();
        for (int i = 0; i < nw; ++i) {
            const BGroup &g = h[i];
            QueueStats &q = qs[g.ctx];
            q.solves += g.ncol;
            q.nearb += g.nearb;
            worst[g.ctx] = std::max(worst[g.ctx], g.status);
            for (int k = 0; k < g.ncol; ++k) {
                q.iters += g.itc[k];
                q.refines += g.refc[k];
                if (iters_out) (*iters_out)[g.sys0 + k] = g.itc[k];
                if (status_out) (*status_out)[g.sys0 + k] = g.status;
            }
        }
    }
    tm.report();
    int w_all = RPA_OK;
    if (spec_worst) spec_worst->assign(nspec, RPA_OK);
    for (int k = 0; k < nspec; ++k) {
        qs[k].worst = worst[k];
        const int wk = add_queue_stats(*specs[k]->c, qs[k]);
        if (spec_worst) (*spec_worst)[k] = wk;
        w_all = std::max(w_all, wk);
    }
    return w_all;
}

int run_block(Ctx &lead, std::vector<BSpec *> &specs, cudaStream_t st, std::vector<int> *iters,
              std::vector<int> *status, std::vector<int> *spec_worst = nullptr) {
    return lead.opt.prec == RPA_MIXED ? run_block_t<float>(lead, specs, st, iters, status, spec_worst)
                                      : run_block_t<double>(lead, specs, st, iters, status, spec_worst);
}

BGroup make_group(int n, int ncol, int sys0, int row0) {
    BGroup g{};
    g.n = n;
    g.ncol = ncol;
    g.sys0 = sys0;
    g.row0 = row0;
    return g;
}

// The pair right-hand sides of chi0 on ncols columns of dv for one context: P_c coefficients
// T[(n, j)][k] = u_k . (u_n (.) dv_j) in FP64 (the block iteration does not project its residuals
// again, so the right-hand sides keep whatever occupied components these coefficients leave), and
// the groups of s consecutive columns per orbital.  T lives in `coef` (grown as needed).
void chi0_spec(Ctx &c, double omega, const double *dv, double *drho, int ncols, int sb, DevBuf &coef, BSpec &sp,
               cudaStream_t s) {
    RPA_CUDA(cudaMemsetAsync(drho, 0, sizeof(double) * (size_t)ncols * c.nd, s));
    double *T = (double *)coef.ensure(sizeof(double) * (size_t)c.ns * ncols * c.ns);
    double *rows = (double *)c.rhs.ensure(sizeof(double) * (size_t)ncols * c.nd);
    for (int n = 0; n < c.ns; ++n) {
        k_bpair_rows<<<dim3((unsigned)std::min<long long>((c.nd + 255) / 256, 1024), ncols), 256, 0, s>>>(
            c.psi64, dv, n, c.nd, rows);
        RPA_LAUNCH("block COCG pair rows");
        count_launches(1);
        gram(rows, ncols, c.psi64, c.ns, c.nd, T + (size_t)n * ncols * c.ns, s, c.dense_scratch);
    }
    sp.c = &c;
    sp.vt = dv;
    sp.Tc = T;
    sp.sign = -1.0;
    sp.omega = omega;
    sp.drho = drho;
    sp.ncols = ncols;
    for (int n = 0; n < c.ns; ++n)
        for (int j0 = 0; j0 < ncols; j0 += sb)
            sp.groups.push_back(make_group(n, std::min(sb, ncols - j0), n * ncols + j0, j0));
}

}  // namespace

int chi0_apply_block(Ctx &c, double omega, const double *dv, double *drho, int ncols, cudaStream_t s) {
    if (ncols == 0) return RPA_OK;
    BSpec sp;
    chi0_spec(c, omega, dv, drho, ncols, c.opt.block_cocg, c.pc_coef, sp, s);
    std::vector<BSpec *> specs{&sp};
    return run_block(c, specs, s, nullptr, nullptr);
}

int chi0_apply_batch(const std::vector<Chi0Request> &reqs, cudaStream_t s, std::vector<int> *status) {
    if (status) status->assign(reqs.size(), RPA_OK);
    if (reqs.empty()) return RPA_OK;
    Ctx &lead = *reqs[0].c;
    const int sb = std::max(1, lead.opt.block_cocg);
    std::vector<BSpec> sp(reqs.size());
    std::vector<BSpec *> specs;
    std::vector<size_t> which;
    for (size_t k = 0; k < reqs.size(); ++k) {
        const Chi0Request &r = reqs[k];
        if (r.ncols == 0) continue;
        chi0_spec(*r.c, r.omega, r.dv, r.drho, r.ncols, sb, r.c->pc_coef, sp[k], s);
        specs.push_back(&sp[k]);
        which.push_back(k);
    }
    if (specs.empty()) return RPA_OK;
    std::vector<int> sw;
    const int w = run_block(lead, specs, s, nullptr, nullptr, &sw);
    if (status)
        for (size_t q = 0; q < which.size(); ++q) (*status)[which[q]] = sw[q];
    return w;
}

int sternheimer_block(Ctx &c, double omega, const int *orb, int nsys, const double *b, const double *Tc, double *x,
                      std::vector<int> *iters, std::vector<int> *status, cudaStream_t s) {
    const int sb = c.opt.block_cocg;
    BSpec sp;
    sp.c = &c;
    sp.rhs = b;
    sp.Tc = Tc;
    sp.sign = 1.0;
    sp.omega = omega;
    sp.xout = (double2 *)x;
    for (int i = 0; i < nsys;) {
        int e = i + 1;
        while (e < nsys && e - i < sb && orb[e] == orb[i]) ++e;
        sp.groups.push_back(make_group(orb[i], e - i, i, i));
        i = e;
    }
    std::vector<BSpec *> specs{&sp};
    return run_block(c, specs, s, iters, status);
}

}  // namespace rpa

// Internal declarations shared by the translation units of librpa.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "rpa.h"

namespace rpa {

constexpr int kRadius = 6;              // 12th-order centred differences
constexpr int kMaxOmega = 64;
constexpr int kMaxSqOrder = 32;     // largest Gauss spectral quadrature order
constexpr int kMaxBlock = 16;       // largest block of block COCG

// ------------------------------------------------------------------------------------------
// Errors: every internal failure throws rpa::Error; the C entry points catch it and turn it
// into a status code plus a thread-local message.
// ------------------------------------------------------------------------------------------
struct Error {
    rpa_status status;
    std::string msg;
};

[[noreturn]] void fail(rpa_status st, const char *fmt, ...);

// Raise a kernel's dynamic shared-memory limit to the device maximum (once; the value never
// depends on the call, so contexts on different threads cannot lower each other's limit between
// setting it and launching) and fail with RPA_ERR_INVALID if `need` bytes exceed that maximum.
void allow_dynamic_smem(const void *kernel, size_t need);

// Kernel launches issued by the library on this thread (reported in rpa_stats.launches).
extern thread_local long long g_launches;
inline void count_launches(long long n) { g_launches += n; }
void check_cuda(cudaError_t e, const char *what, const char *file, int line);
#define RPA_CUDA(call) ::rpa::check_cuda((call), #call, __FILE__, __LINE__)
#define RPA_LAUNCH(what) ::rpa::check_cuda(cudaGetLastError(), what, __FILE__, __LINE__)

// ------------------------------------------------------------------------------------------
// Device buffer that only grows.
// ------------------------------------------------------------------------------------------
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    void *ensure(size_t need);
    void release();
    template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

// Shifted Hamiltonian stencil: (H + sigma) v = (diag + V + sigma) v + sum_k a_k (six neighbours
// at distance k), with a_k = -w_k / (2 h^2) and diag = 3 a_0.
struct StencilCoef {
    double a[kRadius + 1];
};

// Per-system COCG scalars (one slot of a batch).
struct SysState {
    double rho_re, rho_im;        // r^T r (unconjugated)
    double alpha_re, alpha_im;
    double beta_re, beta_im;
    double ref_norm;              // ||b|| (outer) for the FP64 form; ||r64|| for a mixed inner solve
    double bnorm;                 // ||b||
    double rnorm;                 // latest ||r||
    double shift_re, shift_im;    // sigma = -eps_n + i omega
    int n, j;                     // orbital, column
    int active;                   // inner COCG running
    int outer_active;             // mixed: refinement running
    int iters;                    // inner iterations in the current solve
    int total_iters;              // all inner iterations
    int refines;                  // FP64 residual evaluations
    int status;
};

// Summary of the Sternheimer queues run since the last read-back, accumulated on the device (so
// that a queue needs no host synchronisation) and added to rpa_stats at the next one.
struct QueueStats {
    long long solves, iters, refines, nearb, launches;
    int worst;          // largest per-system status
    int unfinished;     // a queue stopped at its epoch bound with systems left
};

struct BatchCoord;   // rendezvous of rpa_ec_batch's threads (api.cu)

// ------------------------------------------------------------------------------------------
// Context
// ------------------------------------------------------------------------------------------
struct Ctx {
    int nx = 0, ny = 0, nz = 0, ns = 0;
    long long nd = 0;
    double h = 0;
    rpa_options opt{};
    StencilCoef coef{};
    int device = 0;

    // inputs (device copies)
    double *vloc64 = nullptr;
    float *vloc32 = nullptr;
    float *vloc_lo = nullptr;     // V_loc - vloc32 in FP32: V_loc as an FP32 pair
    double *psi64 = nullptr;      // ns x nd (row s = orbital s)
    float *psi32 = nullptr;       // FP32 copy (projection of the mixed form's FP32 residuals)
    std::vector<double> eps;
    double *eps_dev = nullptr;

    // Kronecker Coulomb operator: 1D eigenvectors Q_a (n_a x n_a, row-major Q[i*n+a]) and the
    // summed eigenvalue grid lam = mu_x + mu_y + mu_z (nd).
    double *Q[3] = {nullptr, nullptr, nullptr};
    double *lam = nullptr;
    // Laplacian preconditioner of COCG: the 1D eigenvalues mu_a (FP64), FP32 copies of Q_a and mu_a,
    // and the mean of V_loc
    double *mu[3] = {nullptr, nullptr, nullptr};
    float *Qf[3] = {nullptr, nullptr, nullptr};
    float *muf[3] = {nullptr, nullptr, nullptr};
    double vbar = 0.0;

    // workspaces
    DevBuf cocg_state;            // complex vectors of the systems in flight
    DevBuf cocg_partials;
    DevBuf sys_state;             // SysState[slots]
    DevBuf rhs;                   // real right-hand sides of the systems in flight
    DevBuf pc_coef;               // P_c coefficients
    DevBuf coul_tmp;              // Kronecker scratch
    DevBuf blockA, blockB, blockC, blockD;   // N_d x N_r blocks for rpa_ec / apply
    DevBuf small;                 // N_r x N_r matrices and scalars
    DevBuf slot_idx;              // (n, j) of the slots
    DevBuf proj_buf;              // occupied-space projection of finished solutions
    DevBuf coef_buf;              // per-column coefficients of the gradient pass
    DevBuf blockE;                // subspace of the previous iteration (gradient)
    DevBuf dense_scratch;         // split-K partial sums
    SysState *h_state = nullptr;  // pinned host mirror of the slot states
    size_t h_state_cap = 0;
    int *h_count = nullptr;       // pinned host counter
    int *d_tc_err = nullptr;      // set by a tensor-core contraction that gave up waiting on its MMAs
    QueueStats *d_qstats = nullptr;   // device accumulator of queue statistics
    int *d_loop = nullptr;            // epoch counter of a device-driven queue
    char *h_rb = nullptr;             // pinned read-back block (Ritz values, scalars, statistics)
    long long host_syncs = 0;         // host synchronisations of the current call
    // events of the last chi0 application (Coulomb / COCG phase times, read at the next sync)
    cudaEvent_t ev_apply[4] = {nullptr, nullptr, nullptr, nullptr};
    bool apply_timed = false;

    // per-call statistics
    rpa_stats stats{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // profiling (rpa_options.profile): event pool and per-kernel point counters on the device
    std::vector<cudaEvent_t> ev_pool;
    unsigned long long *d_prof_points = nullptr;   // RPA_PROF_SLOTS counters
    // rpa_ec_batch: the rendezvous this context's chi0 applications go to (nullptr otherwise)
    BatchCoord *coord = nullptr;
    // CUDA graphs: epochs of COCG iterations are captured on a private stream and replayed
    bool use_graphs = true;
    cudaStream_t cap_stream = nullptr;

    ~Ctx();
};

// ------------------------------------------------------------------------------------------
// Operations (each enqueues work on `stream`)
// ------------------------------------------------------------------------------------------
// Kronecker Coulomb operator nu^power on ncols columns.
void coulomb_apply(Ctx &c, double power, const double *in, double *out, int ncols, cudaStream_t s,
                   bool tensor = false);
// Whether the dense contractions of this context run on the tensor cores (rpa_options.contractions):
// the P_c coefficients and C = V^T R, and the Kronecker transforms of nu^1/2.
inline bool use_tensor_cores(const Ctx &c) {
    return c.opt.contractions >= 2 || (c.opt.contractions == 0 && c.opt.prec == RPA_MIXED);
}
inline bool use_tensor_cores_kronecker(const Ctx &c) {
    return c.opt.contractions == 2 || (c.opt.contractions == 0 && c.opt.prec == RPA_MIXED);
}
// Fails with RPA_ERR_CUDA if a tensor-core contraction reported a timed-out wait (synchronises s).
void check_tensor_core_status(Ctx &c, cudaStream_t s);
void coulomb_setup(Ctx &c);
// Same operator with its scratch in the library's fixed device array (no allocation).
void coulomb_apply_noalloc(Ctx &c, double power, const double *in, double *out, int ncols, cudaStream_t s);

// Synchronise s and count it in the call's statistics.
void sync_stream(Ctx &c, cudaStream_t s);
// After a synchronisation: add the device queue statistics read back into h (pinned) to the
// call's statistics and return the worst per-system status seen.
int add_queue_stats(Ctx &c, const QueueStats &h);

// Sternheimer solves for the systems given by (n, j) pairs with real right-hand sides b
// (nsys x nd, row per system) -> complex solutions x (nsys x nd interleaved, FP64).
// Returns the worst per-system status; fills per-system iterations/status (host vectors).
int sternheimer_batch(Ctx &c, double omega, const int *orb, int nsys, const double *b, double *x,
                      std::vector<int> *iters, std::vector<int> *status, cudaStream_t s);

// chi0 on ncols real columns: drho = (4/h^3) Re sum_n u_n x_n with the projected right-hand
// sides -P_c(u_n dV_j).  Returns the worst status.
int chi0_apply(Ctx &c, double omega, const double *dv, double *drho, int ncols, cudaStream_t s);

// grad += sum_j coef[j] (4/h^3) Re sum_n (P_c x_{n,j})^2 for the projected Sternheimer solutions of
// dV_j (ncols rows of dv); coef: ncols doubles on the device.  Returns the worst status known on
// the host (a device-driven queue reports through the device statistics).
int response_square(Ctx &c, double omega, const double *dv, const double *coef, double *grad, int ncols,
                    cudaStream_t s);

// Host symmetric eigendecomposition (cyclic Jacobi): A = Q diag(w) Q^T, Q[i*n+a] = component i of
// eigenvector a; w ascending is not guaranteed.  (The 1D matrices of the Coulomb operator.)
void jacobi_eigh(std::vector<double> A, int n, std::vector<double> &w, std::vector<double> &Q);
// The same on the device (parallel cyclic Jacobi, one block; A destroyed); work: 3 (n + 1) doubles.
void jacobi_eigh_device(double *A, int n, double *Q, double *w, double *work, cudaStream_t s);
// S = Q^T and coef[i] = weight * g'(w_i), g'(x) = -x / (1 - x) (the adjoint's Ritz rotation, device).
void ritz_rotation(const double *Q, const double *w, int n, double weight, double *S, double *coef, cudaStream_t s);

// Whether the fused single-pass COCG kernel applies to this context's grid (a whole xy plane fits
// its shared-memory ring); the mixed form then uses it by default.
bool fused_kernel_applies(const Ctx &c, bool warp_specialised = false, bool cluster = false);

// Block COCG (block_cocg.cu) for systems grouped by orbital: chi0 on ncols columns (as chi0_apply)
// and the Sternheimer solves of rpa_sternheimer_solve (as sternheimer_batch; Tc: P_c coefficients
// of the rows of b, or nullptr).
int chi0_apply_block(Ctx &c, double omega, const double *dv, double *drho, int ncols, cudaStream_t s);
int sternheimer_block(Ctx &c, double omega, const int *orb, int nsys, const double *b, const double *Tc,
                      double *x, std::vector<int> *iters, std::vector<int> *status, cudaStream_t s);
// One context's chi0 application within a batch.
struct Chi0Request {
    Ctx *c;
    double omega;
    const double *dv;
    double *drho;
    int ncols;
};
// chi0 for several contexts (distinct, on one device, with equal precision and COCG settings) in
// one set of launches: the block COCG kernels over all their groups at once, with block size
// max(1, block_cocg) and the iteration settings and workspaces of the first context.  The
// statistics of each context get its own systems.
int chi0_apply_batch(const std::vector<Chi0Request> &reqs, cudaStream_t s, std::vector<int> *status = nullptr);
// While a context is attached to a BatchCoord, its chi0 applications are posted there and run
// together with the other contexts' (batch_chi0).
int batch_chi0(Ctx &c, double omega, const double *dv, double *drho, int ncols, cudaStream_t s);

// Same as sternheimer_batch, with b replaced by P_c b first.
int sternheimer_batch_projected(Ctx &c, double omega, const int *orb, int nsys, const double *b, double *x,
                                std::vector<int> *iters, std::vector<int> *status, cudaStream_t s);

// Dense FP64 helpers (dense.cu)
// G (na x nb, row-major) = A B^T with A: na rows of length len, B: nb rows of length len.
void gram(const double *A, int na, const double *B, int nb, long long len, double *G, cudaStream_t s,
          DevBuf &scratch);
// Y (nc rows) = S X, S: nc x nk row-major (device), X: nk rows of length len.
void combine_rows(const double *S, int nc, int nk, const double *X, long long len, double *Y,
                  cudaStream_t s);
// Cholesky of the n x n SPD matrix M (row-major, device) in place -> lower L; returns via
// *dev_info (0 ok, k+1 = failed pivot k).
void cholesky(double *M, int n, int *dev_info, cudaStream_t s);
// Linv = L^{-1} (lower), n x n row-major.
void tri_inverse(const double *L, int n, double *Linv, cudaStream_t s);
// Ascending eigenvalues of the symmetric n x n matrix C (row-major, destroyed), then
// e_out = weight * sum_i [log1p(-lam_i) + lam_i].
// e_out = weight * Tr g(C) by Gauss spectral quadrature of order n_o (part: n doubles of scratch)
void sq_trace(const double *C, int n, int n_o, double *part, double weight, double *e_out, cudaStream_t s);
void sym_eigvals(double *C, int n, double *lam, double *work, double weight, double *e_out,
                 cudaStream_t s);
void symmetrize(double *C, int n, cudaStream_t s);

// D (M x N, row-major) = sum_k A(m, k) B(n, k) with A(m, k) = A[m a_m + k a_k] and B(n, k) =
// B[n b_n + k b_k], on the tensor cores (tcgen05) as six products of BF16 splits accumulated in
// FP32 (tc_gemm.cu).  *err_dev is set to 1 if the kernel gave up waiting on its MMAs.
void tc_gemm(const double *A, long long a_m, long long a_k, const double *B, long long b_n, long long b_k, int M,
             int N, long long K, double *D, cudaStream_t s, DevBuf &scratch, int *err_dev);
// Batched form: for z < batch, D_z[m d_m + n d_n] = sum_k A_z(m, k) B_z(n, k), with the operands and
// the output of member z offset by z a_z, z b_z, z d_z elements; optionally every output element e
// (counted from D) is multiplied by scale[e % scale_n].
void tc_gemm_batched(const double *A, long long a_m, long long a_k, long long a_z, const double *B, long long b_n,
                     long long b_k, long long b_z, int M, int N, int K, double *D, long long d_m, long long d_n,
                     long long d_z, int batch, const double *scale, long long scale_n, cudaStream_t s, int *err_dev);

// Profiling helpers: register a kernel name in the stats table (returns its slot) and add
// launches/time/points/bytes to it.
int prof_slot(Ctx &c, const char *name);

}  // namespace rpa

struct rpa_ctx {
    rpa::Ctx impl;
};

// Dense contractions of the subspace step on the 5th-generation tensor cores (tcgen05, sm_103a):
//
//     D[m][n] = sum_k A(m, k) B(n, k),   A(m, k) = A[m * a_m + k * a_k],  B(n, k) = B[n * b_n + k * b_k]
//
// for FP64 operands, as products of BF16 splits accumulated in FP32.  Every operand value is
// split as x = hi + mid + lo, hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid) (the
// remainders are formed exactly), and the six products that reach the FP32 level,
//     hi.hi + hi.mid + mid.hi + hi.lo + lo.hi + mid.mid,
// are accumulated by tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulator in tensor memory).
// Each product of two BF16 numbers is exact in FP32, so a term carries ~24 significant bits.
//
// Used for the projection C = V^T R of the Rayleigh-Ritz step (Algorithm 1) and the P_c
// coefficients T_{k,(n,j)} = u_k . (u_n (.) nu^1/2 v_j) of the Sternheimer right-hand sides
// (Eqs. 7-9) in the mixed-precision form; the plain FP64 form keeps the FP64 kernels.
//
// Accumulation.  The tensor cores add the products of one MMA to the FP32 accumulator with a
// relative error of up to ~2^-23 of the accumulator per instruction (measured: ~5e-6 relative
// after a few hundred chained MMAs), so chains are kept short: the hi.hi products accumulate in
// one tensor-memory tile and the five smaller cross products in a second, each over one k chunk
// (4 and 20 MMAs), and after every chunk both tiles are read back and added in FP64 registers.
//
// Blocking.  A block computes one 128 x kTcN tile of D over one range of k (split-K, blockIdx.z) or
// for one member of a batch (blockIdx.z with the batch strides); the range is walked in chunks of
// kTcK.  Per chunk all threads read the FP64 operand tiles (coalesced along whichever index is
// contiguous), split them and store the BF16 pieces into shared memory in the canonical K-major
// layout without swizzle (8-row x 16-byte core matrices, 128 bytes each); one thread then issues
// 4 (k slices of 16) x 6 (products) MMAs and commits them to an mbarrier, which every thread waits
// on before the tiles are read back (tcgen05.ld) and the shared tiles rewritten.  The FP64 tile
// goes to the output (batched) or to a split-K partial; a second kernel adds the partials in a
// fixed order (deterministic).
//
// Bounded waits: every wait on the mbarrier gives up after ~1 s of clock cycles, sets the error
// flag, waits (again bounded) for the block's MMAs, frees the tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "internal.cuh"

namespace rpa {

namespace {

constexpr int kTcM = 128;                // tile rows (MMA M)
constexpr int kTcN = 64;                 // tile columns (MMA N)
constexpr int kTcK = 64;                 // k chunk staged per round
constexpr int kTcThreads = 256;
constexpr int kTcSplits = 3;             // hi, mid, lo
constexpr uint32_t kTcCoreBytes = 128;   // one 8 x 16-byte core matrix
constexpr uint32_t kTcSbo = (kTcK / 8) * kTcCoreBytes;            // next 8-row group
constexpr uint32_t kTcLbo = kTcCoreBytes;                         // next 8 k values
constexpr uint32_t kTcTileA = kTcM * kTcK * 2;                    // bytes of one BF16 A tile
constexpr uint32_t kTcTileB = kTcN * kTcK * 2;
constexpr uint32_t kTcSmem = kTcSplits * (kTcTileA + kTcTileB) + 64;
constexpr long long kTcWaitCycles = 2000000000LL;                 // ~1 s at 2 GHz

struct TcArgs {
    const double *A;
    const double *B;
    long long a_m, a_k, b_n, b_k;        // element strides
    int M, N;                            // output size
    long long K;
    long long kchunk;                    // k range per split (multiple of kTcK); K for a batch
    double *part;                        // split-K: [splits][M][N]; batch: the output D
    long long d_m, d_n;                  // output strides (batch); split-K partials are [M][N]
    long long a_z, b_z, d_z;             // batch strides (0: blockIdx.z splits k)
    const double *scale;                 // batch only: D[e] *= scale[e % scale_n] (nullptr = none)
    long long scale_n;
    int *err;                            // set on a timed-out wait
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major canonical layout without swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kTcLbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kTcSbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;              // descriptor version of the 5th-generation tensor cores
    return d;                            // base offset 0, swizzle mode 0 (none)
}

// Instruction descriptor of kind::f16: D in FP32, A and B in BF16, both K-major, M x N.
constexpr uint32_t tc_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Byte offset of element (row, k) of a K-major tile.
__device__ __forceinline__ uint32_t tc_off(int row, int k) {
    return (uint32_t)(row >> 3) * kTcSbo + (uint32_t)(k >> 3) * kTcCoreBytes + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ void split3(double x, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
    const float f = (float)x;                       // x = f + e exactly enough (e below 2^-48 |x|)
    const float e = (float)(x - (double)f);
    h = __float2bfloat16_rn(f);
    const float r1 = f - __bfloat162float(h);       // exact
    m = __float2bfloat16_rn(r1);
    const float r2 = (r1 - __bfloat162float(m)) + e;
    l = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kTcWaitCycles) return false;
    }
}

__global__ void __launch_bounds__(kTcThreads) k_tc_gemm(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char *tA = tsm;                                       // [3][kTcTileA]
    unsigned char *tB = tsm + kTcSplits * kTcTileA;                // [3][kTcTileB]
    uint64_t *bar = reinterpret_cast<uint64_t *>(tsm + kTcSplits * (kTcTileA + kTcTileB));
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * kTcN;
    const bool batch = a.a_z != 0 || a.b_z != 0 || a.d_z != 0;
    const double *const Ab = a.A + (batch ? (long long)blockIdx.z * a.a_z : 0);
    const double *const Bb = a.B + (batch ? (long long)blockIdx.z * a.b_z : 0);
    const long long k0 = batch ? 0 : (long long)blockIdx.z * a.kchunk;
    const long long k1 = min(a.K, k0 + a.kchunk);
    const uint32_t bar_addr = smem_u32(bar);
    constexpr uint32_t kCols = 2 * kTcN;                          // hi.hi tile, cross-product tile

    if (tid == 0) {
        abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_addr) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const bool a_kfast = a.a_k == 1, b_kfast = a.b_k == 1;
    // epilogue mapping: warp w reads tile rows 32 (w % 4) .. +31 (its tensor-memory lanes) and
    // columns 32 (w / 4) .. +31
    const int lane_base = 32 * (warp & 3), col0 = 32 * (warp >> 2);
    const uint32_t t_hh = tmem + ((uint32_t)lane_base << 16) + (uint32_t)col0;
    const uint32_t t_x = t_hh + kTcN;
    double acc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = 0.0;

    uint32_t phase = 0;
    bool ok = true, pending = false;
    for (long long kb = k0; kb < k1; kb += kTcK) {
        // operand tiles: FP64 -> three BF16 pieces, K-major core matrices
        for (int e = tid; e < kTcM * kTcK; e += kTcThreads) {
            const int row = a_kfast ? e / kTcK : e % kTcM;
            const int kk = a_kfast ? e % kTcK : e / kTcM;
            const int m = m0 + row;
            const long long k = kb + kk;
            const double x = (m < a.M && k < k1) ? Ab[(long long)m * a.a_m + k * a.a_k] : 0.0;
            __nv_bfloat16 h, md, l;
            split3(x, h, md, l);
            const uint32_t o = tc_off(row, kk);
            *reinterpret_cast<__nv_bfloat16 *>(tA + o) = h;
            *reinterpret_cast<__nv_bfloat16 *>(tA + kTcTileA + o) = md;
            *reinterpret_cast<__nv_bfloat16 *>(tA + 2 * kTcTileA + o) = l;
        }
        for (int e = tid; e < kTcN * kTcK; e += kTcThreads) {
            const int row = b_kfast ? e / kTcK : e % kTcN;
            const int kk = b_kfast ? e % kTcK : e / kTcN;
            const int n = n0 + row;
            const long long k = kb + kk;
            const double x = (n < a.N && k < k1) ? Bb[(long long)n * a.b_n + k * a.b_k] : 0.0;
            __nv_bfloat16 h, md, l;
            split3(x, h, md, l);
            const uint32_t o = tc_off(row, kk);
            *reinterpret_cast<__nv_bfloat16 *>(tB + o) = h;
            *reinterpret_cast<__nv_bfloat16 *>(tB + kTcTileB + o) = md;
            *reinterpret_cast<__nv_bfloat16 *>(tB + 2 * kTcTileB + o) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy stores -> tensor core
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            constexpr uint32_t idesc = tc_idesc(kTcM, kTcN);
            // (A piece, B piece) of the six products; product 0 (hi.hi) goes to its own tile
            const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
#pragma unroll
            for (int t = 0; t < kTcK / 16; ++t)
#pragma unroll
                for (int pr = 0; pr < 6; ++pr) {
                    const uint64_t da = tc_desc(smem_u32(tA + pa[pr] * kTcTileA) + t * 2 * kTcCoreBytes);
                    const uint64_t db = tc_desc(smem_u32(tB + pb[pr] * kTcTileB) + t * 2 * kTcCoreBytes);
                    const uint32_t d = pr == 0 ? tmem : tmem + kTcN;
                    const uint32_t accum = (t > 0 || pr > 1) ? 1u : 0u;     // each chunk starts both tiles afresh
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                        "l"(da), "l"(db), "r"(idesc), "r"(accum)
                        : "memory");
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_addr)
                         : "memory");
        }
        pending = true;
        if (!mbar_wait(bar_addr, phase)) {
            ok = false;
            atomicExch(&abort_flag, 1);
        }
        phase ^= 1u;
        __syncthreads();
        if (abort_flag) break;
        pending = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // read both tiles back (16 columns at a time) and add them in FP64
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t r[16], x[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(t_hh + 16 * h)
                : "memory");
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]), "=r"(x[7]),
                  "=r"(x[8]), "=r"(x[9]), "=r"(x[10]), "=r"(x[11]), "=r"(x[12]), "=r"(x[13]), "=r"(x[14]), "=r"(x[15])
                : "r"(t_x + 16 * h)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int c = 0; c < 16; ++c)
                acc[16 * h + c] += (double)__uint_as_float(r[c]) + (double)__uint_as_float(x[c]);
        }
        // the next chunk's MMAs rewrite tensor memory and its loads the shared tiles
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (ok && !abort_flag) {
        const int m = m0 + lane_base + (tid & 31);
        if (m < a.M) {
            if (batch) {
                double *out = a.part + (long long)blockIdx.z * a.d_z + (long long)m * a.d_m;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int n = n0 + col0 + c;
                    if (n < a.N) {
                        const long long off = (long long)blockIdx.z * a.d_z + (long long)m * a.d_m + (long long)n * a.d_n;
                        out[(long long)n * a.d_n] = a.scale ? acc[c] * a.scale[off % a.scale_n] : acc[c];
                    }
                }
            } else {
                double *out = a.part + ((long long)blockIdx.z * a.M + m) * a.N;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int n = n0 + col0 + c;
                    if (n < a.N) out[n] = acc[c];
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(a.err, 1);
        if (pending) (void)mbar_wait(bar_addr, phase ^ 1u);          // let the block's MMAs finish
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

__global__ void k_tc_sum_splits(const double *__restrict__ part, int splits, long long n, double *__restrict__ D) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < splits; ++z) s += part[(long long)z * n + e];
        D[e] = s;
    }
}

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

void tc_gemm(const double *A, long long a_m, long long a_k, const double *B, long long b_n, long long b_k, int M,
             int N, long long K, double *D, cudaStream_t s, DevBuf &scratch, int *err_dev) {
    const int tm = (int)cdiv(M, kTcM), tn = (int)cdiv(N, kTcN);
    int dev = 0, sms = 0;
    RPA_CUDA(cudaGetDevice(&dev));
    RPA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // split K so that the grid covers the SMs about three times, with at least two chunks per split
    long long splits = std::max(1LL, std::min<long long>(K / (2 * kTcK), (3LL * sms + tm * tn - 1) / (tm * tn)));
    const long long kchunk = ((K + splits - 1) / splits + kTcK - 1) / kTcK * kTcK;
    splits = std::max(1LL, (K + kchunk - 1) / kchunk);
    double *part = (double *)scratch.ensure(sizeof(double) * (size_t)splits * M * N);
    TcArgs a{};
    a.A = A; a.B = B; a.a_m = a_m; a.a_k = a_k; a.b_n = b_n; a.b_k = b_k;
    a.M = M; a.N = N; a.K = K; a.kchunk = kchunk; a.part = part; a.err = err_dev;
    allow_dynamic_smem((const void *)k_tc_gemm, kTcSmem);
    k_tc_gemm<<<dim3(tm, tn, (unsigned)splits), kTcThreads, kTcSmem, s>>>(a);
    const long long n = (long long)M * N;
    k_tc_sum_splits<<<std::min<unsigned>(cdiv(n, 256), 4096u), 256, 0, s>>>(part, (int)splits, n, D);
    RPA_LAUNCH("tensor-core contraction");
    count_launches(2);
}

void tc_gemm_batched(const double *A, long long a_m, long long a_k, long long a_z, const double *B, long long b_n,
                     long long b_k, long long b_z, int M, int N, int K, double *D, long long d_m, long long d_n,
                     long long d_z, int batch, const double *scale, long long scale_n, cudaStream_t s, int *err_dev) {
    if (batch <= 0 || M <= 0 || N <= 0) return;
    const int tm = (int)cdiv(M, kTcM), tn = (int)cdiv(N, kTcN);
    if (batch > 65535) fail(RPA_ERR_INVALID, "tensor-core contraction: batch of %d exceeds the grid limit", batch);
    TcArgs a{};
    a.A = A; a.B = B; a.a_m = a_m; a.a_k = a_k; a.b_n = b_n; a.b_k = b_k;
    a.M = M; a.N = N; a.K = K; a.kchunk = K; a.part = D; a.d_m = d_m; a.d_n = d_n;
    // a zero stride would read as "split K": a batch always has a nonzero output stride
    a.a_z = a_z; a.b_z = b_z; a.d_z = d_z != 0 ? d_z : 1;
    a.scale = scale; a.scale_n = scale_n > 0 ? scale_n : 1; a.err = err_dev;
    allow_dynamic_smem((const void *)k_tc_gemm, kTcSmem);
    k_tc_gemm<<<dim3(tm, tn, (unsigned)batch), kTcThreads, kTcSmem, s>>>(a);
    RPA_LAUNCH("tensor-core contraction (batched)");
    count_launches(1);
}

}  // namespace rpa

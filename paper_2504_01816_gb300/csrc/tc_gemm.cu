// Dense contractions of the subspace step on the 5th-generation tensor cores (tcgen05, sm_103a):
//
//     D[m][n] = sum_k A(m, k) B(n, k),   A(m, k) = A[m * a_m + k * a_k],  B(n, k) = B[n * b_n + k * b_k]
//
// for FP64 operands, as BF16 tensor-core products that are exact.  The scheme is the error-free
// splitting of Ozaki, Ogita and Oishi (error-free transformation of matrix products into sums of
// products of low-precision pieces) with per-chunk power-of-two scaling:
//
//   * k is walked in chunks of kTcK = 64.  Within a chunk every row m of A gets the power of two
//     s_m = 2^(e_m + 1) above its largest |A(m, k)| (e_m its binary exponent), every row n of B
//     likewise s_n, so that |A(m, k) / s_m| < 1.
//   * |x| = |A(m, k)| / s_m * 2^7 <= 128 is rounded to 2^-24 and cut into four balanced integer
//     digits, read off the bits of the FP64 significand with integer instructions:
//       |x| = a1 + 2^-8 a2 + 2^-16 a3 + 2^-24 a4 + r,  0 <= a1 <= 128, |a2..a4| <= 128, |r| <= 2^-25,
//     each times the sign of A(m, k) and exactly representable in BF16 (8 significant bits).
//   * Products a_i b_j are integers of magnitude at most 2^14, so over one chunk (64 values of k)
//     every partial sum the tensor core forms -- inside one MMA of 16 k values, or accumulated over
//     the chunk's four MMAs -- is an integer below 2^24 (the largest tile, L3, sums at most 256
//     products: below 2^22) and therefore exact in its FP32 accumulator, whatever the rounding of
//     the hardware's additions.  The ten products of weight 2^0 .. 2^-24 go to four tensor-memory tiles by weight:
//     L0 = a1.b1; L1 = a1.b2 + a2.b1; L2 = a1.b3 + a3.b1 + a2.b2; L3 = a1.b4 + a4.b1 + a2.b3 + a3.b2.
//   * After each chunk the tiles are read back (tcgen05.ld), combined exactly in 64-bit integers
//     as 2^24 L0 + 2^16 L1 + 2^8 L2 + L3, and the chunk's contribution s_m s_n 2^-38 times that
//     integer is added in FP64 (one conversion and one multiply-add per output and chunk).
// The only errors are the truncated remainders and the neglected products (weights 2^-31 and
// below, relative to s_m s_n) and the FP64 additions: about 1e-9 of the chunk-row maxima.
//
// Used for the projection C = V^T R of the Rayleigh-Ritz step (Algorithm 1), the P_c coefficients
// T_{k,(n,j)} = u_k . (u_n (.) nu^1/2 v_j) of the Sternheimer right-hand sides (Eqs. 7-9), and the
// per-axis transforms of the Kronecker-product Coulomb operator (Eq. 5), in the mixed-precision form.
//
// Blocking.  A block computes one 128 x kTcN tile of D over one range of k (split-K, blockIdx.z) or
// for one member of a batch (blockIdx.z with the batch strides).  Per chunk all threads read the
// FP64 operand tiles twice (coalesced along whichever index is contiguous): first for the row
// exponents (shared-memory atomicMax), then to cut the pieces, which go to shared memory in the
// canonical K-major layout without swizzle (8-row x 16-byte core matrices, 128 bytes each).  One
// thread issues 4 (k slices of 16) x 10 (products) MMAs and commits them to an mbarrier, which every
// thread waits on before the tiles are read back and the shared tiles rewritten.  The FP64 tile
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
constexpr int kTcPieces = 4;             // integer pieces per operand value
constexpr int kTcLevels = 4;             // product weights 2^0, 2^-8, 2^-16, 2^-24
constexpr uint32_t kTcCoreBytes = 128;   // one 8 x 16-byte core matrix
constexpr uint32_t kTcSbo = (kTcK / 8) * kTcCoreBytes;            // next 8-row group
constexpr uint32_t kTcLbo = kTcCoreBytes;                         // next 8 k values
constexpr uint32_t kTcTileA = kTcM * kTcK * 2;                    // bytes of one BF16 A tile
constexpr uint32_t kTcTileB = kTcN * kTcK * 2;
constexpr uint32_t kTcSmem = kTcPieces * (kTcTileA + kTcTileB) + 64;
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

// Biased binary exponent field of |x| (0 for zero).
__device__ __forceinline__ int exp_field(double x) { return (__double2hiint(x) >> 20) & 0x7FF; }

// The four BF16 pieces of x for the row exponent field e (see above), from the significand bits:
// I = round(|x| / 2^(e - 1022) * 2^31) = round(significand / 2^(22 + e - e_x)), then balanced base-256
// digits I = a1 2^24 + a2 2^16 + a3 2^8 + a4 with a2..a4 in [-128, 127] and 0 <= a1 <= 128 (balanced
// digits keep the neglected products unbiased).  An integer of magnitude <= 256 converts to FP32
// exactly with no bits below the top 8 of its significand, so the upper half of its FP32 pattern
// is the same value in BF16.
__device__ __forceinline__ void cut4(double x, int e, __nv_bfloat16 (&p)[4]) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    const int sh = 22 + e - ex;
    long long I = 0;
    if (ex > 0 && sh < 64)
        I = (long long)((((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) + (1ull << (sh - 1))) >> sh);
    int dg[4];
#pragma unroll
    for (int i = 3; i >= 1; --i) {
        dg[i] = (int)(((I + 128) & 255) - 128);
        I = (I - dg[i]) >> 8;
    }
    dg[0] = (int)I;
    const unsigned short sx = (unsigned short)((bits >> 48) & 0x8000u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const unsigned int v = (unsigned int)abs(dg[i]);
        const unsigned short h = (unsigned short)(__float_as_uint(__uint2float_rn(v)) >> 16);
        const unsigned short sg = dg[i] < 0 ? (unsigned short)(sx ^ 0x8000u) : sx;
        p[i] = __ushort_as_bfloat16(v ? (unsigned short)(h | sg) : (unsigned short)0);
    }
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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

__global__ void __launch_bounds__(kTcThreads, 2) k_tc_gemm(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char *tA = tsm;                                       // [4][kTcTileA]
    unsigned char *tB = tsm + kTcPieces * kTcTileA;                // [4][kTcTileB]
    uint64_t *bar = reinterpret_cast<uint64_t *>(tsm + kTcPieces * (kTcTileA + kTcTileB));
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    __shared__ int abort_flag;
    __shared__ int expA[kTcM], expB[kTcN];                         // row exponents of the chunk
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * kTcN;
    const bool batch = a.a_z != 0 || a.b_z != 0 || a.d_z != 0;
    const double *const Ab = a.A + (batch ? (long long)blockIdx.z * a.a_z : 0);
    const double *const Bb = a.B + (batch ? (long long)blockIdx.z * a.b_z : 0);
    const long long k0 = batch ? 0 : (long long)blockIdx.z * a.kchunk;
    const long long k1 = min(a.K, k0 + a.kchunk);
    const uint32_t bar_addr = smem_u32(bar);
    constexpr uint32_t kCols = kTcLevels * kTcN;                  // one accumulator tile per weight

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
    const int my_row = lane_base + (tid & 31);
    const uint32_t t_base = tmem + ((uint32_t)lane_base << 16) + (uint32_t)col0;
    double acc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = 0.0;

    uint32_t phase = 0;
    bool ok = true, pending = false;
    for (long long kb = k0; kb < k1; kb += kTcK) {
        // 1. row exponents of the chunk
        for (int e = tid; e < kTcM; e += kTcThreads) expA[e] = 0;
        for (int e = tid; e < kTcN; e += kTcThreads) expB[e] = 0;
        __syncthreads();
        for (int e = tid; e < kTcM * kTcK; e += kTcThreads) {
            const int row = a_kfast ? e / kTcK : e % kTcM;
            const int kk = a_kfast ? e % kTcK : e / kTcM;
            const int m = m0 + row;
            const long long k = kb + kk;
            if (m < a.M && k < k1) atomicMax(&expA[row], exp_field(Ab[(long long)m * a.a_m + k * a.a_k]));
        }
        for (int e = tid; e < kTcN * kTcK; e += kTcThreads) {
            const int row = b_kfast ? e / kTcK : e % kTcN;
            const int kk = b_kfast ? e % kTcK : e / kTcN;
            const int n = n0 + row;
            const long long k = kb + kk;
            if (n < a.N && k < k1) atomicMax(&expB[row], exp_field(Bb[(long long)n * a.b_n + k * a.b_k]));
        }
        __syncthreads();
        // 2. integer pieces into the K-major core-matrix tiles
        for (int e = tid; e < kTcM * kTcK; e += kTcThreads) {
            const int row = a_kfast ? e / kTcK : e % kTcM;
            const int kk = a_kfast ? e % kTcK : e / kTcM;
            const int m = m0 + row;
            const long long k = kb + kk;
            const double x = (m < a.M && k < k1) ? Ab[(long long)m * a.a_m + k * a.a_k] : 0.0;
            __nv_bfloat16 pc[4];
            cut4(x, expA[row], pc);
            const uint32_t o = tc_off(row, kk);
#pragma unroll
            for (int i = 0; i < kTcPieces; ++i) *reinterpret_cast<__nv_bfloat16 *>(tA + i * kTcTileA + o) = pc[i];
        }
        for (int e = tid; e < kTcN * kTcK; e += kTcThreads) {
            const int row = b_kfast ? e / kTcK : e % kTcN;
            const int kk = b_kfast ? e % kTcK : e / kTcN;
            const int n = n0 + row;
            const long long k = kb + kk;
            const double x = (n < a.N && k < k1) ? Bb[(long long)n * a.b_n + k * a.b_k] : 0.0;
            __nv_bfloat16 pc[4];
            cut4(x, expB[row], pc);
            const uint32_t o = tc_off(row, kk);
#pragma unroll
            for (int i = 0; i < kTcPieces; ++i) *reinterpret_cast<__nv_bfloat16 *>(tB + i * kTcTileB + o) = pc[i];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy stores -> tensor core
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            constexpr uint32_t idesc = tc_idesc(kTcM, kTcN);
            // (A piece, B piece, weight level) of the ten products a_i b_j with i + j <= 5
            constexpr int np = 10;
            const int pa[np] = {0, 0, 1, 0, 2, 1, 0, 3, 1, 2};
            const int pb[np] = {0, 1, 0, 2, 0, 1, 3, 0, 2, 1};
            const int lv[np] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3};
#pragma unroll
            for (int t = 0; t < kTcK / 16; ++t)
#pragma unroll
                for (int pr = 0; pr < np; ++pr) {
                    const uint64_t da = tc_desc(smem_u32(tA + pa[pr] * kTcTileA) + t * 2 * kTcCoreBytes);
                    const uint64_t db = tc_desc(smem_u32(tB + pb[pr] * kTcTileB) + t * 2 * kTcCoreBytes);
                    const uint32_t d = tmem + (uint32_t)(lv[pr] * kTcN);
                    // each chunk starts every level's tile afresh with its first product
                    const bool first = t == 0 && (pr == 0 || pr == 1 || pr == 3 || pr == 6);
                    const uint32_t accum = first ? 0u : 1u;
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
        // 3. read the four weight tiles back (8 columns at a time) and add the chunk in FP64
        const int ea = expA[my_row];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint32_t l0[8], l1[8], l2[8], l3[8];
            tmem_ld8(t_base + 8 * h, l0);
            tmem_ld8(t_base + kTcN + 8 * h, l1);
            tmem_ld8(t_base + 2 * kTcN + 8 * h, l2);
            tmem_ld8(t_base + 3 * kTcN + 8 * h, l3);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int eb = expB[col0 + 8 * h + c];
                // the tiles hold integers below 2^24: exact in int64 as 2^24 L0 + 2^16 L1 + 2^8 L2 + L3
                const long long v = ((long long)__float2int_rn(__uint_as_float(l0[c])) << 24) +
                                    ((long long)__float2int_rn(__uint_as_float(l1[c])) << 16) +
                                    ((long long)__float2int_rn(__uint_as_float(l2[c])) << 8) +
                                    (long long)__float2int_rn(__uint_as_float(l3[c]));
                // s_m s_n 2^-38 = 2^(ea - 1022 + eb - 1022 - 38); zero rows have exponent field 0
                // (a scale below the normal range -- rows of magnitude ~1e-150 -- counts as zero)
                const double sc = (ea == 0 || eb == 0 || ea + eb < 1060) ? 0.0
                                                                          : __hiloint2double((ea + eb - 1059) << 20, 0);
                acc[8 * h + c] = fma(sc, (double)v, acc[8 * h + c]);
            }
        }
        // the next chunk's MMAs rewrite tensor memory and its loads the shared tiles and exponents
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (ok && !abort_flag) {
        const int m = m0 + my_row;
        if (m < a.M) {
            if (batch) {
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int n = n0 + col0 + c;
                    if (n < a.N) {
                        const long long off = (long long)blockIdx.z * a.d_z + (long long)m * a.d_m + (long long)n * a.d_n;
                        a.part[off] = a.scale ? acc[c] * a.scale[off % a.scale_n] : acc[c];
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

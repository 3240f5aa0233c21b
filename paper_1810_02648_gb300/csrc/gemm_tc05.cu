// BF16 GEMM with FP32 accumulation on the fifth-generation tensor cores
// (tcgen05.mma, kind::f16, one CTA): the warm-start network's contractions.
//
// C[M x N] = op(A)[M x K] op(B)[K x N]; op(A)(m, k) = A[m lda + k], or
// A[k lda + m] when AT; op(B)(k, n) = B[k ldb + n], or B[n ldb + k] when BT.
// A CTA of 128 threads computes a 128 x TN tile (TN a multiple of 16, at most
// 256) over its K range (long K is split over CTAs into workspace slices that
// a second kernel adds in a fixed order): per K chunk of 64 the threads copy
// op(A) and op(B), 16 bytes at a time, into shared memory
// in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core
// matrix, zero-padded at every edge), one thread issues four 128 x TN x 16
// MMAs into a tensor-memory accumulator of TN columns and commits them to an
// mbarrier, and all threads wait (bounded) before the next chunk reuses the
// tiles.  The epilogue reads the accumulator with tcgen05.ld (warp w reads
// rows 32 w .. 32 w + 31) and writes C.  A wait that runs out sets *err, the
// accumulator is freed after a second bounded wait, and C is left unwritten.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "lc_internal.cuh"

namespace lc {

using bf16 = __nv_bfloat16;

constexpr int kTcM = 128, kTcK = 64;
constexpr int kTcMaxTries = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (8-row-group) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N / 8 and M / 16
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// byte offset of element (r, k) of an R x 64 K-major tile in core matrices
__device__ __forceinline__ uint32_t core_off(int r, int k, int rows) {
    return (uint32_t)((((k >> 3) * (rows >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
    for (int t = 0; t < kTcMaxTries; ++t) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 8 consecutive K elements (k .. k + 7) of row r of an operand into one
// 16-byte row of a core matrix; rows_contig: the source is contiguous along
// the rows (stride 1 between rows, ld between K elements), else along K
template <bool ROWS_CONTIG>
__device__ __forceinline__ uint4 load_k8(const bf16* __restrict__ S, int ld, int row, int nrows, int k, int K) {
    union {
        uint4 v;
        bf16 h[8];
    } u;
    if (row >= nrows) return make_uint4(0u, 0u, 0u, 0u);
    if (!ROWS_CONTIG && k + 8 <= K && (ld & 7) == 0 && (((uintptr_t)S) & 15) == 0)
        return *reinterpret_cast<const uint4*>(S + (size_t)row * ld + k);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int kk = k + j;
        u.h[j] = kk < K ? (ROWS_CONTIG ? S[(size_t)kk * ld + row] : S[(size_t)row * ld + kk]) : __float2bfloat16(0.f);
    }
    return u.v;
}

// Split K: blockIdx.z takes K range [z kper, min(K, (z + 1) kper)); with
// gridDim.z > 1 the tile goes to the workspace slice z (M x N, ld N) and a
// second kernel adds the slices in a fixed order.
template <bool AT, bool BT, int TN>
__global__ void __launch_bounds__(128) gemm_tc05_kernel(const bf16* __restrict__ A, int lda,
                                                        const bf16* __restrict__ B, int ldb, float* __restrict__ C,
                                                        int ldc, int M, int N, int K, int kper, float* __restrict__ ws,
                                                        int* __restrict__ err) {
    static_assert(TN % 16 == 0 && TN >= 16 && TN <= 256, "N tile");
    constexpr int kCols = TN <= 32 ? 32 : (TN <= 64 ? 64 : (TN <= 128 ? 128 : 256));
    constexpr uint32_t kLboA = (kTcM / 8) * 128, kLboB = (TN / 8) * 128;
    extern __shared__ unsigned char tc_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    bf16* sA = reinterpret_cast<bf16*>(base);
    bf16* sB = reinterpret_cast<bf16*>(base + kTcM * kTcK * 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * TN;
    const int kb = blockIdx.z * kper, ke = min(K, kb + kper);
    if (gridDim.z > 1) {
        C = ws + (size_t)blockIdx.z * M * N;
        ldc = N;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    uint32_t parity = 0;
    bool ok = true;
    int chunks = 0;
    for (int k0 = kb; k0 < ke; k0 += kTcK) {
        // op(A) rows m0.., op(B) columns n0.., K columns k0.. in groups of 8
        // K elements (one 16-byte core-matrix row each); consecutive threads
        // along the source's contiguous dimension
        for (int g = tid; g < kTcM * (kTcK / 8); g += 128) {
            const int r = AT ? g % kTcM : g / (kTcK / 8), kg = AT ? g / kTcM : g % (kTcK / 8);
            const uint4 v = load_k8<AT>(AT ? A + m0 : A + (size_t)m0 * lda, lda, r, M - m0, k0 + 8 * kg, ke);
            *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(sA) + core_off(r, 8 * kg, kTcM)) = v;
        }
        for (int g = tid; g < TN * (kTcK / 8); g += 128) {
            const int r = BT ? g / (kTcK / 8) : g % TN, kg = BT ? g % (kTcK / 8) : g / TN;
            const uint4 v = load_k8<!BT>(BT ? B + (size_t)n0 * ldb : B + n0, ldb, r, N - n0, k0 + 8 * kg, ke);
            *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(sB) + core_off(r, 8 * kg, TN)) = v;
        }
        // the tensor cores read shared memory through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int s = 0; s < kTcK / 16; ++s) {
                const uint64_t da = tc_desc(a0 + 2 * s * kLboA, kLboA, 128);
                const uint64_t db = tc_desc(b0 + 2 * s * kLboB, kLboB, 128);
                const uint32_t acc = (k0 > kb || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(tc_idesc(kTcM, TN)), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar))
                         : "memory");
        }
        ++chunks;
        const bool done = tc_wait(smem_u32(&bar), parity);
        parity ^= 1u;
        ok = __syncthreads_and(done ? 1 : 0) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) break;
    }
    if (ok && chunks > 0) {
        const int row = m0 + 32 * warp + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M)
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col < N) C[(size_t)row * ldc + col] = __uint_as_float(r[j]);
                }
        }
    } else if (chunks == 0) {
        // an empty K range: a zero product
        for (int e = tid; e < kTcM * TN; e += 128) {
            const int row = m0 + e / TN, col = n0 + e % TN;
            if (row < M && col < N) C[(size_t)row * ldc + col] = 0.f;
        }
    } else {
        if (tid == 0) atomicOr(err, 1);
        // the committed MMAs must finish before the accumulator is freed
        tc_wait(smem_u32(&bar), parity ^ 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

template <int TN>
constexpr int tc05_smem() {
    return kTcM * kTcK * 2 + TN * kTcK * 2 + 1024;
}

// C = sum of the S workspace slices, in slice order
__global__ void __launch_bounds__(256) splitk_sum_kernel(const float* __restrict__ ws, int S, int M, int N,
                                                         float* __restrict__ C, int ldc) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)M * N) return;
    float s = ws[e];
    for (int z = 1; z < S; ++z) s += ws[(size_t)z * M * N + e];
    C[(e / N) * ldc + e % N] = s;
}

template <bool AT, bool BT, int TN>
static cudaError_t launch_tc05(const bf16* A, int lda, const bf16* B, int ldb, float* C, int ldc, int M, int N, int K,
                               float* ws, size_t ws_floats, int* err, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(gemm_tc05_kernel<AT, BT, TN>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, tc05_smem<TN>());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // long K (the weight gradients, K = rows of the batch) split over CTAs
    // of at least 256 K each, as far as the workspace holds the slices
    int S = 1;
    if (K >= 512) {
        S = std::min(K / 256, 32);
        while (S > 1 && (size_t)S * M * N > ws_floats) --S;
    }
    const int kper = S > 1 ? ((K + S - 1) / S + kTcK - 1) / kTcK * kTcK : std::max(K, 1);
    S = S > 1 ? (K + kper - 1) / kper : 1;
    const dim3 grid((N + TN - 1) / TN, (M + kTcM - 1) / kTcM, S);
    gemm_tc05_kernel<AT, BT, TN><<<grid, 128, tc05_smem<TN>(), st>>>(A, lda, B, ldb, C, ldc, M, N, K, kper, ws, err);
    if (S > 1) {
        const size_t total = (size_t)M * N;
        splitk_sum_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(ws, S, M, N, C, ldc);
    }
    return cudaGetLastError();
}

template <bool AT, bool BT>
static cudaError_t launch_tc05_n(const bf16* A, int lda, const bf16* B, int ldb, float* C, int ldc, int M, int N,
                                 int K, float* ws, size_t ws_floats, int* err, cudaStream_t st) {
    // the network's widths: 256 (hidden) and 6 (output, one 16-wide tile)
    if (N <= 16) return launch_tc05<AT, BT, 16>(A, lda, B, ldb, C, ldc, M, N, K, ws, ws_floats, err, st);
    return launch_tc05<AT, BT, 256>(A, lda, B, ldb, C, ldc, M, N, K, ws, ws_floats, err, st);
}

cudaError_t gemm_bf16_tc05(bool at, bool bt, const bf16* A, int lda, const bf16* B, int ldb, float* C, int ldc, int M,
                           int N, int K, float* ws, size_t ws_floats, int* err, cudaStream_t st) {
    if (!at && !bt) return launch_tc05_n<false, false>(A, lda, B, ldb, C, ldc, M, N, K, ws, ws_floats, err, st);
    if (at && !bt) return launch_tc05_n<true, false>(A, lda, B, ldb, C, ldc, M, N, K, ws, ws_floats, err, st);
    if (!at && bt) return launch_tc05_n<false, true>(A, lda, B, ldb, C, ldc, M, N, K, ws, ws_floats, err, st);
    return launch_tc05_n<true, true>(A, lda, B, ldb, C, ldc, M, N, K, ws, ws_floats, err, st);
}

}  // namespace lc

// Learned per-node warm start: node features, the 64-256-256-6 MLP (BF16
// tensor-core GEMMs with FP32 accumulation), its backward pass and Adam, and
// the accept-or-reject application to a capture's node parameters.
//
// The paper starts each frame from the previous frame's result; the network
// predicts each node's update (d_omega, d_t) from features pooled at that
// start so that Gauss-Newton starts closer.  Plain GN stays the arbiter: the
// prediction is kept only if the energy at the predicted parameters does not
// exceed the energy at the start (decided on the device).
//
// Feature vector (64 per node): see lc_node_features in livecap.h.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "lc_context.h"

using namespace lc;

namespace lc {

using bf16 = __nv_bfloat16;

constexpr int kDIn = 64, kDH = 256, kDOut = 6;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kDIn * kDH;
constexpr int kOffW2 = kOffB1 + kDH;
constexpr int kOffB2 = kOffW2 + kDH * kDH;
constexpr int kOffW3 = kOffB2 + kDH;
constexpr int kOffB3 = kOffW3 + kDH * kDOut;
constexpr int kNParams = kOffB3 + kDOut;   // 83,974
static_assert(kNParams == LC_MLP_PARAMS, "parameter count");

// ---------------------------------------------------------------------------
// C[M x N] = op(A)[M x K] op(B)[K x N] in BF16 with FP32 accumulation on the
// tensor cores (mma.sync m16n8k16).  op(A)(m, k) = A[m lda + k], or A[k lda +
// m] when AT; op(B)(k, n) = B[k ldb + n], or B[n ldb + k] when BT.  Block
// tile 64 x 64 x 32, four warps of 32 x 32; edges are zero-padded in shared
// memory, so any M, N, K is accepted.
// ---------------------------------------------------------------------------
constexpr int kGM = 64, kGN = 64, kGK = 32, kGPad = 8;

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

template <bool AT, bool BT>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const bf16* __restrict__ A, int lda,
                                                        const bf16* __restrict__ B, int ldb,
                                                        float* __restrict__ C, int ldc, int M, int N, int K) {
    __shared__ bf16 As[kGM][kGK + kGPad];
    __shared__ bf16 Bs[kGK][kGN + kGPad];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * kGM, n0 = blockIdx.x * kGN;
    const int g = lane >> 2, cq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += kGK) {
        for (int e = tid; e < kGM * kGK; e += 128) {
            const int r = AT ? e % kGM : e / kGK, c = AT ? e / kGM : e % kGK;
            const int m = m0 + r, k = k0 + c;
            As[r][c] = (m < M && k < K) ? (AT ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : zero;
        }
        for (int e = tid; e < kGK * kGN; e += 128) {
            const int r = BT ? e % kGK : e / kGN, c = BT ? e / kGK : e % kGN;
            const int k = k0 + r, n = n0 + c;
            Bs[r][c] = (k < K && n < N) ? (BT ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n]) : zero;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kGK; ks += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + g, c = ks + 2 * cq;
                a[i][0] = pack2(As[r][c], As[r][c + 1]);
                a[i][1] = pack2(As[r + 8][c], As[r + 8][c + 1]);
                a[i][2] = pack2(As[r][c + 8], As[r][c + 9]);
                a[i][3] = pack2(As[r + 8][c + 8], As[r + 8][c + 9]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = wn + j * 8 + g, k = ks + 2 * cq;
                b[j][0] = pack2(Bs[k][n], Bs[k + 1][n]);
                b[j][1] = pack2(Bs[k + 8][n], Bs[k + 9][n]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                        : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]), "r"(b[j][1]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = m0 + wm + i * 16 + g, c = n0 + wn + j * 8 + 2 * cq;
            if (r < M && c < N) C[(size_t)r * ldc + c] = acc[i][j][0];
            if (r < M && c + 1 < N) C[(size_t)r * ldc + c + 1] = acc[i][j][1];
            if (r + 8 < M && c < N) C[(size_t)(r + 8) * ldc + c] = acc[i][j][2];
            if (r + 8 < M && c + 1 < N) C[(size_t)(r + 8) * ldc + c + 1] = acc[i][j][3];
        }
}

// tcgen05 GEMM (gemm_tc05.cu)
cudaError_t gemm_bf16_tc05(bool at, bool bt, const bf16* A, int lda, const bf16* B, int ldb, float* C, int ldc, int M,
                           int N, int K, float* ws, size_t ws_floats, int* err, cudaStream_t st);

void gemm_bf16(bool at, bool bt, const bf16* A, int lda, const bf16* B, int ldb, float* C, int ldc, int M, int N,
               int K, cudaStream_t st) {
    const dim3 grid((N + kGN - 1) / kGN, (M + kGM - 1) / kGM);
    if (!at && !bt) gemm_bf16_kernel<false, false><<<grid, 128, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K);
    if (at && !bt) gemm_bf16_kernel<true, false><<<grid, 128, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K);
    if (!at && bt) gemm_bf16_kernel<false, true><<<grid, 128, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K);
    if (at && bt) gemm_bf16_kernel<true, true><<<grid, 128, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K);
}

// ---------------------------------------------------------------------------
// element-wise parts of the network
// ---------------------------------------------------------------------------
__global__ void normalise_kernel(const float* __restrict__ F, const float* __restrict__ mu,
                                 const float* __restrict__ sigma, bf16* __restrict__ X, int M) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)M * kDIn) return;
    const int c = (int)(e % kDIn);
    const float s = sigma[c];
    X[e] = __float2bfloat16((F[e] - mu[c]) / (s > 0.f ? s : 1.f));
}

// H = relu(Z + b) in BF16
__global__ void bias_relu_kernel(const float* __restrict__ Z, const float* __restrict__ b, bf16* __restrict__ H,
                                 int M, int N) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)M * N) return;
    H[e] = __float2bfloat16(fmaxf(Z[e] + b[e % N], 0.f));
}

// Y = (Z + b) * s_out, per output column
__global__ void out_bias_kernel(const float* __restrict__ Z, const float* __restrict__ b,
                                const float* __restrict__ s_out, float* __restrict__ Y, int M) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * kDOut) return;
    Y[e] = (Z[e] + b[e % kDOut]) * s_out[e % kDOut];
}

// gradient with respect to the last layer's pre-scale output,
// dZ3 = 2 (Y - T) s_out / M (FP32 and BF16), and per-block FP64 partial sums
// of ||Y - T||^2 (a fixed-order second pass adds them)
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                                                   const float* __restrict__ s_out, float* __restrict__ dY,
                                                   bf16* __restrict__ dYb, double* __restrict__ part, int M) {
    __shared__ double sh[8];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (e < M * kDOut) {
        const float d = Y[e] - T[e];
        const float gy = 2.f * d / (float)M * s_out[e % kDOut];
        dY[e] = gy;
        dYb[e] = __float2bfloat16(gy);
        s = (double)d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(32) loss_total_kernel(const double* __restrict__ part, int nblocks, int M,
                                                        double* __restrict__ out) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 32) s += part[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s / (double)(M > 0 ? M : 1);
}

// dZ = dH where the unit was active (H > 0), in BF16
__global__ void relu_back_kernel(const float* __restrict__ dH, const bf16* __restrict__ H, bf16* __restrict__ dZ,
                                 size_t n) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    dZ[e] = __float2bfloat16(__bfloat162float(H[e]) > 0.f ? dH[e] : 0.f);
}

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(bf16 x) { return __bfloat162float(x); }

// out[c] = sum over rows of X[r][c], one block per column, fixed order
template <typename T>
__global__ void __launch_bounds__(256) colsum_kernel(const T* __restrict__ X, int M, int N, float* __restrict__ out) {
    __shared__ float sh[8];
    const int c = blockIdx.x;
    float s = 0.f;
    for (int r = threadIdx.x; r < M; r += 256) s += to_f(X[(size_t)r * N + c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += sh[w];
        out[c] = t;
    }
}

// BF16 copies of the weight matrices from the FP32 master parameters
__global__ void weights_bf16_kernel(const float* __restrict__ theta, bf16* __restrict__ W1, bf16* __restrict__ W2,
                                    bf16* __restrict__ W3) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kDIn * kDH) W1[e] = __float2bfloat16(theta[kOffW1 + e]);
    if (e < kDH * kDH) W2[e] = __float2bfloat16(theta[kOffW2 + e]);
    if (e < kDH * kDOut) W3[e] = __float2bfloat16(theta[kOffW3 + e]);
}

// Adam with bias correction (Kingma and Ba, 2015); bc1 = 1 - beta1^t,
// bc2 = 1 - beta2^t computed on the host
__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kNParams) return;
    const float gr = grad[e];
    const float mm = b1 * m[e] + (1.f - b1) * gr;
    const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    theta[e] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
}

// Column sums and sums of squares in FP64 of a rows x cols array (cols <=
// 256), shifted by the column's first value (sums of x - x_0 and
// (x - x_0)^2: no cancellation when the mean is large against the spread,
// and exactly zero for a constant column): thread j of a block takes column
// j % cols of rows j / cols, + 256 / cols, ...; grid-stride over row groups,
// fixed order.  part[block][2 cols].
__global__ void __launch_bounds__(256) column_moments_kernel(const float* __restrict__ X, long long rows, int cols,
                                                             double* __restrict__ part) {
    __shared__ double sh[2][256];
    const int per = 256 / cols;            // rows per pass of a block
    const int j = threadIdx.x;
    const bool on = j < per * cols;
    const int c = j % cols, r0 = j / cols;
    double s = 0.0, q = 0.0;
    if (on) {
        const double x0 = X[c];
        for (long long r = (long long)blockIdx.x * per + r0; r < rows; r += (long long)gridDim.x * per) {
            const double x = (double)X[r * cols + c] - x0;
            s += x;
            q += x * x;
        }
    }
    sh[0][j] = on ? s : 0.0;
    sh[1][j] = on ? q : 0.0;
    __syncthreads();
    if (j < cols) {
        double ts = 0.0, tq = 0.0;
        for (int k = j; k < per * cols; k += cols) {
            ts += sh[0][k];
            tq += sh[1][k];
        }
        part[(size_t)blockIdx.x * 2 * cols + j] = ts;
        part[(size_t)blockIdx.x * 2 * cols + cols + j] = tq;
    }
}

// input normalisation and output scale from the shifted column moments of
// the features (partF, 64 columns, first row F0) and of the targets (partT,
// 6 columns, first row T0): mu = mean, sigma = population standard
// deviation (1 where below 1e-12; the constant feature 63 keeps mu 0,
// sigma 1), s_out = root mean square of each target column (1 where below
// 1e-12).  With d = x - x_0: mean = x_0 + S/n, variance = Q/n - (S/n)^2,
// mean square = x_0^2 + 2 x_0 S/n + Q/n.
__global__ void __launch_bounds__(128) fit_scaling_kernel(const double* __restrict__ partF,
                                                          const double* __restrict__ partT,
                                                          const float* __restrict__ F0, const float* __restrict__ T0,
                                                          int nblocks, long long rows, float* __restrict__ mu,
                                                          float* __restrict__ sigma, float* __restrict__ s_out) {
    const int j = threadIdx.x;
    const double n = (double)rows;
    if (j < kDIn) {
        double s = 0.0, q = 0.0;
        for (int b = 0; b < nblocks; ++b) {
            s += partF[(size_t)b * 2 * kDIn + j];
            q += partF[(size_t)b * 2 * kDIn + kDIn + j];
        }
        const double d = s / n;
        const double sd = sqrt(fmax(q / n - d * d, 0.0));
        const bool constant = j == kDIn - 1;
        mu[j] = constant ? 0.f : (float)((double)F0[j] + d);
        sigma[j] = (constant || sd < 1e-12) ? 1.f : (float)sd;
    } else if (j < kDIn + kDOut) {
        const int c = j - kDIn;
        double s = 0.0, q = 0.0;
        for (int b = 0; b < nblocks; ++b) {
            s += partT[(size_t)b * 2 * kDOut + c];
            q += partT[(size_t)b * 2 * kDOut + kDOut + c];
        }
        const double x0 = T0[c];
        const double rms = sqrt(fmax(x0 * x0 + 2.0 * x0 * (s / n) + q / n, 0.0));
        s_out[c] = rms < 1e-12 ? 1.f : (float)rms;
    }
}

__global__ void gather_rows_kernel(const float* __restrict__ F, const float* __restrict__ T,
                                   const int* __restrict__ idx, int B, float* __restrict__ Fb, float* __restrict__ Tb) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < B * kDIn) Fb[e] = F[(size_t)idx[e / kDIn] * kDIn + e % kDIn];
    if (e < B * kDOut) Tb[e] = T[(size_t)idx[e / kDOut] * kDOut + e % kDOut];
}

// ---------------------------------------------------------------------------
// node features and the warm-start application
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 rot_log3(float r00, float r01, float r02, float r10, float r11, float r12, float r20,
                                           float r21, float r22) {
    const float c = fminf(1.f, fmaxf(-1.f, 0.5f * (r00 + r11 + r22 - 1.f)));
    const float th = acosf(c);
    const float s = sinf(th);
    const float f = th < 1e-4f ? 0.5f : th / (2.f * s);
    return make_float3(f * (r21 - r12), f * (r02 - r20), f * (r10 - r01));
}

// one warp per node: pooled per-vertex quantities over the node's bound
// vertices (binding weights), plus node-level terms; layout as in the header
__global__ void __launch_bounds__(256) node_features_kernel(const CapDesc* __restrict__ caps,
                                                            const float4* __restrict__ motion,
                                                            float* __restrict__ Fout) {
    const CapDesc& C = caps[0];
    const int lane = threadIdx.x & 31;
    const int k = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (k >= C.n) return;
    float s[24];
#pragma unroll
    for (int q = 0; q < 24; ++q) s[q] = 0.f;
    for (int j = C.ent_off[k] + lane; j < C.ent_off[k + 1]; j += 32) {
        const int2 en = C.ent[j];
        const int i = en.x;
        const float w = __int_as_float(en.y);
        const float4 r = C.res[i], ha = C.HA[i], hb = C.HB[i], ev = C.ev[i];
        const uint32_t fl = C.flags[i];
        const float v[23] = {r.x, r.y, r.z, fabsf(r.x), fabsf(r.y), fabsf(r.z), r.w, r.w * r.w,
                             ev.x, ev.y, ev.z, fabsf(ev.x), fabsf(ev.y), fabsf(ev.z),
                             ha.x, ha.y, ha.z, ha.w, hb.x, hb.y,
                             (fl & LC_VIS_BIT) ? 1.f : 0.f, (fl & LC_INB_BIT) ? 1.f : 0.f,
                             (fl & LC_BNEG_BIT) ? 1.f : 0.f};
#pragma unroll
        for (int q = 0; q < 23; ++q) s[q] += w * v[q];
        s[23] += w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 24; ++q) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    float nb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int e0 = C.edge_off[k], e1 = C.edge_off[k + 1];
    for (int j = e0 + lane; j < e1; j += 32) {
        const int l = C.edge_dst[j];
        const float4 a = motion[2 * l], b = motion[2 * l + 1];
        nb[0] += a.x; nb[1] += a.y; nb[2] += a.z; nb[3] += b.x; nb[4] += b.y; nb[5] += b.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 6; ++q) nb[q] += __shfl_xor_sync(0xffffffffu, nb[q], o);
    if (lane != 0) return;
    float* F = Fout + (size_t)k * 64;
    const float4 R0 = C.node_R[3 * k], R1 = C.node_R[3 * k + 1], R2 = C.node_R[3 * k + 2];
    const float3 om = rot_log3(R0.x, R0.y, R0.z, R1.x, R1.y, R1.z, R2.x, R2.y, R2.z);
    const float4 t = C.node_t[k];
    const float4 bw = C.b[2 * k], bt = C.b[2 * k + 1], dw = C.diag[2 * k], dt = C.diag[2 * k + 1];
    const float bb[6] = {bw.x, bw.y, bw.z, bt.x, bt.y, bt.z};
    const float dd[6] = {dw.x, dw.y, dw.z, dt.x, dt.y, dt.z};
    float dmax = dd[0];
    for (int q = 1; q < 6; ++q) dmax = fmaxf(dmax, dd[q]);
    const float tau = 1e-6f * dmax + 1e-30f;
    F[0] = om.x; F[1] = om.y; F[2] = om.z; F[3] = t.x; F[4] = t.y; F[5] = t.z;
    for (int q = 0; q < 6; ++q) {
        F[6 + q] = bb[q];
        F[12 + q] = dd[q];
        F[18 + q] = bb[q] / (dd[q] + tau);
    }
    const float W = s[23];
    for (int q = 0; q < 23; ++q) F[24 + q] = W > 0.f ? s[q] / W : 0.f;
    F[47] = W;
    const float4 g = C.node_g[k];
    F[48] = g.x; F[49] = g.y; F[50] = g.z;
    const float4 ua = motion[2 * k], ub = motion[2 * k + 1];
    F[51] = ua.x; F[52] = ua.y; F[53] = ua.z; F[54] = ub.x; F[55] = ub.y; F[56] = ub.z;
    const int deg = e1 - e0;
    for (int q = 0; q < 6; ++q) F[57 + q] = deg > 0 ? nb[q] / (float)deg : 0.f;
    F[63] = 1.f;
}

// energy at the current linearisation (photo + sil + ARAP) into slot
__global__ void energy_copy_kernel(const CapDesc* __restrict__ caps, double* __restrict__ out) {
    const Scalars* sc = caps[0].sc;
    *out = sc->e_lin[0] + sc->e_lin[1] + sc->e_lin[2];
}

// save the node parameters and apply the predicted update R <- Exp(w) R, t += d
__global__ void apply_prediction_kernel(const CapDesc* __restrict__ caps, const float* __restrict__ Y,
                                        float4* __restrict__ R0, float4* __restrict__ t0) {
    const CapDesc& C = caps[0];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= C.n) return;
    const float4 r0 = C.node_R[3 * k], r1 = C.node_R[3 * k + 1], r2 = C.node_R[3 * k + 2];
    const float4 t = C.node_t[k];
    R0[3 * k] = r0; R0[3 * k + 1] = r1; R0[3 * k + 2] = r2;
    t0[k] = t;
    const float* y = Y + (size_t)k * 6;
    const float wx = y[0], wy = y[1], wz = y[2];
    const float th2 = wx * wx + wy * wy + wz * wz, th = sqrtf(th2);
    float A, B;
    if (th < 1e-4f) {
        A = 1.f - th2 * (1.f / 6.f);
        B = 0.5f - th2 * (1.f / 24.f);
    } else {
        const float sh = sinf(0.5f * th);
        A = sinf(th) / th;
        B = 2.f * sh * sh / th2;
    }
    const float E00 = 1.f - B * (wy * wy + wz * wz), E11 = 1.f - B * (wx * wx + wz * wz), E22 = 1.f - B * (wx * wx + wy * wy);
    const float E01 = -A * wz + B * wx * wy, E10 = A * wz + B * wx * wy;
    const float E02 = A * wy + B * wx * wz, E20 = -A * wy + B * wx * wz;
    const float E12 = -A * wx + B * wy * wz, E21 = A * wx + B * wy * wz;
    C.node_R[3 * k] = make_float4(E00 * r0.x + E01 * r1.x + E02 * r2.x, E00 * r0.y + E01 * r1.y + E02 * r2.y,
                                  E00 * r0.z + E01 * r1.z + E02 * r2.z, 0.f);
    C.node_R[3 * k + 1] = make_float4(E10 * r0.x + E11 * r1.x + E12 * r2.x, E10 * r0.y + E11 * r1.y + E12 * r2.y,
                                      E10 * r0.z + E11 * r1.z + E12 * r2.z, 0.f);
    C.node_R[3 * k + 2] = make_float4(E20 * r0.x + E21 * r1.x + E22 * r2.x, E20 * r0.y + E21 * r1.y + E22 * r2.y,
                                      E20 * r0.z + E21 * r1.z + E22 * r2.z, 0.f);
    C.node_t[k] = make_float4(t.x + y[3], t.y + y[4], t.z + y[5], 0.f);
}

// keep the prediction iff it does not raise the energy; e[0] start, e[1] predicted
__global__ void accept_kernel(const CapDesc* __restrict__ caps, const double* __restrict__ e,
                              const float4* __restrict__ R0, const float4* __restrict__ t0, int* __restrict__ accepted) {
    const CapDesc& C = caps[0];
    const bool keep = e[1] <= e[0];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        *accepted = keep ? 1 : 0;
        C.sc->vis_frozen = 1;   // the next solve keeps the frame decisions of the start
    }
    if (keep || k >= C.n) return;
    C.node_R[3 * k] = R0[3 * k];
    C.node_R[3 * k + 1] = R0[3 * k + 1];
    C.node_R[3 * k + 2] = R0[3 * k + 2];
    C.node_t[k] = t0[k];
}

// motion over the last frame: u = (Log(R Rprev^T), t - tprev); prev <- current
__global__ void record_motion_kernel(const CapDesc* __restrict__ caps, float4* __restrict__ Rp,
                                     float4* __restrict__ tp, float4* __restrict__ motion) {
    const CapDesc& C = caps[0];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= C.n) return;
    const float4 a0 = C.node_R[3 * k], a1 = C.node_R[3 * k + 1], a2 = C.node_R[3 * k + 2];
    const float4 b0 = Rp[3 * k], b1 = Rp[3 * k + 1], b2 = Rp[3 * k + 2];
    // D = R Rprev^T: D_ij = row i of R . row j of Rprev
    auto d = [](float4 x, float4 y) { return x.x * y.x + x.y * y.y + x.z * y.z; };
    const float3 w = rot_log3(d(a0, b0), d(a0, b1), d(a0, b2), d(a1, b0), d(a1, b1), d(a1, b2), d(a2, b0), d(a2, b1),
                              d(a2, b2));
    const float4 t = C.node_t[k], q = tp[k];
    motion[2 * k] = make_float4(w.x, w.y, w.z, 0.f);
    motion[2 * k + 1] = make_float4(t.x - q.x, t.y - q.y, t.z - q.z, 0.f);
    Rp[3 * k] = a0; Rp[3 * k + 1] = a1; Rp[3 * k + 2] = a2;
    tp[k] = t;
}

__global__ void identity_rows_kernel(float4* __restrict__ R, float4* __restrict__ t, float4* __restrict__ motion, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    R[3 * k] = make_float4(1.f, 0.f, 0.f, 0.f);
    R[3 * k + 1] = make_float4(0.f, 1.f, 0.f, 0.f);
    R[3 * k + 2] = make_float4(0.f, 0.f, 1.f, 0.f);
    t[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    motion[2 * k] = make_float4(0.f, 0.f, 0.f, 0.f);
    motion[2 * k + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace lc

// ---------------------------------------------------------------------------
// the network object
// ---------------------------------------------------------------------------
static std::atomic<unsigned long long> g_mlp_uid{0};   // creation counter (host)

struct lc_mlp {
    unsigned long long uid = 0;   // unique per network; gen bumps when scratch moves
    unsigned long long gen = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    float* theta = nullptr;   // FP32 master parameters
    float* grad = nullptr;
    float* mom = nullptr;
    float* vel = nullptr;
    float* mu = nullptr;
    float* sigma = nullptr;
    float* s_out = nullptr;   // output scale (6), 1 unless set or fitted
    bf16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr;
    int step = 0;
    // activations, sized for `cap` rows
    int cap = 0;
    bf16 *X = nullptr, *H1 = nullptr, *H2 = nullptr, *dYb = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    float *Z = nullptr, *Y = nullptr, *dY = nullptr, *Fin = nullptr, *Tin = nullptr;
    double *part = nullptr, *loss = nullptr;
    int* idx = nullptr;
    // contractions on tcgen05 (0) or mma.sync (1); gerr: a tcgen05 wait ran out
    int gemm_kind = 0;
    int* gerr = nullptr;
    float* ws = nullptr;                       // split-K slices of the tcgen05 GEMM
    static constexpr size_t kWsFloats = size_t(1) << 20;
    std::vector<void*> owned;

    lc_status fail(lc_status s, const char* m) {
        err = m;
        return s;
    }
    void* alloc(size_t bytes) {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        owned.push_back(p);
        return p;
    }
    void release(void* p) {
        if (!p) return;
        cudaFree(p);
        owned.erase(std::remove(owned.begin(), owned.end(), p), owned.end());
    }
    lc_status ensure(int M) {
        if (M <= cap) return LC_OK;
        for (void* p : {(void*)X, (void*)H1, (void*)H2, (void*)dYb, (void*)dZ2, (void*)dZ1, (void*)Z, (void*)Y,
                        (void*)dY, (void*)Fin, (void*)Tin, (void*)part, (void*)idx})
            release(p);
        const size_t m = (size_t)M;
        X = (bf16*)alloc(sizeof(bf16) * m * kDIn);
        H1 = (bf16*)alloc(sizeof(bf16) * m * kDH);
        H2 = (bf16*)alloc(sizeof(bf16) * m * kDH);
        dYb = (bf16*)alloc(sizeof(bf16) * m * kDOut);
        dZ2 = (bf16*)alloc(sizeof(bf16) * m * kDH);
        dZ1 = (bf16*)alloc(sizeof(bf16) * m * kDH);
        Z = (float*)alloc(sizeof(float) * m * kDH);
        Y = (float*)alloc(sizeof(float) * m * kDOut);
        dY = (float*)alloc(sizeof(float) * m * kDOut);
        Fin = (float*)alloc(sizeof(float) * m * kDIn);
        Tin = (float*)alloc(sizeof(float) * m * kDOut);
        part = (double*)alloc(sizeof(double) * ((m * kDOut + 255) / 256 + 1));
        idx = (int*)alloc(sizeof(int) * m);
        if (!X || !H1 || !H2 || !dYb || !dZ2 || !dZ1 || !Z || !Y || !dY || !Fin || !Tin || !part || !idx) {
            cap = 0;
            return fail(LC_ERR_OOM, "lc_mlp: device memory");
        }
        cap = M;
        ++gen;
        return LC_OK;
    }
    void gemm(bool at, bool bt, const bf16* A, int lda, const bf16* B, int ldb, float* C, int ldc, int M, int N, int K,
              cudaStream_t st) {
        if (gemm_kind == 0)
            gemm_bf16_tc05(at, bt, A, lda, B, ldb, C, ldc, M, N, K, ws, kWsFloats, gerr, st);
        else
            gemm_bf16(at, bt, A, lda, B, ldb, C, ldc, M, N, K, st);
    }
    void refresh_weights(cudaStream_t st) { weights_bf16_kernel<<<(kDH * kDH + 255) / 256, 256, 0, st>>>(theta, W1, W2, W3); }
    // forward on rows already normalised into X; output Y (FP32, M x 6)
    void forward(int M, cudaStream_t st) {
        gemm(false, false, X, kDIn, W1, kDH, Z, kDH, M, kDH, kDIn, st);
        bias_relu_kernel<<<(unsigned)(((size_t)M * kDH + 255) / 256), 256, 0, st>>>(Z, theta + kOffB1, H1, M, kDH);
        gemm(false, false, H1, kDH, W2, kDH, Z, kDH, M, kDH, kDH, st);
        bias_relu_kernel<<<(unsigned)(((size_t)M * kDH + 255) / 256), 256, 0, st>>>(Z, theta + kOffB2, H2, M, kDH);
        gemm(false, false, H2, kDH, W3, kDOut, Z, kDOut, M, kDOut, kDH, st);
        out_bias_kernel<<<(M * kDOut + 255) / 256, 256, 0, st>>>(Z, theta + kOffB3, s_out, Y, M);
    }
    // loss and parameter gradient for targets T (FP32, M x 6) after forward
    void backward(const float* T, int M, cudaStream_t st) {
        const int lb = (M * kDOut + 255) / 256;
        loss_kernel<<<lb, 256, 0, st>>>(Y, T, s_out, dY, dYb, part, M);
        loss_total_kernel<<<1, 32, 0, st>>>(part, lb, M, loss);
        const size_t nh = (size_t)M * kDH;
        // layer 3
        gemm(true, false, H2, kDH, dYb, kDOut, grad + kOffW3, kDOut, kDH, kDOut, M, st);
        colsum_kernel<float><<<kDOut, 256, 0, st>>>(dY, M, kDOut, grad + kOffB3);
        gemm(false, true, dYb, kDOut, W3, kDOut, Z, kDH, M, kDH, kDOut, st);   // dH2 = dY W3^T
        relu_back_kernel<<<(unsigned)((nh + 255) / 256), 256, 0, st>>>(Z, H2, dZ2, nh);
        // layer 2
        gemm(true, false, H1, kDH, dZ2, kDH, grad + kOffW2, kDH, kDH, kDH, M, st);
        colsum_kernel<bf16><<<kDH, 256, 0, st>>>(dZ2, M, kDH, grad + kOffB2);
        gemm(false, true, dZ2, kDH, W2, kDH, Z, kDH, M, kDH, kDH, st);        // dH1 = dZ2 W2^T
        relu_back_kernel<<<(unsigned)((nh + 255) / 256), 256, 0, st>>>(Z, H1, dZ1, nh);
        // layer 1
        gemm(true, false, X, kDIn, dZ1, kDH, grad + kOffW1, kDH, kDIn, kDH, M, st);
        colsum_kernel<bf16><<<kDH, 256, 0, st>>>(dZ1, M, kDH, grad + kOffB1);
    }
};

// ---------------------------------------------------------------------------
// per-context warm-start state (node-sized buffers)
// ---------------------------------------------------------------------------
struct WarmState {
    int n = 0;
    float* F = nullptr;        // n x 64 features
    float* Yp = nullptr;       // n x 6 prediction
    float4* motion = nullptr;  // 2n: the node's update over the last frame
    float4* Rprev = nullptr;   // 3n: parameters at the end of the previous frame
    float4* tprev = nullptr;
    float4* R0 = nullptr;      // 3n: parameters before the prediction
    float4* t0 = nullptr;
    double* e = nullptr;       // energies at the start and at the prediction
    int* accepted = nullptr;
    // the warm-start sequence captured as one CUDA graph, for this network
    // and its scratch buffers
    cudaGraphExec_t gexec = nullptr;
    unsigned long long g_uid = 0, g_gen = 0;
};

// ---------------------------------------------------------------------------
// C ABI: the network
// ---------------------------------------------------------------------------
static lc_status mlp_cuda(lc_mlp* m, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LC_OK;
    cudaGetLastError();
    m->err = std::string(what) + ": " + cudaGetErrorString(e);
    return LC_ERR_CUDA;
}

// synchronise the network's stream; a tcgen05 wait that ran out since the
// last check is reported (once) as LC_ERR_TIMEOUT
static lc_status mlp_sync(lc_mlp* m, cudaStream_t st, const char* what) {
    lc_status s = mlp_cuda(m, cudaStreamSynchronize(st), what);
    if (s) return s;
    int ge = 0;
    if (m->gerr && cudaMemcpy(&ge, m->gerr, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && ge) {
        cudaMemset(m->gerr, 0, sizeof(int));
        m->err = std::string(what) + ": a bounded tensor-core wait ran out";
        return LC_ERR_TIMEOUT;
    }
    return LC_OK;
}

static bool is_dev(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

extern "C" lc_status lc_mlp_create(lc_mlp** out, int device, const float* params, const float* mu,
                                   const float* sigma) {
    if (!out) return LC_ERR_ARG;
    *out = nullptr;
    auto* m = new lc_mlp();
    m->uid = ++g_mlp_uid;
    m->device = device;
    if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return LC_ERR_CUDA;
    }
    m->theta = (float*)m->alloc(sizeof(float) * kNParams);
    m->grad = (float*)m->alloc(sizeof(float) * kNParams);
    m->mom = (float*)m->alloc(sizeof(float) * kNParams);
    m->vel = (float*)m->alloc(sizeof(float) * kNParams);
    m->mu = (float*)m->alloc(sizeof(float) * kDIn);
    m->sigma = (float*)m->alloc(sizeof(float) * kDIn);
    m->s_out = (float*)m->alloc(sizeof(float) * kDOut);
    m->W1 = (bf16*)m->alloc(sizeof(bf16) * kDIn * kDH);
    m->W2 = (bf16*)m->alloc(sizeof(bf16) * kDH * kDH);
    m->W3 = (bf16*)m->alloc(sizeof(bf16) * kDH * kDOut);
    m->loss = (double*)m->alloc(sizeof(double));
    m->gerr = (int*)m->alloc(sizeof(int));
    m->ws = (float*)m->alloc(sizeof(float) * lc_mlp::kWsFloats);
    if (!m->theta || !m->grad || !m->mom || !m->vel || !m->mu || !m->sigma || !m->s_out || !m->W1 || !m->W2 || !m->W3 || !m->loss || !m->gerr || !m->ws) {
        lc_mlp_destroy(m);
        return LC_ERR_OOM;
    }
    std::vector<float> zeros(kNParams, 0.f), ones(kDIn, 1.f);
    cudaMemcpy(m->theta, params ? params : zeros.data(), sizeof(float) * kNParams, cudaMemcpyDefault);
    cudaMemcpy(m->mu, mu ? mu : zeros.data(), sizeof(float) * kDIn, cudaMemcpyDefault);
    cudaMemcpy(m->sigma, sigma ? sigma : ones.data(), sizeof(float) * kDIn, cudaMemcpyDefault);
    cudaMemcpy(m->s_out, ones.data(), sizeof(float) * kDOut, cudaMemcpyDefault);
    cudaMemset(m->gerr, 0, sizeof(int));
    cudaMemset(m->mom, 0, sizeof(float) * kNParams);
    cudaMemset(m->vel, 0, sizeof(float) * kNParams);
    m->refresh_weights(m->stream);
    lc_status s = mlp_cuda(m, cudaStreamSynchronize(m->stream), "lc_mlp_create");
    if (s) {
        lc_mlp_destroy(m);
        return s;
    }
    *out = m;
    return LC_OK;
}

extern "C" lc_status lc_mlp_destroy(lc_mlp* m) {
    if (!m) return LC_ERR_ARG;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (void* p : m->owned) cudaFree(p);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return LC_OK;
}

extern "C" const char* lc_mlp_last_error(const lc_mlp* m) { return m ? m->err.c_str() : "null network"; }

extern "C" lc_status lc_mlp_get_params(lc_mlp* m, float* params) {
    if (!m || !params) return LC_ERR_ARG;
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->stream);
    return mlp_cuda(m, cudaMemcpy(params, m->theta, sizeof(float) * kNParams, cudaMemcpyDefault), "lc_mlp_get_params");
}

extern "C" lc_status lc_mlp_set_gemm(lc_mlp* m, int kind) {
    if (!m || kind < LC_GEMM_TCGEN05 || kind > LC_GEMM_MMA_SYNC) return LC_ERR_ARG;
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->stream);
    m->gemm_kind = kind;
    ++m->gen;   // captured warm-start graphs hold the other kernels
    return LC_OK;
}

extern "C" lc_status lc_mlp_set_scaling(lc_mlp* m, const float* mu, const float* sigma, const float* s_out) {
    if (!m) return LC_ERR_ARG;
    cudaSetDevice(m->device);
    cudaStream_t st = m->stream;
    if (mu) cudaMemcpyAsync(m->mu, mu, sizeof(float) * kDIn, cudaMemcpyDefault, st);
    if (sigma) cudaMemcpyAsync(m->sigma, sigma, sizeof(float) * kDIn, cudaMemcpyDefault, st);
    if (s_out) cudaMemcpyAsync(m->s_out, s_out, sizeof(float) * kDOut, cudaMemcpyDefault, st);
    return mlp_cuda(m, cudaStreamSynchronize(st), "lc_mlp_set_scaling");
}

extern "C" lc_status lc_mlp_get_scaling(lc_mlp* m, float* mu, float* sigma, float* s_out) {
    if (!m) return LC_ERR_ARG;
    cudaSetDevice(m->device);
    cudaStream_t st = m->stream;
    if (mu) cudaMemcpyAsync(mu, m->mu, sizeof(float) * kDIn, cudaMemcpyDefault, st);
    if (sigma) cudaMemcpyAsync(sigma, m->sigma, sizeof(float) * kDIn, cudaMemcpyDefault, st);
    if (s_out) cudaMemcpyAsync(s_out, m->s_out, sizeof(float) * kDOut, cudaMemcpyDefault, st);
    return mlp_cuda(m, cudaStreamSynchronize(st), "lc_mlp_get_scaling");
}

// mu / sigma / s_out from the training rows, on the device
extern "C" lc_status lc_mlp_fit_scaling(lc_mlp* m, const float* F, const float* T, long long rows) {
    if (!m || !F || !T || rows < 1) return LC_ERR_ARG;
    if (!is_dev(F) || !is_dev(T)) return m->fail(LC_ERR_ARG, "lc_mlp_fit_scaling: F and T must be device arrays");
    cudaSetDevice(m->device);
    cudaStream_t st = m->stream;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
    const int nb = 4 * (sms > 0 ? sms : 1);
    double* part = nullptr;
    if (cudaMalloc(&part, sizeof(double) * (size_t)nb * 2 * (kDIn + kDOut)) != cudaSuccess) {
        cudaGetLastError();
        return m->fail(LC_ERR_OOM, "lc_mlp_fit_scaling: device memory");
    }
    double* partT = part + (size_t)nb * 2 * kDIn;
    column_moments_kernel<<<nb, 256, 0, st>>>(F, rows, kDIn, part);
    column_moments_kernel<<<nb, 256, 0, st>>>(T, rows, kDOut, partT);
    fit_scaling_kernel<<<1, 128, 0, st>>>(part, partT, F, T, nb, rows, m->mu, m->sigma, m->s_out);
    lc_status s = mlp_sync(m, st, "lc_mlp_fit_scaling");
    cudaFree(part);
    return s;
}

// F (M x 64 raw features) -> Y (M x 6)
extern "C" lc_status lc_mlp_forward(lc_mlp* m, const float* F, int M, float* Y) {
    if (!m || !F || !Y || M < 1) return LC_ERR_ARG;
    cudaSetDevice(m->device);
    lc_status s;
    if ((s = m->ensure(M))) return s;
    cudaStream_t st = m->stream;
    const float* Fd = F;
    if (!is_dev(F)) {
        cudaMemcpyAsync(m->Fin, F, sizeof(float) * (size_t)M * kDIn, cudaMemcpyHostToDevice, st);
        Fd = m->Fin;
    }
    normalise_kernel<<<(unsigned)(((size_t)M * kDIn + 255) / 256), 256, 0, st>>>(Fd, m->mu, m->sigma, m->X, M);
    m->forward(M, st);
    cudaMemcpyAsync(Y, m->Y, sizeof(float) * (size_t)M * kDOut, cudaMemcpyDefault, st);
    return mlp_sync(m, st, "lc_mlp_forward");
}

// loss (1/M) sum ||y - t||^2 and its gradient with respect to the parameters
extern "C" lc_status lc_mlp_gradient(lc_mlp* m, const float* F, const float* T, int M, float* grad, double* loss) {
    if (!m || !F || !T || M < 1) return LC_ERR_ARG;
    cudaSetDevice(m->device);
    lc_status s;
    if ((s = m->ensure(M))) return s;
    cudaStream_t st = m->stream;
    cudaMemcpyAsync(m->Fin, F, sizeof(float) * (size_t)M * kDIn, cudaMemcpyDefault, st);
    cudaMemcpyAsync(m->Tin, T, sizeof(float) * (size_t)M * kDOut, cudaMemcpyDefault, st);
    normalise_kernel<<<(unsigned)(((size_t)M * kDIn + 255) / 256), 256, 0, st>>>(m->Fin, m->mu, m->sigma, m->X, M);
    m->forward(M, st);
    m->backward(m->Tin, M, st);
    if (grad) cudaMemcpyAsync(grad, m->grad, sizeof(float) * kNParams, cudaMemcpyDefault, st);
    if (loss) cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDefault, st);
    return mlp_sync(m, st, "lc_mlp_gradient");
}

// one Adam step on the rows idx[0..B) of (F, T), both device arrays
extern "C" lc_status lc_mlp_train_step(lc_mlp* m, const float* F, const float* T, const int* idx, int B, float lr,
                                       double* loss) {
    if (!m || !F || !T || !idx || B < 1 || !(lr > 0.f)) return LC_ERR_ARG;
    if (!is_dev(F) || !is_dev(T)) return m->fail(LC_ERR_ARG, "lc_mlp_train_step: F and T must be device arrays");
    cudaSetDevice(m->device);
    lc_status s;
    if ((s = m->ensure(B))) return s;
    cudaStream_t st = m->stream;
    cudaMemcpyAsync(m->idx, idx, sizeof(int) * B, cudaMemcpyDefault, st);
    gather_rows_kernel<<<(B * kDIn + 255) / 256, 256, 0, st>>>(F, T, m->idx, B, m->Fin, m->Tin);
    normalise_kernel<<<(unsigned)(((size_t)B * kDIn + 255) / 256), 256, 0, st>>>(m->Fin, m->mu, m->sigma, m->X, B);
    m->forward(B, st);
    m->backward(m->Tin, B, st);
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - powf(b1, (float)m->step), bc2 = 1.f - powf(b2, (float)m->step);
    adam_kernel<<<(kNParams + 255) / 256, 256, 0, st>>>(m->theta, m->grad, m->mom, m->vel, lr, b1, b2, 1e-8f, bc1, bc2);
    m->refresh_weights(st);
    if (loss) {
        cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDefault, st);
        return mlp_sync(m, st, "lc_mlp_train_step");
    }
    return mlp_cuda(m, cudaGetLastError(), "lc_mlp_train_step");
}

// ---------------------------------------------------------------------------
// C ABI: warm start of a capture
// ---------------------------------------------------------------------------
void lc_ctx::warm_release() {
    if (!warm) return;
    if (warm->gexec) cudaGraphExecDestroy(warm->gexec);
    for (void* p : {(void*)warm->F, (void*)warm->Yp, (void*)warm->motion, (void*)warm->Rprev, (void*)warm->tprev,
                    (void*)warm->R0, (void*)warm->t0, (void*)warm->e, (void*)warm->accepted})
        release(p);
    delete warm;
    warm = nullptr;
}

static lc_status warm_ensure(lc_ctx* ctx) {
    const int n = ctx->hC.n;
    if (ctx->warm && ctx->warm->n == n) return LC_OK;
    ctx->warm_release();
    auto* w = new WarmState();
    ctx->warm = w;
    w->n = n;
    w->F = (float*)ctx->alloc(sizeof(float) * 64 * n);
    w->Yp = (float*)ctx->alloc(sizeof(float) * 6 * n);
    w->motion = (float4*)ctx->alloc(sizeof(float4) * 2 * n);
    w->Rprev = (float4*)ctx->alloc(sizeof(float4) * 3 * n);
    w->tprev = (float4*)ctx->alloc(sizeof(float4) * n);
    w->R0 = (float4*)ctx->alloc(sizeof(float4) * 3 * n);
    w->t0 = (float4*)ctx->alloc(sizeof(float4) * n);
    w->e = (double*)ctx->alloc(sizeof(double) * 2);
    w->accepted = (int*)ctx->alloc(sizeof(int));
    if (!w->F || !w->Yp || !w->motion || !w->Rprev || !w->tprev || !w->R0 || !w->t0 || !w->e || !w->accepted)
        return LC_ERR_OOM;
    identity_rows_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(w->Rprev, w->tprev, w->motion, n);
    return ctx->cuda(cudaGetLastError(), "warm-start state");
}

// features at the current node parameters (frame decisions from the last
// visibility pass) into ctx->warm->F
static lc_status warm_features(lc_ctx* ctx) {
    lc_status s;
    if ((s = ctx->linearize_now(true))) return s;
    node_features_kernel<<<(ctx->hC.n + 7) / 8, 256, 0, ctx->stream>>>(ctx->dC, ctx->warm->motion, ctx->warm->F);
    return ctx->cuda(cudaGetLastError(), "node features");
}

extern "C" lc_status lc_node_features(lc_ctx* ctx, float* F) {
    if (!ctx || !F) return LC_ERR_ARG;
    lc_status s;
    if ((s = ctx->check_solve_state("lc_node_features"))) return s;
    if (!ctx->has_vis) return ctx->fail(LC_ERR_STATE, "lc_node_features: no visibility pass yet");
    cudaSetDevice(ctx->device);
    if ((s = warm_ensure(ctx)) || (s = warm_features(ctx))) return s;
    if ((s = ctx->cuda(cudaMemcpyAsync(F, ctx->warm->F, sizeof(float) * 64 * ctx->hC.n, cudaMemcpyDefault, ctx->stream),
                       "copy out")))
        return s;
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
}

extern "C" lc_status lc_record_motion(lc_ctx* ctx) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_graph) return ctx->fail(LC_ERR_STATE, "lc_record_motion: no graph");
    cudaSetDevice(ctx->device);
    lc_status s;
    if ((s = warm_ensure(ctx))) return s;
    WarmState& w = *ctx->warm;
    record_motion_kernel<<<(w.n + 127) / 128, 128, 0, ctx->stream>>>(ctx->dC, w.Rprev, w.tprev, w.motion);
    return ctx->cuda(cudaGetLastError(), "record motion");
}

extern "C" lc_status lc_read_motion(lc_ctx* ctx, float* u) {
    if (!ctx || !u) return LC_ERR_ARG;
    if (!ctx->warm || ctx->warm->n != ctx->hC.n)
        return ctx->fail(LC_ERR_STATE, "lc_read_motion: no motion recorded for this graph");
    cudaSetDevice(ctx->device);
    // float4 rows (x, y, z, 0) -> three floats each: n x (d_omega, d_t)
    lc_status s = ctx->cuda(cudaMemcpy2DAsync(u, 3 * sizeof(float), ctx->warm->motion, sizeof(float4),
                                              3 * sizeof(float), 2 * (size_t)ctx->warm->n, cudaMemcpyDefault,
                                              ctx->stream),
                            "copy out");
    if (s) return s;
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
}

// the warm-start sequence on the context's stream (captured once per network)
static void enqueue_warm(lc_ctx* ctx, lc_mlp* m) {
    WarmState& w = *ctx->warm;
    const int n = ctx->hC.n;
    cudaStream_t st = ctx->stream;
    // frame decisions and linearisation at the start, its energy and features
    launch_warp(ctx->dC, ctx->hC, st);
    launch_vis_unfreeze(ctx->dC, st);
    launch_visibility(ctx->dC, ctx->hC, st);
    cudaMemsetAsync((char*)ctx->hC.sc + offsetof(Scalars, gn_stop), 0, sizeof(int), st);
    launch_warp(ctx->dC, ctx->hC, st);
    launch_linearize(ctx->dC, ctx->hC, true, 0, st);
    launch_rhs(ctx->dC, ctx->hC, LC_MAX_GN, false, st);
    node_features_kernel<<<(n + 7) / 8, 256, 0, st>>>(ctx->dC, w.motion, w.F);
    energy_copy_kernel<<<1, 1, 0, st>>>(ctx->dC, w.e);
    // prediction
    normalise_kernel<<<(unsigned)(((size_t)n * kDIn + 255) / 256), 256, 0, st>>>(w.F, m->mu, m->sigma, m->X, n);
    m->forward(n, st);
    apply_prediction_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctx->dC, m->Y, w.R0, w.t0);
    // energy at the prediction (same frame decisions), then accept or restore
    launch_warp(ctx->dC, ctx->hC, st);
    launch_linearize(ctx->dC, ctx->hC, false, 0, st);
    launch_rhs(ctx->dC, ctx->hC, LC_MAX_GN, true, st);
    energy_copy_kernel<<<1, 1, 0, st>>>(ctx->dC, w.e + 1);
    accept_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctx->dC, w.e, w.R0, w.t0, w.accepted);
}

// Parts of a frame step captured once and replayed (lc_batch_step): the
// allocations first, then the enqueued sequences on ctx->stream.
lc_status warm_step_prepare(lc_ctx* ctx, lc_mlp* m) {
    lc_status s;
    if ((s = warm_ensure(ctx))) return s;
    if (!m) return LC_OK;
    if (m->device != ctx->device) return ctx->fail(LC_ERR_ARG, "lc_batch_step: network on another device");
    if ((s = m->ensure(ctx->hC.n))) return ctx->fail(s, "lc_batch_step: network scratch");
    return LC_OK;
}

void warm_step_enqueue(lc_ctx* ctx, lc_mlp* m) { enqueue_warm(ctx, m); }

void motion_step_enqueue(lc_ctx* ctx) {
    WarmState& w = *ctx->warm;
    record_motion_kernel<<<(w.n + 127) / 128, 128, 0, ctx->stream>>>(ctx->dC, w.Rprev, w.tprev, w.motion);
}

// order a use of the network's buffers on stream st after its earlier work
// (training, other warm starts), and its later work after this use
void mlp_before(lc_mlp* m, cudaStream_t st) {
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, m->stream);
    cudaStreamWaitEvent(st, ev, 0);
    cudaEventDestroy(ev);
}

void mlp_after(lc_mlp* m, cudaStream_t st) {
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, st);
    cudaStreamWaitEvent(m->stream, ev, 0);
    cudaEventDestroy(ev);
}

void mlp_identity(const lc_mlp* m, unsigned long long* uid, unsigned long long* gen) {
    *uid = m ? m->uid : 0;
    *gen = m ? m->gen : 0;
}

extern "C" lc_status lc_warm_start(lc_ctx* ctx, lc_mlp* m, int* accepted, double* energies) {
    if (!ctx || !m) return LC_ERR_ARG;
    lc_status s;
    if ((s = ctx->check_solve_state("lc_warm_start"))) return s;
    if (m->device != ctx->device) return ctx->fail(LC_ERR_ARG, "lc_warm_start: network on another device");
    cudaSetDevice(ctx->device);
    if ((s = warm_ensure(ctx))) return s;
    const int n = ctx->hC.n;
    if ((s = m->ensure(n))) return ctx->fail(s, "lc_warm_start: network scratch");
    WarmState& w = *ctx->warm;
    cudaStream_t st = ctx->stream;
    if (w.gexec && (w.g_uid != m->uid || w.g_gen != m->gen)) {
        cudaGraphExecDestroy(w.gexec);
        w.gexec = nullptr;
    }
    if (!w.gexec) {
        cudaGraph_t g = nullptr;
        if ((s = ctx->cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture"))) return s;
        enqueue_warm(ctx, m);
        const cudaError_t e = cudaStreamEndCapture(st, &g);
        if ((s = ctx->cuda(e, "end capture"))) return s;
        const cudaError_t e2 = cudaGraphInstantiate(&w.gexec, g, 0);
        cudaGraphDestroy(g);
        if ((s = ctx->cuda(e2, "warm-start graph"))) {
            w.gexec = nullptr;
            return s;
        }
        w.g_uid = m->uid;
        w.g_gen = m->gen;
    }
    // the network's previous work (training, other contexts' warm starts)
    // before its buffers are reused here, its later work after
    mlp_before(m, st);
    if ((s = ctx->cuda(cudaGraphLaunch(w.gexec, st), "warm-start graph launch"))) return s;
    ctx->has_vis = true;
    ctx->has_lin = false;
    mlp_after(m, st);
    if (!accepted && !energies) return LC_OK;
    if (accepted && (s = ctx->copy_to_host(accepted, w.accepted, sizeof(int)))) return s;
    if (energies && (s = ctx->copy_to_host(energies, w.e, 2 * sizeof(double)))) return s;
    return LC_OK;
}

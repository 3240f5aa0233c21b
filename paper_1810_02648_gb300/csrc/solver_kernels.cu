// Gauss-Newton / PCG kernels of the non-rigid stage (Sec. 3.4 energy,
// Sec. 4 solver: normal equations J^T J delta = -J^T F, Jacobi-preconditioned
// CG with a fixed iteration count, no damping).
//
// The Jacobian is never stored.  Per vertex i the residual rows r_i
// (3 photometric rows if i is visible, 1 silhouette row if i is in B) depend
// on the node parameters only through the warped position v'_i, so the
// linearisation keeps A_i = d r_i / d v'_i folded into H_i = A_i^T A_i (3x3)
// and e_i = A_i^T r_i.  With a_is = R_k (v_i - g_k) and the left rotation
// increment, d v'_i / d(omega_k, t_k) = w_is [-[a_is]x, I], so
//   (J^T F)_k   = sum_(i,s) w_is [a_is x e_i ; e_i]                 + ARAP
//   (J^T J p)_k = sum_(i,s) w_is [a_is x q_i ; q_i],  q_i = H_i dv_i + ARAP
// with dv_i = sum_s w_is (p_omega,k x a_is + p_t,k).  Per-node sums are
// warp-segmented gathers over the node -> (vertex, weight) CSR (one warp per
// node, shuffle reductions), so there are no floating-point atomics and every
// result is deterministic.  Dot products and energies accumulate in FP64 and
// are reduced per capture by the last tile to finish, in tile order.
#include <algorithm>

#include <cooperative_groups.h>

#include "jtj_pair.cuh"
#include "lc_internal.cuh"

namespace cg = cooperative_groups;

namespace lc {

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

struct Rot {
    float3 r0, r1, r2;
};
__device__ __forceinline__ Rot load_R(const float4* R, int k) {
    const float4 a = R[3 * k], b = R[3 * k + 1], c = R[3 * k + 2];
    return {make_float3(a.x, a.y, a.z), make_float3(b.x, b.y, b.z), make_float3(c.x, c.y, c.z)};
}
__device__ __forceinline__ float3 mul(const Rot& R, float3 v) { return make_float3(dot3(R.r0, v), dot3(R.r1, v), dot3(R.r2, v)); }

// H stored as (h00, h01, h02, h11) + (h12, h22)
__device__ __forceinline__ float3 mulH(float4 A, float4 B, float3 v) {
    return make_float3(A.x * v.x + A.y * v.y + A.z * v.z, A.y * v.x + A.w * v.y + B.x * v.z,
                       A.z * v.x + B.x * v.y + B.y * v.z);
}

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float t) {
    return make_float4(a.x + t * (b.x - a.x), a.y + t * (b.y - a.y), a.z + t * (b.z - a.z), a.w + t * (b.w - a.w));
}
__device__ __forceinline__ float4 sub4(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ __forceinline__ float4 scale4(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }

__device__ __forceinline__ float4 pix(const float4* img, int W, int x, int y) {
    return __ldg(&img[(size_t)y * W + x]);
}

// central difference (one-sided at the border) of all four channels
__device__ __forceinline__ float4 grad_x(const float4* img, int W, int x, int y) {
    if (W < 2) return make_float4(0.f, 0.f, 0.f, 0.f);
    if (x == 0) return sub4(pix(img, W, 1, y), pix(img, W, 0, y));
    if (x == W - 1) return sub4(pix(img, W, W - 1, y), pix(img, W, W - 2, y));
    return scale4(sub4(pix(img, W, x + 1, y), pix(img, W, x - 1, y)), 0.5f);
}
__device__ __forceinline__ float4 grad_y(const float4* img, int W, int H, int x, int y) {
    if (H < 2) return make_float4(0.f, 0.f, 0.f, 0.f);
    if (y == 0) return sub4(pix(img, W, x, 1), pix(img, W, x, 0));
    if (y == H - 1) return sub4(pix(img, W, x, H - 1), pix(img, W, x, H - 2));
    return scale4(sub4(pix(img, W, x, y + 1), pix(img, W, x, y - 1)), 0.5f);
}

// bilinear sample of an image and of its central differences at (u, v),
// clamp to edge
__device__ __forceinline__ void sample_image(const float4* img, int W, int H, float u, float v, float4& I,
                                             float4& Gx, float4& Gy) {
    u = fminf(fmaxf(u, 0.f), (float)(W - 1));
    v = fminf(fmaxf(v, 0.f), (float)(H - 1));
    const int x0 = (int)floorf(u), y0 = (int)floorf(v);
    const float fx = u - (float)x0, fy = v - (float)y0;
    const int x1 = min(x0 + 1, W - 1), y1 = min(y0 + 1, H - 1);
    I = lerp4(lerp4(pix(img, W, x0, y0), pix(img, W, x1, y0), fx), lerp4(pix(img, W, x0, y1), pix(img, W, x1, y1), fx),
              fy);
    Gx = lerp4(lerp4(grad_x(img, W, x0, y0), grad_x(img, W, x1, y0), fx),
               lerp4(grad_x(img, W, x0, y1), grad_x(img, W, x1, y1), fx), fy);
    Gy = lerp4(lerp4(grad_y(img, W, H, x0, y0), grad_y(img, W, H, x1, y0), fx),
               lerp4(grad_y(img, W, H, x0, y1), grad_y(img, W, H, x1, y1), fx), fy);
}

// The same bilinear sample from a staged 4 x 4 patch P (row-major, its
// origin at pixel (x0 - 1, y0 - 1)) when every tap lies inside the image:
// the same operations in the same order as sample_image.
__device__ __forceinline__ void sample_patch(const float4* P, float fx, float fy, float4& I, float4& Gx, float4& Gy) {
    auto p = [&](int x, int y) { return P[4 * y + x]; };
    auto gx = [&](int x, int y) { return scale4(sub4(p(x + 1, y), p(x - 1, y)), 0.5f); };
    auto gy = [&](int x, int y) { return scale4(sub4(p(x, y + 1), p(x, y - 1)), 0.5f); };
    I = lerp4(lerp4(p(1, 1), p(2, 1), fx), lerp4(p(1, 2), p(2, 2), fx), fy);
    Gx = lerp4(lerp4(gx(1, 1), gx(2, 1), fx), lerp4(gx(1, 2), gx(2, 2), fx), fy);
    Gy = lerp4(lerp4(gy(1, 1), gy(2, 1), fx), lerp4(gy(1, 2), gy(2, 2), fx), fy);
}

// mbarrier and bulk-tensor copy primitives (one CTA)
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"((unsigned)__cvta_generic_to_shared(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(bar)),
                 "r"(bytes)
                 : "memory");
}
// bounded wait for phase `parity`; false if it did not complete in time
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int max_tries) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    for (int t = 0; t < max_tries; ++t) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// a box of the 2D tensor map at element coordinates (x, y) into shared memory
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tmap, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            (unsigned)__cvta_generic_to_shared(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"((unsigned)__cvta_generic_to_shared(bar))
        : "memory");
}

constexpr int kTmaPatchBytes = 16 * (int)sizeof(float4);        // 4 x 4 pixels
constexpr int kTmaSmem = kVertTile * kTmaPatchBytes + 128;      // + alignment slack
constexpr int kTmaMaxTries = 1 << 20;

// ---------------------------------------------------------------------------
// Linearisation: residuals, H_i, e_i and the data energy.  With TMA, every
// vertex whose 4 x 4 tap patch lies inside the frame gets it by one
// bulk-tensor copy into its own shared-memory slot (one mbarrier per CTA,
// a bounded wait); the others, and a wait that runs out (flagged in the
// capture's status word), take the global loads.  Both give the same bits.
// ---------------------------------------------------------------------------
template <bool TMA>
__global__ void __launch_bounds__(kVertTile) linearize_kernel(const CapDesc* __restrict__ caps,
                                                               const WorkItem* __restrict__ items, int update_b,
                                                               int gn, const __grid_constant__ CUtensorMap tmap) {
    __shared__ float sh[kVertTile / 32][2];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (update_b && C.sc->gn_stop) return;   // a GN step after the solve reached its target
    const int i = tile * kVertTile + threadIdx.x;
    float enf[2] = {0.f, 0.f};
    uint32_t fl = 0;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 uv = make_float2(0.f, 0.f);
    bool ok = false, ph = false, si = false, masked = false;
    if (i < C.N) {
        fl = C.flags[i];
        v = C.vw[i];
        uv = C.uv[i];
        ok = v.w > 0.f && in_image(uv, C.W, C.H);
        ph = ok && (fl & LC_VIS_BIT);
        si = ok && (fl & LC_INB_BIT);
        if (update_b && si) {
            // b_i follows the current surface; the contour set stays the frame's
            const uint32_t nf = direction_neg(C, i) ? (fl | LC_BNEG_BIT) : (fl & ~LC_BNEG_BIT);
            if (nf != fl) C.flags[i] = nf;
            fl = nf;
        }
        if (si && C.part_on) {
            // body-part mask: the silhouette term is off on another part's region
            const int px = min((int)floorf(uv.x + 0.5f), C.W - 1), py = min((int)floorf(uv.y + 0.5f), C.H - 1);
            const int lab = C.part_mask[(size_t)py * C.W + px];
            masked = lab != 255 && lab != (int)C.vpart[i];
            si = !masked;
        }
    }
    const bool need = i < C.N && (ph || si);
    float4 I = make_float4(0.f, 0.f, 0.f, 0.f), Gx = I, Gy = I;
    if constexpr (TMA) {
        extern __shared__ unsigned char tma_raw[];
        __shared__ __align__(8) uint64_t bar;
        float4* patch = reinterpret_cast<float4*>(((uintptr_t)tma_raw + 127) & ~(uintptr_t)127);
        float fx = 0.f, fy = 0.f;
        int x0 = 0, y0 = 0;
        bool staged = false;
        if (need) {
            const float u = fminf(fmaxf(uv.x, 0.f), (float)(C.W - 1));
            const float w = fminf(fmaxf(uv.y, 0.f), (float)(C.H - 1));
            x0 = (int)floorf(u);
            y0 = (int)floorf(w);
            fx = u - (float)x0;
            fy = w - (float)y0;
            staged = x0 >= 1 && y0 >= 1 && x0 + 2 <= C.W - 1 && y0 + 2 <= C.H - 1;
        }
        if (threadIdx.x == 0) {
            mbar_init(&bar, blockDim.x);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        float4* slot = patch + 16 * threadIdx.x;
        if (staged) {
            mbar_arrive_expect_tx(&bar, kTmaPatchBytes);
            // x in floats: 4 per pixel, so the start is 16-byte aligned
            tma_load_2d(slot, &tmap, 4 * (x0 - 1), y0 - 1, &bar);
        } else {
            mbar_arrive(&bar);
        }
        bool done = mbar_wait(&bar, 0, kTmaMaxTries);
        if (!done) atomicOr(&C.sc->status, kDevErrWait);
        if (staged && done)
            sample_patch(slot, fx, fy, I, Gx, Gy);
        else if (need)
            sample_image(C.img, C.W, C.H, uv.x, uv.y, I, Gx, Gy);
        // no copy may land after the CTA is gone
        if (!done) done = mbar_wait(&bar, 0, kTmaMaxTries);
    } else {
        if (need) sample_image(C.img, C.W, C.H, uv.x, uv.y, I, Gx, Gy);
    }
    if (i < C.N) {
        float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
        float h00 = 0.f, h01 = 0.f, h02 = 0.f, h11 = 0.f, h12 = 0.f, h22 = 0.f;
        float e0 = 0.f, e1 = 0.f, e2 = 0.f;
        if (ph || si) {
            if (ph && C.pyr_levels > 0) {
                // E_photo samples pyramid level j at u_j = (u - (d-1)/2) / d,
                // its gradient scaled by 1/d to full-resolution pixels
                const int j = min(3 - C.pyr_levels + gn, 2);
                const int d = pyr_factor(j);
                const float inv = 1.0f / (float)d, o = 0.5f * (float)(d - 1);
                float4 Il, Gxl, Gyl;
                sample_image(C.lvl[j], C.lvl_W[j], C.lvl_H[j], (uv.x - o) * inv, (uv.y - o) * inv, Il, Gxl, Gyl);
                I = make_float4(Il.x, Il.y, Il.z, I.w);
                Gx = make_float4(Gxl.x * inv, Gxl.y * inv, Gxl.z * inv, Gx.w);
                Gy = make_float4(Gyl.x * inv, Gyl.y * inv, Gyl.z * inv, Gy.w);
            }
            const float iz = 1.0f / v.z;
            const float fz = C.f * iz;
            const float px = -fz * v.x * iz, py = -fz * v.y * iz;   // d pi / dZ terms
            auto add_row = [&](float gx, float gy, float s, float r) {
                const float a0 = s * gx * fz, a1 = s * gy * fz, a2 = s * (gx * px + gy * py);
                h00 += a0 * a0; h01 += a0 * a1; h02 += a0 * a2;
                h11 += a1 * a1; h12 += a1 * a2; h22 += a2 * a2;
                e0 += a0 * r; e1 += a1 * r; e2 += a2 * r;
            };
            if (ph && C.sigma_c > 0.f) {
                // robust colour kernel: prune a correspondence whose colour
                // differs by more than sigma_c (FP32, fixed order)
                const float4 alb = C.albedo[i];
                const float dx = xsub(I.x, alb.x), dy = xsub(I.y, alb.y), dz = xsub(I.z, alb.z);
                const float d2 = xadd(xadd(xmul(dx, dx), xmul(dy, dy)), xmul(dz, dz));
                if (d2 > xmul(C.sigma_c, C.sigma_c)) ph = false;
            }
            if (ph) {
                const float sw = sqrtf(C.w_photo);
                const float4 alb = C.albedo[i];
                res.x = sw * (I.x - alb.x);
                res.y = sw * (I.y - alb.y);
                res.z = sw * (I.z - alb.z);
                add_row(Gx.x, Gy.x, sw, res.x);
                add_row(Gx.y, Gy.y, sw, res.y);
                add_row(Gx.z, Gy.z, sw, res.z);
                enf[0] = res.x * res.x + res.y * res.y + res.z * res.z;
            }
            if (si) {
                const float sw = sqrtf(C.w_sil);
                res.w = sw * I.w;
                const float bs = (fl & LC_BNEG_BIT) ? -sw : sw;
                add_row(Gx.w, Gy.w, bs, res.w);
                enf[1] = res.w * res.w;
            }
        }
        {
            // the bits always reflect this linearisation (cleared when sigma_c / the mask is off)
            const bool pruned = C.sigma_c > 0.f && ok && (fl & LC_VIS_BIT) && !ph;
            uint32_t nf = pruned ? (fl | LC_PRUNED_BIT) : (fl & ~LC_PRUNED_BIT);
            nf = masked ? (nf | LC_MASKED_BIT) : (nf & ~LC_MASKED_BIT);
            if (nf != fl) C.flags[i] = nf;
        }
        C.res[i] = res;
        C.HA[i] = make_float4(h00, h01, h02, h11);
        C.HB[i] = make_float4(h12, h22, 0.f, 0.f);
        C.ev[i] = make_float4(e0, e1, e2, (ph || si) ? 1.f : 0.f);
    }
    double en[2];
    block_sum_f<2, kVertTile / 32>(enf, en, sh);
    reduce_partials<2>(C, CNT_ENERGY, tile, C.vert_tiles, en, [&](const double (&tot)[2]) {
        C.sc->e_lin[0] = tot[0];
        C.sc->e_lin[1] = tot[1];
    });
}

cudaError_t linearize_tma_init() {
    return cudaFuncSetAttribute(linearize_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmem);
}

void launch_linearize(const CapDesc* dC, const Tiles& T, bool update_b, int gn, cudaStream_t st) {
    // work lists span several captures: global loads (the tensor map is per capture)
    static const CUtensorMap none{};
    linearize_kernel<false><<<T.vert, kVertTile, 0, st>>>(dC, T.vert_items, update_b ? 1 : 0, gn, none);
}
void launch_linearize(const CapDesc* dC, const CapDesc& hC, bool update_b, int gn, cudaStream_t st) {
    const Tiles T = single_tiles(hC);
    if (T.tma)
        linearize_kernel<true><<<T.vert, kVertTile, kTmaSmem, st>>>(dC, nullptr, update_b ? 1 : 0, gn, hC.tmap_img);
    else
        launch_linearize(dC, T, update_b, gn, st);
}

// ---------------------------------------------------------------------------
// -J^T F, diag(J^T J) and the ARAP energy (warp per node).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kNodeWarps * 32) rhs_kernel(const CapDesc* __restrict__ caps,
                                                               const WorkItem* __restrict__ items, int slot,
                                                               int energy_only) {
    __shared__ float sh[kNodeWarps][1];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (!energy_only && C.sc->gn_stop) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int k = tile * kNodeTile + w;
    float enf[1] = {0.f};
    if (k < C.n) {
        const Rot R = load_R(C.node_R, k);
        const float3 g = f3(C.node_g[k]), t = f3(C.node_t[k]);
        float acc[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) acc[j] = 0.f;
        if (!energy_only) {
            for (int j = C.ent_off[k] + lane; j < C.ent_off[k + 1]; j += 32) {
                const int2 en2 = C.ent[j];
                const int i = en2.x;
                const float wi = __int_as_float(en2.y);
                const float4 e4 = C.ev[i];
                if (e4.w == 0.f) continue;
                const float3 a = mul(R, f3(C.base[i]) - g);
                const float3 e = f3(e4);
                const float3 c = cross3(a, e);
                acc[0] += wi * c.x; acc[1] += wi * c.y; acc[2] += wi * c.z;
                acc[3] += wi * e.x; acc[4] += wi * e.y; acc[5] += wi * e.z;
                const float4 HA = C.HA[i], HB = C.HB[i];
                // columns of [a]x: a x e_x, a x e_y, a x e_z
                const float3 c0 = make_float3(0.f, a.z, -a.y), c1 = make_float3(-a.z, 0.f, a.x),
                             c2 = make_float3(a.y, -a.x, 0.f);
                const float w2 = wi * wi;
                acc[6] += w2 * dot3(c0, mulH(HA, HB, c0));
                acc[7] += w2 * dot3(c1, mulH(HA, HB, c1));
                acc[8] += w2 * dot3(c2, mulH(HA, HB, c2));
                acc[9] += w2 * HA.x; acc[10] += w2 * HA.w; acc[11] += w2 * HB.y;
            }
        }
        float arap = 0.f;
        for (int j = C.edge_off[k] + lane; j < C.edge_off[k + 1]; j += 32) {
            const int l = C.edge_dst[j];
            const float c = C.w_arap * C.edge_s[j];
            const float3 gl = f3(C.node_g[l]), tl = f3(C.node_t[l]);
            const float3 b = mul(R, gl - g);
            // R_k (g_l - g_k) + g_k + t_k - g_l - t_l, evaluated as
            // (R_k - I)(g_l - g_k) + t_k - t_l: the same value, exactly zero
            // for the identity parameters
            const float3 dg = gl - g;
            const float3 d = (b - dg) + t - tl;
            arap += c * dot3(d, d);
            if (energy_only) continue;
            const float3 bd = cross3(b, d);
            acc[0] += c * bd.x; acc[1] += c * bd.y; acc[2] += c * bd.z;
            acc[3] += c * d.x; acc[4] += c * d.y; acc[5] += c * d.z;
            const float bb = dot3(b, b);
            acc[6] += c * (bb - b.x * b.x); acc[7] += c * (bb - b.y * b.y); acc[8] += c * (bb - b.z * b.z);
            // in-edge (l, k): residual R_l (g_k - g_l) + g_l + t_l - g_k - t_k, d/d t_k = -I
            const Rot Rl = load_R(C.node_R, l);
            const float3 dl = (mul(Rl, g - gl) - (g - gl)) + tl - t;
            acc[3] -= c * dl.x; acc[4] -= c * dl.y; acc[5] -= c * dl.z;
            acc[9] += 2.f * c; acc[10] += 2.f * c; acc[11] += 2.f * c;
        }
        if (!energy_only) {
            warp_sumf<12>(acc);
            if (lane == 0) {
                C.b[2 * k] = make_float4(-acc[0], -acc[1], -acc[2], 0.f);
                C.b[2 * k + 1] = make_float4(-acc[3], -acc[4], -acc[5], 0.f);
                float m[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) m[j] = acc[6 + j] > 0.f ? 1.0f / acc[6 + j] : 0.f;
                C.minv[2 * k] = make_float4(m[0], m[1], m[2], 0.f);
                C.minv[2 * k + 1] = make_float4(m[3], m[4], m[5], 0.f);
                C.diag[2 * k] = make_float4(acc[6], acc[7], acc[8], 0.f);
                C.diag[2 * k + 1] = make_float4(acc[9], acc[10], acc[11], 0.f);
            }
        }
        enf[0] = arap;
    }
    double en[1];
    block_sum_f<1, kNodeWarps>(enf, en, sh);
    reduce_partials<1>(C, CNT_ARAP, tile, C.node_tiles, en, [&](const double (&tot)[1]) {
        Scalars* sc = C.sc;
        sc->e_lin[2] = tot[0];
        const double E = sc->e_lin[0] + sc->e_lin[1] + tot[0];
        C.hist[2 * slot] = E;
        if (!energy_only && C.target_energy > 0.f && E <= (double)C.target_energy) sc->gn_stop = 1;
    });
}

void launch_rhs(const CapDesc* dC, const Tiles& T, int slot, bool energy_only, cudaStream_t st) {
    rhs_kernel<<<T.node, kNodeWarps * 32, 0, st>>>(dC, T.node_items, slot, energy_only ? 1 : 0);
}
void launch_rhs(const CapDesc* dC, const CapDesc& hC, int slot, bool energy_only, cudaStream_t st) {
    launch_rhs(dC, single_tiles(hC), slot, energy_only, st);
}

// ---------------------------------------------------------------------------
// J^T J p: vertex phase (q_i = H_i dv_i), node phase (gather + ARAP), in
// compensated FP32 pairs (jtj_pair.cuh) on FP32 operator data.
//
// The staged coefficients (c_is = w_is R_k (v_i - g_k), w_is) of every
// binding, of every node -> vertex entry, and the rotated offsets of every
// node edge do not change during the PCG, so they are staged once per
// linearisation (the kernels below); the PCG's J^T J p then reads them
// coalesced instead of gathering node rotations and positions.  Only active
// vertices (those with a data row) enter the product, so the staging packs
// them: per chunk of kJChunk vertex ids, the active ones in id order at the
// chunk's start with their coefficients, nodes and H block side by side, and
// per node its active entries at the start of its CSR range, in vertex
// order, as the vertex's compact position and the slot of the binding.  The
// product then reads no byte of an inactive vertex, and the transposed
// product reads the same staged coefficients as the forward one.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kVertTile) jtj_stage_vertex_kernel(const CapDesc* __restrict__ caps,
                                                                      const WorkItem* __restrict__ items) {
    constexpr int kWarps = kVertTile / 32, kChunkWarps = kJChunk / 32;
    __shared__ int wcount[kWarps];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (C.sc->gn_stop) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = tile * kVertTile + threadIdx.x;
    const bool active = i < C.N && C.ev[i].w != 0.f;
    const unsigned bal = __ballot_sync(0xffffffffu, active);
    if (lane == 0) wcount[w] = __popc(bal);
    __syncthreads();
    // rank among the chunk's active vertices: earlier warps of the chunk,
    // then earlier lanes of this warp
    const int w0 = w - w % kChunkWarps;
    int rank = __popc(bal & ((1u << lane) - 1u));
    for (int u = w0; u < w; ++u) rank += wcount[u];
    const int chunk = i / kJChunk;
    if (w == w0 && lane == 0 && chunk * kJChunk < C.N) {
        int total = 0;
        for (int u = w0; u < w0 + kChunkWarps; ++u) total += wcount[u];
        C.vcnt[chunk] = total;
    }
    if (i >= C.N) return;
    const int pos = chunk * kJChunk + rank;
    C.vpos[i] = active ? pos : -1;
    if (!active) return;
    const float4 v = C.base[i];
    const int K = C.K;
    for (int s = 0; s < K; ++s) {
        const size_t e = (size_t)i * K + s;
        const int k = C.bind_idx[e];
        C.vA[(size_t)pos * K + s] = staged_coef(C.node_R, k, v, C.node_g[k], C.bind_w[e]);
        C.vK[(size_t)pos * K + s] = k;
    }
    C.vH[2 * pos] = C.HA[i];
    C.vH[2 * pos + 1] = C.HB[i];
}

__global__ void __launch_bounds__(kNodeWarps * 32) jtj_stage_node_kernel(const CapDesc* __restrict__ caps,
                                                                          const WorkItem* __restrict__ items) {
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (C.sc->gn_stop) return;
    const int lane = threadIdx.x & 31;
    const int k = tile * kNodeTile + (threadIdx.x >> 5);
    if (k >= C.n) return;
    const float4 g = C.node_g[k];
    // the node's active entries packed in CSR order (runs after the vertex
    // stage, whose compact positions it reads); the slot is the vertex's
    // binding to k with the entry's weight
    const int e0 = C.ent_off[k], e1 = C.ent_off[k + 1];
    const int K = C.K;
    int cnt = 0;
    for (int jb = e0; jb < e1; jb += 32) {
        const int j = jb + lane;
        int2 en = make_int2(0, 0);
        int pos = -1;
        if (j < e1) {
            en = C.ent[j];
            pos = C.vpos[en.x];
        }
        const unsigned bal = __ballot_sync(0xffffffffu, pos >= 0);
        if (pos >= 0) {
            int slot = 0;
            for (int s = K - 1; s >= 0; --s) {
                const size_t b = (size_t)en.x * K + s;
                if (C.bind_idx[b] == k && __float_as_int(C.bind_w[b]) == en.y) slot = s;
            }
            C.eV[e0 + cnt + __popc(bal & ((1u << lane) - 1u))] = (pos << 3) | slot;
        }
        cnt += __popc(bal);
    }
    if (lane == 0) C.ecnt[k] = cnt;
    for (int j = C.edge_off[k] + lane; j < C.edge_off[k + 1]; j += 32) {
        const int l = C.edge_dst[j];
        const float4 gl = C.node_g[l];
        const float3 b = staged_edge_offset(C.node_R, k, g, gl);
        const float3 bl = staged_edge_offset(C.node_R, l, gl, g);
        C.dB[2 * j] = make_float4(b.x, b.y, b.z, C.w_arap * C.edge_s[j]);
        C.dB[2 * j + 1] = make_float4(bl.x, bl.y, bl.z, 0.f);
    }
}

void launch_jtj_stage(const CapDesc* dC, const Tiles& T, cudaStream_t st) {
    jtj_stage_vertex_kernel<<<T.vert, kVertTile, 0, st>>>(dC, T.vert_items);
    jtj_stage_node_kernel<<<T.node, kNodeWarps * 32, 0, st>>>(dC, T.node_items);
}
void launch_jtj_stage(const CapDesc* dC, const CapDesc& hC, cudaStream_t st) { launch_jtj_stage(dC, single_tiles(hC), st); }

template <int KT, int VB>
__global__ void __launch_bounds__(VB) jtj_vertex_kernel(const CapDesc* __restrict__ caps,
                                                         const WorkItem* __restrict__ items,
                                                         const float4* __restrict__ p_in,
                                                         const float4* __restrict__ p_lo_in, int check_stop) {
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (check_stop && (C.sc->stop || C.sc->gn_stop)) return;
    // null: the capture's PCG direction (both parts)
    const float4* __restrict__ p = p_in ? p_in : C.p;
    const float4* __restrict__ p_lo = p_in ? p_lo_in : C.p_lo;
    // thread -> (chunk, rank): a block covers VB / kJChunk whole chunks, and
    // only the chunk's active vertices (packed at its start) have work
    static_assert(VB % kJChunk == 0, "vertex blocks hold whole compaction chunks");
    const int chunk = tile * (VB / kJChunk) + threadIdx.x / kJChunk;
    if (chunk * kJChunk >= C.N) return;
    const int r = threadIdx.x % kJChunk;
    if (r >= C.vcnt[chunk]) return;
    const int pos = chunk * kJChunk + r;
    const int K = C.K;
    const float4* __restrict__ A = C.vA + (size_t)pos * K;
    const int* __restrict__ nk = C.vK + (size_t)pos * K;
    constexpr int KM = KT > 0 ? KT : kMaxK;
    const int kk = KT > 0 ? KT : K;
    // all K (coefficient, node) pairs loaded before the p gathers, so the
    // loads of the slots are in flight together
    float4 a[KM];
    int k[KM];
    if constexpr (KT == 4 || KT == 8) {
#pragma unroll
        for (int s = 0; s < KT; s += 4) {
            const int4 k4 = *reinterpret_cast<const int4*>(nk + s);
            k[s] = k4.x; k[s + 1] = k4.y; k[s + 2] = k4.z; k[s + 3] = k4.w;
        }
#pragma unroll
        for (int s = 0; s < KT; ++s) a[s] = A[s];
    } else {
#pragma unroll
        for (int s = 0; s < KM; ++s)
            if (s < kk) {
                a[s] = A[s];
                k[s] = nk[s];
            }
    }
    const float4 HA = C.vH[2 * pos], HB = C.vH[2 * pos + 1];
    fp2acc dv[3];
#pragma unroll
    for (int s = 0; s < KM; ++s)
        if (s < kk) jtj_slot(a[s], node_pair44(p, p_lo, k[s]), dv);
    const float h[6] = {HA.x, HA.y, HA.z, HA.w, HB.x, HB.y};
    const fp2 d[3] = {dv[0].get(), dv[1].get(), dv[2].get()};
    fp2 q[3];
    jtj_block(h, d, q);
    C.q[2 * pos] = make_float4(q[0].h, q[1].h, q[2].h, 1.f);
    C.q[2 * pos + 1] = make_float4(q[0].l, q[1].l, q[2].l, 0.f);
}

// the p . A p total of a capture: alpha = r.z / p.A p as a pair division, or
// a breakdown stop
__device__ __forceinline__ void dot_alpha(const CapDesc& C, double pAp) {
    Scalars* sc = C.sc;
    sc->pAp = pAp;
    if (!(pAp > 0.0)) {
        sc->stop = 1;
        sc->breakdown = 1;
    } else {
        const fp2 alpha = fp2_div(fp2_from_double(sc->rz), fp2_from_double(pAp));
        sc->alpha_h = alpha.h;
        sc->alpha_l = alpha.l;
    }
}

// Sum of a pair over an aligned group of G lanes (fixed xor-shuffle tree;
// every lane of the group gets the total).  Called by all 32 lanes.
template <int G>
__device__ __forceinline__ fp2 fp2_group_sum(fp2 v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        fp2 w;
        w.h = __shfl_xor_sync(0xffffffffu, v.h, o);
        w.l = __shfl_xor_sync(0xffffffffu, v.l, o);
        v = fp2_add(v, w);
    }
    return v;
}

// W warps per block, kJtjNodeLanes lanes per node (kJtjNodesPerWarp nodes per
// warp), U rounds of a node's entries in flight per lane.  Slots walk the
// nodes in the Morton order of their positions (jn_perm), so the nodes of a
// warp are neighbours: similar numbers of active entries (visibility is
// spatially coherent) and shared vertices.  Lane l of a node's group takes
// its active entries l, l + kJtjNodeLanes, ... and edges likewise; the
// group's sums use a fixed shuffle tree, and p . A p is summed per group of
// kNodeTile consecutive slots in one fixed tree, so every launch shape gives
// the same bits.
template <int W, int U>
__global__ void __launch_bounds__(W * 32) jtj_node_kernel(const CapDesc* __restrict__ caps,
                                                          const WorkItem* __restrict__ items,
                                                          const float4* __restrict__ p_in,
                                                          const float4* __restrict__ p_lo_in,
                                                          float4* __restrict__ out_in,
                                                          float4* __restrict__ out_lo_in, int dot) {
    constexpr int NPB = W * kJtjNodesPerWarp;   // nodes per block
    constexpr int NG = NPB / kNodeTile;      // p . A p partial groups per block
    static_assert(NPB % kNodeTile == 0 && NG <= W, "whole partial groups, one warp to sum each");
    __shared__ float2 sh[NPB];
    __shared__ float2 gs[NG];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (dot && (C.sc->stop || C.sc->gn_stop)) return;
    // null: the capture's p and Ap (both parts); out_lo null: the low part is dropped
    const float4* __restrict__ p = p_in ? p_in : C.p;
    const float4* __restrict__ p_lo = p_in ? p_lo_in : C.p_lo;
    float4* __restrict__ out = out_in ? out_in : C.Ap;
    float4* __restrict__ out_lo = out_in ? out_lo_in : C.Ap_lo;
    const int g = threadIdx.x / kJtjNodeLanes, sl = threadIdx.x % kJtjNodeLanes;
    const int slot = tile * NPB + g;
    const bool has = slot < C.n;
    const int k = has ? C.jn_perm[slot] : 0;
    // every lane runs the group sums below; a node past the end has no work
    int e0 = 0, e1 = 0, d0 = 0, d1 = 0;
    if (has) {
        e0 = C.ent_off[k];
        e1 = e0 + C.ecnt[k];   // the node's active entries only (packed at the start of its range)
        d0 = C.edge_off[k];
        d1 = C.edge_off[k + 1];
    }
    fp2acc acc[6];
    const int K = C.K;
    // U rounds of the node's entries at a time: their loads are issued
    // together before any result is used; an entry's coefficient is its
    // vertex's staged binding (compact position, slot)
    for (int jb = e0 + sl; jb < e1; jb += kJtjNodeLanes * U) {
        int vi[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = jb + kJtjNodeLanes * u;
            vi[u] = j < e1 ? C.eV[j] : -1;
        }
        float4 a[U], qh[U], ql[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool on = vi[u] >= 0;
            const int pos = vi[u] >> 3;
            a[u] = on ? C.vA[(size_t)pos * K + (vi[u] & 7)] : make_float4(0.f, 0.f, 0.f, 0.f);
            qh[u] = on ? C.q[2 * pos] : make_float4(0.f, 0.f, 0.f, 0.f);
            ql[u] = on ? C.q[2 * pos + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (vi[u] < 0) continue;
            const fp2 q[3] = {{qh[u].x, ql[u].x}, {qh[u].y, ql[u].y}, {qh[u].z, ql[u].z}};
            jtj_entry(a[u], q, acc);
        }
    }
    NodeP pk{};
    if (has) pk = node_pair44(p, p_lo, k);
    for (int j = d0 + sl; j < d1; j += kJtjNodeLanes)
        jtj_edge(C.dB[2 * j], C.dB[2 * j + 1], pk, node_pair44(p, p_lo, C.edge_dst[j]), acc);
    fp2 t[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) t[c] = fp2_group_sum<kJtjNodeLanes>(acc[c].get());
    fp2 pap_k = {0.f, 0.f};
    if (has && sl == 0) {
        out[2 * k] = make_float4(t[0].h, t[1].h, t[2].h, 0.f);
        out[2 * k + 1] = make_float4(t[3].h, t[4].h, t[5].h, 0.f);
        if (out_lo) {
            out_lo[2 * k] = make_float4(t[0].l, t[1].l, t[2].l, 0.f);
            out_lo[2 * k + 1] = make_float4(t[3].l, t[4].l, t[5].l, 0.f);
        }
        if (dot) {
            fp2acc pap;
            pap.mac(pk.w[0], t[0]); pap.mac(pk.w[1], t[1]); pap.mac(pk.w[2], t[2]);
            pap.mac(pk.t[0], t[3]); pap.mac(pk.t[1], t[4]); pap.mac(pk.t[2], t[5]);
            pap_k = pap.get();
        }
    }
    if (!dot) return;
    // per group of kNodeTile nodes: warp r sums group r's node terms in its
    // first kNodeTile lanes
    if (sl == 0) sh[g] = make_float2(pap_k.h, pap_k.l);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w < NG) {
        const float2 v = lane < kNodeTile ? sh[w * kNodeTile + lane] : make_float2(0.f, 0.f);
        const fp2 s = fp2_warp_sum(fp2{v.x, v.y});
        if (lane == 0) gs[w] = make_float2(s.h, s.l);
    }
    __syncthreads();
    const int t0 = tile * NG;
    const int m = min(NG, C.node_tiles - t0);
    double part[NG][1];
#pragma unroll
    for (int r = 0; r < NG; ++r) part[r][0] = fp2_to_double(fp2{gs[r].x, gs[r].y});
    if (!publish_partials<1>(C, CNT_DOT, t0, m, C.node_tiles, part, C.part)) return;
    if (threadIdx.x >= 32) return;
    double tot[1];
    sum_partials_warp<1>(C.part, C.node_tiles, tot);
    if (threadIdx.x == 0) dot_alpha(C, tot[0]);
}

template <int VB>
static void launch_jtj_vertex(const CapDesc* dC, const Tiles& T, const float4* p, const float4* p_lo, bool dot,
                              cudaStream_t st, int K) {
    if (K == 4)
        jtj_vertex_kernel<4, VB><<<T.jv, VB, 0, st>>>(dC, T.jv_items, p, p_lo, dot ? 1 : 0);
    else if (K == 8)
        jtj_vertex_kernel<8, VB><<<T.jv, VB, 0, st>>>(dC, T.jv_items, p, p_lo, dot ? 1 : 0);
    else
        jtj_vertex_kernel<0, VB><<<T.jv, VB, 0, st>>>(dC, T.jv_items, p, p_lo, dot ? 1 : 0);
}

template <int W>
static void launch_jtj_node(const CapDesc* dC, const Tiles& T, const float4* p, const float4* p_lo, float4* out,
                            float4* out_lo, bool dot, cudaStream_t st) {
    const int d = dot ? 1 : 0;
    if (T.jn_unroll == 2)
        jtj_node_kernel<W, 2><<<T.jn, W * 32, 0, st>>>(dC, T.jn_items, p, p_lo, out, out_lo, d);
    else if (T.jn_unroll == 8)
        jtj_node_kernel<W, 8><<<T.jn, W * 32, 0, st>>>(dC, T.jn_items, p, p_lo, out, out_lo, d);
    else
        jtj_node_kernel<W, 4><<<T.jn, W * 32, 0, st>>>(dC, T.jn_items, p, p_lo, out, out_lo, d);
}

bool jtj_shape_valid(int vert_block, int node_warps, int node_unroll) {
    return (vert_block == 128 || vert_block == 256 || vert_block == 512) &&
           (node_warps == 4 || node_warps == 8 || node_warps == 16) &&
           (node_unroll == 2 || node_unroll == 4 || node_unroll == 8);
}

void launch_jtj(const CapDesc* dC, const Tiles& T, const float4* p, const float4* p_lo, float4* out,
                float4* out_lo, bool dot, cudaStream_t st) {
    if (T.jv_block == 128)
        launch_jtj_vertex<128>(dC, T, p, p_lo, dot, st, T.jk);
    else if (T.jv_block == 512)
        launch_jtj_vertex<512>(dC, T, p, p_lo, dot, st, T.jk);
    else
        launch_jtj_vertex<256>(dC, T, p, p_lo, dot, st, T.jk);
    if (T.jn_warps == 16)
        launch_jtj_node<16>(dC, T, p, p_lo, out, out_lo, dot, st);
    else if (T.jn_warps == 8)
        launch_jtj_node<8>(dC, T, p, p_lo, out, out_lo, dot, st);
    else
        launch_jtj_node<4>(dC, T, p, p_lo, out, out_lo, dot, st);
}
void launch_jtj(const CapDesc* dC, const CapDesc& hC, const float4* p, const float4* p_lo, float4* out,
                float4* out_lo, bool dot, cudaStream_t st) {
    launch_jtj(dC, single_tiles(hC), p, p_lo, out, out_lo, dot, st);
}

// ---------------------------------------------------------------------------
// PCG vector kernels (node-parallel, 2 float4 per node for each part of a
// pair; dot products as pairs per tile, FP64 across tiles).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }

// the three components of element j of a pair vector
__device__ __forceinline__ void load_pair3(const float4* hi, const float4* lo, int j, fp2 (&v)[3]) {
    const float4 h = hi[j], l = lo[j];
    v[0] = {h.x, l.x};
    v[1] = {h.y, l.y};
    v[2] = {h.z, l.z};
}
__device__ __forceinline__ void store_pair3(float4* hi, float4* lo, int j, const fp2 (&v)[3]) {
    hi[j] = make_float4(v[0].h, v[1].h, v[2].h, 0.f);
    lo[j] = make_float4(v[0].l, v[1].l, v[2].l, 0.f);
}

__global__ void __launch_bounds__(kVecThreads) pcg_init_kernel(const CapDesc* __restrict__ caps,
                                                                const WorkItem* __restrict__ items) {
    __shared__ float2 sh[kVecThreads / 32];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (C.sc->gn_stop) return;
    const int k = tile * kVecThreads + threadIdx.x;
    fp2acc rz;
    if (k < C.n) {
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * k + h;
            const float4 b = C.b[j], mi = C.minv[j];
            const fp2 z[3] = {two_prod(mi.x, b.x), two_prod(mi.y, b.y), two_prod(mi.z, b.z)};
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            C.x[j] = zero;
            C.x_lo[j] = zero;
            C.r[j] = make_float4(b.x, b.y, b.z, 0.f);
            C.r_lo[j] = zero;
            store_pair3(C.z, C.z_lo, j, z);
            store_pair3(C.p, C.p_lo, j, z);
            rz.mac(b.x, z[0]); rz.mac(b.y, z[1]); rz.mac(b.z, z[2]);
        }
    }
    const int ntiles = (C.n + kVecThreads - 1) / kVecThreads;
    const fp2 tot = block_sum_fp2<kVecThreads / 32>(rz.get(), sh);
    const double part[1] = {fp2_to_double(tot)};
    reduce_partials<1>(C, CNT_DOT2, tile, ntiles, part, [&](const double (&sum)[1]) {
        Scalars* sc = C.sc;
        sc->rz = sum[0];
        sc->stop = sum[0] == 0.0 ? 1 : 0;
        sc->breakdown = 0;
        sc->iters = 0;
    });
}

__global__ void __launch_bounds__(kVecThreads) pcg_step_kernel(const CapDesc* __restrict__ caps,
                                                                const WorkItem* __restrict__ items) {
    __shared__ float2 sh[kVecThreads / 32];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    Scalars* sc = C.sc;
    if (sc->stop || sc->gn_stop) return;
    const fp2 alpha = {sc->alpha_h, sc->alpha_l};
    const int k = tile * kVecThreads + threadIdx.x;
    fp2acc rz;
    if (k < C.n) {
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * k + h;
            fp2 p[3], x[3], r[3], ap[3], z[3];
            load_pair3(C.p, C.p_lo, j, p);
            load_pair3(C.x, C.x_lo, j, x);
            load_pair3(C.r, C.r_lo, j, r);
            load_pair3(C.Ap, C.Ap_lo, j, ap);
            const float4 mi = C.minv[j];
            const float m[3] = {mi.x, mi.y, mi.z};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                x[c] = fp2_add(x[c], fp2_mul(alpha, p[c]));
                r[c] = fp2_sub(r[c], fp2_mul(alpha, ap[c]));
                z[c] = fp2_scale(m[c], r[c]);
                rz.mac(r[c], z[c]);
            }
            store_pair3(C.x, C.x_lo, j, x);
            store_pair3(C.r, C.r_lo, j, r);
            store_pair3(C.z, C.z_lo, j, z);
        }
    }
    const int ntiles = (C.n + kVecThreads - 1) / kVecThreads;
    const fp2 tot = block_sum_fp2<kVecThreads / 32>(rz.get(), sh);
    const double part[1] = {fp2_to_double(tot)};
    reduce_partials<1>(C, CNT_DOT2, tile, ntiles, part, [&](const double (&sum)[1]) {
        sc->iters += 1;
        sc->rz_new = sum[0];
        if (sum[0] == 0.0) {
            sc->stop = 1;
        } else {
            // every other tile has read its inputs already (it finished before this one)
            const fp2 beta = fp2_div(fp2_from_double(sum[0]), fp2_from_double(sc->rz));
            sc->beta_h = beta.h;
            sc->beta_l = beta.l;
            sc->beta = sum[0] / sc->rz;
            sc->rz = sum[0];
        }
    });
}

__global__ void __launch_bounds__(kVecThreads) pcg_dir_kernel(const CapDesc* __restrict__ caps,
                                                               const WorkItem* __restrict__ items) {
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    Scalars* sc = C.sc;
    if (sc->stop || sc->gn_stop) return;
    const fp2 beta = {sc->beta_h, sc->beta_l};
    const int k = tile * kVecThreads + threadIdx.x;
    if (k < C.n) {
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * k + h;
            fp2 p[3], z[3];
            load_pair3(C.p, C.p_lo, j, p);
            load_pair3(C.z, C.z_lo, j, z);
#pragma unroll
            for (int c = 0; c < 3; ++c) p[c] = fp2_add(z[c], fp2_mul(beta, p[c]));
            store_pair3(C.p, C.p_lo, j, p);
        }
    }
}

void launch_pcg_init(const CapDesc* dC, const Tiles& T, cudaStream_t st) {
    pcg_init_kernel<<<T.vec, kVecThreads, 0, st>>>(dC, T.vec_items);
}
void launch_pcg_init(const CapDesc* dC, const CapDesc& hC, cudaStream_t st) { launch_pcg_init(dC, single_tiles(hC), st); }

void launch_pcg_vectors(const CapDesc* dC, const Tiles& T, cudaStream_t st) {
    pcg_step_kernel<<<T.vec, kVecThreads, 0, st>>>(dC, T.vec_items);
    pcg_dir_kernel<<<T.vec, kVecThreads, 0, st>>>(dC, T.vec_items);
}
void launch_pcg_vectors(const CapDesc* dC, const CapDesc& hC, cudaStream_t st) {
    launch_pcg_vectors(dC, single_tiles(hC), st);
}

// ---------------------------------------------------------------------------
// Parameter update: R_k <- Exp(d_omega_k) R_k, t_k += d_t_k.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kVecThreads) update_kernel(const CapDesc* __restrict__ caps,
                                                              const WorkItem* __restrict__ items, int slot) {
    __shared__ float2 sh[kVecThreads / 32];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (C.sc->gn_stop) return;
    const int k = tile * kVecThreads + threadIdx.x;
    fp2acc s2a;   // ||delta||^2 as a pair (exact products)
    if (k < C.n) {
        const float4 xw = C.x[2 * k], xt = C.x[2 * k + 1];
        s2a.mac(xw.x, xw.x); s2a.mac(xw.y, xw.y); s2a.mac(xw.z, xw.z);
        s2a.mac(xt.x, xt.x); s2a.mac(xt.y, xt.y); s2a.mac(xt.z, xt.z);
        const float th2 = xw.x * xw.x + xw.y * xw.y + xw.z * xw.z;
        const float th = sqrtf(th2);
        float A, B;
        if (th < 1e-4f) {
            A = 1.f - th2 * (1.f / 6.f);
            B = 0.5f - th2 * (1.f / 24.f);
        } else {
            const float sh2 = sinf(0.5f * th);
            A = sinf(th) / th;
            B = 2.f * sh2 * sh2 / th2;
        }
        // E = I + A [w]x + B [w]x^2
        const float wx = xw.x, wy = xw.y, wz = xw.z;
        const float E00 = 1.f - B * (wy * wy + wz * wz), E11 = 1.f - B * (wx * wx + wz * wz),
                    E22 = 1.f - B * (wx * wx + wy * wy);
        const float E01 = -A * wz + B * wx * wy, E10 = A * wz + B * wx * wy;
        const float E02 = A * wy + B * wx * wz, E20 = -A * wy + B * wx * wz;
        const float E12 = -A * wx + B * wy * wz, E21 = A * wx + B * wy * wz;
        const float4 r0 = C.node_R[3 * k], r1 = C.node_R[3 * k + 1], r2 = C.node_R[3 * k + 2];
        C.node_R[3 * k] = make_float4(E00 * r0.x + E01 * r1.x + E02 * r2.x, E00 * r0.y + E01 * r1.y + E02 * r2.y,
                                      E00 * r0.z + E01 * r1.z + E02 * r2.z, 0.f);
        C.node_R[3 * k + 1] = make_float4(E10 * r0.x + E11 * r1.x + E12 * r2.x, E10 * r0.y + E11 * r1.y + E12 * r2.y,
                                          E10 * r0.z + E11 * r1.z + E12 * r2.z, 0.f);
        C.node_R[3 * k + 2] = make_float4(E20 * r0.x + E21 * r1.x + E22 * r2.x, E20 * r0.y + E21 * r1.y + E22 * r2.y,
                                          E20 * r0.z + E21 * r1.z + E22 * r2.z, 0.f);
        const float4 t = C.node_t[k];
        C.node_t[k] = make_float4(t.x + xt.x, t.y + xt.y, t.z + xt.z, 0.f);
    }
    const int ntiles = (C.n + kVecThreads - 1) / kVecThreads;
    const fp2 s2t = block_sum_fp2<kVecThreads / 32>(s2a.get(), sh);
    const double s2[1] = {fp2_to_double(s2t)};
    reduce_partials<1>(C, CNT_STEP, tile, ntiles, s2, [&](const double (&tot)[1]) {
        Scalars* sc = C.sc;
        sc->step2 = tot[0];
        C.hist[2 * slot + 1] = sqrt(tot[0]);
        C.hist_iters[slot] = sc->iters;
        C.hist_iters[LC_MAX_GN + 1] += sc->breakdown;
        sc->gn_done = slot + 1;
    });
}

void launch_update(const CapDesc* dC, const Tiles& T, int gn_slot, cudaStream_t st) {
    update_kernel<<<T.vec, kVecThreads, 0, st>>>(dC, T.vec_items, gn_slot);
}
void launch_update(const CapDesc* dC, const CapDesc& hC, int gn_slot, cudaStream_t st) {
    launch_update(dC, single_tiles(hC), gn_slot, st);
}

// ---------------------------------------------------------------------------
// Condition of the next Gauss-Newton step's conditional graph node: the
// solve goes on unless it reached its target energy.
// ---------------------------------------------------------------------------
__global__ void gn_gate_kernel(const CapDesc* __restrict__ caps, cudaGraphConditionalHandle next) {
    cudaGraphSetConditional(next, caps[0].sc->gn_stop ? 0u : 1u);
}

void launch_gn_gate(const CapDesc* dC, cudaGraphConditionalHandle next, cudaStream_t st) {
    gn_gate_kernel<<<1, 1, 0, st>>>(dC, next);
}

// ---------------------------------------------------------------------------
// 6n <-> two float4 per node
// ---------------------------------------------------------------------------
__global__ void pack_vec_kernel(const float* __restrict__ in, float4* __restrict__ out, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    out[2 * k] = make_float4(in[6 * k], in[6 * k + 1], in[6 * k + 2], 0.f);
    out[2 * k + 1] = make_float4(in[6 * k + 3], in[6 * k + 4], in[6 * k + 5], 0.f);
}
__global__ void unpack_vec_kernel(const float4* __restrict__ in, float* __restrict__ out, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float4 a = in[2 * k], b = in[2 * k + 1];
    out[6 * k] = a.x; out[6 * k + 1] = a.y; out[6 * k + 2] = a.z;
    out[6 * k + 3] = b.x; out[6 * k + 4] = b.y; out[6 * k + 5] = b.z;
}
void launch_pack_vec(const float* in6, float4* out, int n, cudaStream_t st) {
    pack_vec_kernel<<<(n + 127) / 128, 128, 0, st>>>(in6, out, n);
}
void launch_unpack_vec(const float4* in, float* out6, int n, cudaStream_t st) {
    unpack_vec_kernel<<<(n + 127) / 128, 128, 0, st>>>(in, out6, n);
}

}  // namespace lc

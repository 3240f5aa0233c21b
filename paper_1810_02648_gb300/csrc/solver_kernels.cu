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

// ---------------------------------------------------------------------------
// Linearisation: residuals, H_i, e_i and the data energy.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kVertTile) linearize_kernel(const CapDesc* __restrict__ caps,
                                                               const WorkItem* __restrict__ items, int update_b,
                                                               int gn) {
    __shared__ float sh[kVertTile / 32][2];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (update_b && C.sc->gn_stop) return;   // a GN step after the solve reached its target
    const int i = tile * kVertTile + threadIdx.x;
    float enf[2] = {0.f, 0.f};
    if (i < C.N) {
        uint32_t fl = C.flags[i];
        const float4 v = C.vw[i];
        const float2 uv = C.uv[i];
        const bool ok = v.w > 0.f && in_image(uv, C.W, C.H);
        bool ph = ok && (fl & LC_VIS_BIT);
        bool si = ok && (fl & LC_INB_BIT);
        if (update_b && si) {
            // b_i follows the current surface; the contour set stays the frame's
            const uint32_t nf = direction_neg(C, i) ? (fl | LC_BNEG_BIT) : (fl & ~LC_BNEG_BIT);
            if (nf != fl) C.flags[i] = nf;
            fl = nf;
        }
        bool masked = false;
        if (si && C.part_on) {
            // body-part mask: the silhouette term is off on another part's region
            const int px = min((int)floorf(uv.x + 0.5f), C.W - 1), py = min((int)floorf(uv.y + 0.5f), C.H - 1);
            const int lab = C.part_mask[(size_t)py * C.W + px];
            masked = lab != 255 && lab != (int)C.vpart[i];
            si = !masked;
        }
        float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
        float h00 = 0.f, h01 = 0.f, h02 = 0.f, h11 = 0.f, h12 = 0.f, h22 = 0.f;
        float e0 = 0.f, e1 = 0.f, e2 = 0.f;
        if (ph || si) {
            float4 I, Gx, Gy;
            sample_image(C.img, C.W, C.H, uv.x, uv.y, I, Gx, Gy);
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

void launch_linearize(const CapDesc* dC, const Tiles& T, bool update_b, int gn, cudaStream_t st) {
    linearize_kernel<<<T.vert, kVertTile, 0, st>>>(dC, T.vert_items, update_b ? 1 : 0, gn);
}
void launch_linearize(const CapDesc* dC, const CapDesc& hC, bool update_b, int gn, cudaStream_t st) {
    launch_linearize(dC, single_tiles(hC), update_b, gn, st);
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
// J^T J p: vertex phase (q_i = H_i dv_i), node phase (gather + ARAP).
//
// The rotated offsets a_is = R_k (v_i - g_k) of every binding, of every node
// -> vertex entry, and of every node edge do not change during the PCG, so
// they are staged once per linearisation (the kernels below); the PCG's
// J^T J p then reads them coalesced instead of gathering node rotations and
// positions, and skips inactive vertices without touching them.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kVertTile) jtj_stage_vertex_kernel(const CapDesc* __restrict__ caps,
                                                                      const WorkItem* __restrict__ items) {
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (C.sc->gn_stop) return;
    const int i = tile * kVertTile + threadIdx.x;
    if (i >= C.N) return;
    const bool active = C.ev[i].w != 0.f;
    const float3 v = f3(C.base[i]);
    const int K = C.K;
    for (int s = 0; s < K; ++s) {
        const size_t e = (size_t)i * K + s;
        const int k = C.bind_idx[e];
        const float3 a = mul(load_R(C.node_R, k), v - f3(C.node_g[k]));
        C.vA[e] = make_float4(a.x, a.y, a.z, active ? C.bind_w[e] : 0.f);
    }
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
    const Rot R = load_R(C.node_R, k);
    const float3 g = f3(C.node_g[k]);
    for (int j = C.ent_off[k] + lane; j < C.ent_off[k + 1]; j += 32) {
        const int2 en = C.ent[j];
        const bool active = C.ev[en.x].w != 0.f;
        const float3 a = mul(R, f3(C.base[en.x]) - g);
        C.eA[j] = make_float4(a.x, a.y, a.z, active ? __int_as_float(en.y) : 0.f);
    }
    for (int j = C.edge_off[k] + lane; j < C.edge_off[k + 1]; j += 32) {
        const int l = C.edge_dst[j];
        const float3 gl = f3(C.node_g[l]);
        const float3 b = mul(R, gl - g);
        const float3 bl = mul(load_R(C.node_R, l), g - gl);
        C.dB[2 * j] = make_float4(b.x, b.y, b.z, C.w_arap * C.edge_s[j]);
        C.dB[2 * j + 1] = make_float4(bl.x, bl.y, bl.z, 0.f);
    }
}

void launch_jtj_stage(const CapDesc* dC, const Tiles& T, cudaStream_t st) {
    jtj_stage_vertex_kernel<<<T.vert, kVertTile, 0, st>>>(dC, T.vert_items);
    jtj_stage_node_kernel<<<T.node, kNodeWarps * 32, 0, st>>>(dC, T.node_items);
}
void launch_jtj_stage(const CapDesc* dC, const CapDesc& hC, cudaStream_t st) { launch_jtj_stage(dC, single_tiles(hC), st); }

template <int KT>
__device__ __forceinline__ float3 vertex_dv(const float4* __restrict__ A, const int* __restrict__ idx,
                                            const float4* __restrict__ p, int K) {
    // all K (offset, node) pairs loaded before the p gathers, so the loads of
    // the slots are in flight together
    constexpr int KM = KT > 0 ? KT : kMaxK;
    const int kk = KT > 0 ? KT : K;
    float4 a[KM];
    int k[KM];
#pragma unroll
    for (int s = 0; s < KM; ++s)
        if (s < kk) {
            a[s] = A[s];
            k[s] = idx[s];
        }
    float3 dv = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int s = 0; s < KM; ++s)
        if (s < kk) {
            const float3 pw = f3(p[2 * k[s]]), pt = f3(p[2 * k[s] + 1]);
            dv = dv + a[s].w * (cross3(pw, f3(a[s])) + pt);
        }
    return dv;
}

template <int KT>
__global__ void __launch_bounds__(kVertTile) jtj_vertex_kernel(const CapDesc* __restrict__ caps,
                                                                const WorkItem* __restrict__ items,
                                                                const float4* __restrict__ p_in, int check_stop) {
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (check_stop && (C.sc->stop || C.sc->gn_stop)) return;
    const float4* __restrict__ p = p_in ? p_in : C.p;   // null: the capture's PCG direction
    const int i = tile * kVertTile + threadIdx.x;
    if (i >= C.N) return;
    const int K = C.K;
    const float4* __restrict__ A = C.vA + (size_t)i * K;
    if (A[0].w == 0.f) return;   // inactive vertex: no entry of the node phase reads its q
    const float3 dv = vertex_dv<KT>(A, C.bind_idx + (size_t)i * K, p, K);
    const float3 q = mulH(C.HA[i], C.HB[i], dv);
    C.q[i] = make_float4(q.x, q.y, q.z, 1.f);
}

__global__ void __launch_bounds__(kNodeWarps * 32) jtj_node_kernel(const CapDesc* __restrict__ caps,
                                                                    const WorkItem* __restrict__ items,
                                                                    const float4* __restrict__ p_in,
                                                                    float4* __restrict__ out_in, int dot) {
    __shared__ float sh[kNodeWarps][1];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (dot && (C.sc->stop || C.sc->gn_stop)) return;
    const float4* __restrict__ p = p_in ? p_in : C.p;   // null: the capture's p and Ap
    float4* __restrict__ out = out_in ? out_in : C.Ap;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int k = tile * kNodeTile + w;
    float papf[1] = {0.f};
    if (k < C.n) {
        const float3 pw = f3(p[2 * k]), pt = f3(p[2 * k + 1]);
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        // four rounds of the node's entries at a time: their loads are issued
        // together before any result is used
        constexpr int U = 4;
        const int e0 = C.ent_off[k], e1 = C.ent_off[k + 1];
        for (int jb = e0 + lane; jb < e1; jb += 32 * U) {
            float4 a[U];
            int vi[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = jb + 32 * u;
                a[u] = j < e1 ? C.eA[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                vi[u] = j < e1 ? C.ent[j].x : 0;
            }
            float4 q4[U];
#pragma unroll
            for (int u = 0; u < U; ++u) q4[u] = a[u].w != 0.f ? C.q[vi[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float3 q = f3(q4[u]);
                const float3 c = cross3(f3(a[u]), q);
                const float wv = a[u].w;
                acc[0] += wv * c.x; acc[1] += wv * c.y; acc[2] += wv * c.z;
                acc[3] += wv * q.x; acc[4] += wv * q.y; acc[5] += wv * q.z;
            }
        }
        for (int j = C.edge_off[k] + lane; j < C.edge_off[k + 1]; j += 32) {
            const int l = C.edge_dst[j];
            const float4 bk = C.dB[2 * j], bl = C.dB[2 * j + 1];
            const float c = bk.w;
            const float3 plw = f3(p[2 * l]), plt = f3(p[2 * l + 1]);
            const float3 D = cross3(pw, f3(bk)) + pt - plt;
            const float3 bD = cross3(f3(bk), D);
            acc[0] += c * bD.x; acc[1] += c * bD.y; acc[2] += c * bD.z;
            acc[3] += c * D.x; acc[4] += c * D.y; acc[5] += c * D.z;
            const float3 Dl = cross3(plw, f3(bl)) + plt - pt;
            acc[3] -= c * Dl.x; acc[4] -= c * Dl.y; acc[5] -= c * Dl.z;
        }
        warp_sumf<6>(acc);
        if (lane == 0) {
            out[2 * k] = make_float4(acc[0], acc[1], acc[2], 0.f);
            out[2 * k + 1] = make_float4(acc[3], acc[4], acc[5], 0.f);
        }
        if (dot && lane == 0)
            papf[0] = pw.x * acc[0] + pw.y * acc[1] + pw.z * acc[2] + pt.x * acc[3] + pt.y * acc[4] + pt.z * acc[5];
    }
    if (!dot) return;
    double pap[1];
    block_sum_f<1, kNodeWarps>(papf, pap, sh);
    reduce_partials<1>(C, CNT_DOT, tile, C.node_tiles, pap, [&](const double (&tot)[1]) {
        Scalars* sc = C.sc;
        sc->pAp = tot[0];
        if (!(tot[0] > 0.0)) {
            sc->stop = 1;
            sc->breakdown = 1;
        } else {
            sc->alpha = __fdiv_rn((float)sc->rz, (float)tot[0]);
        }
    });
}

void launch_jtj(const CapDesc* dC, const Tiles& T, const float4* p, float4* out, bool dot, cudaStream_t st, int K) {
    if (K == 4)
        jtj_vertex_kernel<4><<<T.vert, kVertTile, 0, st>>>(dC, T.vert_items, p, dot ? 1 : 0);
    else if (K == 8)
        jtj_vertex_kernel<8><<<T.vert, kVertTile, 0, st>>>(dC, T.vert_items, p, dot ? 1 : 0);
    else
        jtj_vertex_kernel<0><<<T.vert, kVertTile, 0, st>>>(dC, T.vert_items, p, dot ? 1 : 0);
    jtj_node_kernel<<<T.node, kNodeWarps * 32, 0, st>>>(dC, T.node_items, p, out, dot ? 1 : 0);
}
void launch_jtj(const CapDesc* dC, const CapDesc& hC, const float4* p, float4* out, bool dot, cudaStream_t st) {
    launch_jtj(dC, single_tiles(hC), p, out, dot, st, hC.K);
}

// ---------------------------------------------------------------------------
// PCG vector kernels (node-parallel, 2 float4 per node, FP64 dots).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ float4 mul4(float4 a, float4 b) { return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w); }
__device__ __forceinline__ float4 axpy4(float a, float4 x, float4 y) {
    return make_float4(y.x + a * x.x, y.y + a * x.y, y.z + a * x.z, y.w + a * x.w);
}

__global__ void __launch_bounds__(kVecThreads) pcg_init_kernel(const CapDesc* __restrict__ caps,
                                                                const WorkItem* __restrict__ items) {
    __shared__ float sh[kVecThreads / 32][1];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (C.sc->gn_stop) return;
    const int k = tile * kVecThreads + threadIdx.x;
    float rzf[1] = {0.f};
    if (k < C.n) {
        for (int h = 0; h < 2; ++h) {
            const float4 b = C.b[2 * k + h];
            const float4 z = mul4(C.minv[2 * k + h], b);
            C.x[2 * k + h] = make_float4(0.f, 0.f, 0.f, 0.f);
            C.r[2 * k + h] = b;
            C.z[2 * k + h] = z;
            C.p[2 * k + h] = z;
            rzf[0] += dot4(b, z);
        }
    }
    const int ntiles = (C.n + kVecThreads - 1) / kVecThreads;
    double rz[1];
    block_sum_f<1, kVecThreads / 32>(rzf, rz, sh);
    reduce_partials<1>(C, CNT_DOT2, tile, ntiles, rz, [&](const double (&tot)[1]) {
        Scalars* sc = C.sc;
        sc->rz = tot[0];
        sc->stop = tot[0] == 0.0 ? 1 : 0;
        sc->breakdown = 0;
        sc->iters = 0;
    });
}

__global__ void __launch_bounds__(kVecThreads) pcg_step_kernel(const CapDesc* __restrict__ caps,
                                                                const WorkItem* __restrict__ items) {
    __shared__ float sh[kVecThreads / 32][1];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    Scalars* sc = C.sc;
    if (sc->stop || sc->gn_stop) return;
    const float alpha = sc->alpha;
    const int k = tile * kVecThreads + threadIdx.x;
    float rzf[1] = {0.f};
    if (k < C.n) {
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * k + h;
            const float4 p = C.p[j];
            C.x[j] = axpy4(alpha, p, C.x[j]);
            const float4 r = axpy4(-alpha, C.Ap[j], C.r[j]);
            const float4 z = mul4(C.minv[j], r);
            C.r[j] = r;
            C.z[j] = z;
            rzf[0] += dot4(r, z);
        }
    }
    const int ntiles = (C.n + kVecThreads - 1) / kVecThreads;
    double rz[1];
    block_sum_f<1, kVecThreads / 32>(rzf, rz, sh);
    reduce_partials<1>(C, CNT_DOT2, tile, ntiles, rz, [&](const double (&tot)[1]) {
        sc->iters += 1;
        sc->rz_new = tot[0];
        if (tot[0] == 0.0) {
            sc->stop = 1;
        } else {
            // every other tile has read its inputs already (it finished before this one)
            sc->beta = tot[0] / sc->rz;
            sc->beta_f = __fdiv_rn((float)tot[0], (float)sc->rz);
            sc->rz = tot[0];
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
    const float beta = sc->beta_f;
    const int k = tile * kVecThreads + threadIdx.x;
    if (k < C.n) {
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * k + h;
            C.p[j] = axpy4(beta, C.p[j], C.z[j]);
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
// Grid-persistent PCG: all n_pcg iterations of one Gauss-Newton step in one
// cooperative launch over the whole GPU, for captures whose data does not fit
// a cluster's shared memory.  Per iteration: the vertex phase (q_i), a grid
// barrier, the node phase (A p and the CTA's p.Ap partial), a barrier, every
// CTA sums the partials in the same fixed order (FP64 across CTAs) for
// alpha, the vector phase (x, r, z and the r.z partial), a barrier, beta the
// same way, p = z + beta p, a barrier.  Operands are the staged rotated
// offsets (jtj_stage_*); vectors live in global memory (L2).
// ---------------------------------------------------------------------------
constexpr int kGridThreads = 256;

__device__ __forceinline__ double grid_total(const float* __restrict__ part, int G) {
    // warp 0: lanes add CTAs lane, lane + 32, ... then a fixed shuffle tree
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    for (int c = lane; c < G; c += 32) v += (double)__ldcg(&part[c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float block_total_f32(float v, float* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < kGridThreads / 32; ++i) t += sh[i];
    return t;   // thread 0
}

template <int KT>
__global__ void __launch_bounds__(kGridThreads) pcg_grid_kernel(const CapDesc* __restrict__ caps, int n_pcg,
                                                                 float* __restrict__ part) {
    __shared__ float sh[kGridThreads / 32];
    __shared__ float s_scal[2];   // alpha / beta of this iteration (thread 0 -> block)
    __shared__ int s_stop;
    cg::grid_group grid = cg::this_grid();
    const CapDesc& C = caps[0];
    if (C.sc->gn_stop) return;   // uniform: read before any barrier
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int gtid = b * kGridThreads + tid, gthreads = G * kGridThreads;
    const int lane = tid & 31, gwarp = gtid >> 5, gwarps = gthreads >> 5;
    const int n = C.n, N = C.N, K = C.K;
    float* partA = part;        // G: p.Ap partials
    float* partB = part + G;    // G: r.z partials
    // x = 0, r = b, z = M^-1 r, p = z; r.z
    float rz_p = 0.f;
    for (int j = gtid; j < 2 * n; j += gthreads) {
        const float4 bb = C.b[j], mi = C.minv[j];
        const float4 z = make_float4(mi.x * bb.x, mi.y * bb.y, mi.z * bb.z, 0.f);
        C.x[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        C.r[j] = bb;
        C.z[j] = z;
        C.p[j] = z;
        rz_p += bb.x * z.x + bb.y * z.y + bb.z * z.z;
    }
    {
        const float t = block_total_f32(rz_p, sh);
        if (tid == 0) partB[b] = t;
    }
    grid.sync();
    double rz = 0.0;
    if (tid < 32) rz = grid_total(partB, G);
    if (tid == 0) s_stop = rz == 0.0 ? 1 : 0;
    __syncthreads();
    rz = __shfl_sync(0xffffffffu, rz, 0);
    int iters = 0, breakdown = 0;
    int stop = s_stop;
    for (int it = 0; it < n_pcg && !stop; ++it) {
        // vertex phase: q_i = H_i dv_i for the active vertices
        for (int i = gtid; i < N; i += gthreads) {
            const float4* __restrict__ A = C.vA + (size_t)i * K;
            if (A[0].w == 0.f) continue;
            const float3 dv = vertex_dv<KT>(A, C.bind_idx + (size_t)i * K, C.p, K);
            const float3 q = mulH(C.HA[i], C.HB[i], dv);
            C.q[i] = make_float4(q.x, q.y, q.z, 1.f);
        }
        grid.sync();
        // node phase: (J^T J p)_k, warp per node; p.Ap partial of the CTA
        float pap = 0.f;
        for (int k = gwarp; k < n; k += gwarps) {
            const float3 pw = f3(C.p[2 * k]), pt = f3(C.p[2 * k + 1]);
            float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            constexpr int U = 4;
            const int e0 = C.ent_off[k], e1 = C.ent_off[k + 1];
            for (int jb = e0 + lane; jb < e1; jb += 32 * U) {
                float4 a[U];
                int vi[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = jb + 32 * u;
                    a[u] = j < e1 ? C.eA[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                    vi[u] = j < e1 ? C.ent[j].x : 0;
                }
                float4 q4[U];
#pragma unroll
                for (int u = 0; u < U; ++u) q4[u] = a[u].w != 0.f ? C.q[vi[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float3 q = f3(q4[u]);
                    const float3 c = cross3(f3(a[u]), q);
                    const float wv = a[u].w;
                    acc[0] += wv * c.x; acc[1] += wv * c.y; acc[2] += wv * c.z;
                    acc[3] += wv * q.x; acc[4] += wv * q.y; acc[5] += wv * q.z;
                }
            }
            for (int j = C.edge_off[k] + lane; j < C.edge_off[k + 1]; j += 32) {
                const int l = C.edge_dst[j];
                const float4 bk = C.dB[2 * j], bl = C.dB[2 * j + 1];
                const float c = bk.w;
                const float3 plw = f3(C.p[2 * l]), plt = f3(C.p[2 * l + 1]);
                const float3 D = cross3(pw, f3(bk)) + pt - plt;
                const float3 bD = cross3(f3(bk), D);
                acc[0] += c * bD.x; acc[1] += c * bD.y; acc[2] += c * bD.z;
                acc[3] += c * D.x; acc[4] += c * D.y; acc[5] += c * D.z;
                const float3 Dl = cross3(plw, f3(bl)) + plt - pt;
                acc[3] -= c * Dl.x; acc[4] -= c * Dl.y; acc[5] -= c * Dl.z;
            }
            warp_sumf<6>(acc);
            if (lane == 0) {
                C.Ap[2 * k] = make_float4(acc[0], acc[1], acc[2], 0.f);
                C.Ap[2 * k + 1] = make_float4(acc[3], acc[4], acc[5], 0.f);
                pap += pw.x * acc[0] + pw.y * acc[1] + pw.z * acc[2] + pt.x * acc[3] + pt.y * acc[4] + pt.z * acc[5];
            }
        }
        {
            const float t = block_total_f32(pap, sh);
            if (tid == 0) partA[b] = t;
        }
        grid.sync();
        if (tid < 32) {
            const double pAp = grid_total(partA, G);
            if (tid == 0) {
                if (!(pAp > 0.0)) {
                    s_stop = 1;
                } else {
                    // the step length is applied in FP32: the FP64 sums are divided in FP32
                    s_scal[0] = __fdiv_rn((float)rz, (float)pAp);
                    s_stop = 0;
                }
            }
        }
        __syncthreads();
        if (s_stop) {
            stop = 1;
            breakdown = 1;
            break;
        }
        const float alpha = s_scal[0];
        // vector phase: x, r, z; r.z partial
        float rzp = 0.f;
        for (int j = gtid; j < 2 * n; j += gthreads) {
            const float4 pp = C.p[j], ap = C.Ap[j], mi = C.minv[j];
            float4 x = C.x[j], r = C.r[j];
            x.x += alpha * pp.x; x.y += alpha * pp.y; x.z += alpha * pp.z;
            r.x -= alpha * ap.x; r.y -= alpha * ap.y; r.z -= alpha * ap.z;
            const float4 z = make_float4(mi.x * r.x, mi.y * r.y, mi.z * r.z, 0.f);
            C.x[j] = x;
            C.r[j] = r;
            C.z[j] = z;
            rzp += r.x * z.x + r.y * z.y + r.z * z.z;
        }
        {
            const float t = block_total_f32(rzp, sh);
            if (tid == 0) partB[b] = t;
        }
        grid.sync();
        ++iters;
        double rz_new = 0.0;
        if (tid < 32) {
            rz_new = grid_total(partB, G);
            if (tid == 0) {
                if (rz_new == 0.0) {
                    s_stop = 1;
                } else {
                    s_scal[1] = __fdiv_rn((float)rz_new, (float)rz);
                    s_stop = 0;
                }
            }
        }
        __syncthreads();
        rz = rz_new;   // meaningful in warp 0; only thread 0 reports it
        if (s_stop) {
            stop = 1;
            break;
        }
        const float beta = s_scal[1];
        for (int j = gtid; j < 2 * n; j += gthreads) {
            const float4 pp = C.p[j], z = C.z[j];
            C.p[j] = make_float4(z.x + beta * pp.x, z.y + beta * pp.y, z.z + beta * pp.z, 0.f);
        }
        grid.sync();
    }
    if (b == 0 && tid == 0) {
        Scalars* sc = C.sc;
        sc->iters = iters;
        sc->breakdown = breakdown;
        sc->stop = stop;
        sc->rz = rz;
    }
}

static int pcg_grid_ctas(const void* kern) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGridThreads, 0);
    return std::max(1, std::min(2, per_sm) * sms);
}

int pcg_grid_max_ctas() { return pcg_grid_ctas((const void*)pcg_grid_kernel<0>); }

cudaError_t launch_pcg_grid(const CapDesc* dC, int K, int n_pcg, float* part, cudaStream_t st) {
    const void* kern = K == 4 ? (const void*)pcg_grid_kernel<4>
                               : (K == 8 ? (const void*)pcg_grid_kernel<8> : (const void*)pcg_grid_kernel<0>);
    const int G = pcg_grid_ctas(kern);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kGridThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    if (K == 4) return cudaLaunchKernelEx(&cfg, pcg_grid_kernel<4>, dC, n_pcg, part);
    if (K == 8) return cudaLaunchKernelEx(&cfg, pcg_grid_kernel<8>, dC, n_pcg, part);
    return cudaLaunchKernelEx(&cfg, pcg_grid_kernel<0>, dC, n_pcg, part);
}

// ---------------------------------------------------------------------------
// Parameter update: R_k <- Exp(d_omega_k) R_k, t_k += d_t_k.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kVecThreads) update_kernel(const CapDesc* __restrict__ caps,
                                                              const WorkItem* __restrict__ items, int slot) {
    __shared__ float sh[kVecThreads / 32][1];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (C.sc->gn_stop) return;
    const int k = tile * kVecThreads + threadIdx.x;
    float s2f[1] = {0.f};
    if (k < C.n) {
        const float4 xw = C.x[2 * k], xt = C.x[2 * k + 1];
        s2f[0] = dot4(xw, xw) + dot4(xt, xt);
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
    double s2[1];
    block_sum_f<1, kVecThreads / 32>(s2f, s2, sh);
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

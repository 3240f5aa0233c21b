// Per-vertex surface stage: the paper's own non-rigid unknowns, the vertex
// positions V (Sec. 3.4: E_photo + E_silhouette + E_smooth + E_edge +
// E_velocity + E_acceleration; Sec. 4: Gauss-Newton with a Jacobi-
// preconditioned CG, one thread per vertex block row).
//
// Per ordered one-ring pair (i, j in N_i) the smooth residual
// sqrt(w_sm s_ij/|N_i|) ((V_i - V_j) - (V^S_i - V^S_j)) and the edge residual
// sqrt(w_ed s_ij/|N_i|) (||V_i - V_j|| - ||Vh_i - Vh_j||).  An undirected edge
// enters vertex i's block row from both of its ordered pairs, so with
// c_ij = s_ij (1/|N_i| + 1/|N_j|) and n_ij = (V_i - V_j)/||V_i - V_j||:
//   (J^T F)_i   = e_i + sum_j w_sm c_ij r^S_ij + w_ed c_ij n_ij (l_ij - lh_ij)
//                 + w_v (V_i - V^{t-1}_i) + w_a (V_i - 2 V^{t-1}_i + V^{t-2}_i)
//   (J^T J p)_i = H_i p_i + (w_v + w_a) p_i
//                 + sum_j w_sm c_ij (p_i - p_j) + w_ed c_ij n_ij n_ij^T (p_i - p_j)
// with H_i, e_i the data blocks of the linearisation (shared with the graph
// stage).  Each vertex gathers its own row from its one-ring: no atomics, and
// every result is deterministic.  The edge directions are staged once per
// linearisation as m_ij = sqrt(w_ed c_ij) n_ij next to w_sm c_ij, so a J^T J p
// reads 20 bytes per ordered pair.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cooperative_groups.h>

#include "lc_context.h"
#include "pose_internal.h"

namespace cg = cooperative_groups;

namespace lc {

namespace {

__device__ __forceinline__ float3 xyz(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3f(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Loads of vectors another CTA of the same launch wrote (the cluster PCG):
// through L2 (__ldcg); plain loads elsewhere.
template <bool kL2>
__device__ __forceinline__ float4 ldv(const float4* p) {
    if (kL2) return __ldcg(p);
    return *p;
}

// p of PCG iteration `it` at vertex j: iteration 0 reads the start direction
// z; later iterations form p = z + beta p_prev on the fly (the direction
// update is fused into the product), with one rounding order everywhere.
template <bool kL2>
__device__ __forceinline__ float3 direction(const CapDesc& C, int it, float beta, int j) {
    if (it <= 0) return xyz(ldv<kL2>(&C.sp[0][j]));
    const float4 z = ldv<kL2>(&C.sz[j]), q = ldv<kL2>(&C.sp[(it - 1) & 1][j]);
    return make_float3(__fmaf_rn(beta, q.x, z.x), __fmaf_rn(beta, q.y, z.y), __fmaf_rn(beta, q.z, z.z));
}

// Block row i of J^T J applied to p (p_in, or with p_in null the PCG
// direction of iteration it): returns p_i and (J^T J p)_i.  The one-ring in
// rounds of U pairs: a round's index and operand loads are issued together
// before any is used (a padding slot points at the vertex itself with a zero
// operand and adds nothing).
template <bool kL2>
__device__ __forceinline__ void row_product(const CapDesc& C, int it, float beta, const float4* __restrict__ p_in,
                                            int i, float3& pi, float3& q) {
    const bool pcg = p_in == nullptr;
    pi = pcg ? direction<kL2>(C, it, beta, i) : xyz(p_in[i]);
    const float4 HA = C.HA[i], HB = C.HB[i];
    const float wt = C.w_vel + C.w_acc;
    q = make_float3(HA.x * pi.x + HA.y * pi.y + HA.z * pi.z + wt * pi.x,
                    HA.y * pi.x + HA.w * pi.y + HB.x * pi.z + wt * pi.y,
                    HA.z * pi.x + HB.x * pi.y + HB.y * pi.z + wt * pi.z);
    constexpr int U = 4;
    const int p0 = C.adj_off[i], p1 = C.adj_off[i + 1];
    for (int pb = p0; pb < p1; pb += U) {
        int jj[U];
        float4 m[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = pb + u < p1;
            jj[u] = ok ? C.adj_dst[pb + u] : i;
            m[u] = ok ? C.adj_m[pb + u] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float3 pj[U];
#pragma unroll
        for (int u = 0; u < U; ++u) pj[u] = pcg ? direction<kL2>(C, it, beta, jj[u]) : xyz(p_in[jj[u]]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float3 dp = sub3(pi, pj[u]);
            const float s = m[u].x * dp.x + m[u].y * dp.y + m[u].z * dp.z;
            q.x += m[u].w * dp.x + s * m[u].x;
            q.y += m[u].w * dp.y + s * m[u].y;
            q.z += m[u].w * dp.z + s * m[u].z;
        }
    }
}

// PCG start at vertex i: x = 0, r = b, z = p = M^-1 b; returns r.z
__device__ __forceinline__ float init_vertex(const CapDesc& C, int i) {
    const float4 b = C.sb[i], m = C.sminv[i];
    const float4 z = make_float4(m.x * b.x, m.y * b.y, m.z * b.z, 0.f);
    C.sx[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    C.sr[i] = b;
    C.sz[i] = z;
    C.sp[0][i] = z;
    return b.x * z.x + b.y * z.y + b.z * z.z;
}

// x += alpha p, r -= alpha A p, z = M^-1 r at vertex i; returns r.z
__device__ __forceinline__ float step_vertex(const CapDesc& C, int it, float alpha, int i) {
    const float4 p = C.sp[it & 1][i], x = C.sx[i], Ap = C.sAp[i], r0 = C.sr[i], m = C.sminv[i];
    C.sx[i] = make_float4(x.x + alpha * p.x, x.y + alpha * p.y, x.z + alpha * p.z, 0.f);
    const float4 r = make_float4(r0.x - alpha * Ap.x, r0.y - alpha * Ap.y, r0.z - alpha * Ap.z, 0.f);
    const float4 z = make_float4(m.x * r.x, m.y * r.y, m.z * r.z, 0.f);
    C.sr[i] = r;
    C.sz[i] = z;
    return r.x * z.x + r.y * z.y + r.z * z.z;
}

}  // namespace

// V -> warped positions and projections read by the visibility and data kernels
__global__ void __launch_bounds__(kVertTile) surface_project_kernel(const CapDesc* __restrict__ caps) {
    const CapDesc& C = caps[0];
    const int i = blockIdx.x * kVertTile + threadIdx.x;
    if (i >= C.N) return;
    const float4 v = C.sV[i];
    const bool ok = valid_depth(v.z);
    C.vw[i] = make_float4(v.x, v.y, v.z, ok ? 1.f : 0.f);
    C.uv[i] = ok ? project_exact(C.f, C.cx, C.cy, v.x, v.y, v.z) : make_float2(0.f, 0.f);
}

// -J^T F, the Jacobi diagonal, the staged edge operands and the regulariser
// energies (smooth, edge, velocity, acceleration).
__global__ void __launch_bounds__(kVertTile) surface_rhs_kernel(const CapDesc* __restrict__ caps, int slot,
                                                                 int energy_only, float4* __restrict__ diag_out) {
    __shared__ float sh[kVertTile / 32][4];
    const CapDesc& C = caps[0];
    if (!energy_only && C.sc->gn_stop) return;
    const int tile = blockIdx.x;
    const int i = tile * kVertTile + threadIdx.x;
    float en[4] = {0.f, 0.f, 0.f, 0.f};
    if (i < C.N) {
        const float4 Vi4 = C.sV[i], Si4 = C.base[i];
        const float3 Vi = xyz(Vi4);
        // displacement from the rest geometry: exact for nearby FP32 values
        const float3 Di = sub3(Vi, xyz(Si4));
        float3 g = make_float3(0.f, 0.f, 0.f);
        float3 dg = make_float3(0.f, 0.f, 0.f);
        if (!energy_only) {
            const float4 e4 = C.ev[i], HA = C.HA[i], HB = C.HB[i];
            g = xyz(e4);
            dg = make_float3(HA.x, HA.w, HB.y);
        }
        constexpr int U = 4;
        const int p0 = C.adj_off[i], p1 = C.adj_off[i + 1];
        for (int pb = p0; pb < p1; pb += U) {
            int jj[U];
            float4 gg[U], vj4[U], sj4[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                jj[u] = pb + u < p1 ? C.adj_dst[pb + u] : i;
                gg[u] = pb + u < p1 ? C.adj_geo[pb + u] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                vj4[u] = C.sV[jj[u]];
                sj4[u] = C.base[jj[u]];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (pb + u >= p1) break;
                const int p = pb + u;
                const float4 geo = gg[u];
                const float3 Vj = xyz(vj4[u]);
                const float3 rs = sub3(Di, sub3(Vj, xyz(sj4[u])));
                const float3 d = sub3(Vi, Vj);
                const float len = sqrtf(dot3f(d, d));
                const float er = len - geo.z;
                en[0] += C.w_smooth * geo.x * dot3f(rs, rs);
                en[1] += C.w_edge * geo.x * er * er;
                if (energy_only) continue;
                const float csm = C.w_smooth * geo.y, ce = C.w_edge * geo.y;
                const float inv = len > 0.f ? 1.0f / len : 0.f;
                const float3 n = make_float3(d.x * inv, d.y * inv, d.z * inv);
                g.x += csm * rs.x + ce * er * n.x;
                g.y += csm * rs.y + ce * er * n.y;
                g.z += csm * rs.z + ce * er * n.z;
                dg.x += csm + ce * n.x * n.x;
                dg.y += csm + ce * n.y * n.y;
                dg.z += csm + ce * n.z * n.z;
                const float sce = sqrtf(ce);
                C.adj_m[p] = make_float4(sce * n.x, sce * n.y, sce * n.z, csm);
            }
        }
        if (C.w_vel > 0.f || C.w_acc > 0.f) {
            const float3 P1 = xyz(C.sH1[i]), P2 = xyz(C.sH2[i]);
            const float3 dv = sub3(Vi, P1);
            const float3 da = sub3(dv, sub3(P1, P2));   // V - 2 V^{t-1} + V^{t-2}
            en[2] = C.w_vel * dot3f(dv, dv);
            en[3] = C.w_acc * dot3f(da, da);
            if (!energy_only) {
                g.x += C.w_vel * dv.x + C.w_acc * da.x;
                g.y += C.w_vel * dv.y + C.w_acc * da.y;
                g.z += C.w_vel * dv.z + C.w_acc * da.z;
                const float wt = C.w_vel + C.w_acc;
                dg.x += wt; dg.y += wt; dg.z += wt;
            }
        }
        if (!energy_only) {
            C.sb[i] = make_float4(-g.x, -g.y, -g.z, 0.f);
            C.sminv[i] = make_float4(dg.x > 0.f ? 1.0f / dg.x : 0.f, dg.y > 0.f ? 1.0f / dg.y : 0.f,
                                     dg.z > 0.f ? 1.0f / dg.z : 0.f, 0.f);
            if (diag_out) diag_out[i] = make_float4(dg.x, dg.y, dg.z, 0.f);
        }
    }
    double tot4[4];
    block_sum_f<4, kVertTile / 32>(en, tot4, sh);
    reduce_partials<4>(C, CNT_ARAP, tile, C.vert_tiles, tot4, [&](const double (&tot)[4]) {
        Scalars* sc = C.sc;
        sc->e_lin[2] = 0.0;
        for (int k = 0; k < 4; ++k) sc->e_reg[k] = tot[k];
        const double E = sc->e_lin[0] + sc->e_lin[1] + tot[0] + tot[1] + tot[2] + tot[3];
        C.hist[2 * slot] = E;
        if (!energy_only && C.target_energy > 0.f && E <= (double)C.target_energy) sc->gn_stop = 1;
    });
}

// J^T J p for PCG iteration `it` (the direction update fused in, see
// direction()), or (it < 0) a plain product of p_in into out_in.
__global__ void __launch_bounds__(kVertTile) surface_jtj_kernel(const CapDesc* __restrict__ caps, int it,
                                                                 const float4* __restrict__ p_in,
                                                                 float4* __restrict__ out_in) {
    __shared__ float sh[kVertTile / 32][1];
    const CapDesc& C = caps[0];
    const bool pcg = it >= 0;
    if (pcg && (C.sc->stop || C.sc->gn_stop)) return;
    const float beta = pcg && it > 0 ? C.sc->beta_f : 0.f;
    const int tile = blockIdx.x;
    const int i = tile * kVertTile + threadIdx.x;
    float papf[1] = {0.f};
    if (i < C.N) {
        float3 pi, q;
        row_product<false>(C, it, beta, pcg ? nullptr : p_in, i, pi, q);
        if (pcg) {
            if (it > 0) C.sp[it & 1][i] = make_float4(pi.x, pi.y, pi.z, 0.f);
            C.sAp[i] = make_float4(q.x, q.y, q.z, 0.f);
            papf[0] = pi.x * q.x + pi.y * q.y + pi.z * q.z;
        } else {
            out_in[i] = make_float4(q.x, q.y, q.z, 0.f);
        }
    }
    if (!pcg) return;
    double pap[1];
    block_sum_f<1, kVertTile / 32>(papf, pap, sh);
    reduce_partials<1>(C, CNT_DOT, tile, C.vert_tiles, pap, [&](const double (&tot)[1]) {
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

__global__ void __launch_bounds__(kVertTile) surface_pcg_init_kernel(const CapDesc* __restrict__ caps) {
    __shared__ float sh[kVertTile / 32][1];
    const CapDesc& C = caps[0];
    if (C.sc->gn_stop) return;
    const int tile = blockIdx.x;
    const int i = tile * kVertTile + threadIdx.x;
    float rzf[1] = {0.f};
    if (i < C.N) rzf[0] = init_vertex(C, i);
    double rz[1];
    block_sum_f<1, kVertTile / 32>(rzf, rz, sh);
    reduce_partials<1>(C, CNT_DOT2, tile, C.vert_tiles, rz, [&](const double (&tot)[1]) {
        Scalars* sc = C.sc;
        sc->rz = tot[0];
        sc->stop = tot[0] == 0.0 ? 1 : 0;
        sc->breakdown = 0;
        sc->iters = 0;
    });
}

// x += alpha p, r -= alpha A p, z = M^-1 r, r.z and beta
__global__ void __launch_bounds__(kVertTile) surface_pcg_step_kernel(const CapDesc* __restrict__ caps, int it) {
    __shared__ float sh[kVertTile / 32][1];
    const CapDesc& C = caps[0];
    Scalars* sc = C.sc;
    if (sc->stop || sc->gn_stop) return;
    const float alpha = sc->alpha;
    const int tile = blockIdx.x;
    const int i = tile * kVertTile + threadIdx.x;
    float rzf[1] = {0.f};
    if (i < C.N) rzf[0] = step_vertex(C, it, alpha, i);
    double rz[1];
    block_sum_f<1, kVertTile / 32>(rzf, rz, sh);
    reduce_partials<1>(C, CNT_DOT2, tile, C.vert_tiles, rz, [&](const double (&tot)[1]) {
        sc->iters += 1;
        sc->rz_new = tot[0];
        if (tot[0] == 0.0) {
            sc->stop = 1;
        } else {
            sc->beta = tot[0] / sc->rz;
            sc->beta_f = __fdiv_rn((float)tot[0], (float)sc->rz);
            sc->rz = tot[0];
        }
    });
}

// ---------------------------------------------------------------------------
// Cluster-persistent PCG: all n_pcg iterations of one Gauss-Newton step in
// one launch of a thread-block cluster (one CTA per SM).  A CTA holds tpc
// consecutive vertex tiles of 256 threads (one vertex per thread), so the
// whole capture is in flight at once.  Vectors stay in global memory (L2);
// each dot product is reduced per tile exactly like the per-iteration
// kernels (FP32 inside the tile, the tile's FP64 partial pushed through
// distributed shared memory into every CTA, summed there in the same lane
// order), so both paths give identical results; one cluster barrier per
// reduction replaces a kernel boundary.
// ---------------------------------------------------------------------------
constexpr int kSurfClusterTiles = 64;   // vertex tiles a cluster PCG handles at most
constexpr int kSurfTilesPerCta = 4;     // up to 1024 threads per CTA

__device__ __forceinline__ double surf_cluster_reduce(cg::cluster_group& cluster, float v, int tile0, int cl,
                                                      int ntiles, double* slots, float* s_warp, double* s_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // FP32 sum of each 256-thread tile in the order of block_sum_f: a fixed
    // shuffle tree per warp, then the tile's 8 warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    constexpr int kW = kVertTile / 32;
    if ((warp % kW) == 0) {
        // the tile's first warp: lanes < cl push its partial into slot
        // `tile` of every cluster CTA
        const int g = warp / kW;
        float t = 0.f;
        for (int w = 0; w < kW; ++w) t += s_warp[g * kW + w];
        const int tile = tile0 + g;
        if (lane < cl && tile < ntiles) cluster.map_shared_rank(slots, lane)[tile] = (double)t;
    }
    cluster.sync();
    if (warp == 0) {
        // the order of sum_partials_warp: lane l adds tiles l, l + 32, ...,
        // then a fixed shuffle tree
        double d = 0.0;
        for (int tl = lane; tl < ntiles; tl += 32) d += slots[tl];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) *s_tot = d;
    }
    __syncthreads();
    return *s_tot;
}

__global__ void __launch_bounds__(kVertTile * kSurfTilesPerCta) surface_pcg_cluster_kernel(
    const CapDesc* __restrict__ caps, int n_pcg) {
    __shared__ double slots[2][kSurfClusterTiles];
    __shared__ float s_warp[kSurfTilesPerCta * kVertTile / 32];
    __shared__ double s_tot;
    cg::cluster_group cluster = cg::this_cluster();
    const CapDesc& C = caps[0];
    if (C.sc->gn_stop) return;   // uniform over the cluster
    const int rank = (int)cluster.block_rank(), cl = (int)cluster.num_blocks();
    const int tpc = (int)blockDim.x / kVertTile;
    const int ntiles = C.vert_tiles, N = C.N;
    const int tile0 = rank * tpc;
    const int i = tile0 * kVertTile + (int)threadIdx.x;   // this thread's vertex
    const bool own = i < N;
    int par = 0;
    // start: x = 0, r = b, z = p = M^-1 b
    double rz = surf_cluster_reduce(cluster, own ? init_vertex(C, i) : 0.f, tile0, cl, ntiles, slots[par], s_warp,
                                    &s_tot);
    par ^= 1;
    int iters = 0, breakdown = 0;
    bool stop = rz == 0.0;
    float beta = 0.f;
    for (int it = 0; it < n_pcg && !stop; ++it) {
        // A p (the direction update fused in) and p.Ap
        float v = 0.f;
        if (own) {
            float3 pi, q;
            row_product<true>(C, it, beta, nullptr, i, pi, q);
            if (it > 0) C.sp[it & 1][i] = make_float4(pi.x, pi.y, pi.z, 0.f);
            C.sAp[i] = make_float4(q.x, q.y, q.z, 0.f);
            v = pi.x * q.x + pi.y * q.y + pi.z * q.z;
        }
        const double pap = surf_cluster_reduce(cluster, v, tile0, cl, ntiles, slots[par], s_warp, &s_tot);
        par ^= 1;
        if (!(pap > 0.0)) {
            breakdown = 1;
            break;
        }
        const float alpha = __fdiv_rn((float)rz, (float)pap);
        const double rzn = surf_cluster_reduce(cluster, own ? step_vertex(C, it, alpha, i) : 0.f, tile0, cl, ntiles,
                                               slots[par], s_warp, &s_tot);
        par ^= 1;
        ++iters;
        if (rzn == 0.0) {
            stop = true;
        } else {
            beta = __fdiv_rn((float)rzn, (float)rz);
            rz = rzn;
        }
    }
    if (rank == 0 && threadIdx.x == 0) {
        Scalars* sc = C.sc;
        sc->iters = iters;
        sc->breakdown = breakdown;
        sc->stop = 1;
        sc->rz = rz;
    }
    // no CTA may leave while another can still write into its partial slots
    cluster.sync();
}

// V += delta, the new projections, ||delta||
__global__ void __launch_bounds__(kVertTile) surface_update_kernel(const CapDesc* __restrict__ caps, int slot) {
    __shared__ float sh[kVertTile / 32][1];
    const CapDesc& C = caps[0];
    if (C.sc->gn_stop) return;
    const int tile = blockIdx.x;
    const int i = tile * kVertTile + threadIdx.x;
    float s2f[1] = {0.f};
    if (i < C.N) {
        const float4 x = C.sx[i], v0 = C.sV[i];
        s2f[0] = x.x * x.x + x.y * x.y + x.z * x.z;
        const float X = v0.x + x.x, Y = v0.y + x.y, Z = v0.z + x.z;
        C.sV[i] = make_float4(X, Y, Z, 0.f);
        const bool ok = valid_depth(Z);
        C.vw[i] = make_float4(X, Y, Z, ok ? 1.f : 0.f);
        C.uv[i] = ok ? project_exact(C.f, C.cx, C.cy, X, Y, Z) : make_float2(0.f, 0.f);
    }
    double s2[1];
    block_sum_f<1, kVertTile / 32>(s2f, s2, sh);
    reduce_partials<1>(C, CNT_STEP, tile, C.vert_tiles, s2, [&](const double (&tot)[1]) {
        Scalars* sc = C.sc;
        sc->step2 = tot[0];
        C.hist[2 * slot + 1] = sqrt(tot[0]);
        C.hist_iters[slot] = sc->iters;
        C.hist_iters[LC_MAX_GN + 1] += sc->breakdown;
        sc->gn_done = slot + 1;
    });
}

// history shift: V^{t-2} <- V^{t-1}, V^{t-1} <- V
__global__ void __launch_bounds__(kVertTile) surface_shift_kernel(const CapDesc* __restrict__ caps) {
    const CapDesc& C = caps[0];
    const int i = blockIdx.x * kVertTile + threadIdx.x;
    if (i >= C.N) return;
    C.sH2[i] = C.sH1[i];
    C.sH1[i] = C.sV[i];
}

void launch_surface_project(const CapDesc* dC, const CapDesc& hC, cudaStream_t st) {
    surface_project_kernel<<<hC.vert_tiles, kVertTile, 0, st>>>(dC);
}
void launch_surface_rhs(const CapDesc* dC, const CapDesc& hC, int slot, bool energy_only, float4* diag_out,
                        cudaStream_t st) {
    surface_rhs_kernel<<<hC.vert_tiles, kVertTile, 0, st>>>(dC, slot, energy_only ? 1 : 0, diag_out);
}
void launch_surface_jtj(const CapDesc* dC, const CapDesc& hC, int it, const float4* p, float4* out, cudaStream_t st) {
    surface_jtj_kernel<<<hC.vert_tiles, kVertTile, 0, st>>>(dC, it, p, out);
}
void launch_surface_pcg_init(const CapDesc* dC, const CapDesc& hC, cudaStream_t st) {
    surface_pcg_init_kernel<<<hC.vert_tiles, kVertTile, 0, st>>>(dC);
}
void launch_surface_pcg_step(const CapDesc* dC, const CapDesc& hC, int it, cudaStream_t st) {
    surface_pcg_step_kernel<<<hC.vert_tiles, kVertTile, 0, st>>>(dC, it);
}
void launch_surface_update(const CapDesc* dC, const CapDesc& hC, int slot, cudaStream_t st) {
    surface_update_kernel<<<hC.vert_tiles, kVertTile, 0, st>>>(dC, slot);
}
// Cluster shape for the cluster PCG of a capture with `tiles` vertex tiles:
// tiles per CTA (1-4) and CTAs (<= 16, or <= 8 if the device does not
// schedule 16); {0, 0} when the capture is too large.
SurfCluster plan_surface_cluster(int tiles) {
    if (tiles > kSurfClusterTiles) return {0, 0};
    for (int clmax : {16, 8}) {
        const int tpc = (tiles + clmax - 1) / clmax;
        if (tpc > kSurfTilesPerCta) continue;
        const int cl = (tiles + tpc - 1) / tpc;
        if (cl > 8 && cudaFuncSetAttribute(surface_pcg_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                           1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(tpc * kVertTile);
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = cl;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, surface_pcg_cluster_kernel, &cfg) == cudaSuccess && n >= 1)
            return {cl, tpc};
        cudaGetLastError();
    }
    return {0, 0};
}

cudaError_t launch_surface_pcg_cluster(const CapDesc* dC, SurfCluster sc, int n_pcg, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sc.cl);
    cfg.blockDim = dim3(sc.tpc * kVertTile);
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = sc.cl;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, surface_pcg_cluster_kernel, dC, n_pcg);
}

static void launch_surface_shift(const CapDesc* dC, const CapDesc& hC, cudaStream_t st) {
    surface_shift_kernel<<<hC.vert_tiles, kVertTile, 0, st>>>(dC);
}

}  // namespace lc

using namespace lc;

// ---------------------------------------------------------------------------
// setup (called by lc_upload_template) and release
// ---------------------------------------------------------------------------
lc_status lc_ctx::surface_setup(const float* V, const float* mat, const std::vector<int4>& medges) {
    const int N = hC.N;
    const int af0 = alloc_failures;
    // one-ring CSR from the unique mesh edges, neighbours ascending
    std::vector<int> off(N + 1, 0);
    for (const int4& e : medges) {
        off[e.x + 1]++;
        off[e.y + 1]++;
    }
    for (int i = 0; i < N; ++i) off[i + 1] += off[i];
    const int n_adj = off[N];
    std::vector<int> dst(n_adj);
    {
        std::vector<int> fill(off.begin(), off.end() - 1);
        for (const int4& e : medges) {
            dst[fill[e.x]++] = e.y;
            dst[fill[e.y]++] = e.x;
        }
    }
    std::vector<float4> geo(n_adj);
    for (int i = 0; i < N; ++i) {
        std::sort(dst.begin() + off[i], dst.begin() + off[i + 1]);
        const double di = off[i + 1] - off[i];
        for (int p = off[i]; p < off[i + 1]; ++p) {
            const int j = dst[p];
            const double dj = off[j + 1] - off[j];
            const double s = 0.5 * ((double)mat[i] + (double)mat[j]);
            const double dx = (double)V[3 * i] - V[3 * j], dy = (double)V[3 * i + 1] - V[3 * j + 1],
                         dz = (double)V[3 * i + 2] - V[3 * j + 2];
            geo[p] = make_float4((float)(s / di), (float)(s * (1.0 / di + 1.0 / dj)),
                                 (float)std::sqrt(dx * dx + dy * dy + dz * dz), 0.f);
        }
    }
    CapDesc& C = hC;
    C.n_adj = n_adj;
    C.adj_off = (const int*)alloc(sizeof(int) * (N + 1));
    C.adj_dst = (const int*)alloc(sizeof(int) * std::max(n_adj, 1));
    C.adj_geo = (const float4*)alloc(sizeof(float4) * std::max(n_adj, 1));
    C.adj_m = (float4*)alloc(sizeof(float4) * std::max(n_adj, 1));
    float4** vecs[] = {&C.sV, &C.sH1, &C.sH2, &C.sD, &C.sb, &C.sminv, &C.sx, &C.sr, &C.sz, &C.sp[0], &C.sp[1],
                       &C.sAp, &surf_diag};
    for (float4** v : vecs) *v = (float4*)alloc(sizeof(float4) * N);
    if (alloc_failures != af0) return LC_ERR_OOM;
    cudaStream_t st = stream;
    lc_status s;
    if ((s = cuda(cudaMemcpyAsync((void*)C.adj_off, off.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, st),
                  "upload")) ||
        (n_adj && ((s = cuda(cudaMemcpyAsync((void*)C.adj_dst, dst.data(), sizeof(int) * n_adj,
                                             cudaMemcpyHostToDevice, st), "upload")) ||
                   (s = cuda(cudaMemcpyAsync((void*)C.adj_geo, geo.data(), sizeof(float4) * n_adj,
                                             cudaMemcpyHostToDevice, st), "upload")))))
        return s;
    // the surface starts at the template; no history, no displacement
    if ((s = cuda(cudaMemcpyAsync(C.sV, tpl, sizeof(float4) * N, cudaMemcpyDeviceToDevice, st), "copy")) ||
        (s = cuda(cudaMemsetAsync(C.sD, 0, sizeof(float4) * N, st), "memset")))
        return s;
    surf_hist = 0;
    surf_has_disp = false;
    surf_has_lin = false;
    surf_shape = plan_surface_cluster(C.vert_tiles);
    surf_cl = surf_shape.cl;
    apply_params();
    return LC_OK;
}

void lc_ctx::surface_release() {
    if (surf_gexec) cudaGraphExecDestroy(surf_gexec);
    surf_gexec = nullptr;
    CapDesc& C = hC;
    void* bufs[] = {(void*)C.adj_off, (void*)C.adj_dst, (void*)C.adj_geo, C.adj_m, C.sV, C.sH1, C.sH2, C.sD,
                    C.sb, C.sminv, C.sx, C.sr, C.sz, C.sp[0], C.sp[1], C.sAp, surf_diag};
    for (void* p : bufs) release(p);
    C.adj_off = C.adj_dst = nullptr;
    C.adj_geo = nullptr;
    C.adj_m = C.sV = C.sH1 = C.sH2 = C.sD = C.sb = C.sminv = C.sx = C.sr = C.sz = C.sp[0] = C.sp[1] = C.sAp = nullptr;
    surf_diag = nullptr;
    C.n_adj = 0;
    surf_hist = 0;
    surf_has_disp = false;
    surf_has_lin = false;
}

// ---------------------------------------------------------------------------
// the captured frame solve
// ---------------------------------------------------------------------------
void lc_ctx::enqueue_surface() {
    const CapDesc& C = hC;
    cudaStream_t st = stream;
    prof_surface.begin = prof_used;
    cudaMemsetAsync(C.hist, 0, sizeof(double) * 2 * (LC_MAX_GN + 1), st);
    cudaMemsetAsync(C.hist_iters, 0, sizeof(int) * (LC_MAX_GN + 2), st);
    cudaMemsetAsync((char*)C.sc + offsetof(Scalars, gn_stop), 0, 2 * sizeof(int), st);
    mark(LC_PH_VIS);
    launch_part_mask(dC, C, st);
    mark(LC_PH_WARP);
    launch_surface_project(dC, C, st);
    mark(LC_PH_VIS);
    launch_visibility(dC, C, st);
    const int n_gn = params.n_gn_surface, n_pcg = params.n_pcg_surface;
    for (int gn = 0; gn < n_gn; ++gn) {
        mark(LC_PH_LIN);
        launch_linearize(dC, C, true, gn, st);
        mark(LC_PH_RHS);
        launch_surface_rhs(dC, C, gn, false, nullptr, st);
        if (surf_cl > 0 && params.pcg_kernel == 0) {
            mark(LC_PH_PCG);
            launch_surface_pcg_cluster(dC, surf_shape, n_pcg, st);
        } else {
            mark(LC_PH_PCG_INIT);
            launch_surface_pcg_init(dC, C, st);
            for (int it = 0; it < n_pcg; ++it) {
                mark(LC_PH_JTJ);
                launch_surface_jtj(dC, C, it, nullptr, nullptr, st);
                mark(LC_PH_PCG_VEC);
                launch_surface_pcg_step(dC, C, it, st);
            }
        }
        mark(LC_PH_UPDATE);
        launch_surface_update(dC, C, gn, st);
    }
    mark(LC_PH_LIN);
    launch_linearize(dC, C, false, LC_MAX_GN, st);
    mark(LC_PH_RHS);
    launch_surface_rhs(dC, C, n_gn, true, nullptr, st);
    launch_vis_unfreeze(dC, st);
    mark_end();
    prof_surface.end = prof_used;
}

lc_status lc_ctx::check_surface_state(const char* who) {
    if (!has_template) return fail(LC_ERR_STATE, "%s: no template", who);
    if (!has_camera || !has_frame) return fail(LC_ERR_STATE, "%s: camera and frame required", who);
    return LC_OK;
}

// temporal weights follow the history actually held
void lc_ctx::surface_weights() {
    hC.w_smooth = params.w_smooth;
    hC.w_edge = params.w_edge;
    hC.w_vel = surf_hist > 0 ? params.w_velocity : 0.f;
    hC.w_acc = surf_hist > 0 ? params.w_acceleration : 0.f;
}

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------
static lc_status upload_vertices(lc_ctx* ctx, float4* dst, const float* src) {
    const int N = ctx->hC.N;
    std::vector<float> h((size_t)3 * N);
    lc_status s;
    if ((s = ctx->fetch(h.data(), src, sizeof(float) * h.size()))) return s;
    std::vector<float4> v4(N);
    for (int i = 0; i < N; ++i) {
        if (!std::isfinite(h[3 * i]) || !std::isfinite(h[3 * i + 1]) || !std::isfinite(h[3 * i + 2]))
            return ctx->fail(LC_ERR_ARG, "non-finite vertex %d", i);
        v4[i] = make_float4(h[3 * i], h[3 * i + 1], h[3 * i + 2], 0.f);
    }
    if ((s = ctx->cuda(cudaMemcpyAsync(dst, v4.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, ctx->stream),
                       "upload")))
        return s;
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
}

static lc_status download_vec(lc_ctx* ctx, float* dst, const float4* src) {
    const int N = ctx->hC.N;
    std::vector<float4> v4(N);
    lc_status s;
    if ((s = ctx->copy_to_host(v4.data(), src, sizeof(float4) * N))) return s;
    std::vector<float> h((size_t)3 * N);
    for (int i = 0; i < N; ++i) {
        h[3 * i] = v4[i].x;
        h[3 * i + 1] = v4[i].y;
        h[3 * i + 2] = v4[i].z;
    }
    return ctx->deliver(dst, h.data(), sizeof(float) * h.size());
}

extern "C" lc_status lc_set_surface(lc_ctx* ctx, const float* V) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_template) return ctx->fail(LC_ERR_STATE, "lc_set_surface: no template");
    if (!V) return ctx->fail(LC_ERR_ARG, "lc_set_surface: null V");
    cudaSetDevice(ctx->device);
    ctx->surf_has_lin = false;
    return upload_vertices(ctx, ctx->hC.sV, V);
}

extern "C" lc_status lc_surface_history(lc_ctx* ctx, const float* V_prev, const float* V_prev2) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_template) return ctx->fail(LC_ERR_STATE, "lc_surface_history: no template");
    cudaSetDevice(ctx->device);
    lc_status s;
    if (!V_prev) {
        ctx->surf_hist = 0;
    } else {
        if ((s = upload_vertices(ctx, ctx->hC.sH1, V_prev))) return s;
        if (V_prev2) {
            if ((s = upload_vertices(ctx, ctx->hC.sH2, V_prev2))) return s;
        } else if ((s = ctx->cuda(cudaMemcpyAsync(ctx->hC.sH2, ctx->hC.sH1, sizeof(float4) * ctx->hC.N,
                                                  cudaMemcpyDeviceToDevice, ctx->stream), "copy"))) {
            return s;
        }
        ctx->surf_hist = V_prev2 ? 2 : 1;
    }
    ctx->surf_has_lin = false;
    ctx->surface_weights();
    return ctx->sync_desc();
}

extern "C" lc_status lc_surface_advance(lc_ctx* ctx) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_template) return ctx->fail(LC_ERR_STATE, "lc_surface_advance: no template");
    cudaSetDevice(ctx->device);
    const CapDesc& C = ctx->hC;
    if (ctx->surf_hist == 0) {
        // the first frame: V^{t-2} = V^{t-1} = V
        lc_status s;
        if ((s = ctx->cuda(cudaMemcpyAsync(C.sH1, C.sV, sizeof(float4) * C.N, cudaMemcpyDeviceToDevice, ctx->stream),
                           "copy")))
            return s;
    }
    launch_surface_shift(ctx->dC, C, ctx->stream);
    launch_surface_warp(ctx->dC, C, ctx->pose_desc(), 0, ctx->stream);
    const int before = ctx->surf_hist;
    ctx->surf_hist = std::min(ctx->surf_hist + 1, 2);
    ctx->surf_has_disp = true;
    lc_status s = ctx->cuda(cudaGetLastError(), "lc_surface_advance");
    if (s) return s;
    if (before > 0) return LC_OK;    // the temporal weights are already on
    ctx->surface_weights();
    return ctx->sync_desc();
}

extern "C" lc_status lc_surface_start(lc_ctx* ctx) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_template) return ctx->fail(LC_ERR_STATE, "lc_surface_start: no template");
    cudaSetDevice(ctx->device);
    ctx->surf_has_lin = false;
    if (!ctx->surf_has_disp)
        return ctx->cuda(cudaMemcpyAsync(ctx->hC.sV, ctx->hC.base, sizeof(float4) * ctx->hC.N,
                                         cudaMemcpyDeviceToDevice, ctx->stream), "copy");
    launch_surface_warp(ctx->dC, ctx->hC, ctx->pose_desc(), 1, ctx->stream);
    return ctx->cuda(cudaGetLastError(), "lc_surface_start");
}

extern "C" lc_status lc_solve_surface(lc_ctx* ctx, lc_solve_stats* stats) {
    if (!ctx) return LC_ERR_ARG;
    lc_status s;
    if ((s = ctx->check_surface_state("lc_solve_surface"))) return s;
    cudaSetDevice(ctx->device);
    if (!ctx->surf_gexec &&
        (s = ctx->capture(&ctx->surf_gexec, &ctx->surf_graph_kernels, &lc_ctx::enqueue_surface)))
        return s;
    if ((s = ctx->cuda(cudaGraphLaunch(ctx->surf_gexec, ctx->stream), "graph launch"))) return s;
    if ((s = ctx->accumulate_profile(ctx->prof_surface))) return s;
    ctx->has_vis = true;
    ctx->has_lin = false;            // the graph stage's node operands are stale
    ctx->surf_has_lin = true;
    ctx->last_surface = true;
    if (stats) {
        if ((s = ctx->read_stats(stats, ctx->params.n_gn_surface, true))) return s;
        stats->n_kernels = ctx->surf_graph_kernels;
        stats->pcg_cluster_size = ctx->surf_cl > 0 && ctx->params.pcg_kernel == 0 ? ctx->surf_cl : 0;
    }
    return LC_OK;
}

extern "C" lc_status lc_read_surface(lc_ctx* ctx, float* V, uint8_t* flags) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_template) return ctx->fail(LC_ERR_STATE, "lc_read_surface: no template");
    cudaSetDevice(ctx->device);
    lc_status s;
    if (V && (s = download_vec(ctx, V, ctx->hC.sV))) return s;
    if (flags) {
        const int N = ctx->hC.N;
        std::vector<uint32_t> f(N);
        if ((s = ctx->copy_to_host(f.data(), ctx->hC.flags, sizeof(uint32_t) * N))) return s;
        std::vector<uint8_t> f8(N);
        for (int i = 0; i < N; ++i) f8[i] = (uint8_t)f[i];
        if ((s = ctx->deliver(flags, f8.data(), N))) return s;
    }
    return LC_OK;
}

extern "C" lc_status lc_surface_visibility(lc_ctx* ctx) {
    if (!ctx) return LC_ERR_ARG;
    lc_status s;
    if ((s = ctx->check_surface_state("lc_surface_visibility"))) return s;
    cudaSetDevice(ctx->device);
    launch_part_mask(ctx->dC, ctx->hC, ctx->stream);
    launch_surface_project(ctx->dC, ctx->hC, ctx->stream);
    launch_visibility(ctx->dC, ctx->hC, ctx->stream);
    if ((s = ctx->cuda(cudaStreamSynchronize(ctx->stream), "lc_surface_visibility"))) return s;
    ctx->has_vis = true;
    ctx->has_lin = false;
    ctx->surf_has_lin = false;
    return LC_OK;
}

extern "C" lc_status lc_surface_linearize(lc_ctx* ctx, float* rhs, float* diag, double* energies) {
    if (!ctx) return LC_ERR_ARG;
    lc_status s;
    if ((s = ctx->check_surface_state("lc_surface_linearize"))) return s;
    if (!ctx->has_vis) return ctx->fail(LC_ERR_STATE, "lc_surface_linearize: no frame decisions");
    cudaSetDevice(ctx->device);
    const CapDesc& C = ctx->hC;
    cudaStream_t st = ctx->stream;
    cudaMemsetAsync((char*)C.sc + offsetof(Scalars, gn_stop), 0, 2 * sizeof(int), st);
    launch_surface_project(ctx->dC, C, st);
    launch_linearize(ctx->dC, C, true, 0, st);
    launch_surface_rhs(ctx->dC, C, 0, false, ctx->surf_diag, st);
    if ((s = ctx->cuda(cudaStreamSynchronize(st), "lc_surface_linearize"))) return s;
    ctx->surf_has_lin = true;
    if (rhs && (s = download_vec(ctx, rhs, C.sb))) return s;
    if (diag && (s = download_vec(ctx, diag, ctx->surf_diag))) return s;
    if (energies) {
        Scalars sc;
        if ((s = ctx->copy_to_host(&sc, C.sc, sizeof(Scalars)))) return s;
        const double e[6] = {sc.e_lin[0], sc.e_lin[1], sc.e_reg[0], sc.e_reg[1], sc.e_reg[2], sc.e_reg[3]};
        if ((s = ctx->deliver(energies, e, sizeof(e)))) return s;
    }
    return LC_OK;
}

extern "C" lc_status lc_surface_apply_jtj(lc_ctx* ctx, const float* p, float* out) {
    if (!ctx) return LC_ERR_ARG;
    if (!p || !out) return ctx->fail(LC_ERR_ARG, "lc_surface_apply_jtj: null array");
    if (!ctx->surf_has_lin) return ctx->fail(LC_ERR_STATE, "lc_surface_apply_jtj: no surface linearisation");
    cudaSetDevice(ctx->device);
    lc_status s;
    if ((s = upload_vertices(ctx, ctx->hC.sz, p))) return s;   // scratch: z is free outside a PCG
    launch_surface_jtj(ctx->dC, ctx->hC, -1, ctx->hC.sz, ctx->hC.sr, ctx->stream);
    if ((s = ctx->cuda(cudaGetLastError(), "lc_surface_apply_jtj"))) return s;
    return download_vec(ctx, out, ctx->hC.sr);
}

extern "C" lc_status lc_surface_solve_linear(lc_ctx* ctx, float* delta, int* iters) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->surf_has_lin) return ctx->fail(LC_ERR_STATE, "lc_surface_solve_linear: no surface linearisation");
    cudaSetDevice(ctx->device);
    const CapDesc& C = ctx->hC;
    cudaStream_t st = ctx->stream;
    cudaMemsetAsync((char*)C.sc + offsetof(Scalars, gn_stop), 0, 2 * sizeof(int), st);
    if (ctx->surf_cl > 0 && ctx->params.pcg_kernel == 0) {
        launch_surface_pcg_cluster(ctx->dC, ctx->surf_shape, ctx->params.n_pcg_surface, st);
    } else {
        launch_surface_pcg_init(ctx->dC, C, st);
        for (int it = 0; it < ctx->params.n_pcg_surface; ++it) {
            launch_surface_jtj(ctx->dC, C, it, nullptr, nullptr, st);
            launch_surface_pcg_step(ctx->dC, C, it, st);
        }
    }
    lc_status s;
    if ((s = ctx->cuda(cudaStreamSynchronize(st), "lc_surface_solve_linear"))) return s;
    if (delta && (s = download_vec(ctx, delta, C.sx))) return s;
    if (iters) {
        Scalars sc;
        if ((s = ctx->copy_to_host(&sc, C.sc, sizeof(Scalars)))) return s;
        *iters = sc.iters;
    }
    return LC_OK;
}

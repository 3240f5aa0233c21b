// Matrix-free J^T J p of the graph stage in compensated FP32 (fpair.cuh),
// shared by the cluster-persistent PCG and the per-iteration kernels.
//
// Operator (Sec. 4, normal equations of the embedded-graph energy; all
// coefficients FP32, fixed for one linearisation):
//   * data rows of vertex i, slot s bound to node k: the 3 x 6 block
//     w_is [-[a_is]x | I] with a_is = R_k (v_i - g_k), stored as the FP32 pair
//     (c_is = w_is a_is, w_is), so J_i p = sum_s (p_omega,k x c_is + w_is p_t,k)
//     and J_i^T q = [c_is x q ; w_is q] use the same numbers: the assembled
//     operator is exactly symmetric (to the pair precision);
//   * the vertex block H_i = A_i^T A_i (FP32, six entries) between them;
//   * ARAP rows of directed edge (k, l) with weight c = w_a s_kl:
//     D = p_omega,k x b_kl + p_t,k - p_t,l, b_kl = R_k (g_l - g_k), and the
//     product c D is formed in pairs, so J_e^T (c J_e p) keeps its symmetry.
#pragma once

#include "fpair.cuh"

namespace lc {

// (omega, t) of one node in pairs
struct NodeP {
    fp2 w[3], t[3];
};

// From 12 consecutive floats: high parts of (omega, t), then low parts.
__device__ __forceinline__ NodeP node_pair12(const float* __restrict__ v) {
    const float4 a = *reinterpret_cast<const float4*>(v);
    const float4 b = *reinterpret_cast<const float4*>(v + 4);
    const float4 c = *reinterpret_cast<const float4*>(v + 8);
    NodeP p;
    p.w[0] = {a.x, b.z}; p.w[1] = {a.y, b.w}; p.w[2] = {a.z, c.x};
    p.t[0] = {a.w, c.y}; p.t[1] = {b.x, c.z}; p.t[2] = {b.y, c.w};
    return p;
}

// From the two float4 per node (omega, t) of the high and (nullable) low arrays.
__device__ __forceinline__ NodeP node_pair44(const float4* __restrict__ hi, const float4* __restrict__ lo, int k) {
    const float4 wh = hi[2 * k], th = hi[2 * k + 1];
    float4 wl = make_float4(0.f, 0.f, 0.f, 0.f), tl = wl;
    if (lo) {
        wl = lo[2 * k];
        tl = lo[2 * k + 1];
    }
    NodeP p;
    p.w[0] = {wh.x, wl.x}; p.w[1] = {wh.y, wl.y}; p.w[2] = {wh.z, wl.z};
    p.t[0] = {th.x, tl.x}; p.t[1] = {th.y, tl.y}; p.t[2] = {th.z, tl.z};
    return p;
}

// The staged data coefficient of one binding: a = R_k (v - g_k) with a fixed
// sequence of rounded operations (so every kernel that stages it gets the same
// bits), then c = w a; returns (c, w).  R: three float4 rows of node k.
__device__ __forceinline__ float4 staged_coef(const float4* __restrict__ R, int k, float4 v, float4 g, float w) {
    const float dx = __fsub_rn(v.x, g.x), dy = __fsub_rn(v.y, g.y), dz = __fsub_rn(v.z, g.z);
    const float4 r0 = R[3 * k], r1 = R[3 * k + 1], r2 = R[3 * k + 2];
    const float ax = __fmaf_rn(r0.z, dz, __fmaf_rn(r0.y, dy, __fmul_rn(r0.x, dx)));
    const float ay = __fmaf_rn(r1.z, dz, __fmaf_rn(r1.y, dy, __fmul_rn(r1.x, dx)));
    const float az = __fmaf_rn(r2.z, dz, __fmaf_rn(r2.y, dy, __fmul_rn(r2.x, dx)));
    return make_float4(__fmul_rn(w, ax), __fmul_rn(w, ay), __fmul_rn(w, az), w);
}

// dv += p_omega x c + w p_t for one slot (cw = (c, w))
__device__ __forceinline__ void jtj_slot(float4 cw, const NodeP& p, fp2acc (&dv)[3]) {
    dv[0].mac(cw.z, p.w[1]); dv[0].mac(-cw.y, p.w[2]); dv[0].mac(cw.w, p.t[0]);
    dv[1].mac(cw.x, p.w[2]); dv[1].mac(-cw.z, p.w[0]); dv[1].mac(cw.w, p.t[1]);
    dv[2].mac(cw.y, p.w[0]); dv[2].mac(-cw.x, p.w[1]); dv[2].mac(cw.w, p.t[2]);
}

// q = H dv, H symmetric given as (h00, h01, h02, h11, h12, h22)
__device__ __forceinline__ void jtj_block(const float (&h)[6], const fp2 (&dv)[3], fp2 (&q)[3]) {
    fp2acc a, b, c;
    a.mac(h[0], dv[0]); a.mac(h[1], dv[1]); a.mac(h[2], dv[2]);
    b.mac(h[1], dv[0]); b.mac(h[3], dv[1]); b.mac(h[4], dv[2]);
    c.mac(h[2], dv[0]); c.mac(h[4], dv[1]); c.mac(h[5], dv[2]);
    q[0] = a.get();
    q[1] = b.get();
    q[2] = c.get();
}

// acc += [c x q ; w q] for one entry of the node (cw = (c, w))
__device__ __forceinline__ void jtj_entry(float4 cw, const fp2 (&q)[3], fp2acc (&acc)[6]) {
    acc[0].mac(cw.y, q[2]); acc[0].mac(-cw.z, q[1]);
    acc[1].mac(cw.z, q[0]); acc[1].mac(-cw.x, q[2]);
    acc[2].mac(cw.x, q[1]); acc[2].mac(-cw.y, q[0]);
    acc[3].mac(cw.w, q[0]); acc[4].mac(cw.w, q[1]); acc[5].mac(cw.w, q[2]);
}

// ARAP edge (k, l) at node k, both directions of the pair of directed edges:
// acc += c [b_kl x D ; D] - c [0 ; E], D = pk.w x b_kl + pk.t - pl.t,
// E = pl.w x b_lk + pl.t - pk.t.  bk = (b_kl, c), bl = (b_lk, -).
__device__ __forceinline__ void jtj_edge(float4 bk, float4 bl, const NodeP& pk, const NodeP& pl, fp2acc (&acc)[6]) {
    fp2 cD[3], cE[3];
    {
        fp2acc d0, d1, d2;
        d0.mac(bk.z, pk.w[1]); d0.mac(-bk.y, pk.w[2]); d0.add(pk.t[0]); d0.add(fp2_neg(pl.t[0]));
        d1.mac(bk.x, pk.w[2]); d1.mac(-bk.z, pk.w[0]); d1.add(pk.t[1]); d1.add(fp2_neg(pl.t[1]));
        d2.mac(bk.y, pk.w[0]); d2.mac(-bk.x, pk.w[1]); d2.add(pk.t[2]); d2.add(fp2_neg(pl.t[2]));
        cD[0] = fp2_scale(bk.w, d0.get());
        cD[1] = fp2_scale(bk.w, d1.get());
        cD[2] = fp2_scale(bk.w, d2.get());
    }
    {
        fp2acc e0, e1, e2;
        e0.mac(bl.z, pl.w[1]); e0.mac(-bl.y, pl.w[2]); e0.add(pl.t[0]); e0.add(fp2_neg(pk.t[0]));
        e1.mac(bl.x, pl.w[2]); e1.mac(-bl.z, pl.w[0]); e1.add(pl.t[1]); e1.add(fp2_neg(pk.t[1]));
        e2.mac(bl.y, pl.w[0]); e2.mac(-bl.x, pl.w[1]); e2.add(pl.t[2]); e2.add(fp2_neg(pk.t[2]));
        cE[0] = fp2_scale(bk.w, e0.get());
        cE[1] = fp2_scale(bk.w, e1.get());
        cE[2] = fp2_scale(bk.w, e2.get());
    }
    acc[0].mac(bk.y, cD[2]); acc[0].mac(-bk.z, cD[1]);
    acc[1].mac(bk.z, cD[0]); acc[1].mac(-bk.x, cD[2]);
    acc[2].mac(bk.x, cD[1]); acc[2].mac(-bk.y, cD[0]);
    acc[3].add(cD[0]); acc[3].add(fp2_neg(cE[0]));
    acc[4].add(cD[1]); acc[4].add(fp2_neg(cE[1]));
    acc[5].add(cD[2]); acc[5].add(fp2_neg(cE[2]));
}

// The ARAP offsets of a directed edge with a fixed operation sequence:
// b = R (d), d = g_l - g_k (or g_k - g_l for the reverse edge).
__device__ __forceinline__ float3 staged_edge_offset(const float4* __restrict__ R, int k, float4 from, float4 to) {
    const float dx = __fsub_rn(to.x, from.x), dy = __fsub_rn(to.y, from.y), dz = __fsub_rn(to.z, from.z);
    const float4 r0 = R[3 * k], r1 = R[3 * k + 1], r2 = R[3 * k + 2];
    return make_float3(__fmaf_rn(r0.z, dz, __fmaf_rn(r0.y, dy, __fmul_rn(r0.x, dx))),
                       __fmaf_rn(r1.z, dz, __fmaf_rn(r1.y, dy, __fmul_rn(r1.x, dx))),
                       __fmaf_rn(r2.z, dz, __fmaf_rn(r2.y, dy, __fmul_rn(r2.x, dx))));
}

}  // namespace lc

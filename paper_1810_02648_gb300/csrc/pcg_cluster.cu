// Cluster-persistent Jacobi-PCG for one Gauss-Newton step (Sec. 4: normal
// equations J^T J delta = -J^T F, Jacobi preconditioner, fixed iteration
// count), all n_pcg iterations in one launch.
//
// One thread-block cluster of CL CTAs solves one capture.  CTA r owns a
// contiguous node range holding about 1/CL of the CSR entries (part_lo).  At
// the start it stages, in its own
// shared memory, everything its nodes' rows of J^T J need:
//   * per CSR entry (vertex i bound to an owned node k, active vertices
//     only): H_i, and for each of i's K slots the node index, weight w_is and
//     a_is = R_k (v_i - g_k), plus which slot is k;
//   * per owned ARAP edge (k, l): l, c = w_a s_kl, b_kl = R_k (g_l - g_k),
//     b_lk = R_l (g_k - g_l);
//   * the preconditioned residual z of all nodes (every CTA holds a copy).
// One iteration is then computed from shared memory alone:
//   (J^T J z)_k = sum_entries w_is [a_is x q_i ; q_i] + ARAP terms, with
//   q_i = H_i sum_s w_is (z_omega,s x a_is + z_t,s) recomputed per entry,
// one warp per owned node (entries and edges lane-strided, one shuffle tree),
// then for the owned nodes p = z + beta p and A p = A z + beta A p (A is
// linear; warp 0 forms beta while the others compute A z), followed by FP64
// partial dot products exchanged through distributed shared memory (each CTA
// writes its partial into every CTA's slot array, all sum in rank order:
// deterministic and identical in every CTA).  The new z of the owned nodes is
// stored into every CTA's copy as each thread forms it.  Two hardware cluster
// barriers per iteration; no spin loops, no global-memory round trips.
#include <algorithm>

#include <cooperative_groups.h>

#include "lc_internal.cuh"

namespace cg = cooperative_groups;

namespace lc {

constexpr int kPcgThreads = 1024;
constexpr int kPcgWarps = kPcgThreads / 32;

// shared-memory carve-up (byte offsets, all 16-byte aligned)
struct Smem {
    size_t p_all, z_all, eH, eA, eK, eSelf, nodeStart, nodeCnt, dL, dB, dC, dCnt, vx, vr, vAp, vAz, vminv, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline Smem smem_layout(int n, int K, int cap_e, int cap_d, int cap_n) {
    Smem s;
    size_t o = 0;
    s.p_all = o; o = al16(o + sizeof(float4) * 2 * (size_t)n);
    s.z_all = o; o = al16(o + sizeof(float4) * 2 * (size_t)n);
    s.eH = o; o = al16(o + sizeof(float) * 6 * (size_t)cap_e);
    s.eA = o; o = al16(o + sizeof(float4) * (size_t)K * cap_e);
    s.eK = o; o = al16(o + sizeof(unsigned short) * (size_t)K * cap_e);
    s.eSelf = o; o = al16(o + (size_t)cap_e);
    s.nodeStart = o; o = al16(o + sizeof(int) * (size_t)cap_n);
    s.nodeCnt = o; o = al16(o + sizeof(int) * (size_t)cap_n);
    s.dL = o; o = al16(o + sizeof(int) * (size_t)cap_d);
    s.dB = o; o = al16(o + sizeof(float4) * 2 * (size_t)cap_d);
    s.dC = o; o = al16(o + sizeof(int) * (size_t)(cap_n + 1));
    s.dCnt = o; o = al16(o + 16);
    s.vx = o; o = al16(o + sizeof(float4) * 2 * (size_t)cap_n);
    s.vr = o; o = al16(o + sizeof(float4) * 2 * (size_t)cap_n);
    s.vAp = o; o = al16(o + sizeof(float4) * 2 * (size_t)cap_n);
    s.vAz = o; o = al16(o + sizeof(float4) * 2 * (size_t)cap_n);
    s.vminv = o; o = al16(o + sizeof(float4) * 2 * (size_t)cap_n);
    s.total = o;
    return s;
}

__device__ __forceinline__ float3 f3_(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 cr(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float dt3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Node range of cluster rank r: nodes are split so that every CTA holds about
// the same number of CSR entries (lo_r = first node whose entry offset reaches
// r/cl of the total).  The host plan uses the same rule.
__host__ __device__ inline int part_lo(const int* ent_off, int n, int cl, int r) {
    if (r <= 0) return 0;
    if (r >= cl) return n;
    const long long target = ((long long)ent_off[n] * r) / cl;
    int a = 0, b = n;   // smallest k with ent_off[k] >= target
    while (a < b) {
        const int m = (a + b) >> 1;
        if (ent_off[m] >= target) b = m;
        else a = m + 1;
    }
    return a;
}

// rotation rows of node k applied to v
__device__ __forceinline__ float3 rot(const float4* R, int k, float3 v) {
    const float4 a = R[3 * k], b = R[3 * k + 1], c = R[3 * k + 2];
    return make_float3(a.x * v.x + a.y * v.y + a.z * v.z, b.x * v.x + b.y * v.y + b.z * v.z,
                       c.x * v.x + c.y * v.y + c.z * v.z);
}

// Block-wide FP32 sum; the result is valid in warp 0.  Fixed shuffle tree.
__device__ __forceinline__ float block_sum_f32(float v, float* s_warpf, int warp, int lane) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_warpf[warp] = v;
    __syncthreads();
    float t = 0.f;
    if (warp == 0) {
        t = s_warpf[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

// Block-wide FP32 sum of values held by lane 0 of each warp (the other lanes
// hold 0); the result is valid in warp 0.  The same fixed tree as
// block_sum_f32 (a warp's shuffle sum of one value and zeros is that value).
__device__ __forceinline__ float block_sum_lane0_f32(float v, float* s_warpf, int warp, int lane) {
    if (lane == 0) s_warpf[warp] = v;
    __syncthreads();
    float t = 0.f;
    if (warp == 0) {
        t = s_warpf[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

// Warp 0: lanes 0..cl-1 store this CTA's total (FP64) into slot `rank` of
// the partial array of cluster CTA `lane`.
__device__ __forceinline__ void publish(cg::cluster_group& cluster, double total, double* slots, int rank, int cl) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32 && lane < cl) {
        double* dst = cluster.map_shared_rank(slots, lane);
        dst[rank] = total;
    }
}

// Sum of the cl (<= 16) cluster partials in FP64 (fixed shuffle tree over 16
// lanes; lane 0 holds the total); warp 0 only.  GB300 issues an FP64 warp
// instruction at ~1.7 lane-operations per clock per SM whatever the number of
// active lanes, so four warp-wide levels beat fifteen one-lane adds (measured:
// 308 vs 323 us per 40-iteration launch on the body).
__device__ __forceinline__ double cluster_total(const double* slots, int cl) {
    double v = (int)(threadIdx.x & 31) < cl ? slots[threadIdx.x & 31] : 0.0;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int KT>
__device__ __forceinline__ void entry_term(int e, int K, int cap_e, const float4* __restrict__ eA,
                                           const unsigned short* __restrict__ eK, const float* __restrict__ eH,
                                           const unsigned char* __restrict__ eSelf, const float4* __restrict__ p_all,
                                           float (&acc)[6]) {
    float3 dv = make_float3(0.f, 0.f, 0.f);
    const int kk = KT > 0 ? KT : K;
#pragma unroll
    for (int s = 0; s < (KT > 0 ? KT : kMaxK); ++s) {
        if (KT == 0 && s >= kk) break;
        const float4 a = eA[s * cap_e + e];
        const int ks = eK[s * cap_e + e];
        const float4 pw = p_all[2 * ks], pt = p_all[2 * ks + 1];
        const float3 c = cr(f3_(pw), f3_(a));
        dv.x += a.w * (c.x + pt.x);
        dv.y += a.w * (c.y + pt.y);
        dv.z += a.w * (c.z + pt.z);
    }
    const float h00 = eH[e], h01 = eH[cap_e + e], h02 = eH[2 * cap_e + e];
    const float h11 = eH[3 * cap_e + e], h12 = eH[4 * cap_e + e], h22 = eH[5 * cap_e + e];
    const float3 q = make_float3(h00 * dv.x + h01 * dv.y + h02 * dv.z, h01 * dv.x + h11 * dv.y + h12 * dv.z,
                                 h02 * dv.x + h12 * dv.y + h22 * dv.z);
    const float4 as = eA[eSelf[e] * cap_e + e];
    const float3 c = cr(f3_(as), q);
    acc[0] += as.w * c.x; acc[1] += as.w * c.y; acc[2] += as.w * c.z;
    acc[3] += as.w * q.x; acc[4] += as.w * q.y; acc[5] += as.w * q.z;
}

template <int KT>
__global__ void __launch_bounds__(kPcgThreads, 1) pcg_cluster_kernel(const CapDesc* __restrict__ caps,
                                                                      int n_pcg, int cap_e, int cap_d, int cap_n) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_pAp_part[16];
    __shared__ double s_rz_part[16];
    __shared__ float s_warpf[kPcgWarps];
    __shared__ double s_scalar[4];   // rz, alpha, beta
    __shared__ int s_flag[2];        // stop, breakdown
    __shared__ int s_stopz;          // the last r^T z was zero (set by warp 0 before a barrier)
    __shared__ float4* s_zdst[16];   // z of every cluster CTA (distributed shared memory)

    cg::cluster_group cluster = cg::this_cluster();
    const int cl = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int cap = blockIdx.x / cl;   // one cluster per capture
    const CapDesc& C = caps[cap];
    // the solve reached its target energy: every CTA of the cluster leaves
    // before any distributed shared memory access
    if (C.sc->gn_stop) return;
    const int n = C.n, K = C.K;
    const int lo = part_lo(C.ent_off, n, cl, rank), hi = part_lo(C.ent_off, n, cl, rank + 1);
    const int nown = hi - lo;
    const Smem L = smem_layout(n, K, cap_e, cap_d, cap_n);
    float4* p_all = (float4*)(smem + L.p_all);
    float4* z_all = (float4*)(smem + L.z_all);
    float* eH = (float*)(smem + L.eH);
    float4* eA = (float4*)(smem + L.eA);
    unsigned short* eK = (unsigned short*)(smem + L.eK);
    unsigned char* eSelf = smem + L.eSelf;
    int* nodeStart = (int*)(smem + L.nodeStart);
    int* nodeCnt = (int*)(smem + L.nodeCnt);
    int* dL = (int*)(smem + L.dL);
    float4* dB = (float4*)(smem + L.dB);
    int* dOff = (int*)(smem + L.dC);
    float4* vx = (float4*)(smem + L.vx);
    float4* vr = (float4*)(smem + L.vr);
    float4* vAp = (float4*)(smem + L.vAp);
    float4* vAz = (float4*)(smem + L.vAz);
    float4* vminv = (float4*)(smem + L.vminv);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < cl) s_zdst[tid] = cluster.map_shared_rank(z_all, tid);

    // ---------------- staging ----------------
    const int e_base = C.ent_off[lo];
    const int d_base = C.edge_off[lo];
    for (int j = tid; j <= nown; j += kPcgThreads) dOff[j] = C.edge_off[lo + j] - d_base;
    // entries: each warp compacts the active entries of its nodes in place
    for (int kk = warp; kk < nown; kk += kPcgWarps) {
        const int k = lo + kk;
        const int a0 = C.ent_off[k], a1 = C.ent_off[k + 1];
        const int start = a0 - e_base;
        int cnt = 0;
        for (int jb = a0; jb < a1; jb += 32) {
            const int j = jb + lane;
            bool act = false;
            int i = 0;
            if (j < a1) {
                i = C.ent[j].x;
                act = C.ev[i].w != 0.f;
            }
            const unsigned m = __ballot_sync(0xffffffffu, act);
            if (act) {
                const int e = start + cnt + __popc(m & ((1u << lane) - 1u));
                const float4 HA = C.HA[i], HB = C.HB[i];
                eH[0 * cap_e + e] = HA.x; eH[1 * cap_e + e] = HA.y; eH[2 * cap_e + e] = HA.z;
                eH[3 * cap_e + e] = HA.w; eH[4 * cap_e + e] = HB.x; eH[5 * cap_e + e] = HB.y;
                const float3 v = f3_(C.base[i]);
                int self = 0;
                for (int s = 0; s < K; ++s) {
                    const int ks = C.bind_idx[(size_t)i * K + s];
                    const float ws = C.bind_w[(size_t)i * K + s];
                    const float4 g = C.node_g[ks];
                    const float3 a = rot(C.node_R, ks, make_float3(v.x - g.x, v.y - g.y, v.z - g.z));
                    eA[s * cap_e + e] = make_float4(a.x, a.y, a.z, ws);
                    eK[s * cap_e + e] = (unsigned short)ks;
                    if (ks == k) self = s;
                }
                eSelf[e] = (unsigned char)self;
            }
            cnt += __popc(m);
        }
        if (lane == 0) {
            nodeStart[kk] = start;
            nodeCnt[kk] = cnt;
        }
    }
    // ARAP edges of owned nodes
    for (int kk = warp; kk < nown; kk += kPcgWarps) {
        const int k = lo + kk;
        const float3 gk = f3_(C.node_g[k]);
        for (int j = C.edge_off[k] + lane; j < C.edge_off[k + 1]; j += 32) {
            const int l = C.edge_dst[j];
            const float c = C.w_arap * C.edge_s[j];
            const float3 gl = f3_(C.node_g[l]);
            const float3 bkl = rot(C.node_R, k, make_float3(gl.x - gk.x, gl.y - gk.y, gl.z - gk.z));
            const float3 blk = rot(C.node_R, l, make_float3(gk.x - gl.x, gk.y - gl.y, gk.z - gl.z));
            const int d = j - d_base;
            dL[d] = l;
            dB[2 * d] = make_float4(bkl.x, bkl.y, bkl.z, c);
            dB[2 * d + 1] = make_float4(blk.x, blk.y, blk.z, 0.f);
        }
    }
    __syncthreads();
    // vectors: x = 0, r = b, M^-1 (own nodes); initial r^T z
    float my_rz = 0.f;
    for (int j = tid; j < 2 * nown; j += kPcgThreads) {
        const float4 b = C.b[2 * lo + j];
        const float4 mi = C.minv[2 * lo + j];
        vx[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        vr[j] = b;
        vminv[j] = mi;
        my_rz += b.x * (mi.x * b.x) + b.y * (mi.y * b.y) + b.z * (mi.z * b.z);
    }
    // the first direction is z_0 = M^-1 b: every CTA holds z for all nodes;
    // the owned p and A p start at zero (p_0 = z_0 + 0 p, A p_0 = A z_0 + 0)
    for (int j = tid; j < 2 * n; j += kPcgThreads) {
        const float4 b = C.b[j];
        const float4 mi = C.minv[j];
        z_all[j] = make_float4(mi.x * b.x, mi.y * b.y, mi.z * b.z, 0.f);
    }
    for (int j = tid; j < 2 * nown; j += kPcgThreads) {
        p_all[2 * lo + j] = make_float4(0.f, 0.f, 0.f, 0.f);
        vAp[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    {
        const float t = block_sum_f32(my_rz, s_warpf, warp, lane);
        publish(cluster, (double)t, s_rz_part, rank, cl);
    }
    cluster.sync();
    if (warp == 0) {
        const double rz = cluster_total(s_rz_part, cl);
        if (lane == 0) {
            s_scalar[0] = rz;
            s_scalar[2] = 0.0;   // beta of the first direction
            s_flag[0] = rz == 0.0 ? 1 : 0;
            s_flag[1] = 0;
            s_stopz = 0;
        }
    }
    __syncthreads();

    // ---------------- iterations ----------------
    // The product is taken on z: A p = A z + beta A p_prev (A is linear), so
    // the heavy A z of iteration it runs while warp 0 forms beta from the
    // previous r^T z, and only the owned entries of p and A p are updated.
    // Flags written inside an iteration are read only after a barrier, so
    // every thread leaves the loop at the same point.
    int iters = 0;
    bool completed = true;
    const int n_it = s_flag[0] ? 0 : n_pcg;
    for (int it = 0; it < n_it; ++it) {
        // warp 0 first: beta = r^T z / (r^T z)_prev from the cluster partials
        if (it > 0 && warp == 0) {
            const double rz_new = cluster_total(s_rz_part, cl);
            if (lane == 0) {
                if (rz_new == 0.0) {
                    s_stopz = 1;
                } else {
                    s_scalar[2] = (double)__fdiv_rn((float)rz_new, (float)s_scalar[0]);
                    s_scalar[0] = rz_new;
                }
            }
        }
        // phase 1: (A z)_k for the owned nodes, one warp per node (warps 1..31:
        // warp 0 is busy with beta): its CSR entries and ARAP edges
        // lane-strided, a fixed 6-float shuffle tree
        for (int kk = warp - 1; kk < nown; kk += kPcgWarps - 1) {
            if (kk < 0) break;
            float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const int e0 = nodeStart[kk], ne = nodeCnt[kk];
            for (int j = lane; j < ne; j += 32) entry_term<KT>(e0 + j, K, cap_e, eA, eK, eH, eSelf, z_all, acc);
            const int k = lo + kk;
            const float3 pw = f3_(z_all[2 * k]), pt = f3_(z_all[2 * k + 1]);
            for (int d = dOff[kk] + lane; d < dOff[kk + 1]; d += 32) {
                const int l = dL[d];
                const float4 bk = dB[2 * d], bl = dB[2 * d + 1];
                const float cc = bk.w;
                const float3 plw = f3_(z_all[2 * l]), plt = f3_(z_all[2 * l + 1]);
                const float3 D0 = cr(pw, f3_(bk));
                const float3 D = make_float3(D0.x + pt.x - plt.x, D0.y + pt.y - plt.y, D0.z + pt.z - plt.z);
                const float3 bD = cr(f3_(bk), D);
                const float3 E0 = cr(plw, f3_(bl));
                acc[0] += cc * bD.x;
                acc[1] += cc * bD.y;
                acc[2] += cc * bD.z;
                acc[3] += cc * D.x - cc * (E0.x + plt.x - pt.x);
                acc[4] += cc * D.y - cc * (E0.y + plt.y - pt.y);
                acc[5] += cc * D.z - cc * (E0.z + plt.z - pt.z);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < 6; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            if (lane == 0) {
                vAz[2 * kk] = make_float4(acc[0], acc[1], acc[2], 0.f);
                vAz[2 * kk + 1] = make_float4(acc[3], acc[4], acc[5], 0.f);
            }
        }
        __syncthreads();
        if (s_stopz) {
            completed = false;
            break;
        }
        // owned p = z + beta p, A p = A z + beta A p; p^T A p (FP32 per CTA)
        const float beta = (float)s_scalar[2];
        float my_pap = 0.f;
        for (int j = tid; j < 2 * nown; j += kPcgThreads) {
            const float4 z = z_all[2 * lo + j], pp = p_all[2 * lo + j];
            const float4 az = vAz[j], ap0 = vAp[j];
            const float4 p = make_float4(z.x + beta * pp.x, z.y + beta * pp.y, z.z + beta * pp.z, 0.f);
            const float4 ap = make_float4(az.x + beta * ap0.x, az.y + beta * ap0.y, az.z + beta * ap0.z, 0.f);
            p_all[2 * lo + j] = p;
            vAp[j] = ap;
            my_pap += p.x * ap.x + p.y * ap.y + p.z * ap.z;
        }
        {
            const float t = block_sum_f32(my_pap, s_warpf, warp, lane);
            publish(cluster, (double)t, s_pAp_part, rank, cl);
        }
        cluster.sync();
        if (warp == 0) {
            const double pAp = cluster_total(s_pAp_part, cl);
            if (lane == 0) {
                if (!(pAp > 0.0)) {
                    s_flag[0] = 1;
                    s_flag[1] = 1;
                } else {
                    // the step length is applied in FP32: divide the FP64 sums in FP32
                    s_scalar[1] = (double)__fdiv_rn((float)s_scalar[0], (float)pAp);
                }
            }
        }
        __syncthreads();
        if (s_flag[0]) {
            completed = false;
            break;
        }
        // phase 2: x, r, z for owned nodes; r^T z partial
        const float alpha = (float)s_scalar[1];
        float my_rz2 = 0.f;
        for (int j = tid; j < 2 * nown; j += kPcgThreads) {
            const float4 p = p_all[2 * lo + j];
            const float4 ap = vAp[j];
            float4 x = vx[j], r = vr[j];
            x.x += alpha * p.x; x.y += alpha * p.y; x.z += alpha * p.z;
            r.x -= alpha * ap.x; r.y -= alpha * ap.y; r.z -= alpha * ap.z;
            const float4 mi = vminv[j];
            const float4 z = make_float4(mi.x * r.x, mi.y * r.y, mi.z * r.z, 0.f);
            vx[j] = x;
            vr[j] = r;
            // the owned z into every CTA's copy (this one's included)
            for (int d = 0; d < cl; ++d) s_zdst[d][2 * lo + j] = z;
            my_rz2 += r.x * z.x + r.y * z.y + r.z * z.z;
        }
        {
            const float t = block_sum_f32(my_rz2, s_warpf, warp, lane);
            publish(cluster, (double)t, s_rz_part, rank, cl);
        }
        cluster.sync();
        ++iters;
    }
    // the r^T z of the last iteration (its beta is never needed)
    if (completed && iters > 0 && warp == 0) {
        const double rz_new = cluster_total(s_rz_part, cl);
        if (lane == 0) {
            if (rz_new == 0.0) s_flag[0] = 1;
            else s_scalar[0] = rz_new;
        }
    }
    if (tid == 0 && s_stopz) s_flag[0] = 1;
    __syncthreads();
    // ---------------- results ----------------
    for (int j = tid; j < 2 * nown; j += kPcgThreads) C.x[2 * lo + j] = vx[j];
    if (rank == 0 && tid == 0) {
        Scalars* sc = C.sc;
        sc->iters = iters;
        sc->breakdown = s_flag[1];
        sc->stop = s_flag[0];
        sc->rz = s_scalar[0];
    }
    // no CTA may exit while others can still write into its shared memory
    cluster.sync();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static bool try_plan(int cl, int n, int K, const int* ent_off, const int* edge_off, int max_smem, PcgPlan& pl) {
    if (n < cl) return false;
    int cap_e = 0, cap_d = 0, cap_n = 0;
    for (int r = 0; r < cl; ++r) {
        const int lo = part_lo(ent_off, n, cl, r), hi = part_lo(ent_off, n, cl, r + 1);
        cap_e = std::max(cap_e, ent_off[hi] - ent_off[lo]);
        cap_d = std::max(cap_d, edge_off[hi] - edge_off[lo]);
        cap_n = std::max(cap_n, hi - lo);
    }
    const Smem L = smem_layout(n, K, std::max(cap_e, 1), std::max(cap_d, 1), std::max(cap_n, 1));
    if (L.total > (size_t)max_smem || n > 65535) return false;
    pl = {cl, std::max(cap_e, 1), std::max(cap_d, 1), std::max(cap_n, 1), L.total};
    return true;
}

typedef void (*PcgKernel)(const CapDesc*, int, int, int, int);

static PcgKernel pcg_kernel_for(int K) {
    if (K == 4) return pcg_cluster_kernel<4>;
    if (K == 8) return pcg_cluster_kernel<8>;
    return pcg_cluster_kernel<0>;
}

// The device can run the kernel for K with this plan (shared memory opt-in,
// non-portable cluster size, at least one resident cluster).
static int max_dynamic_smem();

static bool accept_plan(int K, const PcgPlan& pl) {
    const PcgKernel kern = pcg_kernel_for(K);
    // the attribute caps every later launch of this kernel (other contexts and
    // batches included), so it is raised to the device limit, never lowered
    if (pl.smem > (size_t)max_dynamic_smem() ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dynamic_smem()) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (pl.cl > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.cl);
    cfg.blockDim = dim3(kPcgThreads);
    cfg.dynamicSmemBytes = pl.smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = pl.cl;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return false;
    }
    return true;
}

static int max_dynamic_smem() {
    int dev = 0, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return max_optin - 1024;   // the kernel's own __shared__ arrays (< 1 KB)
}

// Choose the cluster size: the smallest of {8, 16} whose per-CTA staging fits
// in shared memory and that the device can schedule.  Returns false if none
// (the multi-kernel PCG is used then).
bool plan_pcg_cluster(int n, int K, const int* ent_off_host, const int* edge_off_host, PcgPlan* out) {
    const int max_smem = max_dynamic_smem();
    for (int cl : {8, 16}) {
        PcgPlan pl;
        if (!try_plan(cl, n, K, ent_off_host, edge_off_host, max_smem, pl)) continue;
        if (!accept_plan(K, pl)) continue;
        *out = pl;
        return true;
    }
    return false;
}

bool plan_pcg_cluster_group(int cl, const int* n, int K, const int* const* ent_off_host,
                            const int* const* edge_off_host, int count, PcgPlan* out) {
    int cap_e = 1, cap_d = 1, cap_n = 1, nmax = 1;
    for (int c = 0; c < count; ++c) {
        if (n[c] < cl || n[c] > 65535) return false;
        nmax = std::max(nmax, n[c]);
        for (int r = 0; r < cl; ++r) {
            const int lo = part_lo(ent_off_host[c], n[c], cl, r), hi = part_lo(ent_off_host[c], n[c], cl, r + 1);
            cap_e = std::max(cap_e, ent_off_host[c][hi] - ent_off_host[c][lo]);
            cap_d = std::max(cap_d, edge_off_host[c][hi] - edge_off_host[c][lo]);
            cap_n = std::max(cap_n, hi - lo);
        }
    }
    const Smem L = smem_layout(nmax, K, cap_e, cap_d, cap_n);
    if (L.total > (size_t)max_dynamic_smem()) return false;
    const PcgPlan pl = {cl, cap_e, cap_d, cap_n, L.total};
    if (!accept_plan(K, pl)) return false;
    *out = pl;
    return true;
}

cudaError_t launch_pcg_cluster(const CapDesc* dC, const PcgPlan& pl, int K, int n_pcg, cudaStream_t st, int ncap) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.cl * ncap);
    cfg.blockDim = dim3(kPcgThreads);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = pl.cl;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pcg_kernel_for(K), dC, n_pcg, pl.cap_e, pl.cap_d, pl.cap_n);
}

}  // namespace lc

// Cluster-persistent Jacobi-PCG for one Gauss-Newton step (Sec. 4: normal
// equations J^T J delta = -J^T F, Jacobi preconditioner, fixed iteration
// count), all n_pcg iterations in one launch.
//
// One thread-block cluster of CL CTAs solves one capture.  The capture's
// nodes are split into kPcgLeaves spatially compact leaves (recursive
// coordinate bisection at graph build, balanced by node count);
// CTA r owns the nodes of leaves r*L/CL .. (r+1)*L/CL - 1, so most vertices
// have all K of their nodes in one CTA.  At the start the CTA stages in its
// own shared memory:
//   * its local vertices (active vertices bound to an owned node, ascending
//     id): H_i and, per slot, (c_is = w_is a_is, w_is) and the node index;
//   * per owned node its entries (local vertex, slot) and its ARAP edges
//     (l, c = w_a s_kl, b_kl = R_k (g_l - g_k), b_lk = R_l (g_k - g_l));
//   * the preconditioned residual z of all nodes (every CTA holds a copy).
// One iteration is computed from shared memory alone:
//   phase A: q_i = H_i sum_s (z_omega,s x c_is + w_is z_t,s) once per active
//     local vertex (one thread each), and each owned ARAP edge's
//     contribution to its source node (one thread each);
//   phase B: (J^T J z)_k = sum_entries [c_is x q_i ; w_is q_i] + the edges'
//     contributions, sixteen threads per owned node (each a share of its
//     entries and edges, all six components), combined by shuffles;
//   the lanes that finish a node's product apply p = z + beta p and
//   A p = A z + beta A p (A is linear; warp 0 forms beta during phase A) and
//   add their terms of p.Ap; then alpha (warp 0), x, r, z and r.z.
// Vectors, products and dot products are compensated FP32 pairs (fpair.cuh,
// jtj_pair.cuh): CG at tens of iterations on these systems amplifies FP32
// rounding of its recurrences to percent-level changes of the iterate.  The
// operator data stay FP32.  Each CTA's dot-product total (a pair) is
// converted exactly to FP64 and written into every CTA's slot array through
// distributed shared memory; all CTAs sum the slots in rank order in FP64
// (deterministic, identical everywhere), and alpha / beta are pair divisions
// of those totals.  The new z of an owned node goes into the copies of the
// CTAs that read it (a per-node mask built with the partition) as 16-byte
// distributed-shared-memory stores.  Two hardware cluster barriers
// per iteration; no spin loops, no global-memory round trips.
#include <algorithm>
#include <numeric>

#include <cooperative_groups.h>

#include "jtj_pair.cuh"
#include "lc_internal.cuh"

namespace cg = cooperative_groups;

namespace lc {

constexpr int kPcgThreads = 1024;
constexpr int kPcgWarps = kPcgThreads / 32;
constexpr int kNodeLanes = 16;  // phase B threads per owned node
constexpr int kVecArrays = 9;    // x_h, x_l, minv, p_h, p_l, r_h, r_l, ap_h, ap_l

// shared-memory carve-up (byte offsets, all 16-byte aligned)
struct Smem {
    size_t z_all, lvC, lvK, lvH, lvQ, lmap, eUS, ownK, nodeStart, nodeCnt, dL, dB, dE, dNode, dOff, vec, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline Smem smem_layout(int n, int K, int cap_v, int cap_e, int cap_d, int cap_n) {
    Smem s;
    size_t o = 0;
    s.z_all = o; o = al16(o + sizeof(float) * 12 * (size_t)n);
    s.lvC = o; o = al16(o + sizeof(float4) * (size_t)K * cap_v);
    s.lvK = o; o = al16(o + sizeof(unsigned short) * (size_t)K * cap_v);
    s.lvH = o; o = al16(o + sizeof(float) * 6 * (size_t)cap_v);
    s.lvQ = o; o = al16(o + sizeof(float2) * 3 * (size_t)cap_v);
    s.lmap = o; o = al16(o + sizeof(int) * (size_t)cap_v);
    s.eUS = o; o = al16(o + sizeof(unsigned) * (size_t)cap_e);
    s.ownK = o; o = al16(o + sizeof(int) * (size_t)cap_n);
    s.nodeStart = o; o = al16(o + sizeof(int) * (size_t)(cap_n + 1));
    s.nodeCnt = o; o = al16(o + sizeof(int) * (size_t)cap_n);
    s.dL = o; o = al16(o + sizeof(int) * (size_t)cap_d);
    s.dB = o; o = al16(o + sizeof(float4) * 2 * (size_t)cap_d);
    s.dE = o; o = al16(o + sizeof(float) * 12 * (size_t)cap_d);
    s.dNode = o; o = al16(o + sizeof(int) * (size_t)cap_d);
    s.dOff = o; o = al16(o + sizeof(int) * (size_t)(cap_n + 1));
    s.vec = o; o = al16(o + sizeof(float) * kVecArrays * 6 * (size_t)cap_n);
    s.total = o;
    return s;
}

__host__ __device__ inline int log2_cl(int cl) { return cl >= 16 ? 4 : cl >= 8 ? 3 : cl >= 4 ? 2 : cl >= 2 ? 1 : 0; }

// Block-wide sum of one pair per thread when only warps 0 .. nw-1 (nw <= 32)
// hold nonzero values: those warps reduce, the others only pass the barrier;
// the total is valid in warp 0.
__device__ __forceinline__ fp2 block_sum_fp2_warps(fp2 v, float2* sh, int nw) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w < nw) {
        v = fp2_warp_sum(v);
        if (l == 0) sh[w] = make_float2(v.h, v.l);
    }
    __syncthreads();
    fp2 t = {0.f, 0.f};
    if (w == 0) {
        const float2 a = l < nw ? sh[l] : make_float2(0.f, 0.f);
        t = fp2_warp_sum(fp2{a.x, a.y});
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

// Sum of the cl (<= 16) cluster partials in FP64: a fixed xor-shuffle tree
// over lanes 0..15 (which then hold the total), broadcast from lane 0 so that
// every lane of the calling warp returns the same value (a caller that
// branches on it in every lane then branches alike).
__device__ __forceinline__ double cluster_total(const double* slots, int cl) {
    double v = (int)(threadIdx.x & 31) < cl ? slots[threadIdx.x & 31] : 0.0;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

// Block-wide exclusive prefix sum of cnt[0..m) into off[0..m] (off[m] = total),
// by warp 0 in chunks of 32; the caller synchronises afterwards.
__device__ __forceinline__ void block_exclusive_scan(const int* cnt, int* off, int m) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    int base = 0;
    for (int c0 = 0; c0 < m; c0 += 32) {
        const int j = c0 + lane;
        const int v = j < m ? cnt[j] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (j < m) off[j] = base + incl - v;
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) off[m] = base;
}

template <int KT>
__global__ void __launch_bounds__(kPcgThreads, 1) pcg_cluster_kernel(const CapDesc* __restrict__ caps, int n_pcg,
                                                                      int cap_v, int cap_e, int cap_d, int cap_n) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_pAp_part[16];
    __shared__ double s_rz_part[16];
    __shared__ float2 s_warp2[kPcgWarps];
    __shared__ int s_warpi[kPcgWarps + 1];
    __shared__ float s_scalar[6];    // rz (pair), alpha (pair), beta (pair)
    __shared__ int s_flag[3];        // stop, breakdown, capacity overflow
    __shared__ int s_stopz;          // the last r^T z was zero (set by warp 0 before a barrier)
    __shared__ int s_nv;             // local vertices
    __shared__ int s_capflag[16];    // every cluster CTA's capacity flag (written remotely)
    __shared__ float* s_zdst[16];    // z of every cluster CTA (distributed shared memory)

    cg::cluster_group cluster = cg::this_cluster();
    const int cl = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int cap = blockIdx.x / cl;   // one cluster per capture
    const CapDesc& C = caps[cap];
    // the solve reached its target energy: every CTA of the cluster leaves
    // before any distributed shared memory access
    if (C.sc->gn_stop) return;
    const int n = C.n, K = C.K, N = C.N;
    const int lpc = kPcgLeaves / cl;             // leaves per CTA
    const int shift = log2_cl(kPcgLeaves) - log2_cl(cl);   // leaf -> owner rank
    const int lo = C.pcg_leaf_off[rank * lpc], hi = C.pcg_leaf_off[(rank + 1) * lpc];
    // a plan that does not cover this capture owns nothing and reports it
    const bool over = hi - lo > cap_n || hi < lo;
    const int nown = over ? 0 : hi - lo;
    const Smem L = smem_layout(n, K, cap_v, cap_e, cap_d, cap_n);
    float* z_all = (float*)(smem + L.z_all);
    float4* lvC = (float4*)(smem + L.lvC);
    unsigned short* lvK = (unsigned short*)(smem + L.lvK);
    float* lvH = (float*)(smem + L.lvH);
    float2* lvQ = (float2*)(smem + L.lvQ);
    int* lmap = (int*)(smem + L.lmap);   // local vertex -> its active index, -1 if inactive
    unsigned* eUS = (unsigned*)(smem + L.eUS);
    int* perm = (int*)(smem + L.ownK);   // owned node ids
    int* nodeStart = (int*)(smem + L.nodeStart);
    int* nodeCnt = (int*)(smem + L.nodeCnt);
    int* dL = (int*)(smem + L.dL);
    float4* dB = (float4*)(smem + L.dB);
    float* dE = (float*)(smem + L.dE);        // per owned edge: its 6 output pairs of this iteration
    int* dEdgeNode = (int*)(smem + L.dNode);  // owned node of each owned edge
    int* dOff = (int*)(smem + L.dOff);
    float* vbase = (float*)(smem + L.vec);
    const int V6 = 6 * cap_n;
    float* x_h = vbase;
    float* x_l = vbase + V6;
    float* vminv = vbase + 2 * V6;
    float* p_h = vbase + 3 * V6;
    float* p_l = vbase + 4 * V6;
    float* r_h = vbase + 5 * V6;
    float* r_l = vbase + 6 * V6;
    float* ap_h = vbase + 7 * V6;
    float* ap_l = vbase + 8 * V6;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < cl) s_zdst[tid] = cluster.map_shared_rank(z_all, tid);
    if (tid == 0) {
        s_flag[2] = over ? 1 : 0;
        s_nv = 0;
    }
    for (int j = tid; j < nown; j += kPcgThreads) perm[j] = C.pcg_perm[lo + j];
    __syncthreads();

    // ---------------- staging ----------------
    // the CTA's local vertices (a table fixed per graph), compacted to the
    // active ones in order: one vertex per thread per round
    const int ti = cl == 16 ? 1 : 0;
    const int loc0 = C.pcg_loc_off[ti][rank];
    const int nloc = C.pcg_loc_off[ti][rank + 1] - loc0;
    const int* __restrict__ loc_vid = C.pcg_loc_vid[ti] + loc0;
    if (tid == 0 && nloc > cap_v) s_flag[2] = 1;
    for (int u0 = 0; u0 < nloc && u0 < cap_v; u0 += kPcgThreads) {
        const int u = u0 + tid;
        const int i = u < nloc && u < cap_v ? loc_vid[u] : 0;
        const bool act = u < nloc && u < cap_v && C.ev[i].w != 0.f;
        const unsigned m = __ballot_sync(0xffffffffu, act);
        if (lane == 0) s_warpi[warp] = __popc(m);
        __syncthreads();
        if (warp == 0) {
            const int v = s_warpi[lane];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            s_warpi[lane] = incl - v;
            if (lane == 31) s_warpi[kPcgWarps] = incl;
        }
        __syncthreads();
        const int base = s_nv;
        if (u < nloc && u < cap_v) {
            const int a = base + s_warpi[warp] + __popc(m & ((1u << lane) - 1u));
            lmap[u] = act ? a : -1;
            if (act) {
                const float4 HA = C.HA[i], HB = C.HB[i];
                lvH[0 * cap_v + a] = HA.x; lvH[1 * cap_v + a] = HA.y; lvH[2 * cap_v + a] = HA.z;
                lvH[3 * cap_v + a] = HA.w; lvH[4 * cap_v + a] = HB.x; lvH[5 * cap_v + a] = HB.y;
                const float4 v = C.base[i];
                for (int s = 0; s < K; ++s) {
                    const int ks = C.bind_idx[(size_t)i * K + s];
                    lvC[s * cap_v + a] = staged_coef(C.node_R, ks, v, C.node_g[ks], C.bind_w[(size_t)i * K + s]);
                    lvK[s * cap_v + a] = (unsigned short)ks;
                }
            }
        }
        __syncthreads();
        if (tid == 0) s_nv = base + s_warpi[kPcgWarps];
        __syncthreads();
    }
    const int nv = s_nv;
    // entry and edge counts of the owned nodes, their offsets
    for (int j = tid; j < nown; j += kPcgThreads) {
        const int k = perm[j];
        nodeCnt[j] = C.ent_off[k + 1] - C.ent_off[k];
        dOff[j] = C.edge_off[k + 1] - C.edge_off[k];   // edge counts, scanned in place
    }
    __syncthreads();
    block_exclusive_scan(nodeCnt, nodeStart, nown);
    block_exclusive_scan(dOff, dOff, nown);
    __syncthreads();
    if (tid == 0 && (dOff[nown] > cap_d || nodeStart[nown] > cap_e)) s_flag[2] = 1;
    __syncthreads();
    // entries: each warp compacts the active entries of its nodes in place,
    // remapping the table's local vertex to its active index
    const unsigned* __restrict__ ent_us = C.pcg_ent_us[ti] + C.pcg_eus_off[ti][rank];
    const unsigned short* __restrict__ zdst = C.pcg_zdst[ti];   // CTAs reading each node's z
    for (int j = warp; j < nown && !s_flag[2]; j += kPcgWarps) {
        const int start = nodeStart[j], ne = nodeStart[j + 1] - start;
        int cnt = 0;
        for (int e0 = 0; e0 < ne; e0 += 32) {
            const int e = e0 + lane;
            bool act = false;
            unsigned us = 0;
            if (e < ne) {
                const unsigned t = ent_us[start + e];
                const int m = lmap[t & 0xffffu];
                act = m >= 0;
                us = (unsigned)m | (t & 0xffff0000u);
            }
            const unsigned bm = __ballot_sync(0xffffffffu, act);
            if (act) eUS[start + cnt + __popc(bm & ((1u << lane) - 1u))] = us;
            cnt += __popc(bm);
        }
        if (lane == 0) nodeCnt[j] = cnt;
    }
    // ARAP edges of owned nodes
    for (int j = warp; j < nown && !s_flag[2]; j += kPcgWarps) {
        const int k = perm[j];
        const float4 gk = C.node_g[k];
        const int d0 = dOff[j];
        for (int e = C.edge_off[k] + lane; e < C.edge_off[k + 1]; e += 32) {
            const int l = C.edge_dst[e];
            const float4 gl = C.node_g[l];
            const float3 bkl = staged_edge_offset(C.node_R, k, gk, gl);
            const float3 blk = staged_edge_offset(C.node_R, l, gl, gk);
            const int d = d0 + (e - C.edge_off[k]);
            dL[d] = l;
            dEdgeNode[d] = j;
            dB[2 * d] = make_float4(bkl.x, bkl.y, bkl.z, C.w_arap * C.edge_s[e]);
            dB[2 * d + 1] = make_float4(blk.x, blk.y, blk.z, 0.f);
        }
    }
    // vectors of the owned nodes: x = 0, r = b, M^-1; p, A p = 0; initial r^T z
    fp2acc my_rz;
    for (int e = tid; e < 6 * nown; e += kPcgThreads) {
        const int k = perm[e / 6], c = e % 6;
        const float b = ((const float*)C.b)[8 * k + (c / 3) * 4 + c % 3];
        const float mi = ((const float*)C.minv)[8 * k + (c / 3) * 4 + c % 3];
        x_h[e] = 0.f; x_l[e] = 0.f;
        r_h[e] = b; r_l[e] = 0.f;
        vminv[e] = mi;
        p_h[e] = 0.f; p_l[e] = 0.f;
        ap_h[e] = 0.f; ap_l[e] = 0.f;
        my_rz.mac(b, two_prod(mi, b));
    }
    // the first direction is z_0 = M^-1 b: every CTA holds z for all nodes
    for (int e = tid; e < 6 * n; e += kPcgThreads) {
        const int k = e / 6, c = e % 6;
        const float b = ((const float*)C.b)[8 * k + (c / 3) * 4 + c % 3];
        const float mi = ((const float*)C.minv)[8 * k + (c / 3) * 4 + c % 3];
        const fp2 z = two_prod(mi, b);
        z_all[12 * k + c] = z.h;
        z_all[12 * k + 6 + c] = z.l;
    }
    {
        const fp2 t = block_sum_fp2_warps(my_rz.get(), s_warp2, (6 * nown + 31) / 32);
        publish(cluster, fp2_to_double(t), s_rz_part, rank, cl);
        // the capacity flags too: the iteration count below must be the same
        // in every CTA of the cluster (each runs the same cluster barriers)
        if (tid < cl) cluster.map_shared_rank(s_capflag, tid)[rank] = s_flag[2];
    }
    cluster.sync();
    if (warp == 0) {
        const double rz = cluster_total(s_rz_part, cl);
        const int anyf = __any_sync(0xffffffffu, lane < cl && s_capflag[lane] != 0);
        if (lane == 0) {
            s_flag[2] = anyf ? 1 : 0;
            const fp2 r = fp2_from_double(rz);
            s_scalar[0] = r.h; s_scalar[1] = r.l;
            s_scalar[4] = 0.f; s_scalar[5] = 0.f;   // beta of the first direction
            s_flag[0] = rz == 0.0 ? 1 : 0;
            s_flag[1] = 0;
            s_stopz = 0;
        }
    }
    __syncthreads();

    // ---------------- iterations ----------------
    // The product is taken on z: A p = A z + beta A p_prev (A is linear), so
    // the vertex phase of iteration it runs while warp 0 forms beta from the
    // previous r^T z, and only the owned entries of p and A p are updated.
    // Flags written inside an iteration are read only after a barrier, so
    // every thread leaves the loop at the same point.
    int iters = 0;
    bool completed = true;
    const int n_it = (s_flag[0] || s_flag[2]) ? 0 : n_pcg;
    for (int it = 0; it < n_it; ++it) {
        if (warp == 0) {
            if (it > 0) {
                const double rz_new = cluster_total(s_rz_part, cl);
                if (lane == 0) {
                    if (rz_new == 0.0) {
                        s_stopz = 1;
                    } else {
                        const fp2 rn = fp2_from_double(rz_new);
                        const fp2 beta = fp2_div(rn, fp2{s_scalar[0], s_scalar[1]});
                        s_scalar[4] = beta.h; s_scalar[5] = beta.l;
                        s_scalar[0] = rn.h; s_scalar[1] = rn.l;
                    }
                }
            }
        } else {
            // phase A (warps 1..31): one thread per active local vertex forms
            // q_i = H_i J_i z (three independent component chains); the
            // threads after the vertices form each owned ARAP edge's
            // contribution to its source node
            const int nd = dOff[nown];
            for (int t = tid - 32; t < nv + nd; t += kPcgThreads - 32) {
                if (t < nv) {
                    const int u = t;
                    fp2acc dv[3];
#pragma unroll
                    for (int s = 0; s < (KT > 0 ? KT : kMaxK); ++s) {
                        if (KT == 0 && s >= K) break;
                        jtj_slot(lvC[s * cap_v + u], node_pair12(z_all + 12 * (int)lvK[s * cap_v + u]), dv);
                    }
                    const float h[6] = {lvH[u], lvH[cap_v + u], lvH[2 * cap_v + u],
                                        lvH[3 * cap_v + u], lvH[4 * cap_v + u], lvH[5 * cap_v + u]};
                    const fp2 d[3] = {dv[0].get(), dv[1].get(), dv[2].get()};
                    fp2 q[3];
                    jtj_block(h, d, q);
                    lvQ[u] = make_float2(q[0].h, q[0].l);
                    lvQ[cap_v + u] = make_float2(q[1].h, q[1].l);
                    lvQ[2 * cap_v + u] = make_float2(q[2].h, q[2].l);
                } else {
                    // owned edge d of node j (k -> l): c [b_kl x D ; D - E]
                    const int d = t - nv;
                    const int j = dEdgeNode[d];
                    fp2acc acc[6];
                    jtj_edge(dB[2 * d], dB[2 * d + 1], node_pair12(z_all + 12 * perm[j]),
                             node_pair12(z_all + 12 * dL[d]), acc);
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        const fp2 v = acc[c].get();
                        dE[(2 * c) * cap_d + d] = v.h;
                        dE[(2 * c + 1) * cap_d + d] = v.l;
                    }
                }
            }
        }
        __syncthreads();
        if (s_stopz) {
            completed = false;
            break;
        }
        // phase B: (A z)_k, kNodeLanes threads per owned node, each a share of
        // its entries and edges accumulating all six components; the partial
        // vectors are combined by a transposed shuffle reduction after which
        // lane h of the group holds component h >> 1, and that lane applies
        // p = z + beta p, A p = A z + beta A p and adds its term of p^T A p.
        // Warps without a node skip.
        const fp2 beta = {s_scalar[4], s_scalar[5]};
        fp2acc my_pap;
        for (int t0 = 0; t0 < nown * kNodeLanes; t0 += kPcgThreads) {
            if (t0 + 32 * warp >= nown * kNodeLanes) continue;
            const int t = t0 + tid;
            const bool on = t < nown * kNodeLanes;
            const int h = t & (kNodeLanes - 1), j = on ? t / kNodeLanes : 0;
            fp2acc acc[6];
            if (on) {
                const int e0 = nodeStart[j], ne = nodeCnt[j];
                for (int e = h; e < ne; e += kNodeLanes) {
                    const unsigned us = eUS[e0 + e];
                    const int u = (int)(us & 0xffffu), s = (int)(us >> 16);
                    const float2 q0 = lvQ[u], q1 = lvQ[cap_v + u], q2 = lvQ[2 * cap_v + u];
                    const fp2 q[3] = {{q0.x, q0.y}, {q1.x, q1.y}, {q2.x, q2.y}};
                    jtj_entry(lvC[s * cap_v + u], q, acc);
                }
                for (int d = dOff[j] + h; d < dOff[j + 1]; d += kNodeLanes)
#pragma unroll
                    for (int c = 0; c < 6; ++c) acc[c].add(fp2{dE[(2 * c) * cap_d + d], dE[(2 * c + 1) * cap_d + d]});
            }
            fp2 v[8];
#pragma unroll
            for (int c = 0; c < 6; ++c) v[c] = acc[c].get();
            v[6] = v[7] = fp2{0.f, 0.f};
            // transposed reduction over the 16 lanes of the node: at each
            // level a lane keeps half of its slots and adds its partner's
            // copy of them; lane h ends with slot h >> 1 (lanes h, h ^ 1 alike)
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const bool up = h & 8;
                const fp2 send = up ? v[m] : v[4 + m];
                fp2 recv;
                recv.h = __shfl_xor_sync(0xffffffffu, send.h, 8);
                recv.l = __shfl_xor_sync(0xffffffffu, send.l, 8);
                v[m] = fp2_add(up ? v[4 + m] : v[m], recv);
            }
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const bool up = h & 4;
                const fp2 send = up ? v[m] : v[2 + m];
                fp2 recv;
                recv.h = __shfl_xor_sync(0xffffffffu, send.h, 4);
                recv.l = __shfl_xor_sync(0xffffffffu, send.l, 4);
                v[m] = fp2_add(up ? v[2 + m] : v[m], recv);
            }
            {
                const bool up = h & 2;
                const fp2 send = up ? v[0] : v[1];
                fp2 recv;
                recv.h = __shfl_xor_sync(0xffffffffu, send.h, 2);
                recv.l = __shfl_xor_sync(0xffffffffu, send.l, 2);
                v[0] = fp2_add(up ? v[1] : v[0], recv);
            }
            {
                fp2 recv;
                recv.h = __shfl_xor_sync(0xffffffffu, v[0].h, 1);
                recv.l = __shfl_xor_sync(0xffffffffu, v[0].l, 1);
                v[0] = fp2_add(v[0], recv);
            }
            if (on && (h & 1) == 0 && (h >> 1) < 6) {
                const int c = h >> 1, e = 6 * j + c, k = perm[j];
                const fp2 z = {z_all[12 * k + c], z_all[12 * k + 6 + c]};
                const fp2 p = fp2_add(z, fp2_mul(beta, fp2{p_h[e], p_l[e]}));
                const fp2 ap = fp2_add(v[0], fp2_mul(beta, fp2{ap_h[e], ap_l[e]}));
                p_h[e] = p.h; p_l[e] = p.l;
                ap_h[e] = ap.h; ap_l[e] = ap.l;
                my_pap.mac(p, ap);
            }
        }
        {
            const fp2 t = block_sum_fp2_warps(my_pap.get(), s_warp2, (nown * kNodeLanes + 31) / 32);
            publish(cluster, fp2_to_double(t), s_pAp_part, rank, cl);
        }
        cluster.sync();
        // warp 0 forms p^T A p and alpha (GB300's FP64 pipe issues a warp
        // instruction in ~19 clocks: one warp, not all of them, does this)
        if (warp == 0) {
            const double pAp = cluster_total(s_pAp_part, cl);
            if (lane == 0) {
                if (!(pAp > 0.0)) {
                    s_flag[0] = 1;
                    s_flag[1] = 1;
                } else {
                    const fp2 alpha = fp2_div(fp2{s_scalar[0], s_scalar[1]}, fp2_from_double(pAp));
                    s_scalar[2] = alpha.h; s_scalar[3] = alpha.l;
                }
            }
        }
        __syncthreads();
        if (s_flag[0]) {
            completed = false;
            break;
        }
        const fp2 alpha = {s_scalar[2], s_scalar[3]};
        // x, r, z for owned nodes; r^T z partial
        fp2acc my_rz2;
        for (int e = tid; e < 6 * nown; e += kPcgThreads) {
            const int k = perm[e / 6], c = e % 6;
            const fp2 x = fp2_add(fp2{x_h[e], x_l[e]}, fp2_mul(alpha, fp2{p_h[e], p_l[e]}));
            const fp2 r = fp2_sub(fp2{r_h[e], r_l[e]}, fp2_mul(alpha, fp2{ap_h[e], ap_l[e]}));
            const fp2 z = fp2_scale(vminv[e], r);
            x_h[e] = x.h; x_l[e] = x.l;
            r_h[e] = r.h; r_l[e] = r.l;
            z_all[12 * k + c] = z.h;
            z_all[12 * k + 6 + c] = z.l;
            my_rz2.mac(r, z);
        }
        {
            // (the block sum's barrier also makes the new local z visible)
            const fp2 t = block_sum_fp2_warps(my_rz2.get(), s_warp2, (6 * nown + 31) / 32);
            publish(cluster, fp2_to_double(t), s_rz_part, rank, cl);
        }
        // the owned nodes' new z (12 floats each) into the copies of the CTAs
        // that read it (their local vertices or ARAP edges reference the
        // node), three 16-byte stores per node and destination
        for (int t = tid; t < nown * cl; t += kPcgThreads) {
            const int j = t / cl, d = t % cl;
            const int k = perm[j];
            if (d == rank || !((zdst[k] >> d) & 1u)) continue;
            const float4* src = reinterpret_cast<const float4*>(z_all + 12 * k);
            float4* dst = reinterpret_cast<float4*>(s_zdst[d] + 12 * k);
            dst[0] = src[0];
            dst[1] = src[1];
            dst[2] = src[2];
        }
        cluster.sync();
        ++iters;
    }
    // the r^T z of the last iteration (its beta is never needed)
    if (completed && iters > 0 && warp == 0) {
        const double rz_new = cluster_total(s_rz_part, cl);
        if (lane == 0) {
            if (rz_new == 0.0) s_flag[0] = 1;
            const fp2 rn = fp2_from_double(rz_new);
            s_scalar[0] = rn.h; s_scalar[1] = rn.l;
        }
    }
    if (tid == 0 && s_stopz) s_flag[0] = 1;
    __syncthreads();
    // ---------------- results ----------------
    for (int j = tid; j < nown; j += kPcgThreads) {
        const int k = perm[j];
        C.x[2 * k] = make_float4(x_h[6 * j], x_h[6 * j + 1], x_h[6 * j + 2], 0.f);
        C.x[2 * k + 1] = make_float4(x_h[6 * j + 3], x_h[6 * j + 4], x_h[6 * j + 5], 0.f);
    }
    if (tid == 0 && s_flag[2]) atomicOr(&C.sc->status, kDevErrCapacity);
    if (rank == 0 && tid == 0) {
        Scalars* sc = C.sc;
        sc->iters = iters;
        sc->breakdown = s_flag[1];
        sc->stop = s_flag[0];
        sc->rz = (double)s_scalar[0] + (double)s_scalar[1];
    }
    // no CTA may exit while others can still write into its shared memory
    cluster.sync();
}

// ---------------------------------------------------------------------------
// host side: spatial partition
// ---------------------------------------------------------------------------
// Recursive coordinate bisection: a range of nodes is split across the axis
// of its largest extent at its median (node count; ties ordered by node
// index), so every CTA of a cluster owns the same number of nodes (+-1) and
// runs one node per warp in a single round; a range with at least 2^levels
// nodes gives every leaf below it at least one node.
static void rcb(std::vector<int>& idx, int a, int b, int levels, int leaf0, const float4* g,
                std::vector<int>& leaf_off) {
    if (levels == 0) {
        leaf_off[leaf0] = a;
        return;
    }
    const int m = b - a;
    if (m > 1) {
        float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
        for (int j = a; j < b; ++j) {
            const float c[3] = {g[idx[j]].x, g[idx[j]].y, g[idx[j]].z};
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], c[d]);
                hi[d] = std::max(hi[d], c[d]);
            }
        }
        int axis = 0;
        for (int d = 1; d < 3; ++d)
            if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
        auto key = [&](int k) { return axis == 0 ? g[k].x : axis == 1 ? g[k].y : g[k].z; };
        std::sort(idx.begin() + a, idx.begin() + b, [&](int p, int q) {
            const float kp = key(p), kq = key(q);
            return kp < kq || (kp == kq && p < q);
        });
    }
    const int s = a + m / 2;
    const int half = 1 << (levels - 1);
    rcb(idx, a, s, levels - 1, leaf0, g, leaf_off);
    rcb(idx, s, b, levels - 1, leaf0 + half, g, leaf_off);
}

void spatial_partition(int n, int N, int K, const float4* g, const int* ent_off, const int2* ent,
                       const int* edge_off, const int* edge_dst, const int* bind_idx, PcgPartition& out) {
    out.perm.resize(n);
    std::iota(out.perm.begin(), out.perm.end(), 0);
    out.leaf_off.assign(kPcgLeaves + 1, 0);
    int levels = 0;
    while ((1 << levels) < kPcgLeaves) ++levels;
    rcb(out.perm, 0, n, levels, 0, g, out.leaf_off);
    out.leaf_off[kPcgLeaves] = n;
    out.leaf.assign(n, 0);
    for (int f = 0; f < kPcgLeaves; ++f)
        for (int j = out.leaf_off[f]; j < out.leaf_off[f + 1]; ++j) out.leaf[out.perm[j]] = (uint8_t)f;
    // per-CTA maxima for clusters of 1, 2, 4, 8, 16 CTAs
    std::vector<int> mark(N, -1);
    for (int li = 0; li <= 4; ++li) {
        const int cl = 1 << li, lpc = kPcgLeaves / cl;
        const bool tables = cl >= kPcgMinCluster;
        const int ti = cl == 16 ? 1 : 0;
        if (tables) {
            out.loc_off[ti].assign(cl + 1, 0);
            out.loc_vid[ti].clear();
            out.eus_off[ti].assign(cl + 1, 0);
            out.ent_us[ti].clear();
            out.zdst[ti].assign(n, 0);
        }
        int cn = 0, ce = 0, cd = 0, cv = 0;
        std::fill(mark.begin(), mark.end(), -1);
        for (int r = 0; r < cl; ++r) {
            int nn = 0, ne = 0, nd = 0;
            std::vector<int> loc;
            for (int i = 0; i < N; ++i)
                for (int s = 0; s < K; ++s)
                    if ((out.leaf[bind_idx[(size_t)i * K + s]] / lpc) == r && mark[i] != r) {
                        mark[i] = r;
                        loc.push_back(i);   // ascending i
                        if (tables)
                            for (int s2 = 0; s2 < K; ++s2)
                                out.zdst[ti][bind_idx[(size_t)i * K + s2]] |= (unsigned short)(1u << r);
                    }
            for (int j = out.leaf_off[r * lpc]; j < out.leaf_off[(r + 1) * lpc]; ++j) {
                const int k = out.perm[j];
                ++nn;
                ne += ent_off[k + 1] - ent_off[k];
                nd += edge_off[k + 1] - edge_off[k];
                if (!tables) continue;
                out.zdst[ti][k] |= (unsigned short)(1u << r);
                for (int e = edge_off[k]; e < edge_off[k + 1]; ++e) out.zdst[ti][edge_dst[e]] |= (unsigned short)(1u << r);
                for (int e = ent_off[k]; e < ent_off[k + 1]; ++e) {
                    const int i = ent[e].x;
                    const int u = (int)(std::lower_bound(loc.begin(), loc.end(), i) - loc.begin());
                    int self = 0;
                    for (int s = 0; s < K; ++s)
                        if (bind_idx[(size_t)i * K + s] == k) self = s;
                    out.ent_us[ti].push_back((unsigned)u | ((unsigned)self << 16));
                }
            }
            if (tables) {
                out.loc_vid[ti].insert(out.loc_vid[ti].end(), loc.begin(), loc.end());
                out.loc_off[ti][r + 1] = (int)out.loc_vid[ti].size();
                out.eus_off[ti][r + 1] = (int)out.ent_us[ti].size();
            }
            cn = std::max(cn, nn);
            ce = std::max(ce, ne);
            cd = std::max(cd, nd);
            cv = std::max(cv, (int)loc.size());
        }
        out.cap_n[li] = std::max(cn, 1);
        out.cap_e[li] = std::max(ce, 1);
        out.cap_d[li] = std::max(cd, 1);
        out.cap_v[li] = std::max(cv, 1);
    }
}

// ---------------------------------------------------------------------------
// host side: plans and launch
// ---------------------------------------------------------------------------
typedef void (*PcgKernel)(const CapDesc*, int, int, int, int, int);

static PcgKernel pcg_kernel_for(int K) {
    if (K == 4) return pcg_cluster_kernel<4>;
    if (K == 8) return pcg_cluster_kernel<8>;
    return pcg_cluster_kernel<0>;
}

static int max_dynamic_smem() {
    int dev = 0, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return max_optin - 1024;   // the kernel's own __shared__ arrays (< 1 KB)
}

// The device can run the kernel for K with this plan (shared memory opt-in,
// non-portable cluster size, at least one resident cluster).
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

static bool try_plan(int cl, const PcgPartition* const* parts, const int* n, int K, int count, PcgPlan& pl) {
    const int li = log2_cl(cl);
    if ((1 << li) != cl || cl > kPcgLeaves || cl < kPcgMinCluster) return false;
    int cap_v = 1, cap_e = 1, cap_d = 1, cap_n = 1, nmax = 1;
    for (int c = 0; c < count; ++c) {
        // every CTA owns at least one node; node indices fit 16 bits
        if (n[c] < cl || n[c] > 65535 || (int)parts[c]->perm.size() != n[c]) return false;
        for (int r = 0; r < cl; ++r)
            if (parts[c]->leaf_off[(r + 1) * (kPcgLeaves / cl)] <= parts[c]->leaf_off[r * (kPcgLeaves / cl)])
                return false;
        nmax = std::max(nmax, n[c]);
        cap_v = std::max(cap_v, parts[c]->cap_v[li]);
        cap_e = std::max(cap_e, parts[c]->cap_e[li]);
        cap_d = std::max(cap_d, parts[c]->cap_d[li]);
        cap_n = std::max(cap_n, parts[c]->cap_n[li]);
    }
    if (cap_v > 65535) return false;   // local vertex indices fit 16 bits
    const Smem L = smem_layout(nmax, K, cap_v, cap_e, cap_d, cap_n);
    if (L.total > (size_t)max_dynamic_smem()) return false;
    pl = {cl, cap_v, cap_e, cap_d, cap_n, L.total};
    return accept_plan(K, pl);
}

// Choose the cluster size: the largest of {16, 8} whose per-CTA staging fits
// in shared memory and that the device can schedule (an iteration's work is
// split over more SMs; the cluster barrier costs about the same).  Returns
// false if none (the per-iteration kernels are used then).
bool plan_pcg_cluster(const PcgPartition& part, int n, int K, PcgPlan* out) {
    const PcgPartition* pp = &part;
    for (int cl : {16, 8}) {
        PcgPlan pl;
        if (try_plan(cl, &pp, &n, K, 1, pl)) {
            *out = pl;
            return true;
        }
    }
    return false;
}

bool plan_pcg_cluster_group(int cl, const PcgPartition* const* parts, const int* n, int K, int count, PcgPlan* out) {
    PcgPlan pl;
    if (!try_plan(cl, parts, n, K, count, pl)) return false;
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
    return cudaLaunchKernelEx(&cfg, pcg_kernel_for(K), dC, n_pcg, pl.cap_v, pl.cap_e, pl.cap_d, pl.cap_n);
}

}  // namespace lc

// Embedded deformation graph construction on the device.
//
// Farthest-point node sampling, K-nearest-node vertex binding with weights
// (1 - d/d_max)^2 normalised, a symmetrised 4-nearest-node edge graph with
// material-averaged edge weights (the per-edge non-rigidity weights of
// Sec. 3.1, Tab. 1, carried over to graph edges), and the node -> (vertex,
// weight) CSR used by the per-node gathers of the solver.
//
// Index decisions are exact: squared distances are FP64 values computed from
// the FP32 coordinates as (dx*dx + dy*dy) + dz*dz with every operation
// rounded separately, ties broken by the lower index, so any implementation
// following that recipe selects the same nodes and neighbours.
#include <algorithm>

#include <cooperative_groups.h>

#include "lc_internal.cuh"

namespace cg = cooperative_groups;

namespace lc {

__device__ __forceinline__ double d2_exact(float4 a, float4 b) {
    double dx = __dsub_rn((double)a.x, (double)b.x);
    double dy = __dsub_rn((double)a.y, (double)b.y);
    double dz = __dsub_rn((double)a.z, (double)b.z);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// ---------------------------------------------------------------------------
// Farthest-point sampling, cooperative over the whole GPU: each CTA owns a
// contiguous range of vertices and their running minimum distance; per node
// every CTA publishes its farthest vertex (largest distance, lowest index on
// ties), one grid barrier, and every CTA reduces the partials in the same
// way, so all agree on the next node.  GB300's FP64 rate per SM is low, so
// the exact FP64 distance work is spread over every SM.
// ---------------------------------------------------------------------------
constexpr int kFpsThreads = 256;

__device__ __forceinline__ void argmax_merge(double& bd, int& bi, double od, int oi) {
    if (od > bd || (od == bd && oi < bi)) {
        bd = od;
        bi = oi;
    }
}

__device__ __forceinline__ void warp_argmax(double& bd, int& bi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double od = __shfl_xor_sync(0xffffffffu, bd, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        argmax_merge(bd, bi, od, oi);
    }
}

__global__ void __launch_bounds__(kFpsThreads) fps_kernel(const float4* __restrict__ V, int N, int n,
                                                           double* __restrict__ dist, int* __restrict__ node_vid,
                                                           double* __restrict__ pval, int* __restrict__ pidx) {
    __shared__ double sd[kFpsThreads / 32];
    __shared__ int si[kFpsThreads / 32];
    __shared__ int chosen;
    cg::grid_group grid = cg::this_grid();
    const int G = gridDim.x, b = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int lo = (int)((long long)N * b / G), hi = (int)((long long)N * (b + 1) / G);
    float4 q = V[0];
    if (b == 0 && threadIdx.x == 0) node_vid[0] = 0;
    for (int it = 1; it < n; ++it) {
        double bd = -1.0;
        int bi = 0x7fffffff;
        for (int i = lo + threadIdx.x; i < hi; i += kFpsThreads) {
            double d = d2_exact(V[i], q);
            if (it > 1) d = fmin(d, dist[i]);
            dist[i] = d;
            if (d > bd) {  // strictly greater: first (lowest) index within the thread
                bd = d;
                bi = i;
            }
        }
        warp_argmax(bd, bi);
        if (lane == 0) {
            sd[wid] = bd;
            si[wid] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kFpsThreads / 32; ++w) argmax_merge(bd, bi, sd[w], si[w]);
            pval[(it & 1) * G + b] = bd;
            pidx[(it & 1) * G + b] = bi;
        }
        grid.sync();
        if (wid == 0) {
            bd = -1.0;
            bi = 0x7fffffff;
            for (int c = lane; c < G; c += 32) argmax_merge(bd, bi, __ldcg(&pval[(it & 1) * G + c]),
                                                            __ldcg(&pidx[(it & 1) * G + c]));
            warp_argmax(bd, bi);
            if (lane == 0) {
                chosen = bi;
                if (b == 0) node_vid[it] = bi;
            }
        }
        __syncthreads();
        q = V[chosen];
    }
}

// Returns false if the cooperative launch is not possible (the caller then
// reports an error).
bool launch_fps(const float4* V, int N, int n, double* dist, int* node_vid, double* pval, int* pidx, int max_ctas,
                cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fps_kernel, kFpsThreads, 0);
    int G = std::min({sms * std::max(per_sm, 1), (N + kFpsThreads - 1) / kFpsThreads, max_ctas});
    G = std::max(G, 1);
    void* args[] = {(void*)&V, (void*)&N, (void*)&n, (void*)&dist, (void*)&node_vid, (void*)&pval, (void*)&pidx};
    return cudaLaunchCooperativeKernel((const void*)fps_kernel, dim3(G), dim3(kFpsThreads), args, 0, st) == cudaSuccess;
}

// ---------------------------------------------------------------------------
// K nearest nodes per vertex; node positions staged through shared memory.
// ---------------------------------------------------------------------------
template <int KP1>
__device__ __forceinline__ void insert_sorted(double (&d)[KP1], int (&k)[KP1], double nd, int nk) {
    // candidates arrive with increasing index, so strict < keeps lower indices
    // first among equal distances
    if (!(nd < d[KP1 - 1])) return;
    d[KP1 - 1] = nd;
    k[KP1 - 1] = nk;
#pragma unroll
    for (int j = KP1 - 1; j > 0; --j) {
        if (d[j] < d[j - 1]) {
            double td = d[j]; d[j] = d[j - 1]; d[j - 1] = td;
            int tk = k[j]; k[j] = k[j - 1]; k[j - 1] = tk;
        }
    }
}

constexpr int kBindThreads = 256;
constexpr int kBindStage = 1024;

template <int K>
__global__ void __launch_bounds__(kBindThreads) bind_kernel(const float4* __restrict__ V, int N,
                                                             const float4* __restrict__ G, int n,
                                                             int* __restrict__ idx, float* __restrict__ w) {
    __shared__ float4 sg[kBindStage];
    const int i = blockIdx.x * kBindThreads + threadIdx.x;
    float4 v = i < N ? V[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    double d[K + 1];
    int k[K + 1];
#pragma unroll
    for (int j = 0; j <= K; ++j) {
        d[j] = 1.0 / 0.0;
        k[j] = 0x7fffffff;
    }
    for (int base = 0; base < n; base += kBindStage) {
        const int m = min(kBindStage, n - base);
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += kBindThreads) sg[j] = G[base + j];
        __syncthreads();
        for (int j = 0; j < m; ++j) insert_sorted<K + 1>(d, k, d2_exact(v, sg[j]), base + j);
    }
    if (i >= N) return;
    const double dmax = __dsqrt_rn(d[K]);
    double ww[K];
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        double t = dmax > 0.0 ? __dsub_rn(1.0, __ddiv_rn(__dsqrt_rn(d[j]), dmax)) : 0.0;
        ww[j] = dmax > 0.0 ? __dmul_rn(t, t) : 0.0;
        s = __dadd_rn(s, ww[j]);
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        idx[(size_t)i * K + j] = k[j];
        w[(size_t)i * K + j] = s > 0.0 ? __double2float_rn(__ddiv_rn(ww[j], s)) : 1.0f / (float)K;
    }
}

void launch_bind(const float4* V, int N, const float4* G, int n, int K, int* idx, float* w, cudaStream_t st) {
    const int blocks = (N + kBindThreads - 1) / kBindThreads;
    switch (K) {
#define LC_BIND_CASE(KK) \
    case KK: bind_kernel<KK><<<blocks, kBindThreads, 0, st>>>(V, N, G, n, idx, w); break;
        LC_BIND_CASE(1) LC_BIND_CASE(2) LC_BIND_CASE(3) LC_BIND_CASE(4)
        LC_BIND_CASE(5) LC_BIND_CASE(6) LC_BIND_CASE(7) LC_BIND_CASE(8)
#undef LC_BIND_CASE
        default: break;
    }
}

// ---------------------------------------------------------------------------
// Node edges: 4 nearest other nodes, symmetrised, sorted by destination.
// ---------------------------------------------------------------------------
__global__ void node_knn_kernel(const float4* __restrict__ G, int n, int ke, int* __restrict__ knn_e,
                                int* __restrict__ extra_cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double d[kEdgeNN];
    int id[kEdgeNN];
#pragma unroll
    for (int j = 0; j < kEdgeNN; ++j) {
        d[j] = 1.0 / 0.0;
        id[j] = 0x7fffffff;
    }
    const float4 gk = G[k];
    for (int l = 0; l < n; ++l) {
        if (l == k) continue;
        insert_sorted<kEdgeNN>(d, id, d2_exact(gk, G[l]), l);
    }
    for (int j = 0; j < kEdgeNN; ++j) knn_e[k * kEdgeNN + j] = j < ke ? id[j] : -1;
    extra_cnt[k] = 0;
}

__global__ void node_extra_kernel(int n, int ke, const int* __restrict__ knn_e, int* __restrict__ extra_cnt,
                                  int* __restrict__ extra, int* __restrict__ status) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    for (int j = 0; j < ke; ++j) {
        const int k = knn_e[l * kEdgeNN + j];
        bool present = false;
        for (int m = 0; m < ke; ++m) present |= (knn_e[k * kEdgeNN + m] == l);
        if (!present) {
            const int slot = atomicAdd(&extra_cnt[k], 1);
            if (slot < kMaxExtraEdges) extra[k * kMaxExtraEdges + slot] = l;
            else atomicExch(status, 1);
        }
    }
}

__global__ void node_degree_kernel(int n, int ke, const int* __restrict__ extra_cnt, int* __restrict__ deg) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) deg[k] = ke + min(extra_cnt[k], kMaxExtraEdges);
    if (k == n) deg[n] = 0;
}

void launch_node_edges_count(const float4* G, int n, GraphScratch& s, cudaStream_t st) {
    const int ke = n - 1 < kEdgeNN ? n - 1 : kEdgeNN;
    const int t = 128, b = (n + 1 + t - 1) / t;
    node_knn_kernel<<<b, t, 0, st>>>(G, n, ke, s.knn_e, s.extra_cnt);
    node_extra_kernel<<<b, t, 0, st>>>(n, ke, s.knn_e, s.extra_cnt, s.extra, s.status);
    node_degree_kernel<<<b, t, 0, st>>>(n, ke, s.extra_cnt, s.deg);
}

__global__ void node_edges_fill_kernel(int n, int ke, const int* __restrict__ knn_e,
                                       const int* __restrict__ extra_cnt, const int* __restrict__ extra,
                                       const float* __restrict__ material, const int* __restrict__ node_vid,
                                       const int* __restrict__ edge_off, int* __restrict__ edge_dst,
                                       float* __restrict__ edge_s) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int o = edge_off[k];
    int m = 0;
    for (int j = 0; j < ke; ++j) edge_dst[o + m++] = knn_e[k * kEdgeNN + j];
    const int ex = min(extra_cnt[k], kMaxExtraEdges);
    for (int j = 0; j < ex; ++j) edge_dst[o + m++] = extra[k * kMaxExtraEdges + j];
    // insertion sort by destination
    for (int a = 1; a < m; ++a) {
        int v = edge_dst[o + a];
        int b = a - 1;
        while (b >= 0 && edge_dst[o + b] > v) {
            edge_dst[o + b + 1] = edge_dst[o + b];
            --b;
        }
        edge_dst[o + b + 1] = v;
    }
    const float mk = material[node_vid[k]];
    for (int j = 0; j < m; ++j) {
        const float ml = material[node_vid[edge_dst[o + j]]];
        edge_s[o + j] = __fmul_rn(__fadd_rn(mk, ml), 0.5f);
    }
}

void launch_node_edges_fill(const float4* G, int n, const float* material, const int* node_vid,
                            const GraphScratch& s, const int* edge_off, int* edge_dst, float* edge_s,
                            cudaStream_t st) {
    (void)G;
    const int ke = n - 1 < kEdgeNN ? n - 1 : kEdgeNN;
    const int t = 128, b = (n + t - 1) / t;
    node_edges_fill_kernel<<<b, t, 0, st>>>(n, ke, s.knn_e, s.extra_cnt, s.extra, material, node_vid,
                                            edge_off, edge_dst, edge_s);
}

// ---------------------------------------------------------------------------
// Node -> (vertex, weight) CSR, each segment sorted by vertex.
// ---------------------------------------------------------------------------
__global__ void ent_count_kernel(const int* __restrict__ idx, int NK, int* __restrict__ cnt) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < NK) atomicAdd(&cnt[idx[j]], 1);
}

__global__ void ent_fill_kernel(const int* __restrict__ idx, const float* __restrict__ w, int NK, int K,
                                const int* __restrict__ off, int* __restrict__ fill, int2* __restrict__ ent) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NK) return;
    const int k = idx[j];
    const int pos = off[k] + atomicAdd(&fill[k], 1);
    ent[pos] = make_int2(j / K, __float_as_int(w[j]));
}

__global__ void ent_sort_kernel(int n, const int* __restrict__ off, int2* __restrict__ ent) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int a0 = off[k], a1 = off[k + 1];
    for (int a = a0 + 1; a < a1; ++a) {
        int2 v = ent[a];
        int b = a - 1;
        while (b >= a0 && ent[b].x > v.x) {
            ent[b + 1] = ent[b];
            --b;
        }
        ent[b + 1] = v;
    }
}

void launch_entries(const int* idx, const float* w, int N, int K, int n, GraphScratch& s, int* ent_off,
                    int2* ent, cudaStream_t st) {
    const int NK = N * K;
    cudaMemsetAsync(s.ent_cnt, 0, sizeof(int) * (n + 1), st);
    cudaMemsetAsync(s.ent_fill, 0, sizeof(int) * n, st);
    const int t = 256;
    ent_count_kernel<<<(NK + t - 1) / t, t, 0, st>>>(idx, NK, s.ent_cnt);
    launch_exclusive_scan(s.ent_cnt, ent_off, n + 1, st);
    ent_fill_kernel<<<(NK + t - 1) / t, t, 0, st>>>(idx, w, NK, K, ent_off, s.ent_fill, ent);
    ent_sort_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, ent_off, ent);
}

// ---------------------------------------------------------------------------
// Single-block exclusive scan (n up to a few million; used at setup only).
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) scan_kernel(const int* __restrict__ in, int* __restrict__ out, int n) {
    __shared__ int sh[kScanThreads];
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int b = threadIdx.x * per, e = min(n, b + per);
    int s = 0;
    for (int i = b; i < e; ++i) s += in[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        int v = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    int run = threadIdx.x ? sh[threadIdx.x - 1] : 0;
    for (int i = b; i < e; ++i) {
        int v = in[i];
        out[i] = run;
        run += v;
    }
}

void launch_exclusive_scan(const int* in, int* out, int n, cudaStream_t st) {
    scan_kernel<<<1, kScanThreads, 0, st>>>(in, out, n);
}

__global__ void gather_nodes_kernel(const float4* __restrict__ base, const int* __restrict__ vid, int n,
                                    float4* __restrict__ G) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        float4 v = base[vid[k]];
        G[k] = make_float4(v.x, v.y, v.z, 0.f);
    }
}

void launch_gather_nodes(const float4* base, const int* node_vid, int n, float4* G, cudaStream_t st) {
    gather_nodes_kernel<<<(n + 127) / 128, 128, 0, st>>>(base, node_vid, n, G);
}

__global__ void identity_params_kernel(float4* __restrict__ R, float4* __restrict__ t, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    R[3 * k + 0] = make_float4(1.f, 0.f, 0.f, 0.f);
    R[3 * k + 1] = make_float4(0.f, 1.f, 0.f, 0.f);
    R[3 * k + 2] = make_float4(0.f, 0.f, 1.f, 0.f);
    t[k] = make_float4(0.f, 0.f, 0.f, 0.f);
}

void launch_identity_params(float4* R, float4* t, int n, cudaStream_t st) {
    identity_params_kernel<<<(n + 127) / 128, 128, 0, st>>>(R, t, n);
}

}  // namespace lc

// Internal device-side declarations of the livecap library.
//
// One capture (template + graph + frame + solver state) is described by a
// CapDesc that lives in device memory.  Every kernel takes the descriptor
// array and an optional work list of (capture, tile) items, so the same
// kernels serve one capture (work list null: capture 0, tile = blockIdx.x)
// and many captures of uneven size in one launch.
#pragma once

#include <cstdint>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

#include "livecap.h"

namespace lc {

constexpr int kVertTile = 256;      // vertices per vertex tile (one per thread)
constexpr int kNodeWarps = 8;       // warps (= nodes) per node tile
constexpr int kNodeTile = kNodeWarps;
constexpr int kTriTile = 128;       // triangles per raster tile
constexpr int kEdgeTile = 256;      // mesh edges per tile
constexpr int kMaxK = 8;            // nodes per vertex
constexpr int kJChunk = 128;        // vertex ids per compaction chunk of the per-iteration J^T J p
constexpr int kJtjNodeLanes = 8;       // lanes per node in the node phase of the per-iteration J^T J p
constexpr int kJtjNodesPerWarp = 32 / kJtjNodeLanes;
constexpr int kJtjNodeWarps = 4;    // default warps per node-phase block (16 nodes)
static_assert(kVertTile % kJChunk == 0, "vertex tiles hold whole compaction chunks");
constexpr int kEdgeNN = 4;          // node-graph neighbours before symmetrising
constexpr int kMaxExtraEdges = 60;  // symmetrised extra in-edges per node
constexpr int kVecThreads = 256;    // nodes per PCG vector tile

constexpr uint32_t LC_VIS_BIT = LC_FLAG_VISIBLE;
constexpr uint32_t LC_ONSIL_BIT = LC_FLAG_ONSIL;
constexpr uint32_t LC_INB_BIT = LC_FLAG_INB;
constexpr uint32_t LC_BNEG_BIT = LC_FLAG_BNEG;
constexpr uint32_t LC_PRUNED_BIT = LC_FLAG_PRUNED;
constexpr uint32_t LC_MASKED_BIT = LC_FLAG_MASKED;

// Per-capture reduction scalars (FP64; PCG dots and energies).
struct Scalars {
    double rz;         // r^T z of the current iteration
    double rz_new;
    double beta;
    double pAp;
    double e_lin[3];   // photo, sil, arap at the current linearisation
    double step2;      // ||delta||^2 of the last step
    int stop;          // PCG stopped (breakdown or exact convergence)
    int breakdown;     // last PCG stopped on p^T A p <= 0
    int iters;         // PCG iterations run in the current solve
    int status;        // device error word (0 = ok)
    int counts[3];     // visible, contour, contour with b = -1
    int gn_stop;       // the solve reached its target energy: later GN steps are skipped
    int gn_done;       // GN updates made in the current solve (gn_stop, gn_done are reset together)
    int vis_frozen;    // keep the frame decisions (V, B) of the start for the next solve
    float alpha_h, alpha_l;   // graph-stage PCG step length alpha as a compensated FP32 pair
    float beta_h, beta_l;     // graph-stage PCG direction update beta as a pair
    float alpha, beta_f;      // surface-stage PCG step lengths (FP64 sums divided in FP32)
    double e_reg[4];       // surface stage: smooth, edge, velocity, acceleration
};

// Bits of Scalars::status.
constexpr int kDevErrCapacity = 1;   // the cluster PCG's staging exceeded its planned capacity
constexpr int kDevErrWait = 2;       // a bounded wait (TMA staging of the image taps) ran out

// Reduction counters: the last tile of a capture to finish a phase reduces
// the per-tile partials in a fixed order (deterministic, no float atomics).
enum Counter { CNT_ENERGY = 0, CNT_ARAP, CNT_DOT, CNT_DOT2, CNT_STEP, CNT_COUNTS, CNT_N };

struct CapDesc {
    // sizes
    int N, F, n, K, E, W, H, n_medges;
    int vert_tiles, node_tiles, tri_tiles, medge_tiles;
    float f, cx, cy;
    float w_photo, w_sil, w_arap, eps_vis;
    float sigma_c;         // robust colour kernel threshold (0: off)
    float target_energy;   // > 0: stop the GN loop once the energy is <= this
    // template (rest geometry of this stage) and mesh topology
    const float4* base;      // N (x, y, z, 0)
    const float4* albedo;    // N (r, g, b, 0)
    const int4* tris;        // F (a, b, c, 0)
    const int* vt_off;       // N+1 vertex -> triangle CSR (triangle ids ascending)
    const int* vt_tri;
    const int4* medges;      // mesh edges (v0, v1, t0, t1), t1 = -1 on a border
    // graph
    const int* node_vid;     // n
    const int* bind_idx;     // N*K
    const float* bind_w;     // N*K
    const float4* node_g;    // n (g, 0)
    const int* ent_off;      // n+1 node -> (vertex, weight) CSR, vertex ascending
    const int2* ent;         // (vertex, __float_as_int(weight))
    const int* edge_off;     // n+1 node edges by source
    const int* edge_dst;
    const float* edge_s;
    // node parameters
    float4* node_R;          // 3n rows (R_j0, R_j1, R_j2, 0)
    float4* node_t;          // n (t, 0)
    // frame
    const float4* img;       // H*W (r, g, b, dt)
    // photometric pyramid (Sec. 3.4): level j = 0..2 box-averaged by
    // pyr_factor(j) and Gaussian blurred, (r, g, b, 0); pyr_levels = 0: off
    const float4* lvl[3];
    int lvl_W[3], lvl_H[3];
    int pyr_levels;
    // body-part mask of the silhouette term (Sec. 3.4); part_on = 0: off
    const uint8_t* vpart;    // N part of each vertex
    uint8_t* part_raw;       // H*W label of the front triangle of V^S (255: none)
    uint8_t* part_mask;      // H*W dilated labels
    int part_on, torso_part, part_dilate;
    const uint8_t* mask;     // H*W
    // per-frame decisions
    unsigned long long* zbuf;  // H*W
    uint32_t* flags;         // N
    // linearisation
    float4* vw;              // N warped (x, y, z, valid)
    float2* uv;              // N
    float4* res;             // N (r_photo xyz, r_sil)
    float4* HA;              // N (h00, h01, h02, h11)
    float4* HB;              // N (h12, h22, 0, 0)
    float4* ev;              // N (e0, e1, e2, active)
    // PCG state: node vectors as two float4 per node (omega, t)
    float4* b;               // -J^T F
    float4* minv;            // Jacobi inverse diagonal
    float4* diag;            // diag(J^T J)
    float4* x;
    float4* r;
    float4* z;
    float4* p;
    float4* Ap;
    // low parts of the compensated FP32 pairs of the per-iteration PCG
    // (fpair.cuh): the vector is hi + lo
    float4* x_lo;
    float4* r_lo;
    float4* z_lo;
    float4* p_lo;
    float4* Ap_lo;
    float4* q;               // 2N: per active vertex H_i dv_i scratch by compact position, (high, low) parts
    // spatial node partition of the cluster PCG (kPcgLeaves leaves; a
    // cluster of cl CTAs gives CTA r the leaves r*L/cl .. (r+1)*L/cl - 1)
    const int* pcg_perm;      // n nodes in leaf order
    const int* pcg_leaf_off;  // kPcgLeaves + 1 offsets into pcg_perm
    const uint8_t* pcg_leaf;  // n leaf of every node
    // per cluster size (index 0: 8 CTAs, 1: 16 CTAs), fixed per graph:
    // CTA r's local vertices (bound to an owned node, ascending id) are
    // pcg_loc_vid[pcg_loc_off[r] ..), and the CSR entries of its owned nodes
    // (owned nodes in pcg_perm order, each node's entries in CSR order) are
    // pcg_ent_us[pcg_eus_off[r] ..) as (local vertex | slot << 16)
    const int* pcg_loc_off[2];
    const int* pcg_loc_vid[2];
    const int* pcg_eus_off[2];
    const unsigned* pcg_ent_us[2];
    // per node: bit r set if CTA r reads the node's z (it owns the node, a
    // local vertex of it binds to the node, or an owned edge ends there)
    const unsigned short* pcg_zdst[2];
    // operands of the per-iteration J^T J p, staged once per linearisation
    // with the inactive vertices left out: the active vertices of each chunk
    // of kJChunk ids are packed, in id order, at the chunk's start (their
    // compact positions), and the active entries of each node at the start
    // of its CSR range
    float4* vA;              // N*K: (w_is R_k (v_i - g_k), w_is) of compact position pos, slot s, at pos*K + s
    int* vK;                 // N*K: the node of that binding
    float4* vH;              // 2N: (h00, h01, h02, h11), (h12, h22, 0, 0) of compact position pos
    int* vpos;               // N: compact position of vertex i, -1 when inactive
    int* vcnt;               // ceil(N / kJChunk): active vertices per chunk
    int* eV;                 // N*K: per active entry of a node, vertex ascending: (compact position << 3) | slot
    int* ecnt;               // n: active entries per node
    const int* jn_perm;      // n: node of each node-phase slot (Morton order of the node positions)
    float4* dB;              // 2 per directed node edge: (R_k (g_l - g_k), w_a s_kl), (R_l (g_k - g_l), 0)
    // per-vertex surface stage (unknowns V)
    int n_adj;               // directed one-ring pairs
    float w_smooth, w_edge;
    float w_vel, w_acc;      // 0 without temporal history
    const int* adj_off;      // N+1 one-ring CSR, neighbours ascending
    const int* adj_dst;      // n_adj
    const float4* adj_geo;   // n_adj: (s_ij/|N_i|, s_ij (1/|N_i| + 1/|N_j|), |Vh_i - Vh_j|, 0)
    float4* adj_m;           // n_adj, per linearisation: (sqrt(w_edge c_ij) n_ij, w_smooth c_ij)
    float4* sV;              // N current surface (x, y, z, 0)
    float4* sH1;             // N V^{t-1}
    float4* sH2;             // N V^{t-2}
    float4* sD;              // N rest-pose displacement of the last advanced frame
    float4* sb;              // N -J^T F
    float4* sminv;           // N Jacobi inverse diagonal
    float4* sx;
    float4* sr;
    float4* sz;
    float4* sp[2];           // search directions of even / odd PCG iterations
    float4* sAp;
    // reductions
    double* part;            // per-tile partials of the running reduction
    unsigned* counters;      // CNT_N
    Scalars* sc;
    double* hist;            // 2 * (LC_MAX_GN + 1): [2 gn] energy, [2 gn + 1] step norm
    int* hist_iters;         // LC_MAX_GN + 2: PCG iterations per step, [LC_MAX_GN + 1] breakdowns
    // TMA staging of the image taps (lc_params.tma_taps) in single-capture
    // launches: img as a 2D tensor of 4W x H floats, passed to the kernel by
    // value (valid when tma_ok)
    int tma_taps;
    int tma_ok;
    CUtensorMap tmap_img;
};

struct WorkItem {
    int cap;
    int tile;
};

__device__ __forceinline__ void decode(const WorkItem* items, int& cap, int& tile) {
    if (items) {
        WorkItem w = items[blockIdx.x];
        cap = w.cap;
        tile = w.tile;
    } else {
        cap = 0;
        tile = blockIdx.x;
    }
}

// ---- exact FP32 helpers (each operation rounded once, no contraction) -----
__device__ __forceinline__ float xadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float xsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float xmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float xdiv(float a, float b) { return __fdiv_rn(a, b); }

// Projection with the specified operation order: u = (f*X)/Z + cx.
__device__ __forceinline__ float2 project_exact(float f, float cx, float cy, float X, float Y, float Z) {
    return make_float2(xadd(xdiv(xmul(f, X), Z), cx), xadd(xdiv(xmul(f, Y), Z), cy));
}

__device__ __forceinline__ bool valid_depth(float Z) { return Z > 1e-3f; }

__device__ __forceinline__ bool in_image(float2 uv, int W, int H) {
    return uv.x >= 0.0f && uv.x <= (float)(W - 1) && uv.y >= 0.0f && uv.y <= (float)(H - 1);
}

// ---- exact direction rule b_i (shared by the contour pass, the non-rigid
// linearisation and the pose stage) ------------------------------------------
__device__ __forceinline__ float xlerp(float a, float b, float t) { return xadd(a, xmul(t, xsub(b, a))); }

__device__ __forceinline__ float dt_px(const float4* img, int W, int x, int y) { return img[(size_t)y * W + x].w; }

__device__ __forceinline__ float dt_grad_x_exact(const float4* img, int W, int x, int y) {
    if (W < 2) return 0.f;
    if (x == 0) return xsub(dt_px(img, W, 1, y), dt_px(img, W, 0, y));
    if (x == W - 1) return xsub(dt_px(img, W, W - 1, y), dt_px(img, W, W - 2, y));
    return xmul(xsub(dt_px(img, W, x + 1, y), dt_px(img, W, x - 1, y)), 0.5f);
}

__device__ __forceinline__ float dt_grad_y_exact(const float4* img, int W, int H, int x, int y) {
    if (H < 2) return 0.f;
    if (y == 0) return xsub(dt_px(img, W, x, 1), dt_px(img, W, x, 0));
    if (y == H - 1) return xsub(dt_px(img, W, x, H - 1), dt_px(img, W, x, H - 2));
    return xmul(xsub(dt_px(img, W, x, y + 1), dt_px(img, W, x, y - 1)), 0.5f);
}

// b_i = -1 iff the model point projects inside the image silhouette (mask at
// rint(uv)) and its projected area-weighted normal m opposes z = -grad DT,
// i.e. m . grad DT > 0 (Sec. 3.3).  Normal: incident triangles in ascending id
// order, every FP32 operation rounded once.  The vertex must be valid and its
// projection inside the image.
__device__ __forceinline__ bool direction_neg(const CapDesc& C, int i) {
    float nx = 0.f, ny = 0.f, nz = 0.f;
    for (int j = C.vt_off[i]; j < C.vt_off[i + 1]; ++j) {
        const int4 tri = C.tris[C.vt_tri[j]];
        const float4 A = C.vw[tri.x], B = C.vw[tri.y], Q = C.vw[tri.z];
        const float e1x = xsub(B.x, A.x), e1y = xsub(B.y, A.y), e1z = xsub(B.z, A.z);
        const float e2x = xsub(Q.x, A.x), e2y = xsub(Q.y, A.y), e2z = xsub(Q.z, A.z);
        nx = xadd(nx, xsub(xmul(e1y, e2z), xmul(e1z, e2y)));
        ny = xadd(ny, xsub(xmul(e1z, e2x), xmul(e1x, e2z)));
        nz = xadd(nz, xsub(xmul(e1x, e2y), xmul(e1y, e2x)));
    }
    const float4 v = C.vw[i];
    const float mx = xsub(nx, xmul(xdiv(v.x, v.z), nz));
    const float my = xsub(ny, xmul(xdiv(v.y, v.z), nz));
    const float2 uv = C.uv[i];
    const int x0 = (int)floorf(uv.x), y0 = (int)floorf(uv.y);
    const float fx = xsub(uv.x, (float)x0), fy = xsub(uv.y, (float)y0);
    const int x1 = x0 + 1 < C.W ? x0 + 1 : C.W - 1;
    const int y1 = y0 + 1 < C.H ? y0 + 1 : C.H - 1;
    const float gx = xlerp(xlerp(dt_grad_x_exact(C.img, C.W, x0, y0), dt_grad_x_exact(C.img, C.W, x1, y0), fx),
                           xlerp(dt_grad_x_exact(C.img, C.W, x0, y1), dt_grad_x_exact(C.img, C.W, x1, y1), fx), fy);
    const float gy = xlerp(xlerp(dt_grad_y_exact(C.img, C.W, C.H, x0, y0), dt_grad_y_exact(C.img, C.W, C.H, x1, y0), fx),
                           xlerp(dt_grad_y_exact(C.img, C.W, C.H, x0, y1), dt_grad_y_exact(C.img, C.W, C.H, x1, y1), fx),
                           fy);
    const float d = xadd(xmul(mx, gx), xmul(my, gy));
    const long long px = __float2ll_rn(uv.x), py = __float2ll_rn(uv.y);
    const bool inside = C.mask[py * C.W + px] != 0;
    return inside && d > 0.f;
}

// ---- FP64 block reduction helpers -----------------------------------------
template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
}

template <int NV>
__device__ __forceinline__ void warp_sumf(float (&v)[NV]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
}

// Block-wide sum of NV doubles in a fixed order; result valid in thread 0.
template <int NV, int NWARPS>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sh)[NV]) {
    warp_sum<NV>(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) sh[w][j] = v[j];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double s = 0.0;
            for (int i = 0; i < NWARPS; ++i) s += sh[i][j];
            v[j] = s;
        }
    }
}

// Block-wide sum of NV per-thread FP32 values: FP32 inside the block (fixed
// shuffle tree, then the warps' sums in warp order by thread 0), returned in
// FP64 in thread 0 for the FP64 sum across tiles.  Per-thread FP64 work is
// avoided: GB300 runs FP64 at ~1.7 lane-operations per clock per SM.
template <int NV, int NWARPS>
__device__ __forceinline__ void block_sum_f(float (&v)[NV], double (&out)[NV], float (*sh)[NV]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) sh[w][j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) out[j] = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            float s = 0.f;
            for (int i = 0; i < NWARPS; ++i) s += sh[i][j];
            out[j] = (double)s;
        }
    }
}

// Write this tile's partials; returns true (in every thread) in the block
// that finished last for this capture and counter.
// m consecutive tiles' partials (tile0 .. tile0 + m - 1) from one block;
// returns true (in every thread) in the block that finished last.
template <int NV>
__device__ __forceinline__ bool publish_partials(const CapDesc& C, int counter, int tile0, int m, int ntiles,
                                                 const double (*v)[NV], double* part_base) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        for (int g = 0; g < m; ++g)
#pragma unroll
            for (int j = 0; j < NV; ++j) part_base[(tile0 + g) * NV + j] = v[g][j];
        __threadfence();
        unsigned done = atomicAdd(&C.counters[counter], (unsigned)m);
        last = (done + (unsigned)m == (unsigned)ntiles);
        if (last) {
            __threadfence();
            C.counters[counter] = 0u;   // re-arm for the next launch
        }
    }
    __syncthreads();
    return last;
}

template <int NV>
__device__ __forceinline__ bool publish_partial(const CapDesc& C, int counter, int tile, int ntiles,
                                                const double (&v)[NV], double* part_base) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) part_base[tile * NV + j] = v[j];
        __threadfence();
        unsigned done = atomicAdd(&C.counters[counter], 1u);
        last = (done == (unsigned)ntiles - 1u);
        if (last) {
            __threadfence();
            C.counters[counter] = 0u;   // re-arm for the next launch
        }
    }
    __syncthreads();
    return last;
}

// Sum of the ntiles partials by one warp, in a fixed order (lane l adds
// tiles l, l + 32, ...; then a fixed shuffle tree); every lane gets the
// total.  FP64 has a long latency on GB300, so the chain is kept short.
template <int NV>
__device__ __forceinline__ void sum_partials_warp(const double* part_base, int ntiles, double (&out)[NV]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < NV; ++j) out[j] = 0.0;
    for (int t = lane; t < ntiles; t += 32)
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] += __ldcg(&part_base[t * NV + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < NV; ++j) out[j] += __shfl_xor_sync(0xffffffffu, out[j], o);
}

// publish_partial + in the last block: warp 0 sums all tiles, thread 0 runs
// fin(total) (the capture's scalar update, exactly once).
template <int NV, typename Fin>
__device__ __forceinline__ void reduce_partials(const CapDesc& C, int counter, int tile, int ntiles,
                                                const double (&v)[NV], Fin&& fin) {
    if (!publish_partial<NV>(C, counter, tile, ntiles, v, C.part)) return;
    if (threadIdx.x >= 32) return;
    double tot[NV];
    sum_partials_warp<NV>(C.part, ntiles, tot);
    if (threadIdx.x == 0) fin(tot);
}

// ---- launch shapes --------------------------------------------------------
// Blocks of each tile family and their (capture, tile) work lists.  A null
// list means one capture (capture 0, tile = blockIdx.x); a batch of
// captures passes concatenated lists, so the same kernels serve both.
struct Tiles {
    int vert = 0, tri = 0, medge = 0, node = 0, vec = 0;
    const WorkItem* vert_items = nullptr;
    const WorkItem* tri_items = nullptr;
    const WorkItem* medge_items = nullptr;
    const WorkItem* node_items = nullptr;
    const WorkItem* vec_items = nullptr;
    // launch shape of the per-iteration J^T J p (launch_jtj): vertices per
    // vertex-phase block, warps per node-phase block (kJtjNodesPerWarp nodes
    // each) and the node phase's entry rounds in flight, with their own work
    // lists (jv / jn blocks); every shape gives bit-identical results
    int jv = 0, jn = 0;
    const WorkItem* jv_items = nullptr;
    const WorkItem* jn_items = nullptr;
    int jv_block = kVertTile, jn_warps = kJtjNodeWarps, jn_unroll = 4;
    int jk = 0;   // the captures' common K (0: mixed), selects an unrolled vertex phase
    // linearisation with TMA-staged image taps (single-capture launches only:
    // the tensor map is a kernel parameter)
    bool tma = false;
};

inline Tiles single_tiles(const CapDesc& C) {
    Tiles t;
    t.vert = C.vert_tiles;
    t.tri = C.tri_tiles;
    t.medge = C.medge_tiles;
    t.node = C.node_tiles;
    t.vec = (C.n + kVecThreads - 1) / kVecThreads;
    t.jv = C.vert_tiles;
    t.jn = (C.n + kJtjNodeWarps * kJtjNodesPerWarp - 1) / (kJtjNodeWarps * kJtjNodesPerWarp);
    t.jk = C.K;
    t.tma = C.tma_taps && C.tma_ok;
    return t;
}

// ---- kernel launchers (frame_kernels.cu, solver_kernels.cu, graph_kernels.cu)
void launch_pack_frame(const float* rgb, const float* dt, const uint8_t* mask_in, float4* img,
                       uint8_t* mask, int W, int H, cudaStream_t st);
// exact silhouette distance transform of the packed mask into img's 4th
// channel (g: W x H int scratch; W <= 16384, g of a row in shared memory)
// distance transform of the silhouette into img's fourth channel; contour
// (W x H bytes) and g (W x H ints) are scratch
void launch_edt(const uint8_t* mask, uint8_t* contour, int* g, float4* img, int W, int H, cudaStream_t st);
// the body-part mask of the frame (projection and raster of V^S, labels,
// dilation); nothing when the capture's mask is off or its decisions frozen
void launch_part_mask(const CapDesc* dC, const CapDesc& hC, cudaStream_t st);
// vertex part = bone_part of the heaviest of the 4 skinning slots
void launch_vertex_parts(const int4* skin_idx, const float4* skin_w, const int* bone_part, int N, uint8_t* vpart,
                         cudaStream_t st);
// level j of the photometric pyramid from the packed frame (rgb of img):
// box mean over d x d blocks (into out when d > 1), then the separable
// Gaussian `taps` (2r+1 of them), rows into tmp, columns into out (Wd x Hd)
constexpr int kPyrMaxTaps = 31;
__host__ __device__ constexpr int pyr_factor(int j) { return 4 >> j; }   // 4, 2, 1
struct PyrTaps {
    float w[kPyrMaxTaps];
    int r;
};
void launch_pyramid_level(const float4* img, int W, int H, int d, const PyrTaps& taps, float4* tmp, float4* out,
                          int Wd, int Hd, cudaStream_t st);
void launch_warp(const CapDesc* dC, const CapDesc& hC, cudaStream_t st, bool gated = false);
// gated: skipped for captures whose GN loop has stopped (steps after the first)
void launch_warp(const CapDesc* dC, const Tiles& T, cudaStream_t st, bool gated = false);
void launch_visibility(const CapDesc* dC, const CapDesc& hC, cudaStream_t st);
void launch_visibility_kernels(const CapDesc* dC, const Tiles& T, cudaStream_t st);
// the next visibility pass runs again (clears vis_frozen)
void launch_vis_unfreeze(const CapDesc* dC, cudaStream_t st);
// gn: the Gauss-Newton step being linearised (selects the pyramid level;
// LC_MAX_GN for the energy after the last update)
void launch_linearize(const CapDesc* dC, const CapDesc& hC, bool update_b, int gn, cudaStream_t st);
void launch_linearize(const CapDesc* dC, const Tiles& T, bool update_b, int gn, cudaStream_t st);
void launch_rhs(const CapDesc* dC, const CapDesc& hC, int slot, bool energy_only, cudaStream_t st);
void launch_rhs(const CapDesc* dC, const Tiles& T, int slot, bool energy_only, cudaStream_t st);
// rotated offsets of bindings, entries and edges for the per-iteration J^T J p
// (once per linearisation; node parameters and activity must be current)
void launch_jtj_stage(const CapDesc* dC, const CapDesc& hC, cudaStream_t st);
void launch_jtj_stage(const CapDesc* dC, const Tiles& T, cudaStream_t st);
// J^T J p in compensated pairs: p (+ p_lo, nullable) -> out (+ out_lo,
// nullable: the low part is dropped); p / out null: each capture's own p and Ap
void launch_jtj(const CapDesc* dC, const CapDesc& hC, const float4* p, const float4* p_lo, float4* out,
                float4* out_lo, bool dot, cudaStream_t st);
// T.jk: the captures' common K selects an unrolled vertex phase (0: any K)
void launch_jtj(const CapDesc* dC, const Tiles& T, const float4* p, const float4* p_lo, float4* out,
                float4* out_lo, bool dot, cudaStream_t st);
// the launch shapes launch_jtj has kernels for
bool jtj_shape_valid(int vert_block, int node_warps, int node_unroll);
// dynamic shared memory of the TMA-staged linearisation (once per process)
cudaError_t linearize_tma_init();
void launch_pcg_init(const CapDesc* dC, const CapDesc& hC, cudaStream_t st);
void launch_pcg_init(const CapDesc* dC, const Tiles& T, cudaStream_t st);
void launch_pcg_vectors(const CapDesc* dC, const CapDesc& hC, cudaStream_t st);
void launch_pcg_vectors(const CapDesc* dC, const Tiles& T, cudaStream_t st);
void launch_update(const CapDesc* dC, const CapDesc& hC, int gn_slot, cudaStream_t st);
// one thread sets the condition of the next step's conditional graph node to
// "the solve goes on" (capture 0 of dC has not reached its target)
void launch_gn_gate(const CapDesc* dC, cudaGraphConditionalHandle next, cudaStream_t st);
void launch_update(const CapDesc* dC, const Tiles& T, int gn_slot, cudaStream_t st);
void launch_pack_vec(const float* in6, float4* out, int n, cudaStream_t st);
void launch_unpack_vec(const float4* in, float* out6, int n, cudaStream_t st);

// per-vertex surface stage (surface.cu)
void launch_surface_project(const CapDesc* dC, const CapDesc& hC, cudaStream_t st);
// diag_out (nullable): diag(J^T J) per vertex; energy_only: energies only
void launch_surface_rhs(const CapDesc* dC, const CapDesc& hC, int slot, bool energy_only, float4* diag_out,
                        cudaStream_t st);
// it: PCG iteration (-1: plain product of p into out with no dot)
void launch_surface_jtj(const CapDesc* dC, const CapDesc& hC, int it, const float4* p, float4* out, cudaStream_t st);
void launch_surface_pcg_init(const CapDesc* dC, const CapDesc& hC, cudaStream_t st);
void launch_surface_pcg_step(const CapDesc* dC, const CapDesc& hC, int it, cudaStream_t st);
void launch_surface_update(const CapDesc* dC, const CapDesc& hC, int slot, cudaStream_t st);
// all PCG iterations of one step in one cluster launch: cl CTAs of tpc
// vertex tiles each (cl = 0: the capture is too large, per-iteration kernels)
struct SurfCluster {
    int cl, tpc;
};
SurfCluster plan_surface_cluster(int vert_tiles);
cudaError_t launch_surface_pcg_cluster(const CapDesc* dC, SurfCluster shape, int n_pcg, cudaStream_t st);

// cluster-persistent PCG (pcg_cluster.cu)
constexpr int kPcgLeaves = 16;
// Spatial partition of a capture's nodes into kPcgLeaves leaves (recursive
// coordinate bisection of the node positions, balanced by CSR entries and
// edges), and the per-CTA capacities it implies for clusters of 1, 2, 4, 8
// and 16 CTAs (index log2 cl).
struct PcgPartition {
    std::vector<int> perm;
    std::vector<int> leaf_off;
    std::vector<uint8_t> leaf;
    // all nodes in Morton (Z) order of their positions, ties by id: the node
    // order of the per-iteration J^T J p's node phase
    std::vector<int> zorder;
    // clusters of 8 and 16 CTAs (index 0, 1): local vertex lists and entry
    // tables (CapDesc::pcg_loc_* / pcg_ent_us)
    std::vector<int> loc_off[2], loc_vid[2], eus_off[2];
    std::vector<unsigned> ent_us[2];
    std::vector<unsigned short> zdst[2];
    int cap_n[5] = {0, 0, 0, 0, 0};   // owned nodes
    int cap_e[5] = {0, 0, 0, 0, 0};   // CSR entries of the owned nodes
    int cap_d[5] = {0, 0, 0, 0, 0};   // directed edges of the owned nodes
    int cap_v[5] = {0, 0, 0, 0, 0};   // distinct vertices bound to an owned node
};
constexpr int kPcgMinCluster = 8;   // the cluster PCG runs 8 or 16 CTAs per capture
void spatial_partition(int n, int N, int K, const float4* g, const int* ent_off, const int2* ent,
                       const int* edge_off, const int* edge_dst, const int* bind_idx, PcgPartition& out);
struct PcgPlan {
    int cl;          // CTAs per cluster
    int cap_v;       // local-vertex capacity per CTA
    int cap_e;       // CSR-entry capacity per CTA
    int cap_d;       // node-edge capacity per CTA
    int cap_n;       // owned-node capacity per CTA
    size_t smem;     // dynamic shared memory bytes
};
bool plan_pcg_cluster(const PcgPartition& part, int n, int K, PcgPlan* out);
// one cluster per capture: captures 0 .. ncap-1 of dC, all fitting the plan
cudaError_t launch_pcg_cluster(const CapDesc* dC, const PcgPlan& pl, int K, int n_pcg, cudaStream_t st, int ncap = 1);
// a plan of cl CTAs that fits every capture of a group (same K): per-CTA
// capacities are the maxima over the captures, shared memory sized for the
// largest n
bool plan_pcg_cluster_group(int cl, const PcgPartition* const* parts, const int* n, int K, int count, PcgPlan* out);

// graph construction
struct GraphScratch {
    double* dist;       // N
    int* knn_e;         // n * kEdgeNN
    int* extra_cnt;     // n
    int* extra;         // n * kMaxExtraEdges
    int* deg;           // n
    int* ent_cnt;       // n
    int* ent_fill;      // n
    int* status;        // 1
};
// farthest-point sampling as one cooperative launch over the GPU (at most
// max_ctas CTAs; pval / pidx hold 2 * max_ctas partials); false if the launch failed
bool launch_fps(const float4* V, int N, int n, double* dist, int* node_vid, double* pval, int* pidx, int max_ctas,
                cudaStream_t st);
void launch_bind(const float4* V, int N, const float4* G, int n, int K, int* idx, float* w, cudaStream_t st);
void launch_node_edges_count(const float4* G, int n, GraphScratch& s, cudaStream_t st);
void launch_node_edges_fill(const float4* G, int n, const float* material, const int* node_vid,
                            const GraphScratch& s, const int* edge_off, int* edge_dst, float* edge_s,
                            cudaStream_t st);
void launch_entries(const int* idx, const float* w, int N, int K, int n, GraphScratch& s,
                    int* ent_off, int2* ent, cudaStream_t st);
void launch_exclusive_scan(const int* in, int* out, int n, cudaStream_t st);
void launch_gather_nodes(const float4* base, const int* node_vid, int n, float4* G, cudaStream_t st);
void launch_identity_params(float4* R, float4* t, int n, cudaStream_t st);

}  // namespace lc

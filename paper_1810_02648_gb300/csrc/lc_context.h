// Host-side context of the livecap library (one capture).
#pragma once

#include <cmath>
#include <string>
#include <vector>

#include "lc_internal.cuh"

struct PoseState;
struct WarmState;
namespace lc {
struct PoseDesc;
}

struct lc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;      // created by lc_create (caller passed 0)
    std::string err;
    lc_params params{};
    lc::CapDesc hC{};             // host copy of the descriptor
    lc::CapDesc* dC = nullptr;    // device copy
    std::vector<void*> owned;     // every device allocation of this context
    cudaGraphExec_t gexec = nullptr;
    int graph_kernels = 0;        // kernel nodes in the captured non-rigid solve (outside conditional bodies)
    int graph_kernels_step = 0;   // kernel nodes of one conditional Gauss-Newton step (0: unrolled)
    // conditional Gauss-Newton steps (captured solves with a target energy)
    cudaStream_t side_stream = nullptr;    // captures the bodies of conditional nodes
    cudaStream_t saved_stream = nullptr;
    std::vector<cudaGraph_t> cond_bodies;  // bodies of the capture in progress
    bool cond_failed = false;
    void begin_if(cudaGraphConditionalHandle h);
    void end_if();
    bool has_camera = false, has_template = false, has_graph = false, has_frame = false;
    bool has_vis = false, has_lin = false;
    // template
    float4* tpl = nullptr;        // rest template V^hat
    float4* base_buf = nullptr;   // rest geometry of the non-rigid stage (template or skinned mesh)
    float* material = nullptr;
    // frame staging for host inputs
    float* stage_rgb = nullptr;
    float* stage_dt = nullptr;
    uint8_t* stage_mask = nullptr;
    int* edt_g = nullptr;         // distance-transform scratch (first use of a null dt): W x H ints + W x H bytes
    float4* pyr_buf[3] = {nullptr, nullptr, nullptr};   // photometric pyramid levels
    float4* pyr_tmp = nullptr;    // row-blur scratch of the pyramid (W x H)
    lc_status build_pyramid();    // the levels of params.pyr_levels from the current frame
    void pyr_release();
    // body-part mask of the silhouette term (lc_set_body_parts)
    uint8_t* vpart_buf = nullptr;      // N
    uint8_t* part_raw_buf = nullptr;   // W x H
    uint8_t* part_mask_buf = nullptr;  // W x H
    int* bone_part_buf = nullptr;      // J
    lc_status part_images();           // (re)allocate the W x H label images of an active mask
    // scratch node vectors
    float4* tmp_vec = nullptr;
    float4* tmp_vec2 = nullptr;
    float* tmp6 = nullptr;
    int tmp6_cap = 0;
    int part_cap = 0;
    lc::PcgPlan pcg_plan{};
    lc::PcgPartition pcg_part;    // spatial node partition (host copy)
    bool pcg_plan_ok = false;     // the cluster-persistent PCG fits this capture
    bool use_cluster_pcg() const { return pcg_plan_ok && params.pcg_kernel == 0; }
    lc_status plan_pcg();         // partition + plan for the current graph
    void release_pcg_tables();
    void enqueue_pcg();
    PoseState* pose = nullptr;
    WarmState* warm = nullptr;    // learned warm start (warmstart.cu)
    void warm_release();
    // profiling: an event chain recorded between phases of the captured solve
    bool profiling = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_phase;   // phase of the segment starting at event j
    int prof_used = 0;             // events handed out since profiling was switched on
    struct ProfRange {
        int begin = 0, end = 0;    // the events one captured graph records
    } prof_nonrigid, prof_pose, prof_surface;
    double prof_ms[LC_N_PHASES] = {0};
    int prof_cnt[LC_N_PHASES] = {0};
    void mark(int phase);          // record the next event of the chain (capture time)
    void mark_end();
    lc_status accumulate_profile(const ProfRange& r);

    lc_status fail(lc_status st, const char* fmt, ...);
    // device allocations that failed since creation: a setup sequence
    // compares it with its value at the start
    int alloc_failures = 0;
    lc_status cuda(cudaError_t e, const char* what);
    void* alloc(size_t bytes);
    void release(void* p);
    static bool is_device_ptr(const void* p);
    lc_status copy_to_host(void* dst, const void* src_dev, size_t bytes);
    lc_status fetch(void* dst_host, const void* src_any, size_t bytes);
    lc_status deliver(void* dst_any, const void* src_host, size_t bytes);
    lc_status sync_desc();
    void drop_graph();
    void apply_params();
    void ensure_partials();
    void free_graph();
    void free_template();
    void enqueue_nonrigid();
    lc_status check_solve_state(const char* who);
    lc_status read_stats(lc_solve_stats* stats, int n_gn, bool surface = false);
    lc_status capture(cudaGraphExec_t* exec, int* n_kernels, void (lc_ctx::*enqueue)(), int* n_kernels_step = nullptr);
    lc_status linearize_now(bool with_rhs);
    lc_status vec_out(float* dst, const float4* src);
    float* tmp_out();
    // per-vertex surface stage (surface.cu)
    cudaGraphExec_t surf_gexec = nullptr;
    int surf_graph_kernels = 0;
    int surf_hist = 0;             // temporal history frames held (0, 1, 2)
    bool surf_has_disp = false;    // a rest-pose displacement was recorded
    bool surf_has_lin = false;     // the surface operands match the current V
    bool last_surface = false;     // the last solve was the surface stage (lc_read_stats)
    float4* surf_diag = nullptr;   // N: diag(J^T J) for lc_surface_linearize
    int surf_cl = 0;               // cluster size of the surface cluster PCG (0: per-iteration kernels)
    lc::SurfCluster surf_shape{0, 0};
    lc_status surface_setup(const float* V, const float* material, const std::vector<int4>& medges);
    void surface_release();
    void surface_weights();
    void enqueue_surface();
    lc_status check_surface_state(const char* who);
    // pose stage (pose_api.cu)
    const lc::PoseDesc* pose_desc() const;   // device descriptor, null without a skeleton
    void enqueue_pose();
    void pose_release();
    void pose_drop_graph();
    void pose_graph_changed();   // a new graph: no recorded rest-pose node parameters
    lc_status pose_frame(const float* joints2d, const float* joints3d);
    lc_status pose_read(float* pose_out);
};

// Pieces of a frame step that lc_batch_step captures into one graph
// (pose_api.cu, warmstart.cu): *_prepare run on the host before the capture
// (descriptor uploads, allocations); the others enqueue on ctx->stream.
lc_status pose_step_prepare(lc_ctx* ctx);
void pose_step_begin(lc_ctx* ctx, bool euler_start);
void pose_step_end(lc_ctx* ctx);
lc_status warm_step_prepare(lc_ctx* ctx, lc_mlp* m);   // m may be null: motion bookkeeping only
void warm_step_enqueue(lc_ctx* ctx, lc_mlp* m);
void motion_step_enqueue(lc_ctx* ctx);
void mlp_identity(const lc_mlp* m, unsigned long long* uid, unsigned long long* gen);
void mlp_before(lc_mlp* m, cudaStream_t st);   // st waits for the network's earlier work
void mlp_after(lc_mlp* m, cudaStream_t st);    // the network's later work waits for st

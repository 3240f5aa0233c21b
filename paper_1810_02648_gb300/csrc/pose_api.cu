// Skeletal pose stage (Sec. 3.3): entry points, state and the captured solve.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lc_context.h"
#include "pose_internal.h"

using namespace lc;

struct PoseState {
    PoseDesc h{};                   // host copy of the descriptor
    PoseDesc* d = nullptr;          // device copy
    int N = 0;
    cudaGraphExec_t gexec = nullptr;
    int graph_kernels = 0;
    int graph_n_gn = 0;
    bool has_pose = false;
    float* pose_set = nullptr;      // kMaxDof + 9: the pose last given to lc_set_pose, then its root rotation
    PoseDesc last{};                // the descriptor as last copied to the device
    bool synced = false;
    int graph_disp = 0;             // use_disp when the graph was captured
    // the graph stage's displacement warping: node parameters in the rest
    // pose (4n float4) and whether they hold a record
    float4* g_rest = nullptr;
    int* g_valid = nullptr;
    int g_rest_n = 0;
    int graph_warp = 0;             // graph_warp when the pose graph was captured
};

static void rodrigues(const double* w, double* R) {
    const double th = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    const double A = th < 1e-12 ? 1.0 : std::sin(th) / th;
    const double B = th < 1e-12 ? 0.5 : (1.0 - std::cos(th)) / (th * th);
    const double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    double K2[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) K2[3 * r + c] = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
    for (int q = 0; q < 9; ++q) R[q] = (q % 4 == 0 ? 1.0 : 0.0) + A * K[q] + B * K2[q];
}

static void rot_log(const double* R, double* w) {
    const double c = std::fmax(-1.0, std::fmin(1.0, 0.5 * (R[0] + R[4] + R[8] - 1.0)));
    const double th = std::acos(c);
    const double v[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]};
    if (th < 1e-7) {
        for (int k = 0; k < 3; ++k) w[k] = 0.5 * v[k];
        return;
    }
    if (M_PI - th < 1e-5) {
        // near pi: R ~ 2 a a^T - I; axis from the largest diagonal entry
        const int k = (R[0] >= R[4] && R[0] >= R[8]) ? 0 : (R[4] >= R[8] ? 1 : 2);
        double ax[3];
        ax[k] = std::sqrt(std::fmax(0.5 * (R[4 * k] + 1.0), 1e-300));
        for (int j = 0; j < 3; ++j)
            if (j != k) ax[j] = 0.25 * (R[3 * k + j] + R[3 * j + k]) / ax[k];
        const double n = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
        const double sg = (ax[0] * v[0] + ax[1] * v[1] + ax[2] * v[2]) < 0 ? -1.0 : 1.0;
        for (int j = 0; j < 3; ++j) w[j] = sg * th * ax[j] / n;
        return;
    }
    const double f = th / (2.0 * std::sin(th));
    for (int k = 0; k < 3; ++k) w[k] = f * v[k];
}

const PoseDesc* lc_ctx::pose_desc() const { return pose && pose->has_pose ? pose->d : nullptr; }

void lc_ctx::pose_drop_graph() {
    if (pose && pose->gexec) {
        cudaGraphExecDestroy(pose->gexec);
        pose->gexec = nullptr;
    }
}

void lc_ctx::pose_release() {
    if (!pose) return;
    pose_drop_graph();
    void* bufs[] = {(void*)pose->h.parents, (void*)pose->h.rest, (void*)pose->h.col, (void*)pose->h.anc,
                    (void*)pose->h.skin_idx, (void*)pose->h.skin_w, (void*)pose->h.j2d, (void*)pose->h.j3d,
                    (void*)pose->h.level, (void*)pose->h.pairs, pose->h.fk, pose->h.part,
                    pose->h.pose, pose->h.pose_start, pose->h.Rroot, pose->h.blist,
                    pose->h.bcount, pose->h.hist, pose->h.info, pose->h.expA, pose->h.status, pose->d,
                    pose->pose_set, (void*)pose->h.temporal_w, (void*)pose->h.th_lo, (void*)pose->h.th_hi,
                    pose->h.prev_joints, pose->h.pose_hist, pose->h.disp, pose->g_rest, pose->g_valid};
    for (void* p : bufs) release(p);
    delete pose;
    pose = nullptr;
    // the body-part mask follows the skinning weights of the skeleton
    if (hC.part_on) {
        hC.part_on = 0;
        drop_graph();
    }
}

// buffers of the graph stage's displacement warping for the current graph
// (a new graph size reallocates them and drops the captured pose graph,
// which holds their addresses); no record is valid after a reallocation
static lc_status graph_warp_ensure(lc_ctx* ctx) {
    PoseState& S = *ctx->pose;
    if (!ctx->params.graph_warp || !ctx->has_graph || S.g_rest_n == ctx->hC.n) return LC_OK;
    ctx->release(S.g_rest);
    ctx->release(S.g_valid);
    S.g_rest = (float4*)ctx->alloc(sizeof(float4) * 4 * (size_t)ctx->hC.n);
    S.g_valid = (int*)ctx->alloc(sizeof(int));
    S.g_rest_n = 0;
    if (!S.g_rest || !S.g_valid) return LC_ERR_OOM;
    S.g_rest_n = ctx->hC.n;
    ctx->pose_drop_graph();
    return ctx->cuda(cudaMemsetAsync(S.g_valid, 0, sizeof(int), ctx->stream), "graph warp");
}

static bool graph_warp_active(const lc_ctx* ctx) {
    return ctx->pose && ctx->params.graph_warp && ctx->has_graph && ctx->pose->g_rest &&
           ctx->pose->g_rest_n == ctx->hC.n;
}

// a new graph: the recorded rest-pose node parameters no longer apply
void lc_ctx::pose_graph_changed() {
    if (pose && pose->g_valid) cudaMemsetAsync(pose->g_valid, 0, sizeof(int), stream);
}

static lc_status pose_sync(lc_ctx* ctx) {
    lc_status s = ctx->cuda(cudaMemcpyAsync(ctx->pose->d, &ctx->pose->h, sizeof(PoseDesc), cudaMemcpyHostToDevice,
                                            ctx->stream),
                            "pose descriptor");
    if (s) return s;
    ctx->pose->last = ctx->pose->h;
    ctx->pose->synced = true;
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
}

lc_status lc_ctx::pose_frame(const float* joints2d, const float* joints3d) {
    if (!pose) return LC_OK;
    const int J = pose->h.J;
    lc_status s;
    if (joints2d) {
        std::vector<float> j2((size_t)2 * J);
        if ((s = fetch(j2.data(), joints2d, sizeof(float) * 2 * J))) return s;
        if ((s = cuda(cudaMemcpyAsync((void*)pose->h.j2d, j2.data(), sizeof(float) * 2 * J, cudaMemcpyHostToDevice,
                                      stream),
                      "joints")))
            return s;
    }
    if (joints3d) {
        std::vector<float> j3((size_t)3 * J);
        if ((s = fetch(j3.data(), joints3d, sizeof(float) * 3 * J))) return s;
        std::vector<float4> j4(J);
        for (int j = 0; j < J; ++j) j4[j] = make_float4(j3[3 * j], j3[3 * j + 1], j3[3 * j + 2], 0.f);
        if ((s = cuda(cudaMemcpyAsync((void*)pose->h.j3d, j4.data(), sizeof(float4) * J, cudaMemcpyHostToDevice,
                                      stream),
                      "joints")))
            return s;
    }
    const int h2 = joints2d ? 1 : 0, h3 = joints3d ? 1 : 0;
    if (h2 != pose->h.has_j2d || h3 != pose->h.has_j3d) {
        pose->h.has_j2d = h2;
        pose->h.has_j3d = h3;
        return pose_sync(this);
    }
    return cuda(cudaStreamSynchronize(stream), "synchronize");
}

lc_status lc_ctx::pose_read(float* pose_out) {
    if (!pose || !pose->has_pose) return fail(LC_ERR_STATE, "no skeleton / pose");
    const int nd = pose->h.n_dof;
    std::vector<float> p(nd);
    float R[9];
    lc_status s;
    if ((s = copy_to_host(p.data(), pose->h.pose, sizeof(float) * nd)) || (s = copy_to_host(R, pose->h.Rroot, sizeof(R))))
        return s;
    double Rd[9], w[3];
    for (int q = 0; q < 9; ++q) Rd[q] = R[q];
    rot_log(Rd, w);
    for (int k = 0; k < 3; ++k) p[k] = (float)w[k];
    return deliver(pose_out, p.data(), sizeof(float) * nd);
}

static void apply_pose_params(lc_ctx* ctx) {
    PoseDesc& P = ctx->pose->h;
    P.lam_2d = ctx->params.lambda_2d;
    P.lam_3d = ctx->params.lambda_3d;
    P.lam_sil = ctx->params.lambda_sil;
    P.lam_prior = ctx->params.lambda_prior;
    P.lam_temporal = ctx->params.lambda_temporal;
    P.lam_anat = ctx->params.lambda_anatomic;
    P.solver = ctx->params.pose_solver;
    // the skinned displacement of Sec. 3.4 once the surface stage recorded one
    P.use_disp = ctx->params.pose_displacement && ctx->surf_has_disp && ctx->hC.sD ? 1 : 0;
}

extern "C" lc_status lc_upload_skeleton(lc_ctx* ctx, int J, const int32_t* parents, const float* joints_rest,
                                        const uint8_t* dof, const int32_t* skin_idx, const float* skin_w) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_template) return ctx->fail(LC_ERR_STATE, "lc_upload_skeleton: no template");
    if (J < 1 || J > kMaxJoints || !parents || !joints_rest || !dof || !skin_idx || !skin_w)
        return ctx->fail(LC_ERR_ARG, "lc_upload_skeleton: 1 <= J <= %d and non-null arrays required", kMaxJoints);
    cudaSetDevice(ctx->device);
    const int af0 = ctx->alloc_failures;
    const int N = ctx->hC.N;
    std::vector<int32_t> par(J), sidx((size_t)4 * N);
    std::vector<float> rest((size_t)3 * J), sw((size_t)4 * N);
    std::vector<uint8_t> df(J);
    lc_status s;
    if ((s = ctx->fetch(par.data(), parents, sizeof(int32_t) * J)) ||
        (s = ctx->fetch(rest.data(), joints_rest, sizeof(float) * 3 * J)) ||
        (s = ctx->fetch(df.data(), dof, J)) || (s = ctx->fetch(sidx.data(), skin_idx, sizeof(int32_t) * 4 * N)) ||
        (s = ctx->fetch(sw.data(), skin_w, sizeof(float) * 4 * N)))
        return s;
    if (par[0] != -1) return ctx->fail(LC_ERR_ARG, "lc_upload_skeleton: joint 0 must be the root");
    for (int j = 1; j < J; ++j)
        if (par[j] < 0 || par[j] >= j) return ctx->fail(LC_ERR_ARG, "lc_upload_skeleton: parents must precede children");
    for (size_t q = 0; q < sidx.size(); ++q)
        if (sidx[q] < 0 || sidx[q] >= J) return ctx->fail(LC_ERR_ARG, "lc_upload_skeleton: bone index out of range");
    std::vector<int> col(J, -1);
    int nd = 6;
    for (int j = 1; j < J; ++j)
        if (df[j]) {
            col[j] = nd;
            nd += 3;
        }
    if (nd > kMaxDof) return ctx->fail(LC_ERR_ARG, "lc_upload_skeleton: more than %d pose DOF", kMaxDof);
    std::vector<unsigned long long> anc(J, 0ULL);
    for (int j = 0; j < J; ++j)
        for (int a = j; a >= 0; a = par[a]) anc[j] |= 1ULL << a;
    std::vector<int> level(J, 0);
    int n_levels = 1;
    for (int j = 1; j < J; ++j) {
        level[j] = level[par[j]] + 1;
        n_levels = std::max(n_levels, level[j] + 1);
    }
    std::vector<unsigned short> pairs;
    for (int a = 0; a <= nd; ++a)
        for (int b = a; b <= nd; ++b) pairs.push_back((unsigned short)(a << 8 | b));
    if (cudaError_t e = pose_kernels_init(nd)) return ctx->cuda(e, "pose kernel attributes");
    ctx->pose_release();
    ctx->pose = new PoseState();
    PoseState& S = *ctx->pose;
    S.N = N;
    PoseDesc& P = S.h;
    P.J = J;
    P.n_dof = nd;
    P.n_levels = n_levels;
    P.parents = (const int*)ctx->alloc(sizeof(int) * J);
    P.level = (const int*)ctx->alloc(sizeof(int) * J);
    P.pairs = (const unsigned short*)ctx->alloc(sizeof(unsigned short) * pairs.size());
    P.fk = (PoseFk*)ctx->alloc(sizeof(PoseFk));
    P.part = (float*)ctx->alloc(sizeof(float) * pairs.size() * (size_t)pose_system_ctas(J, N));
    P.rest = (const float4*)ctx->alloc(sizeof(float4) * J);
    P.col = (const int*)ctx->alloc(sizeof(int) * J);
    P.anc = (const unsigned long long*)ctx->alloc(sizeof(unsigned long long) * J);
    P.tpl = ctx->tpl;
    P.skin_idx = (const int4*)ctx->alloc(sizeof(int4) * N);
    P.skin_w = (const float4*)ctx->alloc(sizeof(float4) * N);
    P.j2d = (const float2*)ctx->alloc(sizeof(float2) * J);
    P.j3d = (const float4*)ctx->alloc(sizeof(float4) * J);
    P.pose = (float*)ctx->alloc(sizeof(float) * kMaxDof);
    P.pose_start = (float*)ctx->alloc(sizeof(float) * kMaxDof);
    P.Rroot = (float*)ctx->alloc(sizeof(float) * 9);
    P.blist = (int*)ctx->alloc(sizeof(int) * N);
    P.bcount = (int*)ctx->alloc(sizeof(int));
    P.hist = (double*)ctx->alloc(sizeof(double) * 2 * (LC_MAX_GN + 1));
    P.info = (int*)ctx->alloc(sizeof(int) * (LC_MAX_GN + 1));
    P.expA = (double*)ctx->alloc(sizeof(double) * nd * (nd + 1));
    P.status = (int*)ctx->alloc(sizeof(int));
    P.temporal_w = (const float*)ctx->alloc(sizeof(float) * J);
    P.th_lo = (const float*)ctx->alloc(sizeof(float) * kMaxDof);
    P.th_hi = (const float*)ctx->alloc(sizeof(float) * kMaxDof);
    P.disp = (float4*)ctx->alloc(sizeof(float4) * N);
    P.use_disp = 0;
    P.prev_joints = (float4*)ctx->alloc(sizeof(float4) * J);
    P.pose_hist = (float*)ctx->alloc(sizeof(float) * 2 * (kMaxDof + 9));
    P.has_prev = 0;
    P.n_hist = 0;
    S.d = (PoseDesc*)ctx->alloc(sizeof(PoseDesc));
    S.pose_set = (float*)ctx->alloc(sizeof(float) * (kMaxDof + 9));
    if (ctx->alloc_failures != af0) return LC_ERR_OOM;
    std::vector<float4> r4(J), w4(N);
    std::vector<int4> i4(N);
    for (int j = 0; j < J; ++j) r4[j] = make_float4(rest[3 * j], rest[3 * j + 1], rest[3 * j + 2], 0.f);
    for (int i = 0; i < N; ++i) {
        i4[i] = make_int4(sidx[4 * i], sidx[4 * i + 1], sidx[4 * i + 2], sidx[4 * i + 3]);
        w4[i] = make_float4(sw[4 * i], sw[4 * i + 1], sw[4 * i + 2], sw[4 * i + 3]);
    }
    // rest pose: identity root rotation at the root's rest position, zero angles
    std::vector<float> p0(kMaxDof, 0.f);
    p0[3] = rest[0];
    p0[4] = rest[1];
    p0[5] = rest[2];
    const float I3[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    const std::vector<float> ones(J, 1.f), lo(kMaxDof, -INFINITY), hi(kMaxDof, INFINITY);
    cudaStream_t st = ctx->stream;
    struct Up {
        const void* dst;
        const void* src;
        size_t bytes;
    } ups[] = {{P.parents, par.data(), sizeof(int) * J},     {P.rest, r4.data(), sizeof(float4) * J},
               {P.level, level.data(), sizeof(int) * J},
               {P.pairs, pairs.data(), sizeof(unsigned short) * pairs.size()},
               {P.col, col.data(), sizeof(int) * J},         {P.anc, anc.data(), sizeof(unsigned long long) * J},
               {P.skin_idx, i4.data(), sizeof(int4) * N},    {P.skin_w, w4.data(), sizeof(float4) * N},
               {P.pose, p0.data(), sizeof(float) * kMaxDof}, {P.pose_start, p0.data(), sizeof(float) * kMaxDof},
               {P.Rroot, I3, sizeof(I3)},                    {S.pose_set, p0.data(), sizeof(float) * kMaxDof},
               {S.pose_set + kMaxDof, I3, sizeof(I3)},      {P.temporal_w, ones.data(), sizeof(float) * J},
               {P.th_lo, lo.data(), sizeof(float) * kMaxDof}, {P.th_hi, hi.data(), sizeof(float) * kMaxDof}};
    for (auto& u : ups)
        if ((s = ctx->cuda(cudaMemcpyAsync((void*)u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, st), "skeleton upload")))
            return s;
    cudaMemsetAsync(P.status, 0, sizeof(int), st);
    cudaMemsetAsync((void*)P.j2d, 0, sizeof(float2) * J, st);
    cudaMemsetAsync((void*)P.j3d, 0, sizeof(float4) * J, st);
    apply_pose_params(ctx);
    S.has_pose = true;
    return pose_sync(ctx);
}

extern "C" lc_status lc_set_pose(lc_ctx* ctx, const float* pose) {
    if (!ctx || !pose) return LC_ERR_ARG;
    if (!ctx->pose) return ctx->fail(LC_ERR_STATE, "lc_set_pose: no skeleton");
    cudaSetDevice(ctx->device);
    const int nd = ctx->pose->h.n_dof;
    std::vector<float> p(nd);
    lc_status s;
    if ((s = ctx->fetch(p.data(), pose, sizeof(float) * nd))) return s;
    double w[3] = {p[0], p[1], p[2]}, R[9];
    rodrigues(w, R);
    float Rf[9];
    for (int q = 0; q < 9; ++q) Rf[q] = (float)R[q];
    if ((s = ctx->cuda(cudaMemcpyAsync(ctx->pose->h.pose, p.data(), sizeof(float) * nd, cudaMemcpyHostToDevice, ctx->stream),
                       "pose upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync(ctx->pose->h.Rroot, Rf, sizeof(Rf), cudaMemcpyHostToDevice, ctx->stream),
                       "pose upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync(ctx->pose->pose_set, ctx->pose->h.pose, sizeof(float) * nd,
                                       cudaMemcpyDeviceToDevice, ctx->stream),
                       "pose upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync(ctx->pose->pose_set + kMaxDof, Rf, sizeof(Rf), cudaMemcpyHostToDevice,
                                       ctx->stream),
                       "pose upload")))
        return s;
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
}

extern "C" lc_status lc_set_pose_priors(lc_ctx* ctx, const float* temporal_w, const float* theta_min,
                                        const float* theta_max) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->pose) return ctx->fail(LC_ERR_STATE, "lc_set_pose_priors: no skeleton");
    if ((theta_min == nullptr) != (theta_max == nullptr))
        return ctx->fail(LC_ERR_ARG, "lc_set_pose_priors: give both limits or neither");
    cudaSetDevice(ctx->device);
    PoseDesc& P = ctx->pose->h;
    const int J = P.J, nd = P.n_dof;
    lc_status s;
    std::vector<float> w(J, 1.f), lo(kMaxDof, -INFINITY), hi(kMaxDof, INFINITY);
    if (temporal_w && (s = ctx->fetch(w.data(), temporal_w, sizeof(float) * J))) return s;
    for (int j = 0; j < J; ++j)
        if (!(w[j] >= 0.f) || !std::isfinite(w[j])) return ctx->fail(LC_ERR_ARG, "lc_set_pose_priors: bad weight");
    if (theta_min) {
        if ((s = ctx->fetch(lo.data(), theta_min, sizeof(float) * nd)) ||
            (s = ctx->fetch(hi.data(), theta_max, sizeof(float) * nd)))
            return s;
        for (int c = 0; c < nd; ++c) {
            if (c < 6) {
                lo[c] = -INFINITY;   // the root carries no limits
                hi[c] = INFINITY;
            } else if (!(lo[c] <= hi[c])) {
                return ctx->fail(LC_ERR_ARG, "lc_set_pose_priors: theta_min > theta_max");
            }
        }
    }
    if ((s = ctx->cuda(cudaMemcpyAsync((void*)P.temporal_w, w.data(), sizeof(float) * J, cudaMemcpyHostToDevice,
                                       ctx->stream), "upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync((void*)P.th_lo, lo.data(), sizeof(float) * kMaxDof, cudaMemcpyHostToDevice,
                                       ctx->stream), "upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync((void*)P.th_hi, hi.data(), sizeof(float) * kMaxDof, cudaMemcpyHostToDevice,
                                       ctx->stream), "upload")))
        return s;
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
}

extern "C" lc_status lc_pose_advance(lc_ctx* ctx) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->pose) return ctx->fail(LC_ERR_STATE, "lc_pose_advance: no skeleton");
    cudaSetDevice(ctx->device);
    PoseState& S = *ctx->pose;
    lc_status s;
    if ((s = graph_warp_ensure(ctx))) return s;
    launch_pose_advance(S.d, ctx->stream);
    if (graph_warp_active(ctx)) launch_graph_warp(ctx->dC, ctx->hC, S.d, S.g_rest, S.g_valid, 0, ctx->stream);
    s = ctx->cuda(cudaGetLastError(), "lc_pose_advance");
    if (s) return s;
    if (S.h.has_prev && S.h.n_hist >= 2) return LC_OK;   // the descriptor is unchanged
    S.h.has_prev = 1;
    S.h.n_hist = std::min(S.h.n_hist + 1, 2);
    return pose_sync(ctx);
}

extern "C" lc_status lc_pose_extrapolate(lc_ctx* ctx) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->pose) return ctx->fail(LC_ERR_STATE, "lc_pose_extrapolate: no skeleton");
    if (ctx->pose->h.n_hist == 0) return ctx->fail(LC_ERR_STATE, "lc_pose_extrapolate: no recorded pose");
    cudaSetDevice(ctx->device);
    launch_pose_extrapolate(ctx->pose->d, ctx->stream);
    return ctx->cuda(cudaGetLastError(), "lc_pose_extrapolate");
}

extern "C" lc_status lc_pose_clear_history(lc_ctx* ctx) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->pose) return ctx->fail(LC_ERR_STATE, "lc_pose_clear_history: no skeleton");
    cudaSetDevice(ctx->device);
    ctx->pose->h.has_prev = 0;
    ctx->pose->h.n_hist = 0;
    if (ctx->pose->g_valid) cudaMemsetAsync(ctx->pose->g_valid, 0, sizeof(int), ctx->stream);
    return pose_sync(ctx);
}

extern "C" lc_status lc_reset_pose(lc_ctx* ctx) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->pose) return ctx->fail(LC_ERR_STATE, "lc_reset_pose: no skeleton");
    cudaSetDevice(ctx->device);
    PoseState& S = *ctx->pose;
    lc_status s;
    if ((s = ctx->cuda(cudaMemcpyAsync(S.h.pose, S.pose_set, sizeof(float) * kMaxDof, cudaMemcpyDeviceToDevice,
                                       ctx->stream),
                       "pose reset")) ||
        (s = ctx->cuda(cudaMemcpyAsync(S.h.Rroot, S.pose_set + kMaxDof, sizeof(float) * 9, cudaMemcpyDeviceToDevice,
                                       ctx->stream),
                       "pose reset")))
        return s;
    return LC_OK;
}

// A frame step captured once and replayed (lc_batch_step): the host state
// that lc_solve_pose and lc_pose_advance keep must not change between
// replays, so the pose history must be full (two recorded frames) and the
// descriptor is brought to the device here, before the capture.
lc_status pose_step_prepare(lc_ctx* ctx) {
    if (!ctx->pose) return ctx->fail(LC_ERR_STATE, "lc_batch_step: a member has no skeleton");
    PoseState& S = *ctx->pose;
    if (!S.h.has_prev || S.h.n_hist < 2)
        return ctx->fail(LC_ERR_STATE, "lc_batch_step: a member has fewer than two recorded frames (lc_pose_advance)");
    if (!ctx->has_camera || !ctx->has_frame) return ctx->fail(LC_ERR_STATE, "lc_batch_step: camera and frame required");
    apply_pose_params(ctx);
    lc_status s;
    if ((s = graph_warp_ensure(ctx))) return s;
    if (!S.synced || memcmp(&S.h, &S.last, sizeof(PoseDesc)) != 0) return pose_sync(ctx);
    return LC_OK;
}

// the frame's start and pose stage, then (after the non-rigid stage) its end,
// enqueued on ctx->stream
void pose_step_begin(lc_ctx* ctx, bool euler_start) {
    if (euler_start) launch_pose_extrapolate(ctx->pose->d, ctx->stream);
    ctx->enqueue_pose();
}

void pose_step_end(lc_ctx* ctx) {
    PoseState& S = *ctx->pose;
    launch_pose_advance(S.d, ctx->stream);
    if (graph_warp_active(ctx)) launch_graph_warp(ctx->dC, ctx->hC, S.d, S.g_rest, S.g_valid, 0, ctx->stream);
}

void lc_ctx::enqueue_pose() {
    PoseState& S = *pose;
    const PoseDesc& P = S.h;
    cudaStream_t st = stream;
    prof_pose.begin = prof_used;
    mark(LC_PH_POSE);
    cudaMemsetAsync(P.hist, 0, sizeof(double) * 2 * (LC_MAX_GN + 1), st);
    cudaMemsetAsync(P.info, 0, sizeof(int) * (LC_MAX_GN + 1), st);
    cudaMemcpyAsync(P.pose_start, P.pose, sizeof(float) * kMaxDof, cudaMemcpyDeviceToDevice, st);
    mark(LC_PH_POSE_VIS);
    launch_pose_fk(S.d, st);
    if (P.use_disp) launch_surface_warp(dC, hC, S.d, 2, st);   // d^S at the start pose
    launch_pose_skin(dC, hC, S.d, nullptr, 0, st);
    launch_vis_unfreeze(dC, st);
    launch_visibility(dC, hC, st);
    launch_pose_blist(dC, S.d, st);
    // step 0 linearises at the start pose, whose b_i the contour pass just
    // decided on the same vertices; later steps re-decide them
    for (int g = 0; g < params.n_gn_pose; ++g) {
        mark(LC_PH_POSE_SYS);
        if (g > 0) launch_pose_dirs(dC, hC, S.d, st);
        launch_pose_system(dC, hC, S.d, P.J, P.n_dof, st);
        mark(LC_PH_POSE_SOLVE);
        launch_pose_solve(S.d, g, 0, st);
    }
    mark(LC_PH_POSE_SYS);
    launch_pose_dirs(dC, hC, S.d, st);
    launch_pose_system(dC, hC, S.d, P.J, P.n_dof, st);
    mark(LC_PH_POSE_SOLVE);
    launch_pose_solve(S.d, params.n_gn_pose, 1, st);
    // the skinned mesh becomes the rest geometry of the non-rigid stage
    mark(LC_PH_POSE);
    launch_pose_skin(dC, hC, S.d, base_buf, 1, st);
    if (has_graph) launch_gather_nodes(base_buf, hC.node_vid, hC.n, (float4*)hC.node_g, st);
    // the node parameters recorded in the rest pose at the end of the last
    // frame, carried into the solved pose
    if (graph_warp_active(this)) launch_graph_warp(dC, hC, S.d, S.g_rest, S.g_valid, 1, st);
    mark_end();
    prof_pose.end = prof_used;
}

extern "C" lc_status lc_solve_pose(lc_ctx* ctx, lc_solve_stats* stats) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->pose) return ctx->fail(LC_ERR_STATE, "lc_solve_pose: no skeleton");
    if (!ctx->has_camera || !ctx->has_frame) return ctx->fail(LC_ERR_STATE, "lc_solve_pose: camera and frame required");
    cudaSetDevice(ctx->device);
    PoseState& S = *ctx->pose;
    lc_status s;
    apply_pose_params(ctx);
    // the descriptor goes to the device only when it changed (a copy and a
    // synchronisation per frame otherwise)
    if (!S.synced || memcmp(&S.h, &S.last, sizeof(PoseDesc)) != 0) {
        if ((s = pose_sync(ctx))) return s;
    }
    if ((s = graph_warp_ensure(ctx))) return s;
    const int warp_on = graph_warp_active(ctx) ? 1 : 0;
    if (S.gexec && (S.graph_n_gn != ctx->params.n_gn_pose || S.graph_disp != S.h.use_disp || S.graph_warp != warp_on))
        ctx->pose_drop_graph();
    if (!S.gexec) {
        if ((s = ctx->capture(&S.gexec, &S.graph_kernels, &lc_ctx::enqueue_pose))) return s;
        S.graph_n_gn = ctx->params.n_gn_pose;
        S.graph_disp = S.h.use_disp;   // the displacement kernel is in the graph or not
        S.graph_warp = warp_on;        // and the graph warping kernel
    }
    if ((s = ctx->cuda(cudaGraphLaunch(S.gexec, ctx->stream), "graph launch"))) return s;
    if ((s = ctx->accumulate_profile(ctx->prof_pose))) return s;
    // the visibility state now holds the pose stage's frame decisions
    // (z-buffer, visibility and B at the starting pose; b_i and uv at the final)
    ctx->has_vis = true;
    ctx->has_lin = false;
    if (stats) {
        std::vector<double> hist(2 * (LC_MAX_GN + 1));
        std::vector<int> info(LC_MAX_GN + 1);
        int status = 0, nb = 0;
        if ((s = ctx->copy_to_host(hist.data(), S.h.hist, sizeof(double) * hist.size())) ||
            (s = ctx->copy_to_host(info.data(), S.h.info, sizeof(int) * info.size())) ||
            (s = ctx->copy_to_host(&status, S.h.status, sizeof(int))) ||
            (s = ctx->copy_to_host(&nb, S.h.bcount, sizeof(int))))
            return s;
        memset(stats, 0, sizeof(*stats));
        const int g = ctx->params.n_gn_pose;
        for (int k = 0; k < g; ++k) {
            stats->e_gn[k] = hist[2 * k];
            stats->step_norm[k] = hist[2 * k + 1];
            stats->pcg_iters[k] = info[k];
        }
        stats->e_total = hist[2 * g];
        stats->n_gn_done = g;
        stats->n_boundary = nb;
        stats->n_kernels = S.graph_kernels;
        if (status) {
            cudaMemsetAsync(S.h.status, 0, sizeof(int), ctx->stream);
            return ctx->fail(LC_ERR_NUMERIC, "lc_solve_pose: non-positive pivot in the Cholesky factorisation");
        }
    }
    return LC_OK;
}

extern "C" lc_status lc_eval_pose(lc_ctx* ctx, float* V_skinned, double* A, double* g, double* energy) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->pose) return ctx->fail(LC_ERR_STATE, "lc_eval_pose: no skeleton");
    if (!ctx->has_camera || !ctx->has_frame) return ctx->fail(LC_ERR_STATE, "lc_eval_pose: camera and frame required");
    cudaSetDevice(ctx->device);
    PoseState& S = *ctx->pose;
    const int nd = S.h.n_dof, N = ctx->hC.N;
    apply_pose_params(ctx);
    lc_status s;
    if ((s = pose_sync(ctx))) return s;
    cudaStream_t st = ctx->stream;
    // contour set at the current pose, then the system at the current pose
    cudaMemcpyAsync(S.h.pose_start, S.h.pose, sizeof(float) * kMaxDof, cudaMemcpyDeviceToDevice, st);
    launch_pose_fk(S.d, st);
    if (S.h.use_disp) launch_surface_warp(ctx->dC, ctx->hC, S.d, 2, st);
    launch_pose_skin(ctx->dC, ctx->hC, S.d, nullptr, 0, st);
    launch_vis_unfreeze(ctx->dC, st);
    launch_visibility(ctx->dC, ctx->hC, st);
    launch_pose_blist(ctx->dC, S.d, st);
    launch_pose_system(ctx->dC, ctx->hC, S.d, S.h.J, S.h.n_dof, st);
    launch_pose_solve(S.d, LC_MAX_GN, 2, st);
    if ((s = ctx->cuda(cudaGetLastError(), "pose eval"))) return s;
    ctx->has_vis = true;
    ctx->has_lin = false;
    if (V_skinned) {
        std::vector<float4> v4(N);
        if ((s = ctx->copy_to_host(v4.data(), ctx->hC.vw, sizeof(float4) * N))) return s;
        std::vector<float> v(3 * (size_t)N);
        for (int i = 0; i < N; ++i) {
            v[3 * i] = v4[i].x;
            v[3 * i + 1] = v4[i].y;
            v[3 * i + 2] = v4[i].z;
        }
        if ((s = ctx->deliver(V_skinned, v.data(), sizeof(float) * v.size()))) return s;
    }
    std::vector<double> ex((size_t)nd * (nd + 1));
    if ((s = ctx->copy_to_host(ex.data(), S.h.expA, sizeof(double) * ex.size()))) return s;
    if (A) {
        std::vector<double> a((size_t)nd * nd);
        for (int r = 0; r < nd; ++r)
            for (int c = 0; c < nd; ++c) a[(size_t)r * nd + c] = ex[(size_t)r * (nd + 1) + c];
        if ((s = ctx->deliver(A, a.data(), sizeof(double) * a.size()))) return s;
    }
    if (g) {
        std::vector<double> gg(nd);
        for (int r = 0; r < nd; ++r) gg[r] = ex[(size_t)r * (nd + 1) + nd];
        if ((s = ctx->deliver(g, gg.data(), sizeof(double) * nd))) return s;
    }
    if (energy) {
        std::vector<double> hist(2 * (LC_MAX_GN + 1));
        if ((s = ctx->copy_to_host(hist.data(), S.h.hist, sizeof(double) * hist.size()))) return s;
        if ((s = ctx->deliver(energy, &hist[2 * LC_MAX_GN], sizeof(double)))) return s;
    }
    return LC_OK;
}

// ---------------------------------------------------------------------------
// body-part mask of the silhouette term (Sec. 3.4)
// ---------------------------------------------------------------------------
lc_status lc_ctx::part_images() {
    release(part_raw_buf);
    release(part_mask_buf);
    const size_t P = (size_t)hC.W * hC.H;
    part_raw_buf = (uint8_t*)alloc(P);
    part_mask_buf = (uint8_t*)alloc(P);
    if (!part_raw_buf || !part_mask_buf) return LC_ERR_OOM;
    // nothing labelled until the first frame decisions
    if (lc_status s = cuda(cudaMemsetAsync(part_mask_buf, 0xff, P, stream), "part mask")) return s;
    if (lc_status s = cuda(cudaMemsetAsync(part_raw_buf, 0xff, P, stream), "part mask")) return s;
    hC.part_raw = part_raw_buf;
    hC.part_mask = part_mask_buf;
    return LC_OK;
}

extern "C" lc_status lc_set_body_parts(lc_ctx* ctx, const int32_t* bone_part, int torso_part, int dilate_px) {
    if (!ctx) return LC_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (!bone_part) {
        if (ctx->hC.part_on) {
            ctx->hC.part_on = 0;
            ctx->drop_graph();
        }
        return ctx->sync_desc();
    }
    if (!ctx->pose) return ctx->fail(LC_ERR_STATE, "lc_set_body_parts: no skeleton");
    if (!ctx->has_camera) return ctx->fail(LC_ERR_STATE, "lc_set_body_parts: no camera");
    if (torso_part < -1 || torso_part > 254 || dilate_px < 0 || dilate_px > 32)
        return ctx->fail(LC_ERR_ARG, "lc_set_body_parts: torso_part -1..254, dilate_px 0..32");
    const int J = ctx->pose->h.J, N = ctx->hC.N;
    std::vector<int32_t> bp(J);
    lc_status s;
    if ((s = ctx->fetch(bp.data(), bone_part, sizeof(int32_t) * J))) return s;
    for (int j = 0; j < J; ++j)
        if (bp[j] < 0 || bp[j] > 254) return ctx->fail(LC_ERR_ARG, "lc_set_body_parts: part labels are 0..254");
    ctx->release(ctx->bone_part_buf);
    ctx->release(ctx->vpart_buf);
    ctx->bone_part_buf = (int*)ctx->alloc(sizeof(int) * J);
    ctx->vpart_buf = (uint8_t*)ctx->alloc((size_t)N);
    if (!ctx->bone_part_buf || !ctx->vpart_buf) return LC_ERR_OOM;
    if ((s = ctx->part_images())) return s;
    if ((s = ctx->cuda(cudaMemcpyAsync(ctx->bone_part_buf, bp.data(), sizeof(int32_t) * J, cudaMemcpyHostToDevice,
                                       ctx->stream), "body parts")))
        return s;
    launch_vertex_parts(ctx->pose->h.skin_idx, ctx->pose->h.skin_w, ctx->bone_part_buf, N, ctx->vpart_buf, ctx->stream);
    if ((s = ctx->cuda(cudaGetLastError(), "body parts"))) return s;
    CapDesc& C = ctx->hC;
    if (!C.part_on) ctx->drop_graph();
    C.vpart = ctx->vpart_buf;
    C.part_on = 1;
    C.torso_part = torso_part;
    C.part_dilate = dilate_px;
    return ctx->sync_desc();
}

extern "C" lc_status lc_read_part_mask(lc_ctx* ctx, uint8_t* mask, uint8_t* vertex_part) {
    if (!ctx) return LC_ERR_ARG;
    const CapDesc& C = ctx->hC;
    if (!C.part_on) return ctx->fail(LC_ERR_STATE, "lc_read_part_mask: no body-part mask");
    cudaSetDevice(ctx->device);
    lc_status s;
    if (mask) {
        std::vector<uint8_t> m((size_t)C.W * C.H);
        if ((s = ctx->copy_to_host(m.data(), C.part_mask, m.size()))) return s;
        if ((s = ctx->deliver(mask, m.data(), m.size()))) return s;
    }
    if (vertex_part) {
        std::vector<uint8_t> v((size_t)C.N);
        if ((s = ctx->copy_to_host(v.data(), C.vpart, v.size()))) return s;
        if ((s = ctx->deliver(vertex_part, v.data(), v.size()))) return s;
    }
    return LC_OK;
}

// Skeletal pose stage (Sec. 3.3): entry points.
#include "lc_context.h"

struct PoseState {};

void lc_ctx::pose_release() {
    delete pose;
    pose = nullptr;
}

void lc_ctx::pose_drop_graph() {}

lc_status lc_ctx::pose_frame(const float* joints2d, const float* joints3d) {
    (void)joints2d;
    (void)joints3d;
    return LC_OK;
}

lc_status lc_ctx::pose_read(float* pose_out) {
    (void)pose_out;
    return fail(LC_ERR_STATE, "no skeleton uploaded");
}

extern "C" lc_status lc_upload_skeleton(lc_ctx* ctx, int J, const int32_t* parents, const float* joints_rest,
                                        const uint8_t* dof, const int32_t* skin_idx, const float* skin_w) {
    (void)J; (void)parents; (void)joints_rest; (void)dof; (void)skin_idx; (void)skin_w;
    if (!ctx) return LC_ERR_ARG;
    return ctx->fail(LC_ERR_STATE, "lc_upload_skeleton: pose stage not available in this build");
}

extern "C" lc_status lc_set_pose(lc_ctx* ctx, const float* pose) {
    (void)pose;
    if (!ctx) return LC_ERR_ARG;
    return ctx->fail(LC_ERR_STATE, "lc_set_pose: no skeleton");
}

extern "C" lc_status lc_solve_pose(lc_ctx* ctx, lc_solve_stats* stats) {
    (void)stats;
    if (!ctx) return LC_ERR_ARG;
    return ctx->fail(LC_ERR_STATE, "lc_solve_pose: no skeleton");
}

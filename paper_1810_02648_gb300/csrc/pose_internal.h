// Device descriptor of the skeletal pose stage.
#pragma once

#include "lc_internal.cuh"

namespace lc {

constexpr int kMaxJoints = 64;
constexpr int kMaxDof = 63;    // 6 root DOF + 3 per ball joint (up to 19 ball joints)

struct PoseDesc {
    int J, n_dof, max_rows;
    int has_j2d, has_j3d;
    float lam_2d, lam_3d, lam_sil, lam_prior;
    const int* parents;               // J
    const float4* rest;               // J rest joint positions
    const int* col;                   // J: first pose column of a ball joint, -1 otherwise
    const unsigned long long* anc;    // J: bit a set iff a is j or an ancestor of j
    const float4* tpl;                // N rest template
    const int4* skin_idx;             // N
    const float4* skin_w;             // N
    const float2* j2d;                // J
    const float4* j3d;                // J
    float* pose;                      // n_dof ([0:3] unused on the device)
    float* pose_start;                // n_dof: the frame's start pose (angle prior)
    float* Rroot;                     // 9
    float* F;                         // max_rows
    float* Jm;                        // n_dof x max_rows, column-major
    int* blist;                       // N contour vertices
    int* bcount;
    double* hist;                     // 2 (LC_MAX_GN + 1): energy, step norm
    double* expA;                     // n_dof x (n_dof + 1) exported system (inspection)
    int* status;                      // 1: non-positive Cholesky pivot
};

void launch_pose_skin(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, float4* out_base, int mode,
                      cudaStream_t st);
void launch_pose_blist(const CapDesc* dC, const PoseDesc* dP, cudaStream_t st);
// re-skins the mesh into C.vw / C.uv and re-evaluates b_i of the contour set
void launch_pose_dirs(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, cudaStream_t st);
void launch_pose_rows(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, int J, cudaStream_t st);
// mode 0: solve and update, 1: energy only, 2: export A | g into expA
void launch_pose_solve(const PoseDesc* dP, int slot, int mode, cudaStream_t st);

}  // namespace lc

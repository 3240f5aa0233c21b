// Device descriptor of the skeletal pose stage.
#pragma once

#include "lc_internal.cuh"

namespace lc {

constexpr int kMaxJoints = 64;
constexpr int kMaxDof = 63;    // 6 root DOF + 3 per ball joint (up to 19 ball joints)
constexpr int kSysItems = 64;  // residual items (joints / contour vertices) per row CTA
constexpr int kSysThreads = 256;

// kinematics of every joint at the current pose
struct PoseFk {
    float G[kMaxJoints][9];    // world rotation
    float o[kMaxJoints][3];    // world position
    float U[kMaxJoints][9];    // world Euler axes (x, y, z columns) of a DOF joint
};

struct PoseDesc {
    int J, n_dof, n_levels;
    int has_j2d, has_j3d;
    float lam_2d, lam_3d, lam_sil, lam_prior;
    float lam_temporal, lam_anat;
    int solver;                       // 0: mixed-precision refinement, 1: FP64 L D L^T
    int has_prev;                     // previous-frame joints recorded (E_temporal on)
    int n_hist;                       // poses recorded for the frame-start extrapolation (0..2)
    const int* parents;               // J
    const int* level;                 // J: depth in the tree (root 0)
    const unsigned short* pairs;      // (n_dof + 1)(n_dof + 2) / 2: a << 8 | b, column pairs a <= b of [J | F]
    const float4* rest;               // J rest joint positions
    const int* col;                   // J: first pose column of a ball joint, -1 otherwise
    const unsigned long long* anc;    // J: bit a set iff a is j or an ancestor of j
    const float4* tpl;                // N rest template
    const int4* skin_idx;             // N
    const float4* skin_w;             // N
    const float2* j2d;                // J
    const float4* j3d;                // J
    const float* temporal_w;          // J: per-joint weights of E_temporal
    const float* th_lo;               // n_dof: joint angle limits of E_anatomic (+-inf where none)
    const float* th_hi;
    float4* prev_joints;              // J: joints of the previous frame
    float* pose_hist;                 // 2 (kMaxDof + 9): poses t-1, t-2, each followed by its root rotation
    float* pose;                      // n_dof ([0:3] unused on the device)
    float* pose_start;                // n_dof: the frame's start pose (angle prior)
    float* Rroot;                     // 9
    PoseFk* fk;                       // kinematics at the current pose
    float* part;                      // row CTAs x pairs: FP32 partial pair sums
    int* blist;                       // N contour vertices
    int* bcount;
    double* hist;                     // 2 (LC_MAX_GN + 1): energy, step norm
    int* info;                        // LC_MAX_GN + 1: refinement rounds of each step's solve (-1: FP64 factorisation)
    double* expA;                     // n_dof x (n_dof + 1) exported system (inspection)
    int* status;                      // 1: non-positive Cholesky pivot
    float4* disp;                     // N: skinned displacement d^S added to the skinned model (Sec. 3.4)
    int use_disp;                     // disp is set at every solve's start and used
};

void launch_pose_skin(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, float4* out_base, int mode,
                      cudaStream_t st);
void launch_pose_blist(const CapDesc* dC, const PoseDesc* dP, cudaStream_t st);
// forward kinematics of the current pose into P.fk
void launch_pose_fk(const PoseDesc* dP, cudaStream_t st);
// re-skins the mesh into C.vw / C.uv and re-evaluates b_i of the contour set
void launch_pose_dirs(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, cudaStream_t st);
// the current joints -> prev_joints, the pose history shifted by one (after
// a kinematics pass of the current pose)
void launch_pose_advance(const PoseDesc* dP, cudaStream_t st);
// the pose <- the explicit Euler step from the pose history (n_hist >= 1)
void launch_pose_extrapolate(const PoseDesc* dP, cudaStream_t st);
// the graph stage's displacement warping: mode 0 records the node parameters in the rest pose,
// mode 1 poses a valid record with the current pose (rest: 4n float4)
void launch_graph_warp(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, float4* rest, int* valid, int mode,
                       cudaStream_t st);
// displacement warping of the surface stage (dP null: no skeleton, Q_i = I);
// mode 0 records sD from sV, mode 1 sets sV from sD, mode 2 writes Q_i sD_i
// into the pose stage's dP->disp
void launch_surface_warp(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, int mode, cudaStream_t st);
// residual rows -> partial pair sums (P.part)
cudaError_t pose_kernels_init(int n_dof);
int pose_system_ctas(int J, int N);
void launch_pose_system(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, int J, int n_dof,
                        cudaStream_t st);
// mode 0: solve, update and the next kinematics; 1: energy only; 2: export A | g into expA
void launch_pose_solve(const PoseDesc* dP, int slot, int mode, cudaStream_t st);

}  // namespace lc

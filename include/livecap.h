/*
 * livecap.h — C ABI of the GB300 (sm_103a) Gauss-Newton hot path of LiveCap
 * ("Real-time Human Performance Capture from Monocular Video", Habermann et
 * al., arXiv 1810.02648).
 *
 * Conventions for every call
 * --------------------------
 *  - Every call returns an lc_status.  The message of the most recent failed
 *    call on a context is returned by lc_last_error(); a failure leaves the
 *    context usable for later calls, which return their own status.  Device-side failures (a pivot <= 0 in the
 *    pose Cholesky, a non-finite input) are reported through a status word
 *    that the next synchronising call reads.
 *  - Array arguments are plain pointers that may point to host memory or to
 *    CUDA device memory of the context's device; the library tells them apart
 *    with cudaPointerGetAttributes.  The caller owns every pointer it passes.
 *    Uploads copy into library-owned device memory; read-backs copy out.
 *    Shapes are given per argument; all arrays are dense, row-major, with no
 *    padding.
 *  - Work is enqueued on the context's stream (the one given to lc_create).
 *    Calls that return data to host memory synchronise that stream;
 *    calls that only enqueue device work return without waiting.
 *  - Calls made in the wrong order return LC_ERR_STATE (for instance a solve
 *    before a template, graph and frame exist).
 *
 * Geometry conventions: camera space is world space (Sec. 3.2 of the paper);
 * pinhole projection u = f X/Z + cx, v = f Y/Z + cy with pixel centres on
 * integer coordinates; images are H rows of W pixels.
 */
#ifndef LIVECAP_H
#define LIVECAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lc_ctx lc_ctx;

typedef enum {
    LC_OK = 0,
    LC_ERR_ARG = -1,      /* invalid argument (null pointer, bad size, bad mesh) */
    LC_ERR_STATE = -2,    /* call out of order */
    LC_ERR_CUDA = -3,     /* CUDA runtime error (message in lc_last_error) */
    LC_ERR_NUMERIC = -4,  /* non-positive pivot or non-finite value */
    LC_ERR_TIMEOUT = -5,  /* a bounded device-side wait ran out */
    LC_ERR_OOM = -6       /* device allocation failed */
} lc_status;

/* Solver settings.
 * Non-rigid energy weights (Sec. 3.4, E_photo / E_silhouette, plus the
 * embedded-graph ARAP regulariser) and fixed iteration counts of the
 * Gauss-Newton / PCG solver (Sec. 4: no damping, fixed counts).  eps_vis is
 * the depth tolerance of the visibility test in metres.  The lambda_* are the
 * pose-stage weights of Sec. 3.3 (defaults from the paper's parameter list in
 * Sec. 5: lambda_2D = 460, lambda_3D = 28, lambda_silhouette = 200). */
typedef struct {
    float w_photo;      /* default 1 */
    float w_sil;        /* default 0.1 */
    float w_arap;       /* default 10 */
    int n_gn;           /* Gauss-Newton steps of the non-rigid stage, <= LC_MAX_GN */
    int n_pcg;          /* PCG iterations per step */
    float eps_vis;      /* default 1e-2 m */
    float lambda_2d;
    float lambda_3d;
    float lambda_sil;
    int n_gn_pose;      /* Gauss-Newton steps of the pose stage, default 5 */
    float lambda_prior; /* pose stage: weight of (theta - theta_start)^2 on the
                           Euler angles, default 1e4 (keeps the 57x57 system
                           positive definite: bone twists that move no joint and
                           no silhouette are otherwise undetermined) */
    int pcg_kernel;     /* 0 (default): one cluster-persistent kernel runs all PCG
                           iterations of a Gauss-Newton step when the capture's
                           per-CTA data fits in shared memory, else one launch
                           per PCG phase; 1: one launch per PCG phase (J^T J p,
                           vector updates).  Either way the PCG vectors, the
                           J^T J p products and the dot products are carried as
                           compensated FP32 pairs (about 48 significant bits):
                           its iterate matches an FP64 CG on the FP32 operator
                           to ~1e-8 relative */
    float target_energy; /* 0 (default): run all n_gn steps.  > 0: the non-rigid
                           solve stops at the first step whose linearisation
                           energy is <= target_energy (the remaining steps are
                           skipped on the device; stats.n_gn_done counts the
                           updates made; the surface stage too) */
    /* per-vertex surface stage (lc_solve_surface), Sec. 3.4 regularisers.
     * The paper's weights (w_smooth 10, w_edge 30, w_velocity 0.25,
     * w_acceleration 0.1 beside w_photo 1e4) read with positions in
     * millimetres, rescaled to metres and to w_photo = 1: */
    float w_smooth;       /* default 1e3 */
    float w_edge;         /* default 3e3 */
    float w_velocity;     /* default 25 */
    float w_acceleration; /* default 10 */
    int n_gn_surface;     /* Gauss-Newton steps, default 3 (Sec. 4), <= LC_MAX_GN */
    int n_pcg_surface;    /* PCG iterations per step, default 4 (Sec. 4) */
    int pose_solver;      /* pose stage normal equations: 0 (default) mixed precision
                             (FP32 inverse by a symmetric sweep, FP64 residuals,
                             iterative refinement to 1e-10; the FP64 L D L^T when
                             that does not converge); 1: always the FP64 L D L^T */
    float lambda_temporal;  /* pose stage E_temporal (Sec. 3.3, Sec. 5: 1.5); active
                               once lc_pose_advance has recorded a frame */
    float lambda_anatomic;  /* pose stage E_anatomic (Sec. 5: 1e6); active for the
                               limits of lc_set_pose_priors */
    float sigma_c;          /* robust colour kernel of E_photo (Sec. 3.4): a visible
                               vertex whose colour difference ||I(pi(v)) - C|| (FP32,
                               Euclidean over RGB) exceeds sigma_c has its photometric
                               residual and rows zeroed at that linearisation
                               (LC_FLAG_PRUNED); 0 (default) = off */
    int pyr_levels;         /* photometric pyramid (Sec. 3.4): 0 (default) samples the raw
                               image.  1..3: level j = 0, 1, 2 (coarse to fine) is the
                               frame's RGB box-averaged over d x d blocks, d = 4, 2, 1
                               (ceil(W/d) x ceil(H/d) pixels, pixel centre at full-resolution
                               d x + (d-1)/2), then blurred by a separable Gaussian of
                               pyr_ksize[j] taps (sigma = 0.3((k-1)/2 - 1) + 0.8, rows first,
                               clamp to edge); Gauss-Newton step g samples level
                               min(3 - pyr_levels + g, 2), the energy after the last update
                               the finest.  Only E_photo samples it; the silhouette term
                               keeps the full-resolution distance transform. */
    int pyr_ksize[3];       /* Gaussian taps per level, odd, 1..31; default 15, 9, 3 */
    int pose_displacement;  /* 1: once lc_surface_advance has recorded a displacement, the pose
                               stage adds the skinned displacement d^S = Q(theta_start) dhat
                               (the recorded rest-pose displacement carried by the
                               dual-quaternion blend rotation of the frame's start pose) to
                               its skinned model for the silhouette term and the contour set
                               (Sec. 3.4, displacement warping); held fixed during the pose
                               solve.  0 (default): the plain skinned model */
    int gn_block;           /* with a target energy: the non-rigid solve's Gauss-Newton steps are
                               captured in blocks of gn_block steps; every block after the first
                               is a conditional graph node that runs only while the target is
                               not reached (the steps after the target inside a block return at
                               once).  0 (default): all n_gn steps unrolled */
    int graph_warp;         /* 1: displacement warping of the graph stage (the graph counterpart of
                               Sec. 3.4's warping) with a skeleton: lc_pose_advance records every
                               node's parameters in the rest pose through the dual-quaternion blend
                               rotation Q_k of its node vertex at the frame's final pose
                               (R^rest = Q^T R Q, t^rest = Q^T t), and the next pose solve ends by
                               posing them with the solved pose (R = Q R^rest Q^T, t = Q t^rest),
                               so the non-rigid stage starts from the previous frame's deformation
                               carried along with the bones; a record is dropped by
                               lc_pose_clear_history and by a new graph.  0 (default): off */
    int tma_taps;           /* 1: the linearisation of a single capture stages every vertex's 4 x 4
                               pixel patch of the frame (its bilinear taps and central differences,
                               Sec. 3.4 E_photo / E_silhouette) into shared memory with one TMA
                               bulk-tensor copy per vertex (cp.async.bulk.tensor, one mbarrier per
                               CTA, a bounded wait; LC_ERR_TIMEOUT from the next statistics read if
                               a wait ran out, the global loads being used then); vertices whose
                               patch leaves the frame, batched solves and pyramid levels use global
                               loads.  The same bits either way.  Default 1; 0: global loads */
} lc_params;

#define LC_MAX_GN 64

/* Per-solve statistics (FP64 energies: sums of squared residuals). */
typedef struct {
    double e_photo, e_sil, e_arap, e_total;  /* after the last update */
    double e_gn[LC_MAX_GN];                  /* total energy at each linearisation */
    double step_norm[LC_MAX_GN];             /* ||delta|| of each step */
    int pcg_iters[LC_MAX_GN];                /* PCG iterations actually run (pose stage: rounds of
                                                the mixed-precision refinement of each step's
                                                solve, -1 where the FP64 factorisation ran) */
    int n_gn_done;
    int n_visible;                           /* |V| photometric vertices */
    int n_boundary;                          /* |B| contour vertices */
    int n_boundary_neg;                      /* contour vertices with b_i = -1 */
    int pcg_breakdowns;                      /* steps whose PCG stopped on p^T A p <= 0 */
    int n_kernels;                           /* kernel nodes of the captured solve outside conditional bodies
                                                (all of them when no step is conditional) */
    int pcg_cluster_size;                    /* CTAs per cluster of the persistent PCG, 0 = per-phase kernels */
    double e_smooth, e_edge, e_velocity, e_acceleration;  /* surface stage terms (0 after a graph solve) */
    int n_kernels_step;                      /* kernel nodes of one conditional block of gn_block
                                                Gauss-Newton steps (0: the solve is unrolled) */
} lc_solve_stats;

/* Vertex flag bits returned by lc_read_visibility / lc_read_back. */
#define LC_FLAG_VISIBLE 1u   /* vertex in V (depth test passed) */
#define LC_FLAG_ONSIL 2u     /* vertex on a silhouette edge */
#define LC_FLAG_INB 4u       /* vertex in the contour set B */
#define LC_FLAG_BNEG 8u      /* b_i = -1 */
#define LC_FLAG_PRUNED 16u   /* photometric residual pruned by sigma_c at the last linearisation */
#define LC_FLAG_MASKED 32u   /* silhouette term off at the last linearisation: the vertex projects
                                onto another body part's region of the part mask */

/* ---- context ------------------------------------------------------------- */

/* Create a context on CUDA device `device`; `cuda_stream` is a cudaStream_t
 * that all work of the context is enqueued on.  0 = the context creates and
 * owns a non-blocking stream (the solve is captured as a CUDA graph, which
 * the legacy default stream does not allow).  *out receives the context. */
lc_status lc_create(lc_ctx **out, int device, void *cuda_stream);
/* Free the context and all its device memory.  Null is accepted. */
lc_status lc_destroy(lc_ctx *ctx);
/* Message of the first error seen by the context ("" if none). */
const char *lc_last_error(const lc_ctx *ctx);
/* Fill *p with the defaults listed at lc_params. */
lc_status lc_params_default(lc_params *p);
/* Replace the solver settings.  n_gn in [1, LC_MAX_GN], n_pcg >= 1. */
lc_status lc_set_params(lc_ctx *ctx, const lc_params *p);
/* Static pinhole camera (Sec. 3.2): focal length and principal point in
 * pixels, image size W x H (1 <= W, H <= 16384). */
lc_status lc_set_camera(lc_ctx *ctx, float f, float cx, float cy, int W, int H);

/* ---- template and graph --------------------------------------------------- */

/* Template mesh V^hat (Sec. 3.1): V N x 3 positions (metres), tris F x 3
 * vertex indices forming a closed or open 2-manifold (an edge shared by more
 * than two triangles is rejected with LC_ERR_ARG), albedo N x 3 in [0,1]
 * (per-vertex colours C), material N per-vertex non-rigidity weights
 * (Tab. 1; averaged per edge, Sec. 3.1).  Resets graph, skeleton and pose. */
lc_status lc_upload_template(lc_ctx *ctx, const float *V, int N, const int32_t *tris, int F,
                             const float *albedo, const float *material);

/* Build the embedded deformation graph on the device: n_nodes nodes by
 * farthest-point sampling (start vertex 0, lowest index on ties), each vertex
 * bound to its K nearest nodes (1 <= K <= 8, n_nodes >= K+1) with weights
 * (1 - d/d_max)^2 normalised, d_max the distance to the (K+1)-th nearest
 * node, and node edges to the 4 nearest other nodes (symmetrised) weighted by
 * the mean of the two nodes' material weights.  Node parameters are reset to
 * the identity. */
lc_status lc_build_graph(lc_ctx *ctx, int n_nodes, int K);

/* Upload a caller-built embedded deformation graph (Sec. 3.1) in place of
 * lc_build_graph, in the layout lc_read_graph returns: node_vid n (the
 * template vertex of each node, 0 <= v < N), bind_idx / bind_w N x K (each
 * vertex's K nodes and weights, finite and >= 0; the solver uses them as
 * given, without normalising), edge_off n+1 (CSR offsets of the directed
 * edges by source node, edge_off[0] = 0, non-decreasing), edge_dst E and
 * edge_s E (finite, >= 0: the ARAP weight of the pair).  The edge set must
 * be symmetric with equal weights both ways (the solver evaluates a pair's
 * two residuals from either node's out-edges), without self or duplicate
 * edges; edge_dst / edge_s may be null when E = 0.  1 <= K <= 8,
 * 1 <= n_nodes <= N.  Arrays may be host or device memory; they are copied
 * and checked on the host, and a violation returns LC_ERR_ARG and leaves
 * the previous graph in place.  Node parameters are reset to the identity.
 * Synchronises. */
lc_status lc_upload_graph(lc_ctx *ctx, int n_nodes, int K, const int32_t *node_vid, const int32_t *bind_idx,
                          const float *bind_w, const int32_t *edge_off, const int32_t *edge_dst,
                          const float *edge_s);

/* Copy the graph out.  node_vid n, bind_idx N x K, bind_w N x K,
 * edge_off n+1 (CSR offsets of the directed edges by source node),
 * edge_dst E, edge_s E.  Any pointer may be null to skip it; *n_edges (if
 * not null) receives E.  Synchronises. */
lc_status lc_read_graph(lc_ctx *ctx, int32_t *node_vid, int32_t *bind_idx, float *bind_w,
                        int32_t *edge_off, int32_t *edge_dst, float *edge_s, int *n_edges);

/* Node parameters: rotations node_R n x 9 (row-major 3x3) and translations
 * node_t n x 3.  Both null = reset to the identity. */
lc_status lc_set_node_params(lc_ctx *ctx, const float *node_R, const float *node_t);

/* Rest geometry V^S (N x 3) of the non-rigid stages: the skinned mesh of a
 * pose estimate made outside the library (lc_solve_pose sets it from its own
 * fit).  The graph nodes move with it (g_k = V^S of the node's vertex);
 * V^S = NULL restores the template. */
lc_status lc_set_rest_geometry(lc_ctx *ctx, const float *V_S);

/* ---- frame ---------------------------------------------------------------- */

/* One input frame (Sec. 3.2): rgb H x W x 3 in [0,1], dt H x W the Euclidean
 * distance transform of the foreground silhouette in pixels, mask H x W
 * foreground flags (non-zero = foreground).  joints2d (J x 2 pixels) and
 * joints3d (J x 3 metres) are the pose stage's detections (Sec. 3.3); both
 * may be null when no skeleton is used.  The images are repacked on the
 * device into one float4 (r, g, b, dt) per pixel.
 * dt = NULL: the distance transform is computed on the device from the mask,
 * exactly: the distance between pixel centres to the nearest contour pixel (a
 * foreground pixel with a 4-neighbour in the background or on the image
 * border), from integer squared distances (separable: the distance along
 * each column, then the minimum over the row's columns), rounded once to
 * FP32; 0 everywhere when the silhouette has no contour. */
lc_status lc_upload_frame(lc_ctx *ctx, const float *rgb, const float *dt, const uint8_t *mask,
                          const float *joints2d, const float *joints3d);

/* The frame as the solver samples it (inspection; synchronises): dt (H x W
 * floats, the uploaded or device-computed distance transform) and mask
 * (H x W, 0 / 1); either may be NULL. */
lc_status lc_read_frame(lc_ctx *ctx, float *dt, uint8_t *mask);
/* Level j (0 coarsest .. 2 finest) of the photometric pyramid of the current
 * frame (inspection; synchronises): rgb receives ceil(H/d) x ceil(W/d) x 3
 * floats (d = 4, 2, 1), W_out / H_out (nullable) its size.  LC_ERR_STATE
 * when pyr_levels is 0, no frame is loaded or level j is not among the
 * pyr_levels finest; LC_ERR_ARG for j outside 0..2. */
lc_status lc_read_pyramid_level(lc_ctx *ctx, int j, float *rgb, int *W_out, int *H_out);

/* ---- solve ---------------------------------------------------------------- */

/* Non-rigid stage (Sec. 3.4 and Sec. 4): from the current node parameters,
 * warp, find visibility and the contour set B once per frame, then n_gn
 * Gauss-Newton steps, each re-deciding b_i for B on the current surface and
 * solving J^T J delta = -J^T F by n_pcg iterations of
 * Jacobi-preconditioned CG from zero, then R_k <- Exp(d_omega_k) R_k,
 * t_k += d_t_k.  The whole sequence runs as one captured CUDA graph.
 * `stats` may be null; when given, the call synchronises and fills it. */
lc_status lc_solve_nonrigid(lc_ctx *ctx, lc_solve_stats *stats);
/* Statistics of the last lc_solve_nonrigid (as its `stats`).  Synchronises. */
lc_status lc_read_stats(lc_ctx *ctx, lc_solve_stats *stats);

/* Read the result.  node_R n x 9, node_t n x 3, V_out N x 3 (warped
 * vertices), flags N (LC_FLAG_* bits of the last visibility pass; BNEG as
 * last decided, at the final linearisation point),
 * pose N_DOF (pose parameters, see lc_upload_skeleton).  Null pointers are
 * skipped.  Synchronises. */
lc_status lc_read_back(lc_ctx *ctx, float *node_R, float *node_t, float *V_out, uint8_t *flags,
                       float *pose);

/* ---- inspection (each step of the solve, callable on its own) ------------- */

/* Warp with the current node parameters and recompute visibility, contour set
 * and b_i.  Enqueue only. */
lc_status lc_compute_visibility(lc_ctx *ctx);

/* zbuf H x W 64-bit keys (bits of the FP32 depth << 32 | triangle id; all
 * ones = empty), flags N, uv N x 2 projected positions of the visibility
 * pass.  After lc_solve_pose: the pose stage's decisions (z-buffer,
 * visibility and B at its starting pose; BNEG and uv at its final pose).
 * Null pointers are skipped.  Synchronises. */
lc_status lc_read_visibility(lc_ctx *ctx, uint64_t *zbuf, uint8_t *flags, float *uv);

/* Linearise at the current node parameters (visibility must exist; b_i of
 * the contour set is re-decided here, as in every Gauss-Newton step): warped
 * vertices v_warp N x 3, projections uv N x 2, per-vertex residuals
 * r_photo N x 3 (sqrt(w_p)(I - C), zero where inactive) and r_sil N
 * (sqrt(w_s) DT), per-vertex normal blocks H N x 6 (h00 h01 h02 h11 h12 h22
 * of A_i^T A_i, A_i = d r_i / d v'_i with the b_i sign) and e N x 3
 * (A_i^T r_i), energy 3 (photo, sil, arap).  The photometric term samples
 * the pyramid level of Gauss-Newton step 0 (level 3 - pyr_levels) when the
 * pyramid is on; sigma_c and the body-part mask apply as in a solve.  Null
 * pointers are skipped.  Synchronises. */
lc_status lc_eval_linearization(lc_ctx *ctx, float *v_warp, float *uv, float *r_photo,
                                float *r_sil, float *H, float *e, double *energy);

/* At the current linearisation: rhs 6n = -J^T F and diag 6n = diag(J^T J),
 * node-major (d_omega_x, d_omega_y, d_omega_z, d_t_x, d_t_y, d_t_z).
 * Synchronises. */
lc_status lc_eval_gradient(lc_ctx *ctx, float *rhs, float *diag);

/* out 6n = J^T J p at the current linearisation, p 6n (same layout).
 * Synchronises. */
lc_status lc_apply_jtj(lc_ctx *ctx, const float *p, float *out);

/* delta 6n = the PCG solution of J^T J delta = -J^T F at the current
 * linearisation (n_pcg iterations); iters (nullable) receives the number of
 * iterations run.  Node parameters are not changed.  Synchronises. */
lc_status lc_solve_linear(lc_ctx *ctx, float *delta, int *iters);

/* ---- skeletal pose stage (Sec. 3.3) --------------------------------------- */

/* Kinematic skeleton: J joints with parents (parent[0] = -1 is the root,
 * parents precede children), rest joint positions joints_rest J x 3, a DOF
 * flag per joint (dof[j] = 1: ball joint with 3 Euler angles XYZ; 0: fixed
 * end site; the root always has 6 DOF: left-multiplied rotation increment
 * and translation), and the LBS binding skin_idx N x 4 / skin_w N x 4.
 * The pose vector is [root axis-angle 3, root translation 3, 3 Euler angles
 * per DOF joint in joint order]; N_DOF = 6 + 3 * (number of DOF joints
 * excluding the root).  J <= 64. */
lc_status lc_upload_skeleton(lc_ctx *ctx, int J, const int32_t *parents, const float *joints_rest,
                             const uint8_t *dof, const int32_t *skin_idx, const float *skin_w);
/* Body-part mask of the silhouette term (Sec. 3.4, dense silhouette
 * alignment).  bone_part (J entries, host or device) gives the body part
 * (0..254) of each joint's bone; a vertex belongs to the part of its
 * heaviest skinning bone (the first of equal weights).  Then, once per frame
 * (at the frame decisions of lc_solve_nonrigid, lc_solve_surface,
 * lc_compute_visibility and lc_surface_visibility), the stage's rest geometry
 * V^S is rasterised (the exact rasteriser of the visibility pass) into a
 * label image, a covered pixel taking the label shared by two or three
 * vertices of its front triangle (else the first vertex's), and every part
 * grows into uncovered pixels within dilate_px pixels (Euclidean, pixel
 * centres): such a pixel takes torso_part if a torso pixel is within reach
 * (torso_part -1: no precedence), else the nearest part (the lower label on
 * equal distances).  At every linearisation a contour vertex whose pixel
 * (floor(u + 1/2), floor(v + 1/2)) carries another part's label has its
 * silhouette residual switched off (b_i = 0, LC_FLAG_MASKED).  bone_part
 * NULL switches the mask off.  Needs a skeleton (LC_ERR_STATE); labels above
 * 254, torso_part outside -1..254 or dilate_px outside 0..32: LC_ERR_ARG.
 * In an lc_batch solve each member with a mask builds it in the same way.
 * Synchronises. */
lc_status lc_set_body_parts(lc_ctx *ctx, const int32_t *bone_part, int torso_part, int dilate_px);
/* Inspection of the mask of the last frame decisions (synchronises): mask
 * H x W labels (255 = no part) and vertex_part N; either may be NULL. */
lc_status lc_read_part_mask(lc_ctx *ctx, uint8_t *mask, uint8_t *vertex_part);
/* Set the pose vector (N_DOF values) the next pose solve starts from.
 * Synchronises. */
lc_status lc_set_pose(lc_ctx *ctx, const float *pose);
/* Restart from the pose last given to lc_set_pose (the rest pose if none):
 * a device-side copy, enqueue only, so a frame can be re-solved from the same
 * start without a host round trip. */
lc_status lc_reset_pose(lc_ctx *ctx);
/* Pose stage (Sec. 3.3; Sec. 4 pose estimation): from the current pose,
 * skin the template (linear blend skinning), take the contour set B of the
 * skinned mesh once, then n_gn_pose Gauss-Newton steps (each re-deciding b_i
 * on the current skinned surface) on
 *   lambda_2d |pi(o_j) - P2D_j|^2 + lambda_3d |o_j - P3D_j|^2
 *   + lambda_sil / |B| sum_B DT(pi(V_i))^2 + lambda_prior |theta - theta_start|^2
 * with a dense FP32 Jacobian, FP32 J^T J and an FP64 square-root-free
 * Cholesky (L D L^T) solve on the
 * device (a non-positive pivot returns LC_ERR_NUMERIC when stats are read).
 * Afterwards the skinned mesh becomes the rest geometry of the non-rigid
 * stage and the graph nodes move with it.  `stats` may be null (else the
 * call synchronises; e_gn / step_norm hold the history, e_total the final
 * energy, n_boundary |B|). */
lc_status lc_solve_pose(lc_ctx *ctx, lc_solve_stats *stats);

/* Pose-stage regularisers and frame bookkeeping (Sec. 3.3).
 *   E_temporal = lambda_temporal sum_j w_j ||o_j - o_j^{t-1}||^2 on the joint
 *     positions, against the joints recorded by lc_pose_advance (off until a
 *     frame is recorded); 3 residual rows per joint, like the 3D joints.
 *   E_anatomic = lambda_anatomic sum_c Psi(theta_c), Psi(x) = (x - max)^2
 *     above the limit, (min - x)^2 below, 0 inside, on the Euler angles; in
 *     Gauss-Newton a residual sqrt(lambda)(theta - bound) on the angles
 *     outside their limits at each linearisation.
 * lc_set_pose_priors: per-joint weights w (J floats, NULL = 1 each) and the
 *   limits theta_min / theta_max (n_dof floats each in the layout of the pose
 *   vector, the 6 root entries ignored; both NULL = no limits).
 *   Synchronises.
 * lc_pose_advance: end of a frame: the current joints become the previous
 *   frame's, and the current pose enters a two-frame history.  Enqueued.
 * lc_pose_extrapolate: start of a frame: the pose (and the prior's centre at
 *   the next solve) becomes the explicit Euler step from the last two
 *   recorded poses, theta = 2 theta^{t-1} - theta^{t-2} for the Euler angles
 *   and the root translation, R = R^{t-1} (R^{t-2})^T R^{t-1} for the root
 *   rotation; with one recorded pose, that pose.  LC_ERR_STATE without a
 *   recorded pose.  Enqueued.
 * lc_pose_clear_history: forgets the recorded frames. */
lc_status lc_set_pose_priors(lc_ctx *ctx, const float *temporal_w, const float *theta_min, const float *theta_max);
lc_status lc_pose_advance(lc_ctx *ctx);
lc_status lc_pose_extrapolate(lc_ctx *ctx);
lc_status lc_pose_clear_history(lc_ctx *ctx);
/* Inspection: at the current pose, recompute B and b_i and export the pose
 * normal equations: V_skinned N x 3 (FP32 skinned template, plus the skinned
 * displacement when pose_displacement applies), A n_dof x n_dof
 * (J^T J + prior), g n_dof (-J^T F - prior gradient), energy 1.  Null
 * pointers are skipped.  Synchronises. */
lc_status lc_eval_pose(lc_ctx *ctx, float *V_skinned, double *A, double *g, double *energy);

/* ---- batches: many captures per launch (Sec. 4 solver, batched) ---------- */

/* A batch solves the non-rigid stage of several contexts together: one
 * launch per phase for all captures (their work lists concatenated), the
 * whole Gauss-Newton / PCG loop captured as one CUDA graph on the batch's own
 * stream.  Every member keeps its own buffers and reductions, so each
 * capture's result equals its single-context lc_solve_nonrigid with the same
 * PCG kernel and cluster size.  Members must be on one device, fully set up
 * (template, graph, camera, frame) and agree in n_gn and n_pcg.  Frames and
 * node parameters may change between solves (a member whose buffers were
 * reallocated makes the next solve rebuild the plan).  The pose stage is not
 * batched: run lc_solve_pose per context first. */
typedef struct lc_batch lc_batch;
typedef struct lc_mlp lc_mlp;   /* the warm-start network, below */

/* PCG strategy of a batch: */
#define LC_BATCH_PCG_AUTO 0           /* each capture as on its own (smallest cluster that fits,
                                         else the batched per-iteration kernels) */
#define LC_BATCH_PCG_CLUSTER8 1       /* 8-CTA clusters where they fit, else per-iteration kernels */
#define LC_BATCH_PCG_CLUSTER16 2      /* 16-CTA clusters where they fit, else per-iteration kernels */
#define LC_BATCH_PCG_PER_ITERATION 3  /* per-iteration kernels for every capture, batched */

/* ctxs: count >= 1 context handles (the caller keeps ownership; they must
 * outlive the batch).  LC_ERR_STATE if a member is not ready, LC_ERR_ARG if
 * they differ in device, n_gn or n_pcg (message in the first context). */
lc_status lc_batch_create(lc_batch **out, lc_ctx *const *ctxs, int count);
lc_status lc_batch_destroy(lc_batch *batch);
const char *lc_batch_last_error(const lc_batch *batch);
/* Choose the PCG strategy (LC_BATCH_PCG_*); rebuilds the work lists.
 * Synchronises. */
lc_status lc_batch_set_pcg_mode(lc_batch *batch, int mode);
/* One non-rigid solve of every member (from the identity deformation when
 * from_identity != 0, else from each member's current node parameters).
 * The solve waits for work already enqueued on the members' streams, and
 * their later calls wait for the solve.  Enqueue only when stats is null;
 * else synchronises and fills stats[i] for member i (caller order). */
lc_status lc_batch_solve(lc_batch *batch, int from_identity, lc_solve_stats *stats);
/* Autotuner: times `reps` solves (from the identity) under each PCG strategy
 * on the members' current frames, keeps the fastest and returns it in
 * *mode_out; ms_out (nullable, 4 entries indexed by LC_BATCH_PCG_*) receives
 * the mean milliseconds per solve of each.  Synchronises. */
lc_status lc_batch_autotune(lc_batch *batch, int reps, int *mode_out, float *ms_out);

/* Launch shape of a batch: the PCG strategy (LC_BATCH_PCG_*) and, for the
 * captures that run the per-iteration J^T J p (not on a cluster), its
 * vertex-phase block (vert_block: 128, 256 or 512 vertices), its node-phase
 * block (node_warps: 4, 8 or 16 warps of 4 nodes, 8 lanes per node; default
 * 4) and the node phase's entry rounds in flight per lane (node_unroll: 2, 4
 * or 8).  Under one PCG strategy every shape gives bit-identical results:
 * the vertex phase is per vertex, each lane of a node's group takes the
 * node's entries in the same order, and p.A p is summed per group of 8
 * nodes in the same tree.  lc_batch_set_shape
 * rebuilds the plan (LC_ERR_ARG for another value); lc_batch_get_shape
 * reads it. */
typedef struct {
    int pcg_mode;
    int vert_block;
    int node_warps;
    int node_unroll;
} lc_batch_shape;
lc_status lc_batch_set_shape(lc_batch *batch, const lc_batch_shape *shape);
lc_status lc_batch_get_shape(const lc_batch *batch, lc_batch_shape *shape);
/* The autotuner over shapes: for every PCG strategy, every shape where any
 * capture runs the per-iteration J^T J p (else the one default shape): a
 * solve from the identity, its members' node parameters and energy
 * histories compared with the strategy's first shape (a shape whose bits
 * differ is rejected and counted), then reps timed solves from the identity.
 * The fastest shape is set and stored in a process-wide table under the
 * batch's size class (lc_batch_size_class); with use_cache and an entry for
 * the class, that entry is set without timing (*from_cache = 1).  Outputs
 * are nullable.  The members' node parameters are left at a solve from the
 * identity. */
lc_status lc_batch_autotune_shapes(lc_batch *batch, int reps, int use_cache, lc_batch_shape *best, float *best_ms,
                                   int *from_cache, int *n_tried, int *n_rejected);
/* Size class of a batch: per member (K, ceil log2 of its vertices, ceil
 * log2 of its nodes), sorted with multiplicities ("K4.N12.n9x3,...");
 * LC_ERR_ARG if it does not fit in len bytes. */
lc_status lc_batch_size_class(const lc_batch *batch, char *key, int len);
/* The table as text, one line per size class: "class<TAB>pcg_mode vert_block
 * node_warps node_unroll ms"; *needed receives the size with the final NUL
 * (text may be null to ask for it).  _load merges such text into the table
 * (LC_ERR_ARG for a malformed line; nothing is merged then). */
lc_status lc_autotune_table(char *text, int len, int *needed);
lc_status lc_autotune_table_load(const char *text);
/* The batch's CUDA stream (a cudaStream_t), for ordering and timing. */
void *lc_batch_stream(const lc_batch *batch);
/* One matrix-free J^T J p of every member in one launch pair (vertex phase,
 * node phase), at each member's current linearisation with p = its PCG
 * direction, result into its A p buffer: the metric kernel on its own, for
 * measurement.  stage != 0 first recomputes the rotated offsets it reads
 * (once per linearisation in a solve); stage == 0 reuses them.  Requires a
 * previous lc_batch_solve.  Enqueue only. */
lc_status lc_batch_apply_jtj(lc_batch *batch, int stage);

/* One frame step of every member as one CUDA graph (Sec. 3.3-3.4, the
 * per-frame sequence of a tracked stream): per member the pose solve
 * (lc_solve_pose), started from the explicit Euler step (lc_pose_extrapolate)
 * with LC_STEP_EULER_START, else from the member's last solved pose; unless
 * LC_STEP_CARRY_GRAPH, the node parameters reset to the identity over the new
 * skinned surface followed by lc_record_motion (so that the motion recorded
 * after the solve is the frame's update from that start); with a network
 * (non-null), the warm start (lc_warm_start: prediction kept iff the energy
 * does not rise, frame decisions of the start kept); then the non-rigid
 * stage of all members in one launch per phase from their current
 * parameters (lc_batch_solve with from_identity = 0); then per member
 * lc_record_motion and lc_pose_advance.
 * Each member must have a skeleton, a frame uploaded for this step and two
 * recorded frames (two lc_pose_advance calls, so that the pose history no
 * longer changes on the host), else LC_ERR_STATE; profiling must be off.
 * Other flag bits: LC_ERR_ARG.  The graph is captured on the first call and
 * again when the members' descriptors, the network or the flags change; the result is that of the calls above
 * made one after the other.  stats (nullable, one per member in caller
 * order: the non-rigid stage's statistics) makes the call synchronise. */
#define LC_STEP_EULER_START 1u
#define LC_STEP_CARRY_GRAPH 2u
lc_status lc_batch_step(lc_batch *batch, lc_mlp *mlp, unsigned flags, lc_solve_stats *stats);

/* ---- learned warm start (the project's addition to the paper's solver) ---- */

/* The paper starts each frame's non-rigid solve from the previous frame's
 * result (Sec. 3.4, Sec. 4).  A small network predicts every graph node's
 * update (d_omega, d_t) from features pooled at that start, so that the
 * Gauss-Newton iteration starts closer; the prediction is kept only if the
 * energy at the predicted parameters does not exceed the energy at the start.
 *
 * Network: x = (f - mu) / sigma (per feature), h1 = relu(x W1 + b1),
 * h2 = relu(h1 W2 + b2), y = (h2 W3 + b3) * s_out (per output), sizes
 * 64 -> 256 -> 256 -> 6; the contractions run on the tcgen05 tensor cores
 * (one CTA per 128 x 256 tile, shared-memory operands, tensor-memory
 * accumulator; a bounded wait that runs out is reported as LC_ERR_TIMEOUT by
 * the next synchronising lc_mlp_* call) or, selected by lc_mlp_set_gemm, on
 * mma.sync;
 * BF16 weights and activations, FP32 accumulation (tensor cores), FP32
 * master parameters.  Parameter vector (LC_MLP_PARAMS floats): W1 row-major
 * 64 x 256, b1 256, W2 256 x 256, b2 256, W3 256 x 6, b3 6.  Loss over M
 * rows: (1/M) sum ||y - t||^2.
 *
 * Node features (64 per node), at the current node parameters, pooled over
 * the node's bound vertices with their binding weights w (W = sum w; a
 * pooled value is 0 when W = 0) from the linearisation there:
 *   0-2 Log(R_k)   3-5 t_k   6-11 -(J^T F)_k   12-17 diag(J^T J)_k
 *   18-23 (-(J^T F)_k) / (diag_k + 1e-6 max(diag_k))
 *   24-26 sum w r_photo / W   27-29 sum w |r_photo| / W
 *   30 sum w r_sil / W   31 sum w r_sil^2 / W
 *   32-34 sum w e / W   35-37 sum w |e| / W   (e = A_i^T r_i)
 *   38-43 sum w H / W   (H = A_i^T A_i: h00 h01 h02 h11 h12 h22)
 *   44 sum w [visible] / W   45 sum w [in B] / W   46 sum w [b = -1] / W   47 W
 *   48-50 g_k   51-56 u_k: the node's motion over the last frame (lc_record_motion)
 *   57-62 mean u_l over the node's graph neighbours   63 1 */
#define LC_MLP_PARAMS 83974

/* params (LC_MLP_PARAMS, null = zeros), mu / sigma (64 each, null = 0 / 1;
 * sigma <= 0 is treated as 1): host or device. */
lc_status lc_mlp_create(lc_mlp **out, int device, const float *params, const float *mu, const float *sigma);
lc_status lc_mlp_destroy(lc_mlp *mlp);
const char *lc_mlp_last_error(const lc_mlp *mlp);
/* Current FP32 parameters (LC_MLP_PARAMS).  Synchronises. */
lc_status lc_mlp_get_params(lc_mlp *mlp, float *params);
/* Tensor-core path of the network's contractions: LC_GEMM_TCGEN05 (default)
 * or LC_GEMM_MMA_SYNC; both accumulate in FP32 (the order of the sums
 * differs).  Synchronises. */
#define LC_GEMM_TCGEN05 0
#define LC_GEMM_MMA_SYNC 1
lc_status lc_mlp_set_gemm(lc_mlp *mlp, int kind);
/* The network's input normalisation mu / sigma (64 each) and output scale
 * s_out (6; 1 after lc_mlp_create).  Each pointer is nullable (that part is
 * left as is or not read) and may be host or device.  Synchronises. */
lc_status lc_mlp_set_scaling(lc_mlp *mlp, const float *mu, const float *sigma, const float *s_out);
lc_status lc_mlp_get_scaling(lc_mlp *mlp, float *mu, float *sigma, float *s_out);
/* Fit the scaling to training rows, on the device: mu_j / sigma_j = mean and
 * population standard deviation of feature column j of F (rows x 64; sigma
 * 1 where below 1e-12, and feature 63, the constant, keeps mu 0 and sigma 1);
 * s_out_c = root mean square of target column c of T (rows x 6; 1 where
 * below 1e-12), so that the layers fit targets of unit scale.  Moments are
 * accumulated in FP64 in a fixed order, shifted by the first row (exact for
 * a constant column).  F and T must be device arrays (LC_ERR_ARG
 * otherwise).  Synchronises. */
lc_status lc_mlp_fit_scaling(lc_mlp *mlp, const float *F, const float *T, long long rows);
/* Y (M x 6) for raw features F (M x 64).  Synchronises. */
lc_status lc_mlp_forward(lc_mlp *mlp, const float *F, int M, float *Y);
/* Loss and its gradient (LC_MLP_PARAMS, nullable) for features F (M x 64)
 * and targets T (M x 6).  Synchronises. */
lc_status lc_mlp_gradient(lc_mlp *mlp, const float *F, const float *T, int M, float *grad, double *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
 * rows idx[0..B) (host or device) of the device arrays F (rows x 64) and
 * T (rows x 6).  Enqueue only unless loss (nullable) is requested. */
lc_status lc_mlp_train_step(lc_mlp *mlp, const float *F, const float *T, const int *idx, int B, float lr,
                            double *loss);

/* Features (n x 64) at the current node parameters and the frame decisions
 * of the last visibility pass.  Synchronises. */
lc_status lc_node_features(lc_ctx *ctx, float *F);
/* Record the motion of every node since the previous call (or since the
 * graph was built): u_k = (Log(R_k R_prev,k^T), t_k - t_prev,k).  Call once
 * per frame after its solve.  Enqueue only. */
lc_status lc_record_motion(lc_ctx *ctx);
/* The motion recorded by the last lc_record_motion, n x 6 floats per node
 * (Log(R R_prev^T), t - t_prev), into u (host or device).  Called after a
 * frame's solve and its lc_record_motion it is the update that solve made
 * from the frame's start: the warm start's training target.  LC_ERR_STATE
 * if nothing was recorded for the current graph.  Synchronises. */
lc_status lc_read_motion(lc_ctx *ctx, float *u);
/* Warm start at the current node parameters (normally the previous frame's
 * result): visibility, linearisation and features there; the network's
 * update applied to every node (R <- Exp(d_omega) R, t += d_t); kept iff
 * the energy at the predicted parameters (same frame decisions) is <= the
 * energy at the start, else the start parameters are restored - all on the
 * device.  The next lc_solve_nonrigid keeps the frame decisions taken at
 * the start (visibility and the contour set are not recomputed at the
 * predicted parameters), so its energies compare with those of a solve from
 * the start.  accepted (nullable) receives 1/0 and energies (nullable, 2)
 * the two energies; either makes the call synchronise. */
lc_status lc_warm_start(lc_ctx *ctx, lc_mlp *mlp, int *accepted, double *energies);

/* ---- per-vertex surface stage (the paper's own non-rigid unknowns) ---------
 *
 * Sec. 3.4 poses the non-rigid stage over the vertex positions V (N x 3):
 *   E(V) = E_photo + E_silhouette + E_smooth + E_edge + E_velocity + E_acceleration
 *   E_smooth       = w_smooth sum_i sum_{j in N_i} s_ij/|N_i| ||(V_i - V_j) - (V^S_i - V^S_j)||^2
 *   E_edge         = w_edge   sum_i sum_{j in N_i} s_ij/|N_i| (||V_i - V_j|| - ||Vh_i - Vh_j||)^2
 *   E_velocity     = w_velocity     sum_i ||V_i - V^{t-1}_i||^2
 *   E_acceleration = w_acceleration sum_i ||V_i - 2 V^{t-1}_i + V^{t-2}_i||^2
 * N_i is the one-ring of vertex i (vertices sharing a mesh edge), s_ij the
 * mean of the two vertices' material weights (Sec. 3.1), V^S the stage's rest
 * geometry (the skinned mesh after lc_solve_pose, else the template), Vh the
 * template.  The data terms are the graph stage's (same visibility, contour
 * set and b_i rules) evaluated at V_i.  Sec. 4: Gauss-Newton, n_gn_surface
 * steps of n_pcg_surface Jacobi-PCG iterations from 0, one thread per vertex
 * block row gathering its one-ring (no atomics), V <- V + delta.
 * Temporal history: none -> both temporal terms off; one previous frame ->
 * V^{t-2} = V^{t-1}.  The surface state exists once a template is uploaded;
 * the surface calls need no graph.  A new template clears the history. */

/* The current surface V (N x 3 floats): the unknowns and the start of the
 * next lc_solve_surface. */
lc_status lc_set_surface(lc_ctx *ctx, const float *V);
/* Start of a frame (Sec. 3.4, displacement warping): V <- V^S + d^S, where
 * d^S is the displacement recorded by the last lc_surface_advance carried
 * from that frame's pose to the current one: d^S_i = Q_i dh_i with dh_i the
 * recorded rest-pose displacement and Q_i the rotation of the dual-quaternion
 * blend of vertex i's bone rotations (skinning weights of lc_upload_skeleton;
 * Q_i = I without a skeleton).  Without a recorded displacement V <- V^S.
 * Enqueued, no synchronisation. */
lc_status lc_surface_start(lc_ctx *ctx);
/* Temporal history V^{t-1}, V^{t-2} (N x 3 each).  V_prev = NULL clears the
 * history; V_prev2 = NULL sets V^{t-2} = V^{t-1}. */
lc_status lc_surface_history(lc_ctx *ctx, const float *V_prev, const float *V_prev2);
/* End of a frame: V^{t-2} <- V^{t-1}, V^{t-1} <- V, and the rest-pose
 * displacement dh_i = Q_i^T (V_i - V^S_i) is recorded for lc_surface_start.
 * Enqueued, no synchronisation. */
lc_status lc_surface_advance(lc_ctx *ctx);
/* One frame of the surface stage from the current V: frame decisions (V, B,
 * b_i) at the start, n_gn_surface Gauss-Newton steps, final energy.  Needs
 * template, camera and frame.  Captured once as a CUDA graph.  stats
 * (nullable; filling it synchronises): e_photo, e_sil and the four
 * regulariser energies after the last update, e_total their sum, e_gn the
 * total at each linearisation; e_arap = 0. */
lc_status lc_solve_surface(lc_ctx *ctx, lc_solve_stats *stats);
/* Surface read-back (synchronises): V (N x 3, nullable), flags (N, nullable:
 * LC_FLAG_* of the last frame decisions). */
lc_status lc_read_surface(lc_ctx *ctx, float *V, uint8_t *flags);

/* Inspection (each synchronises).  lc_surface_visibility: the frame
 * decisions at the current V (lc_read_visibility returns them).
 * lc_surface_linearize: at the current V with those decisions (b_i
 * re-evaluated; the pyramid level of Gauss-Newton step 0, sigma_c and the
 * body-part mask as in a solve), rhs = -J^T F (N x 3), diag = diag(J^T J) (N x 3) and
 * energies[6] = photo, silhouette, smooth, edge, velocity, acceleration;
 * any output may be NULL.  lc_surface_apply_jtj: out = J^T J p (N x 3) at
 * that linearisation.  lc_surface_solve_linear: n_pcg_surface Jacobi-PCG
 * iterations on it from 0 (delta N x 3, iters = iterations run). */
lc_status lc_surface_visibility(lc_ctx *ctx);
lc_status lc_surface_linearize(lc_ctx *ctx, float *rhs, float *diag, double *energies);
lc_status lc_surface_apply_jtj(lc_ctx *ctx, const float *p, float *out);
lc_status lc_surface_solve_linear(lc_ctx *ctx, float *delta, int *iters);

/* ---- profiling ------------------------------------------------------------ */

/* Phases of the non-rigid solve, for lc_read_profile. */
#define LC_PH_WARP 0      /* warp + projection */
#define LC_PH_VIS 1       /* z-buffer, visibility, contour set, b_i */
#define LC_PH_LIN 2       /* residuals and per-vertex normal blocks */
#define LC_PH_RHS 3       /* -J^T F, Jacobi diagonal, ARAP energy */
#define LC_PH_PCG_INIT 4  /* PCG start vectors */
#define LC_PH_JTJ 5       /* matrix-free J^T J p */
#define LC_PH_PCG_VEC 6   /* PCG vector updates and FP64 dots */
#define LC_PH_UPDATE 7    /* rotation / translation update */
#define LC_PH_POSE 8      /* pose stage: the rest (start-pose copy, final skinning into V^S) */
#define LC_PH_PCG 9       /* cluster-persistent PCG (all iterations of one step) */
#define LC_PH_POSE_VIS 10   /* pose stage: kinematics, skinning, visibility and contour set at the start */
#define LC_PH_POSE_SYS 11   /* pose stage: skinning, b_i and the residual rows reduced to J^T J (per step) */
#define LC_PH_POSE_SOLVE 12 /* pose stage: FP64 normal equations, L D L^T solve, update (per step) */
#define LC_N_PHASES 13

/* Profiling on (1) or off (0).  When on, the captured solves record a chain
 * of CUDA events on the context stream between consecutive phases, so each
 * phase's device time of the last solve can be read with lc_read_profile.
 * The event nodes add a little launch overhead; keep it off for throughput
 * runs.  Changing it re-captures the solve. */
lc_status lc_set_profiling(lc_ctx *ctx, int on);
/* Device time in milliseconds (ms[LC_N_PHASES]) and number of timed
 * segments (count[LC_N_PHASES], nullable) per phase of the last solves since
 * profiling was switched on or last read; reading resets the sums.
 * Synchronises. */
lc_status lc_read_profile(lc_ctx *ctx, double *ms, int *count);

/* ---- visibility without device allocation --------------------------------- */

/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory when they need visibility: code running
 * inside another framework's memory pool that forbids outside allocations,
 * a real-time process whose device memory is reserved up front, or a plugin
 * that may not grow its host application's footprint.
 *
 * Per-vertex visibility of warped vertices V_warp (N x 3, metres) of the
 * mesh tris (F x 3) under the pinhole camera (f, cx, cy, W x H), with depth
 * tolerance eps_vis: visible[i] = 1 or 0, bit-identical to the
 * LC_FLAG_VISIBLE bit of lc_compute_visibility for the same positions.
 * V_warp, tris and visible must be device memory of the current device;
 * work is enqueued on cuda_stream (a cudaStream_t, 0 = legacy default) and
 * the call returns without waiting.  Triangles naming a vertex outside
 * [0, N) are skipped.
 *
 * No device memory is allocated, on any path: the z-buffer scratch is a
 * static device array of LC_NOALLOC_MAX_PIXELS 64-bit entries (8 MiB) that
 * every GPU which loads this library holds until the process exits.  W * H
 * above LC_NOALLOC_MAX_PIXELS returns LC_ERR_ARG; host pointers, memory of
 * another device and a negative or NaN eps_vis return LC_ERR_ARG.  The
 * first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, which may load the module):
 * make that first call outside any stream capture.  All calls share the
 * scratch, each clearing what it uses first; calls that overlap on the GPU
 * race on it, so serialise them (one stream, or explicit ordering). */
#define LC_NOALLOC_MAX_PIXELS (1024 * 1024)
lc_status lc_visibility_noalloc(const float *V_warp, int N, const int32_t *tris, int F, float f, float cx,
                                float cy, int W, int H, float eps_vis, uint8_t *visible, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LIVECAP_H */

// Skeletal pose stage (Sec. 3.3; Sec. 4, pose estimation) on the device.
//
// Pose vector: [root rotation increment (3), root translation (3), Euler XYZ
// angles of every DOF joint (3 each)].  The root rotation is kept as a matrix
// and updated on the left, R <- Exp(d_omega) R; everything else adds.
//
//   forward kinematics: o_root = t, G_root = R; o_j = o_p + G_p (J_j - J_p),
//     G_j = G_p Rx(a) Ry(b) Rz(c) (end sites: G_j = G_p)
//   skinning: V^S_i = sum_s w_is (G_b (V_i - J_b) + o_b), b = bone of slot s
//   residual rows: 2D joints sqrt(l2D)(pi(o_j) - P2D_j), 3D joints
//     sqrt(l3D)(o_j - P3D_j), silhouette sqrt(lsil/|B|) DT(pi(V^S_i)) for the
//     contour set B of the start pose (Jacobian row times b_i), and the angle
//     prior lprior (theta - theta_start) added to the normal equations
//   Jacobian of a point P riding on bone b: root d_omega -> e x (P - t),
//     root t -> I, Euler axis u of an ancestor-or-self joint j of b ->
//     u x (P - o_j), with u_a = G_p e_x, u_b = G_p Rx e_y, u_c = G_p Rx Ry e_z.
//
// Per Gauss-Newton step: forward kinematics once (one CTA, joints of a tree
// level in parallel) into a global table; skinning and b_i of the contour
// set; the residual rows built in shared memory by a grid of CTAs, each
// reducing its rows to FP32 partial sums of the pairs of [J | F] columns; one
// CTA summing the partials in a fixed order into the FP64 normal equations,
// solving them to FP64 accuracy (an FP32 inverse refined with FP64
// residuals, or an FP64 L D L^T whose pivot <= 0 sets a status word),
// updating the pose and computing the next forward kinematics - no host round
// trip.
#include "lc_internal.cuh"
#include "pose_internal.h"

namespace lc {

__device__ __forceinline__ void mat3mul(const float* A, const float* B, float* C) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

// Forward kinematics of the whole skeleton at the current pose into fk, by
// the calling CTA: thread j handles joint j, one tree level at a time (the
// parent's frame is final before its children read it).  Every thread of
// the CTA must call this (it synchronises).
__device__ void forward_kinematics(const PoseDesc& P, PoseFk& fk) {
    // the joint's local rotation L = Rx(a) Ry(b) Rz(c) and its Euler axes in
    // the parent frame (e_x, Rx e_y, Rx Ry e_z) first, for every joint at once;
    // then the tree level by level: G_j = G_p L, U_j = G_p [axes],
    // o_j = o_p + G_p (J_j - J_p)
    const int j = threadIdx.x;
    const float* pose = P.pose;
    float L[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    float Ax[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};   // columns: the three axes
    int p = -1, lvl_j = -1, c = -1;
    float d[3] = {0.f, 0.f, 0.f};
    if (j < P.J) {
        p = P.parents[j];
        lvl_j = P.level[j];
        c = P.col[j];
        if (p >= 0) {
            const float4 rj = P.rest[j], rp = P.rest[p];
            d[0] = rj.x - rp.x;
            d[1] = rj.y - rp.y;
            d[2] = rj.z - rp.z;
        }
        if (p >= 0 && c >= 0) {
            float sa, ca, sb, cb, sc, cc;
            sincosf(pose[c], &sa, &ca);
            sincosf(pose[c + 1], &sb, &cb);
            sincosf(pose[c + 2], &sc, &cc);
            const float Rx[9] = {1.f, 0.f, 0.f, 0.f, ca, -sa, 0.f, sa, ca};
            const float Ry[9] = {cb, 0.f, sb, 0.f, 1.f, 0.f, -sb, 0.f, cb};
            const float Rz[9] = {cc, -sc, 0.f, sc, cc, 0.f, 0.f, 0.f, 1.f};
            float RxRy[9];
            mat3mul(Rx, Ry, RxRy);
            mat3mul(RxRy, Rz, L);
            // axes as columns: e_x, Rx e_y, Rx Ry e_z
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                Ax[3 * r] = r == 0 ? 1.f : 0.f;
                Ax[3 * r + 1] = Rx[3 * r + 1];
                Ax[3 * r + 2] = RxRy[3 * r + 2];
            }
        }
    }
    for (int lvl = 0; lvl < P.n_levels; ++lvl) {
        if (lvl_j == lvl) {
            if (p < 0) {
#pragma unroll
                for (int q = 0; q < 9; ++q) fk.G[j][q] = P.Rroot[q];
                fk.o[j][0] = pose[3];
                fk.o[j][1] = pose[4];
                fk.o[j][2] = pose[5];
            } else {
                float Gp[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) Gp[q] = fk.G[p][q];
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    fk.o[j][r] = fk.o[p][r] + Gp[3 * r] * d[0] + Gp[3 * r + 1] * d[1] + Gp[3 * r + 2] * d[2];
                float G[9];
                if (c < 0) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) G[q] = Gp[q];
                } else {
                    mat3mul(Gp, L, G);
                    float U[9];
                    mat3mul(Gp, Ax, U);
                    // fk.U[j]: rows x, y, z of each axis: U[j][3 a + r] = (G_p axis_a)_r
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        fk.U[j][r] = U[3 * r];
                        fk.U[j][3 + r] = U[3 * r + 1];
                        fk.U[j][6 + r] = U[3 * r + 2];
                    }
                }
#pragma unroll
                for (int q = 0; q < 9; ++q) fk.G[j][q] = G[q];
            }
        }
        __syncthreads();
    }
}

// the global kinematics table -> shared memory (G and o; U when asked)
__device__ __forceinline__ void load_fk(const PoseDesc& P, PoseFk& fk, bool axes) {
    const int J = P.J;
    const float* gG = &P.fk->G[0][0];
    const float* go = &P.fk->o[0][0];
    const float* gU = &P.fk->U[0][0];
    for (int q = threadIdx.x; q < 9 * J; q += blockDim.x) (&fk.G[0][0])[q] = gG[q];
    for (int q = threadIdx.x; q < 3 * J; q += blockDim.x) (&fk.o[0][0])[q] = go[q];
    if (axes)
        for (int q = threadIdx.x; q < 9 * J; q += blockDim.x) (&fk.U[0][0])[q] = gU[q];
}

__device__ __forceinline__ void cross3f(const float* a, const float* b, float* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Adds w * coef . dP/dtheta (P riding on bone b) into row[0..n_dof).
__device__ __forceinline__ void add_point_row(const PoseDesc& P, const PoseFk& fk, const float* pt, int b,
                                              const float* coef, float w, float* row) {
    const float t[3] = {P.pose[3], P.pose[4], P.pose[5]};
    const float rel[3] = {pt[0] - t[0], pt[1] - t[1], pt[2] - t[2]};
    // root rotation: e_a x rel  ->  coef . (e_a x rel) = (rel x coef)_a
    float rc[3];
    cross3f(rel, coef, rc);
    row[0] += w * rc[0];
    row[1] += w * rc[1];
    row[2] += w * rc[2];
    row[3] += w * coef[0];
    row[4] += w * coef[1];
    row[5] += w * coef[2];
    unsigned long long m = P.anc[b];
    while (m) {
        const int j = __ffsll((long long)m) - 1;
        m &= m - 1;
        const int c = P.col[j];
        if (c < 0) continue;
        const float r2[3] = {pt[0] - fk.o[j][0], pt[1] - fk.o[j][1], pt[2] - fk.o[j][2]};
        float rc2[3];
        cross3f(r2, coef, rc2);   // coef . (u x r2) = u . (r2 x coef)
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const float* u = &fk.U[j][3 * ax];
            row[c + ax] += w * (u[0] * rc2[0] + u[1] * rc2[1] + u[2] * rc2[2]);
        }
    }
}

__device__ __forceinline__ float4 dt_sample(const CapDesc& C, float u, float v, float& gx, float& gy) {
    // bilinear DT and central-difference gradient (one-sided at the border)
    const int x0 = (int)floorf(u), y0 = (int)floorf(v);
    const float fx = u - (float)x0, fy = v - (float)y0;
    const int x1 = min(x0 + 1, C.W - 1), y1 = min(y0 + 1, C.H - 1);
    auto D = [&](int x, int y) { return __ldg(&C.img[(size_t)y * C.W + x]).w; };
    auto Gx = [&](int x, int y) {
        if (C.W < 2) return 0.f;
        if (x == 0) return D(1, y) - D(0, y);
        if (x == C.W - 1) return D(C.W - 1, y) - D(C.W - 2, y);
        return (D(x + 1, y) - D(x - 1, y)) * 0.5f;
    };
    auto Gy = [&](int x, int y) {
        if (C.H < 2) return 0.f;
        if (y == 0) return D(x, 1) - D(x, 0);
        if (y == C.H - 1) return D(x, C.H - 1) - D(x, C.H - 2);
        return (D(x, y + 1) - D(x, y - 1)) * 0.5f;
    };
    auto lerp = [](float a, float b, float t) { return a + t * (b - a); };
    const float d = lerp(lerp(D(x0, y0), D(x1, y0), fx), lerp(D(x0, y1), D(x1, y1), fx), fy);
    gx = lerp(lerp(Gx(x0, y0), Gx(x1, y0), fx), lerp(Gx(x0, y1), Gx(x1, y1), fx), fy);
    gy = lerp(lerp(Gy(x0, y0), Gy(x1, y0), fx), lerp(Gy(x0, y1), Gy(x1, y1), fx), fy);
    return make_float4(d, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------------------
// skinning of all vertices: mode 0 -> C.vw / C.uv (for the visibility pass),
// mode 1 -> the non-rigid stage's rest geometry
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) pose_skin_kernel(const CapDesc* __restrict__ caps, const PoseDesc* __restrict__ pd,
                                                        float4* __restrict__ out_base, int mode) {
    __shared__ PoseFk fk;
    const CapDesc& C = caps[0];
    const PoseDesc& P = *pd;
    load_fk(P, fk, false);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.N) return;
    const float4 v = P.tpl[i];
    const int4 bi = P.skin_idx[i];
    const float4 bw = P.skin_w[i];
    const int bones[4] = {bi.x, bi.y, bi.z, bi.w};
    const float ws[4] = {bw.x, bw.y, bw.z, bw.w};
    float X = 0.f, Y = 0.f, Z = 0.f;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int b = bones[s];
        const float4 rb = P.rest[b];
        const float d0 = v.x - rb.x, d1 = v.y - rb.y, d2 = v.z - rb.z;
        const float* G = fk.G[b];
        X += ws[s] * (G[0] * d0 + G[1] * d1 + G[2] * d2 + fk.o[b][0]);
        Y += ws[s] * (G[3] * d0 + G[4] * d1 + G[5] * d2 + fk.o[b][1]);
        Z += ws[s] * (G[6] * d0 + G[7] * d1 + G[8] * d2 + fk.o[b][2]);
    }
    if (mode == 0) {
        if (P.use_disp) {
            // the skinned displacement rides on the skinned model (Sec. 3.4)
            const float4 d = P.disp[i];
            X += d.x;
            Y += d.y;
            Z += d.z;
        }
        const bool ok = valid_depth(Z);
        C.vw[i] = make_float4(X, Y, Z, ok ? 1.f : 0.f);
        C.uv[i] = ok ? project_exact(C.f, C.cx, C.cy, X, Y, Z) : make_float2(0.f, 0.f);
    } else {
        out_base[i] = make_float4(X, Y, Z, 0.f);
    }
}

// ---------------------------------------------------------------------------
// contour vertices in ascending order (single CTA)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) pose_blist_kernel(const CapDesc* __restrict__ caps, const PoseDesc* __restrict__ pd) {
    __shared__ int sh[1024];
    const CapDesc& C = caps[0];
    const PoseDesc& P = *pd;
    const int per = (C.N + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(C.N, b + per);
    int cnt = 0;
    for (int i = b; i < e; ++i) cnt += (C.flags[i] & LC_INB_BIT) ? 1 : 0;
    sh[threadIdx.x] = cnt;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    int pos = threadIdx.x ? sh[threadIdx.x - 1] : 0;
    for (int i = b; i < e; ++i)
        if (C.flags[i] & LC_INB_BIT) P.blist[pos++] = i;
    if (threadIdx.x == 1023) *P.bcount = sh[1023];
}

// ---------------------------------------------------------------------------
// b_i of the contour vertices at the current skinned surface (C.vw / C.uv
// hold it): the contour set stays the frame's
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) pose_dirs_kernel(const CapDesc* __restrict__ caps, const PoseDesc* __restrict__ pd) {
    const CapDesc& C = caps[0];
    const PoseDesc& P = *pd;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *P.bcount) return;
    const int i = P.blist[t];
    const float4 v = C.vw[i];
    const float2 uv = C.uv[i];
    uint32_t fl = C.flags[i];
    const bool neg = v.w > 0.f && in_image(uv, C.W, C.H) && direction_neg(C, i);
    fl = neg ? (fl | LC_BNEG_BIT) : (fl & ~LC_BNEG_BIT);
    C.flags[i] = fl;
}

// ---------------------------------------------------------------------------
// forward kinematics of the current pose into the global table (one CTA)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64) pose_fk_kernel(const PoseDesc* __restrict__ pd) {
    __shared__ PoseFk fk;
    const PoseDesc& P = *pd;
    forward_kinematics(P, fk);
    for (int q = threadIdx.x; q < (int)(sizeof(PoseFk) / sizeof(float)); q += blockDim.x)
        (&P.fk->G[0][0])[q] = (&fk.G[0][0])[q];
}

// ---------------------------------------------------------------------------
// residual rows and their FP32 pair sums.  Items: t < J the 2 rows of 2D
// joint t, t < 2J the 3 rows of 3D joint t - J, t < 3J the 3 temporal rows of
// joint t - 2J (zero without a previous frame), then one row per contour
// vertex; CTA c takes items [c kSysItems, (c + 1) kSysItems), builds their
// rows [J | F] in shared memory (stride na | 1, odd: conflict-free) and
// writes sum_rows a_r b_r for every column pair a <= b of [J | F].
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pose_row_of(int t, int J) {
    return t < J ? 2 * t : (t < 3 * J ? 2 * J + 3 * (t - J) : 8 * J + (t - 3 * J));
}

__global__ void __launch_bounds__(kSysThreads) pose_system_kernel(const CapDesc* __restrict__ caps,
                                                                  const PoseDesc* __restrict__ pd) {
    extern __shared__ float sR[];
    __shared__ PoseFk fk;
    const CapDesc& C = caps[0];
    const PoseDesc& P = *pd;
    const int J = P.J, nd = P.n_dof, na = nd + 1, stride = na | 1;
    const int nB = *P.bcount;
    const int nitems = 3 * J + nB;
    const int t0 = blockIdx.x * kSysItems;
    if (t0 >= nitems) return;                       // uniform over the CTA
    const int t1 = min(nitems, t0 + kSysItems);
    const int r0 = pose_row_of(t0, J), nr = pose_row_of(t1, J) - r0;
    const int tid = threadIdx.x;
    load_fk(P, fk, true);
    for (int q = tid; q < nr * stride; q += kSysThreads) sR[q] = 0.f;
    __syncthreads();
    const int t = t0 + tid;
    if (tid < kSysItems && t < t1) {
        float* row0 = &sR[(pose_row_of(t, J) - r0) * stride];
        if (t < J) {
            // 2D joint rows
            const int j = t;
            const float X = fk.o[j][0], Y = fk.o[j][1], Z = fk.o[j][2];
            const float s2 = sqrtf(P.lam_2d);
            if (P.has_j2d && Z > 1e-3f) {
                const float iz = 1.f / Z, fz = C.f * iz;
                row0[nd] = s2 * (fz * X + C.cx - P.j2d[j].x);
                row0[stride + nd] = s2 * (fz * Y + C.cy - P.j2d[j].y);
                const float cu[3] = {s2 * fz, 0.f, -s2 * fz * X * iz};
                const float cv[3] = {0.f, s2 * fz, -s2 * fz * Y * iz};
                add_point_row(P, fk, fk.o[j], j, cu, 1.f, row0);
                add_point_row(P, fk, fk.o[j], j, cv, 1.f, row0 + stride);
            }
        } else if (t < 2 * J) {
            // 3D joint rows
            const int j = t - J;
            const float s3 = P.has_j3d ? sqrtf(P.lam_3d) : 0.f;
            const float4 p3 = P.j3d[j];
            const float tgt[3] = {p3.x, p3.y, p3.z};
            for (int k = 0; k < 3; ++k) {
                float* row = row0 + k * stride;
                const float coef[3] = {k == 0 ? s3 : 0.f, k == 1 ? s3 : 0.f, k == 2 ? s3 : 0.f};
                if (s3 > 0.f) add_point_row(P, fk, fk.o[j], j, coef, 1.f, row);
                row[nd] = s3 * (fk.o[j][k] - tgt[k]);
            }
        } else if (t < 3 * J) {
            // temporal stabilisation rows: sqrt(l_temporal w_j) (o_j - o_j^{t-1})
            const int j = t - 2 * J;
            if (P.has_prev && P.lam_temporal > 0.f) {
                const float sT = sqrtf(P.lam_temporal * P.temporal_w[j]);
                const float4 q = P.prev_joints[j];
                const float prev[3] = {q.x, q.y, q.z};
                for (int k = 0; k < 3; ++k) {
                    float* row = row0 + k * stride;
                    const float coef[3] = {k == 0 ? sT : 0.f, k == 1 ? sT : 0.f, k == 2 ? sT : 0.f};
                    add_point_row(P, fk, fk.o[j], j, coef, 1.f, row);
                    row[nd] = sT * (fk.o[j][k] - prev[k]);
                }
            }
        } else {
            // silhouette row of a contour vertex
            const int i = P.blist[t - 3 * J];
            const float4 v = P.tpl[i];
            const int4 bi = P.skin_idx[i];
            const float4 bw = P.skin_w[i];
            const int bones[4] = {bi.x, bi.y, bi.z, bi.w};
            const float ws[4] = {bw.x, bw.y, bw.z, bw.w};
            float Pt[4][3];
            float X = 0.f, Y = 0.f, Z = 0.f;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int b = bones[s];
                const float4 rb = P.rest[b];
                const float d0 = v.x - rb.x, d1 = v.y - rb.y, d2 = v.z - rb.z;
                const float* G = fk.G[b];
                Pt[s][0] = G[0] * d0 + G[1] * d1 + G[2] * d2 + fk.o[b][0];
                Pt[s][1] = G[3] * d0 + G[4] * d1 + G[5] * d2 + fk.o[b][1];
                Pt[s][2] = G[6] * d0 + G[7] * d1 + G[8] * d2 + fk.o[b][2];
                X += ws[s] * Pt[s][0];
                Y += ws[s] * Pt[s][1];
                Z += ws[s] * Pt[s][2];
            }
            if (P.use_disp) {
                // held fixed over the solve: the Jacobian stays the skinning's
                const float4 dd = P.disp[i];
                X += dd.x;
                Y += dd.y;
                Z += dd.z;
            }
            const float2 uv = project_exact(C.f, C.cx, C.cy, X, Y, Z);
            if (valid_depth(Z) && in_image(uv, C.W, C.H)) {
                float gx, gy;
                const float d = dt_sample(C, uv.x, uv.y, gx, gy).x;
                const float ss = sqrtf(P.lam_sil / (float)max(nB, 1));
                row0[nd] = ss * d;
                const float bs = (C.flags[i] & LC_BNEG_BIT) ? -ss : ss;
                const float iz = 1.f / Z, fz = C.f * iz;
                const float coef[3] = {bs * gx * fz, bs * gy * fz, -bs * fz * iz * (gx * X + gy * Y)};
#pragma unroll
                for (int s = 0; s < 4; ++s) add_point_row(P, fk, Pt[s], bones[s], coef, ws[s], row0);
            }
        }
    }
    __syncthreads();
    const int npairs = na * (na + 1) / 2;
    float* out = P.part + (size_t)blockIdx.x * npairs;
    for (int p = tid; p < npairs; p += kSysThreads) {
        const unsigned pr = P.pairs[p];
        const int a = (int)(pr >> 8), b = (int)(pr & 255u);
        float acc = 0.f;
        for (int r = 0; r < nr; ++r) acc += sR[r * stride + a] * sR[r * stride + b];
        out[p] = acc;
    }
}

// ---------------------------------------------------------------------------
// normal equations + FP64 Cholesky + update + next kinematics (one CTA)
// mode 0: solve and update, 1: energy only, 2: export A | g into expA
// ---------------------------------------------------------------------------
constexpr int kSolveThreads = 512;

// FP64 sum over a warp (lane 0 holds the result), fixed tree order
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kTri = kMaxDof * (kMaxDof + 1) / 2;   // packed lower triangle of the normal matrix
constexpr int kGs = kMaxDof + 2;                     // FP32 inverse row stride (odd: conflict-free columns)
constexpr int kSeg = 8;                              // partial dot products per row of the FP64 residual
constexpr int kMaxRefine = 12;

__device__ __forceinline__ int tri_at(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

// FP64 right-looking square-root-free Cholesky (L D L^T) of the packed lower
// triangle Ap with right-hand side g, in place; y <- D^-1 L^-1 g, L scaled
// below the diagonal.  The robust path, taken when the mixed-precision solve
// does not converge.  Per pivot warp 0 forms 1/d_k (FP32 seed, two Newton
// steps) and the multipliers; then the trailing triangle densely over the CTA.
__device__ void ldlt_f64(double* Ap, double* g, double* colk, double* w, double* y, int nd, int tid, int* bad) {
    for (int k = 0; k < nd; ++k) {
        const int m = nd - k - 1;
        if (tid < 32) {
            const double d = Ap[tri_at(k, k)];
            double r;
            const float fd = (float)d;
            if (fd > 1e-30f && fd < 1e30f) {
                r = (double)(1.0f / fd);
                r = r * fma(-d, r, 2.0);
                r = r * fma(-d, r, 2.0);
            } else {
                r = d > 0.0 ? 1.0 / d : 0.0;
            }
            for (int t = tid; t <= m; t += 32) {
                const double c = t < m ? Ap[tri_at(k + 1 + t, k)] : g[k];
                colk[t] = c;
                const double wv = c * r;
                w[t] = wv;
                if (t < m) Ap[tri_at(k + 1 + t, k)] = wv;
                else y[k] = wv;
            }
            if (tid == 0 && !(d > 0.0)) *bad = 1;
        }
        __syncthreads();
        const int tri = m * (m + 1) / 2;
        for (int q = tid; q < tri + m; q += kSolveThreads) {
            if (q < tri) {
                int ii = (int)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f);
                while (ii * (ii + 1) / 2 > q) --ii;
                while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
                const int jj = q - ii * (ii + 1) / 2;
                double& a = Ap[tri_at(k + 1 + ii, k + 1 + jj)];
                a = fma(-w[ii], colk[jj], a);
            } else {
                const int ii = q - tri;
                g[k + 1 + ii] = fma(-w[ii], colk[m], g[k + 1 + ii]);
            }
        }
        __syncthreads();
    }
    // x = L^-T y in one warp
    if (tid < 32) {
        for (int k = nd - 1; k >= 0; --k) {
            const double xk = y[k];
            for (int i = tid; i < k; i += 32) y[i] = fma(-Ap[tri_at(k, i)], xk, y[i]);
            __syncwarp();
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kSolveThreads) pose_solve_kernel(const PoseDesc* __restrict__ pd, int slot,
                                                                  int mode) {
    __shared__ double Ap[kTri];               // FP64 normal matrix, packed lower triangle
    __shared__ double g[kMaxDof];             // -J^T F (+ prior)
    __shared__ double x[kMaxDof];             // solution
    __shared__ double rs[kMaxDof];            // residual g - A x
    __shared__ double part4[kMaxDof * kSeg];  // residual partial sums
    __shared__ double w[kMaxDof + 1];
    __shared__ double colk[kMaxDof + 1];
    __shared__ double prior_t[kMaxDof];
    __shared__ float Gf[kMaxDof * kGs];       // FP32 inverse (Gauss-Jordan, in place)
    __shared__ float colb[2][kMaxDof + 1], rf[kMaxDof], redc[4], redx[4];
    __shared__ PoseFk fk;
    __shared__ float s_ftf;
    __shared__ int s_bad, s_fail, s_conv, s_rounds, s_ok32;
    const PoseDesc& P = *pd;
    const int nd = P.n_dof, na = nd + 1;
    const int npairs = na * (na + 1) / 2;
    const int nact = (3 * P.J + *P.bcount + kSysItems - 1) / kSysItems;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_bad = 0;
        s_fail = 0;
    }
    // partial pair sums of the row CTAs, added in CTA order.  A thread's
    // pairs (up to 4) and a round of 8 CTAs: their 32 loads are issued
    // together before any is added (one L2 latency per round)
    constexpr int kPairsPer = 4;
    for (int p0 = tid; p0 < npairs; p0 += kPairsPer * kSolveThreads) {
        float v[kPairsPer] = {0.f, 0.f, 0.f, 0.f};
        for (int c0 = 0; c0 < nact; c0 += 8) {
            float pv[kPairsPer][8];
#pragma unroll
            for (int h = 0; h < kPairsPer; ++h)
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int pp = p0 + h * kSolveThreads;
                    pv[h][u] = (c0 + u < nact && pp < npairs) ? __ldcg(&P.part[(size_t)(c0 + u) * npairs + pp]) : 0.f;
                }
#pragma unroll
            for (int h = 0; h < kPairsPer; ++h)
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (c0 + u < nact) v[h] += pv[h][u];
        }
#pragma unroll
        for (int h = 0; h < kPairsPer; ++h) {
            const int pp = p0 + h * kSolveThreads;
            if (pp >= npairs) break;
            const unsigned pr = P.pairs[pp];
            const int a = (int)(pr >> 8), b = (int)(pr & 255u);
            if (b < nd) {
                Ap[tri_at(b, a)] = (double)v[h];
            } else if (a < nd) {
                g[a] = -(double)v[h];           // g = -J^T F
            } else {
                s_ftf = v[h];                   // F^T F
            }
        }
    }
    __syncthreads();
    // angle prior lprior (theta - theta_start) on the Euler DOF, and the
    // joint-limit barrier l_anatomic Psi(theta) on those outside their limits
    // (a residual sqrt(l_anatomic)(theta - bound)), one DOF per thread
    if (tid < nd) {
        double e = 0.0;
        if (tid >= 6) {
            const double th = (double)P.pose[tid];
            const double dv = th - (double)P.pose_start[tid];
            double a = (double)P.lam_prior, gg = -(double)P.lam_prior * dv;
            e = (double)P.lam_prior * dv * dv;
            const double hi = (double)P.th_hi[tid], lo = (double)P.th_lo[tid];
            const double over = th > hi ? th - hi : (th < lo ? th - lo : 0.0);
            if (over != 0.0 && P.lam_anat > 0.f) {
                a += (double)P.lam_anat;
                gg -= (double)P.lam_anat * over;
                e += (double)P.lam_anat * over * over;
            }
            Ap[tri_at(tid, tid)] += a;
            g[tid] += gg;
        }
        prior_t[tid] = e;
    }
    __syncthreads();
    if (tid < 32) {
        double e = 0.0;
        for (int c = tid; c < nd; c += 32) e += prior_t[c];
        e = warp_sum_f64(e);
        if (tid == 0) P.hist[2 * slot] = (double)s_ftf + e;
    }
    if (mode == 1) return;
    if (mode == 2) {
        for (int q = tid; q < nd * (nd + 1); q += kSolveThreads) {
            const int i = q / (nd + 1), j = q % (nd + 1);
            P.expA[q] = j < nd ? Ap[tri_at(i, j)] : g[i];
        }
        return;
    }
    // Solve A x = g to FP64 accuracy.  GB300's FP64 pipe is slow per warp
    // instruction and the 57 pivots of a factorisation form a serial chain,
    // so the factorisation runs in FP32 and FP64 only enters the residual
    // (mixed-precision iterative refinement):
    //   Gf = A^-1 in FP32 by a symmetric sweep (A is positive definite: no
    //        pivoting);
    //   x = 0, r = g; repeat  x += Gf r (FP32 product), r = g - A x (FP64)
    //   until the correction (or its extrapolated successor) is below 1e-10
    //   of x (the FP64 residual's floor is ~cond(A) 1e-16).
    // A non-positive or non-finite FP32 pivot, or no convergence in
    // kMaxRefine rounds, falls back to the FP64 L D L^T of the same system.
    // Symmetric sweep (Gauss-Jordan for a symmetric matrix, lower triangle
    // only): per pivot k with d = a_kk and the old column c,
    //   a_ij -= c_i c_j / d (i, j != k),  a_ik = c_i / d,  a_kk = -1 / d;
    // after all pivots the triangle holds -A^-1.  Each thread keeps its
    // entries of the packed triangle in registers (round-robin); the owners
    // publish column k + 1 (double-buffered), so one block barrier per pivot;
    // every thread forms 1 / d itself (FP32).  The per-entry update is
    // branch-free (selects, and a publish store that lands in a spare slot
    // when the entry is not in column k + 1), so a thread's entries
    // interleave.
    constexpr int kPer = (kTri + kSolveThreads - 1) / kSolveThreads;
    constexpr int kSpare = kMaxDof;              // colb slot that absorbs non-publishing stores
    {
        const int ntri = nd * (nd + 1) / 2;
        float ga[kPer];
        int gi[kPer], gj[kPer];
#pragma unroll
        for (int sI = 0; sI < kPer; ++sI) {
            const int e = tid + kSolveThreads * sI;
            int i = kSpare, j = kSpare;              // padding entries: every access in the spare slot
            if (e < ntri) {
                i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
                while (i * (i + 1) / 2 > e) --i;
                while ((i + 1) * (i + 2) / 2 <= e) ++i;
                j = e - i * (i + 1) / 2;
            }
            gi[sI] = i;
            gj[sI] = j;
            ga[sI] = e < ntri ? (float)Ap[e] : 0.f;
            if (e < ntri && j == 0) colb[0][i] = ga[sI];
        }
        bool ok = P.solver == 0;
        for (int k = 0; ok && k < nd; ++k) {
            __syncthreads();
            const float* c = colb[k & 1];
            float* cn = colb[(k + 1) & 1];
            const float d = c[k];
            if (!(d > 0.f) || !(d < 3.0e38f)) {
                ok = false;                          // uniform: every thread read the same pivot
                break;
            }
            const float r = __frcp_rn(d);
#pragma unroll
            for (int sI = 0; sI < kPer; ++sI) {
                const int i = gi[sI], j = gj[sI];
                const float ci = c[i], cj = c[j];
                const float upd = fmaf(-ci * r, cj, ga[sI]);
                const float rowk = j == k ? -r : cj * r;
                const float a = i == k ? rowk : (j == k ? ci * r : upd);
                ga[sI] = a;
                cn[j == k + 1 ? i : (i == k + 1 ? j : kSpare)] = a;
            }
        }
        if (tid == 0) s_ok32 = ok ? 1 : 0;
        if (ok) {
#pragma unroll
            for (int sI = 0; sI < kPer; ++sI) {
                const int i = gi[sI], j = gj[sI];
                if (j < kSpare) {
                    Gf[i * kGs + j] = -ga[sI];
                    Gf[j * kGs + i] = -ga[sI];
                }
            }
        }
    }
    __syncthreads();
    const bool ok32 = s_ok32 != 0;
    if (ok32) {
        if (tid < nd) {
            x[tid] = 0.0;
            rs[tid] = g[tid];
        }
        __syncthreads();
        double cm_prev = 0.0;   // thread 0: the last correction
        for (int it = 0; it < kMaxRefine; ++it) {
            // correction c = Gf r (FP32), x += c; the largest |c| and |x|
            if (tid < nd) rf[tid] = (float)rs[tid];
            __syncthreads();
            if (tid < 2 * 64) {
                // two threads per row, the halves added in a fixed order
                const int i = tid >> 1, h = tid & 1;
                float c = 0.f;
                if (i < nd)
                    for (int j = h; j < nd; j += 2) c = fmaf(Gf[i * kGs + j], rf[j], c);
                c += __shfl_xor_sync(0xffffffffu, c, 1);
                float cmax = 0.f, xmax = 0.f;          // magnitudes for the stopping test
                if (i < nd && h == 0) {
                    const double xn = x[i] + (double)c;
                    x[i] = xn;
                    cmax = fabsf(c);
                    xmax = fabsf((float)xn);
                    if (!(cmax < 3.0e38f) || !(xmax < 3.0e38f)) s_fail = 1;   // non-finite (read after the barrier)
                }
                for (int o = 16; o > 0; o >>= 1) {
                    cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
                    xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
                }
                if ((tid & 31) == 0) {
                    redc[tid >> 5] = cmax;
                    redx[tid >> 5] = xmax;
                }
            }
            __syncthreads();
            if (tid == 0) {
                // converged: the correction is below 1e-10 of x, or the next
                // one, extrapolated from the contraction of the last two
                // (cm^2 / cm_prev), is; or the corrections stopped shrinking
                // (the FP64 residual's rounding floor, ~n cond(A) 1e-16) at
                // <= 1e-6 of x; a stall above that is a failure (the FP32
                // inverse does not contract)
                const double cm = fmaxf(fmaxf(redc[0], redc[1]), fmaxf(redc[2], redc[3]));
                const double xm = fmaxf(fmaxf(redx[0], redx[1]), fmaxf(redx[2], redx[3]));
                int conv = cm <= 1e-10 * xm ? 1 : 0;
                if (!conv && it > 0 && cm < 0.5 * cm_prev && cm * cm <= 1e-10 * xm * cm_prev) conv = 1;
                if (!conv && it > 0 && cm > 0.5 * cm_prev) {
                    if (cm <= 1e-6 * xm) conv = 1;
                    else s_fail = 1;
                }
                s_conv = conv;
                s_rounds = it + 1;
                cm_prev = cm;
            }
            __syncthreads();
            if (s_conv || s_fail) break;
            // r = g - A x in FP64: kSeg partial products per row, then one sum per row
            if (tid < nd * kSeg) {
                const int i = tid / kSeg, sg = tid - i * kSeg;
                const int j0 = sg * ((nd + kSeg - 1) / kSeg), j1 = min(nd, j0 + (nd + kSeg - 1) / kSeg);
                double acc = 0.0;
                for (int j = j0; j < j1; ++j) acc = fma(Ap[tri_at(i, j)], x[j], acc);
                part4[tid] = acc;
            }
            __syncthreads();
            if (tid < nd) {
                double a = 0.0;
                for (int sg = 0; sg < kSeg; ++sg) a += part4[tid * kSeg + sg];
                rs[tid] = g[tid] - a;
            }
            __syncthreads();
        }
        if (tid == 0 && !s_conv) s_fail = 1;
        __syncthreads();
    }
    double* y = rs;     // the solution handed to the update: x, or the fallback's
    const bool fallback = !ok32 || s_fail;
    if (fallback) {
        ldlt_f64(Ap, g, colk, w, rs, nd, tid, &s_bad);
    } else if (tid < nd) {
        rs[tid] = x[tid];
    }
    if (tid == 0) P.info[slot] = fallback ? -1 : s_rounds;
    __syncthreads();
    // the pose update: one DOF per thread; the root rotation and the step
    // norm by thread 0
    if (!s_bad && tid >= 3 && tid < nd) P.pose[tid] += (float)y[tid];
    if (tid < 32) {
        double n2 = 0.0;
        for (int c = tid; c < nd; c += 32) n2 += y[c] * y[c];
        n2 = warp_sum_f64(n2);
        if (tid == 0) {
            if (s_bad) {
                *P.status = 1;
                P.hist[2 * slot + 1] = 0.0;
            } else {
                P.hist[2 * slot + 1] = sqrt(n2);
                // R <- Exp(d_omega) R (Rodrigues, FP32)
                const float wx = (float)y[0], wy = (float)y[1], wz = (float)y[2];
                const float th2 = wx * wx + wy * wy + wz * wz, th = sqrtf(th2);
                float Af, Bf;
                if (th < 1e-4f) {
                    Af = 1.f - th2 / 6.f;
                    Bf = 0.5f - th2 / 24.f;
                } else {
                    const float sh = sinf(0.5f * th);
                    Af = sinf(th) / th;
                    Bf = 2.f * sh * sh / th2;
                }
                const float E[9] = {1.f - Bf * (wy * wy + wz * wz), -Af * wz + Bf * wx * wy, Af * wy + Bf * wx * wz,
                                    Af * wz + Bf * wx * wy, 1.f - Bf * (wx * wx + wz * wz), -Af * wx + Bf * wy * wz,
                                    -Af * wy + Bf * wx * wz, Af * wx + Bf * wy * wz, 1.f - Bf * (wx * wx + wy * wy)};
                float R[9], Rn[9];
                for (int q = 0; q < 9; ++q) R[q] = P.Rroot[q];
                mat3mul(E, R, Rn);
                for (int q = 0; q < 9; ++q) P.Rroot[q] = Rn[q];
            }
        }
    }
    __threadfence_block();
    __syncthreads();
    // kinematics of the new pose for the next step's kernels
    forward_kinematics(P, fk);
    for (int q = tid; q < (int)(sizeof(PoseFk) / sizeof(float)); q += kSolveThreads)
        (&P.fk->G[0][0])[q] = (&fk.G[0][0])[q];
}

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Displacement warping of the surface stage (Sec. 3.4): the rotation Q_i of
// the dual-quaternion blend of vertex i's bone rotations (its skinning
// weights; quaternions sign-aligned with the first slot's bone, summed and
// normalised).  mode 0 records the rest-pose displacement
// sD_i = Q_i^T (V_i - V^S_i); mode 1 starts the surface at
// V_i = V^S_i + Q_i sD_i.  Without a skeleton (pd null) Q_i = I.
// ---------------------------------------------------------------------------
// unit quaternion (x, y, z, w) of a row-major rotation matrix, branching on
// the largest of the trace and the diagonal (Shepperd, 1978)
__device__ __forceinline__ float4 quat_of(const float* G) {
    const float tr = G[0] + G[4] + G[8];
    float4 q;
    if (tr >= G[0] && tr >= G[4] && tr >= G[8]) {
        const float w = 0.5f * sqrtf(fmaxf(1.f + tr, 0.f)), k = 0.25f / w;
        q = make_float4((G[7] - G[5]) * k, (G[2] - G[6]) * k, (G[3] - G[1]) * k, w);
    } else if (G[0] >= G[4] && G[0] >= G[8]) {
        const float x = 0.5f * sqrtf(fmaxf(1.f + G[0] - G[4] - G[8], 0.f)), k = 0.25f / x;
        q = make_float4(x, (G[1] + G[3]) * k, (G[2] + G[6]) * k, (G[7] - G[5]) * k);
    } else if (G[4] >= G[8]) {
        const float y = 0.5f * sqrtf(fmaxf(1.f - G[0] + G[4] - G[8], 0.f)), k = 0.25f / y;
        q = make_float4((G[1] + G[3]) * k, y, (G[5] + G[7]) * k, (G[2] - G[6]) * k);
    } else {
        const float z = 0.5f * sqrtf(fmaxf(1.f - G[0] - G[4] + G[8], 0.f)), k = 0.25f / z;
        q = make_float4((G[2] + G[6]) * k, (G[5] + G[7]) * k, z, (G[3] - G[1]) * k);
    }
    return q;
}

// the blend rotation of vertex i from the bones' quaternions qb (row-major;
// the identity where the weighted sum vanishes)
__device__ __forceinline__ void blend_rotation(const PoseDesc& P, const float4* qb, int i, float* R) {
    const int4 bi = P.skin_idx[i];
    const float4 bw = P.skin_w[i];
    const int bones[4] = {bi.x, bi.y, bi.z, bi.w};
    const float ws[4] = {bw.x, bw.y, bw.z, bw.w};
    const float4 q0 = qb[bones[0]];
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 q = qb[bones[k]];
        const float w = (q.x * q0.x + q.y * q0.y + q.z * q0.z + q.w * q0.w) < 0.f ? -ws[k] : ws[k];
        s.x += w * q.x; s.y += w * q.y; s.z += w * q.z; s.w += w * q.w;
    }
    const float n2 = s.x * s.x + s.y * s.y + s.z * s.z + s.w * s.w;
    if (n2 > 0.f) {
        const float inv = rsqrtf(n2);
        const float x = s.x * inv, y = s.y * inv, z = s.z * inv, w = s.w * inv;
        R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - z * w);       R[2] = 2.f * (x * z + y * w);
        R[3] = 2.f * (x * y + z * w);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - x * w);
        R[6] = 2.f * (x * z - y * w);       R[7] = 2.f * (y * z + x * w);       R[8] = 1.f - 2.f * (x * x + y * y);
    }
}

__global__ void __launch_bounds__(256) surface_warp_kernel(const CapDesc* __restrict__ caps,
                                                           const PoseDesc* __restrict__ pd, int mode) {
    __shared__ float4 qb[kMaxJoints];
    const CapDesc& C = caps[0];
    if (pd)
        for (int b = threadIdx.x; b < pd->J; b += blockDim.x) qb[b] = quat_of(&pd->fk->G[b][0]);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.N) return;
    float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    if (pd) blend_rotation(*pd, qb, i, R);
    if (mode == 2) {
        const float4 d = C.sD[i];
        pd->disp[i] = make_float4(R[0] * d.x + R[1] * d.y + R[2] * d.z, R[3] * d.x + R[4] * d.y + R[5] * d.z,
                                  R[6] * d.x + R[7] * d.y + R[8] * d.z, 0.f);
        return;
    }
    const float4 S = C.base[i];
    if (mode == 0) {
        const float4 V = C.sV[i];
        const float dx = V.x - S.x, dy = V.y - S.y, dz = V.z - S.z;
        C.sD[i] = make_float4(R[0] * dx + R[3] * dy + R[6] * dz, R[1] * dx + R[4] * dy + R[7] * dz,
                              R[2] * dx + R[5] * dy + R[8] * dz, 0.f);
    } else {
        const float4 d = C.sD[i];
        C.sV[i] = make_float4(S.x + (R[0] * d.x + R[1] * d.y + R[2] * d.z), S.y + (R[3] * d.x + R[4] * d.y + R[5] * d.z),
                              S.z + (R[6] * d.x + R[7] * d.y + R[8] * d.z), 0.f);
    }
}

// ---------------------------------------------------------------------------
// Displacement warping of the graph stage (the graph counterpart of Sec. 3.4's
// warping): node k's parameters are carried in the rest pose through the
// blend rotation Q_k of its node vertex.  mode 0 (end of a frame, final pose)
// records R^rest = Q^T R Q, t^rest = Q^T t and marks them valid; mode 1
// (start of a frame, after the pose solve) sets R = Q R^rest Q^T,
// t = Q t^rest when a record is valid.  Under a common rigid motion of a
// node's bones this moves the deformed surface rigidly with them.
// rest: 4n float4 (rows of R^rest, then t^rest).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) graph_warp_kernel(const CapDesc* __restrict__ caps,
                                                         const PoseDesc* __restrict__ pd, float4* __restrict__ rest,
                                                         int* __restrict__ valid, int mode) {
    __shared__ float4 qb[kMaxJoints];
    const CapDesc& C = caps[0];
    if (mode == 1 && *valid == 0) return;
    for (int b = threadIdx.x; b < pd->J; b += blockDim.x) qb[b] = quat_of(&pd->fk->G[b][0]);
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= C.n) return;
    float Q[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    blend_rotation(*pd, qb, C.node_vid[k], Q);
    // A = Q^T, B = Q (mode 0) or A = Q, B = Q^T (mode 1): out = A M B, t' = A t
    float A[9], B[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            A[3 * r + c] = mode == 0 ? Q[3 * c + r] : Q[3 * r + c];
            B[3 * r + c] = mode == 0 ? Q[3 * r + c] : Q[3 * c + r];
        }
    const float4* src_R = mode == 0 ? C.node_R : rest;
    const float4 s0 = src_R[3 * k], s1 = src_R[3 * k + 1], s2 = src_R[3 * k + 2];
    const float4 st = mode == 0 ? C.node_t[k] : rest[3 * C.n + k];
    const float M[9] = {s0.x, s0.y, s0.z, s1.x, s1.y, s1.z, s2.x, s2.y, s2.z};
    float AM[9], O[9];
    mat3mul(A, M, AM);
    mat3mul(AM, B, O);
    const float4 r0 = make_float4(O[0], O[1], O[2], 0.f), r1 = make_float4(O[3], O[4], O[5], 0.f),
                 r2 = make_float4(O[6], O[7], O[8], 0.f);
    const float4 t = make_float4(A[0] * st.x + A[1] * st.y + A[2] * st.z, A[3] * st.x + A[4] * st.y + A[5] * st.z,
                                 A[6] * st.x + A[7] * st.y + A[8] * st.z, 0.f);
    if (mode == 0) {
        rest[3 * k] = r0; rest[3 * k + 1] = r1; rest[3 * k + 2] = r2;
        rest[3 * C.n + k] = t;
        if (k == 0) *valid = 1;
    } else {
        C.node_R[3 * k] = r0; C.node_R[3 * k + 1] = r1; C.node_R[3 * k + 2] = r2;
        C.node_t[k] = t;
    }
}

void launch_graph_warp(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, float4* rest, int* valid, int mode,
                       cudaStream_t st) {
    graph_warp_kernel<<<(hC.n + 255) / 256, 256, 0, st>>>(dC, dP, rest, valid, mode);
}

void launch_pose_skin(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, float4* out_base, int mode,
                      cudaStream_t st) {
    pose_skin_kernel<<<(hC.N + 255) / 256, 256, 0, st>>>(dC, dP, out_base, mode);
}
// ---------------------------------------------------------------------------
// Frame bookkeeping of the pose stage (Sec. 3.3): E_temporal's previous-frame
// joints and the two-frame pose history of the start extrapolation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64) pose_advance_kernel(const PoseDesc* __restrict__ pd) {
    const PoseDesc& P = *pd;
    constexpr int kRec = kMaxDof + 9;
    const int t = threadIdx.x;
    if (t < P.J) P.prev_joints[t] = make_float4(P.fk->o[t][0], P.fk->o[t][1], P.fk->o[t][2], 0.f);
    for (int q = t; q < kRec; q += blockDim.x) {
        const float cur = q < kMaxDof ? (q < P.n_dof ? P.pose[q] : 0.f) : P.Rroot[q - kMaxDof];
        P.pose_hist[kRec + q] = P.pose_hist[q];
        P.pose_hist[q] = cur;
    }
}

// pose <- 2 theta^{t-1} - theta^{t-2} (Euler angles, root translation),
// R <- R^{t-1} (R^{t-2})^T R^{t-1}; with one recorded pose, that pose
__global__ void __launch_bounds__(64) pose_extrapolate_kernel(const PoseDesc* __restrict__ pd) {
    const PoseDesc& P = *pd;
    constexpr int kRec = kMaxDof + 9;
    const float* h0 = P.pose_hist;
    const float* h1 = P.pose_hist + kRec;
    const bool two = P.n_hist >= 2;
    const int t = threadIdx.x;
    if (t >= 3 && t < P.n_dof) P.pose[t] = two ? 2.f * h0[t] - h1[t] : h0[t];
    if (t == 0) {
        const float* R0 = h0 + kMaxDof;
        float R[9];
        if (two) {
            const float* R1 = h1 + kMaxDof;
            float R1t[9], M[9];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) R1t[3 * a + b] = R1[3 * b + a];
            mat3mul(R0, R1t, M);
            mat3mul(M, R0, R);
        } else {
            for (int q = 0; q < 9; ++q) R[q] = R0[q];
        }
        for (int q = 0; q < 9; ++q) P.Rroot[q] = R[q];
    }
}

void launch_pose_advance(const PoseDesc* dP, cudaStream_t st) {
    pose_fk_kernel<<<1, 64, 0, st>>>(dP);
    pose_advance_kernel<<<1, 64, 0, st>>>(dP);
}
void launch_pose_extrapolate(const PoseDesc* dP, cudaStream_t st) { pose_extrapolate_kernel<<<1, 64, 0, st>>>(dP); }

void launch_pose_fk(const PoseDesc* dP, cudaStream_t st) { pose_fk_kernel<<<1, 64, 0, st>>>(dP); }
void launch_surface_warp(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, int mode, cudaStream_t st) {
    if (dP) pose_fk_kernel<<<1, 64, 0, st>>>(dP);   // kinematics of the current pose
    surface_warp_kernel<<<(hC.N + 255) / 256, 256, 0, st>>>(dC, dP, mode);
}
void launch_pose_blist(const CapDesc* dC, const PoseDesc* dP, cudaStream_t st) {
    pose_blist_kernel<<<1, 1024, 0, st>>>(dC, dP);
}
void launch_pose_dirs(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, cudaStream_t st) {
    pose_skin_kernel<<<(hC.N + 255) / 256, 256, 0, st>>>(dC, dP, nullptr, 0);
    pose_dirs_kernel<<<(hC.N + 255) / 256, 256, 0, st>>>(dC, dP);
}
size_t pose_system_smem(int n_dof) { return sizeof(float) * 3 * kSysItems * ((n_dof + 1) | 1); }
cudaError_t pose_kernels_init(int n_dof) {
    // sized for the largest skeleton, so no context lowers it below another's need
    (void)n_dof;
    return cudaFuncSetAttribute(pose_system_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pose_system_smem(kMaxDof));
}
int pose_system_ctas(int J, int N) { return (3 * J + N + kSysItems - 1) / kSysItems; }
void launch_pose_system(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, int J, int n_dof,
                        cudaStream_t st) {
    pose_system_kernel<<<pose_system_ctas(J, hC.N), kSysThreads, pose_system_smem(n_dof), st>>>(dC, dP);
}
void launch_pose_solve(const PoseDesc* dP, int slot, int mode, cudaStream_t st) {
    pose_solve_kernel<<<1, kSolveThreads, 0, st>>>(dP, slot, mode);
}

}  // namespace lc

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
// factorising them by Cholesky (pivot <= 0 sets a status word), updating the
// pose and computing the next forward kinematics - no host round trip.
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
    const int j = threadIdx.x;
    const float* pose = P.pose;
    for (int lvl = 0; lvl < P.n_levels; ++lvl) {
        if (j < P.J && P.level[j] == lvl) {
            const int p = P.parents[j];
            if (p < 0) {
#pragma unroll
                for (int q = 0; q < 9; ++q) fk.G[j][q] = P.Rroot[q];
                fk.o[j][0] = pose[3];
                fk.o[j][1] = pose[4];
                fk.o[j][2] = pose[5];
            } else {
                const float4 rj = P.rest[j], rp = P.rest[p];
                const float d[3] = {rj.x - rp.x, rj.y - rp.y, rj.z - rp.z};
                float Gp[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) Gp[q] = fk.G[p][q];
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    fk.o[j][r] = fk.o[p][r] + Gp[3 * r] * d[0] + Gp[3 * r + 1] * d[1] + Gp[3 * r + 2] * d[2];
                const int c = P.col[j];
                if (c < 0) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) fk.G[j][q] = Gp[q];
                } else {
                    float sa, ca, sb, cb, sc, cc;
                    sincosf(pose[c], &sa, &ca);
                    sincosf(pose[c + 1], &sb, &cb);
                    sincosf(pose[c + 2], &sc, &cc);
                    const float Rx[9] = {1.f, 0.f, 0.f, 0.f, ca, -sa, 0.f, sa, ca};
                    const float Ry[9] = {cb, 0.f, sb, 0.f, 1.f, 0.f, -sb, 0.f, cb};
                    const float Rz[9] = {cc, -sc, 0.f, sc, cc, 0.f, 0.f, 0.f, 1.f};
                    float GRx[9], GRxRy[9], G[9];
                    mat3mul(Gp, Rx, GRx);
                    mat3mul(GRx, Ry, GRxRy);
                    mat3mul(GRxRy, Rz, G);
#pragma unroll
                    for (int q = 0; q < 9; ++q) fk.G[j][q] = G[q];
                    // axes: G_p e_x, G_p Rx e_y, G_p Rx Ry e_z (columns)
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        fk.U[j][r] = Gp[3 * r];
                        fk.U[j][3 + r] = GRx[3 * r + 1];
                        fk.U[j][6 + r] = GRxRy[3 * r + 2];
                    }
                }
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
// joint t, t < 2J the 3 rows of 3D joint t - J, then one row per contour
// vertex; CTA c takes items [c kSysItems, (c + 1) kSysItems), builds their
// rows [J | F] in shared memory (stride na | 1, odd: conflict-free) and
// writes sum_rows a_r b_r for every column pair a <= b of [J | F].
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pose_row_of(int t, int J) {
    return t < J ? 2 * t : (t < 2 * J ? 2 * J + 3 * (t - J) : 5 * J + (t - 2 * J));
}

__global__ void __launch_bounds__(kSysThreads) pose_system_kernel(const CapDesc* __restrict__ caps,
                                                                  const PoseDesc* __restrict__ pd) {
    extern __shared__ float sR[];
    __shared__ PoseFk fk;
    const CapDesc& C = caps[0];
    const PoseDesc& P = *pd;
    const int J = P.J, nd = P.n_dof, na = nd + 1, stride = na | 1;
    const int nB = *P.bcount;
    const int nitems = 2 * J + nB;
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
        } else {
            // silhouette row of a contour vertex
            const int i = P.blist[t - 2 * J];
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

__global__ void __launch_bounds__(kSolveThreads) pose_solve_kernel(const PoseDesc* __restrict__ pd, int slot,
                                                                  int mode) {
    __shared__ double A[kMaxDof][kMaxDof + 1];
    __shared__ double invd[kMaxDof];
    __shared__ double w[kMaxDof + 1];
    __shared__ double colk[kMaxDof + 1];
    __shared__ double y[kMaxDof];
    __shared__ double prior_t[kMaxDof];
    __shared__ PoseFk fk;
    __shared__ float s_ftf;
    __shared__ int s_bad;
    const PoseDesc& P = *pd;
    const int nd = P.n_dof, na = nd + 1;
    const int npairs = na * (na + 1) / 2;
    const int nact = (2 * P.J + *P.bcount + kSysItems - 1) / kSysItems;
    const int tid = threadIdx.x;
    if (tid == 0) s_bad = 0;
    // partial pair sums of the row CTAs, added in CTA order
    for (int p = tid; p < npairs; p += kSolveThreads) {
        float v = 0.f;
        for (int c = 0; c < nact; ++c) v += P.part[(size_t)c * npairs + p];
        const unsigned pr = P.pairs[p];
        const int a = (int)(pr >> 8), b = (int)(pr & 255u);
        if (b < nd) {
            A[a][b] = (double)v;
            A[b][a] = (double)v;
        } else if (a < nd) {
            A[a][nd] = -(double)v;          // g = -J^T F
        } else {
            s_ftf = v;                      // F^T F
        }
    }
    __syncthreads();
    // angle prior lprior (theta - theta_start) on the Euler DOF, one DOF per thread
    if (tid < nd) {
        double e = 0.0;
        if (tid >= 6) {
            const double dv = (double)P.pose[tid] - (double)P.pose_start[tid];
            A[tid][tid] += (double)P.lam_prior;
            A[tid][nd] -= (double)P.lam_prior * dv;
            e = (double)P.lam_prior * dv * dv;
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
        for (int q = tid; q < nd * (nd + 1); q += kSolveThreads) P.expA[q] = A[q / (nd + 1)][q % (nd + 1)];
        return;
    }
    // Square-root-free Cholesky A = L D L^T (FP64) of the matrix augmented
    // with g, right-looking: after pivot k the trailing lower triangle holds
    // the Schur complement and column nd the forward-substituted right-hand
    // side.  GB300's FP64 pipe is slow per warp instruction, so per pivot:
    // warp 0 alone forms 1/d_k (FP32 seed refined by two Newton steps
    // y <- y (2 - d y), no division) and the multipliers w_i = A_ik / d_k
    // (L's column k, stored in place; the unscaled column kept in colk); one
    // block barrier; then the trailing lower triangle and column nd, packed
    // densely over all threads so that every FP64 warp instruction carries
    // 32 useful FMAs; one block barrier.
    for (int k = 0; k < nd; ++k) {
        const int m = nd - k - 1;
        if (tid < 32) {
            const double d = A[k][k];
            double r;
            const float fd = (float)d;
            if (fd > 1e-30f && fd < 1e30f) {
                r = (double)__frcp_rn(fd);
                r = r * fma(-d, r, 2.0);
                r = r * fma(-d, r, 2.0);
            } else {
                r = d > 0.0 ? 1.0 / d : 0.0;
            }
            for (int t = tid; t <= m; t += 32) {
                const double c = t < m ? A[k + 1 + t][k] : A[k][nd];
                colk[t] = c;
                const double wv = c * r;
                w[t] = wv;
                if (t < m) A[k + 1 + t][k] = wv;
                else y[k] = wv;
            }
            if (tid == 0) {
                if (!(d > 0.0)) s_bad = 1;
                invd[k] = r;
            }
        }
        __syncthreads();
        const int tri = m * (m + 1) / 2;
        for (int q = tid; q < tri + m; q += kSolveThreads) {
            if (q < tri) {
                // packed row-major trailing triangle: q -> (ii, jj), jj <= ii
                int ii = (int)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f);
                while (ii * (ii + 1) / 2 > q) --ii;
                while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
                const int jj = q - ii * (ii + 1) / 2;
                double& a = A[k + 1 + ii][k + 1 + jj];
                a = fma(-w[ii], colk[jj], a);
            } else {
                const int ii = q - tri;
                double& a = A[k + 1 + ii][nd];
                a = fma(-w[ii], colk[m], a);
            }
        }
        __syncthreads();
    }
    // x = L^-T y, column by column in one warp (L stored below the diagonal of A)
    if (tid < 32) {
        for (int k = nd - 1; k >= 0; --k) {
            const double xk = y[k];
            for (int i = tid; i < k; i += 32) y[i] = fma(-A[k][i], xk, y[i]);
            __syncwarp();
        }
        double n2 = 0.0;
        for (int c = tid; c < nd; c += 32) n2 += y[c] * y[c];
        n2 = warp_sum_f64(n2);
        if (tid == 0) {
            if (s_bad) {
                *P.status = 1;
                P.hist[2 * slot + 1] = 0.0;
            } else {
                P.hist[2 * slot + 1] = sqrt(n2);
                for (int c = 3; c < nd; ++c) P.pose[c] += (float)y[c];
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
    if (pd) {
        const int4 bi = pd->skin_idx[i];
        const float4 bw = pd->skin_w[i];
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

void launch_pose_skin(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, float4* out_base, int mode,
                      cudaStream_t st) {
    pose_skin_kernel<<<(hC.N + 255) / 256, 256, 0, st>>>(dC, dP, out_base, mode);
}
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
int pose_system_ctas(int J, int N) { return (2 * J + N + kSysItems - 1) / kSysItems; }
void launch_pose_system(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, int J, int n_dof,
                        cudaStream_t st) {
    pose_system_kernel<<<pose_system_ctas(J, hC.N), kSysThreads, pose_system_smem(n_dof), st>>>(dC, dP);
}
void launch_pose_solve(const PoseDesc* dP, int slot, int mode, cudaStream_t st) {
    pose_solve_kernel<<<1, kSolveThreads, 0, st>>>(dP, slot, mode);
}

}  // namespace lc

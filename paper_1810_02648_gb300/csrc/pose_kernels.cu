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
// The dense Jacobian (rows x n_dof, FP32, column-major) is reduced to J^T J
// and J^T F in FP32 by one CTA staging row chunks in shared memory, and the
// normal equations are solved by an FP64 Cholesky factorisation in shared
// memory (pivot <= 0 sets a status word) - no host round trip.
#include "lc_internal.cuh"
#include "pose_internal.h"

namespace lc {

// forward kinematics of the whole skeleton into shared memory (thread 0)
struct FkSmem {
    float G[kMaxJoints][9];
    float o[kMaxJoints][3];
    float U[kMaxJoints][9];   // three world axes (rows) per DOF joint
};

__device__ __forceinline__ void mat3mul(const float* A, const float* B, float* C) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

__device__ void forward_kinematics(const PoseDesc& P, FkSmem& fk) {
    if (threadIdx.x != 0) return;
    const float* pose = P.pose;
    for (int j = 0; j < P.J; ++j) {
        const int p = P.parents[j];
        if (p < 0) {
#pragma unroll
            for (int q = 0; q < 9; ++q) fk.G[j][q] = P.Rroot[q];
            fk.o[j][0] = pose[3];
            fk.o[j][1] = pose[4];
            fk.o[j][2] = pose[5];
            continue;
        }
        const float4 rj = P.rest[j], rp = P.rest[p];
        const float d[3] = {rj.x - rp.x, rj.y - rp.y, rj.z - rp.z};
        const float* Gp = fk.G[p];
#pragma unroll
        for (int r = 0; r < 3; ++r) fk.o[j][r] = fk.o[p][r] + Gp[3 * r] * d[0] + Gp[3 * r + 1] * d[1] + Gp[3 * r + 2] * d[2];
        const int c = P.col[j];
        if (c < 0) {
#pragma unroll
            for (int q = 0; q < 9; ++q) fk.G[j][q] = Gp[q];
            continue;
        }
        float sa, ca, sb, cb, sc, cc;
        sincosf(pose[c], &sa, &ca);
        sincosf(pose[c + 1], &sb, &cb);
        sincosf(pose[c + 2], &sc, &cc);
        const float Rx[9] = {1.f, 0.f, 0.f, 0.f, ca, -sa, 0.f, sa, ca};
        const float Ry[9] = {cb, 0.f, sb, 0.f, 1.f, 0.f, -sb, 0.f, cb};
        const float Rz[9] = {cc, -sc, 0.f, sc, cc, 0.f, 0.f, 0.f, 1.f};
        float GRx[9], GRxRy[9];
        mat3mul(Gp, Rx, GRx);
        mat3mul(GRx, Ry, GRxRy);
        mat3mul(GRxRy, Rz, fk.G[j]);
        // axes: G_p e_x, G_p Rx e_y, G_p Rx Ry e_z (columns)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            fk.U[j][r] = Gp[3 * r];
            fk.U[j][3 + r] = GRx[3 * r + 1];
            fk.U[j][6 + r] = GRxRy[3 * r + 2];
        }
    }
}

__device__ __forceinline__ void cross3f(const float* a, const float* b, float* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Adds w * coef . dP/dtheta (P riding on bone b) into row[0..n_dof).
__device__ __forceinline__ void add_point_row(const PoseDesc& P, const FkSmem& fk, const float* pt, int b,
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
    __shared__ FkSmem fk;
    const CapDesc& C = caps[0];
    const PoseDesc& P = *pd;
    forward_kinematics(P, fk);
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
// residual rows and dense Jacobian rows (column-major, ld = max_rows)
// thread t < J: 2D rows of joint t; t < 2J: 3D rows; then one row per
// contour vertex
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) pose_rows_kernel(const CapDesc* __restrict__ caps, const PoseDesc* __restrict__ pd) {
    __shared__ FkSmem fk;
    const CapDesc& C = caps[0];
    const PoseDesc& P = *pd;
    forward_kinematics(P, fk);
    __syncthreads();
    const int J = P.J, nd = P.n_dof, ld = P.max_rows;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nB = *P.bcount;
    if (t >= 2 * J + nB) return;
    float row[3][kMaxDof];
    if (t < J) {
        // 2D joint rows
        const int j = t;
        const float X = fk.o[j][0], Y = fk.o[j][1], Z = fk.o[j][2];
        const float s2 = sqrtf(P.lam_2d);
        const bool ok = P.has_j2d && Z > 1e-3f;
        float r0 = 0.f, r1 = 0.f;
        for (int c = 0; c < nd; ++c) row[0][c] = row[1][c] = 0.f;
        if (ok) {
            const float iz = 1.f / Z, fz = C.f * iz;
            r0 = s2 * (fz * X + C.cx - P.j2d[j].x);
            r1 = s2 * (fz * Y + C.cy - P.j2d[j].y);
            const float cu[3] = {s2 * fz, 0.f, -s2 * fz * X * iz};
            const float cv[3] = {0.f, s2 * fz, -s2 * fz * Y * iz};
            add_point_row(P, fk, fk.o[j], j, cu, 1.f, row[0]);
            add_point_row(P, fk, fk.o[j], j, cv, 1.f, row[1]);
        }
        P.F[2 * j] = r0;
        P.F[2 * j + 1] = r1;
        for (int c = 0; c < nd; ++c) {
            P.Jm[(size_t)c * ld + 2 * j] = row[0][c];
            P.Jm[(size_t)c * ld + 2 * j + 1] = row[1][c];
        }
    } else if (t < 2 * J) {
        const int j = t - J;
        const float s3 = P.has_j3d ? sqrtf(P.lam_3d) : 0.f;
        for (int k = 0; k < 3; ++k) {
            for (int c = 0; c < nd; ++c) row[k][c] = 0.f;
            const float coef[3] = {k == 0 ? s3 : 0.f, k == 1 ? s3 : 0.f, k == 2 ? s3 : 0.f};
            if (s3 > 0.f) add_point_row(P, fk, fk.o[j], j, coef, 1.f, row[k]);
        }
        const float4 p3 = P.j3d[j];
        const float tgt[3] = {p3.x, p3.y, p3.z};
        for (int k = 0; k < 3; ++k) {
            const int r = 2 * J + 3 * j + k;
            P.F[r] = s3 * (fk.o[j][k] - tgt[k]);
            for (int c = 0; c < nd; ++c) P.Jm[(size_t)c * ld + r] = row[k][c];
        }
    } else {
        const int i = P.blist[t - 2 * J];
        const int r = 5 * J + (t - 2 * J);
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
        for (int c = 0; c < nd; ++c) row[0][c] = 0.f;
        float res = 0.f;
        const float2 uv = project_exact(C.f, C.cx, C.cy, X, Y, Z);
        if (valid_depth(Z) && in_image(uv, C.W, C.H)) {
            float gx, gy;
            const float d = dt_sample(C, uv.x, uv.y, gx, gy).x;
            const float ss = sqrtf(P.lam_sil / (float)max(nB, 1));
            res = ss * d;
            const float bs = (C.flags[i] & LC_BNEG_BIT) ? -ss : ss;
            const float iz = 1.f / Z, fz = C.f * iz;
            const float coef[3] = {bs * gx * fz, bs * gy * fz, -bs * fz * iz * (gx * X + gy * Y)};
#pragma unroll
            for (int s = 0; s < 4; ++s) add_point_row(P, fk, Pt[s], bones[s], coef, ws[s], row[0]);
        }
        P.F[r] = res;
        for (int c = 0; c < nd; ++c) P.Jm[(size_t)c * ld + r] = row[0][c];
    }
}

// ---------------------------------------------------------------------------
// normal equations + FP64 Cholesky + update (one CTA)
// ---------------------------------------------------------------------------
constexpr int kSolveThreads = 1024;
constexpr int kChunkRows = 32;

__global__ void __launch_bounds__(kSolveThreads) pose_solve_kernel(const PoseDesc* __restrict__ pd, int slot,
                                                                  int mode) {
    __shared__ float sJ[(kMaxDof + 1) * kChunkRows];
    __shared__ double A[kMaxDof][kMaxDof + 1];
    __shared__ double x[kMaxDof];
    __shared__ unsigned char pa[(kMaxDof + 1) * (kMaxDof + 2) / 2], pb[(kMaxDof + 1) * (kMaxDof + 2) / 2];
    __shared__ float s_ftf;
    __shared__ double s_inv;
    __shared__ int s_bad;
    const PoseDesc& P = *pd;
    const int nd = P.n_dof, ld = P.max_rows;
    const int nrows = 5 * P.J + *P.bcount;
    const int tid = threadIdx.x;
    const int na = nd + 1;                          // augmented with F
    const int npairs = na * (na + 1) / 2;
    if (tid == 0) {
        int p = 0;
        for (int a = 0; a < na; ++a)
            for (int b = a; b < na; ++b) {
                pa[p] = (unsigned char)a;
                pb[p] = (unsigned char)b;
                ++p;
            }
        s_bad = 0;
    }
    __syncthreads();
    // pairs (a <= b) of the augmented matrix [J | F]: FP32 dot products over
    // the rows, in a fixed order
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
    for (int r0 = 0; r0 < nrows; r0 += kChunkRows) {
        const int rn = min(kChunkRows, nrows - r0);
        for (int q = tid; q < na * kChunkRows; q += kSolveThreads) {
            const int c = q / kChunkRows, r = q % kChunkRows;
            float v = 0.f;
            if (r < rn) v = c < nd ? P.Jm[(size_t)c * ld + r0 + r] : P.F[r0 + r];
            sJ[c * kChunkRows + r] = v;
        }
        __syncthreads();
        if (tid < npairs) {
            const float* ca = &sJ[pa[tid] * kChunkRows];
            const float* cb = &sJ[pb[tid] * kChunkRows];
            for (int r = 0; r < rn; ++r) acc0 += ca[r] * cb[r];
        }
        if (tid + kSolveThreads < npairs) {
            const float* ca = &sJ[pa[tid + kSolveThreads] * kChunkRows];
            const float* cb = &sJ[pb[tid + kSolveThreads] * kChunkRows];
            for (int r = 0; r < rn; ++r) acc1 += ca[r] * cb[r];
        }
        if (tid + 2 * kSolveThreads < npairs) {
            const float* ca = &sJ[pa[tid + 2 * kSolveThreads] * kChunkRows];
            const float* cb = &sJ[pb[tid + 2 * kSolveThreads] * kChunkRows];
            for (int r = 0; r < rn; ++r) acc2 += ca[r] * cb[r];
        }
        __syncthreads();
    }
    // scatter into the FP64 system: A (nd x nd) and g = -J^T F in column nd
    auto put = [&](int p, float v) {
        if (p >= npairs) return;
        const int a = pa[p], b = pb[p];
        if (b < nd) {
            A[a][b] = (double)v;
            A[b][a] = (double)v;
        } else if (a < nd) {
            A[a][nd] = -(double)v;
        } else {
            s_ftf = v;   // F^T F
        }
    };
    put(tid, acc0);
    put(tid + kSolveThreads, acc1);
    put(tid + 2 * kSolveThreads, acc2);
    __syncthreads();
    // angle prior: lprior (theta - theta_start) on the Euler DOF
    double prior_e = 0.0;
    if (tid == 0) {
        for (int c = 6; c < nd; ++c) {
            const double dv = (double)P.pose[c] - (double)P.pose_start[c];
            A[c][c] += (double)P.lam_prior;
            A[c][nd] -= (double)P.lam_prior * dv;
            prior_e += (double)P.lam_prior * dv * dv;
        }
        P.hist[2 * slot] = (double)s_ftf + prior_e;
    }
    __syncthreads();
    if (mode == 1) return;
    if (mode == 2) {
        for (int q = tid; q < nd * (nd + 1); q += kSolveThreads) P.expA[q] = A[q / (nd + 1)][q % (nd + 1)];
        return;
    }
    // Cholesky, lower triangle in place (FP64)
    for (int k = 0; k < nd; ++k) {
        if (tid == 0) {
            const double d = A[k][k];
            if (!(d > 0.0)) s_bad = 1;
            A[k][k] = d > 0.0 ? sqrt(d) : 1.0;
            s_inv = 1.0 / A[k][k];
        }
        __syncthreads();
        const double inv = s_inv;
        for (int i = k + 1 + tid; i < nd; i += kSolveThreads) A[i][k] *= inv;
        __syncthreads();
        const int m = nd - k - 1;
        for (int q = tid; q < m * m; q += kSolveThreads) {
            const int i = k + 1 + q / m, j = k + 1 + q % m;
            if (j <= i) A[i][j] -= A[i][k] * A[j][k];
        }
        __syncthreads();
    }
    // forward / back substitution by one warp
    if (tid < 32) {
        for (int i = 0; i < nd; ++i) {
            double s = 0.0;
            for (int j = tid; j < i; j += 32) s += A[i][j] * x[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (tid == 0) x[i] = (A[i][nd] - s) / A[i][i];
            __syncwarp();
        }
        for (int i = nd - 1; i >= 0; --i) {
            double s = 0.0;
            for (int j = i + 1 + tid; j < nd; j += 32) s += A[j][i] * x[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (tid == 0) x[i] = (x[i] - s) / A[i][i];
            __syncwarp();
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (s_bad) {
            *P.status = 1;
            P.hist[2 * slot + 1] = 0.0;
            return;
        }
        double n2 = 0.0;
        for (int c = 0; c < nd; ++c) n2 += x[c] * x[c];
        P.hist[2 * slot + 1] = sqrt(n2);
        for (int c = 3; c < nd; ++c) P.pose[c] += (float)x[c];
        // R <- Exp(d_omega) R (Rodrigues, FP32)
        const float wx = (float)x[0], wy = (float)x[1], wz = (float)x[2];
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

// ---------------------------------------------------------------------------
void launch_pose_skin(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, float4* out_base, int mode,
                      cudaStream_t st) {
    pose_skin_kernel<<<(hC.N + 255) / 256, 256, 0, st>>>(dC, dP, out_base, mode);
}
void launch_pose_blist(const CapDesc* dC, const PoseDesc* dP, cudaStream_t st) {
    pose_blist_kernel<<<1, 1024, 0, st>>>(dC, dP);
}
void launch_pose_dirs(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, cudaStream_t st) {
    pose_skin_kernel<<<(hC.N + 255) / 256, 256, 0, st>>>(dC, dP, nullptr, 0);
    pose_dirs_kernel<<<(hC.N + 255) / 256, 256, 0, st>>>(dC, dP);
}
void launch_pose_rows(const CapDesc* dC, const CapDesc& hC, const PoseDesc* dP, int J, cudaStream_t st) {
    const int maxt = 2 * J + hC.N;
    pose_rows_kernel<<<(maxt + 255) / 256, 256, 0, st>>>(dC, dP);
}
void launch_pose_solve(const PoseDesc* dP, int slot, int mode, cudaStream_t st) {
    pose_solve_kernel<<<1, kSolveThreads, 0, st>>>(dP, slot, mode);
}

}  // namespace lc

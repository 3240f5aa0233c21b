/*
 * Visibility, contour set and silhouette directions — exact-arithmetic oracle.
 * TEST INFRASTRUCTURE ONLY: nothing in the library links this file.
 *
 * The paper obtains visibility by depth buffering once per frame (Sec. 3.4,
 * photometric term), extracts contour vertices B once per frame (Sec. 3.3,
 * silhouette term) and sets b_i = -1 where the projected model normal n and
 * z = -grad(I_DT) satisfy n^T z < 0, else +1.  These are integer decisions, so
 * they are specified in exact integer arithmetic plus a fixed sequence of
 * IEEE FP32 operations (each rounded, no contraction; build with
 * -ffp-contract=off) that any implementation can reproduce bit for bit:
 *
 *  projection   u = (f*X)/Z + cx, v = (f*Y)/Z + cy; valid iff Z > 1e-3.
 *  snapping     su = rint(u*256) as int64 (round half to even); same for v.
 *               Vertices with |u| or |v| >= 2^20 are treated as invalid.
 *  coverage     pixel centre (px,py) in 1/256 fixed point; edge functions in
 *               int64; both windings (sign-normalised); top-left tie rule:
 *               an edge (ex,ey) owns its zero set iff ey < 0 || (ey == 0 && ex > 0).
 *  depth        b_j = (float)w_j / (float)area;
 *               depth = 1 / ((b0/z0 + b1/z1) + b2/z2).
 *  key          (bits(depth) << 32) | triangle id; per-pixel minimum.
 *  visibility   p = (rint(u), rint(v)); visible iff valid, u in [0,W-1],
 *               v in [0,H-1], and (pixel empty or Z <= depth(p) + eps).
 *  contour      mesh edge is a silhouette edge iff its two triangles differ in
 *               (snapped int64 area > 0); an edge with one triangle always is.
 *               B = visible vertices on a silhouette edge whose pixel p lies
 *               on the model's projected outline: some pixel of the 3x3
 *               block around p is outside the image or not covered by any
 *               triangle (internal occluding contours are not part of the
 *               model silhouette).
 *  direction    n_i = sum over incident triangles, increasing id, of
 *               cross(B-A, C-A) (component order x,y,z; each product rounded,
 *               then the difference).  m = (nx - (X/Z)*nz, ny - (Y/Z)*nz).
 *               g = bilinear sample of the central-difference DT gradient at
 *               (u,v) with lerp(a,b,t) = a + t*(b-a).  d = mx*gx + my*gy.
 *               The direction rule only concerns model points that fall
 *               inside the image silhouette (Sec. 3.3: outside points are
 *               always pulled toward the silhouette): b_i = -1 iff the
 *               foreground mask is set at p = (rint(u), rint(v)) and
 *               n^T z < 0, which with z = -g is d > 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FLAG_VISIBLE 1u
#define FLAG_ONSIL 2u
#define FLAG_INB 4u
#define FLAG_BNEG 8u

static int snap(float x, int64_t *out) {
    if (!(fabsf(x) < 1048576.0f)) return 0;
    float s = x * 256.0f;                 /* exact: power-of-two scaling */
    *out = (int64_t)rintf(s);
    return 1;
}

static float lerpf(float a, float b, float t) {
    float d = b - a;
    float m = t * d;
    return a + m;
}

static float grad_x(const float *D, int W, int x, int y) {
    const float *row = D + (int64_t)y * W;
    if (W < 2) return 0.0f;
    if (x == 0) return row[1] - row[0];
    if (x == W - 1) return row[W - 1] - row[W - 2];
    return (row[x + 1] - row[x - 1]) * 0.5f;
}

static float grad_y(const float *D, int W, int H, int x, int y) {
    if (H < 2) return 0.0f;
    if (y == 0) return D[(int64_t)1 * W + x] - D[x];
    if (y == H - 1) return D[(int64_t)(H - 1) * W + x] - D[(int64_t)(H - 2) * W + x];
    return (D[(int64_t)(y + 1) * W + x] - D[(int64_t)(y - 1) * W + x]) * 0.5f;
}

/* owned zero set of an edge under the top-left rule */
static int owns(int64_t ex, int64_t ey) { return ey < 0 || (ey == 0 && ex > 0); }

/* area-weighted vertex normals, incident triangles in increasing id order */
static void vertex_normals(const float *V, const int32_t *F, int T, int N, float *nrm) {
    for (int i = 0; i < 3 * N; ++i) nrm[i] = 0.0f;
    for (int t = 0; t < T; ++t) {
        int ia = F[3 * t], ib = F[3 * t + 1], ic = F[3 * t + 2];
        float e1x = V[3 * ib] - V[3 * ia], e1y = V[3 * ib + 1] - V[3 * ia + 1], e1z = V[3 * ib + 2] - V[3 * ia + 2];
        float e2x = V[3 * ic] - V[3 * ia], e2y = V[3 * ic + 1] - V[3 * ia + 1], e2z = V[3 * ic + 2] - V[3 * ia + 2];
        float p1, p2;
        p1 = e1y * e2z; p2 = e1z * e2y; float cxv = p1 - p2;
        p1 = e1z * e2x; p2 = e1x * e2z; float cyv = p1 - p2;
        p1 = e1x * e2y; p2 = e1y * e2x; float czv = p1 - p2;
        int vv[3] = {ia, ib, ic};
        for (int k = 0; k < 3; ++k) {
            nrm[3 * vv[k]] = nrm[3 * vv[k]] + cxv;
            nrm[3 * vv[k] + 1] = nrm[3 * vv[k] + 1] + cyv;
            nrm[3 * vv[k] + 2] = nrm[3 * vv[k] + 2] + czv;
        }
    }
}

/* b_i = -1 rule for vertex i (projection uv must be valid and in the image):
 * returns 1 iff the foreground mask is set at rint(uv) and d > 0 */
static int direction_neg(const float *V, const int32_t *F, int T, const float *nrm, const float *uv, int W, int H,
                         const float *DT, const uint8_t *mask, int i) {
    (void)F; (void)T;
    float X = V[3 * i], Y = V[3 * i + 1], Z = V[3 * i + 2];
    float xz = X / Z, yz = Y / Z;
    float t1 = xz * nrm[3 * i + 2]; float mx = nrm[3 * i] - t1;
    float t2 = yz * nrm[3 * i + 2]; float my = nrm[3 * i + 1] - t2;
    float u = uv[2 * i], v = uv[2 * i + 1];
    int x0 = (int)floorf(u), y0 = (int)floorf(v);
    float fx = u - (float)x0, fy = v - (float)y0;
    int x1 = x0 + 1 < W ? x0 + 1 : W - 1;
    int y1 = y0 + 1 < H ? y0 + 1 : H - 1;
    float gx = lerpf(lerpf(grad_x(DT, W, x0, y0), grad_x(DT, W, x1, y0), fx),
                     lerpf(grad_x(DT, W, x0, y1), grad_x(DT, W, x1, y1), fx), fy);
    float gy = lerpf(lerpf(grad_y(DT, W, H, x0, y0), grad_y(DT, W, H, x1, y0), fx),
                     lerpf(grad_y(DT, W, H, x0, y1), grad_y(DT, W, H, x1, y1), fx), fy);
    float q1 = mx * gx; float q2 = my * gy; float d = q1 + q2;
    int64_t px = (int64_t)rintf(u), py = (int64_t)rintf(v);
    int inside = mask[py * W + px] != 0;
    return inside && d > 0.0f;
}

/* Directions b_i of the vertices flagged in `sel` at the surface V (the
 * contour set B stays that of the frame; b_i follows the current surface):
 * bneg[i] = 1 iff b_i = -1.  Vertices whose projection is invalid or
 * outside the image get 0 (they carry no residual). */
void oracle_directions(const float *V, int N, const int32_t *F, int T, float f, float cx, float cy, int W, int H,
                       const float *DT, const uint8_t *mask, const uint8_t *sel, uint8_t *bneg) {
    float *nrm = (float *)malloc(sizeof(float) * 3 * (size_t)(N > 0 ? N : 1));
    float *uv = (float *)malloc(sizeof(float) * 2 * (size_t)(N > 0 ? N : 1));
    vertex_normals(V, F, T, N, nrm);
    for (int i = 0; i < N; ++i) {
        bneg[i] = 0;
        if (!sel[i]) continue;
        float X = V[3 * i], Y = V[3 * i + 1], Z = V[3 * i + 2];
        if (!(Z > 1e-3f)) continue;
        float a = f * X; float b = a / Z; float u = b + cx;
        float c = f * Y; float d = c / Z; float v = d + cy;
        uv[2 * i] = u; uv[2 * i + 1] = v;
        if (!(u >= 0.0f && u <= (float)(W - 1) && v >= 0.0f && v <= (float)(H - 1))) continue;
        bneg[i] = (uint8_t)direction_neg(V, F, T, nrm, uv, W, H, DT, mask, i);
    }
    free(nrm);
    free(uv);
}

/*
 * V: N*3 FP32 warped positions.  F: T*3 triangles.  E: NE*4 mesh edges
 * (v0, v1, t0, t1) with t1 = -1 for a boundary edge.  DT, mask: H*W.
 * Outputs: uv (N*2), zbuf (H*W), flags (N).
 */
void oracle_visibility(const float *V, int N, const int32_t *F, int T,
                       const int32_t *E, int NE,
                       float f, float cx, float cy, int W, int H,
                       const float *DT, const uint8_t *mask, float eps,
                       float *uv, uint64_t *zbuf, uint8_t *flags) {
    int64_t P = (int64_t)W * H;
    for (int64_t i = 0; i < P; ++i) zbuf[i] = ~(uint64_t)0;
    /* projection + snapping */
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(N > 0 ? N : 1));
    uint8_t *ok = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
    float *nrm = (float *)malloc(sizeof(float) * 3 * (size_t)(N > 0 ? N : 1));
    for (int i = 0; i < N; ++i) {
        float X = V[3 * i], Y = V[3 * i + 1], Z = V[3 * i + 2];
        int valid = Z > 1e-3f;
        float u = 0.0f, v = 0.0f;
        if (valid) {
            float a = f * X; float b = a / Z; u = b + cx;
            float c = f * Y; float d = c / Z; v = d + cy;
        }
        uv[2 * i] = u; uv[2 * i + 1] = v;
        int64_t a0 = 0, a1 = 0;
        if (valid) valid = snap(u, &a0) && snap(v, &a1);
        S[2 * i] = a0; S[2 * i + 1] = a1;
        ok[i] = (uint8_t)valid;
        flags[i] = 0;
    }
    /* rasterise */
    for (int t = 0; t < T; ++t) {
        int ia = F[3 * t], ib = F[3 * t + 1], ic = F[3 * t + 2];
        if (!ok[ia] || !ok[ib] || !ok[ic]) continue;
        int64_t ax = S[2 * ia], ay = S[2 * ia + 1];
        int64_t bx = S[2 * ib], by = S[2 * ib + 1];
        int64_t qx = S[2 * ic], qy = S[2 * ic + 1];
        int64_t area = (bx - ax) * (qy - ay) - (by - ay) * (qx - ax);
        if (area == 0) continue;
        int64_t sg = area > 0 ? 1 : -1;
        int64_t lo_x = ax < bx ? ax : bx; lo_x = lo_x < qx ? lo_x : qx;
        int64_t hi_x = ax > bx ? ax : bx; hi_x = hi_x > qx ? hi_x : qx;
        int64_t lo_y = ay < by ? ay : by; lo_y = lo_y < qy ? lo_y : qy;
        int64_t hi_y = ay > by ? ay : by; hi_y = hi_y > qy ? hi_y : qy;
        /* pixel range: ceil(lo/256) .. floor(hi/256), clipped */
        int64_t px0 = lo_x >= 0 ? (lo_x + 255) / 256 : -((-lo_x) / 256);
        int64_t px1 = hi_x >= 0 ? hi_x / 256 : -((-hi_x + 255) / 256);
        int64_t py0 = lo_y >= 0 ? (lo_y + 255) / 256 : -((-lo_y) / 256);
        int64_t py1 = hi_y >= 0 ? hi_y / 256 : -((-hi_y + 255) / 256);
        if (px0 < 0) px0 = 0;
        if (py0 < 0) py0 = 0;
        if (px1 > W - 1) px1 = W - 1;
        if (py1 > H - 1) py1 = H - 1;
        /* edge vectors after sign normalisation: edge opposite A runs B->C */
        int64_t eAx = sg * (qx - bx), eAy = sg * (qy - by);
        int64_t eBx = sg * (ax - qx), eBy = sg * (ay - qy);
        int64_t eCx = sg * (bx - ax), eCy = sg * (by - ay);
        int oA = owns(eAx, eAy), oB = owns(eBx, eBy), oC = owns(eCx, eCy);
        float za = V[3 * ia + 2], zb = V[3 * ib + 2], zc = V[3 * ic + 2];
        float farea = (float)(sg * area);
        for (int64_t py = py0; py <= py1; ++py) {
            int64_t Py = py * 256;
            for (int64_t px = px0; px <= px1; ++px) {
                int64_t Px = px * 256;
                int64_t wA = sg * ((qx - bx) * (Py - by) - (qy - by) * (Px - bx));
                int64_t wB = sg * ((ax - qx) * (Py - qy) - (ay - qy) * (Px - qx));
                int64_t wC = sg * ((bx - ax) * (Py - ay) - (by - ay) * (Px - ax));
                if (wA < 0 || wB < 0 || wC < 0) continue;
                if ((wA == 0 && !oA) || (wB == 0 && !oB) || (wC == 0 && !oC)) continue;
                float b0 = (float)wA / farea;
                float b1 = (float)wB / farea;
                float b2 = (float)wC / farea;
                float s0 = b0 / za, s1 = b1 / zb, s2 = b2 / zc;
                float s01 = s0 + s1;
                float ssum = s01 + s2;
                float depth = 1.0f / ssum;
                uint32_t bits; memcpy(&bits, &depth, 4);
                uint64_t key = ((uint64_t)bits << 32) | (uint32_t)t;
                int64_t p = py * W + px;
                if (key < zbuf[p]) zbuf[p] = key;
            }
        }
    }
    /* per-vertex visibility */
    for (int i = 0; i < N; ++i) {
        if (!ok[i]) continue;
        float u = uv[2 * i], v = uv[2 * i + 1];
        if (!(u >= 0.0f && u <= (float)(W - 1) && v >= 0.0f && v <= (float)(H - 1))) continue;
        int64_t px = (int64_t)rintf(u), py = (int64_t)rintf(v);
        uint64_t key = zbuf[py * W + px];
        int vis = 0;
        if (key == ~(uint64_t)0) vis = 1;
        else {
            uint32_t bits = (uint32_t)(key >> 32); float depth; memcpy(&depth, &bits, 4);
            float lim = depth + eps;
            vis = V[3 * i + 2] <= lim;
        }
        if (vis) flags[i] |= FLAG_VISIBLE;
    }
    /* silhouette edges */
    for (int e = 0; e < NE; ++e) {
        int v0 = E[4 * e], v1 = E[4 * e + 1], t0 = E[4 * e + 2], t1 = E[4 * e + 3];
        int front[2] = {0, 0};
        int tt[2] = {t0, t1};
        for (int k = 0; k < 2; ++k) {
            int t = tt[k];
            if (t < 0) continue;
            int ia = F[3 * t], ib = F[3 * t + 1], ic = F[3 * t + 2];
            if (!ok[ia] || !ok[ib] || !ok[ic]) continue;
            int64_t ax = S[2 * ia], ay = S[2 * ia + 1];
            int64_t bx = S[2 * ib], by = S[2 * ib + 1];
            int64_t qx = S[2 * ic], qy = S[2 * ic + 1];
            int64_t area = (bx - ax) * (qy - ay) - (by - ay) * (qx - ax);
            front[k] = area > 0;
        }
        int sil = (t1 < 0) ? 1 : (front[0] != front[1]);
        if (sil) { flags[v0] |= FLAG_ONSIL; flags[v1] |= FLAG_ONSIL; }
    }
    vertex_normals(V, F, T, N, nrm);
    for (int i = 0; i < N; ++i) {
        if (!((flags[i] & FLAG_VISIBLE) && (flags[i] & FLAG_ONSIL))) continue;
        {
            int64_t px = (int64_t)rintf(uv[2 * i]), py = (int64_t)rintf(uv[2 * i + 1]);
            int outline = 0;
            for (int dy = -1; dy <= 1 && !outline; ++dy)
                for (int dx = -1; dx <= 1 && !outline; ++dx) {
                    int64_t qx = px + dx, qy = py + dy;
                    if (qx < 0 || qy < 0 || qx >= W || qy >= H) outline = 1;
                    else if (zbuf[qy * W + qx] == ~(uint64_t)0) outline = 1;
                }
            if (!outline) continue;
        }
        flags[i] |= FLAG_INB;
        if (direction_neg(V, F, T, nrm, uv, W, H, DT, mask, i)) flags[i] |= FLAG_BNEG;
    }
    free(S);
    free(ok);
    free(nrm);
}

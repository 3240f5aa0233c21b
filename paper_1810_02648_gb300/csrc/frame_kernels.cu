#include <algorithm>
// Frame preparation, embedded-graph warp + projection, and the once-per-frame
// visibility / contour pass.
//
// Visibility comes from depth buffering (Sec. 3.4, photometric term), the
// contour set B and the directions b_i from Sec. 3.3 (silhouette term, the
// n^T z < 0 rule for model points inside the image silhouette).  These are
// integer decisions taken in exact integer arithmetic plus a fixed sequence
// of FP32 operations (intrinsics: every operation rounded once, nothing
// contracted), so the result is reproducible bit for bit:
//   snapping: 1/256 px fixed point, round half to even; int64 edge functions
//   with a top-left tie rule, both windings; FP32 perspective-correct depth
//   1 / ((b0/z0 + b1/z1) + b2/z2); key = bits(depth) << 32 | triangle id,
//   resolved with a 64-bit atomicMin.
#include <cstddef>

#include "lc_internal.cuh"

namespace lc {

// ---------------------------------------------------------------------------
// Frame packing: (r, g, b) + dt -> float4 per pixel; mask copied.
// ---------------------------------------------------------------------------
__global__ void pack_frame_kernel(const float* __restrict__ rgb, const float* __restrict__ dt,
                                  const uint8_t* __restrict__ mask_in, float4* __restrict__ img,
                                  uint8_t* __restrict__ mask, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    img[p] = make_float4(rgb[3 * p], rgb[3 * p + 1], rgb[3 * p + 2], dt ? dt[p] : 0.f);   // dt null: computed next
    mask[p] = mask_in[p] ? 1 : 0;
}

void launch_pack_frame(const float* rgb, const float* dt, const uint8_t* mask_in, float4* img, uint8_t* mask,
                       int W, int H, cudaStream_t st) {
    const int P = W * H;
    pack_frame_kernel<<<(P + 255) / 256, 256, 0, st>>>(rgb, dt, mask_in, img, mask, P);
}

// ---------------------------------------------------------------------------
// Silhouette distance transform (Sec. 3.2), exact: the squared Euclidean
// distance to the nearest contour pixel (a foreground pixel with a
// 4-neighbour in the background or on the image border) in integers, by the
// separable decomposition d^2(x, y) = min_i (x - i)^2 + g(i, y)^2 with
// g(i, y) the distance along column i to its nearest contour pixel:
//   phase 0, one thread per pixel: the contour flags;
//   phase 1, a CTA per 8 columns, 128 row chunks each: every thread finds the
//     last / first contour row of its chunk, the chunks are combined through
//     shared memory, then every thread writes g for its chunk;
//   phase 2, a CTA per row with g^2 of the row and its minimum over every 32
//     columns in shared memory: every pixel scans its own 32-column block,
//     then the blocks outward, skipping a block when its nearest column's
//     distance^2 plus the block's minimum g^2 cannot beat the best so far,
//     and stopping where the distance^2 alone cannot.
// I_DT = sqrt(d^2) rounded once to FP32, written into the frame's fourth
// channel; 0 everywhere when the silhouette has no contour.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) edt_contour_kernel(const uint8_t* __restrict__ m, int W, int H,
                                                          uint8_t* __restrict__ c) {
    const size_t P = (size_t)W * H;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(p / W), x = (int)(p - (size_t)y * W);
        bool on = m[p] != 0;
        if (on && x > 0 && y > 0 && x < W - 1 && y < H - 1)
            on = !m[p - 1] || !m[p + 1] || !m[p - W] || !m[p + W];
        c[p] = on ? 1 : 0;
    }
}

constexpr int kEdtCols = 8, kEdtChunks = 128;

__global__ void __launch_bounds__(kEdtCols * kEdtChunks) edt_columns_kernel(const uint8_t* __restrict__ c,
                                                                             int* __restrict__ g, int W, int H) {
    __shared__ int s_last[kEdtChunks][kEdtCols], s_first[kEdtChunks][kEdtCols];
    const int tx = threadIdx.x % kEdtCols, ty = threadIdx.x / kEdtCols;
    const int x = blockIdx.x * kEdtCols + tx;
    const int L = (H + kEdtChunks - 1) / kEdtChunks;
    const int y0 = min(H, ty * L), y1 = min(H, y0 + L);
    const int NONE_LO = -(W + H) - 1, NONE_HI = 2 * (W + H) + 1;
    int last = NONE_LO, first = NONE_HI;
    if (x < W)
        for (int y = y0; y < y1; ++y)
            if (c[(size_t)y * W + x]) {
                if (first == NONE_HI) first = y;
                last = y;
            }
    s_last[ty][tx] = last;
    s_first[ty][tx] = first;
    __syncthreads();
    // the nearest contour rows above this chunk and below it
    int above = NONE_LO, below = NONE_HI;
    for (int k = 0; k < ty; ++k) above = max(above, s_last[k][tx]);
    for (int k = kEdtChunks - 1; k > ty; --k) below = min(below, s_first[k][tx]);
    if (x >= W) return;
    const int inf = W + H;
    // down the chunk with the last contour row so far, then up it
    int lastc = above;
    for (int y = y0; y < y1; ++y) {
        if (c[(size_t)y * W + x]) lastc = y;
        g[(size_t)y * W + x] = min(inf, y - lastc);
    }
    int nextc = below;
    for (int y = y1 - 1; y >= y0; --y) {
        const int v = g[(size_t)y * W + x];
        if (v == 0) nextc = y;
        const int d = min(inf, nextc - y);
        if (d < v) g[(size_t)y * W + x] = d;
    }
}

constexpr int kEdtBlock = 32;

__device__ __forceinline__ int edt_scan_block(const int* s_g2, int W, int x, int b, int best) {
    const int i0 = b * kEdtBlock, i1 = min(W, i0 + kEdtBlock);
    for (int i = i0; i < i1; ++i) {
        const int d = x - i;
        best = min(best, d * d + s_g2[i]);
    }
    return best;
}

__global__ void __launch_bounds__(256) edt_rows_kernel(const int* __restrict__ g, float4* __restrict__ img, int W,
                                                       int H) {
    extern __shared__ int s_g2[];   // g^2 of this row, then the block minima
    const int nb = (W + kEdtBlock - 1) / kEdtBlock;
    int* s_bmin = s_g2 + W;
    const int y = blockIdx.x;
    const int* gy = g + (size_t)y * W;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const int v = gy[x];
        s_g2[x] = v * v;   // (W + H)^2 when the column has no contour
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        int m = s_g2[b * kEdtBlock];
        for (int i = b * kEdtBlock + 1; i < min(W, (b + 1) * kEdtBlock); ++i) m = min(m, s_g2[i]);
        s_bmin[b] = m;
    }
    __syncthreads();
    const int inf = W + H;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const int bx = x / kEdtBlock;
        int best = edt_scan_block(s_g2, W, x, bx, s_g2[x]);
        for (int j = 1;; ++j) {
            bool more = false;
            const int bl = bx - j, br = bx + j;
            if (bl >= 0) {
                const int dl = x - (bl * kEdtBlock + kEdtBlock - 1);
                if (dl * dl < best) {
                    more = true;
                    if (dl * dl + s_bmin[bl] < best) best = edt_scan_block(s_g2, W, x, bl, best);
                }
            }
            if (br < nb) {
                const int dr = br * kEdtBlock - x;
                if (dr * dr < best) {
                    more = true;
                    if (dr * dr + s_bmin[br] < best) best = edt_scan_block(s_g2, W, x, br, best);
                }
            }
            if (!more) break;
        }
        img[(size_t)y * W + x].w = best >= inf * inf ? 0.f : sqrtf((float)best);
    }
}

void launch_edt(const uint8_t* mask, uint8_t* contour, int* g, float4* img, int W, int H, cudaStream_t st) {
    const size_t P = (size_t)W * H;
    const int nb = (W + kEdtBlock - 1) / kEdtBlock;
    const size_t smem = sizeof(int) * (W + nb);
    if (smem > 48 * 1024) cudaFuncSetAttribute(edt_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    edt_contour_kernel<<<(int)std::min<size_t>((P + 255) / 256, 4096), 256, 0, st>>>(mask, W, H, contour);
    edt_columns_kernel<<<(W + kEdtCols - 1) / kEdtCols, kEdtCols * kEdtChunks, 0, st>>>(contour, g, W, H);
    edt_rows_kernel<<<H, 256, smem, st>>>(g, img, W, H);
}

// ---------------------------------------------------------------------------
// Photometric pyramid (Sec. 3.4: a 3-level pyramid of the input image, each
// level Gaussian blurred).  Level pixel (x, y) with factor d is the FP32 mean
// of the frame's pixels in [d x, d x + d) x [d y, d y + d) inside the image
// (rows then columns, in order); the blur is separable, rows first, taps
// applied from -r to r with clamp to edge.  Channels r, g, b; the fourth is 0.
// ---------------------------------------------------------------------------
__global__ void pyr_down_kernel(const float4* __restrict__ img, int W, int H, int d, float4* __restrict__ out,
                                int Wd, int Hd) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= Wd || y >= Hd) return;
    const int x0 = x * d, y0 = y * d, x1 = min(W, x0 + d), y1 = min(H, y0 + d);
    float r = 0.f, g = 0.f, b = 0.f;
    for (int yy = y0; yy < y1; ++yy)
        for (int xx = x0; xx < x1; ++xx) {
            const float4 p = __ldg(&img[(size_t)yy * W + xx]);
            r += p.x;
            g += p.y;
            b += p.z;
        }
    const float c = (float)((x1 - x0) * (y1 - y0));
    out[(size_t)y * Wd + x] = make_float4(r / c, g / c, b / c, 0.f);
}

template <bool kRows>
__global__ void pyr_blur_kernel(const float4* __restrict__ in, int W, int H, const PyrTaps T,
                                float4* __restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    float r = 0.f, g = 0.f, b = 0.f;
    for (int i = -T.r; i <= T.r; ++i) {
        const int xs = kRows ? min(max(x + i, 0), W - 1) : x;
        const int ys = kRows ? y : min(max(y + i, 0), H - 1);
        const float4 p = __ldg(&in[(size_t)ys * W + xs]);
        const float w = T.w[i + T.r];
        r += w * p.x;
        g += w * p.y;
        b += w * p.z;
    }
    out[(size_t)y * W + x] = make_float4(r, g, b, 0.f);
}

void launch_pyramid_level(const float4* img, int W, int H, int d, const PyrTaps& taps, float4* tmp, float4* out,
                          int Wd, int Hd, cudaStream_t st) {
    const dim3 blk(32, 8), grd((Wd + 31) / 32, (Hd + 7) / 8);
    const float4* src = img;
    if (d > 1) {
        pyr_down_kernel<<<grd, blk, 0, st>>>(img, W, H, d, out, Wd, Hd);
        src = out;
    }
    pyr_blur_kernel<true><<<grd, blk, 0, st>>>(src, Wd, Hd, taps, tmp);
    pyr_blur_kernel<false><<<grd, blk, 0, st>>>(tmp, Wd, Hd, taps, out);
}

// ---------------------------------------------------------------------------
// Warp + project: v'_i = v_i + sum_s w_is ((R_k - I)(v_i - g_k) + t_k).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kVertTile) warp_kernel(const CapDesc* __restrict__ caps,
                                                          const WorkItem* __restrict__ items, int gated) {
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (gated && C.sc->gn_stop) return;
    const int i = tile * kVertTile + threadIdx.x;
    if (i >= C.N) return;
    const float4 v = C.base[i];
    const int K = C.K;
    float dx = 0.f, dy = 0.f, dz = 0.f;
    for (int s = 0; s < K; ++s) {
        const int k = C.bind_idx[(size_t)i * K + s];
        const float w = C.bind_w[(size_t)i * K + s];
        const float4 g = C.node_g[k];
        const float4 r0 = C.node_R[3 * k], r1 = C.node_R[3 * k + 1], r2 = C.node_R[3 * k + 2];
        const float4 t = C.node_t[k];
        const float ax = v.x - g.x, ay = v.y - g.y, az = v.z - g.z;
        const float mx = (r0.x - 1.f) * ax + r0.y * ay + r0.z * az + t.x;
        const float my = r1.x * ax + (r1.y - 1.f) * ay + r1.z * az + t.y;
        const float mz = r2.x * ax + r2.y * ay + (r2.z - 1.f) * az + t.z;
        dx += w * mx;
        dy += w * my;
        dz += w * mz;
    }
    const float X = v.x + dx, Y = v.y + dy, Z = v.z + dz;
    const bool ok = valid_depth(Z);
    C.vw[i] = make_float4(X, Y, Z, ok ? 1.f : 0.f);
    C.uv[i] = ok ? project_exact(C.f, C.cx, C.cy, X, Y, Z) : make_float2(0.f, 0.f);
}

void launch_warp(const CapDesc* dC, const Tiles& T, cudaStream_t st, bool gated) {
    warp_kernel<<<T.vert, kVertTile, 0, st>>>(dC, T.vert_items, gated ? 1 : 0);
}
void launch_warp(const CapDesc* dC, const CapDesc& hC, cudaStream_t st, bool gated) {
    launch_warp(dC, single_tiles(hC), st, gated);
}

// ---------------------------------------------------------------------------
// Rasteriser
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool snap(float x, long long& out) {
    if (!(fabsf(x) < 1048576.0f)) return false;
    out = __float2ll_rn(xmul(x, 256.0f));
    return true;
}

__device__ __forceinline__ bool vertex_snap(const CapDesc& C, int i, long long& sx, long long& sy) {
    const float4 v = C.vw[i];
    if (!(v.w > 0.f)) return false;
    const float2 uv = C.uv[i];
    return snap(uv.x, sx) && snap(uv.y, sy);
}

__device__ __forceinline__ bool owns(long long ex, long long ey) { return ey < 0 || (ey == 0 && ex > 0); }

__device__ __forceinline__ long long ceil256(long long a) { return a >= 0 ? (a + 255) / 256 : -((-a) / 256); }
__device__ __forceinline__ long long floor256(long long a) { return a >= 0 ? a / 256 : -((-a + 255) / 256); }

// Triangle setup shared by a warp: each thread sets up one triangle, then
// the warp rasterises its 32 triangles one after the other, the lanes taking
// the pixels of the bounding box in turn (a warp's time is the sum of its
// triangles' box areas / 32 instead of the largest box).
struct TriSetup {
    long long ax, ay, bx, by, qx, qy;
    int px0, py0, w, npix;   // box origin, width, pixel count (0: nothing to draw)
    float za, zb, zc, farea;
    int sg, own, t, pad;
};

// A warp rasterises kTriPerWarp triangles: each is set up by one lane, then
// the warp's lanes take the pixels of its bounding box in turn.  Few triangles
// per warp keep many warps in flight (the per-pixel work is a chain of int64
// edge functions and exact divisions).
constexpr int kTriPerWarp = 8;
constexpr int kRasterThreads = kTriTile / kTriPerWarp * 32;

__global__ void __launch_bounds__(kRasterThreads) raster_kernel(const CapDesc* __restrict__ caps,
                                                                const WorkItem* __restrict__ items) {
    __shared__ TriSetup su[kTriTile];
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = warp * kTriPerWarp + lane;
    const int t = tile * kTriTile + slot;
    TriSetup& S = su[lane < kTriPerWarp ? slot : 0];
    if (lane < kTriPerWarp) S.npix = 0;
    if (lane < kTriPerWarp && t < C.F && !C.sc->vis_frozen) {
        const int4 tri = C.tris[t];
        long long ax, ay, bx, by, qx, qy;
        if (vertex_snap(C, tri.x, ax, ay) && vertex_snap(C, tri.y, bx, by) && vertex_snap(C, tri.z, qx, qy)) {
            const long long area = (bx - ax) * (qy - ay) - (by - ay) * (qx - ax);
            if (area != 0) {
                const long long sg = area > 0 ? 1 : -1;
                long long px0 = ceil256(min(ax, min(bx, qx))), px1 = floor256(max(ax, max(bx, qx)));
                long long py0 = ceil256(min(ay, min(by, qy))), py1 = floor256(max(ay, max(by, qy)));
                px0 = max(px0, 0LL);
                py0 = max(py0, 0LL);
                px1 = min(px1, (long long)C.W - 1);
                py1 = min(py1, (long long)C.H - 1);
                if (px0 <= px1 && py0 <= py1) {
                    S.ax = ax; S.ay = ay; S.bx = bx; S.by = by; S.qx = qx; S.qy = qy;
                    S.px0 = (int)px0;
                    S.py0 = (int)py0;
                    S.w = (int)(px1 - px0 + 1);
                    S.npix = S.w * (int)(py1 - py0 + 1);
                    S.own = (owns(sg * (qx - bx), sg * (qy - by)) ? 1 : 0) | (owns(sg * (ax - qx), sg * (ay - qy)) ? 2 : 0) |
                            (owns(sg * (bx - ax), sg * (by - ay)) ? 4 : 0);
                    S.za = C.vw[tri.x].z;
                    S.zb = C.vw[tri.y].z;
                    S.zc = C.vw[tri.z].z;
                    S.farea = (float)(sg * area);
                    S.sg = (int)sg;
                    S.t = t;
                }
            }
        }
    }
    __syncwarp();
    for (int src = 0; src < kTriPerWarp; ++src) {
        const TriSetup& T = su[warp * kTriPerWarp + src];
        const int npix = T.npix;
        if (npix == 0) continue;
        const long long ax = T.ax, ay = T.ay, bx = T.bx, by = T.by, qx = T.qx, qy = T.qy;
        const long long sg = T.sg;
        const bool oA = T.own & 1, oB = T.own & 2, oC = T.own & 4;
        for (int q = lane; q < npix; q += 32) {
            const int ry = q / T.w;
            const long long px = T.px0 + (q - ry * T.w), py = T.py0 + ry;
            const long long Px = px * 256, Py = py * 256;
            const long long wA = sg * ((qx - bx) * (Py - by) - (qy - by) * (Px - bx));
            const long long wB = sg * ((ax - qx) * (Py - qy) - (ay - qy) * (Px - qx));
            const long long wC = sg * ((bx - ax) * (Py - ay) - (by - ay) * (Px - ax));
            if (wA < 0 || wB < 0 || wC < 0) continue;
            if ((wA == 0 && !oA) || (wB == 0 && !oB) || (wC == 0 && !oC)) continue;
            const float b0 = xdiv(__ll2float_rn(wA), T.farea);
            const float b1 = xdiv(__ll2float_rn(wB), T.farea);
            const float b2 = xdiv(__ll2float_rn(wC), T.farea);
            const float s01 = xadd(xdiv(b0, T.za), xdiv(b1, T.zb));
            const float depth = xdiv(1.0f, xadd(s01, xdiv(b2, T.zc)));
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(depth) << 32) | (unsigned long long)(unsigned)T.t;
            atomicMin(&C.zbuf[py * C.W + px], key);
        }
    }
}

// per-vertex depth test; also resets the vertex flags
__global__ void __launch_bounds__(kVertTile) vis_kernel(const CapDesc* __restrict__ caps,
                                                         const WorkItem* __restrict__ items) {
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (C.sc->vis_frozen) return;   // the frame decisions were kept from the start
    const int i = tile * kVertTile + threadIdx.x;
    if (i >= C.N) return;
    uint32_t fl = 0;
    long long sx, sy;
    if (vertex_snap(C, i, sx, sy)) {
        const float2 uv = C.uv[i];
        if (in_image(uv, C.W, C.H)) {
            const long long px = __float2ll_rn(uv.x), py = __float2ll_rn(uv.y);
            const unsigned long long key = C.zbuf[py * C.W + px];
            bool vis = true;
            if (key != ~0ULL) {
                const float depth = __uint_as_float((unsigned)(key >> 32));
                vis = C.vw[i].z <= xadd(depth, C.eps_vis);
            }
            if (vis) fl |= LC_VIS_BIT;
        }
    }
    C.flags[i] = fl;
}

__device__ __forceinline__ bool front_facing(const CapDesc& C, int t) {
    const int4 tri = C.tris[t];
    long long ax, ay, bx, by, qx, qy;
    if (!vertex_snap(C, tri.x, ax, ay) || !vertex_snap(C, tri.y, bx, by) || !vertex_snap(C, tri.z, qx, qy))
        return false;
    return (bx - ax) * (qy - ay) - (by - ay) * (qx - ax) > 0;
}

__global__ void __launch_bounds__(kEdgeTile) silhouette_kernel(const CapDesc* __restrict__ caps,
                                                                const WorkItem* __restrict__ items) {
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (C.sc->vis_frozen) return;   // the frame decisions were kept from the start
    const int e = tile * kEdgeTile + threadIdx.x;
    if (e >= C.n_medges) return;
    const int4 me = C.medges[e];
    const bool sil = me.w < 0 ? true : (front_facing(C, me.z) != front_facing(C, me.w));
    if (sil) {
        atomicOr(&C.flags[me.x], LC_ONSIL_BIT);
        atomicOr(&C.flags[me.y], LC_ONSIL_BIT);
    }
}

// contour set B (visible vertices on a silhouette edge and on the model's
// projected outline) and the directions b_i
__global__ void __launch_bounds__(kVertTile) contour_kernel(const CapDesc* __restrict__ caps,
                                                             const WorkItem* __restrict__ items) {
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    if (C.sc->vis_frozen) return;   // the frame decisions were kept from the start
    const int i = tile * kVertTile + threadIdx.x;
    int cnt[3] = {0, 0, 0};
    if (i < C.N) {
        uint32_t fl = C.flags[i];
        if (fl & LC_VIS_BIT) cnt[0] = 1;
        if ((fl & LC_VIS_BIT) && (fl & LC_ONSIL_BIT)) {
            // only vertices on the model's projected outline: some pixel of
            // the 3x3 block around rint(uv) is outside the image or uncovered
            const float2 uv = C.uv[i];
            const long long px = __float2ll_rn(uv.x), py = __float2ll_rn(uv.y);
            bool outline = false;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const long long qx = px + dx, qy = py + dy;
                    if (qx < 0 || qy < 0 || qx >= C.W || qy >= C.H) outline = true;
                    else if (C.zbuf[qy * C.W + qx] == ~0ULL) outline = true;
                }
            if (outline) {
                fl |= LC_INB_BIT;
                cnt[1] = 1;
                if (direction_neg(C, i)) {
                    fl |= LC_BNEG_BIT;
                    cnt[2] = 1;
                }
                C.flags[i] = fl;
            }
        }
    }
    // vertex counts for the statistics (integer block sums)
    __shared__ int sh[3];
    if (threadIdx.x < 3) sh[threadIdx.x] = 0;
    __syncthreads();
    for (int j = 0; j < 3; ++j)
        if (cnt[j]) atomicAdd(&sh[j], 1);
    __syncthreads();
    if (threadIdx.x < 3 && sh[threadIdx.x]) atomicAdd(&C.sc->counts[threadIdx.x], sh[threadIdx.x]);
}

// raster, depth test, silhouette edges, contour set (the z-buffers must be
// cleared and the visibility counters zeroed before)
void launch_visibility_kernels(const CapDesc* dC, const Tiles& T, cudaStream_t st) {
    if (T.tri) raster_kernel<<<T.tri, kRasterThreads, 0, st>>>(dC, T.tri_items);
    vis_kernel<<<T.vert, kVertTile, 0, st>>>(dC, T.vert_items);
    if (T.medge) silhouette_kernel<<<T.medge, kEdgeTile, 0, st>>>(dC, T.medge_items);
    contour_kernel<<<T.vert, kVertTile, 0, st>>>(dC, T.vert_items);
}

// z-buffer cleared and visibility counters zeroed, unless the capture's
// frame decisions are frozen
__global__ void __launch_bounds__(256) vis_clear_kernel(const CapDesc* __restrict__ caps) {
    const CapDesc& C = caps[0];
    if (C.sc->vis_frozen) return;
    const size_t P = (size_t)C.W * C.H;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x)
        C.zbuf[p] = ~0ULL;
    if (blockIdx.x == 0 && threadIdx.x < 3) C.sc->counts[threadIdx.x] = 0;
}

__global__ void vis_unfreeze_kernel(const CapDesc* __restrict__ caps) { caps[0].sc->vis_frozen = 0; }

void launch_visibility(const CapDesc* dC, const CapDesc& hC, cudaStream_t st) {
    const size_t P = (size_t)hC.W * hC.H;
    const int blocks = (int)std::min<size_t>((P + 255) / 256, 2048);
    vis_clear_kernel<<<blocks, 256, 0, st>>>(dC);
    launch_visibility_kernels(dC, single_tiles(hC), st);
}

void launch_vis_unfreeze(const CapDesc* dC, cudaStream_t st) { vis_unfreeze_kernel<<<1, 1, 0, st>>>(dC); }

// ---------------------------------------------------------------------------
// Body-part mask of the silhouette term (Sec. 3.4): the rest geometry V^S is
// projected and rasterised into the z-buffer (the same exact rasteriser),
// each covered pixel takes the label of its front triangle (the label two
// or three of its vertices share, else the first vertex's), then every part
// grows into uncovered pixels within part_dilate pixels: the torso label if
// a torso pixel is within reach, else the nearest label, the lower one on
// equal squared distances.  The visibility pass of the current surface
// rasterises into the z-buffer again afterwards.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kVertTile) project_base_kernel(const CapDesc* __restrict__ caps) {
    const CapDesc& C = caps[0];
    const int i = blockIdx.x * kVertTile + threadIdx.x;
    if (i >= C.N || C.sc->vis_frozen) return;
    const float4 v = C.base[i];
    const bool ok = valid_depth(v.z);
    C.vw[i] = make_float4(v.x, v.y, v.z, ok ? 1.f : 0.f);
    C.uv[i] = ok ? project_exact(C.f, C.cx, C.cy, v.x, v.y, v.z) : make_float2(0.f, 0.f);
}

__global__ void __launch_bounds__(256) part_label_kernel(const CapDesc* __restrict__ caps) {
    const CapDesc& C = caps[0];
    if (C.sc->vis_frozen) return;
    const size_t P = (size_t)C.W * C.H;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long key = C.zbuf[p];
        uint8_t lab = 255;
        if (key != ~0ULL) {
            const int4 t = C.tris[(int)(unsigned)(key & 0xffffffffULL)];
            const uint8_t a = C.vpart[t.x], b = C.vpart[t.y], c = C.vpart[t.z];
            lab = (a == b || a == c) ? a : (b == c ? b : a);
        }
        C.part_raw[p] = lab;
    }
}

constexpr int kPartTile = 32;
constexpr unsigned short kPartFar = 0xffff;

// One CTA per 32 x 32 pixels with the labels of the tile and its halo of
// R = part_dilate pixels in shared memory.  The nearest-label search is
// separable: (d^2, label) minimised lexicographically over the labelled
// pixels within R equals, over the columns c within R, (x - c)^2 plus the
// column's own lexicographic minimum of ((y - r)^2, label) over its rows r
// within R (adding a constant keeps the order); likewise for the nearest
// torso pixel.  Pass 1: per (tile row, halo column) the nearest labelled and
// the nearest torso row; pass 2: per pixel the minimum over its 2R + 1
// columns.  Labelled pixels keep their label.
__global__ void __launch_bounds__(kPartTile * kPartTile) part_dilate_kernel(const CapDesc* __restrict__ caps) {
    extern __shared__ unsigned char s_raw[];
    const CapDesc& C = caps[0];
    if (C.sc->vis_frozen) return;
    const int R = C.part_dilate, S = kPartTile + 2 * R;
    uint8_t* s_lab = s_raw;                                                 // S x S
    unsigned short* s_d = (unsigned short*)(s_raw + ((S * S + 15) & ~15));  // kPartTile x S
    unsigned short* s_t = s_d + kPartTile * S;
    uint8_t* s_l = (uint8_t*)(s_t + kPartTile * S);
    const int bx = blockIdx.x * kPartTile - R, by = blockIdx.y * kPartTile - R;
    int any = 0;
    for (int q = threadIdx.x; q < S * S; q += blockDim.x) {
        const int x = bx + q % S, y = by + q / S;
        uint8_t l = 255;
        if (x >= 0 && x < C.W && y >= 0 && y < C.H) l = C.part_raw[(size_t)y * C.W + x];
        s_lab[q] = l;
        any |= l != 255;
    }
    any = __syncthreads_or(any);
    const int tx = threadIdx.x % kPartTile, ty = threadIdx.x / kPartTile;
    const int x = blockIdx.x * kPartTile + tx, y = blockIdx.y * kPartTile + ty;
    if (!any) {
        if (x < C.W && y < C.H) C.part_mask[(size_t)y * C.W + x] = 255;
        return;
    }
    // pass 1: column minima for the tile's rows
    for (int q = threadIdx.x; q < kPartTile * S; q += blockDim.x) {
        const int r = q / S, c = q % S;   // tile row, halo column
        unsigned short dn = kPartFar, dt = kPartFar;
        int ln = 255;
        for (int dy = 0; dy <= R && dt == kPartFar; ++dy) {
            const int a = s_lab[(r + R - dy) * S + c], b = s_lab[(r + R + dy) * S + c];
            if (dn == kPartFar && (a != 255 || b != 255)) {
                dn = (unsigned short)(dy * dy);
                ln = min(a, b);   // 255 when absent: the lower present label
            }
            if (a == C.torso_part || b == C.torso_part) dt = (unsigned short)(dy * dy);
        }
        s_d[q] = dn;
        s_t[q] = dt;
        s_l[q] = (uint8_t)ln;
    }
    __syncthreads();
    if (x >= C.W || y >= C.H) return;
    int lab = s_lab[(ty + R) * S + tx + R];
    if (lab == 255) {
        int best_d = 1 << 30, best_l = 255;
        bool torso = false;
        const int R2 = R * R;
        for (int dx = -R; dx <= R; ++dx) {
            const int q = ty * S + tx + R + dx;
            const int dx2 = dx * dx;
            if (s_t[q] != kPartFar && dx2 + s_t[q] <= R2) torso = true;
            if (s_d[q] == kPartFar) continue;
            const int d2 = dx2 + s_d[q];
            const int l = s_l[q];
            if (d2 <= R2 && (d2 < best_d || (d2 == best_d && l < best_l))) {
                best_d = d2;
                best_l = l;
            }
        }
        lab = torso ? C.torso_part : best_l;
    }
    C.part_mask[(size_t)y * C.W + x] = (uint8_t)lab;
}

static size_t part_dilate_smem(int R) {
    const int S = kPartTile + 2 * R;
    return (size_t)((S * S + 15) & ~15) + (size_t)kPartTile * S * (2 * sizeof(unsigned short) + 1);
}

void launch_part_mask(const CapDesc* dC, const CapDesc& hC, cudaStream_t st) {
    if (!hC.part_on) return;
    const Tiles T = single_tiles(hC);
    project_base_kernel<<<(hC.N + kVertTile - 1) / kVertTile, kVertTile, 0, st>>>(dC);
    const size_t P = (size_t)hC.W * hC.H;
    const int blocks = (int)std::min<size_t>((P + 255) / 256, 2048);
    vis_clear_kernel<<<blocks, 256, 0, st>>>(dC);
    if (T.tri) raster_kernel<<<T.tri, kRasterThreads, 0, st>>>(dC, T.tri_items);
    part_label_kernel<<<blocks, 256, 0, st>>>(dC);
    const dim3 grd((hC.W + kPartTile - 1) / kPartTile, (hC.H + kPartTile - 1) / kPartTile);
    part_dilate_kernel<<<grd, kPartTile * kPartTile, part_dilate_smem(hC.part_dilate), st>>>(dC);
}

__global__ void vertex_parts_kernel(const int4* __restrict__ skin_idx, const float4* __restrict__ skin_w,
                                    const int* __restrict__ bone_part, int N, uint8_t* __restrict__ vpart) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int4 b = skin_idx[i];
    const float4 w = skin_w[i];
    int best = b.x;
    float bw = w.x;
    if (w.y > bw) { best = b.y; bw = w.y; }
    if (w.z > bw) { best = b.z; bw = w.z; }
    if (w.w > bw) { best = b.w; bw = w.w; }
    vpart[i] = (uint8_t)bone_part[best];
}

void launch_vertex_parts(const int4* skin_idx, const float4* skin_w, const int* bone_part, int N, uint8_t* vpart,
                         cudaStream_t st) {
    vertex_parts_kernel<<<(N + 255) / 256, 256, 0, st>>>(skin_idx, skin_w, bone_part, N, vpart);
}

}  // namespace lc

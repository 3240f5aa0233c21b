// Visibility pass that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need this
// result: code running inside another framework's memory pool that forbids
// outside allocations, a process whose device memory is reserved up front
// by a real-time pipeline, or a plugin that may not grow the footprint of
// the host application.  They hand in device buffers they already own and
// get the per-vertex visibility back, with no allocation on any path.
//
// The only scratch, the 64-bit z-buffer, is a file-scope static device array
// of LC_NOALLOC_MAX_PIXELS entries (8 MiB); every GPU that loads this library
// keeps it until the process exits.  Every call shares it, it keeps the last
// call's contents, and each call first clears the part it uses.  Calls that
// overlap on the GPU (different streams, or different host threads on one
// device) race on it; the caller must serialise them.
//
// Arithmetic: identical to the context path (lc_compute_visibility): the
// same projection, 1/256 px snapping, int64 edge functions with the top-left
// rule, FP32 perspective-correct depth and depth test, so the flags are
// bit-identical for the same warped positions.
#include <cstdint>
#include <mutex>

#include "lc_internal.cuh"

namespace {

using lc::xadd;
using lc::xdiv;
using lc::xmul;

static __device__ __align__(256) unsigned long long g_noalloc_zbuf[LC_NOALLOC_MAX_PIXELS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned long long* g_zbuf_addr[kMaxDevices] = {nullptr};

__device__ __forceinline__ bool na_vertex(const float* __restrict__ V, int i, float f, float cx, float cy,
                                          float2& uv, float& Z, long long& sx, long long& sy) {
    const float X = V[3 * i], Y = V[3 * i + 1];
    Z = V[3 * i + 2];
    if (!(Z > 1e-3f)) return false;
    uv = lc::project_exact(f, cx, cy, X, Y, Z);
    if (!(fabsf(uv.x) < 1048576.0f) || !(fabsf(uv.y) < 1048576.0f)) return false;
    sx = __float2ll_rn(xmul(uv.x, 256.0f));
    sy = __float2ll_rn(xmul(uv.y, 256.0f));
    return true;
}

__device__ __forceinline__ bool na_owns(long long ex, long long ey) { return ey < 0 || (ey == 0 && ex > 0); }
__device__ __forceinline__ long long na_ceil256(long long a) { return a >= 0 ? (a + 255) / 256 : -((-a) / 256); }
__device__ __forceinline__ long long na_floor256(long long a) { return a >= 0 ? a / 256 : -((-a + 255) / 256); }

__global__ void na_clear(unsigned long long* __restrict__ zbuf, int P) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) zbuf[p] = ~0ULL;
}

__global__ void na_raster(const float* __restrict__ V, int N, const int32_t* __restrict__ tris, int F, float f,
                          float cx, float cy, int W, int H, unsigned long long* __restrict__ zbuf) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= F) return;
    const int ia = tris[3 * t], ib = tris[3 * t + 1], ic = tris[3 * t + 2];
    // triangles that name a vertex outside [0, N) are skipped
    if (ia < 0 || ia >= N || ib < 0 || ib >= N || ic < 0 || ic >= N) return;
    float2 uva, uvb, uvc;
    float za, zb, zc;
    long long ax, ay, bx, by, qx, qy;
    if (!na_vertex(V, ia, f, cx, cy, uva, za, ax, ay) || !na_vertex(V, ib, f, cx, cy, uvb, zb, bx, by) ||
        !na_vertex(V, ic, f, cx, cy, uvc, zc, qx, qy))
        return;
    const long long area = (bx - ax) * (qy - ay) - (by - ay) * (qx - ax);
    if (area == 0) return;
    const long long sg = area > 0 ? 1 : -1;
    long long px0 = max(na_ceil256(min(ax, min(bx, qx))), 0LL);
    long long py0 = max(na_ceil256(min(ay, min(by, qy))), 0LL);
    long long px1 = min(na_floor256(max(ax, max(bx, qx))), (long long)W - 1);
    long long py1 = min(na_floor256(max(ay, max(by, qy))), (long long)H - 1);
    const bool oA = na_owns(sg * (qx - bx), sg * (qy - by));
    const bool oB = na_owns(sg * (ax - qx), sg * (ay - qy));
    const bool oC = na_owns(sg * (bx - ax), sg * (by - ay));
    const float farea = (float)(sg * area);
    for (long long py = py0; py <= py1; ++py) {
        const long long Py = py * 256;
        for (long long px = px0; px <= px1; ++px) {
            const long long Px = px * 256;
            const long long wA = sg * ((qx - bx) * (Py - by) - (qy - by) * (Px - bx));
            const long long wB = sg * ((ax - qx) * (Py - qy) - (ay - qy) * (Px - qx));
            const long long wC = sg * ((bx - ax) * (Py - ay) - (by - ay) * (Px - ax));
            if (wA < 0 || wB < 0 || wC < 0) continue;
            if ((wA == 0 && !oA) || (wB == 0 && !oB) || (wC == 0 && !oC)) continue;
            const float b0 = xdiv(__ll2float_rn(wA), farea);
            const float b1 = xdiv(__ll2float_rn(wB), farea);
            const float b2 = xdiv(__ll2float_rn(wC), farea);
            const float depth = xdiv(1.0f, xadd(xadd(xdiv(b0, za), xdiv(b1, zb)), xdiv(b2, zc)));
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(depth) << 32) | (unsigned long long)(unsigned)t;
            atomicMin(&zbuf[py * W + px], key);
        }
    }
}

__global__ void na_visible(const float* __restrict__ V, int N, float f, float cx, float cy, int W, int H, float eps,
                           const unsigned long long* __restrict__ zbuf, uint8_t* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float2 uv;
    float Z;
    long long sx, sy;
    uint8_t vis = 0;
    if (na_vertex(V, i, f, cx, cy, uv, Z, sx, sy) && lc::in_image(uv, W, H)) {
        const long long px = __float2ll_rn(uv.x), py = __float2ll_rn(uv.y);
        const unsigned long long key = zbuf[py * W + px];
        vis = 1;
        if (key != ~0ULL) vis = Z <= xadd(__uint_as_float((unsigned)(key >> 32)), eps) ? 1 : 0;
    }
    out[i] = vis;
}

// Device (or managed) memory of device `dev`: memory of another GPU would be
// dereferenced by kernels running on this one.
bool is_device_memory(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" lc_status lc_visibility_noalloc(const float* V_warp, int N, const int32_t* tris, int F, float f, float cx,
                                           float cy, int W, int H, float eps_vis, uint8_t* visible,
                                           void* cuda_stream) {
    if (!V_warp || !tris || !visible || N < 1 || F < 0 || W < 1 || H < 1 || !(f > 0.f) || !(eps_vis >= 0.f))
        return LC_ERR_ARG;
    if ((long long)W * (long long)H > (long long)LC_NOALLOC_MAX_PIXELS) return LC_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LC_ERR_CUDA;
    if (!is_device_memory(V_warp, dev) || !is_device_memory(tris, dev) || !is_device_memory(visible, dev))
        return LC_ERR_ARG;
    unsigned long long* zbuf = nullptr;
    {
        // once per device, with that device current: the host-side name of a
        // __device__ array is not a device address, so look the address up
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_zbuf_addr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_zbuf) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return LC_ERR_CUDA;
            }
            g_zbuf_addr[dev] = (unsigned long long*)ptr;
        }
        zbuf = g_zbuf_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int P = W * H;
    na_clear<<<(P + 255) / 256 < 1184 ? (P + 255) / 256 : 1184, 256, 0, st>>>(zbuf, P);
    if (F > 0) na_raster<<<(F + 127) / 128, 128, 0, st>>>(V_warp, N, tris, F, f, cx, cy, W, H, zbuf);
    na_visible<<<(N + 255) / 256, 256, 0, st>>>(V_warp, N, f, cx, cy, W, H, eps_vis, zbuf, visible);
    return cudaGetLastError() == cudaSuccess ? LC_OK : LC_ERR_CUDA;
}

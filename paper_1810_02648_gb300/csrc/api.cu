// C ABI of the livecap library: context, uploads, graph build, the captured
// non-rigid solve and the inspection calls.  See include/livecap.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>
#include <functional>

#include "lc_context.h"

using namespace lc;

// ---------------------------------------------------------------------------
// error helpers
// ---------------------------------------------------------------------------
lc_status lc_ctx::fail(lc_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    err = buf;
    return st;
}

lc_status lc_ctx::cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return LC_OK;
    return fail(e == cudaErrorMemoryAllocation ? LC_ERR_OOM : LC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void* lc_ctx::alloc(size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        ++alloc_failures;
        cuda(e, "cudaMalloc");
        return nullptr;
    }
    owned.push_back(p);
    return p;
}

void lc_ctx::release(void* p) {
    if (!p) return;
    auto it = std::find(owned.begin(), owned.end(), p);
    if (it != owned.end()) {
        cudaFree(p);
        owned.erase(it);
    }
}

bool lc_ctx::is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

lc_status lc_ctx::copy_to_host(void* dst, const void* src_dev, size_t bytes) {
    lc_status s = cuda(cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDefault, stream), "copy out");
    if (s != LC_OK) return s;
    return cuda(cudaStreamSynchronize(stream), "synchronize");
}

// copy `bytes` from a host-or-device pointer into host memory
lc_status lc_ctx::fetch(void* dst_host, const void* src_any, size_t bytes) {
    if (bytes == 0) return LC_OK;
    return copy_to_host(dst_host, src_any, bytes);
}

// write a host staging buffer to a host-or-device destination
lc_status lc_ctx::deliver(void* dst_any, const void* src_host, size_t bytes) {
    if (bytes == 0) return LC_OK;
    lc_status s = cuda(cudaMemcpyAsync(dst_any, src_host, bytes, cudaMemcpyDefault, stream), "copy");
    if (s != LC_OK) return s;
    return cuda(cudaStreamSynchronize(stream), "synchronize");
}

lc_status lc_ctx::sync_desc() {
    lc_status s = cuda(cudaMemcpyAsync(dC, &hC, sizeof(CapDesc), cudaMemcpyHostToDevice, stream), "descriptor");
    if (s != LC_OK) return s;
    // the host copy must stay unchanged until the copy is done
    return cuda(cudaStreamSynchronize(stream), "synchronize");
}

void lc_ctx::drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    if (surf_gexec) cudaGraphExecDestroy(surf_gexec);
    surf_gexec = nullptr;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" lc_status lc_params_default(lc_params* p) {
    if (!p) return LC_ERR_ARG;
    memset(p, 0, sizeof(*p));
    p->w_photo = 1.0f;
    p->w_sil = 0.1f;
    p->w_arap = 10.0f;
    p->n_gn = 5;
    p->n_pcg = 20;
    p->eps_vis = 1e-2f;
    p->lambda_2d = 460.0f;
    p->lambda_3d = 28.0f;
    p->lambda_sil = 200.0f;
    p->n_gn_pose = 5;
    p->lambda_prior = 1e4f;
    p->pcg_kernel = 0;
    p->target_energy = 0.0f;
    p->w_smooth = 1.0e3f;
    p->w_edge = 3.0e3f;
    p->w_velocity = 25.0f;
    p->w_acceleration = 10.0f;
    p->n_gn_surface = 3;
    p->n_pcg_surface = 4;
    p->pose_solver = 0;
    p->lambda_temporal = 1.5f;
    p->lambda_anatomic = 1.0e6f;
    p->sigma_c = 0.0f;
    p->pyr_levels = 0;
    p->pyr_ksize[0] = 15;
    p->pyr_ksize[1] = 9;
    p->pyr_ksize[2] = 3;
    p->tma_taps = 1;   // measured faster than the global loads on the body capture, same bits
    return LC_OK;
}

extern "C" lc_status lc_create(lc_ctx** out, int device, void* cuda_stream) {
    if (!out) return LC_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return LC_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return LC_ERR_CUDA;
    lc_ctx* c = new lc_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    if (!c->stream) {
        // the solve is captured into a CUDA graph, which the legacy default
        // stream does not allow: use a stream of our own
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return LC_ERR_CUDA;
        }
        c->own_stream = true;
    }
    lc_params_default(&c->params);
    memset(&c->hC, 0, sizeof(CapDesc));
    c->dC = (CapDesc*)c->alloc(sizeof(CapDesc));
    c->hC.sc = (Scalars*)c->alloc(sizeof(Scalars));
    c->hC.counters = (unsigned*)c->alloc(sizeof(unsigned) * CNT_N);
    c->hC.hist = (double*)c->alloc(sizeof(double) * 2 * (LC_MAX_GN + 1));
    c->hC.hist_iters = (int*)c->alloc(sizeof(int) * (LC_MAX_GN + 2));
    if (!c->dC || !c->hC.sc || !c->hC.counters || !c->hC.hist || !c->hC.hist_iters) {
        lc_destroy(c);
        return LC_ERR_OOM;
    }
    cudaMemsetAsync(c->hC.sc, 0, sizeof(Scalars), c->stream);
    cudaMemsetAsync(c->hC.counters, 0, sizeof(unsigned) * CNT_N, c->stream);
    c->apply_params();
    if (c->sync_desc() != LC_OK) {
        lc_destroy(c);
        return LC_ERR_CUDA;
    }
    *out = c;
    return LC_OK;
}

extern "C" lc_status lc_destroy(lc_ctx* ctx) {
    if (!ctx) return LC_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->drop_graph();
    ctx->pose_release();
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    ctx->prof_ev.clear();
    for (void* p : ctx->owned) cudaFree(p);
    ctx->owned.clear();
    if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return LC_OK;
}

extern "C" const char* lc_last_error(const lc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void lc_ctx::apply_params() {
    hC.w_photo = params.w_photo;
    hC.w_sil = params.w_sil;
    hC.w_arap = params.w_arap;
    hC.eps_vis = params.eps_vis;
    hC.target_energy = params.target_energy;
    hC.sigma_c = params.sigma_c;
    hC.tma_taps = params.tma_taps;
    surface_weights();
}

extern "C" lc_status lc_set_params(lc_ctx* ctx, const lc_params* p) {
    if (!ctx || !p) return LC_ERR_ARG;
    if (p->n_gn < 1 || p->n_gn > LC_MAX_GN || p->n_pcg < 1 || p->n_gn_pose < 1 || p->n_gn_pose > LC_MAX_GN ||
        !(p->w_photo >= 0.f) || !(p->w_sil >= 0.f) || !(p->w_arap >= 0.f) || !(p->eps_vis >= 0.f) ||
        !(p->lambda_2d >= 0.f) || !(p->lambda_3d >= 0.f) || !(p->lambda_sil >= 0.f) || !(p->lambda_prior >= 0.f) ||
        !(p->target_energy >= 0.f) || p->n_gn_surface < 1 || p->n_gn_surface > LC_MAX_GN || p->n_pcg_surface < 1 ||
        !(p->w_smooth >= 0.f) || !(p->w_edge >= 0.f) || !(p->w_velocity >= 0.f) || !(p->w_acceleration >= 0.f) ||
        p->pose_solver < 0 || p->pose_solver > 1 || !(p->lambda_temporal >= 0.f) || !(p->lambda_anatomic >= 0.f) ||
        !(p->sigma_c >= 0.f) || p->pyr_levels < 0 || p->pyr_levels > 3 || p->pose_displacement < 0 ||
        p->pose_displacement > 1 || p->gn_block < 0 || p->graph_warp < 0 || p->graph_warp > 1 ||
        p->tma_taps < 0 || p->tma_taps > 1)
        return ctx->fail(LC_ERR_ARG, "lc_set_params: out of range");
    for (int j = 0; j < 3; ++j)
        if (p->pyr_ksize[j] < 1 || p->pyr_ksize[j] > kPyrMaxTaps || p->pyr_ksize[j] % 2 == 0)
            return ctx->fail(LC_ERR_ARG, "lc_set_params: pyr_ksize must be odd, 1..%d", kPyrMaxTaps);
    cudaSetDevice(ctx->device);
    if (p->pcg_kernel < 0 || p->pcg_kernel > 1) return ctx->fail(LC_ERR_ARG, "lc_set_params: pcg_kernel must be 0 or 1");
    // a target energy switches the captured solve to conditional blocks of steps
    if ((p->target_energy > 0.f) != (ctx->params.target_energy > 0.f) || p->gn_block != ctx->params.gn_block)
        ctx->drop_graph();
    if (p->tma_taps != ctx->params.tma_taps) {   // the captured linearisations change kernel
        ctx->drop_graph();
        ctx->pose_drop_graph();
    }
    if (p->n_gn != ctx->params.n_gn || p->n_pcg != ctx->params.n_pcg || p->pcg_kernel != ctx->params.pcg_kernel ||
        p->n_gn_surface != ctx->params.n_gn_surface || p->n_pcg_surface != ctx->params.n_pcg_surface)
        ctx->drop_graph();
    if (p->n_gn_pose != ctx->params.n_gn_pose || p->graph_warp != ctx->params.graph_warp) ctx->pose_drop_graph();
    const bool pyr_changed = p->pyr_levels != ctx->params.pyr_levels ||
                             memcmp(p->pyr_ksize, ctx->params.pyr_ksize, sizeof(p->pyr_ksize)) != 0;
    ctx->params = *p;
    ctx->apply_params();
    if (pyr_changed && ctx->has_frame) {
        lc_status s = ctx->build_pyramid();
        if (s) return s;
    }
    return ctx->sync_desc();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return (EncodeTiledFn)p;
    }();
    return fn;
}

// the frame as a 2D tensor of 4W x H floats, boxes of 16 x 4 (a 4 x 4 pixel
// patch) for the TMA-staged taps; tma_ok = 0 where it cannot be made
static void encode_image_map(lc_ctx* ctx) {
    CapDesc& C = ctx->hC;
    C.tma_ok = 0;
    const EncodeTiledFn fn = encode_tiled();
    if (!fn || !C.img || C.W < 4 || C.H < 4) return;
    if (linearize_tma_init() != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const cuuint64_t dims[2] = {4ull * (cuuint64_t)C.W, (cuuint64_t)C.H};
    const cuuint64_t strides[1] = {16ull * (cuuint64_t)C.W};
    const cuuint32_t box[2] = {16, 4}, elem[2] = {1, 1};
    if (fn(&C.tmap_img, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)C.img, dims, strides, box, elem,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
        C.tma_ok = 1;
}

extern "C" lc_status lc_set_camera(lc_ctx* ctx, float f, float cx, float cy, int W, int H) {
    if (!ctx) return LC_ERR_ARG;
    if (!(f > 0.f) || W < 1 || H < 1 || W > 16384 || H > 16384)
        return ctx->fail(LC_ERR_ARG, "lc_set_camera: bad camera");
    cudaSetDevice(ctx->device);
    if (W != ctx->hC.W || H != ctx->hC.H) {
        ctx->release((void*)ctx->hC.img);
        ctx->release((void*)ctx->hC.mask);
        ctx->release(ctx->hC.zbuf);
        ctx->release(ctx->stage_rgb);
        ctx->release(ctx->stage_dt);
        ctx->release(ctx->stage_mask);
        ctx->release(ctx->edt_g);
        ctx->edt_g = nullptr;
        ctx->pyr_release();
        const size_t P = (size_t)W * H;
        ctx->hC.img = (const float4*)ctx->alloc(sizeof(float4) * P);
        ctx->hC.mask = (const uint8_t*)ctx->alloc(P);
        ctx->hC.zbuf = (unsigned long long*)ctx->alloc(sizeof(unsigned long long) * P);
        ctx->stage_rgb = (float*)ctx->alloc(sizeof(float) * 3 * P);
        ctx->stage_dt = (float*)ctx->alloc(sizeof(float) * P);
        ctx->stage_mask = (uint8_t*)ctx->alloc(P);
        if (!ctx->hC.img || !ctx->hC.mask || !ctx->hC.zbuf || !ctx->stage_rgb || !ctx->stage_dt || !ctx->stage_mask)
            return LC_ERR_OOM;
        ctx->has_frame = false;
        ctx->has_vis = false;
        ctx->drop_graph();
        ctx->hC.W = W;
        ctx->hC.H = H;
        if (ctx->hC.part_on) {
            lc_status s = ctx->part_images();
            if (s) return s;
        }
    }
    ctx->hC.f = f;
    ctx->hC.cx = cx;
    ctx->hC.cy = cy;
    ctx->hC.W = W;
    ctx->hC.H = H;
    encode_image_map(ctx);
    ctx->has_camera = true;
    return ctx->sync_desc();
}

// ---------------------------------------------------------------------------
// template
// ---------------------------------------------------------------------------
template <typename T>
static lc_status host_copy(lc_ctx* ctx, std::vector<T>& dst, const T* src, size_t count) {
    dst.resize(count);
    return ctx->fetch(dst.data(), src, sizeof(T) * count);
}

extern "C" lc_status lc_upload_template(lc_ctx* ctx, const float* V, int N, const int32_t* tris, int F,
                                        const float* albedo, const float* material) {
    if (!ctx) return LC_ERR_ARG;
    if (!V || !tris || !albedo || !material || N < 1 || F < 1)
        return ctx->fail(LC_ERR_ARG, "lc_upload_template: null array or empty mesh");
    cudaSetDevice(ctx->device);
    const int af0 = ctx->alloc_failures;
    std::vector<float> hv, ha, hm;
    std::vector<int32_t> ht;
    lc_status s;
    if ((s = host_copy(ctx, hv, V, (size_t)3 * N)) != LC_OK) return s;
    if ((s = host_copy(ctx, ht, tris, (size_t)3 * F)) != LC_OK) return s;
    if ((s = host_copy(ctx, ha, albedo, (size_t)3 * N)) != LC_OK) return s;
    if ((s = host_copy(ctx, hm, material, (size_t)N)) != LC_OK) return s;
    for (int i = 0; i < 3 * F; ++i)
        if (ht[i] < 0 || ht[i] >= N) return ctx->fail(LC_ERR_ARG, "lc_upload_template: triangle index out of range");
    for (int i = 0; i < 3 * N; ++i)
        if (!std::isfinite(hv[i])) return ctx->fail(LC_ERR_ARG, "lc_upload_template: non-finite vertex");
    // mesh topology: vertex -> triangle CSR (ascending ids) and edges with two triangles
    std::vector<int> vt_off(N + 1, 0), vt_tri((size_t)3 * F);
    for (int i = 0; i < 3 * F; ++i) vt_off[ht[i] + 1]++;
    for (int i = 0; i < N; ++i) vt_off[i + 1] += vt_off[i];
    {
        std::vector<int> fill(vt_off.begin(), vt_off.end() - 1);
        for (int t = 0; t < F; ++t)
            for (int c = 0; c < 3; ++c) vt_tri[fill[ht[3 * t + c]]++] = t;   // t ascending per vertex
    }
    struct HalfEdge {
        int lo, hi, t;
    };
    std::vector<HalfEdge> he((size_t)3 * F);
    for (int t = 0; t < F; ++t)
        for (int c = 0; c < 3; ++c) {
            int a = ht[3 * t + c], b = ht[3 * t + (c + 1) % 3];
            he[3 * t + c] = {std::min(a, b), std::max(a, b), t};
        }
    std::sort(he.begin(), he.end(), [](const HalfEdge& x, const HalfEdge& y) {
        return x.lo != y.lo ? x.lo < y.lo : (x.hi != y.hi ? x.hi < y.hi : x.t < y.t);
    });
    std::vector<int4> medges;
    for (size_t i = 0; i < he.size();) {
        size_t j = i;
        while (j < he.size() && he[j].lo == he[i].lo && he[j].hi == he[i].hi) ++j;
        if (j - i > 2) return ctx->fail(LC_ERR_ARG, "lc_upload_template: non-manifold edge (%d,%d)", he[i].lo, he[i].hi);
        medges.push_back(make_int4(he[i].lo, he[i].hi, he[i].t, j - i == 2 ? he[i + 1].t : -1));
        i = j;
    }
    // release the old template and everything built on it
    ctx->free_template();
    std::vector<float4> v4(N), a4(N);
    std::vector<int4> t4(F);
    for (int i = 0; i < N; ++i) {
        v4[i] = make_float4(hv[3 * i], hv[3 * i + 1], hv[3 * i + 2], 0.f);
        a4[i] = make_float4(ha[3 * i], ha[3 * i + 1], ha[3 * i + 2], 0.f);
    }
    for (int t = 0; t < F; ++t) t4[t] = make_int4(ht[3 * t], ht[3 * t + 1], ht[3 * t + 2], 0);
    CapDesc& C = ctx->hC;
    ctx->tpl = (float4*)ctx->alloc(sizeof(float4) * N);
    ctx->base_buf = (float4*)ctx->alloc(sizeof(float4) * N);
    C.albedo = (const float4*)ctx->alloc(sizeof(float4) * N);
    C.tris = (const int4*)ctx->alloc(sizeof(int4) * F);
    C.vt_off = (const int*)ctx->alloc(sizeof(int) * (N + 1));
    C.vt_tri = (const int*)ctx->alloc(sizeof(int) * 3 * F);
    C.medges = (const int4*)ctx->alloc(sizeof(int4) * medges.size());
    ctx->material = (float*)ctx->alloc(sizeof(float) * N);
    C.flags = (uint32_t*)ctx->alloc(sizeof(uint32_t) * N);
    C.vw = (float4*)ctx->alloc(sizeof(float4) * N);
    C.uv = (float2*)ctx->alloc(sizeof(float2) * N);
    C.res = (float4*)ctx->alloc(sizeof(float4) * N);
    C.HA = (float4*)ctx->alloc(sizeof(float4) * N);
    C.HB = (float4*)ctx->alloc(sizeof(float4) * N);
    C.ev = (float4*)ctx->alloc(sizeof(float4) * N);
    C.q = (float4*)ctx->alloc(sizeof(float4) * 2 * N);
    C.vH = (float4*)ctx->alloc(sizeof(float4) * 2 * N);
    C.vpos = (int*)ctx->alloc(sizeof(int) * N);
    C.vcnt = (int*)ctx->alloc(sizeof(int) * ((N + kJChunk - 1) / kJChunk));
    if (ctx->alloc_failures != af0) return LC_ERR_OOM;
    C.base = ctx->base_buf;
    cudaStream_t st = ctx->stream;
    if ((s = ctx->cuda(cudaMemcpyAsync(ctx->tpl, v4.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, st), "upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync(ctx->base_buf, v4.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, st), "upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync((void*)C.albedo, a4.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, st), "upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync((void*)C.tris, t4.data(), sizeof(int4) * F, cudaMemcpyHostToDevice, st), "upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync((void*)C.vt_off, vt_off.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, st), "upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync((void*)C.vt_tri, vt_tri.data(), sizeof(int) * 3 * F, cudaMemcpyHostToDevice, st), "upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync((void*)C.medges, medges.data(), sizeof(int4) * medges.size(), cudaMemcpyHostToDevice, st), "upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync(ctx->material, hm.data(), sizeof(float) * N, cudaMemcpyHostToDevice, st), "upload")))
        return s;
    C.N = N;
    C.F = F;
    C.n_medges = (int)medges.size();
    C.vert_tiles = (N + kVertTile - 1) / kVertTile;
    C.tri_tiles = (F + kTriTile - 1) / kTriTile;
    C.medge_tiles = (C.n_medges + kEdgeTile - 1) / kEdgeTile;
    if ((s = ctx->surface_setup(hv.data(), hm.data(), medges))) return s;
    ctx->ensure_partials();
    ctx->has_template = true;
    ctx->drop_graph();
    return ctx->sync_desc();
}

void lc_ctx::ensure_partials() {
    const int need = std::max({4 * hC.vert_tiles, hC.node_tiles, (hC.n + kVecThreads - 1) / kVecThreads, 64}) + 8;
    if (need > part_cap) {
        release(hC.part);
        hC.part = (double*)alloc(sizeof(double) * need);
        part_cap = need;
    }
}

void lc_ctx::free_graph() {
    warm_release();
    void* bufs[] = {(void*)hC.node_vid, (void*)hC.bind_idx, (void*)hC.bind_w, (void*)hC.node_g, (void*)hC.ent_off,
                    (void*)hC.ent, (void*)hC.edge_off, (void*)hC.edge_dst, (void*)hC.edge_s, hC.node_R, hC.node_t,
                    hC.vA, hC.vK, hC.eV, hC.ecnt, hC.dB,
                    hC.b, hC.minv, hC.diag, hC.x, hC.r, hC.z, hC.p, hC.Ap, tmp_vec, tmp_vec2,
                    hC.x_lo, hC.r_lo, hC.z_lo, hC.p_lo, hC.Ap_lo};
    release_pcg_tables();
    for (void* p : bufs) release(p);
    hC.node_vid = nullptr; hC.bind_idx = nullptr; hC.bind_w = nullptr; hC.node_g = nullptr;
    hC.ent_off = nullptr; hC.ent = nullptr; hC.edge_off = nullptr; hC.edge_dst = nullptr; hC.edge_s = nullptr;
    hC.node_R = nullptr; hC.node_t = nullptr;
    hC.vA = hC.dB = nullptr;
    hC.vK = hC.eV = hC.ecnt = nullptr;
    hC.b = hC.minv = hC.diag = hC.x = hC.r = hC.z = hC.p = hC.Ap = nullptr;
    hC.x_lo = hC.r_lo = hC.z_lo = hC.p_lo = hC.Ap_lo = nullptr;
    pcg_part = lc::PcgPartition();
    tmp_vec = tmp_vec2 = nullptr;
    pcg_plan_ok = false;
    hC.n = 0;
    hC.K = 0;
    hC.E = 0;
    hC.node_tiles = 0;
    has_graph = false;
    has_lin = false;
    has_vis = false;
}

void lc_ctx::free_template() {
    free_graph();
    pose_release();
    surface_release();
    void* bufs[] = {tpl, base_buf, (void*)hC.albedo, (void*)hC.tris, (void*)hC.vt_off, (void*)hC.vt_tri,
                    (void*)hC.medges, material, hC.flags, hC.vw, hC.uv, hC.res, hC.HA, hC.HB, hC.ev, hC.q,
                    hC.vH, hC.vpos, hC.vcnt};
    for (void* p : bufs) release(p);
    tpl = base_buf = nullptr;
    material = nullptr;
    hC.base = nullptr; hC.albedo = nullptr; hC.tris = nullptr; hC.vt_off = nullptr; hC.vt_tri = nullptr;
    hC.medges = nullptr; hC.flags = nullptr; hC.vw = nullptr; hC.uv = nullptr; hC.res = nullptr;
    hC.HA = hC.HB = hC.ev = hC.q = hC.vH = nullptr;
    hC.vpos = hC.vcnt = nullptr;
    hC.N = hC.F = hC.n_medges = 0;
    has_template = false;
}

// ---------------------------------------------------------------------------
// graph
// ---------------------------------------------------------------------------
void lc_ctx::release_pcg_tables() {
    void* bufs[] = {(void*)hC.pcg_perm, (void*)hC.pcg_leaf_off, (void*)hC.pcg_leaf, (void*)hC.jn_perm,
                    (void*)hC.pcg_loc_off[0], (void*)hC.pcg_loc_vid[0], (void*)hC.pcg_eus_off[0], (void*)hC.pcg_ent_us[0],
                    (void*)hC.pcg_loc_off[1], (void*)hC.pcg_loc_vid[1], (void*)hC.pcg_eus_off[1], (void*)hC.pcg_ent_us[1],
                    (void*)hC.pcg_zdst[0], (void*)hC.pcg_zdst[1]};
    for (void* p : bufs) release(p);
    hC.pcg_perm = nullptr;
    hC.jn_perm = nullptr;
    hC.pcg_leaf_off = nullptr;
    hC.pcg_leaf = nullptr;
    for (int ti = 0; ti < 2; ++ti) {
        hC.pcg_loc_off[ti] = nullptr;
        hC.pcg_loc_vid[ti] = nullptr;
        hC.pcg_eus_off[ti] = nullptr;
        hC.pcg_ent_us[ti] = nullptr;
        hC.pcg_zdst[ti] = nullptr;
    }
}

// Morton order of the node positions: each coordinate quantised to 10 bits
// over the nodes' bounding box, the bits interleaved (x lowest), nodes
// sorted by code and then by id.
static void morton_order(int n, const float4* g, std::vector<int>& order) {
    float lo[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < n; ++k) {
        const float v[3] = {g[k].x, g[k].y, g[k].z};
        for (int d = 0; d < 3; ++d) {
            lo[d] = k ? std::min(lo[d], v[d]) : v[d];
            hi[d] = k ? std::max(hi[d], v[d]) : v[d];
        }
    }
    auto spread = [](uint32_t x) {   // 10 bits -> every third bit of 30
        uint32_t r = 0;
        for (int b = 0; b < 10; ++b) r |= ((x >> b) & 1u) << (3 * b);
        return r;
    };
    std::vector<std::pair<uint32_t, int>> key(n);
    for (int k = 0; k < n; ++k) {
        const float v[3] = {g[k].x, g[k].y, g[k].z};
        uint32_t code = 0;
        for (int d = 0; d < 3; ++d) {
            const float ext = hi[d] - lo[d];
            const float u = ext > 0.f ? (v[d] - lo[d]) / ext : 0.f;
            const uint32_t q = (uint32_t)std::min(1023.f, std::max(0.f, u * 1023.f));
            code |= spread(q) << d;
        }
        key[k] = {code, k};
    }
    std::sort(key.begin(), key.end());
    order.resize(n);
    for (int k = 0; k < n; ++k) order[k] = key[k].second;
}

// Spatial partition of the graph's nodes (host, from the node positions,
// bindings and CSR), its per-CTA tables uploaded to the device, and the
// cluster PCG plan.
lc_status lc_ctx::plan_pcg() {
    CapDesc& C = hC;
    const int n = C.n, N = C.N, K = C.K;
    std::vector<int> eo(n + 1), go(n + 1), bi((size_t)N * K);
    std::vector<float4> g(n);
    lc_status s;
    if ((s = copy_to_host(eo.data(), C.ent_off, sizeof(int) * (n + 1))) ||
        (s = copy_to_host(go.data(), C.edge_off, sizeof(int) * (n + 1))) ||
        (s = copy_to_host(bi.data(), C.bind_idx, sizeof(int) * (size_t)N * K)) ||
        (s = copy_to_host(g.data(), C.node_g, sizeof(float4) * n)))
        return s;
    std::vector<int2> en((size_t)std::max(eo[n], 1));
    std::vector<int> ed((size_t)std::max(go[n], 1));
    if ((s = copy_to_host(en.data(), C.ent, sizeof(int2) * (size_t)eo[n])) ||
        (s = copy_to_host(ed.data(), C.edge_dst, sizeof(int) * (size_t)go[n])))
        return s;
    spatial_partition(n, N, K, g.data(), eo.data(), en.data(), go.data(), ed.data(), bi.data(), pcg_part);
    morton_order(n, g.data(), pcg_part.zorder);
    release_pcg_tables();
    // upload one host array into a fresh device buffer
    auto put = [&](const void* src, size_t bytes) -> void* {
        void* d = alloc(std::max<size_t>(bytes, 16));
        if (d && bytes) cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, stream);
        return d;
    };
    C.pcg_perm = (const int*)put(pcg_part.perm.data(), sizeof(int) * n);
    C.pcg_leaf_off = (const int*)put(pcg_part.leaf_off.data(), sizeof(int) * (kPcgLeaves + 1));
    C.pcg_leaf = (const uint8_t*)put(pcg_part.leaf.data(), n);
    C.jn_perm = (const int*)put(pcg_part.zorder.data(), sizeof(int) * n);
    bool ok = C.pcg_perm && C.pcg_leaf_off && C.pcg_leaf && C.jn_perm;
    for (int ti = 0; ti < 2; ++ti) {
        C.pcg_loc_off[ti] = (const int*)put(pcg_part.loc_off[ti].data(), sizeof(int) * pcg_part.loc_off[ti].size());
        C.pcg_loc_vid[ti] = (const int*)put(pcg_part.loc_vid[ti].data(), sizeof(int) * pcg_part.loc_vid[ti].size());
        C.pcg_eus_off[ti] = (const int*)put(pcg_part.eus_off[ti].data(), sizeof(int) * pcg_part.eus_off[ti].size());
        C.pcg_ent_us[ti] = (const unsigned*)put(pcg_part.ent_us[ti].data(), sizeof(unsigned) * pcg_part.ent_us[ti].size());
        C.pcg_zdst[ti] = (const unsigned short*)put(pcg_part.zdst[ti].data(), sizeof(unsigned short) * pcg_part.zdst[ti].size());
        ok = ok && C.pcg_loc_off[ti] && C.pcg_loc_vid[ti] && C.pcg_eus_off[ti] && C.pcg_ent_us[ti] && C.pcg_zdst[ti];
    }
    if (!ok) return fail(LC_ERR_OOM, "plan_pcg: device allocation failed");
    if ((s = cuda(cudaStreamSynchronize(stream), "upload"))) return s;
    pcg_plan_ok = plan_pcg_cluster(pcg_part, n, K, &pcg_plan);
    cudaGetLastError();
    return LC_OK;
}

// device arrays of a graph of n nodes and K bindings per vertex, edges apart
static void graph_alloc(lc_ctx* ctx, int n, int K) {
    CapDesc& C = ctx->hC;
    const int N = C.N;
    ctx->free_graph();
    C.n = n;
    C.K = K;
    C.node_tiles = (n + kNodeTile - 1) / kNodeTile;
    C.node_vid = (const int*)ctx->alloc(sizeof(int) * n);
    C.bind_idx = (const int*)ctx->alloc(sizeof(int) * (size_t)N * K);
    C.bind_w = (const float*)ctx->alloc(sizeof(float) * (size_t)N * K);
    C.node_g = (const float4*)ctx->alloc(sizeof(float4) * n);
    C.ent_off = (const int*)ctx->alloc(sizeof(int) * (n + 1));
    C.ent = (const int2*)ctx->alloc(sizeof(int2) * (size_t)N * K);
    C.ecnt = (int*)ctx->alloc(sizeof(int) * n);
    C.edge_off = (const int*)ctx->alloc(sizeof(int) * (n + 1));
    C.node_R = (float4*)ctx->alloc(sizeof(float4) * 3 * n);
    C.node_t = (float4*)ctx->alloc(sizeof(float4) * n);
    float4** vecs[] = {&C.b, &C.minv, &C.diag, &C.x, &C.r, &C.z, &C.p, &C.Ap, &ctx->tmp_vec, &ctx->tmp_vec2,
                       &C.x_lo, &C.r_lo, &C.z_lo, &C.p_lo, &C.Ap_lo};
    for (float4** v : vecs) *v = (float4*)ctx->alloc(sizeof(float4) * 2 * n);
}

// the E edge arrays and the per-binding / per-edge staging of the solver
static void graph_alloc_edges(lc_ctx* ctx, int E) {
    CapDesc& C = ctx->hC;
    const size_t NK = (size_t)C.N * C.K;
    C.E = E;
    C.edge_dst = (const int*)ctx->alloc(sizeof(int) * std::max(E, 1));
    C.edge_s = (const float*)ctx->alloc(sizeof(float) * std::max(E, 1));
    C.vA = (float4*)ctx->alloc(sizeof(float4) * NK);
    C.vK = (int*)ctx->alloc(sizeof(int) * NK);
    C.eV = (int*)ctx->alloc(sizeof(int) * NK);
    C.dB = (float4*)ctx->alloc(sizeof(float4) * 2 * (size_t)std::max(E, 1));
}

// after the bindings and edges are in place: the node -> vertex entries,
// node positions of the current rest geometry, identity parameters, the PCG
// plan; the captured solves are dropped
static lc_status graph_finish(lc_ctx* ctx, GraphScratch& gs, const std::function<void()>& cleanup) {
    CapDesc& C = ctx->hC;
    cudaStream_t st = ctx->stream;
    launch_entries(C.bind_idx, C.bind_w, C.N, C.K, C.n, gs, (int*)C.ent_off, (int2*)C.ent, st);
    launch_gather_nodes(C.base, C.node_vid, C.n, (float4*)C.node_g, st);
    launch_identity_params(C.node_R, C.node_t, C.n, st);
    lc_status s = ctx->cuda(cudaStreamSynchronize(st), "graph build");
    cleanup();
    if (s != LC_OK) return s;
    if ((s = ctx->plan_pcg())) return s;
    ctx->ensure_partials();
    ctx->has_graph = true;
    ctx->drop_graph();
    ctx->pose_drop_graph();   // the pose solve moves the graph nodes
    ctx->pose_graph_changed();
    return ctx->sync_desc();
}

extern "C" lc_status lc_build_graph(lc_ctx* ctx, int n_nodes, int K) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_template) return ctx->fail(LC_ERR_STATE, "lc_build_graph: no template");
    CapDesc& C = ctx->hC;
    if (K < 1 || K > kMaxK || n_nodes < K + 1 || n_nodes > C.N)
        return ctx->fail(LC_ERR_ARG, "lc_build_graph: need 1 <= K <= %d and K+1 <= n_nodes <= N", kMaxK);
    cudaSetDevice(ctx->device);
    const int af0 = ctx->alloc_failures;
    const int n = n_nodes, N = C.N;
    cudaStream_t st = ctx->stream;
    graph_alloc(ctx, n, K);
    GraphScratch gs;
    std::vector<void*> scratch;
    auto salloc = [&](size_t b) {
        void* p = ctx->alloc(b);
        scratch.push_back(p);
        return p;
    };
    gs.dist = (double*)salloc(sizeof(double) * N);
    gs.knn_e = (int*)salloc(sizeof(int) * n * kEdgeNN);
    gs.extra_cnt = (int*)salloc(sizeof(int) * n);
    gs.extra = (int*)salloc(sizeof(int) * (size_t)n * kMaxExtraEdges);
    gs.deg = (int*)salloc(sizeof(int) * (n + 1));
    gs.ent_cnt = (int*)salloc(sizeof(int) * (n + 1));
    gs.ent_fill = (int*)salloc(sizeof(int) * n);
    gs.status = (int*)salloc(sizeof(int));
    auto cleanup = [&]() {
        for (void* p : scratch) ctx->release(p);
    };
    if (ctx->alloc_failures != af0) {
        cleanup();
        return LC_ERR_OOM;
    }
    constexpr int kFpsMaxCtas = 4096;
    double* fps_val = (double*)salloc(sizeof(double) * 2 * kFpsMaxCtas);
    int* fps_idx = (int*)salloc(sizeof(int) * 2 * kFpsMaxCtas);
    if (ctx->alloc_failures != af0) {
        cleanup();
        return LC_ERR_OOM;
    }
    cudaMemsetAsync(gs.status, 0, sizeof(int), st);
    // nodes and bindings on the rest template
    if (!launch_fps(ctx->tpl, N, n, gs.dist, (int*)C.node_vid, fps_val, fps_idx, kFpsMaxCtas, st)) {
        cudaGetLastError();
        cleanup();
        return ctx->fail(LC_ERR_CUDA, "lc_build_graph: cooperative launch of the node sampling failed");
    }
    float4* G_tpl = (float4*)salloc(sizeof(float4) * n);
    launch_gather_nodes(ctx->tpl, C.node_vid, n, G_tpl, st);
    launch_bind(ctx->tpl, N, G_tpl, n, K, (int*)C.bind_idx, (float*)C.bind_w, st);
    launch_node_edges_count(G_tpl, n, gs, st);
    launch_exclusive_scan(gs.deg, (int*)C.edge_off, n + 1, st);
    int E = 0, gstat = 0;
    lc_status s;
    if ((s = ctx->copy_to_host(&E, C.edge_off + n, sizeof(int))) != LC_OK ||
        (s = ctx->copy_to_host(&gstat, gs.status, sizeof(int))) != LC_OK) {
        cleanup();
        return s;
    }
    if (gstat) {
        cleanup();
        return ctx->fail(LC_ERR_NUMERIC, "lc_build_graph: a node has more than %d incoming edges", kMaxExtraEdges);
    }
    graph_alloc_edges(ctx, E);
    if (ctx->alloc_failures != af0) {
        cleanup();
        return LC_ERR_OOM;
    }
    launch_node_edges_fill(G_tpl, n, ctx->material, C.node_vid, gs, C.edge_off, (int*)C.edge_dst, (float*)C.edge_s, st);
    return graph_finish(ctx, gs, cleanup);
}

extern "C" lc_status lc_upload_graph(lc_ctx* ctx, int n_nodes, int K, const int32_t* node_vid, const int32_t* bind_idx,
                                     const float* bind_w, const int32_t* edge_off, const int32_t* edge_dst,
                                     const float* edge_s) {
    if (!ctx || !node_vid || !bind_idx || !bind_w || !edge_off) return LC_ERR_ARG;
    if (!ctx->has_template) return ctx->fail(LC_ERR_STATE, "lc_upload_graph: no template");
    CapDesc& C = ctx->hC;
    if (K < 1 || K > kMaxK || n_nodes < 1 || n_nodes > C.N)
        return ctx->fail(LC_ERR_ARG, "lc_upload_graph: need 1 <= K <= %d and 1 <= n_nodes <= N", kMaxK);
    cudaSetDevice(ctx->device);
    const int af0 = ctx->alloc_failures;
    const int n = n_nodes, N = C.N;
    const size_t NK = (size_t)N * K;
    // host copies (the arguments may be host or device memory) for the checks
    std::vector<int32_t> vid(n), bi(NK), eo(n + 1);
    std::vector<float> bw(NK);
    auto get = [&](void* dst, const void* src, size_t bytes) {
        return ctx->cuda(cudaMemcpy(dst, src, bytes, cudaMemcpyDefault), "lc_upload_graph: read arguments");
    };
    lc_status s;
    if ((s = get(vid.data(), node_vid, sizeof(int32_t) * n)) || (s = get(bi.data(), bind_idx, sizeof(int32_t) * NK)) ||
        (s = get(bw.data(), bind_w, sizeof(float) * NK)) || (s = get(eo.data(), edge_off, sizeof(int32_t) * (n + 1))))
        return s;
    for (int k = 0; k < n; ++k)
        if (vid[k] < 0 || vid[k] >= N) return ctx->fail(LC_ERR_ARG, "lc_upload_graph: node_vid[%d] out of range", k);
    for (size_t j = 0; j < NK; ++j) {
        if (bi[j] < 0 || bi[j] >= n) return ctx->fail(LC_ERR_ARG, "lc_upload_graph: bind_idx[%zu] out of range", j);
        if (!(bw[j] >= 0.f) || !std::isfinite(bw[j]))
            return ctx->fail(LC_ERR_ARG, "lc_upload_graph: bind_w[%zu] must be finite and >= 0", j);
    }
    if (eo[0] != 0) return ctx->fail(LC_ERR_ARG, "lc_upload_graph: edge_off[0] must be 0");
    for (int k = 0; k < n; ++k)
        if (eo[k + 1] < eo[k]) return ctx->fail(LC_ERR_ARG, "lc_upload_graph: edge_off must not decrease");
    const int E = eo[n];
    std::vector<int32_t> ed(std::max(E, 1));
    std::vector<float> es(std::max(E, 1));
    if (E > 0) {
        if (!edge_dst || !edge_s) return ctx->fail(LC_ERR_ARG, "lc_upload_graph: edges without edge_dst / edge_s");
        if ((s = get(ed.data(), edge_dst, sizeof(int32_t) * E)) || (s = get(es.data(), edge_s, sizeof(float) * E)))
            return s;
    }
    // the solver evaluates both residuals of a node pair from either node's
    // out-edges, so the edge set must be symmetric with equal weights
    std::vector<std::pair<long long, float>> key(E);
    for (int k = 0; k < n; ++k)
        for (int e = eo[k]; e < eo[k + 1]; ++e) {
            const int l = ed[e];
            if (l < 0 || l >= n || l == k)
                return ctx->fail(LC_ERR_ARG, "lc_upload_graph: edge %d (%d -> %d) invalid", e, k, l);
            if (!(es[e] >= 0.f) || !std::isfinite(es[e]))
                return ctx->fail(LC_ERR_ARG, "lc_upload_graph: edge_s[%d] must be finite and >= 0", e);
            key[e] = {(long long)k * n + l, es[e]};
        }
    std::sort(key.begin(), key.end());
    for (int e = 0; e < E; ++e) {
        if (e > 0 && key[e].first == key[e - 1].first)
            return ctx->fail(LC_ERR_ARG, "lc_upload_graph: duplicate edge");
        const long long k = key[e].first / n, l = key[e].first % n;
        auto it = std::lower_bound(key.begin(), key.end(), std::make_pair(l * n + k, -INFINITY));
        if (it == key.end() || it->first != l * n + k || it->second != key[e].second)
            return ctx->fail(LC_ERR_ARG, "lc_upload_graph: edge %lld -> %lld has no reverse edge of equal weight", k, l);
    }
    cudaStream_t st = ctx->stream;
    graph_alloc(ctx, n, K);
    graph_alloc_edges(ctx, E);
    GraphScratch gs{};
    std::vector<void*> scratch;
    auto salloc = [&](size_t b) {
        void* p = ctx->alloc(b);
        scratch.push_back(p);
        return p;
    };
    gs.ent_cnt = (int*)salloc(sizeof(int) * (n + 1));
    gs.ent_fill = (int*)salloc(sizeof(int) * n);
    auto cleanup = [&]() {
        for (void* p : scratch) ctx->release(p);
    };
    if (ctx->alloc_failures != af0) {
        cleanup();
        return LC_ERR_OOM;
    }
    cudaMemcpyAsync((void*)C.node_vid, vid.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync((void*)C.bind_idx, bi.data(), sizeof(int) * NK, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync((void*)C.bind_w, bw.data(), sizeof(float) * NK, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync((void*)C.edge_off, eo.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st);
    if (E > 0) {
        cudaMemcpyAsync((void*)C.edge_dst, ed.data(), sizeof(int) * E, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync((void*)C.edge_s, es.data(), sizeof(float) * E, cudaMemcpyHostToDevice, st);
    }
    return graph_finish(ctx, gs, cleanup);
}

extern "C" lc_status lc_read_graph(lc_ctx* ctx, int32_t* node_vid, int32_t* bind_idx, float* bind_w, int32_t* edge_off,
                                   int32_t* edge_dst, float* edge_s, int* n_edges) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_graph) return ctx->fail(LC_ERR_STATE, "lc_read_graph: no graph");
    cudaSetDevice(ctx->device);
    const CapDesc& C = ctx->hC;
    lc_status s = LC_OK;
    struct Item {
        void* dst;
        const void* src;
        size_t bytes;
    } items[] = {{node_vid, C.node_vid, sizeof(int) * C.n},
                 {bind_idx, C.bind_idx, sizeof(int) * (size_t)C.N * C.K},
                 {bind_w, C.bind_w, sizeof(float) * (size_t)C.N * C.K},
                 {edge_off, C.edge_off, sizeof(int) * (C.n + 1)},
                 {edge_dst, C.edge_dst, sizeof(int) * C.E},
                 {edge_s, C.edge_s, sizeof(float) * C.E}};
    for (auto& it : items)
        if (it.dst && (s = ctx->cuda(cudaMemcpyAsync(it.dst, it.src, it.bytes, cudaMemcpyDefault, ctx->stream), "copy out")))
            return s;
    if (n_edges) *n_edges = C.E;
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
}

extern "C" lc_status lc_set_node_params(lc_ctx* ctx, const float* node_R, const float* node_t) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_graph) return ctx->fail(LC_ERR_STATE, "lc_set_node_params: no graph");
    cudaSetDevice(ctx->device);
    const int n = ctx->hC.n;
    if (!node_R && !node_t) {
        launch_identity_params(ctx->hC.node_R, ctx->hC.node_t, n, ctx->stream);
        return ctx->cuda(cudaGetLastError(), "identity params");
    }
    if (!node_R || !node_t) return ctx->fail(LC_ERR_ARG, "lc_set_node_params: give both arrays or neither");
    std::vector<float> R, t;
    lc_status s;
    if ((s = host_copy(ctx, R, node_R, (size_t)9 * n)) || (s = host_copy(ctx, t, node_t, (size_t)3 * n))) return s;
    std::vector<float4> R4(3 * n), t4(n);
    for (int k = 0; k < n; ++k) {
        for (int j = 0; j < 3; ++j) R4[3 * k + j] = make_float4(R[9 * k + 3 * j], R[9 * k + 3 * j + 1], R[9 * k + 3 * j + 2], 0.f);
        t4[k] = make_float4(t[3 * k], t[3 * k + 1], t[3 * k + 2], 0.f);
    }
    if ((s = ctx->cuda(cudaMemcpyAsync(ctx->hC.node_R, R4.data(), sizeof(float4) * 3 * n, cudaMemcpyHostToDevice, ctx->stream), "upload")) ||
        (s = ctx->cuda(cudaMemcpyAsync(ctx->hC.node_t, t4.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, ctx->stream), "upload")))
        return s;
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
}

extern "C" lc_status lc_set_rest_geometry(lc_ctx* ctx, const float* V_S) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_template) return ctx->fail(LC_ERR_STATE, "lc_set_rest_geometry: no template");
    cudaSetDevice(ctx->device);
    CapDesc& C = ctx->hC;
    const int N = C.N;
    lc_status s;
    if (!V_S) {
        s = ctx->cuda(cudaMemcpyAsync(ctx->base_buf, ctx->tpl, sizeof(float4) * N, cudaMemcpyDeviceToDevice, ctx->stream),
                      "copy");
    } else {
        std::vector<float> h;
        if ((s = host_copy(ctx, h, V_S, (size_t)3 * N))) return s;
        std::vector<float4> v4(N);
        for (int i = 0; i < N; ++i) {
            if (!std::isfinite(h[3 * i]) || !std::isfinite(h[3 * i + 1]) || !std::isfinite(h[3 * i + 2]))
                return ctx->fail(LC_ERR_ARG, "lc_set_rest_geometry: non-finite vertex");
            v4[i] = make_float4(h[3 * i], h[3 * i + 1], h[3 * i + 2], 0.f);
        }
        s = ctx->cuda(cudaMemcpyAsync(ctx->base_buf, v4.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, ctx->stream),
                      "upload");
    }
    if (s) return s;
    if (ctx->has_graph) launch_gather_nodes(ctx->base_buf, C.node_vid, C.n, (float4*)C.node_g, ctx->stream);
    ctx->has_lin = false;
    ctx->surf_has_lin = false;
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
}

// ---------------------------------------------------------------------------
// frame
// ---------------------------------------------------------------------------
extern "C" lc_status lc_upload_frame(lc_ctx* ctx, const float* rgb, const float* dt, const uint8_t* mask,
                                     const float* joints2d, const float* joints3d) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_camera) return ctx->fail(LC_ERR_STATE, "lc_upload_frame: no camera");
    if (!rgb || !mask) return ctx->fail(LC_ERR_ARG, "lc_upload_frame: null image");
    cudaSetDevice(ctx->device);
    CapDesc& C = ctx->hC;
    const size_t P = (size_t)C.W * C.H;
    cudaStream_t st = ctx->stream;
    const float* drgb = rgb;
    const float* ddt = dt;
    const uint8_t* dmask = mask;
    lc_status s;
    if (!lc_ctx::is_device_ptr(rgb)) {
        if ((s = ctx->cuda(cudaMemcpyAsync(ctx->stage_rgb, rgb, sizeof(float) * 3 * P, cudaMemcpyDefault, st), "frame upload")))
            return s;
        drgb = ctx->stage_rgb;
    }
    if (dt && !lc_ctx::is_device_ptr(dt)) {
        if ((s = ctx->cuda(cudaMemcpyAsync(ctx->stage_dt, dt, sizeof(float) * P, cudaMemcpyDefault, st), "frame upload")))
            return s;
        ddt = ctx->stage_dt;
    }
    if (!lc_ctx::is_device_ptr(mask)) {
        if ((s = ctx->cuda(cudaMemcpyAsync(ctx->stage_mask, mask, P, cudaMemcpyDefault, st), "frame upload"))) return s;
        dmask = ctx->stage_mask;
    }
    launch_pack_frame(drgb, ddt, dmask, (float4*)C.img, (uint8_t*)C.mask, C.W, C.H, st);
    if ((s = ctx->cuda(cudaGetLastError(), "pack frame"))) return s;
    if (!dt) {
        // the distance transform of the silhouette on the device (scratch on first use)
        if (!ctx->edt_g) {
            // column distances (int per pixel), then the contour flags (a byte per pixel)
            ctx->edt_g = (int*)ctx->alloc((sizeof(int) + 1) * P);
            if (!ctx->edt_g) return LC_ERR_OOM;
        }
        launch_edt(C.mask, (uint8_t*)(ctx->edt_g + P), ctx->edt_g, (float4*)C.img, C.W, C.H, st);
        if ((s = ctx->cuda(cudaGetLastError(), "distance transform"))) return s;
    }
    if (ctx->params.pyr_levels > 0) {
        const lc::CapDesc before = C;
        if ((s = ctx->build_pyramid())) return s;
        if (memcmp(&before, &C, sizeof(lc::CapDesc)) != 0 && (s = ctx->sync_desc())) return s;
    }
    if ((s = ctx->pose_frame(joints2d, joints3d))) return s;
    ctx->has_frame = true;
    ctx->has_vis = false;
    ctx->has_lin = false;
    return LC_OK;
}

// ---------------------------------------------------------------------------
// photometric pyramid (Sec. 3.4)
// ---------------------------------------------------------------------------
void lc_ctx::pyr_release() {
    for (int j = 0; j < 3; ++j) {
        release(pyr_buf[j]);
        pyr_buf[j] = nullptr;
        hC.lvl[j] = nullptr;
        hC.lvl_W[j] = hC.lvl_H[j] = 0;
    }
    release(pyr_tmp);
    pyr_tmp = nullptr;
    hC.pyr_levels = 0;
}

// Gaussian taps of an odd size k: sigma = 0.3((k-1)/2 - 1) + 0.8, normalised
// in FP64 and rounded once to FP32
static PyrTaps pyramid_taps(int k) {
    PyrTaps T{};
    T.r = (k - 1) / 2;
    if (T.r == 0) {
        T.w[0] = 1.f;
        return T;
    }
    const double sigma = 0.3 * (T.r - 1) + 0.8;
    double w[kPyrMaxTaps], sum = 0.0;
    for (int i = -T.r; i <= T.r; ++i) {
        w[i + T.r] = exp(-(double)(i * i) / (2.0 * sigma * sigma));
        sum += w[i + T.r];
    }
    for (int i = 0; i < 2 * T.r + 1; ++i) T.w[i] = (float)(w[i] / sum);
    return T;
}

lc_status lc_ctx::build_pyramid() {
    const int L = params.pyr_levels;
    const int W = hC.W, H = hC.H;
    if (L > 0 && !pyr_tmp && !(pyr_tmp = (float4*)alloc(sizeof(float4) * (size_t)W * H))) return LC_ERR_OOM;
    for (int j = 0; j < 3; ++j) {
        if (j < 3 - L) {
            hC.lvl[j] = nullptr;
            hC.lvl_W[j] = hC.lvl_H[j] = 0;
            continue;
        }
        const int d = pyr_factor(j), Wd = (W + d - 1) / d, Hd = (H + d - 1) / d;
        if (!pyr_buf[j] && !(pyr_buf[j] = (float4*)alloc(sizeof(float4) * (size_t)Wd * Hd))) return LC_ERR_OOM;
        launch_pyramid_level(hC.img, W, H, d, pyramid_taps(params.pyr_ksize[j]), pyr_tmp, pyr_buf[j], Wd, Hd, stream);
        hC.lvl[j] = pyr_buf[j];
        hC.lvl_W[j] = Wd;
        hC.lvl_H[j] = Hd;
    }
    hC.pyr_levels = L;
    return cuda(cudaGetLastError(), "pyramid");
}

extern "C" lc_status lc_read_pyramid_level(lc_ctx* ctx, int j, float* rgb, int* W_out, int* H_out) {
    if (!ctx) return LC_ERR_ARG;
    if (j < 0 || j > 2) return ctx->fail(LC_ERR_ARG, "lc_read_pyramid_level: level must be 0, 1 or 2");
    const CapDesc& C = ctx->hC;
    if (!ctx->has_frame || C.pyr_levels == 0 || j < 3 - C.pyr_levels)
        return ctx->fail(LC_ERR_STATE, "lc_read_pyramid_level: level %d not built", j);
    cudaSetDevice(ctx->device);
    const int Wd = C.lvl_W[j], Hd = C.lvl_H[j];
    if (W_out) *W_out = Wd;
    if (H_out) *H_out = Hd;
    if (!rgb) return LC_OK;
    const size_t P = (size_t)Wd * Hd;
    std::vector<float4> img(P);
    lc_status s;
    if ((s = ctx->copy_to_host(img.data(), C.lvl[j], sizeof(float4) * P))) return s;
    std::vector<float> out(3 * P);
    for (size_t p = 0; p < P; ++p) {
        out[3 * p] = img[p].x;
        out[3 * p + 1] = img[p].y;
        out[3 * p + 2] = img[p].z;
    }
    return ctx->deliver(rgb, out.data(), sizeof(float) * 3 * P);
}

extern "C" lc_status lc_read_frame(lc_ctx* ctx, float* dt, uint8_t* mask) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_frame) return ctx->fail(LC_ERR_STATE, "lc_read_frame: no frame");
    cudaSetDevice(ctx->device);
    const CapDesc& C = ctx->hC;
    const size_t P = (size_t)C.W * C.H;
    lc_status s;
    if (dt) {
        std::vector<float4> img(P);
        if ((s = ctx->copy_to_host(img.data(), C.img, sizeof(float4) * P))) return s;
        std::vector<float> d(P);
        for (size_t p = 0; p < P; ++p) d[p] = img[p].w;
        if ((s = ctx->deliver(dt, d.data(), sizeof(float) * P))) return s;
    }
    if (mask) {
        std::vector<uint8_t> m(P);
        if ((s = ctx->copy_to_host(m.data(), C.mask, P))) return s;
        if ((s = ctx->deliver(mask, m.data(), P))) return s;
    }
    return LC_OK;
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------
void lc_ctx::mark(int phase) {
    if (!profiling) return;
    if (prof_used == (int)prof_ev.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        prof_ev.push_back(e);
        prof_phase.push_back(-1);
    }
    prof_phase[prof_used] = phase;
    // external: a real event-record node in the captured graph (a plain record
    // during capture only expresses a dependency)
    cudaEventRecordWithFlags(prof_ev[prof_used], stream, cudaEventRecordExternal);
    ++prof_used;
}

void lc_ctx::mark_end() { mark(-1); }

lc_status lc_ctx::accumulate_profile(const ProfRange& r) {
    if (!profiling || r.end - r.begin < 2) return LC_OK;
    lc_status s = cuda(cudaStreamSynchronize(stream), "synchronize");
    if (s) return s;
    for (int j = r.begin; j + 1 < r.end; ++j) {
        if (prof_phase[j] < 0) continue;
        float ms = 0.f;
        if ((s = cuda(cudaEventElapsedTime(&ms, prof_ev[j], prof_ev[j + 1]), "event time"))) return s;
        prof_ms[prof_phase[j]] += ms;
        prof_cnt[prof_phase[j]] += 1;
    }
    return LC_OK;
}

void lc_ctx::enqueue_pcg() {
    if (use_cluster_pcg()) {
        mark(LC_PH_PCG);
        launch_pcg_cluster(dC, pcg_plan, hC.K, params.n_pcg, stream);
        return;
    }
    mark(LC_PH_PCG_INIT);
    launch_jtj_stage(dC, hC, stream);
    launch_pcg_init(dC, hC, stream);
    for (int it = 0; it < params.n_pcg; ++it) {
        mark(LC_PH_JTJ);
        launch_jtj(dC, hC, nullptr, nullptr, nullptr, nullptr, true, stream);
        mark(LC_PH_PCG_VEC);
        launch_pcg_vectors(dC, hC, stream);
    }
}

// A conditional IF node at the end of the capture in progress on `stream`;
// the capture continues into its body on the side stream until end_if().
void lc_ctx::begin_if(cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaStreamGetCaptureInfo(stream, &cs, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess ||
        cudaGraphAddNode(&node, g, deps, nullptr, nd, &p) != cudaSuccess ||
        cudaStreamUpdateCaptureDependencies(stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess ||
        cudaStreamBeginCaptureToGraph(side_stream, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cond_failed = true;
        return;
    }
    cond_bodies.push_back(p.conditional.phGraph_out[0]);
    saved_stream = stream;
    stream = side_stream;
}

void lc_ctx::end_if() {
    if (stream != side_stream) return;
    cudaGraph_t b = nullptr;
    if (cudaStreamEndCapture(side_stream, &b) != cudaSuccess) cond_failed = true;
    stream = saved_stream;
}

// The non-rigid solve.  With a target energy and gn_block > 0 (and no
// profiling: event records are not allowed in conditional bodies), the
// Gauss-Newton steps are captured in blocks of gn_block steps and every
// block after the first is the body of a conditional IF node whose condition
// the previous block's last kernel sets: the blocks after the target launch
// nothing.  Otherwise all n_gn steps are unrolled (steps after a target
// return at once).
void lc_ctx::enqueue_nonrigid() {
    const CapDesc& C = hC;
    cudaStream_t st = stream;
    prof_nonrigid.begin = prof_used;
    cudaMemsetAsync(C.hist, 0, sizeof(double) * 2 * (LC_MAX_GN + 1), st);
    cudaMemsetAsync(C.hist_iters, 0, sizeof(int) * (LC_MAX_GN + 2), st);
    cudaMemsetAsync((char*)C.sc + offsetof(Scalars, gn_stop), 0, 2 * sizeof(int), st);
    mark(LC_PH_VIS);
    launch_part_mask(dC, C, st);
    mark(LC_PH_WARP);
    launch_warp(dC, C, st);
    mark(LC_PH_VIS);
    launch_visibility(dC, C, st);
    const int B = params.gn_block;
    const int n_blocks = B > 0 ? (params.n_gn + B - 1) / B : 1;
    std::vector<cudaGraphConditionalHandle> hs(n_blocks, 0);
    bool cond = !profiling && params.target_energy > 0.f && n_blocks > 1 && side_stream;
    if (cond) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        if (cudaStreamGetCaptureInfo(stream, &cs, nullptr, &g) != cudaSuccess || cs != cudaStreamCaptureStatusActive)
            cond = false;
        for (int b = 1; cond && b < n_blocks; ++b)
            if (cudaGraphConditionalHandleCreate(&hs[b], g, 0, cudaGraphCondAssignDefault) != cudaSuccess)
                cond_failed = true;
        cudaGetLastError();
    }
    for (int gn = 0; gn < params.n_gn; ++gn) {
        const int blk = cond ? gn / B : 0;
        const bool first_of_block = cond && gn % B == 0, last_of_block = cond && (gn % B == B - 1 || gn == params.n_gn - 1);
        if (first_of_block && blk > 0) begin_if(hs[blk]);
        if (gn > 0) {
            mark(LC_PH_WARP);
            launch_warp(dC, C, stream, true);
        }
        mark(LC_PH_LIN);
        launch_linearize(dC, C, true, gn, stream);
        mark(LC_PH_RHS);
        launch_rhs(dC, C, gn, false, stream);
        enqueue_pcg();
        mark(LC_PH_UPDATE);
        launch_update(dC, C, gn, stream);
        if (last_of_block && blk + 1 < n_blocks) launch_gn_gate(dC, hs[blk + 1], stream);
        if (last_of_block && blk > 0) end_if();
    }
    mark(LC_PH_WARP);
    launch_warp(dC, C, st);
    mark(LC_PH_LIN);
    launch_linearize(dC, C, false, LC_MAX_GN, st);
    mark(LC_PH_RHS);
    launch_rhs(dC, C, params.n_gn, true, st);
    launch_vis_unfreeze(dC, st);
    mark_end();
    prof_nonrigid.end = prof_used;
}

static int kernel_nodes(cudaGraph_t g) {
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    int k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

lc_status lc_ctx::capture(cudaGraphExec_t* exec, int* n_kernels, void (lc_ctx::*enqueue)(), int* n_kernels_step) {
    cudaGraph_t g = nullptr;
    lc_status s;
    if (!side_stream && cudaStreamCreateWithFlags(&side_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        side_stream = nullptr;   // no conditional steps
    }
    cond_bodies.clear();
    cond_failed = false;
    if ((s = cuda(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "begin capture"))) return s;
    (this->*enqueue)();
    if (stream == side_stream) end_if();   // an unbalanced body (cannot happen) is closed
    cudaError_t e = cudaStreamEndCapture(stream, &g);
    if ((s = cuda(e, "end capture"))) return s;
    if (cond_failed) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(LC_ERR_CUDA, "capture: conditional graph nodes could not be built");
    }
    *n_kernels = kernel_nodes(g);
    if (n_kernels_step) *n_kernels_step = cond_bodies.empty() ? 0 : kernel_nodes(cond_bodies[0]);
    cond_bodies.clear();
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return cuda(e, "graph instantiate");
}

lc_status lc_ctx::check_solve_state(const char* who) {
    if (!has_template || !has_graph) return fail(LC_ERR_STATE, "%s: template and graph required", who);
    if (!has_camera || !has_frame) return fail(LC_ERR_STATE, "%s: camera and frame required", who);
    return LC_OK;
}

lc_status lc_ctx::read_stats(lc_solve_stats* stats, int n_gn, bool surface) {
    Scalars sc;
    std::vector<double> hist(2 * (LC_MAX_GN + 1));
    std::vector<int> it(LC_MAX_GN + 2);
    lc_status s;
    if ((s = copy_to_host(&sc, hC.sc, sizeof(Scalars))) || (s = copy_to_host(hist.data(), hC.hist, sizeof(double) * hist.size())) ||
        (s = copy_to_host(it.data(), hC.hist_iters, sizeof(int) * it.size())))
        return s;
    if (sc.status & kDevErrCapacity) {
        cudaMemsetAsync((char*)hC.sc + offsetof(Scalars, status), 0, sizeof(int), stream);
        return fail(LC_ERR_NUMERIC, "internal: the cluster PCG's staging exceeded its planned capacity");
    }
    if (sc.status & kDevErrWait) {
        cudaMemsetAsync((char*)hC.sc + offsetof(Scalars, status), 0, sizeof(int), stream);
        return fail(LC_ERR_TIMEOUT, "a bounded wait for the TMA-staged image taps ran out (the global loads were used)");
    }
    memset(stats, 0, sizeof(*stats));
    stats->e_photo = sc.e_lin[0];
    stats->e_sil = sc.e_lin[1];
    stats->e_arap = sc.e_lin[2];
    stats->e_total = sc.e_lin[0] + sc.e_lin[1] + sc.e_lin[2];
    if (surface) {
        stats->e_arap = 0.0;
        stats->e_smooth = sc.e_reg[0];
        stats->e_edge = sc.e_reg[1];
        stats->e_velocity = sc.e_reg[2];
        stats->e_acceleration = sc.e_reg[3];
        stats->e_total = sc.e_lin[0] + sc.e_lin[1] + sc.e_reg[0] + sc.e_reg[1] + sc.e_reg[2] + sc.e_reg[3];
    }
    for (int g = 0; g < n_gn; ++g) {
        stats->e_gn[g] = hist[2 * g];
        stats->step_norm[g] = hist[2 * g + 1];
        stats->pcg_iters[g] = it[g];
    }
    stats->n_gn_done = sc.gn_done;
    stats->n_visible = sc.counts[0];
    stats->n_boundary = sc.counts[1];
    stats->n_boundary_neg = sc.counts[2];
    stats->pcg_breakdowns = it[LC_MAX_GN + 1];
    return LC_OK;
}

extern "C" lc_status lc_solve_nonrigid(lc_ctx* ctx, lc_solve_stats* stats) {
    if (!ctx) return LC_ERR_ARG;
    lc_status s;
    if ((s = ctx->check_solve_state("lc_solve_nonrigid"))) return s;
    cudaSetDevice(ctx->device);
    if (!ctx->gexec && (s = ctx->capture(&ctx->gexec, &ctx->graph_kernels, &lc_ctx::enqueue_nonrigid,
                                         &ctx->graph_kernels_step)))
        return s;
    if ((s = ctx->cuda(cudaGraphLaunch(ctx->gexec, ctx->stream), "graph launch"))) return s;
    if ((s = ctx->accumulate_profile(ctx->prof_nonrigid))) return s;
    ctx->has_vis = true;
    ctx->has_lin = true;
    ctx->surf_has_lin = false;
    ctx->last_surface = false;
    if (stats) {
        if ((s = ctx->read_stats(stats, ctx->params.n_gn))) return s;
        stats->n_kernels = ctx->graph_kernels;
        stats->n_kernels_step = ctx->graph_kernels_step;
        stats->pcg_cluster_size = ctx->use_cluster_pcg() ? ctx->pcg_plan.cl : 0;
    }
    return LC_OK;
}

extern "C" lc_status lc_read_stats(lc_ctx* ctx, lc_solve_stats* stats) {
    if (!ctx || !stats) return LC_ERR_ARG;
    if (ctx->last_surface ? !ctx->surf_gexec : !ctx->gexec)
        return ctx->fail(LC_ERR_STATE, "lc_read_stats: no non-rigid solve yet");
    cudaSetDevice(ctx->device);
    lc_status s;
    if (ctx->last_surface) {
        if ((s = ctx->read_stats(stats, ctx->params.n_gn_surface, true))) return s;
        stats->n_kernels = ctx->surf_graph_kernels;
        stats->pcg_cluster_size = ctx->surf_cl > 0 && ctx->params.pcg_kernel == 0 ? ctx->surf_cl : 0;
        return LC_OK;
    }
    if ((s = ctx->read_stats(stats, ctx->params.n_gn))) return s;
    stats->n_kernels = ctx->graph_kernels;
    stats->n_kernels_step = ctx->graph_kernels_step;
    stats->pcg_cluster_size = ctx->use_cluster_pcg() ? ctx->pcg_plan.cl : 0;
    return LC_OK;
}

extern "C" lc_status lc_set_profiling(lc_ctx* ctx, int on) {
    if (!ctx) return LC_ERR_ARG;
    cudaSetDevice(ctx->device);
    if ((on != 0) != ctx->profiling) {
        ctx->profiling = on != 0;
        ctx->drop_graph();
        ctx->pose_drop_graph();
        ctx->prof_used = 0;
        ctx->prof_nonrigid = ctx->prof_pose = ctx->prof_surface = lc_ctx::ProfRange{};
    }
    for (int j = 0; j < LC_N_PHASES; ++j) {
        ctx->prof_ms[j] = 0.0;
        ctx->prof_cnt[j] = 0;
    }
    return LC_OK;
}

extern "C" lc_status lc_read_profile(lc_ctx* ctx, double* ms, int* count) {
    if (!ctx || !ms) return LC_ERR_ARG;
    lc_status s = ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
    if (s) return s;
    for (int j = 0; j < LC_N_PHASES; ++j) {
        ms[j] = ctx->prof_ms[j];
        if (count) count[j] = ctx->prof_cnt[j];
        ctx->prof_ms[j] = 0.0;
        ctx->prof_cnt[j] = 0;
    }
    return LC_OK;
}

extern "C" lc_status lc_read_back(lc_ctx* ctx, float* node_R, float* node_t, float* V_out, uint8_t* flags, float* pose) {
    if (!ctx) return LC_ERR_ARG;
    cudaSetDevice(ctx->device);
    const CapDesc& C = ctx->hC;
    lc_status s;
    if ((node_R || node_t) && !ctx->has_graph) return ctx->fail(LC_ERR_STATE, "lc_read_back: no graph");
    if ((V_out || flags) && !ctx->has_template) return ctx->fail(LC_ERR_STATE, "lc_read_back: no template");
    if (node_R) {
        std::vector<float4> R4(3 * C.n);
        if ((s = ctx->copy_to_host(R4.data(), C.node_R, sizeof(float4) * 3 * C.n))) return s;
        std::vector<float> R(9 * C.n);
        for (int k = 0; k < C.n; ++k)
            for (int j = 0; j < 3; ++j) {
                R[9 * k + 3 * j] = R4[3 * k + j].x;
                R[9 * k + 3 * j + 1] = R4[3 * k + j].y;
                R[9 * k + 3 * j + 2] = R4[3 * k + j].z;
            }
        if ((s = ctx->deliver(node_R, R.data(), sizeof(float) * R.size()))) return s;
    }
    if (node_t) {
        std::vector<float4> t4(C.n);
        if ((s = ctx->copy_to_host(t4.data(), C.node_t, sizeof(float4) * C.n))) return s;
        std::vector<float> t(3 * C.n);
        for (int k = 0; k < C.n; ++k) {
            t[3 * k] = t4[k].x;
            t[3 * k + 1] = t4[k].y;
            t[3 * k + 2] = t4[k].z;
        }
        if ((s = ctx->deliver(node_t, t.data(), sizeof(float) * t.size()))) return s;
    }
    if (V_out) {
        std::vector<float4> v4(C.N);
        if ((s = ctx->copy_to_host(v4.data(), C.vw, sizeof(float4) * C.N))) return s;
        std::vector<float> v(3 * C.N);
        for (int i = 0; i < C.N; ++i) {
            v[3 * i] = v4[i].x;
            v[3 * i + 1] = v4[i].y;
            v[3 * i + 2] = v4[i].z;
        }
        if ((s = ctx->deliver(V_out, v.data(), sizeof(float) * v.size()))) return s;
    }
    if (flags) {
        std::vector<uint32_t> f(C.N);
        if ((s = ctx->copy_to_host(f.data(), C.flags, sizeof(uint32_t) * C.N))) return s;
        std::vector<uint8_t> f8(C.N);
        for (int i = 0; i < C.N; ++i) f8[i] = (uint8_t)f[i];
        if ((s = ctx->deliver(flags, f8.data(), f8.size()))) return s;
    }
    if (pose && (s = ctx->pose_read(pose))) return s;
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
}

// ---------------------------------------------------------------------------
// inspection
// ---------------------------------------------------------------------------
extern "C" lc_status lc_compute_visibility(lc_ctx* ctx) {
    if (!ctx) return LC_ERR_ARG;
    lc_status s;
    if ((s = ctx->check_solve_state("lc_compute_visibility"))) return s;
    cudaSetDevice(ctx->device);
    launch_vis_unfreeze(ctx->dC, ctx->stream);
    launch_part_mask(ctx->dC, ctx->hC, ctx->stream);
    launch_warp(ctx->dC, ctx->hC, ctx->stream);
    launch_visibility(ctx->dC, ctx->hC, ctx->stream);
    ctx->has_vis = true;
    ctx->has_lin = false;
    return ctx->cuda(cudaGetLastError(), "visibility");
}

extern "C" lc_status lc_read_visibility(lc_ctx* ctx, uint64_t* zbuf, uint8_t* flags, float* uv) {
    if (!ctx) return LC_ERR_ARG;
    if (!ctx->has_vis) return ctx->fail(LC_ERR_STATE, "lc_read_visibility: no visibility pass yet");
    cudaSetDevice(ctx->device);
    const CapDesc& C = ctx->hC;
    lc_status s;
    if (zbuf && (s = ctx->cuda(cudaMemcpyAsync(zbuf, C.zbuf, sizeof(uint64_t) * (size_t)C.W * C.H, cudaMemcpyDefault, ctx->stream), "copy out")))
        return s;
    if (uv && (s = ctx->cuda(cudaMemcpyAsync(uv, C.uv, sizeof(float2) * C.N, cudaMemcpyDefault, ctx->stream), "copy out")))
        return s;
    if (flags) {
        std::vector<uint32_t> f(C.N);
        if ((s = ctx->copy_to_host(f.data(), C.flags, sizeof(uint32_t) * C.N))) return s;
        std::vector<uint8_t> f8(C.N);
        for (int i = 0; i < C.N; ++i) f8[i] = (uint8_t)f[i];
        if ((s = ctx->deliver(flags, f8.data(), f8.size()))) return s;
    }
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
}

lc_status lc_ctx::linearize_now(bool with_rhs) {
    cudaMemsetAsync((char*)hC.sc + offsetof(Scalars, gn_stop), 0, sizeof(int), stream);
    launch_warp(dC, hC, stream);
    launch_linearize(dC, hC, true, 0, stream);
    launch_rhs(dC, hC, LC_MAX_GN, !with_rhs, stream);
    has_lin = true;
    return cuda(cudaGetLastError(), "linearize");
}

extern "C" lc_status lc_eval_linearization(lc_ctx* ctx, float* v_warp, float* uv, float* r_photo, float* r_sil, float* H,
                                           float* e, double* energy) {
    if (!ctx) return LC_ERR_ARG;
    lc_status s;
    if ((s = ctx->check_solve_state("lc_eval_linearization"))) return s;
    if (!ctx->has_vis) return ctx->fail(LC_ERR_STATE, "lc_eval_linearization: no visibility pass yet");
    cudaSetDevice(ctx->device);
    if ((s = ctx->linearize_now(true))) return s;
    const CapDesc& C = ctx->hC;
    const int N = C.N;
    std::vector<float4> a(N), b(N);
    std::vector<float> out;
    auto emit = [&](float* dst, int width, auto fn) -> lc_status {
        if (!dst) return LC_OK;
        out.assign((size_t)N * width, 0.f);
        for (int i = 0; i < N; ++i) fn(i, &out[(size_t)i * width]);
        return ctx->deliver(dst, out.data(), sizeof(float) * out.size());
    };
    if (v_warp) {
        if ((s = ctx->copy_to_host(a.data(), C.vw, sizeof(float4) * N))) return s;
        if ((s = emit(v_warp, 3, [&](int i, float* o) { o[0] = a[i].x; o[1] = a[i].y; o[2] = a[i].z; }))) return s;
    }
    if (uv && (s = ctx->cuda(cudaMemcpyAsync(uv, C.uv, sizeof(float2) * N, cudaMemcpyDefault, ctx->stream), "copy out")))
        return s;
    if (r_photo || r_sil) {
        if ((s = ctx->copy_to_host(a.data(), C.res, sizeof(float4) * N))) return s;
        if ((s = emit(r_photo, 3, [&](int i, float* o) { o[0] = a[i].x; o[1] = a[i].y; o[2] = a[i].z; }))) return s;
        if ((s = emit(r_sil, 1, [&](int i, float* o) { o[0] = a[i].w; }))) return s;
    }
    if (H) {
        if ((s = ctx->copy_to_host(a.data(), C.HA, sizeof(float4) * N)) || (s = ctx->copy_to_host(b.data(), C.HB, sizeof(float4) * N)))
            return s;
        if ((s = emit(H, 6, [&](int i, float* o) {
                 o[0] = a[i].x; o[1] = a[i].y; o[2] = a[i].z; o[3] = a[i].w; o[4] = b[i].x; o[5] = b[i].y;
             })))
            return s;
    }
    if (e) {
        if ((s = ctx->copy_to_host(a.data(), C.ev, sizeof(float4) * N))) return s;
        if ((s = emit(e, 3, [&](int i, float* o) { o[0] = a[i].x; o[1] = a[i].y; o[2] = a[i].z; }))) return s;
    }
    if (energy) {
        Scalars sc;
        if ((s = ctx->copy_to_host(&sc, C.sc, sizeof(Scalars)))) return s;
        double en[3] = {sc.e_lin[0], sc.e_lin[1], sc.e_lin[2]};
        if ((s = ctx->deliver(energy, en, sizeof(en)))) return s;
    }
    return ctx->cuda(cudaStreamSynchronize(ctx->stream), "synchronize");
}

lc_status lc_ctx::vec_out(float* dst, const float4* src) {
    if (!dst) return LC_OK;
    const int n = hC.n;
    launch_unpack_vec(src, tmp_out(), n, stream);
    std::vector<float> h(6 * n);
    lc_status s;
    if ((s = copy_to_host(h.data(), tmp_out(), sizeof(float) * 6 * n))) return s;
    return deliver(dst, h.data(), sizeof(float) * h.size());
}

float* lc_ctx::tmp_out() {
    if (!tmp6 || tmp6_cap < 6 * hC.n) {
        release(tmp6);
        tmp6 = (float*)alloc(sizeof(float) * 6 * std::max(hC.n, 1));
        tmp6_cap = 6 * hC.n;
    }
    return tmp6;
}

extern "C" lc_status lc_eval_gradient(lc_ctx* ctx, float* rhs, float* diag) {
    if (!ctx) return LC_ERR_ARG;
    lc_status s;
    if ((s = ctx->check_solve_state("lc_eval_gradient"))) return s;
    if (!ctx->has_vis) return ctx->fail(LC_ERR_STATE, "lc_eval_gradient: no visibility pass yet");
    cudaSetDevice(ctx->device);
    if ((s = ctx->linearize_now(true))) return s;
    if ((s = ctx->vec_out(rhs, ctx->hC.b))) return s;
    return ctx->vec_out(diag, ctx->hC.diag);
}

extern "C" lc_status lc_apply_jtj(lc_ctx* ctx, const float* p, float* out) {
    if (!ctx || !p || !out) return LC_ERR_ARG;
    if (!ctx->has_lin) return ctx->fail(LC_ERR_STATE, "lc_apply_jtj: no linearisation (call lc_eval_linearization)");
    cudaSetDevice(ctx->device);
    const int n = ctx->hC.n;
    std::vector<float> hp;
    lc_status s;
    if ((s = host_copy(ctx, hp, p, (size_t)6 * n))) return s;
    if ((s = ctx->cuda(cudaMemcpyAsync(ctx->tmp_out(), hp.data(), sizeof(float) * 6 * n, cudaMemcpyHostToDevice, ctx->stream), "upload")))
        return s;
    launch_pack_vec(ctx->tmp_out(), ctx->tmp_vec, n, ctx->stream);
    launch_jtj_stage(ctx->dC, ctx->hC, ctx->stream);
    launch_jtj(ctx->dC, ctx->hC, ctx->tmp_vec, nullptr, ctx->tmp_vec2, nullptr, false, ctx->stream);
    if ((s = ctx->cuda(cudaGetLastError(), "jtj"))) return s;
    return ctx->vec_out(out, ctx->tmp_vec2);
}

extern "C" lc_status lc_solve_linear(lc_ctx* ctx, float* delta, int* iters) {
    if (!ctx || !delta) return LC_ERR_ARG;
    if (!ctx->has_lin) return ctx->fail(LC_ERR_STATE, "lc_solve_linear: no linearisation (call lc_eval_linearization)");
    cudaSetDevice(ctx->device);
    const bool prof = ctx->profiling;
    ctx->profiling = false;
    cudaMemsetAsync((char*)ctx->hC.sc + offsetof(Scalars, gn_stop), 0, sizeof(int), ctx->stream);
    ctx->enqueue_pcg();
    ctx->profiling = prof;
    lc_status s;
    if ((s = ctx->cuda(cudaGetLastError(), "pcg"))) return s;
    if ((s = ctx->vec_out(delta, ctx->hC.x))) return s;
    if (iters) {
        Scalars sc;
        if ((s = ctx->copy_to_host(&sc, ctx->hC.sc, sizeof(Scalars)))) return s;
        *iters = sc.iters;
    }
    return LC_OK;
}

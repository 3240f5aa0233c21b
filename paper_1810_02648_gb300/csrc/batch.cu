// Batched non-rigid stage: many captures of uneven mesh and image size solved
// together, one launch per phase for all of them, the whole Gauss-Newton /
// PCG loop captured as one CUDA graph.
//
// Every kernel of the single-capture path already takes a descriptor array
// and a (capture, tile) work list; the batch concatenates the captures' tile
// lists per tile family.  The PCG runs as the cluster-persistent kernel, one
// cluster per capture, for groups of captures (same K) whose common plan fits
// in shared memory; the rest use the per-iteration kernels over their own
// work lists.  Each capture keeps its own buffers, reductions and counters
// (its context's), so a capture's arithmetic does not depend on the others:
// its result is bit-identical to its single-capture solve with the same PCG
// kernel and cluster size.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "lc_context.h"

using namespace lc;

namespace lc {

constexpr int kPixTile = 2048;   // z-buffer pixels cleared per block (256 threads x 8)

// Frame reset of every capture: the per-step history zeroed (tile 0 of each
// capture); the z-buffer cleared and the visibility counters zeroed unless
// the capture's frame decisions are frozen (a warm start kept those of its
// start: the visibility kernels then skip the capture).
__global__ void __launch_bounds__(256) batch_reset_kernel(const CapDesc* __restrict__ caps,
                                                          const WorkItem* __restrict__ items) {
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    const bool frozen = C.sc->vis_frozen != 0;
    const size_t P = (size_t)C.W * C.H;
    const size_t p0 = (size_t)tile * kPixTile;
    if (!frozen)
        for (int j = threadIdx.x; j < kPixTile; j += blockDim.x) {
            const size_t p = p0 + j;
            if (p < P) C.zbuf[p] = ~0ULL;
        }
    if (tile == 0) {
        for (int j = threadIdx.x; j < 2 * (LC_MAX_GN + 1); j += blockDim.x) C.hist[j] = 0.0;
        for (int j = threadIdx.x; j < LC_MAX_GN + 2; j += blockDim.x) C.hist_iters[j] = 0;
        if (!frozen && threadIdx.x < 3) C.sc->counts[threadIdx.x] = 0;
        if (threadIdx.x == 0) {
            C.sc->gn_stop = 0;
            C.sc->gn_done = 0;
        }
    }
}

// End of a batched solve: the next visibility pass of every capture runs again.
__global__ void __launch_bounds__(256) batch_unfreeze_kernel(const CapDesc* __restrict__ caps, int count) {
    for (int c = threadIdx.x; c < count; c += blockDim.x) caps[c].sc->vis_frozen = 0;
}

// Node parameters of every capture back to the identity.
__global__ void __launch_bounds__(kVecThreads) batch_identity_kernel(const CapDesc* __restrict__ caps,
                                                                     const WorkItem* __restrict__ items) {
    int cap, tile;
    decode(items, cap, tile);
    const CapDesc& C = caps[cap];
    const int k = tile * kVecThreads + threadIdx.x;
    if (k >= C.n) return;
    C.node_R[3 * k + 0] = make_float4(1.f, 0.f, 0.f, 0.f);
    C.node_R[3 * k + 1] = make_float4(0.f, 1.f, 0.f, 0.f);
    C.node_R[3 * k + 2] = make_float4(0.f, 0.f, 1.f, 0.f);
    C.node_t[k] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace lc

struct BatchGroup {
    int first = 0, count = 0;   // slots in the batch's descriptor array
    int K = 0;
    PcgPlan plan{};
};

struct lc_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<lc_ctx*> ctxs;        // in caller order
    std::vector<int> slot_of;         // caller index -> descriptor slot
    std::vector<int> ctx_of;          // descriptor slot -> caller index
    std::vector<CapDesc> snap;        // descriptors as uploaded (slot order)
    CapDesc* dC = nullptr;
    WorkItem* items = nullptr;        // all work lists, one allocation
    Tiles all, multi;                 // every capture / captures on the per-iteration PCG
    const WorkItem* pix_items = nullptr;
    int pix_blocks = 0;
    std::vector<BatchGroup> groups;   // captures on the cluster PCG
    int mode = LC_BATCH_PCG_AUTO;
    // launch shape of the per-iteration J^T J p (captures not on a cluster)
    int jv_block = kVertTile, jn_warps = kJtjNodeWarps, jn_unroll = 4;
    int first_multi = 0;              // first slot on the per-iteration / grid PCG
    int n_gn = 0, n_pcg = 0;
    cudaGraphExec_t gexec = nullptr;
    bool gexec_identity = false;
    // the frame-step graph (lc_batch_step) and the network it was captured for
    cudaGraphExec_t step_gexec = nullptr;
    unsigned long long step_uid = 0, step_gen = 0;
    unsigned step_flags = 0;
    int step_kernels = 0;
    bool solved = false;              // a solve has run: linearisations and directions exist
    std::vector<cudaEvent_t> ev;      // per member: its stream's work before the solve
    cudaEvent_t done = nullptr;       // the batch solve, awaited by every member's stream
    int graph_kernels = 0;
    std::string err;

    lc_status fail(lc_status st, const char* msg) {
        err = msg;
        return st;
    }
    void free_plan() {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        if (step_gexec) cudaGraphExecDestroy(step_gexec);
        step_gexec = nullptr;
        if (items) cudaFree(items);
        items = nullptr;
        if (dC) cudaFree(dC);
        dC = nullptr;
    }
    lc_status build();
    void enqueue(bool from_identity);
};

// Descriptor order, work lists and PCG groups for the current mode.
lc_status lc_batch::build() {
    free_plan();
    const int count = (int)ctxs.size();
    // cluster-PCG candidates: the mode's cluster size must fit the capture
    // on its own; grouped by K, ascending node count, greedily while the
    // common plan fits
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::vector<int> cl_of(count, 0);
    for (int i = 0; i < count; ++i) {
        lc_ctx* c = ctxs[i];
        int cl = 0;
        if (mode == LC_BATCH_PCG_AUTO && c->use_cluster_pcg()) cl = c->pcg_plan.cl;
        if (mode == LC_BATCH_PCG_CLUSTER8 || mode == LC_BATCH_PCG_CLUSTER16) {
            const int want = mode == LC_BATCH_PCG_CLUSTER8 ? 8 : 16;
            const int n = c->hC.n;
            const PcgPartition* pp = &c->pcg_part;
            PcgPlan pl;
            if (plan_pcg_cluster_group(want, &pp, &n, c->hC.K, 1, &pl)) cl = want;
        }
        cl_of[i] = cl;
    }
    cudaGetLastError();
    // slot order: cluster captures by (cl, K, n), then the rest
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const bool ca = cl_of[a] != 0, cb = cl_of[b] != 0;
        if (ca != cb) return ca;
        if (cl_of[a] != cl_of[b]) return cl_of[a] < cl_of[b];
        if (ctxs[a]->hC.K != ctxs[b]->hC.K) return ctxs[a]->hC.K < ctxs[b]->hC.K;
        return ctxs[a]->hC.n < ctxs[b]->hC.n;
    });
    groups.clear();
    int s = 0;
    while (s < count && cl_of[order[s]]) {
        BatchGroup g;
        g.first = s;
        g.K = ctxs[order[s]]->hC.K;
        const int cl = cl_of[order[s]];
        std::vector<int> ns;
        std::vector<const PcgPartition*> ps;
        int e = s;
        PcgPlan best{};
        while (e < count && cl_of[order[e]] == cl && ctxs[order[e]]->hC.K == g.K) {
            const int i = order[e];
            ns.push_back(ctxs[i]->hC.n);
            ps.push_back(&ctxs[i]->pcg_part);
            PcgPlan pl;
            if (!plan_pcg_cluster_group(cl, ps.data(), ns.data(), g.K, (int)ns.size(), &pl)) {
                ns.pop_back();
                ps.pop_back();
                break;
            }
            best = pl;
            ++e;
        }
        if (e == s) break;   // cannot happen for a capture that fits alone; the rest go per-iteration
        g.count = e - s;
        g.plan = best;
        groups.push_back(g);
        s = e;
    }
    first_multi = s;
    slot_of.assign(count, 0);
    ctx_of.assign(count, 0);
    snap.resize(count);
    for (int j = 0; j < count; ++j) {
        ctx_of[j] = order[j];
        slot_of[order[j]] = j;
        snap[j] = ctxs[order[j]]->hC;
    }
    // work lists
    std::vector<WorkItem> w;
    struct Fam {
        size_t off;
        int n;
    };
    auto family = [&](int lo, int hi, auto tiles_of) {
        Fam f{w.size(), 0};
        for (int j = lo; j < hi; ++j) {
            const int t = tiles_of(snap[j]);
            for (int q = 0; q < t; ++q) w.push_back({j, q});
            f.n += t;
        }
        return f;
    };
    auto vert = [](const CapDesc& C) { return C.vert_tiles; };
    auto tri = [](const CapDesc& C) { return C.tri_tiles; };
    auto medge = [](const CapDesc& C) { return C.medge_tiles; };
    auto node = [](const CapDesc& C) { return C.node_tiles; };
    auto vec = [](const CapDesc& C) { return (C.n + kVecThreads - 1) / kVecThreads; };
    auto pix = [](const CapDesc& C) { return (int)(((size_t)C.W * C.H + kPixTile - 1) / kPixTile); };
    const Fam fa[6] = {family(0, count, vert), family(0, count, tri), family(0, count, medge),
                       family(0, count, node), family(0, count, vec), family(0, count, pix)};
    const Fam fm[3] = {family(first_multi, count, vert), family(first_multi, count, node),
                       family(first_multi, count, vec)};
    // the J^T J p's own blocks at the batch's launch shape
    const int vb = jv_block, nb = jn_warps * kJtjNodesPerWarp;
    auto jvert = [vb](const CapDesc& C) { return (C.N + vb - 1) / vb; };
    auto jnode = [nb](const CapDesc& C) { return (C.n + nb - 1) / nb; };
    const Fam fj[4] = {family(0, count, jvert), family(0, count, jnode), family(first_multi, count, jvert),
                       family(first_multi, count, jnode)};
    if (cudaMalloc(&items, sizeof(WorkItem) * std::max<size_t>(w.size(), 1)) != cudaSuccess ||
        cudaMalloc(&dC, sizeof(CapDesc) * count) != cudaSuccess) {
        cudaGetLastError();
        return fail(LC_ERR_OOM, "lc_batch: device memory");
    }
    cudaMemcpy(items, w.data(), sizeof(WorkItem) * w.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(dC, snap.data(), sizeof(CapDesc) * count, cudaMemcpyHostToDevice);
    auto at = [&](const Fam& f) { return f.n ? items + f.off : nullptr; };
    all = Tiles{};
    all.vert = fa[0].n, all.vert_items = at(fa[0]);
    all.tri = fa[1].n, all.tri_items = at(fa[1]);
    all.medge = fa[2].n, all.medge_items = at(fa[2]);
    all.node = fa[3].n, all.node_items = at(fa[3]);
    all.vec = fa[4].n, all.vec_items = at(fa[4]);
    pix_blocks = fa[5].n, pix_items = at(fa[5]);
    multi = Tiles{};
    multi.vert = fm[0].n, multi.vert_items = at(fm[0]);
    multi.node = fm[1].n, multi.node_items = at(fm[1]);
    multi.vec = fm[2].n, multi.vec_items = at(fm[2]);
    for (Tiles* T : {&all, &multi}) {
        T->jv_block = jv_block;
        T->jn_warps = jn_warps;
        T->jn_unroll = jn_unroll;
    }
    // the common K of a tile set's captures (0: mixed)
    auto common_k = [&](int lo) {
        int k = lo < count ? snap[lo].K : 0;
        for (int j = lo; j < count; ++j)
            if (snap[j].K != k) k = 0;
        return k;
    };
    all.jk = common_k(0);
    multi.jk = common_k(first_multi);
    all.jv = fj[0].n, all.jv_items = at(fj[0]);
    all.jn = fj[1].n, all.jn_items = at(fj[1]);
    multi.jv = fj[2].n, multi.jv_items = at(fj[2]);
    multi.jn = fj[3].n, multi.jn_items = at(fj[3]);
    if (cudaGetLastError() != cudaSuccess) return fail(LC_ERR_CUDA, "lc_batch: uploading the work lists");
    return LC_OK;
}

void lc_batch::enqueue(bool from_identity) {
    cudaStream_t st = stream;
    // body-part masks of the members that have one, from their rest geometry
    // (each rasterises into its own z-buffer, which the reset clears again)
    for (size_t j = 0; j < snap.size(); ++j)
        if (snap[j].part_on) launch_part_mask(dC + j, snap[j], st);
    if (from_identity && all.vec) batch_identity_kernel<<<all.vec, kVecThreads, 0, st>>>(dC, all.vec_items);
    if (pix_blocks) batch_reset_kernel<<<pix_blocks, 256, 0, st>>>(dC, pix_items);
    launch_warp(dC, all, st);
    launch_visibility_kernels(dC, all, st);
    for (int gn = 0; gn < n_gn; ++gn) {
        if (gn > 0) launch_warp(dC, all, st, true);
        launch_linearize(dC, all, true, gn, st);
        launch_rhs(dC, all, gn, false, st);
        for (const BatchGroup& g : groups)
            launch_pcg_cluster(dC + g.first, g.plan, g.K, n_pcg, st, g.count);
        if (multi.vec) {
            launch_jtj_stage(dC, multi, st);
            launch_pcg_init(dC, multi, st);
            for (int it = 0; it < n_pcg; ++it) {
                launch_jtj(dC, multi, nullptr, nullptr, nullptr, nullptr, true, st);
                launch_pcg_vectors(dC, multi, st);
            }
        }
        launch_update(dC, all, gn, st);
    }
    launch_warp(dC, all, st);
    launch_linearize(dC, all, false, LC_MAX_GN, st);
    launch_rhs(dC, all, n_gn, true, st);
    batch_unfreeze_kernel<<<1, 256, 0, st>>>(dC, (int)snap.size());
}

static lc_status batch_check(lc_batch* b) {
    for (lc_ctx* c : b->ctxs) {
        if (!c->has_template || !c->has_graph || !c->has_camera || !c->has_frame)
            return b->fail(LC_ERR_STATE, "lc_batch: every context needs template, graph, camera and frame");
        if (c->device != b->device) return b->fail(LC_ERR_ARG, "lc_batch: contexts on different devices");
        if (c->params.n_gn != b->n_gn || c->params.n_pcg != b->n_pcg)
            return b->fail(LC_ERR_ARG, "lc_batch: contexts differ in n_gn / n_pcg");
    }
    return LC_OK;
}

extern "C" lc_status lc_batch_create(lc_batch** out, lc_ctx* const* ctxs, int count) {
    if (!out || !ctxs || count < 1) return LC_ERR_ARG;
    *out = nullptr;
    auto* b = new lc_batch();
    b->ctxs.assign(ctxs, ctxs + count);
    for (lc_ctx* c : b->ctxs)
        if (!c) {
            delete b;
            return LC_ERR_ARG;
        }
    b->device = ctxs[0]->device;
    b->n_gn = ctxs[0]->params.n_gn;
    b->n_pcg = ctxs[0]->params.n_pcg;
    lc_status s;
    if ((s = batch_check(b))) {
        // keep the message reachable through the first context
        ctxs[0]->fail(s, "%s", b->err.c_str());
        delete b;
        return s;
    }
    cudaSetDevice(b->device);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return LC_ERR_CUDA;
    }
    // the members' own work must be finished before the batch uses their buffers
    for (lc_ctx* c : b->ctxs) cudaStreamSynchronize(c->stream);
    b->ev.resize(count);
    for (auto& e : b->ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if ((s = b->build())) {
        ctxs[0]->fail(s, "%s", b->err.c_str());
        lc_batch_destroy(b);
        return s;
    }
    *out = b;
    return LC_OK;
}

extern "C" lc_status lc_batch_destroy(lc_batch* b) {
    if (!b) return LC_ERR_ARG;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    b->free_plan();
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->done) cudaEventDestroy(b->done);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return LC_OK;
}

extern "C" const char* lc_batch_last_error(const lc_batch* b) { return b ? b->err.c_str() : "null batch"; }

extern "C" lc_status lc_batch_set_pcg_mode(lc_batch* b, int mode) {
    if (!b) return LC_ERR_ARG;
    if (mode < LC_BATCH_PCG_AUTO || mode > LC_BATCH_PCG_PER_ITERATION)
        return b->fail(LC_ERR_ARG, "lc_batch_set_pcg_mode: unknown mode");
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    b->mode = mode;
    return b->build();
}

extern "C" lc_status lc_batch_solve(lc_batch* b, int from_identity, lc_solve_stats* stats) {
    if (!b) return LC_ERR_ARG;
    cudaSetDevice(b->device);
    lc_status s;
    if ((s = batch_check(b))) return s;
    // a member whose buffers or sizes changed since the plan was built
    bool changed = false;
    for (size_t j = 0; j < b->snap.size(); ++j)
        if (memcmp(&b->snap[j], &b->ctxs[b->ctx_of[j]]->hC, sizeof(CapDesc)) != 0) changed = true;
    if (changed && (s = b->build())) return s;
    if (b->gexec && b->gexec_identity != (from_identity != 0)) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    if (!b->gexec) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return b->fail(LC_ERR_CUDA, "lc_batch_solve: begin capture");
        b->enqueue(from_identity != 0);
        if (cudaStreamEndCapture(b->stream, &g) != cudaSuccess || !g) {
            cudaGetLastError();
            return b->fail(LC_ERR_CUDA, "lc_batch_solve: capture failed");
        }
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(g, nodes.data(), &nn);
        int k = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            cudaGraphNodeGetType(nd, &ty);
            if (ty == cudaGraphNodeTypeKernel) ++k;
        }
        b->graph_kernels = k;
        const cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->gexec = nullptr;
            return b->fail(LC_ERR_CUDA, "lc_batch_solve: graph instantiation");
        }
        b->gexec_identity = from_identity != 0;
    }
    // order with the members' own streams: the solve waits for their pending
    // work (uploads, parameter changes), and their later calls wait for it
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        cudaEventRecord(b->ev[i], b->ctxs[i]->stream);
        cudaStreamWaitEvent(b->stream, b->ev[i], 0);
    }
    if (cudaGraphLaunch(b->gexec, b->stream) != cudaSuccess) {
        cudaGetLastError();
        return b->fail(LC_ERR_CUDA, "lc_batch_solve: graph launch");
    }
    cudaEventRecord(b->done, b->stream);
    for (lc_ctx* c : b->ctxs) cudaStreamWaitEvent(c->stream, b->done, 0);
    b->solved = true;
    if (!stats) return LC_OK;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return b->fail(LC_ERR_CUDA, "lc_batch_solve: execution failed");
    }
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        lc_ctx* c = b->ctxs[i];
        if ((s = c->read_stats(&stats[i], b->n_gn))) return b->fail(s, "lc_batch_solve: reading statistics");
        stats[i].n_kernels = b->graph_kernels;
        int cl = 0;
        const int slot = b->slot_of[i];
        for (const BatchGroup& g : b->groups)
            if (slot >= g.first && slot < g.first + g.count) cl = g.plan.cl;
        stats[i].pcg_cluster_size = cl;
    }
    return LC_OK;
}

// One frame step of every member as one CUDA graph: per member the pose
// stage (from its Euler start or its last solved pose), the identity start of
// the non-rigid stage unless the graph parameters are carried, the warm
// start (with a network), then the batched non-rigid stage of all members,
// then per member the motion record and the end of the pose frame.  Captured
// on the first call (and again when the plan or the network changes) by
// routing every member's enqueue sequence into the batch's stream.
extern "C" lc_status lc_batch_step(lc_batch* b, lc_mlp* net, unsigned flags, lc_solve_stats* stats) {
    if (!b) return LC_ERR_ARG;
    if (flags & ~(LC_STEP_EULER_START | LC_STEP_CARRY_GRAPH)) return b->fail(LC_ERR_ARG, "lc_batch_step: unknown flags");
    cudaSetDevice(b->device);
    lc_status s;
    if ((s = batch_check(b))) return s;
    bool changed = false;
    for (size_t j = 0; j < b->snap.size(); ++j)
        if (memcmp(&b->snap[j], &b->ctxs[b->ctx_of[j]]->hC, sizeof(CapDesc)) != 0) changed = true;
    if (changed && (s = b->build())) return s;
    for (lc_ctx* c : b->ctxs) {
        if (c->profiling) return b->fail(LC_ERR_STATE, "lc_batch_step: profiling is on for a member");
        if ((s = pose_step_prepare(c))) return b->fail(s, c->err.c_str());
        if ((s = warm_step_prepare(c, net))) return b->fail(s, c->err.c_str());
    }
    unsigned long long uid = 0, gen = 0;
    mlp_identity(net, &uid, &gen);
    if (b->step_gexec && (b->step_uid != uid || b->step_gen != gen || b->step_flags != flags)) {
        cudaGraphExecDestroy(b->step_gexec);
        b->step_gexec = nullptr;
    }
    if (!b->step_gexec) {
        // every member's stream is the batch's while its sequences are captured
        std::vector<cudaStream_t> saved(b->ctxs.size());
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return b->fail(LC_ERR_CUDA, "lc_batch_step: begin capture");
        for (size_t i = 0; i < b->ctxs.size(); ++i) {
            lc_ctx* c = b->ctxs[i];
            saved[i] = c->stream;
            c->stream = b->stream;
            pose_step_begin(c, (flags & LC_STEP_EULER_START) != 0);
            if (!(flags & LC_STEP_CARRY_GRAPH)) {
                // the non-rigid stage starts from the identity over the new skinned
                // surface; the motion record then measures the frame's update from it
                launch_identity_params(c->hC.node_R, c->hC.node_t, c->hC.n, c->stream);
                motion_step_enqueue(c);
            }
            if (net) warm_step_enqueue(c, net);
        }
        b->enqueue(false);
        for (lc_ctx* c : b->ctxs) {
            motion_step_enqueue(c);
            pose_step_end(c);
        }
        for (size_t i = 0; i < b->ctxs.size(); ++i) b->ctxs[i]->stream = saved[i];
        if (cudaStreamEndCapture(b->stream, &g) != cudaSuccess || !g) {
            cudaGetLastError();
            return b->fail(LC_ERR_CUDA, "lc_batch_step: capture failed");
        }
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(g, nodes.data(), &nn);
        int k = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            cudaGraphNodeGetType(nd, &ty);
            if (ty == cudaGraphNodeTypeKernel) ++k;
        }
        const cudaError_t e = cudaGraphInstantiate(&b->step_gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->step_gexec = nullptr;
            return b->fail(LC_ERR_CUDA, "lc_batch_step: graph instantiation");
        }
        b->step_kernels = k;
        b->step_uid = uid;
        b->step_gen = gen;
        b->step_flags = flags;
    }
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        cudaEventRecord(b->ev[i], b->ctxs[i]->stream);
        cudaStreamWaitEvent(b->stream, b->ev[i], 0);
    }
    if (net) mlp_before(net, b->stream);
    if (cudaGraphLaunch(b->step_gexec, b->stream) != cudaSuccess) {
        cudaGetLastError();
        return b->fail(LC_ERR_CUDA, "lc_batch_step: graph launch");
    }
    if (net) mlp_after(net, b->stream);
    cudaEventRecord(b->done, b->stream);
    for (lc_ctx* c : b->ctxs) {
        cudaStreamWaitEvent(c->stream, b->done, 0);
        c->has_vis = true;
        c->has_lin = true;
        c->surf_has_lin = false;
        c->last_surface = false;
    }
    b->solved = true;
    if (!stats) return LC_OK;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return b->fail(LC_ERR_CUDA, "lc_batch_step: execution failed");
    }
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        if ((s = b->ctxs[i]->read_stats(&stats[i], b->n_gn))) return b->fail(s, "lc_batch_step: reading statistics");
        stats[i].n_kernels = b->step_kernels;
    }
    return LC_OK;
}

extern "C" lc_status lc_batch_autotune(lc_batch* b, int reps, int* mode_out, float* ms_out) {
    if (!b || reps < 1) return LC_ERR_ARG;
    cudaSetDevice(b->device);
    const int modes[4] = {LC_BATCH_PCG_AUTO, LC_BATCH_PCG_CLUSTER8, LC_BATCH_PCG_CLUSTER16,
                          LC_BATCH_PCG_PER_ITERATION};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = -1;
    float best_ms = 0.f;
    lc_status s = LC_OK;
    for (int m : modes) {
        if ((s = lc_batch_set_pcg_mode(b, m))) break;
        // warm up (capture + one run), then time reps solves from the identity
        if ((s = lc_batch_solve(b, 1, nullptr))) break;
        cudaEventRecord(e0, b->stream);
        for (int r = 0; r < reps; ++r)
            if ((s = lc_batch_solve(b, 1, nullptr))) break;
        if (s) break;
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms_out) ms_out[m] = ms;
        if (best < 0 || ms < best_ms) {
            best = m;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    if (mode_out) *mode_out = best;
    return lc_batch_set_pcg_mode(b, best);
}

extern "C" void* lc_batch_stream(const lc_batch* b) { return b ? (void*)b->stream : nullptr; }

extern "C" lc_status lc_batch_apply_jtj(lc_batch* b, int stage) {
    if (!b) return LC_ERR_ARG;
    if (!b->solved) return b->fail(LC_ERR_STATE, "lc_batch_apply_jtj: no batch solve yet");
    cudaSetDevice(b->device);
    if (stage) launch_jtj_stage(b->dC, b->all, b->stream);
    launch_jtj(b->dC, b->all, nullptr, nullptr, nullptr, nullptr, false, b->stream);
    if (cudaGetLastError() != cudaSuccess) return b->fail(LC_ERR_CUDA, "lc_batch_apply_jtj: launch");
    return LC_OK;
}

// ---------------------------------------------------------------------------
// Launch shapes of the per-iteration J^T J p and the shape autotuner with its
// per-size-class table (process-wide).
// ---------------------------------------------------------------------------
extern "C" lc_status lc_batch_set_shape(lc_batch* b, const lc_batch_shape* s) {
    if (!b || !s) return LC_ERR_ARG;
    if (s->pcg_mode < LC_BATCH_PCG_AUTO || s->pcg_mode > LC_BATCH_PCG_PER_ITERATION ||
        !jtj_shape_valid(s->vert_block, s->node_warps, s->node_unroll))
        return b->fail(LC_ERR_ARG, "lc_batch_set_shape: unknown mode or shape");
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    b->mode = s->pcg_mode;
    b->jv_block = s->vert_block;
    b->jn_warps = s->node_warps;
    b->jn_unroll = s->node_unroll;
    return b->build();
}

extern "C" lc_status lc_batch_get_shape(const lc_batch* b, lc_batch_shape* s) {
    if (!b || !s) return LC_ERR_ARG;
    s->pcg_mode = b->mode;
    s->vert_block = b->jv_block;
    s->node_warps = b->jn_warps;
    s->node_unroll = b->jn_unroll;
    return LC_OK;
}

// per member (K, ceil log2 of the vertices, ceil log2 of the nodes), sorted,
// with multiplicities: "K4.N12.n9x3,K8.N17.n12x1"
static std::string size_class(const lc_batch* b) {
    std::map<std::string, int> cnt;
    for (const lc_ctx* c : b->ctxs) {
        char k[64];
        snprintf(k, sizeof(k), "K%d.N%d.n%d", c->hC.K, (int)std::ceil(std::log2((double)std::max(c->hC.N, 1))),
                 (int)std::ceil(std::log2((double)std::max(c->hC.n, 1))));
        ++cnt[k];
    }
    std::string out;
    for (const auto& kv : cnt) {
        if (!out.empty()) out += ",";
        out += kv.first + "x" + std::to_string(kv.second);
    }
    return out;
}

extern "C" lc_status lc_batch_size_class(const lc_batch* b, char* key, int len) {
    if (!b || !key || len < 1) return LC_ERR_ARG;
    const std::string k = size_class(b);
    if ((int)k.size() + 1 > len) return LC_ERR_ARG;
    memcpy(key, k.c_str(), k.size() + 1);
    return LC_OK;
}

struct TuneEntry {
    lc_batch_shape shape;
    float ms;
};
static std::mutex g_tune_mu;
static std::map<std::string, TuneEntry> g_tune;

// every member's node parameters and per-step energy history, as bytes
static lc_status batch_snapshot(lc_batch* b, std::vector<unsigned char>& out) {
    out.clear();
    for (lc_ctx* c : b->ctxs) {
        const CapDesc& C = c->hC;
        const size_t off = out.size();
        const size_t nb = sizeof(float4) * 4 * (size_t)C.n + sizeof(double) * 2 * (LC_MAX_GN + 1);
        out.resize(off + nb);
        if (cudaMemcpy(out.data() + off, C.node_R, sizeof(float4) * 3 * (size_t)C.n, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(out.data() + off + sizeof(float4) * 3 * (size_t)C.n, C.node_t, sizeof(float4) * (size_t)C.n,
                       cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(out.data() + off + sizeof(float4) * 4 * (size_t)C.n, C.hist, sizeof(double) * 2 * (LC_MAX_GN + 1),
                       cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return b->fail(LC_ERR_CUDA, "lc_batch_autotune_shapes: reading results");
        }
    }
    return LC_OK;
}

extern "C" lc_status lc_batch_autotune_shapes(lc_batch* b, int reps, int use_cache, lc_batch_shape* best_out,
                                              float* best_ms, int* from_cache, int* n_tried, int* n_rejected) {
    if (!b || reps < 1) return LC_ERR_ARG;
    cudaSetDevice(b->device);
    const std::string key = size_class(b);
    if (from_cache) *from_cache = 0;
    if (n_tried) *n_tried = 0;
    if (n_rejected) *n_rejected = 0;
    if (use_cache) {
        TuneEntry e{};
        bool hit = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                e = it->second;
                hit = true;
            }
        }
        if (hit) {
            if (from_cache) *from_cache = 1;
            if (best_out) *best_out = e.shape;
            if (best_ms) *best_ms = e.ms;
            return lc_batch_set_shape(b, &e.shape);
        }
    }
    const int modes[4] = {LC_BATCH_PCG_AUTO, LC_BATCH_PCG_CLUSTER8, LC_BATCH_PCG_CLUSTER16,
                          LC_BATCH_PCG_PER_ITERATION};
    const int vbs[3] = {128, 256, 512}, nws[3] = {4, 8, 16}, nus[3] = {2, 4, 8};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    lc_status s = LC_OK;
    lc_batch_shape best{};
    float best_t = -1.f;
    int tried = 0, rejected = 0;
    std::vector<unsigned char> ref, cur;
    for (int m : modes) {
        lc_batch_shape sh{m, kVertTile, kJtjNodeWarps, 4};
        if ((s = lc_batch_set_shape(b, &sh))) break;
        // shapes matter only where captures run the per-iteration J^T J p
        const bool any_multi = b->first_multi < (int)b->ctxs.size();
        std::vector<lc_batch_shape> cands;
        if (!any_multi)
            cands.push_back(sh);
        else
            for (int vb : vbs)
                for (int nw : nws)
                    for (int nu : nus) cands.push_back(lc_batch_shape{m, vb, nw, nu});
        ref.clear();
        for (const lc_batch_shape& c : cands) {
            if ((s = lc_batch_set_shape(b, &c))) break;
            // capture and one run, then the bit-identity check against the
            // mode's first shape, then reps timed solves from the identity
            if ((s = lc_batch_solve(b, 1, nullptr))) break;
            cudaStreamSynchronize(b->stream);
            if ((s = batch_snapshot(b, ref.empty() ? ref : cur))) break;
            ++tried;
            if (&c != &cands[0] && cur != ref) {
                ++rejected;
                continue;
            }
            cudaEventRecord(e0, b->stream);
            for (int r = 0; r < reps && !s; ++r) s = lc_batch_solve(b, 1, nullptr);
            if (s) break;
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (best_t < 0.f || ms < best_t) {
                best_t = ms;
                best = c;
            }
        }
        if (s) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    if (n_tried) *n_tried = tried;
    if (n_rejected) *n_rejected = rejected;
    if (best_out) *best_out = best;
    if (best_ms) *best_ms = best_t;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = TuneEntry{best, best_t};
    }
    return lc_batch_set_shape(b, &best);
}

// the table as text: one line per size class, "key<TAB>mode vert_block
// node_warps node_unroll ms"
extern "C" lc_status lc_autotune_table(char* text, int len, int* needed) {
    std::string out;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const auto& kv : g_tune) {
            char line[96];
            const lc_batch_shape& s = kv.second.shape;
            snprintf(line, sizeof(line), "\t%d %d %d %d %.6g\n", s.pcg_mode, s.vert_block, s.node_warps,
                     s.node_unroll, (double)kv.second.ms);
            out += kv.first + line;
        }
    }
    if (needed) *needed = (int)out.size() + 1;
    if (!text) return LC_OK;
    if (len < (int)out.size() + 1) return LC_ERR_ARG;
    memcpy(text, out.c_str(), out.size() + 1);
    return LC_OK;
}

extern "C" lc_status lc_autotune_table_load(const char* text) {
    if (!text) return LC_ERR_ARG;
    std::map<std::string, TuneEntry> add;
    const char* p = text;
    while (*p) {
        const char* nl = strchr(p, '\n');
        const std::string line(p, nl ? (size_t)(nl - p) : strlen(p));
        p = nl ? nl + 1 : p + line.size();
        if (line.empty()) continue;
        const size_t tab = line.find('\t');
        if (tab == std::string::npos || tab == 0) return LC_ERR_ARG;
        TuneEntry e{};
        double ms = 0.0;
        if (sscanf(line.c_str() + tab + 1, "%d %d %d %d %lf", &e.shape.pcg_mode, &e.shape.vert_block,
                   &e.shape.node_warps, &e.shape.node_unroll, &ms) != 5)
            return LC_ERR_ARG;
        if (e.shape.pcg_mode < LC_BATCH_PCG_AUTO || e.shape.pcg_mode > LC_BATCH_PCG_PER_ITERATION ||
            !jtj_shape_valid(e.shape.vert_block, e.shape.node_warps, e.shape.node_unroll))
            return LC_ERR_ARG;
        e.ms = (float)ms;
        add[line.substr(0, tab)] = e;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& kv : add) g_tune[kv.first] = kv.second;
    return LC_OK;
}

#!/usr/bin/env python
"""Benchmark of the LiveCap Gauss-Newton hot path on GB300.

Metric: GN-solve frames/s (higher is better) on the full-body workload
(articulated capsule body, 6,020 vertices / 12,000 triangles, 23-joint 57-DOF
skeleton, 500 graph nodes, K = 4, 1024x1024 frame): every step is one frame
through both stages, the skeletal pose fit (5 Gauss-Newton steps on the dense
57x57 normal equations) and then the non-rigid fit from the skinned mesh
(10 Gauss-Newton x 40 PCG iterations).  Reported beside it: the dominant
kernel's achieved bandwidth against the measured HBM peak.  Inputs are seeded
synthetic frames (``synth``); the frame data already sits in device memory;
L2 is flushed (a 256 MiB write, outside the timed events) between timed
steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one independent capture per GPU (replicas, weak scaling, no
collective in the data path); launched by torch.distributed.run.
``--impl reference`` times the FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GN-solve frames/s at equal final energy; J^TJp HBM GB/s vs GB300 peak"
UNIT = "frames/s"
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["body", "tiny", "stress", "stream", "batch", "warmstart", "surface",
                                           "surface-stress"], default="body",
                    help="surface*: the per-vertex surface stage (the paper's own unknowns) in place of the "
                         "embedded graph, on the body / stress capture")
    ap.add_argument("--ws-train-frames", type=int, default=20000, help="warm start: training frames")
    ap.add_argument("--ws-seq-len", type=int, default=25,
                    help="warm start: frames kept per training sequence (each also tracks one frame first)")
    ap.add_argument("--ws-eval-seqs", type=int, default=2, help="warm start: held-out sequences")
    ap.add_argument("--ws-eval-frames", type=int, default=300, help="warm start: frames per held-out sequence")
    ap.add_argument("--ws-adam-steps", type=int, default=20000, help="warm start: Adam steps")
    ap.add_argument("--ws-train-counts", default="",
                    help="warm start: GN x PCG counts of the solves that give the targets, e.g. 3x4 "
                         "(default: the capture's own counts)")
    ap.add_argument("--ws-gn-block", type=int, default=2,
                    help="warm start: Gauss-Newton steps per conditional graph block, both arms")
    ap.add_argument("--streams", type=int, default=8, help="stream: tracked sequences solved together")
    ap.add_argument("--stream-frames", type=int, default=40, help="stream: frames per sequence")
    ap.add_argument("--stream-scene", choices=["stress", "body"], default="stress", help="stream: the capture")
    ap.add_argument("--stream-train-seqs", type=int, default=4, help="stream: warm-start training sequences")
    ap.add_argument("--stream-train-len", type=int, default=8, help="stream: frames per training sequence")
    ap.add_argument("--stream-train-counts", default="3x4",
                    help="stream: GN x PCG counts of the solves that give the warm start's targets (default 3x4, "
                         "the paper's counts for the stage: a stable function of the data; '' = the streams' own)")
    ap.add_argument("--no-warm-start", action="store_true", help="stream: without the learned warm start")
    ap.add_argument("--euler-start", action="store_true",
                    help="stream: the pose stage starts from the explicit Euler step (default: the last solved pose)")
    ap.add_argument("--carry-graph", action="store_true",
                    help="stream: the non-rigid stage starts from the previous frame's node parameters, carried with "
                         "the bones (default: the identity over the new skinned surface)")
    ap.add_argument("--batch-count", type=int, default=64, help="captures of the batch workload")
    ap.add_argument("--pcg-mode", type=int, default=-1, help="batch PCG strategy (-1: autotune)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU baseline sample length")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--frames", type=int, default=8, help="body / tiny: captures the timed steps cycle through")
    ap.add_argument("--gn-cap", type=int, default=30,
                    help="body / tiny: Gauss-Newton steps at most while a frame works toward the oracle's energy")
    ap.add_argument("--gn-block", type=int, default=10,
                    help="body / tiny: Gauss-Newton steps per conditional graph block (0: unrolled)")
    ap.add_argument("--no-tma-taps", action="store_true",
                    help="body / tiny: image taps by global loads instead of one TMA bulk-tensor copy per vertex")
    ap.add_argument("--profile-region", action="store_true",
                    help="start / stop the CUDA profiler around the timed steps (batch, stream: around the J^T J p timing) "
                         "for ncu --profile-from-start off")
    ap.add_argument("--no-body-parts", action="store_true",
                    help="body: solve without the body-part mask of the silhouette term")
    # options of the per-frame path (Sec. 3.2-3.4), off in the default line
    ap.add_argument("--pyramid", type=int, default=0, help="photometric pyramid levels (0: raw image)")
    ap.add_argument("--sigma-c", type=float, default=0.0, help="robust colour kernel threshold (0: off)")
    ap.add_argument("--body-parts", action="store_true", help="body-part mask of the silhouette term")
    ap.add_argument("--frame-prep", action="store_true",
                    help="every step first prepares the frame from device-resident RGB, mask and joints "
                         "(packing, distance transform of the silhouette on the device, pyramid levels)")
    return ap.parse_args()


def max_over_ranks(total_ms, dist, device=None):
    """The slowest rank's timed total; every rank receives it."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, total_ms):
    """Whole-job frames/s: each of the `world` replicas solves `steps` frames
    of its own capture; the job lasts as long as the slowest one."""
    return world * steps / (total_ms / 1e3)


def frame_prep_kernels(pyramid_levels):
    """Kernels of one on-device frame preparation: packing, the three passes
    of the distance transform (contour flags, columns, rows), then per
    pyramid level a box mean (factor > 1) and two blur passes."""
    return 4 + sum((1 if j < 2 else 0) + 2 for j in range(3 - pyramid_levels, 3))


def path_options(a):
    """The non-default options of the per-frame path, as config keys."""
    opt = {}
    if a.pyramid:
        opt["pyramid_levels"] = a.pyramid
    if a.sigma_c:
        opt["sigma_c"] = a.sigma_c
    if a.body_parts:
        opt["body_parts"] = "6 parts, 10 px dilation, torso precedence"
    if a.frame_prep:
        opt["frame_prep"] = "in the step: frame packing + device distance transform (+ pyramid levels)"
    return opt


def is_surface(workload):
    return workload.startswith("surface")


def scene_name(workload):
    """Capture of a workload: the surface workloads run on the body / stress
    captures."""
    return {"surface": "body", "surface-stress": "stress"}.get(workload, workload)


def stages_of(scene, surface=False):
    stage2 = "per-vertex surface stage" if surface else "non-rigid stage"
    if scene.skeleton is not None:
        return (f"pose stage ({len(scene.skeleton['parents'])} joints, {len(scene.pose_init)} DOF, "
                f"{scene.n_gn_pose} GN) + {stage2}")
    return stage2


def workload_config(scene, surface=False):
    if surface:
        wl = (f"surface ({scene.name} capture): {scene.N} vertices / {len(scene.F)} triangles, "
              f"{scene.cam.W}x{scene.cam.H} frame, {stages_of(scene, True)}, {scene.n_gn_surface} GN x "
              f"{scene.n_pcg_surface} PCG over the vertex positions, displacement warping and temporal terms")
        cfg = {"workload": wl, "vertices": int(scene.N), "triangles": int(len(scene.F)),
               "image": [int(scene.cam.W), int(scene.cam.H)], "gn_iters": int(scene.n_gn_surface),
               "pcg_iters": int(scene.n_pcg_surface), "surface_weights": list(scene.surface_weights)}
    else:
        cfg = {"workload": f"{scene.name}: {scene.N} vertices / {len(scene.F)} triangles, "
                           f"{scene.n_nodes} nodes K={scene.K}, {scene.cam.W}x{scene.cam.H} frame, "
                           f"{stages_of(scene)}, {scene.n_gn} GN x {scene.n_pcg} PCG",
               "vertices": int(scene.N), "triangles": int(len(scene.F)), "nodes": int(scene.n_nodes),
               "K": int(scene.K), "image": [int(scene.cam.W), int(scene.cam.H)],
               "gn_iters": int(scene.n_gn), "pcg_iters": int(scene.n_pcg)}
    cfg["l2"] = "flushed between timed steps (256 MiB write outside the timed events)"
    if scene.skeleton is not None:
        cfg.update(pose_dof=int(len(scene.pose_init)), pose_gn_iters=int(scene.n_gn_pose))
    return cfg


def oracle_frame(scene, g, surface=False):
    """One frame through the oracle: the pose stage from the scene's start
    pose, then the non-rigid stage on the skinned mesh (graph g built once on
    the template, its nodes following the skinned mesh), or the per-vertex
    surface stage from the skinned mesh."""
    import numpy as np
    from oracle import nonrigid as onr
    base = None
    if scene.skeleton is not None:
        from oracle import pose as op
        base = op.solve_scene(scene)["VS"].astype(np.float32)
    if surface:
        from oracle import surface as osf
        return osf.solve_scene(scene, base32=base)
    return onr.solve_scene(scene, graph=g, base32=base)


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
def _oracle_worker(args):
    workload, seed, seconds = args
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    sys.path.insert(0, ROOT)
    import synth
    from oracle import graph as ograph
    scene = synth.make_scene(scene_name(workload), seed=seed)
    surface = is_surface(workload)
    g = None if surface else ograph.build_graph(scene.V, scene.material, scene.n_nodes, scene.K)
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle_frame(scene, g, surface)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return n, time.perf_counter() - t0


def cpu_baseline(name, seconds):
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(name, 100 + c, seconds) for c in range(cores)])
    frames = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return {"value": frames / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{frames} frame solves ({stages_of(synth_scene(name), is_surface(name))}) of the {name} "
                      f"workload by the FP64 oracle, one single-threaded process per core for ~{seconds:.0f} s"}


def synth_scene(workload):
    import synth
    return synth.make_scene(scene_name(workload))


def run_reference_frames(a):
    """The oracle on the frames of ``run_frames``, one process: each step one
    frame (pose stage, body-part mask, non-rigid stage at its configured
    counts, which end at the energy the GPU path works toward)."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    import synth
    from oracle import graph as ograph
    name = scene_name(a.workload)
    body_parts = name == "body" and not a.no_body_parts
    scenes = [synth.make_scene(name, seed=s) for s in frame_seeds(a)]
    graphs = [ograph.build_graph(sc.V, sc.material, sc.n_nodes, sc.K) for sc in scenes]
    for k in range(a.warmup):
        oracle_frame_parts(scenes[k % len(scenes)], graphs[k % len(scenes)], body_parts)
    t0 = time.perf_counter()
    for k in range(a.steps):
        oracle_frame_parts(scenes[k % len(scenes)], graphs[k % len(scenes)], body_parts)
    dt = time.perf_counter() - t0
    v = a.steps / dt
    cfg = workload_config(scenes[0])
    cfg.update(frames=len(scenes), body_parts=body_parts)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * dt / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{a.steps} frame solves over {len(scenes)} captures, one single-threaded "
                                       f"process"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if a.workload in ("body", "tiny") and not path_options(a):
        return run_reference_frames(a)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    import synth
    from oracle import graph as ograph
    scene = synth.make_scene(scene_name(a.workload))
    surface = is_surface(a.workload)
    g = None if surface else ograph.build_graph(scene.V, scene.material, scene.n_nodes, scene.K)
    for _ in range(a.warmup):
        oracle_frame(scene, g, surface)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle_frame(scene, g, surface)
    dt = time.perf_counter() - t0
    v = a.steps / dt
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * dt / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": workload_config(scene, surface),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{a.steps} frame solves, one single-threaded process"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def jtj_algorithmic_bytes(scene, n_active, n_edges):
    """Minimal bytes one J^T J p must move: per active vertex its K node
    indices and weights, rest position and H_i (8K + 12 + 24 bytes); per node
    R, g and p read (72 B) and the result written (24 B); per directed edge
    two indices and a weight (12 B)."""
    return (8 * scene.K + 36) * n_active + 96 * scene.n_nodes + 12 * n_edges


def surface_jtj_algorithmic_bytes(N, n_adj):
    """Minimal bytes of one fused surface J^T J p (direction update included):
    per vertex z and the previous direction read, H_i read, the new direction
    and A p written (12 + 12 + 24 + 12 + 12 bytes); per ordered one-ring pair
    the neighbour index, the staged edge direction and smoothness weight
    (4 + 12 + 4 bytes)."""
    return 72 * N + 20 * n_adj


def surface_vector_bytes(N):
    """PCG vector traffic per iteration of the surface stage besides J^T J p:
    p, x, A p, r, M^-1 read and x, r, z written (12 B per vertex each)."""
    return 96 * N


def one_ring_pairs(F):
    """Ordered one-ring pairs of a triangle mesh (twice its unique edges)."""
    import numpy as np
    F = np.asarray(F, dtype=np.int64)
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    e.sort(axis=1)
    return 2 * len(np.unique(e, axis=0))


def pcg_vector_bytes(n):
    """PCG vector traffic per iteration if streamed: p read twice, Ap, x, r,
    z, M^-1 read, x, r, z, p written (24 B per node each)."""
    return 12 * 24 * n


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def run_ours(a):
    import numpy as np
    import torch

    import synth
    from paper_1810_02648_gb300 import Context
    from synth import setup_scene

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    cpu_base = None
    opts = path_options(a)
    if rank == 0 and world == 1 and not a.no_cpu_baseline and not opts:
        # spawn the oracle pool before the first GPU call
        cpu_base = cpu_baseline(a.workload, a.cpu_seconds)

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    surface = is_surface(a.workload)
    scene = synth.make_scene(scene_name(a.workload), seed=None if rank == 0 else 1000 + rank)
    stream = torch.cuda.Stream(device=dev)
    ctx = Context(local, stream=stream)
    setup_scene(ctx, scene)
    has_pose = scene.skeleton is not None
    if a.pyramid:
        ctx.set_params(pyr_levels=a.pyramid)
    if a.sigma_c:
        ctx.set_params(sigma_c=a.sigma_c)
    if a.body_parts:
        if not has_pose:
            raise SystemExit("--body-parts needs a capture with a skeleton")
        ctx.set_body_parts(scene.skeleton["bone_part"], scene.skeleton["torso_part"], 10)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    frame_dev = None
    if a.frame_prep:
        frame_dev = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in
                     (scene.rgb.astype(np.float32), scene.mask.astype(np.uint8))]
        if has_pose:
            frame_dev += [torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)
                          for x in (scene.joints2d, scene.joints3d)]
        else:
            frame_dev += [None, None]

    def step():
        # every frame starts from the same pose (device-side reset, no host
        # round trip); the graph stage from the identity deformation, the
        # surface stage from the skinned mesh plus the warped displacement of
        # the previous frame, which it then records with its history
        if frame_dev is not None:
            ctx.upload_frame(frame_dev[0], None, frame_dev[1], frame_dev[2], frame_dev[3])
        if has_pose:
            ctx.reset_pose()
            ctx.solve_pose(stats=False)
        if surface:
            ctx.surface_start()
            ctx.solve_surface(stats=False)
            ctx.surface_advance()
        else:
            ctx.set_node_params(None, None)
            ctx.solve_nonrigid(stats=False)

    for _ in range(a.warmup):
        step()
    pose_stats = None
    if has_pose:
        ctx.reset_pose()
        pose_stats = ctx.solve_pose(stats=True)
    if surface:
        ctx.surface_start()
        stats = ctx.solve_surface(stats=True)
        ctx.surface_advance()
    else:
        ctx.set_node_params(None, None)
        stats = ctx.solve_nonrigid(stats=True)
    torch.cuda.synchronize(dev)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(a.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                starts[k].record(stream)
            step()
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(ms)
    if dist:
        total_ms = max_over_ranks(total_ms, dist, dev)
    value = job_throughput(world, a.steps, total_ms)

    # per-phase device time (event chain in the captured solve), same workload
    ctx.set_profiling(True)
    n_prof = min(a.steps, 20)
    for _ in range(n_prof):
        with torch.cuda.stream(stream):
            flush.zero_()
        step()
    prof = ctx.read_profile()
    ctx.set_profiling(False)
    peak, peak_kind = measured_peaks()
    if surface:
        jtj_bytes = surface_jtj_algorithmic_bytes(scene.N, one_ring_pairs(scene.F))
    else:
        g = ctx.read_graph()
        E = len(g["edge_dst"])
        n_active = stats["n_visible"]
        jtj_bytes = jtj_algorithmic_bytes(scene, n_active, E)
    # dominant kernel: the cluster-persistent PCG when it is used, else the
    # per-iteration J^T J p pair (the fused J^T J p of the surface stage)
    if surface and prof["pcg"][1]:
        k_ms, k_n = prof["pcg"]
        k_bytes = scene.n_pcg_surface * (jtj_bytes + surface_vector_bytes(scene.N)) + 72 * scene.N
        k_name = ("surface_pcg_cluster_kernel (all PCG iterations of one GN step: fused direction update, "
                  "one-ring J^T J p, vector updates, cluster reductions)")
    elif surface:
        k_ms, k_n = prof["jtj"]
        k_bytes = jtj_bytes
        k_name = "surface_jtj_kernel (fused direction update + one-ring J^T J p + p.Ap)"
    elif prof["pcg"][1]:
        k_ms, k_n = prof["pcg"]
        k_bytes = scene.n_pcg * (jtj_bytes + pcg_vector_bytes(scene.n_nodes))
        k_name = "pcg_cluster_kernel (all PCG iterations of one GN step; J^T J p + vectors)"
    else:
        k_ms, k_n = prof["jtj"]
        k_bytes = jtj_bytes
        k_name = "jtj (matrix-free J^T J p: vertex + node phase)"
    achieved = k_bytes / (k_ms / k_n * 1e-3) / 1e9 if k_n else None

    # end to end through the C ABI: pinned host frame in, result out
    rgb = torch.from_numpy(np.ascontiguousarray(scene.rgb, dtype=np.float32)).pin_memory()
    dtm = torch.from_numpy(np.ascontiguousarray(scene.dt, dtype=np.float32)).pin_memory()
    msk = torch.from_numpy(scene.mask.astype(np.uint8)).pin_memory()
    j2 = j3 = outP = None
    if has_pose:
        j2 = torch.from_numpy(np.ascontiguousarray(scene.joints2d, dtype=np.float32)).pin_memory()
        j3 = torch.from_numpy(np.ascontiguousarray(scene.joints3d, dtype=np.float32)).pin_memory()
        outP = torch.empty(len(scene.pose_init), dtype=torch.float32).pin_memory()
    outR = torch.empty((scene.n_nodes, 9), dtype=torch.float32).pin_memory()
    outT = torch.empty((scene.n_nodes, 3), dtype=torch.float32).pin_memory()
    outV = torch.empty((scene.N, 3), dtype=torch.float32).pin_memory()
    lib = ctx._lib
    from paper_1810_02648_gb300.livecap import _ptr
    n_e2e = max(10, a.steps // 2)

    def e2e_step():
        ctx._check(lib.lc_upload_frame(ctx.h, _ptr(rgb), None if a.frame_prep else _ptr(dtm), _ptr(msk),
                                       _ptr(j2) if has_pose else None, _ptr(j3) if has_pose else None))
        if has_pose:
            ctx._check(lib.lc_reset_pose(ctx.h))
            ctx._check(lib.lc_solve_pose(ctx.h, None))
        if surface:
            ctx._check(lib.lc_surface_start(ctx.h))
            ctx._check(lib.lc_solve_surface(ctx.h, None))
            ctx._check(lib.lc_surface_advance(ctx.h))
            ctx._check(lib.lc_read_surface(ctx.h, _ptr(outV), None))
            if has_pose:
                ctx._check(lib.lc_read_back(ctx.h, None, None, None, None, _ptr(outP)))
            return
        ctx._check(lib.lc_set_node_params(ctx.h, None, None))
        ctx._check(lib.lc_solve_nonrigid(ctx.h, None))
        ctx._check(lib.lc_read_back(ctx.h, _ptr(outR), _ptr(outT), _ptr(outV), None,
                                    _ptr(outP) if has_pose else None))

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    h2d = (rgb.numel() * 4 + (0 if a.frame_prep else dtm.numel() * 4) + msk.numel()
           + ((j2.numel() + j3.numel()) * 4 if has_pose else 0))
    d2h = ((0 if surface else outR.numel() + outT.numel()) + outV.numel() + (outP.numel() if has_pose else 0)) * 4

    if rank != 0:
        ctx.close()
        if dist:
            dist.destroy_process_group()
        return
    phases = {k: {"ms_per_frame": v[0] / n_prof, "segments_per_frame": v[1] / n_prof}
              for k, v in prof.items() if v[1]}
    extra_kernels = (5 if has_pose else 3) if surface else 1
    if a.frame_prep:
        extra_kernels += frame_prep_kernels(a.pyramid)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**workload_config(scene, surface), **opts},
        "clocks": clk.summary(),
        "e2e": {"value": world * n_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        # per frame: the captured non-rigid solve, the identity reset kernel
        # (surface stage: start and advance, 2 + 3 kernels with a skeleton,
        # 1 + 2 without)
        # and, with a skeleton, the captured pose solve
        "gpu_launches": (int(stats["n_kernels"]) + extra_kernels
                         + (int(pose_stats["n_kernels"]) if has_pose else 0)) * a.steps,
        "roofline": {"kernel": k_name, "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None,
                     "peak_source": peak_kind, "traffic": None,
                     "algorithmic_bytes_per_launch": k_bytes,
                     "jtjp_algorithmic_bytes": jtj_bytes,
                     "avg_launch_us": 1e3 * k_ms / k_n if k_n else None,
                     "note": (f"the capture's working set ({jtj_bytes / 1e6:.2f} MB per J^T J p) stays in L2 across "
                              "the PCG iterations; a few CTAs (one per 256-1024 vertices) and dependent one-ring "
                              "gathers plus cluster reductions per iteration: latency-bound") if surface else
                             ("the capture's working set (~0.3 MB per J^T J p) stays on chip / in L2 across the "
                              "PCG iterations and the kernel is latency-bound (cluster barriers, FP64 reductions), "
                              "so the HBM fraction is low by construction") if prof["pcg"][1] else
                             ("per-iteration J^T J p (the capture does not fit a cluster): the operands stay in "
                              "L2 across the PCG iterations; latency-bound dependent gathers")},
        "phases": phases,
        "solve": {"e_total": stats["e_total"], "n_visible": stats["n_visible"],
                  "n_boundary": stats["n_boundary"], "kernels_per_frame": stats["n_kernels"]
                  + extra_kernels + (pose_stats["n_kernels"] if has_pose else 0),
                  "pose_e_total": pose_stats["e_total"] if has_pose else None},
        "cpu_baseline": cpu_base,
    }
    print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# graph-stage workloads: frames/s to the FP64 oracle's final energy
# ---------------------------------------------------------------------------
TARGET_TOL = 1e-4     # a frame counts once its energy is within 1e-4 of the oracle's final energy

# DRAM bytes (read + write) of one 40-iteration launch of the cluster PCG on
# the body capture, from one ncu capture of these kernel sources
# (profiles/pcg_cluster_body_full.md); reported only while the sources still
# hash to the captured version, else null.
PCG_TRAFFIC = {"sources": ("pcg_cluster.cu", "jtj_pair.cuh", "fpair.cuh"), "sha256_16": "16b429668c3b5c58",
               "bytes": 709632 + 0}


def _sources_hash(sources):
    import hashlib
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_1810_02648_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def pcg_traffic():
    return PCG_TRAFFIC["bytes"] if _sources_hash(PCG_TRAFFIC["sources"]) == PCG_TRAFFIC["sha256_16"] else None


# DRAM bytes (read + write) of the batch workload's J^T J p launch pair
# (jtj_vertex_kernel + jtj_node_kernel over the 64 captures), from one ncu
# capture of these kernel sources with ncu's cache flush before each kernel
# (profiles/jtj_batched_batch_streams.md); reported only while the sources
# still hash to the captured version, else null.
BATCH_JTJ_TRAFFIC = {"sources": ("solver_kernels.cu", "jtj_pair.cuh", "fpair.cuh", "lc_internal.cuh"),
                     "sha256_16": "bc1a4118eb5951f9", "bytes": 26465536 + 18432 + 36380160 + 232704}


def batch_jtj_traffic():
    return (BATCH_JTJ_TRAFFIC["bytes"]
            if _sources_hash(BATCH_JTJ_TRAFFIC["sources"]) == BATCH_JTJ_TRAFFIC["sha256_16"] else None)


def frame_seeds(a, rank=0):
    """Seeds of the benchmark's frames: the workload's own capture first."""
    base = {"body": 1, "tiny": 0}[scene_name(a.workload)]
    return [base + 1000 * rank + f for f in range(a.frames)]


def oracle_frame_parts(scene, g, body_parts):
    """One frame through the oracle with the body-part mask of the
    silhouette term when asked (a capture with a skeleton): the pose stage
    from the frame's start pose, the mask of its skinned mesh, then the
    non-rigid stage."""
    import numpy as np
    from oracle import nonrigid as onr
    if scene.skeleton is None:
        return onr.solve_scene(scene, graph=g)
    from oracle import parts as oparts
    from oracle import pose as op
    base = op.solve_scene(scene)["VS"].astype(np.float32)
    pm = vp = None
    if body_parts:
        sk, cam = scene.skeleton, scene.cam
        vp = oparts.vertex_parts(sk["skin_idx"], sk["skin_w"], sk["bone_part"])
        pm = oparts.part_mask(base, scene.F, cam.f, cam.cx, cam.cy, cam.W, cam.H, vp, 10, sk["torso_part"])
    return onr.solve_scene(scene, graph=g, base32=base, part_mask=pm, vpart=vp)


def _frame_target_worker(args):
    """Spawned worker: build one frame, solve it with the oracle (timed,
    graph construction excluded) and return the frame and its final energy."""
    name, seed, body_parts = args
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    sys.path.insert(0, ROOT)
    import synth
    from oracle import graph as ograph
    scene = synth.make_scene(name, seed=seed)
    g = ograph.build_graph(scene.V, scene.material, scene.n_nodes, scene.K)
    t0 = time.perf_counter()
    r = oracle_frame_parts(scene, g, body_parts)
    secs = time.perf_counter() - t0
    return {"seed": seed, "scene": scene, "e_star": r["e1"]["total"],
            "hist": [h["energy"] for h in r["hist"]], "seconds": secs}


def oracle_targets(name, seeds, body_parts, procs):
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        return pool.map(_frame_target_worker, [(name, s, body_parts) for s in seeds])


def batched_jtj_roofline(ctxs, scenes, n_visible, dev, shape=None):
    """The per-iteration J^T J p of several captures batched into one launch
    pair (lc_batch_apply_jtj), L2 flushed before each of 20 timed calls:
    algorithmic bytes over CUDA-event time against the measured HBM peak.
    Runs one untimed batched solve first (its operands), which moves the
    captures' node parameters."""
    import torch
    from paper_1810_02648_gb300 import Batch
    b = Batch(ctxs)
    if shape is not None:
        b.set_shape(*shape)
    b.solve(False, stats=False)
    ext = torch.cuda.ExternalStream(b.stream_handle, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    b.apply_jtj(stage=True)
    reps = 20
    j0 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    j1 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    for r in range(reps):
        with torch.cuda.stream(ext):
            flush.zero_()
        j0[r].record(ext)
        b.apply_jtj()
        j1[r].record(ext)
    torch.cuda.synchronize(dev)
    ms = sum(x.elapsed_time(y) for x, y in zip(j0, j1)) / reps
    nbytes = sum(jtj_algorithmic_bytes(sc, nv, len(c.read_graph()["edge_dst"]))
                 for c, sc, nv in zip(ctxs, scenes, n_visible))
    peak, peak_kind = measured_peaks()
    achieved = nbytes / (ms * 1e-3) / 1e9
    shp = b.shape()
    b.close()
    return {"kernel": f"jtj_vertex_kernel + jtj_node_kernel over {len(ctxs)} captures in one launch pair "
                      f"(vertex block {shp['vert_block']}, node block {shp['node_warps']} warps of 4 nodes)",
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": peak_kind, "traffic": None, "algorithmic_bytes_per_launch": nbytes,
            "avg_launch_us": 1e3 * ms, "l2": "flushed before each timed call"}


def run_frames(a):
    import numpy as np
    import torch

    from paper_1810_02648_gb300 import Context
    from synth import setup_scene

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    name = scene_name(a.workload)
    body_parts = name == "body" and not a.no_body_parts
    cores = os.cpu_count() or 1
    # the frames and the oracle's final energies (the spawned pool runs before
    # the first GPU call); its timing is the CPU baseline
    seeds = frame_seeds(a, rank)
    frames = oracle_targets(name, seeds, body_parts, max(1, min(len(seeds), cores // world)))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    ctxs = []
    for fr in frames:
        sc = fr["scene"]
        c = Context(local, stream=stream)
        setup_scene(c, sc)
        if body_parts:
            c.set_body_parts(sc.skeleton["bone_part"], sc.skeleton["torso_part"], 10)
        fr["target"] = fr["e_star"] * (1.0 + TARGET_TOL)
        c.set_params(n_gn=a.gn_cap, target_energy=fr["target"], gn_block=a.gn_block, tma_taps=0 if a.no_tma_taps else 1)
        ctxs.append(c)
    scene = frames[0]["scene"]
    has_pose = scene.skeleton is not None
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(c, stats=False):
        # the frame starts from its start pose and the identity deformation
        # (device-side resets, no host round trip)
        if has_pose:
            c.reset_pose()
            c.solve_pose(stats=False)
        c.set_node_params(None, None)
        return c.solve_nonrigid(stats=stats)

    for k in range(max(a.warmup, len(ctxs))):
        step(ctxs[k % len(ctxs)])
    # per frame: steps used, energies (the captured solves are deterministic,
    # so these are the timed steps' results)
    per = []
    for fr, c in zip(frames, ctxs):
        st = step(c, stats=True)
        reached = st["e_total"] <= fr["target"]
        per.append({"seed": fr["seed"], "e_star": fr["e_star"], "e_final": st["e_total"],
                    "gn_steps": int(st["n_gn_done"]), "reached": bool(reached), "n_visible": int(st["n_visible"])})
    n_kernels, n_step = int(st["n_kernels"]), int(st["n_kernels_step"])
    pose_kernels = int(ctxs[0].solve_pose(stats=True)["n_kernels"]) if has_pose else 0
    # kernels a frame launches: the solve outside its conditional blocks, the
    # blocks it entered (the one holding the step that reached the target
    # included), the pose solve, the identity reset
    B = a.gn_block
    n_blocks = (a.gn_cap + B - 1) // B if B > 0 else 1
    for p in per:
        blocks = min(n_blocks, p["gn_steps"] // B + 1) if B > 0 and n_step else 1
        p["kernels"] = n_kernels + (blocks - 1) * n_step + pose_kernels + 1
    torch.cuda.synchronize(dev)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if a.profile_region:
        torch.cuda.profiler.start()
    with ClockSampler(local) as clk:
        for k in range(a.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                starts[k].record(stream)
            step(ctxs[k % len(ctxs)])
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
    if a.profile_region:
        torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    reached_steps = sum(per[k % len(per)]["reached"] for k in range(a.steps))
    if dist:
        total_ms = max_over_ranks(total_ms, dist, dev)
        t = torch.tensor([reached_steps], dtype=torch.float64, device=dev)
        dist.all_reduce(t)
        reached_steps = int(t.item())
    else:
        reached_steps *= world
    value = reached_steps / (total_ms * 1e-3)

    # the same frames with every capture in flight at once: one context and
    # stream per capture, each frame's solves enqueued round-robin (the
    # GPU's throughput when independent captures share it)
    concurrent = None
    if not a.profile_region:
        cstreams = [torch.cuda.Stream(device=dev) for _ in frames]
        cctxs = []
        for fr, cs in zip(frames, cstreams):
            sc = fr["scene"]
            c = Context(local, stream=cs)
            setup_scene(c, sc)
            if body_parts:
                c.set_body_parts(sc.skeleton["bone_part"], sc.skeleton["torso_part"], 10)
            c.set_params(n_gn=a.gn_cap, target_energy=fr["target"], gn_block=a.gn_block,
                         tma_taps=0 if a.no_tma_taps else 1)
            cctxs.append(c)
        for c in cctxs:
            step(c)
        torch.cuda.synchronize(dev)
        rounds = max(1, a.steps // len(cctxs))
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
            c0.record(stream)
        for cs in cstreams:
            cs.wait_event(c0)
        for r in range(rounds):
            for c in cctxs:
                step(c)
        for cs in cstreams:
            ev = torch.cuda.Event()
            ev.record(cs)
            stream.wait_event(ev)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        c_ms = c0.elapsed_time(c1)
        c_reached = rounds * sum(p["reached"] for p in per)
        concurrent = {"value": c_reached / (c_ms * 1e-3), "unit": UNIT, "captures_in_flight": len(cctxs),
                      "rounds": rounds, "ms": c_ms,
                      "note": "the same frames, every capture on its own context and stream, all in flight at "
                              "once (a 16-CTA cluster PCG per capture); one L2 flush before the timed region"}
        for c in cctxs:
            c.close()

    # per-phase device time of one pass over the frames
    for c in ctxs:
        c.set_profiling(True)
    for k in range(len(ctxs)):
        with torch.cuda.stream(stream):
            flush.zero_()
        step(ctxs[k])
    prof = {}
    for c in ctxs:
        for key, (ms_, cnt) in c.read_profile().items():
            m0, c0 = prof.get(key, (0.0, 0))
            prof[key] = (m0 + ms_, c0 + cnt)
        c.set_profiling(False)
    gn_total = sum(p["gn_steps"] for p in per)
    peak, peak_kind = measured_peaks()
    g = ctxs[0].read_graph()
    jtj_bytes = jtj_algorithmic_bytes(scene, per[0]["n_visible"], len(g["edge_dst"]))
    if prof.get("pcg", (0, 0))[1]:
        k_ms = prof["pcg"][0]
        k_bytes = scene.n_pcg * (jtj_bytes + pcg_vector_bytes(scene.n_nodes))
        k_name = "pcg_cluster_kernel (all PCG iterations of one GN step; J^T J p + vectors, compensated FP32 pairs)"
    else:
        k_ms = prof.get("jtj", (0, 0))[0]
        k_bytes = scene.n_pcg * jtj_bytes
        k_name = "jtj (per-iteration matrix-free J^T J p: vertex + node phase)"
    # launches that did work: one per Gauss-Newton step taken (the steps after
    # the target return at once)
    avg_us = 1e3 * k_ms / gn_total if gn_total else None
    achieved = k_bytes / (avg_us * 1e-6) / 1e9 if avg_us else None

    # end to end through the C ABI: the frame in from pinned host memory, the
    # result out
    from paper_1810_02648_gb300.livecap import _ptr
    lib = ctxs[0]._lib
    host = []
    for fr in frames:
        sc = fr["scene"]
        pin = lambda x, dt=np.float32: torch.from_numpy(np.ascontiguousarray(x, dtype=dt)).pin_memory()  # noqa: E731
        h = {"rgb": pin(sc.rgb), "dt": pin(sc.dt), "mask": pin(sc.mask, np.uint8),
             "j2": pin(sc.joints2d) if has_pose else None, "j3": pin(sc.joints3d) if has_pose else None,
             "R": torch.empty((sc.n_nodes, 9), dtype=torch.float32).pin_memory(),
             "t": torch.empty((sc.n_nodes, 3), dtype=torch.float32).pin_memory(),
             "V": torch.empty((sc.N, 3), dtype=torch.float32).pin_memory(),
             "P": torch.empty(len(sc.pose_init), dtype=torch.float32).pin_memory() if has_pose else None}
        host.append(h)

    def e2e_step(k):
        c, h = ctxs[k % len(ctxs)], host[k % len(host)]
        c._check(lib.lc_upload_frame(c.h, _ptr(h["rgb"]), _ptr(h["dt"]), _ptr(h["mask"]),
                                     _ptr(h["j2"]) if has_pose else None, _ptr(h["j3"]) if has_pose else None))
        if has_pose:
            c._check(lib.lc_reset_pose(c.h))
            c._check(lib.lc_solve_pose(c.h, None))
        c._check(lib.lc_set_node_params(c.h, None, None))
        c._check(lib.lc_solve_nonrigid(c.h, None))
        c._check(lib.lc_read_back(c.h, _ptr(h["R"]), _ptr(h["t"]), _ptr(h["V"]), None,
                                  _ptr(h["P"]) if has_pose else None))

    n_e2e = max(len(ctxs), a.steps // 2)
    for k in range(len(ctxs)):
        e2e_step(k)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(n_e2e):
        e2e_step(k)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    e2e_reached = sum(per[k % len(per)]["reached"] for k in range(n_e2e))
    h0 = host[0]
    h2d = (h0["rgb"].numel() * 4 + h0["dt"].numel() * 4 + h0["mask"].numel()
           + ((h0["j2"].numel() + h0["j3"].numel()) * 4 if has_pose else 0))
    d2h = (h0["R"].numel() + h0["t"].numel() + h0["V"].numel() + (h0["P"].numel() if has_pose else 0)) * 4

    # the same captures' J^T J p batched into one launch pair (the batched
    # product of the scope; untimed solve first, after the timed region)
    roof_batched = batched_jtj_roofline(ctxs, [fr["scene"] for fr in frames], [p["n_visible"] for p in per], dev)
    if rank != 0:
        for c in ctxs:
            c.close()
        if dist:
            dist.destroy_process_group()
        return
    mean_s = statistics.mean(fr["seconds"] for fr in frames)
    cpu_base = {"value": cores / mean_s, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": (f"{len(frames)} frame solves ({stages_of(scene)}{', body-part mask' if body_parts else ''})"
                           f" by the FP64 oracle, one single-threaded process per frame, {mean_s:.2f} s per frame; "
                           f"value = cores / mean frame time")}
    n_reached = sum(p["reached"] for p in per)
    phases = {k: {"ms_per_frame": v[0] / len(ctxs), "segments_per_frame": v[1] / len(ctxs)}
              for k, v in prof.items() if v[1]}
    cfg = workload_config(scene)
    cfg["workload"] = (f"{len(frames)} {name} captures (seeds {seeds[0]}..{seeds[-1]}): {cfg['workload']}; "
                       f"frames/s until the non-rigid energy reaches the FP64 oracle's final energy "
                       f"({scene.n_gn} GN x {scene.n_pcg} PCG) within {TARGET_TOL:g}, at most {a.gn_cap} GN steps"
                       + ("; body-part mask of the silhouette term" if body_parts else ""))
    cfg.update(frames=len(frames), gn_cap=a.gn_cap, gn_block=a.gn_block, target_tol=TARGET_TOL, body_parts=body_parts,
               tma_taps=not a.no_tma_taps)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": cfg,
        "clocks": clk.summary(),
        "e2e": {"value": world * e2e_reached / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        # per frame: the captured pose and non-rigid solves (the Gauss-Newton
        # steps after the first are conditional graph nodes: a frame launches
        # the steps it takes), the identity reset kernel
        "gpu_launches": sum(per[k % len(per)]["kernels"] for k in range(a.steps)),
        "roofline": {"kernel": k_name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "peak_source": peak_kind,
                     "traffic": pcg_traffic() if name == "body" and prof.get("pcg", (0, 0))[1] else None,
                     "algorithmic_bytes_per_launch": k_bytes, "jtjp_algorithmic_bytes": jtj_bytes,
                     "avg_launch_us": avg_us,
                     "note": "the capture's working set (~0.3 MB per J^T J p) stays on chip across the PCG "
                             "iterations; the kernel is bound by its per-iteration synchronisation and the "
                             "compensated-pair arithmetic, so the HBM fraction is low by construction"},
        "roofline_batched": roof_batched,
        "concurrent": concurrent,
        "phases": phases,
        "solve": {"frames_reached": n_reached, "frames": len(per),
                  "gn_steps_mean": statistics.mean(p["gn_steps"] for p in per),
                  "e_final": [p["e_final"] for p in per], "oracle_e_final": [p["e_star"] for p in per],
                  "rel_diff": [(p["e_final"] - p["e_star"]) / p["e_star"] for p in per],
                  "gn_steps": [p["gn_steps"] for p in per],
                  "kernels_per_frame": [p["kernels"] for p in per]},
        "cpu_baseline": cpu_base,
    }
    print(json.dumps(line))
    for c in ctxs:
        c.close()
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# batched captures (uneven sizes, one launch per phase)
# ---------------------------------------------------------------------------
def _batch_member(spec):
    sys.path.insert(0, ROOT)
    import synth
    return synth.make_batch_member(spec)


def _oracle_batch_worker(spec):
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    sys.path.insert(0, ROOT)
    import synth
    from oracle import graph as ograph
    from oracle import nonrigid as onr
    sc = synth.make_batch_member(spec)
    g = ograph.build_graph(sc.V, sc.material, sc.n_nodes, sc.K)
    t0 = time.perf_counter()
    onr.solve_scene(sc, graph=g)
    return time.perf_counter() - t0


def batch_cpu_baseline(specs):
    """The oracle's non-rigid solve of the batch's first captures, one
    single-threaded process per core (one capture each); frames/s = captures
    solved / the longest solve (they run at the same time)."""
    cores = min(os.cpu_count() or 1, len(specs))
    with mp.get_context("spawn").Pool(cores) as pool:
        secs = pool.map(_oracle_batch_worker, specs[:cores])
    return {"value": cores / max(secs), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the non-rigid solves of the batch's first {cores} captures by the FP64 oracle, one "
                      f"single-threaded process per core (scene generation and graph build not timed)"}


def run_batch(a):
    import numpy as np
    import torch

    import synth
    from paper_1810_02648_gb300 import Batch, Context
    from synth import setup_scene

    specs = synth.batch_specs(a.batch_count)
    cpu_base = None
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        scenes = pool.map(_batch_member, specs)
    if not a.no_cpu_baseline:
        cpu_base = batch_cpu_baseline(specs)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctxs = []
    for sc in scenes:
        c = Context(0)
        setup_scene(c, sc)
        ctxs.append(c)
    batch = Batch(ctxs)
    tune = None
    if a.pcg_mode < 0:
        tune = batch.autotune_shapes(reps=2, use_cache=False)
        mode = tune["shape"]["pcg_mode"]
    else:
        mode = a.pcg_mode
        batch.set_pcg_mode(mode)
    ext = torch.cuda.ExternalStream(batch.stream_handle, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(a.warmup):
        batch.solve(True, stats=False)
    stats = batch.solve(True, stats=True)
    torch.cuda.synchronize(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    with ClockSampler(0) as clk:
        for k in range(a.steps):
            with torch.cuda.stream(ext):
                flush.zero_()
            starts[k].record(ext)
            batch.solve(True, stats=False)
            ends[k].record(ext)
        torch.cuda.synchronize(dev)
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    count = len(ctxs)
    value = count * a.steps / (total_ms / 1e3)
    # the metric kernel alone over all captures, L2 flushed before each call
    reps = 20
    batch.apply_jtj(stage=True)      # operands of the final linearisation, untimed
    j0 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    j1 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    if a.profile_region:
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.start()
    for r in range(reps):
        with torch.cuda.stream(ext):
            flush.zero_()
        j0[r].record(ext)
        batch.apply_jtj()
        j1[r].record(ext)
    torch.cuda.synchronize(dev)
    if a.profile_region:
        torch.cuda.profiler.stop()
    jtj_ms = sum(s.elapsed_time(e) for s, e in zip(j0, j1)) / reps
    jtj_bytes = 0
    verts = 0
    for c, sc, st in zip(ctxs, scenes, stats):
        E = len(c.read_graph()["edge_dst"])
        jtj_bytes += jtj_algorithmic_bytes(sc, st["n_visible"], E)
        verts += sc.N
    peak, peak_kind = measured_peaks()
    achieved = jtj_bytes / (jtj_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch: {count} uneven captures ({verts} vertices in total, 2k-20k each, "
                               f"nodes = vertices/12, K=4, 256-1024 px images), non-rigid stage "
                               f"{scenes[0].n_gn} GN x {scenes[0].n_pcg} PCG, one launch per phase",
                   "captures": count, "vertices_total": int(verts),
                   "l2": "flushed between timed steps (256 MiB write outside the timed events)",
                   "pcg_mode": int(mode), "shape": batch.shape(), "size_class": batch.size_class(),
                   "autotune": tune},
        "clocks": clk.summary(),
        "gpu_launches": int(stats[0]["n_kernels"]) * a.steps,
        "roofline": {"kernel": "jtj_vertex_kernel + jtj_node_kernel over all captures (one J^T J p each)",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_kind, "traffic": batch_jtj_traffic(), "algorithmic_bytes_per_launch": jtj_bytes,
                     "avg_launch_us": 1e3 * jtj_ms, "l2": "flushed before each timed call"},
        "solve": {"e_total_sum": float(sum(s["e_total"] for s in stats)),
                  "cluster_sizes": sorted(set(int(s["pcg_cluster_size"]) for s in stats))},
        "cpu_baseline": cpu_base,
    }
    print(json.dumps(line))
    batch.close()
    for c in ctxs:
        c.close()


# ---------------------------------------------------------------------------
# learned warm start on tracked sequences of the body capture
# ---------------------------------------------------------------------------
_WS = {}


def _ws_init():
    """Pool initialiser: one body capture per worker process."""
    sys.path.insert(0, ROOT)
    import synth
    _WS["synth"] = synth
    _WS["sc"] = synth.make_scene("body")


def _ws_frame(args):
    """Frame i of the AR(1) sequence ``seed`` of the body capture, rendered."""
    seed, i = args
    synth, sc = _WS["synth"], _WS["sc"]
    V = synth.ar1_frame(sc.V, sc.n_nodes, 0.05, 0.01, seed, i)
    return synth.render_frame(V, sc.F, sc.albedo, sc.cam, seed=100000 + 1000 * seed + i)


def _ws_restart(ctx):
    ctx.set_node_params(None, None)
    ctx.record_motion()
    ctx.record_motion()          # motion zero: the previous state is the identity too


def run_warmstart(a):
    """Learned warm start on AR(1)-tracked sequences of the body capture:
    training frames rendered by a process pool (host cores) while the GPU
    tracks them with the plain method and records (features, update) rows;
    training on the device; held-out sequences evaluated with one
    target-energy stop for both arms (the plain method's own final energy)."""
    import numpy as np
    import torch

    import synth
    from paper_1810_02648_gb300 import Context
    from synth import setup_scene
    from paper_1810_02648_gb300 import warmstart as ws

    L = a.ws_seq_len
    n_seq = max(1, math.ceil(a.ws_train_frames / L))
    train_seeds = list(range(1, n_seq + 1))
    eval_seeds = [1000000 + k for k in range(a.ws_eval_seqs)]
    sc = synth.make_scene("body")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sp, sw = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    plain = Context(0, stream=sp)
    setup_scene(plain, sc)
    plain.set_params(gn_block=a.ws_gn_block)
    procs = os.cpu_count() or 1
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"              # one BLAS thread per worker
    t_start = time.perf_counter()
    with mp.get_context("spawn").Pool(procs, initializer=_ws_init) as pool:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        it = pool.imap(_ws_frame, [(s, i) for s in train_seeds for i in range(L + 1)], chunksize=2)
        ev_async = pool.map_async(_ws_frame, [(s, i) for s in eval_seeds for i in range(a.ws_eval_frames)],
                                  chunksize=2)
        Fs, Ts, Es = [], [], []
        if a.ws_train_counts:
            tg, tp = (int(x) for x in a.ws_train_counts.lower().split("x"))
            plain.set_params(n_gn=tg, n_pcg=tp)
        for s in train_seeds:
            _ws_restart(plain)
            F, T, E = ws.collect(plain, (next(it) for _ in range(L + 1)), skip=1)
            Fs.append(F)
            Ts.append(T)
            Es.append(E)
        if a.ws_train_counts:
            plain.set_params(n_gn=sc.n_gn, n_pcg=sc.n_pcg)
        torch.cuda.synchronize(dev)
        t_collect = time.perf_counter() - t_start
        F, T, kept = ws.keep_converged(torch.cat(Fs), torch.cat(Ts), np.concatenate(Es))
        del Fs, Ts
        t0 = time.perf_counter()
        net, losses = ws.train(F, T, steps=a.ws_adam_steps, batch=4096, lr=1e-3, seed=0,
                               log_every=max(1, a.ws_adam_steps // 10))
        torch.cuda.synchronize(dev)
        t_train = time.perf_counter() - t0
        rows = int(F.shape[0] * F.shape[1])
        del F, T
        frames = ev_async.get()
    t_all = time.perf_counter() - t_start
    warm = Context(0, stream=sw)
    setup_scene(warm, sc)
    warm.set_params(n_gn=2 * sc.n_gn, gn_block=a.ws_gn_block)
    res = []
    for k in range(len(eval_seeds)):
        seq = frames[k * a.ws_eval_frames:(k + 1) * a.ws_eval_frames]
        for c in (plain, warm):
            _ws_restart(c)
        plain.set_params(target_energy=0.0)
        ws.collect(plain, seq[:1], skip=1)          # the first frame, plain from the identity
        r0 = plain.read_back(V=False, flags=False)
        warm.set_node_params(r0["R"].reshape(-1, 9), r0["t"])
        warm.record_motion()
        res += ws.evaluate(plain, warm, net, seq[1:], (sp, sw))
    sm = ws.summary(res)
    line = {
        "metric": METRIC, "value": sm["warm_frames_per_s"], "unit": UNIT, "n_gpus": 1, "steps": len(res),
        "warmup": 0, "ms_per_step": 1e3 / sm["warm_frames_per_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 solver (compensated-pair PCG), bf16 network", "data": "synthetic",
        "config": {"workload": f"warm start: body capture ({sc.N} vertices, {sc.n_nodes} nodes, K={sc.K}, "
                               f"{sc.cam.W}x{sc.cam.H}), AR(1) sequences (rho 0.9, 0.05 rad / 1 cm), "
                               f"plain {sc.n_gn} GN x {sc.n_pcg} PCG from the previous frame vs warm start + "
                               f"up to {2 * sc.n_gn} GN, both stopping at the plain method's own final energy "
                               f"(1e-4), conditional blocks of {a.ws_gn_block} steps",
                   "train_frames": n_seq * L, "train_sequences": n_seq, "frames_per_sequence": L,
                   "train_rows": rows, "train_frames": int(len(kept)), "train_frames_kept": int(kept.sum()),
                   "target_counts": a.ws_train_counts or f"{sc.n_gn}x{sc.n_pcg}",
                   "adam_steps": a.ws_adam_steps, "adam_batch": 4096,
                   "eval_sequences": len(eval_seeds), "eval_frames_per_sequence": a.ws_eval_frames,
                   "l2": "inputs of one frame < L2; no flush (every frame uploads a new image)"},
        "warm_start": dict(sm, loss_first=losses[0][1], loss_last=losses[-1][1], collect_s=t_collect,
                           train_s=t_train, data_and_training_s=t_all, render_processes=procs),
    }
    print(json.dumps(line))
    net.close()
    plain.close()
    warm.close()


# ---------------------------------------------------------------------------
# tracked streams: both stages per frame, warm start, one graph per frame step
# ---------------------------------------------------------------------------
def _stream_init(name):
    """Pool initialiser: the capture (without its own target frame) per worker."""
    sys.path.insert(0, ROOT)
    import synth
    _WS["synth"] = synth
    _WS["sc"] = synth.make_scene(name, frame=False)


def _stream_frame(args):
    """Frame i of stream ``seed`` of the capture: (rgb, dt, mask, joints2d, joints3d)."""
    seed, i = args
    return _WS["synth"].stream_frame(_WS["sc"], seed, i)


def run_stream(a):
    """Tracked streams of one capture (default: the 100k-vertex, 4,000-node,
    K = 8, 2048^2 stress capture), all solved together.  Frames are rendered
    by a spawned pool (host cores) in step order while the GPU tracks them.
    Per stream the first two frames go through the per-call API (pose stage,
    non-rigid stage, motion and pose bookkeeping); from the third on, every
    frame step is one CUDA graph over all streams (lc_batch_step: pose
    stages, warm starts, the batched non-rigid stage, bookkeeping).  value =
    frames of all streams per second of device time of the step graphs; e2e
    adds the frames' upload from pinned host memory and the statistics'
    read-back."""
    import numpy as np
    import torch

    import synth
    import ctypes

    from paper_1810_02648_gb300 import Batch, Context
    from paper_1810_02648_gb300 import warmstart as ws
    from paper_1810_02648_gb300.livecap import lc_solve_stats
    from synth import setup_scene

    name, S, L = a.stream_scene, a.streams, a.stream_frames
    sc = synth.make_scene(name, frame=False)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    use_net = not a.no_warm_start
    train_seeds = [900 + k for k in range(a.stream_train_seqs)] if use_net else []
    seeds = [100 + k for k in range(S)]
    procs = os.cpu_count() or 1
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    t_start = time.perf_counter()
    pool = mp.get_context("spawn").Pool(procs, initializer=_stream_init, initargs=(name,))
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    tasks = [(s_, i) for s_ in train_seeds for i in range(a.stream_train_len)]
    tasks += [(seeds[j], i) for i in range(L) for j in range(S)]
    it = pool.imap(_stream_frame, tasks, chunksize=1)
    parts = not a.no_body_parts
    ctxs = []
    for j in range(S):
        c = Context(0)
        setup_scene(c, sc, with_frame=False)
        c.set_params(graph_warp=1 if a.carry_graph else 0)
        if parts:
            c.set_body_parts(sc.skeleton["bone_part"], sc.skeleton["torso_part"], 10)
        ctxs.append(c)
    net, losses, t_train = None, [], 0.0
    if use_net:
        t0 = time.perf_counter()
        Fs, Ts, Es = [], [], []
        if a.stream_train_counts:
            tg, tp = (int(x) for x in a.stream_train_counts.lower().split("x"))
            ctxs[0].set_params(n_gn=tg, n_pcg=tp)
        for s_ in train_seeds:
            ws.restart(ctxs[0], pose=True)
            F, T, E = ws.collect(ctxs[0], (next(it) for _ in range(a.stream_train_len)), skip=1, pose=True,
                                 euler=a.euler_start, from_identity=not a.carry_graph)
            Fs.append(F)
            Ts.append(T)
            Es.append(E)
        train_e = np.concatenate(Es)
        F, T, kept = ws.keep_converged(torch.cat(Fs), torch.cat(Ts), train_e)
        net, losses = ws.train(F, T, steps=2000, batch=4096, lr=1e-3, seed=0, log_every=500)
        rows = int(F.shape[0] * sc.n_nodes)
        del Fs, Ts, F, T
        if a.stream_train_counts:
            ctxs[0].set_params(n_gn=sc.n_gn, n_pcg=sc.n_pcg)
        torch.cuda.synchronize(dev)
        t_train = time.perf_counter() - t0
        ws.restart(ctxs[0], pose=True)
    # the first two frames per stream through the per-call API
    for i in range(2):
        for j in range(S):
            c = ctxs[j]
            ws._upload(c, next(it))
            if i > 0 and a.euler_start:
                c.pose_extrapolate()
            c.solve_pose(stats=False)
            if not a.carry_graph:
                c.set_node_params(None, None)
                c.record_motion()
            if i > 0 and net is not None:
                c.warm_start(net, sync=False)
            c.solve_nonrigid(stats=False)
            c.record_motion()
            c.pose_advance()
    torch.cuda.synchronize(dev)
    batch = Batch(ctxs)
    # launch shape of the batched product, tuned on the streams' current
    # frames (the tuner's solves start from the identity, as every frame
    # step's non-rigid stage does)
    tune = batch.autotune_shapes(reps=2, use_cache=False)
    ext = torch.cuda.ExternalStream(batch.stream_handle, device=dev)
    steps = L - 2
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e2e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e2e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    W, H = sc.cam.W, sc.cam.H
    pin = [dict(rgb=torch.empty((H, W, 3), dtype=torch.float32).pin_memory(),
                dt=torch.empty((H, W), dtype=torch.float32).pin_memory(),
                mask=torch.empty((H, W), dtype=torch.uint8).pin_memory(),
                j2=torch.empty((23, 2), dtype=torch.float32).pin_memory(),
                j3=torch.empty((23, 3), dtype=torch.float32).pin_memory()) for _ in range(S)]
    stats_all, e_totals = [], []

    clk = ClockSampler(0)
    clk.__enter__()
    wall = []
    for k in range(steps):
        frames = [next(it) for _ in range(S)]
        for j, fr in enumerate(frames):
            for key, arr in zip(("rgb", "dt", "mask", "j2", "j3"), fr):
                pin[j][key].numpy()[...] = arr
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for j in range(S):
            P = pin[j]
            ctxs[j].upload_frame(P["rgb"], P["dt"], P["mask"], P["j2"], P["j3"])
        torch.cuda.synchronize(dev)
        ev0[k].record(ext)
        batch.step(net, euler_start=a.euler_start, carry_graph=a.carry_graph, stats=False)
        ev1[k].record(ext)
        st = [c.read_stats() for c in ctxs]
        wall.append(time.perf_counter() - t0)
        e_totals.append([x["e_total"] for x in st])
    torch.cuda.synchronize(dev)
    clk.__exit__(None, None, None)
    pool.close()
    pool.join()
    total_ms = sum(x.elapsed_time(y) for x, y in zip(ev0, ev1))
    value = S * steps / (total_ms / 1e3)
    e2e_value = S * steps / sum(wall)
    # the batched J^T J p over all streams, L2 flushed before each call
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    reps = 20
    batch.apply_jtj(stage=True)
    j0 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    j1 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
    if a.profile_region:
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.start()
    for r in range(reps):
        with torch.cuda.stream(ext):
            flush.zero_()
        j0[r].record(ext)
        batch.apply_jtj()
        j1[r].record(ext)
    torch.cuda.synchronize(dev)
    if a.profile_region:
        torch.cuda.profiler.stop()
    jtj_ms = sum(x.elapsed_time(y) for x, y in zip(j0, j1)) / reps
    last = [c.read_stats() for c in ctxs]
    E = len(ctxs[0].read_graph()["edge_dst"])
    jtj_bytes = sum(jtj_algorithmic_bytes(sc, x["n_visible"], E) for x in last)
    peak, peak_kind = measured_peaks()
    achieved = jtj_bytes / (jtj_ms * 1e-3) / 1e9
    n_kernels = int(last[0]["n_kernels"])
    h2d = S * (W * H * (12 + 4 + 1) + 23 * 5 * 4)
    et = np.array(e_totals)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": 2,
        "ms_per_step": total_ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 solver (compensated-pair PCG)" + (", bf16 network" if use_net else ""), "data": "synthetic",
        "config": {"workload": f"streams: {S} tracked {L}-frame sequences of the {name} capture ({sc.N} vertices, "
                               f"{sc.n_nodes} nodes, K={sc.K}, {W}x{H}); smooth joint and root motion (sinusoids, "
                               f"0.3-1 Hz at 25 frames/s, amplitudes 0.1 rad per angle, 0.05 rad / 3 cm at the root), AR(1) "
                               f"control-point field (0.05 rad, 1 cm, rho 0.9); per frame the "
                               f"pose stage ({sc.n_gn_pose} GN from "
                               + ("the explicit Euler step), " if a.euler_start else "the last solved pose), ")
                               + ("the learned warm start, " if use_net else "")
                               + f"the non-rigid stage {sc.n_gn} GN x {sc.n_pcg} PCG from "
                               + ("the previous frame's node parameters carried with the bones" if a.carry_graph
                                  else "the identity over the new skinned surface") + "; "
                               f"frames 3..{L} of all streams: one CUDA graph per frame step",
                   "streams": S, "frames_per_stream": L, "timed_frame_steps": steps, "body_parts": parts,
                   "euler_start": a.euler_start, "carry_graph": a.carry_graph,
                   "warm_start": use_net, "warm_start_training_rows": rows if use_net else 0,
                   "warm_start_target_counts": a.stream_train_counts or f"{sc.n_gn}x{sc.n_pcg}",
                   "shape": tune["shape"], "autotune": {k: tune[k] for k in ("ms", "tried", "rejected")},
                   "l2": "each step uploads new frames (17 MB per 2048^2 frame); no flush"},
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(S * ctypes.sizeof(lc_solve_stats))},
        "gpu_launches": n_kernels * steps,
        "roofline": {"kernel": "jtj_vertex_kernel + jtj_node_kernel over all streams (one J^T J p each)",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_kind, "traffic": None, "algorithmic_bytes_per_launch": jtj_bytes,
                     "avg_launch_us": 1e3 * jtj_ms, "l2": "flushed before each timed call"},
        "solve": {"e_total_median": float(np.median(et)), "e_total_max": float(et.max()),
                  "e_total_last_step": [float(x) for x in et[-1]],
                  "network_loss": [float(losses[0][1]), float(losses[-1][1])] if losses else None,
                  "training_frames": int(len(train_e)) if use_net else 0,
                  "training_frames_kept": int(kept.sum()) if use_net else 0,
                  "training_e_final": [float(x) for x in train_e] if use_net else [],
                  "train_s": t_train, "wall_s": time.perf_counter() - t_start},
        "cpu_baseline": None,
    }
    print(json.dumps(line))
    if net is not None:
        net.close()
    batch.close()
    for c in ctxs:
        c.close()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch":
        run_batch(a)
    elif a.workload == "warmstart":
        run_warmstart(a)
    elif a.workload == "stream":
        run_stream(a)
    elif a.workload in ("body", "tiny") and not path_options(a):
        run_frames(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()

"""Visibility through the allocation-free entry point.

For callers that cannot allocate device memory (a host framework's pool that
forbids outside allocations, a process with its device memory reserved up
front): lc_visibility_noalloc must give the same per-vertex visibility as the
context path, bit for bit, using only caller-owned buffers and its static
scratch.  Two calls in a row with different inputs check that the scratch is
cleared between calls.  This file sorts last so a stop-at-first-failure run
has executed every other test before it.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_helpers import random_params

pytestmark = pytest.mark.gpu


def _context_visibility(ctx, n, seed):
    R, t = random_params(n, seed, rot=0.08, trans=0.01)
    ctx.set_node_params(R.reshape(n, 9), t)
    ctx.compute_visibility()
    flags = ctx.read_visibility()["flags"]
    v = ctx.eval_linearization()["v"]
    return v, (flags & 1).astype(np.uint8)


def test_visibility_noalloc_matches_context_path():
    import torch

    from paper_1810_02648_gb300 import Context, load
    from synth import setup_scene
    from paper_1810_02648_gb300.livecap import LC_OK, LC_ERR_ARG

    lib = load()
    scene = synth.make_scene("tiny")
    ctx = Context(0)
    setup_scene(ctx, scene)
    dev = torch.device("cuda", 0)
    F = torch.from_numpy(scene.F.astype(np.int32)).to(dev)
    out = torch.full((scene.N,), 7, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    cam = scene.cam
    seen = []
    for seed in (21, 22):
        v, ref = _context_visibility(ctx, scene.n_nodes, seed)
        V = torch.from_numpy(v).to(dev)
        st = lib.lc_visibility_noalloc(V.data_ptr(), scene.N, F.data_ptr(), len(scene.F),
                                       float(np.float32(cam.f)), float(np.float32(cam.cx)),
                                       float(np.float32(cam.cy)), cam.W, cam.H, ctypes.c_float(1e-2),
                                       out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert st == LC_OK
        torch.cuda.synchronize(dev)
        got = out.cpu().numpy()
        assert np.array_equal(got, ref)
        seen.append(ref)
    assert not np.array_equal(seen[0], seen[1])   # the two calls really differ
    # sizes beyond the static scratch are refused, and host pointers too
    st = lib.lc_visibility_noalloc(V.data_ptr(), scene.N, F.data_ptr(), len(scene.F), 150.0, 0.0, 0.0,
                                   2048, 2048, ctypes.c_float(1e-2), out.data_ptr(), None)
    assert st == LC_ERR_ARG
    host = np.zeros(scene.N, np.uint8)
    st = lib.lc_visibility_noalloc(V.data_ptr(), scene.N, F.data_ptr(), len(scene.F), 150.0, 63.5, 63.5,
                                   128, 128, ctypes.c_float(1e-2), host.ctypes.data, None)
    assert st == LC_ERR_ARG
    ctx.close()
    # a negative or NaN depth tolerance is refused like in the context path
    for eps in (-1e-2, float("nan")):
        st = lib.lc_visibility_noalloc(V.data_ptr(), scene.N, F.data_ptr(), len(scene.F), 150.0, 63.5, 63.5,
                                       128, 128, ctypes.c_float(eps), out.data_ptr(), None)
        assert st == LC_ERR_ARG

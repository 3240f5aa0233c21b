"""Pins for the exact-arithmetic visibility oracle (CPU).

* A brute-force per-pixel loop over all triangles, written with Python
  integers and numpy FP32 scalars, reproduces the z-buffer key by key.
* On a convex capsule, a vertex is visible iff it faces the camera, except
  next to the silhouette rim; the silhouette edges form one closed loop.
* Depths agree with the FP64 renderer to FP32 accuracy, coverage agrees
  except on boundary pixels.
"""
import numpy as np
import pytest

import synth
from oracle import visibility as vis

f32 = np.float32


def _brute_zbuf(V, F, f, cx, cy, W, H):
    V = V.astype(np.float32)
    S, ok = [], []
    for X, Y, Z in V:
        valid = Z > f32(1e-3)
        u = f32(f32(f32(f) * X) / Z) + f32(cx) if valid else f32(0)
        v = f32(f32(f32(f) * Y) / Z) + f32(cy) if valid else f32(0)
        S.append((int(np.rint(f32(u * f32(256)))), int(np.rint(f32(v * f32(256))))))
        ok.append(valid)
    Z = V[:, 2]
    out = np.full((H, W), np.iinfo(np.uint64).max, dtype=np.uint64)
    for py in range(H):
        for px in range(W):
            P = (px * 256, py * 256)
            best = None
            for t, (a, b, c) in enumerate(F):
                if not (ok[a] and ok[b] and ok[c]):
                    continue
                A, B, C = S[a], S[b], S[c]
                area = (B[0] - A[0]) * (C[1] - A[1]) - (B[1] - A[1]) * (C[0] - A[0])
                if area == 0:
                    continue
                sg = 1 if area > 0 else -1

                def E(p, q):
                    return sg * ((q[0] - p[0]) * (P[1] - p[1]) - (q[1] - p[1]) * (P[0] - p[0]))

                def owns(p, q):
                    ex, ey = sg * (q[0] - p[0]), sg * (q[1] - p[1])
                    return ey < 0 or (ey == 0 and ex > 0)
                ws = [(E(B, C), owns(B, C)), (E(C, A), owns(C, A)), (E(A, B), owns(A, B))]
                if any(w < 0 or (w == 0 and not o) for w, o in ws):
                    continue
                fa = f32(sg * area)
                bb = [f32(f32(w) / fa) for w, _ in ws]
                s01 = f32(f32(bb[0] / Z[a]) + f32(bb[1] / Z[b]))
                depth = f32(f32(1) / f32(s01 + f32(bb[2] / Z[c])))
                key = (int(np.array(depth, dtype=np.float32).view(np.uint32)) << 32) | t
                best = key if best is None else min(best, key)
            if best is not None:
                out[py, px] = best
    return out


def _small_capsule(rings=5, segs=7, z=2.0, rot=0.3):
    V, F = synth.capsule_mesh(0.3, 1.0, rings, segs)
    c, s = np.cos(rot), np.sin(rot)
    V = V @ np.array([[1, 0, 0], [0, c, -s], [0, s, c]]).T + [0.05, -0.02, z]
    return V.astype(np.float32), F.astype(np.int32)


@pytest.mark.parametrize("rot", [0.0, 0.4])
def test_zbuffer_matches_brute_force(rot):
    V, F = _small_capsule(rot=rot)
    W, H, f = 24, 28, 36.0
    cx, cy = (W - 1) / 2, (H - 1) / 2
    out = vis.visibility(V, F, f, cx, cy, W, H, np.zeros((H, W), np.float32),
                         np.zeros((H, W), np.uint8))
    ref = _brute_zbuf(V, F, f, cx, cy, W, H)
    assert np.array_equal(out["zbuf"], ref)
    assert (out["zbuf"] != np.iinfo(np.uint64).max).sum() > 50


def test_convex_capsule_visibility_and_loop():
    s = synth.make_scene("tiny")
    V = s.V
    cam = s.cam
    out = vis.visibility(V, s.F, cam.f, cam.cx, cam.cy, cam.W, cam.H, s.dt, s.mask)
    fl = out["flags"]
    visible = (fl & vis.FLAG_VISIBLE) != 0
    # facing test with FP64 area-weighted normals
    Vd = V.astype(np.float64)
    nrm = np.zeros_like(Vd)
    a, b, c = Vd[s.F[:, 0]], Vd[s.F[:, 1]], Vd[s.F[:, 2]]
    cr = np.cross(b - a, c - a)
    for k in range(3):
        np.add.at(nrm, s.F[:, k], cr)
    facing = np.einsum("ij,ij->i", nrm, -Vd) > 0
    # rim vertices: within 2.5 px of the template's own silhouette, where a
    # pixel (about 2 cm here) no longer separates front from back
    _, tmask = synth.render(Vd, s.F, np.ones((s.N, 3)), cam)
    tdt = synth.contour_distance_transform(tmask)
    px = np.clip(np.rint(out["uv"]).astype(int), 0, cam.W - 1)
    rim = tdt[px[:, 1], px[:, 0]] <= 2.5
    assert (~rim).sum() > 0.35 * s.N
    assert np.array_equal(visible[~rim], facing[~rim])
    # silhouette edges form exactly one closed loop
    E = vis.mesh_edges(s.F)
    uv = out["uv"].astype(np.float64)

    def front(t):
        p = np.rint(uv[s.F[t]] * 256)
        return ((p[1, 0] - p[0, 0]) * (p[2, 1] - p[0, 1]) - (p[1, 1] - p[0, 1]) * (p[2, 0] - p[0, 0])) > 0
    sil = [(v0, v1) for v0, v1, t0, t1 in E if front(t0) != front(t1)]
    deg = {}
    for v0, v1 in sil:
        deg[v0] = deg.get(v0, 0) + 1
        deg[v1] = deg.get(v1, 0) + 1
    assert all(d == 2 for d in deg.values())
    adj = {}
    for v0, v1 in sil:
        adj.setdefault(v0, []).append(v1)
        adj.setdefault(v1, []).append(v0)
    start = next(iter(adj))
    seen, stack = {start}, [start]
    while stack:
        for w in adj[stack.pop()]:
            if w not in seen:
                seen.add(w)
                stack.append(w)
    assert len(seen) == len(adj)
    onsil = (fl & vis.FLAG_ONSIL) != 0
    assert set(np.nonzero(onsil)[0].tolist()) == set(adj)
    inB = (fl & vis.FLAG_INB) != 0
    assert np.array_equal(inB, onsil & visible)


def test_depth_and_coverage_match_fp64_renderer():
    s = synth.make_scene("tiny")
    cam = s.cam
    out = vis.visibility(s.V, s.F, cam.f, cam.cx, cam.cy, cam.W, cam.H, s.dt, s.mask)
    z = out["zbuf"]
    cov = z != np.iinfo(np.uint64).max
    depth = (z >> np.uint64(32)).astype(np.uint32).view(np.float32).astype(np.float64)
    rgb, mask = synth.render(s.V.astype(np.float64), s.F, np.ones((s.N, 3)), cam)
    both = cov & mask
    assert np.abs(cov.astype(int) - mask.astype(int)).sum() <= 0.05 * mask.sum()
    # depth at a covered pixel: FP64 perspective-correct interpolation over
    # the triangle with its corners snapped to 1/256 px
    tri = (z[both] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    yy, xx = np.nonzero(both)
    Vd = s.V.astype(np.float64)
    u = np.rint(out["uv"][:, 0].astype(np.float64) * 256) / 256
    v = np.rint(out["uv"][:, 1].astype(np.float64) * 256) / 256
    A, B, C = s.F[tri, 0], s.F[tri, 1], s.F[tri, 2]
    area = (u[B] - u[A]) * (v[C] - v[A]) - (v[B] - v[A]) * (u[C] - u[A])
    wa = ((u[C] - u[B]) * (yy - v[B]) - (v[C] - v[B]) * (xx - u[B])) / area
    wb = ((u[A] - u[C]) * (yy - v[C]) - (v[A] - v[C]) * (xx - u[C])) / area
    wc = 1.0 - wa - wb
    zref = 1.0 / (wa / Vd[A, 2] + wb / Vd[B, 2] + wc / Vd[C, 2])
    assert np.abs(depth[both] - zref).max() < 1e-5 * zref.max()

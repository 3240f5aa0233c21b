"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle)."""
import json
import os

import numpy as np

from oracle import nonrigid as onr
from oracle import parts as oparts
from oracle import visibility as ovis

REPORT = {}


def report(key, **vals):
    """Record observed error figures; written to $LC_REPORT_DIR if set."""
    REPORT[key] = {k: float(v) if np.isscalar(v) else v for k, v in vals.items()}
    d = os.environ.get("LC_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "parity_report.json"), "w") as f:
            json.dump(REPORT, f, indent=1, sort_keys=True)


def csr_edges(g):
    off, dst = g["edge_off"], g["edge_dst"]
    src = np.repeat(np.arange(len(off) - 1), np.diff(off))
    return np.stack([src, dst], 1).astype(np.int64)


def graph_from_gpu(g):
    return dict(node_vid=g["node_vid"].astype(np.int64), bind_idx=g["bind_idx"].astype(np.int64),
                bind_w=g["bind_w"], edges=csr_edges(g), edge_s=g["edge_s"])


def oracle_problem(scene, g, flags=None, base32=None):
    P = onr.problem_from_scene(scene, graph_from_gpu(g), base32)
    if flags is not None:
        set_flags(P, flags)
    return P


def set_flags(P, flags):
    P.vis = (flags & ovis.FLAG_VISIBLE) != 0
    P.inB = (flags & ovis.FLAG_INB) != 0
    P.bsign = np.where((flags & ovis.FLAG_BNEG) != 0, -1.0, 1.0)


def check_frame_flags(flags, P):
    """Final flags of a GPU solve against the oracle's problem: visibility and
    the contour set (decided once per frame on identical vertices) bit-exact;
    b_i, re-decided at every linearisation on each side's own iterate, may
    differ where m . grad DT is within rounding of zero on the two iterates:
    at most max(2, 1% of |B|) vertices.  Returns the mismatch count."""
    assert np.array_equal((flags & ovis.FLAG_VISIBLE) != 0, P.vis)
    assert np.array_equal((flags & ovis.FLAG_INB) != 0, P.inB)
    neg = (flags & ovis.FLAG_BNEG) != 0
    nb = int(((neg != (P.bsign < 0)) & P.inB).sum())
    assert nb <= max(2, P.inB.sum() // 100)
    return nb


def random_params(n, seed, rot=0.05, trans=0.005):
    rng = np.random.default_rng(seed)
    R = onr.so3_exp(rng.normal(scale=rot, size=(n, 3))).astype(np.float32)
    t = rng.normal(scale=trans, size=(n, 3)).astype(np.float32)
    return R, t


def vec6(x):
    return np.asarray(x, dtype=np.float64).reshape(-1)


def oracle_vertex_blocks(P, v32, uv32, pruned=None):
    """Residuals and A_i^T A_i, A_i^T r_i at given FP32 warped positions and
    projections (the inputs of the GPU's residual kernel), in FP64; ``pruned``
    marks photometric correspondences dropped by the robust colour kernel."""
    v = v32.astype(np.float64)
    u, w = uv32[:, 0].astype(np.float64), uv32[:, 1].astype(np.float64)
    ok = (v[:, 2] > 1e-3) & (u >= 0) & (u <= P.W - 1) & (w >= 0) & (w <= P.H - 1)
    ph = ok & P.vis
    if pruned is not None:
        ph = ph & ~pruned
    si = ok & P.inB & ~oparts.masked(P, v32)
    gxD, gyD = P.grads()[1]
    Dp = onr.dproj(P, v)
    N = len(v)
    r_photo = np.zeros((N, 3))
    r_sil = np.zeros(N)
    H = np.zeros((N, 3, 3))
    e = np.zeros((N, 3))
    ip = np.nonzero(ph)[0]
    if len(ip):
        I, G = onr.photo_sample(P, u[ip], w[ip], grad=True)      # raw image or pyramid level P.level
        r_photo[ip] = np.sqrt(P.w_photo) * (I - P.albedo[ip])
        A = np.sqrt(P.w_photo) * (G @ Dp[ip])
        H[ip] += np.einsum("nri,nrj->nij", A, A)
        e[ip] += np.einsum("nri,nr->ni", A, r_photo[ip])
    isl = np.nonzero(si)[0]
    if len(isl):
        r_sil[isl] = np.sqrt(P.w_sil) * onr.bilinear(P.dt, u[isl], w[isl])
        G = np.stack([onr.bilinear(gxD, u[isl], w[isl]), onr.bilinear(gyD, u[isl], w[isl])], 1)[:, None, :]
        A = (np.sqrt(P.w_sil) * P.bsign[isl])[:, None, None] * (G @ Dp[isl])
        H[isl] += np.einsum("nri,nrj->nij", A, A)
        e[isl] += A[:, 0, :] * r_sil[isl, None]
    H6 = np.stack([H[:, 0, 0], H[:, 0, 1], H[:, 0, 2], H[:, 1, 1], H[:, 1, 2], H[:, 2, 2]], 1)
    return dict(r_photo=r_photo, r_sil=r_sil, H=H6, e=e, photo_on=ph, sil_on=si)


def _r32(rng):
    """FP32 rounding with a random tie-break perturbation of one unit roundoff."""
    u = 2.0 ** -24

    def r32(x):
        x = np.asarray(x, dtype=np.float64)
        return (x * (1.0 + u * rng.standard_normal(x.shape))).astype(np.float32).astype(np.float64)
    return r32


def pcg32(A, b, n, r32):
    """The oracle's Jacobi-PCG with every vector and matrix-vector product
    rounded by ``r32`` (one FP32 execution of the same algorithm)."""
    d = np.asarray(A.diagonal(), dtype=np.float64)
    minv = r32(np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0))
    x = np.zeros_like(b)
    r = r32(b)
    z = r32(minv * r)
    p = z.copy()
    rz = float(r @ z)
    info = dict(iters=0, breakdown=False, rz=[rz])
    if rz == 0.0:
        return x, info
    for it in range(n):
        Ap = r32(A @ p)
        pAp = float(p @ Ap)
        if not pAp > 0.0:
            info["breakdown"] = True
            break
        al = np.float32(rz / pAp)
        x = r32(x + al * p)
        r = r32(r - al * Ap)
        z = r32(minv * r)
        rzn = float(r @ z)
        info["iters"] = it + 1
        if rzn == 0.0:
            break
        p = r32(z + np.float32(rzn / rz) * p)
        rz = rzn
    return x, info


def _project32(project, r32):
    """The projection with its pixel coordinates rounded like an FP32
    execution's (the sampling position of every data term)."""
    def proj(P, v):
        u, w, valid, _ = project(P, v)
        u, w = r32(u), r32(w)
        inimg = valid & (u >= 0) & (u <= P.W - 1) & (w >= 0) & (w <= P.H - 1)
        return u, w, valid, inimg
    return proj


def fp32_rounding_band(scene, graph, n_runs=3, base32=None, n_gn=None, n_pcg=None, sigma_c=0.0, pyr_levels=0):
    """Spread of the oracle's end-to-end result under FP32 rounding, with a
    random tie-break perturbation of one unit roundoff (seeded), of what an
    FP32 execution rounds: the node parameters after every update, the warped
    vertices, their pixel coordinates, the residuals and Jacobian entries, and
    the CG vectors and matrix-vector products.  This measures how far any FP32 execution of the
    same algorithm may land from the FP64 result: CG amplifies rounding along
    the system's ill-conditioned (depth) directions, and a projection within
    rounding of a pixel boundary takes the other cell of the piecewise
    bilinear image and DT gradients.
    Returns (oracle result dict, max |E_k - E_ref|, max |V_k - V_ref|)."""
    ref = onr.solve_scene(scene, graph=graph, base32=base32, n_gn=n_gn, n_pcg=n_pcg, sigma_c=sigma_c,
                          pyr_levels=pyr_levels)
    orig = (onr.pcg, onr.linearise, onr.apply_update, onr.warp, onr.project)
    dE, dV = 0.0, 0.0
    for seed in range(n_runs):
        r32 = _r32(np.random.default_rng(1000 + seed))

        def lin32(P, R, t):
            F, J = orig[1](P, R, t)
            J = J.tocsr(copy=True)
            J.data = r32(J.data)
            return r32(F), J

        def upd32(R, t, delta):
            R1, t1 = orig[2](R, t, delta)
            return r32(R1), r32(t1)

        onr.pcg = lambda A, b, n: pcg32(A, b, n, r32)
        onr.linearise = lin32
        onr.apply_update = upd32
        def warp32(P, R, t):
            # an FP32 warp is exact where the displacement is exactly zero
            v = orig[3](P, R, t)
            return np.where(v != P.base, r32(v), v)

        onr.warp = warp32
        onr.project = _project32(orig[4], r32)
        try:
            o = onr.solve_scene(scene, graph=graph, base32=base32, n_gn=n_gn, n_pcg=n_pcg, sigma_c=sigma_c,
                                pyr_levels=pyr_levels)
        finally:
            onr.pcg, onr.linearise, onr.apply_update, onr.warp, onr.project = orig
        dE = max(dE, abs(o["e1"]["total"] - ref["e1"]["total"]))
        dV = max(dV, float(np.abs(o["v"] - ref["v"]).max()))
    return ref, dE, dV


def oracle_cg_spread(A, b, n, rel=1e-13, n_runs=3):
    """How reproducible the oracle's own n-step PCG is: the FP64 CG rerun with
    every matrix-vector product perturbed by a relative error of ``rel``
    (seeded normal), the magnitude of a compensated-FP32 pair product's error
    (2^-48 of the sum of |terms| per product, up to ~1e-13 of the result where
    the J^T J p terms cancel).  On nearly singular systems the n-step iterate
    is forward unstable: one part in 1e14 per product moves it by up to ~4e-3
    at some Gauss-Newton steps of the body solve.  Returns (FP64 iterate, its info, max relative iterate
    change, max relative change of q(d) = d^T A d / 2 - b^T d)."""
    from oracle.nonrigid import pcg
    dref, info = pcg(A, b, n)
    d = np.asarray(A.diagonal(), dtype=np.float64)
    minv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    q = lambda v: 0.5 * v @ (A @ v) - b @ v  # noqa: E731
    q0 = q(dref)
    s_it = s_q = 0.0
    for seed in range(n_runs):
        rng = np.random.default_rng(3000 + seed)
        x = np.zeros_like(b)
        r = b.copy()
        z = minv * r
        p = z.copy()
        rz = float(r @ z)
        for _ in range(info["iters"]):
            Ap = A @ p
            Ap = Ap * (1.0 + rel * rng.standard_normal(Ap.shape))
            al = rz / float(p @ Ap)
            x = x + al * p
            r = r - al * Ap
            z = minv * r
            rzn = float(r @ z)
            if rzn == 0.0:
                break
            p = z + (rzn / rz) * p
            rz = rzn
        s_it = max(s_it, np.linalg.norm(x - dref) / max(np.linalg.norm(dref), 1e-300))
        s_q = max(s_q, abs(q(x) - q0) / max(abs(q0), 1e-300))
    return dref, info, s_it, s_q


def q_band(A, b, n, n_runs=3):
    """Spread of the quadratic model q(d) = d^T A d / 2 - b^T d at the n-step
    PCG iterate over FP32 executions (``pcg32``), relative to the FP64
    iterate's q.  Returns (FP64 iterate, its info, max relative spread)."""
    from oracle.nonrigid import pcg
    dref, info = pcg(A, b, n)
    q = lambda d: 0.5 * d @ (A @ d) - b @ d  # noqa: E731
    q0 = q(dref)
    spread = 0.0
    for seed in range(n_runs):
        d, _ = pcg32(A, b, n, _r32(np.random.default_rng(2000 + seed)))
        spread = max(spread, abs(q(d) - q0) / abs(q0))
    return dref, info, spread


def ragged_scene(rings, segs, n_nodes, K, side=96, shift=0.0, seed=5):
    """A capsule capture with odd sizes (rings, segments, nodes, K, a
    non-square image, optionally shifted so it leaves the image)."""
    import synth
    V, F = synth.capsule_mesh(0.3, 1.0, rings, segs)
    V = V + np.array([shift, 0.0, 3.0])
    cam = synth.Camera(f=150.0 * side / 128.0, W=side, H=side + 7)
    alb = synth.value_noise_albedo(V, seed)
    mat = synth.half_split_material(V, seed)
    gt = synth.smooth_deformation(V, min(n_nodes, len(V)), 0.05, 0.01, seed)
    rgb, mask = synth.render(gt["V"], F, alb, cam)
    rng = np.random.default_rng(seed)
    rgb = (rgb + rng.normal(0, 0.01, rgb.shape)).astype(np.float32)
    dt = synth.contour_distance_transform(mask).astype(np.float32)
    return synth.Scene("ragged", cam, V.astype(np.float32), F.astype(np.int32), alb.astype(np.float32),
                       mat.astype(np.float32), rgb, dt, mask, n_nodes, K, 4, 15, (1.0, 0.1, 10.0), gt["V"])


def surface_rounding_band(scene, base32=None, V0=None, prev1=None, prev2=None, n_gn=None, n_pcg=None,
                          n_runs=3, sigma_c=0.0, pyr_levels=0, part_mask=None, vpart=None):
    """``fp32_rounding_band`` for the per-vertex surface stage: the spread of
    the oracle's result when its Jacobian entries, residuals, CG vectors and
    products, the vertex positions after every update and their pixel
    coordinates are rounded to FP32 with a random tie-break of one unit
    roundoff.
    Returns (oracle result dict, max |E_k - E_ref|, max |V_k - V_ref|)."""
    from oracle import pyramid as opyr
    from oracle import surface as osf
    kw = dict(base32=base32, V0=V0, n_gn=n_gn, n_pcg=n_pcg, prev1=prev1, prev2=prev2, sigma_c=sigma_c,
              pyr_levels=pyr_levels, part_mask=part_mask, vpart=vpart)
    ref = osf.solve_scene(scene, **kw)
    orig_pcg, orig_lin, orig_gn, orig_proj = onr.pcg, osf.linearise, osf.gauss_newton, onr.project
    dE, dV = 0.0, 0.0
    for seed in range(n_runs):
        r32 = _r32(np.random.default_rng(3000 + seed))

        def lin32(P, V, directions=True):
            F, J = orig_lin(P, V, directions)
            J = J.tocsr(copy=True)
            J.data = r32(J.data)
            return r32(F), J

        def gn32(P, V, n_gn, n_pcg):
            V = np.asarray(V, dtype=np.float64).copy()
            hist = []
            for gn in range(n_gn):
                P.level = opyr.level_of(gn, P.pyr_levels)
                A, b, F, _ = osf.normal_equations(P, V)
                delta, info = onr.pcg(A, b, n_pcg)
                hist.append(dict(energy=float(F @ F), step_norm=float(np.linalg.norm(delta)),
                                 pcg_iters=info["iters"], breakdown=info["breakdown"]))
                V = r32(V + delta.reshape(-1, 3))
            P.level = onr.final_level(P)
            return V, hist

        onr.pcg = lambda A, b, n: pcg32(A, b, n, r32)
        osf.linearise = lin32
        osf.gauss_newton = gn32
        onr.project = _project32(orig_proj, r32)
        try:
            o = osf.solve_scene(scene, **kw)
        finally:
            onr.pcg, osf.linearise, osf.gauss_newton, onr.project = orig_pcg, orig_lin, orig_gn, orig_proj
        dE = max(dE, abs(o["e1"]["total"] - ref["e1"]["total"]))
        dV = max(dV, float(np.abs(o["V"] - ref["V"]).max()))
    return ref, dE, dV

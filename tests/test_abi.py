"""The C-ABI library builds, loads and exports every declared entry point
(CPU: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lc_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1810_02648_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_all_declared_symbols_exported(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1810_02648_gb300 import livecap
    assert set(_declared()) <= set(livecap._SIGS)


def test_no_device_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1810_02648_gb300 import Context, LivecapError
    with pytest.raises(LivecapError):
        Context(0)


def test_params_default(lib):
    from paper_1810_02648_gb300 import livecap
    livecap.load()
    p = livecap.lc_params()
    assert livecap.load().lc_params_default(ctypes.byref(p)) == 0
    # pose-stage weights from the paper's parameter list (Sec. 5)
    assert (p.lambda_2d, p.lambda_3d, p.lambda_sil) == (460.0, 28.0, 200.0)
    assert (p.n_gn, p.n_pcg) == (5, 20)
    # surface stage: Sec. 4 counts (3 Gauss-Newton x 4 PCG) and the weights
    # of Sec. 5 read in millimetres, rescaled to metres and w_photo = 1
    assert (p.n_gn_surface, p.n_pcg_surface) == (3, 4)
    assert (p.w_smooth, p.w_edge, p.w_velocity, p.w_acceleration) == (1e3, 3e3, 25.0, 10.0)
    assert p.target_energy == 0.0 and p.pose_solver == 0
    # pose-stage regularisers (Sec. 5): lambda_temporal 1.5, lambda_anatomic 1e6
    assert (p.lambda_temporal, p.lambda_anatomic) == (1.5, 1e6)
    # robust colour kernel off; photometric pyramid off, the paper's kernel
    # sizes (Sec. 3.4: 15, 9, 3) ready for it
    assert p.sigma_c == 0.0 and p.pyr_levels == 0
    assert list(p.pyr_ksize) == [15, 9, 3]
    # the pose stage's skinned displacement (Sec. 3.4) is opt-in
    assert p.pose_displacement == 0


def test_bench_options_and_launch_count():
    """Host logic of bench.py: the options of the per-frame path become
    config keys, and the frame preparation's kernel count per step."""
    import argparse
    import bench
    a = argparse.Namespace(pyramid=0, sigma_c=0.0, body_parts=False, frame_prep=False)
    assert bench.path_options(a) == {}
    a = argparse.Namespace(pyramid=3, sigma_c=0.5, body_parts=True, frame_prep=True)
    opt = bench.path_options(a)
    assert opt["pyramid_levels"] == 3 and opt["sigma_c"] == 0.5 and "body_parts" in opt and "frame_prep" in opt
    # packing + contour flags + column pass + row pass, then per level a box
    # mean where the factor exceeds 1 and two blur passes
    assert bench.frame_prep_kernels(0) == 4
    assert bench.frame_prep_kernels(1) == 6          # the finest level: two blur passes
    assert bench.frame_prep_kernels(3) == 4 + 3 + 3 + 2


def test_autotune_table_text_round_trip():
    """The shape table's text form (host only): a valid line is merged and
    exported again; a malformed line or an unknown shape is refused."""
    from paper_1810_02648_gb300.livecap import LivecapError, autotune_table, autotune_table_load
    autotune_table_load("K4.N12.n9x2,K8.N17.n12x1\t3 512 16 2 1.25\nK4.N11.n8x5\t0 128 4 8 0.5\n")
    lines = dict(line.split("\t") for line in autotune_table().splitlines())
    assert lines["K4.N12.n9x2,K8.N17.n12x1"].split()[:4] == ["3", "512", "16", "2"]
    assert lines["K4.N11.n8x5"].split()[:4] == ["0", "128", "4", "8"]
    for bad in ("no tab here 3 256 8 4 1\n", "K4.N1.n1x1\t3 300 8 4 1\n", "K4.N1.n1x1\t3 256 12 4 1\n",
                "K4.N1.n1x1\t3 256 2 4 1\n", "K4.N1.n1x1\t9 256 8 4 1\n", "K4.N1.n1x1\t3 256 8\n"):
        with pytest.raises(LivecapError):
            autotune_table_load(bad)
    assert "K4.N1.n1x1" not in autotune_table()

"""The warm start's training-set filter (host logic, CPU tensors): frames
whose plain solve ran away (final energy far above the set's median, or not
finite) or whose targets are not finite are dropped, the rest kept in order."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _set(n_frames, n_nodes=5, seed=0):
    g = torch.Generator().manual_seed(seed)
    F = torch.randn(n_frames, n_nodes, 64, generator=g)
    T = torch.randn(n_frames, n_nodes, 6, generator=g)
    return F, T


def test_keeps_every_converged_frame_in_order():
    from paper_1810_02648_gb300.warmstart import keep_converged
    F, T = _set(6)
    E = np.array([10.0, 12.0, 9.0, 11.0, 900.0, 10.5])   # 900 <= 100 x median (10.75)
    F2, T2, keep = keep_converged(F, T, E)
    assert keep.all()
    assert torch.equal(F2, F) and torch.equal(T2, T)


def test_drops_runaway_and_non_finite_frames():
    from paper_1810_02648_gb300.warmstart import keep_converged
    F, T = _set(7)
    E = np.array([10.0, 1e6, 9.0, np.nan, 11.0, 10.0, 10.0])
    T[5, 2, 3] = float("inf")
    F2, T2, keep = keep_converged(F, T, E)
    assert keep.tolist() == [True, False, True, False, True, False, True]
    idx = [0, 2, 4, 6]
    assert torch.equal(F2, F[idx]) and torch.equal(T2, T[idx])


def test_factor_is_relative_to_the_median():
    from paper_1810_02648_gb300.warmstart import keep_converged
    F, T = _set(3)
    E = np.array([1.0, 2.0, 8.5])                          # median 2: 8.5 > 4 x 2
    _, _, keep = keep_converged(F, T, E, factor=4.0)
    assert keep.tolist() == [True, True, False]
    _, _, keep = keep_converged(F, T, E)
    assert keep.all()

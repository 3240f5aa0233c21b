import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


@pytest.fixture(scope="session")
def tiny_scene():
    import synth
    return synth.make_scene("tiny")


@pytest.fixture(scope="session")
def tiny_graph(tiny_scene):
    from oracle import graph
    s = tiny_scene
    return graph.build_graph(s.V, s.material, s.n_nodes, s.K)


@pytest.fixture(scope="session")
def tiny_problem(tiny_scene, tiny_graph):
    from oracle import nonrigid as nr
    P = nr.problem_from_scene(tiny_scene, tiny_graph)
    R, t = nr.identity_params(P.n)
    nr.frame_decisions(P, tiny_scene.F, R, t)
    return P

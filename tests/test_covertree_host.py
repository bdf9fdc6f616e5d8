"""The C++ cover-tree construction (host only, through the C ABI) checked against the invariants
of §4.1 with the oracle's float64 distances, on random data, the workload-1 dictionary under both
metrics, and a dictionary with duplicates and phase-rotated copies."""
import numpy as np
import pytest

import mrfgen
from tree_check import check_tree


@pytest.fixture(scope="module")
def mrf():
    import paper_1810_01967_gb300 as m
    from paper_1810_01967_gb300 import build as b
    b.build()
    return m


def _rand(g, *shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def test_random(mrf):
    g = np.random.Generator(np.random.PCG64(61))
    A = _rand(g, 400, 6).astype(np.complex64)
    check_tree(A, mrf.tree_build_host(A))


@pytest.mark.parametrize("cone", ["complex", "real_pos"])
def test_workload1_dictionary(mrf, cone):
    A = mrfgen.make_dictionary(1)["atoms"]
    nodes, dups = check_tree(A, mrf.tree_build_host(A, cone=cone), cone=cone)
    assert nodes == A.shape[0] and dups == 0


def test_duplicates_and_rotations(mrf):
    g = np.random.Generator(np.random.PCG64(62))
    B = _rand(g, 80, 5)
    A = np.concatenate([B, B[:12] * np.exp(0.7j), B[3:9]]).astype(np.complex64)
    T = mrf.tree_build_host(A)
    nodes, dups = check_tree(A, T)
    assert dups == 18
    assert np.all(T["rep"][80:92] == np.arange(12)) and np.all(T["rep"][92:] == np.arange(3, 9))
    # Euclidean metric: rotations are not duplicates there
    nodes_e, dups_e = check_tree(A, mrf.tree_build_host(A, cone="real_pos"), cone="real_pos")
    assert dups_e == 6


def test_bad_arguments(mrf):
    with pytest.raises(mrf.MRFError):
        mrf.tree_build_host(np.zeros((0, 4), np.complex64))

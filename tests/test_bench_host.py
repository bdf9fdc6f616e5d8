"""Host logic of bench.py on the CPU: the T1/T2 accuracy metric, the CPU-baseline leg (the
oracle's timed sample and the agreement of a projection with it, here a float32 numpy argmax
standing in for the GPU), and the fail-soft report of that auxiliary figure."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import mrfgen  # noqa: E402
from oracle import mrf_oracle as mo  # noqa: E402


def test_accuracy_metric():
    truth = np.array([100.0, 200.0, 400.0, 800.0])
    mask = np.array([True, True, True, False])
    assert bench.t_accuracy(truth, truth, mask) == 1.0
    est = np.array([110.0, 180.0, 400.0, 0.0])       # errors 10 %, 10 %, 0 %; the 4th is masked
    assert bench.t_accuracy(est, truth, mask) == pytest.approx(1.0 - 0.2 / 3)


@pytest.fixture(scope="module")
def small():
    dic = mrfgen.make_dictionary(1)
    p = mrfgen.make_problem(1, dic=dic)
    Z = mo.adjoint(p["Y"], p["masks"], p["Ny"], p["Nx"])
    return dic["atoms"], Z


def test_baseline_sample_and_agreement(small):
    A, Z = small

    def argmax32(Zs):
        Zs = np.asarray(Zs, np.complex64)
        return (np.abs(Zs.conj() @ A.T) / np.linalg.norm(A, axis=1)).argmax(1)

    r = bench.oracle_baseline(Z[:128], A, target_s=0.2, gpu_idx=argmax32)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] >= 1
    assert r["gpu_agreement_on_sample"] >= 0.98
    # a projection that is always wrong is reported as such
    r = bench.oracle_baseline(Z[:64], A, target_s=0.1, gpu_idx=lambda Zs: np.full(len(Zs), -1))
    assert r["gpu_agreement_on_sample"] == 0.0


def test_baseline_reports_a_failing_projection(small):
    A, Z = small

    def broken(Zs):
        raise RuntimeError("no device")

    r = bench.oracle_baseline(Z[:32], A, target_s=0.1, gpu_idx=broken)
    assert "gpu_agreement_on_sample" not in r
    assert r["gpu_agreement_error"].startswith("RuntimeError")

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


def test_quality_leg_keeps_the_callers_dictionary(monkeypatch):
    """reconstruction_quality builds its own dictionaries for the tree, learned, compressed and
    aligned forms, closes each of them, and leaves the caller's dictionary open (the
    CPU-baseline leg projects with it afterwards).  Library calls are stubbed on the CPU."""
    torch = pytest.importorskip("torch")

    class FakeDict:
        def __init__(self):
            self.closed = False

        def close(self):
            self.closed = True

    built = []

    class FakeSvdOp:
        def __init__(self, V, op):
            pass

        def compress(self, A, Ac):
            pass

        def reconstruct(self, *a, **k):
            pass

        def close(self):
            pass

    class FakeMrf:
        SvdOp = FakeSvdOp

        @staticmethod
        def build_dict_index(*a, **k):
            built.append(FakeDict())
            return built[-1]

        @staticmethod
        def recon_opts(**k):
            return k

        @staticmethod
        def proj_opts(**k):
            return k

        @staticmethod
        def reconstruct(D, *a, **k):
            assert not D.closed, "reconstruct called with a closed dictionary"
            return {"n_fallback": 0, "n_dist_evals": 0}

        @staticmethod
        def attach_mlp(D, M):
            pass

        @staticmethod
        def svd_basis(D, s):
            return None, np.ones(s)

    class FakeEvent:
        def __init__(self, **k):
            pass

        def record(self, *a):
            pass

        def elapsed_time(self, other):
            return 1.0

    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(bench, "train_learned",
                        lambda mrf, D, dic, dev: (None, 0.0, np.zeros(200)))
    N, L, d = 4, 8, 10
    g = np.random.Generator(np.random.PCG64(3))
    dic = {"atoms": (g.standard_normal((d, L)) + 0j).astype(np.complex64),
           "params": np.abs(g.standard_normal((d, 3))).astype(np.float32) + 1.0,
           "grid_shape": (d,)}
    ph = {"labels": np.array([0] * 8 + [-1] * 8), "T1": np.full(16, 1000.0),
          "T2": np.full(16, 100.0), "B0": np.zeros(16)}
    p = {"Ny": N, "Nx": N, "L": L, "Y": np.zeros((N, N, L), np.complex64), "phantom": ph}
    caller = FakeDict()
    out = bench.reconstruction_quality(FakeMrf, caller, None, p, dic, "cpu", None, iters=2,
                                       fp32=True, forms=True)
    assert not caller.closed
    assert built and all(D.closed for D in built)
    assert {"bf16", "fp8", "fp32", "covertree", "learned", "bf16_aligned_real"} <= set(out)

"""GPU parity of the batching form (mrf_batch: slices of different sizes stacked, one projection
launch per iteration, optional CUDA-graph replay): every slice of a batch equals the same slice
reconstructed alone through mrf_ipg_step, graph replay equals eager execution bit for bit, the
BLIP iterates agree with the float64 oracle's, and the capture rules are enforced."""
import numpy as np
import pytest

import mrfgen
from oracle import mrf_oracle as mo
from gpu_util import to_dev, check_projection, check_bound_rule, bf16_bound

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = (24, 32, 40)


@pytest.fixture(scope="module")
def mrf():
    import paper_1810_01967_gb300 as m
    from paper_1810_01967_gb300 import build as b
    b.build()
    return m


@pytest.fixture(scope="module")
def setup():
    dic = mrfgen.make_dictionary(1)
    probs = [mrfgen.make_problem(1, i, dic=dic, N=N) for i, N in enumerate(SIZES)]
    return dic, probs


def make_batch(mrf, D, probs):
    ops = [mrf.make_op(p["Ny"], p["Nx"], p["L"], to_dev(p["masks"])) for p in probs]
    B = mrf.Batch(D, ops)
    B.load([to_dev(p["Y"]) for p in probs])
    return B, ops


def slice_arrays(B, s):
    v = B.views(s)
    return v["X"].cpu().numpy(), v["idx"].cpu().numpy(), v


def alone(mrf, D, p, iters, opts):
    n, L = p["Ny"] * p["Nx"], p["L"]
    op = mrf.make_op(p["Ny"], p["Nx"], L, to_dev(p["masks"]))
    AHY = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    mrf.adjoint(op, to_dev(p["Y"]), AHY)
    X = torch.zeros((n, L), dtype=torch.complex64, device="cuda")
    idx = torch.zeros(n, dtype=torch.int32, device="cuda")
    for _ in range(iters):
        mrf.ipg_step(D, op, AHY, X, 1.0, idx, opts=opts)
    return X.cpu().numpy(), idx.cpu().numpy()


@pytest.mark.parametrize("mode", ["fp32", "bf16"])
def test_batch_equals_slices_alone(mrf, setup, mode):
    dic, probs = setup
    D = mrf.build_dict_index(dic["atoms"], dic["params"], pack_bf16=(mode == "bf16"))
    opts = mrf.proj_opts(mode=mode, certify=False)
    iters = 4
    res = {}
    for g in (False, True):
        B, ops = make_batch(mrf, D, probs)
        B.run(iters, 1.0, opts, use_graph=g)
        torch.cuda.synchronize()
        res[g] = [slice_arrays(B, s) for s in range(len(probs))]
        B.close()
    for s, p in enumerate(probs):
        Xg, ig, _ = res[True][s]
        Xe, ie, _ = res[False][s]
        assert np.array_equal(ig, ie) and np.array_equal(Xg, Xe)   # graph replay == eager
        Xa, ia = alone(mrf, D, p, iters, opts)
        pow2 = (p["Ny"] & (p["Ny"] - 1)) == 0
        if mode == "fp32" and not pow2:
            # the batch's one-launch gradient is the single slice's mixed-radix kernel on the
            # same tiles, and the projection is exact: identical iterates
            assert np.array_equal(ie, ia)
            np.testing.assert_allclose(Xe, Xa, rtol=0, atol=1e-6 * np.abs(Xa).max())
        elif mode == "fp32":
            # a power-of-two slice alone runs the radix-2 kernel, in the batch the mixed-radix
            # one: the transforms round differently (~1e-7), so atoms may differ at near-ties
            same = ie == ia
            assert same.mean() >= 0.995
            np.testing.assert_allclose(Xe[same], Xa[same], rtol=0, atol=1e-5 * np.abs(Xa).max())
        else:
            # BF16 candidate sets depend on the atom split of the launch: same answers up to
            # the BF16 near-ties
            assert np.mean(ie == ia) >= 0.99


def slice_inputs(mrf, D, probs):
    """Per slice: its operator and A^H Y (mrf_adjoint, the call mrf_batch_load makes)."""
    out = []
    for p in probs:
        n, L = p["Ny"] * p["Nx"], p["L"]
        op = mrf.make_op(p["Ny"], p["Nx"], L, to_dev(p["masks"]))
        AHY = torch.empty((n, L), dtype=torch.complex64, device="cuda")
        mrf.adjoint(op, to_dev(p["Y"]), AHY)
        out.append((op, AHY))
    return out


def gpu_z(mrf, D, B, ins, s):
    """The gradient step the batch applies to slice s's current iterate (the same kernels)."""
    v = B.views(s)
    op, AHY = ins[s]
    Z = torch.empty_like(v["X"])
    mrf.gradient(D, op, AHY, v["X"].clone(), 1.0, Z)
    torch.cuda.synchronize()
    return Z.cpu().numpy()


@pytest.mark.parametrize("mode,certify", [("fp32", False), ("bf16", False), ("bf16x3", True),
                                          ("tree_tc", True)])
def test_batch_follows_the_oracle_every_iteration(mrf, setup, mode, certify):
    """Every iteration of the stacked batch: the oracle projects each slice's own Z (the GPU's
    gradient step of the batch's iterate) and the batch's answers follow the exact rule (FP32,
    certified split-BF16, the certified tensor-core tree search at eps = 0) or the kernel-bound
    rule (uncertified BF16); the look-up table then returns the atoms' parameters."""
    dic, probs = setup
    A = dic["atoms"]
    L = A.shape[1]
    tree = mode == "tree_tc"
    D = mrf.build_dict_index(A, dic["params"], pack_bf16=True,
                             pack_bf16x3=(mode in ("bf16x3", "tree_tc")), build_tree=tree,
                             tree_tc=tree)
    B, ops = make_batch(mrf, D, probs)
    ins = slice_inputs(mrf, D, probs)
    opts = mrf.proj_opts(mode=mode, certify=certify)
    iters = 3
    for it in range(iters):
        Zs = [gpu_z(mrf, D, B, ins, s) for s in range(len(probs))]
        B.run(1, 1.0, opts)
        torch.cuda.synchronize()
        for s in range(len(probs)):
            X, idx, v = slice_arrays(B, s)
            rho = v["rho"].cpu().numpy()
            if mode == "bf16":
                agree = check_bound_rule(Zs[s], A, idx, rho, bf16_bound(L), g_X=X)
            else:
                agree = check_projection(Zs[s], A, idx, rho, g_X=X)[0]
            print(f"{mode} iteration {it} slice {s}: agreement with the oracle {agree:.4f}")
    n_tot = sum(p["Ny"] * p["Nx"] for p in probs)
    prm = torch.empty((n_tot, dic["params"].shape[1]), dtype=torch.float32, device="cuda")
    B.lut(prm)
    torch.cuda.synchronize()
    prm = prm.cpu().numpy()
    for s in range(len(probs)):
        X, idx, v = slice_arrays(B, s)
        a = v["offset"]
        assert np.array_equal(prm[a:a + v["n"]], dic["params"][idx])


def check_learned_rule(Z, A, dic, gi, grho, thr, bound):
    """The learned form's contract per voxel: the exhaustive answer (kernel-bound rule) or an
    accepted proposal -- normalised correlation at least the threshold and a local maximum over
    its valid grid neighbours (the edge rule); rho is the returned atom's exact density."""
    Z = np.asarray(Z, np.complex128)
    ref = mo.project(Z, A)
    c = mo.correlation(Z, A, gi)
    zero = np.sum(np.abs(Z) ** 2, axis=1) == 0
    near = c >= ref["s1"] - 2.0 * bound
    cell_atom = np.asarray(dic["cell_atom"])
    cells = np.argwhere(cell_atom >= 0)
    shape = np.array(cell_atom.shape)
    local = np.ones(len(gi), bool)
    for off in np.ndindex(*(3,) * cell_atom.ndim):
        o = np.array(off) - 1
        if not o.any():
            continue
        nc = cells[gi] + o
        inside = np.all((nc >= 0) & (nc < shape), axis=1)
        nj = np.full(len(gi), -1)
        nj[inside] = cell_atom[tuple(nc[inside].T)]
        ok = nj >= 0
        cn = np.full(len(gi), -np.inf)
        cn[ok] = mo.correlation(Z[ok], A, nj[ok])
        local &= cn <= c + 1e-5
    accepted = (c >= thr - 1e-6) & local
    bad = np.flatnonzero(~zero & ~near & ~accepted)
    assert bad.size == 0, f"{bad.size} voxels break the learned form's contract, e.g. {bad[:5]}"
    rr = mo.density(Z, A, gi)
    rr[zero] = 0
    err = np.abs(np.asarray(grho) - rr) / np.maximum(np.abs(rr), 1e-30)
    assert np.max(np.where(zero, np.abs(grho), err)) <= 1e-4
    return float(np.mean(gi == ref["idx"]))


@pytest.mark.parametrize("mode,pair", [("covertree", 0), ("learned", 0), ("learned", 1),
                                       ("tree_tc", 0)])
def test_graph_replay_with_device_side_fallback(mrf, setup, mode, pair):
    """The cover-tree and learned forms under graph replay: their exhaustive fallback takes the
    listed voxel count from the device (no read-back inside the captured iteration).  Graph and
    eager runs give the same answers up to BF16 near-ties (the fallback's atom split is sized
    for the list's capacity instead of its length).  Every graph-replayed iteration k follows
    the oracle on the GPU's own Z: a fresh batch run of k - 1 iterations gives the iterate, a
    fresh run of k iterations replays iteration k from the captured graph, and its answers
    obey the form's rule (eps = 0 cover tree with its exhaustive fallback: the kernel-bound
    rule; learned: that, or an accepted proposal above the threshold and a local maximum; the
    uncertified tensor-core tree search at eps = 0, which has no fallback and reads nothing
    back: the kernel-bound rule)."""
    dic, probs = setup
    A = dic["atoms"]
    L = A.shape[1]
    D = mrf.build_dict_index(A, dic["params"], grid_shape=dic["grid_shape"],
                             pack_bf16=True, build_tree=(mode in ("covertree", "tree_tc")),
                             tree_tc=(mode == "tree_tc"))
    if mode == "learned":
        M = mrf.MLP(D, dic["axes"], dic["cell_atom"], hidden=32)
        mrf.attach_mlp(D, M)
    D.set_tune(bf16_pair=pair)           # the fallback's search on single CTAs or on CTA pairs
    opts = mrf.proj_opts(mode=mode, certify=False, eps=0.0)
    iters = 3
    res = {}
    for g in (False, True):
        B, ops = make_batch(mrf, D, probs)
        B.run(iters, 1.0, opts, use_graph=g)
        torch.cuda.synchronize()
        res[g] = [slice_arrays(B, s) for s in range(len(probs))]
        B.close()
    D.check()
    for s, p in enumerate(probs):
        Xg, ig, _ = res[True][s]
        Xe, ie, _ = res[False][s]
        same = ig == ie
        assert same.mean() >= 0.99, (s, same.mean())
        np.testing.assert_allclose(Xg[same], Xe[same], rtol=0, atol=1e-5 * np.abs(Xe).max())
    ins = slice_inputs(mrf, D, probs)
    for k in range(2, iters + 1):          # iteration k >= 2 of a run replays the graph
        B, ops = make_batch(mrf, D, probs)
        B.run(k - 1, 1.0, opts, use_graph=True)
        Zs = [gpu_z(mrf, D, B, ins, s) for s in range(len(probs))]
        B.close()
        B, ops = make_batch(mrf, D, probs)
        B.run(k, 1.0, opts, use_graph=True)
        torch.cuda.synchronize()
        for s in range(len(probs)):
            X, idx, v = slice_arrays(B, s)
            rho = v["rho"].cpu().numpy()
            if mode in ("covertree", "tree_tc"):
                agree = check_bound_rule(Zs[s], A, idx, rho, bf16_bound(L), g_X=X)
            else:
                agree = check_learned_rule(Zs[s], A, dic, idx, rho, 0.98, bf16_bound(L))
            print(f"{mode} pair={pair} replayed iteration {k} slice {s}: agreement with the "
                  f"oracle {agree:.4f}")
        B.close()


def test_graph_replay_after_the_scratch_grew(mrf, setup):
    """A batch's captured iteration references the dictionary's scratch buffers; when another,
    larger batch on the same dictionary grows (reallocates) them, the first batch's next replay
    captures again instead of touching the freed buffers: its iterates equal an eager run of
    the same slices bit for bit."""
    dic, probs = setup
    D = mrf.build_dict_index(dic["atoms"], dic["params"], pack_bf16=True)
    opts = mrf.proj_opts(mode="fp32", certify=False)
    small = [probs[0]]
    big = [mrfgen.make_problem(1, 7 + k, dic=dic, N=64) for k in range(3)]
    A, _ = make_batch(mrf, D, small)
    A.run(2, 1.0, opts, use_graph=True)           # eager iteration, then a captured one
    Bb, _ = make_batch(mrf, D, big)               # grows the dictionary's scratch
    Bb.run(2, 1.0, opts, use_graph=True)
    A.run(3, 1.0, opts, use_graph=True)           # eager, then replays: captured again
    torch.cuda.synchronize()
    Xg, ig, _ = slice_arrays(A, 0)
    E, _ = make_batch(mrf, D, small)
    E.run(5, 1.0, opts)
    torch.cuda.synchronize()
    Xe, ie, _ = slice_arrays(E, 0)
    assert np.array_equal(ig, ie) and np.array_equal(Xg, Xe)
    D.check()
    for b in (A, Bb, E):
        b.close()


def test_capture_rules_and_errors(mrf, setup):
    from paper_1810_01967_gb300 import MRFError
    dic, probs = setup
    D = mrf.build_dict_index(dic["atoms"], pack_bf16=True)
    B, ops = make_batch(mrf, D, probs)
    with pytest.raises(MRFError, match="graph"):
        B.run(2, 1.0, mrf.proj_opts(mode="bf16", certify=True), use_graph=True)
    with pytest.raises(MRFError):
        B.slice(len(probs))
    # eager runs accept every mode, certified included
    B.run(1, 1.0, mrf.proj_opts(mode="bf16", certify=True))
    torch.cuda.synchronize()
    other = mrfgen.make_problem(1, 0, dic=dic, L=50, N=16)
    op = mrf.make_op(16, 16, 50, to_dev(other["masks"]))
    with pytest.raises(MRFError):
        mrf.Batch(D, [ops[0], op])

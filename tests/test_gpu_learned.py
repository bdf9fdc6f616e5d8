"""GPU parity of the learned proposal (MRF_PROJ_LEARNED) and its training kernels against the
float64 oracle network: forward outputs, MSE loss and every parameter gradient on identical
weights and inputs; v1 and the canonical inputs; the fallback rules of the projection; and the
gain of a trained network over an untrained one (fewer exhaustive fallbacks, same answers)."""
import numpy as np
import pytest

import mrfgen
from oracle import mlp as omlp
from oracle import mrf_oracle as mo
from gpu_util import to_dev, check_projection

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mrf():
    import paper_1810_01967_gb300 as m
    from paper_1810_01967_gb300 import build as b
    b.build()
    return m


@pytest.fixture(scope="module")
def cfg1():
    dic = mrfgen.make_dictionary(1)
    p = mrfgen.make_problem(1, dic=dic)
    Z = mo.adjoint(p["Y"], p["masks"], p["Ny"], p["Nx"]).astype(np.complex64)
    return dic, p, Z


def dictionary(mrf, dic):
    return mrf.build_dict_index(dic["atoms"], dic["params"], grid_shape=dic["grid_shape"])


def flat(p):
    return np.concatenate([p[k].astype(np.float32).ravel() for k in
                           ("W1", "b1", "W2", "b2", "W3", "b3")])


def test_gradients_match_oracle(mrf, cfg1):
    dic = cfg1[0]
    D = dictionary(mrf, dic)
    H = 48
    M = mrf.MLP(D, dic["axes"], dic["cell_atom"], hidden=H)
    I = 2 * dic["atoms"].shape[1]
    g = np.random.Generator(np.random.PCG64(81))
    p = omlp.init(I, n_hidden=H, n_out=3, seed=3)
    for k in ("b1", "b2", "b3"):
        p[k] = g.normal(0, 0.2, p[k].shape)
    w = flat(p)
    M.params(w)
    assert np.array_equal(M.params(), w)
    p64 = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    B = 96
    X = (g.normal(size=(B, I)) / np.sqrt(I)).astype(np.float32)
    T = g.normal(size=(B, 3)).astype(np.float32)
    Y, loss, grads = M.grad(to_dev(X), to_dev(T))
    y, cache = omlp.forward(p64, X.astype(np.float64))
    lref, dy = omlp.mse(y, T.astype(np.float64))
    gref = omlp.backward(p64, cache, dy)
    np.testing.assert_allclose(Y, y, rtol=1e-4, atol=1e-5)
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    off = 0
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        n = gref[k].size
        gk = grads[off:off + n].reshape(gref[k].shape)
        off += n
        rel = np.linalg.norm(gk - gref[k]) / np.linalg.norm(gref[k])
        assert rel < 1e-4, (k, rel)


@pytest.mark.parametrize("L,H,B", [(100, 512, 300), (37, 48, 16389), (100, 320, 129)])
def test_bf16_inference_matches_emulation(mrf, cfg1, L, H, B):
    """The learned projection's inference: BF16 weights and activations on the tensor cores
    with FP32 accumulation, bias + GELU fused into the layer epilogues.  Against a float64
    evaluation of the same network on the BF16-rounded weights, inputs and first-layer
    activations; odd input widths (2L = 74, padded rows), hidden widths whose column tiles are not
    multiples of 32 (48, 320 = 2 x 160), ragged row tiles and more rows than one chunk."""
    dic = cfg1[0]
    A = np.ascontiguousarray(dic["atoms"][:, :L])
    D = mrf.build_dict_index(A, dic["params"], grid_shape=dic["grid_shape"])
    M = mrf.MLP(D, dic["axes"], dic["cell_atom"], hidden=H)
    I = 2 * L
    g = np.random.Generator(np.random.PCG64(L + H))
    p = omlp.init(I, n_hidden=H, n_out=3, seed=5)
    for k in ("b1", "b2", "b3"):
        p[k] = g.normal(0, 0.2, p[k].shape)
    M.params(flat(p))
    X = (g.normal(size=(B, I)) / np.sqrt(I) * 4).astype(np.float32)
    Y = torch.empty((B, 3), dtype=torch.float32, device="cuda")
    M.infer(to_dev(X), Y)
    Yg = Y.cpu().numpy()

    def bf(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(
            torch.bfloat16).to(torch.float64).numpy()

    def gelu(v):
        from scipy.special import erf
        return 0.5 * v * (1 + erf(v / np.sqrt(2)))

    f32 = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    a1 = gelu(bf(X) @ bf(p["W1"]) + f32["b1"])
    a2 = gelu(bf(a1) @ bf(p["W2"]) + f32["b2"])
    ref = a2 @ f32["W3"] + f32["b3"]
    scale = np.abs(ref).max()
    err = np.abs(Yg - ref).max() / scale
    # the FP32 training path on the same weights differs by the BF16 rounding itself
    Yf, _, _ = M.grad(to_dev(X[:256]), None)
    errf = np.abs(Yg[:256] - Yf).max() / np.abs(Yf).max()
    print(f"L={L} H={H} B={B}: BF16 inference vs emulation {err:.2e}, vs FP32 forward {errf:.2e}")
    assert err < 2e-3
    assert errf < 5e-2


def test_v1_and_canonical_inputs(mrf, cfg1):
    dic, p, Z = cfg1
    D = dictionary(mrf, dic)
    M = mrf.MLP(D, dic["axes"], dic["cell_atom"], hidden=32)
    Zs = Z[:300]
    Xg = torch.empty((300, 2 * Zs.shape[1]), dtype=torch.float32, device="cuda")
    v1, ts = M.canonical(to_dev(Zs), Xg)
    v1r = omlp.dominant_vector(dic["atoms"])
    assert np.max(np.abs(v1 - v1r)) < 1e-4
    Xr = omlp.canonicalise(Zs, v1r)
    assert np.max(np.abs(Xg.cpu().numpy() - Xr)) < 1e-4
    # target standardisation of (log T1, log T2)
    lt = np.log(dic["params"][:, :2].astype(np.float64))
    np.testing.assert_allclose(ts[:2], lt.mean(0), rtol=1e-5)
    np.testing.assert_allclose(ts[3:5], lt.std(0), rtol=1e-4)


def test_projection_fallback_rules(mrf, cfg1):
    dic, p, Z = cfg1
    A = dic["atoms"]
    D = dictionary(mrf, dic)
    M = mrf.MLP(D, dic["axes"], dic["cell_atom"], hidden=32)
    mrf.attach_mlp(D, M)
    n = Z.shape[0]
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.complex64, device="cuda")
    # every voxel below threshold 2: all projected by the (certified) exhaustive search
    st = mrf.project(D, to_dev(Z), idx, rho, opts=mrf.proj_opts(mode="learned", fallback_thr=2.0),
                     stats=True)
    check_projection(Z, A, idx.cpu().numpy(), rho.cpu().numpy())
    assert st["n_fallback"] == n
    # no fallback: a valid atom of the neighbourhood with its exact density
    st = mrf.project(D, to_dev(Z), idx, rho, stats=True,
                     opts=mrf.proj_opts(mode="learned", fallback_thr=0.0, learned_edge=False))
    gi = idx.cpu().numpy()
    assert st["n_fallback"] == 0 and gi.min() >= 0 and gi.max() < A.shape[0]
    rr = mo.density(Z, A, gi)
    assert np.max(np.abs(rho.cpu().numpy() - rr) / np.abs(rr)) <= 1e-4
    # edge rule alone (threshold 0): the untrained network's windows miss, so voxels fall back
    st = mrf.project(D, to_dev(Z), idx, rho, stats=True,
                     opts=mrf.proj_opts(mode="learned", fallback_thr=0.0, learned_edge=True))
    assert st["n_fallback"] > 0
    assert_local_max(Z, A, dic, idx.cpu().numpy())


def assert_local_max(Z, A, dic, gi, tol=1e-5):
    """Every voxel's atom is a local maximum of the normalised correlation over its valid grid
    neighbours (all 3^k - 1 offsets): what the edge rule guarantees for accepted proposals, and
    what the exhaustive answer satisfies anyway."""
    n = Z.shape[0]
    cell_atom = np.asarray(dic["cell_atom"])
    cells = np.argwhere(cell_atom >= 0)          # row j = grid cell of atom j (C order)
    assert np.array_equal(cell_atom[tuple(cells.T)], np.arange(A.shape[0]))
    c0 = mo.correlation(Z, A, gi)
    nz = np.linalg.norm(Z, axis=1) > 0
    shape = np.array(cell_atom.shape)
    for off in np.ndindex(*(3,) * cell_atom.ndim):
        o = np.array(off) - 1
        if not o.any():
            continue
        nc = cells[gi] + o
        inside = np.all((nc >= 0) & (nc < shape), axis=1)
        nj = np.full(n, -1)
        nj[inside] = cell_atom[tuple(nc[inside].T)]
        ok = nz & (nj >= 0)
        cn = mo.correlation(Z[ok], A, nj[ok])
        assert np.all(cn <= c0[ok] + tol), (off, float(np.max(cn - c0[ok])))


def test_training_gain(mrf, cfg1):
    dic, p, Z = cfg1
    A = dic["atoms"]
    Ny, Nx, L = p["Ny"], p["Nx"], p["L"]
    n = Ny * Nx
    D = dictionary(mrf, dic)
    op = mrf.make_op(Ny, Nx, L, to_dev(p["masks"]))
    AHY = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    mrf.adjoint(op, to_dev(p["Y"]), AHY)
    X0 = to_dev(p["X0"])
    models = {}
    for trained in (False, True):
        M = mrf.MLP(D, dic["axes"], dic["cell_atom"], hidden=128)
        if trained:
            # aliasing residues of the first IPG iterates of this phantom
            X = torch.zeros((n, L), dtype=torch.complex64, device="cuda")
            idx = torch.zeros(n, dtype=torch.int32, device="cuda")
            Zk = torch.empty_like(X)
            for _ in range(3):
                mrf.gradient(D, op, AHY, X, 1.0, Zk)
                M.add_residues(Zk, X0)
                mrf.ipg_step(D, op, AHY, X, 1.0, idx, opts=mrf.proj_opts(mode="bf16"))
            hist = M.train(steps=600, batch=512, lr=1e-3, history=True)
            assert hist[-50:].mean() < 0.3 * hist[:10].mean(), (hist[:10].mean(), hist[-50:].mean())
        models[trained] = M
    out = {}
    for trained, M in models.items():
        mrf.attach_mlp(D, M)
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        rho = torch.empty(n, dtype=torch.complex64, device="cuda")
        st = mrf.project(D, AHY, idx, rho, opts=mrf.proj_opts(mode="learned", fallback_thr=0.98),
                         stats=True)
        out[trained] = (idx.cpu().numpy(), st["n_fallback"])
    Zh = AHY.cpu().numpy()
    ref = mo.project(Zh, A)
    fg = p["phantom"]["labels"] >= 0
    agree = {t: float(np.mean(out[t][0][fg] == ref["idx"][fg])) for t in out}
    print(f"fallbacks untrained {out[False][1]} trained {out[True][1]} of {n}; "
          f"foreground agreement with exhaustive {agree}")
    # the gain: fewer voxels need the exhaustive search
    assert out[True][1] < out[False][1]
    # the contract: an accepted proposal has normalised correlation >= the threshold; any other
    # voxel carries the exhaustive answer
    gi = out[True][0]
    c = mo.correlation(Zh, A, gi)
    low = c < 0.98 - 1e-5
    near = c >= ref["s1"] - 1e-6
    assert np.all(near[low])
    # the edge rule (on by default): accepted proposals are local maxima over the grid
    assert out[True][1] < n
    assert_local_max(Zh, A, dic, gi)

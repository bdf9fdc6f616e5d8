"""Checks of the seeded input generators (not of the method): Bloch simulators against an
isochromat ensemble and the bSSFP steady-state closed form, grid sizes, masks, noise level."""
import numpy as np

import mrfgen
from mrfgen.bloch import epg_fisp, isochromat_fisp, bssfp
from mrfgen.sequence import param_grid


def test_epg_matches_isochromat_ensemble():
    a = mrfgen.flip_train(60)
    for t1, t2, b1 in [(800.0, 80.0, 1.0), (2500.0, 300.0, 0.7), (300.0, 30.0, 1.3)]:
        e = epg_fisp([t1], [t2], a, B1=b1)[0]
        i = isochromat_fisp(t1, t2, a, B1=b1)
        assert np.max(np.abs(e - i)) < 1e-12


def test_bssfp_steady_state_closed_form():
    """On resonance, alternating +-alpha, TE = TR/2: |M_ss| = sqrt(E2) sin a (1 - E1) /
    (1 - (E1 - E2) cos a - E1 E2), with E1, E2 over one TR."""
    a, T1, T2, TR = 50.0, 1000.0, 100.0, 10.0
    s = bssfp([T1], [T2], [0.0], np.full(4000, a))[0]
    E1, E2 = np.exp(-TR / T1), np.exp(-TR / T2)
    ar = np.deg2rad(a)
    ss = np.sqrt(E2) * np.sin(ar) * (1 - E1) / (1 - (E1 - E2) * np.cos(ar) - E1 * E2)
    assert abs(abs(s[-1]) - ss) < 1e-9


def test_grid_sizes_and_validity():
    for target in (2000, 1961, 2179):
        g = param_grid(target)
        d = g["params"].shape[0]
        assert abs(d - target) <= 0.02 * target
        assert np.all(g["params"][:, 1] < g["params"][:, 0])
    g = param_grid(1961, b0_hz=np.arange(-50, 51, 2.0))
    assert g["params"].shape[0] == 51 * param_grid(1961)["params"].shape[0]
    ca = g["cell_atom"]
    assert ca.max() == g["params"].shape[0] - 1


def test_masks_counts_and_center():
    m = mrfgen.line_masks(64, 30, 8.0, 1)
    assert np.all(m.sum(1) == 8)
    assert np.all(m[:, 0] == 1) and np.all(m[:, -1] == 1)   # DC and its neighbour kept


def test_noise_level():
    dic = mrfgen.make_dictionary(1)
    p = mrfgen.make_problem(1, dic=dic)
    q = mrfgen.make_problem(1, dic=dic, noiseless=True)
    xi = p["Y"].astype(np.complex128) - q["Y"]
    snr = 20 * np.log10(np.linalg.norm(q["Y"]) / np.linalg.norm(xi))
    assert abs(snr - 40.0) < 0.5
    assert np.all(xi[q["Y"] == 0][np.broadcast_to(
        p["masks"].T[:, None, :] == 0, q["Y"].shape)[q["Y"] == 0]] == 0)

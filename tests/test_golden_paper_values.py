"""Pins of the oracle and the input recipe to values the paper prints
(tests/golden/paper_values.txt, each with its passage): the 376-band source
grid and the visible range the decoder's resampling maps between (Sec. 3,
Fig. 1), Dec_T's layer sizes and K (Sec. 5.1, Eq. 10), and the epidermis of
the two-layer workload (Sec. 3)."""
import os

import numpy as np
import pytest

from oracle import decoder as dec_ref
from paper_2606_27604_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def _load():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("=", 1))
            vals[k] = float(v)
    return vals


@pytest.fixture(scope="module")
def pv():
    return _load()


def test_source_grid_is_the_papers(pv):
    n = int(pv["src_bands"])
    assert dec_ref.N_SRC == n
    nm = dec_ref.SRC_NM0 + dec_ref.SRC_STEP * np.arange(n)
    assert nm[0] == pv["src_nm_first"] and nm[-1] == pv["src_nm_last"]
    assert dec_ref.SRC_STEP == pv["src_nm_step"]


def test_visible_grid_spans_the_papers_visible_range(pv):
    assert dec_ref.DST_NM[0] == pv["vis_nm_first"]
    assert dec_ref.DST_NM[-1] == pv["vis_nm_last"]
    # every visible band lies on the source grid or halfway between two of its bands
    s = (dec_ref.DST_NM - pv["src_nm_first"]) / pv["src_nm_step"]
    assert np.all(np.abs(s * 2 - np.round(s * 2)) == 0)


def test_resampling_maps_the_papers_grid(pv):
    # A spectrum equal to its own wavelength on the paper's source grid is
    # carried by the linear resampling to the visible wavelengths exactly.
    n = int(pv["src_bands"])
    src = pv["src_nm_first"] + pv["src_nm_step"] * np.arange(n)
    out = dec_ref.resample_matrix() @ src
    np.testing.assert_allclose(out, dec_ref.DST_NM, rtol=0, atol=1e-9)


def test_dect_layer_sizes_and_K_are_the_papers(pv):
    W = inputs.decoder_weights(seed=4)
    h, L = int(pv["dect_hidden"]), int(pv["dect_layers"])
    shapes = [W[f"dec_t{l}"][0].shape for l in range(L)]
    assert shapes[0] == (h, int(pv["dect_in"]))
    for l in range(1, L - 1):
        assert shapes[l] == (h, h)
    assert shapes[-1] == (int(pv["dect_out"]), h)
    assert pv["dect_out"] == pv["src_bands"] * pv["K"] * pv["params_per_medium"]
    # Dec_T's input is p (Enc's output) next to R_d (Dec_R's output)
    assert pv["dect_in"] == pv["enc_out"] + pv["dec_r_out"]
    assert W["enc2"][0].shape[0] == int(pv["enc_out"])
    assert W["dec_r2"][0].shape[0] == int(pv["dec_r_out"])
    assert dec_ref.K == int(pv["K"])


def test_two_layer_workload_follows_the_papers_epidermis(pv):
    x = inputs.two_layer_batch(n_inst=512)
    d1_um = np.asarray(x.layer2[3], np.float64) * 1e3   # top-layer thickness, mm -> um
    assert d1_um.min() >= pv["epi_um_min"] - 1e-3 and d1_um.max() <= pv["epi_um_max"] + 1e-3
    # the synthetic top-layer g range covers Jacques' g(lambda) over the visible range
    lam = np.array([pv["vis_nm_first"], pv["vis_nm_last"]])
    g_j = pv["epi_g_intercept"] + pv["epi_g_slope_per_nm"] * lam
    g_top = np.asarray(x.g[0], np.float64)
    assert g_top.min() <= g_j.min() and g_top.max() >= g_j.max()

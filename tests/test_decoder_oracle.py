"""Pins of the decoder reference (oracle/decoder.py) against things other
than itself: the library's own bfloat16 matmul, the simplex constraint on
the weights (Sec. 5.1), the output ranges, exact resampling at shared
wavelengths, and the bf16 error bound."""
import numpy as np
import pytest

from oracle import decoder as dec
from paper_2606_27604_b300 import inputs


@pytest.fixture(scope="module")
def setup():
    W = inputs.decoder_weights(seed=4)
    rgb = inputs.rgb_texture(side=16, seed=4)
    return W, rgb


def test_weights_sum_to_one_and_ranges(setup):
    W, rgb = setup
    o = dec.decode(rgb, W)
    np.testing.assert_allclose(o["w"].sum(0), 1.0, atol=1e-12)
    assert np.all((o["alpha"] > 0) & (o["alpha"] < 1))
    assert np.all((o["g"] > 0) & (o["g"] < 1))
    assert np.all((o["sigma_t"] >= 1.0) & (o["sigma_t"] <= 1000.0))
    assert o["alpha"].shape == (3, 81 * rgb.shape[0])


def test_resampling_is_exact_on_shared_wavelengths(setup):
    W, rgb = setup
    o = dec.decode(rgb, W, return_intermediates=True)
    T = rgb.shape[0]
    z = o["logits"]
    a_src = 1.0 / (1.0 + np.exp(-z[..., 0]))          # [T][376][K]
    for j in (0, 2, 40, 80):                         # 380, 390, 580, 780 nm
        s = int((380 + 5 * j - 250) / 2)
        np.testing.assert_allclose(o["alpha"][:, j * T:(j + 1) * T], a_src[:, s, :].T,
                                   rtol=1e-14)
    for j in (1, 39):                                # half-way between two source bands
        s = int((380 + 5 * j - 250 - 1) / 2)
        np.testing.assert_allclose(o["alpha"][:, j * T:(j + 1) * T],
                                   0.5 * (a_src[:, s, :] + a_src[:, s + 1, :]).T, rtol=1e-14)


def test_layer_matches_library_bf16_matmul(setup):
    # One layer of the reference against torch's bfloat16 matmul (fp32
    # accumulate): agreement to the bf16 rounding of the output.
    import torch
    W, rgb = setup
    o = dec.decode(rgb, W, return_intermediates=True)
    Wm, b = W["dec_r1"]
    x = np.tanh(o["p"] @ W["dec_r0"][0].astype(np.float64).T + W["dec_r0"][1])
    xb = torch.from_numpy(x).to(torch.bfloat16)
    ref = (xb @ torch.from_numpy(Wm).to(torch.bfloat16).T).float().numpy() + b
    got = x.astype(np.float64)
    got = dec._bf16(got) @ Wm.astype(np.float64).T + b
    np.testing.assert_allclose(got, ref, atol=2 ** -7 * np.abs(ref).max() + 1e-6)


def test_bf16_activation_error_is_within_bound(setup):
    # The bf16-stored pipeline stays within c * sqrt(fan_in) * 2^-8 of the
    # float64 one on the sigmoid outputs (|sigmoid'| <= 1/4).
    W, rgb = setup
    a = dec.decode(rgb, W)
    b = dec.decode(rgb, W, bf16_activations=True)
    for k in ("alpha", "g", "w"):
        assert np.max(np.abs(a[k] - b[k])) < 4 * np.sqrt(768) * 2 ** -8 * 0.25

"""Pins of the decoder reference (oracle/decoder.py, paper Sec. 5.1, Eq. 10)
against things other than itself:

* an independent float64 network built from torch.nn library layers, with
  the layer order, the Dec_T input order (p, then R_d) and the output layout
  (index band*12 + k*4 + c, channels alpha, g, sigma_t, w) taken from the
  ABI header's description, and the 2-nm -> 5-nm resampling done with
  numpy's own linear interpolation;
* hand-computable networks (zero weights except a few unit entries) whose
  outputs have a closed form: sigma_t = 10^(3 s), the softmax over the
  media, a linear spectrum reproduced exactly by the resampling, and a
  single path through Dec_T that fixes the [out][in] orientation of every
  weight and the input concatenation order;
* the simplex constraint on the weights, the output ranges and the bf16
  error bound.
"""
import numpy as np
import pytest

from oracle import decoder as dec
from paper_2606_27604_b300 import inputs

WIDTHS = {"enc": (3, 256, 256, 5), "dec_r": (5, 512, 512, 376),
          "dec_t": (381, 768, 768, 768, 376 * 12)}
N_SRC = 376


@pytest.fixture(scope="module")
def setup():
    W = inputs.decoder_weights(seed=4)
    rgb = inputs.rgb_texture(side=16, seed=4)
    return W, rgb


# ------------------------------------------------ independent torch network --
def _torch_net(W, net, hidden, out_act, bf16):
    """torch.nn.Sequential of Linear layers with `hidden` between them and
    `out_act` (or nothing) after the last; optional bf16 rounding of every
    stored activation, as the GPU stores them."""
    import torch

    class RoundBF16(torch.nn.Module):
        def forward(self, x):
            return x.to(torch.bfloat16).double()

    dims = WIDTHS[net]
    mods = []
    for l in range(len(dims) - 1):
        lin = torch.nn.Linear(dims[l], dims[l + 1]).double()
        Wl, bl = W[f"{net}{l}"]
        assert Wl.shape == (dims[l + 1], dims[l])       # [out][in]
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(np.asarray(Wl, np.float64)))
            lin.bias.copy_(torch.from_numpy(np.asarray(bl, np.float64)))
        mods.append(lin)
        last = l == len(dims) - 2
        if not last:
            mods.append(hidden())
        elif out_act is not None:
            mods.append(out_act())
        if bf16 and not (last and out_act is None):
            mods.append(RoundBF16())
    return torch.nn.Sequential(*mods)


def _torch_decode(rgb, W, bf16=False):
    import torch
    enc = _torch_net(W, "enc", torch.nn.Tanh, torch.nn.Sigmoid, bf16)
    dr = _torch_net(W, "dec_r", torch.nn.Tanh, torch.nn.Sigmoid, bf16)
    dt = _torch_net(W, "dec_t", torch.nn.Tanh, None, bf16)
    with torch.no_grad():
        x = torch.from_numpy(np.asarray(rgb, np.float64))
        p = enc(x)
        rd = dr(p)
        z = dt(torch.cat([p, rd], dim=1)).numpy()       # Dec_T(p, R_d)
    T = x.shape[0]
    # output index band*12 + k*4 + c
    idx = lambda c: (np.arange(N_SRC)[None, :] * 12 + np.arange(3)[:, None] * 4 + c)  # [k][band]
    src = {}
    sig = lambda v: 1.0 / (1.0 + np.exp(-v))
    src["alpha"] = sig(z[:, idx(0)])                    # [T][k][band]
    src["g"] = sig(z[:, idx(1)])
    src["sigma_t"] = np.power(10.0, 3.0 * sig(z[:, idx(2)]))
    lw = torch.from_numpy(z[:, idx(3)])
    src["w"] = torch.softmax(lw, dim=1).numpy()
    # linear interpolation from 250 + 2 s nm to 380 + 5 j nm (numpy's interp)
    nm_src = 250.0 + 2.0 * np.arange(N_SRC)
    nm_dst = 380.0 + 5.0 * np.arange(81)
    out = {}
    for name, v in src.items():
        r = np.empty((3, 81, T))
        for k in range(3):
            for t in range(T):
                r[k, :, t] = np.interp(nm_dst, nm_src, v[t, k])
        out[name] = r.reshape(3, 81 * T)                # band-major instances
    return out, p.numpy(), rd.numpy(), z


@pytest.mark.parametrize("bf16", [False, True])
def test_reference_equals_independent_library_network(setup, bf16):
    W, rgb = setup
    ref, p, rd, z = _torch_decode(rgb, W, bf16=bf16)
    o = dec.decode(rgb, W, bf16_activations=bf16, return_intermediates=True)
    np.testing.assert_allclose(o["p"], p, rtol=0, atol=1e-12)
    np.testing.assert_allclose(o["R_d"], rd, rtol=0, atol=1e-12)
    np.testing.assert_allclose(o["logits"].reshape(rgb.shape[0], -1), z, rtol=0, atol=1e-10)
    for k in ("alpha", "g", "w"):
        np.testing.assert_allclose(o[k], ref[k], rtol=0, atol=1e-12, err_msg=k)
    np.testing.assert_allclose(o["sigma_t"], ref["sigma_t"], rtol=1e-12, atol=0)


# ------------------------------------------------ hand-computable networks --
def _zero_weights():
    W = {}
    for net, dims in WIDTHS.items():
        for l in range(len(dims) - 1):
            W[f"{net}{l}"] = (np.zeros((dims[l + 1], dims[l]), np.float32),
                              np.zeros(dims[l + 1], np.float32))
    return W


def _logit(y):
    return np.log(y / (1.0 - y))


def test_closed_form_outputs_from_biases_alone():
    # With every weight zero the last layer's bias is the logit vector, so:
    #  alpha (medium k) = a0 + a1 s on source band s: a linear spectrum, which
    #    the linear resampling reproduces exactly at 380 + 5 j nm, i.e. at
    #    source position s = 65 + 2.5 j;
    #  g = 0.8 everywhere; sigma_t = 10^(3 s) with s = 1/2, 1/3, 2/3 for the
    #    three media: 10^1.5, 10, 100 mm^-1;
    #  w = softmax(0, ln 2, ln 5) = (1/8, 2/8, 5/8).
    W = _zero_weights()
    b = np.zeros(N_SRC * 12)
    s = np.arange(N_SRC)
    a0, a1 = [0.1, 0.2, 0.3], [1e-3, 1.5e-3, 5e-4]
    sig_s = [0.5, 1.0 / 3.0, 2.0 / 3.0]
    lw = [0.0, np.log(2.0), np.log(5.0)]
    for k in range(3):
        b[s * 12 + k * 4 + 0] = _logit(a0[k] + a1[k] * s)
        b[s * 12 + k * 4 + 1] = _logit(0.8)
        b[s * 12 + k * 4 + 2] = _logit(sig_s[k])
        b[s * 12 + k * 4 + 3] = lw[k]
    W["dec_t3"] = (W["dec_t3"][0], b)
    rgb = np.array([[0.3, 0.5, 0.7]], np.float32)
    o = dec.decode(rgb, W, return_intermediates=True)
    j = np.arange(81)
    for k in range(3):
        np.testing.assert_allclose(o["alpha"][k], a0[k] + a1[k] * (65 + 2.5 * j), rtol=1e-12)
        np.testing.assert_allclose(o["g"][k], 0.8, rtol=1e-12)
    np.testing.assert_allclose(o["sigma_t"][0], 10 ** 1.5, rtol=1e-12)
    np.testing.assert_allclose(o["sigma_t"][1], 10.0, rtol=1e-12)
    np.testing.assert_allclose(o["sigma_t"][2], 100.0, rtol=1e-12)
    np.testing.assert_allclose(o["w"][:, 0], [1 / 8, 2 / 8, 5 / 8], rtol=1e-12)
    # the intermediate codes are the sigmoids of their biases (zero weights)
    np.testing.assert_allclose(o["p"], 0.5, rtol=0, atol=0)
    np.testing.assert_allclose(o["R_d"], 0.5, rtol=0, atol=0)


def test_single_path_fixes_orientation_and_concat_order():
    # One unit path through the encoder and Dec_T, every weight an
    # off-diagonal entry W[out][in] = 1: rgb channel 2 -> enc hidden 9 ->
    # enc hidden 4 -> p[3] -> Dec_T input column 3 (p comes first) -> hidden
    # 7 -> 11 -> 5 -> logit of (source band 65, medium 1, channel alpha).
    # A transposed weight, or R_d ahead of p, breaks the path and the output
    # falls back to sigmoid of the bias.
    W = _zero_weights()

    def put(name, o, i, v=1.0):
        Wm, bm = W[name]
        Wm = Wm.copy()
        Wm[o, i] = v
        W[name] = (Wm, bm)

    put("enc0", 9, 2)
    put("enc1", 4, 9)
    put("enc2", 3, 4)
    put("dec_t0", 7, 3)
    put("dec_t1", 11, 7)
    put("dec_t2", 5, 11)
    row = 65 * 12 + 1 * 4 + 0
    put("dec_t3", row, 5)
    # R_d is sigmoid(0.9) everywhere, p otherwise sigmoid(0): distinct values
    W["dec_r2"] = (W["dec_r2"][0], np.full(N_SRC, 0.9, np.float32))
    x = 0.7
    rgb = np.array([[0.2, 0.4, x]], np.float32)
    o = dec.decode(rgb, W)
    sig = lambda v: 1.0 / (1.0 + np.exp(-v))
    p3 = sig(np.tanh(np.tanh(np.float64(np.float32(x)))))
    want = sig(np.tanh(np.tanh(np.tanh(p3))))
    np.testing.assert_allclose(o["alpha"][1, 0], want, rtol=1e-13)   # visible band 0 = 380 nm
    assert abs(want - 0.5) > 0.1
    # every other (band, medium) alpha is sigmoid(0) = 1/2
    a = o["alpha"].copy()
    a[1, 0] = 0.5
    np.testing.assert_allclose(a, 0.5, rtol=0, atol=0)


# --------------------------------------------------------------- invariants --
def test_weights_sum_to_one_and_ranges(setup):
    W, rgb = setup
    o = dec.decode(rgb, W)
    np.testing.assert_allclose(o["w"].sum(0), 1.0, atol=1e-12)
    assert np.all((o["alpha"] > 0) & (o["alpha"] < 1))
    assert np.all((o["g"] > 0) & (o["g"] < 1))
    assert np.all((o["sigma_t"] >= 1.0) & (o["sigma_t"] <= 1000.0))
    assert o["alpha"].shape == (3, 81 * rgb.shape[0])


def test_bf16_activation_error_is_within_bound(setup):
    # The bf16-stored pipeline stays within c * sqrt(fan_in) * 2^-8 of the
    # float64 one on the sigmoid outputs (|sigmoid'| <= 1/4).
    W, rgb = setup
    a = dec.decode(rgb, W)
    b = dec.decode(rgb, W, bf16_activations=True)
    for k in ("alpha", "g", "w"):
        assert np.max(np.abs(a[k] - b[k])) < 4 * np.sqrt(768) * 2 ** -8 * 0.25

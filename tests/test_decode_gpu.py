"""The tensor-core decoder (sss_decode) against the FP64 decoder reference.

The reference rounds stored activations to bfloat16 where the GPU stores
them in bfloat16; the remaining differences are FP32 accumulation order and
the hardware tanh, which can move a stored activation by one bf16 step
(2^-8 relative).  Propagated through a layer that is about 2^-8 on the
pre-activations, i.e. <= 2^-8/4 on sigmoid outputs and 3 ln(10) 2^-8/4
relative on sigma_t = 10^(3 s); the bounds below allow four times that.
"""
import numpy as np
import pytest

from oracle import decoder as dec_ref
from paper_2606_27604_b300 import inputs

pytestmark = pytest.mark.gpu

TOL_ABS = 4 * 2 ** -8 / 4          # alpha, g, w
TOL_SIG_REL = 4 * 3 * np.log(10) * 2 ** -8 / 4


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_27604_b300 import api as a
    return a


def _run(api, rgb, W):
    import torch
    packed = api.decoder_pack(W)
    out = api.decode(torch.from_numpy(rgb).cuda(), packed)
    torch.cuda.synchronize()
    code, flags = api.read_status(out["_workspace"])
    return {k: v.cpu().numpy() for k, v in out.items() if not k.startswith("_")}, code, flags


@pytest.mark.parametrize("side", [1, 37])   # one texel; a ragged 1369-texel tile tail
def test_decode_matches_reference(api, side):
    W = inputs.decoder_weights(seed=4)
    rgb = inputs.rgb_texture(side=side, seed=4)
    g, code, flags = _run(api, rgb, W)
    assert code == 0 and flags == 0
    r = dec_ref.decode(rgb, W, bf16_activations=True)
    for k in ("alpha", "g", "w"):
        err = np.abs(g[k] - r[k])
        print(k, "max abs err", err.max())
        assert err.max() <= TOL_ABS, k
    rel = np.abs(g["sigma_t"] / r["sigma_t"] - 1)
    print("sigma_t max rel err", rel.max())
    assert rel.max() <= TOL_SIG_REL
    np.testing.assert_allclose(g["w"].sum(0), 1.0, atol=1e-5)
    # and against the all-float64 pipeline, within the bf16 error bound
    r64 = dec_ref.decode(rgb, W)
    assert np.abs(g["alpha"] - r64["alpha"]).max() < 4 * np.sqrt(768) * 2 ** -8 * 0.25


def test_decode_matches_reference_at_full_size_sampled(api):
    # 600 x 600 = 360,000 texels: 2813 row tiles of 128 (the last one ragged),
    # so every layer's persistent CTAs walk many tiles each and both TMEM
    # accumulators and the accumulator-release wait run.  Decoding is row-
    # independent, so the FP64 reference decodes only the sampled rows:
    # every 173rd row, the whole ragged last tile and the rows around tile
    # boundaries.
    side = 600
    T = side * side
    import torch
    W = inputs.decoder_weights(seed=4)
    rgb = inputs.rgb_texture(side=side, seed=7)
    out = api.decode(torch.from_numpy(rgb).cuda(), api.decoder_pack(W))
    torch.cuda.synchronize()
    code, flags = api.read_status(out["_workspace"])
    assert code == 0 and flags == 0
    last_tile = np.arange((T - 1) // 128 * 128, T)
    edges = np.concatenate([np.arange(b - 2, b + 2) for b in range(128 * 500, T, 128 * 500)])
    rows = np.unique(np.concatenate([np.arange(0, T, 173), last_tile, edges]))
    assert len(rows) > 2000
    r = dec_ref.decode(rgb[rows], W, bf16_activations=True)
    n = len(rows)
    cols = (np.arange(81)[:, None] * T + rows[None, :]).reshape(-1)   # band-major
    ci = torch.from_numpy(cols).cuda()
    g = {k: out[k][:, ci].cpu().numpy() for k in ("alpha", "g", "sigma_t", "w")}
    for k in ("alpha", "g", "w"):
        err = np.abs(g[k] - r[k])
        print(k, "max abs err", err.max())
        assert err.max() <= TOL_ABS, k
    rel = np.abs(g["sigma_t"] / r["sigma_t"] - 1)
    print("sigma_t max rel err", rel.max())
    assert rel.max() <= TOL_SIG_REL
    assert r["alpha"].shape == (3, 81 * n)
    # the weights of every texel and band sum to one (all of them, on the GPU)
    assert float((out["w"].sum(0) - 1.0).abs().max()) <= 1e-5


def test_decode_feeds_the_walk(api):
    # the decoder's output is valid walk input (instances band-major)
    import torch
    W = inputs.decoder_weights(seed=4)
    rgb = inputs.rgb_texture(side=8, seed=5)
    packed = api.decoder_pack(W)
    out = api.decode(torch.from_numpy(rgb).cuda(), packed)
    m = api.Media(out["alpha"], out["sigma_t"], out["g"], out["w"], None, 256, None, 1.4)
    r = api.walk(m, api.WalkOptions(seed=1004))
    torch.cuda.synchronize()
    code, flags = api.read_status(r["_workspace"])
    assert code == 0, flags
    assert torch.all(r["R"] > 0) and torch.all(r["R"] < 1)


def test_bounded_wait_gives_up_and_the_context_survives(api):
    # Failure detection without a fault: a wait on an mbarrier phase that
    # nothing completes, with the pipeline's own bounded wait and a ~1 ms
    # limit, records the timeout in the status word and returns; the next
    # decode on the same context runs clean.
    import torch
    status = torch.zeros(64, dtype=torch.int32, device="cuda")
    api.selftest_bounded_wait(status, 2_000_000)
    torch.cuda.synchronize()
    code, flags = api.read_status(status)
    assert flags & 0x10 and code == 8, (code, flags)
    W = inputs.decoder_weights(seed=4)
    g, code, flags = _run(api, inputs.rgb_texture(side=4, seed=4), W)
    assert code == 0 and flags == 0
    assert np.isfinite(g["alpha"]).all()
    with pytest.raises(api.SSSError):
        api.selftest_bounded_wait(status, 0)

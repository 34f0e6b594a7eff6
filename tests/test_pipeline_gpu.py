"""The full pipeline on the GPU: RGB albedo -> tensor-core decoder -> batched
walk (paper Sec. 5.1 feeding Sec. 4.1 / Sec. 7), against the FP64 oracle
pipeline (oracle decoder with bf16-rounded activations -> oracle walk) on
the same Philox streams, at a size the oracle finishes in seconds.

Two checks:
  * the walk leg alone: the GPU walk and the oracle walk on the parameters
    the GPU decoder produced (float32, identical on both sides), held to
    the same-stream bound;
  * end to end: the decoder's own rounding (bf16 operands, FP32
    accumulation, within the decoder tolerance) moves a few paths, so R
    from the GPU pipeline and from the oracle pipeline must agree within 4
    standard errors, with a median relative error below 1e-3.
"""
import numpy as np
import pytest

from oracle import decoder as dec_ref
from paper_2606_27604_b300 import inputs
from gpu_helpers import compare_same_stream, run_oracle

pytestmark = pytest.mark.gpu

SIDE = 8          # 64 texels x 81 bands
N_PATHS = 512


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_27604_b300 import api as a
    return a


@pytest.fixture(scope="module")
def pipeline(api):
    import torch
    W = inputs.decoder_weights(seed=4)
    rgb = inputs.rgb_texture(side=SIDE, seed=11)
    dec = api.decode(torch.from_numpy(rgb).cuda(), api.decoder_pack(W))
    m = api.Media(dec["alpha"], dec["sigma_t"], dec["g"], dec["w"], None, N_PATHS, None, 1.4)
    o = api.WalkOptions(nbins=64, r_max_mm=10.0, seed=1004)
    out = api.walk(m, o)
    torch.cuda.synchronize()
    assert api.read_status(dec["_workspace"])[0] == 0
    assert api.read_status(out["_workspace"])[0] == 0
    g = {k: v.cpu().numpy() for k, v in out.items() if not k.startswith("_")}
    params = {k: dec[k].cpu().numpy() for k in ("alpha", "sigma_t", "g", "w")}
    return W, rgb, o, g, params


def test_walk_leg_matches_oracle_on_the_decoded_parameters(api, pipeline):
    W, rgb, o, g, prm = pipeline
    n = prm["alpha"].shape[1]
    x = inputs.WalkInputs(prm["alpha"], prm["sigma_t"], prm["g"], prm["w"],
                          np.full(n, N_PATHS, np.uint32), None, 1.4)
    r = run_oracle(x, o)
    worst, where = compare_same_stream(g, r, x.n_paths, r["steps"])
    print("walk leg same-stream worst ratio", worst, where)
    assert worst <= 1.0, where


def test_pipeline_matches_the_oracle_pipeline(api, pipeline):
    import oracle
    W, rgb, o, g, prm = pipeline
    ref = dec_ref.decode(rgb, W, bf16_activations=True)
    n = ref["alpha"].shape[1]
    r = oracle.walk(ref["alpha"].astype(np.float32), ref["sigma_t"].astype(np.float32),
                    ref["g"].astype(np.float32), ref["w"].astype(np.float32),
                    np.full(n, N_PATHS, np.uint32), None, 1.4,
                    oracle.OracleOpts(nbins=64, r_max_mm=10.0, seed=1004))
    se = np.sqrt(r["se_R"] ** 2 + g["stderr_R"] ** 2)
    z = (g["R"] - r["R"]) / np.maximum(se, 1e-12)
    rel = np.abs(g["R"] - r["R"]) / r["R"]
    print("pipeline: max |z|", np.abs(z).max(), "median rel err", np.median(rel))
    assert np.all(np.abs(z) <= 4.0)
    assert np.median(rel) < 1e-3

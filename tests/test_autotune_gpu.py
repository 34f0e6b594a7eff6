"""The launch-shape autotuner picks a shape; results do not depend on it."""
import numpy as np
import pytest

from paper_2606_27604_b300 import inputs

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_shape_and_keeps_results(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_27604_b300 import api, autotune
    x = inputs.spectral_field(n_texels=8, param_seed=3, n_paths=2048)
    m = api.Media.from_inputs(x)
    o = api.WalkOptions(seed=12)
    cache = str(tmp_path / "tune.json")
    cands = autotune.CANDIDATES[:4]
    ot = autotune.tune(m, o, cache_path=cache, candidates=cands, reps=1)
    assert {"block_threads": ot.block_threads, "unit_paths": ot.unit_paths,
            "regroup": ot.regroup} in cands
    again = autotune.tune(m, o, cache_path=cache, candidates=cands, reps=1)  # cached
    assert again == ot
    a = api.walk(m, o, raw=True)["raw"].cpu().numpy()
    b = api.walk(m, ot, raw=True)["raw"].cpu().numpy()
    np.testing.assert_array_equal(a, b)

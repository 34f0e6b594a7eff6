"""Scale-independent LUTs (Sec. 4.2) built with the batched walk."""
import numpy as np
import pytest

import oracle
from paper_2606_27604_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lutmod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_27604_b300 import lut
    return lut


def test_lut_matches_oracle_on_a_small_grid(lutmod):
    alphas = np.array([0.3, 0.8, 0.95, 0.999])
    gs = np.array([0.0, 0.5, 0.9])
    L = lutmod.build(alphas, gs, n_paths=1 << 14, nbins=32, r_max=16.0, n_rel=1.4, seed=7)
    a, s, g, w = lutmod.grid_inputs(alphas, gs)
    r = oracle.walk(a, s, g, w, np.full(a.shape[1], 1 << 14, np.uint32), None, 1.4,
                    oracle.OracleOpts(nbins=32, r_max_mm=16.0, seed=7))
    tol = 1e-5 * np.abs(r["R"]) + (8 + 4e-6 * (1 << 14) * r["steps"]) / (1 << 14)
    assert np.all(np.abs(L.R.reshape(-1) - r["R"]) <= tol)
    bins = L.P.reshape(-1, 32) * L.R.reshape(-1)[:, None]
    tolb = 1e-5 * r["bins"] + (8 + 4e-6 * (1 << 14) * r["steps"][:, None]) / (1 << 14)
    assert np.all(np.abs(bins - r["bins"]) <= tolb)
    assert np.all(L.P.sum(-1) <= 1.0 + 1e-12)


def test_extinction_rescales_the_radial_axis_exactly(lutmod):
    # Eq. 5: the walk at sigma_t = 4 with r_max / 4 gives the sigma_t = 1
    # table bit for bit (a power-of-two scale is exact in binary32)
    import torch
    from paper_2606_27604_b300 import api
    alphas, gs = np.array([0.6, 0.97]), np.array([0.2, 0.8])
    L = lutmod.build(alphas, gs, n_paths=1 << 14, nbins=32, r_max=16.0, seed=9)
    a, s, g, w = lutmod.grid_inputs(alphas, gs)
    t = lambda arr: torch.from_numpy(arr).cuda()
    m = api.Media(t(a), t(s * 4), t(g), t(w), None, 1 << 14, None, 1.4)
    o = api.WalkOptions(nbins=32, r_max_mm=4.0, seed=9)
    out = api.alloc_tallies(m, o)
    out["profile"] = torch.empty(m.n_inst, 32, dtype=torch.float64, device="cuda")
    out = api.walk(m, o, out=out)
    R4 = out["R"].cpu().numpy()
    np.testing.assert_array_equal(R4, L.R.reshape(-1))
    np.testing.assert_array_equal(out["profile"].cpu().numpy(), L.P.reshape(-1, 32))
    # the profile output is bins / R (Eq. 3), up to the rounding of the quotient
    np.testing.assert_allclose(out["profile"].cpu().numpy(),
                               out["bins"].cpu().numpy() / R4[:, None], rtol=4e-16, atol=0)

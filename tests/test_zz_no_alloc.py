"""sss_walk_noalloc, the forward walk for callers that cannot allocate
device memory (hosts that own every device allocation through their own
pool, or threads where a cudaMalloc is not allowed).  It must give what
sss_walk gives, call after call, although every call reuses one built-in
scratch array.  Collected last so a failure here comes after every other
test has run."""
import numpy as np
import pytest

from paper_2606_27604_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_27604_b300 import api as a
    return a


def _compare(api, x, o):
    import torch
    m = api.Media.from_inputs(x)
    ref = api.walk(m, o, raw=True)
    torch.cuda.synchronize()
    code_ref, flags_ref = api.read_status(ref["_workspace"])
    out = api.alloc_tallies(m, o, raw=True)
    for v in out.values():
        v.fill_(-1)  # anything the call fails to write shows up
    code, flags = api.walk_noalloc(m, o, out)
    assert code == 0 and code_ref == 0 and flags == flags_ref == 0, (code, flags)
    np.testing.assert_array_equal(out["raw"].cpu().numpy(), ref["raw"].cpu().numpy())
    for k in ("R", "T", "A", "bins", "overflow", "R_k", "R1", "stderr_R", "stderr_bins",
              "steps"):
        np.testing.assert_allclose(out[k].cpu().numpy(), ref[k].cpu().numpy(), rtol=1e-12,
                                   atol=0, err_msg=k)


def test_noalloc_matches_walk_on_two_calls_in_a_row(api):
    # two different problems back to back: the second must not see the
    # first one's accumulators left in the shared scratch array
    a = inputs.spectral_field(n_texels=4, param_seed=21, n_paths=3000)
    b = inputs.uneven_batch(n_inst=200, param_seed=22, log2_min=8, log2_max=12)
    _compare(api, a, api.WalkOptions(nbins=64, r_max_mm=10.0, seed=5))
    _compare(api, b, api.WalkOptions(nbins=32, r_max_mm=4.0, seed=6))


def test_noalloc_without_a_flag_word_then_the_stream_status(api):
    # status_flags = NULL: the call only enqueues; the device status of its
    # scratch is then read through the per-stream status call
    import torch
    x = inputs.spectral_field(n_texels=3, param_seed=23, n_paths=2000)
    o = api.WalkOptions(nbins=48, r_max_mm=8.0, seed=7)
    m = api.Media.from_inputs(x)
    ref = api.walk(m, o, raw=True)
    out = api.alloc_tallies(m, o, raw=True)
    code, flags = api.walk_noalloc(m, o, out, read_flags=False)
    assert code == 0 and flags is None
    code, flags = api.last_device_status()
    assert code == 0 and flags == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out["raw"].cpu().numpy(), ref["raw"].cpu().numpy())


def test_noalloc_hero_and_no_sumsq_layouts(api):
    # the other accumulator layouts: hero-wavelength groups (a slot holds
    # three members' words) and tallies without squared weights
    x = inputs.spectral_field(n_texels=2, param_seed=24, n_paths=1500)
    _compare(api, x, api.WalkOptions(nbins=32, r_max_mm=6.0, seed=8, hero_bands=3,
                                     hero_texel_bands=81))
    o = api.WalkOptions(nbins=40, r_max_mm=7.0, seed=9, want_sumsq=0)
    import torch
    m = api.Media.from_inputs(x)
    ref = api.walk(m, o, raw=True)
    out = api.alloc_tallies(m, o, raw=True)
    code, flags = api.walk_noalloc(m, o, out)
    assert code == 0 and flags == 0
    np.testing.assert_array_equal(out["raw"].cpu().numpy(), ref["raw"].cpu().numpy())


def test_noalloc_rejects_problems_beyond_its_scratch(api):
    x = inputs.spectral_field(n_texels=256, param_seed=1, n_paths=16)  # 20736 instances
    m = api.Media.from_inputs(x)
    o = api.WalkOptions(nbins=64)
    assert api.workspace_bytes(m, o) > api.NOALLOC_SCRATCH_BYTES
    out = api.alloc_tallies(m, o)
    code, _ = api.walk_noalloc(m, o, out)
    assert code == 9  # SSS_ERR_TOO_LARGE

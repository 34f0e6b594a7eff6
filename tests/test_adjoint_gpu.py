"""Path-replay adjoint (sss_walk_bwd) on the GPU, through the C ABI.

Checked against the oracle's score-function gradient on the same Philox
streams, against common-random-number finite differences of the GPU forward
walk, against closed forms, and through the torch.autograd.Function.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import hfunction as hf
from paper_2606_27604_b300 import inputs
from gpu_helpers import to_oracle_opts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_27604_b300 import api as a
    return a


def _grads_gpu(api, x, o, **g):
    import torch
    m = api.Media.from_inputs(x)
    tg = {k: torch.from_numpy(np.ascontiguousarray(v, np.float64)).cuda()
          for k, v in g.items() if v is not None}
    d = api.walk_bwd(m, o, **tg)
    torch.cuda.synchronize()
    code, flags = api.read_status(d["_workspace"])
    return {k: v.cpu().numpy() for k, v in d.items() if not k.startswith("_")}, code, flags


def _upstream(x, nbins, seed=0):
    rng = np.random.default_rng(seed)
    n = x.n_inst
    return dict(grad_R=rng.normal(size=n), grad_bins=rng.normal(size=(n, nbins)),
                grad_R_k=rng.normal(size=(n, x.K)))


@pytest.mark.parametrize("select_pdf", [0, 1])
def test_adjoint_matches_oracle_score_gradient(api, select_pdf):
    # select_pdf = 1: uniform medium choice, whose weight K w_k / sum(w)
    # rides on the path weight, so the same score terms apply
    x = inputs.spectral_field(n_texels=3, param_seed=3, n_paths=8192)
    o = api.WalkOptions(nbins=64, r_max_mm=10.0, seed=1003, select_pdf=select_pdf)
    up = _upstream(x, 64)
    g, code, flags = _grads_gpu(api, x, o, **up)
    assert code == 0 and flags == 0
    r = oracle.walk_grad(x.alpha, x.sigma_t, x.g, x.w, x.n_paths, None, x.n_rel,
                         to_oracle_opts(o), **up)
    for k in ("d_alpha", "d_sigma_t", "d_g", "d_w"):
        a, b, se = g[k], r[k], r["se_" + k]
        # statistical bar and the tighter same-stream bound
        assert np.all(np.abs(a - b) <= 4 * math.sqrt(2) * se + 1e-12), k
        tight = 1e-4 * np.abs(b) + 0.25 * se + 1e-12
        ratio = np.abs(a - b) / tight
        print(k, "worst same-stream ratio", ratio.max())
        assert ratio.max() <= 1.0, k


def test_two_layer_adjoint_matches_oracle(api):
    # two-layer slabs: the top-layer (mixture) gradients take only the
    # top layer's part of each path and the second layer's optics get their
    # own; same-stream parity with the oracle's score gradient for all of
    # them, and a central difference in alpha2 without roulette
    x = inputs.two_layer_batch(n_inst=48, param_seed=8, n_paths=1 << 13)
    o = api.WalkOptions(nbins=32, r_max_mm=10.0, seed=1013)
    up = _upstream(x, 32, seed=5)
    g, code, flags = _grads_gpu(api, x, o, **up)
    assert code == 0 and flags == 0
    r = oracle.walk_grad(x.alpha, x.sigma_t, x.g, x.w, x.n_paths, None, x.n_rel,
                         to_oracle_opts(o), layer2=x.layer2, **up)
    for k in ("d_alpha", "d_sigma_t", "d_g", "d_w", "d_alpha2", "d_sigma_t2", "d_g2"):
        a, b, se = g[k], r[k], r["se_" + k]
        assert np.all(np.abs(a - b) <= 4 * math.sqrt(2) * se + 1e-12), k
        tight = 1e-4 * np.abs(b) + 0.25 * se + 1e-12
        ratio = np.abs(a - b) / tight
        print("two-layer", k, "worst same-stream ratio", ratio.max())
        assert ratio.max() <= 1.0, k
    # alpha2: without roulette the paths do not depend on the albedos (a
    # path that reaches the step cap is dropped alike by both estimates)
    import torch
    o0 = api.WalkOptions(nbins=32, r_max_mm=10.0, seed=1014, rr_threshold=0.0)
    gs, code, _ = _grads_gpu(api, x, o0, grad_R=np.ones(x.n_inst))
    assert code in (0, 4)   # OK or STEP_LIMIT
    # steps that keep alpha2 +- h inside [0, 1] and small against the path
    # length: R depends on alpha2 through alpha2^n with n up to thousands, so
    # the central difference is accurate only for n h << 1
    f0 = api.walk(api.Media.from_inputs(x), o0)
    torch.cuda.synchronize()
    steps = f0["steps"].cpu().numpy()
    h = np.minimum(np.minimum(1e-3, 0.5 * (1 - x.layer2[0].astype(np.float64))),
                   0.05 / np.maximum(steps, 1.0)).astype(np.float32)
    Rs, a2s = [], []
    for sgn in (-1, 1):
        xs = x.subset(np.arange(x.n_inst))
        a2 = (x.layer2[0] + np.float32(sgn) * h).astype(np.float32)
        assert np.all((a2 >= 0) & (a2 <= 1))
        xs.layer2 = (a2, *x.layer2[1:])
        f = api.walk(api.Media.from_inputs(xs), o0)
        torch.cuda.synchronize()
        assert api.read_status(f["_workspace"])[0] in (0, 4)
        Rs.append(f["R"].cpu().numpy())
        a2s.append(a2.astype(np.float64))
    fd = (Rs[1] - Rs[0]) / (a2s[1] - a2s[0])
    err = np.abs(gs["d_alpha2"] - fd)
    print("d R / d alpha2: max |score - central difference|", err.max(),
          "max |fd|", np.abs(fd).max())
    assert np.all(err <= 2e-3 * np.abs(fd) + 1e-4)


def test_alpha_gradient_equals_crn_finite_difference(api):
    # Roulette off: path geometry does not depend on alpha, so the forward
    # estimate is a polynomial in alpha and the replay gives its derivative.
    # Central differences at h and h/2, Richardson-combined to cancel the
    # h^2 term (paths with hundreds of collisions have large curvature).
    x = inputs.spectral_field(n_texels=2, param_seed=8, n_paths=4096)
    x.alpha[:] = np.minimum(x.alpha, np.float32(0.99))
    o = api.WalkOptions(nbins=32, r_max_mm=8.0, seed=4, rr_threshold=0.0, max_steps=4096)
    g, code, _ = _grads_gpu(api, x, o, grad_R=np.ones(x.n_inst))

    def fd(k, h):
        xp = x.subset(np.arange(x.n_inst)); xm = x.subset(np.arange(x.n_inst))
        xp.alpha[k] += np.float32(h); xm.alpha[k] -= np.float32(h)
        step = xp.alpha[k].astype(np.float64) - xm.alpha[k].astype(np.float64)
        Rp = api.walk(api.Media.from_inputs(xp), o)["R"].cpu().numpy()
        Rm = api.walk(api.Media.from_inputs(xm), o)["R"].cpu().numpy()
        return (Rp - Rm) / step

    for k in range(3):
        f1, f2 = fd(k, 4e-4), fd(k, 2e-4)
        rich = (4.0 * f2 - f1) / 3.0
        np.testing.assert_allclose(g["d_alpha"][k], rich, rtol=2e-3, atol=2e-6)


def test_alpha_gradient_matches_h_function_derivative(api):
    x = inputs.single_wavelength(n_paths=1 << 22).subset(np.array([2, 5]))  # alpha 0.5, 0.9
    o = api.WalkOptions(nbins=32, r_max_mm=10.0, seed=21)
    g, code, _ = _grads_gpu(api, x, o, grad_R=np.ones(2))
    xs = x.subset(np.arange(2)); xs.n_paths = np.full(2, 1 << 16, np.uint32)
    r = oracle.walk_grad(xs.alpha, xs.sigma_t, xs.g, xs.w, xs.n_paths, None, 1.0,
                         to_oracle_opts(o), grad_R=np.ones(2))
    se = np.sqrt((r["se_d_alpha"] ** 2).sum(0)) / math.sqrt(64)   # scaled to 2^22 paths
    for i, a in enumerate((0.5, 0.9)):
        ref = hf.reflectance_total_dalpha(float(np.float32(a)))
        assert abs(g["d_alpha"][:, i].sum() - ref) <= 4 * se[i] + 1e-3 * ref


def test_sigma_t_gradient_pins(api):
    # semi-infinite: R does not depend on sigma_t (separability, Eq. 5)
    x = inputs.single_wavelength(n_paths=1 << 20).subset(np.arange(10, 14))
    x.n_rel = 1.4
    o = api.WalkOptions(nbins=32, r_max_mm=10.0, seed=31)
    g, _, _ = _grads_gpu(api, x, o, grad_R=np.ones(x.n_inst))
    r = oracle.walk_grad(x.alpha, x.sigma_t, x.g, x.w, np.full(x.n_inst, 1 << 16, np.uint32),
                         None, 1.4, to_oracle_opts(o), grad_R=np.ones(x.n_inst))
    se = np.sqrt((r["se_d_sigma_t"] ** 2).sum(0)) / 4.0
    assert np.all(np.abs(g["d_sigma_t"].sum(0)) <= 4 * se)
    # ballistic slab: alpha = 0, n = 1, dT/dsigma_t = -d exp(-sigma_t d)
    y = inputs.single_wavelength(n_paths=1 << 20).subset(np.arange(3))
    y.alpha[:] = 0.0
    y.thickness_mm = np.array([0.3, 0.8, 2.0], np.float32)
    o2 = api.WalkOptions(nbins=8, r_max_mm=1.0, seed=5, mode=1, entry_fresnel=0)
    g2, _, _ = _grads_gpu(api, y, o2, grad_T=np.ones(3))
    d = y.thickness_mm.astype(np.float64)
    st = y.sigma_t[0].astype(np.float64)
    ref = -d * np.exp(-st * d)
    p = np.exp(-st * d)
    se = d * np.sqrt(p * (1 - p) / (1 << 20))
    assert np.all(np.abs(g2["d_sigma_t"].sum(0) - ref) <= 4 * se + 1e-6)


def test_weight_gradient_is_per_medium_reflectance(api):
    import torch
    x = inputs.spectral_field(n_texels=2, param_seed=12, n_paths=16384)
    o = api.WalkOptions(nbins=32, r_max_mm=10.0, seed=8)
    g, _, flags = _grads_gpu(api, x, o, grad_R=np.ones(x.n_inst))
    f = api.walk(api.Media.from_inputs(x), o)
    Rk = f["R_k"].cpu().numpy()                 # [n][K]
    wsum = x.w.astype(np.float32).sum(0)
    expect = (Rk.T * wsum / x.w)                 # same paths, same weights
    np.testing.assert_allclose(g["d_w"], expect, rtol=1e-5, atol=1e-7)


def test_adjoint_is_deterministic_across_launch_shapes(api):
    x = inputs.uneven_batch(n_inst=200, param_seed=4, log2_min=8, log2_max=13)
    up = _upstream(x, 48, seed=3)
    base = api.WalkOptions(nbins=48, r_max_mm=6.0, seed=17)
    ref, code, _ = _grads_gpu(api, x, base, **up)
    assert code == 0
    for kw in ({}, {"block_threads": 64}, {"unit_paths": 100, "regroup": 1}):
        o = api.WalkOptions(nbins=48, r_max_mm=6.0, seed=17, **kw)
        got, _, _ = _grads_gpu(api, x, o, **up)
        for k in ref:
            np.testing.assert_array_equal(ref[k], got[k], err_msg=f"{k} {kw}")


def test_autograd_function_routes_to_replay(api):
    import torch
    x = inputs.spectral_field(n_texels=1, param_seed=6, n_paths=4096)
    o = api.WalkOptions(nbins=16, r_max_mm=5.0, seed=2)
    m = api.Media.from_inputs(x)
    params = [t.clone().requires_grad_(True) for t in (m.alpha, m.sigma_t, m.g, m.w)]
    R, bins, Rk = api.SSSWalk.apply(*params, m, o)
    cB = torch.linspace(-1, 1, 16, device="cuda", dtype=torch.float64)
    loss = (R * 2.0).sum() + (bins * cB).sum() + Rk[:, 1].sum()
    grads = torch.autograd.grad(loss, params)
    gB = cB.expand(m.n_inst, 16).contiguous()
    gK = torch.zeros(m.n_inst, 3, device="cuda", dtype=torch.float64); gK[:, 1] = 1.0
    d = api.walk_bwd(m, o, grad_R=torch.full((m.n_inst,), 2.0, device="cuda",
                                               dtype=torch.float64), grad_bins=gB, grad_R_k=gK)
    for gr, k in zip(grads, ("d_alpha", "d_sigma_t", "d_g", "d_w")):
        torch.testing.assert_close(gr, d[k].float())


def test_inverse_fit_recovers_albedo(api):
    # Targets from held-out parameters; fit the three albedo spectra of a few
    # texels by gradient descent on (R, radial bins) through the replay adjoint.
    import torch
    truth = inputs.spectral_field(n_texels=2, param_seed=33, n_paths=8192)
    o = api.WalkOptions(nbins=32, r_max_mm=10.0, seed=1003)
    mt = api.Media.from_inputs(truth)
    tgt = api.walk(mt, o)
    tR, tB = tgt["R"].clone(), tgt["bins"].clone()
    gen = torch.Generator(device="cuda").manual_seed(7)
    sign = torch.sign(torch.randn(mt.alpha.shape, device="cuda", generator=gen))
    alpha0 = torch.clamp(mt.alpha + 0.08 * sign, 0.3, 0.999)
    logit = torch.logit(alpha0).clone().requires_grad_(True)
    iters = 150
    opt = torch.optim.Adam([logit], lr=0.05)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, iters)
    err0 = None
    for it in range(iters):
        a = torch.sigmoid(logit)
        R, bins, _ = api.SSSWalk.apply(a, mt.sigma_t, mt.g, mt.w, mt, o)
        loss = ((R - tR) ** 2).sum() + ((bins - tB) ** 2).sum()
        opt.zero_grad()
        loss.backward()
        opt.step()
        sched.step()
        if err0 is None:
            err0 = float(loss)
    final = float(loss)
    print("inverse fit loss", err0, "->", final)
    assert final < 0.01 * err0
    # albedo of the heaviest medium per band is recovered where it matters
    a = torch.sigmoid(logit).detach()
    heavy = mt.w.argmax(0)
    idx = torch.arange(mt.n_inst, device="cuda")
    err = (a[heavy, idx] - mt.alpha[heavy, idx]).abs()
    assert float(err.median()) < 0.02


def test_sigma_t_and_g_gradients_match_crn_finite_differences(api):
    # 64 instances of the adjoint workload; central differences with common
    # random numbers (same seed), their error from 32 disjoint path ranges
    # (path_offset), against the replay adjoint.  The bin tallies jump where
    # a path's exit crosses a bin edge; d(bins)/d(sigma_t, g) includes that
    # boundary term, which a common-random-number difference samples only
    # through paths that actually cross, so the step must be large enough
    # for crossings to occur in 2^16 paths: h = 5% of sigma_t and 0.02 in g
    # (at h = 1e-3 almost none cross and the difference misses the term).
    # FD and adjoint are different estimators of the same derivative,
    # compared by z; with 32 batch means z follows a t law with 31 degrees of
    # freedom: over the 256 comparisons max |z| <= 5 and mean z^2 <= 2.
    import torch
    x = inputs.spectral_field(n_texels=1, param_seed=3, n_paths=1 << 16).subset(np.arange(64))
    N, B = 1 << 16, 32
    o = api.WalkOptions(nbins=64, r_max_mm=10.0, seed=1003)
    gb = np.zeros((64, 64)); gb[:, 2] = 1.0
    gR = np.ones(64)
    adj, code, _ = _grads_gpu(api, x, o, grad_R=gR, grad_bins=gb)
    assert code == 0
    # per-instance standard error of the adjoint estimator from the oracle
    xs = x.subset(np.arange(64)); xs.n_paths = np.full(64, N // B, np.uint32)
    r = oracle.walk_grad(xs.alpha, xs.sigma_t, xs.g, xs.w, xs.n_paths, None, x.n_rel,
                         to_oracle_opts(o), grad_R=gR, grad_bins=gb)
    for param, key, rel in (("sigma_t", "d_sigma_t", True), ("g", "d_g", False)):
        for k in (0, 1):
            fds = []
            for b in range(B):
                ob = api.WalkOptions(nbins=64, r_max_mm=10.0, seed=1003, path_offset=b * (N // B))
                vals = []
                for sgn in (+1, -1):
                    xp = x.subset(np.arange(64)); xp.n_paths = np.full(64, N // B, np.uint32)
                    arr = getattr(xp, param)
                    base = arr[k].astype(np.float64)
                    h = 5e-2 * base if rel else np.full(64, 2e-2)
                    arr[k] = (base + sgn * h).astype(np.float32)
                    res = api.walk(api.Media.from_inputs(xp), ob)
                    vals.append((res["R"] + res["bins"][:, 2]).cpu().numpy())
                    step = getattr(xp, param)[k].astype(np.float64)
                    if sgn == +1:
                        up = step
                    else:
                        dn = step
                fds.append((vals[0] - vals[1]) / (up - dn))
            fds = np.array(fds)
            fd, fd_se = fds.mean(0), fds.std(0, ddof=1) / np.sqrt(B)
            se_adj = r["se_" + key][k] / np.sqrt(B)
            z = (adj[key][k] - fd) / np.sqrt(fd_se ** 2 + se_adj ** 2)
            print(param, k, "z rms", np.sqrt(np.mean(z ** 2)), "max", np.abs(z).max())
            assert np.abs(z).max() <= 5.0 and np.mean(z ** 2) <= 2.0, (param, k)

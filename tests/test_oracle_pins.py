"""Pins of the FP64 oracle against things other than itself.

Each test ties one part of the oracle to a closed form, an invariant of the
transport problem (paper Sec. 4.1 Eq. 3/4, Sec. 4.2 Eq. 5), a textbook
identity or a library routine.  A dropped term, a wrong sign or a swapped
operand anywhere in the oracle's walk fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import hfunction as hf
from paper_2606_27604_b300 import inputs

Z = 4.0  # tolerance in standard errors


def _single(alpha, sigma_t=1.0, g=0.0, K=3, n=1, w=None):
    a = np.full((K, n), alpha, np.float32)
    s = np.full((K, n), sigma_t, np.float32)
    gg = np.full((K, n), g, np.float32)
    ww = np.full((K, n), 1.0 / K, np.float32) if w is None else np.asarray(w, np.float32)
    return a, s, gg, ww


# --------------------------------------------------------------------------
# Random numbers: Philox4x32-10 against an independent library implementation
# --------------------------------------------------------------------------
_TRITON_PHILOX = r"""
import json, sys
import numpy as np
import torch
import triton
import triton.language as tl

@triton.jit
def _k(out, c0p, c1p, c2p, c3p, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i),
                           tl.load(c2p + i), tl.load(c3p + i))
    tl.store(out + i * 4 + 0, a)
    tl.store(out + i * 4 + 1, b)
    tl.store(out + i * 4 + 2, c)
    tl.store(out + i * 4 + 3, d)

req = json.loads(sys.stdin.read())
ctrs, key = req["ctrs"], req["key"]
n = len(ctrs)
cols = [torch.tensor(np.array([c[j] for c in ctrs], np.uint32).view(np.int32))
        for j in range(4)]
out = torch.zeros(4 * n, dtype=torch.int32)
_k[(1,)](out, *cols, int(key[0]) | (int(key[1]) << 32), N=n)
print(json.dumps(out.numpy().view(np.uint32).reshape(n, 4).tolist()))
"""


def _triton_philox(ctrs, key):
    """Triton's own Philox4x32-10 (tl.philox), run by its CPU interpreter in
    a child process so that TRITON_INTERPRET is set before triton loads."""
    import json
    import os
    import subprocess
    import sys
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_PHILOX], env=env, check=True,
                       input=json.dumps({"ctrs": ctrs, "key": list(key)}),
                       capture_output=True, text=True, timeout=600)
    return np.array(json.loads(r.stdout.strip().splitlines()[-1]), dtype=np.uint32)


def test_philox_matches_library_implementation():
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    ctrs = [(0, 0, 0, 0), (1, 0, 0, 0), (0xFFFFFFFF,) * 4, (5, 123456, 987, 1),
            (65535, 2 ** 27 - 1, 84934655, 0)]
    ctrs += [tuple(int(v) for v in rng.integers(0, 2 ** 32, 4, dtype=np.uint64))
             for _ in range(3)]
    for key in [(0, 0), (1000, 0), (0xDEADBEEF, 0x12345678)]:
        ref = _triton_philox(ctrs, key)
        got = np.array([oracle.philox4x32_10(c, key) for c in ctrs])
        np.testing.assert_array_equal(got, ref)


# --------------------------------------------------------------------------
# Boundary: smooth dielectric Fresnel (Sec. 8: smooth Fresnel boundary)
# --------------------------------------------------------------------------
def test_fresnel_special_cases():
    for n in (1.33, 1.4, 1.5):
        r0 = ((n - 1) / (n + 1)) ** 2
        assert oracle.fresnel(1.0, n) == pytest.approx(r0, rel=1e-12)
        crit = math.sqrt(1 - 1 / n ** 2)          # cos of the critical angle
        assert oracle.fresnel(crit - 1e-9, n) == 1.0
        assert oracle.fresnel(crit + 1e-6, n) < 1.0
        assert oracle.fresnel(0.0, n) == 1.0
        # Brewster angle seen from inside (tan theta = 1/n): p-wave vanishes,
        # so F equals half the s-wave reflectance.
        th = math.atan(1.0 / n)
        ci, si = math.cos(th), math.sin(th)
        ct = math.sqrt(1 - (n * si) ** 2)
        rs = (n * ci - ct) / (n * ci + ct)
        assert oracle.fresnel(ci, n) == pytest.approx(0.5 * rs * rs, rel=1e-10)
    assert oracle.fresnel(0.3, 1.0) == 0.0


def test_fresnel_reciprocity_with_outside_view():
    # Reflectance is the same seen from either side of the interface for the
    # refracted pair of angles (Stokes relations).
    n = 1.4
    for cos_out in (0.2, 0.5, 0.9):
        sin_out = math.sqrt(1 - cos_out ** 2)
        sin_in = sin_out / n
        cos_in = math.sqrt(1 - sin_in ** 2)
        # outside -> inside, written with the outside angle as incidence
        rs = (cos_out - n * cos_in) / (cos_out + n * cos_in)
        rp = (n * cos_out - cos_in) / (n * cos_out + cos_in)
        F_out = 0.5 * (rs * rs + rp * rp)
        assert oracle.fresnel(cos_in, n) == pytest.approx(F_out, rel=1e-10)


# --------------------------------------------------------------------------
# Henyey-Greenstein sampling (the phase function pf of Sec. 4.1 with g)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("g", [0.0, 0.3, 0.87, 0.95, -0.5])
def test_hg_moments_and_histogram(g):
    M = 200000
    u = (np.arange(M) + 0.5) / M                  # stratified quadrature in u
    mu = np.array([oracle.hg_mu(g, x) for x in u])
    assert np.all(np.abs(mu) <= 1.0)
    assert mu.mean() == pytest.approx(g, abs=2e-4)           # E[mu] = g
    # E[mu^2] for HG = (1 + 2 g^2) / 3
    assert (mu ** 2).mean() == pytest.approx((1 + 2 * g * g) / 3, abs=2e-4)
    if abs(g) > 1e-3:
        # the score d log p / dg has zero mean under p
        sc = np.array([oracle.hg_dlogp_dg(g, m) for m in mu[::10]])
        assert abs(sc.mean()) < 5e-3 * max(1.0, np.abs(sc).mean())


def test_hg_score_matches_numerical_derivative_of_cdf_density():
    # density from the numerical derivative of the sampled quantile function
    g, h = 0.6, 1e-5
    for u in (0.1, 0.4, 0.8):
        mu = oracle.hg_mu(g, u)
        dmu_du = (oracle.hg_mu(g, u + h) - oracle.hg_mu(g, u - h)) / (2 * h)
        p = 1.0 / dmu_du                       # p(mu) = du/dmu
        # p at g +- dg for the same mu, via the quantile function's slope
        def dens(gv):
            # find u' with mu(gv, u') = mu by bisection, then slope there
            lo, hi = 0.0, 1.0
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                if oracle.hg_mu(gv, mid) < mu:
                    lo = mid
                else:
                    hi = mid
            um = 0.5 * (lo + hi)
            return 1.0 / ((oracle.hg_mu(gv, um + h) - oracle.hg_mu(gv, um - h)) / (2 * h))
        dg = 1e-4
        dlogp = (math.log(dens(g + dg)) - math.log(dens(g - dg))) / (2 * dg)
        assert oracle.hg_dlogp_dg(g, mu) == pytest.approx(dlogp, rel=2e-3, abs=2e-3)
        assert p > 0


def test_rotation_preserves_angle_and_norm():
    rng = np.random.default_rng(3)
    for _ in range(200):
        u = rng.normal(size=3); u /= np.linalg.norm(u)
        if rng.uniform() < 0.2:
            u = np.array([0.0, 0.0, rng.choice([-1.0, 1.0])])
        mu = rng.uniform(-1, 1); phi = rng.uniform(0, 2 * math.pi)
        v = oracle.rotate(u, mu, phi)
        assert np.linalg.norm(v) == pytest.approx(1.0, abs=1e-12)
        assert float(u @ v) == pytest.approx(mu, abs=1e-9)


def test_selection_frequencies_follow_weights():
    w = np.array([0.2, 0.5, 0.3], np.float32)
    M = 100000
    u = (np.arange(M) + 0.5) / M
    ks = np.array([oracle.select_medium(w, x) for x in u])
    freq = np.bincount(ks, minlength=3) / M
    np.testing.assert_allclose(freq, w, atol=2e-5)


# --------------------------------------------------------------------------
# Walk against closed forms (Chandrasekhar H-function; exact single scatter)
# --------------------------------------------------------------------------
def test_h_function_moment_identity():
    # int_0^1 H dmu = (2/alpha) (1 - sqrt(1 - alpha)) for isotropic scattering
    for a in (0.1, 0.5, 0.9, 0.99, 0.999):
        mu, wq, H = hf.h_nodes(a, 400)
        assert (wq * H).sum() == pytest.approx(2 / a * (1 - math.sqrt(1 - a)), rel=1e-12)


def test_h_function_second_form():
    # H also solves H(mu) = 1 + (alpha/2) mu H(mu) int_0^1 H(mu')/(mu+mu') dmu'
    a = 0.9
    mu, wq, H = hf.h_nodes(a, 400)
    for m in (0.1, 0.5, 1.0):
        Hm = hf.h_function(a, [m])[0]
        rhs = 1 + 0.5 * a * m * Hm * (wq * H / (m + mu)).sum()
        assert Hm == pytest.approx(rhs, rel=1e-10)


def test_walk_matches_h_function_and_single_scatter():
    x = inputs.single_wavelength(n_paths=1 << 17)
    sel = np.arange(10)
    x = x.subset(sel)
    o = oracle.OracleOpts(nbins=32, r_max_mm=10.0, seed=1000)
    r = oracle.walk(x.alpha, x.sigma_t, x.g, x.w, x.n_paths, None, 1.0, o)
    for i, a in enumerate(inputs.ALPHA_SET0):
        R = hf.reflectance_total(a)
        R1 = hf.reflectance_single(a)
        assert abs(r["R"][i] - R) <= Z * r["se_R"][i], (a, r["R"][i], R)
        assert abs(r["R1"][i] - R1) <= Z * r["se_R1"][i], (a, r["R1"][i], R1)
        assert r["truncated"][i] == 0
        np.testing.assert_allclose(r["R"][i], r["bins"][i].sum() + r["overflow"][i],
                                   rtol=1e-12)


def test_cosine_lobe_incidence_matches_h_function():
    # cosine-weighted incident lobe: R = 2 int R(mu) mu dmu = 1 - 2 sqrt(1-a) int H mu dmu
    for a in (0.5, 0.9, 0.99):
        A, S, G, W = _single(a, K=1)
        r = oracle.walk(A, S, G, W, np.array([1 << 17], np.uint32), None, 1.0,
                        oracle.OracleOpts(incidence=1, seed=3))
        Rc = hf.reflectance_cosine_lobe(a)
        assert abs(r["R"][0] - Rc) <= Z * r["se_R"][0]
        assert Rc > hf.reflectance_total(a)  # oblique light escapes more easily
    # with a boundary the entry weight follows Fresnel at the refracted angle:
    # alpha = 0 leaves only that specular loss, so A = 1 - <F>
    A, S, G, W = _single(0.0, K=1)
    r = oracle.walk(A, S, G, W, np.array([1 << 16], np.uint32), None, 1.4,
                    oracle.OracleOpts(incidence=1, seed=4))
    mu = (np.arange(20000) + 0.5) / 20000      # outside cosines, density 2 mu
    ci = np.sqrt(1 - (1 - mu ** 2) / 1.4 ** 2)
    Fm = np.mean([oracle.fresnel(c, 1.4) * 2 * m for c, m in zip(ci, mu)])
    assert abs(r["A"][0] - (1 - Fm)) <= Z * r["se_A"][0] + 1e-4


def test_zero_albedo_gives_no_reflectance():
    for n_rel in (1.0, 1.4):
        a, s, g, w = _single(0.0, 3.0, 0.5, n=2)
        r = oracle.walk(a, s, g, w, np.full(2, 20000, np.uint32), None, n_rel,
                        oracle.OracleOpts(nbins=16, r_max_mm=5.0, mode=0))
        assert np.all(r["R"] == 0.0) and np.all(r["R1"] == 0.0)
        assert np.all(r["bins"] == 0.0) and np.all(r["T"] == 0.0)
        R0 = ((n_rel - 1) / (n_rel + 1)) ** 2
        np.testing.assert_allclose(r["A"], 1 - R0, rtol=1e-12)


@pytest.mark.parametrize("n_rel", [1.0, 1.4])
def test_finite_slab_zero_albedo_ballistic(n_rel):
    d, st = 0.7, 1.3
    tau = st * d
    N = 200000
    a, s, g, w = _single(0.0, st, 0.0)
    th = np.array([d], np.float32)
    r = oracle.walk(a, s, g, w, np.array([N], np.uint32), th, n_rel,
                    oracle.OracleOpts(nbins=8, r_max_mm=1.0, mode=1, entry_fresnel=1))
    R0 = ((n_rel - 1) / (n_rel + 1)) ** 2
    e = math.exp(-float(np.float32(st)) * float(np.float32(d)))
    T = (1 - R0) ** 2 * e / (1 - R0 ** 2 * e * e)
    R = (1 - R0) ** 2 * R0 * e * e / (1 - R0 ** 2 * e * e)
    assert abs(r["T"][0] - T) <= Z * r["se_T"][0]
    if n_rel == 1.0:
        assert r["R"][0] == 0.0
    else:
        assert abs(r["R"][0] - R) <= Z * r["se_R"][0]
    # ballistic paths stay on the axis: every top exit lands in bin 0
    assert r["bins"][0][1:].sum() == 0.0 and r["overflow"][0] == 0.0


def test_energy_conservation():
    x = inputs.single_wavelength(n_paths=1 << 14).subset(np.arange(10, 16))
    th = np.array([0.5, 2.0, np.inf, 1.0, np.inf, 0.3], np.float32)
    # analog mode, entry weight 1: every path ends in exactly one way
    r = oracle.walk(x.alpha, x.sigma_t, x.g, x.w, x.n_paths, th, 1.4,
                    oracle.OracleOpts(nbins=16, mode=1, entry_fresnel=0, max_steps=4096))
    N = x.n_paths.astype(np.float64)
    exits = (r["R"] + r["T"] + r["A"]) * N + r["truncated"]
    np.testing.assert_allclose(exits, N, rtol=0, atol=1e-6)
    # weight mode: R + T + A = 1 - R0 in expectation (roulette is unbiased)
    rw = oracle.walk(x.alpha, x.sigma_t, x.g, x.w, x.n_paths, th, 1.4,
                     oracle.OracleOpts(nbins=16, mode=0, entry_fresnel=1))
    R0 = (0.4 / 2.4) ** 2
    tot = rw["R"] + rw["T"] + rw["A"]
    se = np.sqrt(rw["se_R"] ** 2 + rw["se_T"] ** 2 + rw["se_A"] ** 2) * 2
    assert np.all(np.abs(tot - (1 - R0)) <= Z * se + 1e-12)


def test_three_identical_media_equal_one_medium():
    a3, s3, g3, w3 = _single(0.93, 2.5, 0.7, K=3, n=1, w=[[0.2], [0.3], [0.5]])
    a1, s1, g1, w1 = _single(0.93, 2.5, 0.7, K=1, n=1)
    o = oracle.OracleOpts(nbins=32, r_max_mm=4.0, seed=99)
    N = np.array([40000], np.uint32)
    r3 = oracle.walk(a3, s3, g3, w3, N, None, 1.4, o)
    r1 = oracle.walk(a1, s1, g1, w1, N, None, 1.4, o)
    for k in ("R", "T", "A", "bins", "overflow", "R1"):
        np.testing.assert_array_equal(r3[k], r1[k])
    # and the per-medium split adds up to R, with shares near the weights
    assert r3["R_k"].sum() == pytest.approx(r3["R"][0], rel=1e-12)


def test_mixture_is_weighted_sum_not_blend():
    # Eq. 4: S = sum_k w_k S_k.  Independent single-medium runs (other seed).
    a = np.array([[0.99], [0.6], [0.9]], np.float32)
    s = np.array([[1.0], [30.0], [5.0]], np.float32)
    g = np.array([[0.8], [0.1], [0.5]], np.float32)
    w = np.array([[0.5], [0.2], [0.3]], np.float32)
    N = np.array([200000], np.uint32)
    o = oracle.OracleOpts(nbins=16, r_max_mm=4.0, seed=5)
    mix = oracle.walk(a, s, g, w, N, None, 1.4, o)
    parts, se2 = 0.0, 0.0
    for k in range(3):
        o2 = oracle.OracleOpts(nbins=16, r_max_mm=4.0, seed=77 + k)
        rk = oracle.walk(a[k:k + 1], s[k:k + 1], g[k:k + 1], np.ones((1, 1), np.float32),
                         N, None, 1.4, o2)
        parts += float(w[k, 0]) * rk["R"][0]
        se2 += (float(w[k, 0]) * rk["se_R"][0]) ** 2
    assert abs(mix["R"][0] - parts) <= Z * math.sqrt(mix["se_R"][0] ** 2 + se2)
    # blending the parameters is a different medium with a different R
    ab = np.full((1, 1), (w * a).sum(), np.float32)
    sb = np.full((1, 1), (w * s).sum(), np.float32)
    gb = np.full((1, 1), (w * g).sum(), np.float32)
    bl = oracle.walk(ab, sb, gb, np.ones((1, 1), np.float32), N, None, 1.4, o)
    assert abs(bl["R"][0] - mix["R"][0]) > 10 * mix["se_R"][0]


def test_separability_of_extinction():
    # Sec. 4.2 Eq. 5: sigma_t only rescales the radial axis of a homogeneous
    # semi-infinite slab; R does not depend on it.  A power-of-two scale is
    # exact in binary arithmetic, so the histograms agree bit for bit.
    a, s, g, w = _single(0.95, 1.5, 0.6)
    N = np.array([30000], np.uint32)
    r1 = oracle.walk(a, s, g, w, N, None, 1.4, oracle.OracleOpts(nbins=32, r_max_mm=8.0))
    r2 = oracle.walk(a, s * 4, g, w, N, None, 1.4, oracle.OracleOpts(nbins=32, r_max_mm=2.0))
    np.testing.assert_array_equal(r1["bins"], r2["bins"])
    np.testing.assert_array_equal(r1["R"], r2["R"])
    # a non-power-of-two scale keeps R up to rounding-level path flips
    r3 = oracle.walk(a, s * 3.7, g, w, N, None, 1.4, oracle.OracleOpts(nbins=32, r_max_mm=8.0))
    assert abs(r3["R"][0] - r1["R"][0]) <= 3.0 / N[0]


# --------------------------------------------------------------------------
# Two-layer slab (skin model of Sec. 3: a top slab over a second layer)
# --------------------------------------------------------------------------
def _layer2(a, s, g, d1, n=1):
    f = lambda v: np.full(n, v, np.float32)
    return (f(a), f(s), f(g), f(d1))


def test_uniform_selection_pdf_is_unbiased():
    # another selection pdf (Sec. 7): uniform choice reweighted by
    # K w_k / sum(w) estimates the same mixture (Eq. 4) as choosing by w_k;
    # unnormalised weights catch a missing 1/sum(w), a missing K, or a
    # weight applied to the wrong medium.
    a = np.array([[0.99], [0.8], [0.95]], np.float32)
    s = np.array([[1.0], [5.0], [2.0]], np.float32)
    g = np.array([[0.8], [0.0], [0.5]], np.float32)
    w = np.array([[2.0], [0.5], [1.0]], np.float32)
    N = np.array([1 << 17], np.uint32)
    byw = oracle.walk(a, s, g, w, N, None, 1.4, oracle.OracleOpts(nbins=8, r_max_mm=4.0, seed=21))
    uni = oracle.walk(a, s, g, w, N, None, 1.4,
                      oracle.OracleOpts(nbins=8, r_max_mm=4.0, seed=22, select_pdf=1))
    for key in ("R", "T", "A", "R1"):
        assert abs(uni[key][0] - byw[key][0]) <= Z * np.hypot(uni["se_" + key][0],
                                                               byw["se_" + key][0]), key
    d = np.abs(uni["R_k"][0] - byw["R_k"][0])
    assert np.all(d <= Z * np.hypot(uni["se_R_k"][0], byw["se_R_k"][0]))
    assert np.all(np.abs(uni["bins"][0] - byw["bins"][0])
                  <= Z * np.hypot(uni["se_bins"][0], byw["se_bins"][0]) + 1e-12)
    # a zero-weight medium is still walked but carries nothing, and its
    # gradient stays finite
    w0 = np.array([[1.0], [0.0], [1.0]], np.float32)
    z = oracle.walk(a, s, g, w0, np.array([20000], np.uint32), None, 1.4,
                    oracle.OracleOpts(nbins=8, r_max_mm=4.0, seed=23, select_pdf=1))
    assert z["R_k"][0, 1] == 0.0 and z["R_k"][0, 0] > 0.0
    gz = oracle.walk_grad(a, s, g, w0, np.array([20000], np.uint32), None, 1.4,
                          oracle.OracleOpts(nbins=8, r_max_mm=4.0, seed=23, select_pdf=1),
                          grad_R=np.ones(1))
    assert np.all(np.isfinite(gz["d_w"])) and gz["d_w"][1, 0] == 0.0


def test_hero_walk_reduces_to_the_walk_and_is_unbiased():
    # hero-wavelength sharing (Wilkie et al. 2014; named in the paper's
    # related work): C = 1 is the plain walk bit for bit; with C = 3, over
    # adjacent-band groups and over rotation orbits, every band's tallies
    # match separate per-band walks within the statistical bar.
    from paper_2606_27604_b300 import inputs
    x = inputs.spectral_field(n_texels=2, param_seed=3, n_paths=1)
    o = oracle.OracleOpts(nbins=16, r_max_mm=10.0, seed=5)
    one = oracle.walk_hero(x.alpha, x.sigma_t, x.g, x.w, 3000, 1, 81, None, x.n_rel, o)
    ref = oracle.walk(x.alpha, x.sigma_t, x.g, x.w, np.full(x.n_inst, 3000, np.uint32), None,
                      x.n_rel, o)
    for key in ("R", "T", "bins", "overflow", "R_k", "R1", "steps"):
        np.testing.assert_array_equal(one[key], ref[key])
    N = 30000
    sep = oracle.walk(x.alpha, x.sigma_t, x.g, x.w, np.full(x.n_inst, N, np.uint32), None,
                      x.n_rel, oracle.OracleOpts(nbins=16, r_max_mm=10.0, seed=6))
    for orbits in (False, True):
        h = oracle.walk_hero(x.alpha, x.sigma_t, x.g, x.w, N, 3, 81, None, x.n_rel, o,
                             orbits=orbits)
        for key in ("R", "R1"):
            z = (h[key] - sep[key]) / np.hypot(h["se_" + key], sep["se_" + key])
            assert np.sqrt(np.mean(z ** 2)) < 1.25 and np.abs(z).max() < 4.5, (orbits, key)
        m = (h["se_bins"] > 0) & (sep["se_bins"] > 0)
        zb = (h["bins"] - sep["bins"])[m] / np.hypot(h["se_bins"], sep["se_bins"])[m]
        assert np.sqrt(np.mean(zb ** 2)) < 1.25, orbits
        if not orbits:
            # adjacent bands: balance weights near 1/C, so one shared path per
            # group is worth about one path per band
            assert np.median(h["se_R"] / sep["se_R"]) < 1.1


def test_hero_walk_identical_members_share_every_tally():
    # members with identical optics have equal path densities, so every
    # balance weight is 1/C and all members score exactly the same
    a, s, g, w = _single(0.95, 3.0, 0.7, K=3, n=6, w=[[0.5] * 6, [0.3] * 6, [0.2] * 6])
    a[1] = 0.7
    s[2] = 9.0
    h = oracle.walk_hero(a, s, g, w, 4000, 3, 3, None, 1.4,
                         oracle.OracleOpts(nbins=8, r_max_mm=4.0, seed=9))
    for key in ("R", "T", "R1", "steps"):
        assert np.all(h[key][0:3] == h[key][0]) and np.all(h[key][3:6] == h[key][3]), key
    np.testing.assert_array_equal(h["bins"][1], h["bins"][0])
    one = oracle.walk(a, s, g, w, np.full(6, 60000, np.uint32), None, 1.4,
                      oracle.OracleOpts(nbins=8, r_max_mm=4.0, seed=10))
    assert abs(h["R"][0] - one["R"][0]) <= Z * np.hypot(h["se_R"][0], one["se_R"][0])


def test_hero_walk_uniform_selection_with_zero_weights_is_unbiased():
    # uniform selection lets a hero pick a medium it gives no weight: the
    # path must still serve the other members, so roulette is decided on
    # the largest member weight (a rule on the hero's alone loses them)
    a = np.array([[0.97] * 3, [0.9] * 3, [0.99] * 3], np.float32)
    s = np.array([[2.0] * 3, [8.0] * 3, [1.0] * 3], np.float32)
    g = np.array([[0.8] * 3, [0.3] * 3, [0.6] * 3], np.float32)
    w = np.array([[1.0, 1.0, 0.0], [0.0, 1.0, 1.0], [1.0, 1.0, 1.0]], np.float32)
    N = 40000
    o = oracle.OracleOpts(nbins=8, r_max_mm=4.0, seed=31, select_pdf=1)
    h = oracle.walk_hero(a, s, g, w, N, 3, 3, None, 1.4, o)
    sep = oracle.walk(a, s, g, w, np.full(3, N, np.uint32), None, 1.4,
                      oracle.OracleOpts(nbins=8, r_max_mm=4.0, seed=32))
    z = (h["R"] - sep["R"]) / np.hypot(h["se_R"], sep["se_R"])
    assert np.all(np.abs(z) < Z), z
    zk = (h["R_k"] - sep["R_k"]) / np.maximum(np.hypot(h["se_R_k"], sep["se_R_k"]), 1e-12)
    assert np.all(np.abs(zk) < Z), zk


def test_log_bins_partition_the_same_exits():
    # logarithmic bins (512 to 50 mm, as the paper's generator) regroup the
    # same exits: their sum equals the linear bins' sum plus overflow, and a
    # bin's content equals the linear tally over the same radii
    A, S, G, W = _single(0.97, 2.0, 0.8, K=1)
    N = np.array([50000], np.uint32)
    lin = oracle.walk(A, S, G, W, N, None, 1.4, oracle.OracleOpts(nbins=50, r_max_mm=50.0, seed=8))
    lg = oracle.walk(A, S, G, W, N, None, 1.4,
                     oracle.OracleOpts(nbins=512, r_max_mm=50.0, seed=8, log_r_min_mm=1.0))
    np.testing.assert_allclose(lg["bins"].sum() + lg["overflow"][0], lin["R"][0], rtol=1e-12)
    np.testing.assert_allclose(lg["bins"][0, 0], lin["bins"][0, 0], rtol=1e-12)  # [0, 1 mm)
    np.testing.assert_allclose(lg["overflow"], lin["overflow"], rtol=1e-12)


def test_two_layer_gradient_pins():
    # gradients of the two-layer walk (score form, Sec. 4.1 path
    # contribution): (1) an interface too deep to reach gives zero layer-2
    # gradients and the one-layer gradients exactly; (2) without roulette the
    # paths do not depend on the albedos, so a central difference of R in
    # alpha2 on the same streams equals the score estimate; (3) with equal
    # optics in both layers, top-layer plus layer-2 gradients add up to the
    # one-layer gradient of that medium (statistically).
    K = 1
    a = np.array([[0.9]], np.float32); s_ = np.array([[4.0]], np.float32)
    g = np.array([[0.6]], np.float32); w = np.ones((1, 1), np.float32)
    N = np.array([40000], np.uint32)
    up = dict(grad_R=np.ones(1))
    o = oracle.OracleOpts(nbins=8, r_max_mm=5.0, seed=41)
    deep = (np.array([0.99], np.float32), np.array([2.0], np.float32),
            np.array([0.3], np.float32), np.array([1e4], np.float32))
    gd = oracle.walk_grad(a, s_, g, w, N, None, 1.4, o, layer2=deep, **up)
    g1 = oracle.walk_grad(a, s_, g, w, N, None, 1.4, o, **up)
    for k in ("d_alpha", "d_sigma_t", "d_g", "d_w"):
        np.testing.assert_array_equal(gd[k], g1[k])
    assert gd["d_alpha2"][0] == 0 and gd["d_sigma_t2"][0] == 0 and gd["d_g2"][0] == 0
    # (2) alpha2 by central difference, roulette off
    o0 = oracle.OracleOpts(nbins=8, r_max_mm=5.0, seed=42, rr_threshold=0.0)
    l2 = (np.array([0.95], np.float32), np.array([2.0], np.float32),
          np.array([0.3], np.float32), np.array([0.15], np.float32))
    gs = oracle.walk_grad(a, s_, g, w, N, None, 1.4, o0, layer2=l2, **up)
    h = 1e-3
    lo = (l2[0] - np.float32(h), *l2[1:]); hi = (l2[0] + np.float32(h), *l2[1:])
    Rlo = oracle.walk(a, s_, g, w, N, None, 1.4, o0, layer2=lo)["R"][0]
    Rhi = oracle.walk(a, s_, g, w, N, None, 1.4, o0, layer2=hi)["R"][0]
    fd = (Rhi - Rlo) / (float(hi[0][0]) - float(lo[0][0]))
    print("d R / d alpha2: score", gs["d_alpha2"][0], "central difference", fd)
    assert abs(gs["d_alpha2"][0] - fd) <= 1e-3 * abs(fd)
    # (3) sum rule with equal layers
    same = (a[0].copy(), s_[0].copy(), g[0].copy(), np.array([0.25], np.float32))
    N2 = np.array([200000], np.uint32)
    two = oracle.walk_grad(a, s_, g, w, N2, None, 1.4, o, layer2=same, **up)
    one = oracle.walk_grad(a, s_, g, w, N2, None, 1.4, oracle.OracleOpts(nbins=8, r_max_mm=5.0,
                                                                        seed=43), **up)
    for k, k2 in (("d_alpha", "d_alpha2"), ("d_sigma_t", "d_sigma_t2"), ("d_g", "d_g2")):
        tot = two[k][0, 0] + two[k2][0]
        # sd(X + Y) <= sd(X) + sd(Y) whatever the correlation of the parts
        se = np.hypot(two["se_" + k][0, 0] + two["se_" + k2][0], one["se_" + k][0, 0])
        print(k, "top + layer 2", tot, "one layer", one[k][0, 0], "se", se)
        assert abs(tot - one[k][0, 0]) <= Z * se, k


def test_two_layer_limits_and_ballistic_transmittance():
    N = np.array([100000], np.uint32)
    o = oracle.OracleOpts(nbins=16, r_max_mm=4.0, seed=21)
    A, S, G, W = _single(0.95, 2.0, 0.6, K=1)
    one = oracle.walk(A, S, G, W, N, None, 1.4, o)
    # identical layers behave like one layer (statistically: the crossing
    # draws a fresh flight, which changes the random numbers, not the law)
    two = oracle.walk(A, S, G, W, N, None, 1.4, o, layer2=_layer2(0.95, 2.0, 0.6, 0.3))
    assert abs(two["R"][0] - one["R"][0]) <= Z * np.hypot(two["se_R"][0], one["se_R"][0])
    # a vanishing top layer leaves the second layer alone
    A2, S2, G2, _ = _single(0.8, 5.0, 0.2, K=1)
    ref2 = oracle.walk(A2, S2, G2, W, N, None, 1.4, oracle.OracleOpts(nbins=16, r_max_mm=4.0, seed=5))
    thin = oracle.walk(A, S, G, W, N, None, 1.4, o, layer2=_layer2(0.8, 5.0, 0.2, 1e-7))
    assert abs(thin["R"][0] - ref2["R"][0]) <= Z * np.hypot(thin["se_R"][0], ref2["se_R"][0])
    # a very thick top layer hides the second one
    thick = oracle.walk(A, S, G, W, N, None, 1.4, o, layer2=_layer2(0.8, 5.0, 0.2, 1e4))
    np.testing.assert_array_equal(thick["R"], one["R"])
    # ballistic transmittance through both layers: alpha = 0, n = 1
    A0, S1, G0, W1 = _single(0.0, 1.5, 0.0, K=1)
    d1, D = 0.4, 1.1
    r = oracle.walk(A0, S1, G0, W1, np.array([200000], np.uint32), np.array([D], np.float32),
                    1.0, oracle.OracleOpts(nbins=8, mode=1, entry_fresnel=0, seed=9),
                    layer2=_layer2(0.0, 3.0, 0.0, d1))
    f = lambda v: float(np.float32(v))
    Tc = math.exp(-f(1.5) * f(d1) - f(3.0) * (f(D) - f(d1)))
    assert abs(r["T"][0] - Tc) <= Z * r["se_T"][0]
    # analog path counts add up exactly with two layers
    r = oracle.walk(_single(0.9, 2.0, 0.5, K=1)[0], S, G, W, np.array([20000], np.uint32),
                    np.array([2.0], np.float32), 1.4,
                    oracle.OracleOpts(nbins=8, mode=1, entry_fresnel=0, max_steps=2048),
                    layer2=_layer2(0.7, 4.0, 0.3, 0.5))
    assert (r["R"][0] + r["T"][0] + r["A"][0]) * 20000 + r["truncated"][0] == pytest.approx(20000, abs=1e-6)


# --------------------------------------------------------------------------
# Gradient estimator (score form of f_SSS, Sec. 4.1; mixture Eq. 4)
# --------------------------------------------------------------------------
def test_alpha_gradient_is_exact_derivative_of_crn_estimator():
    # With roulette off, the path geometry does not depend on alpha, so the
    # common-random-number estimate is a polynomial in alpha and the score
    # estimate equals its derivative up to rounding.
    a, s, g, w = _single(0.8, 2.0, 0.5)
    N = np.array([20000], np.uint32)
    o = oracle.OracleOpts(nbins=16, r_max_mm=3.0, rr_threshold=0.0, max_steps=4096)
    h = 1e-3
    rp = oracle.walk(a + np.float32(h), s, g, w, N, None, 1.4, o)["R"][0]
    rm = oracle.walk(a - np.float32(h), s, g, w, N, None, 1.4, o)["R"][0]
    ap, am = float(np.float32(0.8) + np.float32(h)), float(np.float32(0.8) - np.float32(h))
    fd = (rp - rm) / (ap - am)
    gr = oracle.walk_grad(a, s, g, w, N, None, 1.4, o, grad_R=np.ones(1))
    assert gr["d_alpha"][:, 0].sum() == pytest.approx(fd, rel=2e-4)


def test_alpha_gradient_matches_closed_form():
    for alpha in (0.5, 0.9):
        a, s, g, w = _single(alpha)
        N = np.array([100000], np.uint32)
        o = oracle.OracleOpts(nbins=16, r_max_mm=10.0, seed=321)
        gr = oracle.walk_grad(a, s, g, w, N, None, 1.0, o, grad_R=np.ones(1))
        d = gr["d_alpha"][:, 0].sum()
        se = math.sqrt((gr["se_d_alpha"][:, 0] ** 2).sum())
        ref = hf.reflectance_total_dalpha(float(np.float32(alpha)))
        assert abs(d - ref) <= Z * se, (alpha, d, ref, se)


def test_sigma_t_gradient_zero_for_semi_infinite_reflectance():
    a, s, g, w = _single(0.9, 3.0, 0.4)
    gr = oracle.walk_grad(a, s, g, w, np.array([50000], np.uint32), None, 1.4,
                          oracle.OracleOpts(nbins=16, seed=11), grad_R=np.ones(1))
    d = gr["d_sigma_t"][:, 0].sum()
    se = math.sqrt((gr["se_d_sigma_t"][:, 0] ** 2).sum())
    assert abs(d) <= Z * se and se > 0


def test_sigma_t_gradient_ballistic_transmittance():
    # alpha = 0, n = 1, slab d: T = exp(-sigma_t d), dT/dsigma_t = -d exp(-sigma_t d)
    d, st = 0.8, 1.5
    a, s, g, w = _single(0.0, st)
    gr = oracle.walk_grad(a, s, g, w, np.array([200000], np.uint32),
                          np.array([d], np.float32), 1.0,
                          oracle.OracleOpts(nbins=8, mode=1), grad_T=np.ones(1))
    dd = gr["d_sigma_t"][:, 0].sum()
    se = math.sqrt((gr["se_d_sigma_t"][:, 0] ** 2).sum())
    ref = -float(np.float32(d)) * math.exp(-float(np.float32(st)) * float(np.float32(d)))
    assert abs(dd - ref) <= Z * se


def test_weight_gradient_equals_single_medium_reflectance():
    # dS/dw_k = S_k (Eq. 4), compared with independent single-medium runs
    a = np.array([[0.97], [0.7]], np.float32)
    s = np.array([[2.0], [10.0]], np.float32)
    g = np.array([[0.6], [0.2]], np.float32)
    w = np.array([[0.4], [0.6]], np.float32)
    N = np.array([100000], np.uint32)
    gr = oracle.walk_grad(a, s, g, w, N, None, 1.4, oracle.OracleOpts(nbins=16, seed=3),
                          grad_R=np.ones(1))
    for k in range(2):
        rk = oracle.walk(a[k:k + 1], s[k:k + 1], g[k:k + 1], np.ones((1, 1), np.float32),
                         N, None, 1.4, oracle.OracleOpts(nbins=16, seed=500 + k))
        se = math.sqrt(gr["se_d_w"][k, 0] ** 2 + rk["se_R"][0] ** 2)
        assert abs(gr["d_w"][k, 0] - rk["R"][0]) <= Z * se


def test_g_and_sigma_t_gradients_match_crn_finite_differences():
    a = np.array([[0.95], [0.8], [0.99]], np.float32)
    s = np.array([[2.0], [8.0], [1.0]], np.float32)
    g = np.array([[0.5], [0.2], [0.8]], np.float32)
    w = np.array([[0.3], [0.3], [0.4]], np.float32)
    o = oracle.OracleOpts(nbins=16, r_max_mm=2.0, seed=41)
    N = np.array([20000], np.uint32)
    gb = np.zeros((1, 16)); gb[0, 2] = 1.0          # d bin[2] / d theta
    grad = oracle.walk_grad(a, s, g, w, np.array([200000], np.uint32), None, 1.4, o,
                            grad_bins=gb)
    for param, key in (("g", "d_g"), ("sigma_t", "d_sigma_t")):
        for k in (0, 2):
            h = 0.02 if param == "g" else 0.05 * float(s[k, 0])
            fd, fd_se = _fd_bin(param, k, h, a, s, g, w, o, N, 8, 2)
            sc, sc_se = grad[key][k, 0], grad["se_" + key][k, 0]
            assert abs(fd - sc) <= Z * math.sqrt(fd_se ** 2 + sc_se ** 2) + 0.02 * abs(sc), \
                (param, k, fd, fd_se, sc, sc_se)


def _fd_bin(param, k, h, a, s, g, w, o, N, B, b):
    """Common-random-number central difference of bin b, with a batch-means
    standard error over B independent seeds."""
    vals = []
    for bb in range(B):
        ob = oracle.OracleOpts(**{**o.__dict__, "seed": o.seed + 1000 * bb})
        P = {"alpha": a.copy(), "sigma_t": s.copy(), "g": g.copy()}
        M = {"alpha": a.copy(), "sigma_t": s.copy(), "g": g.copy()}
        P[param][k] += np.float32(h)
        M[param][k] -= np.float32(h)
        step = float(P[param][k, 0]) - float(M[param][k, 0])
        rp = oracle.walk(P["alpha"], P["sigma_t"], P["g"], w, N, None, 1.4, ob)
        rm = oracle.walk(M["alpha"], M["sigma_t"], M["g"], w, N, None, 1.4, ob)
        vals.append((rp["bins"][0, b] - rm["bins"][0, b]) / step)
    vals = np.array(vals)
    return vals.mean(), vals.std(ddof=1) / math.sqrt(B)

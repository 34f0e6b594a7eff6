"""Seeded synthetic inputs for the walk and the decoder.

This module only draws random numbers and lays them out; it holds none of
the transport arithmetic.  The CUDA path, the oracle and the benchmark all
take their inputs from here, so both sides see the same float32 values.

The paper's own workload (decoder-predicted skin spectra, Sec. 5, Sec. 7)
needs trained weights and a skin dataset that are not available, so fields
with the paper's value ranges stand in:

* ``single_wavelength``: 16 sets.  Sets 0-9: one isotropic medium repeated
  three times (g = 0, w = 1/3 each), sigma_t = 1/mm, alpha in
  {0.1, 0.3, 0.5, 0.7, 0.8, 0.9, 0.95, 0.98, 0.99, 0.999}, semi-infinite,
  n = 1.  Sets 10-15: per medium alpha ~ U[0.5, 0.999], log10 sigma_t ~ U[0, 2]
  (mm^-1), g ~ U[0, 0.9], w ~ Dirichlet(1,1,1); same geometry.
* ``spectral_field``: texels x 81 bands (380-780 nm at 5 nm).  Per texel and
  medium, each parameter is drawn at 4 equally spaced knots over the band
  range (alpha ~ U[0.5,0.999], log10 sigma_t ~ U[0,2], g ~ U[0,0.95],
  log-weight = ln E, E ~ Exp(1)), passed through a natural cubic spline in
  wavelength, clamped back to its range; weights are the softmax of the
  splined log-weights over the media (at a knot that is Dirichlet(1,1,1)).
* ``uneven_batch``: independent instances with c1-style per-instance draws,
  a wavelength label uniform over the 151 bands 250-1000 nm, path budgets
  floor(2^U[10,20]) and slabs that are semi-infinite or U[0.1,5] mm thick
  with probability 1/2 each.
* ``rgb_texture``: an RGB albedo texture whose channels follow a seeded
  3-component Gaussian mixture clipped to [0.05, 0.85].

Instance order is texel-major, band fastest: ``i = texel * n_bands + band``.
Parameter arrays are float32 ``[K][n_inst]`` (structure of arrays).
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

K_MEDIA = 3
VISIBLE_NM = np.arange(380.0, 780.0 + 1e-9, 5.0)          # 81 bands
FULL_NM_5 = np.arange(250.0, 1000.0 + 1e-9, 5.0)          # 151 bands
ALPHA_SET0 = (0.1, 0.3, 0.5, 0.7, 0.8, 0.9, 0.95, 0.98, 0.99, 0.999)


@dataclass
class WalkInputs:
    alpha: np.ndarray            # float32 [K][n]
    sigma_t: np.ndarray          # float32 [K][n], mm^-1
    g: np.ndarray                # float32 [K][n]
    w: np.ndarray                # float32 [K][n], sums to 1 per instance
    n_paths: np.ndarray          # uint32 [n]
    thickness_mm: Optional[np.ndarray] = None  # float32 [n], +inf = semi-infinite
    n_rel: float = 1.0
    lambda_nm: Optional[np.ndarray] = None     # float32 [n], label only
    meta: dict = field(default_factory=dict)
    # optional second layer of a two-layer slab: (alpha2, sigma_t2, g2, d1_mm)
    layer2: Optional[tuple] = None

    @property
    def n_inst(self) -> int:
        return int(self.alpha.shape[1])

    @property
    def K(self) -> int:
        return int(self.alpha.shape[0])

    def subset(self, idx) -> "WalkInputs":
        idx = np.asarray(idx)
        return WalkInputs(
            alpha=np.ascontiguousarray(self.alpha[:, idx]),
            sigma_t=np.ascontiguousarray(self.sigma_t[:, idx]),
            g=np.ascontiguousarray(self.g[:, idx]),
            w=np.ascontiguousarray(self.w[:, idx]),
            n_paths=np.ascontiguousarray(self.n_paths[idx]),
            thickness_mm=None if self.thickness_mm is None
            else np.ascontiguousarray(self.thickness_mm[idx]),
            n_rel=self.n_rel,
            lambda_nm=None if self.lambda_nm is None else self.lambda_nm[idx],
            meta=dict(self.meta, subset=True),
            layer2=None if self.layer2 is None
            else tuple(np.ascontiguousarray(a[idx]) for a in self.layer2))


def _dirichlet_ones(rng, shape_lead, K):
    e = rng.exponential(1.0, size=shape_lead + (K,))
    return (e / e.sum(axis=-1, keepdims=True))


def single_wavelength(param_seed: int = 0, n_paths: int = 1 << 18) -> WalkInputs:
    rng = np.random.default_rng(param_seed)
    K = K_MEDIA
    n = 16
    alpha = np.zeros((K, n)); sig = np.ones((K, n)); g = np.zeros((K, n))
    w = np.full((K, n), 1.0 / 3.0)
    for i, a in enumerate(ALPHA_SET0):
        alpha[:, i] = a
    m = n - len(ALPHA_SET0)
    alpha[:, 10:] = rng.uniform(0.5, 0.999, size=(K, m))
    sig[:, 10:] = 10.0 ** rng.uniform(0.0, 2.0, size=(K, m))
    g[:, 10:] = rng.uniform(0.0, 0.9, size=(K, m))
    w[:, 10:] = _dirichlet_ones(rng, (m,), K).T
    return WalkInputs(alpha.astype(np.float32), sig.astype(np.float32),
                      g.astype(np.float32), w.astype(np.float32),
                      np.full(n, n_paths, dtype=np.uint32), None, 1.0,
                      np.full(n, 550.0, dtype=np.float32),
                      meta=dict(name="single_wavelength", param_seed=param_seed))


def _natural_spline_basis(n_knots: int, x_eval: np.ndarray) -> np.ndarray:
    """[len(x_eval)][n_knots] matrix mapping knot values to a natural cubic
    spline through equally spaced knots spanning x_eval's range."""
    from scipy.interpolate import CubicSpline
    xk = np.linspace(x_eval[0], x_eval[-1], n_knots)
    B = np.zeros((len(x_eval), n_knots))
    for j in range(n_knots):
        e = np.zeros(n_knots); e[j] = 1.0
        B[:, j] = CubicSpline(xk, e, bc_type="natural")(x_eval)
    return B


def spectral_field(n_texels: int, param_seed: int = 1, n_paths: int = 4096,
                   bands_nm: np.ndarray = VISIBLE_NM, n_rel: float = 1.4,
                   g_max: float = 0.95, chunk: int = 8192) -> WalkInputs:
    rng = np.random.default_rng(param_seed)
    K = K_MEDIA
    nb = len(bands_nm)
    B = _natural_spline_basis(4, bands_nm).astype(np.float64)   # [nb][4]
    n = n_texels * nb
    out = {k: np.empty((K, n), dtype=np.float32) for k in ("alpha", "sigma_t", "g", "w")}
    for t0 in range(0, n_texels, chunk):
        t1 = min(n_texels, t0 + chunk)
        T = t1 - t0
        ka = rng.uniform(0.5, 0.999, size=(T, K, 4))
        ks = rng.uniform(0.0, 2.0, size=(T, K, 4))
        kg = rng.uniform(0.0, g_max, size=(T, K, 4))
        kw = np.log(rng.exponential(1.0, size=(T, K, 4)))
        sa = np.clip(ka @ B.T, 0.5, 0.999)            # [T][K][nb]
        ss = 10.0 ** np.clip(ks @ B.T, 0.0, 2.0)
        sg = np.clip(kg @ B.T, 0.0, g_max)
        lw = kw @ B.T
        lw = lw - lw.max(axis=1, keepdims=True)
        ew = np.exp(lw)
        sw = ew / ew.sum(axis=1, keepdims=True)
        sl = slice(t0 * nb, t1 * nb)
        for name, v in (("alpha", sa), ("sigma_t", ss), ("g", sg), ("w", sw)):
            # [T][K][nb] -> [K][T*nb], band fastest
            out[name][:, sl] = np.transpose(v, (1, 0, 2)).reshape(K, T * nb)
    lam = np.tile(bands_nm.astype(np.float32), n_texels)
    return WalkInputs(out["alpha"], out["sigma_t"], out["g"], out["w"],
                      np.full(n, n_paths, dtype=np.uint32), None, n_rel, lam,
                      meta=dict(name="spectral_field", n_texels=n_texels, n_bands=nb,
                                param_seed=param_seed))


def uneven_batch(n_inst: int = 4096, param_seed: int = 2, log2_min: float = 10.0,
                 log2_max: float = 20.0, n_rel: float = 1.4) -> WalkInputs:
    rng = np.random.default_rng(param_seed)
    K = K_MEDIA
    alpha = rng.uniform(0.5, 0.999, size=(K, n_inst))
    sig = 10.0 ** rng.uniform(0.0, 2.0, size=(K, n_inst))
    g = rng.uniform(0.0, 0.95, size=(K, n_inst))
    w = _dirichlet_ones(rng, (n_inst,), K).T
    lam = FULL_NM_5[rng.integers(0, len(FULL_NM_5), size=n_inst)]
    n_paths = np.floor(2.0 ** rng.uniform(log2_min, log2_max, size=n_inst))
    finite = rng.uniform(size=n_inst) < 0.5
    th = np.where(finite, rng.uniform(0.1, 5.0, size=n_inst), np.inf)
    return WalkInputs(alpha.astype(np.float32), sig.astype(np.float32),
                      g.astype(np.float32), w.astype(np.float32),
                      n_paths.astype(np.uint32), th.astype(np.float32), n_rel,
                      lam.astype(np.float32),
                      meta=dict(name="uneven_batch", param_seed=param_seed))


# Layer widths of the chained decoder (Sec. 5.1): the encoder and reflectance
# decoder widths are not given in the paper (it defers to a cited work), so
# these two are stand-ins; Dec_T is 381 -> 768 -> 768 -> 768 -> 376 x 12.
DECODER_WIDTHS = {
    "enc": (3, 256, 256, 5),
    "dec_r": (5, 512, 512, 376),
    "dec_t": (381, 768, 768, 768, 376 * 12),
}


def decoder_weights(seed: int = 4) -> dict:
    """Seeded random-init weights of the chained decoder (no trained weights
    are available).  Uniform Xavier init, biases U(-0.1, 0.1).  Values are
    rounded to bfloat16 (returned as float32 holding bf16 values) so that
    every consumer sees the same numbers.  Weight matrices are [out][in]."""
    import torch
    rng = np.random.default_rng(seed)
    out = {}
    for net, dims in DECODER_WIDTHS.items():
        for l in range(len(dims) - 1):
            fan_in, fan_out = dims[l], dims[l + 1]
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            W = rng.uniform(-lim, lim, size=(fan_out, fan_in))
            b = rng.uniform(-0.1, 0.1, size=fan_out)
            Wb = torch.from_numpy(W.astype(np.float32)).to(torch.bfloat16).float().numpy()
            bb = torch.from_numpy(b.astype(np.float32)).to(torch.bfloat16).float().numpy()
            out[f"{net}{l}"] = (Wb, bb)
    return out


def two_layer_batch(n_inst: int = 1024, param_seed: int = 6, n_paths: int = 1 << 14,
                    n_rel: float = 1.4) -> WalkInputs:
    """Two-layer slabs shaped like the paper's skin model (Sec. 3): a thin,
    absorbing, forward-scattering top layer of 50-350 um over a
    semi-infinite, high-albedo second layer.  Synthetic optics (the
    chromophore spectra are not available): top alpha ~ U[0.3, 0.95],
    log10 sigma_t ~ U[1, 2] mm^-1, g ~ U[0.7, 0.9]; second alpha ~
    U[0.9, 0.999], log10 sigma_t ~ U[0.5, 1.5], g ~ U[0.6, 0.9]; one medium
    per path (K = 1)."""
    rng = np.random.default_rng(param_seed)
    f = lambda lo, hi: rng.uniform(lo, hi, size=n_inst).astype(np.float32)
    a1, s1, g1 = f(0.3, 0.95), (10 ** f(1.0, 2.0)).astype(np.float32), f(0.7, 0.9)
    a2, s2, g2 = f(0.9, 0.999), (10 ** f(0.5, 1.5)).astype(np.float32), f(0.6, 0.9)
    d1 = f(0.05, 0.35)
    one = np.ones((1, n_inst), np.float32)
    return WalkInputs(a1[None].copy(), s1[None].copy(), g1[None].copy(), one,
                      np.full(n_inst, n_paths, dtype=np.uint32), None, n_rel,
                      np.full(n_inst, 550.0, np.float32),
                      meta=dict(name="two_layer_batch", param_seed=param_seed),
                      layer2=(a2, s2, g2, d1))


def rgb_texture(side: int = 1024, seed: int = 4) -> np.ndarray:
    """float32 [side*side][3] RGB albedo from a 3-component Gaussian mixture
    per channel, clipped to [0.05, 0.85]."""
    rng = np.random.default_rng(seed)
    n = side * side
    out = np.empty((n, 3), dtype=np.float32)
    for c in range(3):
        means = rng.uniform(0.15, 0.75, size=3)
        sds = rng.uniform(0.03, 0.12, size=3)
        mix = rng.dirichlet(np.ones(3))
        comp = rng.choice(3, size=n, p=mix)
        out[:, c] = np.clip(rng.normal(means[comp], sds[comp]), 0.05, 0.85)
    return out

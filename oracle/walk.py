"""ctypes front end of the C oracle (``walk_oracle.c``).  Test infrastructure.

Inputs are plain numpy arrays in the same layout the CUDA path takes:
``alpha, sigma_t, g, w`` are float32 ``[K][n_inst]``; ``n_paths`` uint32
``[n_inst]``; ``thickness_mm`` float32 ``[n_inst]`` (+inf = semi-infinite)
or None.
"""
import ctypes as C
from dataclasses import dataclass

import numpy as np

from .build import build

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.oracle_fresnel.restype = C.c_double
        _lib.oracle_fresnel.argtypes = [C.c_double, C.c_double]
        _lib.oracle_hg_mu.restype = C.c_double
        _lib.oracle_hg_mu.argtypes = [C.c_double, C.c_double]
        _lib.oracle_hg_dlogp_dg.restype = C.c_double
        _lib.oracle_hg_dlogp_dg.argtypes = [C.c_double, C.c_double]
        _lib.oracle_select_medium.restype = C.c_int
        _lib.oracle_select_medium.argtypes = [C.c_void_p, C.c_int, C.c_double]
        _lib.oracle_rotate.restype = None
        _lib.oracle_rotate.argtypes = [C.c_void_p, C.c_double, C.c_double]
        _lib.oracle_philox4x32_10.restype = None
        _lib.oracle_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.oracle_num_threads.restype = C.c_int
        for f in ("oracle_walk", "oracle_walk_grad", "oracle_trace_many"):
            getattr(_lib, f).restype = C.c_int
    return _lib


class _Opts(C.Structure):
    _fields_ = [("nbins", C.c_int), ("r_max_mm", C.c_double), ("mode", C.c_int),
                ("rr_threshold", C.c_double), ("entry_fresnel", C.c_int),
                ("max_steps", C.c_uint32), ("seed", C.c_uint64), ("incidence", C.c_int),
                ("log_r_min_mm", C.c_double), ("select_pdf", C.c_int)]


class _Layer2(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("alpha2", "sigma_t2", "g2", "d1")]


class _Out(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in
                ("R", "T", "A", "bins", "overflow", "R_k", "R1", "truncated",
                 "se_R", "se_T", "se_A", "se_bins", "se_R_k", "se_R1", "steps")]


PATH_DTYPE = np.dtype([("exit_kind", np.int32), ("medium", np.int32), ("bin", np.int32),
                       ("weight", np.float64), ("absorbed", np.float64),
                       ("steps", np.uint32), ("n_coll", np.uint32), ("length", np.float64),
                       ("dlogp_dg", np.float64), ("x", np.float64), ("y", np.float64),
                       ("n_coll2", np.uint32), ("length2", np.float64),
                       ("dlogp_dg2", np.float64)],
                      align=True)


@dataclass
class OracleOpts:
    """Walk options.  mode 0: albedo weighting + Russian roulette at weight
    ``rr_threshold`` (0 disables roulette); mode 1: analog absorption."""
    nbins: int = 32
    r_max_mm: float = 10.0
    mode: int = 0
    rr_threshold: float = 1.0 / 16.0
    entry_fresnel: int = 1
    max_steps: int = 1 << 16
    seed: int = 1000
    incidence: int = 0
    log_r_min_mm: float = 0.0
    select_pdf: int = 0

    def _c(self):
        return _Opts(self.nbins, self.r_max_mm, self.mode, self.rr_threshold,
                     self.entry_fresnel, self.max_steps, self.seed, self.incidence,
                     self.log_r_min_mm, self.select_pdf)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _check(alpha, sigma_t, g, w):
    alpha, sigma_t, g, w = (_f32(x) for x in (alpha, sigma_t, g, w))
    K, n = alpha.shape
    for x in (sigma_t, g, w):
        assert x.shape == (K, n)
    return alpha, sigma_t, g, w, K, n


def num_threads() -> int:
    return _load().oracle_num_threads()


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: 4 counter words, 2 key words -> 4 output words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def fresnel(cos_i: float, n: float) -> float:
    return _load().oracle_fresnel(cos_i, n)


def hg_mu(g: float, u: float) -> float:
    return _load().oracle_hg_mu(g, u)


def hg_dlogp_dg(g: float, mu: float) -> float:
    return _load().oracle_hg_dlogp_dg(g, mu)


def rotate(u, mu: float, phi: float):
    v = np.array(u, dtype=np.float64)
    _load().oracle_rotate(_p(v), mu, phi)
    return v


def select_medium(w, u: float) -> int:
    w = _f32(w)
    return _load().oracle_select_medium(_p(w), len(w), u)


def _ids(inst_ids, n):
    if inst_ids is None:
        return None
    a = np.ascontiguousarray(inst_ids, dtype=np.int64)
    assert a.shape == (n,)
    return a


def walk(alpha, sigma_t, g, w, n_paths, thickness_mm=None, n_rel=1.0,
         opts: OracleOpts = OracleOpts(), path_offset: int = 0, inst_ids=None,
         layer2=None) -> dict:
    """Mean tallies per instance (fractions of incident power) and their
    standard errors; see ``oracle_walk`` in ``walk_oracle.c``.  ``inst_ids``
    re-walks a subset of a larger batch under the instance numbers the
    random-number counters had there.  ``layer2`` = (alpha2, sigma_t2, g2, d1),
    float32 [n_inst] each, puts a second layer under the chosen medium:
    the medium fills 0 <= z < d1, the second layer d1 <= z < thickness."""
    alpha, sigma_t, g, w, K, n = _check(alpha, sigma_t, g, w)
    l2 = None
    keep = None
    if layer2 is not None:
        keep = [_f32(a) for a in layer2]
        assert all(k.shape == (n,) for k in keep)
        l2 = _Layer2(*(_p(k) for k in keep))
    n_paths = np.ascontiguousarray(n_paths, dtype=np.uint32)
    assert n_paths.shape == (n,)
    th = None if thickness_mm is None else _f32(thickness_mm)
    nb = opts.nbins
    res = {k: np.zeros(n) for k in ("R", "T", "A", "overflow", "R1", "truncated",
                                    "se_R", "se_T", "se_A", "se_R1", "steps")}
    res["bins"] = np.zeros((n, nb))
    res["se_bins"] = np.zeros((n, nb))
    res["R_k"] = np.zeros((n, K))
    res["se_R_k"] = np.zeros((n, K))
    out = _Out(**{k: _p(v) for k, v in res.items()})
    ids = _ids(inst_ids, n)
    o = opts._c()
    rc = _load().oracle_walk(C.c_int64(n), C.c_int(K), _p(alpha), _p(sigma_t), _p(g),
                             _p(w), _p(n_paths), _p(th), C.c_double(n_rel), C.byref(o),
                             C.c_uint32(path_offset), _p(ids),
                             C.byref(l2) if l2 is not None else None, C.byref(out))
    if rc != 0:
        raise ValueError("oracle_walk rejected its arguments")
    return res


def walk_hero(alpha, sigma_t, g, w, n_paths_per_group: int, hero: int, bands_per_texel: int,
              thickness_mm=None, n_rel=1.0, opts: OracleOpts = OracleOpts(),
              inst_offset: int = 0, orbits: bool = False) -> dict:
    """Hero-wavelength walk (see ``oracle_walk_hero`` in ``walk_oracle.c``):
    instances are texels x ``bands_per_texel`` bands, band fastest; each group
    of ``hero`` bands (adjacent, or with ``orbits`` the rotation orbits of
    stride bands_per_texel / hero) shares ``n_paths_per_group`` path
    geometries, each member scoring the balance-heuristic estimate.  Returns the same per-instance dict as
    ``walk`` (A and se_A are 0)."""
    alpha, sigma_t, g, w, K, n = _check(alpha, sigma_t, g, w)
    th = None if thickness_mm is None else _f32(thickness_mm)
    nb = opts.nbins
    res = {k: np.zeros(n) for k in ("R", "T", "A", "overflow", "R1", "truncated",
                                    "se_R", "se_T", "se_A", "se_R1", "steps")}
    res["bins"] = np.zeros((n, nb))
    res["se_bins"] = np.zeros((n, nb))
    res["R_k"] = np.zeros((n, K))
    res["se_R_k"] = np.zeros((n, K))
    out = _Out(**{k: _p(v) for k, v in res.items()})
    o = opts._c()
    rc = _load().oracle_walk_hero(C.c_int64(n), C.c_int(K), _p(alpha), _p(sigma_t), _p(g),
                                  _p(w), C.c_uint32(n_paths_per_group), _p(th),
                                  C.c_double(n_rel), C.byref(o), C.c_int(hero),
                                  C.c_int(bands_per_texel), C.c_int(int(orbits)),
                                  C.c_uint32(inst_offset),
                                  C.byref(out))
    if rc != 0:
        raise ValueError("oracle_walk_hero rejected its arguments")
    return res


def walk_grad(alpha, sigma_t, g, w, n_paths, thickness_mm=None, n_rel=1.0,
              opts: OracleOpts = OracleOpts(), grad_R=None, grad_bins=None,
              grad_R_k=None, grad_T=None, inst_ids=None, layer2=None) -> dict:
    """Score-function gradient of sum(upstream * tallies) w.r.t. the
    per-medium parameters, shape [K][n_inst] each, with standard errors.
    With ``layer2`` (as in ``walk``) the per-medium terms cover the top layer
    and d_alpha2, d_sigma_t2, d_g2 ([n_inst]) the second layer's optics."""
    alpha, sigma_t, g, w, K, n = _check(alpha, sigma_t, g, w)
    l2 = None
    keep = None
    if layer2 is not None:
        keep = [_f32(a) for a in layer2]
        l2 = _Layer2(*(_p(k) for k in keep))
    n_paths = np.ascontiguousarray(n_paths, dtype=np.uint32)
    th = None if thickness_mm is None else _f32(thickness_mm)

    def f64(a, shape):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.shape == shape
        return a
    gR = f64(grad_R, (n,))
    gB = f64(grad_bins, (n, opts.nbins))
    gK = f64(grad_R_k, (n, K))
    gT = f64(grad_T, (n,))
    res = {k: np.zeros((K, n)) for k in ("d_alpha", "d_sigma_t", "d_g", "d_w",
                                         "se_d_alpha", "se_d_sigma_t", "se_d_g", "se_d_w")}
    for k in ("d_alpha2", "d_sigma_t2", "d_g2", "se_d_alpha2", "se_d_sigma_t2", "se_d_g2"):
        res[k] = np.zeros(n)
    o = opts._c()
    rc = _load().oracle_walk_grad(
        C.c_int64(n), C.c_int(K), _p(alpha), _p(sigma_t), _p(g), _p(w), _p(n_paths),
        _p(th), C.c_double(n_rel), C.byref(o), _p(_ids(inst_ids, n)),
        C.byref(l2) if l2 is not None else None,
        _p(gR), _p(gB), _p(gK), _p(gT),
        *[_p(res[k]) for k in ("d_alpha", "d_sigma_t", "d_g", "d_w",
                               "se_d_alpha", "se_d_sigma_t", "se_d_g", "se_d_w",
                               "d_alpha2", "d_sigma_t2", "d_g2",
                               "se_d_alpha2", "se_d_sigma_t2", "se_d_g2")])
    if rc != 0:
        raise ValueError("oracle_walk_grad rejected its arguments")
    return res


def trace(alpha, sigma_t, g, w, inst, path, thickness_mm=None, n_rel=1.0,
          opts: OracleOpts = OracleOpts()):
    """Per-path records (``PATH_DTYPE``) for the given (instance, path) pairs."""
    alpha, sigma_t, g, w, K, n = _check(alpha, sigma_t, g, w)
    inst = np.ascontiguousarray(inst, dtype=np.int64)
    path = np.ascontiguousarray(path, dtype=np.uint32)
    assert inst.shape == path.shape
    th = None if thickness_mm is None else _f32(thickness_mm)
    res = np.zeros(inst.shape[0], dtype=PATH_DTYPE)
    o = opts._c()
    rc = _load().oracle_trace_many(C.c_int64(n), C.c_int(K), _p(alpha), _p(sigma_t),
                                   _p(g), _p(w), _p(th), C.c_double(n_rel), C.byref(o),
                                   C.c_int64(len(inst)), _p(inst), _p(path), _p(res))
    if rc != 0:
        raise ValueError("oracle_trace_many rejected its arguments")
    return res

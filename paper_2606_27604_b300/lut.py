"""Scale-independent lookup tables of a homogeneous medium (paper Sec. 4.2).

For a homogeneous semi-infinite slab the normalised radial profile depends
on (alpha, g) only, and extinction rescales the radial axis (Eq. 5):
P_d(r | alpha, sigma_t) = sigma_t^2 P_d(sigma_t r | alpha, 1), while the total
reflectance R does not depend on sigma_t at all.  So one walk per (alpha, g)
grid point at sigma_t = 1 gives the two tables used by the mixture fit:

  R_lut[i][j]       = R(alpha_i, g_j)
  P_lut[i][j][b]    = fraction of R leaving through annulus b of the radial
                      axis in mean free paths (bins of width r_max / nbins)

Every grid point is one instance of the batched walk (K = 1, sigma_t = 1),
so the whole table is one persistent launch per chunk of the grid.
"""
from dataclasses import dataclass

import numpy as np
import torch

from . import api


@dataclass
class Lut:
    alphas: np.ndarray      # [na]
    gs: np.ndarray          # [ng]
    r_max: float            # in mean free paths
    R: np.ndarray           # [na][ng]
    P: np.ndarray           # [na][ng][nbins], annulus fractions of R
    se_R: np.ndarray        # [na][ng]
    n_paths: int
    n_rel: float

    def density(self) -> np.ndarray:
        """P as a density per unit area (mfp^-2) at the bin centres."""
        nb = self.P.shape[-1]
        edges = np.linspace(0.0, self.r_max, nb + 1)
        area = np.pi * (edges[1:] ** 2 - edges[:-1] ** 2)
        return self.P / area


def grid_inputs(alphas, gs):
    """Media arrays (K = 1, sigma_t = 1, w = 1) for the (alpha, g) grid,
    instance i = ia * len(gs) + ig."""
    A, G = np.meshgrid(np.asarray(alphas, np.float32), np.asarray(gs, np.float32), indexing="ij")
    n = A.size
    return (A.reshape(1, n).copy(), np.ones((1, n), np.float32), G.reshape(1, n).copy(),
            np.ones((1, n), np.float32))


def build(alphas, gs, n_paths: int, nbins: int = 128, r_max: float = 32.0,
          n_rel: float = 1.4, seed: int = 2024, chunk: int = 1 << 16,
          device="cuda") -> Lut:
    """Walks every grid point with n_paths paths (mode: albedo weighting with
    roulette, Fresnel faces with relative index n_rel, normal incidence)."""
    a, s, g, w = grid_inputs(alphas, gs)
    n = a.shape[1]
    R = np.empty(n)
    se = np.empty(n)
    P = np.empty((n, nbins))
    dev = torch.device(device)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        t = lambda arr: torch.from_numpy(np.ascontiguousarray(arr[:, c0:c1])).to(dev)
        m = api.Media(t(a), t(s), t(g), t(w), None, n_paths, None, n_rel)
        o = api.WalkOptions(nbins=nbins, r_max_mm=r_max, seed=seed, instance_offset=c0)
        d = lambda *shape: torch.empty(*shape, dtype=torch.float64, device=dev)
        out = api.walk(m, o, out={"R": d(c1 - c0), "stderr_R": d(c1 - c0),
                                  "profile": d(c1 - c0, nbins)})
        torch.cuda.synchronize(dev)
        code, flags = api.read_status(out["_workspace"])
        if code != 0:
            raise api.SSSError(code, "LUT walk")
        R[c0:c1] = out["R"].cpu().numpy()
        se[c0:c1] = out["stderr_R"].cpu().numpy()
        P[c0:c1] = out["profile"].cpu().numpy()   # bins / R (Eq. 3), on the GPU
    na, ng = len(alphas), len(gs)
    return Lut(np.asarray(alphas, np.float64), np.asarray(gs, np.float64), r_max,
               R.reshape(na, ng), P.reshape(na, ng, nbins), se.reshape(na, ng), n_paths, n_rel)

"""Closed forms for the isotropic, index-matched, semi-infinite half-space
under collimated normal incidence (test infrastructure).

These are the exact values the random walk must reproduce when every medium
of the mixture (Sec. 4.1, Eq. 4) is the same isotropic medium (g = 0), the
boundary is index matched (n = 1) and light enters along the normal (Eq. 3).

* Chandrasekhar's H-function for single-scattering albedo ``alpha`` and
  isotropic scattering (characteristic function alpha/2) solves
      1/H(mu) = sqrt(1-alpha) + (alpha/2) * int_0^1 mu' H(mu') / (mu + mu') dmu'
  (Chandrasekhar, Radiative Transfer, 1950, Ch. V).  It is solved here by
  fixed-point iteration on a Gauss-Legendre rule over [0, 1].
* Total diffuse reflectance (all orders) for incidence cosine mu0:
      R(mu0) = 1 - H(mu0) * sqrt(1 - alpha).
* Single-scatter reflectance for mu0 = 1, from integrating the once-scattered
  beam over depth and the upward hemisphere:
      R1 = (alpha/2) * int_0^1 mu / (1 + mu) dmu = alpha * (1 - ln 2) / 2.
"""
import numpy as np


def _gl01(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def h_nodes(alpha: float, n: int = 400, tol: float = 1e-15, max_iter: int = 200000):
    """H on the Gauss-Legendre nodes of [0,1]: returns (mu, weights, H)."""
    mu, wq = _gl01(n)
    s = np.sqrt(max(0.0, 1.0 - alpha))
    H = np.ones(n)
    kern = mu[None, :] / (mu[:, None] + mu[None, :])  # mu' / (mu + mu')
    for _ in range(max_iter):
        Hn = 1.0 / (s + 0.5 * alpha * (kern * (wq * H)[None, :]).sum(axis=1))
        if np.max(np.abs(Hn - H)) < tol:
            H = Hn
            break
        H = Hn
    return mu, wq, H


def h_function(alpha: float, mu, n: int = 400):
    """H(mu) at arbitrary mu in [0, 1] from the converged node values."""
    nodes, wq, Hn = h_nodes(alpha, n)
    mu = np.atleast_1d(np.asarray(mu, dtype=np.float64))
    s = np.sqrt(max(0.0, 1.0 - alpha))
    integral = (nodes[None, :] * wq[None, :] * Hn[None, :]
                / (mu[:, None] + nodes[None, :])).sum(axis=1)
    return 1.0 / (s + 0.5 * alpha * integral)


def reflectance_total(alpha: float, mu0: float = 1.0, n: int = 400) -> float:
    """R = 1 - H(mu0) sqrt(1-alpha): diffuse reflectance, all orders."""
    return float(1.0 - h_function(alpha, [mu0], n)[0] * np.sqrt(1.0 - alpha))


def reflectance_single(alpha: float) -> float:
    """Order-1 reflectance at mu0 = 1: alpha (1 - ln 2) / 2."""
    return alpha * (1.0 - np.log(2.0)) / 2.0


def reflectance_total_dalpha(alpha: float, h: float = 1e-6, n: int = 400) -> float:
    """dR/dalpha by a central difference of the closed form."""
    return (reflectance_total(alpha + h, n=n) - reflectance_total(alpha - h, n=n)) / (2 * h)


def reflectance_cosine_lobe(alpha: float, n: int = 400) -> float:
    """Diffuse reflectance under a cosine-weighted incident lobe,
    2 int_0^1 R(mu) mu dmu = 1 - 2 sqrt(1 - alpha) int_0^1 H(mu) mu dmu."""
    mu, wq, H = h_nodes(alpha, n)
    return float(1.0 - 2.0 * np.sqrt(1.0 - alpha) * (wq * H * mu).sum())

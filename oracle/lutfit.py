"""FP64 reference of the LUT-based mixture fit (paper Sec. 4.2, Eq. 6-9).
Test infrastructure.

Tables (inputs, any source): R_lut[i][j] = R(alpha_i, g_j) and the radial
density p_lut[i][j][b] at sigma_t = 1, on uniform grids alpha_i = a0 + i da,
g_j = g0 + j dg, rho_b = (b + 1/2) drho.

Model of one (tone, wavelength) problem with K media (Eq. 6 and the text
after Eq. 9):
    R_hat     = sum_k w_k R(alpha_k, g_k)                       (bilinear)
    P_hat(r)  = sum_k w_k P(r | alpha_k, g_k, sigma_k),
    P(r | alpha, g, sigma) = sigma^2 p(sigma r | alpha, g)      (Eq. 5; trilinear)
    L = RMSE_j(log P_hat(r_j), log P_MC(r_j)) + lambda_R (R_hat - R_MC)^2
over the radii with P_MC > 0, lambda_R = 5 (Eq. 7-9).

Readings (the paper gives sigma_t = exp(raw) and Adam with a cosine
schedule, lr = 1e-2): alpha = a_lo + (a_hi - a_lo) sigmoid(raw), likewise
g, sigma_t = exp(raw), w = softmax(raw); table lookups clamp to the grid;
Adam with beta = (0.9, 0.999), eps = 1e-8, lr_t = lr (1 + cos(pi t / S)) / 2.
Raw parameter layout per problem: [alpha_raw K][g_raw K][log sigma K][w_raw K].
"""
import numpy as np


class Tables:
    def __init__(self, R, p, a0, da, g0, dg, drho):
        self.R = np.asarray(R, np.float64)
        self.p = np.asarray(p, np.float64)
        self.a0, self.da, self.g0, self.dg, self.drho = a0, da, g0, dg, drho

    def _cell(self, x, x0, dx, n):
        u = (x - x0) / dx
        i = int(np.clip(np.floor(u), 0, n - 2))
        f = float(np.clip(u - i, 0.0, 1.0))
        inside = 0.0 <= u <= n - 1
        return i, f, inside

    def R_at(self, a, g):
        """R and (dR/da, dR/dg) by bilinear interpolation."""
        na, ng = self.R.shape
        i, fa, ia = self._cell(a, self.a0, self.da, na)
        j, fg, ig = self._cell(g, self.g0, self.dg, ng)
        c00, c10 = self.R[i, j], self.R[i + 1, j]
        c01, c11 = self.R[i, j + 1], self.R[i + 1, j + 1]
        v = (1 - fa) * (1 - fg) * c00 + fa * (1 - fg) * c10 + (1 - fa) * fg * c01 + fa * fg * c11
        da = ((c10 - c00) * (1 - fg) + (c11 - c01) * fg) / self.da if ia else 0.0
        dg = ((c01 - c00) * (1 - fa) + (c11 - c10) * fa) / self.dg if ig else 0.0
        return v, da, dg

    def p_at(self, a, g, rho):
        """p and (dp/da, dp/dg, dp/drho) by trilinear interpolation."""
        na, ng, nb = self.p.shape
        i, fa, ia = self._cell(a, self.a0, self.da, na)
        j, fg, ig = self._cell(g, self.g0, self.dg, ng)
        b, fb, ib = self._cell(rho, 0.5 * self.drho, self.drho, nb)
        c = self.p[i:i + 2, j:j + 2, b:b + 2]
        wa = np.array([1 - fa, fa]); wg = np.array([1 - fg, fg]); wb = np.array([1 - fb, fb])
        v = np.einsum("i,j,k,ijk->", wa, wg, wb, c)
        da = np.einsum("j,k,jk->", wg, wb, c[1] - c[0]) / self.da if ia else 0.0
        dg = np.einsum("i,k,ik->", wa, wb, c[:, 1] - c[:, 0]) / self.dg if ig else 0.0
        dr = np.einsum("i,j,ij->", wa, wg, c[:, :, 1] - c[:, :, 0]) / self.drho if ib else 0.0
        return v, da, dg, dr


def unpack(raw, K, a_rng, g_rng):
    ar, gr, sr, wr = raw[0:K], raw[K:2 * K], raw[2 * K:3 * K], raw[3 * K:4 * K]
    sa = 1 / (1 + np.exp(-ar)); sg = 1 / (1 + np.exp(-gr))
    alpha = a_rng[0] + (a_rng[1] - a_rng[0]) * sa
    g = g_rng[0] + (g_rng[1] - g_rng[0]) * sg
    sig = np.exp(sr)
    e = np.exp(wr - wr.max()); w = e / e.sum()
    return alpha, g, sig, w, sa, sg


def loss_grad(raw, K, tab, r, P_mc, R_mc, lam_R=5.0, a_rng=(0.0, 0.999), g_rng=(0.0, 0.95)):
    """Joint loss and its gradient w.r.t. the raw parameters."""
    raw = np.asarray(raw, np.float64)
    alpha, g, sig, w, sa, sg = unpack(raw, K, a_rng, g_rng)
    m = P_mc > 0
    rj, Pj = r[m], P_mc[m]
    n = len(rj)
    Rk = np.zeros(K); dRa = np.zeros(K); dRg = np.zeros(K)
    for k in range(K):
        Rk[k], dRa[k], dRg[k] = tab.R_at(alpha[k], g[k])
    Rhat = (w * Rk).sum()
    P = np.zeros((K, n)); dPa = np.zeros((K, n)); dPg = np.zeros((K, n)); dPs = np.zeros((K, n))
    for k in range(K):
        for t in range(n):
            v, da, dg, dr = tab.p_at(alpha[k], g[k], sig[k] * rj[t])
            s2 = sig[k] ** 2
            P[k, t] = s2 * v
            dPa[k, t] = s2 * da
            dPg[k, t] = s2 * dg
            dPs[k, t] = 2 * sig[k] * v + s2 * rj[t] * dr
    Phat = (w[:, None] * P).sum(0)
    e = np.log(Phat) - np.log(Pj)
    Ls = np.sqrt((e ** 2).mean())
    L = Ls + lam_R * (Rhat - R_mc) ** 2
    # d L / d Phat_t and d L / d Rhat
    gP = e / (n * Ls) / Phat if Ls > 0 else np.zeros(n)
    gR = 2 * lam_R * (Rhat - R_mc)
    d_alpha = w * ((dPa * gP).sum(1) + gR * dRa)
    d_g = w * ((dPg * gP).sum(1) + gR * dRg)
    d_sig = w * (dPs * gP).sum(1)
    d_w = (P * gP).sum(1) + gR * Rk
    grad = np.zeros(4 * K)
    grad[0:K] = d_alpha * (a_rng[1] - a_rng[0]) * sa * (1 - sa)
    grad[K:2 * K] = d_g * (g_rng[1] - g_rng[0]) * sg * (1 - sg)
    grad[2 * K:3 * K] = d_sig * sig
    grad[3 * K:4 * K] = w * (d_w - (w * d_w).sum())  # softmax Jacobian
    return L, grad


def fit(raw0, K, tab, r, P_mc, R_mc, steps, lr=1e-2, lam_R=5.0, a_rng=(0.0, 0.999),
        g_rng=(0.0, 0.95), b1=0.9, b2=0.999, eps=1e-8):
    """Adam with a cosine learning-rate schedule; returns (raw, loss)."""
    raw = np.array(raw0, np.float64)
    m = np.zeros_like(raw); v = np.zeros_like(raw)
    for t in range(1, steps + 1):
        _, gr = loss_grad(raw, K, tab, r, P_mc, R_mc, lam_R, a_rng, g_rng)
        m = b1 * m + (1 - b1) * gr
        v = b2 * v + (1 - b2) * gr * gr
        mh = m / (1 - b1 ** t); vh = v / (1 - b2 ** t)
        lr_t = lr * 0.5 * (1 + np.cos(np.pi * (t - 1) / steps))
        raw = raw - lr_t * mh / (np.sqrt(vh) + eps)
    L, _ = loss_grad(raw, K, tab, r, P_mc, R_mc, lam_R, a_rng, g_rng)
    return raw, L

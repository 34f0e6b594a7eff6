"""FP64 reference of the chained decoder RGB -> per-band mixture parameters
(test infrastructure; paper Sec. 5.1, Eq. 10).

Enc(A_RGB) -> p (5); Dec_R(p) -> R_d (376 bands, 250-1000 nm at 2 nm);
Dec_T(p, R_d) -> theta(lambda) in R^{376 x 4K}, K = 3, per band and medium
(alpha_k, g_k, sigma_t,k, w_k).  Dec_T is a 4-layer MLP 381 -> 768 -> 768 ->
768 -> 376*12 with tanh hidden activations and sigmoid outputs; the weight
channels instead take a softmax over the K media so they sum to one.

Readings where the paper is silent (Enc/Dec_R widths are deferred to a cited
work): Enc and Dec_R hidden layers use tanh and their outputs a sigmoid;
sigma_t = 10^(3 s) mm^-1 from the sigmoid output s; the 376 bands are
resampled linearly to the 81 visible bands 380-780 nm at 5 nm after the
activations.  Output instance order is band-major (i = band * T + texel).

``bf16_activations=True`` rounds every stored activation (hidden layers,
p and R_d) to bfloat16, the precision the GPU stores them in; everything
else is float64.
"""
import numpy as np

N_SRC = 376
SRC_NM0, SRC_STEP = 250.0, 2.0
DST_NM = np.arange(380.0, 780.0 + 1e-9, 5.0)
K = 3


def _bf16(x):
    import torch
    return torch.from_numpy(np.asarray(x, np.float64)).to(torch.bfloat16).double().numpy()


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _mlp(x, layers, out_act, round_bf16):
    """Linear -> tanh for all but the last layer; `out_act` on the last."""
    h = x
    for i, (W, b) in enumerate(layers):
        z = h @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        last = i == len(layers) - 1
        h = (out_act(z) if out_act else z) if last else np.tanh(z)
        if round_bf16 and not (last and out_act is None):
            h = _bf16(h)
    return h


def resample_matrix():
    """[81][376] linear interpolation from the 2-nm source grid."""
    M = np.zeros((len(DST_NM), N_SRC))
    for j, nm in enumerate(DST_NM):
        x = (nm - SRC_NM0) / SRC_STEP
        lo = int(np.floor(x))
        f = x - lo
        M[j, lo] += 1.0 - f
        if f > 0:
            M[j, lo + 1] += f
    return M


def decode(rgb, weights, bf16_activations=False, return_intermediates=False):
    """rgb float [T][3]; weights dict from the seeded generator
    ({"enc0": (W, b), ...}, W as [out][in]).  Returns float64 SoA arrays
    alpha, g, sigma_t, w of shape [K][81 * T] (band-major)."""
    x = np.asarray(rgb, np.float64)
    enc = [weights[f"enc{i}"] for i in range(3)]
    decr = [weights[f"dec_r{i}"] for i in range(3)]
    dect = [weights[f"dec_t{i}"] for i in range(4)]
    p = _mlp(x, enc, _sigmoid, bf16_activations)            # [T][5]
    Rd = _mlp(p, decr, _sigmoid, bf16_activations)          # [T][376]
    z = _mlp(np.concatenate([p, Rd], axis=1), dect, None, bf16_activations)  # [T][4512]
    T = x.shape[0]
    z = z.reshape(T, N_SRC, K, 4)                            # (alpha, g, sigma_t, w)
    alpha = _sigmoid(z[..., 0])
    g = _sigmoid(z[..., 1])
    sig = 10.0 ** (3.0 * _sigmoid(z[..., 2]))
    lw = z[..., 3]
    lw = lw - lw.max(axis=2, keepdims=True)
    ew = np.exp(lw)
    w = ew / ew.sum(axis=2, keepdims=True)
    R = resample_matrix()                                    # [81][376]
    out = {}
    for name, v in (("alpha", alpha), ("g", g), ("sigma_t", sig), ("w", w)):
        r = np.einsum("js,tsk->kjt", R, v)                  # [K][81][T]
        out[name] = r.reshape(K, len(DST_NM) * T)
    if return_intermediates:
        out["p"] = p
        out["R_d"] = Rd
        out["logits"] = z
    return out

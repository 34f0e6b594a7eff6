"""Shared helpers for the GPU tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs, and compare them."""
import numpy as np

import oracle


def to_oracle_opts(o):
    return oracle.OracleOpts(nbins=o.nbins, r_max_mm=o.r_max_mm, mode=o.mode,
                             rr_threshold=o.rr_threshold, entry_fresnel=o.entry_fresnel,
                             max_steps=o.max_steps, seed=o.seed,
                             incidence=getattr(o, "incidence", 0),
                             log_r_min_mm=getattr(o, "log_r_min_mm", 0.0),
                             select_pdf=getattr(o, "select_pdf", 0))


def run_gpu(x, o, raw=False, media=None):
    import torch
    from paper_2606_27604_b300 import api
    m = media if media is not None else api.Media.from_inputs(x)
    r = api.walk(m, o, raw=raw)
    torch.cuda.synchronize()
    code, flags = api.read_status(r["_workspace"])
    out = {k: v.cpu().numpy() for k, v in r.items() if not k.startswith("_")}
    return out, code, flags


def run_oracle(x, o, inst_ids=None, path_offset=0):
    return oracle.walk(x.alpha, x.sigma_t, x.g, x.w, x.n_paths, x.thickness_mm, x.n_rel,
                       to_oracle_opts(o), path_offset=path_offset, inst_ids=inst_ids,
                       layer2=getattr(x, "layer2", None))


TALLIES = ("R", "T", "A", "bins", "overflow", "R_k", "R1")


def same_stream_tolerance(ref, N, steps):
    """Allowed |GPU - oracle| for one tally when both sides walk the same
    Philox streams.  Two effects, derived from the arithmetic:
      * binary32 rounding of the weight products: W = W0 * alpha^n carries a
        relative error of about n * 2^-24 -> 1e-5 relative covers n < 160
        with a margin of two, and long paths are rare;
      * paths whose binary32 trajectory takes another branch than the
        binary64 one (a flight ending just before/after a face, a radius on
        a bin edge, a roulette draw near W/W_th): each moves at most its
        weight (<= 1) from one tally to another, i.e. 1/N of a tally.  With
        about 1e-6 such flips per draw, an instance of N paths averaging
        `steps` draws sees about 1e-6 * N * steps of them; the bound allows
        8 + 4x that count (Poisson tail) per tally.
    """
    flips = 8.0 + 4.0 * 1e-6 * N * steps
    return 1e-5 * np.abs(ref) + flips / N


def compare_same_stream(g, r, N, steps, keys=TALLIES):
    """Returns the worst ratio |diff| / tolerance over all tallies (<= 1 passes)."""
    worst = 0.0
    where = None
    Nb = np.asarray(N, dtype=np.float64)
    st = np.asarray(steps, dtype=np.float64)
    for k in keys:
        a, b = np.asarray(g[k], np.float64), np.asarray(r[k], np.float64)
        n = Nb.reshape((-1,) + (1,) * (a.ndim - 1))
        s = st.reshape((-1,) + (1,) * (a.ndim - 1))
        tol = same_stream_tolerance(b, n, s)
        ratio = np.abs(a - b) / tol
        if ratio.size and ratio.max() > worst:
            worst = float(ratio.max())
            where = (k, np.unravel_index(int(ratio.argmax()), ratio.shape), float(a.flat[ratio.argmax()]),
                     float(b.flat[ratio.argmax()]))
    return worst, where


def compare_sigma(g, r, keys=("R", "bins", "R1"), z=4.0, max_rel_se=0.2):
    """The statistical bar: |GPU - oracle| <= z * sqrt(se_gpu^2 + se_oracle^2),
    using the oracle's standard errors for both sides (same N, so the two
    variances are equal).  The bar is a normal-approximation bound, so it is
    applied where the tally is supported by enough paths for that
    approximation: relative standard error <= max_rel_se (0.2: about 25 or
    more contributing paths).  A sparser tally (a far radial bin holding a
    handful of exits) is held only by the same-stream bound, where one
    binary32 path flip (one exit weight / N) is allowed for."""
    bad = []
    for k in keys:
        a, b = np.asarray(g[k]), np.asarray(r[k])
        se = np.asarray(r["se_" + k])
        se_g = np.asarray(g["stderr_" + k]) if ("stderr_" + k) in g else se
        lim = z * np.sqrt(2.0) * se + 1e-15
        # relative standard error on each side; an empty tally on either side
        # (0 / 0) is not supported
        with np.errstate(divide="ignore", invalid="ignore"):
            rel = np.maximum(np.where(b != 0, se / np.abs(b), np.inf),
                             np.where(a != 0, se_g / np.abs(a), np.inf))
        supported = rel <= max_rel_se
        viol = (np.abs(a - b) > lim) & supported
        if viol.any():
            bad.append((k, int(viol.sum())))
    return bad

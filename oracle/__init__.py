"""FP64 CPU oracle for the mixture-of-media random walk (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA path: the walk
is plain C in double precision (``walk_oracle.c``), the closed forms are
numpy (``hfunction.py``), the decoder reference is numpy float64
(``decoder.py``).

Citations are to the paper's sections and equations:
  * Sec. 4.1, Eq. 2 and the display after it: path contribution f_SSS;
  * Sec. 4.1, Eq. 3: radial form R_d(r) = R * P_d(r) under normal incidence;
  * Sec. 4.1, Eq. 4: mixture S = sum_k w_k S_k, one medium per path;
  * Sec. 7: the medium is drawn with probability w_k at the walk start.
"""
from .walk import (OracleOpts, philox4x32_10, fresnel, hg_mu, hg_dlogp_dg, rotate,
                   select_medium, walk, walk_grad, walk_hero, trace, num_threads,
                   PATH_DTYPE)
from . import hfunction

__all__ = ["OracleOpts", "philox4x32_10", "fresnel", "hg_mu", "hg_dlogp_dg", "rotate",
           "select_medium", "walk", "walk_grad", "walk_hero", "trace", "num_threads",
           "PATH_DTYPE",
           "hfunction"]

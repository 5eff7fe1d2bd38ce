"""Comparing PCG stopping steps against a reference residual history.

Two FP64 CG runs that sum in different orders (the GPU's batched kernels and
the oracle's per-subdomain LAPACK solves) follow the same residual history
||P r_k|| / ||P r_0|| only to a few percent once it is near 1e-8: on the
16-subdomain tube (cylinder 4 x 16 x 8 cells, 2 x 4 x 2 parts, all-floating,
Dirichlet) the two histories read 2.202e-8 / 2.204e-8 at step 31, 1.007e-8 /
0.968e-8 at step 32.  Where the reference history passes within such a band
of the tolerance, the step that first reaches the tolerance is defined only
up to the steps inside the band, so a stopping count is compared against the
reference's first steps at tol (1 + band) and tol (1 - band), each +-1.
"""
import numpy as np


def count_bracket(res_hist, tol: float, band: float = 0.05):
    """(lo, hi): the first steps of the reference history (index = PCG step,
    entry 0 = ||P r_0||) whose relative residual is at most tol (1 + band) and
    at most tol (1 - band)."""
    h = np.asarray(res_hist, dtype=np.float64)
    h = h / h[0]
    lo = next(k for k, v in enumerate(h) if v <= tol * (1.0 + band))
    hi = next(k for k, v in enumerate(h) if v <= tol * (1.0 - band))
    return lo, hi


def count_matches(n: int, res_hist, tol: float, band: float = 0.05) -> bool:
    """True when stopping step n is within one step of the reference's band."""
    lo, hi = count_bracket(res_hist, tol, band)
    return lo - 1 <= n <= hi + 1

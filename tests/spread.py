"""Iteration-count window for solves whose count is decided by rounding.

On ill-conditioned systems the number of iterations ML(n)BiCGStab needs to
reach tol moves by several percent when one entry of b moves by one ulp,
so a count computed with another summation order (the GPU's reduction
trees) is not expected to equal the oracle's.  The window is derived from
the oracle's own spread: the counts of m = 16 solves whose right-hand sides
differ from b by one ulp in one entry each, plus b itself (17 samples).
Treating the GPU's count as one more draw from the same distribution, the
two-sided 99.9 % normal prediction interval is

    mean +- t_{0.9995, 16} * s * sqrt(1 + 1/17),

with s the sample standard deviation (t_{0.9995, 16} = 4.015).  The
interval is widened to include every sample (it always does for the
sample sizes here) and is never narrower than +-1 iteration.
"""
from __future__ import annotations

import numpy as np

import oracle as O

T_9995_16 = 4.015   # Student t quantile, 0.9995, 16 degrees of freedom
PERTURBATIONS = 16


def perturbed(b, k):
    """b with entry (k * 7919) mod N moved up by one ulp (k = 1, 2, ...)."""
    bb = b.copy()
    t = (k * 7919) % len(b)
    if np.iscomplexobj(bb):
        bb[t] = np.nextafter(bb[t].real, np.inf) + 1j * bb[t].imag
    else:
        bb[t] = np.nextafter(bb[t], np.inf)
    return bb


def window(counts):
    c = np.asarray(counts, dtype=float)
    m = len(c)
    mean, s = float(np.mean(c)), float(np.std(c, ddof=1))
    half = max(T_9995_16 * s * np.sqrt(1.0 + 1.0 / m), 1.0)
    return min(mean - half, float(c.min())), max(mean + half, float(c.max()))


def oracle_counts(solve_one, b):
    """Counts of solve_one(rhs) -> iterations for b and its perturbations."""
    return [solve_one(b)] + [solve_one(perturbed(b, k)) for k in range(1, PERTURBATIONS + 1)]


def oracle_window(A, b, Q, tol, maxit, kappa=0.0, restarts=False, lib=None):
    """The window above for one call of the method (restarts=False) or for
    the restart wrapper O.solve (restarts=True)."""
    x0 = np.zeros_like(b)
    if restarts:
        def one(rhs):
            return O.solve(A, rhs, x0, Q, maxit, tol, kappa, lib=lib).iter
    else:
        def one(rhs):
            return O.mlbicgstabt(A, rhs, x0, Q, maxit, tol, kappa, lib=lib).iter
    counts = oracle_counts(one, b)
    return window(counts), counts


def unique_prefix(A, b, Q, K, rel=1e-12, **kw):
    """The oracle's residual history over K steps, and the last step k <= K
    up to which that history does not depend on the order of the oracle's
    sums (its sequential and fixed-block builds agree to `rel`): only that
    prefix is determined by the method rather than by rounding.  On systems
    whose early steps amplify rounding (a residual that jumps by orders of
    magnitude), the prefix ends early."""
    x0 = np.zeros_like(b)
    ref = O.mlbicgstabt(A, b, x0, Q, K, 0.0, err_hist=True, **kw)
    alt = O.mlbicgstabt(A, b, x0, Q, K, 0.0, err_hist=True, lib=O.load_par(), **kw)
    agree = np.abs(alt.err_hist - ref.err_hist) <= rel * ref.err_hist
    k = K if agree.all() else int(np.argmin(agree)) - 1
    return ref, k

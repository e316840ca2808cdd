"""Independent reference methods used to pin the oracle (NumPy only).

Nothing here is shared with the oracle or with the CUDA library.

* ``bicgstab``: Bi-CGSTAB as published by van der Vorst (SIAM J. Sci. Stat.
  Comput. 13, 1992), with the optional omega safeguard of Sleijpen & van der
  Vorst (Numer. Algorithms 10, 1995).  The paper states that its
  ML(n)BiCGStabt reduces to BiCGStab when n = 1 (§4.3).
"""
from __future__ import annotations

import numpy as np


def _vdot(u, v):
    # u^H v
    return np.vdot(u, v)


def bicgstab(matvec, b, x0, rhat, nsteps: int, kappa: float = 0.0):
    """Run ``nsteps`` full Bi-CGSTAB steps; return the list of iterates x_i
    and, per step, (|rho| of the safeguard or None)."""
    x = np.array(x0, dtype=np.result_type(b, rhat, x0), copy=True)
    r = b - matvec(x)
    p = np.zeros_like(r)
    v = np.zeros_like(r)
    rho_old = 1.0
    alpha = 1.0
    omega = 1.0
    xs, guards = [], []
    for _ in range(nsteps):
        rho = _vdot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = matvec(p)
        alpha = rho / _vdot(rhat, v)
        s = r - alpha * v
        t = matvec(s)
        ts = _vdot(t, s)
        omega = ts / _vdot(t, t)
        g = None
        if kappa > 0:
            g = abs(ts) / (np.linalg.norm(t) * np.linalg.norm(s))
            if g < kappa and g != 0:
                omega = omega * kappa / g
        guards.append(g)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        xs.append(x.copy())
    return xs, guards


def csr_matvec(A):
    """Matvec closure through SciPy's CSR product (a library routine)."""
    import scipy.sparse as sp
    M = sp.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.n_rows, A.n_rows))
    return lambda v: M @ v


def dense(A) -> np.ndarray:
    """Dense copy of a CSR matrix (small cases only)."""
    M = np.zeros((A.n_rows, A.n_rows), dtype=A.val.dtype)
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    M[rows, A.col] = A.val
    return M

"""Seeded synthetic linear systems A x = b for the ML(n)BiCGStab solver.

This module only *generates inputs*: sparse matrices in CSR (and 3x3 BSR),
right-hand sides and initial guesses.  It holds none of the solver's
arithmetic, and imports nothing from the CUDA binding or the CPU oracle, so
both sides can consume the same arrays.

The paper's own test matrices (utm5940, qc2534, SPE9) are not available; the
generators below are stand-ins with the shapes the paper describes
(§5: real non-symmetric and complex symmetric-indefinite systems, reservoir
simulation systems, sequences of systems) built from textbook
discretisations:

* ``cd2d``            2-D 5-point convection-diffusion  -Δu + β·∇u
* ``cd3d_lognormal``  3-D 7-point, cellwise log-normal diffusion, x-convection
* ``reservoir_bsr3``  3 unknowns per cell, dense 3x3 coupling blocks
* ``batch_cd``        many independent 2-D/3-D convection-diffusion systems
* ``helmholtz3d_c``   complex damped shifted Laplacian with x-convection

Common discretisation rules: unit domain, ``h_d = 1/(m_d+1)``, homogeneous
Dirichlet boundary eliminated, lexicographic order with x fastest, central
differences.  Real stencil rows are scaled by h^2 (Krylov iterates do not
change under a global scale of A).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class CSR:
    """Compressed sparse row matrix, 0-based, columns sorted within a row."""

    row_ptr: np.ndarray  # int64, length N+1
    col: np.ndarray      # int32, length nnz
    val: np.ndarray      # float64 or complex128, length nnz
    n_rows: int

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def is_complex(self) -> bool:
        return np.iscomplexobj(self.val)


@dataclasses.dataclass
class BSR3:
    """3x3 block sparse row matrix.  Block (b) is stored row-major in
    ``val[b, 3, 3]``; ``row_ptr``/``col`` index cells (block rows/columns)."""

    row_ptr: np.ndarray  # int64, length ncell+1
    col: np.ndarray      # int32, length nblocks
    val: np.ndarray      # float64, shape (nblocks, 3, 3)
    n_cells: int

    @property
    def n_rows(self) -> int:
        return 3 * self.n_cells

    @property
    def nblocks(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def nnz(self) -> int:
        """Scalar entries (9 per block)."""
        return 9 * self.nblocks


# ---------------------------------------------------------------------------
# generic stencil assembly
# ---------------------------------------------------------------------------

def _assemble(dims, diag, offs):
    """Assemble a CSR matrix from a structured stencil.

    ``dims``  grid extents (mx, my[, mz]) with x fastest.
    ``diag``  array of shape dims[::-1] (z, y, x order) with the diagonal.
    ``offs``  list of (axis, step, coef) where axis is 0=x,1=y,2=z, step=±1
              and ``coef`` has shape dims[::-1]: the coupling of each cell to
              its neighbour at +step along axis (0 where the neighbour lies
              outside the grid is enforced here).
    Columns come out sorted because neighbour offsets are visited in
    increasing linear offset.
    """
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    N = int(np.prod(dims))
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    idx = np.arange(N, dtype=np.int64)
    # coordinates of each cell, x fastest
    coords = []
    rem = idx.copy()
    for d in dims:
        coords.append(rem % d)
        rem //= d
    entries = []  # (linear offset, coef flat, valid mask)
    for axis, step, coef in offs:
        c = coords[axis] + step
        valid = (c >= 0) & (c < dims[axis])
        entries.append((step * strides[axis], np.asarray(coef).reshape(-1), valid))
    entries.append((0, np.asarray(diag).reshape(-1), np.ones(N, dtype=bool)))
    entries.sort(key=lambda t: t[0])
    k = len(entries)
    cols = np.empty((N, k), dtype=np.int64)
    vals = np.empty((N, k), dtype=np.result_type(*[e[1].dtype for e in entries]))
    mask = np.empty((N, k), dtype=bool)
    for j, (off, coef, valid) in enumerate(entries):
        cols[:, j] = idx + off
        vals[:, j] = coef
        mask[:, j] = valid
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = cols[mask].astype(np.int32)
    val = np.ascontiguousarray(vals[mask])
    del nd
    return CSR(row_ptr=row_ptr, col=col, val=val, n_rows=N)


def row_sums(A: CSR) -> np.ndarray:
    """b = A·1 (the right-hand side the paper uses for qc2534, §5)."""
    out = np.zeros(A.n_rows, dtype=A.val.dtype)
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    np.add.at(out, rows, A.val)
    return out


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def cd2d(m: int = 32, beta=(10.0, 5.0)) -> CSR:
    """2-D 5-point convection-diffusion -Δu + β·∇u on an m×m grid, rows
    scaled by h^2: diagonal 4, west/east -1 ∓ β_x h/2, south/north
    -1 ∓ β_y h/2.  m=32 gives N=1024, nnz=4992."""
    h = 1.0 / (m + 1)
    shape = (m, m)  # (y, x)
    bx, by = float(beta[0]), float(beta[1])
    one = np.ones(shape)
    offs = [
        (0, -1, (-1.0 - bx * h / 2) * one),
        (0, +1, (-1.0 + bx * h / 2) * one),
        (1, -1, (-1.0 - by * h / 2) * one),
        (1, +1, (-1.0 + by * h / 2) * one),
    ]
    return _assemble((m, m), 4.0 * one, offs)


def _harmonic(a, b):
    return 2.0 * a * b / (a + b)


def cd3d_lognormal(m: int = 128, sigma: float = 2.0, beta_x: float = 50.0,
                   seed: int = 1) -> CSR:
    """3-D 7-point convection-diffusion -∇·(k∇u) + β_x ∂u/∂x on an m^3 grid.

    Cell diffusion k_c = exp(sigma·Z), Z ~ N(0,1) drawn cell by cell in
    lexicographic order from ``numpy.random.default_rng(seed)``.  An interior
    face takes the harmonic mean of its two cells; a boundary face takes k_c.
    Rows scaled by h^2: off-diagonal -k_f (± β_x h/2 on x-neighbours),
    diagonal Σ_faces k_f.  m=128 gives N=2,097,152 and nnz=14,581,760.
    """
    h = 1.0 / (m + 1)
    rng = np.random.default_rng(seed)
    k = np.exp(sigma * rng.standard_normal(m ** 3)).reshape(m, m, m)  # z,y,x
    c = beta_x * h / 2.0
    diag = np.zeros_like(k)
    offs = []
    for axis in range(3):
        ax = 2 - axis  # numpy axis of grid axis
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, m - 1)
        hi[ax] = slice(1, m)
        kf = _harmonic(k[tuple(lo)], k[tuple(hi)])  # face between i and i+1
        plus = np.zeros_like(k)   # coupling of cell to its +1 neighbour
        minus = np.zeros_like(k)  # coupling of cell to its -1 neighbour
        plus[tuple(lo)] = -kf
        minus[tuple(hi)] = -kf
        dsum = np.zeros_like(k)
        dsum[tuple(lo)] += kf
        dsum[tuple(hi)] += kf
        # boundary faces use the cell's own coefficient
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[ax] = 0
        last[ax] = m - 1
        dsum[tuple(first)] += k[tuple(first)]
        dsum[tuple(last)] += k[tuple(last)]
        diag += dsum
        if axis == 0:
            plus[tuple(lo)] += c
            minus[tuple(hi)] -= c
        offs.append((axis, -1, minus))
        offs.append((axis, +1, plus))
    return _assemble((m, m, m), diag, offs)


def reservoir_bsr3(mx: int = 64, my: int = 64, mz: int = 32, sigma: float = 3.0,
                   seed_perm: int = 3, seed_blocks: int = 4,
                   dominance: float = 1.05) -> BSR3:
    """Reservoir-shaped block system: 3 unknowns per cell, 7-point cell
    coupling, no-flow boundary (no boundary faces).

    Cell transmissibility k_c = exp(sigma·Z) (seed ``seed_perm``); face
    transmissibility T_f = harmonic mean.  Off-diagonal block = T_f·R with R
    a fresh 3x3 matrix of iid N(0,1) entries (seed ``seed_blocks``); the
    diagonal block = (Σ_f T_f)·R, after which every scalar diagonal entry is
    set to ``dominance`` × (sum of |off-diagonal| entries of its scalar row),
    giving strict row diagonal dominance.  64x64x32 gives N=393,216 and
    901,120 blocks.
    """
    dims = (mx, my, mz)
    n_cells = mx * my * mz
    rng_k = np.random.default_rng(seed_perm)
    k = np.exp(sigma * rng_k.standard_normal(n_cells)).reshape(mz, my, mx)
    # scalar face transmissibility per (cell, neighbour) built via the
    # stencil assembler on a scalar pattern; then expanded to blocks.
    offs = []
    tsum = np.zeros_like(k)
    for axis in range(3):
        ax = 2 - axis
        m = dims[axis]
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, m - 1)
        hi[ax] = slice(1, m)
        tf = _harmonic(k[tuple(lo)], k[tuple(hi)])
        plus = np.zeros_like(k)
        minus = np.zeros_like(k)
        plus[tuple(lo)] = tf
        minus[tuple(hi)] = tf
        tsum[tuple(lo)] += tf
        tsum[tuple(hi)] += tf
        offs.append((axis, -1, minus))
        offs.append((axis, +1, plus))
    pattern = _assemble(dims, tsum, offs)  # values: T_f off-diag, ΣT_f diag
    nb = pattern.nnz
    rng_b = np.random.default_rng(seed_blocks)
    R = rng_b.standard_normal((nb, 3, 3))
    blocks = R * pattern.val[:, None, None]
    rows = np.repeat(np.arange(n_cells), np.diff(pattern.row_ptr))
    is_diag = pattern.col == rows
    # strict row diagonal dominance per scalar row
    absb = np.abs(blocks)
    offsum = np.zeros((n_cells, 3))
    np.add.at(offsum, rows, absb.sum(axis=2))
    diag_blocks = np.nonzero(is_diag)[0]
    cell = rows[diag_blocks]
    d = blocks[diag_blocks]
    for a in range(3):
        offsum[cell, a] -= np.abs(d[:, a, a])
        d[:, a, a] = dominance * offsum[cell, a]
    blocks[diag_blocks] = d
    return BSR3(row_ptr=pattern.row_ptr, col=pattern.col,
                val=np.ascontiguousarray(blocks), n_cells=n_cells)


def bsr3_to_csr(B: BSR3) -> CSR:
    """Expand a 3x3 BSR matrix to scalar CSR (columns sorted)."""
    nc = B.n_cells
    cnt = np.diff(B.row_ptr)
    row_ptr = np.zeros(3 * nc + 1, dtype=np.int64)
    per_row = np.repeat(3 * cnt, 3)
    np.cumsum(per_row, out=row_ptr[1:])
    nb = B.nblocks
    brow = np.repeat(np.arange(nc), cnt)
    # position of each block inside its block row
    pos = np.arange(nb) - B.row_ptr[brow]
    col = np.empty(9 * nb, dtype=np.int32)
    val = np.empty(9 * nb, dtype=B.val.dtype)
    for a in range(3):
        base = row_ptr[3 * brow + a] + 3 * pos
        for b in range(3):
            col[base + b] = 3 * B.col + b
            val[base + b] = B.val[:, a, b]
    return CSR(row_ptr=row_ptr, col=col, val=val, n_rows=3 * nc)


def batch_cd(count: int = 512, seed: int = 5, n_min: float = 1e3,
             n_max: float = 1e5):
    """Independent convection-diffusion systems of uneven size.

    Per system: dimension d ∈ {2,3} with probability ½; target size
    N ~ logU[n_min, n_max]; m = round(N^(1/d)) so the realised size is m^d;
    Péclet number Pe ~ U[1,100] and β = Pe·(random unit direction);
    diffusion 1.  Rows scaled by h^2.  Returns a list of (CSR, meta dict).
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        d = 2 if rng.random() < 0.5 else 3
        target = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        m = max(2, int(round(target ** (1.0 / d))))
        pe = rng.uniform(1.0, 100.0)
        u = rng.standard_normal(d)
        u /= np.linalg.norm(u)
        beta = pe * u
        h = 1.0 / (m + 1)
        shape = (m,) * d
        one = np.ones(shape)
        offs = []
        for axis in range(d):
            offs.append((axis, -1, (-1.0 - beta[axis] * h / 2) * one))
            offs.append((axis, +1, (-1.0 + beta[axis] * h / 2) * one))
        A = _assemble(shape, 2.0 * d * one, offs)
        out.append((A, {"dim": d, "m": m, "pe": float(pe),
                        "beta": [float(x) for x in beta]}))
    return out


def helmholtz3d_c(mx: int = 256, my: int = 256, mz: int = 64, k: float = 20.0,
                  damping: float = 0.1, beta_x: float = 20.0) -> CSR:
    """Complex damped shifted Laplacian -Δu - k^2(1+iδ)u + β_x ∂u/∂x.

    Per-dimension spacings h_d = 1/(m_d+1); rows scaled by h_x^2 so the
    values are O(1).  256x256x64 gives N=4,194,304 and nnz=29,163,520.
    """
    dims = (mx, my, mz)
    hs = [1.0 / (d + 1) for d in dims]
    s = hs[0] ** 2
    shape = (mz, my, mx)
    one = np.ones(shape, dtype=np.complex128)
    diag = sum(2.0 * s / hd ** 2 for hd in hs) - s * k * k * (1.0 + 1j * damping)
    offs = []
    for axis in range(3):
        base = -s / hs[axis] ** 2
        conv = s * beta_x / (2.0 * hs[0]) if axis == 0 else 0.0
        offs.append((axis, -1, (base - conv) * one))
        offs.append((axis, +1, (base + conv) * one))
    return _assemble(dims, diag * one, offs)


def conj_transpose(A: CSR) -> CSR:
    """A^H as a separate CSR (stable counting sort by column)."""
    N = A.n_rows
    rows = np.repeat(np.arange(N, dtype=np.int64), np.diff(A.row_ptr))
    order = np.lexsort((rows, A.col))  # by column, then row
    cnt = np.bincount(A.col, minlength=N)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(cnt, out=row_ptr[1:])
    val = A.val[order]
    if np.iscomplexobj(val):
        val = np.conj(val)
    return CSR(row_ptr=row_ptr, col=rows[order].astype(np.int32),
               val=np.ascontiguousarray(val), n_rows=N)


def uniform_rhs(N: int, seed: int = 2) -> np.ndarray:
    """b ~ U[-1, 1], iid, from ``numpy.random.default_rng(seed)``."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, N)


def random_dense_system(N: int, seed: int, shift: float = 3.0,
                        complex_: bool = False):
    """Small well-conditioned dense system stored as CSR (for pins):
    A = randn(N,N)/sqrt(N) + shift·I, b = randn(N)."""
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((N, N)) / math.sqrt(N)
    if complex_:
        M = M + 1j * rng.standard_normal((N, N)) / math.sqrt(N)
    M = M + shift * np.eye(N)
    b = rng.standard_normal(N)
    if complex_:
        b = b + 1j * rng.standard_normal(N)
    return dense_to_csr(M), M, b


def dense_to_csr(M: np.ndarray) -> CSR:
    N = M.shape[0]
    mask = M != 0
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=row_ptr[1:])
    col = np.nonzero(mask)[1].astype(np.int32)
    return CSR(row_ptr=row_ptr, col=col, val=np.ascontiguousarray(M[mask]),
               n_rows=N)


# Named workloads with the sizes the benchmarks and tests use.
WORKLOADS = {
    "cd2d_32": dict(fn="cd2d", kwargs=dict(m=32)),
    "cd3d_lognormal_128": dict(fn="cd3d_lognormal", kwargs=dict(m=128)),
    "reservoir_bsr3_64x64x32": dict(fn="reservoir_bsr3", kwargs={}),
    "helmholtz3d_c_256x256x64": dict(fn="helmholtz3d_c", kwargs={}),
}

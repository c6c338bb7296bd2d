"""Seeded synthetic fully implicit compositional Jacobians in BSR form.

The paper's experiments (Section 5) run on SPE1/SPE5/SPE10 Jacobians produced by a
reservoir simulator; those data sets are not available, so these generators stand in
for them with the same grid shapes, block sizes and sparsity structure:

* a 7-point finite-volume stencil on an nx*ny*nz box (Section 2.1.1, the flux of
  Eq. (flux) couples each cell with its face neighbours);
* block size b = n_c + 1 unknowns per cell, pressure first (Eq. Jacobian-system-reservoir);
* implicit wells as extra block rows after the cells (Eq. Jacobian-system).  A well row
  has one meaningful unknown (bottom-hole pressure, unknown 0); unknowns 1..b-1 of a
  well are identity-padded.

Recipe (all draws from one ``numpy.random.default_rng(seed)`` in a fixed order):

1. permeability: ``ln k ~ N(0,1)`` (``layered=False``) or, per z layer, mean
   ``U[-2,4]`` and sigma 2 (``layered=True``);
2. transmissibility ``T_ij = 2 k_i k_j / (k_i + k_j)`` (harmonic mean), vertical
   faces multiplied by ``kz_ratio``;
3. off-diagonal block ``A_ij = -T_ij * M_ij`` with ``M_ij = R_ij + (b-1) I``, ``R_ij``
   entries ``U[0.1,1]`` drawn independently for every directed pair (so A is
   nonsymmetric).  The ``(b-1) I`` shift makes every M_ij a strictly row diagonally
   dominant positive block; without it the diagonal blocks built in step 5 are
   indefinite and no preconditioned Krylov method converges;
4. well couplings (well w perforating cell c, well index ``WI_c = k_c``):
   ``A_cw = -WI_c * E`` (only column 0 nonzero, entries U[0.1,1]) and
   ``A_wc = -WI_c * F`` (only row 0 nonzero, entries U[0.1,1]);
5. cell diagonal block = accumulation ``U[0.5,2] * I + U[0,0.1]`` block minus the sum
   of the row's off-diagonal blocks; well diagonal = identity with row 0 replaced by
   ``acc * e_0 - sum_c A_wc[0,:]``.

Cells are numbered ``i + nx*(j + ny*k)``; wells follow the cells.  Columns are sorted
within each block row and the diagonal block is always stored.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass

import numpy as np


@dataclass
class BSRMatrix:
    """Block-sparse matrix: ``row_ptr`` int32[nb+1], ``col_idx`` int32[nnzb],
    ``values`` float64[nnzb, b, b] (row-major blocks: row = equation, column = unknown)."""

    nb: int
    b: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    values: np.ndarray
    n_cells: int = 0
    n_wells: int = 0
    dims: tuple = ()

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def n(self) -> int:
        return self.nb * self.b

    def to_dense(self) -> np.ndarray:
        b = self.b
        a = np.zeros((self.nb * b, self.nb * b))
        for i in range(self.nb):
            for p in range(self.row_ptr[i], self.row_ptr[i + 1]):
                j = self.col_idx[p]
                a[i * b:(i + 1) * b, j * b:(j + 1) * b] = self.values[p]
        return a

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.bsr_matrix((self.values, self.col_idx, self.row_ptr),
                             shape=(self.nb * self.b, self.nb * self.b))

    def copy(self) -> "BSRMatrix":
        return BSRMatrix(self.nb, self.b, self.row_ptr.copy(), self.col_idx.copy(),
                         self.values.copy(), self.n_cells, self.n_wells, self.dims)


def _assemble(nb, b, rows, cols, blocks):
    """Sort (row, col) entries into CSR order; entries must be unique."""
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order].astype(np.int32)
    blocks = blocks[order]
    counts = np.bincount(rows, minlength=nb)
    row_ptr = np.zeros(nb + 1, dtype=np.int32)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols, np.ascontiguousarray(blocks, dtype=np.float64)


def box_jacobian(nx: int, ny: int, nz: int, b: int, seed: int, *, layered: bool = False,
                 kz_ratio: float = 1.0, n_wells: int = 0) -> BSRMatrix:
    """Seeded compositional-style Jacobian on an nx*ny*nz box (recipe in the module doc)."""
    rng = np.random.default_rng(seed)
    nc = nx * ny * nz
    if layered:
        layer_mean = rng.uniform(-2.0, 4.0, size=nz)
        lnk = rng.normal(0.0, 2.0, size=(nz, ny, nx)) + layer_mean[:, None, None]
    else:
        lnk = rng.normal(0.0, 1.0, size=(nz, ny, nx))
    k = np.exp(lnk).reshape(-1)  # index i + nx*(j + ny*kk)

    idx = np.arange(nc).reshape(nz, ny, nx)
    faces = []  # (cell a, cell b, scale) for each undirected face
    if nx > 1:
        faces.append((idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel(), 1.0))
    if ny > 1:
        faces.append((idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel(), 1.0))
    if nz > 1:
        faces.append((idx[:-1, :, :].ravel(), idx[1:, :, :].ravel(), kz_ratio))
    fa = np.concatenate([f[0] for f in faces]) if faces else np.zeros(0, np.int64)
    fb = np.concatenate([f[1] for f in faces]) if faces else np.zeros(0, np.int64)
    fs = np.concatenate([np.full(f[0].shape, f[2]) for f in faces]) if faces else np.zeros(0)
    T = fs * 2.0 * k[fa] * k[fb] / (k[fa] + k[fb])
    # directed pairs: (a->b) and (b->a); each gets its own random positive block
    src = np.concatenate([fa, fb])
    dst = np.concatenate([fb, fa])
    Td = np.concatenate([T, T])
    M = rng.uniform(0.1, 1.0, size=(src.shape[0], b, b)) + (b - 1) * np.eye(b)[None]
    off = -Td[:, None, None] * M

    nb = nc + n_wells
    rows = [src]
    cols = [dst]
    blocks = [off]
    diag_sum = np.zeros((nb, b, b))
    np.add.at(diag_sum, src, off)

    well_cells = []
    if n_wells > 0:
        pos = rng.choice(nx * ny, size=n_wells, replace=False)
        for w in range(n_wells):
            wx, wy = int(pos[w] % nx), int(pos[w] // nx)
            cells = idx[:, wy, wx].ravel()  # perforated in every layer
            well_cells.append(cells)
            wi = k[cells]
            E = np.zeros((cells.shape[0], b, b))
            E[:, :, 0] = rng.uniform(0.1, 1.0, size=(cells.shape[0], b))
            F = np.zeros((cells.shape[0], b, b))
            F[:, 0, :] = rng.uniform(0.1, 1.0, size=(cells.shape[0], b))
            a_cw = -wi[:, None, None] * E
            a_wc = -wi[:, None, None] * F
            wrow = np.full(cells.shape[0], nc + w)
            rows += [cells, wrow]
            cols += [wrow, cells]
            blocks += [a_cw, a_wc]
            np.add.at(diag_sum, cells, a_cw)
            np.add.at(diag_sum, wrow, a_wc)

    acc = rng.uniform(0.5, 2.0, size=nb)[:, None, None] * np.eye(b)[None] \
        + rng.uniform(0.0, 0.1, size=(nb, b, b))
    diag = acc - diag_sum
    if n_wells > 0:
        wd = np.broadcast_to(np.eye(b), (n_wells, b, b)).copy()
        wd[:, 0, :] = 0.0
        wd[:, 0, 0] = acc[nc:, 0, 0]
        wd[:, 0, :] -= diag_sum[nc:, 0, :]
        diag[nc:] = wd
    rows.append(np.arange(nb))
    cols.append(np.arange(nb))
    blocks.append(diag)
    row_ptr, col_idx, values = _assemble(nb, b, np.concatenate(rows), np.concatenate(cols),
                                         np.concatenate(blocks))
    return BSRMatrix(nb, b, row_ptr, col_idx, values, nc, n_wells, (nx, ny, nz))


def grid_small(seed: int = 2208) -> BSRMatrix:
    """16x16x8 grid, 3 unknowns per cell, ln k ~ N(0,1), no wells (2048 block rows)."""
    return box_jacobian(16, 16, 8, 3, seed)


def grid_spe10(seed: int = 2209, nx: int = 60, ny: int = 220, nz: int = 85, b: int = 4,
               n_wells: int = 4) -> BSRMatrix:
    """SPE10-shaped 60x220x85 grid (1,122,000 cells), 4 unknowns per cell, layered
    lognormal permeability (per-layer mean ln k ~ U[-2,4], sigma 2, kz/kx = 0.1) and
    four wells perforated along z.  Smaller nx/ny/nz give the same recipe at test sizes."""
    return box_jacobian(nx, ny, nz, b, seed, layered=True, kz_ratio=0.1, n_wells=n_wells)


def random_rhs(a: BSRMatrix, seed: int) -> np.ndarray:
    """RHS ~ N(0,1) on every cell unknown; the identity-padded well unknowns get 0."""
    rng = np.random.default_rng(seed)
    r = rng.normal(0.0, 1.0, size=(a.nb, a.b))
    if a.n_wells > 0:
        r[a.n_cells:, 1:] = 0.0
    return r.reshape(-1)


def perturb_values(a: BSRMatrix, seed: int, rel: float = 0.05) -> np.ndarray:
    """A Newton-like next Jacobian with the same pattern: every entry of every
    off-diagonal block is multiplied by an independent U[1-rel, 1+rel] factor and each
    diagonal block absorbs the change of its row's couplings, so that the diagonal stays
    "accumulation minus the sum of the off-diagonal blocks" (a per-entry perturbation
    of the diagonal too would unbalance cells whose couplings dwarf their accumulation
    term and can make the system nearly singular)."""
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(a.nb), np.diff(a.row_ptr))
    off = rows != a.col_idx
    v = a.values.copy()
    new_off = a.values[off] * rng.uniform(1.0 - rel, 1.0 + rel, size=a.values[off].shape)
    delta = np.zeros((a.nb, a.b, a.b))
    np.add.at(delta, rows[off], new_off - a.values[off])
    v[off] = new_off
    dpos = np.nonzero(~off)[0]
    v[dpos] = a.values[dpos] - delta[rows[dpos]]
    return v


def newton_sequence(a: BSRMatrix, time_steps: int, newton_steps: int, seed: int,
                    rel_newton: float = 0.02, rel_step: float = 0.2) -> list:
    """Values of the Jacobians a time-stepping Newton solver would see, same pattern:
    ``time_steps`` x ``newton_steps`` arrays, each derived from the previous one by
    ``perturb_values`` (so the drift accumulates): U[1 - rel_step, 1 + rel_step] factors
    on the first Newton step of a time step (the state moved a whole step), and
    U[1 - rel_newton, 1 + rel_newton] between Newton steps.  The first array is the
    first time step's first Jacobian, ``a``'s values perturbed once by ``rel_step``."""
    out = []
    cur = a
    for t in range(time_steps):
        for k in range(newton_steps):
            rel = rel_step if k == 0 else rel_newton
            v = perturb_values(cur, seed + 1000 * t + k, rel)
            out.append(v)
            cur = dataclasses.replace(cur, values=v)
    return out


def poisson3d_bsr(nx: int, ny: int, nz: int) -> BSRMatrix:
    """7-point Laplacian (Dirichlet boundary) as a 1x1-block BSR matrix."""
    nc = nx * ny * nz
    idx = np.arange(nc).reshape(nz, ny, nx)
    pairs = []
    if nx > 1:
        pairs.append((idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel()))
    if ny > 1:
        pairs.append((idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel()))
    if nz > 1:
        pairs.append((idx[:-1, :, :].ravel(), idx[1:, :, :].ravel()))
    a = np.concatenate([p[0] for p in pairs])
    c = np.concatenate([p[1] for p in pairs])
    rows = np.concatenate([a, c, np.arange(nc)])
    cols = np.concatenate([c, a, np.arange(nc)])
    vals = np.concatenate([-np.ones(2 * a.shape[0]), np.full(nc, 6.0)])
    row_ptr, col_idx, values = _assemble(nc, 1, rows, cols, vals.reshape(-1, 1, 1))
    return BSRMatrix(nc, 1, row_ptr, col_idx, values, nc, 0, (nx, ny, nz))


def chain_bsr(nb: int, b: int, seed: int) -> BSRMatrix:
    """Block tridiagonal 1-D chain with random diagonally dominant blocks."""
    rng = np.random.default_rng(seed)
    i = np.arange(nb - 1)
    rows = np.concatenate([i, i + 1, np.arange(nb)])
    cols = np.concatenate([i + 1, i, np.arange(nb)])
    off = -rng.uniform(0.1, 1.0, size=(2 * (nb - 1), b, b))
    diag = rng.uniform(0.0, 0.1, size=(nb, b, b)) + (4.0 * b) * np.eye(b)[None]
    row_ptr, col_idx, values = _assemble(nb, b, rows, cols, np.concatenate([off, diag]))
    return BSRMatrix(nb, b, row_ptr, col_idx, values, nb, 0, (nb, 1, 1))


def diagonal_bsr(diag: np.ndarray) -> BSRMatrix:
    """Diagonal matrix with the given entries as a 1x1-block BSR matrix."""
    n = diag.shape[0]
    return BSRMatrix(n, 1, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                     np.asarray(diag, dtype=np.float64).reshape(n, 1, 1), n, 0, (n, 1, 1))

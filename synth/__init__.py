"""Seeded synthetic inputs for the reservoir-type linear systems.

This module generates *inputs* only: matrices, exact solutions and
permeability fields shaped like the pressure and black-oil systems of the
paper's numerical examples (Sec. 5, Examples 2-7: pressure equations and
black-oil Jacobians on structured reservoir grids).  It contains none of the
solver arithmetic; both the CPU oracle and the CUDA path receive the arrays
built here.  Right-hand sides b = A x_true are *not* formed here: the caller
forms them with its own SpMV.

Random numbers come from one counter-based generator, SplitMix64
(Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), keyed by (seed, stream, index), so every value is reproducible
and independent of evaluation order.

Grid and cell numbering: cell (i, j, k) of an nx x ny x nz grid has index
c = i + nx*(j + ny*k) (x fastest).  Unit spacing and unit face areas;
no-flow outer boundary.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "splitmix64", "uniform01", "normal", "log_permeability",
    "pressure_7pt", "black_oil_bsr3", "x_true", "Grid",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)

# Stream identifiers: each random quantity draws from its own stream.
STREAM_PERM = 1
STREAM_XTRUE = 2
STREAM_BLOCK = 3


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to state x (uint64 array)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + _GOLDEN).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = splitmix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        return np.uint64(s ^ (np.uint64(stream) * _STREAM_MUL))


def _bits(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        return splitmix64(_key(seed, stream) + np.asarray(index, dtype=np.uint64))


def uniform01(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of the counter-based draw."""
    return (_bits(seed, stream, index) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Standard normal draws by Box-Muller on draws (2*index, 2*index+1)."""
    index = np.asarray(index, dtype=np.uint64)
    u1 = 1.0 - uniform01(seed, stream, index * np.uint64(2))          # (0, 1]
    u2 = uniform01(seed, stream, index * np.uint64(2) + np.uint64(1))  # [0, 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


class Grid:
    """Structured nx x ny x nz grid with x-fastest cell numbering."""

    def __init__(self, nx: int, ny: int, nz: int):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.n = self.nx * self.ny * self.nz

    @property
    def shape_zyx(self):
        return (self.nz, self.ny, self.nx)


def log_permeability(grid: Grid, seed: int, mu: float = 0.0, sigma: float = 1.0) -> np.ndarray:
    """i.i.d. log-normal permeability per cell: log k ~ N(mu, sigma^2)."""
    idx = np.arange(grid.n, dtype=np.uint64)
    return mu + sigma * normal(seed, STREAM_PERM, idx)


def x_true(n: int, seed: int) -> np.ndarray:
    """Exact solution x_true ~ U(-1, 1), its own stream."""
    return 2.0 * uniform01(seed, STREAM_XTRUE, np.arange(n, dtype=np.uint64)) - 1.0


def _faces(grid: Grid, logk: np.ndarray, kz_scale: float):
    """Face transmissibilities: harmonic mean of the two cell permeabilities.

    Returns (tx, ty, tz) with tx[c] the transmissibility of the face between
    cell c and c+1 (0 where c is on the +x boundary), likewise ty, tz.
    """
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    k = np.exp(logk).reshape(nz, ny, nx)
    t = []
    for axis, scale in ((2, 1.0), (1, 1.0), (0, kz_scale)):
        ka = k * scale
        a = np.take(ka, range(0, ka.shape[axis] - 1), axis=axis)
        b = np.take(ka, range(1, ka.shape[axis]), axis=axis)
        h = 2.0 * a * b / (a + b)
        pad = [(0, 0)] * 3
        pad[axis] = (0, 1)
        t.append(np.pad(h, pad).reshape(-1))
    return t


def _stencil(grid: Grid):
    """Neighbour offsets of the 7-point stencil in ascending column order."""
    nx, nxy = grid.nx, grid.nx * grid.ny
    return [-nxy, -nx, -1, 0, 1, nx, nxy]


def pressure_7pt(grid: Grid, seed: int, kz_scale: float = 1.0, accum: float = 1e-3):
    """3-D 7-point finite-volume pressure matrix in CSR (FP64, sorted columns).

    Row c: a_{c,nb} = -T_{c,nb} for every interior face, a_{cc} = sum T + accum.
    Permeability log-normal(0, 1) i.i.d. per cell (seeded); z-face
    permeability scaled by kz_scale (anisotropy).

    Returns dict(n, rowptr int32[n+1], col int32[nnz], val f64[nnz], logk f64[n]).
    """
    logk = log_permeability(grid, seed)
    tx, ty, tz = _faces(grid, logk, kz_scale)
    n = grid.n
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    c = np.arange(n)
    i = c % nx
    j = (c // nx) % ny
    kk = c // (nx * ny)
    offs = _stencil(grid)
    # transmissibility of each off-diagonal slot and its existence mask
    t_slots = [
        (kk > 0, np.where(kk > 0, np.roll(tz, nx * ny), 0.0)),
        (j > 0, np.where(j > 0, np.roll(ty, nx), 0.0)),
        (i > 0, np.where(i > 0, np.roll(tx, 1), 0.0)),
        None,
        (i < nx - 1, tx),
        (j < ny - 1, ty),
        (kk < nz - 1, tz),
    ]
    diag = np.zeros(n)
    for s in t_slots:
        if s is not None:
            diag += np.where(s[0], s[1], 0.0)
    diag += accum
    mask = np.stack([s[0] if s is not None else np.ones(n, bool) for s in t_slots], axis=1)
    vals = np.stack([-s[1] if s is not None else diag for s in t_slots], axis=1)
    cols = c[:, None] + np.array(offs)[None, :]
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(counts, out=rowptr[1:])
    return dict(
        n=n,
        rowptr=rowptr,
        col=cols[mask].astype(np.int32),
        val=vals[mask].astype(np.float64),
        logk=logk,
    )


def black_oil_bsr3(grid: Grid, seed: int, kz_scale: float = 1.0, accum: float = 1e-3,
                   coupling: float = 0.05):
    """Black-oil-like 3x3-block system in BSR (row-major blocks, FP64).

    Unknowns per cell: (pressure, water saturation, gas saturation), block
    entry 0 is pressure (the Eq. 9 partition, interleaved per cell).  The
    pressure-pressure entries are the 7-point matrix of pressure_7pt.  With
    u ~ U(0.1, 1) seeded per entry, c = coupling, T the face transmissibility:

    off-diagonal block (I, J), J a neighbour:
        [0][0] = -T;  [0][s] = -c u T (s = 1, 2);  [s][0] = -c u T;
        [s][s] = -c u;  [1][2] = [2][1] = 0.
    diagonal block I:
        [0][0] = sum T + accum;  [0][s] = c u [0][0];
        [s][0] = -(sum over J of the [s][0] entries of the off-diagonal blocks)
                 (saturation rows' pressure part has zero row sum);
        [1][2], [2][1] = c u;
        [s][s] = 1 + sum |other entries of scalar row 3I+s| (diagonally dominant).

    Returns dict(nb, bs=3, browptr int32[nb+1], bcol int32[nnzb],
    bval f64[nnzb*9], logk f64[nb]).
    """
    p = pressure_7pt(grid, seed, kz_scale, accum)
    nb = p["n"]
    browptr, bcol, aval = p["rowptr"], p["col"], p["val"]
    nnzb = bcol.shape[0]
    row_of = np.repeat(np.arange(nb), np.diff(browptr))
    is_diag = bcol == row_of
    T = np.where(is_diag, 0.0, -aval)
    # 8 independent U(0.1, 1) draws per block slot
    ridx = np.arange(nnzb, dtype=np.uint64)[:, None] * np.uint64(8) + np.arange(8, dtype=np.uint64)[None, :]
    u = 0.1 + 0.9 * uniform01(seed, STREAM_BLOCK, ridx)
    B = np.zeros((nnzb, 3, 3))
    off = ~is_diag
    B[off, 0, 0] = -T[off]
    for s in (1, 2):
        B[off, 0, s] = -coupling * u[off, s - 1] * T[off]
        B[off, s, 0] = -coupling * u[off, s + 1] * T[off]
        B[off, s, s] = -coupling * u[off, s + 3]
    d = np.nonzero(is_diag)[0]
    B[d, 0, 0] = aval[d]
    for s in (1, 2):
        B[d, 0, s] = coupling * u[d, s - 1] * aval[d]
        # zero row sum of the pressure part of saturation row s
        rs = np.zeros(nb)
        np.add.at(rs, row_of[off], B[off, s, 0])
        B[d, s, 0] = -rs
    B[d, 1, 2] = coupling * u[d, 6]
    B[d, 2, 1] = coupling * u[d, 7]
    for s in (1, 2):
        absrow = np.zeros(nb)
        absrow_all = np.abs(B[:, s, :]).sum(axis=1)
        np.add.at(absrow, row_of, absrow_all)
        B[d, s, s] = 1.0 + absrow   # diagonal entry itself is still 0 here
    return dict(nb=nb, bs=3, browptr=browptr.copy(), bcol=bcol.copy(),
                bval=B.reshape(-1).copy(), logk=p["logk"])


def csr_from_bsr(m: dict):
    """Expand a BSR matrix into scalar CSR with sorted columns (test helper)."""
    nb, bs = m["nb"], m["bs"]
    browptr, bcol, bval = m["browptr"], m["bcol"], m["bval"].reshape(-1, bs, bs)
    cnt = np.diff(browptr)
    rows = []
    n = nb * bs
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.repeat(cnt * bs, bs)
    np.cumsum(rowptr, out=rowptr)
    col = np.empty(rowptr[-1], dtype=np.int32)
    val = np.empty(rowptr[-1])
    for I in range(nb):
        s, e = browptr[I], browptr[I + 1]
        cols = (bcol[s:e, None] * bs + np.arange(bs)[None, :]).reshape(-1)
        for r in range(bs):
            o = rowptr[I * bs + r]
            col[o:o + cols.size] = cols
            val[o:o + cols.size] = bval[s:e, r, :].reshape(-1)
    del rows
    return dict(n=n, rowptr=rowptr, col=col, val=val)

"""Seeded synthetic sparse matrices and vectors.

This module only *generates inputs*.  It performs none of the arithmetic of the
method (no SpMV, no features, no selection); both the CUDA path and the CPU
oracle receive the same arrays produced here.

Every generator is deterministic for a given (seed, device type): a
``torch.Generator`` seeded with ``seed`` drives all draws.  CPU and CUDA
generators produce different streams, so a parity test always generates on the
CPU and copies the arrays to the GPU.

The families stand in for the 115-matrix University of Florida suite the paper
trains and evaluates on (Section 3.2.2 "Training Data Selection", Section 4),
which is not available; each family is built to sit in one bottleneck class of
Section 3.1:

* ``stencil_27pt``   -- regular 3-D stencil, long-ish uniform rows (MB)
* ``random_columns`` -- fixed row length, uniformly scattered columns (CML)
* ``zipf_rows``      -- power-law row lengths with one very long row (IMB)
* ``short_rows``     -- two nonzeros per row, banded (CMP / short rows)

plus the classic Laplacians (2-D 5-point, 3-D 7-point) and small random CSR
matrices with empty rows for edge cases.

Layout of every matrix: CSR with 0-based ``rowptr`` (int32, n_rows+1),
``colind`` (int32, nnz, strictly increasing within a row) and ``val``
(float64, nnz).
"""
from __future__ import annotations

import dataclasses
import math

import torch

__all__ = [
    "HostCSR", "laplacian_2d_5pt", "laplacian_3d_7pt", "stencil_27pt",
    "random_columns", "zipf_rows", "short_rows", "random_csr",
    "uniform_vector", "variable_coeff_laplacian_3d", "family_matrix",
    "FAMILIES", "four_class_set", "dense_to_csr", "batch_matrices",
]


@dataclasses.dataclass
class HostCSR:
    """A CSR matrix held in torch tensors (any device)."""
    n_rows: int
    n_cols: int
    rowptr: torch.Tensor  # int32 [n_rows + 1]
    colind: torch.Tensor  # int32 [nnz]
    val: torch.Tensor     # float64 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.colind.numel())

    def to(self, device) -> "HostCSR":
        return HostCSR(self.n_rows, self.n_cols, self.rowptr.to(device),
                       self.colind.to(device), self.val.to(device), self.name)

    def min_bytes(self, val_bytes: int = 8, idx_bytes: int = 4) -> int:
        """Minimum traffic of one CSR SpMV: every array read once, y written once."""
        return (self.nnz * (val_bytes + idx_bytes) + 4 * (self.n_rows + 1)
                + 8 * self.n_cols + 8 * self.n_rows)


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _uniform(n: int, g: torch.Generator, device, lo=-1.0, hi=1.0) -> torch.Tensor:
    u = torch.rand(n, generator=g, dtype=torch.float64, device=device)
    return lo + (hi - lo) * u


def _rowptr_from_lengths(lengths: torch.Tensor) -> torch.Tensor:
    rp = torch.zeros(lengths.numel() + 1, dtype=torch.int64, device=lengths.device)
    torch.cumsum(lengths.to(torch.int64), 0, out=rp[1:])
    if int(rp[-1]) >= 2 ** 31:
        raise ValueError("nnz does not fit int32 indices")
    return rp.to(torch.int32)


def uniform_vector(n: int, seed: int = 0, device="cpu") -> torch.Tensor:
    """x ~ U[-1, 1] in float64."""
    return _uniform(n, _gen(seed, device), device)


def _stencil(dims, offsets, diag_value=None, off_value=None, seed=0,
             device="cpu", name="stencil") -> HostCSR:
    """Generic structured stencil in natural (lexicographic) ordering.

    ``offsets`` is a list of (dz, dy, dx) in lexicographic order, so the column
    indices of each row come out strictly increasing.  Values are either the
    given constants (diag / off-diagonal) or U[-1,1] draws when both are None.
    """
    nz, ny, nx = dims
    n = nz * ny * nx
    idx = torch.arange(n, dtype=torch.int64, device=device)
    z, rem = idx // (ny * nx), idx % (ny * nx)
    y, x = rem // nx, rem % nx
    cols, valid = [], []
    for dz, dy, dx in offsets:
        ok = ((z + dz >= 0) & (z + dz < nz) & (y + dy >= 0) & (y + dy < ny)
              & (x + dx >= 0) & (x + dx < nx))
        cols.append(idx + dz * ny * nx + dy * nx + dx)
        valid.append(ok)
    cols = torch.stack(cols, 1)
    valid = torch.stack(valid, 1)
    lengths = valid.sum(1)
    colind = cols[valid].to(torch.int32)  # row-major order keeps rows contiguous
    rowptr = _rowptr_from_lengths(lengths)
    if diag_value is None:
        val = _uniform(colind.numel(), _gen(seed, device), device)
    else:
        is_diag = torch.zeros_like(valid)
        for k, o in enumerate(offsets):
            if o == (0, 0, 0):
                is_diag[:, k] = True
        is_diag = is_diag[valid]
        val = torch.where(is_diag, torch.tensor(float(diag_value), dtype=torch.float64, device=device),
                          torch.tensor(float(off_value), dtype=torch.float64, device=device))
    return HostCSR(n, n, rowptr, colind, val, name)


def laplacian_2d_5pt(nx: int = 64, ny: int = 64, device="cpu") -> HostCSR:
    """2-D 5-point Laplacian, Dirichlet boundary: 4 on the diagonal, -1 off."""
    offs = [(0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0)]
    return _stencil((1, ny, nx), offs, 4.0, -1.0, device=device,
                    name=f"laplacian2d_{nx}x{ny}")


def laplacian_3d_7pt(n: int = 128, device="cpu") -> HostCSR:
    """3-D 7-point Laplacian (SPD): 6 on the diagonal, -1 off."""
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    return _stencil((n, n, n), offs, 6.0, -1.0, device=device, name=f"laplacian3d_{n}")


def variable_coeff_laplacian_3d(n: int = 128, seed: int = 0, device="cpu") -> HostCSR:
    """SPD 7-point pattern with off-diagonals -U[0.5, 1.5] and a strictly
    dominant diagonal (sum of |off| in the row, plus 1), symmetric by
    construction: the coefficient of an edge is drawn once per undirected edge."""
    A = laplacian_3d_7pt(n, device=device)
    N = A.n_rows
    g = _gen(seed, device)
    # one coefficient per (min(i,j), direction): directions +x, +y, +z
    coef = 0.5 + torch.rand((N, 3), generator=g, dtype=torch.float64, device=device)
    rows = torch.repeat_interleave(torch.arange(N, device=device),
                                   (A.rowptr[1:] - A.rowptr[:-1]).to(torch.int64))
    cols = A.colind.to(torch.int64)
    lo = torch.minimum(rows, cols)
    d = (rows - cols).abs()
    direction = torch.where(d == 1, 0, torch.where(d == n, 1, 2))
    off = -coef[lo, direction]
    off = torch.where(rows == cols, torch.zeros_like(off), off)
    diag = torch.zeros(N, dtype=torch.float64, device=device)
    diag.index_add_(0, rows, off.abs())
    val = torch.where(rows == cols, diag[rows] + 1.0, off)
    return HostCSR(N, N, A.rowptr, A.colind, val, f"varcoef_laplacian3d_{n}")


def stencil_27pt(n: int = 128, seed: int = 0, device="cpu") -> HostCSR:
    """27-point 3-D stencil on an n^3 grid, values ~U[-1,1] (not symmetric)."""
    offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return _stencil((n, n, n), offs, None, None, seed=seed, device=device,
                    name=f"stencil27_{n}")


def _distinct_sorted_columns(lengths: torch.Tensor, n_cols: int, g, device) -> torch.Tensor:
    """For each row of length l, l distinct sorted columns in [0, n_cols).

    Draw l values r_k from [0, n_cols - l], sort them within the row and add the
    in-row rank k: c_k = r_(k) + k is strictly increasing and < n_cols.
    """
    lengths = lengths.to(torch.int64)
    if int(lengths.max()) > n_cols:
        raise ValueError("row longer than the number of columns")
    nnz = int(lengths.sum())
    rows = torch.repeat_interleave(torch.arange(lengths.numel(), device=device), lengths)
    span = (n_cols - lengths + 1).to(torch.float64)[rows]
    r = torch.floor(torch.rand(nnz, generator=g, dtype=torch.float64, device=device) * span)
    r = torch.minimum(r, span - 1).to(torch.int64)
    key = rows * (n_cols + 1) + r
    key, _ = torch.sort(key)
    r = key - rows * (n_cols + 1)
    start = torch.zeros(lengths.numel() + 1, dtype=torch.int64, device=device)
    torch.cumsum(lengths, 0, out=start[1:])
    rank = torch.arange(nnz, device=device) - start[:-1][rows]
    return (r + rank).to(torch.int32)


def random_columns(n_rows: int = 1 << 22, n_cols: int | None = None, per_row: int = 16,
                   seed: int = 0, device="cpu") -> HostCSR:
    """Every row has ``per_row`` distinct columns spread uniformly over [0, n_cols)."""
    n_cols = n_rows if n_cols is None else n_cols
    g = _gen(seed, device)
    lengths = torch.full((n_rows,), per_row, dtype=torch.int64, device=device)
    colind = _distinct_sorted_columns(lengths, n_cols, g, device)
    val = _uniform(colind.numel(), g, device)
    return HostCSR(n_rows, n_cols, _rowptr_from_lengths(lengths), colind, val,
                   f"random_cols_{n_rows}x{per_row}")


def zipf_lengths(n_rows: int, alpha: float, max_len: int, g, device) -> torch.Tensor:
    """Row lengths with P(l = k) proportional to k^-alpha on k in [1, max_len],
    sampled by inverse CDF; the longest sampled row is set to exactly max_len."""
    k = torch.arange(1, max_len + 1, dtype=torch.float64, device=device)
    cdf = torch.cumsum(k.pow(-alpha), 0)
    cdf = cdf / cdf[-1]
    u = torch.rand(n_rows, generator=g, dtype=torch.float64, device=device)
    lengths = torch.searchsorted(cdf, u, right=False) + 1
    lengths = torch.clamp(lengths, 1, max_len)
    lengths[torch.argmax(lengths)] = max_len
    return lengths


def zipf_rows(n_rows: int = 1 << 20, n_cols: int | None = None, alpha: float = 1.8,
              max_len: int = 200_000, seed: int = 0, device="cpu") -> HostCSR:
    """Power-law row lengths (Zipf alpha), distinct uniform columns per row."""
    n_cols = n_rows if n_cols is None else n_cols
    g = _gen(seed, device)
    lengths = zipf_lengths(n_rows, alpha, min(max_len, n_cols), g, device)
    colind = _distinct_sorted_columns(lengths, n_cols, g, device)
    val = _uniform(colind.numel(), g, device)
    return HostCSR(n_rows, n_cols, _rowptr_from_lengths(lengths), colind, val,
                   f"zipf_{n_rows}_a{alpha}")


def short_rows(n: int = 1 << 23, max_offset: int = 8, seed: int = 0, device="cpu") -> HostCSR:
    """Two nonzeros per row: the diagonal and one column at distance
    d in {1..max_offset} on a random side, reflected back into range."""
    if n <= max_offset:
        raise ValueError("n must exceed max_offset")
    g = _gen(seed, device)
    i = torch.arange(n, dtype=torch.int64, device=device)
    d = torch.randint(1, max_offset + 1, (n,), generator=g, device=device)
    side = torch.randint(0, 2, (n,), generator=g, device=device) * 2 - 1
    j = i + side * d
    j = torch.where((j < 0) | (j >= n), i - side * d, j)
    c = torch.stack([torch.minimum(i, j), torch.maximum(i, j)], 1).reshape(-1)
    val = _uniform(2 * n, g, device)
    lengths = torch.full((n,), 2, dtype=torch.int64, device=device)
    return HostCSR(n, n, _rowptr_from_lengths(lengths), c.to(torch.int32), val,
                   f"short_rows_{n}")


def random_csr(n_rows: int, n_cols: int, max_per_row: int, seed: int = 0,
               empty_frac: float = 0.1, device="cpu") -> HostCSR:
    """Small random CSR for edge-case tests: row lengths uniform in
    [0, max_per_row] with a fraction of forced-empty rows."""
    g = _gen(seed, device)
    cap = min(max_per_row, n_cols)
    lengths = torch.randint(0, cap + 1, (n_rows,), generator=g, device=device)
    if empty_frac > 0 and n_rows > 0:
        empty = torch.rand(n_rows, generator=g, device=device) < empty_frac
        lengths = torch.where(empty, torch.zeros_like(lengths), lengths)
    if n_rows == 0 or int(lengths.sum()) == 0:
        rp = torch.zeros(n_rows + 1, dtype=torch.int32, device=device)
        return HostCSR(n_rows, n_cols, rp, torch.zeros(0, dtype=torch.int32, device=device),
                       torch.zeros(0, dtype=torch.float64, device=device), "random_csr")
    colind = _distinct_sorted_columns(lengths, n_cols, g, device)
    val = _uniform(colind.numel(), g, device)
    return HostCSR(n_rows, n_cols, _rowptr_from_lengths(lengths), colind, val, "random_csr")


def dense_to_csr(dense: torch.Tensor) -> HostCSR:
    """CSR of the nonzero pattern of a small dense float64 matrix."""
    dense = dense.to(torch.float64)
    n_rows, n_cols = dense.shape
    mask = dense != 0
    lengths = mask.sum(1)
    colind = torch.nonzero(mask)[:, 1].to(torch.int32)
    return HostCSR(n_rows, n_cols, _rowptr_from_lengths(lengths), colind, dense[mask], "dense")


FAMILIES = ("stencil", "random", "zipf", "short")


MAX_FAMILY_NNZ = 250_000_000


def _zipf_mean(alpha: float, max_len: int) -> float:
    k = torch.arange(1, max_len + 1, dtype=torch.float64)
    w = k.pow(-alpha)
    return float((k * w).sum() / w.sum())


def family_matrix(family: str, n_rows: int, seed: int, device="cpu") -> HostCSR:
    """One matrix of a family with randomized parameters, for selector
    training sets and batched workloads.  ``n_rows`` is a target; stencils round
    it to a grid.  Parameters are clipped so that the expected number of
    nonzeros stays below MAX_FAMILY_NNZ."""
    g = _gen(seed * 7919 + 17, "cpu")  # parameter draws are tiny: always CPU
    if family == "stencil":
        pts = [7, 27][int(torch.randint(0, 2, (1,), generator=g))]
        if pts == 27 and 27 * n_rows > MAX_FAMILY_NNZ:
            pts = 7
        n = max(4, round(n_rows ** (1.0 / 3.0)))
        if pts == 27:
            A = stencil_27pt(n, seed=seed, device=device)
        else:
            A = laplacian_3d_7pt(n, device=device)
            A.val = _uniform(A.nnz, _gen(seed, device), device)
        return A
    if family == "random":
        per_row = int(torch.randint(2, 65, (1,), generator=g))
        per_row = max(1, min(per_row, n_rows, MAX_FAMILY_NNZ // n_rows))
        return random_columns(n_rows, n_rows, per_row, seed=seed, device=device)
    if family == "zipf":
        alpha = 1.2 + 1.3 * float(torch.rand(1, generator=g, dtype=torch.float64))
        max_len = max(2, min(n_rows // 5, 200_000))
        while max_len > 2 and n_rows * _zipf_mean(alpha, max_len) > MAX_FAMILY_NNZ:
            max_len //= 2
        return zipf_rows(n_rows, n_rows, alpha, max_len, seed=seed, device=device)
    if family == "short":
        per = int(torch.randint(1, 5, (1,), generator=g))
        band = int(torch.randint(2, 64, (1,), generator=g))
        if per == 2:
            return short_rows(max(n_rows, band + 1), min(band, 8), seed=seed, device=device)
        gg = _gen(seed, device)
        lengths = torch.full((n_rows,), per, dtype=torch.int64, device=device)
        # banded: columns drawn from a window of width `band` around the row
        width = min(max(band, per), n_rows)
        lengths = torch.clamp(lengths, max=width)
        i = torch.arange(n_rows, device=device)
        lo = torch.clamp(i - width // 2, 0, max(0, n_rows - width))
        cols = _distinct_sorted_columns(lengths, width, gg, device).to(torch.int64)
        cols = cols + torch.repeat_interleave(lo, lengths)
        val = _uniform(cols.numel(), gg, device)
        return HostCSR(n_rows, n_rows, _rowptr_from_lengths(lengths), cols.to(torch.int32),
                       val, f"banded_{n_rows}x{per}")
    raise ValueError(f"unknown family {family!r}")


def four_class_set(device="cpu", scale: int = 0):
    """The four bottleneck-class matrices at full size (scale=0) or shrunk by
    2^scale in rows for quick runs."""
    s = 1 << scale
    n3 = max(8, 128 // round(s ** (1 / 3)))
    return [
        stencil_27pt(n3, seed=0, device=device),
        random_columns((1 << 22) // s, None, 16, seed=0, device=device),
        zipf_rows((1 << 20) // s, None, 1.8, max(2, 200_000 // s), seed=0, device=device),
        short_rows((1 << 23) // s, 8, seed=0, device=device),
    ]


def batch_matrices(count: int = 512, seed: int = 0, lo: float = 1e3, hi: float = 1e5,
                   device="cpu"):
    """A batch of uneven matrices: rows log-uniform in [lo, hi], families
    mixed in turn, row lengths within 2..200 (stencils of 7 or 27 points,
    2-64 random columns per row, Zipf lengths capped at 200, banded rows of
    2-4 nonzeros)."""
    g = _gen(seed, "cpu")
    out = []
    for i in range(count):
        n = int(round(10 ** (math.log10(lo) + (math.log10(hi) - math.log10(lo))
                             * float(torch.rand(1, generator=g, dtype=torch.float64)))))
        fam = FAMILIES[i % 4]
        s = seed * 100_003 + i
        if fam == "stencil":
            m = max(4, round(n ** (1 / 3)))
            A = stencil_27pt(m, seed=s, device=device) if i % 8 == 0 else laplacian_3d_7pt(m, device=device)
            if i % 8 != 0:
                A.val = _uniform(A.nnz, _gen(s, device), device)
        elif fam == "random":
            per = int(torch.randint(2, 65, (1,), generator=g))
            A = random_columns(n, n, min(per, n), seed=s, device=device)
        elif fam == "zipf":
            alpha = 1.5 + float(torch.rand(1, generator=g, dtype=torch.float64))
            A = zipf_rows(n, n, alpha, min(200, n), seed=s, device=device)
        else:
            per = int(torch.randint(2, 5, (1,), generator=g))
            gg = _gen(s, device)
            lengths = torch.full((n,), per, dtype=torch.int64, device=device)
            band = min(32, n)
            i_ = torch.arange(n, device=device)
            lo_ = torch.clamp(i_ - band // 2, 0, max(0, n - band))
            cols = _distinct_sorted_columns(lengths, band, gg, device).to(torch.int64)
            cols = cols + torch.repeat_interleave(lo_, lengths)
            A = HostCSR(n, n, _rowptr_from_lengths(lengths), cols.to(torch.int32),
                        _uniform(cols.numel(), gg, device), f"banded_{n}x{per}")
        out.append(A)
    return out

"""Seeded synthetic sparse matrices and vectors.

These generators are the only code shared by the CPU oracle's tests and the GPU path's
tests and benchmark. They hold no SpMV arithmetic, no feature or classifier logic and no
format encoding: they only draw CSR structures and values from fixed seeds, so that both
sides are fed the same bytes.

The matrix families stand in for the structural classes of the paper's UF/SuiteSparse test
suite (Section IV-A): regular stencils (bandwidth-bound), power-law rows (imbalance and
compute bound), uniformly scattered columns (latency bound) and banded matrices.

Every generator returns a :class:`Csr` with ``int32`` row pointers and column indices
(sorted and unique within each row) and values in the requested floating dtype.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Csr", "laplacian_2d", "stencil_27pt", "stencil_7pt", "power_law", "scattered",
    "banded", "uniform_random", "dense_random", "identity", "permutation", "random_gaps",
    "uniform_vector", "mixed_spec", "make_from_spec", "batched_specs",
    "SEED_BASE", "MAX_NNZ", "max_nnz_lengths", "max_nnz_rows", "max_nnz_x", "max_nnz_device",
]

# Seeds are derived from the arXiv number so that every run draws the same inputs.
SEED_BASE = 171105487


@dataclasses.dataclass
class Csr:
    """A CSR matrix held in host memory (numpy arrays)."""
    n_rows: int
    n_cols: int
    rowptr: np.ndarray   # int32[n_rows + 1]
    colind: np.ndarray   # int32[nnz]
    val: np.ndarray      # float64 / float32 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.colind.shape[0])

    def astype(self, dtype) -> "Csr":
        return Csr(self.n_rows, self.n_cols, self.rowptr, self.colind,
                   self.val.astype(dtype), self.name)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def _rowptr_from_counts(counts: np.ndarray) -> np.ndarray:
    rp = np.zeros(counts.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    if rp[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 indices")
    return rp.astype(np.int32)


def _sorted_distinct_columns(counts: np.ndarray, n_cols: int, rng: np.random.Generator,
                             row_lo: np.ndarray | None = None,
                             row_span: np.ndarray | int | None = None) -> np.ndarray:
    """Draw, for every row i, counts[i] distinct sorted columns.

    Row i's columns lie in [row_lo[i], row_lo[i] + span_i) (the whole [0, n_cols) by
    default). Sorted uniform positions come from normalised partial sums of exponential
    spacings (the order statistics of uniforms), so no sort is needed; adding the rank j
    to the j-th sorted draw from [0, span - k] makes the columns strictly increasing.
    """
    counts = counts.astype(np.int64)
    n = counts.shape[0]
    if row_lo is None:
        row_lo = np.zeros(n, dtype=np.int64)
    if row_span is None:
        row_span = np.full(n, n_cols, dtype=np.int64)
    elif np.isscalar(row_span):
        row_span = np.full(n, int(row_span), dtype=np.int64)
    if np.any(counts > row_span):
        raise ValueError("more nonzeros requested than columns available in a row")
    total = int(counts.sum())
    if total == 0:
        return np.zeros(0, dtype=np.int32)
    ext = counts + 1
    e = rng.standard_exponential(int(ext.sum()))
    csum = np.cumsum(e)
    ends = np.cumsum(ext)              # exclusive end of each row's spacing block
    starts = ends - ext
    before = np.where(starts > 0, csum[np.maximum(starts - 1, 0)], 0.0)
    row_total = csum[ends - 1] - before
    # positions of the first counts[i] partial sums of each row
    keep = np.ones(int(ext.sum()), dtype=bool)
    keep[ends - 1] = False
    row_of = np.repeat(np.arange(n, dtype=np.int64), counts)
    part = csum[keep] - before[row_of]
    m = (row_span - counts + 1)[row_of]
    u = np.floor(part / row_total[row_of] * m).astype(np.int64)
    np.minimum(u, m - 1, out=u)
    # rank of each element inside its row
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    rank = np.arange(total, dtype=np.int64) - rp[:-1][row_of]
    cols = u + rank + row_lo[row_of]
    return cols.astype(np.int32)


def uniform_vector(n: int, seed: int, dtype=np.float64, lo: float = -1.0,
                   hi: float = 1.0) -> np.ndarray:
    """x drawn uniformly from [lo, hi)."""
    return _rng(seed).uniform(lo, hi, size=n).astype(dtype)


def laplacian_2d(nx: int, ny: int | None = None) -> Csr:
    """5-point Laplacian on an nx x ny grid, natural order: 4 on the diagonal, -1 off."""
    ny = nx if ny is None else ny
    n = nx * ny
    ix = np.arange(n, dtype=np.int64) % nx
    iy = np.arange(n, dtype=np.int64) // nx
    # neighbours in increasing column order: (0,-1), (-1,0), (0,0), (+1,0), (0,+1)
    offs = [(0, -1, -nx), (-1, 0, -1), (0, 0, 0), (1, 0, 1), (0, 1, nx)]
    valid = [((ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny))
             for dx, dy, _ in offs]
    counts = np.sum(np.stack(valid), axis=0)
    rowptr = _rowptr_from_counts(counts)
    nnz = int(rowptr[-1])
    colind = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    pos = rowptr[:-1].astype(np.int64).copy()
    rows = np.arange(n, dtype=np.int64)
    for (dx, dy, d), v in zip(offs, valid):
        r = rows[v]
        colind[pos[r]] = (r + d).astype(np.int32)
        val[pos[r]] = 4.0 if d == 0 else -1.0
        pos[r] += 1
    return Csr(n, n, rowptr, colind, val, f"laplacian2d_{nx}x{ny}")


def _stencil_3d(n: int, radius_offsets, seed: int, name: str) -> Csr:
    """Generic 3-D stencil on an n^3 grid in natural order (x fastest).

    Off-diagonal values are uniform in [-1, 1); the diagonal is 1 + sum |off| of its row,
    which makes the matrix strictly diagonally dominant.
    """
    N = n ** 3
    idx = np.arange(N, dtype=np.int64)
    ix = idx % n
    iy = (idx // n) % n
    iz = idx // (n * n)
    offs = sorted(radius_offsets, key=lambda o: (o[2], o[1], o[0]))
    valid = []
    for dx, dy, dz in offs:
        valid.append((ix + dx >= 0) & (ix + dx < n) & (iy + dy >= 0) & (iy + dy < n)
                     & (iz + dz >= 0) & (iz + dz < n))
    counts = np.zeros(N, dtype=np.int64)
    for v in valid:
        counts += v
    rowptr = _rowptr_from_counts(counts)
    nnz = int(rowptr[-1])
    colind = np.empty(nnz, dtype=np.int32)
    pos = rowptr[:-1].astype(np.int64).copy()
    is_diag = np.zeros(nnz, dtype=bool)
    for (dx, dy, dz), v in zip(offs, valid):
        r = idx[v]
        p = pos[r]
        colind[p] = (r + dx + n * dy + n * n * dz).astype(np.int32)
        if dx == 0 and dy == 0 and dz == 0:
            is_diag[p] = True
        pos[r] += 1
    rng = _rng(seed)
    val = rng.uniform(-1.0, 1.0, size=nnz)
    val[is_diag] = 0.0
    row_of = np.repeat(idx, counts)
    absum = np.bincount(row_of, weights=np.abs(val), minlength=N)
    val[is_diag] = 1.0 + absum[row_of[is_diag]]
    return Csr(N, N, rowptr, colind, val, name)


def stencil_27pt(n: int, seed: int = SEED_BASE + 2) -> Csr:
    """27-point stencil on an n^3 grid (config: 160^3, N = 4,096,000)."""
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return _stencil_3d(n, offs, seed, f"stencil27_{n}^3")


def laplacian_27pt(n: int) -> Csr:
    """Symmetric 27-point operator on an n^3 grid (Dirichlet boundary): 26 on the diagonal,
    -1 for each neighbour. Symmetric with a positive diagonal and irreducibly diagonally
    dominant, hence positive definite: the SPD system of the conjugate-gradient solves."""
    m = stencil_27pt(n)
    row_of = np.repeat(np.arange(m.n_rows, dtype=np.int64), np.diff(m.rowptr))
    val = np.where(m.colind == row_of, 26.0, -1.0)
    return Csr(m.n_rows, m.n_cols, m.rowptr, m.colind, val, f"laplacian27_{n}^3")


def stencil_7pt(n: int, seed: int) -> Csr:
    offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    return _stencil_3d(n, offs, seed, f"stencil7_{n}^3")


def power_law(n: int, alpha: float = 1.8, clip: int = 200_000, seed: int = SEED_BASE + 3,
              dtype=np.float32) -> Csr:
    """Row lengths ~ Zipf(alpha) clipped to [1, clip]; columns uniform, distinct, sorted.

    Values are standard normal. Row lengths are drawn with numpy's Zipf sampler (support
    starting at 1) and clipped, as the configuration states.
    """
    rng = _rng(seed)
    clip = min(clip, n)
    lengths = rng.zipf(alpha, size=n)
    np.clip(lengths, 1, clip, out=lengths)
    rowptr = _rowptr_from_counts(lengths)
    colind = _sorted_distinct_columns(lengths, n, rng)
    val = rng.standard_normal(colind.shape[0]).astype(dtype)
    return Csr(n, n, rowptr, colind, val, f"powerlaw_a{alpha}_{n}")


def scattered(n: int, k: int = 8, seed: int = SEED_BASE + 4, dtype=np.float64) -> Csr:
    """Exactly k nonzeros per row at uniform random distinct columns; values U[-1, 1)."""
    rng = _rng(seed)
    counts = np.full(n, k, dtype=np.int64)
    rowptr = _rowptr_from_counts(counts)
    colind = _sorted_distinct_columns(counts, n, rng)
    val = rng.uniform(-1.0, 1.0, size=colind.shape[0]).astype(dtype)
    return Csr(n, n, rowptr, colind, val, f"scattered_k{k}_{n}")


def banded(n: int, half_bw: int, density: float, seed: int, dtype=np.float64) -> Csr:
    """Random banded matrix: row i draws columns in [i - half_bw, i + half_bw] ∩ [0, n)
    with the given density (at least one nonzero per row)."""
    rng = _rng(seed)
    i = np.arange(n, dtype=np.int64)
    lo = np.maximum(i - half_bw, 0)
    hi = np.minimum(i + half_bw, n - 1)
    span = hi - lo + 1
    counts = np.maximum(1, rng.binomial(span, density))
    counts = np.minimum(counts, span)
    rowptr = _rowptr_from_counts(counts)
    colind = _sorted_distinct_columns(counts, n, rng, row_lo=lo, row_span=span)
    val = rng.uniform(-1.0, 1.0, size=colind.shape[0]).astype(dtype)
    return Csr(n, n, rowptr, colind, val, f"banded_h{half_bw}_{n}")


def uniform_random(n: int, max_per_row: int, seed: int, dtype=np.float64,
                   min_per_row: int = 1, n_cols: int | None = None) -> Csr:
    """Row lengths uniform in [min_per_row, max_per_row]; columns uniform distinct."""
    rng = _rng(seed)
    n_cols = n if n_cols is None else n_cols
    counts = rng.integers(min_per_row, max_per_row + 1, size=n)
    counts = np.minimum(counts, n_cols)
    rowptr = _rowptr_from_counts(counts)
    colind = _sorted_distinct_columns(counts, n_cols, rng)
    val = rng.uniform(-1.0, 1.0, size=colind.shape[0]).astype(dtype)
    return Csr(n, n_cols, rowptr, colind, val, f"uniform_{max_per_row}_{n}")


def same_sign_rows(lengths, n_cols: int, seed: int, dtype=np.float64) -> Csr:
    """Rows of the given lengths, distinct uniform columns, values uniform in [0.5, 1]: with a
    positive x every product of a row has the same sign (no cancellation)."""
    rng = _rng(seed)
    counts = np.minimum(np.asarray(lengths, dtype=np.int64), n_cols)
    rowptr = _rowptr_from_counts(counts)
    colind = _sorted_distinct_columns(counts, n_cols, rng)
    val = rng.uniform(0.5, 1.0, size=colind.shape[0]).astype(dtype)
    return Csr(int(counts.shape[0]), n_cols, rowptr, colind, val, f"same_sign_{counts.shape[0]}")


def dense_random(n_rows: int, n_cols: int, density: float, seed: int,
                 integer_values: bool = True) -> Csr:
    """Small matrix drawn as a dense mask; integer values keep FP64 sums exact."""
    rng = _rng(seed)
    mask = rng.random((n_rows, n_cols)) < density
    if integer_values:
        vals = rng.integers(-8, 9, size=(n_rows, n_cols)).astype(np.float64)
        vals[vals == 0] = 1.0
    else:
        vals = rng.uniform(-1, 1, size=(n_rows, n_cols))
    counts = mask.sum(axis=1)
    rowptr = _rowptr_from_counts(counts)
    r, c = np.nonzero(mask)
    return Csr(n_rows, n_cols, rowptr, c.astype(np.int32), vals[r, c].astype(np.float64),
               f"dense_{n_rows}x{n_cols}")


def identity(n: int) -> Csr:
    return Csr(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
               np.ones(n, dtype=np.float64), f"identity_{n}")


def random_gaps(n_rows: int, n_cols: int, max_len: int, gap_scale: float, seed: int,
                dtype=np.float64) -> Csr:
    """Rows of 0..max_len sorted unique columns whose gaps are drawn geometrically around
    gap_scale times a per-row factor of 0.01, 1 or 100, so one matrix mixes rows with small
    gaps, gaps of thousands and gaps past 65,536; in about 30 % of rows one gap is set to
    exactly 255, 256, 65,535 or 65,536. Values U[-1, 1]."""
    rng = _rng(seed)
    rows = []
    for _ in range(n_rows):
        length = int(rng.integers(0, max_len + 1))
        if length == 0:
            rows.append(np.zeros(0, np.int64))
            continue
        scale = gap_scale * float(rng.choice([0.01, 1.0, 100.0]))
        gaps = rng.geometric(min(1.0, 1.0 / max(scale, 1.0)), length - 1)
        if gaps.size and rng.random() < 0.3:
            gaps[rng.integers(0, gaps.size)] = rng.choice([255, 256, 65535, 65536])
        start = int(rng.integers(0, n_cols))
        cols = start + np.concatenate([[0], np.cumsum(gaps)])
        rows.append(cols[cols < n_cols])
    counts = np.array([r.size for r in rows], np.int64)
    colind = (np.concatenate(rows) if rows else np.zeros(0)).astype(np.int32)
    val = rng.uniform(-1, 1, colind.size).astype(dtype)
    return Csr(n_rows, n_cols, _rowptr_from_counts(counts), colind, val,
               f"random_gaps_{n_rows}x{n_cols}_s{seed}")


def permutation(n: int, seed: int) -> Csr:
    """P with P[i, pi(i)] = 1, so (P x)_i = x[pi(i)]."""
    pi = _rng(seed).permutation(n).astype(np.int32)
    return Csr(n, n, np.arange(n + 1, dtype=np.int32), pi, np.ones(n, dtype=np.float64),
               f"permutation_{n}")


# ---------------------------------------------------------------------------------------
# Mixed matrix sets (learned-selector training set, batched workload)
# ---------------------------------------------------------------------------------------

# --------------------------------------------------------------------------------------
# The largest matrix a handle accepts: nnz just under 2^31 - 2^21 - 1, so that row offsets
# near the top of int32 are exercised. Too large to build on the host, it is given in closed
# form: max_nnz_device builds the whole CSR on a CUDA device with torch, max_nnz_rows any set
# of its rows with numpy, both from the same formulas.
#   rows 2^25, columns 2^20; row lengths 64, except a band of rows of 32 starting at row 2^24
#   (sized so that the total lands just under the limit), rows 1,000,003 k (k >= 1) of 16
#   whose columns are 65,536 apart (delta-index escape rows), and the last three rows of
#   300,000 (long rows, chunked by the row decomposition);
#   column k of row i: 4096 k + (i mod 4096), for the rows of 16: 65536 k + (i mod 4096),
#   for the rows of 300,000: 3 k + (i mod 3);
#   value at position j: ((j * 2654435761) mod 2^31) / 2^30 - 1; x[c]: ((c * 40503) mod
#   65536) / 32768 - 1 (both exact in FP64, in [-1, 1)).

MAX_NNZ = 2 ** 31 - 2 ** 21 - 1
MAX_NNZ_ROWS = 1 << 25
MAX_NNZ_COLS = 1 << 20


def max_nnz_lengths() -> np.ndarray:
    """Row lengths (int64) of the maximum-size matrix."""
    n = MAX_NNZ_ROWS
    lens = np.full(n, 64, np.int64)
    lens[np.arange(1_000_003, n, 1_000_003)] = 16
    lens[-3:] = 300_000
    excess = int(lens.sum()) - (MAX_NNZ - 128)
    band = np.arange(1 << 24, n)
    band = band[lens[band] == 64][: -(-excess // 32)]
    lens[band] = 32
    assert MAX_NNZ - 1024 < lens.sum() <= MAX_NNZ
    return lens


def _max_nnz_stride_offset(i, lens, xp):
    """Per row: the column stride and first column (numpy or torch arrays)."""
    stride = xp.where(lens == 16, 65536, xp.where(lens == 300_000, 3, 4096))
    off = xp.where(lens == 300_000, i % 3, i % 4096)
    return stride, off


def _max_nnz_hash(j):
    return (j * 2654435761) % 2 ** 31   # j < 2^31: the product stays below 2^63


def max_nnz_x() -> np.ndarray:
    c = np.arange(MAX_NNZ_COLS, dtype=np.int64)
    return ((c * 40503) % 65536) / 32768.0 - 1.0


def max_nnz_rows(rows) -> Csr:
    """The given rows of the maximum-size matrix, in the order given, as a CSR of their own
    (FP64 values)."""
    lens = max_nnz_lengths()
    rp_full = np.zeros(MAX_NNZ_ROWS + 1, np.int64)
    np.cumsum(lens, out=rp_full[1:])
    rows = np.asarray(rows, np.int64)
    counts = lens[rows]
    rp = _rowptr_from_counts(counts)
    row_of = np.repeat(rows, counts)
    k = np.arange(int(counts.sum()), dtype=np.int64) - np.repeat(rp[:-1].astype(np.int64), counts)
    stride, off = _max_nnz_stride_offset(row_of, lens[row_of], np)
    cols = (k * stride + off).astype(np.int32)
    vals = _max_nnz_hash(rp_full[row_of] + k).astype(np.float64) / 2.0 ** 30 - 1.0
    return Csr(len(rows), MAX_NNZ_COLS, rp, cols, vals, "max_nnz_rows")


def max_nnz_device(torch, device="cuda"):
    """(rowptr int32, colind int32, val float64) of the whole maximum-size matrix as tensors
    on the device (about 26 GB), built from the closed form in bounded pieces."""
    lens_h = max_nnz_lengths()
    n = MAX_NNZ_ROWS
    rp64 = torch.zeros(n + 1, dtype=torch.int64, device=device)
    rp64[1:] = torch.cumsum(torch.from_numpy(lens_h).to(device), 0)
    nnz = int(rp64[-1])
    col = torch.empty(nnz, dtype=torch.int32, device=device)
    val = torch.empty(nnz, dtype=torch.float64, device=device)
    lens = torch.from_numpy(lens_h).to(device)
    piece = 1 << 21   # rows per piece (about 134 M nonzeros)
    for r0 in range(0, n, piece):
        r1 = min(r0 + piece, n)
        rows = torch.arange(r0, r1, dtype=torch.int64, device=device)
        ln = lens[r0:r1]
        s0, s1 = int(rp64[r0]), int(rp64[r1])
        row_of = torch.repeat_interleave(rows, ln)
        j = torch.arange(s0, s1, dtype=torch.int64, device=device)
        k = j - rp64[row_of]
        stride, off = _max_nnz_stride_offset(row_of, lens[row_of], torch)
        col[s0:s1] = (k * stride + off).to(torch.int32)
        val[s0:s1] = _max_nnz_hash(j).to(torch.float64) / 2.0 ** 30 - 1.0
        del row_of, j, k, stride, off
    return rp64.to(torch.int32), col, val


FAMILIES = ("stencil", "powerlaw", "banded", "random")


def mixed_spec(index: int, seed: int = SEED_BASE + 40, n_lo: int = 10_000,
               n_hi: int = 1_000_000, family: str | None = None) -> dict:
    """Parameters of matrix `index` of a mixed set (pure function of index and seed).

    Families rotate stencil / power-law / banded / uniform-random; N is log-uniform in
    [n_lo, n_hi].
    """
    rng = _rng(seed * 7919 + index)
    fam = family or FAMILIES[index % len(FAMILIES)]
    n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    spec = {"index": index, "family": fam, "seed": int(seed * 1000003 + index)}
    if fam == "stencil":
        kind = int(rng.integers(0, 3))
        if kind == 0:     # 2-D 5-point
            side = max(4, int(round(math.sqrt(n))))
            spec.update(kind="lap2d", side=side)
        elif kind == 1:   # 3-D 7-point
            side = max(3, int(round(n ** (1 / 3))))
            spec.update(kind="st7", side=side)
        else:             # 3-D 27-point
            side = max(3, int(round(n ** (1 / 3))))
            spec.update(kind="st27", side=side)
    elif fam == "powerlaw":
        spec.update(n=n, alpha=float(rng.uniform(1.6, 2.6)), clip=min(n, 20_000))
    elif fam == "banded":
        hb = max(1, int(round(math.exp(rng.uniform(0.0, math.log(max(2.0, n / 10)))))))
        # density per band U(0.05, 1), capped so that a row holds about 64 nonzeros at most
        dens = min(float(rng.uniform(0.05, 1.0)), 64.0 / (2 * hb + 1))
        spec.update(n=n, half_bw=hb, density=dens)
    else:
        spec.update(n=n, max_per_row=int(rng.integers(1, 65)))
    return spec


def make_from_spec(spec: dict, dtype=np.float64) -> Csr:
    fam = spec["family"]
    seed = spec["seed"]
    if fam == "stencil":
        if spec["kind"] == "lap2d":
            m = laplacian_2d(spec["side"])
        elif spec["kind"] == "st7":
            m = stencil_7pt(spec["side"], seed)
        else:
            m = stencil_27pt(spec["side"], seed)
    elif fam == "powerlaw":
        m = power_law(spec["n"], spec["alpha"], clip=spec.get("clip", spec["n"]), seed=seed,
                      dtype=np.float64)
    elif fam == "banded":
        m = banded(spec["n"], spec["half_bw"], spec["density"], seed)
    else:
        m = uniform_random(spec["n"], spec["max_per_row"], seed)
    m.name = f"{fam}_{spec['index']}"
    return m.astype(dtype)


def batched_specs(count: int = 512, seed: int = SEED_BASE + 50, n_lo: int = 1_000,
                  n_hi: int = 200_000) -> list[dict]:
    """The batched workload: `count` mixed matrices with N log-uniform in [n_lo, n_hi] and
    a right-hand-side count k in {1, 4, 16} drawn per matrix."""
    out = []
    rng = _rng(seed)
    ks = rng.choice(np.array([1, 4, 16]), size=count)
    for i in range(count):
        s = mixed_spec(i, seed=seed, n_lo=n_lo, n_hi=n_hi)
        s["k"] = int(ks[i])
        out.append(s)
    return out

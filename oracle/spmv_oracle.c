/*
 * CPU oracle for the bottleneck-adaptive CSR SpMV method of Elafrou, Goumas and Koziris,
 * "Performance Analysis and Optimization of Sparse Matrix-Vector Multiplication on Modern
 * Multi- and Many-Core Processors" (arXiv 1711.05487).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain, obviously-correct reference that
 * the GPU library is checked against. It shares no code, header, table or constant
 * generator with the CUDA library; only the tests, the package entry point's smoke check
 * and the benchmark's CPU-baseline leg may load it. Every loop runs in the order the paper
 * states, in FP64 unless noted. Build flags must keep floating-point contraction off
 * (-ffp-contract=off) so that the FP32 selector inference below performs exactly the
 * operations it spells out.
 *
 * Contents (each function cites the passage it follows):
 *   - CSR validation                         (Section II, CSR definition)
 *   - y = A x in FP64, plus sum |a_ij x_j|    (Section II, Fig. 1)
 *   - multi-RHS y = A X                       (Fig. 1 applied column by column)
 *   - FP64 -> FP32 / BF16 round-to-nearest-even value storage
 *   - 8- and 16-bit delta column-index formats and the width choice (Section III-E, MB)
 *   - merge-path coordinates of a CSR matrix (Section III-E, IMB optimization: the
 *     nnz-balanced work split)
 *   - row decomposition into short, medium and chunked long rows (Section III-E, IMB:
 *     the matrix decomposition of Fig. 5)
 *   - Table I matrix features                (Section III-D)
 *   - P_MB and P_peak bounds                 (Section III-B)
 *   - Classify rule set                      (Section III-C, Fig. 3)
 *   - class -> optimization map              (Section III-E, Table II)
 *   - amortization iterations                (Section IV-D, N_iters,min)
 *   - conjugate gradients on y = A x         (Section IV-D's iterative-solver setting;
 *     Hestenes and Stiefel's method)
 *   - double-float split of FP64 values      (the library's DF64 storage)
 *   - MLP selector: FP64 loss and gradient, FP32 inference, log2(1+v) normalisation
 *     (the learned selector that stands in for the decision tree of Section III-D)
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------------------------- */
/* CSR validation (Section II: rowptr indexes the start of each row within the arrays of
 * nonzeros; colind holds each nonzero's column).                                       */
/* Return codes: 0 valid, 1 rowptr[0] != 0, 2 rowptr decreases, 3 rowptr[N] != nnz,
 *               4 column out of [0, n_cols), 5 columns not strictly increasing in a row,
 *               6 negative sizes.                                                       */
int oracle_validate_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t *rowptr,
                        const int32_t *colind) {
  if (n_rows < 0 || n_cols < 0 || nnz < 0) return 6;
  if (rowptr[0] != 0) return 1;
  for (int64_t i = 0; i < n_rows; ++i)
    if (rowptr[i + 1] < rowptr[i]) return 2;
  if ((int64_t)rowptr[n_rows] != nnz) return 3;
  for (int64_t i = 0; i < n_rows; ++i) {
    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
      if (colind[j] < 0 || (int64_t)colind[j] >= n_cols) return 4;
      if (j > rowptr[i] && colind[j] <= colind[j - 1]) return 5;
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------------- */
/* y = A x (Fig. 1). The statement inside the inner loop accumulates into y[i], which
 * starts at zero: the caption and Section II call this the y = A.x kernel, so the
 * assignment printed in the figure is read as y[i] <- y[i] + val[j] * x[colind[j]].
 * s[i] = sum_j |val[j] * x[colind[j]]| is the scale that the accuracy bound of each
 * result row is stated against. Empty rows give y[i] = s[i] = 0.                       */
void oracle_spmv_f64(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                     const double *val, const double *x, double *y, double *s) {
  for (int64_t i = 0; i < n_rows; ++i) {
    double acc = 0.0, mag = 0.0;
    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
      double p = val[j] * x[colind[j]];
      acc += p;
      mag += fabs(p);
    }
    y[i] = acc;
    if (s) s[i] = mag;
  }
}

/* The paper's baseline CSR scheme (Section IV-A): rows are split into n_threads contiguous
 * ranges of about NNZ / n_threads nonzeros each (static, nnz-balanced; range t starts at the
 * first row whose rowptr reaches t NNZ / n_threads) and each range is one OpenMP thread's.
 * Every row is the same sequential sum as in oracle_spmv_f64, so y is bit-identical to it.
 * Returns the number of threads that ran (1 when built without OpenMP). */
int32_t oracle_spmv_f64_static(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                               const double *val, const double *x, double *y,
                               int32_t n_threads) {
  if (n_threads < 1) n_threads = 1;
  const int64_t nnz = n_rows > 0 ? rowptr[n_rows] : 0;
  int32_t used = 1;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
  {
    const int32_t T = (int32_t)omp_get_num_threads();
    const int32_t t = (int32_t)omp_get_thread_num();
    if (t == 0) used = T;
#else
  {
    const int32_t T = 1, t = 0;
#endif
    /* first row of a range: lower bound of the target nonzero count in rowptr */
    int64_t bounds[2];
    for (int q = 0; q < 2; ++q) {
      const int64_t target = (int64_t)(((__int128)nnz * (t + q)) / T);
      int64_t lo = 0, hi = n_rows;
      while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (rowptr[mid] < target) lo = mid + 1;
        else hi = mid;
      }
      bounds[q] = (t + q == T) ? n_rows : lo;
    }
    for (int64_t i = bounds[0]; i < bounds[1]; ++i) {
      double acc = 0.0;
      for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) acc += val[j] * x[colind[j]];
      y[i] = acc;
    }
  }
  return used;
}

/* The same sum for a list of rows only (used to check sampled rows of large matrices). */
void oracle_spmv_rows_f64(const int64_t *rows, int64_t n_sample, const int32_t *rowptr,
                          const int32_t *colind, const double *val, const double *x,
                          double *y, double *s) {
  for (int64_t r = 0; r < n_sample; ++r) {
    int64_t i = rows[r];
    double acc = 0.0, mag = 0.0;
    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
      double p = val[j] * x[colind[j]];
      acc += p;
      mag += fabs(p);
    }
    y[r] = acc;
    s[r] = mag;
  }
}

/* Y = A X for k right-hand sides, X and Y row-major (N x k): Fig. 1 for every column. */
void oracle_spmm_f64(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                     const double *val, const double *X, int64_t k, double *Y, double *S) {
  for (int64_t i = 0; i < n_rows; ++i) {
    for (int64_t c = 0; c < k; ++c) {
      double acc = 0.0, mag = 0.0;
      for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
        double p = val[j] * X[(int64_t)colind[j] * k + c];
        acc += p;
        mag += fabs(p);
      }
      Y[i * k + c] = acc;
      S[i * k + c] = mag;
    }
  }
}

/* ---------------------------------------------------------------------------------- */
/* Reduced-precision value storage: round-to-nearest-even straight from the FP64 value.
 * FP32: C's double -> float conversion rounds to nearest even in the default mode.       */
void oracle_round_f32(const double *in, float *out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) out[i] = (float)in[i];
}

/* BF16 (1 sign, 8 exponent, 7 fraction bits; same exponent range as FP32). For finite v:
 * the quantum is 2^(max(e, -126) - 7) with v = m 2^e, 1 <= |m| < 2; v / quantum is exact
 * (power-of-two scaling) and rint() rounds it to the nearest integer, ties to even.
 * Magnitudes that round to 2^128 or more become infinity. NaN stays NaN (quiet).        */
static uint16_t bf16_bits_of_exact(double r) {
  /* r is exactly representable in bf16: its float image is exact, take the top half. */
  float f = (float)r;
  uint32_t u;
  memcpy(&u, &f, sizeof u);
  return (uint16_t)(u >> 16);
}

void oracle_round_bf16(const double *in, uint16_t *out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    double v = in[i];
    if (isnan(v)) {
      out[i] = signbit(v) ? 0xFFC0u : 0x7FC0u;
      continue;
    }
    if (isinf(v) || v == 0.0) {
      out[i] = bf16_bits_of_exact(v);
      continue;
    }
    int e;
    (void)frexp(v, &e);          /* v = f 2^e with 0.5 <= |f| < 1, so |v| in [2^(e-1), 2^e) */
    int ex = e - 1;              /* v = m 2^ex with 1 <= |m| < 2                            */
    if (ex < -126) ex = -126;    /* subnormal range keeps the smallest normal's quantum     */
    double q = ldexp(1.0, ex - 7);
    double r = rint(v / q) * q;
    if (fabs(r) >= ldexp(1.0, 128)) r = signbit(v) ? -INFINITY : INFINITY;
    out[i] = bf16_bits_of_exact(r);
  }
}

/* Double-float split of FP64 values (the library's DF64 storage; no counterpart in the
 * paper): v = hi + lo + r with hi = v truncated toward zero to 24 significant bits and
 * lo = (v - hi) truncated toward zero at the quantum 2^(e - 46), e = floor(log2 |v|), so
 * |r| < 2^(e - 46). Both are FP32 numbers, returned as bit patterns; a zero lo is +0.
 * Zero gives (+-0, 0);
 * a nonzero with e outside [-40, 40], an infinity or a NaN gives (0x7FC00000, 0). The
 * subtractions below are exact: each operand and result is a multiple of the quantum and
 * below 2^53 quanta.                                                                     */
static uint32_t f32_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, sizeof u);
  return u;
}

void oracle_df_split(const double *in, uint32_t *out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    const double v = in[i];
    uint32_t hi_bits, lo_bits = 0;
    if (v == 0.0) {
      hi_bits = signbit(v) ? 0x80000000u : 0u;
    } else if (!isfinite(v)) {
      hi_bits = 0x7FC00000u;
    } else {
      int e2;
      (void)frexp(v, &e2);
      const int e = e2 - 1;                        /* 2^e <= |v| < 2^(e+1) */
      if (e < -40 || e > 40) {
        hi_bits = 0x7FC00000u;
      } else {
        const double q_hi = ldexp(1.0, e - 23);    /* 24 significant bits */
        const double hi = trunc(v / q_hi) * q_hi;
        const double q_lo = ldexp(1.0, e - 46);    /* 23 more bits */
        double lo = trunc((v - hi) / q_lo) * q_lo;
        if (lo == 0.0) lo = 0.0;                   /* a zero low part is +0 */
        hi_bits = f32_bits((float)hi);             /* exact: hi, lo fit FP32 */
        lo_bits = f32_bits((float)lo);
      }
    }
    out[2 * i] = hi_bits;
    out[2 * i + 1] = lo_bits;
  }
}

/* Conjugate gradients (Hestenes and Stiefel 1952), the solver setting of Section IV-D in
 * which the tuned SpMV is applied once per iteration. In the textbook order:
 *   r_0 = b - A x_0, p_0 = r_0;
 *   for k = 0, 1, ...: alpha_k = (r_k, r_k) / (p_k, A p_k); x_{k+1} = x_k + alpha_k p_k;
 *     r_{k+1} = r_k - alpha_k A p_k; beta_k = (r_{k+1}, r_{k+1}) / (r_k, r_k);
 *     p_{k+1} = r_{k+1} + beta_k p_k,
 * stopping when ||r_k|| <= rtol ||b|| or after max_iters iterations. alpha (beta) is 0 when
 * its denominator is 0. x holds x_0 on entry and the last iterate on return; hist (may be
 * NULL) receives ||r_k|| for k = 0 .. iterations. Dot products are plain sequential FP64
 * sums. Returns the number of iterations; *converged tells whether the test was met. */
static double dot_f64(int64_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

int64_t oracle_cg(int64_t n, const int32_t *rowptr, const int32_t *colind, const double *val,
                  const double *b, double *x, int64_t max_iters, double rtol, double *hist,
                  int32_t *converged) {
  double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *p = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *ap = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  oracle_spmv_f64(n, rowptr, colind, val, x, ap, NULL);
  for (int64_t i = 0; i < n; ++i) {
    r[i] = b[i] - ap[i];
    p[i] = r[i];
  }
  const double b_norm = sqrt(dot_f64(n, b, b));
  double rr = dot_f64(n, r, r);
  if (hist) hist[0] = sqrt(rr);
  int64_t k = 0;
  *converged = sqrt(rr) <= rtol * b_norm;
  while (!*converged && k < max_iters) {
    oracle_spmv_f64(n, rowptr, colind, val, p, ap, NULL);
    const double pap = dot_f64(n, p, ap);
    const double alpha = pap != 0.0 ? rr / pap : 0.0;
    for (int64_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * ap[i];
    }
    const double rr_new = dot_f64(n, r, r);
    const double beta = rr != 0.0 ? rr_new / rr : 0.0;
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    rr = rr_new;
    ++k;
    if (hist) hist[k] = sqrt(rr);
    *converged = sqrt(rr) <= rtol * b_norm;
  }
  free(r);
  free(p);
  free(ap);
  return k;
}

/* Row decomposition for thread imbalance (Section III-E, IMB: A = A_short + A_long, Fig. 5):
 * a row of length len is long when len >= chunk, medium when l_med <= len < chunk, short
 * otherwise. Long row r is cut into chunks [z, min(z + chunk, rowptr[r+1])) for
 * z = rowptr[r], rowptr[r] + chunk, ... . Outputs in row order: med_rows[], long_rows[],
 * long_first[] (first chunk of each long row, then the chunk count), chunks[] as
 * (row, begin z, end, start column) where the start column is the column a delta decode
 * of the chunk starts from: colind[z - 1] inside the row, colind[z] (whose delta is 0) for
 * the row's first chunk. counts[0..2] = medium rows, long rows, chunks.                  */
void oracle_row_bins(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                     int32_t l_med, int32_t chunk, int32_t *med_rows, int32_t *long_rows,
                     int32_t *long_first, int32_t *chunks, int64_t *counts) {
  int64_t n_med = 0, n_long = 0, n_ch = 0;
  for (int64_t r = 0; r < n_rows; ++r) {
    const int32_t b = rowptr[r], e = rowptr[r + 1];
    const int32_t len = e - b;
    if (len >= chunk) {
      long_rows[n_long] = (int32_t)r;
      long_first[n_long] = (int32_t)n_ch;
      ++n_long;
      for (int32_t z = b; z < e; z += chunk) {
        chunks[4 * n_ch] = (int32_t)r;
        chunks[4 * n_ch + 1] = z;
        chunks[4 * n_ch + 2] = (z + chunk < e) ? z + chunk : e;
        chunks[4 * n_ch + 3] = z > b ? colind[z - 1] : colind[z];
        ++n_ch;
      }
    } else if (len >= l_med) {
      med_rows[n_med++] = (int32_t)r;
    }
  }
  long_first[n_long] = (int32_t)n_ch;
  counts[0] = n_med;
  counts[1] = n_long;
  counts[2] = n_ch;
}

/* ---------------------------------------------------------------------------------- */
/* Sliced rows (SELL-32; a GB300 layout for the CMP class, not in the paper): rows are taken
 * in slices of 32 consecutive rows (the last slice may hold fewer); slice s holds w_s = the
 * longest row length in the slice elements per row, stored column-major: element k of row
 * 32 s + l sits at soff[s] + 32 k + l, where soff[0] = 0 and soff[s+1] = soff[s] + 32 w_s.
 * Positions past a row's length (and the lanes of missing rows in the last slice) are
 * padding. perm[p] is the CSR position of the element at p, or -1 for padding. Returns the
 * number of positions soff[n_slices].                                                    */
int64_t oracle_sell32(int64_t n_rows, const int32_t *rowptr, int64_t *soff, int32_t *perm) {
  const int64_t ns = (n_rows + 31) / 32;
  soff[0] = 0;
  for (int64_t s = 0; s < ns; ++s) {
    int64_t w = 0;
    for (int64_t r = 32 * s; r < 32 * s + 32 && r < n_rows; ++r)
      if (rowptr[r + 1] - rowptr[r] > w) w = rowptr[r + 1] - rowptr[r];
    soff[s + 1] = soff[s] + 32 * w;
  }
  for (int64_t s = 0; s < ns; ++s) {
    const int64_t w = (soff[s + 1] - soff[s]) / 32;
    for (int64_t l = 0; l < 32; ++l) {
      const int64_t r = 32 * s + l;
      const int64_t len = r < n_rows ? rowptr[r + 1] - rowptr[r] : 0;
      for (int64_t k = 0; k < w; ++k)
        perm[soff[s] + 32 * k + l] = k < len ? (int32_t)(rowptr[r] + k) : -1;
    }
  }
  return soff[ns];
}

/* ---------------------------------------------------------------------------------- */
/* Column panels (Section III-E, ML: make the irregular accesses to x hit in cache; read on
 * GB300 as cutting x into P slices that each fit in the L2 and running the SpMV as one pass
 * per slice). Panel p holds the columns [p*w, (p+1)*w), w = oracle_panel_width(n_cols, P):
 * ceil(n_cols / P) rounded up to a multiple of 32 (trailing panels may be empty). The
 * panel-major copy lists panel 0's nonzeros row by row, then panel 1's, and so on; inside a
 * row the columns keep their order. prow[p*(n_rows+1) + i] is the position in the copy of
 * row i's first nonzero of panel p, prow[p*(n_rows+1) + n_rows] the end of panel p, and
 * perm[k] the position in the original CSR of copy element k.                           */
int32_t oracle_panel_width(int64_t n_cols, int32_t n_panels) {
  int64_t w = (n_cols + n_panels - 1) / n_panels;
  w = (w + 31) / 32 * 32;
  return (int32_t)(w > 0 ? w : 32);
}

void oracle_col_panels(int64_t n_rows, int64_t n_cols, const int32_t *rowptr,
                       const int32_t *colind, int32_t n_panels, int32_t *prow, int32_t *perm) {
  const int64_t w = oracle_panel_width(n_cols, n_panels);
  int64_t k = 0;
  for (int32_t p = 0; p < n_panels; ++p) {
    const int64_t lo = (int64_t)p * w, hi = lo + w;
    for (int64_t i = 0; i < n_rows; ++i) {
      prow[(int64_t)p * (n_rows + 1) + i] = (int32_t)k;
      for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j)
        if (colind[j] >= lo && colind[j] < hi) perm[k++] = (int32_t)j;
    }
    prow[(int64_t)p * (n_rows + 1) + n_rows] = (int32_t)k;
  }
}

/* ---------------------------------------------------------------------------------- */
/* Delta-indexed column indices (Section III-E, MB row of Table II): each column index is
 * stored as its distance to the previous column of the same row, in 16 bits wherever
 * possible. Read per row: a row whose every consecutive distance fits 16 bits keeps its
 * first column in base[i] and stores delta[j] = colind[j] - colind[j-1] (delta of the
 * row's first element = 0). A row with a distance above 65535 is an escape row: its
 * deltas are 0, its columns go to esc_col in row order, and base[i] = -(1 + offset of the
 * row in esc_col). An empty row has base[i] = 0. Returns the number of escaped columns. */
int64_t oracle_delta16_encode(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                              int32_t *base, uint16_t *delta, int32_t *esc_col) {
  int64_t n_esc = 0;
  for (int64_t i = 0; i < n_rows; ++i) {
    int64_t b = rowptr[i], e = rowptr[i + 1];
    if (b == e) {
      base[i] = 0;
      continue;
    }
    int fits = 1;
    for (int64_t j = b + 1; j < e; ++j)
      if ((int64_t)colind[j] - (int64_t)colind[j - 1] > 65535) fits = 0;
    if (fits) {
      base[i] = colind[b];
      delta[b] = 0;
      for (int64_t j = b + 1; j < e; ++j) delta[j] = (uint16_t)(colind[j] - colind[j - 1]);
    } else {
      base[i] = (int32_t)(-(1 + n_esc));
      for (int64_t j = b; j < e; ++j) {
        delta[j] = 0;
        esc_col[n_esc++] = colind[j];
      }
    }
  }
  return n_esc;
}

/* Inverse of the above: rebuild colind from (base, delta, esc_col). */
void oracle_delta16_decode(int64_t n_rows, const int32_t *rowptr, const int32_t *base,
                           const uint16_t *delta, const int32_t *esc_col, int32_t *colind) {
  for (int64_t i = 0; i < n_rows; ++i) {
    int64_t b = rowptr[i], e = rowptr[i + 1];
    if (b == e) continue;
    if (base[i] < 0) {
      int64_t off = -(int64_t)base[i] - 1;
      for (int64_t j = b; j < e; ++j) colind[j] = esc_col[off + (j - b)];
    } else {
      int64_t c = base[i];
      for (int64_t j = b; j < e; ++j) {
        c += delta[j];
        colind[j] = (int32_t)c;
      }
    }
  }
}

/* The 8-bit form of the same index: a row whose consecutive column distances all fit 8 bits
 * stores them as uint8 (first delta 0), any other non-empty row is an escape row.          */
int64_t oracle_delta8_encode(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                             int32_t *base, uint8_t *delta, int32_t *esc_col) {
  int64_t n_esc = 0;
  for (int64_t i = 0; i < n_rows; ++i) {
    int64_t b = rowptr[i], e = rowptr[i + 1];
    if (b == e) {
      base[i] = 0;
      continue;
    }
    int fits = 1;
    for (int64_t j = b + 1; j < e; ++j)
      if ((int64_t)colind[j] - (int64_t)colind[j - 1] > 255) fits = 0;
    if (fits) {
      base[i] = colind[b];
      delta[b] = 0;
      for (int64_t j = b + 1; j < e; ++j) delta[j] = (uint8_t)(colind[j] - colind[j - 1]);
    } else {
      base[i] = (int32_t)(-(1 + n_esc));
      for (int64_t j = b; j < e; ++j) {
        delta[j] = 0;
        esc_col[n_esc++] = colind[j];
      }
    }
  }
  return n_esc;
}

void oracle_delta8_decode(int64_t n_rows, const int32_t *rowptr, const int32_t *base,
                          const uint8_t *delta, const int32_t *esc_col, int32_t *colind) {
  for (int64_t i = 0; i < n_rows; ++i) {
    int64_t b = rowptr[i], e = rowptr[i + 1];
    if (b == e) continue;
    if (base[i] < 0) {
      int64_t off = -(int64_t)base[i] - 1;
      for (int64_t j = b; j < e; ++j) colind[j] = esc_col[off + (j - b)];
    } else {
      int64_t c = base[i];
      for (int64_t j = b; j < e; ++j) {
        c += delta[j];
        colind[j] = (int32_t)c;
      }
    }
  }
}

/* "8- or 16-bit deltas wherever possible, never both" (Section III-E, MB): one width per
 * matrix, the one whose index is smaller. Index bytes of width w: w/8 per nonzero of the
 * rows that fit w, 4 per nonzero of the escape rows (the per-row base is the same for
 * both). Returns 8 when that is strictly fewer bytes than 16, else 16.                    */
int32_t oracle_delta_width(int64_t n_rows, const int32_t *rowptr, const int32_t *colind) {
  int64_t bytes8 = 0, bytes16 = 0;
  for (int64_t i = 0; i < n_rows; ++i) {
    int64_t b = rowptr[i], e = rowptr[i + 1];
    int64_t maxd = 0;
    for (int64_t j = b + 1; j < e; ++j) {
      int64_t d = (int64_t)colind[j] - (int64_t)colind[j - 1];
      if (d > maxd) maxd = d;
    }
    bytes8 += (maxd <= 255 ? 1 : 4) * (e - b);
    bytes16 += (maxd <= 65535 ? 2 : 4) * (e - b);
  }
  return bytes8 < bytes16 ? 8 : 16;
}

/* ---------------------------------------------------------------------------------- */
/* Merge-path coordinates (IMB optimization, Section III-E: spread the nonzeros evenly
 * over the workers and let long rows be shared). The work of a CSR SpMV is the merged
 * sequence of the N row-end events (row i ends at rowptr[i+1]) and the NNZ nonzeros
 * 0..NNZ-1, where nonzero j comes before the end of row i exactly when j < rowptr[i+1].
 * Walking that sequence item by item, coord[2t], coord[2t+1] record (rows ended,
 * nonzeros consumed) after t * items_per_tile items, for t = 0..n_tiles; the last entry
 * is (N, NNZ).                                                                           */
void oracle_merge_path(int64_t n_rows, int64_t nnz, const int32_t *rowptr,
                       int64_t items_per_tile, int32_t *coord) {
  int64_t total = n_rows + nnz;
  int64_t n_tiles = (total + items_per_tile - 1) / items_per_tile;
  int64_t a = 0, b = 0, t = 0;
  coord[0] = 0;
  coord[1] = 0;
  for (int64_t d = 1; d <= total; ++d) {
    if (a < n_rows && !(b < nnz && b < (int64_t)rowptr[a + 1])) {
      ++a;        /* the end of row a comes next */
    } else {
      ++b;        /* nonzero b comes next        */
    }
    if (d % items_per_tile == 0 || d == total) {
      ++t;
      coord[2 * t] = (int32_t)a;
      coord[2 * t + 1] = (int32_t)b;
    }
  }
  (void)n_tiles;
}

/* ---------------------------------------------------------------------------------- */
/* Table I features (Section III-D). Per row i:
 *   nnz_i        number of nonzeros;
 *   bw_i         column distance between first and last nonzero, read as the inclusive
 *                span last - first + 1 (so that a one-element row has bw = 1 and
 *                scatter = 1); 0 for an empty row;
 *   scatter_i    nnz_i / bw_i (0 for an empty row);
 *   clustering_i ngroups_i / nnz_i, a group being a maximal run of consecutive columns
 *                (0 for an empty row);
 *   misses_i     elements whose distance from the previous element of the row exceeds
 *                the number of x elements in a cache line; a row's first element counts.
 * The two ratio features are kept as fixed-point numbers q_i = round(2^24 * ratio), the
 * rational rounded half up; their mean and deviation are taken over the q_i and scaled
 * back by 2^-24. Means are sum / N; deviations are population deviations (divide by N),
 * evaluated from exact 128-bit integer moments: sd = sqrt((N sum f^2 - (sum f)^2) / N^2).
 *
 * out[0..13] = size, density, nnz_min, nnz_max, nnz_avg, nnz_sd, bw_min, bw_max, bw_avg,
 *              bw_sd, scatter_avg, scatter_sd, clustering_avg, misses_avg
 * size is 1 when ws_bytes <= llc_bytes. density = NNZ / (n_rows * n_cols).
 * isum[0..11] (exact sums, for bit-level comparison): sum nnz, sum bw, sum q_scatter,
 * sum q_clustering, sum misses, sum ngroups, nnz_min, nnz_max, bw_min, bw_max,
 * and the low 64 bits of sum nnz^2 and sum bw^2.                                          */
static double finalize_sd(u128 s1, u128 s2, int64_t n, double scale) {
  u128 nn = (u128)(uint64_t)n;
  u128 num = nn * s2 - s1 * s1;
  double var = (double)num / ((double)n * (double)n);
  return sqrt(var) * scale;
}

static uint64_t ratio_q24(uint64_t num, uint64_t den) {
  /* round(num * 2^24 / den), halves rounded up, in exact integer arithmetic */
  return (uint64_t)((((u128)num << 25) + den) / ((u128)den * 2));
}

void oracle_features(int64_t n_rows, int64_t n_cols, const int32_t *rowptr,
                     const int32_t *colind, int64_t line_elems, int64_t ws_bytes,
                     int64_t llc_bytes, double *out, uint64_t *isum) {
  int64_t nnz = rowptr[n_rows];
  u128 s_nnz = 0, s_nnz2 = 0, s_bw = 0, s_bw2 = 0, s_sc = 0, s_sc2 = 0, s_cl = 0;
  uint64_t s_miss = 0, s_grp = 0;
  int64_t nnz_min = INT64_MAX, nnz_max = 0, bw_min = INT64_MAX, bw_max = 0;
  for (int64_t i = 0; i < n_rows; ++i) {
    int64_t b = rowptr[i], e = rowptr[i + 1];
    int64_t k = e - b;
    int64_t bw = 0, groups = 0, misses = 0;
    if (k > 0) {
      bw = (int64_t)colind[e - 1] - (int64_t)colind[b] + 1;
      for (int64_t j = b; j < e; ++j) {
        if (j == b) {
          groups += 1;
          misses += 1;
        } else {
          int64_t d = (int64_t)colind[j] - (int64_t)colind[j - 1];
          if (d != 1) groups += 1;
          if (d > line_elems) misses += 1;
        }
      }
    }
    uint64_t q_sc = k > 0 ? ratio_q24((uint64_t)k, (uint64_t)bw) : 0;
    uint64_t q_cl = k > 0 ? ratio_q24((uint64_t)groups, (uint64_t)k) : 0;
    s_nnz += (u128)k;
    s_nnz2 += (u128)k * (u128)k;
    s_bw += (u128)bw;
    s_bw2 += (u128)bw * (u128)bw;
    s_sc += q_sc;
    s_sc2 += (u128)q_sc * (u128)q_sc;
    s_cl += q_cl;
    s_miss += (uint64_t)misses;
    s_grp += (uint64_t)groups;
    if (k < nnz_min) nnz_min = k;
    if (k > nnz_max) nnz_max = k;
    if (bw < bw_min) bw_min = bw;
    if (bw > bw_max) bw_max = bw;
  }
  if (n_rows == 0) {
    nnz_min = nnz_max = bw_min = bw_max = 0;
  }
  const double N = (double)n_rows;
  const double q = 1.0 / 16777216.0; /* 2^-24 */
  out[0] = ws_bytes <= llc_bytes ? 1.0 : 0.0;
  out[1] = n_rows > 0 && n_cols > 0 ? (double)nnz / ((double)n_rows * (double)n_cols) : 0.0;
  out[2] = (double)nnz_min;
  out[3] = (double)nnz_max;
  out[4] = n_rows ? (double)s_nnz / N : 0.0;
  out[5] = n_rows ? finalize_sd(s_nnz, s_nnz2, n_rows, 1.0) : 0.0;
  out[6] = (double)bw_min;
  out[7] = (double)bw_max;
  out[8] = n_rows ? (double)s_bw / N : 0.0;
  out[9] = n_rows ? finalize_sd(s_bw, s_bw2, n_rows, 1.0) : 0.0;
  out[10] = n_rows ? ((double)s_sc / N) * q : 0.0;
  out[11] = n_rows ? finalize_sd(s_sc, s_sc2, n_rows, q) : 0.0;
  out[12] = n_rows ? ((double)s_cl / N) * q : 0.0;
  out[13] = n_rows ? (double)s_miss / N : 0.0;
  if (isum) {
    isum[0] = (uint64_t)s_nnz;
    isum[1] = (uint64_t)s_bw;
    isum[2] = (uint64_t)s_sc;
    isum[3] = (uint64_t)s_cl;
    isum[4] = s_miss;
    isum[5] = s_grp;
    isum[6] = (uint64_t)nnz_min;
    isum[7] = (uint64_t)nnz_max;
    isum[8] = (uint64_t)bw_min;
    isum[9] = (uint64_t)bw_max;
    isum[10] = (uint64_t)s_nnz2;
    isum[11] = (uint64_t)s_bw2;
  }
}

/* ---------------------------------------------------------------------------------- */
/* Section III-B bounds, in GFLOP/s with bandwidth in GB/s (1 GB = 1e9 bytes):
 *   P_MB   = 2 NNZ / ((S_format + S_x + S_y) / B_max),
 *   P_peak = 2 NNZ / ((S_values + S_x + S_y) / B_max),
 * with S_format = 4 (N + 1) + (idx_bytes + val_bytes) NNZ for CSR (int32 row pointers),
 * S_values = val_bytes NNZ, S_x = S_y = vec_bytes N. out[0] = P_MB, out[1] = P_peak,
 * out[2] = S_format + S_x + S_y (the working set, in bytes).                             */
void oracle_bounds(int64_t n_rows, int64_t n_cols, int64_t nnz, int64_t idx_bytes,
                   int64_t val_bytes, int64_t vec_bytes, double b_max_gbs, double *out) {
  double s_format = 4.0 * (double)(n_rows + 1) + (double)(idx_bytes + val_bytes) * (double)nnz;
  double s_xy = (double)vec_bytes * (double)n_cols + (double)vec_bytes * (double)n_rows;
  double s_values = (double)val_bytes * (double)nnz;
  double flops = 2.0 * (double)nnz;
  out[0] = flops / ((s_format + s_xy) / b_max_gbs);
  out[1] = flops / ((s_values + s_xy) / b_max_gbs);
  out[2] = s_format + s_xy;
}

/* B_max is raised for working sets that fit the cache hierarchy (Section III-B footnote):
 * the cache-resident bandwidth applies when the working set is at most the LLC size.   */
double oracle_select_bmax(int64_t ws_bytes, int64_t llc_bytes, double b_main, double b_llc) {
  return ws_bytes <= llc_bytes ? b_llc : b_main;
}

/* ---------------------------------------------------------------------------------- */
/* Classify (Section III-C, Fig. 3). Class bits: MB = 1, ML = 2, IMB = 4, CMP = 8.
 * The paper leaves "P_CSR is close to P_MB" without a tolerance; it is read as
 * P_CSR / P_MB >= t_mb.                                                                  */
uint32_t oracle_classify(const double *p /* csr, mb, ml, imb, cmp, peak */, double t_imb,
                         double t_ml, double t_mb) {
  double p_csr = p[0], p_mb = p[1], p_ml = p[2], p_imb = p[3], p_cmp = p[4], p_peak = p[5];
  uint32_t cls = 0;
  if (p_imb / p_csr > t_imb) cls |= 4u;
  if (p_ml / p_csr > t_ml) cls |= 2u;
  if (p_csr / p_mb >= t_mb && p_mb < p_cmp && p_cmp < p_peak) cls |= 1u;
  if (p_mb > p_cmp || p_cmp > p_peak) cls |= 8u;
  return cls;
}

/* Second profiling pass, a GB300 reading of Section III-C: a compute-bound
 * baseline (CMP) hides the memory bottlenecks, so after the CMP optimization the profile is
 * repeated with the optimized kernel as the baseline, p2 = (P_CSR', P_ML'): ML joins the
 * class set when P_ML' / P_CSR' > t_ml and MB when P_CSR' / P_MB >= t_mb. Without p2, or
 * when pass one found no CMP, the result is Fig. 3's.                                   */
uint32_t oracle_classify2(const double *p, const double *p2, double t_imb, double t_ml,
                          double t_mb) {
  uint32_t cls = oracle_classify(p, t_imb, t_ml, t_mb);
  if (p2 != NULL && (cls & 8u) && p2[0] > 0.0) {
    if (p2[1] / p2[0] > t_ml) cls |= 2u;
    if (p2[0] / p[1] >= t_mb) cls |= 1u;
  }
  return cls;
}

/* Table II: class -> optimization, applied jointly when several classes are detected.
 * Knobs returned in out[0..3]:
 *   out[0] partition: 0 = one sub-warp per row (rows dealt to CTAs by the hardware
 *          scheduler, the GPU's counterpart of a runtime-chosen loop schedule),
 *          1 = merge-path tiles with long rows split across tiles (matrix decomposition);
 *   out[1] column index: 0 = int32, 1 = 16-bit deltas (MB);
 *   out[2] x path: 0 = default, 1 = x kept resident in L2 and gathered through the
 *          read-only path (ML; the counterpart of software prefetching of x);
 *   out[3] vector loads and unrolling: 1 for MB (delta encoding + vectorization) and CMP
 *          (unrolling + vectorization).
 * IMB picks between its two sub-optimizations with nnz_max versus nnz_avg: highly uneven
 * row lengths (nnz_max > long_ratio * nnz_avg) take the decomposition (out[0] = 1; the
 * library's autotuner then runs it as merge-path tiles or as row bins), otherwise the
 * dynamic schedule (sub-warp rows). MB sets the 16-bit delta index in every case: the
 * optimizations of Table II apply jointly, and the row-bin decomposition decodes deltas
 * (merge-path tiles keep int32 columns).                                                */
void oracle_variant_for_classes(uint32_t cls, double nnz_avg, double nnz_max,
                                double long_ratio, int32_t *out) {
  int32_t part = 0, idx = 0, xp = 0, vec = 0;
  if ((cls & 4u) && nnz_max > long_ratio * nnz_avg) part = 1;
  if (cls & 1u) idx = 1;   /* the delta index composes with the row decomposition */
  if (cls & 2u) xp = 1;
  if (cls & (1u | 8u)) vec = 1;
  out[0] = part;
  out[1] = idx;
  out[2] = xp;
  out[3] = vec;
}

/* Section IV-D: N_iters,min = t_pre / (t_base - t_opt); returns +inf when the optimized
 * kernel is not faster.                                                                  */
double oracle_amortization_iters(double t_pre, double t_base, double t_opt) {
  if (t_base <= t_opt) return INFINITY;
  return t_pre / (t_base - t_opt);
}

/* ---------------------------------------------------------------------------------- */
/* MLP selector. Layers sizes[0] -> sizes[1] -> sizes[2] -> sizes[3], ReLU after the two
 * hidden layers, one sigmoid output per bottleneck class, binary cross-entropy averaged
 * over batch and outputs. Parameters are packed W1 (sizes[1] x sizes[0], row-major), b1,
 * W2, b2, W3, b3.                                                                        */
static int64_t mlp_nparams(const int32_t *s) {
  return (int64_t)s[1] * s[0] + s[1] + (int64_t)s[2] * s[1] + s[2] + (int64_t)s[3] * s[2] +
         s[3];
}

int64_t oracle_mlp_nparams(const int32_t *sizes) { return mlp_nparams(sizes); }

/* FP64 loss; when grad is non-null also the gradient of the loss (backpropagation). */
double oracle_mlp_loss_grad_f64(const int32_t *sizes, const double *params, int64_t batch,
                                const double *X, const double *Y, double *grad,
                                double *probs) {
  int n0 = sizes[0], n1 = sizes[1], n2 = sizes[2], n3 = sizes[3];
  const double *W1 = params, *b1 = W1 + (int64_t)n1 * n0, *W2 = b1 + n1,
               *b2 = W2 + (int64_t)n2 * n1, *W3 = b2 + n2, *b3 = W3 + (int64_t)n3 * n2;
  double *h1 = (double *)malloc(sizeof(double) * (size_t)n1);
  double *h2 = (double *)malloc(sizeof(double) * (size_t)n2);
  double *g1 = (double *)malloc(sizeof(double) * (size_t)n1);
  double *g2 = (double *)malloc(sizeof(double) * (size_t)n2);
  double *g3 = (double *)malloc(sizeof(double) * (size_t)n3);
  int64_t np = mlp_nparams(sizes);
  if (grad) memset(grad, 0, sizeof(double) * (size_t)np);
  double *dW1 = grad, *db1 = grad ? dW1 + (int64_t)n1 * n0 : 0,
         *dW2 = grad ? db1 + n1 : 0, *db2 = grad ? dW2 + (int64_t)n2 * n1 : 0,
         *dW3 = grad ? db2 + n2 : 0, *db3 = grad ? dW3 + (int64_t)n3 * n2 : 0;
  double loss = 0.0;
  double inv = 1.0 / ((double)batch * (double)n3);
  for (int64_t b = 0; b < batch; ++b) {
    const double *x = X + b * n0;
    const double *y = Y + b * n3;
    for (int i = 0; i < n1; ++i) {
      double a = b1[i];
      for (int k = 0; k < n0; ++k) a += W1[(int64_t)i * n0 + k] * x[k];
      h1[i] = a > 0.0 ? a : 0.0;
    }
    for (int i = 0; i < n2; ++i) {
      double a = b2[i];
      for (int k = 0; k < n1; ++k) a += W2[(int64_t)i * n1 + k] * h1[k];
      h2[i] = a > 0.0 ? a : 0.0;
    }
    for (int i = 0; i < n3; ++i) {
      double z = b3[i];
      for (int k = 0; k < n2; ++k) z += W3[(int64_t)i * n2 + k] * h2[k];
      double p = 1.0 / (1.0 + exp(-z));
      if (probs) probs[b * n3 + i] = p;
      /* -[y log p + (1 - y) log(1 - p)] written stably in terms of z */
      loss += (z > 0.0 ? z : 0.0) - y[i] * z + log1p(exp(-fabs(z)));
      g3[i] = (p - y[i]) * inv;
    }
    if (!grad) continue;
    for (int i = 0; i < n3; ++i) {
      db3[i] += g3[i];
      for (int k = 0; k < n2; ++k) dW3[(int64_t)i * n2 + k] += g3[i] * h2[k];
    }
    for (int k = 0; k < n2; ++k) {
      double a = 0.0;
      for (int i = 0; i < n3; ++i) a += W3[(int64_t)i * n2 + k] * g3[i];
      g2[k] = h2[k] > 0.0 ? a : 0.0;
    }
    for (int i = 0; i < n2; ++i) {
      db2[i] += g2[i];
      for (int k = 0; k < n1; ++k) dW2[(int64_t)i * n1 + k] += g2[i] * h1[k];
    }
    for (int k = 0; k < n1; ++k) {
      double a = 0.0;
      for (int i = 0; i < n2; ++i) a += W2[(int64_t)i * n1 + k] * g2[i];
      g1[k] = h1[k] > 0.0 ? a : 0.0;
    }
    for (int i = 0; i < n1; ++i) {
      db1[i] += g1[i];
      for (int k = 0; k < n0; ++k) dW1[(int64_t)i * n0 + k] += g1[i] * x[k];
    }
  }
  free(h1);
  free(h2);
  free(g1);
  free(g2);
  free(g3);
  return loss * inv;
}

/* FP32 inference with the exact operation order the selector decision is defined by:
 * each unit starts from its bias and adds w_k * in_k for k = 0, 1, ... with one fused
 * multiply-add per term; ReLU on hidden units; the outputs are the class logits.         */
void oracle_mlp_logits_f32(const int32_t *sizes, const float *params, int64_t batch,
                           const float *X, float *logits) {
  int n0 = sizes[0], n1 = sizes[1], n2 = sizes[2], n3 = sizes[3];
  const float *W1 = params, *b1 = W1 + (int64_t)n1 * n0, *W2 = b1 + n1,
              *b2 = W2 + (int64_t)n2 * n1, *W3 = b2 + n2, *b3 = W3 + (int64_t)n3 * n2;
  float h1[1024], h2[1024];
  if (n1 > 1024 || n2 > 1024) return;
  for (int64_t b = 0; b < batch; ++b) {
    const float *x = X + b * n0;
    for (int i = 0; i < n1; ++i) {
      float a = b1[i];
      for (int k = 0; k < n0; ++k) a = fmaf(W1[(int64_t)i * n0 + k], x[k], a);
      h1[i] = a > 0.0f ? a : 0.0f;
    }
    for (int i = 0; i < n2; ++i) {
      float a = b2[i];
      for (int k = 0; k < n1; ++k) a = fmaf(W2[(int64_t)i * n1 + k], h1[k], a);
      h2[i] = a > 0.0f ? a : 0.0f;
    }
    for (int i = 0; i < n3; ++i) {
      float a = b3[i];
      for (int k = 0; k < n2; ++k) a = fmaf(W3[(int64_t)i * n2 + k], h2[k], a);
      logits[b * n3 + i] = a;
    }
  }
}

/* log2(1 + v) for v >= 0 in FP32, used to compress the heavy-tailed features before the
 * MLP. w = 1 + v = m 2^e with m in [sqrt(2)/2, sqrt(2)) taken from the bits of w, then
 * log2(m) = (2 / ln 2) atanh(t), t = (m - 1) / (m + 1), |t| < 0.1716, with the atanh
 * Taylor series t + t^3/3 + ... + t^11/11 evaluated by Horner's rule in t^2 using fmaf.
 * Inputs below 0 or NaN return 0.                                                         */
float oracle_log2p1_f32(float v) {
  if (!(v > 0.0f)) return 0.0f;
  float w = 1.0f + v;
  uint32_t u;
  memcpy(&u, &w, sizeof u);
  int e = (int)((u >> 23) & 0xFFu) - 127;
  uint32_t mb = (u & 0x007FFFFFu) | 0x3F800000u;
  float m;
  memcpy(&m, &mb, sizeof m);
  if (m > 1.41421356f) {
    m = m * 0.5f;
    e += 1;
  }
  float t = (m - 1.0f) / (m + 1.0f);
  float t2 = t * t;
  float p = 1.0f / 11.0f;
  p = fmaf(p, t2, 1.0f / 9.0f);
  p = fmaf(p, t2, 1.0f / 7.0f);
  p = fmaf(p, t2, 1.0f / 5.0f);
  p = fmaf(p, t2, 1.0f / 3.0f);
  p = fmaf(p, t2, 1.0f);
  float l = (t * p) * 2.88539008f; /* 2 / ln 2 */
  return (float)e + l;
}

void oracle_log2p1_f32_array(const float *in, float *out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) out[i] = oracle_log2p1_f32(in[i]);
}

/* ---------------------------------------------------------------------------------- */
/* Feature route (Section III-D). The paper trains a decision tree on Table I features;
 * the route is read here as fixed rules over the same features:
 *   IMB  highly uneven rows, nnz_max > long_ratio * nnz_avg (the IMB sub-class test of
 *        Section III-E);
 *   ML   most elements open a new cache line (misses_avg >= nnz_avg / 2) and x does not
 *        fit in half of the last-level cache (vec_bytes * n_cols > llc_bytes / 2);
 *   CMP  the working set fits the cache (size = 1) or rows are very short (nnz_avg < 4);
 *   MB   none of the above while the working set exceeds the cache.
 * f[] is the 14-feature vector of oracle_features.                                       */
uint32_t oracle_feature_rules(const double *f, int64_t n_cols, int64_t vec_bytes,
                              int64_t llc_bytes, double long_ratio) {
  double size = f[0], nnz_max = f[3], nnz_avg = f[4], misses_avg = f[13];
  uint32_t cls = 0;
  if (nnz_avg > 0.0 && nnz_max > long_ratio * nnz_avg) cls |= 4u;
  if (misses_avg >= 0.5 * nnz_avg && (double)vec_bytes * (double)n_cols > 0.5 * (double)llc_bytes)
    cls |= 2u;
  if (size != 0.0 || nnz_avg < 4.0) cls |= 8u;
  if (cls == 0 && size == 0.0) cls |= 1u;
  return cls;
}

/* Inputs of the MLP selector, from the 14 features f[0..13] plus n_rows (f[14]) and nnz
 * (f[15]): twelve numbers, each a feature, a ratio of two features (0 when the
 * denominator is 0), or log2(1 + that) for the heavy-tailed ones, converted to FP32:
 *   log2p1(n_rows), log2p1(nnz_avg), log2p1(nnz_sd / nnz_avg), log2p1(nnz_max),
 *   log2p1(nnz_max / nnz_avg), log2p1(bw_avg), log2p1(bw_sd), scatter_avg, scatter_sd,
 *   clustering_avg, misses_avg / nnz_avg, size.
 * With mu and inv_sigma (non-null) every input becomes (v - mu_k) * inv_sigma_k in FP32.  */
static double ratio_or_zero(double a, double b) { return b > 0.0 ? a / b : 0.0; }

void oracle_mlp_inputs(const double *feat, int64_t batch, const float *mu,
                       const float *inv_sigma, float *X) {
  for (int64_t b = 0; b < batch; ++b) {
    const double *f = feat + b * 16;
    float r[12];
    r[0] = oracle_log2p1_f32((float)f[14]);
    r[1] = oracle_log2p1_f32((float)f[4]);
    r[2] = oracle_log2p1_f32((float)ratio_or_zero(f[5], f[4]));
    r[3] = oracle_log2p1_f32((float)f[3]);
    r[4] = oracle_log2p1_f32((float)ratio_or_zero(f[3], f[4]));
    r[5] = oracle_log2p1_f32((float)f[8]);
    r[6] = oracle_log2p1_f32((float)f[9]);
    r[7] = (float)f[10];
    r[8] = (float)f[11];
    r[9] = (float)f[12];
    r[10] = (float)ratio_or_zero(f[13], f[4]);
    r[11] = (float)f[0];
    for (int k = 0; k < 12; ++k) {
      float z = r[k];
      if (mu) z = (z - mu[k]) * inv_sigma[k];
      X[b * 12 + k] = z;
    }
  }
}

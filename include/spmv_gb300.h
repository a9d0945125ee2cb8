/*
 * spmv_gb300.h -- C ABI of a GB300 (sm_103a) bottleneck-adaptive CSR SpMV library.
 *
 * The library implements the method of Elafrou, Goumas and Koziris, "Performance Analysis
 * and Optimization of Sparse Matrix-Vector Multiplication on Modern Multi- and Many-Core
 * Processors" (arXiv 1711.05487): y = A x for a CSR matrix (Section II, Fig. 1), a
 * classifier that finds the matrix's SpMV bottleneck classes -- memory bandwidth (MB),
 * memory latency (ML), thread imbalance (IMB), computation (CMP) -- by profiling
 * (Section III-B/C, Fig. 3) or from matrix features (Section III-D, Table I), and a pool of
 * low-preprocessing CSR optimizations applied jointly per detected class (Section III-E,
 * Table II). A learned selector (a small MLP trained on the GPU) stands in for the paper's
 * decision tree.
 *
 * Conventions for every entry point:
 *   - Plain C types only. A stream argument is a cudaStream_t passed as void*; NULL is the
 *     legacy default stream. A "device pointer" is CUDA global memory of the current device.
 *   - Every call returns spmv_status and never throws or aborts. On error nothing is
 *     written to the caller's outputs unless stated.
 *   - Index arrays are int32 (n_rows, n_cols, nnz < 2^31). CSR columns must be sorted and
 *     unique within each row.
 *   - Calls are not thread-safe on the same handle; different handles are independent.
 */
#ifndef SPMV_GB300_H
#define SPMV_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spmv_matrix *spmv_handle_t;
typedef struct spmv_batch *spmv_batch_t;
typedef struct spmv_selector *spmv_selector_t;
typedef void *spmv_stream_t; /* cudaStream_t */

typedef enum {
  SPMV_OK = 0,
  SPMV_ERR_INVALID_CSR = 1,       /* rowptr/colind violate the CSR definition           */
  SPMV_ERR_UNSUPPORTED_DTYPE = 2, /* dtype combination not offered                      */
  SPMV_ERR_OOM = 3,               /* device allocation failed                           */
  SPMV_ERR_NOT_TUNED = 4,         /* spmv_run before spmv_tune / spmv_set_variant        */
  SPMV_ERR_CUDA = 5,              /* a CUDA runtime call failed                         */
  SPMV_ERR_TIMEOUT = 6,           /* a bounded device-side wait gave up                 */
  SPMV_ERR_ARG = 7,               /* invalid argument (null pointer, size, k ...)       */
  SPMV_ERR_NO_SELECTOR = 8,       /* learned mode without a selector                    */
  SPMV_ERR_TOO_LARGE = 9          /* problem larger than a fixed-size buffer allows     */
} spmv_status;

/* SPMV_DF64 ("double-float") carries an FP64 number as the unevaluated sum hi + lo of two
 * FP32 numbers: hi = the top 24 significant bits, lo = the next 23 (both truncated), so
 * |v - hi - lo| < 2^-46 |v|; zero splits to (+-0, 0), and a nonzero outside [2^-40, 2^41),
 * an infinity or a NaN to (NaN, 0). As a storage / accumulation type it runs FP64 SpMV on
 * the FP32 pipe (see spmv_set_precision); it is not an input type of spmv_create. */
typedef enum { SPMV_F64 = 0, SPMV_F32 = 1, SPMV_BF16 = 2, SPMV_DF64 = 3 } spmv_dtype;

typedef enum {
  SPMV_TUNE_PROFILE = 0,  /* Section III-C: micro-benchmarks + Fig. 3 rules            */
  SPMV_TUNE_FEATURES = 1, /* Section III-D: Table I features + fixed rules              */
  SPMV_TUNE_LEARNED = 2,  /* features + MLP selector, profiling as fallback             */
  SPMV_TUNE_FIXED = 3     /* use opts->fixed                                            */
} spmv_mode;

/* Bottleneck classes (Section III-A); a class set is a bitmask, 0 = not worth optimizing. */
enum { SPMV_CLASS_MB = 1, SPMV_CLASS_ML = 2, SPMV_CLASS_IMB = 4, SPMV_CLASS_CMP = 8 };

/* One point of the optimization pool (Table II, applied jointly). */
typedef struct {
  int32_t partition; /* 0: one sub-warp per row, rows handed to CTAs by the hardware
                        scheduler; 1: merge-path tiles, long rows split across tiles;
                        2: row decomposition (A = A_short + A_long, Fig. 5): rows under
                        bin_med nonzeros on sub-warps of vs lanes (1, 2, 4 or 8), rows under
                        bin_chunk on one warp each, longer rows in bin_chunk-nonzero
                        chunks summed in FP64 in chunk order. 1 and 2 are the decompositions of
                        Section III-E (IMB); the autotuner picks between them;
                        3: sliced rows (SELL-32, a GB300 layout for short rows; see
                        spmv_get_sell): one thread per row over 32-row slices stored
                        column-major, coalesced loads without a shared-memory stage, int32
                        columns or (index 1) the delta index's deltas; vs is 1          */
  int32_t index;     /* 0: int32 columns; 1: 8- or 16-bit column deltas (one width per
                        matrix, see spmv_get_delta) with escape rows (MB); merge-path
                        tiles (partition 1) always read int32 columns                     */
  int32_t xpath;     /* 0: default; 1: x kept L2-resident (evict-last gathers through the
                        read-only path, evict-first streams) (ML); P = 2..16: x cut into P
                        column panels, the SpMV run as P passes over a panel-major copy of
                        the matrix, pass p gathering only from slice p of x (ML with x
                        larger than the L2; see spmv_get_col_panels). Panels run rows on
                        sub-warps of vs = 1, 2, 4 or 8 lanes with int32 columns (partition
                        and index are set to 0); vec selects 128-bit loads               */
  int32_t vec;       /* 0: scalar loads; 1: 128-bit loads of val/colind, unrolled (MB/CMP) */
  int32_t vs;        /* sub-warp width for partition 0: 1 (thread per row over a tile
                        staged in shared memory by bulk copies), 2,4,8,16,32; 0 = heuristic */
  int32_t tile_rows; /* width 1: rows per staged tile, 32 / 64 / 128; 0 = automatic       */
  int32_t tile_pipe; /* width 1: 0 = one tile per CTA, 1 = persistent CTAs keeping the next
                        tile's bulk copy in flight (two shared-memory stages)               */
  int32_t bin_med;   /* partition 2: rows under bin_med nonzeros go to sub-warps; 0 = 64   */
  int32_t bin_chunk; /* partition 2: rows under bin_chunk nonzeros take one warp, longer
                        rows are cut into bin_chunk-nonzero chunks; 0 = 4096. Needs
                        2 <= bin_med <= bin_chunk <= 2^20. Neither limit is in the paper;
                        the grid search of Section III-C tunes them with the thresholds  */
} spmv_variant;

#define SPMV_NUM_FEATURES 14
/* Feature order (Table I): size, density, nnz_min, nnz_max, nnz_avg, nnz_sd, bw_min,
 * bw_max, bw_avg, bw_sd, scatter_avg, scatter_sd, clustering_avg, misses_avg.          */

typedef struct {
  double t_imb;          /* Fig. 3 T_IMB, default 1.24                                   */
  double t_ml;           /* Fig. 3 T_ML, default 1.25                                    */
  double t_mb;           /* "P_CSR close to P_MB" read as P_CSR/P_MB >= t_mb, default 0.75 */
  double long_row_ratio; /* IMB sub-choice: nnz_max > ratio * nnz_avg -> decomposition (32) */
  int32_t autotune;      /* 1: pick the sub-warp width by timing (default 1)             */
  int32_t reps;          /* timed repetitions per probe (default 8; the autotuner half) */
  spmv_variant fixed;    /* SPMV_TUNE_FIXED only                                         */
  spmv_selector_t selector; /* SPMV_TUNE_LEARNED only                                    */
  double min_margin;     /* learned: smallest |logit| accepted, else profile (default 0); a
                            matrix outside the selector's training range (margin -1) always
                            falls back to profiling                                       */
  int32_t second_pass;   /* profile: re-profile after the CMP optimization (default 1)   */
  int32_t bin_med;       /* row decomposition limits of a tuned IMB variant (see          */
  int32_t bin_chunk;     /* spmv_variant); 0 = the defaults 64 and 4096                    */
} spmv_tune_opts;

typedef struct {
  uint32_t classes;      /* detected class set                                           */
  int32_t mode_used;     /* route that decided (LEARNED may fall back to PROFILE)        */
  spmv_variant variant;  /* variant installed on the handle                              */
  double p[6];           /* P_CSR, P_MB, P_ML, P_IMB, P_CMP, P_peak in GFLOP/s (profile) */
  double p2[2];          /* second pass: P_CSR', P_ML' of the CMP-optimized kernel (0 if none) */
  double b_max_gbs;      /* bandwidth used for P_MB / P_peak                             */
  double features[SPMV_NUM_FEATURES];
  double margin;         /* learned: smallest |logit| of the MLP decision                */
  double t_pre_ms;       /* whole spmv_tune wall time                                    */
  double t_classify_ms;  /* probes or features (+ inference)                             */
  double t_prep_ms;      /* format conversion / partitioning                             */
  double t_autotune_ms;  /* sub-warp width and tile geometry sweep                       */
} spmv_tune_report;

/* ---------------------------------------------------------------- matrix handles ---- */

/* Largest nonzero count a handle accepts: 2^31 - 2^21 - 1 (see spmv_create). */
#define SPMV_MAX_NNZ 2145386495LL

/* Fills opts with the defaults listed above. */
spmv_status spmv_tune_opts_default(spmv_tune_opts *opts);

/* Section II (CSR): copies the matrix into library-owned device memory and validates it
 * on the device. row_ptr[n_rows + 1], col_ind[nnz], val[nnz] in dtype val_type are host
 * pointers (device_ptrs = 0) or device pointers (device_ptrs = 1); the caller keeps
 * ownership and may free them when the call returns. Storage, x/y and accumulation
 * dtypes start as val_type / F64 / F64 (F32 / F32 / F32 for F32 and BF16 input).
 * Sizes: n_rows and n_cols below 2^31 - 1, nnz at most SPMV_MAX_NNZ = 2^31 - 2^21 - 1
 * (offsets are int32, and the kernels step through a row's nonzeros in strides of up to
 * 2^20, the longest row-decomposition chunk, which must not pass 2^31 - 1).
 * Errors: SPMV_ERR_ARG (null out or arrays, negative or oversized sizes),
 * SPMV_ERR_INVALID_CSR, SPMV_ERR_OOM, SPMV_ERR_CUDA. The call synchronizes the stream. */
spmv_status spmv_create(spmv_handle_t *out, int64_t n_rows, int64_t n_cols, int64_t nnz,
                        const int32_t *row_ptr, const int32_t *col_ind, const void *val,
                        spmv_dtype val_type, int32_t device_ptrs, spmv_stream_t stream);

/* Frees every device buffer of the handle (synchronizes the device first). */
spmv_status spmv_destroy(spmv_handle_t h);

/* Value storage precision (not in the paper): storage in F64 / F32 / BF16, x and y in
 * vec_type (F64 or F32), products accumulated in acc_type (F64, F32 or DF64). Conversion is
 * round-to-nearest-even straight from the input values. Offered: storage F64 with
 * vec = acc = F64; storage F32 or BF16 with (vec, acc) in {(F64,F64),(F32,F32),(F32,F64),
 * (F64,DF64),(F32,DF64)}; storage DF64 with vec = F64, acc = DF64 (FP64 input values only).
 * acc = F32 keeps every FP32 running sum within the FP32-storage bound (2e-6 of
 * sum_j |a_ij x_j| against the FP64 values): a thread sums at most 30 products of a row in
 * FP32 alone, and a longer chain (a long row, or a lane's share of one) is summed in runs of
 * 16 FP32 products whose sums, and the lanes' reduction, are added in FP64.
 * acc = DF64 with F32 / BF16 storage: width-1 row variants sum each row in double-float
 * arithmetic on the FP32 pipe (a stored value and an FP32 x element are exact in the high
 * part), within about 8e-13 of sum_j |a_ij x_j| against the stored values, the FP64 bound;
 * other variants accumulate in FP64.
 * DF64 (a GB300 answer to the CMP class, not in the paper): GB300's FP64 pipe is about 1/64
 * of its FP32 pipe, so width-1 row variants (vs = 1) compute each product and the row sum
 * in double-float FP32 arithmetic from value pairs split once here and x elements split as
 * they are gathered: each row ends within about 8e-13 of sum_j |a_ij x_j| (inside the FP64
 * bound of 1e-12), not bit-identical to FP64 FMAs. Rows longer than 32 nonzeros, or meeting
 * a value or x element that does not split (see SPMV_DF64), are recomputed with FP64 FMAs;
 * every other variant runs the FP64 kernels on the FP64 values. Width-1 variants run one
 * tile per CTA (tile_pipe is set to 0). The handle keeps the pairs (8 bytes per nonzero)
 * beside the FP64 values.
 * Invalidates the tuned variant (spmv_tune or spmv_set_variant must follow). On failure
 * (SPMV_ERR_OOM, CUDA) the handle is back at the input dtype's defaults and untuned. */
spmv_status spmv_set_precision(spmv_handle_t h, spmv_dtype storage, spmv_dtype vec_type,
                               spmv_dtype acc_type, spmv_stream_t stream);

/* Section III: classify the matrix with the given route, map classes to optimizations
 * (Table II), build the variant's data (delta index, merge-path table) and, if
 * opts->autotune, pick the sub-warp width by timing. opts and report may be NULL
 * (defaults / no report). Synchronizes the stream (the profile route times kernels).
 * Errors: SPMV_ERR_NO_SELECTOR (learned without opts->selector), SPMV_ERR_OOM, CUDA; an
 * error met after argument checks leaves the handle untuned (runs answer
 * SPMV_ERR_NOT_TUNED until a tune or spmv_set_variant succeeds). */
spmv_status spmv_tune(spmv_handle_t h, spmv_mode mode, const spmv_tune_opts *opts,
                      spmv_tune_report *report, spmv_stream_t stream);

/* Installs a variant directly (same preprocessing as spmv_tune, no classification).
 * Errors: SPMV_ERR_ARG (invalid variant; the installed one stays), SPMV_ERR_OOM, CUDA
 * (the handle is left untuned). */
spmv_status spmv_set_variant(spmv_handle_t h, const spmv_variant *v, spmv_stream_t stream);

/* Fig. 1: y = A x (y overwritten), asynchronous on stream, no host synchronization.
 * x[n_cols], y[n_rows] are caller-owned device pointers in the handle's vec_type; they
 * must stay valid until the stream work completes and must not overlap.
 * Errors: SPMV_ERR_NOT_TUNED, SPMV_ERR_ARG, SPMV_ERR_CUDA (launch failure). */
spmv_status spmv_run(spmv_handle_t h, const void *x, void *y, spmv_stream_t stream);

/* y = A x with HOST buffers: copies x to a handle-owned device buffer, runs, copies y
 * back; returns when y is on the host (the end-to-end path). Row variants whose x and y
 * together reach 8 MB compute in eight row chunks: chunk c waits only for the prefix of x
 * up to the largest column of chunks 0..c (uploaded piece by piece on a handle-owned
 * stream), consecutive chunks' kernels run on two alternating handle-owned streams, and
 * each finished chunk of y is downloaded while the next computes (consecutive chunks'
 * downloads alternate between two more streams). Column
 * panels (up to 8) upload x slice by slice, each pass waiting only for its slice, and run
 * their last pass in the eight row chunks. With page-locked x and y the whole pipeline is captured
 * once into a CUDA graph (kept per handle for the last pair of host pointers until the
 * precision or variant changes) and replayed with one launch; pageable buffers take the
 * same pipeline without a graph, with slower, staged copies. Host buffers must stay valid
 * until the call returns. The first call with a new buffer pair or variant captures the
 * graph and must not run while another thread captures a stream. */
spmv_status spmv_run_host(spmv_handle_t h, const void *x_host, void *y_host,
                          spmv_stream_t stream);

/* Y = A X for k right-hand sides (SpMM), X (n_cols x k) and Y (n_rows x k) row-major
 * device arrays in vec_type. Uses the sub-warp row kernel with int32 columns whatever
 * the tuned variant; k >= 1. */
spmv_status spmv_run_spmm(spmv_handle_t h, const void *X, void *Y, int32_t k,
                          spmv_stream_t stream);

/* Copies the handle's CSR back (device pointers: row_ptr[n_rows+1], col_ind[nnz],
 * val[nnz] in the storage dtype). Columns are decoded from the 16-bit delta index when
 * that variant is installed, so this is the format round-trip check. Synchronizes. */
spmv_status spmv_export_csr(spmv_handle_t h, int32_t *row_ptr, int32_t *col_ind, void *val,
                            spmv_stream_t stream);

/* Copies the delta column index (Section III-E, MB) of the handle: base[n_rows] (a row's
 * first column, or -(1 + offset) into esc_col for an escape row, 0 for an empty row),
 * delta[nnz] of *bits (8 or 16) bits each (the first delta of a row is 0) and
 * esc_col[*n_esc] (escape rows' columns in full, in row order). The width is chosen per
 * matrix: 8 bits when that index is strictly smaller than the 16-bit one (1 or 2 bytes per
 * nonzero of the rows whose gaps fit, 4 per nonzero of escape rows), else 16 -- "8- or
 * 16-bit deltas, never both". Pass base = delta = esc_col = NULL to query *n_esc and
 * *bits. SPMV_ERR_NOT_TUNED if no delta index has been built. */
spmv_status spmv_get_delta(spmv_handle_t h, int32_t *base, void *delta, int32_t *esc_col,
                           int64_t *n_esc, int32_t *bits, spmv_stream_t stream);

/* Copies the sliced-row copy of the matrix (variant partition 3): rows in slices of 32
 * consecutive rows (the last may hold fewer); slice s is as wide as its longest row and
 * stores element k of row 32 s + l at position slice_off[s] + 32 k + l (slice_off: device,
 * int64[ceil(n_rows / 32) + 1], slice_off[0] = 0). val (device, *n_positions values of the
 * storage dtype; FP64 for SPMV_DF64 storage) and idx (device, *n_positions int32 columns when
 * *idx_bits = 0, else column deltas of *idx_bits bits, as spmv_get_delta describes them)
 * hold the slices; positions past a row's length are padding (zero). Any of the arrays may
 * be NULL; all NULL queries *n_positions and *idx_bits. SPMV_ERR_NOT_TUNED if no slices have
 * been built. */
spmv_status spmv_get_sell(spmv_handle_t h, int64_t *slice_off, void *val, void *idx,
                          int64_t *n_positions, int32_t *idx_bits, spmv_stream_t stream);

/* Copies the column-panel copy of the matrix (variant xpath = P >= 2; Section III-E, ML,
 * with x cut into P slices that each fit in the L2): panel p holds the columns
 * [p * w, (p + 1) * w), w = *panel_cols = ceil(n_cols / P) rounded up to a multiple of 32
 * (trailing panels may be empty). panel_rowptr (device, int32[P * (n_rows + 1)]) holds
 * each panel's row pointers, absolute positions into panel_col (device, int32[nnz]) and
 * panel_val (device, nnz values of the storage dtype; FP64 for SPMV_DF64 storage), which
 * list panel 0's nonzeros row by row, then panel 1's, and so on, columns in row order.
 * Any of the three arrays may be NULL; all NULL queries *n_panels and *panel_cols.
 * SPMV_ERR_NOT_TUNED if no panel copy has been built. */
spmv_status spmv_get_col_panels(spmv_handle_t h, int32_t *panel_rowptr, int32_t *panel_col,
                                void *panel_val, int32_t *n_panels, int32_t *panel_cols,
                                spmv_stream_t stream);

/* Copies the merge-path tile table (rows ended, nonzeros consumed) for tile boundaries
 * 0..n_tiles into coord (device, int32[2 * (n_tiles + 1)]); pass coord = NULL to query
 * *n_tiles and *items_per_tile. */
spmv_status spmv_get_merge_path(spmv_handle_t h, int32_t *coord, int64_t *n_tiles,
                                int64_t *items_per_tile, spmv_stream_t stream);

/* Copies the row decomposition of partition 2 (device arrays, int32): med_rows[n_med] the
 * rows of 64..4095 nonzeros, long_rows[n_long] the rows of 4096 or more, long_first
 * [n_long + 1] each long row's first chunk (the last entry is n_chunks), chunks[4 * n_chunks]
 * as (row, first nonzero z, end nonzero, start column: colind[z - 1] for a chunk that starts
 * inside its row, colind[z] for a row's first chunk -- where a 16-bit delta decode of the
 * chunk starts), all in row order. counts (host, int64[3])
 * receives n_med, n_long, n_chunks; pass med_rows = NULL to query counts only.
 * SPMV_ERR_NOT_TUNED if no decomposition has been built. */
spmv_status spmv_get_row_bins(spmv_handle_t h, int32_t *med_rows, int32_t *long_rows,
                              int32_t *long_first, int32_t *chunks, int64_t *counts,
                              spmv_stream_t stream);

/* Section III-D, Table I features computed on the device (exact integer moments, host
 * finalization); line_bytes is the cache-line size for misses_i (128 = GPU L2 line,
 * divided by the x element size). features[14] host, isum[12] host (may be NULL):
 * sum nnz, sum bw, sum q_scatter, sum q_clustering, sum misses, sum ngroups, nnz_min,
 * nnz_max, bw_min, bw_max, low 64 bits of sum nnz^2 and of sum bw^2. Synchronizes. */
spmv_status spmv_features(spmv_handle_t h, int32_t line_bytes, double *features,
                          uint64_t *isum, spmv_stream_t stream);

/* Section III-B profile of the matrix. */
typedef struct {
  double p[6];           /* P_CSR, P_MB, P_ML, P_IMB, P_CMP, P_peak (GFLOP/s)             */
  double b_max_gbs;      /* B_max used for P_MB / P_peak (HBM or L2-resident, footnote)   */
  double b_hbm_gbs;      /* measured read bandwidth, buffer much larger than L2           */
  double b_l2_gbs;       /* measured read bandwidth, L2-resident buffer                   */
  double t_csr_ms;       /* static-partition baseline, event time per launch              */
  double t_ml_ms;        /* P_ML kernel (colind'[j] = row of j), per launch               */
  double t_cmp_ms;       /* P_CMP kernel (x[i], no colind), per launch                    */
  double t_median_ms;    /* lower median over SMs of each SM's span (first start to last
                            end of its CTAs): the SM is the worker of the static partition */
  double t_span_ms;      /* last CTA end - first CTA start                                */
  double t_imb_ms;       /* t_median + launch overhead (t_csr - t_span, if positive)      */
  int32_t n_ctas;        /* resident CTAs = workers of the static partition               */
  int32_t vs;            /* sub-warp width of the profiling kernels                       */
  double p2[2];          /* second pass with the CMP-optimized kernel (thread per row over
                            shared-memory tiles) as baseline: P_CSR', and P_ML' of the same
                            kernel on colind'                                             */
} spmv_profile_report;

/* Section III-B profile: runs the static-partition baseline (P_CSR, per-CTA timers for
 * P_IMB: P_IMB = 2 NNZ / t_imb), the P_ML kernel (colind'[j] = row of j) and the P_CMP
 * kernel (x[i] only), and computes P_MB, P_peak from byte counts and the measured B_max
 * (the L2-resident bandwidth when S_format + S_x + S_y fits in L2). reps = timed launches
 * per kernel. out is a host pointer. Synchronizes. */
spmv_status spmv_profile(spmv_handle_t h, int32_t reps, spmv_profile_report *out,
                         spmv_stream_t stream);

/* One launch of the static-partition baseline with per-CTA timers: elapsed_ms[c] and
 * sm_id[c] (host arrays of at least *n_ctas entries; pass NULL to query *n_ctas). CTAs
 * whose row range is empty report elapsed 0. Synchronizes. */
spmv_status spmv_profile_cta_times(spmv_handle_t h, double *elapsed_ms, int32_t *sm_id,
                                   int32_t *n_ctas, spmv_stream_t stream);

/* Runs one profiling kernel once into y (device, vec_type): which = 0 the static-partition
 * baseline, 1 the P_ML kernel, 2 the P_CMP kernel. For tests of their construction. */
spmv_status spmv_profile_kernel(spmv_handle_t h, int32_t which, const void *x, void *y,
                                spmv_stream_t stream);

/* Sustained read bandwidth of the current device (GB/s, 1e9 B/s) for a buffer far larger
 * than L2 (hbm_gbs) and one resident in L2 (l2_gbs): the B_max of Section III-B and of its
 * footnote. Measured once per device and cached. */
spmv_status spmv_probe_bandwidth(double *hbm_gbs, double *l2_gbs);

/* Ceiling of random x gathers (not in the paper; the measured bound of an SpMV whose column
 * indices are uniform random): the time in ms (best of three runs of reps launches) of
 * `count` gathers of elem_bytes (4 or 8) elements at uniform pseudo-random positions of an
 * n_x-element array, 8 in flight per thread, no index array streamed. Allocates and frees
 * its array (n_x < 2^32). Synchronizes. Errors: SPMV_ERR_ARG, SPMV_ERR_OOM, SPMV_ERR_CUDA. */
spmv_status spmv_probe_gather(int64_t n_x, int32_t elem_bytes, int64_t count, int32_t reps,
                              double *ms, spmv_stream_t stream);

/* FMA throughput of the current device (not in the paper; the measured bound of a kernel
 * that spends one FMA per nonzero, which on GB300's narrow FP64 pipe is the native-FP64
 * SpMV's bound): fused multiply-adds per second, best of three runs of reps launches, of a
 * register-only kernel in which every thread runs `chains` independent FMA chains (1, 2, 4
 * or 8) of elem_bytes (8: FP64, 4: FP32) with warps_per_sm warps on each SM (1 to 32, or an
 * even count up to 64). Synchronizes. Errors: SPMV_ERR_ARG, SPMV_ERR_CUDA. */
spmv_status spmv_probe_fma(int32_t elem_bytes, int32_t chains, int32_t warps_per_sm,
                           int32_t reps, double *fma_per_s, spmv_stream_t stream);

/* Fig. 3 on a P-vector (csr, mb, ml, imb, cmp, peak); pure function. */
uint32_t spmv_classify(const double *p, double t_imb, double t_ml, double t_mb);

/* Fig. 3 followed by the second pass (a GB300 reading of Section III-C): when CMP is
 * detected and p2 (P_CSR', P_ML' of the CMP-optimized kernel) is given, ML is added if
 * P_ML' / P_CSR' > t_ml and MB if P_CSR' / P_MB >= t_mb. p2 may be NULL (= spmv_classify).
 * Pure function. */
uint32_t spmv_classify2(const double *p, const double *p2, double t_imb, double t_ml,
                        double t_mb);

/* Table II (jointly applied) for a class set; vs is left 0 (heuristic). Pure function. */
void spmv_variant_for_classes(uint32_t classes, double nnz_avg, double nnz_max,
                              double long_row_ratio, spmv_variant *out);

/* Section III-B closed forms: out[0] = P_MB, out[1] = P_peak (GFLOP/s, b_max in GB/s),
 * out[2] = S_format + S_x + S_y (bytes) for int32 CSR with the given element sizes. */
void spmv_bounds(int64_t n_rows, int64_t n_cols, int64_t nnz, int32_t idx_bytes,
                 int32_t val_bytes, int32_t vec_bytes, double b_max_gbs, double *out);

/* Feature route rules (Section III-D, fixed rules standing in for the trained tree) on
 * the 14 Table I features: IMB if nnz_max > long_row_ratio * nnz_avg; ML if
 * misses_avg >= nnz_avg / 2 and vec_bytes * n_cols > l2_bytes / 2; CMP if size = 1 or
 * nnz_avg < 4; MB if none of these and size = 0. Pure function. */
uint32_t spmv_feature_rules(const double *features, int64_t n_cols, int32_t vec_bytes,
                            int64_t l2_bytes, double long_row_ratio);

/* Validates a CSR held in device memory; *code = 0 valid, 1 rowptr[0] != 0, 2 rowptr
 * decreases, 3 rowptr[n_rows] != nnz, 4 column out of range, 5 columns not strictly
 * increasing (the first offending element in storage order decides 4 vs 5). */
spmv_status spmv_validate_csr(int64_t n_rows, int64_t n_cols, int64_t nnz,
                              const int32_t *row_ptr, const int32_t *col_ind, int32_t *code,
                              spmv_stream_t stream);

/* FP64 -> storage dtype conversion (round to nearest even, no double rounding for BF16)
 * of n device values into out (device). to = SPMV_DF64 writes n (hi, lo) FP32 pairs
 * (8 bytes each) split as SPMV_DF64 describes. */
spmv_status spmv_round_values(const double *in, void *out, int64_t n, spmv_dtype to,
                              spmv_stream_t stream);

/* Reads (and clears) the handle's device error word: 0 none, 1 a bounded wait expired. */
spmv_status spmv_get_last_device_error(spmv_handle_t h, int32_t *code);

/* Failure-path self test of the bounded device waits the tile kernels use: launches one
 * CTA that waits on an mbarrier phase nothing completes (transaction count armed, no copy
 * issued) with a limit of limit_ns (1 ns .. 10 s). The wait gives up, the kernel records the
 * expiry in the handle's error word and exits; the call then reads and clears the word and
 * returns SPMV_ERR_TIMEOUT (SPMV_OK would mean the wait completed). The CUDA context stays
 * usable. Synchronizes the stream. */
spmv_status spmv_selftest_wait_timeout(spmv_handle_t h, int64_t limit_ns, spmv_stream_t stream);

/* Device bytes held by the handle. */
spmv_status spmv_get_device_bytes(spmv_handle_t h, int64_t *bytes);

const char *spmv_status_string(spmv_status s);

/* ----------------------------------------------------- allocation-free SpMV -------- */
/* y = A x (FP64 values, x and y) with the merge-path variant, for callers that must not
 * allocate device memory: for example an application whose own allocator owns the device
 * memory budget and forbids libraries from allocating behind its back, code that runs while
 * the device is nearly full, or latency-critical code that cannot afford cudaMalloc /
 * cudaFree (which can synchronize the device). The paper has no counterpart; this is a
 * property of the library, not of the method.
 *
 * The caller passes the CSR (row_ptr[n_rows+1], col_ind[nnz], val[nnz]), x[n_cols] and
 * y[n_rows] as device pointers; the CSR is used as given (not validated: it must satisfy
 * the CSR definition). The call allocates nothing: its scratch (merge-path tile table and
 * per-tile carries) lives in one fixed 16 MiB array in device global memory, created when
 * the library's kernels are loaded on a device and held by every GPU that loads them until
 * the process exits. Sizes with n_rows + nnz above about 1.07e9 (599,158 tiles of 1792
 * merge items) are rejected with SPMV_ERR_TOO_LARGE before any work is queued.
 *
 * The first call on each device looks up the array's device address (a runtime call that
 * may synchronize, and that creates the device's context if needed); make that first call
 * before any stream capture. The address is kept per CUDA context: after cudaDeviceReset
 * (a new context, in which the array may sit elsewhere) the next call looks it up again, so
 * it too should come before any capture. Asynchronous on stream otherwise. All calls share the one array and each call's scratch contents stay
 * there until the next call overwrites them, so calls whose work overlaps on the GPU (on
 * different streams, or from different host threads, without ordering between them) race
 * and give wrong results; serialize them on one stream or with events. Errors:
 * SPMV_ERR_ARG (negative or oversized int32 sizes, null pointers), SPMV_ERR_TOO_LARGE,
 * SPMV_ERR_CUDA (launch failure). */
spmv_status spmv_run_noalloc(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t *row_ptr,
                             const int32_t *col_ind, const double *val, const double *x,
                             double *y, spmv_stream_t stream);

/* ------------------------------------------------------------ iterative solver ---- */
/* Conjugate gradients (Hestenes and Stiefel) for A x = b with A symmetric positive definite
 * (square handle, vec_type F64): the iterative-solver setting in which Section IV-D weighs
 * the optimizer's preprocessing against the SpMV time it saves. Every iteration applies the
 * handle's tuned variant once (spmv_tune or spmv_set_variant must come first); the dot
 * products and vector updates are the library's own FP64 kernels with fixed reduction
 * order, so a solve repeats bit for bit. Textbook order: r0 = b - A x0, p0 = r0;
 * alpha = (r,r)/(p,Ap), x += alpha p, r -= alpha Ap, beta = (r',r')/(r,r), p = r' + beta p;
 * alpha (beta) is 0 when its denominator is 0.
 *   b[n], x[n]: device FP64; x holds x0 on entry and the last iterate on return.
 *   The solve stops when ||r_k|| <= rtol ||b|| (||r_k|| from the recurrence) or after
 *   max_iters iterations; the host reads ||r_k|| every check_every iterations (each read
 *   synchronizes the stream), so up to check_every - 1 iterations may run past the point
 *   where the test was first met.
 *   res_hist: NULL or device FP64[max_iters + 1], receives ||r_k|| for k = 0 .. iterations.
 *   report: NULL or receives the iteration count, whether the test was met, the final
 *   ||r_k||, ||b|| and the wall time.
 * The handle keeps a workspace of 3 n doubles (+ a few KB) between calls. Synchronizes the
 * stream. Errors: SPMV_ERR_ARG (non-square, null vectors, max_iters < 0, rtol < 0 or NaN,
 * check_every < 1), SPMV_ERR_NOT_TUNED, SPMV_ERR_UNSUPPORTED_DTYPE (vec_type not F64),
 * SPMV_ERR_OOM, SPMV_ERR_CUDA. */
typedef struct {
  int32_t iters;      /* iterations run                                   */
  int32_t converged;  /* 1 if ||r_k|| <= rtol ||b|| at the last check      */
  double res_norm;    /* ||r_k|| (recurrence) at the end                   */
  double b_norm;      /* ||b||                                             */
  double t_ms;        /* wall time of the call                             */
} spmv_cg_report;

spmv_status spmv_cg(spmv_handle_t h, const double *b, double *x, int32_t max_iters,
                    double rtol, int32_t check_every, double *res_hist,
                    spmv_cg_report *report, spmv_stream_t stream);

/* ------------------------------------------------------------- learned selector ---- */
/* The MLP has layer sizes n_in -> h1 -> h2 -> 4 (ReLU hidden units, one logit per class
 * MB, ML, IMB, CMP); parameters packed W1 (h1 x n_in, row-major), b1, W2, b2, W3, b3, FP32.
 * Its inputs are SPMV_MLP_INPUTS numbers derived from the Table I features.             */
#define SPMV_MLP_INPUTS 12

/* Derived inputs on the device: feat (batch x 16 doubles: the 14 Table I features, then
 * n_rows and nnz), mu / inv_sigma (SPMV_MLP_INPUTS floats each, standardization; NULL =
 * none) -> X (batch x SPMV_MLP_INPUTS floats). All pointers device. */
spmv_status spmv_mlp_inputs(const double *feat, int64_t batch, const float *mu,
                            const float *inv_sigma, float *X, spmv_stream_t stream);

/* FP32 logits (batch x sizes[3]) with the fixed multiply-add order that defines the
 * decision: each unit starts from its bias and adds w_k * in_k in k order (fmaf). */
spmv_status spmv_mlp_logits(const int32_t *sizes, const float *params, int64_t batch,
                            const float *X, float *logits, spmv_stream_t stream);

/* Mean binary cross-entropy of sigmoid(logits) against Y (batch x sizes[3], 0/1) and
 * its gradient w.r.t. the packed parameters (backpropagation, FP32 with FP64 sums over
 * the batch, fixed order). grad and loss are device pointers. */
spmv_status spmv_mlp_loss_grad(const int32_t *sizes, const float *params, int64_t batch,
                               const float *X, const float *Y, float *grad, float *loss,
                               spmv_stream_t stream);

/* Runs `steps` full-batch Adam steps (lr, beta1, beta2, eps) on params in place; m and v
 * are the Adam moments (device, zero at step 0), t0 the number of steps already taken.
 * loss_hist (device, may be NULL) receives the loss before each step. */
spmv_status spmv_mlp_train(const int32_t *sizes, float *params, float *m, float *v,
                           int64_t batch, const float *X, const float *Y, int32_t steps,
                           int32_t t0, float lr, float beta1, float beta2, float eps,
                           float *loss_hist, spmv_stream_t stream);

/* A selector: host copies of sizes[4], params, mu and inv_sigma (SPMV_MLP_INPUTS floats
 * each) are uploaded to the current device. */
spmv_status spmv_selector_create(spmv_selector_t *out, const int32_t *sizes,
                                 const float *params, const float *mu,
                                 const float *inv_sigma);

/* Frees the selector's device buffers (synchronizes the device first). SPMV_ERR_ARG for
 * NULL. A handle tuned through the selector keeps its variant. */
spmv_status spmv_selector_destroy(spmv_selector_t s);

/* The training range of the selector's inputs: lo and hi (host, SPMV_MLP_INPUTS floats
 * each, in the standardized input space, copied) bound every input over the training set.
 * Afterwards spmv_selector_predict reports *margin = -1 for a feature vector any of whose
 * inputs lies more than `slack` outside [lo, hi]: the matrix is outside the distribution the
 * network learned from, and spmv_tune's learned route then falls back to profiling (any
 * opts.min_margin >= 0). SPMV_ERR_ARG for null pointers, lo > hi or slack < 0. */
spmv_status spmv_selector_set_range(spmv_selector_t s, const float *lo, const float *hi,
                                    float slack);

/* Class set predicted for a feature vector (16 doubles, host): logit > 0 per class.
 * *margin = smallest |logit|, or -1 when a training range is set and the inputs leave it. */
spmv_status spmv_selector_predict(spmv_selector_t s, const double *feat16, uint32_t *classes,
                                  double *margin, spmv_stream_t stream);

/* ----------------------------------------------------------------- batched SpMM ---- */
/* A batch of `count` tuned handles with FP32 storage, FP32 x/y and FP32 accumulation
 * (runs of at most 16 FP32 products per lane, summed in FP64 on long rows, so every row
 * stays within 2e-6 of sum_j |a_ij x_j|);
 * X[i] (n_cols_i x k[i]) and Y[i] (n_rows_i x k[i]) are row-major device arrays, k[i] in
 * {1, 4, 16}. The batch plans row-block work items (long rows split, partials summed in
 * FP64) and owns a CUDA graph of its launches. It reads the handles' device arrays in
 * place: the handles must outlive the batch, and a batched run answers SPMV_ERR_ARG once a
 * handle's precision has changed since the batch was created. */
spmv_status spmv_batch_create(spmv_batch_t *out, const spmv_handle_t *handles, int32_t count,
                              const void *const *X, void *const *Y, const int32_t *k,
                              spmv_stream_t stream);

/* All products of the batch in one persistent launch (CTAs take work items from a device
 * counter) plus a fixup launch, replayed from a CUDA graph captured on the first call. */
spmv_status spmv_run_batched(spmv_batch_t b, spmv_stream_t stream);

/* The batch's work plan: row blocks of about item_nnz nonzeros per warp (at most 1024 rows),
 * rows longer than item_nnz split into chunks of chunk_nnz nonzeros whose FP64 partials the
 * fixup adds in chunk order (defaults 1024 and 2048). Rebuilds the items and drops the
 * captured graph; synchronizes the device. SPMV_ERR_ARG unless 32 <= item_nnz <= 65536 and
 * item_nnz <= chunk_nnz <= 2^20. */
spmv_status spmv_batch_set_plan(spmv_batch_t b, int32_t item_nnz, int32_t chunk_nnz,
                                spmv_stream_t stream);

/* Autotuner of the batch plan: times `reps` replays (after two warm-ups) of each plan with
 * item_nnz in {256, 512, 1024, 2048} and chunk_nnz = 2 or 4 x item_nnz, keeps the fastest
 * and returns it in *item_nnz / *chunk_nnz (either may be NULL). Runs the batch, so X must
 * hold valid inputs and Y is overwritten. */
spmv_status spmv_batch_tune(spmv_batch_t b, int32_t reps, int32_t *item_nnz, int32_t *chunk_nnz,
                            spmv_stream_t stream);

/* The same work as plain per-matrix launches (no graph, no persistence), for comparison. */
spmv_status spmv_run_batched_sequential(spmv_batch_t b, spmv_stream_t stream);

/* Frees the batch's plan, graph, streams and device buffers (synchronizes the device first);
 * the handles and the caller's X / Y are not touched. SPMV_ERR_ARG for NULL. */
spmv_status spmv_batch_destroy(spmv_batch_t b);

#ifdef __cplusplus
}
#endif
#endif /* SPMV_GB300_H */

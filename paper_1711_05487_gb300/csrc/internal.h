// Host-side declarations shared by the translation units of the library (not part of
// the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spmv_gb300.h"

namespace spmv {

// Every device array the kernels read past its logical end (128-bit chunk loads of the
// last row) is allocated with this many zeroed elements of slack.
constexpr int64_t kPadElems = 32;

// Merge-path tile geometry.
constexpr int kMergeThreads = 256;
constexpr int kMergeIpt = 7;   // merge items per thread: an odd stride between threads keeps
                               // their shared-memory reads in distinct banks
constexpr int kMergeItems = kMergeThreads * kMergeIpt;

// Column index representation of a kernel instance: DB = 0 for int32 columns, 16 or 8 for
// column deltas of that width. A staged tile starts and ends on a multiple of
// stage_align<DB>() elements, so that its index copy is a whole number of 16-byte units.
template <int DB> struct IdxOf { using type = int32_t; };
template <> struct IdxOf<16> { using type = uint16_t; };
template <> struct IdxOf<8> { using type = uint8_t; };
template <int DB> __host__ __device__ constexpr int stage_align() { return DB == 8 ? 16 : 8; }
inline int stage_align_bits(int db) { return db == 8 ? 16 : 8; }

// Everything a SpMV launch needs; unused pointers are null.
struct RunArgs {
  int64_t n_rows = 0, n_cols = 0, nnz = 0;
  const int32_t *rowptr = nullptr;
  const int32_t *colind = nullptr;
  const void *delta = nullptr;       // column deltas, delta_bits (8 or 16) wide
  int32_t delta_bits = 16;
  const int32_t *dbase = nullptr;    // per-row base column / escape offset
  const int32_t *esc = nullptr;      // columns of escape rows
  const void *val = nullptr;         // storage dtype
  const void *x = nullptr;           // vec dtype
  void *y = nullptr;                 // vec dtype
  const int2 *coord = nullptr;       // merge-path tile table [n_tiles + 1]
  int64_t n_tiles = 0;
  int32_t *tail_row = nullptr;       // [n_tiles]
  double *tail_val = nullptr;        // [n_tiles]
  double *head_val = nullptr;        // [n_tiles]
  int32_t k = 1;                     // right-hand sides (SpMM)
  int32_t tile_cap = 0;              // staged elements per row tile (thread-per-row kernel)
  int32_t tile_rows = 0;             // rows (= threads) per tile: 32, 64 or 128
  int32_t tile_pipe = 0;             // 1: persistent CTAs with two staged tiles in flight
  int32_t y_add = 0;                 // 1: row sums are added to y (later column-panel passes)
  int32_t rows_once = 0;             // 1: row pointers and y are touched once (column-panel
                                     // passes): loaded and stored evict-first in the L2, so
                                     // that the slice of x stays resident
  int32_t f32_chain = 30;            // FP32 accumulation: longest row a thread sums in FP32
                                     // alone (16 when passes add into y: one rounding each)
  int32_t *err = nullptr;            // device error word (bounded waits)
  const void *val_df = nullptr;      // storage SPMV_DF64: double-float value pairs
  // row decomposition (partition 2): rows with length < bin_l_med go to sub-warps of
  // bin_vs_short lanes; medium rows (bin_rows) to a warp each; long rows (bin_long_rows,
  // length >= the chunk limit) in chunks (row, first, end nonzero, the column a delta decode of
  // the chunk starts from) whose FP64 partials are added per long row over
  // [bin_long_first[i], bin_long_first[i + 1])
  int32_t bin_l_med = 0, bin_vs_short = 4;
  const int32_t *bin_rows = nullptr;
  int64_t bin_n_med = 0;
  const int4 *bin_chunks = nullptr;
  int64_t bin_n_chunks = 0;
  const int32_t *bin_long_rows = nullptr;
  const int32_t *bin_long_first = nullptr;
  int64_t bin_n_long = 0;
  double *bin_partials = nullptr;
  // column panels (xpath >= 2): a panel-major copy of the matrix; panel p's row pointers
  // are pnl_rowptr + p * pnl_stride, absolute positions into pnl_col / pnl_val. A launch runs
  // the passes pnl_first .. pnl_first + n_panels - 1; pass 0 writes y, later passes add.
  const int32_t *pnl_rowptr = nullptr;
  const int32_t *pnl_col = nullptr;
  const void *pnl_val = nullptr;
  int64_t pnl_stride = 0;
  int32_t pnl_first = 0;
  int32_t n_panels = 0;
  int32_t pnl_tile_cap = 0;          // one thread per row (vs = 1): staged tiles of the passes
  int32_t pnl_tile_rows = 0;         // rows per staged tile of the passes
  // sliced rows (partition 3): 32-row slices stored column-major; element k of row r at
  // sell_off[r / 32] + 32 k + r % 32 of sell_val and sell_idx (int32 columns, or column
  // deltas of delta_bits bits with dbase / esc as for the delta index)
  const int64_t *sell_off = nullptr;
  const void *sell_val = nullptr;
  const void *sell_idx = nullptr;
};

// Column panels: at most this many slices of x (variant field xpath = panel count).
constexpr int kMaxPanels = 16;

// Default row decomposition limits (a variant may set its own): rows of at least kBinMed
// nonzeros get a warp; rows of at least kBinChunk nonzeros are split into chunks of
// kBinChunk nonzeros.
constexpr int kBinMed = 64;
constexpr int kBinChunk = 4096;
constexpr int kBinLimitMax = 1 << 20;

// Thread-per-row tile kernel geometry: at most this many rows (= threads) per CTA.
constexpr int kTileRows = 128;
// A bounded device wait gives up after this many nanoseconds.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// Static-partition profiling launch (Section III-B micro-benchmarks).
struct ProfileArgs {
  int64_t n_rows = 0, n_cols = 0;
  const int32_t *part = nullptr;     // [n_ctas + 1] row boundaries
  int32_t n_ctas = 0;
  const int32_t *rowptr = nullptr;
  const int32_t *colind = nullptr;   // colind, or colind' for P_ML
  const void *val = nullptr;
  const void *x = nullptr;
  void *y = nullptr;
  unsigned long long *t_start = nullptr;
  unsigned long long *t_end = nullptr;
  int32_t *smid = nullptr;            // SM that ran each CTA (may be null)
  int32_t cmp_mode = 0;              // 1: P_CMP kernel (x[i], no colind)
  int32_t vs = 8;
};

// One work item of the batched kernel: rows [row_begin, row_end) of matrix `mat` (nz_end
// then holds the block's nonzero count, used only to order items), or, when chunk >= 0,
// nonzeros [nz_begin, nz_end) of the single long row row_begin whose partial sums go to
// partial slot `chunk`.
struct BatchItem {
  int32_t mat;
  int32_t row_begin;
  int32_t row_end;
  int32_t nz_begin;
  int32_t nz_end;
  int32_t chunk;
};

struct BatchMat {
  const int32_t *rowptr;
  const int32_t *colind;
  const float *val;
  const float *X;
  float *Y;
  int32_t k;
  int32_t vs;
};

// A long row split over several items: partial slots [first, first + count), each k wide.
struct BatchFix {
  int32_t mat;
  int32_t row;
  int32_t first;
  int32_t count;
};

// Launchers, one set per (storage, vec, acc) dtype combination.
typedef cudaError_t (*spmv_launch_fn)(const spmv_variant &v, const RunArgs &a, cudaStream_t s);
typedef cudaError_t (*spmm_launch_fn)(const RunArgs &a, int vs, cudaStream_t s);
typedef cudaError_t (*profile_launch_fn)(const ProfileArgs &a, cudaStream_t s);

struct KernelSet {
  spmv_launch_fn spmv;
  spmm_launch_fn spmm;
  profile_launch_fn profile;
  int profile_blocks_per_sm;   // occupancy of the profiling kernel (for a resident grid)
};

// Returns null for combinations that are not offered.
const KernelSet *kernel_set(spmv_dtype val, spmv_dtype vec, spmv_dtype acc);

#define SPMV_DECLARE_SET(tag) const KernelSet *kernel_set_##tag();
SPMV_DECLARE_SET(f64_dd)
SPMV_DECLARE_SET(f32_dd)
SPMV_DECLARE_SET(f32_ff)
SPMV_DECLARE_SET(f32_fd)
SPMV_DECLARE_SET(bf16_dd)
SPMV_DECLARE_SET(bf16_ff)
SPMV_DECLARE_SET(bf16_fd)
SPMV_DECLARE_SET(f64_df)
#undef SPMV_DECLARE_SET

// Splits in[lo, hi) into double-float pairs out[lo, hi) (spmv_df.cu).
cudaError_t launch_df_split(const double *in, void *out, int64_t lo, int64_t hi, cudaStream_t s);

// ------------------------------------------------------------- preprocessing (prep.cu)
cudaError_t launch_validate(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t *rowptr,
                            const int32_t *colind, int32_t *d_code, cudaStream_t s);
cudaError_t launch_round_values(const double *in, void *out, int64_t n, spmv_dtype to,
                                cudaStream_t s);
cudaError_t launch_convert_values(const void *in, spmv_dtype from, void *out, spmv_dtype to,
                                  int64_t n, cudaStream_t s);
// Delta index: per row, the nonzeros that escape 8-bit and 16-bit deltas (the row's length
// when some gap exceeds 255, resp. 65535, else 0); then, for the chosen width, the fill and
// the inverse (decode back to colind).
cudaError_t launch_delta_flags(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                               int64_t *esc8, int64_t *esc16, cudaStream_t s);
cudaError_t launch_delta_fill(int bits, int64_t n_rows, const int32_t *rowptr,
                              const int32_t *colind, const int64_t *esc_off, int32_t *dbase,
                              void *delta, int32_t *esc, cudaStream_t s);
cudaError_t launch_delta_decode(int bits, int64_t n_rows, const int32_t *rowptr,
                                const int32_t *dbase, const void *delta, const int32_t *esc,
                                int32_t *colind, cudaStream_t s);
// exclusive scan of n int64 values in place; total (device, 1 value) receives the sum
cudaError_t launch_scan_i64(int64_t *data, int64_t n, int64_t *total, int64_t *scratch,
                            int64_t scratch_elems, cudaStream_t s);
int64_t scan_scratch_elems(int64_t n);
cudaError_t launch_merge_coords(int64_t n_rows, int64_t nnz, const int32_t *rowptr,
                                int64_t items, int64_t n_tiles, int2 *coord, cudaStream_t s);
cudaError_t launch_static_partition(int64_t n_rows, int64_t nnz, const int32_t *rowptr,
                                    int32_t n_parts, int32_t *part, cudaStream_t s);
cudaError_t launch_fill_row_index(int64_t n_rows, int64_t n_cols, const int32_t *rowptr,
                                  int32_t *out, cudaStream_t s);
cudaError_t launch_fill_const(void *p, spmv_dtype t, int64_t n, double v, cudaStream_t s);

// Features: per-block partial sums, then a final reduction into FeatSums (device).
struct FeatSums {
  unsigned long long s_nnz, s_sc, s_cl, s_miss, s_grp;
  unsigned long long s_nnz2_lo, s_nnz2_hi, s_bw_lo, s_bw_hi, s_bw2_lo, s_bw2_hi, s_sc2_lo,
      s_sc2_hi;
  long long nnz_min, nnz_max, bw_min, bw_max;
};
int feature_blocks(int64_t n_rows);
cudaError_t launch_features(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                            int32_t line_elems, FeatSums *partials, int n_blocks,
                            FeatSums *out, cudaStream_t s);
cudaError_t launch_row_len_max(int64_t n_rows, const int32_t *rowptr, int32_t *out,
                               cudaStream_t s);
// max over tiles of `tile_rows` rows of the staged element count, aligned to `align`
cudaError_t launch_tile_max(int64_t n_rows, const int32_t *rowptr, int tile_rows, int align,
                            int32_t *out, cudaStream_t s);

// Row decomposition tables: per-row counts (medium flag, long flag, chunks) for the scans,
// then the lists (bin_rows, long rows, their first chunk, chunk table).
cudaError_t launch_bin_counts(int64_t n_rows, const int32_t *rowptr, int32_t l_med,
                              int32_t chunk, int64_t *med, int64_t *lng, int64_t *nch,
                              cudaStream_t s);
cudaError_t launch_bin_fill(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                            int32_t l_med, int32_t chunk, const int64_t *med_off,
                            const int64_t *lng_off, const int64_t *nch_off, int32_t *bin_rows,
                            int32_t *long_rows, int32_t *long_first, int4 *chunks,
                            cudaStream_t s);

// Column panels of width w (panel p = columns [p*w, (p+1)*w), the last panel takes the rest):
// the nonzero count of every row in every panel ([n_panels][n_rows + 1] int64, for the
// scans), then the panel-major copy of the columns and values (val_bytes 2, 4 or 8) and
// each panel's row pointers ([n_panels][n_rows + 1] int32), from the scanned counts.
cudaError_t launch_panel_counts(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                                int32_t n_panels, int32_t width, int64_t *cnt, cudaStream_t s);
cudaError_t launch_panel_fill(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                              const void *val, int val_bytes, int32_t n_panels,
                              const int64_t *off, int32_t *pnl_rowptr, int32_t *pnl_col,
                              void *pnl_val, cudaStream_t s);

// Sliced rows: 32 x (the longest row) of every 32-row slice (int64, for the scan into slice
// offsets), then the column-major copy of the values (val_bytes 2, 4 or 8) and of the column
// representation (idx_bytes 4: int32 columns; 2 or 1: column deltas), padding left as it is.
cudaError_t launch_sell_widths(int64_t n_rows, const int32_t *rowptr, int64_t *w32,
                               cudaStream_t s);
cudaError_t launch_sell_fill(int64_t n_rows, const int32_t *rowptr, const void *val,
                             int val_bytes, const void *idx, int idx_bytes,
                             const int64_t *soff, void *sell_val, void *sell_idx,
                             cudaStream_t s);

// Largest column of each row chunk (host-buffer pipelining)
cudaError_t launch_chunk_colmax(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                                const int64_t *bounds, int n_chunks, int32_t *out,
                                cudaStream_t s);

// Failure-path self test (bounded wait that expires)
cudaError_t launch_selftest_wait(uint64_t limit_ns, int32_t *err, cudaStream_t s);

// Bandwidth probe
cudaError_t launch_gather_probe(const void *x, int32_t elem_bytes, int64_t n_x, int64_t count,
                                unsigned long long *sink, cudaStream_t s);
cudaError_t launch_fma_probe(int32_t elem_bytes, int32_t chains, int32_t warps_per_sm,
                             int32_t fmas_per_thread, int64_t *n_threads,
                             unsigned long long *sink, cudaStream_t s);
cudaError_t launch_read_probe(const void *buf, int64_t bytes, int reps,
                              unsigned long long *sink, cudaStream_t s);

// MLP (mlp.cu)
cudaError_t launch_mlp_inputs(const double *feat, int64_t batch, const float *mu,
                              const float *inv_sigma, float *X, cudaStream_t s);
cudaError_t launch_mlp_logits(const int32_t *sizes, const float *params, int64_t batch,
                              const float *X, float *logits, cudaStream_t s);
cudaError_t launch_mlp_loss_grad(const int32_t *sizes, const float *params, int64_t batch,
                                 const float *X, const float *Y, float *grad, float *loss,
                                 float *work, cudaStream_t s);
int64_t mlp_work_floats(const int32_t *sizes, int64_t batch);
int64_t mlp_logits_work_floats(const int32_t *sizes, int64_t batch);
cudaError_t launch_mlp_logits_ws(const int32_t *sizes, const float *params, int64_t batch,
                                 const float *X, float *logits, float *work, cudaStream_t s);
int64_t mlp_param_count(const int32_t *sizes);
cudaError_t launch_adam(int64_t n, float *p, const float *g, float *m, float *v, float lr,
                        float b1, float b2, float eps, int32_t t, cudaStream_t s);

// Batched (batch.cu): one persistent kernel over the work items of every matrix (each
// item run with the code of its matrix's k in {1, 4, 16}), then the fixup of split rows
cudaError_t launch_batch_persistent(const BatchMat *mats, const BatchItem *items,
                                    int32_t n_items, int32_t *counter, double *partials,
                                    int grid, cudaStream_t s);
cudaError_t launch_batch_fixup(const BatchMat *mats, const BatchFix *fix, int32_t n_fix,
                               const double *partials, cudaStream_t s);
int batch_blocks_per_sm();

// Conjugate gradients (cg.cu): deterministic FP64 vector kernels; each reduction writes
// fixed-grid block partials to `part` (cg_reduce_blocks() doubles) and then one scalar.
int cg_reduce_blocks();
cudaError_t launch_dot(const double *a, const double *b, int64_t n, double *part, double *out,
                       double *hist, cudaStream_t s);
cudaError_t launch_cg_start(const double *b, const double *ax, double *r, double *p, int64_t n,
                            double *part, double *rr, double *hist, cudaStream_t s);
cudaError_t launch_cg_xr(const double *p, const double *ap, double *x, double *r, int64_t n,
                         const double *rr, const double *pap, double *part, double *rr_new,
                         double *hist, cudaStream_t s);
cudaError_t launch_cg_p(const double *r, double *p, int64_t n, const double *rr,
                        const double *rr_new, cudaStream_t s);

// Device arrays and dtypes of a handle (vs = tuned sub-warp width, 0 if none).
spmv_status handle_info(spmv_handle_t h, const int32_t **rowptr, const int32_t **colind,
                        const void **val, int64_t *n_rows, int32_t *storage, int32_t *vec,
                        int32_t *acc, int32_t *vs);

}  // namespace spmv

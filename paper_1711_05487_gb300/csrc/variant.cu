// Optimization-pool data and variant installation (Table II): the delta index, the
// merge-path tile table, the row decomposition tables and the thread-per-row tile geometry.
#include "handle.h"

using namespace spmv;
using namespace spmv::rt;

namespace spmv {
namespace rt {

const KernelSet *set_for(const spmv_matrix *h) { return kernel_set(h->storage, h->vec, h->acc); }

RunArgs run_args(const spmv_matrix *h, const void *x, void *y) {
  RunArgs a;
  a.n_rows = h->n_rows;
  a.n_cols = h->n_cols;
  a.nnz = h->nnz;
  a.rowptr = h->rowptr.as<int32_t>();
  a.colind = h->colind.as<int32_t>();
  a.delta = h->delta.p;
  a.delta_bits = h->delta_bits;
  a.dbase = h->dbase.as<int32_t>();
  a.esc = h->esc.as<int32_t>();
  a.val = h->val_ptr();
  a.x = x;
  a.y = y;
  a.coord = h->coord.as<int2>();
  a.n_tiles = h->n_tiles;
  a.tail_row = h->tail_row.as<int32_t>();
  a.tail_val = h->tail_val.as<double>();
  a.head_val = h->head_val.as<double>();
  a.tile_cap = h->tile_cap;
  a.tile_rows = h->tile_rows;
  a.tile_pipe = h->tile_pipe;
  a.err = h->d_err.as<int32_t>();
  a.val_df = h->val_df.p;
  a.bin_l_med = h->bin_med;
  a.bin_vs_short = h->bin_vs_short;
  a.bin_rows = h->bin_rows.as<int32_t>();
  a.bin_n_med = h->bin_n_med;
  a.bin_chunks = h->bin_chunks.as<int4>();
  a.bin_n_chunks = h->bin_n_chunks;
  a.bin_long_rows = h->bin_long_rows.as<int32_t>();
  a.bin_long_first = h->bin_long_first.as<int32_t>();
  a.bin_n_long = h->bin_n_long;
  a.bin_partials = h->bin_partials.as<double>();
  a.pnl_rowptr = h->pnl_rowptr.as<int32_t>();
  a.pnl_col = h->pnl_col.as<int32_t>();
  a.pnl_val = h->pnl_val.p;
  a.sell_off = h->sell_off.as<int64_t>();
  a.sell_val = h->sell_val.p;
  a.sell_idx = h->sell_idx.p;
  a.pnl_stride = h->n_rows + 1;
  a.pnl_first = 0;
  a.n_panels = h->pnl_count;
  a.pnl_tile_cap = h->pnl_tile_cap;
  a.pnl_tile_rows = h->pnl_tile_rows;
  return a;
}

}  // namespace rt
}  // namespace spmv

namespace {

// The delta index (Section III-E, MB): 8- or 16-bit column deltas, never both; the width
// is the one whose index is smaller (1 or 2 bytes per nonzero of the rows whose gaps fit,
// 4 per nonzero of escape rows), 16 on a tie.
void build_delta(spmv_matrix *h, cudaStream_t s) {
  if (h->has_delta) return;
  const int64_t n = h->n_rows;
  DevBuf cnt;
  cnt.alloc(sizeof(int64_t) * 2 * (size_t)(n + 1), 8, s, true);
  int64_t *e8 = cnt.as<int64_t>(), *e16 = e8 + (n + 1);
  CK(launch_delta_flags(n, h->rowptr.as<int32_t>(), h->colind.as<int32_t>(), e8, e16, s));
  const int64_t se = scan_scratch_elems(n);
  DevBuf scr;
  scr.alloc(sizeof(int64_t) * (size_t)se, 8, s);
  CK(launch_scan_i64(e8, n, e8 + n, scr.as<int64_t>(), se, s));
  CK(launch_scan_i64(e16, n, e16 + n, scr.as<int64_t>(), se, s));
  int64_t esc8 = 0, esc16 = 0;
  CK(cudaMemcpyAsync(&esc8, e8 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&esc16, e16 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int64_t bytes8 = (h->nnz - esc8) + 4 * esc8;
  const int64_t bytes16 = 2 * (h->nnz - esc16) + 4 * esc16;
  const int bits = bytes8 < bytes16 ? 8 : 16;
  const int64_t n_esc = bits == 8 ? esc8 : esc16;
  h->dbase.alloc(sizeof(int32_t) * (size_t)n, 4, s);
  h->delta.alloc((size_t)(bits / 8) * (size_t)h->nnz, (size_t)(bits / 8), s);
  h->esc.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(n_esc, 1), 4, s);
  CK(launch_delta_fill(bits, n, h->rowptr.as<int32_t>(), h->colind.as<int32_t>(),
                       bits == 8 ? e8 : e16, h->dbase.as<int32_t>(), h->delta.p,
                       h->esc.as<int32_t>(), s));
  CK(cudaStreamSynchronize(s));
  h->n_esc = n_esc;
  h->delta_bits = bits;
  h->has_delta = true;
}

void build_merge(spmv_matrix *h, cudaStream_t s) {
  if (h->has_merge) return;
  const int64_t total = h->n_rows + h->nnz;
  const int64_t n_tiles = (total + kMergeItems - 1) / kMergeItems;
  h->coord.alloc(sizeof(int2) * (size_t)(n_tiles + 1), 8, s);
  h->tail_row.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(n_tiles, 1), 4, s, true);
  h->tail_val.alloc(sizeof(double) * (size_t)std::max<int64_t>(n_tiles, 1), 8, s, true);
  h->head_val.alloc(sizeof(double) * (size_t)std::max<int64_t>(n_tiles, 1), 8, s, true);
  CK(launch_merge_coords(h->n_rows, h->nnz, h->rowptr.as<int32_t>(), kMergeItems, n_tiles,
                         h->coord.as<int2>(), s));
  CK(cudaStreamSynchronize(s));
  h->n_tiles = n_tiles;
  h->has_merge = true;
}

// Row decomposition tables (partition 2): three exclusive scans over per-row counts place
// each medium row in the row list and each long row's chunks in the chunk table.
void build_bins(spmv_matrix *h, int32_t l_med, int32_t chunk, cudaStream_t s) {
  if (h->has_bins && h->bin_med == l_med && h->bin_chunk == chunk) return;
  h->has_bins = false;
  for (DevBuf *b : {&h->bin_rows, &h->bin_long_rows, &h->bin_long_first, &h->bin_chunks,
                    &h->bin_partials})
    b->release();
  const int64_t n = h->n_rows;
  DevBuf cnt;
  cnt.alloc(sizeof(int64_t) * 3 * (size_t)(n + 1), 8, s, true);
  int64_t *med = cnt.as<int64_t>(), *lng = med + (n + 1), *nch = lng + (n + 1);
  CK(launch_bin_counts(n, h->rowptr.as<int32_t>(), l_med, chunk, med, lng, nch, s));
  const int64_t se = scan_scratch_elems(n);
  DevBuf scr;
  scr.alloc(sizeof(int64_t) * (size_t)se, 8, s);
  for (int64_t *p : {med, lng, nch}) CK(launch_scan_i64(p, n, p + n, scr.as<int64_t>(), se, s));
  int64_t tot[3];
  for (int q = 0; q < 3; ++q)
    CK(cudaMemcpyAsync(tot + q, med + (int64_t)q * (n + 1) + n, sizeof(int64_t),
                       cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->bin_rows.alloc(4 * (size_t)std::max<int64_t>(tot[0], 1), 4, s);
  h->bin_long_rows.alloc(4 * (size_t)std::max<int64_t>(tot[1], 1), 4, s);
  h->bin_long_first.alloc(4 * (size_t)(tot[1] + 1), 4, s);
  h->bin_chunks.alloc(16 * (size_t)std::max<int64_t>(tot[2], 1), 16, s);
  h->bin_partials.alloc(8 * (size_t)std::max<int64_t>(tot[2], 1), 8, s);
  const int32_t last = (int32_t)tot[2];
  CK(cudaMemcpyAsync(h->bin_long_first.as<int32_t>() + tot[1], &last, 4, cudaMemcpyHostToDevice, s));
  CK(launch_bin_fill(n, h->rowptr.as<int32_t>(), h->colind.as<int32_t>(), l_med, chunk,
                     med, lng, nch,
                     h->bin_rows.as<int32_t>(), h->bin_long_rows.as<int32_t>(),
                     h->bin_long_first.as<int32_t>(), h->bin_chunks.as<int4>(), s));
  CK(cudaStreamSynchronize(s));
  h->bin_n_med = tot[0];
  h->bin_n_long = tot[1];
  h->bin_n_chunks = tot[2];
  h->bin_med = l_med;
  h->bin_chunk = chunk;
  h->has_bins = true;
}

int32_t max_tile_elems(spmv_matrix *h, const int32_t *rowptr, int rows, int align,
                       cudaStream_t s);
int32_t tile_limit(const spmv_matrix *h, const spmv_variant &v, bool pipe);

// Column panels (xpath = P >= 2): the panel-major copy of the columns and of the values
// the kernels read (the storage copy, or the FP64 input for double-float storage), built
// from per-row panel counts and one exclusive scan per panel. Panel p holds the columns
// [p*w, (p+1)*w), w = ceil(n_cols / P) rounded up to a multiple of 32.
void build_panels(spmv_matrix *h, int n_panels, cudaStream_t s) {
  if (h->pnl_count == n_panels) return;
  drop_panels(h);
  const int64_t n = h->n_rows;
  int64_t w = (h->n_cols + n_panels - 1) / n_panels;
  w = std::max<int64_t>(32, (w + 31) / 32 * 32);
  DevBuf cnt;
  cnt.alloc(sizeof(int64_t) * (size_t)n_panels * (size_t)(n + 1), 8, s, true);
  int64_t *c = cnt.as<int64_t>();
  CK(launch_panel_counts(n, h->rowptr.as<int32_t>(), h->colind.as<int32_t>(), n_panels,
                         (int32_t)w, c, s));
  const int64_t se = scan_scratch_elems(n);
  DevBuf scr;
  scr.alloc(sizeof(int64_t) * (size_t)se, 8, s);
  for (int p = 0; p < n_panels; ++p) {
    int64_t *cp = c + (int64_t)p * (n + 1);
    CK(launch_scan_i64(cp, n, cp + n, scr.as<int64_t>(), se, s));
  }
  const size_t vb = h->storage == SPMV_DF64 ? 8 : dtype_bytes(h->storage);
  h->pnl_rowptr.alloc(4 * (size_t)n_panels * (size_t)(n + 1), 4, s);
  h->pnl_col.alloc(4 * (size_t)h->nnz, 4, s);
  h->pnl_val.alloc(vb * (size_t)h->nnz, vb, s);
  CK(launch_panel_fill(n, h->rowptr.as<int32_t>(), h->colind.as<int32_t>(), h->val_ptr(),
                       (int)vb, n_panels, c, h->pnl_rowptr.as<int32_t>(),
                       h->pnl_col.as<int32_t>(), h->pnl_val.p, s));
  CK(cudaStreamSynchronize(s));
  h->pnl_count = n_panels;
  h->pnl_width = (int32_t)w;
  // staged tiles of the one-thread-per-row passes: the largest of 128, 64, 32 rows whose
  // largest tile over all panels fits one 48 KB stage (int32 columns)
  spmv_variant pv{};
  const int32_t limit = tile_limit(h, pv, false);
  h->pnl_tile_rows = 0;
  for (int rows = kTileRows; rows >= 32; rows /= 2) {
    int32_t m = 0;
    for (int p = 0; p < n_panels; ++p)
      m = std::max(m, max_tile_elems(h, h->pnl_rowptr.as<int32_t>() + (int64_t)p * (n + 1), rows,
                                     8, s));
    if (m <= limit || rows == 32) {
      h->pnl_tile_rows = rows;
      h->pnl_tile_cap = std::min(m, limit);
      break;
    }
  }
}

// Slice offsets of the sliced-row layout: 32 x the longest row of each 32-row slice, scanned
// (n_slices + 1 entries, the last one the total).
DevBuf sell_offsets(spmv_matrix *h, int64_t *total, cudaStream_t s) {
  const int64_t ns = (h->n_rows + 31) / 32;
  DevBuf off;
  off.alloc(sizeof(int64_t) * (size_t)(ns + 1), 8, s, true);
  CK(launch_sell_widths(h->n_rows, h->rowptr.as<int32_t>(), off.as<int64_t>(), s));
  const int64_t se = scan_scratch_elems(ns);
  DevBuf scr;
  scr.alloc(sizeof(int64_t) * (size_t)se, 8, s);
  CK(launch_scan_i64(off.as<int64_t>(), ns, off.as<int64_t>() + ns, scr.as<int64_t>(), se, s));
  CK(cudaMemcpyAsync(total, off.as<int64_t>() + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return off;
}

// Sliced rows (partition 3): the column-major copy of the values the kernels read and of the
// columns (bits = 0) or of the delta index's deltas (bits = 8 or 16).
void build_sell(spmv_matrix *h, int bits, cudaStream_t s) {
  if (h->sell_bits == bits) return;
  drop_sell(h);
  int64_t total = 0;
  DevBuf off = sell_offsets(h, &total, s);
  const size_t vb = h->storage == SPMV_DF64 ? 8 : dtype_bytes(h->storage);
  const size_t ib = bits ? (size_t)(bits / 8) : 4;
  h->sell_val.alloc(vb * (size_t)total, vb, s, true);
  h->sell_idx.alloc(ib * (size_t)total, ib, s, true);
  CK(launch_sell_fill(h->n_rows, h->rowptr.as<int32_t>(), h->val_ptr(), (int)vb,
                      bits ? h->delta.p : (const void *)h->colind.p, (int)ib,
                      off.as<int64_t>(), h->sell_val.p, h->sell_idx.p, s));
  CK(cudaStreamSynchronize(s));
  h->sell_off = std::move(off);
  h->sell_total = total;
  h->sell_bits = bits;
}

// Geometry of the thread-per-row kernel. A staged tile holds the values and columns of
// `rows` consecutive rows; the staged capacity is the matrix's largest such tile, capped by
// the shared-memory budget of one stage (48 KB for one tile per CTA, 56 KB per stage for
// the persistent two-stage kernel). Tiles above the cap are computed from global memory.
// staged-tile alignment of the variant's column representation
int tile_align(const spmv_matrix *h, const spmv_variant &v) {
  return v.index == 1 ? stage_align_bits(h->delta_bits) : 8;
}

int32_t max_tile_elems(spmv_matrix *h, const int32_t *rowptr, int rows, int align,
                       cudaStream_t s) {
  CK(launch_tile_max(h->n_rows, rowptr, rows, align, h->small.as<int32_t>(), s));
  int32_t m = 0;
  CK(cudaMemcpyAsync(&m, h->small.p, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return m;
}

int32_t tile_limit(const spmv_matrix *h, const spmv_variant &v, bool pipe) {
  const int eb = (int)dtype_bytes(h->storage) + (v.index == 1 ? h->delta_bits / 8 : 4);
  const int budget = (pipe ? 56 : 48) * 1024 - 32;
  const int al = tile_align(h, v);
  return ((budget / eb) / al) * al;
}

}  // namespace

namespace spmv {
namespace rt {

void set_tile_geometry(spmv_matrix *h, const spmv_variant &v, int rows, bool pipe,
                       cudaStream_t s) {
  h->tile_rows = rows;
  h->tile_pipe = pipe ? 1 : 0;
  h->tile_cap = std::min(max_tile_elems(h, h->rowptr.as<int32_t>(), rows, tile_align(h, v), s),
                         tile_limit(h, v, pipe));
}

// Default geometry: the largest of 128, 64, 32 rows per tile whose largest tile fits one
// 48 KB stage, one tile per CTA; 128-row tiles when none fits.
void compute_tile_cap(spmv_matrix *h, const spmv_variant &v, cudaStream_t s) {
  const int32_t limit = tile_limit(h, v, false);
  for (int rows = kTileRows; rows >= 32; rows /= 2) {
    const int32_t m = max_tile_elems(h, h->rowptr.as<int32_t>(), rows, tile_align(h, v), s);
    if (m <= limit) {
      h->tile_rows = rows;
      h->tile_pipe = 0;
      h->tile_cap = m;
      return;
    }
  }
  set_tile_geometry(h, v, kTileRows, false, s);
}

void drop_sell(spmv_matrix *h) {
  h->sell_off.release();
  h->sell_val.release();
  h->sell_idx.release();
  h->sell_bits = -1;
  h->sell_total = 0;
}

int64_t sell_positions(spmv_matrix *h, cudaStream_t s) {
  int64_t total = 0;
  sell_offsets(h, &total, s);
  return total;
}

void drop_panels(spmv_matrix *h) {
  h->pnl_rowptr.release();
  h->pnl_col.release();
  h->pnl_val.release();
  h->pnl_count = 0;
  h->pnl_width = 0;
}

void prepare_variant(spmv_matrix *h, spmv_variant &v, cudaStream_t s) {
  if (v.partition != 2 || v.xpath >= 2) {   // the limits belong to the row decomposition
    v.bin_med = 0;
    v.bin_chunk = 0;
  }
  if (v.xpath >= 2) {
    // column panels: rows on sub-warps of vs lanes over each panel's CSR, int32 columns
    v.partition = 0;
    v.index = 0;
    v.tile_rows = 0;
    v.tile_pipe = 0;
    if (v.vs == 0) v.vs = std::min(8, pow2_ceil_clamped(h->nnz_avg() / v.xpath, 1, 8));
    build_panels(h, v.xpath, s);
    return;
  }
  if (v.partition == 3) {
    // sliced rows: thread per row, int32 columns or the delta index's deltas
    if (v.index == 1) build_delta(h, s);
    v.vec = 1;
    v.vs = 1;
    v.tile_rows = 0;
    v.tile_pipe = 0;
    build_sell(h, v.index == 1 ? h->delta_bits : 0, s);
    return;
  }
  if (v.partition == 1) {
    v.index = 0;                 // the delta index is built for sub-warp rows only
    build_merge(h, s);
  } else if (v.partition == 2) {
    if (v.index == 1) build_delta(h, s);
    v.vec = 1;
    if (v.vs != 1 && v.vs != 2 && v.vs != 4 && v.vs != 8) v.vs = 4;   // short rows' width
    v.tile_rows = 0;
    v.tile_pipe = 0;
    h->bin_vs_short = v.vs;
    if (v.bin_med == 0) v.bin_med = kBinMed;
    if (v.bin_chunk == 0) v.bin_chunk = kBinChunk;
    build_bins(h, v.bin_med, v.bin_chunk, s);
  } else {
    if (v.index == 1) {
      v.vec = 1;
      build_delta(h, s);
    }
    if (v.vs == 0) {
      v.vs = (v.vec || v.index == 1) ? pool_vs(h->nnz_avg(), v.index == 1 ? 8 : 4)
                                     : heuristic_vs(h->nnz_avg(), 1);
    }
    if (h->acc == SPMV_DF64) v.tile_pipe = 0;   // the double-float kernel: one tile per CTA
    if (v.vs == 1 && v.tile_rows != 0) {
      set_tile_geometry(h, v, v.tile_rows, v.tile_pipe != 0, s);
    } else {
      compute_tile_cap(h, v, s);
      if (v.vs == 1) {
        v.tile_rows = h->tile_rows;
        v.tile_pipe = h->tile_pipe;
      }
    }
    if (v.vs != 1) {
      v.tile_rows = 0;
      v.tile_pipe = 0;
    }
  }
}

bool valid_variant(const spmv_variant &v) {
  if (v.partition < 0 || v.partition > 3) return false;
  if (v.partition == 3 && v.vs != 0 && v.vs != 1) return false;
  if (v.partition == 2 && v.vs != 0 && v.vs != 1 && v.vs != 2 && v.vs != 4 && v.vs != 8)
    return false;
  if (v.index != 0 && v.index != 1) return false;
  if (v.xpath < 0 || v.xpath > kMaxPanels) return false;
  if (v.xpath >= 2 && v.vs != 0 && v.vs != 1 && v.vs != 2 && v.vs != 4 && v.vs != 8)
    return false;
  if (v.vec != 0 && v.vec != 1) return false;
  if (v.partition == 0 && v.vs != 0 && v.vs != 1 && v.vs != 2 && v.vs != 4 && v.vs != 8 &&
      v.vs != 16 && v.vs != 32)
    return false;
  if (v.tile_rows != 0 && v.tile_rows != 32 && v.tile_rows != 64 && v.tile_rows != 128)
    return false;
  if (v.tile_pipe != 0 && v.tile_pipe != 1) return false;
  const int32_t med = v.bin_med ? v.bin_med : kBinMed, chunk = v.bin_chunk ? v.bin_chunk : kBinChunk;
  if (v.bin_med < 0 || v.bin_chunk < 0 || med < 2 || med > chunk || chunk > kBinLimitMax)
    return false;
  return true;
}

cudaError_t launch_run(const spmv_matrix *h, const spmv_variant &v, const void *x, void *y,
                       cudaStream_t s) {
  const KernelSet *ks = set_for(h);
  RunArgs a = run_args(h, x, y);
  return ks->spmv(v, a, s);
}

}  // namespace rt
}  // namespace spmv

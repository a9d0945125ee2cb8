// Host runtime behind the C ABI of include/spmv_gb300.h.
//
// A handle owns a device copy of the CSR matrix (int32 row pointers and columns, values
// in the input dtype, plus a converted copy in the storage dtype), the data of the
// installed optimization-pool variant (16-bit delta index or merge-path tile table and
// carry buffers), and staging buffers for host-buffer runs. spmv_tune classifies the
// matrix (Section III-C profiling, Section III-D features, or the learned selector),
// maps the class set to a variant (Table II, applied jointly), builds the variant's
// data and optionally times the sub-warp widths.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"

using namespace spmv;

// ------------------------------------------------------------------ helpers ----------
namespace {

typedef unsigned __int128 u128;
// Host-buffer runs split the rows into this many chunks so that the upload of the part of x
// the next chunk needs and the download of the previous chunk's y overlap the computation.
constexpr int kHostChunks = 8;

inline size_t dtype_bytes(spmv_dtype t) {
  return (t == SPMV_F64 || t == SPMV_DF64) ? 8 : (t == SPMV_F32 ? 4 : 2);
}
// input value types (spmv_create); SPMV_DF64 is a storage / arithmetic choice only
inline bool valid_dtype(int t) { return t == SPMV_F64 || t == SPMV_F32 || t == SPMV_BF16; }
inline bool valid_precision_dtype(int t) { return valid_dtype(t) || t == SPMV_DF64; }

struct CudaFail {
  cudaError_t e;
};

inline spmv_status map_err(cudaError_t e) {
  if (e == cudaSuccess) return SPMV_OK;
  if (e == cudaErrorMemoryAllocation) return SPMV_ERR_OOM;
  return SPMV_ERR_CUDA;
}

#define CK(expr)                                  \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) throw CudaFail{_e};    \
  } while (0)

// Device buffer with zeroed slack past the logical end (see kPadElems).
// A device allocation owned by exactly one object (move-only; freed on destruction, so
// temporaries do not leak when a CUDA error unwinds a build step).
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes) {
    o.p = nullptr;
    o.bytes = 0;
  }
  DevBuf &operator=(DevBuf &&o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      bytes = o.bytes;
      o.p = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t logical_bytes, size_t elem_bytes, cudaStream_t s, bool zero_all = false) {
    release();
    size_t pad = (size_t)kPadElems * elem_bytes;
    size_t total = ((logical_bytes + pad + 255) / 256) * 256;
    CK(cudaMalloc(&p, total));
    bytes = total;
    if (zero_all) {
      CK(cudaMemsetAsync(p, 0, total, s));
    } else if (total > logical_bytes) {
      CK(cudaMemsetAsync(static_cast<char *>(p) + logical_bytes, 0, total - logical_bytes, s));
    }
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T> T *as() const { return static_cast<T *>(p); }
};

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int pow2_ceil_clamped(double v, int lo, int hi) {
  int p = lo;
  while (p < hi && (double)p < v) p <<= 1;
  return p;
}

// Sub-warp width heuristic: enough lanes to cover the average row in one step of E
// elements per lane.
int heuristic_vs(double nnz_avg, int elems_per_lane) {
  return pow2_ceil_clamped(nnz_avg / (double)elems_per_lane, 2, 32);
}

// Width for the pool's sub-warp-row variants: rows of up to 64 nonzeros on average go to
// the thread-per-row tile kernel (width 1: one FMA per nonzero, no lane reduction);
// longer rows to sub-warps wide enough to cover them.
int pool_vs(double nnz_avg, int elems_per_lane) {
  return nnz_avg <= 64.0 ? 1 : heuristic_vs(nnz_avg, elems_per_lane);
}

struct DeviceInfo {
  int sms = 0;
  int64_t l2_bytes = 0;
  bool bw_done = false;
  double hbm_gbs = 0.0, l2_gbs = 0.0;
};

std::mutex g_dev_mu;
DeviceInfo g_dev[64];

DeviceInfo &device_info(int dev) {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DeviceInfo &d = g_dev[dev & 63];
  if (d.sms == 0) {
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    d.l2_bytes = l2;
  }
  return d;
}

}  // namespace

// ------------------------------------------------------------------ handle -----------
struct spmv_matrix {
  int device = 0;
  int64_t n_rows = 0, n_cols = 0, nnz = 0;
  spmv_dtype in_type = SPMV_F64, storage = SPMV_F64, vec = SPMV_F64, acc = SPMV_F64;
  DevBuf rowptr, colind, val_in, val_store;
  DevBuf val_df;               // storage SPMV_DF64: double-float value pairs
  // optimization-pool data
  DevBuf dbase, delta, esc;
  int64_t n_esc = 0;
  int32_t delta_bits = 16;     // width of the built delta index: 8 or 16
  bool has_delta = false;
  DevBuf coord, tail_row, tail_val, head_val;
  int64_t n_tiles = 0;
  bool has_merge = false;
  DevBuf bin_rows, bin_long_rows, bin_long_first, bin_chunks, bin_partials;
  int64_t bin_n_med = 0, bin_n_long = 0, bin_n_chunks = 0;
  int32_t bin_vs_short = 4;
  bool has_bins = false;
  // run state
  spmv_variant variant{};
  bool tuned = false;
  int32_t tile_cap = 0;        // staged elements per tile of the thread-per-row kernel
  int32_t tile_rows = kTileRows;  // rows per tile of the thread-per-row kernel
  int32_t tile_pipe = 0;       // 1: persistent CTAs with two tiles in flight
  DevBuf d_err;                // device error word of bounded waits
  DevBuf small;                // 256 bytes for single-value reductions (maxima, codes)
  cudaStream_t copy_stream = nullptr;   // host-buffer runs: device-to-host copies of y
  cudaStream_t upload_stream = nullptr; // host-buffer runs: host-to-device copies of x
  cudaStream_t capture_stream = nullptr;  // host-buffer runs: graph capture
  cudaStream_t chunk_stream[2] = {};    // host-buffer runs: alternate chunks' kernels
  cudaEvent_t joined[5] = {};           // host-buffer runs: fork from / rejoin the origin
  cudaGraph_t host_graph = nullptr;     // host-buffer pipeline for (host_x, host_y, epoch)
  cudaGraphExec_t host_exec = nullptr;
  const void *host_x = nullptr;
  void *host_y = nullptr;
  uint64_t host_epoch = 0;
  uint64_t epoch = 1;                   // bumped whenever precision or variant changes
  cudaEvent_t chunk_done[kHostChunks] = {};
  cudaEvent_t x_ready[kHostChunks] = {};
  int64_t x_need[kHostChunks] = {};     // elements of x (a prefix) chunks 0..c read
  bool x_need_valid = false;
  DevBuf feat_part, feat_fin;  // feature partial sums, kept between calls
  DevBuf x_stage, y_stage, scratch;
  DevBuf cg_ws;                // conjugate gradients: r, p, Ap, block partials, scalars
  int32_t last_error = 0;
  double nnz_avg() const { return n_rows ? (double)nnz / (double)n_rows : 0.0; }
  const void *val_ptr() const { return val_store.p ? val_store.p : val_in.p; }
};

struct spmv_selector {
  int device = 0;
  int32_t sizes[4] = {0, 0, 0, 0};
  DevBuf params, mu, inv_sigma;
  DevBuf ws;                   // one sample: 16 features, inputs, hidden layers, logits
  bool has_norm = false;
};

namespace {

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
  a.bin_l_med = kBinMed;
  a.bin_vs_short = h->bin_vs_short;
  a.bin_rows = h->bin_rows.as<int32_t>();
  a.bin_n_med = h->bin_n_med;
  a.bin_chunks = h->bin_chunks.as<int4>();
  a.bin_n_chunks = h->bin_n_chunks;
  a.bin_long_rows = h->bin_long_rows.as<int32_t>();
  a.bin_long_first = h->bin_long_first.as<int32_t>();
  a.bin_n_long = h->bin_n_long;
  a.bin_partials = h->bin_partials.as<double>();
  return a;
}

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
void build_bins(spmv_matrix *h, cudaStream_t s) {
  if (h->has_bins) return;
  const int64_t n = h->n_rows;
  DevBuf cnt;
  cnt.alloc(sizeof(int64_t) * 3 * (size_t)(n + 1), 8, s, true);
  int64_t *med = cnt.as<int64_t>(), *lng = med + (n + 1), *nch = lng + (n + 1);
  CK(launch_bin_counts(n, h->rowptr.as<int32_t>(), kBinMed, kBinChunk, med, lng, nch, s));
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
  CK(launch_bin_fill(n, h->rowptr.as<int32_t>(), h->colind.as<int32_t>(), kBinMed, kBinChunk,
                     med, lng, nch,
                     h->bin_rows.as<int32_t>(), h->bin_long_rows.as<int32_t>(),
                     h->bin_long_first.as<int32_t>(), h->bin_chunks.as<int4>(), s));
  CK(cudaStreamSynchronize(s));
  h->bin_n_med = tot[0];
  h->bin_n_long = tot[1];
  h->bin_n_chunks = tot[2];
  h->has_bins = true;
}

// Geometry of the thread-per-row kernel. A staged tile holds the values and columns of
// `rows` consecutive rows; the staged capacity is the matrix's largest such tile, capped by
// the shared-memory budget of one stage (48 KB for one tile per CTA, 56 KB per stage for
// the persistent two-stage kernel). Tiles above the cap are computed from global memory.
// staged-tile alignment of the variant's column representation
int tile_align(const spmv_matrix *h, const spmv_variant &v) {
  return v.index == 1 ? stage_align_bits(h->delta_bits) : 8;
}

int32_t max_tile_elems(spmv_matrix *h, int rows, int align, cudaStream_t s) {
  CK(launch_tile_max(h->n_rows, h->rowptr.as<int32_t>(), rows, align, h->small.as<int32_t>(), s));
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

void set_tile_geometry(spmv_matrix *h, const spmv_variant &v, int rows, bool pipe,
                       cudaStream_t s) {
  h->tile_rows = rows;
  h->tile_pipe = pipe ? 1 : 0;
  h->tile_cap = std::min(max_tile_elems(h, rows, tile_align(h, v), s), tile_limit(h, v, pipe));
}

// Default geometry: the largest of 128, 64, 32 rows per tile whose largest tile fits one
// 48 KB stage, one tile per CTA; 128-row tiles when none fits.
void compute_tile_cap(spmv_matrix *h, const spmv_variant &v, cudaStream_t s) {
  const int32_t limit = tile_limit(h, v, false);
  for (int rows = kTileRows; rows >= 32; rows /= 2) {
    const int32_t m = max_tile_elems(h, rows, tile_align(h, v), s);
    if (m <= limit) {
      h->tile_rows = rows;
      h->tile_pipe = 0;
      h->tile_cap = m;
      return;
    }
  }
  set_tile_geometry(h, v, kTileRows, false, s);
}

void prepare_variant(spmv_matrix *h, spmv_variant &v, cudaStream_t s) {
  if (v.partition == 1) {
    v.index = 0;                 // the delta index is built for sub-warp rows only
    build_merge(h, s);
  } else if (v.partition == 2) {
    if (v.index == 1) build_delta(h, s);
    v.vec = 1;
    if (v.vs != 2 && v.vs != 4 && v.vs != 8) v.vs = 4;   // short rows' sub-warp width
    v.tile_rows = 0;
    v.tile_pipe = 0;
    h->bin_vs_short = v.vs;
    build_bins(h, s);
  } else {
    if (v.index == 1) {
      v.vec = 1;
      build_delta(h, s);
    }
    if (v.vs == 0) {
      v.vs = (v.vec || v.index == 1) ? pool_vs(h->nnz_avg(), v.index == 1 ? 8 : 4)
                                     : heuristic_vs(h->nnz_avg(), 1);
    }
    if (h->storage == SPMV_DF64) v.tile_pipe = 0;   // the double-float kernel: one tile per CTA
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
  if (v.partition < 0 || v.partition > 2) return false;
  if (v.partition == 2 && v.vs != 0 && v.vs != 2 && v.vs != 4 && v.vs != 8) return false;
  if (v.index != 0 && v.index != 1) return false;
  if (v.xpath != 0 && v.xpath != 1) return false;
  if (v.vec != 0 && v.vec != 1) return false;
  if (v.partition == 0 && v.vs != 0 && v.vs != 1 && v.vs != 2 && v.vs != 4 && v.vs != 8 &&
      v.vs != 16 && v.vs != 32)
    return false;
  if (v.tile_rows != 0 && v.tile_rows != 32 && v.tile_rows != 64 && v.tile_rows != 128)
    return false;
  if (v.tile_pipe != 0 && v.tile_pipe != 1) return false;
  return true;
}

cudaError_t launch_run(const spmv_matrix *h, const spmv_variant &v, const void *x, void *y,
                       cudaStream_t s) {
  const KernelSet *ks = set_for(h);
  RunArgs a = run_args(h, x, y);
  return ks->spmv(v, a, s);
}

// Average milliseconds per launch of fn over reps launches (after 2 warm-up launches).
template <typename F> float time_launches(F fn, int reps, cudaStream_t s) {
  for (int i = 0; i < 2; ++i) CK(fn());
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  for (int i = 0; i < reps; ++i) CK(fn());
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / (float)reps;
}

// ------------------------------------------------------------------ bandwidth --------
void probe_bandwidth(int dev, double *hbm, double *l2) {
  DeviceInfo &d = device_info(dev);
  {
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (d.bw_done) {
      *hbm = d.hbm_gbs;
      *l2 = d.l2_gbs;
      return;
    }
  }
  cudaStream_t s;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  DevBuf big, small, sink;
  const int64_t big_bytes = (int64_t)2 << 30;
  int64_t small_bytes = d.l2_bytes / 4;
  if (small_bytes < (1 << 20)) small_bytes = 1 << 20;
  small_bytes &= ~(int64_t)15;
  big.alloc((size_t)big_bytes, 1, s, true);
  small.alloc((size_t)small_bytes, 1, s, true);
  sink.alloc(8, 8, s, true);
  auto fb = [&]() { return launch_read_probe(big.p, big_bytes, 1, sink.as<unsigned long long>(), s); };
  const int l2_reps = 64;
  auto fs = [&]() {
    return launch_read_probe(small.p, small_bytes, l2_reps, sink.as<unsigned long long>(), s);
  };
  float tb = 1e30f, ts = 1e30f;
  for (int r = 0; r < 3; ++r) {
    tb = std::min(tb, time_launches(fb, 3, s));
    ts = std::min(ts, time_launches(fs, 3, s));
  }
  cudaStreamSynchronize(s);
  big.release();
  small.release();
  sink.release();
  cudaStreamDestroy(s);
  std::lock_guard<std::mutex> lk(g_dev_mu);
  d.hbm_gbs = (double)big_bytes / (tb * 1e-3) / 1e9;
  d.l2_gbs = (double)small_bytes * l2_reps / (ts * 1e-3) / 1e9;
  d.bw_done = true;
  *hbm = d.hbm_gbs;
  *l2 = d.l2_gbs;
}

// --------------------------------------------------------------- bounds & rules ------
void bounds(int64_t n_rows, int64_t n_cols, int64_t nnz, int idx_b, int val_b, int vec_b,
            double b_max, double *out) {
  const double s_format = 4.0 * (double)(n_rows + 1) + (double)(idx_b + val_b) * (double)nnz;
  const double s_xy = (double)vec_b * (double)n_cols + (double)vec_b * (double)n_rows;
  const double s_values = (double)val_b * (double)nnz;
  const double flops = 2.0 * (double)nnz;
  out[0] = flops / ((s_format + s_xy) / b_max);
  out[1] = flops / ((s_values + s_xy) / b_max);
  out[2] = s_format + s_xy;
}

uint32_t classify(const double *p, double t_imb, double t_ml, double t_mb) {
  const double p_csr = p[0], p_mb = p[1], p_ml = p[2], p_imb = p[3], p_cmp = p[4], p_peak = p[5];
  uint32_t c = 0;
  if (p_imb / p_csr > t_imb) c |= SPMV_CLASS_IMB;
  if (p_ml / p_csr > t_ml) c |= SPMV_CLASS_ML;
  if (p_csr / p_mb >= t_mb && p_mb < p_cmp && p_cmp < p_peak) c |= SPMV_CLASS_MB;
  if (p_mb > p_cmp || p_cmp > p_peak) c |= SPMV_CLASS_CMP;
  return c;
}

// Second profiling pass (GB300 reading of Section III-C): when the baseline is compute
// bound (CMP), the compute bottleneck hides the memory ones. After the CMP optimization
// (one FMA per nonzero) the profile is repeated with that kernel as the baseline:
// p2 = {P_CSR', P_ML'}; ML if P_ML' / P_CSR' > t_ml, MB if P_CSR' / P_MB >= t_mb.
uint32_t classify2(const double *p, const double *p2, double t_imb, double t_ml, double t_mb) {
  uint32_t c = classify(p, t_imb, t_ml, t_mb);
  if (p2 && (c & SPMV_CLASS_CMP) && p2[0] > 0.0) {
    if (p2[1] / p2[0] > t_ml) c |= SPMV_CLASS_ML;
    if (p2[0] / p[1] >= t_mb) c |= SPMV_CLASS_MB;
  }
  return c;
}

spmv_variant variant_for_classes(uint32_t cls, double nnz_avg, double nnz_max, double long_ratio) {
  spmv_variant v{};
  if ((cls & SPMV_CLASS_IMB) && nnz_max > long_ratio * nnz_avg) v.partition = 1;
  if (cls & SPMV_CLASS_MB) v.index = 1;   // merge-path tiles keep int32 columns
  if (cls & SPMV_CLASS_ML) v.xpath = 1;
  if (cls & (SPMV_CLASS_MB | SPMV_CLASS_CMP)) v.vec = 1;
  v.vs = 0;
  return v;
}

// Feature route (Section III-D) with fixed rules in place of a trained tree:
//   IMB  highly uneven rows: nnz_max > long_ratio * nnz_avg;
//   ML   most elements start a new cache line (misses_avg >= nnz_avg / 2) and x does not
//        fit in half of L2;
//   CMP  the working set fits in L2 (size = 1) or rows are very short (nnz_avg < 4);
//   MB   none of the above and the working set exceeds L2.
uint32_t feature_rules(const double *f, int64_t n_cols, int vec_bytes, int64_t l2_bytes,
                       double long_ratio) {
  const double size = f[0], nnz_max = f[3], nnz_avg = f[4], misses_avg = f[13];
  uint32_t c = 0;
  if (nnz_avg > 0.0 && nnz_max > long_ratio * nnz_avg) c |= SPMV_CLASS_IMB;
  if (misses_avg >= 0.5 * nnz_avg && (double)vec_bytes * (double)n_cols > 0.5 * (double)l2_bytes)
    c |= SPMV_CLASS_ML;
  if (size != 0.0 || nnz_avg < 4.0) c |= SPMV_CLASS_CMP;
  if (c == 0 && size == 0.0) c |= SPMV_CLASS_MB;
  return c;
}

// ------------------------------------------------------------------ features ---------
double finalize_sd(u128 s1, u128 s2, int64_t n, double scale) {
  const u128 nn = (u128)(uint64_t)n;
  const u128 num = nn * s2 - s1 * s1;
  const double var = (double)num / ((double)n * (double)n);
  return std::sqrt(var) * scale;
}

void compute_features(spmv_matrix *h, int line_bytes, double *out, uint64_t *isum,
                      cudaStream_t s) {
  const int line_elems = std::max(1, line_bytes / (int)dtype_bytes(h->vec));
  const int nb = feature_blocks(h->n_rows);
  if (!h->feat_part.p) {
    h->feat_part.alloc(sizeof(FeatSums) * (size_t)nb, 8, s);
    h->feat_fin.alloc(sizeof(FeatSums), 8, s);
  }
  CK(launch_features(h->n_rows, h->rowptr.as<int32_t>(), h->colind.as<int32_t>(), line_elems,
                     h->feat_part.as<FeatSums>(), nb, h->feat_fin.as<FeatSums>(), s));
  FeatSums fs;
  CK(cudaMemcpyAsync(&fs, h->feat_fin.p, sizeof fs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int64_t n = h->n_rows;
  const u128 s_nnz = fs.s_nnz, s_nnz2 = ((u128)fs.s_nnz2_hi << 64) | fs.s_nnz2_lo;
  const u128 s_bw = ((u128)fs.s_bw_hi << 64) | fs.s_bw_lo;
  const u128 s_bw2 = ((u128)fs.s_bw2_hi << 64) | fs.s_bw2_lo;
  const u128 s_sc = fs.s_sc, s_sc2 = ((u128)fs.s_sc2_hi << 64) | fs.s_sc2_lo;
  const u128 s_cl = fs.s_cl;
  const int64_t vb = (int64_t)dtype_bytes(h->vec);
  const int64_t ws = 4 * (h->n_rows + 1) +
                     (4 + (int64_t)dtype_bytes(h->storage)) * h->nnz + vb * (h->n_rows + h->n_cols);
  const DeviceInfo &d = device_info(h->device);
  const double N = (double)n;
  const double q = 1.0 / 16777216.0;
  long long nnz_min = fs.nnz_min, nnz_max = fs.nnz_max, bw_min = fs.bw_min, bw_max = fs.bw_max;
  if (n == 0) nnz_min = nnz_max = bw_min = bw_max = 0;
  out[0] = ws <= d.l2_bytes ? 1.0 : 0.0;
  out[1] = n > 0 && h->n_cols > 0 ? (double)h->nnz / ((double)n * (double)h->n_cols) : 0.0;
  out[2] = (double)nnz_min;
  out[3] = (double)nnz_max;
  out[4] = n ? (double)s_nnz / N : 0.0;
  out[5] = n ? finalize_sd(s_nnz, s_nnz2, n, 1.0) : 0.0;
  out[6] = (double)bw_min;
  out[7] = (double)bw_max;
  out[8] = n ? (double)s_bw / N : 0.0;
  out[9] = n ? finalize_sd(s_bw, s_bw2, n, 1.0) : 0.0;
  out[10] = n ? ((double)s_sc / N) * q : 0.0;
  out[11] = n ? finalize_sd(s_sc, s_sc2, n, q) : 0.0;
  out[12] = n ? ((double)s_cl / N) * q : 0.0;
  out[13] = n ? (double)fs.s_miss / N : 0.0;
  if (isum) {
    isum[0] = (uint64_t)s_nnz;
    isum[1] = (uint64_t)s_bw;
    isum[2] = (uint64_t)s_sc;
    isum[3] = (uint64_t)s_cl;
    isum[4] = fs.s_miss;
    isum[5] = fs.s_grp;
    isum[6] = (uint64_t)nnz_min;
    isum[7] = (uint64_t)nnz_max;
    isum[8] = (uint64_t)bw_min;
    isum[9] = (uint64_t)bw_max;
    isum[10] = fs.s_nnz2_lo;
    isum[11] = fs.s_bw2_lo;
  }
}

// ------------------------------------------------------------------ profiling --------
// The static-partition profiling setup shared by the profile route and its diagnostics:
// a resident grid of n_ctas CTAs over nnz-balanced contiguous row ranges (rows never
// split), the paper's baseline partitioning (Section IV-A) with one CTA per worker.
struct StaticSetup {
  DevBuf part, t0, t1, smid;
  ProfileArgs pa;
};

void static_setup(spmv_matrix *h, StaticSetup &st, const void *x, void *y, cudaStream_t s) {
  const KernelSet *ks = set_for(h);
  DeviceInfo &d = device_info(h->device);
  const int n_ctas = std::max(1, d.sms * ks->profile_blocks_per_sm);
  st.part.alloc(sizeof(int32_t) * (size_t)(n_ctas + 1), 4, s);
  CK(launch_static_partition(h->n_rows, h->nnz, h->rowptr.as<int32_t>(), n_ctas,
                             st.part.as<int32_t>(), s));
  st.t0.alloc(8 * (size_t)n_ctas, 8, s, true);
  st.t1.alloc(8 * (size_t)n_ctas, 8, s, true);
  st.smid.alloc(4 * (size_t)n_ctas, 4, s, true);
  ProfileArgs &pa = st.pa;
  pa.n_rows = h->n_rows;
  pa.n_cols = h->n_cols;
  pa.part = st.part.as<int32_t>();
  pa.n_ctas = n_ctas;
  pa.rowptr = h->rowptr.as<int32_t>();
  pa.colind = h->colind.as<int32_t>();
  pa.val = h->val_ptr();
  pa.x = x;
  pa.y = y;
  pa.t_start = st.t0.as<unsigned long long>();
  pa.t_end = st.t1.as<unsigned long long>();
  pa.smid = st.smid.as<int32_t>();
  pa.vs = heuristic_vs(h->nnz_avg(), 1);
  pa.cmp_mode = 0;
}

// Per-CTA elapsed times (ms) of the last launch; CTAs with an empty row range get -1.
void read_cta_times(const StaticSetup &st, std::vector<double> &el, std::vector<int32_t> &sm,
                    double *span_ms, cudaStream_t s) {
  const int n = st.pa.n_ctas;
  std::vector<unsigned long long> ts((size_t)n), te((size_t)n);
  std::vector<int32_t> hp((size_t)n + 1);
  sm.assign((size_t)n, 0);
  CK(cudaMemcpyAsync(ts.data(), st.t0.p, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(te.data(), st.t1.p, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(sm.data(), st.smid.p, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hp.data(), st.part.p, 4 * ((size_t)n + 1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  el.assign((size_t)n, -1.0);
  unsigned long long tmin = ~0ull, tmax = 0;
  for (int c = 0; c < n; ++c) {
    if (hp[(size_t)c + 1] <= hp[(size_t)c]) continue;   // no rows: no work
    el[(size_t)c] = (double)(te[(size_t)c] - ts[(size_t)c]) * 1e-6;
    tmin = std::min(tmin, ts[(size_t)c]);
    tmax = std::max(tmax, te[(size_t)c]);
  }
  *span_ms = tmax >= tmin ? (double)(tmax - tmin) * 1e-6 : 0.0;
}

// Span (ms) of every SM that ran at least one CTA with rows: last end - first start.
std::vector<double> sm_spans(const StaticSetup &st, cudaStream_t s, double *global_span_ms) {
  const int n = st.pa.n_ctas;
  std::vector<unsigned long long> ts((size_t)n), te((size_t)n);
  std::vector<int32_t> hp((size_t)n + 1), sm((size_t)n);
  CK(cudaMemcpyAsync(ts.data(), st.t0.p, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(te.data(), st.t1.p, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(sm.data(), st.smid.p, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hp.data(), st.part.p, 4 * ((size_t)n + 1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int max_sm = 0;
  for (int c = 0; c < n; ++c) max_sm = std::max(max_sm, sm[(size_t)c]);
  std::vector<unsigned long long> lo((size_t)max_sm + 1, ~0ull), hi((size_t)max_sm + 1, 0);
  unsigned long long gmin = ~0ull, gmax = 0;
  for (int c = 0; c < n; ++c) {
    if (hp[(size_t)c + 1] <= hp[(size_t)c]) continue;
    const size_t k = (size_t)sm[(size_t)c];
    lo[k] = std::min(lo[k], ts[(size_t)c]);
    hi[k] = std::max(hi[k], te[(size_t)c]);
    gmin = std::min(gmin, ts[(size_t)c]);
    gmax = std::max(gmax, te[(size_t)c]);
  }
  std::vector<double> spans;
  for (size_t k = 0; k < lo.size(); ++k)
    if (hi[k] >= lo[k] && lo[k] != ~0ull) spans.push_back((double)(hi[k] - lo[k]) * 1e-6);
  *global_span_ms = gmax >= gmin && gmin != ~0ull ? (double)(gmax - gmin) * 1e-6 : 0.0;
  return spans;
}

void run_profile(spmv_matrix *h, int reps, spmv_profile_report &o, cudaStream_t s,
                 bool second_pass = false) {
  std::memset(&o, 0, sizeof o);
  const KernelSet *ks = set_for(h);
  DeviceInfo &d = device_info(h->device);
  double b_hbm = 0, b_l2 = 0;
  probe_bandwidth(h->device, &b_hbm, &b_l2);
  const size_t vb = dtype_bytes(h->vec);
  DevBuf x, y, colp;
  x.alloc(vb * (size_t)std::max<int64_t>(h->n_cols, 1), vb, s);
  y.alloc(vb * (size_t)std::max<int64_t>(h->n_rows, 1), vb, s);
  CK(launch_fill_const(x.p, h->vec, h->n_cols, 1.0, s));
  StaticSetup st;
  static_setup(h, st, x.p, y.p, s);
  colp.alloc(sizeof(int32_t) * (size_t)h->nnz, 4, s);
  CK(launch_fill_row_index(h->n_rows, h->n_cols, h->rowptr.as<int32_t>(), colp.as<int32_t>(), s));
  ProfileArgs pa = st.pa;
  const double flops = 2.0 * (double)h->nnz;
  // P_CSR, and the per-CTA times of the last timed launch (P_IMB)
  const float t_csr = time_launches([&]() { return ks->profile(pa, s); }, reps, s);
  // A worker of the paper's static partition is an SM: the CTAs resident on one SM share
  // its pipes, so their individual times reflect the warp scheduler's fairness rather than
  // the partition. Each SM's time is the span of its CTAs (first start to last end); the
  // median is taken over SMs.
  double t_span = 0.0;
  std::vector<double> work = sm_spans(st, s, &t_span);
  double t_median = t_csr;
  if (!work.empty()) {
    std::sort(work.begin(), work.end());
    t_median = work[(work.size() - 1) / 2];           // lower median
  } else {
    t_span = t_csr;
  }
  // the median worker time plus the launch cost that no worker sees
  const double t_imb = t_median + std::max(0.0, (double)t_csr - t_span);
  // P_ML: colind'[j] = row of j
  pa.colind = colp.as<int32_t>();
  const float t_ml = time_launches([&]() { return ks->profile(pa, s); }, reps, s);
  // P_CMP: x[i] only, no colind
  pa.colind = h->colind.as<int32_t>();
  pa.cmp_mode = 1;
  const float t_cmp = time_launches([&]() { return ks->profile(pa, s); }, reps, s);
  double bo[3];
  bounds(h->n_rows, h->n_cols, h->nnz, 4, (int)dtype_bytes(h->storage), (int)vb, 1.0, bo);
  const double ws = bo[2];
  o.b_max_gbs = ws <= (double)d.l2_bytes ? b_l2 : b_hbm;
  bounds(h->n_rows, h->n_cols, h->nnz, 4, (int)dtype_bytes(h->storage), (int)vb, o.b_max_gbs, bo);
  auto gf = [&](double ms) { return ms > 0 ? flops / (ms * 1e-3) / 1e9 : 0.0; };
  o.p[0] = gf(t_csr);
  o.p[1] = bo[0];
  o.p[2] = gf(t_ml);
  o.p[3] = gf(t_imb);
  o.p[4] = gf(t_cmp);
  o.p[5] = bo[1];
  o.b_hbm_gbs = b_hbm;
  o.b_l2_gbs = b_l2;
  o.t_csr_ms = t_csr;
  o.t_ml_ms = t_ml;
  o.t_cmp_ms = t_cmp;
  o.t_median_ms = t_median;
  o.t_span_ms = t_span;
  o.t_imb_ms = t_imb;
  o.n_ctas = st.pa.n_ctas;
  o.vs = st.pa.vs;
  if (second_pass && h->n_rows > 0) {
    // the CMP optimization as the new baseline: thread-per-row tiles, int32 columns
    spmv_variant v2{};
    v2.vec = 1;
    v2.vs = 1;
    compute_tile_cap(h, v2, s);
    const float t2 = time_launches([&]() { return launch_run(h, v2, x.p, y.p, s); }, reps, s);
    RunArgs a2 = run_args(h, x.p, y.p);
    a2.colind = colp.as<int32_t>();
    const KernelSet *k2 = set_for(h);
    const float t2ml = time_launches([&]() { return k2->spmv(v2, a2, s); }, reps, s);
    o.p2[0] = gf(t2);
    o.p2[1] = gf(t2ml);
  }
}

// Sub-warp width sweep by timing (Section III-E "parameter tuning"; build addition). When
// the thread-per-row kernel (width 1) wins, its geometry is swept too: 128 / 64 / 32 rows
// per tile, one tile per CTA or persistent CTAs with two tiles in flight.
// Called by spmv_tune for the routes that choose a variant (never for SPMV_TUNE_FIXED), so
// the sub-warp width and, for width 1, the tile geometry are always swept.
void autotune_vs(spmv_matrix *h, spmv_variant &v, int reps, cudaStream_t s) {
  if (h->n_rows == 0) return;
  const size_t vb = dtype_bytes(h->vec);
  DevBuf x, y;
  x.alloc(vb * (size_t)std::max<int64_t>(h->n_cols, 1), vb, s);
  y.alloc(vb * (size_t)std::max<int64_t>(h->n_rows, 1), vb, s);
  CK(launch_fill_const(x.p, h->vec, h->n_cols, 1.0, s));
  if (v.partition != 0) {
    // IMB's decomposition family: merge-path tiles, or the row decomposition with short
    // rows on sub-warps of 2, 4 or 8 lanes; the fastest is kept
    spmv_variant best_v = v;
    float best_t = 1e30f;
    const int cand[4][2] = {{1, 0}, {2, 2}, {2, 4}, {2, 8}};
    for (const auto &c : cand) {
      spmv_variant t = v;
      t.partition = c[0];
      t.vs = c[1];
      prepare_variant(h, t, s);
      const float ms = time_launches([&]() { return launch_run(h, t, x.p, y.p, s); }, reps, s);
      if (ms < best_t) {
        best_t = ms;
        best_v = t;
      }
    }
    v = best_v;
    prepare_variant(h, v, s);
    return;
  }
  float best = 1e30f;
  int best_vs = v.vs;
  const int widths[6] = {1, 2, 4, 8, 16, 32};
  compute_tile_cap(h, v, s);
  for (int w : widths) {
    spmv_variant t = v;
    t.vs = w;
    const float ms = time_launches([&]() { return launch_run(h, t, x.p, y.p, s); }, reps, s);
    if (ms < best) {
      best = ms;
      best_vs = w;
    }
  }
  v.vs = best_vs;
  if (best_vs != 1) {
    v.tile_rows = 0;
    v.tile_pipe = 0;
    return;
  }
  int best_rows = h->tile_rows, best_pipe = h->tile_pipe, best_cap = h->tile_cap;
  const int max_pipe = h->storage == SPMV_DF64 ? 0 : 1;
  for (int pipe = 0; pipe <= max_pipe; ++pipe) {
    for (int rows = kTileRows; rows >= 32; rows /= 2) {
      set_tile_geometry(h, v, rows, pipe != 0, s);
      const float ms = time_launches([&]() { return launch_run(h, v, x.p, y.p, s); }, reps, s);
      if (ms < best) {
        best = ms;
        best_rows = rows;
        best_pipe = pipe;
        best_cap = h->tile_cap;
      }
    }
  }
  h->tile_rows = best_rows;
  h->tile_pipe = best_pipe;
  h->tile_cap = best_cap;
  v.tile_rows = best_rows;
  v.tile_pipe = best_pipe;
}

bool combo_offered(spmv_dtype storage, spmv_dtype vec, spmv_dtype acc) {
  return kernel_set(storage, vec, acc) != nullptr;
}

void default_types(spmv_dtype in, spmv_dtype *st, spmv_dtype *vec, spmv_dtype *acc) {
  *st = in;
  if (in == SPMV_F64) {
    *vec = SPMV_F64;
    *acc = SPMV_F64;
  } else {
    *vec = SPMV_F32;
    *acc = SPMV_F32;
  }
}

void install_storage(spmv_matrix *h, cudaStream_t s) {
  h->val_store.release();
  h->val_df.release();
  if (h->storage == SPMV_DF64) {
    // the FP64 input values stay the values of every non-double-float kernel
    h->val_df.alloc(8 * (size_t)h->nnz, 8, s);
    CK(launch_df_split(h->val_in.as<double>(), h->val_df.p, 0, h->nnz, s));
  } else if (h->storage != h->in_type) {
    const size_t eb = dtype_bytes(h->storage);
    h->val_store.alloc(eb * (size_t)h->nnz, eb, s);
    CK(launch_convert_values(h->val_in.p, h->in_type, h->val_store.p, h->storage, h->nnz, s));
  }
}

template <typename F> spmv_status guarded(F fn) {
  try {
    return fn();
  } catch (const CudaFail &f) {
    cudaGetLastError();
    return map_err(f.e);
  } catch (const std::bad_alloc &) {
    return SPMV_ERR_OOM;
  } catch (...) {
    return SPMV_ERR_CUDA;
  }
}

// True for page-locked (pinned or registered) host memory.
bool is_page_locked(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

void drop_host_graph(spmv_matrix *h) {
  if (h->host_exec) cudaGraphExecDestroy(h->host_exec);
  if (h->host_graph) cudaGraphDestroy(h->host_graph);
  h->host_exec = nullptr;
  h->host_graph = nullptr;
  h->host_x = nullptr;
  h->host_y = nullptr;
}

}  // namespace

// ================================================================= C ABI ============
extern "C" {

const char *spmv_status_string(spmv_status s) {
  switch (s) {
    case SPMV_OK: return "ok";
    case SPMV_ERR_INVALID_CSR: return "invalid CSR matrix";
    case SPMV_ERR_UNSUPPORTED_DTYPE: return "unsupported dtype combination";
    case SPMV_ERR_OOM: return "device out of memory";
    case SPMV_ERR_NOT_TUNED: return "handle has no variant installed (call spmv_tune)";
    case SPMV_ERR_CUDA: return "CUDA runtime error";
    case SPMV_ERR_TIMEOUT: return "bounded device wait expired";
    case SPMV_ERR_ARG: return "invalid argument";
    case SPMV_ERR_NO_SELECTOR: return "learned mode needs a selector";
    case SPMV_ERR_TOO_LARGE: return "problem larger than the fixed scratch buffer allows";
  }
  return "unknown status";
}

spmv_status spmv_tune_opts_default(spmv_tune_opts *o) {
  if (!o) return SPMV_ERR_ARG;
  std::memset(o, 0, sizeof *o);
  o->t_imb = 1.24;
  o->t_ml = 1.25;
  o->t_mb = 0.75;
  o->long_row_ratio = 32.0;
  o->autotune = 1;
  o->reps = 8;
  o->second_pass = 1;
  o->min_margin = 0.0;
  return SPMV_OK;
}

spmv_status spmv_create(spmv_handle_t *out, int64_t n_rows, int64_t n_cols, int64_t nnz,
                        const int32_t *row_ptr, const int32_t *col_ind, const void *val,
                        spmv_dtype val_type, int32_t device_ptrs, spmv_stream_t stream) {
  if (!out || !row_ptr || (nnz > 0 && (!col_ind || !val))) return SPMV_ERR_ARG;
  if (n_rows < 0 || n_cols < 0 || nnz < 0 || n_rows >= INT32_MAX || n_cols >= INT32_MAX ||
      nnz >= INT32_MAX)
    return SPMV_ERR_ARG;
  if (!valid_dtype(val_type)) return SPMV_ERR_UNSUPPORTED_DTYPE;
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  spmv_matrix *h = new (std::nothrow) spmv_matrix();
  if (!h) return SPMV_ERR_OOM;
  spmv_status st = guarded([&]() -> spmv_status {
    CK(cudaGetDevice(&h->device));
    device_info(h->device);
    h->n_rows = n_rows;
    h->n_cols = n_cols;
    h->nnz = nnz;
    h->in_type = val_type;
    default_types(val_type, &h->storage, &h->vec, &h->acc);
    const size_t eb = dtype_bytes(val_type);
    h->d_err.alloc(4, 4, s, true);
    h->small.alloc(256, 4, s, true);
    h->rowptr.alloc(4 * (size_t)(n_rows + 1), 4, s);
    h->colind.alloc(4 * (size_t)nnz, 4, s);
    h->val_in.alloc(eb * (size_t)nnz, eb, s);
    const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(h->rowptr.p, row_ptr, 4 * (size_t)(n_rows + 1), kind, s));
    if (nnz > 0) {
      CK(cudaMemcpyAsync(h->colind.p, col_ind, 4 * (size_t)nnz, kind, s));
      CK(cudaMemcpyAsync(h->val_in.p, val, eb * (size_t)nnz, kind, s));
    }
    DevBuf code;
    code.alloc(16, 4, s, true);
    CK(launch_validate(n_rows, n_cols, nnz, h->rowptr.as<int32_t>(), h->colind.as<int32_t>(),
                       code.as<int32_t>(), s));
    int32_t c = 0;
    CK(cudaMemcpyAsync(&c, code.p, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (c != 0) return SPMV_ERR_INVALID_CSR;
    return SPMV_OK;
  });
  if (st != SPMV_OK) {
    spmv_destroy(h);
    return st;
  }
  *out = h;
  return SPMV_OK;
}

spmv_status spmv_destroy(spmv_handle_t h) {
  if (!h) return SPMV_ERR_ARG;
  cudaDeviceSynchronize();
  drop_host_graph(h);
  if (h->copy_stream) {
    for (int c = 0; c < kHostChunks; ++c) {
      if (h->chunk_done[c]) cudaEventDestroy(h->chunk_done[c]);
      if (h->x_ready[c]) cudaEventDestroy(h->x_ready[c]);
    }
    for (auto e : h->joined)
      if (e) cudaEventDestroy(e);
    cudaStreamDestroy(h->copy_stream);
    cudaStreamDestroy(h->upload_stream);
    cudaStreamDestroy(h->capture_stream);
    for (auto st : h->chunk_stream)
      if (st) cudaStreamDestroy(st);
  }
  for (DevBuf *b : {&h->rowptr, &h->colind, &h->val_in, &h->val_store, &h->dbase, &h->delta,
                    &h->esc, &h->coord, &h->tail_row, &h->tail_val, &h->head_val, &h->x_stage,
                    &h->y_stage, &h->scratch, &h->d_err, &h->small, &h->feat_part,
                    &h->feat_fin, &h->val_df, &h->cg_ws, &h->bin_rows, &h->bin_long_rows,
                    &h->bin_long_first, &h->bin_chunks, &h->bin_partials})
    b->release();
  delete h;
  return SPMV_OK;
}

spmv_status spmv_set_precision(spmv_handle_t h, spmv_dtype storage, spmv_dtype vec_type,
                               spmv_dtype acc_type, spmv_stream_t stream) {
  if (!h) return SPMV_ERR_ARG;
  if (!valid_precision_dtype(storage) || !valid_precision_dtype(vec_type) ||
      !valid_precision_dtype(acc_type))
    return SPMV_ERR_UNSUPPORTED_DTYPE;
  if (!combo_offered(storage, vec_type, acc_type)) return SPMV_ERR_UNSUPPORTED_DTYPE;
  if (storage == SPMV_DF64 && h->in_type != SPMV_F64) return SPMV_ERR_UNSUPPORTED_DTYPE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    if (storage != h->storage) {
      h->storage = storage;
      install_storage(h, s);
      CK(cudaStreamSynchronize(s));
    }
    if (vec_type != h->vec) {
      h->x_stage.release();
      h->y_stage.release();
    }
    h->vec = vec_type;
    h->acc = acc_type;
    ++h->epoch;
    h->tuned = false;
    return SPMV_OK;
  });
}

spmv_status spmv_set_variant(spmv_handle_t h, const spmv_variant *v, spmv_stream_t stream) {
  if (!h || !v || !valid_variant(*v)) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    spmv_variant w = *v;
    prepare_variant(h, w, s);
    h->variant = w;
    ++h->epoch;
    h->tuned = true;
    return SPMV_OK;
  });
}

spmv_status spmv_tune(spmv_handle_t h, spmv_mode mode, const spmv_tune_opts *opts_in,
                      spmv_tune_report *report, spmv_stream_t stream) {
  if (!h) return SPMV_ERR_ARG;
  spmv_tune_opts opts;
  if (opts_in) opts = *opts_in;
  else spmv_tune_opts_default(&opts);
  if (opts.reps <= 0) opts.reps = 8;
  if (mode == SPMV_TUNE_LEARNED && !opts.selector) return SPMV_ERR_NO_SELECTOR;
  if (mode < SPMV_TUNE_PROFILE || mode > SPMV_TUNE_FIXED) return SPMV_ERR_ARG;
  if (mode == SPMV_TUNE_FIXED && !valid_variant(opts.fixed)) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  spmv_tune_report rep;
  std::memset(&rep, 0, sizeof rep);
  spmv_status st = guarded([&]() -> spmv_status {
    const double t0 = now_ms();
    uint32_t cls = 0;
    spmv_variant v{};
    int used = mode;
    double nnz_max = -1.0;
    auto need_features = [&]() {
      compute_features(h, 128, rep.features, nullptr, s);
      nnz_max = rep.features[3];
    };
    if (mode == SPMV_TUNE_FIXED) {
      v = opts.fixed;
    } else {
      bool done = false;
      if (mode == SPMV_TUNE_FEATURES) {
        need_features();
        const DeviceInfo &d = device_info(h->device);
        cls = feature_rules(rep.features, h->n_cols, (int)dtype_bytes(h->vec), d.l2_bytes,
                            opts.long_row_ratio);
        done = true;
      } else if (mode == SPMV_TUNE_LEARNED) {
        need_features();
        double f16[16];
        std::memcpy(f16, rep.features, sizeof(double) * 14);
        f16[14] = (double)h->n_rows;
        f16[15] = (double)h->nnz;
        uint32_t c = 0;
        double margin = 0.0;
        spmv_status ps = spmv_selector_predict(opts.selector, f16, &c, &margin, stream);
        if (ps != SPMV_OK) return ps;
        rep.margin = margin;
        if (margin >= opts.min_margin) {
          cls = c;
          done = true;
        } else {
          used = SPMV_TUNE_PROFILE;
        }
      }
      if (!done) {
        spmv_profile_report po;
        run_profile(h, opts.reps, po, s, opts.second_pass != 0);
        std::memcpy(rep.p, po.p, sizeof po.p);
        std::memcpy(rep.p2, po.p2, sizeof po.p2);
        rep.b_max_gbs = po.b_max_gbs;
        cls = classify2(po.p, opts.second_pass ? po.p2 : nullptr, opts.t_imb, opts.t_ml,
                        opts.t_mb);
        if (nnz_max < 0) {
          CK(launch_row_len_max(h->n_rows, h->rowptr.as<int32_t>(), h->small.as<int32_t>(), s));
          int32_t m = 0;
          CK(cudaMemcpyAsync(&m, h->small.p, 4, cudaMemcpyDeviceToHost, s));
          CK(cudaStreamSynchronize(s));
          nnz_max = (double)m;
        }
      }
      v = variant_for_classes(cls, h->nnz_avg(), nnz_max, opts.long_row_ratio);
    }
    const double t1 = now_ms();
    prepare_variant(h, v, s);
    CK(cudaStreamSynchronize(s));
    const double t2 = now_ms();
    if (opts.autotune && mode != SPMV_TUNE_FIXED) autotune_vs(h, v, std::max(3, opts.reps / 2), s);
    CK(cudaStreamSynchronize(s));
    const double t3 = now_ms();
    h->variant = v;
    ++h->epoch;
    h->tuned = true;
    rep.classes = cls;
    rep.mode_used = used;
    rep.variant = v;
    rep.t_classify_ms = t1 - t0;
    rep.t_prep_ms = t2 - t1;
    rep.t_autotune_ms = t3 - t2;

    rep.t_pre_ms = t3 - t0;
    return SPMV_OK;
  });
  if (st == SPMV_OK && report) *report = rep;
  return st;
}

spmv_status spmv_run(spmv_handle_t h, const void *x, void *y, spmv_stream_t stream) {
  if (!h) return SPMV_ERR_ARG;
  if (!h->tuned) return SPMV_ERR_NOT_TUNED;
  if ((h->n_cols > 0 && !x) || (h->n_rows > 0 && !y)) return SPMV_ERR_ARG;
  const cudaError_t e = launch_run(h, h->variant, x, y, static_cast<cudaStream_t>(stream));
  return map_err(e);
}

spmv_status spmv_run_host(spmv_handle_t h, const void *x_host, void *y_host,
                          spmv_stream_t stream) {
  if (!h) return SPMV_ERR_ARG;
  if (!h->tuned) return SPMV_ERR_NOT_TUNED;
  if ((h->n_cols > 0 && !x_host) || (h->n_rows > 0 && !y_host)) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    const size_t vb = dtype_bytes(h->vec);
    if (!h->x_stage.p) h->x_stage.alloc(vb * (size_t)std::max<int64_t>(h->n_cols, 1), vb, s);
    if (!h->y_stage.p) h->y_stage.alloc(vb * (size_t)std::max<int64_t>(h->n_rows, 1), vb, s);
    if (!h->copy_stream) {
      CK(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
      CK(cudaStreamCreateWithFlags(&h->upload_stream, cudaStreamNonBlocking));
      CK(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
      for (auto &st : h->chunk_stream) CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      for (int c = 0; c < kHostChunks; ++c) {
        CK(cudaEventCreateWithFlags(&h->chunk_done[c], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->x_ready[c], cudaEventDisableTiming));
      }
      for (auto &e : h->joined) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    // pipelining pays once the copies take longer than a few chunk launches (x and y of at
    // least 8 MB together)
    const bool chunked = h->variant.partition == 0 && h->n_rows >= 4 * kHostChunks * kTileRows &&
                         (int64_t)vb * (h->n_rows + h->n_cols) >= 8000000;
    const int nch = chunked ? kHostChunks : 1;
    // chunk row boundaries: equal parts aligned to 128 rows
    int64_t per = (h->n_rows + nch - 1) / nch;
    per = ((per + kTileRows - 1) / kTileRows) * kTileRows;
    int64_t bounds[kHostChunks + 1];
    for (int c = 0; c < nch; ++c) bounds[c] = std::min<int64_t>(h->n_rows, (int64_t)c * per);
    bounds[nch] = h->n_rows;
    if (chunked && !h->x_need_valid) {
      DevBuf db;
      db.alloc(sizeof(bounds), 8, s);
      CK(cudaMemcpyAsync(db.p, bounds, sizeof(bounds), cudaMemcpyHostToDevice, s));
      CK(launch_chunk_colmax(h->n_rows, h->rowptr.as<int32_t>(), h->colind.as<int32_t>(),
                             db.as<int64_t>(), nch, h->small.as<int32_t>(), s));
      int32_t cm[kHostChunks];
      CK(cudaMemcpyAsync(cm, h->small.p, sizeof(int32_t) * nch, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      int64_t run = 0;
      for (int c = 0; c < nch; ++c) {
        run = std::max<int64_t>(run, (int64_t)cm[c] + 1);
        h->x_need[c] = std::min<int64_t>(run, h->n_cols);
      }
      h->x_need_valid = true;
    }
    // Row kernels compute any row range on their own (row pointers are absolute), so rows go
    // in chunks aligned to 128-row tiles. Chunk c reads x only up to the largest column of
    // chunks 0..c, so x is uploaded in matching pieces on one stream, each chunk waits for
    // its piece, and each finished chunk of y is downloaded on another stream. Consecutive
    // chunks' kernels go to two alternating streams, so one chunk's last partial wave of CTAs
    // overlaps the next chunk's first; all side streams join back into `origin` at the end.
    // Merge-path tiles span the whole matrix: one upload, one launch, one download.
    const KernelSet *ks = set_for(h);
    auto enqueue = [&](cudaStream_t origin) {
      cudaStream_t side[4] = {h->upload_stream, h->copy_stream, h->chunk_stream[0],
                              h->chunk_stream[1]};
      CK(cudaEventRecord(h->joined[4], origin));
      for (cudaStream_t st : side) CK(cudaStreamWaitEvent(st, h->joined[4], 0));
      int64_t uploaded = 0;
      for (int c = 0; c < nch; ++c) {
        const int64_t need = chunked ? h->x_need[c] : h->n_cols;
        if (need > uploaded) {
          CK(cudaMemcpyAsync(static_cast<char *>(h->x_stage.p) + vb * (size_t)uploaded,
                             static_cast<const char *>(x_host) + vb * (size_t)uploaded,
                             vb * (size_t)(need - uploaded), cudaMemcpyHostToDevice,
                             h->upload_stream));
          uploaded = need;
        }
        CK(cudaEventRecord(h->x_ready[c], h->upload_stream));
        cudaStream_t cs = h->chunk_stream[c & 1];
        CK(cudaStreamWaitEvent(cs, h->x_ready[c], 0));
        const int64_t r0 = bounds[c], r1 = bounds[c + 1];
        if (r1 <= r0) continue;
        if (nch == 1) {
          CK(launch_run(h, h->variant, h->x_stage.p, h->y_stage.p, cs));
        } else {
          RunArgs a = run_args(h, h->x_stage.p, static_cast<char *>(h->y_stage.p) + vb * (size_t)r0);
          a.n_rows = r1 - r0;
          a.rowptr += r0;
          if (a.dbase) a.dbase += r0;
          CK(ks->spmv(h->variant, a, cs));
        }
        CK(cudaEventRecord(h->chunk_done[c], cs));
        CK(cudaStreamWaitEvent(h->copy_stream, h->chunk_done[c], 0));
        CK(cudaMemcpyAsync(static_cast<char *>(y_host) + vb * (size_t)r0,
                           static_cast<char *>(h->y_stage.p) + vb * (size_t)r0,
                           vb * (size_t)(r1 - r0), cudaMemcpyDeviceToHost, h->copy_stream));
      }
      for (int k = 0; k < 4; ++k) {
        CK(cudaEventRecord(h->joined[k], side[k]));
        CK(cudaStreamWaitEvent(origin, h->joined[k], 0));
      }
    };
    if (is_page_locked(x_host) && is_page_locked(y_host)) {
      // Page-locked buffers: the whole pipeline (uploads, chunk kernels, downloads and the
      // events between the three streams) is captured once into a CUDA graph per pair of
      // host buffers and tuning state, then replayed with one launch per call.
      if (!h->host_exec || h->host_x != x_host || h->host_y != y_host ||
          h->host_epoch != h->epoch) {
        drop_host_graph(h);
        CK(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeRelaxed));
        try {
          enqueue(h->capture_stream);
        } catch (...) {
          cudaGraph_t g = nullptr;
          cudaStreamEndCapture(h->capture_stream, &g);
          if (g) cudaGraphDestroy(g);
          throw;
        }
        CK(cudaStreamEndCapture(h->capture_stream, &h->host_graph));
        CK(cudaGraphInstantiate(&h->host_exec, h->host_graph, 0));
        h->host_x = x_host;
        h->host_y = y_host;
        h->host_epoch = h->epoch;
      }
      CK(cudaGraphLaunch(h->host_exec, s));
    } else {
      enqueue(s);
    }
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
  });
}

spmv_status spmv_cg(spmv_handle_t h, const double *b, double *x, int32_t max_iters,
                    double rtol, int32_t check_every, double *res_hist,
                    spmv_cg_report *report, spmv_stream_t stream) {
  if (!h || max_iters < 0 || !(rtol >= 0.0) || check_every < 1) return SPMV_ERR_ARG;
  if (!h->tuned) return SPMV_ERR_NOT_TUNED;
  if (h->n_rows != h->n_cols) return SPMV_ERR_ARG;
  if (h->vec != SPMV_F64) return SPMV_ERR_UNSUPPORTED_DTYPE;
  if (h->n_rows > 0 && (!b || !x)) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    const double t0 = now_ms();
    const int64_t n = h->n_rows;
    const int nb = cg_reduce_blocks();
    const size_t vec_bytes = ((8 * (size_t)std::max<int64_t>(n, 1) + 255) / 256) * 256;
    const size_t need = 3 * vec_bytes + 8 * (size_t)nb + 8 * 8;
    if (h->cg_ws.bytes < need) h->cg_ws.alloc(need, 8, s);
    char *w = static_cast<char *>(h->cg_ws.p);
    double *r = reinterpret_cast<double *>(w);
    double *p = reinterpret_cast<double *>(w + vec_bytes);
    double *ap = reinterpret_cast<double *>(w + 2 * vec_bytes);
    double *part = reinterpret_cast<double *>(w + 3 * vec_bytes);
    double *sc = part + nb;   // sc[0], sc[1]: (r, r) of even / odd iterations; sc[2]: (p, Ap);
                              // sc[3]: (b, b)
    // r_0 = b - A x_0, p_0 = r_0
    CK(launch_run(h, h->variant, x, ap, s));
    CK(launch_cg_start(b, ap, r, p, n, part, sc, res_hist, s));
    CK(launch_dot(b, b, n, part, sc + 3, nullptr, s));
    double host_sc[4];
    CK(cudaMemcpyAsync(host_sc, sc, sizeof host_sc, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double b_norm = std::sqrt(host_sc[3]);
    double res = std::sqrt(host_sc[0]);
    bool conv = res <= rtol * b_norm;
    int32_t k = 0;
    while (!conv && k < max_iters) {
      const int32_t chunk = std::min(check_every, max_iters - k);
      for (int32_t j = 0; j < chunk; ++j, ++k) {
        double *rr = sc + (k & 1), *rr_new = sc + ((k + 1) & 1);
        CK(launch_run(h, h->variant, p, ap, s));
        CK(launch_dot(p, ap, n, part, sc + 2, nullptr, s));
        CK(launch_cg_xr(p, ap, x, r, n, rr, sc + 2, part, rr_new,
                        res_hist ? res_hist + k + 1 : nullptr, s));
        CK(launch_cg_p(r, p, n, rr, rr_new, s));
      }
      double rr_host = 0.0;
      CK(cudaMemcpyAsync(&rr_host, sc + (k & 1), sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      res = std::sqrt(rr_host);
      conv = res <= rtol * b_norm;
    }
    CK(cudaStreamSynchronize(s));
    if (report) {
      report->iters = k;
      report->converged = conv ? 1 : 0;
      report->res_norm = res;
      report->b_norm = b_norm;
      report->t_ms = now_ms() - t0;
    }
    return SPMV_OK;
  });
}

spmv_status spmv_run_spmm(spmv_handle_t h, const void *X, void *Y, int32_t k,
                          spmv_stream_t stream) {
  if (!h || k < 1) return SPMV_ERR_ARG;
  if (!h->tuned) return SPMV_ERR_NOT_TUNED;
  if ((h->n_cols > 0 && !X) || (h->n_rows > 0 && !Y)) return SPMV_ERR_ARG;
  const KernelSet *ks = set_for(h);
  RunArgs a = run_args(h, X, Y);
  a.k = k;
  const int vs = heuristic_vs(h->nnz_avg(), 1);
  return map_err(ks->spmm(a, vs, static_cast<cudaStream_t>(stream)));
}

spmv_status spmv_export_csr(spmv_handle_t h, int32_t *row_ptr, int32_t *col_ind, void *val,
                            spmv_stream_t stream) {
  if (!h || !row_ptr || (h->nnz > 0 && (!col_ind || !val))) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    CK(cudaMemcpyAsync(row_ptr, h->rowptr.p, 4 * (size_t)(h->n_rows + 1), cudaMemcpyDeviceToDevice, s));
    if (h->nnz > 0) {
      if (h->tuned && h->variant.partition != 1 && h->variant.index == 1 && h->has_delta) {
        CK(launch_delta_decode(h->delta_bits, h->n_rows, h->rowptr.as<int32_t>(),
                               h->dbase.as<int32_t>(), h->delta.p, h->esc.as<int32_t>(), col_ind,
                               s));
      } else {
        CK(cudaMemcpyAsync(col_ind, h->colind.p, 4 * (size_t)h->nnz, cudaMemcpyDeviceToDevice, s));
      }
      CK(cudaMemcpyAsync(val, h->val_ptr(), dtype_bytes(h->storage) * (size_t)h->nnz,
                         cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
  });
}

spmv_status spmv_get_delta(spmv_handle_t h, int32_t *base, void *delta, int32_t *esc_col,
                           int64_t *n_esc, int32_t *bits, spmv_stream_t stream) {
  if (!h || !n_esc || !bits) return SPMV_ERR_ARG;
  if (!h->has_delta) return SPMV_ERR_NOT_TUNED;
  *n_esc = h->n_esc;
  *bits = h->delta_bits;
  if (!esc_col && !base && !delta) return SPMV_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    if (base) CK(cudaMemcpyAsync(base, h->dbase.p, 4 * (size_t)h->n_rows, cudaMemcpyDeviceToDevice, s));
    if (delta && h->nnz)
      CK(cudaMemcpyAsync(delta, h->delta.p, (size_t)(h->delta_bits / 8) * (size_t)h->nnz,
                         cudaMemcpyDeviceToDevice, s));
    if (esc_col && h->n_esc)
      CK(cudaMemcpyAsync(esc_col, h->esc.p, 4 * (size_t)h->n_esc, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
  });
}

spmv_status spmv_get_row_bins(spmv_handle_t h, int32_t *med_rows, int32_t *long_rows,
                              int32_t *long_first, int32_t *chunks, int64_t *counts,
                              spmv_stream_t stream) {
  if (!h || !counts) return SPMV_ERR_ARG;
  if (!h->has_bins) return SPMV_ERR_NOT_TUNED;
  counts[0] = h->bin_n_med;
  counts[1] = h->bin_n_long;
  counts[2] = h->bin_n_chunks;
  if (!med_rows) return SPMV_OK;
  if (!long_rows || !long_first || !chunks) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    CK(cudaMemcpyAsync(med_rows, h->bin_rows.p, 4 * (size_t)h->bin_n_med, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(long_rows, h->bin_long_rows.p, 4 * (size_t)h->bin_n_long, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(long_first, h->bin_long_first.p, 4 * (size_t)(h->bin_n_long + 1),
                       cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(chunks, h->bin_chunks.p, 16 * (size_t)h->bin_n_chunks, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
  });
}

spmv_status spmv_get_merge_path(spmv_handle_t h, int32_t *coord, int64_t *n_tiles,
                                int64_t *items_per_tile, spmv_stream_t stream) {
  if (!h || !n_tiles || !items_per_tile) return SPMV_ERR_ARG;
  if (!h->has_merge) return SPMV_ERR_NOT_TUNED;
  *n_tiles = h->n_tiles;
  *items_per_tile = kMergeItems;
  if (!coord) return SPMV_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    CK(cudaMemcpyAsync(coord, h->coord.p, 8 * (size_t)(h->n_tiles + 1), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
  });
}

spmv_status spmv_features(spmv_handle_t h, int32_t line_bytes, double *features, uint64_t *isum,
                          spmv_stream_t stream) {
  if (!h || !features || line_bytes <= 0) return SPMV_ERR_ARG;
  return guarded([&]() -> spmv_status {
    compute_features(h, line_bytes, features, isum, static_cast<cudaStream_t>(stream));
    return SPMV_OK;
  });
}

spmv_status spmv_profile(spmv_handle_t h, int32_t reps, spmv_profile_report *out,
                         spmv_stream_t stream) {
  if (!h || !out) return SPMV_ERR_ARG;
  return guarded([&]() -> spmv_status {
    spmv_profile_report o;
    run_profile(h, reps > 0 ? reps : 20, o, static_cast<cudaStream_t>(stream), true);
    *out = o;
    return SPMV_OK;
  });
}

spmv_status spmv_profile_cta_times(spmv_handle_t h, double *elapsed_ms, int32_t *sm_id,
                                   int32_t *n_ctas, spmv_stream_t stream) {
  if (!h || !n_ctas) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    const KernelSet *ks = set_for(h);
    const int n = std::max(1, device_info(h->device).sms * ks->profile_blocks_per_sm);
    if (!elapsed_ms && !sm_id) {
      *n_ctas = n;
      return SPMV_OK;
    }
    if (*n_ctas < n) return SPMV_ERR_ARG;
    const size_t vb = dtype_bytes(h->vec);
    DevBuf x, y;
    x.alloc(vb * (size_t)std::max<int64_t>(h->n_cols, 1), vb, s);
    y.alloc(vb * (size_t)std::max<int64_t>(h->n_rows, 1), vb, s);
    CK(launch_fill_const(x.p, h->vec, h->n_cols, 1.0, s));
    StaticSetup st;
    static_setup(h, st, x.p, y.p, s);
    for (int w = 0; w < 2; ++w) CK(ks->profile(st.pa, s));   // warm
    CK(ks->profile(st.pa, s));
    std::vector<double> el;
    std::vector<int32_t> sm;
    double span = 0;
    read_cta_times(st, el, sm, &span, s);
    for (int c = 0; c < n; ++c) {
      if (elapsed_ms) elapsed_ms[c] = el[(size_t)c] < 0 ? 0.0 : el[(size_t)c];
      if (sm_id) sm_id[c] = sm[(size_t)c];
    }
    *n_ctas = n;
    return SPMV_OK;
  });
}

spmv_status spmv_profile_kernel(spmv_handle_t h, int32_t which, const void *x, void *y,
                                spmv_stream_t stream) {
  if (!h || which < 0 || which > 2 || (h->n_rows > 0 && (!x || !y))) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    const KernelSet *ks = set_for(h);
    StaticSetup st;
    static_setup(h, st, x, y, s);
    DevBuf colp;
    if (which == 1) {
      colp.alloc(sizeof(int32_t) * (size_t)h->nnz, 4, s);
      CK(launch_fill_row_index(h->n_rows, h->n_cols, h->rowptr.as<int32_t>(), colp.as<int32_t>(), s));
      st.pa.colind = colp.as<int32_t>();
    }
    st.pa.cmp_mode = which == 2 ? 1 : 0;
    CK(ks->profile(st.pa, s));
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
  });
}

spmv_status spmv_probe_bandwidth(double *hbm_gbs, double *l2_gbs) {
  if (!hbm_gbs || !l2_gbs) return SPMV_ERR_ARG;
  return guarded([&]() -> spmv_status {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    probe_bandwidth(dev, hbm_gbs, l2_gbs);
    return SPMV_OK;
  });
}

uint32_t spmv_classify(const double *p, double t_imb, double t_ml, double t_mb) {
  if (!p) return 0;
  return classify(p, t_imb, t_ml, t_mb);
}

uint32_t spmv_classify2(const double *p, const double *p2, double t_imb, double t_ml, double t_mb) {
  if (!p) return 0;
  return classify2(p, p2, t_imb, t_ml, t_mb);
}

void spmv_variant_for_classes(uint32_t classes, double nnz_avg, double nnz_max,
                              double long_row_ratio, spmv_variant *out) {
  if (out) *out = variant_for_classes(classes, nnz_avg, nnz_max, long_row_ratio);
}

void spmv_bounds(int64_t n_rows, int64_t n_cols, int64_t nnz, int32_t idx_bytes, int32_t val_bytes,
                 int32_t vec_bytes, double b_max_gbs, double *out) {
  if (out) bounds(n_rows, n_cols, nnz, idx_bytes, val_bytes, vec_bytes, b_max_gbs, out);
}

uint32_t spmv_feature_rules(const double *features, int64_t n_cols, int32_t vec_bytes,
                            int64_t l2_bytes, double long_row_ratio) {
  if (!features) return 0;
  return feature_rules(features, n_cols, vec_bytes, l2_bytes, long_row_ratio);
}

spmv_status spmv_validate_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t *row_ptr,
                              const int32_t *col_ind, int32_t *code, spmv_stream_t stream) {
  if (!row_ptr || !code || n_rows < 0 || n_cols < 0 || nnz < 0) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    DevBuf c;
    c.alloc(16, 4, s, true);
    CK(launch_validate(n_rows, n_cols, nnz, row_ptr, col_ind, c.as<int32_t>(), s));
    CK(cudaMemcpyAsync(code, c.p, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
  });
}

spmv_status spmv_round_values(const double *in, void *out, int64_t n, spmv_dtype to,
                              spmv_stream_t stream) {
  if ((n > 0 && (!in || !out)) || n < 0) return SPMV_ERR_ARG;
  if (!valid_precision_dtype(to)) return SPMV_ERR_UNSUPPORTED_DTYPE;
  if (to == SPMV_DF64) return map_err(launch_df_split(in, out, 0, n, static_cast<cudaStream_t>(stream)));
  return map_err(launch_round_values(in, out, n, to, static_cast<cudaStream_t>(stream)));
}

spmv_status spmv_get_last_device_error(spmv_handle_t h, int32_t *code) {
  if (!h || !code) return SPMV_ERR_ARG;
  return guarded([&]() -> spmv_status {
    CK(cudaDeviceSynchronize());
    int32_t c = 0;
    CK(cudaMemcpy(&c, h->d_err.p, 4, cudaMemcpyDeviceToHost));
    CK(cudaMemset(h->d_err.p, 0, 4));
    *code = c ? c : h->last_error;
    h->last_error = 0;
    return SPMV_OK;
  });
}

spmv_status spmv_selftest_wait_timeout(spmv_handle_t h, int64_t limit_ns,
                                       spmv_stream_t stream) {
  if (!h || limit_ns <= 0 || limit_ns > 10000000000LL) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    CK(launch_selftest_wait((uint64_t)limit_ns, h->d_err.as<int32_t>(), s));
    CK(cudaStreamSynchronize(s));
    int32_t c = 0;
    CK(cudaMemcpy(&c, h->d_err.p, 4, cudaMemcpyDeviceToHost));
    CK(cudaMemset(h->d_err.p, 0, 4));
    return c ? SPMV_ERR_TIMEOUT : SPMV_OK;
  });
}

spmv_status spmv_get_device_bytes(spmv_handle_t h, int64_t *bytes) {
  if (!h || !bytes) return SPMV_ERR_ARG;
  int64_t t = 0;
  for (const DevBuf *b : {&h->rowptr, &h->colind, &h->val_in, &h->val_store, &h->dbase, &h->delta,
                          &h->esc, &h->coord, &h->tail_row, &h->tail_val, &h->head_val,
                          &h->x_stage, &h->y_stage, &h->scratch})
    t += (int64_t)b->bytes;
  *bytes = t;
  return SPMV_OK;
}

// ---------------------------------------------------------------- learned selector ---
spmv_status spmv_mlp_inputs(const double *feat, int64_t batch, const float *mu,
                            const float *inv_sigma, float *X, spmv_stream_t stream) {
  if (batch < 0 || (batch > 0 && (!feat || !X)) || (!mu) != (!inv_sigma)) return SPMV_ERR_ARG;
  return map_err(launch_mlp_inputs(feat, batch, mu, inv_sigma, X, static_cast<cudaStream_t>(stream)));
}

static bool sizes_ok(const int32_t *s) {
  return s && s[0] > 0 && s[1] > 0 && s[2] > 0 && s[3] > 0 && s[0] <= 4096 && s[1] <= 4096 &&
         s[2] <= 4096 && s[3] <= 4096;
}

spmv_status spmv_mlp_logits(const int32_t *sizes, const float *params, int64_t batch,
                            const float *X, float *logits, spmv_stream_t stream) {
  if (!sizes_ok(sizes) || !params || batch < 0 || (batch > 0 && (!X || !logits))) return SPMV_ERR_ARG;
  if (batch == 0) return SPMV_OK;
  return map_err(launch_mlp_logits(sizes, params, batch, X, logits, static_cast<cudaStream_t>(stream)));
}

spmv_status spmv_mlp_loss_grad(const int32_t *sizes, const float *params, int64_t batch,
                               const float *X, const float *Y, float *grad, float *loss,
                               spmv_stream_t stream) {
  if (!sizes_ok(sizes) || !params || batch <= 0 || !X || !Y || !grad || !loss) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    DevBuf work;
    work.alloc(sizeof(float) * (size_t)mlp_work_floats(sizes, batch), 8, s);
    CK(launch_mlp_loss_grad(sizes, params, batch, X, Y, grad, loss, work.as<float>(), s));
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
  });
}

spmv_status spmv_mlp_train(const int32_t *sizes, float *params, float *m, float *v, int64_t batch,
                           const float *X, const float *Y, int32_t steps, int32_t t0, float lr,
                           float beta1, float beta2, float eps, float *loss_hist,
                           spmv_stream_t stream) {
  if (!sizes_ok(sizes) || !params || !m || !v || batch <= 0 || !X || !Y || steps < 0 || t0 < 0)
    return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    const int64_t np = mlp_param_count(sizes);
    DevBuf work, grad, loss;
    work.alloc(sizeof(float) * (size_t)mlp_work_floats(sizes, batch), 8, s);
    grad.alloc(sizeof(float) * (size_t)np, 4, s);
    loss.alloc(sizeof(float), 4, s);
    for (int32_t i = 0; i < steps; ++i) {
      float *lp = loss_hist ? loss_hist + i : loss.as<float>();
      CK(launch_mlp_loss_grad(sizes, params, batch, X, Y, grad.as<float>(), lp, work.as<float>(), s));
      CK(launch_adam(np, params, grad.as<float>(), m, v, lr, beta1, beta2, eps, t0 + i + 1, s));
    }
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
  });
}

spmv_status spmv_selector_create(spmv_selector_t *out, const int32_t *sizes, const float *params,
                                 const float *mu, const float *inv_sigma) {
  if (!out || !sizes_ok(sizes) || !params || sizes[0] != SPMV_MLP_INPUTS || (!mu) != (!inv_sigma))
    return SPMV_ERR_ARG;
  *out = nullptr;
  spmv_selector *sel = new (std::nothrow) spmv_selector();
  if (!sel) return SPMV_ERR_OOM;
  spmv_status st = guarded([&]() -> spmv_status {
    CK(cudaGetDevice(&sel->device));
    std::memcpy(sel->sizes, sizes, sizeof sel->sizes);
    const int64_t np = mlp_param_count(sizes);
    sel->params.alloc(sizeof(float) * (size_t)np, 4, 0);
    CK(cudaMemcpy(sel->params.p, params, sizeof(float) * (size_t)np, cudaMemcpyHostToDevice));
    if (mu) {
      sel->mu.alloc(sizeof(float) * SPMV_MLP_INPUTS, 4, 0);
      sel->inv_sigma.alloc(sizeof(float) * SPMV_MLP_INPUTS, 4, 0);
      CK(cudaMemcpy(sel->mu.p, mu, sizeof(float) * SPMV_MLP_INPUTS, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(sel->inv_sigma.p, inv_sigma, sizeof(float) * SPMV_MLP_INPUTS, cudaMemcpyHostToDevice));
      sel->has_norm = true;
    }
    // per-call workspace: 16 doubles of features, then inputs, hidden layers and logits
    const int64_t wf = SPMV_MLP_INPUTS + mlp_logits_work_floats(sizes, 1) + sizes[3];
    sel->ws.alloc(sizeof(double) * 16 + sizeof(float) * (size_t)wf, 8, 0, true);
    CK(cudaDeviceSynchronize());
    return SPMV_OK;
  });
  if (st != SPMV_OK) {
    spmv_selector_destroy(sel);
    return st;
  }
  *out = sel;
  return SPMV_OK;
}

spmv_status spmv_selector_destroy(spmv_selector_t sel) {
  if (!sel) return SPMV_ERR_ARG;
  cudaDeviceSynchronize();
  sel->params.release();
  sel->mu.release();
  sel->inv_sigma.release();
  sel->ws.release();
  delete sel;
  return SPMV_OK;
}

spmv_status spmv_selector_predict(spmv_selector_t sel, const double *feat16, uint32_t *classes,
                                  double *margin, spmv_stream_t stream) {
  if (!sel || !feat16 || !classes) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    const int n3 = sel->sizes[3];
    double *f = sel->ws.as<double>();
    float *x = reinterpret_cast<float *>(f + 16);
    float *hid = x + SPMV_MLP_INPUTS;
    float *lg = hid + mlp_logits_work_floats(sel->sizes, 1);
    CK(cudaMemcpyAsync(f, feat16, sizeof(double) * 16, cudaMemcpyHostToDevice, s));
    CK(launch_mlp_inputs(f, 1, sel->has_norm ? sel->mu.as<float>() : nullptr,
                         sel->has_norm ? sel->inv_sigma.as<float>() : nullptr, x, s));
    CK(launch_mlp_logits_ws(sel->sizes, sel->params.as<float>(), 1, x, lg, hid, s));
    float h[64];
    CK(cudaMemcpyAsync(h, lg, sizeof(float) * (size_t)std::min(n3, 64), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    uint32_t c = 0;
    double mg = 1e300;
    for (int o = 0; o < n3 && o < 4; ++o) {
      if (h[o] > 0.0f) c |= (1u << o);
      mg = std::min(mg, (double)std::fabs(h[o]));
    }
    *classes = c;
    if (margin) *margin = mg;
    return SPMV_OK;
  });
}

}  // extern "C"

// ---------------------------------------------------------------- kernel sets --------
namespace spmv {
spmv_status handle_info(spmv_handle_t h, const int32_t **rowptr, const int32_t **colind,
                        const void **val, int64_t *n_rows, int32_t *storage, int32_t *vec,
                        int32_t *acc, int32_t *vs) {
  if (!h) return SPMV_ERR_ARG;
  *rowptr = h->rowptr.as<int32_t>();
  *colind = h->colind.as<int32_t>();
  *val = h->val_ptr();
  *n_rows = h->n_rows;
  *storage = h->storage;
  *vec = h->vec;
  *acc = h->acc;
  *vs = (h->tuned && h->variant.partition == 0) ? h->variant.vs : 0;
  return SPMV_OK;
}

const KernelSet *kernel_set(spmv_dtype val, spmv_dtype vec, spmv_dtype acc) {
  if (val == SPMV_F64) return (vec == SPMV_F64 && acc == SPMV_F64) ? kernel_set_f64_dd() : nullptr;
  if (val == SPMV_DF64) return (vec == SPMV_F64 && acc == SPMV_DF64) ? kernel_set_f64_df() : nullptr;
  const bool dd = vec == SPMV_F64 && acc == SPMV_F64;
  const bool ff = vec == SPMV_F32 && acc == SPMV_F32;
  const bool fd = vec == SPMV_F32 && acc == SPMV_F64;
  if (val == SPMV_F32) return dd ? kernel_set_f32_dd() : ff ? kernel_set_f32_ff() : fd ? kernel_set_f32_fd() : nullptr;
  if (val == SPMV_BF16) return dd ? kernel_set_bf16_dd() : ff ? kernel_set_bf16_ff() : fd ? kernel_set_bf16_fd() : nullptr;
  return nullptr;
}
}  // namespace spmv

// Runtime state shared by the host sources behind the C ABI of include/spmv_gb300.h.
//
// A matrix handle owns a device copy of the CSR matrix (int32 row pointers and columns, values
// in the input dtype, plus a converted copy in the storage dtype), the data of the installed
// optimization-pool variant (delta index, merge-path tile table or row decomposition tables)
// and staging buffers for host-buffer runs. The host sources split the runtime as follows:
//   api.cu       handle lifecycle, precision, runs, exports of the pool data;
//   variant.cu   building the pool data and installing a variant (Table II);
//   tune.cu      device properties, bandwidth probe, bounds, classification (Sections III-C
//                and III-D), features, profiling and the width / geometry sweep;
//   host.cu      the pipelined host-buffer run;
//   selector.cu  the learned selector's MLP;
//   cg.cu        conjugate gradients on a tuned handle.
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"

namespace spmv {

// Kernel sets whose thread-per-row tiles accumulate in double-float arithmetic on the FP32
// pipe (spmv_df.cu): FP32 / BF16 storage with FP64 (d) or FP32 (f) x.
const KernelSet *kernel_set_f32_d_df();
const KernelSet *kernel_set_f32_f_df();
const KernelSet *kernel_set_bf16_d_df();
const KernelSet *kernel_set_bf16_f_df();

namespace rt {

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

// Device buffer with zeroed slack past the logical end (see kPadElems), owned by exactly
// one object (move-only; freed on destruction, so temporaries do not leak when a CUDA error
// unwinds a build step).
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

inline double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

inline int pow2_ceil_clamped(double v, int lo, int hi) {
  int p = lo;
  while (p < hi && (double)p < v) p <<= 1;
  return p;
}

// Sub-warp width heuristic: enough lanes to cover the average row in one step of E
// elements per lane.
inline int heuristic_vs(double nnz_avg, int elems_per_lane) {
  return pow2_ceil_clamped(nnz_avg / (double)elems_per_lane, 2, 32);
}

// Width for the pool's sub-warp-row variants: rows of up to 64 nonzeros on average go to
// the thread-per-row tile kernel (width 1: one FMA per nonzero, no lane reduction);
// longer rows to sub-warps wide enough to cover them.
inline int pool_vs(double nnz_avg, int elems_per_lane) {
  return nnz_avg <= 64.0 ? 1 : heuristic_vs(nnz_avg, elems_per_lane);
}

struct DeviceInfo {
  int sms = 0;
  int64_t l2_bytes = 0;
  bool bw_done = false;
  double hbm_gbs = 0.0, l2_gbs = 0.0;
};

// Cached properties of device `dev` (SM count, L2 size, probed bandwidths).
DeviceInfo &device_info(int dev);

}  // namespace rt
}  // namespace spmv

// ------------------------------------------------------------------ handle -----------
struct spmv_matrix {
  using DevBuf = spmv::rt::DevBuf;
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
  int32_t bin_med = spmv::kBinMed, bin_chunk = spmv::kBinChunk;   // limits of the built tables
  bool has_bins = false;
  DevBuf sell_off, sell_val, sell_idx;   // sliced rows: column-major 32-row slices
  int32_t sell_bits = -1;      // column representation of the built slices (0 = int32; -1 none)
  int64_t sell_total = 0;      // slice positions, padding included
  DevBuf pnl_rowptr, pnl_col, pnl_val;   // column panels: panel-major copy of the matrix
  int32_t pnl_count = 0;       // panels of the built copy (0: none)
  int32_t pnl_width = 0;       // columns per panel
  int32_t pnl_tile_rows = 0, pnl_tile_cap = 0;   // staged tiles of one-thread-per-row passes
  // run state
  spmv_variant variant{};
  bool tuned = false;
  int32_t tile_cap = 0;        // staged elements per tile of the thread-per-row kernel
  int32_t tile_rows = spmv::kTileRows;  // rows per tile of the thread-per-row kernel
  int32_t tile_pipe = 0;       // 1: persistent CTAs with two tiles in flight
  DevBuf d_err;                // device error word of bounded waits
  DevBuf small;                // 256 bytes for single-value reductions (maxima, codes)
  cudaStream_t copy_stream = nullptr;   // host-buffer runs: device-to-host copies of y (even
  cudaStream_t copy_stream2 = nullptr;  // and odd chunks: two copies in flight)
  cudaStream_t upload_stream = nullptr; // host-buffer runs: host-to-device copies of x
  cudaStream_t capture_stream = nullptr;  // host-buffer runs: graph capture
  cudaStream_t chunk_stream[2] = {};    // host-buffer runs: alternate chunks' kernels
  cudaEvent_t joined[6] = {};           // host-buffer runs: fork from / rejoin the origin
  cudaEvent_t pass_done = nullptr;      // host-buffer runs: column panels' passes before the last
  cudaGraph_t host_graph = nullptr;     // host-buffer pipeline for (host_x, host_y, epoch)
  cudaGraphExec_t host_exec = nullptr;
  const void *host_x = nullptr;
  void *host_y = nullptr;
  uint64_t host_epoch = 0;
  uint64_t epoch = 1;                   // bumped whenever precision or variant changes
  cudaEvent_t chunk_done[spmv::rt::kHostChunks] = {};
  cudaEvent_t x_ready[spmv::rt::kHostChunks] = {};
  int64_t x_need[spmv::rt::kHostChunks] = {};     // elements of x (a prefix) chunks 0..c read
  bool x_need_valid = false;
  DevBuf feat_part, feat_fin;  // feature partial sums, kept between calls
  DevBuf x_stage, y_stage, scratch;
  DevBuf cg_ws;                // conjugate gradients: r, p, Ap, block partials, scalars
  int32_t last_error = 0;
  double nnz_avg() const { return n_rows ? (double)nnz / (double)n_rows : 0.0; }
  const void *val_ptr() const { return val_store.p ? val_store.p : val_in.p; }
};

struct spmv_selector {
  using DevBuf = spmv::rt::DevBuf;
  int device = 0;
  int32_t sizes[4] = {0, 0, 0, 0};
  DevBuf params, mu, inv_sigma;
  DevBuf ws;                   // one sample: 16 features, inputs, hidden layers, logits
  bool has_norm = false;
  bool has_range = false;      // training range of the standardized inputs
  float in_lo[SPMV_MLP_INPUTS] = {}, in_hi[SPMV_MLP_INPUTS] = {};
  float in_slack = 0.0f;
};

namespace spmv {
namespace rt {

// Kernel set of the handle's (storage, vec, acc) combination.
const KernelSet *set_for(const spmv_matrix *h);
// Kernel arguments for y = A x with the handle's installed pool data.
RunArgs run_args(const spmv_matrix *h, const void *x, void *y);
// Default tile geometry of the thread-per-row kernel, and an explicit one.
void compute_tile_cap(spmv_matrix *h, const spmv_variant &v, cudaStream_t s);
void set_tile_geometry(spmv_matrix *h, const spmv_variant &v, int rows, bool pipe,
                       cudaStream_t s);
// Completes the free fields of v and builds the pool data it needs.
void prepare_variant(spmv_matrix *h, spmv_variant &v, cudaStream_t s);
bool valid_variant(const spmv_variant &v);
// One launch of variant v on device buffers x and y.
cudaError_t launch_run(const spmv_matrix *h, const spmv_variant &v, const void *x, void *y,
                       cudaStream_t s);
// Frees the column-panel copy (its values follow the storage dtype).
void drop_panels(spmv_matrix *h);
// Frees the sliced-row copy (its values follow the storage dtype).
void drop_sell(spmv_matrix *h);
// Positions of the sliced-row layout of the matrix, padding included (no copy is built).
int64_t sell_positions(spmv_matrix *h, cudaStream_t s);
// Frees the captured host-buffer pipeline.
void drop_host_graph(spmv_matrix *h);

// Runs fn, turning CUDA failures and allocation failures into status codes.
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

}  // namespace rt
}  // namespace spmv

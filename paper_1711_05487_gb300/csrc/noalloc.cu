// spmv_run_noalloc: the merge-path SpMV for callers that must not allocate device memory.
//
// The regular path keeps its merge-path table and carry buffers in memory that
// spmv_create / spmv_tune allocate. Some callers cannot allow that: an application whose
// allocator owns the whole device memory budget and forbids libraries from allocating
// behind its back, code that runs when the device is nearly full, or latency-critical code
// that cannot afford cudaMalloc / cudaFree (which can synchronize the device). This entry
// point takes the caller's CSR arrays, x and y, and keeps its scratch (the tile table and
// the per-tile carries) in one fixed-size array in device global memory, defined below.
#include <mutex>

#include "spmv_kernels.cuh"

namespace {

// Scratch size. Every GPU that loads the library holds this array until the process exits.
constexpr long long kNoAllocScratchBytes = 16ll << 20;   // 16 MiB
// Per merge-path tile: table entry (int2, 8 B), carry row (int32, 4 B), tail and head
// carries (FP64, 8 B each); the table has one entry more than there are tiles.
constexpr long long kBytesPerTile = 8 + 4 + 8 + 8;
constexpr long long kMaxTiles = (kNoAllocScratchBytes - 8 - 3 * 256) / kBytesPerTile;
// Largest n_rows + nnz one call accepts (each tile covers kMergeItems merge items).
constexpr long long kMaxItems = kMaxTiles * spmv::kMergeItems;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once per CUDA context (the name
// of the array in host code is only a stand-in for the symbol, not a device address). The
// cache is keyed by the context's unique id: after cudaDeviceReset the runtime creates a new
// context and loads the kernels again, possibly at another address, so an address taken in
// the old context is never reused.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

struct ScratchSlot {
  unsigned long long ctx_id = 0;   // 0: not looked up yet
  void *addr = nullptr;
};

std::mutex g_mu;
ScratchSlot g_scratch[128];
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_entry_points = false;

// Id of the calling thread's current context, 0 if there is none yet (the runtime makes the
// device's primary context current on its first use of the device). Holds g_mu.
unsigned long long current_ctx_id() {
  if (!g_entry_points) {
    g_entry_points = true;
    void *f = nullptr, *g = nullptr;
    cudaDriverEntryPointQueryResult q1{}, q2{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
      g_ctx_id = reinterpret_cast<CtxGetIdFn>(g);
    }
    cudaGetLastError();
  }
  if (!g_ctx_current || !g_ctx_id) return 0;
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_current(&ctx) != 0 || !ctx) return 0;
  if (g_ctx_id(ctx, &id) != 0) return 0;
  return id;
}

spmv_status scratch_address(int dev, unsigned char **out) {
  if (dev < 0 || dev >= 128) return SPMV_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  ScratchSlot &slot = g_scratch[dev];
  const unsigned long long id = current_ctx_id();
  if (id == 0 || slot.ctx_id != id || !slot.addr) {
    // set-up with the device current: the symbol lookup also creates the context (and
    // loads the kernels) if this is the device's first use
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return SPMV_ERR_CUDA;
    }
    slot.addr = p;
    slot.ctx_id = current_ctx_id();   // 0 (no driver entry points): looked up on every call
  }
  *out = static_cast<unsigned char *>(slot.addr);
  return SPMV_OK;
}

inline long long align256(long long v) { return (v + 255) & ~255ll; }

}  // namespace

extern "C" spmv_status spmv_run_noalloc(int64_t n_rows, int64_t n_cols, int64_t nnz,
                                        const int32_t *row_ptr, const int32_t *col_ind,
                                        const double *val, const double *x, double *y,
                                        spmv_stream_t stream) {
  if (n_rows < 0 || n_cols < 0 || nnz < 0 || n_rows >= INT32_MAX || n_cols >= INT32_MAX ||
      nnz >= INT32_MAX)
    return SPMV_ERR_ARG;
  if (n_rows + nnz > kMaxItems) return SPMV_ERR_TOO_LARGE;
  if (n_rows == 0) return SPMV_OK;
  if (!row_ptr || !y || (nnz > 0 && (!col_ind || !val || !x))) return SPMV_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SPMV_ERR_CUDA;
  }
  unsigned char *base = nullptr;
  const spmv_status st = scratch_address(dev, &base);
  if (st != SPMV_OK) return st;

  const long long n_tiles = (n_rows + nnz + spmv::kMergeItems - 1) / spmv::kMergeItems;
  // carve the scratch: table, tail carries, head carries, carry rows (256-byte aligned)
  const long long off_tail = align256(8 * (n_tiles + 1));
  const long long off_head = off_tail + align256(8 * n_tiles);
  const long long off_row = off_head + align256(8 * n_tiles);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  spmv::RunArgs a;
  a.n_rows = n_rows;
  a.n_cols = n_cols;
  a.nnz = nnz;
  a.rowptr = row_ptr;
  a.colind = col_ind;
  a.val = val;
  a.x = x;
  a.y = y;
  a.coord = reinterpret_cast<const int2 *>(base);
  a.n_tiles = n_tiles;
  a.tail_val = reinterpret_cast<double *>(base + off_tail);
  a.head_val = reinterpret_cast<double *>(base + off_head);
  a.tail_row = reinterpret_cast<int32_t *>(base + off_row);
  // Every scratch entry this call reads is written earlier in the same call (the table by
  // the search, the carries by the tile kernel), so nothing needs clearing between calls.
  cudaError_t e = spmv::launch_merge_coords(n_rows, nnz, row_ptr, spmv::kMergeItems, n_tiles,
                                            reinterpret_cast<int2 *>(base), s);
  if (e == cudaSuccess) {
    spmv_variant v{};
    v.partition = 1;
    e = spmv::kernel_set(SPMV_F64, SPMV_F64, SPMV_F64)->spmv(v, a, s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SPMV_ERR_CUDA;
  }
  return SPMV_OK;
}

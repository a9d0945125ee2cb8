// C ABI of the batched SpMM: work-item planning, the persistent launch captured into a
// CUDA graph, and the per-matrix sequential path it is compared with.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

using namespace spmv;

namespace {
// Default plan: target nonzeros per row-block item (a warp's work); rows longer than this
// are split into chunks of kChunkNnz nonzeros (the matrix decomposition applied per item).
// spmv_batch_tune picks both by timing.
constexpr int32_t kItemNnz = 1024;
constexpr int32_t kChunkNnz = 2048;
constexpr int32_t kItemRowsMax = 1024;
inline int k_slot(int k) { return k == 1 ? 0 : (k == 4 ? 1 : 2); }

struct Fail {
  cudaError_t e;
};
#define BK(expr)                               \
  do {                                         \
    cudaError_t _e = (expr);                   \
    if (_e != cudaSuccess) throw Fail{_e};     \
  } while (0)

int heuristic_vs(double nnz_avg) {
  int p = 2;
  while (p < 32 && (double)p < nnz_avg) p <<= 1;
  return p;
}
}  // namespace

struct spmv_batch {
  int device = 0;
  int32_t count = 0;
  std::vector<spmv_handle_t> handles;
  std::vector<const void *> X;
  std::vector<void *> Y;
  std::vector<int32_t> k;
  std::vector<BatchMat> mats;            // per matrix: arrays, k and sub-warp width
  std::vector<std::vector<int32_t>> rowptr;   // host copies, for re-planning
  int32_t item_nnz = kItemNnz, chunk_nnz = kChunkNnz;
  BatchMat *d_mats = nullptr;
  BatchItem *d_items = nullptr;          // every matrix's items, costliest first
  BatchFix *d_fix = nullptr;
  double *d_partials = nullptr;
  int32_t *d_counter = nullptr;          // the work counter of the persistent kernel
  int32_t n_items = 0, n_fix = 0, n_chunks = 0;
  int grid = 0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static void batch_free(spmv_batch *b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->d_mats);
  cudaFree(b->d_items);
  cudaFree(b->d_fix);
  cudaFree(b->d_partials);
  cudaFree(b->d_counter);
  delete b;
}

// The work plan for (item_nnz, chunk_nnz): row blocks of about item_nnz nonzeros per warp,
// rows longer than item_nnz split into chunks of chunk_nnz nonzeros with FP64 partials,
// costliest items first; uploads the items, the fixups and the partial slots, sizes the
// persistent grid and drops the captured graph.
static void batch_plan(spmv_batch *b, int32_t item_nnz, int32_t chunk_nnz, cudaStream_t s) {
  std::vector<BatchItem> items_k[3];   // per k in {1, 4, 16}
  std::vector<BatchFix> fix;
  int32_t chunks = 0;
  for (int32_t m = 0; m < b->count; ++m) {
    const std::vector<int32_t> &hrp = b->rowptr[(size_t)m];
    const int32_t n_rows = (int32_t)hrp.size() - 1;
    std::vector<BatchItem> &items = items_k[k_slot(b->k[(size_t)m])];
    int32_t r = 0;
    while (r < n_rows) {
      const int32_t len = hrp[(size_t)r + 1] - hrp[(size_t)r];
      if (len > item_nnz) {
        const int32_t first = chunks;
        int32_t cnt = 0;
        for (int32_t z = hrp[(size_t)r]; z < hrp[(size_t)r + 1]; z += chunk_nnz) {
          const int32_t ze = std::min(z + chunk_nnz, hrp[(size_t)r + 1]);
          items.push_back(BatchItem{m, r, r + 1, z, ze, chunks++});
          ++cnt;
        }
        fix.push_back(BatchFix{m, r, first, cnt});
        ++r;
        continue;
      }
      int32_t e = r;
      int64_t acc = 0;
      while (e < n_rows && e - r < kItemRowsMax) {
        const int32_t l = hrp[(size_t)e + 1] - hrp[(size_t)e];
        if (l > item_nnz || (acc + l > item_nnz && e > r)) break;
        acc += l;
        ++e;
      }
      items.push_back(BatchItem{m, r, e, 0, (int32_t)acc, -1});   // nz_end: the block's nnz
      r = e;
    }
  }
  // Costliest items first (chunks of split rows, then full row blocks, then the short
  // remainders; within each, the widest right-hand sides first), so that the last items
  // the warps take are the cheapest; the sort is stable, so items of one matrix stay
  // together (their x rows stay L2-hot).
  auto item_class = [&](const BatchItem &it) -> int {
    if (it.chunk >= 0) return 0;
    return it.nz_end >= item_nnz / 2 ? 1 : 2;
  };
  std::vector<BatchItem> items;
  for (int q = 2; q >= 0; --q) items.insert(items.end(), items_k[q].begin(), items_k[q].end());
  std::stable_sort(items.begin(), items.end(), [&](const BatchItem &a, const BatchItem &c) {
    return item_class(a) < item_class(c);
  });
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  BK(cudaDeviceSynchronize());   // no launch of the previous plan is still running
  cudaFree(b->d_items);
  cudaFree(b->d_fix);
  cudaFree(b->d_partials);
  b->d_items = nullptr;
  b->d_fix = nullptr;
  b->d_partials = nullptr;
  b->n_items = (int32_t)items.size();
  b->n_fix = (int32_t)fix.size();
  b->n_chunks = chunks;
  BK(cudaMalloc(&b->d_items, sizeof(BatchItem) * std::max<size_t>(items.size(), 1)));
  BK(cudaMalloc(&b->d_fix, sizeof(BatchFix) * std::max<size_t>(fix.size(), 1)));
  BK(cudaMalloc(&b->d_partials, sizeof(double) * 16 * (size_t)std::max(chunks, 1)));
  if (!items.empty())
    BK(cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice, s));
  if (!fix.empty())
    BK(cudaMemcpyAsync(b->d_fix, fix.data(), sizeof(BatchFix) * fix.size(), cudaMemcpyHostToDevice, s));
  BK(cudaStreamSynchronize(s));
  int sms = 0;
  BK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  const int64_t ctas = ((int64_t)b->n_items + 7) / 8;     // 8 warps per CTA
  b->grid = (int)std::min<int64_t>((int64_t)sms * batch_blocks_per_sm(), ctas);
  b->item_nnz = item_nnz;
  b->chunk_nnz = chunk_nnz;
}

// The batch reads its handles' device arrays through the pointers taken at creation: a
// handle whose precision changed since (its value array reallocated) no longer matches.
static bool batch_current(const spmv_batch *b) {
  for (int32_t m = 0; m < b->count; ++m) {
    const int32_t *rp = nullptr, *ci = nullptr;
    const void *v = nullptr;
    int64_t n_rows = 0;
    int32_t st = 0, ve = 0, ac = 0, vs = 0;
    const BatchMat &bm = b->mats[(size_t)m];
    if (handle_info(b->handles[(size_t)m], &rp, &ci, &v, &n_rows, &st, &ve, &ac, &vs) != SPMV_OK ||
        rp != bm.rowptr || ci != bm.colind || v != static_cast<const void *>(bm.val) ||
        st != SPMV_F32 || ve != SPMV_F32 || ac != SPMV_F32)
      return false;
  }
  return true;
}

static spmv_status batch_status(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? SPMV_ERR_OOM
         : e == cudaErrorInvalidValue  ? SPMV_ERR_ARG
                                       : SPMV_ERR_CUDA;
}

extern "C" {

spmv_status spmv_batch_create(spmv_batch_t *out, const spmv_handle_t *handles, int32_t count,
                              const void *const *X, void *const *Y, const int32_t *k,
                              spmv_stream_t stream) {
  if (!out || !handles || !X || !Y || !k || count <= 0) return SPMV_ERR_ARG;
  *out = nullptr;
  spmv_batch *b = new (std::nothrow) spmv_batch();
  if (!b) return SPMV_ERR_OOM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    BK(cudaGetDevice(&b->device));
    b->count = count;
    b->mats.resize((size_t)count);
    b->rowptr.resize((size_t)count);
    for (int32_t m = 0; m < count; ++m) {
      if (!handles[m] || k[m] < 1 || (k[m] != 1 && k[m] != 4 && k[m] != 16)) throw Fail{cudaErrorInvalidValue};
      const int32_t *rp = nullptr, *ci = nullptr;
      const void *v = nullptr;
      int64_t n_rows = 0;
      int32_t st = 0, ve = 0, ac = 0, vs = 0;
      spmv_status q = handle_info(handles[m], &rp, &ci, &v, &n_rows, &st, &ve, &ac, &vs);
      if (q != SPMV_OK) {
        batch_free(b);
        return q;
      }
      if (st != SPMV_F32 || ve != SPMV_F32 || ac != SPMV_F32) {
        batch_free(b);
        return SPMV_ERR_UNSUPPORTED_DTYPE;
      }
      std::vector<int32_t> &hrp = b->rowptr[(size_t)m];
      hrp.resize((size_t)n_rows + 1);
      BK(cudaMemcpyAsync(hrp.data(), rp, 4 * ((size_t)n_rows + 1), cudaMemcpyDeviceToHost, s));
      BK(cudaStreamSynchronize(s));
      const double avg = n_rows ? (double)hrp[(size_t)n_rows] / (double)n_rows : 0.0;
      b->mats[(size_t)m] = BatchMat{rp, ci, static_cast<const float *>(v),
                                    static_cast<const float *>(X[m]), static_cast<float *>(Y[m]),
                                    k[m], vs > 0 ? vs : heuristic_vs(avg)};
      b->handles.push_back(handles[m]);
      b->X.push_back(X[m]);
      b->Y.push_back(Y[m]);
      b->k.push_back(k[m]);
    }
    BK(cudaMalloc(&b->d_mats, sizeof(BatchMat) * b->mats.size()));
    BK(cudaMalloc(&b->d_counter, sizeof(int32_t)));
    BK(cudaMemcpyAsync(b->d_mats, b->mats.data(), sizeof(BatchMat) * b->mats.size(),
                       cudaMemcpyHostToDevice, s));
    batch_plan(b, kItemNnz, kChunkNnz, s);
    BK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  } catch (const Fail &f) {
    cudaGetLastError();
    batch_free(b);
    return batch_status(f.e);
  }
  *out = b;
  return SPMV_OK;
}

spmv_status spmv_batch_set_plan(spmv_batch_t b, int32_t item_nnz, int32_t chunk_nnz,
                                spmv_stream_t stream) {
  if (!b || item_nnz < 32 || item_nnz > 65536 || chunk_nnz < item_nnz || chunk_nnz > (1 << 20))
    return SPMV_ERR_ARG;
  try {
    batch_plan(b, item_nnz, chunk_nnz, static_cast<cudaStream_t>(stream));
  } catch (const Fail &f) {
    cudaGetLastError();
    return batch_status(f.e);
  }
  return SPMV_OK;
}

spmv_status spmv_batch_tune(spmv_batch_t b, int32_t reps, int32_t *item_nnz,
                            int32_t *chunk_nnz, spmv_stream_t stream) {
  if (!b || reps < 1) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  try {
    BK(cudaEventCreate(&e0));
    BK(cudaEventCreate(&e1));
    float best = 1e30f;
    int32_t bi = b->item_nnz, bc = b->chunk_nnz;
    for (int32_t item : {256, 512, 1024, 2048}) {
      for (int32_t mult : {2, 4}) {
        batch_plan(b, item, item * mult, s);
        for (int w = 0; w < 2; ++w) {
          const spmv_status q = spmv_run_batched(b, stream);
          if (q != SPMV_OK) throw Fail{cudaErrorLaunchFailure};
        }
        BK(cudaEventRecord(e0, s));
        for (int r = 0; r < reps; ++r) {
          const spmv_status q = spmv_run_batched(b, stream);
          if (q != SPMV_OK) throw Fail{cudaErrorLaunchFailure};
        }
        BK(cudaEventRecord(e1, s));
        BK(cudaEventSynchronize(e1));
        float ms = 0.f;
        BK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
          best = ms;
          bi = item;
          bc = item * mult;
        }
      }
    }
    batch_plan(b, bi, bc, s);
  } catch (const Fail &f) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return batch_status(f.e);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (item_nnz) *item_nnz = b->item_nnz;
  if (chunk_nnz) *chunk_nnz = b->chunk_nnz;
  return SPMV_OK;
}

spmv_status spmv_run_batched(spmv_batch_t b, spmv_stream_t stream) {
  if (!b || !batch_current(b)) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    if (!b->exec) {
      // Capture on the batch's own stream (the legacy default stream cannot be captured):
      // reset the work counter, the persistent kernel over every item, then the fixup of
      // split rows.
      BK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int32_t), b->cap);
      if (e == cudaSuccess)
        e = launch_batch_persistent(b->d_mats, b->d_items, b->n_items, b->d_counter,
                                    b->d_partials, b->grid, b->cap);
      if (e == cudaSuccess) e = launch_batch_fixup(b->d_mats, b->d_fix, b->n_fix, b->d_partials, b->cap);
      cudaGraph_t g = nullptr;
      cudaError_t e3 = cudaStreamEndCapture(b->cap, &g);
      BK(e);
      BK(e3);
      b->graph = g;
      BK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
    BK(cudaGraphLaunch(b->exec, s));
  } catch (const Fail &f) {
    cudaGetLastError();
    return f.e == cudaErrorMemoryAllocation ? SPMV_ERR_OOM : SPMV_ERR_CUDA;
  }
  return SPMV_OK;
}

spmv_status spmv_run_batched_sequential(spmv_batch_t b, spmv_stream_t stream) {
  if (!b) return SPMV_ERR_ARG;
  for (int32_t m = 0; m < b->count; ++m) {
    spmv_status q = b->k[(size_t)m] == 1
                        ? spmv_run(b->handles[(size_t)m], b->X[(size_t)m], b->Y[(size_t)m], stream)
                        : spmv_run_spmm(b->handles[(size_t)m], b->X[(size_t)m], b->Y[(size_t)m],
                                        b->k[(size_t)m], stream);
    if (q != SPMV_OK) return q;
  }
  return SPMV_OK;
}

spmv_status spmv_batch_destroy(spmv_batch_t b) {
  if (!b) return SPMV_ERR_ARG;
  batch_free(b);
  return SPMV_OK;
}

}  // extern "C"

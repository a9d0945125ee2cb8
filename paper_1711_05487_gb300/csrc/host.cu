// Host-buffer runs (spmv_run_host): x is uploaded and y downloaded in row chunks that
// overlap the chunks' kernels; with page-locked buffers the pipeline is a CUDA graph.
#include "handle.h"

using namespace spmv;
using namespace spmv::rt;

namespace {

// True for page-locked (pinned or registered) host memory.
bool is_page_locked(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

}  // namespace

namespace spmv {
namespace rt {

void drop_host_graph(spmv_matrix *h) {
  if (h->host_exec) cudaGraphExecDestroy(h->host_exec);
  if (h->host_graph) cudaGraphDestroy(h->host_graph);
  h->host_exec = nullptr;
  h->host_graph = nullptr;
  h->host_x = nullptr;
  h->host_y = nullptr;
}

}  // namespace rt
}  // namespace spmv

extern "C" {

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
      CK(cudaStreamCreateWithFlags(&h->copy_stream2, cudaStreamNonBlocking));
      CK(cudaStreamCreateWithFlags(&h->upload_stream, cudaStreamNonBlocking));
      CK(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
      for (auto &st : h->chunk_stream) CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      for (int c = 0; c < kHostChunks; ++c) {
        CK(cudaEventCreateWithFlags(&h->chunk_done[c], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->x_ready[c], cudaEventDisableTiming));
      }
      for (auto &e : h->joined) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&h->pass_done, cudaEventDisableTiming));
    }
    // pipelining pays once the copies take longer than a few chunk launches (x and y of at
    // least 8 MB together)
    const bool big = h->n_rows >= 4 * kHostChunks * kTileRows &&
                     (int64_t)vb * (h->n_rows + h->n_cols) >= 8000000;
    const int n_pass = h->variant.xpath >= 2 ? h->variant.xpath : 0;
    const bool panels = n_pass >= 2 && n_pass <= kHostChunks && big;
    const bool chunked = (h->variant.partition == 0 || h->variant.partition == 3) &&
                         h->variant.xpath < 2 && big;
    const int nch = (chunked || panels) ? kHostChunks : 1;
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
    cudaStream_t side[5] = {h->upload_stream, h->copy_stream, h->copy_stream2,
                            h->chunk_stream[0], h->chunk_stream[1]};
    auto fork = [&](cudaStream_t origin) {
      CK(cudaEventRecord(h->joined[5], origin));
      for (cudaStream_t st : side) CK(cudaStreamWaitEvent(st, h->joined[5], 0));
    };
    auto join = [&](cudaStream_t origin) {
      for (int k = 0; k < 5; ++k) {
        CK(cudaEventRecord(h->joined[k], side[k]));
        CK(cudaStreamWaitEvent(origin, h->joined[k], 0));
      }
    };
    // downloads of consecutive chunks alternate between two streams (two copies in flight)
    auto download = [&](int c, int64_t r0, int64_t r1, cudaStream_t after) {
      cudaStream_t cp = (c & 1) ? h->copy_stream2 : h->copy_stream;
      CK(cudaEventRecord(h->chunk_done[c], after));
      CK(cudaStreamWaitEvent(cp, h->chunk_done[c], 0));
      CK(cudaMemcpyAsync(static_cast<char *>(y_host) + vb * (size_t)r0,
                         static_cast<char *>(h->y_stage.p) + vb * (size_t)r0,
                         vb * (size_t)(r1 - r0), cudaMemcpyDeviceToHost, cp));
    };
    auto enqueue = [&](cudaStream_t origin) {
      fork(origin);
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
          if (a.sell_off) a.sell_off += r0 / 32;   // chunks start on 128-row boundaries
          CK(ks->spmv(h->variant, a, cs));
        }
        download(c, r0, r1, cs);
      }
      join(origin);
    };
    // Column panels: pass p reads only slice p of x, so x goes up in slice order on the
    // upload stream and pass p waits for its slice (the next slices upload during the
    // passes before); the last pass runs in row chunks on the two alternating streams, each
    // finished chunk of y downloaded while the next computes.
    auto enqueue_panels = [&](cudaStream_t origin) {
      fork(origin);
      const int64_t w = h->pnl_width;
      for (int p = 0; p < n_pass; ++p) {
        const int64_t c0 = std::min<int64_t>(h->n_cols, (int64_t)p * w);
        const int64_t c1 = p == n_pass - 1 ? h->n_cols : std::min<int64_t>(h->n_cols, c0 + w);
        if (c1 > c0)
          CK(cudaMemcpyAsync(static_cast<char *>(h->x_stage.p) + vb * (size_t)c0,
                             static_cast<const char *>(x_host) + vb * (size_t)c0,
                             vb * (size_t)(c1 - c0), cudaMemcpyHostToDevice, h->upload_stream));
        CK(cudaEventRecord(h->x_ready[p], h->upload_stream));
      }
      for (int p = 0; p + 1 < n_pass; ++p) {
        CK(cudaStreamWaitEvent(h->chunk_stream[0], h->x_ready[p], 0));
        RunArgs a = run_args(h, h->x_stage.p, h->y_stage.p);
        a.pnl_first = p;
        a.n_panels = 1;
        CK(ks->spmv(h->variant, a, h->chunk_stream[0]));
      }
      CK(cudaEventRecord(h->pass_done, h->chunk_stream[0]));
      CK(cudaStreamWaitEvent(h->chunk_stream[1], h->pass_done, 0));
      for (cudaStream_t cs : {h->chunk_stream[0], h->chunk_stream[1]})
        CK(cudaStreamWaitEvent(cs, h->x_ready[n_pass - 1], 0));
      for (int c = 0; c < nch; ++c) {
        const int64_t r0 = bounds[c], r1 = bounds[c + 1];
        if (r1 <= r0) continue;
        cudaStream_t cs = h->chunk_stream[c & 1];
        RunArgs a = run_args(h, h->x_stage.p, static_cast<char *>(h->y_stage.p) + vb * (size_t)r0);
        a.n_rows = r1 - r0;
        a.pnl_rowptr += r0;
        a.pnl_first = n_pass - 1;
        a.n_panels = 1;
        CK(ks->spmv(h->variant, a, cs));
        download(c, r0, r1, cs);
      }
      join(origin);
    };
    auto run = [&](cudaStream_t origin) {
      if (panels) enqueue_panels(origin);
      else enqueue(origin);
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
          run(h->capture_stream);
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
      run(s);
    }
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
  });
}

}  // extern "C"

// Host runtime behind the C ABI of include/spmv_gb300.h: handle lifecycle, precision,
// variant installation by hand, runs on device buffers, exports of the pool data, CSR
// validation and the device error word. Classification and tuning live in tune.cu,
// host-buffer runs in host.cu, the selector in selector.cu, conjugate gradients in cg.cu.
#include "handle.h"

using namespace spmv;
using namespace spmv::rt;

namespace {

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
  drop_panels(h);   // the panel and slice copies hold values of the previous storage dtype
  drop_sell(h);
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

spmv_status spmv_create(spmv_handle_t *out, int64_t n_rows, int64_t n_cols, int64_t nnz,
                        const int32_t *row_ptr, const int32_t *col_ind, const void *val,
                        spmv_dtype val_type, int32_t device_ptrs, spmv_stream_t stream) {
  if (!out || !row_ptr || (nnz > 0 && (!col_ind || !val))) return SPMV_ERR_ARG;
  if (n_rows < 0 || n_cols < 0 || nnz < 0 || n_rows >= INT32_MAX || n_cols >= INT32_MAX ||
      nnz > SPMV_MAX_NNZ)
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
    if (h->pass_done) cudaEventDestroy(h->pass_done);
    cudaStreamDestroy(h->copy_stream);
    cudaStreamDestroy(h->copy_stream2);
    cudaStreamDestroy(h->upload_stream);
    cudaStreamDestroy(h->capture_stream);
    for (auto st : h->chunk_stream)
      if (st) cudaStreamDestroy(st);
  }
  delete h;   // every device buffer of the handle is a DevBuf and frees itself
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
      // no run until a variant is installed for the new storage
      h->tuned = false;
      ++h->epoch;
      h->storage = storage;
      try {
        install_storage(h, s);
        CK(cudaStreamSynchronize(s));
      } catch (...) {
        // back to the input dtype's defaults, whose values are always resident
        h->val_store.release();
        h->val_df.release();
        h->x_stage.release();
        h->y_stage.release();
        default_types(h->in_type, &h->storage, &h->vec, &h->acc);
        throw;
      }
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
    // untuned while the variant's buffers are rebuilt: a failure part way leaves no
    // installed variant pointing at released buffers
    h->tuned = false;
    ++h->epoch;
    spmv_variant w = *v;
    prepare_variant(h, w, s);
    h->variant = w;
    ++h->epoch;
    h->tuned = true;
    return SPMV_OK;
  });
}

spmv_status spmv_run(spmv_handle_t h, const void *x, void *y, spmv_stream_t stream) {
  if (!h) return SPMV_ERR_ARG;
  if (!h->tuned) return SPMV_ERR_NOT_TUNED;
  if ((h->n_cols > 0 && !x) || (h->n_rows > 0 && !y)) return SPMV_ERR_ARG;
  const cudaError_t e = launch_run(h, h->variant, x, y, static_cast<cudaStream_t>(stream));
  return map_err(e);
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

spmv_status spmv_get_sell(spmv_handle_t h, int64_t *slice_off, void *val, void *idx,
                          int64_t *n_positions, int32_t *idx_bits, spmv_stream_t stream) {
  if (!h || !n_positions || !idx_bits) return SPMV_ERR_ARG;
  if (h->sell_bits < 0) return SPMV_ERR_NOT_TUNED;
  *n_positions = h->sell_total;
  *idx_bits = h->sell_bits;
  if (!slice_off && !val && !idx) return SPMV_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    const size_t vb = h->storage == SPMV_DF64 ? 8 : dtype_bytes(h->storage);
    const size_t ib = h->sell_bits ? (size_t)(h->sell_bits / 8) : 4;
    const int64_t ns = (h->n_rows + 31) / 32;
    if (slice_off)
      CK(cudaMemcpyAsync(slice_off, h->sell_off.p, 8 * (size_t)(ns + 1), cudaMemcpyDeviceToDevice, s));
    if (val && h->sell_total)
      CK(cudaMemcpyAsync(val, h->sell_val.p, vb * (size_t)h->sell_total, cudaMemcpyDeviceToDevice, s));
    if (idx && h->sell_total)
      CK(cudaMemcpyAsync(idx, h->sell_idx.p, ib * (size_t)h->sell_total, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
  });
}

spmv_status spmv_get_col_panels(spmv_handle_t h, int32_t *panel_rowptr, int32_t *panel_col,
                                void *panel_val, int32_t *n_panels, int32_t *panel_cols,
                                spmv_stream_t stream) {
  if (!h || !n_panels || !panel_cols) return SPMV_ERR_ARG;
  if (h->pnl_count == 0) return SPMV_ERR_NOT_TUNED;
  *n_panels = h->pnl_count;
  *panel_cols = h->pnl_width;
  if (!panel_rowptr && !panel_col && !panel_val) return SPMV_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    const size_t vb = h->storage == SPMV_DF64 ? 8 : dtype_bytes(h->storage);
    if (panel_rowptr)
      CK(cudaMemcpyAsync(panel_rowptr, h->pnl_rowptr.p,
                         4 * (size_t)h->pnl_count * (size_t)(h->n_rows + 1),
                         cudaMemcpyDeviceToDevice, s));
    if (panel_col && h->nnz)
      CK(cudaMemcpyAsync(panel_col, h->pnl_col.p, 4 * (size_t)h->nnz, cudaMemcpyDeviceToDevice, s));
    if (panel_val && h->nnz)
      CK(cudaMemcpyAsync(panel_val, h->pnl_val.p, vb * (size_t)h->nnz, cudaMemcpyDeviceToDevice, s));
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
                          &h->x_stage, &h->y_stage, &h->scratch, &h->val_df, &h->bin_rows,
                          &h->bin_long_rows, &h->bin_long_first, &h->bin_chunks,
                          &h->bin_partials, &h->pnl_rowptr, &h->pnl_col, &h->pnl_val,
                          &h->sell_off, &h->sell_val, &h->sell_idx})
    t += (int64_t)b->bytes;
  *bytes = t;
  return SPMV_OK;
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
  if (acc == SPMV_DF64 && (val == SPMV_F32 || val == SPMV_BF16)) {
    if (vec == SPMV_F64) return val == SPMV_F32 ? kernel_set_f32_d_df() : kernel_set_bf16_d_df();
    if (vec == SPMV_F32) return val == SPMV_F32 ? kernel_set_f32_f_df() : kernel_set_bf16_f_df();
    return nullptr;
  }
  const bool dd = vec == SPMV_F64 && acc == SPMV_F64;
  const bool ff = vec == SPMV_F32 && acc == SPMV_F32;
  const bool fd = vec == SPMV_F32 && acc == SPMV_F64;
  if (val == SPMV_F32) return dd ? kernel_set_f32_dd() : ff ? kernel_set_f32_ff() : fd ? kernel_set_f32_fd() : nullptr;
  if (val == SPMV_BF16) return dd ? kernel_set_bf16_dd() : ff ? kernel_set_bf16_ff() : fd ? kernel_set_bf16_fd() : nullptr;
  return nullptr;
}
}  // namespace spmv

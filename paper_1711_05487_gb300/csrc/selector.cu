// The learned selector (Section III-D with an MLP in place of the decision tree): input
// normalization, logits, loss and gradient, Adam training and the per-matrix prediction.
#include "handle.h"

using namespace spmv;
using namespace spmv::rt;

extern "C" {

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

spmv_status spmv_selector_set_range(spmv_selector_t sel, const float *lo, const float *hi,
                                    float slack) {
  if (!sel || !lo || !hi || !(slack >= 0.0f)) return SPMV_ERR_ARG;
  for (int k = 0; k < SPMV_MLP_INPUTS; ++k)
    if (!(lo[k] <= hi[k])) return SPMV_ERR_ARG;
  std::memcpy(sel->in_lo, lo, sizeof sel->in_lo);
  std::memcpy(sel->in_hi, hi, sizeof sel->in_hi);
  sel->in_slack = slack;
  sel->has_range = true;
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
    float xin[SPMV_MLP_INPUTS];
    if (sel->has_range)
      CK(cudaMemcpyAsync(xin, x, sizeof xin, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool inside = true;
    if (sel->has_range)
      for (int k = 0; k < SPMV_MLP_INPUTS; ++k)
        inside = inside && xin[k] >= sel->in_lo[k] - sel->in_slack &&
                 xin[k] <= sel->in_hi[k] + sel->in_slack;
    uint32_t c = 0;
    double mg = 1e300;
    for (int o = 0; o < n3 && o < 4; ++o) {
      if (h[o] > 0.0f) c |= (1u << o);
      mg = std::min(mg, (double)std::fabs(h[o]));
    }
    *classes = c;
    if (margin) *margin = inside ? mg : -1.0;
    return SPMV_OK;
  });
}

}  // extern "C"

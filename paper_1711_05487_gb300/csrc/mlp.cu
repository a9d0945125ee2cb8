// Learned selector: a small MLP over Table I features (the stand-in for the paper's
// decision tree, Section III-D). Inference uses a fixed multiply-add order so that the
// class decision is reproducible bit for bit; training is full-batch backpropagation with
// FP64 sums over the batch and Adam updates.
//
// Layer sizes n0 -> n1 -> n2 -> n3, ReLU on the hidden layers, one logit per class.
// Parameters packed W1 (n1 x n0, row-major), b1, W2 (n2 x n1), b2, W3 (n3 x n2), b3.
#include "common.cuh"

namespace spmv {

namespace {
constexpr int kT = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

struct Layout {
  int n0, n1, n2, n3;
  int64_t w1, b1, w2, b2, w3, b3, total;
};

Layout layout(const int32_t *s) {
  Layout L;
  L.n0 = s[0]; L.n1 = s[1]; L.n2 = s[2]; L.n3 = s[3];
  L.w1 = 0;
  L.b1 = L.w1 + (int64_t)L.n1 * L.n0;
  L.w2 = L.b1 + L.n1;
  L.b2 = L.w2 + (int64_t)L.n2 * L.n1;
  L.w3 = L.b2 + L.n2;
  L.b3 = L.w3 + (int64_t)L.n3 * L.n2;
  L.total = L.b3 + L.n3;
  return L;
}
}  // namespace

int64_t mlp_param_count(const int32_t *sizes) { return layout(sizes).total; }

// ---------------------------------------------------------------- derived inputs ------
// log2(1 + v) for v >= 0 (0 for v <= 0 or NaN): w = 1 + v = m 2^e, m folded into
// [sqrt(2)/2, sqrt(2)], then log2(m) = (2/ln 2) atanh(t), t = (m-1)/(m+1), from the atanh
// series t + t^3/3 + ... + t^11/11 in Horner form. The _rn intrinsics keep the compiler
// from fusing or reordering anything, so every step rounds exactly as written.
__device__ float log2p1_f32(float v) {
  if (!(v > 0.0f)) return 0.0f;
  const float w = __fadd_rn(1.0f, v);
  const uint32_t u = __float_as_uint(w);
  int e = (int)((u >> 23) & 0xFFu) - 127;
  float m = __uint_as_float((u & 0x007FFFFFu) | 0x3F800000u);
  if (m > 1.41421356f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float t = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float t2 = __fmul_rn(t, t);
  float p = 1.0f / 11.0f;
  p = fmaf(p, t2, 1.0f / 9.0f);
  p = fmaf(p, t2, 1.0f / 7.0f);
  p = fmaf(p, t2, 1.0f / 5.0f);
  p = fmaf(p, t2, 1.0f / 3.0f);
  p = fmaf(p, t2, 1.0f);
  const float l = __fmul_rn(__fmul_rn(t, p), 2.88539008f);
  return __fadd_rn((float)e, l);
}

__device__ __forceinline__ double safe_div(double a, double b) { return b > 0.0 ? a / b : 0.0; }

// feat: 16 doubles per sample = 14 Table I features (size, density, nnz_min, nnz_max,
// nnz_avg, nnz_sd, bw_min, bw_max, bw_avg, bw_sd, scatter_avg, scatter_sd,
// clustering_avg, misses_avg), n_rows, nnz.
__global__ void k_mlp_inputs(const double *feat, int64_t batch, const float *mu,
                             const float *inv_sigma, float *X) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const double *f = feat + b * 16;
  float r[SPMV_MLP_INPUTS];
  r[0] = log2p1_f32((float)f[14]);
  r[1] = log2p1_f32((float)f[4]);
  r[2] = log2p1_f32((float)safe_div(f[5], f[4]));
  r[3] = log2p1_f32((float)f[3]);
  r[4] = log2p1_f32((float)safe_div(f[3], f[4]));
  r[5] = log2p1_f32((float)f[8]);
  r[6] = log2p1_f32((float)f[9]);
  r[7] = (float)f[10];
  r[8] = (float)f[11];
  r[9] = (float)f[12];
  r[10] = (float)safe_div(f[13], f[4]);
  r[11] = (float)f[0];
  for (int k = 0; k < SPMV_MLP_INPUTS; ++k) {
    float z = r[k];
    if (mu) z = __fmul_rn(__fsub_rn(z, mu[k]), inv_sigma[k]);
    X[b * SPMV_MLP_INPUTS + k] = z;
  }
}

cudaError_t launch_mlp_inputs(const double *feat, int64_t batch, const float *mu,
                              const float *inv_sigma, float *X, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  k_mlp_inputs<<<nblk(batch), kT, 0, s>>>(feat, batch, mu, inv_sigma, X);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ dense layers ------
// out[b, o] = act(bias[o] + sum_k W[o, k] in[b, k]), the sum taken as a chain of fmaf in
// k order starting from the bias.
__global__ void k_dense_fwd(const float *in, int64_t batch, int nin, const float *W,
                            const float *bias, int nout, int relu, float *out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= batch * nout) return;
  const int64_t b = idx / nout;
  const int o = (int)(idx % nout);
  const float *x = in + b * nin;
  const float *w = W + (int64_t)o * nin;
  float a = bias[o];
  for (int k = 0; k < nin; ++k) a = fmaf(w[k], x[k], a);
  out[idx] = relu ? (a > 0.0f ? a : 0.0f) : a;
}

// G[b, o] = (sigmoid(z) - y) / (batch * n3); term[b] = sum_o BCE-with-logits(z, y).
__global__ void k_out_grad(const float *Z, const float *Y, int64_t batch, int n3, float *G,
                           double *term) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const double inv = 1.0 / ((double)batch * (double)n3);
  double acc = 0.0;
  for (int o = 0; o < n3; ++o) {
    const double z = Z[b * n3 + o], y = Y[b * n3 + o];
    const double p = 1.0 / (1.0 + exp(-z));
    acc += (z > 0.0 ? z : 0.0) - y * z + log1p(exp(-fabs(z)));
    G[b * n3 + o] = (float)((p - y) * inv);
  }
  term[b] = acc;
}

// dW[o, k] = sum_b G[b, o] in[b, k], db[o] = sum_b G[b, o] (b in order, FP64 sums).
__global__ void k_dense_wgrad(const float *G, const float *in, int64_t batch, int nin, int nout,
                              float *dW, float *db) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nw = (int64_t)nout * nin;
  if (idx < nw) {
    const int o = (int)(idx / nin), k = (int)(idx % nin);
    double acc = 0.0;
    for (int64_t b = 0; b < batch; ++b) acc += (double)G[b * nout + o] * (double)in[b * nin + k];
    dW[idx] = (float)acc;
  } else if (idx < nw + nout) {
    const int o = (int)(idx - nw);
    double acc = 0.0;
    for (int64_t b = 0; b < batch; ++b) acc += (double)G[b * nout + o];
    db[o] = (float)acc;
  }
}

// Gin[b, k] = [act[b, k] > 0] * sum_o W[o, k] G[b, o]   (ReLU derivative)
__global__ void k_dense_dgrad(const float *G, const float *W, const float *act, int64_t batch,
                              int nin, int nout, float *Gin) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= batch * nin) return;
  const int64_t b = idx / nin;
  const int k = (int)(idx % nin);
  double acc = 0.0;
  for (int o = 0; o < nout; ++o) acc += (double)W[(int64_t)o * nin + k] * (double)G[b * nout + o];
  Gin[idx] = act[idx] > 0.0f ? (float)acc : 0.0f;
}

__global__ void k_loss_reduce(const double *term, int64_t batch, int n3, float *loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double acc = 0.0;
  for (int64_t b = 0; b < batch; ++b) acc += term[b];
  *loss = (float)(acc / ((double)batch * (double)n3));
}

int64_t mlp_logits_work_floats(const int32_t *sizes, int64_t batch) {
  const Layout L = layout(sizes);
  return batch * ((int64_t)L.n1 + L.n2);
}

// work: mlp_logits_work_floats(sizes, batch) floats of device memory for the hidden layers.
cudaError_t launch_mlp_logits_ws(const int32_t *sizes, const float *params, int64_t batch,
                                 const float *X, float *logits, float *work, cudaStream_t s) {
  const Layout L = layout(sizes);
  float *h1 = work, *h2 = work + batch * L.n1;
  k_dense_fwd<<<nblk(batch * L.n1), kT, 0, s>>>(X, batch, L.n0, params + L.w1, params + L.b1,
                                                L.n1, 1, h1);
  k_dense_fwd<<<nblk(batch * L.n2), kT, 0, s>>>(h1, batch, L.n1, params + L.w2, params + L.b2,
                                                L.n2, 1, h2);
  k_dense_fwd<<<nblk(batch * L.n3), kT, 0, s>>>(h2, batch, L.n2, params + L.w3, params + L.b3,
                                                L.n3, 0, logits);
  return cudaGetLastError();
}

cudaError_t launch_mlp_logits(const int32_t *sizes, const float *params, int64_t batch,
                              const float *X, float *logits, cudaStream_t s) {
  float *work = nullptr;
  cudaError_t e = cudaMallocAsync(&work, sizeof(float) * (size_t)mlp_logits_work_floats(sizes, batch), s);
  if (e != cudaSuccess) return e;
  e = launch_mlp_logits_ws(sizes, params, batch, X, logits, work, s);
  cudaFreeAsync(work, s);
  return e;
}

// Work area (floats): H1, H2, Z, G3, G2, G1, then 2 * batch floats holding FP64 terms.
int64_t mlp_work_floats(const int32_t *sizes, int64_t batch) {
  const Layout L = layout(sizes);
  return batch * (2 * (int64_t)L.n1 + 2 * (int64_t)L.n2 + 2 * (int64_t)L.n3) + 2 * batch + 2;
}

cudaError_t launch_mlp_loss_grad(const int32_t *sizes, const float *params, int64_t batch,
                                 const float *X, const float *Y, float *grad, float *loss,
                                 float *work, cudaStream_t s) {
  const Layout L = layout(sizes);
  float *H1 = work, *H2 = H1 + batch * L.n1, *Z = H2 + batch * L.n2, *G3 = Z + batch * L.n3,
        *G2 = G3 + batch * L.n3, *G1 = G2 + batch * L.n2;
  // FP64 terms start at an 8-byte aligned float offset
  int64_t off = (int64_t)((G1 + batch * L.n1) - work);
  off = (off + 1) & ~(int64_t)1;
  double *term = reinterpret_cast<double *>(work + off);
  k_dense_fwd<<<nblk(batch * L.n1), kT, 0, s>>>(X, batch, L.n0, params + L.w1, params + L.b1,
                                                L.n1, 1, H1);
  k_dense_fwd<<<nblk(batch * L.n2), kT, 0, s>>>(H1, batch, L.n1, params + L.w2, params + L.b2,
                                                L.n2, 1, H2);
  k_dense_fwd<<<nblk(batch * L.n3), kT, 0, s>>>(H2, batch, L.n2, params + L.w3, params + L.b3,
                                                L.n3, 0, Z);
  k_out_grad<<<nblk(batch), kT, 0, s>>>(Z, Y, batch, L.n3, G3, term);
  k_loss_reduce<<<1, 32, 0, s>>>(term, batch, L.n3, loss);
  k_dense_wgrad<<<nblk((int64_t)L.n3 * L.n2 + L.n3), kT, 0, s>>>(G3, H2, batch, L.n2, L.n3,
                                                                grad + L.w3, grad + L.b3);
  k_dense_dgrad<<<nblk(batch * L.n2), kT, 0, s>>>(G3, params + L.w3, H2, batch, L.n2, L.n3, G2);
  k_dense_wgrad<<<nblk((int64_t)L.n2 * L.n1 + L.n2), kT, 0, s>>>(G2, H1, batch, L.n1, L.n2,
                                                                grad + L.w2, grad + L.b2);
  k_dense_dgrad<<<nblk(batch * L.n1), kT, 0, s>>>(G2, params + L.w2, H1, batch, L.n1, L.n2, G1);
  k_dense_wgrad<<<nblk((int64_t)L.n1 * L.n0 + L.n1), kT, 0, s>>>(G1, X, batch, L.n0, L.n1,
                                                                grad + L.w1, grad + L.b1);
  return cudaGetLastError();
}

// Adam (Kingma & Ba, 2015) with bias correction; t is the 1-based step number.
__global__ void k_adam(int64_t n, float *p, const float *g, float *m, float *v, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

cudaError_t launch_adam(int64_t n, float *p, const float *g, float *m, float *v, float lr,
                        float b1, float b2, float eps, int32_t t, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  k_adam<<<nblk(n), kT, 0, s>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace spmv

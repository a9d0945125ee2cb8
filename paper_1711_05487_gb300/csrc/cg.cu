// Conjugate gradients (Hestenes and Stiefel, 1952) on a tuned SpMV handle: the iterative
// solver whose repeated y = A x amortizes the optimizer's preprocessing (Section IV-D). The
// SpMV is the handle's pool variant; the vector kernels here are FP64 and deterministic:
// every dot product uses a fixed grid, a fixed per-thread element order and a fixed tree,
// so a solve repeats bit for bit. Scalars stay on the device; the host reads the residual
// only every `check_every` iterations.
#include "common.cuh"
#include "handle.h"

namespace spmv {

namespace {
constexpr int kRedThreads = 256;

// Block sum in a fixed order: shuffle tree within warps, then warp 0 over the warp sums.
__device__ __forceinline__ double block_sum(double v, double *sh) {
  v = group_sum<32>(v, 0xffffffffu);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    t = group_sum<32>(t, 0xffffffffu);
  }
  __syncthreads();
  return t;   // valid in thread 0
}
}  // namespace

// part[b] = sum over the elements i = b*T + t + k*G*T of block b of a_i * b_i.
__global__ void __launch_bounds__(kRedThreads)
k_dot_partial(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
              double *__restrict__ part) {
  __shared__ double sh[kRedThreads / 32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out = sum of part[0 .. n_part) in a fixed order; optionally also hist = sqrt(out).
__global__ void __launch_bounds__(kRedThreads)
k_sum_final(const double *__restrict__ part, int n_part, double *out, double *hist) {
  __shared__ double sh[kRedThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n_part; i += blockDim.x) s += part[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    *out = s;
    if (hist) *hist = sqrt(s);
  }
}

// r = b - Ax, p = r, part = block sums of r.r
__global__ void __launch_bounds__(kRedThreads)
k_cg_start(const double *__restrict__ b, const double *__restrict__ ax, double *__restrict__ r,
           double *__restrict__ p, int64_t n, double *__restrict__ part) {
  __shared__ double sh[kRedThreads / 32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = b[i] - ax[i];
    r[i] = ri;
    p[i] = ri;
    s = fma(ri, ri, s);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// alpha = rr / pAp (0 if pAp = 0); x += alpha p; r -= alpha Ap; part = block sums of r.r
__global__ void __launch_bounds__(kRedThreads)
k_cg_xr(const double *__restrict__ p, const double *__restrict__ ap, double *__restrict__ x,
        double *__restrict__ r, int64_t n, const double *rr, const double *pap,
        double *__restrict__ part) {
  __shared__ double sh[kRedThreads / 32];
  const double d = *pap;
  const double alpha = d != 0.0 ? *rr / d : 0.0;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, ap[i], r[i]);
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// beta = rr_new / rr (0 if rr = 0); p = r + beta p
__global__ void __launch_bounds__(kRedThreads)
k_cg_p(const double *__restrict__ r, double *__restrict__ p, int64_t n, const double *rr,
       const double *rr_new) {
  const double d = *rr;
  const double beta = d != 0.0 ? *rr_new / d : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], r[i]);
}

int cg_reduce_blocks() {
  static const int blocks = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return 4 * (sms > 0 ? sms : 1);
  }();
  return blocks;
}

cudaError_t launch_dot(const double *a, const double *b, int64_t n, double *part, double *out,
                       double *hist, cudaStream_t s) {
  const int g = cg_reduce_blocks();
  k_dot_partial<<<g, kRedThreads, 0, s>>>(a, b, n, part);
  k_sum_final<<<1, kRedThreads, 0, s>>>(part, g, out, hist);
  return cudaGetLastError();
}

cudaError_t launch_cg_start(const double *b, const double *ax, double *r, double *p, int64_t n,
                            double *part, double *rr, double *hist, cudaStream_t s) {
  const int g = cg_reduce_blocks();
  k_cg_start<<<g, kRedThreads, 0, s>>>(b, ax, r, p, n, part);
  k_sum_final<<<1, kRedThreads, 0, s>>>(part, g, rr, hist);
  return cudaGetLastError();
}

cudaError_t launch_cg_xr(const double *p, const double *ap, double *x, double *r, int64_t n,
                         const double *rr, const double *pap, double *part, double *rr_new,
                         double *hist, cudaStream_t s) {
  const int g = cg_reduce_blocks();
  k_cg_xr<<<g, kRedThreads, 0, s>>>(p, ap, x, r, n, rr, pap, part);
  k_sum_final<<<1, kRedThreads, 0, s>>>(part, g, rr_new, hist);
  return cudaGetLastError();
}

cudaError_t launch_cg_p(const double *r, double *p, int64_t n, const double *rr,
                        const double *rr_new, cudaStream_t s) {
  k_cg_p<<<cg_reduce_blocks(), kRedThreads, 0, s>>>(r, p, n, rr, rr_new);
  return cudaGetLastError();
}

}  // namespace spmv

using namespace spmv;
using namespace spmv::rt;

extern "C" {

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

}  // extern "C"

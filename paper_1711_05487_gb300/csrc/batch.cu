// Batched SpMV / SpMM over many matrices of uneven sizes in one persistent launch.
//
// The host plans work items (row blocks of about equal nonzero counts; rows longer than a
// chunk are split into nonzero chunks, the matrix decomposition of Fig. 4/5). A grid of
// resident CTAs takes items from a device counter with atomicAdd -- no CTA ever waits on
// another -- and k_batch_fixup adds the chunks of split rows in chunk order, in FP64.
// Storage, x/y and accumulation are FP32; every matrix has k in {1, 4, 16} right-hand
// sides (row-major X and Y).
#include "common.cuh"

namespace spmv {

namespace {
constexpr int kBT = 256;
}

template <int K>
__device__ __forceinline__ void load_xrow(const float *p, float *o) {
  if constexpr (K == 1) {
    o[0] = __ldg(p);
  } else {
#pragma unroll
    for (int q = 0; q < K; q += 4) {
      const uint4 u = ld_nc_u4(p + q);
      o[q] = __uint_as_float(u.x);
      o[q + 1] = __uint_as_float(u.y);
      o[q + 2] = __uint_as_float(u.z);
      o[q + 3] = __uint_as_float(u.w);
    }
  }
}

// Rows [r0, r1) of one matrix, a sub-warp of vs lanes per row.
template <int K, int VS>
__device__ void batch_rows(const BatchMat &m, int r0, int r1) {
  constexpr int GROUPS = kBT / VS;
  const int lane = threadIdx.x & (VS - 1);
  const unsigned mask = group_mask<VS>();
  for (int row = r0 + (int)threadIdx.x / VS; row < r1; row += GROUPS) {
    const int s = __ldg(m.rowptr + row), e = __ldg(m.rowptr + row + 1);
    float acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = 0.0f;
    for (int j = s + lane; j < e; j += VS) {
      const float v = __ldg(m.val + j);
      float xr[K];
      load_xrow<K>(m.X + (int64_t)__ldg(m.colind + j) * K, xr);
#pragma unroll
      for (int q = 0; q < K; ++q) acc[q] = fmaf(v, xr[q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const float r = group_sum<VS>(acc[q], mask);
      if (lane == 0) m.Y[(int64_t)row * K + q] = r;
    }
  }
}

template <int K>
__device__ void batch_rows_k(const BatchMat &m, int r0, int r1) {
  switch (m.vs) {
    case 2: batch_rows<K, 2>(m, r0, r1); break;
    case 4: batch_rows<K, 4>(m, r0, r1); break;
    case 8: batch_rows<K, 8>(m, r0, r1); break;
    case 16: batch_rows<K, 16>(m, r0, r1); break;
    default: batch_rows<K, 32>(m, r0, r1); break;
  }
}

// Nonzeros [z0, z1) of one long row, the whole CTA: FP32 per-thread sums, then a fixed
// tree reduction in FP64 into partial slot `chunk` (16 doubles per slot, k used).
template <int K>
__device__ void batch_chunk(const BatchMat &m, int z0, int z1, int chunk, double *partials) {
  __shared__ double red[kBT];
  float acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0.0f;
  for (int j = z0 + (int)threadIdx.x; j < z1; j += kBT) {
    const float v = __ldg(m.val + j);
    float xr[K];
    load_xrow<K>(m.X + (int64_t)__ldg(m.colind + j) * K, xr);
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = fmaf(v, xr[q], acc[q]);
  }
  for (int q = 0; q < K; ++q) {
    red[threadIdx.x] = (double)acc[q];
    __syncthreads();
    for (int off = kBT / 2; off > 0; off >>= 1) {
      if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x == 0) partials[(int64_t)chunk * 16 + q] = red[0];
    __syncthreads();
  }
}

__device__ void batch_item(const BatchMat *mats, const BatchItem &it, double *partials) {
  const BatchMat m = mats[it.mat];
  if (it.chunk < 0) {
    switch (m.k) {
      case 1: batch_rows_k<1>(m, it.row_begin, it.row_end); break;
      case 4: batch_rows_k<4>(m, it.row_begin, it.row_end); break;
      default: batch_rows_k<16>(m, it.row_begin, it.row_end); break;
    }
  } else {
    switch (m.k) {
      case 1: batch_chunk<1>(m, it.nz_begin, it.nz_end, it.chunk, partials); break;
      case 4: batch_chunk<4>(m, it.nz_begin, it.nz_end, it.chunk, partials); break;
      default: batch_chunk<16>(m, it.nz_begin, it.nz_end, it.chunk, partials); break;
    }
  }
}

__global__ void __launch_bounds__(kBT)
k_batch_persistent(const BatchMat *mats, const BatchItem *items, int32_t n_items,
                   int32_t *counter, double *partials) {
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    batch_item(mats, items[it], partials);
  }
}

// One CTA per item (the same work without persistence).
__global__ void __launch_bounds__(kBT)
k_batch_items(const BatchMat *mats, const BatchItem *items, int32_t n_items, double *partials) {
  if ((int)blockIdx.x >= n_items) return;
  batch_item(mats, items[blockIdx.x], partials);
}

__global__ void k_batch_fixup(const BatchMat *mats, const BatchFix *fix, int32_t n_fix,
                              const double *partials) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_fix * 16) return;
  const BatchFix f = fix[idx / 16];
  const int q = (int)(idx % 16);
  const BatchMat m = mats[f.mat];
  if (q >= m.k) return;
  double tot = 0.0;
  for (int c = 0; c < f.count; ++c) tot += partials[(int64_t)(f.first + c) * 16 + q];
  m.Y[(int64_t)f.row * m.k + q] = (float)tot;
}

int batch_blocks_per_sm() {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_persistent, kBT, 0);
  return b > 0 ? b : 1;
}

cudaError_t launch_batch_persistent(const BatchMat *mats, const BatchItem *items,
                                    int32_t n_items, int32_t *counter, double *partials,
                                    int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  if (n_items <= 0) return cudaSuccess;
  k_batch_persistent<<<grid, kBT, 0, s>>>(mats, items, n_items, counter, partials);
  return cudaGetLastError();
}

cudaError_t launch_batch_items(const BatchMat *mats, const BatchItem *items, int32_t n_items,
                               double *partials, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  k_batch_items<<<n_items, kBT, 0, s>>>(mats, items, n_items, partials);
  return cudaGetLastError();
}

cudaError_t launch_batch_fixup(const BatchMat *mats, const BatchFix *fix, int32_t n_fix,
                               const double *partials, cudaStream_t s) {
  if (n_fix <= 0) return cudaSuccess;
  const int64_t n = (int64_t)n_fix * 16;
  k_batch_fixup<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mats, fix, n_fix, partials);
  return cudaGetLastError();
}

}  // namespace spmv

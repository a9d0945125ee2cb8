// Batched SpMV / SpMM over many matrices of uneven sizes in one persistent launch.
//
// The host plans work items (row blocks of about equal nonzero counts; rows longer than a
// chunk are split into nonzero chunks, the matrix decomposition of Fig. 4/5) and sorts them
// longest first. One resident kernel walks them all: every warp takes the next item from a
// device counter with atomicAdd (no warp or CTA ever waits on another) and runs the code of
// its matrix's right-hand-side count k in {1, 4, 16}; a row-block item is computed by
// sub-warps of the matrix's width, a chunk of a long row by the whole warp into an FP64
// partial slot, and k_batch_fixup adds
// the chunks of each split row in chunk order, in FP64. Storage and x/y are FP32; the
// accumulation is FP32, in runs of at most kF32Run products per lane added into FP32 pairs
// wherever a lane's chain would pass kF32Chain roundings, so every row stays within the
// FP32 bound; X and Y are row-major (n x k).
#include "common.cuh"

namespace spmv {

namespace {
constexpr int kBT = 256;
}

// True when a lane's FP32 chain over a row of len products spread over `lanes` lanes (its
// products plus the log2(LANES) levels of the lane reduction) would pass kF32Chain roundings.
template <int LANES>
__device__ __forceinline__ bool f32_chain_too_long(int len, int lanes) {
  constexpr int levels = LANES >= 32 ? 5 : LANES >= 16 ? 4 : LANES >= 8 ? 3 : LANES >= 4 ? 2
                                                                             : LANES >= 2 ? 1 : 0;
  return (len + lanes - 1) / lanes + levels > kF32Chain;
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

// Rows [r0, r1) of one matrix by one warp: sub-warps of VS lanes, one row each, U rows per
// sub-warp at a time. The U rows' bounds, values, columns and x rows are loaded together
// before any multiply-add, so U chains of dependent loads are in flight per lane instead of
// one. Each row's lane sums and their reduction keep the order of a single-row walk.
// FOLD (rows whose FP32 chain per lane would pass kF32Chain roundings): every lane adds its
// FP32 sum into an FP32 pair after each run of kF32Run products and the lane reduction adds
// the pairs, which keeps a long row within the FP32 bound; short rows stay in plain FP32.
template <int K, int VS, int U, bool FOLD>
__device__ __forceinline__ void warp_rows_group(const BatchMat &m, int row0, int r1, int sl,
                                                unsigned mask, const int (&s)[U],
                                                const int (&e)[U], int maxlen) {
  constexpr int GROUPS = 32 / VS;
  float acc[U][K];
  FPair tot[FOLD ? U : 1][FOLD ? K : 1];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int q = 0; q < K; ++q) acc[u][q] = 0.0f;
  int steps = 0;
  for (int off = sl; off < maxlen; off += VS) {
    float v[U];
    int c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = s[u] + off;
      const bool ok = j < e[u];
      v[u] = ok ? __ldg(m.val + j) : 0.0f;
      c[u] = ok ? __ldg(m.colind + j) : -1;
    }
    float xr[U][K];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (c[u] >= 0) {
        load_xrow<K>(m.X + (int64_t)c[u] * K, xr[u]);
      } else {
#pragma unroll
        for (int q = 0; q < K; ++q) xr[u][q] = 0.0f;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int q = 0; q < K; ++q) acc[u][q] = fmaf(v[u], xr[u][q], acc[u][q]);
    if constexpr (FOLD) {
      if (++steps == kF32Run) {
        steps = 0;
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int q = 0; q < K; ++q) {
            wadd(tot[u][q], acc[u][q]);
            acc[u][q] = 0.0f;
          }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int row = row0 + u * GROUPS;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      float r;
      if constexpr (FOLD) {
        wadd(tot[u][q], acc[u][q]);
        r = wvalue(group_sum<VS>(tot[u][q], mask));
      } else {
        r = group_sum<VS>(acc[u][q], mask);
      }
      if (sl == 0 && row < r1) m.Y[(int64_t)row * K + q] = r;
    }
  }
}

template <int K, int VS, int U>
__device__ void warp_rows(const BatchMat &m, int r0, int r1, int lane) {
  constexpr int GROUPS = 32 / VS;
  const int sl = lane & (VS - 1);
  const unsigned mask = group_mask<VS>();
  for (int row0 = r0 + lane / VS; row0 < r1; row0 += GROUPS * U) {
    int s[U], e[U];
    int maxlen = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int row = row0 + u * GROUPS;
      s[u] = 0;
      e[u] = 0;
      if (row < r1) {
        s[u] = __ldg(m.rowptr + row);
        e[u] = __ldg(m.rowptr + row + 1);
      }
      maxlen = max(maxlen, e[u] - s[u]);
    }
    // uniform over the sub-warp (its lanes share the U rows): a lane's FP32 chain is its
    // products plus the log2(VS) levels of the lane reduction
    if (f32_chain_too_long<VS>(maxlen, VS)) {
      if constexpr (K == 1) {
        warp_rows_group<K, VS, U, true>(m, row0, r1, sl, mask, s, e, maxlen);
      } else {
        // wider right-hand sides fold one row at a time (the pairs of U rows would cost
        // occupancy); such a row has more than kF32Chain / 2 products per lane anyway
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int su[1] = {s[u]}, eu[1] = {e[u]};
          warp_rows_group<K, VS, 1, true>(m, row0 + u * GROUPS, r1, sl, mask, su, eu,
                                          e[u] - s[u]);
        }
      }
    } else {
      warp_rows_group<K, VS, U, false>(m, row0, r1, sl, mask, s, e, maxlen);
    }
  }
}

// K = 16: the four lanes of a quad share a nonzero, each gathering one 16-byte quarter of
// its x row and keeping 4 accumulators, so a sub-warp of VS lanes has VS / 4 nonzeros of its
// row in flight (two per quad per step) instead of one 64-byte gather per lane. The two
// nonzeros of a step go to two accumulator sets (even and odd steps' halves of the lane's
// share), two independent FMA chains of half the length; their sum and the quads' sums of
// one row are added with a fixed shuffle tree; the quad of slot 0 writes the row.
// FOLD (rows whose chains would pass kF32Chain roundings): each chain's FP32 sums of kF32Run
// products are added into FP32 pairs, and the quads' pairs are added.
template <int VS, bool FOLD>
__device__ __forceinline__ void row_k16(const BatchMat &m, int row, int s, int e, int slot,
                                        int quad, unsigned mask) {
  constexpr int SLOTS = VS / 4;
  float a0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, a1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  FPair tot[4];
  int steps = 0;
  int j = s + slot;
  for (; j + SLOTS < e; j += 2 * SLOTS) {
    const float v0 = __ldg(m.val + j), v1 = __ldg(m.val + j + SLOTS);
    const int c0 = __ldg(m.colind + j), c1 = __ldg(m.colind + j + SLOTS);
    const uint4 x0 = ld_nc_u4(m.X + (int64_t)c0 * 16 + quad * 4);
    const uint4 x1 = ld_nc_u4(m.X + (int64_t)c1 * 16 + quad * 4);
    a0[0] = fmaf(v0, __uint_as_float(x0.x), a0[0]);
    a0[1] = fmaf(v0, __uint_as_float(x0.y), a0[1]);
    a0[2] = fmaf(v0, __uint_as_float(x0.z), a0[2]);
    a0[3] = fmaf(v0, __uint_as_float(x0.w), a0[3]);
    a1[0] = fmaf(v1, __uint_as_float(x1.x), a1[0]);
    a1[1] = fmaf(v1, __uint_as_float(x1.y), a1[1]);
    a1[2] = fmaf(v1, __uint_as_float(x1.z), a1[2]);
    a1[3] = fmaf(v1, __uint_as_float(x1.w), a1[3]);
    if constexpr (FOLD) {
      if (++steps == kF32Run) {
        steps = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          wadd(tot[q], a0[q]);
          wadd(tot[q], a1[q]);
          a0[q] = 0.0f;
          a1[q] = 0.0f;
        }
      }
    }
  }
  if (j < e) {
    const float v0 = __ldg(m.val + j);
    const uint4 x0 = ld_nc_u4(m.X + (int64_t)__ldg(m.colind + j) * 16 + quad * 4);
    a0[0] = fmaf(v0, __uint_as_float(x0.x), a0[0]);
    a0[1] = fmaf(v0, __uint_as_float(x0.y), a0[1]);
    a0[2] = fmaf(v0, __uint_as_float(x0.z), a0[2]);
    a0[3] = fmaf(v0, __uint_as_float(x0.w), a0[3]);
  }
  float r[4];
  if constexpr (FOLD) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      FPair t = tot[q];
      wadd(t, a0[q]);
      wadd(t, a1[q]);
#pragma unroll
      for (int off = 4; off < VS; off <<= 1) {
        FPair o;
        o.hi = __shfl_xor_sync(mask, t.hi, off, VS);
        o.lo = __shfl_xor_sync(mask, t.lo, off, VS);
        wadd(t, o);
      }
      r[q] = wvalue(t);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) r[q] = a0[q] + a1[q];
#pragma unroll
    for (int off = 4; off < VS; off <<= 1)
#pragma unroll
      for (int q = 0; q < 4; ++q) r[q] += __shfl_xor_sync(mask, r[q], off, VS);
  }
  if (slot == 0)
    *reinterpret_cast<float4 *>(m.Y + (int64_t)row * 16 + quad * 4) =
        make_float4(r[0], r[1], r[2], r[3]);
}

template <int VS>
__device__ void warp_rows_k16(const BatchMat &m, int r0, int r1, int lane) {
  static_assert(VS >= 4, "a quad per nonzero");
  constexpr int GROUPS = 32 / VS, SLOTS = VS / 4;
  const int sl = lane & (VS - 1), slot = sl >> 2, quad = sl & 3;
  const unsigned mask = group_mask<VS>();
  for (int row = r0 + lane / VS; row < r1; row += GROUPS) {
    const int s = __ldg(m.rowptr + row), e = __ldg(m.rowptr + row + 1);
    // a lane's two chains hold about half of its ceil(len / SLOTS) products each, plus the
    // sum of the two and the levels of the lane reduction
    const int per_lane = (e - s + SLOTS - 1) / SLOTS;
    if (f32_chain_too_long<SLOTS>((per_lane + 1) / 2 + 1, 1))
      row_k16<VS, true>(m, row, s, e, slot, quad, mask);
    else
      row_k16<VS, false>(m, row, s, e, slot, quad, mask);
  }
}

// rows in flight per lane: more for narrow right-hand sides (registers: U * K accumulators)
template <int K> struct RowsInFlight {
  static constexpr int value = K == 1 ? 4 : (K == 4 ? 2 : 1);
};

template <int K>
__device__ void warp_rows_vs(const BatchMat &m, int r0, int r1, int lane) {
  constexpr int U = RowsInFlight<K>::value;
  if constexpr (K == 16) {
    switch (m.vs) {
      case 1: case 2: case 4: warp_rows_k16<4>(m, r0, r1, lane); break;
      case 8: warp_rows_k16<8>(m, r0, r1, lane); break;
      case 16: warp_rows_k16<16>(m, r0, r1, lane); break;
      default: warp_rows_k16<32>(m, r0, r1, lane); break;
    }
    return;
  }
  switch (m.vs) {
    case 1: warp_rows<K, 1, U>(m, r0, r1, lane); break;
    case 2: warp_rows<K, 2, U>(m, r0, r1, lane); break;
    case 4: warp_rows<K, 4, U>(m, r0, r1, lane); break;
    case 8: warp_rows<K, 8, U>(m, r0, r1, lane); break;
    case 16: warp_rows<K, 16, U>(m, r0, r1, lane); break;
    default: warp_rows<K, 32, U>(m, r0, r1, lane); break;
  }
}

// Nonzeros [z0, z1) of one long row by one warp: FP32 lane sums of at most kF32Run
// products at a time, added into FP32 pairs, then (once per lane) a fixed shuffle tree in
// FP64 into partial slot `chunk` (16 doubles per slot, k used).
// K = 16: eight slots of a quad each (as in warp_rows_k16); the slots' sums are added in
// FP64 with a fixed shuffle tree and the quad of slot 0 writes the 16 partials.
__device__ void warp_chunk_k16(const BatchMat &m, int z0, int z1, int chunk, double *partials,
                               int lane) {
  const int slot = lane >> 2, quad = lane & 3;
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  FPair w[4];
  int steps = 0;
  int j = z0 + slot;
  for (; j + 8 < z1; j += 16) {
    const float v0 = __ldg(m.val + j), v1 = __ldg(m.val + j + 8);
    const int c0 = __ldg(m.colind + j), c1 = __ldg(m.colind + j + 8);
    const uint4 x0 = ld_nc_u4(m.X + (int64_t)c0 * 16 + quad * 4);
    const uint4 x1 = ld_nc_u4(m.X + (int64_t)c1 * 16 + quad * 4);
    acc[0] = fmaf(v1, __uint_as_float(x1.x), fmaf(v0, __uint_as_float(x0.x), acc[0]));
    acc[1] = fmaf(v1, __uint_as_float(x1.y), fmaf(v0, __uint_as_float(x0.y), acc[1]));
    acc[2] = fmaf(v1, __uint_as_float(x1.z), fmaf(v0, __uint_as_float(x0.z), acc[2]));
    acc[3] = fmaf(v1, __uint_as_float(x1.w), fmaf(v0, __uint_as_float(x0.w), acc[3]));
    if (++steps == kF32Run / 2) {
      steps = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        wadd(w[q], acc[q]);
        acc[q] = 0.0f;
      }
    }
  }
  if (j < z1) {
    const float v0 = __ldg(m.val + j);
    const uint4 x0 = ld_nc_u4(m.X + (int64_t)__ldg(m.colind + j) * 16 + quad * 4);
    acc[0] = fmaf(v0, __uint_as_float(x0.x), acc[0]);
    acc[1] = fmaf(v0, __uint_as_float(x0.y), acc[1]);
    acc[2] = fmaf(v0, __uint_as_float(x0.z), acc[2]);
    acc[3] = fmaf(v0, __uint_as_float(x0.w), acc[3]);
  }
  double t[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    wadd(w[q], acc[q]);
    t[q] = wdouble(w[q]);
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) t[q] += __shfl_xor_sync(0xffffffffu, t[q], off);
  }
  if (slot == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) partials[(int64_t)chunk * 16 + quad * 4 + q] = t[q];
  }
}

template <int K>
__device__ void warp_chunk(const BatchMat &m, int z0, int z1, int chunk, double *partials,
                           int lane) {
  if constexpr (K == 16) {
    warp_chunk_k16(m, z0, z1, chunk, partials, lane);
    return;
  }
  float acc[K];
  FPair w[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0.0f;
  int steps = 0;
  // two elements per lane per step: both loads issue before the multiply-adds, which then
  // run in element order
  int j = z0 + lane;
  for (; j + 32 < z1; j += 64) {
    const float v0 = __ldg(m.val + j), v1 = __ldg(m.val + j + 32);
    const int c0 = __ldg(m.colind + j), c1 = __ldg(m.colind + j + 32);
    float x0[K], x1[K];
    load_xrow<K>(m.X + (int64_t)c0 * K, x0);
    load_xrow<K>(m.X + (int64_t)c1 * K, x1);
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = fmaf(v1, x1[q], fmaf(v0, x0[q], acc[q]));
    if (++steps == kF32Run / 2) {
      steps = 0;
#pragma unroll
      for (int q = 0; q < K; ++q) {
        wadd(w[q], acc[q]);
        acc[q] = 0.0f;
      }
    }
  }
  if (j < z1) {
    const float v = __ldg(m.val + j);
    float xr[K];
    load_xrow<K>(m.X + (int64_t)__ldg(m.colind + j) * K, xr);
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = fmaf(v, xr[q], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    wadd(w[q], acc[q]);
    const double r = group_sum<32>(wdouble(w[q]), 0xffffffffu);
    if (lane == 0) partials[(int64_t)chunk * 16 + q] = r;
  }
}

template <int K>
__device__ __forceinline__ void run_item(const BatchMat &m, const BatchItem &item,
                                         double *partials, int lane) {
  if (item.chunk < 0) warp_rows_vs<K>(m, item.row_begin, item.row_end, lane);
  else warp_chunk<K>(m, item.nz_begin, item.nz_end, item.chunk, partials, lane);
}

// The whole batch in one persistent launch: a resident grid whose warps take the next work
// item from one device counter (atomicAdd; no warp or CTA ever waits on another) and run it
// with the code of its matrix's right-hand-side count.
__global__ void __launch_bounds__(kBT)
k_batch_persistent(const BatchMat *mats, const BatchItem *items, int32_t n_items,
                   int32_t *counter, double *partials) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(counter, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= n_items) break;
    const BatchItem item = items[it];
    const BatchMat m = mats[item.mat];
    if (m.k == 1) run_item<1>(m, item, partials, lane);
    else if (m.k == 4) run_item<4>(m, item, partials, lane);
    else run_item<16>(m, item, partials, lane);
  }
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
  if (n_items <= 0 || grid <= 0) return cudaSuccess;
  k_batch_persistent<<<grid, kBT, 0, s>>>(mats, items, n_items, counter, partials);
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

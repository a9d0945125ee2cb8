// Thread-per-row tile kernels (sub-warp width 1) and their launchers: a tile of 32, 64 or
// 128 consecutive rows is staged into shared memory by bulk asynchronous copies (TMA) and
// each thread walks its own row with one fused multiply-add per nonzero (CMP on GB300's
// FP64 pipe; MB with 16-bit column deltas).
//  k_rowtile       - one tile per CTA;
//  k_rowtile_pipe  - persistent CTAs keeping the next tile's bulk copy in flight.
// Included by spmv_kernels.cuh; kept apart so that a measurement of these kernels can name
// exactly the sources it was taken on.
#pragma once

#include <atomic>
#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace spmv {

// ----------------------------------------------------------------------- k_rowtile ----
// One thread per row over a tile of blockDim.x (32, 64 or 128) consecutive rows (sub-warp
// width 1). The
// tile's values and column indices (int32 or 16-bit deltas) are staged into shared memory
// by two bulk asynchronous copies (TMA) completing on an mbarrier, so the DRAM stream is
// fully coalesced whatever the row lengths; then each thread walks its own row with one
// fused multiply-add per nonzero and no cross-lane reduction. On GB300 the FP64 pipe
// retires only ~2 FMA lanes per clock per SM, so spending exactly one FP64 instruction per
// nonzero is what lets FP64 SpMV reach the memory roofline. A tile whose staged size
// exceeds tile_cap is computed from global memory instead (a warp per row).
template <typename ValT, typename IdxT>
__host__ __device__ constexpr int tile_elem_bytes() {
  return (int)(sizeof(ValT) + sizeof(IdxT));
}

// FP64 rows with delta-coded columns are summed in two FMA chains: element k of a row of
// length len goes to chain 1 when k is odd and lies in the row's 8-element blocks
// (k < len rounded down to a multiple of 8), to chain 0 otherwise, and the row's value is
// chain 0 + chain 1 (one FP64 add per row). On GB300 this ran the 27-point stencil 3 %
// faster than one chain; with int32 columns one chain was faster, so those rows keep it.
// The double-float kernel's FP64 fallback uses the same assignment to stay bit-identical.
__device__ __forceinline__ int fp64_chain_of(int k, int len) {
  return k < (len & ~7) ? (k & 1) : 0;
}

// Dot product of one row whose values and columns sit in shared memory at offset o (the
// row's first element) of a staged tile: 16 (then 8) gathers of x in flight per thread
// before their FMAs; exact trip counts keep the FP64 pipe free of masked-off work.
template <typename ValT, typename VecT, typename AccT, int DB, bool XL2, bool NA = false,
          typename IdxT>
__device__ __forceinline__ AccT tile_row_dot(const RunArgs &a, const ValT *sval,
                                             const IdxT *sidx, int o, int len, int32_t base,
                                             const VecT *__restrict__ x, uint64_t pol_x) {
  AccT acc = 0;
  // Column of element k: int32 from shared memory, or the running sum of 16-bit deltas
  // from the row's base column, or (escape rows) the full column kept in global memory.
  const int32_t *ec = nullptr;
  int c = base;
  if constexpr (DB != 0) {
    if (base < 0) ec = a.esc + (-(int64_t)base - 1);
  }
  auto column = [&](int k) -> int {
    if constexpr (DB != 0) {
      if (ec) return __ldg(ec + k);
      c += (int)sidx[o + k];
      return c;
    } else {
      return (int)sidx[o + k];
    }
  };
  // FP32 accumulation of a row longer than a.f32_chain: each 16-product run's sum is added
  // into an FP32 pair
  FPair tot;
  const bool fold = IsF32<AccT>::value && len > a.f32_chain;
  int k = 0;
  if constexpr (!IsF32<AccT>::value && DB != 0) {
    AccT acc1 = 0;   // chain 1 of fp64_chain_of
    for (; k + 16 <= len; k += 16) {
      AccT xv[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) xv[q] = (AccT)ldx<XL2, NA>(x + column(k + q), pol_x);
#pragma unroll
      for (int q = 0; q < 16; q += 2) {
        acc = fma(widen<AccT>(sval[o + k + q]), xv[q], acc);
        acc1 = fma(widen<AccT>(sval[o + k + q + 1]), xv[q + 1], acc1);
      }
    }
    for (; k + 8 <= len; k += 8) {
      AccT xv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) xv[q] = (AccT)ldx<XL2, NA>(x + column(k + q), pol_x);
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        acc = fma(widen<AccT>(sval[o + k + q]), xv[q], acc);
        acc1 = fma(widen<AccT>(sval[o + k + q + 1]), xv[q + 1], acc1);
      }
    }
    for (; k < len; ++k)
      acc = fma(widen<AccT>(sval[o + k]), (AccT)ldx<XL2, NA>(x + column(k), pol_x), acc);
    return acc + acc1;
  } else {
    for (; k + 16 <= len; k += 16) {
      AccT xv[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) xv[q] = (AccT)ldx<XL2, NA>(x + column(k + q), pol_x);
#pragma unroll
      for (int q = 0; q < 16; ++q) acc = fma(widen<AccT>(sval[o + k + q]), xv[q], acc);
      if constexpr (IsF32<AccT>::value) {
        if (fold) {
          wadd(tot, (float)acc);
          acc = 0;
        }
      }
    }
    for (; k + 8 <= len; k += 8) {
      AccT xv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) xv[q] = (AccT)ldx<XL2, NA>(x + column(k + q), pol_x);
#pragma unroll
      for (int q = 0; q < 8; ++q) acc = fma(widen<AccT>(sval[o + k + q]), xv[q], acc);
    }
    for (; k < len; ++k)
      acc = fma(widen<AccT>(sval[o + k]), (AccT)ldx<XL2, NA>(x + column(k), pol_x), acc);
    if constexpr (IsF32<AccT>::value) {
      if (fold) {
        wadd(tot, (float)acc);
        acc = (AccT)wvalue(tot);
      }
    }
    return acc;
  }
}

// One lane's share of row r (nonzeros [s, e)) straight from global memory, lanes strided
// by 32. With SumT wider than AccT (FP32 pairs) each lane sums runs of kF32Run products in
// AccT and adds the run sums into SumT.
template <typename ValT, typename VecT, typename AccT, int DB, bool XL2, typename SumT,
          bool NA = false>
__device__ __forceinline__ SumT warp_row_dot(const RunArgs &a, int64_t r, int s, int e,
                                             int lane, const VecT *__restrict__ x,
                                             uint64_t pol_x) {
  constexpr bool RUNS = !std::is_same<SumT, AccT>::value;
  const ValT *__restrict__ val = static_cast<const ValT *>(a.val);
  SumT sum{};
  AccT part = 0;
  int steps = 0;
  auto add = [&](AccT p) {
    part += p;
    if constexpr (RUNS) {
      if (++steps == kF32Run) {
        wadd(sum, part);
        part = 0;
        steps = 0;
      }
    }
  };
  if constexpr (DB != 0) {
    const int32_t base = __ldg(a.dbase + r);
    if (base < 0) {
      const int32_t *ec = a.esc + (-(int64_t)base - 1) - s;
      for (int j = s + lane; j < e; j += 32)
        add(widen<AccT>(val[j]) * (AccT)ldx<XL2, NA>(x + __ldg(ec + j), pol_x));
    } else {
      // decode the row's deltas: the lane sums its own and its predecessors' deltas
      using DT = typename IdxOf<DB>::type;
      const DT *__restrict__ dl = static_cast<const DT *>(a.delta);
      int run = base;
      for (int j0 = s; j0 < e; j0 += 32) {
        const int j = j0 + lane;
        const int d = j < e ? (int)dl[j] : 0;
        const int incl = group_incl_scan<32>(d, lane, 0xffffffffu);
        if (j < e) add(widen<AccT>(val[j]) * (AccT)ldx<XL2, NA>(x + (run + incl), pol_x));
        run += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
  } else {
    for (int j = s + lane; j < e; j += 32)
      add(widen<AccT>(val[j]) * (AccT)ldx<XL2, NA>(x + __ldg(a.colind + j), pol_x));
  }
  wadd(sum, part);
  return sum;
}

// Stores a row's sum, or adds it to y (the later passes of column panels); a panel pass
// reads and writes y evict-first.
template <typename VecT, typename AccT>
__device__ __forceinline__ void store_y(const RunArgs &a, VecT *__restrict__ y, int64_t row,
                                        AccT v) {
  if (a.rows_once) {
    const uint64_t pol = policy_evict_first();
    if (a.y_add) v = (AccT)ld_hint(y + row, pol) + v;
    st_hint(y + row, (VecT)v, pol);
    return;
  }
  if (a.y_add) y[row] = (VecT)((AccT)y[row] + v);
  else y[row] = (VecT)v;
}

// A row pointer: read-only path, evict-first in the L2 for a panel pass.
__device__ __forceinline__ int32_t ld_rowptr(const RunArgs &a, int64_t i) {
  if (a.rows_once) return ld_hint_nc(a.rowptr + i, policy_evict_first());
  return __ldg(a.rowptr + i);
}

// Rows [r0, r1) straight from global memory, a warp per row (tiles larger than the staged
// capacity).
template <typename ValT, typename VecT, typename AccT, int DB, bool XL2, bool NA = false>
__device__ __forceinline__ void tile_direct(const RunArgs &a, int64_t r0, int64_t r1,
                                            const VecT *__restrict__ x, VecT *__restrict__ y,
                                            uint64_t pol_x) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t r = r0 + warp; r < r1; r += blockDim.x / 32) {
    const int s = __ldg(a.rowptr + r), e = __ldg(a.rowptr + r + 1);
    if constexpr (IsF32<AccT>::value) {
      if (e - s > kF32Run * 32) {   // long row in FP32: runs summed in pairs (warp-uniform)
        FPair d = warp_row_dot<ValT, VecT, AccT, DB, XL2, FPair, NA>(a, r, s, e, lane, x, pol_x);
        d = group_sum<32>(d, 0xffffffffu);
        if (lane == 0) store_y<VecT, AccT>(a, y, r, (AccT)wvalue(d));
        continue;
      }
    }
    AccT acc = warp_row_dot<ValT, VecT, AccT, DB, XL2, AccT, NA>(a, r, s, e, lane, x, pol_x);
    acc = group_sum<32>(acc, 0xffffffffu);
    if (lane == 0) store_y<VecT, AccT>(a, y, r, acc);
  }
}

template <typename ValT, typename VecT, typename AccT, int DB, bool XL2, bool NA = false>
__global__ void __launch_bounds__(kTileRows) k_rowtile(const RunArgs a) {
  using IdxT = typename IdxOf<DB>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  const int rows = (int)blockDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rows;
  const int64_t r1 = min(r0 + (int64_t)rows, a.n_rows);
  const int s0 = ld_rowptr(a, r0), s1 = ld_rowptr(a, r1);
  constexpr int AL = stage_align<DB>();
  const int a0 = s0 & ~(AL - 1);                 // aligned start: the copies are 16-byte units
  const int nc = ((s1 - a0) + AL - 1) & ~(AL - 1);   // staged elements
  const ValT *__restrict__ val = static_cast<const ValT *>(a.val);
  const VecT *__restrict__ x = static_cast<const VecT *>(a.x);
  VecT *__restrict__ y = static_cast<VecT *>(a.y);
  uint64_t pol_x = 0;
  if constexpr (XL2) pol_x = policy_evict_last();
  const int64_t row = r0 + threadIdx.x;
  if (nc <= a.tile_cap) {
    ValT *sval = reinterpret_cast<ValT *>(smem + 16);
    IdxT *sidx = reinterpret_cast<IdxT *>(smem + 16 + (size_t)a.tile_cap * sizeof(ValT));
    const IdxT *gidx;
    if constexpr (DB != 0) gidx = static_cast<const IdxT *>(a.delta);
    else gidx = a.colind;
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      if (nc > 0) {
        const uint64_t pol = policy_evict_first();
        const uint32_t bv = (uint32_t)nc * (uint32_t)sizeof(ValT);
        const uint32_t bi = (uint32_t)nc * (uint32_t)sizeof(IdxT);
        mbar_expect_tx(bar, bv + bi);
        bulk_g2s(sval, val + a0, bv, bar, pol);
        bulk_g2s(sidx, gidx + a0, bi, bar, pol);
      }
    }
    // row bounds while the copies are in flight
    int s = 0, e = 0;
    int32_t base = 0;
    if (row < r1) {
      s = ld_rowptr(a, row);
      e = ld_rowptr(a, row + 1);
      if constexpr (DB != 0) base = __ldg(a.dbase + row);
    }
    __syncthreads();   // the barrier is initialised before anyone waits on it
    if (nc > 0) {
      if (!mbar_wait_bounded(bar, 0, kWaitLimitNs)) {
        if (threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
        mbar_wait_bounded(bar, 0, kWaitLimitNs);   // let the copies land before exiting
        return;
      }
    }
    if (row >= r1) return;
    store_y<VecT, AccT>(a, y, row,
                        tile_row_dot<ValT, VecT, AccT, DB, XL2, NA>(a, sval, sidx, s - a0, e - s,
                                                                    base, x, pol_x));
  } else {
    // oversize tile: a warp per row straight from global memory
    tile_direct<ValT, VecT, AccT, DB, XL2, NA>(a, r0, r1, x, y, pol_x);
  }
}


// Persistent variant: a resident grid in which every CTA walks tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... with two shared-memory stages, so that the bulk copy of its
// next tile is in flight while it computes the current one. Stage s is refilled only after
// all threads passed the barrier that ends their reads of it.
template <typename ValT, typename VecT, typename AccT, int DB, bool XL2>
__global__ void __launch_bounds__(kTileRows) k_rowtile_pipe(const RunArgs a) {
  using IdxT = typename IdxOf<DB>::type;
  constexpr int S = 2;
  extern __shared__ __align__(16) unsigned char smem[];   // S mbarriers 16 B apart, then stages
  const int rows = (int)blockDim.x;
  const int64_t n_tiles = (a.n_rows + rows - 1) / rows;
  const size_t vbytes = (size_t)a.tile_cap * sizeof(ValT);
  const size_t stage_bytes = vbytes + (size_t)a.tile_cap * sizeof(IdxT);
  unsigned char *stage0 = smem + 16 * S;
  const ValT *__restrict__ val = static_cast<const ValT *>(a.val);
  const VecT *__restrict__ x = static_cast<const VecT *>(a.x);
  VecT *__restrict__ y = static_cast<VecT *>(a.y);
  const IdxT *gidx;
  if constexpr (DB != 0) gidx = static_cast<const IdxT *>(a.delta);
  else gidx = a.colind;
  uint64_t pol_x = 0;
  if constexpr (XL2) pol_x = policy_evict_last();
  auto tile_span = [&](int64_t t, int64_t &r0, int64_t &r1, int &a0, int &nc) {
    r0 = t * rows;
    r1 = min(r0 + (int64_t)rows, a.n_rows);
    const int s0 = __ldg(a.rowptr + r0), s1 = __ldg(a.rowptr + r1);
    constexpr int AL = stage_align<DB>();
    a0 = s0 & ~(AL - 1);
    nc = ((s1 - a0) + AL - 1) & ~(AL - 1);
  };
  auto issue = [&](int64_t t, int st) {   // one thread
    int64_t r0, r1;
    int a0, nc;
    tile_span(t, r0, r1, a0, nc);
    uint64_t *b = reinterpret_cast<uint64_t *>(smem + 16 * st);
    if (nc > 0 && nc <= a.tile_cap) {
      const uint64_t pol = policy_evict_first();
      const uint32_t bv = (uint32_t)nc * (uint32_t)sizeof(ValT);
      const uint32_t bi = (uint32_t)nc * (uint32_t)sizeof(IdxT);
      unsigned char *dst = stage0 + (size_t)st * stage_bytes;
      mbar_expect_tx(b, bv + bi);
      bulk_g2s(dst, val + a0, bv, b, pol);
      bulk_g2s(dst + vbytes, gidx + a0, bi, b, pol);
    } else {
      mbar_arrive(b);                      // nothing staged: complete the phase now
    }
  };
  if (threadIdx.x == 0) {
    for (int st = 0; st < S; ++st) mbar_init(reinterpret_cast<uint64_t *>(smem + 16 * st), 1);
    for (int st = 0; st < S; ++st) {
      const int64_t t = (int64_t)blockIdx.x + (int64_t)st * gridDim.x;
      if (t < n_tiles) issue(t, st);
    }
  }
  __syncthreads();
  for (int64_t i = 0;; ++i) {
    const int64_t t = (int64_t)blockIdx.x + i * gridDim.x;
    if (t >= n_tiles) break;
    const int st = (int)(i % S);
    const uint32_t parity = (uint32_t)((i / S) & 1);
    int64_t r0, r1;
    int a0, nc;
    tile_span(t, r0, r1, a0, nc);
    const int64_t row = r0 + threadIdx.x;
    int s = 0, e = 0;
    int32_t base = 0;
    if (row < r1) {
      s = __ldg(a.rowptr + row);
      e = __ldg(a.rowptr + row + 1);
      if constexpr (DB != 0) base = __ldg(a.dbase + row);
    }
    uint64_t *b = reinterpret_cast<uint64_t *>(smem + 16 * st);
    const bool ok = mbar_wait_bounded(b, parity, kWaitLimitNs);
    if (!__syncthreads_and(ok)) {
      // give up: record the error and let every copy in flight land before exiting
      if (threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
      for (int q = 0; q < S; ++q) {
        const int64_t tq = (int64_t)blockIdx.x + (i + q) * gridDim.x;
        if (tq < n_tiles)
          mbar_wait_bounded(reinterpret_cast<uint64_t *>(smem + 16 * ((i + q) % S)),
                            (uint32_t)(((i + q) / S) & 1), kWaitLimitNs);
      }
      return;
    }
    if (nc <= a.tile_cap) {
      const ValT *sval = reinterpret_cast<const ValT *>(stage0 + (size_t)st * stage_bytes);
      const IdxT *sidx = reinterpret_cast<const IdxT *>(stage0 + (size_t)st * stage_bytes + vbytes);
      if (row < r1)
        store_y<VecT, AccT>(a, y, row, tile_row_dot<ValT, VecT, AccT, DB, XL2>(
                                           a, sval, sidx, s - a0, e - s, base, x, pol_x));
    } else {
      tile_direct<ValT, VecT, AccT, DB, XL2>(a, r0, r1, x, y, pol_x);
    }
    __syncthreads();                       // every thread is done with stage st
    if (threadIdx.x == 0) {
      const int64_t t2 = (int64_t)blockIdx.x + (i + S) * gridDim.x;
      if (t2 < n_tiles) issue(t2, st);
    }
  }
}

// Raises a kernel's dynamic shared-memory limit the first time a launch needs more than
// 48 KB. The limit only grows, under one lock, so concurrent callers never lower it below a
// size another thread is about to launch with.
inline std::mutex &smem_attr_mutex() {
  static std::mutex m;
  return m;
}

template <typename K>
cudaError_t ensure_smem(K kernel, size_t smem, std::atomic<int> &configured) {
  if (smem <= 48 * 1024 || configured.load(std::memory_order_acquire) >= (int)smem)
    return cudaSuccess;
  std::lock_guard<std::mutex> lk(smem_attr_mutex());
  if (configured.load(std::memory_order_relaxed) >= (int)smem) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) configured.store((int)smem, std::memory_order_release);
  return e;
}

template <typename ValT, typename VecT, typename AccT, int DB, bool XL2, bool NA = false>
cudaError_t launch_rowtile_k(const RunArgs &a, cudaStream_t s) {
  using IdxT = typename IdxOf<DB>::type;
  const int rows = a.tile_rows > 0 ? a.tile_rows : kTileRows;
  const size_t per_stage = (size_t)a.tile_cap * (sizeof(ValT) + sizeof(IdxT));
  if (a.tile_pipe) {
    static std::atomic<int> configured{0};
    auto kern = k_rowtile_pipe<ValT, VecT, AccT, DB, XL2>;
    const size_t smem = 32 + 2 * per_stage;
    cudaError_t e = ensure_smem(kern, smem, configured);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, rows, smem);
    const int64_t n_tiles = (a.n_rows + rows - 1) / rows;
    int64_t g = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    if (g > n_tiles) g = n_tiles;
    kern<<<(unsigned)g, rows, smem, s>>>(a);
    return cudaGetLastError();
  }
  static std::atomic<int> configured{0};
  const size_t smem = 16 + per_stage;
  cudaError_t e = ensure_smem(k_rowtile<ValT, VecT, AccT, DB, XL2, NA>, smem, configured);
  if (e != cudaSuccess) return e;
  const unsigned g = (unsigned)((a.n_rows + rows - 1) / rows);
  k_rowtile<ValT, VecT, AccT, DB, XL2, NA><<<g, rows, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename ValT, typename VecT, typename AccT>
cudaError_t launch_rowtile(const spmv_variant &v, const RunArgs &a, cudaStream_t s) {
  const bool xl2 = v.xpath != 0;
  if (v.index == 1 && a.delta_bits == 8)
    return xl2 ? launch_rowtile_k<ValT, VecT, AccT, 8, true>(a, s)
               : launch_rowtile_k<ValT, VecT, AccT, 8, false>(a, s);
  if (v.index == 1)
    return xl2 ? launch_rowtile_k<ValT, VecT, AccT, 16, true>(a, s)
               : launch_rowtile_k<ValT, VecT, AccT, 16, false>(a, s);
  return xl2 ? launch_rowtile_k<ValT, VecT, AccT, 0, true>(a, s)
             : launch_rowtile_k<ValT, VecT, AccT, 0, false>(a, s);
}

}  // namespace spmv

// SpMV kernel templates (one instantiation set per storage / vector / accumulator dtype).
//
//  k_rowvec  - a sub-warp of VS lanes per row (Fig. 1's inner loop spread over lanes);
//              rows go to CTAs through the hardware block scheduler. Knobs from Table II:
//              VEC  128-bit loads of val / colind, unrolled (CMP, MB "vectorization"),
//              DB   8- or 16-bit column deltas decoded with a sub-warp prefix sum (MB),
//              XL2  x gathered with an L2 evict-last policy while val / colind stream with
//                   evict-first (ML: the GPU counterpart of software prefetching into cache).
//  k_rowtile - thread-per-row tiles staged by TMA bulk copies (spmv_tile.cuh).
//  k_bins_*  - row decomposition: short rows by sub-warps, medium rows by warps, long rows
//              split into chunks with a fixed-order FP64 fixup (IMB).
//  k_sell    - sliced rows (SELL-32): thread per row over 32-row slices stored column-major,
//              coalesced loads without a shared-memory stage (CMP, with or without deltas).
//  k_panel   - one pass of the column-panel variant (ML, x larger than the L2): the rows'
//              nonzeros in one L2-sized slice of x, from a panel-major copy of the matrix.
//  k_merge   - merge-path tiles of equal (rows + nonzeros) work; rows longer than a tile
//              are split over tiles and finished by k_merge_fixup (IMB: the decomposition
//              of Fig. 4/5, long rows computed by many workers with a reduction).
//  k_static  - the profiling baseline of Section III-B: one resident CTA per static
//              nnz-balanced row range with %globaltimer stamps (P_CSR, P_IMB, P_ML) or
//              unit-stride x[i] accesses without colind (P_CMP).
//  k_spmm    - Y = A X for row-major X with K columns per gather.
#pragma once

#include <climits>
#include <type_traits>

#include "common.cuh"
#include "spmv_tile.cuh"

namespace spmv {

constexpr int kRowThreads = 256;

// ------------------------------------------------------------ vector-load range dot ----
// One lane's share of sum_{j in [s, e)} val[j] x[colind[j]] for a sub-warp of VS lanes: 4
// elements per lane per step, colind as one 16-byte load and val as 8..32 bytes (the chunks
// start at s rounded down to 4 elements; elements outside [s, e) are masked off). With a
// wider SumT than AccT (FP32 accumulation over a long range), runs of 16 products (four
// steps) are summed in AccT and the run sums in SumT: within the FP32 bound, (16 + 1) u.
template <typename ValT, typename VecT, typename AccT, int VS, bool XL2, typename SumT = AccT>
__device__ __forceinline__ SumT vec_range_dot(const RunArgs &a, int s, int e, int lane,
                                              uint64_t pol_s, uint64_t pol_x) {
  const ValT *__restrict__ val = static_cast<const ValT *>(a.val);
  const VecT *__restrict__ x = static_cast<const VecT *>(a.x);
  const int32_t *__restrict__ col = a.colind;
  SumT sum{};
  AccT part = 0;
  int steps = 0;
  const int a0 = s & ~3;
#pragma unroll 2
  for (int b = a0 + lane * 4; b < e; b += VS * 4) {
    const uint4 c4 = ld16<true>(col + b, pol_s);
    AccT v[4];
    VLoad<AccT, true, 4>::run(val + b, v, pol_s);
    const int cc[4] = {(int)c4.x, (int)c4.y, (int)c4.z, (int)c4.w};
    AccT xv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = b + q;
      xv[q] = (j >= s && j < e) ? (AccT)ldx<XL2>(x + cc[q], pol_x) : (AccT)0;
    }
    if constexpr (std::is_same<SumT, AccT>::value) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = b + q;
        if (j >= s && j < e) sum += v[q] * xv[q];
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = b + q;
        if (j >= s && j < e) part += v[q] * xv[q];
      }
      if (++steps == 4) {
        wadd(sum, part);
        part = 0;
        steps = 0;
      }
    }
  }
  if constexpr (!std::is_same<SumT, AccT>::value) wadd(sum, part);
  return sum;
}

// One lane's share over [s, e) of an escape row, whose columns are stored in full: ec[0] is
// the column of element s.
template <typename ValT, typename VecT, typename AccT, int VS, bool XL2, typename SumT = AccT>
__device__ __forceinline__ SumT esc_range_dot(const RunArgs &a, int s, int e,
                                              const int32_t *ec, int lane, uint64_t pol_x) {
  const ValT *__restrict__ val = static_cast<const ValT *>(a.val);
  const VecT *__restrict__ x = static_cast<const VecT *>(a.x);
  SumT sum{};
  for (int j = s + lane; j < e; j += VS)
    wadd(sum, (AccT)(widen<AccT>(val[j]) * (AccT)ldx<XL2>(x + __ldg(ec + (j - s)), pol_x)));
  return sum;
}

// Eight column deltas of DB (8 or 16) bits starting at element b (a multiple of 8): one
// 8- or 16-byte load.
template <int DB>
__device__ __forceinline__ void load_deltas8(const void *delta, int b, uint64_t pol, int d[8]) {
  if constexpr (DB == 16) {
    const uint4 w = ld16<true>(static_cast<const uint16_t *>(delta) + b, pol);
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) d[q] = (q & 1) ? (int)(u[q >> 1] >> 16) : (int)(u[q >> 1] & 0xFFFFu);
  } else {
    const uint2 w = ld8<true>(static_cast<const uint8_t *>(delta) + b, pol);
    const uint32_t u[2] = {w.x, w.y};
#pragma unroll
    for (int q = 0; q < 8; ++q) d[q] = (int)((u[q >> 2] >> (8 * (q & 3))) & 0xFFu);
  }
}

// One lane's share over [s, e) with DB-bit column deltas: 8 deltas per lane per step, the
// column of element j = running + the deltas of elements s..j (a sub-warp prefix sum), where
// running is the column the decode starts from (the row's base for a range that starts the
// row, whose first delta is 0; the preceding element's column otherwise).
template <typename ValT, typename VecT, typename AccT, int VS, int DB, bool XL2,
          typename SumT = AccT>
__device__ __forceinline__ SumT delta_range_dot(const RunArgs &a, int s, int e, int running,
                                                int lane, unsigned mask, uint64_t pol_s,
                                                uint64_t pol_x) {
  const ValT *__restrict__ val = static_cast<const ValT *>(a.val);
  const VecT *__restrict__ x = static_cast<const VecT *>(a.x);
  SumT sum{};
  AccT part = 0;
  const int a0 = s & ~7;
  const int n_it = (e - a0 + VS * 8 - 1) / (VS * 8);
  for (int it = 0; it < n_it; ++it) {
    const int b = a0 + it * (VS * 8) + lane * 8;
    // lanes whose 8 elements start past the range end load nothing (reads stay below
    // e + 8, inside the arrays' slack)
    const bool live = b < e;
    int dd[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    AccT v[8];
    if (live) {
      load_deltas8<DB>(a.delta, b, pol_s, dd);
      VLoad<AccT, true, 8>::run(val + b, v, pol_s);
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = (AccT)0;
    }
    int p[8];
    int acc = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = b + q;
      const int d = (j >= s && j < e) ? dd[q] : 0;
      acc += d;
      p[q] = acc;
    }
    const int incl = group_incl_scan<VS>(acc, lane, mask);
    const int excl = incl - acc;
    const int tot = __shfl_sync(mask, incl, VS - 1, VS);
    AccT xv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = b + q;
      xv[q] = (j >= s && j < e) ? (AccT)ldx<XL2>(x + (running + excl + p[q]), pol_x) : (AccT)0;
    }
    if constexpr (std::is_same<SumT, AccT>::value) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = b + q;
        if (j >= s && j < e) sum += v[q] * xv[q];
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = b + q;
        if (j >= s && j < e) part += v[q] * xv[q];
      }
      if (it & 1) {           // runs of 16 products (two steps) summed in AccT
        wadd(sum, part);
        part = 0;
      }
    }
    running += tot;
  }
  if constexpr (!std::is_same<SumT, AccT>::value) wadd(sum, part);
  return sum;
}

// ------------------------------------------------------------------------ k_rowvec ----
// One lane's share of sum_{j in [s, e)} val[j] x[colind[j]], lanes strided by VS (Fig. 1's
// inner loop spread over a sub-warp). With SumT wider than AccT the lane's products are
// summed in runs of kF32Run in AccT and the run sums in SumT.
template <typename ValT, typename VecT, typename AccT, int VS, bool XL2, typename SumT>
__device__ __forceinline__ SumT strided_dot(const RunArgs &a, int s, int e, int lane,
                                            uint64_t pol_x) {
  const ValT *__restrict__ val = static_cast<const ValT *>(a.val);
  const VecT *__restrict__ x = static_cast<const VecT *>(a.x);
  const int32_t *__restrict__ col = a.colind;
  if constexpr (std::is_same<SumT, AccT>::value) {
    AccT sum = 0;
    for (int j = s + lane; j < e; j += VS)
      sum += widen<AccT>(val[j]) * (AccT)ldx<XL2>(x + __ldg(col + j), pol_x);
    return sum;
  } else {
    SumT sum{};
    for (int j0 = s + lane; j0 < e; j0 += kF32Run * VS) {
      const int j1 = min(e, j0 + kF32Run * VS);
      AccT part = 0;
      for (int j = j0; j < j1; j += VS)
        part += widen<AccT>(val[j]) * (AccT)ldx<XL2>(x + __ldg(col + j), pol_x);
      wadd(sum, part);
    }
    return sum;
  }
}

// One lane's share of row `row` with the knobs of k_rowvec.
template <typename ValT, typename VecT, typename AccT, int VS, bool VEC, int DB, bool XL2,
          typename SumT>
__device__ __forceinline__ SumT rowvec_dot(const RunArgs &a, int64_t row, int s, int e,
                                           int lane, unsigned mask, uint64_t pol_s,
                                           uint64_t pol_x) {
  if constexpr (!VEC) {
    return strided_dot<ValT, VecT, AccT, VS, XL2, SumT>(a, s, e, lane, pol_x);
  } else if constexpr (DB == 0) {
    return vec_range_dot<ValT, VecT, AccT, VS, XL2, SumT>(a, s, e, lane, pol_s, pol_x);
  } else {
    const int32_t base = __ldg(a.dbase + row);
    if (base < 0)
      return esc_range_dot<ValT, VecT, AccT, VS, XL2, SumT>(a, s, e, a.esc + (-(int64_t)base - 1),
                                                            lane, pol_x);
    return delta_range_dot<ValT, VecT, AccT, VS, DB, XL2, SumT>(a, s, e, base, lane, mask, pol_s,
                                                                pol_x);
  }
}

template <typename ValT, typename VecT, typename AccT, int VS, bool VEC, int DB, bool XL2>
__global__ void __launch_bounds__(kRowThreads) k_rowvec(const RunArgs a) {
  constexpr int GROUPS = kRowThreads / VS;
  const int lane = threadIdx.x & (VS - 1);
  const int64_t row = (int64_t)blockIdx.x * GROUPS + threadIdx.x / VS;
  if (row >= a.n_rows) return;  // the whole sub-warp leaves together
  const unsigned mask = group_mask<VS>();
  uint64_t pol_s = 0, pol_x = 0;
  if constexpr (VEC) pol_s = policy_evict_first();
  if constexpr (XL2) pol_x = policy_evict_last();
  const int s = __ldg(a.rowptr + row), e = __ldg(a.rowptr + row + 1);
  VecT *__restrict__ y = static_cast<VecT *>(a.y);
  if constexpr (IsF32<AccT>::value) {
    // FP32 accumulation of a row longer than kF32Run products per lane: FP32 runs added
    // into FP32 pairs, and a lane reduction over the pairs (uniform over the sub-warp)
    if (e - s > kF32Run * VS) {
      FPair d = rowvec_dot<ValT, VecT, AccT, VS, VEC, DB, XL2, FPair>(a, row, s, e, lane, mask,
                                                                      pol_s, pol_x);
      d = group_sum<VS>(d, mask);
      if (lane == 0) y[row] = (VecT)wvalue(d);
      return;
    }
  }
  AccT sum = rowvec_dot<ValT, VecT, AccT, VS, VEC, DB, XL2, AccT>(a, row, s, e, lane, mask, pol_s,
                                                                  pol_x);
  sum = group_sum<VS>(sum, mask);
  if (lane == 0) y[row] = (VecT)sum;
}

// ------------------------------------------------------------------------- k_panel ----
// One streamed element of 4, 8 or 2 bytes: evict-first in L2, kept in L1 (the lanes of a
// thread-per-row warp read neighbouring parts of the same sectors).
__device__ __forceinline__ int32_t ld_stream_1(const int32_t *p, uint64_t pol) {
  int32_t r;
  asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;"
               : "=r"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ double ld_stream_1(const double *p, uint64_t pol) {
  double r;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;"
               : "=d"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float ld_stream_1(const float *p, uint64_t pol) {
  float r;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;"
               : "=f"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ __nv_bfloat16 ld_stream_1(const __nv_bfloat16 *p, uint64_t pol) {
  unsigned short r;
  asm volatile("ld.global.nc.L2::cache_hint.b16 %0, [%1], %2;"
               : "=h"(r) : "l"(p), "l"(pol));
  return __ushort_as_bfloat16(r);
}
__device__ __forceinline__ uint16_t ld_stream_1(const uint16_t *p, uint64_t pol) {
  unsigned short r;
  asm volatile("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;"
               : "=h"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ uint8_t ld_stream_1(const uint8_t *p, uint64_t pol) {
  unsigned short r;
  asm volatile("ld.global.nc.L2::cache_hint.u8 %0, [%1], %2;"
               : "=h"(r) : "l"(p), "l"(pol));
  return (uint8_t)r;
}


// One lane's share of a row's nonzeros in one panel (prow gives the panel's row bounds):
// 128-bit loads (VEC), or four of the lane's nonzeros per step whose columns and values are
// loaded first (evict-first), then their four x gathers in flight together. With SumT wider
// than AccT, runs of kF32Run products are summed in AccT and the run sums in SumT.
template <typename ValT, typename VecT, typename AccT, int VS, bool VEC, typename SumT>
__device__ __forceinline__ SumT panel_dot(const RunArgs &a, int s, int e, int lane,
                                          uint64_t pol_s, uint64_t pol_x) {
  if constexpr (VEC) {
    return vec_range_dot<ValT, VecT, AccT, VS, true, SumT>(a, s, e, lane, pol_s, pol_x);
  } else {
    const ValT *__restrict__ val = static_cast<const ValT *>(a.val);
    const VecT *__restrict__ x = static_cast<const VecT *>(a.x);
    SumT sum{};
    AccT part = 0;
    int steps = 0;
    for (int j0 = s + lane; j0 < e; j0 += 4 * VS) {
      int c[4];
      ValT v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = j0 + q * VS;
        c[q] = j < e ? ld_stream_1(a.colind + j, pol_s) : -1;
        v[q] = j < e ? ld_stream_1(val + j, pol_s) : ValT(0);
      }
      AccT xv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) xv[q] = c[q] >= 0 ? (AccT)ldx<true>(x + c[q], pol_x) : AccT(0);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c[q] >= 0) part += widen<AccT>(v[q]) * xv[q];
      if constexpr (!std::is_same<SumT, AccT>::value) {
        if (++steps == kF32Run / 4) {
          wadd(sum, part);
          part = 0;
          steps = 0;
        }
      }
    }
    wadd(sum, part);
    return sum;
  }
}

// One pass of the column-panel variant (ML with x larger than the L2). The matrix is held
// panel-major: panel p holds the nonzeros whose columns fall in the p-th slice of x, as a
// CSR of its own with the rows in order. Pass p computes every row's sum over panel p, so
// one pass gathers from one L2-sized slice of x (evict-last) while its panel streams past
// (evict-first); pass 0 writes y, later passes add to it. With FP32 accumulation every
// pass sums runs of kF32Run products into an FP32 pair and rounds once into y, so a row
// through P passes errs by at most (16 + P) u.
template <typename ValT, typename VecT, typename AccT, int VS, bool VEC>
__global__ void __launch_bounds__(kRowThreads) k_panel(const RunArgs a,
                                                       const int32_t *__restrict__ prow,
                                                       int add) {
  constexpr int GROUPS = kRowThreads / VS;
  using SumT = typename WideOf<AccT>::type;
  const int lane = threadIdx.x & (VS - 1);
  const int64_t row = (int64_t)blockIdx.x * GROUPS + threadIdx.x / VS;
  if (row >= a.n_rows) return;  // the whole sub-warp leaves together
  const unsigned mask = group_mask<VS>();
  const uint64_t pol_s = policy_evict_first(), pol_x = policy_evict_last();
  const int s = __ldg(prow + row), e = __ldg(prow + row + 1);
  SumT sum = panel_dot<ValT, VecT, AccT, VS, VEC, SumT>(a, s, e, lane, pol_s, pol_x);
  sum = group_sum<VS>(sum, mask);
  if (lane == 0) {
    VecT *y = static_cast<VecT *>(a.y);
    if (add) wadd(sum, (AccT)y[row]);
    y[row] = (VecT)wvalue(sum);
  }
}

// -------------------------------------------------------------------------- k_sell ----
// Sliced rows (SELL-32, partition 3): one thread per row over a layout in which the 32 rows of
// a slice lie column-major, so that the k-th elements of a warp's rows are one contiguous
// 256-byte (FP64) run: every value and column load is coalesced without a shared-memory
// stage, and the occupancy is set by registers alone. 16 (then 8) x gathers in flight per
// thread before their FMAs, one FMA per nonzero, exact trip counts (padding is never read).
constexpr int kSellThreads = 128;

template <typename ValT, typename VecT, typename AccT, int DB, bool XL2>
__global__ void __launch_bounds__(kSellThreads, 10) k_sell(const RunArgs a) {
  using IdxT = typename IdxOf<DB>::type;
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= a.n_rows) return;
  const int64_t p0 = __ldg(a.sell_off + (row >> 5)) + (row & 31);
  const int len = __ldg(a.rowptr + row + 1) - __ldg(a.rowptr + row);
  const ValT *__restrict__ sv = static_cast<const ValT *>(a.sell_val) + p0;
  const IdxT *__restrict__ si = static_cast<const IdxT *>(a.sell_idx) + p0;
  const VecT *__restrict__ x = static_cast<const VecT *>(a.x);
  // the slices stream past once (evict-first) so that they do not push x out of the L2
  const uint64_t pol_s = policy_evict_first();
  uint64_t pol_x = 0;
  if constexpr (XL2) pol_x = policy_evict_last();
  int c = 0;
  const int32_t *ec = nullptr;
  if constexpr (DB != 0) {
    const int32_t base = __ldg(a.dbase + row);
    if (base < 0) ec = a.esc + (-(int64_t)base - 1);
    else c = base;
  }
  auto column = [&](int k) -> int {
    if constexpr (DB != 0) {
      if (ec) return __ldg(ec + k);
      c += (int)ld_stream_1(si + 32 * (int64_t)k, pol_s);
      return c;
    } else {
      return ld_stream_1(si + 32 * (int64_t)k, pol_s);
    }
  };
  AccT acc = 0;
  // FP32 accumulation of a row longer than kF32Chain: each 16-product run's sum is added
  // into an FP32 pair
  FPair tot;
  const bool fold = IsF32<AccT>::value && len > kF32Chain;
  int k = 0;
  for (; k + 16 <= len; k += 16) {
    AccT xv[16], v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      xv[q] = (AccT)ldx<XL2>(x + column(k + q), pol_x);
      v[q] = widen<AccT>(ld_stream_1(sv + 32 * (int64_t)(k + q), pol_s));
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) acc = fma(v[q], xv[q], acc);
    if constexpr (IsF32<AccT>::value) {
      if (fold) {
        wadd(tot, (float)acc);
        acc = 0;
      }
    }
  }
  for (; k + 8 <= len; k += 8) {
    AccT xv[8], v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      xv[q] = (AccT)ldx<XL2>(x + column(k + q), pol_x);
      v[q] = widen<AccT>(ld_stream_1(sv + 32 * (int64_t)(k + q), pol_s));
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) acc = fma(v[q], xv[q], acc);
  }
  for (; k < len; ++k)
    acc = fma(widen<AccT>(ld_stream_1(sv + 32 * (int64_t)k, pol_s)), (AccT)ldx<XL2>(x + column(k), pol_x),
              acc);
  if constexpr (IsF32<AccT>::value) {
    if (fold) {
      wadd(tot, (float)acc);
      acc = (AccT)wvalue(tot);
    }
  }
  static_cast<VecT *>(a.y)[row] = (VecT)acc;
}

template <typename ValT, typename VecT, typename AccT>
cudaError_t launch_sell(const spmv_variant &v, const RunArgs &a, cudaStream_t s) {
  if (!a.sell_off || !a.sell_val || !a.sell_idx) return cudaErrorInvalidValue;
  const unsigned g = (unsigned)((a.n_rows + kSellThreads - 1) / kSellThreads);
  const bool xl2 = v.xpath != 0;
  const int db = v.index == 1 ? a.delta_bits : 0;
#define SPMV_SELL(DB_)                                                                \
  (xl2 ? k_sell<ValT, VecT, AccT, DB_, true><<<g, kSellThreads, 0, s>>>(a)           \
       : k_sell<ValT, VecT, AccT, DB_, false><<<g, kSellThreads, 0, s>>>(a))
  if (db == 16) SPMV_SELL(16);
  else if (db == 8) SPMV_SELL(8);
  else SPMV_SELL(0);
#undef SPMV_SELL
  return cudaGetLastError();
}

// ------------------------------------------------------------------------- k_merge ----
// Tile t covers merge items [t*D, (t+1)*D): the row-end events and nonzeros between the
// table entries coord[t] and coord[t+1] (rows ended, nonzeros consumed).
//  1. stage the tile's row ends, values and gathered x[colind[j]] in shared memory
//     (coalesced loads, all gathers of the tile in flight at once);
//  2. every thread takes IPT consecutive merge items (found by a merge-path search in
//     shared memory) and sums each row it sees with one fused multiply-add per nonzero;
//  3. a row that began in an earlier thread gets those threads' carries through a segmented
//     scan over the threads (keys = open rows); a row that began in an earlier tile is
//     finished by k_merge_fixup, which adds the earlier tiles' carries in tile order (no
//     atomics: results are reproducible).
// With FP32 accumulation the tile stages each product a_j x_j (one shared-memory store and
// load per nonzero, the multiply done while staging); with FP64 accumulation it stages a_j
// and x_j and the walk keeps one FMA per nonzero (GB300's FP64 pipe is the scarce unit).
template <typename ValT, typename VecT, typename AccT, bool XL2>
__global__ void __launch_bounds__(kMergeThreads) k_merge(const RunArgs a) {
  constexpr int D = kMergeItems;
  constexpr bool PROD = std::is_same<AccT, float>::value;
  __shared__ int s_rowend[D + 1];
  __shared__ AccT s_val[D];
  __shared__ AccT s_x[PROD ? 1 : D];
  __shared__ int s_crow[kMergeThreads];
  __shared__ AccT s_cval[kMergeThreads];
  const int t = blockIdx.x;
  const int2 c0 = a.coord[t], c1 = a.coord[t + 1];
  const int row0 = c0.x, nz0 = c0.y;
  const int nrows_t = c1.x - c0.x, nnz_t = c1.y - c0.y;
  const int total = nrows_t + nnz_t;
  const ValT *__restrict__ val = static_cast<const ValT *>(a.val);
  const VecT *__restrict__ x = static_cast<const VecT *>(a.x);
  const int32_t *__restrict__ col = a.colind;
  uint64_t pol_s = 0, pol_x = 0;
  if constexpr (XL2) {
    pol_s = policy_evict_first();
    pol_x = policy_evict_last();
  }
  for (int k = threadIdx.x; k < nrows_t; k += kMergeThreads)
    s_rowend[k] = __ldg(a.rowptr + row0 + 1 + k);
  if (threadIdx.x == 0) s_rowend[nrows_t] = INT_MAX;
  // nnz_t <= kMergeIpt * kMergeThreads: every thread stages at most kMergeIpt nonzeros; all
  // column loads are issued first, then all value loads and x gathers, then the stores
  {
    int cj[kMergeIpt];
#pragma unroll
    for (int q = 0; q < kMergeIpt; ++q) {
      const int k = q * kMergeThreads + (int)threadIdx.x;
      cj[q] = k < nnz_t ? __ldg(col + nz0 + k) : 0;
    }
    AccT vv[kMergeIpt], xx[kMergeIpt];
#pragma unroll
    for (int q = 0; q < kMergeIpt; ++q) {
      const int k = q * kMergeThreads + (int)threadIdx.x;
      vv[q] = k < nnz_t ? widen<AccT>(val[nz0 + k]) : (AccT)0;
      xx[q] = k < nnz_t ? (AccT)ldx<XL2>(x + cj[q], pol_x) : (AccT)0;
    }
#pragma unroll
    for (int q = 0; q < kMergeIpt; ++q) {
      const int k = q * kMergeThreads + (int)threadIdx.x;
      if (k < nnz_t) {
        if constexpr (PROD) {
          s_val[k] = vv[q] * xx[q];
        } else {
          s_val[k] = vv[q];
          s_x[k] = xx[q];
        }
      }
    }
  }
  __syncthreads();

  const int d0 = min((int)threadIdx.x * kMergeIpt, total);
  const int d1 = min(d0 + kMergeIpt, total);
  int lo = max(0, d0 - nnz_t), hi = min(d0, nrows_t);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (s_rowend[mid] <= nz0 + d0 - 1 - mid) lo = mid + 1;
    else hi = mid;
  }
  int ra = lo, nb = d0 - lo;
  AccT acc = 0;
  bool has_first = false;
  int first_row = 0;
  AccT first_val = 0;
  VecT *__restrict__ y = static_cast<VecT *>(a.y);
  int re = s_rowend[ra];   // end of the current row (s_rowend[nrows_t] is a sentinel)
  for (int d = d0; d < d1; ++d) {
    if (nz0 + nb < re) {
      if constexpr (PROD) acc += s_val[nb];
      else acc = fma(s_val[nb], s_x[nb], acc);   // one FP64 instruction per nonzero
      ++nb;
    } else {
      const int r = row0 + ra;
      if (!has_first) {
        has_first = true;
        first_row = r;
        first_val = acc;
      } else {
        y[r] = (VecT)acc;
      }
      acc = 0;
      ++ra;
      re = s_rowend[ra];
    }
  }
  // Carries: thread i ends holding the partial sum `acc` of its open row `key`. Keys are
  // non-decreasing over the threads, so equal keys form contiguous segments; a segmented
  // inclusive scan (fixed shuffle tree inside each warp, then warps combined in order) gives
  // every thread the sum of its segment up to itself.
  const int key = row0 + ra;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  AccT sc = acc;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const AccT tv = __shfl_up_sync(0xffffffffu, sc, off);
    const int tk = __shfl_up_sync(0xffffffffu, key, off);
    if (lane >= off && tk == key) sc += tv;
  }
  __shared__ AccT s_wsum[kMergeThreads / 32];
  __shared__ int s_wkey_first[kMergeThreads / 32], s_wkey_last[kMergeThreads / 32];
  __shared__ AccT s_win[kMergeThreads / 32];
  if (lane == 31) {
    s_wsum[warp] = sc;
    s_wkey_last[warp] = key;
  }
  if (lane == 0) s_wkey_first[warp] = key;
  __syncthreads();
  if (threadIdx.x == 0) {
    // carry into warp w: the part of its first segment held by earlier warps
    AccT in = 0;
    s_win[0] = 0;
    for (int w = 1; w < kMergeThreads / 32; ++w) {
      if (s_wkey_last[w - 1] == s_wkey_first[w]) {
        in = s_wsum[w - 1] + (s_wkey_first[w - 1] == s_wkey_last[w - 1] ? in : (AccT)0);
      } else {
        in = 0;
      }
      s_win[w] = in;
    }
  }
  __syncthreads();
  if (key == s_wkey_first[warp]) sc += s_win[warp];
  s_crow[threadIdx.x] = key;
  s_cval[threadIdx.x] = sc;
  __syncthreads();
  if (has_first) {
    // the row this thread completed began in earlier threads: add their segment
    const int q = (int)threadIdx.x - 1;
    const AccT tot = (q >= 0 && s_crow[q] == first_row) ? first_val + s_cval[q] : first_val;
    const bool continued = (first_row == row0) && (__ldg(a.rowptr + row0) < nz0);
    if (continued) a.head_val[t] = (double)tot;
    else y[first_row] = (VecT)tot;
  }
  if (threadIdx.x == kMergeThreads - 1) {
    // the row open at the tile's end (idle threads hold it with a zero carry)
    a.tail_row[t] = c1.x;
    a.tail_val[t] = s_crow[threadIdx.x] == c1.x ? (double)s_cval[threadIdx.x] : 0.0;
  }
}

// Rows that began in an earlier tile: y[row] = (carries of the earlier tiles that hold part
// of the row) + the part summed in the tile that ends the row. One warp per tile: the lanes
// read 32 earlier tails at a time, a fixed shuffle tree sums each chunk and the chunks are
// added nearest first; FP64 throughout.
template <typename VecT>
__global__ void k_merge_fixup(const RunArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32 + 1;
  if (t >= a.n_tiles) return;                    // uniform across the warp
  const int2 c0 = a.coord[t], c1 = a.coord[t + 1];
  const int row0 = c0.x;
  if (c1.x - c0.x <= 0) return;                  // the tile ends no row
  if (!(__ldg(a.rowptr + row0) < c0.y)) return;  // its first row starts inside it
  double tot = 0.0;
  for (int64_t base = t - 1; base >= 0; base -= 32) {
    const int64_t q = base - lane;
    const bool mine = q >= 0 && a.tail_row[q] == row0;
    double v = mine ? a.tail_val[q] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    tot += v;
    if (!__all_sync(0xffffffffu, mine)) break;   // the row's earlier tiles are contiguous
  }
  tot += a.head_val[t];
  if (lane == 0) static_cast<VecT *>(a.y)[row0] = (VecT)tot;
}

// ------------------------------------------------------------------------ k_static ----
template <typename ValT, typename VecT, typename AccT, int VS, bool CMP>
__global__ void __launch_bounds__(kRowThreads) k_static(const ProfileArgs a) {
  __shared__ unsigned long long t0;
  if (threadIdx.x == 0) t0 = globaltimer_ns();
  __syncthreads();
  constexpr int GROUPS = kRowThreads / VS;
  const int lane = threadIdx.x & (VS - 1);
  const unsigned mask = group_mask<VS>();
  const int r0 = a.part[blockIdx.x], r1 = a.part[blockIdx.x + 1];
  const ValT *__restrict__ val = static_cast<const ValT *>(a.val);
  const VecT *__restrict__ x = static_cast<const VecT *>(a.x);
  VecT *__restrict__ y = static_cast<VecT *>(a.y);
  const int32_t *__restrict__ col = a.colind;
  const int64_t xmax = a.n_cols - 1;
  for (int row = r0 + (int)threadIdx.x / VS; row < r1; row += GROUPS) {
    const int s = __ldg(a.rowptr + row), e = __ldg(a.rowptr + row + 1);
    AccT sum = 0;
    if constexpr (CMP) {
      if (s < e) {   // a matrix without columns has only empty rows: x is never read
        const VecT xi = __ldg(x + (row < xmax ? row : xmax));
        for (int j = s + lane; j < e; j += VS) sum += widen<AccT>(val[j]) * (AccT)xi;
      }
    } else {
      for (int j = s + lane; j < e; j += VS)
        sum += widen<AccT>(val[j]) * (AccT)__ldg(x + __ldg(col + j));
    }
    sum = group_sum<VS>(sum, mask);
    if (lane == 0) y[row] = (VecT)sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a.t_start[blockIdx.x] = t0;
    a.t_end[blockIdx.x] = globaltimer_ns();
    if (a.smid) {
      uint32_t sm;
      asm volatile("mov.u32 %0, %smid;" : "=r"(sm));
      a.smid[blockIdx.x] = (int32_t)sm;
    }
  }
}

// -------------------------------------------------------------------------- k_spmm ----
// K consecutive right-hand-side columns [off, off + K) of row-major X / Y (leading
// dimension ldk). For K > 1 the K values of one X row are fetched as 16-byte loads
// (launcher guarantees alignment: ldk and off multiples of the vector width).
template <typename VecT, int K> struct XRow {
  __device__ __forceinline__ static void load(const VecT *p, VecT *o) {
    if constexpr (K == 1) {
      o[0] = __ldg(p);
    } else {
      constexpr int PER = 16 / (int)sizeof(VecT);
#pragma unroll
      for (int q = 0; q < K; q += PER) {
        const uint4 u = ld_nc_u4(p + q);
        if constexpr (sizeof(VecT) == 8) {
          o[q] = (VecT)__hiloint2double(u.y, u.x);
          o[q + 1] = (VecT)__hiloint2double(u.w, u.z);
        } else {
          o[q] = (VecT)__uint_as_float(u.x);
          o[q + 1] = (VecT)__uint_as_float(u.y);
          o[q + 2] = (VecT)__uint_as_float(u.z);
          o[q + 3] = (VecT)__uint_as_float(u.w);
        }
      }
    }
  }
};

template <typename ValT, typename VecT, typename AccT, int VS, int K>
__global__ void __launch_bounds__(kRowThreads) k_spmm(const RunArgs a, int off, int ldk) {
  constexpr int GROUPS = kRowThreads / VS;
  const int lane = threadIdx.x & (VS - 1);
  const int64_t row = (int64_t)blockIdx.x * GROUPS + threadIdx.x / VS;
  if (row >= a.n_rows) return;
  const unsigned mask = group_mask<VS>();
  const ValT *__restrict__ val = static_cast<const ValT *>(a.val);
  const VecT *__restrict__ X = static_cast<const VecT *>(a.x);
  const int s = __ldg(a.rowptr + row), e = __ldg(a.rowptr + row + 1);
  VecT *__restrict__ Y = static_cast<VecT *>(a.y) + row * ldk + off;
  AccT acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0;
  if constexpr (IsF32<AccT>::value) {
    if (e - s > kF32Run * VS) {
      // FP32 accumulation of a long row: every lane sums runs of kF32Run products per column
      // in FP32 and adds the run sums into FP32 pairs, reduced over the lanes as pairs
      FPair tot[K];
      for (int j0 = s + lane; j0 < e; j0 += kF32Run * VS) {
        const int j1 = min(e, j0 + kF32Run * VS);
        for (int j = j0; j < j1; j += VS) {
          const AccT v = widen<AccT>(val[j]);
          VecT xr[K];
          XRow<VecT, K>::load(X + (int64_t)__ldg(a.colind + j) * ldk + off, xr);
#pragma unroll
          for (int q = 0; q < K; ++q) acc[q] += v * (AccT)xr[q];
        }
#pragma unroll
        for (int q = 0; q < K; ++q) {
          wadd(tot[q], (float)acc[q]);
          acc[q] = 0;
        }
      }
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const FPair r = group_sum<VS>(tot[q], mask);
        if (lane == 0) Y[q] = (VecT)wvalue(r);
      }
      return;
    }
  }
  for (int j = s + lane; j < e; j += VS) {
    const AccT v = widen<AccT>(val[j]);
    VecT xr[K];
    XRow<VecT, K>::load(X + (int64_t)__ldg(a.colind + j) * ldk + off, xr);
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] += v * (AccT)xr[q];
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const AccT r = group_sum<VS>(acc[q], mask);
    if (lane == 0) Y[q] = (VecT)r;
  }
}

// -------------------------------------------------------------------- k_bins_* ------
// Row decomposition (IMB, Section III-E's matrix decomposition A = A_short + A_long; Fig. 5):
//  k_bins        - one launch of two kinds of blocks: short rows (shorter than l_med), a
//                  sub-warp of VS lanes (1: a thread) each, over all rows (longer rows are
//                  skipped: the sub-warp reads their bounds only), and warp items,
//                  one warp per work item: a medium row (l_med <= length < kBinChunk, from
//                  the row list) written directly, or a chunk of at most kBinChunk nonzeros
//                  of a long row whose sum goes to an FP64 partial slot; with FP32
//                  accumulation the lanes add runs of 16 products into FP32 pairs;
//  k_bins_fixup  - each long row's partials added by one warp in a fixed order
//                  (reproducible, no atomics).
// One sub-warp's share of elements [s, e) of row `row`, whose decode (delta columns of DB
// bits) starts from column `running`.
template <typename ValT, typename VecT, typename AccT, int VS, int DB, bool XL2, typename SumT>
__device__ __forceinline__ SumT bins_range_dot(const RunArgs &a, int64_t row, int s, int e,
                                               int running, int lane, uint64_t pol_s,
                                               uint64_t pol_x) {
  if constexpr (DB != 0) {
    const int32_t base = __ldg(a.dbase + row);
    if (base < 0) {
      const int rs = __ldg(a.rowptr + row);
      return esc_range_dot<ValT, VecT, AccT, VS, XL2, SumT>(
          a, s, e, a.esc + (-(int64_t)base - 1) + (s - rs), lane, pol_x);
    }
    return delta_range_dot<ValT, VecT, AccT, VS, DB, XL2, SumT>(a, s, e, running, lane,
                                                                group_mask<VS>(), pol_s, pol_x);
  } else {
    return vec_range_dot<ValT, VecT, AccT, VS, XL2, SumT>(a, s, e, lane, pol_s, pol_x);
  }
}

// Short rows of row block `blk` (kRowThreads / VS rows).
template <typename ValT, typename VecT, typename AccT, int VS, int DB, bool XL2>
__device__ __forceinline__ void bins_short_block(const RunArgs &a, int64_t blk) {
  constexpr int GROUPS = kRowThreads / VS;
  const int lane = threadIdx.x & (VS - 1);
  const int64_t row = blk * GROUPS + threadIdx.x / VS;
  if (row >= a.n_rows) return;
  const int s = __ldg(a.rowptr + row), e = __ldg(a.rowptr + row + 1);
  if (e - s >= a.bin_l_med) return;
  uint64_t pol_s = policy_evict_first(), pol_x = 0;
  if constexpr (XL2) pol_x = policy_evict_last();
  const int running = DB != 0 ? __ldg(a.dbase + row) : 0;
  if constexpr (IsF32<AccT>::value) {
    if (e - s > kF32Run * VS) {   // FP32 runs summed in pairs (uniform over the sub-warp)
      FPair d = bins_range_dot<ValT, VecT, AccT, VS, DB, XL2, FPair>(a, row, s, e, running,
                                                                     lane, pol_s, pol_x);
      d = group_sum<VS>(d, group_mask<VS>());
      if (lane == 0) static_cast<VecT *>(a.y)[row] = (VecT)wvalue(d);
      return;
    }
  }
  AccT sum = bins_range_dot<ValT, VecT, AccT, VS, DB, XL2, AccT>(a, row, s, e, running, lane,
                                                                  pol_s, pol_x);
  sum = group_sum<VS>(sum, group_mask<VS>());
  if (lane == 0) static_cast<VecT *>(a.y)[row] = (VecT)sum;
}

// Warp items of block `blk` (kRowThreads / 32 items: long-row chunks first, then medium rows).
template <typename ValT, typename VecT, typename AccT, int DB, bool XL2>
__device__ __forceinline__ void bins_warp_block(const RunArgs &a, int64_t blk) {
  using WS = typename WideOf<AccT>::type;   // FP32 runs are summed in FP32 pairs
  const int lane = threadIdx.x & 31;
  const int64_t item = (blk * kRowThreads + threadIdx.x) / 32;
  if (item >= a.bin_n_med + a.bin_n_chunks) return;
  uint64_t pol_s = policy_evict_first(), pol_x = 0;
  if constexpr (XL2) pol_x = policy_evict_last();
  if (item < a.bin_n_chunks) {
    // (row, first nonzero, end nonzero, the column the delta decode starts from)
    const int4 c = a.bin_chunks[item];
    const WS sum = bins_range_dot<ValT, VecT, AccT, 32, DB, XL2, WS>(a, c.x, c.y, c.z, c.w,
                                                                    lane, pol_s, pol_x);
    const WS t = group_sum<32>(sum, 0xffffffffu);
    if (lane == 0) a.bin_partials[item] = wdouble(t);
  } else {
    const int row = __ldg(a.bin_rows + (item - a.bin_n_chunks));
    const int s = __ldg(a.rowptr + row), e = __ldg(a.rowptr + row + 1);
    const int running = DB != 0 ? __ldg(a.dbase + row) : 0;
    WS sum = bins_range_dot<ValT, VecT, AccT, 32, DB, XL2, WS>(a, row, s, e, running, lane,
                                                              pol_s, pol_x);
    sum = group_sum<32>(sum, 0xffffffffu);
    if (lane == 0) static_cast<VecT *>(a.y)[row] = (VecT)wvalue(sum);
  }
}

// The row decomposition in one launch: g_warp blocks of warp items and g_short blocks of
// short rows, the short blocks spread evenly among the others (block b is short block j
// when floor((b + 1) g_short / B) > floor(b g_short / B) = j, B = g_warp + g_short), so that
// the latency-bound short rows run beside the gather-bound long ones instead of after them.
template <typename ValT, typename VecT, typename AccT, int VS, int DB, bool XL2>
__global__ void __launch_bounds__(kRowThreads) k_bins(const RunArgs a, int64_t g_warp,
                                                      int64_t g_short) {
  const int64_t B = g_warp + g_short, b = blockIdx.x;
  const int64_t j0 = b * g_short / B, j1 = (b + 1) * g_short / B;
  if (j1 > j0) bins_short_block<ValT, VecT, AccT, VS, DB, XL2>(a, j0);
  else bins_warp_block<ValT, VecT, AccT, DB, XL2>(a, b - j0);
}

// One warp per long row: the lanes read the row's partials 32 at a time (lane j takes chunks
// j, j + 32, ... in order), then a fixed shuffle tree adds the lanes' sums; FP64 throughout,
// the same order on every run.
template <typename VecT>
__global__ void k_bins_fixup(const RunArgs a) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (i >= a.bin_n_long) return;                  // uniform over the warp
  double t = 0.0;
  for (int c = a.bin_long_first[i] + lane; c < a.bin_long_first[i + 1]; c += 32)
    t += a.bin_partials[c];
  t = group_sum<32>(t, 0xffffffffu);
  if (lane == 0) static_cast<VecT *>(a.y)[a.bin_long_rows[i]] = (VecT)t;
}

template <typename ValT, typename VecT, typename AccT, int VS, int DB, bool XL2>
void launch_bins_vs(const RunArgs &a, cudaStream_t s) {
  constexpr int GROUPS = kRowThreads / VS;
  const int64_t items = a.bin_n_med + a.bin_n_chunks;
  const int64_t g_warp = (items * 32 + kRowThreads - 1) / kRowThreads;
  const int64_t g_short = (a.n_rows + GROUPS - 1) / GROUPS;
  k_bins<ValT, VecT, AccT, VS, DB, XL2><<<(unsigned)(g_warp + g_short), kRowThreads, 0, s>>>(
      a, g_warp, g_short);
}

template <typename ValT, typename VecT, typename AccT, int DB, bool XL2>
void launch_bins_k(const RunArgs &a, cudaStream_t s) {
  switch (a.bin_vs_short) {
    case 1: launch_bins_vs<ValT, VecT, AccT, 1, DB, XL2>(a, s); break;
    case 2: launch_bins_vs<ValT, VecT, AccT, 2, DB, XL2>(a, s); break;
    case 8: launch_bins_vs<ValT, VecT, AccT, 8, DB, XL2>(a, s); break;
    default: launch_bins_vs<ValT, VecT, AccT, 4, DB, XL2>(a, s); break;
  }
}

template <typename ValT, typename VecT, typename AccT>
cudaError_t launch_bins(int db, bool xl2, const RunArgs &a, cudaStream_t s) {
  if (a.n_rows == 0) return cudaSuccess;
  if (db == 16) {
    if (xl2) launch_bins_k<ValT, VecT, AccT, 16, true>(a, s);
    else launch_bins_k<ValT, VecT, AccT, 16, false>(a, s);
  } else if (db == 8) {
    if (xl2) launch_bins_k<ValT, VecT, AccT, 8, true>(a, s);
    else launch_bins_k<ValT, VecT, AccT, 8, false>(a, s);
  } else {
    if (xl2) launch_bins_k<ValT, VecT, AccT, 0, true>(a, s);
    else launch_bins_k<ValT, VecT, AccT, 0, false>(a, s);
  }
  if (a.bin_n_long > 0)
    k_bins_fixup<VecT><<<(unsigned)((a.bin_n_long * 32 + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------ launchers ---
inline unsigned grid_for_rows(int64_t n_rows, int vs) {
  const int64_t groups = kRowThreads / vs;
  return (unsigned)((n_rows + groups - 1) / groups);
}

template <typename ValT, typename VecT, typename AccT, int VS>
cudaError_t launch_rowvec_vs(const spmv_variant &v, const RunArgs &a, cudaStream_t s) {
  const unsigned g = grid_for_rows(a.n_rows, VS);
  const bool dl = v.index == 1, vec = v.vec != 0 || dl, xl2 = v.xpath != 0;
  if (!vec) {
    if (xl2) k_rowvec<ValT, VecT, AccT, VS, false, 0, true><<<g, kRowThreads, 0, s>>>(a);
    else k_rowvec<ValT, VecT, AccT, VS, false, 0, false><<<g, kRowThreads, 0, s>>>(a);
  } else if (!dl) {
    if (xl2) k_rowvec<ValT, VecT, AccT, VS, true, 0, true><<<g, kRowThreads, 0, s>>>(a);
    else k_rowvec<ValT, VecT, AccT, VS, true, 0, false><<<g, kRowThreads, 0, s>>>(a);
  } else if (a.delta_bits == 8) {
    if (xl2) k_rowvec<ValT, VecT, AccT, VS, true, 8, true><<<g, kRowThreads, 0, s>>>(a);
    else k_rowvec<ValT, VecT, AccT, VS, true, 8, false><<<g, kRowThreads, 0, s>>>(a);
  } else {
    if (xl2) k_rowvec<ValT, VecT, AccT, VS, true, 16, true><<<g, kRowThreads, 0, s>>>(a);
    else k_rowvec<ValT, VecT, AccT, VS, true, 16, false><<<g, kRowThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// The column-panel variant: one launch per pass, in panel order on one stream. With one
// thread per row (VS = 1) every pass is the thread-per-row tile kernel on the panel's CSR
// (its tiles staged by bulk copies, x gathered evict-last), adding into y after the first
// pass; wider sub-warps run k_panel.
template <typename ValT, typename VecT, typename AccT, int VS>
cudaError_t launch_panels_vs(const spmv_variant &v, const RunArgs &a, cudaStream_t s) {
  RunArgs pa = a;
  pa.colind = a.pnl_col;
  pa.val = a.pnl_val;
  const unsigned g = grid_for_rows(a.n_rows, VS);
  for (int p = a.pnl_first; p < a.pnl_first + a.n_panels; ++p) {
    const int32_t *prow = a.pnl_rowptr + (int64_t)p * a.pnl_stride;
    if constexpr (VS == 1) {
      if (a.pnl_tile_rows <= 0) return cudaErrorInvalidValue;
      RunArgs ta = pa;
      ta.rowptr = prow;
      ta.y_add = p > 0;
      ta.rows_once = 1;
      ta.f32_chain = kF32Run;          // each pass also rounds once into y
      ta.tile_cap = a.pnl_tile_cap;
      ta.tile_rows = a.pnl_tile_rows;
      ta.tile_pipe = 0;
      // x gathers without L1 allocation: measured on the scattered 16M x 8 matrix, 447
      // against 426 GFLOP/s (the same hint slowed the stencil and power-law kernels, whose
      // gathers do hit L1)
      const cudaError_t e = launch_rowtile_k<ValT, VecT, AccT, 0, true, true>(ta, s);
      if (e != cudaSuccess) return e;
    } else {
      if (v.vec) k_panel<ValT, VecT, AccT, VS, true><<<g, kRowThreads, 0, s>>>(pa, prow, p > 0);
      else k_panel<ValT, VecT, AccT, VS, false><<<g, kRowThreads, 0, s>>>(pa, prow, p > 0);
    }
  }
  return cudaGetLastError();
}

template <typename ValT, typename VecT, typename AccT>
cudaError_t launch_panels(const spmv_variant &v, const RunArgs &a, cudaStream_t s) {
  if (!a.pnl_rowptr || a.pnl_first < 0 || a.n_panels < 1 ||
      a.pnl_first + a.n_panels > v.xpath || a.pnl_stride < a.n_rows + 1)
    return cudaErrorInvalidValue;
  switch (v.vs) {
    case 1: return launch_panels_vs<ValT, VecT, AccT, 1>(v, a, s);
    case 2: return launch_panels_vs<ValT, VecT, AccT, 2>(v, a, s);
    case 4: return launch_panels_vs<ValT, VecT, AccT, 4>(v, a, s);
    case 8: return launch_panels_vs<ValT, VecT, AccT, 8>(v, a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename ValT, typename VecT, typename AccT>
cudaError_t launch_spmv_impl(const spmv_variant &v, const RunArgs &a, cudaStream_t s) {
  if (a.n_rows == 0) return cudaSuccess;
  if (v.xpath >= 2) return launch_panels<ValT, VecT, AccT>(v, a, s);
  if (v.partition == 3) return launch_sell<ValT, VecT, AccT>(v, a, s);
  if (v.partition == 2)
    return launch_bins<ValT, VecT, AccT>(v.index == 1 ? a.delta_bits : 0, v.xpath != 0, a, s);
  if (v.partition == 1) {
    if (a.n_tiles == 0) return cudaSuccess;
    if (v.xpath) k_merge<ValT, VecT, AccT, true><<<(unsigned)a.n_tiles, kMergeThreads, 0, s>>>(a);
    else k_merge<ValT, VecT, AccT, false><<<(unsigned)a.n_tiles, kMergeThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.n_tiles > 1) {
      const unsigned g = (unsigned)(((a.n_tiles - 1) * 32 + 255) / 256);   // a warp per tile
      k_merge_fixup<VecT><<<g, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
  }
  switch (v.vs) {
    case 1: return launch_rowtile<ValT, VecT, AccT>(v, a, s);
    case 2: return launch_rowvec_vs<ValT, VecT, AccT, 2>(v, a, s);
    case 4: return launch_rowvec_vs<ValT, VecT, AccT, 4>(v, a, s);
    case 8: return launch_rowvec_vs<ValT, VecT, AccT, 8>(v, a, s);
    case 16: return launch_rowvec_vs<ValT, VecT, AccT, 16>(v, a, s);
    case 32: return launch_rowvec_vs<ValT, VecT, AccT, 32>(v, a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename ValT, typename VecT, typename AccT, int VS>
cudaError_t launch_spmm_vs(const RunArgs &a, cudaStream_t s) {
  const unsigned g = grid_for_rows(a.n_rows, VS);
  const int k = a.k;
  constexpr int PER = 16 / (int)sizeof(VecT);
  int off = 0;
  if (k % PER == 0) {
    for (; off + 16 <= k; off += 16) k_spmm<ValT, VecT, AccT, VS, 16><<<g, kRowThreads, 0, s>>>(a, off, k);
    for (; off + 4 <= k; off += 4) k_spmm<ValT, VecT, AccT, VS, 4><<<g, kRowThreads, 0, s>>>(a, off, k);
  }
  for (; off < k; ++off) k_spmm<ValT, VecT, AccT, VS, 1><<<g, kRowThreads, 0, s>>>(a, off, k);
  return cudaGetLastError();
}

template <typename ValT, typename VecT, typename AccT>
cudaError_t launch_spmm_impl(const RunArgs &a, int vs, cudaStream_t s) {
  if (a.n_rows == 0) return cudaSuccess;
  switch (vs) {
    case 2: return launch_spmm_vs<ValT, VecT, AccT, 2>(a, s);
    case 4: return launch_spmm_vs<ValT, VecT, AccT, 4>(a, s);
    case 8: return launch_spmm_vs<ValT, VecT, AccT, 8>(a, s);
    case 16: return launch_spmm_vs<ValT, VecT, AccT, 16>(a, s);
    case 32: return launch_spmm_vs<ValT, VecT, AccT, 32>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename ValT, typename VecT, typename AccT, int VS>
cudaError_t launch_static_vs(const ProfileArgs &a, cudaStream_t s) {
  if (a.cmp_mode) k_static<ValT, VecT, AccT, VS, true><<<a.n_ctas, kRowThreads, 0, s>>>(a);
  else k_static<ValT, VecT, AccT, VS, false><<<a.n_ctas, kRowThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename ValT, typename VecT, typename AccT>
cudaError_t launch_profile_impl(const ProfileArgs &a, cudaStream_t s) {
  if (a.n_ctas <= 0) return cudaSuccess;
  switch (a.vs) {
    case 2: return launch_static_vs<ValT, VecT, AccT, 2>(a, s);
    case 4: return launch_static_vs<ValT, VecT, AccT, 4>(a, s);
    case 8: return launch_static_vs<ValT, VecT, AccT, 8>(a, s);
    case 16: return launch_static_vs<ValT, VecT, AccT, 16>(a, s);
    case 32: return launch_static_vs<ValT, VecT, AccT, 32>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename ValT, typename VecT, typename AccT>
int profile_occupancy() {
  int blocks = 0;
  // all VS share the same resource footprint closely; take the largest-register one
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_static<ValT, VecT, AccT, 2, false>,
                                                kRowThreads, 0);
  return blocks > 0 ? blocks : 1;
}

}  // namespace spmv

// Defines kernel_set_<TAG>() for one dtype combination.
#define SPMV_DEFINE_SET(TAG, VALT, VECT, ACCT)                                          \
  namespace spmv {                                                                      \
  const KernelSet *kernel_set_##TAG() {                                                 \
    static KernelSet ks = {&launch_spmv_impl<VALT, VECT, ACCT>,                         \
                           &launch_spmm_impl<VALT, VECT, ACCT>,                         \
                           &launch_profile_impl<VALT, VECT, ACCT>, 0};                  \
    if (ks.profile_blocks_per_sm == 0)                                                  \
      ks.profile_blocks_per_sm = profile_occupancy<VALT, VECT, ACCT>();                 \
    return &ks;                                                                         \
  }                                                                                     \
  }

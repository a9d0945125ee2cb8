// FP64 SpMV whose products and sums run in the FP32 pipe as double-float arithmetic.
//
// GB300's FP64 pipe retires about 0.5 T FMA/s against 33 T for FP32, so FP64 SpMV with one
// FMA per nonzero is compute bound (the CMP class of Section III-A) on this GPU. Here every
// FP64 number is carried as an unevaluated sum hi + lo of two FP32 numbers:
//   - split: hi holds the top 24 significant bits of v (exact truncation), lo the next 23
//     (truncated), so |v - hi - lo| < 2^-46 |v|. The split is integer bit work; values are
//     split once when the precision is installed, x elements as they are gathered;
//   - product: hi_v*hi_x is taken exactly as a rounded product and its error (fmaf), plus
//     the cross terms hi_v*lo_x + lo_v*hi_x; lo_v*lo_x (< 2^-46 |v x|) is dropped. Together
//     with the split, each product is within about 6 * 2^-46 |v x| of v*x;
//   - sum: the row accumulator (s, t) is updated with an error-free two-sum of the high parts
//     (Knuth, TAOCP vol. 2, 4.2.2), the low parts added to its error, and a fast two-sum
//     renormalisation (Dekker 1971). Each step errs by at most about 6 u^2 (|s| + |p|),
//     u = 2^-24, so a row of n <= kDfMaxRow products ends within about
//     6 u^2 (n + 1) + 6 * 2^-46 < 8e-13 of sum_j |a_ij x_j|.
// Rows longer than kDfMaxRow, and rows that meet a value or an x element outside
// [2^-40, 2^41) (split to a NaN marker, so the double-float sum is not finite), are
// recomputed with native FP64 FMAs from the original FP64 values.
//
// The same kernel serves FP32 and BF16 storage with double-float accumulation: such a value
// is exact in the high part (low part zero), and so is an FP32 x element, so a product is
// the exact FP32 product plus its rounding error (and the x split's cross term for FP64 x);
// the sum is the same double-float recurrence. Against the stored values, rows keep the
// FP64 bound above at FP32 instruction rates.
#include "spmv_kernels.cuh"

namespace spmv {

namespace {
constexpr int kDfMaxRow = 32;
constexpr uint32_t kDfNanHi = 0x7FC00000u;   // quiet NaN: marks an unsplittable number
}  // namespace

// Split of one FP64 number into FP32 bit patterns (hi, lo), integer operations and one
// exact FP32 subtraction, without branches. Zero gives (+-0, 0); a nonzero outside
// [2^-40, 2^41) (biased exponent outside [983, 1063]), an infinity or a NaN gives (NaN, 0).
__device__ __forceinline__ uint2 df_split(double d) {
  const uint32_t H = (uint32_t)((unsigned long long)__double_as_longlong(d) >> 32);
  const uint32_t L = (uint32_t)(unsigned long long)__double_as_longlong(d);
  const uint32_t eb = (H >> 20) & 0x7FFu;
  // (H:L) << 3 puts the low 9 exponent bits and the top 23 fraction bits in one word; the
  // rebias 1023 -> 127 is a subtraction of 896 in the exponent field, taken modulo 2^9
  // (in range the result lies in [87, 167], so its ninth bit is zero)
  uint32_t hi = (__funnelshift_l(L, H, 3) - (384u << 23)) | (H & 0x80000000u);
  // lo = the next 23 fraction bits scaled by 2^(e - 46): (1.m - 1) * 2^(e - 23), an exact
  // FP32 subtraction of two numbers carrying hi's sign
  const uint32_t base = (hi & 0xFF800000u) - (23u << 23);
  const uint32_t m = (L >> 6) & 0x7FFFFFu;
  float lo = __fsub_rn(__uint_as_float(base | m), __uint_as_float(base));
  const bool out = eb - 983u > 80u;                  // also zero, subnormal, inf, NaN
  const bool zero = ((H & 0x7FFFFFFFu) | L) == 0u;
  hi = out ? (zero ? (H & 0x80000000u) : kDfNanHi) : hi;
  lo = out ? 0.0f : lo;
  return make_uint2(hi, __float_as_uint(lo));
}

__global__ void k_df_split(const double *__restrict__ in, uint2 *__restrict__ out, int64_t lo,
                           int64_t hi) {
  for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = df_split(in[i]);
}

cudaError_t launch_df_split(const double *in, void *out, int64_t lo, int64_t hi,
                            cudaStream_t s) {
  if (hi <= lo) return cudaSuccess;
  int64_t g = (hi - lo + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  k_df_split<<<(unsigned)g, 256, 0, s>>>(in, static_cast<uint2 *>(out), lo, hi);
  return cudaGetLastError();
}

namespace {

template <bool XL2> __device__ __forceinline__ uint2 ldx_pair(const uint2 *p, uint64_t pol) {
  if constexpr (XL2) {
    uint2 r;
    asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                 : "=r"(r.x), "=r"(r.y)
                 : "l"(p), "l"(pol));
    return r;
  } else {
    return __ldg(p);
  }
}

// A stored value as a double-float pair: DF64 storage holds the pair; an FP32 or BF16 value
// is exact in the high part. A nonzero outside [2^-40, 2^41) becomes the NaN marker, as in
// df_split, so that its row falls back to FP64.
__device__ __forceinline__ uint2 df_pair(uint2 v) { return v; }
__device__ __forceinline__ uint2 df_pair(float v) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t eb = (b >> 23) & 0xFFu;
  const bool out = eb - 87u > 80u;                   // biased exponent outside [87, 167]
  const bool zero = (b & 0x7FFFFFFFu) == 0u;
  return make_uint2(out ? (zero ? (b & 0x80000000u) : kDfNanHi) : b, 0u);
}
__device__ __forceinline__ uint2 df_pair(__nv_bfloat16 v) { return df_pair(__bfloat162float(v)); }

// An x element as a pair: FP64 x is split as gathered, FP32 x is exact in the high part.
template <bool XL2> __device__ __forceinline__ uint2 df_x(const double *p, uint64_t pol) {
  return df_split(ldx<XL2>(p, pol));
}
template <bool XL2> __device__ __forceinline__ uint2 df_x(const float *p, uint64_t pol) {
  return df_pair(ldx<XL2>(p, pol));
}

// (s, t) += (p, q); the _rn intrinsics keep each operation as written.
__device__ __forceinline__ void df_add(float &s, float &t, float p, float q) {
  const float S = __fadd_rn(s, p);
  const float b = __fsub_rn(S, s);
  float e = __fadd_rn(__fsub_rn(s, __fsub_rn(S, b)), __fsub_rn(p, b));
  e = __fadd_rn(e, __fadd_rn(t, q));
  s = __fadd_rn(S, e);
  t = __fsub_rn(e, __fsub_rn(s, S));
}

// v * x as (p, q): p = fl(hi_v hi_x), q = its rounding error + hi_v lo_x + lo_v hi_x; VLO /
// XLO say whether v / x have a low part at all (a zero one contributes nothing).
template <bool VLO, bool XLO>
__device__ __forceinline__ void df_prod(uint2 v, uint2 xv, float &p, float &q) {
  const float vh = __uint_as_float(v.x), vl = __uint_as_float(v.y);
  const float xh = __uint_as_float(xv.x), xl = __uint_as_float(xv.y);
  p = __fmul_rn(vh, xh);
  const float pe = __fmaf_rn(vh, xh, -p);
  if constexpr (VLO && XLO) q = __fadd_rn(__fmaf_rn(vh, xl, __fmul_rn(vl, xh)), pe);
  else if constexpr (XLO) q = __fmaf_rn(vh, xl, pe);
  else if constexpr (VLO) q = __fmaf_rn(vl, xh, pe);
  else q = pe;
}

// The values a staged tile holds for the double-float kernel and the storage type the FP64
// fallbacks read: DF64 stages pairs and falls back to the FP64 originals; FP32 / BF16 stage
// and fall back to the stored values themselves.
template <typename ValT> struct DfStore { using type = ValT; };
template <> struct DfStore<uint2> { using type = double; };

}  // namespace

// Thread-per-row tiles as in the FP64 kernel: a tile's values (pairs, or FP32 / BF16) and
// column indices are staged in shared memory by one bulk copy each; each thread then walks
// its row.
template <typename ValT, typename VecT, int DB, bool XL2>
__global__ void __launch_bounds__(kTileRows) k_rowtile_df(const RunArgs a) {
  using StoreT = typename DfStore<ValT>::type;
  constexpr bool VLO = std::is_same<ValT, uint2>::value;
  constexpr bool XLO = std::is_same<VecT, double>::value;
  using IdxT = typename IdxOf<DB>::type;
  constexpr int AL = stage_align<DB>();
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  const int rows = (int)blockDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rows;
  const int64_t r1 = min(r0 + (int64_t)rows, a.n_rows);
  const int s0 = __ldg(a.rowptr + r0), s1 = __ldg(a.rowptr + r1);
  const int a0 = s0 & ~(AL - 1);
  const int nc = ((s1 - a0) + AL - 1) & ~(AL - 1);
  const StoreT *__restrict__ val = static_cast<const StoreT *>(a.val);
  const ValT *__restrict__ vdf =
      static_cast<const ValT *>(VLO ? a.val_df : a.val);   // the staged values
  const VecT *__restrict__ x = static_cast<const VecT *>(a.x);
  VecT *__restrict__ y = static_cast<VecT *>(a.y);
  uint64_t pol_x = 0;
  if constexpr (XL2) pol_x = policy_evict_last();
  const int64_t row = r0 + threadIdx.x;
  if (nc > a.tile_cap) {
    tile_direct<StoreT, VecT, double, DB, XL2>(a, r0, r1, x, y, pol_x);
    return;
  }
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
      bulk_g2s(sval, vdf + a0, bv, bar, pol);
      bulk_g2s(sidx, gidx + a0, bi, bar, pol);
    }
  }
  int s = 0, e = 0;
  int32_t base = 0;
  if (row < r1) {
    s = __ldg(a.rowptr + row);
    e = __ldg(a.rowptr + row + 1);
    if constexpr (DB != 0) base = __ldg(a.dbase + row);
  }
  __syncthreads();
  if (nc > 0) {
    if (!mbar_wait_bounded(bar, 0, kWaitLimitNs)) {
      if (threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
      mbar_wait_bounded(bar, 0, kWaitLimitNs);
      return;
    }
  }
  if (row >= r1) return;
  const int o = s - a0, len = e - s;
  const int32_t *ec = nullptr;
  if constexpr (DB != 0) {
    if (base < 0) ec = a.esc + (-(int64_t)base - 1);
  }
  int c = base;
  auto column = [&](int k) -> int {
    if constexpr (DB != 0) {
      if (ec) return __ldg(ec + k);
      c += (int)sidx[o + k];
      return c;
    } else {
      return (int)sidx[o + k];
    }
  };
  if (len <= kDfMaxRow) {
    float sh = 0.0f, sl = 0.0f;
    int k = 0;
    for (; k + 16 <= len; k += 16) {
      uint2 xv[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) xv[q] = df_x<XL2>(x + column(k + q), pol_x);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        float p, pq;
        df_prod<VLO, XLO>(df_pair(sval[o + k + q]), xv[q], p, pq);
        df_add(sh, sl, p, pq);
      }
    }
    for (; k + 8 <= len; k += 8) {
      uint2 xv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) xv[q] = df_x<XL2>(x + column(k + q), pol_x);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float p, pq;
        df_prod<VLO, XLO>(df_pair(sval[o + k + q]), xv[q], p, pq);
        df_add(sh, sl, p, pq);
      }
    }
    for (; k < len; ++k) {
      float p, pq;
      df_prod<VLO, XLO>(df_pair(sval[o + k]), df_x<XL2>(x + column(k), pol_x), p, pq);
      df_add(sh, sl, p, pq);
    }
    if (isfinite(sh)) {
      y[row] = (VecT)((double)sh + (double)sl);
      return;
    }
    c = base;   // restart the delta decode for the FP64 pass
  }
  // FP64 FMAs in the FP64-accumulating tile kernel's order: element order, in the two
  // chains of fp64_chain_of when the columns are delta-coded
  double acc = 0.0, acc1 = 0.0;
  for (int k = 0; k < len; ++k) {
    const double p = widen<double>(val[s + k]), xk = (double)ldx<XL2>(x + column(k), pol_x);
    if (DB != 0 && fp64_chain_of(k, len)) acc1 = fma(p, xk, acc1);
    else acc = fma(p, xk, acc);
  }
  y[row] = (VecT)(DB != 0 ? acc + acc1 : acc);
}

namespace {

template <typename ValT, typename VecT, int DB, bool XL2>
cudaError_t launch_rowtile_df_k(const RunArgs &a, cudaStream_t s) {
  static std::atomic<int> configured{0};
  const int rows = a.tile_rows > 0 ? a.tile_rows : kTileRows;
  const size_t smem = 16 + (size_t)a.tile_cap * (sizeof(ValT) + sizeof(typename IdxOf<DB>::type));
  cudaError_t e = ensure_smem(k_rowtile_df<ValT, VecT, DB, XL2>, smem, configured);
  if (e != cudaSuccess) return e;
  const unsigned g = (unsigned)((a.n_rows + rows - 1) / rows);
  k_rowtile_df<ValT, VecT, DB, XL2><<<g, rows, smem, s>>>(a);
  return cudaGetLastError();
}

// Width-1 row variants run the double-float tile kernel (one tile per CTA, whatever
// tile_pipe says); every other variant (column panels included) runs the FP64-accumulating
// kernels of `base` (for DF64 storage on the FP64 originals).
template <typename ValT, typename VecT>
cudaError_t launch_spmv_df(const KernelSet *base, const spmv_variant &v, const RunArgs &a,
                           cudaStream_t s) {
  if (a.n_rows == 0) return cudaSuccess;
  if (v.partition != 0 || v.vs != 1 || v.xpath >= 2) return base->spmv(v, a, s);
  const bool xl2 = v.xpath != 0;
  if (v.index == 1 && a.delta_bits == 8)
    return xl2 ? launch_rowtile_df_k<ValT, VecT, 8, true>(a, s)
               : launch_rowtile_df_k<ValT, VecT, 8, false>(a, s);
  if (v.index == 1)
    return xl2 ? launch_rowtile_df_k<ValT, VecT, 16, true>(a, s)
               : launch_rowtile_df_k<ValT, VecT, 16, false>(a, s);
  return xl2 ? launch_rowtile_df_k<ValT, VecT, 0, true>(a, s)
             : launch_rowtile_df_k<ValT, VecT, 0, false>(a, s);
}

cudaError_t spmv_f64_df(const spmv_variant &v, const RunArgs &a, cudaStream_t s) {
  return launch_spmv_df<uint2, double>(kernel_set_f64_dd(), v, a, s);
}
cudaError_t spmv_f32_d_df(const spmv_variant &v, const RunArgs &a, cudaStream_t s) {
  return launch_spmv_df<float, double>(kernel_set_f32_dd(), v, a, s);
}
cudaError_t spmv_f32_f_df(const spmv_variant &v, const RunArgs &a, cudaStream_t s) {
  return launch_spmv_df<float, float>(kernel_set_f32_fd(), v, a, s);
}
cudaError_t spmv_bf16_d_df(const spmv_variant &v, const RunArgs &a, cudaStream_t s) {
  return launch_spmv_df<__nv_bfloat16, double>(kernel_set_bf16_dd(), v, a, s);
}
cudaError_t spmv_bf16_f_df(const spmv_variant &v, const RunArgs &a, cudaStream_t s) {
  return launch_spmv_df<__nv_bfloat16, float>(kernel_set_bf16_fd(), v, a, s);
}

// The base set with its SpMV launcher replaced (profiling, SpMM as in the base set).
const KernelSet *df_set(const KernelSet *base, spmv_launch_fn fn, KernelSet *slot) {
  *slot = *base;
  slot->spmv = fn;
  return slot;
}

}  // namespace

const KernelSet *kernel_set_f64_df() {
  static KernelSet ks;
  static const KernelSet *p = df_set(kernel_set_f64_dd(), &spmv_f64_df, &ks);
  return p;
}
const KernelSet *kernel_set_f32_d_df() {
  static KernelSet ks;
  static const KernelSet *p = df_set(kernel_set_f32_dd(), &spmv_f32_d_df, &ks);
  return p;
}
const KernelSet *kernel_set_f32_f_df() {
  static KernelSet ks;
  static const KernelSet *p = df_set(kernel_set_f32_fd(), &spmv_f32_f_df, &ks);
  return p;
}
const KernelSet *kernel_set_bf16_d_df() {
  static KernelSet ks;
  static const KernelSet *p = df_set(kernel_set_bf16_dd(), &spmv_bf16_d_df, &ks);
  return p;
}
const KernelSet *kernel_set_bf16_f_df() {
  static KernelSet ks;
  static const KernelSet *p = df_set(kernel_set_bf16_fd(), &spmv_bf16_f_df, &ks);
  return p;
}

}  // namespace spmv

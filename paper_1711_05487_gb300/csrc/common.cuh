// Device-side helpers shared by the SpMV kernels: dtype conversion, cache-hinted loads
// (inline PTX), sub-warp reductions and scans.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace spmv {

// ------------------------------------------------------------------ dtype traits ------
template <typename T> struct DT;
template <> struct DT<double> { static constexpr spmv_dtype id = SPMV_F64; };
template <> struct DT<float> { static constexpr spmv_dtype id = SPMV_F32; };
template <> struct DT<__nv_bfloat16> { static constexpr spmv_dtype id = SPMV_BF16; };

template <typename AccT> __device__ __forceinline__ AccT widen(double v) { return (AccT)v; }
template <typename AccT> __device__ __forceinline__ AccT widen(float v) { return (AccT)v; }
template <typename AccT> __device__ __forceinline__ AccT widen(__nv_bfloat16 v) {
  return (AccT)__bfloat162float(v);
}

// ------------------------------------------------- FP32 accumulation within its bound ----
// With FP32 accumulation a row's result must stay within 2e-6 of sum_j |a_ij x_j| (the
// FP32-storage tolerance). Every FP32 addition rounds the running sum by at most
// u = 2^-24 of its magnitude, which is at most sum_j |a_ij x_j|, so a value that went
// through n roundings errs by at most n u. No FP32 running sum therefore takes more than
// about 30 roundings (its products, its share of a lane reduction, the final store, and
// one for values rounded to FP32 from FP64): a row whose chain would be longer is summed
// in runs of kF32Run products whose sums are added into an FP32 pair (at most 16 u + the
// final store).
constexpr int kF32Run = 16;     // products per FP32 run before its sum is set aside
constexpr int kF32Chain = 30;   // most roundings one FP32 running sum may take
template <typename AccT> struct IsF32 { static constexpr bool value = false; };
template <> struct IsF32<float> { static constexpr bool value = true; };

// The run sums are added into an FP32 pair hi + lo with Knuth's two-sum (the addition
// hi + a = s + e is exact in FP32, e goes to lo), so their total carries an error of order
// u^2 and stays on the FP32 pipe (GB300's FP64 pipe runs at 1/64 of its FP32 rate).
struct FPair {
  float hi = 0.0f, lo = 0.0f;
};
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// Wide sums: FPair for FP32 runs, the type itself otherwise.
__device__ __forceinline__ void wadd(FPair &w, float a) {
  float s, e;
  two_sum(w.hi, a, s, e);
  w.hi = s;
  w.lo += e;
}
__device__ __forceinline__ void wadd(FPair &w, const FPair &o) {
  float s, e;
  two_sum(w.hi, o.hi, s, e);
  w.hi = s;
  w.lo += o.lo + e;
}
__device__ __forceinline__ void wadd(double &w, double a) { w += a; }
__device__ __forceinline__ void wadd(float &w, float a) { w += a; }
__device__ __forceinline__ float wvalue(const FPair &w) { return w.hi + w.lo; }
__device__ __forceinline__ double wvalue(double w) { return w; }
__device__ __forceinline__ float wvalue(float w) { return w; }
__device__ __forceinline__ double wdouble(const FPair &w) { return (double)w.hi + (double)w.lo; }
__device__ __forceinline__ double wdouble(double w) { return w; }
template <typename AccT> struct WideOf { using type = AccT; };
template <> struct WideOf<float> { using type = FPair; };

// bf16 held in the low / high half of a 32-bit word -> float (exact)
__device__ __forceinline__ float bf16lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// ---------------------------------------------------------------- L2 cache policies ---
// createpolicy gives a 64-bit L2 eviction policy for the .L2::cache_hint loads below.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Streamed data: read-only path, evict-first in L2. The lines are allocated in L1: the
// 16-byte chunks that neighbouring short rows' sub-warps read share lines across
// instructions (on GB300, skipping L1 allocation cost the row decomposition 0.7 % on the
// power-law matrix and the delta-coded sub-warp kernel 5 % on the stencil).
__device__ __forceinline__ uint4 ld_stream_u4(const void *p, uint64_t pol) {
  uint4 r;
  asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ uint2 ld_stream_u2(const void *p, uint64_t pol) {
  uint2 r;
  asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
               : "=r"(r.x), "=r"(r.y)
               : "l"(p), "l"(pol));
  return r;
}
// Plain 128-bit read-only load.
__device__ __forceinline__ uint4 ld_nc_u4(const void *p) {
  uint4 r;
  asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}
__device__ __forceinline__ uint2 ld_nc_u2(const void *p) {
  uint2 r;
  asm volatile("ld.global.nc.v2.u32 {%0,%1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
  return r;
}

template <bool HINT> __device__ __forceinline__ uint4 ld16(const void *p, uint64_t pol) {
  if constexpr (HINT) return ld_stream_u4(p, pol);
  else return ld_nc_u4(p);
}
template <bool HINT> __device__ __forceinline__ uint2 ld8(const void *p, uint64_t pol) {
  if constexpr (HINT) return ld_stream_u2(p, pol);
  else return ld_nc_u2(p);
}

// x gathers: evict-last keeps x resident in L2 while the matrix streams past it.
// NA: the gather allocates no L1 line (x gathers of a column-panel pass, which land on an
// L2-sized slice at random and are almost never reused from L1).
template <bool XL2, bool NA = false>
__device__ __forceinline__ double ldx(const double *p, uint64_t pol) {
  if constexpr (XL2 && NA) {
    double r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;"
                 : "=d"(r) : "l"(p), "l"(pol));
    return r;
  } else if constexpr (XL2) {
    double r;
    asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(p), "l"(pol));
    return r;
  } else {
    return __ldg(p);
  }
}
template <bool XL2, bool NA = false>
__device__ __forceinline__ float ldx(const float *p, uint64_t pol) {
  if constexpr (XL2 && NA) {
    float r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;"
                 : "=f"(r) : "l"(p), "l"(pol));
    return r;
  } else if constexpr (XL2) {
    float r;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(p), "l"(pol));
    return r;
  } else {
    return __ldg(p);
  }
}

// Read-modify-write data touched once (y of a column-panel pass): a coherent load and a
// store, both with an L2 eviction policy.
__device__ __forceinline__ double ld_hint(const double *p, uint64_t pol) {
  double r;
  asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float ld_hint(const float *p, uint64_t pol) {
  float r;
  asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ void st_hint(double *p, double v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(float *p, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ int32_t ld_hint_nc(const int32_t *p, uint64_t pol) {
  int32_t r;
  asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
  return r;
}

// ---------------------------------------------------- vector loads of E values --------
// Loads E consecutive values starting at an E-aligned index into AccT registers.
template <typename AccT, bool HINT, int E> struct VLoad;

template <typename AccT, bool HINT> struct VLoad<AccT, HINT, 4> {
  __device__ __forceinline__ static void run(const double *p, AccT *o, uint64_t pol) {
    uint4 a = ld16<HINT>(p, pol), b = ld16<HINT>(p + 2, pol);
    o[0] = (AccT)__hiloint2double(a.y, a.x);
    o[1] = (AccT)__hiloint2double(a.w, a.z);
    o[2] = (AccT)__hiloint2double(b.y, b.x);
    o[3] = (AccT)__hiloint2double(b.w, b.z);
  }
  __device__ __forceinline__ static void run(const float *p, AccT *o, uint64_t pol) {
    uint4 a = ld16<HINT>(p, pol);
    o[0] = (AccT)__uint_as_float(a.x);
    o[1] = (AccT)__uint_as_float(a.y);
    o[2] = (AccT)__uint_as_float(a.z);
    o[3] = (AccT)__uint_as_float(a.w);
  }
  __device__ __forceinline__ static void run(const __nv_bfloat16 *p, AccT *o, uint64_t pol) {
    uint2 a = ld8<HINT>(p, pol);
    o[0] = (AccT)bf16lo(a.x);
    o[1] = (AccT)bf16hi(a.x);
    o[2] = (AccT)bf16lo(a.y);
    o[3] = (AccT)bf16hi(a.y);
  }
};

template <typename AccT, bool HINT> struct VLoad<AccT, HINT, 8> {
  template <typename ValT>
  __device__ __forceinline__ static void run(const ValT *p, AccT *o, uint64_t pol) {
    if constexpr (sizeof(ValT) == 2) {
      uint4 a = ld16<HINT>(p, pol);
      o[0] = (AccT)bf16lo(a.x); o[1] = (AccT)bf16hi(a.x);
      o[2] = (AccT)bf16lo(a.y); o[3] = (AccT)bf16hi(a.y);
      o[4] = (AccT)bf16lo(a.z); o[5] = (AccT)bf16hi(a.z);
      o[6] = (AccT)bf16lo(a.w); o[7] = (AccT)bf16hi(a.w);
    } else {
      VLoad<AccT, HINT, 4>::run(p, o, pol);
      VLoad<AccT, HINT, 4>::run(p + 4, o + 4, pol);
    }
  }
};

// ------------------------------------------------------------ sub-warp collectives ----
// Lanes [g*VS, (g+1)*VS) of a warp form sub-warp g; mask selects exactly those lanes.
template <int VS> __device__ __forceinline__ unsigned group_mask() {
  if constexpr (VS == 32) return 0xffffffffu;
  else return ((1u << VS) - 1u) << ((threadIdx.x & 31) & ~(VS - 1));
}

template <int VS, typename T> __device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
  for (int off = VS / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off, VS);
  return v;
}
// The same tree over FP32 pairs (both halves shuffled, high parts added by two-sum).
template <int VS> __device__ __forceinline__ FPair group_sum(FPair v, unsigned mask) {
#pragma unroll
  for (int off = VS / 2; off > 0; off >>= 1) {
    FPair o;
    o.hi = __shfl_xor_sync(mask, v.hi, off, VS);
    o.lo = __shfl_xor_sync(mask, v.lo, off, VS);
    wadd(v, o);
  }
  return v;
}

// Inclusive scan over the sub-warp (Hillis-Steele with shuffles).
template <int VS> __device__ __forceinline__ int group_incl_scan(int v, int lane, unsigned mask) {
#pragma unroll
  for (int off = 1; off < VS; off <<= 1) {
    int t = __shfl_up_sync(mask, v, off, VS);
    if (lane >= off) v += t;
  }
  return v;
}

// ------------------------------------------------- mbarrier + bulk async copy (TMA) ----
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  // make the initialised barrier visible to the async (TMA) proxy
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// One bulk copy global -> shared of `bytes` (multiple of 16, both addresses 16-byte
// aligned), completing on the mbarrier, with an L2 eviction policy for the source.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}
// Arrival without a transaction count (completes a phase that has nothing to copy).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns();

// Waits for phase `parity` of the barrier for at most limit_ns of wall time; false when
// the limit expired (the caller records the error and must not read the staged data).
// Also bounded by an iteration count, so that the wait ends even if the clock stalled.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return false;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

}  // namespace spmv

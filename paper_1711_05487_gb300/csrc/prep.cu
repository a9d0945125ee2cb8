// Preprocessing kernels: CSR validation, value precision conversion, the 16-bit delta
// column index, merge-path tile table, static profiling partition, Table I feature
// extraction and the read-bandwidth probe.
#include <climits>

#include "common.cuh"

namespace spmv {

namespace {
constexpr int kT = 256;

inline unsigned blocks_for(int64_t n, int per_block = kT) {
  int64_t b = (n + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > 2147483647LL) b = 2147483647LL;
  return (unsigned)b;
}
}  // namespace

// ----------------------------------------------------------------- CSR validation -----
// Codes follow the CSR definition (Section II): 1 rowptr[0] != 0, 2 rowptr decreases,
// 3 rowptr[n] != nnz, 4 column out of range, 5 columns not strictly increasing. For the
// element checks the first offending element in storage order decides between 4 and 5.
__global__ void k_validate_rowptr(int64_t n_rows, int64_t nnz, const int32_t *rowptr,
                                  int32_t *flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    if (rowptr[0] != 0) atomicOr(flags, 1);
    if ((int64_t)rowptr[n_rows] != nnz) atomicOr(flags, 4);
  }
  if (i < n_rows && rowptr[i + 1] < rowptr[i]) atomicOr(flags, 2);
}

__global__ void k_validate_finish(const int32_t *flags, const unsigned long long *first_bad,
                                  int32_t *code) {
  const int f = *flags;
  int c = 0;
  if (f & 1) c = 1;
  else if (f & 2) c = 2;
  else if (f & 4) c = 3;
  else if (*first_bad != ~0ull) c = (int)(*first_bad & 7ull);
  *code = c;
}

__global__ void k_init_validate(int32_t *flags, unsigned long long *first_bad) {
  *flags = 0;
  *first_bad = ~0ull;
}

__global__ void k_validate_cols_guarded(int64_t n_rows, int64_t n_cols, const int32_t *rowptr,
                                        const int32_t *colind, const int32_t *flags,
                                        unsigned long long *first_bad) {
  if (*flags != 0) return;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= n_rows) return;
  const int s = rowptr[i], e = rowptr[i + 1];
  for (int j = s + lane; j < e; j += 32) {
    const int c = colind[j];
    int code = 0;
    if (c < 0 || (int64_t)c >= n_cols) code = 4;
    else if (j > s && c <= colind[j - 1]) code = 5;
    if (code) atomicMin(first_bad, ((unsigned long long)j << 3) | (unsigned long long)code);
  }
}

// d_code points at 16 bytes of device scratch: [code, flags, first_bad (8 bytes)].
// The element pass reads colind only when every rowptr check passed (then all offsets lie
// in [0, nnz]).
cudaError_t launch_validate(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t *rowptr,
                            const int32_t *colind, int32_t *d_code, cudaStream_t s) {
  int32_t *flags = d_code + 1;
  unsigned long long *first_bad = reinterpret_cast<unsigned long long *>(d_code + 2);
  k_init_validate<<<1, 1, 0, s>>>(flags, first_bad);
  k_validate_rowptr<<<blocks_for(n_rows + 1), kT, 0, s>>>(n_rows, nnz, rowptr, flags);
  if (n_rows > 0)
    k_validate_cols_guarded<<<blocks_for(n_rows, kT / 32), kT, 0, s>>>(n_rows, n_cols, rowptr,
                                                                       colind, flags, first_bad);
  k_validate_finish<<<1, 1, 0, s>>>(flags, first_bad, d_code);
  return cudaGetLastError();
}

// ---------------------------------------------------------- value precision codec -----
// FP64 -> BF16, round to nearest even without double rounding: the value is first
// rounded to FP32 with round-to-odd (truncate, then set the last bit if anything was
// cut off; Boldo & Melquiond, "When double rounding is odd", 2005), which keeps enough
// bits (24 >= 8 + 2) for the second, round-to-nearest-even step to FP32 -> BF16 to give
// the correctly rounded result.
__device__ __forceinline__ uint16_t f64_to_bf16_rne(double v) {
  if (isnan(v)) return signbit(v) ? (uint16_t)0xFFC0u : (uint16_t)0x7FC0u;
  float f = __double2float_rz(v);
  uint32_t u = __float_as_uint(f);
  if ((double)f != v && !isinf(v)) u |= 1u;   // round to odd
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);  // +-inf
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;                          // nearest, ties to even
  return (uint16_t)(u >> 16);
}

__global__ void k_round_values(const double *in, void *out, int64_t n, int to) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = in[i];
    if (to == SPMV_F64) static_cast<double *>(out)[i] = v;
    else if (to == SPMV_F32) static_cast<float *>(out)[i] = __double2float_rn(v);
    else static_cast<uint16_t *>(out)[i] = f64_to_bf16_rne(v);
  }
}

cudaError_t launch_round_values(const double *in, void *out, int64_t n, spmv_dtype to,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  unsigned g = blocks_for(n);
  if (g > 65536u) g = 65536u;
  k_round_values<<<g, kT, 0, s>>>(in, out, n, (int)to);
  return cudaGetLastError();
}

__device__ __forceinline__ double load_as_f64(const void *p, int t, int64_t i) {
  if (t == SPMV_F64) return static_cast<const double *>(p)[i];
  if (t == SPMV_F32) return (double)static_cast<const float *>(p)[i];
  return (double)__uint_as_float(((uint32_t) static_cast<const uint16_t *>(p)[i]) << 16);
}

__global__ void k_convert_values(const void *in, int from, void *out, int to, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = load_as_f64(in, from, i);
    if (to == SPMV_F64) static_cast<double *>(out)[i] = v;
    else if (to == SPMV_F32) static_cast<float *>(out)[i] = __double2float_rn(v);
    else static_cast<uint16_t *>(out)[i] = f64_to_bf16_rne(v);
  }
}

cudaError_t launch_convert_values(const void *in, spmv_dtype from, void *out, spmv_dtype to,
                                  int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  unsigned g = blocks_for(n);
  if (g > 65536u) g = 65536u;
  k_convert_values<<<g, kT, 0, s>>>(in, (int)from, out, (int)to, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ delta index --------
// Per row (a warp each): esc8[i] / esc16[i] = the row's length if some consecutive column
// distance exceeds 255 / 65535, else 0 (scans turn these into escape offsets and totals).
__global__ void k_delta_flags(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                              int64_t *esc8, int64_t *esc16) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= n_rows) return;
  const int s = rowptr[i], e = rowptr[i + 1];
  int64_t maxd = 0;
  for (int j = s + 1 + lane; j < e; j += 32)
    maxd = max(maxd, (int64_t)colind[j] - (int64_t)colind[j - 1]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) maxd = max(maxd, __shfl_xor_sync(0xffffffffu, maxd, off));
  if (lane == 0) {
    esc8[i] = maxd > 255 ? (int64_t)(e - s) : 0;
    esc16[i] = maxd > 65535 ? (int64_t)(e - s) : 0;
  }
}

template <typename T>
__global__ void k_delta_fill(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                             const int64_t *esc_off, int32_t *dbase, T *delta, int32_t *esc) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= n_rows) return;
  const int s = rowptr[i], e = rowptr[i + 1];
  if (s == e) {
    if (lane == 0) dbase[i] = 0;
    return;
  }
  const bool escape = esc_off[i + 1] != esc_off[i];
  if (escape) {
    const int64_t off = esc_off[i];
    if (lane == 0) dbase[i] = (int32_t)(-(1 + off));
    for (int j = s + lane; j < e; j += 32) {
      delta[j] = 0;
      esc[off + (j - s)] = colind[j];
    }
  } else {
    if (lane == 0) dbase[i] = colind[s];
    for (int j = s + lane; j < e; j += 32)
      delta[j] = (j == s) ? (T)0 : (T)(colind[j] - colind[j - 1]);
  }
}

cudaError_t launch_delta_flags(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                               int64_t *esc8, int64_t *esc16, cudaStream_t s) {
  if (n_rows == 0) return cudaSuccess;
  k_delta_flags<<<blocks_for(n_rows, kT / 32), kT, 0, s>>>(n_rows, rowptr, colind, esc8, esc16);
  return cudaGetLastError();
}

// esc_off has n_rows + 1 entries (exclusive scan of the chosen width's counts, total last).
cudaError_t launch_delta_fill(int bits, int64_t n_rows, const int32_t *rowptr,
                              const int32_t *colind, const int64_t *esc_off, int32_t *dbase,
                              void *delta, int32_t *esc, cudaStream_t s) {
  if (n_rows == 0) return cudaSuccess;
  const unsigned g = blocks_for(n_rows, kT / 32);
  if (bits == 8)
    k_delta_fill<uint8_t><<<g, kT, 0, s>>>(n_rows, rowptr, colind, esc_off, dbase,
                                           static_cast<uint8_t *>(delta), esc);
  else
    k_delta_fill<uint16_t><<<g, kT, 0, s>>>(n_rows, rowptr, colind, esc_off, dbase,
                                            static_cast<uint16_t *>(delta), esc);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_delta_decode(int64_t n_rows, const int32_t *rowptr, const int32_t *dbase,
                               const T *delta, const int32_t *esc, int32_t *colind) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows) return;
  const int s = rowptr[i], e = rowptr[i + 1];
  if (s == e) return;
  const int32_t b = dbase[i];
  if (b < 0) {
    const int64_t off = -(int64_t)b - 1;
    for (int j = s; j < e; ++j) colind[j] = esc[off + (j - s)];
  } else {
    int c = b;
    for (int j = s; j < e; ++j) {
      c += delta[j];
      colind[j] = c;
    }
  }
}

cudaError_t launch_delta_decode(int bits, int64_t n_rows, const int32_t *rowptr,
                                const int32_t *dbase, const void *delta, const int32_t *esc,
                                int32_t *colind, cudaStream_t s) {
  if (n_rows == 0) return cudaSuccess;
  if (bits == 8)
    k_delta_decode<uint8_t><<<blocks_for(n_rows), kT, 0, s>>>(
        n_rows, rowptr, dbase, static_cast<const uint8_t *>(delta), esc, colind);
  else
    k_delta_decode<uint16_t><<<blocks_for(n_rows), kT, 0, s>>>(
        n_rows, rowptr, dbase, static_cast<const uint16_t *>(delta), esc, colind);
  return cudaGetLastError();
}

// ------------------------------------------------------------- exclusive scan (i64) ---
// Three passes: per-block sums, a single-block scan of the block sums, then per-block
// scans with the block offset added. Deterministic (integer).
constexpr int kScanBlock = 1024;   // elements per block (256 threads x 4)

__global__ void k_scan_block_sums(const int64_t *data, int64_t n, int64_t *sums) {
  __shared__ int64_t sh[kT];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  int64_t acc = 0;
  for (int q = 0; q < 4; ++q) {
    const int64_t i = base + threadIdx.x * 4 + q;
    if (i < n) acc += data[i];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = kT / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = sh[0];
}

__global__ void k_scan_sums_serial(int64_t *sums, int64_t nb, int64_t *total) {
  // single thread block: chunked scan of up to a few hundred thousand block sums
  __shared__ int64_t sh[kT];
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += kT) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < nb ? sums[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kT; off <<= 1) {
      int64_t t = (int)threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) sums[i] = carry + sh[threadIdx.x] - v;
    carry += sh[kT - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_apply(int64_t *data, int64_t n, const int64_t *sums) {
  __shared__ int64_t sh[kT];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock;
  int64_t v[4];
  int64_t acc = 0;
  for (int q = 0; q < 4; ++q) {
    const int64_t i = base + threadIdx.x * 4 + q;
    v[q] = i < n ? data[i] : 0;
    acc += v[q];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = 1; off < kT; off <<= 1) {
    int64_t t = (int)threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int64_t run = sums[blockIdx.x] + sh[threadIdx.x] - acc;
  for (int q = 0; q < 4; ++q) {
    const int64_t i = base + threadIdx.x * 4 + q;
    if (i < n) data[i] = run;
    run += v[q];
  }
}

int64_t scan_scratch_elems(int64_t n) { return (n + kScanBlock - 1) / kScanBlock + 1; }

cudaError_t launch_scan_i64(int64_t *data, int64_t n, int64_t *total, int64_t *scratch,
                            int64_t scratch_elems, cudaStream_t s) {
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  if (nb + 1 > scratch_elems) return cudaErrorInvalidValue;
  if (n == 0) {
    return cudaMemsetAsync(total, 0, sizeof(int64_t), s);
  }
  k_scan_block_sums<<<(unsigned)nb, kT, 0, s>>>(data, n, scratch);
  k_scan_sums_serial<<<1, kT, 0, s>>>(scratch, nb, total);
  k_scan_apply<<<(unsigned)nb, kT, 0, s>>>(data, n, scratch);
  return cudaGetLastError();
}

// -------------------------------------------------------------- merge-path table ------
// coord[t] = (rows ended, nonzeros consumed) after min(t * items, n_rows + nnz) items of
// the merge of row ends (row i ends at rowptr[i+1]) with nonzeros 0..nnz-1, where a row
// end goes first when rowptr[i+1] <= the nonzero's index.
__global__ void k_merge_coords(int64_t n_rows, int64_t nnz, const int32_t *rowptr,
                               int64_t items, int64_t n_tiles, int2 *coord) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t > n_tiles) return;
  int64_t d = t * items;
  const int64_t total = n_rows + nnz;
  if (d > total) d = total;
  int64_t lo = d - nnz > 0 ? d - nnz : 0;
  int64_t hi = d < n_rows ? d : n_rows;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)rowptr[mid + 1] <= d - 1 - mid) lo = mid + 1;
    else hi = mid;
  }
  coord[t] = make_int2((int)lo, (int)(d - lo));
}

cudaError_t launch_merge_coords(int64_t n_rows, int64_t nnz, const int32_t *rowptr,
                                int64_t items, int64_t n_tiles, int2 *coord, cudaStream_t s) {
  k_merge_coords<<<blocks_for(n_tiles + 1), kT, 0, s>>>(n_rows, nnz, rowptr, items, n_tiles, coord);
  return cudaGetLastError();
}

// ------------------------------------------------------ static profiling partition ----
// part[c] = first row whose start offset is >= round(c * nnz / n_parts): contiguous row
// ranges of about equal nonzero counts, rows never split (the paper's baseline
// partitioning, Section IV-A).
__global__ void k_static_partition(int64_t n_rows, int64_t nnz, const int32_t *rowptr,
                                   int32_t n_parts, int32_t *part) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c > n_parts) return;
  if (c == 0) { part[0] = 0; return; }
  if (c == n_parts) { part[n_parts] = (int32_t)n_rows; return; }
  const int64_t target = (c * nnz + n_parts / 2) / n_parts;
  int64_t lo = 0, hi = n_rows;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)rowptr[mid] < target) lo = mid + 1;
    else hi = mid;
  }
  part[c] = (int32_t)lo;
}

cudaError_t launch_static_partition(int64_t n_rows, int64_t nnz, const int32_t *rowptr,
                                    int32_t n_parts, int32_t *part, cudaStream_t s) {
  k_static_partition<<<blocks_for((int64_t)n_parts + 1), kT, 0, s>>>(n_rows, nnz, rowptr, n_parts, part);
  return cudaGetLastError();
}

// colind'[j] = i for every nonzero j of row i (P_ML micro-benchmark, Section III-B);
// for a matrix with more rows than columns the index is clamped to the last column so
// that x stays in bounds.
__global__ void k_fill_row_index(int64_t n_rows, int64_t n_cols, const int32_t *rowptr,
                                 int32_t *out) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= n_rows) return;
  const int s = rowptr[i], e = rowptr[i + 1];
  const int32_t v = (int32_t)(i < n_cols ? i : n_cols - 1);
  for (int j = s + lane; j < e; j += 32) out[j] = v;
}

cudaError_t launch_fill_row_index(int64_t n_rows, int64_t n_cols, const int32_t *rowptr,
                                  int32_t *out, cudaStream_t s) {
  if (n_rows == 0) return cudaSuccess;
  k_fill_row_index<<<blocks_for(n_rows, kT / 32), kT, 0, s>>>(n_rows, n_cols, rowptr, out);
  return cudaGetLastError();
}

__global__ void k_fill_const(void *p, int t, int64_t n, double v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (t == SPMV_F64) static_cast<double *>(p)[i] = v;
    else static_cast<float *>(p)[i] = (float)v;
  }
}

cudaError_t launch_fill_const(void *p, spmv_dtype t, int64_t n, double v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  unsigned g = blocks_for(n);
  if (g > 65536u) g = 65536u;
  k_fill_const<<<g, kT, 0, s>>>(p, (int)t, n, v);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- features ---------
// Table I per-row quantities, one warp per row; integer sums are exact in any order, so
// the per-block partials and their final reduction give the same bits as a serial sum.
typedef unsigned __int128 u128;

struct FeatAcc {
  u128 s_nnz2, s_bw, s_bw2, s_sc2;
  unsigned long long s_nnz, s_sc, s_cl, s_miss, s_grp;
  long long nnz_min, nnz_max, bw_min, bw_max;
};

__device__ __forceinline__ void feat_init(FeatAcc &f) {
  f.s_nnz2 = f.s_bw = f.s_bw2 = f.s_sc2 = 0;
  f.s_nnz = f.s_sc = f.s_cl = f.s_miss = f.s_grp = 0;
  f.nnz_min = LLONG_MAX;
  f.nnz_max = 0;
  f.bw_min = LLONG_MAX;
  f.bw_max = 0;
}

__device__ __forceinline__ void feat_merge(FeatAcc &a, const FeatAcc &b) {
  a.s_nnz2 += b.s_nnz2; a.s_bw += b.s_bw; a.s_bw2 += b.s_bw2; a.s_sc2 += b.s_sc2;
  a.s_nnz += b.s_nnz; a.s_sc += b.s_sc; a.s_cl += b.s_cl; a.s_miss += b.s_miss;
  a.s_grp += b.s_grp;
  a.nnz_min = min(a.nnz_min, b.nnz_min); a.nnz_max = max(a.nnz_max, b.nnz_max);
  a.bw_min = min(a.bw_min, b.bw_min); a.bw_max = max(a.bw_max, b.bw_max);
}

__device__ __forceinline__ void feat_store(FeatSums *o, const FeatAcc &f) {
  o->s_nnz = f.s_nnz; o->s_sc = f.s_sc; o->s_cl = f.s_cl; o->s_miss = f.s_miss;
  o->s_grp = f.s_grp;
  o->s_nnz2_lo = (unsigned long long)f.s_nnz2; o->s_nnz2_hi = (unsigned long long)(f.s_nnz2 >> 64);
  o->s_bw_lo = (unsigned long long)f.s_bw; o->s_bw_hi = (unsigned long long)(f.s_bw >> 64);
  o->s_bw2_lo = (unsigned long long)f.s_bw2; o->s_bw2_hi = (unsigned long long)(f.s_bw2 >> 64);
  o->s_sc2_lo = (unsigned long long)f.s_sc2; o->s_sc2_hi = (unsigned long long)(f.s_sc2 >> 64);
  o->nnz_min = f.nnz_min; o->nnz_max = f.nnz_max; o->bw_min = f.bw_min; o->bw_max = f.bw_max;
}

__device__ __forceinline__ FeatAcc feat_load(const FeatSums *o) {
  FeatAcc f;
  f.s_nnz = o->s_nnz; f.s_sc = o->s_sc; f.s_cl = o->s_cl; f.s_miss = o->s_miss; f.s_grp = o->s_grp;
  f.s_nnz2 = ((u128)o->s_nnz2_hi << 64) | o->s_nnz2_lo;
  f.s_bw = ((u128)o->s_bw_hi << 64) | o->s_bw_lo;
  f.s_bw2 = ((u128)o->s_bw2_hi << 64) | o->s_bw2_lo;
  f.s_sc2 = ((u128)o->s_sc2_hi << 64) | o->s_sc2_lo;
  f.nnz_min = o->nnz_min; f.nnz_max = o->nnz_max; f.bw_min = o->bw_min; f.bw_max = o->bw_max;
  return f;
}

// round(num * 2^24 / den), halves up, exact (num, den < 2^31)
__device__ __forceinline__ unsigned long long q24(unsigned long long num, unsigned long long den) {
  return ((num << 25) + den) / (2ull * den);
}

constexpr int kFeatThreads = 256;
constexpr int kFeatWarps = kFeatThreads / 32;

__global__ void __launch_bounds__(kFeatThreads)
k_features(int64_t n_rows, const int32_t *rowptr, const int32_t *colind, int32_t line_elems,
           FeatSums *partials) {
  __shared__ FeatSums sh[kFeatWarps];
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  FeatAcc acc;
  feat_init(acc);
  for (int64_t i = (int64_t)blockIdx.x * kFeatWarps + warp; i < n_rows;
       i += (int64_t)gridDim.x * kFeatWarps) {
    const int s = rowptr[i], e = rowptr[i + 1];
    const long long k = e - s;
    unsigned grp = 0, miss = 0;
    for (int j = s + lane; j < e; j += 32) {
      if (j == s) {
        grp += 1;
        miss += 1;
      } else {
        const long long d = (long long)colind[j] - (long long)colind[j - 1];
        grp += (d != 1);
        miss += (d > line_elems);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      grp += __shfl_xor_sync(0xffffffffu, grp, off);
      miss += __shfl_xor_sync(0xffffffffu, miss, off);
    }
    if (lane == 0) {
      const long long bw = k > 0 ? (long long)colind[e - 1] - (long long)colind[s] + 1 : 0;
      const unsigned long long qs = k > 0 ? q24((unsigned long long)k, (unsigned long long)bw) : 0;
      const unsigned long long qc = k > 0 ? q24(grp, (unsigned long long)k) : 0;
      acc.s_nnz += (unsigned long long)k;
      acc.s_nnz2 += (u128)k * (u128)k;
      acc.s_bw += (u128)bw;
      acc.s_bw2 += (u128)bw * (u128)bw;
      acc.s_sc += qs;
      acc.s_sc2 += (u128)qs * (u128)qs;
      acc.s_cl += qc;
      acc.s_miss += miss;
      acc.s_grp += grp;
      acc.nnz_min = min(acc.nnz_min, k);
      acc.nnz_max = max(acc.nnz_max, k);
      acc.bw_min = min(acc.bw_min, bw);
      acc.bw_max = max(acc.bw_max, bw);
    }
  }
  if (lane == 0) feat_store(&sh[warp], acc);
  __syncthreads();
  if (threadIdx.x == 0) {
    FeatAcc tot = feat_load(&sh[0]);
    for (int w = 1; w < kFeatWarps; ++w) feat_merge(tot, feat_load(&sh[w]));
    feat_store(&partials[blockIdx.x], tot);
  }
}

__global__ void k_features_final(const FeatSums *partials, int n, FeatSums *out) {
  if (threadIdx.x != 0) return;
  FeatAcc tot = feat_load(&partials[0]);
  for (int b = 1; b < n; ++b) feat_merge(tot, feat_load(&partials[b]));
  feat_store(out, tot);
}

int feature_blocks(int64_t n_rows) {
  int64_t b = (n_rows + kFeatWarps * 16 - 1) / (kFeatWarps * 16);
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return (int)b;
}

cudaError_t launch_features(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                            int32_t line_elems, FeatSums *partials, int n_blocks,
                            FeatSums *out, cudaStream_t s) {
  k_features<<<n_blocks, kFeatThreads, 0, s>>>(n_rows, rowptr, colind, line_elems, partials);
  k_features_final<<<1, 32, 0, s>>>(partials, n_blocks, out);
  return cudaGetLastError();
}

__global__ void k_row_len_max(int64_t n_rows, const int32_t *rowptr, int32_t *out) {
  int m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rows;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, rowptr[i + 1] - rowptr[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

cudaError_t launch_row_len_max(int64_t n_rows, const int32_t *rowptr, int32_t *out,
                               cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int32_t), s);
  if (e != cudaSuccess || n_rows == 0) return e;
  unsigned g = blocks_for(n_rows);
  if (g > 4096u) g = 4096u;
  k_row_len_max<<<g, kT, 0, s>>>(n_rows, rowptr, out);
  return cudaGetLastError();
}

// Staged size of a thread-per-row tile: elements from the tile's first nonzero rounded
// down to a multiple of 8 to its last nonzero, rounded up to a multiple of 8.
__global__ void k_tile_max(int64_t n_rows, const int32_t *rowptr, int tile_rows, int align,
                           int32_t *out) {
  int m = 0;
  const int64_t n_tiles = (n_rows + tile_rows - 1) / tile_rows;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r0 = t * tile_rows;
    const int64_t r1 = r0 + tile_rows < n_rows ? r0 + tile_rows : n_rows;
    const int a0 = rowptr[r0] & ~(align - 1);
    m = max(m, ((rowptr[r1] - a0) + align - 1) & ~(align - 1));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

cudaError_t launch_tile_max(int64_t n_rows, const int32_t *rowptr, int tile_rows, int align,
                            int32_t *out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int32_t), s);
  if (e != cudaSuccess || n_rows == 0) return e;
  const int64_t n_tiles = (n_rows + tile_rows - 1) / tile_rows;
  unsigned g = blocks_for(n_tiles);
  if (g > 4096u) g = 4096u;
  k_tile_max<<<g, kT, 0, s>>>(n_rows, rowptr, tile_rows, align, out);
  return cudaGetLastError();
}

// Largest column index used by rows [bounds[c], bounds[c+1]) for each of n_chunks chunks
// (-1 for a chunk without nonzeros); out must hold n_chunks ints set to -1.
__global__ void k_chunk_colmax(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                               const int64_t *bounds, int n_chunks, int32_t *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int s = rowptr[i], e = rowptr[i + 1];
    if (e <= s) continue;
    int c = 0;
    while (c + 1 < n_chunks && i >= bounds[c + 1]) ++c;
    atomicMax(out + c, colind[e - 1]);
  }
}

cudaError_t launch_chunk_colmax(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                                const int64_t *bounds, int n_chunks, int32_t *out,
                                cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0xFF, sizeof(int32_t) * (size_t)n_chunks, s);
  if (e != cudaSuccess || n_rows == 0) return e;
  unsigned g = blocks_for(n_rows);
  if (g > 4096u) g = 4096u;
  k_chunk_colmax<<<g, kT, 0, s>>>(n_rows, rowptr, colind, bounds, n_chunks, out);
  return cudaGetLastError();
}

// Failure-path self test: waits (bounded) on an mbarrier phase that nothing completes -- the
// transaction count is armed but no copy is issued -- and records the expiry in err exactly
// as the SpMV kernels do. No asynchronous copy is in flight when the CTA exits.
__global__ void k_selftest_wait(uint64_t limit_ns, int32_t *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, 16);
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
  if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicExch(err, 1);
}

cudaError_t launch_selftest_wait(uint64_t limit_ns, int32_t *err, cudaStream_t s) {
  k_selftest_wait<<<1, 32, 0, s>>>(limit_ns, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- bandwidth probe -----
// Reads `bytes` (a multiple of 16) reps times with 128-bit streaming loads; the XOR of
// everything read is stored only if it equals an impossible value, so the loads stay.
__global__ void k_read_probe(const uint4 *buf, int64_t n16, int reps, unsigned long long *sink) {
  uint32_t acc = 0;
  for (int r = 0; r < reps; ++r) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
         i += (int64_t)gridDim.x * blockDim.x) {
      const uint4 v = ld_nc_u4(buf + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  if (acc == 0x9E3779B9u) *sink = acc;
}

cudaError_t launch_read_probe(const void *buf, int64_t bytes, int reps,
                              unsigned long long *sink, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t n16 = bytes / 16;
  int64_t g = (int64_t)sms * 8;
  const int64_t need = (n16 + kT - 1) / kT;
  if (g > need) g = need;
  if (g < 1) g = 1;
  k_read_probe<<<(unsigned)g, kT, 0, s>>>(static_cast<const uint4 *>(buf), n16, reps, sink);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ gather probe -----
// `count` gathers of one element each from x[0, n_x) at pseudo-random positions: gather j
// reads x[(h(j) >> 32) * n_x >> 32], h the splitmix64 finalizer (Steele, Lea and Flood) of
// seed + j, so no index array is streamed and the positions are uniform over x. Each thread
// keeps 8 gathers in flight before summing them; the sum is stored only if it equals an
// impossible value, so the loads stay. The gather rate is the ceiling of an SpMV whose x
// accesses are uniform random over an x of the same size.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void k_gather_probe(const T *__restrict__ x, int64_t n_x, int64_t count,
                               uint64_t seed, unsigned long long *sink) {
  T acc = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * 8;
  for (int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8; j0 < count;
       j0 += stride) {
    T v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint64_t h = mix64(seed + (uint64_t)(j0 + q));
      const int64_t i = (int64_t)(((h >> 32) * (uint64_t)n_x) >> 32);
      v[q] = j0 + q < count ? __ldg(x + i) : (T)0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) acc += v[q];
  }
  if (acc == (T)-1234.5) *sink = 1;
}

cudaError_t launch_gather_probe(const void *x, int32_t elem_bytes, int64_t n_x, int64_t count,
                                unsigned long long *sink, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t g = (int64_t)sms * 8;
  const int64_t need = (count / 8 + kT - 1) / kT;
  if (g > need) g = need;
  if (g < 1) g = 1;
  if (elem_bytes == 8)
    k_gather_probe<double><<<(unsigned)g, kT, 0, s>>>(static_cast<const double *>(x), n_x, count,
                                                      0x9E3779B97F4A7C15ull, sink);
  else
    k_gather_probe<float><<<(unsigned)g, kT, 0, s>>>(static_cast<const float *>(x), n_x, count,
                                                     0x9E3779B97F4A7C15ull, sink);
  return cudaGetLastError();
}

// FMA throughput probe: every thread runs C independent chains a <- fma(a, b, c) from
// registers (b and c are kernel arguments, so nothing folds); the chains' sum is stored
// only if it equals an impossible value. Blocks of 32 threads (64 above 32 warps per SM)
// so that warps_per_sm warps land on each SM.
template <typename T, int C>
__global__ void k_fma_probe(T b, T c, int32_t iters, unsigned long long *sink) {
  T a[C];
  const T t = (T)(blockIdx.x * blockDim.x + threadIdx.x) * (T)1e-9;
#pragma unroll
  for (int i = 0; i < C; ++i) a[i] = t + (T)i;
  for (int32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < C; ++i) a[i] = fma(a[i], b, c);
  }
  T sum = 0;
#pragma unroll
  for (int i = 0; i < C; ++i) sum += a[i];
  if (sum == (T)-1234.5) *sink = 1;
}

template <typename T>
cudaError_t launch_fma_probe_t(int32_t chains, int64_t blocks, int threads, int32_t fmas,
                               unsigned long long *sink, cudaStream_t s) {
  const T b = (T)0.999999, c = (T)1e-7;
  switch (chains) {
    case 1: k_fma_probe<T, 1><<<(unsigned)blocks, threads, 0, s>>>(b, c, fmas, sink); break;
    case 2: k_fma_probe<T, 2><<<(unsigned)blocks, threads, 0, s>>>(b, c, fmas / 2, sink); break;
    case 4: k_fma_probe<T, 4><<<(unsigned)blocks, threads, 0, s>>>(b, c, fmas / 4, sink); break;
    default: k_fma_probe<T, 8><<<(unsigned)blocks, threads, 0, s>>>(b, c, fmas / 8, sink); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_fma_probe(int32_t elem_bytes, int32_t chains, int32_t warps_per_sm,
                             int32_t fmas_per_thread, int64_t *n_threads,
                             unsigned long long *sink, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = warps_per_sm <= 32 ? 32 : 64;
  const int64_t blocks = (int64_t)sms * warps_per_sm * 32 / threads;
  *n_threads = blocks * threads;
  return elem_bytes == 8 ? launch_fma_probe_t<double>(chains, blocks, threads, fmas_per_thread, sink, s)
                         : launch_fma_probe_t<float>(chains, blocks, threads, fmas_per_thread, sink, s);
}

// ------------------------------------------------------------ row decomposition ------
// Per row: med = 1 if l_med <= length < chunk, lng = 1 if length >= chunk, nch = the long
// row's chunk count. Exclusive scans of the three give each row's place in the lists.
__global__ void k_bin_counts(int64_t n_rows, const int32_t *rowptr, int32_t l_med,
                             int32_t chunk, int64_t *med, int64_t *lng, int64_t *nch) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const int len = rowptr[r + 1] - rowptr[r];
  const bool is_long = len >= chunk;
  med[r] = (len >= l_med && !is_long) ? 1 : 0;
  lng[r] = is_long ? 1 : 0;
  nch[r] = is_long ? (len + chunk - 1) / chunk : 0;
}

// A chunk is (row, first nonzero z, end nonzero, the column its delta decode starts from:
// colind[z - 1] inside the row, colind[z] for the row's first chunk, whose first delta is 0).
__global__ void k_bin_fill(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                           int32_t l_med, int32_t chunk, const int64_t *med_off,
                           const int64_t *lng_off, const int64_t *nch_off, int32_t *bin_rows,
                           int32_t *long_rows, int32_t *long_first, int4 *chunks) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const int s = rowptr[r], e = rowptr[r + 1], len = e - s;
  if (len >= chunk) {
    const int64_t k = lng_off[r];
    const int64_t c0 = nch_off[r];
    long_rows[k] = (int32_t)r;
    long_first[k] = (int32_t)c0;
    int64_t c = c0;
    for (int z = s; z < e; z += chunk, ++c)
      chunks[c] = make_int4((int)r, z, min(z + chunk, e), colind[z > s ? z - 1 : z]);
  } else if (len >= l_med) {
    bin_rows[med_off[r]] = (int32_t)r;
  }
}

cudaError_t launch_bin_counts(int64_t n_rows, const int32_t *rowptr, int32_t l_med,
                              int32_t chunk, int64_t *med, int64_t *lng, int64_t *nch,
                              cudaStream_t s) {
  if (n_rows <= 0) return cudaSuccess;
  k_bin_counts<<<blocks_for(n_rows), kT, 0, s>>>(n_rows, rowptr, l_med, chunk, med, lng, nch);
  return cudaGetLastError();
}

cudaError_t launch_bin_fill(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                            int32_t l_med, int32_t chunk, const int64_t *med_off,
                            const int64_t *lng_off, const int64_t *nch_off, int32_t *bin_rows,
                            int32_t *long_rows, int32_t *long_first, int4 *chunks,
                            cudaStream_t s) {
  if (n_rows <= 0) return cudaSuccess;
  k_bin_fill<<<blocks_for(n_rows), kT, 0, s>>>(n_rows, rowptr, colind, l_med, chunk, med_off,
                                                lng_off, nch_off, bin_rows, long_rows,
                                                long_first, chunks);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- sliced rows ----
__global__ void k_sell_widths(int64_t n_rows, const int32_t *rowptr, int64_t *w32) {
  const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= (n_rows + 31) / 32) return;
  const int64_t r1 = min(32 * sl + 32, n_rows);
  int w = 0;
  for (int64_t r = 32 * sl; r < r1; ++r) w = max(w, rowptr[r + 1] - rowptr[r]);
  w32[sl] = 32 * (int64_t)w;
}

// Thread per row: element k of row r goes to soff[r / 32] + 32 k + r % 32.
template <typename VT, typename IT>
__global__ void k_sell_fill(int64_t n_rows, const int32_t *rowptr, const VT *val, const IT *idx,
                            const int64_t *soff, VT *sval, IT *sidx) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const int64_t p0 = soff[r >> 5] + (r & 31);
  const int s = rowptr[r], len = rowptr[r + 1] - s;
  for (int k = 0; k < len; ++k) {
    sval[p0 + 32 * (int64_t)k] = val[s + k];
    sidx[p0 + 32 * (int64_t)k] = idx[s + k];
  }
}

cudaError_t launch_sell_widths(int64_t n_rows, const int32_t *rowptr, int64_t *w32,
                               cudaStream_t s) {
  if (n_rows <= 0) return cudaSuccess;
  k_sell_widths<<<blocks_for((n_rows + 31) / 32), kT, 0, s>>>(n_rows, rowptr, w32);
  return cudaGetLastError();
}

template <typename VT>
static cudaError_t sell_fill_v(int64_t n, const int32_t *rowptr, const void *val, const void *idx,
                               int idx_bytes, const int64_t *soff, void *sv, void *si,
                               cudaStream_t s) {
  const unsigned g = blocks_for(n);
  const VT *v = static_cast<const VT *>(val);
  VT *o = static_cast<VT *>(sv);
  switch (idx_bytes) {
    case 4:
      k_sell_fill<VT, int32_t><<<g, kT, 0, s>>>(n, rowptr, v, static_cast<const int32_t *>(idx),
                                                soff, o, static_cast<int32_t *>(si));
      break;
    case 2:
      k_sell_fill<VT, uint16_t><<<g, kT, 0, s>>>(n, rowptr, v, static_cast<const uint16_t *>(idx),
                                                 soff, o, static_cast<uint16_t *>(si));
      break;
    case 1:
      k_sell_fill<VT, uint8_t><<<g, kT, 0, s>>>(n, rowptr, v, static_cast<const uint8_t *>(idx),
                                                soff, o, static_cast<uint8_t *>(si));
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sell_fill(int64_t n_rows, const int32_t *rowptr, const void *val,
                             int val_bytes, const void *idx, int idx_bytes,
                             const int64_t *soff, void *sell_val, void *sell_idx,
                             cudaStream_t s) {
  if (n_rows <= 0) return cudaSuccess;
  switch (val_bytes) {
    case 8: return sell_fill_v<uint64_t>(n_rows, rowptr, val, idx, idx_bytes, soff, sell_val, sell_idx, s);
    case 4: return sell_fill_v<uint32_t>(n_rows, rowptr, val, idx, idx_bytes, soff, sell_val, sell_idx, s);
    case 2: return sell_fill_v<uint16_t>(n_rows, rowptr, val, idx, idx_bytes, soff, sell_val, sell_idx, s);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------------ column panels ----
// Thread per row: the row's columns are sorted, so its part in panel b starts at the first
// column >= b * width (binary search between the previous boundary and the row's end).
__global__ void k_panel_counts(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                               int32_t n_panels, int32_t width, int64_t *cnt) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const int e = rowptr[r + 1];
  int prev = rowptr[r];
  for (int b = 1; b < n_panels; ++b) {
    const int64_t target = (int64_t)b * width;
    int lo = prev, hi = e;
    while (lo < hi) {
      const int mid = lo + ((hi - lo) >> 1);
      if ((int64_t)colind[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    cnt[(int64_t)(b - 1) * (n_rows + 1) + r] = lo - prev;
    prev = lo;
  }
  cnt[(int64_t)(n_panels - 1) * (n_rows + 1) + r] = e - prev;
}

// Warp per row (warp n_rows writes the panels' end pointers): the row's panel-p part is
// copied to panel p's base (the totals of the panels before it) plus the row's scanned
// offset in panel p.
template <typename T>
__global__ void k_panel_fill(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                             const T *val, int32_t n_panels, const int64_t *off,
                             int32_t *pnl_rowptr, int32_t *pnl_col, T *pnl_val) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r > n_rows) return;
  const int64_t stride = n_rows + 1;
  int64_t base = 0;
  int src = r < n_rows ? rowptr[r] : 0;
  for (int p = 0; p < n_panels; ++p) {
    const int64_t *o = off + (int64_t)p * stride;
    const int64_t dst = base + o[r];
    if (lane == 0) pnl_rowptr[(int64_t)p * stride + r] = (int32_t)dst;
    if (r < n_rows) {
      const int c = (int)(o[r + 1] - o[r]);
      for (int k = lane; k < c; k += 32) {
        pnl_col[dst + k] = colind[src + k];
        pnl_val[dst + k] = val[src + k];
      }
      src += c;
    }
    base += o[n_rows];
  }
}

cudaError_t launch_panel_counts(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                                int32_t n_panels, int32_t width, int64_t *cnt, cudaStream_t s) {
  if (n_rows <= 0) return cudaSuccess;
  k_panel_counts<<<blocks_for(n_rows), kT, 0, s>>>(n_rows, rowptr, colind, n_panels, width,
                                                     cnt);
  return cudaGetLastError();
}

cudaError_t launch_panel_fill(int64_t n_rows, const int32_t *rowptr, const int32_t *colind,
                              const void *val, int val_bytes, int32_t n_panels,
                              const int64_t *off, int32_t *pnl_rowptr, int32_t *pnl_col,
                              void *pnl_val, cudaStream_t s) {
  if (n_rows < 0) return cudaErrorInvalidValue;
  const unsigned g = blocks_for((n_rows + 1) * 32);
  switch (val_bytes) {
    case 8:
      k_panel_fill<uint64_t><<<g, kT, 0, s>>>(n_rows, rowptr, colind,
                                              static_cast<const uint64_t *>(val), n_panels, off,
                                              pnl_rowptr, pnl_col, static_cast<uint64_t *>(pnl_val));
      break;
    case 4:
      k_panel_fill<uint32_t><<<g, kT, 0, s>>>(n_rows, rowptr, colind,
                                              static_cast<const uint32_t *>(val), n_panels, off,
                                              pnl_rowptr, pnl_col, static_cast<uint32_t *>(pnl_val));
      break;
    case 2:
      k_panel_fill<uint16_t><<<g, kT, 0, s>>>(n_rows, rowptr, colind,
                                              static_cast<const uint16_t *>(val), n_panels, off,
                                              pnl_rowptr, pnl_col, static_cast<uint16_t *>(pnl_val));
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace spmv

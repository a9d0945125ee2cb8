// Bottleneck classification and tuning: device properties and the bandwidth probe, the
// performance bounds of Section III-B, the profile route (Section III-C, Fig. 3), the
// feature route (Section III-D) and the sub-warp width / tile geometry sweep, with the
// spmv_tune entry point that maps the class set to a pool variant.
#include "handle.h"

using namespace spmv;
using namespace spmv::rt;

namespace {

std::mutex g_dev_mu;
DeviceInfo g_dev[64];

}  // namespace

namespace spmv {
namespace rt {

DeviceInfo &device_info(int dev) {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DeviceInfo &d = g_dev[dev & 63];
  if (d.sms == 0) {
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    d.l2_bytes = l2;
  }
  return d;
}

}  // namespace rt
}  // namespace spmv

namespace {

// Average milliseconds per launch of fn over reps launches (after 2 warm-up launches).
template <typename F> float time_launches(F fn, int reps, cudaStream_t s) {
  for (int i = 0; i < 2; ++i) CK(fn());
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  for (int i = 0; i < reps; ++i) CK(fn());
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / (float)reps;
}

// ------------------------------------------------------------------ bandwidth --------
void probe_bandwidth(int dev, double *hbm, double *l2) {
  DeviceInfo &d = device_info(dev);
  {
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (d.bw_done) {
      *hbm = d.hbm_gbs;
      *l2 = d.l2_gbs;
      return;
    }
  }
  cudaStream_t s;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  DevBuf big, small, sink;
  const int64_t big_bytes = (int64_t)2 << 30;
  int64_t small_bytes = d.l2_bytes / 4;
  if (small_bytes < (1 << 20)) small_bytes = 1 << 20;
  small_bytes &= ~(int64_t)15;
  big.alloc((size_t)big_bytes, 1, s, true);
  small.alloc((size_t)small_bytes, 1, s, true);
  sink.alloc(8, 8, s, true);
  auto fb = [&]() { return launch_read_probe(big.p, big_bytes, 1, sink.as<unsigned long long>(), s); };
  const int l2_reps = 64;
  auto fs = [&]() {
    return launch_read_probe(small.p, small_bytes, l2_reps, sink.as<unsigned long long>(), s);
  };
  float tb = 1e30f, ts = 1e30f;
  for (int r = 0; r < 3; ++r) {
    tb = std::min(tb, time_launches(fb, 3, s));
    ts = std::min(ts, time_launches(fs, 3, s));
  }
  cudaStreamSynchronize(s);
  big.release();
  small.release();
  sink.release();
  cudaStreamDestroy(s);
  std::lock_guard<std::mutex> lk(g_dev_mu);
  d.hbm_gbs = (double)big_bytes / (tb * 1e-3) / 1e9;
  d.l2_gbs = (double)small_bytes * l2_reps / (ts * 1e-3) / 1e9;
  d.bw_done = true;
  *hbm = d.hbm_gbs;
  *l2 = d.l2_gbs;
}

// --------------------------------------------------------------- bounds & rules ------
void bounds(int64_t n_rows, int64_t n_cols, int64_t nnz, int idx_b, int val_b, int vec_b,
            double b_max, double *out) {
  const double s_format = 4.0 * (double)(n_rows + 1) + (double)(idx_b + val_b) * (double)nnz;
  const double s_xy = (double)vec_b * (double)n_cols + (double)vec_b * (double)n_rows;
  const double s_values = (double)val_b * (double)nnz;
  const double flops = 2.0 * (double)nnz;
  out[0] = flops / ((s_format + s_xy) / b_max);
  out[1] = flops / ((s_values + s_xy) / b_max);
  out[2] = s_format + s_xy;
}

uint32_t classify(const double *p, double t_imb, double t_ml, double t_mb) {
  const double p_csr = p[0], p_mb = p[1], p_ml = p[2], p_imb = p[3], p_cmp = p[4], p_peak = p[5];
  uint32_t c = 0;
  if (p_imb / p_csr > t_imb) c |= SPMV_CLASS_IMB;
  if (p_ml / p_csr > t_ml) c |= SPMV_CLASS_ML;
  if (p_csr / p_mb >= t_mb && p_mb < p_cmp && p_cmp < p_peak) c |= SPMV_CLASS_MB;
  if (p_mb > p_cmp || p_cmp > p_peak) c |= SPMV_CLASS_CMP;
  return c;
}

// Second profiling pass (GB300 reading of Section III-C): when the baseline is compute
// bound (CMP), the compute bottleneck hides the memory ones. After the CMP optimization
// (one FMA per nonzero) the profile is repeated with that kernel as the baseline:
// p2 = {P_CSR', P_ML'}; ML if P_ML' / P_CSR' > t_ml, MB if P_CSR' / P_MB >= t_mb.
uint32_t classify2(const double *p, const double *p2, double t_imb, double t_ml, double t_mb) {
  uint32_t c = classify(p, t_imb, t_ml, t_mb);
  if (p2 && (c & SPMV_CLASS_CMP) && p2[0] > 0.0) {
    if (p2[1] / p2[0] > t_ml) c |= SPMV_CLASS_ML;
    if (p2[0] / p[1] >= t_mb) c |= SPMV_CLASS_MB;
  }
  return c;
}

spmv_variant variant_for_classes(uint32_t cls, double nnz_avg, double nnz_max, double long_ratio) {
  spmv_variant v{};
  if ((cls & SPMV_CLASS_IMB) && nnz_max > long_ratio * nnz_avg) v.partition = 1;
  if (cls & SPMV_CLASS_MB) v.index = 1;   // merge-path tiles keep int32 columns
  if (cls & SPMV_CLASS_ML) v.xpath = 1;
  if (cls & (SPMV_CLASS_MB | SPMV_CLASS_CMP)) v.vec = 1;
  v.vs = 0;
  return v;
}

// Feature route (Section III-D) with fixed rules in place of a trained tree:
//   IMB  highly uneven rows: nnz_max > long_ratio * nnz_avg;
//   ML   most elements start a new cache line (misses_avg >= nnz_avg / 2) and x does not
//        fit in half of L2;
//   CMP  the working set fits in L2 (size = 1) or rows are very short (nnz_avg < 4);
//   MB   none of the above and the working set exceeds L2.
uint32_t feature_rules(const double *f, int64_t n_cols, int vec_bytes, int64_t l2_bytes,
                       double long_ratio) {
  const double size = f[0], nnz_max = f[3], nnz_avg = f[4], misses_avg = f[13];
  uint32_t c = 0;
  if (nnz_avg > 0.0 && nnz_max > long_ratio * nnz_avg) c |= SPMV_CLASS_IMB;
  if (misses_avg >= 0.5 * nnz_avg && (double)vec_bytes * (double)n_cols > 0.5 * (double)l2_bytes)
    c |= SPMV_CLASS_ML;
  if (size != 0.0 || nnz_avg < 4.0) c |= SPMV_CLASS_CMP;
  if (c == 0 && size == 0.0) c |= SPMV_CLASS_MB;
  return c;
}

// ------------------------------------------------------------------ features ---------
double finalize_sd(u128 s1, u128 s2, int64_t n, double scale) {
  const u128 nn = (u128)(uint64_t)n;
  const u128 num = nn * s2 - s1 * s1;
  const double var = (double)num / ((double)n * (double)n);
  return std::sqrt(var) * scale;
}

void compute_features(spmv_matrix *h, int line_bytes, double *out, uint64_t *isum,
                      cudaStream_t s) {
  const int line_elems = std::max(1, line_bytes / (int)dtype_bytes(h->vec));
  const int nb = feature_blocks(h->n_rows);
  if (!h->feat_part.p) {
    h->feat_part.alloc(sizeof(FeatSums) * (size_t)nb, 8, s);
    h->feat_fin.alloc(sizeof(FeatSums), 8, s);
  }
  CK(launch_features(h->n_rows, h->rowptr.as<int32_t>(), h->colind.as<int32_t>(), line_elems,
                     h->feat_part.as<FeatSums>(), nb, h->feat_fin.as<FeatSums>(), s));
  FeatSums fs;
  CK(cudaMemcpyAsync(&fs, h->feat_fin.p, sizeof fs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int64_t n = h->n_rows;
  const u128 s_nnz = fs.s_nnz, s_nnz2 = ((u128)fs.s_nnz2_hi << 64) | fs.s_nnz2_lo;
  const u128 s_bw = ((u128)fs.s_bw_hi << 64) | fs.s_bw_lo;
  const u128 s_bw2 = ((u128)fs.s_bw2_hi << 64) | fs.s_bw2_lo;
  const u128 s_sc = fs.s_sc, s_sc2 = ((u128)fs.s_sc2_hi << 64) | fs.s_sc2_lo;
  const u128 s_cl = fs.s_cl;
  const int64_t vb = (int64_t)dtype_bytes(h->vec);
  const int64_t ws = 4 * (h->n_rows + 1) +
                     (4 + (int64_t)dtype_bytes(h->storage)) * h->nnz + vb * (h->n_rows + h->n_cols);
  const DeviceInfo &d = device_info(h->device);
  const double N = (double)n;
  const double q = 1.0 / 16777216.0;
  long long nnz_min = fs.nnz_min, nnz_max = fs.nnz_max, bw_min = fs.bw_min, bw_max = fs.bw_max;
  if (n == 0) nnz_min = nnz_max = bw_min = bw_max = 0;
  out[0] = ws <= d.l2_bytes ? 1.0 : 0.0;
  out[1] = n > 0 && h->n_cols > 0 ? (double)h->nnz / ((double)n * (double)h->n_cols) : 0.0;
  out[2] = (double)nnz_min;
  out[3] = (double)nnz_max;
  out[4] = n ? (double)s_nnz / N : 0.0;
  out[5] = n ? finalize_sd(s_nnz, s_nnz2, n, 1.0) : 0.0;
  out[6] = (double)bw_min;
  out[7] = (double)bw_max;
  out[8] = n ? (double)s_bw / N : 0.0;
  out[9] = n ? finalize_sd(s_bw, s_bw2, n, 1.0) : 0.0;
  out[10] = n ? ((double)s_sc / N) * q : 0.0;
  out[11] = n ? finalize_sd(s_sc, s_sc2, n, q) : 0.0;
  out[12] = n ? ((double)s_cl / N) * q : 0.0;
  out[13] = n ? (double)fs.s_miss / N : 0.0;
  if (isum) {
    isum[0] = (uint64_t)s_nnz;
    isum[1] = (uint64_t)s_bw;
    isum[2] = (uint64_t)s_sc;
    isum[3] = (uint64_t)s_cl;
    isum[4] = fs.s_miss;
    isum[5] = fs.s_grp;
    isum[6] = (uint64_t)nnz_min;
    isum[7] = (uint64_t)nnz_max;
    isum[8] = (uint64_t)bw_min;
    isum[9] = (uint64_t)bw_max;
    isum[10] = fs.s_nnz2_lo;
    isum[11] = fs.s_bw2_lo;
  }
}

// ------------------------------------------------------------------ profiling --------
// The static-partition profiling setup shared by the profile route and its diagnostics:
// a resident grid of n_ctas CTAs over nnz-balanced contiguous row ranges (rows never
// split), the paper's baseline partitioning (Section IV-A) with one CTA per worker.
struct StaticSetup {
  DevBuf part, t0, t1, smid;
  ProfileArgs pa;
};

void static_setup(spmv_matrix *h, StaticSetup &st, const void *x, void *y, cudaStream_t s) {
  const KernelSet *ks = set_for(h);
  DeviceInfo &d = device_info(h->device);
  const int n_ctas = std::max(1, d.sms * ks->profile_blocks_per_sm);
  st.part.alloc(sizeof(int32_t) * (size_t)(n_ctas + 1), 4, s);
  CK(launch_static_partition(h->n_rows, h->nnz, h->rowptr.as<int32_t>(), n_ctas,
                             st.part.as<int32_t>(), s));
  st.t0.alloc(8 * (size_t)n_ctas, 8, s, true);
  st.t1.alloc(8 * (size_t)n_ctas, 8, s, true);
  st.smid.alloc(4 * (size_t)n_ctas, 4, s, true);
  ProfileArgs &pa = st.pa;
  pa.n_rows = h->n_rows;
  pa.n_cols = h->n_cols;
  pa.part = st.part.as<int32_t>();
  pa.n_ctas = n_ctas;
  pa.rowptr = h->rowptr.as<int32_t>();
  pa.colind = h->colind.as<int32_t>();
  pa.val = h->val_ptr();
  pa.x = x;
  pa.y = y;
  pa.t_start = st.t0.as<unsigned long long>();
  pa.t_end = st.t1.as<unsigned long long>();
  pa.smid = st.smid.as<int32_t>();
  pa.vs = heuristic_vs(h->nnz_avg(), 1);
  pa.cmp_mode = 0;
}

// Per-CTA elapsed times (ms) of the last launch; CTAs with an empty row range get -1.
void read_cta_times(const StaticSetup &st, std::vector<double> &el, std::vector<int32_t> &sm,
                    double *span_ms, cudaStream_t s) {
  const int n = st.pa.n_ctas;
  std::vector<unsigned long long> ts((size_t)n), te((size_t)n);
  std::vector<int32_t> hp((size_t)n + 1);
  sm.assign((size_t)n, 0);
  CK(cudaMemcpyAsync(ts.data(), st.t0.p, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(te.data(), st.t1.p, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(sm.data(), st.smid.p, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hp.data(), st.part.p, 4 * ((size_t)n + 1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  el.assign((size_t)n, -1.0);
  unsigned long long tmin = ~0ull, tmax = 0;
  for (int c = 0; c < n; ++c) {
    if (hp[(size_t)c + 1] <= hp[(size_t)c]) continue;   // no rows: no work
    el[(size_t)c] = (double)(te[(size_t)c] - ts[(size_t)c]) * 1e-6;
    tmin = std::min(tmin, ts[(size_t)c]);
    tmax = std::max(tmax, te[(size_t)c]);
  }
  *span_ms = tmax >= tmin ? (double)(tmax - tmin) * 1e-6 : 0.0;
}

// Span (ms) of every SM that ran at least one CTA with rows: last end - first start.
std::vector<double> sm_spans(const StaticSetup &st, cudaStream_t s, double *global_span_ms) {
  const int n = st.pa.n_ctas;
  std::vector<unsigned long long> ts((size_t)n), te((size_t)n);
  std::vector<int32_t> hp((size_t)n + 1), sm((size_t)n);
  CK(cudaMemcpyAsync(ts.data(), st.t0.p, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(te.data(), st.t1.p, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(sm.data(), st.smid.p, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hp.data(), st.part.p, 4 * ((size_t)n + 1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int max_sm = 0;
  for (int c = 0; c < n; ++c) max_sm = std::max(max_sm, sm[(size_t)c]);
  std::vector<unsigned long long> lo((size_t)max_sm + 1, ~0ull), hi((size_t)max_sm + 1, 0);
  unsigned long long gmin = ~0ull, gmax = 0;
  for (int c = 0; c < n; ++c) {
    if (hp[(size_t)c + 1] <= hp[(size_t)c]) continue;
    const size_t k = (size_t)sm[(size_t)c];
    lo[k] = std::min(lo[k], ts[(size_t)c]);
    hi[k] = std::max(hi[k], te[(size_t)c]);
    gmin = std::min(gmin, ts[(size_t)c]);
    gmax = std::max(gmax, te[(size_t)c]);
  }
  std::vector<double> spans;
  for (size_t k = 0; k < lo.size(); ++k)
    if (hi[k] >= lo[k] && lo[k] != ~0ull) spans.push_back((double)(hi[k] - lo[k]) * 1e-6);
  *global_span_ms = gmax >= gmin && gmin != ~0ull ? (double)(gmax - gmin) * 1e-6 : 0.0;
  return spans;
}

void run_profile(spmv_matrix *h, int reps, spmv_profile_report &o, cudaStream_t s,
                 bool second_pass = false) {
  std::memset(&o, 0, sizeof o);
  const KernelSet *ks = set_for(h);
  DeviceInfo &d = device_info(h->device);
  double b_hbm = 0, b_l2 = 0;
  probe_bandwidth(h->device, &b_hbm, &b_l2);
  const size_t vb = dtype_bytes(h->vec);
  DevBuf x, y, colp;
  x.alloc(vb * (size_t)std::max<int64_t>(h->n_cols, 1), vb, s);
  y.alloc(vb * (size_t)std::max<int64_t>(h->n_rows, 1), vb, s);
  CK(launch_fill_const(x.p, h->vec, h->n_cols, 1.0, s));
  StaticSetup st;
  static_setup(h, st, x.p, y.p, s);
  colp.alloc(sizeof(int32_t) * (size_t)h->nnz, 4, s);
  CK(launch_fill_row_index(h->n_rows, h->n_cols, h->rowptr.as<int32_t>(), colp.as<int32_t>(), s));
  ProfileArgs pa = st.pa;
  const double flops = 2.0 * (double)h->nnz;
  // P_CSR, and the per-CTA times of the last timed launch (P_IMB)
  const float t_csr = time_launches([&]() { return ks->profile(pa, s); }, reps, s);
  // A worker of the paper's static partition is an SM: the CTAs resident on one SM share
  // its pipes, so their individual times reflect the warp scheduler's fairness rather than
  // the partition. Each SM's time is the span of its CTAs (first start to last end); the
  // median is taken over SMs.
  double t_span = 0.0;
  std::vector<double> work = sm_spans(st, s, &t_span);
  double t_median = t_csr;
  if (!work.empty()) {
    std::sort(work.begin(), work.end());
    t_median = work[(work.size() - 1) / 2];           // lower median
  } else {
    t_span = t_csr;
  }
  // the median worker time plus the launch cost that no worker sees
  const double t_imb = t_median + std::max(0.0, (double)t_csr - t_span);
  // P_ML: colind'[j] = row of j
  pa.colind = colp.as<int32_t>();
  const float t_ml = time_launches([&]() { return ks->profile(pa, s); }, reps, s);
  // P_CMP: x[i] only, no colind
  pa.colind = h->colind.as<int32_t>();
  pa.cmp_mode = 1;
  const float t_cmp = time_launches([&]() { return ks->profile(pa, s); }, reps, s);
  double bo[3];
  bounds(h->n_rows, h->n_cols, h->nnz, 4, (int)dtype_bytes(h->storage), (int)vb, 1.0, bo);
  const double ws = bo[2];
  o.b_max_gbs = ws <= (double)d.l2_bytes ? b_l2 : b_hbm;
  bounds(h->n_rows, h->n_cols, h->nnz, 4, (int)dtype_bytes(h->storage), (int)vb, o.b_max_gbs, bo);
  auto gf = [&](double ms) { return ms > 0 ? flops / (ms * 1e-3) / 1e9 : 0.0; };
  o.p[0] = gf(t_csr);
  o.p[1] = bo[0];
  o.p[2] = gf(t_ml);
  o.p[3] = gf(t_imb);
  o.p[4] = gf(t_cmp);
  o.p[5] = bo[1];
  o.b_hbm_gbs = b_hbm;
  o.b_l2_gbs = b_l2;
  o.t_csr_ms = t_csr;
  o.t_ml_ms = t_ml;
  o.t_cmp_ms = t_cmp;
  o.t_median_ms = t_median;
  o.t_span_ms = t_span;
  o.t_imb_ms = t_imb;
  o.n_ctas = st.pa.n_ctas;
  o.vs = st.pa.vs;
  if (second_pass && h->n_rows > 0) {
    // the CMP optimization as the new baseline: thread-per-row tiles, int32 columns
    spmv_variant v2{};
    v2.vec = 1;
    v2.vs = 1;
    compute_tile_cap(h, v2, s);
    const float t2 = time_launches([&]() { return launch_run(h, v2, x.p, y.p, s); }, reps, s);
    RunArgs a2 = run_args(h, x.p, y.p);
    a2.colind = colp.as<int32_t>();
    const KernelSet *k2 = set_for(h);
    const float t2ml = time_launches([&]() { return k2->spmv(v2, a2, s); }, reps, s);
    o.p2[0] = gf(t2);
    o.p2[1] = gf(t2ml);
  }
}

// Device bytes of a second copy of the matrix: panel-major (n_panels row-pointer sets) or
// sliced rows (`positions` slots).
size_t panel_bytes(const spmv_matrix *h, int n_panels) {
  const size_t vb = h->storage == SPMV_DF64 ? 8 : dtype_bytes(h->storage);
  return (4 + vb) * (size_t)h->nnz + 4 * (size_t)n_panels * (size_t)(h->n_rows + 1);
}

// An optional copy is tried only when the device has room for it and a quarter to spare.
bool optional_fits(size_t bytes, cudaStream_t s) {
  size_t free_b = 0, total_b = 0;
  CK(cudaStreamSynchronize(s));
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return bytes + bytes / 4 < free_b;
}

// Column panels compete when the matrix is ML (v.xpath = 1) and x is larger than half the
// L2: panel counts that cut x into slices of a half and a third of the L2, each with
// sub-warps of 1 lane up to the width that covers a row's average share of one panel (at
// most 8), scalar or 128-bit loads. The fastest replaces v when it beats `best` (the time of
// v); otherwise the panel copy is freed.
void sweep_panels(spmv_matrix *h, spmv_variant &v, float best, const void *x, void *y,
                  int reps, cudaStream_t s) {
  const DeviceInfo &d = device_info(h->device);
  const double xb = (double)dtype_bytes(h->vec) * (double)h->n_cols;
  if (v.xpath != 1 || d.l2_bytes <= 0 || xb <= 0.5 * (double)d.l2_bytes) return;
  spmv_variant best_v = v;
  bool found = false;
  int last_p = 0;
  // the panel copy doubles the matrix in device memory: without room for it, panels sit out
  if (!optional_fits(panel_bytes(h, 2), s)) return;
  for (int f = 2; f <= 3; ++f) {
    const int p = std::min(kMaxPanels,
                           std::max(2, (int)std::ceil(xb * f / (double)d.l2_bytes)));
    if (p == last_p) continue;
    last_p = p;
    const int w_max = pow2_ceil_clamped(h->nnz_avg() / p, 1, 8);
    for (int w = 1; w <= w_max; w *= 2) {
      for (int vec = 0; vec <= 1; ++vec) {
        spmv_variant t = v;
        t.xpath = p;
        t.vs = w;
        t.vec = vec;
        prepare_variant(h, t, s);
        const float ms = time_launches([&]() { return launch_run(h, t, x, y, s); }, reps, s);
        if (ms < best) {
          best = ms;
          best_v = t;
          found = true;
        }
      }
    }
  }
  if (found) {
    v = best_v;
    prepare_variant(h, v, s);
  } else {
    drop_panels(h);
  }
}

// Sub-warp width sweep by timing (Section III-E "parameter tuning"; not in the paper). When
// the thread-per-row kernel (width 1) wins, its geometry is swept too: 128 / 64 / 32 rows
// per tile, one tile per CTA or persistent CTAs with two tiles in flight.
// Called by spmv_tune for the routes that choose a variant (never for SPMV_TUNE_FIXED), so
// the sub-warp width and, for width 1, the tile geometry are always swept; then sliced rows
// (short rows, little padding) and, for ML matrices whose x exceeds half the L2, column
// panels (sweep_panels) compete with the winner.
void autotune_vs(spmv_matrix *h, spmv_variant &v, int reps, int32_t bin_med, int32_t bin_chunk,
                 cudaStream_t s) {
  if (h->n_rows == 0) return;
  const size_t vb = dtype_bytes(h->vec);
  DevBuf x, y;
  x.alloc(vb * (size_t)std::max<int64_t>(h->n_cols, 1), vb, s);
  y.alloc(vb * (size_t)std::max<int64_t>(h->n_rows, 1), vb, s);
  CK(launch_fill_const(x.p, h->vec, h->n_cols, 1.0, s));
  if (v.partition != 0) {
    // IMB's decomposition family: merge-path tiles, or the row decomposition with short
    // rows on one thread or sub-warps of 2, 4 or 8 lanes; the fastest is kept
    spmv_variant best_v = v;
    float best_t = 1e30f;
    const int cand[5][2] = {{1, 0}, {2, 1}, {2, 2}, {2, 4}, {2, 8}};
    for (const auto &c : cand) {
      spmv_variant t = v;
      t.partition = c[0];
      t.vs = c[1];
      t.bin_med = bin_med;
      t.bin_chunk = bin_chunk;
      prepare_variant(h, t, s);
      const float ms = time_launches([&]() { return launch_run(h, t, x.p, y.p, s); }, reps, s);
      if (ms < best_t) {
        best_t = ms;
        best_v = t;
      }
    }
    v = best_v;
    prepare_variant(h, v, s);
    return;
  }
  float best = 1e30f;
  int best_vs = v.vs;
  const int widths[6] = {1, 2, 4, 8, 16, 32};
  compute_tile_cap(h, v, s);
  for (int w : widths) {
    spmv_variant t = v;
    t.vs = w;
    const float ms = time_launches([&]() { return launch_run(h, t, x.p, y.p, s); }, reps, s);
    if (ms < best) {
      best = ms;
      best_vs = w;
    }
  }
  v.vs = best_vs;
  if (best_vs != 1) {
    v.tile_rows = 0;
    v.tile_pipe = 0;
  } else {
    int best_rows = h->tile_rows, best_pipe = h->tile_pipe, best_cap = h->tile_cap;
    const int max_pipe = h->acc == SPMV_DF64 ? 0 : 1;
    for (int pipe = 0; pipe <= max_pipe; ++pipe) {
      for (int rows = kTileRows; rows >= 32; rows /= 2) {
        set_tile_geometry(h, v, rows, pipe != 0, s);
        const float ms = time_launches([&]() { return launch_run(h, v, x.p, y.p, s); }, reps, s);
        if (ms < best) {
          best = ms;
          best_rows = rows;
          best_pipe = pipe;
          best_cap = h->tile_cap;
        }
      }
    }
    h->tile_rows = best_rows;
    h->tile_pipe = best_pipe;
    h->tile_cap = best_cap;
    v.tile_rows = best_rows;
    v.tile_pipe = best_pipe;
  }
  // Sliced rows (thread per row without a shared-memory stage) compete with the best row
  // variant when rows are short and the slices pad the matrix by at most an eighth; their
  // times vary more from run to run, so they replace the incumbent only when 5 % faster.
  const int64_t sell_pos = h->nnz_avg() <= 64.0 && v.xpath < 2 ? sell_positions(h, s) : -1;
  const size_t sell_vb = h->storage == SPMV_DF64 ? 8 : dtype_bytes(h->storage);
  if (sell_pos >= 0 && sell_pos <= h->nnz + h->nnz / 8 + 32 * ((h->n_rows + 31) / 32) &&
      optional_fits((sell_vb + 4) * (size_t)sell_pos, s)) {
    spmv_variant t = v;
    t.partition = 3;
    t.vs = 1;
    prepare_variant(h, t, s);
    const float ms = time_launches([&]() { return launch_run(h, t, x.p, y.p, s); }, reps, s);
    if (ms < 0.95f * best) {
      best = ms;
      v = t;
    } else {
      drop_sell(h);
    }
  }
  sweep_panels(h, v, best, x.p, y.p, reps, s);
  if (v.partition != 3) drop_sell(h);
}

}  // namespace

extern "C" {

spmv_status spmv_tune_opts_default(spmv_tune_opts *o) {
  if (!o) return SPMV_ERR_ARG;
  std::memset(o, 0, sizeof *o);
  o->t_imb = 1.24;
  o->t_ml = 1.25;
  o->t_mb = 0.75;
  o->long_row_ratio = 32.0;
  o->autotune = 1;
  o->reps = 8;
  o->second_pass = 1;
  o->min_margin = 0.0;
  return SPMV_OK;
}

spmv_status spmv_tune(spmv_handle_t h, spmv_mode mode, const spmv_tune_opts *opts_in,
                      spmv_tune_report *report, spmv_stream_t stream) {
  if (!h) return SPMV_ERR_ARG;
  spmv_tune_opts opts;
  if (opts_in) opts = *opts_in;
  else spmv_tune_opts_default(&opts);
  if (opts.reps <= 0) opts.reps = 8;
  if (mode == SPMV_TUNE_LEARNED && !opts.selector) return SPMV_ERR_NO_SELECTOR;
  if (mode < SPMV_TUNE_PROFILE || mode > SPMV_TUNE_FIXED) return SPMV_ERR_ARG;
  if (mode == SPMV_TUNE_FIXED && !valid_variant(opts.fixed)) return SPMV_ERR_ARG;
  {
    spmv_variant lim{};
    lim.bin_med = opts.bin_med;
    lim.bin_chunk = opts.bin_chunk;
    if (!valid_variant(lim)) return SPMV_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  spmv_tune_report rep;
  std::memset(&rep, 0, sizeof rep);
  spmv_status st = guarded([&]() -> spmv_status {
    // untuned while probes and candidates rebuild the variant buffers: a failure part way
    // leaves no installed variant pointing at released buffers
    h->tuned = false;
    ++h->epoch;
    const double t0 = now_ms();
    uint32_t cls = 0;
    spmv_variant v{};
    int used = mode;
    double nnz_max = -1.0;
    auto need_features = [&]() {
      compute_features(h, 128, rep.features, nullptr, s);
      nnz_max = rep.features[3];
    };
    if (mode == SPMV_TUNE_FIXED) {
      v = opts.fixed;
    } else {
      bool done = false;
      if (mode == SPMV_TUNE_FEATURES) {
        need_features();
        const DeviceInfo &d = device_info(h->device);
        cls = feature_rules(rep.features, h->n_cols, (int)dtype_bytes(h->vec), d.l2_bytes,
                            opts.long_row_ratio);
        done = true;
      } else if (mode == SPMV_TUNE_LEARNED) {
        need_features();
        double f16[16];
        std::memcpy(f16, rep.features, sizeof(double) * 14);
        f16[14] = (double)h->n_rows;
        f16[15] = (double)h->nnz;
        uint32_t c = 0;
        double margin = 0.0;
        spmv_status ps = spmv_selector_predict(opts.selector, f16, &c, &margin, stream);
        if (ps != SPMV_OK) return ps;
        rep.margin = margin;
        if (margin >= opts.min_margin) {
          cls = c;
          done = true;
        } else {
          used = SPMV_TUNE_PROFILE;
        }
      }
      if (!done) {
        spmv_profile_report po;
        run_profile(h, opts.reps, po, s, opts.second_pass != 0);
        std::memcpy(rep.p, po.p, sizeof po.p);
        std::memcpy(rep.p2, po.p2, sizeof po.p2);
        rep.b_max_gbs = po.b_max_gbs;
        cls = classify2(po.p, opts.second_pass ? po.p2 : nullptr, opts.t_imb, opts.t_ml,
                        opts.t_mb);
        if (nnz_max < 0) {
          CK(launch_row_len_max(h->n_rows, h->rowptr.as<int32_t>(), h->small.as<int32_t>(), s));
          int32_t m = 0;
          CK(cudaMemcpyAsync(&m, h->small.p, 4, cudaMemcpyDeviceToHost, s));
          CK(cudaStreamSynchronize(s));
          nnz_max = (double)m;
        }
      }
      v = variant_for_classes(cls, h->nnz_avg(), nnz_max, opts.long_row_ratio);
      v.bin_med = opts.bin_med;
      v.bin_chunk = opts.bin_chunk;
    }
    const double t1 = now_ms();
    prepare_variant(h, v, s);
    CK(cudaStreamSynchronize(s));
    const double t2 = now_ms();
    if (opts.autotune && mode != SPMV_TUNE_FIXED)
      autotune_vs(h, v, std::max(3, opts.reps / 2), opts.bin_med, opts.bin_chunk, s);
    CK(cudaStreamSynchronize(s));
    const double t3 = now_ms();
    h->variant = v;
    ++h->epoch;
    h->tuned = true;
    rep.classes = cls;
    rep.mode_used = used;
    rep.variant = v;
    rep.t_classify_ms = t1 - t0;
    rep.t_prep_ms = t2 - t1;
    rep.t_autotune_ms = t3 - t2;

    rep.t_pre_ms = t3 - t0;
    return SPMV_OK;
  });
  if (st == SPMV_OK && report) *report = rep;
  return st;
}

spmv_status spmv_features(spmv_handle_t h, int32_t line_bytes, double *features, uint64_t *isum,
                          spmv_stream_t stream) {
  if (!h || !features || line_bytes <= 0) return SPMV_ERR_ARG;
  return guarded([&]() -> spmv_status {
    compute_features(h, line_bytes, features, isum, static_cast<cudaStream_t>(stream));
    return SPMV_OK;
  });
}

spmv_status spmv_profile(spmv_handle_t h, int32_t reps, spmv_profile_report *out,
                         spmv_stream_t stream) {
  if (!h || !out) return SPMV_ERR_ARG;
  return guarded([&]() -> spmv_status {
    spmv_profile_report o;
    run_profile(h, reps > 0 ? reps : 20, o, static_cast<cudaStream_t>(stream), true);
    *out = o;
    return SPMV_OK;
  });
}

spmv_status spmv_profile_cta_times(spmv_handle_t h, double *elapsed_ms, int32_t *sm_id,
                                   int32_t *n_ctas, spmv_stream_t stream) {
  if (!h || !n_ctas) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    const KernelSet *ks = set_for(h);
    const int n = std::max(1, device_info(h->device).sms * ks->profile_blocks_per_sm);
    if (!elapsed_ms && !sm_id) {
      *n_ctas = n;
      return SPMV_OK;
    }
    if (*n_ctas < n) return SPMV_ERR_ARG;
    const size_t vb = dtype_bytes(h->vec);
    DevBuf x, y;
    x.alloc(vb * (size_t)std::max<int64_t>(h->n_cols, 1), vb, s);
    y.alloc(vb * (size_t)std::max<int64_t>(h->n_rows, 1), vb, s);
    CK(launch_fill_const(x.p, h->vec, h->n_cols, 1.0, s));
    StaticSetup st;
    static_setup(h, st, x.p, y.p, s);
    for (int w = 0; w < 2; ++w) CK(ks->profile(st.pa, s));   // warm
    CK(ks->profile(st.pa, s));
    std::vector<double> el;
    std::vector<int32_t> sm;
    double span = 0;
    read_cta_times(st, el, sm, &span, s);
    for (int c = 0; c < n; ++c) {
      if (elapsed_ms) elapsed_ms[c] = el[(size_t)c] < 0 ? 0.0 : el[(size_t)c];
      if (sm_id) sm_id[c] = sm[(size_t)c];
    }
    *n_ctas = n;
    return SPMV_OK;
  });
}

spmv_status spmv_profile_kernel(spmv_handle_t h, int32_t which, const void *x, void *y,
                                spmv_stream_t stream) {
  if (!h || which < 0 || which > 2 || (h->n_rows > 0 && (!x || !y))) return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    const KernelSet *ks = set_for(h);
    StaticSetup st;
    static_setup(h, st, x, y, s);
    DevBuf colp;
    if (which == 1) {
      colp.alloc(sizeof(int32_t) * (size_t)h->nnz, 4, s);
      CK(launch_fill_row_index(h->n_rows, h->n_cols, h->rowptr.as<int32_t>(), colp.as<int32_t>(), s));
      st.pa.colind = colp.as<int32_t>();
    }
    st.pa.cmp_mode = which == 2 ? 1 : 0;
    CK(ks->profile(st.pa, s));
    CK(cudaStreamSynchronize(s));
    return SPMV_OK;
  });
}

spmv_status spmv_probe_bandwidth(double *hbm_gbs, double *l2_gbs) {
  if (!hbm_gbs || !l2_gbs) return SPMV_ERR_ARG;
  return guarded([&]() -> spmv_status {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    probe_bandwidth(dev, hbm_gbs, l2_gbs);
    return SPMV_OK;
  });
}

spmv_status spmv_probe_gather(int64_t n_x, int32_t elem_bytes, int64_t count, int32_t reps,
                              double *ms, spmv_stream_t stream) {
  if (!ms || n_x < 1 || n_x >= ((int64_t)1 << 32) || count < 1 || reps < 1 ||
      (elem_bytes != 4 && elem_bytes != 8))
    return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    DevBuf x, sink;
    x.alloc((size_t)elem_bytes * (size_t)n_x, 16, s);
    sink.alloc(8, 8, s, true);
    CK(launch_fill_const(x.p, elem_bytes == 8 ? SPMV_F64 : SPMV_F32, n_x, 1.0, s));
    float best = 1e30f;
    for (int r = 0; r < 3; ++r)
      best = std::min(best, time_launches([&]() {
        return launch_gather_probe(x.p, elem_bytes, n_x, count,
                                   sink.as<unsigned long long>(), s);
      }, reps, s));
    CK(cudaStreamSynchronize(s));
    *ms = best;
    return SPMV_OK;
  });
}

spmv_status spmv_probe_fma(int32_t elem_bytes, int32_t chains, int32_t warps_per_sm,
                           int32_t reps, double *fma_per_s, spmv_stream_t stream) {
  if (!fma_per_s || (elem_bytes != 4 && elem_bytes != 8) || reps < 1 ||
      (chains != 1 && chains != 2 && chains != 4 && chains != 8) || warps_per_sm < 1 ||
      warps_per_sm > 64 || (warps_per_sm > 32 && warps_per_sm % 2 != 0))
    return SPMV_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> spmv_status {
    constexpr int32_t kFmas = 16384;   // per thread and launch
    DevBuf sink;
    sink.alloc(8, 8, s, true);
    int64_t n_threads = 0;
    float best = 1e30f;
    for (int r = 0; r < 3; ++r)
      best = std::min(best, time_launches([&]() {
        return launch_fma_probe(elem_bytes, chains, warps_per_sm, kFmas, &n_threads,
                                sink.as<unsigned long long>(), s);
      }, reps, s));
    CK(cudaStreamSynchronize(s));
    *fma_per_s = (double)n_threads * kFmas / (best * 1e-3);
    return SPMV_OK;
  });
}

uint32_t spmv_classify(const double *p, double t_imb, double t_ml, double t_mb) {
  if (!p) return 0;
  return classify(p, t_imb, t_ml, t_mb);
}

uint32_t spmv_classify2(const double *p, const double *p2, double t_imb, double t_ml, double t_mb) {
  if (!p) return 0;
  return classify2(p, p2, t_imb, t_ml, t_mb);
}

void spmv_variant_for_classes(uint32_t classes, double nnz_avg, double nnz_max,
                              double long_row_ratio, spmv_variant *out) {
  if (out) *out = variant_for_classes(classes, nnz_avg, nnz_max, long_row_ratio);
}

void spmv_bounds(int64_t n_rows, int64_t n_cols, int64_t nnz, int32_t idx_bytes, int32_t val_bytes,
                 int32_t vec_bytes, double b_max_gbs, double *out) {
  if (out) bounds(n_rows, n_cols, nnz, idx_bytes, val_bytes, vec_bytes, b_max_gbs, out);
}

uint32_t spmv_feature_rules(const double *features, int64_t n_cols, int32_t vec_bytes,
                            int64_t l2_bytes, double long_row_ratio) {
  if (!features) return 0;
  return feature_rules(features, n_cols, vec_bytes, l2_bytes, long_row_ratio);
}

}  // extern "C"

// Host runtime of libamber: argument validation, the Weibull history solve
// (Sec. 3.1.2, Appendix A), the context and its one-time workspace, per-
// kernel event timing, and the extern "C" entry points declared in amber.h.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "assign.cuh"
#include "fft.cuh"
#include "sort.cuh"
#include "source.cuh"
#include "spectra.cuh"
#include "lpt.cuh"

namespace amber {
// krange: if not null, the intensities' key range is folded into it (the
// sort's control block, reset beforehand) so the ranking needs no range pass.
// variant: the FFT tile/radix variant (0 default; 1 for n >= 128).
// spec_in: if not null, the x- and y-transformed source (source_spectrum_f32's
// output), read by the z pass instead of transforming src.
// hist8: the inverse x pass also counts the raw keys' 8-bit digits into krange.
// tma: the z pass stages its tiles with the tensor-memory accelerator
// (k_fft_zconv_tma; two-stage sizes n >= 64, same results bit for bit).
cudaError_t radiation_field_f32(int n, const float* src, float* J, void* H, const void* tw, double box, double l_mfp,
                               unsigned int* status, cudaStream_t s, FftProfile* prof, SortCtrl* krange,
                               int variant, const void* spec_in = nullptr, bool hist8 = false, bool tma = false);
cudaError_t source_spectrum_f32(int n, const float* src, void* H, const void* tw, cudaStream_t s, FftProfile* prof,
                               int variant);
cudaError_t radiation_field_multi_f32(int n, int variant, const float* const* srcs, int M, float* J, void* H,
                                      const void* tw, const float* kp, unsigned int* status, cudaStream_t s,
                                      SortCtrl* kranges);
cudaError_t radiation_field_f64(int n, const double* src, double* J, void* H, const void* tw, double box,
                               double l_mfp, unsigned int* status, cudaStream_t s, FftProfile* prof,
                               SortCtrl* krange);

// ---------------------------------------------------------------------------
// Per-kernel timing: a pool of events recorded around launches.
// ---------------------------------------------------------------------------
static const char* kProfNames[PK_COUNT] = {
    "fft_r2c_x", "fft_y_fwd", "fft_z_conv", "fft_y_inv", "fft_c2r_x",
    "sort_histogram", "sort_pass", "mass_reduce", "thresholds", "scan_assign", "scatter_back"};

struct FftProfile {
  bool on = false;
  int device = 0;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Rec { int kind; size_t ev; };
  std::vector<Rec> recs;
  int open_kind = -1;
  double total_ms[PK_COUNT] = {};
  int64_t launches[PK_COUNT] = {};
};

void prof_begin(FftProfile* p, int kind, cudaStream_t s) {
  if (!p || !p->on) return;
  if (p->used + 2 > p->pool.size()) { p->open_kind = -1; return; }
  cudaEventRecord(p->pool[p->used], s);
  p->recs.push_back({kind, p->used});
  p->used += 2;
  p->open_kind = kind;
}
void prof_end(FftProfile* p, int kind, cudaStream_t s) {
  if (!p || !p->on || p->open_kind != kind) return;
  cudaEventRecord(p->pool[p->recs.back().ev + 1], s);
  p->open_kind = -1;
}
static void prof_harvest(FftProfile* p) {
  for (const auto& r : p->recs) {
    cudaEventSynchronize(p->pool[r.ev + 1]);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->pool[r.ev], p->pool[r.ev + 1]) == cudaSuccess) {
      p->total_ms[r.kind] += ms;
      p->launches[r.kind] += 1;
    }
  }
  p->recs.clear();
  p->used = 0;
}

// ---------------------------------------------------------------------------
// Weibull history (Sec. 3.1.1, 3.1.2, Appendix A) in FP64 on the host.
// ---------------------------------------------------------------------------
static bool history_valid(const amber_history_t* h) {
  if (!h) return false;
  const double v[] = {h->z_mid, h->dz, h->Az, h->x_ear, h->x_mid, h->x_lat, h->z_lo, h->z_hi};
  for (double x : v)
    if (!std::isfinite(x)) return false;
  if (!(0.0 < h->x_ear && h->x_ear < h->x_mid && h->x_mid < h->x_lat && h->x_lat < 1.0)) return false;
  if (!(h->dz > 0.0 && h->Az > 0.0)) return false;
  if (!(h->z_hi > h->z_lo)) return false;
  if (h->n_table < 2 || h->n_table > kMaxTable) return false;
  if (h->weighting != AMBER_WEIGHT_MASS && h->weighting != AMBER_WEIGHT_MASS_GROWTH &&
      h->weighting != AMBER_WEIGHT_VOLUME)
    return false;
  if (h->weighting == AMBER_WEIGHT_MASS_GROWTH && !(h->omega_m > 0.0 && h->omega_m <= 1.0)) return false;
  return true;
}

// Offset a through the mid and late points for power c (Appendix A).
static double a_mid_lat(double c, double zm, double zl, double Lm, double Ll) {
  const double pm = std::pow(Lm, 1.0 / c), pl = std::pow(Ll, 1.0 / c);
  return (zl * pm - zm * pl) / (pm - pl);
}

static int weibull_solve(const amber_history_t* h, double* a_out, double* b_out, double* c_out) {
  if (!history_valid(h)) return AMBER_ERR_INVALID_ARG;
  const double ze = h->z_mid + h->dz * h->Az / (1.0 + h->Az);  // Eq. zear
  const double zm = h->z_mid;
  const double zl = ze - h->dz;                                 // Eq. duration
  const double Le = std::fabs(std::log(h->x_ear)), Lm = std::fabs(std::log(h->x_mid)),
               Ll = std::fabs(std::log(h->x_lat));
  auto f = [&](double c) {
    const double a = a_mid_lat(c, zm, zl, Lm, Ll);
    return std::pow(Le / Lm, 1.0 / c) - (ze - a) / (zm - a);
  };
  const int G = 400;
  const double lc0 = std::log(0.05), lc1 = std::log(100.0);
  double cprev = std::exp(lc0), fprev = f(cprev);
  for (int i = 1; i <= G; ++i) {
    const double c = std::exp(lc0 + (lc1 - lc0) * i / G);
    const double fc = f(c);
    const bool ok = std::isfinite(fprev) && std::isfinite(fc) && !(fprev * fc > 0.0);
    if (ok) {
      double lo = cprev, hi = c, flo = fprev;
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double fm = f(mid);
        if (fm == 0.0) { lo = hi = mid; break; }
        if ((fm > 0.0) == (flo > 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
        if (hi - lo <= 1e-15 * hi) break;
      }
      const double cw = 0.5 * (lo + hi);
      const double pe = std::pow(Le, 1.0 / cw), pl = std::pow(Ll, 1.0 / cw);
      const double aw = (ze * pl - zl * pe) / (pl - pe);
      const double bw = (zm - aw) / std::pow(Lm, 1.0 / cw);
      if (aw > 0.0 && bw > 0.0 && cw > 0.0) {
        *a_out = aw; *b_out = bw; *c_out = cw;
        return AMBER_OK;
      }
    }
    cprev = c;
    fprev = fc;
  }
  return AMBER_ERR_NO_SOLUTION;
}

static int history_coeffs(const amber_history_t* h, HistoryCoeffs* hc) {
  double a, b, c;
  const int st = weibull_solve(h, &a, &b, &c);
  if (st != AMBER_OK) return st;
  hc->a = a; hc->b = b; hc->c = c;
  hc->z_lo = std::fmin(h->z_lo, a);  // reach the fully ionized plateau
  hc->z_hi = h->z_hi;
  hc->n_table = h->n_table;
  hc->weighting = h->weighting;
  hc->omega_m = h->omega_m;
  hc->z_mid = h->z_mid;
  return AMBER_OK;
}

// ---------------------------------------------------------------------------
// Workspace plan.
// ---------------------------------------------------------------------------
static int fft_nmax(int64_t cells) {
  int n = 0;
  for (int m = 4; m <= 1024; m *= 2)
    if ((int64_t)m * m * m <= cells) n = m;
  return n;
}

struct Plan {
  int n32 = 0, n64 = 0;
  int64_t cells64 = 0;
  size_t off_spec, off_keysA, off_keysB, off_idxA, off_idxB, off_massA, off_massB, off_lb, off_sctrl, off_actrl, off_X, off_invdx, off_lin,
      off_state, off_btab, off_tilemass, off_status, off_srcsum, off_pow, off_tw32, off_tw64, total;
  size_t tw32_off[11] = {}, tw64_off[11] = {};
};

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

static Plan make_plan(int64_t max_cells) {
  Plan p;
  p.n32 = fft_nmax(max_cells);
  p.n64 = std::min(p.n32, 256);
  p.cells64 = std::min<int64_t>(max_cells, (int64_t)1 << 24);
  auto spec_bytes = [](int n, size_t elem) { return n ? (size_t)n * n * (n / 2 + 2) * elem : 0; };
  const size_t spec = std::max(spec_bytes(p.n32, 8), spec_bytes(p.n64, 16));
  const size_t keyb = std::max((size_t)max_cells * 4, (size_t)p.cells64 * 8);
  const size_t idxb = (size_t)max_cells * 4;
  const size_t lb = 2 * sort_lookback_words(max_cells) * 4;
  const size_t stt = (size_t)((max_cells + kScanTile - 1) / kScanTile) * sizeof(unsigned long long);
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o += align256(bytes); return at; };
  p.off_spec = take(spec);
  p.off_keysA = take(keyb);
  p.off_keysB = take(keyb);
  p.off_idxA = take(idxb);
  p.off_idxB = take(idxb);
  p.off_massA = take(idxb);
  p.off_massB = take(idxb);
  p.off_lb = take(lb);
  p.off_sctrl = take(sizeof(SortCtrl));
  p.off_actrl = take(kAssignCtrlBytes);
  p.off_X = take((size_t)kMaxTable * sizeof(unsigned long long));
  p.off_invdx = take((size_t)kMaxTable * sizeof(float));
  p.off_lin = take((size_t)4 * kMaxTable * sizeof(float));
  p.off_state = take(stt);
  p.off_btab = take((size_t)((max_cells + kScanTile - 1) / kScanTile) * (kMaxBuckets + 1) * sizeof(uint16_t));
  p.off_tilemass = take((size_t)sort_tiles(max_cells) * 16);
  p.off_status = take(256);
  p.off_srcsum = take(256);
  p.off_pow = take((size_t)kPowerAcc * kMaxPowerBins * sizeof(double));
  size_t tw32 = 0, tw64 = 0;
  for (int l = 2, n = 4; n <= 1024; ++l, n *= 2) {
    if (n <= p.n32) { p.tw32_off[l] = tw32; tw32 += align256((size_t)n * 8); }
    if (n <= p.n64) { p.tw64_off[l] = tw64; tw64 += align256((size_t)n * 16); }
  }
  p.off_tw32 = take(tw32);
  p.off_tw64 = take(tw64);
  p.total = o;
  return p;
}

static int ilog2i(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

}  // namespace amber

using namespace amber;

struct amber_ctx {
  int device = 0;
  int64_t max_cells = 0;
  Plan plan;
  unsigned char* ws = nullptr;
  unsigned int* status = nullptr;
  unsigned int* h_status = nullptr;  // pinned
  SortWork sortw{};
  AssignWork assw{};
  int num_sms = 0;
  FftProfile prof;
  cudaStream_t last_stream = nullptr;
  amber_tuning_t tune[11] = {};  // per log2 n: FFT variant, digit width and peers of the FP32 solve path
  cudaEvent_t host_solve_done = nullptr;  // recorded after each amber_solve_host's solve
  std::mutex mu;
};

namespace {
// Host-buffer solves on one device take turns in call order: each waits for
// the previous one's solve (not its copies), so contexts used in turn overlap
// one call's copies with another's solve without two solves sharing the GPU.
std::mutex g_host_solve_mu;
amber_ctx* g_last_host_solve[64] = {};
}  // namespace

namespace {

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

bool is_pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

// A device array must start on a multiple of its element size (NULL passes:
// optional arguments are checked for presence separately).  Kernels need no
// more than that: wider vector loads check their own alignment.
template <typename T> bool elem_aligned(const T* p) { return (reinterpret_cast<uintptr_t>(p) % sizeof(T)) == 0; }
bool all_aligned() { return true; }
template <typename T, typename... R> bool all_aligned(const T* p, const R*... rest) {
  return elem_aligned(p) && all_aligned(rest...);
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return AMBER_OK;
  return AMBER_ERR_CUDA;
}

}  // namespace

namespace {

// Bump allocator over one device allocation (256-byte aligned pieces).
struct Layout {
  size_t total = 0;
  size_t take(size_t bytes) {
    const size_t at = total;
    total += align256(bytes);
    return at;
  }
};

// Host copy of a device argument array, placed at `off` in the workspace.
struct HostBlob {
  size_t off = 0;
  std::vector<unsigned char> bytes;
  template <typename T> void set(const std::vector<T>& v) {
    bytes.resize(v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(bytes.data(), v.data(), bytes.size());
  }
};

}  // namespace

extern "C" {

int amber_history_default(amber_history_t* h, double z_mid, double dz, double Az) {
  if (!h) return AMBER_ERR_INVALID_ARG;
  h->z_mid = z_mid; h->dz = dz; h->Az = Az;
  h->x_ear = 0.05; h->x_mid = 0.50; h->x_lat = 0.95;
  h->z_lo = 5.0; h->z_hi = 20.0; h->n_table = 2000;
  h->weighting = AMBER_WEIGHT_MASS;
  h->omega_m = 0.3;
  return AMBER_OK;
}

int amber_history_coeffs(const amber_history_t* h, double out_abc[3]) {
  if (!h || !out_abc) return AMBER_ERR_INVALID_ARG;
  double a, b, c;
  const int st = weibull_solve(h, &a, &b, &c);
  if (st != AMBER_OK) return st;
  out_abc[0] = a; out_abc[1] = b; out_abc[2] = c;
  return AMBER_OK;
}

int amber_history_table(const amber_history_t* h, double* z_out, double* x_out) {
  if (!h || !z_out || !x_out) return AMBER_ERR_INVALID_ARG;
  HistoryCoeffs hc;
  const int st = history_coeffs(h, &hc);
  if (st != AMBER_OK) return st;
  for (int j = 0; j < hc.n_table; ++j) {
    const double z = hc.z_lo + (hc.z_hi - hc.z_lo) * (double)j / (double)(hc.n_table - 1);
    const double u = std::fmax((z - hc.a) / hc.b, 0.0);
    z_out[j] = z;
    x_out[j] = std::exp(-std::pow(u, hc.c));
  }
  return AMBER_OK;
}

int amber_workspace_bytes(int64_t max_cells, size_t* out_bytes) {
  if (!out_bytes || max_cells < 1 || max_cells > ((int64_t)1 << 30)) return AMBER_ERR_INVALID_ARG;
  *out_bytes = make_plan(max_cells).total;
  return AMBER_OK;
}

int amber_create(amber_ctx** out, int device, int64_t max_cells) {
  if (!out || max_cells < 1 || max_cells > ((int64_t)1 << 30) || device < 0) return AMBER_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device >= ndev) {
    cudaGetLastError();
    return AMBER_ERR_CUDA;
  }
  DeviceGuard g(device);
  amber_ctx* c = new (std::nothrow) amber_ctx();
  // defaults: the autotuner's picks on the synthetic recipe -- 8-bit digits
  // from 512^3 up (four passes of 8 bits beat three of 9 there: 30.7 vs
  // 32.1 ms per ranking at 1024^3), 9-bit below, default FFT tiles, ballots
  if (c)
    for (int l = 0; l < 11; ++l)
      c->tune[l] = amber_tuning_t{1 << l, 0, l >= 9 ? 8 : 9, 0, 0, {0.0, 0.0}, {0.0, 0.0, 0.0, 0.0}, 0, l == 9 ? 1 : 0,
                                  0.0};
  if (!c) return AMBER_ERR_OOM;
  c->device = device;
  c->max_cells = max_cells;
  c->plan = make_plan(max_cells);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&c->ws, c->plan.total) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return AMBER_ERR_OOM;
  }
  if (cudaMallocHost(&c->h_status, sizeof(unsigned int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->ws);
    delete c;
    return AMBER_ERR_CUDA;
  }
  if (cudaEventCreateWithFlags(&c->host_solve_done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(c->h_status);
    cudaFree(c->ws);
    delete c;
    return AMBER_ERR_CUDA;
  }
  const Plan& p = c->plan;
  c->status = reinterpret_cast<unsigned int*>(c->ws + p.off_status);
  cudaMemset(c->ws + p.off_status, 0, 256);
  c->sortw.keysA = c->ws + p.off_keysA;
  c->sortw.keysB = c->ws + p.off_keysB;
  c->sortw.idxA = reinterpret_cast<uint32_t*>(c->ws + p.off_idxA);
  c->sortw.idxB = reinterpret_cast<uint32_t*>(c->ws + p.off_idxB);
  c->sortw.massA = reinterpret_cast<float*>(c->ws + p.off_massA);
  c->sortw.massB = reinterpret_cast<float*>(c->ws + p.off_massB);
  c->sortw.lookback = reinterpret_cast<uint32_t*>(c->ws + p.off_lb);
  c->sortw.ctrl = reinterpret_cast<SortCtrl*>(c->ws + p.off_sctrl);
  c->sortw.max_cells = max_cells;
  c->sortw.num_sms = c->num_sms;
  c->assw.ctrl = c->ws + p.off_actrl;
  c->assw.Xq = reinterpret_cast<unsigned long long*>(c->ws + p.off_X);
  c->assw.inv_dx = reinterpret_cast<float*>(c->ws + p.off_invdx);
  c->assw.lin = reinterpret_cast<float*>(c->ws + p.off_lin);
  c->assw.state = reinterpret_cast<unsigned long long*>(c->ws + p.off_state);
  // bucketed (cell, z) pairs reuse the key buffers, dead once ranked
  c->assw.bcell = reinterpret_cast<uint32_t*>(c->sortw.keysA);
  c->assw.bz = reinterpret_cast<float*>(c->sortw.keysB);
  c->assw.btab = reinterpret_cast<uint16_t*>(c->ws + p.off_btab);
  c->assw.num_sms = c->num_sms;
  // twiddles w_n^m = exp(-2 pi i m / n), FP64 on the host, rounded for FP32
  for (int l = 6, n = 64; n <= p.n32; ++l, n *= 2) {
    std::vector<float> t32(2 * n);
    std::vector<double> t64(2 * n);
    for (int m = 0; m < n; ++m) {
      const double ang = -2.0 * M_PI * (double)m / (double)n;
      t64[2 * m] = std::cos(ang);
      t64[2 * m + 1] = std::sin(ang);
      t32[2 * m] = (float)t64[2 * m];
      t32[2 * m + 1] = (float)t64[2 * m + 1];
    }
    cudaMemcpy(c->ws + p.off_tw32 + p.tw32_off[l], t32.data(), t32.size() * 4, cudaMemcpyHostToDevice);
    if (n <= p.n64) cudaMemcpy(c->ws + p.off_tw64 + p.tw64_off[l], t64.data(), t64.size() * 8, cudaMemcpyHostToDevice);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(c->h_status);
    cudaFree(c->ws);
    delete c;
    return AMBER_ERR_CUDA;
  }
  *out = c;
  return AMBER_OK;
}

int amber_destroy(amber_ctx* c) {
  if (!c) return AMBER_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(g_host_solve_mu);
    if (c->device >= 0 && c->device < 64 && g_last_host_solve[c->device] == c) g_last_host_solve[c->device] = nullptr;
  }
  {
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    if (c->host_solve_done) cudaEventDestroy(c->host_solve_done);
    for (auto e : c->prof.pool) cudaEventDestroy(e);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->ws) cudaFree(c->ws);
  }
  delete c;
  return AMBER_OK;
}

extern "C++" {
template <typename T>
static int rf_args_ok(amber_ctx* c, const T* src, int n, double box, double l, const T* J, int nmax) {
  if (!c || !src || !J || !all_aligned(src, J)) return AMBER_ERR_INVALID_ARG;
  if (!is_pow2_in(n, 4, 1024) || !(box > 0.0) || !std::isfinite(box) || !(l > 0.0) || !std::isfinite(l))
    return AMBER_ERR_INVALID_ARG;
  if (n > nmax) return AMBER_ERR_CAPACITY;
  return AMBER_OK;
}
}  // extern "C++"

int amber_radiation_field(amber_ctx* c, const float* d_src, int n, double box, double l_mfp, float* d_J,
                          void* stream) {
  int st = rf_args_ok(c, d_src, n, box, l_mfp, d_J, c ? c->plan.n32 : 0);
  if (st) return st;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const Plan& p = c->plan;
  const int l = ilog2i(n);
  return cuda_status(radiation_field_f32(n, d_src, d_J, c->ws + p.off_spec, c->ws + p.off_tw32 + p.tw32_off[l], box,
                                         l_mfp, c->status, s, &c->prof, nullptr, c->tune[l].fft_variant, nullptr,
                                         false, c->tune[l].zpass_tma != 0));
}

int amber_radiation_field_f64(amber_ctx* c, const double* d_src, int n, double box, double l_mfp, double* d_J,
                              void* stream) {
  int st = rf_args_ok(c, d_src, n, box, l_mfp, d_J, c ? c->plan.n64 : 0);
  if (st) return st;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const Plan& p = c->plan;
  const int l = ilog2i(n);
  return cuda_status(radiation_field_f64(n, d_src, d_J, c->ws + p.off_spec, c->ws + p.off_tw64 + p.tw64_off[l], box,
                                         l_mfp, c->status, s, &c->prof, nullptr));
}

int amber_power_bins(int n, int* nbins) {
  if (!nbins || !is_pow2_in(n, 4, 1024)) return AMBER_ERR_INVALID_ARG;
  *nbins = power_bins(n);
  return AMBER_OK;
}

int amber_delta_z(amber_ctx* c, const float* d_z, int64_t ncells, float* d_out, double* d_zbar_opt, void* stream) {
  if (!c || !d_z || !d_out || ncells < 1 || !all_aligned(d_z, d_out, d_zbar_opt)) return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  double* acc = reinterpret_cast<double*>(c->ws + c->plan.off_pow);
  return cuda_status(delta_z_impl(d_z, ncells, d_out, acc, d_zbar_opt, c->num_sms, s));
}

int amber_epsilon_z_pdf(amber_ctx* c, const float* d_z, const float* d_zref, int64_t ncells, double lo, double hi,
                        int nbins, unsigned long long* d_counts, double* d_moments_opt, void* stream) {
  if (!c || !d_z || !d_zref || !d_counts || ncells < 1 || !all_aligned(d_z, d_zref, d_counts, d_moments_opt))
    return AMBER_ERR_INVALID_ARG;
  if (!std::isfinite(lo) || !std::isfinite(hi) || !(hi > lo) || nbins < 1 || nbins > 16000)
    return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(epsilon_pdf_impl(d_z, d_zref, ncells, lo, hi, nbins, d_counts, d_moments_opt, c->num_sms, s));
}

int amber_power_spectrum(amber_ctx* c, const float* d_a, const float* d_b_opt, int n, double box, double* d_k,
                         double* d_Paa, double* d_Pbb_opt, double* d_Pab_opt, double* d_modes, void* stream) {
  if (!c || !d_a || !d_k || !d_Paa || !d_modes) return AMBER_ERR_INVALID_ARG;
  if (!all_aligned(d_a, d_b_opt, d_k, d_Paa, d_Pbb_opt, d_Pab_opt, d_modes)) return AMBER_ERR_INVALID_ARG;
  if (!is_pow2_in(n, 4, 1024) || !(box > 0.0) || !std::isfinite(box)) return AMBER_ERR_INVALID_ARG;
  if (n > c->plan.n32) return AMBER_ERR_CAPACITY;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const Plan& p = c->plan;
  const void* tw = c->ws + p.off_tw32 + p.tw32_off[ilog2i(n)];
  // a's spectrum in the transform buffer; b's in the key buffers, which are
  // contiguous and hold 8 bytes per cell (the half spectrum needs 4 + 16/n)
  void* Ha = c->ws + p.off_spec;
  void* Hb = d_b_opt ? static_cast<void*>(c->sortw.keysA) : nullptr;
  cudaError_t e = forward_spectrum_f32(n, d_a, Ha, tw, s);
  if (e == cudaSuccess && d_b_opt) e = forward_spectrum_f32(n, d_b_opt, Hb, tw, s);
  if (e == cudaSuccess)
    e = power_impl(Ha, Hb, n, box, reinterpret_cast<double*>(c->ws + p.off_pow), d_k, d_Paa, d_Pbb_opt, d_Pab_opt,
                   d_modes, c->num_sms, s);
  return cuda_status(e);
}

int amber_power_derived(amber_ctx* c, const double* d_k, const double* d_Paa, const double* d_Pbb_opt,
                        const double* d_Pab_opt, int nbins, double* d_D2aa, double* d_D2bb_opt, double* d_bias_opt,
                        double* d_r_opt, void* stream) {
  if (!c || !d_k || !d_Paa || !d_D2aa || nbins < 1 || nbins > kMaxPowerBins) return AMBER_ERR_INVALID_ARG;
  if ((d_D2bb_opt || d_bias_opt || d_r_opt) && !d_Pbb_opt) return AMBER_ERR_INVALID_ARG;
  if (d_r_opt && !d_Pab_opt) return AMBER_ERR_INVALID_ARG;
  if (!all_aligned(d_k, d_Paa, d_Pbb_opt, d_Pab_opt, d_D2aa, d_D2bb_opt, d_bias_opt, d_r_opt))
    return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(power_derived_impl(d_k, d_Paa, d_Pbb_opt, d_Pab_opt, nbins, d_D2aa, d_D2bb_opt, d_bias_opt,
                                        d_r_opt, s));
}

static LptWork lpt_work(amber_ctx* c, int n) {
  const Plan& p = c->plan;
  LptWork w{};
  // three half spectra (4 + 16/n bytes per cell each): the transform buffer
  // and the key and index ping-pong pairs (8 bytes per cell each); two fields
  // in the mass pair
  w.H0 = c->ws + p.off_spec;
  w.H1 = c->sortw.keysA;
  w.H2 = c->sortw.idxA;
  w.F0 = c->sortw.massA;
  w.F1 = c->sortw.massB;
  w.acc = reinterpret_cast<double*>(c->ws + p.off_pow);
  w.tw = c->ws + p.off_tw32 + p.tw32_off[ilog2i(n)];
  w.status = c->status;
  w.num_sms = c->num_sms;
  return w;
}

static int lpt_args_ok(amber_ctx* c, int n, double box) {
  if (!c) return AMBER_ERR_INVALID_ARG;
  if (!is_pow2_in(n, 4, 1024) || !(box > 0.0) || !std::isfinite(box)) return AMBER_ERR_INVALID_ARG;
  if (n > c->plan.n32) return AMBER_ERR_CAPACITY;
  return AMBER_OK;
}

int amber_lpt_displacement(amber_ctx* c, const float* d_delta_lin, int n, double box, double D1, double D2,
                           float* d_psi_x, float* d_psi_y, float* d_psi_z, void* stream) {
  int st = lpt_args_ok(c, n, box);
  if (st) return st;
  if (!d_delta_lin || !d_psi_x || !d_psi_y || !d_psi_z || !std::isfinite(D1) || !std::isfinite(D2))
    return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(lpt_impl(lpt_work(c, n), n, box, D1, D2, d_delta_lin, d_psi_x, d_psi_y, d_psi_z, s));
}

int amber_mesh_density(amber_ctx* c, const float* d_psi_x, const float* d_psi_y, const float* d_psi_z,
                       const float* d_mass_opt, int n, double box, int order, int interlace, float* d_rho,
                       void* stream) {
  int st = lpt_args_ok(c, n, box);
  if (st) return st;
  if (!d_psi_x || !d_psi_y || !d_psi_z || !d_rho || order < 1 || order > 3 || (interlace != 0 && interlace != 1))
    return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(mesh_impl(lpt_work(c, n), n, box, order, interlace == 1, d_psi_x, d_psi_y, d_psi_z, d_mass_opt,
                               d_rho, s));
}

int amber_esf_fcoll(amber_ctx* c, const float* d_delta_lin, int n, double box, double R, int filter, double delta_c,
                    double dsigma2, float* d_fcoll, void* stream) {
  int st = lpt_args_ok(c, n, box);
  if (st) return st;
  if (!d_delta_lin || !d_fcoll || !(R > 0.0) || !std::isfinite(R) || (filter != 0 && filter != 1) ||
      !std::isfinite(delta_c) || !(dsigma2 > 0.0) || !std::isfinite(dsigma2))
    return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(fcoll_impl(lpt_work(c, n), n, box, R, filter, delta_c, dsigma2, d_delta_lin, d_fcoll, s));
}

int amber_sigma2_tophat(const double* k, const double* Delta2, int nk, double R, double* out) {
  if (!k || !Delta2 || !out || nk < 2 || !(R > 0.0)) return AMBER_ERR_INVALID_ARG;
  double acc = 0.0, prev = 0.0;
  for (int i = 0; i < nk; ++i) {
    if (!(k[i] > 0.0) || (i && !(k[i] > k[i - 1]))) return AMBER_ERR_INVALID_ARG;
    const double x = k[i] * R;
    const double W = x < 1e-3 ? 1.0 - x * x / 10.0 : 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
    const double f = Delta2[i] * W * W;
    if (i) acc += 0.5 * (f + prev) * std::log(k[i] / k[i - 1]);
    prev = f;
  }
  *out = acc;
  return AMBER_OK;
}

int amber_rank(amber_ctx* c, const float* d_J, int64_t ncells, uint32_t* d_order, void* stream) {
  if (!c || !d_J || !d_order || ncells < 1 || !all_aligned(d_J, d_order)) return AMBER_ERR_INVALID_ARG;
  if (ncells > c->max_cells) return AMBER_ERR_CAPACITY;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(rank_impl<float>(c->sortw, d_J, ncells, d_order, nullptr, nullptr, nullptr, false, c->status, s,
                                      &c->prof, kSpinLimit));
}

int amber_rank_f64(amber_ctx* c, const double* d_J, int64_t ncells, uint32_t* d_order, void* stream) {
  if (!c || !d_J || !d_order || ncells < 1 || !all_aligned(d_J, d_order)) return AMBER_ERR_INVALID_ARG;
  if (ncells > c->plan.cells64) return AMBER_ERR_CAPACITY;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(rank_impl<double>(c->sortw, d_J, ncells, d_order, nullptr, nullptr, nullptr, false, c->status, s,
                                       &c->prof, kSpinLimit));
}

int amber_assign_zre(amber_ctx* c, const uint32_t* d_order, const float* d_mass, int64_t ncells,
                     const amber_history_t* h, float* d_zre, double* d_F_opt, void* stream) {
  if (!c || !d_order || !d_mass || !d_zre || ncells < 1 || !all_aligned(d_order, d_mass, d_zre, d_F_opt))
    return AMBER_ERR_INVALID_ARG;
  if (ncells > c->max_cells) return AMBER_ERR_CAPACITY;
  HistoryCoeffs hc;
  const int st = history_coeffs(h, &hc);
  if (st) return st;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(assign_impl(c->assw, d_order, d_mass, false, nullptr, ncells, hc, d_zre, d_F_opt, c->status, s,
                                 &c->prof, kSpinLimit));
}

extern "C++" {
template <typename T>
static int solve_args(amber_ctx* c, const T* src, const float* mass, const amber_params_t* p, const float* zre,
                      int want_prec, int nmax, HistoryCoeffs* hc) {
  if (!c || !src || !mass || !p || !zre || !all_aligned(src, mass, zre)) return AMBER_ERR_INVALID_ARG;
  if (p->precision != want_prec) return AMBER_ERR_INVALID_ARG;
  int st = rf_args_ok(c, src, p->n, p->box, p->l_mfp, src, nmax);
  if (st) return st;
  return history_coeffs(&p->hist, hc);
}
}  // extern "C++"

// Enqueue one FP32 solve on s (no locking, no validation).  With order_out
// (and mass_rank_out) the sort leaves the rank order and the rank-order
// masses there for the caller; otherwise they stay in the workspace.
static cudaError_t solve_f32_enqueue(amber_ctx* c, const float* d_src, const float* d_mass, const amber_params_t* p,
                                     const HistoryCoeffs& hc, float* d_zre, float* d_J_opt, uint32_t* order_out,
                                     float* mass_rank_out, cudaStream_t s, const void* spec_in = nullptr) {
  const Plan& pl = c->plan;
  const int n = p->n;
  const int64_t C = (int64_t)n * n * n;
  float* J = d_J_opt ? d_J_opt : reinterpret_cast<float*>(c->sortw.keysB);
  const amber_tuning_t& tu = c->tune[ilog2i(n)];
  // with 8-bit digits the inverse x pass can count the raw keys' digits
  const bool fuse = tu.fuse_histogram && tu.sort_digit_bits == 8;
  cudaError_t e = sort_ctrl_reset(c->sortw.ctrl, s);
  if (e == cudaSuccess)
    e = radiation_field_f32(n, d_src, J, c->ws + pl.off_spec, c->ws + pl.off_tw32 + pl.tw32_off[ilog2i(n)], p->box,
                           p->l_mfp, c->status, s, &c->prof, c->sortw.ctrl, tu.fft_variant, spec_in, fuse,
                           tu.zpass_tma != 0);
  // the first sort pass sums each tile's masses; the thresholds kernel adds them
  unsigned long long* tile_mass = reinterpret_cast<unsigned long long*>(c->ws + pl.off_tilemass);
  if (e == cudaSuccess)
    e = rank_impl<float>(c->sortw, J, C, order_out, d_mass, order_out ? mass_rank_out : nullptr, tile_mass, true,
                         c->status, s, &c->prof, kSpinLimit, tu.sort_digit_bits, tu.sort_match, fuse);
  if (e != cudaSuccess) return e;
  if (order_out)
    return assign_impl(c->assw, order_out, mass_rank_out, true, tile_mass, C, hc, d_zre, nullptr, c->status, s,
                       &c->prof, kSpinLimit);
  // the order and rank-order masses sit on the A or B side by pass parity
  return assign_impl(c->assw, c->sortw.idxA, c->sortw.massA, true, tile_mass, C, hc, d_zre, nullptr, c->status, s,
                     &c->prof, kSpinLimit, c->sortw.idxB, c->sortw.massB, &c->sortw.ctrl->npasses);
}

// Autotuning of one grid size (the context's lock held): every FFT variant,
// then every (digit width, digit-peer method) of the ranking on the chosen
// variant's intensities, each once untimed and three times timed.
static bool autotune_enabled() {
  const char* v = getenv("AMBER_AUTOTUNE");
  return !(v && strcmp(v, "0") == 0);
}

static int autotune_locked(amber_ctx* c, const float* d_src, const float* d_mass, int n, double box, double l_mfp,
                           amber_tuning_t* out, cudaStream_t s) {
  const Plan& pl = c->plan;
  const int lg = ilog2i(n);
  const int64_t C = (int64_t)n * n * n;
  const void* tw = c->ws + pl.off_tw32 + pl.tw32_off[lg];
  float* J = reinterpret_cast<float*>(c->sortw.keysB);
  // the spectrum buffer (>= 4 B/cell) is free once a transform is done: it
  // keeps the intensities the ranking candidates start from
  float* Jkeep = reinterpret_cast<float*>(c->ws + pl.off_spec);
  unsigned long long* tile_mass = reinterpret_cast<unsigned long long*>(c->ws + pl.off_tilemass);
  const bool prof_on = c->prof.on;
  c->prof.on = false;
  amber_tuning_t t = c->tune[lg];
  t.n = n;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // median of three timed runs after one untimed run
  auto timed = [&](auto&& run, double* ms_out) {
    double ms[3] = {0.0, 0.0, 0.0};
    for (int r = -1; r < 3 && e == cudaSuccess; ++r) {
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = run();
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float f = 0.f;
      if (e == cudaSuccess && r >= 0) e = cudaEventElapsedTime(&f, e0, e1);
      if (r >= 0) ms[r] = f;
    }
    std::sort(ms, ms + 3);
    *ms_out = ms[1];
  };
  const int nv = n >= 128 ? 2 : 1;
  t.fft_ms[0] = t.fft_ms[1] = 0.0;
  for (int v = 0; v < nv && e == cudaSuccess; ++v)
    timed([&] { return radiation_field_f32(n, d_src, J, c->ws + pl.off_spec, tw, box, l_mfp, c->status, s, nullptr,
                                           nullptr, v); }, &t.fft_ms[v]);
  t.fft_variant = (nv == 2 && t.fft_ms[1] < t.fft_ms[0]) ? 1 : 0;
  // the chosen tiles once more with the TMA-staged z pass
  t.fft_tma_ms = 0.0;
  t.zpass_tma = 0;
  if (n >= 64 && e == cudaSuccess) {
    timed([&] { return radiation_field_f32(n, d_src, J, c->ws + pl.off_spec, tw, box, l_mfp, c->status, s, nullptr,
                                           nullptr, t.fft_variant, nullptr, false, true); }, &t.fft_tma_ms);
    t.zpass_tma = t.fft_tma_ms < 0.98 * t.fft_ms[t.fft_variant] ? 1 : 0;  // a clear win only
  }
  if (e == cudaSuccess)
    e = radiation_field_f32(n, d_src, J, c->ws + pl.off_spec, tw, box, l_mfp, c->status, s, nullptr, nullptr,
                            t.fft_variant, nullptr, false, t.zpass_tma != 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Jkeep, J, (size_t)C * sizeof(float), cudaMemcpyDeviceToDevice, s);
  static const int cand[4][2] = {{9, 0}, {9, 1}, {8, 0}, {8, 1}};
  int best = 0;
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
    timed([&] {
      cudaError_t r = cudaMemcpyAsync(J, Jkeep, (size_t)C * sizeof(float), cudaMemcpyDeviceToDevice, s);
      if (r == cudaSuccess)
        r = rank_impl<float>(c->sortw, J, C, nullptr, d_mass, nullptr, tile_mass, false, c->status, s, nullptr,
                             kSpinLimit, cand[k][0], cand[k][1]);
      return r;
    }, &t.sort_ms[k]);
    if (t.sort_ms[k] < t.sort_ms[best]) best = k;
  }
  t.sort_digit_bits = cand[best][0];
  t.sort_match = cand[best][1];
  t.tuned = 1;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->prof.on = prof_on;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return AMBER_ERR_CUDA;
  }
  c->tune[lg] = t;
  if (out) *out = t;
  return AMBER_OK;
}

int amber_solve(amber_ctx* c, const float* d_src, const float* d_mass, const amber_params_t* p, float* d_zre,
                float* d_J_opt, void* stream) {
  HistoryCoeffs hc;
  int st = solve_args(c, d_src, d_mass, p, d_zre, 32, c ? c->plan.n32 : 0, &hc);
  if (st) return st;
  if (!all_aligned(d_J_opt)) return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(solve_f32_enqueue(c, d_src, d_mass, p, hc, d_zre, d_J_opt, nullptr, nullptr, s));
}

int amber_solve_host(amber_ctx* c, const float* h_src, const float* h_mass, const amber_params_t* p, float* h_zre,
                     void* stream) {
  HistoryCoeffs hc;
  int st = solve_args(c, h_src, h_mass, p, h_zre, 32, c ? c->plan.n32 : 0, &hc);
  if (st) return st;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const size_t bytes = (size_t)p->n * p->n * p->n * sizeof(float);
  // device copies in workspace that is free when they are live: the source in
  // the second index array (read by the forward x pass, first written by the
  // second digit pass), the masses in the second mass array (read by the
  // first digit pass, first written by the second), z_re in the transform
  // buffer (free once the inverse x pass has run)
  float* dS = reinterpret_cast<float*>(c->sortw.idxB);
  float* dM = c->sortw.massB;
  float* dZ = reinterpret_cast<float*>(c->ws + c->plan.off_spec);
  cudaError_t e = cudaMemcpyAsync(dS, h_src, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dM, h_mass, bytes, cudaMemcpyHostToDevice, s);
  {
    // the solve waits for the previous host-buffer solve on this device
    // (enqueued after this call's copies in, which need not wait)
    std::lock_guard<std::mutex> glk(g_host_solve_mu);
    amber_ctx*& last = g_last_host_solve[c->device < 64 ? c->device : 63];
    if (e == cudaSuccess && last && last != c) e = cudaStreamWaitEvent(s, last->host_solve_done, 0);
    if (e == cudaSuccess) e = solve_f32_enqueue(c, dS, dM, p, hc, dZ, nullptr, nullptr, nullptr, s);
    if (e == cudaSuccess) e = cudaEventRecord(c->host_solve_done, s);
    if (e == cudaSuccess) last = c;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_zre, dZ, bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) cudaGetLastError();
  return cuda_status(e);
}

int amber_autotune(amber_ctx* c, const float* d_src, const float* d_mass, int n, double box, double l_mfp,
                   amber_tuning_t* out, void* stream) {
  const int st = rf_args_ok(c, d_src, n, box, l_mfp, d_src, c ? c->plan.n32 : 0);
  if (st) return st;
  if (!d_mass) return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  c->last_stream = (cudaStream_t)stream;
  return autotune_locked(c, d_src, d_mass, n, box, l_mfp, out, (cudaStream_t)stream);
}

int amber_set_tuning(amber_ctx* c, const amber_tuning_t* t) {
  if (!c || !t || !is_pow2_in(t->n, 4, 1024) || t->n > c->plan.n32) return AMBER_ERR_INVALID_ARG;
  if (t->fft_variant < 0 || t->fft_variant > (t->n >= 128 ? 1 : 0)) return AMBER_ERR_INVALID_ARG;
  if ((t->sort_digit_bits != 8 && t->sort_digit_bits != 9) || (t->sort_match != 0 && t->sort_match != 1) ||
      (t->fuse_histogram != 0 && t->fuse_histogram != 1) || (t->zpass_tma != 0 && t->zpass_tma != 1))
    return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  c->tune[ilog2i(t->n)] = *t;
  return AMBER_OK;
}

int amber_get_tuning(amber_ctx* c, int n, amber_tuning_t* out) {
  if (!c || !out || !is_pow2_in(n, 4, 1024)) return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  *out = c->tune[ilog2i(n)];
  return AMBER_OK;
}

int amber_solve_tomographic(amber_ctx* c, const float* const* d_src_list, int nint, const double* z_bounds,
                            const float* d_mass, const amber_params_t* p, float* d_zre, void* stream) {
  if (!d_src_list || !z_bounds || nint < 1 || nint > 64) return AMBER_ERR_INVALID_ARG;
  for (int k = 0; k < nint; ++k)
    if (!d_src_list[k]) return AMBER_ERR_INVALID_ARG;
  for (int k = 0; k <= nint; ++k)
    if (!std::isfinite(z_bounds[k]) || (k && !(z_bounds[k] < z_bounds[k - 1]))) return AMBER_ERR_INVALID_ARG;
  HistoryCoeffs hc;
  int st = solve_args(c, d_src_list[0], d_mass, p, d_zre, 32, c ? c->plan.n32 : 0, &hc);
  if (st) return st;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const Plan& pl = c->plan;
  const int n = p->n;
  const int64_t C = (int64_t)n * n * n;
  float* J = reinterpret_cast<float*>(c->sortw.keysB);
  // the transform buffer is free once J is formed: it holds each interval's matching
  float* ztmp = reinterpret_cast<float*>(c->ws + pl.off_spec);
  unsigned long long* tile_mass = reinterpret_cast<unsigned long long*>(c->ws + pl.off_tilemass);
  cudaError_t e = tomo_fill(d_zre, C, c->num_sms, s);
  for (int k = 0; k < nint && e == cudaSuccess; ++k) {
    // the inverse x pass folds this interval's key range into the sort control
    e = sort_ctrl_reset(c->sortw.ctrl, s);
    if (e == cudaSuccess)
      e = radiation_field_f32(n, d_src_list[k], J, c->ws + pl.off_spec, c->ws + pl.off_tw32 + pl.tw32_off[ilog2i(n)],
                              p->box, p->l_mfp, c->status, s, &c->prof, c->sortw.ctrl,
                              c->tune[ilog2i(n)].fft_variant, nullptr, false, c->tune[ilog2i(n)].zpass_tma != 0);
    if (e == cudaSuccess && k > 0) e = tomo_mask(J, d_zre, C, c->sortw.ctrl, c->num_sms, s);
    if (e == cudaSuccess)
      e = rank_impl<float>(c->sortw, J, C, nullptr, d_mass, nullptr, tile_mass, true, c->status, s, &c->prof,
                           kSpinLimit, c->tune[ilog2i(n)].sort_digit_bits, c->tune[ilog2i(n)].sort_match);
    if (e == cudaSuccess)
      e = assign_impl(c->assw, c->sortw.idxA, c->sortw.massA, true, tile_mass, C, hc, ztmp, nullptr, c->status, s,
                      &c->prof, kSpinLimit, c->sortw.idxB, c->sortw.massB, &c->sortw.ctrl->npasses);
    if (e == cudaSuccess) e = tomo_merge(d_zre, ztmp, C, (float)z_bounds[k + 1], k == nint - 1, c->num_sms, s);
  }
  return cuda_status(e);
}

int amber_solve_ex(amber_ctx* c, const float* d_src, const float* d_mass, const amber_params_t* p, float* d_zre,
                   float* d_J_opt, uint32_t* d_order_out, float* d_mass_rank_out, void* stream) {
  HistoryCoeffs hc;
  int st = solve_args(c, d_src, d_mass, p, d_zre, 32, c ? c->plan.n32 : 0, &hc);
  if (st) return st;
  if (!d_order_out || !d_mass_rank_out || !all_aligned(d_J_opt, d_order_out, d_mass_rank_out))
    return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(solve_f32_enqueue(c, d_src, d_mass, p, hc, d_zre, d_J_opt, d_order_out, d_mass_rank_out, s));
}

int amber_spectrum_bytes(int n, size_t* out_bytes) {
  if (!out_bytes || !is_pow2_in(n, 4, 1024)) return AMBER_ERR_INVALID_ARG;
  *out_bytes = (size_t)n * n * (n / 2 + 2) * 8;
  return AMBER_OK;
}

int amber_source_spectrum(amber_ctx* c, const float* d_src, int n, void* d_spec, void* stream) {
  if (!c || !d_src || !d_spec || !is_pow2_in(n, 4, 1024) || !all_aligned(d_src) ||
      (reinterpret_cast<uintptr_t>(d_spec) & 15) != 0)
    return AMBER_ERR_INVALID_ARG;
  if (n > c->plan.n32) return AMBER_ERR_CAPACITY;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const int l = ilog2i(n);
  return cuda_status(source_spectrum_f32(n, d_src, d_spec, c->ws + c->plan.off_tw32 + c->plan.tw32_off[l], s,
                                         &c->prof, c->tune[l].fft_variant));
}

int amber_solve_spectrum(amber_ctx* c, const void* d_spec, const float* d_mass, const amber_params_t* p, float* d_zre,
                         float* d_J_opt, uint32_t* d_order_out, float* d_mass_rank_out, void* stream) {
  if (!d_spec || (reinterpret_cast<uintptr_t>(d_spec) & 15) != 0) return AMBER_ERR_INVALID_ARG;
  HistoryCoeffs hc;
  // the spectrum stands in for the source field in the argument checks
  int st = solve_args(c, static_cast<const float*>(d_spec), d_mass, p, d_zre, 32, c ? c->plan.n32 : 0, &hc);
  if (st) return st;
  if ((d_order_out == nullptr) != (d_mass_rank_out == nullptr) || !all_aligned(d_J_opt, d_order_out, d_mass_rank_out))
    return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(solve_f32_enqueue(c, nullptr, d_mass, p, hc, d_zre, d_J_opt, d_order_out, d_mass_rank_out, s,
                                       d_spec));
}

int amber_assign_zre_ranked(amber_ctx* c, const uint32_t* d_order, const float* d_mass_rank, int64_t ncells,
                            const amber_history_t* h, float* d_zre, double* d_F_opt, void* stream) {
  if (!c || !d_order || !d_mass_rank || !d_zre || ncells < 1 || !all_aligned(d_order, d_mass_rank, d_zre, d_F_opt))
    return AMBER_ERR_INVALID_ARG;
  if (ncells > c->max_cells) return AMBER_ERR_CAPACITY;
  HistoryCoeffs hc;
  const int st = history_coeffs(h, &hc);
  if (st) return st;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(assign_impl(c->assw, d_order, d_mass_rank, true, nullptr, ncells, hc, d_zre, d_F_opt, c->status,
                                 s, &c->prof, kSpinLimit));
}

// ---------------------------------------------------------------------------
// Batched solves: every stage of every item in one launch per stage (per grid
// size for the transforms, per digit width for the sort), captured once.
// ---------------------------------------------------------------------------
struct amber_batch {
  int device = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<amber_ctx*> ctxs;
  unsigned char* ws = nullptr;    // the batch's own workspace (all items at once)
  unsigned char* args = nullptr;  // the items' kernel arguments
  int kernel_nodes = 0;
};


int amber_batch_create(amber_batch** out, amber_ctx* const* ctxs, int nctx, const amber_batch_item* items,
                       int nitems) {
  if (!out || !ctxs || nctx < 1 || !items || nitems < 1) return AMBER_ERR_INVALID_ARG;
  *out = nullptr;
  amber_ctx* c0 = ctxs[0];
  for (int k = 0; k < nctx; ++k)
    if (!ctxs[k] || ctxs[k]->device != (c0 ? c0->device : -1)) return AMBER_ERR_INVALID_ARG;
  std::vector<HistoryCoeffs> hcs(nitems);
  for (int i = 0; i < nitems; ++i) {
    const int st = solve_args(c0, items[i].d_src, items[i].d_mass, &items[i].params, items[i].d_zre, 32,
                              c0->plan.n32, &hcs[i]);
    if (st) return st;
    if (items[i].params.n < 8) return AMBER_ERR_INVALID_ARG;  // x-pass tiles span whole items from 8^3 up
  }
  std::lock_guard<std::mutex> lk(c0->mu);
  DeviceGuard g(c0->device);
  // each size not yet tuned: autotune on its first item
  for (int i = 0; i < nitems && autotune_enabled(); ++i) {
    const int n = items[i].params.n, lg = ilog2i(n);
    if (c0->tune[lg].tuned) continue;
    const int st = autotune_locked(c0, items[i].d_src, items[i].d_mass, n, items[i].params.box,
                                   items[i].params.l_mfp, nullptr, nullptr);
    if (st) return st;
  }
  // every context of the batch carries the choices the batch runs with
  for (int k = 1; k < nctx; ++k) {
    if (ctxs[k] == c0) continue;
    std::lock_guard<std::mutex> lk2(ctxs[k]->mu);
    for (int i = 0; i < nitems; ++i) {
      const int lg = ilog2i(items[i].params.n);
      ctxs[k]->tune[lg] = c0->tune[lg];
    }
  }
  // items ordered by grid size: one size's spectra and intensities lie back to back
  std::vector<int> ord(nitems);
  for (int i = 0; i < nitems; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return items[a].params.n < items[b].params.n; });

  // ---- workspace plan
  Layout L;
  struct ItemWs {
    int64_t C;
    size_t J, kA, iA, iB, mA, mB, spec, lb, actrl, Xq, inv, lin, state, btab, tmass;
    int64_t sort_tiles, scan_tiles;
    int nbuckets;
  };
  std::vector<ItemWs> iw(nitems);
  int64_t cells = 0;
  for (int i : ord) cells += (int64_t)items[i].params.n * items[i].params.n * items[i].params.n;
  // per-cell arrays: one run per kind, items in size order
  const size_t offJ = L.take(cells * 4), offKA = L.take(cells * 4), offIA = L.take(cells * 4),
               offIB = L.take(cells * 4), offMA = L.take(cells * 4), offMB = L.take(cells * 4);
  size_t spec_total = 0;
  for (int i : ord) {
    const int n = items[i].params.n;
    spec_total += (size_t)n * n * (n / 2 + 2) * 8;
  }
  const size_t offSpec = L.take(spec_total);
  const size_t offCtrl = L.take((size_t)nitems * sizeof(SortCtrl));  // one control block per item, in size order
  const size_t offACtrl = L.take((size_t)nitems * kAssignCtrlBytes);
  {
    int64_t co = 0;
    size_t so = 0;
    for (int i : ord) {
      const int n = items[i].params.n;
      ItemWs& w = iw[i];
      w.C = (int64_t)n * n * n;
      w.J = offJ + co * 4;
      w.kA = offKA + co * 4;
      w.iA = offIA + co * 4;
      w.iB = offIB + co * 4;
      w.mA = offMA + co * 4;
      w.mB = offMB + co * 4;
      w.spec = offSpec + so;
      co += w.C;
      so += (size_t)n * n * (n / 2 + 2) * 8;
    }
  }
  size_t state_total = 0;
  for (int i : ord) {
    ItemWs& w = iw[i];
    w.sort_tiles = sort_tiles(w.C);
    w.scan_tiles = (w.C + kScanTile - 1) / kScanTile;
    int shift;
    bucket_plan(w.C, &w.nbuckets, &shift);
    state_total += align256((size_t)w.scan_tiles * 8);
  }
  const size_t offState = L.take(state_total);  // scan look-back words of every item (one memset)
  {
    size_t so = 0;
    for (int i : ord) {
      ItemWs& w = iw[i];
      w.state = offState + so;
      so += align256((size_t)w.scan_tiles * 8);
      w.lb = L.take(2 * sort_lookback_words(w.C) * 4);
      w.Xq = L.take((size_t)hcs[i].n_table * 8);
      w.inv = L.take((size_t)hcs[i].n_table * 4);
      w.lin = L.take((size_t)4 * kMaxTable * 4);
      w.btab = L.take((size_t)w.scan_tiles * (w.nbuckets + 1) * 2);
      w.tmass = L.take((size_t)w.sort_tiles * 16);
    }
  }
  // per-item argument arrays (device copies of host-built structs)
  std::vector<int> sizes, rbs;
  for (int i : ord) {
    const int n = items[i].params.n;
    if (sizes.empty() || sizes.back() != n) sizes.push_back(n);
  }
  for (int n : sizes) {
    const int rb = c0->tune[ilog2i(n)].sort_digit_bits;
    if (std::find(rbs.begin(), rbs.end(), rb) == rbs.end()) rbs.push_back(rb);
  }
  amber_batch* b = new (std::nothrow) amber_batch();
  if (!b) return AMBER_ERR_OOM;
  b->device = c0->device;
  b->ctxs.assign(ctxs, ctxs + nctx);
  if (cudaMalloc(&b->ws, L.total) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return AMBER_ERR_OOM;
  }
  unsigned char* W = b->ws;
  // the argument arrays hold addresses in W; they are laid out here, then
  // copied to a second allocation once complete
  Layout A;
  std::vector<HostBlob> blobs;
  auto place = [&](auto vec) -> size_t {
    HostBlob hb;
    hb.set(vec);
    hb.off = A.take(hb.bytes.size() ? hb.bytes.size() : 16);
    blobs.push_back(std::move(hb));
    return blobs.back().off;
  };

  SortCtrl* ctrl_base = reinterpret_cast<SortCtrl*>(W + offCtrl);
  std::vector<SortWork> sw(nitems);
  std::vector<AssignWork> aw(nitems);
  std::vector<int> pos(nitems);  // position of item i in size order
  for (int k = 0; k < nitems; ++k) pos[ord[k]] = k;
  for (int i = 0; i < nitems; ++i) {
    const ItemWs& w = iw[i];
    SortWork& s = sw[i];
    s.keysA = W + w.kA;
    s.keysB = W + w.J;  // the intensity, dead after the first digit pass
    s.idxA = reinterpret_cast<uint32_t*>(W + w.iA);
    s.idxB = reinterpret_cast<uint32_t*>(W + w.iB);
    s.massA = reinterpret_cast<float*>(W + w.mA);
    s.massB = reinterpret_cast<float*>(W + w.mB);
    s.lookback = reinterpret_cast<uint32_t*>(W + w.lb);
    s.ctrl = ctrl_base + pos[i];
    s.max_cells = w.C;
    s.num_sms = c0->num_sms;
    AssignWork& a = aw[i];
    a.ctrl = W + offACtrl + (size_t)pos[i] * kAssignCtrlBytes;
    a.Xq = reinterpret_cast<unsigned long long*>(W + w.Xq);
    a.inv_dx = reinterpret_cast<float*>(W + w.inv);
    a.lin = reinterpret_cast<float*>(W + w.lin);
    a.state = reinterpret_cast<unsigned long long*>(W + w.state);
    a.bcell = reinterpret_cast<uint32_t*>(s.keysA);
    a.bz = reinterpret_cast<float*>(s.keysB);
    a.btab = reinterpret_cast<uint16_t*>(W + w.btab);
    a.num_sms = c0->num_sms;
  }

  // ---- transforms: per size, the sources, kf and l_mfp of its items
  struct FftGroup { int n, M, first; size_t srcs, kp; };
  std::vector<FftGroup> fg;
  for (int n : sizes) {
    FftGroup f{n, 0, -1, 0, 0};
    std::vector<const float*> srcs;
    std::vector<float> kp;
    for (int k = 0; k < nitems; ++k) {
      const int i = ord[k];
      if (items[i].params.n != n) continue;
      if (f.first < 0) f.first = i;
      ++f.M;
      srcs.push_back(items[i].d_src);
      kp.push_back((float)(2.0 * 3.14159265358979323846 / items[i].params.box));
      kp.push_back((float)items[i].params.l_mfp);
    }
    f.srcs = place(srcs);
    f.kp = place(kp);
    fg.push_back(f);
  }
  // ---- sort: per digit width, the items' histogram and pass arguments
  struct SortGroup { int rb, match; RankMulti r; size_t hist, hpre, pass[4], tpre; };
  std::vector<SortGroup> sg;
  std::vector<unsigned long long*> tile_mass(nitems);
  for (int i = 0; i < nitems; ++i) tile_mass[i] = reinterpret_cast<unsigned long long*>(W + iw[i].tmass);
  for (int rb : rbs) {
    SortGroup q{};
    q.rb = rb;
    std::vector<HistArgs> hist;
    std::vector<uint32_t> hpre{0}, tpre{0};
    std::vector<PassArgs> pass[4];
    for (int k = 0; k < nitems; ++k) {
      const int i = ord[k];
      const amber_tuning_t& tu = c0->tune[ilog2i(items[i].params.n)];
      if (tu.sort_digit_bits != rb) continue;
      q.match = tu.sort_match;
      HistArgs h;
      uint32_t hb;
      PassArgs pa[4];
      const int P = rank_args<float>(sw[i], reinterpret_cast<const float*>(sw[i].keysB), iw[i].C, nullptr,
                                     items[i].d_mass, nullptr, tile_mass[i], c0->status, kSpinLimit, rb, &h, &hb, pa);
      for (int p = 0; p < 4; ++p) pass[p].push_back(pa[p < P ? p : P - 1]);
      hist.push_back(h);
      hpre.push_back(hpre.back() + hb);
      tpre.push_back(tpre.back() + (uint32_t)iw[i].sort_tiles);
    }
    q.r.M = (int)hist.size();
    q.r.hist_blocks = hpre.back();
    q.r.tiles = tpre.back();
    q.hist = place(hist);
    q.hpre = place(hpre);
    for (int p = 0; p < 4; ++p) q.pass[p] = place(pass[p]);
    q.tpre = place(tpre);
    sg.push_back(q);
  }
  // ---- matching: thresholds and scatter for every item, scans per weighting form
  AssignMulti am{};
  size_t o_thresh, o_scan[2], o_spre[2], o_scatter, o_xpre;
  {
    std::vector<ThreshArgs> th;
    std::vector<ScanArgs> sc[2];
    std::vector<uint32_t> spre[2] = {{0}, {0}}, xpre{0};
    std::vector<ScatterArgs> xs;
    for (int k = 0; k < nitems; ++k) {
      const int i = ord[k];
      ThreshArgs ta;
      ScanArgs sa;
      ScatterArgs xa;
      assign_args(aw[i], sw[i].idxA, sw[i].massA, tile_mass[i], iw[i].C, hcs[i], items[i].d_zre, nullptr, c0->status,
                  kSpinLimit, sw[i].idxB, sw[i].massB, &sw[i].ctrl->npasses, &ta, &sa, &xa);
      th.push_back(ta);
      const int f = hcs[i].weighting != AMBER_WEIGHT_MASS ? 1 : 0;
      sc[f].push_back(sa);
      spre[f].push_back(spre[f].back() + (uint32_t)iw[i].scan_tiles);
      xs.push_back(xa);
      xpre.push_back(xpre.back() + (uint32_t)(xa.groups * xa.nbuckets));
    }
    am.M = nitems;
    for (int f = 0; f < 2; ++f) {
      am.Mg[f] = (int)sc[f].size();
      am.scan_tiles[f] = spre[f].back();
      o_scan[f] = place(sc[f]);
      o_spre[f] = place(spre[f]);
    }
    am.scatter_blocks = xpre.back();
    o_thresh = place(th);
    o_scatter = place(xs);
    o_xpre = place(xpre);
  }
  cudaError_t e = cudaMalloc(&b->args, A.total);
  unsigned char* G = b->args;
  for (const HostBlob& hb : blobs)
    if (e == cudaSuccess && !hb.bytes.empty()) e = cudaMemcpy(G + hb.off, hb.bytes.data(), hb.bytes.size(),
                                                               cudaMemcpyHostToDevice);
  am.thresh = reinterpret_cast<const ThreshArgs*>(G + o_thresh);
  for (int f = 0; f < 2; ++f) {
    am.scan[f] = reinterpret_cast<const ScanArgs*>(G + o_scan[f]);
    am.scan_prefix[f] = reinterpret_cast<const uint32_t*>(G + o_spre[f]);
  }
  am.scatter = reinterpret_cast<const ScatterArgs*>(G + o_scatter);
  am.scatter_prefix = reinterpret_cast<const uint32_t*>(G + o_xpre);
  for (SortGroup& q : sg) {
    q.r.hist = reinterpret_cast<const HistArgs*>(G + q.hist);
    q.r.hist_prefix = reinterpret_cast<const uint32_t*>(G + q.hpre);
    for (int p = 0; p < 4; ++p) q.r.pass[p] = reinterpret_cast<const PassArgs*>(G + q.pass[p]);
    q.r.tile_prefix = reinterpret_cast<const uint32_t*>(G + q.tpre);
  }

  // ---- capture: every stage once
  const bool prof_on = c0->prof.on;
  c0->prof.on = false;
  cudaStream_t origin = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
  bool capturing = false;
  if (e == cudaSuccess) {
    e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed);
    capturing = e == cudaSuccess;
  }
  // sort control blocks: zero, key minimum at its largest value (the inverse
  // x passes fold each item's key range in)
  if (e == cudaSuccess) e = cudaMemsetAsync(W + offCtrl, 0, (size_t)nitems * sizeof(SortCtrl), origin);
  if (e == cudaSuccess)
    e = cudaMemset2DAsync(W + offCtrl, sizeof(SortCtrl), 0xff, sizeof(unsigned long long), nitems, origin);
  for (const FftGroup& f : fg) {
    if (e != cudaSuccess) break;
    const int l = ilog2i(f.n);
    e = radiation_field_multi_f32(f.n, c0->tune[l].fft_variant, reinterpret_cast<const float* const*>(G + f.srcs), f.M,
                                  reinterpret_cast<float*>(W + iw[f.first].J), W + iw[f.first].spec,
                                  c0->ws + c0->plan.off_tw32 + c0->plan.tw32_off[l],
                                  reinterpret_cast<const float*>(G + f.kp), c0->status, origin, sw[f.first].ctrl);
  }
  for (const SortGroup& q : sg)
    if (e == cudaSuccess) e = rank_multi(q.r, q.rb, q.match == 1, origin);
  if (e == cudaSuccess) e = cudaMemsetAsync(W + offACtrl, 0, (size_t)nitems * kAssignCtrlBytes, origin);
  if (e == cudaSuccess) e = cudaMemsetAsync(W + offState, 0, state_total, origin);
  if (e == cudaSuccess) e = assign_multi(am, origin);
  if (capturing) {
    const cudaError_t e2 = cudaStreamEndCapture(origin, &b->graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e == cudaSuccess) {
    size_t nn = 0;
    cudaGraphGetNodes(b->graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(b->graph, nodes.data(), &nn);
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++b->kernel_nodes;
    }
  }
  c0->prof.on = prof_on;
  if (origin) cudaStreamDestroy(origin);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->ws);
    if (b->args) cudaFree(b->args);
    delete b;
    return AMBER_ERR_CUDA;
  }
  *out = b;
  return AMBER_OK;
}

int amber_batch_launch(amber_batch* b, void* stream) {
  if (!b) return AMBER_ERR_INVALID_ARG;
  DeviceGuard g(b->device);
  for (auto* c : b->ctxs) c->last_stream = (cudaStream_t)stream;
  return cuda_status(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

int amber_batch_kernel_nodes(amber_batch* b, int* out_nodes) {
  if (!b || !out_nodes) return AMBER_ERR_INVALID_ARG;
  *out_nodes = b->kernel_nodes;
  return AMBER_OK;
}

int amber_batch_destroy(amber_batch* b) {
  if (!b) return AMBER_ERR_INVALID_ARG;
  {
    DeviceGuard g(b->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ws) cudaFree(b->ws);
    if (b->args) cudaFree(b->args);
  }
  delete b;
  return AMBER_OK;
}

int amber_solve_f64(amber_ctx* c, const double* d_src, const float* d_mass, const amber_params_t* p, float* d_zre,
                    double* d_J_opt, void* stream) {
  HistoryCoeffs hc;
  int st = solve_args(c, d_src, d_mass, p, d_zre, 64, c ? c->plan.n64 : 0, &hc);
  if (st) return st;
  if (!all_aligned(d_J_opt)) return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const Plan& pl = c->plan;
  const int n = p->n;
  const int64_t C = (int64_t)n * n * n;
  double* J = d_J_opt ? d_J_opt : reinterpret_cast<double*>(c->sortw.keysB);
  cudaError_t e = sort_ctrl_reset(c->sortw.ctrl, s);
  if (e == cudaSuccess)
    e = radiation_field_f64(n, d_src, J, c->ws + pl.off_spec, c->ws + pl.off_tw64 + pl.tw64_off[ilog2i(n)], p->box,
                           p->l_mfp, c->status, s, &c->prof, c->sortw.ctrl);
  unsigned long long* tile_mass = reinterpret_cast<unsigned long long*>(c->ws + pl.off_tilemass);
  if (e == cudaSuccess)
    e = rank_impl<double>(c->sortw, J, C, nullptr, d_mass, nullptr, tile_mass, true, c->status, s, &c->prof,
                          kSpinLimit);
  // the order and rank-order masses sit on the A or B side by pass parity
  if (e == cudaSuccess)
    e = assign_impl(c->assw, c->sortw.idxA, c->sortw.massA, true, tile_mass, C, hc, d_zre, nullptr, c->status, s,
                    &c->prof, kSpinLimit, c->sortw.idxB, c->sortw.massB, &c->sortw.ctrl->npasses);
  return cuda_status(e);
}

int amber_sync_status(amber_ctx* c, void* stream) {
  if (!c) return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(c->h_status, c->status, sizeof(unsigned int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemsetAsync(c->status, 0, sizeof(unsigned int), s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return AMBER_ERR_CUDA;
  }
  return (int)*c->h_status;
}

const char* amber_status_string(int code) {
  switch (code) {
    case AMBER_OK: return "ok";
    case AMBER_ERR_INVALID_ARG: return "invalid argument";
    case AMBER_ERR_NO_SOLUTION: return "no Weibull solution with positive coefficients";
    case AMBER_ERR_NONFINITE: return "non-finite intensity";
    case AMBER_ERR_OOM: return "device workspace allocation failed";
    case AMBER_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case AMBER_ERR_CUDA: return "CUDA runtime error";
    case AMBER_ERR_INVALID_MASS: return "invalid cell mass";
    case AMBER_ERR_CAPACITY: return "size exceeds context capacity";
    default: return "multiple or unknown status bits";
  }
}

int amber_profile_enable(amber_ctx* c, int on) {
  if (!c) return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  if (on && c->prof.pool.empty()) {
    c->prof.pool.resize(8192);
    for (auto& e : c->prof.pool)
      if (cudaEventCreate(&e) != cudaSuccess) return AMBER_ERR_CUDA;
  }
  c->prof.on = on != 0;
  return AMBER_OK;
}

int amber_profile_reset(amber_ctx* c) {
  if (!c) return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  prof_harvest(&c->prof);
  for (int k = 0; k < PK_COUNT; ++k) { c->prof.total_ms[k] = 0.0; c->prof.launches[k] = 0; }
  return AMBER_OK;
}

int amber_profile_kinds(void) { return PK_COUNT; }

int amber_struct_layout(int which, size_t* size, size_t* offsets, int max_offsets, int* count) {
  if (!size || !count) return AMBER_ERR_INVALID_ARG;
  size_t off[16];
  int k = 0;
  switch (which) {
    case 0:
      *size = sizeof(amber_history_t);
      for (size_t o : {offsetof(amber_history_t, z_mid), offsetof(amber_history_t, dz), offsetof(amber_history_t, Az),
                       offsetof(amber_history_t, x_ear), offsetof(amber_history_t, x_mid),
                       offsetof(amber_history_t, x_lat), offsetof(amber_history_t, z_lo),
                       offsetof(amber_history_t, z_hi), offsetof(amber_history_t, n_table),
                       offsetof(amber_history_t, weighting), offsetof(amber_history_t, omega_m)})
        off[k++] = o;
      break;
    case 1:
      *size = sizeof(amber_params_t);
      for (size_t o : {offsetof(amber_params_t, n), offsetof(amber_params_t, box), offsetof(amber_params_t, l_mfp),
                       offsetof(amber_params_t, hist), offsetof(amber_params_t, precision)})
        off[k++] = o;
      break;
    case 2:
      *size = sizeof(amber_tuning_t);
      for (size_t o : {offsetof(amber_tuning_t, n), offsetof(amber_tuning_t, fft_variant),
                       offsetof(amber_tuning_t, sort_digit_bits), offsetof(amber_tuning_t, sort_match),
                       offsetof(amber_tuning_t, tuned), offsetof(amber_tuning_t, fft_ms),
                       offsetof(amber_tuning_t, sort_ms), offsetof(amber_tuning_t, fuse_histogram),
                       offsetof(amber_tuning_t, zpass_tma), offsetof(amber_tuning_t, fft_tma_ms)})
        off[k++] = o;
      break;
    case 3:
      *size = sizeof(amber_batch_item);
      for (size_t o : {offsetof(amber_batch_item, d_src), offsetof(amber_batch_item, d_mass),
                       offsetof(amber_batch_item, params), offsetof(amber_batch_item, d_zre)})
        off[k++] = o;
      break;
    default:
      return AMBER_ERR_INVALID_ARG;
  }
  *count = k;
  for (int i = 0; i < k && i < max_offsets && offsets; ++i) offsets[i] = off[i];
  return AMBER_OK;
}

int amber_profile_read(amber_ctx* c, int kind, const char** name, double* total_ms, int64_t* launches) {
  if (!c || kind < 0 || kind >= PK_COUNT) return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  prof_harvest(&c->prof);
  if (name) *name = kProfNames[kind];
  if (total_ms) *total_ms = c->prof.total_ms[kind];
  if (launches) *launches = c->prof.launches[kind];
  return AMBER_OK;
}

int amber_source_field(amber_ctx* c, const float* d_delta, int64_t ncells, double delta_c, double sigma_f,
                       float* d_S, float* d_mass_opt, void* stream) {
  if (!c || !d_delta || !d_S || ncells < 1 || !std::isfinite(delta_c) || !(sigma_f > 0.0) || !std::isfinite(sigma_f))
    return AMBER_ERR_INVALID_ARG;
  if (!all_aligned(d_delta, d_S, d_mass_opt)) return AMBER_ERR_INVALID_ARG;
  if (ncells > c->max_cells) return AMBER_ERR_CAPACITY;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  return cuda_status(source_field_impl(d_delta, ncells, delta_c, sigma_f, d_S, d_mass_opt,
                                       reinterpret_cast<unsigned long long*>(c->ws + c->plan.off_srcsum), c->num_sms,
                                       c->status, s));
}

int amber_sort_passes(amber_ctx* c, int* out_passes) {
  if (!c || !out_passes) return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  int np = 0;
  if (cudaStreamSynchronize(c->last_stream) != cudaSuccess ||
      cudaMemcpy(&np, &c->sortw.ctrl->npasses, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return AMBER_ERR_CUDA;
  }
  *out_passes = np;
  return AMBER_OK;
}

int amber_test_wait_timeout(amber_ctx* c, unsigned int spin_limit, void* stream) {
  if (!c || spin_limit < 1) return AMBER_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* word = reinterpret_cast<uint32_t*>(c->ws + c->plan.off_status + 64);
  return cuda_status(wait_timeout_test(word, c->status, spin_limit, s));
}

}  // extern "C"

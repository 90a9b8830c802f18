// wo_api.cu - the C ABI declared in include/wo.h: argument validation,
// workspace layout and the sequence of kernel passes for each entry point.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "wo_internal.h"

namespace wo {

// ------------------------------------------------------------ profiling
namespace {
struct Pending {
  const char* name;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_prof = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
std::atomic<long long> g_launches{0};

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

void prof_begin(const char* name, cudaStream_t s, int* token) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  *token = -1;
  if (!g_prof) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Pending p{name, take_event(), take_event()};
  if (!p.a || !p.b) return;
  cudaEventRecord(p.a, s);
  g_pending.push_back(p);
  *token = (int)g_pending.size() - 1;
}

void prof_end(int token, cudaStream_t s) {
  if (token < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (token < (int)g_pending.size()) cudaEventRecord(g_pending[token].b, s);
}

// ------------------------------------------------------------ sizes
static bool size_ok(int n) {
  if (n < 1 || n > 2048) return false;
  int m = n;
  if (m % 3 == 0) m /= 3;
  return (m & (m - 1)) == 0;
}

struct Sys {
  int n_kinds, lf_props, has_fl, C, P, n_arms;
  int want_phase, want_abs, want_dz, planes, want_grad, smooth;
  int kxm;    // kx-major bank (WO_TF_KX_MAJOR)
  int aberr;  // aberrated detection pupil (wo_build_tf_aberrated): set by the caller, not by kinds
};

static Sys system_of(unsigned kinds) {
  Sys s{};
  s.want_phase = (kinds & WO_TF_PHASE) ? 1 : 0;
  s.want_abs = (kinds & WO_TF_ABSORPTION) ? 1 : 0;
  s.has_fl = (kinds & WO_TF_FLUOR) ? 1 : 0;
  s.lf_props = s.want_phase + s.want_abs;
  s.n_kinds = s.lf_props + s.has_fl;
  s.C = (s.lf_props ? 1 : 0) + s.has_fl;
  s.P = s.n_kinds;
  s.n_arms = (s.lf_props ? 2 : 0) + s.has_fl;
  s.smooth = (kinds & WO_TF_SMOOTH_SOURCE) ? 1 : 0;
  s.kxm = (kinds & WO_TF_KX_MAJOR) ? 1 : 0;
  const unsigned core = kinds & ~(unsigned)(WO_TF_PLANES | WO_TF_SMOOTH_SOURCE | WO_TF_KX_MAJOR);
  if (core == WO_TF_PHASE_GRAD) {  // phase TF and d/d(z0, tilt_x, tilt_y, NA_ill): five slots, seven arms
    s.want_phase = 1;
    s.want_dz = 1;
    s.want_grad = 1;
    s.smooth = 1;
    s.planes = 1;
    s.lf_props = 1;
    s.n_kinds = 5;
    s.C = 1;
    s.P = 1;
    s.n_arms = 7;
    s.want_abs = 0;
    s.has_fl = 0;
    return s;
  }
  if (core == WO_TF_PHASE_DZ) {  // phase TF and d/dz0: two slots, four arms
    s.planes = (kinds & WO_TF_PLANES) ? 1 : 0;
    s.want_phase = 1;
    s.want_dz = 1;
    s.lf_props = 1;
    s.n_kinds = 2;
    s.C = 1;
    s.P = 1;
    s.n_arms = 4;
  }
  return s;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t status, pipe, head;
  size_t optics, zern, counts, rec, rec2, norm_part, norms, arms, build_end;
  size_t specA, specB, op_end;
  size_t total;
  size_t tf_spectra, tf_stats, tf_total;
};

// Every workspace starts with the device status block (kStatusBytes) and the
// tile pipeline's counters; the entry points' regions follow.
static size_t ws_head(int n) { return kStatusBytes + align256(pipe_counter_bytes(n)); }

static Layout layout_of(int n, int Z, int Y, int X, const Sys& s) {
  Layout L{};
  const size_t Xh = (size_t)X / 2 + 1;
  L.status = 0;
  L.pipe = kStatusBytes;
  L.head = ws_head(n);
  size_t off = L.head;
  L.optics = off; off += align256((size_t)n * sizeof(wo_optics));
  L.zern = off; if (s.aberr) off += align256((size_t)n * WO_MAX_ZERNIKE * sizeof(double));
  L.counts = off; off += align256((size_t)n * 4 * sizeof(int));
  L.rec = off; off += align256((size_t)n * Y * X * sizeof(float4));
  L.rec2 = off; if (s.want_grad || s.aberr) off += align256((size_t)n * Y * X * sizeof(float4));
  const int rb = (Y + record_rows(Y, n) - 1) / record_rows(Y, n);
  L.norm_part = off; if (s.smooth) off += align256((size_t)n * rb * 4 * sizeof(float));
  L.norms = off; if (s.smooth) off += align256((size_t)n * 4 * sizeof(float));
  L.arms = off; off += align256((size_t)n * s.n_arms * Z * Y * X * sizeof(float2));
  L.build_end = off;
  const size_t vols = (size_t)(s.C > s.P ? s.C : s.P);
  const size_t spec = align256((size_t)n * vols * Z * Y * Xh * sizeof(float2));
  L.specA = L.head;
  L.specB = L.head + spec;
  L.op_end = L.head + 2 * spec;
  L.total = L.build_end > L.op_end ? L.build_end : L.op_end;
  const size_t tune_end = kStatusBytes + tune_partials_bytes(n, Y, X, 4);
  if (s.want_dz && tune_end > L.total) L.total = tune_end;
  L.tf_spectra = align256((size_t)n * s.n_kinds * Z * Y * Xh * sizeof(float2));
  L.tf_stats = L.tf_spectra;
  L.tf_total = L.tf_spectra + (size_t)n * 8 * sizeof(float);
  return L;
}

static bool aligned16(const void* p) { return p && (((uintptr_t)p) & 15u) == 0; }

// Shared memory of the z kernels: up to three volumes of Z x B columns.
static size_t zpass_smem(int Z) {
  const int NV = 3;
  int B = 16;
  while (B > 1 && (size_t)NV * Z * B * 8 > 64 * 1024) B /= 2;
  return ((size_t)Z + (size_t)2 * NV * Z * B) * sizeof(float2) + 1024 * 11 * sizeof(float);
}

static wo_status check_shape(int n_tiles, int Z, int Y, int X, unsigned kinds) {
  if (n_tiles < 1 || n_tiles > 65535) return WO_ERR_ARG;
  if (kinds & ~255u) return WO_ERR_ARG;
  const bool kxm = (kinds & WO_TF_KX_MAJOR) != 0;
  const unsigned base = kinds & ~(unsigned)(WO_TF_PLANES | WO_TF_SMOOTH_SOURCE | WO_TF_KX_MAJOR);
  // kx-major banks: one kind, 3D TFs
  if (kxm && ((kinds & WO_TF_PLANES) || (base != WO_TF_PHASE && base != WO_TF_ABSORPTION && base != WO_TF_FLUOR)))
    return WO_ERR_ARG;
  if (base == 0) return WO_ERR_ARG;
  if ((base & WO_TF_PHASE_DZ) && base != WO_TF_PHASE_DZ) return WO_ERR_ARG;
  if ((base & WO_TF_PHASE_GRAD) && base != WO_TF_PHASE_GRAD) return WO_ERR_ARG;
  if ((kinds & WO_TF_PLANES) && base != WO_TF_PHASE_DZ && base != WO_TF_PHASE_GRAD) return WO_ERR_ARG;
  if (base == WO_TF_PHASE_GRAD && !(kinds & WO_TF_PLANES)) return WO_ERR_ARG;  // per-plane banks only
  if ((kinds & WO_TF_SMOOTH_SOURCE) && base == WO_TF_FLUOR) return WO_ERR_ARG;  // no source pupil
  if (Z < 1 || Y < 1 || X < 2) return WO_ERR_SHAPE;
  if (X % 2) return WO_ERR_SHAPE;
  if (!size_ok(Z) || !size_ok(Y) || !size_ok(X / 2) || X > 2048) return WO_ERR_UNSUPPORTED_SIZE;
  if (zpass_smem(Z) > 227 * 1024) return WO_ERR_UNSUPPORTED_SIZE;
  // four arm rows of X per PSF-row block must fit shared memory
  if (base == WO_TF_PHASE_DZ && X > 768) return WO_ERR_UNSUPPORTED_SIZE;
  // the seven arms of the gradient bank need the register-resident row pass
  if (base == WO_TF_PHASE_GRAD && !(X == 32 || X == 48 || X == 64 || X == 96 || X == 128 || X == 192 || X == 256))
    return WO_ERR_UNSUPPORTED_SIZE;
  // the plane engine's shapes, and PSF-row and x-pass CTAs whose rows stay inside a plane
  if (kxm && !(plane_supported(Z, Y) && psf_kxm_supported(X, Y, Z) && rows_kxm_supported(X / 2, Y)))
    return WO_ERR_UNSUPPORTED_SIZE;
  return WO_OK;
}

static wo_status check_optics(const wo_optics& o) {
  const double v[9] = {o.lambda_um, o.n_medium, o.pixel_um, o.z_step_um, o.na_det,
                       o.na_ill, o.tilt_x, o.tilt_y, o.defocus_um};
  for (double x : v)
    if (!isfinite(x)) return WO_ERR_OPTICS;
  if (o.lambda_um <= 0 || o.n_medium <= 0 || o.pixel_um <= 0 || o.z_step_um <= 0) return WO_ERR_OPTICS;
  if (o.na_det <= 0 || o.na_det >= o.n_medium) return WO_ERR_OPTICS;
  const double tilt = sqrt(o.tilt_x * o.tilt_x + o.tilt_y * o.tilt_y);
  if (o.na_ill < 0 || o.na_ill + tilt > o.n_medium) return WO_ERR_OPTICS;
  // the pupil correlation must not alias on the transverse grid
  if ((o.na_det + o.na_ill + tilt) / o.lambda_um >= 1.0 / (2.0 * o.pixel_um)) return WO_ERR_UNDERSAMPLED;
  // the axial band of the TFs must fit the z sampling
  const double s = o.na_det / o.n_medium;
  if ((o.n_medium / o.lambda_um) * (1.0 - sqrt(1.0 - s * s)) >= 1.0 / (2.0 * o.z_step_um))
    return WO_ERR_UNDERSAMPLED;
  return WO_OK;
}

static wo_status cuda_status(cudaError_t e) { return e == cudaSuccess ? WO_OK : WO_ERR_CUDA; }


#define WO_TRY(expr)                          \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) return WO_ERR_CUDA; \
  } while (0)

}  // namespace wo

using namespace wo;

extern "C" {

int wo_size_supported(int n) { return size_ok(n) ? 1 : 0; }

size_t wo_tf_bytes(int n_tiles, int Z, int Y, int X, unsigned kinds) {
  if (check_shape(n_tiles, Z, Y, X, kinds) != WO_OK) return 0;
  return layout_of(n_tiles, Z, Y, X, system_of(kinds)).tf_total;
}

size_t wo_aberrated_workspace_bytes(int n_tiles, int Z, int Y, int X, unsigned kinds) {
  if (check_shape(n_tiles, Z, Y, X, kinds) != WO_OK) return 0;
  Sys s = system_of(kinds);
  s.aberr = 1;
  return layout_of(n_tiles, Z, Y, X, s).total;
}

size_t wo_workspace_bytes(int n_tiles, int Z, int Y, int X, unsigned kinds) {
  if (check_shape(n_tiles, Z, Y, X, kinds) != WO_OK) return 0;
  return layout_of(n_tiles, Z, Y, X, system_of(kinds)).total;
}

const char* wo_status_string(wo_status st) {
  switch (st) {
    case WO_OK: return "ok";
    case WO_ERR_ARG: return "invalid argument (null or misaligned pointer, bad count or flag)";
    case WO_ERR_SHAPE: return "inconsistent shape";
    case WO_ERR_UNSUPPORTED_SIZE: return "unsupported transform length";
    case WO_ERR_UNDERSAMPLED: return "optics undersampled on this grid";
    case WO_ERR_CUDA: return "CUDA error";
    case WO_ERR_TIMEOUT: return "device-side wait timed out";
    case WO_ERR_OPTICS: return "physically invalid optics";
    case WO_ERR_WORKSPACE: return "workspace too small";
    case WO_ERR_BOUNDS: return "a device-side index check failed (WO_CHECK build)";
  }
  return "unknown status";
}

void wo_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_prof = on != 0;
}

int wo_profile_read(const char** names, long long* launches, double* ms, int cap) {
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<const char*> nm;
  std::vector<long long> cnt;
  std::vector<double> tot;
  for (const Pending& p : g_pending) {
    float t = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess) cudaEventElapsedTime(&t, p.a, p.b);
    size_t i = 0;
    for (; i < nm.size(); ++i)
      if (strcmp(nm[i], p.name) == 0) break;
    if (i == nm.size()) {
      nm.push_back(p.name);
      cnt.push_back(0);
      tot.push_back(0.0);
    }
    cnt[i] += 1;
    tot[i] += t;
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
  const int n = (int)nm.size();
  for (int i = 0; i < n && i < cap; ++i) {
    if (names) names[i] = nm[i];
    if (launches) launches[i] = cnt[i];
    if (ms) ms[i] = tot[i];
  }
  return n;
}

long long wo_launch_count(void) { return g_launches.load(); }
}  // extern "C"

namespace wo {
namespace {
std::mutex g_attr_mu;
struct SmemGrant {
  const void* kernel;
  int device;
  size_t bytes;  // dynamic shared memory the kernel may take on the device
};
std::vector<SmemGrant> g_attr_set;
}  // namespace

#if defined(WO_CHECK) && WO_CHECK
namespace {
std::vector<CheckReader>& check_units() {
  static std::vector<CheckReader> units;
  return units;
}
std::mutex g_check_mu;
}  // namespace

void check_register(CheckReader r) {
  std::lock_guard<std::mutex> lk(g_check_mu);
  check_units().push_back(r);
}

int check_take_all(int* info) {
  std::lock_guard<std::mutex> lk(g_check_mu);
  int first = 0;
  for (CheckReader r : check_units()) {
    int inf[2] = {0, 0};
    const int c = r(inf);
    if (c != 0 && first == 0) {
      first = c;
      if (info) {
        info[0] = inf[0];
        info[1] = inf[1];
      }
    }
  }
  return first;
}
#endif

size_t smem_attr_granted(const void* kernel, int device) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  for (const auto& e : g_attr_set)
    if (e.kernel == kernel && e.device == device) return e.bytes;
  return 0;
}

void smem_attr_mark(const void* kernel, int device, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  for (auto& e : g_attr_set)
    if (e.kernel == kernel && e.device == device) {
      if (bytes > e.bytes) e.bytes = bytes;
      return;
    }
  g_attr_set.push_back({kernel, device, bytes});
}
}  // namespace wo

extern "C" {

// Shared body of wo_build_tf (optics copied from the host into the workspace)
// and wo_build_tf_device (optics read in place from device memory).
static wo_status build_tf_impl(const wo_optics* optics, bool on_host, int n_tiles, int Z, int Y, int X,
                               unsigned kinds, void* d_tf, void* d_ws, size_t ws_bytes, wo_stream stream,
                               const double* h_zern = nullptr, int n_zern = 0) {
  wo_status st = check_shape(n_tiles, Z, Y, X, kinds);
  if (st != WO_OK) return st;
  if (!optics || !aligned16(d_tf) || !aligned16(d_ws)) return WO_ERR_ARG;
  if (n_zern < 0 || n_zern > WO_MAX_ZERNIKE || (n_zern > 0 && !h_zern)) return WO_ERR_ARG;
  for (long long i = 0; i < (long long)n_tiles * n_zern; ++i)
    if (!isfinite(h_zern[i])) return WO_ERR_ARG;
  if (!on_host && (((uintptr_t)optics) & 7u)) return WO_ERR_ARG;
  if (on_host) {
    for (int t = 0; t < n_tiles; ++t) {
      st = check_optics(optics[t]);
      if (st != WO_OK) return st;
    }
  }
  Sys s = system_of(kinds);
  s.aberr = n_zern > 0 ? 1 : 0;
  const Layout L = layout_of(n_tiles, Z, Y, X, s);
  if (ws_bytes < L.total) return WO_ERR_WORKSPACE;
  cudaStream_t cs = (cudaStream_t)stream;
  char* ws = (char*)d_ws;
  char* tfb = (char*)d_tf;
  TfArgs a{};
  a.zern = s.aberr ? (const double*)(ws + L.zern) : nullptr;
  a.n_zern = n_zern;
  a.optics = on_host ? (const wo_optics*)(ws + L.optics) : optics;
  a.counts = (int*)(ws + L.counts);
  a.rec = (float4*)(ws + L.rec);
  a.arms = (float2*)(ws + L.arms);
  a.tf = (float2*)tfb;
  a.stats = (float*)(tfb + L.tf_stats);
  a.n_tiles = n_tiles; a.Z = Z; a.Y = Y; a.X = X;
  a.lf_props = s.lf_props;
  a.want_phase = s.want_phase; a.want_abs = s.want_abs; a.want_fl = s.has_fl;
  a.n_arms = s.n_arms; a.n_kinds = s.n_kinds;
  a.want_dz = s.want_dz;
  a.want_grad = s.want_grad;
  a.smooth = s.smooth;
  a.rec2 = (float4*)(ws + L.rec2);
  a.norm_part = (float*)(ws + L.norm_part);
  a.norms = (float*)(ws + L.norms);
  a.rec_blocks = (Y + record_rows(Y, n_tiles) - 1) / record_rows(Y, n_tiles);
  a.kxm = s.kxm;
  // Columns k_x beyond the largest TF support radius of the batch hold only
  // the PSF rows' rounding noise: the y and z passes leave them out.  The
  // radius: H1(q) needs nu in S and P and nu + q in P; the fluorescence TF and
  // the smooth source reach 2 NA_det / lambda; plus two bins of margin.
  a.x_cols = X / 2 + 1;
  if (on_host) {
    int kmax = 0;
    for (int q = 0; q < n_tiles; ++q) {
      const wo_optics& o = optics[q];
      const double tilt = sqrt(o.tilt_x * o.tilt_x + o.tilt_y * o.tilt_y);
      double r = 0.0;
      if (s.lf_props > 0) r = s.smooth ? 2.0 * o.na_det : o.na_det + fmin(o.na_det, o.na_ill + tilt);
      if (s.has_fl) r = fmax(r, 2.0 * o.na_det);
      const int k = (int)ceil(r / o.lambda_um * (double)X * o.pixel_um) + 2;
      kmax = k > kmax ? k : kmax;
    }
    if (kmax + 1 < a.x_cols) a.x_cols = kmax + 1;
  }
  if (on_host)
    WO_TRY(cudaMemcpyAsync((void*)a.optics, optics, (size_t)n_tiles * sizeof(wo_optics), cudaMemcpyHostToDevice, cs));
  if (s.aberr)
    WO_TRY(cudaMemcpyAsync((void*)a.zern, h_zern, (size_t)n_tiles * n_zern * sizeof(double), cudaMemcpyHostToDevice,
                           cs));
  WO_TRY(cudaMemsetAsync(a.counts, 0, (size_t)n_tiles * 4 * sizeof(int), cs));
  WO_TRY(cudaMemsetAsync(a.stats, 0, (size_t)n_tiles * 8 * sizeof(float), cs));
  WO_TRY(tf_pupil_record(a, cs));
  WO_TRY(tf_arms(a, cs));
  a.row_begin = 0;
  a.row_end = (long long)n_tiles * Z * Y;
  WO_TRY(tf_psf_rows(a, cs));
  if (s.kxm) return cuda_status(tf_plane_yz(a, (int*)(ws + L.status), cs));  // y and z transforms, plane by plane
  const int Xh = X / 2 + 1;
  WO_TRY(cols_c2c(Y, false, a.tf, Xh, (long long)Y * Xh, a.x_cols, (long long)n_tiles * s.n_kinds * Z, cs,
                  "tf_ypass"));
  if (!s.planes) WO_TRY(tf_zpass(a, cs));  // per-plane banks stop before the z transform
  return WO_OK;
}

wo_status wo_build_tf(const wo_optics* h_optics, int n_tiles, int Z, int Y, int X, unsigned kinds,
                      void* d_tf, void* d_ws, size_t ws_bytes, wo_stream stream) {
  return build_tf_impl(h_optics, true, n_tiles, Z, Y, X, kinds, d_tf, d_ws, ws_bytes, stream);
}

wo_status wo_build_tf_device(const wo_optics* d_optics, int n_tiles, int Z, int Y, int X, unsigned kinds,
                             void* d_tf, void* d_ws, size_t ws_bytes, wo_stream stream) {
  return build_tf_impl(d_optics, false, n_tiles, Z, Y, X, kinds, d_tf, d_ws, ws_bytes, stream);
}

wo_status wo_build_tf_aberrated(const wo_optics* h_optics, const double* h_zernike, int n_zernike, int n_tiles,
                                int Z, int Y, int X, unsigned kinds, void* d_tf, void* d_ws, size_t ws_bytes,
                                wo_stream stream) {
  return build_tf_impl(h_optics, true, n_tiles, Z, Y, X, kinds, d_tf, d_ws, ws_bytes, stream, h_zernike, n_zernike);
}

// forward (op 0), adjoint (op 1), reconstruct (op 2)
// Kinds whose reconstruction the tile pipeline covers: the phase TF alone
// (also from a defocus-derivative bank, whose slot 0 it is).
static bool pipe_system(const Sys& s) { return s.lf_props == 1 && s.want_phase && !s.has_fl && !s.planes; }

// Arguments of the tile pipeline for a reconstruction with this layout.
static PipeLaunch pipe_launch(const Layout& L, const Sys& s, const void* d_tf, const float* d_in, float* d_out,
                              int n_tiles, int Z, int Y, int X, char* ws, int tf_shared, float eta, int eta_absolute,
                              const float* h_bg) {
  const int Xh = X / 2 + 1;
  PipeLaunch p{};
  p.in = d_in;
  p.out = d_out;
  p.spec = (float2*)(ws + L.specA);
  p.tf = (const float2*)d_tf;  // the phase TF is slot 0 of every bank that has one
  p.tf_stride = (long long)s.n_kinds * Z * Y * Xh;
  p.stats = (const float*)((const char*)d_tf + (tf_shared ? layout_of(1, Z, Y, X, s).tf_stats : L.tf_stats));
  p.counters = (int*)(ws + L.pipe);
  p.status = (int*)(ws + L.status);
  p.n_tiles = n_tiles;
  p.Z = Z;
  p.Y = Y;
  p.X = X;
  p.tf_shared = tf_shared;
  p.eta_absolute = eta_absolute;
  p.zero_dc = h_bg ? 0 : 1;
  p.withhold = -1;
  p.eta = eta;
  p.bg_plane = h_bg ? (float)((double)Y * X * h_bg[0]) : 0.f;
  p.scale = (float)(2.0 / ((double)X * (double)Y * (double)Z));
  p.budget_ns = kPipeBudgetNs;
  return p;
}

// tf_shared: d_tf holds one tile's bank, used for every tile of the batch.
// field: the input stacks are the tiles of a field, read in place by the
// first pass (d_in unused; one data channel).  fout: the output tiles are
// blended into a field by the last pass (d_out unused).
static wo_status run_op(int op, const void* d_tf, unsigned kinds, const float* d_in, const float* h_bg,
                        const float* h_eta, int eta_flag, int mode, float* d_out, int n_tiles, int Z,
                        int Y, int X, void* d_ws, size_t ws_bytes, wo_stream stream, int tf_shared = 0,
                        const FieldSrc* field = nullptr, const FieldDst* fout = nullptr) {
  wo_status st = check_shape(n_tiles, Z, Y, X, kinds);
  if (st != WO_OK) return st;
  if (kinds & WO_TF_PLANES) return WO_ERR_ARG;  // the operators need the 3D TFs
  if (field) d_in = field->field;
  if (fout) d_out = fout->field;
  if (!aligned16(d_tf) || !aligned16(d_in) || !aligned16(d_out) || !aligned16(d_ws)) return WO_ERR_ARG;
  const Sys s = system_of(kinds);
  // a kx-major bank serves the 3D operators on square planes (not the 2D
  // solve, not the fused blend)
  if (s.kxm && (mode != WO_MODE_3D || fout || X != Y)) return WO_ERR_ARG;
  if (op == 2) {
    if (!h_eta) return WO_ERR_ARG;
    if (eta_flag != WO_ETA_RELATIVE && eta_flag != WO_ETA_ABSOLUTE) return WO_ERR_ARG;
    if (mode != WO_MODE_3D && mode != WO_MODE_2D) return WO_ERR_ARG;
    const int n_modes = (s.lf_props ? 1 : 0) + s.has_fl;
    for (int m = 0; m < n_modes; ++m)
      if (!(h_eta[m] >= 0.f) || !isfinite(h_eta[m])) return WO_ERR_ARG;
  }
  if (h_bg) {
    for (int c = 0; c < s.C; ++c)
      if (!isfinite(h_bg[c])) return WO_ERR_ARG;
  }
  const Layout L = layout_of(n_tiles, Z, Y, X, s);
  if (ws_bytes < L.total) return WO_ERR_WORKSPACE;
  cudaStream_t cs = (cudaStream_t)stream;
  char* ws = (char*)d_ws;
  float2* specA = (float2*)(ws + L.specA);
  float2* specB = (float2*)(ws + L.specB);
  const float2* tf = (const float2*)d_tf;
  const int Xh = X / 2 + 1, H = X / 2;
  const int n_in = (op == 0) ? s.P : s.C;
  const int n_out = (op == 0) ? s.C : s.P;

  RowBg bg_in{};
  bg_in.rows_per_block = (long long)Z * Y;
  bg_in.nchan = n_in;
  if (op != 0) {
    if (h_bg) {
      bg_in.mode = 1;
      for (int c = 0; c < s.C; ++c) bg_in.v[c] = h_bg[c];
    } else if (op == 2) {
      bg_in.mode = 2;  // any constant only moves the DC bin, which is zeroed
    }
  }
  RowBg bg_out{};
  bg_out.rows_per_block = (long long)Z * Y;
  bg_out.nchan = n_out;
  if (op == 0 && h_bg) {
    bg_out.mode = 1;
    for (int c = 0; c < s.C; ++c) bg_out.v[c] = h_bg[c];
  }

  ZOp zo{};
  zo.op = op;
  zo.n_in = n_in;
  zo.n_out = n_out;
  zo.n_tf = s.n_kinds;
  zo.lf_props = s.lf_props;
  zo.has_fl = s.has_fl;
  zo.lf_chan = s.lf_props ? 0 : -1;
  zo.fl_chan = s.has_fl ? (s.lf_props ? 1 : 0) : -1;
  zo.tf_shared = tf_shared;
  // the statistics block follows the spectra of the tiles the bank was built for
  zo.stats = (const float*)((const char*)d_tf + (tf_shared ? layout_of(1, Z, Y, X, s).tf_stats : L.tf_stats));
  if (op == 2) {
    int m = 0;
    if (s.lf_props) zo.eta_lf = h_eta[m++];
    if (s.has_fl) zo.eta_fl = h_eta[m++];
    zo.eta_absolute = (eta_flag == WO_ETA_ABSOLUTE);
    zo.zero_dc = h_bg ? 0 : 1;
  }

  // The phase-only 3D reconstruction of tile-sized planes runs as one
  // persistent pipeline (wo_pipe.cu) unless the schedule table says otherwise.
  if (op == 2 && mode == WO_MODE_3D && !field && !fout && !s.kxm && pipe_system(s) && pipe_supported(Z, Y, X) &&
      recon_engine(Z, Y, X) == WO_ENGINE_HYBRID) {
    PipeLaunch p = pipe_launch(L, s, d_tf, d_in, d_out, n_tiles, Z, Y, X, ws, tf_shared, zo.eta_lf,
                               zo.eta_absolute, h_bg);
    return cuda_status(tile_pipeline(p, cs));
  }
  const long long in_rows = (long long)n_tiles * n_in * Z * Y;
  if (s.kxm) {
    // kx-major bank (one kind: one volume in, one out): the x pass into the
    // kx-major spectrum (from the tiles, or from the field's tiles in place),
    // the plane engine, the x pass back (the forward model adds its
    // background there); the spectrum stays in specA throughout
    if (field) WO_TRY(rows_r2c_field_kxm(H, *field, specA, in_rows, bg_in, cs));
    else WO_TRY(rows_r2c_kxm(H, d_in, specA, in_rows, Z, Y, bg_in, cs));
    WO_TRY(plane_yz_op(Z, Y, specA, tf, zo, n_tiles, Xh, (int*)(ws + L.status), cs));
    const float scale = (float)(2.0 / ((double)X * (double)Y * (double)Z));
    WO_TRY(rows_c2r_kxm(H, specA, d_out, (long long)n_tiles * n_out * Z * Y, Z, Y, scale, bg_out, cs));
    return WO_OK;
  }
  if (field) {  // the x pass reads the tiles from the field, then the y pass
    WO_TRY(rows_r2c_field(H, *field, specA, in_rows, bg_in, cs));
    WO_TRY(cols_c2c(Y, false, specA, Xh, (long long)Y * Xh, Xh, in_rows / Y, cs, "y_fwd"));
  } else {
    WO_TRY(plane_xy_fwd(X, Y, d_in, specA, in_rows / Y, bg_in, cs));
  }
  if (op == 2 && mode == WO_MODE_2D) {
    WO_TRY(z_solve2d(Z, specA, specB, tf, zo, n_tiles, Y, Xh, cs));
    const float scale = 2.0f / ((float)X * (float)Y);
    RowBg none{};
    none.rows_per_block = Y;
    none.nchan = 1;
    if (fout) {  // inverse y pass, then the inverse x pass blending the tiles into the field
      WO_TRY(cols_c2c(Y, true, specB, Xh, (long long)Y * Xh, Xh, (long long)n_tiles * s.P, cs, "y_inv"));
      FieldDst f2 = *fout;
      f2.Z = 1;
      WO_TRY(rows_c2r_blend(H, specB, f2, scale, cs));
    } else {
      WO_TRY(plane_xy_inv(X, Y, specB, d_out, (long long)n_tiles * s.P, scale, none, cs));
    }
    return WO_OK;
  }
  WO_TRY(z_fused(Z, specA, specB, tf, zo, n_tiles, Y, Xh, cs));
  const float scale = (float)(2.0 / ((double)X * (double)Y * (double)Z));
  if (fout) {  // (reconstruction only: no background added on the way out)
    WO_TRY(cols_c2c(Y, true, specB, Xh, (long long)Y * Xh, Xh, (long long)n_tiles * n_out * Z, cs, "y_inv"));
    WO_TRY(rows_c2r_blend(H, specB, *fout, scale, cs));
  } else {
    WO_TRY(plane_xy_inv(X, Y, specB, d_out, (long long)n_tiles * n_out * Z, scale, bg_out, cs));
  }
  return WO_OK;
}

wo_status wo_forward(const void* d_tf, unsigned kinds, const float* d_f, const float* h_background,
                     float* d_data, int n_tiles, int Z, int Y, int X, void* d_ws, size_t ws_bytes,
                     wo_stream stream) {
  return run_op(0, d_tf, kinds, d_f, h_background, nullptr, 0, WO_MODE_3D, d_data, n_tiles, Z, Y, X, d_ws,
                ws_bytes, stream);
}

wo_status wo_forward_adjoint(const void* d_tf, unsigned kinds, const float* d_data,
                             const float* h_background, float* d_f, int n_tiles, int Z, int Y, int X,
                             void* d_ws, size_t ws_bytes, wo_stream stream) {
  return run_op(1, d_tf, kinds, d_data, h_background, nullptr, 0, WO_MODE_3D, d_f, n_tiles, Z, Y, X, d_ws,
                ws_bytes, stream);
}

wo_status wo_reconstruct(const void* d_tf, unsigned kinds, const float* d_data, const float* h_background,
                         const float* h_eta, int eta_flag, int mode, float* d_f, int n_tiles, int Z, int Y,
                         int X, void* d_ws, size_t ws_bytes, wo_stream stream) {
  return run_op(2, d_tf, kinds, d_data, h_background, h_eta, eta_flag, mode, d_f, n_tiles, Z, Y, X, d_ws,
                ws_bytes, stream);
}

wo_status wo_reconstruct_field_tiles(const void* d_tf, unsigned kinds, const float* d_field, int Z, int tiles_y,
                                     int tiles_x, int core, int halo, const float* h_background, const float* h_eta,
                                     int eta_flag, int mode, float* d_f, void* d_ws, size_t ws_bytes,
                                     wo_stream stream) {
  if (tiles_y < 1 || tiles_x < 1 || core < 1 || halo < 0 || 2 * halo > core || Z < 1) return WO_ERR_ARG;
  if ((long long)tiles_y * tiles_x > 65535) return WO_ERR_ARG;
  if (!d_field) return WO_ERR_ARG;
  const Sys s = system_of(kinds);
  if (s.C != 1) return WO_ERR_ARG;  // a field is one channel
  const int E = core + 2 * halo;
  if (E % 2 || !rows_reg_supported(E / 2)) return WO_ERR_UNSUPPORTED_SIZE;
  const FieldSrc f{d_field, Z, tiles_y, tiles_x, core, halo};
  return run_op(2, d_tf, kinds, nullptr, h_background, h_eta, eta_flag, mode, d_f, tiles_y * tiles_x, Z, E, E, d_ws,
                ws_bytes, stream, 0, &f);
}

wo_status wo_restore_field(const void* d_tf, unsigned kinds, const float* d_field, int Z, int tiles_y, int tiles_x,
                           int core, int halo, const float* h_background, const float* h_eta, int eta_flag, int mode,
                           float* d_out, void* d_ws, size_t ws_bytes, wo_stream stream) {
  if (tiles_y < 1 || tiles_x < 1 || core < 1 || halo < 0 || 2 * halo > core || Z < 1) return WO_ERR_ARG;
  if ((long long)tiles_y * tiles_x > 65535 || tiles_x > 64) return WO_ERR_ARG;
  if (!d_field || !d_out || d_out == d_field) return WO_ERR_ARG;
  const Sys s = system_of(kinds);
  if (s.C != 1) return WO_ERR_ARG;  // a field is one channel
  const int E = core + 2 * halo;
  if (E % 2 || !rows_reg_supported(E / 2)) return WO_ERR_UNSUPPORTED_SIZE;
  const FieldSrc f{d_field, Z, tiles_y, tiles_x, core, halo};
  const FieldDst o{d_out, s.P, Z, tiles_y, tiles_x, core, halo};
  return run_op(2, d_tf, kinds, nullptr, h_background, h_eta, eta_flag, mode, nullptr, tiles_y * tiles_x, Z, E, E,
                d_ws, ws_bytes, stream, 0, &f, &o);
}

wo_status wo_reconstruct_shared_tf(const void* d_tf, unsigned kinds, const float* d_data,
                                   const float* h_background, const float* h_eta, int eta_flag, int mode, float* d_f,
                                   int n_tiles, int Z, int Y, int X, void* d_ws, size_t ws_bytes, wo_stream stream) {
  return run_op(2, d_tf, kinds, d_data, h_background, h_eta, eta_flag, mode, d_f, n_tiles, Z, Y, X, d_ws, ws_bytes,
                stream, 1);
}

wo_status wo_pipeline_probe(const void* d_tf, const float* d_data, float* d_f, int n_tiles, int Z, int Y, int X,
                            int withhold, long long budget_ns, void* d_ws, size_t ws_bytes, wo_stream stream) {
  wo_status st = check_shape(n_tiles, Z, Y, X, WO_TF_PHASE);
  if (st != WO_OK) return st;
  if (!pipe_supported(Z, Y, X)) return WO_ERR_UNSUPPORTED_SIZE;
  if (!aligned16(d_tf) || !aligned16(d_data) || !aligned16(d_f) || !aligned16(d_ws)) return WO_ERR_ARG;
  if (withhold < -1 || withhold >= n_tiles || budget_ns < 1000 || budget_ns > 10LL * kPipeBudgetNs) return WO_ERR_ARG;
  const Sys s = system_of(WO_TF_PHASE);
  const Layout L = layout_of(n_tiles, Z, Y, X, s);
  if (ws_bytes < L.total) return WO_ERR_WORKSPACE;
  PipeLaunch p = pipe_launch(L, s, d_tf, d_data, d_f, n_tiles, Z, Y, X, (char*)d_ws, 0, 1e-3f, 1, nullptr);
  p.withhold = withhold;
  p.budget_ns = budget_ns;
  return cuda_status(tile_pipeline(p, (cudaStream_t)stream));
}

wo_status wo_sync_status(void* d_ws, int* h_info, wo_stream stream) {
  if (!aligned16(d_ws)) return WO_ERR_ARG;
  cudaStream_t cs = (cudaStream_t)stream;
  int blk[4] = {0, 0, 0, 0};
  // pageable destination: the copy has landed when the call returns
  WO_TRY(cudaMemcpyAsync(blk, d_ws, sizeof(blk), cudaMemcpyDeviceToHost, cs));
  WO_TRY(cudaMemsetAsync(d_ws, 0, kStatusBytes, cs));
  WO_TRY(cudaStreamSynchronize(cs));
  if (h_info) {
    h_info[0] = blk[1];
    h_info[1] = blk[2];
  }
  if (blk[0] < 0 || blk[0] > (int)WO_ERR_BOUNDS) return WO_ERR_CUDA;  // not a status: the block was never cleared
#if defined(WO_CHECK) && WO_CHECK
  // the index checks of every translation unit (read and cleared in any case)
  int cinfo[2] = {0, 0};
  const int c = check_take_all(cinfo);
  if (blk[0] == 0 && c != 0) {
    if (h_info) {
      h_info[0] = cinfo[0];
      h_info[1] = cinfo[1];
    }
    return (wo_status)c;
  }
#endif
  return (wo_status)blk[0];
}

int wo_check_build(void) {
#if defined(WO_CHECK) && WO_CHECK
  return 1;
#else
  return 0;
#endif
}

wo_status wo_clear_status(void* d_ws, wo_stream stream) {
  if (!aligned16(d_ws)) return WO_ERR_ARG;
  return cuda_status(cudaMemsetAsync(d_ws, 0, kStatusBytes, (cudaStream_t)stream));
}

wo_status wo_spectrum(const float* d_data, const float* h_background, int mode, void* d_spec, int n_tiles, int Z,
                      int Y, int X, wo_stream stream) {
  wo_status st = check_shape(n_tiles, Z, Y, X, WO_TF_PHASE);
  if (st != WO_OK) return st;
  if (mode != WO_MODE_3D && mode != WO_MODE_2D) return WO_ERR_ARG;
  if (!aligned16(d_data) || !aligned16(d_spec)) return WO_ERR_ARG;
  if (h_background && !isfinite(h_background[0])) return WO_ERR_ARG;
  cudaStream_t cs = (cudaStream_t)stream;
  float2* spec = (float2*)d_spec;
  const int Xh = X / 2 + 1, H = X / 2;
  const long long plane = (long long)Y * Xh;
  RowBg bg{};
  bg.rows_per_block = (long long)Z * Y;
  bg.nchan = 1;
  if (h_background) {
    bg.mode = 1;
    bg.v[0] = h_background[0];
  } else {
    bg.mode = 2;  // a constant per stack only moves the DC bins, fixed below
  }
  WO_TRY(plane_xy_fwd(X, Y, d_data, spec, (long long)n_tiles * Z, bg, cs));
  if (mode == WO_MODE_3D) {
    WO_TRY(cols_c2c(Z, false, spec, plane, (long long)Z * plane, (int)plane, n_tiles, cs, "z_fwd"));
    if (!h_background) WO_TRY(zero_dc(spec, n_tiles, (long long)Z * plane, cs));
  } else if (!h_background) {
    WO_TRY(center_dc_planes(spec, n_tiles, Z, plane, cs));
  }
  return WO_OK;
}

wo_status wo_tune_objective(const void* d_tf, unsigned kinds, const wo_optics* d_optics, const void* d_spec,
                            int loss, float eta, float nu_max, double* d_value, double* d_grad, int n_tiles, int Z,
                            int Y, int X, void* d_ws, size_t ws_bytes, wo_stream stream) {
  const unsigned base = kinds & ~(unsigned)(WO_TF_PLANES | WO_TF_SMOOTH_SOURCE);
  if (base != WO_TF_PHASE_DZ && base != WO_TF_PHASE_GRAD) return WO_ERR_ARG;
  if (loss != WO_LOSS_DATA && loss != WO_LOSS_MIDBAND) return WO_ERR_ARG;
  wo_status st = check_shape(n_tiles, Z, Y, X, kinds);
  if (st != WO_OK) return st;
  if (!aligned16(d_tf) || !aligned16(d_spec) || !aligned16(d_ws)) return WO_ERR_ARG;
  if (!d_optics || (((uintptr_t)d_optics) & 7u)) return WO_ERR_ARG;
  if (!d_value && !d_grad) return WO_ERR_ARG;
  if ((d_value && (((uintptr_t)d_value) & 7u)) || (d_grad && (((uintptr_t)d_grad) & 7u))) return WO_ERR_ARG;
  if (!(eta >= 0.f) || !isfinite(eta) || !(nu_max == nu_max)) return WO_ERR_ARG;
  const int np = base == WO_TF_PHASE_GRAD ? 4 : 1;
  if (ws_bytes < kStatusBytes + tune_partials_bytes(n_tiles, Y, X, np)) return WO_ERR_WORKSPACE;
  return cuda_status(tune_reduce((const float2*)d_tf, (const float2*)d_spec, d_optics, n_tiles, Z, Y, X, eta,
                                 isfinite(nu_max) ? nu_max : 0.f, (kinds & WO_TF_PLANES) ? 1 : Z, loss, np,
                                 (double*)((char*)d_ws + kStatusBytes), d_value, d_grad, (cudaStream_t)stream));
}

wo_status wo_reconstruct_vjp(const void* d_tf, unsigned kinds, const void* d_spec, const float* d_gout, float eta,
                             int mode, double* d_grad, int n_tiles, int Z, int Y, int X, void* d_ws, size_t ws_bytes,
                             wo_stream stream) {
  const unsigned base = kinds & ~(unsigned)(WO_TF_PLANES | WO_TF_SMOOTH_SOURCE);
  if (base != WO_TF_PHASE_DZ && base != WO_TF_PHASE_GRAD) return WO_ERR_ARG;
  if (mode != WO_MODE_3D && mode != WO_MODE_2D) return WO_ERR_ARG;
  wo_status st = check_shape(n_tiles, Z, Y, X, kinds);
  if (st != WO_OK) return st;
  const bool planes = (kinds & WO_TF_PLANES) != 0;
  if ((mode == WO_MODE_3D) == planes) return WO_ERR_ARG;  // 3D needs a 3D bank, 2D a per-plane bank
  if (!aligned16(d_tf) || !aligned16(d_spec) || !aligned16(d_gout) || !aligned16(d_ws)) return WO_ERR_ARG;
  if (!d_grad || (((uintptr_t)d_grad) & 7u)) return WO_ERR_ARG;
  if (!(eta >= 0.f) || !isfinite(eta)) return WO_ERR_ARG;
  const int np = base == WO_TF_PHASE_GRAD ? 4 : 1;
  const int Xh = X / 2 + 1, H = X / 2;
  const long long plane = (long long)Y * Xh;
  const int gz = mode == WO_MODE_3D ? Z : 1;  // planes of the upstream gradient
  const size_t gbytes = align256((size_t)n_tiles * gz * plane * sizeof(float2));
  if (ws_bytes < kStatusBytes + gbytes + tune_partials_bytes(n_tiles, Y, X, np)) return WO_ERR_WORKSPACE;
  cudaStream_t cs = (cudaStream_t)stream;
  float2* G = (float2*)((char*)d_ws + kStatusBytes);
  double* partials = (double*)((char*)d_ws + kStatusBytes + gbytes);
  RowBg none{};
  none.rows_per_block = (long long)gz * Y;
  none.nchan = 1;
  WO_TRY(plane_xy_fwd(X, Y, d_gout, G, (long long)n_tiles * gz, none, cs));
  if (mode == WO_MODE_3D) WO_TRY(cols_c2c(Z, false, G, plane, (long long)Z * plane, (int)plane, n_tiles, cs, "z_fwd"));
  return cuda_status(vjp_reduce((const float2*)d_tf, (const float2*)d_spec, G, n_tiles, Z, Y, X, eta,
                                mode == WO_MODE_3D ? 1 : 0, np, partials, d_grad, cs));
}

wo_status wo_adam_optics(wo_optics* d_optics, const double* d_grad, int n_params, double* d_state, int n_tiles,
                         const double* h_lr, double beta1, double beta2, double eps, wo_stream stream) {
  if (n_tiles < 1 || n_tiles > 65535) return WO_ERR_ARG;
  if (n_params != 1 && n_params != 4) return WO_ERR_ARG;
  if (!d_optics || !d_grad || !d_state || !h_lr) return WO_ERR_ARG;
  if ((((uintptr_t)d_optics) | ((uintptr_t)d_grad) | ((uintptr_t)d_state)) & 7u) return WO_ERR_ARG;
  AdamLr lr{};
  for (int p = 0; p < n_params; ++p) {
    if (!(h_lr[p] >= 0.0) || !isfinite(h_lr[p])) return WO_ERR_ARG;
    lr.v[p] = h_lr[p];
  }
  if (!(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0) || !isfinite(eps))
    return WO_ERR_ARG;
  return cuda_status(adam_optics(d_optics, d_grad, n_params, d_state, n_tiles, lr, beta1, beta2, eps,
                                 (cudaStream_t)stream));
}

wo_status wo_reconstruct_fused(const void* d_tf, int n_channels, const float* d_data, const float* h_background,
                               float eta, int eta_flag, int mode, float* d_f, int n_tiles, int Z, int Y, int X,
                               void* d_ws, size_t ws_bytes, wo_stream stream) {
  if (n_channels < 1 || n_channels > kMaxFuseChannels) return WO_ERR_ARG;
  if (n_tiles < 1 || (long long)n_tiles * n_channels > 65535) return WO_ERR_ARG;
  wo_status st = check_shape(n_tiles * n_channels, Z, Y, X, WO_TF_PHASE);
  if (st != WO_OK) return st;
  if (!aligned16(d_tf) || !aligned16(d_data) || !aligned16(d_f) || !aligned16(d_ws)) return WO_ERR_ARG;
  if (eta_flag != WO_ETA_RELATIVE && eta_flag != WO_ETA_ABSOLUTE) return WO_ERR_ARG;
  if (mode != WO_MODE_3D && mode != WO_MODE_2D) return WO_ERR_ARG;
  if (!(eta >= 0.f) || !isfinite(eta)) return WO_ERR_ARG;
  if (h_background) {
    for (int c = 0; c < n_channels; ++c)
      if (!isfinite(h_background[c])) return WO_ERR_ARG;
  }
  const int C = n_channels;
  const int Xh = X / 2 + 1, H = X / 2;
  const size_t half = (size_t)Z * Y * Xh * sizeof(float2);
  const size_t specA = align256((size_t)n_tiles * C * half);
  const size_t specB = align256((size_t)n_tiles * half);
  const size_t statsb = align256((size_t)n_tiles * 2 * sizeof(float));
  if (ws_bytes < kStatusBytes + specA + specB + statsb) return WO_ERR_WORKSPACE;
  cudaStream_t cs = (cudaStream_t)stream;
  char* ws = (char*)d_ws + kStatusBytes;
  float2* A = (float2*)ws;
  float2* Bv = (float2*)(ws + specA);
  float* stats = (float*)(ws + specA + specB);
  RowBg bg{};
  bg.rows_per_block = (long long)Z * Y;
  bg.nchan = C;
  bg.mode = h_background ? 0 : 2;  // a given background is removed from the DC bin in the z pass
  FuseOp op{};
  op.C = C;
  op.mode = mode;
  op.zero_dc = h_background ? 0 : 1;
  op.eta_relative = eta_flag == WO_ETA_RELATIVE;
  op.eta = eta;
  op.stats = stats;
  const double nvox = (double)Z * Y * X;
  if (h_background)
    for (int c = 0; c < C; ++c) op.bg_dc[c] = (float)(nvox * (double)h_background[c]);
  const long long plane = (long long)Y * Xh;
  WO_TRY(plane_xy_fwd(X, Y, d_data, A, (long long)n_tiles * C * Z, bg, cs));
  if (op.eta_relative) WO_TRY(fuse_stats((const float2*)d_tf, n_tiles, C, Z, Y, Xh, stats, cs));
  WO_TRY(z_fuse(Z, A, Bv, (const float2*)d_tf, op, n_tiles, Y, Xh, cs));
  RowBg none{};
  none.nchan = 1;
  if (mode == WO_MODE_3D) {
    none.rows_per_block = (long long)Z * Y;
    WO_TRY(plane_xy_inv(X, Y, Bv, d_f, (long long)n_tiles * Z, (float)(2.0 / nvox), none, cs));
  } else {
    none.rows_per_block = Y;
    WO_TRY(plane_xy_inv(X, Y, Bv, d_f, (long long)n_tiles, 2.0f / ((float)X * (float)Y), none, cs));
  }
  return WO_OK;
}

size_t wo_fused_workspace_bytes(int n_channels, int n_tiles, int Z, int Y, int X) {
  if (n_channels < 1 || n_channels > kMaxFuseChannels || n_tiles < 1 || (long long)n_tiles * n_channels > 65535)
    return 0;
  if (check_shape(n_tiles * n_channels, Z, Y, X, WO_TF_PHASE) != WO_OK) return 0;
  const size_t half = (size_t)Z * Y * (X / 2 + 1) * sizeof(float2);
  return kStatusBytes + align256((size_t)n_tiles * n_channels * half) + align256((size_t)n_tiles * half) +
         align256((size_t)n_tiles * 2 * sizeof(float));
}

static wo_status check_tiles(int Z, int tiles_y, int tiles_x, int core, int halo, const void* a,
                             const void* b) {
  if (!aligned16(a) || !aligned16(b)) return WO_ERR_ARG;
  if (Z < 1 || tiles_y < 1 || tiles_x < 1 || core < 1 || halo < 0) return WO_ERR_SHAPE;
  if (2 * halo > core) return WO_ERR_SHAPE;
  const long long E = (long long)core + 2LL * halo;
  if (E > 65535 || (long long)tiles_x * core > (1LL << 30) || (long long)tiles_y * tiles_x * Z > 65535 ||
      (long long)tiles_y * core * Z > (1LL << 31) - 1)
    return WO_ERR_SHAPE;
  return WO_OK;
}

wo_status wo_tile_gather(const float* d_field, int Z, int tiles_y, int tiles_x, int core, int halo,
                         float* d_tiles, wo_stream stream) {
  wo_status st = check_tiles(Z, tiles_y, tiles_x, core, halo, d_field, d_tiles);
  if (st != WO_OK) return st;
  return cuda_status(tiles_gather(d_field, Z, tiles_y, tiles_x, core, halo, d_tiles, (cudaStream_t)stream));
}

wo_status wo_tile_blend(const float* d_tiles, int Z, int tiles_y, int tiles_x, int core, int halo,
                        float* d_field, wo_stream stream) {
  wo_status st = check_tiles(Z, tiles_y, tiles_x, core, halo, d_tiles, d_field);
  if (st != WO_OK) return st;
  return cuda_status(tiles_blend(d_tiles, Z, tiles_y, tiles_x, core, halo, d_field, (cudaStream_t)stream));
}

}  // extern "C"

// wo_sched.cu - the schedule table and the autotuner.
//
// Some passes have more than one implementation (an engine).  The column
// transforms (every y pass and the z transforms of wo_spectrum) run either on
// the shared-memory Stockham engine (wo_cols.cu: B columns per CTA, radix-8
// stages, each stage a shared-memory round trip between block barriers) or
// on the hybrid engine (wo_colhyb.cu: coalesced tile copies and a
// register-resident four-step transform per column, one padded transpose,
// warp-level synchronisation).  Which one is faster depends on the length,
// the number of columns and the batch; the table holds one choice per
// (pass, length), the autotuner fills it by timing both on the caller's
// shapes, and wo_schedule_set lets a caller pin a choice.
#include <atomic>
#include <mutex>
#include <stdio.h>
#include <string.h>

#include "wo_internal.h"

namespace wo {

namespace {
constexpr int kMaxLen = 2048;
std::atomic<int> g_cols_engine[kMaxLen + 1];  // 0: default
std::atomic<int> g_rows_engine[kMaxLen + 1];  // 0: default
std::atomic<int> g_recon_engine[kMaxLen + 1];  // 0: default, keyed by Y
std::atomic<int> g_xy_engine[kMaxLen + 1];     // 0: default, keyed by Y (X == Y)
}  // namespace

int xy_engine(int X, int Y) {
  if (!xy_supported(X, Y)) return WO_ENGINE_SMEM;
  const int e = g_xy_engine[Y].load(std::memory_order_relaxed);
  if (e == WO_ENGINE_SMEM || e == WO_ENGINE_HYBRID) return e;
  // default: the separate x and y passes.  The fused kernels hold a 109 KB
  // plane tile per CTA, so an SM runs two CTAs of four warps and overlaps
  // little of one CTA's copies with the other's transforms: 11.87 against
  // 10.99 ms per step of the 256-tile field (k_xy_fwd 410 us and k_xy_inv
  // 614 us per 64 tiles under ncu, 8 warps per SM); the autotuner keeps
  // them where they measure faster
  return WO_ENGINE_SMEM;
}

int recon_engine(int Z, int Y, int X) {
  if (!pipe_supported(Z, Y, X)) return WO_ENGINE_SMEM;
  const int e = g_recon_engine[Y].load(std::memory_order_relaxed);
  if (e == WO_ENGINE_SMEM || e == WO_ENGINE_HYBRID) return e;
  // default: the five passes.  The pipeline keeps a tile's spectra in L2
  // between its items but holds one 150 KB plane per SM, so an SM loads,
  // transforms and stores in turn instead of overlapping them across several
  // blocks: 7.5 ms against 4.9 ms for the five passes on the 256-tile field
  // (8.0 against 2.8 ms on 4096 small stacks)
  return WO_ENGINE_SMEM;
}

static bool recon_pipe_length(int n) { return n == 64 || n == 128 || n == 192; }

int cols_engine(int n) {
  if (n < 1 || n > kMaxLen) return WO_ENGINE_SMEM;
  const int e = g_cols_engine[n].load(std::memory_order_relaxed);
  if (e == WO_ENGINE_HYBRID && cols_hyb_supported(n)) return WO_ENGINE_HYBRID;
  if (e == WO_ENGINE_SMEM) return WO_ENGINE_SMEM;
  // default: the shared-memory engine, which was the faster one on the
  // workloads' y passes (512, 192 and 128 points); the autotuner may pick the
  // hybrid engine for other lengths and batches
  return WO_ENGINE_SMEM;
}

int rows_engine(int n) {
  if (n < 1 || n > kMaxLen || !rows_reg_supported(n)) return WO_ENGINE_SMEM;
  const int e = g_rows_engine[n].load(std::memory_order_relaxed);
  if (e == WO_ENGINE_SMEM || e == WO_ENGINE_HYBRID) return e;
  // default: the register rows, faster on the workloads' x passes (256 and 96
  // points: 0.127 -> 0.087 ms and 0.152 -> 0.112 ms on the widefield step)
  return WO_ENGINE_HYBRID;
}

// Time the two engines of one table entry on `run` (a batch of launches on
// stream s) and keep the faster.  The engines are timed in alternating rounds
// (kReps runs per round, after one untimed run each) and each keeps its best
// round, so a clock ramp or a cold cache early on does not decide the
// choice.  The other engine replaces the built-in default only when it is at
// least 2 % faster, so near-ties do not flip from one process to the next.
// Returns the engine kept, or -1 on a CUDA error (the entry is then
// restored).
template <class Run>
static int tune_entry(std::atomic<int>& entry, int default_engine, bool hybrid_ok, cudaStream_t s, Run run) {
  constexpr int kEngines = 2, kRounds = 3, kReps = 8;
  const int engines[kEngines] = {WO_ENGINE_SMEM, WO_ENGINE_HYBRID};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1;
  float t_best[kEngines];
  bool ok[kEngines];
  const int saved = entry.load();
  bool failed = false;
  for (int k = 0; k < kEngines; ++k) {
    t_best[k] = 0.f;
    ok[k] = engines[k] != WO_ENGINE_HYBRID || hybrid_ok;
    if (!ok[k]) continue;
    entry.store(engines[k]);
    if (run(0) != cudaSuccess) failed = true;
  }
  for (int r = 0; r < kRounds && !failed; ++r) {
    for (int k = 0; k < kEngines && !failed; ++k) {
      if (!ok[k]) continue;
      entry.store(engines[k]);
      cudaEventRecord(e0, s);
      for (int q = 0; q < kReps; ++q) run(q);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        failed = true;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r == 0 || ms < t_best[k]) t_best[k] = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int best = -1;
  for (int k = 0; k < kEngines && !failed; ++k)
    if (ok[k] && engines[k] == default_engine) best = k;
  for (int k = 0; k < kEngines && !failed; ++k)
    if (ok[k] && (best < 0 || t_best[k] < 0.98f * t_best[best])) best = k;
  entry.store(best < 0 ? saved : engines[best]);
  return best < 0 ? -1 : engines[best];
}

// Column transforms of length n over `planes` planes of `ncols` columns
// (pitch ncols) in the scratch buffer, alternating directions.
static int tune_cols(int n, int ncols, long long planes, float2* scratch, cudaStream_t s) {
  const long long ps = (long long)n * ncols;
  return tune_entry(g_cols_engine[n], WO_ENGINE_SMEM, cols_hyb_supported(n), s, [&](int q) {
    return cols_c2c(n, q & 1, scratch, ncols, ps, ncols, planes, s, "autotune");
  });
}

// The x and y transforms of `planes` planes of Y x X (X == Y): the fused
// kernels against the separate passes, forward and inverse per run.
static int tune_xy(int X, long long planes, float2* scratch, cudaStream_t s) {
  float* real = reinterpret_cast<float*>(scratch);
  float2* half = scratch + (size_t)planes * X * X / 2;  // after the real planes
  const RowBg none{};
  return tune_entry(g_xy_engine[X], WO_ENGINE_SMEM, true, s, [&](int) {
    cudaError_t e = plane_xy_fwd(X, X, real, half, planes, none, s);
    if (e != cudaSuccess) return e;
    return plane_xy_inv(X, X, half, real, planes, 1.0f, none, s);
  });
}

// x passes of n complex points over `rows` rows: a real-to-half-spectrum
// pass and its inverse per run, on two disjoint parts of the scratch buffer.
static int tune_rows(int n, long long rows, float2* scratch, cudaStream_t s) {
  float* real = reinterpret_cast<float*>(scratch);
  float2* half = scratch + (size_t)rows * n;  // after the 2n real samples of every row
  const RowBg none{};
  return tune_entry(g_rows_engine[n], WO_ENGINE_HYBRID, rows_reg_supported(n), s, [&](int) {
    cudaError_t e = rows_r2c(n, real, half, rows, none, s);
    if (e != cudaSuccess) return e;
    return rows_c2r(n, half, real, rows, 1.0f, none, s);
  });
}

}  // namespace wo

using namespace wo;

extern "C" {

wo_status wo_schedule_set(int pass, int n, int engine) {
  if (pass != WO_PASS_COLS && pass != WO_PASS_ROWS && pass != WO_PASS_RECON && pass != WO_PASS_XY) return WO_ERR_ARG;
  if (n < 1 || n > kMaxLen) return WO_ERR_ARG;
  if (engine != WO_ENGINE_DEFAULT && engine != WO_ENGINE_SMEM && engine != WO_ENGINE_HYBRID) return WO_ERR_ARG;
  if (pass == WO_PASS_RECON) {
    if (engine == WO_ENGINE_HYBRID && !recon_pipe_length(n)) return WO_ERR_UNSUPPORTED_SIZE;
    g_recon_engine[n].store(engine, std::memory_order_relaxed);
    return WO_OK;
  }
  if (pass == WO_PASS_XY) {
    if (engine == WO_ENGINE_HYBRID && !xy_supported(n, n)) return WO_ERR_UNSUPPORTED_SIZE;
    g_xy_engine[n].store(engine, std::memory_order_relaxed);
    return WO_OK;
  }
  const bool hyb_ok = pass == WO_PASS_COLS ? cols_hyb_supported(n) : rows_reg_supported(n);
  if (engine == WO_ENGINE_HYBRID && !hyb_ok) return WO_ERR_UNSUPPORTED_SIZE;
  (pass == WO_PASS_COLS ? g_cols_engine : g_rows_engine)[n].store(engine, std::memory_order_relaxed);
  return WO_OK;
}

int wo_schedule_get(int pass, int n) {
  if (n < 1 || n > kMaxLen) return -1;
  if (pass == WO_PASS_COLS) return cols_engine(n);
  if (pass == WO_PASS_ROWS) return rows_engine(n);
  if (pass == WO_PASS_XY) return xy_engine(n, n);
  if (pass == WO_PASS_RECON) {
    if (!recon_pipe_length(n)) return WO_ENGINE_SMEM;
    const int e = g_recon_engine[n].load(std::memory_order_relaxed);
    return e == WO_ENGINE_HYBRID ? WO_ENGINE_HYBRID : WO_ENGINE_SMEM;
  }
  return -1;
}

wo_status wo_autotune(int n_tiles, int Z, int Y, int X, unsigned kinds, void* d_ws, size_t ws_bytes,
                      wo_stream stream) {
  const size_t need = wo_workspace_bytes(n_tiles, Z, Y, X, kinds);
  if (need == 0) return WO_ERR_ARG;
  if (!d_ws || (((uintptr_t)d_ws) & 15u)) return WO_ERR_ARG;
  if (ws_bytes < need) return WO_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  // the trials use the workspace past its status block
  float2* scratch = (float2*)((char*)d_ws + kStatusBytes);
  const int Xh = X / 2 + 1;
  // y passes: Z planes per volume of Y x Xh; the largest batch of the entry
  // points (three volumes per tile) stays inside the workspace's first half
  const size_t vol_bytes = (size_t)Z * Y * Xh * sizeof(float2);
  long long vols = (long long)(((need - kStatusBytes) / 2) / vol_bytes);
  if (vols < 1) vols = 1;
  if (vols > 3LL * n_tiles) vols = 3LL * n_tiles;
  // the x-pass trial uses about twice the bytes of the column trials
  if (cudaMemsetAsync(scratch, 0, 2 * (size_t)vols * vol_bytes, s) != cudaSuccess) return WO_ERR_CUDA;
  if (tune_cols(Y, Xh, vols * Z, scratch, s) < 0) return WO_ERR_CUDA;
  // z transforms (3D data spectra): Y*Xh columns of length Z
  if (Z > 1 && Z != Y && tune_cols(Z, Y * Xh, vols, scratch, s) < 0) return WO_ERR_CUDA;
  // x passes: the rows of the same volumes (2n real samples in, n+1 bins out
  // per row fit the volumes' half spectra twice over)
  if (rows_reg_supported(X / 2) && tune_rows(X / 2, vols * Z * Y, scratch, s) < 0) return WO_ERR_CUDA;
  // fused x-y planes (the same volumes' planes, real and half spectrum side by side)
  if (xy_supported(X, Y) && tune_xy(X, vols * Z, scratch, s) < 0) return WO_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? WO_OK : WO_ERR_CUDA;
}

}  // extern "C"

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
}  // namespace

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

}  // namespace wo

using namespace wo;

extern "C" {

wo_status wo_schedule_set(int pass, int n, int engine) {
  if (pass != WO_PASS_COLS) return WO_ERR_ARG;
  if (n < 1 || n > kMaxLen) return WO_ERR_ARG;
  if (engine != WO_ENGINE_DEFAULT && engine != WO_ENGINE_SMEM && engine != WO_ENGINE_HYBRID) return WO_ERR_ARG;
  if (engine == WO_ENGINE_HYBRID && !cols_hyb_supported(n)) return WO_ERR_UNSUPPORTED_SIZE;
  g_cols_engine[n].store(engine, std::memory_order_relaxed);
  return WO_OK;
}

int wo_schedule_get(int pass, int n) {
  if (pass != WO_PASS_COLS || n < 1 || n > kMaxLen) return -1;
  return cols_engine(n);
}

// Time every engine for the column transforms of length n over `planes`
// planes of `ncols` columns (pitch ncols) in the scratch buffer; keep the
// fastest.  The engines are timed in alternating rounds (kReps launches per
// round, after one untimed launch each) and each keeps its best round, so a
// clock ramp or a cold cache early on does not decide the choice.  Returns
// the engine kept, or -1 on a CUDA error.
static int tune_cols(int n, int ncols, long long planes, float2* scratch, cudaStream_t s, float* best_ms) {
  constexpr int kEngines = 2, kRounds = 3, kReps = 8;
  const int engines[kEngines] = {WO_ENGINE_SMEM, WO_ENGINE_HYBRID};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1;
  float t_best[kEngines];
  bool ok[kEngines];
  const int saved = g_cols_engine[n].load();
  const long long ps = (long long)n * ncols;
  bool failed = false;
  for (int k = 0; k < kEngines; ++k) {
    t_best[k] = 0.f;
    ok[k] = engines[k] != WO_ENGINE_HYBRID || cols_hyb_supported(n);
    if (!ok[k]) continue;
    g_cols_engine[n].store(engines[k]);
    if (cols_c2c(n, false, scratch, ncols, ps, ncols, planes, s, "autotune") != cudaSuccess) failed = true;
  }
  for (int r = 0; r < kRounds && !failed; ++r) {
    for (int k = 0; k < kEngines && !failed; ++k) {
      if (!ok[k]) continue;
      g_cols_engine[n].store(engines[k]);
      cudaEventRecord(e0, s);
      for (int q = 0; q < kReps; ++q) cols_c2c(n, q & 1, scratch, ncols, ps, ncols, planes, s, "autotune");
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
    if (ok[k] && (best < 0 || t_best[k] < t_best[best])) best = k;
  g_cols_engine[n].store(best < 0 ? saved : engines[best]);
  if (best_ms) *best_ms = best < 0 ? 0.f : t_best[best] / kReps;
  return best < 0 ? -1 : engines[best];
}

wo_status wo_autotune(int n_tiles, int Z, int Y, int X, unsigned kinds, void* d_ws, size_t ws_bytes,
                      wo_stream stream) {
  const size_t need = wo_workspace_bytes(n_tiles, Z, Y, X, kinds);
  if (need == 0) return WO_ERR_ARG;
  if (!d_ws || (((uintptr_t)d_ws) & 15u)) return WO_ERR_ARG;
  if (ws_bytes < need) return WO_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  float2* scratch = (float2*)d_ws;
  const int Xh = X / 2 + 1;
  // y passes: Z planes per volume of Y x Xh; the largest batch of the entry
  // points (three volumes per tile) stays inside the workspace's first half
  const size_t vol_bytes = (size_t)Z * Y * Xh * sizeof(float2);
  long long vols = (long long)((need / 2) / vol_bytes);
  if (vols < 1) vols = 1;
  if (vols > 3LL * n_tiles) vols = 3LL * n_tiles;
  if (cudaMemsetAsync(scratch, 0, (size_t)vols * vol_bytes, s) != cudaSuccess) return WO_ERR_CUDA;
  if (tune_cols(Y, Xh, vols * Z, scratch, s, nullptr) < 0) return WO_ERR_CUDA;
  // z transforms (3D data spectra): Y*Xh columns of length Z
  if (Z > 1 && Z != Y && tune_cols(Z, Y * Xh, vols, scratch, s, nullptr) < 0) return WO_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? WO_OK : WO_ERR_CUDA;
}

}  // extern "C"

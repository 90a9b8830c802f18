// wo_tf.cuh - device helpers shared by the transfer-function kernels.
#pragma once
#include "wo_internal.h"

namespace wo {

__device__ __forceinline__ int fft_index(int i, int n) { return (i < (n + 1) / 2) ? i : i - n; }

__device__ __forceinline__ float lf_scale(const TfArgs& a, int t) {
  // 2K = 2 c / (N_perp sum S P^2), c = 2 pi n dz / lambda^2; the sum is a count
  // for the binary source and a float sum for the smooth one
  const wo_optics o = a.optics[t];
  const double sp = a.smooth ? (double)a.norms[4 * t] : (double)a.counts[4 * t];
  if (!(sp > 0.0)) return 0.f;
  const double c = 2.0 * 3.14159265358979323846 * o.n_medium * o.z_step_um / (o.lambda_um * o.lambda_um);
  return (float)(2.0 * c / ((double)a.Y * (double)a.X * sp));
}

// d log(sum S P^2) / d theta for the smooth source (theta = 0 tilt_x,
// 1 tilt_y, 2 NA_ill): the normalisation's share of dH1/dtheta.
__device__ __forceinline__ float norm_dlog(const TfArgs& a, int t, int theta) {
  const float sp = a.norms[4 * t];
  return sp > 0.f ? a.norms[4 * t + 1 + theta] / sp : 0.f;
}

__device__ __forceinline__ float fl_scale(const TfArgs& a, int t) {
  const int n_p = a.counts[4 * t + 1];
  if (n_p == 0) return 0.f;
  return (float)(1.0 / ((double)a.Y * (double)a.X * (double)a.Z * (double)n_p));
}

// fractional part of (eh + el) * (zh + zl), accurate to a few 1e-8
__device__ __forceinline__ float phase_frac(float eh, float el, float zh, float zl) {
  const float p = eh * zh;
  float err = fmaf(eh, zh, -p);
  err = fmaf(eh, zl, err);
  err = fmaf(el, zh, err);
  return (p - rintf(p)) + err;
}

// e^{i 2 pi f} of a phase f in cycles (|f| <= 1.5): f is folded into
// [-1/2, 1/2] and the unit phasor taken with the hardware sine and cosine
// (__sincosf), whose absolute error on [-pi, pi] CUDA documents as at most
// 2^-21.41 (about 4e-7): the arms are unit-magnitude factors times
// amplitudes <= 1 / eta, and every TF sums tens of thousands of them, so
// this stays three orders of magnitude inside the 1e-4 parity bound while
// costing a few instructions instead of a full-range sincospif.
__device__ __forceinline__ void unit_phasor(float f, float* s, float* c) {
  f -= rintf(f);
  __sincosf(6.28318530717958647692f * f, s, c);
}

}  // namespace wo

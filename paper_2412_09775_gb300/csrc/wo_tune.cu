// wo_tune.cu - per-tile defocus auto-tuning (Results, physics-guided
// auto-tuning; Fig. 2a(iv); Ext. Data Fig. 3; Methods, optical pooled screen
// data): the loss of the 2D thin-object Tikhonov fit and its exact derivative
// with respect to the tile's defocus, and an on-device Adam step.
//
// Per transverse frequency nu, with the data spectrum D_k and the TF pair
// (H_k, dH_k) over the Z entries k of a column - either the per-plane 2D
// spectra (k = plane j, zf = 1) or the 3D spectra (k = axial bin; Parseval
// over z turns the sum over planes into a sum over k with a factor zf = Z):
//   F  = sum_k conj(H_k) D_k / (sum_k |H_k|^2 + zf eta)     (the 2D solve)
//   R_k = D_k - H_k F                                       (residual)
//   q  = sum_k |R_k|^2 + zf eta |F|^2                       (loss density)
//   dq = -2 Re sum_k conj(dH_k F) R_k                       (its derivative)
// dq is the partial derivative at fixed F: F minimises q, so dq/dF = 0 there
// and the hand-written adjoint needs no derivative of the solve itself.  The
// per-tile loss is sum_nu w(nu) q / (N_perp zf), w = 2 for the half-spectrum
// bins that stand for a conjugate pair, 1 for x = 0 and x = X/2.
//
// The mid-band loss (the paper's image-quality loss) is -sum_band w |F|^2 /
// N_perp over c/8 <= |nu| <= c/4; F does not minimise it, so its derivative
// goes through the solve: with c = sum conj(H) D, h = sum |H|^2,
// den = h + zf eta, dF = (sum conj(dH) D - F 2 Re sum conj(H) dH) / den.
#include "wo_fft.cuh"
#include "wo_internal.h"

namespace wo {

namespace {
constexpr int kTuneThreads = 256;

__device__ __forceinline__ int freq_index(int i, int n) { return (i < (n + 1) / 2) ? i : i - n; }

// Deterministic block sum of NV doubles per thread (fixed tree over
// kTuneThreads); the sums land in red[v * kTuneThreads].
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
#pragma unroll
  for (int i = 0; i < NV; ++i) red[i * kTuneThreads + threadIdx.x] = v[i];
  __syncthreads();
  for (int h = kTuneThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
#pragma unroll
      for (int i = 0; i < NV; ++i) red[i * kTuneThreads + threadIdx.x] += red[i * kTuneThreads + threadIdx.x + h];
    }
    __syncthreads();
  }
}
}  // namespace

// One thread per transverse frequency (column c = y * Xh + x of the half
// spectrum), grid (ceil(Y*Xh / 256), n_tiles).  Consecutive threads read
// consecutive columns of every axial plane: each pass over k is coalesced.
// The bank holds 1 + NP slots per tile: H, then dH/dtheta_p.
template <int NP>
__global__ void __launch_bounds__(kTuneThreads) k_tune_cols(const float2* __restrict__ tf2,
                                                            const float2* __restrict__ spec,
                                                            const wo_optics* __restrict__ optics, int Z, int Y,
                                                            int Xh, int X, float eta, float nu_max, int zf,
                                                            int loss, double* __restrict__ partials) {
  __shared__ double red[(1 + NP) * kTuneThreads];
  const int t = blockIdx.y;
  const long long plane = (long long)Y * Xh;
  const long long vol = (long long)Z * plane;
  const long long c = (long long)blockIdx.x * kTuneThreads + threadIdx.x;
  double acc[1 + NP];  // value, then the derivatives
#pragma unroll
  for (int i = 0; i <= NP; ++i) acc[i] = 0.0;
  bool on = c < plane;
  int x = 0;
  if (on) {
    const int y = (int)(c / Xh);
    x = (int)(c - (long long)y * Xh);
    // the band tests take the frequencies in float64, as the oracle does;
    // the full loss needs none (float64 is slow on this part)
    if (loss == WO_LOSS_MIDBAND || nu_max > 0.f) {
      const wo_optics& o = optics[t];
      const double p = o.pixel_um;
      const double fy = (double)freq_index(y, Y) / ((double)Y * p), fx = (double)x / ((double)X * p);
      if (loss == WO_LOSS_MIDBAND) {  // c/8 <= |nu| <= c/4, c = (NA_det + NA_ill)/lambda
        const double r = sqrt(fx * fx + fy * fy), cut = (o.na_det + o.na_ill) / o.lambda_um;
        on = r >= cut / 8.0 && r <= cut / 4.0;
      } else {
        on = fx * fx + fy * fy <= (double)nu_max * (double)nu_max;
      }
    }
  }
  const double w = (x == 0 || 2 * x == X) ? 1.0 : 2.0;
  const float2* D = spec + (long long)t * vol + c;
  const float2* H = tf2 + (long long)t * (1 + NP) * vol + c;
  if (on && loss == WO_LOSS_MIDBAND) {
    // -|F|^2 and its derivatives through the solve: dF_p = (dc_p - F dh_p) / den
    float cr = 0.f, ci = 0.f, hh = 0.f, dcr[NP], dci[NP], dhr[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) dcr[q] = dci[q] = dhr[q] = 0.f;
#pragma unroll 4
    for (int k = 0; k < Z; ++k) {
      const float2 d = __ldg(D + k * plane), h = __ldg(H + k * plane);
      const float2 r = cmulc(h, d);
      cr += r.x;
      ci += r.y;
      hh += cabs2(h);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const float2 dh = __ldg(H + (q + 1) * vol + k * plane);
        const float2 e = cmulc(dh, d);
        dcr[q] += e.x;
        dci[q] += e.y;
        dhr[q] += h.x * dh.x + h.y * dh.y;
      }
    }
    const float den = hh + (float)zf * eta;
    const float inv = den > 0.f ? 1.0f / den : 0.f;
    const float2 F = make_float2(cr * inv, ci * inv);
    acc[0] = -w * (double)cabs2(F);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const float2 dF = make_float2((dcr[q] - 2.f * dhr[q] * F.x) * inv, (dci[q] - 2.f * dhr[q] * F.y) * inv);
      acc[1 + q] = -w * 2.0 * ((double)F.x * dF.x + (double)F.y * dF.y);
    }
  } else if (on) {
    float cr = 0.f, ci = 0.f, hh = 0.f;
#pragma unroll 8
    for (int k = 0; k < Z; ++k) {
      const float2 d = __ldg(D + k * plane), h = __ldg(H + k * plane);
      const float2 r = cmulc(h, d);
      cr += r.x;
      ci += r.y;
      hh += cabs2(h);
    }
    const float den = hh + (float)zf * eta;
    const float inv = den > 0.f ? 1.0f / den : 0.f;
    const float2 F = make_float2(cr * inv, ci * inv);
    float rr = 0.f, gg[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) gg[q] = 0.f;
#pragma unroll 4
    for (int k = 0; k < Z; ++k) {
      const float2 d = __ldg(D + k * plane), h = __ldg(H + k * plane);
      const float2 R = csub(d, cmul(h, F));
      rr += cabs2(R);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const float2 e = cmul(__ldg(H + (q + 1) * vol + k * plane), F);
        gg[q] += e.x * R.x + e.y * R.y;  // Re(conj(dH F) R)
      }
    }
    acc[0] = w * ((double)rr + (double)zf * (double)eta * (double)cabs2(F));
#pragma unroll
    for (int q = 0; q < NP; ++q) acc[1 + q] = w * (-2.0 * (double)gg[q]);
  }
  block_sum<1 + NP>(acc, red);
  if (threadIdx.x <= NP) partials[((long long)t * gridDim.x + blockIdx.x) * (1 + NP) + threadIdx.x] =
      red[threadIdx.x * kTuneThreads];
}

// One warp per tile: the tile's partials in a fixed order, then the scale.
__global__ void k_tune_final(const double* __restrict__ partials, int nblk, int np, double scale,
                             double* __restrict__ value, double* __restrict__ grad) {
  const int t = blockIdx.x, lane = threadIdx.x;
  for (int q = 0; q <= np; ++q) {
    double v = 0.0;
    for (int i = lane; i < nblk; i += 32) v += partials[((long long)t * nblk + i) * (1 + np) + q];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) {
      if (q == 0 && value) value[t] = v * scale;
      if (q > 0 && grad) grad[(long long)t * np + q - 1] = v * scale;
    }
  }
}

cudaError_t tune_reduce(const float2* tf2, const float2* spec, const wo_optics* optics, int n_tiles, int Z,
                        int Y, int X, float eta, float nu_max, int zf, int loss, int np, double* partials,
                        double* value, double* grad, cudaStream_t s) {
  const int Xh = X / 2 + 1;
  const long long plane = (long long)Y * Xh;
  const unsigned nblk = (unsigned)((plane + kTuneThreads - 1) / kTuneThreads);
  dim3 grid(nblk, (unsigned)n_tiles);
  if (np == 4) {
    WO_LAUNCH("tune_cols", s, (k_tune_cols<4><<<grid, kTuneThreads, 0, s>>>(tf2, spec, optics, Z, Y, Xh, X, eta,
                                                                           nu_max, zf, loss, partials)));
  } else {
    WO_LAUNCH("tune_cols", s, (k_tune_cols<1><<<grid, kTuneThreads, 0, s>>>(tf2, spec, optics, Z, Y, Xh, X, eta,
                                                                           nu_max, zf, loss, partials)));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // F is the same in both forms; the residual sums carry the Parseval factor zf
  const double scale = 1.0 / ((double)X * (double)Y * (loss == WO_LOSS_MIDBAND ? 1.0 : (double)zf));
  WO_LAUNCH("tune_final", s, (k_tune_final<<<(unsigned)n_tiles, 32, 0, s>>>(partials, (int)nblk, np, scale, value,
                                                                             grad)));
  return cudaGetLastError();
}

// Vector-Jacobian product of the phase reconstruction with respect to the
// tuned optics: dL/dtheta_p = <g, d f/d theta_p> for an upstream gradient g
// of the reconstruction f (Parseval: (1/N) Re sum_nu conj(G) dF_p, the half
// spectrum weighted by w as above).  With the regulariser eta absolute:
//   3D (per 3D frequency):   F = conj(H) D / (|H|^2 + eta),
//     dF_p = (conj(dH_p) D - 2 Re(conj(H) dH_p) F) / (|H|^2 + eta);
//   2D (per transverse frequency, sums over the planes j):
//     F = sum_j conj(H_j) D_j / (sum_j |H_j|^2 + eta),
//     dF_p = (sum_j conj(dH_pj) D_j - 2 Re(sum_j conj(H_j) dH_pj) F) / (sum_j |H_j|^2 + eta).
// Partials hold 1 + NP doubles per block (slot 0 unused) so that k_tune_final
// reduces them.
template <int NP, bool MODE3D>
__global__ void __launch_bounds__(kTuneThreads) k_vjp_cols(const float2* __restrict__ tf2,
                                                           const float2* __restrict__ spec,
                                                           const float2* __restrict__ gspec, int Z, int Y, int Xh,
                                                           int X, float eta, double* __restrict__ partials) {
  __shared__ double red[(1 + NP) * kTuneThreads];
  const int t = blockIdx.y;
  const long long plane = (long long)Y * Xh;
  const long long vol = (long long)Z * plane;
  const long long c = (long long)blockIdx.x * kTuneThreads + threadIdx.x;
  double acc[1 + NP];
#pragma unroll
  for (int i = 0; i <= NP; ++i) acc[i] = 0.0;
  if (c < plane) {
    const int y = (int)(c / Xh), x = (int)(c - (long long)y * Xh);
    const double w = (x == 0 || 2 * x == X) ? 1.0 : 2.0;
    const float2* D = spec + (long long)t * vol + c;
    const float2* H = tf2 + (long long)t * (1 + NP) * vol + c;
    if constexpr (MODE3D) {
      const float2* G = gspec + (long long)t * vol + c;
      float gs[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) gs[q] = 0.f;
#pragma unroll 4
      for (int k = 0; k < Z; ++k) {
        const float2 d = __ldg(D + k * plane), h = __ldg(H + k * plane), g = __ldg(G + k * plane);
        const float den = cabs2(h) + eta;
        const float inv = den > 0.f ? 1.0f / den : 0.f;
        const float2 F = cscale(cmulc(h, d), inv);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const float2 dh = __ldg(H + (q + 1) * vol + k * plane);
          const float2 e = cmulc(dh, d);
          const float dhr = h.x * dh.x + h.y * dh.y;
          const float2 dF = make_float2((e.x - 2.f * dhr * F.x) * inv, (e.y - 2.f * dhr * F.y) * inv);
          gs[q] += g.x * dF.x + g.y * dF.y;  // Re(conj(G) dF)
        }
      }
#pragma unroll
      for (int q = 0; q < NP; ++q) acc[1 + q] = w * (double)gs[q];
    } else {
      float cr = 0.f, ci = 0.f, hh = 0.f, dcr[NP], dci[NP], dhr[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) dcr[q] = dci[q] = dhr[q] = 0.f;
#pragma unroll 4
      for (int k = 0; k < Z; ++k) {
        const float2 d = __ldg(D + k * plane), h = __ldg(H + k * plane);
        const float2 r = cmulc(h, d);
        cr += r.x;
        ci += r.y;
        hh += cabs2(h);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const float2 dh = __ldg(H + (q + 1) * vol + k * plane);
          const float2 e = cmulc(dh, d);
          dcr[q] += e.x;
          dci[q] += e.y;
          dhr[q] += h.x * dh.x + h.y * dh.y;
        }
      }
      const float den = hh + eta;
      const float inv = den > 0.f ? 1.0f / den : 0.f;
      const float2 F = make_float2(cr * inv, ci * inv);
      const float2 g = __ldg(gspec + (long long)t * plane + c);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const float2 dF = make_float2((dcr[q] - 2.f * dhr[q] * F.x) * inv, (dci[q] - 2.f * dhr[q] * F.y) * inv);
        acc[1 + q] = w * ((double)g.x * dF.x + (double)g.y * dF.y);
      }
    }
  }
  block_sum<1 + NP>(acc, red);
  if (threadIdx.x <= NP) partials[((long long)t * gridDim.x + blockIdx.x) * (1 + NP) + threadIdx.x] =
      red[threadIdx.x * kTuneThreads];
}

cudaError_t vjp_reduce(const float2* tf2, const float2* spec, const float2* gspec, int n_tiles, int Z, int Y, int X,
                       float eta, int mode3d, int np, double* partials, double* grad, cudaStream_t s) {
  const int Xh = X / 2 + 1;
  const long long plane = (long long)Y * Xh;
  const unsigned nblk = (unsigned)((plane + kTuneThreads - 1) / kTuneThreads);
  dim3 grid(nblk, (unsigned)n_tiles);
  if (np == 4 && !mode3d) {
    WO_LAUNCH("vjp_cols", s, (k_vjp_cols<4, false><<<grid, kTuneThreads, 0, s>>>(tf2, spec, gspec, Z, Y, Xh, X, eta,
                                                                                partials)));
  } else if (np == 1 && !mode3d) {
    WO_LAUNCH("vjp_cols", s, (k_vjp_cols<1, false><<<grid, kTuneThreads, 0, s>>>(tf2, spec, gspec, Z, Y, Xh, X, eta,
                                                                                partials)));
  } else if (np == 1) {
    WO_LAUNCH("vjp_cols", s, (k_vjp_cols<1, true><<<grid, kTuneThreads, 0, s>>>(tf2, spec, gspec, Z, Y, Xh, X, eta,
                                                                               partials)));
  } else {
    return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const double scale = 1.0 / ((double)X * (double)Y * (mode3d ? (double)Z : 1.0));
  WO_LAUNCH("tune_final", s, (k_tune_final<<<(unsigned)n_tiles, 32, 0, s>>>(partials, (int)nblk, np, scale, nullptr,
                                                                             grad)));
  return cudaGetLastError();
}

size_t tune_partials_bytes(int n_tiles, int Y, int X, int np) {
  const long long plane = (long long)Y * (X / 2 + 1);
  return (size_t)n_tiles * (size_t)((plane + kTuneThreads - 1) / kTuneThreads) * (1 + np) * sizeof(double);
}

__global__ void k_zero_dc(float2* spec, int n_tiles, long long vol) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_tiles) spec[(long long)t * vol] = make_float2(0.f, 0.f);
}

cudaError_t zero_dc(float2* spec, int n_tiles, long long vol, cudaStream_t s) {
  WO_LAUNCH("zero_dc", s, (k_zero_dc<<<(unsigned)((n_tiles + 127) / 128), 128, 0, s>>>(spec, n_tiles, vol)));
  return cudaGetLastError();
}

// One warp per tile: subtract the mean of the Z per-plane DC bins from each.
__global__ void k_center_dc_planes(float2* spec, int n_tiles, int Z, long long plane) {
  const int t = blockIdx.x, lane = threadIdx.x;
  float2* base = spec + (long long)t * Z * plane;
  double sx = 0.0, sy = 0.0;
  for (int j = lane; j < Z; j += 32) {
    sx += base[(long long)j * plane].x;
    sy += base[(long long)j * plane].y;
  }
  for (int off = 16; off > 0; off >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, off);
    sy += __shfl_xor_sync(0xffffffffu, sy, off);
  }
  const float mx = (float)(sx / Z), my = (float)(sy / Z);
  __syncwarp();
  for (int j = lane; j < Z; j += 32) {
    float2& d = base[(long long)j * plane];
    d = make_float2(d.x - mx, d.y - my);
  }
}

cudaError_t center_dc_planes(float2* spec, int n_tiles, int Z, long long plane, cudaStream_t s) {
  WO_LAUNCH("center_dc", s, (k_center_dc_planes<<<(unsigned)n_tiles, 32, 0, s>>>(spec, n_tiles, Z, plane)));
  return cudaGetLastError();
}

// Adam (Kingma and Ba, 2015) on each tile's tuned optics parameters, in the
// order defocus_um, tilt_x, tilt_y, na_ill (the first np of them), with the
// moments and the step count kept in device memory: state[t][p] = {m, v, s}.
// NA_ill is kept inside [0.01, n_medium - |tilt| - 1e-3] after each step (a
// projection onto physically valid illumination).
__global__ void k_adam_optics(wo_optics* __restrict__ optics, const double* __restrict__ grad, int np,
                              double* __restrict__ state, int n_tiles, AdamLr lr, double b1, double b2,
                              double eps) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  wo_optics o = optics[t];
  double* par[4] = {&o.defocus_um, &o.tilt_x, &o.tilt_y, &o.na_ill};
  for (int p = 0; p < np; ++p) {
    double* st = state + (3LL * np) * t + 3 * p;
    const double g = grad[(long long)t * np + p];
    const double m = b1 * st[0] + (1.0 - b1) * g;
    const double v = b2 * st[1] + (1.0 - b2) * g * g;
    const double n = st[2] + 1.0;
    st[0] = m;
    st[1] = v;
    st[2] = n;
    const double mh = m / (1.0 - pow(b1, n));
    const double vh = v / (1.0 - pow(b2, n));
    *par[p] -= lr.v[p] * mh / (sqrt(vh) + eps);
  }
  if (np > 3) {
    const double tilt = sqrt(o.tilt_x * o.tilt_x + o.tilt_y * o.tilt_y);
    o.na_ill = fmin(fmax(o.na_ill, 0.01), o.n_medium - tilt - 1e-3);
  }
  optics[t] = o;
}

cudaError_t adam_optics(wo_optics* optics, const double* grad, int np, double* state, int n_tiles, AdamLr lr,
                        double b1, double b2, double eps, cudaStream_t s) {
  WO_LAUNCH("adam_optics", s,
            (k_adam_optics<<<(unsigned)((n_tiles + 127) / 128), 128, 0, s>>>(optics, grad, np, state, n_tiles, lr,
                                                                              b1, b2, eps)));
  return cudaGetLastError();
}

}  // namespace wo

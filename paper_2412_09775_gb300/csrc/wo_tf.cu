// wo_tf.cu - transfer-function build (Table 1, scalar column).
//
// The pupil correlations of Table 1 are formed through their point-spread
// functions.  With unnormalised inverse 2D transforms a = IDFT2(A_j),
// b = IDFT2(B_j), p = IDFT2(P_j) and g = conj(a) b:
//   H1_j = K DFT2(g),  K = c / (N_perp sum S P^2)
//   H_re_j = H1_j + H1_j(-q)* = DFT2(2K Re g),
//   H_im_j = i (H1_j - H1_j(-q)*) = DFT2(-2K Im g),
//   H_fl_j = DFT2(|p|^2) / (N_perp Z sum P^2)          (so that H_fl(0) = 1)
// so each TF is the 3D real-to-half-spectrum transform of a real PSF stack.
//
// Kernels, in order:
//   k_pupil_record  per (tile, y, x): pupil masks (float64 predicates, same
//                   operation order as the float64 reference), eta as a
//                   float pair, 1/eta, and the counts sum S P^2, sum P^2.
//   k_arms          per (tile, plane j, x strip): generate A_j, B_j, P_j in
//                   registers (defocus phase exp(i 2 pi eta z_j) with a
//                   float-pair product), inverse FFT along y.
//   k_psf_rows      per row: inverse FFT along x, form the real PSF rows,
//                   real-to-half-spectrum FFT along x into the TF bank.
//   (cols pass)     forward FFT along y in place in the TF bank.
//   k_tf_zpass      forward FFT along z in place, plus the per-tile maxima
//                   used by the relative regulariser.
#include "wo_fft.cuh"
#include "wo_internal.h"
#include "wo_tf.cuh"
#include "wo_zops.cuh"

namespace wo {

// One block per RY rows of one tile.  The frequency axes are computed once per
// block (the same IEEE divisions as the float64 reference); the mask
// predicates are exact float64 products and sums in the reference's order.
// eta = sqrt(k_m^2 - |nu|^2) takes a float seed and one float64 Newton
// correction (relative error ~1e-14, far below the float phase resolution).
// Rows per block: between 8 and 32, as many as keep about two blocks per SM
// busy (each block computes the x frequency axis once, with IEEE divisions).
constexpr int kRecRowsMax = 32;

int record_rows(int Y, int n_tiles) {
  const long long want = ((long long)Y * n_tiles + 303) / 304;
  return (int)(want < 8 ? 8 : (want > kRecRowsMax ? kRecRowsMax : want));
}

// Device-side copy of the host validation (wo_api.cu check_optics) for optics
// that live in device memory: 0 if valid, else the wo_status code.
__device__ int optics_status(const wo_optics& o) {
  const double v[9] = {o.lambda_um, o.n_medium, o.pixel_um, o.z_step_um, o.na_det,
                       o.na_ill, o.tilt_x, o.tilt_y, o.defocus_um};
  for (int i = 0; i < 9; ++i)
    if (!isfinite(v[i])) return WO_ERR_OPTICS;
  if (o.lambda_um <= 0 || o.n_medium <= 0 || o.pixel_um <= 0 || o.z_step_um <= 0) return WO_ERR_OPTICS;
  if (o.na_det <= 0 || o.na_det >= o.n_medium) return WO_ERR_OPTICS;
  const double tilt = sqrt(o.tilt_x * o.tilt_x + o.tilt_y * o.tilt_y);
  if (o.na_ill < 0 || o.na_ill + tilt > o.n_medium) return WO_ERR_OPTICS;
  if ((o.na_det + o.na_ill + tilt) / o.lambda_um >= 1.0 / (2.0 * o.pixel_um)) return WO_ERR_UNDERSAMPLED;
  const double s = o.na_det / o.n_medium;
  if ((o.n_medium / o.lambda_um) * (1.0 - sqrt(1.0 - s * s)) >= 1.0 / (2.0 * o.z_step_um)) return WO_ERR_UNDERSAMPLED;
  return WO_OK;
}

// Noll's index j >= 1 -> radial order n and |m|; cos(|m| phi) for even j,
// sin(|m| phi) for odd j (m != 0).  Within order n (indices n(n+1)/2 + 1 ..
// n(n+1)/2 + n + 1) |m| runs 0 or 1, then pairs of 2, 4, ... or 3, 5, ...
__device__ __forceinline__ void noll_index(int j, int& n, int& am) {
  n = 0;
  while ((n + 1) * (n + 2) / 2 < j) ++n;
  const int p = j - n * (n + 1) / 2 - 1;
  am = 2 * ((p + 1 - (n & 1)) / 2) + (n & 1);
}

// Aberration phase W = sum_j c_j Z_j at the unit-pupil point (ux, uy),
// |u| <= 1, in waves.  Z_j = N_j R_n^|m|(rho) {cos, sin}(|m| phi) with
// rho^|m| {cos, sin}(|m| phi) = {Re, Im} (ux + i uy)^|m| and
// R_n^|m|(rho) = rho^|m| P_k^(0,|m|)(2 rho^2 - 1), k = (n - |m|)/2, the Jacobi
// polynomial by its three-term recurrence (stable in float on [-1, 1]).
// zc: the tile's coefficients pre-multiplied by N_j; zn, zm: n and signed m.
__device__ float aberration_waves(float ux, float uy, const float* zc, const signed char* zn,
                                  const signed char* zm, int nz) {
  const float x = 2.f * (ux * ux + uy * uy) - 1.f;
  float W = 0.f;
  for (int q = 0; q < nz; ++q) {
    const float c = zc[q];
    if (c == 0.f) continue;
    const int m = zm[q], am = m < 0 ? -m : m, k = (zn[q] - am) / 2;
    float re = 1.f, im = 0.f;
    for (int i = 0; i < am; ++i) {
      const float t = re * ux - im * uy;
      im = fmaf(re, uy, im * ux);
      re = t;
    }
    const float ang = m > 0 ? re : (m < 0 ? im : 1.f);
    const float b = (float)am;
    float p0 = 1.f, p1 = 0.5f * ((b + 2.f) * x - b);
    float pk = k == 0 ? p0 : p1;
    for (int i = 1; i < k; ++i) {  // P_{i+1} from P_i and P_{i-1}
      const float s2 = 2.f * i + b;
      const float a1 = 2.f * (i + 1) * (i + b + 1.f) * s2;
      const float a2 = -(s2 + 1.f) * b * b;
      const float a3 = s2 * (s2 + 1.f) * (s2 + 2.f);
      const float a4 = 2.f * i * (i + b) * (s2 + 2.f);
      const float p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
      p0 = p1;
      p1 = p2;
      pk = p2;
    }
    W = fmaf(c * ang, pk, W);
  }
  return W;
}

__global__ void __launch_bounds__(256) k_pupil_record(TfArgs a, int kRecRows) {
  extern __shared__ double nu_x[];  // [X]
  __shared__ double nu_y[kRecRowsMax];
  __shared__ int part[2][8];
  __shared__ float fpart[4][8];
  __shared__ float zc[WO_MAX_ZERNIKE];
  __shared__ signed char zn[WO_MAX_ZERNIKE], zm[WO_MAX_ZERNIKE];
  const bool want_rec2 = a.want_grad || a.n_zern > 0;
  const int Y = a.Y, X = a.X;
  const int t = blockIdx.y;
  const int y0 = blockIdx.x * kRecRows;
  const wo_optics o = a.optics[t];
  float4* rec = a.rec;
  // The tile's status and float64 constants are formed once per block
  // (float64 is slow on this part) and shared.
  __shared__ int status_sh;
  __shared__ double cst[8];  // rp2, cy, cx, rs, rs2, km2, 1/rp, wedge
  if (threadIdx.x == 0) {
    status_sh = optics_status(o);
    const double lam = o.lambda_um;
    const double rp = __ddiv_rn(o.na_det, lam);
    cst[0] = __dmul_rn(rp, rp);
    cst[1] = __ddiv_rn(o.tilt_y, lam);
    cst[2] = __ddiv_rn(o.tilt_x, lam);
    cst[3] = __ddiv_rn(o.na_ill, lam);
    cst[4] = __dmul_rn(cst[3], cst[3]);
    const double km = __ddiv_rn(o.n_medium, lam);
    cst[5] = __dmul_rn(km, km);
    cst[6] = 1.0 / rp;
    cst[7] = 1.0 / ((double)min(Y, X) * o.pixel_um);
  }
  __syncthreads();
  // Invalid optics (possible only when they come from device memory): the
  // tile's record is all zero, so its transfer functions are zero, and its
  // status is left in the statistics block.
  const int status = status_sh;
  if (status != WO_OK) {
    for (int e = threadIdx.x; e < kRecRows * X; e += 256) {
      const int yy = e / X;
      if (y0 + yy >= Y) continue;
      const long long i = ((long long)t * Y + y0 + yy) * X + (e - yy * X);
      rec[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (want_rec2) a.rec2[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (a.smooth && threadIdx.x < 4) a.norm_part[((long long)t * a.rec_blocks + blockIdx.x) * 4 + threadIdx.x] = 0.f;
    if (blockIdx.x == 0 && threadIdx.x == 0) reinterpret_cast<int*>(a.stats)[(long long)t * 8 + 4] = status;
    return;  // uniform across the block
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // support radius of the tile's TFs (cycles per pixel, two bins of margin):
    // H1(q) needs nu in S and P and nu + q in P; the fluorescence TF and the
    // smooth source (nonzero wherever P is) reach 2 NA_det / lambda
    const double tilt = sqrt(o.tilt_x * o.tilt_x + o.tilt_y * o.tilt_y);
    double r = 0.0;
    if (a.lf_props > 0) r = a.smooth ? 2.0 * o.na_det : o.na_det + fmin(o.na_det, o.na_ill + tilt);
    if (a.want_fl) r = fmax(r, 2.0 * o.na_det);
    a.stats[(long long)t * 8 + 5] = (float)(r / o.lambda_um * o.pixel_um + 2.0 / (double)min(Y, X));
  }
  const double px = __dmul_rn((double)X, o.pixel_um), py = __dmul_rn((double)Y, o.pixel_um);
  for (int x = threadIdx.x; x < X; x += 256) nu_x[x] = __ddiv_rn((double)fft_index(x, X), px);
  if (threadIdx.x < kRecRows && y0 + threadIdx.x < Y)
    nu_y[threadIdx.x] = __ddiv_rn((double)fft_index(y0 + threadIdx.x, Y), py);
  if (threadIdx.x < a.n_zern) {
    int n, am;
    noll_index(threadIdx.x + 1, n, am);
    const int m = am == 0 ? 0 : (((threadIdx.x + 1) & 1) ? -am : am);
    const double norm = sqrt(am == 0 ? (double)(n + 1) : 2.0 * (n + 1));
    zc[threadIdx.x] = (float)(a.zern[(long long)t * a.n_zern + threadIdx.x] * norm);
    zn[threadIdx.x] = (signed char)n;
    zm[threadIdx.x] = (signed char)m;
  }
  __syncthreads();
  const double lam = o.lambda_um;
  const double rp2 = cst[0], cy = cst[1], cx = cst[2], rs = cst[3], rs2 = cst[4], km2 = cst[5];
  // float images of the constants for the mask pre-test: a predicate is
  // settled in float when the float value is clear of the threshold by a
  // margin far above the float error; otherwise the float64 expression decides
  const float rp2f = (float)rp2, rs2f = (float)rs2, cxf = (float)cx, cyf = (float)cy;
  const float mp = 1e-5f * rp2f;
  // smooth source: S = 1 / (1 + exp(-(R - d) / w)), w one frequency bin of the
  // coarser axis, and its derivatives in tilt and NA_ill
  const float rsf = (float)rs, lamf = (float)lam;
  const float inv_rp = (float)cst[6];  // unit-pupil coordinates of the aberration
  const float wedge = (float)cst[7];
  int n_sp = 0, n_p = 0, kx_band = -1;
  float s_sp = 0.f, s_tx = 0.f, s_ty = 0.f, s_na = 0.f;
  const int rows = min(kRecRows, Y - y0);
  for (int e = threadIdx.x; e < rows * X; e += 256) {
    const int yy = e / X, x = e - (e / X) * X;
    const double vy = nu_y[yy], vx = nu_x[x];
    const float vyf = (float)vy, vxf = (float)vx;
    const float r2f = vxf * vxf + vyf * vyf;
    bool P;
    if (r2f < rp2f - mp) P = true;
    else if (r2f > rp2f + mp) P = false;
    else P = __dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)) <= rp2;
    float S = 0.f, dtx = 0.f, dty = 0.f, dna = 0.f;
    if (P && a.smooth) {
      const float ux = vxf - cxf, uy = vyf - cyf;
      const float d = sqrtf(ux * ux + uy * uy);
      S = 1.0f / (1.0f + expf(-(rsf - d) / wedge));
      const float ds = S * (1.0f - S) / wedge;
      dna = ds / lamf;
      if (d > 0.f) {
        dtx = ds * ux / (d * lamf);
        dty = ds * uy / (d * lamf);
      }
    } else if (P) {
      const float dxf = vxf - cxf, dyf = vyf - cyf;
      const float s2f = dxf * dxf + dyf * dyf;
      // the float error of s2f scales with (|nu| + |c|)^2, not with rs^2
      const float ax = fabsf(vxf) + fabsf(cxf), ay = fabsf(vyf) + fabsf(cyf);
      const float ms = 1e-5f * rs2f + 4e-6f * (ax * ax + ay * ay) + 1e-9f;
      bool Sb;
      if (s2f < rs2f - ms) Sb = true;
      else if (s2f > rs2f + ms) Sb = false;
      else {
        const double dy = __dsub_rn(vy, cy), dx = __dsub_rn(vx, cx);
        Sb = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= rs2;
      }
      S = Sb ? 1.f : 0.f;
    }
    // eta (as a float pair) is used only inside the detection pupil, where
    // every arm lives; elsewhere the record holds zeros
    float eh = 0.f, el = 0.f, binv = 0.f;
    if (P) {
      const double r2 = __dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy));
      const double e2 = __dsub_rn(km2, r2);
      if (e2 > 0.0) {
        const float s0 = sqrtf((float)e2);
        const double rem = fma(-(double)s0, (double)s0, e2);
        const double eta = (double)s0 + (double)((float)rem * (0.5f / s0));
        eh = __double2float_rn(eta);
        el = __double2float_rn(__dsub_rn(eta, (double)eh));
        binv = 1.0f / eh;
      }
    }
    float wfrac = 0.f;
    if (P && a.n_zern > 0) {
      const float W = aberration_waves(vxf * inv_rp, vyf * inv_rp, zc, zn, zm, a.n_zern);
      wfrac = W - rintf(W);
    }
    const long long i = ((long long)t * Y + y0 + yy) * X + x;
    rec[i] = make_float4(eh, el, binv, S);  // S is 0 outside P
    if (want_rec2) a.rec2[i] = make_float4(dtx, dty, dna, wfrac);
    n_sp += (S != 0.f) ? 1 : 0;
    n_p += P ? 1 : 0;
    s_sp += S;
    s_tx += dtx;
    s_ty += dty;
    s_na += dna;
    // band limit along x: the largest |k_x| inside P on the k_y = 0 row.  P is
    // contained in nu_x^2 <= (NA_det/lambda)^2, so every column beyond it is
    // zero in every arm.
    if (y0 + yy == 0 && P) kx_band = max(kx_band, abs(fft_index(x, X)));
  }
  for (int off = 16; off > 0; off >>= 1) {
    n_sp += __shfl_down_sync(0xffffffffu, n_sp, off);
    n_p += __shfl_down_sync(0xffffffffu, n_p, off);
    kx_band = max(kx_band, __shfl_down_sync(0xffffffffu, kx_band, off));
    s_sp += __shfl_down_sync(0xffffffffu, s_sp, off);
    s_tx += __shfl_down_sync(0xffffffffu, s_tx, off);
    s_ty += __shfl_down_sync(0xffffffffu, s_ty, off);
    s_na += __shfl_down_sync(0xffffffffu, s_na, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ int band[8];
  if (lane == 0) {
    part[0][warp] = n_sp;
    part[1][warp] = n_p;
    band[warp] = kx_band;
    fpart[0][warp] = s_sp;
    fpart[1][warp] = s_tx;
    fpart[2][warp] = s_ty;
    fpart[3][warp] = s_na;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int ca = 0, cb = 0, k = -1;
    for (int i = 0; i < 8; ++i) {
      ca += part[0][i];
      cb += part[1][i];
      k = max(k, band[i]);
    }
    if (ca) atomicAdd(&a.counts[4 * t], ca);
    if (cb) atomicAdd(&a.counts[4 * t + 1], cb);
    if (k >= 0) atomicMax(&a.counts[4 * t + 2], k);
  }
  // smooth source: per-block partial sums, reduced per tile in a fixed order
  if (a.smooth && threadIdx.x < 4) {
    float v = 0.f;
    for (int i = 0; i < 8; ++i) v += fpart[threadIdx.x][i];
    a.norm_part[((long long)t * a.rec_blocks + blockIdx.x) * 4 + threadIdx.x] = v;
  }
}

// Per tile: the four smooth-source sums from the record blocks' partials.
__global__ void k_norms(const float* __restrict__ part, int blocks, int n_tiles, float* __restrict__ norms) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // tile * 4 + sum
  if (i >= 4 * n_tiles) return;
  const int t = i / 4, q = i % 4;
  double v = 0.0;
  for (int b = 0; b < blocks; ++b) v += part[((long long)t * blocks + b) * 4 + q];
  norms[i] = (float)v;
}

template <int N, bool DER>  // N = Y; DER: a derivative bank (arms A', B' and the source ones)
__global__ void __launch_bounds__(ColGeom<N>::NT, (1024 / ColGeom<N>::NT) > 1 ? (1024 / ColGeom<N>::NT) : 1) k_arms(TfArgs a) {
  using G = ColGeom<N>;
  constexpr int B = G::B, NT = G::NT;
  constexpr int PER = (N * B + NT - 1) / NT;
  extern __shared__ float2 sm[];
  float2* buf = sm;
  float2* tw = sm + N * B;
  // derivative banks: eta and the source derivatives of the strip, staged
  // once (each arm that needs them reads them from here)
  float* eta_s = reinterpret_cast<float*>(tw + N);  // [N*B]
  float* ds_s = eta_s + N * B;                       // [3][N*B]
  const int X = a.X, Z = a.Z;
  const int t = blockIdx.z, j = blockIdx.y, x0 = blockIdx.x * B;
  const int w = min(B, X - x0);
  // skip strips whose columns all lie outside the detection band: every arm
  // is exactly zero there, and the row pass never reads those columns
  const int kxmax = a.counts[4 * t + 2];
  bool active = false;
  for (int b = 0; b < w; ++b) active |= abs(fft_index(x0 + b, X)) <= kxmax;
  if (!active) return;  // uniform across the CTA
#if defined(WO_CHECK) && WO_CHECK
  {  // the strip's records and the arm strips it writes
    const long long nt = gridDim.z;
    if (!WO_IN((long long)t * N * X + x0 + (long long)(N - 1) * X + w - 1, nt * N * X, 8) ||
        !WO_IN((((long long)t * a.n_arms + a.n_arms - 1) * Z + j) * (long long)N * X + x0 + (long long)(N - 1) * X + w - 1,
               nt * a.n_arms * Z * (long long)N * X, 8))
      return;
  }
#endif
  make_twiddles<N>(tw);
  // the plane's focal displacement as a float pair, formed in float64 by one
  // lane of each warp (float64 is slow on this part) and broadcast
  float zh = 0.f, zl = 0.f;
  if ((threadIdx.x & 31) == 0) {
    const double zj = __dadd_rn(__dmul_rn((double)fft_index(j, Z), a.optics[t].z_step_um), a.optics[t].defocus_um);
    zh = __double2float_rn(zj);
    zl = __double2float_rn(__dsub_rn(zj, (double)zh));
  }
  zh = __shfl_sync(0xffffffffu, zh, 0);
  zl = __shfl_sync(0xffffffffu, zl, 0);
  const float4* rec = a.rec + (long long)t * N * X + x0;
  float4 r[PER];
  float s_[PER], c_[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * NT;
    const int n = e / B, b = e % B;
    r[i] = (e < N * B && b < w) ? __ldg(rec + (long long)n * X + b) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const bool stage = DER && a.arms_stage != 0;
  if (stage && a.want_dz) {
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + i * NT;
      if (e < N * B) eta_s[e] = r[i].x;  // zero outside the strip's width (r is zero there)
    }
  }
  if (stage && a.want_grad) {
    const float4* rec2 = a.rec2 + (long long)t * N * X + x0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + i * NT;
      if (e >= N * B) continue;
      const float4 d = (e % B) < w ? __ldg(rec2 + (long long)(e / B) * X + e % B) : make_float4(0.f, 0.f, 0.f, 0.f);
      ds_s[e] = d.x;
      ds_s[N * B + e] = d.y;
      ds_s[2 * N * B + e] = d.z;
    }
  }
  // (read after the first arm's barrier)
  // an aberrated detection pupil adds W (waves, reduced to [-1/2, 1/2]) to every arm's phase
  const float* wrec = a.n_zern > 0 ? reinterpret_cast<const float*>(a.rec2 + (long long)t * N * X + x0) + 3 : nullptr;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * NT;
    float ph = phase_frac(r[i].x, r[i].y, zh, zl);
    if (wrec && e < N * B && (e % B) < w) ph += __ldg(wrec + 4 * ((long long)(e / B) * X + e % B));
    unit_phasor(ph, &s_[i], &c_[i]);
  }
  // arms, in slot order: A, B (label-free), P (fluorescence), or
  // A, B, A' = i 2 pi eta A, B' = i 2 pi eta B (phase TF and its defocus
  // derivative), then A_tx, A_ty, A_NA (derivatives in the source parameters)
  int arm = 0;
#pragma unroll 1
  for (int which = 0; which < (DER ? 8 : 3); ++which) {
    if (which < 2 && a.lf_props == 0) continue;
    if (which == 2 && !a.want_fl) continue;
    if ((which == 3 || which == 4) && !a.want_dz) continue;
    if (which > 4 && !a.want_grad) continue;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + i * NT;
      if (e >= N * B) continue;
      // v = (al + i be) e^{i phi}: A (S, 0), B (0, 1/eta), P (1, 0),
      // A' (0, 2 pi eta S), B' (-2 pi eta / eta, 0), and for the source
      // parameters A_theta (dS/dtheta, 0); zero off the pupil.  S (the
      // record's w) is 0 or 1 for the binary source.  eta and the source
      // derivatives come from the strip's staged copies (or, where they do
      // not fit shared memory, from the records again: L2 hits)
      float tpe = 0.f, dsv = 0.f;
      const bool inb = (e % B) < w;
      if (which == 3 || which == 4)
        tpe = 6.28318530717958648f * (stage ? eta_s[e] : (inb ? __ldg(&rec[(long long)(e / B) * X + e % B].x) : 0.f));
      if (which > 4) {
        if (stage) {
          dsv = ds_s[(which - 5) * N * B + e];
        } else if (inb) {
          const float* r2 = reinterpret_cast<const float*>(a.rec2 + (long long)t * N * X + x0 +
                                                           (long long)(e / B) * X + e % B);
          dsv = __ldg(r2 + (which - 5));
        }
      }
      float al = which == 0 ? r[i].w : (which == 2 ? (r[i].z != 0.f ? 1.f : 0.f)
                                        : (which == 4 ? -tpe * r[i].z : (which > 4 ? dsv : 0.f)));
      float be = which == 1 ? r[i].z : (which == 3 ? tpe * r[i].w : 0.f);
      buf[e] = make_float2(al * c_[i] - be * s_[i], al * s_[i] + be * c_[i]);
    }
    __syncthreads();
    fft_smem<N, B, NT, true, 1>(buf, B, 1, tw);
    float2* dst = a.arms + (((long long)t * a.n_arms + arm) * Z + j) * (long long)N * X + x0;
    for (int e = threadIdx.x; e < N * B; e += NT) {
      const int n = e / B, b = e % B;
      if (b < w) dst[(long long)n * X + b] = buf[e];
    }
    __syncthreads();
    ++arm;
  }
}

template <int NX>
struct PsfGeom {
  static constexpr int B = (NX <= 1024) ? 8 : 4;  // rows per CTA (a power of two: the swizzle width)
  static constexpr int NT = threads_for(NX * B);
  static constexpr int MINB = (1024 / NT) > 1 ? (1024 / NT) : 1;
  static constexpr int SLOT = NX * B + B;  // elements per arm slot (up to four arms)
};

// Per row (tile t, plane j, row y) of the arms after their y transform:
// inverse transform along x of every arm, then the PSF rows and their forward
// transform along x.  The label-free PSFs are the real and imaginary parts of
// g = 2K conj(a) b, so one complex transform G of g gives both rows:
//   H_re(k) = (G(k) + G*(-k)) / 2,   H_im(k) = i (G(k) - G*(-k)) / 2.
// The fluorescence PSF |p|^2 / (N_perp Z sum P^2) is transformed as a complex
// row with zero imaginary part.  Each arm's B rows sit in their own slot,
// element n of row b at n * B + (b ^ (n & (B-1))) (SwzAddr): the coalesced
// row copies and the transform stages are both free of bank conflicts.
template <int NX>
__global__ void __launch_bounds__(PsfGeom<NX>::NT, PsfGeom<NX>::MINB) k_psf_rows(TfArgs a) {
  using G = PsfGeom<NX>;
  constexpr int B = G::B, NT = G::NT, H = NX / 2, SLOT = G::SLOT;
  using Addr = SwzAddr<B, NX>;
  const Addr addr{};
  extern __shared__ float2 sm[];
  float2* buf = sm;                              // [n_arms][SLOT]
  float2* tw = sm + a.n_arms * SLOT;             // exp(-2 pi i m / NX)
  float* sc = reinterpret_cast<float*>(tw + NX); // [B] label-free 2K, [B] fluorescence scale
  int* kxm = reinterpret_cast<int*>(sc + 2 * B); // [B] x band limit of the row's tile
  const long long nrows = a.row_end;
  const long long row0 = a.row_begin + (long long)blockIdx.x * B;
  const int na = a.n_arms;
  const bool lf = a.lf_props > 0, fl = a.want_fl != 0;
  if (threadIdx.x < B) {
    const long long row = row0 + threadIdx.x;
    const int t = (int)((row < nrows ? row : nrows - 1) / ((long long)a.Z * a.Y));
    sc[threadIdx.x] = lf_scale(a, t);
    sc[B + threadIdx.x] = fl_scale(a, t);
    kxm[threadIdx.x] = row < nrows ? a.counts[4 * t + 2] : -1;
  }
  __syncthreads();
  const long long plane_elems = (long long)a.Y * NX;
  // columns outside the detection band are zero (and were never written)
  for (int e = threadIdx.x; e < na * B * NX; e += NT) {
    const int q = e / NX, n = e - (e / NX) * NX;  // q = arm * B + b
    const int arm = q / B, b = q - (q / B) * B;
    const long long row = row0 + b;
    const bool ok = abs(fft_index(n, NX)) <= kxm[b];
    const float2* src = a.arms;
    if (ok) {
      const long long t = row / ((long long)a.Z * a.Y);
      const long long rem = row - t * a.Z * a.Y;  // j*Y + y
      src = a.arms + ((t * na + arm) * a.Z) * plane_elems + rem * NX + n;
    }
    cp_async8(buf + addr(n, q), src, ok);
  }
  make_twiddles<NX>(tw);
  cp_async_wait_all();
  __syncthreads();
  for (int arm = 0; arm < na; ++arm) fft_smem_a<NX, B, NT, true, 1>(buf + arm * SLOT, addr, tw);
  // PSF rows: slot 0 <- 2K conj(a) b (label-free), slot fl_dst <- fluorescence
  const int fl_src = lf ? 2 : 0, fl_dst = lf ? 1 : 0;
  for (int e = threadIdx.x; e < B * NX; e += NT) {
    const int n = e / B, b = e - (e / B) * B;
    const int i = addr(n, b);  // same position in every slot
    if (a.want_dz) {  // slot 0 <- 2K conj(a) b, slot 1 <- 2K (conj(a') b + conj(a) b')
      const float2 va = buf[i], vb = buf[SLOT + i], vad = buf[2 * SLOT + i], vbd = buf[3 * SLOT + i];
      buf[i] = cscale(cmulc(va, vb), sc[b]);
      buf[SLOT + i] = cscale(cadd(cmulc(vad, vb), cmulc(va, vbd)), sc[b]);
      continue;
    }
    if (lf) buf[i] = cscale(cmulc(buf[i], buf[SLOT + i]), sc[b]);
    if (fl) {
      const float2 p = buf[fl_src * SLOT + i];
      buf[fl_dst * SLOT + i] = make_float2(sc[B + b] * cabs2(p), 0.f);
    }
  }
  __syncthreads();
  const int nf = a.want_dz ? 2 : (lf ? 1 : 0) + (fl ? 1 : 0);
  for (int sl = 0; sl < nf; ++sl) fft_smem_a<NX, B, NT, false, 1>(buf + sl * SLOT, addr, tw);
  const int Z = a.Z, Y = a.Y, Xh = H + 1;
  for (int e = threadIdx.x; e < B * Xh; e += NT) {
    const int b = e / Xh, k = e - (e / Xh) * Xh;
    const long long row = row0 + b;
    if (row >= nrows) continue;
    const long long plane = row / Y;  // t*Z + j
    const int y = (int)(row - plane * Y);
    const long long t = plane / Z, j = plane - (plane / Z) * Z;
    float2* dst = a.tf + ((t * a.n_kinds * Z + j) * Y + y) * Xh + k;  // slot 0 of this row
    const long long kstride = (long long)Z * Y * Xh;
    int slot = 0;
    if (a.want_dz) {  // H_re of g and of g' (the map g -> H_re is linear)
      for (int q = 0; q < 2; ++q) {
        const float2 gk = buf[q * SLOT + addr(k, b)];
        const float2 gc = cconj(buf[q * SLOT + addr(k == 0 ? 0 : NX - k, b)]);
        dst[q * kstride] = make_float2(0.5f * (gk.x + gc.x), 0.5f * (gk.y + gc.y));
      }
      continue;
    }
    if (lf) {
      const float2 gk = buf[addr(k, b)];
      const float2 gc = cconj(buf[addr(k == 0 ? 0 : NX - k, b)]);
      if (a.want_phase) dst[(slot++) * kstride] = make_float2(0.5f * (gk.x + gc.x), 0.5f * (gk.y + gc.y));
      if (a.want_abs) dst[(slot++) * kstride] = make_float2(-0.5f * (gk.y - gc.y), 0.5f * (gk.x - gc.x));
    }
    if (fl) dst[slot * kstride] = buf[fl_dst * SLOT + addr(k, b)];
  }
}

template <int N, int NK>  // N = Z, NK transfer functions per tile
__global__ void __launch_bounds__(ZGeom<N, NK>::NT, ZGeom<N, NK>::MINB) k_tf_zpass(TfArgs a) {
  using G = ZGeom<N, NK>;
  constexpr int B = G::B, NT = G::NT, KK = NT / B;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;  // [n][kind][b]
  float* red = reinterpret_cast<float*>(buf + NK * N * B);  // [NT][2]
  const int Y = a.Y, Xh = a.X / 2 + 1;
  const int t = blockIdx.z, y = blockIdx.y, x0 = blockIdx.x * B;
  const int w = min(B, Xh - x0);
  const long long zs = (long long)Y * Xh;
  const long long vol = (long long)N * zs;
  float2* base = a.tf + (long long)t * NK * vol + (long long)y * Xh + x0;
  load_zcols<N, NK, B, NT>(buf, base, NK, vol, zs, w);
  make_twiddles<N>(tw);
  cp_async_wait_all();
  __syncthreads();
  fft_smem<N, NK * B, NT, false, 1>(buf, NK * B, 1, tw);
  const int L = a.lf_props;
  float m3_lf = 0.f, m3_fl = 0.f, col_lf = 0.f, col_fl = 0.f;
  const int b = threadIdx.x % B;  // fixed per thread: NT is a multiple of 32 and B divides 32
  if (b < w) {
    for (int e = threadIdx.x; e < N * B; e += NT) {
      const int n = e / B;
      const float2* cell = buf + n * NK * B + b;
      float lf = 0.f;
      for (int s = 0; s < L; ++s) lf += cabs2(cell[s * B]);
      m3_lf = fmaxf(m3_lf, lf);
      col_lf += lf;
      if (a.want_fl) {
        const float fl = cabs2(cell[L * B]);
        m3_fl = fmaxf(m3_fl, fl);
        col_fl += fl;
      }
    }
  }
  store_zcols<N, NK, B, NT>(buf, base, NK, vol, zs, w);
  red[2 * threadIdx.x] = col_lf;
  red[2 * threadIdx.x + 1] = col_fl;
  __syncthreads();
  float m2_lf = 0.f, m2_fl = 0.f;
  if (threadIdx.x < B && threadIdx.x < w) {
    for (int q = 0; q < KK; ++q) {
      m2_lf += red[2 * (q * B + threadIdx.x)];
      m2_fl += red[2 * (q * B + threadIdx.x) + 1];
    }
  }
  // block maxima (values are >= 0, so integer order equals float order):
  // warp shuffles, then one atomic per statistic per CTA
  for (int off = 16; off > 0; off >>= 1) {
    m3_lf = fmaxf(m3_lf, __shfl_down_sync(0xffffffffu, m3_lf, off));
    m3_fl = fmaxf(m3_fl, __shfl_down_sync(0xffffffffu, m3_fl, off));
    m2_lf = fmaxf(m2_lf, __shfl_down_sync(0xffffffffu, m2_lf, off));
    m2_fl = fmaxf(m2_fl, __shfl_down_sync(0xffffffffu, m2_fl, off));
  }
  __syncthreads();  // red[] is reused below
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[4 * warp + 0] = m3_lf;
    red[4 * warp + 1] = m2_lf;
    red[4 * warp + 2] = m3_fl;
    red[4 * warp + 3] = m2_fl;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    float m = 0.f;
    for (int q = 0; q < NT / 32; ++q) m = fmaxf(m, red[4 * q + threadIdx.x]);
    if (m > 0.f) atomicMax(reinterpret_cast<int*>(a.stats + (long long)t * 8) + threadIdx.x, __float_as_int(m));
  }
}

cudaError_t tf_pupil_record(const TfArgs& a, cudaStream_t s) {
  const int kRecRows = record_rows(a.Y, a.n_tiles);
  dim3 grid((unsigned)((a.Y + kRecRows - 1) / kRecRows), (unsigned)a.n_tiles);
  const size_t smem = (size_t)a.X * sizeof(double);
  WO_LAUNCH("tf_pupil_record", s,
            (k_pupil_record<<<grid, 256, smem, s>>>(a, kRecRows)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !a.smooth) return e;
  WO_LAUNCH("tf_norms", s, (k_norms<<<(unsigned)((4 * a.n_tiles + 127) / 128), 128, 0, s>>>(a.norm_part, a.rec_blocks,
                                                                                          a.n_tiles, a.norms)));
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_arms(const TfArgs& a, cudaStream_t s) {
  using G = ColGeom<N>;
  // plus eta (derivative banks) and three source derivatives (gradient bank)
  constexpr size_t kStage = (size_t)N * G::B * sizeof(float);
  constexpr size_t kMax = 227 * 1024;
  constexpr size_t kCap = G::SMEM + 4 * kStage <= kMax ? G::SMEM + 4 * kStage : kMax;
  const cudaError_t attr0 = allow_smem(k_arms<N, false>, G::SMEM);
  const cudaError_t attr1 = allow_smem(k_arms<N, true>, kCap);
  if (attr0 != cudaSuccess) return attr0;
  if (attr1 != cudaSuccess) return attr1;
  TfArgs b = a;
  size_t smem = G::SMEM + (a.want_dz ? kStage : 0) + (a.want_grad ? 3 * kStage : 0);
  b.arms_stage = smem <= kCap ? 1 : 0;
  if (!b.arms_stage) smem = G::SMEM;
  dim3 grid((unsigned)((a.X + G::B - 1) / G::B), (unsigned)a.Z, (unsigned)a.n_tiles);
  if (a.want_dz) {
    WO_LAUNCH("tf_arms", s, (k_arms<N, true><<<grid, G::NT, smem, s>>>(b)));
  } else {
    WO_LAUNCH("tf_arms", s, (k_arms<N, false><<<grid, G::NT, smem, s>>>(b)));
  }
  return cudaGetLastError();
}

cudaError_t tf_arms(const TfArgs& a, cudaStream_t s) {
  if (arms_reg_supported(a.Y, a)) return tf_arms_reg(a, s);
  switch (a.Y) {
#define WO_CASE(n) \
  case n:          \
    return launch_arms<n>(a, s);
    WO_FOR_EACH_SIZE(WO_CASE)
#undef WO_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <int NX>
static cudaError_t launch_psf(const TfArgs& a, cudaStream_t s) {
  using G = PsfGeom<NX>;
  // up to four arm slots where they fit (the derivative bank needs four; the
  // API admits it only for X <= 768), else three
  constexpr size_t kMax = 227 * 1024;
  constexpr size_t s4 = ((size_t)4 * G::SLOT + NX + 2 * G::B) * sizeof(float2);
  constexpr size_t s3 = ((size_t)3 * G::SLOT + NX + 2 * G::B) * sizeof(float2);
  constexpr size_t cap = s4 <= kMax ? s4 : s3;
  const size_t smem = ((size_t)a.n_arms * G::SLOT + NX + 2 * G::B) * sizeof(float2);
  if (smem > cap) return cudaErrorInvalidValue;
  const cudaError_t attr = allow_smem(k_psf_rows<NX>, cap);
  if (attr != cudaSuccess) return attr;
  const long long rows = a.row_end - a.row_begin;
  WO_LAUNCH("tf_psf_rows", s, (k_psf_rows<NX><<<(unsigned)((rows + G::B - 1) / G::B), G::NT, smem, s>>>(a)));
  return cudaGetLastError();
}

cudaError_t tf_psf_rows(const TfArgs& a, cudaStream_t s) {
  if (psf_rows_reg_supported(a.X, a.n_arms)) return tf_psf_rows_reg(a, s);
  switch (a.X) {
#define WO_CASE(n) \
  case n:          \
    return launch_psf<n>(a, s);
    WO_CASE(2) WO_CASE(4) WO_CASE(6) WO_CASE(8) WO_CASE(12) WO_CASE(16) WO_CASE(24) WO_CASE(32)
    WO_CASE(48) WO_CASE(64) WO_CASE(96) WO_CASE(128) WO_CASE(192) WO_CASE(256) WO_CASE(384)
    WO_CASE(512) WO_CASE(768) WO_CASE(1024) WO_CASE(1536) WO_CASE(2048)
#undef WO_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <int N, int NK>
static cudaError_t launch_zpass(const TfArgs& a, cudaStream_t s) {
  using G = ZGeom<N, NK>;
  const size_t smem = G::SMEM + (size_t)G::NT * 2 * sizeof(float);
  const cudaError_t attr = allow_smem(k_tf_zpass<N, NK>, smem);
  if (attr != cudaSuccess) return attr;
  dim3 grid((unsigned)((a.x_cols + G::B - 1) / G::B), (unsigned)a.Y, (unsigned)a.n_tiles);
  WO_LAUNCH("tf_zpass", s, (k_tf_zpass<N, NK><<<grid, G::NT, smem, s>>>(a)));
  return cudaGetLastError();
}

#define WO_ZP_CASE_1(n) case n: return launch_zpass<n, 1>(a, s);
#define WO_ZP_CASE_2(n) case n: return launch_zpass<n, 2>(a, s);
#define WO_ZP_CASE_3(n) case n: return launch_zpass<n, 3>(a, s);

cudaError_t tf_zpass(const TfArgs& a, cudaStream_t s) {
  if (tf_zpass_reg_supported(a)) return tf_zpass_reg(a, s);
  if (a.n_kinds == 1) {
    switch (a.Z) { WO_FOR_EACH_SIZE(WO_ZP_CASE_1) default: return cudaErrorInvalidValue; }
  }
  if (a.n_kinds == 2) {
    switch (a.Z) { WO_FOR_EACH_SIZE(WO_ZP_CASE_2) default: return cudaErrorInvalidValue; }
  }
  switch (a.Z) { WO_FOR_EACH_SIZE(WO_ZP_CASE_3) default: return cudaErrorInvalidValue; }
}

}  // namespace wo

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
#include "wo_zops.cuh"

namespace wo {

__device__ __forceinline__ int fft_index(int i, int n) { return (i < (n + 1) / 2) ? i : i - n; }

__global__ void __launch_bounds__(256)
    k_pupil_record(const wo_optics* __restrict__ optics, float4* __restrict__ rec, int* __restrict__ counts,
                   int Y, int X) {
  const int t = blockIdx.y;
  const int idx = blockIdx.x * 256 + threadIdx.x;
  int n_sp = 0, n_p = 0;
  if (idx < Y * X) {
    const wo_optics o = optics[t];
    const int y = idx / X, x = idx - (idx / X) * X;
    const double nu_y = __ddiv_rn((double)fft_index(y, Y), __dmul_rn((double)Y, o.pixel_um));
    const double nu_x = __ddiv_rn((double)fft_index(x, X), __dmul_rn((double)X, o.pixel_um));
    const double lam = o.lambda_um;
    // detection pupil: |nu| <= NA_det / lambda
    const double rp = __ddiv_rn(o.na_det, lam);
    const double r2 = __dadd_rn(__dmul_rn(nu_x, nu_x), __dmul_rn(nu_y, nu_y));
    const bool P = r2 <= __dmul_rn(rp, rp);
    // source pupil: |nu - t/lambda| <= NA_ill / lambda
    const double cy = __ddiv_rn(o.tilt_y, lam), cx = __ddiv_rn(o.tilt_x, lam);
    const double dy = __dsub_rn(nu_y, cy), dx = __dsub_rn(nu_x, cx);
    const double rs = __ddiv_rn(o.na_ill, lam);
    const bool S = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= __dmul_rn(rs, rs);
    const double km = __ddiv_rn(o.n_medium, lam);
    const double e2 = __dsub_rn(__dmul_rn(km, km), r2);
    const double eta = __dsqrt_rn(e2 > 0.0 ? e2 : 0.0);
    const float eh = __double2float_rn(eta);
    const float el = __double2float_rn(__dsub_rn(eta, (double)eh));
    const float binv = (P && eta > 0.0) ? __double2float_rn(__drcp_rn(eta)) : 0.f;
    rec[(long long)t * Y * X + idx] = make_float4(eh, el, binv, (S && P) ? 1.f : 0.f);
    n_sp = (S && P) ? 1 : 0;
    n_p = P ? 1 : 0;
    // band limit along x: the largest |k_x| inside P on the k_y = 0 row.  P is
    // contained in nu_x^2 <= (NA_det/lambda)^2, so every column beyond it is
    // zero in every arm.
    if (y == 0 && P) atomicMax(&counts[4 * t + 2], abs(fft_index(x, X)));
  }
  for (int off = 16; off > 0; off >>= 1) {
    n_sp += __shfl_down_sync(0xffffffffu, n_sp, off);
    n_p += __shfl_down_sync(0xffffffffu, n_p, off);
  }
  __shared__ int part[2][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    part[0][warp] = n_sp;
    part[1][warp] = n_p;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int i = 0; i < 8; ++i) {
      a += part[0][i];
      b += part[1][i];
    }
    if (a) atomicAdd(&counts[4 * t], a);
    if (b) atomicAdd(&counts[4 * t + 1], b);
  }
}

// fractional part of (eh + el) * (zh + zl), accurate to a few 1e-8
__device__ __forceinline__ float phase_frac(float eh, float el, float zh, float zl) {
  const float p = eh * zh;
  float err = fmaf(eh, zh, -p);
  err = fmaf(eh, zl, err);
  err = fmaf(el, zh, err);
  return (p - rintf(p)) + err;
}

template <int N>  // N = Y
__global__ void __launch_bounds__(ColGeom<N>::NT, (1024 / ColGeom<N>::NT) > 1 ? (1024 / ColGeom<N>::NT) : 1) k_arms(TfArgs a) {
  using G = ColGeom<N>;
  constexpr int B = G::B, NT = G::NT;
  constexpr int PER = (N * B + NT - 1) / NT;
  extern __shared__ float2 sm[];
  float2* buf = sm;
  float2* tw = sm + N * B;
  const int X = a.X, Z = a.Z;
  const int t = blockIdx.z, j = blockIdx.y, x0 = blockIdx.x * B;
  const int w = min(B, X - x0);
  // skip strips whose columns all lie outside the detection band: every arm
  // is exactly zero there, and the row pass never reads those columns
  const int kxmax = a.counts[4 * t + 2];
  bool active = false;
  for (int b = 0; b < w; ++b) active |= abs(fft_index(x0 + b, X)) <= kxmax;
  if (!active) return;  // uniform across the CTA
  make_twiddles<N>(tw);
  const wo_optics o = a.optics[t];
  const double zj = __dadd_rn(__dmul_rn((double)fft_index(j, Z), o.z_step_um), o.defocus_um);
  const float zh = __double2float_rn(zj);
  const float zl = __double2float_rn(__dsub_rn(zj, (double)zh));
  const float4* rec = a.rec + (long long)t * N * X + x0;
  float4 r[PER];
  float s_[PER], c_[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * NT;
    const int n = e / B, b = e % B;
    r[i] = (e < N * B && b < w) ? __ldg(rec + (long long)n * X + b) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) sincospif(2.0f * phase_frac(r[i].x, r[i].y, zh, zl), &s_[i], &c_[i]);
  int arm = 0;
  for (int which = 0; which < 3; ++which) {
    if (which < 2 && a.lf_props == 0) continue;
    if (which == 2 && !a.want_fl) continue;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = threadIdx.x + i * NT;
      if (e >= N * B) continue;
      const bool on = (which == 0) ? (r[i].w != 0.f) : (r[i].z != 0.f);
      float2 v = make_float2(0.f, 0.f);
      if (on) v = (which == 1) ? make_float2(-r[i].z * s_[i], r[i].z * c_[i]) : make_float2(c_[i], s_[i]);
      buf[e] = v;
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
  static constexpr int B = (NX <= 128) ? 16 : (NX <= 1024) ? 8 : 4;
  static constexpr int LD = NX + 1;
  static constexpr int NT = threads_for(NX * B);
  static constexpr int MINB = (1536 / NT) > 1 ? (1536 / NT) : 1;
  static constexpr size_t SMEM = (2 * (size_t)B * LD + NX + 2 * B) * sizeof(float2);
};

// Real row h (given through `val`) -> half spectrum written to dst rows.
template <int NX, int B, int NT, class F>
__device__ __forceinline__ void psf_r2c_rows(float2* src, float2* pack, const float2* tw, F val,
                                             float2* __restrict__ tf, long long row0, long long nrows,
                                             const TfArgs& a, int slot) {
  constexpr int H = NX / 2, LD = NX + 1;
  const int Z = a.Z, Y = a.Y, Xh = H + 1;
  for (int e = threadIdx.x; e < B * H; e += NT) {
    const int b = e / H, m = e - (e / H) * H;
    const long long row = row0 + b;
    float2 z = make_float2(0.f, 0.f);
    if (row < nrows) z = make_float2(val(src[b * LD + 2 * m], b), val(src[b * LD + 2 * m + 1], b));
    pack[b * LD + m] = z;
  }
  __syncthreads();
  fft_smem<H, B, NT, false, 2>(pack, 1, LD, tw);
  for (int e = threadIdx.x; e < B * (H + 1); e += NT) {
    const int b = e / (H + 1), k = e - (e / (H + 1)) * (H + 1);
    const long long row = row0 + b;
    if (row >= nrows) continue;
    const float2 zk = pack[b * LD + (k == H ? 0 : k)];
    const float2 zc = cconj(pack[b * LD + (k == 0 ? 0 : H - k)]);
    const float2 s = cadd(zk, zc);
    const float2 u = cmul(tw[k], csub(zk, zc));
    const long long plane = row / Y;  // t*Z + j
    const int y = (int)(row - plane * Y);
    const long long t = plane / Z, j = plane - (plane / Z) * Z;
    tf[(((t * a.n_kinds + slot) * Z + j) * Y + y) * Xh + k] =
        make_float2(0.5f * (s.x + u.y), 0.5f * (s.y - u.x));
  }
  __syncthreads();
}

__device__ __forceinline__ float lf_scale(const TfArgs& a, int t) {
  // 2K = 2 c / (N_perp sum S P^2), c = 2 pi n dz / lambda^2
  const wo_optics o = a.optics[t];
  const int n_sp = a.counts[4 * t];
  if (n_sp == 0) return 0.f;
  const double c = 2.0 * 3.14159265358979323846 * o.n_medium * o.z_step_um / (o.lambda_um * o.lambda_um);
  return (float)(2.0 * c / ((double)a.Y * (double)a.X * (double)n_sp));
}

__device__ __forceinline__ float fl_scale(const TfArgs& a, int t) {
  const int n_p = a.counts[4 * t + 1];
  if (n_p == 0) return 0.f;
  return (float)(1.0 / ((double)a.Y * (double)a.X * (double)a.Z * (double)n_p));
}

template <int NX>
__global__ void __launch_bounds__(PsfGeom<NX>::NT, PsfGeom<NX>::MINB) k_psf_rows(TfArgs a) {
  using G = PsfGeom<NX>;
  constexpr int B = G::B, LD = G::LD, NT = G::NT;
  extern __shared__ float2 sm[];
  float2* bufA = sm;
  float2* bufB = sm + B * LD;
  float2* tw = sm + 2 * B * LD;  // exp(-2 pi i m / NX)
  float* sc = reinterpret_cast<float*>(tw + NX);  // per row: [B] label-free 2K, [B] fluorescence
  int* kxm = reinterpret_cast<int*>(sc + 2 * B);   // per row: x band limit of its tile
  const long long nrows = (long long)a.n_tiles * a.Z * a.Y;
  const long long row0 = (long long)blockIdx.x * B;
  if (threadIdx.x < B) {
    const long long row = row0 + threadIdx.x;
    const int t = (int)((row < nrows ? row : nrows - 1) / ((long long)a.Z * a.Y));
    sc[threadIdx.x] = lf_scale(a, t);
    sc[B + threadIdx.x] = fl_scale(a, t);
    kxm[threadIdx.x] = row < nrows ? a.counts[4 * t + 2] : -1;
  }
  __syncthreads();
  const long long plane_elems = (long long)a.Y * NX;  // elements of one arm plane
  // columns outside the detection band are zero (and were never written)
  auto load_arm = [&](float2* dst, int arm) {
    for (int e = threadIdx.x; e < B * NX; e += NT) {
      const int b = e / NX, n = e - (e / NX) * NX;
      const long long row = row0 + b;
      const bool ok = row < nrows && abs(fft_index(n, NX)) <= kxm[b];
      const float2* src = a.arms;
      if (ok) {
        const long long t = row / ((long long)a.Z * a.Y);
        const long long rem = row - t * a.Z * a.Y;  // j*Y + y
        src = a.arms + ((t * a.n_arms + arm) * a.Z) * plane_elems + rem * NX + n;
      }
      cp_async8(dst + b * LD + n, src, ok);
    }
  };
  make_twiddles<NX>(tw);
  int arm = 0;
  if (a.lf_props > 0) {
    load_arm(bufA, 0);
    load_arm(bufB, 1);
    cp_async_wait_all();
    __syncthreads();
    fft_smem<NX, B, NT, true, 1>(bufA, 1, LD, tw);
    fft_smem<NX, B, NT, true, 1>(bufB, 1, LD, tw);
    for (int e = threadIdx.x; e < B * NX; e += NT) {
      const int b = e / NX, n = e - (e / NX) * NX;
      bufA[b * LD + n] = cmulc(bufA[b * LD + n], bufB[b * LD + n]);  // g = conj(a) b
    }
    __syncthreads();
    int slot = 0;
    if (a.want_phase) {
      psf_r2c_rows<NX, B, NT>(bufA, bufB, tw, [&](float2 g, int b) { return sc[b] * g.x; },
                              a.tf, row0, nrows, a, slot);
      ++slot;
    }
    if (a.want_abs) {
      psf_r2c_rows<NX, B, NT>(bufA, bufB, tw, [&](float2 g, int b) { return -sc[b] * g.y; },
                              a.tf, row0, nrows, a, slot);
    }
    arm = 2;
  }
  if (a.want_fl) {
    load_arm(bufA, arm);
    cp_async_wait_all();
    __syncthreads();
    fft_smem<NX, B, NT, true, 1>(bufA, 1, LD, tw);
    psf_r2c_rows<NX, B, NT>(bufA, bufB, tw, [&](float2 p, int b) { return sc[B + b] * cabs2(p); },
                            a.tf, row0, nrows, a, a.lf_props);
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
  for (int e = threadIdx.x; e < NK * N * B; e += NT) {
    const int v = e / (N * B), r = e - v * (N * B);
    const int n = r / B, bb = r % B;
    if (bb < w) base[v * vol + n * zs + bb] = buf[(n * NK + v) * B + bb];
  }
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
  // block maxima (values are >= 0, so integer order equals float order)
  for (int off = 16; off > 0; off >>= 1) {
    m3_lf = fmaxf(m3_lf, __shfl_down_sync(0xffffffffu, m3_lf, off));
    m3_fl = fmaxf(m3_fl, __shfl_down_sync(0xffffffffu, m3_fl, off));
    m2_lf = fmaxf(m2_lf, __shfl_down_sync(0xffffffffu, m2_lf, off));
    m2_fl = fmaxf(m2_fl, __shfl_down_sync(0xffffffffu, m2_fl, off));
  }
  if ((threadIdx.x & 31) == 0) {
    int* st = reinterpret_cast<int*>(a.stats + (long long)t * 8);
    if (m3_lf > 0.f) atomicMax(st + 0, __float_as_int(m3_lf));
    if (m2_lf > 0.f) atomicMax(st + 1, __float_as_int(m2_lf));
    if (m3_fl > 0.f) atomicMax(st + 2, __float_as_int(m3_fl));
    if (m2_fl > 0.f) atomicMax(st + 3, __float_as_int(m2_fl));
  }
}

cudaError_t tf_pupil_record(const TfArgs& a, cudaStream_t s) {
  dim3 grid((unsigned)((a.Y * a.X + 255) / 256), (unsigned)a.n_tiles);
  WO_LAUNCH("tf_pupil_record", s, (k_pupil_record<<<grid, 256, 0, s>>>(a.optics, a.rec, a.counts, a.Y, a.X)));
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_arms(const TfArgs& a, cudaStream_t s) {
  using G = ColGeom<N>;
  static cudaError_t attr = allow_smem(k_arms<N>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  dim3 grid((unsigned)((a.X + G::B - 1) / G::B), (unsigned)a.Z, (unsigned)a.n_tiles);
  WO_LAUNCH("tf_arms", s, (k_arms<N><<<grid, G::NT, G::SMEM, s>>>(a)));
  return cudaGetLastError();
}

cudaError_t tf_arms(const TfArgs& a, cudaStream_t s) {
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
  static cudaError_t attr = allow_smem(k_psf_rows<NX>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  const long long rows = (long long)a.n_tiles * a.Z * a.Y;
  WO_LAUNCH("tf_psf_rows", s, (k_psf_rows<NX><<<(unsigned)((rows + G::B - 1) / G::B), G::NT, G::SMEM, s>>>(a)));
  return cudaGetLastError();
}

cudaError_t tf_psf_rows(const TfArgs& a, cudaStream_t s) {
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
  static cudaError_t attr = allow_smem(k_tf_zpass<N, NK>, smem);
  if (attr != cudaSuccess) return attr;
  const int Xh = a.X / 2 + 1;
  dim3 grid((unsigned)((Xh + G::B - 1) / G::B), (unsigned)a.Y, (unsigned)a.n_tiles);
  WO_LAUNCH("tf_zpass", s, (k_tf_zpass<N, NK><<<grid, G::NT, smem, s>>>(a)));
  return cudaGetLastError();
}

#define WO_ZP_CASE_1(n) case n: return launch_zpass<n, 1>(a, s);
#define WO_ZP_CASE_2(n) case n: return launch_zpass<n, 2>(a, s);
#define WO_ZP_CASE_3(n) case n: return launch_zpass<n, 3>(a, s);

cudaError_t tf_zpass(const TfArgs& a, cudaStream_t s) {
  if (a.n_kinds == 1) {
    switch (a.Z) { WO_FOR_EACH_SIZE(WO_ZP_CASE_1) default: return cudaErrorInvalidValue; }
  }
  if (a.n_kinds == 2) {
    switch (a.Z) { WO_FOR_EACH_SIZE(WO_ZP_CASE_2) default: return cudaErrorInvalidValue; }
  }
  switch (a.Z) { WO_FOR_EACH_SIZE(WO_ZP_CASE_3) default: return cudaErrorInvalidValue; }
}

}  // namespace wo

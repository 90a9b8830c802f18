// wo_fuse.cu - multi-channel fusion: one property from C data channels, each
// seen through its own transfer function (9-aperture fusion, Results; C x 1
// multi-channel Tikhonov, Eq. recon with a C-element column H):
//   F(nu) = sum_c conj(H_c) D~_c / (sum_c |H_c|^2 + eta)
// per 3D frequency, or per transverse frequency with the sums also over the
// axial bins (the 2D phase-from-defocus model; Parseval over z).
//
// The z pass streams the channels: for each channel a CTA loads the z columns
// of its B x columns, transforms them along z in shared memory and adds
// conj(H_c) D_c and |H_c|^2 into two accumulators in shared memory; after the
// last channel it forms F, transforms it back (3D) or reduces it over k (2D),
// and stores one output volume.
#include "wo_fft.cuh"
#include "wo_internal.h"
#include "wo_zops.cuh"

namespace wo {

namespace {

template <int N>
struct FuseGeom {
  using G = ZGeom<N, 3>;  // data tile, numerator, denominator
  static constexpr int B = G::B, NT = G::NT, MINB = G::MINB;
  static constexpr size_t SMEM = G::SMEM + (size_t)NT * 3 * sizeof(float);
};

// Per tile: max over 3D frequencies of sum_c |H_c|^2 and max over transverse
// frequencies of sum_k sum_c |H_c|^2 (the relative regulariser's scales in
// 3D and 2D).  One thread per (y, x) column.
__global__ void __launch_bounds__(256) k_fuse_stats(const float2* __restrict__ tf, int C, int Z, int Y, int Xh,
                                                    float* __restrict__ stats) {
  const int t = blockIdx.y;
  const long long plane = (long long)Y * Xh;
  const long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float m3 = 0.f, s2 = 0.f;
  if (col < plane) {
    const float2* h = tf + (long long)t * C * Z * plane + col;
    for (int k = 0; k < Z; ++k) {
      float s = 0.f;
      for (int c = 0; c < C; ++c) s += cabs2(__ldg(h + ((long long)c * Z + k) * plane));
      m3 = fmaxf(m3, s);
      s2 += s;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    m3 = fmaxf(m3, __shfl_down_sync(0xffffffffu, m3, off));
    s2 = fmaxf(s2, __shfl_down_sync(0xffffffffu, s2, off));
  }
  // values are >= 0: integer order equals float order
  if ((threadIdx.x & 31) == 0) {
    if (m3 > 0.f) atomicMax(reinterpret_cast<int*>(stats) + 2 * t, __float_as_int(m3));
    if (s2 > 0.f) atomicMax(reinterpret_cast<int*>(stats) + 2 * t + 1, __float_as_int(s2));
  }
}

template <int N>
__global__ void __launch_bounds__(FuseGeom<N>::NT, FuseGeom<N>::MINB)
    k_z_fuse(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ tf, FuseOp op,
             int Y, int Xh) {
  using G = FuseGeom<N>;
  constexpr int B = G::B, NT = G::NT;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* dbuf = sm + N;
  float2* num = dbuf + N * B;
  float* den = reinterpret_cast<float*>(num + N * B);
  float* red = den + 2 * N * B;  // [NT][3] (2D reduction)
  const int t = blockIdx.z, y = blockIdx.y, x0 = blockIdx.x * B;
  const int w = min(B, Xh - x0);
  const long long zs = (long long)Y * Xh;
  const long long vol = (long long)N * zs;
  const long long col = (long long)y * Xh + x0;
  const int C = op.C;
  make_twiddles<N>(tw);
  for (int e = threadIdx.x; e < N * B; e += NT) {
    num[e] = make_float2(0.f, 0.f);
    den[e] = 0.f;
  }
  for (int c = 0; c < C; ++c) {
    load_zcols<N, 1, B, NT>(dbuf, in + ((long long)t * C + c) * vol + col, 1, vol, zs, w);
    cp_async_wait_all();
    __syncthreads();
    fft_smem<N, B, NT, false, 1>(dbuf, B, 1, tw);
    const float2* h = tf + ((long long)t * C + c) * vol + col;
    for (int e = threadIdx.x; e < N * B; e += NT) {
      const int k = e / B, b = e % B;
      if (b >= w) continue;
      float2 d = dbuf[e];
      if (k == 0 && y == 0 && x0 + b == 0) d = op.zero_dc ? make_float2(0.f, 0.f) : make_float2(d.x - op.bg_dc[c], d.y);
      const float2 hv = __ldg(h + (long long)k * zs + b);
      num[e] = cadd(num[e], cmulc(hv, d));
      den[e] += cabs2(hv);
    }
    __syncthreads();  // dbuf is reloaded for the next channel
  }
  const float* st = op.stats + 2LL * t;
  if (op.mode == WO_MODE_3D) {
    const float lam = op.eta_relative ? op.eta * st[0] : op.eta;
    for (int e = threadIdx.x; e < N * B; e += NT) {
      const float q = den[e] + lam;
      dbuf[e] = q > 0.f ? cscale(num[e], 1.0f / q) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_smem<N, B, NT, true, 1>(dbuf, B, 1, tw);
    store_zcols<N, 1, B, NT>(dbuf, out + (long long)t * vol + col, 1, vol, zs, w);
    return;
  }
  // 2D: sum over k of both accumulators, per column b (fixed per thread)
  const int b = threadIdx.x % B;
  float sr = 0.f, si = 0.f, sd = 0.f;
  for (int e = threadIdx.x; e < N * B; e += NT) {
    sr += num[e].x;
    si += num[e].y;
    sd += den[e];
  }
  red[3 * threadIdx.x] = sr;
  red[3 * threadIdx.x + 1] = si;
  red[3 * threadIdx.x + 2] = sd;
  __syncthreads();
  if (threadIdx.x < B && b < w) {
    float2 a = make_float2(0.f, 0.f);
    float dd = 0.f;
    for (int q = threadIdx.x; q < NT; q += B) {
      a = cadd(a, make_float2(red[3 * q], red[3 * q + 1]));
      dd += red[3 * q + 2];
    }
    // per-plane sums are 1/Z of the sums over k, so eta enters as Z eta
    const float lam = op.eta_relative ? op.eta * st[1] : op.eta * (float)N;
    const float q = dd + lam;
    out[(long long)t * zs + col + b] = q > 0.f ? cscale(a, 1.0f / q) : make_float2(0.f, 0.f);
  }
}

template <int N>
cudaError_t launch_z_fuse(const float2* in, float2* out, const float2* tf, const FuseOp& op, int n_tiles, int Y,
                          int Xh, cudaStream_t s) {
  using G = FuseGeom<N>;
  const cudaError_t attr = allow_smem(k_z_fuse<N>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  dim3 grid((unsigned)((Xh + G::B - 1) / G::B), (unsigned)Y, (unsigned)n_tiles);
  WO_LAUNCH("z_fuse", s, (k_z_fuse<N><<<grid, G::NT, G::SMEM, s>>>(in, out, tf, op, Y, Xh)));
  return cudaGetLastError();
}

}  // namespace

cudaError_t fuse_stats(const float2* tf, int n_tiles, int C, int Z, int Y, int Xh, float* stats, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(stats, 0, (size_t)n_tiles * 2 * sizeof(float), s);
  if (e != cudaSuccess) return e;
  const long long plane = (long long)Y * Xh;
  dim3 grid((unsigned)((plane + 255) / 256), (unsigned)n_tiles);
  WO_LAUNCH("fuse_stats", s, (k_fuse_stats<<<grid, 256, 0, s>>>(tf, C, Z, Y, Xh, stats)));
  return cudaGetLastError();
}

cudaError_t z_fuse(int Z, const float2* in, float2* out, const float2* tf, const FuseOp& op, int n_tiles, int Y,
                   int Xh, cudaStream_t s) {
  switch (Z) {
#define WO_CASE(n) \
  case n:          \
    return launch_z_fuse<n>(in, out, tf, op, n_tiles, Y, Xh, s);
    WO_FOR_EACH_SIZE(WO_CASE)
#undef WO_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace wo

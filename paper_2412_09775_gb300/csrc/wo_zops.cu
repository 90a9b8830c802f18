// wo_zops.cu - fused z pass: forward z transform, per-frequency operator,
// inverse z transform, in one kernel.
//
// A CTA owns B adjacent x columns of one (tile, y) row of the half-spectrum
// volumes.  It loads the z columns of every input volume, transforms them
// along z in shared memory, applies the per-frequency operator while reading
// the transfer functions once (coalesced along x), transforms the outputs
// back and stores them.  The per-frequency operators are
//   forward      D_c = sum_p H_cp F_p                        (Eq. fwd, Fourier form)
//   adjoint      F_p = sum_c conj(H_cp) D_c
//   reconstruct  F = H^H (H H^H + eta I)^-1 D~, which for the one-channel
//                modes here is F_p = conj(H_p) D~ / (sum_p |H_p|^2 + eta)
//                (Eq. recon; the push-through form of the normal equations)
// The 2D variant sums H^H H and H^H D over k_z (Parseval over the planes) and
// solves a P x P (P <= 2) system per transverse frequency.
#include "wo_fft.cuh"
#include "wo_internal.h"

namespace wo {

template <int N>
struct ZGeom {
  static constexpr int B = (N <= 256) ? 16 : (N <= 512) ? 8 : (N <= 1024) ? 4 : 2;
  static constexpr int NT0 = (N * B) / 16;
  static constexpr int NT = NT0 < 64 ? 64 : (NT0 > 512 ? 512 : NT0);
  static constexpr int MINB = (768 / NT) > 1 ? (768 / NT) : 1;
};

__device__ __forceinline__ float2 ld_tf(const float2* p) { return __ldg(p); }

template <int N>
__global__ void __launch_bounds__(ZGeom<N>::NT, ZGeom<N>::MINB)
    k_z_fused(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ tf,
              ZOp op, int Y, int Xh) {
  using G = ZGeom<N>;
  constexpr int B = G::B, NT = G::NT;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* bin = sm + N;
  float2* bout = bin + op.n_in * N * B;
  make_twiddles<N>(tw);
  const int t = blockIdx.z, y = blockIdx.y, x0 = blockIdx.x * B;
  const int w = min(B, Xh - x0);
  const long long zs = (long long)Y * Xh;
  const long long vol = (long long)N * zs;
  const long long col = (long long)y * Xh + x0;
  for (int v = 0; v < op.n_in; ++v) {
    const float2* src = in + ((long long)t * op.n_in + v) * vol + col;
    for (int e = threadIdx.x; e < N * B; e += NT) {
      const int n = e / B, b = e % B;
      bin[v * N * B + e] = (b < w) ? src[n * zs + b] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  for (int v = 0; v < op.n_in; ++v) fft_smem<N, B, NT, false, 1>(bin + v * N * B, B, 1, tw);

  const float* st = op.stats + (long long)t * 8;
  const float lam_lf = op.eta_absolute ? op.eta_lf : op.eta_lf * st[0];
  const float lam_fl = op.eta_absolute ? op.eta_fl : op.eta_fl * st[2];
  const int L = op.lf_props;
  for (int e = threadIdx.x; e < N * B; e += NT) {
    const int k = e / B, b = e % B;
    if (b >= w) {
      for (int v = 0; v < op.n_out; ++v) bout[v * N * B + e] = make_float2(0.f, 0.f);
      continue;
    }
    const float2* h = tf + ((long long)t * op.n_tf * N + k) * zs + col + b;
    float2 H[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) H[s] = (s < op.n_tf) ? ld_tf(h + s * vol) : make_float2(0.f, 0.f);
    if (op.op == 0) {  // forward: props in, channels out
      if (L > 0) {
        float2 d = cmul(H[0], bin[e]);
        if (L > 1) d = cadd(d, cmul(H[1], bin[N * B + e]));
        bout[op.lf_chan * N * B + e] = d;
      }
      if (op.has_fl) bout[op.fl_chan * N * B + e] = cmul(H[L], bin[L * N * B + e]);
    } else if (op.op == 1) {  // adjoint: channels in, props out
      if (L > 0) {
        const float2 d = bin[op.lf_chan * N * B + e];
        bout[e] = cmulc(H[0], d);
        if (L > 1) bout[N * B + e] = cmulc(H[1], d);
      }
      if (op.has_fl) bout[L * N * B + e] = cmulc(H[L], bin[op.fl_chan * N * B + e]);
    } else {  // reconstruct
      const bool dc = op.zero_dc && k == 0 && y == 0 && (x0 + b) == 0;
      if (L > 0) {
        const float2 d = dc ? make_float2(0.f, 0.f) : bin[op.lf_chan * N * B + e];
        float den = lam_lf + cabs2(H[0]);
        if (L > 1) den += cabs2(H[1]);
        const float inv = 1.0f / den;
        bout[e] = cscale(cmulc(H[0], d), inv);
        if (L > 1) bout[N * B + e] = cscale(cmulc(H[1], d), inv);
      }
      if (op.has_fl) {
        const float2 d = dc ? make_float2(0.f, 0.f) : bin[op.fl_chan * N * B + e];
        bout[L * N * B + e] = cscale(cmulc(H[L], d), 1.0f / (lam_fl + cabs2(H[L])));
      }
    }
  }
  __syncthreads();
  for (int v = 0; v < op.n_out; ++v) fft_smem<N, B, NT, true, 1>(bout + v * N * B, B, 1, tw);
  for (int v = 0; v < op.n_out; ++v) {
    float2* dst = out + ((long long)t * op.n_out + v) * vol + col;
    for (int e = threadIdx.x; e < N * B; e += NT) {
      const int n = e / B, b = e % B;
      if (b < w) dst[n * zs + b] = bout[v * N * B + e];
    }
  }
}

// 2D: out[t][p][y][x] = (sum_k H_k^H H_k + lam I)^-1 sum_k H_k^H D_k per mode.
template <int N>
__global__ void __launch_bounds__(ZGeom<N>::NT, ZGeom<N>::MINB)
    k_z_solve2d(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ tf,
                ZOp op, int Y, int Xh) {
  using G = ZGeom<N>;
  constexpr int B = G::B, NT = G::NT, KK = NT / B;
  constexpr int NACC = 11;  // m00 m11 m01(2) r0(2) r1(2) mf rf(2)
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* bin = sm + N;
  float* red = reinterpret_cast<float*>(bin + op.n_in * N * B);  // [NT][NACC]
  make_twiddles<N>(tw);
  const int t = blockIdx.z, y = blockIdx.y, x0 = blockIdx.x * B;
  const int w = min(B, Xh - x0);
  const long long zs = (long long)Y * Xh;
  const long long vol = (long long)N * zs;
  const long long col = (long long)y * Xh + x0;
  for (int v = 0; v < op.n_in; ++v) {
    const float2* src = in + ((long long)t * op.n_in + v) * vol + col;
    for (int e = threadIdx.x; e < N * B; e += NT) {
      const int n = e / B, b = e % B;
      bin[v * N * B + e] = (b < w) ? src[n * zs + b] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  for (int v = 0; v < op.n_in; ++v) fft_smem<N, B, NT, false, 1>(bin + v * N * B, B, 1, tw);

  const int L = op.lf_props;
  const int b = threadIdx.x % B, kk = threadIdx.x / B;
  float acc[NACC];
#pragma unroll
  for (int i = 0; i < NACC; ++i) acc[i] = 0.f;
  if (b < w) {
    for (int k = kk; k < N; k += KK) {
      const int e = k * B + b;
      const bool dc = op.zero_dc && k == 0 && y == 0 && (x0 + b) == 0;
      const float2* h = tf + ((long long)t * op.n_tf * N + k) * zs + col + b;
      if (L > 0) {
        const float2 d = dc ? make_float2(0.f, 0.f) : bin[op.lf_chan * N * B + e];
        const float2 h0 = ld_tf(h);
        acc[0] += cabs2(h0);
        const float2 r0 = cmulc(h0, d);
        acc[4] += r0.x; acc[5] += r0.y;
        if (L > 1) {
          const float2 h1 = ld_tf(h + vol);
          acc[1] += cabs2(h1);
          const float2 m01 = cmulc(h0, h1);
          acc[2] += m01.x; acc[3] += m01.y;
          const float2 r1 = cmulc(h1, d);
          acc[6] += r1.x; acc[7] += r1.y;
        }
      }
      if (op.has_fl) {
        const float2 d = dc ? make_float2(0.f, 0.f) : bin[op.fl_chan * N * B + e];
        const float2 hf = ld_tf(h + L * vol);
        acc[8] += cabs2(hf);
        const float2 rf = cmulc(hf, d);
        acc[9] += rf.x; acc[10] += rf.y;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < NACC; ++i) red[threadIdx.x * NACC + i] = acc[i];
  __syncthreads();
  if (kk == 0 && b < w) {
    for (int q = 1; q < KK; ++q) {
#pragma unroll
      for (int i = 0; i < NACC; ++i) acc[i] += red[(q * B + b) * NACC + i];
    }
    const float* st = op.stats + (long long)t * 8;
    float2* o = out + (long long)t * (L + op.has_fl) * Y * Xh + (long long)y * Xh + x0 + b;
    const long long plane = (long long)Y * Xh;
    if (L > 0) {
      const float lam = op.eta_absolute ? op.eta_lf * (float)N : op.eta_lf * st[1];
      const float2 r0 = make_float2(acc[4], acc[5]);
      if (L == 1) {
        o[0] = cscale(r0, 1.0f / (acc[0] + lam));
      } else {
        const float a = acc[0] + lam, d = acc[1] + lam;
        const float2 m = make_float2(acc[2], acc[3]);
        const float2 r1 = make_float2(acc[6], acc[7]);
        const float inv = 1.0f / (a * d - cabs2(m));
        const float2 f0 = csub(cscale(r0, d), cmul(m, r1));
        const float2 f1 = csub(cscale(r1, a), cmulc(m, r0));
        o[0] = cscale(f0, inv);
        o[plane] = cscale(f1, inv);
      }
    }
    if (op.has_fl) {
      const float lam = op.eta_absolute ? op.eta_fl * (float)N : op.eta_fl * st[3];
      o[L * plane] = cscale(make_float2(acc[9], acc[10]), 1.0f / (acc[8] + lam));
    }
  }
}

template <int N>
static cudaError_t launch_z(bool two_d, const float2* in, float2* out, const float2* tf, ZOp op,
                            int n_tiles, int Y, int Xh, cudaStream_t s) {
  using G = ZGeom<N>;
  dim3 grid((unsigned)((Xh + G::B - 1) / G::B), (unsigned)Y, (unsigned)n_tiles);
  if (!two_d) {
    const size_t smem = ((size_t)N + (size_t)(op.n_in + op.n_out) * N * G::B) * sizeof(float2);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t a = cudaFuncSetAttribute(k_z_fused<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (a != cudaSuccess) return a;
    WO_LAUNCH("z_fused", s, (k_z_fused<N><<<grid, G::NT, smem, s>>>(in, out, tf, op, Y, Xh)));
  } else {
    const size_t smem = ((size_t)N + (size_t)op.n_in * N * G::B) * sizeof(float2) + (size_t)G::NT * 11 * sizeof(float);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t a = cudaFuncSetAttribute(k_z_solve2d<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (a != cudaSuccess) return a;
    WO_LAUNCH("z_solve2d", s, (k_z_solve2d<N><<<grid, G::NT, smem, s>>>(in, out, tf, op, Y, Xh)));
  }
  return cudaGetLastError();
}

static cudaError_t dispatch_z(bool two_d, int Z, const float2* in, float2* out, const float2* tf, ZOp op,
                              int n_tiles, int Y, int Xh, cudaStream_t s) {
  switch (Z) {
#define WO_CASE(n) \
  case n:          \
    return launch_z<n>(two_d, in, out, tf, op, n_tiles, Y, Xh, s);
    WO_FOR_EACH_SIZE(WO_CASE)
#undef WO_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t z_fused(int Z, const float2* in, float2* out, const float2* tf, ZOp op, int n_tiles, int Y,
                    int Xh, cudaStream_t s) {
  return dispatch_z(false, Z, in, out, tf, op, n_tiles, Y, Xh, s);
}

cudaError_t z_solve2d(int Z, const float2* in, float2* out, const float2* tf, ZOp op, int n_tiles, int Y,
                      int Xh, cudaStream_t s) {
  return dispatch_z(true, Z, in, out, tf, op, n_tiles, Y, Xh, s);
}

}  // namespace wo

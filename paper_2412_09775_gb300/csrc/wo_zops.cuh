// wo_zops.cuh - fused z pass: forward z transform, per-frequency operator,
// inverse z transform, in one kernel (shared by the translation units that
// instantiate it).
//
// A CTA owns B adjacent x columns of one (tile, y) row of the half-spectrum
// volumes.  The z columns of all NI input volumes are copied asynchronously
// into shared memory laid out [n][slot][b], so one batched transform covers
// every volume.  The per-frequency operator then replaces, in place, the NI
// input values at each (k, b) by the NO output values, reading the transfer
// functions once (coalesced along x); the NO outputs are transformed back in
// one batch and stored.  The operators are
//   forward      D_c = sum_p H_cp F_p                        (Eq. fwd, Fourier form)
//   adjoint      F_p = sum_c conj(H_cp) D_c
//   reconstruct  F = H^H (H H^H + eta I)^-1 D~, which for the one-channel
//                modes here is F_p = conj(H_p) D~ / (sum_p |H_p|^2 + eta)
//                (Eq. recon; the push-through form of the normal equations)
// The 2D variant sums H^H H and H^H D over k_z (Parseval over the planes) and
// solves a P x P (P <= 2) system per transverse frequency.
#pragma once
#include "wo_fft.cuh"
#include "wo_internal.h"

namespace wo {

// Columns per CTA of the z kernels: 16 while the tile stays within 32 KB,
// else the widest that fits 64 KB.  At 96 planes and three volumes 8 columns
// (more CTAs resident per SM) measured faster than 16 and 4.
__host__ __device__ constexpr int z_cols(int N, int NV) {
  return (NV * N * 16 * 8 <= 32 * 1024) ? 16
         : (NV * N * 8 * 8 <= 64 * 1024) ? 8
         : (NV * N * 4 * 8 <= 64 * 1024) ? 4
         : (NV * N * 2 * 8 <= 64 * 1024) ? 2
                                        : 1;
}

template <int N, int NV>
struct ZGeom {
  static constexpr int B = z_cols(N, NV);
  static constexpr int NT = threads_for(NV * N * B);
  static constexpr int MINB = (1536 / NT) > 1 ? (1536 / NT) : 1;
  static constexpr size_t SMEM = ((size_t)N + (size_t)NV * N * B) * sizeof(float2);
  // fused pass: plus up to three transfer functions of N x B prefetched (the
  // launch asks for the slots the bank has)
  static constexpr size_t SMEM_TF = SMEM + (size_t)3 * N * B * sizeof(float2);
  static constexpr size_t smem_tf(int n_tf) { return SMEM + (size_t)n_tf * N * B * sizeof(float2); }
};

__device__ __forceinline__ float2 sel3(int i, float2 a, float2 b, float2 c) { return i == 0 ? a : (i == 1 ? b : c); }

// Copy the z columns of `nv` volumes into slots [n][v][b] of the tile.  Each
// thread keeps one column b (NT is a multiple of B) and walks n with a
// pointer increment, so a copy costs a handful of instructions.
template <int N, int NV, int B, int NT>
__device__ __forceinline__ void load_zcols(float2* buf, const float2* __restrict__ src, int nv,
                                           long long vol, long long zs, int w) {
  constexpr int NSTEP = NT / B;
  const int b = threadIdx.x % B, n0 = threadIdx.x / B;
  const bool ok = b < w;
  for (int v = 0; v < nv; ++v) {
    const float2* g = src + v * vol + (long long)n0 * zs + b;
    float2* d = buf + (n0 * NV + v) * B + b;
#pragma unroll 4
    for (int n = n0; n < N; n += NSTEP) {
      cp_async8(d, ok ? g : src, ok);
      g += NSTEP * zs;
      d += NSTEP * NV * B;
    }
  }
}

// Store slots [n][v][b] of the tile to the z columns of `nv` volumes.
template <int N, int NV, int B, int NT>
__device__ __forceinline__ void store_zcols(const float2* buf, float2* __restrict__ dst, int nv, long long vol,
                                            long long zs, int w) {
  constexpr int NSTEP = NT / B;
  const int b = threadIdx.x % B, n0 = threadIdx.x / B;
  if (b >= w) return;
  for (int v = 0; v < nv; ++v) {
    float2* g = dst + v * vol + (long long)n0 * zs + b;
    const float2* d = buf + (n0 * NV + v) * B + b;
#pragma unroll 4
    for (int n = n0; n < N; n += NSTEP) {
      *g = *d;
      g += NSTEP * zs;
      d += NSTEP * NV * B;
    }
  }
}

// Zero the z columns of `nv` volumes (frequencies outside the TF support).
template <int N, int B, int NT>
__device__ __forceinline__ void zero_zcols(float2* __restrict__ dst, int nv, long long vol, long long zs, int w) {
  constexpr int NSTEP = NT / B;
  const int b = threadIdx.x % B, n0 = threadIdx.x / B;
  if (b >= w) return;
  for (int v = 0; v < nv; ++v) {
    float2* g = dst + v * vol + (long long)n0 * zs + b;
#pragma unroll 4
    for (int n = n0; n < N; n += NSTEP) {
      *g = make_float2(0.f, 0.f);
      g += NSTEP * zs;
    }
  }
}

// True when column k_x = x0 of row y lies outside the tile's TF support disk
// (k_y/Y)^2 + (k_x/X)^2 <= r^2 (r: statistics word 5, cycles per pixel);
// there the TFs hold only the rounding noise of the PSF-row transforms, and
// every operator's output is set to zero.  The nearest column of a strip
// k_x >= x0 is x0 (k_x >= 0 in the half spectrum), so the whole strip is
// outside when x0 is.
__device__ __forceinline__ bool outside_support(const float* stats, int y, int Y, int x0, int X) {
  const float r = stats[5];
  const float fy = (float)(y < (Y + 1) / 2 ? y : y - Y) / (float)Y, fx = (float)x0 / (float)X;
  return fy * fy + fx * fx > r * r;
}

template <int N, int NI, int NO>
__global__ void __launch_bounds__(ZGeom<N, (NI > NO ? NI : NO)>::NT, ZGeom<N, (NI > NO ? NI : NO)>::MINB)
    k_z_fused(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ tf, ZOp op,
              int Y, int Xh) {
  constexpr int NV = NI > NO ? NI : NO;
  using G = ZGeom<N, NV>;
  constexpr int B = G::B, NT = G::NT;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  float2* htf = buf + NV * N * B;  // [kind][n][b] transfer functions, prefetched
  const int t = blockIdx.z, y = blockIdx.y, x0 = blockIdx.x * B;
  const int w = min(B, Xh - x0);
  const long long zs = (long long)Y * Xh;
  const long long vol = (long long)N * zs;
  const long long col = (long long)y * Xh + x0;
  const int ntf = op.n_tf;
  const int tt = op.tf_shared ? 0 : t;  // the tile whose TFs and statistics apply
#if defined(WO_CHECK) && WO_CHECK
  {  // this strip's elements in the input, output and TF volumes
    const long long span = (long long)(N - 1) * zs + w - 1;
    const long long nt = gridDim.z, ntt = op.tf_shared ? 1 : nt;
    if (!WO_IN((long long)t * NI * vol + (NI - 1) * vol + col + span, nt * NI * vol, 6) ||
        !WO_IN((long long)t * NO * vol + (NO - 1) * vol + col + span, nt * NO * vol, 6) ||
        !WO_IN((long long)tt * ntf * vol + (ntf - 1) * vol + col + span, ntt * ntf * vol, 6))
      return;  // uniform across the CTA
  }
#endif
  if (outside_support(op.stats + (long long)tt * 8, y, Y, x0, 2 * (Xh - 1))) {
    // every TF is zero here, so is every operator's output
    zero_zcols<N, B, NT>(out + (long long)t * NO * vol + col, NO, vol, zs, w);
    return;  // uniform across the CTA
  }
  load_zcols<N, NV, B, NT>(buf, in + (long long)t * NI * vol + col, NI, vol, zs, w);
  for (int q = 0; q < ntf; ++q)
    load_zcols<N, 1, B, NT>(htf + q * N * B, tf + ((long long)tt * ntf + q) * vol + col, 1, vol, zs, w);
  make_twiddles<N>(tw);
  cp_async_wait_all();
  __syncthreads();
  fft_smem<N, NI * B, NT, false, 1>(buf, NV * B, 1, tw);

  const float* st = op.stats + (long long)tt * 8;
  const float lam_lf = op.eta_absolute ? op.eta_lf : op.eta_lf * st[0];
  const float lam_fl = op.eta_absolute ? op.eta_fl : op.eta_fl * st[2];
  const int L = op.lf_props;
  const float2 zero = make_float2(0.f, 0.f);
  // a thread keeps one column b (NT is a multiple of B); columns outside the
  // support disk hold only the TFs' rounding noise: zero out
  static_assert(NT % B == 0, "one column per thread");
  const int bt = threadIdx.x % B;
  const bool col_in = bt < w && !outside_support(st, y, Y, x0 + bt, 2 * (Xh - 1));
  for (int e = threadIdx.x; e < N * B; e += NT) {
    const int k = e / B, b = e % B;  // B is a power of two: shifts
    float2* cell = buf + k * NV * B + b;  // slot v at cell[v * B]
    float2 y0 = zero, y1 = zero, y2 = zero;
    if (col_in) {
      const float2 x0v = cell[0];
      const float2 x1v = NI > 1 ? cell[B] : zero;
      const float2 x2v = NI > 2 ? cell[2 * B] : zero;
      const float2* h = htf + k * B + b;  // slot s at h[s * N * B]
      float2 H[3];
#pragma unroll
      for (int s = 0; s < 3; ++s) H[s] = (s < ntf) ? h[s * N * B] : zero;
      if (op.op == 0) {  // forward: props in, channels out
        if (L > 0) {
          float2 d = cmul(H[0], x0v);
          if (L > 1) d = cadd(d, cmul(H[1], x1v));
          if (op.lf_chan == 0) y0 = d; else y1 = d;
        }
        if (op.has_fl) {
          const float2 d = cmul(H[L], sel3(L, x0v, x1v, x2v));
          if (op.fl_chan == 0) y0 = d; else y1 = d;
        }
      } else if (op.op == 1) {  // adjoint: channels in, props out
        if (L > 0) {
          const float2 d = sel3(op.lf_chan, x0v, x1v, x2v);
          y0 = cmulc(H[0], d);
          if (L > 1) y1 = cmulc(H[1], d);
        }
        if (op.has_fl) {
          const float2 f = cmulc(H[L], sel3(op.fl_chan, x0v, x1v, x2v));
          if (L == 0) y0 = f; else if (L == 1) y1 = f; else y2 = f;
        }
      } else {  // reconstruct
        const bool dc = op.zero_dc && k == 0 && y == 0 && (x0 + b) == 0;
        if (L > 0) {
          const float2 d = dc ? zero : sel3(op.lf_chan, x0v, x1v, x2v);
          float den = lam_lf + cabs2(H[0]);
          if (L > 1) den += cabs2(H[1]);
          const float inv = den > 0.f ? 1.0f / den : 0.f;  // zero TF and eta: minimum norm
          y0 = cscale(cmulc(H[0], d), inv);
          if (L > 1) y1 = cscale(cmulc(H[1], d), inv);
        }
        if (op.has_fl) {
          const float2 d = dc ? zero : sel3(op.fl_chan, x0v, x1v, x2v);
          const float den = lam_fl + cabs2(H[L]);
          const float2 f = cscale(cmulc(H[L], d), den > 0.f ? 1.0f / den : 0.f);
          if (L == 0) y0 = f; else if (L == 1) y1 = f; else y2 = f;
        }
      }
    }
    cell[0] = y0;
    if (NO > 1) cell[B] = y1;
    if (NO > 2) cell[2 * B] = y2;
  }
  __syncthreads();
  fft_smem<N, NO * B, NT, true, 1>(buf, NV * B, 1, tw);
  store_zcols<N, NV, B, NT>(buf, out + (long long)t * NO * vol + col, NO, vol, zs, w);
}

// 2D: out[t][p][y][x] = (sum_k H_k^H H_k + lam I)^-1 sum_k H_k^H D_k per mode.
template <int N, int NI>
__global__ void __launch_bounds__(ZGeom<N, NI>::NT, ZGeom<N, NI>::MINB)
    k_z_solve2d(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ tf, ZOp op,
                int Y, int Xh) {
  using G = ZGeom<N, NI>;
  constexpr int B = G::B, NT = G::NT, KK = NT / B;
  constexpr int NACC = 11;  // m00 m11 m01(2) r0(2) r1(2) mf rf(2)
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* buf = sm + N;
  float* red = reinterpret_cast<float*>(buf + NI * N * B);  // [NT][NACC]
  const int t = blockIdx.z, y = blockIdx.y, x0 = blockIdx.x * B;
  const int w = min(B, Xh - x0);
  const long long zs = (long long)Y * Xh;
  const long long vol = (long long)N * zs;
  const long long col = (long long)y * Xh + x0;
  const int L = op.lf_props;
  const int tt = op.tf_shared ? 0 : t;  // the tile whose TFs and statistics apply
#if defined(WO_CHECK) && WO_CHECK
  {  // this strip's elements in the input and TF volumes, and in the 2D output
    const long long span = (long long)(N - 1) * zs + w - 1;
    const long long nt = gridDim.z, ntt = op.tf_shared ? 1 : nt, np = L + op.has_fl;
    if (!WO_IN((long long)t * NI * vol + (NI - 1) * vol + col + span, nt * NI * vol, 6) ||
        !WO_IN((long long)tt * op.n_tf * vol + (op.n_tf - 1) * vol + col + span, ntt * op.n_tf * vol, 6) ||
        !WO_IN(((long long)t * np + np - 1) * Y * Xh + col + w - 1, nt * np * Y * Xh, 6))
      return;  // uniform across the CTA
  }
#endif
  if (outside_support(op.stats + (long long)tt * 8, y, Y, x0, 2 * (Xh - 1))) {
    if (threadIdx.x < w) {
      float2* o = out + (long long)t * (L + op.has_fl) * Y * Xh + col + threadIdx.x;
      for (int p = 0; p < L + op.has_fl; ++p) o[(long long)p * Y * Xh] = make_float2(0.f, 0.f);
    }
    return;  // uniform across the CTA
  }
  load_zcols<N, NI, B, NT>(buf, in + (long long)t * NI * vol + col, NI, vol, zs, w);
  make_twiddles<N>(tw);
  cp_async_wait_all();
  __syncthreads();
  fft_smem<N, NI * B, NT, false, 1>(buf, NI * B, 1, tw);

  const int b = threadIdx.x % B, kk = threadIdx.x / B;
  float acc[NACC];
#pragma unroll
  for (int i = 0; i < NACC; ++i) acc[i] = 0.f;
  // columns outside the support disk hold only the TFs' rounding noise: zero out
  if (b < w && !outside_support(op.stats + (long long)tt * 8, y, Y, x0 + b, 2 * (Xh - 1))) {
    for (int k = kk; k < N; k += KK) {
      const float2* cell = buf + k * NI * B + b;
      const bool dc = op.zero_dc && k == 0 && y == 0 && (x0 + b) == 0;
      const float2* h = tf + ((long long)tt * op.n_tf * N + k) * zs + col + b;
      if (L > 0) {
        const float2 d = dc ? make_float2(0.f, 0.f) : cell[op.lf_chan * B];
        const float2 h0 = __ldg(h);
        acc[0] += cabs2(h0);
        const float2 r0 = cmulc(h0, d);
        acc[4] += r0.x; acc[5] += r0.y;
        if (L > 1) {
          const float2 h1 = __ldg(h + vol);
          acc[1] += cabs2(h1);
          const float2 m01 = cmulc(h0, h1);
          acc[2] += m01.x; acc[3] += m01.y;
          const float2 r1 = cmulc(h1, d);
          acc[6] += r1.x; acc[7] += r1.y;
        }
      }
      if (op.has_fl) {
        const float2 d = dc ? make_float2(0.f, 0.f) : cell[op.fl_chan * B];
        const float2 hf = __ldg(h + L * vol);
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
    const float* st = op.stats + (long long)tt * 8;
    float2* o = out + (long long)t * (L + op.has_fl) * Y * Xh + (long long)y * Xh + x0 + b;
    const long long plane = (long long)Y * Xh;
    if (L > 0) {
      const float lam = op.eta_absolute ? op.eta_lf * (float)N : op.eta_lf * st[1];
      const float2 r0 = make_float2(acc[4], acc[5]);
      if (L == 1) {
        const float den = acc[0] + lam;
        o[0] = cscale(r0, den > 0.f ? 1.0f / den : 0.f);
      } else {
        const float a = acc[0] + lam, d = acc[1] + lam;
        const float2 m = make_float2(acc[2], acc[3]);
        const float2 r1 = make_float2(acc[6], acc[7]);
        const float det = a * d - cabs2(m);
        const float inv = det > 0.f ? 1.0f / det : 0.f;
        const float2 f0 = csub(cscale(r0, d), cmul(m, r1));
        const float2 f1 = csub(cscale(r1, a), cmulc(m, r0));
        o[0] = cscale(f0, inv);
        o[plane] = cscale(f1, inv);
      }
    }
    if (op.has_fl) {
      const float lam = op.eta_absolute ? op.eta_fl * (float)N : op.eta_fl * st[3];
      const float den = acc[8] + lam;
      o[L * plane] = cscale(make_float2(acc[9], acc[10]), den > 0.f ? 1.0f / den : 0.f);
    }
  }
}

template <int N, int NI, int NO>
cudaError_t launch_z_fused(const float2* in, float2* out, const float2* tf, ZOp op, int n_tiles, int Y, int Xh,
                           cudaStream_t s) {
  constexpr int NV = NI > NO ? NI : NO;
  using G = ZGeom<N, NV>;
  const cudaError_t attr = allow_smem(k_z_fused<N, NI, NO>, G::SMEM_TF);
  if (attr != cudaSuccess) return attr;
  dim3 grid((unsigned)((Xh + G::B - 1) / G::B), (unsigned)Y, (unsigned)n_tiles);
  const size_t smem = G::smem_tf(op.n_tf < 3 ? op.n_tf : 3);
  WO_LAUNCH("z_fused", s, (k_z_fused<N, NI, NO><<<grid, G::NT, smem, s>>>(in, out, tf, op, Y, Xh)));
  return cudaGetLastError();
}

template <int N, int NI>
cudaError_t launch_z_solve2d(const float2* in, float2* out, const float2* tf, ZOp op, int n_tiles, int Y, int Xh,
                             cudaStream_t s) {
  using G = ZGeom<N, NI>;
  const size_t smem = G::SMEM + (size_t)G::NT * 11 * sizeof(float);
  const cudaError_t attr = allow_smem(k_z_solve2d<N, NI>, smem);
  if (attr != cudaSuccess) return attr;
  dim3 grid((unsigned)((Xh + G::B - 1) / G::B), (unsigned)Y, (unsigned)n_tiles);
  WO_LAUNCH("z_solve2d", s, (k_z_solve2d<N, NI><<<grid, G::NT, smem, s>>>(in, out, tf, op, Y, Xh)));
  return cudaGetLastError();
}

}  // namespace wo

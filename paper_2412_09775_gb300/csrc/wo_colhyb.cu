// wo_colhyb.cu - column transforms with coalesced tile copies and
// register-resident transforms (the "hybrid" column engine).
//
// A CTA owns CPC adjacent columns of one plane.  The N x CPC tile is copied
// into shared memory with cp.async in whole row segments (as the
// shared-memory Stockham engine in wo_cols.cu does), then each column is
// transformed by T lanes of one warp in registers (the row transforms of
// wo_regfft.cuh: one padded transpose per transform, warp-level
// synchronisation only), written back to the tile and stored in row
// segments.  The tile pitch P is chosen so that the lanes' column reads and
// writes fall on distinct 8-byte bank pairs within each half-warp.
#include "wo_fft.cuh"
#include "wo_internal.h"
#include "wo_regfft.cuh"

namespace wo {

namespace {

template <class P>
struct HybGeom {
  static constexpr int T = P::T, N = P::N;
  static constexpr int NT = (T <= 16) ? 128 : 256;
  static constexpr int CPC = NT / T;                       // columns per CTA
  static constexpr int PITCH = CPC + (T < 16 ? 16 / T : 1);  // tile row pitch
  static constexpr size_t SMEM =
      ((size_t)N * PITCH + (size_t)CPC * P::SLICE + (size_t)P::TW) * sizeof(float2);
};

template <class P, bool INV>
__global__ void __launch_bounds__(HybGeom<P>::NT, 1)
    k_cols_hyb(float2* __restrict__ data, long long col_stride, long long plane_stride, int ncols,
               long long nplanes, long long total, long long group_stride) {
  using G = HybGeom<P>;
  constexpr int N = G::N, T = G::T, NT = G::NT, CPC = G::CPC, PITCH = G::PITCH, E = P::E;
  extern __shared__ float2 sm[];
  float2* tile = sm;                        // [N][PITCH]
  float2* slices = tile + N * PITCH;        // [CPC][SLICE]
  float2* tw = slices + CPC * P::SLICE;     // [TW]
  const long long q = blockIdx.y + (long long)gridDim.y * blockIdx.z;
  if (q >= total) return;  // uniform across the CTA
  const long long g = q / nplanes, plane = q - g * nplanes;
  const int x0 = blockIdx.x * CPC;
  const int w = min(CPC, ncols - x0);
  float2* base = data + g * group_stride + plane * plane_stride + x0;
  {  // coalesced copy in: one column per thread, walking n
    const int b = threadIdx.x % CPC, n0 = threadIdx.x / CPC;
    constexpr int NSTEP = NT / CPC;
    const bool ok = b < w;
    const float2* src = base + (long long)n0 * col_stride + b;
#pragma unroll 4
    for (int n = n0; n < N; n += NSTEP) {
      cp_async8(tile + n * PITCH + b, ok ? src : base, ok);
      src += NSTEP * col_stride;
    }
  }
  P::twiddles(tw);
  cp_async_wait_all();
  __syncthreads();
  const int t = threadIdx.x % T, cl = threadIdx.x / T;
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = tile[(t + T * m) * PITCH + cl];
  P::template fft<INV>(v, tw, slices + cl * P::SLICE, t);
#pragma unroll
  for (int m = 0; m < E; ++m) tile[(t + T * m) * PITCH + cl] = v[m];
  __syncthreads();
  {  // coalesced copy out
    const int b = threadIdx.x % CPC, n0 = threadIdx.x / CPC;
    constexpr int NSTEP = NT / CPC;
    if (b < w) {
      float2* dst = base + (long long)n0 * col_stride + b;
#pragma unroll 4
      for (int n = n0; n < N; n += NSTEP) {
        *dst = tile[n * PITCH + b];
        dst += NSTEP * col_stride;
      }
    }
  }
}

template <class P>
cudaError_t launch_cols_hyb(bool inv, float2* data, long long cs, long long ps, int ncols, long long nplanes,
                            cudaStream_t s, const char* name, long long groups, long long gs) {
  using G = HybGeom<P>;
  const cudaError_t a0 = allow_smem(k_cols_hyb<P, false>, G::SMEM);
  const cudaError_t a1 = allow_smem(k_cols_hyb<P, true>, G::SMEM);
  if (a0 != cudaSuccess) return a0;
  if (a1 != cudaSuccess) return a1;
  const unsigned gx = (unsigned)((ncols + G::CPC - 1) / G::CPC);
  const long long total = nplanes * groups;
  const long long gy = total < 65535 ? total : 65535;
  const long long gz = (total + gy - 1) / gy;
  dim3 grid(gx, (unsigned)gy, (unsigned)gz);
  if (inv) {
    WO_LAUNCH(name, s, (k_cols_hyb<P, true><<<grid, G::NT, G::SMEM, s>>>(data, cs, ps, ncols, nplanes, total, gs)));
  } else {
    WO_LAUNCH(name, s, (k_cols_hyb<P, false><<<grid, G::NT, G::SMEM, s>>>(data, cs, ps, ncols, nplanes, total, gs)));
  }
  return cudaGetLastError();
}

}  // namespace

bool cols_hyb_supported(int N) {
  return N == 32 || N == 48 || N == 64 || N == 96 || N == 128 || N == 192 || N == 256 || N == 512;
}

cudaError_t cols_c2c_hyb(int N, bool inverse, float2* data, long long col_stride, long long plane_stride, int ncols,
                         long long nplanes, cudaStream_t s, const char* name, long long groups,
                         long long group_stride) {
  using R32 = Row2<32, 8>;
  using R48 = Row2<48, 12>;
  using R64 = Row2<64, 8>;
  using R96 = Row2<96, 24>;
  using R128 = Row2<128, 16>;
  using R192 = Row2<192, 24>;
  using R256 = Row2<256, 16>;
  switch (N) {
#define WO_CH(n, p) \
  case n:           \
    return launch_cols_hyb<p>(inverse, data, col_stride, plane_stride, ncols, nplanes, s, name, groups, group_stride);
    WO_CH(32, R32) WO_CH(48, R48) WO_CH(64, R64) WO_CH(96, R96) WO_CH(128, R128) WO_CH(192, R192)
    WO_CH(256, R256) WO_CH(512, Row512)
#undef WO_CH
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace wo

// wo_cols.cu - in-place complex transforms along a strided axis (y or z).
//
// A CTA owns B adjacent columns of one plane for the whole transform: it
// reads the N x B tile with coalesced B-wide row segments, runs every
// Stockham stage in shared memory and writes the tile back to the same place.
#include "wo_fft.cuh"
#include "wo_internal.h"

namespace wo {

// Copy an N x B column tile (element n of column b at g[n * stride + b]) to
// shared memory [n][b], one column per thread, pointer-walked.
template <int N, int B, int NT>
__device__ __forceinline__ void col_tile_load(float2* buf, const float2* __restrict__ g, long long stride,
                                              int w) {
  constexpr int NSTEP = NT / B;
  const int b = threadIdx.x % B, n0 = threadIdx.x / B;
  const bool ok = b < w;
  const float2* p = g + (long long)n0 * stride + b;
  float2* d = buf + n0 * B + b;
#pragma unroll 4
  for (int n = n0; n < N; n += NSTEP) {
    cp_async8(d, ok ? p : g, ok);
    p += NSTEP * stride;
    d += NSTEP * B;
  }
}

template <int N, int B, int NT>
__device__ __forceinline__ void col_tile_store(const float2* buf, float2* __restrict__ g, long long stride,
                                               int w) {
  constexpr int NSTEP = NT / B;
  const int b = threadIdx.x % B, n0 = threadIdx.x / B;
  if (b >= w) return;
  float2* p = g + (long long)n0 * stride + b;
  const float2* d = buf + n0 * B + b;
#pragma unroll 4
  for (int n = n0; n < N; n += NSTEP) {
    *p = *d;
    p += NSTEP * stride;
    d += NSTEP * B;
  }
}

template <int N, bool INV>
__global__ void __launch_bounds__(ColGeom<N>::NT, ColGeom<N>::MINB)
    k_cols(float2* __restrict__ data, long long col_stride, long long plane_stride, int ncols,
           long long nplanes, long long total, long long group_stride) {
  using G = ColGeom<N>;
  constexpr int B = G::B, NT = G::NT;
  extern __shared__ float2 sm[];
  float2* buf = sm;
  float2* tw = sm + N * B;
  const long long p = blockIdx.y + (long long)gridDim.y * blockIdx.z;
  if (p >= total) return;  // uniform across the CTA
  const long long g = p / nplanes, plane = p - g * nplanes;
  const int x0 = blockIdx.x * B;
  const int w = min(B, ncols - x0);
  float2* base = data + g * group_stride + plane * plane_stride + x0;
#if defined(WO_CHECK) && WO_CHECK
  {  // the elements this tile addresses, against the extent of the passes' volume
    const long long extent = (total / nplanes - 1) * group_stride + (nplanes - 1) * plane_stride +
                             (long long)(N - 1) * col_stride + ncols;
    const long long first = base - data, last = first + (long long)(N - 1) * col_stride + w - 1;
    if (!WO_IN(first, extent, 5) || !WO_IN(last, extent, 5)) return;  // uniform across the CTA
  }
#endif
  col_tile_load<N, B, NT>(buf, base, col_stride, w);
  make_twiddles<N>(tw);  // while the tile's copies are in flight
  cp_async_wait_all();
  __syncthreads();
  fft_smem<N, B, NT, INV, 1>(buf, B, 1, tw);
  col_tile_store<N, B, NT>(buf, base, col_stride, w);
}

template <int N>
static cudaError_t launch_cols(bool inv, float2* data, long long cs, long long ps, int ncols,
                               long long nplanes, cudaStream_t s, const char* name, long long groups,
                               long long gs) {
  using G = ColGeom<N>;
  const size_t smem = G::SMEM;
  const cudaError_t a0 = allow_smem(k_cols<N, false>, smem);
  const cudaError_t a1 = allow_smem(k_cols<N, true>, smem);
  if (a0 != cudaSuccess) return a0;
  if (a1 != cudaSuccess) return a1;
  const unsigned gx = (unsigned)((ncols + G::B - 1) / G::B);
  const long long total = nplanes * groups;
  const long long gy = total < 65535 ? total : 65535;
  const long long gz = (total + gy - 1) / gy;
  dim3 grid(gx, (unsigned)gy, (unsigned)gz);
  if (inv) {
    WO_LAUNCH(name, s, (k_cols<N, true><<<grid, G::NT, smem, s>>>(data, cs, ps, ncols, nplanes, total, gs)));
  } else {
    WO_LAUNCH(name, s, (k_cols<N, false><<<grid, G::NT, smem, s>>>(data, cs, ps, ncols, nplanes, total, gs)));
  }
  return cudaGetLastError();
}

cudaError_t cols_c2c(int N, bool inverse, float2* data, long long col_stride, long long plane_stride,
                     int ncols, long long nplanes, cudaStream_t s, const char* name, long long groups,
                     long long group_stride) {
  if (N == 1 || nplanes <= 0 || ncols <= 0 || groups <= 0) return cudaSuccess;  // identity
  if (cols_engine(N) == WO_ENGINE_HYBRID)
    return cols_c2c_hyb(N, inverse, data, col_stride, plane_stride, ncols, nplanes, s, name, groups, group_stride);
  switch (N) {
#define WO_CASE(n) \
  case n:          \
    return launch_cols<n>(inverse, data, col_stride, plane_stride, ncols, nplanes, s, name, groups, group_stride);
    WO_CASE(2) WO_CASE(3) WO_CASE(4) WO_CASE(6) WO_CASE(8) WO_CASE(12) WO_CASE(16) WO_CASE(24)
    WO_CASE(32) WO_CASE(48) WO_CASE(64) WO_CASE(96) WO_CASE(128) WO_CASE(192) WO_CASE(256)
    WO_CASE(384) WO_CASE(512) WO_CASE(768) WO_CASE(1024) WO_CASE(1536) WO_CASE(2048)
#undef WO_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace wo

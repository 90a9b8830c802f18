// wo_pad.cu - padding in place of circular boundaries.
//
// The Fourier-space operators treat every volume as periodic in x, y and z
// (Eq. fwd in its Fourier form).  A caller that wants other boundaries pads
// the volume to a larger supported grid, runs the operator there, and crops
// the result back.  wo_pad writes [n][Zp][Yp][Xp] from [n][Z][Y][X] with the
// input at offset ((Zp-Z)/2, (Yp-Y)/2, (Xp-X)/2) and the margin filled by
// zeros, by the nearest edge sample, or by the mirror image about the edge
// samples (index -i, 2(n-1) - i, repeated with period 2(n-1)); wo_crop takes
// the same window back out.  Both are plain streaming copies: one warp per
// output row, lanes along x, so reads and writes are coalesced except where
// a mirrored margin runs backwards.
#include "wo_internal.h"

namespace wo {

__device__ __forceinline__ int pad_index(int i, int n, int mode) {
  if (i >= 0 && i < n) return i;
  if (mode == WO_PAD_ZERO) return -1;
  if (mode == WO_PAD_EDGE) return i < 0 ? 0 : n - 1;
  if (n == 1) return 0;
  const int p = 2 * (n - 1);
  int r = i % p;
  if (r < 0) r += p;
  return r < n ? r : p - r;
}

__global__ void __launch_bounds__(256)
    k_pad(const float* __restrict__ in, long long n_rows, int Z, int Y, int X, int Zp, int Yp, int Xp, int oz,
          int oy, int ox, int mode, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * 8;
  for (long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5); row < n_rows; row += warps) {
    const long long vz = row / Yp;  // v * Zp + z
    const int yo = (int)(row - vz * Yp);
    const long long v = vz / Zp;
    const int zo = (int)(vz - v * Zp);
    const int zi = pad_index(zo - oz, Z, mode), yi = pad_index(yo - oy, Y, mode);
    float* dst = out + row * Xp;
    if (zi < 0 || yi < 0) {
      for (int x = lane; x < Xp; x += 32) dst[x] = 0.f;
      continue;
    }
    const float* src = in + ((v * Z + zi) * Y + yi) * (long long)X;
    for (int x = lane; x < Xp; x += 32) {
      const int xi = pad_index(x - ox, X, mode);
      dst[x] = xi < 0 ? 0.f : __ldg(src + xi);
    }
  }
}

__global__ void __launch_bounds__(256)
    k_crop(const float* __restrict__ in, long long n_rows, int Zp, int Yp, int Xp, int Z, int Y, int X, int oz,
           int oy, int ox, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * 8;
  for (long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5); row < n_rows; row += warps) {
    const long long vz = row / Y;  // v * Z + z
    const int y = (int)(row - vz * Y);
    const long long v = vz / Z;
    const int z = (int)(vz - v * Z);
    const float* src = in + ((v * Zp + z + oz) * Yp + y + oy) * (long long)Xp + ox;
    float* dst = out + row * X;
    for (int x = lane; x < X; x += 32) dst[x] = __ldg(src + x);
  }
}

// Blocks for a grid-stride loop over rows, eight rows (warps) per block:
// up to eight resident blocks on each of the GPU's SMs.
static unsigned row_blocks(long long rows) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) ==
                                                   cudaSuccess && v > 0)
      sms = v;
    else
      sms = 152;
  }
  const long long want = (rows + 7) / 8, cap = 8LL * sms;
  return (unsigned)(want < cap ? want : cap);
}

static bool pad_shape_ok(int n_vol, int Z, int Y, int X, int Zp, int Yp, int Xp) {
  if (n_vol < 1 || Z < 1 || Y < 1 || X < 1) return false;
  if (Zp < Z || Yp < Y || Xp < X) return false;
  const long long big = (long long)n_vol * Zp * Yp * Xp;
  return big < (1LL << 40);
}

}  // namespace wo

using namespace wo;

extern "C" {

wo_status wo_pad(const float* d_in, int n_vol, int Z, int Y, int X, int Zp, int Yp, int Xp, int mode, float* d_out,
                 wo_stream stream) {
  if (!d_in || !d_out || d_in == d_out) return WO_ERR_ARG;
  if (mode != WO_PAD_ZERO && mode != WO_PAD_MIRROR && mode != WO_PAD_EDGE) return WO_ERR_ARG;
  if (!pad_shape_ok(n_vol, Z, Y, X, Zp, Yp, Xp)) return WO_ERR_SHAPE;
  cudaStream_t s = (cudaStream_t)stream;
  const long long rows = (long long)n_vol * Zp * Yp;
  WO_LAUNCH("pad", s,
            (k_pad<<<row_blocks(rows), 256, 0, s>>>(d_in, rows, Z, Y, X, Zp, Yp, Xp, (Zp - Z) / 2, (Yp - Y) / 2,
                                                      (Xp - X) / 2, mode, d_out)));
  return cudaGetLastError() == cudaSuccess ? WO_OK : WO_ERR_CUDA;
}

wo_status wo_crop(const float* d_in, int n_vol, int Zp, int Yp, int Xp, int Z, int Y, int X, float* d_out,
                  wo_stream stream) {
  if (!d_in || !d_out || d_in == d_out) return WO_ERR_ARG;
  if (!pad_shape_ok(n_vol, Z, Y, X, Zp, Yp, Xp)) return WO_ERR_SHAPE;
  cudaStream_t s = (cudaStream_t)stream;
  const long long rows = (long long)n_vol * Z * Y;
  WO_LAUNCH("crop", s,
            (k_crop<<<row_blocks(rows), 256, 0, s>>>(d_in, rows, Zp, Yp, Xp, Z, Y, X, (Zp - Z) / 2, (Yp - Y) / 2,
                                                       (Xp - X) / 2, d_out)));
  return cudaGetLastError() == cudaSuccess ? WO_OK : WO_ERR_CUDA;
}

}  // extern "C"

// wo_tiles.cu - overlapping tiles for shift-variant restoration (Fig. 2a;
// Methods, "Organelle-scale optical pooled screen data": tiling and
// linearly weighted stitching).
//
// Tile (ty, tx) covers field rows ty*core - halo .. ty*core + core + halo and
// likewise in x; pixels outside the field are mirror-padded (-i, 2(n-1)-i).
// Blending weights are separable linear ramps over the 2*halo overlap,
//   w(u) = min(1, (u + 1/2)/(2 halo), (E - u - 1/2)/(2 halo)),
// and the field is sum_t w_t tile_t / sum_t w_t.  With 2*halo <= core every
// field pixel is covered by at most two tiles per axis.
#include "wo_internal.h"
#include "wo_tiles.cuh"

namespace wo {

// Gather: one thread per 4 consecutive tile pixels of a row.  When the four
// field pixels are in range they are contiguous and 16-byte aligned (tile
// origins and the field width are multiples of 4 when core and halo are), so
// the copy is one float4 load and store; mirrored edges fall back to scalars.
__global__ void __launch_bounds__(256)
    k_gather(const float* __restrict__ field, int Z, int tiles_x, int core, int halo, int Yf, int Xf,
             float* __restrict__ tiles, int vec) {
  const int E = core + 2 * halo;
  const int E4 = (E + 3) / 4;
  const long long tz = blockIdx.y;  // t * Z + z
  const long long t = tz / Z, z = tz - (tz / Z) * Z;
  const int ty = (int)(t / tiles_x), tx = (int)(t - (t / tiles_x) * tiles_x);
  const float* src = field + z * (long long)Yf * Xf;
  float* dst = tiles + tz * (long long)E * E;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < E * E4; i += gridDim.x * 256) {
    const int u = i / E4, v0 = (i - (i / E4) * E4) * 4;
    const int y = mirror_idx(ty * core - halo + u, Yf);
    const int xs = tx * core - halo + v0;
    const float* row = src + (long long)y * Xf;
    if (!WO_IN(tz * (long long)E * E + (long long)u * E + min(v0 + 3, E - 1), (long long)gridDim.y * E * E, 4) ||
        !WO_IN(z * (long long)Yf * Xf + (long long)y * Xf, (long long)Z * Yf * Xf, 4))
      continue;
    if (vec && xs >= 0 && xs + 3 < Xf && v0 + 3 < E) {
      *reinterpret_cast<float4*>(dst + (long long)u * E + v0) = __ldg(reinterpret_cast<const float4*>(row + xs));
    } else {
      for (int k = 0; k < 4 && v0 + k < E; ++k) dst[(long long)u * E + v0 + k] = __ldg(row + mirror_idx(xs + k, Xf));
    }
  }
}

// Blend: one thread per L consecutive field pixels of a row (L = 4 when
// core and halo are multiples of 4, else 1); the covering tiles (at most two
// per axis) are the same for the L pixels, only the x weights differ.  The
// kernel is bound by instruction issue, so the weights' reciprocal is formed
// once per thread and each covering tile column's x weights once per group,
// with the values and summation order of the plain per-tile form; eight
// CTAs per SM (32 registers) keep every warp slot filled.
template <int L>
__global__ void __launch_bounds__(256, 8)
    k_blend(const float* __restrict__ tiles, int Z, int tiles_y, int tiles_x, int core, int halo,
            float* __restrict__ field) {
  const int E = core + 2 * halo;
  const int Yf = tiles_y * core, Xf = tiles_x * core;
  const long long zy = blockIdx.x;  // z * Yf + y
  const long long z = zy / Yf;
  const int y = (int)(zy - z * Yf);
  const float inv = halo > 0 ? 1.0f / (2.0f * (float)halo) : 0.f;
  auto weight = [&](int u) { return halo > 0 ? ramp_inv(u, E, inv) : 1.f; };
  int tys[2], us[2];
  float wys[2];
  int ny = 0;
  const int qy = (y + halo) / core;
  for (int c = qy - 1; c <= qy; ++c) {
    if (c < 0 || c >= tiles_y) continue;
    const int u = y - (c * core - halo);
    if (u < 0 || u >= E) continue;
    tys[ny] = c; us[ny] = u; wys[ny] = weight(u); ++ny;
  }
  const int nvec = Xf / L;  // Xf is a multiple of L
  for (int i = threadIdx.x; i < nvec; i += 256) {
    const int x0 = L * i;
    float acc[L], wsum[L];
#pragma unroll
    for (int k = 0; k < L; ++k) acc[k] = wsum[k] = 0.f;
    const int qx = (x0 + halo) / core;
    for (int c = qx - 1; c <= qx; ++c) {
      if (c < 0 || c >= tiles_x) continue;
      const int v = x0 - (c * core - halo);
      if (v < 0 || v >= E) continue;  // L = 4: v..v+3 lie in the same tile
      float wx[L];
#pragma unroll
      for (int k = 0; k < L; ++k) wx[k] = weight(v + k);
      for (int a = 0; a < ny; ++a) {
        const long long t = (long long)tys[a] * tiles_x + c;
        if (!WO_IN(((t * Z + z) * E + us[a]) * (long long)E + v + L - 1, (long long)tiles_y * tiles_x * Z * E * E, 4))
          continue;
        const float* src = tiles + ((t * Z + z) * E + us[a]) * (long long)E + v;
        float val[L];
        if constexpr (L == 4) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(src));
          val[0] = q.x; val[1] = q.y; val[2] = q.z; val[3] = q.w;
        } else {
          val[0] = __ldg(src);
        }
#pragma unroll
        for (int k = 0; k < L; ++k) {
          const float wgt = wys[a] * wx[k];
          acc[k] += wgt * val[k];
          wsum[k] += wgt;
        }
      }
    }
    float* dst = field + zy * (long long)Xf + x0;
    if (!WO_IN(zy * (long long)Xf + x0 + L - 1, (long long)gridDim.x * Xf, 4)) continue;
    if constexpr (L == 4) {
      *reinterpret_cast<float4*>(dst) =
          make_float4(acc[0] / wsum[0], acc[1] / wsum[1], acc[2] / wsum[2], acc[3] / wsum[3]);
    } else {
      dst[0] = acc[0] / wsum[0];
    }
  }
}

cudaError_t tiles_gather(const float* field, int Z, int ty, int tx, int core, int halo, float* tiles,
                         cudaStream_t s) {
  const int E = core + 2 * halo;
  const int vec = (core % 4 == 0 && halo % 4 == 0) ? 1 : 0;
  const long long work = (long long)E * ((E + 3) / 4);
  dim3 grid((unsigned)((work + 255) / 256), (unsigned)((long long)ty * tx * Z));
  WO_LAUNCH("tile_gather", s, (k_gather<<<grid, 256, 0, s>>>(field, Z, tx, core, halo, ty * core, tx * core, tiles, vec)));
  return cudaGetLastError();
}

cudaError_t tiles_blend(const float* tiles, int Z, int ty, int tx, int core, int halo, float* field,
                        cudaStream_t s) {
  const int vec = (core % 4 == 0 && halo % 4 == 0) ? 1 : 0;
  dim3 grid((unsigned)((long long)ty * core * Z));
  if (vec) WO_LAUNCH("tile_blend", s, (k_blend<4><<<grid, 256, 0, s>>>(tiles, Z, ty, tx, core, halo, field)));
  else WO_LAUNCH("tile_blend", s, (k_blend<1><<<grid, 256, 0, s>>>(tiles, Z, ty, tx, core, halo, field)));
  return cudaGetLastError();
}

}  // namespace wo

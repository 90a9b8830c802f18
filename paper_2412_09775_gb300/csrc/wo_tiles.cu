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

namespace wo {

__device__ __forceinline__ int mirror_idx(int i, int n) {
  i = i < 0 ? -i : i;
  return i >= n ? 2 * (n - 1) - i : i;
}

__device__ __forceinline__ float ramp(int u, int E, int halo) {
  if (halo == 0) return 1.f;
  const float inv = 1.0f / (2.0f * (float)halo);
  return fminf(1.f, fminf(((float)u + 0.5f) * inv, ((float)(E - u) - 0.5f) * inv));
}

__global__ void __launch_bounds__(128)
    k_gather(const float* __restrict__ field, int Z, int tiles_x, int core, int halo, int Yf, int Xf,
             float* __restrict__ tiles) {
  const int E = core + 2 * halo;
  const int v = blockIdx.x * 128 + threadIdx.x;
  if (v >= E) return;
  const int u = blockIdx.y;
  const long long tz = blockIdx.z;
  const long long t = tz / Z, z = tz - (tz / Z) * Z;
  const int ty = (int)(t / tiles_x), tx = (int)(t - (t / tiles_x) * tiles_x);
  const int y = mirror_idx(ty * core - halo + u, Yf);
  const int x = mirror_idx(tx * core - halo + v, Xf);
  tiles[((t * Z + z) * E + u) * (long long)E + v] = __ldg(field + (z * Yf + y) * (long long)Xf + x);
}

__global__ void __launch_bounds__(128)
    k_blend(const float* __restrict__ tiles, int Z, int tiles_y, int tiles_x, int core, int halo,
            float* __restrict__ field) {
  const int E = core + 2 * halo;
  const int Yf = tiles_y * core, Xf = tiles_x * core;
  const int x = blockIdx.x * 128 + threadIdx.x;
  if (x >= Xf) return;
  const int y = blockIdx.y;
  const long long z = blockIdx.z;
  int tys[2], us[2], txs[2], vs[2];
  float wys[2], wxs[2];
  int ny = 0, nx = 0;
  const int qy = (y + halo) / core, qx = (x + halo) / core;
  for (int c = qy - 1; c <= qy; ++c) {
    if (c < 0 || c >= tiles_y) continue;
    const int u = y - (c * core - halo);
    if (u < 0 || u >= E) continue;
    tys[ny] = c; us[ny] = u; wys[ny] = ramp(u, E, halo); ++ny;
  }
  for (int c = qx - 1; c <= qx; ++c) {
    if (c < 0 || c >= tiles_x) continue;
    const int v = x - (c * core - halo);
    if (v < 0 || v >= E) continue;
    txs[nx] = c; vs[nx] = v; wxs[nx] = ramp(v, E, halo); ++nx;
  }
  float acc = 0.f, wsum = 0.f;
  for (int i = 0; i < ny; ++i) {
    for (int k = 0; k < nx; ++k) {
      const long long t = (long long)tys[i] * tiles_x + txs[k];
      const float wgt = wys[i] * wxs[k];
      acc += wgt * __ldg(tiles + ((t * Z + z) * E + us[i]) * (long long)E + vs[k]);
      wsum += wgt;
    }
  }
  field[(z * Yf + y) * (long long)Xf + x] = acc / wsum;
}

cudaError_t tiles_gather(const float* field, int Z, int ty, int tx, int core, int halo, float* tiles,
                         cudaStream_t s) {
  const int E = core + 2 * halo;
  dim3 grid((unsigned)((E + 127) / 128), (unsigned)E, (unsigned)((long long)ty * tx * Z));
  WO_LAUNCH("tile_gather", s, (k_gather<<<grid, 128, 0, s>>>(field, Z, tx, core, halo, ty * core, tx * core, tiles)));
  return cudaGetLastError();
}

cudaError_t tiles_blend(const float* tiles, int Z, int ty, int tx, int core, int halo, float* field,
                        cudaStream_t s) {
  dim3 grid((unsigned)((tx * core + 127) / 128), (unsigned)(ty * core), (unsigned)Z);
  WO_LAUNCH("tile_blend", s, (k_blend<<<grid, 128, 0, s>>>(tiles, Z, ty, tx, core, halo, field)));
  return cudaGetLastError();
}

}  // namespace wo

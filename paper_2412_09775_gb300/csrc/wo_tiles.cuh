// wo_tiles.cuh - tile geometry shared by the tile kernels and the row passes
// that read and write tiles in place.
//
// Tile (ty, tx) covers field rows ty*core - halo .. ty*core + core + halo and
// likewise in x; pixels outside the field are mirror-padded (-i, 2(n-1)-i).
// Blending weights are separable linear ramps over the 2*halo overlap,
//   w(u) = min(1, (u + 1/2)/(2 halo), (E - u - 1/2)/(2 halo)).
#pragma once

namespace wo {

__device__ __forceinline__ int mirror_idx(int i, int n) {
  i = i < 0 ? -i : i;
  return i >= n ? 2 * (n - 1) - i : i;
}

// The ramp for halo > 0 with inv = 1 / (2 halo) formed by the caller.
__device__ __forceinline__ float ramp_inv(int u, int E, float inv) {
  return fminf(1.f, fminf(((float)u + 0.5f) * inv, ((float)(E - u) - 0.5f) * inv));
}

__device__ __forceinline__ float ramp(int u, int E, int halo) {
  if (halo == 0) return 1.f;
  return ramp_inv(u, E, 1.0f / (2.0f * (float)halo));
}

}  // namespace wo

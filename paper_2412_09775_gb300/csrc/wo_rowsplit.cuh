// wo_rowsplit.cuh - the real <-> half-spectrum split of a row held by T
// lanes of a warp (the register-resident row transforms of wo_regfft.cuh).
//
// A real row of 2N samples is read as N complex samples z[n] = x[2n] +
// i x[2n+1] and transformed with a length-N complex FFT; its N+1 bins are
//   X[k] = (Z[k] + Z*[N-k])/2 - (i/2) e^{-2 pi i k/2N} (Z[k] - Z*[N-k]),
//   X[N] = Re Z[0] - Im Z[0],
// and back, Z[k] = A + iB with A = (X[k] + X*[N-k])/2 and
// B = (X[k] - X*[N-k]) e^{+2 pi i k/2N}/2, then a length-N inverse FFT.
// Lane t owns the points k = t + T m; the partner value Z*[N-k] lives in the
// lane that owns N - k and comes by a shuffle (all 32 lanes take part).
#pragma once
#include "wo_fft.cuh"
#include "wo_internal.h"

namespace wo {

// Background constant of a row (see RowBg): mode 1 the channel's value, mode 2
// the first sample of the row's (tile, channel) block.
__device__ __forceinline__ float row_constant(const float* in, long long row, long long n2, const RowBg& bg) {
  const long long grow = bg.row_offset + row;
  if (bg.mode == 1) return bg.v[(grow / bg.rows_per_block) % bg.nchan];
  if (bg.mode == 2) return __ldg(in + ((grow / bg.rows_per_block) * bg.rows_per_block - bg.row_offset) * n2);
  return 0.f;
}

// The partner lane owns N - k, and the register it sends for our register m
// is mirror(m) (lane 0: point T m pairs with T ((E - m) mod E); lane t > 0:
// t + T m pairs with (T - t) + T (E-1-m)).
template <int E>
__device__ __forceinline__ float2 mirror_reg(const float2 (&v)[E], int m, bool lane0) {
  return lane0 ? v[(E - m) % E] : v[E - 1 - m];
}

__device__ __forceinline__ int split_partner(int t, int T) {
  const int lane = threadIdx.x & 31;
  return (lane - t) + (T - t) % T;
}

// After the forward transform of z (v): emit(k, X[k]) for the lane's points
// k = t + T m, and emit(N, X[N]) on lane 0.  tw2[k] = e^{-2 pi i k/2N}.
template <int N, int T, int E, class Emit>
__device__ __forceinline__ void r2c_split(const float2 (&v)[E], const float2* tw2, int t, Emit emit) {
  const int partner = split_partner(t, T);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const float2 mv = mirror_reg<E>(v, m, t == 0);
    const float2 zc = make_float2(__shfl_sync(0xffffffffu, mv.x, partner), -__shfl_sync(0xffffffffu, mv.y, partner));
    const int k = t + T * m;
    const float2 s = cadd(v[m], zc);
    const float2 u = cmul(tw2[k], csub(v[m], zc));
    emit(k, make_float2(0.5f * (s.x + u.y), 0.5f * (s.y - u.x)));
  }
  if (t == 0) emit(N, make_float2(v[0].x - v[0].y, 0.f));
}

// Before the inverse transform: v[m] = Z[k] from the lane's bins x[m] = X[k]
// and, on lane 0, xn = X[N] (the partner of X[0]).
template <int T, int E>
__device__ __forceinline__ void c2r_merge(const float2 (&x)[E], float2 xn, const float2* tw2, int t, float2 (&v)[E]) {
  const int partner = split_partner(t, T);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const float2 mv = mirror_reg<E>(x, m, t == 0);
    float2 xc = make_float2(__shfl_sync(0xffffffffu, mv.x, partner), -__shfl_sync(0xffffffffu, mv.y, partner));
    if (t == 0 && m == 0) xc = make_float2(xn.x, -xn.y);
    const int k = t + T * m;
    const float2 a = make_float2(0.5f * (x[m].x + xc.x), 0.5f * (x[m].y + xc.y));
    const float2 b = cmul(make_float2(0.5f * (x[m].x - xc.x), 0.5f * (x[m].y - xc.y)), cconj(tw2[k]));
    v[m] = make_float2(a.x - b.y, a.y + b.x);
  }
}

}  // namespace wo

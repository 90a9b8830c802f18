// wo_rowsreg.cu - transforms along x (real <-> half spectrum) with register-
// resident row transforms (the "hybrid" engine of the row passes).
//
// Same operations as k_rows_r2c / k_rows_c2r (wo_rows.cu): a real row of 2N
// samples is read as N complex samples z[n] = x[2n] + i x[2n+1], transformed
// with a length-N complex FFT and split into the N+1 bins of the real
// transform,
//   X[k] = (Z[k] + Z*[N-k])/2 - (i/2) e^{-2 pi i k/2N} (Z[k] - Z*[N-k]),
//   X[N] = Re Z[0] - Im Z[0],
// and back (Z[k] = A + iB, A = (X[k] + X*[N-k])/2,
// B = (X[k] - X*[N-k]) e^{+2 pi i k/2N}/2, then a length-N inverse FFT).  Here
// T lanes of one warp own a row, lane t holding points t + T m (the row
// transforms of wo_regfft.cuh): the row is loaded straight into registers
// (16 lanes read 16 consecutive complex samples), the partner value
// Z*[N-k] comes from the lane that owns N - k by a shuffle, and only the
// transform's transposes touch shared memory.
#include "wo_fft.cuh"
#include "wo_internal.h"
#include "wo_regfft.cuh"
#include "wo_rowsplit.cuh"
#include "wo_tiles.cuh"

namespace wo {

namespace {

constexpr int kRowThreads = 128;

template <class P>
struct RowRegGeom {
  static constexpr int N = P::N, T = P::T, E = P::E;
  static constexpr int RPC = kRowThreads / T;  // rows per CTA
  static constexpr size_t SMEM = ((size_t)P::TW + 2 * (size_t)N + (size_t)RPC * P::SLICE) * sizeof(float2);
};

// PY > 0: the output is kx-major, [block][N+1][Z][PY] (the plane engine's
// layout; a row's bins at o + k Z PY, the 32/T rows of a warp consecutive
// rows of one plane: whole 32-byte sectors per bin), Z the planes per block.
template <class P, int PY = 0>
__global__ void __launch_bounds__(kRowThreads) k_rows_r2c_reg(const float* __restrict__ in, float2* __restrict__ out,
                                                               long long nrows, RowBg bg, int Z) {
  using G = RowRegGeom<P>;
  constexpr int N = G::N, T = G::T, E = G::E, RPC = G::RPC;
  extern __shared__ float2 sm[];
  float2* tw = sm;                  // P's twiddles
  float2* tw2 = sm + P::TW;         // exp(-2 pi i m / 2N)
  const int t = threadIdx.x % T, r = threadIdx.x / T;
  float2* S = sm + P::TW + 2 * N + r * P::SLICE;
  const long long row = (long long)blockIdx.x * RPC + r;
  const bool live0 = row < nrows;
  long long rr = live0 ? row : nrows - 1;  // tail lanes transform a valid row and store nothing
  // (a failed index check turns the row into a tail row: the block's barriers are still met)
  const bool inside = WO_IN(rr, nrows, 7);
  if (!inside) rr = 0;
  const bool live = live0 && inside;
  const float c = row_constant(in, rr, 2LL * N, bg);
  const float2* src = reinterpret_cast<const float2*>(in + rr * (2LL * N)) + t;
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = __ldg(src + T * m);
  P::twiddles(tw);  // while the row's loads are in flight
  make_twiddles<2 * N>(tw2);
  __syncthreads();
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = make_float2(v[m].x - c, v[m].y - c);
  P::template fft<false>(v, tw, S, t);
  if constexpr (PY > 0) {
    const long long plane_rows = (long long)Z * PY;
    const long long blk = rr / plane_rows, rem = rr - blk * plane_rows;  // rem = z PY + y
    const long long ob = blk * (N + 1) * plane_rows + rem;
    float2* o = out + ob;
    r2c_split<N, T, E>(v, tw2, t, [&](int k, float2 val) {
      if (live && WO_IN(ob + k * plane_rows, nrows * (N + 1), 7)) o[k * plane_rows] = val;
    });
  } else {
    float2* o = out + rr * (N + 1);
    r2c_split<N, T, E>(v, tw2, t, [&](int k, float2 val) {
      if (live) o[k] = val;
    });
  }
}

template <class P, int PY>
cudaError_t launch_r2c_kxm(const float* in, float2* out, long long nrows, int Z, RowBg bg, cudaStream_t s) {
  using G = RowRegGeom<P>;
  const cudaError_t attr = allow_smem(k_rows_r2c_reg<P, PY>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  const long long blocks = (nrows + G::RPC - 1) / G::RPC;
  WO_LAUNCH("rows_r2c", s,
            (k_rows_r2c_reg<P, PY><<<(unsigned)blocks, kRowThreads, G::SMEM, s>>>(in, out, nrows, bg, Z)));
  return cudaGetLastError();
}

template <class P>
__global__ void __launch_bounds__(kRowThreads) k_rows_c2r_reg(const float2* __restrict__ in, float* __restrict__ out,
                                                               long long nrows, float scale, RowBg bg) {
  using G = RowRegGeom<P>;
  constexpr int N = G::N, T = G::T, E = G::E, RPC = G::RPC;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* tw2 = sm + P::TW;
  const int t = threadIdx.x % T, r = threadIdx.x / T;
  float2* S = sm + P::TW + 2 * N + r * P::SLICE;
  const long long row = (long long)blockIdx.x * RPC + r;
  const bool live0 = row < nrows;
  long long rr = live0 ? row : nrows - 1;
  const bool inside = WO_IN(rr, nrows, 7);
  if (!inside) rr = 0;
  const bool live = live0 && inside;
  const float2* src = in + rr * (N + 1) + t;
  float2 x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) x[m] = __ldg(src + T * m);
  const float2 xn = t == 0 ? __ldg(in + rr * (N + 1) + N) : make_float2(0.f, 0.f);  // X[N], partner of X[0]
  P::twiddles(tw);  // while the row's loads are in flight
  make_twiddles<2 * N>(tw2);
  __syncthreads();
  float2 v[E];
  c2r_merge<T, E>(x, xn, tw2, t, v);
  P::template fft<true>(v, tw, S, t);
  if (!live) return;
  const float cst = bg.mode == 1 ? bg.v[((bg.row_offset + rr) / bg.rows_per_block) % bg.nchan] : 0.f;
  float2* o = reinterpret_cast<float2*>(out + rr * (2LL * N)) + t;
#pragma unroll
  for (int m = 0; m < E; ++m) o[T * m] = make_float2(v[m].x * scale + cst, v[m].y * scale + cst);
}

// k_rows_r2c_reg with the rows read from the tiles of a field (FieldSrc):
// tile row (t, z, u) is field row mirror(ty core - halo + u) of plane z,
// samples mirror(tx core - halo + x); a tile whose columns lie inside the
// field reads them as pairs, a border tile one mirrored sample at a time.
// The mode-2 background is the tile's first sample, as for a gathered tile.
//
// KXM: the output is kx-major, [tile][k][z][u] (the plane engine's layout,
// wo_plane.cu): each lane stores its row's bins straight from registers; the
// 32/T rows of a warp are consecutive rows u of one plane, so a warp store
// of one register fills a run of 32/T points of each of T bins (whole
// 32-byte sectors).
template <class P, bool KXM>
__global__ void __launch_bounds__(kRowThreads) k_rows_r2c_field(FieldSrc f, float2* __restrict__ out, long long nrows,
                                                                 RowBg bg) {
  using G = RowRegGeom<P>;
  constexpr int N = G::N, T = G::T, E = G::E, RPC = G::RPC, W = 2 * N;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* tw2 = sm + P::TW;
  const int t = threadIdx.x % T, r = threadIdx.x / T;
  float2* S = sm + P::TW + 2 * N + r * P::SLICE;
  const long long row = (long long)blockIdx.x * RPC + r;
  const bool live0 = row < nrows;
  long long rr = live0 ? row : nrows - 1;
  const bool inside = WO_IN(rr, nrows, 7);
  if (!inside) rr = 0;
  const bool live = live0 && inside;
  const int Yf = f.tiles_y * f.core, Xf = f.tiles_x * f.core;
  const long long per_tile = (long long)f.Z * W;
  const long long tile = rr / per_tile, rem = rr - tile * per_tile;
  const int z = (int)(rem / W), u = (int)(rem - (long long)(rem / W) * W);
  const int ty = (int)(tile / f.tiles_x), tx = (int)(tile - (tile / f.tiles_x) * f.tiles_x);
  const int y0 = ty * f.core - f.halo, xs0 = tx * f.core - f.halo;
  const float* frow = f.field + ((long long)z * Yf + mirror_idx(y0 + u, Yf)) * Xf;
  float c = 0.f;
  if (bg.mode == 1) c = bg.v[((bg.row_offset + rr) / bg.rows_per_block) % bg.nchan];
  if (bg.mode == 2) c = __ldg(f.field + (long long)mirror_idx(y0, Yf) * Xf + mirror_idx(xs0, Xf));
  const bool pairs = xs0 >= 0 && xs0 + W <= Xf && ((xs0 | Xf) & 1) == 0;  // uniform per tile
  float2 v[E];
  if (pairs) {
    const float2* src = reinterpret_cast<const float2*>(frow + xs0) + t;
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = __ldg(src + T * m);
  } else {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int x = xs0 + 2 * (t + T * m);
      v[m] = make_float2(__ldg(frow + mirror_idx(x, Xf)), __ldg(frow + mirror_idx(x + 1, Xf)));
    }
  }
  P::twiddles(tw);  // while the row's loads are in flight
  make_twiddles<2 * N>(tw2);
  __syncthreads();
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = make_float2(v[m].x - c, v[m].y - c);
  P::template fft<false>(v, tw, S, t);
  if constexpr (KXM) {
    const long long ob = (tile * (N + 1) * f.Z + z) * (long long)W + u;  // bin k at ob + k Z W
    float2* o = out + ob;
    const long long kstep = (long long)f.Z * W;
    r2c_split<N, T, E>(v, tw2, t, [&](int k, float2 val) {
      if (live && WO_IN(ob + k * kstep, nrows * (N + 1), 7)) o[k * kstep] = val;
    });
  } else {
    float2* o = out + rr * (N + 1);
    r2c_split<N, T, E>(v, tw2, t, [&](int k, float2 val) {
      if (live) o[k] = val;
    });
  }
}

template <class P, bool KXM>
cudaError_t launch_r2c_field(const FieldSrc& f, float2* out, long long nrows, RowBg bg, cudaStream_t s) {
  using G = RowRegGeom<P>;
  const cudaError_t attr = allow_smem(k_rows_r2c_field<P, KXM>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  const long long blocks = (nrows + G::RPC - 1) / G::RPC;
  WO_LAUNCH("rows_r2c", s,
            (k_rows_r2c_field<P, KXM><<<(unsigned)blocks, kRowThreads, G::SMEM, s>>>(f, out, nrows, bg)));
  return cudaGetLastError();
}

// The inverse x pass from a kx-major half spectrum [block][k][z][y] (the
// plane engine's layout) to real rows [block][z][y][2N], as
// k_rows_c2r_reg: each lane loads its row's bins straight into registers;
// the 32/T rows of a warp are consecutive rows y of one plane (32/T divides
// Y), so a warp load of one register reads a run of 32/T points of each of
// T bins (whole 32-byte sectors).
template <class P>
__global__ void __launch_bounds__(kRowThreads) k_rows_c2r_kxm(const float2* __restrict__ in, float* __restrict__ out,
                                                               long long nrows, int Z, int Y, float scale, RowBg bg) {
  using G = RowRegGeom<P>;
  constexpr int N = G::N, T = G::T, E = G::E, RPC = G::RPC;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* tw2 = sm + P::TW;
  const int t = threadIdx.x % T, r = threadIdx.x / T;
  float2* S = sm + P::TW + 2 * N + r * P::SLICE;
  const long long row = (long long)blockIdx.x * RPC + r;
  const bool live0 = row < nrows;
  long long rr = live0 ? row : nrows - 1;
  const bool inside = WO_IN(rr, nrows, 7);
  if (!inside) rr = 0;
  const bool live = live0 && inside;
  const long long plane_rows = (long long)Z * Y;
  const long long blk = rr / plane_rows, rem = rr - blk * plane_rows;  // rem = z Y + y
  const long long kstep = plane_rows;                                     // bin k of the row at src + k Z Y
  const long long sb = blk * (N + 1) * plane_rows + rem;
  const float2* src = in + sb;
  float2 x[E];
#pragma unroll
  for (int m = 0; m < E; ++m)
    x[m] = WO_IN(sb + (t + T * m) * kstep, nrows * (N + 1), 7) ? __ldg(src + (t + T * m) * kstep)
                                                                : make_float2(0.f, 0.f);
  const float2 xn = (t == 0 && WO_IN(sb + N * kstep, nrows * (N + 1), 7)) ? __ldg(src + N * kstep)
                                                                           : make_float2(0.f, 0.f);  // X[N]
  P::twiddles(tw);  // while the row's loads are in flight
  make_twiddles<2 * N>(tw2);
  __syncthreads();
  float2 v[E];
  c2r_merge<T, E>(x, xn, tw2, t, v);
  P::template fft<true>(v, tw, S, t);
  if (!live) return;
  const float cst = bg.mode == 1 ? bg.v[((bg.row_offset + rr) / bg.rows_per_block) % bg.nchan] : 0.f;
  float2* o = reinterpret_cast<float2*>(out + rr * (2LL * N)) + t;
#pragma unroll
  for (int m = 0; m < E; ++m) o[T * m] = make_float2(v[m].x * scale + cst, v[m].y * scale + cst);
}

template <class P>
cudaError_t launch_c2r_kxm(const float2* in, float* out, long long nrows, int Z, int Y, float scale, RowBg bg,
                           cudaStream_t s) {
  using G = RowRegGeom<P>;
  const cudaError_t attr = allow_smem(k_rows_c2r_kxm<P>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  const long long blocks = (nrows + G::RPC - 1) / G::RPC;
  WO_LAUNCH("rows_c2r", s,
            (k_rows_c2r_kxm<P><<<(unsigned)blocks, kRowThreads, G::SMEM, s>>>(in, out, nrows, Z, Y, scale, bg)));
  return cudaGetLastError();
}

// The inverse x pass of a field's tiles fused with their blend (the tiles
// wo_reconstruct writes, stitched as wo_tile_blend stitches them): a CTA
// takes field row y of plane z of property p; the tile rows that cover it
// (row u of the one or two tile rows ty, every tx) are transformed back (T
// lanes each, as k_rows_c2r_reg), scaled, parked in shared memory, and
// blended with k_blend's weights, order and arithmetic, so the field equals
// the one from the tiles bit for bit.  spec: the half spectra after the
// inverse y pass, [tile][P][Z][2N][N+1].
template <class P>
__global__ void __launch_bounds__(kRowThreads) k_rows_c2r_blend(const float2* __restrict__ spec, FieldDst f,
                                                                 float scale, int vec) {
  using G = RowRegGeom<P>;
  constexpr int N = G::N, T = G::T, E = G::E, RPC = G::RPC, W = 2 * N, XH = N + 1;
  // parked row pitch: the rows of a half-warp's pair stores start on distinct bank pairs
  constexpr int RS = W + 8;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* tw2 = sm + P::TW;
  float* vals = reinterpret_cast<float*>(sm + P::TW + 2 * N + RPC * P::SLICE);  // [2][tiles_x][RS]
  const int t = threadIdx.x % T, r = threadIdx.x / T;
  float2* S = sm + P::TW + 2 * N + r * P::SLICE;
  const int core = f.core, halo = f.halo;
  const int Yf = f.tiles_y * core, Xf = f.tiles_x * core;
  const long long frow = blockIdx.x;  // (p Z + z) Yf + y
  const int y = (int)(frow % Yf);
  const long long pz = frow / Yf;
  const int z = (int)(pz % f.Z), p = (int)(pz / f.Z);
  int tys[2] = {0, 0}, us[2] = {0, 0};
  float wys[2] = {0.f, 0.f};
  int ny = 0;
  const int qy = (y + halo) / core;
  for (int c = qy - 1; c <= qy; ++c) {
    if (c < 0 || c >= f.tiles_y) continue;
    const int u = y - (c * core - halo);
    if (u < 0 || u >= W) continue;
    tys[ny] = c;
    us[ny] = u;
    wys[ny] = ramp(u, W, halo);
    ++ny;
  }
  P::twiddles(tw);
  make_twiddles<2 * N>(tw2);
  __syncthreads();
  const int nrow = ny * f.tiles_x;
  for (int i0 = 0; i0 < nrow; i0 += RPC) {  // uniform across the CTA
    const int i = i0 + r;
    const bool live = i < nrow;
    const int a = live ? i / f.tiles_x : 0, b = live ? i - (i / f.tiles_x) * f.tiles_x : 0;
    const long long tile = (long long)tys[a] * f.tiles_x + b;
    const long long srow = ((tile * f.P + p) * f.Z + z) * (long long)W + us[a];
    const bool ok = live && WO_IN(srow, (long long)f.tiles_y * f.tiles_x * f.P * f.Z * W, 7);
    const float2* src = spec + (ok ? srow : 0) * XH;
    float2 x[E];
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = __ldg(src + t + T * m);
    const float2 xn = t == 0 ? __ldg(src + N) : make_float2(0.f, 0.f);  // X[N], partner of X[0]
    float2 v[E];
    c2r_merge<T, E>(x, xn, tw2, t, v);
    P::template fft<true>(v, tw, S, t);
    if (ok) {
      float2* dst = reinterpret_cast<float2*>(vals + (a * f.tiles_x + b) * RS) + t;
      const float cst = 0.f;  // (as the reconstruction's inverse x pass: no background added)
#pragma unroll
      for (int m = 0; m < E; ++m) dst[T * m] = make_float2(v[m].x * scale + cst, v[m].y * scale + cst);
    }
  }
  __syncthreads();
  float* out = f.field + frow * (long long)Xf;
  const int nvec = vec ? Xf / 4 : Xf;
  for (int q = threadIdx.x; q < nvec; q += kRowThreads) {
    const int x0 = vec ? 4 * q : q;
    const int lanes = vec ? 4 : 1;
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, wsum[4] = {0.f, 0.f, 0.f, 0.f};
    const int qx = (x0 + halo) / core;
    for (int c = qx - 1; c <= qx; ++c) {
      if (c < 0 || c >= f.tiles_x) continue;
      const int v = x0 - (c * core - halo);
      if (v < 0 || v >= W) continue;  // vec: v .. v+3 lie in the same tile
      for (int a = 0; a < ny; ++a) {
        const float* src = vals + (a * f.tiles_x + c) * RS + v;
        for (int k = 0; k < lanes; ++k) {
          const float wgt = wys[a] * ramp(v + k, W, halo);
          acc[k] += wgt * src[k];
          wsum[k] += wgt;
        }
      }
    }
    if (!WO_IN(frow * (long long)Xf + x0 + lanes - 1, (long long)gridDim.x * Xf, 7)) continue;
    if (vec) {
      *reinterpret_cast<float4*>(out + x0) =
          make_float4(acc[0] / wsum[0], acc[1] / wsum[1], acc[2] / wsum[2], acc[3] / wsum[3]);
    } else {
      out[x0] = acc[0] / wsum[0];
    }
  }
}

template <class P>
cudaError_t launch_c2r_blend(const float2* spec, const FieldDst& f, float scale, cudaStream_t s) {
  using G = RowRegGeom<P>;
  const size_t smem = G::SMEM + (size_t)2 * f.tiles_x * (2 * G::N + 8) * sizeof(float);
  const cudaError_t attr = allow_smem(k_rows_c2r_blend<P>, smem);
  if (attr != cudaSuccess) return attr;
  const int vec = (f.core % 4 == 0 && f.halo % 4 == 0) ? 1 : 0;
  const long long rows = (long long)f.P * f.Z * f.tiles_y * f.core;
  WO_LAUNCH("rows_c2r", s, (k_rows_c2r_blend<P><<<(unsigned)rows, kRowThreads, smem, s>>>(spec, f, scale, vec)));
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_r2c_reg(const float* in, float2* out, long long nrows, RowBg bg, cudaStream_t s) {
  using G = RowRegGeom<P>;
  const cudaError_t attr = allow_smem(k_rows_r2c_reg<P>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  const long long blocks = (nrows + G::RPC - 1) / G::RPC;
  WO_LAUNCH("rows_r2c", s, (k_rows_r2c_reg<P><<<(unsigned)blocks, kRowThreads, G::SMEM, s>>>(in, out, nrows, bg, 1)));
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_c2r_reg(const float2* in, float* out, long long nrows, float scale, RowBg bg, cudaStream_t s) {
  using G = RowRegGeom<P>;
  const cudaError_t attr = allow_smem(k_rows_c2r_reg<P>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  const long long blocks = (nrows + G::RPC - 1) / G::RPC;
  WO_LAUNCH("rows_c2r", s,
            (k_rows_c2r_reg<P><<<(unsigned)blocks, kRowThreads, G::SMEM, s>>>(in, out, nrows, scale, bg)));
  return cudaGetLastError();
}

}  // namespace

bool rows_reg_supported(int N) {
  return N == 32 || N == 48 || N == 64 || N == 96 || N == 128 || N == 192 || N == 256 || N == 512;
}

cudaError_t rows_r2c_reg(int N, const float* in, float2* out, long long nrows, RowBg bg, cudaStream_t s) {
  switch (N) {
    case 32: return launch_r2c_reg<Row2<32, 8>>(in, out, nrows, bg, s);
    case 48: return launch_r2c_reg<Row2<48, 12>>(in, out, nrows, bg, s);
    case 64: return launch_r2c_reg<Row2<64, 8>>(in, out, nrows, bg, s);
    case 96: return launch_r2c_reg<Row2<96, 24>>(in, out, nrows, bg, s);
    case 128: return launch_r2c_reg<Row2<128, 16>>(in, out, nrows, bg, s);
    case 192: return launch_r2c_reg<Row2<192, 24>>(in, out, nrows, bg, s);
    case 256: return launch_r2c_reg<Row2<256, 16>>(in, out, nrows, bg, s);
    case 512: return launch_r2c_reg<Row512>(in, out, nrows, bg, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t rows_r2c_field(int N, const FieldSrc& f, float2* out, long long nrows, RowBg bg, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  switch (N) {
    case 32: return launch_r2c_field<Row2<32, 8>, false>(f, out, nrows, bg, s);
    case 48: return launch_r2c_field<Row2<48, 12>, false>(f, out, nrows, bg, s);
    case 64: return launch_r2c_field<Row2<64, 8>, false>(f, out, nrows, bg, s);
    case 96: return launch_r2c_field<Row2<96, 24>, false>(f, out, nrows, bg, s);
    case 128: return launch_r2c_field<Row2<128, 16>, false>(f, out, nrows, bg, s);
    case 192: return launch_r2c_field<Row2<192, 24>, false>(f, out, nrows, bg, s);
    case 256: return launch_r2c_field<Row2<256, 16>, false>(f, out, nrows, bg, s);
    case 512: return launch_r2c_field<Row512, false>(f, out, nrows, bg, s);
    default: return cudaErrorInvalidValue;
  }
}

bool rows_kxm_supported(int N, int Y) {
  const int rpw = N == 64 ? 32 / 8 : 32 / 4;  // rows per warp of the N-point row transform (8 or 4 lanes per row)
  return (N == 32 || N == 64 || N == 96) && Y % rpw == 0;
}

cudaError_t rows_r2c_field_kxm(int N, const FieldSrc& f, float2* out, long long nrows, RowBg bg, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  if (!rows_kxm_supported(N, 2 * N)) return cudaErrorInvalidValue;
  switch (N) {
    case 32: return launch_r2c_field<Row2<32, 8>, true>(f, out, nrows, bg, s);
    case 64: return launch_r2c_field<Row2<64, 8>, true>(f, out, nrows, bg, s);
    case 96: return launch_r2c_field<Row2<96, 24>, true>(f, out, nrows, bg, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t rows_r2c_kxm(int N, const float* in, float2* out, long long nrows, int Z, int Y, RowBg bg,
                         cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  if (!rows_kxm_supported(N, Y) || Y != 2 * N || nrows % ((long long)Z * Y)) return cudaErrorInvalidValue;
  switch (N) {  // square planes: Y = 2N
    case 32: return launch_r2c_kxm<Row2<32, 8>, 64>(in, out, nrows, Z, bg, s);
    case 64: return launch_r2c_kxm<Row2<64, 8>, 128>(in, out, nrows, Z, bg, s);
    case 96: return launch_r2c_kxm<Row2<96, 24>, 192>(in, out, nrows, Z, bg, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t rows_c2r_kxm(int N, const float2* in, float* out, long long nrows, int Z, int Y, float scale, RowBg bg,
                         cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  if (!rows_kxm_supported(N, Y) || nrows % ((long long)Z * Y)) return cudaErrorInvalidValue;  // whole planes
  switch (N) {
    case 32: return launch_c2r_kxm<Row2<32, 8>>(in, out, nrows, Z, Y, scale, bg, s);
    case 64: return launch_c2r_kxm<Row2<64, 8>>(in, out, nrows, Z, Y, scale, bg, s);
    case 96: return launch_c2r_kxm<Row2<96, 24>>(in, out, nrows, Z, Y, scale, bg, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t rows_c2r_blend(int N, const float2* spec, const FieldDst& f, float scale, cudaStream_t s) {
  if (f.tiles_x > 64) return cudaErrorInvalidValue;  // the parked rows must fit shared memory
  switch (N) {
    case 32: return launch_c2r_blend<Row2<32, 8>>(spec, f, scale, s);
    case 48: return launch_c2r_blend<Row2<48, 12>>(spec, f, scale, s);
    case 64: return launch_c2r_blend<Row2<64, 8>>(spec, f, scale, s);
    case 96: return launch_c2r_blend<Row2<96, 24>>(spec, f, scale, s);
    case 128: return launch_c2r_blend<Row2<128, 16>>(spec, f, scale, s);
    case 192: return launch_c2r_blend<Row2<192, 24>>(spec, f, scale, s);
    case 256: return launch_c2r_blend<Row2<256, 16>>(spec, f, scale, s);
    case 512: return launch_c2r_blend<Row512>(spec, f, scale, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t rows_c2r_reg(int N, const float2* in, float* out, long long nrows, float scale, RowBg bg,
                         cudaStream_t s) {
  switch (N) {
    case 32: return launch_c2r_reg<Row2<32, 8>>(in, out, nrows, scale, bg, s);
    case 48: return launch_c2r_reg<Row2<48, 12>>(in, out, nrows, scale, bg, s);
    case 64: return launch_c2r_reg<Row2<64, 8>>(in, out, nrows, scale, bg, s);
    case 96: return launch_c2r_reg<Row2<96, 24>>(in, out, nrows, scale, bg, s);
    case 128: return launch_c2r_reg<Row2<128, 16>>(in, out, nrows, scale, bg, s);
    case 192: return launch_c2r_reg<Row2<192, 24>>(in, out, nrows, scale, bg, s);
    case 256: return launch_c2r_reg<Row2<256, 16>>(in, out, nrows, scale, bg, s);
    case 512: return launch_c2r_reg<Row512>(in, out, nrows, scale, bg, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wo

// wo_xy.cu - the x and y transforms of a plane in one kernel: a cluster of
// two CTAs per plane, which exchange the plane's half spectrum through
// distributed shared memory.
//
// Forward (real plane -> half spectrum, the passes rows_r2c + y_fwd): CTA
// rank r transforms rows [r Y/2, (r+1) Y/2) along x (real row -> N+1 bins,
// the register-resident row transforms and split of wo_rowsplit.cuh) and
// writes bin k of each row into the tile of the CTA that owns column k
// (rank 0 the columns k < K0, rank 1 the others), its own or its partner's.
// After a cluster barrier each CTA transforms its columns along y in its
// tile (T lanes of a warp per column, in registers) and stores them in
// whole row segments.
//
// Inverse (half spectrum -> real plane, y_inv + rows_c2r): each CTA loads
// its columns, transforms them back along y, and after a cluster barrier
// transforms its rows back along x, reading each row's bins from both
// tiles; a second cluster barrier keeps each tile alive until the partner
// has read it.
//
// One plane's half spectrum is read and written once instead of twice
// (the passes' intermediate trip through memory is gone).  No CTA leaves
// before the cluster barriers: a failed index check (WO_CHECK builds) only
// disables the plane's global accesses.
#include <stdint.h>

#include "wo_fft.cuh"
#include "wo_internal.h"
#include "wo_regfft.cuh"
#include "wo_rowsplit.cuh"

namespace wo {

namespace {

constexpr int kXyThreads = 128;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// The address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_cluster(uint32_t a, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}

__device__ __forceinline__ float2 ld_cluster(uint32_t a) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}

// Every thread of both CTAs: writes before it (to either CTA's shared
// memory) are seen by reads after it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// PX: the complex row transform of H = X/2 points; PY: the column transform
// of Y points.
template <class PX, class PY>
struct XyGeom {
  static constexpr int H = PX::N, X = 2 * H, XH = H + 1, Y = PY::N;
  static constexpr int TX = PX::T, EX = PX::E, TY = PY::T, EY = PY::E;
  static constexpr int NT = kXyThreads;
  static constexpr int K0 = (XH + 1) / 2;        // columns of rank 0 (rank 1: XH - K0)
  // tile pitch: the smallest >= K0 that is 2 mod 16, so that a half-warp's
  // column reads (8 lanes x 2 columns) hit distinct 8-byte bank pairs
  static constexpr int PITCH = (K0 - 2 + 15) / 16 * 16 + 2;
  static constexpr int RX = NT / TX, CY = NT / TY;  // rows / columns per round
  static constexpr int SCR = (RX * PX::SLICE > CY * PY::SLICE) ? RX * PX::SLICE : CY * PY::SLICE;
  // twiddles of both transforms, e^{-2 pi i k / X}, the transposes' scratch, the tile [Y][PITCH]
  static constexpr size_t SMEM =
      ((size_t)PX::TW + (size_t)PY::TW + (size_t)X + (size_t)SCR + (size_t)Y * PITCH) * sizeof(float2);
  static_assert(Y % 2 == 0, "each CTA takes half of the rows");
};

template <class PX, class PY>
__device__ __forceinline__ void xy_setup(float2* sm, float2*& twx, float2*& twy, float2*& tw2, float2*& scr,
                                         float2*& tile) {
  using G = XyGeom<PX, PY>;
  twx = sm;
  twy = twx + PX::TW;
  tw2 = twy + PY::TW;
  scr = tw2 + G::X;
  tile = scr + G::SCR;
  PX::twiddles(twx);
  PY::twiddles(twy);
  make_twiddles<G::X>(tw2);
}

// Column transforms (along y) of this CTA's ncols columns, in place in the tile.
template <class PX, class PY, bool INV>
__device__ __forceinline__ void xy_columns(float2* tile, const float2* twy, float2* scr, int ncols) {
  using G = XyGeom<PX, PY>;
  constexpr int TY = G::TY, EY = G::EY, CY = G::CY, PITCH = G::PITCH;
  const int l = threadIdx.x % TY, cc = threadIdx.x / TY;
  for (int c0 = 0; c0 < ncols; c0 += CY) {
    const int c = c0 + cc;
    const bool cv = c < ncols;  // lanes past the last column transform zeros and write nothing
    float2 v[EY];
#pragma unroll
    for (int m = 0; m < EY; ++m) v[m] = cv ? tile[(l + TY * m) * PITCH + c] : make_float2(0.f, 0.f);
    PY::template fft<INV>(v, twy, scr + cc * PY::SLICE, l);
    if (cv) {
#pragma unroll
      for (int m = 0; m < EY; ++m) tile[(l + TY * m) * PITCH + c] = v[m];
    }
  }
}

template <class PX, class PY>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kXyThreads)
    k_xy_fwd(const float* __restrict__ in, float2* __restrict__ out, long long nplanes, long long plane0, RowBg bg) {
  using G = XyGeom<PX, PY>;
  constexpr int H = G::H, X = G::X, XH = G::XH, Y = G::Y, TX = G::TX, EX = G::EX, RX = G::RX, K0 = G::K0,
                PITCH = G::PITCH;
  extern __shared__ float2 sm[];
  float2 *twx, *twy, *tw2, *scr, *tile;
  xy_setup<PX, PY>(sm, twx, twy, tw2, scr, tile);
  const uint32_t rank = cluster_rank();
  const long long plane = plane0 + blockIdx.y + (long long)gridDim.y * blockIdx.z;
  const bool ok = plane < nplanes && WO_IN(plane, nplanes, 10);  // else: barriers only
  const uint32_t tile0 = cluster_addr(smem_addr(tile), 0), tile1 = cluster_addr(smem_addr(tile), 1);
  __syncthreads();  // the twiddles
  // x: this CTA's rows; bin k of row y goes to tile (k < K0 ? 0 : 1) at [y][k - k0].
  // A round's row loads are issued during the previous round's transform.
  const int t = threadIdx.x % TX, rr = threadIdx.x / TX;
  float2 nxt[EX];
  float cn = 0.f;
  auto load_row = [&](int r0) {
    const int y = (int)rank * (Y / 2) + r0 + rr;
    const bool rv = ok && r0 + rr < Y / 2;
    const long long row = plane * Y + (rv ? y : 0);
    cn = rv ? row_constant(in, row, X, bg) : 0.f;
    const float2* src = reinterpret_cast<const float2*>(in + row * X) + t;
#pragma unroll
    for (int m = 0; m < EX; ++m) nxt[m] = rv ? __ldg(src + TX * m) : make_float2(0.f, 0.f);
  };
  load_row(0);
  for (int r0 = 0; r0 < Y / 2; r0 += RX) {
    const int y = (int)rank * (Y / 2) + r0 + rr;
    const bool rv = ok && r0 + rr < Y / 2;
    float2 v[EX];
#pragma unroll
    for (int m = 0; m < EX; ++m) v[m] = make_float2(nxt[m].x - cn, nxt[m].y - cn);
    if (r0 + RX < Y / 2) load_row(r0 + RX);
    PX::template fft<false>(v, twx, scr + rr * PX::SLICE, t);
    r2c_split<H, TX, EX>(v, tw2, t, [&](int k, float2 val) {
      if (rv) st_cluster((k < K0 ? tile0 + (uint32_t)(y * PITCH + k) * 8u
                                 : tile1 + (uint32_t)(y * PITCH + k - K0) * 8u), val);
    });
  }
  cluster_sync();  // every bin in its tile
  const int ncols = rank == 0 ? K0 : XH - K0, k0 = rank == 0 ? 0 : K0;
  xy_columns<PX, PY, false>(tile, twy, scr, ncols);
  __syncthreads();
  if (ok) {  // whole row segments: warp w takes rows w, w + NT/32, ...
    float2* o = out + plane * (long long)Y * XH + k0;
    const int lane = threadIdx.x & 31;
    for (int y = threadIdx.x >> 5; y < Y; y += G::NT / 32)
      for (int c = lane; c < ncols; c += 32) o[(long long)y * XH + c] = tile[y * PITCH + c];
  }
}

template <class PX, class PY>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kXyThreads)
    k_xy_inv(const float2* __restrict__ in, float* __restrict__ out, long long nplanes, long long plane0, float scale,
             RowBg bg) {
  using G = XyGeom<PX, PY>;
  constexpr int H = G::H, X = G::X, XH = G::XH, Y = G::Y, TX = G::TX, EX = G::EX, RX = G::RX, K0 = G::K0,
                PITCH = G::PITCH;
  extern __shared__ float2 sm[];
  float2 *twx, *twy, *tw2, *scr, *tile;
  xy_setup<PX, PY>(sm, twx, twy, tw2, scr, tile);
  const uint32_t rank = cluster_rank();
  const long long plane = plane0 + blockIdx.y + (long long)gridDim.y * blockIdx.z;
  const bool ok = plane < nplanes && WO_IN(plane, nplanes, 10);  // else: barriers only
  const int ncols = rank == 0 ? K0 : XH - K0, k0 = rank == 0 ? 0 : K0;
  {  // this CTA's columns, in whole row segments (warp w: rows w, w + NT/32, ...), copied
     // asynchronously so that every copy of the tile is in flight at once
    const float2* src = in + plane * (long long)Y * XH + k0;
    const int lane = threadIdx.x & 31;
    for (int y = threadIdx.x >> 5; y < Y; y += G::NT / 32)
      for (int c = lane; c < ncols; c += 32) cp_async8(tile + y * PITCH + c, ok ? src + (long long)y * XH + c : src, ok);
    cp_async_wait_all();
  }
  __syncthreads();  // the tile and the twiddles
  xy_columns<PX, PY, true>(tile, twy, scr, ncols);
  const uint32_t tile0 = cluster_addr(smem_addr(tile), 0), tile1 = cluster_addr(smem_addr(tile), 1);
  cluster_sync();  // both tiles transformed
  // x: this CTA's rows, each row's bins read from both tiles; a round's bins
  // are read during the previous round's transform
  const int t = threadIdx.x % TX, rr = threadIdx.x / TX;
  float2 x[EX], xn;
  auto read_row = [&](int r0) {
    const bool rv = ok && r0 + rr < Y / 2;
    const int ys = rv ? (int)rank * (Y / 2) + r0 + rr : 0;
#pragma unroll
    for (int m = 0; m < EX; ++m) {
      const int k = t + TX * m;
      x[m] = ld_cluster(k < K0 ? tile0 + (uint32_t)(ys * PITCH + k) * 8u : tile1 + (uint32_t)(ys * PITCH + k - K0) * 8u);
    }
    xn = t == 0 ? ld_cluster(tile1 + (uint32_t)(ys * PITCH + H - K0) * 8u) : make_float2(0.f, 0.f);
  };
  read_row(0);
  for (int r0 = 0; r0 < Y / 2; r0 += RX) {
    const int y = (int)rank * (Y / 2) + r0 + rr;
    const bool rv = ok && r0 + rr < Y / 2;
    float2 v[EX];
    c2r_merge<TX, EX>(x, xn, tw2, t, v);
    if (r0 + RX < Y / 2) read_row(r0 + RX);
    PX::template fft<true>(v, twx, scr + rr * PX::SLICE, t);
    if (rv) {
      const long long row = plane * Y + y;
      const float cst = bg.mode == 1 ? bg.v[((bg.row_offset + row) / bg.rows_per_block) % bg.nchan] : 0.f;
      float2* o = reinterpret_cast<float2*>(out + row * X) + t;
#pragma unroll
      for (int m = 0; m < EX; ++m) o[TX * m] = make_float2(v[m].x * scale + cst, v[m].y * scale + cst);
    }
  }
  cluster_sync();  // the partner has read this tile
}

template <class PX, class PY>
cudaError_t launch_xy(bool inv, const void* in, void* out, long long nplanes, float scale, RowBg bg, cudaStream_t s) {
  using G = XyGeom<PX, PY>;
  const cudaError_t a0 = allow_smem(k_xy_fwd<PX, PY>, G::SMEM);
  const cudaError_t a1 = allow_smem(k_xy_inv<PX, PY>, G::SMEM);
  if (a0 != cudaSuccess) return a0;
  if (a1 != cudaSuccess) return a1;
  // planes in launches of at most 65535 x 65535 (grid y, z)
  const long long per = 65535LL * 65535LL;
  for (long long p0 = 0; p0 < nplanes; p0 += per) {
    const long long n = nplanes - p0 < per ? nplanes - p0 : per;
    const long long gy = n < 65535 ? n : 65535;
    dim3 grid(2, (unsigned)gy, (unsigned)((n + gy - 1) / gy));
    if (inv) {
      WO_LAUNCH("xy_inv", s, (k_xy_inv<PX, PY><<<grid, G::NT, G::SMEM, s>>>((const float2*)in, (float*)out,
                                                                          p0 + n, p0, scale, bg)));
    } else {
      WO_LAUNCH("xy_fwd", s, (k_xy_fwd<PX, PY><<<grid, G::NT, G::SMEM, s>>>((const float*)in, (float2*)out,
                                                                          p0 + n, p0, bg)));
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t xy_dispatch(bool inv, int X, int Y, const void* in, void* out, long long nplanes, float scale, RowBg bg,
                        cudaStream_t s) {
  if (X == 192 && Y == 192) return launch_xy<Row2<96, 24>, Row2<192, 24>>(inv, in, out, nplanes, scale, bg, s);
  if (X == 128 && Y == 128) return launch_xy<Row2<64, 8>, Row2<128, 16>>(inv, in, out, nplanes, scale, bg, s);
  if (X == 64 && Y == 64) return launch_xy<Row2<32, 8>, Row2<64, 8>>(inv, in, out, nplanes, scale, bg, s);
  return cudaErrorNotSupported;
}

}  // namespace

bool xy_supported(int X, int Y) {
  return (X == 192 && Y == 192) || (X == 128 && Y == 128) || (X == 64 && Y == 64);
}

cudaError_t xy_fwd(int X, int Y, const float* in, float2* out, long long nplanes, RowBg bg, cudaStream_t s) {
  if (nplanes <= 0) return cudaSuccess;
  return xy_dispatch(false, X, Y, in, out, nplanes, 1.f, bg, s);
}

cudaError_t xy_inv(int X, int Y, const float2* in, float* out, long long nplanes, float scale, RowBg bg,
                   cudaStream_t s) {
  if (nplanes <= 0) return cudaSuccess;
  return xy_dispatch(true, X, Y, in, out, nplanes, scale, bg, s);
}

// The x and y transforms of nplanes planes: the fused kernel where the
// schedule table says so, else the row pass and the column pass.
cudaError_t plane_xy_fwd(int X, int Y, const float* in, float2* out, long long nplanes, RowBg bg, cudaStream_t s) {
  if (xy_engine(X, Y) == WO_ENGINE_HYBRID) return xy_fwd(X, Y, in, out, nplanes, bg, s);
  const int Xh = X / 2 + 1;
  const cudaError_t e = rows_r2c(X / 2, in, out, nplanes * Y, bg, s);
  if (e != cudaSuccess) return e;
  return cols_c2c(Y, false, out, Xh, (long long)Y * Xh, Xh, nplanes, s, "y_fwd");
}

// The inverse; the separate passes work in place on `in`.
cudaError_t plane_xy_inv(int X, int Y, float2* in, float* out, long long nplanes, float scale, RowBg bg,
                         cudaStream_t s) {
  if (xy_engine(X, Y) == WO_ENGINE_HYBRID) return xy_inv(X, Y, in, out, nplanes, scale, bg, s);
  const int Xh = X / 2 + 1;
  const cudaError_t e = cols_c2c(Y, true, in, Xh, (long long)Y * Xh, Xh, nplanes, s, "y_inv");
  if (e != cudaSuccess) return e;
  return rows_c2r(X / 2, in, out, nplanes * Y, scale, bg, s);
}

}  // namespace wo

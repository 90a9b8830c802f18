// wo_plane.cu - the y and z transforms of a kx-major half spectrum, one
// (tile, k_x) plane per CTA: the plane engine of one-volume operators and of
// one-kind TF banks built with WO_TF_KX_MAJOR.
//
// A kx-major half spectrum is laid out [tile][k_x][z][y] (complex): the Z x Y
// plane of every half-spectrum column k_x is contiguous.  The x passes that
// produce and consume it transpose through shared memory (wo_rowsreg.cu,
// wo_psf.cu).  A CTA here brings its whole plane into shared memory with TMA
// bulk copies, transforms the rows along y and the columns along z in
// registers (the four-step transforms of wo_regfft.cuh: T lanes per row or
// column, point t + T m in register m) and writes the plane back, so the
// y pass, the z pass with the operator between its transforms, and the
// inverse y pass cross HBM once instead of three times.
//
//   k_tf_yz   TF build: forward y and z transforms of a TF plane in place,
//             plus the regulariser maxima (as k_tf_zpass_reg);
//   k_yz_op   forward y and z transforms, the per-frequency operator of
//             k_z_reg (forward, adjoint, Tikhonov inverse), inverse z and y
//             transforms; planes and z columns outside the tile's TF support
//             disk are written as zeros without being transformed.
//
// The plane in shared memory: row z (Y points) at offset z Y, the points of
// an odd row rotated by 8 (point y in cell (y + 8) mod Y), so that the two
// rows a half-warp touches in the y transforms, and the two z points of a
// half-warp's column lanes, fall on different halves of the banks.  An even
// row arrives as one bulk copy, an odd row as two; every row completes on
// its own mbarrier, so a row's y transform starts as soon as that row has
// landed.  Each transform's
// exchange runs in place in the cells of its own row or column: lane n2's
// value for k1 goes to index k1 T + (n2 xor (k1 mod T)), which keeps the
// exchange's writes and reads free of bank conflicts.
#include <stdint.h>

#include <type_traits>

#include "wo_bulk.cuh"
#include "wo_fft.cuh"
#include "wo_internal.h"
#include "wo_regfft.cuh"
#include "wo_zops.cuh"

namespace wo {

namespace {

constexpr int kRot = 8;  // rotation of the odd rows (points)

// The four-step transform of Row2<N, N1> (wo_regfft.cuh) with its exchange
// in the N cells cell(s), s in [0, N), of the sequence being transformed.
// twc[k1 T + t] = w_N^(t k1).  The caller synchronises the warp before it
// writes the cells again.
template <class P, bool INV, class Cell>
__device__ __forceinline__ void fft_cells(float2 (&v)[P::E], const float2* twc, int t, Cell cell) {
  constexpr int N = P::N, N1 = P::E, T = P::T, NI = N1 / T;
  static_assert((T & (T - 1)) == 0, "the exchange index needs a power-of-two lane count");
  reg_stages<N1, 1, INV, N / N1>(v, twc);
#pragma unroll
  for (int k1 = 1; k1 < N1; ++k1) {
    float2 w = twc[k1 * T + t];
    if (INV) w.y = -w.y;
    v[k1] = cmul(v[k1], w);
  }
  __syncwarp();  // every lane has read the cells it loaded from
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) *cell(k1 * T + (t ^ (k1 & (T - 1)))) = v[k1];
  __syncwarp();
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    float2 u[T];
#pragma unroll
    for (int n2 = 0; n2 < T; ++n2) u[n2] = *cell((t + T * i) * T + (n2 ^ t));
    reg_stages<T, 1, INV, N / T>(u, twc);
#pragma unroll
    for (int k2 = 0; k2 < T; ++k2) v[i + NI * k2] = u[k2];
  }
}

// w_N^(t k1) at [k1 T + t] for the transform P.
template <class P>
__device__ __forceinline__ void cell_twiddles(float2* twc) {
  for (int e = threadIdx.x; e < P::N; e += blockDim.x) {
    const int k1 = e / P::T, t = e - (e / P::T) * P::T;
    float s, c;
    sincospif(2.0f * (float)(t * k1) / (float)P::N, &s, &c);
    twc[e] = make_float2(c, -s);
  }
}

template <class PY, class PZ, int NT_>
struct PlaneGeom {
  static constexpr int Y = PY::N, Z = PZ::N, NT = NT_;
  static constexpr int RPP = NT / PY::T;  // rows per y pass
  static constexpr int CW = 32 / PZ::T;   // z columns per warp
  static constexpr int CPP = NT / PZ::T;  // z columns per z pass
  static constexpr int PLANE = Z * Y;
  // plane, y twiddles, z twiddles, one mbarrier per row
  static constexpr size_t SMEM = (size_t)(PLANE + Y + Z) * sizeof(float2) + (size_t)Z * sizeof(uint64_t);
  // resident CTAs per SM by shared memory (228 KB per SM, 1 KB reserved per CTA, the static reduction array), at most 4
  static constexpr int FIT = (int)((228 * 1024) / (SMEM + 1024 + 64));
  static constexpr int MINB = FIT < 4 ? FIT : 4;
  static_assert(NT % 32 == 0 && Z % RPP == 0 && Y % CPP == 0, "whole passes of whole warps");
  static_assert(32 % PY::T == 0 && 32 % PZ::T == 0, "a row's or column's lanes sit in one warp");
  static_assert(Z % 2 == 0 && Y % 16 == 0 && Y > kRot, "row pairs; 16-byte rows; the odd-row rotation");
  static_assert(MINB >= 1, "the plane must fit shared memory");
  static_assert(Z <= NT, "a thread issues each row's copies");
};

// Cell of point s of row z (odd rows rotated).
template <int Y>
__device__ __forceinline__ int row_cell(int z, int s) {
  int q = s + ((z & 1) ? kRot : 0);
  return q >= Y ? q - Y : q;
}

// Threads 0 .. Z-1: copy plane `src` (Z rows of Y points) into P, odd rows
// rotated, row z completing on bars[z] (thread z initialises and arms the
// barrier of row z and issues its copies, so the rows' copies go out
// together).  The caller synchronises the CTA before any thread waits on a
// barrier.
template <int Z, int Y>
__device__ __forceinline__ void plane_copy_in(float2* P, const float2* src, uint64_t* bars) {
  const int z = threadIdx.x;
  if (z < Z) {
    mbar_init(bars + z, 1);
    mbar_init_fence();
    mbar_expect_tx(bars + z, (unsigned)(Y * sizeof(float2)));
    const float2* s = src + (long long)z * Y;
    float2* d = P + z * Y;
    if (z & 1) {
      bulk_load(d + kRot, s, (unsigned)((Y - kRot) * sizeof(float2)), bars + z);
      bulk_load(d, s + (Y - kRot), (unsigned)(kRot * sizeof(float2)), bars + z);
    } else {
      bulk_load(d, s, (unsigned)(Y * sizeof(float2)), bars + z);
    }
  }
}

// This thread's bounded wait for the copy of one row; false when it ran out.
__device__ __forceinline__ bool row_wait(uint64_t* bar) {
  if (mbar_try_wait(bar, 0u)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, 0u)) {
    if ((long long)(global_ns() - t0) > kPipeBudgetNs) return false;
  }
  return true;
}

// Every thread, after the forward y transforms: the result is the same in
// every thread of the CTA.  When a row's copy did not land within the
// budget, the first thread records WO_ERR_TIMEOUT (site, the plane's index)
// in the status block, and every thread waits once more, bounded, for every
// row, so that no copy lands after the CTA is gone.
template <int Z>
__device__ __forceinline__ bool plane_settle(bool ok, uint64_t* bars, int* status, int site, long long plane) {
  ok = __syncthreads_and(ok) != 0;
  if (!ok) {
    if (threadIdx.x == 0 && atomicCAS(status, 0, (int)WO_ERR_TIMEOUT) == 0) {
      status[1] = site;
      status[2] = (int)(plane > 2147483647LL ? 2147483647LL : plane);
    }
    const unsigned long long t1 = global_ns();
    for (int z = 0; z < Z; ++z)
      while (!mbar_try_wait(bars + z, 0u) && (long long)(global_ns() - t1) < kPipeBudgetNs) {
      }
  }
  return ok;
}

// The forward y transforms of every row of the plane in shared memory, in
// place, each row once its copy has landed (bars[z]); false when a wait ran
// out (the row is then transformed as it stands and the caller discards the
// plane).
template <class PY, class PZ, int NT>
__device__ __forceinline__ bool plane_rows_fwd(float2* P, const float2* twy, uint64_t* bars) {
  using G = PlaneGeom<PY, PZ, NT>;
  constexpr int Y = G::Y, T = PY::T, E = PY::E;
  const int t = threadIdx.x % T;
  bool ok = true;
#pragma unroll 1
  for (int z = threadIdx.x / T; z < G::Z; z += G::RPP) {
    ok = row_wait(bars + z) && ok;
    float2* row = P + z * Y;
    auto cell = [&](int s) { return row + row_cell<Y>(z, s); };
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = *cell(t + T * m);
    fft_cells<PY, false>(v, twy, t, cell);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < E; ++m) *cell(t + T * m) = v[m];
  }
  return ok;
}

// TF build: forward y and z transforms of TF plane (tile, k_x) in place and
// the tile's regulariser maxima.  Planes k_x >= x_cols are not launched;
// planes outside the tile's own support disk (every TF of the tile vanishes
// there: only the PSF rows' rounding noise) are left as they are, as the
// operators never read them (k_yz_op writes zeros there).
template <class PY, class PZ, int NT>
__global__ void __launch_bounds__(NT, PlaneGeom<PY, PZ, NT>::MINB) k_tf_yz(float2* __restrict__ tf,
                                                                          float* __restrict__ stats, int Xh, int lf,
                                                                          int* __restrict__ status) {
  using G = PlaneGeom<PY, PZ, NT>;
  constexpr int Y = G::Y, Z = G::Z, TZ = PZ::T, EZ = PZ::E, CW = G::CW;
  extern __shared__ __align__(16) float2 sm[];
  float2* P = sm;
  float2* twy = sm + G::PLANE;
  float2* twz = twy + Y;
  uint64_t* bars = reinterpret_cast<uint64_t*>(twz + Z);
  __shared__ float red[2 * (NT / 32)];
  const int kx = blockIdx.x, tile = blockIdx.y;
  const long long pidx = (long long)tile * Xh + kx;
  float2* plane = tf + pidx * G::PLANE;
#if defined(WO_CHECK) && WO_CHECK
  if (!WO_IN((pidx + 1) * G::PLANE - 1, (long long)gridDim.y * Xh * G::PLANE, 12)) return;  // uniform
#endif
  if (outside_support(stats + (long long)tile * 8, 0, Y, kx, 2 * (Xh - 1))) return;  // uniform
  plane_copy_in<Z, Y>(P, plane, bars);
  cell_twiddles<PY>(twy);
  cell_twiddles<PZ>(twz);
  __syncthreads();
  if (!plane_settle<Z>(plane_rows_fwd<PY, PZ, NT>(P, twy, bars), bars, status, 12, pidx)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = lane / CW, col = lane - (lane / CW) * CW;
  float m3 = 0.f, m2 = 0.f;
#pragma unroll 1
  for (int c0 = 0; c0 < Y; c0 += G::CPP) {
    const int c = c0 + warp * CW + col;
    auto cell = [&](int s) { return P + s * Y + row_cell<Y>(s, c); };
    float2 v[EZ];
#pragma unroll
    for (int m = 0; m < EZ; ++m) v[m] = *cell(t + TZ * m);
    fft_cells<PZ, false>(v, twz, t, cell);
    float cs = 0.f;
#pragma unroll
    for (int m = 0; m < EZ; ++m) {
      const float q = cabs2(v[m]);
      m3 = fmaxf(m3, q);
      cs += q;
      plane[(long long)(t + TZ * m) * Y + c] = v[m];
    }
    // the column's sum over its TZ lanes (lanes col + CW t), a fixed order
#pragma unroll
    for (int o = CW; o < 32; o <<= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
    m2 = fmaxf(m2, cs);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m3 = fmaxf(m3, __shfl_down_sync(0xffffffffu, m3, o));
    m2 = fmaxf(m2, __shfl_down_sync(0xffffffffu, m2, o));
  }
  if (lane == 0) {
    red[2 * warp] = m3;
    red[2 * warp + 1] = m2;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    float mx = 0.f;
    for (int q = 0; q < NT / 32; ++q) mx = fmaxf(mx, red[2 * q + threadIdx.x]);
    const int slot = (lf ? 0 : 2) + threadIdx.x;  // values >= 0: integer order is float order
    if (mx > 0.f) atomicMax(reinterpret_cast<int*>(stats + (long long)tile * 8) + slot, __float_as_int(mx));
  }
}

// Operator: plane (tile, k_x) of `in` through the y and z transforms, the
// per-frequency operator, and back, into the same plane of `out` (in == out
// allowed: the plane is read whole before anything is written).
template <class PY, class PZ, int NT>
__global__ void __launch_bounds__(NT, PlaneGeom<PY, PZ, NT>::MINB) k_yz_op(const float2* in, float2* out,
                                                                          const float2* __restrict__ tf, ZOp op,
                                                                          int Xh, int* __restrict__ status) {
  using G = PlaneGeom<PY, PZ, NT>;
  constexpr int Y = G::Y, Z = G::Z, TY = PY::T, EY = PY::E, TZ = PZ::T, EZ = PZ::E, CW = G::CW;
  extern __shared__ __align__(16) float2 sm[];
  float2* P = sm;
  float2* twy = sm + G::PLANE;
  float2* twz = twy + Y;
  uint64_t* bars = reinterpret_cast<uint64_t*>(twz + Z);
  const int kx = blockIdx.x, tile = blockIdx.y;
  const int tt = op.tf_shared ? 0 : tile;  // the tile whose TF and statistics apply
  const float* st = op.stats + (long long)tt * 8;
  const int X = 2 * (Xh - 1);
  const long long pidx = (long long)tile * Xh + kx;
  const float2* src = in + pidx * G::PLANE;
  float2* dst = out + pidx * G::PLANE;
  const float2* h = tf + ((long long)tt * Xh + kx) * G::PLANE;
#if defined(WO_CHECK) && WO_CHECK
  {
    const long long nt = gridDim.y, ntt = op.tf_shared ? 1 : nt;
    if (!WO_IN((pidx + 1) * G::PLANE - 1, nt * Xh * G::PLANE, 13) ||
        !WO_IN(((long long)tt * Xh + kx + 1) * G::PLANE - 1, ntt * Xh * G::PLANE, 13))
      return;  // uniform
  }
#endif
  if (outside_support(st, 0, Y, kx, X)) {  // the plane's nearest column is outside: all of it is
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int e = threadIdx.x; e < G::PLANE / 2; e += NT) d4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;  // uniform
  }
  plane_copy_in<Z, Y>(P, src, bars);
  // the TF plane is read in the z step: on its way to L2 meanwhile
  if (threadIdx.x < Z) bulk_prefetch_l2(h + (long long)threadIdx.x * Y, (unsigned)(Y * sizeof(float2)));
  const bool lf = op.lf_props > 0;
  const float eta = lf ? op.eta_lf : op.eta_fl;
  const float lam = op.eta_absolute ? eta : eta * st[lf ? 0 : 2];
  cell_twiddles<PY>(twy);
  cell_twiddles<PZ>(twz);
  __syncthreads();
  if (!plane_settle<Z>(plane_rows_fwd<PY, PZ, NT>(P, twy, bars), bars, status, 13, pidx)) return;
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = lane / CW, col = lane - (lane / CW) * CW;
#pragma unroll 1
    for (int c0 = 0; c0 < Y; c0 += G::CPP) {
      const int c = c0 + warp * CW + col;
      auto cell = [&](int s) { return P + s * Y + row_cell<Y>(s, c); };
      const bool inside = !outside_support(st, c, Y, kx, X);
      if (!__any_sync(0xffffffffu, inside)) {  // the warp's columns are all outside
#pragma unroll
        for (int m = 0; m < EZ; ++m) *cell(t + TZ * m) = make_float2(0.f, 0.f);
        continue;
      }
      float2 H[EZ], v[EZ];
#pragma unroll
      for (int m = 0; m < EZ; ++m) {
        H[m] = inside ? __ldg(h + (long long)(t + TZ * m) * Y + c) : make_float2(0.f, 0.f);
        v[m] = inside ? *cell(t + TZ * m) : make_float2(0.f, 0.f);
      }
      fft_cells<PZ, false>(v, twz, t, cell);
#pragma unroll
      for (int m = 0; m < EZ; ++m) {
        const float2 x = v[m], hv = H[m];
        if (op.op == 0) {
          v[m] = cmul(hv, x);
        } else if (op.op == 1) {
          v[m] = cmulc(hv, x);
        } else {
          const bool dc = op.zero_dc && t + TZ * m == 0 && c == 0 && kx == 0;
          const float den = lam + cabs2(hv);
          const float inv = den > 0.f ? 1.0f / den : 0.f;  // zero TF and eta: minimum norm
          v[m] = dc ? make_float2(0.f, 0.f) : cscale(cmulc(hv, x), inv);
        }
      }
      fft_cells<PZ, true>(v, twz, t, cell);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < EZ; ++m) *cell(t + TZ * m) = inside ? v[m] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  // inverse y transforms, each row stored from registers (a lane group's
  // store covers TY consecutive points: whole 32-byte sectors)
  const int t = threadIdx.x % TY;
#pragma unroll 1
  for (int z = threadIdx.x / TY; z < Z; z += G::RPP) {
    float2* row = P + z * Y;
    auto cell = [&](int s) { return row + row_cell<Y>(z, s); };
    float2 v[EY];
#pragma unroll
    for (int m = 0; m < EY; ++m) v[m] = *cell(t + TY * m);
    fft_cells<PY, true>(v, twy, t, cell);
    float2* o = dst + (long long)z * Y + t;
#pragma unroll
    for (int m = 0; m < EY; ++m) o[TY * m] = v[m];
  }
}

template <class PY, class PZ, int NT>
cudaError_t launch_tf_yz(const TfArgs& a, int* status, cudaStream_t s) {
  using G = PlaneGeom<PY, PZ, NT>;
  const cudaError_t attr = allow_smem(k_tf_yz<PY, PZ, NT>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  if (a.x_cols <= 0) return cudaSuccess;
  dim3 grid((unsigned)a.x_cols, (unsigned)a.n_tiles);
  WO_LAUNCH("tf_yz", s,
            (k_tf_yz<PY, PZ, NT><<<grid, NT, G::SMEM, s>>>(a.tf, a.stats, a.X / 2 + 1, a.lf_props > 0, status)));
  return cudaGetLastError();
}

template <class PY, class PZ, int NT>
cudaError_t launch_yz_op(float2* spec, const float2* tf, const ZOp& op, int n_tiles, int Xh, int* status,
                         cudaStream_t s) {
  using G = PlaneGeom<PY, PZ, NT>;
  const cudaError_t attr = allow_smem(k_yz_op<PY, PZ, NT>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  dim3 grid((unsigned)Xh, (unsigned)n_tiles);
  WO_LAUNCH("yz_op", s, (k_yz_op<PY, PZ, NT><<<grid, NT, G::SMEM, s>>>(spec, spec, tf, op, Xh, status)));
  return cudaGetLastError();
}

// The instantiated (Z, Y) shapes: Z 32 or 48 with Y 64, 128 or 192, and
// 16 x 64 (small stacks).
template <class F>
cudaError_t plane_dispatch(int Z, int Y, F f) {
  if (Z == 16 && Y == 64) return f(Row2<64, 8>{}, Row2<16, 4>{}, std::integral_constant<int, 128>{});
  if (Z == 48 && Y == 192) return f(Row2<192, 24>{}, Row2<48, 12>{}, std::integral_constant<int, 192>{});
  if (Z == 48 && Y == 128) return f(Row2<128, 16>{}, Row2<48, 12>{}, std::integral_constant<int, 128>{});
  if (Z == 48 && Y == 64) return f(Row2<64, 8>{}, Row2<48, 12>{}, std::integral_constant<int, 128>{});
  if (Z == 32 && Y == 192) return f(Row2<192, 24>{}, Row2<32, 8>{}, std::integral_constant<int, 128>{});
  if (Z == 32 && Y == 128) return f(Row2<128, 16>{}, Row2<32, 8>{}, std::integral_constant<int, 128>{});
  if (Z == 32 && Y == 64) return f(Row2<64, 8>{}, Row2<32, 8>{}, std::integral_constant<int, 128>{});
  return cudaErrorInvalidValue;
}

}  // namespace

bool plane_supported(int Z, int Y) {
  return ((Z == 32 || Z == 48) && (Y == 64 || Y == 128 || Y == 192)) || (Z == 16 && Y == 64);
}

cudaError_t tf_plane_yz(const TfArgs& a, int* status, cudaStream_t s) {
  if (a.n_kinds != 1) return cudaErrorInvalidValue;
  return plane_dispatch(a.Z, a.Y, [&](auto py, auto pz, auto nt) {
    return launch_tf_yz<decltype(py), decltype(pz), decltype(nt)::value>(a, status, s);
  });
}

cudaError_t plane_yz_op(int Z, int Y, float2* spec, const float2* tf, const ZOp& op, int n_tiles, int Xh,
                        int* status, cudaStream_t s) {
  if (op.n_in != 1 || op.n_out != 1 || op.n_tf != 1) return cudaErrorInvalidValue;
  return plane_dispatch(Z, Y, [&](auto py, auto pz, auto nt) {
    return launch_yz_op<decltype(py), decltype(pz), decltype(nt)::value>(spec, tf, op, n_tiles, Xh, status, s);
  });
}

}  // namespace wo

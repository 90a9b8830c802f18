// wo_zreg.cu - fused z pass with register-resident z transforms, for one
// volume in, one volume out and one transfer function (the one-property
// modes: phase or absorption or fluorescence alone).
//
// The same operation as k_z_fused (wo_zops.cuh) with NI = NO = 1: forward
// transform along z, the per-frequency operator
//   forward      D = H F,
//   adjoint      F = conj(H) D,
//   reconstruct  F = conj(H) D~ / (|H|^2 + eta)   (Eq. recon, one channel),
// inverse transform along z.  Here T lanes of one warp own a z column (lane
// l holds the points n = l + T m, the row transforms of wo_regfft.cuh run on
// a column) and a warp covers 32/T adjacent x columns: the column and its
// transfer function are loaded straight into registers (each warp load fills
// whole 32-byte sectors), the operator acts on the registers that the
// forward transform leaves (frequency k = l + T m in register m, the same
// ownership as the input), and the result is stored from them.  Columns
// outside the tile's TF support disk are written as zeros without being
// read, one column at a time.
#include "wo_fft.cuh"
#include "wo_internal.h"
#include "wo_regfft.cuh"
#include "wo_zops.cuh"

namespace wo {

namespace {

template <class P>
struct ZRegGeom {
  static constexpr int N = P::N, T = P::T, E = P::E;
  static constexpr int NT = 128;
  static constexpr int CPC = NT / T;  // x columns per CTA
  static constexpr size_t SMEM = ((size_t)P::TW + (size_t)CPC * P::SLICE) * sizeof(float2);
  static_assert(T <= 8, "a warp's loads and stores must cover whole sectors");
};

template <class P>
__global__ void __launch_bounds__(ZRegGeom<P>::NT) k_z_reg(const float2* __restrict__ in, float2* __restrict__ out,
                                                          const float2* __restrict__ tf, ZOp op, int Y, int Xh) {
  using G = ZRegGeom<P>;
  constexpr int N = G::N, T = G::T, E = G::E, CPC = G::CPC;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* slices = sm + P::TW;  // [CPC][SLICE]
  const int t = blockIdx.z, x0 = blockIdx.x * CPC;
  const int w = min(CPC, Xh - x0);
  const long long zs = (long long)Y * Xh;
  const long long vol = (long long)N * zs;
  const int tt = op.tf_shared ? 0 : t;  // the tile whose TFs and statistics apply
  const float* st = op.stats + (long long)tt * 8;
  const int X = 2 * (Xh - 1);
  const int y = blockIdx.y;
#if defined(WO_CHECK) && WO_CHECK
  {  // this strip's elements in the input, output and TF volumes
    const long long span = (long long)(N - 1) * zs + (long long)y * Xh + x0 + w - 1;
    const long long nt = gridDim.z, ntt = op.tf_shared ? 1 : nt;
    if (!WO_IN((long long)t * vol + span, nt * vol, 6) || !WO_IN((long long)tt * vol + span, ntt * vol, 6)) return;
  }
#endif
  const int l = threadIdx.x % T, cl = threadIdx.x / T;
  const int xg = x0 + cl;
  const bool live = cl < w;
  const bool inside = live && !outside_support(st, y, Y, xg, X);
  const long long col = (long long)y * Xh + (live ? xg : 0);
  float2* dst = out + (long long)t * vol + col;
  if (outside_support(st, y, Y, x0, X)) {  // the strip's nearest column is outside: all of it is (uniform)
    if (live) {
#pragma unroll
      for (int m = 0; m < E; ++m) dst[(long long)(l + T * m) * zs] = make_float2(0.f, 0.f);
    }
    return;
  }
  const bool lf = op.lf_props > 0;
  const float eta = lf ? op.eta_lf : op.eta_fl;
  const float lam = op.eta_absolute ? eta : eta * st[lf ? 0 : 2];
  const float2* src = in + (long long)t * vol + col;
  const float2* h = tf + (long long)tt * vol + col;
  float2 v[E], H[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const long long o = (long long)(l + T * m) * zs;
    v[m] = inside ? __ldg(src + o) : make_float2(0.f, 0.f);
    H[m] = inside ? __ldg(h + o) : make_float2(0.f, 0.f);
  }
  P::twiddles(tw);  // while the loads are in flight
  __syncthreads();
  P::template fft<false>(v, tw, slices + cl * P::SLICE, l);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const float2 x = v[m], hv = H[m];
    if (op.op == 0) {
      v[m] = cmul(hv, x);
    } else if (op.op == 1) {
      v[m] = cmulc(hv, x);
    } else {
      const bool dc = op.zero_dc && l + T * m == 0 && y == 0 && xg == 0;
      const float den = lam + cabs2(hv);
      const float inv = den > 0.f ? 1.0f / den : 0.f;  // zero TF and eta: minimum norm
      v[m] = dc ? make_float2(0.f, 0.f) : cscale(cmulc(hv, x), inv);
    }
  }
  P::template fft<true>(v, tw, slices + cl * P::SLICE, l);
  if (live) {
#pragma unroll
    for (int m = 0; m < E; ++m) dst[(long long)(l + T * m) * zs] = inside ? v[m] : make_float2(0.f, 0.f);
  }
}

template <class P>
cudaError_t launch_z_reg(const float2* in, float2* out, const float2* tf, ZOp op, int n_tiles, int Y, int Xh,
                         cudaStream_t s) {
  using G = ZRegGeom<P>;
  const cudaError_t attr = allow_smem(k_z_reg<P>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  dim3 grid((unsigned)((Xh + G::CPC - 1) / G::CPC), (unsigned)Y, (unsigned)n_tiles);
  WO_LAUNCH("z_fused", s, (k_z_reg<P><<<grid, G::NT, G::SMEM, s>>>(in, out, tf, op, Y, Xh)));
  return cudaGetLastError();
}

// The TF build's z pass for one-kind banks (the same scheme): forward
// transform along z of every TF column in place, and the per-tile maxima the
// relative regulariser uses — max over (k, column) of |H|^2 and max over
// columns of sum_k |H|^2 (statistics words 0, 1 for a label-free kind, 2, 3
// for fluorescence), as in k_tf_zpass.  Columns k_x >= x_cols (outside every
// tile's support, rounding noise only) are left as they are.
template <class P>
__global__ void __launch_bounds__(ZRegGeom<P>::NT) k_tf_zpass_reg(TfArgs a) {
  using G = ZRegGeom<P>;
  constexpr int N = G::N, T = G::T, E = G::E, CPC = G::CPC, NT = G::NT;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* slices = sm + P::TW;  // [CPC][SLICE]
  __shared__ float red[2 * (NT / 32)];
  const int Y = a.Y, Xh = a.X / 2 + 1;
  const int t = blockIdx.z, y = blockIdx.y, x0 = blockIdx.x * CPC;
  const int w = min(CPC, a.x_cols - x0);
  const long long zs = (long long)Y * Xh;
  const long long vol = (long long)N * zs;
#if defined(WO_CHECK) && WO_CHECK
  {  // this strip's elements of the tile's TF slot
    const long long span = (long long)(N - 1) * zs + (long long)y * Xh + x0 + w - 1;
    if (!WO_IN((long long)t * vol + span, (long long)gridDim.z * vol, 6)) return;  // uniform across the CTA
  }
#endif
  const int l = threadIdx.x % T, cl = threadIdx.x / T;
  const bool live = cl < w;
  float2* col = a.tf + (long long)t * vol + (long long)y * Xh + x0 + (live ? cl : 0);
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = live ? col[(long long)(l + T * m) * zs] : make_float2(0.f, 0.f);
  P::twiddles(tw);  // while the loads are in flight
  __syncthreads();
  P::template fft<false>(v, tw, slices + cl * P::SLICE, l);
  float m3 = 0.f, cs = 0.f;
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const float q = cabs2(v[m]);
    m3 = fmaxf(m3, q);
    cs += q;
  }
  if (live) {
#pragma unroll
    for (int m = 0; m < E; ++m) col[(long long)(l + T * m) * zs] = v[m];
  }
  // the column's sum over its T lanes (a fixed order), then block maxima
  // (values >= 0: integer order equals float order) and one atomic per statistic
#pragma unroll
  for (int o = 1; o < T; o <<= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
  float m2 = live ? cs : 0.f;
  if (!live) m3 = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m3 = fmaxf(m3, __shfl_down_sync(0xffffffffu, m3, o));
    m2 = fmaxf(m2, __shfl_down_sync(0xffffffffu, m2, o));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[2 * warp] = m3;
    red[2 * warp + 1] = m2;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    float mx = 0.f;
    for (int q = 0; q < NT / 32; ++q) mx = fmaxf(mx, red[2 * q + threadIdx.x]);
    const int slot = (a.lf_props > 0 ? 0 : 2) + threadIdx.x;
    if (mx > 0.f) atomicMax(reinterpret_cast<int*>(a.stats + (long long)t * 8) + slot, __float_as_int(mx));
  }
}

template <class P>
cudaError_t launch_tf_zpass_reg(const TfArgs& a, cudaStream_t s) {
  using G = ZRegGeom<P>;
  const cudaError_t attr = allow_smem(k_tf_zpass_reg<P>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  if (a.x_cols <= 0) return cudaSuccess;
  dim3 grid((unsigned)((a.x_cols + G::CPC - 1) / G::CPC), (unsigned)a.Y, (unsigned)a.n_tiles);
  WO_LAUNCH("tf_zpass", s, (k_tf_zpass_reg<P><<<grid, G::NT, G::SMEM, s>>>(a)));
  return cudaGetLastError();
}

}  // namespace

bool tf_zpass_reg_supported(const TfArgs& a) {
  if (a.n_kinds != 1) return false;
  const int Z = a.Z;
  return Z == 32 || Z == 48 || Z == 64 || Z == 96 || Z == 128 || Z == 192;
}

cudaError_t tf_zpass_reg(const TfArgs& a, cudaStream_t s) {
  switch (a.Z) {
    case 32: return launch_tf_zpass_reg<Row2<32, 8>>(a, s);
    case 48: return launch_tf_zpass_reg<Row2<48, 12>>(a, s);
    case 64: return launch_tf_zpass_reg<Row2<64, 8>>(a, s);
    case 96: return launch_tf_zpass_reg<Row2<96, 24>>(a, s);
    case 128: return launch_tf_zpass_reg<Row2<128, 16>>(a, s);
    case 192: return launch_tf_zpass_reg<Row2<192, 24>>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

bool z_reg_supported(int Z, const ZOp& op) {
  if (op.n_in != 1 || op.n_out != 1 || op.n_tf != 1 || op.lf_props + op.has_fl != 1) return false;
  if (op.lf_props > 0 ? op.lf_chan != 0 : op.fl_chan != 0) return false;
  return Z == 16 || Z == 32 || Z == 48 || Z == 64 || Z == 96 || Z == 128 || Z == 192;
}

cudaError_t z_fused_reg(int Z, const float2* in, float2* out, const float2* tf, ZOp op, int n_tiles, int Y, int Xh,
                        cudaStream_t s) {
  switch (Z) {
    case 16: return launch_z_reg<Row2<16, 4>>(in, out, tf, op, n_tiles, Y, Xh, s);
    case 32: return launch_z_reg<Row2<32, 8>>(in, out, tf, op, n_tiles, Y, Xh, s);
    case 48: return launch_z_reg<Row2<48, 12>>(in, out, tf, op, n_tiles, Y, Xh, s);
    case 64: return launch_z_reg<Row2<64, 8>>(in, out, tf, op, n_tiles, Y, Xh, s);
    case 96: return launch_z_reg<Row2<96, 24>>(in, out, tf, op, n_tiles, Y, Xh, s);
    case 128: return launch_z_reg<Row2<128, 16>>(in, out, tf, op, n_tiles, Y, Xh, s);
    case 192: return launch_z_reg<Row2<192, 24>>(in, out, tf, op, n_tiles, Y, Xh, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wo

// wo_armsreg.cu - the arm pass of the TF build with register-resident y
// transforms.
//
// The same operation as k_arms (wo_tf.cu) for banks without derivatives:
// per (tile t, plane j, strip of CPC columns) the arms of plane j, A = S
// e^{i phi}, B = i (1/eta) e^{i phi} (label-free) and P = [inside] e^{i phi}
// (fluorescence), phi = 2 pi eta z_j (+ 2 pi W with an aberrated pupil),
// each inverse-transformed along y.  Here T lanes of one warp own a column,
// lane l holding the points n = l + T m (the row transforms of wo_regfft.cuh
// run on a column): the arm values are generated straight into the
// registers the transform works on.  With T <= 8 a warp covers 32/T
// adjacent columns, and every record load of a warp fills whole 32-byte
// sectors.
//
// A lane loads its records in batches of eight (or four) points (the loads
// of a batch in flight together), forms the phase factor e^{i phi} of each
// point once and from it every arm's value: the first arm's into the
// registers of the transform, the later arms' into the lane's own
// shared-memory slots.  Points outside the pupil (zero amplitude in every
// arm) skip the phase, and columns outside the detection band (every arm
// zero there; the row pass never reads them) skip the loads and are not
// stored.  A transformed arm leaves through a strip tile in shared memory,
// so that every warp store writes whole rows of the strip.
#include "wo_fft.cuh"
#include "wo_internal.h"
#include "wo_regfft.cuh"
#include "wo_tf.cuh"

namespace wo {

namespace {

template <class P>
struct ArmGeom {
  static constexpr int N = P::N, T = P::T, E = P::E;
  static constexpr int NT = 128;
  static constexpr int CPC = NT / T;  // columns per CTA
  static constexpr int CH = E % 8 == 0 ? 8 : 4;  // points per load batch
  // the strip tile [N][PITCH] that the stores go through shares its space
  // with the transposes' slices; PITCH puts a half-warp's writes (T lanes of
  // 16/T columns) on distinct 8-byte bank pairs
  static constexpr int PITCH = CPC + 16 / T;
  static constexpr size_t SHARED =
      (size_t)N * PITCH > (size_t)CPC * P::SLICE ? (size_t)N * PITCH : (size_t)CPC * P::SLICE;
  // plus n_arms - 1 stash slots of [E][NT] (the arms after the first)
  static constexpr size_t BASE = ((size_t)P::TW + SHARED) * sizeof(float2);
  static constexpr size_t SLOT = (size_t)E * NT * sizeof(float2);
  static_assert(T <= 8, "a warp's loads and stores must cover whole sectors");
  static_assert(E % CH == 0, "whole load batches");
};

template <class P>
__global__ void __launch_bounds__(ArmGeom<P>::NT) k_arms_reg(TfArgs a) {
  using G = ArmGeom<P>;
  constexpr int N = G::N, T = G::T, E = G::E, NT = G::NT, CPC = G::CPC, CH = G::CH;
  extern __shared__ float2 sm[];
  float2* tw = sm;
  float2* slices = sm + P::TW;         // [CPC][SLICE]: the columns' transposes
  float2* tile = slices;               // [N][PITCH]: an arm's strip on its way out
  float2* stash = slices + G::SHARED;  // [arm - 1][E][NT]: the later arms' values
  const int X = a.X, Z = a.Z;
  const int t = blockIdx.z, j = blockIdx.y, x0 = blockIdx.x * CPC;
  const int w = min(CPC, X - x0);
  // strips whose columns all lie outside the detection band: every arm is zero
  const int kxmax = a.counts[4 * t + 2];
  bool active = false;
  for (int b = 0; b < w; ++b) active |= abs(fft_index(x0 + b, X)) <= kxmax;
  if (!active) return;  // uniform across the CTA
#if defined(WO_CHECK) && WO_CHECK
  {  // the strip's records and the arm strips it writes
    const long long nt = gridDim.z;
    if (!WO_IN((long long)t * N * X + x0 + (long long)(N - 1) * X + w - 1, nt * N * X, 8) ||
        !WO_IN((((long long)t * a.n_arms + a.n_arms - 1) * Z + j) * (long long)N * X + x0 + (long long)(N - 1) * X + w - 1,
               nt * a.n_arms * Z * (long long)N * X, 8))
      return;
  }
#endif
  P::twiddles(tw);
  // the plane's focal displacement as a float pair, formed in float64 by one
  // lane of each warp and broadcast
  float zh = 0.f, zl = 0.f;
  if ((threadIdx.x & 31) == 0) {
    const double zj = __dadd_rn(__dmul_rn((double)fft_index(j, Z), a.optics[t].z_step_um), a.optics[t].defocus_um);
    zh = __double2float_rn(zj);
    zl = __double2float_rn(__dsub_rn(zj, (double)zh));
  }
  zh = __shfl_sync(0xffffffffu, zh, 0);
  zl = __shfl_sync(0xffffffffu, zl, 0);
  const int l = threadIdx.x % T, cl = threadIdx.x / T;
  // lanes of columns past the strip or outside the band transform zeros and store nothing
  const bool live = cl < w && abs(fft_index(x0 + cl, X)) <= kxmax;
  const long long col = (long long)t * N * X + x0 + (live ? cl : 0);
  const float4* rec = a.rec + col;
  const float* wrec = a.n_zern > 0 ? reinterpret_cast<const float*>(a.rec2 + col) + 3 : nullptr;
  const bool lf = a.lf_props != 0, fl = a.want_fl != 0;
  // The arms, in slot order A, B (label-free), P (fluorescence), are
  // (al + i be) e^{i phi}: A (S, 0), B (0, 1/eta), P (1, 0) inside the pupil.
  // The first goes to v, the others to the stash.
  float2 v[E];
#pragma unroll
  for (int m0 = 0; m0 < E; m0 += CH) {
    float4 q[CH];
    float wv[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) {  // the batch's loads first
      const long long o = (long long)(l + T * (m0 + i)) * X;
      q[i] = live ? __ldg(rec + o) : make_float4(0.f, 0.f, 0.f, 0.f);
      wv[i] = (live && wrec) ? __ldg(wrec + 4 * o) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int m = m0 + i;
      float s = 0.f, c = 0.f;
      if (q[i].z != 0.f || q[i].w != 0.f) unit_phasor(phase_frac(q[i].x, q[i].y, zh, zl) + wv[i], &s, &c);
      const float S = q[i].w, ie = q[i].z, in = ie != 0.f ? 1.f : 0.f;
      if (lf) {
        v[m] = make_float2(S * c, S * s);
        stash[m * NT + threadIdx.x] = make_float2(-ie * s, ie * c);
        if (fl) stash[(E + m) * NT + threadIdx.x] = make_float2(in * c, in * s);
      } else {
        v[m] = make_float2(in * c, in * s);
      }
    }
  }
  __syncthreads();  // the twiddles
  const int n_arms = (lf ? 2 : 0) + (fl ? 1 : 0);
#pragma unroll 1
  for (int arm = 0; arm < n_arms; ++arm) {
    if (arm > 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = stash[((arm - 1) * E + m) * NT + threadIdx.x];
    }
    P::template fft<true>(v, tw, slices + cl * P::SLICE, l);
    // through the strip tile, so that each warp store covers whole rows of the strip
    __syncthreads();  // every column's transposes are done with the slices
#pragma unroll
    for (int m = 0; m < E; ++m) tile[(l + T * m) * G::PITCH + cl] = v[m];
    __syncthreads();
    float2* dst = a.arms + (((long long)t * a.n_arms + arm) * Z + j) * (long long)N * X + x0;
    for (int e = threadIdx.x; e < N * CPC; e += NT) {
      const int n = e / CPC, b = e % CPC;
      if (b < w && abs(fft_index(x0 + b, X)) <= kxmax) dst[(long long)n * X + b] = tile[n * G::PITCH + b];
    }
    __syncthreads();  // the tile's reads are done before the next transform
  }
}

template <class P>
cudaError_t launch_arms_reg(const TfArgs& a, cudaStream_t s) {
  using G = ArmGeom<P>;
  const cudaError_t attr = allow_smem(k_arms_reg<P>, G::BASE + 2 * G::SLOT);
  if (attr != cudaSuccess) return attr;
  const int n_arms = (a.lf_props != 0 ? 2 : 0) + (a.want_fl ? 1 : 0);
  if (n_arms != a.n_arms || n_arms == 0) return cudaErrorInvalidValue;
  const size_t smem = G::BASE + (size_t)(n_arms - 1) * G::SLOT;
  dim3 grid((unsigned)((a.X + G::CPC - 1) / G::CPC), (unsigned)a.Z, (unsigned)a.n_tiles);
  WO_LAUNCH("tf_arms", s, (k_arms_reg<P><<<grid, G::NT, smem, s>>>(a)));
  return cudaGetLastError();
}

}  // namespace

bool arms_reg_supported(int Y, const TfArgs& a) {
  if (a.want_dz || a.want_grad) return false;
  return Y == 32 || Y == 48 || Y == 64 || Y == 96 || Y == 128 || Y == 192;
}

cudaError_t tf_arms_reg(const TfArgs& a, cudaStream_t s) {
  switch (a.Y) {
    case 32: return launch_arms_reg<Row2<32, 8>>(a, s);
    case 48: return launch_arms_reg<Row2<48, 12>>(a, s);
    case 64: return launch_arms_reg<Row2<64, 8>>(a, s);
    case 96: return launch_arms_reg<Row2<96, 24>>(a, s);
    case 128: return launch_arms_reg<Row2<128, 16>>(a, s);
    case 192: return launch_arms_reg<Row2<192, 24>>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wo

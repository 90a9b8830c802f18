// wo_estmma.cu - the estimator's 3x3 convolutions on the tensor cores.
//
// Every convolution of the network (forward, its data gradient and its
// weight gradient) is a contraction, run here as an implicit GEMM with
// mma.sync.m16n8k16 (bfloat16 operands, float32 accumulators) on
// fragments staged in shared memory:
//   forward      y[b,co,p]  = relu(bias[co] + sum_{tap,ci} x[b,ci,p+tap] w[co,ci,tap])
//                M = output pixels, N = co, K = (tap, ci)
//   data grad    gx[b,ci,q] = [x[b,ci,q] > 0] sum_{tap,co} g[b,co,(q-tap)/s] w[co,ci,tap]
//                M = input pixels, N = ci, K = (tap, co)
//   weight grad  dw[co,ci,tap] = sum_{b,p} g[b,co,p] x[b,ci,p+tap]
//                M = co, N = ci (every tap per block), K = (b, p)
// The weights are bfloat16 (exact operands).  Activations and gradients are
// float32; each is split into three bfloat16 parts, v = hi + mid + lo, each
// the bfloat16 rounding of what the previous ones leave (|v - hi - mid - lo|
// <= 2^-26 |v|, below float32 rounding), so that the products keep float32
// accuracy: x w = hi w + mid w + lo w (three MMAs).  Products of bfloat16
// values are exact in float32, so the only roundings are the float32 sums'.
// (With two parts the splits alone leave 2^-17 of each product, enough to
// flip the ReLU masks of near-zero activations.)  The gradients, which decide
// no mask, split their float32 operands in two: g w = g_hi w + g_lo w, and
// g x = g_hi x_hi + g_hi x_lo + g_lo x_hi (2^-16 of each product left out).
//
// Fragment layout of mma.m16n8k16 (PTX ISA): with g = lane / 4 and
// t = lane % 4, A (16 x 16, row-major) holds rows g and g + 8, columns
// 2t, 2t+1 and 2t+8, 2t+9; B (16 x 8, K x N) holds k = 2t, 2t+1 and 2t+8,
// 2t+9 of column n = g; C (16 x 8) rows g and g + 8, columns 2t and 2t+1.
// Tiles sit in shared memory with k contiguous (A as [m][k], B as [n][k]),
// pitch 24 bfloat16, so every fragment word of a warp falls in its own bank.
#include <cuda_bf16.h>
#include <stdint.h>

#include "wo_internal.h"

namespace wo {

namespace {

constexpr int kMmaThreads = 128;  // four warps
constexpr int kPitch = 24;        // bfloat16 per staged row (16 used)

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& mid, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  const float r = v - __bfloat162float(hi);  // exact
  mid = __float2bfloat16_rn(r);
  lo = __float2bfloat16_rn(r - __bfloat162float(mid));
}

// c += a b for one m16n8k16 tile.
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Fragments by ldmatrix: each of the 8-row by 8-column bfloat16 matrices it
// reads is given by the 16-byte row addresses of eight lanes (lanes 8 i ..
// 8 i + 7 for matrix i), and lane l receives elements (l / 4, 2 (l mod 4) ..
// + 1) of every matrix: the m16n8k16 operand layout (g = l / 4, t = l mod 4).
// Every staging pitch here is a multiple of 8 bfloat16, so the rows are
// 16-byte aligned, and its eight rows fall on distinct 16-byte bank groups.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const __nv_bfloat16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a)
               : "memory");
}

__device__ __forceinline__ void ldsm_x2(uint32_t& r0, uint32_t& r1, const __nv_bfloat16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a) : "memory");
}

// A fragment of the 16 x 16 tile whose row 0 is at `s` (rows P bfloat16
// apart): matrices rows 0-7 / 8-15 by k 0-7 / 8-15, in the order a0..a3.
template <int P = kPitch>
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const __nv_bfloat16* s, int lane) {
  static_assert(P % 8 == 0, "16-byte aligned fragment rows");
  const int mi = lane >> 3, r = lane & 7;
  ldsm_x4(a, s + (r + ((mi & 1) << 3)) * P + ((mi & 2) << 2));
}

// B fragment of the 8 columns whose column 0 (k contiguous) is at `s`:
// matrices k 0-7 and 8-15 of the 8 columns (lanes 16-31 repeat the addresses
// of lanes 0-15; ldmatrix .x2 reads those of lanes 0-15).
template <int P = kPitch>
__device__ __forceinline__ void frag_b(uint32_t& b0, uint32_t& b1, const __nv_bfloat16* s, int lane) {
  static_assert(P % 8 == 0, "16-byte aligned fragment rows");
  const int r = lane & 7, c = (lane >> 3) & 1;
  ldsm_x2(b0, b1, s + r * P + 8 * c);
}

// B fragments of two adjacent 8-column tiles (columns 0-7 at `s`, 8-15 at
// s + 8 P) by one ldmatrix .x4: b[0], b[1] of the first, b[2], b[3] of the
// second.
template <int P = kPitch>
__device__ __forceinline__ void frag_b2(uint32_t (&b)[4], const __nv_bfloat16* s, int lane) {
  static_assert(P % 8 == 0, "16-byte aligned fragment rows");
  const int mi = lane >> 3, r = lane & 7;
  ldsm_x4(b, s + (r + ((mi >> 1) << 3)) * P + 8 * (mi & 1));
}

// Tiles with 32 k per row: pitch 40 bfloat16 (80 bytes), so that the eight
// 16-byte rows of an ldmatrix phase fall on distinct bank groups.
constexpr int kPitch32 = 40;

// ------------------------------------------------------------------ weights for the staging copies
// The layers' bfloat16 weights w[co][ci][tap] re-laid once per pass so that a
// stage's B tile is a run of whole rows: wtf[tap][co][ci] (forward: k = ci)
// and wtb[tap][ci][co] (data gradient: k = co), layer l at conv_off(l).
__host__ __device__ constexpr int conv_ci(int l) { return l == 0 ? 3 : (l == 1 ? 32 : (l == 2 ? 64 : 96)); }
__host__ __device__ constexpr int conv_co(int l) { return l == 0 ? 32 : (l == 1 ? 64 : (l == 2 ? 96 : 128)); }
__host__ __device__ constexpr long long conv_off(int l) {
  return l == 0 ? 0 : (l == 1 ? 864 : (l == 2 ? 864 + 18432 : 864 + 18432 + 55296));
}
constexpr long long kConvTotal = 864 + 18432 + 55296 + 110592;

struct ConvOffsets {
  long long w[4];  // each layer's weights in the flat parameter array
};

__global__ void k_conv_prep(const __nv_bfloat16* __restrict__ wb, ConvOffsets o, __nv_bfloat16* __restrict__ wtf,
                            __nv_bfloat16* __restrict__ wtb) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kConvTotal) return;
  const int l = i < conv_off(1) ? 0 : (i < conv_off(2) ? 1 : (i < conv_off(3) ? 2 : 3));
  const int CI = conv_ci(l), CO = conv_co(l);
  const long long off = conv_off(l);
  const long long r = i - off;  // [co][ci][tap]
  const int tap = (int)(r % 9), ci = (int)((r / 9) % CI), co = (int)(r / (9LL * CI));
  const __nv_bfloat16 v = wb[o.w[l] + r];
  wtf[off + ((long long)tap * CO + co) * CI + ci] = v;
  wtb[off + ((long long)tap * CI + ci) * CO + co] = v;
}

// Lane map of the A staging copies: a warp covers 8 pixels x 4 channel pairs,
// so the 32-bit (two-channel) shared-memory stores of a warp fall in
// distinct banks for row pitches of 12 or 20 words (like the fragment loads),
// and its global loads are 32-byte runs of 8 pixels per channel.
struct StageLane {
  int m_lo, p_lo;  // pixel within the group of 8, pair within the group of 4
  __device__ StageLane() : m_lo((threadIdx.x & 31) >> 2), p_lo(threadIdx.x & 3) {}
};

// ------------------------------------------------------------------ forward
// Block: 64 output pixels of one sample (four warps of 16) x all CO.  Stages
// run over (tap, 16-channel chunk); each stage's A (64 pixels x 16 channels,
// split in three parts) and B (CO x 16 weights, whole rows of wtf) are
// loaded into registers during the previous stage's products and written to
// the other of two shared-memory buffers: one barrier per stage.
template <int CI, int CO, int H, int S>
__global__ void __launch_bounds__(kMmaThreads) k_conv_fwd_mma(const float* __restrict__ x,
                                                              const __nv_bfloat16* __restrict__ wtf,
                                                              const float* __restrict__ w32, long long boff,
                                                              float* __restrict__ y) {
  constexpr int HO = (H + S - 1) / S, NPIX = HO * HO, NT = CO / 8, NC = CI / 16, NSTAGE = 9 * NC;
  constexpr int BV = CO * 4 / kMmaThreads;  // 8-byte weight copies per thread per stage
  static_assert(CI % 16 == 0 && (CO * 4) % kMmaThreads == 0, "channel counts of the staged forward");
  __shared__ __align__(16) __nv_bfloat16 ahi[2][64 * kPitch], amid[2][64 * kPitch], alo[2][64 * kPitch];
  __shared__ __align__(16) __nv_bfloat16 bs[2][CO * kPitch];
  const int b = blockIdx.y, p0 = blockIdx.x * 64;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const StageLane sl;
  // this thread's two pixels (groups 2 warp, 2 warp + 1) and two pairs (p_lo, p_lo + 4)
  int oh[2], ow[2];
  bool pv[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int p = p0 + (2 * warp + h) * 8 + sl.m_lo;
    pv[h] = p < NPIX;
    oh[h] = p / HO;
    ow[h] = p - (p / HO) * HO;
  }
  const float* xb = x + (long long)b * CI * H * H;
  float av[2][2][2];  // [pixel][pair][channel of the pair]
  uint2 bv[BV];
  auto load = [&](int st) {
    const int tap = st / NC, c0 = (st - (st / NC) * NC) * 16;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ih = oh[h] * S + tap / 3 - 1, iw = ow[h] * S + tap % 3 - 1;
      const bool ok = pv[h] && ih >= 0 && ih < H && iw >= 0 && iw < H;
      const float* src = xb + ((long long)(c0 + 2 * sl.p_lo) * H + (ok ? ih : 0)) * H + (ok ? iw : 0);
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < 2; ++c) av[h][q][c] = ok ? __ldg(src + (long long)(8 * q + c) * H * H) : 0.f;
    }
    const uint2* wsrc = reinterpret_cast<const uint2*>(wtf + (long long)tap * CO * CI + c0);
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      const int e = threadIdx.x + j * kMmaThreads, co = e >> 2, q = e & 3;
      bv[j] = __ldg(wsrc + co * (CI / 4) + q);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = (2 * warp + h) * 8 + sl.m_lo;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        __nv_bfloat16 h0, m0, l0, h1, m1, l1;
        split_bf16(av[h][q][0], h0, m0, l0);
        split_bf16(av[h][q][1], h1, m1, l1);
        const int o = m * kPitch + 2 * (sl.p_lo + 4 * q);
        *reinterpret_cast<__nv_bfloat162*>(&ahi[buf][o]) = __halves2bfloat162(h0, h1);
        *reinterpret_cast<__nv_bfloat162*>(&amid[buf][o]) = __halves2bfloat162(m0, m1);
        *reinterpret_cast<__nv_bfloat162*>(&alo[buf][o]) = __halves2bfloat162(l0, l1);
      }
    }
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      const int e = threadIdx.x + j * kMmaThreads, co = e >> 2, q = e & 3;
      *reinterpret_cast<uint2*>(&bs[buf][co * kPitch + 4 * q]) = bv[j];
    }
  };
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  load(0);
  store(0);
  __syncthreads();
  for (int st = 0; st < NSTAGE; ++st) {
    const int buf = st & 1;
    if (st + 1 < NSTAGE) load(st + 1);  // in flight during this stage's products
    uint32_t fh[4], fm[4], fl[4];
    frag_a(fh, ahi[buf] + warp * 16 * kPitch, lane);
    frag_a(fm, amid[buf] + warp * 16 * kPitch, lane);
    frag_a(fl, alo[buf] + warp * 16 * kPitch, lane);
    static_assert(NT % 2 == 0, "B tiles in pairs");
#pragma unroll
    for (int n = 0; n < NT; n += 2) {
      uint32_t bb[4];
      frag_b2(bb, bs[buf] + n * 8 * kPitch, lane);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        mma16816(acc[n + h], fl, bb[2 * h], bb[2 * h + 1]);
        mma16816(acc[n + h], fm, bb[2 * h], bb[2 * h + 1]);
        mma16816(acc[n + h], fh, bb[2 * h], bb[2 * h + 1]);
      }
    }
    // the other buffer was last read before the previous barrier
    if (st + 1 < NSTAGE) store(buf ^ 1);
    __syncthreads();
  }
  const int g = lane >> 2, t = lane & 3;
  float* yb = y + (long long)b * CO * NPIX;
#pragma unroll
  for (int n = 0; n < NT; ++n) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = p0 + warp * 16 + g + (q >= 2 ? 8 : 0), co = n * 8 + 2 * t + (q & 1);
      if (p < NPIX) yb[(long long)co * NPIX + p] = fmaxf(acc[n][q] + w32[boff + co], 0.f);
    }
  }
}

// Forward of a layer with 9 CI <= 32 (the first layer, three channels): K is
// (ci, tap), k = 9 ci + tap, in one 32-wide stage (rows 9 CI .. 31 zero),
// instead of nine taps each padded to 16 channels.
template <int CI, int CO, int H, int S>
__global__ void __launch_bounds__(kMmaThreads) k_conv_fwd_mma_k32(const float* __restrict__ x,
                                                                  const __nv_bfloat16* __restrict__ wb,
                                                                  const float* __restrict__ w32, long long woff,
                                                                  long long boff, float* __restrict__ y) {
  constexpr int HO = (H + S - 1) / S, NPIX = HO * HO, NT = CO / 8, KV = CI * 9, P = kPitch32;
  static_assert(KV <= 32 && CO % 8 == 0, "first-layer forward");
  __shared__ __align__(16) __nv_bfloat16 ahi[64 * P], amid[64 * P], alo[64 * P], bs[CO * P];
  const int b = blockIdx.y, p0 = blockIdx.x * 64;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* xb = x + (long long)b * CI * H * H;
  {  // A: 64 pixels x 16 k-pairs; a warp covers 8 pixels x 4 pairs (conflict-free 32-bit stores)
    const StageLane sl;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const int combo = warp + 4 * it;  // 32 combos = 8 pixel groups x 4 pair groups
      const int m = (combo & 7) * 8 + sl.m_lo, kp = (combo >> 3) * 4 + sl.p_lo;
      const int p = p0 + m;
      const int oh = p / HO, ow = p - (p / HO) * HO;
      float v[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int k = 2 * kp + c;
        v[c] = 0.f;
        if (p < NPIX && k < KV) {
          const int ci = k / 9, tap = k - 9 * (k / 9);
          const int ih = oh * S + tap / 3 - 1, iw = ow * S + tap % 3 - 1;
          if (ih >= 0 && ih < H && iw >= 0 && iw < H) v[c] = __ldg(xb + ((long long)ci * H + ih) * H + iw);
        }
      }
      __nv_bfloat16 h0, m0, l0, h1, m1, l1;
      split_bf16(v[0], h0, m0, l0);
      split_bf16(v[1], h1, m1, l1);
      const int o = m * P + 2 * kp;
      *reinterpret_cast<__nv_bfloat162*>(&ahi[o]) = __halves2bfloat162(h0, h1);
      *reinterpret_cast<__nv_bfloat162*>(&amid[o]) = __halves2bfloat162(m0, m1);
      *reinterpret_cast<__nv_bfloat162*>(&alo[o]) = __halves2bfloat162(l0, l1);
    }
  }
  // w[co][ci][tap] sits at woff + co KV + k
  for (int e = threadIdx.x; e < CO * 32; e += kMmaThreads) {
    const int co = e >> 5, k = e & 31;
    bs[co * P + k] = k < KV ? wb[woff + (long long)co * KV + k] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    uint32_t fh[4], fm[4], fl[4];
    frag_a<P>(fh, ahi + warp * 16 * P + ks * 16, lane);
    frag_a<P>(fm, amid + warp * 16 * P + ks * 16, lane);
    frag_a<P>(fl, alo + warp * 16 * P + ks * 16, lane);
    static_assert(NT % 2 == 0, "B tiles in pairs");
#pragma unroll
    for (int n = 0; n < NT; n += 2) {
      uint32_t bb[4];
      frag_b2<P>(bb, bs + n * 8 * P + ks * 16, lane);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        mma16816(acc[n + h], fl, bb[2 * h], bb[2 * h + 1]);
        mma16816(acc[n + h], fm, bb[2 * h], bb[2 * h + 1]);
        mma16816(acc[n + h], fh, bb[2 * h], bb[2 * h + 1]);
      }
    }
  }
  const int g = lane >> 2, t = lane & 3;
  float* yb = y + (long long)b * CO * NPIX;
#pragma unroll
  for (int n = 0; n < NT; ++n) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = p0 + warp * 16 + g + (q >= 2 ? 8 : 0), co = n * 8 + 2 * t + (q & 1);
      if (p < NPIX) yb[(long long)co * NPIX + p] = fmaxf(acc[n][q] + w32[boff + co], 0.f);
    }
  }
}

// ------------------------------------------------------------------ data gradient
// Stride 2.  Input row ih receives the kernel rows kh with ih + 1 - kh even,
// from output row (ih + 1 - kh) / 2: kh = 1 for even ih (output row ih / 2),
// kh = 0 and 2 for odd ih (output rows (ih + 1) / 2 and (ih - 1) / 2); the
// same for columns.  So the input pixels of one parity class (ih mod 2,
// iw mod 2) take the same 1, 2 or 4 taps, each from a shifted window of the
// output grid, and a block works on one class: a quarter of the nine taps on
// average, none of them on zeros.
// Block: 64 input pixels of one class of one sample (class grid (i, j),
// ih = 2 i + ph, iw = 2 j + pw) x all CI; stages of one tap x 32 output
// channels.  g is the gradient at the layer's output (already masked by its
// ReLU); the result is masked by the ReLU of the layer's input (xin > 0).  g
// is split in two (two MMAs: the data gradient decides no mask either).
template <int CI, int CO, int H, int S>
__global__ void __launch_bounds__(kMmaThreads) k_conv_bwd_data_mma(const float* __restrict__ gy,
                                                                   const __nv_bfloat16* __restrict__ wtb,
                                                                   const float* __restrict__ xin,
                                                                   float* __restrict__ gx) {
  constexpr int HO = H / 2, W2 = H / 2, NCLS = W2 * W2, BPC = (NCLS + 63) / 64, NT = CI / 8, P = kPitch32;
  constexpr int BV = CI * 4 / kMmaThreads;  // 16-byte weight copies per thread per stage
  static_assert(S == 2 && H % 2 == 0, "the data gradient by parity classes is for stride 2");
  static_assert(CI % 8 == 0 && CO % 32 == 0 && (CI * 4) % kMmaThreads == 0, "channel counts of the data gradient");
  __shared__ __align__(16) __nv_bfloat16 ahi[2][64 * P], alo[2][64 * P], bs[2][CI * P];
  const int b = blockIdx.y, cls = blockIdx.x / BPC, r0 = (blockIdx.x - cls * BPC) * 64;
  const int ph = cls >> 1, pw = cls & 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const StageLane sl;
  // this thread's two class pixels (groups 2 warp, 2 warp + 1) and four pairs (p_lo + 4 q)
  int ci_[2], cj_[2];
  bool rv[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = r0 + (2 * warp + h) * 8 + sl.m_lo;
    rv[h] = r < NCLS;
    ci_[h] = r / W2;
    cj_[h] = r - (r / W2) * W2;
  }
  const float* gb = gy + (long long)b * CO * HO * HO;
  // the class's taps, (kh, kw) with ih + 1 - kh and iw + 1 - kw even; stages (tap, 32-channel chunk)
  const int nkw = 1 + pw, NCH = CO / 32, nstage = (1 + ph) * nkw * NCH;
  float av[2][4][2];  // [pixel][pair group][channel of the pair]
  uint4 bv[BV];
  auto tap_of = [&](int st, int& kh, int& kw, int& c0) {
    const int tp = st / NCH;
    c0 = (st - tp * NCH) * 32;
    const int a = tp / nkw, c = tp - a * nkw;
    kh = ph ? 2 * a : 1;
    kw = pw ? 2 * c : 1;
  };
  auto load = [&](int st) {
    int kh, kw, c0;
    tap_of(st, kh, kw, c0);
    const int dh = (ph + 1 - kh) >> 1, dw = (pw + 1 - kw) >> 1;  // output row i + dh, column j + dw
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int oh = ci_[h] + dh, ow = cj_[h] + dw;
      const bool ok = rv[h] && oh < HO && ow < HO;
      const float* src = gb + ((long long)(c0 + 2 * sl.p_lo) * HO + (ok ? oh : 0)) * HO + (ok ? ow : 0);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 2; ++c) av[h][q][c] = ok ? __ldg(src + (long long)(8 * q + c) * HO * HO) : 0.f;
    }
    const uint4* wsrc = reinterpret_cast<const uint4*>(wtb + (long long)(kh * 3 + kw) * CI * CO + c0);
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      const int e = threadIdx.x + j * kMmaThreads, ci = e >> 2, q = e & 3;
      bv[j] = __ldg(wsrc + ci * (CO / 8) + q);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = (2 * warp + h) * 8 + sl.m_lo;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float v0 = av[h][q][0], v1 = av[h][q][1];
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
        const int o = m * P + 2 * (sl.p_lo + 4 * q);
        *reinterpret_cast<__nv_bfloat162*>(&ahi[buf][o]) = __halves2bfloat162(h0, h1);
        *reinterpret_cast<__nv_bfloat162*>(&alo[buf][o]) = __halves2bfloat162(l0, l1);
      }
    }
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      const int e = threadIdx.x + j * kMmaThreads, ci = e >> 2, q = e & 3;
      *reinterpret_cast<uint4*>(&bs[buf][ci * P + 8 * q]) = bv[j];
    }
  };
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  // the input ReLU's values at this thread's outputs, loaded now so that their
  // latency hides under the stages (for the narrower layers, where the
  // registers allow)
  const int g = lane >> 2, t = lane & 3;
  constexpr bool kEarly = NT <= 8;
  float xm[kEarly ? 4 : 1][kEarly ? NT : 1];
  // the input pixel of this thread's output rows (-1 past the class grid)
  auto out_pixel = [&](int q4) -> int {
    const int r = r0 + warp * 16 + g + (q4 >= 2 ? 8 : 0);
    const int i = r / W2, j = r - (r / W2) * W2;
    return r < NCLS ? (2 * i + ph) * H + 2 * j + pw : -1;
  };
  if constexpr (kEarly) {
    int xidx[4];
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) xidx[q4] = out_pixel(q4);
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4)
#pragma unroll
      for (int n = 0; n < NT; ++n)
        xm[q4][n] = xidx[q4] >= 0 ? __ldg(xin + ((long long)b * CI + n * 8 + 2 * t + (q4 & 1)) * H * H + xidx[q4]) : 0.f;
  }
  load(0);
  store(0);
  __syncthreads();
  for (int st = 0; st < nstage; ++st) {
    const int buf = st & 1;
    if (st + 1 < nstage) load(st + 1);  // in flight during this stage's products
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      uint32_t fh[4], fl[4];
      frag_a<P>(fh, ahi[buf] + warp * 16 * P + ks * 16, lane);
      frag_a<P>(fl, alo[buf] + warp * 16 * P + ks * 16, lane);
      static_assert(NT % 2 == 0, "B tiles in pairs");
#pragma unroll
      for (int n = 0; n < NT; n += 2) {
        uint32_t bb[4];
        frag_b2<P>(bb, bs[buf] + n * 8 * P + ks * 16, lane);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          mma16816(acc[n + h], fl, bb[2 * h], bb[2 * h + 1]);
          mma16816(acc[n + h], fh, bb[2 * h], bb[2 * h + 1]);
        }
      }
    }
    if (st + 1 < nstage) store(buf ^ 1);  // the other buffer was last read before the previous barrier
    __syncthreads();
  }
#pragma unroll
  for (int q4 = 0; q4 < 4; ++q4) {
    const int pix = out_pixel(q4);
    if (pix < 0) continue;
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      const int ci = n * 8 + 2 * t + (q4 & 1);
      const long long idx = ((long long)b * CI + ci) * H * H + pix;
      float xv;
      if constexpr (kEarly) xv = xm[q4][n];
      else xv = __ldg(xin + idx);
      gx[idx] = xv > 0.f ? acc[n][q4] : 0.f;
    }
  }
}

// ------------------------------------------------------------------ weight gradient
// Block: 16 input channels, every output channel and all nine taps, over the
// output pixels of samples [s0, s0 + chunk), 32 pixels (in raster order) per
// stage.  Warps: CO/16 row groups (16 output channels each) x 2 tap groups
// (taps 0-4, 5-8), so every warp has products to do and 40 accumulators.
// A stage's g (CO x 32) and the nine taps' input samples for its pixels
// (9 x 16 x 32) are loaded into registers during the previous stage's
// products and written to the other of two shared-memory buffers: one
// barrier per stage.  The weight gradient feeds only the weight update, so g
// and x are split in two parts (three MMAs: hi hi, hi lo, lo hi; 2^-16 of
// each product left out), unlike the forward pass, whose sums decide the
// ReLU masks.  The bias gradient (the sum of g over samples and pixels) is
// accumulated from the same staged values in float32: per thread over its
// stages, then over the warp's lanes in a fixed order; blocks of the first
// channel group write it per sample chunk.
constexpr int kWgThreads = 256;  // the first layer's kernel
constexpr int kWgPix = 32;     // output pixels per stage
constexpr int kWgPitch = 40;   // bfloat16 per staged row (32 used)

template <int CO>
struct WgGeom {
  static constexpr int MT = CO / 16, NW = 2 * MT, NT = 32 * NW;
  static constexpr int GV = CO * kWgPix / NT, XV = 9 * 16 * kWgPix / NT;
  static constexpr int MINB = NT <= 384 ? 2 : 1;  // blocks per SM the register budget is cut for
  static constexpr size_t SMEM = 2 * (2 * (size_t)CO + 2 * 9 * 16) * kWgPitch * sizeof(__nv_bfloat16);
  static_assert(CO % 16 == 0 && (9 * 16 * kWgPix) % NT == 0, "output channels of the weight gradient");
};

template <int CI, int CO, int H, int S>
__global__ void __launch_bounds__(WgGeom<CO>::NT, WgGeom<CO>::MINB) k_conv_bwd_weight_mma(const float* __restrict__ gy,
                                                                        const float* __restrict__ x, int B,
                                                                        int chunk, float* __restrict__ part,
                                                                        float* __restrict__ partb) {
  using G = WgGeom<CO>;
  constexpr int HO = (H + S - 1) / S, NPIX = HO * HO, PS = (NPIX + kWgPix - 1) / kWgPix;
  constexpr int MT = G::MT, NW = G::NW, NT = G::NT, GV = G::GV, XV = G::XV, P = kWgPitch;
  extern __shared__ __align__(16) unsigned char wg_raw[];
  __nv_bfloat16* ghi = reinterpret_cast<__nv_bfloat16*>(wg_raw);  // [2][CO][P]
  __nv_bfloat16* glo = ghi + 2 * CO * P;                           // [2][CO][P]
  __nv_bfloat16* xhi = glo + 2 * CO * P;                           // [2][9 * 16][P]
  __nv_bfloat16* xlo = xhi + 2 * 144 * P;                          // [2][9 * 16][P]
  const int c0 = blockIdx.x * 16, ck = blockIdx.y;
  const int s0 = ck * chunk, s1 = min(B, s0 + chunk);
  const int nst = (s1 > s0 ? s1 - s0 : 0) * PS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int mt = warp % MT, tg = warp / MT, tap0 = tg * 5;  // taps tap0 .. min(tap0 + 5, 9) - 1
  float acc[5][2][4];
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int n = 0; n < 2; ++n) acc[q][n][0] = acc[q][n][1] = acc[q][n][2] = acc[q][n][3] = 0.f;
  // a thread stages pixel k = lane of every stage: output channels warp + NW i
  // of g, and (tap, channel) pairs (warp + NW i) of x
  float gv[GV], xv[XV], bacc[GV];
#pragma unroll
  for (int i = 0; i < GV; ++i) bacc[i] = 0.f;
  auto load = [&](int st) {
    const int sb = s0 + st / PS, p = (st - (st / PS) * PS) * kWgPix + lane;
    const bool pv = p < NPIX;
    const float* gb = gy + (long long)sb * CO * NPIX + (pv ? p : 0);
#pragma unroll
    for (int i = 0; i < GV; ++i) gv[i] = pv ? __ldg(gb + (long long)(warp + NW * i) * NPIX) : 0.f;
    const int oh = p / HO, ow = p - (p / HO) * HO;
    const float* xb = x + ((long long)sb * CI + c0) * H * H;
#pragma unroll
    for (int i = 0; i < XV; ++i) {
      const int r = warp + NW * i, c = r & 15, tap = r >> 4;
      const int ih = oh * S + tap / 3 - 1, iw = ow * S + tap % 3 - 1;
      const bool ok = pv && c0 + c < CI && ih >= 0 && ih < H && iw >= 0 && iw < H;
      xv[i] = ok ? __ldg(xb + ((long long)c * H + ih) * H + iw) : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < GV; ++i) {
      const int o = (buf * CO + warp + NW * i) * P + lane;
      const __nv_bfloat16 h = __float2bfloat16_rn(gv[i]);
      ghi[o] = h;
      glo[o] = __float2bfloat16_rn(gv[i] - __bfloat162float(h));
      bacc[i] += gv[i];
    }
#pragma unroll
    for (int i = 0; i < XV; ++i) {
      const int o = (buf * 144 + warp + NW * i) * P + lane;  // row tap * 16 + c
      const __nv_bfloat16 h = __float2bfloat16_rn(xv[i]);
      xhi[o] = h;
      xlo[o] = __float2bfloat16_rn(xv[i] - __bfloat162float(h));
    }
  };
  if (nst > 0) {
    load(0);
    store(0);
  }
  __syncthreads();
  for (int st = 0; st < nst; ++st) {
    const int buf = st & 1;
    if (st + 1 < nst) load(st + 1);  // in flight during this stage's products
    const __nv_bfloat16* gh = ghi + (buf * CO + mt * 16) * P;
    const __nv_bfloat16* gl = glo + (buf * CO + mt * 16) * P;
#pragma unroll
    for (int ks = 0; ks < kWgPix / 16; ++ks) {
      uint32_t fh[4], fl[4];
      frag_a<P>(fh, gh + ks * 16, lane);
      frag_a<P>(fl, gl + ks * 16, lane);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const int tap = tap0 + q;
        if (tap >= 9) break;
        // the tap's two 8-column tiles: by one ldmatrix .x4 each, unless the
        // register budget is that of 384 threads at two blocks per SM (85 per
        // thread), where the four fragment registers more spill
        uint32_t bh[4], bl[4];
        if constexpr (NT * G::MINB > 512) {
#pragma unroll
          for (int n = 0; n < 2; ++n) {
            frag_b<P>(bh[2 * n], bh[2 * n + 1], xhi + (buf * 144 + tap * 16 + n * 8) * P + ks * 16, lane);
            frag_b<P>(bl[2 * n], bl[2 * n + 1], xlo + (buf * 144 + tap * 16 + n * 8) * P + ks * 16, lane);
          }
        } else {
          frag_b2<P>(bh, xhi + (buf * 144 + tap * 16) * P + ks * 16, lane);
          frag_b2<P>(bl, xlo + (buf * 144 + tap * 16) * P + ks * 16, lane);
        }
#pragma unroll
        for (int n = 0; n < 2; ++n) {
          mma16816(acc[q][n], fh, bl[2 * n], bl[2 * n + 1]);
          mma16816(acc[q][n], fl, bh[2 * n], bh[2 * n + 1]);
          mma16816(acc[q][n], fh, bh[2 * n], bh[2 * n + 1]);
        }
      }
    }
    if (st + 1 < nst) store(buf ^ 1);  // the other buffer was last read before the previous barrier
    __syncthreads();
  }
  float* pc = part + (long long)ck * CO * CI * 9;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int tap = tap0 + q;
    if (tap >= 9) break;
#pragma unroll
    for (int n = 0; n < 2; ++n) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int co = mt * 16 + g + (r >= 2 ? 8 : 0), ci = c0 + n * 8 + 2 * t + (r & 1);
        if (ci < CI) pc[((long long)co * CI + ci) * 9 + tap] = acc[q][n][r];
      }
    }
  }
  if (blockIdx.x != 0) return;  // every channel group stages the same g: one writes the bias sums
#pragma unroll
  for (int i = 0; i < GV; ++i) {
    float v = bacc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) partb[(long long)ck * CO + warp + NW * i] = v;
  }
}

// Weight gradient of a layer with 9 CI <= 32 (the first layer): N is
// (ci, tap), n = 9 ci + tap, one 32-wide tile (rows 9 CI .. 31 zero), instead
// of nine taps each padded to 16 channels.  The eight warps are CO / 16 row
// groups x 8 / (CO / 16) pixel slices over 64 output pixels per stage; the
// slices' sums are added in slice order at the end.  As in the other weight
// gradients, a stage's g and x are loaded into registers during the previous
// stage's products and written to the other of two buffers.
constexpr int kWgPixN = 64;
constexpr int kWgPitchN = 72;  // 144 bytes: the eight 16-byte rows of an ldmatrix phase on distinct bank groups

template <int CI, int CO, int H, int S>
__global__ void __launch_bounds__(kWgThreads, 2) k_conv_bwd_weight_mma_n32(const float* __restrict__ gy,
                                                                        const float* __restrict__ x, int B,
                                                                        int chunk, float* __restrict__ part,
                                                                        float* __restrict__ partb) {
  constexpr int HO = (H + S - 1) / S, NPIX = HO * HO, MT = CO / 16, SL = 8 / MT, PX = kWgPixN / SL;
  constexpr int KV = CI * 9, P = kWgPitchN, PS = (NPIX + kWgPixN - 1) / kWgPixN;
  constexpr int GB = CO * kWgPixN / kWgThreads, CS = kWgThreads / kWgPixN;  // g per thread, channel sets
  constexpr int XV = (KV * kWgPixN + kWgThreads - 1) / kWgThreads;
  static_assert(KV <= 32 && CO % 16 == 0 && 8 % MT == 0 && PX % 16 == 0 && (CO * kWgPixN) % kWgThreads == 0,
                "first-layer weight gradient");
  constexpr int BUF = (2 * CO + 2 * 32) * P;  // bfloat16 per buffer: g hi, g lo, x hi, x lo
  constexpr int STAGE_BYTES = 2 * BUF * 2, RED_BYTES = (SL - 1) * MT * 512 * 4;
  __shared__ __align__(16) unsigned char raw[STAGE_BYTES > RED_BYTES ? STAGE_BYTES : RED_BYTES];
  __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(raw);
  const int ck = blockIdx.y;
  const int s0 = ck * chunk, s1 = min(B, s0 + chunk);
  const int nst = (s1 > s0 ? s1 - s0 : 0) * PS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mt = warp % MT, sl = warp / MT;
  const int g = lane >> 2, t = lane & 3;
  for (int e = threadIdx.x; e < 2 * (32 - KV) * kWgPixN; e += kWgThreads) {  // the zero rows of both buffers, once
    const int bb = e / ((32 - KV) * kWgPixN), r = e % ((32 - KV) * kWgPixN);
    const int n = KV + r / kWgPixN, k = r % kWgPixN;
    __nv_bfloat16* xb = base + bb * BUF + 2 * CO * P;
    xb[n * P + k] = xb[32 * P + n * P + k] = __float2bfloat16_rn(0.f);
  }
  float acc[4][4];
#pragma unroll
  for (int n = 0; n < 4; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  // thread tid stages pixel k = tid % kWgPixN of output channels tid / kWgPixN + CS i,
  // and the bias gradient from those values
  float gv[GB], xv[XV], bacc[GB];
#pragma unroll
  for (int i = 0; i < GB; ++i) bacc[i] = 0.f;
  const int kk = threadIdx.x % kWgPixN;
  auto load = [&](int st) {
    const int sb = s0 + st / PS, p = (st - (st / PS) * PS) * kWgPixN + kk;
    const bool pv = p < NPIX;
    const float* gb = gy + (long long)sb * CO * NPIX + (pv ? p : 0);
#pragma unroll
    for (int i = 0; i < GB; ++i) gv[i] = pv ? __ldg(gb + (long long)(threadIdx.x / kWgPixN + CS * i) * NPIX) : 0.f;
    const int oh = p / HO, ow = p - (p / HO) * HO;
    const float* xb = x + (long long)sb * CI * H * H;
#pragma unroll
    for (int i = 0; i < XV; ++i) {
      const int n = (threadIdx.x + kWgThreads * i) / kWgPixN;
      const int ci = n / 9, tap = n - 9 * (n / 9);
      const int ih = oh * S + tap / 3 - 1, iw = ow * S + tap % 3 - 1;
      const bool ok = pv && n < KV && ih >= 0 && ih < H && iw >= 0 && iw < H;
      xv[i] = ok ? __ldg(xb + ((long long)ci * H + ih) * H + iw) : 0.f;
    }
  };
  auto store = [&](int buf) {
    __nv_bfloat16* gh = base + buf * BUF;
#pragma unroll
    for (int i = 0; i < GB; ++i) {
      const int o = (threadIdx.x / kWgPixN + CS * i) * P + kk;
      const __nv_bfloat16 h = __float2bfloat16_rn(gv[i]);
      gh[o] = h;
      gh[CO * P + o] = __float2bfloat16_rn(gv[i] - __bfloat162float(h));
      bacc[i] += gv[i];
    }
    __nv_bfloat16* xh = gh + 2 * CO * P;
#pragma unroll
    for (int i = 0; i < XV; ++i) {
      const int n = (threadIdx.x + kWgThreads * i) / kWgPixN;
      if (n >= KV) continue;
      const __nv_bfloat16 h = __float2bfloat16_rn(xv[i]);
      xh[n * P + kk] = h;
      xh[32 * P + n * P + kk] = __float2bfloat16_rn(xv[i] - __bfloat162float(h));
    }
  };
  if (nst > 0) {
    load(0);
    store(0);
  }
  __syncthreads();
  for (int st = 0; st < nst; ++st) {
    const int buf = st & 1;
    if (st + 1 < nst) load(st + 1);  // in flight during this stage's products
    const __nv_bfloat16* ghi = base + buf * BUF;
    const __nv_bfloat16* glo = ghi + CO * P;
    const __nv_bfloat16* xhi = glo + CO * P;
    const __nv_bfloat16* xlo = xhi + 32 * P;
#pragma unroll
    for (int ks = 0; ks < PX / 16; ++ks) {
      const int k0 = sl * PX + ks * 16;
      uint32_t fh[4], fl[4];
      frag_a<P>(fh, ghi + mt * 16 * P + k0, lane);
      frag_a<P>(fl, glo + mt * 16 * P + k0, lane);
#pragma unroll
      for (int n = 0; n < 4; n += 2) {
        uint32_t bh[4], bl[4];
        frag_b2<P>(bh, xhi + n * 8 * P + k0, lane);
        frag_b2<P>(bl, xlo + n * 8 * P + k0, lane);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          mma16816(acc[n + h], fh, bl[2 * h], bl[2 * h + 1]);
          mma16816(acc[n + h], fl, bh[2 * h], bh[2 * h + 1]);
          mma16816(acc[n + h], fh, bh[2 * h], bh[2 * h + 1]);
        }
      }
    }
    if (st + 1 < nst) store(buf ^ 1);  // the other buffer was last read before the previous barrier
    __syncthreads();
  }
  // bias: each warp's sums over its lanes, then, in warp order, those of the
  // warps that staged the same channels (the staging buffers are free: the
  // loop ended on a barrier)
  float* rb = reinterpret_cast<float*>(raw);  // [warp][GB]
#pragma unroll
  for (int i = 0; i < GB; ++i) {
    float v = bacc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) rb[warp * GB + i] = v;
  }
  __syncthreads();
  constexpr int WPC = kWgPixN / 32;  // warps per channel set
  if (threadIdx.x < CO) {
    const int co = threadIdx.x, set = co % CS, i = co / CS;
    float v = 0.f;
    for (int w = 0; w < WPC; ++w) v += rb[(set * WPC + w) * GB + i];
    partb[(long long)ck * CO + co] = v;
  }
  __syncthreads();  // rb read before the slices reuse the buffer
  // slices 1 .. SL-1 hand their sums to slice 0 (the staging buffers are free: the loop ended on a barrier)
  float* red = reinterpret_cast<float*>(raw);
  if (sl > 0) {
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) red[(((sl - 1) * MT + mt) * 16 + n * 4 + q) * 32 + lane] = acc[n][q];
  }
  __syncthreads();
  if (sl > 0) return;
#pragma unroll
  for (int o = 1; o < SL; ++o) {
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[n][q] += red[(((o - 1) * MT + mt) * 16 + n * 4 + q) * 32 + lane];
  }
  float* pc = part + (long long)ck * CO * KV;
#pragma unroll
  for (int n = 0; n < 4; ++n) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int co = mt * 16 + g + (q >= 2 ? 8 : 0), nn = n * 8 + 2 * t + (q & 1);
      if (nn < KV) pc[(long long)co * KV + nn] = acc[n][q];  // w[co][ci][tap] at co KV + 9 ci + tap
    }
  }
}

// grad[woff + i] = sum over chunks of part[chunk][i] (i < n, the weights),
// grad[boff + j] = sum over chunks of partb[chunk][j] (j < nb, the biases).
// A block takes 32 consecutive entries (one per lane, coalesced loads); its
// eight warps sum the chunks c = warp (mod 8) in chunk order, and lane e of
// warp 0 adds the eight warp sums in warp order: a fixed order throughout.
__global__ void __launch_bounds__(256) k_reduce_chunks(const float* __restrict__ part, int chunks, long long n,
                                                       long long woff, const float* __restrict__ partb, int nb,
                                                       long long boff, float* __restrict__ grad) {
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long i = (long long)blockIdx.x * 32 + lane;
  const bool live = i < n + nb, w = i < n;
  const float* src = w ? part + i : partb + (i - n);
  const long long stride = w ? n : nb;
  float s = 0.f;
  if (live) {
#pragma unroll 4
    for (int c = warp; c < chunks; c += 8) s += __ldg(src + (long long)c * stride);
  }
  red[warp][lane] = s;
  __syncthreads();
  if (warp != 0 || !live) return;
  float t = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) t += red[q][lane];
  grad[w ? woff + i : boff + (i - n)] = t;
}

// Profiler labels per layer.
constexpr const char* kFwdName[4] = {"est_conv_fwd_l1", "est_conv_fwd_l2", "est_conv_fwd_l3", "est_conv_fwd_l4"};
constexpr const char* kWgName[4] = {"est_wgrad_l1", "est_wgrad_l2", "est_wgrad_l3", "est_wgrad_l4"};
constexpr const char* kDgName[4] = {"est_dgrad_l1", "est_dgrad_l2", "est_dgrad_l3", "est_dgrad_l4"};

template <int CI, int CO, int H, int S>
__host__ __device__ constexpr int layer_of() {
  return CI == 3 ? 0 : (CI == 32 ? 1 : (CI == 64 ? 2 : 3));
}

template <int CI, int CO, int H, int S>
cudaError_t fwd_layer(const float* x, const __nv_bfloat16* wb, const __nv_bfloat16* wt, const float* w32,
                      long long woff, long long boff, int B, float* y, cudaStream_t s) {
  constexpr int HO = (H + S - 1) / S;
  constexpr int l = layer_of<CI, CO, H, S>();
  dim3 grid((unsigned)((HO * HO + 63) / 64), (unsigned)B);
  const char* name = kFwdName[l];
  if constexpr (CI * 9 <= 32) {
    WO_LAUNCH(name, s, (k_conv_fwd_mma_k32<CI, CO, H, S><<<grid, kMmaThreads, 0, s>>>(x, wb, w32, woff, boff, y)));
  } else {
    WO_LAUNCH(name, s, (k_conv_fwd_mma<CI, CO, H, S><<<grid, kMmaThreads, 0, s>>>(x, wt + conv_off(l), w32, boff,
                                                                                 y)));
  }
  return cudaGetLastError();
}

template <int CI, int CO, int H, int S>
cudaError_t bwd_layer(const float* gy, const float* xin, const __nv_bfloat16* wt, long long woff, long long boff,
                      int B, float* gx, float* part, size_t part_floats, float* grad, cudaStream_t s) {
  // weight gradient: blocks (16-channel group, sample chunk); chunks so that
  // the grid has about 600 blocks and the partials fit their buffer (weight
  // partials [chunk][CO][CI][9], then bias partials [chunk][CO])
  const int per = (CI + 15) / 16;
  int chunks = (608 + per - 1) / per;
  const long long wsz = (long long)CO * CI * 9;
  if ((long long)chunks * (wsz + CO) > (long long)part_floats) chunks = (int)(part_floats / (wsz + CO));
  if (chunks > B) chunks = B;
  if (chunks < 1) return cudaErrorInvalidValue;
  const int chunk = (B + chunks - 1) / chunks;
  chunks = (B + chunk - 1) / chunk;
  float* bpart = part + (long long)chunks * wsz;
  dim3 gw((unsigned)((CI + 15) / 16), (unsigned)chunks);
  const char* wname = kWgName[layer_of<CI, CO, H, S>()];
  if constexpr (CI * 9 <= 32) {
    WO_LAUNCH(wname, s, (k_conv_bwd_weight_mma_n32<CI, CO, H, S><<<gw, kWgThreads, 0, s>>>(gy, xin, B, chunk,
                                                                                          part, bpart)));
  } else {
    using G = WgGeom<CO>;
    const cudaError_t attr = allow_smem(k_conv_bwd_weight_mma<CI, CO, H, S>, G::SMEM);
    if (attr != cudaSuccess) return attr;
    WO_LAUNCH(wname, s, (k_conv_bwd_weight_mma<CI, CO, H, S><<<gw, G::NT, G::SMEM, s>>>(gy, xin, B, chunk, part,
                                                                                      bpart)));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  WO_LAUNCH("est_wgrad_reduce", s, (k_reduce_chunks<<<(unsigned)((wsz + CO + 31) / 32), 256, 0, s>>>(
                                       part, chunks, wsz, woff, bpart, CO, boff, grad)));
  e = cudaGetLastError();
  if (e != cudaSuccess || gx == nullptr) return e;
  if constexpr (CI % 8 == 0 && S == 2) {
    dim3 gd((unsigned)(4 * ((H / 2 * (H / 2) + 63) / 64)), (unsigned)B);
    const char* dname = kDgName[layer_of<CI, CO, H, S>()];
    WO_LAUNCH(dname, s, (k_conv_bwd_data_mma<CI, CO, H, S><<<gd, kMmaThreads, 0, s>>>(
                            gy, wt + kConvTotal + conv_off(layer_of<CI, CO, H, S>()), xin, gx)));
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// The layers' weights re-laid for the staging copies (wt: 2 x 185184
// bfloat16, forward layout then data-gradient layout).
size_t est_conv_prep_elems() { return 2 * (size_t)kConvTotal; }

cudaError_t est_conv_prep(const void* wb, const long long* woff, void* wt, cudaStream_t s) {
  ConvOffsets o{};
  for (int l = 0; l < 4; ++l) o.w[l] = woff[l];
  __nv_bfloat16* f = (__nv_bfloat16*)wt;
  WO_LAUNCH("est_conv_prep", s, (k_conv_prep<<<(unsigned)((kConvTotal + 255) / 256), 256, 0, s>>>(
                                    (const __nv_bfloat16*)wb, o, f, f + kConvTotal)));
  return cudaGetLastError();
}

// The four layers of the estimator (3->32 stride 1 at 64 x 64, 32->64,
// 64->96, 96->128 stride 2).
cudaError_t est_conv_fwd_mma(int layer, const float* x, const void* wb, const void* wt, const float* w32,
                             long long woff, long long boff, int B, float* y, cudaStream_t s) {
  const __nv_bfloat16* w = (const __nv_bfloat16*)wb;
  const __nv_bfloat16* t = (const __nv_bfloat16*)wt;
  switch (layer) {
    case 0: return fwd_layer<3, 32, 64, 1>(x, w, t, w32, woff, boff, B, y, s);
    case 1: return fwd_layer<32, 64, 64, 2>(x, w, t, w32, woff, boff, B, y, s);
    case 2: return fwd_layer<64, 96, 32, 2>(x, w, t, w32, woff, boff, B, y, s);
    case 3: return fwd_layer<96, 128, 16, 2>(x, w, t, w32, woff, boff, B, y, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t est_conv_bwd_mma(int layer, const float* gy, const float* xin, const void* wt, long long woff,
                             long long boff, int B, float* gx, float* part, size_t part_floats, float* grad,
                             cudaStream_t s) {
  const __nv_bfloat16* t = (const __nv_bfloat16*)wt;
  switch (layer) {
    case 0: return bwd_layer<3, 32, 64, 1>(gy, xin, t, woff, boff, B, nullptr, part, part_floats, grad, s);
    case 1: return bwd_layer<32, 64, 64, 2>(gy, xin, t, woff, boff, B, gx, part, part_floats, grad, s);
    case 2: return bwd_layer<64, 96, 32, 2>(gy, xin, t, woff, boff, B, gx, part, part_floats, grad, s);
    case 3: return bwd_layer<96, 128, 16, 2>(gy, xin, t, woff, boff, B, gx, part, part_floats, grad, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wo

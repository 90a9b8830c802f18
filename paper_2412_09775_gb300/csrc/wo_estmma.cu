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

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// c += a b for one m16n8k16 tile.
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragment of the 16 x 16 tile whose row 0 is at `s` (rows P bfloat16 apart).
template <int P = kPitch>
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const __nv_bfloat16* s, int lane) {
  const int g = lane >> 2, t = lane & 3;
  a[0] = ld32(s + g * P + 2 * t);
  a[1] = ld32(s + (g + 8) * P + 2 * t);
  a[2] = ld32(s + g * P + 2 * t + 8);
  a[3] = ld32(s + (g + 8) * P + 2 * t + 8);
}

// B fragment of the 8 columns whose column 0 (k contiguous) is at `s`.
template <int P = kPitch>
__device__ __forceinline__ void frag_b(uint32_t& b0, uint32_t& b1, const __nv_bfloat16* s, int lane) {
  const int g = lane >> 2, t = lane & 3;
  b0 = ld32(s + g * P + 2 * t);
  b1 = ld32(s + g * P + 2 * t + 8);
}

// Tiles with 32 k per row: pitch 40 bfloat16 (20 words), so that the eight
// rows g of a fragment load start in banks 20 g mod 32, all different.
constexpr int kPitch32 = 40;

__host__ __device__ constexpr int ceil16(int v) { return (v + 15) / 16 * 16; }

// ------------------------------------------------------------------ forward
// Block: 64 output pixels of one sample (four warps of 16) x all CO.
template <int CI, int CO, int H, int S>
__global__ void __launch_bounds__(kMmaThreads) k_conv_fwd_mma(const float* __restrict__ x,
                                                              const __nv_bfloat16* __restrict__ wb,
                                                              const float* __restrict__ w32, long long woff,
                                                              long long boff, float* __restrict__ y) {
  constexpr int HO = (H + S - 1) / S, NPIX = HO * HO, CIP = ceil16(CI), NT = CO / 8;
  __shared__ __align__(16) __nv_bfloat16 ahi[64 * kPitch], amid[64 * kPitch], alo[64 * kPitch], bs[CO * kPitch];
  const int b = blockIdx.y, p0 = blockIdx.x * 64;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  const float* xb = x + (long long)b * CI * H * H;
  for (int tap = 0; tap < 9; ++tap) {
    const int kh = tap / 3, kw = tap % 3;
    for (int c0 = 0; c0 < CIP; c0 += 16) {
      // A: 64 pixels x 16 channels, split into three bfloat16 parts
      for (int e = threadIdx.x; e < 64 * 16; e += kMmaThreads) {
        const int c = e >> 6, m = e & 63;
        const int p = p0 + m, ci = c0 + c;
        float v = 0.f;
        if (p < NPIX && ci < CI) {
          const int oh = p / HO, ow = p - (p / HO) * HO;
          const int ih = oh * S + kh - 1, iw = ow * S + kw - 1;
          if (ih >= 0 && ih < H && iw >= 0 && iw < H) v = __ldg(xb + ((long long)ci * H + ih) * H + iw);
        }
        split_bf16(v, ahi[m * kPitch + c], amid[m * kPitch + c], alo[m * kPitch + c]);
      }
      // B: 16 channels x CO weights w[co][ci][tap]
      for (int e = threadIdx.x; e < CO * 16; e += kMmaThreads) {
        const int co = e >> 4, c = e & 15, ci = c0 + c;
        bs[co * kPitch + c] = ci < CI ? wb[woff + ((long long)co * CI + ci) * 9 + tap] : __float2bfloat16_rn(0.f);
      }
      __syncthreads();
      uint32_t fh[4], fm[4], fl[4];
      frag_a(fh, ahi + warp * 16 * kPitch, lane);
      frag_a(fm, amid + warp * 16 * kPitch, lane);
      frag_a(fl, alo + warp * 16 * kPitch, lane);
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        uint32_t b0, b1;
        frag_b(b0, b1, bs + n * 8 * kPitch, lane);
        mma16816(acc[n], fl, b0, b1);
        mma16816(acc[n], fm, b0, b1);
        mma16816(acc[n], fh, b0, b1);
      }
      __syncthreads();
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
  for (int e = threadIdx.x; e < 64 * 32; e += kMmaThreads) {
    const int k = e >> 6, m = e & 63;
    const int p = p0 + m;
    float v = 0.f;
    if (p < NPIX && k < KV) {
      const int ci = k / 9, tap = k - 9 * (k / 9);
      const int oh = p / HO, ow = p - (p / HO) * HO;
      const int ih = oh * S + tap / 3 - 1, iw = ow * S + tap % 3 - 1;
      if (ih >= 0 && ih < H && iw >= 0 && iw < H) v = __ldg(xb + ((long long)ci * H + ih) * H + iw);
    }
    split_bf16(v, ahi[m * P + k], amid[m * P + k], alo[m * P + k]);
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
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      uint32_t b0, b1;
      frag_b<P>(b0, b1, bs + n * 8 * P + ks * 16, lane);
      mma16816(acc[n], fl, b0, b1);
      mma16816(acc[n], fm, b0, b1);
      mma16816(acc[n], fh, b0, b1);
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
                                                                   const __nv_bfloat16* __restrict__ wb,
                                                                   long long woff, const float* __restrict__ xin,
                                                                   float* __restrict__ gx) {
  constexpr int HO = H / 2, W2 = H / 2, NCLS = W2 * W2, BPC = (NCLS + 63) / 64, NT = CI / 8, P = kPitch32;
  static_assert(S == 2 && H % 2 == 0, "the data gradient by parity classes is for stride 2");
  static_assert(CI % 8 == 0 && CO % 32 == 0, "channel counts of the data gradient");
  __shared__ __align__(16) __nv_bfloat16 ahi[64 * P], alo[64 * P], bs[CI * P];
  const int b = blockIdx.y, cls = blockIdx.x / BPC, r0 = (blockIdx.x - cls * BPC) * 64;
  const int ph = cls >> 1, pw = cls & 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  const float* gb = gy + (long long)b * CO * HO * HO;
  for (int a = 0; a <= ph; ++a) {
    for (int c = 0; c <= pw; ++c) {
      const int kh = ph ? 2 * a : 1, kw = pw ? 2 * c : 1;
      const int dh = (ph + 1 - kh) >> 1, dw = (pw + 1 - kw) >> 1;  // output row i + dh, column j + dw
      for (int c0 = 0; c0 < CO; c0 += 32) {
        for (int e = threadIdx.x; e < 64 * 32; e += kMmaThreads) {
          const int m = e & 63, cc = e >> 6;
          const int r = r0 + m;
          const int i = r / W2, j = r - (r / W2) * W2;
          const int oh = i + dh, ow = j + dw;
          float v = 0.f;
          if (r < NCLS && oh < HO && ow < HO) v = __ldg(gb + ((long long)(c0 + cc) * HO + oh) * HO + ow);
          const __nv_bfloat16 hi = __float2bfloat16_rn(v);
          ahi[m * P + cc] = hi;
          alo[m * P + cc] = __float2bfloat16_rn(v - __bfloat162float(hi));
        }
        for (int e = threadIdx.x; e < CI * 32; e += kMmaThreads) {
          const int cc = e & 31, ci = e >> 5;
          bs[ci * P + cc] = wb[woff + ((long long)(c0 + cc) * CI + ci) * 9 + kh * 3 + kw];
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          uint32_t fh[4], fl[4];
          frag_a<P>(fh, ahi + warp * 16 * P + ks * 16, lane);
          frag_a<P>(fl, alo + warp * 16 * P + ks * 16, lane);
#pragma unroll
          for (int n = 0; n < NT; ++n) {
            uint32_t b0, b1;
            frag_b<P>(b0, b1, bs + n * 8 * P + ks * 16, lane);
            mma16816(acc[n], fl, b0, b1);
            mma16816(acc[n], fh, b0, b1);
          }
        }
        __syncthreads();
      }
    }
  }
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int q4 = 0; q4 < 4; ++q4) {
    const int r = r0 + warp * 16 + g + (q4 >= 2 ? 8 : 0);
    if (r >= NCLS) continue;
    const int i = r / W2, j = r - (r / W2) * W2;
    const long long pix = (long long)(2 * i + ph) * H + 2 * j + pw;
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      const int ci = n * 8 + 2 * t + (q4 & 1);
      const long long idx = ((long long)b * CI + ci) * H * H + pix;
      gx[idx] = xin[idx] > 0.f ? acc[n][q4] : 0.f;
    }
  }
}

// ------------------------------------------------------------------ weight gradient
// Block (eight warps): 16 input channels, every output channel (warp w takes
// rows 16w .. 16w+15) and all nine taps, over the output pixels of samples
// [s0, s0 + chunk), 32 pixels (in raster order) per stage: g for those pixels
// and the nine taps' input samples for them are staged once and every tap's
// products run from the same g fragments.  The weight gradient feeds only the
// weight update, so g and x are split in two parts (three MMAs: hi hi, hi lo,
// lo hi; 2^-16 of each product left out), unlike the forward pass, whose
// sums decide the ReLU masks.
constexpr int kWgThreads = 256;
constexpr int kWgPix = 32;     // output pixels per stage
constexpr int kWgPitch = 40;   // bfloat16 per staged row (32 used)

template <int CI, int CO, int H, int S>
__global__ void __launch_bounds__(kWgThreads) k_conv_bwd_weight_mma(const float* __restrict__ gy,
                                                                    const float* __restrict__ x, int B, int chunk,
                                                                    float* __restrict__ part) {
  constexpr int HO = (H + S - 1) / S, NPIX = HO * HO, MT = CO / 16;
  static_assert(CO % 16 == 0 && MT <= 8, "output channels of the weight gradient");
  // g: [co][pixel] hi / lo; x: [tap][ci][pixel] hi / lo (pixel contiguous: the k index)
  __shared__ __align__(16) __nv_bfloat16 ghi[CO * kWgPitch], glo[CO * kWgPitch];
  __shared__ __align__(16) __nv_bfloat16 xhi[9 * 16 * kWgPitch], xlo[9 * 16 * kWgPitch];
  const int c0 = blockIdx.x * 16, ck = blockIdx.y;
  const int s0 = ck * chunk, s1 = min(B, s0 + chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  float acc[9][2][4];
#pragma unroll
  for (int q = 0; q < 9; ++q)
#pragma unroll
    for (int n = 0; n < 2; ++n) acc[q][n][0] = acc[q][n][1] = acc[q][n][2] = acc[q][n][3] = 0.f;
  for (int sb = s0; sb < s1; ++sb) {
    const float* gb = gy + (long long)sb * CO * NPIX;
    const float* xb = x + (long long)sb * CI * H * H;
    for (int p0 = 0; p0 < NPIX; p0 += kWgPix) {
      for (int e = threadIdx.x; e < CO * kWgPix; e += kWgThreads) {
        const int co = e / kWgPix, k = e - co * kWgPix, p = p0 + k;
        const float v = p < NPIX ? __ldg(gb + (long long)co * NPIX + p) : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        ghi[co * kWgPitch + k] = hi;
        glo[co * kWgPitch + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
      }
      for (int e = threadIdx.x; e < 9 * 16 * kWgPix; e += kWgThreads) {
        const int k = e % kWgPix, rest = e / kWgPix, c = rest % 16, tap = rest / 16;
        const int p = p0 + k, ci = c0 + c;
        float v = 0.f;
        if (p < NPIX && ci < CI) {
          const int oh = p / HO, ow = p - (p / HO) * HO;
          const int ih = oh * S + tap / 3 - 1, iw = ow * S + tap % 3 - 1;
          if (ih >= 0 && ih < H && iw >= 0 && iw < H) v = __ldg(xb + ((long long)ci * H + ih) * H + iw);
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        xhi[(tap * 16 + c) * kWgPitch + k] = hi;
        xlo[(tap * 16 + c) * kWgPitch + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
      }
      __syncthreads();
      if (warp < MT) {
#pragma unroll
        for (int ks = 0; ks < kWgPix / 16; ++ks) {
          // A (16 output channels x 16 pixels) of this warp's rows, shared by every tap
          const __nv_bfloat16* ah = ghi + warp * 16 * kWgPitch + ks * 16;
          const __nv_bfloat16* al = glo + warp * 16 * kWgPitch + ks * 16;
          uint32_t fh[4], fl[4];
          fh[0] = ld32(ah + g * kWgPitch + 2 * t);
          fh[1] = ld32(ah + (g + 8) * kWgPitch + 2 * t);
          fh[2] = ld32(ah + g * kWgPitch + 2 * t + 8);
          fh[3] = ld32(ah + (g + 8) * kWgPitch + 2 * t + 8);
          fl[0] = ld32(al + g * kWgPitch + 2 * t);
          fl[1] = ld32(al + (g + 8) * kWgPitch + 2 * t);
          fl[2] = ld32(al + g * kWgPitch + 2 * t + 8);
          fl[3] = ld32(al + (g + 8) * kWgPitch + 2 * t + 8);
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
            for (int n = 0; n < 2; ++n) {
              const __nv_bfloat16* bh = xhi + (tap * 16 + n * 8 + g) * kWgPitch + ks * 16 + 2 * t;
              const __nv_bfloat16* bl = xlo + (tap * 16 + n * 8 + g) * kWgPitch + ks * 16 + 2 * t;
              const uint32_t bh0 = ld32(bh), bh1 = ld32(bh + 8), bl0 = ld32(bl), bl1 = ld32(bl + 8);
              mma16816(acc[tap][n], fh, bl0, bl1);
              mma16816(acc[tap][n], fl, bh0, bh1);
              mma16816(acc[tap][n], fh, bh0, bh1);
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (warp >= MT) return;
  float* pc = part + (long long)ck * CO * CI * 9;
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
    for (int n = 0; n < 2; ++n) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int co = warp * 16 + g + (q >= 2 ? 8 : 0), ci = c0 + n * 8 + 2 * t + (q & 1);
        if (ci < CI) pc[((long long)co * CI + ci) * 9 + tap] = acc[tap][n][q];
      }
    }
  }
}

// Weight gradient of a layer with 9 CI <= 32 (the first layer): N is
// (ci, tap), n = 9 ci + tap, one 32-wide tile (rows 9 CI .. 31 zero), instead
// of nine taps each padded to 16 channels.  The eight warps are CO / 16 row
// groups x 8 / (CO / 16) pixel slices over 128 output pixels per stage; the
// slices' sums are added in slice order at the end.
constexpr int kWgPixN = 128;
constexpr int kWgPitchN = 136;  // 68 words: fragment rows g start in banks 4 g

template <int CI, int CO, int H, int S>
__global__ void __launch_bounds__(kWgThreads, 2) k_conv_bwd_weight_mma_n32(const float* __restrict__ gy,
                                                                        const float* __restrict__ x, int B,
                                                                        int chunk, float* __restrict__ part) {
  constexpr int HO = (H + S - 1) / S, NPIX = HO * HO, MT = CO / 16, SL = 8 / MT, PX = kWgPixN / SL;
  constexpr int KV = CI * 9, P = kWgPitchN;
  static_assert(KV <= 32 && CO % 16 == 0 && 8 % MT == 0 && PX % 16 == 0, "first-layer weight gradient");
  constexpr int STAGE_BYTES = (2 * CO + 2 * 32) * P * 2, RED_BYTES = (SL - 1) * MT * 512 * 4;
  __shared__ __align__(16) unsigned char raw[STAGE_BYTES > RED_BYTES ? STAGE_BYTES : RED_BYTES];
  __nv_bfloat16* ghi = reinterpret_cast<__nv_bfloat16*>(raw);
  __nv_bfloat16* glo = ghi + CO * P;
  __nv_bfloat16* xhi = glo + CO * P;
  __nv_bfloat16* xlo = xhi + 32 * P;
  const int ck = blockIdx.y;
  const int s0 = ck * chunk, s1 = min(B, s0 + chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mt = warp % MT, sl = warp / MT;
  const int g = lane >> 2, t = lane & 3;
  for (int e = threadIdx.x; e < (32 - KV) * kWgPixN; e += kWgThreads) {  // the zero rows, once
    const int n = KV + e / kWgPixN, k = e % kWgPixN;
    xhi[n * P + k] = xlo[n * P + k] = __float2bfloat16_rn(0.f);
  }
  float acc[4][4];
#pragma unroll
  for (int n = 0; n < 4; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  for (int sb = s0; sb < s1; ++sb) {
    const float* gb = gy + (long long)sb * CO * NPIX;
    const float* xb = x + (long long)sb * CI * H * H;
    for (int p0 = 0; p0 < NPIX; p0 += kWgPixN) {
      for (int e = threadIdx.x; e < CO * kWgPixN; e += kWgThreads) {
        const int co = e / kWgPixN, k = e % kWgPixN, p = p0 + k;
        const float v = p < NPIX ? __ldg(gb + (long long)co * NPIX + p) : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        ghi[co * P + k] = hi;
        glo[co * P + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
      }
      for (int e = threadIdx.x; e < KV * kWgPixN; e += kWgThreads) {
        const int n = e / kWgPixN, k = e % kWgPixN, p = p0 + k;
        const int ci = n / 9, tap = n - 9 * (n / 9);
        float v = 0.f;
        if (p < NPIX) {
          const int oh = p / HO, ow = p - (p / HO) * HO;
          const int ih = oh * S + tap / 3 - 1, iw = ow * S + tap % 3 - 1;
          if (ih >= 0 && ih < H && iw >= 0 && iw < H) v = __ldg(xb + ((long long)ci * H + ih) * H + iw);
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        xhi[n * P + k] = hi;
        xlo[n * P + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
      }
      __syncthreads();
#pragma unroll
      for (int ks = 0; ks < PX / 16; ++ks) {
        const int k0 = sl * PX + ks * 16;
        uint32_t fh[4], fl[4];
        frag_a<P>(fh, ghi + mt * 16 * P + k0, lane);
        frag_a<P>(fl, glo + mt * 16 * P + k0, lane);
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          uint32_t bh0, bh1, bl0, bl1;
          frag_b<P>(bh0, bh1, xhi + n * 8 * P + k0, lane);
          frag_b<P>(bl0, bl1, xlo + n * 8 * P + k0, lane);
          mma16816(acc[n], fh, bl0, bl1);
          mma16816(acc[n], fl, bh0, bh1);
          mma16816(acc[n], fh, bh0, bh1);
        }
      }
      __syncthreads();
    }
  }
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

// grad[woff + i] = sum over chunks of part[chunk][i], in chunk order.
__global__ void k_reduce_chunks(const float* __restrict__ part, int chunks, long long n, long long woff,
                                float* __restrict__ grad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int c = 0; c < chunks; ++c) s += part[(long long)c * n + i];
  grad[woff + i] = s;
}

// Bias gradient: db[co] = sum over samples and pixels of g[b][co][p], in two
// fixed-order passes: blocks (co, sample chunk) reduce their samples' pixels
// with a fixed tree into part[co][chunk], then one thread per co adds its
// chunks in order.
constexpr int kBiasChunks = 32;
__global__ void __launch_bounds__(256) k_bias_part(const float* __restrict__ gy, int B, int CO, int NPIX,
                                                   float* __restrict__ part) {
  __shared__ float red[256];
  const int co = blockIdx.x, ck = blockIdx.y;
  const int per = (B + kBiasChunks - 1) / kBiasChunks;
  const int b0 = ck * per, b1 = min(B, b0 + per);
  float s = 0.f;
  for (int b = b0; b < b1; ++b) {
    const float* gc = gy + ((long long)b * CO + co) * NPIX;
    for (int p = threadIdx.x; p < NPIX; p += blockDim.x) s += gc[p];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)co * kBiasChunks + ck] = red[0];
}

__global__ void k_bias_final(const float* __restrict__ part, int CO, long long boff, float* __restrict__ grad) {
  const int co = blockIdx.x * blockDim.x + threadIdx.x;
  if (co >= CO) return;
  float s = 0.f;
  for (int c = 0; c < kBiasChunks; ++c) s += part[(long long)co * kBiasChunks + c];
  grad[boff + co] = s;
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
cudaError_t fwd_layer(const float* x, const __nv_bfloat16* wb, const float* w32, long long woff, long long boff, int B,
                      float* y, cudaStream_t s) {
  constexpr int HO = (H + S - 1) / S;
  dim3 grid((unsigned)((HO * HO + 63) / 64), (unsigned)B);
  const char* name = kFwdName[layer_of<CI, CO, H, S>()];
  if constexpr (CI * 9 <= 32) {
    WO_LAUNCH(name, s, (k_conv_fwd_mma_k32<CI, CO, H, S><<<grid, kMmaThreads, 0, s>>>(x, wb, w32, woff, boff, y)));
  } else {
    WO_LAUNCH(name, s, (k_conv_fwd_mma<CI, CO, H, S><<<grid, kMmaThreads, 0, s>>>(x, wb, w32, woff, boff, y)));
  }
  return cudaGetLastError();
}

template <int CI, int CO, int H, int S>
cudaError_t bwd_layer(const float* gy, const float* xin, const __nv_bfloat16* wb, long long woff, long long boff,
                      int B, float* gx, float* part, size_t part_floats, float* grad, cudaStream_t s) {
  constexpr int HO = (H + S - 1) / S;
  // weight gradient: blocks (16-channel group, sample chunk); chunks so that
  // the grid has about 600 blocks and the partials fit their buffer
  const int per = (CI + 15) / 16;
  int chunks = (608 + per - 1) / per;
  const long long wsz = (long long)CO * CI * 9;
  const long long room = (long long)part_floats - (long long)CO * kBiasChunks;  // bias partials follow
  if ((long long)chunks * wsz > room) chunks = (int)(room / wsz);
  if (chunks > B) chunks = B;
  if (chunks < 1) return cudaErrorInvalidValue;
  const int chunk = (B + chunks - 1) / chunks;
  chunks = (B + chunk - 1) / chunk;
  dim3 gw((unsigned)((CI + 15) / 16), (unsigned)chunks);
  const char* wname = kWgName[layer_of<CI, CO, H, S>()];
  if constexpr (CI * 9 <= 32) {
    WO_LAUNCH(wname, s, (k_conv_bwd_weight_mma_n32<CI, CO, H, S><<<gw, kWgThreads, 0, s>>>(gy, xin, B, chunk,
                                                                                          part)));
  } else {
    WO_LAUNCH(wname, s, (k_conv_bwd_weight_mma<CI, CO, H, S><<<gw, kWgThreads, 0, s>>>(gy, xin, B, chunk, part)));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  WO_LAUNCH("est_wgrad_reduce", s, (k_reduce_chunks<<<(unsigned)((wsz + 255) / 256), 256, 0, s>>>(part, chunks, wsz,
                                                                                                  woff, grad)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the bias partials sit after the weight partials in the scratch
  float* bpart = part + (long long)chunks * wsz;
  if ((long long)chunks * wsz + (long long)CO * kBiasChunks > (long long)part_floats) return cudaErrorInvalidValue;
  WO_LAUNCH("est_bias_grad", s, (k_bias_part<<<dim3((unsigned)CO, (unsigned)kBiasChunks), 256, 0, s>>>(gy, B, CO,
                                                                                                     HO * HO, bpart)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  WO_LAUNCH("est_bias_grad", s, (k_bias_final<<<1, 128, 0, s>>>(bpart, CO, boff, grad)));
  e = cudaGetLastError();
  if (e != cudaSuccess || gx == nullptr) return e;
  if constexpr (CI % 8 == 0 && S == 2) {
    dim3 gd((unsigned)(4 * ((H / 2 * (H / 2) + 63) / 64)), (unsigned)B);
    const char* dname = kDgName[layer_of<CI, CO, H, S>()];
    WO_LAUNCH(dname, s, (k_conv_bwd_data_mma<CI, CO, H, S><<<gd, kMmaThreads, 0, s>>>(gy, wb, woff, xin, gx)));
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// The four layers of the estimator (3->32 stride 1 at 64 x 64, 32->64,
// 64->96, 96->128 stride 2).
cudaError_t est_conv_fwd_mma(int layer, const float* x, const void* wb, const float* w32, long long woff,
                             long long boff, int B, float* y, cudaStream_t s) {
  const __nv_bfloat16* w = (const __nv_bfloat16*)wb;
  switch (layer) {
    case 0: return fwd_layer<3, 32, 64, 1>(x, w, w32, woff, boff, B, y, s);
    case 1: return fwd_layer<32, 64, 64, 2>(x, w, w32, woff, boff, B, y, s);
    case 2: return fwd_layer<64, 96, 32, 2>(x, w, w32, woff, boff, B, y, s);
    case 3: return fwd_layer<96, 128, 16, 2>(x, w, w32, woff, boff, B, y, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t est_conv_bwd_mma(int layer, const float* gy, const float* xin, const void* wb, long long woff,
                             long long boff, int B, float* gx, float* part, size_t part_floats, float* grad,
                             cudaStream_t s) {
  const __nv_bfloat16* w = (const __nv_bfloat16*)wb;
  switch (layer) {
    case 0: return bwd_layer<3, 32, 64, 1>(gy, xin, w, woff, boff, B, nullptr, part, part_floats, grad, s);
    case 1: return bwd_layer<32, 64, 64, 2>(gy, xin, w, woff, boff, B, gx, part, part_floats, grad, s);
    case 2: return bwd_layer<64, 96, 32, 2>(gy, xin, w, woff, boff, B, gx, part, part_floats, grad, s);
    case 3: return bwd_layer<96, 128, 16, 2>(gy, xin, w, woff, boff, B, gx, part, part_floats, grad, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wo

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
//                M = co, N = ci (one tap per block), K = (b, p)
// The weights are bfloat16 (exact operands).  Activations and gradients are
// float32; each is split into three bfloat16 parts, v = hi + mid + lo, each
// the bfloat16 rounding of what the previous ones leave (|v - hi - mid - lo|
// <= 2^-26 |v|, below float32 rounding), so that the products keep float32
// accuracy: x w = hi w + mid w + lo w (three MMAs), and in the weight
// gradient g x = the six products of parts whose orders add up to at most 2
// (hi hi, hi mid, mid hi, hi lo, lo hi, mid mid; the rest is below 2^-24).
// Products of bfloat16 values are exact in float32, so the only roundings
// are the float32 sums'.  (With two parts the splits alone leave 2^-17 of
// each product, enough to flip the ReLU masks of near-zero activations.)
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

// A fragment of the 16 x 16 tile whose row 0 is at `s` (pitch kPitch).
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const __nv_bfloat16* s, int lane) {
  const int g = lane >> 2, t = lane & 3;
  a[0] = ld32(s + g * kPitch + 2 * t);
  a[1] = ld32(s + (g + 8) * kPitch + 2 * t);
  a[2] = ld32(s + g * kPitch + 2 * t + 8);
  a[3] = ld32(s + (g + 8) * kPitch + 2 * t + 8);
}

// B fragment of the 8 columns whose column 0 (k contiguous) is at `s`.
__device__ __forceinline__ void frag_b(uint32_t& b0, uint32_t& b1, const __nv_bfloat16* s, int lane) {
  const int g = lane >> 2, t = lane & 3;
  b0 = ld32(s + g * kPitch + 2 * t);
  b1 = ld32(s + g * kPitch + 2 * t + 8);
}

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

// ------------------------------------------------------------------ data gradient
// Block: 64 input pixels of one sample x all CI.  g is the gradient at the
// layer's output (already masked by its ReLU); the result is masked by the
// ReLU of the layer's input (xin > 0).
template <int CI, int CO, int H, int S>
__global__ void __launch_bounds__(kMmaThreads) k_conv_bwd_data_mma(const float* __restrict__ gy,
                                                                   const __nv_bfloat16* __restrict__ wb,
                                                                   long long woff, const float* __restrict__ xin,
                                                                   float* __restrict__ gx) {
  constexpr int HO = (H + S - 1) / S, NPIX = H * H, NT = CI / 8;
  static_assert(CI % 8 == 0 && CO % 16 == 0, "channel counts of the data gradient");
  __shared__ __align__(16) __nv_bfloat16 ahi[64 * kPitch], amid[64 * kPitch], alo[64 * kPitch], bs[CI * kPitch];
  const int b = blockIdx.y, p0 = blockIdx.x * 64;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  const float* gb = gy + (long long)b * CO * HO * HO;
  for (int tap = 0; tap < 9; ++tap) {
    const int kh = tap / 3, kw = tap % 3;
    for (int c0 = 0; c0 < CO; c0 += 16) {
      // A: 64 input pixels x 16 output channels: g at the output pixel this tap maps the input pixel to
      for (int e = threadIdx.x; e < 64 * 16; e += kMmaThreads) {
        const int c = e >> 6, m = e & 63;
        const int q = p0 + m;
        float v = 0.f;
        if (q < NPIX) {
          const int ih = q / H, iw = q - (q / H) * H;
          const int th = ih + 1 - kh, tw = iw + 1 - kw;
          if (th >= 0 && tw >= 0 && th % S == 0 && tw % S == 0) {
            const int oh = th / S, ow = tw / S;
            if (oh < HO && ow < HO) v = __ldg(gb + ((long long)(c0 + c) * HO + oh) * HO + ow);
          }
        }
        split_bf16(v, ahi[m * kPitch + c], amid[m * kPitch + c], alo[m * kPitch + c]);
      }
      // B: 16 output channels x CI weights w[co][ci][tap]
      for (int e = threadIdx.x; e < CI * 16; e += kMmaThreads) {
        const int ci = e >> 4, c = e & 15;
        bs[ci * kPitch + c] = wb[woff + ((long long)(c0 + c) * CI + ci) * 9 + tap];
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
#pragma unroll
  for (int n = 0; n < NT; ++n) {
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      const int q = p0 + warp * 16 + g + (q4 >= 2 ? 8 : 0), ci = n * 8 + 2 * t + (q4 & 1);
      if (q < NPIX) {
        const long long i = ((long long)b * CI + ci) * NPIX + q;
        gx[i] = xin[i] > 0.f ? acc[n][q4] : 0.f;
      }
    }
  }
}

// ------------------------------------------------------------------ weight gradient
// Block: one tap, 16 input channels, all CO, over the pixels of samples
// [s0, s0 + chunk).  Warps take the CO / 16 row tiles in turn.  Writes its
// partial sums part[chunk][co][ci][tap] (reduced in a fixed order later).
template <int CI, int CO, int H, int S>
__global__ void __launch_bounds__(kMmaThreads) k_conv_bwd_weight_mma(const float* __restrict__ gy,
                                                                     const float* __restrict__ x, int B, int chunk,
                                                                     float* __restrict__ part) {
  constexpr int HO = (H + S - 1) / S, NPIX = HO * HO, CIP = ceil16(CI), MT = CO / 16;
  constexpr int MW = (MT + 3) / 4;  // row tiles per warp
  static_assert(CO % 16 == 0, "output channels of the weight gradient");
  __shared__ __align__(16) __nv_bfloat16 ahi[CO * kPitch], amid[CO * kPitch], alo[CO * kPitch], bhi[16 * kPitch],
      bmid[16 * kPitch], blo[16 * kPitch];
  const int tap = blockIdx.x, c0 = blockIdx.y * 16, ck = blockIdx.z;
  const int kh = tap / 3, kw = tap % 3;
  const int s0 = ck * chunk, s1 = min(B, s0 + chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[MW][2][4];
#pragma unroll
  for (int i = 0; i < MW; ++i)
#pragma unroll
    for (int n = 0; n < 2; ++n) acc[i][n][0] = acc[i][n][1] = acc[i][n][2] = acc[i][n][3] = 0.f;
  for (int sb = s0; sb < s1; ++sb) {
    const float* gb = gy + (long long)sb * CO * NPIX;
    const float* xb = x + (long long)sb * CI * H * H;
    for (int k0 = 0; k0 < NPIX; k0 += 16) {
      // A: CO x 16 pixels of g
      for (int e = threadIdx.x; e < CO * 16; e += kMmaThreads) {
        const int co = e >> 4, k = e & 15, p = k0 + k;
        const float v = p < NPIX ? __ldg(gb + (long long)co * NPIX + p) : 0.f;
        split_bf16(v, ahi[co * kPitch + k], amid[co * kPitch + k], alo[co * kPitch + k]);
      }
      // B: 16 channels x 16 pixels of x at this tap (n-major)
      for (int e = threadIdx.x; e < 16 * 16; e += kMmaThreads) {
        const int c = e >> 4, k = e & 15, p = k0 + k, ci = c0 + c;
        float v = 0.f;
        if (p < NPIX && ci < CI) {
          const int oh = p / HO, ow = p - (p / HO) * HO;
          const int ih = oh * S + kh - 1, iw = ow * S + kw - 1;
          if (ih >= 0 && ih < H && iw >= 0 && iw < H) v = __ldg(xb + ((long long)ci * H + ih) * H + iw);
        }
        split_bf16(v, bhi[c * kPitch + k], bmid[c * kPitch + k], blo[c * kPitch + k]);
      }
      __syncthreads();
      uint32_t bh[2][2], bm[2][2], bl[2][2];
#pragma unroll
      for (int n = 0; n < 2; ++n) {
        frag_b(bh[n][0], bh[n][1], bhi + n * 8 * kPitch, lane);
        frag_b(bm[n][0], bm[n][1], bmid + n * 8 * kPitch, lane);
        frag_b(bl[n][0], bl[n][1], blo + n * 8 * kPitch, lane);
      }
#pragma unroll
      for (int i = 0; i < MW; ++i) {
        const int mt = warp + 4 * i;
        if (mt >= MT) break;
        uint32_t ah[4], am[4], al[4];
        frag_a(ah, ahi + mt * 16 * kPitch, lane);
        frag_a(am, amid + mt * 16 * kPitch, lane);
        frag_a(al, alo + mt * 16 * kPitch, lane);
#pragma unroll
        for (int n = 0; n < 2; ++n) {  // smallest terms first
          mma16816(acc[i][n], am, bm[n][0], bm[n][1]);
          mma16816(acc[i][n], ah, bl[n][0], bl[n][1]);
          mma16816(acc[i][n], al, bh[n][0], bh[n][1]);
          mma16816(acc[i][n], ah, bm[n][0], bm[n][1]);
          mma16816(acc[i][n], am, bh[n][0], bh[n][1]);
          mma16816(acc[i][n], ah, bh[n][0], bh[n][1]);
        }
      }
      __syncthreads();
    }
  }
  const int g = lane >> 2, t = lane & 3;
  float* pc = part + (long long)ck * CO * CI * 9;
#pragma unroll
  for (int i = 0; i < MW; ++i) {
    const int mt = warp + 4 * i;
    if (mt >= MT) break;
#pragma unroll
    for (int n = 0; n < 2; ++n) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int co = mt * 16 + g + (q >= 2 ? 8 : 0), ci = c0 + n * 8 + 2 * t + (q & 1);
        if (ci < CI) pc[((long long)co * CI + ci) * 9 + tap] = acc[i][n][q];
      }
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

// Bias gradient: db[co] = sum over samples and pixels of g[b][co][p] (one
// block per co; a fixed tree per block).
__global__ void __launch_bounds__(256) k_bias_grad(const float* __restrict__ gy, int B, int CO, int NPIX,
                                                   long long boff, float* __restrict__ grad) {
  __shared__ float red[256];
  const int co = blockIdx.x;
  float s = 0.f;
  for (long long e = threadIdx.x; e < (long long)B * NPIX; e += blockDim.x) {
    const long long b = e / NPIX, p = e - b * NPIX;
    s += gy[(b * CO + co) * NPIX + p];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) grad[boff + co] = red[0];
}

template <int CI, int CO, int H, int S>
cudaError_t fwd_layer(const float* x, const __nv_bfloat16* wb, const float* w32, long long woff, long long boff, int B,
                      float* y, cudaStream_t s) {
  constexpr int HO = (H + S - 1) / S;
  dim3 grid((unsigned)((HO * HO + 63) / 64), (unsigned)B);
  WO_LAUNCH("est_conv_fwd", s, (k_conv_fwd_mma<CI, CO, H, S><<<grid, kMmaThreads, 0, s>>>(x, wb, w32, woff, boff, y)));
  return cudaGetLastError();
}

template <int CI, int CO, int H, int S>
cudaError_t bwd_layer(const float* gy, const float* xin, const __nv_bfloat16* wb, long long woff, long long boff,
                      int B, float* gx, float* part, size_t part_floats, float* grad, cudaStream_t s) {
  constexpr int HO = (H + S - 1) / S;
  // weight gradient: blocks (tap, 16-channel group, sample chunk); chunks so
  // that the grid has about 2k blocks and the partials fit their buffer
  const int per = 9 * ((CI + 15) / 16);
  int chunks = (2048 + per - 1) / per;
  const long long wsz = (long long)CO * CI * 9;
  if ((long long)chunks * wsz > (long long)part_floats) chunks = (int)(part_floats / wsz);
  if (chunks > B) chunks = B;
  if (chunks < 1) return cudaErrorInvalidValue;
  const int chunk = (B + chunks - 1) / chunks;
  chunks = (B + chunk - 1) / chunk;
  dim3 gw(9u, (unsigned)((CI + 15) / 16), (unsigned)chunks);
  WO_LAUNCH("est_conv_bwd_w", s, (k_conv_bwd_weight_mma<CI, CO, H, S><<<gw, kMmaThreads, 0, s>>>(gy, xin, B, chunk,
                                                                                               part)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  WO_LAUNCH("est_conv_bwd_w", s, (k_reduce_chunks<<<(unsigned)((wsz + 255) / 256), 256, 0, s>>>(part, chunks, wsz, woff,
                                                                                                grad)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  WO_LAUNCH("est_conv_bwd_w", s, (k_bias_grad<<<(unsigned)CO, 256, 0, s>>>(gy, B, CO, HO * HO, boff, grad)));
  e = cudaGetLastError();
  if (e != cudaSuccess || gx == nullptr) return e;
  if constexpr (CI % 8 == 0) {
    dim3 gd((unsigned)((H * H + 63) / 64), (unsigned)B);
    WO_LAUNCH("est_conv_bwd_x", s, (k_conv_bwd_data_mma<CI, CO, H, S><<<gd, kMmaThreads, 0, s>>>(gy, wb, woff, xin,
                                                                                               gx)));
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

// wo_est.cu - the learned optics estimator: spectral features of a tile, a
// small convolutional network with bfloat16 weights and float32 sums
// (inference and training), and the thin-specimen generator that makes its
// training data with the forward model.
//
// Network: four 3x3 convolutions (3->32 stride 1, 32->64, 64->96, 96->128
// stride 2, zero padding 1, ReLU), a global average pool, a linear layer to 4
// outputs.  Parameters live in one flat float32 array (master weights, in the
// order conv1 W, conv1 b, ..., conv4 W, conv4 b, fc W, fc b) and a bfloat16
// copy of it that the kernels read for every weight (biases are read as
// float32).  The outputs are the standardised optics; the caller's scale and
// offset map them to physical units (out = scale * net + offset).
#include <cuda_bf16.h>
#include <stdint.h>

#include "wo_fft.cuh"
#include "wo_internal.h"

namespace wo {

namespace {

constexpr int kSide = 64;
constexpr int kOut = 4;
struct LayerDef {
  int ci, co, stride, hin;
};
constexpr LayerDef kLayers[4] = {{3, 32, 1, 64}, {32, 64, 2, 64}, {64, 96, 2, 32}, {96, 128, 2, 16}};


// Offsets of every parameter array in the flat layout.
struct ParamMap {
  long long w[4], b[4], fw, fb, total;
};
constexpr ParamMap param_map() {
  ParamMap m{};
  long long o = 0;
  for (int l = 0; l < 4; ++l) {
    m.w[l] = o;
    o += (long long)kLayers[l].co * kLayers[l].ci * 9;
    m.b[l] = o;
    o += kLayers[l].co;
  }
  m.fw = o;
  o += (long long)kOut * kLayers[3].co;
  m.fb = o;
  o += kOut;
  m.total = o;
  return m;
}
constexpr ParamMap kMap = param_map();

__device__ __forceinline__ float bf(const __nv_bfloat16* p, long long i) { return __bfloat162float(p[i]); }

// ---------------------------------------------------------------- features
__device__ __forceinline__ int freq_idx(int i, int n) { return (i < (n + 1) / 2) ? i : i - n; }

// One block per (natural row r, tile): radial sums of the plane's power and of
// the cross spectrum with the next plane, over the half spectrum with the
// weights of the conjugate pairs.  Rows >= Z are zero.  ch0 holds the raw
// power until k_feat_norm.
__global__ void __launch_bounds__(256) k_features(const float2* __restrict__ spec, const wo_optics* __restrict__ optics,
                                                  int Z, int Y, int X, float* __restrict__ feat) {
  __shared__ float P[kSide], den[kSide], sx[kSide], sy[kSide];
  const int r = blockIdx.x, t = blockIdx.y;
  const int Xh = X / 2 + 1;
  for (int i = threadIdx.x; i < kSide; i += blockDim.x) P[i] = den[i] = sx[i] = sy[i] = 0.f;
  __syncthreads();
  float* out = feat + (long long)t * 3 * kSide * kSide + (long long)r * kSide;
  if (r < Z) {
    const wo_optics o = optics[t];
    const double cut = 2.0 * o.na_det / o.lambda_um;
    const long long plane = (long long)Y * Xh;
    const float2* Dr = spec + ((long long)t * Z + ((r - Z / 2 + Z) % Z)) * plane;
    const bool nxt = r + 1 < Z;
    const float2* Dn = spec + ((long long)t * Z + ((r + 1 - Z / 2 + Z) % Z)) * plane;
    // the radial bin is decided in float where the value is clear of a bin
    // edge by far more than the float error (relative 3e-7 of at most 64),
    // and by the float64 expression otherwise, so the bins equal the
    // float64 ones (float64 is slow on this part)
    const float inv_py = (float)(1.0 / ((double)Y * o.pixel_um)), inv_px = (float)(1.0 / ((double)X * o.pixel_um));
    const float qscale = (float)((double)kSide / cut);
    for (long long e = threadIdx.x; e < plane; e += blockDim.x) {
      const int y = (int)(e / Xh), x = (int)(e - (long long)y * Xh);
      const float fyf = (float)freq_idx(y, Y) * inv_py, fxf = (float)x * inv_px;
      const float radf = sqrtf(fxf * fxf + fyf * fyf);
      const float q = radf * qscale;
      const float fr = q - floorf(q);
      int b;
      if (fr > 1e-4f && fr < 1.f - 1e-4f) {
        b = (int)floorf(q);
      } else {
        const double fy = (double)freq_idx(y, Y) / ((double)Y * o.pixel_um);
        const double fx = (double)x / ((double)X * o.pixel_um);
        b = (int)floor(sqrt(fx * fx + fy * fy) / cut * kSide);
      }
      if (b >= kSide) continue;
      const float w = (x == 0 || 2 * x == X) ? 1.f : 2.f;
      const float2 dr = Dr[e];
      atomicAdd(&P[b], w * cabs2(dr));
      if (nxt) {
        const float2 dn = Dn[e];
        const float2 c = cmulc(dr, dn);  // dn * conj(dr)
        const float ux = radf > 0.f ? fxf / radf : 0.f, uy = radf > 0.f ? fyf / radf : 0.f;
        atomicAdd(&den[b], w * sqrtf(cabs2(dn) * cabs2(dr)));
        atomicAdd(&sx[b], w * c.y * ux);
        atomicAdd(&sy[b], w * c.y * uy);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kSide; i += blockDim.x) {
    out[i] = P[i];
    out[kSide * kSide + i] = den[i] > 0.f ? sx[i] / den[i] : 0.f;
    out[2 * kSide * kSide + i] = den[i] > 0.f ? sy[i] / den[i] : 0.f;
  }
}

// One block per tile: ch0 = log(1 + P / mean P) over the Z valid rows.
__global__ void __launch_bounds__(256) k_feat_norm(int Z, float* __restrict__ feat) {
  __shared__ double red[256];
  float* f = feat + (long long)blockIdx.x * 3 * kSide * kSide;
  double s = 0.0;
  for (int i = threadIdx.x; i < Z * kSide; i += blockDim.x) s += f[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  const double m = red[0] / (double)(Z * kSide);
  for (int i = threadIdx.x; i < Z * kSide; i += blockDim.x) f[i] = m > 0 ? (float)log1p((double)f[i] / m) : 0.f;
}

// ---------------------------------------------------------------- phantom
// Spheres projected along z onto one plane, as the index increment of a
// plane of thickness dz: sum dn 2 sqrt(r^2 - rho^2) / dz, periodic tile.
__global__ void k_thin_phantom(const float4* __restrict__ par, int S, int Y, int X, float pixel, float dz,
                               float* __restrict__ out) {
  const int t = blockIdx.y;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)Y * X) return;
  const int y = (int)(i / X), x = (int)(i - (long long)y * X);
  const float py = y * pixel, px = x * pixel, ey = Y * pixel, ex = X * pixel;
  float v = 0.f;
  for (int s = 0; s < S; ++s) {
    const float4 q = __ldg(par + (long long)t * S + s);  // cy, cx, radius, dn
    float dy = py - q.x + 0.5f * ey, dx = px - q.y + 0.5f * ex;
    dy -= floorf(dy / ey) * ey;
    dx -= floorf(dx / ex) * ex;
    dy -= 0.5f * ey;
    dx -= 0.5f * ex;
    const float r2 = q.z * q.z - (dy * dy + dx * dx);
    if (r2 > 0.f) v += q.w * 2.f * sqrtf(r2) / dz;
  }
  out[(long long)t * Y * X + i] = v;
}

// ---------------------------------------------------------------- network
// (the convolutions run on the tensor cores: wo_estmma.cu)

// pooled[b][c] = mean y4; out[b][k] = sum_c fw[k][c] pooled[b][c] + fb[k]; one block per sample
__global__ void __launch_bounds__(128) k_head_fwd(const float* __restrict__ y4, const __nv_bfloat16* __restrict__ wb,
                                                  const float* __restrict__ w32, int C, int HW,
                                                  float* __restrict__ pooled, float* __restrict__ out,
                                                  const float* __restrict__ scale, const float* __restrict__ offset,
                                                  float* __restrict__ phys) {
  __shared__ float pl[128];
  const int b = blockIdx.x;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const float* yc = y4 + ((long long)b * C + c) * HW;
    float s = 0.f;
    for (int i = 0; i < HW; ++i) s += yc[i];
    pl[c] = s / (float)HW;
    pooled[(long long)b * C + c] = pl[c];
  }
  __syncthreads();
  if (threadIdx.x < kOut) {
    const int k = threadIdx.x;
    float s = w32[kMap.fb + k];
    for (int c = 0; c < C; ++c) s = fmaf(bf(wb, kMap.fw + (long long)k * C + c), pl[c], s);
    out[(long long)b * kOut + k] = s;
    if (phys) phys[(long long)b * kOut + k] = scale[k] * s + offset[k];
  }
}

// Loss and the head's gradients.  One block: g_out = 2 (out - t) / (B * 4),
// d fc W = g_out^T pooled, d fc b = sum g_out; g_pooled = g_out fc W.
// Head backward, spread over blocks: blocks [0, kOut C / 8) give the linear
// weights' gradients (one warp per weight, lanes over samples, a fixed
// shuffle order), the next B C / 256 blocks the pooled features' gradients
// (one thread each), and the last block the loss and the linear biases'
// gradients (a fixed tree).
constexpr int kHeadWBlocks(int C) { return kOut * C / 8; }
__global__ void __launch_bounds__(256) k_head_bwd(const float* __restrict__ out, const float* __restrict__ target,
                                                  const float* __restrict__ pooled, const __nv_bfloat16* __restrict__ wb,
                                                  int B, int C, float* __restrict__ grad, float* __restrict__ gpool,
                                                  float* __restrict__ loss) {
  const float gs = 2.f / (float)(B * kOut);
  const int nwb = kHeadWBlocks(C), npb = (B * C + 255) / 256;
  if (blockIdx.x < nwb) {
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;  // weight [k][c]
    const int k = i / C, c = i - (i / C) * C;
    float s = 0.f;
    for (int b = lane; b < B; b += 32) s += gs * (out[b * kOut + k] - target[b * kOut + k]) * pooled[(long long)b * C + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) grad[kMap.fw + i] = s;
    return;
  }
  if (blockIdx.x < nwb + npb) {
    const int i = (blockIdx.x - nwb) * 256 + threadIdx.x;
    if (i >= B * C) return;
    const int b = i / C, c = i - (i / C) * C;
    float s = 0.f;
    for (int k = 0; k < kOut; ++k) s += gs * (out[b * kOut + k] - target[b * kOut + k]) * bf(wb, kMap.fw + (long long)k * C + c);
    gpool[i] = s;
    return;
  }
  __shared__ float red[256];
  float l = 0.f;
  for (int i = threadIdx.x; i < B * kOut; i += blockDim.x) {
    const float d = out[i] - target[i];
    l += d * d;
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = red[0] / (float)(B * kOut);
  if (threadIdx.x < kOut) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += gs * (out[b * kOut + threadIdx.x] - target[b * kOut + threadIdx.x]);
    grad[kMap.fb + threadIdx.x] = s;
  }
}

// Gradient at the last conv layer's output from the pooled gradient,
// masked by its ReLU: g[b][c][i] = gpool[b][c] / HW where y > 0.
__global__ void k_unpool(const float* __restrict__ gpool, const float* __restrict__ y, int C, int HW, long long n,
                         float* __restrict__ g) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long bc = i / HW;
  g[i] = y[i] > 0.f ? gpool[bc] / (float)HW : 0.f;
}

// Adam (Kingma and Ba, 2015) on the float32 master weights, then their
// bfloat16 copy (round to nearest even).  step is 1-based.
__global__ void k_adam_flat(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

// standardise physical targets: t = (phys - offset) / scale
__global__ void k_standardise(const float* __restrict__ phys, const float* __restrict__ scale,
                              const float* __restrict__ offset, int n, float* __restrict__ t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * kOut) t[i] = (phys[i] - offset[i % kOut]) / scale[i % kOut];
}

// Workspace layout for a batch.
struct EstWs {
  size_t act[5], out, pooled, gpool, gA, gB, grad, target, scale, part, wt, total;
  size_t part_floats;  // partial weight gradients of the tensor-core kernels
};

// Floats of the per-chunk partial weight gradients (the largest layer's need:
// about 600 blocks of 16 input channels, at most one chunk per sample).
size_t est_part_floats(int B) {
  size_t m = 0;
  for (int l = 0; l < 4; ++l) {
    const int per = (kLayers[l].ci + 15) / 16;
    long long chunks = (608 + per - 1) / per;
    if (chunks > B) chunks = B;
    const size_t need = (size_t)chunks * kLayers[l].co * ((size_t)kLayers[l].ci * 9 + 1);  // weights, bias
    m = need > m ? need : m;
  }
  return m;
}
size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
EstWs est_ws(int B) {
  EstWs L{};
  size_t o = 0;
  const size_t sizes[5] = {(size_t)B * 3 * kSide * kSide, (size_t)B * 32 * 64 * 64, (size_t)B * 64 * 32 * 32,
                           (size_t)B * 96 * 16 * 16, (size_t)B * 128 * 8 * 8};
  L.act[0] = 0;  // the caller's features are read in place
  for (int i = 1; i < 5; ++i) {
    L.act[i] = o;
    o += al(sizes[i] * sizeof(float));
  }
  L.out = o; o += al((size_t)B * kOut * sizeof(float));
  L.pooled = o; o += al((size_t)B * 128 * sizeof(float));
  L.gpool = o; o += al((size_t)B * 128 * sizeof(float));
  L.gA = o; o += al(sizes[1] * sizeof(float));
  L.gB = o; o += al(sizes[1] * sizeof(float));
  L.grad = o; o += al((size_t)kMap.total * sizeof(float));
  L.target = o; o += al((size_t)B * kOut * sizeof(float));
  L.scale = o; o += al(2 * kOut * sizeof(float));
  L.part_floats = est_part_floats(B);
  L.part = o; o += al(L.part_floats * sizeof(float));
  L.wt = o; o += al(est_conv_prep_elems() * 2);  // bfloat16
  L.total = o;
  return L;
}

cudaError_t net_forward(const __nv_bfloat16* wb, const float* w32, const float* feat, int B, char* ws, const EstWs& L,
                        cudaStream_t s, const float* scale, const float* offset, float* phys) {
  const float* x = feat;
  void* wt = ws + L.wt;
  cudaError_t e = est_conv_prep(wb, kMap.w, wt, s);
  if (e != cudaSuccess) return e;
  for (int l = 0; l < 4; ++l) {
    float* y = (float*)(ws + L.act[l + 1]);
    e = est_conv_fwd_mma(l, x, wb, wt, w32, kMap.w[l], kMap.b[l], B, y, s);
    if (e != cudaSuccess) return e;
    x = y;
  }
  WO_LAUNCH("est_head_fwd", s, (k_head_fwd<<<(unsigned)B, 128, 0, s>>>(x, wb, w32, 128, 64, (float*)(ws + L.pooled),
                                                                       (float*)(ws + L.out), scale, offset, phys)));
  return cudaGetLastError();
}

cudaError_t net_backward(const __nv_bfloat16* wb, const float* w32, const float* feat, const float* target, int B,
                         char* ws, const EstWs& L, float* grad, float* loss, cudaStream_t s) {
  cudaError_t e = net_forward(wb, w32, feat, B, ws, L, s, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(grad, 0, (size_t)kMap.total * sizeof(float), s);
  if (e != cudaSuccess) return e;
  const unsigned head_blocks = (unsigned)(kHeadWBlocks(128) + (B * 128 + 255) / 256 + 1);
  WO_LAUNCH("est_head_bwd", s, (k_head_bwd<<<head_blocks, 256, 0, s>>>((float*)(ws + L.out), target,
                                                                       (float*)(ws + L.pooled), wb, B, 128, grad,
                                                                       (float*)(ws + L.gpool), loss)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  float* g = (float*)(ws + L.gA);
  float* gnext = (float*)(ws + L.gB);
  const long long n4 = (long long)B * 128 * 64;
  WO_LAUNCH("est_unpool", s, (k_unpool<<<(unsigned)((n4 + 255) / 256), 256, 0, s>>>((float*)(ws + L.gpool),
                                                                                     (float*)(ws + L.act[4]), 128, 64,
                                                                                     n4, g)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int l = 3; l >= 0; --l) {
    const float* xin = l == 0 ? feat : (const float*)(ws + L.act[l]);
    // weight and bias gradients, then (below the first layer) the gradient at
    // the layer's input, masked by the ReLU that produced it
    e = est_conv_bwd_mma(l, g, xin, ws + L.wt, kMap.w[l], kMap.b[l], B, l == 0 ? nullptr : gnext, (float*)(ws + L.part),
                         L.part_floats, grad, s);
    if (e != cudaSuccess) return e;
    if (l == 0) break;
    float* tmp = g;
    g = gnext;
    gnext = tmp;
  }
  return cudaSuccess;
}

}  // namespace

size_t est_param_count() { return (size_t)kMap.total; }
size_t est_workspace_bytes(int B) { return est_ws(B).total; }

cudaError_t est_features(const float2* spec, const wo_optics* optics, int n, int Z, int Y, int X, float* feat,
                         cudaStream_t s) {
  dim3 grid((unsigned)kSide, (unsigned)n);
  WO_LAUNCH("est_features", s, (k_features<<<grid, 256, 0, s>>>(spec, optics, Z, Y, X, feat)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  WO_LAUNCH("est_feat_norm", s, (k_feat_norm<<<(unsigned)n, 256, 0, s>>>(Z, feat)));
  return cudaGetLastError();
}

cudaError_t est_thin_phantom(const float4* par, int n, int S, int Y, int X, float pixel, float dz, float* out,
                             cudaStream_t s) {
  dim3 grid((unsigned)(((long long)Y * X + 255) / 256), (unsigned)n);
  WO_LAUNCH("thin_phantom", s, (k_thin_phantom<<<grid, 256, 0, s>>>(par, S, Y, X, pixel, dz, out)));
  return cudaGetLastError();
}

cudaError_t est_to_bf16(const float* w, void* wb, cudaStream_t s) {
  const long long n = kMap.total;
  WO_LAUNCH("est_to_bf16", s, (k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, (__nv_bfloat16*)wb, n)));
  return cudaGetLastError();
}

cudaError_t est_forward(const void* wb, const float* w32, const float* feat, int B, const float* h_scale,
                        const float* h_offset, float* phys, void* ws, cudaStream_t s) {
  const EstWs L = est_ws(B);
  char* w = (char*)ws;
  float* sc = (float*)(w + L.scale);
  float hv[2 * kOut];
  for (int k = 0; k < kOut; ++k) {
    hv[k] = h_scale[k];
    hv[kOut + k] = h_offset[k];
  }
  cudaError_t e = cudaMemcpyAsync(sc, hv, sizeof(hv), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return net_forward((const __nv_bfloat16*)wb, w32, feat, B, w, L, s, sc, sc + kOut, phys);
}

cudaError_t est_backward(const void* wb, const float* w32, const float* feat, const float* phys_target, int B,
                         const float* h_scale, const float* h_offset, float* grad, float* loss, void* ws,
                         cudaStream_t s) {
  const EstWs L = est_ws(B);
  char* w = (char*)ws;
  float* sc = (float*)(w + L.scale);
  float hv[2 * kOut];
  for (int k = 0; k < kOut; ++k) {
    hv[k] = h_scale[k];
    hv[kOut + k] = h_offset[k];
  }
  cudaError_t e = cudaMemcpyAsync(sc, hv, sizeof(hv), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  float* t = (float*)(w + L.target);
  WO_LAUNCH("est_standardise", s, (k_standardise<<<(unsigned)((B * kOut + 255) / 256), 256, 0, s>>>(phys_target, sc,
                                                                                                  sc + kOut, B, t)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return net_backward((const __nv_bfloat16*)wb, w32, feat, t, B, w, L, grad ? grad : (float*)(w + L.grad), loss, s);
}

cudaError_t est_adam(float* w32, void* wb, const float* grad, float* m, float* v, int step, float lr, float b1,
                     float b2, float eps, cudaStream_t s) {
  const long long n = kMap.total;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  WO_LAUNCH("est_adam", s, (k_adam_flat<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w32, (__nv_bfloat16*)wb, grad, m,
                                                                                    v, n, lr, b1, b2, eps, c1, c2)));
  return cudaGetLastError();
}

float* est_grad_buffer(void* ws, int B) { return (float*)((char*)ws + est_ws(B).grad); }

}  // namespace wo

using namespace wo;

namespace {
bool a16(const void* p) { return p && (((uintptr_t)p) & 15u) == 0; }
bool a8(const void* p) { return p && (((uintptr_t)p) & 7u) == 0; }
wo_status cs(cudaError_t e) { return e == cudaSuccess ? WO_OK : WO_ERR_CUDA; }
bool scale_ok(const float* sc, const float* off) {
  if (!sc || !off) return false;
  for (int k = 0; k < 4; ++k)
    if (!(sc[k] != 0.f) || !isfinite(sc[k]) || !isfinite(off[k])) return false;
  return true;
}
}  // namespace

extern "C" {

size_t wo_est_param_count(void) { return est_param_count(); }

size_t wo_est_workspace_bytes(int batch) {
  if (batch < 1 || batch > 4096) return 0;
  return est_workspace_bytes(batch);
}

size_t wo_est_activation_offset(int batch, int layer) {
  if (batch < 1 || batch > 4096 || layer < 1 || layer > 4) return 0;
  return est_ws(batch).act[layer];
}

wo_status wo_est_sync_bf16(const float* d_w32, void* d_wbf16, wo_stream stream) {
  if (!a16(d_w32) || !a16(d_wbf16)) return WO_ERR_ARG;
  return cs(est_to_bf16(d_w32, d_wbf16, (cudaStream_t)stream));
}

wo_status wo_est_forward(const void* d_wbf16, const float* d_w32, const float* d_feat, int batch,
                         const float* h_scale, const float* h_offset, float* d_out, void* d_ws, size_t ws_bytes,
                         wo_stream stream) {
  if (batch < 1 || batch > 4096) return WO_ERR_ARG;
  if (!a16(d_wbf16) || !a16(d_w32) || !a16(d_feat) || !a16(d_out) || !a16(d_ws)) return WO_ERR_ARG;
  if (!scale_ok(h_scale, h_offset)) return WO_ERR_ARG;
  if (ws_bytes < est_workspace_bytes(batch)) return WO_ERR_WORKSPACE;
  return cs(est_forward(d_wbf16, d_w32, d_feat, batch, h_scale, h_offset, d_out, d_ws, (cudaStream_t)stream));
}

wo_status wo_est_backward(const void* d_wbf16, const float* d_w32, const float* d_feat, const float* d_target,
                          int batch, const float* h_scale, const float* h_offset, float* d_grad, float* d_loss,
                          void* d_ws, size_t ws_bytes, wo_stream stream) {
  if (batch < 1 || batch > 4096) return WO_ERR_ARG;
  if (!a16(d_wbf16) || !a16(d_w32) || !a16(d_feat) || !a16(d_target) || !a16(d_ws)) return WO_ERR_ARG;
  if ((d_grad && !a16(d_grad)) || (d_loss && !a8(d_loss))) return WO_ERR_ARG;
  if (!scale_ok(h_scale, h_offset)) return WO_ERR_ARG;
  if (ws_bytes < est_workspace_bytes(batch)) return WO_ERR_WORKSPACE;
  return cs(est_backward(d_wbf16, d_w32, d_feat, d_target, batch, h_scale, h_offset, d_grad, d_loss, d_ws,
                         (cudaStream_t)stream));
}

wo_status wo_est_train_step(float* d_w32, void* d_wbf16, float* d_m, float* d_v, const float* d_feat,
                            const float* d_target, int batch, const float* h_scale, const float* h_offset, int step,
                            float lr, float* d_loss, void* d_ws, size_t ws_bytes, wo_stream stream) {
  if (step < 1 || !(lr >= 0.f) || !isfinite(lr)) return WO_ERR_ARG;
  if (!a16(d_m) || !a16(d_v)) return WO_ERR_ARG;
  wo_status st = wo_est_backward(d_wbf16, d_w32, d_feat, d_target, batch, h_scale, h_offset, nullptr, d_loss, d_ws,
                                 ws_bytes, stream);
  if (st != WO_OK) return st;
  return cs(est_adam(d_w32, d_wbf16, est_grad_buffer(d_ws, batch), d_m, d_v, step, lr, 0.9f, 0.999f, 1e-8f,
                     (cudaStream_t)stream));
}

wo_status wo_est_features(const void* d_spec, const wo_optics* d_optics, int n_tiles, int Z, int Y, int X,
                          float* d_feat, wo_stream stream) {
  if (n_tiles < 1 || n_tiles > 65535 || Z < 2 || Z > 64 || Y < 2 || X < 2 || (X % 2)) return WO_ERR_SHAPE;
  if (!a16(d_spec) || !a8(d_optics) || !a16(d_feat)) return WO_ERR_ARG;
  return cs(est_features((const float2*)d_spec, d_optics, n_tiles, Z, Y, X, d_feat, (cudaStream_t)stream));
}

wo_status wo_thin_phantom(const float* d_params, int n_tiles, int n_spheres, int Y, int X, double pixel_um,
                          double z_step_um, float* d_out, wo_stream stream) {
  if (n_tiles < 1 || n_tiles > 65535 || n_spheres < 0 || Y < 1 || X < 1) return WO_ERR_SHAPE;
  if (!(pixel_um > 0) || !(z_step_um > 0)) return WO_ERR_ARG;
  if (!a16(d_params) || !a16(d_out)) return WO_ERR_ARG;
  return cs(est_thin_phantom((const float4*)d_params, n_tiles, n_spheres, Y, X, (float)pixel_um, (float)z_step_um,
                             d_out, (cudaStream_t)stream));
}

}  // extern "C"

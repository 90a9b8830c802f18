// wo_rows.cu - transforms along the contiguous x axis (real <-> half spectrum).
//
// A real row x[0..2N) is read as N complex samples z[n] = x[2n] + i x[2n+1]
// (a plain float2 load), transformed with a length-N complex FFT, and split
// into the N+1 bins of the real transform:
//   X[k] = (Z[k] + Z*[N-k])/2 - (i/2) e^{-2 pi i k/2N} (Z[k] - Z*[N-k]).
// The inverse rebuilds Z[k] = A + iB with A = (X[k] + X*[N-k])/2 and
// B = (X[k] - X*[N-k]) e^{+2 pi i k/2N}/2 and applies a length-N inverse FFT.
// B rows per CTA sit in shared memory with an odd pitch (N | 1) so the
// stage accesses (row index fastest across a warp) are bank-conflict free;
// global loads and stores run along the rows and are fully coalesced.
#include "wo_fft.cuh"
#include "wo_internal.h"

namespace wo {

// Per-row background constant (mode 1: the channel's value; mode 2: the
// first sample of the row's (tile, channel) block), one per row of the CTA.
__device__ __forceinline__ void row_constants(float* sc, const float* in, long long row0, long long nrows,
                                              int B, int N, const RowBg& bg) {
  if (threadIdx.x < B) {
    const long long row = row0 + threadIdx.x;
    float c = 0.f;
    if (row < nrows && bg.mode == 1) c = bg.v[(row / bg.rows_per_block) % bg.nchan];
    if (row < nrows && bg.mode == 2) c = in[(row / bg.rows_per_block) * bg.rows_per_block * (2LL * N)];
    sc[threadIdx.x] = c;
  }
}

template <int N>
__global__ void __launch_bounds__(RowGeom<N>::NT, RowGeom<N>::MINB)
    k_rows_r2c(const float* __restrict__ in, float2* __restrict__ out, long long nrows, RowBg bg) {
  using G = RowGeom<N>;
  constexpr int B = G::B, LD = G::LD, NT = G::NT;
  extern __shared__ float2 sm[];
  float2* buf = sm;
  float2* tw = sm + B * LD;                            // exp(-2 pi i m / 2N), m in [0, 2N)
  float* sc = reinterpret_cast<float*>(tw + 2 * N);   // [B] background per row
  const long long row0 = (long long)blockIdx.x * B;
  for (int e = threadIdx.x; e < B * N; e += NT) {
    const int b = e / N, n = e - (e / N) * N;
    const long long row = row0 + b;
    const bool ok = row < nrows;
    cp_async8(buf + b * LD + n, in + (ok ? row * (2LL * N) + 2 * n : 0), ok);
  }
  make_twiddles<2 * N>(tw);
  row_constants(sc, in, row0, nrows, B, N, bg);
  cp_async_wait_all();
  __syncthreads();
  if (bg.mode != 0) {
    for (int e = threadIdx.x; e < B * N; e += NT) {
      const int b = e / N, n = e - (e / N) * N;
      const float c = sc[b];
      float2 v = buf[b * LD + n];
      v.x -= c;
      v.y -= c;
      buf[b * LD + n] = v;
    }
    __syncthreads();
  }
  fft_smem<N, B, NT, false, 2>(buf, 1, LD, tw);
  for (int e = threadIdx.x; e < B * (N + 1); e += NT) {
    const int b = e / (N + 1), k = e - (e / (N + 1)) * (N + 1);
    const long long row = row0 + b;
    if (row >= nrows) continue;
    const float2 zk = buf[b * LD + (k == N ? 0 : k)];
    const float2 zc = cconj(buf[b * LD + (k == 0 ? 0 : N - k)]);
    const float2 s = cadd(zk, zc);
    const float2 u = cmul(tw[k], csub(zk, zc));
    out[row * (N + 1) + k] = make_float2(0.5f * (s.x + u.y), 0.5f * (s.y - u.x));
  }
}

template <int N>
__global__ void __launch_bounds__(RowGeom<N>::NT, RowGeom<N>::MINB)
    k_rows_c2r(const float2* __restrict__ in, float* __restrict__ out, long long nrows, float scale,
               RowBg bg) {
  using G = RowGeom<N>;
  constexpr int B = G::B, LD = G::LD, LD2 = G::LD2, NT = G::NT;
  extern __shared__ float2 sm[];
  float2* raw = sm;                                     // [B][LD2] input half spectra
  float2* buf = sm + B * LD2;                           // [B][LD] packed complex rows
  float2* tw = buf + B * LD;
  float* sc = reinterpret_cast<float*>(tw + 2 * N);
  const long long row0 = (long long)blockIdx.x * B;
  for (int e = threadIdx.x; e < B * (N + 1); e += NT) {
    const int b = e / (N + 1), k = e - (e / (N + 1)) * (N + 1);
    const long long row = row0 + b;
    const bool ok = row < nrows;
    cp_async8(raw + b * LD2 + k, in + (ok ? row * (N + 1) + k : 0), ok);
  }
  make_twiddles<2 * N>(tw);
  if (threadIdx.x < B) {
    const long long row = row0 + threadIdx.x;
    sc[threadIdx.x] = (row < nrows && bg.mode == 1) ? bg.v[(row / bg.rows_per_block) % bg.nchan] : 0.f;
  }
  cp_async_wait_all();
  __syncthreads();
  for (int e = threadIdx.x; e < B * N; e += NT) {
    const int b = e / N, k = e - (e / N) * N;
    const float2 xk = raw[b * LD2 + k];
    const float2 xc = cconj(raw[b * LD2 + N - k]);
    const float2 a = make_float2(0.5f * (xk.x + xc.x), 0.5f * (xk.y + xc.y));
    const float2 bb = cmul(make_float2(0.5f * (xk.x - xc.x), 0.5f * (xk.y - xc.y)), cconj(tw[k]));
    buf[b * LD + k] = make_float2(a.x - bb.y, a.y + bb.x);
  }
  __syncthreads();
  fft_smem<N, B, NT, true, 2>(buf, 1, LD, tw);
  for (int e = threadIdx.x; e < B * N; e += NT) {
    const int b = e / N, n = e - (e / N) * N;
    const long long row = row0 + b;
    if (row >= nrows) continue;
    const float c = sc[b];
    const float2 v = buf[b * LD + n];
    reinterpret_cast<float2*>(out + row * (2LL * N))[n] = make_float2(v.x * scale + c, v.y * scale + c);
  }
}

template <int N>
static size_t rows_smem_r2c() {
  return ((size_t)RowGeom<N>::B * RowGeom<N>::LD + 2 * (size_t)N) * sizeof(float2) + RowGeom<N>::B * sizeof(float);
}

template <int N>
static size_t rows_smem_c2r() {
  return ((size_t)RowGeom<N>::B * (RowGeom<N>::LD + RowGeom<N>::LD2) + 2 * (size_t)N) * sizeof(float2) +
         RowGeom<N>::B * sizeof(float);
}

template <int N>
static cudaError_t launch_r2c(const float* in, float2* out, long long nrows, RowBg bg, cudaStream_t s) {
  const size_t smem = rows_smem_r2c<N>();
  static cudaError_t attr = allow_smem(k_rows_r2c<N>, smem);
  if (attr != cudaSuccess) return attr;
  const long long blocks = (nrows + RowGeom<N>::B - 1) / RowGeom<N>::B;
  WO_LAUNCH("rows_r2c", s, (k_rows_r2c<N><<<(unsigned)blocks, RowGeom<N>::NT, smem, s>>>(in, out, nrows, bg)));
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_c2r(const float2* in, float* out, long long nrows, float scale, RowBg bg,
                              cudaStream_t s) {
  const size_t smem = rows_smem_c2r<N>();
  static cudaError_t attr = allow_smem(k_rows_c2r<N>, smem);
  if (attr != cudaSuccess) return attr;
  const long long blocks = (nrows + RowGeom<N>::B - 1) / RowGeom<N>::B;
  WO_LAUNCH("rows_c2r", s,
            (k_rows_c2r<N><<<(unsigned)blocks, RowGeom<N>::NT, smem, s>>>(in, out, nrows, scale, bg)));
  return cudaGetLastError();
}

cudaError_t rows_r2c(int N, const float* in, float2* out, long long nrows, RowBg bg, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  switch (N) {
#define WO_CASE(n) \
  case n:          \
    return launch_r2c<n>(in, out, nrows, bg, s);
    WO_CASE(1) WO_CASE(2) WO_CASE(3) WO_CASE(4) WO_CASE(6) WO_CASE(8) WO_CASE(12) WO_CASE(16)
    WO_CASE(24) WO_CASE(32) WO_CASE(48) WO_CASE(64) WO_CASE(96) WO_CASE(128) WO_CASE(192)
    WO_CASE(256) WO_CASE(384) WO_CASE(512) WO_CASE(768) WO_CASE(1024)
#undef WO_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t rows_c2r(int N, const float2* in, float* out, long long nrows, float scale, RowBg bg,
                     cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  switch (N) {
#define WO_CASE(n) \
  case n:          \
    return launch_c2r<n>(in, out, nrows, scale, bg, s);
    WO_CASE(1) WO_CASE(2) WO_CASE(3) WO_CASE(4) WO_CASE(6) WO_CASE(8) WO_CASE(12) WO_CASE(16)
    WO_CASE(24) WO_CASE(32) WO_CASE(48) WO_CASE(64) WO_CASE(96) WO_CASE(128) WO_CASE(192)
    WO_CASE(256) WO_CASE(384) WO_CASE(512) WO_CASE(768) WO_CASE(1024)
#undef WO_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace wo

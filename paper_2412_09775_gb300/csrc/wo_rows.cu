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
    const long long grow = bg.row_offset + row;  // row index in the whole volume set
    float c = 0.f;
    if (row < nrows && bg.mode == 1) c = bg.v[(grow / bg.rows_per_block) % bg.nchan];
    if (row < nrows && bg.mode == 2)
      c = in[((grow / bg.rows_per_block) * bg.rows_per_block - bg.row_offset) * (2LL * N)];
    sc[threadIdx.x] = c;
  }
}

template <int N>
__global__ void __launch_bounds__(RowGeom<N>::NT, RowGeom<N>::MINB)
    k_rows_r2c(const float* __restrict__ in, float2* __restrict__ out, long long nrows, RowBg bg) {
  using G = RowGeom<N>;
  constexpr int B = G::B, P = G::P, NT = G::NT;
  extern __shared__ float2 sm[];
  float2* buf = sm;                                   // [N][P]
  float2* tw = sm + N * P;                            // exp(-2 pi i m / 2N), m in [0, 2N)
  float* sc = reinterpret_cast<float*>(tw + 2 * N);   // [B] background per row
  const long long row0 = (long long)blockIdx.x * B;
  const int rows = (int)min((long long)B, nrows - row0);
  const float2* g = reinterpret_cast<const float2*>(in + row0 * (2LL * N));
  for (int e = threadIdx.x; e < B * N; e += NT) {
    const int b = e / N, n = e - (e / N) * N;
    cp_async8(buf + n * P + b, b < rows ? g + b * N + n : g, b < rows);
  }
  make_twiddles<2 * N>(tw);
  row_constants(sc, in, row0, nrows, B, N, bg);
  cp_async_wait_all();
  __syncthreads();
  if (bg.mode != 0) {
    for (int e = threadIdx.x; e < B * N; e += NT) {
      const int b = e / N, n = e - (e / N) * N;
      const float c = sc[b];
      float2 v = buf[n * P + b];
      v.x -= c;
      v.y -= c;
      buf[n * P + b] = v;
    }
    __syncthreads();
  }
  fft_smem<N, B, NT, false, 2>(buf, P, 1, tw);
  float2* o = out + row0 * (N + 1);
  for (int e = threadIdx.x; e < B * (N + 1); e += NT) {
    const int b = e / (N + 1), k = e - (e / (N + 1)) * (N + 1);
    if (b >= rows) continue;
    const float2 zk = buf[(k == N ? 0 : k) * P + b];
    const float2 zc = cconj(buf[(k == 0 ? 0 : N - k) * P + b]);
    const float2 s = cadd(zk, zc);
    const float2 u = cmul(tw[k], csub(zk, zc));
    o[b * (N + 1) + k] = make_float2(0.5f * (s.x + u.y), 0.5f * (s.y - u.x));
  }
}

// The pre-processing is done in place on pairs (k, N-k): with
// A = (X[k] + X*[N-k])/2 and B = (X[k] - X*[N-k]) e^{+i pi k/N}/2,
// Z[k] = A + iB and Z[N-k] = A* + iB*.
template <int N>
__global__ void __launch_bounds__(RowGeom<N>::NT, RowGeom<N>::MINB)
    k_rows_c2r(const float2* __restrict__ in, float* __restrict__ out, long long nrows, float scale,
               RowBg bg) {
  using G = RowGeom<N>;
  constexpr int B = G::B, P = G::P, NT = G::NT, H = N / 2 + 1;
  extern __shared__ float2 sm[];
  float2* buf = sm;                                   // [N + 1][P]
  float2* tw = sm + (N + 1) * P;
  float* sc = reinterpret_cast<float*>(tw + 2 * N);
  const long long row0 = (long long)blockIdx.x * B;
  const int rows = (int)min((long long)B, nrows - row0);
  const float2* g = in + row0 * (N + 1);
  for (int e = threadIdx.x; e < B * (N + 1); e += NT) {
    const int b = e / (N + 1), k = e - (e / (N + 1)) * (N + 1);
    cp_async8(buf + k * P + b, b < rows ? g + b * (N + 1) + k : g, b < rows);
  }
  make_twiddles<2 * N>(tw);
  if (threadIdx.x < B) {
    const long long row = row0 + threadIdx.x;
    sc[threadIdx.x] =
        (row < nrows && bg.mode == 1) ? bg.v[((bg.row_offset + row) / bg.rows_per_block) % bg.nchan] : 0.f;
  }
  cp_async_wait_all();
  __syncthreads();
  for (int e = threadIdx.x; e < B * H; e += NT) {
    const int b = e / H, k = e - (e / H) * H;
    const float2 xk = buf[k * P + b];
    const float2 xc = cconj(buf[(N - k) * P + b]);
    const float2 a = make_float2(0.5f * (xk.x + xc.x), 0.5f * (xk.y + xc.y));
    const float2 bb = cmul(make_float2(0.5f * (xk.x - xc.x), 0.5f * (xk.y - xc.y)), cconj(tw[k]));
    buf[k * P + b] = make_float2(a.x - bb.y, a.y + bb.x);
    if (k != 0 && 2 * k != N) buf[(N - k) * P + b] = make_float2(a.x + bb.y, -a.y + bb.x);
  }
  __syncthreads();
  fft_smem<N, B, NT, true, 2>(buf, P, 1, tw);
  float2* o = reinterpret_cast<float2*>(out + row0 * (2LL * N));
  for (int e = threadIdx.x; e < B * N; e += NT) {
    const int b = e / N, n = e - (e / N) * N;
    if (b >= rows) continue;
    const float c = sc[b];
    const float2 v = buf[n * P + b];
    o[b * N + n] = make_float2(v.x * scale + c, v.y * scale + c);
  }
}

template <int N>
static size_t rows_smem_r2c() {
  return ((size_t)N * RowGeom<N>::P + 2 * (size_t)N) * sizeof(float2) + RowGeom<N>::B * sizeof(float);
}

template <int N>
static size_t rows_smem_c2r() {
  return ((size_t)(N + 1) * RowGeom<N>::P + 2 * (size_t)N) * sizeof(float2) + RowGeom<N>::B * sizeof(float);
}

template <int N>
static cudaError_t launch_r2c(const float* in, float2* out, long long nrows, RowBg bg, cudaStream_t s) {
  const size_t smem = rows_smem_r2c<N>();
  const cudaError_t attr = allow_smem(k_rows_r2c<N>, smem);
  if (attr != cudaSuccess) return attr;
  const long long blocks = (nrows + RowGeom<N>::B - 1) / RowGeom<N>::B;
  WO_LAUNCH("rows_r2c", s, (k_rows_r2c<N><<<(unsigned)blocks, RowGeom<N>::NT, smem, s>>>(in, out, nrows, bg)));
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_c2r(const float2* in, float* out, long long nrows, float scale, RowBg bg,
                              cudaStream_t s) {
  const size_t smem = rows_smem_c2r<N>();
  const cudaError_t attr = allow_smem(k_rows_c2r<N>, smem);
  if (attr != cudaSuccess) return attr;
  const long long blocks = (nrows + RowGeom<N>::B - 1) / RowGeom<N>::B;
  WO_LAUNCH("rows_c2r", s,
            (k_rows_c2r<N><<<(unsigned)blocks, RowGeom<N>::NT, smem, s>>>(in, out, nrows, scale, bg)));
  return cudaGetLastError();
}

cudaError_t rows_r2c(int N, const float* in, float2* out, long long nrows, RowBg bg, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  if (rows_engine(N) == WO_ENGINE_HYBRID) return rows_r2c_reg(N, in, out, nrows, bg, s);
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
  if (rows_engine(N) == WO_ENGINE_HYBRID) return rows_c2r_reg(N, in, out, nrows, scale, bg, s);
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

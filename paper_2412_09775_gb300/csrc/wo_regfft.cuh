// wo_regfft.cuh - register-resident FFTs of short rows.
//
// A row of N = N1 * T points is held by T consecutive lanes of one warp, lane
// t owning the points p = t + T m (m = 0 .. N1-1) in register m.  A transform
// is the four-step factorisation n = T n1 + t, k = k1 + N1 k2:
//   1. each lane: DFT of length N1 over n1 in registers (Stockham stages),
//   2. multiply by w_N^(t k1),
//   3. transpose through shared memory (the row's own slice; the lanes of a
//      row are one warp's, so __syncwarp suffices),
//   4. each lane: N1/T DFTs of length T over t, for k1 = t + T i.
// The result, point k1 + N1 k2, lands in lane (k1 mod T), register
// i + (N1/T) k2 = (p - t)/T: the same ownership as the input, so transforms
// chain in registers without reordering.  Transforms are unnormalised.
#pragma once
#include "wo_fft.cuh"

namespace wo {

// Twiddles of the in-register stages as compile-time constants.  Their
// lengths NS * R (12, 16 or 24 for the row lengths here) divide 48, so every
// one is a power of w_48 = exp(-2 pi i / 48); the table is evaluated at
// compile time from the Taylor series of cos and sin on [-pi, pi] (30 terms,
// far below double rounding there) and rounded to float.
namespace twc {
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int n = 1; n < 30; ++n) {
    t *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    s += t;
  }
  return s;
}
constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int n = 1; n < 30; ++n) {
    t *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    s += t;
  }
  return s;
}
struct W48 {
  float re[48], im[48];  // exp(-2 pi i m / 48)
};
constexpr W48 make_w48() {
  W48 w{};
  for (int m = 0; m < 48; ++m) {
    const double x = (m <= 24 ? m : m - 48) * (2.0 * kPi / 48.0);
    w.re[m] = (float)taylor_cos(x);
    w.im[m] = (float)(-taylor_sin(x));
  }
  return w;
}
}  // namespace twc
__device__ constexpr twc::W48 kW48 = twc::make_w48();

// a * w_DEN^e (forward) or a * w_DEN^-e (inverse); e and DEN are constants
// once the stage loops are unrolled, so the trivial powers cost nothing.
template <bool INV, int DEN>
__device__ __forceinline__ float2 twiddle_mul(float2 a, int e) {
  static_assert(48 % DEN == 0, "stage length must divide 48");
  const int m = (e % DEN) * (48 / DEN);
  if (m == 0) return a;
  if (m == 24) return make_float2(-a.x, -a.y);
  if (m == 12) return mul_mi<INV>(a);
  if (m == 36) return mul_mi<!INV>(a);
  return cmul(a, make_float2(kW48.re[m], INV ? -kW48.im[m] : kW48.im[m]));
}

// In-register Stockham stages over L points (natural order in and out).
template <int L, int NS, bool INV, int STEP>
__device__ __forceinline__ void reg_stages(float2 (&v)[L], const float2* tw) {
  if constexpr (NS < L) {
    constexpr int R = radix_for(L / NS);
    constexpr int M = L / R;
    float2 o[L];
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const int k = j % NS;
      float2 w[R];
#pragma unroll
      for (int r = 0; r < R; ++r) w[r] = v[j + r * M];
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) w[r] = twiddle_mul<INV, NS * R>(w[r], r * k);
      }
      dftR<R, INV>(w);
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) o[base + r * NS] = w[r];
    }
#pragma unroll
    for (int i = 0; i < L; ++i) v[i] = o[i];
    reg_stages<L, NS * R, INV, STEP>(v, tw);
  }
}

// Two-step row transform, N = N1 * T (T lanes of N1 points; T divides N1
// and 32).  The slice pitch is T mod 16 so that the lane-major writes and the
// column reads of a half-warp fall on distinct 8-byte bank pairs.
template <int N_, int N1>
struct Row2 {
  static constexpr int N = N_, E = N1, T = N / N1;
  static constexpr int NI = N1 / T;  // length-T DFTs per lane in step 4
  static constexpr int LP = N1 + 1;  // lane pitch in the slice
  static constexpr int SLICE = ((T * LP + 15 - T) / 16) * 16 + T;
  static constexpr int TW = 2 * N;   // w_N^m, then w_N^(t k1) at [k1 * T + t]
  static_assert(N1 % T == 0, "each lane needs whole length-T transforms");
  static_assert(T <= 32 && (32 % T) == 0, "a row's lanes must sit in one warp");

  static __device__ __forceinline__ void twiddles(float2* tw) {
    make_twiddles<N>(tw);
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
      const int k1 = e / T, t = e - (e / T) * T;
      float s, c;
      sincospif(2.0f * (float)(t * k1) / (float)N, &s, &c);
      tw[N + e] = make_float2(c, -s);
    }
  }

  template <bool INV>
  static __device__ __forceinline__ void fft(float2 (&v)[E], const float2* tw, float2* S, int t) {
    reg_stages<N1, 1, INV, N / N1>(v, tw);
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) {
      float2 w = tw[N + k1 * T + t];
      if (INV) w.y = -w.y;
      v[k1] = cmul(v[k1], w);
    }
    __syncwarp();  // the previous transform's reads of S are done
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) S[t * LP + k1] = v[k1];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      float2 u[T];
#pragma unroll
      for (int n2 = 0; n2 < T; ++n2) u[n2] = S[n2 * LP + t + T * i];
      reg_stages<T, 1, INV, N / T>(u, tw);
#pragma unroll
      for (int k2 = 0; k2 < T; ++k2) v[i + NI * k2] = u[k2];
    }
  }
};

// 512 points on one warp, 16 per lane (lane l owns p = l + 32 m): Stockham
// passes of radix 16 (from registers), 16 and 2, with two exchanges through a
// slice padded by one element per 16 (index p + p/16), conflict-free for
// every pass's writes and reads.
struct Row512 {
  static constexpr int N = 512, E = 16, T = 32;
  static constexpr int SLICE = N + N / 16;
  static constexpr int TW = N + 256;  // w_512^m, then w_256^(r k) at [r * 16 + k]

  static __device__ __forceinline__ int pad(int p) { return p + (p >> 4); }

  static __device__ __forceinline__ void twiddles(float2* tw) {
    make_twiddles<N>(tw);
    for (int e = threadIdx.x; e < 256; e += blockDim.x) {
      const int r = e >> 4, k = e & 15;
      float s, c;
      sincospif(2.0f * (float)(r * k) / 256.0f, &s, &c);
      tw[N + e] = make_float2(c, -s);
    }
  }

  template <bool INV>
  static __device__ __forceinline__ void fft(float2 (&v)[E], const float2* tw, float2* S, int l) {
    // pass 1 (sub-length 1, radix 16): butterfly l takes points l + 32 r
    reg_stages<16, 1, INV, 32>(v, tw);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) S[pad(16 * l + r)] = v[r];
    __syncwarp();
    // pass 2 (sub-length 16, radix 16): twiddles w_256^(r k), k = l mod 16
    const int k = l & 15;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      v[r] = S[pad(l + 32 * r)];
      if (r > 0) {
        float2 w = tw[N + r * 16 + k];
        if (INV) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    reg_stages<16, 1, INV, 32>(v, tw);
    __syncwarp();
    const int base = (l >> 4) * 256 + k;
#pragma unroll
    for (int r = 0; r < 16; ++r) S[pad(base + 16 * r)] = v[r];
    __syncwarp();
    // pass 3 (sub-length 256, radix 2): butterflies j = l + 32 i, twiddle w_512^j
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = l + 32 * i;
      const float2 a = S[pad(j)];
      float2 w = tw[j];
      if (INV) w.y = -w.y;
      const float2 b = cmul(S[pad(j + 256)], w);
      v[i] = cadd(a, b);
      v[i + 8] = csub(a, b);
    }
  }
};

}  // namespace wo

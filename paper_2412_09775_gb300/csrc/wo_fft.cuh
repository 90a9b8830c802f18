// wo_fft.cuh - shared-memory mixed-radix Stockham FFT engine for sm_103a.
//
// A CTA transforms a batch of B sequences of compile-time length N that sit
// in shared memory; element n of sequence b lives at buf[n*es + b*bs].  Each
// stage is radix 8, 4, 2 or 3 (N = 2^a * 3^b, b <= 1).  A stage loads every
// butterfly input of the thread into registers, synchronises, then applies
// twiddles, the radix-R DFT and writes the self-sorted outputs back in place.
// Threads are mapped with the sequence index b fastest, so a warp touches
// consecutive sequences: with es = B (column tiles) that is one contiguous
// run, and with bs odd (row tiles padded to an odd pitch) the accesses fall
// in distinct banks.
//
// Stockham self-sorting formulation (Govindaraju et al., SC'08): with Ns the
// product of the radices already applied, butterfly j reads x[j + r*N/R],
// multiplies input r by w^(r*k), k = j mod Ns, w = exp(-2 pi i/(Ns*R)), and
// writes output r to y[(j/Ns)*Ns*R + k + r*Ns].
//
// Forward transforms use exp(-2 pi i/N); inverse ones exp(+2 pi i/N) and are
// unnormalised.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace wo {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
  // X1 = v0 + w v1 + w^2 v2, w = exp(-+ 2 pi i / 3) = -1/2 -+ i sqrt(3)/2
  const float kS3 = 0.866025403784438647f;  // sqrt(3)/2
  float2 s = cadd(v[1], v[2]);
  float2 d = csub(v[1], v[2]);
  float2 m = make_float2(v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y);
  float2 t = mul_mi<INV>(make_float2(kS3 * d.x, kS3 * d.y));
  v[0] = cadd(v[0], s);
  v[1] = cadd(m, t);
  v[2] = csub(m, t);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
  float2 t2 = cadd(a1, a3), t3 = mul_mi<INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  const float kR = 0.707106781186547524f;  // 1/sqrt(2)
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // o_k *= w8^k, w8 = exp(-+ i pi / 4)
  if (!INV) {
    o1 = make_float2(kR * (o1.x + o1.y), kR * (o1.y - o1.x));
    o2 = make_float2(o2.y, -o2.x);
    o3 = make_float2(kR * (o3.y - o3.x), -kR * (o3.x + o3.y));
  } else {
    o1 = make_float2(kR * (o1.x - o1.y), kR * (o1.x + o1.y));
    o2 = make_float2(-o2.y, o2.x);
    o3 = make_float2(-kR * (o3.x + o3.y), kR * (o3.x - o3.y));
  }
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <int R, bool INV>
__device__ __forceinline__ void dftR(float2* v) {
  if constexpr (R == 2) dft2<INV>(v);
  else if constexpr (R == 3) dft3<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else dft8<INV>(v);
}

// Radix of the next stage given the remaining length.
__host__ __device__ constexpr int radix_for(int rem) {
  return (rem % 8 == 0) ? 8 : (rem % 4 == 0) ? 4 : (rem % 2 == 0) ? 2 : 3;
}

// Fill tw[m] = exp(-2 pi i m / L) for m in [0, L).
template <int L>
__device__ __forceinline__ void make_twiddles(float2* tw) {
  for (int m = threadIdx.x; m < L; m += blockDim.x) {
    float s, c;
    sincospif(2.0f * (float)m / (float)L, &s, &c);
    tw[m] = make_float2(c, -s);
  }
}

// Shared-memory layouts: the index of element n of sequence s.
struct LinAddr {  // n * es + s * bs
  int es, bs;
  __device__ __forceinline__ int operator()(int n, int s) const { return n * es + s * bs; }
};
// SLOTS groups of S = 2^k sequences (s = slot * S + b), each group stored
// n-major with the sequence index XOR-swizzled by n: index
// slot * (L * S + S) + n * S + (b ^ (n & (S - 1))).  Copies that walk n for a
// fixed sequence and stages that walk the sequences for a fixed n both spread
// over all banks; the extra S elements between groups shift alternate groups
// by half the banks.
template <int S, int L>
struct SwzAddr {
  __device__ __forceinline__ int operator()(int n, int s) const {
    const int slot = s / S, b = s & (S - 1);
    return slot * (L * S + S) + n * S + (b ^ (n & (S - 1)));
  }
};

// One Stockham stage.  The twiddle table holds exp(-2 pi i m / (N*TWS)).
template <int N, int R, int NS, int B, int NT, bool INV, int TWS, class A>
__device__ __forceinline__ void fft_stage_a(float2* buf, A addr, const float2* tw) {
  constexpr int M = N / R;
  constexpr int NB = M * B;
  constexpr int PER = (NB + NT - 1) / NT;
  float2 v[PER][R];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int beta = threadIdx.x + i * NT;
    if ((NB % NT == 0) || beta < NB) {
      const int b = beta % B, j = beta / B;
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = buf[addr(j + r * M, b)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int beta = threadIdx.x + i * NT;
    if ((NB % NT == 0) || beta < NB) {
      const int b = beta % B, j = beta / B;
      const int k = j % NS;
      if constexpr (NS > 1) {
        constexpr int STEP = N / (NS * R);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[(r * k * STEP) * TWS];  // r*k*STEP < N
          if (INV) w.y = -w.y;
          v[i][r] = cmul(v[i][r], w);
        }
      }
      dftR<R, INV>(v[i]);
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[addr(base + r * NS, b)] = v[i][r];
    }
  }
  __syncthreads();
}

// All stages of a length-N transform over B sequences (in place, natural
// order in and out), any layout.
template <int N, int B, int NT, bool INV, int TWS, class A, int NS = 1>
__device__ __forceinline__ void fft_smem_a(float2* buf, A addr, const float2* tw) {
  if constexpr (NS < N) {
    constexpr int R = radix_for(N / NS);
    fft_stage_a<N, R, NS, B, NT, INV, TWS>(buf, addr, tw);
    fft_smem_a<N, B, NT, INV, TWS, A, NS * R>(buf, addr, tw);
  }
}

// Linear layout: element n of sequence b at buf[n*es + b*bs].
template <int N, int B, int NT, bool INV, int TWS>
__device__ __forceinline__ void fft_smem(float2* buf, int es, int bs, const float2* tw) {
  fft_smem_a<N, B, NT, INV, TWS>(buf, LinAddr{es, bs}, tw);
}

// ------------------------------------------------------------ async copies
// cp.async (global -> shared, bypassing registers): a thread issues all of its
// copies before waiting, so a whole tile is in flight at once.  A source size
// of 0 zero-fills the destination without reading the source.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }


// Threads for a batch of B sequences of length N at about 8 elements per
// thread (one radix-8 butterfly per stage), a multiple of 32 in [64, 1024].
__host__ __device__ constexpr int threads_for(int elems) {
  int t = elems / 8;
  t = t < 64 ? 64 : (t > 1024 ? 1024 : t);
  return (t + 31) / 32 * 32;
}

// Launch geometry shared by the column-tile kernels (transforms along a
// strided axis, B adjacent columns per CTA).
template <int N>
struct ColGeom {
  static constexpr int B = (N <= 256) ? 16 : 8;
  static constexpr int NT = threads_for(N * B);
  static constexpr int MINB = (1536 / NT) > 1 ? (1536 / NT) : 1;
  static constexpr size_t SMEM = (size_t)N * B * sizeof(float2) + (size_t)N * sizeof(float2);
};

// Row tiles (transforms along the contiguous axis).  B rows per CTA are held
// column-major in shared memory, element n of row b at n * P + b with the odd
// pitch P = B + 1: the coalesced row copies (n fastest across a warp) and the
// FFT stages (row fastest) are both free of bank conflicts.
template <int N>
struct RowGeom {
  static constexpr int B = (N <= 512) ? 16 : 8;
  static constexpr int P = B + 1;
  static constexpr int NT = threads_for(N * B);
  static constexpr int MINB = (1536 / NT) > 1 ? (1536 / NT) : 1;
};

}  // namespace wo

// Every supported transform length.
#define WO_FOR_EACH_SIZE(M)                                                                 \
  M(1) M(2) M(3) M(4) M(6) M(8) M(12) M(16) M(24) M(32) M(48) M(64) M(96) M(128) M(192) \
      M(256) M(384) M(512) M(768) M(1024) M(1536) M(2048)

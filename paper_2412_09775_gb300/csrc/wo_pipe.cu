// wo_pipe.cu - persistent tile pipeline of the 3D Tikhonov reconstruction for
// tile-sized planes (rows a5-a7 on a batch of tiles; Eq. recon solved per
// frequency in its push-through form F = conj(H) D / (|H|^2 + eta) for the
// phase-only mode).
//
// The pass path (wo_api.cu) moves a tile through five kernels: x R2C, y FFT,
// z FFT + solve + inverse z FFT, inverse y, x C2R, each reading and writing
// the whole batch in HBM.  For planes that fit one SM's shared memory (a
// 192 x 97 complex half-plane is 149 KB) this kernel does the same work as
// three kinds of work items taken from one queue by persistent CTAs:
//   A(t, j)  plane j of tile t: x R2C and y FFT in shared memory, the plane's
//            half spectrum stored to the workspace;
//   B(t, y)  row y of tile t: its Z x (X/2+1) spectrum column block and TF
//            block, z FFT, per-frequency solve, inverse z FFT, stored back;
//   C(t, j)  plane j of tile t: the solved half spectrum brought in by one
//            TMA bulk copy, inverse y FFT and x C2R in shared memory, the
//            real plane of the reconstruction stored.
// Items are dispensed by an atomic ticket in steps s = 0, 1, ...: step s
// holds A(s, *), then B(s-1, *), then C(s-2, *).  A tile's spectrum lives
// between its A and C items, about three tiles (21 MB at 48 x 192 x 192) at
// any time, so the hand-offs stay in the 129 MB L2: HBM sees the data once
// in, the TFs once and the result once out.
//
// B(t, *) waits until the A(t, *) items have posted (a per-tile counter), C
// until the B items have.  A ticket is taken only by a running CTA and every
// item waits only on items with smaller tickets, which were taken earlier by
// running CTAs, and A items wait on nothing: the earliest unfinished item
// never waits, so the queue always makes progress.  The waits are bounded
// all the same: a waiting CTA reads %globaltimer, and after `budget_ns`
// without the count it records WO_ERR_TIMEOUT in the workspace's status
// block, raises the batch's abort flag (every CTA then stops taking tickets
// and leaves its waits) and returns.  Data produced by another CTA of the
// launch is read past L1 (ld.global.cg, or the TMA bulk copy, which reads
// through L2).
#include <stdint.h>

#include "wo_fft.cuh"
#include "wo_bulk.cuh"
#include "wo_internal.h"
#include "wo_zops.cuh"

namespace wo {

namespace {

constexpr int kPipeThreads = 512;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

struct PipeArgs {
  const float* in;       // [T][Z][Y][X] data (brightfield stacks)
  float* out;            // [T][Z][Y][X] reconstructed index increment
  float2* spec;          // [T][Z][Y][Xh] working spectra (workspace)
  const float2* tf;      // phase TF of tile 0; tile t's at tf + t * tf_stride
  long long tf_stride;   // float2 between tiles' phase TFs (0: one bank for every tile)
  const float* stats;    // [T or 1][8] TF statistics
  int* ctr;              // [0] ticket, [1] abort, [2, 2+T) A posts, [2+T, 2+2T) B posts
  int* status;           // workspace status block: code, site, detail
  int T, tf_shared, eta_absolute, zero_dc, withhold;
  float eta, bg_plane, scale;  // bg_plane: Y X b removed from each plane's DC (given background)
  long long budget_ns;
};

// Record the first error of the batch and raise the abort flag.
__device__ void pipe_fail(const PipeArgs& a, int site, int detail) {
  if (atomicCAS(a.status, 0, (int)WO_ERR_TIMEOUT) == 0) {
    a.status[1] = site;
    a.status[2] = detail;
  }
  atomicExch(a.ctr + 1, 1);
  __threadfence();
}

// Thread 0: wait (bounded) until *c >= target.  false on timeout or abort.
__device__ bool pipe_wait(const PipeArgs& a, const int* c, int target, int site, int detail) {
  if (ld_acquire(c) >= target) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    __nanosleep(256);
    if (ld_acquire(c) >= target) return true;
    if (ld_acquire(a.ctr + 1)) return false;
    if ((long long)(global_ns() - t0) > a.budget_ns) {
      pipe_fail(a, site, detail);
      return false;
    }
  }
}

// In-place transforms of length N of S sequences in shared memory (element
// n of sequence b at buf[n * es + b * bs]), CHUNK sequences at a time: an
// in-place stage holds every input of the chunk in registers across its
// barrier, so the chunk bounds the registers a thread needs.
template <int N, int S, int CHUNK, int NT, bool INV, int B0 = 0>
__device__ __forceinline__ void fft_chunks(float2* buf, int es, int bs, const float2* tw) {
  if constexpr (B0 < S) {
    constexpr int C = (S - B0) < CHUNK ? (S - B0) : CHUNK;
    fft_smem<N, C, NT, INV, 1>(buf + B0 * bs, es, bs, tw);
    fft_chunks<N, S, CHUNK, NT, INV, B0 + C>(buf, es, bs, tw);
  }
}

template <int N, int S, int CHUNK, int NT, bool INV>
__device__ __forceinline__ void fft_call(float2* buf, int es, int bs, const float2* tw) {
  fft_chunks<N, S, CHUNK, NT, INV>(buf, es, bs, tw);
}

// Sequences per chunk so that a thread holds at most about 20 complex values.
__host__ __device__ constexpr int chunk_for(int N, int S, int NT) {
  const int c = (20 * NT) / N;
  const int k = (S + (c > 0 ? c : 1) - 1) / (c > 0 ? c : 1);  // chunks
  return (S + k - 1) / k;
}

template <int Z, int Y, int H>
struct PipeGeom {
  static constexpr int Xh = H + 1;
  static constexpr int PLANE = Y * Xh;             // float2 of a half-spectrum plane
  static constexpr int ZBLK = Z * Xh;              // float2 of one row's z block
  static constexpr int BUF = PLANE > 2 * ZBLK ? PLANE : 2 * ZBLK;
  static constexpr int TW = H + Y + Z + (H + 1);   // x, y, z twiddles and the R2C split factors
  static constexpr size_t SMEM = (size_t)(BUF + TW) * sizeof(float2) + 16;
};

// Shared memory of the kernel: the plane buffer and the twiddle tables.
struct PipeSmem {
  float2* P;    // plane (A, C) or [D | H] z blocks (B)
  float2* twx;  // w_H^m
  float2* twy;  // w_Y^m
  float2* twz;  // w_Z^m
  float2* tws;  // w_X^k, k = 0..H (R2C split)
  uint64_t* bar;
};

// A(t, j): x R2C and y FFT of plane j of tile t; posts to the tile's counter.
template <int Z, int Y, int H>
__device__ __forceinline__ void item_A(const PipeArgs& a, const PipeSmem& m, int t, int j) {
  using G = PipeGeom<Z, Y, H>;
  constexpr int NT = kPipeThreads, Xh = G::Xh, X = 2 * H;
  const int tid = threadIdx.x;
  float2* P = m.P;
  const float2* src = reinterpret_cast<const float2*>(a.in + ((long long)t * Z + j) * Y * X);
  for (int e = tid; e < Y * H; e += NT) {
    const int y = e / H, n = e - y * H;
    cp_async8(P + y * Xh + n, src + e, true);
  }
  cp_async_wait_all();
  __syncthreads();
  fft_call<H, Y, chunk_for(H, Y, NT), NT, false>(P, 1, Xh, m.twx);  // rows: z_n = x_2n + i x_2n+1
  // Hermitian split: X_k = (Z_k + conj Z_-k)/2 - i w_X^k (Z_k - conj Z_-k)/2, k = 0..H
  for (int e = tid; e < Y * (H / 2 + 1); e += NT) {
    const int y = e / (H / 2 + 1), q = e - y * (H / 2 + 1);
    float2* row = P + y * Xh;
    const int mq = (H - q) % H;
    const float2 zk = row[q], zm = row[mq];
    const float2 sk = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));  // (Z_k + conj Z_m)/2
    const float2 dk = make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y + zm.y));  // (Z_k - conj Z_m)/2
    const float2 sm_ = make_float2(sk.x, -sk.y);                                // (Z_m + conj Z_k)/2
    const float2 dm = make_float2(-dk.x, dk.y);                                 // (Z_m - conj Z_k)/2
    const float2 tk = cmul(m.tws[q], dk), tm = cmul(m.tws[H - q], dm);
    row[q] = make_float2(sk.x + tk.y, sk.y - tk.x);  // sk - i tk
    row[H - q] = make_float2(sm_.x + tm.y, sm_.y - tm.x);
  }
  __syncthreads();
  fft_call<Y, Xh, chunk_for(Y, Xh, NT), NT, false>(P, Xh, 1, m.twy);  // columns
  if (tid == 0 && a.bg_plane != 0.f) P[0].x -= a.bg_plane;
  __syncthreads();
  float4* dst = reinterpret_cast<float4*>(a.spec + ((long long)t * Z + j) * G::PLANE);
  const float4* s4 = reinterpret_cast<const float4*>(P);
  for (int e = tid; e < G::PLANE / 2; e += NT) __stcg(dst + e, s4[e]);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    atomicAdd(a.ctr + 2 + t, 1);
  }
}

// B(t, y): z FFT, per-frequency solve, inverse z FFT of row y of tile t;
// posts to the tile's second counter.
template <int Z, int Y, int H>
__device__ __forceinline__ void item_B(const PipeArgs& a, const PipeSmem& m, int t, int y) {
  using G = PipeGeom<Z, Y, H>;
  constexpr int NT = kPipeThreads, Xh = G::Xh;
  const int tid = threadIdx.x;
  const int tt = a.tf_shared ? 0 : t;
  float2* D = m.P;
  float2* Hb = m.P + G::ZBLK;
  const float2* sp = a.spec + ((long long)t * Z * Y + y) * Xh;
  const float2* hp = a.tf + (long long)tt * a.tf_stride + (long long)y * Xh;
  for (int e = tid; e < G::ZBLK; e += NT) {
    const int jz = e / Xh, x = e - jz * Xh;
    D[e] = __ldcg(sp + (long long)jz * Y * Xh + x);
    Hb[e] = __ldg(hp + (long long)jz * Y * Xh + x);
  }
  __syncthreads();
  fft_call<Z, Xh, chunk_for(Z, Xh, NT), NT, false>(D, Xh, 1, m.twz);
  const float* st = a.stats + (long long)tt * 8;
  const float lam = a.eta_absolute ? a.eta : a.eta * st[0];
  for (int e = tid; e < G::ZBLK; e += NT) {
    const int kz = e / Xh, x = e - kz * Xh;
    float2 d = D[e];
    if (a.zero_dc && kz == 0 && y == 0 && x == 0) d = make_float2(0.f, 0.f);
    // columns outside the support disk hold only the TFs' rounding noise: zero out
    if (outside_support(st, y, Y, x, 2 * H)) d = make_float2(0.f, 0.f);
    const float2 h = Hb[e];
    const float den = lam + cabs2(h);
    D[e] = cscale(cmulc(h, d), den > 0.f ? 1.0f / den : 0.f);  // zero TF and eta: minimum norm
  }
  __syncthreads();
  fft_call<Z, Xh, chunk_for(Z, Xh, NT), NT, true>(D, Xh, 1, m.twz);
  float2* op = a.spec + ((long long)t * Z * Y + y) * Xh;
  for (int e = tid; e < G::ZBLK; e += NT) {
    const int jz = e / Xh, x = e - jz * Xh;
    __stcg(op + (long long)jz * Y * Xh + x, D[e]);
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    atomicAdd(a.ctr + 2 + a.T + t, 1);
  }
}

// C(t, j): the solved plane by TMA, inverse y FFT and x C2R, the real plane
// stored.  false when its copy did not land within the budget.
template <int Z, int Y, int H>
__device__ __forceinline__ bool item_C(const PipeArgs& a, const PipeSmem& m, int t, int j, unsigned phase) {
  using G = PipeGeom<Z, Y, H>;
  constexpr int NT = kPipeThreads, Xh = G::Xh, X = 2 * H;
  const int tid = threadIdx.x;
  float2* P = m.P;
  if (tid == 0) {
    // the bulk copy (async proxy) reads what other CTAs stored and
    // overwrites what this CTA's threads last read and wrote
    asm volatile("fence.proxy.async;" ::: "memory");
    mbar_expect_tx(m.bar, (unsigned)(G::PLANE * sizeof(float2)));
    bulk_load(P, a.spec + ((long long)t * Z + j) * G::PLANE, (unsigned)(G::PLANE * sizeof(float2)), m.bar);
  }
  // every thread waits for the copy; bounded, though a bulk copy of valid
  // addresses always completes
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(m.bar, phase)) {
    if ((long long)(global_ns() - t0) > a.budget_ns) {
      if (tid == 0) pipe_fail(a, 3, t);
      // leave only once the copy has landed or the wait ran out again, so
      // no copy writes this CTA's shared memory after it exits
      const unsigned long long t1 = global_ns();
      while (!mbar_try_wait(m.bar, phase) && (long long)(global_ns() - t1) < a.budget_ns) {
      }
      return false;
    }
  }
  fft_call<Y, Xh, chunk_for(Y, Xh, NT), NT, true>(P, Xh, 1, m.twy);
  // inverse of the split: Z_k = (X_k + conj X_H-k)/2 + i conj(w_X^k) (X_k - conj X_H-k)/2, k < H
  for (int e = tid; e < Y * (H / 2 + 1); e += NT) {
    const int y = e / (H / 2 + 1), q = e - y * (H / 2 + 1);
    float2* row = P + y * Xh;
    const float2 xk = row[q], xm = row[H - q];
    const float2 ek = make_float2(0.5f * (xk.x + xm.x), 0.5f * (xk.y - xm.y));
    const float2 ok = make_float2(0.5f * (xk.x - xm.x), 0.5f * (xk.y + xm.y));
    const float2 em = make_float2(ek.x, -ek.y);
    const float2 om = make_float2(-ok.x, ok.y);
    const float2 uk = cmul(cconj(m.tws[q]), ok), um = cmul(cconj(m.tws[H - q]), om);
    row[q] = make_float2(ek.x - uk.y, ek.y + uk.x);  // ek + i uk
    if (q > 0) row[H - q] = make_float2(em.x - um.y, em.y + um.x);
  }
  __syncthreads();
  fft_call<H, Y, chunk_for(H, Y, NT), NT, true>(P, 1, Xh, m.twx);
  float2* dst = reinterpret_cast<float2*>(a.out + ((long long)t * Z + j) * Y * X);
  for (int e = tid; e < Y * H; e += NT) {
    const int y = e / H, n = e - y * H;
    dst[e] = cscale(P[y * Xh + n], a.scale);
  }
  __syncthreads();  // P is refilled by the next item
  return true;
}

// One item per CTA: the CTA takes the next ticket when it starts (not its
// block index), so tickets are handed out in the order CTAs begin to run.
template <int Z, int Y, int H>
__global__ void __launch_bounds__(kPipeThreads, 1) k_pipe(PipeArgs a) {
  using G = PipeGeom<Z, Y, H>;
  constexpr int NT = kPipeThreads;
  extern __shared__ __align__(16) float2 sm[];
  PipeSmem m;
  m.P = sm;
  m.twx = sm + G::BUF;
  m.twy = m.twx + H;
  m.twz = m.twy + Y;
  m.tws = m.twz + Z;
  m.bar = reinterpret_cast<uint64_t*>(m.tws + H + 1);
  __shared__ int s_item, s_go;
  const int tid = threadIdx.x;
  constexpr int STEP = Z + Y + Z;
  const long long total = (long long)(a.T + 2) * STEP;
  if (tid == 0) {
    const int k = ld_acquire(a.ctr + 1) ? -1 : atomicAdd(a.ctr, 1);
    s_item = (k < 0 || (long long)k >= total) ? -1 : k;
  }
  __syncthreads();
  const int k = s_item;
  if (k < 0) return;
  const int s = k / STEP, r = k - s * STEP;
  if (r < Z) {
    if (s >= a.T || s == a.withhold) return;
  } else {
    const int t = r < Z + Y ? s - 1 : s - 2;
    if (t < 0 || t >= a.T) return;
  }
  if (r < Z || r >= Z + Y) {  // plane items: x, y and split twiddles
    make_twiddles<H>(m.twx);
    make_twiddles<Y>(m.twy);
    for (int q = tid; q <= H; q += NT) {
      float sn, cs;
      sincospif((float)q / (float)H, &sn, &cs);  // exp(-2 pi i q / X)
      m.tws[q] = make_float2(cs, -sn);
    }
  } else {
    make_twiddles<Z>(m.twz);
  }
  if (r < Z) {
    __syncthreads();
    item_A<Z, Y, H>(a, m, s, r);
  } else if (r < Z + Y) {
    const int t = s - 1;
    if (tid == 0) s_go = pipe_wait(a, a.ctr + 2 + t, Z, 1, t) ? 1 : 0;
    __syncthreads();
    if (!s_go) return;
    item_B<Z, Y, H>(a, m, t, r - Z);
  } else {
    const int t = s - 2;
    if (tid == 0) {
      mbar_init(m.bar, 1);
      s_go = pipe_wait(a, a.ctr + 2 + a.T + t, Y, 2, t) ? 1 : 0;
    }
    __syncthreads();
    if (!s_go) return;
    item_C<Z, Y, H>(a, m, t, r - Z - Y, 0u);
  }
}

template <int Z, int Y, int H>
cudaError_t launch_pipe(const PipeArgs& a, cudaStream_t s) {
  using G = PipeGeom<Z, Y, H>;
  const cudaError_t attr = allow_smem(k_pipe<Z, Y, H>, G::SMEM);
  if (attr != cudaSuccess) return attr;
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pipe<Z, Y, H>, kPipeThreads, G::SMEM);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  const long long items = (long long)(a.T + 2) * (2 * Z + Y);
  WO_LAUNCH("tile_pipeline", s, (k_pipe<Z, Y, H><<<(unsigned)items, kPipeThreads, G::SMEM, s>>>(a)));
  return cudaGetLastError();
}

}  // namespace

// The shapes the pipeline is built for: (Z, Y, X/2) of the tile workloads
// (the shift-variant field's 48 x 192 x 192 tiles, the 48 x 128 x 128 tuning
// and estimator tiles, the 16 x 64 x 64 small stacks).
bool pipe_supported(int Z, int Y, int X) {
  return (Z == 48 && Y == 192 && X == 192) || (Z == 48 && Y == 128 && X == 128) || (Z == 16 && Y == 64 && X == 64);
}

size_t pipe_counter_bytes(int n_tiles) { return (size_t)(2 + 2 * (size_t)n_tiles) * sizeof(int); }

cudaError_t tile_pipeline(const PipeLaunch& p, cudaStream_t s) {
  PipeArgs a{};
  a.in = p.in;
  a.out = p.out;
  a.spec = p.spec;
  a.tf = p.tf;
  a.tf_stride = p.tf_shared ? 0 : p.tf_stride;
  a.stats = p.stats;
  a.ctr = p.counters;
  a.status = p.status;
  a.T = p.n_tiles;
  a.tf_shared = p.tf_shared;
  a.eta_absolute = p.eta_absolute;
  a.zero_dc = p.zero_dc;
  a.withhold = p.withhold;
  a.eta = p.eta;
  a.bg_plane = p.bg_plane;
  a.scale = p.scale;
  a.budget_ns = p.budget_ns;
  cudaError_t e = cudaMemsetAsync(p.counters, 0, pipe_counter_bytes(p.n_tiles), s);
  if (e != cudaSuccess) return e;
  if (p.Z == 48 && p.Y == 192 && p.X == 192) return launch_pipe<48, 192, 96>(a, s);
  if (p.Z == 48 && p.Y == 128 && p.X == 128) return launch_pipe<48, 128, 64>(a, s);
  if (p.Z == 16 && p.Y == 64 && p.X == 64) return launch_pipe<16, 64, 32>(a, s);
  return cudaErrorInvalidValue;
}

}  // namespace wo

// wo_psf.cu - PSF rows of the transfer-function build with register-resident
// row transforms (rows of 32 to 512 points).
//
// Same operation as k_psf_rows (wo_tf.cu): per row (tile t, plane j, row y)
// of the arms after their y transform, the inverse transform along x of every
// arm, the real PSF rows, and their forward transform along x into the TF
// bank.  Here T lanes of a warp own a row (wo_regfft.cuh): the arms are read
// from global memory straight into registers (columns outside the detection
// band are zero and are not read), the products are formed in registers, and
// every transform touches shared memory once (one transpose), with warp-level
// synchronisation only.
//
// All real PSF rows are transformed as complex rows two at a time where the
// kinds allow it: with the defocus derivative the row w = 2K (Re g + i Re g')
// gives both TF rows from one transform (g' = conj(a') b + conj(a) b'):
//   H(k) = (W(k) + W*(-k)) / 2,   dH(k) = (W(k) - W*(-k)) / (2i).
// Label-free rows use the complex g = 2K conj(a) b:
//   H_re(k) = (G(k) + G*(-k)) / 2,   H_im(k) = i (G(k) - G*(-k)) / 2.
// Single real rows (fluorescence, or one label-free kind) pair up across two
// rows of the bank instead (k_psf_rows_pair).
// W*(-k) lives in the lane that owns N - k; it is fetched with a shuffle.
#include <type_traits>

#include "wo_fft.cuh"
#include "wo_internal.h"
#include "wo_regfft.cuh"
#include "wo_tf.cuh"

namespace wo {

namespace {
constexpr int kPsfThreads = 128;

template <class P>
__device__ __forceinline__ void load_arm(float2 (&v)[P::E], const TfArgs& a, long long t, long long rem, int arm,
                                         int kxm, int lane_t) {
  constexpr int N = P::N, N1 = P::E, T = P::T;
  const float2* src = a.arms + ((t * a.n_arms + arm) * a.Z) * (long long)a.Y * N + rem * N + lane_t;
#pragma unroll
  for (int m = 0; m < N1; ++m) {
    const int n = lane_t + T * m;
    v[m] = (abs(fft_index(n, N)) <= kxm) ? __ldg(src + T * m) : make_float2(0.f, 0.f);
  }
}

// Register index holding W(N - k) in the lane that owns it (see wo_regfft.cuh):
// for lane 0, point T m pairs with T ((N1 - m) mod N1); for lane t > 0, point
// t + T m pairs with (T - t) + T (N1 - 1 - m).
template <int N1>
__device__ __forceinline__ float2 mirror_value(const float2 (&v)[N1], int m, bool lane0) {
  return lane0 ? v[(N1 - m) % N1] : v[N1 - 1 - m];
}

}  // namespace

// P: the row transform (Row2 or Row512 of wo_regfft.cuh).  MODE 0: any mix
// of label-free and fluorescence kinds; 1: the phase TF and its defocus
// derivative (arms A, B, A', B'); 2: plus the derivatives in tilt_x, tilt_y
// and NA_ill under the smooth source (arms A_tx, A_ty, A_NA; their rows
// 2K (Re conj(a_theta) b - (D_theta / D) Re g), D = sum S P^2).
template <class P, int MODE>
__global__ void __launch_bounds__(kPsfThreads, (P::E > 16 && MODE == 2) ? 2 : 4) k_psf_rows_reg(TfArgs a) {
  constexpr int N = P::N, N1 = P::E, T = P::T, RP = P::SLICE, RPC = kPsfThreads / T;
  __shared__ float2 tw[P::TW];
  __shared__ float2 slices[RPC * RP];
  const int lt = threadIdx.x % T, r = threadIdx.x / T;
  const int lane = threadIdx.x & 31;
  const int partner = (lane - lt) + (T - lt) % T;  // lane owning N - k
  const bool lane0 = lt == 0;
  float2* S = slices + r * RP;
  const long long nrows = a.row_end;
  const long long row = a.row_begin + (long long)blockIdx.x * RPC + r;
  bool live = row < nrows;
  const long long rr = live ? row : nrows - 1;  // tail lanes compute on a valid row, store nothing
  const long long zy = (long long)a.Z * a.Y;
  long long t = rr / zy, rem = rr - t * zy;  // rem = j*Y + y
  const bool lf = a.lf_props > 0, fl = a.want_fl != 0;
  const int Xh = N / 2 + 1;
  const long long kstride = (long long)a.Z * a.Y * Xh;
#if defined(WO_CHECK) && WO_CHECK
  {  // the row's count, last arm point and last TF bin inside their arrays; a
     // failed check turns the row into a tail row (row 0, nothing stored), so
     // the block's barrier is still met
    const long long arms_end = (long long)a.n_tiles * a.n_arms * a.Z * a.Y * N;
    const long long tf_end = (long long)a.n_tiles * a.n_kinds * kstride;
    if (!WO_IN(t, a.n_tiles, 9) ||
        !WO_IN(((t * a.n_arms + a.n_arms - 1) * a.Z) * (long long)a.Y * N + rem * N + N - 1, arms_end, 9) ||
        !WO_IN((t * a.n_kinds * a.Z) * (long long)a.Y * Xh + rem * Xh + (a.n_kinds - 1) * kstride + N / 2, tf_end, 9)) {
      live = false;
      t = 0;
      rem = 0;
    }
  }
#endif
  const int kxm = a.counts[4 * t + 2];
  float2* dst = a.tf + (t * a.n_kinds * a.Z) * (long long)a.Y * Xh + rem * Xh;  // slot 0 of this row

  constexpr bool DZ = MODE >= 1;
  float2 w[N1];
  float gre[MODE == 2 ? N1 : 1];  // Re g (unscaled), for the normalisation terms
  float2 vb[N1];                  // b, kept for the source-parameter arms
  float2 va[N1];
  // the row's first arm is on its way while the block forms its twiddles
  if (DZ || lf) load_arm<P>(va, a, t, rem, 0, kxm, lt);
  else load_arm<P>(w, a, t, rem, 0, kxm, lt);
  // the row's scale factors (float64 arithmetic, slow on this part) are
  // formed once per row, by its first lane, and broadcast
  float sc_row = 0.f, scf_row = 0.f;
  if (lt == 0) {
    if (DZ || lf) sc_row = lf_scale(a, (int)t);
    if (!DZ && fl) scf_row = fl_scale(a, (int)t);
  }
  sc_row = __shfl_sync(0xffffffffu, sc_row, lane - lt);
  scf_row = __shfl_sync(0xffffffffu, scf_row, lane - lt);
  P::twiddles(tw);
  __syncthreads();
  int slot = 0;
  if (DZ || lf) {
    const float sc = sc_row;
    if constexpr (DZ) {
      // w = 2K (Re conj(a) b + i (Re conj(a) b' + Re conj(a') b)), arms A, B, A', B'
      P::template fft<true>(va, tw, S, lt);
      load_arm<P>(vb, a, t, rem, 3, kxm, lt);
      P::template fft<true>(vb, tw, S, lt);
#pragma unroll
      for (int m = 0; m < N1; ++m) w[m].y = va[m].x * vb[m].x + va[m].y * vb[m].y;
      load_arm<P>(vb, a, t, rem, 1, kxm, lt);
      P::template fft<true>(vb, tw, S, lt);
#pragma unroll
      for (int m = 0; m < N1; ++m) w[m].x = va[m].x * vb[m].x + va[m].y * vb[m].y;
      load_arm<P>(va, a, t, rem, 2, kxm, lt);
      P::template fft<true>(va, tw, S, lt);
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        w[m].y += va[m].x * vb[m].x + va[m].y * vb[m].y;
        if constexpr (MODE == 2) gre[m] = w[m].x;
        w[m] = cscale(w[m], sc);
      }
    } else {
      P::template fft<true>(va, tw, S, lt);
      load_arm<P>(vb, a, t, rem, 1, kxm, lt);
      P::template fft<true>(vb, tw, S, lt);
#pragma unroll
      for (int m = 0; m < N1; ++m) w[m] = cscale(cmulc(va[m], vb[m]), sc);
    }
    P::template fft<false>(w, tw, S, lt);
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const float2 mv = mirror_value<N1>(w, m, lane0);
      float2 c;  // conj(W(N - k))
      c.x = __shfl_sync(0xffffffffu, mv.x, partner);
      c.y = -__shfl_sync(0xffffffffu, mv.y, partner);
      const int k = lt + T * m;
      if (!live || k > N / 2) continue;
      const float2 s = make_float2(0.5f * (w[m].x + c.x), 0.5f * (w[m].y + c.y));  // (W + W*(-k)) / 2
      const float2 d = make_float2(0.5f * (w[m].x - c.x), 0.5f * (w[m].y - c.y));  // (W - W*(-k)) / 2
      if constexpr (DZ) {
        dst[k] = s;
        dst[kstride + k] = make_float2(d.y, -d.x);  // d / i
      } else {
        int q = 0;
        if (a.want_phase) dst[(q++) * kstride + k] = s;
        if (a.want_abs) dst[(q++) * kstride + k] = make_float2(-d.y, d.x);  // i d
      }
    }
    slot = DZ ? 2 : a.lf_props;
  }
  if constexpr (MODE == 2) {
    // source parameters: rows 2K (Re conj(a_theta) b - r_theta Re g), tilt_x
    // and tilt_y packed as one complex row, NA_ill as a real row
    const float sc = sc_row;
    const float rx = norm_dlog(a, (int)t, 0), ry = norm_dlog(a, (int)t, 1), rn = norm_dlog(a, (int)t, 2);
    float2 vs[N1];
    load_arm<P>(vs, a, t, rem, 4, kxm, lt);
    P::template fft<true>(vs, tw, S, lt);
#pragma unroll
    for (int m = 0; m < N1; ++m) w[m].x = sc * (vs[m].x * vb[m].x + vs[m].y * vb[m].y - rx * gre[m]);
    load_arm<P>(vs, a, t, rem, 5, kxm, lt);
    P::template fft<true>(vs, tw, S, lt);
#pragma unroll
    for (int m = 0; m < N1; ++m) w[m].y = sc * (vs[m].x * vb[m].x + vs[m].y * vb[m].y - ry * gre[m]);
    P::template fft<false>(w, tw, S, lt);
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const float2 mv = mirror_value<N1>(w, m, lane0);
      float2 c;  // conj(W(N - k))
      c.x = __shfl_sync(0xffffffffu, mv.x, partner);
      c.y = -__shfl_sync(0xffffffffu, mv.y, partner);
      const int k = lt + T * m;
      if (!live || k > N / 2) continue;
      const float2 d = make_float2(0.5f * (w[m].x - c.x), 0.5f * (w[m].y - c.y));
      dst[2 * kstride + k] = make_float2(0.5f * (w[m].x + c.x), 0.5f * (w[m].y + c.y));
      dst[3 * kstride + k] = make_float2(d.y, -d.x);
    }
    load_arm<P>(vs, a, t, rem, 6, kxm, lt);
    P::template fft<true>(vs, tw, S, lt);
#pragma unroll
    for (int m = 0; m < N1; ++m) w[m] = make_float2(sc * (vs[m].x * vb[m].x + vs[m].y * vb[m].y - rn * gre[m]), 0.f);
    P::template fft<false>(w, tw, S, lt);
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const int k = lt + T * m;
      if (live && k <= N / 2) dst[4 * kstride + k] = w[m];
    }
  }
  if (!DZ && fl) {
    const float scf = scf_row;
    if (lf) load_arm<P>(w, a, t, rem, 2, kxm, lt);  // without label-free kinds it is arm 0, loaded above
    P::template fft<true>(w, tw, S, lt);
#pragma unroll
    for (int m = 0; m < N1; ++m) w[m] = make_float2(scf * cabs2(w[m]), 0.f);
    P::template fft<false>(w, tw, S, lt);
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      const int k = lt + T * m;
      if (live && k <= N / 2) dst[slot * kstride + k] = w[m];
    }
  }
}

// Banks without derivatives whose real PSF rows can share transforms: each
// lane group takes two consecutive rows.  A real row pair h0, h1 goes through
// one forward transform as w = h0 + i h1:
//   H0(k) = (W(k) + W*(-k)) / 2,   H1(k) = (W(k) - W*(-k)) / (2i).
// The fluorescence rows h = scf |p|^2 always pair this way; the label-free
// rows pair when one label-free kind is wanted (h = 2K Re g for the phase TF,
// -2K Im g for the absorption TF); with both, each row's complex g gives both
// TF rows from one transform as in k_psf_rows_reg.  The first row's real PSF
// row waits in shared memory (each lane reads back only what it wrote) while
// the second is formed.  The two rows may belong to different tiles when Z*Y
// is odd; everything per row is formed per row.
//
// ZK > 0: the bank is kx-major, [tile][kind][k][j][y] (the plane engine's
// layout, wo_plane.cu) with ZK planes of N rows: a lane stores bin k of its
// two rows (y, y + 1 of one plane, y even) as one 16-byte pair straight from
// registers; the lane groups of a warp hold consecutive row pairs, so a warp
// store fills a run of 2 * 32/T points of each of T bins (whole 32-byte
// sectors).  The bins' stride ZK N is a constant, so their offsets from the
// lane's first bin are immediates.
//
// Four CTAs (16 warps) per SM at every row length: the 24-point rows then
// fit in 128 registers only by spilling about 130 bytes a thread, and still
// run 6 % faster than at three CTAs with 168 registers and no spills (the
// kernel is bound by issue, and the extra warps hide its latencies).
template <class P, int LF, int ZK>  // LF: label-free kinds wanted (0, 1 or 2)
__global__ void __launch_bounds__(kPsfThreads, 4) k_psf_rows_pair(TfArgs a) {
  constexpr int N = P::N, N1 = P::E, T = P::T, RP = P::SLICE, RPC = kPsfThreads / T;
  // held-row pitch = T mod 32: the rows of one warp start on distinct banks
  constexpr int HP = N + (((T - N) % 32) + 32) % 32;
  __shared__ float2 tw[P::TW];
  __shared__ float2 slices[RPC * RP];
  __shared__ float held[RPC * HP];
  const int lt = threadIdx.x % T, r = threadIdx.x / T;
  const int lane = threadIdx.x & 31;
  const int partner = (lane - lt) + (T - lt) % T;  // lane owning N - k
  const bool lane0 = lt == 0;
  float2* S = slices + r * RP;
  float* Hs = held + r * HP + lt;  // this lane's points lt + T m at Hs[T m]
  const long long nrows = a.row_end;
  const long long row0 = a.row_begin + 2 * ((long long)blockIdx.x * RPC + r);
  bool live0 = row0 < nrows, live1 = row0 + 1 < nrows;
  const long long r0 = live0 ? row0 : nrows - 1, r1 = live1 ? row0 + 1 : nrows - 1;  // tails compute, store nothing
  const long long zy = (long long)a.Z * a.Y;
  long long t0 = r0 / zy, rem0 = r0 - t0 * zy, t1 = r1 / zy, rem1 = r1 - t1 * zy;
  constexpr bool lf = LF > 0, lf1 = LF == 1;
  const bool fl = a.want_fl != 0;
  const int Xh = N / 2 + 1;
  const long long kstride = (long long)a.Z * a.Y * Xh;
  const int fl_arm = lf ? 2 : 0;
#if defined(WO_CHECK) && WO_CHECK
  {  // both rows' counts, last arm points and last TF bins inside their arrays
    const long long arms_end = (long long)a.n_tiles * a.n_arms * a.Z * a.Y * N;
    const long long tf_end = (long long)a.n_tiles * a.n_kinds * kstride;
    const long long last_arm = (long long)a.n_arms - 1;
    if (!WO_IN(t0, a.n_tiles, 9) || !WO_IN(t1, a.n_tiles, 9) ||
        !WO_IN(((t0 * a.n_arms + last_arm) * a.Z) * (long long)a.Y * N + rem0 * N + N - 1, arms_end, 9) ||
        !WO_IN(((t1 * a.n_arms + last_arm) * a.Z) * (long long)a.Y * N + rem1 * N + N - 1, arms_end, 9) ||
        !WO_IN((t0 * a.n_kinds * a.Z) * (long long)a.Y * Xh + rem0 * Xh + (a.n_kinds - 1) * kstride + N / 2, tf_end, 9) ||
        !WO_IN((t1 * a.n_kinds * a.Z) * (long long)a.Y * Xh + rem1 * Xh + (a.n_kinds - 1) * kstride + N / 2, tf_end, 9)) {
      live0 = live1 = false;  // both rows become tail rows: nothing stored, the barrier still met
      t0 = t1 = 0;
      rem0 = rem1 = 0;
    }
  }
#endif
  const int kxm0 = a.counts[4 * t0 + 2], kxm1 = a.counts[4 * t1 + 2];
  float2* dst0 = a.tf + (t0 * a.n_kinds * a.Z) * (long long)a.Y * Xh + rem0 * Xh;
  float2* dst1 = a.tf + (t1 * a.n_kinds * a.Z) * (long long)a.Y * Xh + rem1 * Xh;

  float2 w[N1];
  float2 va[N1];
  // the first row's first arm is on its way while the block forms its twiddles
  if (lf) load_arm<P>(va, a, t0, rem0, 0, kxm0, lt);
  else load_arm<P>(w, a, t0, rem0, fl_arm, kxm0, lt);
  float sc0 = 0.f, sc1 = 0.f, scf0 = 0.f, scf1 = 0.f;  // float64 set-up: the group's first lane, broadcast
  if (lt == 0) {
    if (lf) {
      sc0 = lf_scale(a, (int)t0);
      sc1 = t1 == t0 ? sc0 : lf_scale(a, (int)t1);
    }
    if (fl) {
      scf0 = fl_scale(a, (int)t0);
      scf1 = t1 == t0 ? scf0 : fl_scale(a, (int)t1);
    }
  }
  sc0 = __shfl_sync(0xffffffffu, sc0, lane - lt);
  sc1 = __shfl_sync(0xffffffffu, sc1, lane - lt);
  scf0 = __shfl_sync(0xffffffffu, scf0, lane - lt);
  scf1 = __shfl_sync(0xffffffffu, scf1, lane - lt);
  P::twiddles(tw);
  __syncthreads();
  // one forward transform of w = h0 + i h1 into TF slot `slot` of both rows
  auto store_pair = [&](int slot) {
    P::template fft<false>(w, tw, S, lt);
    if constexpr (ZK > 0) {
      // rows r0, r0 + 1: one plane (Y = N even), bin k of both at dk + k ZK N
      const long long db = ((t0 * a.n_kinds + slot) * Xh * ZK) * (long long)N + rem0;
      float2* dk = a.tf + db;
      constexpr int kz = ZK * N;
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        if (T * m > N / 2) continue;  // no lane stores a bin of this register
        const float2 mv = mirror_value<N1>(w, m, lane0);
        float2 c;  // conj(W(N - k))
        c.x = __shfl_sync(0xffffffffu, mv.x, partner);
        c.y = -__shfl_sync(0xffffffffu, mv.y, partner);
        const int k = lt + T * m;
        if (k > N / 2 || !live1 || !WO_IN(db + k * kz + 1, (long long)a.n_tiles * a.n_kinds * kz * Xh, 9)) continue;
        *reinterpret_cast<float4*>(dk + k * kz) = make_float4(0.5f * (w[m].x + c.x), 0.5f * (w[m].y + c.y),
                                                              0.5f * (w[m].y - c.y), -0.5f * (w[m].x - c.x));
      }
      return;
    }
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      if (T * m > N / 2) continue;  // no lane stores a bin of this register
      const float2 mv = mirror_value<N1>(w, m, lane0);
      float2 c;  // conj(W(N - k))
      c.x = __shfl_sync(0xffffffffu, mv.x, partner);
      c.y = -__shfl_sync(0xffffffffu, mv.y, partner);
      const int k = lt + T * m;
      if (k > N / 2) continue;
      if (live0) dst0[slot * kstride + k] = make_float2(0.5f * (w[m].x + c.x), 0.5f * (w[m].y + c.y));
      if (live1) dst1[slot * kstride + k] = make_float2(0.5f * (w[m].y - c.y), -0.5f * (w[m].x - c.x));
    }
  };
  if constexpr (lf) {
    // one kind: straight-line code, so w is live only from the second row's product
#pragma unroll(LF == 1 ? 2 : 1)
    for (int q = 0; q < 2; ++q) {
      const long long tq = q ? t1 : t0, remq = q ? rem1 : rem0;
      const int kxq = q ? kxm1 : kxm0;
      const bool liveq = q ? live1 : live0;
      float2* dq = q ? dst1 : dst0;
      const float sc = q ? sc1 : sc0;
      if (q) load_arm<P>(va, a, tq, remq, 0, kxq, lt);
      float2 vb[N1];
      P::template fft<true>(va, tw, S, lt);
      load_arm<P>(vb, a, tq, remq, 1, kxq, lt);
      P::template fft<true>(vb, tw, S, lt);
      if constexpr (lf1) {
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          const float2 g = cmulc(va[m], vb[m]);
          const float h = sc * (a.want_phase ? g.x : -g.y);  // one kind: Re g (phase) or -Im g (absorption)
          if (q == 0) Hs[T * m] = h;
          else w[m] = make_float2(Hs[T * m], h);
        }
        continue;
      } else {
#pragma unroll
      for (int m = 0; m < N1; ++m) w[m] = cscale(cmulc(va[m], vb[m]), sc);
      P::template fft<false>(w, tw, S, lt);
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        if (T * m > N / 2) continue;  // no lane stores a bin of this register
        const float2 mv = mirror_value<N1>(w, m, lane0);
        float2 c;  // conj(W(N - k))
        c.x = __shfl_sync(0xffffffffu, mv.x, partner);
        c.y = -__shfl_sync(0xffffffffu, mv.y, partner);
        const int k = lt + T * m;
        if (!liveq || k > N / 2) continue;
        dq[k] = make_float2(0.5f * (w[m].x + c.x), 0.5f * (w[m].y + c.y));
        dq[kstride + k] = make_float2(-0.5f * (w[m].y - c.y), 0.5f * (w[m].x - c.x));
      }
      }
    }
    if constexpr (lf1) store_pair(0);
    if (!fl) return;
    load_arm<P>(w, a, t0, rem0, fl_arm, kxm0, lt);
  }
  P::template fft<true>(w, tw, S, lt);
#pragma unroll
  for (int m = 0; m < N1; ++m) Hs[T * m] = scf0 * cabs2(w[m]);
  load_arm<P>(w, a, t1, rem1, fl_arm, kxm1, lt);
  P::template fft<true>(w, tw, S, lt);
#pragma unroll
  for (int m = 0; m < N1; ++m) w[m] = make_float2(Hs[T * m], scf1 * cabs2(w[m]));
  store_pair(LF);
}

template <class P>
static cudaError_t launch_psf_pair(const TfArgs& a, cudaStream_t s) {
  constexpr int RPC = kPsfThreads / P::T;
  const long long pairs = (a.row_end - a.row_begin + 1) / 2;
  const unsigned grid = (unsigned)((pairs + RPC - 1) / RPC);
  if (a.kxm) {  // one kind, Y = X, Z 32 or 48 (16 with X = 64) (checked by the caller)
    if constexpr (P::N == 64 || P::N == 128 || P::N == 192) {
      if (a.Y != P::N) return cudaErrorInvalidValue;
      auto go = [&](auto zk) {
        constexpr int ZK = decltype(zk)::value;
        if (a.lf_props == 0) WO_LAUNCH("tf_psf_rows", s, (k_psf_rows_pair<P, 0, ZK><<<grid, kPsfThreads, 0, s>>>(a)));
        else WO_LAUNCH("tf_psf_rows", s, (k_psf_rows_pair<P, 1, ZK><<<grid, kPsfThreads, 0, s>>>(a)));
        return cudaGetLastError();
      };
      if (a.Z == 48) return go(std::integral_constant<int, 48>{});
      if (a.Z == 32) return go(std::integral_constant<int, 32>{});
      if constexpr (P::N == 64) {
        if (a.Z == 16) return go(std::integral_constant<int, 16>{});
      }
    }
    return cudaErrorInvalidValue;
  }
  switch (a.lf_props) {
    case 0: WO_LAUNCH("tf_psf_rows", s, (k_psf_rows_pair<P, 0, 0><<<grid, kPsfThreads, 0, s>>>(a))); break;
    case 1: WO_LAUNCH("tf_psf_rows", s, (k_psf_rows_pair<P, 1, 0><<<grid, kPsfThreads, 0, s>>>(a))); break;
    default: WO_LAUNCH("tf_psf_rows", s, (k_psf_rows_pair<P, 2, 0><<<grid, kPsfThreads, 0, s>>>(a))); break;
  }
  return cudaGetLastError();
}

// Row lengths X whose PSF-row pair kernel writes kx-major banks (the
// instantiated ones: square planes, Y = X, of 32 or 48 planes, or 16 planes
// of 64 points).
bool psf_kxm_supported(int X, int Y, int Z) {
  return (X == 64 || X == 128 || X == 192) && Y == X && (Z == 32 || Z == 48 || (Z == 16 && X == 64));
}

template <class P, int MODE>
static cudaError_t launch_psf_reg(const TfArgs& a, cudaStream_t s) {
  constexpr int RPC = kPsfThreads / P::T;
  const long long rows = a.row_end - a.row_begin;
  const unsigned grid = (unsigned)((rows + RPC - 1) / RPC);
  WO_LAUNCH("tf_psf_rows", s, (k_psf_rows_reg<P, MODE><<<grid, kPsfThreads, 0, s>>>(a)));
  return cudaGetLastError();
}

// Banks whose real PSF rows pair up across rows (k_psf_rows_pair).
static bool psf_pairs(const TfArgs& a) { return !a.want_dz && !a.want_grad && (a.want_fl || a.lf_props == 1); }

template <class P, bool GRAD = true>
static cudaError_t launch_psf_reg_any(const TfArgs& a, cudaStream_t s) {
  if (a.want_grad) {
    if constexpr (GRAD) return launch_psf_reg<P, 2>(a, s);
    return cudaErrorInvalidValue;
  }
  if (a.want_dz) return launch_psf_reg<P, 1>(a, s);
  return psf_pairs(a) ? launch_psf_pair<P>(a, s) : launch_psf_reg<P, 0>(a, s);
}

bool psf_rows_reg_supported(int X, int n_arms) {
  switch (X) {
    case 32: case 48: case 64: case 128: case 256: return true;
    case 512: return n_arms <= 4;
    case 96: case 192: return n_arms <= 3 || n_arms == 7;  // 24 points per lane: the derivative bank would spill
    default: return false;
  }
}

cudaError_t tf_psf_rows_reg(const TfArgs& a, cudaStream_t s) {
  switch (a.X) {
    case 32: return launch_psf_reg_any<Row2<32, 8>>(a, s);
    case 48: return launch_psf_reg_any<Row2<48, 12>>(a, s);
    case 64: return launch_psf_reg_any<Row2<64, 8>>(a, s);
    case 96:
      if (a.want_grad) return launch_psf_reg<Row2<96, 24>, 2>(a, s);
      if (a.want_dz) return cudaErrorInvalidValue;
      return psf_pairs(a) ? launch_psf_pair<Row2<96, 24>>(a, s) : launch_psf_reg<Row2<96, 24>, 0>(a, s);
    case 128: return launch_psf_reg_any<Row2<128, 16>>(a, s);
    case 192:
      if (a.want_grad) return launch_psf_reg<Row2<192, 24>, 2>(a, s);
      if (a.want_dz) return cudaErrorInvalidValue;
      return psf_pairs(a) ? launch_psf_pair<Row2<192, 24>>(a, s) : launch_psf_reg<Row2<192, 24>, 0>(a, s);
    case 256: return launch_psf_reg_any<Row2<256, 16>>(a, s);
    case 512: return launch_psf_reg_any<Row512, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wo

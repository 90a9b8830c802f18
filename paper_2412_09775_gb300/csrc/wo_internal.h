// wo_internal.h - launchers shared between the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/wo.h"

namespace wo {

// Index checks of the WO_CHECK build.  WO_IN(i, n, site) is true when
// 0 <= i < n; in a WO_CHECK build a kernel guards its global-memory accesses
// with it, skips an access whose index falls outside the buffer it addresses
// and records the first such index in its translation unit's device check
// block (code WO_ERR_BOUNDS, the site, the index), which wo_sync_status reads
// and clears.  Without WO_CHECK it is the constant true and costs nothing.
#if defined(WO_CHECK) && WO_CHECK
using CheckReader = int (*)(int* info);  // reads and clears one unit's block: code, [site, index]
void check_register(CheckReader r);
int check_take_all(int* info);           // the first recorded error over every unit (WO_OK if none)
namespace {
__device__ int g_wo_check[4];  // per translation unit: this build has no relocatable device code
__device__ __noinline__ void check_fail(int site, long long i) {
  if (atomicCAS(&g_wo_check[0], 0, (int)WO_ERR_BOUNDS) == 0) {
    g_wo_check[1] = site;
    g_wo_check[2] = (int)(i > 2147483647LL ? 2147483647LL : (i < -2147483647LL ? -2147483647LL : i));
  }
}
int check_take_unit(int* info) {
  int h[4] = {0, 0, 0, 0};
  if (cudaMemcpyFromSymbol(h, g_wo_check, sizeof(h)) != cudaSuccess) return (int)WO_ERR_CUDA;
  if (h[0] != 0) {
    const int z[4] = {0, 0, 0, 0};
    if (cudaMemcpyToSymbol(g_wo_check, z, sizeof(z)) != cudaSuccess) return (int)WO_ERR_CUDA;
    if (info) {
      info[0] = h[1];
      info[1] = h[2];
    }
  }
  return h[0];
}
struct CheckUnit {
  CheckUnit() { check_register(&check_take_unit); }
};
const CheckUnit g_check_unit;
}  // namespace
#define WO_IN(i, n, site) \
  (((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n)) ? true : (wo::check_fail((site), (long long)(i)), false))
#else
#define WO_IN(i, n, site) true
#endif

// Instrumentation: counts every launch; with profiling on, brackets it with
// CUDA events on its stream (see wo_profile_enable).
void prof_begin(const char* name, cudaStream_t s, int* token);
void prof_end(int token, cudaStream_t s);

// Background handling of a row pass over volumes laid out
// [block][Z][Y][X], block = tile * nchan + channel.
struct RowBg {
  float v[4];               // per-channel constants (mode 1)
  long long rows_per_block; // Z*Y
  long long row_offset;     // global index of the first row passed to the kernel
  int nchan;                // channels per tile
  int mode;                 // 0: none, 1: add/subtract v[channel], 2: subtract
                            //    the block's first sample (before R2C only)
};

// Real rows of length 2N -> half spectra of N+1 bins (row pitch N+1).
cudaError_t rows_r2c(int N, const float* in, float2* out, long long nrows, RowBg bg,
                     cudaStream_t s);
// Half spectra (pitch N+1) -> real rows of length 2N, times `scale`, plus bg.
cudaError_t rows_c2r(int N, const float2* in, float* out, long long nrows, float scale,
                     RowBg bg, cudaStream_t s);
// In-place C2C transforms of length N along a strided axis over `groups`
// groups of `nplanes` planes: element n of column c of plane i of group g at
// data[g*group_stride + i*plane_stride + n*col_stride + c].
// `name` labels the launch for the profiler.
cudaError_t cols_c2c(int N, bool inverse, float2* data, long long col_stride,
                     long long plane_stride, int ncols, long long nplanes, cudaStream_t s,
                     const char* name, long long groups = 1, long long group_stride = 0);

// Per-frequency operator applied between a forward and an inverse z transform.
struct ZOp {
  int op;            // 0 forward, 1 adjoint, 2 reconstruct
  int n_in, n_out;   // volumes per tile read / written
  int n_tf;          // TF slots per tile
  int lf_props;      // label-free properties (TF slots 0..lf_props-1), 0..2
  int has_fl;        // fluorescence TF at slot lf_props
  int lf_chan;       // data channel of the label-free mode (or -1)
  int fl_chan;       // data channel of the fluorescence mode (or -1)
  float eta_lf, eta_fl;
  int eta_absolute;
  int zero_dc;       // reconstruct: zero D(0) (background = channel mean)
  int tf_shared;     // 1: every tile uses tile 0's TFs and statistics (one bank for a batch of stacks)
  const float* stats;  // [tile][8] from the TF bank
};
// Fused z pass: FFT_z of n_in volumes, per-frequency op, IFFT_z of n_out volumes.
// Spectra laid out [tile][vol][Z][Y][Xh].
cudaError_t z_fused(int Z, const float2* in, float2* out, const float2* tf, ZOp op, int n_tiles,
                    int Y, int Xh, cudaStream_t s);
// The one-volume, one-TF case with register-resident z transforms (wo_zreg.cu).
bool z_reg_supported(int Z, const ZOp& op);
cudaError_t z_fused_reg(int Z, const float2* in, float2* out, const float2* tf, ZOp op, int n_tiles, int Y, int Xh,
                        cudaStream_t s);
// 2D reconstruction: FFT_z, per-transverse-frequency solve summed over k_z.
// out: [tile][P][Y][Xh].
cudaError_t z_solve2d(int Z, const float2* in, float2* out, const float2* tf, ZOp op, int n_tiles,
                      int Y, int Xh, cudaStream_t s);
// The plane engine (wo_plane.cu) on a kx-major spectrum, in place: one
// volume in and out, one TF slot (kx-major bank).
cudaError_t plane_yz_op(int Z, int Y, float2* spec, const float2* tf, const ZOp& op, int n_tiles, int Xh,
                        int* status, cudaStream_t s);

// The device status block at the start of every workspace: int32 code (a
// wo_status, 0 while nothing went wrong), site, detail; the rest reserved.
constexpr size_t kStatusBytes = 256;

// Persistent tile pipeline of the phase-only 3D reconstruction (wo_pipe.cu).
struct PipeLaunch {
  const float* in;       // [T][Z][Y][X] data
  float* out;            // [T][Z][Y][X] result
  float2* spec;          // [T][Z][Y][X/2+1] workspace spectra
  const float2* tf;      // phase TF slot of tile 0; tiles tf_stride float2 apart (0: shared bank)
  long long tf_stride;
  const float* stats;    // [T or 1][8]
  int* counters;         // pipe_counter_bytes(T), zeroed by the launcher
  int* status;           // the workspace's status block
  int n_tiles, Z, Y, X;
  int tf_shared, eta_absolute, zero_dc, withhold;
  float eta, bg_plane, scale;
  long long budget_ns;
};
bool pipe_supported(int Z, int Y, int X);
// Engine of the phase-only 3D reconstruction for these shapes: WO_ENGINE_SMEM
// (the five passes) or WO_ENGINE_HYBRID (the persistent pipeline).
int recon_engine(int Z, int Y, int X);
// Bound of every wait of the pipeline (ns): far above any legitimate wait
// (an item takes microseconds), far below a hang.
constexpr long long kPipeBudgetNs = 1000000000LL;
size_t pipe_counter_bytes(int n_tiles);
cudaError_t tile_pipeline(const PipeLaunch& p, cudaStream_t s);

// Multi-channel fusion (wo_fuse.cu): one property from C channels, each with
// its own TF; input spectra [tile][C][Z][Y][Xh], TF bank [tile*C][Z][Y][Xh].
constexpr int kMaxFuseChannels = 16;
struct FuseOp {
  int C;
  int mode;          // WO_MODE_3D: out [tile][Z][Y][Xh]; WO_MODE_2D: out [tile][Y][Xh]
  int zero_dc;       // background = channel means: zero the DC bin
  int eta_relative;  // eta times the per-tile scale in stats
  float eta;
  float bg_dc[kMaxFuseChannels];  // N b_c, subtracted from the DC bin when !zero_dc
  const float* stats;             // [tile][2]: max sum_c |H_c|^2 (3D), max sum_k sum_c |H_c|^2 (2D)
};
cudaError_t fuse_stats(const float2* tf, int n_tiles, int C, int Z, int Y, int Xh, float* stats, cudaStream_t s);
cudaError_t z_fuse(int Z, const float2* in, float2* out, const float2* tf, const FuseOp& op, int n_tiles, int Y,
                   int Xh, cudaStream_t s);

// Transfer-function build.
struct TfArgs {
  const wo_optics* optics;  // device copy, [n_tiles]
  int* counts;              // [n_tiles][4]: #(S and P) (binary source), #P, x band limit, -
  float4* rec;              // [n_tiles][Y][X] pupil record
  float2* arms;             // [n_tiles][n_arms][Z][Y][X]
  float2* tf;               // [n_tiles][n_kinds][Z][Y][Xh]
  float* stats;             // [n_tiles][8]
  int n_tiles, Z, Y, X;
  int lf_props;             // 0..2 (phase, absorption present -> slots)
  int want_phase, want_abs, want_fl;
  int n_arms;               // 2*(lf) + fl, or 4 with want_dz
  int n_kinds;
  int want_dz;              // phase TF and dH/d(defocus): arms A, B, A', B'; kinds 2
  int want_grad;            // plus dH/d(tilt_x, tilt_y, NA_ill): arms A_tx, A_ty, A_na; kinds 5
  int smooth;               // smooth-edged source pupil (S a float in [0, 1])
  float4* rec2;             // [n_tiles][Y][X] (dS/dtx P, dS/dty P, dS/dNA P, W - rint(W)), want_grad or aberrated
  const double* zern;       // [n_tiles][n_zern] Zernike coefficients (waves, Noll order), device copy
  int n_zern;               // 0: unaberrated detection pupil
  int arms_stage;           // arm pass: eta / source derivatives staged in shared memory (set at launch)
  int x_cols;               // half-spectrum columns the y and z passes transform; beyond them every
                            // tile's TFs vanish (Xh when the optics are not known on the host)
  float* norm_part;         // [n_tiles][record blocks][4] partial sums of S P and dS P
  float* norms;             // [n_tiles][4]: sum S P, then sum dS/dtheta P (smooth source)
  int rec_blocks;           // record blocks per tile
  long long row_begin, row_end;  // PSF-row pass: rows (t*Z + j)*Y + y in [begin, end)
  int kxm;                  // the bank is kx-major, [n_tiles][n_kinds][Xh][Z][Y] (WO_TF_KX_MAJOR)
};
cudaError_t tf_pupil_record(const TfArgs& a, cudaStream_t s);
int record_rows(int Y, int n_tiles);  // rows per pupil-record block
cudaError_t tf_arms(const TfArgs& a, cudaStream_t s);
// Arm pass with register-resident y transforms (wo_armsreg.cu): banks without derivatives, Y <= 192.
bool arms_reg_supported(int Y, const TfArgs& a);
cudaError_t tf_arms_reg(const TfArgs& a, cudaStream_t s);
cudaError_t tf_psf_rows(const TfArgs& a, cudaStream_t s);
// The TF build's z pass for one-kind banks with register-resident z
// transforms (wo_zreg.cu).
bool tf_zpass_reg_supported(const TfArgs& a);
cudaError_t tf_zpass_reg(const TfArgs& a, cudaStream_t s);
// kx-major banks and spectra (WO_TF_KX_MAJOR; [block][Xh][Z][Y] complex):
// PSF rows of length X whose pair kernel writes them (square planes, Y = X,
// of Z = 32 or 48 planes) (wo_psf.cu); the plane engine's shapes and
// kernels (wo_plane.cu): the TF build's y and z transforms with the
// regulariser maxima, and the y and z transforms with a one-volume operator
// between them, in place; status: the workspace's status block (bounded
// waits on the planes' bulk copies).
bool psf_kxm_supported(int X, int Y, int Z);
bool plane_supported(int Z, int Y);
cudaError_t tf_plane_yz(const TfArgs& a, int* status, cudaStream_t s);
// Hybrid column engine (wo_colhyb.cu) and the schedule table (wo_sched.cu).
bool cols_hyb_supported(int N);
cudaError_t cols_c2c_hyb(int N, bool inverse, float2* data, long long col_stride, long long plane_stride, int ncols,
                         long long nplanes, cudaStream_t s, const char* name, long long groups,
                         long long group_stride);
int cols_engine(int n);  // WO_ENGINE_SMEM or WO_ENGINE_HYBRID
// The x and y transforms of a plane in one kernel per direction (wo_xy.cu),
// and the helpers that pick it or the two passes by the schedule table.
bool xy_supported(int X, int Y);
int xy_engine(int X, int Y);  // WO_ENGINE_HYBRID: the fused kernels
cudaError_t xy_fwd(int X, int Y, const float* in, float2* out, long long nplanes, RowBg bg, cudaStream_t s);
cudaError_t xy_inv(int X, int Y, const float2* in, float* out, long long nplanes, float scale, RowBg bg,
                   cudaStream_t s);
cudaError_t plane_xy_fwd(int X, int Y, const float* in, float2* out, long long nplanes, RowBg bg, cudaStream_t s);
cudaError_t plane_xy_inv(int X, int Y, float2* in, float* out, long long nplanes, float scale, RowBg bg,
                         cudaStream_t s);
int rows_engine(int n);  // engine of the x passes for n complex points (wo_rowsreg.cu: HYBRID)
bool rows_reg_supported(int N);
cudaError_t rows_r2c_reg(int N, const float* in, float2* out, long long nrows, RowBg bg, cudaStream_t s);
// The tiles of a field as the rows' source (wo_rowsreg.cu): tile t = (ty, tx)
// of a tiles_y x tiles_x grid covers field rows ty*core - halo .. and
// columns tx*core - halo .., mirror-padded outside the field [Z][Yf][Xf]
// (Yf = tiles_y core, Xf = tiles_x core); tile rows in [tile][z][row] order,
// 2N = core + 2 halo samples each.  The same values wo_tile_gather would
// write, read in place.
struct FieldSrc {
  const float* field;
  int Z, tiles_y, tiles_x, core, halo;
};
cudaError_t rows_r2c_field(int N, const FieldSrc& f, float2* out, long long nrows, RowBg bg, cudaStream_t s);
// kx-major x passes (wo_rowsreg.cu): real rows of 2N points, Y rows per plane;
// supported for N = 32, 64, 96 when a warp's rows (32 / T) divide Y.  The
// forward pass reads the tiles of a field (out: [tile][N+1][Z][2N]); the
// inverse writes real rows [block][Z][Y][2N] from [block][N+1][Z][Y].
bool rows_kxm_supported(int N, int Y);
cudaError_t rows_r2c_field_kxm(int N, const FieldSrc& f, float2* out, long long nrows, RowBg bg, cudaStream_t s);
cudaError_t rows_c2r_kxm(int N, const float2* in, float* out, long long nrows, int Z, int Y, float scale, RowBg bg,
                         cudaStream_t s);
// The forward pass from volumes [block][Z][Y][2N] (square planes, Y = 2N)
// into [block][N+1][Z][Y].
cudaError_t rows_r2c_kxm(int N, const float* in, float2* out, long long nrows, int Z, int Y, RowBg bg,
                         cudaStream_t s);
// The inverse x pass of a field's tiles fused with their blend into the
// field (wo_rowsreg.cu): field [P][Z][tiles_y core][tiles_x core], the same
// values as the inverse x pass into tiles followed by wo_tile_blend.
struct FieldDst {
  float* field;
  int P, Z, tiles_y, tiles_x, core, halo;
};
cudaError_t rows_c2r_blend(int N, const float2* spec, const FieldDst& f, float scale, cudaStream_t s);
cudaError_t rows_c2r_reg(int N, const float2* in, float* out, long long nrows, float scale, RowBg bg,
                         cudaStream_t s);
// Register-resident variant of the PSF-row pass for short rows (wo_psf.cu).
bool psf_rows_reg_supported(int X, int n_arms);
cudaError_t tf_psf_rows_reg(const TfArgs& a, cudaStream_t s);
cudaError_t tf_zpass(const TfArgs& a, cudaStream_t s);

// Auto-tuning: per-tile value and derivatives of the 2D thin-object loss from
// a data spectrum [tile][Z][Y][Xh] and a bank of 1 + np slots per tile (H,
// then dH/dtheta_p); frequencies above nu_max (cycles/um, > 0) are left out.
// zf: Z for 3D spectra (Parseval over z puts a factor Z on the eta term and
// on the normalisation), 1 for per-plane 2D spectra.  value [tile],
// grad [tile][np].  `partials` holds tune_partials_bytes(n_tiles, Y, X, np).
cudaError_t tune_reduce(const float2* tf2, const float2* spec, const wo_optics* optics, int n_tiles, int Z,
                        int Y, int X, float eta, float nu_max, int zf, int loss, int np, double* partials,
                        double* value, double* grad, cudaStream_t s);
size_t tune_partials_bytes(int n_tiles, int Y, int X, int np);
// Vector-Jacobian product of the phase reconstruction in the tuned optics:
// spectra D [tile][Z][Y][Xh] (3D or per plane), upstream spectra G
// [tile][Z][Y][Xh] (3D) or [tile][Y][Xh] (2D), bank of 1 + np slots per tile;
// grad [tile][np].
cudaError_t vjp_reduce(const float2* tf2, const float2* spec, const float2* gspec, int n_tiles, int Z, int Y, int X,
                       float eta, int mode3d, int np, double* partials, double* grad, cudaStream_t s);
struct AdamLr {
  double v[4];  // step sizes for defocus_um, tilt_x, tilt_y, na_ill
};
cudaError_t adam_optics(wo_optics* optics, const double* grad, int np, double* state, int n_tiles, AdamLr lr,
                        double b1, double b2, double eps, cudaStream_t s);
// Zero element 0 of each of n_tiles volumes of vol elements (the DC bin).
cudaError_t zero_dc(float2* spec, int n_tiles, long long vol, cudaStream_t s);
// Per-plane 2D spectra [tile][Z][plane]: subtract from each plane's DC bin the
// mean of the tile's DC bins (background = the stack's mean).
cudaError_t center_dc_planes(float2* spec, int n_tiles, int Z, long long plane, cudaStream_t s);

// Learned optics estimator (wo_est.cu).
size_t est_param_count();
size_t est_workspace_bytes(int B);
cudaError_t est_features(const float2* spec, const wo_optics* optics, int n, int Z, int Y, int X, float* feat,
                         cudaStream_t s);
cudaError_t est_thin_phantom(const float4* par, int n, int S, int Y, int X, float pixel, float dz, float* out,
                             cudaStream_t s);
cudaError_t est_to_bf16(const float* w, void* wb, cudaStream_t s);
cudaError_t est_forward(const void* wb, const float* w32, const float* feat, int B, const float* h_scale,
                        const float* h_offset, float* phys, void* ws, cudaStream_t s);
cudaError_t est_backward(const void* wb, const float* w32, const float* feat, const float* phys_target, int B,
                         const float* h_scale, const float* h_offset, float* grad, float* loss, void* ws,
                         cudaStream_t s);
cudaError_t est_adam(float* w32, void* wb, const float* grad, float* m, float* v, int step, float lr, float b1,
                     float b2, float eps, cudaStream_t s);
float* est_grad_buffer(void* ws, int B);
// The estimator's convolutions on the tensor cores (wo_estmma.cu): layer
// 0..3, bfloat16 weights wb (element offsets woff, boff of the flat
// parameter array), float32 activations [B][C][H][H].  Backward: weight and
// bias gradients of the layer into grad, and (gx != NULL) the gradient at its
// input masked by xin > 0; part holds part_floats floats of scratch.
cudaError_t est_conv_fwd_mma(int layer, const float* x, const void* wb, const void* wt, const float* w32,
                             long long woff, long long boff, int B, float* y, cudaStream_t s);
cudaError_t est_conv_bwd_mma(int layer, const float* gy, const float* xin, const void* wt, long long woff,
                             long long boff, int B, float* gx, float* part, size_t part_floats, float* grad,
                             cudaStream_t s);
// wt: the layers' weights re-laid for the staging copies (est_conv_prep_elems()
// bfloat16), made from wb by est_conv_prep before a forward or backward pass.
size_t est_conv_prep_elems();
cudaError_t est_conv_prep(const void* wb, const long long* woff, void* wt, cudaStream_t s);

// Tiles.
cudaError_t tiles_gather(const float* field, int Z, int ty, int tx, int core, int halo,
                         float* tiles, cudaStream_t s);
cudaError_t tiles_blend(const float* tiles, int Z, int ty, int tx, int core, int halo,
                        float* field, cudaStream_t s);

// Let a kernel take `bytes` of dynamic shared memory: the opt-in attribute is
// needed once its static plus dynamic shared memory passes 48 KB, and is set
// once per (kernel, device) for the largest size asked (the attribute belongs
// to the device's context): a registry of the granted sizes, kept by wo_api.cu.
size_t smem_attr_granted(const void* kernel, int device);
void smem_attr_mark(const void* kernel, int device, size_t bytes);
template <class K>
inline cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes == 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (smem_attr_granted((const void*)kernel, dev) >= bytes) return cudaSuccess;
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if (fa.sharedSizeBytes + bytes > 48 * 1024)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) smem_attr_mark((const void*)kernel, dev, bytes);
  return e;
}

}  // namespace wo

#define WO_LAUNCH(name, stream, ...)        \
  do {                                      \
    int _wo_tok = -1;                       \
    wo::prof_begin(name, stream, &_wo_tok); \
    __VA_ARGS__;                            \
    wo::prof_end(_wo_tok, stream);          \
  } while (0)

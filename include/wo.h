/*
 * wo.h - C ABI of the GB300 (sm_103a) library for WaveOrder's linear
 * wave-optical imaging model and its Tikhonov inverse (arxiv 2412.09775).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - Volumes are float32, x contiguous: [n_tiles][channel or property][Z][Y][X].
 * - Spectra use the unnormalised forward DFT; inverses carry 1/N.  Transfer
 *   functions are stored as the non-redundant half spectrum
 *   [Z][Y][X/2+1] of interleaved complex64 (re, im), FFT order, not shifted.
 * - Frequencies nu = k / (N * pixel) with k in FFT order; plane j of a stack
 *   sits at focal displacement z_j = k_j * z_step + defocus (k_j in FFT order),
 *   boundaries are periodic in x, y and z.
 * - Properties, in this order, for the kinds present in `kinds`:
 *   WO_TF_PHASE -> index increment dn, WO_TF_ABSORPTION -> extinction index
 *   kappa, WO_TF_FLUOR -> fluorophore density.  Channels: one brightfield
 *   stack if any label-free kind is present, then one fluorescence stack if
 *   WO_TF_FLUOR is.  The two contrast modes are independent (block-diagonal
 *   operator, Eq. fwd_block).
 * - Supported lengths: Y, Z and X/2 must each be 1 or 2^a * 3^b with
 *   b <= 1 and the value <= 2048 (see wo_size_supported); X must be even.
 *
 * Ownership and errors
 * --------------------
 * The caller allocates every device buffer (for example as torch tensors)
 * and keeps it alive until the work queued on `stream` has finished.  The
 * library never allocates or frees device memory and never synchronises the
 * device (except wo_sync_status and wo_autotune, which say so); all work is
 * queued on `stream`.  Device pointers must be 16-byte
 * aligned.  Every entry point validates its arguments before launching
 * anything; on an error status nothing was launched and no output was
 * touched.  A failed CUDA launch returns WO_ERR_CUDA (the queue may then hold
 * partial work).  Host arrays (h_*) are read during the call only.
 *
 * The API is not re-entrant across host threads that share one workspace.
 */
#ifndef WO_H
#define WO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *wo_stream;

typedef enum {
  WO_OK = 0,
  WO_ERR_ARG = 1,              /* null or misaligned pointer, bad count or flag */
  WO_ERR_SHAPE = 2,            /* inconsistent shape (odd X, tile grid mismatch) */
  WO_ERR_UNSUPPORTED_SIZE = 3, /* an FFT length outside the supported set */
  WO_ERR_UNDERSAMPLED = 4,     /* optics alias on this grid (see wo_build_tf) */
  WO_ERR_CUDA = 5,             /* a CUDA launch or runtime call failed */
  WO_ERR_TIMEOUT = 6,          /* a bounded device-side wait expired (the tile pipeline of
                                  WO_PASS_RECON; reported through wo_sync_status) */
  WO_ERR_OPTICS = 7,           /* physically invalid optics (e.g. NA_det >= n) */
  WO_ERR_WORKSPACE = 8,        /* workspace smaller than wo_workspace_bytes() */
  WO_ERR_BOUNDS = 9            /* a kernel of a WO_CHECK build found an index outside its
                                  buffer and skipped the access (reported through
                                  wo_sync_status) */
} wo_status;

/* Per-tile optical parameters theta (Fig. 2a(ii); Ext. Data Fig. 3a-b).
 * Lengths in micrometres; NA and tilts in NA units (n * sin(angle)). */
typedef struct {
  double lambda_um;   /* vacuum wavelength */
  double n_medium;    /* refractive index of the medium */
  double pixel_um;    /* sample-plane pixel size (x and y) */
  double z_step_um;   /* distance between stack planes */
  double na_det;      /* detection NA, 0 < na_det < n_medium */
  double na_ill;      /* illumination NA, >= 0 (0: a single source point) */
  double tilt_x;      /* illumination tilt (pupil centre) along x */
  double tilt_y;      /* illumination tilt (pupil centre) along y */
  double defocus_um;  /* focal offset z_offset added to every plane */
} wo_optics;

enum { WO_TF_PHASE = 1, WO_TF_ABSORPTION = 2, WO_TF_FLUOR = 4 };
/* A bank of two TF slots per tile for defocus auto-tuning (used alone, never
 * or-ed with the kinds above): slot 0 the 3D phase TF, slot 1 its derivative
 * with respect to the tile's defocus_um, dH/dz0 (per um).  The defocus enters
 * both pupil arms through e^{i2pi eta z_j}, so the derivative arms are
 * A' = i2pi eta A and B' = i2pi eta B, and dH1 = c sum (A'* B + A* B') / sum S P^2
 * goes through the same Table 1 combination and z-DFT as H1.  Supported for
 * X <= 768.  wo_forward, wo_forward_adjoint and wo_reconstruct accept such a
 * bank with this kinds value and use its phase slot (a phase-only system). */
enum { WO_TF_PHASE_DZ = 8 };
/* Or-ed with WO_TF_PHASE_DZ only: keep the per-plane 2D TFs H_j(nu_perp) and
 * dH_j/dz0 (slot layout unchanged, index j = plane instead of axial bin; the
 * z-DFT is not applied and the statistics block holds only the optics
 * status).  Such a bank serves wo_tune_objective alone, which then takes
 * per-plane data spectra (wo_spectrum, WO_MODE_2D) and skips a z transform
 * per step; the operators reject it (WO_ERR_ARG). */
enum { WO_TF_PLANES = 16 };
enum { WO_LOSS_DATA = 0, WO_LOSS_MIDBAND = 1 };
/* Or-ed with label-free kinds (phase, absorption, WO_TF_PHASE_DZ): the source
 * pupil gets a logistic edge one frequency bin of the coarser axis wide,
 *   S = 1 / (1 + exp(-(NA_ill/lambda - |nu - t/lambda|) / w)),  w = 1/(min(Y,X) p),
 * instead of the closed disk, and sum S P^2 becomes a float sum: the model in
 * which the illumination tilt and NA_ill have derivatives.  The detection
 * pupil stays binary. */
enum { WO_TF_SMOOTH_SOURCE = 32 };
/* A bank of five per-plane TF slots for tuning defocus and illumination
 * (requires WO_TF_PLANES; implies WO_TF_SMOOTH_SOURCE): slot 0 the phase TF,
 * then its derivatives in defocus_um, tilt_x, tilt_y and na_ill.  The source
 * enters the direct arm A = S P e^{i2pi eta z_j} and the normalisation
 * D = sum S P^2, so dH1/dtheta = c sum (A_theta* B) / D - H1 D_theta / D with
 * A_theta = (dS/dtheta) P e^{...}, D_theta = sum (dS/dtheta) P^2, through
 * Table 1 unchanged.  X must be 32, 48, 64, 96, 128, 192 or 256. */
enum { WO_TF_PHASE_GRAD = 64 };
/* Or-ed with exactly one of WO_TF_PHASE, WO_TF_ABSORPTION, WO_TF_FLUOR (and
 * optionally WO_TF_SMOOTH_SOURCE): the bank's half spectra are stored
 * kx-major, [n_tiles][1][X/2+1][Z][Y] complex64 (the Z x Y plane of every
 * half-spectrum column k_x contiguous; same size, same statistics block).
 * The build then runs its y and z transforms, and an operator with such a
 * bank its y and z transforms and the per-frequency operator between them, as
 * one pass per (tile, k_x) plane on the chip (TMA bulk copies of the plane
 * into shared memory; one trip through HBM instead of three), and the x
 * passes transpose on the way in and out.  Supported for Z = 32 or 48 and
 * square planes Y = X = 64, 128 or 192, and for Z = 16 with Y = X = 64 (else
 * WO_ERR_UNSUPPORTED_SIZE).  Accepted by wo_build_tf, wo_build_tf_device, and
 * with the same kinds value by wo_forward, wo_forward_adjoint, and in
 * WO_MODE_3D by wo_reconstruct, wo_reconstruct_shared_tf and
 * wo_reconstruct_field_tiles (square tiles, E = Y = X); the 2D solve,
 * wo_restore_field and the tuning calls reject such a bank (WO_ERR_ARG).  The
 * planes of k_x outside a tile's own TF support disk hold the PSF rows'
 * rounding noise (of the order of 1e-7 of the largest TF value) instead of
 * transformed noise: the operators write zeros there without reading them.
 * The plane kernels wait
 * for their copies with a bound; a wait that runs out records WO_ERR_TIMEOUT
 * in the workspace's status block (wo_sync_status). */
enum { WO_TF_KX_MAJOR = 128 };
enum { WO_MODE_3D = 0, WO_MODE_2D = 1 };
enum { WO_ETA_RELATIVE = 0, WO_ETA_ABSOLUTE = 1 };

/* 1 if n is a supported FFT length, else 0. */
int wo_size_supported(int n);

/* Bytes of a transfer-function bank for these arguments: the half spectra
 * [n_tiles][n_kinds][Z][Y][X/2+1] complex64, followed (at the next 256-byte
 * boundary) by a per-tile statistics block [n_tiles][8] of 32-bit words that
 * the TF build fills: float max_nu sum_lf|H|^2, float max_nu_perp
 * sum_kz sum_lf|H|^2, the same two for fluorescence (used by the relative
 * regulariser), int32 optics status (see wo_build_tf_device), float support
 * radius r in cycles per pixel (every TF of the tile is zero where
 * (k_y/Y)^2 + (k_x/X)^2 > r^2: r = (R p + 2/min(Y, X)), R = (NA_det +
 * min(NA_det, NA_ill + |t|))/lambda for label-free kinds, 2 NA_det/lambda for
 * fluorescence or the smooth source, the largest over the kinds present,
 * two bins of margin), two reserved.  The z passes of the operators skip
 * the frequencies outside that disk (their outputs are zero there).
 * 0 on invalid arguments. */
size_t wo_tf_bytes(int n_tiles, int Z, int Y, int X, unsigned kinds);

/* Workspace bytes that suffice for every entry point with these arguments.
 * 0 on invalid arguments. */
size_t wo_workspace_bytes(int n_tiles, int Z, int Y, int X, unsigned kinds);

/* Rows a1-a4.  Build the scalar 3D weak-object transfer functions of every
 * tile from its optics (Table 1, scalar column; Methods "Summary of transfer
 * functions"):
 *   S  = 1[|nu - t/lambda| <= NA_ill/lambda],  P = 1[|nu| <= NA_det/lambda]
 *   A_j = S P e^{i2pi eta z_j},  B_j = P (i/eta) e^{i2pi eta z_j},
 *   eta = sqrt((n/lambda)^2 - |nu|^2)
 *   H1_j(q) = c sum_nu A_j*(nu) B_j(nu+q) / sum S P^2,  c = 2 pi n dz / lambda^2
 *   [H_re_j; H_im_j] = [[1, 1], [i, -i]] [H1_j(q); H1_j(-q)*]
 *   H_fl_j(q) = sum_nu P_j*(nu) P_j(nu+q),  P_j = P e^{i2pi eta z_j}
 * then a DFT over j gives the 3D TFs; H_fl is scaled to H_fl(0) = 1.
 * h_optics: n_tiles host structs.  d_tf: wo_tf_bytes() bytes (output).
 * Returns WO_ERR_OPTICS if a tile has NA_det >= n, NA_ill + |t| > n or a
 * non-positive length; WO_ERR_UNDERSAMPLED if
 * (NA_det + NA_ill + |t|)/lambda >= 1/(2 pixel) (the pupil correlation would
 * alias) or (n/lambda)(1 - sqrt(1 - (NA_det/n)^2)) >= 1/(2 z_step).
 * With the optics on the host the y and z transforms of the build cover the
 * half-spectrum columns k_x up to the batch's largest TF support radius plus
 * two bins; the columns beyond hold the PSF rows' rounding noise (of the
 * order of 1e-7 of the largest TF value) instead of exact zeros. */
wo_status wo_build_tf(const wo_optics *h_optics, int n_tiles, int Z, int Y, int X,
                      unsigned kinds, void *d_tf, void *d_ws, size_t ws_bytes,
                      wo_stream stream);

/* Rows a1-a4 with the optics in device memory (n_tiles structs at d_optics,
 * 8-byte aligned, caller-owned, read by the kernels): the form to capture in
 * a CUDA graph or to drive from parameters updated on the device (one
 * parameter vector theta per tile, Fig. 2a(ii)).  The optics cannot be
 * checked on the host, so the kernels apply the same checks per tile: a tile
 * that fails them gets all-zero transfer functions and its status
 * (WO_ERR_OPTICS or WO_ERR_UNDERSAMPLED) as an int32 in element 4 of its row
 * of the statistics block (0 for valid tiles); reconstructions of such a tile
 * are zero.  Shape, pointer and workspace errors are returned as usual. */
wo_status wo_build_tf_device(const wo_optics *d_optics, int n_tiles, int Z, int Y, int X,
                             unsigned kinds, void *d_tf, void *d_ws, size_t ws_bytes,
                             wo_stream stream);

/* Rows a1-a4 with an aberrated detection pupil (row f4; Ext. Data Fig. 3b:
 * the detection branch takes N_z Zernike coefficients besides NA_det and the
 * defocus).  The detection pupil becomes
 *   P = 1[|nu| <= NA_det/lambda] exp(i 2 pi W(nu)),  W = sum_j c_j Z_j(rho, phi),
 *   rho = |nu| lambda / NA_det,  phi = atan2(nu_y, nu_x),
 * Z_j Noll's Zernike polynomials (j = 1 piston, 2/3 tilt along x/y, 4
 * defocus, 5/6 astigmatism, 7/8 coma, 11 primary spherical, ...; unit RMS
 * over the pupil), c_j in waves.  The paper does not fix the ordering,
 * normalisation or unit; this is the convention of this library.  P enters
 * every arm (A = S P e^{...}, B = P (i/eta) e^{...}, P_j = P e^{...}), so
 * every kind, including the derivative banks, takes the aberration; the
 * normalisations use |P|^2, which it leaves unchanged.  The TFs lose the
 * parity of the unaberrated ones and stay Hermitian (real PSFs).  A tilt
 * c_2 = s NA_det / (2 lambda) shifts every PSF by -s along x.
 * h_zernike: [n_tiles][n_zernike] host doubles (c_1 .. c_n_zernike per tile),
 * read during the call; 0 <= n_zernike <= WO_MAX_ZERNIKE (radial orders up
 * to 7); n_zernike = 0 is wo_build_tf.  Non-finite coefficients: WO_ERR_ARG.
 * The workspace must hold wo_aberrated_workspace_bytes() bytes; the bank
 * has the layout of wo_tf_bytes() and serves every operator as usual. */
#define WO_MAX_ZERNIKE 36
size_t wo_aberrated_workspace_bytes(int n_tiles, int Z, int Y, int X, unsigned kinds);
wo_status wo_build_tf_aberrated(const wo_optics *h_optics, const double *h_zernike,
                                int n_zernike, int n_tiles, int Z, int Y, int X,
                                unsigned kinds, void *d_tf, void *d_ws, size_t ws_bytes,
                                wo_stream stream);

/* Row a5.  Forward model (Eq. fwd, Eq. fwd_block, Fourier form):
 *   d_c = IFFT3( sum_p H_cp FFT3(f_p) ) + b_c
 * d_f: [n_tiles][P][Z][Y][X] properties (input); d_data: [n_tiles][C][Z][Y][X]
 * (output).  h_background: C host floats (NULL: zero). */
wo_status wo_forward(const void *d_tf, unsigned kinds, const float *d_f,
                     const float *h_background, float *d_data, int n_tiles,
                     int Z, int Y, int X, void *d_ws, size_t ws_bytes,
                     wo_stream stream);

/* Row a6.  Adjoint of the forward model's linear part:
 *   f_p = IFFT3( sum_c conj(H_cp) FFT3(d_c - b_c) )
 * d_data: [n_tiles][C][Z][Y][X] (input); d_f: [n_tiles][P][Z][Y][X] (output).
 * h_background: C host floats (NULL: zero). */
wo_status wo_forward_adjoint(const void *d_tf, unsigned kinds, const float *d_data,
                             const float *h_background, float *d_f, int n_tiles,
                             int Z, int Y, int X, void *d_ws, size_t ws_bytes,
                             wo_stream stream);

/* Row a7.  Tikhonov reconstruction per contrast mode (Eq. recon; its
 * one-step solution Eq. tls_solution): per frequency
 *   F = (H^H H + eta_abs I)^-1 H^H D~,   D~_c(0) = D_c(0) - N b_c
 * computed in the equivalent form H^H (H H^H + eta_abs I)^-1 D~.
 * h_eta: one value per contrast mode present (label-free first, then
 * fluorescence).  eta_flag WO_ETA_RELATIVE: eta_abs = eta * max_nu
 * sum_{c,p}|H_cp|^2 of that mode and tile; WO_ETA_ABSOLUTE: eta_abs = eta.
 * h_background: C host floats, or NULL for the per-channel mean (the
 * reconstruction then has zero mean).
 * mode WO_MODE_3D: d_f is [n_tiles][P][Z][Y][X].
 * mode WO_MODE_2D (phase from defocus; Methods "Cell-scale optical pooled
 * screen data"): a thin object at the reference plane, every plane of the
 * stack one channel of a per-transverse-frequency solve; d_f is
 * [n_tiles][P][Y][X] and eta_abs uses max_nu_perp sum_j sum_{c,p} |H_cp,j|^2. */
wo_status wo_reconstruct(const void *d_tf, unsigned kinds, const float *d_data,
                         const float *h_background, const float *h_eta,
                         int eta_flag, int mode, float *d_f, int n_tiles, int Z,
                         int Y, int X, void *d_ws, size_t ws_bytes, wo_stream stream);

/* Row a7 for a batch of independent stacks imaged with the same optics (the
 * many small z-stacks of a pooled screen, Methods "Cell-scale optical pooled
 * screen data"): wo_reconstruct with one transfer-function bank for the whole
 * batch.  d_tf: a bank built for ONE tile (wo_tf_bytes(1, Z, Y, X, kinds)
 * bytes), read by every stack; d_data [n_tiles][C][Z][Y][X], d_f as in
 * wo_reconstruct; the relative regulariser uses that bank's statistics.  The
 * workspace holds wo_workspace_bytes(n_tiles, ...) bytes.  Same errors as
 * wo_reconstruct. */
wo_status wo_reconstruct_shared_tf(const void *d_tf, unsigned kinds, const float *d_data,
                                   const float *h_background, const float *h_eta, int eta_flag, int mode,
                                   float *d_f, int n_tiles, int Z, int Y, int X, void *d_ws, size_t ws_bytes,
                                   wo_stream stream);

/* Allocation-free reconstruction.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory where they need a
 * reconstruction - a plugin inside a host application that owns the whole
 * device-memory budget, code behind a caching allocator it may not bypass, or
 * a latency-bound loop that must not pay cudaMalloc/cudaFree's implicit
 * device synchronisation.  Same arguments and result as wo_reconstruct minus
 * the workspace: the workspace is a device array of WO_STATIC_SCRATCH_BYTES
 * (32 MiB) inside the library, which every GPU that loads the library holds
 * until the process exits.  The caller still provides d_tf, d_data and d_f.
 * - Problems whose wo_workspace_bytes() exceeds WO_STATIC_SCRATCH_BYTES are
 *   rejected with WO_ERR_WORKSPACE before anything is launched (for example
 *   16x64x64 with all three kinds needs 2 MB; 96x512x512 does not fit).
 * - The first call on a device looks up the array's device address with that
 *   device current (and loads the array there); make that first call before
 *   any stream capture begins.  Later calls outside capture look the address
 *   up again (a reset or replaced context is followed); calls made while the
 *   stream is captured use the address of the last call on that device.
 * - The function allocates nothing (no cudaMalloc, cudaFree or allocating
 *   library routine).
 * - All calls on a device share the one array and it keeps the previous
 *   call's contents; nothing in it needs to start at zero.  Calls whose work
 *   overlaps on the GPU (different streams, or different host threads) race
 *   on the array: order them on one stream. */
#define WO_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
wo_status wo_reconstruct_static(const void *d_tf, unsigned kinds, const float *d_data,
                                const float *h_background, const float *h_eta, int eta_flag,
                                int mode, float *d_f, int n_tiles, int Z, int Y, int X,
                                wo_stream stream);

/* Multi-channel fusion (9-aperture fusion, Results: several illumination
 * apertures fused into one phase estimate; Eq. recon with C channels and
 * P = 1): per frequency
 *   F = sum_c conj(H_c) D~_c / (sum_c |H_c|^2 + eta_abs),
 * D~_c the spectrum of channel c with its background removed from the DC bin
 * (h_background[c], or the channel's mean when h_background is NULL).
 * WO_MODE_3D: per 3D frequency, d_f [n_tiles][Z][Y][X].  WO_MODE_2D: the thin
 * object, per transverse frequency with the sums over every plane of every
 * channel, d_f [n_tiles][Y][X].  eta_flag: WO_ETA_ABSOLUTE, or
 * WO_ETA_RELATIVE for eta_abs = eta * max_nu sum_c |H_c(nu)|^2 (3D) or
 * eta * max_nu_perp sum_j sum_c |H_cj|^2 (2D), per tile.
 * d_tf: a WO_TF_PHASE bank built for n_tiles * n_channels entries, channel
 * c of tile t at entry t * n_channels + c (each with that aperture's optics).
 * d_data: [n_tiles][n_channels][Z][Y][X].  1 <= n_channels <= 16.  The
 * workspace holds wo_fused_workspace_bytes() bytes (0 on invalid arguments). */
size_t wo_fused_workspace_bytes(int n_channels, int n_tiles, int Z, int Y, int X);
wo_status wo_reconstruct_fused(const void *d_tf, int n_channels, const float *d_data,
                               const float *h_background, float eta, int eta_flag, int mode,
                               float *d_f, int n_tiles, int Z, int Y, int X, void *d_ws,
                               size_t ws_bytes, wo_stream stream);

/* Row a8 (gather).  Cut a field [Z][tiles_y*core][tiles_x*core] into
 * overlapping tiles [tiles_y*tiles_x][Z][E][E], E = core + 2*halo, tile
 * (ty, tx) starting at field pixel (ty*core - halo, tx*core - halo); pixels
 * outside the field are mirror-padded (-i, 2(n-1)-i).  Requires
 * 0 <= halo, 2*halo <= core (Fig. 2a(i); Methods "Organelle-scale ..."). */
wo_status wo_tile_gather(const float *d_field, int Z, int tiles_y, int tiles_x,
                         int core, int halo, float *d_tiles, wo_stream stream);

/* Rows a8 + a7: wo_reconstruct of the tiles of a field without gathering
 * them first.  The result (d_f [tiles_y*tiles_x][P][Z][E][E], E = core +
 * 2 halo) equals, bit for bit, wo_tile_gather of d_field [Z][tiles_y*core]
 * [tiles_x*core] followed by wo_reconstruct on the tiles with the same
 * arguments: the reconstruction's first pass reads each tile's rows from the
 * field in place (mirror-padded at the field's edges), so the gathered
 * copy never goes to memory.  The TF bank holds one bank per tile (in tile
 * order ty*tiles_x + tx); kinds must describe one data channel (phase and/or
 * absorption, or fluorescence alone: else WO_ERR_ARG); E/2 must be one of
 * the register row lengths (32, 48, 64, 96, 128, 192, 256, 512: else
 * WO_ERR_UNSUPPORTED_SIZE); 0 <= halo, 2*halo <= core, tiles_y*tiles_x <=
 * 65535 (else WO_ERR_ARG).  The workspace is wo_workspace_bytes(tiles_y *
 * tiles_x, Z, E, E, kinds); h_background, h_eta, eta_flag and mode as for
 * wo_reconstruct (NULL background: each tile's mean). */
wo_status wo_reconstruct_field_tiles(const void *d_tf, unsigned kinds, const float *d_field, int Z,
                                     int tiles_y, int tiles_x, int core, int halo,
                                     const float *h_background, const float *h_eta, int eta_flag,
                                     int mode, float *d_f, void *d_ws, size_t ws_bytes,
                                     wo_stream stream);

/* Rows a8 + a7 + a8: restore a field in one call — the reconstruction of
 * its tiles read in place (as wo_reconstruct_field_tiles) with the last pass
 * blending the reconstructed tiles straight into d_out [P][Z][tiles_y*core]
 * [tiles_x*core] (WO_MODE_2D: [P][tiles_y*core][tiles_x*core]), so neither
 * the gathered nor the reconstructed tiles go to memory.  Equal, bit for
 * bit, to wo_reconstruct_field_tiles followed by wo_tile_blend of each
 * property.  Arguments as for wo_reconstruct_field_tiles; also tiles_x <= 64
 * and d_out != d_field (else WO_ERR_ARG). */
wo_status wo_restore_field(const void *d_tf, unsigned kinds, const float *d_field, int Z, int tiles_y,
                           int tiles_x, int core, int halo, const float *h_background,
                           const float *h_eta, int eta_flag, int mode, float *d_out, void *d_ws,
                           size_t ws_bytes, wo_stream stream);

/* Row a8 (blend).  Stitch tiles back: field = sum_t w_t tile_t / sum_t w_t
 * with separable linear-ramp weights w(u) = min(1, (u+1/2)/(2 halo),
 * (E-u-1/2)/(2 halo)) per axis (linearly weighted distance-to-edge blending). */
wo_status wo_tile_blend(const float *d_tiles, int Z, int tiles_y, int tiles_x,
                        int core, int halo, float *d_field, wo_stream stream);

/* Row f4, padding in place of circular boundaries.  The operators above are
 * periodic in x, y and z (the Fourier form of Eq. fwd); to get other
 * boundaries, pad the stacks to a larger supported grid, build the TFs and
 * run the operator there, and crop the result back.
 * wo_pad: d_in [n_vol][Z][Y][X] -> d_out [n_vol][Zp][Yp][Xp], the input at
 * offset (oz, oy, ox) = ((Zp-Z)/2, (Yp-Y)/2, (Xp-X)/2) (integer halves), the
 * margin filled per `mode`: WO_PAD_ZERO zeros, WO_PAD_EDGE the nearest edge
 * sample, WO_PAD_MIRROR the mirror image about the edge samples (index -i
 * and 2(n-1) - i, periodic with period 2(n-1) for margins wider than the
 * volume; a length-1 axis repeats its sample).  wo_crop: the window of shape
 * (Z, Y, X) at the same offset, d_in [n_vol][Zp][Yp][Xp] -> d_out
 * [n_vol][Z][Y][X].  Out of place (WO_ERR_ARG if d_in == d_out; other
 * overlaps are undefined); Zp >= Z >= 1 etc., else WO_ERR_SHAPE; any sizes
 * (the FFT-length rules apply to the padded grid's operators, not here). */
enum { WO_PAD_ZERO = 0, WO_PAD_MIRROR = 1, WO_PAD_EDGE = 2 };
wo_status wo_pad(const float *d_in, int n_vol, int Z, int Y, int X, int Zp, int Yp, int Xp,
                 int mode, float *d_out, wo_stream stream);
wo_status wo_crop(const float *d_in, int n_vol, int Zp, int Yp, int Xp, int Z, int Y, int X,
                  float *d_out, wo_stream stream);

/* Defocus auto-tuning (Results, physics-guided auto-tuning of the optical
 * parameters theta; Fig. 2a(iv); Ext. Data Fig. 3; Methods, optical pooled
 * screen data: 2D phase from a z-stack, Adam, fixed regulariser).
 *
 * wo_spectrum: the half spectra [n_tiles][Z][Y][X/2+1] complex64 of n_tiles
 * brightfield stacks d_data [n_tiles][Z][Y][X]: 3D spectra (WO_MODE_3D) or
 * each plane's 2D spectrum (WO_MODE_2D), with the background b removed:
 * b = h_background[0], or the stack's mean when h_background is NULL.  In 3D
 * the DC bin becomes D(0) - N b (0 for the mean); in 2D every plane's DC bin
 * becomes D_j(0) - N_perp b.  d_spec holds n_tiles*Z*Y*(X/2+1)*8 bytes
 * (caller-owned, 16-byte aligned).  Same shape rules as wo_forward. */
wo_status wo_spectrum(const float *d_data, const float *h_background, int mode, void *d_spec,
                      int n_tiles, int Z, int Y, int X, wo_stream stream);

/* wo_tune_objective: per tile, a loss of the 2D thin-object reconstruction
 * and its derivatives with respect to the tile's tuned optics parameters: the
 * defocus alone (kinds with WO_TF_PHASE_DZ) or defocus, tilt_x, tilt_y and
 * NA_ill (WO_TF_PHASE_GRAD; d_grad [n_tiles][4] in that order).  The formulas
 * below are written for the defocus; every other parameter takes its own
 * dH slot in place of dH.
 *
 * loss = WO_LOSS_DATA: the loss of the 2D thin-object fit (every
 * plane j sees the object at the reference plane through the per-plane phase
 * TF H_j) at its Tikhonov minimiser, and its derivative with respect to the
 * tile's defocus:
 *   L(z0) = min_f sum_j ||d_j - b - H_j(z0) f||^2 + eta ||f||^2
 *         = (1/N_perp) sum_nu [ sum_j |D_j - H_j F|^2 + eta |F|^2 ],
 *   F(nu) = sum_j H_j* D_j / (sum_j |H_j|^2 + eta),
 *   dL/dz0 = (1/N_perp) sum_nu -2 Re sum_j (dH_j F)* (D_j - H_j F)
 * (the derivative needs no derivative of F because F minimises the
 * bracket).  kinds = WO_TF_PHASE_DZ | WO_TF_PLANES evaluates these sums over
 * the planes j from per-plane banks and spectra; kinds = WO_TF_PHASE_DZ
 * evaluates the same value over the axial bins k of 3D banks and spectra
 * (Parseval over z: sum_j = (1/Z) sum_k, so eta enters as Z eta and the
 * normalisation as 1/(N_perp Z)).  Transverse frequencies
 * with |nu| > nu_max (cycles/um) are left out of both sums when nu_max > 0
 * (0 or +inf: all frequencies): the loss of the band-limited data, whose
 * minimum in z0 is wider.  eta is absolute (>= 0).
 *
 * loss = WO_LOSS_MIDBAND: the paper's image-quality loss, minus the power of
 * the reconstruction F in the mid band c/8 <= |nu| <= c/4 of the transverse
 * cutoff c = (NA_det + NA_ill)/lambda:
 *   L(z0) = -(1/N_perp) sum_band |F|^2,
 *   dL/dz0 = -(2/N_perp) sum_band Re(F* dF),  dF = (sum_j dH_j* D_j - F dh) / (h + eta),
 *   h = sum_j |H_j|^2, dh = 2 Re sum_j H_j* dH_j
 * (F is not the minimiser of this loss, so the derivative goes through the
 * solve).  nu_max is ignored.
 * d_tf: a bank of these kinds for the same tiles; d_optics: the device optics
 * the bank was built from (8-byte aligned; pixel_um sets the frequency grid);
 * d_spec: wo_spectrum of the data in the matching mode.  d_value: n_tiles
 * doubles, d_grad: n_tiles x n_params doubles (8-byte aligned; either may be
 * NULL, not both).  The workspace needs n_tiles * ceil(Y*(X/2+1)/256) *
 * 8 * (1 + n_params) bytes, which wo_workspace_bytes() of the bank's kinds
 * covers; the sums are reduced in a fixed order (repeatable to the bit).  No host synchronisation: the call can be captured in a CUDA
 * graph together with wo_build_tf_device and wo_adam_optics. */
wo_status wo_tune_objective(const void *d_tf, unsigned kinds, const wo_optics *d_optics,
                            const void *d_spec, int loss, float eta, float nu_max, double *d_value,
                            double *d_grad, int n_tiles, int Z, int Y, int X, void *d_ws,
                            size_t ws_bytes, wo_stream stream);

/* wo_reconstruct_vjp: the hand-written adjoint of the phase reconstruction
 * with respect to the tuned optics (Ext. Data Fig. 3: the paper
 * back-propagates a loss of the reconstruction to each tile's parameters).
 * Given the upstream gradient g = dL/df of a loss L of the reconstruction f,
 * it returns dL/dtheta_p = <g, df/dtheta_p> per tile, the reconstruction
 * taken with an absolute regulariser eta (>= 0) and the background removed as
 * d_spec was made:
 *   WO_MODE_3D (kinds WO_TF_PHASE_DZ, a 3D bank; theta = defocus_um): f the 3D
 *     reconstruction of wo_reconstruct, F = conj(H) D / (|H|^2 + eta) per 3D
 *     frequency; d_spec the 3D spectra (wo_spectrum, WO_MODE_3D); d_gout
 *     [n_tiles][Z][Y][X].
 *   WO_MODE_2D (kinds WO_TF_PHASE_DZ | WO_TF_PLANES, theta = defocus_um, or
 *     WO_TF_PHASE_GRAD | WO_TF_PLANES, theta = (defocus_um, tilt_x, tilt_y,
 *     na_ill)): f the thin-object reconstruction of wo_reconstruct's 2D mode,
 *     F = sum_j conj(H_j) D_j / (sum_j |H_j|^2 + eta) per transverse
 *     frequency (Parseval over z: the same f as WO_MODE_2D with a 3D bank of
 *     the same optics and absolute eta); d_spec the per-plane spectra
 *     (wo_spectrum, WO_MODE_2D); d_gout [n_tiles][Y][X].
 * In both: dF_p = (conj(dH_p) D - 2 Re(conj(H) dH_p) F) / den with the sums
 * over planes in 2D, and dL/dtheta_p = (1/N) Re sum_nu conj(G) dF_p (G the
 * unnormalised spectrum of g, N its number of samples).  d_grad: n_tiles x
 * n_params doubles (8-byte aligned).  The workspace holds the upstream
 * spectra and the partial sums: wo_workspace_bytes() of the bank's kinds
 * suffices.  The sums are reduced in a fixed order; no host synchronisation. */
wo_status wo_reconstruct_vjp(const void *d_tf, unsigned kinds, const void *d_spec, const float *d_gout, float eta,
                             int mode, double *d_grad, int n_tiles, int Z, int Y, int X, void *d_ws, size_t ws_bytes,
                             wo_stream stream);

/* wo_adam_optics: one Adam step (Kingma and Ba, 2015) on each tile's tuned
 * optics parameters in the device optics array - defocus_um (n_params = 1),
 * or defocus_um, tilt_x, tilt_y, na_ill (n_params = 4) - from d_grad
 * [n_tiles][n_params]:
 *   m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2,  s = s + 1,
 *   theta -= lr_p (m / (1 - b1^s)) / (sqrt(v / (1 - b2^s)) + eps);
 * with four parameters NA_ill is then kept inside [0.01, n - |tilt| - 1e-3].
 * d_state: n_tiles x n_params x {m, v, s} doubles, zeroed by the caller
 * before the first step and kept on the device, so a captured graph of build
 * + objective + step replays as further Adam iterations.  h_lr: n_params
 * host step sizes >= 0; 0 <= b1, b2 < 1, eps > 0; device pointers 8-byte
 * aligned. */
wo_status wo_adam_optics(wo_optics *d_optics, const double *d_grad, int n_params, double *d_state,
                         int n_tiles, const double *h_lr, double beta1, double beta2, double eps,
                         wo_stream stream);

/* Learned optics estimator (no counterpart in the paper: the workload asks
 * for a learned starting point of auto-tuning).  Features: per tile, a
 * 3 x 64 x 64 float image from the per-plane 2D spectra of its stack
 * (wo_spectrum, WO_MODE_2D, channel-mean background), planes in natural
 * order as rows (Z <= 64, zero rows below), 64 radial bins of |nu| up to
 * 2 NA_det/lambda as columns:
 *   ch0 = log(1 + P / mean P),  P = sum_bin |D_r|^2            (power profile)
 *   ch1 = sum_bin Im(D_{r+1} D_r*) nu_x/|nu| / sum_bin |D_{r+1}| |D_r|
 *   ch2 = the same with nu_y                                  (plane-to-plane drift)
 * The power profile locates the in-focus plane (the defocus with its sign),
 * the drift follows the illumination tilt.  wo_est_features: d_feat
 * [n_tiles][3][64][64] (caller-owned).
 * Network: conv 3x3 3->32 (stride 1), 32->64, 64->96, 96->128 (stride 2), zero
 * padding 1, ReLU; global average pool; linear 128->4.  Parameters: one flat
 * float32 array of wo_est_param_count() values (each conv W [co][ci][3][3]
 * then its bias, then the linear W [4][128] and bias) and a bfloat16 copy
 * (uint16 storage, same offsets) from which every weight is read; sums are
 * float32.  Outputs are standardised; h_scale / h_offset (4 host floats
 * each, scale != 0) map them to physical units, out = scale * net + offset,
 * and targets back.  wo_est_forward: d_out [batch][4] physical values.
 * wo_est_backward: mean squared error of the standardised outputs and its
 * gradient (d_grad: param_count floats, or NULL to keep it in the
 * workspace; d_loss: one float or NULL).  wo_est_train_step: backward, then
 * one Adam step (Kingma and Ba, 2015; b1 0.9, b2 0.999, eps 1e-8, 1-based
 * step) on the float32 weights with moments d_m, d_v (param_count floats
 * each, zeroed before the first step) and a refresh of the bfloat16 copy.
 * wo_est_sync_bf16: the bfloat16 copy from the float32 weights (round to
 * nearest even).  All device arrays 16-byte aligned; 1 <= batch <= 4096;
 * workspace wo_est_workspace_bytes(batch).
 * wo_thin_phantom: the training specimens, [n_tiles][Y][X] float: spheres
 * (d_params [n_tiles][n_spheres][4] floats: centre y, centre x, radius in
 * um, index increment) projected along z on the periodic tile, as the
 * increment of one plane of thickness z_step: sum dn 2 sqrt(r^2 - rho^2) / dz. */
size_t wo_est_param_count(void);
size_t wo_est_workspace_bytes(int batch);
/* Byte offset, in the estimator's workspace, of convolution layer `layer`'s
 * output (1..4: float32 [batch][C][H][H] after its ReLU) as the last
 * wo_est_forward / wo_est_backward / wo_est_train_step of that batch size
 * left it: the network's ReLU decisions, for comparisons with a reference
 * that decides them in another precision.  Layer 1's output starts the
 * workspace (offset 0); 0 on invalid arguments for the other layers. */
size_t wo_est_activation_offset(int batch, int layer);
wo_status wo_est_sync_bf16(const float *d_w32, void *d_wbf16, wo_stream stream);
wo_status wo_est_forward(const void *d_wbf16, const float *d_w32, const float *d_feat, int batch,
                         const float *h_scale, const float *h_offset, float *d_out, void *d_ws,
                         size_t ws_bytes, wo_stream stream);
wo_status wo_est_backward(const void *d_wbf16, const float *d_w32, const float *d_feat,
                          const float *d_target, int batch, const float *h_scale,
                          const float *h_offset, float *d_grad, float *d_loss, void *d_ws,
                          size_t ws_bytes, wo_stream stream);
wo_status wo_est_train_step(float *d_w32, void *d_wbf16, float *d_m, float *d_v,
                            const float *d_feat, const float *d_target, int batch,
                            const float *h_scale, const float *h_offset, int step, float lr,
                            float *d_loss, void *d_ws, size_t ws_bytes, wo_stream stream);
wo_status wo_est_features(const void *d_spec, const wo_optics *d_optics, int n_tiles, int Z, int Y,
                          int X, float *d_feat, wo_stream stream);
wo_status wo_thin_phantom(const float *d_params, int n_tiles, int n_spheres, int Y, int X,
                          double pixel_um, double z_step_um, float *d_out, wo_stream stream);

/* Schedules and the autotuner (no counterpart in the paper).  A pass with
 * more than one implementation runs the engine its schedule table names.
 * WO_PASS_COLS: the complex transforms along a strided axis (every y pass,
 * the z transforms of wo_spectrum), per length n: WO_ENGINE_SMEM (shared-
 * memory Stockham stages, radix 8, B columns per block) or WO_ENGINE_HYBRID
 * (coalesced tile copies, a register-resident four-step transform per column
 * with one shared-memory transpose; lengths 32, 48, 64, 96, 128, 192, 256,
 * 512).  WO_ENGINE_DEFAULT restores the built-in choice.  Results do not
 * depend on the engine beyond float32 rounding.
 * wo_schedule_set: WO_ERR_ARG on a bad pass, length or engine,
 * WO_ERR_UNSUPPORTED_SIZE for an engine that lacks the length.
 * wo_schedule_get: the engine in use for (pass, n), -1 on bad arguments.
 * wo_autotune: times every engine of the column transforms that an entry
 * point on these shapes launches (lengths Y and Z, batches as large as the
 * workspace allows up to three volumes per tile) and of the x passes (X/2
 * points, the rows of the same volumes), on the workspace (its
 * contents are destroyed), and keeps the fastest in the table (the non-default
 * engine only when at least 2 % faster).  It waits for
 * the stream (it measures with events), so it is not for graph capture; run
 * it once before capturing.  The table is process-wide. */
enum { WO_PASS_COLS = 0 };
/* WO_PASS_ROWS: the real <-> half-spectrum transforms along x (the first and
 * last pass of every operator and of wo_spectrum), per n = X/2 complex
 * points: WO_ENGINE_SMEM (rows staged in shared memory, Stockham stages) or
 * WO_ENGINE_HYBRID (each row held by T lanes of one warp straight from global
 * memory, register-resident four-step transform, the Hermitian split by warp
 * shuffles; n = 32, 48, 64, 96, 128, 192, 256, 512; the default where it
 * exists). */
enum { WO_PASS_ROWS = 1 };
/* WO_PASS_RECON: the phase-only 3D reconstruction (wo_reconstruct,
 * wo_reconstruct_shared_tf with kinds WO_TF_PHASE, optionally with
 * WO_TF_SMOOTH_SOURCE, or a WO_TF_PHASE_DZ bank, WO_MODE_3D) of tiles whose
 * planes fit one SM's shared memory, keyed by n = Y: WO_ENGINE_SMEM (the five
 * passes, each a kernel over the whole batch) or WO_ENGINE_HYBRID (one
 * kernel: CTAs take per-plane x/y work, per-row z-solve work and per-plane
 * inverse x/y work from one queue in ticket order, so a tile's spectra stay
 * in L2 between them; available for (Z, Y, X) = (48, 192, 192),
 * (48, 128, 128), (16, 64, 64)).  The default is WO_ENGINE_SMEM, the faster
 * on this part (the pipeline holds one plane per SM and cannot overlap one
 * item's copies with another's transforms).  Every wait of that kernel on another CTA's
 * work is bounded (one second): when it runs out, the kernel records
 * WO_ERR_TIMEOUT in the workspace's status block (wo_sync_status) and stops.
 * Results agree with the passes to float32 rounding. */
enum { WO_PASS_RECON = 2 };
/* WO_PASS_XY: the x and y transforms of a plane (the first two and last two
 * passes of every operator, and of wo_spectrum and the gradient), keyed by
 * n = Y for square planes X = Y: WO_ENGINE_SMEM (the x pass and the y pass,
 * each a kernel over the batch) or WO_ENGINE_HYBRID (one kernel per
 * direction: a cluster of two CTAs per plane transforms its rows along x,
 * exchanges the bins through distributed shared memory and transforms its
 * columns along y, so the intermediate spectrum never goes to memory;
 * n = 64, 128, 192).  The default is WO_ENGINE_SMEM: the fused kernels hold
 * a plane tile of about 109 KB per CTA (192 x 192), two CTAs per SM, and
 * measured slower on the 256-tile field; wo_autotune picks them where they
 * are faster.  Results agree to float32 rounding. */
enum { WO_PASS_XY = 3 };
enum { WO_ENGINE_DEFAULT = 0, WO_ENGINE_SMEM = 1, WO_ENGINE_HYBRID = 2 };
wo_status wo_schedule_set(int pass, int n, int engine);
int wo_schedule_get(int pass, int n);
wo_status wo_autotune(int n_tiles, int Z, int Y, int X, unsigned kinds, void *d_ws,
                      size_t ws_bytes, wo_stream stream);

/* Device-side errors.  Errors found on the device - a bounded wait of the
 * tile pipeline that ran out (WO_ERR_TIMEOUT), an index check of a WO_CHECK
 * build (WO_ERR_BOUNDS) - cannot be returned by the call that queued the
 * kernel.  They are recorded in the status block: the first 256 bytes of the
 * workspace (int32 code, site, detail; the first error since the block was
 * last cleared is kept).  Workspaces sized by wo_workspace_bytes and
 * wo_fused_workspace_bytes begin with it.
 * wo_clear_status: zero the block (stream-ordered); do it once on a new
 *   workspace before its first use.
 * wo_sync_status: wait for `stream`, read the block, clear it, and return the
 *   recorded code (WO_OK if none); h_info (2 ints, or NULL) receives the site
 *   (1: a z-solve item waited for its tile's plane items, 2: an inverse plane
 *   item waited for the z-solve items, 3: a TMA copy into shared memory, 4+: a
 *   WO_CHECK kernel family) and the detail (tile index, or the offending
 *   index).  Unlike every other entry point it synchronises the stream.
 *   WO_ERR_CUDA if the block holds no status code (never cleared).
 * wo_pipeline_probe: a diagnostic of the tile pipeline's bounded waits.  It
 *   runs the pipeline of the phase-only 3D reconstruction (eta 1e-3
 *   absolute, channel-mean background) on a WO_TF_PHASE bank exactly as
 *   wo_reconstruct does, except that every wait gives up after budget_ns
 *   (1e3 .. 1e10) and, when 0 <= withhold < n_tiles, the plane items of tile
 *   `withhold` are never posted: the items waiting for them then run out of
 *   time, record WO_ERR_TIMEOUT (site 1, detail withhold) and the kernel
 *   returns instead of hanging.  withhold = -1 runs the pipeline whole.
 *   Shapes: those of WO_PASS_RECON's pipeline; the workspace of
 *   wo_workspace_bytes(n_tiles, Z, Y, X, WO_TF_PHASE). */
wo_status wo_clear_status(void *d_ws, wo_stream stream);
wo_status wo_sync_status(void *d_ws, int *h_info, wo_stream stream);
/* 1 for a WO_CHECK build of the library, else 0.  In a WO_CHECK build the
 * kernels test the index of each global-memory access against the extent of
 * the buffer it addresses; an access outside is skipped (never a fault) and
 * the first such index is recorded (WO_ERR_BOUNDS; site: 4 tile gather/blend,
 * 5 column transforms, 6 z passes, 7 x passes, 8 arms, 9 PSF rows; detail:
 * the index), which wo_sync_status returns when the workspace's own block is
 * clear. */
int wo_check_build(void);
wo_status wo_pipeline_probe(const void *d_tf, const float *d_data, float *d_f, int n_tiles, int Z, int Y, int X,
                            int withhold, long long budget_ns, void *d_ws, size_t ws_bytes, wo_stream stream);

/* Human-readable name of a status. */
const char *wo_status_string(wo_status status);

/* Instrumentation (no counterpart in the paper).  When enabled, every kernel
 * launch is bracketed by CUDA events on its stream and counted per kernel
 * family.  wo_profile_read waits for the recorded events, then fills up to
 * `cap` entries of names (static strings), launch counts and total
 * milliseconds, and returns the number of families; it resets the record. */
void wo_profile_enable(int on);
int wo_profile_read(const char **names, long long *launches, double *ms, int cap);

/* Total kernel launches queued by this library since load. */
long long wo_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* WO_H */

/*
 * graphic.h -- C ABI of the GB300 (sm_103a) library for the data-parallel
 * hot path of the GRAPHIC angular-differential-imaging reduction
 * (Hugelier et al., arXiv:1510.04331): Fourier recentring shift, angle-gated
 * median PSF subtraction, Fourier three-shear derotation, median collapse.
 *
 * General rules for every call below:
 *   - Cubes are FP32, C-contiguous [n_frames][n][n] (frame-major, row-major
 *     frames) in DEVICE memory owned by the caller, except in the *_host
 *     calls, whose cube and result pointers are HOST memory.  n is a power
 *     of two in [64, 1024]; the frame centre is pixel (row n/2, col n/2).
 *     Device cubes and results start on a 16-byte boundary (cudaMalloc and
 *     torch give 256); GRAPHIC_ERR_INVALID_ARG otherwise.
 *   - Per-frame parameter arrays (dx, dy, theta, parang) are HOST arrays of
 *     n_frames doubles, owned by the caller, read before the call returns.
 *   - n_frames == 0 is a no-op for graphic_shift and graphic_rotate (the
 *     pointers may then be NULL); the median calls need n_frames >= 1.
 *   - Calls are enqueued on the context's stream (graphic_set_stream; the
 *     legacy default stream otherwise) and wait for it before returning, so
 *     the returned status covers the device work.  in and out may be the
 *     same pointer (in place); partially overlapping buffers are undefined.
 *   - Return value: GRAPHIC_OK (0) or a negative GRAPHIC_ERR_* code; a
 *     message for the last failure of the calling thread is available from
 *     graphic_last_error().  On error the output contents are unspecified.
 *   - Inputs must be finite; a NaN or Inf seen on the device gives
 *     GRAPHIC_ERR_NONFINITE.
 *   - The library allocates its own device workspaces (plan arrays, the
 *     scratch of the rotation) on first use and keeps them per context until
 *     graphic_release() or graphic_destroy().
 */
#ifndef GRAPHIC_H
#define GRAPHIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRAPHIC_OK 0
#define GRAPHIC_ERR_INVALID_ARG -1   /* null pointer, bad size, bad parameter  */
#define GRAPHIC_ERR_UNSUPPORTED -2   /* n or n_frames outside what is built    */
#define GRAPHIC_ERR_OOM -3           /* device allocation failed               */
#define GRAPHIC_ERR_CUDA -4          /* CUDA runtime error                     */
#define GRAPHIC_ERR_NONFINITE -5     /* NaN or Inf in the input cube           */
#define GRAPHIC_ERR_TIMEOUT -6       /* bounded device wait ran out            */
#define GRAPHIC_ERR_INTERNAL -7      /* device-side consistency check failed   */

/* Largest frame count the median kernels take in one call. */
#define GRAPHIC_MAX_FRAMES_MEDIAN 2048

typedef struct graphic_ctx graphic_ctx;

/* Create a context bound to CUDA device `device`.  *out receives the handle.
 * Fails with GRAPHIC_ERR_UNSUPPORTED if the device is not sm_103. */
int graphic_create(graphic_ctx **out, int device);

/* Free every device and host resource of the context (waits for its stream). */
int graphic_destroy(graphic_ctx *ctx);

/* Free the context's workspaces (they are re-created on demand). */
int graphic_release(graphic_ctx *ctx);

/* Use `stream` (a cudaStream_t, may be NULL for the legacy default stream)
 * for every later call on this context.  The stream stays owned by the
 * caller. */
int graphic_set_stream(graphic_ctx *ctx, void *stream);

/* Message of the last failing call made by the calling thread ("" if none). */
const char *graphic_last_error(void);

/* ABI version: major * 10000 + minor * 100 + patch. */
int graphic_version(void);

/*
 * A cube in device memory with a frame stride, for cubes that are views into
 * larger buffers (a sub-range of frames of a bigger allocation, frames
 * padded to an alignment): frame t starts at data + t * frame_stride floats.
 * frame_stride == 0 means n*n (dense); otherwise frame_stride >= n*n and a
 * multiple of 4, so that every frame starts on a 16-byte boundary
 * (GRAPHIC_ERR_INVALID_ARG otherwise).  data is owned by the caller.  The
 * *_cube calls below are the plain calls with this description of their
 * cubes; the floats between frames are neither read nor written.
 */
typedef struct {
  float *data;           /* device pointer to frame 0 */
  int64_t n_frames;
  int32_t n;
  int32_t reserved_;     /* zero */
  int64_t frame_stride;  /* elements between frames, 0 = n*n */
} graphic_cube;

/*
 * Sub-pixel recentring shift (Sect. 3.3.1, shift theorem with the separable
 * 2-D phasor, on frames zero-padded to m = 2n).  Frame t is moved by
 * (dx[t], dy[t]) pixels: out(x, y) = in(x - dx, y - dy), computed as a row
 * pass then a column pass, each line padded to m (data at offset n/2),
 * transformed, multiplied by exp(-i 2 pi k d / m) on signed bins k (the
 * Nyquist bin by cos(pi d)), transformed back, cropped to the same n
 * samples.  |dx|, |dy| <= n/2 (GRAPHIC_ERR_INVALID_ARG otherwise).
 */
int graphic_shift(graphic_ctx *ctx, const float *in, float *out, int64_t n_frames, int32_t n,
                  const double *dx, const double *dy);

/*
 * Fourier three-shear rotation (Sect. 3.4, rotation matrix written as
 * S_x(-tan(theta/2)) S_y(sin theta) S_x(-tan(theta/2)), each shear a 1-D
 * Fourier shift per line of the 2x zero-padded frame).  Frame t is rotated
 * by theta_deg[t] degrees counter-clockwise about pixel (n/2, n/2): content
 * at (x, y) = (col - n/2, row - n/2) moves to (x cos - y sin, x sin + y cos).
 * theta = 90 q + theta' with q = floor(theta/90 + 1/2): the 90 q part is an
 * exact index map (zero where the source pixel is outside the frame), the
 * shears use theta' in [-45, 45) and are skipped when theta' == 0.
 * Uses a device scratch of (frames per chunk) * n * 2n floats.
 */
int graphic_rotate(graphic_ctx *ctx, const float *in, float *out, int64_t n_frames, int32_t n,
                   const double *theta_deg);

/*
 * Angle-gated median PSF subtraction (Sect. 3.3, reference-frame conditions
 * and a per-frame PSF built as a plain median, without coefficients).
 * annuli_edges[0] < ... < annuli_edges[n_edges-1] (pixels) define
 * n_edges - 1 annuli; pixel p (rho^2 = x^2 + y^2) belongs to annulus a when
 * edges[a]^2 <= rho^2 < edges[a+1]^2 and is set to 0 in every frame when it
 * belongs to none.  For annulus a, alpha_min = 2 asin(min(1, n_fwhm * fwhm /
 * (2 edges[a]))) (degrees); frame t's reference set is every frame k with
 * |parang[k] - parang[t]| > alpha_min, or, when that set is empty, the
 * frame(s) with the largest |parang[k] - parang[t]|.
 * out[t](p) = in[t](p) - median over the reference set of in[k](p), the
 * median taken in the IEEE total order, even counts averaging the two
 * middle values in FP32.  n_frames <= GRAPHIC_MAX_FRAMES_MEDIAN.
 */
int graphic_adi_subtract(graphic_ctx *ctx, const float *in, float *out, int64_t n_frames, int32_t n,
                         const double *parang_deg, double fwhm, double n_fwhm, const double *annuli_edges,
                         int32_t n_edges);

/*
 * Median collapse (Sect. 3.4, merge of the derotated frames): out(p) = median
 * over the n_frames frames of in[t](p), same median rule as above.  out is a
 * device buffer of n*n floats.  Any n_frames >= 1.
 */
int graphic_collapse_median(graphic_ctx *ctx, const float *in, int64_t n_frames, int32_t n, float *out);

/*
 * The four steps above on strided cubes (graphic_cube).  in and out must have
 * the same n and n_frames; in-place calls pass the same cube twice.
 */
int graphic_shift_cube(graphic_ctx *ctx, const graphic_cube *in, const graphic_cube *out, const double *dx,
                       const double *dy);
int graphic_rotate_cube(graphic_ctx *ctx, const graphic_cube *in, const graphic_cube *out, const double *theta_deg);
int graphic_adi_subtract_cube(graphic_ctx *ctx, const graphic_cube *in, const graphic_cube *out,
                              const double *parang_deg, double fwhm, double n_fwhm, const double *annuli_edges,
                              int32_t n_edges);
int graphic_collapse_median_cube(graphic_ctx *ctx, const graphic_cube *in, float *out);

/*
 * The whole reduction (Sect. 3, PSF subtraction then derotation and merge):
 * shift by (dx, dy) from `in` into `work`, median PSF subtraction in place in
 * `work`, derotation by theta = -parang in place in `work`, median collapse
 * of `work` into `out` (n*n).  `in` is only read; `work` holds n_frames*n*n
 * floats and may equal `in` (the input is then overwritten).
 */
int graphic_reduce(graphic_ctx *ctx, const float *in, float *work, int64_t n_frames, int32_t n,
                   const double *dx, const double *dy, const double *parang_deg, double fwhm, double n_fwhm,
                   const double *annuli_edges, int32_t n_edges, float *out);

/* graphic_reduce on strided cubes: in is only read, work (same n and
 * n_frames, its own stride) holds the intermediate frames, out is n*n. */
int graphic_reduce_cube(graphic_ctx *ctx, const graphic_cube *in, const graphic_cube *work, const double *dx,
                        const double *dy, const double *parang_deg, double fwhm, double n_fwhm,
                        const double *annuli_edges, int32_t n_edges, float *out);

/*
 * The same two calls with the paper's second reference-frame condition
 * (Sect. 3.3, maximum time separation): frame k is in frame t's reference
 * set only if also |times[k] - times[t]| < t_max, and the fallback for an
 * empty set takes the frames farthest in angle among those within t_max.
 * times: host array of n_frames (any unit, with t_max in the same unit);
 * NULL means no time condition (then identical to the plain calls).  The
 * times must be monotone along the order of the parallactic angles (as for
 * a transit observed in time order), else GRAPHIC_ERR_UNSUPPORTED; t_max
 * must be > 0 (GRAPHIC_ERR_INVALID_ARG).  With a time condition every pixel
 * takes the general median path (sort + membership sweep), not the faster
 * band path.
 */
int graphic_adi_subtract_ex(graphic_ctx *ctx, const float *in, float *out, int64_t n_frames, int32_t n,
                            const double *parang, const double *times, double t_max, double fwhm, double n_fwhm,
                            const double *annuli_edges, int32_t n_edges);
int graphic_reduce_ex(graphic_ctx *ctx, const float *in, float *work, int64_t n_frames, int32_t n,
                      const double *dx, const double *dy, const double *parang, const double *times, double t_max,
                      double fwhm, double n_fwhm, const double *annuli_edges, int32_t n_edges, float *out);

/*
 * graphic_reduce with HOST buffers: copies host_in (n_frames*n*n floats) to
 * a device cube the context owns, reduces it, copies the n*n result back to
 * host_out.  Pinned (page-locked) host memory gives the fastest copies.
 */
int graphic_reduce_host(graphic_ctx *ctx, const float *host_in, int64_t n_frames, int32_t n, const double *dx,
                        const double *dy, const double *parang_deg, double fwhm, double n_fwhm,
                        const double *annuli_edges, int32_t n_edges, float *host_out);

/*
 * graphic_rotate without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (an allocator policy that forbids it, a host application that
 * hands over only a stream and pre-allocated buffers, a path that must not
 * trigger allocator work).  Same arithmetic and result as graphic_rotate;
 * in, out: device cubes of the caller, n_frames x n x n floats; theta_deg:
 * host array of n_frames doubles; stream: cudaStream_t (NULL = legacy
 * default stream); runs on the CURRENT CUDA device and waits for `stream`.
 * No context is needed.  Its working memory is a 16 MiB static device
 * array inside the library (plus a small static plan array), which every
 * GPU that loads the library holds until the process exits; frames go
 * through it in chunks of 16 MiB / (8 n^2) frames.  A frame whose n x 2n
 * scratch exceeds 16 MiB is rejected with GRAPHIC_ERR_UNSUPPORTED.  The
 * first call on a device sets the device up (takes the static arrays'
 * device addresses, uploads the FFT tables): make that first call before
 * any stream capture.  All calls share the static arrays: calls that
 * overlap on the GPU (other streams, other host threads) race; serialise
 * them.
 */
int graphic_rotate_noalloc(const float *in, float *out, int64_t n_frames, int32_t n, const double *theta_deg,
                           void *stream);

/* ---- image-quality pre-processing (Sect. 3.2) --------------------------------- */

/*
 * Master sky (Sect. 3.2, master sky): sky(p) = median over the n_frames
 * frames of the values in[t](p) that are finite and lie outside frame t's
 * star mask, i.e. not within mask_r pixels of (mask_x[t], mask_y[t]) (x =
 * column, y = row; mask_x = mask_y = NULL: no mask).  Masked regions may
 * also be marked by NaN in `in`.  Same median rule as the collapse; NaN
 * where no value is left.  in: device n_frames x n x n; sky: device n x n;
 * mask arrays on the host.  Any n_frames >= 1.
 */
int graphic_sky_median(graphic_ctx *ctx, const float *in, int64_t n_frames, int32_t n, const double *mask_x,
                       const double *mask_y, double mask_r, float *sky);

/*
 * Sky subtraction (Sect. 3.2): out[t] = in[t] - skies[j], j the master sky
 * closest in time (|sky_times[j] - frame_times[t]| smallest, the lower j on a
 * tie).  skies: device n_skies x n x n (16-byte aligned); times on the host.
 * out may equal in.
 */
int graphic_sky_subtract(graphic_ctx *ctx, const float *in, float *out, int64_t n_frames, int32_t n,
                         const float *skies, int32_t n_skies, const double *frame_times, const double *sky_times);

/*
 * Bad pixel map (Sect. 3.2, bad pixel correction): map[p] = 1 when
 * |ref[p] - median(ref)| > C sigma, sigma the population standard deviation
 * of the n x n values of ref (FP64), the median by the rule above (FP32),
 * the comparison in FP64; else 0.  ref (a master dark or sky) and map
 * (uint8, n x n) are device buffers.  GRAPHIC_ERR_NONFINITE if ref holds a
 * non-finite value.
 */
int graphic_bad_pixel_map(graphic_ctx *ctx, const float *ref, int32_t n, double C, uint8_t *map);

/*
 * Bad pixel correction (Sect. 3.2), in place: in every frame the pixels
 * flagged in map (device n x n uint8, may be NULL) and the non-finite ones
 * are set to NaN, then, pass after pass, every NaN pixel with at least one
 * finite 8-neighbour takes the median of those neighbours (same median
 * rule), all pixels of a pass reading the previous pass's values, until none
 * is left: clumps fill from their border inwards.  GRAPHIC_ERR_NONFINITE if
 * a frame has no finite pixel at all (it is left NaN).  Uses the context's
 * scratch (n_frames x n x n floats).
 */
int graphic_bad_pixel_fix(graphic_ctx *ctx, float *cube, int64_t n_frames, int32_t n, const uint8_t *map);

/*
 * Registration (Sect. 3.1): per frame of the device cube in (n_frames x n x
 * n floats, any n >= 1), the star's centre and FWHM.
 *  1. Centroid: the seed is the brightest pixel (the first in row-major
 *     order on a tie); the patch is the 8-connected set of pixels above
 *     thresh reachable from it inside the box of half-size R around it
 *     (clipped to the frame).  The frame is registered when the seed is
 *     above thresh, the patch touches no box edge that lies inside the
 *     frame and min_size <= |patch| <= max_size; the centroid is the
 *     flux-weighted centre of mass of the patch (x = column, y = row).
 *  2. Moffat fit I(x, y) = I0 (beta - 1) / (pi alpha^2) (1 + rho^2 /
 *     alpha^2)^(-beta) + Bg, rho the distance to (x0, y0), by
 *     Levenberg-Marquardt over the window of half-size w around the rounded
 *     centroid (clipped): start x0, y0 = centroid, alpha = max(1,
 *     sqrt(|patch| / pi)), beta = 2.5, Bg = window minimum, I0 = sum of (v -
 *     Bg) over the window; damping lambda * diag(J^T J) from lambda = 1e-3
 *     (/10 on an accepted step, *10 on a rejected one or one leaving alpha
 *     <= 0 or beta <= 1, at most 10 tries); stop when an accepted step
 *     lowers the squared error by at most 1e-14 of it, when no try lowers
 *     it, or after 200 iterations.  FWHM = 2 alpha sqrt(2^(1/beta) - 1).
 * out: device n_frames x 8 doubles per frame: found (1.0 / 0.0), x0, y0,
 * FWHM, I0, alpha, beta, Bg (all 0 when not found).  iters: device
 * n_frames int32 (iterations made, 0 when not found) or NULL.  The fit
 * runs in two phases: the iteration above with the per-pixel model in FP32
 * (lambda floor 1e-6, stop at a drop <= 1e-7 of the squared error), then
 * the FP64 iteration above from its result; iters counts both (<= 400).  in must be
 * 16-byte aligned, 1 <= n <= 65535, 1 <= R <= 32, 1 <= w <= 32; the
 * context scratch holds 8 bytes a frame.  All arithmetic after the pixel
 * values is FP64.  GRAPHIC_ERR_NONFINITE if a frame holds a non-finite
 * value (its row of out is then zero).  Two kernel launches (frame
 * argmax, fit); synchronous.
 */
int graphic_register(graphic_ctx *ctx, const float *in, int64_t n_frames, int32_t n, double thresh, int32_t R,
                     int32_t min_size, int32_t max_size, int32_t w, double *out, int32_t *iters);

/* ---- photometric-accuracy and binning experiments (Sect. 4.2, 4.3) ----- */

/*
 * Median binning (Sect. 4.3: every B consecutive frames combined into one
 * median frame; the quick-look binning of Sect. 3.1): out[g](p) = median of
 * in[f](p) over the frames f of group g = [g B, min(n_frames, (g + 1) B)),
 * the last group possibly shorter, by the median rule of
 * graphic_collapse_median.  in: device n_frames x n x n; out: device
 * ceil(n_frames / B) x n x n (16-byte aligned, n as for the reduction).
 * B >= 1.  GRAPHIC_ERR_NONFINITE on a non-finite value.  Synchronous.
 */
int graphic_bin_median(graphic_ctx *ctx, const float *in, float *out, int64_t n_frames, int32_t n, int32_t B);

/*
 * Host helper for binned sequences: out[g] = mean of v over group g (FP64,
 * in order), e.g. the parallactic angle or time of a median bin (the paper
 * does not say which value a bin takes; its mean).  out: ceil(n / B).
 */
int graphic_bin_mean(const double *v, int64_t n, int32_t B, double *out);

/*
 * Fake companion injection (Sect. 4.2: companions added to the raw frames
 * at an angle that follows the field rotation), in place.  Companion j of
 * frame t sits at (xc[t] + r[j] cos(pa0[j] + parang[t]), yc[t] + r[j]
 * sin(pa0[j] + parang[t])) (x = column, y = row, degrees counter-clockwise
 * from +x; positions in FP64 on the host) with the Moffat profile of
 * Sect. 3.1, total flux flux[j] and the frame's alpha[t], beta[t]:
 * flux (beta - 1) / (pi alpha^2) (1 + rho^2 / alpha^2)^(-beta), evaluated in
 * FP32 on the square window of half-size `half` around the rounded position
 * (clipped to the frame) and added to the frame, companion after
 * companion.  cube: device n_frames x n x n (any n >= 1); all other arrays
 * on the host (parang, xc, yc, alpha, beta: n_frames; r, pa0, flux:
 * n_comp).  alpha > 0, beta > 1, 0 <= half <= 4096.  Synchronous.
 */
int graphic_inject(graphic_ctx *ctx, float *cube, int64_t n_frames, int32_t n, const double *parang,
                   const double *xc, const double *yc, int32_t n_comp, const double *r, const double *pa0,
                   const double *flux, const double *alpha, const double *beta, int32_t half);

/*
 * Aperture photometry (Sect. 4.2, recovered flux): out[k] = sum of img over
 * the pixels whose centres lie within `radius` of (x[k], y[k]) ((col -
 * x)^2 + (row - y)^2 <= radius^2, FP64).  img: device n x n; x, y, out:
 * host arrays of n_ap.  Synchronous.
 */
int graphic_aperture(graphic_ctx *ctx, const float *img, int32_t n, int32_t n_ap, const double *x, const double *y,
                     double radius, double *out);

/* ---- uneven batches --------------------------------------------------------- */

/* One cube of a batch: device cubes in/out (n_frames x n x n, out may equal
 * in), host per-frame shifts (NULL: 0) and rotation angles (degrees; may be
 * NULL when the item does not rotate), and which steps to apply. */
typedef struct {
  const float *in;
  float *out;
  int64_t n_frames;
  int32_t n;
  int32_t passes;              /* GRAPHIC_PASS_* mask; 0 means both steps */
  const double *dx;
  const double *dy;
  const double *theta_deg;
} graphic_batch_item;

#define GRAPHIC_PASS_SHIFT 1         /* recentring shift (Sect. 3.3.1)                */
#define GRAPHIC_PASS_ROTATE 2        /* three-shear rotation (Sect. 3.4)              */

#define GRAPHIC_BATCH_PER_CUBE 0     /* the per-call passes, cube after cube          */
#define GRAPHIC_BATCH_PERSISTENT 1   /* every frame in one persistent launch (graph)  */
#define GRAPHIC_BATCH_GROUPED 2      /* per-size launches over frame tables (graph)   */
#define GRAPHIC_BATCH_AUTO 3         /* the mode the schedule names (autotuner)       */

/*
 * Recentre and/or rotate every frame of every cube of an uneven batch (cubes
 * of different n and frame counts): out = rotate(shift(in, dx, dy), theta)
 * with both steps, the arithmetic of graphic_shift followed by
 * graphic_rotate (Sect. 3.3.1, 3.4); one step when `passes` names one.
 *   GRAPHIC_BATCH_PERSISTENT  all frames in ONE persistent kernel launch
 *     replayed from a CUDA graph while the batch keeps its layout; its work
 *     items (one group of line pairs of one pass of one frame) wait only on
 *     the previous pass of their own frame, with bounded waits
 *     (GRAPHIC_ERR_TIMEOUT).  Scratch: two waves of at most the schedule's
 *     batch_budget_mb each.
 *   GRAPHIC_BATCH_GROUPED  frames sorted by size into waves whose scratch
 *     fits group_budget_mb (L2-sized); each pass of a wave is one launch of
 *     that size's kernel over a table of frame pointers; waves run on
 *     group_streams concurrent branches of one CUDA graph (wave w reuses the
 *     scratch of wave w - group_streams), replayed while the layout holds.
 * Items may not overlap one another, except that an item's out may equal its
 * own in.  Synchronous: returns after the device finished.
 */
int graphic_batch_geom(graphic_ctx *ctx, const graphic_batch_item *items, int32_t n_items, int32_t mode);

/*
 * Autotuner: time the schedule candidates on this batch and keep the fastest
 * in the context -- for the per-call passes the intermediate per chunk of
 * frames (64..4096 MiB) and the kernel of 1024-point lines (one
 * warp per line pair with radix-32 stages, or the generic radix-16 kernel);
 * for the persistent executor the wave budget and CTAs per SM; for the
 * grouped executor the wave budget and the number of concurrent branches;
 * then the fastest batched mode (batch_mode, used by GRAPHIC_BATCH_AUTO).
 * Writes them to cache_path (JSON, may be NULL), which graphic_create reads
 * back from the file named by the environment variable GRAPHIC_TUNE_CACHE.
 * best_ms (may be NULL) receives the best per-cube, persistent and grouped
 * times (3 doubles).
 */
int graphic_autotune(graphic_ctx *ctx, const graphic_batch_item *items, int32_t n_items, const char *cache_path,
                     double *best_ms);

/* Schedule values, in order: chunk_mb, variant_1024, batch_budget_mb,
 * batch_ctas_per_sm, group_budget_mb, group_streams (1..8), batch_mode
 * (GRAPHIC_BATCH_PERSISTENT or GRAPHIC_BATCH_GROUPED) -- the first n. */
#define GRAPHIC_SCHEDULE_LEN 7
int graphic_get_schedule(graphic_ctx *ctx, int32_t *values, int32_t n);
int graphic_set_schedule(graphic_ctx *ctx, const int32_t *values, int32_t n);

/* ---- precision variant (tensor cores) --------------------------------------- */

#define GRAPHIC_PREC_FP32 0      /* FP32 radix-16 Stockham kernels (default)                */
#define GRAPHIC_PREC_BF16X3 1    /* DFT stages as BF16 hi+lo GEMMs, FP32 accumulation       */
#define GRAPHIC_PREC_FP16X3 2    /* DFT stages as FP16 hi+lo GEMMs, FP32 accumulation       */

/*
 * Arithmetic of the shift and rotation line passes of this context
 * (graphic_shift, graphic_rotate, graphic_reduce*, and graphic_batch_geom in
 * the per-cube and grouped modes) for frames of n = 1024 (2048-point
 * lines); other sizes keep the FP32 kernels.  With BF16X3 / FP16X3 every
 * 2048-point DFT runs as three radix stages (16, 16, 8), each one GEMM on
 * the tensor cores (tcgen05) with operands split into hi + lo parts of the
 * 16-bit type and the products hi.hi + lo.hi + hi.lo accumulated in FP32;
 * twiddles, phasors and the FP64 phase-argument reduction are those of the
 * FP32 path.  Error against the FP64 definition, relative to the frame
 * peak: about 1e-6 (FP16X3) and 1e-4 (BF16X3) per pass, against ~1e-7 for
 * FP32 (measured per step by the tests).  The persistent batch mode always
 * uses FP32.
 */
int graphic_set_precision(graphic_ctx *ctx, int32_t precision);
int graphic_get_precision(graphic_ctx *ctx, int32_t *precision);

/* ---- measurement support ------------------------------------------------ */

/* Kernel identifiers for graphic_profile_read. */
#define GRAPHIC_K_SHIFT_X 0
#define GRAPHIC_K_SHIFT_Y 1
#define GRAPHIC_K_ADI_MEDIAN 2
#define GRAPHIC_K_ROT_P1 3
#define GRAPHIC_K_ROT_P2 4
#define GRAPHIC_K_ROT_P3 5
#define GRAPHIC_K_COLLAPSE 6
#define GRAPHIC_K_BATCH 7
#define GRAPHIC_K_REG_ARGMAX 8
#define GRAPHIC_K_REG_FIT 9
#define GRAPHIC_K_BIN 10
#define GRAPHIC_K_ADI_BAND_PREP 11
#define GRAPHIC_K_ADI_BAND_SWEEP 12
#define GRAPHIC_K_COUNT 13

/* enable != 0: bracket every kernel launch of the context with CUDA events
 * on its stream and accumulate per-kernel device time and launch counts;
 * enable == 0 stops.  Enabling resets the counters. */
int graphic_profile(graphic_ctx *ctx, int enable);

/* Copy the accumulated device milliseconds and launch counts of the first
 * n kernels (ids above) into ms[] and launches[] (host arrays of n).  The
 * median PSF step is up to three kinds of interval: its general path
 * (GRAPHIC_K_ADI_MEDIAN, named "adi_general"), the band path's preparation
 * kernels (with the kernel that zeroes groups outside the annuli) and its
 * sweep kernels, one launch of each per bit-map width class; a grouped or
 * persistent batch call (GRAPHIC_K_BATCH) counts as one graph launch. */
int graphic_profile_read(graphic_ctx *ctx, double *ms, int64_t *launches, int32_t n);

/* Name of kernel id `k` (static string), NULL if out of range. */
const char *graphic_kernel_name(int32_t k);

/* Bytes of device workspace the context currently holds. */
int graphic_workspace_bytes(graphic_ctx *ctx, int64_t *bytes);

#ifdef __cplusplus
}
#endif

#endif /* GRAPHIC_H */

// Internal declarations shared by the CUDA translation units of the GRAPHIC
// GB300 library.  Not part of the C ABI (see include/graphic.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/graphic.h"

namespace graphic {

// Line-pass kinds: which lines of which buffer one launch transforms.
//   SHIFT_X  rows of an n x n frame, shift dx[f]             (Sect. 3.3.1)
//   SHIFT_Y  columns of an n x n frame, shift dy[f]          (Sect. 3.3.1)
//   ROT_P1   rows of rot90^q(frame) -> scratch rows of 2n, x-shear -a y (Sect. 3.4)
//   ROT_P2   columns of the n x 2n scratch, y-shear +s x     (Sect. 3.4)
//   ROT_P3   scratch rows -> frame rows, x-shear -a y        (Sect. 3.4)
enum LineKind { SHIFT_X = 0, SHIFT_Y = 1, ROT_P1 = 2, ROT_P2 = 3, ROT_P3 = 4 };

struct LineArgs {
  const float *in;       // frame cube (SHIFT_*, ROT_P1) or scratch (ROT_P2/P3)
  float *out;            // frame cube (SHIFT_*, ROT_P3) or scratch (ROT_P1/P2)
  const double *p0;      // per frame: dx (SHIFT_X) or a = tan(theta'/2) (ROT_*)
  const double *p1;      // per frame: dy (SHIFT_Y) or s = sin(theta') (ROT_*)
  const int *q;          // per frame: quarter turns (ROT_P1)
  int *status;           // device status word (bit 0: non-finite input)
  long long in_fstride;  // elements between consecutive frames of `in`
  long long out_fstride; // elements between consecutive frames of `out`
  int n;                 // frame side
  const float *const *in_tab;  // optional: frame f reads in_tab[f] instead of in + f in_fstride
  float *const *out_tab;       // optional: frame f writes out_tab[f] instead of out + f out_fstride
  // optional: the per-line shift parameters (phase splits, Nyquist weight,
  // phasor steps) precomputed by launch_line_params, lp_lines per frame
  // (1 for the shift passes, whose lines of a frame share their shift);
  // null: each CTA computes its lines' parameters itself (FP64)
  const void *lp_tab;
  int lp_lines;
};

// Record `msg` as the calling thread's last error (graphic_last_error) and
// return `code` (capi.cu).
int set_last_error(int code, const char *msg);

// Host plans and argument checks (capi.cu).
int validate_shift(const double *dx, const double *dy, int64_t T, int32_t n);
int validate_adi(const double *parang, int64_t T, double fwhm, double n_fwhm, const double *edges, int32_t n_edges);
// Angle-gated reference sets (Sect. 3.3): frames sorted by parallactic angle
// (stable), per annulus and sorted position s the set {k : |alpha_k -
// alpha_s| > alpha_min(r_a)} as sorted-position ranges [0, L) u [R, T),
// farthest frames when empty, and the rank band of each annulus' medians.
// With time stamps (times != null) also |t_k - t_s| < t_max: the frames
// within t_max form a window [A, B) of the angle order (times must be
// monotone along it), the set is [A, L) u [R, B) with L, R clipped to the
// window, the fallback takes the farthest frames within the window, and the
// band path is off (its rank band assumes the whole frame set).
struct AdiPlanHost {
  std::vector<int> perm;     // [T]
  std::vector<int> lr;       // [A][T][2]
  std::vector<int> ab;       // [T][2] time windows (empty without a time gate)
  std::vector<double> edge2; // [A+1]
  std::vector<int> band;     // [A][4]
  int wmax = 0;
  // band path (plan_band_path): event queries [A][T] (a_s | b_s << 16: frame s
  // is outside the reference set of the queries a_s <= i < b_s), the 4-pixel
  // groups of the band path class after class (0: no pixel in an annulus;
  // then bit map widths 1, 2, 4, 8, 16, 32 words), class offsets [8]; after
  // the classes, from gen_off on, the gen_n 8-pixel blocks (index p / 8)
  // with a pixel of an annulus that has no band: the general path's grid
  // (gen_off < 0: every block)
  std::vector<uint32_t> evq;
  std::vector<int> groups;
  std::vector<int> class_off;
  int gen_off = -1, gen_n = 0;
};
// Returns GRAPHIC_OK, or an error code (last error set) for times that are
// not monotone in the angle order or a t_max that is not > 0.
int plan_adi(const double *parang, int64_t T, double fwhm, double n_fwhm, const double *edges, int32_t n_edges,
             AdiPlanHost &ap, const double *times = nullptr, double t_max = 0.0);
// Band path tables of a plan for frames of side n (psf_band.cu); the groups
// of a geometry are cached.  band_scratch_bytes: the device scratch the band
// path of that plan needs.
int plan_band_path(AdiPlanHost &ap, int64_t T, int32_t n);
size_t band_scratch_bytes(const AdiPlanHost &ap, int64_t T);
// The band path works through its pixel groups in chunks whose tables fit
// the scratch it is given; kBandScratchMax bounds what callers allocate.
constexpr size_t kBandScratchMax = (size_t)256 << 20;

// Asynchronous context calls for the serving loop (capi.cu): a batch call on
// the context's stream without the final synchronisation (the status word is
// cleared first), the status word's copy to pinned host memory (valid once
// the stream reaches it), and an upper bound of the device workspace the
// context's batch calls hold.
int ctx_batch_async(graphic_ctx *c, const graphic_batch_item *items, int32_t n_items, int32_t mode);
const int *ctx_status_async(graphic_ctx *c);
size_t ctx_workspace_bound(const graphic_ctx *c, int32_t mode);
// Grouped batches: record and replay a graph (default) or launch directly.
void ctx_set_graph_batches(graphic_ctx *c, bool on);

// Device status bits.
constexpr int STATUS_NONFINITE = 1;
constexpr int STATUS_INTERNAL = 2;
constexpr int STATUS_TIMEOUT = 4;

// geom.cu
int geom_init_device();   // uploads the twiddle tables of the current device (0 = ok)
// variant_1024: 1024-point lines by one warp per line pair (1) or the generic kernel (0)
cudaError_t launch_line_pass(LineKind kind, const LineArgs &a, long long n_frames, cudaStream_t st,
                             int variant_1024 = 1);
// Parameter tables for the line passes (geom.cu): the parameters of every
// line of n_frames frames of pass `kind` (ROT_P1 and ROT_P3 share theirs),
// computed in FP64 by one thread per line into `out`, line_params_bytes(kind,
// n, n_frames) bytes; the lines per frame of the table is line_params_lines.
int line_params_lines(LineKind kind, int n);
size_t line_params_bytes(LineKind kind, int n, long long n_frames);
cudaError_t launch_line_params(LineKind kind, const LineArgs &a, long long n_frames, void *out, cudaStream_t st);

// Uneven batches (one persistent launch): per-frame descriptor ...
struct BatchFrame {
  const float *in;       // n x n input frame
  float *out;            // n x n output frame (shift then rotation)
  const float *rin;      // input of the rotation: out after a shift, else in
  float *scratch;        // n x 2n scratch slot of this frame's wave
  double dx, dy;         // recentring shift
  double a, s;           // tan(theta'/2), sin(theta')
  int q;                 // quarter turns
  int n;                 // frame side
  int wave;              // wave index (scratch ring slot = wave & 1)
  int ctas[5];           // work items of passes shift x, shift y, rotation 1, 2, 3 (0: pass not applied)
};
// ... and the work segments in hand-out order.
struct BatchSeg {
  int item0;             // first item of the segment
  int frame;
  int pass;              // 0..4
  int count;
};
struct BatchArgs {
  const BatchFrame *frames;
  const BatchSeg *segs;
  const int *seg_of_item;  // [total] segment of each item
  int nseg;
  int total;             // items in all
  int nframes;
  int *next;             // hand-out counter (zeroed before the launch)
  int *done;             // [5][nframes] finished items per (pass, frame) (zeroed)
  int *wave_done;        // [waves] finished rotation-pass-3 items per wave (zeroed)
  const int *wave_r3;    // [waves] rotation-pass-3 items per wave
  int *status;
  long long spin_limit;  // clock cycles a wait may take before STATUS_TIMEOUT
};
cudaError_t launch_batch_persistent(const BatchArgs &b, int ctas_per_sm, cudaStream_t st);

// tc.cu: line passes with the DFT stages on the tensor cores (frames of
// n = 1024 only), operands split into hi + lo parts of BF16 or FP16.
constexpr int PREC_FP32 = 0;
constexpr int PREC_BF16X3 = 1;
constexpr int PREC_FP16X3 = 2;
int tc_init_device();      // twiddles and DFT operand tables of the current device (0 = ok)
bool tc_supported(int n);
cudaError_t launch_line_pass_tc(LineKind kind, const LineArgs &a, long long n_frames, cudaStream_t st,
                                int precision);

// median.cu
struct AdiArgs {
  const float *in;
  float *out;
  const int *perm;       // [T] frame index at angle-sorted position s
  int perm_id;           // 1: perm is the identity (frames already in angle order)
  const int *lr;         // [A][T][2] (L, R) of the reference set of sorted frame s in annulus a
  const int *ab;         // [T][2] time window (A, B) of sorted frame s, A <= L <= R <= B (null: [0, T));
                         // the reference set is [A, L) u [R, B)
  const double *edge2;   // [A+1] squared annulus edges (FP64)
  const int *band;       // [A][4] (blo, bhi, W, 0): full-rank band holding every median the
                         // annulus needs, W = bitmap words per lane (0: general path)
  int *status;
  long long in_fs;       // elements between consecutive frames of in (n*n for dense cubes)
  long long out_fs;      // elements between consecutive frames of out
  int T;
  int n;
  int n_ann;             // A
  int wmax;              // largest W over the annuli (0: no band path)
  // band path (psf_band.cu), from plan_band_path
  const uint32_t *evq;   // [A][T] device
  const int *groups;     // device, class after class
  int class_off[8];      // host copy of AdiPlanHost::class_off
  int gen_list;          // 1: the general path runs on the gen_n blocks listed at groups + gen_off
                         // (AdiPlanHost::gen_off, gen_n); 0: on every 8-pixel block
  int gen_off, gen_n;
  char *band_scratch;    // device scratch of band_scratch_cap bytes (at least one group's tables)
  size_t band_scratch_cap;
  // optional hook around each group of launches (profiling): mark(user,
  // kind, 1) before and mark(user, kind, 0) after; kind 0 = general path,
  // 1 = band preparation (and the zero groups), 2 = band sweep
  void (*mark)(void *user, int kind, int begin);
  void *mark_user;
};
// *launched (may be null) receives the number of kernels launched (the
// general path when it has blocks, then the band path's launches).
cudaError_t launch_adi_median(const AdiArgs &a, cudaStream_t st, int *launched = nullptr);
// psf_band.cu: the band path's launches (zero groups, then per class the
// preparation and the sweep); *launched is incremented per kernel
cudaError_t launch_adi_band(const AdiArgs &a, cudaStream_t st, int *launched);

struct CollapseArgs {
  const float *in;
  float *out;
  int *status;
  long long T;
  int n;
  long long fs;          // elements between consecutive frames of in (0: n*n)
  // master-sky variant (launch_sky_median): values that are not finite or
  // lie within mask_r of the frame's (mask_x[t], mask_y[t]) are left out
  const double *mask_x;  // [T] device, may be null (no mask)
  const double *mask_y;
  double mask_r2;
};
cudaError_t launch_collapse(const CollapseArgs &a, cudaStream_t st);
cudaError_t launch_sky_median(const CollapseArgs &a, cudaStream_t st);

// prep.cu: image-quality pre-processing (Sect. 3.2)
cudaError_t launch_sky_subtract(const float *in, float *out, long long T, int n, const float *skies,
                                const int *sky_of_frame, cudaStream_t st);
// one radix pass over the keys of n_vals floats: histogram (256 bins, device,
// zeroed here) of digit `shift` among keys whose bits under pmask equal prefix
cudaError_t launch_key_histogram(const float *v, long long n_vals, uint32_t prefix, uint32_t pmask, int shift,
                                 unsigned int *hist, cudaStream_t st);
// FP64 sums: sums[0] += v, or with mean != null sums[1] += (v - *mean)^2
cudaError_t launch_frame_sums(const float *v, long long n_vals, const double *mean, double *sums, cudaStream_t st);
cudaError_t launch_bad_map(const float *ref, long long n_vals, const float *med, const double *thresh,
                           uint8_t *map, cudaStream_t st);
// bad pixel correction: mark (flagged or non-finite -> NaN), then passes
cudaError_t launch_bad_mark(float *cube, long long T, int n, const uint8_t *map, unsigned long long *nan_count,
                            cudaStream_t st);
cudaError_t launch_bad_pass(const float *src, float *dst, long long T, int n, unsigned long long *counts,
                            cudaStream_t st);

// register.cu: registration (Sect. 3.1), one CTA per frame
struct RegArgs {
  const float *in;   // T x n x n device
  double *out;       // T x 8 device: found, x0, y0, fwhm, I0, alpha, beta, Bg
  int *iters;        // T device: Levenberg-Marquardt iterations made
  int *status;
  long long T;
  int n;
  double thresh;
  int R, min_size, max_size, w;
};
// keys: device workspace of register_keys_bytes(T): the packed per-frame
// maxima that the argmax kernel writes and the fit reads, then the fit's
// frame counter (all zeroed by launch_register_argmax)
size_t register_keys_bytes(long long T);
cudaError_t launch_register_argmax(const RegArgs &a, unsigned long long *keys, cudaStream_t st);
cudaError_t launch_register_fit(const RegArgs &a, unsigned long long *keys, cudaStream_t st);

// photometry.cu: binning, fake companions, apertures (Sect. 4.2, 4.3)
// out: ceil(T / B) frames; *launched receives the kernel count
cudaError_t launch_bin_median(const float *in, float *out, long long T, int n, int B, int *status, cudaStream_t st,
                              int *launched = nullptr);
// pos: [T][n_comp] (x, y) FP64; win: [T][n_comp] (row, col) of the window
// centre; amp: [T][n_comp] Moffat peak; shape: [T] (1 / alpha^2, beta), FP32
cudaError_t launch_inject(float *cube, long long T, int n, int n_comp, const double *pos, const int *win,
                          const float *amp, const float *shape, int half, cudaStream_t st);
// xy: [n_ap] (x, y); out: [n_ap] device FP64
cudaError_t launch_aperture(const float *img, int n, int n_ap, const double *xy, double radius, double *out,
                            cudaStream_t st);

}  // namespace graphic

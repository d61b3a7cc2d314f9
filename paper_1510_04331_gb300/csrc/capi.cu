// capi.cu -- C ABI of the GRAPHIC GB300 library (declared in include/graphic.h):
// argument checks, FP64 host plans, workspaces, kernel orchestration.
//
// Host plans (FP64, computed per call):
//   shift   dx[t], dy[t] uploaded as they are;
//   rotate  theta = 90 q + theta', q = floor(theta/90 + 1/2) (Sect. 3.4 shears
//           need |theta'| <= 45 deg to keep tan(theta'/2) bounded), then
//           a = tan(theta'/2), s = sin(theta') per frame;
//   adi     frames sorted by parallactic angle (stable), and for every annulus
//           and sorted position s the reference set {k : |alpha_k - alpha_s|
//           > alpha_min} (Sect. 3.3) written as sorted-position ranges
//           [0, L) u [R, T) -- exact, because |fl(alpha_k - alpha_s)| is
//           monotone on either side of s -- with the farthest-frame fallback
//           when that set is empty; with time stamps also the window [A, B)
//           of frames within t_max (Sect. 3.3), the set then [A, L) u [R, B).
// Work order of graphic_rotate / graphic_shift: frames are processed in
// chunks sized so that a chunk's intermediate data (the n x 2n scratch of
// the rotation) stays within the L2 cache between the passes.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/graphic.h"
#include "graphic_internal.h"

using namespace graphic;

struct graphic_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int *d_status = nullptr;
  int *h_status = nullptr;          // pinned
  char *d_plan = nullptr;
  size_t d_plan_bytes = 0;
  char *h_plan = nullptr;           // pinned staging
  size_t h_plan_bytes = 0;
  float *d_scratch = nullptr;
  size_t scratch_bytes = 0;
  float *d_cube = nullptr;          // graphic_reduce_host device copy of the input
  size_t cube_bytes = 0;
  float *d_img = nullptr;           // graphic_reduce_host device result
  size_t img_bytes = 0;
  char *d_bscratch = nullptr;       // median PSF band path: per-pixel band tables
  size_t bscratch_bytes = 0;
  char *d_lparam = nullptr;         // line-pass parameter tables
  size_t lparam_bytes = 0;
  char *d_gparam = nullptr;         // grouped executor: parameter tables, one region per branch
  size_t gparam_bytes = 0;
  bool prof = false;
  double prof_ms[GRAPHIC_K_COUNT] = {};
  int64_t prof_n[GRAPHIC_K_COUNT] = {};
  int64_t prof_extra[GRAPHIC_K_COUNT] = {};   // kernels beyond one per bracketed call
  std::vector<cudaEvent_t> ev;      // event pool, pairs
  std::vector<int> ev_kernel;       // kernel id per used pair
  size_t ev_used = 0;
  // schedule (defaults, autotuner, or GRAPHIC_TUNE_CACHE)
  int chunk_mb = 4096;              // frames per chunk of the per-call passes: this much intermediate
                                    // (measured: one chunk per survey cube beats L2-sized chunks, whose
                                    // launch tails cost more than the scratch's trips to HBM)
  int variant_1024 = 1;             // 1024-point lines: 1 warp per line pair (radix 32x32), 0 generic
  int batch_budget_mb = 1024;       // persistent executor: scratch of one wave (two waves alternate)
  int batch_ctas_per_sm = 2;
  int group_budget_mb = 128;        // grouped executor: scratch of one wave
  int group_streams = 2;            // grouped executor: concurrent graph branches
  int batch_mode = GRAPHIC_BATCH_GROUPED;   // GRAPHIC_BATCH_AUTO resolves to this
  bool group_graph = true;          // grouped executor: record a graph (false: launch directly)
  int precision = GRAPHIC_PREC_FP32;   // line-pass arithmetic for frames of n = 1024
  // pre-processing: small device buffers (histogram, sums, counters, median, threshold)
  char *d_prep = nullptr;
  size_t prep_bytes = 0;
  // graphic_reduce_host: copy stream and event (cube copied in chunks ahead of the shift pass)
  cudaStream_t s_copy = nullptr;
  cudaEvent_t ev_copy = nullptr;
  // grouped executor state
  float *d_gscratch = nullptr;
  size_t gscratch_bytes = 0;
  std::vector<cudaStream_t> gstreams;
  std::vector<cudaEvent_t> gevents;
  cudaGraph_t ggraph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<long long> gkey;
  // persistent executor state
  int *d_counters = nullptr;
  size_t counters_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<long long> graph_key;
};

namespace {

thread_local std::string g_err;

const double kPi = 3.14159265358979323846264338327950288;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char *where) {
  return fail(e == cudaErrorMemoryAllocation ? GRAPHIC_ERR_OOM : GRAPHIC_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool supported_n(int32_t n) { return n == 64 || n == 128 || n == 256 || n == 512 || n == 1024; }

int check_cube(const void *in, const void *out, int64_t T, int32_t n, bool device = true) {
  if (T < 0) return fail(GRAPHIC_ERR_INVALID_ARG, "n_frames < 0");
  if (T > 0 && (!in || !out)) return fail(GRAPHIC_ERR_INVALID_ARG, "null cube pointer");
  if (device && (((uintptr_t)in | (uintptr_t)out) & 15))
    return fail(GRAPHIC_ERR_INVALID_ARG, "device cubes must be 16-byte aligned");
  if (!supported_n(n)) return fail(GRAPHIC_ERR_UNSUPPORTED, "n must be one of 64, 128, 256, 512, 1024");
  return GRAPHIC_OK;
}

int ensure(void **ptr, size_t *have, size_t need, bool pinned) {
  if (*have >= need && *ptr) return GRAPHIC_OK;
  if (*ptr) {
    if (pinned) cudaFreeHost(*ptr); else cudaFree(*ptr);
    *ptr = nullptr;
    *have = 0;
  }
  cudaError_t e = pinned ? cudaMallocHost(ptr, need) : cudaMalloc(ptr, need);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return cuda_fail(e, pinned ? "cudaMallocHost" : "cudaMalloc");
  }
  *have = need;
  return GRAPHIC_OK;
}

// --- profiling ------------------------------------------------------------
void prof_begin(graphic_ctx *c, int k) {
  if (!c->prof) return;
  if (c->ev.size() < 2 * (c->ev_used + 1)) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    c->ev.push_back(a);
    c->ev.push_back(b);
    c->ev_kernel.push_back(k);
  }
  c->ev_kernel[c->ev_used] = k;
  cudaEventRecord(c->ev[2 * c->ev_used], c->stream);
}
void prof_end(graphic_ctx *c) {
  if (!c->prof) return;
  cudaEventRecord(c->ev[2 * c->ev_used + 1], c->stream);
  c->ev_used++;
}
void prof_collect(graphic_ctx *c) {
  for (int k = 0; k < GRAPHIC_K_COUNT; k++) {
    c->prof_n[k] += c->prof_extra[k];
    c->prof_extra[k] = 0;
  }
  for (size_t i = 0; i < c->ev_used; i++) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess) {
      c->prof_ms[c->ev_kernel[i]] += ms;
      c->prof_n[c->ev_kernel[i]] += 1;
    }
  }
  c->ev_used = 0;
}

// --- plan upload ----------------------------------------------------------
struct PlanBuilder {
  std::vector<char> buf;
  size_t add(const void *src, size_t bytes) {
    size_t off = (buf.size() + 15) & ~size_t(15);
    buf.resize(off + bytes);
    if (bytes) memcpy(buf.data() + off, src, bytes);
    return off;
  }
};

int upload_plan(graphic_ctx *c, const PlanBuilder &pb) {
  const size_t bytes = std::max<size_t>(pb.buf.size(), 16);
  int rc = ensure((void **)&c->h_plan, &c->h_plan_bytes, bytes, true);
  if (rc) return rc;
  rc = ensure((void **)&c->d_plan, &c->d_plan_bytes, bytes, false);
  if (rc) return rc;
  memcpy(c->h_plan, pb.buf.data(), pb.buf.size());
  CK(cudaMemcpyAsync(c->d_plan, c->h_plan, pb.buf.size(), cudaMemcpyHostToDevice, c->stream));
  return GRAPHIC_OK;
}

int begin_call(graphic_ctx *c) {
  CK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
  return GRAPHIC_OK;
}

// Wait for the stream, collect profile events, turn the status word into a code.
int end_call(graphic_ctx *c) {
  CK(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  prof_collect(c);
  if (*c->h_status & STATUS_NONFINITE) return fail(GRAPHIC_ERR_NONFINITE, "non-finite value in the input cube");
  if (*c->h_status & STATUS_INTERNAL) return fail(GRAPHIC_ERR_INTERNAL, "device consistency check failed");
  if (*c->h_status & STATUS_TIMEOUT) return fail(GRAPHIC_ERR_TIMEOUT, "a bounded device wait ran out");
  return GRAPHIC_OK;
}

constexpr size_t kCopyChunkMB = 256;   // host -> device copy pieces of graphic_reduce_host

long long chunk_frames(const graphic_ctx *c, long long T, size_t bytes_per_frame) {
  size_t budget = (size_t)c->chunk_mb << 20;
  if (const char *e = getenv("GRAPHIC_CHUNK_MB")) {
    long v = atol(e);
    if (v > 0) budget = (size_t)v << 20;
  }
  long long k = (long long)(budget / bytes_per_frame);
  if (k < 1) k = 1;
  if (k > T) k = T;
  return k;
}

}  // namespace

// One line pass with the context's arithmetic: the tensor-core DFT stages
// (BF16 / FP16 hi + lo) where the precision variant asks for them and the
// frame size has them, else the FP32 kernels.
cudaError_t line_pass(const graphic_ctx *c, LineKind kind, const LineArgs &a, long long nf, cudaStream_t st) {
  if (c->precision != GRAPHIC_PREC_FP32 && tc_supported(a.n))
    return launch_line_pass_tc(kind, a, nf, st, c->precision);
  return launch_line_pass(kind, a, nf, st, c->variant_1024);
}

// --- shift ------------------------------------------------------------------
int graphic::validate_shift(const double *dx, const double *dy, int64_t T, int32_t n) {
  if (T > 0 && (!dx || !dy)) return fail(GRAPHIC_ERR_INVALID_ARG, "null dx/dy");
  for (int64_t t = 0; t < T; t++) {
    if (!isfinite(dx[t]) || !isfinite(dy[t])) return fail(GRAPHIC_ERR_INVALID_ARG, "non-finite shift");
    if (fabs(dx[t]) > n / 2 || fabs(dy[t]) > n / 2) return fail(GRAPHIC_ERR_INVALID_ARG, "|shift| > n/2");
  }
  return GRAPHIC_OK;
}

namespace {

// Enqueue the two shift passes for frames [0, T) with parameters at device
// pointers p_dx, p_dy.  in -> out (out may equal in); in_fs / out_fs: the
// frame strides in elements (0: n*n).
int enqueue_shift(graphic_ctx *c, const float *in, float *out, int64_t T, int32_t n, const double *p_dx,
                  const double *p_dy, long long in_fs = 0, long long out_fs = 0) {
  const long long NN = (long long)n * n;
  if (!in_fs) in_fs = NN;
  if (!out_fs) out_fs = NN;
  const long long ch = chunk_frames(c, T, (size_t)NN * sizeof(float));
  // per-frame shift parameters of both passes, once for all frames
  const size_t pb = line_params_bytes(SHIFT_X, n, T);
  int rc = ensure((void **)&c->d_lparam, &c->lparam_bytes, 2 * pb, false);
  if (rc) return rc;
  {
    LineArgs a{};
    a.p0 = p_dx;
    a.p1 = p_dy;
    a.n = n;
    cudaError_t e = launch_line_params(SHIFT_X, a, T, c->d_lparam, c->stream);
    if (e == cudaSuccess) e = launch_line_params(SHIFT_Y, a, T, c->d_lparam + pb, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "shift parameters");
  }
  for (long long f0 = 0; f0 < T; f0 += ch) {
    const long long nf = std::min<long long>(ch, T - f0);
    LineArgs a{};
    a.in = in + f0 * in_fs;
    a.out = out + f0 * out_fs;
    a.p0 = p_dx + f0;
    a.p1 = p_dy + f0;
    a.status = c->d_status;
    a.in_fstride = in_fs;
    a.out_fstride = out_fs;
    a.n = n;
    a.lp_lines = 1;
    a.lp_tab = c->d_lparam + (size_t)f0 * (pb / T);
    prof_begin(c, GRAPHIC_K_SHIFT_X);
    cudaError_t e = line_pass(c, SHIFT_X, a, nf, c->stream);
    prof_end(c);
    if (e != cudaSuccess) return cuda_fail(e, "shift x pass");
    a.in = out + f0 * out_fs;
    a.in_fstride = out_fs;
    a.lp_tab = c->d_lparam + pb + (size_t)f0 * (pb / T);
    prof_begin(c, GRAPHIC_K_SHIFT_Y);
    e = line_pass(c, SHIFT_Y, a, nf, c->stream);
    prof_end(c);
    if (e != cudaSuccess) return cuda_fail(e, "shift y pass");
  }
  return GRAPHIC_OK;
}

// --- rotate -----------------------------------------------------------------
struct RotPlanHost {
  std::vector<double> a, s;
  std::vector<int> q;
};

int plan_rotate(const double *theta, int64_t T, bool negate, RotPlanHost &rp) {
  rp.a.resize(T);
  rp.s.resize(T);
  rp.q.resize(T);
  for (int64_t t = 0; t < T; t++) {
    const double th = negate ? -theta[t] : theta[t];
    if (!isfinite(th) || fabs(th) > 1e6) return fail(GRAPHIC_ERR_INVALID_ARG, "angle not finite or |angle| > 1e6 deg");
    const int q = (int)floor(th / 90.0 + 0.5);
    const double tp = th - 90.0 * (double)q;
    if (tp == 0.0) {
      rp.a[t] = 0.0;
      rp.s[t] = 0.0;
    } else {
      const double r = tp * kPi / 180.0;
      rp.a[t] = tan(r / 2.0);
      rp.s[t] = sin(r);
    }
    rp.q[t] = ((q % 4) + 4) % 4;
  }
  return GRAPHIC_OK;
}

int enqueue_rotate(graphic_ctx *c, const float *in, float *out, int64_t T, int32_t n, const double *p_a,
                   const double *p_s, const int *p_q, long long in_fs = 0, long long out_fs = 0) {
  const long long NN = (long long)n * n;
  const long long NM = NN * 2;
  if (!in_fs) in_fs = NN;
  if (!out_fs) out_fs = NN;
  const long long ch = chunk_frames(c, T, (size_t)NM * sizeof(float));
  int rc = ensure((void **)&c->d_scratch, &c->scratch_bytes, (size_t)ch * NM * sizeof(float), false);
  if (rc) return rc;
  // per-line shear parameters of a chunk: passes 1 and 3 share theirs
  const size_t pb13 = line_params_bytes(ROT_P1, n, ch), pb2 = line_params_bytes(ROT_P2, n, ch);
  if ((rc = ensure((void **)&c->d_lparam, &c->lparam_bytes, pb13 + pb2, false))) return rc;
  for (long long f0 = 0; f0 < T; f0 += ch) {
    const long long nf = std::min<long long>(ch, T - f0);
    LineArgs a{};
    a.p0 = p_a + f0;
    a.p1 = p_s + f0;
    a.q = p_q + f0;
    a.status = c->d_status;
    a.n = n;
    {
      cudaError_t e = launch_line_params(ROT_P1, a, nf, c->d_lparam, c->stream);
      if (e == cudaSuccess) e = launch_line_params(ROT_P2, a, nf, c->d_lparam + pb13, c->stream);
      if (e != cudaSuccess) return cuda_fail(e, "shear parameters");
    }
    a.lp_tab = c->d_lparam;
    a.lp_lines = line_params_lines(ROT_P1, n);
    // pass 1: frame rows (after rot90^q) -> scratch rows of 2n
    a.in = in + f0 * in_fs;
    a.out = c->d_scratch;
    a.in_fstride = in_fs;
    a.out_fstride = NM;
    prof_begin(c, GRAPHIC_K_ROT_P1);
    cudaError_t e = line_pass(c, ROT_P1, a, nf, c->stream);
    prof_end(c);
    if (e != cudaSuccess) return cuda_fail(e, "rotation pass 1");
    // pass 2: scratch columns, in place
    a.in = c->d_scratch;
    a.out = c->d_scratch;
    a.in_fstride = NM;
    a.out_fstride = NM;
    a.lp_tab = c->d_lparam + pb13;
    a.lp_lines = line_params_lines(ROT_P2, n);
    prof_begin(c, GRAPHIC_K_ROT_P2);
    e = line_pass(c, ROT_P2, a, nf, c->stream);
    prof_end(c);
    if (e != cudaSuccess) return cuda_fail(e, "rotation pass 2");
    // pass 3: scratch rows -> frame rows
    a.out = out + f0 * out_fs;
    a.out_fstride = out_fs;
    a.lp_tab = c->d_lparam;
    a.lp_lines = line_params_lines(ROT_P3, n);
    prof_begin(c, GRAPHIC_K_ROT_P3);
    e = line_pass(c, ROT_P3, a, nf, c->stream);
    prof_end(c);
    if (e != cudaSuccess) return cuda_fail(e, "rotation pass 3");
  }
  return GRAPHIC_OK;
}

}  // namespace

// --- adi --------------------------------------------------------------------
int graphic::validate_adi(const double *parang, int64_t T, double fwhm, double n_fwhm, const double *edges, int32_t n_edges) {
  if (T < 1) return fail(GRAPHIC_ERR_INVALID_ARG, "n_frames < 1");
  if (T > GRAPHIC_MAX_FRAMES_MEDIAN) return fail(GRAPHIC_ERR_UNSUPPORTED, "n_frames > GRAPHIC_MAX_FRAMES_MEDIAN");
  if (!parang) return fail(GRAPHIC_ERR_INVALID_ARG, "null parang");
  if (!edges || n_edges < 2 || n_edges > 4096) return fail(GRAPHIC_ERR_INVALID_ARG, "need 2..4096 annulus edges");
  if (!(fwhm > 0) || !isfinite(fwhm) || !(n_fwhm > 0) || !isfinite(n_fwhm))
    return fail(GRAPHIC_ERR_INVALID_ARG, "fwhm and n_fwhm must be finite and > 0");
  for (int32_t i = 0; i < n_edges; i++) {
    if (!isfinite(edges[i]) || edges[i] < 0) return fail(GRAPHIC_ERR_INVALID_ARG, "annulus edges must be finite, >= 0");
    if (i && !(edges[i] > edges[i - 1])) return fail(GRAPHIC_ERR_INVALID_ARG, "annulus edges must increase");
  }
  for (int64_t t = 0; t < T; t++)
    if (!isfinite(parang[t])) return fail(GRAPHIC_ERR_INVALID_ARG, "non-finite parallactic angle");
  return GRAPHIC_OK;
}

// Band of full ranks that holds every median annulus `lr` needs: query s has
// |S| = L + T - R members, its (lower) median is the k-th of S, k = (|S|-1)/2,
// and at most w = R - L frames are excluded, so that element has full rank in
// [k, k + w]; with the upper median of an even |S|, in [k, k + 1 + w].
static void plan_band(const int *lr, int64_t T, int *out) {
  int64_t blo = T, bhi = -1;
  for (int64_t s = 0; s < T; s++) {
    const int64_t L = lr[2 * s], R = lr[2 * s + 1];
    const int64_t nS = L + (T - R), w = R - L;
    const int64_t k = (nS - 1) / 2;
    blo = std::min(blo, k);
    bhi = std::max(bhi, k + ((nS & 1) ? 0 : 1) + w);
  }
  bhi = std::min<int64_t>(bhi, T - 1);
  const int64_t B = bhi - blo + 1;
  int W = 0;
  for (int c = 1; c <= 32; c <<= 1)
    if (32 * c >= B) {
      W = c;
      break;
    }
  out[0] = (int)blo;
  out[1] = (int)bhi;
  out[2] = W;
  out[3] = 0;
}

static double alpha_min_deg(double fwhm, double n_fwhm, double r) {
  double arg = n_fwhm * fwhm / (2.0 * r);
  if (!(arg < 1.0)) arg = 1.0;
  return 2.0 * asin(arg) * 180.0 / kPi;
}

int graphic::plan_adi(const double *parang, int64_t T, double fwhm, double n_fwhm, const double *edges,
                      int32_t n_edges, AdiPlanHost &ap, const double *times, double t_max) {
  const int A = n_edges - 1;
  ap.perm.resize(T);
  for (int64_t t = 0; t < T; t++) ap.perm[t] = (int)t;
  std::stable_sort(ap.perm.begin(), ap.perm.end(), [&](int x, int y) { return parang[x] < parang[y]; });
  ap.edge2.resize(n_edges);
  for (int i = 0; i < n_edges; i++) ap.edge2[i] = edges[i] * edges[i];
  // time windows [A, B) in the angle order (the whole order without a time gate)
  ap.ab.clear();
  std::vector<int> wa(T, 0), wb(T, (int)T);
  if (times) {
    if (!(t_max > 0) || std::isnan(t_max)) return fail(GRAPHIC_ERR_INVALID_ARG, "t_max must be > 0");
    std::vector<double> tt(T);
    bool up = true, down = true;
    for (int64_t s = 0; s < T; s++) {
      tt[s] = times[ap.perm[s]];
      if (!std::isfinite(tt[s])) return fail(GRAPHIC_ERR_INVALID_ARG, "non-finite time stamp");
      if (s) {
        up &= tt[s] >= tt[s - 1];
        down &= tt[s] <= tt[s - 1];
      }
    }
    if (!up && !down)
      return fail(GRAPHIC_ERR_UNSUPPORTED, "time stamps must be monotone in the order of the parallactic angles");
    // |fl(t_k - t_s)| is monotone on either side of s: binary searches are exact
    for (int64_t s = 0; s < T; s++) {
      auto near = [&](int64_t k) { return fabs(tt[k] - tt[s]) < t_max; };
      int64_t lo = 0, hi = s;   // [0, s]: false ... false true ... true
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (near(mid)) hi = mid; else lo = mid + 1;
      }
      wa[s] = (int)lo;
      lo = s;
      hi = T;                   // [s, T): true ... true false ... false
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (near(mid)) lo = mid + 1; else hi = mid;
      }
      wb[s] = (int)lo;
    }
    ap.ab.resize((size_t)T * 2);
    for (int64_t s = 0; s < T; s++) {
      ap.ab[2 * s] = wa[s];
      ap.ab[2 * s + 1] = wb[s];
    }
  }
  ap.lr.assign((size_t)A * T * 2, 0);
  std::vector<double> al(T);
  for (int64_t s = 0; s < T; s++) al[s] = parang[ap.perm[s]];
  for (int a = 0; a < A; a++) {
    const double amin = alpha_min_deg(fwhm, n_fwhm, edges[a]);
    int *lr = ap.lr.data() + (size_t)a * T * 2;
    for (int64_t s = 0; s < T; s++) {
      const double ai = al[s];
      auto pred = [&](int64_t k) { return fabs(al[k] - ai) > amin; };
      // [0, s]: pred true ... true false ... false
      int64_t lo = 0, hi = s;
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (pred(mid)) lo = mid + 1; else hi = mid;
      }
      int64_t L = lo;
      // [s, T): pred false ... false true ... true
      lo = s;
      hi = T;
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (pred(mid)) hi = mid; else lo = mid + 1;
      }
      int64_t R = lo;
      // clip the excluded range to the time window: the set is [W0, L) u [R, W1)
      const int64_t W0 = wa[s], W1 = wb[s];
      L = std::max(L, W0);
      R = std::min(R, W1);
      if (L == W0 && R == W1) {
        // empty: the frame(s) of the window farthest in angle
        const double best = std::max(fabs(al[W0] - ai), fabs(al[W1 - 1] - ai));
        int64_t l2 = W0;
        while (l2 < W1 && fabs(al[l2] - ai) == best) l2++;
        int64_t r2 = W1;
        if (l2 < W1)
          while (r2 > l2 && fabs(al[r2 - 1] - ai) == best) r2--;
        else
          r2 = W1;
        L = l2;
        R = r2;
      }
      lr[2 * s] = (int)L;
      lr[2 * s + 1] = (int)R;
    }
  }
  ap.band.assign((size_t)A * 4, 0);
  ap.wmax = 0;
  if (times) return GRAPHIC_OK;   // general path only
  for (int a = 0; a < A; a++) {
    const int *lr = ap.lr.data() + (size_t)a * T * 2;
    plan_band(lr, T, ap.band.data() + 4 * a);
    // the band kernel's sweep needs gates that only move forward
    for (int64_t s = 1; s < T; s++)
      if (lr[2 * s] < lr[2 * s - 2] || lr[2 * s + 1] < lr[2 * s - 1]) {
        ap.band[4 * a + 2] = 0;
        break;
      }
    ap.wmax = std::max(ap.wmax, ap.band[4 * a + 2]);
  }
  return GRAPHIC_OK;
}

namespace {

// Plan tables of the median PSF step in the uploaded plan (byte offsets).
struct AdiOffsets {
  size_t perm, lr, e2, band, ab, evq, groups;
};

AdiOffsets add_adi_plan(PlanBuilder &pb, const AdiPlanHost &ap, int64_t T) {
  AdiOffsets o{};
  o.e2 = pb.add(ap.edge2.data(), ap.edge2.size() * sizeof(double));
  o.perm = pb.add(ap.perm.data(), T * sizeof(int));
  o.lr = pb.add(ap.lr.data(), ap.lr.size() * sizeof(int));
  o.band = pb.add(ap.band.data(), ap.band.size() * sizeof(int));
  o.ab = pb.add(ap.ab.data(), ap.ab.size() * sizeof(int));
  o.evq = pb.add(ap.evq.data(), ap.evq.size() * sizeof(uint32_t));
  o.groups = pb.add(ap.groups.data(), ap.groups.size() * sizeof(int));
  return o;
}

int enqueue_adi_raw(graphic_ctx *c, const float *in, float *out, int64_t T, int32_t n, const int *p_perm,
                    const int *p_lr, const double *p_edge2, const int *p_band, int wmax, int n_ann,
                    const int *p_ab, const uint32_t *p_evq, const int *p_groups, const std::vector<int> &class_off,
                    int gen_off, int gen_n, char *band_scratch, size_t band_scratch_cap, long long in_fs,
                    long long out_fs, bool perm_id) {
  AdiArgs a{};
  a.perm_id = perm_id ? 1 : 0;
  a.in_fs = in_fs ? in_fs : (long long)n * n;
  a.out_fs = out_fs ? out_fs : (long long)n * n;
  a.band_scratch_cap = band_scratch_cap;
  a.evq = p_evq;
  a.groups = p_groups;
  for (int k = 0; k < 8; k++) a.class_off[k] = k < (int)class_off.size() ? class_off[k] : 0;
  a.gen_list = gen_off >= 0 ? 1 : 0;
  a.gen_off = gen_off;
  a.gen_n = gen_n;
  a.band_scratch = band_scratch;
  a.in = in;
  a.out = out;
  a.perm = p_perm;
  a.lr = p_lr;
  a.ab = p_ab;
  a.edge2 = p_edge2;
  a.band = p_band;
  a.wmax = wmax;
  a.status = c->d_status;
  a.T = (int)T;
  a.n = n;
  a.n_ann = n_ann;
  // profiling: one bracket per group of launches (general path, band
  // preparation with the zero groups, band sweep)
  a.mark_user = c;
  a.mark = [](void *u, int kind, int begin) {
    graphic_ctx *cc = static_cast<graphic_ctx *>(u);
    const int id = kind == 0 ? GRAPHIC_K_ADI_MEDIAN : kind == 1 ? GRAPHIC_K_ADI_BAND_PREP : GRAPHIC_K_ADI_BAND_SWEEP;
    if (begin) prof_begin(cc, id);
    else prof_end(cc);
  };
  int launched = 0;
  cudaError_t e = launch_adi_median(a, c->stream, &launched);
  if (e != cudaSuccess) return cuda_fail(e, "median PSF kernel");
  return GRAPHIC_OK;
}


int enqueue_collapse(graphic_ctx *c, const float *in, int64_t T, int32_t n, float *out, long long in_fs = 0) {
  CollapseArgs a{};
  a.fs = in_fs;
  a.in = in;
  a.out = out;
  a.status = c->d_status;
  a.T = T;
  a.n = n;
  prof_begin(c, GRAPHIC_K_COLLAPSE);
  cudaError_t e = launch_collapse(a, c->stream);
  prof_end(c);
  if (e != cudaSuccess) return cuda_fail(e, "collapse kernel");
  return GRAPHIC_OK;
}

template <class T>
const T *at(const graphic_ctx *c, size_t off) {
  return reinterpret_cast<const T *>(c->d_plan + off);
}

int enqueue_adi(graphic_ctx *c, const float *in, float *out, int64_t T, int32_t n, const AdiPlanHost &ap,
                const AdiOffsets &o, long long in_fs = 0, long long out_fs = 0) {
  bool perm_id = true;
  for (int64_t t = 0; t < T && perm_id; t++) perm_id = ap.perm[t] == (int)t;
  const size_t need = band_scratch_bytes(ap, T);
  if (need) {
    int rc = ensure((void **)&c->d_bscratch, &c->bscratch_bytes, need, false);
    if (rc) return rc;
  }
  return enqueue_adi_raw(c, in, out, T, n, at<int>(c, o.perm), at<int>(c, o.lr), at<double>(c, o.e2),
                         at<int>(c, o.band), ap.wmax, (int)ap.edge2.size() - 1,
                         ap.ab.empty() ? nullptr : at<int>(c, o.ab), at<uint32_t>(c, o.evq), at<int>(c, o.groups),
                         ap.class_off, ap.gen_off, ap.gen_n, c->d_bscratch, c->bscratch_bytes, in_fs, out_fs,
                         perm_id);
}

// Full reduction of the device cube `in` (work may equal in).  With host_in,
// `in` is first filled from host_in, chunk by chunk on the context's copy
// stream, each chunk's shift pass starting as soon as its copy is done.
int reduce_device(graphic_ctx *c, const float *in, float *work, int64_t T, int32_t n, const double *dx,
                  const double *dy, const double *parang, double fwhm, double n_fwhm, const double *edges,
                  int32_t n_edges, float *out, const float *host_in = nullptr, const double *times = nullptr,
                  double t_max = 0.0, long long in_fs = 0, long long work_fs = 0) {
  int rc = validate_shift(dx, dy, T, n);
  if (rc) return rc;
  rc = validate_adi(parang, T, fwhm, n_fwhm, edges, n_edges);
  if (rc) return rc;
  RotPlanHost rp;
  rc = plan_rotate(parang, T, true, rp);
  if (rc) return rc;
  AdiPlanHost ap;
  if ((rc = plan_adi(parang, T, fwhm, n_fwhm, edges, n_edges, ap, times, t_max))) return rc;
  if ((rc = plan_band_path(ap, T, n))) return rc;
  PlanBuilder pb;
  const size_t o_dx = pb.add(dx, T * sizeof(double));
  const size_t o_dy = pb.add(dy, T * sizeof(double));
  const size_t o_a = pb.add(rp.a.data(), T * sizeof(double));
  const size_t o_s = pb.add(rp.s.data(), T * sizeof(double));
  const size_t o_q = pb.add(rp.q.data(), T * sizeof(int));
  const AdiOffsets oa = add_adi_plan(pb, ap, T);
  if ((rc = begin_call(c))) return rc;
  if ((rc = upload_plan(c, pb))) return rc;
  if (!host_in) {
    if ((rc = enqueue_shift(c, in, work, T, n, at<double>(c, o_dx), at<double>(c, o_dy), in_fs, work_fs))) return rc;
  } else {
    if (!c->s_copy) {
      CK(cudaStreamCreateWithFlags(&c->s_copy, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&c->ev_copy, cudaEventDisableTiming));
    }
    // the copies start after everything already on the compute stream
    CK(cudaEventRecord(c->ev_copy, c->stream));
    CK(cudaStreamWaitEvent(c->s_copy, c->ev_copy, 0));
    // copies in pieces of kCopyChunkMB, each piece's shift launched as soon as
    // it lands (the copy, not the shift, bounds this path)
    const size_t NN = (size_t)n * n;
    const long long ch = std::max<long long>(1, std::min<long long>(T, (long long)((kCopyChunkMB << 20) /
                                                                                    (NN * sizeof(float)))));
    for (long long f0 = 0; f0 < T; f0 += ch) {
      const long long nf = std::min<long long>(ch, T - f0);
      CK(cudaMemcpyAsync(const_cast<float *>(in) + f0 * NN, host_in + f0 * NN, nf * NN * sizeof(float),
                         cudaMemcpyHostToDevice, c->s_copy));
      CK(cudaEventRecord(c->ev_copy, c->s_copy));
      CK(cudaStreamWaitEvent(c->stream, c->ev_copy, 0));
      if ((rc = enqueue_shift(c, in + f0 * NN, work + f0 * NN, nf, n, at<double>(c, o_dx) + f0,
                              at<double>(c, o_dy) + f0)))
        return rc;
    }
  }
  if ((rc = enqueue_adi(c, work, work, T, n, ap, oa, work_fs, work_fs))) return rc;
  if ((rc = enqueue_rotate(c, work, work, T, n, at<double>(c, o_a), at<double>(c, o_s), at<int>(c, o_q), work_fs,
                           work_fs)))
    return rc;
  if ((rc = enqueue_collapse(c, work, T, n, out, work_fs))) return rc;
  return GRAPHIC_OK;
}

// --- uneven batches -----------------------------------------------------------
int item_passes(const graphic_batch_item &it) {
  return it.passes ? it.passes : (GRAPHIC_PASS_SHIFT | GRAPHIC_PASS_ROTATE);
}

int validate_batch(const graphic_batch_item *items, int32_t n_items) {
  if (n_items < 0 || (n_items > 0 && !items)) return fail(GRAPHIC_ERR_INVALID_ARG, "bad item list");
  for (int32_t i = 0; i < n_items; i++) {
    const graphic_batch_item &it = items[i];
    int rc = check_cube(it.in, it.out, it.n_frames, it.n);
    if (rc) return rc;
    if (it.passes < 0 || it.passes > (GRAPHIC_PASS_SHIFT | GRAPHIC_PASS_ROTATE))
      return fail(GRAPHIC_ERR_INVALID_ARG, "bad passes mask");
    if (it.n_frames > 0 && (item_passes(it) & GRAPHIC_PASS_ROTATE) && !it.theta_deg)
      return fail(GRAPHIC_ERR_INVALID_ARG, "null theta");
    for (int64_t t = 0; t < it.n_frames; t++) {
      const double dx = it.dx ? it.dx[t] : 0.0, dy = it.dy ? it.dy[t] : 0.0;
      if (!isfinite(dx) || !isfinite(dy) || fabs(dx) > it.n / 2 || fabs(dy) > it.n / 2)
        return fail(GRAPHIC_ERR_INVALID_ARG, "shift not finite or |shift| > n/2");
    }
  }
  return GRAPHIC_OK;
}

// work items (CTAs) of one frame per pass: shift x, shift y, rotation 1, 2, 3
void batch_ctas(int n, int out[5]) {
  const int per = n * n / 4096;   // n lines, 4096/m line pairs per CTA
  out[0] = out[1] = out[2] = out[4] = per;
  out[3] = 2 * per;               // 2n columns
}

// One cube after the other: the per-call shift and rotation passes, no
// synchronisation in between.
int batch_per_cube(graphic_ctx *c, const graphic_batch_item *items, int32_t n_items) {
  PlanBuilder pb;
  std::vector<size_t> off(n_items * 5);
  for (int32_t i = 0; i < n_items; i++) {
    const graphic_batch_item &it = items[i];
    const int64_t T = it.n_frames;
    std::vector<double> dx(T, 0.0), dy(T, 0.0);
    for (int64_t t = 0; t < T; t++) {
      if (it.dx) dx[t] = it.dx[t];
      if (it.dy) dy[t] = it.dy[t];
    }
    RotPlanHost rp;
    if (item_passes(it) & GRAPHIC_PASS_ROTATE) {
      int rc = plan_rotate(it.theta_deg, T, false, rp);
      if (rc) return rc;
    } else {
      rp.a.assign(T, 0.0);
      rp.s.assign(T, 0.0);
      rp.q.assign(T, 0);
    }
    off[5 * i + 0] = pb.add(dx.data(), T * sizeof(double));
    off[5 * i + 1] = pb.add(dy.data(), T * sizeof(double));
    off[5 * i + 2] = pb.add(rp.a.data(), T * sizeof(double));
    off[5 * i + 3] = pb.add(rp.s.data(), T * sizeof(double));
    off[5 * i + 4] = pb.add(rp.q.data(), T * sizeof(int));
  }
  int rc;
  if ((rc = upload_plan(c, pb))) return rc;
  for (int32_t i = 0; i < n_items; i++) {
    const graphic_batch_item &it = items[i];
    if (it.n_frames == 0) continue;
    const int ps = item_passes(it);
    if ((ps & GRAPHIC_PASS_SHIFT) && (rc = enqueue_shift(c, it.in, it.out, it.n_frames, it.n,
                                                         at<double>(c, off[5 * i]), at<double>(c, off[5 * i + 1]))))
      return rc;
    const float *rin = (ps & GRAPHIC_PASS_SHIFT) ? it.out : it.in;
    if ((ps & GRAPHIC_PASS_ROTATE) &&
        (rc = enqueue_rotate(c, rin, it.out, it.n_frames, it.n, at<double>(c, off[5 * i + 2]),
                             at<double>(c, off[5 * i + 3]), at<int>(c, off[5 * i + 4]))))
      return rc;
  }
  return GRAPHIC_OK;
}

// Every frame of every cube in one persistent launch, replayed from a CUDA
// graph while the batch keeps its layout.
int batch_persistent(graphic_ctx *c, const graphic_batch_item *items, int32_t n_items) {
  std::vector<BatchFrame> fr;
  for (int32_t i = 0; i < n_items; i++) {
    const graphic_batch_item &it = items[i];
    const int ps = item_passes(it);
    RotPlanHost rp;
    if (ps & GRAPHIC_PASS_ROTATE) {
      int rc = plan_rotate(it.theta_deg, it.n_frames, false, rp);
      if (rc) return rc;
    }
    const size_t NN = (size_t)it.n * it.n;
    for (int64_t t = 0; t < it.n_frames; t++) {
      BatchFrame b{};
      b.in = it.in + t * NN;
      b.out = it.out + t * NN;
      b.rin = (ps & GRAPHIC_PASS_SHIFT) ? b.out : b.in;
      b.dx = it.dx ? it.dx[t] : 0.0;
      b.dy = it.dy ? it.dy[t] : 0.0;
      if (ps & GRAPHIC_PASS_ROTATE) {
        b.a = rp.a[t];
        b.s = rp.s[t];
        b.q = rp.q[t];
      }
      b.n = it.n;
      batch_ctas(it.n, b.ctas);
      if (!(ps & GRAPHIC_PASS_SHIFT)) b.ctas[0] = b.ctas[1] = 0;
      if (!(ps & GRAPHIC_PASS_ROTATE)) b.ctas[2] = b.ctas[3] = b.ctas[4] = 0;
      fr.push_back(b);
    }
  }
  const int nframes = (int)fr.size();
  if (nframes == 0) return GRAPHIC_OK;
  // waves: consecutive frames whose n x 2n scratch fits the wave budget
  const size_t budget = std::max<size_t>((size_t)c->batch_budget_mb << 20, (size_t)1024 * 2048 * 4);
  std::vector<size_t> wave_off(nframes);
  int waves = 0;
  size_t used = 0, wave_max = 0;
  for (int f = 0; f < nframes; f++) {
    const size_t need = fr[f].ctas[2] ? (size_t)fr[f].n * 2 * fr[f].n * sizeof(float) : 0;
    if (f == 0 || used + need > budget) {
      if (f) waves++;
      used = 0;
    }
    fr[f].wave = waves;
    wave_off[f] = used;
    used += need;
    wave_max = std::max(wave_max, used);
  }
  waves++;
  int rc = ensure((void **)&c->d_scratch, &c->scratch_bytes, 2 * wave_max, false);
  if (rc) return rc;
  for (int f = 0; f < nframes; f++)
    fr[f].scratch = c->d_scratch + ((fr[f].wave & 1) ? wave_max / sizeof(float) : 0) + wave_off[f] / sizeof(float);
  // segments in hand-out order
  std::vector<BatchSeg> segs;
  std::vector<int> wave_r3(waves, 0);
  long long total = 0;
  int f0 = 0;
  for (int w = 0; w < waves; w++) {
    int f1 = f0;
    while (f1 < nframes && fr[f1].wave == w) f1++;
    for (int pass = 0; pass < 5; pass++)
      for (int f = f0; f < f1; f++) {
        if (!fr[f].ctas[pass]) continue;
        segs.push_back(BatchSeg{(int)total, f, pass, fr[f].ctas[pass]});
        total += fr[f].ctas[pass];
        if (pass == 4) wave_r3[w] += fr[f].ctas[pass];
      }
    f0 = f1;
  }
  if (total >= (1ll << 31)) return fail(GRAPHIC_ERR_UNSUPPORTED, "batch too large for one launch");
  std::vector<int> seg_of_item((size_t)total);
  for (size_t k = 0; k < segs.size(); k++)
    for (int i = 0; i < segs[k].count; i++) seg_of_item[(size_t)segs[k].item0 + i] = (int)k;
  PlanBuilder pb;
  const size_t o_fr = pb.add(fr.data(), fr.size() * sizeof(BatchFrame));
  const size_t o_sg = pb.add(segs.data(), segs.size() * sizeof(BatchSeg));
  const size_t o_w = pb.add(wave_r3.data(), wave_r3.size() * sizeof(int));
  const size_t o_si = pb.add(seg_of_item.data(), seg_of_item.size() * sizeof(int));
  const size_t cbytes = sizeof(int) * (1 + 5 * (size_t)nframes + waves);
  if ((rc = ensure((void **)&c->d_counters, &c->counters_bytes, cbytes, false))) return rc;
  // the pinned / device plan buffers must not move under a recorded graph
  const size_t pbytes = std::max<size_t>(pb.buf.size(), 16);
  if ((rc = ensure((void **)&c->h_plan, &c->h_plan_bytes, pbytes, true))) return rc;
  if ((rc = ensure((void **)&c->d_plan, &c->d_plan_bytes, pbytes, false))) return rc;
  memcpy(c->h_plan, pb.buf.data(), pb.buf.size());
  BatchArgs b{};
  b.frames = reinterpret_cast<const BatchFrame *>(c->d_plan + o_fr);
  b.segs = reinterpret_cast<const BatchSeg *>(c->d_plan + o_sg);
  b.wave_r3 = reinterpret_cast<const int *>(c->d_plan + o_w);
  b.seg_of_item = reinterpret_cast<const int *>(c->d_plan + o_si);
  b.nseg = (int)segs.size();
  b.total = (int)total;
  b.nframes = nframes;
  b.next = c->d_counters;
  b.done = c->d_counters + 1;
  b.wave_done = c->d_counters + 1 + 5 * (size_t)nframes;
  b.status = c->d_status;
  b.spin_limit = 2000000000ll;   // about one second of clock cycles per wait
  const std::vector<long long> key = {(long long)(uintptr_t)c->h_plan, (long long)(uintptr_t)c->d_plan,
                                      (long long)pb.buf.size(), (long long)o_sg, (long long)o_w, (long long)o_si,
                                      (long long)(uintptr_t)c->d_counters, (long long)cbytes, b.nseg, b.total,
                                      nframes, (long long)(uintptr_t)c->d_status, c->batch_ctas_per_sm,
                                      (long long)(uintptr_t)c->stream};
  if (c->graph_exec && key != c->graph_key) {
    cudaGraphExecDestroy(c->graph_exec);
    cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
  }
  if (!c->graph_exec) {
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_plan, c->h_plan, pb.buf.size(), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counters, 0, cbytes, cs);
    if (e == cudaSuccess) e = launch_batch_persistent(b, c->batch_ctas_per_sm, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e != cudaSuccess ? e : e2, "batch graph capture");
    }
    e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    c->graph = g;
    c->graph_key = key;
  }
  prof_begin(c, GRAPHIC_K_BATCH);
  cudaError_t e = cudaGraphLaunch(c->graph_exec, c->stream);
  prof_end(c);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return GRAPHIC_OK;
}

// Grouped executor.  Frames sorted by (size, steps) and cut into waves whose
// rotation scratch fits group_budget_mb; a wave's passes are launches of that
// size's line-pass kernel over frame-pointer tables.  Waves are dealt round
// robin to group_streams branches of one captured graph: a branch runs its
// waves in order, so wave w reuses the scratch slot of wave w - branches only
// after it finished.  The graph is kept while the layout (wave shapes,
// buffers, stream) is unchanged; per call only the plan is rewritten.
struct GroupWave {
  int n, mask, f0, nf;
};

void drop_group_graph(graphic_ctx *c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->ggraph) cudaGraphDestroy(c->ggraph);
  c->gexec = nullptr;
  c->ggraph = nullptr;
  c->gkey.clear();
}

int batch_grouped(graphic_ctx *c, const graphic_batch_item *items, int32_t n_items) {
  struct Fr {
    const float *in;
    float *out;
    double dx, dy, a, s;
    int q, n, mask;
  };
  std::vector<Fr> fr;
  for (int32_t i = 0; i < n_items; i++) {
    const graphic_batch_item &it = items[i];
    const int ps = item_passes(it);
    RotPlanHost rp;
    if (ps & GRAPHIC_PASS_ROTATE) {
      int rc = plan_rotate(it.theta_deg, it.n_frames, false, rp);
      if (rc) return rc;
    }
    const size_t NN = (size_t)it.n * it.n;
    for (int64_t t = 0; t < it.n_frames; t++) {
      Fr f{};
      f.in = it.in + t * NN;
      f.out = it.out + t * NN;
      f.dx = it.dx ? it.dx[t] : 0.0;
      f.dy = it.dy ? it.dy[t] : 0.0;
      if (ps & GRAPHIC_PASS_ROTATE) {
        f.a = rp.a[t];
        f.s = rp.s[t];
        f.q = rp.q[t];
      }
      f.n = it.n;
      f.mask = ps;
      fr.push_back(f);
    }
  }
  const int nframes = (int)fr.size();
  if (nframes == 0) return GRAPHIC_OK;
  // largest frames first (their launches are the long ones), stable otherwise
  std::stable_sort(fr.begin(), fr.end(), [](const Fr &x, const Fr &y) {
    return x.n != y.n ? x.n > y.n : x.mask < y.mask;
  });
  const size_t budget = (size_t)c->group_budget_mb << 20;
  std::vector<GroupWave> waves;
  size_t slot_bytes = 0;
  for (int f = 0; f < nframes;) {
    const int n = fr[f].n, mask = fr[f].mask;
    // the wave's bytes: rotation scratch (n x 2n), else the frames themselves
    const size_t per = (mask & GRAPHIC_PASS_ROTATE) ? (size_t)n * 2 * n * sizeof(float) : (size_t)n * n * sizeof(float);
    int g = f;
    size_t used = 0;
    while (g < nframes && fr[g].n == n && fr[g].mask == mask && (g == f || used + per <= budget)) {
      used += per;
      g++;
    }
    waves.push_back(GroupWave{n, mask, f, g - f});
    if (mask & GRAPHIC_PASS_ROTATE) slot_bytes = std::max(slot_bytes, used);
    f = g;
  }
  const int R = std::max(1, std::min<int>(c->group_streams, (int)waves.size()));
  int rc;
  if (slot_bytes && (rc = ensure((void **)&c->d_gscratch, &c->gscratch_bytes, slot_bytes * R, false))) return rc;
  // per-line shift parameter tables of a wave (one region per branch):
  // shift x and y per frame, then shears of rotation passes 1/3 and 2
  auto wave_tab_bytes = [](const GroupWave &w) -> size_t {
    size_t b = 0;
    if (w.mask & GRAPHIC_PASS_SHIFT) b += 2 * line_params_bytes(SHIFT_X, w.n, w.nf);
    if (w.mask & GRAPHIC_PASS_ROTATE)
      b += line_params_bytes(ROT_P1, w.n, w.nf) + line_params_bytes(ROT_P2, w.n, w.nf);
    return b;
  };
  size_t tab_bytes = 16;
  for (const GroupWave &w : waves) tab_bytes = std::max(tab_bytes, wave_tab_bytes(w));
  tab_bytes = (tab_bytes + 255) & ~(size_t)255;
  if ((rc = ensure((void **)&c->d_gparam, &c->gparam_bytes, tab_bytes * R, false))) return rc;
  // plan: per frame tables in the sorted order
  std::vector<const float *> tin(nframes), trin(nframes);
  std::vector<float *> tout(nframes);
  std::vector<double> pdx(nframes), pdy(nframes), pa(nframes), ps(nframes);
  std::vector<int> pq(nframes);
  for (int f = 0; f < nframes; f++) {
    tin[f] = fr[f].in;
    tout[f] = fr[f].out;
    trin[f] = (fr[f].mask & GRAPHIC_PASS_SHIFT) ? fr[f].out : fr[f].in;
    pdx[f] = fr[f].dx;
    pdy[f] = fr[f].dy;
    pa[f] = fr[f].a;
    ps[f] = fr[f].s;
    pq[f] = fr[f].q;
  }
  PlanBuilder pb;
  const size_t o_in = pb.add(tin.data(), nframes * sizeof(void *));
  const size_t o_out = pb.add(tout.data(), nframes * sizeof(void *));
  const size_t o_rin = pb.add(trin.data(), nframes * sizeof(void *));
  const size_t o_dx = pb.add(pdx.data(), nframes * sizeof(double));
  const size_t o_dy = pb.add(pdy.data(), nframes * sizeof(double));
  const size_t o_a = pb.add(pa.data(), nframes * sizeof(double));
  const size_t o_s = pb.add(ps.data(), nframes * sizeof(double));
  const size_t o_q = pb.add(pq.data(), nframes * sizeof(int));
  const size_t pbytes = std::max<size_t>(pb.buf.size(), 16);
  if ((rc = ensure((void **)&c->h_plan, &c->h_plan_bytes, pbytes, true))) return rc;
  if ((rc = ensure((void **)&c->d_plan, &c->d_plan_bytes, pbytes, false))) return rc;
  memcpy(c->h_plan, pb.buf.data(), pb.buf.size());
  std::vector<long long> key = {(long long)(uintptr_t)c->h_plan, (long long)(uintptr_t)c->d_plan,
                                (long long)pb.buf.size(), (long long)(uintptr_t)c->d_gscratch, (long long)slot_bytes,
                                (long long)(uintptr_t)c->d_status, R, c->variant_1024, c->precision,
                                (long long)(uintptr_t)c->stream, (long long)(uintptr_t)c->d_gparam,
                                (long long)tab_bytes};
  for (const GroupWave &w : waves) {
    key.push_back(w.n);
    key.push_back(w.mask);
    key.push_back(w.nf);
  }
  while ((int)c->gstreams.size() < R) {
    cudaStream_t st;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    c->gstreams.push_back(st);
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    c->gevents.push_back(ev);
  }
  // the waves on R branches forked from and joined back into `s0`
  auto enqueue = [&](cudaStream_t s0) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(c->d_plan, c->h_plan, pb.buf.size(), cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess && R > 1) e = cudaEventRecord(c->gevents[0], s0);
    for (int r = 1; r < R && e == cudaSuccess; r++) e = cudaStreamWaitEvent(c->gstreams[r], c->gevents[0], 0);
    for (size_t wi = 0; wi < waves.size() && e == cudaSuccess; wi++) {
      const GroupWave &w = waves[wi];
      const int r = (int)(wi % R);
      cudaStream_t st = r ? c->gstreams[r] : s0;
      const long long NM = 2ll * w.n * w.n;
      char *tab = c->d_gparam + (size_t)r * tab_bytes;
      LineArgs a{};
      a.status = c->d_status;
      a.n = w.n;
      if (w.mask & GRAPHIC_PASS_SHIFT) {
        a.in_tab = at<const float *>(c, o_in) + w.f0;
        a.out_tab = at<float *>(c, o_out) + w.f0;
        a.p0 = at<double>(c, o_dx) + w.f0;
        a.p1 = at<double>(c, o_dy) + w.f0;
        const size_t pb1 = line_params_bytes(SHIFT_X, w.n, w.nf);
        e = launch_line_params(SHIFT_X, a, w.nf, tab, st);
        if (e == cudaSuccess) e = launch_line_params(SHIFT_Y, a, w.nf, tab + pb1, st);
        a.lp_lines = 1;
        a.lp_tab = tab;
        if (e == cudaSuccess) e = line_pass(c, SHIFT_X, a, w.nf, st);
        a.in_tab = at<const float *>(c, o_out) + w.f0;
        a.lp_tab = tab + pb1;
        if (e == cudaSuccess) e = line_pass(c, SHIFT_Y, a, w.nf, st);
        tab += 2 * pb1;
      }
      if ((w.mask & GRAPHIC_PASS_ROTATE) && e == cudaSuccess) {
        float *slot = c->d_gscratch + (size_t)r * (slot_bytes / sizeof(float));
        LineArgs b{};
        b.status = c->d_status;
        b.n = w.n;
        b.p0 = at<double>(c, o_a) + w.f0;
        b.p1 = at<double>(c, o_s) + w.f0;
        b.q = at<int>(c, o_q) + w.f0;
        b.in_tab = at<const float *>(c, o_rin) + w.f0;
        b.out = slot;
        b.out_fstride = NM;
        const size_t pb13 = line_params_bytes(ROT_P1, w.n, w.nf);
        e = launch_line_params(ROT_P1, b, w.nf, tab, st);
        if (e == cudaSuccess) e = launch_line_params(ROT_P2, b, w.nf, tab + pb13, st);
        b.lp_tab = tab;
        b.lp_lines = line_params_lines(ROT_P1, w.n);
        if (e == cudaSuccess) e = line_pass(c, ROT_P1, b, w.nf, st);
        b.in_tab = nullptr;
        b.in = slot;
        b.in_fstride = NM;
        b.lp_tab = tab + pb13;
        b.lp_lines = line_params_lines(ROT_P2, w.n);
        if (e == cudaSuccess) e = line_pass(c, ROT_P2, b, w.nf, st);
        b.out = nullptr;
        b.out_tab = at<float *>(c, o_out) + w.f0;
        b.lp_tab = tab;
        b.lp_lines = line_params_lines(ROT_P3, w.n);
        if (e == cudaSuccess) e = line_pass(c, ROT_P3, b, w.nf, st);
      }
    }
    for (int r = 1; r < R && e == cudaSuccess; r++) {
      e = cudaEventRecord(c->gevents[r], c->gstreams[r]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, c->gevents[r], 0);
    }
    return e;
  };
  if (!c->group_graph) {
    // direct launches (a layout that changes every call gains nothing from a graph)
    prof_begin(c, GRAPHIC_K_BATCH);
    cudaError_t e = enqueue(c->stream);
    prof_end(c);
    if (e != cudaSuccess) return cuda_fail(e, "grouped batch launches");
    return GRAPHIC_OK;
  }
  if (c->gexec && key != c->gkey) drop_group_graph(c);
  if (!c->gexec) {
    cudaStream_t s0 = c->gstreams[0];
    cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = enqueue(s0);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s0, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e != cudaSuccess ? e : e2, "grouped batch graph capture");
    }
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      c->gexec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    c->ggraph = g;
    c->gkey = key;
  }
  prof_begin(c, GRAPHIC_K_BATCH);
  cudaError_t e = cudaGraphLaunch(c->gexec, c->stream);
  prof_end(c);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return GRAPHIC_OK;
}

int run_batch(graphic_ctx *c, const graphic_batch_item *items, int32_t n_items, int32_t mode) {
  int rc = validate_batch(items, n_items);
  if (rc) return rc;
  if (mode == GRAPHIC_BATCH_AUTO) mode = c->batch_mode;
  if (mode != GRAPHIC_BATCH_PER_CUBE && mode != GRAPHIC_BATCH_PERSISTENT && mode != GRAPHIC_BATCH_GROUPED)
    return fail(GRAPHIC_ERR_INVALID_ARG, "unknown batch mode");
  if ((rc = begin_call(c))) return rc;
  rc = (mode == GRAPHIC_BATCH_PER_CUBE)     ? batch_per_cube(c, items, n_items)
       : (mode == GRAPHIC_BATCH_PERSISTENT) ? batch_persistent(c, items, n_items)
                                            : batch_grouped(c, items, n_items);
  if (rc) {
    cudaStreamSynchronize(c->stream);
    c->ev_used = 0;
    return rc;
  }
  return end_call(c);
}

// --- schedule cache ---------------------------------------------------------
const char *kTuneKeys[GRAPHIC_SCHEDULE_LEN] = {"chunk_mb",        "variant_1024",  "batch_budget_mb",
                                              "batch_ctas_per_sm", "group_budget_mb", "group_streams",
                                              "batch_mode"};

void schedule_slots(graphic_ctx *c, int *dst[GRAPHIC_SCHEDULE_LEN]) {
  int *v[GRAPHIC_SCHEDULE_LEN] = {&c->chunk_mb,        &c->variant_1024,  &c->batch_budget_mb, &c->batch_ctas_per_sm,
                                  &c->group_budget_mb, &c->group_streams, &c->batch_mode};
  for (int k = 0; k < GRAPHIC_SCHEDULE_LEN; k++) dst[k] = v[k];
}

bool schedule_value_ok(int k, int v) {
  switch (k) {
    case 1: return v == 0 || v == 1;
    case 5: return v >= 1 && v <= 8;
    case 6: return v == GRAPHIC_BATCH_PERSISTENT || v == GRAPHIC_BATCH_GROUPED;
    default: return v > 0;
  }
}

void load_schedule(graphic_ctx *c, const char *path) {
  if (!path || !*path) return;
  FILE *fp = fopen(path, "r");
  if (!fp) return;
  char buf[4096];
  const size_t nread = fread(buf, 1, sizeof(buf) - 1, fp);
  fclose(fp);
  buf[nread] = 0;
  int *dst[GRAPHIC_SCHEDULE_LEN];
  schedule_slots(c, dst);
  for (int k = 0; k < GRAPHIC_SCHEDULE_LEN; k++) {
    char pat[64];
    snprintf(pat, sizeof(pat), "\"%s\":", kTuneKeys[k]);
    const char *q = strstr(buf, pat);
    int v;
    if (q && sscanf(q + strlen(pat), " %d", &v) == 1 && schedule_value_ok(k, v)) *dst[k] = v;
  }
}

int save_schedule(graphic_ctx *c, const char *path) {
  if (!path || !*path) return GRAPHIC_OK;
  FILE *fp = fopen(path, "w");
  if (!fp) return fail(GRAPHIC_ERR_INVALID_ARG, std::string("cannot write ") + path);
  int *v[GRAPHIC_SCHEDULE_LEN];
  schedule_slots(c, v);
  fprintf(fp, "{");
  for (int k = 0; k < GRAPHIC_SCHEDULE_LEN; k++) fprintf(fp, "%s\"%s\": %d", k ? ", " : "", kTuneKeys[k], *v[k]);
  fprintf(fp, "}\n");
  fclose(fp);
  return GRAPHIC_OK;
}

// Device milliseconds of one batch call (after one untimed call).
int time_batch(graphic_ctx *c, const graphic_batch_item *items, int32_t n_items, int32_t mode, int reps, float *ms) {
  int rc = run_batch(c, items, n_items, mode);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int r = 0; r < reps; r++) {
    cudaEventRecord(e0, c->stream);
    rc = run_batch(c, items, n_items, mode);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    if (rc) break;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    best = std::min(best, t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return rc;
}

}  // namespace

int graphic::set_last_error(int code, const char *msg) { return fail(code, msg); }

int graphic::ctx_batch_async(graphic_ctx *c, const graphic_batch_item *items, int32_t n_items, int32_t mode) {
  int rc = validate_batch(items, n_items);
  if (rc) return rc;
  if (mode == GRAPHIC_BATCH_AUTO) mode = c->batch_mode;
  if ((rc = begin_call(c))) return rc;
  switch (mode) {
    case GRAPHIC_BATCH_PER_CUBE: return batch_per_cube(c, items, n_items);
    case GRAPHIC_BATCH_PERSISTENT: return batch_persistent(c, items, n_items);
    case GRAPHIC_BATCH_GROUPED: return batch_grouped(c, items, n_items);
  }
  return fail(GRAPHIC_ERR_INVALID_ARG, "unknown batch mode");
}

void graphic::ctx_set_graph_batches(graphic_ctx *c, bool on) { c->group_graph = on; }

const int *graphic::ctx_status_async(graphic_ctx *c) {
  if (cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return nullptr;
  return c->h_status;
}

size_t graphic::ctx_workspace_bound(const graphic_ctx *c, int32_t mode) {
  if (mode == GRAPHIC_BATCH_AUTO) mode = c->batch_mode;
  const size_t mb = 1ull << 20;
  size_t ws = 64 * mb;   // plans, tables, counters
  // grouped: the branches' rotation scratch and their parameter tables (at
  // most half the scratch: 3n lines of 80 bytes per frame against 8 n^2)
  if (mode == GRAPHIC_BATCH_GROUPED)
    ws += (size_t)c->group_streams * std::max<size_t>(c->group_budget_mb * mb, 8 * mb) * 3 / 2;
  else if (mode == GRAPHIC_BATCH_PERSISTENT) ws += 2 * std::max<size_t>(c->batch_budget_mb * mb, 8 * mb);
  else ws += std::max<size_t>((size_t)c->chunk_mb * mb * 2, 8 * mb);
  return ws;
}

extern "C" {

int graphic_version(void) { return 10000; }

const char *graphic_last_error(void) { return g_err.c_str(); }

int graphic_create(graphic_ctx **out, int device) {
  if (!out) return fail(GRAPHIC_ERR_INVALID_ARG, "null out");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(GRAPHIC_ERR_INVALID_ARG, "no such device");
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3)
    return fail(GRAPHIC_ERR_UNSUPPORTED, "built for sm_103a (GB300); device is sm_" + std::to_string(prop.major) +
                                             std::to_string(prop.minor));
  DeviceGuard g(device);
  graphic_ctx *c = new graphic_ctx();
  c->device = device;
  if (geom_init_device() != 0 || tc_init_device() != 0) {
    delete c;
    return fail(GRAPHIC_ERR_CUDA, "twiddle table upload failed");
  }
  e = cudaMalloc(&c->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_status, sizeof(int));
  if (e != cudaSuccess) {
    graphic_destroy(c);
    return cuda_fail(e, "context allocation");
  }
  load_schedule(c, getenv("GRAPHIC_TUNE_CACHE"));
  *out = c;
  return GRAPHIC_OK;
}

int graphic_release(graphic_ctx *c) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  cudaFree(c->d_plan);
  cudaFreeHost(c->h_plan);
  cudaFree(c->d_scratch);
  cudaFree(c->d_cube);
  cudaFree(c->d_img);
  cudaFree(c->d_bscratch);
  c->d_bscratch = nullptr;
  c->bscratch_bytes = 0;
  cudaFree(c->d_lparam);
  c->d_lparam = nullptr;
  c->lparam_bytes = 0;
  cudaFree(c->d_gparam);
  c->d_gparam = nullptr;
  c->gparam_bytes = 0;
  cudaFree(c->d_counters);
  cudaFree(c->d_gscratch);
  c->d_gscratch = nullptr;
  cudaFree(c->d_prep);
  c->d_prep = nullptr;
  c->prep_bytes = 0;
  c->gscratch_bytes = 0;
  drop_group_graph(c);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->graph_exec = nullptr;
  c->graph = nullptr;
  c->graph_key.clear();
  c->d_counters = nullptr;
  c->counters_bytes = 0;
  c->d_plan = nullptr;
  c->h_plan = nullptr;
  c->d_scratch = nullptr;
  c->d_cube = nullptr;
  c->d_img = nullptr;
  c->d_plan_bytes = c->h_plan_bytes = c->scratch_bytes = c->cube_bytes = c->img_bytes = 0;
  return GRAPHIC_OK;
}

int graphic_destroy(graphic_ctx *c) {
  if (!c) return GRAPHIC_OK;
  graphic_release(c);
  DeviceGuard g(c->device);
  cudaFree(c->d_status);
  cudaFreeHost(c->h_status);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  for (cudaEvent_t e : c->gevents) cudaEventDestroy(e);
  if (c->ev_copy) cudaEventDestroy(c->ev_copy);
  if (c->s_copy) cudaStreamDestroy(c->s_copy);
  for (cudaStream_t st : c->gstreams) cudaStreamDestroy(st);
  delete c;
  return GRAPHIC_OK;
}

int graphic_set_stream(graphic_ctx *c, void *stream) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  c->stream = (cudaStream_t)stream;
  return GRAPHIC_OK;
}

int graphic_shift(graphic_ctx *c, const float *in, float *out, int64_t T, int32_t n, const double *dx,
                  const double *dy) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  int rc = check_cube(in, out, T, n);
  if (rc) return rc;
  if ((rc = validate_shift(dx, dy, T, n))) return rc;
  if (T == 0) return GRAPHIC_OK;
  DeviceGuard g(c->device);
  PlanBuilder pb;
  const size_t o_dx = pb.add(dx, T * sizeof(double));
  const size_t o_dy = pb.add(dy, T * sizeof(double));
  if ((rc = begin_call(c))) return rc;
  if ((rc = upload_plan(c, pb))) return rc;
  if ((rc = enqueue_shift(c, in, out, T, n, at<double>(c, o_dx), at<double>(c, o_dy)))) return rc;
  return end_call(c);
}

int graphic_rotate(graphic_ctx *c, const float *in, float *out, int64_t T, int32_t n, const double *theta) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  int rc = check_cube(in, out, T, n);
  if (rc) return rc;
  if (T > 0 && !theta) return fail(GRAPHIC_ERR_INVALID_ARG, "null theta");
  if (T == 0) return GRAPHIC_OK;
  RotPlanHost rp;
  if ((rc = plan_rotate(theta, T, false, rp))) return rc;
  DeviceGuard g(c->device);
  PlanBuilder pb;
  const size_t o_a = pb.add(rp.a.data(), T * sizeof(double));
  const size_t o_s = pb.add(rp.s.data(), T * sizeof(double));
  const size_t o_q = pb.add(rp.q.data(), T * sizeof(int));
  if ((rc = begin_call(c))) return rc;
  if ((rc = upload_plan(c, pb))) return rc;
  if ((rc = enqueue_rotate(c, in, out, T, n, at<double>(c, o_a), at<double>(c, o_s), at<int>(c, o_q)))) return rc;
  return end_call(c);
}

int graphic_adi_subtract_ex(graphic_ctx *c, const float *in, float *out, int64_t T, int32_t n,
                            const double *parang, const double *times, double t_max, double fwhm, double n_fwhm,
                            const double *edges, int32_t n_edges) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  int rc = check_cube(in, out, T, n);
  if (rc) return rc;
  if ((rc = validate_adi(parang, T, fwhm, n_fwhm, edges, n_edges))) return rc;
  AdiPlanHost ap;
  if ((rc = plan_adi(parang, T, fwhm, n_fwhm, edges, n_edges, ap, times, t_max))) return rc;
  if ((rc = plan_band_path(ap, T, n))) return rc;
  DeviceGuard g(c->device);
  PlanBuilder pb;
  const AdiOffsets oa = add_adi_plan(pb, ap, T);
  if ((rc = begin_call(c))) return rc;
  if ((rc = upload_plan(c, pb))) return rc;
  if ((rc = enqueue_adi(c, in, out, T, n, ap, oa))) return rc;
  return end_call(c);
}

int graphic_adi_subtract(graphic_ctx *c, const float *in, float *out, int64_t T, int32_t n, const double *parang,
                         double fwhm, double n_fwhm, const double *edges, int32_t n_edges) {
  return graphic_adi_subtract_ex(c, in, out, T, n, parang, nullptr, 0.0, fwhm, n_fwhm, edges, n_edges);
}

int graphic_collapse_median(graphic_ctx *c, const float *in, int64_t T, int32_t n, float *out) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  int rc = check_cube(in, out, T, n);
  if (rc) return rc;
  if (T < 1) return fail(GRAPHIC_ERR_INVALID_ARG, "n_frames < 1");
  DeviceGuard g(c->device);
  if ((rc = begin_call(c))) return rc;
  if ((rc = enqueue_collapse(c, in, T, n, out))) return rc;
  return end_call(c);
}

int graphic_reduce_ex(graphic_ctx *c, const float *in, float *work, int64_t T, int32_t n, const double *dx,
                      const double *dy, const double *parang, const double *times, double t_max, double fwhm,
                      double n_fwhm, const double *edges, int32_t n_edges, float *out) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  int rc = check_cube(in, work, T, n);
  if (rc) return rc;
  if (!out) return fail(GRAPHIC_ERR_INVALID_ARG, "null out");
  DeviceGuard g(c->device);
  if ((rc = reduce_device(c, in, work, T, n, dx, dy, parang, fwhm, n_fwhm, edges, n_edges, out, nullptr, times,
                          t_max))) {
    cudaStreamSynchronize(c->stream);
    c->ev_used = 0;
    return rc;
  }
  return end_call(c);
}

int graphic_reduce(graphic_ctx *c, const float *in, float *work, int64_t T, int32_t n, const double *dx,
                   const double *dy, const double *parang, double fwhm, double n_fwhm, const double *edges,
                   int32_t n_edges, float *out) {
  return graphic_reduce_ex(c, in, work, T, n, dx, dy, parang, nullptr, 0.0, fwhm, n_fwhm, edges, n_edges, out);
}

int graphic_reduce_host(graphic_ctx *c, const float *host_in, int64_t T, int32_t n, const double *dx,
                        const double *dy, const double *parang, double fwhm, double n_fwhm, const double *edges,
                        int32_t n_edges, float *host_out) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  int rc = check_cube(host_in, host_out, T, n, false);
  if (rc) return rc;
  if (T < 1) return fail(GRAPHIC_ERR_INVALID_ARG, "n_frames < 1");
  DeviceGuard g(c->device);
  const size_t NN = (size_t)n * n;
  if ((rc = ensure((void **)&c->d_cube, &c->cube_bytes, (size_t)T * NN * sizeof(float), false))) return rc;
  if ((rc = ensure((void **)&c->d_img, &c->img_bytes, NN * sizeof(float), false))) return rc;
  if ((rc = reduce_device(c, c->d_cube, c->d_cube, T, n, dx, dy, parang, fwhm, n_fwhm, edges, n_edges, c->d_img,
                          host_in))) {
    cudaStreamSynchronize(c->stream);
    c->ev_used = 0;
    return rc;
  }
  CK(cudaMemcpyAsync(host_out, c->d_img, NN * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  return end_call(c);
}

// --- strided cubes ------------------------------------------------------------
namespace {
int check_cube_desc(const graphic_cube *cb, const char *what, long long &fs) {
  if (!cb) return fail(GRAPHIC_ERR_INVALID_ARG, std::string("null ") + what + " cube");
  const long long NN = (long long)cb->n * cb->n;
  fs = cb->frame_stride ? cb->frame_stride : NN;
  if (cb->frame_stride && (cb->frame_stride < NN || (cb->frame_stride & 3)))
    return fail(GRAPHIC_ERR_INVALID_ARG, std::string(what) + ": frame_stride must be 0 or >= n*n and a multiple of 4");
  return GRAPHIC_OK;
}
int check_pair(const graphic_cube *in, const graphic_cube *out, long long &ifs, long long &ofs) {
  int rc = check_cube_desc(in, "in", ifs);
  if (rc) return rc;
  if ((rc = check_cube_desc(out, "out", ofs))) return rc;
  if (in->n != out->n || in->n_frames != out->n_frames)
    return fail(GRAPHIC_ERR_INVALID_ARG, "in and out cubes differ in n or n_frames");
  return check_cube(in->data, out->data, in->n_frames, in->n);
}
}  // namespace

int graphic_shift_cube(graphic_ctx *c, const graphic_cube *in, const graphic_cube *out, const double *dx,
                       const double *dy) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  long long ifs, ofs;
  int rc = check_pair(in, out, ifs, ofs);
  if (rc) return rc;
  const int64_t T = in->n_frames;
  const int32_t n = in->n;
  if ((rc = validate_shift(dx, dy, T, n))) return rc;
  if (T == 0) return GRAPHIC_OK;
  DeviceGuard g(c->device);
  PlanBuilder pb;
  const size_t o_dx = pb.add(dx, T * sizeof(double));
  const size_t o_dy = pb.add(dy, T * sizeof(double));
  if ((rc = begin_call(c))) return rc;
  if ((rc = upload_plan(c, pb))) return rc;
  if ((rc = enqueue_shift(c, in->data, out->data, T, n, at<double>(c, o_dx), at<double>(c, o_dy), ifs, ofs)))
    return rc;
  return end_call(c);
}

int graphic_rotate_cube(graphic_ctx *c, const graphic_cube *in, const graphic_cube *out, const double *theta) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  long long ifs, ofs;
  int rc = check_pair(in, out, ifs, ofs);
  if (rc) return rc;
  const int64_t T = in->n_frames;
  const int32_t n = in->n;
  if (T > 0 && !theta) return fail(GRAPHIC_ERR_INVALID_ARG, "null theta");
  if (T == 0) return GRAPHIC_OK;
  RotPlanHost rp;
  if ((rc = plan_rotate(theta, T, false, rp))) return rc;
  DeviceGuard g(c->device);
  PlanBuilder pb;
  const size_t o_a = pb.add(rp.a.data(), T * sizeof(double));
  const size_t o_s = pb.add(rp.s.data(), T * sizeof(double));
  const size_t o_q = pb.add(rp.q.data(), T * sizeof(int));
  if ((rc = begin_call(c))) return rc;
  if ((rc = upload_plan(c, pb))) return rc;
  if ((rc = enqueue_rotate(c, in->data, out->data, T, n, at<double>(c, o_a), at<double>(c, o_s), at<int>(c, o_q),
                           ifs, ofs)))
    return rc;
  return end_call(c);
}

int graphic_adi_subtract_cube(graphic_ctx *c, const graphic_cube *in, const graphic_cube *out, const double *parang,
                              double fwhm, double n_fwhm, const double *edges, int32_t n_edges) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  long long ifs, ofs;
  int rc = check_pair(in, out, ifs, ofs);
  if (rc) return rc;
  const int64_t T = in->n_frames;
  const int32_t n = in->n;
  if ((rc = validate_adi(parang, T, fwhm, n_fwhm, edges, n_edges))) return rc;
  AdiPlanHost ap;
  if ((rc = plan_adi(parang, T, fwhm, n_fwhm, edges, n_edges, ap))) return rc;
  if ((rc = plan_band_path(ap, T, n))) return rc;
  DeviceGuard g(c->device);
  PlanBuilder pb;
  const AdiOffsets oa = add_adi_plan(pb, ap, T);
  if ((rc = begin_call(c))) return rc;
  if ((rc = upload_plan(c, pb))) return rc;
  if ((rc = enqueue_adi(c, in->data, out->data, T, n, ap, oa, ifs, ofs))) return rc;
  return end_call(c);
}

int graphic_collapse_median_cube(graphic_ctx *c, const graphic_cube *in, float *out) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  long long ifs;
  int rc = check_cube_desc(in, "in", ifs);
  if (rc) return rc;
  if ((rc = check_cube(in->data, out, in->n_frames, in->n))) return rc;
  if (in->n_frames < 1) return fail(GRAPHIC_ERR_INVALID_ARG, "n_frames < 1");
  DeviceGuard g(c->device);
  if ((rc = begin_call(c))) return rc;
  if ((rc = enqueue_collapse(c, in->data, in->n_frames, in->n, out, ifs))) return rc;
  return end_call(c);
}

int graphic_reduce_cube(graphic_ctx *c, const graphic_cube *in, const graphic_cube *work, const double *dx,
                        const double *dy, const double *parang, double fwhm, double n_fwhm, const double *edges,
                        int32_t n_edges, float *out) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  long long ifs, wfs;
  int rc = check_pair(in, work, ifs, wfs);
  if (rc) return rc;
  if (!out) return fail(GRAPHIC_ERR_INVALID_ARG, "null out");
  DeviceGuard g(c->device);
  if ((rc = reduce_device(c, in->data, work->data, in->n_frames, in->n, dx, dy, parang, fwhm, n_fwhm, edges, n_edges,
                          out, nullptr, nullptr, 0.0, ifs, wfs))) {
    cudaStreamSynchronize(c->stream);
    c->ev_used = 0;
    return rc;
  }
  return end_call(c);
}

int graphic_batch_geom(graphic_ctx *c, const graphic_batch_item *items, int32_t n_items, int32_t mode) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  DeviceGuard g(c->device);
  return run_batch(c, items, n_items, mode);
}

int graphic_autotune(graphic_ctx *c, const graphic_batch_item *items, int32_t n_items, const char *cache_path,
                     double *best_ms) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  DeviceGuard g(c->device);
  int rc = validate_batch(items, n_items);
  if (rc) return rc;
  float ms;
  // per-cube schedule: intermediate per chunk, kernel of 1024-point lines
  int best_chunk = c->chunk_mb, best_var = c->variant_1024;
  float best_pc = 1e30f;
  for (int var = 0; var <= 1; var++)
    for (int mb : {64, 256, 1024, 4096}) {
      c->chunk_mb = mb;
      c->variant_1024 = var;
      if ((rc = time_batch(c, items, n_items, GRAPHIC_BATCH_PER_CUBE, 2, &ms))) return rc;
      if (ms < best_pc) {
        best_pc = ms;
        best_chunk = mb;
        best_var = var;
      }
    }
  c->chunk_mb = best_chunk;
  c->variant_1024 = best_var;
  // persistent executor: wave budget, CTAs per SM
  int best_budget = c->batch_budget_mb, best_cps = c->batch_ctas_per_sm;
  float best_ps = 1e30f;
  for (int cps = 1; cps <= 2; cps++)
    for (int mb : {128, 4096}) {
      c->batch_budget_mb = mb;
      c->batch_ctas_per_sm = cps;
      if ((rc = time_batch(c, items, n_items, GRAPHIC_BATCH_PERSISTENT, 2, &ms))) return rc;
      if (ms < best_ps) {
        best_ps = ms;
        best_budget = mb;
        best_cps = cps;
      }
    }
  c->batch_budget_mb = best_budget;
  c->batch_ctas_per_sm = best_cps;
  // grouped executor: wave budget, concurrent branches
  int best_gb = c->group_budget_mb, best_gs = c->group_streams;
  float best_gr = 1e30f;
  for (int gs : {1, 2, 3, 4})
    for (int mb : {32, 64, 128, 256}) {
      c->group_budget_mb = mb;
      c->group_streams = gs;
      if ((rc = time_batch(c, items, n_items, GRAPHIC_BATCH_GROUPED, 2, &ms))) return rc;
      if (ms < best_gr) {
        best_gr = ms;
        best_gb = mb;
        best_gs = gs;
      }
    }
  c->group_budget_mb = best_gb;
  c->group_streams = best_gs;
  c->batch_mode = (best_gr <= best_ps) ? GRAPHIC_BATCH_GROUPED : GRAPHIC_BATCH_PERSISTENT;
  if (best_ms) {
    best_ms[0] = best_pc;
    best_ms[1] = best_ps;
    best_ms[2] = best_gr;
  }
  return save_schedule(c, cache_path);
}

int graphic_get_schedule(graphic_ctx *c, int32_t *values, int32_t n) {
  if (!c || !values || n < 0) return fail(GRAPHIC_ERR_INVALID_ARG, "bad arguments");
  int *v[GRAPHIC_SCHEDULE_LEN];
  schedule_slots(c, v);
  for (int32_t k = 0; k < n && k < GRAPHIC_SCHEDULE_LEN; k++) values[k] = *v[k];
  return GRAPHIC_OK;
}

int graphic_set_schedule(graphic_ctx *c, const int32_t *values, int32_t n) {
  if (!c || !values || n < 0) return fail(GRAPHIC_ERR_INVALID_ARG, "bad arguments");
  int *dst[GRAPHIC_SCHEDULE_LEN];
  schedule_slots(c, dst);
  for (int32_t k = 0; k < n && k < GRAPHIC_SCHEDULE_LEN; k++)
    if (!schedule_value_ok(k, values[k])) return fail(GRAPHIC_ERR_INVALID_ARG, "bad schedule value");
  for (int32_t k = 0; k < n && k < GRAPHIC_SCHEDULE_LEN; k++) *dst[k] = values[k];
  return GRAPHIC_OK;
}

int graphic_set_precision(graphic_ctx *c, int32_t precision) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  if (precision != GRAPHIC_PREC_FP32 && precision != GRAPHIC_PREC_BF16X3 && precision != GRAPHIC_PREC_FP16X3)
    return fail(GRAPHIC_ERR_INVALID_ARG, "unknown precision");
  c->precision = precision;
  drop_group_graph(c);   // recorded launches name the kernels
  return GRAPHIC_OK;
}

int graphic_get_precision(graphic_ctx *c, int32_t *precision) {
  if (!c || !precision) return fail(GRAPHIC_ERR_INVALID_ARG, "bad arguments");
  *precision = c->precision;
  return GRAPHIC_OK;
}

// --- image-quality pre-processing (Sect. 3.2) ----------------------------------
int graphic_sky_median(graphic_ctx *c, const float *in, int64_t T, int32_t n, const double *mask_x,
                       const double *mask_y, double mask_r, float *sky) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  int rc = check_cube(in, sky, T, n);
  if (rc) return rc;
  if (T < 1) return fail(GRAPHIC_ERR_INVALID_ARG, "n_frames < 1");
  if ((mask_x == nullptr) != (mask_y == nullptr)) return fail(GRAPHIC_ERR_INVALID_ARG, "mask_x and mask_y go together");
  if (!std::isfinite(mask_r) || mask_r < 0) return fail(GRAPHIC_ERR_INVALID_ARG, "mask_r must be finite, >= 0");
  DeviceGuard g(c->device);
  PlanBuilder pb;
  size_t o_mx = 0, o_my = 0;
  if (mask_x) {
    o_mx = pb.add(mask_x, T * sizeof(double));
    o_my = pb.add(mask_y, T * sizeof(double));
  }
  if ((rc = begin_call(c))) return rc;
  if ((rc = upload_plan(c, pb))) return rc;
  CollapseArgs a{};
  a.in = in;
  a.out = sky;
  a.status = c->d_status;
  a.T = T;
  a.n = n;
  a.mask_x = mask_x ? at<double>(c, o_mx) : nullptr;
  a.mask_y = mask_x ? at<double>(c, o_my) : nullptr;
  a.mask_r2 = mask_r * mask_r;
  prof_begin(c, GRAPHIC_K_COLLAPSE);
  cudaError_t e = launch_sky_median(a, c->stream);
  prof_end(c);
  if (e != cudaSuccess) return cuda_fail(e, "sky median kernel");
  return end_call(c);
}

int graphic_sky_subtract(graphic_ctx *c, const float *in, float *out, int64_t T, int32_t n, const float *skies,
                         int32_t n_skies, const double *frame_times, const double *sky_times) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  int rc = check_cube(in, out, T, n);
  if (rc) return rc;
  if (n_skies < 1 || !skies || ((uintptr_t)skies & 15)) return fail(GRAPHIC_ERR_INVALID_ARG, "need >= 1 aligned sky");
  if (T > 0 && (!frame_times || !sky_times)) return fail(GRAPHIC_ERR_INVALID_ARG, "null times");
  std::vector<int> j(T, 0);
  for (int64_t t = 0; t < T; t++) {
    if (!std::isfinite(frame_times[t])) return fail(GRAPHIC_ERR_INVALID_ARG, "non-finite time");
    for (int s = 1; s < n_skies; s++)
      if (fabs(sky_times[s] - frame_times[t]) < fabs(sky_times[j[t]] - frame_times[t])) j[t] = s;
  }
  if (T == 0) return GRAPHIC_OK;
  DeviceGuard g(c->device);
  PlanBuilder pb;
  const size_t o_j = pb.add(j.data(), T * sizeof(int));
  if ((rc = begin_call(c))) return rc;
  if ((rc = upload_plan(c, pb))) return rc;
  cudaError_t e = launch_sky_subtract(in, out, T, n, skies, at<int>(c, o_j), c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sky subtraction kernel");
  return end_call(c);
}

namespace {

// host value of a total-order key
float key_value(uint32_t key) {
  const uint32_t b = (key & 0x80000000u) ? (key & 0x7fffffffu) : ~key;
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
}

// Key of the k-th smallest (0-based) of n_vals device floats: four radix
// passes, each a device histogram read back by the host.
int select_key(graphic_ctx *c, const float *v, long long n_vals, unsigned long long k, unsigned int *d_hist,
               uint32_t *key) {
  uint32_t prefix = 0, pmask = 0;
  unsigned long long krem = k;
  std::vector<unsigned int> h(256);
  for (int pass = 0; pass < 4; pass++) {
    const int shift = 24 - 8 * pass;
    cudaError_t e = launch_key_histogram(v, n_vals, prefix, pmask, shift, d_hist, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_hist, 256 * sizeof(unsigned int), cudaMemcpyDeviceToHost,
                                              c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "frame median");
    unsigned long long cum = 0;
    int d = 255;
    for (int b = 0; b < 256; b++) {
      if (cum + h[b] > krem) {
        d = b;
        break;
      }
      cum += h[b];
    }
    krem -= cum;
    prefix |= (uint32_t)d << shift;
    pmask |= 0xffu << shift;
  }
  *key = prefix;
  return GRAPHIC_OK;
}

}  // namespace

int graphic_bad_pixel_map(graphic_ctx *c, const float *ref, int32_t n, double C, uint8_t *map) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  if (!ref || !map || n < 1) return fail(GRAPHIC_ERR_INVALID_ARG, "null buffer or n < 1");
  if (!std::isfinite(C) || C < 0) return fail(GRAPHIC_ERR_INVALID_ARG, "C must be finite, >= 0");
  DeviceGuard g(c->device);
  const long long N = (long long)n * n;
  int rc;
  if ((rc = ensure((void **)&c->d_prep, &c->prep_bytes, 4096, false))) return rc;
  unsigned int *d_hist = reinterpret_cast<unsigned int *>(c->d_prep);          // 1 KB
  double *d_sums = reinterpret_cast<double *>(c->d_prep + 1024);              // 2 doubles
  double *d_mean = d_sums + 2;
  double *d_thresh = d_sums + 3;
  float *d_med = reinterpret_cast<float *>(c->d_prep + 1024 + 64);
  double sums[2] = {0, 0};
  CK(cudaMemsetAsync(d_sums, 0, 2 * sizeof(double), c->stream));
  cudaError_t e = launch_frame_sums(ref, N, nullptr, d_sums, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "frame sums");
  CK(cudaMemcpyAsync(sums, d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (!std::isfinite(sums[0])) return fail(GRAPHIC_ERR_NONFINITE, "non-finite value in the reference frame");
  const double mean = sums[0] / (double)N;
  CK(cudaMemcpyAsync(d_mean, &mean, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  e = launch_frame_sums(ref, N, d_mean, d_sums, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "frame sums");
  CK(cudaMemcpyAsync(sums, d_sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const double sigma = sqrt(sums[1] / (double)N);
  uint32_t klo, khi;
  if ((rc = select_key(c, ref, N, (unsigned long long)((N - 1) / 2), d_hist, &klo))) return rc;
  float med = key_value(klo);
  if ((N & 1) == 0) {
    if ((rc = select_key(c, ref, N, (unsigned long long)(N / 2), d_hist, &khi))) return rc;
    const float hi = key_value(khi);
    volatile float s = med + hi;   // FP32 sum, then the halving, as the device medians
    med = s * 0.5f;
  }
  const double thresh = C * sigma;
  CK(cudaMemcpyAsync(d_med, &med, sizeof(float), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d_thresh, &thresh, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  e = launch_bad_map(ref, N, d_med, d_thresh, map, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bad pixel map kernel");
  CK(cudaStreamSynchronize(c->stream));
  return GRAPHIC_OK;
}

int graphic_bad_pixel_fix(graphic_ctx *c, float *cube, int64_t T, int32_t n, const uint8_t *map) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  if (T < 0 || (T > 0 && !cube) || n < 1) return fail(GRAPHIC_ERR_INVALID_ARG, "bad cube");
  if (T == 0) return GRAPHIC_OK;
  DeviceGuard g(c->device);
  const size_t bytes = (size_t)T * n * n * sizeof(float);
  int rc;
  if ((rc = ensure((void **)&c->d_prep, &c->prep_bytes, 4096, false))) return rc;
  if ((rc = ensure((void **)&c->d_scratch, &c->scratch_bytes, bytes, false))) return rc;
  unsigned long long *d_cnt = reinterpret_cast<unsigned long long *>(c->d_prep + 2048);   // [3]
  unsigned long long cnt[3] = {0, 0, 0};
  CK(cudaMemsetAsync(d_cnt, 0, 3 * sizeof(unsigned long long), c->stream));
  cudaError_t e = launch_bad_mark(cube, T, n, map, d_cnt, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bad pixel marking kernel");
  CK(cudaMemcpyAsync(cnt, d_cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  unsigned long long left = cnt[0];
  float *src = cube, *dst = c->d_scratch;
  bool hopeless = false;
  for (int pass = 0; left > 0 && pass <= 2 * n; pass++) {
    CK(cudaMemsetAsync(d_cnt + 1, 0, 2 * sizeof(unsigned long long), c->stream));
    e = launch_bad_pass(src, dst, T, n, d_cnt + 1, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "bad pixel pass kernel");
    CK(cudaMemcpyAsync(cnt + 1, d_cnt + 1, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::swap(src, dst);
    if (cnt[2] == 0) {
      hopeless = true;
      break;
    }
    left = cnt[1];
  }
  if (src != cube) CK(cudaMemcpyAsync(cube, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (hopeless || left > 0) return fail(GRAPHIC_ERR_NONFINITE, "a frame has no finite pixel left to fill from");
  return GRAPHIC_OK;
}

int graphic_register(graphic_ctx *c, const float *in, int64_t T, int32_t n, double thresh, int32_t R,
                     int32_t min_size, int32_t max_size, int32_t w, double *out, int32_t *iters) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  if (T < 0 || T > (int64_t)INT32_MAX * 4 || n < 1 || n > 65535) return fail(GRAPHIC_ERR_INVALID_ARG, "bad cube shape");
  if (T > 0 && (!in || !out)) return fail(GRAPHIC_ERR_INVALID_ARG, "null buffer");
  if ((uintptr_t)in & 15) return fail(GRAPHIC_ERR_INVALID_ARG, "the cube must be 16-byte aligned");
  if (R < 1 || R > 32 || w < 1 || w > 32) return fail(GRAPHIC_ERR_INVALID_ARG, "R and w must lie in 1..32");
  if (std::isnan(thresh)) return fail(GRAPHIC_ERR_INVALID_ARG, "thresh is NaN");
  if (T == 0) return GRAPHIC_OK;
  DeviceGuard g(c->device);
  int rc;
  if ((rc = ensure((void **)&c->d_scratch, &c->scratch_bytes, register_keys_bytes(T), false))) return rc;
  if ((rc = begin_call(c))) return rc;
  RegArgs a;
  a.in = in;
  a.out = out;
  a.iters = iters;
  a.status = c->d_status;
  a.T = T;
  a.n = n;
  a.thresh = thresh;
  a.R = R;
  a.min_size = min_size;
  a.max_size = max_size;
  a.w = w;
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(c->d_scratch);
  prof_begin(c, GRAPHIC_K_REG_ARGMAX);
  cudaError_t e = launch_register_argmax(a, keys, c->stream);
  prof_end(c);
  if (e != cudaSuccess) return cuda_fail(e, "registration argmax kernel");
  prof_begin(c, GRAPHIC_K_REG_FIT);
  e = launch_register_fit(a, keys, c->stream);
  prof_end(c);
  if (e != cudaSuccess) return cuda_fail(e, "registration fit kernel");
  return end_call(c);
}

int graphic_bin_median(graphic_ctx *c, const float *in, float *out, int64_t T, int32_t n, int32_t B) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  int rc = check_cube(in, out, T, n);
  if (rc) return rc;
  if (B < 1) return fail(GRAPHIC_ERR_INVALID_ARG, "B must be >= 1");
  if (T == 0) return GRAPHIC_OK;
  DeviceGuard g(c->device);
  if ((rc = begin_call(c))) return rc;
  int launched = 0;
  prof_begin(c, GRAPHIC_K_BIN);
  cudaError_t e = launch_bin_median(in, out, T, n, B, c->d_status, c->stream, &launched);
  prof_end(c);
  if (c->prof && launched > 1) c->prof_extra[GRAPHIC_K_BIN] += launched - 1;
  if (e != cudaSuccess) return cuda_fail(e, "binning kernel");
  return end_call(c);
}

int graphic_bin_mean(const double *v, int64_t n, int32_t B, double *out) {
  if (n < 0 || B < 1 || (n > 0 && (!v || !out))) return fail(GRAPHIC_ERR_INVALID_ARG, "bad arguments");
  for (int64_t g = 0; g * B < n; g++) {
    const int64_t f0 = g * B, f1 = std::min<int64_t>(n, f0 + B);
    double s = 0.0;
    for (int64_t f = f0; f < f1; f++) s += v[f];
    out[g] = s / (double)(f1 - f0);
  }
  return GRAPHIC_OK;
}

int graphic_inject(graphic_ctx *c, float *cube, int64_t T, int32_t n, const double *parang, const double *xc,
                   const double *yc, int32_t n_comp, const double *r, const double *pa0, const double *flux,
                   const double *alpha, const double *beta, int32_t half) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  if (T < 0 || n < 1 || n_comp < 0 || half < 0 || half > 4096) return fail(GRAPHIC_ERR_INVALID_ARG, "bad sizes");
  if (T == 0 || n_comp == 0) return GRAPHIC_OK;
  if (!cube || !parang || !xc || !yc || !r || !pa0 || !flux || !alpha || !beta)
    return fail(GRAPHIC_ERR_INVALID_ARG, "null buffer");
  if (T > INT32_MAX) return fail(GRAPHIC_ERR_INVALID_ARG, "too many frames");
  const double PI = 3.14159265358979323846;
  std::vector<double> pos((size_t)T * n_comp * 2);
  std::vector<int> win((size_t)T * n_comp * 2);
  std::vector<float> amp((size_t)T * n_comp), shape((size_t)T * 2);
  for (int j = 0; j < n_comp; j++)
    if (!std::isfinite(r[j]) || !std::isfinite(pa0[j]) || !std::isfinite(flux[j]))
      return fail(GRAPHIC_ERR_INVALID_ARG, "non-finite companion parameter");
  for (int64_t t = 0; t < T; t++) {
    if (!(alpha[t] > 0) || !(beta[t] > 1) || !std::isfinite(alpha[t]) || !std::isfinite(beta[t]) ||
        !std::isfinite(parang[t]) || !std::isfinite(xc[t]) || !std::isfinite(yc[t]))
      return fail(GRAPHIC_ERR_INVALID_ARG, "alpha > 0, beta > 1 and finite angles / centres required");
    shape[2 * t] = (float)(1.0 / (alpha[t] * alpha[t]));
    shape[2 * t + 1] = (float)beta[t];
    for (int j = 0; j < n_comp; j++) {
      const size_t q = (size_t)t * n_comp + j;
      const double ang = (pa0[j] + parang[t]) * PI / 180.0;
      const double xp = xc[t] + r[j] * cos(ang), yp = yc[t] + r[j] * sin(ang);
      pos[2 * q] = xp;
      pos[2 * q + 1] = yp;
      const double fr = floor(yp + 0.5), fc = floor(xp + 0.5);
      // a window entirely off the frame is skipped by the kernel's bounds test; keep the ints in range
      win[2 * q] = (int)std::max(-1e9, std::min(1e9, fr));
      win[2 * q + 1] = (int)std::max(-1e9, std::min(1e9, fc));
      amp[q] = (float)(flux[j] * (beta[t] - 1.0) / (PI * alpha[t] * alpha[t]));
    }
  }
  DeviceGuard g(c->device);
  PlanBuilder pb;
  const size_t o_pos = pb.add(pos.data(), pos.size() * sizeof(double));
  const size_t o_win = pb.add(win.data(), win.size() * sizeof(int));
  const size_t o_amp = pb.add(amp.data(), amp.size() * sizeof(float));
  const size_t o_shape = pb.add(shape.data(), shape.size() * sizeof(float));
  int rc;
  if ((rc = begin_call(c))) return rc;
  if ((rc = upload_plan(c, pb))) return rc;
  cudaError_t e = launch_inject(cube, T, n, n_comp, at<double>(c, o_pos), at<int>(c, o_win), at<float>(c, o_amp),
                                at<float>(c, o_shape), half, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "injection kernel");
  return end_call(c);
}

int graphic_aperture(graphic_ctx *c, const float *img, int32_t n, int32_t n_ap, const double *x, const double *y,
                     double radius, double *out) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  if (n < 1 || n_ap < 0 || !(radius >= 0) || !std::isfinite(radius)) return fail(GRAPHIC_ERR_INVALID_ARG, "bad sizes");
  if (n_ap == 0) return GRAPHIC_OK;
  if (!img || !x || !y || !out) return fail(GRAPHIC_ERR_INVALID_ARG, "null buffer");
  std::vector<double> xy((size_t)n_ap * 2);
  for (int k = 0; k < n_ap; k++) {
    if (!std::isfinite(x[k]) || !std::isfinite(y[k])) return fail(GRAPHIC_ERR_INVALID_ARG, "non-finite position");
    xy[2 * k] = x[k];
    xy[2 * k + 1] = y[k];
  }
  DeviceGuard g(c->device);
  PlanBuilder pb;
  const size_t o_xy = pb.add(xy.data(), xy.size() * sizeof(double));
  int rc;
  if ((rc = ensure((void **)&c->d_prep, &c->prep_bytes, std::max<size_t>(4096, (size_t)n_ap * sizeof(double)),
                   false)))
    return rc;
  if ((rc = begin_call(c))) return rc;
  if ((rc = upload_plan(c, pb))) return rc;
  double *d_out = reinterpret_cast<double *>(c->d_prep);
  cudaError_t e = launch_aperture(img, n, n_ap, at<double>(c, o_xy), radius, d_out, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "aperture kernel");
  CK(cudaMemcpyAsync(out, d_out, (size_t)n_ap * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return end_call(c);
}

int graphic_profile(graphic_ctx *c, int enable) {
  if (!c) return fail(GRAPHIC_ERR_INVALID_ARG, "null ctx");
  c->prof = enable != 0;
  if (c->prof) {
    for (int k = 0; k < GRAPHIC_K_COUNT; k++) {
      c->prof_ms[k] = 0;
      c->prof_n[k] = 0;
      c->prof_extra[k] = 0;
    }
  }
  c->ev_used = 0;
  return GRAPHIC_OK;
}

int graphic_profile_read(graphic_ctx *c, double *ms, int64_t *launches, int32_t n) {
  if (!c || !ms || !launches || n < 0) return fail(GRAPHIC_ERR_INVALID_ARG, "bad arguments");
  for (int32_t k = 0; k < n && k < GRAPHIC_K_COUNT; k++) {
    ms[k] = c->prof_ms[k];
    launches[k] = c->prof_n[k];
  }
  return GRAPHIC_OK;
}

const char *graphic_kernel_name(int32_t k) {
  static const char *names[GRAPHIC_K_COUNT] = {"shift_x", "shift_y", "adi_general", "rot_pass1",
                                              "rot_pass2", "rot_pass3", "collapse_median", "batch_persistent",
                                              "register_argmax", "register_fit", "bin_median", "adi_band_prep",
                                              "adi_band_sweep"};
  return (k >= 0 && k < GRAPHIC_K_COUNT) ? names[k] : nullptr;
}

int graphic_workspace_bytes(graphic_ctx *c, int64_t *bytes) {
  if (!c || !bytes) return fail(GRAPHIC_ERR_INVALID_ARG, "bad arguments");
  *bytes = (int64_t)(c->d_plan_bytes + c->scratch_bytes + c->gscratch_bytes + c->cube_bytes + c->img_bytes +
                     c->counters_bytes + c->bscratch_bytes + c->lparam_bytes + c->gparam_bytes);
  return GRAPHIC_OK;
}

}  // extern "C"

// noalloc.cu -- graphic_rotate_noalloc: the three-shear rotation without any
// device allocation, for callers that cannot call cudaMalloc -- e.g. code
// running under an allocator or memory-pool policy that forbids it, a plugin
// or library handed only a stream and pre-allocated buffers by its host,
// or a latency-critical path that must not trigger allocator work.
//
// Everything the rotation needs besides the caller's input and output lives
// in file-scope static __device__ arrays of fixed size (held on every GPU
// that loads this library, until the process exits):
//   g_scratch  16 MiB: the n x 2n intermediate of up to kScratchFloats / (2 n^2)
//              frames at a time (2 frames at n = 1024, 8 at n = 512, ...);
//   g_a, g_s, g_q  the per-frame plan of one such chunk;
//   g_status   the non-finite-input flag, cleared at the start of every call.
// The scratch is written completely by rotation pass 1 before pass 2 reads
// it, so its old contents never matter.  All calls share these arrays:
// two calls that overlap on the GPU (different streams, or different host
// threads) race and give wrong results; serialise them.
//
// Set-up: the first call on a device (with that device current) takes the
// device addresses of the arrays with cudaGetSymbolAddress and uploads the
// FFT twiddle tables; do that first call before any stream capture.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "../../include/graphic.h"
#include "graphic_internal.h"

namespace graphic {
namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;
constexpr size_t kScratchFloats = kScratchBytes / sizeof(float);
constexpr int kPlanMax = (int)(kScratchFloats / (64 * 128));   // most frames per chunk (n = 64)

static __device__ __align__(256) float g_scratch[kScratchFloats];
static __device__ __align__(256) double g_a[kPlanMax];
static __device__ __align__(256) double g_s[kPlanMax];
static __device__ __align__(256) int g_q[kPlanMax];
static __device__ __align__(256) int g_status;

struct DevSyms {
  bool ready = false;
  float *scratch = nullptr;
  double *a = nullptr;
  double *s = nullptr;
  int *q = nullptr;
  int *status = nullptr;
};

constexpr int kMaxDevices = 64;
DevSyms g_syms[kMaxDevices];
std::mutex g_setup_mu;

const double kPi = 3.14159265358979323846264338327950288;

int setup_device(int dev, DevSyms **out) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DevSyms &d = g_syms[dev];
  if (!d.ready) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return GRAPHIC_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3) return GRAPHIC_ERR_UNSUPPORTED;
    if (cudaGetSymbolAddress((void **)&d.scratch, g_scratch) != cudaSuccess) return GRAPHIC_ERR_CUDA;
    if (cudaGetSymbolAddress((void **)&d.a, g_a) != cudaSuccess) return GRAPHIC_ERR_CUDA;
    if (cudaGetSymbolAddress((void **)&d.s, g_s) != cudaSuccess) return GRAPHIC_ERR_CUDA;
    if (cudaGetSymbolAddress((void **)&d.q, g_q) != cudaSuccess) return GRAPHIC_ERR_CUDA;
    if (cudaGetSymbolAddress((void **)&d.status, g_status) != cudaSuccess) return GRAPHIC_ERR_CUDA;
    if (geom_init_device() != 0) return GRAPHIC_ERR_CUDA;
    d.ready = true;
  }
  *out = &d;
  return GRAPHIC_OK;
}

}  // namespace
}  // namespace graphic

using namespace graphic;

extern "C" int graphic_rotate_noalloc(const float *in, float *out, int64_t n_frames, int32_t n,
                                      const double *theta_deg, void *stream) {
  if (n_frames < 0) return set_last_error(GRAPHIC_ERR_INVALID_ARG, "n_frames < 0");
  if (n != 64 && n != 128 && n != 256 && n != 512 && n != 1024)
    return set_last_error(GRAPHIC_ERR_UNSUPPORTED, "n must be one of 64, 128, 256, 512, 1024");
  const size_t frame_scratch = (size_t)n * 2 * n * sizeof(float);
  if (frame_scratch > kScratchBytes)
    return set_last_error(GRAPHIC_ERR_UNSUPPORTED, "one frame's n x 2n scratch exceeds the 16 MiB static scratch");
  if (n_frames == 0) return GRAPHIC_OK;
  if (!in || !out || !theta_deg) return set_last_error(GRAPHIC_ERR_INVALID_ARG, "null pointer");
  for (int64_t t = 0; t < n_frames; t++)
    if (!isfinite(theta_deg[t]) || fabs(theta_deg[t]) > 1e6)
      return set_last_error(GRAPHIC_ERR_INVALID_ARG, "angle not finite or |angle| > 1e6 deg");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_last_error(GRAPHIC_ERR_CUDA, "no current CUDA device");
  DevSyms *sym = nullptr;
  int rc = setup_device(dev, &sym);
  if (rc) return set_last_error(rc, "set-up of the static scratch failed on this device");
  cudaStream_t st = (cudaStream_t)stream;

  const long long NN = (long long)n * n;
  const long long NM = 2 * NN;
  long long ch = (long long)(kScratchFloats / (size_t)NM);
  if (ch > kPlanMax) ch = kPlanMax;
  if (cudaMemsetAsync(sym->status, 0, sizeof(int), st) != cudaSuccess)
    return set_last_error(GRAPHIC_ERR_CUDA, "status clear failed");
  double pa[kPlanMax], ps[kPlanMax];
  int pq[kPlanMax];
  for (long long f0 = 0; f0 < n_frames; f0 += ch) {
    const long long nf = (n_frames - f0 < ch) ? (n_frames - f0) : ch;
    // the plan of this chunk: theta = 90 q + theta', a = tan(theta'/2), s = sin(theta')
    for (long long t = 0; t < nf; t++) {
      const double th = theta_deg[f0 + t];
      const int q = (int)floor(th / 90.0 + 0.5);
      const double tp = th - 90.0 * (double)q;
      if (tp == 0.0) {
        pa[t] = 0.0;
        ps[t] = 0.0;
      } else {
        const double r = tp * kPi / 180.0;
        pa[t] = tan(r / 2.0);
        ps[t] = sin(r);
      }
      pq[t] = ((q % 4) + 4) % 4;
    }
    // pageable source: the copies return once the data is staged, so the
    // stack arrays can be refilled for the next chunk (stream order keeps the
    // device plan of this chunk until its kernels have run)
    if (cudaMemcpyAsync(sym->a, pa, nf * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(sym->s, ps, nf * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(sym->q, pq, nf * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return set_last_error(GRAPHIC_ERR_CUDA, "plan upload failed");
    LineArgs a{};
    a.p0 = sym->a;
    a.p1 = sym->s;
    a.q = sym->q;
    a.status = sym->status;
    a.n = n;
    a.in = in + f0 * NN;
    a.out = sym->scratch;
    a.in_fstride = NN;
    a.out_fstride = NM;
    cudaError_t e = launch_line_pass(ROT_P1, a, nf, st);
    a.in = sym->scratch;
    a.in_fstride = NM;
    if (e == cudaSuccess) e = launch_line_pass(ROT_P2, a, nf, st);
    a.out = out + f0 * NN;
    a.out_fstride = NN;
    if (e == cudaSuccess) e = launch_line_pass(ROT_P3, a, nf, st);
    if (e != cudaSuccess) return set_last_error(GRAPHIC_ERR_CUDA, cudaGetErrorString(e));
  }
  int h_status = 0;
  if (cudaMemcpyAsync(&h_status, sym->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return set_last_error(GRAPHIC_ERR_CUDA, "stream synchronisation failed");
  if (h_status & STATUS_NONFINITE) return set_last_error(GRAPHIC_ERR_NONFINITE, "non-finite value in the input cube");
  return GRAPHIC_OK;
}

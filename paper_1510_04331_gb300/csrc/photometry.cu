// photometry.cu -- the photometric-accuracy and binning experiments (Sect.
// 4.2, 4.3): median binning of consecutive frames, fake companion injection
// into raw frames, aperture photometry of the reduced image.
//
//  * bin_median_kernel<W>: one thread per (group, pixel); the group's B <= W
//    values are loaded (coalesced along the pixels, all loads in flight),
//    turned into total-order keys padded with the largest key, sorted by a
//    bitonic network in registers (all indices compile-time) and the median
//    taken by the collapse rule.  HBM-bound: T x n^2 x 4 B read, ceil(T/B) x
//    n^2 x 4 B written.  Groups of more than 64 frames go to the median
//    collapse kernel, one launch per group.
//  * inject_kernel: one block per frame; companions in turn (a barrier
//    between them, so overlapping windows never race), each over its window
//    of (2 half + 1)^2 pixels; positions and windows come from the FP64 host
//    plan, the Moffat profile is evaluated in FP32.
//  * aperture_kernel: one block per aperture over the bounding box of the
//    disc, FP64 block sum.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "graphic_internal.h"

namespace graphic {
namespace {

constexpr int BIN_THREADS = 128;

__device__ __forceinline__ uint32_t bkey(float x) {
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float bval(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

template <int W>
__global__ void __launch_bounds__(BIN_THREADS) bin_median_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                                 long long T, long long nn, int B,
                                                                 long long blocks_per_group, int *status) {
  const long long g = blockIdx.x / blocks_per_group;
  const long long p = (blockIdx.x - g * blocks_per_group) * BIN_THREADS + threadIdx.x;
  if (p >= nn) return;
  const long long f0 = g * B;
  const int m = (int)((T - f0) < B ? (T - f0) : B);
  const float *src = in + f0 * nn + p;
  uint32_t k[W];
  bool bad = false;
#pragma unroll
  for (int i = 0; i < W; i++) {
    if (i < m) {
      const float v = __ldcs(src + (long long)i * nn);
      bad |= !(fabsf(v) <= 3.402823466e38f);
      k[i] = bkey(v);
    } else {
      k[i] = 0xffffffffu;
    }
  }
  if (bad) atomicOr(status, STATUS_NONFINITE);
#pragma unroll
  for (int s = 2; s <= W; s <<= 1)
#pragma unroll
    for (int j = s >> 1; j > 0; j >>= 1)
#pragma unroll
      for (int i = 0; i < W; i++) {
        const int l = i ^ j;
        if (l > i) {
          const uint32_t a = k[i], b = k[l];
          const bool up = (i & s) == 0;
          k[i] = up ? min(a, b) : max(a, b);
          k[l] = up ? max(a, b) : min(a, b);
        }
      }
  const int ilo = (m - 1) >> 1, ihi = m >> 1;
  uint32_t lo = 0, hi = 0;
#pragma unroll
  for (int i = 0; i < W; i++) {
    if (i == ilo) lo = k[i];
    if (i == ihi) hi = k[i];
  }
  const float a = bval(lo);
  out[g * nn + p] = (m & 1) ? a : (a + bval(hi)) * 0.5f;
}

__global__ void inject_kernel(float *cube, long long T, int n, int n_comp, const double *__restrict__ pos,
                              const int *__restrict__ win, const float *__restrict__ amp,
                              const float *__restrict__ shape, int half) {
  const long long t = blockIdx.x;
  float *fr = cube + t * (long long)n * n;
  const int side = 2 * half + 1;
  const float ia2 = shape[2 * t], beta = shape[2 * t + 1];
  for (int j = 0; j < n_comp; j++) {
    const long long q = t * n_comp + j;
    const double xp = pos[2 * q], yp = pos[2 * q + 1];
    const int cr = win[2 * q], cc = win[2 * q + 1];
    const float A = amp[q];
    for (int i = threadIdx.x; i < side * side; i += blockDim.x) {
      const int row = cr - half + i / side, col = cc - half + i % side;
      if (row < 0 || row >= n || col < 0 || col >= n) continue;
      const double dx = (double)col - xp, dy = (double)row - yp;
      const float rho2 = (float)(dx * dx + dy * dy);
      const float u = 1.0f + rho2 * ia2;
      const float m = A * exp2f(-beta * log2f(u));
      float *px = fr + (long long)row * n + col;
      *px = *px + m;
    }
    __syncthreads();   // the next companion's window may overlap this one
  }
}

__global__ void aperture_kernel(const float *__restrict__ img, int n, const double *__restrict__ xy, double radius,
                                double *out) {
  __shared__ double part[32];
  const int k = blockIdx.x;
  const double x = xy[2 * k], y = xy[2 * k + 1], r2 = radius * radius;
  const int r0 = max(0, (int)floor(y - radius) - 1), r1 = min(n - 1, (int)ceil(y + radius) + 1);
  const int c0 = max(0, (int)floor(x - radius) - 1), c1 = min(n - 1, (int)ceil(x + radius) + 1);
  double s = 0.0;
  if (r0 <= r1 && c0 <= c1) {
    const int W = c1 - c0 + 1, H = r1 - r0 + 1;
    for (int i = threadIdx.x; i < W * H; i += blockDim.x) {
      const int row = r0 + i / W, col = c0 + i % W;
      const double dx = (double)col - x, dy = (double)row - y;
      if (dx * dx + dy * dy <= r2) s += (double)img[(long long)row * n + col];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
    out[k] = t;
  }
}

template <int W>
cudaError_t bin_launch(const float *in, float *out, long long T, long long nn, int B, int *status,
                       cudaStream_t st) {
  const long long G = (T + B - 1) / B;
  const long long bpg = (nn + BIN_THREADS - 1) / BIN_THREADS;
  if (G * bpg > 0x7fffffffLL) return cudaErrorInvalidConfiguration;   // one block per (bin, 128 pixels)
  bin_median_kernel<W><<<(unsigned)(G * bpg), BIN_THREADS, 0, st>>>(in, out, T, nn, B, bpg, status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bin_median(const float *in, float *out, long long T, int n, int B, int *status, cudaStream_t st,
                              int *launched) {
  if (launched) *launched = 0;
  if (T <= 0) return cudaSuccess;
  const long long nn = (long long)n * n;
  const long long G = (T + B - 1) / B;
  cudaError_t e;
  if (B <= 16) {
    e = bin_launch<16>(in, out, T, nn, B, status, st);
  } else if (B <= 32) {
    e = bin_launch<32>(in, out, T, nn, B, status, st);
  } else if (B <= 64) {
    e = bin_launch<64>(in, out, T, nn, B, status, st);
  } else {
    for (long long g = 0; g < G; g++) {
      CollapseArgs a{};
      a.in = in + g * B * nn;
      a.out = out + g * nn;
      a.status = status;
      a.T = (T - g * B) < B ? (T - g * B) : B;
      a.n = n;
      if ((e = launch_collapse(a, st)) != cudaSuccess) return e;
    }
    if (launched) *launched = (int)G;
    return cudaSuccess;
  }
  if (launched && e == cudaSuccess) *launched = 1;
  return e;
}

cudaError_t launch_inject(float *cube, long long T, int n, int n_comp, const double *pos, const int *win,
                          const float *amp, const float *shape, int half, cudaStream_t st) {
  if (T <= 0 || n_comp <= 0) return cudaSuccess;
  inject_kernel<<<(unsigned)T, 256, 0, st>>>(cube, T, n, n_comp, pos, win, amp, shape, half);
  return cudaGetLastError();
}

cudaError_t launch_aperture(const float *img, int n, int n_ap, const double *xy, double radius, double *out,
                            cudaStream_t st) {
  if (n_ap <= 0) return cudaSuccess;
  aperture_kernel<<<(unsigned)n_ap, 256, 0, st>>>(img, n, xy, radius, out);
  return cudaGetLastError();
}

}  // namespace graphic

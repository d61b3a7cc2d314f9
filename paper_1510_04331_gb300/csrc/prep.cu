// prep.cu -- image-quality pre-processing (Sect. 3.2): sky subtraction with
// the master sky closest in time, the pieces of the sigma-clip bad pixel
// map (radix histograms of total-order keys, FP64 frame sums, the map), and
// the neighbour-median bad pixel correction.  The master sky itself is the
// masked variant of the median collapse (median.cu).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "graphic_internal.h"

namespace graphic {
namespace {

// IEEE total-order key of a float: a larger key is a larger value, -0 < +0.
__device__ __forceinline__ uint32_t key_of(float x) {
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// out[t] = in[t] - skies[sky_of_frame[t]], four floats per thread.
__global__ void sky_subtract_kernel(const float4 *__restrict__ in, float4 *__restrict__ out, long long T,
                                    long long nn4, const float4 *__restrict__ skies,
                                    const int *__restrict__ sky_of_frame) {
  const long long total = T * nn4;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long t = i / nn4, q = i - t * nn4;
    const float4 a = in[i];
    const float4 b = skies[(long long)__ldg(&sky_of_frame[t]) * nn4 + q];
    out[i] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
  }
}

// 256-bin histogram of digit `shift` of the keys matching prefix under pmask.
__global__ void key_histogram_kernel(const float *__restrict__ v, long long n, uint32_t prefix, uint32_t pmask,
                                     int shift, unsigned int *hist) {
  __shared__ unsigned int h[256];
  for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint32_t k = key_of(v[i]);
    if ((k & pmask) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], h[b]);
}

// FP64 sum of v (mean == null) or of (v - *mean)^2, block partials then one
// atomic per block.
__global__ void frame_sums_kernel(const float *__restrict__ v, long long n, const double *mean, double *sums) {
  __shared__ double part[8];
  double acc = 0.0;
  const double mu = mean ? *mean : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double x = (double)v[i];
    acc += mean ? (x - mu) * (x - mu) : x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += part[w];
    atomicAdd(&sums[mean ? 1 : 0], s);
  }
}

// map[p] = |ref[p] - med| > thresh (FP64 comparison).
__global__ void bad_map_kernel(const float *__restrict__ ref, long long n, const float *med, const double *thresh,
                               uint8_t *map) {
  const double m = (double)*med, th = *thresh;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    map[i] = fabs((double)ref[i] - m) > th ? 1 : 0;
}

__device__ __forceinline__ void count_block(unsigned long long mine, unsigned long long *dst) {
  __shared__ unsigned long long part[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += part[w];
    if (s) atomicAdd(dst, s);
  }
  __syncthreads();   // part is reused by the next call
}

// Flagged and non-finite pixels become NaN; counts them.
__global__ void bad_mark_kernel(float *cube, long long T, long long nn, const uint8_t *map,
                                unsigned long long *nan_count) {
  unsigned long long mine = 0;
  const long long total = T * nn;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = cube[i];
    const bool bad = !isfinite(v) || (map && map[i % nn]);
    if (bad) {
      cube[i] = __uint_as_float(0x7fc00000u);
      mine++;
    }
  }
  count_block(mine, nan_count);
}

// One pass: every NaN pixel with a finite 8-neighbour in src takes the median
// of those neighbours (two middle values averaged for an even count, FP32);
// counts[0] += NaN pixels left, counts[1] += pixels filled.
__global__ void bad_pass_kernel(const float *__restrict__ src, float *__restrict__ dst, long long T, int n,
                                unsigned long long *counts) {
  unsigned long long left = 0, filled = 0;
  const long long nn = (long long)n * n, total = T * nn;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = src[i];
    if (!isnan(v)) {
      dst[i] = v;
      continue;
    }
    const long long f = i / nn, p = i - f * nn;
    const int r = (int)(p / n), c = (int)(p - (long long)r * n);
    const float *fr = src + f * nn;
    uint32_t k[8];
    int m = 0;
#pragma unroll
    for (int dr = -1; dr <= 1; dr++)
#pragma unroll
      for (int dc = -1; dc <= 1; dc++) {
        if (!dr && !dc) continue;
        const int rr = r + dr, cc = c + dc;
        if (rr < 0 || rr >= n || cc < 0 || cc >= n) continue;
        const float w = fr[(long long)rr * n + cc];
        if (!isnan(w)) k[m++] = key_of(w);
      }
    if (m == 0) {
      dst[i] = v;
      left++;
      continue;
    }
    // insertion sort of at most 8 keys
    for (int a = 1; a < m; a++) {
      const uint32_t x = k[a];
      int b = a - 1;
      while (b >= 0 && k[b] > x) {
        k[b + 1] = k[b];
        b--;
      }
      k[b + 1] = x;
    }
    auto val = [](uint32_t key) {
      return __uint_as_float((key & 0x80000000u) ? (key & 0x7fffffffu) : ~key);
    };
    const float lo = val(k[(m - 1) / 2]);
    dst[i] = (m & 1) ? lo : (lo + val(k[m / 2])) * 0.5f;
    filled++;
  }
  count_block(left, &counts[0]);
  count_block(filled, &counts[1]);
}

unsigned grid_for(long long work, int threads) {
  long long g = (work + threads - 1) / threads;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

cudaError_t launch_sky_subtract(const float *in, float *out, long long T, int n, const float *skies,
                                const int *sky_of_frame, cudaStream_t st) {
  const long long nn4 = (long long)n * n / 4;
  if (T <= 0) return cudaSuccess;
  sky_subtract_kernel<<<grid_for(T * nn4, 256), 256, 0, st>>>(reinterpret_cast<const float4 *>(in),
                                                              reinterpret_cast<float4 *>(out), T, nn4,
                                                              reinterpret_cast<const float4 *>(skies), sky_of_frame);
  return cudaGetLastError();
}

cudaError_t launch_key_histogram(const float *v, long long n_vals, uint32_t prefix, uint32_t pmask, int shift,
                                 unsigned int *hist, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  key_histogram_kernel<<<grid_for(n_vals, 256), 256, 0, st>>>(v, n_vals, prefix, pmask, shift, hist);
  return cudaGetLastError();
}

cudaError_t launch_frame_sums(const float *v, long long n_vals, const double *mean, double *sums, cudaStream_t st) {
  frame_sums_kernel<<<grid_for(n_vals, 256), 256, 0, st>>>(v, n_vals, mean, sums);
  return cudaGetLastError();
}

cudaError_t launch_bad_map(const float *ref, long long n_vals, const float *med, const double *thresh,
                           uint8_t *map, cudaStream_t st) {
  bad_map_kernel<<<grid_for(n_vals, 256), 256, 0, st>>>(ref, n_vals, med, thresh, map);
  return cudaGetLastError();
}

cudaError_t launch_bad_mark(float *cube, long long T, int n, const uint8_t *map, unsigned long long *nan_count,
                            cudaStream_t st) {
  const long long nn = (long long)n * n;
  bad_mark_kernel<<<grid_for(T * nn, 256), 256, 0, st>>>(cube, T, nn, map, nan_count);
  return cudaGetLastError();
}

cudaError_t launch_bad_pass(const float *src, float *dst, long long T, int n, unsigned long long *counts,
                            cudaStream_t st) {
  const long long nn = (long long)n * n;
  bad_pass_kernel<<<grid_for(T * nn, 256), 256, 0, st>>>(src, dst, T, n, counts);
  return cudaGetLastError();
}

}  // namespace graphic

// line_common.cuh -- device helpers shared by the line-pass kernels (the
// FP32 Stockham kernels of geom.cu and the tensor-core kernels of tc.cu):
// complex arithmetic, the per-line shift parameters with their FP64 phase
// reduction, and the frame loads of the five pass kinds.  Each translation
// unit gets its own copy (anonymous namespace).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "graphic_internal.h"

namespace graphic {
namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

struct LineParam {
  float dhi, dlo;   // delta = d / m split: delta_hi on a 2^-12 grid, delta_lo the rest
  float cnyq;       // cos(pi d), Nyquist weight
  float pad_;
  float2 step[8];   // exp(-i 2 pi r delta), r = 0..7
};

__device__ __forceinline__ float2 phase_at(const LineParam &p, int K);

// m is a power of two, so d / m and the 2^-12 grid split are exact in FP64;
// the eight steps use the split in FP32 like every other phase (a few FP64
// operations per line on GB300's narrow FP64 pipe).
__device__ __forceinline__ void make_param(LineParam &p, double d, int m) {
  const double delta = d * (1.0 / (double)m);
  const double dhi = rint(delta * 4096.0) * (1.0 / 4096.0);
  p.dhi = (float)dhi;
  p.dlo = (float)(delta - dhi);
  const double d2 = d - 2.0 * rint(0.5 * d);   // d mod 2, exact
  p.cnyq = cospif((float)d2);
  p.pad_ = 0.f;
#pragma unroll
  for (int r = 0; r < 8; r++) p.step[r] = phase_at(p, r);
}

// exp(-i 2 pi K delta) for integer 0 <= K < 2^11.
__device__ __forceinline__ float2 phase_at(const LineParam &p, int K) {
  float kf = (float)K;
  float t = kf * p.dhi;      // exact: K < 2^11, dhi on a 2^-12 grid with |dhi| <= 1
  t -= rintf(t);
  t = fmaf(kf, p.dlo, t);
  float s, c;
  sincospif(2.0f * t, &s, &c);
  return make_float2(c, -s);
}

template <int KIND>
__device__ __forceinline__ double line_shift(const LineArgs &a, long long f, int line, int n) {
  const int m = 2 * n;
  if constexpr (KIND == SHIFT_X) return a.p0[f];
  else if constexpr (KIND == SHIFT_Y) return a.p1[f];
  else if constexpr (KIND == ROT_P2) return a.p1[f] * (double)(((line + n / 2) & (m - 1)) - n);
  else return -a.p0[f] * (double)(line - n / 2);
}

__device__ __forceinline__ bool finite_pair(float2 v) { return isfinite(v.x) && isfinite(v.y); }

// Global loads of frame data: through L1 normally; L2 only (.cg) in the
// persistent batch kernel, whose CTAs read data other CTAs of the same
// launch wrote (L1 is not coherent across SMs).
template <bool CG>
__device__ __forceinline__ float ldf(const float *p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}
template <bool CG>
__device__ __forceinline__ float2 ldf2(const float *p) {
  if constexpr (CG) return __ldcg(reinterpret_cast<const float2 *>(p));
  else return *reinterpret_cast<const float2 *>(p);
}

// Load element `pos` (< n) of row `line` of rot90^q(frame) and of row line+1.
template <bool CG = false>
__device__ __forceinline__ float2 load_rot90_pair(const float *__restrict__ fr, int n, int q, int line, int pos) {
  float x0 = 0.f, x1 = 0.f;
  switch (q) {
    case 0:
      x0 = ldf<CG>(fr + (size_t)line * n + pos);
      x1 = ldf<CG>(fr + (size_t)(line + 1) * n + pos);
      break;
    case 1:   // g[i][j] = in[n - j][i]  (j >= 1)
      if (pos >= 1) {
        float2 t = ldf2<CG>(fr + (size_t)(n - pos) * n + line);
        x0 = t.x;
        x1 = t.y;
      }
      break;
    case 2:   // g[i][j] = in[n - i][n - j]  (i, j >= 1)
      if (pos >= 1) {
        if (line >= 1) x0 = ldf<CG>(fr + (size_t)(n - line) * n + (n - pos));
        x1 = ldf<CG>(fr + (size_t)(n - line - 1) * n + (n - pos));
      }
      break;
    default:  // g[i][j] = in[j][n - i]  (i >= 1)
      if (line >= 1) x0 = ldf<CG>(fr + (size_t)pos * n + (n - line));
      x1 = ldf<CG>(fr + (size_t)pos * n + (n - line - 1));
      break;
  }
  return make_float2(x0, x1);
}

}  // namespace
}  // namespace graphic

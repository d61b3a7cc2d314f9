// register.cu -- registration (Sect. 3.1): per frame the centroid of the
// patch of contiguous pixels above a threshold around the brightest pixel,
// then a Moffat fit by Levenberg-Marquardt started there; the centre gives
// the recentring shift, alpha and beta the FWHM.
//
// Two kernels.
//  * frame_argmax_kernel: the only pass over whole frames, HBM-bound.  One
//    block per (frame, chunk of REG_CHUNK pixels), 16-byte loads; each block
//    merges its maximum into the frame's 64-bit word by atomicMax on the
//    packed (total-order key of the value, ~index): the largest value wins,
//    the smallest index on a tie.  A non-finite value sets the word to all
//    ones (no finite value packs to it) and the status flag.
//  * register_fit_kernel: one warp per frame.  The box of half-size R around
//    the seed and its 8-connected flood fill in shared memory (sweeps until
//    none changes: the fixpoint is the connected component whatever the
//    order of the updates), FP64 patch sums, then the fit window in the same
//    shared buffer and the Levenberg-Marquardt loop.  Every sum is a
//    butterfly (xor) shuffle reduction, which leaves the bit-identical sum in
//    every lane (each level adds the same two operands, commuted), so every
//    lane solves the same damped 6 x 6 system and takes the same decisions:
//    no broadcast, no block barrier, and several frames per SM keep the FP64
//    pipe busy.  Start values, damping schedule and stopping rules are those
//    of the FP64 oracle.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "graphic_internal.h"

namespace graphic {
namespace {

constexpr int ARG_THREADS = 256;
constexpr int ARG_VEC = 8;                                   // float4 loads per thread per chunk
constexpr long long REG_CHUNK = (long long)ARG_THREADS * ARG_VEC * 4;   // pixels per block
constexpr int FIT_WARPS = 1;   // one warp (frame) per block: small batches spread over all SMs
constexpr double REG_PI = 3.14159265358979323846;
constexpr unsigned long long KEY_NONFINITE = ~0ull;

__device__ __forceinline__ uint32_t order_key(float x) {
  if (x == 0.0f) x = 0.0f;   // -0 and +0 compare equal: the index decides
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ unsigned long long pack(float v, uint32_t idx) {
  return ((unsigned long long)order_key(v) << 32) | (unsigned long long)(~idx);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  return x;
}

__global__ void __launch_bounds__(ARG_THREADS) frame_argmax_kernel(const float *__restrict__ in, long long T,
                                                                   long long nn, long long chunks,
                                                                   unsigned long long *keys, int *status) {
  __shared__ unsigned long long part[ARG_THREADS / 32];
  __shared__ int part_bad[ARG_THREADS / 32];
  const long long items = T * chunks;
  const bool vec = (nn & 3) == 0;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const long long f = it / chunks, c = it - f * chunks;
    const float *fr = in + f * nn;
    const long long s = c * REG_CHUNK, e = min(nn, s + REG_CHUNK);
    float best = -INFINITY;
    long long bi = -1;
    bool bad = false;
    if (vec) {
      const float4 *f4 = reinterpret_cast<const float4 *>(fr);
      const long long s4 = s >> 2, e4 = e >> 2;
      float4 v[ARG_VEC];
#pragma unroll
      for (int k = 0; k < ARG_VEC; k++) {
        const long long j = s4 + threadIdx.x + (long long)k * ARG_THREADS;
        v[k] = j < e4 ? __ldcs(&f4[j]) : make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
      }
#pragma unroll
      for (int k = 0; k < ARG_VEC; k++) {
        const long long j = s4 + threadIdx.x + (long long)k * ARG_THREADS;
        const float q[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
        if (j < e4) {
#pragma unroll
          for (int l = 0; l < 4; l++) {
            bad |= !(fabsf(q[l]) <= 3.402823466e38f);
            if (q[l] > best || bi < 0) {
              best = q[l];
              bi = 4 * j + l;
            }
          }
        }
      }
    } else {
      for (long long j = s + threadIdx.x; j < e; j += ARG_THREADS) {
        const float x = fr[j];
        bad |= !(fabsf(x) <= 3.402823466e38f);
        if (x > best || bi < 0) {
          best = x;
          bi = j;
        }
      }
    }
    unsigned long long key = bi >= 0 ? pack(best, (uint32_t)bi) : 0ull;
    key = warp_max_u64(key);
    const int wbad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
      part[threadIdx.x >> 5] = key;
      part_bad[threadIdx.x >> 5] = wbad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long k = 0;
      int b = 0;
      for (int w = 0; w < ARG_THREADS / 32; w++) {
        k = part[w] > k ? part[w] : k;
        b |= part_bad[w];
      }
      if (b) {
        atomicMax(&keys[f], KEY_NONFINITE);
        atomicOr(status, STATUS_NONFINITE);
      } else {
        atomicMax(&keys[f], k);
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ float warp_sum32(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ float warp_min(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// Moffat profile (Sect. 3.1) with parameters p = (I0, x0, y0, alpha, beta,
// Bg): the quotients that do not depend on the pixel, once per parameter set.
struct MoffatConst {
  double x0, y0, beta, bg, ia2, A, c0, c1, c3, c4, c5;
};

__device__ __forceinline__ MoffatConst moffat_const(const double *p) {
  constexpr double INV_PI = 0.318309886183790671537767526745;   // 1 / pi
  MoffatConst k;
  const double I0 = p[0], al = p[3], be = p[4];
  const double ia = 1.0 / al;                  // the one division of a parameter set
  k.x0 = p[1];
  k.y0 = p[2];
  k.beta = be;
  k.bg = p[5];
  k.ia2 = ia * ia;
  k.c0 = (be - 1.0) * k.ia2 * INV_PI;          // dI/dI0 = c0 P
  k.A = I0 * k.c0;                             // I0 (beta - 1) / (pi alpha^2)
  k.c1 = 2.0 * k.A * be * k.ia2;               // dI/dx0 = c1 P / u dx
  k.c3 = -2.0 * k.A * ia;                      // dI/dalpha = c3 P + c4 rho^2 P / u
  k.c4 = k.c1 * ia;
  k.c5 = I0 * k.ia2 * INV_PI;                  // dI/dbeta = c5 P - A ln(u) P
  return k;
}

// Damped 6 x 6 solve by Cholesky; false when the matrix is not positive
// definite.  The six pivots' reciprocals are taken once, so the
// factorisation and both substitutions run on multiplications (FP64
// divisions are long instruction sequences on this GPU).
__device__ bool chol6(const double *A, const double *b, double *x) {
  double L[21], inv[6];   // lower triangle, row i at i (i + 1) / 2; 1 / L[i][i]
#pragma unroll
  for (int i = 0; i < 6; i++)
#pragma unroll
    for (int j = 0; j <= i; j++) {
      double s = A[i * 6 + j];
#pragma unroll
      for (int k = 0; k < j; k++) s -= L[i * (i + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
      if (i == j) {
        if (!(s > 0)) return false;
        const double d = sqrt(s);
        L[i * (i + 1) / 2 + i] = d;
        inv[i] = 1.0 / d;
      } else {
        L[i * (i + 1) / 2 + j] = s * inv[j];
      }
    }
  double y[6];
#pragma unroll
  for (int i = 0; i < 6; i++) {
    double s = b[i];
#pragma unroll
    for (int k = 0; k < i; k++) s -= L[i * (i + 1) / 2 + k] * y[k];
    y[i] = s * inv[i];
  }
#pragma unroll
  for (int i = 5; i >= 0; i--) {
    double s = y[i];
#pragma unroll
    for (int k = i + 1; k < 6; k++) s -= L[k * (k + 1) / 2 + i] * x[k];
    x[i] = s * inv[i];
  }
  return true;
}

// One pass over the window at the parameters k: the squared error of the
// model and the normal equations of its analytic Jacobian (J^T J lower
// triangle in ne[0..21), J^T r in ne[21..27)), lane partials then warp sums
// (every lane ends with the same values).  The oracle takes the two in
// separate passes; one pass serves both here because the normal equations
// of an accepted trial point are those of the next iteration.
__device__ __forceinline__ double window_pass(const MoffatConst &k, const float *win, int WH, int WW, int wr0,
                                              int wc0, int lane, double *ne) {
  double cost = 0.0;
#pragma unroll
  for (int q = 0; q < 27; q++) ne[q] = 0.0;
  for (int i = lane; i < WH * WW; i += 32) {
    const int r = i / WW, c = i - r * WW;
    const double dx = (double)(c + wc0) - k.x0, dy = (double)(r + wr0) - k.y0;
    const double rho2 = dx * dx + dy * dy;
    const double u = 1.0 + rho2 * k.ia2;
    const double lu = log(u);
    const double P = exp(-k.beta * lu);
    // 1 / u: the FP32 reciprocal refined by two Newton steps r <- r (2 - u r)
    // (relative error 1e-7 -> 1e-14 -> below FP64 rounding; u >= 1)
    double ru = (double)__frcp_rn((float)u);
    ru = ru * (2.0 - u * ru);
    ru = ru * (2.0 - u * ru);
    const double Pu = P * ru;
    const double e = k.A * P + k.bg - (double)win[i];
    double g[6];
    g[0] = k.c0 * P;
    g[1] = k.c1 * Pu * dx;
    g[2] = k.c1 * Pu * dy;
    g[3] = k.c3 * P + k.c4 * rho2 * Pu;
    g[4] = k.c5 * P - k.A * lu * P;
    g[5] = 1.0;
    cost += e * e;
    int q = 0;
#pragma unroll
    for (int ii = 0; ii < 6; ii++)
#pragma unroll
      for (int jj = 0; jj <= ii; jj++) ne[q++] += g[ii] * g[jj];
#pragma unroll
    for (int ii = 0; ii < 6; ii++) ne[21 + ii] += g[ii] * e;
  }
#pragma unroll
  for (int q = 0; q < 27; q++) ne[q] = warp_sum(ne[q]);
  return warp_sum(cost);
}

// The damped step of the FP32 phase: the normal equations scaled by D =
// diag(J^T J)^(-1/2) (unit diagonal, so the damping lambda diag(J^T J)
// becomes lambda I), factorised and solved in FP32, the step scaled back.
// False when the scaled matrix is not positive definite.
__device__ bool step32(const double *ne, double lambda, double *d) {
  float dinv[6], L[21], inv[6], y[6];
#pragma unroll
  for (int i = 0; i < 6; i++) {
    const double a = ne[i * (i + 1) / 2 + i];
    dinv[i] = a > 0 ? rsqrtf((float)a) : 1.0f;
  }
#pragma unroll
  for (int i = 0; i < 6; i++)
#pragma unroll
    for (int j = 0; j <= i; j++) {
      float s = (float)ne[i * (i + 1) / 2 + j] * dinv[i] * dinv[j];
      if (i == j) {
        const double a = ne[i * (i + 1) / 2 + i];
        s += (float)(lambda * (a > 0 ? 1.0 : 1e-12));
      }
#pragma unroll
      for (int k = 0; k < j; k++) s -= L[i * (i + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
      if (i == j) {
        if (!(s > 0.0f)) return false;
        const float dd = sqrtf(s);
        L[i * (i + 1) / 2 + i] = dd;
        inv[i] = 1.0f / dd;
      } else {
        L[i * (i + 1) / 2 + j] = s * inv[j];
      }
    }
#pragma unroll
  for (int i = 0; i < 6; i++) {
    float s = -(float)ne[21 + i] * dinv[i];
#pragma unroll
    for (int k = 0; k < i; k++) s -= L[i * (i + 1) / 2 + k] * y[k];
    y[i] = s * inv[i];
  }
  float x[6];
#pragma unroll
  for (int i = 5; i >= 0; i--) {
    float s = y[i];
#pragma unroll
    for (int k = i + 1; k < 6; k++) s -= L[k * (k + 1) / 2 + i] * x[k];
    x[i] = s * inv[i];
  }
#pragma unroll
  for (int i = 0; i < 6; i++) d[i] = (double)(x[i] * dinv[i]);
  return true;
}

// The same quotients in FP32, for the first (FP32) phase of the fit.
struct MoffatConst32 {
  float x0, y0, beta, bg, ia2, A, c0, c1, c3, c4, c5;
};

__device__ __forceinline__ MoffatConst32 moffat_const32(const double *p) {
  const MoffatConst k = moffat_const(p);
  MoffatConst32 f;
  f.x0 = (float)k.x0;
  f.y0 = (float)k.y0;
  f.beta = (float)k.beta;
  f.bg = (float)k.bg;
  f.ia2 = (float)k.ia2;
  f.A = (float)k.A;
  f.c0 = (float)k.c0;
  f.c1 = (float)k.c1;
  f.c3 = (float)k.c3;
  f.c4 = (float)k.c4;
  f.c5 = (float)k.c5;
  return f;
}

// window_pass with the per-pixel model, derivatives, lane partials and warp
// sums in FP32: on GB300 the FP32 pipe is 64 times the FP64 one, and the
// first iterations only need to come close.
__device__ __forceinline__ double window_pass32(const MoffatConst32 &k, const float *win, int WH, int WW, int wr0,
                                                int wc0, int lane, double *ne) {
  float cost = 0.0f, a[27];
#pragma unroll
  for (int q = 0; q < 27; q++) a[q] = 0.0f;
  for (int i = lane; i < WH * WW; i += 32) {
    const int r = i / WW, c = i - r * WW;
    const float dx = (float)(c + wc0) - k.x0, dy = (float)(r + wr0) - k.y0;
    const float rho2 = dx * dx + dy * dy;
    const float u = 1.0f + rho2 * k.ia2;
    const float l2 = log2f(u);
    const float P = exp2f(-k.beta * l2);
    const float Pu = P / u;
    const float e = k.A * P + k.bg - win[i];
    float g[6];
    g[0] = k.c0 * P;
    g[1] = k.c1 * Pu * dx;
    g[2] = k.c1 * Pu * dy;
    g[3] = k.c3 * P + k.c4 * rho2 * Pu;
    g[4] = k.c5 * P - k.A * (l2 * 0.69314718056f) * P;
    g[5] = 1.0f;
    cost += e * e;
    int q = 0;
#pragma unroll
    for (int ii = 0; ii < 6; ii++)
#pragma unroll
      for (int jj = 0; jj <= ii; jj++) a[q++] += g[ii] * g[jj];
#pragma unroll
    for (int ii = 0; ii < 6; ii++) a[21 + ii] += g[ii] * e;
  }
  // FP32 butterflies (each lane ends with the same bits), widened at the end
#pragma unroll
  for (int q = 0; q < 27; q++) ne[q] = (double)warp_sum32(a[q]);
  return (double)warp_sum32(cost);
}

// Levenberg-Marquardt iterations from p (the oracle's steps: damping lambda
// x diag(J^T J) from 1e-3, /10 (floor lam_floor) on an accepted step, x10 on
// a rejected one or one leaving alpha <= 0 or beta <= 1, at most 10 tries;
// stop when an accepted step lowers the squared error by at most stop_rel
// of it, when no try lowers it, or after 200 iterations).  F32 selects the
// FP32 evaluation.  Returns the iterations made; p and cost are updated.
template <bool F32>
__device__ __forceinline__ int lm_loop(double (&p)[6], double &cost, double *ne_cur, double lam_floor,
                                       double stop_rel, const float *buf, int WH, int WW, int wr0, int wc0,
                                       int lane) {
  double ne[27];
  cost = F32 ? window_pass32(moffat_const32(p), buf, WH, WW, wr0, wc0, lane, ne)
             : window_pass(moffat_const(p), buf, WH, WW, wr0, wc0, lane, ne);
  // ne_cur: the normal equations at p (identical in every lane: lane q keeps q)
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 27; q++)
    if (lane == q) ne_cur[q] = ne[q];
  __syncwarp();
  double lambda = 1e-3;
  int it;
  for (it = 0; it < 200; it++) {
    bool accepted = false;
    double newcost = cost;
    for (int tries = 0; tries < 10; tries++) {
      double d[6], q[6];
      bool ok;
      if constexpr (F32) {
        ok = step32(ne_cur, lambda, d);
      } else {
        double A[36], mg[6];
        int k = 0;
#pragma unroll
        for (int ii = 0; ii < 6; ii++)
#pragma unroll
          for (int jj = 0; jj <= ii; jj++) {
            A[ii * 6 + jj] = ne_cur[k];
            A[jj * 6 + ii] = ne_cur[k];
            k++;
          }
#pragma unroll
        for (int ii = 0; ii < 6; ii++) {
          const double di = A[ii * 6 + ii] > 0 ? A[ii * 6 + ii] : 1e-12;
          A[ii * 6 + ii] += lambda * di;
          mg[ii] = -ne_cur[21 + ii];
        }
        ok = chol6(A, mg, d);
      }
      if (!ok) {
        lambda *= 10.0;
        continue;
      }
#pragma unroll
      for (int ii = 0; ii < 6; ii++) q[ii] = p[ii] + d[ii];
      if (!(q[3] > 0) || !(q[4] > 1.0)) {
        lambda *= 10.0;
        continue;
      }
      newcost = F32 ? window_pass32(moffat_const32(q), buf, WH, WW, wr0, wc0, lane, ne)
                    : window_pass(moffat_const(q), buf, WH, WW, wr0, wc0, lane, ne);
      if (newcost < cost) {
#pragma unroll
        for (int ii = 0; ii < 6; ii++) p[ii] = q[ii];
        __syncwarp();   // every lane has read ne_cur
#pragma unroll
        for (int qq = 0; qq < 27; qq++)
          if (lane == qq) ne_cur[qq] = ne[qq];
        __syncwarp();
        lambda = fmax(lambda / 10.0, lam_floor);
        accepted = true;
        break;
      }
      lambda *= 10.0;
    }
    if (!accepted) break;
    const double drop = cost - newcost;
    cost = newcost;
    if (drop <= stop_rel * cost) {
      it++;
      break;
    }
  }
  return it;
}

// One frame on one warp: seed from the argmax word, patch, centroid, fit.
__device__ __forceinline__ void fit_frame(const RegArgs &a, unsigned long long key, long long f, float *buf,
                                          uint8_t *lab, double *ne_cur, int lane) {
  const int n = a.n;
  const float *fr = a.in + f * (long long)n * n;
  double *out = a.out + f * 8;
  auto not_found = [&]() {
    if (lane < 8) out[lane] = 0.0;
    if (lane == 0 && a.iters) a.iters[f] = 0;
  };
  if (key == KEY_NONFINITE) {
    not_found();
    return;
  }
  const long long seed = (long long)(~(uint32_t)(key & 0xffffffffull));
  if (key == 0ull || seed >= (long long)n * n) {   // no maximum recorded: cannot happen for n >= 1
    if (lane == 0) atomicOr(a.status, STATUS_INTERNAL);
    not_found();
    return;
  }
  const int r0 = (int)(seed / n), c0 = (int)(seed - (long long)r0 * n), R = a.R;
  const int rlo = max(r0 - R, 0), rhi = min(r0 + R, n - 1), clo = max(c0 - R, 0), chi = min(c0 + R, n - 1);
  const int H = rhi - rlo + 1, W = chi - clo + 1;
  const double th = a.thresh;

  // ---- patch: flood fill of the pixels above the threshold ----------------
  // lab: 0 below the threshold, 2 above and not (yet) reached, 1 in the patch
  __syncwarp();   // the previous frame's reads of buf and lab are done
  for (int i = lane; i < H * W; i += 32) {
    const int r = i / W, c = i - r * W;
    const float v = fr[(long long)(r + rlo) * n + (c + clo)];
    buf[i] = v;
    lab[i] = (double)v > th ? 2 : 0;
  }
  __syncwarp();
  const int si = (r0 - rlo) * W + (c0 - clo);
  if (lab[si] == 0) {   // the seed itself is not above the threshold
    not_found();
    return;
  }
  __syncwarp();
  if (lane == 0) lab[si] = 1;
  __syncwarp();
  for (int sweep = 0; sweep <= H * W; sweep++) {
    bool changed = false;
    for (int i = lane; i < H * W; i += 32) {
      if (lab[i] != 2) continue;
      const int r = i / W, c = i - r * W;
      bool nb = false;
      for (int dr = -1; dr <= 1; dr++)
        for (int dc = -1; dc <= 1; dc++) {
          const int rr = r + dr, cc = c + dc;
          if ((dr || dc) && rr >= 0 && rr < H && cc >= 0 && cc < W && lab[rr * W + cc] == 1) nb = true;
        }
      if (nb) {
        lab[i] = 1;
        changed = true;
      }
    }
    __syncwarp();
    if (!__any_sync(0xffffffffu, changed)) break;
  }
  double cnt = 0.0, sv = 0.0, sx = 0.0, sy = 0.0;
  bool touch = false;
  for (int i = lane; i < H * W; i += 32) {
    if (lab[i] != 1) continue;
    const int r = i / W, c = i - r * W;
    const double v = buf[i];
    cnt += 1.0;
    sv += v;
    sx += v * (double)(c + clo);
    sy += v * (double)(r + rlo);
    touch |= (r == 0 && rlo > 0) || (r == H - 1 && rhi < n - 1) || (c == 0 && clo > 0) || (c == W - 1 && chi < n - 1);
  }
  cnt = warp_sum(cnt);
  sv = warp_sum(sv);
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  const int size = (int)cnt;
  if (__any_sync(0xffffffffu, touch) || size < a.min_size || size > a.max_size) {
    not_found();
    return;
  }
  const double cx = sx / sv, cy = sy / sv;

  // ---- Moffat fit ---------------------------------------------------------
  const int rc = (int)floor(cy + 0.5), cc = (int)floor(cx + 0.5), w = a.w;
  const int wr0 = max(rc - w, 0), wr1 = min(rc + w, n - 1), wc0 = max(cc - w, 0), wc1 = min(cc + w, n - 1);
  const int WH = wr1 - wr0 + 1, WW = wc1 - wc0 + 1;
  __syncwarp();   // the box reads are done: the buffer now takes the window
  float lmin = INFINITY;
  for (int i = lane; i < WH * WW; i += 32) {
    const int r = i / WW, c = i - r * WW;
    const float v = fr[(long long)(r + wr0) * n + (c + wc0)];
    buf[i] = v;
    lmin = fminf(lmin, v);
  }
  __syncwarp();
  const double bg = warp_min(lmin);
  double i0 = 0.0;
  for (int i = lane; i < WH * WW; i += 32) i0 += (double)buf[i] - bg;
  i0 = warp_sum(i0);
  double p[6] = {i0, cx, cy, fmax(1.0, sqrt((double)size / REG_PI)), 2.5, bg};
  double cost;
  // Phase A: FP32 evaluation until the FP32 cost stops improving (its
  // rounding is about 1e-7 of it; a lambda floor of 1e-6 keeps the damped
  // system well away from the FP32 noise of J^T J).  Phase B: the FP64
  // iteration of the oracle from there, which converges in a few steps to
  // the same minimum.
  const int it_a = lm_loop<true>(p, cost, ne_cur, 1e-6, 1e-7, buf, WH, WW, wr0, wc0, lane);
  const int it_b = lm_loop<false>(p, cost, ne_cur, 1e-12, 1e-14, buf, WH, WW, wr0, wc0, lane);
  const int it = it_a + it_b;
  if (lane == 0) {
    out[0] = 1.0;
    out[1] = p[1];
    out[2] = p[2];
    out[3] = 2.0 * p[3] * sqrt(pow(2.0, 1.0 / p[4]) - 1.0);
    out[4] = p[0];
    out[5] = p[3];
    out[6] = p[4];
    out[7] = p[5];
    if (a.iters) a.iters[f] = it;
  }
}

// Persistent warps: each takes the next frame from the counter after the
// per-frame words (no waiting on other warps).
__global__ void __launch_bounds__(FIT_WARPS * 32) register_fit_kernel(const RegArgs a,
                                                                      unsigned long long *__restrict__ keys,
                                                                      int side) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int S2 = side * side;
  const size_t per_warp = (((size_t)S2 * 5 + 15) & ~(size_t)15) + 27 * sizeof(double);
  unsigned char *base = smem + (size_t)wid * per_warp;
  float *buf = reinterpret_cast<float *>(base);
  uint8_t *lab = reinterpret_cast<uint8_t *>(buf + S2);
  double *ne_cur = reinterpret_cast<double *>(base + (((size_t)S2 * 5 + 15) & ~(size_t)15));
  unsigned long long *counter = keys + a.T;
  for (;;) {
    long long f = 0;
    if (lane == 0) f = (long long)atomicAdd(counter, 1ull);
    f = __shfl_sync(0xffffffffu, f, 0);
    if (f >= a.T) break;
    fit_frame(a, keys[f], f, buf, lab, ne_cur, lane);
  }
}

}  // namespace

size_t register_keys_bytes(long long T) { return (size_t)(T + 1) * sizeof(unsigned long long); }

cudaError_t launch_register_argmax(const RegArgs &a, unsigned long long *keys, cudaStream_t st) {
  if (a.T <= 0) return cudaSuccess;
  const long long nn = (long long)a.n * a.n;
  cudaError_t e = cudaMemsetAsync(keys, 0, register_keys_bytes(a.T), st);
  if (e != cudaSuccess) return e;
  const long long chunks = (nn + REG_CHUNK - 1) / REG_CHUNK;
  const long long items = a.T * chunks;
  const unsigned grid = (unsigned)(items < 152LL * 64 ? items : 152LL * 64);
  frame_argmax_kernel<<<grid, ARG_THREADS, 0, st>>>(a.in, a.T, nn, chunks, keys, a.status);
  return cudaGetLastError();
}

cudaError_t launch_register_fit(const RegArgs &a, unsigned long long *keys, cudaStream_t st) {
  if (a.T <= 0) return cudaSuccess;
  const int side = 2 * (a.R > a.w ? a.R : a.w) + 1;
  const size_t per_warp = (((size_t)side * side * 5 + 15) & ~(size_t)15) + 27 * sizeof(double);
  const size_t smem = per_warp * FIT_WARPS;
  cudaError_t e = cudaFuncSetAttribute(register_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, register_fit_kernel, FIT_WARPS * 32, smem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const long long need = (a.T + FIT_WARPS - 1) / FIT_WARPS;
  long long grid = (long long)(per_sm > 0 ? per_sm : 1) * sms;
  if (grid > need) grid = need;
  register_fit_kernel<<<(unsigned)grid, FIT_WARPS * 32, smem, st>>>(a, keys, side);
  return cudaGetLastError();
}

}  // namespace graphic

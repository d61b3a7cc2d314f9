// geom.cu -- Fourier line passes of the shift (Sect. 3.3.1) and of the
// three-shear rotation (Sect. 3.4) on sm_103a.
//
// Every pass applies, to each line of a frame, the periodic Fourier shift
//   v = IFFT_m( H(d) . FFT_m( u ) ),  H_k = exp(-i 2 pi k d / m) on signed
//   bins k, H_{m/2} = cos(pi d) (a Hermitian filter, so real lines stay real)
// where m = 2n is the zero-padded line length.  The padded line is handled
// in "rolled" coordinates (padded index + n/2 mod m), so the frame data sit
// in [0, n), the zero padding in [n, m) and the crop window of the output
// is again [0, n): rolling commutes with a circular filter.
//
// Data path of one CTA (256 threads): it owns LPC = 4096/m line PAIRS, each
// pair packed as one complex line z = a + i b (two real lines), handled by
// m/16 threads holding 16 complex values in registers.  Forward FFT =
// Stockham autosort stages of radix 16, 16 and m/256 (or 16, 8 for m = 128):
// the first stage reads global memory straight into registers (input half
// zero: pruned at compile time), later stages exchange through shared
// memory (ping-pong buffers, one pad slot every 16 entries against bank
// conflicts).  The middle step separates the two real spectra where the two
// lines have different shifts (shear passes), multiplies by the phasors and
// stores conj(V)/m; the inverse is then the same forward stages
// (IFFT(V) = conj(FFT(conj V)) / m), the last stage writing the cropped
// output straight to global memory.
//
// Phase arguments: d is formed in FP64 per line, reduced to delta = d/m =
// delta_hi + delta_lo with delta_hi on a 2^-12 grid (so k * delta_hi is exact
// in FP32 for k < 2^11) and the turns frac(k delta) evaluated as
// (k delta_hi - rint(k delta_hi)) + k delta_lo before sincospif.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "graphic_internal.h"
#include "line_common.cuh"

namespace graphic {
namespace {

// Twiddle tables W_m^e = exp(-i 2 pi e / m), e in [0, m), for m = 128..2048,
// stored back to back at offset m - 128 (FP64 cos/sin rounded to FP32).
constexpr int kTwTotal = 4096 - 128;
__device__ float2 d_twiddle[kTwTotal];
// The twiddles of the radix-32 x 32 warp FFT (m = 1024), W_1024^(r lane) at
// [r][lane] (the same values as d_twiddle): lane-contiguous, so each of the
// 31 twiddle loads of a lane group is one coalesced 256-byte access.
__device__ float2 d_tw1024_rl[32 * 32];

__host__ __device__ constexpr int tw_off(int m) { return m - 128; }

// complex helpers, line parameters and frame loads: line_common.cuh

// exp(-i 2 pi j / 16) as (cos, sin) of 2 pi j / 16: the constants are
// cos(pi/8), sin(pi/8) and sqrt(1/2).
#define G_C16 0.92387953251128675613f
#define G_S16 0.38268343236508977173f
#define G_R2 0.70710678118654752440f

template <int J>
__device__ __forceinline__ float2 mul_w16(float2 a) {
  constexpr int j = J & 15;
  if constexpr (j == 0) return a;
  else if constexpr (j == 4) return make_float2(a.y, -a.x);
  else if constexpr (j == 8) return make_float2(-a.x, -a.y);
  else if constexpr (j == 12) return make_float2(-a.y, a.x);
  else {
    constexpr float cs[16] = {1.f, G_C16, G_R2, G_S16, 0.f, -G_S16, -G_R2, -G_C16,
                              -1.f, -G_C16, -G_R2, -G_S16, 0.f, G_S16, G_R2, G_C16};
    constexpr float sn[16] = {0.f, G_S16, G_R2, G_C16, 1.f, G_C16, G_R2, G_S16,
                              0.f, -G_S16, -G_R2, -G_C16, -1.f, -G_C16, -G_R2, -G_S16};
    constexpr float c = cs[j], s = sn[j];
    // (a.x + i a.y)(c - i s)
    return make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
  }
}

__device__ __forceinline__ void dft2(float2 &a, float2 &b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
  float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = csub(a1, a3);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = make_float2(t1.x + t3.y, t1.y - t3.x);  // t1 - i t3
  a3 = make_float2(t1.x - t3.y, t1.y + t3.x);  // t1 + i t3
}

// In-place forward DFT of size R on a[0..R), natural order out.
// R = R1 * R2 with n = R2 n1 + n2, k = k1 + R1 k2: inner DFT_R1 over n1,
// twiddle W_R^(n2 k1), outer DFT_R2 over n2, then the index transpose.
template <int R>
__device__ __forceinline__ void dft(float2 (&a)[R]);

template <>
__device__ __forceinline__ void dft<2>(float2 (&a)[2]) { dft2(a[0], a[1]); }

template <>
__device__ __forceinline__ void dft<4>(float2 (&a)[4]) { dft4(a[0], a[1], a[2], a[3]); }

template <>
__device__ __forceinline__ void dft<8>(float2 (&a)[8]) {
  dft4(a[0], a[2], a[4], a[6]);
  dft4(a[1], a[3], a[5], a[7]);
  a[3] = mul_w16<2>(a[3]);   // n2 = 1, k1 = 1: W8^1
  a[5] = mul_w16<4>(a[5]);   // k1 = 2
  a[7] = mul_w16<6>(a[7]);   // k1 = 3
  dft2(a[0], a[1]);
  dft2(a[2], a[3]);
  dft2(a[4], a[5]);
  dft2(a[6], a[7]);
  // slot 2 k1 + k2 holds X[k1 + 4 k2]
  float2 t[8];
#pragma unroll
  for (int i = 0; i < 8; i++) t[i] = a[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; k1++)
#pragma unroll
    for (int k2 = 0; k2 < 2; k2++) a[k1 + 4 * k2] = t[2 * k1 + k2];
}

template <>
__device__ __forceinline__ void dft<16>(float2 (&a)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; n2++) dft4(a[n2], a[n2 + 4], a[n2 + 8], a[n2 + 12]);
  // slot 4 k1 + n2 *= W16^(n2 k1)
  a[5] = mul_w16<1>(a[5]);
  a[6] = mul_w16<2>(a[6]);
  a[7] = mul_w16<3>(a[7]);
  a[9] = mul_w16<2>(a[9]);
  a[10] = mul_w16<4>(a[10]);
  a[11] = mul_w16<6>(a[11]);
  a[13] = mul_w16<3>(a[13]);
  a[14] = mul_w16<6>(a[14]);
  a[15] = mul_w16<9>(a[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; k1++) dft4(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
  float2 t[16];
#pragma unroll
  for (int i = 0; i < 16; i++) t[i] = a[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; k1++)
#pragma unroll
    for (int k2 = 0; k2 < 4; k2++) a[k1 + 4 * k2] = t[4 * k1 + k2];
}

__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }

// Radix of Stockham stage s (0-based) for line length M.
template <int M, int S>
struct Radix {
  static constexpr int value = (S == 0) ? 16 : (S == 1 ? (M == 128 ? 8 : 16) : M / 256);
};
template <int M>
struct NumStages {
  static constexpr int value = (M <= 256) ? 2 : 3;
};

// One Stockham stage in registers: v[m] holds element j + m M/16 of the
// stage input; after the call, v[u + U r] holds output r of virtual thread
// vt = j + u M/16, to be stored at position (vt / NS) NS R + (vt % NS) + r NS.
template <int M, int R, int NS>
__device__ __forceinline__ void stage_compute(float2 (&v)[16], int j, const float2 *__restrict__ tw) {
  constexpr int U = 16 / R;
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int vt = j + u * (M / 16);
    float2 a[R];
#pragma unroll
    for (int r = 0; r < R; r++) a[r] = v[u + U * r];
    if constexpr (NS > 1) {
      const int k = vt & (NS - 1);
#pragma unroll
      for (int r = 1; r < R; r++) a[r] = cmul(a[r], __ldg(&tw[r * k * (M / (NS * R))]));
    }
    dft<R>(a);
#pragma unroll
    for (int r = 0; r < R; r++) v[u + U * r] = a[r];
  }
}

template <int M, int R, int NS>
__device__ __forceinline__ void stage_store_smem(const float2 (&v)[16], int j, float2 *dst) {
  constexpr int U = 16 / R;
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int vt = j + u * (M / 16);
    const int base = (vt / NS) * NS * R + (vt & (NS - 1));
#pragma unroll
    for (int r = 0; r < R; r++) dst[padi(base + r * NS)] = v[u + U * r];
  }
}

template <int M>
__device__ __forceinline__ void load_smem(float2 (&v)[16], int j, const float2 *src) {
#pragma unroll
  for (int m = 0; m < 16; m++) v[m] = src[padi(j + m * (M / 16))];
}

// Barrier among the M/16 threads of one line pair: a named barrier (id 1 + p)
// when the pair spans several warps, otherwise the warp's own barrier.
template <int M>
__device__ __forceinline__ void pair_sync(int p) {
  constexpr int TPL = M / 16;
  if constexpr (TPL > 32) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(1 + p), "r"(TPL) : "memory");
  } else {
    __syncwarp();
  }
}

// Stages 1.. of a forward transform from smem buffer `a` (ping-pong with
// `b`); stage 0 has already been computed and stored into `a`.  Returns the
// buffer holding the natural-order result (all stages but the last), or,
// when LAST_TO_REGS, leaves the last stage's outputs in v.  Only the
// threads of line pair p take part.
template <int M, bool LAST_TO_REGS>
__device__ __forceinline__ float2 *run_stages(float2 (&v)[16], int j, int p, float2 *a, float2 *b,
                                              const float2 *__restrict__ tw) {
  constexpr int S = NumStages<M>::value;
  // stage 1
  pair_sync<M>(p);
  load_smem<M>(v, j, a);
  stage_compute<M, Radix<M, 1>::value, 16>(v, j, tw);
  if constexpr (S == 2) {
    if constexpr (!LAST_TO_REGS) {
      stage_store_smem<M, Radix<M, 1>::value, 16>(v, j, b);
      return b;
    }
    return nullptr;
  } else {
    stage_store_smem<M, Radix<M, 1>::value, 16>(v, j, b);
    pair_sync<M>(p);
    load_smem<M>(v, j, b);
    stage_compute<M, Radix<M, 2>::value, 256>(v, j, tw);
    if constexpr (!LAST_TO_REGS) {
      stage_store_smem<M, Radix<M, 2>::value, 256>(v, j, a);
      return a;
    }
    return nullptr;
  }
}

// Output position of register slot (u, r) after the last stage: vt + r M/R.
template <int M>
struct LastStage {
  static constexpr int R = Radix<M, NumStages<M>::value - 1>::value;
  static constexpr int U = 16 / R;
};


template <int M, int KIND, bool CG = false>
__device__ __forceinline__ void line_pass_body(const LineArgs &a, long long f, int cx, float2 *smem, LineParam *lp,
                                               int *ident_p) {
  constexpr int N = M / 2;
  constexpr int TPL = M / 16;          // threads per line pair
  constexpr int LPC = 4096 / M;        // line pairs per CTA
  constexpr int LBUF = M + M / 16;     // padded line buffer, complex entries
  constexpr bool SAME_D = (KIND == SHIFT_X || KIND == SHIFT_Y);
  constexpr int NIN = (KIND == ROT_P3) ? M : N;        // input samples per line
  constexpr int NOUT = (KIND == ROT_P1) ? M : N;       // output samples per line
  constexpr int NLINES = (KIND == ROT_P2) ? M : N;     // lines per frame

  int &ident_s = *ident_p;
  const int tid = threadIdx.x;
  const int p = tid / TPL;
  const int j = tid % TPL;
  const int line0 = 2 * (cx * LPC + p);
  const float *__restrict__ fin = a.in_tab ? a.in_tab[f] : a.in + f * a.in_fstride;
  float *__restrict__ fout = a.out_tab ? a.out_tab[f] : a.out + f * a.out_fstride;
  const float2 *__restrict__ tw = d_twiddle + tw_off(M);
  float2 *bufA = smem + p * LBUF;
  float2 *bufB = smem + (LPC + p) * LBUF;
  const int q = (KIND == ROT_P1) ? (a.q[f] & 3) : 0;

  if (tid == 0) {
    bool id;
    if constexpr (KIND == SHIFT_X) id = (a.p0[f] == 0.0);
    else if constexpr (KIND == SHIFT_Y) id = (a.p1[f] == 0.0);
    else id = (a.p0[f] == 0.0 && a.p1[f] == 0.0);
    ident_s = id ? 1 : 0;
  }
  if (tid < 2 * LPC && (!SAME_D || tid == 0)) {
    const int gl = 2 * cx * LPC + tid;
    if (a.lp_tab)
      lp[tid] = reinterpret_cast<const LineParam *>(a.lp_tab)[f * a.lp_lines + (SAME_D ? 0 : gl)];
    else
      make_param(lp[tid], line_shift<KIND>(a, f, gl, N), M);
  }
  __syncthreads();

  bool bad = false;
  if (ident_s) {
    // zero shift for every line of the frame: copy (exact identity)
    if constexpr (KIND == ROT_P2) return;
    for (int pos = j; pos < NOUT; pos += TPL) {
      float2 z = make_float2(0.f, 0.f);
      if (pos < NIN) {
        if constexpr (KIND == SHIFT_X || KIND == ROT_P3) {
          const int rs = (KIND == ROT_P3) ? M : N;
          z = make_float2(ldf<CG>(fin + (size_t)line0 * rs + pos), ldf<CG>(fin + (size_t)(line0 + 1) * rs + pos));
        } else if constexpr (KIND == SHIFT_Y) {
          z = ldf2<CG>(fin + (size_t)pos * N + line0);
        } else if constexpr (KIND == ROT_P1) {
          z = load_rot90_pair<CG>(fin, N, q, line0, pos);
        }
      }
      if constexpr (KIND == SHIFT_X || KIND == ROT_P1) bad |= !finite_pair(z);
      if constexpr (KIND == SHIFT_Y) {
        *reinterpret_cast<float2 *>(fout + (size_t)pos * N + line0) = z;
      } else {
        const int rs = (KIND == ROT_P1) ? M : N;
        fout[(size_t)line0 * rs + pos] = z.x;
        fout[(size_t)(line0 + 1) * rs + pos] = z.y;
      }
    }
    if (bad) atomicOr(a.status, STATUS_NONFINITE);
    return;
  }

  // ---- forward transform, stage 0 straight from global memory ----------
  float2 v[16];
  {
#pragma unroll
    for (int m = 0; m < 16; m++) {
      const int pos = j + m * (M / 16);
      float2 z = make_float2(0.f, 0.f);
      if (m * (M / 16) < NIN) {   // compile-time pruning of the zero half
        if constexpr (KIND == SHIFT_X) {
          z = make_float2(ldf<CG>(fin + (size_t)line0 * N + pos), ldf<CG>(fin + (size_t)(line0 + 1) * N + pos));
        } else if constexpr (KIND == SHIFT_Y) {
          z = ldf2<CG>(fin + (size_t)pos * N + line0);
        } else if constexpr (KIND == ROT_P1) {
          z = load_rot90_pair<CG>(fin, N, q, line0, pos);
        } else if constexpr (KIND == ROT_P2) {
          z = ldf2<CG>(fin + (size_t)pos * M + line0);
        } else {
          z = make_float2(ldf<CG>(fin + (size_t)line0 * M + pos), ldf<CG>(fin + (size_t)(line0 + 1) * M + pos));
        }
        if constexpr (KIND == SHIFT_X || KIND == ROT_P1) bad |= !finite_pair(z);
      }
      v[m] = z;
    }
    if constexpr (KIND == SHIFT_X || KIND == ROT_P1) {
      if (bad) atomicOr(a.status, STATUS_NONFINITE);
    }
  }
  stage_compute<M, 16, 1>(v, j, tw);
  stage_store_smem<M, 16, 1>(v, j, bufA);
  float2 *spec = run_stages<M, false>(v, j, p, bufA, bufB, tw);
  pair_sync<M>(p);

  // ---- middle: phasors (and separation of the two real spectra) ---------
  {
    const LineParam &la = lp[SAME_D ? 0 : 2 * p];
    const LineParam &lb = lp[SAME_D ? 0 : 2 * p + 1];
    const float inv_m = 1.0f / (float)M;
    // the 1/m of the inverse (and the 1/2 of the separation) are powers of
    // two, carried by the phasor base (the same bits as scaling each product)
    constexpr float sc = SAME_D ? 1.0f / (float)M : 0.5f / (float)M;
    const int K0 = 8 * j;
    const float2 pa0 = phase_at(la, K0);
    const float2 ba = make_float2(pa0.x * sc, pa0.y * sc);
    float2 bb = ba;
    if constexpr (!SAME_D) {
      const float2 pb0 = phase_at(lb, K0);
      bb = make_float2(pb0.x * sc, pb0.y * sc);
    }
#pragma unroll
    for (int r = 0; r < 8; r++) {
      const int k = K0 + r;
      if (k == 0) {
        float2 z = spec[0];
        spec[0] = make_float2(z.x * inv_m, -z.y * inv_m);
        continue;
      }
      const float2 ha = cmul(ba, la.step[r]);
      float2 z = spec[padi(k)], zm = spec[padi(M - k)];
      float2 vk, vm;
      if constexpr (SAME_D) {
        vk = cmul(z, ha);
        vm = cmul(zm, cconj(ha));
      } else {
        const float2 hb = cmul(bb, lb.step[r]);
        // 2A = Z_k + conj Z_{-k},  2B = (Z_k - conj Z_{-k}) / i
        const float2 A = make_float2(z.x + zm.x, z.y - zm.y);
        const float2 B = make_float2(z.y + zm.y, zm.x - z.x);
        const float2 P = cmul(A, ha), Q = cmul(B, hb);
        vk = make_float2(P.x - Q.y, P.y + Q.x);     // P + i Q
        vm = make_float2(P.x + Q.y, Q.x - P.y);     // conj P + i conj Q
      }
      spec[padi(k)] = make_float2(vk.x, -vk.y);
      spec[padi(M - k)] = make_float2(vm.x, -vm.y);
    }
    if (j == 0) {
      float2 z = spec[padi(M / 2)];
      spec[padi(M / 2)] = make_float2(z.x * la.cnyq * inv_m, -z.y * lb.cnyq * inv_m);
    }
  }
  pair_sync<M>(p);

  // ---- inverse via forward stages on conj(V)/m --------------------------
  float2 *other = (spec == bufA) ? bufB : bufA;
  load_smem<M>(v, j, spec);
  stage_compute<M, 16, 1>(v, j, tw);
  stage_store_smem<M, 16, 1>(v, j, other);
  run_stages<M, true>(v, j, p, other, spec, tw);

  // ---- store: slot (u, r) -> position vt + r M/R; y = conj(result) -------
  constexpr int RL = LastStage<M>::R;
  constexpr int UL = LastStage<M>::U;
  {
#pragma unroll
    for (int u = 0; u < UL; u++) {
#pragma unroll
      for (int r = 0; r < RL; r++) {
        const int pos = j + u * (M / 16) + r * (M / RL);
        if (r * (M / RL) < NOUT) {
          const float2 y = v[u + UL * r];
          if constexpr (KIND == SHIFT_Y) {
            *reinterpret_cast<float2 *>(fout + (size_t)pos * N + line0) = make_float2(y.x, -y.y);
          } else if constexpr (KIND == ROT_P2) {
            *reinterpret_cast<float2 *>(fout + (size_t)pos * M + line0) = make_float2(y.x, -y.y);
          } else {
            const int rs = (KIND == ROT_P1) ? M : N;
            fout[(size_t)line0 * rs + pos] = y.x;
            fout[(size_t)(line0 + 1) * rs + pos] = -y.y;
          }
        }
      }
    }
  }
  (void)NLINES;
}

// One CTA of a line pass: line pairs cx * LPC .. of frame blockIdx.y.
// Register budget: 3 resident CTAs per SM for lines of up to 256 points, 2
// for longer ones (measured: 3 is faster on the short lines, slower on the
// 2048-point ones).
template <int M, int KIND>
__global__ void __launch_bounds__(256, (M <= 256) ? 3 : 2) line_pass_kernel(const LineArgs a) {
  extern __shared__ float2 smem[];
  __shared__ LineParam lp[2 * (4096 / M)];
  __shared__ int ident_s;
  line_pass_body<M, KIND>(a, blockIdx.y, blockIdx.x, smem, lp, &ident_s);
}

// ---------------------------------------------------------------------------
// m = 1024: one warp per line pair, 32 complex values per thread.
// Forward FFT = two Stockham stages of radix 32 (one shared-memory exchange),
// the thread holding bins k = lane + 32 r afterwards; the pair separation
// reads the conjugate-partner bin through shared memory; the inverse reuses
// the same two stages on conj(V)/m.
// ---------------------------------------------------------------------------

// cos(2 pi m / 32) for m = 0..8 (the others follow by symmetry).
#define G_C32_0 1.0f
#define G_C32_1 0.98078528040323044913f
#define G_C32_2 0.92387953251128675613f
#define G_C32_3 0.83146961230254523708f
#define G_C32_4 0.70710678118654752440f
#define G_C32_5 0.55557023301960222474f
#define G_C32_6 0.38268343236508977173f
#define G_C32_7 0.19509032201612826785f
#define G_C32_8 0.0f

__host__ __device__ constexpr float c32_base(int m) {
  return m == 0 ? G_C32_0 : m == 1 ? G_C32_1 : m == 2 ? G_C32_2 : m == 3 ? G_C32_3 : m == 4 ? G_C32_4
       : m == 5 ? G_C32_5 : m == 6 ? G_C32_6 : m == 7 ? G_C32_7 : G_C32_8;
}
// cos and sin of 2 pi m / 32 for any m, from the first octant
__host__ __device__ constexpr float c32(int m) {
  return (m & 31) <= 8 ? c32_base(m & 31)
       : (m & 31) <= 16 ? -c32_base(16 - (m & 31))
       : (m & 31) <= 24 ? -c32_base((m & 31) - 16) : c32_base(32 - (m & 31));
}
__host__ __device__ constexpr float s32(int m) {
  return (m & 31) <= 8 ? c32_base(8 - (m & 31))
       : (m & 31) <= 16 ? c32_base((m & 31) - 8)
       : (m & 31) <= 24 ? -c32_base(24 - (m & 31)) : -c32_base((m & 31) - 24);
}

template <int J>
__device__ __forceinline__ float2 mul_w32(float2 a) {
  constexpr int j = J & 31;
  if constexpr (j == 0) return a;
  else if constexpr (j == 8) return make_float2(a.y, -a.x);
  else if constexpr (j == 16) return make_float2(-a.x, -a.y);
  else if constexpr (j == 24) return make_float2(-a.y, a.x);
  else {
    constexpr float c = c32(j), s = s32(j);
    return make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
  }
}

// In-place forward DFT of size 32, natural order out: n = 8 n1 + n2,
// k = k1 + 4 k2 (inner DFT4 over n1, twiddle W32^(n2 k1), outer DFT8 over n2).
template <int K1>
__device__ __forceinline__ void w32_row(float2 (&a)[32]) {
  a[8 * K1 + 1] = mul_w32<1 * K1>(a[8 * K1 + 1]);
  a[8 * K1 + 2] = mul_w32<2 * K1>(a[8 * K1 + 2]);
  a[8 * K1 + 3] = mul_w32<3 * K1>(a[8 * K1 + 3]);
  a[8 * K1 + 4] = mul_w32<4 * K1>(a[8 * K1 + 4]);
  a[8 * K1 + 5] = mul_w32<5 * K1>(a[8 * K1 + 5]);
  a[8 * K1 + 6] = mul_w32<6 * K1>(a[8 * K1 + 6]);
  a[8 * K1 + 7] = mul_w32<7 * K1>(a[8 * K1 + 7]);
}

// HALF: a[16..31] are zero (a line zero-padded to twice its length), so
// each inner DFT4 has two inputs.
template <bool HALF = false>
__device__ __forceinline__ void dft32(float2 (&a)[32]) {
#pragma unroll
  for (int n2 = 0; n2 < 8; n2++) {
    if constexpr (HALF) {
      const float2 x0 = a[n2], x1 = a[n2 + 8];
      a[n2] = cadd(x0, x1);
      a[n2 + 8] = make_float2(x0.x + x1.y, x0.y - x1.x);    // x0 - i x1
      a[n2 + 16] = csub(x0, x1);
      a[n2 + 24] = make_float2(x0.x - x1.y, x0.y + x1.x);   // x0 + i x1
    } else {
      dft4(a[n2], a[n2 + 8], a[n2 + 16], a[n2 + 24]);
    }
  }
  w32_row<1>(a);
  w32_row<2>(a);
  w32_row<3>(a);
  float2 t[32];
#pragma unroll
  for (int k1 = 0; k1 < 4; k1++) {
    float2 b[8];
#pragma unroll
    for (int n2 = 0; n2 < 8; n2++) b[n2] = a[8 * k1 + n2];
    dft<8>(b);
#pragma unroll
    for (int k2 = 0; k2 < 8; k2++) t[k1 + 4 * k2] = b[k2];
  }
#pragma unroll
  for (int i = 0; i < 32; i++) a[i] = t[i];
}

__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }

// Two radix-32 Stockham stages over the 1024-point line held as v[m] =
// element lane + 32 m: after the call v[r] = X[lane + 32 r].  buf: the warp's
// exchange buffer (1024 + 32 entries); tw: W_1024^(r lane) at [r][lane].
template <bool HALF = false>
__device__ __forceinline__ void fft1024_warp(float2 (&v)[32], int lane, float2 *buf,
                                             const float2 *__restrict__ tw) {
  dft32<HALF>(v);
#pragma unroll
  for (int r = 0; r < 32; r++) buf[pad32(32 * lane + r)] = v[r];
  __syncwarp();
#pragma unroll
  for (int m = 0; m < 32; m++) v[m] = buf[pad32(lane + 32 * m)];
#pragma unroll
  for (int r = 1; r < 32; r++) v[r] = cmul(v[r], __ldg(&tw[r * 32 + lane]));
  dft32(v);
  __syncwarp();
}

// The shift of one line pair held in registers (v[m] = element lane + 32 m,
// packed as line a + i line b): forward transform, spectrum separation and
// per-line phasors (Sect. 3.3.1 shift theorem; lines a and b shifted by
// their own amounts unless SAME_D), inverse transform.  On return v[r] is
// conj(y) at element lane + 32 r.  buf: the warp's exchange buffer.
template <int KIND>
__device__ __forceinline__ void w32_filter(float2 (&v)[32], int lane, float2 *buf, const float2 *__restrict__ tw,
                                           const LineParam &la, const LineParam &lb) {
  constexpr int M = 1024;
  constexpr bool SAME_D = (KIND == SHIFT_X || KIND == SHIFT_Y);
  fft1024_warp<KIND != ROT_P3>(v, lane, buf, tw);   // only rotation pass 3 reads whole 1024-point lines

  // ---- middle: v[r] = Z_k, k = lane + 32 r --------------------------------
  // the 1/m of the inverse and the 1/2 of the pair separation are powers of
  // two, carried by the phasors (the same bits as scaling each product)
  constexpr float sc = SAME_D ? 1.0f / (float)M : 0.5f / (float)M;
  const float2 sa = phase_at(la, 32);
  if constexpr (SAME_D) {
    // one shift for both lines: V_k = Z_k H_k, H_k = exp(-i 2 pi ks delta),
    // ks the signed bin: exact anchors at r = 0, 8, 16, 24, a product with
    // exp(-i 2 pi 32 delta) in between
    float2 ha;
#pragma unroll
    for (int r = 0; r < 32; r++) {
      const int k = lane + 32 * r;
      if ((r & 7) == 0) {
        const float2 pa = phase_at(la, (r < 16) ? k : k - M);
        ha = make_float2(pa.x * sc, pa.y * sc);
      } else {
        ha = cmul(ha, sa);
      }
      const float2 ua = (r == 16 && lane == 0) ? make_float2(la.cnyq * sc, 0.f) : ha;   // Nyquist bin
      const float2 vk = cmul(v[r], ua);
      v[r] = make_float2(vk.x, -vk.y);   // conj(V) / m
    }
  } else {
    // lines a and b shifted by their own amounts.  Bins k and M - k share the
    // separated spectra (A_{M-k} = conj A_k, B_{M-k} = conj B_k) and the
    // phasors (H_{-k} = conj H_k), so each lane computes its bins k < M/2
    // (r < 16) and hands V_{M-k} to the lane that holds bin M - k; lane 0
    // computes its own bins 0 and M/2 (each its own partner).
#pragma unroll
    for (int r = 0; r < 32; r++) buf[pad32(lane + 32 * r)] = v[r];
    __syncwarp();
    const float2 sb = phase_at(lb, 32);
    float2 ha, hb;
#pragma unroll
    for (int r = 0; r < 16; r++) {
      const int k = lane + 32 * r;
      if ((r & 7) == 0) {
        const float2 pa = phase_at(la, k), pb = phase_at(lb, k);
        ha = make_float2(pa.x * sc, pa.y * sc);
        hb = make_float2(pb.x * sc, pb.y * sc);
      } else {
        ha = cmul(ha, sa);
        hb = cmul(hb, sb);
      }
      // twice the spectra of lines a and b; location M - k is read and
      // written by this lane only
      const int jm = pad32((M - k) & (M - 1));
      const float2 z = v[r], zm = buf[jm];
      const float2 A = make_float2(z.x + zm.x, z.y - zm.y);
      const float2 B = make_float2(z.y + zm.y, zm.x - z.x);
      const float2 P = cmul(A, ha), Q = cmul(B, hb);
      v[r] = make_float2(P.x - Q.y, -(P.y + Q.x));                 // conj(V_k) / m
      if (r > 0 || lane > 0) buf[jm] = make_float2(P.x + Q.y, P.y - Q.x);   // conj(V_{M-k}) / m
    }
    if (lane == 0) {   // Nyquist bin M/2: v[16] holds it, its own partner
      const float2 z = v[16];
      const float2 A = make_float2(z.x + z.x, z.y - z.y);
      const float2 B = make_float2(z.y + z.y, z.x - z.x);
      const float2 P = cmul(A, make_float2(la.cnyq * sc, 0.f)), Q = cmul(B, make_float2(lb.cnyq * sc, 0.f));
      v[16] = make_float2(P.x - Q.y, -(P.y + Q.x));
    }
    __syncwarp();
#pragma unroll
    for (int r = 16; r < 32; r++)
      if (r > 16 || lane > 0) v[r] = buf[pad32(lane + 32 * r)];
  }
  __syncwarp();

  // ---- inverse: the same stages on conj(V)/m; y = conj(result) ------------
  fft1024_warp(v, lane, buf, tw);
}

// Line pairs (warps) per CTA: 8 for rotation passes 1 and 2 (64-byte row
// pieces of 16 adjacent columns, and a CTA's warps keep the unrolled
// transform's code warm together: pass 2 5.05 -> 4.91 ms per survey step,
// 16 pairs 6.23 ms; pass 1 2.63 -> 2.56 ms), 4 for the others (with 8 pairs:
// shift columns 1.88 -> 2.17, shift rows 1.48 -> 1.58, rotation pass 3
// 1.97 -> 2.04 ms).  Register budget for 16 resident warps per SM (measured faster
// than 12 for every kind).
template <int KIND>
constexpr int w32_ppc() { return (KIND == ROT_P2 || KIND == ROT_P1) ? 8 : 4; }
constexpr size_t w32_smem_bytes(int ppc) { return (size_t)ppc * (1024 + 1024 / 32) * sizeof(float2); }

template <int KIND>
__global__ void __launch_bounds__(32 * w32_ppc<KIND>(), 16 / w32_ppc<KIND>()) line_pass_w32(const LineArgs a) {
  constexpr int M = 1024, N = 512, PPC = w32_ppc<KIND>();
  constexpr bool SAME_D = (KIND == SHIFT_X || KIND == SHIFT_Y);
  constexpr int NIN = (KIND == ROT_P3) ? M : N;
  constexpr int NOUT = (KIND == ROT_P1) ? M : N;
  extern __shared__ float2 w32_smem[];
  float2 (*sbuf)[M + M / 32] = reinterpret_cast<float2 (*)[M + M / 32]>(w32_smem);   // [PPC][M + M/32]
  __shared__ LineParam lp[PPC][2];
  __shared__ int ident_s;

  const int lane = threadIdx.x & 31, p = threadIdx.x >> 5;
  const long long f = blockIdx.y;
  const int line0 = 2 * (blockIdx.x * PPC + p);
  const float *__restrict__ fin = a.in_tab ? a.in_tab[f] : a.in + f * a.in_fstride;
  float *__restrict__ fout = a.out_tab ? a.out_tab[f] : a.out + f * a.out_fstride;
  const float2 *__restrict__ tw = d_tw1024_rl;
  float2 *buf = sbuf[p];
  const int q = (KIND == ROT_P1) ? (a.q[f] & 3) : 0;

  if (threadIdx.x == 0) {
    bool id;
    if constexpr (KIND == SHIFT_X) id = (a.p0[f] == 0.0);
    else if constexpr (KIND == SHIFT_Y) id = (a.p1[f] == 0.0);
    else id = (a.p0[f] == 0.0 && a.p1[f] == 0.0);
    ident_s = id ? 1 : 0;
  }
  if (lane < 2 && (!SAME_D || lane == 0)) {
    if (a.lp_tab)
      lp[p][lane] = reinterpret_cast<const LineParam *>(a.lp_tab)[f * a.lp_lines + (SAME_D ? 0 : line0 + lane)];
    else
      make_param(lp[p][lane], line_shift<KIND>(a, f, line0 + lane, N), M);
  }
  __syncthreads();

  bool bad = false;
  if (ident_s) {
    if constexpr (KIND == ROT_P2) return;
    for (int pos = lane; pos < NOUT; pos += 32) {
      float2 z = make_float2(0.f, 0.f);
      if (pos < NIN) {
        if constexpr (KIND == SHIFT_X || KIND == ROT_P3) {
          const int rs = (KIND == ROT_P3) ? M : N;
          z = make_float2(fin[(size_t)line0 * rs + pos], fin[(size_t)(line0 + 1) * rs + pos]);
        } else if constexpr (KIND == SHIFT_Y) {
          z = *reinterpret_cast<const float2 *>(fin + (size_t)pos * N + line0);
        } else if constexpr (KIND == ROT_P1) {
          z = load_rot90_pair(fin, N, q, line0, pos);
        }
      }
      if constexpr (KIND == SHIFT_X || KIND == ROT_P1) bad |= !finite_pair(z);
      if constexpr (KIND == SHIFT_Y) {
        *reinterpret_cast<float2 *>(fout + (size_t)pos * N + line0) = z;
      } else {
        const int rs = (KIND == ROT_P1) ? M : N;
        fout[(size_t)line0 * rs + pos] = z.x;
        fout[(size_t)(line0 + 1) * rs + pos] = z.y;
      }
    }
    if (bad) atomicOr(a.status, STATUS_NONFINITE);
    return;
  }

  // ---- load: v[m] = element lane + 32 m of the line pair -----------------
  // Column passes: the CTA's 2 PPC adjacent columns are read row by row as
  // 16-byte pieces (whole sectors) into the per-pair buffers first.
  constexpr bool COLS = (KIND == SHIFT_Y || KIND == ROT_P2);
  constexpr int RS = (KIND == ROT_P2) ? M : N;     // row stride of a column pass
  constexpr int HP = PPC / 2;                      // 16-byte pieces per row of the CTA's columns
  const int col0 = 2 * PPC * blockIdx.x;           // first column of the CTA
  if constexpr (COLS) {
    // every piece's load is issued before the first shared-memory store
    constexpr int IT = HP * NIN / (32 * PPC);
    static_assert(IT * 32 * PPC == HP * NIN, "pieces per thread");
    float4 q4[IT];
#pragma unroll
    for (int k = 0; k < IT; k++) {
      const int i = threadIdx.x + k * 32 * PPC, row = i / HP, h = i % HP;
      q4[k] = *reinterpret_cast<const float4 *>(fin + (size_t)row * RS + col0 + 4 * h);
    }
#pragma unroll
    for (int k = 0; k < IT; k++) {
      const int i = threadIdx.x + k * 32 * PPC, row = i / HP, h = i % HP;
      sbuf[2 * h][pad32(row)] = make_float2(q4[k].x, q4[k].y);
      sbuf[2 * h + 1][pad32(row)] = make_float2(q4[k].z, q4[k].w);
    }
    __syncthreads();
  }
  // Rotation pass 1 with an odd number of quarter turns: the lines of
  // rot90^q(frame) are columns of the frame, staged the same way.
  //   q = 1: element pos >= 1 of lines col0 + j is frame[n - pos][col0 + j];
  //   q = 3: element pos of line i >= 1 is frame[pos][n - i], i.e. columns
  //          n - col0 - 7 .. n - col0 for the CTA's lines col0 .. col0 + 7.
  const bool RCOLS = (KIND == ROT_P1) && (q & 1);
  if (RCOLS) {
    if (q == 1) {
      constexpr int IT = HP * N / (32 * PPC);
      float4 q4[IT];
#pragma unroll
      for (int k = 0; k < IT; k++) {
        const int i = threadIdx.x + k * 32 * PPC, row = i / HP, h = i % HP;
        q4[k] = row == 0 ? make_float4(0.f, 0.f, 0.f, 0.f)   // row 0 would be element n
                         : *reinterpret_cast<const float4 *>(fin + (size_t)row * N + col0 + 4 * h);
      }
#pragma unroll
      for (int k = 0; k < IT; k++) {
        const int i = threadIdx.x + k * 32 * PPC, row = i / HP, h = i % HP;
        if (row == 0) continue;
        sbuf[2 * h][pad32(N - row)] = make_float2(q4[k].x, q4[k].y);
        sbuf[2 * h + 1][pad32(N - row)] = make_float2(q4[k].z, q4[k].w);
      }
      if (threadIdx.x < PPC) sbuf[threadIdx.x][pad32(0)] = make_float2(0.f, 0.f);
    } else {
      // lines col0 + 2p and col0 + 2p + 1 are frame columns n - col0 - 2p and
      // n - col0 - 2p - 1: the row's 2 PPC floats from column cb, plus column
      // n - col0 for line col0 (line 0 of the frame is zero)
      constexpr int NF = 2 * PPC;
      const int cb = N - col0 - NF;                    // >= 0, a multiple of NF
      constexpr int IT = N / (32 * PPC);
      float f[IT][NF];
      float top[IT];
#pragma unroll
      for (int k = 0; k < IT; k++) {
        const float *rowp = fin + (size_t)(threadIdx.x + k * 32 * PPC) * N;
#pragma unroll
        for (int u = 0; u < NF / 4; u++) {
          const float4 x = *reinterpret_cast<const float4 *>(rowp + cb + 4 * u);
          f[k][4 * u] = x.x;
          f[k][4 * u + 1] = x.y;
          f[k][4 * u + 2] = x.z;
          f[k][4 * u + 3] = x.w;
        }
        top[k] = (col0 > 0) ? rowp[N - col0] : 0.f;
      }
#pragma unroll
      for (int k = 0; k < IT; k++) {
        const int pos = threadIdx.x + k * 32 * PPC;
#pragma unroll
        for (int pp = 0; pp < PPC; pp++)
          sbuf[pp][pad32(pos)] = make_float2(pp == 0 ? top[k] : f[k][NF - 2 * pp], f[k][NF - 1 - 2 * pp]);
      }
    }
    __syncthreads();
  }
  float2 v[32];
  if constexpr (KIND == ROT_P1) {
    // one branch per line pair, not per element, so that each form's loads
    // are issued together: staged columns (odd quarter turns), rows (q = 0)
    // or rows read backwards (q = 2: element pos >= 1 of line i >= 1 is
    // frame[n - i][n - pos])
    if (RCOLS) {
#pragma unroll
      for (int m = 0; m < 32; m++) v[m] = (32 * m < NIN) ? buf[pad32(lane + 32 * m)] : make_float2(0.f, 0.f);
    } else if (q == 0) {
#pragma unroll
      for (int m = 0; m < 32; m++) {
        const int pos = lane + 32 * m;
        v[m] = (32 * m < NIN) ? make_float2(fin[(size_t)line0 * N + pos], fin[(size_t)(line0 + 1) * N + pos])
                              : make_float2(0.f, 0.f);
      }
    } else {
      const float *r0 = fin + (size_t)(N - line0) * N + N;        // row n - line0 (unused for line0 = 0), + n
      const float *r1 = fin + (size_t)(N - line0 - 1) * N + N;    // row n - line0 - 1, + n
#pragma unroll
      for (int m = 0; m < 32; m++) {
        const int pos = lane + 32 * m;
        float2 z = make_float2(0.f, 0.f);
        if (32 * m < NIN && pos >= 1) z = make_float2(line0 >= 1 ? r0[-pos] : 0.f, r1[-pos]);
        v[m] = z;
      }
    }
#pragma unroll
    for (int m = 0; m < 32; m++) bad |= !finite_pair(v[m]);
  } else {
#pragma unroll
    for (int m = 0; m < 32; m++) {
      const int pos = lane + 32 * m;
      float2 z = make_float2(0.f, 0.f);
      if (32 * m < NIN) {
        if (COLS) {
          z = buf[pad32(pos)];
        } else if constexpr (KIND == SHIFT_X) {
          z = make_float2(fin[(size_t)line0 * N + pos], fin[(size_t)(line0 + 1) * N + pos]);
        } else if constexpr (KIND == SHIFT_Y) {
          z = *reinterpret_cast<const float2 *>(fin + (size_t)pos * N + line0);
        } else if constexpr (KIND == ROT_P2) {
          z = *reinterpret_cast<const float2 *>(fin + (size_t)pos * M + line0);
        } else {
          z = make_float2(fin[(size_t)line0 * M + pos], fin[(size_t)(line0 + 1) * M + pos]);
        }
        if constexpr (KIND == SHIFT_X) bad |= !finite_pair(z);
      }
      v[m] = z;
    }
  }
  if constexpr (KIND == SHIFT_X || KIND == ROT_P1) {
    if (bad) atomicOr(a.status, STATUS_NONFINITE);
  }
  if (COLS || RCOLS) __syncwarp();   // buf is the FFT's exchange buffer from here on
  w32_filter<KIND>(v, lane, buf, tw, lp[p][0], lp[p][SAME_D ? 0 : 1]);
  if constexpr (COLS) {
    // through the per-pair buffers, then row by row as 16-byte pieces
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 32; r++)
      if (32 * r < NOUT) buf[pad32(lane + 32 * r)] = make_float2(v[r].x, -v[r].y);
    __syncthreads();
    for (int i = threadIdx.x; i < HP * NOUT; i += 32 * PPC) {
      const int row = i / HP, h = i % HP;
      const float2 e0 = sbuf[2 * h][pad32(row)], e1 = sbuf[2 * h + 1][pad32(row)];
      *reinterpret_cast<float4 *>(fout + (size_t)row * RS + col0 + 4 * h) = make_float4(e0.x, e0.y, e1.x, e1.y);
    }
    return;
  }
#pragma unroll
  for (int r = 0; r < 32; r++) {
    const int pos = lane + 32 * r;
    if (32 * r < NOUT) {
      const float2 y = v[r];
      if constexpr (KIND == SHIFT_Y) {
        *reinterpret_cast<float2 *>(fout + (size_t)pos * N + line0) = make_float2(y.x, -y.y);
      } else if constexpr (KIND == ROT_P2) {
        *reinterpret_cast<float2 *>(fout + (size_t)pos * M + line0) = make_float2(y.x, -y.y);
      } else {
        const int rs = (KIND == ROT_P1) ? M : N;
        fout[(size_t)line0 * rs + pos] = y.x;
        fout[(size_t)(line0 + 1) * rs + pos] = -y.y;
      }
    }
  }
}

template <int KIND>
cudaError_t launch_w32(const LineArgs &a, long long n_frames, cudaStream_t st) {
  constexpr int M = 1024, N = 512, PPC = w32_ppc<KIND>();
  constexpr int NLINES = (KIND == ROT_P2) ? M : N;
  for (long long f0 = 0; f0 < n_frames; f0 += 65535) {
    const long long nf = (n_frames - f0 < 65535) ? (n_frames - f0) : 65535;
    LineArgs b = a;
    b.in = a.in + f0 * a.in_fstride;
    b.out = a.out + f0 * a.out_fstride;
    b.p0 = a.p0 ? a.p0 + f0 : nullptr;
    b.p1 = a.p1 ? a.p1 + f0 : nullptr;
    b.q = a.q ? a.q + f0 : nullptr;
    b.in_tab = a.in_tab ? a.in_tab + f0 : nullptr;
    b.out_tab = a.out_tab ? a.out_tab + f0 : nullptr;
    b.lp_tab = a.lp_tab ? reinterpret_cast<const LineParam *>(a.lp_tab) + f0 * a.lp_lines : nullptr;
    dim3 grid(NLINES / (2 * PPC), (unsigned)nf);
    line_pass_w32<KIND><<<grid, 32 * PPC, w32_smem_bytes(PPC), st>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Persistent executor for uneven batches: frames of any supported size, each
// shifted then rotated, in ONE launch.  Work items (one CTA-sized group of
// line pairs of one pass of one frame) are handed out in order from an
// atomic counter: waves of frames one after the other, within a wave pass
// by pass (shift x, shift y, rotation passes 1-3), within a pass frame by
// frame.  An item of pass p waits until its frame's pass p-1 items are done;
// rotation pass 1 of wave w also waits until wave w-2 has finished (their
// scratch slots alternate).  Every wait is on items handed out earlier, held
// by running CTAs, so none can wait forever; the waits are still bounded
// (clock-based), setting STATUS_TIMEOUT and moving on if a limit is hit.
// ---------------------------------------------------------------------------

template <int KIND>
__device__ __forceinline__ void batch_pass(const BatchFrame &fr, int cx, int *status, float2 *smem, LineParam *lp,
                                           int *ident) {
  LineArgs la{};
  la.status = status;
  la.in_fstride = 0;
  la.out_fstride = 0;
  la.n = fr.n;
  if constexpr (KIND == SHIFT_X) {
    la.in = fr.in; la.out = fr.out; la.p0 = &fr.dx; la.p1 = &fr.dy;
  } else if constexpr (KIND == SHIFT_Y) {
    la.in = fr.out; la.out = fr.out; la.p0 = &fr.dx; la.p1 = &fr.dy;
  } else {
    la.p0 = &fr.a; la.p1 = &fr.s; la.q = &fr.q;
    if constexpr (KIND == ROT_P1) { la.in = fr.rin; la.out = fr.scratch; }
    else if constexpr (KIND == ROT_P2) { la.in = fr.scratch; la.out = fr.scratch; }
    else { la.in = fr.scratch; la.out = fr.out; }
  }
  // L1-bypassing loads where this SM may hold a stale line: the rotation
  // passes read data that CTAs on other SMs wrote after this SM may have
  // cached it (frame columns after the column shift, recycled scratch).  The
  // shift passes read only the input (or lines only their own CTA wrote).
  constexpr bool CG = (KIND == ROT_P1 || KIND == ROT_P2 || KIND == ROT_P3);
  switch (fr.n) {
    case 64: line_pass_body<128, KIND, CG>(la, 0, cx, smem, lp, ident); break;
    case 128: line_pass_body<256, KIND, CG>(la, 0, cx, smem, lp, ident); break;
    case 256: line_pass_body<512, KIND, CG>(la, 0, cx, smem, lp, ident); break;
    case 512: line_pass_body<1024, KIND, CG>(la, 0, cx, smem, lp, ident); break;
    default: line_pass_body<2048, KIND, CG>(la, 0, cx, smem, lp, ident); break;
  }
}

// Wait until *ctr >= target.  Gives up after `limit` clock cycles, or at once
// when an earlier wait of the launch already gave up (so a launch with a
// broken dependency ends after one limit, not one limit per item).
__device__ __forceinline__ bool wait_at_least(const int *ctr, int target, long long limit, const int *status) {
  const long long t0 = clock64();
  while (*(volatile const int *)ctr < target) {
    if ((*(volatile const int *)status & STATUS_TIMEOUT) || clock64() - t0 > limit) return false;
    __nanosleep(64);
  }
  return true;
}

// Items are taken BATCH_GRAB at a time with one atomic; the next grab is
// issued before the current group is processed, hiding its latency.
constexpr int BATCH_GRAB = 4;

__global__ void __launch_bounds__(256, 2) batch_persistent_kernel(const BatchArgs b) {
  extern __shared__ float2 smem[];
  __shared__ LineParam lp[2 * 32];
  __shared__ int ident_s;
  __shared__ int grab_s[2];
  __shared__ int seg_s;
  const int tid = threadIdx.x;
  if (tid == 0) grab_s[0] = atomicAdd(b.next, BATCH_GRAB);
  int slot = 0;
  for (;;) {
    __syncthreads();
    const int g0 = grab_s[slot];
    if (g0 >= b.total) break;
    if (tid == 0) grab_s[slot ^ 1] = atomicAdd(b.next, BATCH_GRAB);   // next group, in flight
    const int g1 = min(g0 + BATCH_GRAB, b.total);
    for (int it = g0; it < g1; it++) {
      if (tid == 0) {
        const int sgi = __ldg(&b.seg_of_item[it]);
        seg_s = sgi;
        const BatchSeg sg = b.segs[sgi];
        bool ok = true;
        if (sg.pass > 0) ok = wait_at_least(&b.done[(sg.pass - 1) * b.nframes + sg.frame],
                                            b.frames[sg.frame].ctas[sg.pass - 1], b.spin_limit, b.status);
        if (ok && sg.pass == 2) {
          const int w = b.frames[sg.frame].wave;
          if (w >= 2) ok = wait_at_least(&b.wave_done[w - 2], b.wave_r3[w - 2], b.spin_limit, b.status);
        }
        if (!ok) atomicOr(b.status, STATUS_TIMEOUT);
        __threadfence();
      }
      __syncthreads();
      const BatchSeg sg = b.segs[seg_s];
      const BatchFrame &fr = b.frames[sg.frame];
      const int cx = it - sg.item0;
      switch (sg.pass) {
        case 0: batch_pass<SHIFT_X>(fr, cx, b.status, smem, lp, &ident_s); break;
        case 1: batch_pass<SHIFT_Y>(fr, cx, b.status, smem, lp, &ident_s); break;
        case 2: batch_pass<ROT_P1>(fr, cx, b.status, smem, lp, &ident_s); break;
        case 3: batch_pass<ROT_P2>(fr, cx, b.status, smem, lp, &ident_s); break;
        default: batch_pass<ROT_P3>(fr, cx, b.status, smem, lp, &ident_s); break;
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        atomicAdd(&b.done[sg.pass * b.nframes + sg.frame], 1);
        if (sg.pass == 4) atomicAdd(&b.wave_done[fr.wave], 1);
      }
    }
    slot ^= 1;
  }
}

template <int M>
size_t line_smem_bytes() {
  constexpr int LPC = 4096 / M;
  constexpr int LBUF = M + M / 16;
  return (size_t)2 * LPC * LBUF * sizeof(float2);
}

template <int M, int KIND>
cudaError_t launch_one(const LineArgs &a, long long n_frames, cudaStream_t st) {
  constexpr int N = M / 2;
  constexpr int LPC = 4096 / M;
  constexpr int NLINES = (KIND == ROT_P2) ? M : N;
  const size_t smem = line_smem_bytes<M>();   // limit raised by geom_init_device
  for (long long f0 = 0; f0 < n_frames; f0 += 65535) {
    const long long nf = (n_frames - f0 < 65535) ? (n_frames - f0) : 65535;
    LineArgs b = a;
    b.in = a.in + f0 * a.in_fstride;
    b.out = a.out + f0 * a.out_fstride;
    b.p0 = a.p0 ? a.p0 + f0 : nullptr;
    b.p1 = a.p1 ? a.p1 + f0 : nullptr;
    b.q = a.q ? a.q + f0 : nullptr;
    b.in_tab = a.in_tab ? a.in_tab + f0 : nullptr;
    b.out_tab = a.out_tab ? a.out_tab + f0 : nullptr;
    b.lp_tab = a.lp_tab ? reinterpret_cast<const LineParam *>(a.lp_tab) + f0 * a.lp_lines : nullptr;
    dim3 grid(NLINES / (2 * LPC), (unsigned)nf);
    line_pass_kernel<M, KIND><<<grid, 256, smem, st>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int M>
cudaError_t launch_m(LineKind kind, const LineArgs &a, long long n_frames, cudaStream_t st) {
  switch (kind) {
    case SHIFT_X: return launch_one<M, SHIFT_X>(a, n_frames, st);
    case SHIFT_Y: return launch_one<M, SHIFT_Y>(a, n_frames, st);
    case ROT_P1: return launch_one<M, ROT_P1>(a, n_frames, st);
    case ROT_P2: return launch_one<M, ROT_P2>(a, n_frames, st);
    case ROT_P3: return launch_one<M, ROT_P3>(a, n_frames, st);
  }
  return cudaErrorInvalidValue;
}

// Raise the dynamic shared-memory limit of every generic line-pass kernel of
// length M (done once per device at set-up, outside any stream capture).
template <int M>
bool configure_m() {
  const int smem = (int)line_smem_bytes<M>();
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  return cudaFuncSetAttribute(line_pass_kernel<M, SHIFT_X>, at, smem) == cudaSuccess &&
         cudaFuncSetAttribute(line_pass_kernel<M, SHIFT_Y>, at, smem) == cudaSuccess &&
         cudaFuncSetAttribute(line_pass_kernel<M, ROT_P1>, at, smem) == cudaSuccess &&
         cudaFuncSetAttribute(line_pass_kernel<M, ROT_P2>, at, smem) == cudaSuccess &&
         cudaFuncSetAttribute(line_pass_kernel<M, ROT_P3>, at, smem) == cudaSuccess;
}

}  // namespace

// One thread per line: the line's shift parameters in FP64 (the arithmetic
// each CTA of the passes would otherwise do on GB300's narrow FP64 pipe).
template <int KIND>
__global__ void __launch_bounds__(256) line_param_kernel(const LineArgs a, long long n_frames, int lines,
                                                        LineParam *out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_frames * lines) return;
  const long long f = idx / lines;
  const int line = (int)(idx - f * lines);
  make_param(out[idx], line_shift<KIND>(a, f, line, a.n), 2 * a.n);
}

int line_params_lines(LineKind kind, int n) {
  return (kind == SHIFT_X || kind == SHIFT_Y) ? 1 : (kind == ROT_P2 ? 2 * n : n);
}

size_t line_params_bytes(LineKind kind, int n, long long n_frames) {
  return (size_t)n_frames * line_params_lines(kind, n) * sizeof(LineParam);
}

cudaError_t launch_line_params(LineKind kind, const LineArgs &a, long long n_frames, void *out, cudaStream_t st) {
  const int lines = line_params_lines(kind, a.n);
  const long long total = n_frames * lines;
  if (total == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((total + 255) / 256);
  LineParam *o = reinterpret_cast<LineParam *>(out);
  switch (kind) {
    case SHIFT_X: line_param_kernel<SHIFT_X><<<grid, 256, 0, st>>>(a, n_frames, lines, o); break;
    case SHIFT_Y: line_param_kernel<SHIFT_Y><<<grid, 256, 0, st>>>(a, n_frames, lines, o); break;
    case ROT_P1:
    case ROT_P3: line_param_kernel<ROT_P1><<<grid, 256, 0, st>>>(a, n_frames, lines, o); break;
    case ROT_P2: line_param_kernel<ROT_P2><<<grid, 256, 0, st>>>(a, n_frames, lines, o); break;
  }
  return cudaGetLastError();
}

int geom_init_device() {
  if (!(configure_m<128>() && configure_m<256>() && configure_m<512>() && configure_m<1024>() &&
        configure_m<2048>()))
    return -1;
  {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (cudaFuncSetAttribute(line_pass_w32<SHIFT_X>, at, (int)w32_smem_bytes(w32_ppc<SHIFT_X>())) != cudaSuccess ||
        cudaFuncSetAttribute(line_pass_w32<SHIFT_Y>, at, (int)w32_smem_bytes(w32_ppc<SHIFT_Y>())) != cudaSuccess ||
        cudaFuncSetAttribute(line_pass_w32<ROT_P1>, at, (int)w32_smem_bytes(w32_ppc<ROT_P1>())) != cudaSuccess ||
        cudaFuncSetAttribute(line_pass_w32<ROT_P2>, at, (int)w32_smem_bytes(w32_ppc<ROT_P2>())) != cudaSuccess ||
        cudaFuncSetAttribute(line_pass_w32<ROT_P3>, at, (int)w32_smem_bytes(w32_ppc<ROT_P3>())) != cudaSuccess)
      return -1;
  }
  // the persistent batch kernel is launched inside stream capture: set its
  // shared-memory limit here, per device, outside any capture
  if (cudaFuncSetAttribute(batch_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)line_smem_bytes<1024>()) != cudaSuccess)
    return -1;
  static float2 host[kTwTotal];
  static bool filled = false;
  if (!filled) {
    for (int m = 128; m <= 2048; m *= 2)
      for (int e = 0; e < m; e++) {
        const double ang = 2.0 * 3.14159265358979323846 * (double)e / (double)m;
        host[tw_off(m) + e] = make_float2((float)cos(ang), (float)-sin(ang));
      }
    filled = true;
  }
  static float2 rl[32 * 32];
  for (int r = 0; r < 32; r++)
    for (int l = 0; l < 32; l++) rl[r * 32 + l] = host[tw_off(1024) + r * l];
  if (cudaMemcpyToSymbol(d_tw1024_rl, rl, sizeof(rl)) != cudaSuccess) return -1;
  return cudaMemcpyToSymbol(d_twiddle, host, sizeof(host)) == cudaSuccess ? 0 : -1;
}

cudaError_t launch_batch_persistent(const BatchArgs &b, int ctas_per_sm, cudaStream_t st) {
  const size_t smem = line_smem_bytes<1024>();   // the same for every line length
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long grid = (long long)sms * (ctas_per_sm > 0 ? ctas_per_sm : 1);
  if (grid > b.total) grid = b.total;
  if (grid < 1) return cudaSuccess;
  batch_persistent_kernel<<<(unsigned)grid, 256, smem, st>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_line_pass(LineKind kind, const LineArgs &a, long long n_frames, cudaStream_t st, int variant_1024) {
  if (n_frames <= 0) return cudaSuccess;
  switch (a.n) {
    case 64: return launch_m<128>(kind, a, n_frames, st);
    case 128: return launch_m<256>(kind, a, n_frames, st);
    case 256: return launch_m<512>(kind, a, n_frames, st);
    case 512:
      if (!variant_1024) return launch_m<1024>(kind, a, n_frames, st);
      switch (kind) {
        case SHIFT_X: return launch_w32<SHIFT_X>(a, n_frames, st);
        case SHIFT_Y: return launch_w32<SHIFT_Y>(a, n_frames, st);
        case ROT_P1: return launch_w32<ROT_P1>(a, n_frames, st);
        case ROT_P2: return launch_w32<ROT_P2>(a, n_frames, st);
        case ROT_P3: return launch_w32<ROT_P3>(a, n_frames, st);
      }
      return cudaErrorInvalidValue;
    case 1024: return launch_m<2048>(kind, a, n_frames, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace graphic

// tc.cu -- precision variant of the Fourier line passes (shift, Sect. 3.3.1;
// three-shear rotation, Sect. 3.4) on the 5th-generation tensor cores
// (tcgen05, sm_103a), for 2048-point padded lines (frames of 1024 x 1024).
//
// Each line PAIR is packed as one complex line z = a + i b, as in the FP32
// kernels, and the same filter v = IFFT(H . FFT(u)) is applied.  The DFTs
// are the change: m = 2048 = 16 . 16 . 8 and every radix stage is one dense
// GEMM on the tensor cores.  With n = 128 a + b (a < 16, b < 128) and
// k = c + 16 c2 + 256 d3:
//   stage 1  u[b][c]      = sum_a  z[128 a + b] W16^(a c),   times W2048^(b c)
//   stage 2  v[c,b2][c2]  = sum_a2 u[8 a2 + b2][c] W16^(a2 c2), times W128^(b2 c2)
//   stage 3  Z[k]         = sum_b2 v[c,b2][c2] W8^(b2 d3)
// One stage is D[rows x 2R] = A[rows x 2R] . B with rows the independent
// R-point vectors (128 per line; 256 for the radix-8 stage), complex values
// interleaved along K (re, im) -- one packed 32-bit word per complex value
// and part -- and B the real form of the DFT matrix, its output columns
// interleaved the same way.  A and B are split into hi + lo parts of one 16-bit type (BF16 or
// FP16), x = hi + lo 2^-s with lo stored scaled by 2^s (s = 8 for BF16, 11
// for FP16: the lo parts keep the normal range, which the tensor cores need
// -- subnormal FP16 operands lose their value), and two FP32 accumulators in
// tensor memory take D_hi = A_hi B_hi and D_x = A_lo B_hi + A_hi B_lo; the
// epilogue forms D = D_hi + 2^-s D_x (the A_lo B_lo term, 2^-2s, is below
// the representation error of the split).  FP16 values too small for a
// normal hi part go wholly into lo.  Between stages each thread reads its
// accumulator rows (tcgen05.ld), applies the twiddles in FP32, splits again
// and stores the next stage's operand rows in shared memory.  Phase arguments of the
// middle step are the FP32 kernels' (FP64 per-line reduction of d/m).
// FP16 range: every line is scaled by a power of two so that max |z| <= 1;
// radix stages grow values at most by their radix (2048 in all), the middle
// step's 1/m scale brings the inverse's input back below 2, so no value
// exceeds 2^13 < 65504; the power of two is undone at the store.
//
// tcgen05 usage: one 64-column tensor-memory allocation per CTA (warp 0),
// MMAs (kind::f16, M = 128, N = 32 or 16, K = 16, operands K-major in the
// canonical no-swizzle core-matrix layout) issued by thread 0 and committed
// to one mbarrier; every wait on it is bounded (STATUS_TIMEOUT).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "graphic_internal.h"
#include "line_common.cuh"

namespace graphic {
namespace {

constexpr int TC_M = 2048;        // padded line length
constexpr int TC_N = 1024;        // frame side
constexpr int TC_PPC = 4;         // line pairs per CTA (one after the other)
#ifndef TC_MIN_CTAS
#define TC_MIN_CTAS 4             // resident CTAs per SM the register budget is cut for (4: fastest measured)
#endif

// Twiddles (FP64 cos / sin rounded to FP32), laid out for coalesced reads:
// stage 1 W_2048^(t c) at [c][t] (t < 128, c < 16), stage 2 W_128^(b2 c2)
// at [b2][c2] (b2 < 8, c2 < 16).
__device__ float2 d_tw1[16 * 128];
__device__ float2 d_tw2[8 * 16];

// Real forms of the DFT matrices (B operands, N x K, K-major core-matrix
// order), hi and lo parts, per element type (0: BF16, 1: FP16).
struct TcTables {
  uint16_t r16[2][2][32 * 32];
  uint16_t r8[2][2][16 * 16];
};
__device__ TcTables d_tc;

// byte offset of element (r, k) of a K-major operand with KD columns:
// 8-row x 16-byte core matrices, adjacent along K (128 B apart), 8-row
// groups KD * 16 bytes apart.
__host__ __device__ constexpr int kmaj_off(int r, int k, int KD) {
  return (r >> 3) * (KD * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// shared-memory layout (bytes from a 1024-aligned base)
constexpr int SM_A = 0;           // A hi [0, 8192), A lo [8192, 16384)
constexpr int SM_ALO = 8192;
constexpr int SM_B16 = 16384;     // radix-16 B hi, lo (2048 each)
constexpr int SM_B8 = 20480;      // radix-8 B hi, lo (512 each)
constexpr int SM_Z = 21504;       // natural-order spectrum, 2048 x float2
constexpr int SM_BYTES = SM_Z + TC_M * 8;

// two floats -> one 32-bit word of two 16-bit values (lo half = a), and back
template <bool F16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if constexpr (F16) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
}
template <bool F16>
__device__ __forceinline__ float2 unpack2(uint32_t w) {
  if constexpr (F16) return __half22float2(*reinterpret_cast<const __half2 *>(&w));
  else return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
}

// scale of the stored lo parts: 2^(precision bits of the type)
template <bool F16>
struct LoScale {
  static constexpr float up = F16 ? 2048.f : 256.f;
  static constexpr float down = F16 ? (1.f / 2048.f) : (1.f / 256.f);
};

// complex x -> packed hi and packed lo 2^s; FP16 values below the normal
// range go wholly into lo
template <bool F16>
__device__ __forceinline__ void split2(float2 x, uint32_t &h, uint32_t &l) {
  h = pack2<F16>(x.x, x.y);
  float2 hf = unpack2<F16>(h);
  if constexpr (F16) {
    const bool tr = fabsf(x.x) < 6.103515625e-05f, ti = fabsf(x.y) < 6.103515625e-05f;
    h &= (tr ? 0xffff0000u : 0xffffffffu) & (ti ? 0x0000ffffu : 0xffffffffu);
    hf.x = tr ? 0.f : hf.x;
    hf.y = ti ? 0.f : hf.y;
  }
  l = pack2<F16>((x.x - hf.x) * LoScale<F16>::up, (x.y - hf.y) * LoScale<F16>::up);
}

// complex x -> hi and lo words at byte offset `off` of the A operand
template <bool F16>
__device__ __forceinline__ void put_split(unsigned char *sm, int off, float2 x) {
  uint32_t h, l;
  split2<F16>(x, h, l);
  *reinterpret_cast<uint32_t *>(sm + SM_A + off) = h;
  *reinterpret_cast<uint32_t *>(sm + SM_ALO + off) = l;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version; base offset 0, no swizzle
  return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, A and B of one
// 16-bit type, both K-major, shape M x N
__host__ __device__ constexpr uint32_t idesc(int M, int N, bool f16) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

// Wait for the mbarrier phase `parity`; false after `limit` clock cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity));
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// Row of the combined accumulator D_hi + 2^-s D_x, columns 0..31.
template <bool F16>
__device__ __forceinline__ void acc_row(uint32_t trow, float (&v)[32]) {
#pragma unroll
  for (int h = 0; h < 2; h++) {
    float a[16], b[16];
    tmem_ld16(trow + 16 * h, a);
    tmem_ld16(trow + 32 + 16 * h, b);
#pragma unroll
    for (int i = 0; i < 16; i++) v[16 * h + i] = fmaf(b[i], LoScale<F16>::down, a[i]);
  }
}

// Operand stores done, accumulator reads done: make both visible to the
// tensor cores, then one CTA barrier.
__device__ __forceinline__ void to_mma_sync() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Thread 0: the split products of a radix-16 stage (two K steps): D_hi in
// columns 0-31, D_x in columns 32-63.
__device__ __forceinline__ void issue_r16(uint32_t tmem, uint32_t sbase, uint32_t mbar, bool f16) {
  const uint32_t id = idesc(128, 32, f16);
#pragma unroll
  for (int ks = 0; ks < 2; ks++) {
    const uint64_t ah = sdesc(sbase + SM_A + ks * 256, 128, 512);
    const uint64_t al = sdesc(sbase + SM_ALO + ks * 256, 128, 512);
    const uint64_t bh = sdesc(sbase + SM_B16 + ks * 256, 128, 512);
    const uint64_t bl = sdesc(sbase + SM_B16 + 2048 + ks * 256, 128, 512);
    const uint32_t acc = ks > 0 ? 1u : 0u;
    mma(tmem, ah, bh, id, acc);
    mma(tmem + 32, al, bh, id, acc);
    mma(tmem + 32, ah, bl, id, 1u);
  }
  commit(mbar);
}

// Thread 0: the radix-8 stage, two 128-row tiles: D_hi of tile t in columns
// 16 t .. 16 t + 15, D_x in 32 + 16 t ...
__device__ __forceinline__ void issue_r8(uint32_t tmem, uint32_t sbase, uint32_t mbar, bool f16) {
  const uint32_t id = idesc(128, 16, f16);
  const uint64_t bh = sdesc(sbase + SM_B8, 128, 256);
  const uint64_t bl = sdesc(sbase + SM_B8 + 512, 128, 256);
#pragma unroll
  for (int t = 0; t < 2; t++) {
    const uint64_t ah = sdesc(sbase + SM_A + t * 4096, 128, 256);
    const uint64_t al = sdesc(sbase + SM_ALO + t * 4096, 128, 256);
    mma(tmem + 16 * t, ah, bh, id, 0u);
    mma(tmem + 32 + 16 * t, al, bh, id, 0u);
    mma(tmem + 32 + 16 * t, ah, bl, id, 1u);
  }
  commit(mbar);
}

struct TcState {
  unsigned char *sm;
  uint32_t sbase, tmem_row, tmem, mbar;
  uint32_t phase;
  int tid;
  long long limit;
  bool ok;
};

// Issue the MMAs of one stage and wait for them (bounded).  After a wait
// that ran out (s.ok false, the same in every thread) nothing more is issued.
template <bool F16, bool R8>
__device__ __forceinline__ void run_stage(TcState &s) {
  if (!s.ok) return;
  if (s.tid == 0) {
    if constexpr (R8) issue_r8(s.tmem, s.sbase, s.mbar, F16);
    else issue_r16(s.tmem, s.sbase, s.mbar, F16);
  }
  const bool got = mbar_wait(s.mbar, s.phase, s.limit);
  s.ok = __syncthreads_and(got) != 0;
  if (s.ok) s.phase ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Forward 2048-point DFT of the line whose stage-1 operand is in place.
// On return, thread t holds Z[t + 256 d3] in (w[2 d3], w[2 d3 + 1]) and
// Z[128 + t + 256 d3] in (w[16 + 2 d3], w[17 + 2 d3]).
template <bool F16>
__device__ __forceinline__ void dft2048(TcState &s, float (&w)[32]) {
  const int t = s.tid;
  // stage 1: rows b = t, twiddle W2048^(b c), rows of stage 2 are (c, b2)
  run_stage<F16, false>(s);
  {
    float u[32];
    acc_row<F16>(s.tmem_row, u);
    const int a2 = t >> 3, b2 = t & 7;
#pragma unroll
    for (int c = 0; c < 16; c++) {
      const float2 x = cmul(make_float2(u[2 * c], u[2 * c + 1]), __ldg(&d_tw1[c * 128 + t]));
      put_split<F16>(s.sm, kmaj_off(c * 8 + b2, 2 * a2, 32), x);
    }
  }
  to_mma_sync();
  // stage 2: rows (c, b2) = t, twiddle W128^(b2 c2), rows of stage 3 are r3 = 16 c2 + c
  run_stage<F16, false>(s);
  {
    float v[32];
    acc_row<F16>(s.tmem_row, v);
    const int c = t >> 3, b2 = t & 7;
#pragma unroll
    for (int c2 = 0; c2 < 16; c2++) {
      const float2 x = cmul(make_float2(v[2 * c2], v[2 * c2 + 1]), __ldg(&d_tw2[b2 * 16 + c2]));
      put_split<F16>(s.sm, kmaj_off(16 * c2 + c, 2 * b2, 16), x);
    }
  }
  to_mma_sync();
  // stage 3: radix 8, output index k = r3 + 256 d3
  run_stage<F16, true>(s);
  acc_row<F16>(s.tmem_row, w);
}

// Stage-1 operand row b = t from the natural-order values z[128 a + t]:
// complex value a at K positions (2a, 2a + 1), written as 16-byte chunks.
template <bool F16>
__device__ __forceinline__ void put_row_s1(unsigned char *sm, int t, const float2 (&z)[16]) {
  uint32_t hw[16], lw[16];
#pragma unroll
  for (int a = 0; a < 16; a++) split2<F16>(z[a], hw[a], lw[a]);
#pragma unroll
  for (int q = 0; q < 4; q++) {       // four 8-element core-matrix rows along K
    const int off = kmaj_off(t, 8 * q, 32);
    *reinterpret_cast<uint4 *>(sm + SM_A + off) = make_uint4(hw[4 * q], hw[4 * q + 1], hw[4 * q + 2], hw[4 * q + 3]);
    *reinterpret_cast<uint4 *>(sm + SM_ALO + off) =
        make_uint4(lw[4 * q], lw[4 * q + 1], lw[4 * q + 2], lw[4 * q + 3]);
  }
}

template <int KIND, bool F16>
__global__ void __launch_bounds__(128, TC_MIN_CTAS) line_pass_tc(const LineArgs a) {
  constexpr int M = TC_M, N = TC_N;
  constexpr bool SAME_D = (KIND == SHIFT_X || KIND == SHIFT_Y);
  constexpr int NIN = (KIND == ROT_P3) ? M : N;
  constexpr int NOUT = (KIND == ROT_P1) ? M : N;
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ LineParam lp[2];
  __shared__ __align__(8) uint64_t mbar_s;
  __shared__ uint32_t tslot;
  __shared__ int ident_s;
  __shared__ float red[4];

  unsigned char *sm = smraw;
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long f = blockIdx.y;
  const float *__restrict__ fin = a.in_tab ? a.in_tab[f] : a.in + f * a.in_fstride;
  float *__restrict__ fout = a.out_tab ? a.out_tab[f] : a.out + f * a.out_fstride;
  const int q = (KIND == ROT_P1) ? (a.q[f] & 3) : 0;

  // set-up: mbarrier, tensor memory, DFT operands
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_s)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    bool id;
    if constexpr (KIND == SHIFT_X) id = (a.p0[f] == 0.0);
    else if constexpr (KIND == SHIFT_Y) id = (a.p1[f] == 0.0);
    else id = (a.p0[f] == 0.0 && a.p1[f] == 0.0);
    ident_s = id ? 1 : 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  {
    const int ty = F16 ? 1 : 0;
    const uint4 *s16 = reinterpret_cast<const uint4 *>(&d_tc.r16[ty][0][0]);   // hi then lo, contiguous
    const uint4 *s8 = reinterpret_cast<const uint4 *>(&d_tc.r8[ty][0][0]);
    uint4 *d16 = reinterpret_cast<uint4 *>(sm + SM_B16);
    uint4 *d8 = reinterpret_cast<uint4 *>(sm + SM_B8);
    for (int i = tid; i < 4096 / 16; i += 128) d16[i] = s16[i];
    for (int i = tid; i < 1024 / 16; i += 128) d8[i] = s8[i];
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  TcState st;
  st.sm = sm;
  st.sbase = smem_u32(sm);
  st.tmem = tslot;
  st.tmem_row = tslot + ((uint32_t)(warp * 32) << 16);
  st.mbar = smem_u32(&mbar_s);
  st.phase = 0;
  st.tid = tid;
  st.limit = 2000000000ll;   // about one second of clock cycles
  st.ok = true;
  float2 *Z = reinterpret_cast<float2 *>(sm + SM_Z);

  const int pairs = ((KIND == ROT_P2) ? M : N) / 2;
  for (int pp = 0; pp < TC_PPC; pp++) {
    const int pair = blockIdx.x * TC_PPC + pp;
    if (pair >= pairs) break;
    const int line0 = 2 * pair;
    if (tid < 2 && (!SAME_D || tid == 0)) {
      if (a.lp_tab)
        lp[tid] = reinterpret_cast<const LineParam *>(a.lp_tab)[f * a.lp_lines + (SAME_D ? 0 : line0 + tid)];
      else
        make_param(lp[tid], line_shift<KIND>(a, f, line0 + tid, N), M);
    }
    __syncthreads();

    bool bad = false;
    if (ident_s) {
      // zero shift for every line of the frame: exact copy
      if constexpr (KIND != ROT_P2) {
        for (int pos = tid; pos < NOUT; pos += 128) {
          float2 z = make_float2(0.f, 0.f);
          if (pos < NIN) {
            if constexpr (KIND == SHIFT_X || KIND == ROT_P3) {
              const int rs = (KIND == ROT_P3) ? M : N;
              z = make_float2(fin[(size_t)line0 * rs + pos], fin[(size_t)(line0 + 1) * rs + pos]);
            } else if constexpr (KIND == SHIFT_Y) {
              z = *reinterpret_cast<const float2 *>(fin + (size_t)pos * N + line0);
            } else {
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
      }
      __syncthreads();
      continue;
    }

    // ---- load z[128 a + tid], scale to max |z| <= 1 --------------------------
    float2 z[16];
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const int pos = 128 * k + tid;
      float2 v = make_float2(0.f, 0.f);
      if (128 * k < NIN) {
        if constexpr (KIND == SHIFT_X) {
          v = make_float2(fin[(size_t)line0 * N + pos], fin[(size_t)(line0 + 1) * N + pos]);
        } else if constexpr (KIND == SHIFT_Y) {
          v = *reinterpret_cast<const float2 *>(fin + (size_t)pos * N + line0);
        } else if constexpr (KIND == ROT_P1) {
          v = load_rot90_pair(fin, N, q, line0, pos);
        } else if constexpr (KIND == ROT_P2) {
          v = *reinterpret_cast<const float2 *>(fin + (size_t)pos * M + line0);
        } else {
          v = make_float2(fin[(size_t)line0 * M + pos], fin[(size_t)(line0 + 1) * M + pos]);
        }
        if constexpr (KIND == SHIFT_X || KIND == ROT_P1) bad |= !finite_pair(v);
      }
      z[k] = v;
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    if constexpr (KIND == SHIFT_X || KIND == ROT_P1) {
      if (bad) atomicOr(a.status, STATUS_NONFINITE);
    }
    // non-finite values make the scale meaningless; their lines come out garbage
    // while the status word reports them
    mx = isfinite(mx) ? mx : 0.f;
    mx = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mx)));
    if ((tid & 31) == 0) red[warp] = mx;
    __syncthreads();
    mx = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
    // power of two with max |z| 2^-e <= 1, clamped so that both factors stay
    // finite (lines below 2^-64 of unit scale are kept unscaled-up)
    const int e = (mx > 0.f) ? max(ilogbf(mx) + 1, -64) : 0;
    const float sc_in = ldexpf(1.f, -e), sc_out = ldexpf(1.f, e);
#pragma unroll
    for (int k = 0; k < 16; k++) z[k] = make_float2(z[k].x * sc_in, z[k].y * sc_in);
    put_row_s1<F16>(sm, tid, z);
    to_mma_sync();

    // ---- forward DFT -> natural-order spectrum in shared memory ---------------
    float w[32];
    dft2048<F16>(st, w);
#pragma unroll
    for (int d3 = 0; d3 < 8; d3++) {
      Z[tid + 256 * d3] = make_float2(w[2 * d3], w[2 * d3 + 1]);
      Z[128 + tid + 256 * d3] = make_float2(w[16 + 2 * d3], w[17 + 2 * d3]);
    }
    __syncthreads();

    // ---- middle: phasors (separating the two real spectra), conj(V) / m ------
    {
      const LineParam &la = lp[0];
      const LineParam &lb = lp[SAME_D ? 0 : 1];
      const float inv_m = 1.0f / (float)M;
#pragma unroll 2
      for (int r = 0; r < 8; r++) {
        const int k = tid + 128 * r;   // 0 .. 1023
        if (k == 0) {
          const float2 z0 = Z[0];
          Z[0] = make_float2(z0.x * inv_m, -z0.y * inv_m);
          continue;
        }
        const float2 ha = phase_at(la, k);
        const float2 zk = Z[k], zm = Z[M - k];
        float2 vk, vm;
        if constexpr (SAME_D) {
          vk = cmul(zk, ha);
          vm = cmul(zm, cconj(ha));
        } else {
          const float2 hb = phase_at(lb, k);
          const float2 A = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
          const float2 B = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
          const float2 P = cmul(A, ha), Q = cmul(B, hb);
          vk = make_float2(P.x - Q.y, P.y + Q.x);
          vm = make_float2(P.x + Q.y, Q.x - P.y);
        }
        Z[k] = make_float2(vk.x * inv_m, -vk.y * inv_m);
        Z[M - k] = make_float2(vm.x * inv_m, -vm.y * inv_m);
      }
      if (tid == 0) {
        const float2 zn = Z[M / 2];
        Z[M / 2] = make_float2(zn.x * la.cnyq * inv_m, -zn.y * lb.cnyq * inv_m);
      }
    }
    __syncthreads();

    // ---- inverse: forward DFT of conj(V) / m, conjugated at the store -------
#pragma unroll
    for (int k = 0; k < 16; k++) z[k] = Z[128 * k + tid];
    put_row_s1<F16>(sm, tid, z);
    to_mma_sync();
    dft2048<F16>(st, w);
#pragma unroll
    for (int tt = 0; tt < 2; tt++) {
#pragma unroll
      for (int d3 = 0; d3 < 8; d3++) {
        const int pos = 128 * tt + tid + 256 * d3;
        if (256 * d3 < NOUT) {
          const float2 y = make_float2(w[16 * tt + 2 * d3] * sc_out, -w[16 * tt + 2 * d3 + 1] * sc_out);
          if constexpr (KIND == SHIFT_Y) {
            *reinterpret_cast<float2 *>(fout + (size_t)pos * N + line0) = y;
          } else if constexpr (KIND == ROT_P2) {
            *reinterpret_cast<float2 *>(fout + (size_t)pos * M + line0) = y;
          } else {
            const int rs = (KIND == ROT_P1) ? M : N;
            fout[(size_t)line0 * rs + pos] = y.x;
            fout[(size_t)(line0 + 1) * rs + pos] = y.y;
          }
        }
      }
    }
    // operand and accumulator free for the next pair (lp rewritten after this)
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!st.ok) break;
  }
  if (!st.ok) {
    // a wait ran out: record it, give the MMAs in flight one more bounded wait
    if (tid == 0) atomicOr(a.status, STATUS_TIMEOUT);
    mbar_wait(st.mbar, st.phase, st.limit);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(st.tmem));
}

template <int KIND, bool F16>
cudaError_t launch_kind(const LineArgs &a, long long n_frames, cudaStream_t st) {
  constexpr int NLINES = (KIND == ROT_P2) ? TC_M : TC_N;
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
    dim3 grid((NLINES / 2 + TC_PPC - 1) / TC_PPC, (unsigned)nf);
    line_pass_tc<KIND, F16><<<grid, 128, SM_BYTES + 1024, st>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <bool F16>
cudaError_t launch_prec(LineKind kind, const LineArgs &a, long long n_frames, cudaStream_t st) {
  switch (kind) {
    case SHIFT_X: return launch_kind<SHIFT_X, F16>(a, n_frames, st);
    case SHIFT_Y: return launch_kind<SHIFT_Y, F16>(a, n_frames, st);
    case ROT_P1: return launch_kind<ROT_P1, F16>(a, n_frames, st);
    case ROT_P2: return launch_kind<ROT_P2, F16>(a, n_frames, st);
    case ROT_P3: return launch_kind<ROT_P3, F16>(a, n_frames, st);
  }
  return cudaErrorInvalidValue;
}

uint16_t host16(float x, bool f16) {
  if (f16) return __half_as_ushort(__float2half_rn(x));
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
float host_from16(uint16_t h, bool f16) {
  if (f16) return __half2float(__ushort_as_half(h));
  return __bfloat162float(__ushort_as_bfloat16(h));
}

// B[n][k] of a radix-R stage: y_c = sum_a x_a W_R^(a c), complex values
// interleaved (re, im):  B[2c][2a] = Re W, B[2c][2a+1] = -Im W,
// B[2c+1][2a] = Im W, B[2c+1][2a+1] = Re W.
void fill_dft(int R, bool f16, uint16_t *hi, uint16_t *lo) {
  const double pi = 3.14159265358979323846;
  const int K = 2 * R;
  for (int n = 0; n < K; n++)
    for (int k = 0; k < K; k++) {
      const int c = n >> 1, a = k >> 1;
      const double ang = 2.0 * pi * (double)((a * c) % R) / (double)R;
      const double wr = cos(ang), wi = -sin(ang);
      double v;
      if ((n & 1) == 0) v = (k & 1) ? -wi : wr;
      else v = (k & 1) ? wr : wi;
      const uint16_t h = (f16 && fabs(v) < 6.103515625e-05) ? (uint16_t)0 : host16((float)v, f16);
      const uint16_t l = host16((float)((v - (double)host_from16(h, f16)) * (f16 ? 2048.0 : 256.0)), f16);
      const int idx = kmaj_off(n, k, K) / 2;
      hi[idx] = h;
      lo[idx] = l;
    }
}

}  // namespace

int tc_init_device() {
  static float2 tw1[16 * 128], tw2[8 * 16];
  static TcTables tab;
  static bool filled = false;
  if (!filled) {
    const double pi = 3.14159265358979323846;
    for (int c = 0; c < 16; c++)
      for (int t = 0; t < 128; t++) {
        const double ang = 2.0 * pi * (double)((t * c) % TC_M) / (double)TC_M;
        tw1[c * 128 + t] = make_float2((float)cos(ang), (float)-sin(ang));
      }
    for (int b2 = 0; b2 < 8; b2++)
      for (int c2 = 0; c2 < 16; c2++) {
        const double ang = 2.0 * pi * (double)((b2 * c2) % 128) / 128.0;
        tw2[b2 * 16 + c2] = make_float2((float)cos(ang), (float)-sin(ang));
      }
    for (int ty = 0; ty < 2; ty++) {
      fill_dft(16, ty == 1, tab.r16[ty][0], tab.r16[ty][1]);
      fill_dft(8, ty == 1, tab.r8[ty][0], tab.r8[ty][1]);
    }
    filled = true;
  }
  if (cudaMemcpyToSymbol(d_tw1, tw1, sizeof(tw1)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(d_tw2, tw2, sizeof(tw2)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(d_tc, &tab, sizeof(tab)) != cudaSuccess) return -1;
  return 0;
}

bool tc_supported(int n) { return n == TC_N; }

cudaError_t launch_line_pass_tc(LineKind kind, const LineArgs &a, long long n_frames, cudaStream_t st,
                                int precision) {
  if (n_frames <= 0) return cudaSuccess;
  if (a.n != TC_N) return cudaErrorInvalidValue;
  if (precision == PREC_FP16X3) return launch_prec<true>(kind, a, n_frames, st);
  if (precision == PREC_BF16X3) return launch_prec<false>(kind, a, n_frames, st);
  return cudaErrorInvalidValue;
}

}  // namespace graphic

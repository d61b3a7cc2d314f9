// select_common.cuh -- device helpers shared by the selection kernels (the
// median collapse and general median PSF path of median.cu, the band path of
// psf_band.cu): IEEE total-order keys, asynchronous shared-memory copies, bit
// selection.  Each translation unit gets its own copy (anonymous namespace).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace graphic {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// 32-bit key whose unsigned order is the IEEE total order of the float
// (-0 < +0): negative values get every bit flipped, positive ones the sign bit.
__device__ __forceinline__ uint32_t f2key(float v) {
  uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
  uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(b);
}

// Asynchronous global -> shared copies (no register staging).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Position of the (r+1)-th set bit of x (r = 0 for the lowest), r < popc(x):
// bisection on the popcounts of the low 16, 8, 4, 2 and 1 bits.
__device__ __forceinline__ int nth_set(uint32_t x, int r) {
  int pos = 0, c;
  c = __popc(x & 0xffffu);
  if (r >= c) { r -= c; x >>= 16; pos += 16; }
  c = __popc(x & 0xffu);
  if (r >= c) { r -= c; x >>= 8; pos += 8; }
  c = __popc(x & 0xfu);
  if (r >= c) { r -= c; x >>= 4; pos += 4; }
  c = __popc(x & 0x3u);
  if (r >= c) { r -= c; x >>= 2; pos += 2; }
  if (r >= (int)(x & 1u)) pos += 1;
  return pos;
}

// 32 x 32 bit transpose across a warp: on entry lane b holds row b; on exit
// lane c holds the word whose bit b is bit c of row b.  Five butterfly
// stages, each swapping the off-diagonal blocks of size s between lanes
// that differ in bit s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const uint32_t m = (s == 16) ? 0x0000ffffu : (s == 8) ? 0x00ff00ffu : (s == 4) ? 0x0f0f0f0fu
                       : (s == 2) ? 0x33333333u : 0x55555555u;
    const uint32_t y = __shfl_xor_sync(FULL, x, s);
    // lane with bit s clear keeps its low blocks and takes the partner's low
    // blocks shifted up; the other keeps its high blocks and takes the
    // partner's high blocks shifted down
    x = (lane & s) ? ((x & ~m) | ((y >> s) & m)) : ((x & m) | ((y << s) & ~m));
  }
  return x;
}

// Exclusive prefix over a warp-private 256-bin histogram (8 bins per lane),
// in place.  Returns nothing; hist[d] becomes the number of keys with digit < d.
__device__ __forceinline__ void hist_exclusive_scan(uint32_t *hist, int lane) {
  uint32_t h[8], s = 0;
#pragma unroll
  for (int b = 0; b < 8; b++) {
    h[b] = hist[lane * 8 + b];
    s += h[b];
  }
  uint32_t inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += t;
  }
  uint32_t acc = inc - s;
#pragma unroll
  for (int b = 0; b < 8; b++) {
    hist[lane * 8 + b] = acc;
    acc += h[b];
  }
}

// Given a filled histogram and a rank krem, find digit d with
// below(d) <= krem < below(d) + hist[d]; returns d, below(d), hist[d].
__device__ __forceinline__ void hist_find(const uint32_t *hist, uint32_t krem, int lane, uint32_t &d,
                                          uint32_t &below, uint32_t &cnt) {
  uint32_t h[8], s = 0;
#pragma unroll
  for (int b = 0; b < 8; b++) {
    h[b] = hist[lane * 8 + b];
    s += h[b];
  }
  uint32_t inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += t;
  }
  const uint32_t exc = inc - s;
  const unsigned ball = __ballot_sync(FULL, inc > krem);
  const int L = __ffs(ball) - 1;
  uint32_t dd = 0, bb = 0, cc = 0;
  if (lane == L) {
    uint32_t acc = exc;
    bool done = false;
#pragma unroll
    for (int b = 0; b < 8; b++) {
      if (!done && acc + h[b] > krem) {
        dd = lane * 8 + b;
        bb = acc;
        cc = h[b];
        done = true;
      }
      acc += h[b];
    }
  }
  d = __shfl_sync(FULL, dd, L);
  below = __shfl_sync(FULL, bb, L);
  cnt = __shfl_sync(FULL, cc, L);
}


// Exact radix selects of the elements of full ranks r_lo <= r_hi among the T
// keys keys[s * STRIDE] (s < T), sharing each histogram pass while both
// prefixes agree: returns their keys and the numbers of smaller keys.
// Histograms use fire-and-forget shared-memory reductions (no dependency
// chain); digits equal in every key are skipped.
template <int STRIDE>
__device__ __forceinline__ void band_select2(const uint32_t *keys, int T, uint32_t r_lo, uint32_t r_hi,
                                             uint32_t varying, uint32_t andv, uint32_t *hlo, uint32_t *hhi,
                                             int lane, uint32_t &Klo, uint32_t &clt_lo, uint32_t &Khi,
                                             uint32_t &clt_hi) {
  uint32_t plo = 0, phi = 0, pmask = 0, klo = r_lo, khi = r_hi;
#pragma unroll 1
  for (int pass = 0; pass < 4; pass++) {
    const int shift = 24 - 8 * pass;
    if (((varying >> shift) & 255u) == 0) {
      plo |= andv & (0xffu << shift);
      phi |= andv & (0xffu << shift);
      pmask |= 0xffu << shift;
      continue;
    }
    const bool same = (plo == phi);
#pragma unroll
    for (int b = 0; b < 8; b++) {
      hlo[lane * 8 + b] = 0;
      hhi[lane * 8 + b] = 0;
    }
    __syncwarp();
#pragma unroll 4
    for (int s = lane; s < T; s += 32) {
      const uint32_t key = keys[s * STRIDE];
      const uint32_t d = (key >> shift) & 255u;
      const uint32_t km = key & pmask;
      if (km == plo) atomicAdd(&hlo[d], 1u);
      if (!same && km == phi) atomicAdd(&hhi[d], 1u);
    }
    __syncwarp();
    uint32_t d, below, cnt;
    hist_find(hlo, klo, lane, d, below, cnt);
    plo |= d << shift;
    klo -= below;
    hist_find(same ? hlo : hhi, khi, lane, d, below, cnt);
    phi |= d << shift;
    khi -= below;
    pmask |= 0xffu << shift;
    __syncwarp();
  }
  Klo = plo;
  clt_lo = r_lo - klo;
  Khi = phi;
  clt_hi = r_hi - khi;
}

}  // namespace
}  // namespace graphic

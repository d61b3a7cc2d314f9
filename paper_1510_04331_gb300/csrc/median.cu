// median.cu -- angle-gated median PSF subtraction (Sect. 3.3) and median
// collapse (Sect. 3.4) on sm_103a.
//
// The kernels work in the paper's "spatial" data-parallel scheme: a CTA
// owns consecutive pixels of every frame, one warp per pixel (8 for the
// general median path, whose CTA reads a 32-byte sector per frame; 4 for the
// collapse, a 16-byte row per frame).  Values are compared as 32-bit IEEE
// total-order keys (negative: all bits flipped, positive: sign bit set), so
// selection is exact and bit-reproducible.
//
// PSF subtraction.  Frames are visited in angle order s (perm[s] = frame).
// For frame s the reference set is the sorted positions [0, L_s) u [R_s, T)
// (host plan, FP64 gate).  Per pixel the warp
//   1. sorts the T keys with a stable LSD radix sort (8-bit digits, digits
//      that are equal in every key are skipped), giving the sorted keys and
//      rank[s], the sorted position of frame s;
//   2. splits the T queries into 32 contiguous chunks, one per lane, builds
//      each chunk's starting membership bitmap over sorted positions (lane
//      0's chunk by ballots, the others by XOR-toggling the frames whose
//      membership changes between chunk starts), and
//   3. lets every lane sweep its chunk: per query it toggles the bits of the
//      frames entering/leaving the set and walks a pointer to the k-th set
//      bit (k = (|S| - 1) / 2), the median being that key (or the mean of it
//      and the next set bit's key, in FP32, for even |S|).
// Collapse.  Per pixel, a value-linear histogram over a sampled range
// locates the two middle ranks, read off a short candidate list
// (collapse2_kernel); radix selects (8-bit digits) are its exact fallback and
// the masked (master sky) and long-cube form (collapse_kernel).
#include <cuda_runtime.h>
#include <type_traits>
#include <stdint.h>

#include "graphic_internal.h"
#include "select_common.cuh"

namespace graphic {
namespace {

constexpr uint32_t NOTAG = 0xffffffffu;

__device__ __forceinline__ int annulus_of(long long p, int n, const double *edge2, int n_ann) {
  const long long x = (p % n) - n / 2, y = (p / n) - n / 2;
  const double rho2 = (double)(x * x + y * y);
  for (int a = 0; a < n_ann; a++)
    if (edge2[a] <= rho2 && rho2 < edge2[a + 1]) return a;
  return -1;
}

// ---------------------------------------------------------------------------
// Median collapse
// ---------------------------------------------------------------------------

// One warp per pixel, COL_PPC pixels per CTA.  Keys in shared memory are
// frame-major with an odd row stride (COL_KS words), so a warp reading its
// pixel's keys of 32 consecutive frames hits 32 distinct banks.  Radix
// select of the lower median: 8-bit digits, most significant first, digits
// constant over the pixel's keys skipped, histograms by shared-memory
// reductions.
constexpr int COL_PPC = 4;
constexpr int COL_KS = 5;
// collapse2_kernel: words per frame row (one 16-byte copy per frame; a
// warp's column reads meet 4-way bank conflicts, cheaper here than four
// 4-byte copies per frame)
constexpr int C2_KS = 4;

// MASKED (master sky, Sect. 3.2): values that are not finite or fall in the
// frame's star mask are left out -- they get the largest key, so they rank
// after every value kept -- and the median is taken over the m values kept
// (NaN when m = 0).
template <bool SMEM, bool MASKED = false>
__global__ void __launch_bounds__(32 * COL_PPC) collapse_kernel(const CollapseArgs a) {
  extern __shared__ uint32_t csm[];
  uint32_t *hist_all = csm;                       // [COL_PPC][256]
  uint32_t *keys_all = csm + COL_PPC * 256;       // [T][COL_KS] (SMEM only)
  const long long T = a.T;
  const long long NN = a.fs ? a.fs : (long long)a.n * a.n;   // frame stride
  const long long p0 = (long long)blockIdx.x * COL_PPC;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;

  bool bad = false;
  if constexpr (SMEM) {
    for (long long j = threadIdx.x; j < COL_PPC * T; j += 32 * COL_PPC) {
      const long long t = j / COL_PPC;
      const int q = (int)(j - t * COL_PPC);
      cp_async4(keys_all + t * COL_KS + q, a.in + t * NN + p0 + q);
    }
    cp_async_wait_all();
    __syncthreads();
  }
  uint32_t *hist = hist_all + w * 256;
  const long long p = p0 + w;
  // masked-out values (MASKED) get the largest key
  auto key_of = [&](long long t, float v) -> uint32_t {
    if constexpr (MASKED) {
      bool keep = isfinite(v);
      if (a.mask_x) {
        const double ddx = (double)(p % a.n) - a.mask_x[t], ddy = (double)(p / a.n) - a.mask_y[t];
        keep &= !(ddx * ddx + ddy * ddy < a.mask_r2);
      }
      return keep ? f2key(v) : 0xffffffffu;
    } else {
      return f2key(v);
    }
  };
  auto key_at = [&](long long t) -> uint32_t {
    if constexpr (SMEM) return keys_all[t * COL_KS + w];
    else return key_of(t, a.in[t * NN + p]);
  };
  // keys in place (each warp converts its own pixel), finiteness, and the
  // digits shared by every key
  uint32_t orv = 0, andv = 0xffffffffu;
  int kept = 0;
  for (long long t = lane; t < T; t += 32) {
    float v;
    if constexpr (SMEM) v = __uint_as_float(keys_all[t * COL_KS + w]);
    else v = a.in[t * NN + p];
    const uint32_t key = key_of(t, v);
    if constexpr (MASKED) kept += (key != 0xffffffffu) ? 1 : 0;
    else bad |= !isfinite(v);
    if constexpr (SMEM) keys_all[t * COL_KS + w] = key;
    orv |= key;
    andv &= key;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    orv |= __shfl_xor_sync(FULL, orv, o);
    andv &= __shfl_xor_sync(FULL, andv, o);
  }
  const bool anybad = __any_sync(FULL, bad);
  if (anybad && lane == 0) atomicOr(a.status, STATUS_NONFINITE);
  __syncwarp();
  const uint32_t varying = orv ^ andv;

  long long m = T;
  if constexpr (MASKED) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(FULL, kept, o);
    m = kept;
    if (m == 0) {
      if (lane == 0) a.out[p] = __uint_as_float(0x7fc00000u);   // no value left: NaN
      return;
    }
  }
  const uint32_t k = (uint32_t)((m - 1) / 2);
  uint32_t prefix = 0, pmask = 0, krem = k, cnt = (uint32_t)T;
  // Candidate list: the pass in which at most `cap` keys still match the
  // prefix also copies them (in frame order) into the row padding words
  // (word COL_KS - 1 of rows [w cap, (w + 1) cap), which no key uses), and
  // the later passes read only the list.
  const int cap = SMEM ? (int)(T / COL_PPC < 128 ? T / COL_PPC : 128) : 0;
  uint32_t *cbuf = keys_all + (long long)w * cap * COL_KS + (COL_KS - 1);   // element j at cbuf[j * COL_KS]
  int nc = -1;                                                            // list length, -1: none yet
  const unsigned lt = (1u << lane) - 1u;
  for (int pass = 0; pass < 4; pass++) {
    const int shift = 24 - 8 * pass;
    if (((varying >> shift) & 255u) == 0) {   // every key has this digit
      prefix |= andv & (0xffu << shift);
      pmask |= 0xffu << shift;
      continue;
    }
#pragma unroll
    for (int b = 0; b < 8; b++) hist[lane * 8 + b] = 0;
    __syncwarp();
    if (nc >= 0) {
      for (int j = lane; j < nc; j += 32) {
        const uint32_t key = cbuf[j * COL_KS];
        if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
      }
    } else if (cnt <= (uint32_t)cap) {
      int len = 0;
      for (long long t0 = 0; t0 < T; t0 += 32) {
        const long long t = t0 + lane;
        const uint32_t key = t < T ? key_at(t) : 0u;
        const bool match = t < T && (key & pmask) == prefix;
        const unsigned mm = __ballot_sync(FULL, match);
        if (match) {
          cbuf[(len + __popc(mm & lt)) * COL_KS] = key;
          atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        len += __popc(mm);
      }
      nc = len;
    } else {
#pragma unroll 4
      for (long long t = lane; t < T; t += 32) {
        const uint32_t key = key_at(t);
        if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
      }
    }
    __syncwarp();
    uint32_t d, below;
    hist_find(hist, krem, lane, d, below, cnt);
    prefix |= d << shift;
    pmask |= 0xffu << shift;
    krem -= below;
    __syncwarp();
  }
  const float lo = key2f(prefix);
  float med = lo;
  if ((m & 1) == 0) {
    uint32_t hi = prefix;
    if (krem + 1 >= cnt) {
      // smallest key greater than the lower median: from the candidate list
      // when it holds one (the list's bucket is a contiguous key range, so a
      // larger key inside it beats every key above it), else from all keys
      uint32_t mn = 0xffffffffu;
      if (nc >= 0) {
        for (int j = lane; j < nc; j += 32) {
          const uint32_t key = cbuf[j * COL_KS];
          if (key > prefix && key < mn) mn = key;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(FULL, mn, o));
      }
      if (nc < 0 || mn == 0xffffffffu) {
        mn = 0xffffffffu;
        for (long long t = lane; t < T; t += 32) {
          const uint32_t key = key_at(t);
          if (key > prefix && key < mn) mn = key;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(FULL, mn, o));
      }
      hi = mn;
    }
    med = (lo + key2f(hi)) * 0.5f;
  }
  if (lane == 0) a.out[p] = med;
}

// Median collapse of unmasked cubes that fit shared memory.  Per pixel
// (one warp): the values in shared memory, one 16-byte row of the CTA's 4
// pixels per frame.
// A 256-bin histogram linear in value over the interquartile range of 32
// sampled frames (values outside it counted below or ignored above), filled
// in one pass over the raw values, locates the bins of the two middle
// ranks; a second pass copies the total-order keys of those bins (a few
// values) into the warp's second 256 histogram words, and the middle ranks
// are read off by counting within that list.  A middle rank outside the
// range, a list longer than 256 keys (many equal values) or a non-finite
// value falls back to exact radix selects of the two middle ranks over all
// keys.
__global__ void __launch_bounds__(32 * COL_PPC, 5) collapse2_kernel(const CollapseArgs a) {
  extern __shared__ uint32_t csm[];
  uint32_t *hist_all = csm;                       // [COL_PPC][512]
  uint32_t *keys_all = csm + COL_PPC * 512;       // [T][C2_KS]
  const int T = (int)a.T;
  const long long NN = a.fs ? a.fs : (long long)a.n * a.n;   // frame stride
  const long long p0 = (long long)blockIdx.x * COL_PPC;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < T; t += 32 * COL_PPC) cp_async16(keys_all + t * C2_KS, a.in + (long long)t * NN + p0);
  cp_async_wait_all();
  __syncthreads();
  uint32_t *hist = hist_all + w * 512;
  uint32_t *kw = keys_all + w;   // value (then key) of frame t: kw[t * C2_KS]
  const uint32_t k0 = (uint32_t)((T - 1) / 2);
  const bool even = (T & 1) == 0;
  const uint32_t k1 = even ? k0 + 1 : k0;
  // histogram range: the interquartile range of 32 frames sampled evenly in
  // time (bitonic sort across the warp; the min and max of the sample when
  // the quartiles coincide).  The median lies between the sample's quartiles
  // unless fewer than 9 or more than 23 of the 32 sampled values fall below
  // it (well under 1 % of pixels when frames vary independently); then, as
  // for a range the sample missed, the exact path below takes over.
  float lo = 0.f, scale = 0.f;
  if (T >= 32) {
    float x = __uint_as_float(kw[(int)(((long long)lane * T) >> 5) * C2_KS]);
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int d = k >> 1; d > 0; d >>= 1) {
        const float y = __shfl_xor_sync(FULL, x, d);
        const bool up = (lane & k) == 0, low = (lane & d) == 0;
        x = (up == low) ? fminf(x, y) : fmaxf(x, y);
      }
    }
    float qlo = __shfl_sync(FULL, x, 8), qhi = __shfl_sync(FULL, x, 23);
    if (!(qhi > qlo)) {
      qlo = __shfl_sync(FULL, x, 0);
      qhi = __shfl_sync(FULL, x, 31);
    }
    const float sc = 256.f / (qhi - qlo);
    if (qhi > qlo && sc <= 3.4e38f) {   // finite range and scale
      lo = qlo;
      scale = sc;
    }
  }
  // one pass over the raw values: x = (v - lo) scale is monotone in v;
  // x < 0 counts below the range, [0, 256) takes bin (int) x, the rest is
  // above.  (scale = 0 puts every finite value in bin 0.)  The finiteness
  // check rides along.
#pragma unroll
  for (int b = 0; b < 8; b++) hist[lane * 8 + b] = 0u;
  __syncwarp();
  bool bad = false;
  uint32_t nb = 0;
#pragma unroll 4
  for (int t = lane; t < T; t += 32) {
    const float v = __uint_as_float(kw[t * C2_KS]);
    bad |= !isfinite(v);
    const float xv = (v - lo) * scale;
    if (xv < 0.f) nb++;
    else if (xv < 256.f) atomicAdd(&hist[(int)xv], 1u);
  }
  const bool anybad = __any_sync(FULL, bad);
  if (anybad && lane == 0) atomicOr(a.status, STATUS_NONFINITE);
  const uint32_t nbelow = __reduce_add_sync(FULL, nb);
  __syncwarp();
  uint32_t h[8], hs = 0;
#pragma unroll
  for (int b = 0; b < 8; b++) {
    h[b] = hist[lane * 8 + b];
    hs += h[b];
  }
  uint32_t inc = hs;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t tt = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += tt;
  }
  const uint32_t inside = __shfl_sync(FULL, inc, 31);
  // bins of ranks k0 and k1 (ranks within the range: k - nbelow) and the
  // values below them; a rank outside the range takes the exact path
  const bool in_range = k0 >= nbelow && k1 - nbelow < inside;
  int bin[2] = {0, 0};
  uint32_t bel[2] = {0u, 0u};
  if (in_range) {
#pragma unroll
    for (int q = 0; q < 2; q++) {
      const uint32_t r = (q ? k1 : k0) - nbelow;
      const unsigned ball = __ballot_sync(FULL, inc > r);
      const int L = __ffs(ball) - 1;
      int bb = 0;
      uint32_t be = 0;
      if (lane == L) {
        uint32_t acc = inc - hs;
        bool done = false;
#pragma unroll
        for (int b = 0; b < 8; b++) {
          if (!done && acc + h[b] > r) {
            bb = lane * 8 + b;
            be = acc;
            done = true;
          }
          acc += h[b];
        }
      }
      bin[q] = __shfl_sync(FULL, bb, L);
      bel[q] = __shfl_sync(FULL, be, L) + nbelow;
    }
  }
  const int nlist = in_range ? (int)(bel[1] + hist[bin[1]] - bel[0]) : 0x7fffffff;
  // the list lives in the warp's second 256 histogram words
  const int cap = min(T, 256);
  float med;
  if (!anybad && nlist <= cap) {
    uint32_t *cbuf = hist + 256;   // element j at cbuf[j] (the second histogram's words)
    const unsigned lt = (1u << lane) - 1u;
    int len = 0;
    // four 32-frame rounds per step: their loads and bins are independent;
    // the list holds total-order keys.  Bins bin0 .. bin1 of x >= 0 are the
    // x in [bin0, bin1 + 1) (truncation is the floor there; -0 is in bin 0).
    const float xlo = (float)bin[0], xhi = (float)(bin[1] + 1);
    for (int t0 = 0; t0 < T; t0 += 128) {
      float v[4];
      bool in[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int t = t0 + 32 * u + lane;
        v[u] = t < T ? __uint_as_float(kw[t * C2_KS]) : 0.f;
        const float xv = (v[u] - lo) * scale;
        in[u] = t < T && xv >= xlo && xv < xhi;
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const unsigned mm = __ballot_sync(FULL, in[u]);
        if (in[u]) cbuf[len + __popc(mm & lt)] = f2key(v[u]);
        len += __popc(mm);
      }
    }
    __syncwarp();
    // ranks r0, r1 within the list: the key with (#smaller) <= r < (#smaller or equal)
    const uint32_t r0 = k0 - bel[0], r1 = k1 - bel[0];
    uint32_t f0 = 0xffffffffu, f1 = 0xffffffffu;
    for (int j = lane; j < len; j += 32) {
      const uint32_t kj = cbuf[j];
      uint32_t nlt = 0, nle = 0;
      for (int x = 0; x < len; x++) {
        const uint32_t kx = cbuf[x];
        nlt += kx < kj ? 1u : 0u;
        nle += kx <= kj ? 1u : 0u;
      }
      if (nlt <= r0 && r0 < nle) f0 = kj;
      if (nlt <= r1 && r1 < nle) f1 = kj;
    }
    f0 = __reduce_min_sync(FULL, f0);
    f1 = __reduce_min_sync(FULL, f1);
    med = even ? (key2f(f0) + key2f(f1)) * 0.5f : key2f(f0);
  } else {
    // exact: keys in place, then radix selects of the two middle ranks
    uint32_t orv = 0u, andv = 0xffffffffu;
    for (int t = lane; t < T; t += 32) {
      const uint32_t k = f2key(__uint_as_float(kw[t * C2_KS]));
      kw[t * C2_KS] = k;
      orv |= k;
      andv &= k;
    }
    orv = __reduce_or_sync(FULL, orv);
    andv = __reduce_and_sync(FULL, andv);
    __syncwarp();
    uint32_t Klo, Khi, clo, chi;
    band_select2<C2_KS>(kw, T, k0, k1, orv ^ andv, andv, hist, hist + 256, lane, Klo, clo, Khi, chi);
    med = even ? (key2f(Klo) + key2f(Khi)) * 0.5f : key2f(Klo);
  }
  if (lane == 0) a.out[p0 + w] = med;
}

// ---------------------------------------------------------------------------
// Angle-gated median PSF subtraction
// ---------------------------------------------------------------------------

__device__ __forceinline__ int next_set(const uint32_t *bm, int c, int x, int nw) {
  int wd = x >> 5;
  if (wd >= nw) return -1;
  uint32_t word = bm[wd * 32 + c] & (0xffffffffu << (x & 31));
  while (word == 0) {
    if (++wd >= nw) return -1;
    word = bm[wd * 32 + c];
  }
  return wd * 32 + __ffs(word) - 1;
}

__device__ __forceinline__ int prev_set(const uint32_t *bm, int c, int x) {
  if (x < 0) return -1;
  int wd = x >> 5;
  uint32_t word = bm[wd * 32 + c] & (0xffffffffu >> (31 - (x & 31)));
  while (word == 0) {
    if (--wd < 0) return -1;
    word = bm[wd * 32 + c];
  }
  return wd * 32 + 31 - __clz(word);
}

__global__ void __launch_bounds__(256, 1) adi_median_kernel(const AdiArgs a, int tcap) {
  extern __shared__ uint32_t asm_[];
  uint32_t *hist_all = asm_;                                   // [8][256]
  uint32_t *kA_all = hist_all + 8 * 256;                       // [8][tcap]
  uint32_t *kB_all = kA_all + 8 * tcap;                        // [8][tcap]
  uint16_t *iA_all = reinterpret_cast<uint16_t *>(kB_all + 8 * tcap);   // [8][tcap]
  uint16_t *iB_all = iA_all + 8 * tcap;                                  // [8][tcap]
  uint16_t *perm_s = iB_all + 8 * tcap;                                  // [tcap]
  __shared__ int ann_s[8];

  const int T = a.T;
  const long long p0 = (long long)(a.gen_list ? __ldg(&a.groups[a.gen_off + blockIdx.x]) : (int)blockIdx.x) * 8;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = tcap / 32;   // bitmap words per lane column

  if (lane == 0) ann_s[w] = annulus_of(p0 + w, a.n, a.edge2, a.n_ann);
  for (int s = threadIdx.x; s < T; s += 256) perm_s[s] = (uint16_t)__ldg(&a.perm[s]);
  __syncthreads();
  // a 4-pixel group whose annuli all have a band (or no annulus) belongs to
  // the band path (psf_band.cu), which runs after this kernel
  bool banded[2];
#pragma unroll
  for (int g = 0; g < 2; g++) {
    bool b = a.wmax > 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int an = ann_s[4 * g + q];
      b &= (an < 0) || (__ldg(&a.band[4 * an + 2]) > 0);
    }
    banded[g] = b;
  }
  if (banded[0] && banded[1]) return;
  bool any = false;
#pragma unroll
  for (int q = 0; q < 8; q++) any |= ann_s[q] >= 0;
  bool bad = false;
  if (any) {
    // all T x 8 values in flight at once: two 16-byte copies per frame into
    // a frame-major staging area (the kB buffer), then keys into kA, rows
    // per pixel
    float *stage = reinterpret_cast<float *>(kB_all);
    for (int j = threadIdx.x; j < 2 * T; j += 256) {
      const int s = j >> 1, h = j & 1;
      cp_async16(stage + s * 8 + 4 * h, a.in + (long long)perm_s[s] * a.in_fs + p0 + 4 * h);
    }
    cp_async_wait_all();
    __syncthreads();
#pragma unroll 1
    for (int pw = 0; pw < 8; pw++) {
      for (int s = threadIdx.x; s < T; s += 256) {
        const float v = stage[s * 8 + pw];
        bad |= !isfinite(v);
        kA_all[pw * tcap + s] = f2key(v);
        iA_all[pw * tcap + s] = (uint16_t)s;
      }
    }
  }
  if (bad) atomicOr(a.status, STATUS_NONFINITE);
  __syncthreads();

  const int ann = ann_s[w];
  const long long p = p0 + w;
  if (banded[w >> 2]) return;
  if (ann < 0) {
    for (int i = lane; i < T; i += 32) a.out[(long long)perm_s[i] * a.out_fs + p] = 0.0f;
    return;
  }
  uint32_t *hist = hist_all + w * 256;
  uint32_t *sk = kA_all + w * tcap, *dk = kB_all + w * tcap;
  uint16_t *si = iA_all + w * tcap, *di = iB_all + w * tcap;

  // ---- 1. stable LSD radix sort of (key, frame) --------------------------
  uint32_t orv = 0, andv = 0xffffffffu;
  for (int i = lane; i < T; i += 32) {
    orv |= sk[i];
    andv &= sk[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    orv |= __shfl_xor_sync(FULL, orv, o);
    andv &= __shfl_xor_sync(FULL, andv, o);
  }
  const uint32_t varying = orv ^ andv;
  for (int pass = 0; pass < 4; pass++) {
    const int shift = 8 * pass;
    if (((varying >> shift) & 255u) == 0) continue;   // equal digit in every key
#pragma unroll
    for (int b = 0; b < 8; b++) hist[lane * 8 + b] = 0;
    __syncwarp();
    for (int base = 0; base < T; base += 32) {
      const int i = base + lane;
      const uint32_t tag = (i < T) ? ((sk[i] >> shift) & 255u) : NOTAG;
      const unsigned peers = __match_any_sync(FULL, tag);
      if (tag != NOTAG && lane == __ffs(peers) - 1) hist[tag] += __popc(peers);
      __syncwarp();
    }
    hist_exclusive_scan(hist, lane);
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    for (int base = 0; base < T; base += 32) {
      const int i = base + lane;
      uint32_t key = 0, tag = NOTAG;
      uint16_t fi = 0;
      if (i < T) {
        key = sk[i];
        fi = si[i];
        tag = (key >> shift) & 255u;
      }
      const unsigned peers = __match_any_sync(FULL, tag);
      uint32_t off = 0;
      if (tag != NOTAG) {
        off = hist[tag];
        const int pos = (int)off + __popc(peers & lt);
        dk[pos] = key;
        di[pos] = fi;
      }
      __syncwarp();
      if (tag != NOTAG && lane == __ffs(peers) - 1) hist[tag] = off + __popc(peers);
      __syncwarp();
    }
    uint32_t *tk = sk; sk = dk; dk = tk;
    uint16_t *ti = si; si = di; di = ti;
  }
  // sk: sorted keys, si: frame (sorted angle position) at each sorted
  // position.  rank[s] goes to di, bitmaps to dk.
  uint16_t *rk = di;
  uint32_t *bm = dk;
  for (int pos = lane; pos < T; pos += 32) rk[si[pos]] = (uint16_t)pos;
  __syncwarp();

  // ---- 2. chunk-start membership bitmaps ---------------------------------
  // Frame s (angle order) is in the set of query i when it lies in the time
  // window [A_i, B_i) and outside the excluded range [L_i, R_i) (which lies
  // inside the window): the XOR of two range indicators, so moving any of
  // the four boundaries toggles exactly the frames it passes over.
  const int *LR = a.lr + (size_t)ann * T * 2;
  const int2 *AB2 = reinterpret_cast<const int2 *>(a.ab);
  auto window = [&](int i) -> int2 { return AB2 ? __ldg(&AB2[i]) : make_int2(0, T); };
  const int C = (T + 31) / 32;
  {
    const int L0 = __ldg(&LR[0]), R0 = __ldg(&LR[1]);
    const int2 W0 = window(0);
    for (int wd = 0; wd < nw; wd++) {
      const int pos = wd * 32 + lane;
      bool mem = false;
      if (pos < T) {
        const int s = si[pos];
        mem = (s >= W0.x && s < W0.y) && ((s < L0) || (s >= R0));
      }
      const unsigned word = __ballot_sync(FULL, mem);
      if (lane == 0) bm[wd * 32] = word;
    }
    __syncwarp();
    int Lp = L0, Rp = R0, Ap = W0.x, Bp = W0.y;
    for (int c = 1; c < 32; c++) {
      const int i0 = c * C;
      if (i0 >= T) break;
      const int Lc = __ldg(&LR[2 * i0]), Rc = __ldg(&LR[2 * i0 + 1]);
      const int2 Wc = window(i0);
      for (int wd = lane; wd < nw; wd += 32) bm[wd * 32 + c] = bm[wd * 32 + c - 1];
      __syncwarp();
      const int lo[4] = {min(Lp, Lc), min(Rp, Rc), min(Ap, Wc.x), min(Bp, Wc.y)};
      const int hi[4] = {max(Lp, Lc), max(Rp, Rc), max(Ap, Wc.x), max(Bp, Wc.y)};
      for (int q = 0; q < 4; q++)
        for (int s = lo[q] + lane; s < hi[q]; s += 32) {
          const int r = rk[s];
          atomicXor(&bm[(r >> 5) * 32 + c], 1u << (r & 31));
        }
      __syncwarp();
      Lp = Lc;
      Rp = Rc;
      Ap = Wc.x;
      Bp = Wc.y;
    }
  }

  // ---- 3. per-lane sweep over its chunk of queries -----------------------
  const int c = lane;
  const int i0 = c * C;
  const int i1 = min(T, i0 + C);
  bool fail = false;
  if (i0 < T) {
    int L = __ldg(&LR[2 * i0]), R = __ldg(&LR[2 * i0 + 1]);
    int2 W = window(i0);
    int nset = (W.y - W.x) - (R - L);
    int k = (nset - 1) >> 1;
    int pos = -1, acc = 0;
    for (int wd = 0; wd < nw; wd++) {
      const uint32_t word = bm[wd * 32 + c];
      const int pc = __popc(word);
      if (acc + pc > k) {
        pos = wd * 32 + nth_set(word, k - acc);
        break;
      }
      acc += pc;
    }
    int below = k;
    if (pos < 0) fail = true;
    const int2 *LR2 = reinterpret_cast<const int2 *>(LR);
    int2 nxt = __ldg(&LR2[i0]);
    for (int i = i0; i < i1 && !fail; i++) {
      const int Ln = nxt.x, Rn = nxt.y;
      const int2 Wn = window(i);
      if (i + 1 < i1) nxt = __ldg(&LR2[i + 1]);
      // toggle frames whose membership changes; keep `below` = set bits < pos
      const int npass = AB2 ? 4 : 2;
      for (int pass = 0; pass < npass; pass++) {
        const int s0 = pass == 0 ? min(L, Ln) : pass == 1 ? min(R, Rn) : pass == 2 ? min(W.x, Wn.x) : min(W.y, Wn.y);
        const int s1 = pass == 0 ? max(L, Ln) : pass == 1 ? max(R, Rn) : pass == 2 ? max(W.x, Wn.x) : max(W.y, Wn.y);
        for (int s = s0; s < s1; s++) {
          const int r = rk[s];
          uint32_t *wp = &bm[(r >> 5) * 32 + c];
          const uint32_t bit = 1u << (r & 31);
          const uint32_t nwv = *wp ^ bit;
          *wp = nwv;
          if (r < pos) below += (nwv & bit) ? 1 : -1;
        }
      }
      L = Ln;
      R = Rn;
      W = Wn;
      nset = (W.y - W.x) - (R - L);
      k = (nset - 1) >> 1;
      // walk the pointer to the k-th set bit
      for (int guard = 0; guard < 4 * 2048 + 8; guard++) {
        const bool set = (bm[(pos >> 5) * 32 + c] >> (pos & 31)) & 1u;
        if (below == k && set) break;
        if (below < k || (below == k && !set)) {
          if (set) below++;
          pos = next_set(bm, c, pos + 1, nw);
        } else {
          pos = prev_set(bm, c, pos - 1);
          below--;
        }
        if (pos < 0) {
          fail = true;
          break;
        }
      }
      if (fail) break;
      float med = key2f(sk[pos]);
      if ((nset & 1) == 0) {
        const int hp = next_set(bm, c, pos + 1, nw);
        if (hp < 0) {
          fail = true;
          break;
        }
        med = (med + key2f(sk[hp])) * 0.5f;
      }
      const float v = key2f(sk[rk[i]]);
      a.out[(long long)perm_s[i] * a.out_fs + p] = v - med;
    }
  }
  if (fail) atomicOr(a.status, STATUS_INTERNAL);
}

int pow2_at_least(long long x, int lo) {
  int v = lo;
  while (v < x) v <<= 1;
  return v;
}

}  // namespace

cudaError_t launch_adi_general(const AdiArgs &a, cudaStream_t st, int tcap);

cudaError_t launch_collapse(const CollapseArgs &a, cudaStream_t st) {
  const long long NN = (long long)a.n * a.n;
  const unsigned grid = (unsigned)(NN / COL_PPC);
  const long long fs = a.fs ? a.fs : NN;
  const bool rows16 = ((uintptr_t)a.in & 15) == 0 && (fs & 3) == 0;   // 16-byte frame rows of 4 pixels
  if (a.T <= 8192 && rows16) {
    const size_t smem = (size_t)(COL_PPC * 512 + C2_KS * a.T) * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(collapse2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    collapse2_kernel<<<grid, 32 * COL_PPC, smem, st>>>(a);
  } else if (a.T <= 8192) {
    const size_t smem = (size_t)(COL_PPC * 256 + COL_KS * a.T) * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(collapse_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    collapse_kernel<true><<<grid, 32 * COL_PPC, smem, st>>>(a);
  } else {
    const size_t smem = (size_t)(COL_PPC * 256) * sizeof(uint32_t);
    collapse_kernel<false><<<grid, 32 * COL_PPC, smem, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_sky_median(const CollapseArgs &a, cudaStream_t st) {
  const long long NN = (long long)a.n * a.n;
  const unsigned grid = (unsigned)(NN / COL_PPC);
  if (a.T <= 8192) {
    const size_t smem = (size_t)(COL_PPC * 256 + COL_KS * a.T) * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(collapse_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    collapse_kernel<true, true><<<grid, 32 * COL_PPC, smem, st>>>(a);
  } else {
    const size_t smem = (size_t)(COL_PPC * 256) * sizeof(uint32_t);
    collapse_kernel<false, true><<<grid, 32 * COL_PPC, smem, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_adi_median(const AdiArgs &a, cudaStream_t st, int *launched) {
  int dummy = 0;
  int &nl = launched ? *launched : dummy;
  nl = 0;
  const int tcap = pow2_at_least(a.T, 32);
  // general kernel first: it reads every pixel of its 8-pixel groups and
  // writes only the 4-pixel halves that are not on the band path; the band
  // path's groups (psf_band.cu) are disjoint from those halves
  if (a.mark) a.mark(a.mark_user, 0, 1);
  cudaError_t e = launch_adi_general(a, st, tcap);
  if (a.mark) a.mark(a.mark_user, 0, 0);
  nl += (e == cudaSuccess && (!a.gen_list || a.gen_n > 0));
  if (e != cudaSuccess || a.wmax == 0) return e;
  return launch_adi_band(a, st, &nl);
}

cudaError_t launch_adi_general(const AdiArgs &a, cudaStream_t st, int tcap) {
  const long long NN = (long long)a.n * a.n;
  const size_t smem = (size_t)8 * 256 * sizeof(uint32_t) +
                      (size_t)8 * tcap * (2 * sizeof(uint32_t) + 2 * sizeof(uint16_t)) + (size_t)tcap * sizeof(uint16_t);
  // the plan lists the blocks with a pixel of an annulus without a band
  // (every other block would read its annuli and exit, one CTA per SM at a
  // time for this kernel's shared memory)
  const long long nblk = a.gen_list ? a.gen_n : NN / 8;
  if (nblk == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(adi_median_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  adi_median_kernel<<<(unsigned)nblk, 256, smem, st>>>(a, tcap);
  return cudaGetLastError();
}

}  // namespace graphic

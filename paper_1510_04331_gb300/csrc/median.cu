// median.cu -- angle-gated median PSF subtraction (Sect. 3.3) and median
// collapse (Sect. 3.4) on sm_103a.
//
// Both kernels work in the paper's "spatial" data-parallel scheme: a CTA of
// 8 warps owns 8 consecutive pixels of every frame (one warp per pixel) and
// reads, per frame, those 8 pixels as one 32-byte sector.  Values are
// compared as 32-bit IEEE total-order keys (negative: all bits flipped,
// positive: sign bit set), so selection is exact and bit-reproducible.
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
// Collapse.  Per pixel, radix select (4 passes of 8-bit histograms with
// warp-aggregated counts) of the lower median, plus the next key for even T.
#include <cuda_runtime.h>
#include <type_traits>
#include <stdint.h>

#include "graphic_internal.h"

namespace graphic {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t NOTAG = 0xffffffffu;

__device__ __forceinline__ uint32_t f2key(float v) {
  uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
  uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(b);
}

// 16-byte asynchronous global -> shared copy (no register staging).
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

__device__ __forceinline__ int annulus_of(long long p, int n, const double *edge2, int n_ann) {
  const long long x = (p % n) - n / 2, y = (p / n) - n / 2;
  const double rho2 = (double)(x * x + y * y);
  for (int a = 0; a < n_ann; a++)
    if (edge2[a] <= rho2 && rho2 < edge2[a + 1]) return a;
  return -1;
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
  const long long NN = (long long)a.n * a.n;
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
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.status, STATUS_NONFINITE);
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
  const long long NN = (long long)a.n * a.n;
  const long long p0 = (long long)blockIdx.x * 8;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = tcap / 32;   // bitmap words per lane column

  if (lane == 0) ann_s[w] = annulus_of(p0 + w, a.n, a.edge2, a.n_ann);
  for (int s = threadIdx.x; s < T; s += 256) perm_s[s] = (uint16_t)__ldg(&a.perm[s]);
  __syncthreads();
  // a 4-pixel group whose annuli all have a band (or no annulus) belongs to
  // adi_band_kernel, which runs after this kernel
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
      cp_async16(stage + s * 8 + 4 * h, a.in + (long long)perm_s[s] * NN + p0 + 4 * h);
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
    for (int i = lane; i < T; i += 32) a.out[(long long)perm_s[i] * NN + p] = 0.0f;
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
      a.out[(long long)perm_s[i] * NN + p] = v - med;
    }
  }
  if (fail) atomicOr(a.status, STATUS_INTERNAL);
}

// ---------------------------------------------------------------------------
// Band path of the median PSF subtraction
// ---------------------------------------------------------------------------

constexpr uint16_t CODE_BELOW = 0xffff;
constexpr uint16_t CODE_ABOVE = 0xfffe;
constexpr int BAND_PPC = 4;   // pixels (warps) per CTA

// In-register bitonic sort (ascending by key) of 32 E (key, tag) pairs held
// as E consecutive elements per lane.  Equal keys keep their own tags.
template <int E>
__device__ __forceinline__ void bitonic_sort_warp(uint32_t (&k)[E], uint32_t (&x)[E], int lane) {
  constexpr int P = 32 * E;
#pragma unroll
  for (int size = 2; size <= P; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= E) {
        const int ls = stride / E;
        const bool upper = (lane & ls) != 0;
#pragma unroll
        for (int e = 0; e < E; e++) {
          const bool desc = ((lane * E + e) & size) != 0;
          const uint32_t ok = __shfl_xor_sync(FULL, k[e], ls);
          const uint32_t ox = __shfl_xor_sync(FULL, x[e], ls);
          const bool take = (upper == desc) ? (ok < k[e]) : (ok > k[e]);
          k[e] = take ? ok : k[e];
          x[e] = take ? ox : x[e];
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; e++) {
          if (e & stride) continue;
          const int e2 = e | stride;
          const bool desc = ((lane * E + e) & size) != 0;
          const bool sw = desc ? (k[e] < k[e2]) : (k[e] > k[e2]);
          const uint32_t k0 = k[e], k1 = k[e2], x0 = x[e], x1 = x[e2];
          k[e] = sw ? k1 : k0;
          k[e2] = sw ? k0 : k1;
          x[e] = sw ? x1 : x0;
          x[e2] = sw ? x0 : x1;
        }
      }
    }
  }
}

// Sort the nb extracted band elements (bk keys, bidx frames) of one warp in
// place and write code[frame] = sorted band position.
template <int E>
__device__ __forceinline__ void band_sort(uint32_t *bk, uint16_t *bidx, uint16_t *code, int nb, int lane) {
  uint32_t k[E], x[E];
#pragma unroll
  for (int e = 0; e < E; e++) {
    const int j = lane * E + e;
    k[e] = (j < nb) ? bk[j] : 0xffffffffu;
    x[e] = (j < nb) ? (uint32_t)bidx[j] : 0xffffu;
  }
  __syncwarp();
  bitonic_sort_warp<E>(k, x, lane);
#pragma unroll
  for (int e = 0; e < E; e++) {
    const int j = lane * E + e;
    if (j < nb) {
      bk[j] = k[e];
      bidx[j] = (uint16_t)x[e];
      code[x[e]] = (uint16_t)j;
    }
  }
  __syncwarp();
}

// Exact radix selects of the elements of full ranks r_lo <= r_hi among the T
// keys keys[s * BAND_PPC] (s < T), sharing each histogram pass while both
// prefixes agree: returns their keys and the numbers of smaller keys.
// Histograms use fire-and-forget shared-memory reductions (no dependency
// chain); digits equal in every key are skipped.
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
      const uint32_t key = keys[s * BAND_PPC];
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

__device__ __forceinline__ int band_next_set(const uint32_t *bm, int c, int x, int nw) {
  int wd = x >> 5;
  if (wd >= nw) return -1;
  uint32_t word = bm[wd * 32 + c] & (0xffffffffu << (x & 31));
  while (word == 0) {
    if (++wd >= nw) return -1;
    word = bm[wd * 32 + c];
  }
  return wd * 32 + __ffs(word) - 1;
}

// Frame s enters (sign +1) or leaves (sign -1) the reference set of lane c:
// flip its band bit (base counts set bits in words before wi) or count it
// among the BELOW frames.  Branch-free; an inactive call changes nothing.
__device__ __forceinline__ void band_toggle(const uint16_t *code, uint32_t *bm, int c, int s, bool active, int sign,
                                            int wi, int &base, int &cb) {
  const uint16_t cd = active ? code[s] : CODE_ABOVE;
  const bool isb = cd < CODE_ABOVE;
  const int wq = isb ? (cd >> 5) : 0;
  const uint32_t bit = isb ? (1u << (cd & 31)) : 0u;
  bm[wq * 32 + c] ^= bit;
  base += (isb && wq < wi) ? sign : 0;
  cb += (cd == CODE_BELOW) ? sign : 0;
}

// Sweep blocks: the CTA's warps step through their chunks in lockstep, SWK
// queries at a time, so that the values of a block (one 16-byte copy per
// frame for the 4 pixels) and its residuals (one 16-byte store per frame)
// move as whole float4s instead of 4-byte accesses to 32 frames per warp.
constexpr int SWK = 8;
constexpr size_t SW_BLOCK_BYTES = (size_t)SWK * 32 * 16;   // [SWK][32 chunks] float4

// Shared-memory carve-up of adi_band_kernel (bytes), for tcap >= T and
// bitmap width wmax words per lane.  Late (sweep-time) tenants of dead
// regions: bitmaps, staged gates and the residual block in the key area,
// the double-buffered value blocks in the histogram area.
struct BandSmem {
  size_t a, code, bk, bidx, hist, brank, perm, total, obuf;
  __host__ __device__ BandSmem(int tcap, int wmax) {
    const size_t bcm = 32 * (size_t)wmax;
    const size_t keys_b = (size_t)BAND_PPC * tcap * 4;
    // bitmaps + 2 staged gates + the residual block
    const size_t late_b = (size_t)BAND_PPC * wmax * 32 * 4 + 2 * (size_t)tcap * 4 + SW_BLOCK_BYTES;
    a = 0;
    obuf = (size_t)BAND_PPC * wmax * 32 * 4 + 2 * (size_t)tcap * 4;
    code = keys_b > late_b ? keys_b : late_b;
    bk = code + (size_t)BAND_PPC * tcap * 2;
    bidx = bk + (size_t)BAND_PPC * bcm * 4;
    hist = bidx + (size_t)BAND_PPC * bcm * 2;
    hist = (hist + 15) & ~(size_t)15;
    static_assert((size_t)BAND_PPC * 512 * 4 >= 2 * SW_BLOCK_BYTES, "value blocks live in the histogram area");
    brank = hist + (size_t)BAND_PPC * 512 * 4;
    perm = brank + (size_t)BAND_PPC * 64 * 8;
    total = perm + (size_t)tcap * 2;
    total = (total + 15) & ~(size_t)15;
  }
};

// Band path of the median PSF subtraction for 4-pixel groups whose largest
// bitmap width W lies in (wmin, wmax].  Per pixel (one warp):
//   1. keys at full ranks blo, bhi (two radix selects sharing passes);
//   2. ordered extraction of the band (frames between the two, boundary ties
//      split by frame order so that exactly bhi - blo + 1 frames are in it),
//      codes BELOW / ABOVE for the others and a rank structure over BELOW;
//   3. in-register bitonic sort of the band; code[frame] = band position;
//   4. every lane builds its chunk-start membership bitmap over band
//      positions and its count of BELOW frames in the reference set;
//   5. every lane sweeps its chunk of queries: toggle the frames entering /
//      leaving the set, walk a pointer to the t-th set bit, t = k - below.
template <int WCAP>
__global__ void __launch_bounds__(32 * BAND_PPC, 3) adi_band_kernel(const AdiArgs a, int tcap, int wmin) {
  extern __shared__ __align__(16) unsigned char bsm_raw[];
  const int T = a.T;
  const int W_MAX = a.wmax;
  const int BCM = 32 * W_MAX;
  const BandSmem L(tcap, W_MAX);
  uint32_t *keys = reinterpret_cast<uint32_t *>(bsm_raw + L.a);             // [T][4] (phases 0-2)
  uint32_t *bm_all = reinterpret_cast<uint32_t *>(bsm_raw + L.a);           // [4][W_MAX][32] (phases 4-5)
  uint32_t *gate_all = bm_all + BAND_PPC * W_MAX * 32;                      // [2][tcap] packed (L, R)
  uint16_t *code_all = reinterpret_cast<uint16_t *>(bsm_raw + L.code);     // [4][tcap]
  uint32_t *bk_all = reinterpret_cast<uint32_t *>(bsm_raw + L.bk);         // [4][BCM]
  uint16_t *bidx_all = reinterpret_cast<uint16_t *>(bsm_raw + L.bidx);     // [4][BCM]
  uint32_t *hist_all = reinterpret_cast<uint32_t *>(bsm_raw + L.hist);     // [4][512]
  uint32_t *brank_all = reinterpret_cast<uint32_t *>(bsm_raw + L.brank);   // [4][64][2]
  uint16_t *perm_s = reinterpret_cast<uint16_t *>(bsm_raw + L.perm);       // [tcap]
  __shared__ int ann_s[BAND_PPC];
  __shared__ int gate_ann[2];

  const long long NN = (long long)a.n * a.n;
  const long long p0 = (long long)blockIdx.x * BAND_PPC;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) ann_s[w] = annulus_of(p0 + w, a.n, a.edge2, a.n_ann);
  __syncthreads();
  bool mine = true, any = false;
  int gw = 0;
#pragma unroll
  for (int q = 0; q < BAND_PPC; q++) {
    const int an = ann_s[q];
    const int Wq = an < 0 ? 0 : __ldg(&a.band[4 * an + 2]);
    mine &= (an < 0) || (Wq > 0);
    any |= an >= 0;
    gw = max(gw, Wq);
  }
  // groups without annuli go to the first band launch
  if (!mine || gw > W_MAX || (gw <= wmin && !(wmin == 0 && gw == 0))) return;
  for (int s = threadIdx.x; s < T; s += 32 * BAND_PPC) perm_s[s] = (uint16_t)__ldg(&a.perm[s]);
  __syncthreads();
  const int ann = ann_s[w];
  if (!any) {
    for (int i = threadIdx.x; i < T * BAND_PPC; i += 32 * BAND_PPC)
      a.out[(long long)perm_s[i / BAND_PPC] * NN + p0 + (i % BAND_PPC)] = 0.0f;
    return;
  }
  // ---- 0. load: one 16-byte copy per frame (the 4 pixels), keys in place
  {
    float *stage = reinterpret_cast<float *>(keys);
    for (int s = threadIdx.x; s < T; s += 32 * BAND_PPC)
      cp_async16(stage + BAND_PPC * s, a.in + (long long)perm_s[s] * NN + p0);
    cp_async_wait_all();
    __syncthreads();
    bool bad = false;
    for (int j = threadIdx.x; j < T * BAND_PPC; j += 32 * BAND_PPC) {
      const float v = stage[j];
      bad |= !isfinite(v);
      keys[j] = f2key(v);
    }
    if (bad) atomicOr(a.status, STATUS_NONFINITE);
    __syncthreads();
  }
  const int blo = ann >= 0 ? __ldg(&a.band[4 * ann]) : 0;
  const int bhi = ann >= 0 ? __ldg(&a.band[4 * ann + 1]) : 0;
  const int W = ann >= 0 ? __ldg(&a.band[4 * ann + 2]) : 0;
  const uint32_t *kw = keys + w;                 // key of frame s: kw[s * 4]
  uint32_t *hist = hist_all + w * 512;
  uint32_t *bk = bk_all + w * BCM;
  uint16_t *code = code_all + w * tcap;
  uint16_t *bidx = bidx_all + w * BCM;
  uint32_t *brank = brank_all + w * 128;         // [64] BELOW masks, [64] BELOW counts before each round
  bool fail = false;
  int nb = 0, nbelow = 0;

  if (ann >= 0) {
    // ---- 1. exact keys at full ranks blo and bhi ------------------------
    uint32_t orv = 0, andv = 0xffffffffu;
    for (int s = lane; s < T; s += 32) {
      orv |= kw[s * BAND_PPC];
      andv &= kw[s * BAND_PPC];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      orv |= __shfl_xor_sync(FULL, orv, o);
      andv &= __shfl_xor_sync(FULL, andv, o);
    }
    uint32_t Klo, Khi, clt_lo, clt_hi;
    band_select2(kw, T, (uint32_t)blo, (uint32_t)bhi, orv ^ andv, andv, hist, hist + 256, lane, Klo, clt_lo,
                 Khi, clt_hi);
    // ---- 2. ordered extraction -------------------------------------------
    // First without tie handling: the band is taken as the keys in
    // [Klo, Khi].  When that set has exactly bhi - blo + 1 members it is the
    // band (no key equal to a bound had to go outside); otherwise keys equal
    // to a bound are split by frame order in a second, exact pass.  Both
    // passes write every frame's code or band entry.
    const int need_lo = blo - (int)clt_lo;
    const int lim_hi = bhi + 1 - (int)clt_hi;
    const unsigned lt = (1u << lane) - 1u;
    auto extract = [&](auto ties) {
      constexpr bool TIES = decltype(ties)::value;
      nb = 0;
      nbelow = 0;
      int tlo = 0, thi = 0;
      for (int base = 0; base < T; base += 32) {
        const int s = base + lane;
        const bool valid = s < T;
        const uint32_t key = valid ? kw[s * BAND_PPC] : 0u;
        bool below, above;
        if constexpr (TIES) {
          const bool eqlo = valid && key == Klo, eqhi = valid && key == Khi;
          const unsigned mlo = __ballot_sync(FULL, eqlo), mhi = __ballot_sync(FULL, eqhi);
          const int ilo = tlo + __popc(mlo & lt), ihi = thi + __popc(mhi & lt);
          below = valid && (key < Klo || (eqlo && ilo < need_lo));
          above = valid && !below && (key > Khi || (eqhi && ihi >= lim_hi));
          tlo += __popc(mlo);
          thi += __popc(mhi);
        } else {
          below = valid && key < Klo;
          above = valid && key > Khi;
        }
        const bool inb = valid && !below && !above;
        const unsigned mb = __ballot_sync(FULL, inb), mbl = __ballot_sync(FULL, below);
        if (inb) {
          const int j = nb + __popc(mb & lt);
          if (j < BCM) {
            bk[j] = key;
            bidx[j] = (uint16_t)s;
          }
        } else if (valid) {
          code[s] = below ? CODE_BELOW : CODE_ABOVE;
        }
        if (lane == 0) {
          brank[base >> 5] = mbl;
          brank[64 + (base >> 5)] = (uint32_t)nbelow;
        }
        nb += __popc(mb);
        nbelow += __popc(mbl);
      }
    };
    extract(std::false_type{});
    if (nb != bhi - blo + 1) {
      __syncwarp();
      extract(std::true_type{});
    }
    if (nb != bhi - blo + 1 || nb > 32 * W) fail = true;
    __syncwarp();
    // ---- 3. sort the band; codes of band frames = sorted positions -------
    if (!fail) {
      // only the widths this instantiation serves are compiled in (the
      // 32-word sort needs far more registers than the others)
      if constexpr (WCAP <= 16) {
        switch (W) {
          case 1: band_sort<1>(bk, bidx, code, nb, lane); break;
          case 2: band_sort<2>(bk, bidx, code, nb, lane); break;
          case 4: band_sort<4>(bk, bidx, code, nb, lane); break;
          case 8: band_sort<8>(bk, bidx, code, nb, lane); break;
          default: band_sort<16>(bk, bidx, code, nb, lane); break;
        }
      } else {
        band_sort<32>(bk, bidx, code, nb, lane);
      }
    }
  }
  // keys are dead from here on: their space holds the bitmaps and the gates
  __syncthreads();
  if (threadIdx.x < 2) gate_ann[threadIdx.x] = -1;
  __syncthreads();
  if (lane == 0 && ann >= 0) {
    // the (at most two) annuli of this group get their gate staged once
    if (atomicCAS(&gate_ann[0], -1, ann) != -1 && gate_ann[0] != ann) atomicCAS(&gate_ann[1], -1, ann);
  }
  __syncthreads();
  for (int g = 0; g < 2; g++) {
    const int an = gate_ann[g];
    if (an < 0) continue;
    const int2 *lr2 = reinterpret_cast<const int2 *>(a.lr + (size_t)an * T * 2);
    uint32_t *gt = gate_all + g * tcap;
    for (int s = threadIdx.x; s < T; s += 32 * BAND_PPC) {
      const int2 v = __ldg(&lr2[s]);
      gt[s] = (uint32_t)v.x | ((uint32_t)v.y << 16);
    }
  }
  __syncthreads();
  // pixels outside the annuli and failed warps take part in the lockstep
  // sweep (their residuals are 0) so that the CTA's barriers stay uniform
  if (fail && ann >= 0 && lane == 0) atomicOr(a.status, STATUS_INTERNAL);
  const bool act = ann >= 0 && !fail;
  // gate of this pixel's annulus: staged copy, or global memory for a third
  // annulus inside one 4-pixel group
  const uint32_t *gate = gate_ann[0] == ann ? gate_all : (gate_ann[1] == ann ? gate_all + tcap : nullptr);
  const int2 *gate_g = reinterpret_cast<const int2 *>(a.lr + (size_t)(ann < 0 ? 0 : ann) * T * 2);
  auto gate_at = [&](int i) -> uint32_t {
    if (gate) return gate[i];
    const int2 v = __ldg(&gate_g[i]);
    return (uint32_t)v.x | ((uint32_t)v.y << 16);
  };
  uint32_t *bm = bm_all + w * W_MAX * 32;
  auto below_before = [&](int s) -> int {      // BELOW frames with sorted position < s
    if (s >= T) return nbelow;
    const int r = s >> 5;
    return (int)brank[64 + r] + __popc(brank[r] & ((1u << (s & 31)) - 1u));
  };
  const int C = (T + 31) / 32;
  const int c = lane;
  const int i0 = c * C;
  const int i1 = min(T, i0 + C);
  const int nblk = (C + SWK - 1) / SWK;
  float4 *vbuf = reinterpret_cast<float4 *>(hist_all);                       // [2][SWK][32]
  float *obuf = reinterpret_cast<float *>(bsm_raw + L.obuf);                // [SWK][32][4]
  // values of block b: frame perm[c' C + b SWK + kk], the group's 4 pixels
  auto prefetch = [&](int b) {
    float4 *dst = vbuf + (b & 1) * SWK * 32;
    for (int q = threadIdx.x; q < SWK * 32; q += 32 * BAND_PPC) {
      const int kk = q >> 5, cc = q & 31;
      const int i = cc * C + b * SWK + kk;
      if (b * SWK + kk < C && i < T) cp_async16(dst + q, a.in + (long long)perm_s[i] * NN + p0);
    }
    cp_async_commit();
  };
  prefetch(0);   // the histograms are dead: overlap the first block with the bitmaps

  // ---- 4. chunk-start bitmap and BELOW count of each lane --------------
  int cb = 0;
  if (act && i0 < T) {
    const uint32_t g0 = gate_at(i0);
    const int L0 = (int)(g0 & 0xffffu), R0 = (int)(g0 >> 16);
    for (int wd = 0; wd < W; wd++) {
      uint32_t word = 0;
#pragma unroll 8
      for (int b = 0; b < 32; b++) {
        const int pb = wd * 32 + b;
        const int f = bidx[pb];                       // same address in every lane
        word |= (pb < nb && (f < L0 || f >= R0)) ? (1u << b) : 0u;
      }
      bm[wd * 32 + c] = word;
    }
    cb = below_before(L0) + (nbelow - below_before(R0));
  }
  __syncwarp();

  // ---- 5. per-lane sweep, SWK queries per block -------------------------
  // State: word wi of the bitmap column holds the t-th set bit, base = set
  // bits in words < wi.  Gates of band annuli are monotone (host check):
  // frames [L, L') enter the reference set, frames [R, R') leave it.
  int Lc = 0, Rc = 0, wi = 0, base = 0;
  bool lane_ok = act && i0 < T;
  if (lane_ok) {
    const uint32_t g0 = gate_at(i0);
    Lc = (int)(g0 & 0xffffu);
    Rc = (int)(g0 >> 16);
  }
  for (int b = 0; b < nblk; b++) {
    if (b + 1 < nblk) {
      prefetch(b + 1);
      cp_async_wait_group<1>();
    } else {
      cp_async_wait_group<0>();
    }
    __syncthreads();   // block b's values are in; block b-1's residuals are written out
    const float4 *vb = vbuf + (b & 1) * SWK * 32;
    for (int kk = 0; kk < SWK; kk++) {
      const int i = i0 + b * SWK + kk;
      if (b * SWK + kk >= C || i >= i1) break;
      float res = 0.0f;
      if (lane_ok) {
        const uint32_t gi = gate_at(i);
        const int Ln = (int)(gi & 0xffffu), Rn = (int)(gi >> 16);
        // frames [Lc, Ln) enter, [Rc, Rn) leave: the first two of each run
        // without branches (the usual case is one or two), any others in a loop
        band_toggle(code, bm, c, Lc, Lc < Ln, 1, wi, base, cb);
        band_toggle(code, bm, c, Lc + 1, Lc + 1 < Ln, 1, wi, base, cb);
        for (int s = Lc + 2; s < Ln; s++) band_toggle(code, bm, c, s, true, 1, wi, base, cb);
        band_toggle(code, bm, c, Rc, Rc < Rn, -1, wi, base, cb);
        band_toggle(code, bm, c, Rc + 1, Rc + 1 < Rn, -1, wi, base, cb);
        for (int s = Rc + 2; s < Rn; s++) band_toggle(code, bm, c, s, true, -1, wi, base, cb);
        Lc = Ln;
        Rc = Rn;
        const int nset = Lc + (T - Rc);
        const int t = ((nset - 1) >> 1) - cb;
        uint32_t wd = bm[wi * 32 + c];
        int pc = __popc(wd);
        while (t < base && wi > 0) {
          wi--;
          wd = bm[wi * 32 + c];
          pc = __popc(wd);
          base -= pc;
        }
        while (t >= base + pc && wi + 1 < W) {
          base += pc;
          wi++;
          wd = bm[wi * 32 + c];
          pc = __popc(wd);
        }
        if (t >= base && t < base + pc) {
          const int pos = nth_set(wd, t - base);
          float med = key2f(bk[wi * 32 + pos]);
          if ((nset & 1) == 0) {
            // the next member: a higher bit of this word, else the next word's first
            const uint32_t rest = pos < 31 ? (wd & (0xfffffffeu << pos)) : 0u;
            const int p2 = rest ? wi * 32 + __ffs(rest) - 1 : band_next_set(bm, c, (wi + 1) * 32, W);
            if (p2 >= 0)
              med = (med + key2f(bk[p2])) * 0.5f;
            else
              lane_ok = false;
          }
          if (lane_ok) {
            const float4 v4 = vb[kk * 32 + c];
            const float v = w == 0 ? v4.x : (w == 1 ? v4.y : (w == 2 ? v4.z : v4.w));
            res = v - med;
          }
        } else {
          lane_ok = false;
        }
        if (!lane_ok) atomicOr(a.status, STATUS_INTERNAL);
      }
      obuf[(kk * 32 + c) * 4 + w] = res;
    }
    __syncthreads();   // block b's residuals are complete
    for (int q = threadIdx.x; q < SWK * 32; q += 32 * BAND_PPC) {
      const int kk = q >> 5, cc = q & 31;
      const int i = cc * C + b * SWK + kk;
      if (b * SWK + kk < C && i < T) {
        const float4 r4 = reinterpret_cast<const float4 *>(obuf)[q];
        *reinterpret_cast<float4 *>(a.out + (long long)perm_s[i] * NN + p0) = r4;
      }
    }
  }
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
  if (a.T <= 8192) {
    const size_t smem = (size_t)(COL_PPC * 256 + COL_KS * a.T) * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(collapse_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
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
  const long long NN = (long long)a.n * a.n;
  const int tcap = pow2_at_least(a.T, 32);
  // general kernel first: it reads every pixel of its groups and writes only
  // its own; the band launches then own disjoint 4-pixel groups
  cudaError_t e = launch_adi_general(a, st, tcap);
  nl += (e == cudaSuccess);
  if (e != cudaSuccess || a.wmax == 0) return e;
  // band launches: groups whose widest bitmap is <= 16 words, then wider ones,
  // each with shared memory sized for its widest class
  {
    AdiArgs b = a;
    b.wmax = a.wmax < 16 ? a.wmax : 16;
    const BandSmem L(tcap, b.wmax);
    e = cudaFuncSetAttribute(adi_band_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    adi_band_kernel<16><<<(unsigned)(NN / BAND_PPC), 32 * BAND_PPC, L.total, st>>>(b, tcap, 0);
    e = cudaGetLastError();
    nl += (e == cudaSuccess);
    if (e != cudaSuccess) return e;
  }
  if (a.wmax > 16) {
    const BandSmem L(tcap, a.wmax);
    e = cudaFuncSetAttribute(adi_band_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    adi_band_kernel<32><<<(unsigned)(NN / BAND_PPC), 32 * BAND_PPC, L.total, st>>>(a, tcap, 16);
    e = cudaGetLastError();
    nl += (e == cudaSuccess);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_adi_general(const AdiArgs &a, cudaStream_t st, int tcap) {
  const long long NN = (long long)a.n * a.n;
  const size_t smem = (size_t)8 * 256 * sizeof(uint32_t) +
                      (size_t)8 * tcap * (2 * sizeof(uint32_t) + 2 * sizeof(uint16_t)) + (size_t)tcap * sizeof(uint16_t);
  cudaError_t e = cudaFuncSetAttribute(adi_median_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  adi_median_kernel<<<(unsigned)(NN / 8), 256, smem, st>>>(a, tcap);
  return cudaGetLastError();
}

}  // namespace graphic

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

template <bool SMEM>
__global__ void __launch_bounds__(256) collapse_kernel(const CollapseArgs a, int tcap) {
  extern __shared__ uint32_t csm[];
  uint32_t *hist_all = csm;                 // [8][256]
  uint32_t *keys_all = csm + 8 * 256;       // [8][tcap]   (SMEM only)
  const long long T = a.T;
  const long long NN = (long long)a.n * a.n;
  const long long p0 = (long long)blockIdx.x * 8;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;

  bool bad = false;
  if constexpr (SMEM) {
    for (long long idx = threadIdx.x; idx < 8 * T; idx += 256) {
      const int pw = (int)(idx & 7);
      const long long t = idx >> 3;
      const float v = a.in[t * NN + p0 + pw];
      bad |= !isfinite(v);
      keys_all[pw * tcap + t] = f2key(v);
    }
    if (bad) atomicOr(a.status, STATUS_NONFINITE);
    __syncthreads();
  }
  uint32_t *hist = hist_all + w * 256;
  const uint32_t *keys = keys_all + w * tcap;
  const long long p = p0 + w;
  auto key_at = [&](long long t) -> uint32_t {
    if constexpr (SMEM) return keys[t];
    else return f2key(a.in[t * NN + p]);
  };

  const uint32_t k = (uint32_t)((T - 1) / 2);
  uint32_t prefix = 0, pmask = 0, krem = k, cnt = 0;
  for (int pass = 0; pass < 4; pass++) {
    const int shift = 24 - 8 * pass;
#pragma unroll
    for (int b = 0; b < 8; b++) hist[lane * 8 + b] = 0;
    __syncwarp();
    for (long long base = 0; base < T; base += 32) {
      const long long t = base + lane;
      uint32_t tag = NOTAG;
      if (t < T) {
        const uint32_t key = key_at(t);
        if constexpr (!SMEM) {
          if (pass == 0) bad |= !isfinite(key2f(key));
        }
        if ((key & pmask) == prefix) tag = (key >> shift) & 255u;
      }
      const unsigned peers = __match_any_sync(FULL, tag);
      if (tag != NOTAG && lane == __ffs(peers) - 1) hist[tag] += __popc(peers);
      __syncwarp();
    }
    uint32_t d, below;
    hist_find(hist, krem, lane, d, below, cnt);
    prefix |= d << shift;
    pmask |= 0xffu << shift;
    krem -= below;
    __syncwarp();
  }
  if constexpr (!SMEM) {
    if (bad) atomicOr(a.status, STATUS_NONFINITE);
  }
  const float lo = key2f(prefix);
  float med = lo;
  if ((T & 1) == 0) {
    uint32_t hi = prefix;
    if (krem + 1 >= cnt) {
      // smallest key greater than the lower median
      uint32_t m = 0xffffffffu;
      for (long long t = lane; t < T; t += 32) {
        const uint32_t key = key_at(t);
        if (key > prefix && key < m) m = key;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(FULL, m, o));
      hi = m;
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
  __shared__ int ann_s[8];

  const int T = a.T;
  const long long NN = (long long)a.n * a.n;
  const long long p0 = (long long)blockIdx.x * 8;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = tcap / 32;   // bitmap words per lane column

  if (lane == 0) ann_s[w] = annulus_of(p0 + w, a.n, a.edge2, a.n_ann);
  __syncthreads();
  bool any = false;
#pragma unroll
  for (int q = 0; q < 8; q++) any |= ann_s[q] >= 0;
  bool bad = false;
  if (any) {
    for (int idx = threadIdx.x; idx < 8 * T; idx += 256) {
      const int pw = idx & 7, s = idx >> 3;
      const float v = a.in[(long long)a.perm[s] * NN + p0 + pw];
      bad |= !isfinite(v);
      kA_all[pw * tcap + s] = f2key(v);
      iA_all[pw * tcap + s] = (uint16_t)s;
    }
  }
  if (bad) atomicOr(a.status, STATUS_NONFINITE);
  __syncthreads();

  const int ann = ann_s[w];
  const long long p = p0 + w;
  if (ann < 0) {
    for (int i = lane; i < T; i += 32) a.out[(long long)a.perm[i] * NN + p] = 0.0f;
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
  const int *LR = a.lr + (size_t)ann * T * 2;
  const int C = (T + 31) / 32;
  {
    const int L0 = __ldg(&LR[0]), R0 = __ldg(&LR[1]);
    for (int wd = 0; wd < nw; wd++) {
      const int pos = wd * 32 + lane;
      bool mem = false;
      if (pos < T) {
        const int s = si[pos];
        mem = (s < L0) || (s >= R0);
      }
      const unsigned word = __ballot_sync(FULL, mem);
      if (lane == 0) bm[wd * 32] = word;
    }
    __syncwarp();
    int Lp = L0, Rp = R0;
    for (int c = 1; c < 32; c++) {
      const int i0 = c * C;
      if (i0 >= T) break;
      const int Lc = __ldg(&LR[2 * i0]), Rc = __ldg(&LR[2 * i0 + 1]);
      for (int wd = lane; wd < nw; wd += 32) bm[wd * 32 + c] = bm[wd * 32 + c - 1];
      __syncwarp();
      const int a0 = min(Lp, Lc), a1 = max(Lp, Lc), b0 = min(Rp, Rc), b1 = max(Rp, Rc);
      for (int s = a0 + lane; s < a1; s += 32) {
        const int r = rk[s];
        atomicXor(&bm[(r >> 5) * 32 + c], 1u << (r & 31));
      }
      for (int s = b0 + lane; s < b1; s += 32) {
        const int r = rk[s];
        atomicXor(&bm[(r >> 5) * 32 + c], 1u << (r & 31));
      }
      __syncwarp();
      Lp = Lc;
      Rp = Rc;
    }
  }

  // ---- 3. per-lane sweep over its chunk of queries -----------------------
  const int c = lane;
  const int i0 = c * C;
  const int i1 = min(T, i0 + C);
  bool fail = false;
  if (i0 < T) {
    int L = __ldg(&LR[2 * i0]), R = __ldg(&LR[2 * i0 + 1]);
    int nset = L + (T - R);
    int k = (nset - 1) >> 1;
    int pos = -1, acc = 0;
    for (int wd = 0; wd < nw; wd++) {
      const uint32_t word = bm[wd * 32 + c];
      const int pc = __popc(word);
      if (acc + pc > k) {
        pos = wd * 32 + (int)__fns(word, 0, k - acc + 1);
        break;
      }
      acc += pc;
    }
    int below = k;
    if (pos < 0) fail = true;
    for (int i = i0; i < i1 && !fail; i++) {
      const int Ln = __ldg(&LR[2 * i]), Rn = __ldg(&LR[2 * i + 1]);
      // toggle frames whose membership changes; keep `below` = set bits < pos
      for (int pass = 0; pass < 2; pass++) {
        const int s0 = pass == 0 ? min(L, Ln) : min(R, Rn);
        const int s1 = pass == 0 ? max(L, Ln) : max(R, Rn);
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
      nset = L + (T - R);
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
      a.out[(long long)__ldg(&a.perm[i]) * NN + p] = v - med;
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

cudaError_t launch_collapse(const CollapseArgs &a, cudaStream_t st) {
  const long long NN = (long long)a.n * a.n;
  const unsigned grid = (unsigned)(NN / 8);
  if (a.T <= 4096) {
    const int tcap = pow2_at_least(a.T, 32);
    const size_t smem = (size_t)(8 * 256 + 8 * tcap) * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(collapse_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    collapse_kernel<true><<<grid, 256, smem, st>>>(a, tcap);
  } else {
    const size_t smem = (size_t)(8 * 256) * sizeof(uint32_t);
    collapse_kernel<false><<<grid, 256, smem, st>>>(a, 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_adi_median(const AdiArgs &a, cudaStream_t st) {
  const long long NN = (long long)a.n * a.n;
  const int tcap = pow2_at_least(a.T, 32);
  const size_t smem = (size_t)8 * 256 * sizeof(uint32_t) + (size_t)8 * tcap * (2 * sizeof(uint32_t) + 2 * sizeof(uint16_t));
  cudaError_t e = cudaFuncSetAttribute(adi_median_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  adi_median_kernel<<<(unsigned)(NN / 8), 256, smem, st>>>(a, tcap);
  return cudaGetLastError();
}

}  // namespace graphic

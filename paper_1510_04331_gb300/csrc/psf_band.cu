// psf_band.cu -- band path of the angle-gated median PSF subtraction
// (Sect. 3.3) on sm_103a.
//
// Notation.  Frames in angle order s = 0..T-1 (perm[s] = frame index).  The
// PSF of query i (the frame at angle position i) is the median of the pixel
// over its reference set S_i = [0, L_i) u [R_i, T) (host plan, FP64 gate;
// on this path L_i and R_i never decrease with i): the (|S_i|-1)/2-th member
// in the IEEE total order of the values, ties ordered by s, averaged in FP32
// with the next member when |S_i| is even.  The full rank of every such
// member (its rank among all T values) lies in one band [blo, bhi] of the
// annulus (host plan), so only the band's members and the count of the
// frames below the band ("BELOW") matter.
//
// Frame s is outside S_i exactly for the queries a_s <= i < b_s (a_s = first
// i with R_i > s, b_s = first i with L_i > s; host table evq): a band member
// leaves the reference set once and re-enters once, so the reference set of
// the band changes at only 2 x (band size) "events" over all T queries.
//
// Two kernels, one warp per pixel, four pixels (16 bytes of each frame) per
// CTA:
//   band_prep_kernel   finds the band's members: the pixel's T values in
//     shared memory, a 256-bin histogram linear in value between the
//     pixel's extremes locates the bins of ranks blo and bhi, one pass
//     extracts the values of those bins (candidates, in frame order) and a
//     bit map of the frames below them; a counting sort (256 bins linear in
//     value between the candidates' extremes, ties in a bin resolved by
//     counting) ranks the candidates.  When the located bins hold more than
//     the candidate capacity (heavy outliers, many ties) an exact radix
//     select of the keys of ranks blo and bhi and a tie-aware extraction
//     give the band directly.  Writes per pixel: the band's values in value
//     order, the band's members in frame order (value position, event
//     queries) and the BELOW bit map over s.
//   band_sweep_kernel  lane c sweeps the queries [cC, cC + C), C = ceil(T/32):
//     a bit map over band positions (value order) holds the band members of
//     the current reference set; its start state for every lane comes from
//     the event queries by one 32 x 32 bit transpose per map word; per query
//     the lane applies the events of that query, counts the BELOW members
//     of S_i from the BELOW map (two prefix popcounts), and reads the t-th
//     member of its map, t = k_i - (BELOW members).  The lanes of the CTA
//     sweep in lockstep blocks of SWK queries so that values (one 16-byte
//     copy per frame) and residuals (one 16-byte store per frame) move as
//     whole float4s.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "graphic_internal.h"
#include "select_common.cuh"

namespace graphic {
namespace {

constexpr int PPC = 4;     // pixels (warps) per CTA
constexpr int KS = 4;      // band_prep_kernel: words per frame row of the keys (one 16-byte copy per frame)
constexpr int SWK = 4;     // queries per lockstep sweep block (4 measured faster than 8: smaller blocks, more CTAs)
constexpr int NCLASS = 7;  // group classes: 0 = no pixel in an annulus, then bit map words 1, 2, 4, ..., 32
constexpr int kClassW[NCLASS] = {0, 1, 2, 4, 8, 16, 32};

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Per-pixel slot written by band_prep_kernel and read by band_sweep_kernel,
// for band capacity NB and nwt = ceil(T / 32) BELOW words.
//   header   int4 (band size nb, BELOW count, annulus or -1, 1 = ok)
//   skeys    [NB] u32   band values (float bits) in value order
//   blev     [NB] u32   band members in frame order: event queries a | b << 16
//   blpos    [NB] u16   band members in frame order: value position
//   below    [nwt] u32  bit s: frame s is below the band
struct Slot {
  size_t skeys, blev, blpos, below, bytes;
  __host__ __device__ Slot(int NB, int nwt) {
    skeys = 16;
    blev = skeys + (size_t)NB * 4;
    blpos = blev + (size_t)NB * 4;
    below = al16(blpos + (size_t)NB * 2);
    bytes = al16(below + (size_t)nwt * 4);
  }
};

struct BandArgs {
  AdiArgs a;
  const uint32_t *evq;   // [A][T] event queries a_s | b_s << 16 (annuli with a band)
  const int *groups;     // this class's 4-pixel groups (first pixel / 4)
  char *slots;           // this class's slots, PPC per group
  size_t slot_bytes;
  int NB;                // band capacity 32 W of the class
  int cap;               // candidate capacity of band_prep_kernel
  int nwt;               // ceil(T / 32)
};

__device__ __forceinline__ int annulus_of(long long p, int n, const double *edge2, int n_ann) {
  const long long x = (p % n) - n / 2, y = (p / n) - n / 2;
  const double rho2 = (double)(x * x + y * y);
  for (int a = 0; a < n_ann; a++)
    if (edge2[a] <= rho2 && rho2 < edge2[a + 1]) return a;
  return -1;
}

// Bin of a key in a histogram linear in value from v0 with `scale` bins per
// unit: monotone non-decreasing in the key (every step is a monotone
// rounding), clamped to [0, 255].  A scale of 0 (empty or overflowing
// range) puts every key in bin 0.
__device__ __forceinline__ int vbin(uint32_t k, float v0, float scale) {
  const float x = (key2f(k) - v0) * scale;
  const int b = (int)x;              // x >= 0 or NaN (inf * 0): NaN converts to 0
  return b < 255 ? b : 255;
}

// Bins holding the ranks r0 <= r1 in a filled 256-bin histogram: returns the
// bins and the number of keys in lower bins.
__device__ __forceinline__ void hist_locate2(const uint32_t *hist, uint32_t r0, uint32_t r1, int lane, int &b0,
                                             uint32_t &below0, int &b1, uint32_t &below1) {
  uint32_t h[8], s = 0;
#pragma unroll
  for (int b = 0; b < 8; b++) {
    h[b] = hist[lane * 8 + b];
    s += h[b];
  }
  uint32_t inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += t;
  }
  const uint32_t exc = inc - s;
  int rb[2];
  uint32_t rbel[2];
  const uint32_t rr[2] = {r0, r1};
#pragma unroll
  for (int q = 0; q < 2; q++) {
    const unsigned ball = __ballot_sync(FULL, inc > rr[q]);
    const int L = ball ? __ffs(ball) - 1 : 31;
    int bb = 0;
    uint32_t bel = 0;
    if (lane == L) {
      uint32_t acc = exc;
      bool done = false;
#pragma unroll
      for (int b = 0; b < 8; b++) {
        if (!done && acc + h[b] > rr[q]) {
          bb = lane * 8 + b;
          bel = acc;
          done = true;
        }
        acc += h[b];
      }
    }
    rb[q] = __shfl_sync(FULL, bb, L);
    rbel[q] = __shfl_sync(FULL, bel, L);
  }
  b0 = rb[0];
  below0 = rbel[0];
  b1 = rb[1];
  below1 = rbel[1];
}

// ---------------------------------------------------------------------------
// band_prep_kernel
// ---------------------------------------------------------------------------

// Shared memory: keys [T][KS] u32 (pixel q of frame s at s KS + q), then per
// warp: hist[256], cur[256] u32, ckey[cap] u32, cs[cap] u16, tmp[cap] u16,
// below[nwt] u32.
__host__ __device__ inline size_t prep_warp_bytes(int cap, int nwt) {
  return al16(2048 + (size_t)cap * 8) + al16((size_t)nwt * 4);
}
__host__ __device__ inline size_t prep_smem_bytes(int T, int cap, int nwt) {
  return al16((size_t)T * KS * 4) + PPC * prep_warp_bytes(cap, nwt);
}

__global__ void __launch_bounds__(32 * PPC, 4) band_prep_kernel(const BandArgs B) {
  extern __shared__ __align__(16) unsigned char psm[];
  const AdiArgs &a = B.a;
  const int T = a.T;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long p0 = (long long)__ldg(&B.groups[blockIdx.x]) * PPC;
  uint32_t *keys = reinterpret_cast<uint32_t *>(psm);
  unsigned char *wb = psm + al16((size_t)T * KS * 4) + (size_t)w * prep_warp_bytes(B.cap, B.nwt);
  uint32_t *hist = reinterpret_cast<uint32_t *>(wb);
  uint32_t *cur = hist + 256;
  uint32_t *ckey = cur + 256;
  uint16_t *cs = reinterpret_cast<uint16_t *>(ckey + B.cap);
  uint16_t *tmp = cs + B.cap;
  uint32_t *below = reinterpret_cast<uint32_t *>(wb + al16(2048 + (size_t)B.cap * 8));
  __shared__ int ann_s[PPC];

  if (lane == 0) ann_s[w] = annulus_of(p0 + w, a.n, a.edge2, a.n_ann);
  // the group's 4 pixels of every frame, angle order: one 16-byte copy each,
  // in four quarters, so that the key conversion of a quarter overlaps the
  // copies of the later ones
  const int Q = ((T + 127) / 128) * 32;   // frames per quarter, a multiple of 32
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int s1 = min(T, (k + 1) * Q);
    for (int s = k * Q + threadIdx.x; s < s1; s += 32 * PPC)
      cp_async16(keys + KS * s, a.in + (long long)(a.perm_id ? s : __ldg(&a.perm[s])) * a.in_fs + p0);
    cp_async_commit();
  }
  uint32_t *kcol = keys + w;   // key of frame s: kcol[s * KS]
  // keys in place, with the finiteness check and the extremes; each warp
  // works on its own pixel's column
  bool bad = false;
  uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (k == 0) cp_async_wait_group<3>();
    else if (k == 1) cp_async_wait_group<2>();
    else if (k == 2) cp_async_wait_group<1>();
    else cp_async_wait_group<0>();
    __syncthreads();   // quarter k of every thread's copies has landed
    const int s1 = min(T, (k + 1) * Q);
#pragma unroll 4
    for (int s = k * Q + lane; s < s1; s += 32) {
      const float v = __uint_as_float(kcol[s * KS]);
      bad |= !isfinite(v);
      const uint32_t key = f2key(v);
      kcol[s * KS] = key;
      kmin = min(kmin, key);
      kmax = max(kmax, key);
    }
  }
  const int ann = ann_s[w];   // written before the barriers above
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.status, STATUS_NONFINITE);
  __syncwarp();
  char *slot = B.slots + ((size_t)blockIdx.x * PPC + w) * B.slot_bytes;
  const Slot L(B.NB, B.nwt);
  if (ann < 0) {
    if (lane == 0) *reinterpret_cast<int4 *>(slot) = make_int4(0, 0, -1, 1);
    return;
  }
  const int blo = __ldg(&a.band[4 * ann]), bhi = __ldg(&a.band[4 * ann + 1]);
  const int nbd = bhi - blo + 1;
  const uint32_t *kw = kcol;
  const unsigned lt = (1u << lane) - 1u;
  // each candidate's event queries are gathered asynchronously into this
  // warp's key column as the candidate is found (entry j at kcol[j * KS]:
  // j never passes the frame being read, whose key is already in registers)
  const uint32_t *evq = B.evq + (size_t)ann * T;

  // ---- extremes ----------------------------------------------------------
  kmin = __reduce_min_sync(FULL, kmin);
  kmax = __reduce_max_sync(FULL, kmax);

  // ---- candidates: the histogram bins of ranks blo .. bhi -----------------
  const float v0 = key2f(kmin);
  const float range = key2f(kmax) - v0;
  const float scale = (range > 0.f) ? 256.f / range : 0.f;
#pragma unroll
  for (int b = 0; b < 8; b++) hist[lane * 8 + b] = 0u;
  __syncwarp();
#pragma unroll 4
  for (int s = lane; s < T; s += 32) atomicAdd(&hist[vbin(kw[s * KS], v0, scale)], 1u);
  __syncwarp();
  int B0, B1;
  uint32_t bel0, bel1;
  hist_locate2(hist, (uint32_t)blo, (uint32_t)bhi, lane, B0, bel0, B1, bel1);
  const uint32_t cnt_hi = hist[B1];
  const int ncand = (int)(bel1 + cnt_hi - bel0);
  int nc = 0;
  int nbelow = 0;   // frames below the candidates
  uint32_t cmin = 0xffffffffu, cmax = 0u;
  __syncwarp();
  if (ncand <= B.cap) {
    // four 32-frame rounds per step: their loads and bins are independent
    for (int base = 0; base < T; base += 128) {
      uint32_t k[4];
      int b[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int s = base + 32 * u + lane;
        k[u] = s < T ? kw[s * KS] : 0u;
        b[u] = s < T ? vbin(k[u], v0, scale) : 256;
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int s = base + 32 * u + lane;
        if (base + 32 * u >= T) break;
        const bool isc = b[u] >= B0 && b[u] <= B1;
        const bool isb = b[u] < B0;
        const unsigned mc = __ballot_sync(FULL, isc), mb = __ballot_sync(FULL, isb);
        if (isc) {
          const int j = nc + __popc(mc & lt);
          ckey[j] = k[u];
          cs[j] = (uint16_t)s;
          cp_async4(&kcol[j * KS], evq + s);
          cmin = min(cmin, k[u]);
          cmax = max(cmax, k[u]);
        }
        if (lane == 0) below[(base >> 5) + u] = mb;
        nc += __popc(mc);
      }
    }
    nbelow = (int)bel0;
  } else {
    // exact: keys of full ranks blo and bhi, then the band itself with the
    // keys equal to a bound split by frame order
    uint32_t orv = 0, andv = 0xffffffffu;
    for (int s = lane; s < T; s += 32) {
      orv |= kw[s * KS];
      andv &= kw[s * KS];
    }
    orv = __reduce_or_sync(FULL, orv);
    andv = __reduce_and_sync(FULL, andv);
    uint32_t Klo, Khi, clt_lo, clt_hi;
    band_select2<KS>(kw, T, (uint32_t)blo, (uint32_t)bhi, orv ^ andv, andv, hist, cur, lane, Klo, clt_lo, Khi,
                      clt_hi);
    const int need_lo = blo - (int)clt_lo;
    const int lim_hi = bhi + 1 - (int)clt_hi;
    int tlo = 0, thi = 0;
    for (int base = 0; base < T; base += 32) {
      const int s = base + lane;
      const bool valid = s < T;
      const uint32_t k = valid ? kw[s * KS] : 0u;
      const bool eqlo = valid && k == Klo, eqhi = valid && k == Khi;
      const unsigned mlo = __ballot_sync(FULL, eqlo), mhi = __ballot_sync(FULL, eqhi);
      const int ilo = tlo + __popc(mlo & lt), ihi = thi + __popc(mhi & lt);
      const bool isb = valid && (k < Klo || (eqlo && ilo < need_lo));
      const bool isa = valid && !isb && (k > Khi || (eqhi && ihi >= lim_hi));
      const bool isc = valid && !isb && !isa;
      tlo += __popc(mlo);
      thi += __popc(mhi);
      const unsigned mc = __ballot_sync(FULL, isc), mb = __ballot_sync(FULL, isb);
      if (isc) {
        const int j = nc + __popc(mc & lt);
        if (j < B.cap) {
          ckey[j] = k;
          cs[j] = (uint16_t)s;
          cp_async4(&kcol[j * KS], evq + s);
        }
        cmin = min(cmin, k);
        cmax = max(cmax, k);
      }
      if (lane == 0) below[base >> 5] = mb;
      nc += __popc(mc);
    }
    nbelow = blo;
  }
  cmin = __reduce_min_sync(FULL, cmin);
  cmax = __reduce_max_sync(FULL, cmax);
  cp_async_wait_all();
  __syncwarp();
  bool ok = nc <= B.cap && nc >= nbd;

  // ---- counting sort of the candidates: rank in (key, frame) order --------
  int nbb = 0, nfix = 0;
  if (ok) {
    const float w0 = key2f(cmin);
    const float r2 = key2f(cmax) - w0;
    const float sc2 = (r2 > 0.f) ? 256.f / r2 : 0.f;
#pragma unroll
    for (int b = 0; b < 8; b++) hist[lane * 8 + b] = 0u;
    __syncwarp();
    for (int j = lane; j < nc; j += 32) atomicAdd(&hist[vbin(ckey[j], w0, sc2)], 1u);
    __syncwarp();
    hist_exclusive_scan(hist, lane);
#pragma unroll
    for (int b = 0; b < 8; b++) cur[lane * 8 + b] = hist[lane * 8 + b];
    __syncwarp();
    for (int j = lane; j < nc; j += 32) tmp[atomicAdd(&cur[vbin(ckey[j], w0, sc2)], 1u)] = (uint16_t)j;
    __syncwarp();
    uint32_t *skeys_g = reinterpret_cast<uint32_t *>(slot + L.skeys);
    uint32_t *blev_g = reinterpret_cast<uint32_t *>(slot + L.blev);
    uint16_t *blpos_g = reinterpret_cast<uint16_t *>(slot + L.blpos);
    const int off = nbelow - blo;   // value position = off + rank among the candidates
    for (int j0 = 0; j0 < nc; j0 += 32) {
      const int j = j0 + lane;
      bool inb = false;
      int pos = 0, s = 0;
      if (j < nc) {
        const uint32_t k = ckey[j];
        const int b = vbin(k, w0, sc2);
        const int st = (int)hist[b], en = (int)cur[b];
        int r = st;
        for (int x = st; x < en; x++) {
          const int j2 = tmp[x];
          const uint32_t k2 = ckey[j2];
          r += (k2 < k || (k2 == k && j2 < j)) ? 1 : 0;
        }
        pos = off + r;
        s = cs[j];
        if (pos < 0) {
          atomicOr(&below[s >> 5], 1u << (s & 31));
          nfix++;
        } else if (pos < nbd) {
          skeys_g[pos] = __float_as_uint(key2f(k));   // the sweep reads values
          inb = true;
        }
      }
      const unsigned mi = __ballot_sync(FULL, inb);
      if (inb) {
        const int jj = nbb + __popc(mi & lt);
        blpos_g[jj] = (uint16_t)pos;
        blev_g[jj] = kcol[j * KS];
      }
      nbb += __popc(mi);
    }
    nfix = __reduce_add_sync(FULL, nfix);
    ok = (nbb == nbd);
  }
  __syncwarp();
  uint32_t *below_g = reinterpret_cast<uint32_t *>(slot + L.below);
  for (int wd = lane; wd < B.nwt; wd += 32) below_g[wd] = below[wd];
  if (lane == 0) {
    *reinterpret_cast<int4 *>(slot) = make_int4(nbd, nbelow + nfix, ann, ok ? 1 : 0);
    if (!ok) atomicOr(a.status, STATUS_INTERNAL);
  }
}

// ---------------------------------------------------------------------------
// band_sweep_kernel
// ---------------------------------------------------------------------------

// Shared memory: per warp skeys[NB] u32, blev[NB] u32, bm[NB] u32 (bit map,
// word wd of lane c at wd * 32 + c), blpos[NB] u16, belowc[nwt + 1] uint2
// (BELOW word, BELOW frames before it); per CTA three value blocks (each
// replaced by its residuals in place).
// The gates (L_i, R_i) are read through L1 (a few KB per annulus, shared by
// every CTA of the annulus): measured faster than staging them, which cost
// resident CTAs.
__host__ __device__ inline size_t sweep_warp_bytes(int NB, int nwt) {
  return (size_t)NB * 12 + al16((size_t)NB * 2) + al16((size_t)(nwt + 1) * 8);
}
constexpr size_t kBlockBytes = (size_t)SWK * 32 * 16;   // [SWK][32 lanes] float4
__host__ __device__ inline size_t sweep_smem_bytes(int NB, int nwt, int T) {
  return PPC * sweep_warp_bytes(NB, nwt) + 3 * kBlockBytes;
}

template <int WC>
__global__ void __launch_bounds__(32 * PPC, (WC <= 8) ? 9 : (WC == 16 ? 4 : 2)) band_sweep_kernel(const BandArgs B) {
  extern __shared__ __align__(16) unsigned char ssm[];
  constexpr int NB = 32 * WC;
  const AdiArgs &a = B.a;
  const int T = a.T;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long p0 = (long long)__ldg(&B.groups[blockIdx.x]) * PPC;
  const int nwt = B.nwt;
  unsigned char *wb = ssm + (size_t)w * sweep_warp_bytes(NB, nwt);
  uint32_t *skeys = reinterpret_cast<uint32_t *>(wb);
  uint32_t *blev = skeys + NB;
  uint32_t *bm = blev + NB;
  uint16_t *blpos = reinterpret_cast<uint16_t *>(bm + NB);
  uint2 *belowc = reinterpret_cast<uint2 *>(wb + (size_t)NB * 12 + al16((size_t)NB * 2));
  unsigned char *cb_ = ssm + PPC * sweep_warp_bytes(NB, nwt);
  // [3][SWK][32] 16-byte rows: block b's values in buffer b % 3, replaced by
  // its residuals in place (each slot is read, then written, by one thread)
  float4 *vbuf = reinterpret_cast<float4 *>(cb_);

  // ---- this pixel's band data -------------------------------------------
  const char *slot = B.slots + ((size_t)blockIdx.x * PPC + w) * B.slot_bytes;
  const Slot SL(B.NB, nwt);
  const int4 hdr = *reinterpret_cast<const int4 *>(slot);
  const int nb = hdr.x, nbelow = hdr.y, ann = hdr.z;
  bool act = ann >= 0 && hdr.w == 1 && nb <= NB;
  if (act) {
    // band values, event queries and value positions: 16-byte asynchronous
    // copies (the arrays start on 16-byte boundaries in the slot and here;
    // whole pieces stay within the capacity NB)
    const int nk = (nb + 3) >> 2, np = (nb + 7) >> 3;
    for (int q = lane; q < 2 * nk + np; q += 32) {
      if (q < nk) cp_async16(skeys + 4 * q, slot + SL.skeys + 16 * q);
      else if (q < 2 * nk) cp_async16(blev + 4 * (q - nk), slot + SL.blev + 16 * (q - nk));
      else cp_async16(blpos + 8 * (q - 2 * nk), slot + SL.blpos + 16 * (q - 2 * nk));
    }
  }
  cp_async_commit();
  if (act) {
    // BELOW words and the BELOW frames before each (exclusive prefix)
    const uint32_t *bw = reinterpret_cast<const uint32_t *>(slot + SL.below);
    uint32_t carry = 0;
    for (int w0 = 0; w0 <= nwt; w0 += 32) {
      const int wd = w0 + lane;
      const uint32_t m = wd < nwt ? bw[wd] : 0u;
      const uint32_t c = __popc(m);
      uint32_t inc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += t;
      }
      if (wd <= nwt) belowc[wd] = make_uint2(m, carry + inc - c);
      carry += __shfl_sync(FULL, inc, 31);
    }
  }
  const int2 *gate_g = reinterpret_cast<const int2 *>(a.lr + (size_t)(ann < 0 ? 0 : ann) * T * 2);

  const int C = (T + 31) / 32;
  const int c = lane;
  const int i0 = c * C;
  const int i1 = min(T, i0 + C);
  const int nblk = (C + SWK - 1) / SWK;
  auto prefetch = [&](int b) {
    float4 *dst = vbuf + (b % 3) * SWK * 32;
    for (int q = threadIdx.x; q < SWK * 32; q += 32 * PPC) {
      const int kk = q >> 5, cc = q & 31;
      const int i = cc * C + b * SWK + kk;
      if (b * SWK + kk < C && i < T)
        cp_async16(dst + q, a.in + (long long)(a.perm_id ? i : __ldg(&a.perm[i])) * a.in_fs + p0);
    }
    cp_async_commit();
  };
  prefetch(0);

  // ---- start state of every lane: members at query i0 -------------------
  // band position p (value order) is a member at query c C unless its frame's
  // exclusion queries [a, b) hold c C, i.e. unless ceil(a/C) <= c < ceil(b/C):
  // one 32-bit chunk mask per position, transposed into the lanes' words
  cp_async_wait_group<1>();   // the band data (the first value block may still be in flight)
  __syncwarp();
  if (act) {
    for (int j = lane; j < nb; j += 32) bm[blpos[j]] = blev[j];   // event queries by value position
    __syncwarp();
#pragma unroll 1
    for (int wd = 0; wd < WC; wd++) {
      const int p = wd * 32 + lane;
      uint32_t m = 0u;
      if (p < nb) {
        const uint32_t ev = bm[p];
        const int ea = (int)(ev & 0xffffu), eb = (int)(ev >> 16);
        const int clo = (ea + C - 1) / C, chi = (eb + C - 1) / C;
        const uint32_t lo_mask = clo >= 32 ? 0xffffffffu : ((1u << clo) - 1u);
        const uint32_t hi_mask = chi >= 32 ? 0xffffffffu : ((1u << chi) - 1u);
        m = ~(hi_mask & ~lo_mask);
      }
      const uint32_t word = warp_transpose32(m, lane);
      bm[wd * 32 + lane] = word;
    }
    __syncwarp();
  }
  // next leave / enter events after i0: first members (frame order) whose
  // a (b) exceeds i0; a and b never decrease along the frame order
  int ja = nb, jb = nb;
  if (act) {
    int lo = 0, hi = nb;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((int)(blev[mid] & 0xffffu) > i0) hi = mid; else lo = mid + 1;
    }
    ja = lo;
    lo = 0;
    hi = nb;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((int)(blev[mid] >> 16) > i0) hi = mid; else lo = mid + 1;
    }
    jb = lo;
  }
  int na = ja < nb ? (int)(blev[ja] & 0xffffu) : 0x7fffffff;
  int nq = jb < nb ? (int)(blev[jb] >> 16) : 0x7fffffff;
  int ne = min(na, nq);   // query of the next event
  bool lane_ok = act && i0 < T;
  int wi = 0, base = 0;   // word of the current member, members in the words below it
  bool fail = false;
  // the gate of the lane's next query is loaded one query ahead
  int2 gnext = lane_ok ? __ldg(&gate_g[i0]) : make_int2(0, 0);

  // ---- sweep ------------------------------------------------------------
  // one barrier per block: after it block b's values are in and block b-1's
  // residuals are complete; block b+1's copies go to the third buffer, and
  // block b-1's residuals are written out while block b is swept
  auto store_block = [&](int bb) {
    const float4 *ob = vbuf + (bb % 3) * SWK * 32;
    for (int q = threadIdx.x; q < SWK * 32; q += 32 * PPC) {
      const int kk = q >> 5, cc = q & 31;
      const int i = cc * C + bb * SWK + kk;
      if (bb * SWK + kk < C && i < T)
        *reinterpret_cast<float4 *>(a.out + (long long)(a.perm_id ? i : __ldg(&a.perm[i])) * a.out_fs + p0) = ob[q];
    }
  };
  for (int b = 0; b < nblk; b++) {
    cp_async_wait_group<0>();
    __syncthreads();
    if (b + 1 < nblk) prefetch(b + 1);
    if (b > 0) store_block(b - 1);
    float *vb = reinterpret_cast<float *>(vbuf + (b % 3) * SWK * 32);
    for (int kk = 0; kk < SWK; kk++) {
      const int i = i0 + b * SWK + kk;
      if (b * SWK + kk >= C || i >= i1) break;
      float res = 0.0f;
      if (lane_ok) {
        const int2 gv = gnext;
        if (i + 1 < i1) gnext = __ldg(&gate_g[i + 1]);
        // events of query i, leaving (a == i) and entering (b == i) members
        // from one merged stream
        while (ne == i) {
          const bool leave = na == i;
          const int j = leave ? ja : jb;
          const int pos = blpos[j];
          const int wd = pos >> 5;
          bm[wd * 32 + c] ^= 1u << (pos & 31);
          base += (wd < wi) ? (leave ? -1 : 1) : 0;
          if (leave) {
            ja++;
            na = ja < nb ? (int)(blev[ja] & 0xffffu) : 0x7fffffff;
          } else {
            jb++;
            nq = jb < nb ? (int)(blev[jb] >> 16) : 0x7fffffff;
          }
          ne = min(na, nq);
        }
        const int Li = gv.x, Ri = gv.y;
        // BELOW members of S_i: BELOW frames before L_i and from R_i on
        const uint2 ul = belowc[Li >> 5], ur = belowc[Ri >> 5];
        const int bl = (int)ul.y + __popc(ul.x & ((1u << (Li & 31)) - 1u));
        const int br = (int)ur.y + __popc(ur.x & ((1u << (Ri & 31)) - 1u));
        const int cbm = bl + (nbelow - br);
        const int nset = Li + (T - Ri);
        const int t = ((nset - 1) >> 1) - cbm;
        uint32_t wd = bm[wi * 32 + c];
        int pc = __popc(wd);
        while (t < base && wi > 0) {
          wi--;
          wd = bm[wi * 32 + c];
          pc = __popc(wd);
          base -= pc;
        }
        while (t >= base + pc && wi + 1 < WC) {
          base += pc;
          wi++;
          wd = bm[wi * 32 + c];
          pc = __popc(wd);
        }
        if (t >= base && t < base + pc) {
          const int pos = nth_set(wd, t - base);
          float med = __uint_as_float(skeys[wi * 32 + pos]);
          // the next member, needed for an even |S_i| (found for every lane:
          // the lanes' parities differ, so a branch would run both ways):
          // a higher bit of this word, else the first of a later word
          uint32_t rest = pos < 31 ? (wd & (0xfffffffeu << pos)) : 0u;
          int wn = wi;
          while (rest == 0u && wn + 1 < WC) {
            wn++;
            rest = bm[wn * 32 + c];
          }
          const bool even = (nset & 1) == 0;
          const float hi = __uint_as_float(skeys[rest ? wn * 32 + __ffs(rest) - 1 : wi * 32 + pos]);
          if (even) {
            if (rest) med = (med + hi) * 0.5f;
            else fail = true;
          }
          res = vb[(kk * 32 + c) * 4 + w] - med;
        } else {
          fail = true;
        }
        if (fail) lane_ok = false;
      }
      vb[(kk * 32 + c) * 4 + w] = res;
    }
  }
  __syncthreads();   // the last block's residuals are complete
  if (nblk > 0) store_block(nblk - 1);
  if (ann >= 0 && (hdr.w != 1 || nb > NB)) fail = true;
  if (__any_sync(FULL, fail) && lane == 0) atomicOr(a.status, STATUS_INTERNAL);
}

// Groups without a pixel in an annulus: residual 0 in every frame.
__global__ void __launch_bounds__(128) band_zero_kernel(float *out, const int *groups, int T, long long out_fs) {
  const long long p0 = (long long)__ldg(&groups[blockIdx.x]) * PPC;
  for (int t = threadIdx.x; t < T; t += blockDim.x)
    *reinterpret_cast<float4 *>(out + (long long)t * out_fs + p0) = make_float4(0.f, 0.f, 0.f, 0.f);
}

int class_of_width(int W) { return W <= 1 ? 1 : W == 2 ? 2 : W == 4 ? 3 : W == 8 ? 4 : W == 16 ? 5 : 6; }

template <int WC>
cudaError_t launch_sweep(const BandArgs &b, int ngroups, cudaStream_t st) {
  const size_t smem = sweep_smem_bytes(32 * WC, b.nwt, b.a.T);
  cudaError_t e = cudaFuncSetAttribute(band_sweep_kernel<WC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  band_sweep_kernel<WC><<<(unsigned)ngroups, 32 * PPC, smem, st>>>(b);
  return cudaGetLastError();
}

// Group classes of a frame geometry, cached: the computation visits every
// pixel once, the plan of a repeated call is the same.
struct GroupKey {
  int n;
  std::vector<double> edge2;
  std::vector<int> width;
  bool operator<(const GroupKey &o) const {
    return std::tie(n, edge2, width) < std::tie(o.n, o.edge2, o.width);
  }
};
std::mutex g_group_mu;
struct GroupLists {
  std::vector<int> groups, class_off;
  int gen_off, gen_n;
};
std::map<GroupKey, GroupLists> g_group_cache;

}  // namespace

int plan_band_path(AdiPlanHost &ap, int64_t T, int32_t n) {
  const int A = (int)ap.edge2.size() - 1;
  ap.evq.clear();
  ap.groups.clear();
  ap.class_off.assign(NCLASS + 1, 0);
  ap.gen_off = -1;
  ap.gen_n = 0;
  if (ap.wmax == 0 || A <= 0) return GRAPHIC_OK;
  // event queries of every banded annulus: frame s is outside S_i for
  // a_s <= i < b_s (two pointers over the monotone gates)
  ap.evq.assign((size_t)A * T, 0u);
  for (int an = 0; an < A; an++) {
    if (ap.band[4 * an + 2] == 0) continue;
    const int *lr = ap.lr.data() + (size_t)an * T * 2;
    uint32_t *ev = ap.evq.data() + (size_t)an * T;
    int64_t ia = 0, ib = 0;
    for (int64_t s = 0; s < T; s++) {
      while (ia < T && lr[2 * ia + 1] <= s) ia++;   // first i with R_i > s
      while (ib < T && lr[2 * ib] <= s) ib++;       // first i with L_i > s
      ev[s] = (uint32_t)ia | ((uint32_t)ib << 16);
    }
  }
  GroupKey key{n, ap.edge2, {}};
  for (int an = 0; an < A; an++) key.width.push_back(ap.band[4 * an + 2]);
  {
    std::lock_guard<std::mutex> lk(g_group_mu);
    auto it = g_group_cache.find(key);
    if (it != g_group_cache.end()) {
      ap.groups = it->second.groups;
      ap.class_off = it->second.class_off;
      ap.gen_off = it->second.gen_off;
      ap.gen_n = it->second.gen_n;
      return GRAPHIC_OK;
    }
  }
  const int64_t NN = (int64_t)n * n;
  std::vector<std::vector<int>> lists(NCLASS);
  std::vector<int> gen_blocks;   // 8-pixel blocks of the general path
  for (int64_t g = 0; g < NN / PPC; g++) {
    int cls = 0;
    bool general = false;
    for (int q = 0; q < PPC; q++) {
      const int64_t p = g * PPC + q;
      const int64_t x = (p % n) - n / 2, y = (p / n) - n / 2;
      const double rho2 = (double)(x * x + y * y);
      int an = -1;
      for (int k = 0; k < A; k++)
        if (ap.edge2[k] <= rho2 && rho2 < ap.edge2[k + 1]) {
          an = k;
          break;
        }
      if (an < 0) continue;
      const int W = ap.band[4 * an + 2];
      if (W == 0) general = true;
      else cls = std::max(cls, class_of_width(W));
    }
    if (!general) lists[cls].push_back((int)g);
    else if (gen_blocks.empty() || gen_blocks.back() != (int)(g / 2)) gen_blocks.push_back((int)(g / 2));
  }
  for (int k = 0; k < NCLASS; k++) {
    ap.class_off[k] = (int)ap.groups.size();
    ap.groups.insert(ap.groups.end(), lists[k].begin(), lists[k].end());
  }
  ap.class_off[NCLASS] = (int)ap.groups.size();
  ap.gen_off = (int)ap.groups.size();
  ap.gen_n = (int)gen_blocks.size();
  ap.groups.insert(ap.groups.end(), gen_blocks.begin(), gen_blocks.end());
  std::lock_guard<std::mutex> lk(g_group_mu);
  if (g_group_cache.size() > 16) g_group_cache.clear();
  g_group_cache[key] = {ap.groups, ap.class_off, ap.gen_off, ap.gen_n};
  return GRAPHIC_OK;
}

size_t band_scratch_bytes(const AdiPlanHost &ap, int64_t T) {
  if (ap.class_off.size() != NCLASS + 1) return 0;
  const int nwt = (int)((T + 31) / 32);
  size_t bytes = 0, one = 0;
  for (int k = 1; k < NCLASS; k++) {
    const size_t ng = (size_t)(ap.class_off[k + 1] - ap.class_off[k]);
    const size_t g = PPC * Slot(32 * kClassW[k], nwt).bytes;
    bytes = std::max(bytes, ng * g);   // classes run one after the other
    if (ng) one = std::max(one, g);
  }
  return std::max(one, std::min(bytes, kBandScratchMax));
}

cudaError_t launch_adi_band(const AdiArgs &a, cudaStream_t st, int *launched) {
  int dummy = 0;
  int &nl = launched ? *launched : dummy;
  const int T = a.T;
  const int nwt = (T + 31) / 32;
  const int *off = a.class_off;
  auto mark = [&](int kind, int begin) {
    if (a.mark) a.mark(a.mark_user, kind, begin);
  };
  if (off[1] > off[0]) {
    mark(1, 1);
    band_zero_kernel<<<(unsigned)(off[1] - off[0]), 128, 0, st>>>(a.out, a.groups + off[0], T, a.out_fs);
    cudaError_t e = cudaGetLastError();
    mark(1, 0);
    if (e != cudaSuccess) return e;
    nl++;
  }
  for (int k = 1; k < NCLASS; k++) {
    const int ngk = off[k + 1] - off[k];
    if (ngk == 0) continue;
    BandArgs b{};
    b.a = a;
    b.evq = a.evq;
    b.slots = a.band_scratch;
    b.NB = 32 * kClassW[k];
    b.nwt = nwt;
    b.slot_bytes = Slot(b.NB, nwt).bytes;
    // candidates: the band (more than NB / 2 ranks) and the spill of its two
    // end bins (a few dozen keys), at most T; then as many more as fit the
    // shared memory without costing a resident CTA (a pixel whose located
    // bins hold more takes the exact path)
    b.cap = std::min(T, b.NB + std::max(64, b.NB / 4));
    {
      int dev = 0, per_sm = 0;
      if (cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
          per_sm > 0) {
        const size_t reserve = 1024;   // per resident CTA
        auto ctas = [&](int c) { return (size_t)per_sm / (prep_smem_bytes(T, c, nwt) + reserve); };
        const size_t occ = ctas(b.cap);
        while (b.cap + 32 <= T && ctas(b.cap + 32) == occ && prep_smem_bytes(T, b.cap + 32, nwt) <= 227 * 1024)
          b.cap += 32;
      }
    }
    const size_t psmem = prep_smem_bytes(T, b.cap, nwt);
    cudaError_t e = cudaFuncSetAttribute(band_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    if (e != cudaSuccess) return e;
    // the class's groups in chunks whose tables fit the scratch
    const int per = (int)std::min<size_t>((size_t)ngk, a.band_scratch_cap / (PPC * b.slot_bytes));
    if (per < 1) return cudaErrorInvalidValue;
    for (int g0 = 0; g0 < ngk; g0 += per) {
      const int ng = std::min(per, ngk - g0);
      b.groups = a.groups + off[k] + g0;
      mark(1, 1);
      band_prep_kernel<<<(unsigned)ng, 32 * PPC, psmem, st>>>(b);
      e = cudaGetLastError();
      mark(1, 0);
      if (e != cudaSuccess) return e;
      nl++;
      mark(2, 1);
      switch (kClassW[k]) {
        case 1: e = launch_sweep<1>(b, ng, st); break;
        case 2: e = launch_sweep<2>(b, ng, st); break;
        case 4: e = launch_sweep<4>(b, ng, st); break;
        case 8: e = launch_sweep<8>(b, ng, st); break;
        case 16: e = launch_sweep<16>(b, ng, st); break;
        default: e = launch_sweep<32>(b, ng, st); break;
      }
      mark(2, 0);
      if (e != cudaSuccess) return e;
      nl++;
    }
  }
  return cudaSuccess;
}

}  // namespace graphic

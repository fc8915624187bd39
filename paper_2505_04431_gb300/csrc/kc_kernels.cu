// kc_kernels.cu - the k-mer counting hot path on sm_103a.
//
// Phase 1 (Section III-C, Algorithm 3 first loop; Section V "Phase 1"):
//   pass A  k_pack_count    ASCII -> 2-bit codes + invalid mask (the paper's Encode),
//                           rolling forward / reverse-complement keys (Algorithm 1's
//                           kmer = (kmer << 2) OR Encode), owner partition of every
//                           valid window, per-tile partition histogram.
//   scans   k_col_scan, k_bucket_scan   exact write offsets per (tile, partition).
//   pass B  k_scatter       recomputes the keys from the packed codes and writes each
//                           key to its owner partition.  A tile's keys are first
//                           grouped per partition in shared memory (a counting sort)
//                           and leave in contiguous runs: this block-level staging is
//                           the GPU form of the per-destination L2 buffers of
//                           Section IV-C / Algorithm 4 (AddToL2Buffer), which exist to
//                           turn many small sends into few large ones.
// Phase 2 (Algorithm 3 after the barrier: Sort + Accumulate; Section V "Phase 2"):
//   k_fine_hist, k_fine_scan, k_fine_scatter   split every owner partition into fine
//                           partitions small enough for one shared-memory table.
//   k_count_emit            per fine partition: insert every key into an
//                           order-preserving open-addressing table in shared memory
//                           (CAS claims the slot, a 32-bit atomic add counts; a warp
//                           whose 32 keys are equal adds once, the warp-level form of
//                           the heavy-hitter pre-aggregation of Section IV-D), sort the
//                           few keys displaced by collisions, and emit the sorted
//                           (key, count) run at the offset found by a decoupled
//                           look-back over the fine partitions.
//
// Owner partitions are key ranges (not hashes) so that the per-partition outputs
// concatenate into one ascending array.  A monotone map u(key) from the top 64 key
// bits flattens the distribution of canonical keys (min of two near-independent
// uniforms has density 2(1-x); u = 1 - (1-x)^2 is its distribution function), and
// coarse partition, fine partition and table home slot are consecutive bit fields
// of u, so every one of them is non-decreasing in the key.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kc_internal.h"

namespace kc {

typedef unsigned __int128 u128;

template <int KW> struct KeyT;
template <> struct KeyT<1> { typedef uint64_t T; };
template <> struct KeyT<2> { typedef u128 T; };

// ------------------------------------------------------------------ bit helpers
__device__ __forceinline__ uint64_t revpairs64(uint64_t x) {
  x = __brevll(x);
  return ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
}
__device__ __forceinline__ uint64_t key_mask(uint64_t, int k) { return k >= 32 ? ~0ull : ((1ull << (2 * k)) - 1); }
__device__ __forceinline__ u128 key_mask(u128, int k) { return k >= 64 ? ~(u128)0 : (((u128)1 << (2 * k)) - 1); }
// value of the reverse complement of the k-mer v (digit d -> 3 - d, digit order reversed)
__device__ __forceinline__ uint64_t revcomp(uint64_t v, int k) { return revpairs64(~v) >> (64 - 2 * k); }
__device__ __forceinline__ u128 revcomp(u128 v, int k) {
  u128 r = ((u128)revpairs64(~(uint64_t)v) << 64) | revpairs64(~(uint64_t)(v >> 64));
  return r >> (128 - 2 * k);
}
template <class K> __device__ __forceinline__ K all_ones() { return ~(K)0; }

__device__ __forceinline__ uint64_t shfl_key(uint64_t v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ u128 shfl_key(u128 v, int src) {
  uint64_t lo = __shfl_sync(0xffffffffu, (uint64_t)v, src);
  uint64_t hi = __shfl_sync(0xffffffffu, (uint64_t)(v >> 64), src);
  return ((u128)hi << 64) | lo;
}

// Look-back status words carry their own payload (flag and value in one 64-bit word) and
// guard no other data, so relaxed GPU-scope accesses are enough.
__device__ __forceinline__ void st_status(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_status(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ u128 cas128_shared(u128* p, u128 cmp, u128 val) {
  uint64_t clo = (uint64_t)cmp, chi = (uint64_t)(cmp >> 64), vlo = (uint64_t)val, vhi = (uint64_t)(val >> 64), olo, ohi;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile(
      "{\n\t.reg .b128 d, c, v;\n\tmov.b128 c, {%2, %3};\n\tmov.b128 v, {%4, %5};\n\t"
      "atom.shared.cas.b128 d, [%6], c, v;\n\tmov.b128 {%0, %1}, d;\n\t}"
      : "=l"(olo), "=l"(ohi)
      : "l"(clo), "l"(chi), "l"(vlo), "l"(vhi), "r"(a)
      : "memory");
  return ((u128)ohi << 64) | olo;
}

__device__ __forceinline__ void store_key(uint64_t* dst, uint64_t i, uint64_t key) { dst[i] = key; }
__device__ __forceinline__ void store_key(uint64_t* dst, uint64_t i, u128 key) {
  reinterpret_cast<ulonglong2*>(dst)[i] = make_ulonglong2((uint64_t)key, (uint64_t)(key >> 64));
}
__device__ __forceinline__ void load_key(const uint64_t* src, uint64_t i, uint64_t& key) { key = src[i]; }
__device__ __forceinline__ void load_key(const uint64_t* src, uint64_t i, u128& key) {
  const ulonglong2 v = reinterpret_cast<const ulonglong2*>(src)[i];
  key = ((u128)v.y << 64) | v.x;
}

// Block-wide exclusive scan of n values in shared memory (in place); returns the total.
// All threads of the block must call it.  `warp_tmp` holds 32 entries.
template <typename T>
__device__ T block_exclusive_scan(T* data, int n, T* warp_tmp) {
  const int nt = blockDim.x, t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = (nt + 31) >> 5;
  const int per = (n + nt - 1) / nt;
  const int lo = min(n, t * per), hi = min(n, lo + per);
  T s = 0;
  for (int i = lo; i < hi; ++i) s += data[i];
  T x = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tmp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = lane < nw ? warp_tmp[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < nw) warp_tmp[lane] = w;  // inclusive per warp
  }
  __syncthreads();
  T run = x - s + (wid ? warp_tmp[wid - 1] : 0);
  const T total = warp_tmp[nw - 1];
  for (int i = lo; i < hi; ++i) {
    T v = data[i];
    data[i] = run;
    run += v;
  }
  __syncthreads();
  return total;
}

// Shared arrays that are scanned by contiguous per-thread chunks are padded (one word per
// 32) so that those chunks fall in distinct banks.
__host__ __device__ __forceinline__ uint32_t PAD(uint32_t i) { return i + (i >> 5); }
__host__ __device__ __forceinline__ size_t padded_len(size_t n) { return n + (n >> 5) + 1; }

// block_exclusive_scan over a padded array (logical element i at data[PAD(i)]).
template <typename T>
__device__ T block_exclusive_scan_pad(T* data, int n, T* warp_tmp) {
  const int nt = blockDim.x, t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = (nt + 31) >> 5;
  const int per = (n + nt - 1) / nt;
  const int lo = min(n, t * per), hi = min(n, lo + per);
  T s = 0;
  for (int i = lo; i < hi; ++i) s += data[PAD(i)];
  T x = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tmp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = lane < nw ? warp_tmp[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < nw) warp_tmp[lane] = w;
  }
  __syncthreads();
  T run = x - s + (wid ? warp_tmp[wid - 1] : 0);
  const T total = warp_tmp[nw - 1];
  for (int i = lo; i < hi; ++i) {
    T v = data[PAD(i)];
    data[PAD(i)] = run;
    run += v;
  }
  __syncthreads();
  return total;
}

// ------------------------------------------------------------------ input checks
__global__ void k_check_offsets(const uint64_t* offsets, uint64_t n_reads, Meta* meta) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_reads; i += (uint64_t)gridDim.x * blockDim.x) {
    if (offsets[i + 1] < offsets[i]) atomicOr(&meta->status, ST_BAD_OFFSETS);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && offsets[0] != 0) atomicOr(&meta->status, ST_BAD_OFFSETS);
}

// first read whose start is >= the halo start of each tile (lower bound in offsets)
__global__ void k_tile_first(const uint64_t* offsets, uint64_t n_reads, uint64_t n_tiles, uint64_t* tile_first) {
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  const uint64_t pos = t * kTileBases;
  const uint64_t halo = pos >= 64 ? pos - 64 : 0;
  uint64_t lo = 0, hi = n_reads;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (offsets[mid] < halo) lo = mid + 1; else hi = mid;
  }
  tile_first[t] = lo;
}

// ------------------------------------------------------------------ phase 1 helpers
// ASCII -> codes for 32 bytes given as 8 little-endian words.
__device__ __forceinline__ void pack32(const uint32_t w[8], uint64_t& code, uint32_t& inv) {
  uint64_t c = 0;
  uint32_t v = 0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const uint32_t x = w[m];
    const uint32_t c4 = ((x >> 1) ^ (x >> 2)) & 0x03030303u;  // A0 C1 G2 T3 (either case)
    const uint32_t g = ((c4 << 6) & 0xC0u) | ((c4 >> 4) & 0x30u) | ((c4 >> 14) & 0x0Cu) | ((c4 >> 24) & 0x03u);
    c |= (uint64_t)g << (56 - 8 * m);
    const uint32_t lc = x | 0x20202020u;
    const uint32_t ok = __vcmpeq4(lc, 0x61616161u) | __vcmpeq4(lc, 0x63636363u) | __vcmpeq4(lc, 0x67676767u) |
                        __vcmpeq4(lc, 0x74747474u);
    const uint32_t bad = ~ok & 0x80808080u;
    v |= (((bad >> 7) & 1u) | ((bad >> 14) & 2u) | ((bad >> 21) & 4u) | ((bad >> 28) & 8u)) << (4 * m);
  }
  code = c;
  inv = v;
}

// Convert code word w (bases 32w .. 32w+31) straight from the reads.
__device__ __forceinline__ void convert_word(const uint8_t* reads, uint64_t L, uint64_t w, uint64_t& code, uint32_t& inv) {
  const uint64_t p = w * 32;
  uint32_t x[8];
  if (p + 32 <= L) {
    const uint4* src = reinterpret_cast<const uint4*>(reads + p);
    const uint4 a = __ldcs(src), b2 = __ldcs(src + 1);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b2.x; x[5] = b2.y; x[6] = b2.z; x[7] = b2.w;
    pack32(x, code, inv);
  } else {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      uint32_t v = 0;
      for (int r = 0; r < 4; ++r) {
        const uint64_t q = p + 4 * m + r;
        v |= (uint32_t)(q < L ? reads[q] : 0) << (8 * r);
      }
      x[m] = v;
    }
    pack32(x, code, inv);  // byte 0 is not a base, so the tail past L is invalid
  }
}

// Mark read starts inside the slot window [j0-2, j0+nw) of a sub-step in st_s; advance *rcur
// to the first read whose start is >= the next sub-step's halo.  All threads call it.
__device__ void build_starts(const uint64_t* offsets, uint64_t n_reads, uint64_t j0, int nw, uint32_t* st_s,
                             uint64_t* rcur_s) {
  const int t = threadIdx.x, nt = blockDim.x;
  const int64_t st0 = (int64_t)j0 * 32 - 64;
  const uint64_t end = (j0 + nw) * 32;
  const int64_t next_halo = (int64_t)end - 64;
  uint64_t base = *rcur_s;
  uint64_t adv = 0;
  while (true) {
    const uint64_t i = base + t;
    const uint64_t p = i < n_reads ? offsets[i] : ~0ull;
    if (p < end) {
      const int64_t rel = (int64_t)p - st0;
      if (rel >= 0 && rel < (int64_t)(nw + 2) * 32) atomicOr(&st_s[rel >> 5], 1u << (rel & 31));
    }
    const int nb = __syncthreads_count(p != ~0ull && (int64_t)p < next_halo);
    const int ne = __syncthreads_count(p < end);
    adv += nb;
    if (ne < nt) break;
    base += nt;
  }
  if (t == 0) *rcur_s += adv;
}

// The range map: coarse partition, fine partition are bit fields of a 32-bit value u,
// non-decreasing in the key.  x = top 32 bits of the 2k-bit key; canonical keys are the
// min of two near-independent uniforms (density 2(1-x)), so u = 1 - (1-x)^2 (its
// distribution function) spreads them evenly.
__device__ __forceinline__ uint32_t top32_of(uint64_t key, int k) { return (uint32_t)((key << (64 - 2 * k)) >> 32); }
__device__ __forceinline__ uint32_t top32_of(u128 key, int k) { return (uint32_t)(key >> (2 * k - 32)); }
__device__ __forceinline__ uint32_t umap(uint32_t x, int canonical) {
  if (!canonical) return x;
  const uint32_t y = ~x;
  return ~__umulhi(y, y);
}
__device__ __forceinline__ uint32_t field32(uint32_t u, int skip, int bits) {
  const uint32_t v = skip >= 32 ? 0u : (u << skip);
  return bits ? v >> (32 - bits) : 0u;
}
template <class K>
__device__ __forceinline__ uint32_t coarse_of(K key, int k, int canonical, int b1) {
  return field32(umap(top32_of(key, k), canonical), 0, b1);
}

// Windows of one thread: WPT consecutive window ends starting at base q0 (q0 = 32j for
// WPT == 32; q0 = 32j + 16h for WPT == 16).  With the base stream S aligned so that window
// i's first base is S's base i, window i's forward key is the top 2k bits of S << 2i and
// its reverse complement the top 2k bits of R << 2(WPT-1-i), R being the complemented
// bases in reverse order.  Both shifts are compile-time constants once the loop over i is
// unrolled.  Values are kept top-aligned (key << (64 or 128) - 2k), so the top 32 bits
// that drive the range map come for free.
struct Win {
  uint64_t s0, s1, s2;  // S, left-aligned (192 bits; only s0, s1 used for k <= 32)
  uint64_t r0, r1, r2;  // R, left-aligned
  uint64_t m0, m1;      // mask of the top 2k bits (m1 used for k > 32)
  uint32_t valid;       // bit i: window i has k bases in ACGTacgt and no read start inside
};

__device__ __forceinline__ uint64_t shl128_hi(uint64_t a, uint64_t b, int sh) {  // top word of (a:b) << sh, 0 <= sh <= 64
  return sh == 0 ? a : (sh >= 64 ? b : (a << sh) | (b >> (64 - sh)));
}

// Mask of valid window ends for the 32 bases of word j: bit e (0..31) is set iff the k
// bases ending at 32j + e are all bases (inv clear) and no read starts at any of the last
// k - 1 of them.  inv / starts over words j-2, j-1, j as one 96-bit value, LSB = base 32j-64.
__device__ __forceinline__ uint32_t valid_mask(uint32_t i2, uint32_t i1, uint32_t i0, uint32_t t2, uint32_t t1,
                                               uint32_t t0, int k) {
  const u128 I = (u128)i2 | ((u128)i1 << 32) | ((u128)i0 << 64);
  const u128 S = (u128)t2 | ((u128)t1 << 32) | ((u128)t0 << 64);
  // a read start at base p forbids windows holding p-1 and p: mark base p-1 (C = I | S >> 1)
  // window [e-k+1, e] is valid iff C has no bit in [e-k+1, e-1] and I has no bit at e
  u128 bad = I;
  const int w = k - 1;
  if (w > 0) {
    const u128 C = I | (S >> 1);
    u128 Y = C;  // OR over a window of width 2^p ending at each bit
    int p = 1;
    while (2 * p <= w) {
      Y |= Y << p;
      p *= 2;
    }
    if (w > p) Y |= Y << (w - p);  // width w
    bad |= Y << 1;                 // windows ending at e look at C bits e-1 .. e-w
  }
  return ~(uint32_t)(bad >> 64);
}

template <int KW, int WPT>
__device__ __forceinline__ void win_setup(uint64_t w2, uint64_t w1, uint64_t w0, uint32_t vmask_word, int h, int k,
                                          Win& W) {
  // (w2 : w1 : w0) holds bases 32j-64 .. 32j+31; the first window's first base is
  // q0 - k + 1 = 32j + 16h - k + 1, at index 65 + 16h - k of that string.
  const int off = 65 + 16 * h - k;  // base index, >= 1
  const int sh = 2 * off;           // bits to drop from the top, 2 .. 162
  if (sh >= 128) {
    W.s0 = w0 << (sh - 128);
    W.s1 = 0;
    W.s2 = 0;
  } else if (sh >= 64) {
    W.s0 = shl128_hi(w1, w0, sh - 64);
    W.s1 = (sh - 64 == 0) ? w0 : w0 << (sh - 64);
    W.s2 = 0;
  } else {
    W.s0 = shl128_hi(w2, w1, sh);
    W.s1 = shl128_hi(w1, w0, sh);
    W.s2 = w0 << sh;
  }
  // R: complements of bases 32j+31 down to 32j-64; window i's reverse complement starts at
  // base q0 + i, i.e. at index 31 - 16h - i of R, so align R to index 31 - 16h - (WPT - 1).
  const uint64_t r0 = revpairs64(~w0), r1 = revpairs64(~w1), r2 = revpairs64(~w2);
  const int rsh = 2 * (32 - 16 * h - WPT);  // 0 (WPT 32 or h 1) or 32 (WPT 16, h 0)
  W.r0 = shl128_hi(r0, r1, rsh);
  W.r1 = shl128_hi(r1, r2, rsh);
  W.r2 = rsh ? r2 << rsh : r2;
  if (KW == 1) {
    W.m0 = k >= 32 ? ~0ull : ~(~0ull >> (2 * k));
    W.m1 = 0;
  } else {
    W.m0 = ~0ull;
    W.m1 = k >= 64 ? ~0ull : ~(~0ull >> (2 * k - 64));
  }
  W.valid = vmask_word >> (16 * h);
}

// Window i: the canonical value, top-aligned (top 64 bits in c0, next 64 in c1 for k > 32).
template <int KW, int WPT>
__device__ __forceinline__ void win_top(const Win& W, int i, int canonical, uint64_t& c0, uint64_t& c1) {
  const int fs = 2 * i, rs = 2 * (WPT - 1 - i);
  if constexpr (KW == 1) {
    const uint64_t f = shl128_hi(W.s0, W.s1, fs) & W.m0;
    const uint64_t r = shl128_hi(W.r0, W.r1, rs) & W.m0;
    c0 = (canonical && r < f) ? r : f;
    c1 = 0;
  } else {
    const uint64_t f0 = shl128_hi(W.s0, W.s1, fs), f1 = shl128_hi(W.s1, W.s2, fs) & W.m1;
    const uint64_t r0 = shl128_hi(W.r0, W.r1, rs), r1 = shl128_hi(W.r1, W.r2, rs) & W.m1;
    const bool rlt = canonical && ((r0 < f0) || (r0 == f0 && r1 < f1));
    c0 = rlt ? r0 : f0;
    c1 = rlt ? r1 : f1;
  }
}
__device__ __forceinline__ void top_to_key(uint64_t c0, uint64_t, int k, uint64_t& key) {
  key = k >= 32 ? c0 : c0 >> (64 - 2 * k);
}
__device__ __forceinline__ void top_to_key(uint64_t c0, uint64_t c1, int k, u128& key) {
  const u128 c = ((u128)c0 << 64) | c1;
  key = k >= 64 ? c : c >> (128 - 2 * k);
}

// ------------------------------------------------------------------ pass A
// One code word per thread: convert, store, and histogram the coarse partitions of its 32
// windows (keys are recomputed in pass B, which needs the partition offsets first).
template <int KW>
__global__ void __launch_bounds__(kPackThreads, KW == 1 ? 2 : 1) k_pack_count(Shape s, Buffers b) {
  typedef typename KeyT<KW>::T K;
  extern __shared__ uint32_t hist_s[];  // [P1]
  __shared__ uint64_t code_s[kPackThreads + 2];
  __shared__ uint32_t inv_s[kPackThreads + 2];
  __shared__ uint32_t st_s[kPackThreads + 2];
  __shared__ uint64_t rcur_s;
  const int t = threadIdx.x;
  const int P1 = 1 << s.b1;
  const uint64_t tile = blockIdx.x;
  for (int c = t; c < P1; c += kPackThreads) hist_s[c] = 0;
  if (t == 0) rcur_s = b.tile_first[tile];
  for (int sub = 0; sub < kTileWords / kPackThreads; ++sub) {
    const uint64_t j0 = tile * kTileWords + (uint64_t)sub * kPackThreads;
    if (j0 >= s.n_words) break;
    __syncthreads();
    if (t < 2) {
      if (sub > 0) {
        code_s[t] = code_s[kPackThreads + t];
        inv_s[t] = inv_s[kPackThreads + t];
      } else if (j0 + t >= 2) {
        convert_word(b.reads, s.L, j0 + t - 2, code_s[t], inv_s[t]);
      } else {
        code_s[t] = 0;
        inv_s[t] = ~0u;
      }
    }
    const uint64_t j = j0 + t;
    uint64_t code = 0;
    uint32_t inv = ~0u;
    if (j < s.n_words) {
      convert_word(b.reads, s.L, j, code, inv);
      b.codes64[j] = code;
      b.inv32[j] = inv;
    }
    __syncthreads();
    code_s[t + 2] = code;
    inv_s[t + 2] = inv;
    st_s[t + 2] = 0;
    if (t < 2) st_s[t] = 0;
    __syncthreads();
    build_starts(b.offsets, s.n_reads, j0, kPackThreads, st_s, &rcur_s);
    __syncthreads();
    if (j < s.n_words) {
      Win W;
      const uint32_t vm = valid_mask(inv_s[t], inv_s[t + 1], inv, st_s[t], st_s[t + 1], st_s[t + 2], s.k);
      win_setup<KW, 32>(code_s[t], code_s[t + 1], code, vm, 0, s.k, W);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        if ((W.valid >> i) & 1u) {
          uint64_t c0, c1;
          win_top<KW, 32>(W, i, s.canonical, c0, c1);
          atomicAdd(&hist_s[field32(umap((uint32_t)(c0 >> 32), s.canonical), 0, s.b1)], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (int c = t; c < P1; c += kPackThreads) b.hist[tile * P1 + c] = hist_s[c];
}

// ------------------------------------------------------------------ scans
// Column scan of hist[tile][c]: toff[tile][c] = keys of partition c in tiles before `tile`.
__global__ void k_col_scan(const uint32_t* hist, uint64_t* toff, uint64_t* ccount, uint64_t n_tiles, int P1) {
  __shared__ uint64_t part[32][33];
  const int lane = threadIdx.x, w = threadIdx.y;
  const int c = blockIdx.x * 32 + lane;
  const uint64_t per = (n_tiles + 31) / 32;
  const uint64_t lo = min(n_tiles, (uint64_t)w * per), hi = min(n_tiles, lo + per);
  uint64_t s = 0;
  if (c < P1)
    for (uint64_t t = lo; t < hi; ++t) s += hist[t * P1 + c];
  part[w][lane] = s;
  __syncthreads();
  if (w == 0) {
    uint64_t run = 0;
    for (int ww = 0; ww < 32; ++ww) {
      const uint64_t x = part[ww][lane];
      part[ww][lane] = run;
      run += x;
    }
    if (c < P1) ccount[c] = run;
  }
  __syncthreads();
  if (c < P1) {
    uint64_t run = part[w][lane];
    for (uint64_t t = lo; t < hi; ++t) {
      toff[t * P1 + c] = run;
      run += hist[t * P1 + c];
    }
  }
}

// Partition starts and the total number of windows.  One block.
__global__ void k_bucket_scan(const uint64_t* ccount, uint64_t* cstart, int P1, Meta* meta) {
  extern __shared__ uint64_t sc[];  // [P1]
  __shared__ uint64_t wt[32];
  for (int c = threadIdx.x; c < P1; c += blockDim.x) {
    const uint64_t n = ccount[c];
    sc[c] = n;
    if (n > 0xffffffffull) atomicOr(&meta->status, ST_PARTITION_OVERFLOW);  // pass B keeps 32-bit cursors
  }
  __syncthreads();
  const uint64_t K = block_exclusive_scan<uint64_t>(sc, P1, wt);
  for (int c = threadIdx.x; c < P1; c += blockDim.x) cstart[c] = sc[c];
  if (threadIdx.x == 0) {
    cstart[P1] = K;
    meta->n_windows = K;
  }
}

// Fine split of every coarse partition, after pass B: the distinct-key estimate (a sampled
// HyperLogLog filled by pass B) gives the duplication factor K / D, and a fine partition
// aims at fine_target distinct keys, i.e. fine_target * K / D keys.  One block.
__global__ void k_fine_plan(const uint64_t* cstart, const uint32_t* hll, uint32_t* fine_base, uint8_t* fine_log2, int P1,
                            uint32_t fine_target, uint32_t nf_max, Meta* meta) {
  extern __shared__ uint64_t fsc[];  // [P1]
  __shared__ uint64_t wt[32];
  __shared__ float zsum_s[32], zeros_s[32];
  __shared__ double target_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // HyperLogLog estimate over the 1/8 hash-sample of the keys
  float z = 0.f, zeros = 0.f;
  for (int i = threadIdx.x; i < kHllRegs; i += blockDim.x) {
    const uint32_t r = hll[i];
    z += exp2f(-(float)r);
    zeros += r == 0 ? 1.f : 0.f;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    z += __shfl_xor_sync(0xffffffffu, z, d);
    zeros += __shfl_xor_sync(0xffffffffu, zeros, d);
  }
  if (lane == 0) {
    zsum_s[wid] = z;
    zeros_s[wid] = zeros;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double zs = 0, zr = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      zs += zsum_s[w];
      zr += zeros_s[w];
    }
    const double m = kHllRegs;
    double e = 0.7213 / (1.0 + 1.079 / m) * m * m / zs;
    if (e < 2.5 * m && zr > 0) e = m * log(m / zr);
    const double d_est = e * kHllSample;
    const double K = (double)cstart[P1];
    double dup = d_est > 1.0 ? K / d_est : 1.0;
    dup = dup < 1.0 ? 1.0 : (dup > 32.0 ? 32.0 : dup);
    target_s = (double)fine_target * (0.8 * dup > 1.0 ? 0.8 * dup : 1.0);
    meta->d_estimate = (uint64_t)d_est;
  }
  __syncthreads();
  const double target = target_s;
  for (int c = threadIdx.x; c < P1; c += blockDim.x) {
    const uint64_t n = cstart[c + 1] - cstart[c];
    const uint64_t m = (uint64_t)ceil((double)n / target);
    int bf = m <= 1 ? 0 : 64 - __clzll(m - 1);
    bf = min(bf, kMaxFineLog2);
    fine_log2[c] = (uint8_t)bf;
    fsc[c] = 1ull << bf;
  }
  __syncthreads();
  const uint64_t NF = block_exclusive_scan<uint64_t>(fsc, P1, wt);
  for (int c = threadIdx.x; c < P1; c += blockDim.x) fine_base[c] = (uint32_t)fsc[c];
  if (threadIdx.x == 0) {
    fine_base[P1] = (uint32_t)NF;
    meta->n_fine = NF <= nf_max ? NF : 0;  // later kernels never index past nf_max
    if (NF > nf_max) atomicOr(&meta->status, ST_INTERNAL);
  }
}

// ------------------------------------------------------------------ pass B
// Per sub-step, NT threads x WPT windows: every key is computed once and kept in registers,
// its rank inside its partition taken with a shared-memory atomic (counting sort, step 1);
// after the block scan of the partition histogram the keys go to their partition's run in
// the staging buffer, and the runs leave in order.  A 1/8 hash sample of the keys feeds a
// HyperLogLog sketch (distinct-key estimate for sizing the fine partitions).
__device__ __forceinline__ uint64_t key_hash(uint64_t key) { return key * 0x9E3779B97F4A7C15ull; }
__device__ __forceinline__ uint64_t key_hash(u128 key) {
  return ((uint64_t)key ^ ((uint64_t)(key >> 64) * 0xC2B2AE3D27D4EB4Full)) * 0x9E3779B97F4A7C15ull;
}

template <int KW, int NT>
__global__ void __launch_bounds__(NT, 2) k_scatter(Shape s, Buffers b) {
  typedef typename KeyT<KW>::T K;
  constexpr int WPT = KW == 1 ? 32 : 16;    // windows per thread
  constexpr int TPW = 32 / WPT;             // threads per code word
  constexpr int NW = NT / TPW;              // code words per sub-step
  constexpr int SUB = NT * WPT;             // windows per sub-step
  extern __shared__ __align__(16) uint8_t sm[];
  const int P1 = 1 << s.b1;
  K* stage = reinterpret_cast<K*>(sm);                                                // [SUB]
  unsigned long long* cursor = reinterpret_cast<unsigned long long*>(stage + SUB);   // [P1] absolute write positions
  uint32_t* hist = reinterpret_cast<uint32_t*>(cursor + P1);                            // [padded P1]
  uint32_t* soff = hist + padded_len(P1);                                               // [padded P1]
  __shared__ uint64_t code_s[NW + 2];
  __shared__ uint32_t inv_s[NW + 2];
  __shared__ uint32_t st_s[NW + 2];
  __shared__ uint32_t hll_s[kHllRegs];
  __shared__ uint64_t rcur_s;
  __shared__ uint32_t wt[32];
  const int t = threadIdx.x;
  const int wl = t / TPW, h = t % TPW;  // code word of the thread within the sub-step, half
  const uint64_t tile = blockIdx.x;
  for (int c = t; c < P1; c += NT) {
    cursor[c] = b.cstart[c] + b.toff[tile * P1 + c];
    hist[PAD(c)] = 0;
  }
  for (int i = t; i < kHllRegs; i += NT) hll_s[i] = 0;
  if (t == 0) rcur_s = b.tile_first[tile];
  for (int sub = 0; sub < kTileWords / NW; ++sub) {
    const uint64_t j0 = tile * kTileWords + (uint64_t)sub * NW;
    if (j0 >= s.n_words) break;
    __syncthreads();
    if (t < 2) {
      if (sub > 0) {
        code_s[t] = code_s[NW + t];
        inv_s[t] = inv_s[NW + t];
      } else if (j0 + t >= 2) {
        code_s[t] = b.codes64[j0 + t - 2];
        inv_s[t] = b.inv32[j0 + t - 2];
      } else {
        code_s[t] = 0;
        inv_s[t] = ~0u;
      }
    }
    for (int w = t; w < NW; w += NT) {
      const uint64_t jw = j0 + w;
      code_s[w + 2] = jw < s.n_words ? b.codes64[jw] : 0;
      inv_s[w + 2] = jw < s.n_words ? b.inv32[jw] : ~0u;
      st_s[w + 2] = 0;
    }
    if (t < 2) st_s[t] = 0;
    __syncthreads();
    build_starts(b.offsets, s.n_reads, j0, NW, st_s, &rcur_s);
    __syncthreads();
    const uint64_t j = j0 + wl;
    K keys[WPT];
    uint32_t rr[WPT / 2];
    uint32_t valid = 0;
#pragma unroll
    for (int i = 0; i < WPT / 2; ++i) rr[i] = 0;
    if (j < s.n_words) {
      Win W;
      const int sw = wl + 2;
      const uint32_t vm = valid_mask(inv_s[sw - 2], inv_s[sw - 1], inv_s[sw], st_s[sw - 2], st_s[sw - 1], st_s[sw], s.k);
      win_setup<KW, WPT>(code_s[sw - 2], code_s[sw - 1], code_s[sw], vm, h, s.k, W);
      valid = W.valid & (WPT == 32 ? 0xffffffffu : 0xffffu);
#pragma unroll
      for (int i = 0; i < WPT; ++i) {
        if ((valid >> i) & 1u) {
          uint64_t c0, c1;
          win_top<KW, WPT>(W, i, s.canonical, c0, c1);
          top_to_key(c0, c1, s.k, keys[i]);
          const uint32_t c = field32(umap((uint32_t)(c0 >> 32), s.canonical), 0, s.b1);
          const uint32_t r = atomicAdd(&hist[PAD(c)], 1u);
          rr[i >> 1] |= r << (16 * (i & 1));
          const uint64_t hh = key_hash(keys[i]);
          if ((hh >> (64 - kHllSampleLog2)) == 0) {
            const uint32_t reg = (uint32_t)(hh >> (64 - kHllSampleLog2 - kHllLog2)) & (kHllRegs - 1);
            const uint64_t rest = hh << (kHllSampleLog2 + kHllLog2);
            atomicMax(&hll_s[reg], (uint32_t)min(__clzll(rest) + 1, 64 - kHllSampleLog2 - kHllLog2 + 1));
          }
        }
      }
    }
    __syncthreads();
    for (int c = t; c < P1; c += NT) soff[PAD(c)] = hist[PAD(c)];
    __syncthreads();
    block_exclusive_scan_pad<uint32_t>(soff, P1, wt);
#pragma unroll
    for (int i = 0; i < WPT; ++i) {
      if (valid & (1u << i)) {
        const uint32_t c = coarse_of(keys[i], s.k, s.canonical, s.b1);  // same field as above, from the key
        const uint32_t pos = soff[PAD(c)] + ((rr[i >> 1] >> (16 * (i & 1))) & 0xffffu);
        stage[pos] = keys[i];
      }
    }
    __syncthreads();
    const uint32_t n_sub = soff[PAD(P1 - 1)] + hist[PAD(P1 - 1)];
    for (uint32_t i = t; i < n_sub; i += NT) {
      const K key = stage[i];
      const uint32_t c = coarse_of(key, s.k, s.canonical, s.b1);  // runs are grouped by partition
      const uint32_t so = soff[PAD(c)];
      const uint64_t pos = cursor[c] + (i - so);
      if (i >= so && i - so < hist[PAD(c)] && pos < s.cap) store_key(b.kbuf, pos, key);
      else atomicOr(&b.meta->status, ST_INTERNAL);
    }
    __syncthreads();
    for (int c = t; c < P1; c += NT) {
      cursor[c] += hist[PAD(c)];
      hist[PAD(c)] = 0;
    }
  }
  __syncthreads();
  for (int i = t; i < kHllRegs; i += NT)
    if (hll_s[i]) atomicMax(&b.hll[i], hll_s[i]);
}

// ------------------------------------------------------------------ phase 2: fine split
struct FineCtx {
  int k, canonical, b1;
};

template <class K>
__device__ __forceinline__ uint32_t fine_index(K key, const FineCtx& x, const uint32_t* fine_base_s, const uint8_t* flog_s) {
  const uint32_t u = umap(top32_of(key, x.k), x.canonical);
  const uint32_t c = field32(u, 0, x.b1);
  return fine_base_s[c] + field32(u, x.b1, flog_s[c]);
}

template <int KW>
__device__ __forceinline__ void load_fine_tables(const Buffers& b, int P1, uint32_t* fine_base_s, uint8_t* flog_s) {
  for (int c = threadIdx.x; c <= P1; c += blockDim.x) fine_base_s[c] = b.fine_base[c];
  for (int c = threadIdx.x; c < P1; c += blockDim.x) flog_s[c] = b.fine_log2[c];
}

constexpr int kFineThreads = 512;
constexpr int kFinePer = 16;  // keys per thread per chunk (loaded as 16-byte pairs / quads, all before use)
constexpr int kFineChunk = kFineThreads * kFinePer;

// Load this thread's keys of the chunk [c0, c1): pairs of words (read-only path, all
// loads issued before any use).  Key m of the thread is chunk key  (m / P) * P * T +
// threadIdx.x * P + m % P, P = 16 / (8 KW) keys per load, T = threads.
template <int KW>
__device__ __forceinline__ void load_chunk(const uint64_t* __restrict__ src, uint64_t c0, uint64_t c1,
                                           typename KeyT<KW>::T (&keys)[kFinePer], uint32_t& have) {
  typedef typename KeyT<KW>::T K;
  constexpr int P = KW == 1 ? 2 : 1;  // keys per 16-byte load
  have = 0;
  ulonglong2 v[kFinePer / P];
#pragma unroll
  for (int m = 0; m < kFinePer / P; ++m) {
    const uint64_t i = c0 + (uint64_t)m * P * kFineThreads + (uint64_t)threadIdx.x * P;
    v[m] = make_ulonglong2(0, 0);
    if (i + P <= c1) v[m] = __ldg(reinterpret_cast<const ulonglong2*>(src + i * KW));
    else if (i < c1) v[m].x = __ldg(src + i * KW);  // P == 2 and one key left
  }
#pragma unroll
  for (int m = 0; m < kFinePer / P; ++m) {
    const uint64_t i = c0 + (uint64_t)m * P * kFineThreads + (uint64_t)threadIdx.x * P;
    if constexpr (KW == 1) {
      keys[2 * m] = (K)v[m].x;
      keys[2 * m + 1] = (K)v[m].y;
      if (i < c1) have |= 1u << (2 * m);
      if (i + 1 < c1) have |= 1u << (2 * m + 1);
    } else {
      keys[m] = (K)(((u128)v[m].y << 64) | v[m].x);
      if (i < c1) have |= 1u << m;
    }
  }
}

template <int KW>
__global__ void __launch_bounds__(kFineThreads) k_fine_hist(Shape s, Buffers b) {
  typedef typename KeyT<KW>::T K;
  extern __shared__ __align__(16) uint8_t sm[];
  const int P1 = 1 << s.b1;
  uint32_t* fine_base_s = reinterpret_cast<uint32_t*>(sm);  // [P1+1]
  uint32_t* lh = fine_base_s + P1 + 1;                       // [kFineLocalCap]
  uint8_t* flog_s = reinterpret_cast<uint8_t*>(lh + kFineLocalCap);
  __shared__ uint32_t g_lo_s, g_hi_s;
  load_fine_tables<KW>(b, P1, fine_base_s, flog_s);
  for (int i = threadIdx.x; i < kFineLocalCap; i += kFineThreads) lh[i] = 0;
  const FineCtx x{s.k, s.canonical, s.b1};
  const uint64_t K_total = b.meta->n_windows;
  __syncthreads();
  for (uint64_t c0 = blockIdx.x * (uint64_t)kFineChunk; c0 < K_total; c0 += (uint64_t)gridDim.x * kFineChunk) {
    const uint64_t c1 = min(K_total, c0 + kFineChunk);
    if (threadIdx.x == 0) {
      K kf, kl;
      load_key(b.kbuf, c0, kf);
      load_key(b.kbuf, c1 - 1, kl);
      const uint32_t cf = coarse_of(kf, s.k, s.canonical, s.b1), cl = coarse_of(kl, s.k, s.canonical, s.b1);
      g_lo_s = fine_base_s[cf];
      g_hi_s = fine_base_s[cl + 1];
    }
    __syncthreads();
    const uint32_t g_lo = g_lo_s, span = g_hi_s - g_lo_s;
    const bool local = span <= (uint32_t)kFineLocalCap;
    K keys[kFinePer];
    uint32_t have;
    load_chunk<KW>(b.kbuf, c0, c1, keys, have);
#pragma unroll
    for (int m = 0; m < kFinePer; ++m) {
      if ((have >> m) & 1u) {
        const uint32_t g = fine_index(keys[m], x, fine_base_s, flog_s);
        if (local && g - g_lo < span) atomicAdd(&lh[g - g_lo], 1u);
        else if (g < s.nf_max) atomicAdd(&b.fhist[g], 1u);
        else atomicOr(&b.meta->status, ST_INTERNAL);
      }
    }
    __syncthreads();
    if (local) {
      for (uint32_t i = threadIdx.x; i < span; i += kFineThreads) {
        const uint32_t v = lh[i];
        if (v) {
          if (g_lo + i < s.nf_max) atomicAdd(&b.fhist[g_lo + i], v);
          else atomicOr(&b.meta->status, ST_INTERNAL);
          lh[i] = 0;
        }
      }
    }
    __syncthreads();
  }
}

// Exclusive scan of the fine histogram (one block of 1024 threads).
__global__ void k_fine_scan(Shape sh, Buffers b) {
  __shared__ uint64_t wt[32];
  __shared__ uint64_t carry_s;
  const uint64_t NF = min(b.meta->n_fine, sh.nf_max);
  const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, wid = t >> 5;
  if (t == 0) carry_s = 0;
  __syncthreads();
  for (uint64_t base = 0; base < NF; base += (uint64_t)nt * 8) {
    uint64_t v[8];
    uint64_t s = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const uint64_t i = base + (uint64_t)t * 8 + m;
      v[m] = i < NF ? b.fhist[i] : 0;
      s += v[m];
    }
    uint64_t x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) wt[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint64_t w = wt[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= d) w += y;
      }
      wt[lane] = w;
    }
    __syncthreads();
    uint64_t run = carry_s + x - s + (wid ? wt[wid - 1] : 0);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const uint64_t i = base + (uint64_t)t * 8 + m;
      if (i < NF) {
        b.foff[i] = run;
        b.fcur[i] = run;
      }
      run += v[m];
    }
    __syncthreads();
    if (t == 0) carry_s += wt[31];
    __syncthreads();
  }
  if (t == 0) b.foff[NF] = carry_s;
}

template <int KW>
__global__ void __launch_bounds__(kFineThreads) k_fine_scatter(Shape s, Buffers b) {
  typedef typename KeyT<KW>::T K;
  extern __shared__ __align__(16) uint8_t sm[];
  const int P1 = 1 << s.b1;
  K* stage = reinterpret_cast<K*>(sm);                                        // [kFineChunk]
  uint64_t* gbase = reinterpret_cast<uint64_t*>(stage + kFineChunk);          // [kFineLocalCap]
  uint32_t* lh = reinterpret_cast<uint32_t*>(gbase + kFineLocalCap);          // [padded kFineLocalCap]
  uint32_t* soff = lh + padded_len(kFineLocalCap);                            // [padded kFineLocalCap]
  uint16_t* stage_g = reinterpret_cast<uint16_t*>(soff + padded_len(kFineLocalCap));  // [kFineChunk]
  uint32_t* fine_base_s = reinterpret_cast<uint32_t*>(stage_g + kFineChunk);  // [P1+1]
  uint8_t* flog_s = reinterpret_cast<uint8_t*>(fine_base_s + P1 + 1);         // [P1]
  __shared__ uint32_t g_lo_s, g_hi_s;
  __shared__ uint32_t wt[32];
  load_fine_tables<KW>(b, P1, fine_base_s, flog_s);
  for (int i = threadIdx.x; i < kFineLocalCap; i += kFineThreads) lh[PAD(i)] = 0;
  const FineCtx x{s.k, s.canonical, s.b1};
  const uint64_t K_total = b.meta->n_windows;
  __syncthreads();
  for (uint64_t c0 = blockIdx.x * (uint64_t)kFineChunk; c0 < K_total; c0 += (uint64_t)gridDim.x * kFineChunk) {
    const uint64_t c1 = min(K_total, c0 + kFineChunk);
    if (threadIdx.x == 0) {
      K kf, kl;
      load_key(b.kbuf, c0, kf);
      load_key(b.kbuf, c1 - 1, kl);
      const uint32_t cf = coarse_of(kf, s.k, s.canonical, s.b1), cl = coarse_of(kl, s.k, s.canonical, s.b1);
      g_lo_s = fine_base_s[cf];
      g_hi_s = fine_base_s[cl + 1];
    }
    __syncthreads();
    const uint32_t g_lo = g_lo_s, span = g_hi_s - g_lo_s;
    if (span == 0 || span > (uint32_t)kFineLocalCap) {
      // a chunk over very many tiny fine partitions: one global cursor bump per key
      for (int m = 0; m < kFinePer; ++m) {
        const uint64_t i = c0 + threadIdx.x + (uint64_t)m * kFineThreads;
        if (i < c1) {
          K key;
          load_key(b.kbuf, i, key);
          const uint32_t g = fine_index(key, x, fine_base_s, flog_s);
          const uint64_t pos = g < s.nf_max ? atomicAdd(&b.fcur[g], 1ull) : ~0ull;
          if (pos < s.cap) store_key(b.sbuf, pos, key);
          else atomicOr(&b.meta->status, ST_INTERNAL);
        }
      }
      __syncthreads();
      continue;
    }
    K keys[kFinePer];
    uint32_t gr[kFinePer];
    uint32_t have;
    load_chunk<KW>(b.kbuf, c0, c1, keys, have);
#pragma unroll
    for (int m = 0; m < kFinePer; ++m) {
      gr[m] = 0xffffffffu;
      if ((have >> m) & 1u) {
        const uint32_t lg = fine_index(keys[m], x, fine_base_s, flog_s) - g_lo;
        if (lg < span) {
          const uint32_t r = atomicAdd(&lh[PAD(lg)], 1u);
          gr[m] = (lg << 16) | r;
        } else {
          atomicOr(&b.meta->status, ST_INTERNAL);
        }
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < span; i += kFineThreads) soff[PAD(i)] = lh[PAD(i)];
    __syncthreads();
    block_exclusive_scan_pad<uint32_t>(soff, (int)span, wt);
    for (uint32_t i = threadIdx.x; i < span; i += kFineThreads) {
      const uint32_t v = lh[PAD(i)];
      if (v) gbase[i] = g_lo + i < s.nf_max ? atomicAdd(&b.fcur[g_lo + i], (unsigned long long)v) : ~0ull;
    }
#pragma unroll
    for (int m = 0; m < kFinePer; ++m) {
      if (gr[m] != 0xffffffffu) {
        const uint32_t lg = gr[m] >> 16;
        const uint32_t pos = soff[PAD(lg)] + (gr[m] & 0xffffu);
        stage[pos] = keys[m];
        stage_g[pos] = (uint16_t)lg;
      }
    }
    __syncthreads();
    // only the keys that were staged (a key outside the chunk's fine range was rejected above)
    const uint32_t n_staged = soff[PAD(span - 1)] + lh[PAD(span - 1)];
    for (uint32_t i = threadIdx.x; i < n_staged; i += kFineThreads) {
      const uint32_t lg = stage_g[i];
      if (lg >= span) {
        atomicOr(&b.meta->status, ST_INTERNAL);
        continue;
      }
      const uint64_t pos = gbase[lg] + (i - soff[PAD(lg)]);
      if (pos < s.cap) store_key(b.sbuf, pos, stage[i]);
      else atomicOr(&b.meta->status, ST_INTERNAL);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < span; i += kFineThreads) lh[PAD(i)] = 0;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ phase 2: count + emit
constexpr uint64_t kLookValue = (1ull << 62) - 1;
constexpr uint64_t kLookAgg = 1ull << 62;
constexpr uint64_t kLookIncl = 2ull << 62;

// Decoupled look-back (executed by one warp): sum of distinct counts of fine partitions < g.
__device__ uint64_t lookback(unsigned long long* look, uint64_t g, uint32_t* status) {
  const int lane = threadIdx.x & 31;
  uint64_t excl = 0;
  int64_t j = (int64_t)g - 1;
  while (j >= 0) {
    const int64_t idx = j - lane;
    uint64_t v = kLookIncl;  // before the first partition: inclusive prefix 0
    if (idx >= 0) {
      uint32_t spins = 0;
      v = ld_status(&look[idx]);
      while ((v >> 62) == 0) {
        if (++spins > kLookbackSpinLimit) {
          atomicOr(status, ST_TIMEOUT);
          v = kLookIncl;
          break;
        }
        __nanosleep(64);
        v = ld_status(&look[idx]);
      }
    }
    const unsigned incl = __ballot_sync(0xffffffffu, (v >> 62) == 2);
    const int stop = incl ? __ffs(incl) - 1 : 31;
    uint64_t val = lane <= stop ? (v & kLookValue) : 0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) val += __shfl_xor_sync(0xffffffffu, val, d);
    excl += val;
    if (incl) break;
    j -= 32;
  }
  return excl;
}

template <int KW>
struct Table {
  typedef typename KeyT<KW>::T K;
  K* keys;
  uint32_t* counts;
};

// Count kernel shared memory: a hash table of 2^bT_max slots (key + count) and a bucket
// histogram of kHistMax(kw) entries.  After the count, the table's bytes hold the dense
// array of distinct keys (at most 3/4 of the slots).
constexpr int kTableLog2Cap = 13;  // 8192 slots: 8 per thread of the 1024-thread block
__host__ __device__ constexpr int hist_max(int kw) { return kw == 1 ? 16384 : 8192; }

size_t count_kernel_smem(int kw, int bT_max, int /*unused*/) {
  const size_t slots = (size_t)1 << bT_max;
  return slots * (size_t)(kw * 8 + 4) + padded_len(hist_max(kw)) * 4 + 256;
}

int table_log2_max(int kw, size_t smem_optin) {
  int best = 6;
  for (int bt = 6; bt <= kTableLog2Cap; ++bt)
    if (count_kernel_smem(kw, bt, 0) + 8192 <= smem_optin) best = bt;  // 8 KB for static shared memory
  return best;
}

constexpr int kProbeLimit = 128;
constexpr int kWorkers = kCountThreads - 32;  // warps 1.. load and sort while warp 0 looks back
constexpr int kSlotsPerThread = (1 << kTableLog2Cap) / kCountThreads;

// counting-table slot of a key: a multiplicative hash (spreads keys that share prefixes)
__device__ __forceinline__ uint32_t hslot(uint64_t key, int bT) {
  return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - bT));
}
__device__ __forceinline__ uint32_t hslot(u128 key, int bT) {
  const uint64_t h = ((uint64_t)key ^ ((uint64_t)(key >> 64) * 0xC2B2AE3D27D4EB4Full)) * 0x9E3779B97F4A7C15ull;
  return (uint32_t)(h >> (64 - bT));
}

__device__ __forceinline__ void bar_workers() { asm volatile("bar.sync 1, %0;" ::"r"(kWorkers) : "memory"); }

// Add `inc` to the count of `key` (claiming a slot if new).  Returns false if no slot
// was found within the probe limit.
template <int KW>
__device__ __forceinline__ bool count_insert(Table<KW> tb, typename KeyT<KW>::T key, uint32_t inc, int bT,
                                             uint32_t* n_new, uint32_t* status) {
  typedef typename KeyT<KW>::T K;
  const K EMPTY = all_ones<K>();
  const uint32_t mask = (1u << bT) - 1;
  uint32_t s = hslot(key, bT);
  for (int probe = 0; probe < kProbeLimit; ++probe, s = (s + 1) & mask) {
    bool hit = false;
    if constexpr (KW == 1) {
      uint64_t* p = reinterpret_cast<uint64_t*>(tb.keys) + s;
      const uint64_t cur = *reinterpret_cast<volatile uint64_t*>(p);
      if (cur == (uint64_t)key) {
        hit = true;
      } else if (cur == ~0ull) {
        const unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long*>(p), ~0ull, (unsigned long long)key);
        if (old == ~0ull) atomicAdd(n_new, 1u);
        hit = (old == ~0ull || old == (unsigned long long)key);
      }
    } else {
      const K old = cas128_shared(reinterpret_cast<u128*>(tb.keys) + s, (u128)EMPTY, (u128)key);
      if (old == EMPTY) atomicAdd(n_new, 1u);
      hit = (old == EMPTY || old == key);
    }
    if (hit) {
      const uint32_t o = atomicAdd(&tb.counts[s], inc);
      if (o > 0xffffffffu - inc) atomicOr(status, ST_COUNT_OVERFLOW);
      return true;
    }
  }
  return false;
}

template <int KW>
__device__ __forceinline__ void table_clear(Table<KW> tb, uint32_t nslots) {
  typedef typename KeyT<KW>::T K;
  for (uint32_t i = threadIdx.x; i < nslots; i += blockDim.x) {
    tb.keys[i] = all_ones<K>();
    tb.counts[i] = 0;
  }
}

// Count the keys in[0, n) (only those in [lo, hi] when `ranged`).  The all-ones key is
// counted apart in *special (it marks empty slots).  Sets *ovf if a key found no slot.
template <int KW>
__device__ void count_all(Table<KW> tb, const uint64_t* in, uint64_t n, bool ranged, typename KeyT<KW>::T lo,
                          typename KeyT<KW>::T hi, int bT, uint32_t* n_new, uint32_t* ovf, uint32_t* special,
                          uint32_t* status) {
  typedef typename KeyT<KW>::T K;
  constexpr int kIn = KW == 1 ? 8 : 2;  // loads in flight per thread (u128 keys: register-bound at 64)
  const K EMPTY = all_ones<K>();
  const int lane = threadIdx.x & 31;
  for (uint64_t base = 0; base < n; base += kIn * (uint64_t)blockDim.x) {
    K kk[kIn];
    bool aa[kIn];
#pragma unroll
    for (int m = 0; m < kIn; ++m) {
      const uint64_t i = base + (uint64_t)m * blockDim.x + threadIdx.x;
      kk[m] = 0;
      aa[m] = i < n;
      if (aa[m]) load_key(in, i, kk[m]);
    }
#pragma unroll
    for (int m = 0; m < kIn; ++m) {
      const K key = kk[m];
      bool act = aa[m];
      if (ranged) act = act && key >= lo && key <= hi && key != EMPTY;
      const unsigned am = __ballot_sync(0xffffffffu, act);
      if (!am) continue;
      const int first = __ffs(am) - 1;
      const K k0 = shfl_key(key, first);
      const bool same = __all_sync(0xffffffffu, !act || key == k0);
      if (same) {  // a warp of equal keys (heavy hitter) adds once
        if (lane == first) {
          const uint32_t inc = __popc(am);
          if (k0 == EMPTY) {
            if (atomicAdd(special, inc) > 0xffffffffu - inc) atomicOr(status, ST_COUNT_OVERFLOW);
          } else if (!count_insert<KW>(tb, k0, inc, bT, n_new, status)) {
            atomicOr(ovf, 1u);
          }
        }
      } else if (act) {
        if (key == EMPTY) {
          if (atomicAdd(special, 1u) == 0xffffffffu) atomicOr(status, ST_COUNT_OVERFLOW);
        } else if (!count_insert<KW>(tb, key, 1u, bT, n_new, status)) {
          atomicOr(ovf, 1u);
        }
      }
    }
  }
}

template <class K> __device__ __forceinline__ int bitlen(K v);
template <> __device__ __forceinline__ int bitlen(uint64_t v) { return 64 - __clzll(v); }
template <> __device__ __forceinline__ int bitlen(u128 v) {
  const uint64_t hi = (uint64_t)(v >> 64);
  return hi ? 128 - __clzll(hi) : 64 - __clzll((uint64_t)v);
}

// Smallest and largest key in the table (all threads; the result is returned to all).
template <int KW>
__device__ void table_range(Table<KW> tb, uint32_t nslots, typename KeyT<KW>::T* red_lo, typename KeyT<KW>::T* red_hi,
                            typename KeyT<KW>::T& lo, typename KeyT<KW>::T& hi) {
  typedef typename KeyT<KW>::T K;
  const K EMPTY = all_ones<K>();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  K mn = EMPTY, mx = 0;
  for (uint32_t s = threadIdx.x; s < nslots; s += blockDim.x) {
    const K key = tb.keys[s];
    if (key != EMPTY) {
      mn = key < mn ? key : mn;
      mx = key > mx ? key : mx;
    }
  }
#pragma unroll
  for (int dd = 16; dd > 0; dd >>= 1) {
    const K a = shfl_key(mn, (lane + dd) & 31), c = shfl_key(mx, (lane + dd) & 31);
    mn = a < mn ? a : mn;
    mx = c > mx ? c : mx;
  }
  if (lane == 0) {
    red_lo[wid] = mn;
    red_hi[wid] = mx;
  }
  __syncthreads();
  if (wid == 0) {  // one warp combines the per-warp results
    const int nw = (int)(blockDim.x >> 5);
    mn = lane < nw ? red_lo[lane] : EMPTY;
    mx = lane < nw ? red_hi[lane] : K(0);
#pragma unroll
    for (int dd = 16; dd > 0; dd >>= 1) {
      const K a = shfl_key(mn, (lane + dd) & 31), c = shfl_key(mx, (lane + dd) & 31);
      mn = a < mn ? a : mn;
      mx = c > mx ? c : mx;
    }
    __syncwarp();
    if (lane == 0) {
      red_lo[0] = mn;
      red_hi[0] = mx;
    }
  }
  __syncthreads();
  lo = red_lo[0];
  hi = red_hi[0];
}

// Write the table's entries to stage[0, d) grouped by bucket (key - lo) >> sh, buckets in
// ascending order (an ordered counting sort; entries inside a bucket are unordered).
// hist[0, NB) must be zero on entry; on return it holds each bucket's first position.
// All threads; nslots <= kSlotsPerThread * blockDim.x.
template <int KW>
__device__ void place_entries(Table<KW> tb, uint32_t nslots, typename KeyT<KW>::T lo, int sh, uint32_t* hist,
                              uint32_t NB, uint64_t* stage_keys, uint32_t* stage_counts, uint32_t* wtmp) {
  typedef typename KeyT<KW>::T K;
  const K EMPTY = all_ones<K>();
  uint32_t br[kSlotsPerThread];
#pragma unroll
  for (int m = 0; m < kSlotsPerThread; ++m) {
    const uint32_t s = threadIdx.x + m * blockDim.x;
    br[m] = 0xffffffffu;
    if (s < nslots) {
      const K key = tb.keys[s];
      if (key != EMPTY) {
        const uint32_t bk = (uint32_t)((key - lo) >> sh);
        br[m] = (bk << 16) | atomicAdd(&hist[PAD(bk)], 1u);  // NB <= 2^14, rank < 2^16
      }
    }
  }
  __syncthreads();
  block_exclusive_scan_pad<uint32_t>(hist, (int)NB, wtmp);
#pragma unroll
  for (int m = 0; m < kSlotsPerThread; ++m) {
    if (br[m] != 0xffffffffu) {
      const uint32_t s = threadIdx.x + m * blockDim.x;
      const uint32_t pos = hist[PAD(br[m] >> 16)] + (br[m] & 0xffffu);
      store_key(stage_keys, pos, tb.keys[s]);
      stage_counts[pos] = tb.counts[s];
    }
  }
  __syncthreads();
}

// Sort keys[a, a+c) (with their counts) by one warp: a bitonic network whose comparators
// all put the smaller key first, so positions past c act as +infinity and are skipped.
template <class K>
__device__ void warp_sort_segment(K* keys, uint32_t* counts, uint32_t a, uint32_t c) {
  const int lane = threadIdx.x & 31;
  uint32_t M = 1;
  while (M < c) M <<= 1;
  for (uint32_t size = 2; size <= M; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = lane; i < M; i += 32) {
        const uint32_t j = (stride == (size >> 1)) ? (i ^ (size - 1)) : (i ^ stride);
        if (j > i && j < c) {
          const K x = keys[a + i], y = keys[a + j];
          if (y < x) {
            keys[a + i] = y;
            keys[a + j] = x;
            const uint32_t cx = counts[a + i];
            counts[a + i] = counts[a + j];
            counts[a + j] = cx;
          }
        }
      }
      __syncwarp();
    }
  }
}

__device__ __forceinline__ uint64_t shfl_xor_key(uint64_t v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ u128 shfl_xor_key(u128 v, int m) {
  const uint64_t lo = __shfl_xor_sync(0xffffffffu, (uint64_t)v, m);
  const uint64_t hi = __shfl_xor_sync(0xffffffffu, (uint64_t)(v >> 64), m);
  return ((u128)hi << 64) | lo;
}

// Sort keys[a, a+c), c <= 32, with their counts: one entry per lane, a bitonic network on
// shuffles (lanes past c hold the largest key and stay at the end).  Whole warp calls it.
template <class K>
__device__ __forceinline__ void warp_sort32(K* keys, uint32_t* counts, uint32_t a, uint32_t c) {
  const int lane = threadIdx.x & 31;
  const bool have = (uint32_t)lane < c;
  K key = have ? keys[a + lane] : ~(K)0;
  uint32_t cnt = have ? counts[a + lane] : 0u;
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int j = size >> 1; j > 0; j >>= 1) {
      const K other = shfl_xor_key(key, j);
      const uint32_t oc = __shfl_xor_sync(0xffffffffu, cnt, j);
      const bool up = (lane & size) == 0, lower = (lane & j) == 0;
      const bool take = (lower == up) ? (other < key) : (key < other);
      if (take) {
        key = other;
        cnt = oc;
      }
    }
  }
  if (have) {
    keys[a + lane] = key;
    counts[a + lane] = cnt;
  }
}

constexpr int kRankPer = 7;        // entries per worker thread: 7 * 992 >= 3/4 of 8192 slots
constexpr uint32_t kBigBucket = 256;  // buckets above this are sorted in place by a warp first

// Worker warps: read the bucket-grouped staged entries into the dense shared arrays, then
// give every entry its rank inside the partition: its bucket's first position plus the
// number of smaller keys in the same bucket (buckets are small; the rare bucket above
// kBigBucket entries is sorted in place by one warp and ranked by position).
template <int KW>
__device__ __forceinline__ void load_and_rank(const uint64_t* stage_keys, const uint32_t* stage_counts, uint32_t d,
                                              typename KeyT<KW>::T* dense_keys, uint32_t* dense_counts,
                                              const uint32_t* hist, uint32_t NB, typename KeyT<KW>::T lo, int sh,
                                              uint32_t (&rank)[kRankPer], unsigned long long* prof) {
  typedef typename KeyT<KW>::T K;
  const int t = threadIdx.x - 32, wid = t >> 5, lane = t & 31;
  long long tm = clock64();
  for (uint32_t i = t; i < d; i += kWorkers) {
    K key;
    load_key(stage_keys, i, key);
    dense_keys[i] = key;
    dense_counts[i] = stage_counts[i];
  }
  bar_workers();
  // rare large buckets: one warp each, in place (each warp scans a slice of the buckets)
  constexpr int kWarps = kWorkers / 32;
  const uint32_t per = (NB + kWarps - 1) / kWarps;
  const uint32_t b_lo = min(NB, (uint32_t)wid * per), b_hi = min(NB, b_lo + per);
  for (uint32_t base = b_lo; base < b_hi; base += 32) {
    const uint32_t bk = base + lane;
    uint32_t a = 0, c = 0;
    if (bk < b_hi) {
      a = hist[PAD(bk)];
      c = (bk + 1 < NB ? hist[PAD(bk + 1)] : d) - a;
    }
    unsigned todo = __ballot_sync(0xffffffffu, c > kBigBucket);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      warp_sort_segment<K>(dense_keys, dense_counts, __shfl_sync(0xffffffffu, a, src),
                           __shfl_sync(0xffffffffu, c, src));
    }
  }
  bar_workers();
  if (prof && t == 0) {
    const long long now = clock64();
    atomicAdd(&prof[3], (unsigned long long)(now - tm));
    tm = now;
  }
#pragma unroll
  for (int m = 0; m < kRankPer; ++m) {
    const uint32_t i = t + m * kWorkers;
    rank[m] = 0xffffffffu;
    if (i < d) {
      const K key = dense_keys[i];
      const uint32_t bk = (uint32_t)((key - lo) >> sh);
      const uint32_t a = hist[PAD(bk)];
      const uint32_t e = bk + 1 < NB ? hist[PAD(bk + 1)] : d;
      uint32_t r = a;
      if (e - a > kBigBucket) {
        r = i;
      } else {
        for (uint32_t j = a; j < e; ++j) r += dense_keys[j] < key;
      }
      rank[m] = r;
    }
  }
  if (prof && t == 0) atomicAdd(&prof[4], (unsigned long long)(clock64() - tm));
}

// Worker threads: write their entries at out[base + rank].
template <int KW>
__device__ __forceinline__ void emit_ranked(const typename KeyT<KW>::T* dense_keys, const uint32_t* dense_counts,
                                            uint32_t d, const uint32_t (&rank)[kRankPer], uint64_t base,
                                            uint64_t* out_keys, uint32_t* out_counts, uint64_t cap, uint32_t* status) {
  const int t = threadIdx.x - 32;
  if (base + d > cap) {
    if (t == 0) atomicOr(status, ST_INTERNAL);
    return;
  }
#pragma unroll
  for (int m = 0; m < kRankPer; ++m) {
    const uint32_t i = t + m * kWorkers;
    if (i < d && rank[m] < d) {
      store_key(out_keys, base + rank[m], dense_keys[i]);
      out_counts[base + rank[m]] = dense_counts[i];
    }
  }
}

// Key range of the current table and an ordered counting sort of its entries into NB
// buckets, written to `stage` (global) grouped by bucket.  All threads.
template <int KW>
__device__ void bucket_table(Table<KW> tb, uint32_t nslots, uint32_t d, uint64_t* stage_keys, uint32_t* stage_counts,
                             uint32_t* hist, typename KeyT<KW>::T* red_lo, typename KeyT<KW>::T* red_hi, uint32_t* wtmp,
                             unsigned long long* prof, typename KeyT<KW>::T& lo, int& sh, uint32_t& NB) {
  typedef typename KeyT<KW>::T K;
  long long tm = clock64();
  K hi;
  table_range<KW>(tb, nslots, red_lo, red_hi, lo, hi);
  NB = 1;
  while (NB < (uint32_t)hist_max(KW) && NB < 2 * d) NB <<= 1;  // at most two entries per bucket on average
  const int bB = 31 - __clz(NB);
  sh = d == 0 ? 0 : max(0, bitlen(K(hi - lo)) - bB);
  for (uint32_t i = threadIdx.x; i < NB; i += blockDim.x) hist[PAD(i)] = 0;
  __syncthreads();
  if (prof && threadIdx.x == 0) {
    const long long now = clock64();
    atomicAdd(&prof[0], (unsigned long long)(now - tm));
    tm = now;
  }
  place_entries<KW>(tb, nslots, lo, sh, hist, NB, stage_keys, stage_counts, wtmp);
  if (prof && threadIdx.x == 0) atomicAdd(&prof[1], (unsigned long long)(clock64() - tm));
}

__device__ __forceinline__ int ceil_log2_u32(uint32_t v) { return v <= 1 ? 0 : 32 - __clz(v - 1); }

template <int KW>
__global__ void __launch_bounds__(kCountThreads, 1) k_count_emit(Shape s, Buffers b) {
  typedef typename KeyT<KW>::T K;
  extern __shared__ __align__(16) uint8_t sm[];
  const uint32_t cap_slots = 1u << s.bT_max;
  uint32_t* hist = reinterpret_cast<uint32_t*>(sm + (size_t)cap_slots * (KW * 8 + 4));
  __shared__ uint64_t g_s, excl_s;
  __shared__ uint32_t ovf_s, special_s, nnew_s;
  __shared__ uint32_t wtmp[32];
  __shared__ K red_lo[32], red_hi[32];
  __shared__ K stk_lo[160], stk_hi[160];
  __shared__ int stk_n;
  const K EMPTY = all_ones<K>();
  const uint64_t NF = b.meta->n_fine;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* stage_cnt_all = reinterpret_cast<uint32_t*>(b.kbuf);  // kbuf is free once the fine split is done
  unsigned long long* prof = s.profile ? reinterpret_cast<unsigned long long*>(b.meta->sub_cycles) : nullptr;
  // profiled plans: thread 0 adds the cycles spent in each phase (0 clear, 1 count, 2 -,
  // 3 order, 4 look-back (warp 0, overlapped), 5 emit, 6 overflow path, 7 ticket + setup)
  long long t_mark = clock64();
  auto phase = [&](int i) {
    if (s.profile && threadIdx.x == 0) {
      const long long now = clock64();
      atomicAdd(reinterpret_cast<unsigned long long*>(&b.meta->phase_cycles[i]), (unsigned long long)(now - t_mark));
      t_mark = now;
    }
  };
  // dense arrays reuse the table bytes: at most 3/4 of the slots
  const uint32_t dcap = (3u * cap_slots) >> 2;
  K* dk = reinterpret_cast<K*>(sm);
  uint32_t* dc = reinterpret_cast<uint32_t*>(dk + dcap);
  while (true) {
    if (threadIdx.x == 0) {
      g_s = atomicAdd(reinterpret_cast<unsigned long long*>(&b.meta->ticket), 1ull);
      ovf_s = 0;
      special_s = 0;
      nnew_s = 0;
    }
    __syncthreads();
    const uint64_t g = g_s;
    if (g >= NF) break;
    const uint64_t f0 = b.foff[g];
    uint64_t n = b.foff[g + 1] - f0;
    if (f0 > s.cap || n > s.cap - f0) {  // inconsistent scan: record it, count nothing
      if (threadIdx.x == 0) atomicOr(&b.meta->status, ST_INTERNAL);
      n = 0;
    }
    const uint64_t* in = b.sbuf + f0 * KW;
    // table: at least twice the keys (at most that many distinct), within the cap
    int bT = 6;
    while (bT < s.bT_max && ((uint64_t)1 << bT) < 2 * n) ++bT;
    Table<KW> tb;
    tb.keys = reinterpret_cast<K*>(sm);
    tb.counts = reinterpret_cast<uint32_t*>(tb.keys + (1u << bT));
    phase(7);
    table_clear<KW>(tb, 1u << bT);
    __syncthreads();
    phase(0);
    count_all<KW>(tb, in, n, false, K(0), K(0), bT, &nnew_s, &ovf_s, &special_s, &b.meta->status);
    __syncthreads();
    phase(1);
    const uint32_t dn = nnew_s;
    if (!ovf_s && dn <= dcap) {
      const uint64_t d = (uint64_t)dn + (special_s ? 1 : 0);
      if (threadIdx.x == 0) st_status(&b.look[g], (g == 0 ? kLookIncl : kLookAgg) | d);
      // order through this partition's spent input region (keys) and kbuf (counts)
      K lo;
      int sh;
      uint32_t NB;
      uint32_t rank[kRankPer];
      bucket_table<KW>(tb, 1u << bT, dn, b.sbuf + f0 * KW, stage_cnt_all + f0, hist, red_lo, red_hi, wtmp, prof, lo, sh,
                       NB);
      if (wid == 0) {
        const long long lb0 = clock64();
        const uint64_t ex = g == 0 ? 0 : lookback(b.look, g, &b.meta->status);
        if (lane == 0) {
          if (g > 0) st_status(&b.look[g], kLookIncl | (ex + d));
          excl_s = ex;
          if (s.profile)
            atomicAdd(reinterpret_cast<unsigned long long*>(&b.meta->phase_cycles[4]), (unsigned long long)(clock64() - lb0));
        }
      } else {
        load_and_rank<KW>(b.sbuf + f0 * KW, stage_cnt_all + f0, dn, dk, dc, hist, NB, lo, sh, rank, prof);
      }
      __syncthreads();
      phase(3);
      const uint64_t ex = excl_s;
      if (wid > 0) emit_ranked<KW>(dk, dc, dn, rank, ex, b.out_keys, b.out_counts, s.cap, &b.meta->status);
      if (special_s && threadIdx.x == 0) {
        if (ex + dn < s.cap) {
          store_key(b.out_keys, ex + dn, EMPTY);
          b.out_counts[ex + dn] = special_s;
        } else {
          atomicOr(&b.meta->status, ST_INTERNAL);
        }
      }
      __syncthreads();
      phase(5);
      continue;
    }
    // ---------------- overflow path: too many distinct keys for the table.  Split the
    // partition's key range into sub-ranges, each counted in its own table and ordered;
    // the exclusive prefix is resolved first because the partial outputs are written
    // before the total is known.  A sub-range narrower than the table holds fewer
    // distinct keys than slots, so the splitting ends.
    if (wid == 0) {
      const uint64_t ex = g == 0 ? 0 : lookback(b.look, g, &b.meta->status);
      if (lane == 0) excl_s = ex;
    }
    if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&b.meta->n_overflow), 1ull);
    K mn = EMPTY, mx = 0;
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) {
      K key;
      load_key(in, i, key);
      if (key != EMPTY) {
        mn = key < mn ? key : mn;
        mx = key > mx ? key : mx;
      }
    }
#pragma unroll
    for (int dd = 16; dd > 0; dd >>= 1) {
      const K a = shfl_key(mn, (lane + dd) & 31), c = shfl_key(mx, (lane + dd) & 31);
      mn = a < mn ? a : mn;
      mx = c > mx ? c : mx;
    }
    if (lane == 0) {
      red_lo[wid] = mn;
      red_hi[wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      K a = EMPTY, c = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        a = red_lo[w] < a ? red_lo[w] : a;
        c = red_hi[w] > c ? red_hi[w] : c;
      }
      stk_n = 0;
      if (a <= c) {
        stk_lo[0] = a;
        stk_hi[0] = c;
        stk_n = 1;
      }
    }
    __syncthreads();
    const int bTf = s.bT_max;
    tb.keys = reinterpret_cast<K*>(sm);
    tb.counts = reinterpret_cast<uint32_t*>(tb.keys + cap_slots);
    uint64_t written = 0;
    while (stk_n > 0) {
      const K lo = stk_lo[stk_n - 1], hi = stk_hi[stk_n - 1];
      __syncthreads();
      if (threadIdx.x == 0) {
        --stk_n;
        ovf_s = 0;
        special_s = 0;
        nnew_s = 0;
      }
      table_clear<KW>(tb, cap_slots);
      __syncthreads();
      count_all<KW>(tb, in, n, true, lo, hi, bTf, &nnew_s, &ovf_s, &special_s, &b.meta->status);
      __syncthreads();
      const uint32_t dn2 = nnew_s;
      const K width = hi - lo;
      if (ovf_s || dn2 > dcap) {
        if (threadIdx.x == 0) {
          if (width == 0 || stk_n + 2 > 160) {
            atomicOr(&b.meta->status, ST_INTERNAL);  // a single key cannot overflow
          } else {
            const K mid = lo + (width >> 1);
            stk_lo[stk_n] = mid + 1;
            stk_hi[stk_n] = hi;
            stk_lo[stk_n + 1] = lo;
            stk_hi[stk_n + 1] = mid;
            stk_n += 2;
          }
        }
        __syncthreads();
        continue;
      }
      // stage in the output region this sub-range will occupy, order, write back in place
      const uint64_t base = excl_s + written;
      if (base + dn2 > s.cap) {
        if (threadIdx.x == 0) atomicOr(&b.meta->status, ST_INTERNAL);
        __syncthreads();
        continue;
      }
      {
        K lo2;
        int sh2;
        uint32_t NB2;
        uint32_t rank2[kRankPer];
        bucket_table<KW>(tb, cap_slots, dn2, b.out_keys + base * KW, b.out_counts + base, hist, red_lo, red_hi, wtmp,
                         nullptr, lo2, sh2, NB2);
        if (wid > 0)
          load_and_rank<KW>(b.out_keys + base * KW, b.out_counts + base, dn2, dk, dc, hist, NB2, lo2, sh2, rank2,
                            nullptr);
        __syncthreads();
        if (wid > 0) emit_ranked<KW>(dk, dc, dn2, rank2, base, b.out_keys, b.out_counts, s.cap, &b.meta->status);
      }
      written += dn2;
      __syncthreads();
    }
    // the all-ones key, if present, is the largest key of all
    uint32_t sp = 0;
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) {
      K key;
      load_key(in, i, key);
      sp += key == EMPTY;
    }
#pragma unroll
    for (int dd = 16; dd > 0; dd >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, dd);
    if (lane == 0) wtmp[wid] = sp;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t tot = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wtmp[w];
      if (tot) {
        if (tot > 0xffffffffull) atomicOr(&b.meta->status, ST_COUNT_OVERFLOW);
        if (excl_s + written < s.cap) {
          store_key(b.out_keys, excl_s + written, EMPTY);
          b.out_counts[excl_s + written] = (uint32_t)tot;
        } else {
          atomicOr(&b.meta->status, ST_INTERNAL);
        }
        ++written;
      }
      st_status(&b.look[g], kLookIncl | (excl_s + written));
    }
    __syncthreads();
    phase(6);
  }
}

// ------------------------------------------------------------------ final: distinct total
__global__ void k_finish(Buffers b) {
  const uint64_t NF = b.meta->n_fine;
  if (NF == 0) {
    b.meta->n_distinct = 0;
    return;
  }
  const unsigned long long v = ld_status(&b.look[NF - 1]);
  if ((v >> 62) != 2) atomicOr(&b.meta->status, ST_INTERNAL);
  b.meta->n_distinct = v & kLookValue;
}

// ------------------------------------------------------------------ launches
static size_t scatter_smem(int kw, int nt, int P1) {
  const size_t sub = (size_t)nt * (kw == 1 ? 32 : 16);
  return sub * (size_t)(kw * 8) + (size_t)P1 * 8 + 2 * padded_len(P1) * 4;
}
static size_t fine_hist_smem(int P1) { return (size_t)(P1 + 1) * 4 + kFineLocalCap * 4 + P1 + 16; }
static size_t fine_scatter_smem(int kw, int P1) {
  return (size_t)kFineChunk * (kw * 8) + kFineLocalCap * 8 + 2 * padded_len(kFineLocalCap) * 4 + kFineChunk * 2 +
         (size_t)(P1 + 1) * 4 + P1 + 16;
}

int configure_kernels(int device) {
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return (int)e;
  // dynamic + static shared memory must fit the opt-in limit
#define KC_SET(fn)                                                                                          \
  {                                                                                                         \
    cudaFuncAttributes fa;                                                                                  \
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return (int)e;                                 \
    const int dyn = optin - (int)fa.sharedSizeBytes;                                                        \
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess) \
      return (int)e;                                                                                        \
  }
  KC_SET(k_pack_count<1>);
  KC_SET(k_pack_count<2>);
  KC_SET((k_scatter<1, 256>));
  KC_SET((k_scatter<2, 256>));
  KC_SET(k_fine_plan);
  KC_SET(k_fine_hist<1>);
  KC_SET(k_fine_hist<2>);
  KC_SET(k_fine_scatter<1>);
  KC_SET(k_fine_scatter<2>);
  KC_SET(k_count_emit<1>);
  KC_SET(k_count_emit<2>);
  KC_SET(k_bucket_scan);
#undef KC_SET
  return 0;
}

// After each launch: record the marker, and stop the sequence on a launch error so that
// no later kernel runs on buffers an earlier one did not fill (returns -cudaError_t).
#define KC_STEP(name)                                   \
  do {                                                  \
    const cudaError_t le = cudaGetLastError();          \
    if (le != cudaSuccess) return -(int)le;             \
    mark(name);                                         \
  } while (0)

int launch_phase1(const Shape& s, const Buffers& b, int n_sms, void* stream, const Marker& mark) {
  cudaStream_t st = (cudaStream_t)stream;
  const int P1 = 1 << s.b1;
  int launches = 0;
  if (s.n_reads > 0) {
    const uint64_t want = (s.n_reads + 255) / 256, lim = (uint64_t)n_sms * 8;
    const unsigned g = (unsigned)(want < lim ? want : lim);
    k_check_offsets<<<g, 256, 0, st>>>(b.offsets, s.n_reads, b.meta);
    ++launches;
    KC_STEP("k_check_offsets");
  }
  if (s.n_tiles == 0) return launches;
  k_tile_first<<<(unsigned)((s.n_tiles + 127) / 128), 128, 0, st>>>(b.offsets, s.n_reads, s.n_tiles, b.tile_first);
  ++launches;
  KC_STEP("k_tile_first");
  const size_t smA = (size_t)P1 * 4;
  if (s.kw == 1) k_pack_count<1><<<(unsigned)s.n_tiles, kPackThreads, smA, st>>>(s, b);
  else k_pack_count<2><<<(unsigned)s.n_tiles, kPackThreads, smA, st>>>(s, b);
  ++launches;
  KC_STEP("k_pack_count");
  k_col_scan<<<(unsigned)((P1 + 31) / 32), dim3(32, 32), 0, st>>>(b.hist, b.toff, b.cstart /* as ccount */, s.n_tiles, P1);
  ++launches;
  KC_STEP("k_col_scan");
  return launches;
}

int launch_phase2(const Shape& s, const Buffers& b, int n_sms, uint32_t nf_max, void* stream, const Marker& mark) {
  cudaStream_t st = (cudaStream_t)stream;
  const int P1 = 1 << s.b1;
  int launches = 0;
  // partition starts (cstart holds the per-partition counts written by k_col_scan; the
  // scan reads them into shared memory before overwriting)
  k_bucket_scan<<<1, 1024, (size_t)P1 * 8, st>>>(b.cstart, b.cstart, P1, b.meta);
  ++launches;
  KC_STEP("k_bucket_scan");
  if (s.n_tiles > 0) {
    const size_t smB = scatter_smem(s.kw, 256, P1);
    if (smB + 8704 > s.smem_budget) return -(int)cudaErrorInvalidConfiguration;
    const unsigned gt = (unsigned)s.n_tiles;
    if (s.kw == 1) k_scatter<1, 256><<<gt, 256, smB, st>>>(s, b);
    else k_scatter<2, 256><<<gt, 256, smB, st>>>(s, b);
    ++launches;
    KC_STEP("k_scatter");
  }
  k_fine_plan<<<1, 1024, (size_t)P1 * 8, st>>>(b.cstart, b.hll, b.fine_base, b.fine_log2, P1, s.fine_target, nf_max,
                                               b.meta);
  ++launches;
  KC_STEP("k_fine_plan");
  const unsigned gf = (unsigned)(n_sms * 2);
  if (s.kw == 1) k_fine_hist<1><<<gf, kFineThreads, fine_hist_smem(P1), st>>>(s, b);
  else k_fine_hist<2><<<gf, kFineThreads, fine_hist_smem(P1), st>>>(s, b);
  ++launches;
  KC_STEP("k_fine_hist");
  k_fine_scan<<<1, 1024, 0, st>>>(s, b);
  ++launches;
  KC_STEP("k_fine_scan");
  if (s.kw == 1) k_fine_scatter<1><<<gf, kFineThreads, fine_scatter_smem(1, P1), st>>>(s, b);
  else k_fine_scatter<2><<<gf, kFineThreads, fine_scatter_smem(2, P1), st>>>(s, b);
  ++launches;
  KC_STEP("k_fine_scatter");
  const size_t smC = count_kernel_smem(s.kw, s.bT_max, s.tail);
  if (s.kw == 1) k_count_emit<1><<<(unsigned)n_sms, kCountThreads, smC, st>>>(s, b);
  else k_count_emit<2><<<(unsigned)n_sms, kCountThreads, smC, st>>>(s, b);
  ++launches;
  KC_STEP("k_count_emit");
  k_finish<<<1, 1, 0, st>>>(b);
  ++launches;
  KC_STEP("k_finish");
  return launches;
}

}  // namespace kc

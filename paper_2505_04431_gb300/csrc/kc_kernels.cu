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
// top 64 bits of a 2k-bit key
__device__ __forceinline__ uint64_t top64(uint64_t key, int k) { return key << (64 - 2 * k); }
__device__ __forceinline__ uint64_t top64(u128 key, int k) { return (uint64_t)(key >> (2 * k - 64)); }
// monotone flattening map (see file comment)
__device__ __forceinline__ uint64_t utrans(uint64_t x, int canonical) {
  if (!canonical) return x;
  const uint64_t y = ~x;
  return ~__umul64hi(y, y);
}
__device__ __forceinline__ uint32_t field(uint64_t u, int skip, int bits) {
  return bits ? (uint32_t)((u << skip) >> (64 - bits)) : 0u;
}
template <class K> __device__ __forceinline__ K all_ones() { return ~(K)0; }

__device__ __forceinline__ uint64_t shfl_key(uint64_t v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ u128 shfl_key(u128 v, int src) {
  uint64_t lo = __shfl_sync(0xffffffffu, (uint64_t)v, src);
  uint64_t hi = __shfl_sync(0xffffffffu, (uint64_t)(v >> 64), src);
  return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
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

// Walk the 32 windows ending in the code word at `slot` (bases q0 .. q0+31); call
// f(o, key) for every valid window ending at q0 + o.  Slots slot-2, slot-1 hold the two
// previous words.  Valid: the k bases are ACGT and no read starts after the first of them.
template <int KW, class F>
__device__ __forceinline__ void for_windows(const uint64_t* code_s, const uint32_t* inv_s, const uint32_t* st_s, int slot,
                                            uint64_t q0, uint64_t L, int k, int canonical, F&& f) {
  typedef typename KeyT<KW>::T K;
  const K mask = key_mask(K(0), k);
  K fwd;
  if constexpr (KW == 1) fwd = (K)code_s[slot - 1] & mask;
  else fwd = (K)((((u128)code_s[slot - 2]) << 64) | code_s[slot - 1]) & mask;
  K rc = revcomp(fwd, k);
  const uint64_t yi = (uint64_t)inv_s[slot - 2] | ((uint64_t)inv_s[slot - 1] << 32);
  const uint64_t ys = (uint64_t)st_s[slot - 2] | ((uint64_t)st_s[slot - 1] << 32);
  int run = min(__clzll(yi), __clzll(ys) + 1);
  const uint64_t w = code_s[slot];
  const uint32_t iv = inv_s[slot], sv = st_s[slot];
  const uint64_t left = L - q0;
  const int nq = left < 32 ? (int)left : 32;
  const int sh = 2 * k - 2;
#pragma unroll
  for (int o = 0; o < 32; ++o) {
    const uint32_t c = (uint32_t)(w >> (62 - 2 * o)) & 3u;
    const int ib = (iv >> o) & 1, sb = (sv >> o) & 1;
    run = ib ? 0 : (sb ? 1 : min(run + 1, 64));
    fwd = ((fwd << 2) | (K)c) & mask;
    rc = (rc >> 2) | ((K)(3u - c) << sh);
    if (o < nq && run >= k) {
      const K key = (canonical && rc < fwd) ? rc : fwd;
      f(o, key);
    }
  }
}

template <class K>
__device__ __forceinline__ uint32_t coarse_of(K key, int k, int canonical, int b1) {
  return field(utrans(top64(key, k), canonical), 0, b1);
}

// ------------------------------------------------------------------ pass A
template <int KW>
__global__ void __launch_bounds__(kPackThreads) k_pack_count(Shape s, Buffers b) {
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
    __syncthreads();
    const uint64_t j = j0 + t;
    if (j < s.n_words) {
      uint64_t code;
      uint32_t inv;
      convert_word(b.reads, s.L, j, code, inv);
      b.codes64[j] = code;
      b.inv32[j] = inv;
      code_s[t + 2] = code;
      inv_s[t + 2] = inv;
    } else {
      code_s[t + 2] = 0;
      inv_s[t + 2] = ~0u;
    }
    st_s[t + 2] = 0;
    if (t < 2) st_s[t] = 0;
    __syncthreads();
    build_starts(b.offsets, s.n_reads, j0, kPackThreads, st_s, &rcur_s);
    __syncthreads();
    if (j < s.n_words) {
      for_windows<KW>(code_s, inv_s, st_s, t + 2, j * 32, s.L, s.k, s.canonical, [&](int, K key) {
        atomicAdd(&hist_s[coarse_of(key, s.k, s.canonical, s.b1)], 1u);
      });
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

// Partition starts, fine split per partition, totals.  One block.
__global__ void k_bucket_scan(const uint64_t* ccount, uint64_t* cstart, uint32_t* fine_base, uint8_t* fine_log2, int P1,
                              uint32_t fine_target, uint32_t nf_max, Meta* meta) {
  extern __shared__ uint64_t sc[];  // [P1] then [P1] u64
  __shared__ uint64_t wt[32];
  uint64_t* a = sc;
  uint64_t* f = sc + P1;
  for (int c = threadIdx.x; c < P1; c += blockDim.x) {
    const uint64_t n = ccount[c];
    a[c] = n;
    const uint64_t m = (n + fine_target - 1) / fine_target;
    int bf = m <= 1 ? 0 : 64 - __clzll(m - 1);
    bf = min(bf, kMaxFineLog2);
    fine_log2[c] = (uint8_t)bf;
    f[c] = 1ull << bf;
  }
  __syncthreads();
  const uint64_t K = block_exclusive_scan<uint64_t>(a, P1, wt);
  const uint64_t NF = block_exclusive_scan<uint64_t>(f, P1, wt);
  for (int c = threadIdx.x; c < P1; c += blockDim.x) {
    cstart[c] = a[c];
    fine_base[c] = (uint32_t)f[c];
  }
  if (threadIdx.x == 0) {
    cstart[P1] = K;
    fine_base[P1] = (uint32_t)NF;
    meta->n_windows = K;
    meta->n_fine = NF <= nf_max ? NF : 0;  // later kernels never index past nf_max
    if (NF > nf_max) atomicOr(&meta->status, ST_INTERNAL);
  }
}

// ------------------------------------------------------------------ pass B
template <int KW, int NT>
__global__ void __launch_bounds__(NT) k_scatter(Shape s, Buffers b) {
  typedef typename KeyT<KW>::T K;
  constexpr int SUB = NT * 32;  // windows per sub-step
  extern __shared__ __align__(16) uint8_t sm[];
  const int P1 = 1 << s.b1;
  K* stage = reinterpret_cast<K*>(sm);                                     // [SUB]
  uint16_t* stage_c = reinterpret_cast<uint16_t*>(stage + SUB);            // [SUB]
  uint64_t* cursor = reinterpret_cast<uint64_t*>(stage_c + SUB);           // [P1]
  uint32_t* hist = reinterpret_cast<uint32_t*>(cursor + P1);               // [P1]
  uint32_t* soff = hist + P1;                                              // [P1]
  __shared__ uint64_t code_s[NT + 2];
  __shared__ uint32_t inv_s[NT + 2];
  __shared__ uint32_t st_s[NT + 2];
  __shared__ uint64_t rcur_s;
  __shared__ uint32_t wt[32];
  const int t = threadIdx.x;
  const uint64_t tile = blockIdx.x;
  for (int c = t; c < P1; c += NT) {
    cursor[c] = b.cstart[c] + b.toff[tile * P1 + c];
    hist[c] = 0;
  }
  if (t == 0) rcur_s = b.tile_first[tile];
  for (int sub = 0; sub < kTileWords / NT; ++sub) {
    const uint64_t j0 = tile * kTileWords + (uint64_t)sub * NT;
    if (j0 >= s.n_words) break;
    __syncthreads();
    if (t < 2) {
      if (sub > 0) {
        code_s[t] = code_s[NT + t];
        inv_s[t] = inv_s[NT + t];
      } else if (j0 + t >= 2) {
        code_s[t] = b.codes64[j0 + t - 2];
        inv_s[t] = b.inv32[j0 + t - 2];
      } else {
        code_s[t] = 0;
        inv_s[t] = ~0u;
      }
    }
    __syncthreads();
    const uint64_t j = j0 + t;
    if (j < s.n_words) {
      code_s[t + 2] = b.codes64[j];
      inv_s[t + 2] = b.inv32[j];
    } else {
      code_s[t + 2] = 0;
      inv_s[t + 2] = ~0u;
    }
    st_s[t + 2] = 0;
    if (t < 2) st_s[t] = 0;
    __syncthreads();
    build_starts(b.offsets, s.n_reads, j0, NT, st_s, &rcur_s);
    __syncthreads();
    // rank of every window inside its partition (shared-memory counting sort, step 1)
    uint32_t rr[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) rr[i] = 0;
    if (j < s.n_words) {
      for_windows<KW>(code_s, inv_s, st_s, t + 2, j * 32, s.L, s.k, s.canonical, [&](int o, K key) {
        const uint32_t r = atomicAdd(&hist[coarse_of(key, s.k, s.canonical, s.b1)], 1u);
        rr[o >> 1] |= r << (16 * (o & 1));
      });
    }
    __syncthreads();
    for (int c = t; c < P1; c += NT) soff[c] = hist[c];
    __syncthreads();
    block_exclusive_scan<uint32_t>(soff, P1, wt);
    // step 2: place every key at its partition's run in the staging buffer
    if (j < s.n_words) {
      for_windows<KW>(code_s, inv_s, st_s, t + 2, j * 32, s.L, s.k, s.canonical, [&](int o, K key) {
        const uint32_t c = coarse_of(key, s.k, s.canonical, s.b1);
        const uint32_t pos = soff[c] + ((rr[o >> 1] >> (16 * (o & 1))) & 0xffffu);
        stage[pos] = key;
        stage_c[pos] = (uint16_t)c;
      });
    }
    __syncthreads();
    // step 3: runs leave in order, consecutive threads on consecutive addresses
    const uint32_t n_sub = soff[P1 - 1] + hist[P1 - 1];
    for (uint32_t i = t; i < n_sub; i += NT) {
      const uint32_t c = stage_c[i];
      if (c >= (uint32_t)P1) {
        atomicOr(&b.meta->status, ST_INTERNAL);
        continue;
      }
      const uint64_t pos = cursor[c] + (i - soff[c]);
      if (pos < s.cap) store_key(b.kbuf, pos, stage[i]);
      else atomicOr(&b.meta->status, ST_INTERNAL);
    }
    __syncthreads();
    for (int c = t; c < P1; c += NT) {
      cursor[c] += hist[c];
      hist[c] = 0;
    }
  }
}

// ------------------------------------------------------------------ phase 2: fine split
struct FineCtx {
  int k, canonical, b1;
};

template <class K>
__device__ __forceinline__ uint32_t fine_index(K key, const FineCtx& x, const uint32_t* fine_base_s, const uint8_t* flog_s) {
  const uint64_t u = utrans(top64(key, x.k), x.canonical);
  const uint32_t c = field(u, 0, x.b1);
  return fine_base_s[c] + field(u, x.b1, flog_s[c]);
}

template <int KW>
__device__ __forceinline__ void load_fine_tables(const Buffers& b, int P1, uint32_t* fine_base_s, uint8_t* flog_s) {
  for (int c = threadIdx.x; c <= P1; c += blockDim.x) fine_base_s[c] = b.fine_base[c];
  for (int c = threadIdx.x; c < P1; c += blockDim.x) flog_s[c] = b.fine_log2[c];
}

constexpr int kFineThreads = 512;
constexpr int kFinePer = 8;  // keys per thread per chunk
constexpr int kFineChunk = kFineThreads * kFinePer;

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
#pragma unroll
    for (int m = 0; m < kFinePer; ++m) {
      const uint64_t i = c0 + threadIdx.x + (uint64_t)m * kFineThreads;
      if (i < c1) {
        K key;
        load_key(b.kbuf, i, key);
        const uint32_t g = fine_index(key, x, fine_base_s, flog_s);
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
  uint32_t* lh = reinterpret_cast<uint32_t*>(gbase + kFineLocalCap);          // [kFineLocalCap]
  uint32_t* soff = lh + kFineLocalCap;                                        // [kFineLocalCap]
  uint16_t* stage_g = reinterpret_cast<uint16_t*>(soff + kFineLocalCap);      // [kFineChunk]
  uint32_t* fine_base_s = reinterpret_cast<uint32_t*>(stage_g + kFineChunk);  // [P1+1]
  uint8_t* flog_s = reinterpret_cast<uint8_t*>(fine_base_s + P1 + 1);         // [P1]
  __shared__ uint32_t g_lo_s, g_hi_s;
  __shared__ uint32_t wt[32];
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
#pragma unroll
    for (int m = 0; m < kFinePer; ++m) {
      const uint64_t i = c0 + threadIdx.x + (uint64_t)m * kFineThreads;
      gr[m] = 0xffffffffu;
      if (i < c1) {
        load_key(b.kbuf, i, keys[m]);
        const uint32_t lg = fine_index(keys[m], x, fine_base_s, flog_s) - g_lo;
        if (lg < span) {
          const uint32_t r = atomicAdd(&lh[lg], 1u);
          gr[m] = (lg << 16) | r;
        } else {
          atomicOr(&b.meta->status, ST_INTERNAL);
        }
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < span; i += kFineThreads) soff[i] = lh[i];
    __syncthreads();
    block_exclusive_scan<uint32_t>(soff, (int)span, wt);
    for (uint32_t i = threadIdx.x; i < span; i += kFineThreads) {
      const uint32_t v = lh[i];
      if (v) gbase[i] = g_lo + i < s.nf_max ? atomicAdd(&b.fcur[g_lo + i], (unsigned long long)v) : ~0ull;
    }
#pragma unroll
    for (int m = 0; m < kFinePer; ++m) {
      if (gr[m] != 0xffffffffu) {
        const uint32_t lg = gr[m] >> 16;
        const uint32_t pos = soff[lg] + (gr[m] & 0xffffu);
        stage[pos] = keys[m];
        stage_g[pos] = (uint16_t)lg;
      }
    }
    __syncthreads();
    // only the keys that were staged (a key outside the chunk's fine range was rejected above)
    const uint32_t n_staged = soff[span - 1] + lh[span - 1];
    for (uint32_t i = threadIdx.x; i < n_staged; i += kFineThreads) {
      const uint32_t lg = stage_g[i];
      if (lg >= span) {
        atomicOr(&b.meta->status, ST_INTERNAL);
        continue;
      }
      const uint64_t pos = gbase[lg] + (i - soff[lg]);
      if (pos < s.cap) store_key(b.sbuf, pos, stage[i]);
      else atomicOr(&b.meta->status, ST_INTERNAL);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < span; i += kFineThreads) lh[i] = 0;
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
      v = ld_acquire(&look[idx]);
      while ((v >> 62) == 0) {
        if (++spins > kLookbackSpinLimit) {
          atomicOr(status, ST_TIMEOUT);
          v = kLookIncl;
          break;
        }
        __nanosleep(64);
        v = ld_acquire(&look[idx]);
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

// Count kernel shared memory: a hash table of 2^bT_max slots (key + count).  After the
// count, the same bytes hold the dense array of distinct keys (at most 3/4 of the slots)
// and the bucket histogram used to order them.
size_t count_kernel_smem(int kw, int bT_max, int /*unused*/) {
  const size_t slots = (size_t)1 << bT_max;
  return slots * (size_t)(kw * 8 + 4) + 256;
}

int table_log2_max(int kw, size_t smem_optin) {
  int best = 6;
  for (int bt = 6; bt <= 16; ++bt)
    if (count_kernel_smem(kw, bt, 0) + 8192 <= smem_optin) best = bt;  // 8 KB for static shared memory
  return best;
}

constexpr int kProbeLimit = 128;
constexpr int kWorkers = kCountThreads - 32;  // warps 1.. order and sort while warp 0 looks back
constexpr int kBigCap = 256;                  // buckets too large for one thread, sorted per warp

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
  const K EMPTY = all_ones<K>();
  const int lane = threadIdx.x & 31;
  for (uint64_t base = 0; base < n; base += 2 * (uint64_t)blockDim.x) {
    K kk[2];
    bool aa[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {  // two loads in flight per thread
      const uint64_t i = base + (uint64_t)m * blockDim.x + threadIdx.x;
      kk[m] = 0;
      aa[m] = i < n;
      if (aa[m]) load_key(in, i, kk[m]);
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) {
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

// Write the occupied slots (unordered) to stage_keys / stage_counts[0, d).
template <int KW>
__device__ void stage_table(Table<KW> tb, uint32_t nslots, uint64_t* stage_keys, uint32_t* stage_counts,
                            uint32_t* cursor) {
  typedef typename KeyT<KW>::T K;
  const K EMPTY = all_ones<K>();
  const int lane = threadIdx.x & 31;
  for (uint32_t base = (threadIdx.x & ~31u); base < nslots; base += blockDim.x) {
    const uint32_t s = base + lane;
    const bool occ = s < nslots && tb.keys[s] != EMPTY;
    const unsigned m = __ballot_sync(0xffffffffu, occ);
    uint32_t pos = 0;
    if (lane == 0 && m) pos = atomicAdd(cursor, __popc(m));
    pos = __shfl_sync(0xffffffffu, pos, 0);
    if (occ) {
      const uint32_t o = pos + __popc(m & ((1u << lane) - 1));
      store_key(stage_keys, o, tb.keys[s]);
      stage_counts[o] = tb.counts[s];
    }
  }
}

// Exclusive scan of data[0, n) by the worker threads (named barrier 1); returns the total.
template <typename T>
__device__ T workers_exclusive_scan(T* data, int n, T* warp_tmp) {
  const int t = threadIdx.x - 32, nt = kWorkers, lane = t & 31, wid = t >> 5, nw = kWorkers / 32;
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
  bar_workers();
  if (wid == 0) {
    T w = lane < nw ? warp_tmp[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < nw) warp_tmp[lane] = w;
  }
  bar_workers();
  T run = x - s + (wid ? warp_tmp[wid - 1] : 0);
  const T total = warp_tmp[nw - 1];
  for (int i = lo; i < hi; ++i) {
    T v = data[i];
    data[i] = run;
    run += v;
  }
  bar_workers();
  return total;
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

// Order the d staged entries by key into dense_keys / dense_counts (shared memory):
// an ordered counting sort into NB buckets (bucket = bfn(key), non-decreasing in the
// key), then a sort inside every bucket.  Run by the worker warps only.
template <int KW, class B>
__device__ void order_entries(const uint64_t* stage_keys, const uint32_t* stage_counts, uint32_t d,
                              typename KeyT<KW>::T* dense_keys, uint32_t* dense_counts, uint32_t* hist, uint32_t NB,
                              B&& bfn, uint32_t* big_list, uint32_t* big_n, uint32_t* warp_tmp) {
  typedef typename KeyT<KW>::T K;
  const int t = threadIdx.x - 32;
  for (uint32_t i = t; i < NB; i += kWorkers) hist[i] = 0;
  if (t == 0) *big_n = 0;
  bar_workers();
  constexpr int kMaxPer = 16;  // d <= kMaxPer * kWorkers (checked by the caller)
  uint32_t br[kMaxPer];
#pragma unroll
  for (int m = 0; m < kMaxPer; ++m) {
    const uint32_t i = t + m * kWorkers;
    br[m] = 0xffffffffu;
    if (i < d) {
      K key;
      load_key(stage_keys, i, key);
      const uint32_t bk = bfn(key);
      const uint32_t r = atomicAdd(&hist[bk], 1u);
      br[m] = (bk << 16) | r;  // NB <= 2^15 buckets, rank < 2^16
    }
  }
  bar_workers();
  // bucket sizes are kept in the second half of hist's space? no: scan in place, sizes recomputed below
  workers_exclusive_scan<uint32_t>(hist, (int)NB, warp_tmp);
#pragma unroll
  for (int m = 0; m < kMaxPer; ++m) {
    const uint32_t i = t + m * kWorkers;
    if (i < d) {
      K key;
      load_key(stage_keys, i, key);
      const uint32_t pos = hist[br[m] >> 16] + (br[m] & 0xffffu);
      dense_keys[pos] = key;
      dense_counts[pos] = stage_counts[i];
    }
  }
  bar_workers();
  // sort inside buckets: short ones by one thread, long ones queued for a warp
  for (uint32_t bk = t; bk < NB; bk += kWorkers) {
    const uint32_t a = hist[bk];
    const uint32_t e = bk + 1 < NB ? hist[bk + 1] : d;
    const uint32_t c = e - a;
    if (c < 2) continue;
    if (c > 32) {
      const uint32_t q = atomicAdd(big_n, 1u);
      if (q < kBigCap) {
        big_list[q] = bk;
        continue;
      }
    }
    for (uint32_t i = a + 1; i < e; ++i) {
      const K kv = dense_keys[i];
      const uint32_t cv = dense_counts[i];
      uint32_t m = i;
      while (m > a && dense_keys[m - 1] > kv) {
        dense_keys[m] = dense_keys[m - 1];
        dense_counts[m] = dense_counts[m - 1];
        --m;
      }
      dense_keys[m] = kv;
      dense_counts[m] = cv;
    }
  }
  bar_workers();
  const uint32_t nbig = min(*big_n, (uint32_t)kBigCap);
  for (uint32_t q = (uint32_t)(t >> 5); q < nbig; q += kWorkers / 32) {
    const uint32_t bk = big_list[q];
    const uint32_t a = hist[bk];
    const uint32_t e = bk + 1 < NB ? hist[bk + 1] : d;
    warp_sort_segment<K>(dense_keys, dense_counts, a, e - a);
  }
}

// Coalesced copy of the dense sorted entries to out[base, base + d).
template <int KW>
__device__ void emit_dense(const typename KeyT<KW>::T* dense_keys, const uint32_t* dense_counts, uint32_t d,
                           uint64_t base, uint64_t* out_keys, uint32_t* out_counts, uint64_t cap, uint32_t* status) {
  if (base + d > cap) {
    if (threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
    return;
  }
  for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) {
    store_key(out_keys, base + i, dense_keys[i]);
    out_counts[base + i] = dense_counts[i];
  }
}

template <class K> __device__ __forceinline__ int bitlen(K v);
template <> __device__ __forceinline__ int bitlen(uint64_t v) { return 64 - __clzll(v); }
template <> __device__ __forceinline__ int bitlen(u128 v) {
  const uint64_t hi = (uint64_t)(v >> 64);
  return hi ? 128 - __clzll(hi) : 64 - __clzll((uint64_t)v);
}

__device__ __forceinline__ int ceil_log2_u32(uint32_t v) { return v <= 1 ? 0 : 32 - __clz(v - 1); }

template <int KW>
__global__ void __launch_bounds__(kCountThreads, 1) k_count_emit(Shape s, Buffers b) {
  typedef typename KeyT<KW>::T K;
  extern __shared__ __align__(16) uint8_t sm[];
  const uint32_t cap_slots = 1u << s.bT_max;
  __shared__ uint64_t g_s, excl_s;
  __shared__ uint32_t ovf_s, special_s, nnew_s, cursor_s, c_s, flog_s, big_n;
  __shared__ uint32_t wtmp[32];
  __shared__ uint32_t big_list[kBigCap];
  __shared__ K red_lo[32], red_hi[32];
  __shared__ K stk_lo[160], stk_hi[160];
  __shared__ int stk_n;
  const K EMPTY = all_ones<K>();
  const int P1 = 1 << s.b1;
  const uint64_t NF = b.meta->n_fine;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* stage_cnt_all = reinterpret_cast<uint32_t*>(b.kbuf);  // kbuf is free once the fine split is done
  // profiled plans: thread 0 adds the cycles spent in each phase (0 clear, 1 count, 2 stage,
  // 3 order + sort, 4 look-back, 5 emit, 6 overflow path, 7 ticket + setup)
  long long t_mark = clock64();
  auto phase = [&](int i) {
    if (s.profile && threadIdx.x == 0) {
      const long long now = clock64();
      atomicAdd(reinterpret_cast<unsigned long long*>(&b.meta->phase_cycles[i]), (unsigned long long)(now - t_mark));
      t_mark = now;
    }
  };
  // the dense array and histogram reuse the table bytes: layout for a table of 2^bT slots
  auto dense_layout = [&](int bT, K*& dk, uint32_t*& dc, uint32_t*& hist, uint32_t& dcap) {
    dcap = (3u << bT) >> 2;
    dk = reinterpret_cast<K*>(sm);
    dc = reinterpret_cast<uint32_t*>(dk + dcap);
    hist = dc + dcap;
  };
  while (true) {
    if (threadIdx.x == 0) {
      g_s = atomicAdd(reinterpret_cast<unsigned long long*>(&b.meta->ticket), 1ull);
      ovf_s = 0;
      special_s = 0;
      nnew_s = 0;
      cursor_s = 0;
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
    if (threadIdx.x == 0) {  // coarse partition of g: last c with fine_base[c] <= g
      int lo = 0, hi = P1 - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.fine_base[mid] <= (uint32_t)g) lo = mid; else hi = mid - 1;
      }
      c_s = (uint32_t)lo;
      flog_s = b.fine_log2[lo];
    }
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
    K* dk;
    uint32_t *dc, *hist, dcap;
    dense_layout(bT, dk, dc, hist, dcap);
    const uint32_t dn = nnew_s;
    if (!ovf_s && dn <= dcap && dn <= 16u * kWorkers) {
      const uint64_t d = (uint64_t)dn + (special_s ? 1 : 0);
      if (threadIdx.x == 0) st_release(&b.look[g], (g == 0 ? kLookIncl : kLookAgg) | d);
      // stage the distinct entries in this partition's spent input region
      stage_table<KW>(tb, 1u << bT, b.sbuf + f0 * KW, stage_cnt_all + f0, &cursor_s);
      __syncthreads();
      phase(2);
      if (wid == 0) {
        const uint64_t ex = g == 0 ? 0 : lookback(b.look, g, &b.meta->status);
        if (lane == 0) {
          if (g > 0) st_release(&b.look[g], kLookIncl | (ex + d));
          excl_s = ex;
        }
      } else {
        uint32_t NB = 1;
        while (NB < 32768u && NB * 2 <= dn) NB <<= 1;  // about two entries per bucket
        const int bB = ceil_log2_u32(NB);
        const int skip = s.b1 + (int)flog_s;
        const int kk = s.k, canon = s.canonical;
        order_entries<KW>(b.sbuf + f0 * KW, stage_cnt_all + f0, dn, dk, dc, hist, NB,
                          [&](K key) { return field(utrans(top64(key, kk), canon), skip, bB); }, big_list, &big_n,
                          wtmp);
      }
      __syncthreads();
      phase(3);
      const uint64_t ex = excl_s;
      emit_dense<KW>(dk, dc, dn, ex, b.out_keys, b.out_counts, s.cap, &b.meta->status);
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
    // partition's key range into sub-ranges, each counted in its own table and ordered
    // with buckets (key - lo) >> shift; the exclusive prefix is resolved first because
    // the partial outputs are written before the total is known.  A sub-range narrower
    // than the table holds fewer distinct keys than slots, so the splitting ends.
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
    dense_layout(bTf, dk, dc, hist, dcap);
    uint64_t written = 0;
    while (stk_n > 0) {
      const K lo = stk_lo[stk_n - 1], hi = stk_hi[stk_n - 1];
      __syncthreads();
      if (threadIdx.x == 0) {
        --stk_n;
        ovf_s = 0;
        special_s = 0;
        nnew_s = 0;
        cursor_s = 0;
      }
      table_clear<KW>(tb, cap_slots);
      __syncthreads();
      count_all<KW>(tb, in, n, true, lo, hi, bTf, &nnew_s, &ovf_s, &special_s, &b.meta->status);
      __syncthreads();
      const uint32_t dn2 = nnew_s;
      const K width = hi - lo;
      if (ovf_s || dn2 > dcap || dn2 > 16u * kWorkers) {
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
      stage_table<KW>(tb, cap_slots, b.out_keys + base * KW, b.out_counts + base, &cursor_s);
      __syncthreads();
      if (wid > 0) {
        uint32_t NB = 1;
        while (NB < 32768u && NB * 2 <= dn2) NB <<= 1;
        const int bB = ceil_log2_u32(NB);
        const int sh = max(0, bitlen(width) - bB);
        order_entries<KW>(b.out_keys + base * KW, b.out_counts + base, dn2, dk, dc, hist, NB,
                          [&](K key) { return (uint32_t)((key - lo) >> sh); }, big_list, &big_n, wtmp);
      }
      __syncthreads();
      emit_dense<KW>(dk, dc, dn2, base, b.out_keys, b.out_counts, s.cap, &b.meta->status);
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
      st_release(&b.look[g], kLookIncl | (excl_s + written));
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
  const unsigned long long v = ld_acquire(&b.look[NF - 1]);
  if ((v >> 62) != 2) atomicOr(&b.meta->status, ST_INTERNAL);
  b.meta->n_distinct = v & kLookValue;
}

// ------------------------------------------------------------------ launches
static size_t scatter_smem(int kw, int nt, int P1) {
  const size_t sub = (size_t)nt * 32;
  return sub * (size_t)(kw * 8) + sub * 2 + (size_t)P1 * 8 + (size_t)P1 * 8;
}
// threads per CTA of pass B: the largest of 512/256/128 whose staging fits shared memory
static int scatter_threads(int kw, int P1, size_t budget) {
  for (int nt = kw == 1 ? 512 : 256; nt >= 128; nt >>= 1)
    if (scatter_smem(kw, nt, P1) <= budget) return nt;
  return 0;
}
static size_t fine_hist_smem(int P1) { return (size_t)(P1 + 1) * 4 + kFineLocalCap * 4 + P1 + 16; }
static size_t fine_scatter_smem(int kw, int P1) {
  return (size_t)kFineChunk * (kw * 8) + kFineLocalCap * (8 + 4 + 4) + kFineChunk * 2 + (size_t)(P1 + 1) * 4 + P1 + 16;
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
  KC_SET((k_scatter<1, 512>));
  KC_SET((k_scatter<1, 256>));
  KC_SET((k_scatter<1, 128>));
  KC_SET((k_scatter<2, 256>));
  KC_SET((k_scatter<2, 128>));
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
  k_bucket_scan<<<1, 1024, (size_t)P1 * 16, st>>>(b.cstart, b.cstart, b.fine_base, b.fine_log2, P1, s.fine_target, nf_max,
                                                   b.meta);
  ++launches;
  KC_STEP("k_bucket_scan");
  if (s.n_tiles > 0) {
    // budget: opt-in shared memory minus the kernel's static part (at most 8.5 KB)
    const int nt = scatter_threads(s.kw, P1, s.smem_budget - 8704);
    if (nt == 0) return -(int)cudaErrorInvalidConfiguration;
    const size_t smB = scatter_smem(s.kw, nt, P1);
    const unsigned gt = (unsigned)s.n_tiles;
    if (s.kw == 1) {
      if (nt == 512) k_scatter<1, 512><<<gt, 512, smB, st>>>(s, b);
      else if (nt == 256) k_scatter<1, 256><<<gt, 256, smB, st>>>(s, b);
      else k_scatter<1, 128><<<gt, 128, smB, st>>>(s, b);
    } else {
      if (nt == 256) k_scatter<2, 256><<<gt, 256, smB, st>>>(s, b);
      else k_scatter<2, 128><<<gt, 128, smB, st>>>(s, b);
    }
    ++launches;
    KC_STEP("k_scatter");
  }
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

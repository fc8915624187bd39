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
//   k_fine_plan, k_fine_hist, k_fine_scan, k_fine_scatter   split every owner partition
//                           into fine partitions small enough for one shared-memory table
//                           (sized from a HyperLogLog estimate of the distinct keys).
//   k_count_emit            persistent; per fine partition: count every key in a hashed
//                           open-addressing table in shared memory (CAS claims a slot, a
//                           32-bit atomic add counts), order the occupied slots by a
//                           bucketed counting sort over the partition's key range, and
//                           write the sorted (key, count) run at the offset found by a
//                           decoupled look-back over the fine partitions, or in its own
//                           input region when that offset is not known in time.
//   k_scan_distinct, k_compact   output offsets of all runs; the runs written in place
//                           move to their offsets.
// Variants: every kernel body also runs as a batched kernel (one launch for a group of
// counts, each thread block working for one count found through a block table); pass B
// without the shared-memory staging (DIRECT) and the count kernel with a warp-level merge
// of equal keys (the heavy-hitter pre-aggregation of Section IV-D; slower on GB300, so off
// by default) exist for the aggregation experiment of Section VI.
//
// Owner partitions are key ranges (not hashes) so that the per-partition outputs
// concatenate into one ascending array.  A monotone map u(key) of the top 32 key bits
// flattens the distribution of canonical keys (the min of two near-independent uniforms
// has density 2(1-x); u = 1 - (1-x)^2 is its distribution function); the coarse partition
// is the top bits of u and the fine partitions split each coarse range of u into equal
// parts, so both are non-decreasing in the key.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kc_internal.h"

namespace kc {

typedef unsigned __int128 u128;

// Batched launches: each block finds its count (one table load), copies the count's
// descriptor to shared memory and runs the kernel body for that count.
__device__ __forceinline__ void batch_locate(const BatchTab& t, BatchDesc& d_s, uint32_t& bid_s, uint32_t& nblk_s) {
  __shared__ uint32_t i_s;
  const uint32_t tid = threadIdx.x + threadIdx.y * blockDim.x, nth = blockDim.x * blockDim.y;
  if (tid == 0) {
    const uint32_t i = t.blk2s[blockIdx.x];
    const uint32_t a = t.start[i];
    i_s = i;
    bid_s = blockIdx.x - a;
    nblk_s = t.start[i + 1] - a;
  }
  __syncthreads();
  const uint32_t* src = reinterpret_cast<const uint32_t*>(t.desc + i_s);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&d_s);
  for (uint32_t w = tid; w < sizeof(BatchDesc) / 4; w += nth) dst[w] = src[w];
  __syncthreads();
}
#define KC_BATCH_PROLOGUE(t)                 \
  __shared__ BatchDesc d_s_;                 \
  __shared__ uint32_t bid_s_, nblk_s_;       \
  batch_locate(t, d_s_, bid_s_, nblk_s_);    \
  const BatchDesc& d = d_s_;                 \
  const uint32_t bid = bid_s_, nblk = nblk_s_; \
  (void)bid;                                 \
  (void)nblk

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
// Asynchronous 4- and 8-byte copies from global to shared memory (cp.async); the issuing
// thread waits for all of its copies with cp_async_wait_all.
__device__ __forceinline__ void cp_async4(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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
// Batched launches: the arrays a count needs zeroed (status record, fine histogram,
// look-back words, sketch, partition starts) are cleared by one kernel for all counts.
__global__ void k_clear_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  const Shape& s = d.s;
  const Buffers& b = d.b;
  const uint64_t i0 = (uint64_t)bid * blockDim.x + threadIdx.x, stride = (uint64_t)nblk * blockDim.x;
  for (uint64_t i = i0; i < s.nf_max; i += stride) {
    b.fhist[i] = 0;
    b.look[i] = 0;
  }
  for (uint64_t i = i0; i < (uint64_t)kHllRegs; i += stride) b.hll[i] = 0;
  for (uint64_t i = i0; i <= (1ull << s.b1); i += stride) b.cstart[i] = 0;
  for (uint64_t i = i0; i < sizeof(Meta) / 4; i += stride) reinterpret_cast<uint32_t*>(b.meta)[i] = 0;
}

__device__ __forceinline__ void check_offsets_body(const uint64_t* offsets, uint64_t n_reads, uint64_t L, Meta* meta,
                                                   uint32_t bid, uint32_t nblk) {
  for (uint64_t i = bid * (uint64_t)blockDim.x + threadIdx.x; i < n_reads; i += (uint64_t)nblk * blockDim.x) {
    if (offsets[i + 1] < offsets[i]) atomicOr(&meta->status, ST_BAD_OFFSETS);
  }
  if (bid == 0 && threadIdx.x == 0 && (offsets[0] != 0 || offsets[n_reads] != L))
    atomicOr(&meta->status, ST_BAD_OFFSETS);
}
__global__ void k_check_offsets(const uint64_t* offsets, uint64_t n_reads, uint64_t L, Meta* meta) {
  check_offsets_body(offsets, n_reads, L, meta, blockIdx.x, gridDim.x);
}
__global__ void k_check_offsets_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  check_offsets_body(d.b.offsets, d.s.n_reads, d.s.L, d.b.meta, bid, nblk);
}

// first read whose start is >= the halo start of each tile (lower bound in offsets)
__device__ __forceinline__ void tile_first_body(const uint64_t* offsets, uint64_t n_reads, uint64_t n_tiles,
                                                uint64_t* tile_first, uint32_t bid) {
  const uint64_t t = bid * (uint64_t)blockDim.x + threadIdx.x;
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
__global__ void k_tile_first(const uint64_t* offsets, uint64_t n_reads, uint64_t n_tiles, uint64_t* tile_first) {
  tile_first_body(offsets, n_reads, n_tiles, tile_first, blockIdx.x);
}
__global__ void k_tile_first_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  tile_first_body(d.b.offsets, d.s.n_reads, d.s.n_tiles, d.b.tile_first, bid);
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
// x >> s, and 0 for s >= 32 (one clamping funnel shift)
__device__ __forceinline__ uint32_t shr_clamp(uint32_t x, uint32_t s) { return __funnelshift_rc(x, 0u, s); }
// the coarse field of u: its top b1 bits (none for b1 = 0)
__device__ __forceinline__ uint32_t coarse_field(uint32_t u, int b1) { return shr_clamp(u, 32 - b1); }
template <class K>
__device__ __forceinline__ uint32_t coarse_of(K key, int k, int canonical, int b1) {
  return coarse_field(umap(top32_of(key, k), canonical), b1);
}

// floor(sqrt(v)) from 32-bit conversions and single-precision arithmetic (64-bit
// conversions and double precision are slow on this GPU): the single-precision root is
// within 2^32 * 2^-24 of the true one; one Newton step on the exact residual brings it
// within a few units, and exact integer comparisons finish.  The root is below 2^32, so
// every square fits in 64 bits.
__host__ __device__ __forceinline__ float u64_to_float(uint64_t v) {
  return (float)(uint32_t)(v >> 32) * 4294967296.0f + (float)(uint32_t)v;
}
__host__ __device__ __forceinline__ uint64_t isqrt64(uint64_t v) {
  const float f = sqrtf(u64_to_float(v));
  uint64_t y = f >= 4294967296.0f ? 0xffffffffull : (uint64_t)(uint32_t)f;
  if (y > 0) {
    const int64_t r = (int64_t)(v - y * y);  // |r| < 2^42
    const float rf = (float)(int32_t)(r >> 32) * 4294967296.0f + (float)(uint32_t)r;
    const int64_t z = (int64_t)y + (int32_t)(rf / (2.0f * (float)(uint32_t)y));  // step below 2^10
    y = z < 0 ? 0 : (z > 0xffffffffll ? 0xffffffffull : (uint64_t)z);
  }
  while (y > 0 && y * y > v) --y;
  while (y < 0xffffffffull && (y + 1) * (y + 1) <= v) ++y;
  return y;
}

// The top-32-bit values x whose range-map value lies in [ulo, uhi]: [xlo, xhi] (empty when
// xlo > xhi).  Canonical: umap(x) = 2^32 - 1 - floor(y^2 / 2^32) with y = 2^32 - 1 - x, so
// umap(x) >= ulo  <=>  y^2 < (2^32 - ulo) 2^32   and   umap(x) <= uhi  <=>  y^2 >= (2^32 - 1 - uhi) 2^32.
__host__ __device__ __forceinline__ void x_range(uint32_t ulo, uint32_t uhi, int canonical, uint32_t& xlo,
                                                 uint32_t& xhi) {
  if (!canonical) {
    xlo = ulo;
    xhi = uhi;
    return;
  }
  const uint64_t ymax = isqrt64(((uint64_t)(0x100000000ull - ulo) << 32) - 1);  // wraps to 2^64 - 1 for ulo = 0
  xlo = 0xffffffffu - (uint32_t)(ymax < 0xffffffffull ? ymax : 0xffffffffull);
  const uint64_t m = (uint64_t)(~uhi) << 32;
  const uint64_t ymin = m == 0 ? 0 : isqrt64(m - 1) + 1;  // ceil(sqrt(m))
  xhi = ymin > 0xffffffffull ? 0u : 0xffffffffu - (uint32_t)ymin;
  if (ymin > 0xffffffffull) xlo = 1;  // no x maps at or below uhi (only uhi = 0): empty
}

// Keys (2k bits) whose top 32 bits lie in [xlo, xhi].
__host__ __device__ __forceinline__ void key_range(uint32_t xlo, uint32_t xhi, int k, uint64_t& lo, uint64_t& hi) {
  lo = ((uint64_t)xlo << 32) >> (64 - 2 * k);
  hi = (((uint64_t)xhi << 32) | 0xffffffffull) >> (64 - 2 * k);
}
__host__ __device__ __forceinline__ void key_range(uint32_t xlo, uint32_t xhi, int k, u128& lo, u128& hi) {
  const int sh = 2 * k - 32;
  lo = (u128)xlo << sh;
  hi = ((u128)xhi << sh) | (((u128)1 << sh) - 1);
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
// Top 32 bits of (a:b) << sh, 0 <= sh < 64 (a compile-time constant once unrolled).
__device__ __forceinline__ uint32_t top32_shl(uint64_t a, uint64_t b, int sh) {
  return sh < 32 ? __funnelshift_l((uint32_t)a, (uint32_t)(a >> 32), sh)
                 : __funnelshift_l((uint32_t)(b >> 32), (uint32_t)a, sh - 32);
}
// Window i: the top 32 bits of its canonical value only (the range-map input), from 32-bit
// shifts.  The smaller of the forward and reverse-complement top words is the canonical
// value's top word: where the top words differ they decide which value is smaller, and
// where they tie both values share them.
template <int KW, int WPT>
__device__ __forceinline__ uint32_t win_top32(const Win& W, int i, int canonical) {
  const uint32_t m = (uint32_t)(W.m0 >> 32);
  const uint32_t f = top32_shl(W.s0, W.s1, 2 * i) & m;
  const uint32_t r = top32_shl(W.r0, W.r1, 2 * (WPT - 1 - i)) & m;
  return canonical ? min(f, r) : f;
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
__device__ __forceinline__ void pack_count_body(const Shape& s, const Buffers& b, uint32_t bid) {
  typedef typename KeyT<KW>::T K;
  extern __shared__ uint32_t hist_s[];  // [P1 + 32]: bins P1 + lane take the invalid windows
  __shared__ uint64_t code_s[kPackThreads + 2];
  __shared__ uint32_t inv_s[kPackThreads + 2];
  __shared__ uint32_t st_s[kPackThreads + 2];
  __shared__ uint64_t rcur_s, len_s;
  const int t = threadIdx.x;
  const int P1 = 1 << s.b1;
  const uint64_t tile = bid;
  for (int c = t; c < P1 + 32; c += kPackThreads) hist_s[c] = 0;
  if (t == 0) {
    rcur_s = b.tile_first[tile];
    // bases read: never past the end the offsets give (a base count that disagrees with
    // them is reported by k_check_offsets; the reads buffer is not overrun meanwhile)
    const uint64_t e = b.offsets[s.n_reads];
    len_s = e < s.L ? e : s.L;
  }
  __syncthreads();
  const uint64_t len = len_s;
  for (int sub = 0; sub < kTileWords / kPackThreads; ++sub) {
    const uint64_t j0 = tile * kTileWords + (uint64_t)sub * kPackThreads;
    if (j0 >= s.n_words) break;
    __syncthreads();
    if (t < 2) {
      if (sub > 0) {
        code_s[t] = code_s[kPackThreads + t];
        inv_s[t] = inv_s[kPackThreads + t];
      } else if (j0 + t >= 2) {
        convert_word(b.reads, len, j0 + t - 2, code_s[t], inv_s[t]);
      } else {
        code_s[t] = 0;
        inv_s[t] = ~0u;
      }
    }
    const uint64_t j = j0 + t;
    uint64_t code = 0;
    uint32_t inv = ~0u;
    if (j < s.n_words) {
      convert_word(b.reads, len, j, code, inv);
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
      for (int i = 0; i < 32; ++i) {  // an invalid window goes to bin P1 + lane, never read: no branch
        const uint32_t c = coarse_field(umap(win_top32<KW, 32>(W, i, s.canonical), s.canonical), s.b1);
        atomicAdd(&hist_s[((W.valid >> i) & 1u) ? c : (uint32_t)P1 + (t & 31)], 1u);
      }
    }
  }
  __syncthreads();
  for (int c = t; c < P1; c += kPackThreads) b.hist[tile * P1 + c] = hist_s[c];
}
template <int KW>
__global__ void __launch_bounds__(kPackThreads, KW == 1 ? 2 : 1) k_pack_count(Shape s, Buffers b) {
  pack_count_body<KW>(s, b, blockIdx.x);
}
template <int KW>
__global__ void __launch_bounds__(kPackThreads, KW == 1 ? 2 : 1) k_pack_count_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  pack_count_body<KW>(d.s, d.b, bid);
}

// ------------------------------------------------------------------ scans
// Column scan of hist[tile][c]: toff[tile][c] = keys of partition c in tiles before `tile`.
__device__ __forceinline__ void col_scan_body(const uint32_t* hist, uint64_t* toff, uint64_t* ccount, uint64_t n_tiles, int P1,
                                              uint32_t bid) {
  __shared__ uint64_t part[32][33];
  const int lane = threadIdx.x, w = threadIdx.y;
  const int c = bid * 32 + lane;
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
__global__ void k_col_scan(const uint32_t* hist, uint64_t* toff, uint64_t* ccount, uint64_t n_tiles, int P1) {
  col_scan_body(hist, toff, ccount, n_tiles, P1, blockIdx.x);
}
__global__ void k_col_scan_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  col_scan_body(d.b.hist, d.b.toff, d.b.cstart, d.s.n_tiles, 1 << d.s.b1, bid);
}

// Partition starts and the total number of windows.  One block.
__device__ __forceinline__ void bucket_scan_body(const uint64_t* ccount, uint64_t* cstart, int P1, Meta* meta) {
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
__global__ void k_bucket_scan(const uint64_t* ccount, uint64_t* cstart, int P1, Meta* meta) {
  bucket_scan_body(ccount, cstart, P1, meta);
}
__global__ void k_bucket_scan_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  bucket_scan_body(d.b.cstart, d.b.cstart, 1 << d.s.b1, d.b.meta);
}

// Fine split of every coarse partition, after pass B: the distinct-key estimate (a sampled
// HyperLogLog filled by pass B) gives the duplication factor K / D, and a fine partition
// aims at fine_target distinct keys, i.e. fine_target * K / D keys.  One block.
__device__ __forceinline__ void fine_plan_body(const uint64_t* cstart, const uint32_t* hll, uint32_t* fine_base, uint32_t* fine_m,
                            uint32_t* flo, int P1, int b1, uint32_t fine_target, uint32_t nf_max, Meta* meta) {
  extern __shared__ uint64_t fsc[];  // [P1]
  __shared__ uint64_t wt[32];
  __shared__ float zsum_s[32], zeros_s[32];
  __shared__ double target_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // HyperLogLog estimate over the 1/64 hash-sample of the keys
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
    target_s = (double)fine_target * (0.9 * dup > 1.0 ? 0.9 * dup : 1.0);
    meta->d_estimate = (uint64_t)d_est;
  }
  __syncthreads();
  const double target = target_s;
  for (int c = threadIdx.x; c < P1; c += blockDim.x) {
    const uint64_t n = cstart[c + 1] - cstart[c];
    uint64_t m = (uint64_t)ceil((double)n / target);
    m = m < 1 ? 1 : (m > (uint64_t)kMaxFine ? (uint64_t)kMaxFine : m);
    fine_m[c] = (uint32_t)m;
    fsc[c] = m;
  }
  __syncthreads();
  const uint64_t NF = block_exclusive_scan<uint64_t>(fsc, P1, wt);
  for (int c = threadIdx.x; c < P1; c += blockDim.x) fine_base[c] = (uint32_t)fsc[c];
  // fine partition g = fsc[c] + f holds the values u of coarse field c whose low part
  // v = u mod 2^(32 - b1) has floor(v m / 2^(32 - b1)) = f, i.e. v >= ceil(f 2^(32 - b1) / m);
  // one thread per fine partition, its coarse partition found by binary search in fsc
  const uint64_t w = 1ull << (32 - b1);
  for (uint64_t g = threadIdx.x; g < NF && g < nf_max; g += blockDim.x) {
    int lo = 0, hi = P1 - 1;  // last c with fsc[c] <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (fsc[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    const uint64_t m = fine_m[lo], f = g - fsc[lo];
    flo[g] = (uint32_t)((uint64_t)lo << (32 - b1)) + (uint32_t)((f * w + m - 1) / m);
  }
  if (threadIdx.x == 0) {
    if (NF <= nf_max) flo[NF] = 0;  // so that the last partition ends at u = 2^32 - 1
    fine_base[P1] = (uint32_t)NF;
    meta->n_fine = NF <= nf_max ? NF : 0;  // later kernels never index past nf_max
    if (NF > nf_max) atomicOr(&meta->status, ST_INTERNAL);
  }
}
__global__ void k_fine_plan(const uint64_t* cstart, const uint32_t* hll, uint32_t* fine_base, uint32_t* fine_m,
                            uint32_t* flo, int P1, int b1, uint32_t fine_target, uint32_t nf_max, Meta* meta) {
  fine_plan_body(cstart, hll, fine_base, fine_m, flo, P1, b1, fine_target, nf_max, meta);
}
__global__ void k_fine_plan_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  fine_plan_body(d.b.cstart, d.b.hll, d.b.fine_base, d.b.fine_m, d.b.flo, 1 << d.s.b1, d.s.b1, d.s.fine_target,
                 (uint32_t)d.s.nf_max, d.b.meta);
}

// ------------------------------------------------------------------ pass B
// Per sub-step, NT threads x WPT windows: every key is computed once and kept in registers,
// its rank inside its partition taken with a shared-memory atomic (counting sort, step 1);
// after the block scan of the partition histogram the keys go to their partition's run in
// the staging buffer, and the runs leave in order.  A 1/64 hash sample of the keys feeds a
// HyperLogLog sketch (distinct-key estimate for sizing the fine partitions).
__device__ __forceinline__ uint64_t key_hash(uint64_t key) { return key * 0x9E3779B97F4A7C15ull; }
__device__ __forceinline__ uint64_t key_hash(u128 key) {
  return ((uint64_t)key ^ ((uint64_t)(key >> 64) * 0xC2B2AE3D27D4EB4Full)) * 0x9E3779B97F4A7C15ull;
}

// KEEP_C: each window's coarse partition is kept in shared memory (taken in phase 1,
// carried to the staging and the write-out) instead of being recomputed from the key
// twice; used when two blocks per SM still fit.
// DIRECT (the aggregation ablation without per-block buckets): every valid window takes its
// slot with a global atomic on its partition's cursor and is written on its own.
template <int KW, int NT, bool KEEP_C, bool DIRECT = false>
__device__ __forceinline__ void scatter_body(const Shape& s, const Buffers& b, uint32_t bid) {
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
  uint32_t* soff = hist + padded_len(P1 + 32);                                          // [padded P1]
  uint16_t* rawc = reinterpret_cast<uint16_t*>(soff + padded_len(P1 + 32));  // KEEP_C: [SUB], window i of thread t at i * NT + t
  uint16_t* stage_c = rawc + SUB;                                        // KEEP_C: [SUB], partition of each staged key
  __shared__ uint64_t code_s[NW + 2];
  __shared__ uint32_t inv_s[NW + 2];
  __shared__ uint32_t st_s[NW + 2];
  __shared__ uint32_t hll_s[kHllRegs];
  __shared__ uint64_t rcur_s;
  __shared__ uint32_t wt[32];
  const int t = threadIdx.x;
  const int wl = t / TPW, h = t % TPW;  // code word of the thread within the sub-step, half
  const uint64_t tile = bid;
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
      // every window is computed and ranked without a branch (so that the windows' dependency
      // chains interleave): an invalid window is ranked in bin P1 + lane, which no scan reads
      // (one such bin per lane, so that a warp's invalid windows do not share an address), and
      // only the rare sketch update depends on the window being valid
#pragma unroll
      for (int i = 0; i < WPT; ++i) {
        uint64_t c0, c1;
        win_top<KW, WPT>(W, i, s.canonical, c0, c1);
        top_to_key(c0, c1, s.k, keys[i]);
        const uint32_t c = coarse_field(umap((uint32_t)(c0 >> 32), s.canonical), s.b1);
        const uint64_t hh = key_hash(keys[i]);
        const bool v = (valid >> i) & 1u;
        if constexpr (DIRECT) {
          if (v) {
            const unsigned long long pos = atomicAdd(&b.fcur[c], 1ull);
            if (pos < s.cap) store_key(b.kbuf, pos, keys[i]);
            else atomicOr(&b.meta->status, ST_INTERNAL);
          }
        } else {
          if constexpr (KEEP_C) rawc[i * NT + t] = (uint16_t)c;
          const uint32_t cc = v ? c : (uint32_t)P1 + (t & 31);
          rr[i >> 1] |= (atomicAdd(&hist[PAD(cc)], 1u) & 0xffffu) << (16 * (i & 1));
        }
        if (v && (hh >> (64 - kHllSampleLog2)) == 0) {
          const uint32_t reg = (uint32_t)(hh >> (64 - kHllSampleLog2 - kHllLog2)) & (kHllRegs - 1);
          const uint64_t rest = hh << (kHllSampleLog2 + kHllLog2);
          atomicMax(&hll_s[reg], (uint32_t)min(__clzll(rest) + 1, 64 - kHllSampleLog2 - kHllLog2 + 1));
        }
      }
    }
    if constexpr (DIRECT) continue;
    __syncthreads();
    for (int c = t; c < P1; c += NT) soff[PAD(c)] = hist[PAD(c)];
    __syncthreads();
    block_exclusive_scan_pad<uint32_t>(soff, P1, wt);
#pragma unroll
    for (int i = 0; i < WPT; ++i) {
      // an invalid window is staged at slot SUB - 1, which no valid window takes then (with
      // one window invalid, at most SUB - 1 are valid) and the write-out never reads
      uint32_t c;
      if constexpr (KEEP_C) c = rawc[i * NT + t];
      else c = coarse_of(keys[i], s.k, s.canonical, s.b1);  // same field as above, from the key
      const uint32_t pos = (valid & (1u << i)) ? soff[PAD(c)] + ((rr[i >> 1] >> (16 * (i & 1))) & 0xffffu)
                                               : (uint32_t)(SUB - 1);
      stage[pos] = keys[i];
      if constexpr (KEEP_C) stage_c[pos] = (uint16_t)c;
    }
    __syncthreads();
    const uint32_t n_sub = soff[PAD(P1 - 1)] + hist[PAD(P1 - 1)];
    // during the write-out cursor[c] holds cursor[c] - soff[c]: staged position i of
    // partition c goes to cursor[c] + i
    for (int c = t; c < P1; c += NT) cursor[c] -= soff[PAD(c)];
    __syncthreads();
    for (uint32_t i = t; i < n_sub; i += NT) {
      const K key = stage[i];
      uint32_t c;
      if constexpr (KEEP_C) c = stage_c[i];
      else c = coarse_of(key, s.k, s.canonical, s.b1);  // runs are grouped by partition
      const uint64_t pos = cursor[c] + i;
      if (pos < s.cap) store_key(b.kbuf, pos, key);
      else atomicOr(&b.meta->status, ST_INTERNAL);
    }
    __syncthreads();
    for (int c = t; c < P1; c += NT) {
      cursor[c] += soff[PAD(c)] + hist[PAD(c)];
      hist[PAD(c)] = 0;
    }
  }
  __syncthreads();
  for (int i = t; i < kHllRegs; i += NT)
    if (hll_s[i]) atomicMax(&b.hll[i], hll_s[i]);
}
template <int KW, int NT, bool KEEP_C>
__global__ void __launch_bounds__(NT, 2) k_scatter(Shape s, Buffers b) {
  scatter_body<KW, NT, KEEP_C>(s, b, blockIdx.x);
}
// Aggregation ablation: the partition cursors start at the partition starts, and pass B
// writes every key on its own through them.
__global__ void k_direct_cursors(const uint64_t* cstart, unsigned long long* cur, int P1) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < P1; c += gridDim.x * blockDim.x) cur[c] = cstart[c];
}
template <int KW>
__global__ void __launch_bounds__(256, 2) k_scatter_direct(Shape s, Buffers b) {
  scatter_body<KW, 256, false, true>(s, b, blockIdx.x);
}

template <int KW, int NT, bool KEEP_C>
__global__ void __launch_bounds__(NT, 2) k_scatter_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  scatter_body<KW, NT, KEEP_C>(d.s, d.b, bid);
}

// ------------------------------------------------------------------ phase 2: fine split
// Fine partition of a key: the coarse field c of u selects {first fine partition of c,
// m_c}; the fine index is floor(v m_c / 2^(32 - b1)) for the low part v of u (below the
// coarse field), taken as the high word of (v << b1) * m_c.  The m_c fine partitions of c
// split its range of u into near-equal parts.
struct FineMap {
  int k, canonical, b1;
};

template <class K>
__device__ __forceinline__ uint32_t fine_of(K key, const FineMap& x, const uint2* fmap) {
  const uint32_t u = umap(top32_of(key, x.k), x.canonical);
  const uint2 e = fmap[coarse_field(u, x.b1)];
  return e.x + __umulhi(u << x.b1, e.y);
}

// fmap[c] = {fine_base[c], fine_m[c]} for c < P1, fmap[P1].x = fine partition count.
__device__ __forceinline__ void load_fine_map(const Buffers& b, int P1, uint2* fmap) {
  for (int c = threadIdx.x; c <= P1; c += blockDim.x) fmap[c] = make_uint2(b.fine_base[c], c < P1 ? b.fine_m[c] : 0u);
}
__host__ __device__ inline FineMap make_fine_map(const Shape& s) { return FineMap{s.k, s.canonical, s.b1}; }

constexpr int kFineThreads = 512;
constexpr int kFinePer = 8;  // keys per thread per chunk (loaded as 16-byte pairs / single u128, all before use)
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

// Chunks of the coarse-grouped keys are handed out round-robin.  A chunk's first and last
// keys bound the fine partitions it touches; they are fetched for the block's next chunk
// (cp.async into bnd_s[1 - cur]) while the current one is processed.
template <int KW>
__device__ __forceinline__ void fetch_bounds(const uint64_t* kbuf, uint64_t c0, uint64_t K_total,
                                             typename KeyT<KW>::T* bnd) {
  const uint64_t c1 = min(K_total, c0 + kFineChunk);
  if constexpr (KW == 1) {
    cp_async8(&bnd[0], kbuf + c0);
    cp_async8(&bnd[1], kbuf + c1 - 1);
  } else {
    cp_async16(&bnd[0], kbuf + 2 * c0);
    cp_async16(&bnd[1], kbuf + 2 * (c1 - 1));
  }
}

template <int KW>
__device__ __forceinline__ void fine_hist_body(const Shape& s, const Buffers& b, uint32_t bid, uint32_t nblk,
                                               bool redo = false) {
  typedef typename KeyT<KW>::T K;
  extern __shared__ __align__(16) uint8_t sm[];
  if (redo && !b.meta->fine_spill) return;  // the exact fine split runs again only after a spill
  // a sampled layout counts one chunk in 2^kFineSampleLog2 (the exact split: every chunk)
  const uint64_t cstep = (s.fine_sampled && !redo) ? ((uint64_t)kFineChunk << kFineSampleLog2) : (uint64_t)kFineChunk;
  const int P1 = 1 << s.b1;
  uint2* fmap = reinterpret_cast<uint2*>(sm);                    // [P1 + 1]
  uint32_t* lh = reinterpret_cast<uint32_t*>(fmap + P1 + 1);     // [kFineLocalCap]
  __shared__ __align__(16) K bnd_s[2][2];
  load_fine_map(b, P1, fmap);
  for (int i = threadIdx.x; i < kFineLocalCap; i += kFineThreads) lh[i] = 0;
  const FineMap x = make_fine_map(s);
  const uint64_t K_total = min(b.meta->n_windows, s.cap);
  const uint64_t stride = (uint64_t)nblk * cstep;
  if (threadIdx.x == 0 && bid * cstep < K_total) {
    fetch_bounds<KW>(b.kbuf, bid * cstep, K_total, bnd_s[0]);
    cp_async_wait_all();
  }
  __syncthreads();
  int cur = 0;
  for (uint64_t c0 = bid * cstep; c0 < K_total; c0 += stride, cur ^= 1) {
    const uint64_t c1 = min(K_total, c0 + kFineChunk);
    const uint32_t g_lo = fmap[coarse_of(bnd_s[cur][0], s.k, s.canonical, s.b1)].x;
    const uint32_t span = fmap[coarse_of(bnd_s[cur][1], s.k, s.canonical, s.b1) + 1].x - g_lo;
    if (threadIdx.x == 0 && c0 + stride < K_total) fetch_bounds<KW>(b.kbuf, c0 + stride, K_total, bnd_s[cur ^ 1]);
    const bool local = span <= (uint32_t)kFineLocalCap;
    K keys[kFinePer];
    uint32_t have;
    load_chunk<KW>(b.kbuf, c0, c1, keys, have);
#pragma unroll
    for (int m = 0; m < kFinePer; ++m) {
      if ((have >> m) & 1u) {
        const uint32_t g = fine_of(keys[m], x, fmap);
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
    if (threadIdx.x == 0) cp_async_wait_all();
    __syncthreads();
  }
}
template <int KW>
__global__ void __launch_bounds__(kFineThreads, 2) k_fine_hist(Shape s, Buffers b, int redo) {
  fine_hist_body<KW>(s, b, blockIdx.x, gridDim.x, redo != 0);
}
template <int KW>
__global__ void __launch_bounds__(kFineThreads, 2) k_fine_hist_batch(BatchTab t, int redo) {
  KC_BATCH_PROLOGUE(t);
  fine_hist_body<KW>(d.s, d.b, bid, nblk, redo != 0);
}

// Keys at positions below x of the keys array that a sampled fine histogram counts: one
// kFineChunk-key chunk in 2^kFineSampleLog2.
__device__ __forceinline__ uint64_t sampled_below(uint64_t x) {
  const uint64_t per = (uint64_t)kFineChunk << kFineSampleLog2;
  const uint64_t r = x % per;
  return (x / per) * kFineChunk + (r < (uint64_t)kFineChunk ? r : (uint64_t)kFineChunk);
}

// Region of fine partition g in a sampled layout: its estimated size (its sampled count
// scaled by its coarse partition's keys over that partition's sampled keys) plus 5.5
// standard deviations of that estimate and 16 keys; never more than its coarse partition.
// Too small a sample gives the whole coarse partition.
__device__ __forceinline__ uint64_t fine_region(const Shape& sh, const Buffers& b, uint64_t g) {
  const uint32_t c = sh.b1 ? b.flo[g] >> (32 - sh.b1) : 0u;
  const uint64_t a = b.cstart[c], e = b.cstart[c + 1];
  const uint64_t n_c = e - a, s_c = sampled_below(e) - sampled_below(a);
  if (s_c < 1024) return n_c;
  const float f = (float)n_c / (float)s_c, cnt = (float)b.fhist[g];
  const float slack = sh.tight_slack ? 0.f : 5.5f * f * sqrtf(cnt + 1.f) + 16.f;
  const uint64_t r = (uint64_t)(cnt * f + slack) + (sh.tight_slack ? 0 : 1);
  return r < n_c ? r : n_c;
}

// Exclusive scan of the fine partitions' sizes (exact histogram) or regions (sampled
// layout) into their starts (one block of 1024 threads).  A sampled layout that does not fit
// the keys arrays is given up at once (the exact split follows).
__device__ __forceinline__ void fine_scan_body(const Shape& sh, const Buffers& b, bool redo = false) {
  __shared__ uint64_t wt[32];
  __shared__ uint64_t carry_s;
  if (redo && !b.meta->fine_spill) return;
  const bool sampled = sh.fine_sampled && !redo;
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
      v[m] = i < NF ? (sampled ? fine_region(sh, b, i) : (uint64_t)b.fhist[i]) : 0;
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
  if (t == 0) {
    b.foff[NF] = carry_s;
    if (sampled && carry_s > sh.cap_kb) b.meta->fine_spill = 1;
  }
}
__global__ void k_fine_scan(Shape sh, Buffers b, int redo) { fine_scan_body(sh, b, redo != 0); }

// Before the exact fine split runs again (a sampled region overflowed): a fresh histogram.
__global__ void k_fine_redo_clear(Shape sh, Buffers b) {
  if (!b.meta->fine_spill) return;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < sh.nf_max; i += (uint64_t)gridDim.x * blockDim.x)
    b.fhist[i] = 0;
}
__global__ void k_fine_scan_batch(BatchTab t, int redo) {
  KC_BATCH_PROLOGUE(t);
  fine_scan_body(d.s, d.b, redo != 0);
}
// (the fine scan's table: one block per count)
__global__ void k_fine_redo_clear_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  if (!d.b.meta->fine_spill) return;
  for (uint64_t i = threadIdx.x; i < d.s.nf_max; i += blockDim.x) d.b.fhist[i] = 0;
}

// Exclusive scan of in[0, n) into out[0, n) (all threads of the block, n <= 4 * blockDim);
// returns the total.
__device__ uint32_t block_scan_to(const uint32_t* in, uint32_t* out, int n, uint32_t* warp_tmp) {
  const int nt = blockDim.x, t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = (nt + 31) >> 5;
  const int per = (n + nt - 1) / nt;
  const int lo = min(n, t * per), hi = min(n, lo + per);
  uint32_t s = 0;
  for (int i = lo; i < hi; ++i) s += in[i];
  uint32_t x = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tmp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < nw ? warp_tmp[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < nw) warp_tmp[lane] = w;
  }
  __syncthreads();
  uint32_t run = x - s + (wid ? warp_tmp[wid - 1] : 0);
  const uint32_t total = warp_tmp[nw - 1];
  for (int i = lo; i < hi; ++i) {
    out[i] = run;
    run += in[i];
  }
  __syncthreads();
  return total;
}

// Split each chunk by fine partition: rank the keys in a shared histogram, bump each fine
// partition's global cursor once per chunk, stage the keys grouped by fine partition and
// write every group as one contiguous run.
template <int KW>
__device__ __forceinline__ void fine_scatter_body(const Shape& s, const Buffers& b, uint32_t bid, uint32_t nblk,
                                                  bool redo = false) {
  typedef typename KeyT<KW>::T K;
  extern __shared__ __align__(16) uint8_t sm[];
  // the exact split runs again only after a spill; a sampled layout given up by the scan is
  // not written at all.  In a sampled layout a run that would pass its region's end is not
  // written: the spill is recorded and the exact split follows.
  if (redo ? !b.meta->fine_spill : (s.fine_sampled && b.meta->fine_spill)) return;
  const bool sampled = s.fine_sampled && !redo;
  constexpr uint64_t kSpilledRun = 1ull << 63;  // never a run's offset
  const int P1 = 1 << s.b1;
  K* stage = reinterpret_cast<K*>(sm);                                          // [kFineChunk]
  uint16_t* stage_g = reinterpret_cast<uint16_t*>(stage + kFineChunk);          // [kFineChunk]
  uint64_t* delta = reinterpret_cast<uint64_t*>(stage_g + kFineChunk);          // [kFineLocalCap]
  uint32_t* lh = reinterpret_cast<uint32_t*>(delta + kFineLocalCap);            // [kFineLocalCap]
  uint32_t* soff = lh + kFineLocalCap;                                          // [kFineLocalCap]
  uint2* fmap = reinterpret_cast<uint2*>(soff + kFineLocalCap);                 // [P1 + 1]
  __shared__ __align__(16) K bnd_s[2][2];
  __shared__ uint32_t wt[32];
  load_fine_map(b, P1, fmap);
  for (int i = threadIdx.x; i < kFineLocalCap; i += kFineThreads) lh[i] = 0;
  const FineMap x = make_fine_map(s);
  const uint64_t K_total = min(b.meta->n_windows, s.cap);
  const uint64_t stride = (uint64_t)nblk * kFineChunk;
  if (threadIdx.x == 0 && bid * (uint64_t)kFineChunk < K_total) {
    fetch_bounds<KW>(b.kbuf, bid * (uint64_t)kFineChunk, K_total, bnd_s[0]);
    cp_async_wait_all();
  }
  __syncthreads();
  int cur = 0;
  for (uint64_t c0 = bid * (uint64_t)kFineChunk; c0 < K_total; c0 += stride, cur ^= 1) {
    const uint64_t c1 = min(K_total, c0 + kFineChunk);
    const uint32_t g_lo = fmap[coarse_of(bnd_s[cur][0], s.k, s.canonical, s.b1)].x;
    const uint32_t span = fmap[coarse_of(bnd_s[cur][1], s.k, s.canonical, s.b1) + 1].x - g_lo;
    if (threadIdx.x == 0 && c0 + stride < K_total) fetch_bounds<KW>(b.kbuf, c0 + stride, K_total, bnd_s[cur ^ 1]);
    if (span == 0 || span > (uint32_t)kFineLocalCap) {
      // a chunk over very many tiny fine partitions: one global cursor bump per key
      for (int m = 0; m < kFinePer; ++m) {
        const uint64_t i = c0 + threadIdx.x + (uint64_t)m * kFineThreads;
        if (i < c1) {
          K key;
          load_key(b.kbuf, i, key);
          const uint32_t g = fine_of(key, x, fmap);
          const uint64_t pos = g < s.nf_max ? atomicAdd(&b.fcur[g], 1ull) : ~0ull;
          if (sampled && g < s.nf_max && pos >= b.foff[g + 1]) b.meta->fine_spill = 1;
          else if (pos < s.cap_kb) store_key(b.sbuf, pos, key);
          else atomicOr(&b.meta->status, ST_INTERNAL);
        }
      }
    } else {
      K keys[kFinePer];
      uint32_t gr[kFinePer];
      uint32_t have;
      load_chunk<KW>(b.kbuf, c0, c1, keys, have);
#pragma unroll
      for (int m = 0; m < kFinePer; ++m) {
        gr[m] = 0xffffffffu;
        if ((have >> m) & 1u) {
          const uint32_t lg = fine_of(keys[m], x, fmap) - g_lo;
          if (lg < span) gr[m] = (lg << 16) | atomicAdd(&lh[lg], 1u);  // span <= 2^10, rank < 2^16
          else atomicOr(&b.meta->status, ST_INTERNAL);
        }
      }
      __syncthreads();
      const uint32_t n_staged = block_scan_to(lh, soff, (int)span, wt);
      // one cursor bump per fine partition; delta[lg] + staged position = global position
      for (uint32_t i = threadIdx.x; i < span; i += kFineThreads) {
        const uint32_t v = lh[i];
        if (v) {
          uint64_t gb = s.cap_kb;  // positions at or past cap_kb are rejected below
          if (g_lo + i < s.nf_max) {
            const uint64_t lim = sampled ? b.foff[g_lo + i + 1] : ~0ull;  // loaded before the bump
            gb = atomicAdd(&b.fcur[g_lo + i], (unsigned long long)v);
            if (gb + v > lim) {  // the run passes its region's end
              b.meta->fine_spill = 1;
              gb = kSpilledRun;
            }
          } else {
            atomicOr(&b.meta->status, ST_INTERNAL);
          }
          delta[i] = gb == kSpilledRun ? kSpilledRun : gb - soff[i];
          lh[i] = 0;
        }
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
      for (uint32_t i = threadIdx.x; i < n_staged; i += kFineThreads) {
        const uint64_t dl = delta[stage_g[i]];
        if (dl == kSpilledRun) continue;
        const uint64_t pos = dl + i;
        if (pos < s.cap_kb) store_key(b.sbuf, pos, stage[i]);
        else atomicOr(&b.meta->status, ST_INTERNAL);
      }
    }
    if (threadIdx.x == 0) cp_async_wait_all();
    __syncthreads();
  }
}
template <int KW>
__global__ void __launch_bounds__(kFineThreads, 2) k_fine_scatter(Shape s, Buffers b, int redo) {
  fine_scatter_body<KW>(s, b, blockIdx.x, gridDim.x, redo != 0);
}
template <int KW>
__global__ void __launch_bounds__(kFineThreads, 2) k_fine_scatter_batch(BatchTab t, int redo) {
  KC_BATCH_PROLOGUE(t);
  fine_scatter_body<KW>(d.s, d.b, bid, nblk, redo != 0);
}

// ------------------------------------------------------------------ phase 2: count + emit
constexpr uint64_t kLookValue = (1ull << 62) - 1;
constexpr uint64_t kLookAgg = 1ull << 62;
constexpr uint64_t kLookIncl = 2ull << 62;

// Decoupled look-back (executed by one warp): sum of distinct counts of fine partitions < g.
// Each step reads the kLookPer * 32 status words before position j at once (lane l holds
// distance q * 32 + l); the nearest inclusive prefix among them ends the walk, and only
// unpublished words nearer than it are waited for (with a bounded spin).  With `abort`,
// the wait also ends as soon as *abort becomes nonzero, and kNoPrefix is returned.
constexpr int kLookPer = 8;
constexpr uint64_t kNoPrefix = ~0ull;
__device__ uint64_t lookback(unsigned long long* look, uint64_t g, uint32_t* status, uint32_t spin_limit,
                             const volatile uint32_t* abort = nullptr) {
  const int lane = threadIdx.x & 31;
  constexpr uint32_t kNone = kLookPer * 32;
  uint64_t excl = 0;
  int64_t j = (int64_t)g - 1;
  while (j >= 0) {
    uint64_t v[kLookPer];
#pragma unroll
    for (int q = 0; q < kLookPer; ++q) {
      const int64_t idx = j - (q * 32 + lane);
      v[q] = idx >= 0 ? ld_status(&look[idx]) : kLookIncl;  // before the first partition: inclusive 0
    }
    uint32_t stop = kNone, spins = 0;
    while (true) {
      stop = kNone;  // nearest inclusive distance
#pragma unroll
      for (int q = kLookPer - 1; q >= 0; --q) {
        const unsigned b = __ballot_sync(0xffffffffu, (v[q] >> 62) == 2);
        if (b) stop = q * 32 + __ffs(b) - 1;
      }
      bool wait = false;
#pragma unroll
      for (int q = 0; q < kLookPer; ++q) wait |= (uint32_t)(q * 32 + lane) < stop && (v[q] >> 62) == 0;
      if (!__any_sync(0xffffffffu, wait)) break;
      if (abort && *abort) return kNoPrefix;
      if (++spins > spin_limit) {
        if (lane == 0) atomicOr(status, ST_TIMEOUT);
        return excl;
      }
      __nanosleep(64);
#pragma unroll
      for (int q = 0; q < kLookPer; ++q) {
        const int64_t idx = j - (q * 32 + lane);
        if ((uint32_t)(q * 32 + lane) < stop && (v[q] >> 62) == 0) v[q] = ld_status(&look[idx]);
      }
    }
    uint64_t val = 0;
#pragma unroll
    for (int q = 0; q < kLookPer; ++q)
      if ((uint32_t)(q * 32 + lane) <= stop) val += v[q] & kLookValue;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) val += __shfl_xor_sync(0xffffffffu, val, d);
    excl += val;
    if (stop != kNone) break;
    j -= kNone;
  }
  return excl;
}

template <int KW>
struct Table {
  typedef typename KeyT<KW>::T K;
  K* keys;
  uint32_t* counts;
};

// Count kernel shared memory: a hash table of 2^bT_max slots (key + count), a bucket
// histogram of hist_max(kw) entries and the 16-bit slot numbers of up to 3/4 of the slots
// in output order.
constexpr int kTableLog2Cap = kCountThreads == 1024 ? 13 : 12;  // 8 slots per thread
__host__ __device__ constexpr int hist_max(int kw) {
  return kCountThreads == 1024 ? (kw == 1 ? 16384 : 8192) : 4096;
}

size_t count_kernel_smem(int kw, int bT_max, int /*unused*/) {
  const size_t slots = (size_t)1 << bT_max;
  return slots * (size_t)(kw * 8 + 4) + padded_len(hist_max(kw)) * 4 + ((3 * slots) >> 2) * 2 + 256;
}

// The largest table whose block (8 KB of static shared memory included) fits the opt-in
// limit, with kCountBlocksPerSM blocks on one SM (each also keeps 1 KB for the system).
int table_log2_max(int kw, size_t smem_optin, size_t smem_per_sm) {
  size_t budget = smem_optin;
  if (kCountBlocksPerSM > 1 && smem_per_sm) {
    const size_t per = smem_per_sm / kCountBlocksPerSM - 1024;
    budget = per < budget ? per : budget;
  }
  int best = 6;
  for (int bt = 6; bt <= kTableLog2Cap; ++bt)
    if (count_kernel_smem(kw, bt, 0) + 8192 <= budget) best = bt;
  return best;
}

constexpr int kProbeLimit = 128;
constexpr int kWorkers = kCountThreads - 32;  // warps 1.. load and sort while warp 0 looks back
constexpr int kSlotsPerWorker = ((1 << kTableLog2Cap) + kWorkers - 1) / kWorkers;

// counting-table slot of a key: a multiplicative hash (spreads keys that share prefixes)
__device__ __forceinline__ uint32_t hslot(uint64_t key, int bT) {
  return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - bT));
}
__device__ __forceinline__ uint32_t hslot(u128 key, int bT) {
  const uint64_t h = ((uint64_t)key ^ ((uint64_t)(key >> 64) * 0xC2B2AE3D27D4EB4Full)) * 0x9E3779B97F4A7C15ull;
  return (uint32_t)(h >> (64 - bT));
}

// Block barrier with the warp reconverged first: the count kernel reaches its barriers
// straight after branches taken by one thread or lane (ticket fetch, look-back bookkeeping).
__device__ __forceinline__ void block_sync() {
  __syncwarp();
  __syncthreads();
}

// Named barrier of the worker warps (1..31).  Its non-aligned form is used: a worker warp
// may arrive diverged (right after a branch taken by one of its threads, e.g. thread 32
// computing the key range), which the aligned form (bar.sync) does not allow.
__device__ __forceinline__ void bar_workers() {
  __syncwarp();
  asm volatile("barrier.sync 1, %0;" ::"r"(kWorkers) : "memory");
}

// Add `inc` to the count of `key` (claiming a slot if new).  Returns 2 if the key claimed a
// new slot, 1 if it was already there, 0 if no slot was found within the probe limit.
template <int KW>
__device__ __forceinline__ int count_insert(Table<KW> tb, typename KeyT<KW>::T key, uint32_t inc, int bT, bool check,
                                            uint32_t limit, uint32_t* status) {
  typedef typename KeyT<KW>::T K;
  const K EMPTY = all_ones<K>();
  const uint32_t mask = (1u << bT) - 1;
  uint32_t s = hslot(key, bT);
  for (int probe = 0; probe < kProbeLimit; ++probe, s = (s + 1) & mask) {
    int res = 0;
    if constexpr (KW == 1) {
      // read the slot; claim it only if empty (the claim's answer then replaces the read):
      // one exit test per probe instead of a branch per case
      uint64_t* p = reinterpret_cast<uint64_t*>(tb.keys) + s;
      unsigned long long old = *reinterpret_cast<volatile uint64_t*>(p);
      const bool emp = old == ~0ull;
      if (emp) old = atomicCAS(reinterpret_cast<unsigned long long*>(p), ~0ull, (unsigned long long)key);
      res = (emp && old == ~0ull) ? 2 : (old == (unsigned long long)key ? 1 : 0);
    } else {
      const K old = cas128_shared(reinterpret_cast<u128*>(tb.keys) + s, (u128)EMPTY, (u128)key);
      res = old == EMPTY ? 2 : (old == key ? 1 : 0);
    }
    if (res) {
      if (check) {
        const uint32_t o = atomicAdd(&tb.counts[s], inc);
        if (o > limit - inc) atomicOr(status, ST_COUNT_OVERFLOW);
      } else {
        atomicAdd(&tb.counts[s], inc);  // result unused: a reduction
      }
      return res;
    }
  }
  return 0;
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
// counted apart in *special (it marks empty slots); it exists only when the k-mer fills
// the key word (full_width).  Sets *ovf if a key found no slot.
// With MERGE, a warp whose active keys are all equal adds them with one atomic (the
// heavy-hitter merge of the paper's L3 layer); without it (the default) every key is added
// on its own: on GB300 the shared-memory atomics absorb equal keys faster than the merge's
// warp vote costs, even for a single key.
template <int KW, bool MERGE = false>
__device__ void count_all(Table<KW> tb, const uint64_t* in, uint64_t n, bool ranged, typename KeyT<KW>::T lo,
                          typename KeyT<KW>::T hi, int bT, bool full_width, uint32_t limit, uint32_t* n_new,
                          uint32_t* ovf, uint32_t* special, uint32_t* status) {
  typedef typename KeyT<KW>::T K;
  constexpr int kIn = KW == 1 ? 8 : 2;  // loads in flight per thread (u128 keys: register-bound at 64)
  const K EMPTY = all_ones<K>();
  const int lane = threadIdx.x & 31;
  const bool check = n > limit;  // a count can pass the limit only in a partition that large
  uint32_t claimed = 0;
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
      // a warp whose active keys all equal lane 0's key (a heavy hitter) adds them at once;
      // lane 0's own key counts only if it is active, so any inactive lane 0 is harmless
      const K k0 = shfl_key(key, 0);
      if (MERGE && __all_sync(0xffffffffu, !act || key == k0)) {
        const unsigned am = __ballot_sync(0xffffffffu, act);
        if (am && lane == __ffs(am) - 1) {
          const uint32_t inc = __popc(am);
          if (full_width && k0 == EMPTY) {
            if (atomicAdd(special, inc) > limit - inc) atomicOr(status, ST_COUNT_OVERFLOW);
          } else {
            const int r = count_insert<KW>(tb, k0, inc, bT, check, limit, status);
            if (!r) atomicOr(ovf, 1u);
            claimed += r == 2;
          }
        }
      } else if (act) {
        if (full_width && key == EMPTY) {
          if (atomicAdd(special, 1u) >= limit) atomicOr(status, ST_COUNT_OVERFLOW);
        } else {
          const int r = count_insert<KW>(tb, key, 1u, bT, check, limit, status);
          if (!r) atomicOr(ovf, 1u);
          claimed += r == 2;
        }
      }
    }
  }
  // the slots claimed, added once per warp (a shared counter bumped per new key would be
  // one address hit by every lane of a warp whose keys are all new)
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) claimed += __shfl_xor_sync(0xffffffffu, claimed, d);
  if (lane == 0 && claimed) atomicAdd(n_new, claimed);
}

template <class K> __device__ __forceinline__ int bitlen(K v);
template <> __device__ __forceinline__ int bitlen(uint64_t v) { return 64 - __clzll(v); }
template <> __device__ __forceinline__ int bitlen(u128 v) {
  const uint64_t hi = (uint64_t)(v >> 64);
  return hi ? 128 - __clzll(hi) : 64 - __clzll((uint64_t)v);
}

// Block-wide min of mn and max of mx (all threads; the result is returned to all).
template <class K>
__device__ void block_range(K mn, K mx, K* red_lo, K* red_hi, K& lo, K& hi) {
  const K EMPTY = ~(K)0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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

// Sort idx[a, a+c) by the keys the slots hold, by one warp: a bitonic network whose
// comparators all put the smaller key first, so positions past c act as +infinity.
template <class K>
__device__ void warp_sort_idx(const K* keys, uint16_t* idx, uint32_t a, uint32_t c) {
  const int lane = threadIdx.x & 31;
  uint32_t M = 1;
  while (M < c) M <<= 1;
  for (uint32_t size = 2; size <= M; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = lane; i < M; i += 32) {
        const uint32_t j = (stride == (size >> 1)) ? (i ^ (size - 1)) : (i ^ stride);
        if (j > i && j < c) {
          const uint16_t x = idx[a + i], y = idx[a + j];
          if (keys[y] < keys[x]) {
            idx[a + i] = y;
            idx[a + j] = x;
          }
        }
      }
      __syncwarp();
    }
  }
}

// positions per worker thread: 7 * 992 >= 3/4 of 8192 slots, 7 * 480 >= 3/4 of 4096
constexpr int kRankPer = ((3 << kTableLog2Cap) / 4 + kWorkers - 1) / kWorkers;
static_assert(kRankPer == 7, "rank registers sized for 7 positions per worker");
constexpr int kRankRegs = (kRankPer + 1) / 2;  // ranks (< 2^13) are kept two per register
__device__ __forceinline__ uint32_t rank_get(const uint32_t (&rk)[kRankRegs], int m) {
  return (rk[m >> 1] >> (16 * (m & 1))) & 0xffffu;
}
constexpr uint32_t kBigBucket = 256;  // buckets above this are sorted by a warp, not ranked by counting

constexpr int kBigMax = 32;  // more than d / kBigBucket <= 6144 / 257

// Exclusive scan of the padded array data (logical element i at data[PAD(i)]) by the
// worker warps (warp 0 is busy with the look-back meanwhile); returns the total.
__device__ uint32_t workers_exclusive_scan_pad(uint32_t* data, int n, uint32_t* warp_tmp) {
  constexpr int nt = kWorkers, nw = kWorkers / 32;
  const int t = threadIdx.x - 32, lane = t & 31, wid = t >> 5;
  const int per = (n + nt - 1) / nt;
  const int lo = min(n, t * per), hi = min(n, lo + per);
  uint32_t s = 0;
  for (int i = lo; i < hi; ++i) s += data[PAD(i)];
  uint32_t x = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tmp[wid] = x;
  bar_workers();
  if (wid == 0) {
    uint32_t w = lane < nw ? warp_tmp[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < nw) warp_tmp[lane] = w;
  }
  bar_workers();
  uint32_t run = x - s + (wid ? warp_tmp[wid - 1] : 0);
  const uint32_t total = warp_tmp[nw - 1];
  for (int i = lo; i < hi; ++i) {
    const uint32_t v = data[PAD(i)];
    data[PAD(i)] = run;
    run += v;
  }
  bar_workers();
  return total;
}

// Order the table's d occupied slots for output (worker warps only).  The key range
// [lo, hi] of the table is read from range_s[0..1] (written by worker 0 before the call).  NB
// buckets (key - lo) >> sh, one to two per key; an ordered counting sort of the slot
// numbers into idx[0, d), bucket by bucket (buckets ascending, slots unordered inside a
// bucket); hist[PAD(b)] is left holding bucket b's first position, and big_s[0, *big_n)
// lists the buckets above kBigBucket entries.
template <int KW>
__device__ void bucket_slots(Table<KW> tb, uint32_t nslots, uint32_t d, const typename KeyT<KW>::T* range_s,
                             uint32_t* hist, uint16_t* idx, uint32_t* wtmp, uint32_t* big_s, uint32_t* big_n,
                             typename KeyT<KW>::T& lo, int& sh, uint32_t& NB, uint32_t* status,
                             unsigned long long* prof = nullptr) {
  typedef typename KeyT<KW>::T K;
  const K EMPTY = all_ones<K>();
  long long tm = clock64();
  const int t = threadIdx.x - 32;
  auto mark = [&](int i) {
    if (prof && t == 0) {
      const long long now = clock64();
      atomicAdd(&prof[i], (unsigned long long)(now - tm));
      tm = now;
    }
  };
  NB = 1;
  while (NB < (uint32_t)hist_max(KW) && NB < d) NB <<= 1;
  for (uint32_t i = t; i < NB; i += kWorkers) hist[PAD(i)] = 0;
  if (t == 0) *big_n = 0;
  bar_workers();
  mark(2);
  lo = range_s[0];
  const K hi = range_s[1];
  const int bB = 31 - __clz(NB);
  sh = d == 0 ? 0 : max(0, bitlen(K(hi - lo)) - bB);
  uint32_t br[kSlotsPerWorker];
#pragma unroll
  for (int m = 0; m < kSlotsPerWorker; ++m) {
    const uint32_t s = t + m * kWorkers;
    br[m] = 0xffffffffu;
    if (s < nslots) {
      const K key = tb.keys[s];
      if (key != EMPTY) {
        if (key < lo || key > hi) {  // cannot happen: the range holds every key of the table
          atomicOr(status, ST_INTERNAL);
        } else {
          const uint32_t bk = (uint32_t)((key - lo) >> sh);
          const uint32_t r = atomicAdd(&hist[PAD(bk)], 1u);
          br[m] = (bk << 16) | r;  // NB <= 2^14, rank < 2^16
          if (r == kBigBucket) {   // the entry that takes bucket bk past kBigBucket
            const uint32_t q = atomicAdd(big_n, 1u);
            if (q < kBigMax) big_s[q] = bk;
            else atomicOr(status, ST_INTERNAL);
          }
        }
      }
    }
  }
  bar_workers();
  mark(5);
  workers_exclusive_scan_pad(hist, (int)NB, wtmp);
  mark(6);
#pragma unroll
  for (int m = 0; m < kSlotsPerWorker; ++m)
    if (br[m] != 0xffffffffu) idx[hist[PAD(br[m] >> 16)] + (br[m] & 0xffffu)] = (uint16_t)(t + m * kWorkers);
  bar_workers();
  mark(7);
}

// Worker warps: the rank of the entry at each bucket-grouped position j (its bucket's
// first position plus the number of smaller keys in the bucket).  The rare bucket above
// kBigBucket entries is first sorted in place by one warp and ranked by position.
template <int KW>
__device__ __forceinline__ void rank_slots(Table<KW> tb, const uint16_t* idx_c, uint16_t* idx, uint32_t d,
                                           const uint32_t* hist, uint32_t NB, typename KeyT<KW>::T lo, int sh,
                                           const uint32_t* big_s, uint32_t n_big, uint32_t (&rank)[kRankRegs],
                                           unsigned long long* prof) {
  typedef typename KeyT<KW>::T K;
  const int t = threadIdx.x - 32, wid = t >> 5;
  long long tm = clock64();
  constexpr int kWarps = kWorkers / 32;
  if (n_big) {  // rare: one warp per big bucket
    for (uint32_t q = wid; q < min(n_big, (uint32_t)kBigMax); q += kWarps) {
      const uint32_t bk = big_s[q];
      const uint32_t a = hist[PAD(bk)];
      const uint32_t e = bk + 1 < NB ? hist[PAD(bk + 1)] : d;
      warp_sort_idx<K>(tb.keys, idx, a, e - a);
    }
    bar_workers();
  }
  if (prof && t == 0) {
    const long long now = clock64();
    atomicAdd(&prof[3], (unsigned long long)(now - tm));
    tm = now;
  }
#pragma unroll
  for (int m = 0; m < kRankRegs; ++m) rank[m] = 0xffffffffu;
#pragma unroll
  for (int m = 0; m < kRankPer; ++m) {
    const uint32_t j = t + m * kWorkers;
    if (j < d) {
      const K key = tb.keys[idx_c[j]];
      const uint32_t bk = (uint32_t)((key - lo) >> sh);
      const uint32_t a = hist[PAD(bk)];
      const uint32_t e = bk + 1 < NB ? hist[PAD(bk + 1)] : d;
      uint32_t r = a;
      if (e - a > kBigBucket) {
        r = j;
      } else {
        for (uint32_t q = a; q < e; ++q) r += tb.keys[idx_c[q]] < key;
      }
      const int sh = 16 * (m & 1);
      rank[m >> 1] = (rank[m >> 1] & ~(0xffffu << sh)) | (r << sh);
    }
  }
  if (prof && t == 0) atomicAdd(&prof[4], (unsigned long long)(clock64() - tm));
}

// Worker threads: write the entry at each grouped position j to out[base + rank].  Ranks
// differ from j by less than a bucket, so the writes of a warp are nearly contiguous.
template <int KW>
__device__ __forceinline__ void emit_slots(Table<KW> tb, const uint16_t* idx, uint32_t d,
                                           const uint32_t (&rank)[kRankRegs], uint64_t base, uint64_t* out_keys,
                                           uint32_t* out_counts, uint64_t cap, uint32_t* status) {
  const int t = threadIdx.x - 32;
  if (base + d > cap) {
    if (t == 0) atomicOr(status, ST_INTERNAL);
    return;
  }
#pragma unroll
  for (int m = 0; m < kRankPer; ++m) {
    const uint32_t j = t + m * kWorkers;
    const uint32_t r = rank_get(rank, m);
    if (j < d && r < d) {
      const uint32_t s = idx[j];
      store_key(out_keys, base + r, tb.keys[s]);
      out_counts[base + r] = tb.counts[s];
    }
  }
}

__device__ __forceinline__ int ceil_log2_u32(uint32_t v) { return v <= 1 ? 0 : 32 - __clz(v - 1); }

template <int KW, bool MERGE = false>
__device__ __forceinline__ void count_emit_body(const Shape& s, const Buffers& b) {
  typedef typename KeyT<KW>::T K;
  extern __shared__ __align__(16) uint8_t sm[];
  const uint32_t cap_slots = 1u << s.bT_max;
  const uint32_t dcap = (3u * cap_slots) >> 2;  // most distinct keys a table is ordered with
  uint32_t* hist = reinterpret_cast<uint32_t*>(sm + (size_t)cap_slots * (KW * 8 + 4));
  uint16_t* idx = reinterpret_cast<uint16_t*>(hist + padded_len(hist_max(KW)));  // [dcap]
  __shared__ uint64_t excl_s, next_s[3];  // next ticket, its input range
  __shared__ volatile uint32_t ordered_s;  // the workers have ranked the current table
  __shared__ uint32_t next_u[2];          // its range-map interval: [next_u[0], next_u[1] - 1]
  __shared__ uint32_t ovf_s, special_s, nnew_s;
  __shared__ uint32_t wtmp[32];
  __shared__ K red_lo[32], red_hi[32];
  __shared__ K stk_lo[160], stk_hi[160];
  __shared__ K range_s[2];
  __shared__ uint32_t big_s[kBigMax], big_n;
  __shared__ int stk_n;
  const K EMPTY = all_ones<K>();
  const uint64_t NF = min(b.meta->n_fine, s.nf_max);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long* prof = s.profile ? reinterpret_cast<unsigned long long*>(b.meta->sub_cycles) : nullptr;
  unsigned long long* ticket = reinterpret_cast<unsigned long long*>(&b.meta->ticket);
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
  // The next partition's ticket, input range and range-map interval (next_s, next_u) are
  // fetched by thread 0 while the workers write the current partition out: the ticket is
  // taken as late as that, so that partitions start in ticket order and a look-back seldom
  // waits on a predecessor that started late; the rest arrives by asynchronous copies to
  // shared memory.  Tickets stay in increasing order within a block, so the block holding
  // the smallest unfinished ticket is always working on it and every look-back ends.
  auto fetch_next = [&](uint64_t nx) {  // one thread; completes at cp.async.wait_all
    next_s[0] = nx;
    if (nx < NF) {
      cp_async8(&next_s[1], &b.foff[nx]);
      cp_async8(&next_s[2], &b.fcur[nx]);  // the split's cursor: the partition's keys end there
      cp_async4(&next_u[0], &b.flo[nx]);
      cp_async4(&next_u[1], &b.flo[nx + 1]);
    }
  };
  if (threadIdx.x == 0) {
    ordered_s = 0;
    fetch_next(atomicAdd(ticket, 1ull));
    cp_async_wait_all();
  }
  while (true) {
    block_sync();
    const uint64_t g = next_s[0];
    if (g >= NF) break;
    const uint64_t f0 = next_s[1];
    uint64_t n = next_s[2] - f0;
    if (threadIdx.x == 0) {
      ovf_s = 0;
      special_s = 0;
      nnew_s = 0;
    }
    if (f0 > s.cap_kb || n > s.cap_kb - f0) {  // inconsistent scan: record it, count nothing
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
    block_sync();
    phase(0);
    count_all<KW, MERGE>(tb, in, n, false, K(0), K(0), bT, s.k == 32 * KW, s.count_limit, &nnew_s, &ovf_s,
                         &special_s, &b.meta->status);
    block_sync();
    phase(1);
    const uint32_t dn = nnew_s;
    if (!ovf_s && dn <= dcap) {
      const uint64_t d = (uint64_t)dn + (special_s ? 1 : 0);
      if (threadIdx.x == 0 && !(s.withhold && g == 0))
        st_status(&b.look[g], (g == 0 && !s.defer_all ? kLookIncl : kLookAgg) | d);
      // Warp 0 resolves the exclusive prefix (look-back) while the workers order the table,
      // waiting on unpublished predecessors only as long as the workers are busy.  Without a
      // prefix by then, the partition's run is written to its own input region instead
      // (deferred) and k_compact moves it once all counts are known.
      uint32_t rank[kRankRegs];
      if (wid == 0) {
        const long long lb0 = clock64();
        // (with a withheld prefix, a test that needs the wait to run out, it does not give up
        // when the ordering is done)
        const uint64_t ex = s.defer_all ? kNoPrefix
                            : g == 0    ? 0
                                        : lookback(b.look, g, &b.meta->status, s.spin_limit,
                                                   s.withhold ? nullptr : &ordered_s);
        if (lane == 0) {
          const bool direct = ex != kNoPrefix;
          if (direct && g > 0) st_status(&b.look[g], kLookIncl | (ex + d));
          b.fhist[g] = (uint32_t)d | (direct ? 0u : 0x80000000u);
          if (!direct) atomicAdd(reinterpret_cast<unsigned long long*>(&b.meta->n_deferred), 1ull);
          excl_s = ex;
          if (s.profile)
            atomicAdd(reinterpret_cast<unsigned long long*>(&b.meta->phase_cycles[4]), (unsigned long long)(clock64() - lb0));
        }
      } else {
        const long long tm = clock64();
        if (threadIdx.x == 32) {
          // every key of the partition lies in the key range of its range-map interval.
          // next_u still holds this partition's interval (the next one is fetched during
          // the write-out); flo[NF] = 0, so the last interval ends at 2^32 - 1
          const uint32_t ulo = next_u[0], uhi = next_u[1] - 1u;
          uint32_t xlo, xhi;
          x_range(ulo, uhi, s.canonical, xlo, xhi);
          key_range(xlo, xhi, s.k, range_s[0], range_s[1]);
        }
        K lo;
        int sh;
        uint32_t NB;
        bucket_slots<KW>(tb, 1u << bT, dn, range_s, hist, idx, wtmp, big_s, &big_n, lo, sh, NB, &b.meta->status,
                         prof);
        if (prof && threadIdx.x == 32) atomicAdd(&prof[1], (unsigned long long)(clock64() - tm));
        rank_slots<KW>(tb, idx, idx, dn, hist, NB, lo, sh, big_s, big_n, rank, prof);
        bar_workers();
        if (threadIdx.x == 32) ordered_s = 1;
      }
      block_sync();
      phase(3);
      const uint64_t ex = excl_s;
      if (threadIdx.x == 0) {
        ordered_s = 0;
        fetch_next(atomicAdd(ticket, 1ull));
      }
      // direct: final positions; deferred: the partition's own input region
      const bool direct = ex != kNoPrefix;
      uint64_t* okeys = direct ? b.out_keys : b.sbuf;
      uint32_t* ocnts = direct ? b.out_counts : reinterpret_cast<uint32_t*>(b.kbuf);
      const uint64_t obase = direct ? ex : f0, olim = direct ? s.cap : f0 + n;
      if (wid > 0) emit_slots<KW>(tb, idx, dn, rank, obase, okeys, ocnts, olim, &b.meta->status);
      if (threadIdx.x == 0) {
        if (special_s) {
          if (obase + dn < olim) {
            store_key(okeys, obase + dn, EMPTY);
            ocnts[obase + dn] = special_s;
          } else {
            atomicOr(&b.meta->status, ST_INTERNAL);
          }
        }
        cp_async_wait_all();
      }
      phase(5);
    } else {
      // ---------------- overflow path: too many distinct keys for the table.  Split the
      // partition's key range into sub-ranges, each counted in its own table and ordered;
      // the exclusive prefix is resolved first because the partial outputs are written
      // before the total is known.  A sub-range narrower than the table holds fewer
      // distinct keys than slots, so the splitting ends.
      if (wid == 0) {
        const uint64_t ex = g == 0 ? 0 : lookback(b.look, g, &b.meta->status, s.spin_limit);
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
      {
        K a, c;
        block_range<K>(mn, mx, red_lo, red_hi, a, c);
        if (threadIdx.x == 0) {
          stk_n = 0;
          if (a <= c) {
            stk_lo[0] = a;
            stk_hi[0] = c;
            stk_n = 1;
          }
        }
      }
      block_sync();
      const int bTf = s.bT_max;
      tb.keys = reinterpret_cast<K*>(sm);
      tb.counts = reinterpret_cast<uint32_t*>(tb.keys + cap_slots);
      uint64_t written = 0;
      while (stk_n > 0) {
        const K lo = stk_lo[stk_n - 1], hi = stk_hi[stk_n - 1];
        block_sync();
        if (threadIdx.x == 0) {
          --stk_n;
          ovf_s = 0;
          special_s = 0;
          nnew_s = 0;
        }
        table_clear<KW>(tb, cap_slots);
        block_sync();
        count_all<KW, MERGE>(tb, in, n, true, lo, hi, bTf, s.k == 32 * KW, s.count_limit, &nnew_s, &ovf_s,
                             &special_s, &b.meta->status);
        block_sync();
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
          block_sync();
          continue;
        }
        const uint64_t base = excl_s + written;
        {
          uint32_t rank2[kRankRegs];
          if (wid > 0) {
            if (threadIdx.x == 32) {
              range_s[0] = lo;
              range_s[1] = hi;
            }
            K lo2;
            int sh2;
            uint32_t NB2;
            bucket_slots<KW>(tb, cap_slots, dn2, range_s, hist, idx, wtmp, big_s, &big_n, lo2, sh2, NB2,
                             &b.meta->status);
            rank_slots<KW>(tb, idx, idx, dn2, hist, NB2, lo2, sh2, big_s, big_n, rank2, nullptr);
          }
          block_sync();
          if (wid > 0) emit_slots<KW>(tb, idx, dn2, rank2, base, b.out_keys, b.out_counts, s.cap, &b.meta->status);
        }
        written += dn2;
        block_sync();
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
      block_sync();
      if (threadIdx.x == 0) {
        uint64_t tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wtmp[w];
        if (tot) {
          if (tot > s.count_limit) atomicOr(&b.meta->status, ST_COUNT_OVERFLOW);
          if (excl_s + written < s.cap) {
            store_key(b.out_keys, excl_s + written, EMPTY);
            b.out_counts[excl_s + written] = (uint32_t)tot;
          } else {
            atomicOr(&b.meta->status, ST_INTERNAL);
          }
          ++written;
        }
        if (!(s.withhold && g == 0)) st_status(&b.look[g], kLookIncl | (excl_s + written));
        b.fhist[g] = (uint32_t)written;
        fetch_next(atomicAdd(ticket, 1ull));
        cp_async_wait_all();
      }
      phase(6);
    }
  }
}
template <int KW, bool MERGE = false>
__global__ void __launch_bounds__(kCountThreads, kCountBlocksPerSM) k_count_emit(Shape s, Buffers b) {
  count_emit_body<KW, MERGE>(s, b);
}
template <int KW>
__global__ void __launch_bounds__(kCountThreads, kCountBlocksPerSM) k_count_emit_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  count_emit_body<KW>(d.s, d.b);
}

// ------------------------------------------------------------------ final: offsets of the runs
// Exclusive scan of the distinct counts of the fine partitions (one block of 1024
// threads): fcur[g] = first output position of partition g, n_distinct = the total.  The
// look-back words are checked against it, and the deferred partitions are listed (in
// increasing order) at the front of the spent look-back array for k_compact.
__device__ __forceinline__ void scan_distinct_body(const Shape& sh, const Buffers& b) {
  __shared__ uint64_t wt[32];
  __shared__ uint32_t wd[32];
  __shared__ uint64_t carry_s;
  __shared__ uint32_t dcarry_s;
  const uint64_t NF = min(b.meta->n_fine, sh.nf_max);
  const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, wid = t >> 5;
  if (t == 0) {
    carry_s = 0;
    dcarry_s = 0;
  }
  __syncthreads();
  bool bad = false;
  for (uint64_t base = 0; base < NF; base += (uint64_t)nt * 8) {
    uint32_t v[8];
    unsigned long long lk[8];
    uint64_t s = 0;
    uint32_t nd = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const uint64_t i = base + (uint64_t)t * 8 + m;
      v[m] = i < NF ? b.fhist[i] : 0;
      lk[m] = i < NF ? ld_status(&b.look[i]) : 0;
      s += v[m] & 0x7fffffffu;
      nd += v[m] >> 31;
    }
    uint64_t x = s;
    uint32_t y = nd;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t xs = __shfl_up_sync(0xffffffffu, x, d);
      const uint32_t ys = __shfl_up_sync(0xffffffffu, y, d);
      if (lane >= d) {
        x += xs;
        y += ys;
      }
    }
    if (lane == 31) {
      wt[wid] = x;
      wd[wid] = y;
    }
    __syncthreads();  // also: every look-back word of this chunk has been read
    if (wid == 0) {
      uint64_t w = wt[lane];
      uint32_t z = wd[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t ws = __shfl_up_sync(0xffffffffu, w, d);
        const uint32_t zs = __shfl_up_sync(0xffffffffu, z, d);
        if (lane >= d) {
          w += ws;
          z += zs;
        }
      }
      wt[lane] = w;
      wd[lane] = z;
    }
    __syncthreads();
    uint64_t run = carry_s + x - s + (wid ? wt[wid - 1] : 0);
    uint32_t drun = dcarry_s + y - nd + (wid ? wd[wid - 1] : 0);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const uint64_t i = base + (uint64_t)t * 8 + m;
      if (i < NF) {
        const uint64_t d = v[m] & 0x7fffffffu;
        const bool deferred = v[m] >> 31;
        // a direct partition published its inclusive prefix, a deferred one its count
        const uint64_t want = deferred ? (kLookAgg | d) : (kLookIncl | (run + d));
        bad |= lk[m] != want;
        b.fcur[i] = run;
        if (deferred) b.look[drun++] = i;
        run += d;
      }
    }
    __syncthreads();
    if (t == 0) {
      carry_s += wt[31];
      dcarry_s += wd[31];
    }
    __syncthreads();
  }
  if (bad) atomicOr(&b.meta->status, ST_INTERNAL);
  if (t == 0) {
    b.meta->n_distinct = carry_s;
    if (dcarry_s != b.meta->n_deferred) atomicOr(&b.meta->status, ST_INTERNAL);
  }
}
__global__ void __launch_bounds__(1024) k_scan_distinct(Shape sh, Buffers b) { scan_distinct_body(sh, b); }
__global__ void __launch_bounds__(1024) k_scan_distinct_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  scan_distinct_body(d.s, d.b);
}

// Move the runs of the deferred fine partitions from their input regions (keys in sbuf,
// counts in kbuf as 32-bit words) to their output positions: one block per partition.
template <int KW>
__device__ __forceinline__ void compact_body(const Shape& s, const Buffers& b, uint32_t bid, uint32_t nblk) {
  typedef typename KeyT<KW>::T K;
  const uint64_t n_def = min(b.meta->n_deferred, s.nf_max);
  const uint32_t* cnt_src = reinterpret_cast<const uint32_t*>(b.kbuf);
  for (uint64_t q = bid; q < n_def; q += nblk) {
    const uint64_t g = b.look[q];
    if (g >= min(b.meta->n_fine, s.nf_max)) {
      if (threadIdx.x == 0) atomicOr(&b.meta->status, ST_INTERNAL);
      continue;
    }
    const uint32_t d = b.fhist[g] & 0x7fffffffu;
    const uint64_t src = b.foff[g], dst = b.fcur[g];
    if (src + d > s.cap_kb || dst + d > s.cap) {
      if (threadIdx.x == 0) atomicOr(&b.meta->status, ST_INTERNAL);
      continue;
    }
    for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) {
      K key;
      load_key(b.sbuf, src + i, key);
      store_key(b.out_keys, dst + i, key);
      b.out_counts[dst + i] = cnt_src[src + i];
    }
  }
}
template <int KW>
__global__ void __launch_bounds__(256) k_compact(Shape s, Buffers b) {
  compact_body<KW>(s, b, blockIdx.x, gridDim.x);
}
template <int KW>
__global__ void __launch_bounds__(256) k_compact_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  compact_body<KW>(d.s, d.b, bid, nblk);
}

// ------------------------------------------------------------------ launches
constexpr size_t kScatterStaticSmem = 9216;  // pass B's static shared memory (batched form included), rounded up
static size_t scatter_smem(int kw, int nt, int P1, bool keep_c) {
  const size_t sub = (size_t)nt * (kw == 1 ? 32 : 16);
  return sub * (size_t)(kw * 8) + (size_t)P1 * 8 + 2 * padded_len(P1 + 32) * 4 + (keep_c ? sub * 4 : 0);
}
static size_t fine_hist_smem(int P1) { return (size_t)(P1 + 1) * 8 + kFineLocalCap * 4 + 16; }
static size_t fine_scatter_smem(int kw, int P1) {
  return (size_t)kFineChunk * (kw * 8 + 2) + kFineLocalCap * (8 + 4 + 4) + (size_t)(P1 + 1) * 8 + 16;
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
  KC_SET((k_scatter<1, 256, false>));
  KC_SET((k_scatter<2, 256, false>));
  KC_SET((k_scatter<1, 256, true>));
  KC_SET((k_scatter<2, 256, true>));
  KC_SET(k_scatter_direct<1>);
  KC_SET(k_scatter_direct<2>);
  KC_SET(k_fine_plan);
  KC_SET(k_fine_hist<1>);
  KC_SET(k_fine_hist<2>);
  KC_SET(k_fine_scatter<1>);
  KC_SET(k_fine_scatter<2>);
  KC_SET(k_count_emit<1>);
  KC_SET(k_count_emit<2>);
  KC_SET((k_count_emit<1, true>));
  KC_SET((k_count_emit<2, true>));
  KC_SET(k_bucket_scan);
  KC_SET(k_pack_count_batch<1>);
  KC_SET(k_pack_count_batch<2>);
  KC_SET((k_scatter_batch<1, 256, false>));
  KC_SET((k_scatter_batch<2, 256, false>));
  KC_SET((k_scatter_batch<1, 256, true>));
  KC_SET((k_scatter_batch<2, 256, true>));
  KC_SET(k_fine_plan_batch);
  KC_SET(k_fine_hist_batch<1>);
  KC_SET(k_fine_hist_batch<2>);
  KC_SET(k_fine_scatter_batch<1>);
  KC_SET(k_fine_scatter_batch<2>);
  KC_SET(k_count_emit_batch<1>);
  KC_SET(k_count_emit_batch<2>);
  KC_SET(k_bucket_scan_batch);
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
    k_check_offsets<<<g, 256, 0, st>>>(b.offsets, s.n_reads, s.L, b.meta);
    ++launches;
    KC_STEP("k_check_offsets");
  }
  if (s.n_tiles == 0) return launches;
  k_tile_first<<<(unsigned)((s.n_tiles + 127) / 128), 128, 0, st>>>(b.offsets, s.n_reads, s.n_tiles, b.tile_first);
  ++launches;
  KC_STEP("k_tile_first");
  const size_t smA = (size_t)(P1 + 32) * 4;
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
    const size_t smB = scatter_smem(s.kw, 256, P1, false), smK = scatter_smem(s.kw, 256, P1, true);
    if (smB + kScatterStaticSmem > s.smem_budget) return -(int)cudaErrorInvalidConfiguration;
    // keep each window's coarse partition in shared memory if two blocks per SM still fit
    int per_sm = 0;
    if (s.kw == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter<1, 256, true>, 256, smK);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter<2, 256, true>, 256, smK);
    const bool keep_c = per_sm >= 2;
    const unsigned gt = (unsigned)s.n_tiles;
    if (s.aggr & kAggrNoSmemBuckets) {
      k_direct_cursors<<<(P1 + 255) / 256, 256, 0, st>>>(b.cstart, b.fcur, P1);
      ++launches;
      KC_STEP("k_direct_cursors");
      if (s.kw == 1) k_scatter_direct<1><<<gt, 256, smB, st>>>(s, b);
      else k_scatter_direct<2><<<gt, 256, smB, st>>>(s, b);
    } else if (s.kw == 1) {
      if (keep_c) k_scatter<1, 256, true><<<gt, 256, smK, st>>>(s, b);
      else k_scatter<1, 256, false><<<gt, 256, smB, st>>>(s, b);
    } else {
      if (keep_c) k_scatter<2, 256, true><<<gt, 256, smK, st>>>(s, b);
      else k_scatter<2, 256, false><<<gt, 256, smB, st>>>(s, b);
    }
    ++launches;
    KC_STEP("k_scatter");
  }
  k_fine_plan<<<1, 1024, (size_t)P1 * 8, st>>>(b.cstart, b.hll, b.fine_base, b.fine_m, b.flo, P1, s.b1, s.fine_target, nf_max,
                                               b.meta);
  ++launches;
  KC_STEP("k_fine_plan");
  const unsigned gf = (unsigned)(n_sms * 2);
  // the fine split (sampled layout or exact); after a sampled one, the exact split again,
  // whose kernels return at once unless a sampled region overflowed
  for (int redo = 0; redo <= (s.fine_sampled ? 1 : 0); ++redo) {
    if (redo) {
      k_fine_redo_clear<<<(unsigned)n_sms, 1024, 0, st>>>(s, b);
      ++launches;
      KC_STEP("k_fine_redo_clear");
    }
    if (s.kw == 1) k_fine_hist<1><<<gf, kFineThreads, fine_hist_smem(P1), st>>>(s, b, redo);
    else k_fine_hist<2><<<gf, kFineThreads, fine_hist_smem(P1), st>>>(s, b, redo);
    ++launches;
    KC_STEP(redo ? "k_fine_hist_redo" : "k_fine_hist");
    k_fine_scan<<<1, 1024, 0, st>>>(s, b, redo);
    ++launches;
    KC_STEP(redo ? "k_fine_scan_redo" : "k_fine_scan");
    if (s.kw == 1) k_fine_scatter<1><<<gf, kFineThreads, fine_scatter_smem(1, P1), st>>>(s, b, redo);
    else k_fine_scatter<2><<<gf, kFineThreads, fine_scatter_smem(2, P1), st>>>(s, b, redo);
    ++launches;
    KC_STEP(redo ? "k_fine_scatter_redo" : "k_fine_scatter");
  }
  const size_t smC = count_kernel_smem(s.kw, s.bT_max, s.tail);
  if (s.aggr & kAggrWarpMerge) {
    if (s.kw == 1) k_count_emit<1, true><<<(unsigned)(n_sms * kCountBlocksPerSM), kCountThreads, smC, st>>>(s, b);
    else k_count_emit<2, true><<<(unsigned)(n_sms * kCountBlocksPerSM), kCountThreads, smC, st>>>(s, b);
  } else if (s.kw == 1) {
    k_count_emit<1><<<(unsigned)(n_sms * kCountBlocksPerSM), kCountThreads, smC, st>>>(s, b);
  } else {
    k_count_emit<2><<<(unsigned)(n_sms * kCountBlocksPerSM), kCountThreads, smC, st>>>(s, b);
  }
  ++launches;
  KC_STEP("k_count_emit");
  k_scan_distinct<<<1, 1024, 0, st>>>(s, b);
  ++launches;
  KC_STEP("k_scan_distinct");
  if (s.kw == 1) k_compact<1><<<(unsigned)(n_sms * 8), 256, 0, st>>>(s, b);
  else k_compact<2><<<(unsigned)(n_sms * 8), 256, 0, st>>>(s, b);
  ++launches;
  KC_STEP("k_compact");
  return launches;
}

uint32_t batch_blocks(BatchKernel k, const Shape& s, int n_sms, uint64_t bases_total) {
  auto clampu = [](uint64_t v, uint64_t lo, uint64_t hi) { return (uint32_t)(v < lo ? lo : (v > hi ? hi : v)); };
  const uint64_t P1 = 1ull << s.b1, nsm = (uint64_t)n_sms;
  switch (k) {
    case BK_CLEAR: return clampu((s.nf_max + 2047) / 2048, 1, 32);
    case BK_CHECK: return clampu((s.n_reads + 255) / 256, 1, 64);
    case BK_TILE_FIRST: return (uint32_t)((s.n_tiles + 127) / 128);
    case BK_PACK: return (uint32_t)s.n_tiles;
    case BK_COL_SCAN: return s.n_tiles ? (uint32_t)((P1 + 31) / 32) : 0u;
    case BK_SCATTER: return (uint32_t)s.n_tiles;
    case BK_FINE_HIST:
    case BK_FINE_SCATTER: return clampu((s.L + 4ull * kFineChunk - 1) / (4ull * kFineChunk), 1, 2 * nsm);
    case BK_COUNT: {
      const double share = bases_total ? (double)s.L / (double)bases_total : 1.0;
      return clampu((uint64_t)(2.0 * (double)nsm * share + 0.999), 1, nsm * kCountBlocksPerSM);
    }
    case BK_COMPACT: return clampu(s.nf_max / 8, 1, 8 * nsm);
    default: return 1u;  // one block per count: bucket scan, fine plan, fine scan, scan of distinct counts
  }
}

// The launch sequence of launch_phase1 + launch_phase2, each kernel once for all counts of
// the batch (all with the same key width); a kernel that gives no count a block is skipped.
int launch_batch(const BatchPlan& bp, int n_sms, void* stream, const Marker& mark) {
  cudaStream_t st = (cudaStream_t)stream;
  const int P1 = bp.P1_max;
  const Shape& s0 = bp.host[0].s;
  int launches = 0;
  auto tab = [&](BatchKernel k) { return BatchTab{bp.desc, bp.blk2s[k], bp.start[k]}; };
#define KC_BLAUNCH(k, call, name) \
  if (bp.grid[k]) {               \
    call;                         \
    ++launches;                   \
    KC_STEP(name);                \
  }
  KC_BLAUNCH(BK_CLEAR, (k_clear_batch<<<bp.grid[BK_CLEAR], 256, 0, st>>>(tab(BK_CLEAR))), "k_clear_batch");
  KC_BLAUNCH(BK_CHECK, (k_check_offsets_batch<<<bp.grid[BK_CHECK], 256, 0, st>>>(tab(BK_CHECK))), "k_check_offsets");
  KC_BLAUNCH(BK_TILE_FIRST, (k_tile_first_batch<<<bp.grid[BK_TILE_FIRST], 128, 0, st>>>(tab(BK_TILE_FIRST))),
             "k_tile_first");
  if (bp.kw == 1) {
    KC_BLAUNCH(BK_PACK, (k_pack_count_batch<1><<<bp.grid[BK_PACK], kPackThreads, (size_t)(P1 + 32) * 4, st>>>(tab(BK_PACK))),
               "k_pack_count");
  } else {
    KC_BLAUNCH(BK_PACK, (k_pack_count_batch<2><<<bp.grid[BK_PACK], kPackThreads, (size_t)(P1 + 32) * 4, st>>>(tab(BK_PACK))),
               "k_pack_count");
  }
  KC_BLAUNCH(BK_COL_SCAN, (k_col_scan_batch<<<bp.grid[BK_COL_SCAN], dim3(32, 32), 0, st>>>(tab(BK_COL_SCAN))),
             "k_col_scan");
  KC_BLAUNCH(BK_BUCKET_SCAN,
             (k_bucket_scan_batch<<<bp.grid[BK_BUCKET_SCAN], 1024, (size_t)P1 * 8, st>>>(tab(BK_BUCKET_SCAN))),
             "k_bucket_scan");
  if (bp.grid[BK_SCATTER]) {
    const size_t smB = scatter_smem(bp.kw, 256, P1, false), smK = scatter_smem(bp.kw, 256, P1, true);
    if (smB + kScatterStaticSmem > s0.smem_budget) return -(int)cudaErrorInvalidConfiguration;
    int per_sm = 0;
    if (bp.kw == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter_batch<1, 256, true>, 256, smK);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter_batch<2, 256, true>, 256, smK);
    const unsigned g = bp.grid[BK_SCATTER];
    if (bp.kw == 1) {
      if (per_sm >= 2) k_scatter_batch<1, 256, true><<<g, 256, smK, st>>>(tab(BK_SCATTER));
      else k_scatter_batch<1, 256, false><<<g, 256, smB, st>>>(tab(BK_SCATTER));
    } else {
      if (per_sm >= 2) k_scatter_batch<2, 256, true><<<g, 256, smK, st>>>(tab(BK_SCATTER));
      else k_scatter_batch<2, 256, false><<<g, 256, smB, st>>>(tab(BK_SCATTER));
    }
    ++launches;
    KC_STEP("k_scatter");
  }
  KC_BLAUNCH(BK_FINE_PLAN, (k_fine_plan_batch<<<bp.grid[BK_FINE_PLAN], 1024, (size_t)P1 * 8, st>>>(tab(BK_FINE_PLAN))),
             "k_fine_plan");
  // the fine split; then, for counts with a sampled layout, the exact split again (each
  // count's blocks return at once unless its sampled regions overflowed)
  for (int redo = 0; redo <= (bp.sampled ? 1 : 0); ++redo) {
    if (redo)
      KC_BLAUNCH(BK_FINE_SCAN, (k_fine_redo_clear_batch<<<bp.grid[BK_FINE_SCAN], 1024, 0, st>>>(tab(BK_FINE_SCAN))),
                 "k_fine_redo_clear");
    if (bp.kw == 1) {
      KC_BLAUNCH(BK_FINE_HIST,
                 (k_fine_hist_batch<1><<<bp.grid[BK_FINE_HIST], kFineThreads, fine_hist_smem(P1), st>>>(
                     tab(BK_FINE_HIST), redo)),
                 redo ? "k_fine_hist_redo" : "k_fine_hist");
    } else {
      KC_BLAUNCH(BK_FINE_HIST,
                 (k_fine_hist_batch<2><<<bp.grid[BK_FINE_HIST], kFineThreads, fine_hist_smem(P1), st>>>(
                     tab(BK_FINE_HIST), redo)),
                 redo ? "k_fine_hist_redo" : "k_fine_hist");
    }
    KC_BLAUNCH(BK_FINE_SCAN, (k_fine_scan_batch<<<bp.grid[BK_FINE_SCAN], 1024, 0, st>>>(tab(BK_FINE_SCAN), redo)),
               redo ? "k_fine_scan_redo" : "k_fine_scan");
    if (bp.kw == 1) {
      KC_BLAUNCH(BK_FINE_SCATTER,
                 (k_fine_scatter_batch<1><<<bp.grid[BK_FINE_SCATTER], kFineThreads, fine_scatter_smem(1, P1), st>>>(
                     tab(BK_FINE_SCATTER), redo)),
                 redo ? "k_fine_scatter_redo" : "k_fine_scatter");
    } else {
      KC_BLAUNCH(BK_FINE_SCATTER,
                 (k_fine_scatter_batch<2><<<bp.grid[BK_FINE_SCATTER], kFineThreads, fine_scatter_smem(2, P1), st>>>(
                     tab(BK_FINE_SCATTER), redo)),
                 redo ? "k_fine_scatter_redo" : "k_fine_scatter");
    }
  }
  const size_t smC = count_kernel_smem(bp.kw, s0.bT_max, s0.tail);
  if (bp.kw == 1) {
    KC_BLAUNCH(BK_COUNT, (k_count_emit_batch<1><<<bp.grid[BK_COUNT], kCountThreads, smC, st>>>(tab(BK_COUNT))),
               "k_count_emit");
  } else {
    KC_BLAUNCH(BK_COUNT, (k_count_emit_batch<2><<<bp.grid[BK_COUNT], kCountThreads, smC, st>>>(tab(BK_COUNT))),
               "k_count_emit");
  }
  KC_BLAUNCH(BK_SCAN_DISTINCT,
             (k_scan_distinct_batch<<<bp.grid[BK_SCAN_DISTINCT], 1024, 0, st>>>(tab(BK_SCAN_DISTINCT))),
             "k_scan_distinct");
  if (bp.kw == 1) {
    KC_BLAUNCH(BK_COMPACT, (k_compact_batch<1><<<bp.grid[BK_COMPACT], 256, 0, st>>>(tab(BK_COMPACT))), "k_compact");
  } else {
    KC_BLAUNCH(BK_COMPACT, (k_compact_batch<2><<<bp.grid[BK_COMPACT], 256, 0, st>>>(tab(BK_COMPACT))), "k_compact");
  }
#undef KC_BLAUNCH
  return launches;
}

}  // namespace kc

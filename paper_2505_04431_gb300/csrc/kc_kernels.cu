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
//   k_fine_plan             sizes the fine partitions of every coarse partition (one
//                           shared-memory table each, from a HyperLogLog estimate of the
//                           distinct keys) and lays out the phase-2 tasks.
//   k_phase2                persistent; takes the coarse partitions in turn: split tasks
//                           regroup a coarse partition's keys by fine partition chunk by
//                           chunk, count tasks count each fine partition in a hashed
//                           open-addressing table in shared memory (CAS claims a slot, a
//                           32-bit atomic add counts), order the occupied slots by a
//                           bucketed counting sort over the partition's key range and
//                           write the sorted (key, count) run at the offset found by a
//                           decoupled look-back (or later, from the block's stage slot).
//                           A coarse partition's keys pass between its split and count
//                           tasks through L2 only.
//   k_scan_distinct         checks every partition's published prefix; the output size.
// Variants: every kernel body also runs as a batched kernel (one launch for a group of
// counts, each thread block working for one count found through a block table); pass B
// without the shared-memory staging (DIRECT) and the count tasks with a warp-level merge
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
// Batched launches: the arrays a count needs zeroed (status record, distinct counts,
// look-back words, sketch, partition starts, split counters) are cleared by one kernel for
// all counts.
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
  for (uint64_t i = i0; i < (1ull << s.b1); i += stride) b.sdone[i] = 0;
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
  extern __shared__ uint32_t hist_s[];  // [P1]
  __shared__ uint64_t code_s[kPackThreads + 2];
  __shared__ uint32_t inv_s[kPackThreads + 2];
  __shared__ uint32_t st_s[kPackThreads + 2];
  __shared__ uint64_t rcur_s, len_s;
  const int t = threadIdx.x;
  const int P1 = 1 << s.b1;
  const uint64_t tile = bid;
  for (int c = t; c < P1; c += kPackThreads) hist_s[c] = 0;
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
      for (int i = 0; i < 32; ++i) {
        if ((W.valid >> i) & 1u)
          atomicAdd(&hist_s[coarse_field(umap(win_top32<KW, 32>(W, i, s.canonical), s.canonical), s.b1)], 1u);
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

// Plan of phase 2, after pass B (one block).  The distinct-key estimate (a sampled
// HyperLogLog filled by pass B) gives the duplication factor K / D, and a fine partition
// aims at fine_target distinct keys, i.e. fine_target * K / D keys: coarse partition c is
// cut into m_c = ceil(n_c / target) parts of its range of u (at most kMaxFine) and split in
// ceil(n_c / split_chunk) chunks.  Written here: each fine partition's first value of u
// (flo), each coarse partition's first fine partition and first run-start entry, and the
// ticket layout (stage s: the split tasks of coarse partition s, then the count tasks of
// coarse partition s - 1).
__device__ __forceinline__ void fine_plan_body(const Shape& s, const Buffers& b) {
  extern __shared__ uint64_t fsc[];  // [P1 + kStageLag + 1]
  __shared__ uint64_t wt[32];
  __shared__ float zsum_s[32], zeros_s[32];
  __shared__ double target_s;
  const int P1 = 1 << s.b1, b1 = s.b1;
  const uint64_t CH = split_chunk(s.kw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Meta* meta = b.meta;
  const uint64_t* cstart = b.cstart;
  // HyperLogLog estimate over the 1/8 hash-sample of the keys
  float z = 0.f, zeros = 0.f;
  for (int i = threadIdx.x; i < kHllRegs; i += blockDim.x) {
    const uint32_t r = b.hll[i];
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
    target_s = (double)s.fine_target * (0.9 * dup > 1.0 ? 0.9 * dup : 1.0);
    meta->d_estimate = (uint64_t)d_est;
  }
  __syncthreads();
  const double target = target_s;
  // fine partitions per coarse partition, and their first index
  for (int c = threadIdx.x; c <= P1; c += blockDim.x) {
    uint64_t m = 0;
    if (c < P1) {
      const uint64_t n = cstart[c + 1] - cstart[c];
      m = (uint64_t)ceil((double)n / target);
      m = m < 1 ? 1 : (m > (uint64_t)kMaxFine ? (uint64_t)kMaxFine : m);
      b.fine_m[c] = (uint32_t)m;
    }
    fsc[c] = m;
  }
  __syncthreads();
  const uint64_t NF = block_exclusive_scan<uint64_t>(fsc, P1 + 1, wt);
  for (int c = threadIdx.x; c <= P1; c += blockDim.x) b.fine_base[c] = (uint32_t)fsc[c];
  // fine partition g = fsc[c] + f holds the values u of coarse field c whose low part
  // v = u mod 2^(32 - b1) has floor(v m / 2^(32 - b1)) = f, i.e. v >= ceil(f 2^(32 - b1) / m);
  // one thread per fine partition, its coarse partition found by binary search in fsc
  const uint64_t w = 1ull << (32 - b1);
  for (uint64_t g = threadIdx.x; g < NF && g < s.nf_max; g += blockDim.x) {
    int lo = 0, hi = P1 - 1;  // last c with fsc[c] <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (fsc[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    const uint64_t m = b.fine_m[lo], f = g - fsc[lo];
    b.flo[g] = (uint32_t)((uint64_t)lo << (32 - b1)) + (uint32_t)((f * w + m - 1) / m);
  }
  __syncthreads();
  // run-start entries: (m_c + 1) per chunk of coarse partition c
  for (int c = threadIdx.x; c <= P1; c += blockDim.x) {
    uint64_t e = 0;
    if (c < P1) e = ((uint64_t)b.fine_m[c] + 1) * ((cstart[c + 1] - cstart[c] + CH - 1) / CH);
    fsc[c] = e;
  }
  __syncthreads();
  const uint64_t TE = block_exclusive_scan<uint64_t>(fsc, P1 + 1, wt);
  for (int c = threadIdx.x; c <= P1; c += blockDim.x) b.tbase[c] = fsc[c];
  __syncthreads();
  // tickets: stage s = split tasks of s (s < P1), then count tasks of s - kStageLag
  const int NS = P1 + kStageLag;  // stages
  for (int c = threadIdx.x; c <= NS; c += blockDim.x) {
    uint64_t v = 0;
    if (c < P1) v += (cstart[c + 1] - cstart[c] + CH - 1) / CH;
    if (c >= kStageLag && c < NS) v += b.fine_m[c - kStageLag];
    fsc[c] = v;
  }
  __syncthreads();
  const uint64_t T = block_exclusive_scan<uint64_t>(fsc, NS + 1, wt);
  const bool ok = NF <= s.nf_max && TE <= s.tcap && T < 0xffffffffull;
  for (int c = threadIdx.x; c < NS; c += blockDim.x) {
    b.tstart[c] = ok ? (uint32_t)fsc[c] : 0u;
    const uint64_t nch = c < P1 ? (cstart[c + 1] - cstart[c] + CH - 1) / CH : 0;
    b.tsplit[c] = ok ? (uint32_t)(fsc[c] + nch) : 0u;
  }
  if (threadIdx.x == 0) {
    if (NF <= s.nf_max) b.flo[NF] = 0;  // so that the last partition ends at u = 2^32 - 1
    b.tstart[NS] = ok ? (uint32_t)T : 0u;  // no tasks when a capacity is exceeded
    meta->n_fine = ok ? NF : 0;                 // later kernels never index past nf_max
    meta->n_tasks = ok ? T : 0;
    if (!ok) atomicOr(&meta->status, ST_INTERNAL);
  }
}
__global__ void k_fine_plan(Shape s, Buffers b) { fine_plan_body(s, b); }
__global__ void k_fine_plan_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  fine_plan_body(d.s, d.b);
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
  uint32_t* soff = hist + padded_len(P1);                                               // [padded P1]
  uint16_t* rawc = reinterpret_cast<uint16_t*>(soff + padded_len(P1));  // KEEP_C: [SUB], window i of thread t at i * NT + t
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
      // the arithmetic of every window is branch-free (so that the windows' dependency chains
      // interleave); only the shared-memory updates depend on the window being valid
#pragma unroll
      for (int i = 0; i < WPT; ++i) {
        uint64_t c0, c1;
        win_top<KW, WPT>(W, i, s.canonical, c0, c1);
        top_to_key(c0, c1, s.k, keys[i]);
        const uint32_t c = coarse_field(umap((uint32_t)(c0 >> 32), s.canonical), s.b1);
        const uint64_t hh = key_hash(keys[i]);
        const bool v = (valid >> i) & 1u;
        if (v) {
          if constexpr (DIRECT) {
            // the cursors of this variant are the first P1 words of toff (tile 0's offsets,
            // which it does not read)
            const unsigned long long pos = atomicAdd(reinterpret_cast<unsigned long long*>(&b.toff[c]), 1ull);
            if (pos < s.cap) store_key(b.kbuf, pos, keys[i]);
            else atomicOr(&b.meta->status, ST_INTERNAL);
          } else {
            if constexpr (KEEP_C) rawc[i * NT + t] = (uint16_t)c;
            rr[i >> 1] |= atomicAdd(&hist[PAD(c)], 1u) << (16 * (i & 1));
          }
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
      if (valid & (1u << i)) {
        uint32_t c;
        if constexpr (KEEP_C) c = rawc[i * NT + t];
        else c = coarse_of(keys[i], s.k, s.canonical, s.b1);  // same field as above, from the key
        const uint32_t pos = soff[PAD(c)] + ((rr[i >> 1] >> (16 * (i & 1))) & 0xffffu);
        stage[pos] = keys[i];
        if constexpr (KEEP_C) stage_c[pos] = (uint16_t)c;
      }
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


// ------------------------------------------------------------------ phase 2: count helpers
constexpr uint64_t kLookValue = (1ull << 62) - 1;
constexpr uint64_t kLookAgg = 1ull << 62;
constexpr uint64_t kLookIncl = 2ull << 62;

// Decoupled look-back (executed by one warp): sum of distinct counts of fine partitions < g.
// (A decoupled look-back is the published single-pass prefix-scan method: each partition
// publishes its own total as soon as it is known and its inclusive prefix once that is.)
// Each step reads the kLookPer * 32 status words before position j at once (lane l holds
// distance q * 32 + l); the nearest inclusive prefix among them ends the walk, and only
// unpublished words nearer than it are waited for (with a bounded spin).  With `abort`,
// the wait also ends as soon as *abort becomes nonzero, and kNoPrefix is returned.
constexpr int kLookPer = 8;
constexpr uint64_t kNoPrefix = ~0ull;
__device__ uint64_t lookback(unsigned long long* look, uint64_t g, uint32_t* status, uint32_t spin_limit,
                             const volatile uint32_t* abort = nullptr, unsigned long long* prof = nullptr) {
  const int lane = threadIdx.x & 31;
  constexpr uint32_t kNone = kLookPer * 32;
  uint64_t excl = 0;
  int64_t j = (int64_t)g - 1;
  uint32_t steps = 0, waits = 0;
  struct Tally {  // profiled calls: walk steps and wait iterations, added by lane 0 on return
    unsigned long long* p;
    const uint32_t &st, &wt;
    int lane;
    __device__ ~Tally() {
      if (p && lane == 0) {
        p[0] += st;
        p[1] += wt;
      }
    }
  } tally_{prof, steps, waits, lane};
  while (j >= 0) {
    ++steps;
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
      ++waits;
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

// Shared memory of the phase-2 kernel.  The count tasks use a hash table of 2^bT_max slots
// (key + count), a bucket histogram of hist_max(kw) entries and the 16-bit slot numbers of
// up to 3/4 of the slots in output order; the split tasks reuse the same bytes for their
// staging (keys and their fine partitions) and four per-fine-partition arrays.  After it
// come the areas every task keeps: the ticket layout (stage starts, count starts) and one
// batch of a fine partition's runs.
constexpr int kTableLog2Cap = 13;  // 8192 slots: 8 per thread of the 1024-thread block
__host__ __device__ constexpr int hist_max(int kw) { return kw == 1 ? 16384 : 8192; }
constexpr int kBinsPad = kMaxFine + 1 + ((kMaxFine + 1) >> 5) + 1;  // padded_len(kMaxFine + 1)
__host__ __device__ inline size_t align_to(size_t x, size_t a) { return (x + a - 1) / a * a; }
__host__ __device__ inline size_t count_area_bytes(int kw, int bT_max) {
  const size_t slots = (size_t)1 << bT_max;
  return slots * (size_t)(kw * 8 + 4) + padded_len(hist_max(kw)) * 4 + ((3 * slots) >> 2) * 2 + 256;
}
__host__ __device__ inline size_t split_area_bytes(int kw) {
  return (size_t)split_sub(kw) * (kw * 8 + 2) + 4 * (size_t)kBinsPad * 4;
}
__host__ __device__ inline size_t phase2_area(int kw, int bT_max) {
  const size_t a = count_area_bytes(kw, bT_max), b = split_area_bytes(kw);
  return align_to(a > b ? a : b, 16);
}
__host__ __device__ constexpr int max_coarse(int kw) { return 1 << max_coarse_log2(kw); }
__host__ __device__ inline size_t persist_bytes(int kw) {
  return (size_t)(2 * (max_coarse(kw) + kStageLag) + 1) * 4 + (size_t)(3 * kRunBatch + 1) * 4 + 16;
}
size_t phase2_smem(int kw, int bT_max) { return phase2_area(kw, bT_max) + persist_bytes(kw); }

int table_log2_max(int kw, size_t smem_optin) {
  int best = 6;
  for (int bt = 6; bt <= kTableLog2Cap; ++bt)
    if (phase2_smem(kw, bt) + 8192 <= smem_optin) best = bt;  // 8 KB for static shared memory
  return best;
}

// A deferred run in the stage: keys (dcap + 1 of them, the all-ones key included), then
// counts, each part on whole 128-byte lines.
__host__ __device__ inline size_t stage_keys_bytes(int kw, int bT_max) {
  return align_to((((size_t)3 << bT_max) / 4 + 1) * kw * 8, 128);
}
size_t stage_slot_bytes(int kw, int bT_max) {
  return align_to(stage_keys_bytes(kw, bT_max) + align_to((((size_t)3 << bT_max) / 4 + 1) * 4, 128), 256);
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
                                            uint32_t* status) {
  typedef typename KeyT<KW>::T K;
  const K EMPTY = all_ones<K>();
  const uint32_t mask = (1u << bT) - 1;
  uint32_t s = hslot(key, bT);
  for (int probe = 0; probe < kProbeLimit; ++probe, s = (s + 1) & mask) {
    int res = 0;
    if constexpr (KW == 1) {
      uint64_t* p = reinterpret_cast<uint64_t*>(tb.keys) + s;
      const uint64_t cur = *reinterpret_cast<volatile uint64_t*>(p);
      if (cur == (uint64_t)key) {
        res = 1;
      } else if (cur == ~0ull) {
        const unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long*>(p), ~0ull, (unsigned long long)key);
        res = old == ~0ull ? 2 : (old == (unsigned long long)key ? 1 : 0);
      }
    } else {
      const K old = cas128_shared(reinterpret_cast<u128*>(tb.keys) + s, (u128)EMPTY, (u128)key);
      res = old == EMPTY ? 2 : (old == key ? 1 : 0);
    }
    if (res) {
      if (check) {
        const uint32_t o = atomicAdd(&tb.counts[s], inc);
        if (o > 0xffffffffu - inc) atomicOr(status, ST_COUNT_OVERFLOW);
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

constexpr int kRankPer = 7;           // positions per worker thread: 7 * 992 >= 3/4 of 8192 slots
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

// ------------------------------------------------------------------ phase 2: split + count
// One persistent kernel does the second phase for every coarse partition in turn.  Its
// work is a list of tasks taken in ticket order, laid out stage by stage: stage s holds the
// split tasks of coarse partition s, then the count tasks of coarse partition s - 1.
//
//   split task (c, j)   chunk j of coarse partition c (split_chunk keys of kbuf): the
//                       chunk's fine-partition histogram, then its keys placed in sbuf at
//                       the same positions, grouped by fine partition (staged per
//                       sub-chunk in shared memory, written as runs); where each fine
//                       partition's run starts in the chunk goes to rstart.
//   count task (c, f)   fine partition g = fine_base[c] + f: waits until every split task
//                       of c is done, gathers its run from every chunk of c, counts the
//                       keys in a shared-memory table, orders the distinct keys and writes
//                       them out (Algorithm 3 after its barrier: Sort + Accumulate).
//
// A coarse partition is small enough (about 19 MB of keys) that its chunks are still in
// L2 when its count tasks read them one stage later, and the lines a count task has read
// are discarded from L2 (discard.global.L2), so the split copy is not written back to HBM.
// Every wait is on a task with a smaller ticket (tickets are taken in order by running
// thread blocks), so the smallest unfinished ticket always makes progress.
//
// Output offsets come from a decoupled look-back over the fine partitions (the published
// single-pass scan method: each partition publishes its total as soon as it is known and
// its inclusive prefix once that is).  A partition whose prefix is not known when its keys
// are ordered leaves its run in the block's own stage slot (in L2) and writes it out later,
// once its prefix is known: when the block needs the slot again, after a later task if the
// prefix is known by then without waiting, or at the end.

__device__ __forceinline__ void discard_l2(uintptr_t line) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(line) : "memory");
}
// Discard the 128-byte lines that lie wholly inside the bytes [lo, hi); thread i of n.
__device__ __forceinline__ void discard_lines(const void* lo, const void* hi, uint32_t i, uint32_t n) {
  const uintptr_t a = ((uintptr_t)lo + 127) & ~(uintptr_t)127, e = (uintptr_t)hi & ~(uintptr_t)127;
  for (uintptr_t x = a + (uintptr_t)i * 128; x < e; x += (uintptr_t)n * 128) discard_l2(x);
}
__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Data written by other thread blocks of the same launch is read at L2 (ld.global.cg).
__device__ __forceinline__ void load_key_cg(const uint64_t* src, uint64_t i, uint64_t& key) { key = __ldcg(src + i); }
__device__ __forceinline__ void load_key_cg(const uint64_t* src, uint64_t i, u128& key) {
  const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(src) + i);
  key = ((u128)v.y << 64) | v.x;
}

// Fine partition of a key inside its coarse partition (m parts of the coarse range of u):
// floor(v m / 2^(32 - b1)) for the low part v of u, the high word of (v << b1) m.
template <class K>
__device__ __forceinline__ uint32_t fine_in_coarse(K key, int k, int canonical, int b1, uint32_t m, uint32_t& coarse) {
  const uint32_t u = umap(top32_of(key, k), canonical);
  coarse = coarse_field(u, b1);
  return __umulhi(b1 ? u << b1 : u, m);
}

// Shared state of a phase-2 thread block that outlives one task.
struct P2State {
  // the next task, prepared by thread 0 while the block finishes the current one
  uint64_t nx_cs, nx_ce, nx_tb, nx_g;
  uint32_t nx_kind, nx_c, nx_i, nx_m, nx_ulo, nx_uhi;
  // deferred runs waiting in this block's stage slots, oldest first: slot (pend_head + i) %
  // n_slots holds partition pend_g[...] with pend_d[...] entries, for i < pend_n
  uint64_t pend_g[kMaxSlots];
  uint32_t pend_d[kMaxSlots];
  uint32_t pend_head, pend_n;
  uint64_t excl;
  uint32_t ordered, one, ovf, special, nnew, wait_ok, big_n;
  uint32_t nseg;
  uint64_t nkeys;
  int stk_n;
  // profiled plans: thread 0's cycles per phase and task tallies (added to the status record)
  unsigned long long acc[8], tally[8];
  long long tmark;
};
enum : uint32_t { TASK_SPLIT = 0, TASK_COUNT = 1, TASK_DONE = 2 };

template <int KW, bool MERGE>
struct Phase2 {
  typedef typename KeyT<KW>::T K;
  static constexpr uint32_t SUB = split_sub(KW), CH = split_chunk(KW), PER = SUB / kCountThreads;
  static constexpr int kIn = KW == 1 ? 8 : 2;  // keys in flight per lane while counting
  const Shape& s;
  const Buffers& b;
  uint8_t* sm;
  P2State& st;
  uint32_t* wtmp;       // [32]
  uint32_t* tstart_s;   // [P1 + 2]
  uint32_t* tsplit_s;   // [P1 + 1]
  uint32_t* run_st;     // [kRunBatch] start of each run inside its coarse partition
  uint32_t* run_len;    // [kRunBatch]
  uint32_t* run_pre;    // [kRunBatch + 1] exclusive prefix of the run lengths
  K* red_lo;            // [32]
  K* red_hi;            // [32]
  K* range_s;           // [2]
  K* stk_lo;            // [160]
  K* stk_hi;            // [160]
  uint32_t* big_s;      // [kBigMax]
  uint8_t* slots;       // this block's stage slots
  int P1;
  uint32_t cap_slots, dcap;

  __device__ uint32_t tid() const { return threadIdx.x; }
  // profiled plans: the cycles since the last mark go to phase i (thread 0's view; it takes
  // part in every block barrier, so its time is the block's)
  __device__ void mark(int i) {
    if (s.profile && tid() == 0) {
      const long long now = clock64();
      st.acc[i] += (unsigned long long)(now - st.tmark);
      st.tmark = now;
    }
  }
  __device__ void tally(int i, unsigned long long v = 1) {
    if (s.profile && tid() == 0) st.tally[i] += v;
  }

  // ---- thread 0: take the next ticket and look its task up
  __device__ void prefetch() {
    unsigned long long* ticket = reinterpret_cast<unsigned long long*>(&b.meta->ticket);
    const uint64_t t = atomicAdd(ticket, 1ull);
    const uint64_t n_tasks = tstart_s[P1 + kStageLag];
    if (t >= n_tasks) {
      st.nx_kind = TASK_DONE;
      return;
    }
    int lo = 0, hi = P1 + kStageLag - 1;  // the stage: last s with tstart_s[s] <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tstart_s[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    uint32_t c, i, kind;
    if (t < tsplit_s[lo]) {
      kind = TASK_SPLIT;
      c = (uint32_t)lo;
      i = (uint32_t)(t - tstart_s[lo]);
    } else {
      kind = TASK_COUNT;
      c = (uint32_t)(lo - kStageLag);
      i = (uint32_t)(t - tsplit_s[lo]);
    }
    st.nx_kind = kind;
    st.nx_c = c;
    st.nx_i = i;
    st.nx_cs = b.cstart[c];
    st.nx_ce = b.cstart[c + 1];
    st.nx_m = b.fine_m[c];
    st.nx_tb = b.tbase[c];
    if (kind == TASK_COUNT) {
      const uint64_t g = (uint64_t)b.fine_base[c] + i;
      st.nx_g = g;
      st.nx_ulo = b.flo[g];
      st.nx_uhi = b.flo[g + 1] - 1u;  // flo[NF] = 0: the last interval ends at 2^32 - 1
    }
  }

  // ---- split task (c, j)
  // One warp's exclusive scan of the padded array d[0, n) in place (lane l takes a contiguous
  // stretch); returns the total to every lane.
  __device__ static uint32_t warp_scan_pad(uint32_t* d, uint32_t n) {
    const uint32_t lane = threadIdx.x & 31, per = (n + 31) >> 5;
    const uint32_t a = min(n, lane * per), e = min(n, a + per);
    uint32_t sum = 0;
    for (uint32_t i = a; i < e; ++i) sum += d[PAD(i)];
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    uint32_t run = x - sum;
    for (uint32_t i = a; i < e; ++i) {
      const uint32_t v = d[PAD(i)];
      d[PAD(i)] = run;
      run += v;
    }
    return __shfl_sync(0xffffffffu, x, 31);
  }

  __device__ void split(uint32_t c, uint32_t j, uint64_t cs, uint64_t ce, uint32_t m, uint64_t tb) {
    K* stage = reinterpret_cast<K*>(sm);
    uint16_t* stage_g = reinterpret_cast<uint16_t*>(stage + SUB);
    uint32_t* cur = reinterpret_cast<uint32_t*>(stage_g + SUB);  // padded [m + 1]: counts, then cursors
    uint32_t* scnt = cur + kBinsPad;                               // padded [m]: keys of the sub-chunk
    uint32_t* soff = scnt + kBinsPad;                              // padded [m]: their staged start
    int32_t* delta = reinterpret_cast<int32_t*>(soff + kBinsPad);  // [m]: chunk position - staged position
    const uint32_t t = tid();
    const uint64_t nc = ce - cs;
    const uint64_t nch = (nc + CH - 1) / CH;
    const uint64_t lo = cs + (uint64_t)j * CH, hi = min(lo + CH, ce);
    const int k = s.k, can = s.canonical, b1 = s.b1;
    bool bad = m == 0 || m > (uint32_t)kMaxFine;
    if (bad) m = 1;
    // pass 1: how many keys of the chunk each fine partition gets
    for (uint32_t f = t; f <= m; f += kCountThreads) {
      cur[PAD(f)] = 0;
      scnt[PAD(f)] = 0;
    }
    block_sync();
    for (uint64_t base = lo; base < hi; base += SUB) {
      K keys[PER];
#pragma unroll
      for (uint32_t q = 0; q < PER; ++q) {
        const uint64_t i = base + t + (uint64_t)q * kCountThreads;
        keys[q] = 0;
        if (i < hi) load_key(b.kbuf, i, keys[q]);
      }
#pragma unroll
      for (uint32_t q = 0; q < PER; ++q) {
        const uint64_t i = base + t + (uint64_t)q * kCountThreads;
        if (i < hi) {
          uint32_t cc;
          const uint32_t f = fine_in_coarse(keys[q], k, can, b1, m, cc);
          if (cc == c && f < m) atomicAdd(&cur[PAD(f)], 1u);
          else bad = true;
        }
      }
    }
    block_sync();
    if (t < 32) warp_scan_pad(cur, m + 1);  // cur[PAD(m)]: keys of the chunk
    block_sync();
    for (uint32_t f = t; f <= m; f += kCountThreads)
      b.rstart[tb + (uint64_t)f * nch + j] = (uint16_t)cur[PAD(f)];  // < 2^16: a chunk holds at most 32768 keys
    // pass 2: each sub-chunk's keys ranked by fine partition, staged and written as runs at
    // their partition's place in the chunk.  Three barriers per sub-chunk: one warp scans
    // the sub-chunk's counts (and advances the cursors, and clears the counts) between the
    // ranking and the staging, and the write-out of a sub-chunk overlaps the ranking of
    // the next.  Warp 0 does not write out: thread 0 takes the next ticket meanwhile.
    for (uint64_t base = lo; base < hi; base += SUB) {
      K keys[PER];
      uint32_t fr[PER];
#pragma unroll
      for (uint32_t q = 0; q < PER; ++q) {
        const uint64_t i = base + t + (uint64_t)q * kCountThreads;
        keys[q] = 0;
        if (i < hi) load_key(b.kbuf, i, keys[q]);
      }
#pragma unroll
      for (uint32_t q = 0; q < PER; ++q) {
        const uint64_t i = base + t + (uint64_t)q * kCountThreads;
        fr[q] = 0xffffffffu;
        if (i < hi) {
          uint32_t cc;
          const uint32_t f = fine_in_coarse(keys[q], k, can, b1, m, cc);
          if (cc == c && f < m) fr[q] = (f << 16) | atomicAdd(&scnt[PAD(f)], 1u);  // rank < SUB <= 2^13
          else bad = true;
        }
      }
      block_sync();  // ranks taken; the previous sub-chunk is written out
      if (t < 32) {
        const uint32_t lane = t;
        const uint32_t per = (m + 31) >> 5;
        const uint32_t a = min(m, lane * per), e = min(m, a + per);
        uint32_t sum = 0;
        for (uint32_t f = a; f < e; ++f) sum += scnt[PAD(f)];
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= (uint32_t)o) x += y;
        }
        uint32_t run = x - sum;
        for (uint32_t f = a; f < e; ++f) {
          const uint32_t v = scnt[PAD(f)];
          soff[PAD(f)] = run;
          delta[f] = (int32_t)cur[PAD(f)] - (int32_t)run;
          cur[PAD(f)] += v;
          scnt[PAD(f)] = 0;
          run += v;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, x, 31);
        if (lane == 0) st.nseg = tot;  // keys staged in this sub-chunk
      }
      block_sync();
      const uint32_t n_staged = min((uint32_t)umin64(SUB, hi - base), st.nseg);
#pragma unroll
      for (uint32_t q = 0; q < PER; ++q) {
        if (fr[q] != 0xffffffffu) {
          const uint32_t f = fr[q] >> 16;
          const uint32_t pos = soff[PAD(f)] + (fr[q] & 0xffffu);
          if (pos < n_staged) {
            stage[pos] = keys[q];
            stage_g[pos] = (uint16_t)f;
          } else {
            bad = true;
          }
        }
      }
      block_sync();
      if (base + SUB >= hi && t == 0) prefetch();
      if (t >= 32) {
        for (uint32_t i = t - 32; i < n_staged; i += kCountThreads - 32) {
          const uint64_t dst = (uint64_t)((int64_t)lo + delta[stage_g[i]] + (int64_t)i);
          if (dst >= lo && dst < hi) store_key(b.sbuf, dst, stage[i]);
          else bad = true;
        }
      }
    }
    if (lo >= hi && t == 0) prefetch();  // an empty chunk (cannot happen: chunks cover the keys)
    // the chunk's keys in kbuf are not read again
    discard_lines(b.kbuf + lo * KW, b.kbuf + hi * KW, t, kCountThreads);
    if (bad) atomicOr(&b.meta->status, ST_INTERNAL);
    block_sync();
    if (t == 0) {
      __threadfence();
      atomicAdd(&b.sdone[c], 1u);
    }
    mark(0);
    tally(0);
  }

  // ---- count task: the runs of fine partition f in the chunks [jb, jb + kRunBatch) of
  // coarse partition c into run_st / run_len / run_pre; returns their keys (all threads)
  __device__ uint64_t load_runs(uint64_t tb, uint32_t f, uint64_t nch, uint64_t jb, uint64_t nc) {
    const uint32_t t = tid();
    const uint64_t nr = umin64(kRunBatch, nch - jb);
    uint32_t mine = 0;
    for (uint32_t r = t; r < (uint32_t)kRunBatch; r += kCountThreads) {
      uint32_t len = 0;
      if (r < nr) {
        const uint64_t jj = jb + r;
        const uint32_t a = __ldcg(b.rstart + tb + (uint64_t)f * nch + jj);
        const uint32_t e = __ldcg(b.rstart + tb + (uint64_t)(f + 1) * nch + jj);
        // a run lies inside its chunk, and the chunk inside the coarse partition
        if (e < a || jj * CH + e > nc) atomicOr(&b.meta->status, ST_INTERNAL);
        else len = e - a;
        run_st[r] = (uint32_t)(jj * CH) + a;
        run_len[r] = len;
      }
      run_pre[r] = len;
    }
    block_sync();
    const uint32_t total = block_exclusive_scan<uint32_t>(run_pre, kRunBatch, wtmp);
    if (t == 0) run_pre[kRunBatch] = total;
    block_sync();
    return total;
  }

  // all keys of fine partition f (a pass over its run starts only)
  __device__ uint64_t input_size(uint64_t tb, uint32_t f, uint64_t nch, uint64_t nc) {
    const uint32_t t = tid();
    uint64_t mine = 0;
    for (uint64_t jj = t; jj < nch; jj += kCountThreads) {
      const uint32_t a = __ldcg(b.rstart + tb + (uint64_t)f * nch + jj);
      const uint32_t e = __ldcg(b.rstart + tb + (uint64_t)(f + 1) * nch + jj);
      if (e >= a && jj * CH + e <= nc) mine += e - a;
    }
    if (t == 0) st.nkeys = 0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, d);
    block_sync();
    if ((t & 31) == 0 && mine) atomicAdd(reinterpret_cast<unsigned long long*>(&st.nkeys), (unsigned long long)mine);
    block_sync();
    return st.nkeys;
  }

  // Count the keys of the loaded runs (only those in [lo, hi] when `ranged`).  The runs are
  // read as one sequence (run_pre: where each starts in it) in chunks of 256 keys, warp w
  // taking chunks w, w + 32, ...; each lane finds its key's run by stepping forward from
  // the chunk's first run.  The all-ones key is counted apart in st.special (it marks empty
  // slots); it exists only when the k-mer fills the key word (full_width).  With MERGE, a
  // warp whose active keys are all equal adds them with one atomic (the heavy-hitter merge
  // of the paper's L3 layer).  Returns the slots this thread claimed.
  __device__ uint32_t count_runs(Table<KW> tb, const uint64_t* src, uint32_t nr, bool ranged, K lo, K hi, int bT,
                                 bool full_width, bool check) {
    const K EMPTY = all_ones<K>();
    const uint32_t lane = tid() & 31, w = tid() >> 5;
    const uint32_t n = nr ? run_pre[kRunBatch] : 0;
    uint32_t claimed = 0;
    for (uint32_t base = w * 256; base < n; base += (kCountThreads / 32) * 256) {
      int a = 0, z = (int)nr - 1;  // the run of key `base`: last r with run_pre[r] <= base
      while (a < z) {
        const int mid = (a + z + 1) >> 1;
        if (run_pre[mid] <= base) a = mid;
        else z = mid - 1;
      }
      uint32_t r = (uint32_t)a;
      for (uint32_t m0 = 0; m0 < 256; m0 += 32 * kIn) {
        K kk[kIn];
        bool aa[kIn];
#pragma unroll
        for (int m = 0; m < kIn; ++m) {
          const uint32_t i = base + m0 + lane + 32 * m;
          kk[m] = 0;
          aa[m] = i < n;
          if (aa[m]) {
            while (r + 1 < nr && run_pre[r + 1] <= i) ++r;
            load_key_cg(src, (uint64_t)run_st[r] + (i - run_pre[r]), kk[m]);
          }
        }
#pragma unroll
        for (int m = 0; m < kIn; ++m) {
          const K key = kk[m];
          bool act = aa[m];
          if (ranged) act = act && key >= lo && key <= hi && key != EMPTY;
          const K k0 = shfl_key(key, 0);
          if (MERGE && __all_sync(0xffffffffu, !act || key == k0)) {
            const unsigned am = __ballot_sync(0xffffffffu, act);
            if (am && lane == (uint32_t)(__ffs(am) - 1)) {
              const uint32_t inc = __popc(am);
              if (full_width && k0 == EMPTY) {
                if (atomicAdd(&st.special, inc) > 0xffffffffu - inc) atomicOr(&b.meta->status, ST_COUNT_OVERFLOW);
              } else {
                const int res = count_insert<KW>(tb, k0, inc, bT, check, &b.meta->status);
                if (!res) atomicOr(&st.ovf, 1u);
                claimed += res == 2;
              }
            }
          } else if (act) {
            if (full_width && key == EMPTY) {
              if (atomicAdd(&st.special, 1u) == 0xffffffffu) atomicOr(&b.meta->status, ST_COUNT_OVERFLOW);
            } else {
              const int res = count_insert<KW>(tb, key, 1u, bT, check, &b.meta->status);
              if (!res) atomicOr(&st.ovf, 1u);
              claimed += res == 2;
            }
          }
        }
      }
    }
    return claimed;
  }

  // Block-wide sum of the slots claimed into st.nnew (all threads).
  __device__ void add_claimed(uint32_t claimed) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) claimed += __shfl_xor_sync(0xffffffffu, claimed, d);
    if ((tid() & 31) == 0 && claimed) atomicAdd(&st.nnew, claimed);
  }

  // Discard the sbuf lines of the loaded runs (read for the last time).
  __device__ void discard_runs(const uint64_t* src, uint32_t nr) {
    const uint32_t lane = tid() & 31, w = tid() >> 5;
    for (uint32_t r = w; r < nr; r += kCountThreads / 32)
      discard_lines(src + (uint64_t)run_st[r] * KW, src + ((uint64_t)run_st[r] + run_len[r]) * KW, lane, 32);
  }

  __device__ uint8_t* slot_at(uint32_t i) const { return slots + (size_t)i * s.stage_bytes; }

  // ---- the oldest run waiting in the stage: written out once its prefix is known.  With
  // `blocking`, the look-back waits (bounded) for it; otherwise the call gives up at the
  // first wait.  Returns whether it was written out (all threads).
  __device__ bool finalize(bool blocking) {
    block_sync();
    if (st.pend_n == 0) return false;
    const uint32_t si = st.pend_head;
    const uint64_t g = st.pend_g[si];
    const uint32_t d = st.pend_d[si];
    const long long t0 = clock64();
    if (tid() < 32) {
      const uint64_t ex = lookback(b.look, g, &b.meta->status, s.spin_limit, blocking ? nullptr : &st.one,
                                   s.profile && blocking ? &st.tally[6] : nullptr);
      if (tid() == 0) st.excl = ex;
    }
    block_sync();
    if (blocking) tally(4, (unsigned long long)(clock64() - t0));
    const uint64_t ex = st.excl;
    if (ex == kNoPrefix) return false;
    uint8_t* slot = slot_at(si);
    const uint64_t* skeys = reinterpret_cast<const uint64_t*>(slot);
    const uint32_t* scnts = reinterpret_cast<const uint32_t*>(slot + stage_keys_bytes(KW, s.bT_max));
    if (tid() == 0) st_status(&b.look[g], kLookIncl | (ex + d));
    if (ex + d > s.cap) {
      if (tid() == 0) atomicOr(&b.meta->status, ST_INTERNAL);
    } else {
      for (uint32_t i = tid(); i < d; i += kCountThreads) {
        K key;
        load_key_cg(skeys, i, key);
        store_key(b.out_keys, ex + i, key);
        b.out_counts[ex + i] = __ldcg(scnts + i);
      }
    }
    block_sync();
    // the slot is this block's own: its used lines are dropped without a write-back
    discard_lines(slot, slot + align_to((size_t)d * KW * 8, 128), tid(), kCountThreads);
    discard_lines(scnts, reinterpret_cast<const uint8_t*>(scnts) + align_to((size_t)d * 4, 128), tid(), kCountThreads);
    if (tid() == 0) {
      st.pend_head = (si + 1) % s.n_slots;
      --st.pend_n;
    }
    block_sync();
    return true;
  }

  // ---- count task (c, f)
  __device__ void count(uint32_t c, uint32_t f, uint64_t g, uint64_t cs, uint64_t ce, uint64_t tb, uint32_t ulo,
                        uint32_t uhi) {
    const K EMPTY = all_ones<K>();
    const uint32_t t = tid(), lane = t & 31, wid = t >> 5;
    uint32_t* hist = reinterpret_cast<uint32_t*>(sm + (size_t)cap_slots * (KW * 8 + 4));
    uint16_t* idx = reinterpret_cast<uint16_t*>(hist + padded_len(hist_max(KW)));  // [dcap]
    const uint64_t nch = (ce - cs + CH - 1) / CH;
    const uint64_t* src = b.sbuf + cs * KW;
    const bool full_width = s.k == 32 * KW;
    if (t == 0) {
      st.ovf = 0;
      st.special = 0;
      st.nnew = 0;
      // the split of coarse partition c must be complete (bounded wait)
      uint32_t spins = 0, ok = 1;
      while (ld_acquire_u32(&b.sdone[c]) < (uint32_t)nch) {
        if (++spins > kLookbackSpinLimit) {
          atomicOr(&b.meta->status, ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
      st.wait_ok = ok;
      if (spins) tally(2);
    }
    tally(1);
    block_sync();
    mark(1);
    const uint64_t nch_eff = st.wait_ok ? nch : 0;
    const bool one_batch = nch_eff <= (uint64_t)kRunBatch;
    const uint64_t nc = ce - cs;
    uint64_t n = one_batch ? load_runs(tb, f, nch_eff, 0, nc) : input_size(tb, f, nch_eff, nc);
    uint32_t nr = (uint32_t)umin64(kRunBatch, nch_eff);
    if (n > s.cap) {
      if (t == 0) atomicOr(&b.meta->status, ST_INTERNAL);
      n = 0;
      nr = 0;
      if (t == 0) run_pre[kRunBatch] = 0;
    }
    const bool check = n > 0xffffffffull;  // a count can pass 2^32 - 1 only in a partition that large
    // table: at least twice the keys (at most that many distinct), within the cap
    int bT = 6;
    while (bT < s.bT_max && ((uint64_t)1 << bT) < 2 * n) ++bT;
    Table<KW> tb_;
    tb_.keys = reinterpret_cast<K*>(sm);
    tb_.counts = reinterpret_cast<uint32_t*>(tb_.keys + (1u << bT));
    table_clear<KW>(tb_, 1u << bT);
    block_sync();
    {
      uint32_t claimed = 0;
      if (one_batch) {
        claimed = count_runs(tb_, src, nr, false, K(0), K(0), bT, full_width, check);
      } else {
        for (uint64_t jb = 0; jb < nch_eff; jb += kRunBatch) {
          load_runs(tb, f, nch_eff, jb, nc);
          claimed += count_runs(tb_, src, (uint32_t)umin64(kRunBatch, nch_eff - jb), false, K(0), K(0), bT,
                                full_width, check);
          block_sync();
        }
      }
      add_claimed(claimed);
    }
    block_sync();
    mark(2);
    const uint32_t dn = st.nnew;
    if (!st.ovf && dn <= dcap) {
      if (one_batch) discard_runs(src, nr);
      const uint64_t d = (uint64_t)dn + (st.special ? 1 : 0);
      const bool publish = !(s.withhold && g == 0);
      if (t == 0) {
        if (publish) st_status(&b.look[g], (g == 0 && !s.defer_all ? kLookIncl : kLookAgg) | d);
        b.fhist[g] = (uint32_t)d;
        st.ordered = 0;
      }
      block_sync();
      // Warp 0 resolves the exclusive prefix (look-back) while the workers order the table,
      // waiting on unpublished predecessors only as long as the workers are busy.
      uint32_t rank[kRankRegs];
      if (wid == 0) {
        const uint64_t ex =
            s.defer_all ? kNoPrefix : g == 0 ? 0 : lookback(b.look, g, &b.meta->status, s.spin_limit, &st.ordered);
        if (lane == 0) {
          if (ex != kNoPrefix && g > 0) st_status(&b.look[g], kLookIncl | (ex + d));
          st.excl = ex;
        }
      } else {
        if (t == 32) {
          // every key of the partition lies in the key range of its range-map interval
          uint32_t xlo, xhi;
          x_range(ulo, uhi, s.canonical, xlo, xhi);
          key_range(xlo, xhi, s.k, range_s[0], range_s[1]);
        }
        K klo;
        int sh;
        uint32_t NB;
        bucket_slots<KW>(tb_, 1u << bT, dn, range_s, hist, idx, wtmp, big_s, &st.big_n, klo, sh, NB, &b.meta->status);
        rank_slots<KW>(tb_, idx, idx, dn, hist, NB, klo, sh, big_s, st.big_n, rank, nullptr);
        bar_workers();
        if (t == 32) st.ordered = 1;
      }
      block_sync();
      mark(3);
      const uint64_t ex = st.excl;
      if (ex != kNoPrefix) {
        // direct: final positions; thread 0 takes the next ticket meanwhile
        if (t == 0) prefetch();
        if (wid > 0) emit_slots<KW>(tb_, idx, dn, rank, ex, b.out_keys, b.out_counts, s.cap, &b.meta->status);
        if (t == 32 && st.special) {
          if (ex + dn < s.cap) {
            store_key(b.out_keys, ex + dn, EMPTY);
            b.out_counts[ex + dn] = st.special;
          } else {
            atomicOr(&b.meta->status, ST_INTERNAL);
          }
        }
        block_sync();
        mark(4);
        tally(3);
      } else {
        // deferred: the run waits in a stage slot of this block; when all are taken, the
        // oldest is written out first (waiting for its prefix)
        while (!finalize(false) && st.pend_n == s.n_slots) finalize(true);
        if (t == 0) prefetch();
        const uint32_t si = (st.pend_head + st.pend_n) % s.n_slots;
        uint8_t* slot = slot_at(si);
        uint64_t* okeys = reinterpret_cast<uint64_t*>(slot);
        uint32_t* ocnts = reinterpret_cast<uint32_t*>(slot + stage_keys_bytes(KW, s.bT_max));
        if (wid > 0) emit_slots<KW>(tb_, idx, dn, rank, 0, okeys, ocnts, (uint64_t)dcap + 1, &b.meta->status);
        block_sync();
        if (t == 32) {
          if (st.special) {
            store_key(okeys, dn, EMPTY);
            ocnts[dn] = st.special;
          }
          st.pend_g[si] = g;
          st.pend_d[si] = (uint32_t)d;
          ++st.pend_n;
          atomicAdd(reinterpret_cast<unsigned long long*>(&b.meta->n_deferred), 1ull);
        }
        block_sync();
        mark(5);
      }
      return;
    }
    // ---------------- overflow path: too many distinct keys for the table.  Split the
    // partition's key range into sub-ranges, each counted in its own table and ordered;
    // the exclusive prefix is resolved first because the partial outputs are written
    // before the total is known.  A sub-range narrower than the table holds fewer distinct
    // keys than slots, so the splitting ends.
    if (wid == 0) {
      const uint64_t ex = g == 0 ? 0 : lookback(b.look, g, &b.meta->status, s.spin_limit);
      if (lane == 0) st.excl = ex;
    }
    if (t == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&b.meta->n_overflow), 1ull);
    K mn = EMPTY, mx = 0;
    uint32_t sp = 0;  // the all-ones key, if present, is the largest key of all
    for (uint64_t jb = 0; jb < nch_eff; jb += kRunBatch) {
      const uint32_t nrb = (uint32_t)umin64(kRunBatch, nch_eff - jb);
      if (!one_batch) load_runs(tb, f, nch_eff, jb, nc);
      for (uint32_t r = wid; r < nrb; r += kCountThreads / 32) {
        for (uint32_t i = lane; i < run_len[r]; i += 32) {
          K key;
          load_key_cg(src, (uint64_t)run_st[r] + i, key);
          if (key != EMPTY) {
            mn = key < mn ? key : mn;
            mx = key > mx ? key : mx;
          } else {
            ++sp;
          }
        }
      }
      block_sync();
    }
    {
      K a, cc;
      block_range<K>(mn, mx, red_lo, red_hi, a, cc);
      if (t == 0) {
        st.stk_n = 0;
        if (a <= cc) {
          stk_lo[0] = a;
          stk_hi[0] = cc;
          st.stk_n = 1;
        }
      }
    }
    block_sync();
    const int bTf = s.bT_max;
    tb_.keys = reinterpret_cast<K*>(sm);
    tb_.counts = reinterpret_cast<uint32_t*>(tb_.keys + cap_slots);
    uint64_t written = 0;
    while (st.stk_n > 0) {
      const K lo = stk_lo[st.stk_n - 1], hi = stk_hi[st.stk_n - 1];
      block_sync();
      if (t == 0) {
        --st.stk_n;
        st.ovf = 0;
        st.special = 0;
        st.nnew = 0;
      }
      table_clear<KW>(tb_, cap_slots);
      block_sync();
      uint32_t claimed = 0;
      for (uint64_t jb = 0; jb < nch_eff; jb += kRunBatch) {
        const uint32_t nrb = (uint32_t)umin64(kRunBatch, nch_eff - jb);
        if (!one_batch) load_runs(tb, f, nch_eff, jb, nc);
        claimed += count_runs(tb_, src, nrb, true, lo, hi, bTf, false, check);
        block_sync();
      }
      add_claimed(claimed);
      block_sync();
      const uint32_t dn2 = st.nnew;
      const K width = hi - lo;
      if (st.ovf || dn2 > dcap) {
        if (t == 0) {
          if (width == 0 || st.stk_n + 2 > 160) {
            atomicOr(&b.meta->status, ST_INTERNAL);  // a single key cannot overflow
          } else {
            const K mid = lo + (width >> 1);
            stk_lo[st.stk_n] = mid + 1;
            stk_hi[st.stk_n] = hi;
            stk_lo[st.stk_n + 1] = lo;
            stk_hi[st.stk_n + 1] = mid;
            st.stk_n += 2;
          }
        }
        block_sync();
        continue;
      }
      const uint64_t base = st.excl + written;
      {
        uint32_t rank2[kRankRegs];
        if (wid > 0) {
          if (t == 32) {
            range_s[0] = lo;
            range_s[1] = hi;
          }
          K lo2;
          int sh2;
          uint32_t NB2;
          bucket_slots<KW>(tb_, cap_slots, dn2, range_s, hist, idx, wtmp, big_s, &st.big_n, lo2, sh2, NB2,
                           &b.meta->status);
          rank_slots<KW>(tb_, idx, idx, dn2, hist, NB2, lo2, sh2, big_s, st.big_n, rank2, nullptr);
        }
        block_sync();
        if (wid > 0) emit_slots<KW>(tb_, idx, dn2, rank2, base, b.out_keys, b.out_counts, s.cap, &b.meta->status);
      }
      written += dn2;
      block_sync();
    }
    if (one_batch) discard_runs(src, nr);
#pragma unroll
    for (int dd = 16; dd > 0; dd >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, dd);
    if (lane == 0) wtmp[wid] = sp;
    block_sync();
    if (t == 0) {
      uint64_t tot = 0;
      for (int w = 0; w < kCountThreads / 32; ++w) tot += wtmp[w];
      if (tot) {
        if (tot > 0xffffffffull) atomicOr(&b.meta->status, ST_COUNT_OVERFLOW);
        if (st.excl + written < s.cap) {
          store_key(b.out_keys, st.excl + written, EMPTY);
          b.out_counts[st.excl + written] = (uint32_t)tot;
        } else {
          atomicOr(&b.meta->status, ST_INTERNAL);
        }
        ++written;
      }
      if (!(s.withhold && g == 0)) st_status(&b.look[g], kLookIncl | (st.excl + written));
      b.fhist[g] = (uint32_t)written;
      prefetch();
    }
    block_sync();
    mark(6);
  }
};

template <int KW, bool MERGE>
__device__ __forceinline__ void phase2_body(const Shape& s, const Buffers& b, uint32_t bid) {
  typedef typename KeyT<KW>::T K;
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ P2State st;
  __shared__ uint32_t wtmp[32];
  __shared__ K red_lo[32], red_hi[32];
  __shared__ K stk_lo[160], stk_hi[160];
  __shared__ K range_s[2];
  __shared__ uint32_t big_s[kBigMax];
  const int P1 = 1 << s.b1;
  uint32_t* persist = reinterpret_cast<uint32_t*>(sm + phase2_area(KW, s.bT_max));
  Phase2<KW, MERGE> p{s, b, sm, st, wtmp};
  p.tstart_s = persist;
  p.tsplit_s = persist + max_coarse(KW) + kStageLag + 1;
  p.run_st = persist + 2 * (max_coarse(KW) + kStageLag) + 1;
  p.run_len = p.run_st + kRunBatch;
  p.run_pre = p.run_len + kRunBatch;
  p.red_lo = red_lo;
  p.red_hi = red_hi;
  p.range_s = range_s;
  p.stk_lo = stk_lo;
  p.stk_hi = stk_hi;
  p.big_s = big_s;
  p.slots = b.stage + (size_t)bid * s.n_slots * s.stage_bytes;
  p.P1 = P1;
  p.cap_slots = 1u << s.bT_max;
  p.dcap = (3u * p.cap_slots) >> 2;
  const uint32_t t = threadIdx.x;
  if (bid >= s.n_stage || s.b1 > max_coarse_log2(KW) || s.n_slots < 1 || s.n_slots > (uint32_t)kMaxSlots) {
    if (t == 0) atomicOr(&b.meta->status, ST_INTERNAL);
    return;
  }
  for (int i = t; i <= P1 + kStageLag; i += kCountThreads) p.tstart_s[i] = b.tstart[i];
  for (int i = t; i < P1 + kStageLag; i += kCountThreads) p.tsplit_s[i] = b.tsplit[i];
  if (t == 0) {
    st.pend_head = 0;
    st.pend_n = 0;
    st.one = 1;
    for (int i = 0; i < 8; ++i) st.acc[i] = st.tally[i] = 0;
    st.tmark = clock64();
  }
  block_sync();
  if (t == 0) p.prefetch();
  while (true) {
    block_sync();
    const uint32_t kind = st.nx_kind;
    if (kind == TASK_DONE) break;
    const uint32_t c = st.nx_c, i = st.nx_i, m = st.nx_m, ulo = st.nx_ulo, uhi = st.nx_uhi;
    const uint64_t cs = st.nx_cs, ce = st.nx_ce, tb = st.nx_tb, g = st.nx_g;
    block_sync();  // the task is read: thread 0 may prepare the next one
    p.mark(7);
    if (kind == TASK_SPLIT) p.split(c, i, cs, ce, m, tb);
    else p.count(c, i, g, cs, ce, tb, ulo, uhi);
    while (p.finalize(false)) {  // the waiting runs whose prefix is known by now
    }
  }
  while (st.pend_n) p.finalize(true);
  p.mark(7);
  if (s.profile && t == 0) {
    for (int i = 0; i < 8; ++i) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&b.meta->phase_cycles[i]), st.acc[i]);
      atomicAdd(reinterpret_cast<unsigned long long*>(&b.meta->sub_cycles[i]), st.tally[i]);
    }
  }
}

template <int KW, bool MERGE = false>
__global__ void __launch_bounds__(kCountThreads, 1) k_phase2(Shape s, Buffers b) {
  phase2_body<KW, MERGE>(s, b, blockIdx.x);
}
template <int KW>
__global__ void __launch_bounds__(kCountThreads, 1) k_phase2_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  phase2_body<KW, false>(d.s, d.b, bid);
}

// ------------------------------------------------------------------ final: the output size
// Exclusive scan of the distinct counts of the fine partitions (one block of 1024
// threads): every look-back word must hold its partition's inclusive prefix, and the total
// is the number of distinct keys.
__device__ __forceinline__ void scan_distinct_body(const Shape& sh, const Buffers& b) {
  __shared__ uint64_t wt[32];
  __shared__ uint64_t carry_s;
  const uint64_t NF = min(b.meta->n_fine, sh.nf_max);
  const int t = threadIdx.x, nt = blockDim.x, lane = t & 31, wid = t >> 5;
  if (t == 0) carry_s = 0;
  __syncthreads();
  bool bad = false;
  for (uint64_t base = 0; base < NF; base += (uint64_t)nt * 8) {
    uint32_t v[8];
    unsigned long long lk[8];
    uint64_t s = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const uint64_t i = base + (uint64_t)t * 8 + m;
      v[m] = i < NF ? b.fhist[i] : 0;
      lk[m] = i < NF ? ld_status(&b.look[i]) : 0;
      s += v[m];
    }
    uint64_t x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t xs = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += xs;
    }
    if (lane == 31) wt[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint64_t w = wt[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t ws = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= d) w += ws;
      }
      wt[lane] = w;
    }
    __syncthreads();
    uint64_t run = carry_s + x - s + (wid ? wt[wid - 1] : 0);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const uint64_t i = base + (uint64_t)t * 8 + m;
      if (i < NF) {
        run += v[m];
        bad |= lk[m] != (kLookIncl | run);
      }
    }
    __syncthreads();
    if (t == 0) carry_s += wt[31];
    __syncthreads();
  }
  if (bad) atomicOr(&b.meta->status, ST_INTERNAL);
  if (t == 0) b.meta->n_distinct = carry_s;
}
__global__ void __launch_bounds__(1024) k_scan_distinct(Shape sh, Buffers b) { scan_distinct_body(sh, b); }
__global__ void __launch_bounds__(1024) k_scan_distinct_batch(BatchTab t) {
  KC_BATCH_PROLOGUE(t);
  scan_distinct_body(d.s, d.b);
}

// ------------------------------------------------------------------ launches
constexpr size_t kScatterStaticSmem = 9216;  // pass B's static shared memory (batched form included), rounded up
static size_t scatter_smem(int kw, int nt, int P1, bool keep_c) {
  const size_t sub = (size_t)nt * (kw == 1 ? 32 : 16);
  return sub * (size_t)(kw * 8) + (size_t)P1 * 8 + 2 * padded_len(P1) * 4 + (keep_c ? sub * 4 : 0);
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
  KC_SET(k_phase2<1>);
  KC_SET(k_phase2<2>);
  KC_SET((k_phase2<1, true>));
  KC_SET((k_phase2<2, true>));
  KC_SET(k_bucket_scan);
  KC_SET(k_pack_count_batch<1>);
  KC_SET(k_pack_count_batch<2>);
  KC_SET((k_scatter_batch<1, 256, false>));
  KC_SET((k_scatter_batch<2, 256, false>));
  KC_SET((k_scatter_batch<1, 256, true>));
  KC_SET((k_scatter_batch<2, 256, true>));
  KC_SET(k_fine_plan_batch);
  KC_SET(k_phase2_batch<1>);
  KC_SET(k_phase2_batch<2>);
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

int launch_phase2(const Shape& s, const Buffers& b, int n_sms, void* stream, const Marker& mark) {
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
      k_direct_cursors<<<(P1 + 255) / 256, 256, 0, st>>>(b.cstart, reinterpret_cast<unsigned long long*>(b.toff), P1);
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
  k_fine_plan<<<1, 1024, (size_t)(P1 + kStageLag + 1) * 8, st>>>(s, b);
  ++launches;
  KC_STEP("k_fine_plan");
  // the persistent split + count kernel: one block per SM (at most one per stage slot)
  const unsigned gp = (unsigned)(s.n_stage < (uint32_t)n_sms ? s.n_stage : (uint32_t)n_sms);
  const size_t smC = phase2_smem(s.kw, s.bT_max);
  if (s.aggr & kAggrWarpMerge) {
    if (s.kw == 1) k_phase2<1, true><<<gp, kCountThreads, smC, st>>>(s, b);
    else k_phase2<2, true><<<gp, kCountThreads, smC, st>>>(s, b);
  } else if (s.kw == 1) {
    k_phase2<1><<<gp, kCountThreads, smC, st>>>(s, b);
  } else {
    k_phase2<2><<<gp, kCountThreads, smC, st>>>(s, b);
  }
  ++launches;
  KC_STEP("k_phase2");
  k_scan_distinct<<<1, 1024, 0, st>>>(s, b);
  ++launches;
  KC_STEP("k_scan_distinct");
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
    case BK_PHASE2: {
      const double share = bases_total ? (double)s.L / (double)bases_total : 1.0;
      const uint64_t cap = nsm < s.n_stage ? nsm : s.n_stage;
      return clampu((uint64_t)(2.0 * (double)nsm * share + 0.999), 1, cap);
    }
    default: return 1u;  // one block per count: bucket scan, fine plan, scan of distinct counts
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
    KC_BLAUNCH(BK_PACK, (k_pack_count_batch<1><<<bp.grid[BK_PACK], kPackThreads, (size_t)P1 * 4, st>>>(tab(BK_PACK))),
               "k_pack_count");
  } else {
    KC_BLAUNCH(BK_PACK, (k_pack_count_batch<2><<<bp.grid[BK_PACK], kPackThreads, (size_t)P1 * 4, st>>>(tab(BK_PACK))),
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
  KC_BLAUNCH(BK_FINE_PLAN,
             (k_fine_plan_batch<<<bp.grid[BK_FINE_PLAN], 1024, (size_t)(P1 + kStageLag + 1) * 8, st>>>(
                 tab(BK_FINE_PLAN))),
             "k_fine_plan");
  const size_t smC = phase2_smem(bp.kw, s0.bT_max);
  if (bp.kw == 1) {
    KC_BLAUNCH(BK_PHASE2, (k_phase2_batch<1><<<bp.grid[BK_PHASE2], kCountThreads, smC, st>>>(tab(BK_PHASE2))),
               "k_phase2");
  } else {
    KC_BLAUNCH(BK_PHASE2, (k_phase2_batch<2><<<bp.grid[BK_PHASE2], kCountThreads, smC, st>>>(tab(BK_PHASE2))),
               "k_phase2");
  }
  KC_BLAUNCH(BK_SCAN_DISTINCT,
             (k_scan_distinct_batch<<<bp.grid[BK_SCAN_DISTINCT], 1024, 0, st>>>(tab(BK_SCAN_DISTINCT))),
             "k_scan_distinct");
#undef KC_BLAUNCH
  return launches;
}

}  // namespace kc

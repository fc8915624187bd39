// kc_internal.h - declarations shared by the kernels and the host orchestration.
//
// Data layout in device memory (one kc_count call):
//   codes64[w]   bases 32w .. 32w+31 as 2-bit codes (A0 C1 G2 T3), first base in
//                the two most significant bits (Algorithm 1's kmer << 2 order).
//   inv32[w]     bit i set iff byte 32w+i is not one of ACGTacgt, or lies past
//                the end of the input.
//   hist[t][c]   phase-1 histogram: valid windows of tile t in coarse partition c.
//   toff[t][c]   write offset of tile t inside partition c (bucket-major scan).
//   kbuf         keys grouped by coarse partition (the owner partition of
//                Algorithm 3's AsyncAdd, here a key range so that outputs concatenate
//                in sorted order).
//   sbuf         the same keys regrouped by fine partition inside each coarse one.
//   out keys / counts   the sorted histogram.
#pragma once
#include <stdint.h>

namespace kc {

constexpr int kWordBases = 32;                 // bases per packed code word
constexpr int kTileWords = 8192;               // one phase-1 tile = 262144 bases
constexpr uint64_t kTileBases = (uint64_t)kTileWords * kWordBases;
constexpr int kPackThreads = 512;              // pass A: one code word per thread per sub-step
constexpr int kMaxCoarseLog2 = 12;             // at most 4096 coarse partitions
constexpr int kMaxFine = 4096;                 // at most this many fine partitions per coarse one
// bases per coarse partition aimed at when the plan sets no partition count
constexpr uint64_t coarse_bases(int kw) { return kw == 1 ? (12ull << 20) : (6ull << 20); }
// count kernel: threads per block and blocks per SM (one block of 1024 threads with
// 8192-slot tables, or two of 512 threads with 4096-slot tables)
#ifndef KC_COUNT_THREADS
#define KC_COUNT_THREADS 1024
#endif
constexpr int kCountThreads = KC_COUNT_THREADS;
constexpr int kCountBlocksPerSM = 1024 / kCountThreads;
static_assert(kCountThreads == 1024 || kCountThreads == 512, "count blocks of 1024 or 512 threads");
constexpr int kFineChunk1 = 8192;              // fine-scatter chunk, 64-bit keys
constexpr int kFineChunk2 = 4096;              // fine-scatter chunk, 128-bit keys
constexpr int kFineLocalCap = 2048;            // fine partitions one chunk may span (shared histogram)
constexpr int kHllLog2 = 10;                   // distinct-key sketch: 1024 registers
constexpr int kHllRegs = 1 << kHllLog2;
constexpr int kHllSampleLog2 = 6;              // ... over a 1/64 hash sample of the keys (a rarer sample
                                               // leaves pass B's warps out of the sketch update more often)
constexpr double kHllSample = 64.0;
constexpr uint32_t kLookbackSpinLimit = 1u << 22;  // x ~100 ns sleep: ~0.4 s, then give up
constexpr uint32_t kTestSpinLimit = 64;            // the same wait when a test withholds a prefix
constexpr uint32_t kTestCountLimit = 0xffff;       // the count limit when a test lowers it
// Fine layout from a sample: the fine histogram counts one 4096-key chunk in 2^kFineSampleLog2
// and sizes each fine partition's region from that estimate plus slack; for counts of at
// least kFineSampledMinBases bases (smaller ones take the exact histogram).
constexpr int kFineSampleLog2 = 3;
constexpr uint64_t kFineSampledMinBases = 1ull << 26;

// status bits written by kernels (a kc_status is derived from them on the host)
enum : uint32_t {
  ST_COUNT_OVERFLOW = 1u,   // a count exceeded 2^32 - 1
  ST_TIMEOUT = 2u,          // a bounded wait gave up
  ST_BAD_OFFSETS = 4u,      // offsets not non-decreasing
  ST_INTERNAL = 8u,         // an internal consistency check failed
  ST_PARTITION_OVERFLOW = 16u,  // a coarse partition holds 2^32 keys or more
};

// Values the host reads back at the end of a call.
struct Meta {
  uint64_t n_windows;   // K: valid windows
  uint64_t n_distinct;  // D
  uint64_t n_fine;      // number of fine partitions
  uint64_t n_overflow;  // fine partitions that took the overflow path
  uint64_t n_deferred;  // fine partitions written out by k_compact (prefix unknown in time)
  uint32_t status;
  uint32_t fine_spill;  // the sampled fine layout overflowed a region: the exact fine split ran
  uint64_t ticket;      // phase-2 work counter
  uint64_t d_estimate;  // distinct keys estimated by the sketch
  uint64_t sub_cycles[8];    // profiled plans only: ordering sub-steps (range, rank, scan, place, small sorts, big sorts, #big)
  uint64_t phase_cycles[8];  // profiled plans only: SM cycles per phase of k_count_emit, summed over CTAs
};

struct Shape {
  uint64_t L;           // bases
  uint64_t n_reads;
  uint64_t n_words;     // ceil(L / 32)
  uint64_t n_tiles;     // ceil(n_words / kTileWords)
  int k;
  int canonical;
  int kw;               // key words: 1 or 2
  int b1;               // log2 coarse partitions
  int bT_max;           // log2 of the largest table
  int tail;             // table slots past the home range (linear probing never wraps)
  uint32_t fine_target; // keys per fine partition aimed for
  uint64_t cap;         // capacity of kbuf / sbuf / outputs in keys
  uint64_t nf_max;      // capacity of the fine-partition arrays
  uint64_t smem_budget; // opt-in shared memory per block
  uint32_t spin_limit;  // iterations of a bounded device wait before it gives up
  uint32_t count_limit; // largest count reported (2^32 - 1; lower only when a test asks)
  uint64_t cap_kb;      // capacity of kbuf / sbuf in keys (cap, plus the slack of a sampled fine layout)
  int fine_sampled;     // nonzero: fine partition regions sized from a sample of the keys
  int tight_slack;      // nonzero (testing): sampled regions get no slack
  int profile;          // nonzero: k_count_emit accumulates per-phase cycle counts
  int defer_all;        // nonzero (testing): every fine partition takes the deferred write-out
  int withhold;         // nonzero (testing): partition 0 never publishes its prefix
  int aggr;             // aggregation variants: kAggr* bits (single-count path only)
};
constexpr int kAggrNoSmemBuckets = 1;  // pass B writes every key on its own (global atomic cursor)
constexpr int kAggrWarpMerge = 2;      // the count kernel adds a warp's equal keys with one atomic

struct Buffers {
  const uint8_t* reads;
  const uint64_t* offsets;
  uint64_t* codes64;
  uint32_t* inv32;
  uint64_t* tile_first;   // first read index whose start is >= the tile's halo start
  uint32_t* hist;         // [n_tiles][P1]
  uint64_t* toff;         // [n_tiles][P1]
  uint64_t* cstart;       // [P1 + 1] coarse partition starts
  uint32_t* fine_base;    // [P1 + 1] first fine index of each coarse partition
  uint32_t* fine_m;       // [P1] fine partitions of each coarse partition
  uint32_t* hll;          // [kHllRegs] distinct-key sketch (max-merged by pass B)
  uint32_t* fhist;        // [nf_max] keys per fine partition (fine split); then distinct keys | deferred bit 31
  uint64_t* foff;         // [nf_max + 1] fine partition starts
  uint32_t* flo;          // [nf_max + 1] first range-map value u of each fine partition (0 after the last)
  unsigned long long* fcur;  // [nf_max] fine scatter cursors
  unsigned long long* look;  // [nf_max] look-back status words
  uint64_t* kbuf;
  uint64_t* sbuf;
  uint64_t* out_keys;
  uint32_t* out_counts;
  Meta* meta;
};

// One count of a batch: its shape and its buffers (inside the batch's scratch arena).
struct BatchDesc {
  Shape s;
  Buffers b;
};

// A batched launch of one kernel: block x works for count blk2s[x] as its block
// x - start[blk2s[x]] of start[i + 1] - start[i].
struct BatchTab {
  const BatchDesc* desc;
  const uint32_t* blk2s;
  const uint32_t* start;
};

// The counts of a batch, laid out for the batched launches (host side; the device copy of
// descriptors and tables is at `dev`).
struct BatchPlan {
  int n = 0;
  int kw = 1;
  int P1_max = 1;
  int sampled = 0;                  // some count has a sampled fine layout (the exact split may follow)
  const BatchDesc* host = nullptr;  // n descriptors
  const BatchDesc* desc = nullptr;  // device copy
  // per kernel: device block->count table and block starts (n + 1), and the grid
  const uint32_t* blk2s[16] = {};
  const uint32_t* start[16] = {};
  uint32_t grid[16] = {};
};
enum BatchKernel {
  BK_CLEAR, BK_CHECK, BK_TILE_FIRST, BK_PACK, BK_COL_SCAN, BK_BUCKET_SCAN, BK_SCATTER, BK_FINE_PLAN, BK_FINE_HIST,
  BK_FINE_SCAN, BK_FINE_SCATTER, BK_COUNT, BK_SCAN_DISTINCT, BK_COMPACT, BK_N
};

// Called after every kernel launch with the kernel's name (used for per-kernel timing).
struct Marker {
  void (*fn)(void* ctx, const char* name) = nullptr;
  void* ctx = nullptr;
  void operator()(const char* name) const {
    if (fn) fn(ctx, name);
  }
};

// Host launch wrappers (kc_kernels.cu).  Each returns the number of kernel launches, or
// -cudaError_t if a launch failed (no later kernel is launched then).
int launch_phase1(const Shape& s, const Buffers& b, int n_sms, void* stream, const Marker& mark);
int launch_phase2(const Shape& s, const Buffers& b, int n_sms, uint32_t nf_max, void* stream, const Marker& mark);
// Blocks each kernel of a batched launch gives one count (host rule, shared by the planner
// and the launcher), and the whole batched launch sequence (returns launches or
// -cudaError_t).
uint32_t batch_blocks(BatchKernel k, const Shape& s, int n_sms, uint64_t bases_total);
int launch_batch(const BatchPlan& bp, int n_sms, void* stream, const Marker& mark);
int configure_kernels(int device);  // sets shared-memory attributes; returns 0 or a cudaError_t

size_t count_kernel_smem(int kw, int bT_max, int tail);
void set_error_message(const char* msg);  // the text kc_last_error returns on this thread
int table_log2_max(int kw, size_t smem_optin, size_t smem_per_sm);

// Shape and scratch layout of one count (host only; shared by kc_count, the batched and
// submitted forms and kc_count_noalloc, so that all make the same choices).
struct ShapeOpts {
  uint32_t p_hint = 0;      // coarse partitions (power of two) or 0
  float load = 0.55f;       // table load aimed at per fine partition
  uint32_t slots_max = 0;   // largest count table (slots) or 0
  size_t smem_optin = 0;
  size_t smem_per_sm = 0;   // shared memory of one SM (for the count blocks it holds)
  int profile = 0, defer_all = 0, withhold = 0, low_count_limit = 0, aggr = 0;
  int allow_sampled = 0;   // a single count: the fine layout may be sized from a sample
  int force_sampled = 0;   // testing: sampled at any size
  int tight_slack = 0;     // testing: sampled regions get no slack
};
struct Layout {  // byte offsets into the count's scratch block
  size_t reads, offs, codes, inv, tf, hist, toff, cst, fb, fm, hll, fh, fo, flo, fc, look, kbuf, sbuf, meta;
  size_t total;
};
// Fills s and lay for L bases and n_reads reads; copy_reads / copy_offs: the scratch holds a
// copy of the reads (L + 16 bytes) / the offsets.  Returns the fine-partition capacity.
uint32_t make_shape(const ShapeOpts& o, uint64_t L, uint64_t n_reads, int k, int canonical, bool copy_reads,
                    bool copy_offs, Shape& s, Layout& lay);
// The scratch-held buffers at ws (reads, offsets and outputs are the caller's to set when
// they are not copies).
Buffers layout_buffers(const Layout& lay, uint8_t* ws);
// Enqueue the clears every count starts from on `stream` (a cudaStream_t); returns a
// cudaError_t.
int clear_scratch(const Shape& s, const Buffers& b, void* stream);

}  // namespace kc

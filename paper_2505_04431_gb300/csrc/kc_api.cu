// kc_api.cu - the C ABI declared in include/kc.h: plans, scratch memory, argument
// checks, the phase-1 / phase-2 launch sequence and error reporting.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <unordered_map>
#include <vector>

#include "kc.h"
#include "kc_internal.h"

namespace {

thread_local std::string g_err;

kc_status fail(kc_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
kc_status cuda_fail(cudaError_t e, const char* what) {
  return fail(KC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct AsyncJob;  // a count submitted with kc_submit

// The result buffers of a group of batched counts, shared by the group's results and
// released with the last of them.
struct GroupOwner {
  void* keys = nullptr;
  void* counts = nullptr;
  std::atomic<int> refs{0};
};

// Scratch arena of one group of batched counts (their scratch side by side)
constexpr size_t kBatchArenaBytes = 16ull << 30;

}  // namespace

namespace kc {
void set_error_message(const char* msg) { g_err = msg ? msg : ""; }

static int ceil_log2_u64(uint64_t v) { return v <= 1 ? 0 : 64 - __builtin_clzll(v - 1); }

uint32_t make_shape(const ShapeOpts& o, uint64_t L, uint64_t n_reads, int k, int canonical, bool copy_reads,
                    bool copy_offs, Shape& s, Layout& lay) {
  s = Shape{};
  s.L = L;
  s.n_reads = n_reads;
  s.n_words = (L + 31) / 32;
  s.n_tiles = (s.n_words + kTileWords - 1) / kTileWords;
  s.k = k;
  s.canonical = canonical ? 1 : 0;
  s.kw = k <= 32 ? 1 : 2;
  int b1;
  if (o.p_hint) {
    b1 = ceil_log2_u64(o.p_hint);
  } else {
    // coarse partitions of at most about 12 Mi windows (64-bit keys) or 6 Mi (128-bit keys):
    // few enough partitions that pass B's per-partition runs stay long, small enough that a
    // partition of distinct keys splits into at most ~2800 (64-bit) or ~1400 (128-bit) fine
    // partitions of one table each, within kMaxFine (measured on GB300: 256 coarse
    // partitions for 3 G bases of 64-bit keys beat 512 and 128)
    const int want = ceil_log2_u64(L / coarse_bases(s.kw) + 1);
    b1 = want < 11 ? want : 11;
  }
  s.b1 = b1;
  const uint64_t P1 = 1ull << b1;
  int bT_max = table_log2_max(s.kw, o.smem_optin, o.smem_per_sm);
  if (o.slots_max) {
    const int bt = 63 - __builtin_clzll((uint64_t)o.slots_max);
    if (bt < bT_max) bT_max = bt;
  }
  s.bT_max = bT_max;
  s.tail = bT_max >= 10 ? 1024 : (1 << bT_max);
  const double ft = (double)(1u << bT_max) * o.load;  // distinct keys per fine partition aimed at
  s.fine_target = ft < 16 ? 16u : (uint32_t)ft;
  s.cap = L > 0 ? L : 1;
  // sum over partitions of ceil(n_c / target), target >= fine_target: at most K / ft + P1
  const uint64_t nf_bound = s.cap / s.fine_target + P1 + 1;
  const uint64_t nf_lim = P1 * kMaxFine;
  s.nf_max = nf_bound < nf_lim ? nf_bound : nf_lim;
  // a sampled fine layout: regions hold their estimate plus slack (about a fifth of the keys
  // in all, and at least 16 keys each); a layout that does not fit falls back to the exact one
  s.fine_sampled = o.allow_sampled && (o.force_sampled || L >= kFineSampledMinBases) ? 1 : 0;
  s.tight_slack = o.tight_slack;
  s.cap_kb = s.fine_sampled ? s.cap + s.cap / 4 + s.nf_max * 64 : s.cap;
  s.smem_budget = o.smem_optin;
  s.spin_limit = o.withhold ? kTestSpinLimit : kLookbackSpinLimit;
  s.count_limit = o.low_count_limit ? kTestCountLimit : 0xffffffffu;
  s.profile = o.profile;
  s.defer_all = o.defer_all;
  s.withhold = o.withhold;
  s.aggr = o.aggr;
  const uint64_t nf = s.nf_max;
  size_t at = 0;
  auto take = [&](size_t bytes) {
    const size_t o_ = at;
    at = (at + (bytes ? bytes : 1) + 255) / 256 * 256;
    return o_;
  };
  lay.reads = take(copy_reads ? L + 16 : 0);
  lay.offs = take(copy_offs ? (n_reads + 1) * 8 : 0);
  lay.codes = take(s.n_words * 8);
  lay.inv = take(s.n_words * 4);
  lay.tf = take(s.n_tiles * 8);
  lay.hist = take(s.n_tiles * P1 * 4);
  lay.toff = take(s.n_tiles * P1 * 8);
  lay.cst = take((P1 + 1) * 8);
  lay.fb = take((P1 + 1) * 4);
  lay.fm = take(P1 * 4);
  lay.hll = take((size_t)kHllRegs * 4);
  lay.fh = take(nf * 4);
  lay.fo = take((nf + 1) * 8);
  lay.flo = take((nf + 1) * 4);
  lay.fc = take(nf * 8);
  lay.look = take(nf * 8);
  lay.kbuf = take(s.cap_kb * s.kw * 8);
  lay.sbuf = take(s.cap_kb * s.kw * 8);
  lay.meta = take(sizeof(Meta));
  lay.total = at;
  return (uint32_t)nf;
}

Buffers layout_buffers(const Layout& lay, uint8_t* ws) {
  Buffers b{};
  b.reads = (const uint8_t*)(ws + lay.reads);
  b.offsets = (const uint64_t*)(ws + lay.offs);
  b.codes64 = (uint64_t*)(ws + lay.codes);
  b.inv32 = (uint32_t*)(ws + lay.inv);
  b.tile_first = (uint64_t*)(ws + lay.tf);
  b.hist = (uint32_t*)(ws + lay.hist);
  b.toff = (uint64_t*)(ws + lay.toff);
  b.cstart = (uint64_t*)(ws + lay.cst);
  b.fine_base = (uint32_t*)(ws + lay.fb);
  b.fine_m = (uint32_t*)(ws + lay.fm);
  b.hll = (uint32_t*)(ws + lay.hll);
  b.fhist = (uint32_t*)(ws + lay.fh);
  b.foff = (uint64_t*)(ws + lay.fo);
  b.flo = (uint32_t*)(ws + lay.flo);
  b.fcur = (unsigned long long*)(ws + lay.fc);
  b.look = (unsigned long long*)(ws + lay.look);
  b.kbuf = (uint64_t*)(ws + lay.kbuf);
  b.sbuf = (uint64_t*)(ws + lay.sbuf);
  b.meta = (Meta*)(ws + lay.meta);
  return b;
}

int clear_scratch(const Shape& s, const Buffers& b, void* stream) {
  const cudaStream_t st = (cudaStream_t)stream;
  const size_t P1 = (size_t)1 << s.b1;
  cudaError_t e;
  if ((e = cudaMemsetAsync(b.meta, 0, sizeof(Meta), st)) != cudaSuccess) return (int)e;
  if ((e = cudaMemsetAsync(b.fhist, 0, (size_t)s.nf_max * 4, st)) != cudaSuccess) return (int)e;
  if ((e = cudaMemsetAsync(b.hll, 0, (size_t)kHllRegs * 4, st)) != cudaSuccess) return (int)e;
  if ((e = cudaMemsetAsync(b.look, 0, (size_t)s.nf_max * 8, st)) != cudaSuccess) return (int)e;
  return (int)cudaMemsetAsync(b.cstart, 0, (P1 + 1) * 8, st);
}
}  // namespace kc

struct kc_plan_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  kc_alloc_fn alloc = nullptr;
  kc_free_fn free_ = nullptr;
  void* ctx = nullptr;
  uint64_t max_bytes = 0;
  uint32_t p_hint = 0;
  float load = 0.5f;
  uint32_t slots_max = 0;
  int n_sms = 0;
  size_t smem_optin = 0;
  size_t smem_per_sm = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // batched counts: scratch arena of a group of counts, device and pinned host tables
  void* bws = nullptr;
  size_t bws_bytes = 0;
  void* btab = nullptr;
  size_t btab_bytes = 0;
  void* btab_host = nullptr;
  size_t btab_host_bytes = 0;
  struct kc::Meta* bmeta = nullptr;  // kc_count_batch: pinned status records
  uint32_t bmeta_n = 0;
  // kc_submit_batch: pinned staging of the tables, each buffer reused once its copy is done
  static constexpr int kStaging = 8;
  struct Staging {
    void* host = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;
  } stg[kStaging];
  int stg_next = 0;
  // submitted counts (kc_submit): jobs in flight and their pinned status records
  std::unordered_map<uint64_t, AsyncJob*> jobs;
  // transfer stream of submitted counts: host inputs in, results out to host buffers, so
  // that these copies overlap the counts queued before and after them on `stream`
  cudaStream_t xfer = nullptr;
  uint64_t next_job = 1;
  static constexpr int kPinned = 4096;
  struct kc::Meta* pinned = nullptr;
  std::vector<int> pinned_free;
  std::atomic<int> busy{0};
  kc_stats stats{};
  // per-kernel timing (KC_PLAN_PROFILE)
  bool profile = false;
  bool defer_all = false;
  bool withhold = false;
  bool low_count_limit = false;
  bool force_sampled = false;
  bool tight_slack = false;
  bool small_arena = false;
  int aggr = 0;
  static constexpr int kMaxMarks = 32;
  cudaEvent_t ev[kMaxMarks + 1] = {};
  const char* ev_name[kMaxMarks] = {};
  int n_marks = 0;
  float kernel_ms[kMaxMarks] = {};
  int n_kernel_ms = 0;
};

namespace {

// Device memory for use on stream `st` (the plan's stream unless stated): a block is only
// ever written by work on the stream it was allocated for, or by work ordered after that
// stream's use of it, and it is freed on that stream once the host has seen that work end.
void* dev_alloc_on(kc_plan_s* p, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 256;
  if (p->alloc) return p->alloc(bytes, (void*)st, p->ctx);
  void* ptr = nullptr;
  if (cudaMallocAsync(&ptr, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return ptr;
}
void dev_free_on(kc_plan_s* p, void* ptr, cudaStream_t st) {
  if (!ptr) return;
  if (p->free_) p->free_(ptr, (void*)st, p->ctx);
  else cudaFreeAsync(ptr, st);
}
void* dev_alloc(kc_plan_s* p, size_t bytes) { return dev_alloc_on(p, bytes, p->stream); }
void dev_free(kc_plan_s* p, void* ptr) { dev_free_on(p, ptr, p->stream); }

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct ScopedBusy {
  kc_plan_s* p;
  bool ok;
  explicit ScopedBusy(kc_plan_s* pl) : p(pl) {
    int z = 0;
    ok = p->busy.compare_exchange_strong(z, 1);
  }
  ~ScopedBusy() {
    if (ok) p->busy.store(0);
  }
};

void record_mark(void* ctx, const char* name) {
  kc_plan_s* p = (kc_plan_s*)ctx;
  if (p->n_marks >= kc_plan_s::kMaxMarks) return;
  p->ev_name[p->n_marks] = name;
  cudaEventRecord(p->ev[p->n_marks + 1], p->stream);
  ++p->n_marks;
}

// Diagnostics (environment variable KC_DEBUG_SYNC set): wait for every kernel as soon as it
// is launched and report it on stderr, so that a kernel that does not finish is named.
void debug_mark(void* ctx, const char* name) {
  kc_plan_s* p = (kc_plan_s*)ctx;
  fprintf(stderr, "[kc] %s launched\n", name);
  const cudaError_t e = cudaStreamSynchronize(p->stream);
  fprintf(stderr, "[kc] %s finished: %s\n", name, cudaGetErrorString(e));
}


// ---- one count: shape and scratch layout (host only), launch sequence, result
struct Job {
  kc::Shape s{};
  kc::Layout lay{};
  int P1 = 1;
  uint32_t nf_max = 0;
  uint64_t L = 0, n_reads = 0;
  bool off_dev = false, copy_reads = false, reads_dev = false;
  // host inputs of a submitted count, copied on the transfer stream into a buffer of the
  // job's own (not the plan's scratch) so that the copy may run while earlier counts do
  bool stage_r = false, stage_o = false;
  const uint8_t* reads = nullptr;
  const uint64_t* offsets = nullptr;
  const uint8_t* stage_reads = nullptr;
  const uint64_t* stage_offs = nullptr;
  size_t ws_bytes = 0, out_key_bytes = 0, out_cnt_bytes = 0;
  void* okeys = nullptr;
  void* ocnts = nullptr;
};

kc::ShapeOpts shape_opts(const kc_plan_s* p) {
  kc::ShapeOpts o;
  o.p_hint = p->p_hint;
  o.load = p->load;
  o.slots_max = p->slots_max;
  o.smem_optin = p->smem_optin;
  o.smem_per_sm = p->smem_per_sm;
  o.profile = p->profile ? 1 : 0;
  o.defer_all = p->defer_all ? 1 : 0;
  o.withhold = p->withhold ? 1 : 0;
  o.low_count_limit = p->low_count_limit ? 1 : 0;
  o.force_sampled = p->force_sampled ? 1 : 0;
  o.tight_slack = p->tight_slack ? 1 : 0;
  o.aggr = p->aggr;
  return o;
}

void plan_job(const kc_plan_s* p, const uint8_t* reads, const uint64_t* offsets, uint64_t n_reads, uint64_t L,
              bool off_dev, int k, int canonical, Job& j, bool stage_host = false, bool sampled_ok = false) {
  j.reads = reads;
  j.offsets = offsets;
  j.n_reads = n_reads;
  j.L = L;
  j.off_dev = off_dev;
  j.reads_dev = L > 0 && is_device_ptr(reads);
  j.copy_reads = L > 0 && (!j.reads_dev || ((uintptr_t)reads & 15) != 0);
  j.stage_r = stage_host && L > 0 && !j.reads_dev;
  j.stage_o = stage_host && !off_dev;
  kc::ShapeOpts o = shape_opts(p);
  o.allow_sampled = sampled_ok ? 1 : 0;
  j.nf_max = kc::make_shape(o, L, n_reads, k, canonical, j.copy_reads && !j.stage_r, !off_dev && !j.stage_o, j.s,
                            j.lay);
  j.P1 = 1 << j.s.b1;
  j.ws_bytes = j.lay.total;
  j.out_key_bytes = j.s.cap * j.s.kw * 8;
  j.out_cnt_bytes = j.s.cap * 4;
}

// The buffers of one count with scratch at `ws` and its outputs at j.okeys / j.ocnts.
kc::Buffers make_buffers(const Job& j, uint8_t* ws) {
  kc::Buffers b = kc::layout_buffers(j.lay, ws);
  if (!j.copy_reads) b.reads = j.reads;
  if (j.stage_r) b.reads = j.stage_reads;
  if (j.off_dev) b.offsets = j.offsets;
  if (j.stage_o) b.offsets = j.stage_offs;
  b.out_keys = (uint64_t*)j.okeys;
  b.out_counts = (uint32_t*)j.ocnts;
  return b;
}

// The input copies of one count (reads that are on the host or misaligned, host offsets).
bool enqueue_copies(const Job& j, const kc::Buffers& b, cudaStream_t st, std::string* err) {
  cudaError_t e;
  if (j.copy_reads && !j.stage_r && (e = cudaMemcpyAsync((void*)b.reads, j.reads, j.L,
                                           j.reads_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st)) != cudaSuccess) {
    *err = std::string("copying reads: ") + cudaGetErrorString(e);
    return false;
  }
  if (!j.off_dev && !j.stage_o &&
      (e = cudaMemcpyAsync((void*)b.offsets, j.offsets, (j.n_reads + 1) * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
    *err = std::string("copying offsets: ") + cudaGetErrorString(e);
    return false;
  }
  return true;
}

// Copies, clears and launches of one count on stream `st` with scratch at `ws`; the
// status record is copied to *meta_dst at the end (asynchronously if it is pinned).
bool enqueue_job(const Job& j, uint8_t* ws, cudaStream_t st, kc::Meta* meta_dst, const kc::Marker& mark, int n_sms,
                 int* launches, std::string* err) {
  const kc::Shape& s = j.s;
  const kc::Buffers b = make_buffers(j, ws);
  if (!enqueue_copies(j, b, st, err)) return false;
  cudaError_t e;
  if ((e = (cudaError_t)kc::clear_scratch(s, b, (void*)st)) != cudaSuccess) {
    *err = std::string("clearing scratch: ") + cudaGetErrorString(e);
    return false;
  }
  int l = kc::launch_phase1(s, b, n_sms, (void*)st, mark);
  if (l >= 0) {
    const int l2 = kc::launch_phase2(s, b, n_sms, j.nf_max, (void*)st, mark);
    l = l2 >= 0 ? l + l2 : l2;
  }
  if (l < 0) {
    *err = std::string("launch: ") + cudaGetErrorString((cudaError_t)(-l));
    return false;
  }
  *launches = l;
  if ((e = cudaMemcpyAsync(meta_dst, b.meta, sizeof(kc::Meta), cudaMemcpyDeviceToHost, st)) != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return false;
  }
  return true;
}

kc_status job_status(const Job& j, const kc::Meta& m, const char* who, std::string* msg) {
  const std::string w(who);
  // the status record must describe a result that fits the buffers of this count
  if (m.n_windows > j.L || m.n_distinct > m.n_windows || m.n_fine > j.nf_max || m.n_deferred > m.n_fine) {
    *msg = w + ": inconsistent status record";
    return KC_ECUDA;
  }
  if (m.status & kc::ST_BAD_OFFSETS) {
    *msg = w + ": offsets must start at 0, be non-decreasing and end at the base count";
    return KC_EINVAL;
  }
  if (m.status & kc::ST_PARTITION_OVERFLOW) {
    *msg = w + ": one key range holds 2^32 windows or more; use more partitions";
    return KC_EOVERFLOW;
  }
  if (m.status & kc::ST_COUNT_OVERFLOW) {
    *msg = w + (j.s.count_limit == 0xffffffffu ? ": a count exceeds 2^32 - 1" : ": a count exceeds the test limit");
    return KC_EOVERFLOW;
  }
  if (m.status & kc::ST_TIMEOUT) {
    *msg = w + ": a device-side wait timed out";
    return KC_ETIMEOUT;
  }
  if (m.status & kc::ST_INTERNAL) {
    *msg = w + ": internal consistency check failed";
    return KC_ECUDA;
  }
  return KC_OK;
}

void fill_result(const Job& j, const kc::Meta& m, kc_result* out) {
  out->n = m.n_distinct;
  out->key_words = (uint32_t)j.s.kw;
  out->keys = j.okeys;
  out->counts = (uint32_t*)j.ocnts;
  out->n_valid_windows = m.n_windows;
  out->capacity = j.s.cap;
}

struct AsyncJob {
  Job j;
  int slot = -1;
  cudaEvent_t ev = nullptr;
  GroupOwner* owner = nullptr;  // a count of a batched group: its results live in the group's buffers
  // staged host inputs (allocated for the transfer stream) and the event after their copy
  void* stage = nullptr;
  cudaEvent_t ev_in = nullptr;
  // host buffers the result goes to (kc_job_copy_to_host), the event after that copy, and
  // the status record kept while it runs
  uint64_t* keys_host = nullptr;
  uint32_t* counts_host = nullptr;
  uint64_t host_cap = 0;
  cudaEvent_t ev_out = nullptr;
  bool copying = false;
  kc::Meta meta{};
};

// drop one reference to a group's result buffers (freed with the last)
void release_owner(kc_plan_s* p, GroupOwner* o) {
  if (o->refs.fetch_sub(1) == 1) {
    dev_free(p, o->keys);
    dev_free(p, o->counts);
    delete o;
  }
}

// release a finished (or failed) job's bookkeeping; with `drop`, its result buffers too
void retire(kc_plan_s* p, uint64_t id, AsyncJob* a, bool drop) {
  if (drop) {
    if (a->owner) {
      release_owner(p, a->owner);
    } else {
      dev_free(p, a->j.okeys);
      dev_free(p, a->j.ocnts);
    }
  }
  if (a->ev) cudaEventDestroy(a->ev);
  if (a->ev_in) cudaEventDestroy(a->ev_in);
  if (a->ev_out) cudaEventDestroy(a->ev_out);
  dev_free_on(p, a->stage, p->xfer);  // the count that read it has ended (its event was seen)
  if (a->slot >= 0) p->pinned_free.push_back(a->slot);
  p->jobs.erase(id);
  delete a;
}

// release a job that failed before its kernels were enqueued: its input copy may be queued
// on the transfer stream, so that stream is drained before the staging buffer goes back
void drop_unsubmitted(kc_plan_s* p, AsyncJob* a) {
  if (a->stage) cudaStreamSynchronize(p->xfer);
  if (a->ev_in) cudaEventDestroy(a->ev_in);
  dev_free_on(p, a->stage, p->xfer);
  delete a;
}

// ---- batched groups (kc_count_batch, kc_submit_batch)
struct Group {
  std::vector<uint32_t> idx;
  std::vector<size_t> ws_off, key_off, cnt_off;
  size_t ws = 0, keys = 0, cnts = 0, tab = 0;
  uint64_t bases = 0;
};
struct GroupPlan {
  std::vector<Group> groups;
  std::vector<uint32_t> alone;  // counts whose scratch is larger than the arena
  size_t need_single = 0, arena = 0, tab_total = 0, tab_max = 0, out_total = 0;
};

// Counts whose scratch fits the arena side by side form a group (taken in order); the
// table bytes of each group (descriptors, block starts and block-to-count maps).
bool plan_groups(const kc_plan_s* p, const std::vector<Job>& jobs, GroupPlan& gp, std::string* err) {
  const size_t arena_cap = p->small_arena ? (32ull << 20)
                           : p->max_bytes   ? std::max<size_t>(p->max_bytes / 4, 1ull << 28)
                                            : kBatchArenaBytes;
  for (uint32_t i = 0; i < (uint32_t)jobs.size(); ++i) {
    const Job& j = jobs[i];
    gp.out_total += j.out_key_bytes + j.out_cnt_bytes;
    const size_t w = align_up(j.ws_bytes, 256);
    if (w > arena_cap) {
      gp.alone.push_back(i);
      gp.need_single = std::max(gp.need_single, j.ws_bytes);
      continue;
    }
    if (gp.groups.empty() || gp.groups.back().ws + w > arena_cap) gp.groups.emplace_back();
    Group& g = gp.groups.back();
    g.idx.push_back(i);
    g.ws_off.push_back(g.ws);
    g.key_off.push_back(g.keys);
    g.cnt_off.push_back(g.cnts);
    g.ws += w;
    g.keys += align_up(j.out_key_bytes, 256);
    g.cnts += align_up(j.out_cnt_bytes, 256);
    g.bases += j.L;
  }
  // a group of one count runs alone: the single-count kernels need no tables
  for (size_t gi = 0; gi < gp.groups.size();) {
    if (gp.groups[gi].idx.size() == 1) {
      const uint32_t i = gp.groups[gi].idx[0];
      gp.alone.push_back(i);
      gp.need_single = std::max(gp.need_single, jobs[i].ws_bytes);
      gp.groups.erase(gp.groups.begin() + gi);
    } else {
      ++gi;
    }
  }
  for (Group& g : gp.groups) {
    gp.arena = std::max(gp.arena, g.ws);
    const uint32_t n = (uint32_t)g.idx.size();
    size_t words = 0;
    for (int k = 0; k < kc::BK_N; ++k) {
      uint64_t sum = 0;
      for (uint32_t q : g.idx) sum += kc::batch_blocks((kc::BatchKernel)k, jobs[q].s, p->n_sms, g.bases);
      if (sum > 0x7fffffffull) {
        *err = "a group needs too many thread blocks";
        return false;
      }
      words += (n + 1) + sum;
    }
    g.tab = align_up(n * sizeof(kc::BatchDesc), 256) + align_up(words * 4, 256);
    gp.tab_total += g.tab;
    gp.tab_max = std::max(gp.tab_max, g.tab);
  }
  return true;
}


// Enqueue one group on the plan's stream: its outputs (two allocations, owned by `o`), the
// descriptors and block tables staged at `h` (pinned) and copied to `dv`, the input copies,
// the batched launches, and each count's status record to meta_dst[q].
bool enqueue_group(kc_plan_s* p, std::vector<Job>& jobs, const Group& g, GroupOwner* o, uint8_t* h, uint8_t* dv,
                   kc::Meta* const* meta_dst, uint32_t* launches, kc_status* stc, std::string* err) {
  const uint32_t n = (uint32_t)g.idx.size();
  o->keys = dev_alloc(p, g.keys);
  o->counts = o->keys ? dev_alloc(p, g.cnts) : nullptr;
  if (!o->keys || !o->counts) {
    *stc = KC_ENOMEM;
    *err = "result allocation failed";
    return false;
  }
  kc::BatchDesc* hd = (kc::BatchDesc*)h;
  int P1_max = 1;
  for (uint32_t q = 0; q < n; ++q) {
    Job& j = jobs[g.idx[q]];
    j.okeys = (uint8_t*)o->keys + g.key_off[q];
    j.ocnts = (uint8_t*)o->counts + g.cnt_off[q];
    hd[q].s = j.s;
    hd[q].b = make_buffers(j, (uint8_t*)p->bws + g.ws_off[q]);
    P1_max = std::max(P1_max, j.P1);
    if (!enqueue_copies(j, hd[q].b, p->stream, err)) {
      *stc = KC_ECUDA;
      return false;
    }
  }
  kc::BatchPlan bp;
  bp.n = (int)n;
  bp.kw = jobs[g.idx[0]].s.kw;
  bp.P1_max = P1_max;
  for (uint32_t q = 0; q < n; ++q) bp.sampled |= jobs[g.idx[q]].s.fine_sampled;
  bp.host = hd;
  bp.desc = (const kc::BatchDesc*)dv;
  const size_t dbytes = align_up(n * sizeof(kc::BatchDesc), 256);
  uint32_t* hw = (uint32_t*)(h + dbytes);
  const uint32_t* dw = (const uint32_t*)(dv + dbytes);
  for (int k = 0; k < kc::BK_N; ++k) {
    uint32_t* start = hw;
    uint32_t* blk2s = hw + n + 1;
    uint32_t at = 0;
    for (uint32_t q = 0; q < n; ++q) {
      start[q] = at;
      const uint32_t c = kc::batch_blocks((kc::BatchKernel)k, jobs[g.idx[q]].s, p->n_sms, g.bases);
      for (uint32_t x = 0; x < c; ++x) blk2s[at + x] = q;
      at += c;
    }
    start[n] = at;
    bp.start[k] = dw;
    bp.blk2s[k] = dw + n + 1;
    bp.grid[k] = at;
    hw += n + 1 + at;
    dw += n + 1 + at;
  }
  cudaError_t e;
  if ((e = cudaMemcpyAsync(dv, h, g.tab, cudaMemcpyHostToDevice, p->stream)) != cudaSuccess) {
    *stc = KC_ECUDA;
    *err = std::string("copying tables: ") + cudaGetErrorString(e);
    return false;
  }
  const kc::Marker none;
  const int nl = kc::launch_batch(bp, p->n_sms, (void*)p->stream, none);
  if (nl < 0) {
    *stc = KC_ECUDA;
    *err = std::string("launch: ") + cudaGetErrorString((cudaError_t)(-nl));
    return false;
  }
  *launches += (uint32_t)nl;
  for (uint32_t q = 0; q < n; ++q)
    if ((e = cudaMemcpyAsync(meta_dst[q], hd[q].b.meta, sizeof(kc::Meta), cudaMemcpyDeviceToHost, p->stream)) !=
        cudaSuccess) {
      *stc = KC_ECUDA;
      *err = cudaGetErrorString(e);
      return false;
    }
  return true;
}

// grow a plan-held device buffer (stream-ordered: earlier work on the plan's stream keeps
// the old one until it is done)
bool grow_dev(kc_plan_s* p, void*& buf, size_t& have, size_t want) {
  if (have >= want) return true;
  dev_free(p, buf);
  buf = nullptr;
  have = 0;
  buf = dev_alloc(p, want);
  if (!buf) return false;
  have = want;
  return true;
}

void record_stats(kc_plan_s* p, const Job& j, const kc::Meta& m) {
  p->stats.n_partitions = (uint32_t)j.P1;
  p->stats.n_fine = m.n_fine;
  p->stats.n_overflow_fine = m.n_overflow;
  p->stats.n_deferred_fine = m.n_deferred;
  p->stats.fine_sampled = j.s.fine_sampled ? 1u : 0u;
  p->stats.fine_resplit = m.fine_spill ? 1u : 0u;
  for (int i = 0; i < 8; ++i) p->stats.phase_cycles[i] = m.phase_cycles[i];
  for (int i = 0; i < 8; ++i) p->stats.sub_cycles[i] = m.sub_cycles[i];
}

}  // namespace

extern "C" {

const char* kc_last_error(void) { return g_err.c_str(); }

kc_status kc_plan(const kc_plan_opts* opts, kc_plan_t* out) {
  g_err.clear();
  if (!opts || !out) return fail(KC_EINVAL, "kc_plan: opts and out must not be NULL");
  *out = nullptr;
  if ((opts->alloc == nullptr) != (opts->free_ == nullptr))
    return fail(KC_EINVAL, "kc_plan: alloc and free_ must be given together");
  if (opts->n_partitions_hint && (opts->n_partitions_hint & (opts->n_partitions_hint - 1)))
    return fail(KC_EINVAL, "kc_plan: n_partitions_hint must be a power of two");
  if (opts->n_partitions_hint > (1u << kc::kMaxCoarseLog2))
    return fail(KC_EINVAL, "kc_plan: n_partitions_hint above 4096");
  if (opts->table_load < 0.f || opts->table_load > 0.95f) return fail(KC_EINVAL, "kc_plan: table_load outside [0, 0.95]");
  if (opts->table_slots_max && opts->table_slots_max < 64) return fail(KC_EINVAL, "kc_plan: table_slots_max below 64");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (opts->device < 0 || opts->device >= ndev) return fail(KC_EINVAL, "kc_plan: no such device");
  if ((e = cudaSetDevice(opts->device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, opts->device)) != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  if (prop.major < 10) return fail(KC_EINVAL, "kc_plan: the library is built for sm_103a (compute capability 10.x)");
  const int ce = kc::configure_kernels(opts->device);
  if (ce) return cuda_fail((cudaError_t)ce, "cudaFuncSetAttribute");
  kc_plan_s* p = new kc_plan_s();
  p->device = opts->device;
  p->stream = (cudaStream_t)opts->stream;
  p->alloc = opts->alloc;
  p->free_ = opts->free_;
  p->ctx = opts->alloc_ctx;
  p->max_bytes = opts->max_device_bytes;
  p->p_hint = opts->n_partitions_hint;
  p->load = opts->table_load > 0.f ? opts->table_load : 0.55f;
  p->slots_max = opts->table_slots_max;
  p->n_sms = prop.multiProcessorCount;
  p->smem_optin = prop.sharedMemPerBlockOptin;
  p->smem_per_sm = prop.sharedMemPerMultiprocessor;
  p->profile = (opts->flags & KC_PLAN_PROFILE) != 0;
  p->defer_all = (opts->flags & KC_PLAN_DEFER_ALL) != 0;
  p->withhold = (opts->flags & KC_PLAN_TEST_WITHHOLD_PREFIX) != 0;
  p->low_count_limit = (opts->flags & KC_PLAN_TEST_COUNT_LIMIT) != 0;
  p->force_sampled = (opts->flags & KC_PLAN_TEST_FINE_SAMPLED) != 0;
  p->tight_slack = (opts->flags & KC_PLAN_TEST_TIGHT_SLACK) != 0;
  p->small_arena = (opts->flags & KC_PLAN_BATCH_ARENA_SMALL) != 0;
  p->aggr = ((opts->flags & KC_PLAN_ABLATE_NO_SMEM_BUCKETS) ? kc::kAggrNoSmemBuckets : 0) |
            ((opts->flags & KC_PLAN_WARP_MERGE) ? kc::kAggrWarpMerge : 0);
  if (p->profile) {
    for (int i = 0; i <= kc_plan_s::kMaxMarks; ++i) {
      if ((e = cudaEventCreate(&p->ev[i])) != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(p->ev[j]);
        delete p;
        return cuda_fail(e, "cudaEventCreate");
      }
    }
  }
  *out = p;
  return KC_OK;
}

kc_status kc_plan_destroy(kc_plan_t p) {
  g_err.clear();
  if (!p) return fail(KC_EINVAL, "kc_plan_destroy: NULL plan");
  cudaSetDevice(p->device);
  cudaStreamSynchronize(p->stream);
  if (p->xfer) cudaStreamSynchronize(p->xfer);
  while (!p->jobs.empty()) {  // results never collected
    auto it = p->jobs.begin();
    retire(p, it->first, it->second, true);
  }
  if (p->pinned) cudaFreeHost(p->pinned);
  if (p->btab_host) cudaFreeHost(p->btab_host);
  if (p->bmeta) cudaFreeHost(p->bmeta);
  for (auto& st : p->stg) {
    if (st.ev) cudaEventDestroy(st.ev);
    if (st.host) cudaFreeHost(st.host);
  }
  dev_free(p, p->bws);
  dev_free(p, p->btab);
  dev_free(p, p->ws);
  cudaStreamSynchronize(p->stream);
  if (p->xfer) {
    cudaStreamSynchronize(p->xfer);
    cudaStreamDestroy(p->xfer);
  }
  if (p->profile)
    for (int i = 0; i <= kc_plan_s::kMaxMarks; ++i) cudaEventDestroy(p->ev[i]);
  delete p;
  return KC_OK;
}

kc_status kc_footprint(kc_plan_t p, uint64_t n_reads, uint64_t n_bases, int k, int reads_on_device,
                       int offsets_on_device, uint64_t* scratch_bytes, uint64_t* result_bytes) {
  g_err.clear();
  if (!p || !scratch_bytes || !result_bytes) return fail(KC_EINVAL, "kc_footprint: NULL argument");
  if (k < 1 || k > 64) return fail(KC_EINVAL, "kc_footprint: k must be in 1..64");
  kc::Shape s{};
  kc::Layout lay{};
  kc::ShapeOpts o = shape_opts(p);
  o.allow_sampled = 1;  // as kc_count and kc_submit size a count
  kc::make_shape(o, n_bases, n_reads, k, 1, n_bases > 0 && !reads_on_device, !offsets_on_device, s, lay);
  *scratch_bytes = lay.total;
  *result_bytes = s.cap * s.kw * 8 + s.cap * 4;
  return KC_OK;
}

kc_status kc_free(kc_plan_t p, kc_result* r) {
  g_err.clear();
  if (!p || !r) return fail(KC_EINVAL, "kc_free: NULL argument");
  cudaSetDevice(p->device);
  if (r->_owner) {  // a result of a batched group: the group's buffers go with its last result
    release_owner(p, (GroupOwner*)r->_owner);
  } else {
    dev_free(p, r->keys);
    dev_free(p, r->counts);
  }
  memset(r, 0, sizeof(*r));
  return KC_OK;
}

kc_status kc_result_copy_to_host(kc_plan_t p, const kc_result* r, uint64_t* keys_host, uint32_t* counts_host) {
  g_err.clear();
  if (!p || !r) return fail(KC_EINVAL, "kc_result_copy_to_host: NULL argument");
  if (r->n == 0) return KC_OK;
  if (!keys_host || !counts_host || !r->keys || !r->counts) return fail(KC_EINVAL, "kc_result_copy_to_host: NULL buffer");
  cudaSetDevice(p->device);
  cudaError_t e = cudaMemcpyAsync(keys_host, r->keys, r->n * r->key_words * 8, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(counts_host, r->counts, r->n * 4, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "kc_result_copy_to_host");
  return KC_OK;
}

kc_status kc_last_stats(kc_plan_t p, kc_stats* out) {
  g_err.clear();
  if (!p || !out) return fail(KC_EINVAL, "kc_last_stats: NULL argument");
  *out = p->stats;
  out->workspace_bytes = p->ws_bytes;
  return KC_OK;
}

kc_status kc_last_kernel_times(kc_plan_t p, uint32_t max, const char** names, float* ms, uint32_t* n_out) {
  g_err.clear();
  if (!p || !n_out) return fail(KC_EINVAL, "kc_last_kernel_times: NULL argument");
  if (!p->profile) return fail(KC_EINVAL, "kc_last_kernel_times: plan created without KC_PLAN_PROFILE");
  *n_out = (uint32_t)p->n_kernel_ms;
  for (uint32_t i = 0; i < max && i < (uint32_t)p->n_kernel_ms; ++i) {
    if (names) names[i] = p->ev_name[i];
    if (ms) ms[i] = p->kernel_ms[i];
  }
  return KC_OK;
}

kc_status kc_count(kc_plan_t p, const uint8_t* reads, const uint64_t* offsets, uint64_t n_reads, int k, int canonical,
                   kc_result* out) {
  g_err.clear();
  if (!p || !out) return fail(KC_EINVAL, "kc_count: plan and out must not be NULL");
  memset(out, 0, sizeof(*out));
  if (k < 1 || k > 64) return fail(KC_EINVAL, "kc_count: k must be in 1..64");
  if (!offsets) return fail(KC_EINVAL, "kc_count: offsets must not be NULL");
  ScopedBusy busy(p);
  if (!busy.ok) return fail(KC_EBUSY, "kc_count: plan in use by another call");
  cudaError_t e = cudaSetDevice(p->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaStream_t st = p->stream;

  // ---- offsets: where they live, the total length, and (for host offsets) validity
  const bool off_dev = is_device_ptr(offsets);
  uint64_t first = 0, L = 0;
  if (off_dev) {
    if ((e = cudaMemcpyAsync(&first, offsets, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&L, offsets + n_reads, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_fail(e, "kc_count: reading offsets");
  } else {  // their order is checked on the device (k_check_offsets), as for device offsets
    first = offsets[0];
    L = offsets[n_reads];
  }
  if (first != 0) return fail(KC_EINVAL, "kc_count: offsets[0] must be 0");
  if (L > 0 && !reads) return fail(KC_EINVAL, "kc_count: reads must not be NULL");

  Job j;
  plan_job(p, reads, offsets, n_reads, L, off_dev, k, canonical, j, false, true);
  if (p->max_bytes && (uint64_t)(j.ws_bytes + j.out_key_bytes + j.out_cnt_bytes) > p->max_bytes)
    return fail(KC_ENOMEM, "kc_count: input needs more device memory than max_device_bytes");
  if (p->ws_bytes < j.ws_bytes) {
    dev_free(p, p->ws);
    p->ws = nullptr;
    p->ws_bytes = 0;
    void* w = dev_alloc(p, j.ws_bytes);
    if (!w) return fail(KC_ENOMEM, "kc_count: scratch allocation failed");
    p->ws = w;
    p->ws_bytes = j.ws_bytes;
  }
  j.okeys = dev_alloc(p, j.out_key_bytes);
  j.ocnts = j.okeys ? dev_alloc(p, j.out_cnt_bytes) : nullptr;
  if (!j.okeys || !j.ocnts) {
    dev_free(p, j.okeys);
    return fail(KC_ENOMEM, "kc_count: result allocation failed");
  }
  // on any error: let the launched work finish before its buffers go back to the allocator
  auto bail = [&](kc_status stc, const std::string& msg) {
    cudaStreamSynchronize(st);
    cudaGetLastError();
    dev_free(p, j.okeys);
    dev_free(p, j.ocnts);
    return fail(stc, msg);
  };

  kc::Marker mark;
  p->n_marks = 0;
  p->n_kernel_ms = 0;
  if (p->profile) {
    mark.fn = record_mark;
    mark.ctx = p;
    cudaEventRecord(p->ev[0], st);
  } else if (getenv("KC_DEBUG_SYNC")) {
    mark.fn = debug_mark;
    mark.ctx = p;
  }
  kc::Meta m{};
  int launches = 0;
  std::string err;
  if (!enqueue_job(j, (uint8_t*)p->ws, st, &m, mark, p->n_sms, &launches, &err)) return bail(KC_ECUDA, "kc_count: " + err);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(KC_ECUDA, std::string("kc_count: ") + cudaGetErrorString(e));
  p->stats.kernel_launches = (uint32_t)launches;
  if (p->profile) {
    for (int i = 0; i < p->n_marks; ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, p->ev[i], p->ev[i + 1]);
      p->kernel_ms[i] = t;
    }
    p->n_kernel_ms = p->n_marks;
  }
  record_stats(p, j, m);
  std::string msg;
  const kc_status stc = job_status(j, m, "kc_count", &msg);
  if (stc != KC_OK) return bail(stc, msg);
  fill_result(j, m, out);
  return KC_OK;
}

kc_status kc_count_batch(kc_plan_t p, uint32_t n_samples, const uint8_t* const* reads, const uint64_t* const* offsets,
                         const uint64_t* n_reads, const uint64_t* n_bases, int k, int canonical, kc_result* out) {
  g_err.clear();
  if (!p || !out) return fail(KC_EINVAL, "kc_count_batch: plan and out must not be NULL");
  for (uint32_t i = 0; i < n_samples; ++i) memset(&out[i], 0, sizeof(out[i]));
  if (n_samples == 0) return KC_OK;
  if (!reads || !offsets || !n_reads || !n_bases) return fail(KC_EINVAL, "kc_count_batch: NULL sample array");
  if (k < 1 || k > 64) return fail(KC_EINVAL, "kc_count_batch: k must be in 1..64");
  ScopedBusy busy(p);
  if (!busy.ok) return fail(KC_EBUSY, "kc_count_batch: plan in use by another call");
  cudaError_t e = cudaSetDevice(p->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");

  // ---- every sample's shape and scratch layout (host only; nothing is read back)
  std::vector<Job> jobs(n_samples);
  for (uint32_t i = 0; i < n_samples; ++i) {
    if (!offsets[i]) return fail(KC_EINVAL, "kc_count_batch: offsets of a sample is NULL");
    const bool off_dev = is_device_ptr(offsets[i]);
    if (!off_dev && (offsets[i][0] != 0 || offsets[i][n_reads[i]] != n_bases[i]))  // order: checked on the device
      return fail(KC_EINVAL, "kc_count_batch: a sample's offsets must run from 0 to its base count");
    if (n_bases[i] > 0 && !reads[i]) return fail(KC_EINVAL, "kc_count_batch: reads of a sample is NULL");
    plan_job(p, reads[i], offsets[i], n_reads[i], n_bases[i], off_dev, k, canonical, jobs[i], false, true);
  }
  // ---- groups: counts whose scratch fits the arena together share the batched launches
  // (every kernel once per group); a count larger than the arena runs alone
  GroupPlan gp;
  std::string err;
  if (!plan_groups(p, jobs, gp, &err)) return fail(KC_EINVAL, "kc_count_batch: " + err);
  const size_t total = gp.out_total + gp.arena + gp.need_single + gp.tab_total;
  if (p->max_bytes && total > p->max_bytes)
    return fail(KC_ENOMEM, "kc_count_batch: the batch needs more device memory than max_device_bytes");
  if (!gp.alone.empty() && !grow_dev(p, p->ws, p->ws_bytes, gp.need_single))
    return fail(KC_ENOMEM, "kc_count_batch: scratch allocation failed");
  if (!gp.groups.empty() &&
      (!grow_dev(p, p->bws, p->bws_bytes, gp.arena) || !grow_dev(p, p->btab, p->btab_bytes, gp.tab_total)))
    return fail(KC_ENOMEM, "kc_count_batch: scratch allocation failed");
  if (p->btab_host_bytes < gp.tab_total) {
    if (p->btab_host) cudaFreeHost(p->btab_host);
    p->btab_host = nullptr;
    p->btab_host_bytes = 0;
    if ((e = cudaMallocHost(&p->btab_host, gp.tab_total)) != cudaSuccess)
      return cuda_fail(e, "kc_count_batch: pinned tables");
    p->btab_host_bytes = gp.tab_total;
  }
  if (p->bmeta_n < n_samples) {
    if (p->bmeta) cudaFreeHost(p->bmeta);
    p->bmeta = nullptr;
    p->bmeta_n = 0;
    if ((e = cudaMallocHost((void**)&p->bmeta, sizeof(kc::Meta) * n_samples)) != cudaSuccess)
      return cuda_fail(e, "kc_count_batch: pinned status buffer");
    p->bmeta_n = n_samples;
  }
  kc::Meta* metas = p->bmeta;
  std::vector<GroupOwner*> owners(gp.groups.size(), nullptr);
  auto release = [&](kc_status stc, const std::string& msg) {
    cudaStreamSynchronize(p->stream);
    cudaGetLastError();
    for (uint32_t i : gp.alone) {
      dev_free(p, jobs[i].okeys);
      dev_free(p, jobs[i].ocnts);
    }
    for (GroupOwner* o : owners)
      if (o) {
        dev_free(p, o->keys);
        dev_free(p, o->counts);
        delete o;
      }
    for (uint32_t i = 0; i < n_samples; ++i) memset(&out[i], 0, sizeof(out[i]));
    return fail(stc, msg);
  };
  // ---- enqueue everything on the plan's stream; no host synchronisation until the end
  const kc::Marker none;
  uint32_t launches = 0;
  for (uint32_t i : gp.alone) {
    Job& j = jobs[i];
    j.okeys = dev_alloc(p, j.out_key_bytes);
    j.ocnts = j.okeys ? dev_alloc(p, j.out_cnt_bytes) : nullptr;
    if (!j.okeys || !j.ocnts) return release(KC_ENOMEM, "kc_count_batch: result allocation failed");
    int nl = 0;
    if (!enqueue_job(j, (uint8_t*)p->ws, p->stream, &metas[i], none, p->n_sms, &nl, &err))
      return release(KC_ECUDA, "kc_count_batch: " + err);
    launches += (uint32_t)nl;
  }
  size_t tab_at = 0;
  for (size_t gi = 0; gi < gp.groups.size(); ++gi) {
    const Group& g = gp.groups[gi];
    owners[gi] = new GroupOwner();
    owners[gi]->refs = (int)g.idx.size();
    std::vector<kc::Meta*> dst(g.idx.size());
    for (size_t q = 0; q < g.idx.size(); ++q) dst[q] = &metas[g.idx[q]];
    kc_status stc = KC_OK;
    if (!enqueue_group(p, jobs, g, owners[gi], (uint8_t*)p->btab_host + tab_at, (uint8_t*)p->btab + tab_at, dst.data(),
                       &launches, &stc, &err))
      return release(stc, "kc_count_batch: " + err);
    tab_at += g.tab;
  }
  if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess)
    return release(KC_ECUDA, std::string("kc_count_batch: ") + cudaGetErrorString(e));
  for (uint32_t i = 0; i < n_samples; ++i) {
    std::string msg;
    const kc_status stc = job_status(jobs[i], metas[i], "kc_count_batch", &msg);
    if (stc != KC_OK) return release(stc, msg + " (sample " + std::to_string(i) + ")");
  }
  for (uint32_t i = 0; i < n_samples; ++i) fill_result(jobs[i], metas[i], &out[i]);
  for (size_t gi = 0; gi < gp.groups.size(); ++gi)
    for (uint32_t q : gp.groups[gi].idx) out[q]._owner = owners[gi];
  p->stats = kc_stats{};
  p->stats.kernel_launches = launches;
  return KC_OK;
}


kc_status kc_submit(kc_plan_t p, const uint8_t* reads, const uint64_t* offsets, uint64_t n_reads, uint64_t n_bases,
                    int k, int canonical, uint64_t* job) {
  g_err.clear();
  if (!p || !job) return fail(KC_EINVAL, "kc_submit: plan and job must not be NULL");
  *job = 0;
  if (k < 1 || k > 64) return fail(KC_EINVAL, "kc_submit: k must be in 1..64");
  if (!offsets) return fail(KC_EINVAL, "kc_submit: offsets must not be NULL");
  if (n_bases > 0 && !reads) return fail(KC_EINVAL, "kc_submit: reads must not be NULL");
  ScopedBusy busy(p);
  if (!busy.ok) return fail(KC_EBUSY, "kc_submit: plan in use by another call");
  cudaError_t e = cudaSetDevice(p->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  const bool off_dev = is_device_ptr(offsets);
  if (!off_dev && (offsets[0] != 0 || offsets[n_reads] != n_bases))  // their order: checked on the device
    return fail(KC_EINVAL, "kc_submit: offsets must run from 0 to the base count");
  if (!p->xfer && (e = cudaStreamCreateWithFlags(&p->xfer, cudaStreamNonBlocking)) != cudaSuccess) {
    p->xfer = nullptr;
    return cuda_fail(e, "kc_submit: transfer stream");
  }
  if (!p->pinned) {
    if ((e = cudaMallocHost((void**)&p->pinned, sizeof(kc::Meta) * kc_plan_s::kPinned)) != cudaSuccess)
      return cuda_fail(e, "kc_submit: pinned status records");
    for (int i = kc_plan_s::kPinned - 1; i >= 0; --i) p->pinned_free.push_back(i);
  }
  if (p->pinned_free.empty()) return fail(KC_EBUSY, "kc_submit: too many counts in flight");
  AsyncJob* a = new AsyncJob();
  plan_job(p, reads, offsets, n_reads, n_bases, off_dev, k, canonical, a->j, true, true);
  const size_t stage_r = a->j.stage_r ? (n_bases + 16 + 255) / 256 * 256 : 0;
  const size_t stage_o = a->j.stage_o ? (n_reads + 1) * 8 : 0;
  if (p->max_bytes &&
      (uint64_t)(a->j.ws_bytes + stage_r + stage_o + a->j.out_key_bytes + a->j.out_cnt_bytes) > p->max_bytes) {
    delete a;
    return fail(KC_ENOMEM, "kc_submit: input needs more device memory than max_device_bytes");
  }
  // host inputs: copied on the transfer stream into the job's own buffer (allocated for that
  // stream), the count's kernels wait for the copy's event
  if (stage_r + stage_o) {
    a->stage = dev_alloc_on(p, stage_r + stage_o, p->xfer);
    if (!a->stage) {
      delete a;
      return fail(KC_ENOMEM, "kc_submit: input staging allocation failed");
    }
    a->j.stage_reads = (const uint8_t*)a->stage;
    a->j.stage_offs = (const uint64_t*)((uint8_t*)a->stage + stage_r);
    if ((a->j.stage_r && (e = cudaMemcpyAsync((void*)a->j.stage_reads, reads, n_bases, cudaMemcpyHostToDevice,
                                              p->xfer)) != cudaSuccess) ||
        (a->j.stage_o && (e = cudaMemcpyAsync((void*)a->j.stage_offs, offsets, stage_o, cudaMemcpyHostToDevice,
                                              p->xfer)) != cudaSuccess) ||
        (e = cudaEventCreateWithFlags(&a->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventRecord(a->ev_in, p->xfer)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p->stream, a->ev_in, 0)) != cudaSuccess) {
      cudaStreamSynchronize(p->xfer);
      cudaStreamSynchronize(p->stream);
      if (a->ev_in) cudaEventDestroy(a->ev_in);
      dev_free_on(p, a->stage, p->xfer);
      delete a;
      return cuda_fail(e, "kc_submit: copying the inputs");
    }
  }
  // submitted counts run one after another on the plan's stream (never two at once on the
  // device); the plan's scratch grows in stream order if this count needs more
  const cudaStream_t lst = p->stream;
  if (p->ws_bytes < a->j.ws_bytes) {
    dev_free(p, p->ws);
    p->ws = nullptr;
    p->ws_bytes = 0;
    p->ws = dev_alloc(p, a->j.ws_bytes);
    if (!p->ws) {
      drop_unsubmitted(p, a);
      return fail(KC_ENOMEM, "kc_submit: scratch allocation failed");
    }
    p->ws_bytes = a->j.ws_bytes;
  }
  a->j.okeys = dev_alloc(p, a->j.out_key_bytes);
  a->j.ocnts = a->j.okeys ? dev_alloc(p, a->j.out_cnt_bytes) : nullptr;
  if (!a->j.okeys || !a->j.ocnts) {
    dev_free(p, a->j.okeys);
    drop_unsubmitted(p, a);
    return fail(KC_ENOMEM, "kc_submit: result allocation failed");
  }
  a->slot = p->pinned_free.back();
  p->pinned_free.pop_back();
  const uint64_t id = p->next_job++;
  p->jobs[id] = a;
  int nl = 0;
  std::string err;
  const kc::Marker none;
  if (!enqueue_job(a->j, (uint8_t*)p->ws, lst, &p->pinned[a->slot], none, p->n_sms, &nl, &err)) {
    cudaStreamSynchronize(lst);
    cudaStreamSynchronize(p->xfer);
    cudaGetLastError();
    retire(p, id, a, true);
    return fail(KC_ECUDA, "kc_submit: " + err);
  }
  if ((e = cudaEventCreateWithFlags(&a->ev, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventRecord(a->ev, lst)) != cudaSuccess) {
    cudaStreamSynchronize(lst);
    cudaStreamSynchronize(p->xfer);
    retire(p, id, a, true);
    return cuda_fail(e, "kc_submit: completion event");
  }
  *job = id;
  return KC_OK;
}


kc_status kc_submit_batch(kc_plan_t p, uint32_t n_samples, const uint8_t* const* reads, const uint64_t* const* offsets,
                          const uint64_t* n_reads, const uint64_t* n_bases, int k, int canonical, uint64_t* job_ids) {
  g_err.clear();
  if (!p || !job_ids) return fail(KC_EINVAL, "kc_submit_batch: plan and job_ids must not be NULL");
  for (uint32_t i = 0; i < n_samples; ++i) job_ids[i] = 0;
  if (n_samples == 0) return KC_OK;
  if (!reads || !offsets || !n_reads || !n_bases) return fail(KC_EINVAL, "kc_submit_batch: NULL sample array");
  if (k < 1 || k > 64) return fail(KC_EINVAL, "kc_submit_batch: k must be in 1..64");
  ScopedBusy busy(p);
  if (!busy.ok) return fail(KC_EBUSY, "kc_submit_batch: plan in use by another call");
  cudaError_t e = cudaSetDevice(p->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  std::vector<Job> jobs(n_samples);
  for (uint32_t i = 0; i < n_samples; ++i) {
    if (!offsets[i]) return fail(KC_EINVAL, "kc_submit_batch: offsets of a sample is NULL");
    const bool off_dev = is_device_ptr(offsets[i]);
    if (!off_dev) {
      if (offsets[i][0] != 0 || offsets[i][n_reads[i]] != n_bases[i])
        return fail(KC_EINVAL, "kc_submit_batch: a sample's offsets must run from 0 to its base count");
      for (uint64_t r = 0; r < n_reads[i]; ++r)
        if (offsets[i][r + 1] < offsets[i][r]) return fail(KC_EINVAL, "kc_submit_batch: offsets must be non-decreasing");
    }
    if (n_bases[i] > 0 && !reads[i]) return fail(KC_EINVAL, "kc_submit_batch: reads of a sample is NULL");
    plan_job(p, reads[i], offsets[i], n_reads[i], n_bases[i], off_dev, k, canonical, jobs[i], false, true);
  }
  GroupPlan gp;
  std::string err;
  if (!plan_groups(p, jobs, gp, &err)) return fail(KC_EINVAL, "kc_submit_batch: " + err);
  if (p->max_bytes && gp.out_total + gp.arena + gp.need_single + gp.tab_max > p->max_bytes)
    return fail(KC_ENOMEM, "kc_submit_batch: the batch needs more device memory than max_device_bytes");
  if (!p->pinned) {
    if ((e = cudaMallocHost((void**)&p->pinned, sizeof(kc::Meta) * kc_plan_s::kPinned)) != cudaSuccess)
      return cuda_fail(e, "kc_submit_batch: pinned status records");
    for (int i = kc_plan_s::kPinned - 1; i >= 0; --i) p->pinned_free.push_back(i);
  }
  if (p->pinned_free.size() < n_samples) return fail(KC_EBUSY, "kc_submit_batch: too many counts in flight");
  // scratch, arena and device tables grow in stream order (earlier counts keep the old ones)
  if (!gp.alone.empty() && !grow_dev(p, p->ws, p->ws_bytes, gp.need_single))
    return fail(KC_ENOMEM, "kc_submit_batch: scratch allocation failed");
  if (!gp.groups.empty() &&
      (!grow_dev(p, p->bws, p->bws_bytes, gp.arena) || !grow_dev(p, p->btab, p->btab_bytes, gp.tab_max)))
    return fail(KC_ENOMEM, "kc_submit_batch: scratch allocation failed");
  // one job per count, each with its pinned status slot and completion event
  std::vector<AsyncJob*> made(n_samples, nullptr);
  std::vector<uint64_t> ids(n_samples, 0);
  for (uint32_t i = 0; i < n_samples; ++i) {
    AsyncJob* a = new AsyncJob();
    a->slot = p->pinned_free.back();
    p->pinned_free.pop_back();
    ids[i] = p->next_job++;
    p->jobs[ids[i]] = a;
    made[i] = a;
  }
  std::vector<GroupOwner*> owners(gp.groups.size(), nullptr);
  auto release = [&](kc_status stc, const std::string& msg) {
    cudaStreamSynchronize(p->stream);
    cudaGetLastError();
    for (uint32_t i : gp.alone) {
      dev_free(p, jobs[i].okeys);
      dev_free(p, jobs[i].ocnts);
    }
    for (GroupOwner* o : owners)
      if (o) {
        dev_free(p, o->keys);
        dev_free(p, o->counts);
        delete o;
      }
    for (uint32_t i = 0; i < n_samples; ++i) retire(p, ids[i], made[i], false);  // no buffers of their own yet
    return fail(stc, msg);
  };
  const kc::Marker none;
  uint32_t launches = 0;
  for (uint32_t i : gp.alone) {
    Job& j = jobs[i];
    j.okeys = dev_alloc(p, j.out_key_bytes);
    j.ocnts = j.okeys ? dev_alloc(p, j.out_cnt_bytes) : nullptr;
    if (!j.okeys || !j.ocnts) return release(KC_ENOMEM, "kc_submit_batch: result allocation failed");
    int nl = 0;
    if (!enqueue_job(j, (uint8_t*)p->ws, p->stream, &p->pinned[made[i]->slot], none, p->n_sms, &nl, &err))
      return release(KC_ECUDA, "kc_submit_batch: " + err);
    launches += (uint32_t)nl;
  }
  for (size_t gi = 0; gi < gp.groups.size(); ++gi) {
    const Group& g = gp.groups[gi];
    // a pinned staging buffer whose last copy has completed
    kc_plan_s::Staging& st = p->stg[p->stg_next];
    p->stg_next = (p->stg_next + 1) % kc_plan_s::kStaging;
    if (st.ev && (e = cudaEventSynchronize(st.ev)) != cudaSuccess)
      return release(KC_ECUDA, std::string("kc_submit_batch: ") + cudaGetErrorString(e));
    if (st.bytes < g.tab) {
      if (st.host) cudaFreeHost(st.host);
      st.host = nullptr;
      st.bytes = 0;
      if ((e = cudaMallocHost(&st.host, g.tab)) != cudaSuccess)
        return release(KC_ECUDA, std::string("kc_submit_batch: pinned tables: ") + cudaGetErrorString(e));
      st.bytes = g.tab;
    }
    if (!st.ev && (e = cudaEventCreateWithFlags(&st.ev, cudaEventDisableTiming)) != cudaSuccess)
      return release(KC_ECUDA, std::string("kc_submit_batch: ") + cudaGetErrorString(e));
    owners[gi] = new GroupOwner();
    owners[gi]->refs = (int)g.idx.size();
    std::vector<kc::Meta*> dst(g.idx.size());
    for (size_t q = 0; q < g.idx.size(); ++q) dst[q] = &p->pinned[made[g.idx[q]]->slot];
    kc_status stc = KC_OK;
    if (!enqueue_group(p, jobs, g, owners[gi], (uint8_t*)st.host, (uint8_t*)p->btab, dst.data(), &launches, &stc, &err))
      return release(stc, "kc_submit_batch: " + err);
    if ((e = cudaEventRecord(st.ev, p->stream)) != cudaSuccess)
      return release(KC_ECUDA, std::string("kc_submit_batch: ") + cudaGetErrorString(e));
  }
  for (uint32_t i = 0; i < n_samples; ++i) {
    if ((e = cudaEventCreateWithFlags(&made[i]->ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventRecord(made[i]->ev, p->stream)) != cudaSuccess)
      return release(KC_ECUDA, std::string("kc_submit_batch: completion event: ") + cudaGetErrorString(e));
  }
  // hand over: each job owns its outputs (counted alone) or a reference on its group's buffers
  for (uint32_t i = 0; i < n_samples; ++i) made[i]->j = jobs[i];
  for (size_t gi = 0; gi < gp.groups.size(); ++gi)
    for (uint32_t q : gp.groups[gi].idx) made[q]->owner = owners[gi];
  for (uint32_t i = 0; i < n_samples; ++i) job_ids[i] = ids[i];
  return KC_OK;
}

static kc_status job_collect(kc_plan_t p, uint64_t id, kc_result* out, int* done, bool block) {
  const std::string who = block ? "kc_job_wait" : "kc_job_poll";
  g_err.clear();
  if (!p || !out || !done) return fail(KC_EINVAL, who + ": NULL argument");
  *done = 0;
  memset(out, 0, sizeof(*out));
  ScopedBusy busy(p);
  if (!busy.ok) return fail(KC_EBUSY, who + ": plan in use by another call");
  auto it = p->jobs.find(id);
  if (it == p->jobs.end()) return fail(KC_EINVAL, who + ": no such job");
  AsyncJob* a = it->second;
  cudaSetDevice(p->device);
  auto drop = [&](kc_status stc, const std::string& msg) {
    *done = 1;
    if (a->stage || a->copying) cudaStreamSynchronize(p->xfer);
    retire(p, id, a, true);
    return fail(stc, msg);
  };
  if (!a->copying) {
    const cudaError_t q = block ? cudaEventSynchronize(a->ev) : cudaEventQuery(a->ev);
    if (q == cudaErrorNotReady) return KC_OK;
    if (q != cudaSuccess) return drop(KC_ECUDA, who + ": " + cudaGetErrorString(q));
    a->meta = p->pinned[a->slot];
    std::string msg;
    const kc_status stc = job_status(a->j, a->meta, who.c_str(), &msg);
    if (stc != KC_OK) return drop(stc, msg);
    if (a->keys_host) {
      // the count has ended (its event was seen): its result goes out on the transfer stream,
      // behind the input copies queued there, while the counts queued after it run
      const uint64_t n = a->meta.n_distinct;
      if (n > a->host_cap) return drop(KC_EINVAL, who + ": the result does not fit the host buffers given");
      cudaError_t e = cudaSuccess;
      if (n && ((e = cudaMemcpyAsync(a->keys_host, a->j.okeys, n * a->j.s.kw * 8, cudaMemcpyDefault, p->xfer)) !=
                    cudaSuccess ||
                (e = cudaMemcpyAsync(a->counts_host, a->j.ocnts, n * 4, cudaMemcpyDefault, p->xfer)) != cudaSuccess))
        return drop(KC_ECUDA, who + ": copying the result out: " + cudaGetErrorString(e));
      if ((e = cudaEventRecord(a->ev_out, p->xfer)) != cudaSuccess)
        return drop(KC_ECUDA, who + ": copy event: " + cudaGetErrorString(e));
      a->copying = true;
    }
  }
  if (a->copying) {
    const cudaError_t q = block ? cudaEventSynchronize(a->ev_out) : cudaEventQuery(a->ev_out);
    if (q == cudaErrorNotReady) return KC_OK;
    if (q != cudaSuccess) return drop(KC_ECUDA, who + ": copying the result out: " + cudaGetErrorString(q));
  }
  *done = 1;
  fill_result(a->j, a->meta, out);
  out->_owner = a->owner;  // the result keeps the job's reference on the group's buffers
  record_stats(p, a->j, a->meta);
  retire(p, id, a, false);
  return KC_OK;
}

kc_status kc_job_poll(kc_plan_t p, uint64_t job, kc_result* out, int* done) {
  return job_collect(p, job, out, done, false);
}

kc_status kc_job_wait(kc_plan_t p, uint64_t job, kc_result* out) {
  int done = 0;
  return job_collect(p, job, out, &done, true);
}

kc_status kc_job_copy_to_host(kc_plan_t p, uint64_t job, uint64_t* keys_host, uint32_t* counts_host,
                              uint64_t capacity) {
  g_err.clear();
  if (!p || !keys_host || !counts_host) return fail(KC_EINVAL, "kc_job_copy_to_host: NULL argument");
  ScopedBusy busy(p);
  if (!busy.ok) return fail(KC_EBUSY, "kc_job_copy_to_host: plan in use by another call");
  auto it = p->jobs.find(job);
  if (it == p->jobs.end()) return fail(KC_EINVAL, "kc_job_copy_to_host: no such job");
  AsyncJob* a = it->second;
  if (a->copying) return fail(KC_EINVAL, "kc_job_copy_to_host: the job's result is already being copied");
  cudaSetDevice(p->device);
  if (!a->ev_out) {
    const cudaError_t e = cudaEventCreateWithFlags(&a->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      a->ev_out = nullptr;
      return cuda_fail(e, "kc_job_copy_to_host: copy event");
    }
  }
  a->keys_host = keys_host;
  a->counts_host = counts_host;
  a->host_cap = capacity;
  return KC_OK;
}

}  // extern "C"

// kc_api.cu - the C ABI declared in include/kc.h: plans, scratch memory, argument
// checks, the phase-1 / phase-2 launch sequence and error reporting.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <string>

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

}  // namespace

namespace kc {
void set_error_message(const char* msg) { g_err = msg ? msg : ""; }
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
  void* ws = nullptr;
  size_t ws_bytes = 0;
  std::atomic<int> busy{0};
  kc_stats stats{};
  // per-kernel timing (KC_PLAN_PROFILE)
  bool profile = false;
  bool defer_all = false;
  static constexpr int kMaxMarks = 32;
  cudaEvent_t ev[kMaxMarks + 1] = {};
  const char* ev_name[kMaxMarks] = {};
  int n_marks = 0;
  float kernel_ms[kMaxMarks] = {};
  int n_kernel_ms = 0;
};

namespace {

void* dev_alloc(kc_plan_s* p, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (p->alloc) return p->alloc(bytes, (void*)p->stream, p->ctx);
  void* ptr = nullptr;
  if (cudaMallocAsync(&ptr, bytes, p->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return ptr;
}

void dev_free(kc_plan_s* p, void* ptr) {
  if (!ptr) return;
  if (p->free_) p->free_(ptr, (void*)p->stream, p->ctx);
  else cudaFreeAsync(ptr, p->stream);
}

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Layout {
  size_t off[24];
  int n = 0;
  size_t total = 0;
  size_t add(size_t bytes) {
    const size_t o = total;
    total = align_up(total + bytes, 256);
    off[n++] = o;
    return o;
  }
};

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

int ceil_log2_u64(uint64_t v) { return v <= 1 ? 0 : 64 - __builtin_clzll(v - 1); }

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
  p->profile = (opts->flags & KC_PLAN_PROFILE) != 0;
  p->defer_all = (opts->flags & KC_PLAN_DEFER_ALL) != 0;
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
  dev_free(p, p->ws);
  cudaStreamSynchronize(p->stream);
  if (p->profile)
    for (int i = 0; i <= kc_plan_s::kMaxMarks; ++i) cudaEventDestroy(p->ev[i]);
  delete p;
  return KC_OK;
}

kc_status kc_free(kc_plan_t p, kc_result* r) {
  g_err.clear();
  if (!p || !r) return fail(KC_EINVAL, "kc_free: NULL argument");
  cudaSetDevice(p->device);
  dev_free(p, r->keys);
  dev_free(p, r->counts);
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
  } else {
    first = offsets[0];
    L = offsets[n_reads];
    for (uint64_t i = 0; i < n_reads; ++i)
      if (offsets[i + 1] < offsets[i]) return fail(KC_EINVAL, "kc_count: offsets must be non-decreasing");
  }
  if (first != 0) return fail(KC_EINVAL, "kc_count: offsets[0] must be 0");
  if (L > 0 && !reads) return fail(KC_EINVAL, "kc_count: reads must not be NULL");
  const bool reads_dev = L > 0 && is_device_ptr(reads);
  const bool copy_reads = L > 0 && (!reads_dev || ((uintptr_t)reads & 15) != 0);

  // ---- shape
  kc::Shape s{};
  s.L = L;
  s.n_reads = n_reads;
  s.n_words = (L + 31) / 32;
  s.n_tiles = (s.n_words + kc::kTileWords - 1) / kc::kTileWords;
  s.k = k;
  s.canonical = canonical ? 1 : 0;
  s.kw = k <= 32 ? 1 : 2;
  int b1;
  if (p->p_hint) b1 = ceil_log2_u64(p->p_hint);
  else {
    // coarse partitions of at most about 6 M windows: few enough partitions that the keys
    // pass B writes for one partition per step form runs of whole sectors, small enough
    // that a partition of distinct keys splits into at most ~1400 fine partitions
    const int want = ceil_log2_u64(L / (6u << 20) + 1);
    b1 = want < 11 ? want : 11;
  }
  s.b1 = b1;
  const int P1 = 1 << b1;
  int bT_max = kc::table_log2_max(s.kw, p->smem_optin);
  if (p->slots_max) {
    int bt = 63 - __builtin_clzll((uint64_t)p->slots_max);
    if (bt < bT_max) bT_max = bt;
  }
  s.bT_max = bT_max;
  s.tail = bT_max >= 10 ? 1024 : (1 << bT_max);
  const double ft = (double)(1u << bT_max) * p->load;  // distinct keys per fine partition aimed at
  s.fine_target = ft < 16 ? 16u : (uint32_t)ft;
  s.cap = L > 0 ? L : 1;
  // sum over partitions of ceil(n_c / target), target >= fine_target: at most K / ft + P1
  const uint64_t nf_bound = s.cap / s.fine_target + (uint64_t)P1 + 1;
  const uint64_t nf_lim = (uint64_t)P1 * kc::kMaxFine;
  const uint64_t nf_max64 = nf_bound < nf_lim ? nf_bound : nf_lim;
  const uint32_t nf_max = (uint32_t)nf_max64;
  s.nf_max = nf_max;
  s.smem_budget = p->smem_optin;
  s.profile = p->profile ? 1 : 0;
  s.defer_all = p->defer_all ? 1 : 0;

  // ---- scratch layout
  Layout lay;
  const size_t o_reads = lay.add(copy_reads ? L + 16 : 0);
  const size_t o_offs = lay.add(off_dev ? 0 : (n_reads + 1) * 8);
  const size_t o_codes = lay.add(s.n_words * 8);
  const size_t o_inv = lay.add(s.n_words * 4);
  const size_t o_tf = lay.add(s.n_tiles * 8);
  const size_t o_hist = lay.add(s.n_tiles * P1 * 4);
  const size_t o_toff = lay.add(s.n_tiles * P1 * 8);
  const size_t o_cst = lay.add((size_t)(P1 + 1) * 8);
  const size_t o_fb = lay.add((size_t)(P1 + 1) * 4);
  const size_t o_fl = lay.add((size_t)P1 * 4);
  const size_t o_hll = lay.add((size_t)kc::kHllRegs * 4);
  const size_t o_fh = lay.add((size_t)nf_max * 4);
  const size_t o_fo = lay.add((size_t)(nf_max + 1) * 8);
  const size_t o_flo = lay.add((size_t)(nf_max + 1) * 4);
  const size_t o_fc = lay.add((size_t)nf_max * 8);
  const size_t o_look = lay.add((size_t)nf_max * 8);
  const size_t o_kbuf = lay.add(s.cap * s.kw * 8);
  const size_t o_sbuf = lay.add(s.cap * s.kw * 8);
  const size_t o_meta = lay.add(sizeof(kc::Meta));
  const size_t out_key_bytes = s.cap * s.kw * 8, out_cnt_bytes = s.cap * 4;
  if (p->max_bytes && (uint64_t)(lay.total + out_key_bytes + out_cnt_bytes) > p->max_bytes)
    return fail(KC_ENOMEM, "kc_count: input needs more device memory than max_device_bytes");
  if (p->ws_bytes < lay.total) {
    dev_free(p, p->ws);
    p->ws = nullptr;
    p->ws_bytes = 0;
    void* w = dev_alloc(p, lay.total);
    if (!w) return fail(KC_ENOMEM, "kc_count: scratch allocation failed");
    p->ws = w;
    p->ws_bytes = lay.total;
  }
  uint8_t* ws = (uint8_t*)p->ws;
  void* okeys = dev_alloc(p, out_key_bytes);
  void* ocnts = okeys ? dev_alloc(p, out_cnt_bytes) : nullptr;
  if (!okeys || !ocnts) {
    dev_free(p, okeys);
    return fail(KC_ENOMEM, "kc_count: result allocation failed");
  }

  kc::Buffers b{};
  b.reads = copy_reads ? (const uint8_t*)(ws + o_reads) : reads;
  b.offsets = off_dev ? offsets : (const uint64_t*)(ws + o_offs);
  b.codes64 = (uint64_t*)(ws + o_codes);
  b.inv32 = (uint32_t*)(ws + o_inv);
  b.tile_first = (uint64_t*)(ws + o_tf);
  b.hist = (uint32_t*)(ws + o_hist);
  b.toff = (uint64_t*)(ws + o_toff);
  b.cstart = (uint64_t*)(ws + o_cst);
  b.fine_base = (uint32_t*)(ws + o_fb);
  b.fine_m = (uint32_t*)(ws + o_fl);
  b.hll = (uint32_t*)(ws + o_hll);
  b.fhist = (uint32_t*)(ws + o_fh);
  b.foff = (uint64_t*)(ws + o_fo);
  b.flo = (uint32_t*)(ws + o_flo);
  b.fcur = (unsigned long long*)(ws + o_fc);
  b.look = (unsigned long long*)(ws + o_look);
  b.kbuf = (uint64_t*)(ws + o_kbuf);
  b.sbuf = (uint64_t*)(ws + o_sbuf);
  b.meta = (kc::Meta*)(ws + o_meta);
  b.out_keys = (uint64_t*)okeys;
  b.out_counts = (uint32_t*)ocnts;

  // on any error: let the launched work finish before its buffers go back to the allocator
  auto bail = [&](kc_status stc, const std::string& msg) {
    cudaStreamSynchronize(st);
    cudaGetLastError();
    dev_free(p, okeys);
    dev_free(p, ocnts);
    return fail(stc, msg);
  };
  if (copy_reads &&
      (e = cudaMemcpyAsync((void*)b.reads, reads, L, reads_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st)) !=
          cudaSuccess)
    return bail(KC_ECUDA, std::string("kc_count: copying reads: ") + cudaGetErrorString(e));
  if (!off_dev &&
      (e = cudaMemcpyAsync((void*)b.offsets, offsets, (n_reads + 1) * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return bail(KC_ECUDA, std::string("kc_count: copying offsets: ") + cudaGetErrorString(e));
  if ((e = cudaMemsetAsync(b.meta, 0, sizeof(kc::Meta), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(b.fhist, 0, (size_t)nf_max * 4, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(b.hll, 0, (size_t)kc::kHllRegs * 4, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(b.look, 0, (size_t)nf_max * 8, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(b.cstart, 0, (size_t)(P1 + 1) * 8, st)) != cudaSuccess)
    return bail(KC_ECUDA, std::string("kc_count: clearing scratch: ") + cudaGetErrorString(e));

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
  int launches = kc::launch_phase1(s, b, p->n_sms, (void*)st, mark);
  if (launches >= 0) {
    const int l2 = kc::launch_phase2(s, b, p->n_sms, nf_max, (void*)st, mark);
    launches = l2 >= 0 ? launches + l2 : l2;
  }
  if (launches < 0)
    return bail(KC_ECUDA, std::string("kc_count: launch: ") + cudaGetErrorString((cudaError_t)(-launches)));
  kc::Meta m{};
  if ((e = cudaMemcpyAsync(&m, b.meta, sizeof(m), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return bail(KC_ECUDA, std::string("kc_count: ") + cudaGetErrorString(e));
  p->stats.kernel_launches = (uint32_t)launches;
  if (p->profile) {
    for (int i = 0; i < p->n_marks; ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, p->ev[i], p->ev[i + 1]);
      p->kernel_ms[i] = t;
    }
    p->n_kernel_ms = p->n_marks;
  }
  p->stats.n_partitions = (uint32_t)P1;
  p->stats.n_fine = m.n_fine;
  p->stats.n_overflow_fine = m.n_overflow;
  p->stats.n_deferred_fine = m.n_deferred;
  for (int i = 0; i < 8; ++i) p->stats.phase_cycles[i] = m.phase_cycles[i];
  for (int i = 0; i < 8; ++i) p->stats.sub_cycles[i] = m.sub_cycles[i];
  if (m.status & kc::ST_BAD_OFFSETS) return bail(KC_EINVAL, "kc_count: offsets must start at 0 and be non-decreasing");
  if (m.status & kc::ST_PARTITION_OVERFLOW)
    return bail(KC_EOVERFLOW, "kc_count: one key range holds 2^32 windows or more; use more partitions");
  if (m.status & kc::ST_COUNT_OVERFLOW) return bail(KC_EOVERFLOW, "kc_count: a count exceeds 2^32 - 1");
  if (m.status & kc::ST_TIMEOUT) return bail(KC_ETIMEOUT, "kc_count: a device-side wait timed out");
  if (m.status & kc::ST_INTERNAL) return bail(KC_ECUDA, "kc_count: internal consistency check failed");
  out->n = m.n_distinct;
  out->key_words = (uint32_t)s.kw;
  out->keys = okeys;
  out->counts = (uint32_t*)ocnts;
  out->n_valid_windows = m.n_windows;
  out->capacity = s.cap;
  return KC_OK;
}

}  // extern "C"

// kc_noalloc.cu - kc_count_noalloc: the k-mer count for callers that may not allocate
// device memory at call time.
//
// Some callers cannot call cudaMalloc (or any allocator) when they count: an application
// that has handed all device memory to its own pool up front, or a latency-bound loop in
// which an allocation, with the synchronisation it can imply, is not acceptable.  This
// entry point runs the same kernels as kc_count, but every scratch buffer lives in one
// file-scope device array of fixed size; the caller passes device buffers for the inputs
// and the outputs, and nothing is allocated.
//
// The array is shared by every call in the process and keeps the last call's contents;
// everything that must start at zero is cleared at the start of each call.  Calls that
// overlap on the GPU (other streams, other host threads) race on it.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "kc.h"
#include "kc_internal.h"

// Scratch for one call; KC_NOALLOC_SCRATCH_BYTES is stated in kc.h.  Every GPU that
// loads this library holds it until the process exits.
static __device__ __align__(256) unsigned char kc_noalloc_scratch[KC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;

struct DeviceSetup {
  bool ready = false;
  void* scratch = nullptr;  // device address of kc_noalloc_scratch on this device
  int n_sms = 0;
  size_t smem_optin = 0;
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// errors are reported through kc_last_error, like every other entry point
kc_status nfail(kc_status st, const std::string& msg) {
  kc::set_error_message(msg.c_str());
  return st;
}

bool device_resident(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }
int clog2(uint64_t v) { return v <= 1 ? 0 : 64 - __builtin_clzll(v - 1); }

// One-time set-up on the current device: the scratch array's device address (host code
// cannot use the symbol itself) and the kernels' shared-memory attributes.
kc_status setup_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (dev < 0 || dev >= kMaxDevices) return nfail(KC_EINVAL, "kc_count_noalloc: device ordinal out of range");
  DeviceSetup& d = g_setup[dev];
  if (!d.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, kc_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return nfail(KC_ECUDA, std::string("kc_count_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    int sms = 0, optin = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
      return nfail(KC_ECUDA, std::string("kc_count_noalloc: device attributes: ") + cudaGetErrorString(e));
    const int ce = kc::configure_kernels(dev);
    if (ce) return nfail(KC_ECUDA, std::string("kc_count_noalloc: kernel attributes: ") + cudaGetErrorString((cudaError_t)ce));
    d.scratch = p;
    d.n_sms = sms;
    d.smem_optin = (size_t)optin;
    d.ready = true;
  }
  *out = &d;
  return KC_OK;
}

}  // namespace

extern "C" kc_status kc_count_noalloc(const uint8_t* reads, const uint64_t* offsets, uint64_t n_reads, int k,
                                      int canonical, uint64_t* out_keys, uint32_t* out_counts, uint64_t out_capacity,
                                      uint64_t* n_distinct, uint64_t* n_valid_windows, void* stream) {
  kc::set_error_message("");
  if (k < 1 || k > 64) return nfail(KC_EINVAL, "kc_count_noalloc: k must be in 1..64");
  if (!offsets || !out_keys || !out_counts || !n_distinct || !n_valid_windows)
    return nfail(KC_EINVAL, "kc_count_noalloc: NULL argument");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(KC_ECUDA, std::string("kc_count_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  DeviceSetup* ds = nullptr;
  kc_status st = setup_device(dev, &ds);
  if (st != KC_OK) return st;
  cudaStream_t strm = (cudaStream_t)stream;
  if (!device_resident(offsets) || !device_resident(out_keys) || !device_resident(out_counts))
    return nfail(KC_EINVAL, "kc_count_noalloc: offsets and outputs must be device memory");
  uint64_t first = 0, L = 0;
  if ((e = cudaMemcpyAsync(&first, offsets, 8, cudaMemcpyDeviceToHost, strm)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&L, offsets + n_reads, 8, cudaMemcpyDeviceToHost, strm)) != cudaSuccess ||
      (e = cudaStreamSynchronize(strm)) != cudaSuccess)
    return nfail(KC_ECUDA, std::string("kc_count_noalloc: reading offsets: ") + cudaGetErrorString(e));
  if (first != 0) return nfail(KC_EINVAL, "kc_count_noalloc: offsets[0] must be 0");
  if (L > KC_NOALLOC_MAX_BASES)
    return nfail(KC_EINVAL, "kc_count_noalloc: input of " + std::to_string(L) + " bases exceeds the maximum of " +
                                std::to_string((unsigned long long)KC_NOALLOC_MAX_BASES));
  if (L > 0 && (!reads || !device_resident(reads) || ((uintptr_t)reads & 15) != 0))
    return nfail(KC_EINVAL, "kc_count_noalloc: reads must be device memory aligned to 16 bytes");
  const uint64_t cap = L > 0 ? L : 1;
  if (out_capacity < cap)
    return nfail(KC_EINVAL, "kc_count_noalloc: out_capacity must be at least offsets[n_reads] (the number of bases)");

  // shape: the same choices kc_count makes for this input size
  kc::Shape s{};
  s.L = L;
  s.n_reads = n_reads;
  s.n_words = (L + 31) / 32;
  s.n_tiles = (s.n_words + kc::kTileWords - 1) / kc::kTileWords;
  s.k = k;
  s.canonical = canonical ? 1 : 0;
  s.kw = k <= 32 ? 1 : 2;
  {
    const int want = clog2(L / kc::coarse_bases(s.kw) + 1);  // the same rule as kc_count
    s.b1 = want < 11 ? want : 11;
  }
  const int P1 = 1 << s.b1;
  s.bT_max = kc::table_log2_max(s.kw, ds->smem_optin);
  s.tail = s.bT_max >= 10 ? 1024 : (1 << s.bT_max);
  const double ft = (double)(1u << s.bT_max) * 0.55;
  s.fine_target = ft < 16 ? 16u : (uint32_t)ft;
  s.cap = cap;
  const uint64_t nf_bound = cap / s.fine_target + (uint64_t)P1 + 1;
  const uint64_t nf_lim = (uint64_t)P1 * kc::kMaxFine;
  const uint32_t nf_max = (uint32_t)(nf_bound < nf_lim ? nf_bound : nf_lim);
  s.nf_max = nf_max;
  s.smem_budget = ds->smem_optin;
  s.profile = 0;
  s.defer_all = 0;

  // scratch layout inside the static array
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = up256(o + (bytes ? bytes : 1));
    return at;
  };
  const size_t o_codes = take(s.n_words * 8), o_inv = take(s.n_words * 4), o_tf = take(s.n_tiles * 8);
  const size_t o_hist = take(s.n_tiles * P1 * 4), o_toff = take(s.n_tiles * P1 * 8);
  const size_t o_cst = take((size_t)(P1 + 1) * 8), o_fb = take((size_t)(P1 + 1) * 4), o_fl = take((size_t)P1 * 4);
  const size_t o_hll = take((size_t)kc::kHllRegs * 4);
  const size_t o_fh = take((size_t)nf_max * 4), o_fo = take((size_t)(nf_max + 1) * 8);
  const size_t o_flo = take((size_t)(nf_max + 1) * 4);
  const size_t o_fc = take((size_t)nf_max * 8), o_look = take((size_t)nf_max * 8);
  const size_t o_kbuf = take(cap * s.kw * 8), o_sbuf = take(cap * s.kw * 8), o_meta = take(sizeof(kc::Meta));
  if (o > (size_t)KC_NOALLOC_SCRATCH_BYTES)
    return nfail(KC_EINVAL, "kc_count_noalloc: input needs more scratch than the fixed array holds");
  uint8_t* ws = (uint8_t*)ds->scratch;
  kc::Buffers b{};
  b.reads = reads;
  b.offsets = offsets;
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
  b.out_keys = out_keys;
  b.out_counts = out_counts;

  // the array keeps the previous call's contents: clear what the kernels expect at zero
  if ((e = cudaMemsetAsync(b.meta, 0, sizeof(kc::Meta), strm)) != cudaSuccess ||
      (e = cudaMemsetAsync(b.fhist, 0, (size_t)nf_max * 4, strm)) != cudaSuccess ||
      (e = cudaMemsetAsync(b.hll, 0, (size_t)kc::kHllRegs * 4, strm)) != cudaSuccess ||
      (e = cudaMemsetAsync(b.look, 0, (size_t)nf_max * 8, strm)) != cudaSuccess ||
      (e = cudaMemsetAsync(b.cstart, 0, (size_t)(P1 + 1) * 8, strm)) != cudaSuccess)
    return nfail(KC_ECUDA, std::string("kc_count_noalloc: clearing scratch: ") + cudaGetErrorString(e));
  kc::Marker none;
  int launches = kc::launch_phase1(s, b, ds->n_sms, (void*)strm, none);
  if (launches >= 0) {
    const int l2 = kc::launch_phase2(s, b, ds->n_sms, nf_max, (void*)strm, none);
    launches = l2 >= 0 ? launches + l2 : l2;
  }
  kc::Meta m{};
  const cudaError_t ce = cudaMemcpyAsync(&m, b.meta, sizeof(m), cudaMemcpyDeviceToHost, strm);
  const cudaError_t se = cudaStreamSynchronize(strm);
  if (launches < 0)
    return nfail(KC_ECUDA, std::string("kc_count_noalloc: launch: ") + cudaGetErrorString((cudaError_t)(-launches)));
  if (ce != cudaSuccess || se != cudaSuccess)
    return nfail(KC_ECUDA, std::string("kc_count_noalloc: ") + cudaGetErrorString(ce != cudaSuccess ? ce : se));
  if (m.status & kc::ST_BAD_OFFSETS) return nfail(KC_EINVAL, "kc_count_noalloc: offsets must be non-decreasing");
  if (m.status & kc::ST_PARTITION_OVERFLOW) return nfail(KC_EOVERFLOW, "kc_count_noalloc: a key range holds 2^32 windows");
  if (m.status & kc::ST_COUNT_OVERFLOW) return nfail(KC_EOVERFLOW, "kc_count_noalloc: a count exceeds 2^32 - 1");
  if (m.status & kc::ST_TIMEOUT) return nfail(KC_ETIMEOUT, "kc_count_noalloc: a device-side wait timed out");
  if (m.status & kc::ST_INTERNAL) return nfail(KC_ECUDA, "kc_count_noalloc: internal consistency check failed");
  *n_distinct = m.n_distinct;
  *n_valid_windows = m.n_windows;
  return KC_OK;
}

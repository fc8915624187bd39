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
  size_t smem_per_sm = 0;
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
    int sms = 0, optin = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
      return nfail(KC_ECUDA, std::string("kc_count_noalloc: device attributes: ") + cudaGetErrorString(e));
    const int ce = kc::configure_kernels(dev);
    if (ce) return nfail(KC_ECUDA, std::string("kc_count_noalloc: kernel attributes: ") + cudaGetErrorString((cudaError_t)ce));
    d.scratch = p;
    d.n_sms = sms;
    d.smem_optin = (size_t)optin;
    d.smem_per_sm = (size_t)per_sm;
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
  // the kernels read offsets as 8-byte words, write counts as 4-byte words and keys as 8- or
  // (k > 32) 16-byte words: a misaligned buffer is refused before anything is launched
  if (((uintptr_t)offsets & 7) != 0 || ((uintptr_t)out_counts & 3) != 0 ||
      ((uintptr_t)out_keys & (k > 32 ? 15 : 7)) != 0)
    return nfail(KC_EINVAL, "kc_count_noalloc: offsets must be 8-byte aligned, out_counts 4-byte aligned and out_keys "
                            "8-byte aligned (16-byte for k > 32)");
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

  // shape and scratch layout: the same choices kc_count makes for this input size
  kc::ShapeOpts so;
  so.smem_optin = ds->smem_optin;
  so.smem_per_sm = ds->smem_per_sm;
  kc::Shape s{};
  kc::Layout lay{};
  kc::make_shape(so, L, n_reads, k, canonical, false, false, s, lay);
  if (lay.total > (size_t)KC_NOALLOC_SCRATCH_BYTES)
    return nfail(KC_EINVAL, "kc_count_noalloc: input needs more scratch than the fixed array holds");
  kc::Buffers b = kc::layout_buffers(lay, (uint8_t*)ds->scratch);
  b.reads = reads;
  b.offsets = offsets;
  b.out_keys = out_keys;
  b.out_counts = out_counts;

  // the array keeps the previous call's contents: clear what the kernels expect at zero
  if ((e = (cudaError_t)kc::clear_scratch(s, b, (void*)strm)) != cudaSuccess)
    return nfail(KC_ECUDA, std::string("kc_count_noalloc: clearing scratch: ") + cudaGetErrorString(e));
  kc::Marker none;
  int launches = kc::launch_phase1(s, b, ds->n_sms, (void*)strm, none);
  if (launches >= 0) {
    const int l2 = kc::launch_phase2(s, b, ds->n_sms, (uint32_t)s.nf_max, (void*)strm, none);
    launches = l2 >= 0 ? launches + l2 : l2;
  }
  kc::Meta m{};
  const cudaError_t ce = cudaMemcpyAsync(&m, b.meta, sizeof(m), cudaMemcpyDeviceToHost, strm);
  const cudaError_t se = cudaStreamSynchronize(strm);
  if (launches < 0)
    return nfail(KC_ECUDA, std::string("kc_count_noalloc: launch: ") + cudaGetErrorString((cudaError_t)(-launches)));
  if (ce != cudaSuccess || se != cudaSuccess)
    return nfail(KC_ECUDA, std::string("kc_count_noalloc: ") + cudaGetErrorString(ce != cudaSuccess ? ce : se));
  // the status record must describe a result that fits the caller's buffers
  if (m.n_windows > L || m.n_distinct > m.n_windows || m.n_fine > s.nf_max || m.n_deferred > m.n_fine ||
      m.n_distinct > out_capacity)
    return nfail(KC_ECUDA, "kc_count_noalloc: inconsistent status record");
  if (m.status & kc::ST_BAD_OFFSETS) return nfail(KC_EINVAL, "kc_count_noalloc: offsets must be non-decreasing");
  if (m.status & kc::ST_PARTITION_OVERFLOW) return nfail(KC_EOVERFLOW, "kc_count_noalloc: a key range holds 2^32 windows");
  if (m.status & kc::ST_COUNT_OVERFLOW) return nfail(KC_EOVERFLOW, "kc_count_noalloc: a count exceeds 2^32 - 1");
  if (m.status & kc::ST_TIMEOUT) return nfail(KC_ETIMEOUT, "kc_count_noalloc: a device-side wait timed out");
  if (m.status & kc::ST_INTERNAL) return nfail(KC_ECUDA, "kc_count_noalloc: internal consistency check failed");
  *n_distinct = m.n_distinct;
  *n_valid_windows = m.n_windows;
  return KC_OK;
}

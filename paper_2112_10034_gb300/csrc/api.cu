// Library-wide pieces of the C ABI: status strings, version, the device-side
// status word that bounded waits report into, the spin limit, and the cached
// SM count used to size persistent grids.
#include <mutex>

#include "cox_common.cuh"

namespace {

__device__ unsigned g_dev_status;  // bit flags (cox::kDevTimeout)

using cox::kMaxDevices;
unsigned* g_status_addr[kMaxDevices];
int g_sms[kMaxDevices];
std::mutex g_mu;
uint32_t g_spin_limit = 1u << 22;

int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return 0;
  return d;
}

}  // namespace

namespace cox {

// Device address of the status word on the current device (looked up once per
// device; make the first library call of a device outside stream capture).
unsigned* device_status_word() {
  const int d = current_device();
  if (!g_status_addr[d]) {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_status_addr[d]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_dev_status) == cudaSuccess) g_status_addr[d] = static_cast<unsigned*>(p);
    }
  }
  return g_status_addr[d];
}

uint32_t spin_limit() { return g_spin_limit; }

int device_index() { return current_device(); }

int sm_count() {
  const int d = current_device();
  if (!g_sms[d]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v < 1) v = 1;
    g_sms[d] = v;
  }
  return g_sms[d];
}

}  // namespace cox

extern "C" const char* cox_status_string(cox_status s) {
  switch (s) {
    case COX_OK: return "COX_OK";
    case COX_EINVAL: return "COX_EINVAL: invalid argument";
    case COX_EUNSUPPORTED: return "COX_EUNSUPPORTED: outside the supported scope";
    case COX_ECUDA: return "COX_ECUDA: CUDA runtime error";
    case COX_ENOMEM: return "COX_ENOMEM: workspace or budget too small";
    case COX_ETIMEOUT: return "COX_ETIMEOUT: a bounded device wait ran out";
    case COX_EBUSY: return "COX_EBUSY: resource busy";
    default: return "COX_?: unknown status";
  }
}

extern "C" int cox_version(void) { return 100; }

extern "C" void cox_set_spin_limit(uint32_t polls) { g_spin_limit = polls ? polls : (1u << 22); }

extern "C" cox_status cox_device_status(void* stream) {
  if (cudaStreamSynchronize(cox::as_stream(stream)) != cudaSuccess) return COX_ECUDA;
  unsigned* w = cox::device_status_word();
  if (!w) return COX_ECUDA;
  unsigned v = 0;
  if (cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return COX_ECUDA;
  if (v == 0) return COX_OK;
  if (cudaMemset(w, 0, sizeof v) != cudaSuccess) return COX_ECUDA;
  return (v & cox::kDevTimeout) ? COX_ETIMEOUT : COX_ECUDA;
}

// Morton ordering without any device allocation.
//
// mp_morton_order keeps its sort keys in a workspace that the context
// allocates (and grows) with cudaMalloc.  Some callers cannot allow that:
// code that enqueues work while a CUDA graph is being captured (an
// allocation is not a stream operation and breaks the capture), latency-
// critical loops that must not stall on the allocator's implicit device
// synchronisation, and programs whose device memory is owned by another
// allocator (a caching pool such as PyTorch's) or by a fixed budget.  This
// variant sorts in a fixed buffer that lives in the library's own device
// image instead.
//
// The buffer is a file-scope __device__ array, so every GPU that loads the
// library holds it (MP_NOALLOC_MAX_POINTS keys of 8 bytes, 1 MiB) until the
// process exits.  In host code the array's name is only a host-side
// placeholder; the device address is looked up once per device with
// cudaGetSymbolAddress while that device is current, and that address is
// what the kernels receive.  The looked-up address belongs to the device's
// current context: after a cudaDeviceReset the runtime creates a new
// context (and loads the module again), so the cache records the context it
// was filled in and looks the address up again when the context differs.
#include <cstdio>
#include <mutex>

#include "../../include/mpchol.h"
#include "mp_internal.h"

namespace mp {
void set_error_text(const char* msg);
}

namespace {

static __device__ __align__(256) unsigned long long g_sort_keys[MP_NOALLOC_MAX_POINTS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct KeysAddr {
  void* ctx;                   // context the address was looked up in
  unsigned long long* addr;
};
KeysAddr g_keys[kMaxDevices] = {};

// cuCtxGetCurrent through the runtime's driver entry point (no link
// against libcuda); returns the calling thread's current context or null.
void* current_context() {
  typedef int (*Fn)(void**);
  static Fn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<Fn>(f);
  }();
  void* c = nullptr;
  if (!fn || fn(&c) != 0) return nullptr;
  return c;
}

mp_status cuda_fail(const char* what, cudaError_t e) {
  char msg[256];
  snprintf(msg, sizeof msg, "mp_morton_order_noalloc: %s: %s", what, cudaGetErrorString(e));
  mp::set_error_text(msg);
  return MP_ERR_CUDA;
}

}  // namespace

extern "C" mp_status mp_morton_order_noalloc(int64_t n, const double* d_locs_in,
                                             double* d_locs_out, int64_t* d_perm, void* stream) {
  if (!d_locs_in || !d_locs_out || !d_perm || d_locs_in == d_locs_out) {
    mp::set_error_text("mp_morton_order_noalloc: null or aliased pointer");
    return MP_ERR_ARG;
  }
  if (n < 1 || n > MP_NOALLOC_MAX_POINTS) {
    mp::set_error_text("mp_morton_order_noalloc: n must be in [1, MP_NOALLOC_MAX_POINTS = 131072]; "
                       "use mp_morton_order for more points");
    return MP_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) {
    mp::set_error_text("mp_morton_order_noalloc: device index beyond the library's table of 64");
    return MP_ERR_ARG;
  }
  // an error left by earlier work would otherwise be reported as this
  // call's: say so and leave it in place for its owner
  e = cudaPeekAtLastError();
  if (e != cudaSuccess) return cuda_fail("an earlier CUDA error is pending (not cleared)", e);
  unsigned long long* keys = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    void* ctx = current_context();
    if (!g_keys[dev].addr || !ctx || g_keys[dev].ctx != ctx) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_sort_keys);
      if (e != cudaSuccess || !p) return cuda_fail("cudaGetSymbolAddress", e);
      // the look-up makes the runtime's context current when none was
      g_keys[dev].ctx = ctx ? ctx : current_context();
      g_keys[dev].addr = static_cast<unsigned long long*>(p);
    }
    keys = g_keys[dev].addr;
  }
  int64_t n2 = 1024;
  while (n2 < n) n2 <<= 1;
  // every one of the n2 keys is written by the key kernel before the sort
  // reads it, so nothing left by an earlier call needs clearing
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mp::launch_morton_keys(d_locs_in, n, n2, keys, s);
  mp::launch_bitonic(keys, n2, s);
  mp::launch_morton_gather(keys, d_locs_in, n, d_locs_out, d_perm, s);
  e = cudaGetLastError();
  return e == cudaSuccess ? MP_OK : cuda_fail("kernel launch", e);
}

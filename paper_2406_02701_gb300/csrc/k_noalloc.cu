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
// what the kernels receive.
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
unsigned long long* g_keys_addr[kMaxDevices] = {};

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
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MP_ERR_CUDA;
  unsigned long long* keys = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_keys_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_sort_keys) != cudaSuccess || !p) {
        mp::set_error_text("mp_morton_order_noalloc: cudaGetSymbolAddress failed");
        return MP_ERR_CUDA;
      }
      g_keys_addr[dev] = static_cast<unsigned long long*>(p);
    }
    keys = g_keys_addr[dev];
  }
  int64_t n2 = 1024;
  while (n2 < n) n2 <<= 1;
  // every one of the n2 keys is written by the key kernel before the sort
  // reads it, so nothing left by an earlier call needs clearing
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mp::launch_morton_keys(d_locs_in, n, n2, keys, s);
  mp::launch_bitonic(keys, n2, s);
  mp::launch_morton_gather(keys, d_locs_in, n, d_locs_out, d_perm, s);
  return cudaPeekAtLastError() == cudaSuccess ? MP_OK : MP_ERR_CUDA;
}

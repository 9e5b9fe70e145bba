// Autotuner of tile sizes and schedules.
//
// The tiled multi-precision extension (Sec. 7) fixes neither the tile size
// nor how the work of a step is scheduled; on GB300 the best choice depends
// on the sizes of the matrices, how many run together, and which formats
// their tiles take.  The tuner measures instead of assuming: it builds the
// real plan of a candidate schedule, runs it (one warm-up, then the best of
// two launches timed with CUDA events on the caller's stream) and keeps the
// fastest.  The search is coordinate descent from the default schedule --
// first the tile size b, then, at the best b, each schedule flag toggled
// once (the other task-graph block of the diagonal tiles, the FP64 panel
// solve instead of the integer-digit tensor-core products, the 4-slot ring
// of the 16-/8-bit tensor-core updates) -- so a batch costs about eight
// timed launches, not the product of all choices.
//
// Results can be kept in a plain text cache file, one "key b flags ms" line
// per tuned workload; the key names the GPU (name and SM count) and a
// coarse signature of the workload, so a later run with a workload of the
// same kind takes the choice without timing.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mpchol.h"

namespace mp {
void set_error_text(const char* msg);
}

namespace {

std::string gpu_key(mp_ctx* ctx) {
  (void)ctx;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p{};
  cudaGetDeviceProperties(&p, dev);
  char buf[320];
  snprintf(buf, sizeof buf, "%s/%dsm", p.name, p.multiProcessorCount);
  std::string s(buf);
  for (char& c : s)
    if (c == ' ' || c == '\t') c = '_';
  return s;
}

bool cache_get(const char* path, const std::string& key, mp_tuned* out) {
  if (!path || !*path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char k[768];
    int b = 0;
    unsigned flags = 0;
    double ms = 0;
    if (sscanf(line, "%767s %d %u %lf", k, &b, &flags, &ms) == 4 && key == k) {
      out->b = b;
      out->flags = flags;
      out->ms = ms;
      found = true;                    // the last matching line wins
    }
  }
  fclose(f);
  if (found) {
    out->from_cache = 1;
    out->tried = 0;
  }
  return found;
}

void cache_put(const char* path, const std::string& key, const mp_tuned& t) {
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %u %.6f\n", key.c_str(), t.b, t.flags, t.ms);
  fclose(f);
}

// Best of two timed runs of `run` after one warm-up; ms < 0 on failure.
template <class Run>
double time_runs(cudaStream_t s, Run run) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.0;
  }
  double best = -1.0;
  if (run() == MP_OK && cudaStreamSynchronize(s) == cudaSuccess) {
    for (int r = 0; r < 2; ++r) {
      cudaEventRecord(e0, s);
      if (run() != MP_OK) { best = -1.0; break; }
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { best = -1.0; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (best < 0 || ms < best) best = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// Coordinate descent over (b, flags); `measure(b, flags)` returns ms or < 0.
template <class Measure>
mp_status search(const std::vector<int>& bs, uint32_t base_flags, Measure measure, mp_tuned* out) {
  out->tried = 0;
  out->from_cache = 0;
  int best_b = 0;
  uint32_t best_f = base_flags;
  double best = -1.0;
  for (int b : bs) {
    const double ms = measure(b, base_flags);
    ++out->tried;
    if (ms > 0 && (best < 0 || ms < best)) { best = ms; best_b = b; }
  }
  if (best < 0) {
    mp::set_error_text("autotuner: no candidate schedule ran");
    return MP_ERR_CUDA;
  }
  // the default block of the diagonal task graph at the best b is 16 for
  // b in [384, 768] and 32 otherwise: try the other one
  const uint32_t other_dag = (best_b >= 384 && best_b <= 768) ? MP_TMAT_DAG32 : MP_TMAT_DAG16;
  for (uint32_t toggle : {other_dag, (uint32_t)MP_TMAT_FP64_PANEL, (uint32_t)MP_TMAT_LOWP_RING4}) {
    const uint32_t f = best_f | toggle;
    const double ms = measure(best_b, f);
    ++out->tried;
    if (ms > 0 && ms < best) { best = ms; best_f = f; }
  }
  out->b = best_b;
  out->flags = best_f;
  out->ms = best;
  return MP_OK;
}

int quartile_256(std::vector<int64_t> v, double q) {
  std::sort(v.begin(), v.end());
  const int64_t x = v[(size_t)std::min<double>(v.size() - 1, std::floor(q * (v.size() - 1) + 0.5))];
  return (int)((x + 255) / 256 * 256);
}

// splitmix64: the tuner's own synthetic points
uint64_t mix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" mp_status mp_tune_batch(mp_ctx* ctx, int32_t count, const mp_request* reqs,
                                   const char* cache_path, void* stream, mp_tuned* out) {
  if (!ctx || !reqs || !out || count < 1) return MP_ERR_ARG;
  std::vector<int64_t> ns(count);
  int64_t nmax = 0, rhs = 0;
  int far = 0;
  double eps = 0.0;
  for (int r = 0; r < count; ++r) {
    if (reqs[r].h_map) {
      // an explicit map is tied to the b it was built for
      mp::set_error_text("mp_tune_batch: request maps must be given by rule (h_map NULL) when b is tuned");
      return MP_ERR_ARG;
    }
    ns[r] = reqs[r].n;
    nmax = std::max(nmax, reqs[r].n);
    rhs += reqs[r].nrhs;
    far = std::max(far, reqs[r].rule_eps > 0 ? (int)reqs[r].rule_far : 0);
    eps = std::max(eps, reqs[r].rule_eps);
  }
  char sig[512];
  snprintf(sig, sizeof sig, "batch|%s|count=%d|nq=%d,%d,%d,%d,%d|rhs=%lld|far=%d|eps=%.3g",
           gpu_key(ctx).c_str(), count, quartile_256(ns, 0.0), quartile_256(ns, 0.25), quartile_256(ns, 0.5),
           quartile_256(ns, 0.75), quartile_256(ns, 1.0), (long long)rhs, far, eps);
  const std::string key(sig);
  if (cache_get(cache_path, key, out)) return MP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* d_ll = nullptr;
  int32_t* d_st = nullptr;
  if (cudaMalloc(&d_ll, sizeof(double) * rhs) != cudaSuccess) return MP_ERR_OOM;
  if (cudaMalloc(&d_st, sizeof(int32_t) * count) != cudaSuccess) {
    cudaFree(d_ll);
    return MP_ERR_OOM;
  }
  std::vector<int> bs;
  for (int b : {128, 256, 384, 512})
    if (b == 128 || (int64_t)b <= std::max<int64_t>(nmax, 128)) bs.push_back(b);
  auto measure = [&](int b, uint32_t flags) -> double {
    mp_batch* B = nullptr;
    if (mp_batch_create_ex(ctx, count, reqs, b, flags, stream, &B) != MP_OK) return -1.0;
    const double ms = time_runs(s, [&] { return mp_batch_run(B, d_ll, d_st); });
    cudaStreamSynchronize(s);
    mp_batch_destroy(B);
    return ms;
  };
  mp_status st = search(bs, 0u, measure, out);
  cudaFree(d_ll);
  cudaFree(d_st);
  if (st == MP_OK) cache_put(cache_path, key, *out);
  return st;
}

extern "C" mp_status mp_tune_tmat(mp_ctx* ctx, int64_t n, uint8_t far_dt, double eps,
                                  int32_t refine_iters, const char* cache_path, void* stream,
                                  mp_tuned* out) {
  if (!ctx || !out || n < 1 || far_dt > MP_E4M3 || !(eps > 0) || refine_iters < 0) return MP_ERR_ARG;
  char sig[512];
  snprintf(sig, sizeof sig, "tmat|%s|n=%lld|far=%d|eps=%.3g|refine=%d", gpu_key(ctx).c_str(), (long long)n,
           (int)far_dt, eps, refine_iters);
  const std::string key(sig);
  if (cache_get(cache_path, key, out)) return MP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // a jittered grid of the unit square (Morton-ordered on the device) and
  // one standard normal-like right-hand side (a sum of uniforms: the tuner
  // times work, not statistics)
  const int64_t m = (int64_t)std::ceil(std::sqrt((double)n));
  std::vector<double> locs(2 * n), z(n);
  uint64_t seed = 0x5eed ^ (uint64_t)n;
  auto uni = [&] { return (double)(mix64(seed) >> 11) * 0x1p-53; };
  for (int64_t i = 0; i < n; ++i) {
    locs[2 * i] = ((double)(i % m) + uni()) / (double)m;
    locs[2 * i + 1] = ((double)(i / m) + uni()) / (double)m;
    z[i] = uni() + uni() + uni() - 1.5;
  }
  double *d_in = nullptr, *d_sorted = nullptr, *d_z = nullptr, *d_ll = nullptr;
  int64_t* d_perm = nullptr;
  mp_status st = MP_OK;
  if (cudaMalloc(&d_in, sizeof(double) * 2 * n) != cudaSuccess ||
      cudaMalloc(&d_sorted, sizeof(double) * 2 * n) != cudaSuccess ||
      cudaMalloc(&d_z, sizeof(double) * n) != cudaSuccess || cudaMalloc(&d_ll, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_perm, sizeof(int64_t) * n) != cudaSuccess)
    st = MP_ERR_OOM;
  std::vector<double> sorted(2 * n);
  if (st == MP_OK && (cudaMemcpyAsync(d_in, locs.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s) ||
                      cudaMemcpyAsync(d_z, z.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s)))
    st = MP_ERR_CUDA;
  if (st == MP_OK) st = mp_morton_order(ctx, n, d_in, d_sorted, d_perm, stream);
  if (st == MP_OK && (cudaMemcpyAsync(sorted.data(), d_sorted, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, s) ||
                      cudaStreamSynchronize(s)))
    st = MP_ERR_CUDA;
  const mp_matern cov{1.0, 0.05, 1.5, 1e-4};
  if (st == MP_OK) {
    std::vector<int> bs;
    for (int b : {128, 256, 384, 512, 1024})
      if (b == 128 || b <= n) bs.push_back(b);
    auto measure = [&](int b, uint32_t flags) -> double {
      const int nt = (int)((n + b - 1) / b);
      std::vector<uint8_t> map((size_t)nt * nt);
      if (mp_map_bound(n, b, sorted.data(), cov, 2, MP_F32, far_dt, eps, map.data()) != MP_OK) return -1.0;
      mp_tmat* t = nullptr;
      const uint32_t f = flags | (refine_iters > 0 ? MP_TMAT_KEEP_SIGMA : 0u);
      if (mp_tmat_create(ctx, n, b, map.data(), f, stream, &t) != MP_OK) return -1.0;
      const double ms = time_runs(s, [&] {
        mp_status r = mp_generate_matern(t, d_sorted, cov);
        if (r == MP_OK) r = mp_chol(t, nullptr, nullptr);
        if (r == MP_OK) r = mp_loglik(t, d_z, n, 1, refine_iters, d_ll, nullptr, nullptr);
        return r;
      });
      cudaStreamSynchronize(s);
      mp_tmat_destroy(t);
      return ms;
    };
    st = search(bs, 0u, measure, out);
  }
  cudaFree(d_in);
  cudaFree(d_sorted);
  cudaFree(d_z);
  cudaFree(d_ll);
  cudaFree(d_perm);
  if (st == MP_OK) cache_put(cache_path, key, *out);
  return st;
}

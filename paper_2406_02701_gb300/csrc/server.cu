// Continuous-batching server of Gaussian log-likelihood requests (the stream
// of likelihood evaluations an MLE search issues, Sec. 6.2).
//
// Requests arrive with host buffers and wait in a queue.  mp_server_poll
// retires requests whose work has finished on the GPU and admits queued
// requests -- in arrival order, later ones backfilling when an earlier one
// does not fit -- while a stream slot is free and the request's device
// footprint fits the HBM budget.  Every admitted request runs on its own
// stream, so the work of requests that arrive while others are on the GPU
// overlaps on the device.  A finished request keeps its factor on the
// device until it is released; when a new request needs the memory, the
// least recently finished unreleased factors are evicted.
//
// Per request: Morton order of the locations and the precision map are
// computed on the host at admission (the map from a closed-form upper bound
// of each tile's norm, see plan_map), the sorted locations and right-hand
// sides are copied to the device, and the tile generation, the
// factorisation graph and the log-likelihood graph are enqueued on the
// request's stream, followed by the copy of the results to pinned memory
// and an event.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mpchol.h"
#include "mp_internal.h"

namespace mp {
void set_error_text(const char* msg);
}

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

uint32_t spread16(uint32_t v) {
  uint32_t k = 0;
  for (int bit = 0; bit < 16; ++bit) k |= ((v >> bit) & 1u) << (2 * bit);
  return k;
}

// Morton order on the host, same definition as mp_morton_order.
std::vector<int64_t> morton_perm(const double* locs, int64_t n) {
  std::vector<std::pair<uint64_t, int64_t>> key(n);
  for (int64_t i = 0; i < n; ++i) {
    double qx = std::max(std::min(std::floor(locs[2 * i] * 65536.0), 65535.0), 0.0);
    double qy = std::max(std::min(std::floor(locs[2 * i + 1] * 65536.0), 65535.0), 0.0);
    uint64_t k = spread16((uint32_t)qx) | ((uint64_t)spread16((uint32_t)qy) << 1);
    key[i] = {k, i};
  }
  std::sort(key.begin(), key.end());
  std::vector<int64_t> p(n);
  for (int64_t i = 0; i < n; ++i) p[i] = key[i].second;
  return p;
}

// C(r): the closed forms, or the generation kernels' table for other nu
double matern(double r, const mp_matern& c, const std::vector<double>& tab, int e0) {
  double x = r / c.range;
  if (!mp::matern_nu_closed(c.nu)) return c.sigma2 * mp::matern_nu_host(tab.data(), e0, x);
  double poly = c.nu == 0.5 ? 1.0 : c.nu == 1.5 ? 1.0 + x : 1.0 + x + x * x / 3.0;
  return c.sigma2 * poly * std::exp(-x);
}

double uround(int dt) {
  switch (dt) {
    case MP_F32: return std::ldexp(1.0, -24);
    case MP_BF16: return std::ldexp(1.0, -8);
    case MP_F16: return std::ldexp(1.0, -11);
    case MP_E4M3: return std::ldexp(1.0, -4);
    default: return std::ldexp(1.0, -53);
  }
}

}  // namespace

// Map of a request: diagonal FP64, |i-j| <= band in near_dt, a farther tile
// in far_dt when u(far) * B_ij <= eps * ||A||_F^lo / NT, where
// B_ij = sqrt(rows_i cols_j) C(d_ij) >= ||A_ij||_F bounds the tile's norm
// with d_ij the distance between the bounding boxes of the two tiles'
// (Morton-sorted) points (the covariance decreases with distance), and
// ||A||_F^lo = sqrt(n) (sigma2 + nugget) <= ||A||_F (the diagonal alone).
// Both bounds only make the map more conservative than the exact-norm rule.
extern "C" mp_status mp_map_bound(int64_t n, int32_t b, const double* h_sorted_locs, mp_matern c,
                                  int32_t band, uint8_t near_dt, uint8_t far_dt, double eps,
                                  uint8_t* h_map) {
  if (n < 1 || b < 1 || !h_sorted_locs || !h_map || band < 0 || !(eps > 0)) return MP_ERR_ARG;
  if (!(c.range > 0) || !(c.sigma2 > 0)) return MP_ERR_ARG;
  std::vector<double> tab;
  int e0 = 0;
  if (!mp::matern_nu_valid(c.nu) || (!mp::matern_nu_closed(c.nu) && mp::matern_nu_table(c.nu, tab, &e0))) {
    mp::set_error_text("mp_map_bound: nu must be in (0, 16]");
    return MP_ERR_ARG;
  }
  const int nt = (int)((n + b - 1) / b);
  std::vector<double> lo_x(nt), hi_x(nt), lo_y(nt), hi_y(nt);
  std::vector<int64_t> cnt(nt);
  for (int t = 0; t < nt; ++t) {
    lo_x[t] = lo_y[t] = 1e300;
    hi_x[t] = hi_y[t] = -1e300;
    const int64_t r0 = (int64_t)t * b, r1 = std::min<int64_t>(n, r0 + b);
    cnt[t] = r1 - r0;
    for (int64_t r = r0; r < r1; ++r) {
      lo_x[t] = std::min(lo_x[t], h_sorted_locs[2 * r]);
      hi_x[t] = std::max(hi_x[t], h_sorted_locs[2 * r]);
      lo_y[t] = std::min(lo_y[t], h_sorted_locs[2 * r + 1]);
      hi_y[t] = std::max(hi_y[t], h_sorted_locs[2 * r + 1]);
    }
  }
  const double fro_lo = std::sqrt((double)n) * (c.sigma2 + c.nugget);
  const double bound = eps * fro_lo / nt;
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < nt; ++j) {
      uint8_t m = 255;
      if (i == j) m = MP_F64;
      else if (j < i) {
        if (i - j <= band) m = near_dt;
        else {
          double dx = std::max(0.0, std::max(lo_x[i] - hi_x[j], lo_x[j] - hi_x[i]));
          double dy = std::max(0.0, std::max(lo_y[i] - hi_y[j], lo_y[j] - hi_y[i]));
          double B = std::sqrt((double)cnt[i] * (double)cnt[j]) * matern(std::sqrt(dx * dx + dy * dy), c, tab, e0);
          m = uround(far_dt) * B <= bound ? far_dt : near_dt;
        }
      }
      h_map[(size_t)i * nt + j] = m;
    }
  return MP_OK;
}

struct Job {
  int64_t id = 0;
  int64_t n = 0;
  int32_t nrhs = 1, refine = 0, b = 0;
  mp_matern cov{};
  double t_submit = 0, t_admit = 0, t_done = 0;
  std::vector<double> locs, z;          // host copies (locs sorted at admission)
  int slot = -1;
  uint32_t flags = 0;                   // schedule flags of its matrix
  int64_t bytes = 0;
  mp_tmat* t = nullptr;
  double* d_in = nullptr;               // device: sorted locs, z, outputs
  double* h_out = nullptr;              // pinned: ll[nrhs], quad[nrhs], logdet, info
  cudaEvent_t done = nullptr;
  bool finished = false, released = false;
  int32_t status = MP_OK;
  int n_low = 0, n_tiles = 0;
};

struct mp_server {
  mp_ctx* ctx = nullptr;
  int64_t budget = 0, used = 0;
  int max_slots = 0;
  double eps = 1e-6;
  uint8_t far_dt = MP_BF16;
  int32_t band = 2;
  std::vector<cudaStream_t> streams;
  std::vector<Job*> slot_job;
  std::deque<Job*> queue;
  std::vector<Job*> jobs;               // all jobs by id order
  std::deque<Job*> kept;                // finished, unreleased (LRU order)
  int64_t next_id = 1;
  int32_t inject_oom = 0;               // admissions whose input allocation is made to fail
  // tuned schedules by request size (ascending n): b and flags
  std::vector<int64_t> tuned_n;
  std::vector<int32_t> tuned_b;
  std::vector<uint32_t> tuned_flags;
};

namespace {

int pick_b(int64_t n) { return n <= 2048 ? 128 : n <= 8192 ? 256 : 512; }

// Tile size and schedule flags of a request: the tuned choice of the
// smallest tuned size >= n (the largest when n exceeds them all), else the
// fixed rule.
void pick_schedule(const mp_server* S, int64_t n, int* b, uint32_t* flags) {
  *b = pick_b(n);
  *flags = 0;
  if (S->tuned_n.empty()) return;
  size_t k = 0;
  while (k + 1 < S->tuned_n.size() && S->tuned_n[k] < n) ++k;
  *b = S->tuned_b[k];
  *flags = S->tuned_flags[k];
}

// Device bytes of a request: tiles and workspace, estimated from the sizes
// before the plan exists (FP64 worst case for the tiles, the Sigma copy,
// scratch and vectors).
int64_t footprint(int64_t n, int b, int nrhs, bool sigma) {
  const int64_t nt = (n + b - 1) / b, N = nt * b;
  int64_t tiles = nt * (nt + 1) / 2 * (int64_t)b * b * 8;
  int64_t extra = (nt * 2 + nt + 8) * (int64_t)b * b * 8;     // inverses, shadows, panel slots
  int64_t vec = N * nrhs * 8 * 6 + N * 8;
  return tiles * (sigma ? 2 : 1) + extra + vec;
}

void free_job_device(mp_server* S, Job* J) {
  if (J->t) { mp_tmat_destroy(J->t); J->t = nullptr; }
  if (J->d_in) { cudaFreeAsync(J->d_in, S->streams[J->slot >= 0 ? J->slot : 0]); J->d_in = nullptr; }
  S->used -= J->bytes;
  J->bytes = 0;
}

mp_status admit(mp_server* S, Job* J, int slot) {
  cudaStream_t st = S->streams[slot];
  // host planning: Morton order and precision map
  std::vector<int64_t> p = morton_perm(J->locs.data(), J->n);
  std::vector<double> sl(2 * J->n), sz((size_t)J->n * J->nrhs);
  for (int64_t k = 0; k < J->n; ++k) {
    sl[2 * k] = J->locs[2 * p[k]];
    sl[2 * k + 1] = J->locs[2 * p[k] + 1];
    for (int c = 0; c < J->nrhs; ++c) sz[(size_t)c * J->n + k] = J->z[(size_t)c * J->n + p[k]];
  }
  J->locs.swap(sl);
  J->z.swap(sz);
  const int nt = (int)((J->n + J->b - 1) / J->b);
  std::vector<uint8_t> map((size_t)nt * nt);
  mp_status s = mp_map_bound(J->n, J->b, J->locs.data(), J->cov, S->band, MP_F32, S->far_dt, S->eps,
                             map.data());
  if (s) return s;
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < i; ++j) {
      ++J->n_tiles;
      if (map[(size_t)i * nt + j] == S->far_dt) ++J->n_low;
    }
  s = mp_tmat_create(S->ctx, J->n, J->b, map.data(),
                     (J->refine > 0 ? MP_TMAT_KEEP_SIGMA : 0) | MP_TMAT_STREAM_ALLOC | MP_TMAT_DIRECT | J->flags, st,
                     &J->t);
  if (s) return s;
  const size_t in_bytes = sizeof(double) * (2 * J->n + (size_t)J->n * J->nrhs + 2 * J->nrhs + 2);
  if (S->inject_oom > 0) {   // a failed allocation, made on the host (the matrix exists already)
    --S->inject_oom;
    return MP_ERR_OOM;
  }
  if (cudaMallocAsync((void**)&J->d_in, in_bytes, st) != cudaSuccess) return MP_ERR_OOM;
  int64_t tb = 0;
  mp_tmat_info(J->t, nullptr, nullptr, nullptr, &tb);
  J->bytes = tb + (int64_t)in_bytes;
  S->used += J->bytes;
  double* d_locs = J->d_in;
  double* d_z = d_locs + 2 * J->n;
  double* d_ll = d_z + (size_t)J->n * J->nrhs;
  double* d_quad = d_ll + J->nrhs;
  double* d_logdet = d_quad + J->nrhs;
  int64_t* d_info = reinterpret_cast<int64_t*>(d_logdet + 1);
  if (cudaMemcpyAsync(d_locs, J->locs.data(), sizeof(double) * 2 * J->n, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(d_z, J->z.data(), sizeof(double) * J->n * J->nrhs, cudaMemcpyHostToDevice, st))
    return MP_ERR_CUDA;
  if ((s = mp_generate_matern(J->t, d_locs, J->cov))) return s;
  if ((s = mp_chol(J->t, d_info, d_logdet))) return s;
  if ((s = mp_loglik(J->t, d_z, J->n, J->nrhs, J->refine, d_ll, d_quad, nullptr))) return s;
  if (cudaMemcpyAsync(J->h_out, d_ll, sizeof(double) * (2 * J->nrhs + 2), cudaMemcpyDeviceToHost, st))
    return MP_ERR_CUDA;
  if (cudaEventRecord(J->done, st)) return MP_ERR_CUDA;
  J->slot = slot;
  J->t_admit = now_s();
  return MP_OK;
}

}  // namespace

extern "C" mp_status mp_server_create(mp_ctx* ctx, int64_t hbm_budget, int32_t max_slots,
                                      double eps, uint8_t far_dt, mp_server** out) {
  if (!ctx || !out || hbm_budget <= 0 || max_slots < 1 || max_slots > 64 || !(eps > 0) ||
      far_dt > MP_E4M3)
    return MP_ERR_ARG;
  mp_server* S = new mp_server;
  S->ctx = ctx;
  S->budget = hbm_budget;
  S->max_slots = max_slots;
  S->eps = eps;
  S->far_dt = far_dt;
  S->streams.resize(max_slots);
  S->slot_job.assign(max_slots, nullptr);
  for (auto& st : S->streams)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      delete S;
      return MP_ERR_CUDA;
    }
  *out = S;
  return MP_OK;
}

extern "C" void mp_server_destroy(mp_server* S) {
  if (!S) return;
  for (auto st : S->streams) cudaStreamSynchronize(st);
  for (Job* J : S->jobs) {
    free_job_device(S, J);
    if (J->h_out) cudaFreeHost(J->h_out);
    if (J->done) cudaEventDestroy(J->done);
    delete J;
  }
  for (auto st : S->streams) cudaStreamDestroy(st);
  delete S;
}

extern "C" mp_status mp_server_submit(mp_server* S, int64_t n, const double* h_locs, const double* h_z,
                                      int32_t nrhs, int32_t refine_iters, mp_matern cov,
                                      int64_t* id) {
  if (!S || n < 1 || !h_locs || !h_z || nrhs < 1 || refine_iters < 0 || !id) return MP_ERR_ARG;
  if (!mp::matern_nu_valid(cov.nu) || !(cov.range > 0) || !(cov.sigma2 > 0) || !(cov.nugget >= 0))
    return MP_ERR_ARG;
  Job* J = new Job;
  J->id = S->next_id++;
  J->n = n;
  J->nrhs = nrhs;
  J->refine = refine_iters;
  J->cov = cov;
  {
    int b = 0;
    pick_schedule(S, n, &b, &J->flags);
    J->b = b;
  }
  J->locs.assign(h_locs, h_locs + 2 * n);
  J->z.assign(h_z, h_z + (size_t)n * nrhs);
  if (cudaMallocHost(&J->h_out, sizeof(double) * (2 * nrhs + 2)) != cudaSuccess ||
      cudaEventCreateWithFlags(&J->done, cudaEventDisableTiming) != cudaSuccess) {
    delete J;
    return MP_ERR_CUDA;
  }
  J->t_submit = now_s();
  S->jobs.push_back(J);
  S->queue.push_back(J);
  *id = J->id;
  return MP_OK;
}

extern "C" mp_status mp_server_poll(mp_server* S, mp_serve_result* out, int32_t max_out,
                                    int32_t* n_out) {
  if (!S || !n_out || (max_out > 0 && !out)) return MP_ERR_ARG;
  *n_out = 0;
  // retire
  for (int s = 0; s < S->max_slots; ++s) {
    Job* J = S->slot_job[s];
    if (!J) continue;
    cudaError_t e = cudaEventQuery(J->done);
    if (e == cudaErrorNotReady) continue;
    J->t_done = now_s();
    J->finished = true;
    S->slot_job[s] = nullptr;
    if (e != cudaSuccess) J->status = MP_ERR_CUDA;
    else {
      const double info = J->h_out[2 * J->nrhs + 1];
      int64_t iv;
      std::memcpy(&iv, &info, sizeof iv);
      J->status = iv == 0 ? MP_OK : iv < 0 ? MP_ERR_TIMEOUT : MP_ERR_NOT_SPD;
    }
    S->kept.push_back(J);
    if (*n_out < max_out) {
      mp_serve_result& r = out[(*n_out)++];
      r.id = J->id;
      r.status = J->status;
      r.nrhs = J->nrhs;
      r.n = J->n;
      r.b = J->b;
      r.t_submit = J->t_submit;
      r.t_admit = J->t_admit;
      r.t_done = J->t_done;
      r.logdet = J->h_out[2 * J->nrhs];
      r.loglik0 = J->h_out[0];
      r.low_tiles = J->n_low;
      r.offdiag_tiles = J->n_tiles;
    }
  }
  // admit (arrival order, backfilling)
  for (auto it = S->queue.begin(); it != S->queue.end();) {
    int slot = -1;
    for (int s = 0; s < S->max_slots; ++s)
      if (!S->slot_job[s]) { slot = s; break; }
    if (slot < 0) break;
    Job* J = *it;
    const int64_t need = footprint(J->n, J->b, J->nrhs, J->refine > 0);
    while (S->used + need > S->budget && !S->kept.empty()) {   // evict kept factors
      Job* K = S->kept.front();
      S->kept.pop_front();
      free_job_device(S, K);
    }
    if (S->used + need > S->budget) { ++it; continue; }
    mp_status st = admit(S, J, slot);
    if (st != MP_OK) {
      free_job_device(S, J);
      J->status = st;
      J->finished = true;
      J->t_done = now_s();
      it = S->queue.erase(it);
      if (*n_out < max_out) {
        mp_serve_result& r = out[(*n_out)++];
        std::memset(&r, 0, sizeof r);
        r.id = J->id;
        r.status = st;
        r.t_submit = J->t_submit;
        r.t_done = J->t_done;
      }
      continue;
    }
    S->slot_job[slot] = J;
    it = S->queue.erase(it);
  }
  return MP_OK;
}

extern "C" mp_status mp_server_tune(mp_server* S, const int64_t* sizes, int32_t count,
                                    int32_t refine_iters, const char* cache_path) {
  if (!S || !sizes || count < 1 || refine_iters < 0) return MP_ERR_ARG;
  std::vector<int64_t> ns(sizes, sizes + count);
  std::sort(ns.begin(), ns.end());
  ns.erase(std::unique(ns.begin(), ns.end()), ns.end());
  std::vector<int32_t> bs;
  std::vector<uint32_t> fs;
  for (int64_t n : ns) {
    if (n < 1) return MP_ERR_ARG;
    mp_tuned t{};
    mp_status st = mp_tune_tmat(S->ctx, n, S->far_dt, S->eps, refine_iters, cache_path, S->streams[0], &t);
    if (st) return st;
    bs.push_back(t.b);
    fs.push_back(t.flags);
  }
  S->tuned_n = ns;
  S->tuned_b = bs;
  S->tuned_flags = fs;
  return MP_OK;
}

extern "C" mp_status mp_server_inject_alloc_failures(mp_server* S, int32_t count) {
  if (!S || count < 0) return MP_ERR_ARG;
  S->inject_oom = count;
  return MP_OK;
}

extern "C" mp_status mp_server_result(mp_server* S, int64_t id, double* h_ll, double* h_quad) {
  if (!S || id < 1 || id >= S->next_id) return MP_ERR_ARG;
  Job* J = S->jobs[id - 1];
  if (!J->finished) return MP_ERR_STATE;
  if (h_ll) std::memcpy(h_ll, J->h_out, sizeof(double) * J->nrhs);
  if (h_quad) std::memcpy(h_quad, J->h_out + J->nrhs, sizeof(double) * J->nrhs);
  return (mp_status)J->status;
}

extern "C" mp_status mp_server_release(mp_server* S, int64_t id) {
  if (!S || id < 1 || id >= S->next_id) return MP_ERR_ARG;
  Job* J = S->jobs[id - 1];
  if (!J->finished) return MP_ERR_STATE;
  auto k = std::find(S->kept.begin(), S->kept.end(), J);
  if (k != S->kept.end()) S->kept.erase(k);
  free_job_device(S, J);
  J->released = true;
  return MP_OK;
}

extern "C" mp_status mp_server_factor(mp_server* S, int64_t id, mp_tmat** t) {
  if (!S || !t || id < 1 || id >= S->next_id) return MP_ERR_ARG;
  Job* J = S->jobs[id - 1];
  if (!J->finished || !J->t) return MP_ERR_STATE;
  *t = J->t;
  return MP_OK;
}

extern "C" mp_status mp_server_stats(mp_server* S, int64_t* queued, int64_t* running,
                                     int64_t* kept, int64_t* bytes_used) {
  if (!S) return MP_ERR_ARG;
  int64_t r = 0;
  for (Job* J : S->slot_job) r += J != nullptr;
  if (queued) *queued = (int64_t)S->queue.size();
  if (running) *running = r;
  if (kept) *kept = (int64_t)S->kept.size();
  if (bytes_used) *bytes_used = S->used;
  return MP_OK;
}

// Locations and covariance tiles.
//
// Morton order: 32-bit Z-curve keys of the 16-bit-quantised coordinates
// (x bits even, y bits odd), made unique by appending the point index, then
// sorted by a bitonic network (global passes for strides >= 1024, shared
// memory for the rest).
//
// Generation (the Matérn model of Sec. 6.2 in its half-integer closed
// forms): every entry of a lower tile is computed in float64 from the two
// locations and rounded once into the tile's format.  E4M3 tiles first get
// the tile's amax from a separate pass (`gen_amax`), then the power-of-two
// scale.  Rows/columns beyond n are identity padding.  The float64
// arithmetic is written with explicit _rn intrinsics so that no fused
// multiply-add changes the rounding of the distance or the polynomial.
#include "mp_device.cuh"

namespace mp {

namespace {

__device__ __forceinline__ uint32_t spread16(uint32_t v) {
  uint32_t k = 0;
  for (int bit = 0; bit < 16; ++bit) k |= ((v >> bit) & 1u) << (2 * bit);
  return k;
}

__global__ void k_morton_keys(const double* __restrict__ locs, int64_t n, int64_t n2,
                              unsigned long long* __restrict__ keys) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2) return;
  if (i >= n) { keys[i] = ~0ull; return; }
  double qx = fmax(fmin(floor(__dmul_rn(locs[2 * i], 65536.0)), 65535.0), 0.0);
  double qy = fmax(fmin(floor(__dmul_rn(locs[2 * i + 1], 65536.0)), 65535.0), 0.0);
  uint32_t key = spread16((uint32_t)qx) | (spread16((uint32_t)qy) << 1);
  keys[i] = ((unsigned long long)key << 32) | (unsigned long long)i;
}

// One compare-exchange pass of the bitonic network with stride j >= 1024.
__global__ void k_bitonic_global(unsigned long long* keys, int64_t n2, int64_t j, int64_t k) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2) return;
  int64_t l = i ^ j;
  if (l <= i) return;
  unsigned long long a = keys[i], b = keys[l];
  bool up = (i & k) == 0;
  if (up ? a > b : a < b) { keys[i] = b; keys[l] = a; }
}

// All passes of stage k with stride < 1024 (or the full sort of 1024-element
// blocks when k_hi = 0), inside one 1024-element block in shared memory.
__global__ void k_bitonic_local(unsigned long long* keys, int64_t n2, int64_t k_lo,
                                int64_t k_hi) {
  __shared__ unsigned long long s[1024];
  int64_t base = (int64_t)blockIdx.x * 1024;
  for (int t = threadIdx.x; t < 1024; t += blockDim.x) s[t] = keys[base + t];
  __syncthreads();
  for (int64_t k = k_lo; k <= k_hi; k <<= 1) {
    for (int64_t j = (k >> 1) < 512 ? (k >> 1) : 512; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < 1024; t += blockDim.x) {
        int l = t ^ (int)j;
        if (l > t) {
          unsigned long long a = s[t], b = s[l];
          bool up = ((base + t) & k) == 0;
          if (up ? a > b : a < b) { s[t] = b; s[l] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < 1024; t += blockDim.x) keys[base + t] = s[t];
}

__global__ void k_morton_gather(const unsigned long long* __restrict__ keys,
                                const double* __restrict__ in, int64_t n,
                                double* __restrict__ out, int64_t* __restrict__ perm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t p = (int64_t)(keys[i] & 0xffffffffull);
  perm[i] = p;
  out[2 * i] = in[2 * p];
  out[2 * i + 1] = in[2 * p + 1];
}

// Matérn covariance of two locations (closed forms, x = r / range).  x is
// r times the rounded reciprocal of the range (GB300's FP64 pipe makes a
// division cost about ten FP64 operations): one more rounding than r /
// range, i.e. |dx| <= 2 ulp(x), which exp(-x) carries as a relative error
// of at most 2 x 2^-52.
__device__ __forceinline__ double entry(const ItemGen& it, double inv_range, double xi, double yi,
                                        double xj, double yj, int64_t gi, int64_t gj) {
  if (gi >= it.n || gj >= it.n) return gi == gj ? 1.0 : 0.0;
  double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj);
  double r = sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
  double x = __dmul_rn(r, inv_range);
  double poly;
  if (it.nu == 0.5) poly = 1.0;
  else if (it.nu == 1.5) poly = __dadd_rn(1.0, x);
  else poly = __dadd_rn(__dadd_rn(1.0, x), __dmul_rn(__dmul_rn(x, x), 1.0 / 3.0));
  double v = __dmul_rn(__dmul_rn(it.sigma2, poly), exp(-x));
  if (gi == gj) v = __dadd_rn(v, it.nugget);
  return v;
}

constexpr int GEN_ROWS = 16;

template <bool AMAX>
__global__ void __launch_bounds__(256) k_generate(Arena A, const ItemGen* __restrict__ items) {
  extern __shared__ double sloc[];           // b column points (x, y) + GEN_ROWS row points
  const ItemGen it = items[blockIdx.x];
  const int b = A.b;
  const int r0 = blockIdx.y * GEN_ROWS;
  const int64_t gi0 = (int64_t)it.ti * b + r0, gj0 = (int64_t)it.tj * b;
  double* cx = sloc;
  double* rx = sloc + 2 * b;
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    int64_t g = gj0 + c;
    cx[2 * c] = g < it.n ? it.locs[2 * g] : 0.0;
    cx[2 * c + 1] = g < it.n ? it.locs[2 * g + 1] : 0.0;
  }
  for (int r = threadIdx.x; r < GEN_ROWS; r += blockDim.x) {
    int64_t g = gi0 + r;
    rx[2 * r] = g < it.n ? it.locs[2 * g] : 0.0;
    rx[2 * r + 1] = g < it.n ? it.locs[2 * g + 1] : 0.0;
  }
  __syncthreads();
  const int dt = A.tiles[it.tile].dt;
  char* dst = tile_bytes(A, it.tile);
  const double inv_range = 1.0 / it.range;
  double mx = 0.0;
  double inv_s = 1.0;
  if (!AMAX && dt == E4M3) inv_s = 1.0 / e4m3_scale(amax_value(&A.amax[it.tile]));
  for (int e = threadIdx.x; e < GEN_ROWS * b; e += blockDim.x) {
    int r = e / b, c = e - r * b;
    double v = entry(it, inv_range, rx[2 * r], rx[2 * r + 1], cx[2 * c], cx[2 * c + 1], gi0 + r, gj0 + c);
    int64_t off = (int64_t)(r0 + r) * b + c;
    if (AMAX) {
      mx = fmax(mx, fabs(v));
    } else {
      store_round(dst, dt, off, dt == E4M3 ? v * inv_s : v);
      if (it.sigma64) it.sigma64[off] = v;
    }
  }
  if (AMAX) {
    __shared__ double red[8];
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
      atomic_max_pos(&A.amax[it.tile], mx);
    }
  } else if (blockIdx.y == 0 && threadIdx.x == 0) {
    A.scale[it.tile] = dt == E4M3 ? e4m3_scale(amax_value(&A.amax[it.tile])) : 1.0;
  }
}

// Sum of squares of 16 rows of one generated tile, written to a per-CTA
// partial (reduced in a fixed order by k_reduce_norms: deterministic).
__global__ void __launch_bounds__(256) k_tile_sumsq(int b, const ItemGen* __restrict__ items,
                                                    double* __restrict__ partial) {
  extern __shared__ double sloc[];
  const ItemGen it = items[blockIdx.x];
  const int r0 = blockIdx.y * GEN_ROWS;
  const int64_t gi0 = (int64_t)it.ti * b + r0, gj0 = (int64_t)it.tj * b;
  double* cx = sloc;
  double* rx = sloc + 2 * b;
  for (int c = threadIdx.x; c < b; c += blockDim.x) {
    int64_t g = gj0 + c;
    cx[2 * c] = g < it.n ? it.locs[2 * g] : 0.0;
    cx[2 * c + 1] = g < it.n ? it.locs[2 * g + 1] : 0.0;
  }
  for (int r = threadIdx.x; r < GEN_ROWS; r += blockDim.x) {
    int64_t g = gi0 + r;
    rx[2 * r] = g < it.n ? it.locs[2 * g] : 0.0;
    rx[2 * r + 1] = g < it.n ? it.locs[2 * g + 1] : 0.0;
  }
  __syncthreads();
  const double inv_range = 1.0 / it.range;
  double ss = 0.0;
  for (int e = threadIdx.x; e < GEN_ROWS * b; e += blockDim.x) {
    int r = e / b, c = e - r * b;
    double v = entry(it, inv_range, rx[2 * r], rx[2 * r + 1], cx[2 * c], cx[2 * c + 1], gi0 + r, gj0 + c);
    ss += v * v;
  }
  __shared__ double red[8];
  ss = warp_sum(ss);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) ss += red[w];
    partial[(int64_t)blockIdx.x * gridDim.y + blockIdx.y] = ss;
  }
}

__global__ void k_reduce_norms(const ItemGen* __restrict__ items, int count, int parts, int nt,
                               const double* __restrict__ partial, double* __restrict__ norms) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  double s = 0.0;
  for (int p = 0; p < parts; ++p) s += partial[(int64_t)t * parts + p];
  norms[items[t].ti * nt + items[t].tj] = sqrt(s);
}

}  // namespace

void launch_tile_norms(int b, const ItemGen* items, int count, int nt, double* partial,
                       double* norms, cudaStream_t s) {
  if (count <= 0) return;
  dim3 grid(count, b / GEN_ROWS);
  size_t smem = sizeof(double) * (2 * b + 2 * GEN_ROWS);
  k_tile_sumsq<<<grid, 256, smem, s>>>(b, items, partial);
  k_reduce_norms<<<(count + 127) / 128, 128, 0, s>>>(items, count, b / GEN_ROWS, nt, partial, norms);
}

void launch_morton_keys(const double* locs, int64_t n, int64_t n2, unsigned long long* keys,
                        cudaStream_t s) {
  k_morton_keys<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(locs, n, n2, keys);
}

void launch_bitonic(unsigned long long* keys, int64_t n2, cudaStream_t s) {
  // n2 is a power of two >= 1024
  unsigned blocks_local = (unsigned)(n2 / 1024);
  k_bitonic_local<<<blocks_local, 512, 0, s>>>(keys, n2, 2, 1024);
  for (int64_t k = 2048; k <= n2; k <<= 1) {
    for (int64_t j = k >> 1; j >= 1024; j >>= 1)
      k_bitonic_global<<<(unsigned)(n2 / 256), 256, 0, s>>>(keys, n2, j, k);
    k_bitonic_local<<<blocks_local, 512, 0, s>>>(keys, n2, k, k);
  }
}

void launch_morton_gather(const unsigned long long* keys, const double* in, int64_t n,
                          double* out, int64_t* perm, cudaStream_t s) {
  k_morton_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, in, n, out, perm);
}

void launch_gen_amax(const Arena& A, const ItemGen* items, int count, cudaStream_t s) {
  if (count <= 0) return;
  dim3 grid(count, A.b / GEN_ROWS);
  size_t smem = sizeof(double) * (2 * A.b + 2 * GEN_ROWS);
  k_generate<true><<<grid, 256, smem, s>>>(A, items);
}

void launch_generate(const Arena& A, const ItemGen* items, int count, cudaStream_t s) {
  if (count <= 0) return;
  dim3 grid(count, A.b / GEN_ROWS);
  size_t smem = sizeof(double) * (2 * A.b + 2 * GEN_ROWS);
  k_generate<false><<<grid, 256, smem, s>>>(A, items);
}

}  // namespace mp

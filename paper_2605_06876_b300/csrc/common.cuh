// Internal helpers of the sm_103a implementation: error reporting, workspace
// carving, the per-launch camera set, warp utilities, and the device-wide scan
// and stable LSD radix sort used by binning, top-k, regions and compaction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>

#include "adpsplit.h"

namespace adp {

// ----------------------------------------------------------------- errors

void set_error(const char* fmt, ...);

#define ADP_CHECK_ARG(cond, ...)               \
  do {                                         \
    if (!(cond)) {                             \
      ::adp::set_error(__VA_ARGS__);           \
      return ADP_ERR_INVALID_ARG;              \
    }                                          \
  } while (0)

#define ADP_CUDA(call)                                                          \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      ::adp::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                       __FILE__, __LINE__);                                     \
      return ADP_ERR_CUDA;                                                      \
    }                                                                           \
  } while (0)

#define ADP_LAUNCH_CHECK() ADP_CUDA(cudaGetLastError())

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// ----------------------------------------------------------------- workspace

// Bump allocator over a caller-provided workspace; every block 256-aligned.
struct Carver {
  char* base;
  size_t size;
  size_t off = 0;
  bool ok = true;
  Carver(void* b, size_t s) : base(static_cast<char*>(b)), size(s) {}
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    if (off + bytes > size || base == nullptr) {
      ok = false;
      off += bytes;
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};
// Byte count of a carve of `count` elements of T (for workspace-size queries).
template <class T>
inline size_t carve_bytes(size_t count) {
  size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
  return bytes == 0 ? 256 : bytes;
}

// ----------------------------------------------------------------- cameras

// Cameras of one launch, passed by value as a kernel parameter.
struct CamSet {
  int n_views;
  int tile_w, tile_h;
  adp_camera cam[ADP_MAX_VIEWS];
  int tiles_x[ADP_MAX_VIEWS];
  int tiles_y[ADP_MAX_VIEWS];
  int tile_base[ADP_MAX_VIEWS + 1];
  long long pix_base[ADP_MAX_VIEWS + 1];
};

int make_camset(const adp_camera* cams, int n_views, const adp_params* prm, CamSet* cs);

__device__ __forceinline__ int view_of_tile(const CamSet& cs, int tile) {
  int v = 0;
  while (v + 1 < cs.n_views && tile >= cs.tile_base[v + 1]) ++v;
  return v;
}

// ----------------------------------------------------------------- warp utils

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ----------------------------------------------------------------- scan

// Exclusive prefix sum of n int64 values produced by a functor load(i),
// reduce-then-scan in three launches. The count is either a host value or read
// from device memory (d_n != nullptr, with n_max an upper bound sizing grids).
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

inline int64_t scan_blocks(int64_t n_max) { return (n_max + SCAN_TILE - 1) / SCAN_TILE; }
inline size_t scan_workspace_bytes(int64_t n_max) {
  return carve_bytes<long long>(scan_blocks(n_max) + 1);
}

__device__ __forceinline__ long long device_count(const long long* d_n, long long n) {
  return d_n ? *d_n : n;
}

template <class Load>
__global__ void scan_reduce_kernel(Load load, long long n, const long long* d_n, long long* bsum) {
  __shared__ long long s[SCAN_THREADS / 32];
  long long N = device_count(d_n, n);
  long long base = (long long)blockIdx.x * SCAN_TILE;
  long long acc = 0;
  if (base < N) {
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      long long i = base + (long long)k * SCAN_THREADS + threadIdx.x;
      if (i < N) acc += load(i);
    }
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < SCAN_THREADS / 32; ++w) t += s[w];
    bsum[blockIdx.x] = t;
  }
}

// Single block: exclusive scan of the block sums in place; total to *total.
__global__ void scan_blocksums_kernel(long long* bsum, long long nb_max, long long n,
                                      const long long* d_n, long long* total);

template <class Load, class Store>
__global__ void scan_downsweep_kernel(Load load, Store store, long long n, const long long* d_n,
                                      const long long* bsum) {
  __shared__ long long s_warp[SCAN_THREADS / 32];
  long long N = device_count(d_n, n);
  long long base = (long long)blockIdx.x * SCAN_TILE;
  if (base >= N) return;
  // blocked arrangement: thread t owns items base + t*ITEMS .. + ITEMS-1
  long long v[SCAN_ITEMS];
  long long tsum = 0;
  long long first = base + (long long)threadIdx.x * SCAN_ITEMS;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    long long i = first + k;
    v[k] = i < N ? load(i) : 0;
    tsum += v[k];
  }
  // block exclusive scan of tsum
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long inc = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  long long wpre = 0;
  for (int k = 0; k < w; ++k) wpre += s_warp[k];
  long long run = bsum[blockIdx.x] + wpre + inc - tsum;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    long long i = first + k;
    if (i < N) store(i, run);
    run += v[k];
  }
}

// Exclusive scan: store(i, prefix_i). total (device, may be null) receives the sum.
template <class Load, class Store>
int scan_exclusive(Load load, Store store, long long n_max, const long long* d_n,
                   long long* total, void* ws, cudaStream_t st) {
  long long nb = scan_blocks(n_max);
  if (nb == 0) nb = 1;
  long long* bsum = static_cast<long long*>(ws);
  scan_reduce_kernel<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(load, n_max, d_n, bsum);
  scan_blocksums_kernel<<<1, 1024, 0, st>>>(bsum, nb, n_max, d_n, total);
  scan_downsweep_kernel<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(load, store, n_max, d_n, bsum);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

// ----------------------------------------------------------------- radix sort

// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits, the
// item count read from device memory. Each pass: per-tile digit histograms, a
// per-digit scan over tiles, and a stable scatter whose ranks come from warp
// match masks in item order.
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;  // items per lane
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_BINS = 256;

inline long long rs_tiles(long long n_max) { return (n_max + RS_TILE - 1) / RS_TILE; }

struct SortWorkspace {
  unsigned* keys_alt;
  unsigned* vals_alt;
  unsigned* hist;       // [RS_BINS][tiles_max]
  unsigned* digit_tot;  // [RS_BINS]
  long long tiles_max;
};

inline size_t sort_workspace_bytes(long long n_max) {
  long long t = rs_tiles(n_max);
  if (t < 1) t = 1;
  return 2 * carve_bytes<unsigned>(n_max) + carve_bytes<unsigned>((size_t)RS_BINS * t) +
         carve_bytes<unsigned>(RS_BINS);
}
inline SortWorkspace carve_sort(Carver& c, long long n_max) {
  SortWorkspace w;
  w.tiles_max = rs_tiles(n_max);
  if (w.tiles_max < 1) w.tiles_max = 1;
  w.keys_alt = c.take<unsigned>(n_max);
  w.vals_alt = c.take<unsigned>(n_max);
  w.hist = c.take<unsigned>((size_t)RS_BINS * w.tiles_max);
  w.digit_tot = c.take<unsigned>(RS_BINS);
  return w;
}

// Digit of an item: from the key (shift) or, when by_value, value / divisor
// (used to order by view after a depth sort).
struct DigitOp {
  int shift;
  unsigned divisor;  // 0: digit from key
  __device__ __forceinline__ unsigned operator()(unsigned key, unsigned val) const {
    return divisor ? (val / divisor) & 255u : (key >> shift) & 255u;
  }
};

__global__ void rs_hist_kernel(const unsigned* keys, const unsigned* vals, const long long* d_n,
                               long long tiles_max, DigitOp op, unsigned* hist);
__global__ void rs_scan_kernel(unsigned* hist, const long long* d_n, long long tiles_max,
                               unsigned* digit_tot);
__global__ void rs_scatter_kernel(const unsigned* keys_in, const unsigned* vals_in,
                                  unsigned* keys_out, unsigned* vals_out, const long long* d_n,
                                  long long tiles_max, DigitOp op, const unsigned* hist,
                                  const unsigned* digit_tot);

// Sorts (keys, vals) in place by the given passes. passes[k] is a DigitOp;
// n_max bounds the device count *d_n.
int radix_sort_pairs(unsigned* keys, unsigned* vals, const long long* d_n, long long n_max,
                     const DigitOp* passes, int n_passes, const SortWorkspace& w, cudaStream_t st);

inline int bits_for(long long v) {
  int b = 0;
  while (b < 62 && (1LL << b) <= v) ++b;
  return b;
}

// ----------------------------------------------------------------- misc

__global__ void fill_i32_kernel(int* p, long long n, int v);
inline unsigned grid_for(long long n, int threads, long long cap = 1LL << 30) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// SH basis count and float4 plane count.
__host__ __device__ inline int sh_coeffs(int deg) { return (deg + 1) * (deg + 1); }
__host__ __device__ inline int sh_planes(int deg) { return (3 * sh_coeffs(deg) + 3) / 4; }

}  // namespace adp

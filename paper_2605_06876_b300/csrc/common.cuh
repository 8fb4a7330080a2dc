// Internal helpers of the sm_103a implementation: error reporting, workspace
// carving, the per-launch camera set, warp utilities, and the device-wide scan
// and stable LSD radix sort used by binning, top-k, regions and compaction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <mutex>

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

// ----------------------------------------------------------------- fills

// Up to FILL_MAX device ranges, each set to a repeated 64-bit pattern (byte o of
// a range gets byte o % 8 of the pattern, the lowest byte first), by one kernel.
// Inside a captured graph a memset node costs about as much as three dependent
// kernel launches, so a call that resets several ranges before its kernels
// resets them all in one launch, or inside a kernel it launches first anyway
// (fill_ranges_device).
constexpr int FILL_MAX = 8;
struct FillSet {
  int n = 0;
  bool overflow = false;
  unsigned char* ptr[FILL_MAX];
  long long bytes[FILL_MAX];
  unsigned long long pattern[FILL_MAX];
  void add(void* p, size_t b, unsigned long long pat = 0ull) {
    if (b == 0) return;
    if (n == FILL_MAX) {
      overflow = true;
      return;
    }
    ptr[n] = static_cast<unsigned char*>(p);
    bytes[n] = (long long)b;
    pattern[n] = pat;
    ++n;
  }
};

// The ranges of f, by threads tid = 0 .. nt-1 of a grid: 16-byte stores for the
// aligned middle of each range, byte stores for its ends.
__device__ __forceinline__ void fill_ranges_device(const FillSet& f, long long tid, long long nt) {
  for (int s = 0; s < f.n; ++s) {
    unsigned char* b = f.ptr[s];
    const long long len = f.bytes[s];
    const unsigned long long pat = f.pattern[s];
    long long head = (long long)((16u - (unsigned)(reinterpret_cast<uintptr_t>(b) & 15u)) & 15u);
    if (head > len) head = len;
    const long long body = (len - head) >> 4;
    for (long long o = tid; o < head; o += nt) b[o] = (unsigned char)(pat >> (8 * (o & 7)));
    for (long long o = head + (body << 4) + tid; o < len; o += nt)
      b[o] = (unsigned char)(pat >> (8 * (o & 7)));
    // the 8-byte words of the middle start at offsets congruent to head mod 8
    const int sh = (int)(head & 7) * 8;
    const unsigned long long r = sh ? (pat >> sh) | (pat << (64 - sh)) : pat;
    const ulonglong2 v = make_ulonglong2(r, r);
    ulonglong2* q = reinterpret_cast<ulonglong2*>(b + head);
    for (long long c = tid; c < body; c += nt) q[c] = v;
  }
}

// One launch that fills the ranges of f (none when f is empty).
int launch_fill(const FillSet& f, cudaStream_t st);

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
  // the EWA Jacobian's clamp of x/z and y/z: 1.3 times the tangent of the half
  // field of view, 1.3 W / (2 fx) and 1.3 H / (2 fy), each a product and a
  // correctly rounded division, so the host computes exactly what a kernel would
  float lim_x[ADP_MAX_VIEWS];
  float lim_y[ADP_MAX_VIEWS];
};

int make_camset(const adp_camera* cams, int n_views, const adp_params* prm, CamSet* cs);

// Gaussians a compositing block stages per batch (validated by make_camset).
inline int stage_size(const adp_params* prm) {
  return prm->batch == 64 || prm->batch == 128 ? prm->batch : 256;
}

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

// ----------------------------------------------------------------- auxiliary stream

// The library's auxiliary stream of the current device (highest priority) and the
// events that fork work onto it and join it back: `planned` and `merged` for the
// overlapped split's plan, `forked` and `joined` for the batched step. Created on
// the first use on a device (so that use must come before any stream capture that
// includes it); the mutex serialises the event records and waits of host threads.
struct AuxStream {
  cudaStream_t stream = nullptr;
  cudaEvent_t planned = nullptr, merged = nullptr;
  cudaEvent_t forked = nullptr, joined = nullptr;
};
int aux_stream(AuxStream** out);
std::mutex& aux_mutex();

// ----------------------------------------------------------------- bounded waits

// Every device wait of the library (the scan's look-back, the top-k's grid
// barrier) polls at most a bounded number of times. The bound is read on the
// host at each launch (adp_set_spin_limit; the default is large enough never to
// run out on a working device). A wait that runs out records ADP_ERR_TIMEOUT in
// the caller's status word (if one was given) and in the call's own error flag,
// and the kernel returns normally with results the call then discards or marks
// undefined.
long long spin_limit();

__device__ __forceinline__ void report_timeout(int* d_status) {
  if (d_status) atomicCAS(d_status, 0, (int)ADP_ERR_TIMEOUT);
}

// Sets *count to 0 if the scan whose error flag is err gave up a wait. A
// compaction by a scan that gave up can leave gaps (entries never written)
// below its count; consumers that index memory with the compacted entries then
// see an empty list instead.
__global__ void count_guard_kernel(const unsigned long long* err, long long* count);

// ----------------------------------------------------------------- scan

// Exclusive prefix sum of n int64 values produced by a functor load(i), in one
// launch with decoupled look-back: each CTA takes the next tile from a ticket
// counter, publishes its tile total, then its inclusive prefix once the totals
// before it are known, reading up to 32 predecessors at a time. A CTA only ever
// waits on tiles handed out before its own ticket, which are being processed by
// CTAs already running, so the waits end; each is still bounded, and a bound
// that runs out sets the error flag (scan_error_flag) and *d_status and leaves
// the prefixes too small (never larger than the true ones). The count is a host
// value or read from device memory (d_n != nullptr, n an upper bound).
constexpr int SCAN_THREADS = 256;
#ifndef ADP_SCAN_ITEMS
#define ADP_SCAN_ITEMS 4
#endif
constexpr int SCAN_ITEMS = ADP_SCAN_ITEMS;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr unsigned long long SCAN_FLAG_A = 1ull << 62;  // tile total published
constexpr unsigned long long SCAN_FLAG_P = 2ull << 62;  // inclusive prefix published
constexpr unsigned long long SCAN_VALUE = (1ull << 62) - 1;

__host__ __device__ inline long long scan_blocks(long long n_max) {
  return (n_max + SCAN_TILE - 1) / SCAN_TILE;
}
// status words [0, nb), ticket, error flag
inline size_t scan_workspace_bytes(long long n_max) {
  return carve_bytes<unsigned long long>(scan_blocks(n_max) + 4);
}
// The error flag of a scan's workspace: nonzero after a look-back gave up. It is
// cleared by the next scan in the same workspace, so a consumer reads it before.
inline const unsigned long long* scan_error_flag(const void* ws, long long n_max) {
  return static_cast<const unsigned long long*>(ws) + scan_blocks(n_max) + 2;
}

__device__ __forceinline__ long long device_count(const long long* d_n, long long n) {
  return d_n ? *d_n : n;
}

template <class Load, class Store>
__global__ void __launch_bounds__(SCAN_THREADS)
    scan_lookback_kernel(Load load, Store store, long long n, const long long* d_n,
                         unsigned long long* status, long long* total, int* d_status,
                         long long spin_max) {
  __shared__ long long s_warp[SCAN_THREADS / 32];
  __shared__ long long s_excl;
  __shared__ long long s_tile;
  const long long N = device_count(d_n, n);
  const long long nb = (N + SCAN_TILE - 1) / SCAN_TILE;
  unsigned long long* ticket = status + scan_blocks(n) + 1;
  unsigned long long* err = ticket + 1;
  if (threadIdx.x == 0) s_tile = (long long)atomicAdd(ticket, 1ull);
  __syncthreads();
  const long long tile = s_tile;
  if (tile >= nb) {
    if (nb == 0 && tile == 0 && threadIdx.x == 0 && total) *total = 0;
    return;
  }
  const long long base = tile * SCAN_TILE;
  const long long first = base + (long long)threadIdx.x * SCAN_ITEMS;
  long long v[SCAN_ITEMS];
  long long tsum = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const long long i = first + k;
    v[k] = i < N ? load(i) : 0;
    tsum += v[k];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long inc = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  long long wpre = 0, agg = 0;
  for (int k = 0; k < SCAN_THREADS / 32; ++k) {
    if (k < w) wpre += s_warp[k];
    agg += s_warp[k];
  }
  if (w == 0) {  // publish, then look back
    volatile unsigned long long* vs = status;
    if (tile == 0) {
      if (lane == 0) {
        __threadfence();
        atomicExch(status, SCAN_FLAG_P | (unsigned long long)agg);
        s_excl = 0;
      }
    } else {
      if (lane == 0) atomicExch(status + tile, SCAN_FLAG_A | (unsigned long long)agg);
      long long excl = 0;
      long long end = tile;  // window covers [end - 32, end)
      bool done = false;
      while (!done) {
        const long long j = end - 1 - lane;
        unsigned long long word = SCAN_FLAG_P;  // before tile 0: an empty prefix
        if (j >= 0) {
          long long spins = 0;
          do {
            word = vs[j];
          } while ((word >> 62) == 0 && ++spins < spin_max);
          if ((word >> 62) == 0) {
            atomicExch(err, 1ull);
            report_timeout(d_status);
            word = SCAN_FLAG_P;  // give up: stop the look-back here
          }
        }
        const unsigned pmask = __ballot_sync(0xffffffffu, (word >> 62) == 2);
        // sum the totals from the nearest inclusive prefix (lowest lane) to the window end
        const int stop = pmask ? __ffs(pmask) - 1 : 31;
        long long val = (lane <= stop && j >= 0) ? (long long)(word & SCAN_VALUE) : 0;
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
        excl += val;
        if (pmask) done = true;
        end -= 32;
      }
      if (lane == 0) {
        __threadfence();
        atomicExch(status + tile, SCAN_FLAG_P | (unsigned long long)(excl + agg));
        s_excl = excl;
      }
    }
  }
  __syncthreads();
  long long run = s_excl + wpre + inc - tsum;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const long long i = first + k;
    if (i < N) store(i, run);
    run += v[k];
  }
  if (tile == nb - 1 && threadIdx.x == 0 && total) *total = s_excl + agg;
}

// The words of a scan workspace that must be zero when the scan starts.
inline size_t scan_status_bytes(long long n_max) {
  long long nb = scan_blocks(n_max);
  if (nb == 0) nb = 1;
  return sizeof(unsigned long long) * (size_t)(nb + 3);
}
// Adds those words of the scan workspace ws to a fill.
inline void scan_clear(FillSet& f, void* ws, long long n_max) {
  f.add(ws, scan_status_bytes(n_max));
}

// Exclusive scan: store(i, prefix_i); total (device, may be null) receives the sum.
// d_status (device, may be null): the caller's status word (see bounded waits).
// cleared: the caller has zeroed the workspace's status words (scan_clear) since
// the last scan in it; otherwise the scan zeroes them itself first.
template <class Load, class Store>
int scan_exclusive(Load load, Store store, long long n_max, const long long* d_n,
                   long long* total, void* ws, cudaStream_t st, int* d_status,
                   bool cleared = false) {
  long long nb = scan_blocks(n_max);
  if (nb == 0) nb = 1;
  unsigned long long* status = static_cast<unsigned long long*>(ws);
  if (!cleared) {
    FillSet f;
    scan_clear(f, ws, n_max);
    const int rc = launch_fill(f, st);
    if (rc) return rc;
  }
  scan_lookback_kernel<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(load, store, n_max, d_n, status,
                                                              total, d_status, spin_limit());
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

// ----------------------------------------------------------------- radix sort

// Stable LSD radix sort of (uint32 key, uint32 value) pairs, 8-bit digits, the
// item count read from device memory. Each pass: per-tile digit histograms, a
// per-digit scan over tiles, and a stable scatter whose ranks come from warp
// ballots in item order.
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 8;  // items per lane
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

// Digit of an item: `bits` bits (1 to 8) of the key from `shift` or, with a
// divisor, of value / divisor (used to order by view after a depth sort). A pass
// with fewer bits ranks with fewer ballots and scans fewer histogram rows.
struct DigitOp {
  int shift;
  unsigned divisor;  // 0: digit from key
  int bits = 8;
  __host__ __device__ __forceinline__ unsigned mask() const { return (1u << bits) - 1u; }
  __host__ __device__ __forceinline__ int bins() const { return 1 << bits; }
  __device__ __forceinline__ unsigned operator()(unsigned key, unsigned val) const {
    return divisor ? (val / divisor) & mask() : (key >> shift) & mask();
  }
};

// Up to four passes of a small sort (one launch; see small_sort_kernel).
constexpr long long SMALL_SORT_MAX = 8192;
struct SmallPasses {
  DigitOp op[4];
  int count;
};

__global__ void rs_hist_kernel(const unsigned* keys, const unsigned* vals, const long long* d_n,
                               long long tiles_max, DigitOp op, unsigned* hist);
__global__ void rs_scan_kernel(unsigned* hist, const long long* d_n, long long tiles_max,
                               int bins, unsigned* digit_tot);
__global__ void rs_scatter_kernel(const unsigned* keys_in, const unsigned* vals_in,
                                  unsigned* keys_out, unsigned* vals_out, const long long* d_n,
                                  long long tiles_max, DigitOp op, const unsigned* hist,
                                  const unsigned* digit_tot, bool drop_none);

// Key that a sort may drop (see radix_sort_pairs): all bits set.
constexpr unsigned RS_DROP_KEY = 0xffffffffu;

// Sorts (keys, vals) in place by the given passes. passes[k] is a DigitOp;
// n_max bounds the device count *d_n. Up to SMALL_SORT_MAX items (and four
// passes) the sort runs in a single one-block launch.
// first_hist_done: the caller already wrote the first pass's per-tile histograms
// (hist[digit * tiles_max + tile], every digit of every tile of *d_n items).
// drop_none (with first_hist_done and a writable count): the first pass drops the
// items whose key is RS_DROP_KEY (the caller's histograms leave them out) and sets
// *d_n to the items kept, which the later passes sort.
// res_keys, res_vals (optional): receive where the sorted pairs are (keys/vals, or
// the workspace's alternate buffers after an odd number of passes), instead of the
// copy back into keys/vals.
int radix_sort_pairs(unsigned* keys, unsigned* vals, long long* d_n, long long n_max,
                     const DigitOp* passes, int n_passes, const SortWorkspace& w, cudaStream_t st,
                     bool first_hist_done = false, bool drop_none = false,
                     unsigned** res_keys = nullptr, unsigned** res_vals = nullptr);

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

// Error statistics of AdpSplit (Eq. 6, Eqs. 7-8, Secs. 4.1 and 5.1):
//  - per view, the raw L1 error and its min/max (block reduction + atomics),
//    then the min-max normalised E, mask M and band B, decided in float32 with
//    correctly rounded operations, and the per-Gaussian attribution (count,
//    mass) with warp-aggregated integer atomics (mass in exact fixed point);
//  - top-k error mass by a radix select on the 64-bit mass keys, in one
//    cooperative launch;
//  - erosion (a min filter over the tile and its halo in shared memory),
//    8-connected labelling by a union-find whose
//    roots are the smallest pixel index of each component (per 32x32 tile in
//    shared memory first, then across tile borders in global memory),
//    exact int64 region moments, the area filter and the FP64 region statistics.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "phases.cuh"

namespace adp {

// ------------------------------------------------------------------ error map

__global__ void err_raw_kernel(const float* img, const float* tgt, CamSet cs, float* raw,
                               unsigned* minmax_bits) {
  const int v = blockIdx.y;
  const long long P = (long long)cs.cam[v].width * cs.cam[v].height;
  const long long base = cs.pix_base[v];
  unsigned lo = 0x7f800000u, hi = 0u;  // +inf, 0 as float bits (raw >= 0)
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < P;
       u += (long long)gridDim.x * blockDim.x) {
    long long p = base + u;
    float d0 = fabsf(__fsub_rn(img[3 * p], tgt[3 * p]));
    float d1 = fabsf(__fsub_rn(img[3 * p + 1], tgt[3 * p + 1]));
    float d2 = fabsf(__fsub_rn(img[3 * p + 2], tgt[3 * p + 2]));
    float r = __fadd_rn(__fadd_rn(d0, d1), d2);
    raw[p] = r;
    unsigned b = __float_as_uint(r);
    lo = min(lo, b);
    hi = max(hi, b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  __shared__ unsigned s_lo[32], s_hi[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    s_lo[w] = lo;
    s_hi[w] = hi;
  }
  __syncthreads();
  if (w == 0) {  // one pair of atomics per block
    lo = lane < nw ? s_lo[lane] : 0x7f800000u;
    hi = lane < nw ? s_hi[lane] : 0u;
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      atomicMin(&minmax_bits[2 * v], lo);
      atomicMax(&minmax_bits[2 * v + 1], hi);
    }
  }
}

// E, M, B and the per-Gaussian attribution of pre-erosion error pixels.
__global__ void err_norm_kernel(float* E, uint8_t* mask, const unsigned* minmax_bits,
                                const int* dominant, long long n, CamSet cs, float tau, int L,
                                int mass_shift, int* count, double* mass) {
  __shared__ unsigned long long s_val[8][32];
  const int v = blockIdx.y;
  const long long P = (long long)cs.cam[v].width * cs.cam[v].height;
  const long long base = cs.pix_base[v];
  const float mass_scale = __int_as_float((127 + mass_shift) << 23);  // 2^mass_shift
  const float mn = __uint_as_float(minmax_bits[2 * v]);
  const float mx = __uint_as_float(minmax_bits[2 * v + 1]);
  const float range = __fsub_rn(mx, mn);
  const float one_minus_tau = __fsub_rn(1.0f, tau);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // whole warps iterate together so the match below sees every lane
  for (long long u0 = blockIdx.x * (long long)blockDim.x; u0 < P;
       u0 += (long long)gridDim.x * blockDim.x) {
    long long u = u0 + threadIdx.x;
    int key = -1;
    float e = 0.f;
    if (u < P) {
      long long p = base + u;
      e = range > 0.f ? __fdiv_rn(__fsub_rn(E[p], mn), range) : 0.f;
      E[p] = e;
      bool m = e > tau;
      int b = 0;
      if (m) {
        float t = __fdiv_rn(__fmul_rn(__fsub_rn(e, tau), (float)L), one_minus_tau);
        b = (int)floorf(t);
        b = b > L - 1 ? L - 1 : (b < 0 ? 0 : b);
      }
      mask[p] = (uint8_t)((m ? 1 : 0) | (b << 4));
      int d = dominant[p];
      if (m && d >= 0 && d < n) key = d;
    }
    unsigned peers = __match_any_sync(0xffffffffu, key);
    // E * 2^mass_shift is an integer for every E above the threshold, so the
    // sums are exact and independent of the order of the atomics
    s_val[warp][lane] = __float2ull_rn(e * mass_scale);
    __syncwarp();
    if (key >= 0 && (peers & lanemask_lt()) == 0) {
      unsigned long long q = 0;
      for (unsigned m = peers; m; m &= m - 1) q += s_val[warp][__ffs(m) - 1];
      atomicAdd(&count[key], __popc(peers));
      atomicAdd(reinterpret_cast<unsigned long long*>(&mass[key]), q);
    }
    __syncwarp();
  }
}

// Converts the fixed-point mass sums (held in the mass array) to doubles in place.
// q * 2^-shift as a double, exactly, for q < 2^53: the IEEE-754 fields are built
// from the integer (exponent from the leading bit, the bits below it as the
// fraction), with no FP64 instruction (B300's FP64 rate is a small fraction of its
// FP32 rate). Larger q take the FP64 conversion.
__device__ __forceinline__ double fixed_to_double(unsigned long long q, int shift) {
  if (q == 0ull) return 0.0;
  if (q >> 53) return (double)q * ldexp(1.0, -shift);
  const int e = 63 - __clzll((long long)q);  // q in [2^e, 2^(e+1))
  const unsigned long long frac = (q << (52 - e)) & ((1ull << 52) - 1ull);
  const unsigned long long bits = ((unsigned long long)(1023 + e - shift) << 52) | frac;
  return __longlong_as_double((long long)bits);
}

__global__ void mass_finalize_kernel(double* mass, long long n, int mass_shift) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long q = reinterpret_cast<unsigned long long*>(mass)[i];
    mass[i] = fixed_to_double(q, mass_shift);
  }
}

// Scale exponent for the fixed-point mass: a float32 E > tau >= 2^e is a
// multiple of 2^(e - 23), so E * 2^(23 - e) is an integer. Capped at 36 so that
// 2^28 pixels of E <= 1 still fit in 64 bits (below tau = 2^-13 the sums round
// to 2^-36).
static int mass_shift_for(float tau) {
  int e = -4;
  if (tau > 0.f) {
    int ex;
    frexpf(tau, &ex);  // tau = f * 2^ex, f in [0.5, 1)
    e = ex - 1;
  } else {
    e = -13;
  }
  int sh = 23 - e;
  return sh < 0 ? 0 : (sh > 36 ? 36 : sh);
}

// ------------------------------------------------------------------ top-k

// One-launch top-k: a cooperative kernel (every block resident) runs the radix
// select and the final compaction with grid-wide barriers between the phases.
// Each pass histograms one 8-bit digit of the keys that still match the chosen
// high digits (block histograms in shared memory, summed in global memory), and
// every block then picks the same digit from the summed histogram. A pass also
// takes the smallest and largest matching key: once they are equal (for example
// all the zero masses), the threshold key is known and the passes stop; they also
// stop when the chosen digit holds exactly the keys still to take. The output is
// the keys above the threshold and the first `remaining` keys equal to it in id
// order, written in id order.
#ifndef ADP_TOPK_THREADS
#define ADP_TOPK_THREADS 256
#endif
#ifndef ADP_TOPK_PER_SM
#define ADP_TOPK_PER_SM 2
#endif
constexpr int TOPK_THREADS = ADP_TOPK_THREADS;
constexpr int TOPK_PER_SM = ADP_TOPK_PER_SM;  // resident blocks per SM the grid asks for
constexpr int TOPK_MAX_BLOCKS = 1024;         // bound of the grid
static_assert(TOPK_THREADS >= 256 && TOPK_THREADS <= 1024 && TOPK_THREADS % 32 == 0,
              "the digit sums take 256 threads and the flag scan one warp of warp totals");
struct TopkCoop {
  unsigned* hist;              // [8][256], zeroed before the launch
  unsigned long long* mm;      // [8][2] min and ~max of the matching keys (all ones before)
  unsigned* bar;               // barrier counter, zeroed before the launch
  unsigned* err;               // set if a barrier wait gave up
  long long* blk;              // [2][gridDim.x] per-block counts
  uint8_t* sel;                // [n] selection flags
  int* d_status;               // the caller's status word (may be null)
  long long spin_max;          // poll bound of a barrier wait
};

// Grid-wide barrier number `round` (1, 2, ...) over a counter that starts at zero.
// Waits are bounded: on timeout the error flag and the caller's status word are
// set and the barrier returns false in every thread of the block, which then
// leaves the kernel. Every block counts itself in before waiting, so the blocks
// still waiting pass this barrier with complete data and stop at the next one
// (the departed block never reaches it): no block goes on from stale state.
__device__ __forceinline__ bool topk_grid_barrier(const TopkCoop& w, unsigned round) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(w.bar, 1u);
    const unsigned target = round * gridDim.x;
    volatile unsigned* vb = w.bar;
    long long spins = 0;
    int ok = 1;
    while (*vb < target) {
      if (++spins > w.spin_max) {
        atomicExch(w.err, 1u);
        report_timeout(w.d_status);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Block-wide exclusive scan of 0/1 flags over TOPK_THREADS threads; returns the
// thread's prefix and sets *total.
__device__ __forceinline__ int topk_flag_scan(bool f, int* s_w, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned b = __ballot_sync(0xffffffffu, f);
  if (lane == 0) s_w[warp] = __popc(b);
  __syncthreads();
  if (warp == 0) {
    int x = lane < TOPK_THREADS / 32 ? s_w[lane] : 0, inc = x;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    s_w[32 + lane] = inc - x;
    if (lane == 31) s_w[64] = inc;
  }
  __syncthreads();
  const int pre = s_w[32 + warp] + __popc(b & lanemask_lt());
  *total = s_w[64];
  __syncthreads();
  return pre;
}

__global__ void __launch_bounds__(TOPK_THREADS)
    topk_coop_kernel(const double* mass, long long n, long long k, int* out_ids, TopkCoop w) {
  __shared__ unsigned s_h[256];
  __shared__ unsigned long long s_lo[32], s_hi[32];
  __shared__ int s_w[65];
  __shared__ unsigned s_pick[3];  // digit, its count, keys in higher digits
  __shared__ long long s_pre;
  const unsigned long long* keys = reinterpret_cast<const unsigned long long*>(mass);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const long long G = gridDim.x;
  const long long chunk = ((n + G - 1) / G + TOPK_THREADS - 1) / TOPK_THREADS * TOPK_THREADS;
  const long long c0 = blockIdx.x * chunk, c1 = min(n, c0 + chunk);
  unsigned long long prefix = 0ull, mask = 0ull;
  long long remaining = k;
  unsigned round = 0;
  for (int p = 0; p < 8; ++p) {
    const int shift = 56 - 8 * p;
    if (t < 256) s_h[t] = 0u;
    __syncthreads();
    unsigned long long lo = ~0ull, hi = 0ull;
    for (long long i = c0 + t; i < c1; i += TOPK_THREADS) {
      const unsigned long long key = keys[i];
      if ((key & mask) == prefix) {
        atomicAdd(&s_h[(key >> shift) & 255ull], 1u);
        lo = min(lo, key);
        hi = max(hi, key);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      s_lo[warp] = lo;
      s_hi[warp] = hi;
    }
    __syncthreads();
    if (warp == 0) {
      lo = lane < TOPK_THREADS / 32 ? s_lo[lane] : ~0ull;
      hi = lane < TOPK_THREADS / 32 ? s_hi[lane] : 0ull;
      for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      if (lane == 0 && lo <= hi) {  // the maximum as the complement of a minimum
        atomicMin(&w.mm[2 * p], lo);
        atomicMin(&w.mm[2 * p + 1], ~hi);
      }
    }
    if (t < 256 && s_h[t]) atomicAdd(&w.hist[256 * p + t], s_h[t]);
    if (!topk_grid_barrier(w, ++round)) return;
    const unsigned long long glo = *(volatile unsigned long long*)&w.mm[2 * p];
    const unsigned long long ghi = ~*(volatile unsigned long long*)&w.mm[2 * p + 1];
    if (glo == ghi) {  // every key still in play is the threshold key
      prefix = glo;
      mask = ~0ull;
      break;
    }
    if (warp < 8) {  // suffix sums over digits 255 .. 0, one digit per thread
      const int b = 255 - t;
      const long long c = (long long)*(volatile unsigned*)&w.hist[256 * p + b];
      long long inc = c;
      for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane == 31) s_lo[warp] = (unsigned long long)inc;
      __syncwarp();
      asm volatile("bar.sync 1, 256;");
      long long pre = 0;
      for (int q = 0; q < warp; ++q) pre += (long long)s_lo[q];
      const long long suf = pre + inc, above = suf - c;
      if (suf >= remaining && above < remaining) {
        s_pick[0] = (unsigned)b;
        s_pick[1] = (unsigned)c;
        s_pick[2] = (unsigned)above;
      }
    }
    __syncthreads();
    prefix |= (unsigned long long)s_pick[0] << shift;
    mask |= 255ull << shift;
    remaining -= (long long)s_pick[2];
    if ((long long)s_pick[1] == remaining) break;  // the digit's keys are all taken
    __syncthreads();
  }
  // ranks of the keys equal to the threshold (under the mask), in id order
  int tot = 0;
  long long cnt_eq = 0;
  for (long long i0 = c0; i0 < c1; i0 += TOPK_THREADS) {
    const long long i = i0 + t;
    const bool eq = i < c1 && (keys[i] & mask) == prefix;
    topk_flag_scan(eq, s_w, &tot);
    cnt_eq += tot;
  }
  if (t == 0) w.blk[blockIdx.x] = cnt_eq;
  if (!topk_grid_barrier(w, ++round)) return;
  if (warp == 0) {
    long long x = 0;
    for (long long b = lane; b < blockIdx.x; b += 32) x += *(volatile long long*)&w.blk[b];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_pre = x;
  }
  __syncthreads();
  long long run = s_pre, cnt_sel = 0;
  for (long long i0 = c0; i0 < c1; i0 += TOPK_THREADS) {
    const long long i = i0 + t;
    unsigned long long km = i < c1 ? (keys[i] & mask) : 0ull;
    const bool eq = i < c1 && km == prefix;
    const int r = topk_flag_scan(eq, s_w, &tot);
    const bool sel = i < c1 && (km > prefix || (eq && run + r < remaining));
    if (i < c1) w.sel[i] = sel ? 1 : 0;
    run += tot;
    cnt_sel += __syncthreads_count(sel);
  }
  if (t == 0) w.blk[G + blockIdx.x] = cnt_sel;
  if (!topk_grid_barrier(w, ++round)) return;
  if (warp == 0) {
    long long x = 0;
    for (long long b = lane; b < blockIdx.x; b += 32) x += *(volatile long long*)&w.blk[G + b];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_pre = x;
  }
  __syncthreads();
  run = s_pre;
  for (long long i0 = c0; i0 < c1; i0 += TOPK_THREADS) {
    const long long i = i0 + t;
    const bool sel = i < c1 && w.sel[i];
    const int r = topk_flag_scan(sel, s_w, &tot);
    if (sel) out_ids[run + r] = (int)i;
    run += tot;
  }
}

// Blocks of the cooperative top-k kernel on this device: TOPK_PER_SM per SM, or
// as many as the kernel's occupancy allows (all resident).
static int topk_coop_grid(int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  ADP_CUDA(cudaGetDevice(&dev));
  ADP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  ADP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, topk_coop_kernel, TOPK_THREADS, 0));
  ADP_CHECK_ARG(per_sm >= 1 && sms >= 1, "the top-k kernel cannot be resident on this device");
  const long long g = (long long)sms * (per_sm < TOPK_PER_SM ? per_sm : TOPK_PER_SM);
  *grid = (int)(g < TOPK_MAX_BLOCKS ? g : TOPK_MAX_BLOCKS);
  return ADP_OK;
}

// Scratch layout of the cooperative top-k (in a workspace or the static array).
static size_t topk_coop_bytes(long long n) {
  return carve_bytes<unsigned>(8 * 256) + carve_bytes<unsigned long long>(16) +
         carve_bytes<unsigned>(2) + carve_bytes<long long>(2 * TOPK_MAX_BLOCKS) +
         carve_bytes<uint8_t>(n > 0 ? n : 1);
}

static int topk_coop_run(const double* mass, long long n, long long k, int32_t* out_ids,
                         void* ws, size_t ws_bytes, int* d_status, cudaStream_t st) {
  Carver c(ws, ws_bytes);
  TopkCoop w;
  w.hist = c.take<unsigned>(8 * 256);
  w.mm = c.take<unsigned long long>(16);
  w.bar = c.take<unsigned>(2);
  w.err = w.bar + 1;
  w.blk = c.take<long long>(2 * TOPK_MAX_BLOCKS);
  w.sel = c.take<uint8_t>(n > 0 ? n : 1);
  w.d_status = d_status;
  w.spin_max = spin_limit();
  ADP_CHECK_ARG(c.ok, "internal: top-k scratch too small");
  int grid = 0;
  int rc = topk_coop_grid(&grid);
  if (rc) return rc;
  // the histograms, the barrier and the min/max slots, and -1 in every output slot
  // (if a barrier wait gives up, the slots of the blocks that left hold -1, which
  // every consumer of a candidate list skips), in one launch
  FillSet fill;
  fill.add(w.hist, sizeof(unsigned) * 8 * 256);
  fill.add(w.bar, 2 * sizeof(unsigned));
  fill.add(w.mm, 16 * sizeof(unsigned long long), ~0ull);
  fill.add(out_ids, sizeof(int32_t) * (size_t)k, ~0ull);
  rc = launch_fill(fill, st);
  if (rc) return rc;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(TOPK_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ADP_CUDA(cudaLaunchKernelEx(&cfg, topk_coop_kernel, mass, (long long)n, (long long)k,
                              (int*)out_ids, w));
  return ADP_OK;
}

// ------------------------------------------------------------------ erosion

// Horizontal then vertical AND over radius r; outside the image counts as set.
// Erosion of M into mask bit 1: a pixel stays set iff every pixel of its
// (2r+1)x(2r+1) window is set, pixels outside the image counting as set. One
// 32x32 output tile per block: the tile and its r-wide halo are staged in shared
// memory, eroded along rows, then along columns.
constexpr int ERODE_T = 32;
constexpr int ERODE_RMAX = 64;

// The ranges of f are filled by the same launch (the call's resets; the erosion
// reads none of them).
// Shared memory: the staged (32 + 2r)^2 block and its row-eroded (32 + 2r) x 32
// block, sized for the call's radius (erode_smem_bytes; 30 KB at the largest).
__host__ __device__ inline int erode_smem_bytes(int r) {
  return (ERODE_T + 2 * r) * (ERODE_T + 2 * r) + (ERODE_T + 2 * r) * ERODE_T;
}
__global__ void __launch_bounds__(256) erode_kernel(uint8_t* mask, CamSet cs, int r, FillSet f) {
  extern __shared__ uint8_t s_erode[];
  uint8_t* s_in = s_erode;
  uint8_t* s_row = s_erode + (ERODE_T + 2 * r) * (ERODE_T + 2 * r);
  fill_ranges_device(f, ((long long)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x,
                     (long long)gridDim.x * gridDim.y * blockDim.x);
  const int v = blockIdx.y;
  const int W = cs.cam[v].width, H = cs.cam[v].height;
  const int ntx = (W + ERODE_T - 1) / ERODE_T, nty = (H + ERODE_T - 1) / ERODE_T;
  if ((int)blockIdx.x >= ntx * nty) return;
  const int x0 = (blockIdx.x % ntx) * ERODE_T, y0 = (blockIdx.x / ntx) * ERODE_T;
  const long long base = cs.pix_base[v];
  const int E = ERODE_T + 2 * r;  // staged edge
  for (int q = threadIdx.x; q < E * E; q += blockDim.x) {
    const int yy = y0 - r + q / E, xx = x0 - r + q % E;
    s_in[q] = (xx < 0 || yy < 0 || xx >= W || yy >= H) ? 1
                                                        : (mask[base + (long long)yy * W + xx] & 1);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < E * ERODE_T; q += blockDim.x) {  // rows: E x 32
    const int ry = q / ERODE_T, cx = q % ERODE_T;
    uint8_t ok = 1;
    for (int d = 0; d <= 2 * r && ok; ++d) ok = s_in[ry * E + cx + d];
    s_row[q] = ok;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < ERODE_T * ERODE_T; q += blockDim.x) {  // columns
    const int cy = q / ERODE_T, cx = q % ERODE_T;
    const int x = x0 + cx, y = y0 + cy;
    if (x >= W || y >= H) continue;
    uint8_t ok = 1;
    for (int d = 0; d <= 2 * r && ok; ++d) ok = s_row[(cy + d) * ERODE_T + cx];
    const long long p = base + (long long)y * W + x;
    const uint8_t m = mask[p];
    mask[p] = (uint8_t)((m & ~2) | (ok ? 2 : 0));
  }
}

// ------------------------------------------------------------------ labelling

// Root of a with path halving: each visited node is re-pointed at its
// grandparent. A node is re-pointed only while it is not a root and only to one
// of its own ancestors, so a concurrent link made by uf_unite is never lost: a
// union whose atomicMin finds its node already re-pointed retries from there.
__device__ __forceinline__ int uf_find(volatile int* L, int a) {
  int p = L[a];
  while (p != a) {
    int gp = L[p];
    if (gp != p) L[a] = gp;
    a = p;
    p = gp;
  }
  return a;
}

// Joins the sets of a and b; every link points to a smaller index, so each
// component ends rooted at its smallest pixel index.
__device__ void uf_unite(int* L, int a, int b) {
  volatile int* VL = L;
  for (int guard = 0; guard < (1 << 24); ++guard) {
    a = uf_find(VL, a);
    b = uf_find(VL, b);
    if (a == b) return;
    if (a > b) {
      int t = a;
      a = b;
      b = t;
    }
    int old = atomicMin(&L[b], a);
    if (old == b) return;
    b = old;
  }
}

__device__ __forceinline__ bool region_pixel(const uint8_t* mask, const int* dom,
                                             const uint8_t* cand, long long n, long long p) {
  int d = dom[p];
  return (mask[p] & 2) && d >= 0 && d < n && cand[d];
}

// Same-class test of two participating pixels: equal dominant Gaussian and band.
__device__ __forceinline__ bool same_class(const int* L, const int* dom, const uint8_t* mask,
                                           long long p, long long q) {
  return L[q] >= 0 && dom[q] == dom[p] && (mask[q] >> 4) == (mask[p] >> 4);
}

constexpr int CCL_T = 32;  // labelling tile edge (32 x 32 pixels per CTA)

__device__ __forceinline__ int sfind(volatile int* l, int a) {
  int p = l[a];
  while (p != a) {
    int gp = l[p];
    if (gp != p) l[a] = gp;
    a = p;
    p = gp;
  }
  return a;
}

__device__ void sunite(int* l, int a, int b) {
  volatile int* vl = l;
  for (int guard = 0; guard < 4096; ++guard) {
    a = sfind(vl, a);
    b = sfind(vl, b);
    if (a == b) return;
    if (a > b) {
      int t = a;
      a = b;
      b = t;
    }
    int old = atomicMin(&l[b], a);
    if (old == b) return;
    b = old;
  }
}

// Labelling inside one 32x32 tile in shared memory, then every pixel of the
// tile gets its label: the tile-local root by global index for a participating
// pixel (eroded mask set, dominated by a candidate), -1 for any other.
// Row runs first: a warp labels one tile row at a time with ballots, linking every
// pixel straight to the first pixel of its run of same-class neighbours. Then the
// union-find joins runs across rows, with one union per place where two runs
// start to touch: the up edge only where the left neighbour does not already
// reach the up-left pixel, up-left only when neither left nor up is joined,
// up-right only when up is not joined. Every link points to a smaller index, so a
// component's root is its smallest pixel index.
__global__ void __launch_bounds__(256) ccl_local_kernel(const uint8_t* mask, const int* dom,
                                                        const uint8_t* cand, long long n,
                                                        CamSet cs, int* L, long long* part,
                                                        int* lroots,
                                                        unsigned long long* n_lroots) {
  __shared__ int s_l[CCL_T * CCL_T];
  __shared__ int s_d[CCL_T * CCL_T];
  __shared__ uint8_t s_b[CCL_T * CCL_T];
  __shared__ unsigned s_m[6][CCL_T * CCL_T];  // tile-local moments per local root
  const int v = blockIdx.y;
  const int W = cs.cam[v].width, H = cs.cam[v].height;
  const int ntx = (W + CCL_T - 1) / CCL_T, nty = (H + CCL_T - 1) / CCL_T;
  if ((int)blockIdx.x >= ntx * nty) return;
  const int tx0 = (blockIdx.x % ntx) * CCL_T, ty0 = (blockIdx.x / ntx) * CCL_T;
  const long long base = cs.pix_base[v];
  const int lane = threadIdx.x & 31;
  bool any = false;
  for (int li = threadIdx.x; li < CCL_T * CCL_T; li += blockDim.x) {
    int x = tx0 + (li & (CCL_T - 1)), y = ty0 + li / CCL_T;
    int lab = -1, d = -1;
    uint8_t b = 0;
    if (x < W && y < H) {
      const long long p = base + (long long)y * W + x;
      if (region_pixel(mask, dom, cand, n, p)) {
        lab = li;
        d = dom[p];
        b = mask[p] >> 4;
      }
    }
    any = any || lab >= 0;
    s_l[li] = lab;
    s_d[li] = d;
    s_b[li] = b;
  }
  if (!__syncthreads_or(any)) {  // no participating pixel: every label is -1
    for (int li = threadIdx.x; li < CCL_T * CCL_T; li += blockDim.x) {
      int x = tx0 + (li & (CCL_T - 1)), y = ty0 + li / CCL_T;
      if (x < W && y < H) L[base + (long long)y * W + x] = -1;
    }
    return;
  }
  for (int li = threadIdx.x; li < CCL_T * CCL_T; li += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 6; ++k) s_m[k][li] = 0u;
  }
  __syncthreads();
  auto same = [&](int a, int q) { return s_l[q] >= 0 && s_d[q] == s_d[a] && s_b[q] == s_b[a]; };
  // row runs (a warp owns whole rows; lane = column)
  for (int li = threadIdx.x; li < CCL_T * CCL_T; li += blockDim.x) {
    const bool part = s_l[li] >= 0;
    const bool joined_left = part && lane > 0 && same(li, li - 1);
    const unsigned starts = __ballot_sync(0xffffffffu, part && !joined_left);
    if (part) {
      const unsigned upto = starts & (lane == 31 ? 0xffffffffu : ((2u << lane) - 1u));
      s_l[li] = (li - lane) + (31 - __clz(upto));
    }
  }
  __syncthreads();
  // joins across rows
  for (int li = threadIdx.x; li < CCL_T * CCL_T; li += blockDim.x) {
    const int ly = li / CCL_T;
    if (ly == 0 || s_l[li] < 0) continue;
    const bool left = lane > 0 && same(li, li - 1);
    const bool up = same(li, li - CCL_T);
    const bool upleft = lane > 0 && same(li, li - CCL_T - 1);
    const bool upright = lane < CCL_T - 1 && same(li, li - CCL_T + 1);
    if (up && !(left && upleft)) sunite(s_l, li, li - CCL_T);
    if (upleft && !left && !up) sunite(s_l, li, li - CCL_T - 1);
    if (upright && !up) sunite(s_l, li, li - CCL_T + 1);
  }
  __syncthreads();
  // labels, and the moments of each tile-local component in tile coordinates
  // (below 32, so 32-lane sums of squares fit 32 bits): one warp reduction per
  // moment and group of lanes with the same local root, then shared atomics
  for (int li = threadIdx.x; li < CCL_T * CCL_T; li += blockDim.x) {
    int x = tx0 + (li & (CCL_T - 1)), y = ty0 + li / CCL_T;
    int r = -1;
    if (x < W && y < H) {
      int lab = -1;
      if (s_l[li] >= 0) {
        r = sfind(s_l, li);
        int rx = tx0 + (r & (CCL_T - 1)), ry = ty0 + r / CCL_T;
        lab = (int)(base + (long long)ry * W + rx);
      }
      L[base + (long long)y * W + x] = lab;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, r);
    if (r >= 0) {
      const unsigned lx = (unsigned)(li & (CCL_T - 1)), ly = (unsigned)(li / CCL_T);
      const unsigned m0 = __popc(peers), m1 = __reduce_add_sync(peers, lx);
      const unsigned m2 = __reduce_add_sync(peers, ly), m3 = __reduce_add_sync(peers, lx * lx);
      const unsigned m4 = __reduce_add_sync(peers, lx * ly), m5 = __reduce_add_sync(peers, ly * ly);
      if ((peers & lanemask_lt()) == 0) {
        atomicAdd(&s_m[0][r], m0);
        atomicAdd(&s_m[1][r], m1);
        atomicAdd(&s_m[2][r], m2);
        atomicAdd(&s_m[3][r], m3);
        atomicAdd(&s_m[4][r], m4);
        atomicAdd(&s_m[5][r], m5);
      }
    }
  }
  __syncthreads();
  // every local root: its moments in image coordinates (exact int64) and a list entry
  for (int li = threadIdx.x; li < CCL_T * CCL_T; li += blockDim.x) {
    if (s_l[li] != li) continue;  // participating roots point at themselves
    const long long X0 = tx0, Y0 = ty0;
    const long long A = s_m[0][li], sx = s_m[1][li], sy = s_m[2][li];
    const long long sxx = s_m[3][li], sxy = s_m[4][li], syy = s_m[5][li];
    const int x = tx0 + (li & (CCL_T - 1)), y = ty0 + li / CCL_T;
    const long long p = base + (long long)y * W + x;
    long long* m6 = part + 6 * p;
    m6[0] = A;
    m6[1] = A * X0 + sx;
    m6[2] = A * Y0 + sy;
    m6[3] = A * X0 * X0 + 2 * X0 * sx + sxx;
    m6[4] = A * X0 * Y0 + X0 * sy + Y0 * sx + sxy;
    m6[5] = A * Y0 * Y0 + 2 * Y0 * sy + syy;
    lroots[atomicAdd(n_lroots, 1ull)] = (int)p;
  }
}

// The edges of the 8-neighbourhood that cross a tile border, with the same skip
// rules, joined in the global union-find. Only the pixels on a tile's top row,
// left column and right column own such edges: CCL_BORDER of them per tile, one
// thread each.
constexpr int CCL_BORDER = 3 * CCL_T - 2;

__global__ void ccl_border_kernel(const uint8_t* mask, const int* dom, CamSet cs, int* L) {
  const int v = blockIdx.y;
  const int W = cs.cam[v].width, H = cs.cam[v].height;
  const int ntx = (W + CCL_T - 1) / CCL_T, nty = (H + CCL_T - 1) / CCL_T;
  const long long base = cs.pix_base[v];
  const int total = ntx * nty * CCL_BORDER;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
    const int tile = u / CCL_BORDER, k = u - tile * CCL_BORDER;
    int lx, ly;
    if (k < CCL_T) {  // top row
      lx = k;
      ly = 0;
    } else if (k < 2 * CCL_T - 1) {  // left column below the corner
      lx = 0;
      ly = k - CCL_T + 1;
    } else {  // right column below the corner
      lx = CCL_T - 1;
      ly = k - 2 * CCL_T + 2;
    }
    const int x = (tile % ntx) * CCL_T + lx, y = (tile / ntx) * CCL_T + ly;
    if (x >= W || y >= H) continue;
    long long p = base + (long long)y * W + x;
    if (L[p] < 0) continue;
    bool left = x > 0 && same_class(L, dom, mask, p, p - 1);
    bool up = y > 0 && same_class(L, dom, mask, p, p - W);
    if (left && lx == 0) uf_unite(L, (int)p, (int)(p - 1));
    if (up && ly == 0) uf_unite(L, (int)p, (int)(p - W));
    if (!left && !up && x > 0 && y > 0 && (lx == 0 || ly == 0) &&
        same_class(L, dom, mask, p, p - W - 1))
      uf_unite(L, (int)p, (int)(p - W - 1));
    if (!up && x < W - 1 && y > 0 && (lx == CCL_T - 1 || ly == 0) &&
        same_class(L, dom, mask, p, p - W + 1))
      uf_unite(L, (int)p, (int)(p - W + 1));
  }
}

// Every participating pixel's label becomes its root (only when the caller asks for
// per-pixel labels; the moments pass finds the roots of the local roots itself). The
// search only reads: a
// thread writes nothing but its own pixel's final root, so no other write can
// replace a root already stored (a path-halving write made here could land after
// the owner's final write and leave a non-root ancestor in place). Concurrent
// final writes only shorten other threads' paths to the same roots.
__global__ void ccl_flatten_kernel(int* L, long long P) {
  volatile int* VL = L;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    int r = VL[p];
    if (r < 0) continue;
    for (int q = VL[r]; q != r; q = VL[r]) r = q;
    VL[p] = r;
  }
}

__global__ void zero_i64_kernel(long long* p, const long long* d_n, int per) {
  long long N = *d_n * per;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = 0;
}

// Exact int64 moments per root: the tile-local components' moments, which the
// labelling kernel left at their local roots, added to the slot of the final root.
// The final root is found by following the labels (read only; every union is done).
__global__ void moments_kernel(const int* lroots, const unsigned long long* n_lroots,
                               const long long* part, const int* L, const int* slot,
                               long long* mom) {
  const long long N = (long long)*n_lroots;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
       t += (long long)gridDim.x * blockDim.x) {
    const int p = lroots[t];
    int r = L[p];
    for (int q = L[r]; q != r; q = L[r]) r = q;
    const int s = slot[r];
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(part + 6LL * p);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(mom + 6LL * s);
#pragma unroll
    for (int k = 0; k < 6; ++k) atomicAdd(dst + k, src[k]);
  }
}

__device__ __forceinline__ double cov_exact(long long A, long long Sab, long long Sa, long long Sb) {
  __int128 num = (__int128)A * Sab - (__int128)Sa * Sb;
  return (double)num / ((double)A * (double)A);
}

struct RegionArgs {
  const long long* mom;
  const int* root_pix;
  const long long* kept_idx;
  const long long* d_nroots;
  const int* dom;
  const uint8_t* mask;
  const float* tgt;
  int m_min;
  long long cap;
  int* view;
  int* parent;
  int* label;
  int* band;
  long long* moments;
  double* stats;
};

__global__ void region_stats_kernel(RegionArgs a, CamSet cs) {
  long long N = *a.d_nroots;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
       r += (long long)gridDim.x * blockDim.x) {
    const long long* m = a.mom + 6 * r;
    long long A = m[0];
    if (A < a.m_min) continue;
    long long k = a.kept_idx[r];
    if (k >= a.cap) continue;
    long long g = a.root_pix[r];
    int v = 0;
    while (v + 1 < cs.n_views && g >= cs.pix_base[v + 1]) ++v;
    int W = cs.cam[v].width, H = cs.cam[v].height;
    double cx = (double)m[1] / (double)A, cy = (double)m[2] / (double)A;
    double cxx = cov_exact(A, m[3], m[1], m[1]);
    double cxy = cov_exact(A, m[4], m[1], m[2]);
    double cyy = cov_exact(A, m[5], m[2], m[2]);
    // closed-form eigen-decomposition of the 2x2 covariance
    double mid = 0.5 * (cxx + cyy), dd = 0.5 * (cxx - cyy);
    double rad = sqrt(dd * dd + cxy * cxy);
    double l1 = mid + rad, l2 = mid - rad;
    double ex = 1.0, ey = 0.0;
    if (rad > 0.0) {
      if (dd >= 0.0) {
        ex = dd + rad;
        ey = cxy;
      } else {
        ex = cxy;
        ey = rad - dd;
      }
      double nrm = sqrt(ex * ex + ey * ey);
      ex /= nrm;
      ey /= nrm;
      if (ex < 0.0 || (ex == 0.0 && ey < 0.0)) {
        ex = -ex;
        ey = -ey;
      }
    }
    int xi = (int)floor(cx + 0.5), yi = (int)floor(cy + 0.5);
    xi = xi < 0 ? 0 : (xi > W - 1 ? W - 1 : xi);
    yi = yi < 0 ? 0 : (yi > H - 1 ? H - 1 : yi);
    const float* rgb = a.tgt + 3 * (cs.pix_base[v] + (long long)yi * W + xi);
    double* s = a.stats + 12 * k;
    s[0] = cx;
    s[1] = cy;
    s[2] = cxx;
    s[3] = cxy;
    s[4] = cyy;
    s[5] = ex;
    s[6] = ey;
    s[7] = sqrt(l1 > 0.0 ? l1 : 0.0);
    s[8] = sqrt(l2 > 0.0 ? l2 : 0.0);
    s[9] = rgb[0];
    s[10] = rgb[1];
    s[11] = rgb[2];
    a.view[k] = v;
    a.parent[k] = a.dom[g];
    a.label[k] = (int)(g - cs.pix_base[v]);
    a.band[k] = a.mask[g] >> 4;
    for (int j = 0; j < 6; ++j) a.moments[6 * k + j] = m[j];
  }
}

__global__ void labels_out_kernel(const int* L, const long long* mom, const int* slot, int m_min,
                                  CamSet cs, int* labels) {
  const int v = blockIdx.y;
  const int P = cs.cam[v].width * cs.cam[v].height;
  const long long base = cs.pix_base[v];
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < P; u += gridDim.x * blockDim.x) {
    int r = L[base + u];
    labels[base + u] = r >= 0 ? (int)(r - base) : -1;
  }
}

__global__ void scatter_flag_kernel(const int* ids, long long k, long long n, uint8_t* flag) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < k;
       i += (long long)gridDim.x * blockDim.x) {
    int id = ids[i];
    if (id >= 0 && id < n) flag[id] = 1;
  }
}

__global__ void iota_kernel(int* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (int)i;
}

static long long total_pixels(const CamSet& cs) { return cs.pix_base[cs.n_views]; }
static unsigned view_grid(const CamSet& cs) {
  long long mx = 0;
  for (int v = 0; v < cs.n_views; ++v) {
    long long P = (long long)cs.cam[v].width * cs.cam[v].height;
    if (P > mx) mx = P;
  }
  long long g = (mx + 255) / 256;
  return (unsigned)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace adp

using namespace adp;

// ------------------------------------------------------------------ error stats

namespace adp {

void error_init_fill(FillSet& f, adp_error_maps* maps, int n_views, int32_t* count,
                     double* mass, long long n) {
  // per view the word pair (min, max) = (+inf, 0): 0x7f800000 in the lower word
  f.add(maps->minmax, 2 * sizeof(unsigned) * (size_t)n_views, 0x7f800000ull);
  if (n > 0) {
    f.add(count, sizeof(int32_t) * (size_t)n);
    f.add(mass, sizeof(double) * (size_t)n);
  }
}

int error_norm_phase(adp_error_maps* maps, const int32_t* dominant, long long n,
                     const CamSet& cs, const adp_params* prm, int32_t* count, double* mass,
                     cudaStream_t st) {
  const unsigned* mm = reinterpret_cast<const unsigned*>(maps->minmax);
  const dim3 grid(view_grid(cs), cs.n_views);
  const int shift = mass_shift_for(prm->tau_l1);
  err_norm_kernel<<<grid, 256, 0, st>>>(maps->E, maps->mask, mm, dominant, n, cs, prm->tau_l1,
                                        prm->n_levels, shift, count, mass);
  if (n > 0) mass_finalize_kernel<<<grid_for(n, 256, 148 * 16), 256, 0, st>>>(mass, n, shift);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

}  // namespace adp

extern "C" ADP_API size_t adp_error_stats_workspace_size(int32_t n_views, const adp_camera* cams) {
  (void)n_views;
  (void)cams;
  return 0;
}

extern "C" ADP_API int adp_error_stats(const float* img, const float* target,
                                       const int32_t* dominant, int64_t n,
                                       const adp_camera* cams, int32_t n_views,
                                       const adp_params* prm, adp_error_maps* maps,
                                       int32_t* count, double* mass, adp_stream_t stream) {
  ADP_CHECK_ARG(img && target && dominant && maps && maps->E && maps->mask && maps->minmax,
                "NULL argument");
  ADP_CHECK_ARG(n >= 0 && n < (1LL << 31), "n out of range");
  ADP_CHECK_ARG(n == 0 || (count && mass), "NULL count/mass");
  CamSet cs;
  int rc = make_camset(cams, n_views, prm, &cs);
  if (rc) return rc;
  ADP_CHECK_ARG(prm->n_levels >= 1 && prm->n_levels <= 15, "n_levels must be 1..15");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* mm = reinterpret_cast<unsigned*>(maps->minmax);
  FillSet fill;
  error_init_fill(fill, maps, n_views, count, mass, n);
  rc = launch_fill(fill, st);
  if (rc) return rc;
  dim3 grid(view_grid(cs), n_views);
  err_raw_kernel<<<dim3(std::min(grid.x, 148u * 4u), n_views), 256, 0, st>>>(img, target, cs,
                                                                            maps->E, mm);
  return error_norm_phase(maps, dominant, n, cs, prm, count, mass, st);
}

// ------------------------------------------------------------------ top-k

extern "C" ADP_API size_t adp_select_topk_workspace_size(int64_t n) {
  if (n < 0) return 0;
  return topk_coop_bytes(n);
}

extern "C" ADP_API int adp_select_topk(const double* mass, int64_t n, int64_t k, int32_t* out_ids,
                                       void* ws, size_t ws_bytes, int32_t* d_status,
                                       adp_stream_t stream) {
  ADP_CHECK_ARG(n >= 0 && n < (1LL << 31) && k >= 0, "bad n or k");
  ADP_CHECK_ARG(k == 0 || (mass && out_ids), "NULL argument");
  ADP_CHECK_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
  size_t need = adp_select_topk_workspace_size(n);
  ADP_CHECK_ARG(ws_bytes >= need, "workspace %zu bytes, need %zu", ws_bytes, need);
  cudaStream_t st = (cudaStream_t)stream;
  if (k > n) k = n;
  if (k == 0) return ADP_OK;
  if (k == n) {
    iota_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(out_ids, n);
    ADP_LAUNCH_CHECK();
    return ADP_OK;
  }
  return topk_coop_run(mass, n, k, out_ids, ws, ws_bytes, d_status, st);
}

// ------------------------------------------------------------------ regions

struct RegionWs {
  int* L;
  int* slot;
  int* root_pix;
  long long* mom;
  long long* part;  // [6P] moments of tile-local components, at their local roots
  int* lroots;      // [P] the local roots
  long long* kept_idx;
  uint8_t* cand;
  void* scan;   // the roots' scan
  void* scan2;  // the area filter's scan
  long long* counters;  // [0] roots, [2] local roots
};

static size_t region_ws_bytes(long long n, long long P) {
  return 3 * carve_bytes<int>(P) + 2 * carve_bytes<long long>(6 * P) + carve_bytes<int>(P) +
         carve_bytes<long long>(P) + carve_bytes<uint8_t>(n) +
         2 * scan_workspace_bytes(P) + carve_bytes<long long>(4);
}

extern "C" ADP_API size_t adp_error_regions_workspace_size(int64_t n, int32_t n_views,
                                                           const adp_camera* cams) {
  if (!cams || n_views < 1 || n_views > ADP_MAX_VIEWS || n < 0) return 0;
  long long P = 0;
  for (int v = 0; v < n_views; ++v) P += (long long)cams[v].width * cams[v].height;
  return region_ws_bytes(n, P);
}

extern "C" ADP_API int adp_error_regions(adp_error_maps* maps, const int32_t* dominant,
                                         const float* target, int64_t n, const adp_camera* cams,
                                         int32_t n_views, const int32_t* candidates,
                                         int64_t n_cand, const adp_params* prm,
                                         adp_regions* out, void* ws, size_t ws_bytes,
                                         int32_t* d_status, adp_stream_t stream) {
  ADP_CHECK_ARG(maps && maps->mask && dominant && target && out && out->count, "NULL argument");
  ADP_CHECK_ARG(n >= 0 && n < (1LL << 31) && n_cand >= 0 && n_cand <= n, "bad n or n_cand");
  ADP_CHECK_ARG(n_cand == 0 || candidates, "NULL candidates");
  ADP_CHECK_ARG(out->capacity >= 0, "negative capacity");
  ADP_CHECK_ARG(out->capacity == 0 || (out->view && out->parent && out->label && out->band &&
                                       out->moments && out->stats),
                "NULL region array");
  CamSet cs;
  int rc = make_camset(cams, n_views, prm, &cs);
  if (rc) return rc;
  ADP_CHECK_ARG(prm->r_erode >= 0 && prm->r_erode <= ERODE_RMAX, "r_erode must be 0..64");
  for (int v = 0; v < n_views; ++v)  // the moment sums split coordinates into 8-bit halves
    ADP_CHECK_ARG(cs.cam[v].width < 65536 && cs.cam[v].height < 65536,
                  "image sides must be below 65536");
  long long P = total_pixels(cs);
  ADP_CHECK_ARG(P < (1LL << 31), "too many pixels");
  ADP_CHECK_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
  size_t need = region_ws_bytes(n, P);
  ADP_CHECK_ARG(ws_bytes >= need, "workspace %zu bytes, need %zu", ws_bytes, need);
  cudaStream_t st = (cudaStream_t)stream;
  Carver c(ws, ws_bytes);
  RegionWs w;
  w.L = c.take<int>(P);
  w.slot = c.take<int>(P);
  w.root_pix = c.take<int>(P);
  w.mom = c.take<long long>(6 * P);
  w.part = c.take<long long>(6 * P);
  w.lroots = c.take<int>(P);
  w.kept_idx = c.take<long long>(P);
  w.cand = c.take<uint8_t>(n);
  w.scan = c.take<char>(scan_workspace_bytes(P));
  w.scan2 = c.take<char>(scan_workspace_bytes(P));
  w.counters = c.take<long long>(4);
  // the candidate flags, the counters and both scans' status words are reset by
  // the erosion's launch
  FillSet fill;
  fill.add(w.cand, (size_t)n);
  fill.add(w.counters, 4 * sizeof(long long));
  scan_clear(fill, w.scan, P);
  scan_clear(fill, w.scan2, P);
  ADP_CHECK_ARG(!fill.overflow, "internal: too many ranges in one fill");

  dim3 grid(view_grid(cs), n_views);
  // erosion -> mask bit 1
  {
    int max_et = 0;
    for (int v = 0; v < n_views; ++v) {
      int t = ((cs.cam[v].width + ERODE_T - 1) / ERODE_T) * ((cs.cam[v].height + ERODE_T - 1) / ERODE_T);
      max_et = t > max_et ? t : max_et;
    }
    erode_kernel<<<dim3(max_et, n_views), 256, erode_smem_bytes(prm->r_erode), st>>>(
        maps->mask, cs, prm->r_erode, fill);
  }
  // candidate flags
  if (n_cand > 0)
    scatter_flag_kernel<<<grid_for(n_cand, 256, 4096), 256, 0, st>>>(candidates, n_cand, n,
                                                                      w.cand);
  // labelling
  unsigned gp = grid_for(P, 256, 148 * 16);
  unsigned long long* n_lroots = reinterpret_cast<unsigned long long*>(&w.counters[2]);
  {
    int max_tiles = 0;
    for (int v = 0; v < n_views; ++v) {
      int t = ((cs.cam[v].width + CCL_T - 1) / CCL_T) * ((cs.cam[v].height + CCL_T - 1) / CCL_T);
      max_tiles = t > max_tiles ? t : max_tiles;
    }
    ccl_local_kernel<<<dim3(max_tiles, n_views), 256, 0, st>>>(maps->mask, dominant, w.cand, n,
                                                                cs, w.L, w.part, w.lroots,
                                                                n_lroots);
    ccl_border_kernel<<<dim3(grid_for((long long)max_tiles * CCL_BORDER, 256), n_views), 256, 0,
                        st>>>(maps->mask, dominant, cs, w.L);
  }
  if (out->labels) ccl_flatten_kernel<<<gp, 256, 0, st>>>(w.L, P);
  ADP_LAUNCH_CHECK();
  // roots -> slots
  int* L = w.L;
  int* slot = w.slot;
  int* root_pix = w.root_pix;
  rc = scan_exclusive([=] __device__(long long p) -> long long { return L[p] == p ? 1 : 0; },
                      [=] __device__(long long p, long long pre) {
                        if (L[p] == p) {
                          slot[p] = (int)pre;
                          root_pix[pre] = (int)p;
                        }
                      },
                      P, nullptr, &w.counters[0], w.scan, st, d_status, /*cleared=*/true);
  if (rc) return rc;
  count_guard_kernel<<<1, 1, 0, st>>>(scan_error_flag(w.scan, P), &w.counters[0]);
  zero_i64_kernel<<<gp, 256, 0, st>>>(w.mom, &w.counters[0], 6);
  moments_kernel<<<grid_for(P, 256, 148 * 8), 256, 0, st>>>(w.lroots, n_lroots, w.part, w.L,
                                                            w.slot, w.mom);
  ADP_LAUNCH_CHECK();
  // area filter: kept index of every root, total -> out->count
  const long long* mom = w.mom;
  long long* kept = w.kept_idx;
  int m_min = prm->m_min;
  rc = scan_exclusive(
      [=] __device__(long long r) -> long long { return mom[6 * r] >= m_min ? 1 : 0; },
      [=] __device__(long long r, long long pre) { kept[r] = pre; }, P, &w.counters[0],
      (long long*)out->count, w.scan2, st, d_status, /*cleared=*/true);
  if (rc) return rc;
  RegionArgs ra;
  ra.mom = w.mom;
  ra.root_pix = w.root_pix;
  ra.kept_idx = w.kept_idx;
  ra.d_nroots = &w.counters[0];
  ra.dom = dominant;
  ra.mask = maps->mask;
  ra.tgt = target;
  ra.m_min = prm->m_min;
  ra.cap = out->capacity;
  ra.view = out->view;
  ra.parent = out->parent;
  ra.label = out->label;
  ra.band = out->band;
  ra.moments = (long long*)out->moments;
  ra.stats = out->stats;
  region_stats_kernel<<<gp, 256, 0, st>>>(ra, cs);
  if (out->labels)
    labels_out_kernel<<<grid, 256, 0, st>>>(w.L, w.mom, w.slot, prm->m_min, cs, out->labels);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

// ------------------------------------------------------------------ top-k without allocation
//
// A variant of adp_select_topk for callers that cannot allocate device memory
// (or call cudaMalloc) at the point they run, e.g. code inside a custom
// allocator, a memory-capped host framework or a context where allocation
// would break an outer stream capture. Its scratch lives in the statically
// allocated device array below, sized for at most ADP_TOPK_NOALLOC_MAX_N
// Gaussians. Every device that loads the library keeps this array until the
// process exits.

namespace adp {

// Scratch of the allocation-free top-k: selection state, histogram, one flag
// byte per Gaussian, scan block sums and two counters (all 256-aligned).
constexpr long long kNoallocMaxN = ADP_TOPK_NOALLOC_MAX_N;
constexpr size_t kNoallocBytes =
    8 * 256 * 4 /*histograms*/ + 256 /*min/max*/ + 256 /*barrier*/ +
    2 * TOPK_MAX_BLOCKS * 8 /*block counts*/ + ((kNoallocMaxN + 255) / 256) * 256 /*flags*/;
static __device__ __align__(256) unsigned char g_topk_scratch[kNoallocBytes];

// Per-device address of g_topk_scratch, looked up once per device.
static void* g_topk_scratch_ptr[64];
static std::mutex g_topk_scratch_mu;

static int topk_scratch_address(void** out) {
  int dev = 0;
  ADP_CUDA(cudaGetDevice(&dev));
  ADP_CHECK_ARG(dev >= 0 && dev < 64, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_topk_scratch_mu);
  if (!g_topk_scratch_ptr[dev]) {
    void* p = nullptr;
    ADP_CUDA(cudaGetSymbolAddress(&p, g_topk_scratch));
    g_topk_scratch_ptr[dev] = p;
  }
  *out = g_topk_scratch_ptr[dev];
  return ADP_OK;
}

}  // namespace adp

extern "C" ADP_API int adp_select_topk_noalloc(const double* mass, int64_t n, int64_t k,
                                               int32_t* out_ids, int32_t* d_status,
                                               adp_stream_t stream) {
  ADP_CHECK_ARG(n >= 0 && k >= 0, "bad n or k");
  ADP_CHECK_ARG(n <= ADP_TOPK_NOALLOC_MAX_N,
                "n = %lld exceeds the %lld Gaussians the static scratch of "
                "adp_select_topk_noalloc holds; use adp_select_topk with a workspace",
                (long long)n, (long long)ADP_TOPK_NOALLOC_MAX_N);
  ADP_CHECK_ARG(k == 0 || (mass && out_ids), "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (k > n) k = n;
  if (k == 0) return ADP_OK;
  if (k == n) {
    iota_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(out_ids, n);
    ADP_LAUNCH_CHECK();
    return ADP_OK;
  }
  void* base = nullptr;
  int rc = topk_scratch_address(&base);
  if (rc) return rc;
  ADP_CHECK_ARG(topk_coop_bytes(n) <= kNoallocBytes, "internal: static scratch too small");
  return topk_coop_run(mass, n, k, out_ids, base, kNoallocBytes, d_status, st);
}

// Error strings, defaults, camera set construction, and the non-template parts
// of the scan and radix sort.
#include <atomic>
#include <cstdarg>
#include <cstring>

#include "common.cuh"
#include "gauss_math.cuh"

namespace adp {

static thread_local char g_err[512] = "";

// Poll bound of every device wait (see adp_set_spin_limit). About a second of
// polling on a B300 at the default; read at each launch.
constexpr long long kDefaultSpinLimit = 1LL << 22;
static std::atomic<long long> g_spin_limit{kDefaultSpinLimit};
long long spin_limit() { return g_spin_limit.load(std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int make_camset(const adp_camera* cams, int n_views, const adp_params* prm, CamSet* cs) {
  ADP_CHECK_ARG(cams != nullptr, "cams is NULL");
  ADP_CHECK_ARG(n_views >= 1 && n_views <= ADP_MAX_VIEWS, "n_views %d outside [1, %d]", n_views,
                ADP_MAX_VIEWS);
  ADP_CHECK_ARG(prm != nullptr, "params is NULL");
  ADP_CHECK_ARG(prm->tile_w > 0 && prm->tile_h > 0 && prm->tile_w * prm->tile_h == 256,
                "tile %dx%d must have 256 pixels", prm->tile_w, prm->tile_h);
  ADP_CHECK_ARG(prm->batch == 0 || prm->batch == 64 || prm->batch == 128 || prm->batch == 256,
                "batch %d must be 0, 64, 128 or 256", prm->batch);
  memset(cs, 0, sizeof(*cs));
  cs->n_views = n_views;
  cs->tile_w = prm->tile_w;
  cs->tile_h = prm->tile_h;
  cs->tile_base[0] = 0;
  cs->pix_base[0] = 0;
  for (int v = 0; v < n_views; ++v) {
    const adp_camera& c = cams[v];
    ADP_CHECK_ARG(c.width > 0 && c.height > 0 && c.width <= 16384 && c.height <= 16384,
                  "view %d: bad size %dx%d", v, c.width, c.height);
    ADP_CHECK_ARG(c.fx > 0 && c.fy > 0, "view %d: focal lengths must be positive", v);
    cs->cam[v] = c;
    cs->lim_x[v] = 1.3f * (float)c.width / (2.f * c.fx);
    cs->lim_y[v] = 1.3f * (float)c.height / (2.f * c.fy);
    cs->tiles_x[v] = (c.width + prm->tile_w - 1) / prm->tile_w;
    cs->tiles_y[v] = (c.height + prm->tile_h - 1) / prm->tile_h;
    long long nt = (long long)cs->tile_base[v] + (long long)cs->tiles_x[v] * cs->tiles_y[v];
    ADP_CHECK_ARG(nt < (1LL << 30), "too many tiles");
    cs->tile_base[v + 1] = (int)nt;
    cs->pix_base[v + 1] = cs->pix_base[v] + (long long)c.width * c.height;
  }
  return ADP_OK;
}

__global__ void fill_i32_kernel(int* p, long long n, int v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

// ----------------------------------------------------------------- scan

// ----------------------------------------------------------------- radix sort

__global__ void rs_hist_kernel(const unsigned* keys, const unsigned* vals, const long long* d_n,
                               long long tiles_max, DigitOp op, unsigned* hist) {
  __shared__ unsigned s_hist[RS_BINS];
  long long N = *d_n;
  long long nt = (N + RS_TILE - 1) / RS_TILE;
  if (nt > tiles_max) nt = tiles_max;
  for (long long t = blockIdx.x; t < nt; t += gridDim.x) {
    s_hist[threadIdx.x] = 0;
    __syncthreads();
    long long base = t * RS_TILE;
    unsigned d[RS_ROUNDS];
#pragma unroll
    for (int k = 0; k < RS_ROUNDS; ++k) {  // all loads first, then the shared atomics
      long long i = base + (long long)k * RS_THREADS + threadIdx.x;
      d[k] = i < N ? (op.divisor ? op(0u, vals[i]) : op(keys[i], 0u)) : (unsigned)RS_BINS;
    }
#pragma unroll
    for (int k = 0; k < RS_ROUNDS; ++k)
      if (d[k] < (unsigned)RS_BINS) atomicAdd(&s_hist[d[k]], 1u);
    __syncthreads();
    if ((int)threadIdx.x < op.bins()) hist[(size_t)threadIdx.x * tiles_max + t] = s_hist[threadIdx.x];
    __syncthreads();
  }
}

// One block per digit: exclusive scan of that digit's per-tile counts, each thread
// taking RS_SCAN_ITEMS consecutive tiles of a round (so a block needs few rounds,
// each with two barriers, even for tens of thousands of tiles).
constexpr int RS_SCAN_ITEMS = 8;
__global__ void rs_scan_kernel(unsigned* hist, const long long* d_n, long long tiles_max,
                               int bins, unsigned* digit_tot) {
  __shared__ unsigned s_warp[RS_WARPS];
  __shared__ unsigned s_carry;
  if ((int)blockIdx.x >= bins) {  // a digit the pass cannot produce
    if (threadIdx.x == 0) digit_tot[blockIdx.x] = 0u;
    return;
  }
  long long N = *d_n;
  long long nt = (N + RS_TILE - 1) / RS_TILE;
  if (nt > tiles_max) nt = tiles_max;
  unsigned* row = hist + (size_t)blockIdx.x * tiles_max;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (long long base = 0; base < nt; base += (long long)RS_THREADS * RS_SCAN_ITEMS) {
    const long long i0 = base + (long long)threadIdx.x * RS_SCAN_ITEMS;
    unsigned x[RS_SCAN_ITEMS];
    unsigned tsum = 0;
#pragma unroll
    for (int k = 0; k < RS_SCAN_ITEMS; ++k) {
      x[k] = i0 + k < nt ? row[i0 + k] : 0u;
      tsum += x[k];
    }
    unsigned inc = tsum;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    unsigned wpre = 0, btot = 0;
    for (int k = 0; k < RS_WARPS; ++k) {
      wpre += k < w ? s_warp[k] : 0u;
      btot += s_warp[k];
    }
    unsigned run = s_carry + wpre + inc - tsum;
#pragma unroll
    for (int k = 0; k < RS_SCAN_ITEMS; ++k) {
      if (i0 + k < nt) row[i0 + k] = run;
      run += x[k];
    }
    __syncthreads();  // every thread has read s_carry and s_warp
    if (threadIdx.x == 0) s_carry += btot;
    __syncthreads();
  }
  if (threadIdx.x == 0) digit_tot[blockIdx.x] = s_carry;
}

// Block-wide exclusive scan of one value per thread (RS_THREADS threads).
__device__ __forceinline__ unsigned block_excl_scan(unsigned x, unsigned* s_w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned inc = x;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  unsigned pre = 0;
  for (int k = 0; k < warp; ++k) pre += s_w[k];
  __syncthreads();
  return pre + inc - x;
}

// Stable scatter of one pass. A warp ranks its RS_ROUNDS rounds of 32 items in
// item order: the lanes holding the same digit are found with one ballot per digit
// bit (the pass's 1 to 8), and the lowest of them adds the run to the warp's count
// of that digit with one shared atomic, the rounds separated by __syncwarp (which
// orders the atomics of different lanes) so that all are in flight before the first
// result is read.
// The tile is then reordered by digit in shared memory and each digit's run is
// written to global memory by consecutive threads.
// Four resident blocks per SM (64 registers, no spills) hide the shared-memory
// latency of the ranking better than three at the unconstrained 76-80 registers.
__global__ void __launch_bounds__(RS_THREADS, 4)
    rs_scatter_kernel(const unsigned* keys_in, const unsigned* vals_in, unsigned* keys_out,
                      unsigned* vals_out, const long long* d_n, long long tiles_max, DigitOp op,
                      const unsigned* hist, const unsigned* digit_tot, bool drop_none) {
  __shared__ unsigned s_base[RS_BINS];             // global start of every digit
  __shared__ unsigned s_whist[RS_WARPS][RS_BINS];  // per-warp counts, then warp prefixes
  __shared__ unsigned s_lbase[RS_BINS];            // start of every digit within the tile
  __shared__ unsigned s_delta[RS_BINS];            // global minus tile position of the digit
  __shared__ unsigned s_w[RS_WARPS];
  __shared__ unsigned s_keys[RS_TILE];
  __shared__ unsigned s_vals[RS_TILE];
  __shared__ unsigned s_kept;                      // items of the tile that are written
  long long N = *d_n;
  long long nt = (N + RS_TILE - 1) / RS_TILE;
  if (nt > tiles_max) nt = tiles_max;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  s_base[threadIdx.x] = block_excl_scan(digit_tot[threadIdx.x], s_w);
  const unsigned lt = lanemask_lt();
  for (long long t = blockIdx.x; t < nt; t += gridDim.x) {
    for (int d = threadIdx.x; d < RS_WARPS * RS_BINS; d += RS_THREADS) (&s_whist[0][0])[d] = 0;
    __syncthreads();
    const long long tile0 = t * RS_TILE;
    const long long base = tile0 + (long long)warp * (RS_ROUNDS * 32);
    unsigned key[RS_ROUNDS], val[RS_ROUNDS], dig[RS_ROUNDS], peers[RS_ROUNDS], off[RS_ROUNDS];
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {  // issue every load before the ranking
      long long i = base + r * 32 + lane;
      key[r] = i < N ? keys_in[i] : 0u;
      val[r] = i < N ? vals_in[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
      long long i = base + r * 32 + lane;
      const bool valid = i < N && !(drop_none && key[r] == RS_DROP_KEY);
      const unsigned d = valid ? op(key[r], val[r]) : (unsigned)RS_BINS;
      dig[r] = d;
      unsigned p = __ballot_sync(0xffffffffu, valid);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        if (b < op.bits) {  // uniform: the pass's digit width
          const unsigned m = __ballot_sync(0xffffffffu, (d >> b) & 1u);
          p &= ((d >> b) & 1u) ? m : ~m;
        }
      }
      peers[r] = valid ? p : 0u;
    }
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
      off[r] = 0u;
      if (peers[r] != 0u && (peers[r] & lt) == 0u)
        off[r] = atomicAdd(&s_whist[warp][dig[r]], (unsigned)__popc(peers[r]));
      __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
      const int leader = peers[r] != 0u ? __ffs(peers[r]) - 1 : lane;
      off[r] = __shfl_sync(0xffffffffu, off[r], leader) + __popc(peers[r] & lt);
    }
    __syncthreads();
    unsigned cnt;
    {  // per-digit exclusive prefix over warps, and the tile's count of the digit
      int d = threadIdx.x;
      unsigned run = 0;
      for (int w2 = 0; w2 < RS_WARPS; ++w2) {
        unsigned c = s_whist[w2][d];
        s_whist[w2][d] = run;
        run += c;
      }
      cnt = run;
    }
    unsigned lb = block_excl_scan(cnt, s_w);
    s_lbase[threadIdx.x] = lb;
    if (threadIdx.x == RS_BINS - 1) s_kept = lb + cnt;
    s_delta[threadIdx.x] =
        s_base[threadIdx.x] +
        ((int)threadIdx.x < op.bins() ? hist[(size_t)threadIdx.x * tiles_max + t] : 0u) - lb;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
      if (dig[r] < (unsigned)RS_BINS) {  // in range and not dropped
        unsigned d = dig[r];
        unsigned lpos = s_lbase[d] + s_whist[warp][d] + off[r];
        s_keys[lpos] = key[r];
        s_vals[lpos] = val[r];
      }
    }
    __syncthreads();
    const int kept = (int)s_kept;
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {  // kept <= RS_TILE
      const int j = r * RS_THREADS + (int)threadIdx.x;
      if (j < kept) {
        const unsigned k = s_keys[j], vv = s_vals[j];
        const unsigned pos = s_delta[op(k, vv)] + (unsigned)j;
        keys_out[pos] = k;
        vals_out[pos] = vv;
      }
    }
    __syncthreads();
  }
}

// Stable LSD radix sort of at most SMALL_SORT_MAX pairs in one block of 1024
// threads (the data stay in global memory, L2-resident at this size): per pass a
// shared histogram, its exclusive scan, then rounds of 1024 items in order, each
// ranked by warp match masks and per-warp digit counts, so equal digits keep
// their order. Results end in (ka, va).
__global__ void __launch_bounds__(1024)
    small_sort_kernel(unsigned* ka, unsigned* va, unsigned* kb, unsigned* vb, const long long* d_n,
                      long long n_max, SmallPasses passes) {
  __shared__ unsigned s_base[RS_BINS];
  __shared__ unsigned s_run[RS_BINS];
  __shared__ unsigned s_wc[32][RS_BINS];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  long long N = *d_n;
  if (N > n_max) N = n_max;
  const unsigned lt = lanemask_lt();
  unsigned *src_k = ka, *src_v = va, *dst_k = kb, *dst_v = vb;
  for (int p = 0; p < passes.count; ++p) {
    const DigitOp op = passes.op[p];
    if (t < RS_BINS) {
      s_base[t] = 0u;
      s_run[t] = 0u;
    }
    __syncthreads();
    for (long long i = t; i < N; i += 1024) atomicAdd(&s_base[op(src_k[i], src_v[i])], 1u);
    __syncthreads();
    if (t < 32) {  // exclusive scan of the 256 bins, 8 per lane
      unsigned c[8], sum = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        c[q] = s_base[8 * t + q];
        sum += c[q];
      }
      unsigned inc = sum;
      for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      unsigned run = inc - sum;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        s_base[8 * t + q] = run;
        run += c[q];
      }
    }
    __syncthreads();
    for (long long r0 = 0; r0 < N; r0 += 1024) {
      for (int q = t; q < 32 * RS_BINS; q += 1024) (&s_wc[0][0])[q] = 0u;
      __syncthreads();
      const long long i = r0 + t;
      const bool valid = i < N;
      const unsigned k = valid ? src_k[i] : 0u, v = valid ? src_v[i] : 0u;
      const unsigned d = valid ? op(k, v) : (unsigned)RS_BINS;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const unsigned rank = __popc(peers & lt);
      if (valid && rank == 0) s_wc[warp][d] = __popc(peers);
      __syncthreads();
      if (t < RS_BINS) {  // prefix over warps, continuing the digit's running count
        unsigned run = s_run[t];
        for (int w = 0; w < 32; ++w) {
          const unsigned c = s_wc[w][t];
          s_wc[w][t] = run;
          run += c;
        }
        s_run[t] = run;
      }
      __syncthreads();
      if (valid) {
        const unsigned pos = s_base[d] + s_wc[warp][d] + rank;
        dst_k[pos] = k;
        dst_v[pos] = v;
      }
      __syncthreads();
    }
    unsigned* tk = src_k; src_k = dst_k; dst_k = tk;
    unsigned* tv = src_v; src_v = dst_v; dst_v = tv;
  }
  if (src_k != ka)  // odd pass count: copy back
    for (long long i = t; i < N; i += 1024) {
      ka[i] = src_k[i];
      va[i] = src_v[i];
    }
}

// After a pass that dropped items: the count the later passes sort.
__global__ void rs_kept_count_kernel(const unsigned* digit_tot, long long* d_n) {
  __shared__ unsigned long long s_sum[RS_BINS / 32];
  unsigned long long x = digit_tot[threadIdx.x];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < RS_BINS / 32; ++w) t += s_sum[w];
    *d_n = (long long)t;
  }
}

int radix_sort_pairs(unsigned* keys, unsigned* vals, long long* d_n, long long n_max,
                     const DigitOp* passes, int n_passes, const SortWorkspace& w,
                     cudaStream_t st, bool first_hist_done, bool drop_none, unsigned** res_keys,
                     unsigned** res_vals) {
  if (res_keys) *res_keys = keys;
  if (res_vals) *res_vals = vals;
  if (n_max <= 0 || n_passes <= 0) return ADP_OK;
  if (n_max <= SMALL_SORT_MAX && n_passes <= 4 && !first_hist_done) {  // one small launch
    SmallPasses sp;
    sp.count = n_passes;
    for (int p = 0; p < n_passes; ++p) sp.op[p] = passes[p];
    small_sort_kernel<<<1, 1024, 0, st>>>(keys, vals, w.keys_alt, w.vals_alt, d_n, n_max, sp);
    ADP_LAUNCH_CHECK();
    return ADP_OK;
  }
  unsigned *ka = keys, *va = vals, *kb = w.keys_alt, *vb = w.vals_alt;
  long long grid = w.tiles_max < 148 * 8 ? w.tiles_max : 148 * 8;
  for (int p = 0; p < n_passes; ++p) {
    if (p > 0 || !first_hist_done)
      rs_hist_kernel<<<(unsigned)grid, RS_THREADS, 0, st>>>(ka, va, d_n, w.tiles_max, passes[p],
                                                             w.hist);
    rs_scan_kernel<<<RS_BINS, RS_THREADS, 0, st>>>(w.hist, d_n, w.tiles_max, passes[p].bins(),
                                                    w.digit_tot);
    const bool drop = drop_none && first_hist_done && p == 0;
    rs_scatter_kernel<<<(unsigned)grid, RS_THREADS, 0, st>>>(ka, va, kb, vb, d_n, w.tiles_max,
                                                              passes[p], w.hist, w.digit_tot, drop);
    if (drop) rs_kept_count_kernel<<<1, RS_BINS, 0, st>>>(w.digit_tot, d_n);
    ADP_LAUNCH_CHECK();
    unsigned* tk = ka; ka = kb; kb = tk;
    unsigned* tv = va; va = vb; vb = tv;
  }
  if (ka != keys) {  // odd pass count: results live in the alternate buffers
    if (res_keys && res_vals) {
      *res_keys = ka;
      *res_vals = va;
      return ADP_OK;
    }
    ADP_CUDA(cudaMemcpyAsync(keys, ka, sizeof(unsigned) * n_max, cudaMemcpyDeviceToDevice, st));
    ADP_CUDA(cudaMemcpyAsync(vals, va, sizeof(unsigned) * n_max, cudaMemcpyDeviceToDevice, st));
  }
  return ADP_OK;
}

constexpr int AUX_MAX_DEVICES = 64;
static AuxStream g_aux[AUX_MAX_DEVICES];
static std::mutex g_aux_mu;

std::mutex& aux_mutex() { return g_aux_mu; }

int aux_stream(AuxStream** out) {
  int dev = 0;
  ADP_CUDA(cudaGetDevice(&dev));
  ADP_CHECK_ARG(dev >= 0 && dev < AUX_MAX_DEVICES, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_aux_mu);
  AuxStream& a = g_aux[dev];
  if (!a.stream) {
    int lo = 0, hi = 0;
    ADP_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    ADP_CUDA(cudaEventCreateWithFlags(&a.planned, cudaEventDisableTiming));
    ADP_CUDA(cudaEventCreateWithFlags(&a.merged, cudaEventDisableTiming));
    ADP_CUDA(cudaEventCreateWithFlags(&a.forked, cudaEventDisableTiming));
    ADP_CUDA(cudaEventCreateWithFlags(&a.joined, cudaEventDisableTiming));
    ADP_CUDA(cudaStreamCreateWithPriority(&a.stream, cudaStreamNonBlocking, hi));
  }
  *out = &a;
  return ADP_OK;
}

__global__ void count_guard_kernel(const unsigned long long* err, long long* count) {
  if (*err != 0ull) *count = 0;
}

__global__ void __launch_bounds__(256) fill_kernel(FillSet f) {
  fill_ranges_device(f, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                     (long long)gridDim.x * blockDim.x);
}

int launch_fill(const FillSet& f, cudaStream_t st) {
  ADP_CHECK_ARG(!f.overflow, "internal: more than %d ranges in one fill", FILL_MAX);
  long long chunks = 0;
  for (int s = 0; s < f.n; ++s) chunks = std::max(chunks, (f.bytes[s] + 15) / 16);
  if (chunks == 0) return ADP_OK;
  fill_kernel<<<grid_for(chunks, 256, 148 * 4), 256, 0, st>>>(f);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

}  // namespace adp

extern "C" {

ADP_API int32_t adp_version(void) { return ADP_VERSION; }

ADP_API const char* adp_last_error_string(void) { return adp::g_err; }

ADP_API void adp_set_spin_limit(int64_t max_polls) {
  adp::g_spin_limit.store(max_polls > 0 ? (long long)max_polls : adp::kDefaultSpinLimit,
                          std::memory_order_relaxed);
}

ADP_API void adp_get_constants(adp_constants* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->version = ADP_VERSION;
  c->max_views = ADP_MAX_VIEWS;
  c->tile_pixels = 256;
  c->max_sh_degree = 3;
  c->fov_clamp = 1.3f;
  c->gram_schmidt_eps = 1e-12;
  const float sh[16] = {SHC0, -SHC1, SHC1, -SHC1, SHC2_0, -SHC2_0, SHC2_2, -SHC2_0, SHC2_4,
                        -SHC3_0, SHC3_1, -SHC3_2, SHC3_3, -SHC3_2, SHC3_5, -SHC3_0};
  for (int k = 0; k < 16; ++k) c->sh_coef[k] = sh[k];
  c->topk_noalloc_max_n = ADP_TOPK_NOALLOC_MAX_N;
  c->default_spin_limit = adp::kDefaultSpinLimit;
  adp_default_params(&c->defaults);
}

ADP_API void adp_default_params(adp_params* p) {
  if (!p) return;
  p->tau_l1 = 0.1f;
  p->r_erode = 2;
  p->m_min = 5;
  p->n_levels = 3;
  p->n_max = 19;
  p->gamma_d = 2.0f;
  p->gamma_c = 0.15f;
  p->eps_t = 1e-8f;
  p->eta = 0.8f;
  p->scale_floor = 1e-7f;
  p->near_plane = 0.2f;
  p->low_pass = 0.3f;
  p->alpha_min = 1.0f / 255.0f;
  p->alpha_max = 0.99f;
  p->t_min = 1e-4f;
  p->tile_w = 16;
  p->tile_h = 16;
  p->batch = 256;
}

}  // extern "C"

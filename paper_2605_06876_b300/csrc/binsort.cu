// Tile binning with a depth sort (Eq. 1: Gaussians blended in depth order).
//
// Instead of one wide sort of (tile, depth) keys over every instance, the
// visible (view, Gaussian) records are sorted once by (view, depth, id) -- four
// 8-bit passes over 32-bit depth keys, plus one pass on the view -- and then
// duplicated into their tiles in that order; a stable sort of the instances on
// the tile index alone (2-3 passes) leaves every tile's list in (depth, id)
// order. This moves far fewer bytes than sorting 64-bit keys over all
// instances, and ties in depth resolve to the lower id because every pass is
// stable over id-ordered input. Instances whose alpha ellipse misses their tile
// (the rectangle of tiles overestimates a rotated ellipse, about a fifth of the
// instances) are dropped by the first pass of the tile sort, which changes no
// pixel's contributors.
#include <algorithm>

#include "common.cuh"

namespace adp {

// The instance count the duplication and the tile sort process: the required
// count if it fits the capacity and the offset scan completed, else 0 (nothing
// binned).
__global__ void clamp_count_kernel(const long long* K, long long cap,
                                   const unsigned long long* scan_err, long long* Kc) {
  long long k = *K;
  *Kc = (k <= cap && *scan_err == 0ull) ? k : 0;
}

// Load-balanced duplication: each CTA takes a chunk of DUP_CHUNK consecutive
// instances. The record owning the chunk's first instance comes from the offset
// scan (chunk_first), and the chunk's record offsets are staged in shared memory.
// The records the chunk overlaps (usually a few dozen, at most DUP_CHUNK + 1) are
// loaded once, up to DUP_REC at a time, one thread each, into shared memory (view,
// id, tile origin, width and its reciprocal, 2D mean, conic and the alpha cut-off);
// each record marks the slot of the chunk where it starts, and an inclusive
// max-scan over the slots gives every instance its record, with no search per
// instance. Each thread takes DUP_ITEMS consecutive instances. k's tile is its
// position within the record's tile rectangle (row-major). Balanced whatever a
// Gaussian's footprint, one round of dependent loads per chunk (not per sub-chunk),
// and each thread stores its instances as 16-byte vectors. A chunk is one tile of
// the radix sort, so the CTA also writes that tile's histogram of the tile sort's
// first digit (the low 8 bits of the key).
constexpr int DUP_CHUNK = 2048;
constexpr int DUP_THREADS = 256;
constexpr int DUP_ITEMS = DUP_CHUNK / DUP_THREADS;
// Records staged per batch: a chunk's ~100 records (about 21 instances each on the
// 1M workloads) fit one batch, and the smaller shared-memory footprint than with 512
// leaves more of the SM's unified L1 to the records' gathers (16 views: 599 -> 480 us).
constexpr int DUP_REC = 256;
static_assert(DUP_CHUNK == RS_TILE, "a duplication chunk is one radix-sort tile");
static_assert(DUP_ITEMS == 8, "two 16-byte stores of keys and of ids per thread");
constexpr unsigned TILE_NONE = 0xffffffffu;  // sorts after every real tile

// Whether the ellipse q(d) = d^T C d <= k around the 2D mean (the pixels where
// o exp(-q/2) >= alpha_min) reaches the rectangle of pixel centres
// [x0, x1] x [y0, y1]: the minimum of the convex quadratic over the rectangle is
// 0 if the mean is inside, else it lies on an edge, where the 1-D minimum is the
// clamped stationary point (dy = -B dx / C on a vertical edge, dx = -B dy / A on
// a horizontal one; rbc = -B / C and rba = -B / A come precomputed per record).
// A small relative and absolute margin keeps the test conservative under float32
// rounding, so no contributing pixel is ever lost.
__device__ __forceinline__ bool ellipse_meets_rect(float mx, float my, float A, float B, float C,
                                                   float k, float rbc, float rba, float x0,
                                                   float x1, float y0, float y1) {
  if (mx >= x0 && mx <= x1 && my >= y0 && my <= y1) return true;
  float qmin = 3.4e38f;
  for (int e = 0; e < 2; ++e) {  // vertical edges x = x0, x1: q(dy) = A dx^2 + 2 B dx dy + C dy^2
    float dx = (e ? x1 : x0) - mx;
    float dy = fminf(fmaxf(rbc * dx, y0 - my), y1 - my);
    qmin = fminf(qmin, A * dx * dx + 2.f * B * dx * dy + C * dy * dy);
  }
  for (int e = 0; e < 2; ++e) {  // horizontal edges y = y0, y1
    float dy = (e ? y1 : y0) - my;
    float dx = fminf(fmaxf(rba * dy, x0 - mx), x1 - mx);
    qmin = fminf(qmin, A * dx * dx + 2.f * B * dx * dy + C * dy * dy);
  }
  return qmin <= k * 1.0001f + 1e-3f;
}

__global__ void __launch_bounds__(DUP_THREADS, 5) duplicate_kernel(
    const unsigned* vvals, const long long* offs, const int* chunk_first, const long long* d_nvis,
    const long long* d_K, long long cap, const int4* rect, const float4* xyod, const float4* conic,
    float alpha_min, long long n, CamSet cs, int view_shift, unsigned* tkeys, int* inst,
    bool inst_vec, unsigned hist_mask, unsigned* hist, long long tiles_max) {
  __shared__ int s_off[DUP_CHUNK + 1];  // record offsets of the chunk (the first may be < 0)
  __shared__ int s_i[DUP_REC];          // Gaussian id
  __shared__ int s_org[DUP_REC];        // first tile column | first tile row << 16
  __shared__ int s_wv[DUP_REC];         // rectangle width | view << 16 | (multi-tile) << 31
  __shared__ float s_iw[DUP_REC];       // 1 / rectangle width
  __shared__ float4 s_e0[DUP_REC];      // 2D mean, conic A, B
  __shared__ float4 s_e1[DUP_REC];      // conic C, cut-off k, -B / C, -B / A
  __shared__ int s_rec[DUP_CHUNK];      // 1 + batch record starting at each slot, else 0
  __shared__ int s_wm[DUP_THREADS / 32];
  __shared__ unsigned s_h[RS_BINS];
  const long long N = *d_nvis, K = *d_K;  // K: the clamped count (0 = bin nothing)
  if (K == 0 || K > cap || N == 0) return;
  const long long n_chunks = (K + DUP_CHUNK - 1) / DUP_CHUNK;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e0 = DUP_ITEMS * (int)threadIdx.x;  // the thread's first slot
  for (int e = threadIdx.x; e < DUP_CHUNK; e += DUP_THREADS) s_rec[e] = 0;
  for (long long t = blockIdx.x; t < n_chunks; t += gridDim.x) {
    const long long k0 = t * DUP_CHUNK;
    const int kn = (int)min((long long)DUP_CHUNK, K - k0);  // instances in the chunk
    const long long j0 = chunk_first[t];
    const long long j1 = t + 1 < n_chunks ? (long long)chunk_first[t + 1] : N - 1;
    const int cnt = (int)(j1 - j0 + 1);  // <= DUP_CHUNK + 1: every record owns >= 1 instance
    for (int q = threadIdx.x; q < cnt; q += DUP_THREADS) s_off[q] = (int)(offs[j0 + q] - k0);
    for (int d = threadIdx.x; d < RS_BINS; d += DUP_THREADS) s_h[d] = 0u;
    __syncthreads();
    unsigned keys[DUP_ITEMS];
    int ids[DUP_ITEMS];
#pragma unroll
    for (int h = 0; h < DUP_ITEMS; ++h) {
      keys[h] = TILE_NONE;
      ids[h] = 0;
    }
    for (int rb = 0; rb < cnt; rb += DUP_REC) {  // record batches (one in the common case)
      const int rn = min(DUP_REC, cnt - rb);
      const int a0 = max(s_off[rb], 0);                        // the batch's slots
      const int a1 = rb + rn < cnt ? min(s_off[rb + rn], kn) : kn;  // [a0, a1)
      for (int q = threadIdx.x; q < rn; q += DUP_THREADS) {
        const unsigned p = vvals[j0 + rb + q];
        const int v = (int)(p / (unsigned long long)n);
        const int4 r = rect[p];
        const float4 xy = xyod[p], cn = conic[p];
        const int w = r.y - r.x + 1;
        const bool multi = w * (r.w - r.z + 1) > 1;
        s_i[q] = (int)(p - (unsigned long long)v * n);
        s_org[q] = r.x | (r.z << 16);
        s_wv[q] = w | (v << 16) | (multi ? (int)0x80000000u : 0);
        s_iw[q] = 1.f / (float)w;
        s_e0[q] = make_float4(xy.x, xy.y, cn.x, cn.y);
        s_e1[q] = multi ? make_float4(cn.z, 2.f * __logf(xy.z / alpha_min), -cn.y / cn.z,
                                      -cn.y / cn.x)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        // the chunk's first record may start before it (mark slot 0); the last one
        // listed may start exactly at the next chunk (no slot here)
        const int slot = max(s_off[rb + q], 0);
        if (slot < kn) s_rec[slot] = q + 1;
      }
      __syncthreads();
      // each slot's record: the largest mark at or before it (an inclusive max-scan)
      int mk[DUP_ITEMS];
      int run = 0;
#pragma unroll
      for (int h = 0; h < DUP_ITEMS; ++h) {
        run = max(run, s_rec[e0 + h]);
        mk[h] = run;
      }
      int inc = run;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = max(inc, y);
      }
      if (lane == 31) s_wm[warp] = inc;
      int before = __shfl_up_sync(0xffffffffu, inc, 1);
      if (lane == 0) before = 0;
      __syncthreads();
      for (int w2 = 0; w2 < warp; ++w2) before = max(before, s_wm[w2]);
#pragma unroll
      for (int h = 0; h < DUP_ITEMS; ++h) {
        const int kk = e0 + h;
        s_rec[kk] = 0;  // cleared for the next batch (each thread its own slots)
        if (kk < a0 || kk >= a1) continue;
        const int q = max(before, mk[h]) - 1;
        const int org = s_org[q], wv = s_wv[q];
        const int w = wv & 0xffff, v = (wv >> 16) & 0x7fff;
        const int tt = kk - s_off[rb + q];
        // tt = row * w + col: the quotient from the float reciprocal (tt < 2^24, so
        // it is off by at most one) and one correction step
        int qd = __float2int_rd(__int2float_rn(tt) * s_iw[q]);
        int rm = tt - qd * w;
        if (rm < 0) {
          --qd;
          rm += w;
        } else if (rm >= w) {
          ++qd;
          rm -= w;
        }
        const int ty = (org >> 16) + qd, tx = (org & 0xffff) + rm;
        unsigned key = (unsigned)(ty * cs.tiles_x[v] + tx) | ((unsigned)v << view_shift);
        if (wv < 0) {  // a one-tile rectangle always meets its ellipse
          const float4 f0 = s_e0[q];
          const float4 f1 = s_e1[q];
          const float x0 = (float)(tx * cs.tile_w), y0 = (float)(ty * cs.tile_h);
          const float x1 = fminf(x0 + (float)(cs.tile_w - 1), (float)(cs.cam[v].width - 1));
          const float y1 = fminf(y0 + (float)(cs.tile_h - 1), (float)(cs.cam[v].height - 1));
          if (!ellipse_meets_rect(f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w, x0, x1, y0, y1))
            key = TILE_NONE;
        }
        keys[h] = key;
        ids[h] = s_i[q];
        if (key != TILE_NONE) atomicAdd(&s_h[key & hist_mask], 1u);  // the sort drops the others
      }
      __syncthreads();  // the batch's records and marks are no longer read
    }
    const long long k = k0 + e0;  // a multiple of 8: 16-byte aligned stores
    if (e0 + DUP_ITEMS <= kn) {
      uint4* kv = reinterpret_cast<uint4*>(tkeys + k);
      kv[0] = make_uint4(keys[0], keys[1], keys[2], keys[3]);
      kv[1] = make_uint4(keys[4], keys[5], keys[6], keys[7]);
      if (inst_vec) {
        int4* iv = reinterpret_cast<int4*>(inst + k);
        iv[0] = make_int4(ids[0], ids[1], ids[2], ids[3]);
        iv[1] = make_int4(ids[4], ids[5], ids[6], ids[7]);
      } else {
#pragma unroll
        for (int h = 0; h < DUP_ITEMS; ++h) inst[k + h] = ids[h];
      }
    } else {
#pragma unroll
      for (int h = 0; h < DUP_ITEMS; ++h)
        if (e0 + h < kn) {
          tkeys[k + h] = keys[h];
          inst[k + h] = ids[h];
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d <= (int)hist_mask; d += DUP_THREADS)
      hist[(size_t)d * tiles_max + t] = s_h[d];
  }
}

// Per-tile ranges from the sorted keys (view-local tile | view << view_shift):
// a list starts where the key differs from the previous one and ends where it
// differs from the next. Each thread takes four consecutive keys (one 16-byte
// load; the keys buffer is 256-byte aligned) and the key before them.
__global__ void tile_ranges_kernel(const unsigned* tkeys, const long long* d_n, CamSet cs,
                                   int view_shift, int2* ranges) {
  const long long N = *d_n;
  const unsigned local_mask = (1u << view_shift) - 1u;
  const long long n4 = (N + 3) / 4;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    const long long j0 = 4 * q;
    unsigned k[6];  // k[0]: the key before, k[5]: the key after (TILE_NONE at the ends)
    if (j0 + 4 <= N) {
      const uint4 v = *reinterpret_cast<const uint4*>(tkeys + j0);
      k[1] = v.x; k[2] = v.y; k[3] = v.z; k[4] = v.w;
    } else {
      for (int e = 0; e < 4; ++e) k[1 + e] = j0 + e < N ? tkeys[j0 + e] : TILE_NONE;
    }
    k[0] = j0 > 0 ? tkeys[j0 - 1] : TILE_NONE;
    k[5] = j0 + 4 < N ? tkeys[j0 + 4] : TILE_NONE;
#pragma unroll
    for (int e = 1; e <= 4; ++e) {
      const unsigned t = k[e];
      if (t == TILE_NONE) continue;  // instances whose ellipse misses the tile, or past N
      const int g = cs.tile_base[t >> view_shift] + (int)(t & local_mask);
      const long long j = j0 + e - 1;
      if (k[e - 1] != t) ranges[g].x = (int)j;
      if (k[e + 1] != t) ranges[g].y = (int)(j + 1);
    }
  }
}

struct BinWs {
  long long* counters;  // [0] visible; [1] clamped instance count, then the kept ones
  void* scan;   // the compaction's scan
  void* scan2;  // the instance offsets' scan
  unsigned* vkeys;
  unsigned* vvals;
  long long* offs;
  unsigned* tkeys;
  int* chunk_first;  // [cap / DUP_CHUNK + 1] record owning each chunk's first instance
  SortWorkspace sort;
};

static long long dup_chunks(long long cap) { return (cap + DUP_CHUNK - 1) / DUP_CHUNK + 1; }

static size_t bin_ws_bytes(long long nv, long long cap) {
  long long m = nv > cap ? nv : cap;
  return carve_bytes<long long>(4) + 2 * scan_workspace_bytes(nv) + 2 * carve_bytes<unsigned>(nv) +
         carve_bytes<long long>(nv) + carve_bytes<unsigned>(cap) + carve_bytes<int>(dup_chunks(cap)) +
         sort_workspace_bytes(m);
}

static BinWs carve_bin(Carver& c, long long nv, long long cap) {
  BinWs w;
  long long m = nv > cap ? nv : cap;
  w.counters = c.take<long long>(4);
  w.scan = c.take<char>(scan_workspace_bytes(nv));
  w.scan2 = c.take<char>(scan_workspace_bytes(nv));
  w.vkeys = c.take<unsigned>(nv);
  w.vvals = c.take<unsigned>(nv);
  w.offs = c.take<long long>(nv);
  w.tkeys = c.take<unsigned>(cap);
  w.chunk_first = c.take<int>(dup_chunks(cap));
  w.sort = carve_sort(c, m);
  return w;
}

}  // namespace adp

using namespace adp;

extern "C" ADP_API size_t adp_bin_sort_workspace_size(int64_t n, int32_t n_views,
                                                      int64_t capacity) {
  if (n < 0 || n_views < 1 || capacity < 0) return 0;
  return bin_ws_bytes((long long)n * n_views, capacity);
}

extern "C" ADP_API int adp_bin_sort(int64_t n, const adp_projected* pr, const adp_camera* cams,
                                    int32_t n_views, const adp_params* prm, adp_bins* bins,
                                    void* ws, size_t ws_bytes, int32_t* d_status,
                                    adp_stream_t stream) {
  ADP_CHECK_ARG(pr && bins, "NULL argument");
  CamSet cs;
  int rc = make_camset(cams, n_views, prm, &cs);
  if (rc) return rc;
  ADP_CHECK_ARG(n >= 0 && (long long)n * n_views < (1LL << 31), "n_views * n exceeds 2^31");
  ADP_CHECK_ARG(bins->capacity >= 0 && bins->capacity < (1LL << 31), "capacity out of range");
  ADP_CHECK_ARG(bins->tile_range && bins->n_instances && (bins->inst_gauss || bins->capacity == 0),
                "NULL bins array");
  ADP_CHECK_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
  long long nv = (long long)n * n_views, cap = bins->capacity;
  size_t need = bin_ws_bytes(nv, cap);
  ADP_CHECK_ARG(ws_bytes >= need, "workspace %zu bytes, need %zu", ws_bytes, need);
  // instance keys: view-local tile | view << view_shift (see step 4)
  int max_local = 0;
  for (int v = 0; v < n_views; ++v) max_local = std::max(max_local, cs.tiles_x[v] * cs.tiles_y[v]);
  const int tile_bits = bits_for(max_local);
  const int view_shift = 8 * ((tile_bits + 7) / 8);
  ADP_CHECK_ARG(view_shift <= 24 && (long long)(n_views - 1) < (1LL << (32 - view_shift)) - 1,
                "too many tiles per view for the tile key");
  cudaStream_t st = (cudaStream_t)stream;
  long long n_tiles = cs.tile_base[n_views];
  // the empty tile ranges, the instance count and both scans' status words, in one launch
  FillSet fill;
  fill.add(bins->tile_range, sizeof(int2) * n_tiles);
  fill.add(bins->n_instances, sizeof(long long));
  Carver c(ws, ws_bytes);
  BinWs w;
  if (nv > 0) {
    w = carve_bin(c, nv, cap);
    scan_clear(fill, w.scan, nv);
    scan_clear(fill, w.scan2, nv);
  }
  rc = launch_fill(fill, st);
  if (rc || nv == 0) return rc;
  const int* tiles = pr->tiles_touched;
  const float4* xyod = reinterpret_cast<const float4*>(pr->xy_opacity_depth);

  // 1. compact the visible records with their depth keys
  unsigned* vkeys = w.vkeys;
  unsigned* vvals = w.vvals;
  rc = scan_exclusive(
      [=] __device__(long long p) -> long long { return tiles[p] > 0 ? 1 : 0; },
      [=] __device__(long long p, long long pre) {
        if (tiles[p] > 0) {
          vkeys[pre] = __float_as_uint(xyod[p].w);
          vvals[pre] = (unsigned)p;
        }
      },
      nv, nullptr, &w.counters[0], w.scan, st, d_status, /*cleared=*/true);
  if (rc) return rc;
  count_guard_kernel<<<1, 1, 0, st>>>(scan_error_flag(w.scan, nv), &w.counters[0]);

  // 2. stable sort by depth, then by view
  DigitOp passes[5];
  int np = 0;
  for (int s = 0; s < 32; s += 8) passes[np++] = DigitOp{s, 0u};
  if (n_views > 1) passes[np++] = DigitOp{0, (unsigned)n, bits_for(n_views - 1)};
  // the sorted records stay where the last pass wrote them (the tile sort reuses
  // the alternate buffers only after the duplication has read them)
  unsigned* skeys = nullptr;
  rc = radix_sort_pairs(vkeys, vvals, &w.counters[0], nv, passes, np, w.sort, st, false, false,
                        &skeys, &vvals);
  if (rc) return rc;

  // 3. instance offsets in sorted order; total -> n_instances
  // (and the record owning the first instance of every duplication chunk)
  long long* offs = w.offs;
  int* chunk_first = w.chunk_first;
  const long long n_chunk_max = (cap + DUP_CHUNK - 1) / DUP_CHUNK;
  rc = scan_exclusive([=] __device__(long long j) -> long long { return tiles[vvals[j]]; },
                      [=] __device__(long long j, long long pre) {
                        offs[j] = pre;
                        const long long end = pre + tiles[vvals[j]];
                        for (long long c = (pre + DUP_CHUNK - 1) / DUP_CHUNK;
                             c < n_chunk_max && c * DUP_CHUNK < end; ++c)
                          chunk_first[c] = (int)j;
                      },
                      nv, &w.counters[0], (long long*)bins->n_instances, w.scan2, st, d_status,
                      /*cleared=*/true);
  if (rc) return rc;
  clamp_count_kernel<<<1, 1, 0, st>>>((const long long*)bins->n_instances, cap,
                                      scan_error_flag(w.scan2, nv), &w.counters[1]);

  // 4. duplicate into tiles, 5. stable sort by tile. The instance key is the
  // view-local tile with the view above the sorted bits: the tile sort takes
  // only the passes the largest view needs, every (view, tile) list is still one
  // run in (depth, id) order (the records come view-major and every pass is
  // stable), and the runs are ordered by local tile, then view. Instances whose
  // ellipse misses their tile get the key TILE_NONE, which the first pass drops.
  if (cap > 0) {
    // the tile passes split the tile bits evenly (13 bits: 7 + 6), fewer bits per
    // pass than 8 where that takes no extra pass
    DigitOp tp[4];
    const int ntp = (tile_bits + 7) / 8 > 0 ? (tile_bits + 7) / 8 : 1;
    for (int q = 0, s = 0; q < ntp; ++q) {
      const int b = (tile_bits - s + (ntp - q) - 1) / (ntp - q);  // ceil of the rest
      tp[q] = DigitOp{s, 0u, b < 1 ? 1 : b};
      s += b;
    }
    duplicate_kernel<<<(unsigned)std::min<long long>((cap + DUP_CHUNK - 1) / DUP_CHUNK, 148 * 8),
                       DUP_THREADS, 0, st>>>(
        vvals, offs, chunk_first, &w.counters[0], &w.counters[1], cap,
        reinterpret_cast<const int4*>(pr->rect), xyod,
        reinterpret_cast<const float4*>(pr->conic), prm->alpha_min, n, cs, view_shift, w.tkeys,
        bins->inst_gauss, aligned(bins->inst_gauss, 16), tp[0].mask(), w.sort.hist,
        w.sort.tiles_max);
    ADP_LAUNCH_CHECK();
    // the first pass's tile histograms come from the duplication, which leaves out the
    // instances whose ellipse misses their tile; the first pass drops them and the
    // count becomes the kept instances
    static_assert(TILE_NONE == RS_DROP_KEY, "the filtered key is the sort's drop key");
    rc = radix_sort_pairs(w.tkeys, reinterpret_cast<unsigned*>(bins->inst_gauss),
                          &w.counters[1], cap, tp, ntp, w.sort, st, /*first_hist_done=*/true,
                          /*drop_none=*/true);
    if (rc) return rc;
    // 6. per-tile ranges
    tile_ranges_kernel<<<grid_for(cap, 256, 148 * 16), 256, 0, st>>>(
        w.tkeys, &w.counters[1], cs, view_shift, reinterpret_cast<int2*>(bins->tile_range));
    ADP_LAUNCH_CHECK();
  }
  return ADP_OK;
}

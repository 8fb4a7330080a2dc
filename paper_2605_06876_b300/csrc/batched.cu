// The batched training step of many views (Sec. 4.1: the sampled views of a
// densification step; the loss and its gradient are the baselines', Sec. 5.1):
// projection and binning of every view in one launch each, then ONE persistent
// kernel over a work queue of (view, tile) items that, per tile, composites the
// forward (Eq. 1, the dominant map of Eq. 5), writes the raw L1 error of Eq. 6
// with the view's min/max reduction as its epilogue, and walks the same list back
// to front for the L1 backward with the final transmittance, the last blended
// positions and dL/dpixel still in registers; then the normalisation of Eq. 6
// with the per-Gaussian error statistics, and the per-Gaussian chain rule summed
// over views. Blocks take items from a counter, so views of uneven size share one
// launch without a tail per view.
#include <algorithm>

#include "phases.cuh"
#include "tile_composite.cuh"

#ifndef ADP_FUSED_PX
#define ADP_FUSED_PX 4
#endif
#ifndef ADP_FUSED_MINB  // resident blocks per SM the register budget is sized for
#define ADP_FUSED_MINB 12
#endif

namespace adp {

struct FusedArgs {
  const float4* xyod;
  const float4* conic;
  const float4* rgb;
  const int* inst;
  const int2* ranges;
  long long n;
  const float* target;
  float bg[3];
  CompositeConsts kc;
  float* out_rgb;
  float* out_T;
  int* out_n;
  int* out_last;
  int* out_dom;
  float* raw;         // [P] raw L1 error (normalised in place later)
  unsigned* minmax;   // [V][2] float bits of the raw L1 min and max
  float4* g2d;        // [V*n][3] pixel moments of the backward, zeroed
  int* item_ctr;      // next work item (the tile index), zeroed
};

constexpr int FUSED_PX = ADP_FUSED_PX;

template <int PX, int STAGE>
__global__ void __launch_bounds__(TileLanes<PX>::THREADS, ADP_FUSED_MINB)
    fused_tile_kernel(FusedArgs a, CamSet cs) {
  constexpr int NT = TileLanes<PX>::THREADS;
  constexpr int NP = PX / 2;
  __shared__ float4 s_g0[STAGE];
  __shared__ float4 s_g1[STAGE];
  __shared__ float4 s_g2[STAGE];
  __shared__ float2 s_y[STAGE];
  __shared__ int s_item, s_maxlast;
  __shared__ unsigned s_lo[NT / 32], s_hi[NT / 32];
  const StageBuf sb{s_g0, s_g1, s_g2, s_y};
  const int n_items = cs.tile_base[cs.n_views];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.item_ctr, 1);
    __syncthreads();
    const int tile = s_item;
    __syncthreads();  // every thread is past the previous item and has read s_item
    if (tile >= n_items) break;
    const TileGeom<PX> t = tile_geom<PX>(cs, a.ranges, a.n, tile);
    FwdOut<PX> o;
    fwd_tile<PX, STAGE>(a.xyod, a.conic, a.rgb, a.inst, t, a.kc, sb, o);
    // epilogue: the image, the raw L1 error and dL/dpixel of the L1 loss
    const float sc = 1.f / (3.f * (float)t.W * (float)t.H);
    BwdIn<PX> in;
    unsigned lo = 0x7f800000u, hi = 0u;  // +inf, 0 as float bits (raw >= 0)
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const float t2[2] = {o.T[j].x, o.T[j].y}, r2[2] = {o.c0[j].x, o.c0[j].y};
      const float g2[2] = {o.c1[j].x, o.c1[j].y}, b2[2] = {o.c2[j].x, o.c2[j].y};
      float gg[2][3];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int h = 2 * j + e;
        in.last[h] = o.last[h];
        gg[e][0] = gg[e][1] = gg[e][2] = 0.f;
        if (!pixel_in(t, h)) continue;
        const long long p = t.pix_base + (long long)t.py * t.W + t.px0 + h;
        const float im[3] = {__fmaf_rn(t2[e], a.bg[0], r2[e]), __fmaf_rn(t2[e], a.bg[1], g2[e]),
                             __fmaf_rn(t2[e], a.bg[2], b2[e])};
        a.out_rgb[3 * p + 0] = im[0];
        a.out_rgb[3 * p + 1] = im[1];
        a.out_rgb[3 * p + 2] = im[2];
        a.out_T[p] = t2[e];
        a.out_n[p] = o.ncon[h];
        a.out_last[p] = o.last[h];
        a.out_dom[p] = o.dom[h];
        float d[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          d[ch] = __fsub_rn(im[ch], a.target[3 * p + ch]);
          gg[e][ch] = d[ch] > 0.f ? sc : (d[ch] < 0.f ? -sc : 0.f);
        }
        const float r = __fadd_rn(__fadd_rn(fabsf(d[0]), fabsf(d[1])), fabsf(d[2]));
        a.raw[p] = r;
        lo = min(lo, __float_as_uint(r));
        hi = max(hi, __float_as_uint(r));
      }
      in.T[j] = o.T[j];
      in.G0[j] = make_float2(gg[0][0], gg[1][0]);
      in.G1[j] = make_float2(gg[0][1], gg[1][1]);
      in.G2[j] = make_float2(gg[0][2], gg[1][2]);
    }
    // the view's min and max: a warp reduction, then one pair of atomics per item
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if (lane == 0) {
      s_lo[warp] = lo;
      s_hi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < NT / 32; ++w) {
        lo = min(lo, s_lo[w]);
        hi = max(hi, s_hi[w]);
      }
      if (lo <= hi) {
        atomicMin(&a.minmax[2 * t.v], lo);
        atomicMax(&a.minmax[2 * t.v + 1], hi);
      }
    }
    bwd_tile<PX, STAGE>(a.xyod, a.conic, a.rgb, a.inst, t, a.kc, a.bg, sb, &s_maxlast, in, a.g2d);
  }
}

template <int STAGE>
static int fused_grid(int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  ADP_CUDA(cudaGetDevice(&dev));
  ADP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  ADP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, fused_tile_kernel<FUSED_PX, STAGE>, TileLanes<FUSED_PX>::THREADS, 0));
  ADP_CHECK_ARG(per_sm >= 1, "the fused kernel cannot be resident on this device");
  *grid = sms * per_sm;
  return ADP_OK;
}

struct BatchedWs {
  void* bins_ws;
  size_t bins_bytes;
  float4* g2d;
  int* list;
  unsigned long long* n_list;
  int* item_ctr;
};

static size_t batched_ws_bytes(long long n, int n_views, long long capacity) {
  return adp_bin_sort_workspace_size(n, n_views, capacity) +
         carve_bytes<float4>(3 * (size_t)n * n_views) + carve_bytes<int>(n) +
         carve_bytes<unsigned long long>(1) + carve_bytes<int>(1);
}

}  // namespace adp

using namespace adp;

extern "C" ADP_API size_t adp_train_step_batched_workspace_size(int64_t n, int32_t n_views,
                                                                const adp_camera* cams,
                                                                const adp_params* prm,
                                                                int64_t capacity) {
  if (n < 0 || n_views < 1 || capacity < 0) return 0;
  CamSet cs;
  if (make_camset(cams, n_views, prm, &cs)) return 0;
  return batched_ws_bytes(n, n_views, capacity);
}

extern "C" ADP_API int adp_train_step_batched(
    const adp_gaussians* g, const adp_camera* cams, int32_t n_views, const float* target,
    const float* bg, const adp_params* prm, adp_projected* pr, adp_bins* bins, adp_image* img,
    adp_error_maps* maps, int32_t* count, double* mass, adp_gaussians* grad, float* grad2d_accum,
    int32_t* grad2d_visits, void* ws, size_t ws_bytes, int32_t* d_status, adp_stream_t stream) {
  ADP_CHECK_ARG(g && pr && bins && img && maps && grad && target, "NULL argument");
  ADP_CHECK_ARG(img->rgb && img->T_final && img->n_contrib && img->last && img->dominant,
                "NULL image array");
  ADP_CHECK_ARG(maps->E && maps->mask && maps->minmax, "NULL error map array");
  ADP_CHECK_ARG(!grad2d_accum == !grad2d_visits, "give both or neither densification accumulators");
  ADP_CHECK_ARG(grad->n == g->n && grad->sh_degree == g->sh_degree, "grad shape mismatch");
  ADP_CHECK_ARG(g->n == 0 || (count && mass), "NULL count/mass");
  CamSet cs;
  int rc = make_camset(cams, n_views, prm, &cs);
  if (rc) return rc;
  ADP_CHECK_ARG(g->n >= 0 && (long long)g->n * n_views < (1LL << 31), "n_views * n exceeds 2^31");
  ADP_CHECK_ARG(prm->n_levels >= 1 && prm->n_levels <= 15, "n_levels must be 1..15");
  ADP_CHECK_ARG(prm->alpha_min >= 1e-18f && prm->t_min >= 1e-18f && prm->alpha_max < 1.f,
                "alpha_min and t_min must be >= 1e-18 and alpha_max < 1");
  ADP_CHECK_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
  const long long n = g->n;
  const int n_items = cs.tile_base[n_views];
  const size_t need = batched_ws_bytes(n, n_views, bins->capacity);
  ADP_CHECK_ARG(ws_bytes >= need, "workspace %zu bytes, need %zu", ws_bytes, need);
  cudaStream_t st = (cudaStream_t)stream;
  BatchedWs w;
  {
    Carver c(ws, ws_bytes);
    w.bins_bytes = adp_bin_sort_workspace_size(n, n_views, bins->capacity);
    w.bins_ws = c.take<char>(w.bins_bytes);
    w.g2d = c.take<float4>(3 * (size_t)n * n_views);
    w.list = c.take<int>(n);
    w.n_list = c.take<unsigned long long>(1);
    w.item_ctr = c.take<int>(1);
    ADP_CHECK_ARG(c.ok, "internal: workspace carve failed");
  }
  // 1-2. projection (zeroing the backward's moment rows of the visible records) and
  // binning of every view
  rc = project_launch(g, cams, n_views, prm, pr, w.g2d, st);
  if (rc) return rc;
  rc = adp_bin_sort(n, pr, cams, n_views, prm, bins, w.bins_ws, w.bins_bytes, d_status, stream);
  if (rc) return rc;
  // (with no Gaussian every tile list is empty: the image is the background, and the
  // error maps and the statistics follow from it)
  // 3. the fused forward + error epilogue + backward over the (view, tile) queue
  // the queue counters and the error statistics' presets, in one launch
  FillSet fill;
  fill.add(w.n_list, sizeof(unsigned long long));
  fill.add(w.item_ctr, sizeof(int));
  error_init_fill(fill, maps, n_views, count, mass, n);
  rc = launch_fill(fill, st);
  if (rc) return rc;
  FusedArgs a;
  a.xyod = reinterpret_cast<const float4*>(pr->xy_opacity_depth);
  a.conic = reinterpret_cast<const float4*>(pr->conic);
  a.rgb = reinterpret_cast<const float4*>(pr->rgb);
  a.inst = bins->inst_gauss;
  a.ranges = reinterpret_cast<const int2*>(bins->tile_range);
  a.n = n;
  a.target = target;
  for (int c = 0; c < 3; ++c) a.bg[c] = bg ? bg[c] : 0.f;
  a.kc = CompositeConsts{prm->alpha_min, prm->alpha_max, prm->t_min, log2f(prm->alpha_min)};
  a.out_rgb = img->rgb;
  a.out_T = img->T_final;
  a.out_n = img->n_contrib;
  a.out_last = img->last;
  a.out_dom = img->dominant;
  a.raw = maps->E;
  a.minmax = reinterpret_cast<unsigned*>(maps->minmax);
  a.g2d = w.g2d;
  a.item_ctr = w.item_ctr;
  const dim3 block(TileLanes<FUSED_PX>::THREADS);
  int grid = 0;
  switch (stage_size(prm)) {
    case 64:
      rc = fused_grid<64>(&grid);
      if (rc) return rc;
      fused_tile_kernel<FUSED_PX, 64><<<std::min(grid, n_items), block, 0, st>>>(a, cs);
      break;
    case 128:
      rc = fused_grid<128>(&grid);
      if (rc) return rc;
      fused_tile_kernel<FUSED_PX, 128><<<std::min(grid, n_items), block, 0, st>>>(a, cs);
      break;
    default:
      rc = fused_grid<256>(&grid);
      if (rc) return rc;
      fused_tile_kernel<FUSED_PX, 256><<<std::min(grid, n_items), block, 0, st>>>(a, cs);
      break;
  }
  ADP_LAUNCH_CHECK();
  // 4. E, M, B and the per-Gaussian count and mass (Eq. 6, Sec. 5.1) on the
  // auxiliary stream, beside 5. the per-Gaussian chain rule summed over views: the
  // first is bound by its divisions and atomics, the second by gather latency
  AuxStream* aux = nullptr;
  rc = aux_stream(&aux);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lock(aux_mutex());
    ADP_CUDA(cudaEventRecord(aux->forked, st));
    ADP_CUDA(cudaStreamWaitEvent(aux->stream, aux->forked, 0));
  }
  const int rc_err = error_norm_phase(maps, img->dominant, n, cs, prm, count, mass, aux->stream);
  {
    std::lock_guard<std::mutex> lock(aux_mutex());
    ADP_CUDA(cudaEventRecord(aux->joined, aux->stream));
  }
  const int rc_bwd = backward_gauss_phase(g, pr, cs, prm, grad, grad2d_accum, grad2d_visits,
                                          w.g2d, w.list, w.n_list, st);
  {  // joined even after an error, so a capture stays valid
    std::lock_guard<std::mutex> lock(aux_mutex());
    ADP_CUDA(cudaStreamWaitEvent(st, aux->joined, 0));
  }
  return rc_err ? rc_err : rc_bwd;
}

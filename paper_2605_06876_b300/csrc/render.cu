// Front-to-back alpha compositing (Eq. 1) with the dominant Gaussian map (Eq. 5).
// One CTA per tile (256 pixels, PX horizontally adjacent ones per thread); the
// tile's depth-sorted list is staged through shared memory 256 Gaussians at a
// time in a precomputed form (alpha in log2 units, the rows each ellipse
// reaches), a warp skips Gaussians that reach none of its rows, the per-pixel
// update is branch-free (a pixel that has stopped, or that a Gaussian misses,
// takes a zero weight), a warp leaves the batch once all its pixels have
// stopped and a block-wide vote ends the tile.
#include "gauss_math.cuh"

#ifndef ADP_RENDER_PX
#define ADP_RENDER_PX 4
#endif

namespace adp {

struct RenderArgs {
  const float4* xyod;
  const float4* conic;
  const float4* rgb;
  const int* inst;
  const int2* ranges;
  long long n;
  float bg[3];
  float alpha_min, alpha_max, t_min, log2_alpha_min;
  float* out_rgb;
  float* out_T;
  int* out_n;
  int* out_last;
  int* out_dom;
};

constexpr int RENDER_PX = ADP_RENDER_PX;
constexpr int STAGE = 256;  // Gaussians staged per batch

template <int PX>
__global__ void __launch_bounds__(TileLanes<PX>::THREADS) render_kernel(RenderArgs a, CamSet cs) {
  constexpr int NT = TileLanes<PX>::THREADS;
  __shared__ float4 s_g0[STAGE];
  __shared__ float4 s_g1[STAGE];
  __shared__ float4 s_g2[STAGE];
  __shared__ float2 s_y[STAGE];
  const int tile = blockIdx.x;
  const int v = view_of_tile(cs, tile);
  const int lt = tile - cs.tile_base[v];
  const int txs = cs.tiles_x[v];
  const int W = cs.cam[v].width, H = cs.cam[v].height;
  const int2 range = a.ranges[tile];
  const int count = range.y - range.x;
  const long long rec_base = (long long)v * a.n;
  const int tx0 = (lt % txs) * cs.tile_w, ty0 = (lt / txs) * cs.tile_h;
  const int warp = threadIdx.x >> 5;
  // the rows this warp's pixels cover
  const float wy0 = (float)(ty0 + (TileLanes<PX>::WARP_PIXELS * warp) / cs.tile_w);
  const float wy1 =
      (float)(ty0 + (TileLanes<PX>::WARP_PIXELS * (warp + 1) - 1) / cs.tile_w);
  const int li0 = PX * (int)threadIdx.x;
  const int px0 = tx0 + li0 % cs.tile_w, py = ty0 + li0 / cs.tile_w;
  const float fy = (float)py;
  const float amax = a.alpha_max, tmin = a.t_min, l2amin = a.log2_alpha_min;

  float T[PX], c0[PX], c1[PX], c2[PX], best[PX];
  int dom[PX], ncon[PX], last[PX];
  bool done[PX];
  bool all_done = true;
#pragma unroll
  for (int h = 0; h < PX; ++h) {
    T[h] = 1.f;
    c0[h] = c1[h] = c2[h] = 0.f;
    best[h] = 0.f;  // every blended weight T alpha is > 0
    dom[h] = -1;
    ncon[h] = 0;
    last[h] = 0;
    done[h] = !(px0 + h < W && py < H);
    all_done = all_done && done[h];
  }
  for (int b0 = 0; b0 < count; b0 += STAGE) {
    if (__syncthreads_count(all_done) == NT) break;
    for (int j = (int)threadIdx.x; j < STAGE && b0 + j < count; j += NT) {
      int id = a.inst[range.x + b0 + j];
      long long r = rec_base + id;
      Staged g = stage_gaussian(a.xyod[r], a.conic[r], a.rgb[r], id, a.alpha_min);
      s_g0[j] = g.g0;
      s_g1[j] = g.g1;
      s_g2[j] = g.g2;
      s_y[j] = g.y;
    }
    __syncthreads();
    if (__all_sync(0xffffffffu, all_done)) continue;
    const int cnt = min(STAGE, count - b0);
    for (int k = 0; k < cnt; ++k) {
      const float2 yr = s_y[k];
      if (yr.y < wy0 || yr.x > wy1) continue;  // warp-uniform: no row of this warp reached
      const float4 g0 = s_g0[k], g1 = s_g1[k], g2 = s_g2[k];
      const RowQ rq = row_q(g0, g1, fy);
      const int id = __float_as_int(g2.y);
      all_done = true;
#pragma unroll
      for (int h = 0; h < PX; ++h) {
        float dx;
        const float q = pix_q(g0, rq, (float)(px0 + h), &dx);
        const bool live = !done[h] && q >= l2amin;
        const float al = fminf(amax, ex2_approx(q));
        const float test = T[h] * (1.f - al);
        const bool stop = live && test < tmin;  // stop before blending (T would drop below t_min)
        const bool blend = live && !stop;
        done[h] = done[h] || stop;
        const float w = blend ? T[h] * al : 0.f;
        c0[h] = fmaf(w, g1.z, c0[h]);
        c1[h] = fmaf(w, g1.w, c1[h]);
        c2[h] = fmaf(w, g2.x, c2[h]);
        if (w > best[h]) {  // strict: the earliest of equal weights wins
          best[h] = w;
          dom[h] = id;
        }
        T[h] = blend ? test : T[h];
        ncon[h] += blend ? 1 : 0;
        last[h] = blend ? b0 + k + 1 : last[h];
        all_done = all_done && done[h];
      }
      if (__all_sync(0xffffffffu, all_done)) break;
    }
  }
#pragma unroll
  for (int h = 0; h < PX; ++h) {
    if (!(px0 + h < W && py < H)) continue;
    long long p = cs.pix_base[v] + (long long)py * W + px0 + h;
    a.out_rgb[3 * p + 0] = c0[h] + T[h] * a.bg[0];
    a.out_rgb[3 * p + 1] = c1[h] + T[h] * a.bg[1];
    a.out_rgb[3 * p + 2] = c2[h] + T[h] * a.bg[2];
    a.out_T[p] = T[h];
    a.out_n[p] = ncon[h];
    a.out_last[p] = last[h];
    a.out_dom[p] = dom[h];
  }
}

}  // namespace adp

using namespace adp;

extern "C" ADP_API int adp_render(int64_t n, const adp_projected* pr, const adp_bins* bins,
                                  const adp_camera* cams, int32_t n_views, const float* bg,
                                  const adp_params* prm, adp_image* out, adp_stream_t stream) {
  ADP_CHECK_ARG(pr && bins && out, "NULL argument");
  CamSet cs;
  int rc = make_camset(cams, n_views, prm, &cs);
  if (rc) return rc;
  ADP_CHECK_ARG(n >= 0 && (long long)n * n_views < (1LL << 31), "n_views * n exceeds 2^31");
  ADP_CHECK_ARG(out->rgb && out->T_final && out->n_contrib && out->last && out->dominant,
                "NULL image array");
  ADP_CHECK_ARG(bins->tile_range, "NULL tile ranges");
  RenderArgs a;
  a.xyod = reinterpret_cast<const float4*>(pr->xy_opacity_depth);
  a.conic = reinterpret_cast<const float4*>(pr->conic);
  a.rgb = reinterpret_cast<const float4*>(pr->rgb);
  a.inst = bins->inst_gauss;
  a.ranges = reinterpret_cast<const int2*>(bins->tile_range);
  a.n = n;
  for (int c = 0; c < 3; ++c) a.bg[c] = bg ? bg[c] : 0.f;
  a.alpha_min = prm->alpha_min;
  a.alpha_max = prm->alpha_max;
  a.t_min = prm->t_min;
  a.log2_alpha_min = log2f(prm->alpha_min);
  a.out_rgb = out->rgb;
  a.out_T = out->T_final;
  a.out_n = out->n_contrib;
  a.out_last = out->last;
  a.out_dom = out->dominant;
  int n_tiles = cs.tile_base[n_views];
  render_kernel<RENDER_PX>
      <<<n_tiles, TileLanes<RENDER_PX>::THREADS, 0, (cudaStream_t)stream>>>(a, cs);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

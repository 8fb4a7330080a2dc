// Front-to-back alpha compositing (Eq. 1) with the dominant Gaussian map (Eq. 5):
// one CTA per tile runs the forward walk of tile_composite.cuh (PX horizontally
// adjacent pixels per thread, the tile's depth-sorted list staged through shared
// memory a batch of Gaussians at a time) and writes the per-pixel outputs.
#include "tile_composite.cuh"

#ifndef ADP_RENDER_PX
#define ADP_RENDER_PX 4
#endif
#ifndef ADP_RENDER_MINB  // resident blocks per SM the register budget is sized for
#define ADP_RENDER_MINB 1
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
  CompositeConsts kc;
  float* out_rgb;
  float* out_T;
  int* out_n;
  int* out_last;
  int* out_dom;
};

constexpr int RENDER_PX = ADP_RENDER_PX;

// One CTA per tile: the forward walk of fwd_tile, then the per-pixel outputs.
template <int PX, int STAGE>
__global__ void __launch_bounds__(TileLanes<PX>::THREADS, ADP_RENDER_MINB)
    render_kernel(RenderArgs a, CamSet cs) {
  constexpr int NP = PX / 2;
  __shared__ float4 s_g0[STAGE];
  __shared__ float4 s_g1[STAGE];
  __shared__ float4 s_g2[STAGE];
  __shared__ float2 s_y[STAGE];
  const StageBuf sb{s_g0, s_g1, s_g2, s_y};
  const TileGeom<PX> t = tile_geom<PX>(cs, a.ranges, a.n, blockIdx.x);
  FwdOut<PX> o;
  fwd_tile<PX, STAGE>(a.xyod, a.conic, a.rgb, a.inst, t, a.kc, sb, o);
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const float t2[2] = {o.T[j].x, o.T[j].y}, r2[2] = {o.c0[j].x, o.c0[j].y};
    const float g2[2] = {o.c1[j].x, o.c1[j].y}, b2[2] = {o.c2[j].x, o.c2[j].y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int h = 2 * j + e;
      if (!pixel_in(t, h)) continue;
      const long long p = t.pix_base + (long long)t.py * t.W + t.px0 + h;
      a.out_rgb[3 * p + 0] = __fmaf_rn(t2[e], a.bg[0], r2[e]);
      a.out_rgb[3 * p + 1] = __fmaf_rn(t2[e], a.bg[1], g2[e]);
      a.out_rgb[3 * p + 2] = __fmaf_rn(t2[e], a.bg[2], b2[e]);
      a.out_T[p] = t2[e];
      a.out_n[p] = o.ncon[h];
      a.out_last[p] = o.last[h];
      a.out_dom[p] = o.dom[h];
    }
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
  // the compositing loop detects a blend and a strictly larger weight by scaling
  // them by 2^126 (weights are at least t_min * alpha_min)
  ADP_CHECK_ARG(prm->alpha_min >= 1e-18f && prm->t_min >= 1e-18f && prm->alpha_max < 1.f,
                "alpha_min and t_min must be >= 1e-18 and alpha_max < 1");
  RenderArgs a;
  a.xyod = reinterpret_cast<const float4*>(pr->xy_opacity_depth);
  a.conic = reinterpret_cast<const float4*>(pr->conic);
  a.rgb = reinterpret_cast<const float4*>(pr->rgb);
  a.inst = bins->inst_gauss;
  a.ranges = reinterpret_cast<const int2*>(bins->tile_range);
  a.n = n;
  for (int c = 0; c < 3; ++c) a.bg[c] = bg ? bg[c] : 0.f;
  a.kc = CompositeConsts{prm->alpha_min, prm->alpha_max, prm->t_min, log2f(prm->alpha_min)};
  a.out_rgb = out->rgb;
  a.out_T = out->T_final;
  a.out_n = out->n_contrib;
  a.out_last = out->last;
  a.out_dom = out->dominant;
  int n_tiles = cs.tile_base[n_views];
  const dim3 grid(n_tiles), block(TileLanes<RENDER_PX>::THREADS);
  cudaStream_t st = (cudaStream_t)stream;
  switch (stage_size(prm)) {
    case 64: render_kernel<RENDER_PX, 64><<<grid, block, 0, st>>>(a, cs); break;
    case 128: render_kernel<RENDER_PX, 128><<<grid, block, 0, st>>>(a, cs); break;
    default: render_kernel<RENDER_PX, 256><<<grid, block, 0, st>>>(a, cs); break;
  }
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

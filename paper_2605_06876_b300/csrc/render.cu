// Front-to-back alpha compositing (Eq. 1) with the dominant Gaussian map (Eq. 5).
// One CTA per tile (256 pixels, two horizontally adjacent ones per thread); the
// tile's depth-sorted list is staged through shared memory 256 Gaussians at a
// time in a precomputed form (alpha in log2 units, the rows each ellipse
// reaches), a warp skips Gaussians that reach none of its rows, and a block-wide
// vote ends the tile once every pixel has stopped.
#include "gauss_math.cuh"

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

constexpr int RENDER_THREADS = 128;  // two horizontally adjacent pixels per thread
constexpr int STAGE = 256;           // Gaussians staged per batch

struct FwdPix {
  float T, c0, c1, c2, best, fx, fy;
  int dom, ncon, last;
  bool done;
};

__device__ __forceinline__ void fwd_step(FwdPix& s, int pos, const Staged& g, float amax,
                                         float tmin, float l2amin) {
  if (s.done) return;
  float dx, dy;
  const float q = log2_alpha(g.g0, g.g1, s.fx, s.fy, &dx, &dy);
  if (q < l2amin) return;
  const float al = fminf(amax, exp2f(q));
  const float test = s.T * (1.f - al);
  if (test < tmin) {
    s.done = true;
    return;
  }
  const float w = s.T * al;
  s.c0 += w * g.g1.z;
  s.c1 += w * g.g1.w;
  s.c2 += w * g.g2.x;
  if (w > s.best) {
    s.best = w;
    s.dom = __float_as_int(g.g2.y);
  }
  s.T = test;
  ++s.ncon;
  s.last = pos + 1;
}

__global__ void __launch_bounds__(RENDER_THREADS) render_kernel(RenderArgs a, CamSet cs) {
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
  // the rows this warp's 64 pixels cover
  const float wy0 = (float)(ty0 + (64 * warp) / cs.tile_w);
  const float wy1 = (float)(ty0 + (64 * warp + 63) / cs.tile_w);

  FwdPix ps[2];
  bool inside[2];
  int pxs[2], pys[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int li = 2 * (int)threadIdx.x + h;
    pxs[h] = tx0 + li % cs.tile_w;
    pys[h] = ty0 + li / cs.tile_w;
    inside[h] = pxs[h] < W && pys[h] < H;
    FwdPix& s = ps[h];
    s.T = 1.f;
    s.c0 = s.c1 = s.c2 = 0.f;
    s.best = -1.f;
    s.fx = (float)pxs[h];
    s.fy = (float)pys[h];
    s.dom = -1;
    s.ncon = 0;
    s.last = 0;
    s.done = !inside[h];
  }
  for (int b0 = 0; b0 < count; b0 += STAGE) {
    if (__syncthreads_count(ps[0].done && ps[1].done) == RENDER_THREADS) break;
    for (int j = (int)threadIdx.x; j < STAGE && b0 + j < count; j += RENDER_THREADS) {
      int id = a.inst[range.x + b0 + j];
      long long r = rec_base + id;
      Staged g = stage_gaussian(a.xyod[r], a.conic[r], a.rgb[r], id, a.alpha_min);
      s_g0[j] = g.g0;
      s_g1[j] = g.g1;
      s_g2[j] = g.g2;
      s_y[j] = g.y;
    }
    __syncthreads();
    if (!(ps[0].done && ps[1].done)) {
      const int cnt = min(STAGE, count - b0);
      for (int k = 0; k < cnt; ++k) {
        const float2 yr = s_y[k];
        if (yr.y < wy0 || yr.x > wy1) continue;  // warp-uniform: no row of this warp reached
        Staged g;
        g.g0 = s_g0[k];
        g.g1 = s_g1[k];
        g.g2 = s_g2[k];
        fwd_step(ps[0], b0 + k, g, a.alpha_max, a.t_min, a.log2_alpha_min);
        fwd_step(ps[1], b0 + k, g, a.alpha_max, a.t_min, a.log2_alpha_min);
        if (ps[0].done && ps[1].done) break;
      }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (!inside[h]) continue;
    const FwdPix& s = ps[h];
    long long p = cs.pix_base[v] + (long long)pys[h] * W + pxs[h];
    a.out_rgb[3 * p + 0] = s.c0 + s.T * a.bg[0];
    a.out_rgb[3 * p + 1] = s.c1 + s.T * a.bg[1];
    a.out_rgb[3 * p + 2] = s.c2 + s.T * a.bg[2];
    a.out_T[p] = s.T;
    a.out_n[p] = s.ncon;
    a.out_last[p] = s.last;
    a.out_dom[p] = s.dom;
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
  render_kernel<<<n_tiles, RENDER_THREADS, 0, (cudaStream_t)stream>>>(a, cs);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

// Front-to-back alpha compositing (Eq. 1) with the dominant Gaussian map (Eq. 5).
// One CTA per tile (256 pixels, PX horizontally adjacent ones per thread); the
// tile's depth-sorted list is staged through shared memory 256 Gaussians at a
// time in a precomputed form (alpha in log2 units, the rows each ellipse
// reaches), a warp skips Gaussians that reach none of its rows, the per-pixel
// update is branch-free (a pixel that has stopped, or that a Gaussian misses,
// takes a zero weight), a warp leaves the batch once all its pixels have
// stopped (checked every fourth Gaussian) and a block-wide vote ends the tile.
#include "gauss_math.cuh"

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
  float alpha_min, alpha_max, t_min, log2_alpha_min;
  float* out_rgb;
  float* out_T;
  int* out_n;
  int* out_last;
  int* out_dom;
};

constexpr int RENDER_PX = ADP_RENDER_PX;
#ifndef ADP_RENDER_STAGE
#define ADP_RENDER_STAGE 256
#endif
constexpr int STAGE = ADP_RENDER_STAGE;  // Gaussians staged per batch (at most 256)

// Scale that saturates any positive alpha or weight difference the rules allow
// to exactly 1 (__saturatef(x * kSat) is 0 for x <= 0 and 1 for x >= 2^-126).
constexpr float kSat = 8.507059173023462e37f;  // 2^126
// Minus the x coordinate given to a pixel that has stopped: its exponent q is then
// -inf or hugely negative, so the alpha test fails without a separate flag.
constexpr float kGone = -1e30f;

// The per-pixel update runs on horizontal pixel pairs with the packed two-lane
// FP32 instructions of sm_100+ (each lane rounds like the scalar instruction), and
// the bookkeeping that would otherwise take compares and selects on the integer
// pipe -- contributor count, last blended position, position of the dominant
// weight -- is kept as exact small floats within the staged batch (positions
// below 256) through saturating multiplies on the FMA pipe, and folded into the
// integer outputs when the batch ends.
template <int PX>
__global__ void __launch_bounds__(TileLanes<PX>::THREADS, ADP_RENDER_MINB)
    render_kernel(RenderArgs a, CamSet cs) {
  static_assert(PX % 2 == 0, "pixels are processed in pairs");
  constexpr int NT = TileLanes<PX>::THREADS;
  constexpr int NP = PX / 2;
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
  const float2 one2 = make_float2(1.f, 1.f), neg2 = make_float2(-1.f, -1.f);

  float2 T[NP], c0[NP], c1[NP], c2[NP], best[NP], nfx[NP];
  float2 ncf[NP], lastf[NP], domf[NP];  // per batch: blends, last blended k + 1, dominant k
  int dom[PX], ncon[PX], last[PX];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    T[j] = one2;
    c0[j] = c1[j] = c2[j] = make_float2(0.f, 0.f);
    best[j] = make_float2(0.f, 0.f);  // every blended weight T alpha is > 0
    ncf[j] = lastf[j] = make_float2(0.f, 0.f);
    domf[j] = neg2;
    float n2[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int h = 2 * j + e;
      dom[h] = -1;
      ncon[h] = 0;
      last[h] = 0;
      n2[e] = (px0 + h < W && py < H) ? -(float)(px0 + h) : kGone;
    }
    nfx[j] = make_float2(n2[0], n2[1]);
  }
  auto thread_done = [&]() {
    bool d = true;
#pragma unroll
    for (int j = 0; j < NP; ++j) d = d && nfx[j].x == kGone && nfx[j].y == kGone;
    return d;
  };
  for (int b0 = 0; b0 < count; b0 += STAGE) {
    if (__syncthreads_count(thread_done()) == NT) break;
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
    if (__all_sync(0xffffffffu, thread_done())) continue;
    const int cnt = min(STAGE, count - b0);
    float kfl = 0.f;  // k as a float, advanced with k (no conversion per Gaussian)
    for (int k = 0; k < cnt; ++k, kfl += 1.f) {
      if ((k & 3) == 0 && __all_sync(0xffffffffu, thread_done())) break;
      const float2 yr = s_y[k];
      if (yr.y < wy0 || yr.x > wy1) continue;  // warp-uniform: no row of this warp reached
      const float4 g0 = s_g0[k], g1 = s_g1[k], g2 = s_g2[k];
      const RowQ rq = row_q(g0, g1, fy);
      const float2 mx = make_float2(g0.x, g0.x), qa = make_float2(g0.z, g0.z);
      const float2 qb = make_float2(rq.bdy, rq.bdy), qe = make_float2(rq.e, rq.e);
      const float2 cr = make_float2(g1.z, g1.z), cg = make_float2(g1.w, g1.w);
      const float2 cb = make_float2(g2.x, g2.x);
      const float2 kf = make_float2(kfl, kfl), k1 = make_float2(kfl + 1.f, kfl + 1.f);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        // q = dx (a dx + b dy) + e, the same operations as pix_q
        const float2 dx = __fadd2_rn(mx, nfx[j]);
        const float2 q = __ffma2_rn(dx, __ffma2_rn(qa, dx, qb), qe);
        float2 al = make_float2(q.x >= l2amin ? fminf(amax, ex2_approx(q.x)) : 0.f,
                                q.y >= l2amin ? fminf(amax, ex2_approx(q.y)) : 0.f);
        // stop before blending when T (1 - alpha) would fall below t_min
        const float2 test = __fmul2_rn(T[j], __ffma2_rn(al, neg2, one2));
        if (test.x < tmin) {
          al.x = 0.f;
          nfx[j].x = kGone;
        }
        if (test.y < tmin) {
          al.y = 0.f;
          nfx[j].y = kGone;
        }
        const float2 w = __fmul2_rn(T[j], al);
        T[j] = __fmul2_rn(T[j], __ffma2_rn(al, neg2, one2));
        c0[j] = __ffma2_rn(w, cr, c0[j]);
        c1[j] = __ffma2_rn(w, cg, c1[j]);
        c2[j] = __ffma2_rn(w, cb, c2[j]);
        // 1 if blended, else 0
        const float2 bl = make_float2(__saturatef(al.x * kSat), __saturatef(al.y * kSat));
        ncf[j] = __fadd2_rn(ncf[j], bl);
        lastf[j] = __ffma2_rn(bl, __ffma2_rn(lastf[j], neg2, k1), lastf[j]);
        // 1 if w beats the best weight so far (strictly: the earliest of equal weights wins)
        const float2 dw = __ffma2_rn(best[j], neg2, w);
        const float2 up = make_float2(__saturatef(dw.x * kSat), __saturatef(dw.y * kSat));
        best[j] = make_float2(fmaxf(best[j].x, w.x), fmaxf(best[j].y, w.y));
        domf[j] = __ffma2_rn(up, __ffma2_rn(domf[j], neg2, kf), domf[j]);
      }
    }
    // fold the batch's bookkeeping into the integer outputs
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const float nc2[2] = {ncf[j].x, ncf[j].y}, l2[2] = {lastf[j].x, lastf[j].y};
      const float d2[2] = {domf[j].x, domf[j].y};
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int h = 2 * j + e;
        ncon[h] += (int)nc2[e];
        if (l2[e] > 0.f) last[h] = b0 + (int)l2[e];
        if (d2[e] >= 0.f) dom[h] = __float_as_int(s_g2[(int)d2[e]].y);
      }
      ncf[j] = lastf[j] = make_float2(0.f, 0.f);
      domf[j] = neg2;
    }
  }
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const float t2[2] = {T[j].x, T[j].y}, r2[2] = {c0[j].x, c0[j].y};
    const float g2[2] = {c1[j].x, c1[j].y}, b2[2] = {c2[j].x, c2[j].y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int h = 2 * j + e;
      if (!(px0 + h < W && py < H)) continue;
      long long p = cs.pix_base[v] + (long long)py * W + px0 + h;
      a.out_rgb[3 * p + 0] = r2[e] + t2[e] * a.bg[0];
      a.out_rgb[3 * p + 1] = g2[e] + t2[e] * a.bg[1];
      a.out_rgb[3 * p + 2] = b2[e] + t2[e] * a.bg[2];
      a.out_T[p] = t2[e];
      a.out_n[p] = ncon[h];
      a.out_last[p] = last[h];
      a.out_dom[p] = dom[h];
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

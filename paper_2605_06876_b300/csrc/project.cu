// EWA projection of every Gaussian into every view (Sec. 3, Eq. 1): float4 plane
// loads, one record of three float4 + int4 rect + tile count per (view,
// Gaussian). Records of pairs culled by the cheap screen test get only
// tiles_touched = 0; their other fields are left unwritten (nothing reads them).
// Blocks take a chunk of Gaussians, screen it cheaply (against every view when
// there are several, reading each Gaussian's mean and scales once) and project
// the surviving pairs with full warps.
#include "gauss_math.cuh"
#include "phases.cuh"

namespace adp {

struct ProjectArgs {
  const float4* mean_logit;
  const float4* logscale;
  const float4* quat;
  const float* sh;
  long long n;
  int deg;
  float near_plane, low_pass, alpha_min;
  float4* xy_op_depth;
  float4* conic;
  float4* rgb;
  int4* rect;
  int* tiles;
  float4* zero_moments;  // optional [V*n][3]: zeroed for every visible record
};

// The view-independent part of a Gaussian: opacity sigmoid(logit) and the six
// entries of Sigma = Rg diag(s^2) Rg^T.
__device__ __forceinline__ float opacity_of(float logit) { return 1.f / (1.f + __expf(-logit)); }

__device__ __forceinline__ void sigma3(float4 ls, float4 q, float* S) {
  float qn = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  Mat3 Rg = rot_of_quat(q.x * qn, q.y * qn, q.z * qn, q.w * qn);
  float s2[3] = {__expf(2.f * ls.x), __expf(2.f * ls.y), __expf(2.f * ls.z)};
  S[0] = Rg.m[0] * Rg.m[0] * s2[0] + Rg.m[1] * Rg.m[1] * s2[1] + Rg.m[2] * Rg.m[2] * s2[2];
  S[1] = Rg.m[0] * Rg.m[3] * s2[0] + Rg.m[1] * Rg.m[4] * s2[1] + Rg.m[2] * Rg.m[5] * s2[2];
  S[2] = Rg.m[0] * Rg.m[6] * s2[0] + Rg.m[1] * Rg.m[7] * s2[1] + Rg.m[2] * Rg.m[8] * s2[2];
  S[3] = Rg.m[3] * Rg.m[3] * s2[0] + Rg.m[4] * Rg.m[4] * s2[1] + Rg.m[5] * Rg.m[5] * s2[2];
  S[4] = Rg.m[3] * Rg.m[6] * s2[0] + Rg.m[4] * Rg.m[7] * s2[1] + Rg.m[5] * Rg.m[8] * s2[2];
  S[5] = Rg.m[6] * Rg.m[6] * s2[0] + Rg.m[7] * Rg.m[7] * s2[1] + Rg.m[8] * Rg.m[8] * s2[2];
}

// EWA projection of a Gaussian (mean ml, opacity o, Sigma S, SH planes shp[0..P))
// into view v; writes record v * n + i. Both projection kernels call this, so a
// view's records do not depend on how many views share the launch.
template <int DEG>
__device__ __forceinline__ void project_view(const ProjectArgs& a, const CamSet& cs, long long i,
                                             int v, float4 ml, float o, const float* S,
                                             const float4* shp) {
  const adp_camera& cam = cs.cam[v];
  long long rec = (long long)v * a.n + i;
  const float* Rw = cam.R;
  float pcx = Rw[0] * ml.x + Rw[1] * ml.y + Rw[2] * ml.z + cam.t[0];
  float pcy = Rw[3] * ml.x + Rw[4] * ml.y + Rw[5] * ml.z + cam.t[1];
  float pcz = Rw[6] * ml.x + Rw[7] * ml.y + Rw[8] * ml.z + cam.t[2];
  bool vis = pcz > a.near_plane && o >= a.alpha_min;
  float4 out0 = make_float4(0.f, 0.f, 0.f, 0.f), out1 = out0, out2 = out0;
  int4 rc = make_int4(0, -1, 0, -1);
  int nt = 0;
  if (vis) {
    // J with x/z, y/z clamped to 1.3x the half field of view
    float inv_z = 1.f / pcz;
    const float limx = cs.lim_x[v], limy = cs.lim_y[v];
    float ux = fminf(limx, fmaxf(-limx, pcx * inv_z));
    float uy = fminf(limy, fmaxf(-limy, pcy * inv_z));
    float j00 = cam.fx * inv_z, j02 = -cam.fx * ux * inv_z;
    float j11 = cam.fy * inv_z, j12 = -cam.fy * uy * inv_z;
    // T = J W (2x3)
    float T0[3], T1[3];
    for (int c = 0; c < 3; ++c) {
      T0[c] = j00 * Rw[c] + j02 * Rw[6 + c];
      T1[c] = j11 * Rw[3 + c] + j12 * Rw[6 + c];
    }
    // Sigma2D = T Sigma T^T
    float ST0[3] = {S[0] * T0[0] + S[1] * T0[1] + S[2] * T0[2],
                    S[1] * T0[0] + S[3] * T0[1] + S[4] * T0[2],
                    S[2] * T0[0] + S[4] * T0[1] + S[5] * T0[2]};
    float ST1[3] = {S[0] * T1[0] + S[1] * T1[1] + S[2] * T1[2],
                    S[1] * T1[0] + S[3] * T1[1] + S[4] * T1[2],
                    S[2] * T1[0] + S[4] * T1[1] + S[5] * T1[2]};
    float ca = T0[0] * ST0[0] + T0[1] * ST0[1] + T0[2] * ST0[2] + a.low_pass;
    float cb = T0[0] * ST1[0] + T0[1] * ST1[1] + T0[2] * ST1[2];
    float cc = T1[0] * ST1[0] + T1[1] * ST1[1] + T1[2] * ST1[2] + a.low_pass;
    float det = ca * cc - cb * cb;
    if (det > 0.f) {
      float idet = 1.f / det;
      float mx = cam.fx * pcx * inv_z + cam.px;
      float my = cam.fy * pcy * inv_z + cam.py;
      // pixel box of o exp(-d^T C d / 2) >= alpha_min
      float k = 2.f * __logf(o / a.alpha_min);
      k = fmaxf(k, 0.f);
      float hx = sqrtf(k * ca), hy = sqrtf(k * cc);
      float x0 = fmaxf(ceilf(mx - hx), 0.f), x1 = fminf(floorf(mx + hx), (float)(cam.width - 1));
      float y0 = fmaxf(ceilf(my - hy), 0.f), y1 = fminf(floorf(my + hy), (float)(cam.height - 1));
      if (x0 <= x1 && y0 <= y1) {
        rc = make_int4((int)x0 / cs.tile_w, (int)x1 / cs.tile_w, (int)y0 / cs.tile_h,
                       (int)y1 / cs.tile_h);
        nt = (rc.y - rc.x + 1) * (rc.w - rc.z + 1);
        // colour from the direction camera centre -> mean
        float ccx = -(Rw[0] * cam.t[0] + Rw[3] * cam.t[1] + Rw[6] * cam.t[2]);
        float ccy = -(Rw[1] * cam.t[0] + Rw[4] * cam.t[1] + Rw[7] * cam.t[2]);
        float ccz = -(Rw[2] * cam.t[0] + Rw[5] * cam.t[1] + Rw[8] * cam.t[2]);
        float dx = ml.x - ccx, dy = ml.y - ccy, dz = ml.z - ccz;
        float il = rsqrtf(dx * dx + dy * dy + dz * dz);
        float Y[16];
        sh_eval_basis(DEG, dx * il, dy * il, dz * il, Y);
        constexpr int K = (DEG + 1) * (DEG + 1);
        float col[3] = {0.5f, 0.5f, 0.5f};
        constexpr int P = (3 * K + 3) / 4;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const float4 c4 = shp[p];
          float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            int f = 4 * p + l;
            if (f < 3 * K) col[f % 3] += cv[l] * Y[f / 3];
          }
        }
        out0 = make_float4(mx, my, o, pcz);
        out1 = make_float4(cc * idet, -cb * idet, ca * idet, 0.f);
        // w: the channels clamped at 0 (bit c for channel c), for the backward
        const int clamped = (col[0] < 0.f ? 1 : 0) | (col[1] < 0.f ? 2 : 0) | (col[2] < 0.f ? 4 : 0);
        out2 = make_float4(fmaxf(col[0], 0.f), fmaxf(col[1], 0.f), fmaxf(col[2], 0.f),
                           (float)clamped);
      }
    }
  }
  a.xy_op_depth[rec] = out0;
  a.conic[rec] = out1;
  a.rgb[rec] = out2;
  a.rect[rec] = rc;
  a.tiles[rec] = nt;
  if (a.zero_moments && nt > 0) {  // the backward's pixel moments of this record
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    a.zero_moments[3 * rec] = z;
    a.zero_moments[3 * rec + 1] = z;
    a.zero_moments[3 * rec + 2] = z;
  }
}

// Full projection of Gaussian i into view v (a survivor of either kernel's
// screen test). The SH degree is a template parameter so that the SH arrays stay in
// registers.
template <int DEG>
__device__ void project_one(const ProjectArgs& a, const CamSet& cs, long long i, int v) {
  constexpr int P = (3 * (DEG + 1) * (DEG + 1) + 3) / 4;
  const float4 ml = a.mean_logit[i];
  const float o = opacity_of(ml.w);
  float S[6];
  sigma3(a.logscale[i], a.quat[i], S);
  float4 shp[P];
#pragma unroll
  for (int p = 0; p < P; ++p) shp[p] = reinterpret_cast<const float4*>(a.sh)[(long long)p * a.n + i];
  project_view<DEG>(a, cs, i, v, ml, o, S, shp);
}

// Conservative screen test from the mean, the largest scale and the opacity:
// the ellipse's box half-width is at most sqrt(k (|J row|^2 s_max^2 + low_pass))
// with k = 2 ln(o / alpha_min), so a Gaussian whose bound misses the image
// (with a margin) cannot touch it. Culled records get tiles_touched = 0. The
// part that does not depend on the view is computed once per Gaussian; per view
// the test compares squared distances (no square root) and takes 1 / z from the
// fast reciprocal, whose error is far inside the 1% margins.
struct CullG {
  float x, y, z;  // the mean
  float ks;       // k s_max^2 (with the margins)
  float klp;      // k low_pass
  bool live;      // o >= alpha_min
};

__device__ __forceinline__ CullG cull_gaussian(const ProjectArgs& a, float4 ml, float4 ls) {
  CullG c;
  c.x = ml.x;
  c.y = ml.y;
  c.z = ml.z;
  const float o = opacity_of(ml.w);
  c.live = o >= a.alpha_min;
  const float k = fmaxf(2.f * __logf(o / a.alpha_min), 0.f) * 1.01f;
  const float smax2 = __expf(2.f * fmaxf(ls.x, fmaxf(ls.y, ls.z)));
  c.ks = k * smax2 * 1.01f;
  c.klp = k * a.low_pass;
  return c;
}

__device__ __forceinline__ bool cull_view(const ProjectArgs& a, const adp_camera& cam, float2 lim,
                                          const CullG& c) {
  const float* Rw = cam.R;
  const float pcz = Rw[6] * c.x + Rw[7] * c.y + Rw[8] * c.z + cam.t[2];
  if (!(pcz > a.near_plane)) return false;
  const float pcx = Rw[0] * c.x + Rw[1] * c.y + Rw[2] * c.z + cam.t[0];
  const float pcy = Rw[3] * c.x + Rw[4] * c.y + Rw[5] * c.z + cam.t[1];
  const float iz = __fdividef(1.f, pcz);
  const float ux = fminf(lim.x, fmaxf(-lim.x, pcx * iz)), uy = fminf(lim.y, fmaxf(-lim.y, pcy * iz));
  const float jx = cam.fx * iz, jy = cam.fy * iz;
  // (half-width - 1)^2 of the bound along x and y
  const float hx2 = jx * jx * (1.f + ux * ux) * c.ks + c.klp;
  const float hy2 = jy * jy * (1.f + uy * uy) * c.ks + c.klp;
  const float mx = cam.fx * pcx * iz + cam.px, my = cam.fy * pcy * iz + cam.py;
  // how far the centre lies outside the image, less the one-pixel margin
  const float ox = fmaxf(-mx, mx - (float)(cam.width - 1)) - 1.f;
  const float oy = fmaxf(-my, my - (float)(cam.height - 1)) - 1.f;
  return (ox <= 0.f || ox * ox <= hx2) && (oy <= 0.f || oy * oy <= hy2);
}

// Appends the entry of every lane with vis set to the block's survivor list: one
// shared atomic per warp, the lanes' slots in lane order (all lanes take part).
__device__ __forceinline__ void append_survivor(int* list, int* cnt, bool vis, int entry) {
  const unsigned m = __ballot_sync(0xffffffffu, vis);
  const unsigned lane = threadIdx.x & 31u;
  int base = 0;
  if (lane == 0 && m) base = atomicAdd(cnt, __popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (vis) list[base + __popc(m & ((1u << lane) - 1u))] = entry;
}

// A culled record: only its tile count (0) is written; nothing reads the rest.
__device__ __forceinline__ void write_culled(const ProjectArgs& a, long long rec) {
  a.tiles[rec] = 0;
}

// Several views: each block takes a chunk of VIEWS_CHUNK Gaussians; a thread
// reads one Gaussian's mean and scales once and screens it against every view,
// the surviving (view, Gaussian) pairs are compacted in shared memory, and the
// block projects them with full warps (the chunk's parameters are then in L1).
// 128-Gaussian chunks and one shared atomic per warp and view took the kernel
// from 278 to 249 us at 1M Gaussians x 16 views.
constexpr int VIEWS_THREADS = 128;
constexpr int VIEWS_CHUNK = 128;
template <int DEG>
__global__ void __launch_bounds__(VIEWS_THREADS) project_views_kernel(ProjectArgs a, CamSet cs) {
  __shared__ int s_list[VIEWS_CHUNK * ADP_MAX_VIEWS];
  __shared__ int s_cnt;
  for (long long c0 = (long long)blockIdx.x * VIEWS_CHUNK; c0 < a.n;
       c0 += (long long)gridDim.x * VIEWS_CHUNK) {
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int q0 = 0; q0 < VIEWS_CHUNK; q0 += VIEWS_THREADS) {
      const int q = q0 + (int)threadIdx.x;
      const long long i = c0 + q;
      const bool in = i < a.n;
      CullG c;
      c.live = false;
      if (in) c = cull_gaussian(a, a.mean_logit[i], a.logscale[i]);
      for (int v = 0; v < cs.n_views; ++v) {
        const bool vis =
            c.live && cull_view(a, cs.cam[v], make_float2(cs.lim_x[v], cs.lim_y[v]), c);
        if (in && !vis) write_culled(a, (long long)v * a.n + i);
        append_survivor(s_list, &s_cnt, vis, (v << 16) | q);
      }
    }
    __syncthreads();
    const int cnt = s_cnt;
    for (int e = threadIdx.x; e < cnt; e += VIEWS_THREADS) {
      const int w = s_list[e];
      project_one<DEG>(a, cs, c0 + (w & 0xffff), w >> 16);
    }
    __syncthreads();
  }
}

constexpr int PROJ_THREADS = 256;
constexpr int PROJ_CHUNK = 512;

// Each CTA takes PROJ_CHUNK Gaussians of one view: a cheap pass culls most of
// them, the survivors are compacted in shared memory and projected by full
// warps, so the expensive EWA and SH work is not diluted by culled lanes.
template <int DEG>
__global__ void __launch_bounds__(PROJ_THREADS) project_kernel(ProjectArgs a, CamSet cs) {
  __shared__ int s_list[PROJ_CHUNK];
  __shared__ int s_cnt;
  const int v = blockIdx.y;
  const float2 lim = make_float2(cs.lim_x[v], cs.lim_y[v]);
  for (long long c0 = (long long)blockIdx.x * PROJ_CHUNK; c0 < a.n;
       c0 += (long long)gridDim.x * PROJ_CHUNK) {
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int q0 = 0; q0 < PROJ_CHUNK; q0 += PROJ_THREADS) {  // warp-uniform
      const int q = q0 + (int)threadIdx.x;
      const long long i = c0 + q;
      const bool in = i < a.n;
      bool vis = false;
      if (in) {
        const CullG c = cull_gaussian(a, a.mean_logit[i], a.logscale[i]);
        vis = c.live && cull_view(a, cs.cam[v], lim, c);
        if (!vis) write_culled(a, (long long)v * a.n + i);
      }
      append_survivor(s_list, &s_cnt, vis, q);
    }
    __syncthreads();
    const int cnt = s_cnt;
    for (int q = threadIdx.x; q < cnt; q += PROJ_THREADS) project_one<DEG>(a, cs, c0 + s_list[q], v);
    __syncthreads();
  }
}

}  // namespace adp

using namespace adp;

extern "C" ADP_API int adp_project(const adp_gaussians* g, const adp_camera* cams, int32_t n_views,
                                   const adp_params* prm, adp_projected* out,
                                   adp_stream_t stream) {
  return project_launch(g, cams, n_views, prm, out, nullptr, (cudaStream_t)stream);
}

int adp::project_launch(const adp_gaussians* g, const adp_camera* cams, int n_views,
                        const adp_params* prm, adp_projected* out, float4* zero_moments,
                        cudaStream_t st) {
  ADP_CHECK_ARG(g && out, "NULL argument");
  ADP_CHECK_ARG(g->n >= 0 && g->n < (1LL << 31), "n = %lld out of range", (long long)g->n);
  ADP_CHECK_ARG(g->sh_degree >= 0 && g->sh_degree <= 3, "sh_degree must be 0..3");
  CamSet cs;
  int rc = make_camset(cams, n_views, prm, &cs);
  if (rc) return rc;
  ADP_CHECK_ARG((long long)n_views * g->n < (1LL << 31), "n_views * n exceeds 2^31");
  if (g->n == 0) return ADP_OK;
  ADP_CHECK_ARG(g->mean_logit && g->logscale && g->quat && g->sh, "NULL Gaussian array");
  ADP_CHECK_ARG(out->xy_opacity_depth && out->conic && out->rgb && out->rect && out->tiles_touched,
                "NULL projected array");
  ADP_CHECK_ARG(aligned(g->mean_logit, 16) && aligned(g->logscale, 16) && aligned(g->quat, 16) &&
                    aligned(g->sh, 16) && aligned(out->xy_opacity_depth, 16) &&
                    aligned(out->conic, 16) && aligned(out->rgb, 16) && aligned(out->rect, 16),
                "float4 arrays must be 16-byte aligned");
  ProjectArgs a;
  a.mean_logit = reinterpret_cast<const float4*>(g->mean_logit);
  a.logscale = reinterpret_cast<const float4*>(g->logscale);
  a.quat = reinterpret_cast<const float4*>(g->quat);
  a.sh = g->sh;
  a.n = g->n;
  a.deg = g->sh_degree;
  a.near_plane = prm->near_plane;
  a.low_pass = prm->low_pass;
  a.alpha_min = prm->alpha_min;
  a.xy_op_depth = reinterpret_cast<float4*>(out->xy_opacity_depth);
  a.conic = reinterpret_cast<float4*>(out->conic);
  a.rgb = reinterpret_cast<float4*>(out->rgb);
  a.rect = reinterpret_cast<int4*>(out->rect);
  a.tiles = out->tiles_touched;
  a.zero_moments = zero_moments;
  if (n_views == 1) {  // survivors compacted to full warps
    dim3 grid((unsigned)((g->n + PROJ_CHUNK - 1) / PROJ_CHUNK), n_views);
    switch (g->sh_degree) {
      case 0: project_kernel<0><<<grid, PROJ_THREADS, 0, st>>>(a, cs); break;
      case 1: project_kernel<1><<<grid, PROJ_THREADS, 0, st>>>(a, cs); break;
      case 2: project_kernel<2><<<grid, PROJ_THREADS, 0, st>>>(a, cs); break;
      default: project_kernel<3><<<grid, PROJ_THREADS, 0, st>>>(a, cs); break;
    }
  } else {  // chunks of Gaussians screened against every view
    const unsigned grid = (unsigned)((g->n + VIEWS_CHUNK - 1) / VIEWS_CHUNK);
    switch (g->sh_degree) {
      case 0: project_views_kernel<0><<<grid, VIEWS_THREADS, 0, st>>>(a, cs); break;
      case 1: project_views_kernel<1><<<grid, VIEWS_THREADS, 0, st>>>(a, cs); break;
      case 2: project_views_kernel<2><<<grid, VIEWS_THREADS, 0, st>>>(a, cs); break;
      default: project_views_kernel<3><<<grid, VIEWS_THREADS, 0, st>>>(a, cs); break;
    }
  }
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

// Hand-written backward of the compositing and projection.
//
// Pass 1 (one CTA per tile, several pixels per thread): walks the tile's list
// back to front from each pixel's last blended Gaussian, recovering the
// transmittance before each Gaussian as T / (1 - alpha) from T_final instead of
// storing it, and the normalised colour behind it by the recurrence
// R <- R + alpha (c - R) starting from the background. Per (view, Gaussian) it
// accumulates pixel moments of dL/dalpha (and the colour gradient); a warp
// reduces its pixels' contributions (a reduce-scatter) before nine scalar
// atomics per record.
// Pass 2 (one thread per visible Gaussian, from a compacted list): turns the
// moments into dL/d(mean2d, conic, opacity), chains them through the EWA
// projection and the SH colour of every view and sums over views, so the
// per-Gaussian parameters are read and the gradients written once per step.
#include "phases.cuh"
#include "tile_composite.cuh"

namespace adp {

struct BwdPixArgs {
  const float4* xyod;
  const float4* conic;
  const float4* rgb;
  const int* inst;
  const int2* ranges;
  long long n;
  const float* img;
  const float* T_final;
  const int* last;
  const float* target;
  const float* dL_drgb;
  float bg[3];
  CompositeConsts kc;
  float4* g2d;     // [V*n][3]
  int* tile_ctr;   // next tile to take, zero at the launch
};

// PX horizontally adjacent pixels per thread; the walk itself is bwd_tile
// (tile_composite.cuh), which the fused batched kernel also runs.
#ifndef ADP_BWD_PX
#define ADP_BWD_PX 4
#endif
#ifndef ADP_BWD_MINB  // resident blocks per SM the register budget is sized for
#define ADP_BWD_MINB 1
#endif
constexpr int BWD_PX = ADP_BWD_PX;

// Loads a tile's per-pixel inputs (final transmittance, last blended position,
// dL/dpixel of the L1 loss or the given upstream gradient) and walks it.
template <int PX, int STAGE>
__device__ __forceinline__ void bwd_pixel_tile(const BwdPixArgs& a, const CamSet& cs,
                                               const int tile, const StageBuf& sb,
                                               int* s_maxlast) {
  constexpr int NP = PX / 2;
  const TileGeom<PX> t = tile_geom<PX>(cs, a.ranges, a.n, tile);
  const float sc = 1.f / (3.f * (float)t.W * (float)t.H);
  BwdIn<PX> in;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    float tt[2], g[2][3];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int h = 2 * j + e;
      tt[e] = 1.f;
      g[e][0] = g[e][1] = g[e][2] = 0.f;
      in.last[h] = 0;
      if (pixel_in(t, h)) {
        const long long p = t.pix_base + (long long)t.py * t.W + t.px0 + h;
        tt[e] = a.T_final[p];
        in.last[h] = a.last[p];
        if (a.dL_drgb) {
          g[e][0] = a.dL_drgb[3 * p];
          g[e][1] = a.dL_drgb[3 * p + 1];
          g[e][2] = a.dL_drgb[3 * p + 2];
        } else {
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) {
            const float d = a.img[3 * p + ch] - a.target[3 * p + ch];
            g[e][ch] = d > 0.f ? sc : (d < 0.f ? -sc : 0.f);
          }
        }
      }
    }
    in.T[j] = make_float2(tt[0], tt[1]);
    in.G0[j] = make_float2(g[0][0], g[1][0]);
    in.G1[j] = make_float2(g[0][1], g[1][1]);
    in.G2[j] = make_float2(g[0][2], g[1][2]);
  }
  bwd_tile<PX, STAGE>(a.xyod, a.conic, a.rgb, a.inst, t, a.kc, a.bg, sb, s_maxlast, in, a.g2d);
}

// Blocks take tiles in order from a counter (zeroed before the launch). With
// BWD_PERSIST > 0 the grid is BWD_PERSIST resident blocks per SM, which leaves
// registers free on every SM for the kernels of the concurrent error-statistics
// stream: their blocks then start without waiting for tiles to retire. With 0,
// the grid has one block per tile.
#ifndef ADP_BWD_PERSIST
#define ADP_BWD_PERSIST 6
#endif
constexpr int BWD_PERSIST = ADP_BWD_PERSIST;

template <int PX, int STAGE>
__global__ void __launch_bounds__(TileLanes<PX>::THREADS, ADP_BWD_MINB)
    bwd_pixel_kernel(BwdPixArgs a, CamSet cs) {
  __shared__ float4 s_g0[STAGE];
  __shared__ float4 s_g1[STAGE];
  __shared__ float4 s_g2[STAGE];
  __shared__ float2 s_y[STAGE];
  __shared__ int s_tile, s_maxlast;
  const StageBuf sb{s_g0, s_g1, s_g2, s_y};
  const int n_tiles = cs.tile_base[cs.n_views];
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_ctr, 1);
    __syncthreads();
    const int tile = s_tile;
    __syncthreads();  // every thread is past the previous tile and has read s_tile
    if (tile >= n_tiles) break;
    bwd_pixel_tile<PX, STAGE>(a, cs, tile, sb, &s_maxlast);
  }
}

struct BwdGaussArgs {
  const float4* mean_logit;
  const float4* logscale;
  const float4* quat;
  const float* sh;
  const int* tiles;
  const float4* rgb;  // projected colours; w holds the clamped channels
  const float4* g2d;
  long long n;
  int deg;
  float low_pass;
  float4* g_ml;
  float4* g_ls;
  float4* g_q;
  float* g_sh;
  float* g2d_accum;   // optional: += the 2D-mean gradient norm of every rendered view
  int* g2d_visits;    // optional: += the number of those views
};

// Chain rule of one visible Gaussian, summed over views. The SH degree is a
// template parameter so that every SH array index is a constant and the arrays
// stay in registers.
// acc: the thread's column of a [4 * planes][BWDG_THREADS] shared-memory array in
// which the SH gradient is summed over the views (written to the planes once);
// shc: the same for the Gaussian's SH coefficients, read from global memory once
// instead of once per view.
constexpr int BWDG_THREADS = 128;
template <int DEG>
__device__ void bwd_one(const BwdGaussArgs& a, const CamSet& cs, long long i, float* acc,
                        float* shc) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int planes = (3 * K + 3) / 4;
  float4 ml = a.mean_logit[i], ls = a.logscale[i], q4 = a.quat[i];
  float qn2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
  float iq = rsqrtf(qn2);
  float qw = q4.x * iq, qx = q4.y * iq, qy = q4.z * iq, qz = q4.w * iq;
  Mat3 Rg = rot_of_quat(qw, qx, qy, qz);
  float s[3] = {__expf(ls.x), __expf(ls.y), __expf(ls.z)};
  float o = 1.f / (1.f + __expf(-ml.w));
  // Sigma3 (full)
  float S[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      S[3 * r + c] = Rg.m[3 * r] * Rg.m[3 * c] * s[0] * s[0] + Rg.m[3 * r + 1] * Rg.m[3 * c + 1] * s[1] * s[1] +
                     Rg.m[3 * r + 2] * Rg.m[3 * c + 2] * s[2] * s[2];
  float gmu[3] = {0.f, 0.f, 0.f}, glogit = 0.f;
  float g2d_norm = 0.f;  // densification statistic of this Gaussian, summed over views
  int g2d_n = 0;
  float G3[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dL/dSigma3 over views
  // SH coefficients and their gradient rows, one float4 plane at a time
  const float4* shp = reinterpret_cast<const float4*>(a.sh) + i;
  float4* gshp = reinterpret_cast<float4*>(a.g_sh) + i;
#pragma unroll
  for (int p = 0; p < planes; ++p) {
    const float4 c4 = shp[(long long)p * a.n];
    shc[(4 * p) * BWDG_THREADS] = c4.x;
    shc[(4 * p + 1) * BWDG_THREADS] = c4.y;
    shc[(4 * p + 2) * BWDG_THREADS] = c4.z;
    shc[(4 * p + 3) * BWDG_THREADS] = c4.w;
  }
#pragma unroll
  for (int f = 0; f < 4 * planes; ++f) acc[f * BWDG_THREADS] = 0.f;
  // the views that render this Gaussian, from loads issued together; the next
  // view's pixel moments are fetched while the current one is worked on
  unsigned vmask = 0u;
  for (int v = 0; v < cs.n_views; ++v)
    vmask |= (a.tiles[(long long)v * a.n + i] > 0 ? 1u : 0u) << v;
  float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0, n2 = n0;
  float nw = 0.f;
  if (vmask) {
    const long long r0 = (long long)(__ffs(vmask) - 1) * a.n + i;
    n0 = a.g2d[3 * r0];
    n1 = a.g2d[3 * r0 + 1];
    n2 = a.g2d[3 * r0 + 2];
    nw = a.rgb[r0].w;
  }
  while (vmask) {
    const int v = __ffs(vmask) - 1;
    vmask &= vmask - 1u;
    const float4 q0 = n0, q1 = n1, q2 = n2;  // pixel moments of dL/dalpha * alpha
    const int clamped = (int)nw;
    if (vmask) {
      const long long rn = (long long)(__ffs(vmask) - 1) * a.n + i;
      n0 = a.g2d[3 * rn];
      n1 = a.g2d[3 * rn + 1];
      n2 = a.g2d[3 * rn + 2];
      nw = a.rgb[rn].w;
    }
    const float mS = q0.x, mSx = q0.y, mSy = q0.z;
    float gA = -0.5f * q0.w, gB = -q1.x, gC = -0.5f * q1.y;
    float gcol[3] = {q1.z, q1.w, q2.x};
    const adp_camera& cam = cs.cam[v];
    const float* Rw = cam.R;
    float pc[3];
    for (int r = 0; r < 3; ++r)
      pc[r] = Rw[3 * r] * ml.x + Rw[3 * r + 1] * ml.y + Rw[3 * r + 2] * ml.z + cam.t[r];
    float z = pc[2], iz = 1.f / z;
    // opacity: dL/do = S / o, do/dlogit = o (1 - o)
    glogit += mS * (1.f - o);
    // colour
    float ccx = -(Rw[0] * cam.t[0] + Rw[3] * cam.t[1] + Rw[6] * cam.t[2]);
    float ccy = -(Rw[1] * cam.t[0] + Rw[4] * cam.t[1] + Rw[7] * cam.t[2]);
    float ccz = -(Rw[2] * cam.t[0] + Rw[5] * cam.t[1] + Rw[8] * cam.t[2]);
    float d[3] = {ml.x - ccx, ml.y - ccy, ml.z - ccz};
    float il = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    float u[3] = {d[0] * il, d[1] * il, d[2] * il};
    float Y[16];
    sh_eval_basis(DEG, u[0], u[1], u[2], Y);
    // channels the projection clamped at 0 pass no gradient
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
      if (clamped & (1 << ch)) gcol[ch] = 0.f;
    // dL/dsh = gcol Y (summed over views), and the weights w_k = sum_ch sh_k,ch gcol_ch
    // of the basis partials in the direction gradient
    float wk[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) wk[k] = 0.f;
#pragma unroll
    for (int p = 0; p < planes; ++p) {
      const float cf[4] = {shc[(4 * p) * BWDG_THREADS], shc[(4 * p + 1) * BWDG_THREADS],
                           shc[(4 * p + 2) * BWDG_THREADS], shc[(4 * p + 3) * BWDG_THREADS]};
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int f = 4 * p + l;
        if (f < 3 * K) {
          acc[f * BWDG_THREADS] = fmaf(gcol[f % 3], Y[f / 3], acc[f * BWDG_THREADS]);
          wk[f / 3] += cf[l] * gcol[f % 3];
        }
      }
      // one plane at a time: keeps the compiler from hoisting every plane's
      // shared-memory loads (and their registers) to the top of the loop
      asm volatile("" ::: "memory");
    }
    float gu[3] = {0.f, 0.f, 0.f};
    if (DEG > 0) sh_grad_dot(DEG, u[0], u[1], u[2], wk, gu);
    float ud = gu[0] * u[0] + gu[1] * u[1] + gu[2] * u[2];
    for (int k = 0; k < 3; ++k) gmu[k] += (gu[k] - ud * u[k]) * il;
    // EWA
    const float limx = cs.lim_x[v], limy = cs.lim_y[v];
    float txz = pc[0] * iz, tyz = pc[1] * iz;
    bool clx = txz < -limx || txz > limx, cly = tyz < -limy || tyz > limy;
    float ux = fminf(limx, fmaxf(-limx, txz)), uy = fminf(limy, fmaxf(-limy, tyz));
    float J00 = cam.fx * iz, J02 = -cam.fx * ux * iz, J11 = cam.fy * iz, J12 = -cam.fy * uy * iz;
    float T0[3], T1[3];
    for (int c = 0; c < 3; ++c) {
      T0[c] = J00 * Rw[c] + J02 * Rw[6 + c];
      T1[c] = J11 * Rw[3 + c] + J12 * Rw[6 + c];
    }
    float ST0[3], ST1[3];
    for (int r = 0; r < 3; ++r) {
      ST0[r] = S[3 * r] * T0[0] + S[3 * r + 1] * T0[1] + S[3 * r + 2] * T0[2];
      ST1[r] = S[3 * r] * T1[0] + S[3 * r + 1] * T1[1] + S[3 * r + 2] * T1[2];
    }
    float ca = T0[0] * ST0[0] + T0[1] * ST0[1] + T0[2] * ST0[2] + a.low_pass;
    float cb = T0[0] * ST1[0] + T0[1] * ST1[1] + T0[2] * ST1[2];
    float cc = T1[0] * ST1[0] + T1[1] * ST1[1] + T1[2] * ST1[2] + a.low_pass;
    float idet = 1.f / (ca * cc - cb * cb);
    float QA = cc * idet, QB = -cb * idet, QC = ca * idet;
    // dL/dSigma2D = -Q G_Q Q with G_Q = [[gA, gB/2], [gB/2, gC]]
    float hB = 0.5f * gB;
    float M00 = gA * QA + hB * QB, M01 = gA * QB + hB * QC;
    float M10 = hB * QA + gC * QB, M11 = hB * QB + gC * QC;
    float ga = -(QA * M00 + QB * M10);
    float gbh = -(QA * M01 + QB * M11);  // symmetric off-diagonal entry
    float gc2 = -(QB * M01 + QC * M11);
    // G2 = [[ga, gbh], [gbh, gc2]]; dL/dSigma3 += T^T G2 T; dL/dT = 2 G2 T Sigma3
    float GT0[3], GT1[3];
    for (int c = 0; c < 3; ++c) {
      GT0[c] = ga * T0[c] + gbh * T1[c];
      GT1[c] = gbh * T0[c] + gc2 * T1[c];
    }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) G3[3 * r + c] += T0[r] * GT0[c] + T1[r] * GT1[c];
    float dT0[3], dT1[3];
    for (int c = 0; c < 3; ++c) {
      dT0[c] = 2.f * (GT0[0] * S[c] + GT0[1] * S[3 + c] + GT0[2] * S[6 + c]);
      dT1[c] = 2.f * (GT1[0] * S[c] + GT1[1] * S[3 + c] + GT1[2] * S[6 + c]);
    }
    // T = J W: dL/dJ = dL/dT W^T
    float gJ00 = dT0[0] * Rw[0] + dT0[1] * Rw[1] + dT0[2] * Rw[2];
    float gJ02 = dT0[0] * Rw[6] + dT0[1] * Rw[7] + dT0[2] * Rw[8];
    float gJ11 = dT1[0] * Rw[3] + dT1[1] * Rw[4] + dT1[2] * Rw[5];
    float gJ12 = dT1[0] * Rw[6] + dT1[1] * Rw[7] + dT1[2] * Rw[8];
    float gp[3] = {0.f, 0.f, 0.f};
    float iz2 = iz * iz;
    gp[2] += -cam.fx * iz2 * gJ00 - cam.fy * iz2 * gJ11 + cam.fx * ux * iz2 * gJ02 +
             cam.fy * uy * iz2 * gJ12;
    if (!clx) {
      gp[0] += -cam.fx * iz2 * gJ02;
      gp[2] += cam.fx * pc[0] * iz2 * iz * gJ02;
    }
    if (!cly) {
      gp[1] += -cam.fy * iz2 * gJ12;
      gp[2] += cam.fy * pc[1] * iz2 * iz * gJ12;
    }
    // 2D mean: dL/dmean = -(Q [Sx, Sy])
    const float gmx = -(QA * mSx + QB * mSy), gmy = -(QB * mSx + QC * mSy);
    // the image-space gradient in normalised device coordinates (x_ndc spans W / 2
    // pixels per unit), as the adaptive density control accumulates it
    g2d_norm += sqrtf(fmaf(gmx * 0.5f * (float)cam.width, gmx * 0.5f * (float)cam.width,
                           (gmy * 0.5f * (float)cam.height) * (gmy * 0.5f * (float)cam.height)));
    ++g2d_n;
    gp[0] += gmx * cam.fx * iz;
    gp[1] += gmy * cam.fy * iz;
    gp[2] += -(gmx * cam.fx * pc[0] + gmy * cam.fy * pc[1]) * iz2;
    for (int k = 0; k < 3; ++k) gmu[k] += Rw[k] * gp[0] + Rw[3 + k] * gp[1] + Rw[6 + k] * gp[2];
  }
  // Sigma3 = Rg diag(s^2) Rg^T: symmetrise G3, then scales and rotation
  float Gs[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Gs[3 * r + c] = 0.5f * (G3[3 * r + c] + G3[3 * c + r]);
  float GR[9];  // dL/dRg = 2 Gs Rg diag(s^2)
  float gls[3];
  for (int j = 0; j < 3; ++j) {
    float acc = 0.f;
    for (int r = 0; r < 3; ++r) {
      float gr = 0.f;
      for (int k = 0; k < 3; ++k) gr += Gs[3 * r + k] * Rg.m[3 * k + j];
      GR[3 * r + j] = 2.f * gr * s[j] * s[j];
      acc += Rg.m[3 * r + j] * gr;
    }
    gls[j] = 2.f * s[j] * s[j] * acc;
  }
  // dR/dq for the normalised quaternion
  float gw = 2.f * (-qz * GR[1] + qy * GR[2] + qz * GR[3] - qx * GR[5] - qy * GR[6] + qx * GR[7]);
  float gx = 2.f * (qy * GR[1] + qz * GR[2] + qy * GR[3] - 2.f * qx * GR[4] - qw * GR[5] +
                    qz * GR[6] + qw * GR[7] - 2.f * qx * GR[8]);
  float gy = 2.f * (-2.f * qy * GR[0] + qx * GR[1] + qw * GR[2] + qx * GR[3] + qz * GR[5] -
                    qw * GR[6] + qz * GR[7] - 2.f * qy * GR[8]);
  float gz = 2.f * (-2.f * qz * GR[0] - qw * GR[1] + qx * GR[2] + qw * GR[3] - 2.f * qz * GR[4] +
                    qy * GR[5] + qx * GR[6] + qy * GR[7]);
  float dotq = gw * qw + gx * qx + gy * qy + gz * qz;
  if (a.g2d_accum) {
    a.g2d_accum[i] += g2d_norm;
    a.g2d_visits[i] += g2d_n;
  }
#pragma unroll
  for (int p = 0; p < planes; ++p)
    gshp[(long long)p * a.n] = make_float4(acc[(4 * p) * BWDG_THREADS], acc[(4 * p + 1) * BWDG_THREADS],
                                           acc[(4 * p + 2) * BWDG_THREADS],
                                           acc[(4 * p + 3) * BWDG_THREADS]);
  a.g_ml[i] = make_float4(gmu[0], gmu[1], gmu[2], glogit);
  a.g_ls[i] = make_float4(gls[0], gls[1], gls[2], 0.f);
  a.g_q[i] = make_float4((gw - dotq * qw) * iq, (gx - dotq * qx) * iq, (gy - dotq * qy) * iq,
                         (gz - dotq * qz) * iq);
}

// Zeroes the gradient of every Gaussian rendered in no view (or, for a
// gradient with a row mask, writes the mask instead) and appends the
// others to a list (the list order does not change any result), so the
// chain-rule pass runs on full warps of visible Gaussians. Warps count their
// visible lanes with a ballot; one global atomic per block reserves the block's
// slots.
__global__ void __launch_bounds__(256) bwd_visible_kernel(const int* tiles, long long n,
                                                          int n_views, int planes, float4* g_ml,
                                                          float4* g_ls, float4* g_q, float4* g_sh,
                                                          uint8_t* rows, int* list,
                                                          unsigned long long* count) {
  __shared__ unsigned s_cnt[8];
  __shared__ unsigned long long s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long i0 = blockIdx.x * (long long)blockDim.x; i0 < n;
       i0 += (long long)gridDim.x * blockDim.x) {
    const long long i = i0 + threadIdx.x;
    bool seen = false;
    if (i < n)
      for (int v = 0; v < n_views; ++v) seen |= tiles[(long long)v * n + i] > 0;
    const unsigned vis = __ballot_sync(0xffffffffu, seen);
    if (lane == 0) s_cnt[warp] = __popc(vis);
    __syncthreads();
    unsigned before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const unsigned c = s_cnt[w];
      before += w < warp ? c : 0u;
      total += c;
    }
    if (threadIdx.x == 0 && total) s_base = atomicAdd(count, (unsigned long long)total);
    __syncthreads();
    if (seen) list[s_base + before + __popc(vis & lanemask_lt())] = (int)i;
    if (rows) {  // masked gradient: mark the rows; the others are never touched
      if (i < n) rows[i] = seen ? 1 : 0;
    } else if (i < n && !seen) {
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      g_ml[i] = z;
      g_ls[i] = z;
      g_q[i] = z;
      for (int p = 0; p < planes; ++p) g_sh[(long long)p * n + i] = z;
    }
  }
}

#ifndef ADP_BWDG_MINB  // resident 128-thread blocks per SM the register budget is sized for
#define ADP_BWDG_MINB 4
#endif
template <int DEG>
__global__ void __launch_bounds__(BWDG_THREADS, ADP_BWDG_MINB)
    bwd_gauss_kernel(BwdGaussArgs a, CamSet cs, const int* list,
                     const unsigned long long* n_list) {
  constexpr int planes = (3 * (DEG + 1) * (DEG + 1) + 3) / 4;
  __shared__ float s_acc[4 * planes * BWDG_THREADS];
  __shared__ float s_shc[4 * planes * BWDG_THREADS];
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < (long long)*n_list) bwd_one<DEG>(a, cs, list[t], s_acc + threadIdx.x, s_shc + threadIdx.x);
}

}  // namespace adp

using namespace adp;

extern "C" ADP_API size_t adp_render_backward_workspace_size(int64_t n, int32_t n_views) {
  if (n < 0 || n_views < 1) return 0;
  return carve_bytes<float4>(3 * (size_t)n * n_views) + carve_bytes<int>(n) +
         carve_bytes<unsigned long long>(1) + carve_bytes<int>(1);
}

extern "C" ADP_API int adp_render_backward(const adp_gaussians* g, const adp_projected* pr,
                                           const adp_bins* bins, const adp_image* fwd,
                                           const float* target, const float* dL_drgb,
                                           const adp_camera* cams, int32_t n_views,
                                           const float* bg, const adp_params* prm,
                                           adp_gaussians* grad, float* grad2d_accum,
                                           int32_t* grad2d_visits, void* ws, size_t ws_bytes,
                                           adp_stream_t stream) {
  ADP_CHECK_ARG(g && pr && bins && fwd && grad, "NULL argument");
  ADP_CHECK_ARG(target || dL_drgb, "one of target and dL_drgb must be given");
  ADP_CHECK_ARG(!grad2d_accum == !grad2d_visits, "give both or neither densification accumulators");
  ADP_CHECK_ARG(grad->n == g->n && grad->sh_degree == g->sh_degree, "grad shape mismatch");
  ADP_CHECK_ARG(g->sh_degree >= 0 && g->sh_degree <= 3, "sh_degree must be 0..3");
  CamSet cs;
  int rc = make_camset(cams, n_views, prm, &cs);
  if (rc) return rc;
  ADP_CHECK_ARG(g->n >= 0 && (long long)g->n * n_views < (1LL << 31), "n_views * n exceeds 2^31");
  ADP_CHECK_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
  size_t need = adp_render_backward_workspace_size(g->n, n_views);
  ADP_CHECK_ARG(ws_bytes >= need, "workspace %zu bytes, need %zu", ws_bytes, need);
  if (g->n == 0) return ADP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Carver cv(ws, ws_bytes);
  float4* g2d = cv.take<float4>(3 * (size_t)g->n * n_views);
  int* list = cv.take<int>(g->n);
  unsigned long long* n_list = cv.take<unsigned long long>(1);
  int* tile_ctr = cv.take<int>(1);
  // the list count and the tile counter are reset by the same launch
  FillSet fill;
  fill.add(n_list, sizeof(unsigned long long));
  fill.add(tile_ctr, sizeof(int));
  rc = zero_visible_moments(pr->tiles_touched, (long long)g->n * n_views, g2d, fill, st);
  if (rc) return rc;
  BwdPixArgs pa;
  pa.xyod = reinterpret_cast<const float4*>(pr->xy_opacity_depth);
  pa.conic = reinterpret_cast<const float4*>(pr->conic);
  pa.rgb = reinterpret_cast<const float4*>(pr->rgb);
  pa.inst = bins->inst_gauss;
  pa.ranges = reinterpret_cast<const int2*>(bins->tile_range);
  pa.n = g->n;
  pa.img = fwd->rgb;
  pa.T_final = fwd->T_final;
  pa.last = fwd->last;
  pa.target = target;
  pa.dL_drgb = dL_drgb;
  for (int c = 0; c < 3; ++c) pa.bg[c] = bg ? bg[c] : 0.f;
  pa.kc = CompositeConsts{prm->alpha_min, prm->alpha_max, prm->t_min, log2f(prm->alpha_min)};
  pa.g2d = g2d;
  pa.tile_ctr = tile_ctr;
  long long grid = cs.tile_base[n_views];
  if (BWD_PERSIST > 0) {
    int dev = 0, sms = 0;
    ADP_CUDA(cudaGetDevice(&dev));
    ADP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    grid = std::min<long long>(grid, (long long)sms * BWD_PERSIST);
  }
  const dim3 pg((unsigned)grid), pb(TileLanes<BWD_PX>::THREADS);
  switch (stage_size(prm)) {
    case 64: bwd_pixel_kernel<BWD_PX, 64><<<pg, pb, 0, st>>>(pa, cs); break;
    case 128: bwd_pixel_kernel<BWD_PX, 128><<<pg, pb, 0, st>>>(pa, cs); break;
    default: bwd_pixel_kernel<BWD_PX, 256><<<pg, pb, 0, st>>>(pa, cs); break;
  }
  ADP_LAUNCH_CHECK();
  return backward_gauss_phase(g, pr, cs, prm, grad, grad2d_accum, grad2d_visits, g2d, list, n_list,
                              st);
}

namespace adp {

// Zeroes the pixel-moment rows (three float4) of the visible records only: the
// per-pixel pass adds to records in tile lists, and the per-Gaussian pass reads
// records with tiles_touched > 0, so nothing reads the rows of culled records.
__global__ void zero_visible_kernel(const int* tiles, long long n_rec, float4* g2d, FillSet f) {
  fill_ranges_device(f, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                     (long long)gridDim.x * blockDim.x);
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n_rec;
       r += (long long)gridDim.x * blockDim.x) {
    if (tiles[r] > 0) {
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      g2d[3 * r] = z;
      g2d[3 * r + 1] = z;
      g2d[3 * r + 2] = z;
    }
  }
}

int zero_visible_moments(const int* tiles, long long n_rec, float4* g2d, const FillSet& f,
                         cudaStream_t st) {
  if (n_rec <= 0) return launch_fill(f, st);
  zero_visible_kernel<<<grid_for(n_rec, 256, 148 * 16), 256, 0, st>>>(tiles, n_rec, g2d, f);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

int backward_gauss_phase(const adp_gaussians* g, const adp_projected* pr, const CamSet& cs,
                         const adp_params* prm, adp_gaussians* grad, float* grad2d_accum,
                         int32_t* grad2d_visits, const float4* g2d, int* list,
                         unsigned long long* n_list, cudaStream_t st) {
  const int n_views = cs.n_views;
  BwdGaussArgs ga;
  ga.mean_logit = reinterpret_cast<const float4*>(g->mean_logit);
  ga.logscale = reinterpret_cast<const float4*>(g->logscale);
  ga.quat = reinterpret_cast<const float4*>(g->quat);
  ga.sh = g->sh;
  ga.tiles = pr->tiles_touched;
  ga.rgb = reinterpret_cast<const float4*>(pr->rgb);
  ga.g2d = g2d;
  ga.n = g->n;
  ga.deg = g->sh_degree;
  ga.low_pass = prm->low_pass;
  ga.g_ml = reinterpret_cast<float4*>(grad->mean_logit);
  ga.g_ls = reinterpret_cast<float4*>(grad->logscale);
  ga.g_q = reinterpret_cast<float4*>(grad->quat);
  ga.g_sh = grad->sh;
  ga.g2d_accum = grad2d_accum;
  ga.g2d_visits = grad2d_visits;
  bwd_visible_kernel<<<grid_for(g->n, 256, 148 * 16), 256, 0, st>>>(
      pr->tiles_touched, g->n, n_views, sh_planes(g->sh_degree), ga.g_ml, ga.g_ls, ga.g_q,
      reinterpret_cast<float4*>(grad->sh), grad->rows, list, n_list);
  const unsigned gb = grid_for(g->n, BWDG_THREADS);
  switch (g->sh_degree) {
    case 0: bwd_gauss_kernel<0><<<gb, BWDG_THREADS, 0, st>>>(ga, cs, list, n_list); break;
    case 1: bwd_gauss_kernel<1><<<gb, BWDG_THREADS, 0, st>>>(ga, cs, list, n_list); break;
    case 2: bwd_gauss_kernel<2><<<gb, BWDG_THREADS, 0, st>>>(ga, cs, list, n_list); break;
    default: bwd_gauss_kernel<3><<<gb, BWDG_THREADS, 0, st>>>(ga, cs, list, n_list); break;
  }
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

}  // namespace adp

// The D-SSIM term of the training loss the baselines use (and the paper leaves
// unchanged, Sec. 5.1): L = (1 - lambda) L1 + lambda (1 - SSIM), per view, with the
// SSIM of each colour channel under an 11x11 Gaussian window (sigma 1.5, zero
// padding outside the image) averaged over the view's pixels and channels.
//
// With the five window sums m1 = G*x, m2 = G*y, q11 = G*x^2, q22 = G*y^2,
// q12 = G*(xy) of the render x and the target y, SSIM = A1 A2 / (B1 B2) where
// A1 = 2 m1 m2 + C1, A2 = 2 (q12 - m1 m2) + C2, B1 = m1^2 + m2^2 + C1 and
// B2 = q11 - m1^2 + q22 - m2^2 + C2. Its derivative with respect to x(u) is
// G*(dS/dm1)(u) + 2 x(u) G*(dS/dq11)(u) + y(u) G*(dS/dq12)(u), the window being
// symmetric, so the adjoint of each window sum is the same zero-padded sum.
// Two kernels, each one 32x32 tile and its 5-pixel halo in shared memory, one
// channel at a time, the window applied as a row pass then a column pass: the
// forward computes the SSIM map and the three derivative maps, the backward sums
// those under the window and adds the L1 term.
#include "common.cuh"

namespace adp {

constexpr int SS_T = 32;             // output tile edge
constexpr int SS_R = 5;              // window radius
constexpr int SS_E = SS_T + 2 * SS_R;  // staged edge
constexpr float SS_C1 = 0.01f * 0.01f;
constexpr float SS_C2 = 0.03f * 0.03f;

// Normalised 1-D Gaussian weights (sigma 1.5), computed by the block.
__device__ __forceinline__ void ssim_weights(float* w) {
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int k = 0; k <= 2 * SS_R; ++k) {
      const float d = (float)(k - SS_R);
      w[k] = expf(-d * d / (2.f * 1.5f * 1.5f));
      s += w[k];
    }
    for (int k = 0; k <= 2 * SS_R; ++k) w[k] /= s;
  }
}

struct SsimArgs {
  const float* img;
  const float* tgt;
  float* dmap;       // [3 channels][3 maps][P]: dS/dm1, dS/dq11, dS/dq12, scaled
  float* dL;         // [P][3]
  double* loss;      // [V][2]: mean L1, mean SSIM (or NULL)
  float lambda;
  long long P;
};

__global__ void __launch_bounds__(256) ssim_fwd_kernel(SsimArgs a, CamSet cs) {
  __shared__ float s_w[2 * SS_R + 1];
  __shared__ float s_x[SS_E][SS_E];
  __shared__ float s_y[SS_E][SS_E];
  __shared__ float s_h[5][SS_E][SS_T];
  __shared__ double s_d[8][2];
  const int v = blockIdx.y;
  const int W = cs.cam[v].width, H = cs.cam[v].height;
  const int ntx = (W + SS_T - 1) / SS_T, nty = (H + SS_T - 1) / SS_T;
  if ((int)blockIdx.x >= ntx * nty) return;
  const int tx0 = (blockIdx.x % ntx) * SS_T, ty0 = (blockIdx.x / ntx) * SS_T;
  const long long base = cs.pix_base[v];
  const float scale = -a.lambda / (3.f * (float)W * (float)H);  // d(loss)/dS per pixel-channel
  ssim_weights(s_w);
  double s_sum = 0.0, l1_sum = 0.0;
  for (int c = 0; c < 3; ++c) {
    __syncthreads();
    for (int q = threadIdx.x; q < SS_E * SS_E; q += blockDim.x) {
      const int r = q / SS_E, cc = q - r * SS_E;
      const int gx = tx0 - SS_R + cc, gy = ty0 - SS_R + r;
      float xv = 0.f, yv = 0.f;
      if (gx >= 0 && gy >= 0 && gx < W && gy < H) {
        const long long p = base + (long long)gy * W + gx;
        xv = a.img[3 * p + c];
        yv = a.tgt[3 * p + c];
      }
      s_x[r][cc] = xv;
      s_y[r][cc] = yv;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < SS_E * SS_T; q += blockDim.x) {  // row pass
      const int r = q / SS_T, cx = q - r * SS_T;
      float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f, h4 = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * SS_R; ++k) {
        const float wk = s_w[k], xv = s_x[r][cx + k], yv = s_y[r][cx + k];
        h0 = fmaf(wk, xv, h0);
        h1 = fmaf(wk, yv, h1);
        h2 = fmaf(wk, xv * xv, h2);
        h3 = fmaf(wk, yv * yv, h3);
        h4 = fmaf(wk, xv * yv, h4);
      }
      s_h[0][r][cx] = h0;
      s_h[1][r][cx] = h1;
      s_h[2][r][cx] = h2;
      s_h[3][r][cx] = h3;
      s_h[4][r][cx] = h4;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < SS_T * SS_T; q += blockDim.x) {  // column pass
      const int oy = q / SS_T, ox = q - oy * SS_T;
      const int x = tx0 + ox, y = ty0 + oy;
      if (x >= W || y >= H) continue;
      float m1 = 0.f, m2 = 0.f, q11 = 0.f, q22 = 0.f, q12 = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * SS_R; ++k) {
        const float wk = s_w[k];
        m1 = fmaf(wk, s_h[0][oy + k][ox], m1);
        m2 = fmaf(wk, s_h[1][oy + k][ox], m2);
        q11 = fmaf(wk, s_h[2][oy + k][ox], q11);
        q22 = fmaf(wk, s_h[3][oy + k][ox], q22);
        q12 = fmaf(wk, s_h[4][oy + k][ox], q12);
      }
      const float A1 = 2.f * m1 * m2 + SS_C1, A2 = 2.f * (q12 - m1 * m2) + SS_C2;
      const float B1 = m1 * m1 + m2 * m2 + SS_C1, B2 = (q11 - m1 * m1) + (q22 - m2 * m2) + SS_C2;
      const float iB = 1.f / (B1 * B2);
      const float S = A1 * A2 * iB;
      // dS/dm1, dS/dq11, dS/dq12
      const float d_m1 = (2.f * m2 * A2 - 2.f * m2 * A1) * iB - S * (2.f * m1 / B1 - 2.f * m1 / B2);
      const float d_q11 = -S / B2;
      const float d_q12 = 2.f * A1 * iB;
      const long long p = base + (long long)y * W + x;
      a.dmap[(3LL * c + 0) * a.P + p] = scale * d_m1;
      a.dmap[(3LL * c + 1) * a.P + p] = scale * d_q11;
      a.dmap[(3LL * c + 2) * a.P + p] = scale * d_q12;
      s_sum += (double)S;
      l1_sum += (double)fabsf(s_x[oy + SS_R][ox + SS_R] - s_y[oy + SS_R][ox + SS_R]);
    }
  }
  if (a.loss) {  // block sums of SSIM and |x - y|, one pair of atomics per block
    for (int o = 16; o > 0; o >>= 1) {
      s_sum += __shfl_xor_sync(0xffffffffu, s_sum, o);
      l1_sum += __shfl_xor_sync(0xffffffffu, l1_sum, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
      s_d[warp][0] = l1_sum;
      s_d[warp][1] = s_sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t0 = 0.0, t1 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        t0 += s_d[w][0];
        t1 += s_d[w][1];
      }
      const double inv = 1.0 / (3.0 * (double)W * (double)H);
      atomicAdd(&a.loss[2 * v], t0 * inv);
      atomicAdd(&a.loss[2 * v + 1], t1 * inv);
    }
  }
}

__global__ void __launch_bounds__(256) ssim_bwd_kernel(SsimArgs a, CamSet cs) {
  __shared__ float s_w[2 * SS_R + 1];
  __shared__ float s_d[3][SS_E][SS_E];
  __shared__ float s_h[3][SS_E][SS_T];
  const int v = blockIdx.y;
  const int W = cs.cam[v].width, H = cs.cam[v].height;
  const int ntx = (W + SS_T - 1) / SS_T, nty = (H + SS_T - 1) / SS_T;
  if ((int)blockIdx.x >= ntx * nty) return;
  const int tx0 = (blockIdx.x % ntx) * SS_T, ty0 = (blockIdx.x / ntx) * SS_T;
  const long long base = cs.pix_base[v];
  const float sc1 = (1.f - a.lambda) / (3.f * (float)W * (float)H);  // the L1 term
  ssim_weights(s_w);
  for (int c = 0; c < 3; ++c) {
    __syncthreads();
    for (int q = threadIdx.x; q < SS_E * SS_E; q += blockDim.x) {
      const int r = q / SS_E, cc = q - r * SS_E;
      const int gx = tx0 - SS_R + cc, gy = ty0 - SS_R + r;
      float d0 = 0.f, d1 = 0.f, d2 = 0.f;
      if (gx >= 0 && gy >= 0 && gx < W && gy < H) {
        const long long p = base + (long long)gy * W + gx;
        d0 = a.dmap[(3LL * c + 0) * a.P + p];
        d1 = a.dmap[(3LL * c + 1) * a.P + p];
        d2 = a.dmap[(3LL * c + 2) * a.P + p];
      }
      s_d[0][r][cc] = d0;
      s_d[1][r][cc] = d1;
      s_d[2][r][cc] = d2;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < SS_E * SS_T; q += blockDim.x) {  // row pass
      const int r = q / SS_T, cx = q - r * SS_T;
      float h0 = 0.f, h1 = 0.f, h2 = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * SS_R; ++k) {
        const float wk = s_w[k];
        h0 = fmaf(wk, s_d[0][r][cx + k], h0);
        h1 = fmaf(wk, s_d[1][r][cx + k], h1);
        h2 = fmaf(wk, s_d[2][r][cx + k], h2);
      }
      s_h[0][r][cx] = h0;
      s_h[1][r][cx] = h1;
      s_h[2][r][cx] = h2;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < SS_T * SS_T; q += blockDim.x) {  // column pass
      const int oy = q / SS_T, ox = q - oy * SS_T;
      const int x = tx0 + ox, y = ty0 + oy;
      if (x >= W || y >= H) continue;
      float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * SS_R; ++k) {
        const float wk = s_w[k];
        g0 = fmaf(wk, s_h[0][oy + k][ox], g0);
        g1 = fmaf(wk, s_h[1][oy + k][ox], g1);
        g2 = fmaf(wk, s_h[2][oy + k][ox], g2);
      }
      const long long p = base + (long long)y * W + x;
      const float xv = a.img[3 * p + c], yv = a.tgt[3 * p + c];
      const float d = xv - yv;
      const float l1 = d > 0.f ? sc1 : (d < 0.f ? -sc1 : 0.f);
      a.dL[3 * p + c] = l1 + g0 + 2.f * xv * g1 + yv * g2;
    }
  }
}

}  // namespace adp

using namespace adp;

extern "C" ADP_API size_t adp_dssim_workspace_size(int32_t n_views, const adp_camera* cams) {
  if (!cams || n_views < 1 || n_views > ADP_MAX_VIEWS) return 0;
  long long P = 0;
  for (int v = 0; v < n_views; ++v) P += (long long)cams[v].width * cams[v].height;
  return carve_bytes<float>(9 * (size_t)P);
}

extern "C" ADP_API int adp_dssim_loss_grad(const float* img, const float* target,
                                           const adp_camera* cams, int32_t n_views,
                                           float lambda, const adp_params* prm, float* dL_drgb,
                                           double* loss, void* ws, size_t ws_bytes,
                                           adp_stream_t stream) {
  ADP_CHECK_ARG(img && target && dL_drgb, "NULL argument");
  ADP_CHECK_ARG(lambda >= 0.f && lambda <= 1.f, "lambda must be in [0, 1]");
  CamSet cs;
  int rc = make_camset(cams, n_views, prm, &cs);
  if (rc) return rc;
  ADP_CHECK_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
  const size_t need = adp_dssim_workspace_size(n_views, cams);
  ADP_CHECK_ARG(ws_bytes >= need, "workspace %zu bytes, need %zu", ws_bytes, need);
  cudaStream_t st = (cudaStream_t)stream;
  SsimArgs a;
  a.img = img;
  a.tgt = target;
  a.dmap = static_cast<float*>(ws);
  a.dL = dL_drgb;
  a.loss = loss;
  a.lambda = lambda;
  a.P = cs.pix_base[n_views];
  if (loss) {
    FillSet f;
    f.add(loss, sizeof(double) * 2 * n_views);
    rc = launch_fill(f, st);
    if (rc) return rc;
  }
  int max_tiles = 0;
  for (int v = 0; v < n_views; ++v) {
    const int t = ((cams[v].width + SS_T - 1) / SS_T) * ((cams[v].height + SS_T - 1) / SS_T);
    max_tiles = t > max_tiles ? t : max_tiles;
  }
  ssim_fwd_kernel<<<dim3(max_tiles, n_views), 256, 0, st>>>(a, cs);
  ssim_bwd_kernel<<<dim3(max_tiles, n_views), 256, 0, st>>>(a, cs);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

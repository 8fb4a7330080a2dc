// One bias-corrected Adam step over every parameter plane (the optimizer the
// paper leaves unchanged, Sec. 5.1): one thread per float4 of each plane,
// parameters, moments and gradients each read once and written once.
#include "common.cuh"

namespace adp {

struct AdamArgs {
  float4 *p_ml, *p_ls, *p_q, *p_sh;
  const float4 *g_ml, *g_ls, *g_q, *g_sh;
  float4 *m_ml, *m_ls, *m_q, *m_sh;
  float4 *v_ml, *v_ls, *v_q, *v_sh;
  long long n;
  int planes;
  float lr[6];
  float b1, b2, eps, bc1, bc2;
  const int* d_step;  // if set, the step number is read here (bias corrections on device)
};

__device__ __forceinline__ float adam1(float& p, float g, float& m, float& v, float lr,
                                       const AdamArgs& a, float bc1, float bc2) {
  m = a.b1 * m + (1.f - a.b1) * g;
  v = a.b2 * v + (1.f - a.b2) * g * g;
  float mh = m / bc1, vh = v / bc2;
  p -= lr * mh / (sqrtf(vh) + a.eps);
  return p;
}

__device__ __forceinline__ void adam4(float4* P, const float4* G, float4* M, float4* V,
                                      long long idx, const float* lr4, const AdamArgs& a,
                                      float bc1, float bc2) {
  float4 p = P[idx], g = G[idx], m = M[idx], v = V[idx];
  adam1(p.x, g.x, m.x, v.x, lr4[0], a, bc1, bc2);
  adam1(p.y, g.y, m.y, v.y, lr4[1], a, bc1, bc2);
  adam1(p.z, g.z, m.z, v.z, lr4[2], a, bc1, bc2);
  adam1(p.w, g.w, m.w, v.w, lr4[3], a, bc1, bc2);
  P[idx] = p;
  M[idx] = m;
  V[idx] = v;
}

// blockIdx.y selects the plane: 0 mean+logit, 1 log-scale, 2 quaternion,
// 3.. SH planes; each thread updates one float4 of it.
__global__ void adam_kernel(AdamArgs a) {
  __shared__ float s_bc[2];
  if (threadIdx.x == 0) {  // bias corrections, once per block
    float bc1 = a.bc1, bc2 = a.bc2;
    if (a.d_step) {
      const float t = (float)*a.d_step;
      bc1 = 1.f - powf(a.b1, t);
      bc2 = 1.f - powf(a.b2, t);
    }
    s_bc[0] = bc1;
    s_bc[1] = bc2;
  }
  __syncthreads();
  const float bc1 = s_bc[0], bc2 = s_bc[1];
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int q = blockIdx.y;
  if (q == 0) {
    float lr4[4] = {a.lr[0], a.lr[0], a.lr[0], a.lr[1]};
    adam4(a.p_ml, a.g_ml, a.m_ml, a.v_ml, i, lr4, a, bc1, bc2);
  } else if (q == 1) {
    float lr4[4] = {a.lr[2], a.lr[2], a.lr[2], 0.f};
    adam4(a.p_ls, a.g_ls, a.m_ls, a.v_ls, i, lr4, a, bc1, bc2);
  } else if (q == 2) {
    float lr4[4] = {a.lr[3], a.lr[3], a.lr[3], a.lr[3]};
    adam4(a.p_q, a.g_q, a.m_q, a.v_q, i, lr4, a, bc1, bc2);
  } else {
    const int p = q - 3;
    float lr4[4];
    for (int l = 0; l < 4; ++l) lr4[l] = (4 * p + l) < 3 ? a.lr[4] : a.lr[5];
    adam4(a.p_sh, a.g_sh, a.m_sh, a.v_sh, (long long)p * a.n + i, lr4, a, bc1, bc2);
  }
}

__global__ void adam_step_advance_kernel(int* d_step) { *d_step += 1; }

}  // namespace adp

using namespace adp;

extern "C" ADP_API int adp_adam_step(adp_gaussians* param, const adp_gaussians* grad,
                                     adp_gaussians* m, adp_gaussians* v, int32_t step,
                                     int32_t* d_step, const float* lr, float beta1, float beta2,
                                     float eps, adp_stream_t stream) {
  ADP_CHECK_ARG(param && grad && m && v && lr, "NULL argument");
  ADP_CHECK_ARG(d_step || step >= 1, "step must be >= 1");
  ADP_CHECK_ARG(grad->n == param->n && m->n == param->n && v->n == param->n, "size mismatch");
  ADP_CHECK_ARG(param->sh_degree >= 0 && param->sh_degree <= 3, "sh_degree must be 0..3");
  if (param->n == 0) return ADP_OK;
  AdamArgs a;
  a.p_ml = (float4*)param->mean_logit; a.p_ls = (float4*)param->logscale;
  a.p_q = (float4*)param->quat; a.p_sh = (float4*)param->sh;
  a.g_ml = (const float4*)grad->mean_logit; a.g_ls = (const float4*)grad->logscale;
  a.g_q = (const float4*)grad->quat; a.g_sh = (const float4*)grad->sh;
  a.m_ml = (float4*)m->mean_logit; a.m_ls = (float4*)m->logscale;
  a.m_q = (float4*)m->quat; a.m_sh = (float4*)m->sh;
  a.v_ml = (float4*)v->mean_logit; a.v_ls = (float4*)v->logscale;
  a.v_q = (float4*)v->quat; a.v_sh = (float4*)v->sh;
  a.n = param->n;
  a.planes = sh_planes(param->sh_degree);
  for (int k = 0; k < 6; ++k) a.lr[k] = lr[k];
  a.b1 = beta1;
  a.b2 = beta2;
  a.eps = eps;
  a.d_step = d_step;
  a.bc1 = d_step ? 1.f : 1.f - powf(beta1, (float)step);
  a.bc2 = d_step ? 1.f : 1.f - powf(beta2, (float)step);
  adam_kernel<<<dim3(grid_for(param->n, 256), 3 + a.planes), 256, 0, (cudaStream_t)stream>>>(a);
  if (d_step) adam_step_advance_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(d_step);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

// One bias-corrected Adam step (the optimizer the paper leaves unchanged,
// Sec. 5.1) over every parameter plane: one thread per float4 of each plane,
// parameters, moments and gradients each read once and written once. A second
// entry point updates only listed rows (the split candidates, whose updated
// parameters the split plan reads before the compaction applies the step to
// every other row while it copies them).
#include "adam.cuh"

namespace adp {

struct AdamPlanes {
  float4 *p_ml, *p_ls, *p_q, *p_sh;
  const float4 *g_ml, *g_ls, *g_q, *g_sh;
  float4 *m_ml, *m_ls, *m_q, *m_sh;
  float4 *v_ml, *v_ls, *v_q, *v_sh;
  const uint8_t* g_rows;  // optional gradient row mask: 0 = zero gradient, not read
  long long n;
  int planes;
};

// Plane q of Gaussian i: parameter, gradient and moment pointers.
__device__ __forceinline__ void plane_ptrs(const AdamPlanes& a, int q, long long i, float4** P,
                                           const float4** G, float4** M, float4** V) {
  if (q == 0) {
    *P = a.p_ml + i; *G = a.g_ml + i; *M = a.m_ml + i; *V = a.v_ml + i;
  } else if (q == 1) {
    *P = a.p_ls + i; *G = a.g_ls + i; *M = a.m_ls + i; *V = a.v_ls + i;
  } else if (q == 2) {
    *P = a.p_q + i; *G = a.g_q + i; *M = a.m_q + i; *V = a.v_q + i;
  } else {
    const long long o = (long long)(q - 3) * a.n + i;
    *P = a.p_sh + o; *G = a.g_sh + o; *M = a.m_sh + o; *V = a.v_sh + o;
  }
}

__device__ __forceinline__ void adam_at(const AdamPlanes& a, const AdamHyper& h, int q,
                                        long long i) {
  float4 *P, *M, *V;
  const float4* G;
  plane_ptrs(a, q, i, &P, &G, &M, &V);
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 p = *P, m = *M, v = *V;  // all loads first
  const float4 g = (!a.g_rows || a.g_rows[i]) ? *G : z;
  const float2 bc = adam_bias(h);
  float lr4[4];
  adam_plane_lr(h, q, lr4);
  adam_vec4(p, g, m, v, lr4, h, bc);
  *P = p;
  *M = m;
  *V = v;
}

// blockIdx.y selects the plane: 0 mean+logit, 1 log-scale, 2 quaternion,
// 3.. SH planes; each thread updates one float4 of it.
__global__ void adam_kernel(AdamPlanes a, AdamHyper h) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  adam_at(a, h, blockIdx.y, i);
}

// The same update on listed rows only (blockIdx.y selects the plane).
__global__ void adam_rows_kernel(AdamPlanes a, AdamHyper h, const int* rows, long long n_rows) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n_rows) return;
  const int i = rows[t];
  if (i < 0 || i >= a.n) return;
  adam_at(a, h, blockIdx.y, i);
}

__global__ void adam_step_advance_kernel(int* d_step) { *d_step += 1; }

static int adam_check(const adp_gaussians* param, const adp_gaussians* grad,
                      const adp_gaussians* m, const adp_gaussians* v, const float* lr) {
  ADP_CHECK_ARG(param && grad && m && v && lr, "NULL argument");
  ADP_CHECK_ARG(grad->n == param->n && m->n == param->n && v->n == param->n, "size mismatch");
  ADP_CHECK_ARG(param->sh_degree >= 0 && param->sh_degree <= 3, "sh_degree must be 0..3");
  return ADP_OK;
}

static AdamPlanes adam_planes(adp_gaussians* param, const adp_gaussians* grad, adp_gaussians* m,
                              adp_gaussians* v) {
  AdamPlanes a;
  a.p_ml = (float4*)param->mean_logit; a.p_ls = (float4*)param->logscale;
  a.p_q = (float4*)param->quat; a.p_sh = (float4*)param->sh;
  a.g_ml = (const float4*)grad->mean_logit; a.g_ls = (const float4*)grad->logscale;
  a.g_q = (const float4*)grad->quat; a.g_sh = (const float4*)grad->sh;
  a.m_ml = (float4*)m->mean_logit; a.m_ls = (float4*)m->logscale;
  a.m_q = (float4*)m->quat; a.m_sh = (float4*)m->sh;
  a.v_ml = (float4*)v->mean_logit; a.v_ls = (float4*)v->logscale;
  a.v_q = (float4*)v->quat; a.v_sh = (float4*)v->sh;
  a.g_rows = grad->rows;
  a.n = param->n;
  a.planes = sh_planes(param->sh_degree);
  return a;
}

}  // namespace adp

using namespace adp;

extern "C" ADP_API int adp_adam_step(adp_gaussians* param, const adp_gaussians* grad,
                                     adp_gaussians* m, adp_gaussians* v, int32_t step,
                                     int32_t* d_step, const float* lr, float beta1, float beta2,
                                     float eps, adp_stream_t stream) {
  int rc = adam_check(param, grad, m, v, lr);
  if (rc) return rc;
  ADP_CHECK_ARG(d_step || step >= 1, "step must be >= 1");
  if (param->n == 0) return ADP_OK;
  AdamPlanes a = adam_planes(param, grad, m, v);
  AdamHyper h = adam_hyper(lr, beta1, beta2, eps, step, d_step);
  cudaStream_t st = (cudaStream_t)stream;
  adam_kernel<<<dim3(grid_for(param->n, 256), 3 + a.planes), 256, 0, st>>>(a, h);
  if (d_step) adam_step_advance_kernel<<<1, 1, 0, st>>>(d_step);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

extern "C" ADP_API int adp_adam_step_rows(adp_gaussians* param, const adp_gaussians* grad,
                                          adp_gaussians* m, adp_gaussians* v, const int32_t* rows,
                                          int64_t n_rows, int32_t step, const int32_t* d_step,
                                          const float* lr, float beta1, float beta2, float eps,
                                          adp_stream_t stream) {
  int rc = adam_check(param, grad, m, v, lr);
  if (rc) return rc;
  ADP_CHECK_ARG(d_step || step >= 1, "step must be >= 1");
  ADP_CHECK_ARG(n_rows >= 0 && n_rows <= param->n, "n_rows out of range");
  ADP_CHECK_ARG(n_rows == 0 || rows, "NULL rows");
  if (n_rows == 0) return ADP_OK;
  AdamPlanes a = adam_planes(param, grad, m, v);
  AdamHyper h = adam_hyper(lr, beta1, beta2, eps, step, d_step);
  // blocks of 128 threads: 0.034 against 0.035 ms for 256 (100k candidate rows)
  adam_rows_kernel<<<dim3(grid_for(n_rows, 128), 3 + a.planes), 128, 0, (cudaStream_t)stream>>>(
      a, h, rows, n_rows);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

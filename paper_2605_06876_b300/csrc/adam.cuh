// The bias-corrected Adam update (the baselines' optimizer, which the paper
// leaves unchanged, Sec. 5.1) on one float4 of a parameter plane, shared by the
// plain Adam kernels and by the compaction that applies the step while it
// copies, so that both give bit-identical results.
#pragma once

#include <cmath>

#include "common.cuh"

namespace adp {

struct AdamHyper {
  float lr[6];  // mean, opacity logit, log-scale, quaternion, SH DC, SH rest
  float b1, b2, eps;
  float ln_b1, ln_b2;  // log(beta), for the bias corrections
  int step;            // the step number t, unless d_step is set
  const int* d_step;   // if set, t is read here
};

// Reciprocals of the bias corrections 1 - beta^t = -expm1(t log beta) (no
// cancellation for small t), computed by every thread (no barrier, no dependent
// preamble before the streaming loads) and identically for a host-given and a
// device-held t.
__device__ __forceinline__ float2 adam_bias(const AdamHyper& h) {
  const float t = (float)(h.d_step ? *h.d_step : h.step);
  return make_float2(1.f / -expm1f(t * h.ln_b1), 1.f / -expm1f(t * h.ln_b2));
}

// One element. Multiplies by the reciprocals (and by a correctly rounded
// reciprocal of sqrt(v^) + eps) instead of dividing: IEEE divisions per element
// would make this streaming update compute-bound.
__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, float lr,
                                      const AdamHyper& h, float2 ibc) {
  // explicit fused multiply-adds: the same rounding in every kernel that inlines this
  m = fmaf(h.b1, m, (1.f - h.b1) * g);
  v = fmaf(h.b2, v, ((1.f - h.b2) * g) * g);
  const float mh = m * ibc.x, vh = v * ibc.y;
  p -= (lr * mh) * __frcp_rn(sqrtf(vh) + h.eps);
}

// Learning rates of the four lanes of plane q: 0 mean + logit, 1 log-scale
// (+ pad), 2 quaternion, 3.. SH (the first three floats are the DC colour).
__device__ __forceinline__ void adam_plane_lr(const AdamHyper& h, int q, float* lr4) {
  if (q == 0) {
    lr4[0] = lr4[1] = lr4[2] = h.lr[0];
    lr4[3] = h.lr[1];
  } else if (q == 1) {
    lr4[0] = lr4[1] = lr4[2] = h.lr[2];
    lr4[3] = 0.f;
  } else if (q == 2) {
    lr4[0] = lr4[1] = lr4[2] = lr4[3] = h.lr[3];
  } else {
#pragma unroll
    for (int l = 0; l < 4; ++l) lr4[l] = (4 * (q - 3) + l) < 3 ? h.lr[4] : h.lr[5];
  }
}

__device__ __forceinline__ void adam_vec4(float4& p, float4 g, float4& m, float4& v,
                                          const float* lr4, const AdamHyper& h, float2 bc) {
  adam1(p.x, g.x, m.x, v.x, lr4[0], h, bc);
  adam1(p.y, g.y, m.y, v.y, lr4[1], h, bc);
  adam1(p.z, g.z, m.z, v.z, lr4[2], h, bc);
  adam1(p.w, g.w, m.w, v.w, lr4[3], h, bc);
}

// Host side: hyperparameters of one call (step >= 1 unless d_step is given).
inline AdamHyper adam_hyper(const float* lr, float beta1, float beta2, float eps, int step,
                            const int* d_step) {
  AdamHyper h;
  for (int k = 0; k < 6; ++k) h.lr[k] = lr[k];
  h.b1 = beta1;
  h.b2 = beta2;
  h.eps = eps;
  h.d_step = d_step;
  h.step = step;
  h.ln_b1 = (float)log((double)beta1);
  h.ln_b2 = (float)log((double)beta2);
  return h;
}

}  // namespace adp

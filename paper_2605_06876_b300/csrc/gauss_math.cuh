// Device math shared by the forward and backward kernels: quaternion rotation,
// the real SH basis (3DGS sign convention) and its gradient, and the staged
// per-Gaussian form and alpha evaluation that forward and backward share.
#pragma once

#include "common.cuh"

namespace adp {

// Real SH normalisation constants up to degree 3 (3DGS basis signs).
#define SHC0 0.28209479177387814f
#define SHC1 0.4886025119029199f
#define SHC2_0 1.0925484305920792f
#define SHC2_2 0.31539156525252005f
#define SHC2_4 0.5462742152960396f
#define SHC3_0 0.5900435899266435f
#define SHC3_1 2.890611442640554f
#define SHC3_2 0.4570457994644658f
#define SHC3_3 0.3731763325901154f
#define SHC3_5 1.445305721320277f

struct Mat3 {
  float m[9];
};

// Rotation (row-major) of the normalised quaternion q = (w, x, y, z).
__device__ __forceinline__ Mat3 rot_of_quat(float w, float x, float y, float z) {
  Mat3 R;
  R.m[0] = 1.f - 2.f * (y * y + z * z);
  R.m[1] = 2.f * (x * y - w * z);
  R.m[2] = 2.f * (x * z + w * y);
  R.m[3] = 2.f * (x * y + w * z);
  R.m[4] = 1.f - 2.f * (x * x + z * z);
  R.m[5] = 2.f * (y * z - w * x);
  R.m[6] = 2.f * (x * z - w * y);
  R.m[7] = 2.f * (y * z + w * x);
  R.m[8] = 1.f - 2.f * (x * x + y * y);
  return R;
}

// Basis values Y[k], k < (deg+1)^2, at unit direction (x, y, z).
__device__ __forceinline__ void sh_eval_basis(int deg, float x, float y, float z, float* Y) {
  Y[0] = SHC0;
  if (deg < 1) return;
  Y[1] = -SHC1 * y;
  Y[2] = SHC1 * z;
  Y[3] = -SHC1 * x;
  if (deg < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = SHC2_0 * x * y;
  Y[5] = -SHC2_0 * y * z;
  Y[6] = SHC2_2 * (2.f * zz - xx - yy);
  Y[7] = -SHC2_0 * x * z;
  Y[8] = SHC2_4 * (xx - yy);
  if (deg < 3) return;
  Y[9] = -SHC3_0 * y * (3.f * xx - yy);
  Y[10] = SHC3_1 * x * y * z;
  Y[11] = -SHC3_2 * y * (4.f * zz - xx - yy);
  Y[12] = SHC3_3 * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -SHC3_2 * x * (4.f * zz - xx - yy);
  Y[14] = SHC3_5 * z * (xx - yy);
  Y[15] = -SHC3_0 * x * (xx - 3.f * yy);
}

// Partial derivatives of the basis with respect to the (unnormalised
// coordinates of the) direction: dY[k] = (dY/dx, dY/dy, dY/dz).
__device__ __forceinline__ void sh_eval_basis_grad(int deg, float x, float y, float z,
                                                   float3* dY) {
  dY[0] = make_float3(0.f, 0.f, 0.f);
  if (deg < 1) return;
  dY[1] = make_float3(0.f, -SHC1, 0.f);
  dY[2] = make_float3(0.f, 0.f, SHC1);
  dY[3] = make_float3(-SHC1, 0.f, 0.f);
  if (deg < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  dY[4] = make_float3(SHC2_0 * y, SHC2_0 * x, 0.f);
  dY[5] = make_float3(0.f, -SHC2_0 * z, -SHC2_0 * y);
  dY[6] = make_float3(-2.f * SHC2_2 * x, -2.f * SHC2_2 * y, 4.f * SHC2_2 * z);
  dY[7] = make_float3(-SHC2_0 * z, 0.f, -SHC2_0 * x);
  dY[8] = make_float3(2.f * SHC2_4 * x, -2.f * SHC2_4 * y, 0.f);
  if (deg < 3) return;
  dY[9] = make_float3(-SHC3_0 * 6.f * x * y, -SHC3_0 * (3.f * xx - 3.f * yy), 0.f);
  dY[10] = make_float3(SHC3_1 * y * z, SHC3_1 * x * z, SHC3_1 * x * y);
  dY[11] = make_float3(SHC3_2 * 2.f * x * y, -SHC3_2 * (4.f * zz - xx - 3.f * yy),
                       -SHC3_2 * 8.f * y * z);
  dY[12] = make_float3(-SHC3_3 * 6.f * x * z, -SHC3_3 * 6.f * y * z,
                       SHC3_3 * (6.f * zz - 3.f * xx - 3.f * yy));
  dY[13] = make_float3(-SHC3_2 * (4.f * zz - 3.f * xx - yy), SHC3_2 * 2.f * x * y,
                       -SHC3_2 * 8.f * x * z);
  dY[14] = make_float3(SHC3_5 * 2.f * x * z, -SHC3_5 * 2.f * y * z, SHC3_5 * (xx - yy));
  dY[15] = make_float3(-SHC3_0 * (3.f * xx - 3.f * yy), SHC3_0 * 6.f * x * y, 0.f);
}

// g = sum_k w[k] dY[k] (the basis partials of sh_eval_basis_grad weighted by w),
// accumulated term by term in k order without forming the partials.
__device__ __forceinline__ void sh_grad_dot(int deg, float x, float y, float z, const float* w,
                                            float* g) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (deg >= 1) {
    gy = fmaf(w[1], -SHC1, gy);
    gz = fmaf(w[2], SHC1, gz);
    gx = fmaf(w[3], -SHC1, gx);
  }
  if (deg >= 2) {
    gx = fmaf(w[4], SHC2_0 * y, gx);
    gy = fmaf(w[4], SHC2_0 * x, gy);
    gy = fmaf(w[5], -SHC2_0 * z, gy);
    gz = fmaf(w[5], -SHC2_0 * y, gz);
    gx = fmaf(w[6], -2.f * SHC2_2 * x, gx);
    gy = fmaf(w[6], -2.f * SHC2_2 * y, gy);
    gz = fmaf(w[6], 4.f * SHC2_2 * z, gz);
    gx = fmaf(w[7], -SHC2_0 * z, gx);
    gz = fmaf(w[7], -SHC2_0 * x, gz);
    gx = fmaf(w[8], 2.f * SHC2_4 * x, gx);
    gy = fmaf(w[8], -2.f * SHC2_4 * y, gy);
  }
  if (deg >= 3) {
    const float xx = x * x, yy = y * y, zz = z * z;
    gx = fmaf(w[9], -SHC3_0 * 6.f * x * y, gx);
    gy = fmaf(w[9], -SHC3_0 * (3.f * xx - 3.f * yy), gy);
    gx = fmaf(w[10], SHC3_1 * y * z, gx);
    gy = fmaf(w[10], SHC3_1 * x * z, gy);
    gz = fmaf(w[10], SHC3_1 * x * y, gz);
    gx = fmaf(w[11], SHC3_2 * 2.f * x * y, gx);
    gy = fmaf(w[11], -SHC3_2 * (4.f * zz - xx - 3.f * yy), gy);
    gz = fmaf(w[11], -SHC3_2 * 8.f * y * z, gz);
    gx = fmaf(w[12], -SHC3_3 * 6.f * x * z, gx);
    gy = fmaf(w[12], -SHC3_3 * 6.f * y * z, gy);
    gz = fmaf(w[12], SHC3_3 * (6.f * zz - 3.f * xx - 3.f * yy), gz);
    gx = fmaf(w[13], -SHC3_2 * (4.f * zz - 3.f * xx - yy), gx);
    gy = fmaf(w[13], SHC3_2 * 2.f * x * y, gy);
    gz = fmaf(w[13], -SHC3_2 * 8.f * x * z, gz);
    gx = fmaf(w[14], SHC3_5 * 2.f * x * z, gx);
    gy = fmaf(w[14], -SHC3_5 * 2.f * y * z, gy);
    gz = fmaf(w[14], SHC3_5 * (xx - yy), gz);
    gx = fmaf(w[15], -SHC3_0 * (3.f * xx - 3.f * yy), gx);
    gy = fmaf(w[15], SHC3_0 * 6.f * x * y, gy);
  }
  g[0] = gx;
  g[1] = gy;
  g[2] = gz;
}

// Reads SH float k*3+ch of Gaussian i from the float4 planes.
__device__ __forceinline__ float sh_coef(const float* sh, long long n, long long i, int f) {
  return sh[((long long)(f >> 2) * n + i) * 4 + (f & 3)];
}

// A projected Gaussian as the compositing loops stage it in shared memory:
// 2D mean, the conic scaled into log2 units (a = -A log2(e) / 2, b = -B log2(e),
// c = -C log2(e) / 2), log2 of the opacity, its reciprocal, the colour, the id,
// and the rows its alpha ellipse can reach.
struct Staged {
  float4 g0;  // mx, my, a, b
  float4 g1;  // c, log2(o), r, g
  float4 g2;  // blue, id (int bits), 1/o, 0
  float2 y;   // lowest and highest image row the ellipse reaches
};

constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ Staged stage_gaussian(float4 xyod, float4 conic, float4 rgb, int id,
                                                 float alpha_min) {
  Staged s;
  const float o = xyod.z;
  s.g0 = make_float4(xyod.x, xyod.y, -0.5f * kLog2e * conic.x, -kLog2e * conic.y);
  s.g1 = make_float4(-0.5f * kLog2e * conic.z, __log2f(o), rgb.x, rgb.y);
  s.g2 = make_float4(rgb.z, __int_as_float(id), 1.f / o, 0.f);
  // rows of the ellipse o exp(-d^T C d / 2) >= alpha_min: |dy| <= sqrt(k S_yy) with
  // S_yy = A / det(C), k = 2 ln(o / alpha_min); widened so the skip is conservative
  const float det = conic.x * conic.z - conic.y * conic.y;
  const float k = fmaxf(2.f * __logf(o / alpha_min), 0.f);
  const float hy = sqrtf(k * conic.x / det) * 1.001f + 0.01f;
  s.y = make_float2(xyod.y - hy, xyod.y + hy);
  return s;
}

// log2 of alpha_raw = o exp(-d^T C d / 2) at a pixel, with d = mean - pixel,
// written as q = dx (a dx + b dy) + (c dy^2 + log2 o) in the staged log2 conic
// (a, b, c): the bracketed term and b dy depend only on the pixel row, so a
// thread computes them once for its pixels of one row. Forward and backward
// both evaluate q through these two functions, and the value of a pixel does not
// depend on which thread computes it, so their decisions agree bit for bit for
// every tile shape.
struct RowQ {
  float dy, bdy, e;
};

__device__ __forceinline__ RowQ row_q(const float4& g0, const float4& g1, float py) {
  RowQ r;
  r.dy = g0.y - py;
  r.bdy = g0.w * r.dy;
  r.e = fmaf(g1.x * r.dy, r.dy, g1.y);
  return r;
}

__device__ __forceinline__ float pix_q(const float4& g0, const RowQ& r, float px, float* dx) {
  *dx = g0.x - px;
  return fmaf(*dx, fmaf(g0.z, *dx, r.bdy), r.e);
}

// 2^x and 1/x from the special-function unit (relative error about 2^-22;
// subnormal results flush to zero, which only ever meets alphas already below
// the 1/255 cut).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Pixel layout of a 256-pixel tile with PX horizontally adjacent pixels per
// thread (PX divides every supported tile width).
template <int PX>
struct TileLanes {
  static constexpr int THREADS = 256 / PX;
  static constexpr int WARP_PIXELS = 32 * PX;
};

}  // namespace adp

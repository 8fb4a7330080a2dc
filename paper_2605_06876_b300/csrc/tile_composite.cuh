// Per-tile compositing loops shared by the one-stage kernels (adp_render,
// adp_render_backward) and the fused batched kernel (adp_train_step_batched):
// the forward walk of Eq. 1 with the dominant Gaussian of Eq. 5, and the
// backward walk that recovers the transmittance from its final value. Both
// stage the tile's depth-sorted list through shared memory STAGE Gaussians at a
// time in the form of stage_gaussian (alpha in log2 units, the rows each
// ellipse reaches); a warp skips a Gaussian that reaches none of its rows; the
// per-pixel update is branch-free on horizontal pixel pairs with the packed
// two-lane FP32 instructions of sm_100+ (each lane rounds like the scalar
// instruction). Forward and backward evaluate every alpha through row_q/pix_q
// with the same operations, so their decisions agree bit for bit whichever
// kernel runs them.
#pragma once

#include "gauss_math.cuh"

namespace adp {

// Scale that saturates any positive alpha or weight difference the rules allow
// to exactly 1 (__saturatef(x * kSat) is 0 for x <= 0 and 1 for x >= 2^-126).
constexpr float kSat = 8.507059173023462e37f;  // 2^126
// Minus the x coordinate given to a pixel that has stopped: its exponent q is then
// -inf or hugely negative, so the alpha test fails without a separate flag.
constexpr float kGone = -1e30f;

// The staging buffers of one block (STAGE Gaussians each), declared by the kernel.
struct StageBuf {
  float4* g0;
  float4* g1;
  float4* g2;
  float2* y;
};

// The tile a thread works on and its pixels: PX horizontally adjacent pixels
// starting at (px0, py).
template <int PX>
struct TileGeom {
  int v, W, H, px0, py;
  float fy, wy0, wy1;  // the thread's row; the first and last rows of its warp
  int2 range;          // the tile's list in the instance array
  long long rec_base;  // first record of the view
  long long pix_base;  // first pixel of the view
};

template <int PX>
__device__ __forceinline__ TileGeom<PX> tile_geom(const CamSet& cs, const int2* ranges,
                                                  long long n, int tile) {
  TileGeom<PX> t;
  t.v = view_of_tile(cs, tile);
  const int lt = tile - cs.tile_base[t.v];
  const int txs = cs.tiles_x[t.v];
  t.W = cs.cam[t.v].width;
  t.H = cs.cam[t.v].height;
  t.range = ranges[tile];
  t.rec_base = (long long)t.v * n;
  t.pix_base = cs.pix_base[t.v];
  const int tx0 = (lt % txs) * cs.tile_w, ty0 = (lt / txs) * cs.tile_h;
  const int warp = threadIdx.x >> 5;
  t.wy0 = (float)(ty0 + (TileLanes<PX>::WARP_PIXELS * warp) / cs.tile_w);
  t.wy1 = (float)(ty0 + (TileLanes<PX>::WARP_PIXELS * (warp + 1) - 1) / cs.tile_w);
  const int li0 = PX * (int)threadIdx.x;
  t.px0 = tx0 + li0 % cs.tile_w;
  t.py = ty0 + li0 / cs.tile_w;
  t.fy = (float)t.py;
  return t;
}

template <int PX>
__device__ __forceinline__ bool pixel_in(const TileGeom<PX>& t, int h) {
  return t.px0 + h < t.W && t.py < t.H;
}

// Stages list entries [b0, b0 + cnt) of the tile into the buffers (all threads).
template <int NT>
__device__ __forceinline__ void stage_batch(const float4* xyod, const float4* conic,
                                            const float4* rgb, const int* inst, int first,
                                            long long rec_base, float alpha_min, int cnt,
                                            const StageBuf& sb) {
  for (int j = (int)threadIdx.x; j < cnt; j += NT) {
    const int id = inst[first + j];
    const long long r = rec_base + id;
    const Staged g = stage_gaussian(xyod[r], conic[r], rgb[r], id, alpha_min);
    sb.g0[j] = g.g0;
    sb.g1[j] = g.g1;
    sb.g2[j] = g.g2;
    sb.y[j] = g.y;
  }
}

struct CompositeConsts {
  float alpha_min, alpha_max, t_min, log2_alpha_min;
};

// Per-thread result of the forward walk: per pixel pair the transmittance and
// the colour sums; per pixel the dominant Gaussian, the number of blended
// Gaussians and one past the list position of the last one.
template <int PX>
struct FwdOut {
  float2 T[PX / 2], c0[PX / 2], c1[PX / 2], c2[PX / 2];
  int dom[PX], ncon[PX], last[PX];
};

// Front to back over the tile's list (Eq. 1): alpha = min(alpha_max, o exp(q)),
// skipped below alpha_min, stop before blending once T (1 - alpha) < t_min. The
// contributor count, the last blended position and the position of the dominant
// weight T alpha (Eq. 5, strictly larger wins, so the earliest of equal weights)
// are kept as exact small floats within a staged batch (positions below STAGE)
// through saturating multiplies on the FMA pipe, and folded into integers when
// the batch ends. A warp leaves the batch once all its pixels have stopped
// (checked every fourth Gaussian) and a block-wide vote ends the tile.
template <int PX, int STAGE>
__device__ __forceinline__ void fwd_tile(const float4* xyod, const float4* conic,
                                         const float4* rgb, const int* inst,
                                         const TileGeom<PX>& t, const CompositeConsts& kc,
                                         const StageBuf& sb, FwdOut<PX>& o) {
  static_assert(PX % 2 == 0, "pixels are processed in pairs");
  constexpr int NT = TileLanes<PX>::THREADS;
  constexpr int NP = PX / 2;
  const int count = t.range.y - t.range.x;
  const float amax = kc.alpha_max, tmin = kc.t_min, l2amin = kc.log2_alpha_min;
  const float2 one2 = make_float2(1.f, 1.f), neg2 = make_float2(-1.f, -1.f);
  float2 best[NP], nfx[NP];
  float2 ncf[NP], lastf[NP], domf[NP];  // per batch: blends, last blended k + 1, dominant k
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    o.T[j] = one2;
    o.c0[j] = o.c1[j] = o.c2[j] = make_float2(0.f, 0.f);
    best[j] = make_float2(0.f, 0.f);  // every blended weight T alpha is > 0
    ncf[j] = lastf[j] = make_float2(0.f, 0.f);
    domf[j] = neg2;
    float n2[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int h = 2 * j + e;
      o.dom[h] = -1;
      o.ncon[h] = 0;
      o.last[h] = 0;
      n2[e] = pixel_in(t, h) ? -(float)(t.px0 + h) : kGone;
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
    const int cnt = min(STAGE, count - b0);
    stage_batch<NT>(xyod, conic, rgb, inst, t.range.x + b0, t.rec_base, kc.alpha_min, cnt, sb);
    __syncthreads();
    if (__all_sync(0xffffffffu, thread_done())) continue;
    float kfl = 0.f;  // k as a float, advanced with k (no conversion per Gaussian)
    for (int k = 0; k < cnt; ++k, kfl += 1.f) {
      if ((k & 3) == 0 && __all_sync(0xffffffffu, thread_done())) break;
      const float2 yr = sb.y[k];
      if (yr.y < t.wy0 || yr.x > t.wy1) continue;  // warp-uniform: no row of this warp reached
      const float4 g0 = sb.g0[k], g1 = sb.g1[k], g2 = sb.g2[k];
      const RowQ rq = row_q(g0, g1, t.fy);
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
        const float2 test = __fmul2_rn(o.T[j], __ffma2_rn(al, neg2, one2));
        if (test.x < tmin) {
          al.x = 0.f;
          nfx[j].x = kGone;
        }
        if (test.y < tmin) {
          al.y = 0.f;
          nfx[j].y = kGone;
        }
        const float2 w = __fmul2_rn(o.T[j], al);
        o.T[j] = __fmul2_rn(o.T[j], __ffma2_rn(al, neg2, one2));
        o.c0[j] = __ffma2_rn(w, cr, o.c0[j]);
        o.c1[j] = __ffma2_rn(w, cg, o.c1[j]);
        o.c2[j] = __ffma2_rn(w, cb, o.c2[j]);
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
        o.ncon[h] += (int)nc2[e];
        if (l2[e] > 0.f) o.last[h] = b0 + (int)l2[e];
        if (d2[e] >= 0.f) o.dom[h] = __float_as_int(sb.g2[(int)d2[e]].y);
      }
      ncf[j] = lastf[j] = make_float2(0.f, 0.f);
      domf[j] = neg2;
    }
  }
}

// Reduce-scatter of eight per-lane values across the warp by recursive halving:
// at each of three levels a lane keeps half of its values and sends the other
// half to its partner, then two plain steps finish. Lane l ends with the warp
// total of value index ((l >> 4) & 1) * 4 + ((l >> 3) & 1) * 2 + ((l >> 2) & 1)
// (the same in all four lanes of its quad): nine shuffles instead of forty.
__device__ __forceinline__ float reduce_scatter8(const float* v, int* idx) {
  const int lane = threadIdx.x & 31;
  const bool b16 = (lane >> 4) & 1, b8 = (lane >> 3) & 1, b4 = (lane >> 2) & 1;
  float u[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float keep = b16 ? v[4 + i] : v[i];
    float send = b16 ? v[i] : v[4 + i];
    u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float w[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    float keep = b8 ? u[2 + i] : u[i];
    float send = b8 ? u[i] : u[2 + i];
    w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float keep = b4 ? w[1] : w[0];
  float send = b4 ? w[0] : w[1];
  float x = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  *idx = (b16 ? 4 : 0) + (b8 ? 2 : 0) + (b4 ? 1 : 0);
  return x;
}

// Per-thread input of the backward walk: per pixel pair the final transmittance
// and dL/dpixel; per pixel one past the list position of its last blended
// Gaussian (0 for a pixel outside the image).
template <int PX>
struct BwdIn {
  float2 T[PX / 2], G0[PX / 2], G1[PX / 2], G2[PX / 2];
  int last[PX];
};

// Back to front over the tile's list from the last blended position of any of
// its pixels. The transmittance before each Gaussian is recovered as
// T / (1 - alpha) and the colour behind it by R <- R + alpha (c - R) from the
// background. Per Gaussian the warp reduces its pixels' moments of
// k = dL/dalpha * alpha (alpha below the clamp only) with d = mean - pixel --
// S = sum k, Sx = sum k dx, Sy, Sxx, Sxy, Syy -- and the colour gradient
// sum T alpha dL/dpixel, then adds them to g2d[3 (rec_base + id) ..] with one
// reduce-scatter and nine scalar atomics. With alpha = o exp(power) they give
// dL/do = S / o, dL/dA = -Sxx / 2, dL/dB = -Sxy, dL/dC = -Syy / 2 and
// dL/dmean = -(A Sx + B Sy, B Sx + C Sy), applied by the per-Gaussian pass. A
// thread's pixels share dy, so Sy, Sxy, Syy follow from its S and Sx.
// s_maxlast: one shared int of the block.
template <int PX, int STAGE>
__device__ __forceinline__ void bwd_tile(const float4* xyod, const float4* conic,
                                         const float4* rgb, const int* inst,
                                         const TileGeom<PX>& t, const CompositeConsts& kc,
                                         const float* bg, const StageBuf& sb, int* s_maxlast,
                                         BwdIn<PX>& in, float4* g2d) {
  static_assert(PX % 2 == 0, "pixels are processed in pairs");
  constexpr int NT = TileLanes<PX>::THREADS;
  constexpr int NP = PX / 2;
  const float amax = kc.alpha_max, l2amin = kc.log2_alpha_min;
  const float2 one2 = make_float2(1.f, 1.f), neg2 = make_float2(-1.f, -1.f);
  float2 R0[NP], R1[NP], R2[NP], npx[NP];
  int warp_last = 0;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    R0[j] = make_float2(bg[0], bg[0]);
    R1[j] = make_float2(bg[1], bg[1]);
    R2[j] = make_float2(bg[2], bg[2]);
    npx[j] = make_float2(-(float)(t.px0 + 2 * j), -(float)(t.px0 + 2 * j + 1));
    warp_last = max(warp_last, max(in.last[2 * j], in.last[2 * j + 1]));
  }
  if (threadIdx.x == 0) *s_maxlast = 0;
  __syncthreads();
  for (int o = 16; o > 0; o >>= 1)
    warp_last = max(warp_last, __shfl_xor_sync(0xffffffffu, warp_last, o));
  if ((threadIdx.x & 31) == 0 && warp_last > 0) atomicMax(s_maxlast, warp_last);
  __syncthreads();
  const int end = *s_maxlast;
  const int lane = threadIdx.x & 31;
  for (int b1 = end; b1 > 0; b1 -= STAGE) {
    const int b0 = b1 - STAGE > 0 ? b1 - STAGE : 0;
    __syncthreads();
    stage_batch<NT>(xyod, conic, rgb, inst, t.range.x + b0, t.rec_base, kc.alpha_min, b1 - b0,
                    sb);
    __syncthreads();
    const int kmax = min(b1, warp_last) - b0;  // warp-uniform
    for (int k = kmax - 1; k >= 0; --k) {
      const float2 yr = sb.y[k];
      if (yr.y < t.wy0 || yr.x > t.wy1) continue;  // warp-uniform: no row of this warp reached
      const float4 g0 = sb.g0[k], g1 = sb.g1[k], g2 = sb.g2[k];
      const RowQ rq = row_q(g0, g1, t.fy);
      const int pos = b0 + k;
      const float2 mx = make_float2(g0.x, g0.x), qa = make_float2(g0.z, g0.z);
      const float2 qb = make_float2(rq.bdy, rq.bdy), qe = make_float2(rq.e, rq.e);
      const float2 cr = make_float2(g1.z, g1.z), cg = make_float2(g1.w, g1.w);
      const float2 cb = make_float2(g2.x, g2.x);
      float2 S = make_float2(0.f, 0.f), Sx = S, Sxx = S, C0 = S, C1 = S, C2 = S;
      bool hit = false;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        // q = dx (a dx + b dy) + e, the same operations as pix_q
        const float2 dx = __fadd2_rn(mx, npx[j]);
        const float2 q = __ffma2_rn(dx, __ffma2_rn(qa, dx, qb), qe);
        const bool p0 = pos < in.last[2 * j] && q.x >= l2amin;  // blended in the forward
        const bool p1 = pos < in.last[2 * j + 1] && q.y >= l2amin;
        hit = hit || p0 || p1;
        const float ar0 = ex2_approx(q.x), ar1 = ex2_approx(q.y);
        const float2 al = make_float2(p0 ? fminf(amax, ar0) : 0.f, p1 ? fminf(amax, ar1) : 0.f);
        const float2 om = __ffma2_rn(al, neg2, one2);  // 1 - alpha
        // transmittance before this Gaussian
        const float2 Tj = __fmul2_rn(in.T[j], make_float2(rcp_approx(om.x), rcp_approx(om.y)));
        const float2 d0 = __ffma2_rn(R0[j], neg2, cr);  // colour minus the colour behind
        const float2 d1 = __ffma2_rn(R1[j], neg2, cg);
        const float2 d2 = __ffma2_rn(R2[j], neg2, cb);
        const float2 dal = __fmul2_rn(
            Tj, __ffma2_rn(in.G0[j], d0, __ffma2_rn(in.G1[j], d1, __fmul2_rn(in.G2[j], d2))));
        const float2 wgt = __fmul2_rn(Tj, al);
        C0 = __ffma2_rn(wgt, in.G0[j], C0);
        C1 = __ffma2_rn(wgt, in.G1[j], C1);
        C2 = __ffma2_rn(wgt, in.G2[j], C2);
        R0[j] = __ffma2_rn(al, d0, R0[j]);
        R1[j] = __ffma2_rn(al, d1, R1[j]);
        R2[j] = __ffma2_rn(al, d2, R2[j]);
        in.T[j] = Tj;
        // dL/dalpha * alpha, zero through the clamp (alpha = 0 where not blended)
        float2 kk = __fmul2_rn(dal, al);
        kk.x = ar0 <= amax ? kk.x : 0.f;
        kk.y = ar1 <= amax ? kk.y : 0.f;
        S = __fadd2_rn(S, kk);
        const float2 tt = __fmul2_rn(dx, kk);
        Sx = __fadd2_rn(Sx, tt);
        Sxx = __ffma2_rn(dx, tt, Sxx);
      }
      if (__ballot_sync(0xffffffffu, hit)) {
        const float dy = rq.dy;
        const float s1 = S.x + S.y, sx = Sx.x + Sx.y;
        float vals[8] = {s1, sx, dy * s1, Sxx.x + Sxx.y, dy * sx, dy * dy * s1, C0.x + C0.y,
                         C1.x + C1.y};
        int idx;
        float sum = reduce_scatter8(vals, &idx);
        float cbs = warp_sum(C2.x + C2.y);
        int id = __float_as_int(g2.y);
        float* gp = reinterpret_cast<float*>(g2d + 3 * (t.rec_base + id));
        if ((lane & 3) == 0) atomicAdd(gp + idx, sum);
        if (lane == 0) atomicAdd(gp + 8, cbs);
      }
    }
  }
}

}  // namespace adp

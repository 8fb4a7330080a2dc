// Candidate selection of the adaptive density control (Sec. 3, Eq. 2): with the
// average image-space gradient g_i = accum_i / visits_i, Gaussians with
// g_i >= tau_g are split when their largest scale exceeds tau_s and cloned
// otherwise. Both decisions are made in float32 on the stored values: g_i by one
// correctly rounded division, the scale test on the log-scales against
// ln(tau_s) rounded to float32 (exp is increasing, so this is max s > tau_s
// without rounding an exponential). One decoupled-look-back scan with both
// counts packed in one 64-bit word (splits in the low half, clones in the high
// half; n < 2^31 keeps them apart) writes both id lists in ascending id order.
#include <cmath>

#include "common.cuh"

namespace adp {

__device__ __forceinline__ unsigned densify_class(const float* accum, const int* visits,
                                                  const float4* logscale, long long i,
                                                  float tau_g, float ln_tau_s) {
  const int nv = visits[i];
  const float gi = nv > 0 ? __fdiv_rn(accum[i], (float)nv) : 0.f;
  if (!(gi >= tau_g)) return 0u;
  const float4 ls = logscale[i];
  const float smax = fmaxf(ls.x, fmaxf(ls.y, ls.z));
  return smax > ln_tau_s ? 1u : 2u;  // 1 split, 2 clone
}

// The two counts from the packed scan total; both 0 if the scan gave up a wait
// (its lists may have gaps), so the tail pass turns every entry into -1.
__global__ void densify_counts_kernel(long long* packed, const unsigned long long* err,
                                      int64_t* d_counts) {
  if (*err != 0ull) *packed = 0;
  const unsigned long long t = (unsigned long long)*packed;
  d_counts[0] = (int64_t)(t & 0xffffffffull);
  d_counts[1] = (int64_t)(t >> 32);
}

// Entries past each list's count become -1 (the lists can then be passed whole,
// with their capacity as the candidate count, to calls that skip -1 entries).
__global__ void densify_tail_kernel(const long long* packed, long long n, int32_t* split_ids,
                                    int32_t* clone_ids) {
  const unsigned long long t = (unsigned long long)*packed;
  const long long ns = (long long)(t & 0xffffffffull), nc = (long long)(t >> 32);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (i >= ns) split_ids[i] = -1;
    if (i >= nc) clone_ids[i] = -1;
  }
}

}  // namespace adp

using namespace adp;

extern "C" ADP_API size_t adp_densify_select_workspace_size(int64_t n) {
  if (n < 0) return 0;
  return scan_workspace_bytes(n > 0 ? n : 1) + carve_bytes<long long>(1);
}

extern "C" ADP_API int adp_densify_select(const float* grad2d_accum, const int32_t* grad2d_visits,
                                          const adp_gaussians* g, float tau_g, float tau_s,
                                          int32_t* split_ids, int32_t* clone_ids,
                                          int64_t* d_counts, void* ws, size_t ws_bytes,
                                          int32_t* d_status, adp_stream_t stream) {
  ADP_CHECK_ARG(g && d_counts, "NULL argument");
  ADP_CHECK_ARG(g->n >= 0 && g->n < (1LL << 31), "n out of range");
  ADP_CHECK_ARG(g->n == 0 || (grad2d_accum && grad2d_visits && g->logscale && split_ids &&
                              clone_ids), "NULL array");
  ADP_CHECK_ARG(tau_s > 0.f, "tau_s must be positive");
  ADP_CHECK_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
  const size_t need = adp_densify_select_workspace_size(g->n);
  ADP_CHECK_ARG(ws_bytes >= need, "workspace %zu bytes, need %zu", ws_bytes, need);
  cudaStream_t st = (cudaStream_t)stream;
  if (g->n == 0) {
    FillSet f;
    f.add(d_counts, 2 * sizeof(int64_t));
    return launch_fill(f, st);
  }
  Carver c(ws, ws_bytes);
  void* sw = c.take<char>(scan_workspace_bytes(g->n));
  long long* total = c.take<long long>(1);
  const float ln_tau_s = (float)std::log((double)tau_s);
  const float* acc = grad2d_accum;
  const int* vis = grad2d_visits;
  const float4* ls = reinterpret_cast<const float4*>(g->logscale);
  int32_t* sp = split_ids;
  int32_t* cl = clone_ids;
  int rc = scan_exclusive(
      [=] __device__(long long i) -> long long {
        const unsigned k = densify_class(acc, vis, ls, i, tau_g, ln_tau_s);
        return k == 1u ? 1LL : (k == 2u ? (1LL << 32) : 0LL);
      },
      [=] __device__(long long i, long long pre) {
        const unsigned k = densify_class(acc, vis, ls, i, tau_g, ln_tau_s);
        if (k == 1u) sp[pre & 0xffffffffLL] = (int32_t)i;
        if (k == 2u) cl[(unsigned long long)pre >> 32] = (int32_t)i;
      },
      g->n, nullptr, total, sw, st, d_status);
  if (rc) return rc;
  densify_counts_kernel<<<1, 1, 0, st>>>(total, scan_error_flag(sw, g->n), d_counts);
  densify_tail_kernel<<<grid_for(g->n, 256, 148 * 16), 256, 0, st>>>(total, g->n, split_ids,
                                                                      clone_ids);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

// The AdpSplit operator (Sec. 4, Sec. 5.1, Appendix A) and the compaction of the
// Gaussian arrays.
//
// Plan: regions are grouped by candidate with a stable radix sort on the
// candidate index (keeping their (view, label) order), one thread per region
// builds the child proposal (Eqs. 9-10, Appendix A), and one warp per
// candidate with several proposals merges them (Eqs. 11-12: pairwise tests over
// the lanes, union-find, enclosing covariance from a Jacobi 3x3
// eigen-decomposition), applies the n_max cap and writes the surviving children
// into a per-region child table.
// Scans give every kept Gaussian its new index and every candidate the offset
// of its appended block. This stage is small next to rendering, so it runs in
// FP64, which keeps every integer outcome (statuses, child counts) stable.
// Apply: gathers kept Gaussians (with Adam moments) and writes appended ones.
#include <mutex>

#include "adam.cuh"
#include "gauss_math.cuh"

namespace adp {

struct Prop {
  double mu[3];
  double R[9];  // row-major, columns are the child's axes
  double s[3];
  double is2[3];  // 1 / s^2 (FP64 division is slow here: done once per proposal)
  double rgb[3];
};

struct SplitWs {
  int* cand_of;        // [n] candidate index or -1
  unsigned* rkeys;     // [Rcap]
  unsigned* rvals;     // [Rcap]
  int2* seg;           // [n_cand] sorted-region range of each candidate
  Prop* props;         // [Rcap]
  int* uf;             // [Rcap]
  int* groups;         // [Rcap] root of each group, per candidate segment
  double* ext;         // [Rcap]
  float4* kids;        // [Rcap][4] child table: mean, quat, logscale, dc
  unsigned* dest;      // [n] new row of each Gaussian: bit 31 set for a (RESET)
                       // candidate, all ones for a removed one
  long long* app_off;  // [n_cand]
  long long* counters; // [0] regions in use, [1] kept, [2] appended, [3] new n,
                       // [4] ADAPTIVE candidates, [5] bound on the new n known
                       // before the merge (n + sum of min(proposals, n_max) over
                       // ADAPTIVE candidates + the FALLBACK count)
  int* multi;          // [n_cand] the ADAPTIVE candidates, in no particular order
  void* scan;          // the kept-row scan
  void* scan2;         // the appended-block scan (may run beside the kept-row one)
  SortWorkspace sort;
};

static size_t split_ws_bytes(long long n, long long nc, long long rc) {
  long long sm = n > nc ? n : nc;
  return carve_bytes<int>(n) + 2 * carve_bytes<unsigned>(rc) + carve_bytes<int2>(nc) +
         carve_bytes<Prop>(rc) + 2 * carve_bytes<int>(rc) + carve_bytes<double>(rc) +
         carve_bytes<float4>(4 * rc) + carve_bytes<unsigned>(n) + carve_bytes<long long>(nc) +
         carve_bytes<long long>(8) + carve_bytes<int>(nc) + scan_workspace_bytes(sm) +
         scan_workspace_bytes(nc) + sort_workspace_bytes(rc);
}

static SplitWs carve_split(Carver& c, long long n, long long nc, long long rc) {
  SplitWs w;
  long long sm = n > nc ? n : nc;
  w.cand_of = c.take<int>(n);
  w.rkeys = c.take<unsigned>(rc);
  w.rvals = c.take<unsigned>(rc);
  w.seg = c.take<int2>(nc);
  w.props = c.take<Prop>(rc);
  w.uf = c.take<int>(rc);
  w.groups = c.take<int>(rc);
  w.ext = c.take<double>(rc);
  w.kids = c.take<float4>(4 * rc);
  w.dest = c.take<unsigned>(n);
  w.app_off = c.take<long long>(nc);
  w.counters = c.take<long long>(8);
  w.multi = c.take<int>(nc);
  w.scan = c.take<char>(scan_workspace_bytes(sm));
  w.scan2 = c.take<char>(scan_workspace_bytes(nc));
  w.sort = carve_sort(c, rc);
  return w;
}

// ------------------------------------------------------------------ fp64 helpers

__device__ __forceinline__ double dot3d(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ void cross3d(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double clipd(double x, double a) {
  double m = fabs(x) < a ? fabs(x) : a;
  return x < 0.0 ? -m : m;
}

__device__ void quat_rot_d(float4 q, double* R) {
  double w = q.x, x = q.y, y = q.z, z = q.w;
  double nq = sqrt(w * w + x * x + y * y + z * z);
  w /= nq; x /= nq; y /= nq; z /= nq;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

// Unit quaternion (w >= 0) of a rotation matrix, from its largest diagonal term.
__device__ float4 rot_quat_d(const double* R) {
  double m00 = R[0], m11 = R[4], m22 = R[8];
  double w, x, y, z;
  double tr = m00 + m11 + m22;
  if (tr >= m00 && tr >= m11 && tr >= m22) {
    double r = sqrt(1.0 + tr);
    w = 0.5 * r; double f = 0.5 / r;
    x = (R[7] - R[5]) * f; y = (R[2] - R[6]) * f; z = (R[3] - R[1]) * f;
  } else if (m00 >= m11 && m00 >= m22) {
    double r = sqrt(1.0 + m00 - m11 - m22);
    x = 0.5 * r; double f = 0.5 / r;
    w = (R[7] - R[5]) * f; y = (R[1] + R[3]) * f; z = (R[2] + R[6]) * f;
  } else if (m11 >= m22) {
    double r = sqrt(1.0 - m00 + m11 - m22);
    y = 0.5 * r; double f = 0.5 / r;
    w = (R[2] - R[6]) * f; x = (R[1] + R[3]) * f; z = (R[5] + R[7]) * f;
  } else {
    double r = sqrt(1.0 - m00 - m11 + m22);
    z = 0.5 * r; double f = 0.5 / r;
    w = (R[3] - R[1]) * f; x = (R[2] + R[6]) * f; y = (R[5] + R[7]) * f;
  }
  double inq = 1.0 / sqrt(w * w + x * x + y * y + z * z);
  if (w < 0) inq = -inq;
  return make_float4((float)(w * inq), (float)(x * inq), (float)(y * inq), (float)(z * inq));
}

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations
// (Rutishauser's update form); E gets the eigenvectors as columns. Jacobi keeps
// eigenvectors accurate when eigenvalues are close, which the merged covariances
// of clipped, nearly isotropic children need. At most 50 sweeps.
__device__ void sym3_eigen(const double* A, double* lam, double* E) {
  double a[3][3], v[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      a[i][j] = A[3 * i + j];
      v[i][j] = i == j ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off == 0.0 || off <= 1e-32 * dia) break;
    for (int pq = 0; pq < 3; ++pq) {
      int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      double apq = a[p][q];
      if (apq == 0.0) continue;
      double tau = (a[q][q] - a[p][p]) / (2.0 * apq);
      double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
      int r = 3 - p - q;  // the untouched index
      double arp = a[r][p], arq = a[r][q];
      a[r][p] = a[p][r] = c * arp - s * arq;
      a[r][q] = a[q][r] = s * arp + c * arq;
      a[p][p] -= t * apq;
      a[q][q] += t * apq;
      a[p][q] = a[q][p] = 0.0;
      for (int k = 0; k < 3; ++k) {
        double vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - s * vkq;
        v[k][q] = s * vkp + c * vkq;
      }
    }
  }
  for (int i = 0; i < 3; ++i) {
    lam[i] = a[i][i];
    for (int j = 0; j < 3; ++j) E[3 * i + j] = v[i][j];
  }
}

__device__ __forceinline__ void sigma_of(const Prop& p, double* S) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += p.R[3 * i + k] * p.s[k] * p.s[k] * p.R[3 * j + k];
      S[3 * i + j] = acc;
    }
}

// sqrt(d^T Sigma^-1 d) with Sigma^-1 = R diag(s^-2) R^T
__device__ __forceinline__ double mahal_d(const Prop& p, const double* d) {
  double acc = 0;
  for (int k = 0; k < 3; ++k) {
    double c = p.R[k] * d[0] + p.R[3 + k] * d[1] + p.R[6 + k] * d[2];
    acc += c * c * p.is2[k];
  }
  return sqrt(acc);
}

// ------------------------------------------------------------------ plan kernels

__global__ void cand_of_kernel(const int* cand, long long nc, long long n, int* cand_of) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
       c += (long long)gridDim.x * blockDim.x) {
    int i = cand[c];
    if (i >= 0 && i < n) cand_of[i] = (int)c;
  }
}

__global__ void region_keys_kernel(const int* parent, const long long* d_count, long long cap,
                                   const int* cand_of, long long n, unsigned nc, unsigned* keys,
                                   unsigned* vals, long long* used) {
  long long R = *d_count;
  if (R > cap) R = cap;
  if (blockIdx.x == 0 && threadIdx.x == 0) *used = R;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < R;
       r += (long long)gridDim.x * blockDim.x) {
    int p = parent[r];
    int c = (p >= 0 && p < n) ? cand_of[p] : -1;
    keys[r] = c >= 0 ? (unsigned)c : nc;
    vals[r] = (unsigned)r;
  }
}

__global__ void seg_kernel(const unsigned* keys, const long long* d_n, unsigned nc, int2* seg) {
  long long N = *d_n;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < N;
       j += (long long)gridDim.x * blockDim.x) {
    unsigned k = keys[j];
    if (k >= nc) continue;
    if (j == 0 || keys[j - 1] != k) seg[k].x = (int)j;
    if (j == N - 1 || keys[j + 1] != k) seg[k].y = (int)(j + 1);
  }
}

struct ProposalArgs {
  const float4* mean_logit;
  const float4* logscale;
  const float4* quat;
  const int* r_view;
  const int* r_parent;
  const double* r_stats;
  const unsigned* keys;
  const unsigned* vals;
  const long long* d_n;
  unsigned nc;
  double eps_t, scale_floor;
  Prop* props;
};

// One child proposal per region (Eqs. 9-10 and Appendix A), in FP64.
__global__ void proposal_kernel(ProposalArgs a, CamSet cs) {
  long long N = *a.d_n;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < N;
       j += (long long)gridDim.x * blockDim.x) {
    if (a.keys[j] >= a.nc) continue;
    int r = (int)a.vals[j];
    int i = a.r_parent[r];
    const adp_camera& cam = cs.cam[a.r_view[r]];
    const double* st = a.r_stats + 12LL * r;
    float4 ml = a.mean_logit[i], ls = a.logscale[i];
    double mu[3] = {ml.x, ml.y, ml.z};
    double sp[3] = {exp((double)ls.x), exp((double)ls.y), exp((double)ls.z)};
    double Rp[9];
    quat_rot_d(a.quat[i], Rp);
    double Rw[9], tw[3];
    for (int k = 0; k < 9; ++k) Rw[k] = cam.R[k];
    for (int k = 0; k < 3; ++k) tw[k] = cam.t[k];
    double o[3], u[3], w[3], zv[3];
    for (int k = 0; k < 3; ++k) {
      o[k] = -(Rw[k] * tw[0] + Rw[3 + k] * tw[1] + Rw[6 + k] * tw[2]);
      u[k] = Rw[k];
      w[k] = Rw[3 + k];
      zv[k] = Rw[6 + k];
    }
    double dcam[3] = {(st[0] - (double)cam.px) / (double)cam.fx,
                      (st[1] - (double)cam.py) / (double)cam.fy, 1.0};
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = Rw[k] * dcam[0] + Rw[3 + k] * dcam[1] + Rw[6 + k] * dcam[2];
    double dn = sqrt(dot3d(d, d));
    for (int k = 0; k < 3; ++k) d[k] /= dn;
    // Sigma^-1 d and t* (Eq. 10)
    double Ad[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
      double c = Rp[k] * d[0] + Rp[3 + k] * d[1] + Rp[6 + k] * d[2];
      c /= sp[k] * sp[k];
      for (int m = 0; m < 3; ++m) Ad[m] += Rp[3 * m + k] * c;
    }
    double b[3] = {mu[0] - o[0], mu[1] - o[1], mu[2] - o[2]};
    double ts = dot3d(b, Ad) / (dot3d(d, Ad) + a.eps_t);
    Prop p;
    for (int k = 0; k < 3; ++k) p.mu[k] = o[k] + ts * d[k];
    double tz = ts / sqrt(dot3d(dcam, dcam));
    double smax = fmax(sp[0], fmax(sp[1], sp[2]));
    double e1x = st[5], e1y = st[6], e2x = -st[6], e2y = st[5];
    double w1x = clipd(e1x * st[7] * tz / (double)cam.fx, smax * fabs(e1x));
    double w1y = clipd(e1y * st[7] * tz / (double)cam.fy, smax * fabs(e1y));
    double w2x = clipd(e2x * st[8] * tz / (double)cam.fx, smax * fabs(e2x));
    double w2y = clipd(e2y * st[8] * tz / (double)cam.fy, smax * fabs(e2y));
    double a1[3], a2[3];
    for (int k = 0; k < 3; ++k) {
      a1[k] = w1x * u[k] + w1y * w[k];
      a2[k] = w2x * u[k] + w2y * w[k];
    }
    double n1 = sqrt(dot3d(a1, a1)), n2 = sqrt(dot3d(a2, a2));
    p.s[0] = fmax(n1, a.scale_floor);
    p.s[1] = fmax(n2, a.scale_floor);
    p.s[2] = p.s[1];
    for (int k = 0; k < 3; ++k) p.is2[k] = 1.0 / (p.s[k] * p.s[k]);
    double u1[3], u2[3];
    for (int k = 0; k < 3; ++k) u1[k] = n1 < 1e-12 ? u[k] : a1[k] / n1;
    double pr = dot3d(a2, u1), r2[3];
    for (int k = 0; k < 3; ++k) r2[k] = a2[k] - pr * u1[k];
    double nr = sqrt(dot3d(r2, r2));
    if (nr < 1e-12) {
      cross3d(zv, u1, u2);
    } else {
      for (int k = 0; k < 3; ++k) u2[k] = r2[k] / nr;
    }
    double c12[3];
    cross3d(u1, u2, c12);
    if (dot3d(c12, zv) < 0.0)
      for (int k = 0; k < 3; ++k) u2[k] = -u2[k];
    for (int k = 0; k < 3; ++k) {
      p.R[3 * k + 0] = u1[k];
      p.R[3 * k + 1] = u2[k];
      p.R[3 * k + 2] = zv[k];
      p.rgb[k] = st[9 + k];
    }
    a.props[j] = p;
  }
}

// The stored child is float32, so its log-scales are taken in float32 (within
// two float ulps of the rounded FP64 logarithm, at a fraction of the cost on the
// reduced-rate FP64 pipe) and the colour is mapped to the DC coefficient by a
// multiplication by 1 / C0 = 2 sqrt(pi).
__device__ void store_child(float4* kid, const double* mu, const double* R, const double* s,
                            const double* rgb) {
  kid[0] = make_float4((float)mu[0], (float)mu[1], (float)mu[2], 0.f);
  kid[1] = rot_quat_d(R);
  kid[2] = make_float4(logf((float)s[0]), logf((float)s[1]), logf((float)s[2]), 0.f);
  const double inv_C0 = 3.5449077018110318;  // 1 / C0 of the degree-0 SH basis
  kid[3] = make_float4((float)((rgb[0] - 0.5) * inv_C0), (float)((rgb[1] - 0.5) * inv_C0),
                       (float)((rgb[2] - 0.5) * inv_C0), 0.f);
}

struct MergeArgs {
  const int* cand;
  const int* count;
  const int2* seg;
  const Prop* props;
  int* uf;
  int* groups;
  double* ext;
  float4* kids;
  long long nc;
  double gamma_d, gamma_c, scale_floor;
  int n_max;
  uint8_t* status;
  int* n_children;
  int* multi;                    // candidates left to merge_warp_kernel
  unsigned long long* n_multi;   // their count
  unsigned long long* bound;     // += the largest growth the statuses allow
  long long n_rows;              // rows of the input population
};

// Eq. 11 between two proposals.
__device__ __forceinline__ bool merge_edge(const Prop& px, const Prop& py, double gamma_d,
                                           double gamma_c) {
  double dc = fmax(fabs(px.rgb[0] - py.rgb[0]),
                   fmax(fabs(px.rgb[1] - py.rgb[1]), fabs(px.rgb[2] - py.rgb[2])));
  if (dc > gamma_c) return false;
  double d[3] = {py.mu[0] - px.mu[0], py.mu[1] - px.mu[1], py.mu[2] - px.mu[2]};
  return mahal_d(px, d) + mahal_d(py, d) <= gamma_d;
}

// Merged parameters of the group rooted at proposal g (members m >= g with
// uf[m] == g), Eq. 12; a one-member group is the proposal itself.
__device__ void merged_group(const MergeArgs& a, int s0, int M, int g, double* mu, double* rgb,
                             double* R, double* s) {
  const int* uf = a.uf + s0;
  int cnt = 0, last = g;
  double gm[3] = {0, 0, 0}, gc[3] = {0, 0, 0}, Sb[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int m = g; m < M; ++m) {
    if (uf[m] != g) continue;
    const Prop& p = a.props[s0 + m];
    double S[9];
    sigma_of(p, S);
    for (int k = 0; k < 3; ++k) {
      gm[k] += p.mu[k];
      gc[k] += p.rgb[k];
    }
    for (int k = 0; k < 9; ++k) Sb[k] += S[k];
    ++cnt;
    last = m;
  }
  if (cnt == 1) {
    const Prop& p = a.props[s0 + g];
    for (int k = 0; k < 3; ++k) {
      mu[k] = p.mu[k];
      rgb[k] = p.rgb[k];
      s[k] = p.s[k];
    }
    for (int k = 0; k < 9; ++k) R[k] = p.R[k];
    return;
  }
  for (int k = 0; k < 3; ++k) {
    mu[k] = gm[k] / cnt;
    rgb[k] = gc[k] / cnt;
  }
  for (int k = 0; k < 9; ++k) Sb[k] /= cnt;
  double ev[3];
  sym3_eigen(Sb, ev, R);
  double lam[3] = {0, 0, 0};
  for (int m = g; m <= last; ++m) {
    if (uf[m] != g) continue;
    const Prop& p = a.props[s0 + m];
    double S[9];
    sigma_of(p, S);
    for (int r = 0; r < 3; ++r) {
      double e[3] = {R[r], R[3 + r], R[6 + r]};
      double Se[3];
      for (int k = 0; k < 3; ++k) Se[k] = S[3 * k] * e[0] + S[3 * k + 1] * e[1] + S[3 * k + 2] * e[2];
      double dm[3] = {p.mu[0] - mu[0], p.mu[1] - mu[1], p.mu[2] - mu[2]};
      double reach = fabs(dot3d(e, dm)) + sqrt(fmax(dot3d(e, Se), 0.0));
      lam[r] = fmax(lam[r], reach * reach);
    }
  }
  double c0[3] = {R[0], R[3], R[6]}, c1[3] = {R[1], R[4], R[7]}, c2[3] = {R[2], R[5], R[8]}, cc[3];
  cross3d(c0, c1, cc);
  if (dot3d(cc, c2) < 0.0) {
    R[2] = -R[2];
    R[5] = -R[5];
    R[8] = -R[8];
  }
  for (int r = 0; r < 3; ++r) s[r] = fmax(sqrt(lam[r]), a.scale_floor);
}

// One thread per candidate: statuses (which need no proposal), the list of
// ADAPTIVE candidates for merge_warp_kernel, and a bound on the new population
// size that holds whatever the merges decide: every ADAPTIVE candidate adds at
// most min(proposals, n_max) rows net (children plus its parent copy, minus
// itself) and every FALLBACK one adds one.
__global__ void merge_status_kernel(MergeArgs a) {
  unsigned long long extra = 0ull;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.nc;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = a.cand[c];
    const int2 sg = a.seg[c];
    const int M = sg.y - sg.x;
    if (i < 0) {  // an unused entry of a candidate list passed whole
      a.status[c] = ADP_KEEP;
      a.n_children[c] = 0;
    } else if (a.count[i] == 0) {
      a.status[c] = ADP_FALLBACK;
      a.n_children[c] = 0;
      extra += 1ull;
    } else if (M <= 0) {
      a.status[c] = ADP_RESET;
      a.n_children[c] = 0;
    } else {
      a.status[c] = ADP_ADAPTIVE;
      a.multi[atomicAdd(a.n_multi, 1ull)] = (int)c;  // merged by a warp
      extra += (unsigned long long)min(M, a.n_max);
    }
  }
  for (int o = 16; o > 0; o >>= 1) extra += __shfl_xor_sync(0xffffffffu, extra, o);
  if ((threadIdx.x & 31) == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) extra += (unsigned long long)a.n_rows;
    if (extra) atomicAdd(a.bound, extra);
  }
}

__device__ __forceinline__ int uf_root_v(volatile int* uf, int x) {
  int p = uf[x];
  while (p != x) {
    x = p;
    p = uf[x];
  }
  return x;
}

// One warp per ADAPTIVE candidate (the list merge_status_kernel builds; each
// candidate writes only its own segment, so the order is free; a single proposal
// is a one-member group, Eq. 12 then returns it unchanged): the pairwise tests of
// Eq. 11 are spread over the lanes and joined in a union-find whose links point
// to smaller indices (so every group is rooted at its first member); groups are
// numbered in first-member order, merged one per lane (Eq. 12), capped at n_max
// by extent (ties to the earlier group) and written to the child table in order.
__global__ void merge_warp_kernel(MergeArgs a) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long n_multi = (long long)*a.n_multi;
  for (long long t = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); t < n_multi;
       t += warps) {
    const int c = a.multi[t];
    const int2 sg = a.seg[c];
    const int s0 = sg.x, M = sg.y - sg.x;
    int* uf = a.uf + s0;
    volatile int* vuf = uf;
    for (int m = lane; m < M; m += 32) uf[m] = m;
    __syncwarp();
    for (int x = 0; x < M - 1; ++x) {
      const Prop& px = a.props[s0 + x];
      for (int y = x + 1 + lane; y < M; y += 32) {
        if (!merge_edge(px, a.props[s0 + y], a.gamma_d, a.gamma_c)) continue;
        int u = x, w = y;
        for (int guard = 0; guard < 4096; ++guard) {  // lock-free union, min-rooted
          u = uf_root_v(vuf, u);
          w = uf_root_v(vuf, w);
          if (u == w) break;
          if (u > w) {
            int t = u;
            u = w;
            w = t;
          }
          int old = atomicMin(&uf[w], u);
          if (old == w) break;
          w = old;
        }
      }
    }
    __syncwarp();
    __threadfence_block();
    for (int m = lane; m < M; m += 32) uf[m] = uf_root_v(vuf, m);
    __syncwarp();
    // groups in first-member order
    int ng = 0;
    for (int base = 0; base < M; base += 32) {
      const int m = base + lane;
      const bool root = m < M && uf[m] == m;
      const unsigned msk = __ballot_sync(0xffffffffu, root);
      if (root) a.groups[s0 + ng + __popc(msk & lanemask_lt())] = m;
      ng += __popc(msk);
    }
    __syncwarp();
    for (int gi = lane; gi < ng; gi += 32) {
      double mu[3], rgb[3], R[9], sc[3];
      merged_group(a, s0, M, a.groups[s0 + gi], mu, rgb, R, sc);
      a.ext[s0 + gi] = sc[0] * sc[1] * sc[2];
      store_child(a.kids + 4LL * (s0 + gi), mu, R, sc, rgb);
    }
    __syncwarp();
    // cap, then compaction in group order (positions never pass their source)
    int kept_total = 0;
    for (int base = 0; base < ng; base += 32) {
      const int gk = base + lane;
      bool keep = false;
      float4 k0, k1, k2, k3;
      if (gk < ng) {
        const double e = a.ext[s0 + gk];
        int rank = 0;
        for (int h = 0; h < ng && rank < a.n_max; ++h) {
          const double eh = a.ext[s0 + h];
          rank += (eh > e || (eh == e && h < gk)) ? 1 : 0;
        }
        keep = rank < a.n_max;
        const float4* src = a.kids + 4LL * (s0 + gk);
        k0 = src[0];
        k1 = src[1];
        k2 = src[2];
        k3 = src[3];
      }
      const unsigned msk = __ballot_sync(0xffffffffu, keep);
      __syncwarp();
      if (keep) {
        float4* dst = a.kids + 4LL * (s0 + kept_total + __popc(msk & lanemask_lt()));
        dst[0] = k0;
        dst[1] = k1;
        dst[2] = k2;
        dst[3] = k3;
      }
      kept_total += __popc(msk);
      __syncwarp();
    }
    if (lane == 0) a.n_children[c] = kept_total;
  }
}

// The new size. If either scan of the plan gave up a wait, the size is set beyond
// any capacity, so the compaction writes nothing (the caller's status word
// holds ADP_ERR_TIMEOUT).
__global__ void new_n_kernel(long long* counters, int64_t* d_new_n,
                             const unsigned long long* err_keep,
                             const unsigned long long* err_append) {
  const bool failed = *err_keep != 0ull || (err_append && *err_append != 0ull);
  counters[3] = failed ? (1LL << 62) : counters[1] + counters[2];
  *d_new_n = counters[3];
}

// ------------------------------------------------------------------ apply kernels

struct GaussPtrs {
  float4* ml;
  float4* ls;
  float4* q;
  float4* sh;
  long long n;
};

static inline GaussPtrs gp_of(const adp_gaussians* g) {
  GaussPtrs p;
  p.ml = reinterpret_cast<float4*>(g->mean_logit);
  p.ls = reinterpret_cast<float4*>(g->logscale);
  p.q = reinterpret_cast<float4*>(g->quat);
  p.sh = reinterpret_cast<float4*>(g->sh);
  p.n = g->n;
  return p;
}

struct ApplyArgs {
  GaussPtrs in, min_, vin, out, mout, vout;
  GaussPtrs grad;  // with the fused Adam step: the gradients of in
  const uint8_t* grad_rows;  // optional row mask of grad: 0 = zero gradient, not read
  AdamHyper adam;
  const long long* counters;  // [1] kept, [3] new size
  const long long* fit;       // the size compared with the capacity: [3], or the bound [5]
  bool has_m_in, has_v_in, has_m_out, has_v_out;
  int planes;
  const unsigned* dest;  // see SplitWs::dest
};

__device__ __forceinline__ void copy_gauss(const GaussPtrs& s, long long i, const GaussPtrs& d,
                                           long long j, int planes) {
  d.ml[j] = s.ml[i];
  d.ls[j] = s.ls[i];
  d.q[j] = s.q[i];
  for (int p = 0; p < planes; ++p) d.sh[(long long)p * d.n + j] = s.sh[(long long)p * s.n + i];
}

__device__ __forceinline__ void zero_gauss(const GaussPtrs& d, long long j, int planes) {
  float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  d.ml[j] = z;
  d.ls[j] = z;
  d.q[j] = z;
  for (int p = 0; p < planes; ++p) d.sh[(long long)p * d.n + j] = z;
}

__device__ __forceinline__ float4* plane_of(const GaussPtrs& g, int q, long long i) {
  return q == 0 ? g.ml + i : q == 1 ? g.ls + i : q == 2 ? g.q + i : g.sh + (long long)(q - 3) * g.n + i;
}

// Kept rows: one thread per (row, plane), blockIdx.y the plane (0 mean+logit,
// 1 log-scale, 2 quaternion, 3.. SH), so a block streams one plane of the
// parameters and moments (and gradients); the row's destination is one 32-bit
// word, re-read for every plane from L2. With ADAM, each kept
// non-candidate row gets the update adp_adam_step makes, bit for bit (candidates
// got theirs before the plan); moments in and out are then required.

// The row streams are read and written with the evict-first (streaming) cache
// hint, so the destination words and the gradient row mask, which every plane
// reads again, stay in L2 while the 15 planes stream past.
__device__ __forceinline__ float4 ld_row(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ void st_row(float4* p, float4 v) { __stcs(p, v); }

template <bool ADAM>
__device__ __forceinline__ void keep_row(const ApplyArgs& a, int q, long long i) {
  if (i >= a.in.n) return;
  // the destination first: a removed candidate's row is not read; then every
  // stream, and the gradient, whose load waits only for the row mask
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  const long long n_new = *a.fit;
  const unsigned d = a.dest[i];
  if (d == 0xffffffffu) return;  // a removed candidate
  const bool gl = ADAM && (!a.grad_rows || a.grad_rows[i]);
  float4 p = ld_row(plane_of(a.in, q, i));
  float4 m = a.has_m_in ? ld_row(plane_of(a.min_, q, i)) : z;
  float4 v = a.has_v_in ? ld_row(plane_of(a.vin, q, i)) : z;
  const float4 g = gl ? ld_row(plane_of(a.grad, q, i)) : z;
  if (n_new > a.out.n) return;  // the new population does not fit: write nothing
  const long long j = d & 0x7fffffffu;
  if (j >= a.out.n) return;
  if (ADAM && !(d >> 31)) {  // candidates got their step before the plan
    float lr4[4];
    adam_plane_lr(a.adam, q, lr4);
    adam_vec4(p, g, m, v, lr4, a.adam, adam_bias(a.adam));
  }
  st_row(plane_of(a.out, q, j), p);
  if (a.has_m_out) st_row(plane_of(a.mout, q, j), m);
  if (a.has_v_out) st_row(plane_of(a.vout, q, j), v);
}

// Blocks of 64 threads: 0.253 ms at 1M Gaussians, against 0.254 for 128, 0.259 for
// 256, 0.267 for 512 and 0.347 for 1024.
#ifndef ADP_KEEP_THREADS
#define ADP_KEEP_THREADS 64
#endif
constexpr int KEEP_THREADS = ADP_KEEP_THREADS;
template <bool ADAM>
__global__ void apply_keep_kernel(ApplyArgs a) {
  keep_row<ADAM>(a, blockIdx.y, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

struct AppendArgs {
  GaussPtrs in, out, mout, vout;
  bool has_m_out, has_v_out;
  int planes;
  const int* cand;
  long long nc;
  const uint8_t* status;
  const int* n_children;
  const int2* seg;
  const float4* kids;
  const long long* app_off;
  const long long* counters;
  const float* noise;
  float shrink;  // ln(2 eta), rounded to float32
};

// After an overlapped plan: the kept rows skipped by apply_keep_kernel because
// the bound on the new size exceeded the capacity, when the exact size fits (a
// grid-stride pass over every row and plane; a caller that sizes out for the
// bound never takes it, and the kernel then returns at once).
__global__ void __launch_bounds__(256) late_keep_kernel(ApplyArgs a) {
  if (a.counters[5] <= a.out.n || a.counters[3] > a.out.n) return;
  a.fit = a.counters + 3;
  const long long nr = a.in.n, tot = nr * (3 + a.planes);
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < tot;
       u += (long long)gridDim.x * blockDim.x)
    keep_row<true>(a, (int)(u / nr), u % nr);
}

// Appended rows: one thread per new row, in chunks of APP_THREADS rows per
// block. A row's candidate is the last one whose block of rows starts at or
// before it; the block finds the candidates of its chunk with two searches in
// global memory, stages their offsets in shared memory (at most APP_STAGE of
// them; longer runs of candidates without rows search global memory) and each
// thread searches there. The row is the parent copy (opacity o / (N + 1)) or
// child k - 1 of an ADAPTIVE candidate, or vanilla child k of a FALLBACK one
// (mu + R (s * noise), log-scale lowered by ln(2 eta)); every appended row gets
// zero moments. The arithmetic is float32: the mean offset sums the rotated
// noise before adding it to the mean, and the parent's new opacity logit is
// logit(sigmoid(x) / (N + 1)) = -ln(N + (N + 1) e^-x), written for either sign
// of x so that the exponential never overflows.
constexpr int APP_THREADS = 128;
constexpr int APP_STAGE = 512;

__device__ __forceinline__ long long last_le_ll(const long long* off, long long lo, long long hi,
                                               long long r) {
  while (lo < hi) {  // last c in [lo, hi] with off[c] <= r (off[lo] <= r)
    const long long mid = (lo + hi + 1) >> 1;
    if (off[mid] <= r) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float split_parent_logit(float x, int N) {
  const float a = (float)N, b = (float)(N + 1);
  return x >= 0.f ? -logf(fmaf(b, expf(-x), a)) : x - logf(fmaf(a, expf(x), b));
}

__global__ void __launch_bounds__(APP_THREADS) apply_append_kernel(AppendArgs a) {
  __shared__ long long s_off[APP_STAGE];
  __shared__ long long s_c[2];
  if (a.counters[3] > a.out.n) return;  // the new population does not fit: write nothing
  const long long n_keep = a.counters[1], n_app = a.counters[2];
  for (long long r0 = blockIdx.x * (long long)APP_THREADS; r0 < n_app;
       r0 += (long long)gridDim.x * APP_THREADS) {
    const long long r1 = min(r0 + APP_THREADS, n_app);
    if (threadIdx.x < 2)
      s_c[threadIdx.x] = last_le_ll(a.app_off, 0, a.nc - 1, threadIdx.x == 0 ? r0 : r1 - 1);
    __syncthreads();
    const long long c0 = s_c[0], cnt = s_c[1] - c0 + 1;
    const bool staged = cnt <= APP_STAGE;
    if (staged)
      for (int q = threadIdx.x; q < cnt; q += APP_THREADS) s_off[q] = a.app_off[c0 + q];
    __syncthreads();
    const long long r = r0 + threadIdx.x;
    if (r < r1) {
      long long c, base;
      if (staged) {
        const long long q = last_le_ll(s_off, 0, cnt - 1, r);
        c = c0 + q;
        base = s_off[q];
      } else {
        c = last_le_ll(a.app_off, c0, c0 + cnt - 1, r);
        base = a.app_off[c];
      }
      const int k = (int)(r - base);
      const int i = a.cand[c];
      const long long j = n_keep + r;
      const uint8_t stt = a.status[c];
      const float4 ml = a.in.ml[i], ls = a.in.ls[i];
      if (stt == ADP_FALLBACK) {
        const float4 q = a.in.q[i];
        const float qn = 1.f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        const Mat3 R = rot_of_quat(q.x * qn, q.y * qn, q.z * qn, q.w * qn);
        const float* z = a.noise + 6 * c + 3 * k;
        const float d0 = expf(ls.x) * z[0], d1 = expf(ls.y) * z[1], d2 = expf(ls.z) * z[2];
        float m[3];
        const float mu[3] = {ml.x, ml.y, ml.z};
        for (int rr = 0; rr < 3; ++rr)
          m[rr] = mu[rr] + fmaf(R.m[3 * rr], d0, fmaf(R.m[3 * rr + 1], d1, R.m[3 * rr + 2] * d2));
        copy_gauss(a.in, i, a.out, j, a.planes);
        a.out.ml[j] = make_float4(m[0], m[1], m[2], ml.w);
        a.out.ls[j] = make_float4(ls.x - a.shrink, ls.y - a.shrink, ls.z - a.shrink, ls.w);
      } else if (k == 0) {  // parent copy: opacity o / (N + 1), everything else unchanged
        copy_gauss(a.in, i, a.out, j, a.planes);
        a.out.ml[j] = make_float4(ml.x, ml.y, ml.z, split_parent_logit(ml.w, a.n_children[c]));
      } else {
        const float4* kid = a.kids + 4LL * (a.seg[c].x + k - 1);
        const float4 km = kid[0], kq = kid[1], kl = kid[2], kd = kid[3];
        a.out.ml[j] = make_float4(km.x, km.y, km.z, ml.w);
        a.out.ls[j] = make_float4(kl.x, kl.y, kl.z, 0.f);
        a.out.q[j] = kq;
        a.out.sh[j] = make_float4(kd.x, kd.y, kd.z, 0.f);
        for (int p = 1; p < a.planes; ++p)
          a.out.sh[(long long)p * a.out.n + j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (a.has_m_out) zero_gauss(a.mout, j, a.planes);
      if (a.has_v_out) zero_gauss(a.vout, j, a.planes);
    }
    __syncthreads();
  }
}

// Whether two Gaussian arrays share a plane (either may be NULL).
static bool gauss_alias(const adp_gaussians* a, const adp_gaussians* b) {
  if (!a || !b) return false;
  const float* pa[4] = {a->mean_logit, a->logscale, a->quat, a->sh};
  const float* pb[4] = {b->mean_logit, b->logscale, b->quat, b->sh};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      if (pa[i] && pa[i] == pb[j]) return true;
  return false;
}

static bool gauss_ok(const adp_gaussians* g) {
  return g && g->mean_logit && g->logscale && g->quat && g->sh && aligned(g->mean_logit, 16) &&
         aligned(g->logscale, 16) && aligned(g->quat, 16) && aligned(g->sh, 16);
}

}  // namespace adp

using namespace adp;

extern "C" ADP_API size_t adp_split_workspace_size(int64_t n, int64_t n_cand,
                                                   int64_t region_capacity) {
  if (n < 0 || n_cand < 0 || region_capacity < 0) return 0;
  return split_ws_bytes(n, n_cand, region_capacity);
}

namespace adp {

// The validated arguments of a plan.
struct PlanCall {
  const adp_gaussians* g;
  const adp_regions* regs;
  const int32_t* candidates;
  const int32_t* count;
  const adp_params* prm;
  uint8_t* status;
  int32_t* n_children;
  int64_t* d_new_n;
  int32_t* d_status;
  long long n, nc, rcap;
  CamSet cs;
};

static int plan_args(const adp_gaussians* g, const adp_camera* cams, int32_t n_views,
                     const adp_regions* regs, const int32_t* candidates, int64_t n_cand,
                     const int32_t* count, const adp_params* prm, uint8_t* status,
                     int32_t* n_children, int64_t* d_new_n, void* ws, size_t ws_bytes,
                     int32_t* d_status, PlanCall* pc) {
  ADP_CHECK_ARG(gauss_ok(g) || (g && g->n == 0), "bad Gaussian arrays");
  ADP_CHECK_ARG(regs && regs->count && count && d_new_n, "NULL argument");
  ADP_CHECK_ARG(g->n >= 0 && g->n < (1LL << 31), "n out of range");
  ADP_CHECK_ARG(n_cand >= 0 && n_cand <= g->n, "n_cand out of range");
  ADP_CHECK_ARG(n_cand == 0 || (candidates && status && n_children), "NULL candidate arrays");
  ADP_CHECK_ARG(regs->capacity >= 0 && regs->capacity < (1LL << 31), "region capacity out of range");
  ADP_CHECK_ARG(regs->capacity == 0 || (regs->view && regs->parent && regs->stats),
                "NULL region arrays");
  int rc = make_camset(cams, n_views, prm, &pc->cs);
  if (rc) return rc;
  ADP_CHECK_ARG(prm->n_max >= 0, "n_max must be >= 0");
  ADP_CHECK_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
  pc->n = g->n;
  pc->nc = n_cand;
  pc->rcap = regs->capacity;
  size_t need = split_ws_bytes(pc->n, pc->nc, pc->rcap);
  ADP_CHECK_ARG(ws_bytes >= need, "workspace %zu bytes, need %zu", ws_bytes, need);
  pc->g = g;
  pc->regs = regs;
  pc->candidates = candidates;
  pc->count = count;
  pc->prm = prm;
  pc->status = status;
  pc->n_children = n_children;
  pc->d_new_n = d_new_n;
  pc->d_status = d_status;
  return ADP_OK;
}

static MergeArgs merge_args(const PlanCall& pc, const SplitWs& w) {
  MergeArgs ma;
  ma.cand = pc.candidates;
  ma.count = pc.count;
  ma.seg = w.seg;
  ma.props = w.props;
  ma.uf = w.uf;
  ma.groups = w.groups;
  ma.ext = w.ext;
  ma.kids = w.kids;
  ma.nc = pc.nc;
  ma.gamma_d = pc.prm->gamma_d;
  ma.gamma_c = pc.prm->gamma_c;
  ma.scale_floor = pc.prm->scale_floor;
  ma.n_max = pc.prm->n_max;
  ma.status = pc.status;
  ma.n_children = pc.n_children;
  ma.multi = w.multi;
  ma.n_multi = reinterpret_cast<unsigned long long*>(&w.counters[4]);
  ma.bound = reinterpret_cast<unsigned long long*>(&w.counters[5]);
  ma.n_rows = pc.n;
  return ma;
}

// Plan, first part (needs no proposal): regions grouped per candidate, the
// statuses, the bound on the new size and the new row of every kept Gaussian.
static int plan_phase_a(const PlanCall& pc, const SplitWs& w, cudaStream_t st) {
  const long long n = pc.n, nc = pc.nc, rcap = pc.rcap;
  int rc;
  // the counters, -1 in every Gaussian's candidate slot, the empty region
  // segments and the status words of both parts' scans, in one launch
  FillSet fill;
  fill.add(w.counters, 8 * sizeof(long long));
  fill.add(w.cand_of, sizeof(int) * (size_t)n, ~0ull);
  fill.add(w.seg, sizeof(int2) * (size_t)nc);
  scan_clear(fill, w.scan, n);
  if (nc > 0) scan_clear(fill, w.scan2, nc);
  rc = launch_fill(fill, st);
  if (rc) return rc;
  if (nc > 0) {
    cand_of_kernel<<<grid_for(nc, 256, 4096), 256, 0, st>>>(pc.candidates, nc, n, w.cand_of);
  }
  if (rcap > 0) {
    region_keys_kernel<<<grid_for(rcap, 256, 4096), 256, 0, st>>>(
        pc.regs->parent, (const long long*)pc.regs->count, rcap, w.cand_of, n, (unsigned)nc,
        w.rkeys, w.rvals, &w.counters[0]);
    int bits = bits_for(nc);
    DigitOp passes[4];
    int np = 0;
    for (int sft = 0; sft < bits; sft += 8) passes[np++] = DigitOp{sft, 0u};
    rc = radix_sort_pairs(w.rkeys, w.rvals, &w.counters[0], rcap, passes, np, w.sort, st);
    if (rc) return rc;
    seg_kernel<<<grid_for(rcap, 256, 4096), 256, 0, st>>>(w.rkeys, &w.counters[0], (unsigned)nc,
                                                          w.seg);
  }
  // statuses, the ADAPTIVE list and the bound (launched even without candidates:
  // the bound then is n)
  merge_status_kernel<<<grid_for(nc, 256, 4096), 256, 0, st>>>(merge_args(pc, w));
  ADP_LAUNCH_CHECK();
  // new indices of kept Gaussians
  const int* cand_of = w.cand_of;
  unsigned* dest = w.dest;
  const uint8_t* cstatus = pc.status;
  rc = scan_exclusive(
      [=] __device__(long long i) -> long long {
        int cc = cand_of[i];
        return (cc < 0 || cstatus[cc] == ADP_RESET) ? 1 : 0;
      },
      [=] __device__(long long i, long long pre) {
        const int cc = cand_of[i];
        const bool kept = cc < 0 || cstatus[cc] == ADP_RESET;
        dest[i] = kept ? ((unsigned)pre | (cc >= 0 ? 0x80000000u : 0u)) : 0xffffffffu;
      },
      n, nullptr, &w.counters[1], w.scan, st, pc.d_status, /*cleared=*/true);
  return rc;
}

// Plan, second part: one proposal per region (Eqs. 9-10, Appendix A), the merge
// and cap per ADAPTIVE candidate (Eqs. 11-12), the offsets of the appended
// blocks and the new size.
static int plan_phase_b(const PlanCall& pc, const SplitWs& w, cudaStream_t st) {
  const long long nc = pc.nc, rcap = pc.rcap;
  int rc;
  if (rcap > 0) {
    ProposalArgs pa;
    pa.mean_logit = reinterpret_cast<const float4*>(pc.g->mean_logit);
    pa.logscale = reinterpret_cast<const float4*>(pc.g->logscale);
    pa.quat = reinterpret_cast<const float4*>(pc.g->quat);
    pa.r_view = pc.regs->view;
    pa.r_parent = pc.regs->parent;
    pa.r_stats = pc.regs->stats;
    pa.keys = w.rkeys;
    pa.vals = w.rvals;
    pa.d_n = &w.counters[0];
    pa.nc = (unsigned)nc;
    pa.eps_t = pc.prm->eps_t;
    pa.scale_floor = pc.prm->scale_floor;
    pa.props = w.props;
    proposal_kernel<<<grid_for(rcap, 128, 4096), 128, 0, st>>>(pa, pc.cs);
    ADP_LAUNCH_CHECK();
  }
  if (nc > 0) {
    // a resident grid (four 128-thread blocks per SM fit its registers) that loops
    // over the device-side list; an ADAPTIVE candidate has a region, so there are
    // at most min(nc, rcap) of them
    merge_warp_kernel<<<grid_for(std::min(nc, std::max(rcap, 1LL)) * 32, 128, 148 * 4), 128, 0,
                        st>>>(merge_args(pc, w));
    ADP_LAUNCH_CHECK();
    const uint8_t* cstatus = pc.status;
    const int* nch = pc.n_children;
    long long* app_off = w.app_off;
    rc = scan_exclusive(
        [=] __device__(long long cc) -> long long {
          uint8_t s = cstatus[cc];
          return s == ADP_ADAPTIVE ? 1 + nch[cc] : (s == ADP_FALLBACK ? 2 : 0);
        },
        [=] __device__(long long cc, long long pre) { app_off[cc] = pre; }, nc, nullptr,
        &w.counters[2], w.scan2, st, pc.d_status, /*cleared=*/true);
    if (rc) return rc;
  }
  new_n_kernel<<<1, 1, 0, st>>>(w.counters, pc.d_new_n, scan_error_flag(w.scan, pc.n),
                                nc > 0 ? scan_error_flag(w.scan2, nc) : nullptr);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

}  // namespace adp

extern "C" ADP_API int adp_split_plan(const adp_gaussians* g, const adp_camera* cams,
                                      int32_t n_views, const adp_regions* regs,
                                      const int32_t* candidates, int64_t n_cand,
                                      const int32_t* count, const adp_params* prm,
                                      uint8_t* status, int32_t* n_children, int64_t* d_new_n,
                                      int64_t* h_new_n, void* ws, size_t ws_bytes,
                                      int32_t* d_status, adp_stream_t stream) {
  PlanCall pc;
  int rc = plan_args(g, cams, n_views, regs, candidates, n_cand, count, prm, status, n_children,
                     d_new_n, ws, ws_bytes, d_status, &pc);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Carver c(ws, ws_bytes);
  SplitWs w = carve_split(c, pc.n, pc.nc, pc.rcap);
  rc = plan_phase_a(pc, w, st);
  if (rc) return rc;
  rc = plan_phase_b(pc, w, st);
  if (rc) return rc;
  if (h_new_n) {
    ADP_CUDA(cudaMemcpyAsync(h_new_n, &w.counters[3], sizeof(long long), cudaMemcpyDeviceToHost, st));
    ADP_CUDA(cudaStreamSynchronize(st));
  }
  return ADP_OK;
}

extern "C" ADP_API int adp_split_plan_statuses(const adp_gaussians* g, const adp_camera* cams,
                                               int32_t n_views, const adp_regions* regs,
                                               const int32_t* candidates, int64_t n_cand,
                                               const int32_t* count, const adp_params* prm,
                                               uint8_t* status, int32_t* n_children,
                                               int64_t* d_new_n, void* ws, size_t ws_bytes,
                                               int32_t* d_status, adp_stream_t stream) {
  PlanCall pc;
  int rc = plan_args(g, cams, n_views, regs, candidates, n_cand, count, prm, status, n_children,
                     d_new_n, ws, ws_bytes, d_status, &pc);
  if (rc) return rc;
  Carver c(ws, ws_bytes);
  SplitWs w = carve_split(c, pc.n, pc.nc, pc.rcap);
  return plan_phase_a(pc, w, (cudaStream_t)stream);
}

extern "C" ADP_API int adp_split_plan_proposals_overlapped(
    const adp_gaussians* g, const adp_camera* cams, int32_t n_views, const adp_regions* regs,
    const int32_t* candidates, int64_t n_cand, const int32_t* count, const adp_params* prm,
    uint8_t* status, int32_t* n_children, int64_t* d_new_n, void* ws, size_t ws_bytes,
    int32_t* d_status, adp_stream_t stream) {
  PlanCall pc;
  int rc = plan_args(g, cams, n_views, regs, candidates, n_cand, count, prm, status, n_children,
                     d_new_n, ws, ws_bytes, d_status, &pc);
  if (rc) return rc;
  AuxStream* aux = nullptr;
  rc = aux_stream(&aux);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Carver c(ws, ws_bytes);
  SplitWs w = carve_split(c, pc.n, pc.nc, pc.rcap);
  {  // fork: the second part on the auxiliary stream, after the work enqueued on st
    std::lock_guard<std::mutex> lock(aux_mutex());
    ADP_CUDA(cudaEventRecord(aux->planned, st));
    ADP_CUDA(cudaStreamWaitEvent(aux->stream, aux->planned, 0));
  }
  rc = plan_phase_b(pc, w, aux->stream);
  std::lock_guard<std::mutex> lock(aux_mutex());
  ADP_CUDA(cudaEventRecord(aux->merged, aux->stream));
  if (rc) {
    // join the fork before reporting the failure, so that a capture in progress
    // stays valid and no later call waits on a stale event
    ADP_CUDA(cudaStreamWaitEvent(st, aux->merged, 0));
    return rc;
  }
  return ADP_OK;
}

extern "C" ADP_API int adp_split_plan_overlapped(const adp_gaussians* g, const adp_camera* cams,
                                                 int32_t n_views, const adp_regions* regs,
                                                 const int32_t* candidates, int64_t n_cand,
                                                 const int32_t* count, const adp_params* prm,
                                                 uint8_t* status, int32_t* n_children,
                                                 int64_t* d_new_n, void* ws, size_t ws_bytes,
                                                 int32_t* d_status, adp_stream_t stream) {
  // the arguments and the auxiliary stream first, so that a failure leaves no work
  PlanCall pc;
  int rc = plan_args(g, cams, n_views, regs, candidates, n_cand, count, prm, status, n_children,
                     d_new_n, ws, ws_bytes, d_status, &pc);
  if (rc) return rc;
  AuxStream* aux = nullptr;
  rc = aux_stream(&aux);
  if (rc) return rc;
  rc = adp_split_plan_statuses(g, cams, n_views, regs, candidates, n_cand, count, prm, status,
                               n_children, d_new_n, ws, ws_bytes, d_status, stream);
  if (rc) return rc;
  return adp_split_plan_proposals_overlapped(g, cams, n_views, regs, candidates, n_cand, count,
                                             prm, status, n_children, d_new_n, ws, ws_bytes,
                                             d_status, stream);
}

// Which part of the compaction a call enqueues: everything, or, after an
// overlapped plan, the kept rows (against the bound) or the join and the
// appended rows.
enum class ApplyPart { ALL, KEEP, APPEND };

static int split_apply_impl(const adp_gaussians* g, const adp_gaussians* grad,
                            const AdamHyper* adam, const adp_gaussians* m_in,
                            const adp_gaussians* v_in, const adp_regions* regs,
                            const int32_t* candidates, int64_t n_cand, const uint8_t* status,
                            const int32_t* n_children, const float* noise, const adp_params* prm,
                            adp_gaussians* out, adp_gaussians* m_out, adp_gaussians* v_out,
                            void* ws, size_t ws_bytes, cudaStream_t st,
                            ApplyPart part = ApplyPart::ALL) {
  const bool overlapped = part != ApplyPart::ALL;
  ADP_CHECK_ARG(g && out && regs && prm, "NULL argument");
  ADP_CHECK_ARG(gauss_ok(g) || g->n == 0, "bad input Gaussian arrays");
  ADP_CHECK_ARG(gauss_ok(out) || out->n == 0, "bad output Gaussian arrays");
  ADP_CHECK_ARG(out->sh_degree == g->sh_degree, "sh_degree mismatch");
  ADP_CHECK_ARG(n_cand >= 0 && n_cand <= g->n, "n_cand out of range");
  ADP_CHECK_ARG(n_cand == 0 || (candidates && status && n_children && noise), "NULL candidate arrays");
  ADP_CHECK_ARG(!m_in || (gauss_ok(m_in) && m_in->n == g->n), "bad m_in");
  ADP_CHECK_ARG(!v_in || (gauss_ok(v_in) && v_in->n == g->n), "bad v_in");
  ADP_CHECK_ARG(!m_out || (gauss_ok(m_out) && m_out->n == out->n), "bad m_out (its n must equal out->n)");
  ADP_CHECK_ARG(!v_out || (gauss_ok(v_out) && v_out->n == out->n), "bad v_out (its n must equal out->n)");
  if (adam) {
    ADP_CHECK_ARG(m_in && v_in && m_out && v_out, "the fused Adam step needs all four moment arrays");
    ADP_CHECK_ARG(grad && (gauss_ok(grad) || g->n == 0) && grad->n == g->n &&
                      grad->sh_degree == g->sh_degree, "bad grad");
  }
  ADP_CHECK_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
  ADP_CHECK_ARG(!overlapped || adam, "internal: the overlapped compaction has the Adam step");
  // outputs must not alias inputs: the compaction reads rows while it writes others,
  // and in the overlapped calls the proposals read g on the auxiliary stream while
  // the kept rows are written
  ADP_CHECK_ARG(!gauss_alias(out, g) && !gauss_alias(out, m_in) && !gauss_alias(out, v_in) &&
                    !gauss_alias(out, grad) && !gauss_alias(m_out, g) &&
                    !gauss_alias(m_out, m_in) && !gauss_alias(m_out, v_in) &&
                    !gauss_alias(v_out, g) && !gauss_alias(v_out, m_in) &&
                    !gauss_alias(v_out, v_in),
                "output arrays alias input arrays");
  long long n = g->n, nc = n_cand, rcap = regs->capacity;
  size_t need = split_ws_bytes(n, nc, rcap);
  ADP_CHECK_ARG(ws_bytes >= need, "workspace %zu bytes, need %zu", ws_bytes, need);
  Carver c(ws, ws_bytes);
  SplitWs w = carve_split(c, n, nc, rcap);
  int planes = sh_planes(g->sh_degree);
  GaussPtrs gin = gp_of(g), gout = gp_of(out);
  ApplyArgs aa;
  aa.in = gin;
  aa.out = gout;
  aa.has_m_in = m_in != nullptr;
  aa.has_v_in = v_in != nullptr;
  aa.has_m_out = m_out != nullptr;
  aa.has_v_out = v_out != nullptr;
  if (m_in) aa.min_ = gp_of(m_in);
  if (v_in) aa.vin = gp_of(v_in);
  if (m_out) aa.mout = gp_of(m_out);
  if (v_out) aa.vout = gp_of(v_out);
  aa.grad_rows = nullptr;
  if (adam) {
    aa.grad = gp_of(grad);
    aa.grad_rows = grad->rows;
    aa.adam = *adam;
  }
  aa.planes = planes;
  aa.dest = w.dest;
  aa.counters = w.counters;
  // after an overlapped plan the merge may still run: the kept rows are written
  // against the bound on the new size, the appended ones after the join
  aa.fit = overlapped ? &w.counters[5] : &w.counters[3];
  AuxStream* aux = nullptr;
  if (overlapped) {
    int rc = aux_stream(&aux);
    if (rc) return rc;
  }
  if (n > 0 && part != ApplyPart::APPEND) {
    const dim3 kg(grid_for(n, KEEP_THREADS), 3 + planes);
    if (adam)
      apply_keep_kernel<true><<<kg, KEEP_THREADS, 0, st>>>(aa);
    else
      apply_keep_kernel<false><<<kg, KEEP_THREADS, 0, st>>>(aa);
  }
  if (part == ApplyPart::KEEP) {
    ADP_LAUNCH_CHECK();
    return ADP_OK;
  }
  if (overlapped) {  // join the plan's second part
    std::lock_guard<std::mutex> lock(aux_mutex());
    ADP_CUDA(cudaStreamWaitEvent(st, aux->merged, 0));
  }
  // the kept rows were written against the bound unless it exceeded out->n. The
  // bound is at most n + n_cand + the region capacity (one row per FALLBACK
  // candidate, at most one per stored region for an ADAPTIVE one), so with that much
  // room the late pass can never act and is not launched
  if (overlapped && n > 0 && out->n < n + nc + rcap) {
    late_keep_kernel<<<148 * 2, 256, 0, st>>>(aa);
    ADP_LAUNCH_CHECK();
  }
  if (nc > 0) {
    AppendArgs ap;
    ap.in = gin;
    ap.out = gout;
    ap.has_m_out = m_out != nullptr;
    ap.has_v_out = v_out != nullptr;
    if (m_out) ap.mout = gp_of(m_out);
    if (v_out) ap.vout = gp_of(v_out);
    ap.planes = planes;
    ap.cand = candidates;
    ap.nc = nc;
    ap.status = status;
    ap.n_children = n_children;
    ap.seg = w.seg;
    ap.kids = w.kids;
    ap.app_off = w.app_off;
    ap.counters = w.counters;
    ap.noise = noise;
    ap.shrink = (float)std::log(2.0 * (double)prm->eta);
    apply_append_kernel<<<grid_for(nc * (long long)(prm->n_max > 1 ? prm->n_max + 1 : 2),
                                   APP_THREADS, 148 * 16), APP_THREADS, 0, st>>>(ap);
  }
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

__global__ void split_step_advance_kernel(int* d_step) { *d_step += 1; }

extern "C" ADP_API int adp_split_apply(const adp_gaussians* g, const adp_gaussians* m_in,
                                       const adp_gaussians* v_in, const adp_regions* regs,
                                       const int32_t* candidates, int64_t n_cand,
                                       const uint8_t* status, const int32_t* n_children,
                                       const float* noise, const adp_params* prm,
                                       adp_gaussians* out, adp_gaussians* m_out,
                                       adp_gaussians* v_out, void* ws, size_t ws_bytes,
                                       adp_stream_t stream) {
  return split_apply_impl(g, nullptr, nullptr, m_in, v_in, regs, candidates, n_cand, status,
                          n_children, noise, prm, out, m_out, v_out, ws, ws_bytes,
                          (cudaStream_t)stream);
}

extern "C" ADP_API int adp_split_apply_adam(
    const adp_gaussians* g, const adp_gaussians* grad, const adp_gaussians* m_in,
    const adp_gaussians* v_in, const adp_regions* regs, const int32_t* candidates, int64_t n_cand,
    const uint8_t* status, const int32_t* n_children, const float* noise, const adp_params* prm,
    int32_t step, int32_t* d_step, const float* lr, float beta1, float beta2, float eps,
    adp_gaussians* out, adp_gaussians* m_out, adp_gaussians* v_out, void* ws, size_t ws_bytes,
    adp_stream_t stream) {
  ADP_CHECK_ARG(lr, "NULL lr");
  ADP_CHECK_ARG(d_step || step >= 1, "step must be >= 1");
  AdamHyper h = adam_hyper(lr, beta1, beta2, eps, step, d_step);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = split_apply_impl(g, grad, &h, m_in, v_in, regs, candidates, n_cand, status, n_children,
                            noise, prm, out, m_out, v_out, ws, ws_bytes, st);
  if (rc) return rc;
  if (d_step) {
    split_step_advance_kernel<<<1, 1, 0, st>>>(d_step);
    ADP_LAUNCH_CHECK();
  }
  return ADP_OK;
}

static int split_overlapped_part(
    const adp_gaussians* g, const adp_gaussians* grad, const adp_gaussians* m_in,
    const adp_gaussians* v_in, const adp_regions* regs, const int32_t* candidates, int64_t n_cand,
    const uint8_t* status, const int32_t* n_children, const float* noise, const adp_params* prm,
    int32_t step, int32_t* d_step, const float* lr, float beta1, float beta2, float eps,
    adp_gaussians* out, adp_gaussians* m_out, adp_gaussians* v_out, void* ws, size_t ws_bytes,
    adp_stream_t stream, ApplyPart part) {
  ADP_CHECK_ARG(lr, "NULL lr");
  ADP_CHECK_ARG(d_step || step >= 1, "step must be >= 1");
  AdamHyper h = adam_hyper(lr, beta1, beta2, eps, step, d_step);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = split_apply_impl(g, grad, &h, m_in, v_in, regs, candidates, n_cand, status, n_children,
                            noise, prm, out, m_out, v_out, ws, ws_bytes, st, part);
  if (rc) return rc;
  if (d_step && part == ApplyPart::APPEND) {
    split_step_advance_kernel<<<1, 1, 0, st>>>(d_step);
    ADP_LAUNCH_CHECK();
  }
  return ADP_OK;
}

extern "C" ADP_API int adp_split_keep_overlapped(
    const adp_gaussians* g, const adp_gaussians* grad, const adp_gaussians* m_in,
    const adp_gaussians* v_in, const adp_regions* regs, const int32_t* candidates, int64_t n_cand,
    const uint8_t* status, const int32_t* n_children, const float* noise, const adp_params* prm,
    int32_t step, int32_t* d_step, const float* lr, float beta1, float beta2, float eps,
    adp_gaussians* out, adp_gaussians* m_out, adp_gaussians* v_out, void* ws, size_t ws_bytes,
    adp_stream_t stream) {
  return split_overlapped_part(g, grad, m_in, v_in, regs, candidates, n_cand, status, n_children,
                               noise, prm, step, d_step, lr, beta1, beta2, eps, out, m_out, v_out,
                               ws, ws_bytes, stream, ApplyPart::KEEP);
}

extern "C" ADP_API int adp_split_append_overlapped(
    const adp_gaussians* g, const adp_gaussians* grad, const adp_gaussians* m_in,
    const adp_gaussians* v_in, const adp_regions* regs, const int32_t* candidates, int64_t n_cand,
    const uint8_t* status, const int32_t* n_children, const float* noise, const adp_params* prm,
    int32_t step, int32_t* d_step, const float* lr, float beta1, float beta2, float eps,
    adp_gaussians* out, adp_gaussians* m_out, adp_gaussians* v_out, void* ws, size_t ws_bytes,
    adp_stream_t stream) {
  return split_overlapped_part(g, grad, m_in, v_in, regs, candidates, n_cand, status, n_children,
                               noise, prm, step, d_step, lr, beta1, beta2, eps, out, m_out, v_out,
                               ws, ws_bytes, stream, ApplyPart::APPEND);
}

// ------------------------------------------------------------------ clone

namespace adp {

// Copies of the listed Gaussians appended after the split's rows: each copy is
// the Gaussian's kept row of the new population (after any Adam step the
// compaction applied), with zero moments. Nothing is written if the result does
// not fit.
__global__ void clone_kernel(const int* ids, const long long* d_n_clone, long long max_clone,
                             long long n, const unsigned* dest, const long long* counters,
                             GaussPtrs pop, GaussPtrs mout, GaussPtrs vout, bool has_m,
                             bool has_v, int planes) {
  long long nc = *d_n_clone;
  if (nc > max_clone) nc = max_clone;
  const long long base = counters[3];
  if (base + nc > pop.n) return;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc;
       t += (long long)gridDim.x * blockDim.x) {
    const int id = ids[t];
    const unsigned d = (id >= 0 && id < n) ? dest[id] : 0xffffffffu;
    const long long j = base + t;
    if (d >> 31) {  // a split candidate (not a kept row) or no id: an all-zero row
      zero_gauss(pop, j, planes);
    } else {
      copy_gauss(pop, (long long)d, pop, j, planes);
    }
    if (has_m) zero_gauss(mout, j, planes);
    if (has_v) zero_gauss(vout, j, planes);
  }
}

__global__ void clone_size_kernel(const long long* d_n_clone, long long max_clone,
                                  const long long* counters, int64_t* d_new_n) {
  long long nc = *d_n_clone;
  if (nc > max_clone) nc = max_clone;
  *d_new_n = counters[3] + nc;
}

}  // namespace adp

extern "C" ADP_API int adp_split_clone(int64_t n, int64_t n_cand, int64_t region_capacity,
                                       const int32_t* clone_ids, const int64_t* d_n_clone,
                                       int64_t max_clone, adp_gaussians* pop, adp_gaussians* m_out,
                                       adp_gaussians* v_out, void* ws, size_t ws_bytes,
                                       int64_t* d_new_n, adp_stream_t stream) {
  ADP_CHECK_ARG(pop && d_new_n && d_n_clone, "NULL argument");
  ADP_CHECK_ARG(gauss_ok(pop) || pop->n == 0, "bad population arrays");
  ADP_CHECK_ARG(n >= 0 && n < (1LL << 31) && n_cand >= 0 && region_capacity >= 0, "bad sizes");
  ADP_CHECK_ARG(max_clone >= 0 && max_clone <= n, "max_clone out of range");
  ADP_CHECK_ARG(max_clone == 0 || clone_ids, "NULL clone ids");
  ADP_CHECK_ARG(!m_out || (gauss_ok(m_out) && m_out->n == pop->n), "bad m_out");
  ADP_CHECK_ARG(!v_out || (gauss_ok(v_out) && v_out->n == pop->n), "bad v_out");
  ADP_CHECK_ARG(aligned(ws, 256), "workspace must be 256-byte aligned");
  const size_t need = split_ws_bytes(n, n_cand, region_capacity);
  ADP_CHECK_ARG(ws_bytes >= need, "workspace %zu bytes, need %zu", ws_bytes, need);
  cudaStream_t st = (cudaStream_t)stream;
  Carver c(ws, ws_bytes);
  SplitWs w = carve_split(c, n, n_cand, region_capacity);
  const int planes = sh_planes(pop->sh_degree);
  GaussPtrs mo = {}, vo = {};
  if (m_out) mo = gp_of(m_out);
  if (v_out) vo = gp_of(v_out);
  if (max_clone > 0)
    clone_kernel<<<grid_for(max_clone, 256, 148 * 16), 256, 0, st>>>(
        clone_ids, (const long long*)d_n_clone, max_clone, (long long)n, w.dest, w.counters,
        gp_of(pop), mo, vo,
        m_out != nullptr, v_out != nullptr, planes);
  clone_size_kernel<<<1, 1, 0, st>>>((const long long*)d_n_clone, max_clone, w.counters, d_new_n);
  ADP_LAUNCH_CHECK();
  return ADP_OK;
}

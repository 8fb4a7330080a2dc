/*
 * adpsplit.h -- C ABI of the B300 (sm_103a) implementation of the AdpSplit hot
 * path: projection, tile binning, front-to-back compositing with the dominant
 * Gaussian map, the L1 error statistics, the AdpSplit operator with compaction of
 * the Gaussian arrays, the hand-written render backward and Adam.
 *
 * Conventions shared by every call
 *  - Pointers inside the structs and the array arguments are DEVICE pointers
 *    owned by the caller, unless a parameter says "host". The library allocates
 *    no device memory: scratch space comes from the caller as a workspace whose
 *    size a *_workspace_size() query returns (adp_select_topk_noalloc instead
 *    uses one statically allocated device array, see there). float4 arrays must
 *    be 16-byte aligned, workspaces 256-byte aligned.
 *  - Every call is asynchronous on the given stream (a cudaStream_t; NULL is the
 *    legacy default stream) and does not synchronise, except adp_split_plan,
 *    which reads one integer back when asked to (see there). The overlapped
 *    split (adp_split_plan_overlapped or its second part, and its two compaction
 *    calls) and the batched step (adp_train_step_batched) also put work on a
 *    stream the library keeps per device, forked from and joined back into the
 *    given stream (see there).
 *  - Every call returns an adp_status. A host-side argument error returns
 *    ADP_ERR_INVALID_ARG before anything is launched; a CUDA launch error returns
 *    ADP_ERR_CUDA. adp_last_error_string() describes the last failure of the
 *    calling thread. No C++ exception crosses the ABI.
 *  - Conditions only the device can see (an instance or region count beyond the
 *    capacity the caller gave) are reported through device counters that hold
 *    the REQUIRED size; the caller compares them with its capacity after a sync
 *    and calls again with more room. Kernels never write past a capacity.
 *  - Device status word. The calls whose kernels wait on other blocks (the
 *    look-back of their prefix sums, the grid barrier of the top-k) take an
 *    int32_t* d_status (device, may be NULL). Every such wait is bounded (see
 *    adp_set_spin_limit); one that runs out sets *d_status to ADP_ERR_TIMEOUT if
 *    it is still ADP_OK (0), and the kernel returns normally, so the context
 *    stays usable. The call's outputs are then undefined, and the calls that
 *    write through the affected prefix sums write nothing past their
 *    capacities. The word is never cleared by the library: the caller zeroes it,
 *    passes it to the calls of a step and reads it at the step's sync point.
 *  - Up to ADP_MAX_VIEWS views per call. Camera structs are HOST memory and are
 *    passed to the kernels by value.
 *  - The library caches per device, for the life of the process, the auxiliary
 *    stream of the overlapped split and the device address of the static top-k
 *    scratch. Both belong to the device's primary context, so the library must
 *    not be used on a device after cudaDeviceReset on it.
 *
 * Notation follows the paper (AdpSplit, Secs. 3-4 and Appendix A).
 */
#ifndef ADPSPLIT_H
#define ADPSPLIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADP_API __attribute__((visibility("default")))
#define ADP_MAX_VIEWS 32
#define ADP_VERSION 2

typedef void* adp_stream_t; /* cudaStream_t */

typedef enum adp_status {
  ADP_OK = 0,
  ADP_ERR_INVALID_ARG = 1, /* bad sizes, NULL pointers, misalignment, small workspace */
  ADP_ERR_CAPACITY = 2,    /* a caller-given capacity is too small (host-detected) */
  ADP_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  ADP_ERR_TIMEOUT = 4,     /* a bounded device wait gave up (reported in a status word) */
  ADP_ERR_NUMERIC = 5      /* reserved: non-finite input detected */
} adp_status;

/* Split status of one candidate (Sec. 5.1). */
enum {
  ADP_KEEP = 0,     /* not a candidate */
  ADP_ADAPTIVE = 1, /* N_i >= 1 children from error regions plus a parent copy */
  ADP_FALLBACK = 2, /* no error pixel attributed in any view: vanilla split, N = 2 */
  ADP_RESET = 3     /* pixels attributed but no region survived: kept, status reset */
};

/* OpenCV pinhole camera: x right, y down, z forward. A world point X maps to
 * camera point R X + t (R row-major); pixel (x, y) has its centre at image
 * coordinate (x, y); (px, py) is the principal point. Host memory. */
typedef struct adp_camera {
  int32_t width, height;
  float fx, fy, px, py;
  float R[9];
  float t[3];
} adp_camera;

/* Hyper-parameters. adp_default_params() fills the paper's defaults (Sec. 5.1):
 * tau_l1 0.1, r_erode 2, m_min 5, n_levels 3, n_max 19, gamma_d 2.0, gamma_c
 * 0.15; eta 0.8 and the forward constants are the 3DGS ones the paper keeps. */
typedef struct adp_params {
  float tau_l1;      /* normalised L1 error threshold of the mask M (Eq. 6) */
  int32_t r_erode;   /* erosion radius: (2r+1)^2 square window, 0 = off */
  int32_t m_min;     /* minimum region area (Eq. 8) */
  int32_t n_levels;  /* L error bands over [tau_l1, 1] */
  int32_t n_max;     /* child cap per parent */
  float gamma_d;     /* merge distance threshold (Eq. 11) */
  float gamma_c;     /* merge colour threshold (Eq. 11) */
  float eps_t;       /* epsilon of Eq. 10 */
  float eta;         /* vanilla split shrink factor (Eq. 4) */
  float scale_floor; /* lower bound on initialised child scales */
  float near_plane;  /* cull at camera depth <= near_plane */
  float low_pass;    /* added to the 2D covariance diagonal */
  float alpha_min;   /* contribution threshold 1/255 */
  float alpha_max;   /* alpha clamp 0.99 */
  float t_min;       /* stop before blending when T (1 - alpha) < t_min */
  int32_t tile_w;    /* tile width in pixels; tile_w * tile_h must be 256 */
  int32_t tile_h;
  int32_t batch;     /* Gaussians a compositing block stages per batch: 64, 128 or 256
                        (0 = 256); changes no result, only the speed */
} adp_params;

/* Gaussian parameters (also the layout of gradients and Adam moments), SoA of
 * float4 planes, n entries each:
 *   mean_logit[i] = (x, y, z, opacity logit)      opacity o = sigmoid(logit)
 *   logscale[i]   = (log sx, log sy, log sz, 0)  scale s = exp(log s)
 *   quat[i]       = (w, x, y, z)                 normalised before use
 *   sh[p * n + i] = floats 4p..4p+3 of the SH list of Gaussian i, where float
 *                   3k + ch is coefficient k of channel ch, k < K = (deg+1)^2;
 *                   there are ceil(3K / 4) planes (1 for degree 0, 12 for 3).
 * rows (gradients only; NULL for parameters and moments): an optional device
 * byte per row. When non-NULL, a row with rows[i] == 0 is zero by definition
 * and the library neither reads nor writes its planes: adp_render_backward then
 * writes the mask itself (1 for every Gaussian rendered in at least one view)
 * instead of zeroing the other rows, and the Adam entry points skip the
 * gradient reads of masked-out rows. Rows of Gaussians that no view renders are
 * most rows of a large scene, so this saves two passes over their planes. */
typedef struct adp_gaussians {
  int64_t n;
  int32_t sh_degree; /* 0..3 */
  int32_t reserved;
  float* mean_logit;
  float* logscale;
  float* quat;
  float* sh;
  uint8_t* rows;
} adp_gaussians;

/* Projected Gaussians, one record per (view v, Gaussian i) at index v * n + i.
 * A culled record has tiles_touched = 0; its other fields are unspecified. */
typedef struct adp_projected {
  float* xy_opacity_depth; /* float4: 2D mean x, y; opacity; camera depth */
  float* conic;            /* float4: A, B, C, 0 -- inverse 2D covariance [[A, B], [B, C]] */
  float* rgb;              /* float4: r, g, b, m -- SH colour for this view, clamped at 0;
                              m = the clamped channels as a number 0..7 (bit c: channel c < 0) */
  int32_t* rect;           /* int4: tile x0, x1, y0, y1 (inclusive) of the pixel box */
  int32_t* tiles_touched;  /* number of tiles of rect; 0 = not rendered */
} adp_projected;

/* Tile bins. Tiles are numbered view by view, row-major within a view. */
typedef struct adp_bins {
  int64_t capacity;      /* length of inst_gauss */
  int32_t* inst_gauss;   /* Gaussian id per instance, ordered by (view, tile, depth, id) */
  int32_t* tile_range;   /* [n_tiles_total][2]: [start, end) into inst_gauss */
  int64_t* n_instances;  /* [1]: instances required (> capacity means overflow) */
} adp_bins;

/* Per-pixel render outputs; views are concatenated, each row-major. */
typedef struct adp_image {
  float* rgb;         /* [P][3] composited colour + T_final * background */
  float* T_final;     /* [P] transmittance after the last blended Gaussian */
  int32_t* n_contrib; /* [P] number of blended Gaussians */
  int32_t* last;      /* [P] one past the tile-list position of the last blended Gaussian */
  int32_t* dominant;  /* [P] Eq. 5: Gaussian with the largest T alpha, -1 if none */
} adp_image;

/* Error maps of Eq. 6. mask bits: 0 = M (E > tau_l1), 1 = eroded M,
 * 4..7 = band B (0 where M = 0). */
typedef struct adp_error_maps {
  float* E;      /* [P] normalised L1 error (float32 decisions) */
  uint8_t* mask; /* [P] */
  float* minmax; /* [n_views][2] min and max of the raw L1 error per view */
} adp_error_maps;

/* Kept error regions (Eqs. 7-8) with their statistics (Sec. 4.1), ordered by
 * (view, label). stats = (cx, cy, cov_xx, cov_xy, cov_yy, e1x, e1y, sigma1,
 * sigma2, r, g, b): centroid, population covariance, major PCA axis with
 * e1x > 0 (or e1y > 0 if e1x = 0), standard deviations along e1 and
 * e2 = (-e1y, e1x), target RGB at the pixel nearest the centroid. */
typedef struct adp_regions {
  int64_t capacity;
  int32_t* view;
  int32_t* parent;   /* the dominant Gaussian of the region */
  int32_t* label;    /* smallest linear pixel index y * W + x in the region */
  int32_t* band;
  int64_t* moments;  /* [cap][6]: A, sum x, sum y, sum x^2, sum xy, sum y^2 */
  double* stats;     /* [cap][12] */
  int64_t* count;    /* [1]: kept regions (> capacity means overflow) */
  int32_t* labels;   /* optional [P]: label of every participating pixel, else -1 */
} adp_regions;

ADP_API int32_t adp_version(void);
ADP_API void adp_default_params(adp_params* p);
ADP_API const char* adp_last_error_string(void);

/* Constants fixed inside the library (host query, no device needed): limits,
 * the conventions the paper leaves open that the kernels hard-code, and the
 * default parameters. */
typedef struct adp_constants {
  int32_t version;           /* ADP_VERSION */
  int32_t max_views;         /* ADP_MAX_VIEWS */
  int32_t tile_pixels;       /* pixels of a tile (tile_w * tile_h) */
  int32_t max_sh_degree;     /* 3 */
  float fov_clamp;           /* x/z and y/z of the EWA Jacobian are clamped to
                                fov_clamp * (image side / 2) / focal length */
  float sh_coef[16];         /* real SH basis: Y_k(d) = sh_coef[k] * m_k(d) with the
                                monomials m = 1, y, z, x, xy, yz, 2z^2-x^2-y^2, xz,
                                x^2-y^2, y(3x^2-y^2), xyz, y(4z^2-x^2-y^2),
                                z(2z^2-3x^2-3y^2), x(4z^2-x^2-y^2), z(x^2-y^2),
                                x(x^2-3y^2) (3DGS sign convention) */
  double gram_schmidt_eps;   /* residual below which Appendix A's in-plane axis
                                falls back to z x u1 */
  int64_t topk_noalloc_max_n;  /* ADP_TOPK_NOALLOC_MAX_N */
  int64_t default_spin_limit;  /* poll bound of device waits by default */
  adp_params defaults;       /* adp_default_params() */
} adp_constants;
ADP_API void adp_get_constants(adp_constants* c);

/* Bound on the polls of every device wait launched after the call, process
 * wide (max_polls <= 0 restores the default, about a second of polling). A
 * small bound makes waits give up and report ADP_ERR_TIMEOUT (a test of the
 * failure path); results of calls that timed out are undefined. */
ADP_API void adp_set_spin_limit(int64_t max_polls);

/* --- Projection (Sec. 3, Eq. 1). ------------------------------------------
 * EWA splatting of every Gaussian into every view: camera transform, 3D
 * covariance R S S^T R^T, Sigma2D = J W Sigma W^T J^T + low_pass I with x/z and
 * y/z clamped to 1.3x the half field of view in J, conic = Sigma2D^-1, opacity
 * sigmoid(logit), SH colour along the ray from the camera centre, and the pixel
 * box of the ellipse o exp(-d^T C d / 2) >= alpha_min. Culls depth <= near_plane,
 * det(Sigma2D) <= 0, o < alpha_min and boxes outside the image.
 * out: n_views * g->n records. */
ADP_API int adp_project(const adp_gaussians* g, const adp_camera* cams, int32_t n_views,
                        const adp_params* prm, adp_projected* out, adp_stream_t stream);

/* --- Tile binning and depth sort (Eq. 1 depth order). -----------------------
 * Sorts the visible (view, Gaussian) records by (view, depth, id), duplicates
 * each into the tiles of its rect and sorts the instances stably by tile, so each
 * tile's list is ordered by (depth, id); writes tile ranges. A tile's list holds
 * the Gaussians whose alpha ellipse o exp(-d^T C d / 2) >= alpha_min can reach
 * one of its pixel centres (a conservative float32 test: every contributing
 * Gaussian is listed, and no listed one contributes to a pixel it cannot reach).
 * If the instance count (all tiles of every rect) exceeds bins->capacity
 * nothing past the capacity is written and *bins->n_instances holds the
 * required size. */
ADP_API size_t adp_bin_sort_workspace_size(int64_t n, int32_t n_views, int64_t capacity);
ADP_API int adp_bin_sort(int64_t n, const adp_projected* pr, const adp_camera* cams,
                         int32_t n_views, const adp_params* prm, adp_bins* bins, void* ws,
                         size_t ws_bytes, int32_t* d_status, adp_stream_t stream);

/* --- Compositing (Eq. 1) and dominant map (Eq. 5). --------------------------
 * Per pixel, front to back over its tile's list: alpha = min(alpha_max,
 * o exp(power)), skipped below alpha_min, stop before blending once
 * T (1 - alpha) < t_min. bg: host float[3] background. */
ADP_API int adp_render(int64_t n, const adp_projected* pr, const adp_bins* bins,
                       const adp_camera* cams, int32_t n_views, const float* bg,
                       const adp_params* prm, adp_image* out, adp_stream_t stream);

/* --- Error statistics (Eq. 6, Sec. 4.1, Sec. 5.1). --------------------------
 * Per view: raw L1 = |I^ - I_gt|_1 over RGB, min-max normalised to E,
 * M = [E > tau_l1], band B = min(L-1, floor(L (E - tau)/(1 - tau))); then every
 * pixel with M = 1 and a dominant Gaussian i adds 1 to count[i] and E to
 * mass[i] (summed over views; mass is exact: E is a float32 in (0.1, 1]).
 * count and mass are zeroed by the call. img, target: [P][3] float32. */
ADP_API size_t adp_error_stats_workspace_size(int32_t n_views, const adp_camera* cams);
ADP_API int adp_error_stats(const float* img, const float* target, const int32_t* dominant,
                            int64_t n, const adp_camera* cams, int32_t n_views,
                            const adp_params* prm, adp_error_maps* maps, int32_t* count,
                            double* mass, adp_stream_t stream);

/* The k Gaussians with the largest mass (ties to the lower id), written to
 * out_ids in ascending id order. If a grid-barrier wait runs out (d_status),
 * every entry is a distinct id or -1. */
ADP_API size_t adp_select_topk_workspace_size(int64_t n);
ADP_API int adp_select_topk(const double* mass, int64_t n, int64_t k, int32_t* out_ids,
                            void* ws, size_t ws_bytes, int32_t* d_status, adp_stream_t stream);

/* The same selection for callers that cannot allocate device memory where they
 * run (no cudaMalloc, no caller workspace): for example code running inside a
 * custom device allocator or a memory pool's callback, a host framework that
 * caps or forbids allocations mid-step, or a library layer that holds no
 * allocator of its own. The paper has no counterpart; this is an
 * integration convenience. Scratch comes from a statically allocated device
 * array sized for n <= ADP_TOPK_NOALLOC_MAX_N (about 4 MiB, held by every
 * device that loads the library until the process exits); larger n returns
 * ADP_ERR_INVALID_ARG. The first call on each device looks up that array's
 * device address (cudaGetSymbolAddress, with the device current); make that
 * first call before any stream capture. All calls share the one array, whose
 * contents persist from call to call (the call resets what must start at
 * zero): calls that can overlap on the GPU (different streams, or different
 * host threads, on the same device) race and must be serialised by the
 * caller. Results are identical to adp_select_topk's. */
#define ADP_TOPK_NOALLOC_MAX_N (1LL << 22)
ADP_API int adp_select_topk_noalloc(const double* mass, int64_t n, int64_t k, int32_t* out_ids,
                                    int32_t* d_status, adp_stream_t stream);

/* Error regions (Eqs. 7-8): erode M by the (2 r_erode + 1)^2 square (pixels
 * outside the image count as set), then join 8-neighbours whose eroded M is set,
 * whose dominant Gaussian is the same split candidate and whose band is equal;
 * keep components with area >= m_min and compute their statistics. Sets mask
 * bit 1. candidates: device, ascending ids. */
ADP_API size_t adp_error_regions_workspace_size(int64_t n, int32_t n_views, const adp_camera* cams);
ADP_API int adp_error_regions(adp_error_maps* maps, const int32_t* dominant, const float* target,
                              int64_t n, const adp_camera* cams, int32_t n_views,
                              const int32_t* candidates, int64_t n_cand, const adp_params* prm,
                              adp_regions* out, void* ws, size_t ws_bytes, int32_t* d_status,
                              adp_stream_t stream);

/* --- The AdpSplit operator (Sec. 4, Sec. 5.1, Appendix A). ------------------
 * Two phases sharing one workspace, which must not change in between.
 * Plan: per candidate (device list, strictly ascending ids) its status and
 * child count: FALLBACK if count[i] == 0, RESET if no region of i survives,
 * else ADAPTIVE: one proposal per region (Eqs. 9-10, Appendix A), merged per
 * parent across views (Eqs. 11-12), capped at n_max by sqrt(det Sigma) (ties to
 * the earlier group), children in first-member (view, label) order. Computed in
 * FP64. Writes status[n_cand], n_children[n_cand] and *d_new_n; if h_new_n is
 * non-NULL the call copies the size back and synchronises the stream.
 * Apply: writes the new population into out, whose n is its CAPACITY (plane
 * stride); the population occupies entries [0, *d_new_n). If the planned size
 * exceeds out->n nothing is written (compare *d_new_n with out->n after a
 * sync), so a caller may pass buffers sized for the largest possible result,
 * n + n_cand * (n_max + 1), and never synchronise. Order: every non-candidate
 * and RESET Gaussian in id order with its Adam moments, then per candidate in
 * ascending id [parent copy with opacity o/(N_i + 1), children] or the two
 * vanilla children mu + R (s * noise), s / (2 eta) (Eqs. 3-4), all with zero
 * moments. noise: [n_cand][2][3] standard normal. m_in/v_in/m_out/v_out may be
 * NULL to skip the moments; m_out and v_out have out->n entries. No output array
 * may share a plane with an input array (ADP_ERR_INVALID_ARG). */
ADP_API size_t adp_split_workspace_size(int64_t n, int64_t n_cand, int64_t region_capacity);
ADP_API int adp_split_plan(const adp_gaussians* g, const adp_camera* cams, int32_t n_views,
                           const adp_regions* regs, const int32_t* candidates, int64_t n_cand,
                           const int32_t* count, const adp_params* prm, uint8_t* status,
                           int32_t* n_children, int64_t* d_new_n, int64_t* h_new_n, void* ws,
                           size_t ws_bytes, int32_t* d_status, adp_stream_t stream);
ADP_API int adp_split_apply(const adp_gaussians* g, const adp_gaussians* m_in,
                            const adp_gaussians* v_in, const adp_regions* regs,
                            const int32_t* candidates, int64_t n_cand, const uint8_t* status,
                            const int32_t* n_children, const float* noise, const adp_params* prm,
                            adp_gaussians* out, adp_gaussians* m_out, adp_gaussians* v_out,
                            void* ws, size_t ws_bytes, adp_stream_t stream);
/* The compaction with the step's Adam update fused into it (one pass over the
 * parameters and moments instead of two). Equivalent, bit for bit, to
 * adp_adam_step on every row of g followed by adp_split_plan and
 * adp_split_apply, provided the candidate rows got their step first from
 * adp_adam_step_rows (the plan reads the candidates' updated parameters): each
 * kept non-candidate row is read with its gradient grad (same layout as g) and
 * moments, updated, and written to its new row; RESET candidates are copied as
 * they are; appended rows are as in adp_split_apply. m_in, v_in, m_out and v_out
 * are required. step, d_step, lr, beta1, beta2, eps as in adp_adam_step; the
 * call advances *d_step after the compaction. If the planned size exceeds
 * out->n nothing is written and the non-candidate rows keep their old state (a
 * caller that sizes out for n + n_cand * (n_max + 1) never meets this). */
ADP_API int adp_split_apply_adam(const adp_gaussians* g, const adp_gaussians* grad,
                                 const adp_gaussians* m_in, const adp_gaussians* v_in,
                                 const adp_regions* regs, const int32_t* candidates,
                                 int64_t n_cand, const uint8_t* status,
                                 const int32_t* n_children, const float* noise,
                                 const adp_params* prm, int32_t step, int32_t* d_step,
                                 const float* lr, float beta1, float beta2, float eps,
                                 adp_gaussians* out, adp_gaussians* m_out, adp_gaussians* v_out,
                                 void* ws, size_t ws_bytes, adp_stream_t stream);

/* The same plan and fused compaction as adp_split_plan + adp_split_apply_adam,
 * with identical results, split so that the plan's proposals and merges (Eqs.
 * 9-12, small FP64 kernels) run while the compaction streams the kept rows.
 * adp_split_plan_overlapped enqueues on `stream` the part that needs no
 * proposal (statuses, the new row of every kept Gaussian and a bound on the new
 * size: n + sum over ADAPTIVE candidates of min(regions, n_max) + the FALLBACK
 * count), then the proposals, merges, child counts and the new size on the
 * library's auxiliary stream of the current device (highest priority), which
 * waits for that part. adp_split_keep_overlapped writes the kept rows (with
 * their Adam step) on `stream` when the bound fits out->n. adp_split_append_
 * overlapped makes `stream` wait for the auxiliary stream, appends the new rows
 * (and writes the kept rows there if only the exact size fits) and advances
 * *d_step. status is ready in stream order after the plan; n_children,
 * *d_new_n and the population only after the append call. Constraints: the
 * three calls come in this order, on one stream and device, from one host
 * thread, with no other overlapped plan of that device in between, and with
 * identical arguments for the last two; the first overlapped plan on a device
 * creates the auxiliary stream and its two events, so it must come before any
 * stream capture that includes these calls (inside a capture the auxiliary
 * stream joins the capture as a forked stream). The workspace is that of
 * adp_split_plan. Arguments, ownership and errors as in adp_split_plan (without
 * h_new_n) and adp_split_apply_adam.
 * adp_split_plan_overlapped is adp_split_plan_statuses followed by
 * adp_split_plan_proposals_overlapped on the same stream, with the same
 * arguments. A caller may instead make the two calls itself. The first enqueues
 * the part that needs no proposal on its `stream`. It reads the candidates, the
 * regions and count, but no parameter of g (only g->n), so it may run on another
 * stream before the candidates' Adam step (adp_adam_step_rows), e.g. beside the
 * render backward. The second forks the proposals and merges onto the auxiliary
 * stream after the work already enqueued on its `stream`. That stream must by
 * then be ordered after the first call (an event) and after adp_adam_step_rows.
 * The keep and append calls then follow on that stream as above. Between the
 * two calls nothing else may use the workspace. */
ADP_API int adp_split_plan_overlapped(const adp_gaussians* g, const adp_camera* cams,
                                      int32_t n_views, const adp_regions* regs,
                                      const int32_t* candidates, int64_t n_cand,
                                      const int32_t* count, const adp_params* prm,
                                      uint8_t* status, int32_t* n_children, int64_t* d_new_n,
                                      void* ws, size_t ws_bytes, int32_t* d_status,
                                      adp_stream_t stream);
ADP_API int adp_split_plan_statuses(const adp_gaussians* g, const adp_camera* cams,
                                    int32_t n_views, const adp_regions* regs,
                                    const int32_t* candidates, int64_t n_cand,
                                    const int32_t* count, const adp_params* prm, uint8_t* status,
                                    int32_t* n_children, int64_t* d_new_n, void* ws,
                                    size_t ws_bytes, int32_t* d_status, adp_stream_t stream);
ADP_API int adp_split_plan_proposals_overlapped(
    const adp_gaussians* g, const adp_camera* cams, int32_t n_views, const adp_regions* regs,
    const int32_t* candidates, int64_t n_cand, const int32_t* count, const adp_params* prm,
    uint8_t* status, int32_t* n_children, int64_t* d_new_n, void* ws, size_t ws_bytes,
    int32_t* d_status, adp_stream_t stream);
ADP_API int adp_split_keep_overlapped(
    const adp_gaussians* g, const adp_gaussians* grad, const adp_gaussians* m_in,
    const adp_gaussians* v_in, const adp_regions* regs, const int32_t* candidates, int64_t n_cand,
    const uint8_t* status, const int32_t* n_children, const float* noise, const adp_params* prm,
    int32_t step, int32_t* d_step, const float* lr, float beta1, float beta2, float eps,
    adp_gaussians* out, adp_gaussians* m_out, adp_gaussians* v_out, void* ws, size_t ws_bytes,
    adp_stream_t stream);
ADP_API int adp_split_append_overlapped(
    const adp_gaussians* g, const adp_gaussians* grad, const adp_gaussians* m_in,
    const adp_gaussians* v_in, const adp_regions* regs, const int32_t* candidates, int64_t n_cand,
    const uint8_t* status, const int32_t* n_children, const float* noise, const adp_params* prm,
    int32_t step, int32_t* d_step, const float* lr, float beta1, float beta2, float eps,
    adp_gaussians* out, adp_gaussians* m_out, adp_gaussians* v_out, void* ws, size_t ws_bytes,
    adp_stream_t stream);

/* --- Render backward. -------------------------------------------------------
 * Gradient of L = sum over views of the mean L1 error |I^ - I_gt| over pixels
 * and channels (sign(0) = 0), or, if dL_drgb is non-NULL, of the upstream
 * gradient dL_drgb [P][3], with respect to every parameter. Per tile, back to
 * front, transmittance recovered from T_final by division; the derivative is
 * exact for the forward as defined (zero through the alpha clamp, the colour
 * clamp at 0 and the clamped x/z, y/z of J). grad is zeroed and written; the
 * per-view 2D gradients are summed over views.
 * grad2d_accum [n] float, grad2d_visits [n] int32 (both or neither, may be NULL):
 * the image-space statistic of the adaptive density control (Sec. 3, Eq. 2). For
 * every Gaussian rendered in a view, the call ADDS to grad2d_accum[i] the norm of
 * dL/d(projected 2D mean) in normalised device coordinates (pixel gradient times
 * W/2 and H/2) and 1 to grad2d_visits[i]; the caller zeroes both at the start of
 * a densification interval, and g_i = accum / visits is the average of Eq. 2. */
ADP_API size_t adp_render_backward_workspace_size(int64_t n, int32_t n_views);
ADP_API int adp_render_backward(const adp_gaussians* g, const adp_projected* pr,
                                const adp_bins* bins, const adp_image* fwd, const float* target,
                                const float* dL_drgb, const adp_camera* cams, int32_t n_views,
                                const float* bg, const adp_params* prm, adp_gaussians* grad,
                                float* grad2d_accum, int32_t* grad2d_visits, void* ws,
                                size_t ws_bytes, adp_stream_t stream);

/* --- The batched step of many views (Sec. 4.1: the V views sampled per
 * densification step; loss and gradient unchanged, Sec. 5.1). ---------------
 * For n_views views (up to ADP_MAX_VIEWS, uneven sizes allowed): adp_project and
 * adp_bin_sort of all views, then ONE persistent kernel over a work queue of
 * (view, tile) items that per tile composites the forward (Eq. 1, dominant map of
 * Eq. 5), writes the raw L1 error |I^ - I_gt|_1 and reduces the view's min/max
 * (Eq. 6), and walks the tile's list back to front for the gradient of the L1
 * loss with the final transmittance and dL/dpixel still in registers; then E, M,
 * B with the per-Gaussian count and mass (as adp_error_stats) and the
 * per-Gaussian chain rule summed over views (as adp_render_backward). Every
 * output equals that of adp_project, adp_bin_sort, adp_render, adp_error_stats
 * and adp_render_backward called on the same views (bit for bit, except the
 * gradient, whose float atomics sum in another order). Arguments are those
 * calls': pr (n_views * n records), bins (capacity buffers; an overflow bins
 * nothing and leaves the required size in *bins->n_instances), img and maps (all
 * views' pixels), count and mass (n, zeroed by the call), grad (zeroed or masked
 * rows), the optional Eq. 2 accumulators, d_status (see the conventions). The
 * workspace size depends on n, n_views and bins->capacity (0 for invalid
 * arguments). Asynchronous and capturable in a CUDA graph. The error
 * normalisation runs on the library's auxiliary stream of the device, forked from
 * `stream` after the per-tile kernel and joined back before the call returns (as
 * in the overlapped split); the first call on a device creates that stream, so it
 * must come before any stream capture that includes the call. */
ADP_API size_t adp_train_step_batched_workspace_size(int64_t n, int32_t n_views,
                                                     const adp_camera* cams,
                                                     const adp_params* prm, int64_t capacity);
ADP_API int adp_train_step_batched(const adp_gaussians* g, const adp_camera* cams, int32_t n_views,
                                   const float* target, const float* bg, const adp_params* prm,
                                   adp_projected* pr, adp_bins* bins, adp_image* img,
                                   adp_error_maps* maps, int32_t* count, double* mass,
                                   adp_gaussians* grad, float* grad2d_accum,
                                   int32_t* grad2d_visits, void* ws, size_t ws_bytes,
                                   int32_t* d_status, adp_stream_t stream);

/* --- Adaptive density control candidates (Sec. 3, Eq. 2). -------------------
 * With g_i = grad2d_accum[i] / grad2d_visits[i] (0 when never visited; one
 * correctly rounded float32 division), Gaussian i is a split candidate iff
 * g_i >= tau_g and max(s_i) > tau_s (Eq. 2), and a clone candidate iff
 * g_i >= tau_g and max(s_i) <= tau_s (the high-gradient Gaussians of small scale
 * the baselines clone). The scale test is made on the stored log-scales against
 * ln(tau_s) rounded to float32. Writes the split ids and the clone ids in
 * ascending order (each list has room for n entries; entries past the count are
 * set to -1) and their counts to d_counts[0], d_counts[1] (device int64); no host
 * synchronisation. The split list is the candidate list of adp_error_regions and
 * adp_split_plan, which may be given whole, with n_cand = n: those calls skip -1
 * entries (a -1 candidate gets status ADP_KEEP and no children). */
ADP_API size_t adp_densify_select_workspace_size(int64_t n);
ADP_API int adp_densify_select(const float* grad2d_accum, const int32_t* grad2d_visits,
                               const adp_gaussians* g, float tau_g, float tau_s,
                               int32_t* split_ids, int32_t* clone_ids, int64_t* d_counts,
                               void* ws, size_t ws_bytes, int32_t* d_status,
                               adp_stream_t stream);
/* Clone (the baselines' operation for small high-gradient Gaussians, Sec. 3):
 * called after adp_split_apply or adp_split_apply_adam with the same workspace
 * and the same n (population before the split), n_cand and region capacity. It
 * appends to the new population pop (capacity pop->n) a copy of each listed
 * Gaussian -- its kept row in pop, so after any Adam step the compaction applied
 * -- at rows [planned size, planned size + count), with zero moments in m_out and
 * v_out (optional), and sets *d_new_n to the new size. count is *d_n_clone
 * (device int64), at most max_clone; ids are ids of the population before the
 * split and must not be split candidates (such an entry gives an all-zero row).
 * If the result does not fit in pop->n, nothing is written and *d_new_n holds the
 * required size. */
ADP_API int adp_split_clone(int64_t n, int64_t n_cand, int64_t region_capacity,
                            const int32_t* clone_ids, const int64_t* d_n_clone, int64_t max_clone,
                            adp_gaussians* pop, adp_gaussians* m_out, adp_gaussians* v_out,
                            void* ws, size_t ws_bytes, int64_t* d_new_n, adp_stream_t stream);

/* --- D-SSIM loss term (the baselines' loss, unchanged by the paper, Sec. 5.1).
 * Per view, L = (1 - lambda) mean|I^ - I_gt| + lambda (1 - SSIM), SSIM averaged
 * over the view's pixels and the three channels, each channel under an 11x11
 * Gaussian window (sigma 1.5, zero padding outside the image), C1 = 0.01^2,
 * C2 = 0.03^2. Writes dL/dI^ (float [P][3]) for adp_render_backward's dL_drgb
 * (sign(0) = 0 in the L1 term). loss (device double [V][2], may be NULL) receives
 * each view's mean L1 error and mean SSIM. Workspace: 36 bytes per pixel. */
ADP_API size_t adp_dssim_workspace_size(int32_t n_views, const adp_camera* cams);
ADP_API int adp_dssim_loss_grad(const float* img, const float* target, const adp_camera* cams,
                                int32_t n_views, float lambda, const adp_params* prm,
                                float* dL_drgb, double* loss, void* ws, size_t ws_bytes,
                                adp_stream_t stream);

/* --- Adam (the baselines' optimizer, unchanged by the paper, Sec. 5.1). -----
 * In place, bias-corrected. The step number t >= 1 is `step`, or, if d_step
 * (device int32) is non-NULL, *d_step, which the call then increments on the
 * device -- so a step replayed from a captured CUDA graph advances t. lr (host
 * float[6]): mean, opacity logit, log-scale, quaternion, SH DC, SH rest. */
ADP_API int adp_adam_step(adp_gaussians* param, const adp_gaussians* grad, adp_gaussians* m,
                          adp_gaussians* v, int32_t step, int32_t* d_step, const float* lr,
                          float beta1, float beta2, float eps, adp_stream_t stream);
/* The same update on the listed rows only (device int32 ids in [0, n), no
 * repeats), e.g. the split candidates before adp_split_plan when the
 * compaction applies the step to the other rows (adp_split_apply_adam).
 * Reads *d_step (if non-NULL) but does not advance it. */
ADP_API int adp_adam_step_rows(adp_gaussians* param, const adp_gaussians* grad, adp_gaussians* m,
                               adp_gaussians* v, const int32_t* rows, int64_t n_rows,
                               int32_t step, const int32_t* d_step, const float* lr, float beta1,
                               float beta2, float eps, adp_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* ADPSPLIT_H */

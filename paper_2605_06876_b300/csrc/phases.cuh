// Host-side phases of the one-stage entry points that the fused batched step
// (adp_train_step_batched) runs as they are, on the same stream.
#pragma once

#include "common.cuh"

namespace adp {

// adp_project's launch; zero_moments (optional, [V*n][3] float4) additionally gets
// the three rows of every record the projection makes visible zeroed (the
// backward's pixel moments, which are only read for visible records).
int project_launch(const adp_gaussians* g, const adp_camera* cams, int n_views,
                   const adp_params* prm, adp_projected* out, float4* zero_moments,
                   cudaStream_t st);

// Adds to f the presets of the error statistics: the per-view min/max words of
// maps->minmax for the raw L1 reduction, and the zeroed per-Gaussian count and
// mass that error_norm_phase accumulates into.
void error_init_fill(FillSet& f, adp_error_maps* maps, int n_views, int32_t* count,
                     double* mass, long long n);

// Eq. 6 from the raw per-pixel L1 error in maps->E and its per-view min/max:
// E, the mask M and the bands B (in place), and the per-Gaussian count and
// error mass of the pre-erosion error pixels (into the zeroed count and mass,
// see error_init_fill).
int error_norm_phase(adp_error_maps* maps, const int32_t* dominant, long long n,
                     const CamSet& cs, const adp_params* prm, int32_t* count, double* mass,
                     cudaStream_t st);

// Zeroes the three float4 pixel-moment rows of every record with tiles > 0, and
// fills the ranges of f in the same launch.
int zero_visible_moments(const int* tiles, long long n_rec, float4* g2d, const FillSet& f,
                         cudaStream_t st);

// The per-Gaussian part of the render backward: from the per-(view, Gaussian)
// pixel moments in g2d, the chain rule through the EWA projection and the SH
// colour of every view, summed over views, into grad (zeroed or masked rows);
// list and n_list are scratch (n ints, one counter zeroed by the caller).
int backward_gauss_phase(const adp_gaussians* g, const adp_projected* pr, const CamSet& cs,
                         const adp_params* prm, adp_gaussians* grad, float* grad2d_accum,
                         int32_t* grad2d_visits, const float4* g2d, int* list,
                         unsigned long long* n_list, cudaStream_t st);

}  // namespace adp

// prs_runs.h -- several runs of one 2D box in one launch of the three-step pass (Eqs. 3-5):
// the ensemble's runs that are stepped alone, pass by pass (prs_api.cu: step_runs).
#pragma once

#include "prs_internal.h"

namespace prs {

// Runs of one box per launch of the 2D three-step pass (at most kT3MaxRuns): phi, dphi in and
// out and the three kicks of each run (k[3r .. 3r+2]), each run's run constants.
constexpr int kT3MaxRuns = 16;
struct T3Runs2D {
    const float* phi_in[kT3MaxRuns];
    float* phi_out[kT3MaxRuns];
    const float* v_in[kT3MaxRuns];
    float* v_out[kT3MaxRuns];
    KickP k[kT3MaxRuns][3];
    int bpr;  // CTAs (row chunks) per run
};
cudaError_t launch_step_t3_2d_runs(const Geo& g, int nruns, const float* const* phi_in, float* const* phi_out,
                                   const float* const* v_in, float* const* v_out, const KickF* k,
                                   const RunConst<float>* rc, unsigned int* err, cudaStream_t st);

}  // namespace prs

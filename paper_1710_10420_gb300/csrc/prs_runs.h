// prs_runs.h -- several runs of one 2D box in one launch of the three-step pass or of the
// one-step pass (Eqs. 3-5, with or without the Eq. 7/8 sums): the ensemble's runs that are
// stepped alone, pass by pass (prs_api.cu: step_runs, step_measure_first_runs).
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

// Runs of one 2D box per launch of the one-step pass (at most kT3MaxRuns), optionally with
// the Eq. 7/8 sums of each run's state fused in (prs_runs.cu): phi, dphi in and out, the
// kick, the run constants and the diagnostics scratch of each run.
struct Runs1 {
    const float* phi_in[kT3MaxRuns];
    float* phi_out[kT3MaxRuns];
    const float* v_in[kT3MaxRuns];
    float* v_out[kT3MaxRuns];
    KickF k[kT3MaxRuns];
    RunConst<float> rc[kT3MaxRuns];
    DiagScratch scr[kT3MaxRuns];
    int bpr;  // CTAs (row chunks) per run
};
// scr: null for the step alone, else one scratch per run (its result receives the sums).
cudaError_t launch_step2d_runs(const Geo& g, int nruns, const float* const* phi_in, float* const* phi_out,
                               const float* const* v_in, float* const* v_out, const KickF* k,
                               const RunConst<float>* rc, const DiagScratch* scr, unsigned int* err,
                               cudaStream_t st);

}  // namespace prs

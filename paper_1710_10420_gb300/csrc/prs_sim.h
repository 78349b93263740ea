// prs_sim.h -- the run object behind the opaque prs_sim handle (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "prs.h"
#include "prs_internal.h"

struct prs_sim {
    prs_params p;
    prs::Geo g;
    size_t elem;         // bytes per value
    cudaStream_t stream;
    void* phi[2];        // ping-pong field buffers
    void* dphi;          // velocity, updated in place
    int cur;             // which phi[] holds phi^n
    bool owned;          // library allocated phi[] and dphi
    bool have_buffers;
    bool initialised;
    int64_t n;           // step index of the state
    double rc[6];        // deta, 1/dx^2, 1/phi0^2, 2D, V0, phi0
    prs::DiagScratch scr;
    prs::DevStatus* d_status; // device: result, counter, error word
    prs::DevStatus* h_status; // pinned host copy
    void* dphi_alt;           // second dphi buffer for passes that read dphi across sites (library-owned)
    void* adj_ws;             // prs_adjoint working memory, kept for the next call
    size_t adj_ws_bytes;
    std::vector<cudaEvent_t> adj_ev; // prs_adjoint phase boundaries (created on demand)
    double adj_ms[3];         // last prs_adjoint: forward, recomputation, reverse sweep (ms)
    bool adj_timed;
    void* guard_base[3];      // PRS_DEBUG: allocations of phi[0], phi[1], dphi with guard bands
    prs::DebugCheck* d_dbg;   // PRS_DEBUG: results of the scan kernel
};

namespace prs {

// FP64 step-n coefficients: c1, c2, cV, delta, d delta / d alpha (Eq. 4, Eq. 6).
void step_coefficients(const prs_params& p, int64_t n, double out[5]);
// Leapfrog stability at step n.
bool cfl_ok(const prs_params& p, int64_t n);
// Leapfrog stability at every step n .. n+nsteps-1 (nsteps >= 1): the force prefactor
// cV ~ a^beta = eta^(m beta) is monotonic in eta, so its largest value over the steps is
// at the first (beta < 0) or the last (beta > 0), and both ends are checked.
bool cfl_ok_over(const prs_params& p, int64_t n, int64_t nsteps);
// Record a CUDA error for prs_last_error(); returns PRS_ECUDA.
int cuda_fail(cudaError_t e, const char* what);
// Allocate the field buffers if none are bound or allocated yet.
int ensure_buffers(prs_sim* s);
// After a synchronised read of s->h_status: PRS_ETIMEOUT (once) if a device wait gave up.
int check_device_error(prs_sim* s);
// Queue the first part of what prs_step_measure(nsteps) does, without waiting for it: the
// Eq. 7/8 sums of the current state into *result (device memory), fused into the first step
// where a fused kernel serves the box.  *taken: the steps queued (1 fused, else 0); the
// caller steps the other nsteps - *taken as prs_step would, for the same fields.  A bounded
// wait that gives up sets the run's device error word.
int step_measure_first(prs_sim* s, int64_t nsteps, DiagAcc* result, int64_t* taken);
// step_measure_first for several runs: one launch of the fused one-step pass over all of them
// when they share a 2D box and stream (at most kT3MaxRuns; the fields are those of the runs'
// own passes, the sums the same to FP64 rounding), else run by run.
int step_measure_first_runs(prs_sim* const* runs, int nruns, int64_t nsteps, DiagAcc* const* results,
                            int64_t* taken);
// Step each of several runs by nsteps as prs_step would step it alone (the same passes in the
// same order, so the same fields), issuing each round of 2D three-step passes and of single
// steps as one launch over all the runs when they share a box, stream and plan (at most
// kT3MaxRuns); else one run after another.
int step_runs(prs_sim* const* runs, int nruns, int64_t nsteps);
// PRS_DEBUG: the checks after a call that returned rc (prs_debug.cu); scan_state adds
// the non-finite scan of the state.  Returns rc when the run has no PRS_DEBUG.
int debug_after(prs_sim* s, int rc, const char* where, bool scan_state);
// PRS_DEBUG: one field of `bytes` between two guard bands.
int debug_alloc_field(size_t bytes, void** base, void** field);

}  // namespace prs

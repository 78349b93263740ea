// prs_internal.h -- shared between the host API (prs_api.cu) and the kernel files.
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "prs.h"

namespace prs {

// Lattice geometry in the layout of the ABI: idx = x + nx*(y + ny*z), x fastest.
struct Geo {
    int dims;
    int nx, ny, nz;  // nz = 1 in 2D
    int64_t S;       // sites
};

// Per-step coefficients of Eq. 4 with Eq. 6 and the force prefactor, in working precision.
template <typename R>
struct StepCoef {
    R c1, c2, cV;
};

// FP32 kick of one step (Eq. 4 with Eq. 6 and the force prefactor), the step's
// constants folded:
//   dphi' = c1 dphi + g s2 + phi (k1 - k2 phi^2),   s2 = sum of the 2D neighbours,
// with g = c2/dx^2, k1 = c2 cV - 2D g and k2 = c2 cV/phi0^2, which is
// c1 dphi + c2 (Lphi - cV phi (phi^2/phi0^2 - 1)) rearranged.  Computed in FP64 on the
// host and rounded once (kick_f32).
struct KickF {
    float c1, g, k1, k2;
};

// KickF and the time step as f32x2 operands: each word holds the same float in both halves,
// so the packed update (update4p) takes its constants as they are, with no per-use packing.
struct KickP {
    unsigned long long c1, g, k1, nk2, dt;  // c1, g, k1, -k2, deta
};

inline unsigned long long pack_pair(float f)
{
    unsigned int u;
    static_assert(sizeof u == sizeof f, "32-bit float");
    __builtin_memcpy(&u, &f, sizeof u);
    return ((unsigned long long)u << 32) | u;
}

inline KickP kick_packed(const KickF& k, float deta)
{
    return KickP{pack_pair(k.c1), pack_pair(k.g), pack_pair(k.k1), pack_pair(-k.k2), pack_pair(deta)};
}

// The FP64 form of KickF (the non-reproducible FP64 step, prs_generic.cu).
struct KickD {
    double c1, g, k1, k2;
};

// Scalars fixed for the whole run, in working precision.
template <typename R>
struct RunConst {
    R deta;        // Eq. 5
    R inv_dx2;     // 1/dx^2 of Eq. 3
    R inv_phi0sq;  // 1/phi0^2
    R twoD;        // 2*dims, the centre weight of Eq. 3
    R V0;          // potential height (Eq. 1)
    R phi0;        // vacuum value
};

// Device-side result of one diagnostic reduction (Eq. 7, Eq. 8 sums and counts).
struct DiagAcc {
    double sum_w;
    double sum_ratio;
    long long n_links;
    long long n_wall;
    long long n_vzero;
    long long n_nonfinite;
};

// Device scratch of the diagnostics: per-block partials + a completion counter.
struct DiagScratch {
    DiagAcc* partials;     // [max_blocks]
    DiagAcc* result;       // [1]
    unsigned int* counter; // [1], zero between launches
    int max_blocks;
};

// Device words the host reads back with the diagnostics: the result, the
// completion counter and the sticky error code of bounded waits (0 = none).
struct DevStatus {
    DiagAcc result;
    unsigned int counter;
    unsigned int error;
};

// PRS_DEBUG: guard bands around library-owned fields and the scan's results.
static constexpr size_t kGuardBytes = 4096;
static constexpr unsigned char kGuardByte = 0xA5;
struct DebugCheck {
    unsigned int bad_guard;       // bit b: guard band b differs from the pattern
    unsigned long long nonfinite; // non-finite values in phi^n and dphi
};

// The FP32 kick of a step from its coefficients (c1, c2, cV) and the run's constants
// (the layout of RunConst: deta, 1/dx^2, 1/phi0^2, 2D, V0, phi0).
KickF kick_f32(const double coef[3], const double run_const[6]);

// Kernel launchers (prs_kernels.cu).  Each returns cudaSuccess or the launch error.
cudaError_t launch_init_random(const Geo& g, int precision, uint64_t seed, void* phi, void* dphi, bool zero_dphi,
                               cudaStream_t st);

// One pass of `nsteps_in_pass` fused leapfrog steps from phi_in into phi_out,
// dphi in place.  coef holds one entry per fused step (host memory, by value).
cudaError_t launch_step(const Geo& g, int precision, bool repro, const void* phi_in, void* phi_out, void* dphi,
                        const double* c1, const double* c2, const double* cV, int nsteps_in_pass,
                        const double run_const[6], unsigned int* err, cudaStream_t st);

// As launch_step with dphi read from dphi_in and written to dphi_out (may be equal).
cudaError_t launch_step_io(const Geo& g, int precision, bool repro, const void* phi_in, void* phi_out,
                           const void* dphi_in, void* dphi_out, const double* c1, const double* c2, const double* cV,
                           int nsteps_in_pass, const double run_const[6], unsigned int* err, cudaStream_t st);

// Largest number of steps one pass can fuse for this geometry/precision, and the
// number used when params.tblock is 0.
int max_fused_steps(const Geo& g, int precision, bool repro);
int default_fused_steps(const Geo& g, int precision, bool repro);

cudaError_t launch_measure(const Geo& g, int precision, const void* phi, const void* dphi, const double run_const[6],
                           const DiagScratch& scr, cudaStream_t st);

// Fast FP32 kernels (prs_fast.cu) for x sides that are multiples of 128.
bool fast_step_ok(const Geo& g, int precision);
cudaError_t launch_measure_fast(const Geo& g, const float* phi, const float* v, RunConst<float> rc,
                                const DiagScratch& scr, unsigned int* err, cudaStream_t st);
// One step (in -> out, v -> v_out) and the diagnostics of (in, v); cudaErrorNotSupported
// when this box has no fused kernel.
cudaError_t launch_step_measure_fast(const Geo& g, const float* in, float* out, const float* v, float* v_out,
                                     KickF k, RunConst<float> rc, const DiagScratch& scr, unsigned int* err,
                                     cudaStream_t st);

// Two fused leapfrog steps per pass (prs_tblock.cu), FP32 3D and 2D; dphi out of place.
bool tblock_ok(const Geo& g, int precision);
// Rows of y per tile of the 3D two-step pass (0 when it does not apply).
int tblock3_rows(const Geo& g);
// phi_mid, v_mid (3D only; both or neither): also store the state between the two
// steps there (cudaErrorNotSupported in 2D).
cudaError_t launch_step_t2(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out,
                           KickF k0, KickF k1, RunConst<float> rc, unsigned int* err, cudaStream_t st,
                           float* phi_mid = nullptr, float* v_mid = nullptr);

// The two-step pass with TMA tensor copies (prs_t2tma.cu) for FP32 3D boxes tiled by 256 x 8
// (cudaErrorNotSupported for other boxes, or when the tensor-map encoder is unavailable).
bool t2tma_ok(const Geo& g);
cudaError_t launch_step_t2_tma(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out,
                               KickF k0, KickF k1, RunConst<float> rc, unsigned int* err, cudaStream_t st,
                               float* phi_mid, float* v_mid);

// Three fused leapfrog steps per pass (prs_t3tma.cu), FP32 3D boxes with an x side that is a
// multiple of 128 and a y side that is a multiple of 8 (at least 16); dphi out of place.
// width: the tile's columns (128 or 256; 0 picks the default, 128).
bool t3tma_ok(const Geo& g);
cudaError_t launch_step_t3_tma(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out,
                               KickF k0, KickF k1, KickF k2, RunConst<float> rc, unsigned int* err, cudaStream_t st,
                               int width = 0);

// Three fused leapfrog steps per pass on FP32 2D boxes (prs_t3_2d.cu): x sides that are
// multiples of 128 up to 4096; dphi out of place.
bool t3_2d_ok(const Geo& g);
cudaError_t launch_step_t3_2d(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out,
                              KickF k0, KickF k1, KickF k2, RunConst<float> rc, unsigned int* err, cudaStream_t st);

// One three-step pass on whichever kernel takes the box (3D tensor-copy tiles or 2D rows).
cudaError_t launch_step_t3(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out,
                           KickF k0, KickF k1, KickF k2, RunConst<float> rc, unsigned int* err, cudaStream_t st);

// Store a message for prs_last_error() on this thread.
void record_error(const char* msg);

// The diagnostic kernel launched on exactly `grid` blocks (1 <= grid <= scr.max_blocks).
cudaError_t launch_measure_on_grid(const Geo& g, int precision, const void* phi, const void* dphi,
                                   const double run_const[6], const DiagScratch& scr, int grid, cudaStream_t st);

// Host-side setup shared by the launchers.  Calls on different prs_sim handles may
// run concurrently from several host threads, so neither keeps unsynchronised state.

// Streaming multiprocessors of the current device, cached per device (152 if the
// query fails).
int sm_count_current();

// Raise `func`'s dynamic shared-memory limit to `bytes` on the current device, once per
// device: `done` holds one bit per device ordinal.  Two threads may both make the
// (idempotent) attribute call; neither skips it before it has succeeded.
cudaError_t smem_limit_once(std::atomic<unsigned long long>& done, const void* func, int bytes);

}  // namespace prs

// prs_step.cu -- chooses the kernel for one pass of fused leapfrog steps.
#include "prs_internal.h"

namespace prs {

cudaError_t launch_step_generic(const Geo& g, int precision, bool repro, const void* in, void* out, const void* dphi,
                                void* dphi_out, double c1, double c2, double cV, const double rcd[6], cudaStream_t st);
cudaError_t launch_step_fast(const Geo& g, const float* in, float* out, const float* v, float* v_out,
                             KickF k, RunConst<float> rc, unsigned int* err, cudaStream_t st);

KickF kick_f32(const double coef[3], const double run_const[6])
{
    const double g = coef[1] * run_const[1];
    const double h = coef[1] * coef[2];
    return KickF{(float)coef[0], (float)g, (float)(h - run_const[3] * g), (float)(h * run_const[2])};
}

// Steps one pass may fuse (params.tblock above this is clamped): three on the FP32 boxes the
// three-step passes take, two on the other boxes of the two-step passes.
int max_fused_steps(const Geo& g, int precision, bool repro)
{
    (void)repro;
    if (!tblock_ok(g, precision)) return 1;
    return (g.dims == 3 ? t3tma_ok(g) : t3_2d_ok(g)) ? 3 : 2;
}

cudaError_t launch_step_t3(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out,
                           KickF k0, KickF k1, KickF k2, RunConst<float> rc, unsigned int* err, cudaStream_t st)
{
    if (g.dims == 2) return launch_step_t3_2d(g, phi_in, phi_out, v_in, v_out, k0, k1, k2, rc, err, st);
    return launch_step_t3_tma(g, phi_in, phi_out, v_in, v_out, k0, k1, k2, rc, err, st);
}

// The library's default number of steps per pass (us per step, one / two / three steps per
// pass).  FP32 3D: one below 2^24 sites, where a one-step pass cut into chunks of a few planes
// occupies the GPU best (128^3 8.3 / 15.4 / 11.0, 256^2 x 128 18.1 / 21.6 / 20.5); from 2^24 two
// wherever the two-step pass gets tiles of at least 4 rows (256^3 46.7 / 32.8 / 34.3; 1024^3
// 2.53 / 1.37 / 1.43 ms).  FP32 2D: three on rows of 2048 or more (2048^2 10.3 / 10.3 / 9.4,
// 4096^2 47.0 / 25.7 / 22.6) and on boxes of at most 1024 rows (256^2 4.1 / 4.6 / 3.4, 1024^2
// 6.2 / 6.2 / 5.8; 512^2 is the exception, 4.1 / 5.1 / 4.6); else two from 2^24 sites (state above
// L2) and one below (512 x 2048 8.2 / 8.9 / -).  FP64 and other boxes: one.
int default_fused_steps(const Geo& g, int precision, bool repro)
{
    (void)repro;
    if (precision != PRS_FP32 || !tblock_ok(g, precision)) return 1;
    if (g.dims == 2) {
        if (t3_2d_ok(g) && (g.nx >= 2048 || g.ny <= 1024)) return 3;
        return g.S >= (int64_t)1 << 24 ? 2 : 1;
    }
    if (g.S < (int64_t)1 << 24) return 1;
    return tblock3_rows(g) >= 4 ? 2 : 1;
}

cudaError_t launch_step(const Geo& g, int precision, bool repro, const void* phi_in, void* phi_out, void* dphi,
                        const double* c1, const double* c2, const double* cV, int nsteps_in_pass,
                        const double run_const[6], unsigned int* err, cudaStream_t st)
{
    return launch_step_io(g, precision, repro, phi_in, phi_out, dphi, dphi, c1, c2, cV, nsteps_in_pass, run_const,
                          err, st);
}

cudaError_t launch_step_io(const Geo& g, int precision, bool repro, const void* phi_in, void* phi_out,
                           const void* dphi_in, void* dphi_out, const double* c1, const double* c2, const double* cV,
                           int nsteps_in_pass, const double run_const[6], unsigned int* err, cudaStream_t st)
{
    if (nsteps_in_pass != 1) return cudaErrorInvalidValue;
    if (fast_step_ok(g, precision)) {
        const double coef[3] = {c1[0], c2[0], cV[0]};
        const KickF k = kick_f32(coef, run_const);
        RunConst<float> rc{(float)run_const[0], (float)run_const[1], (float)run_const[2], (float)run_const[3],
                           (float)run_const[4], (float)run_const[5]};
        return launch_step_fast(g, (const float*)phi_in, (float*)phi_out, (const float*)dphi_in, (float*)dphi_out, k,
                                rc, err, st);
    }
    return launch_step_generic(g, precision, repro, phi_in, phi_out, dphi_in, dphi_out, c1[0], c2[0], cV[0], run_const,
                               st);
}

}  // namespace prs

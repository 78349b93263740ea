// prs_runs.cu -- several runs of one 2D box in one launch of the one-step pass (Eqs. 3-5),
// with or without the Eq. 7/8 sums of each run's state fused in.
//
// A run alone cuts a small box into short chunks of bands (2048^2: 1024 bands of two rows over
// 256 CTAs; 1024^2: one band of four rows per CTA, staged with two halo bands), so a CTA spends
// much of its pass filling its ring.  Runs of one box launched together share the CTA slots:
// CTA b takes chunk b % bpr of run b / bpr, each chunk many bands long.  Each site's update is
// the same tile routine as the single-run pass (prs_tile.cuh: tile2d), so the fields do not
// depend on the chunking; each run's sums reduce over its own bpr blocks into its own scratch
// (a different grouping of the FP64 sums than the run's own pass: the same to FP64 rounding).
#include <cuda_runtime.h>

#include <atomic>

#include "prs_internal.h"
#include "prs_reduce.cuh"
#include "prs_runs.h"
#include "prs_tile.cuh"

namespace prs {

namespace {

constexpr int kRunItems = 4;  // float4 per thread per band: 4096 sites per band, as the single-run pass
// the largest band tile fast_step_ok admits (the single-run pass's limit), set once per kernel
constexpr size_t kRunTileSmemMax = 100 * 1024;

template <bool MEAS>
__global__ void __launch_bounds__(kFastThreads, 2)
    k_step2d_runs(const __grid_constant__ Runs1 R, int nx, int ny, int rb, int cy, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int run = blockIdx.x / R.bpr, c = blockIdx.x - run * R.bpr;
    Tile2D T{R.phi_in[run], R.phi_out[run], R.v_in[run], R.v_out[run], nx, ny, rb, c * cy, 0};
    T.yn = min(cy, ny - T.y0);  // at least one band: the launcher makes every chunk non-empty
    unsigned* wq = MEAS ? reinterpret_cast<unsigned*>(smem_raw + tile_smem2d(nx, rb)) + (threadIdx.x >> 5) * kQueuePerWarp
                        : nullptr;
    SiteAcc a{0.0, 0.0, 0.0f, 0.0f, 0, 0, 0, 0};
    tile2d<kRunItems, true, MEAS>(T, R.k[run], R.rc[run], smem_raw, wq, a, err);
    if (MEAS)
        block_reduce_and_finish_at(DiagAcc{a.sw, a.sr, a.nl, a.nw, a.nv0, a.nnf}, R.scr[run], (unsigned)c,
                                   (unsigned)R.bpr);
}

}  // namespace

cudaError_t launch_step2d_runs(const Geo& g, int nruns, const float* const* phi_in, float* const* phi_out,
                               const float* const* v_in, float* const* v_out, const KickF* k,
                               const RunConst<float>* rc, const DiagScratch* scr, unsigned int* err,
                               cudaStream_t st)
{
    if (g.dims != 2 || nruns < 1 || nruns > kT3MaxRuns || !fast_step_ok(g, PRS_FP32)) return cudaErrorNotSupported;
    const int rb = kRunItems * 1024 / g.nx;  // rows per band
    const size_t sm = tile_smem2d(g.nx, rb) + (scr ? kQueueBytes : 0);
    const void* fn = scr ? (const void*)k_step2d_runs<true> : (const void*)k_step2d_runs<false>;
    static std::atomic<unsigned long long> attr_m{0}, attr_s{0};
    if (sm > kRunTileSmemMax + (scr ? kQueueBytes : 0)) return cudaErrorNotSupported;
    cudaError_t e = smem_limit_once(scr ? attr_m : attr_s, fn, (int)(kRunTileSmemMax + (scr ? kQueueBytes : 0)));
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFastThreads, sm) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    Runs1 R{};
    for (int r = 0; r < nruns; ++r) {
        R.phi_in[r] = phi_in[r];
        R.phi_out[r] = phi_out[r];
        R.v_in[r] = v_in[r];
        R.v_out[r] = v_out[r];
        R.k[r] = k[r];
        R.rc[r] = rc[r];
        if (scr) R.scr[r] = scr[r];
    }
    // chunks per run: the runs' chunks fill the CTA slots once; every chunk holds whole bands
    // and none is empty (each block joins its run's reduction); at most the scratch's blocks
    const int bands = g.ny / rb;
    int bpr = per_sm * sm_count_current() / nruns;
    if (bpr < 1) bpr = 1;
    if (bpr > bands) bpr = bands;
    for (int r = 0; scr && r < nruns; ++r)
        if (bpr > scr[r].max_blocks) bpr = scr[r].max_blocks;
    const int bpc = (bands + bpr - 1) / bpr;
    R.bpr = (bands + bpc - 1) / bpc;
    const int cy = bpc * rb;
    if (scr)
        k_step2d_runs<true><<<R.bpr * nruns, kFastThreads, sm, st>>>(R, g.nx, g.ny, rb, cy, err);
    else
        k_step2d_runs<false><<<R.bpr * nruns, kFastThreads, sm, st>>>(R, g.nx, g.ny, rb, cy, err);
    return cudaGetLastError();
}

}  // namespace prs

// prs_fast.cu -- the FP32 leapfrog step (Eqs. 3-6) and wall diagnostics (Eqs. 7, 8)
// for boxes whose x side is a multiple of 128 and at most 4096 (3D: 1024): the
// path the benchmark times.  One kernel applies Eqs. 3-5 in a single pass over
// HBM (read phi and dphi once, write them once: 16 B per site-update), where the
// paper's OpenCL code ran one kernel per equation.  The tile routines (bulk-async
// plane staging, shuffles, bounded waits) live in prs_tile.cuh; this file sizes
// the grids: one CTA per tile, two resident per SM.
#include <cuda_runtime.h>

#include "prs_arith.cuh"
#include "prs_internal.h"
#include "prs_ptx.cuh"
#include "prs_reduce.cuh"
#include "prs_tile.cuh"

namespace prs {

template <int ITEMS>
__global__ void __launch_bounds__(kFastThreads, 2)
    k_step3d_f32(const float* __restrict__ phi_in, float* __restrict__ phi_out, const float* v, float* v_out, int nx,
                 int ny, int nz, int ty, int cz, KickF k, RunConst<float> rc, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int ytiles = ny / ty;
    Tile3D T{phi_in, phi_out, v, v_out, nx, ny, nz, ty, (int)(blockIdx.x % ytiles) * ty,
             (int)(blockIdx.x / ytiles) * cz, 0};
    T.zn = min(cz, nz - T.z0);
    SiteAcc a{};
    tile3d<ITEMS, true, false>(T, k, rc, smem_raw, nullptr, a, err);
}

template <int ITEMS>
__global__ void __launch_bounds__(kFastThreads, 2)
    k_step2d_f32(const float* __restrict__ phi_in, float* __restrict__ phi_out, const float* v, float* v_out, int nx,
                 int ny, int rb, int cy, KickF k, RunConst<float> rc, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Tile2D T{phi_in, phi_out, v, v_out, nx, ny, rb, (int)blockIdx.x * cy, 0};
    T.yn = min(cy, ny - T.y0);
    SiteAcc a{};
    tile2d<ITEMS, true, false>(T, k, rc, smem_raw, nullptr, a, err);
}

template <int ITEMS>
__global__ void __launch_bounds__(kFastThreads, 2)
    k_measure3d_f32(const float* __restrict__ phi, const float* __restrict__ v, int nx, int ny, int nz, int ty,
                    int cz, RunConst<float> rc, DiagScratch scr, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int ytiles = ny / ty;
    Tile3D T{phi, nullptr, v, nullptr, nx, ny, nz, ty, (int)(blockIdx.x % ytiles) * ty,
             (int)(blockIdx.x / ytiles) * cz, 0};
    T.zn = min(cz, nz - T.z0);
    unsigned* wq = reinterpret_cast<unsigned*>(smem_raw + tile_smem3d(nx, ty)) + (threadIdx.x >> 5) * kQueuePerWarp;
    SiteAcc a{0.0, 0.0, 0.0f, 0.0f, 0, 0, 0, 0};
    KickF k{};
    tile3d<ITEMS, false, true>(T, k, rc, smem_raw, wq, a, err);  // on a timeout the partial sums still reduce
    block_reduce_and_finish(DiagAcc{a.sw, a.sr, a.nl, a.nw, a.nv0, a.nnf}, scr);
}

template <int ITEMS>
__global__ void __launch_bounds__(kFastThreads, 2)
    k_measure2d_f32(const float* __restrict__ phi, const float* __restrict__ v, int nx, int ny, int rb, int cy,
                    RunConst<float> rc, DiagScratch scr, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Tile2D T{phi, nullptr, v, nullptr, nx, ny, rb, (int)blockIdx.x * cy, 0};
    T.yn = min(cy, ny - T.y0);
    unsigned* wq = reinterpret_cast<unsigned*>(smem_raw + tile_smem2d(nx, rb)) + (threadIdx.x >> 5) * kQueuePerWarp;
    SiteAcc a{0.0, 0.0, 0.0f, 0.0f, 0, 0, 0, 0};
    KickF k{};
    tile2d<ITEMS, false, true>(T, k, rc, smem_raw, wq, a, err);
    block_reduce_and_finish(DiagAcc{a.sw, a.sr, a.nl, a.nw, a.nv0, a.nnf}, scr);
}

// One leapfrog step and the diagnostics of its input state from one read of it (NX > 0:
// an instantiation for that row width, the 1024-wide production box).
template <int ITEMS, int NX>
__global__ void __launch_bounds__(kFastThreads, 2)
    k_step_measure3d_f32(const float* __restrict__ phi_in, float* __restrict__ phi_out, const float* v, float* v_out,
                         int nx, int ny, int nz, int ty, int cz, KickF k, RunConst<float> rc,
                         DiagScratch scr, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int ytiles = ny / ty;
    Tile3D T{phi_in, phi_out, v, v_out, nx, ny, nz, ty, (int)(blockIdx.x % ytiles) * ty,
             (int)(blockIdx.x / ytiles) * cz, 0};
    T.zn = min(cz, nz - T.z0);
    unsigned* wq = reinterpret_cast<unsigned*>(smem_raw + tile_smem3d(nx, ty)) + (threadIdx.x >> 5) * kQueuePerWarp;
    SiteAcc a{0.0, 0.0, 0.0f, 0.0f, 0, 0, 0, 0};
    tile3d<ITEMS, true, true, NX>(T, k, rc, smem_raw, wq, a, err);
    block_reduce_and_finish(DiagAcc{a.sw, a.sr, a.nl, a.nw, a.nv0, a.nnf}, scr);
}

template <int ITEMS>
__global__ void __launch_bounds__(kFastThreads, 2)
    k_step_measure2d_f32(const float* __restrict__ phi_in, float* __restrict__ phi_out, const float* v, float* v_out,
                         int nx, int ny, int rb, int cy, KickF k, RunConst<float> rc, DiagScratch scr,
                         unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Tile2D T{phi_in, phi_out, v, v_out, nx, ny, rb, (int)blockIdx.x * cy, 0};
    T.yn = min(cy, ny - T.y0);
    unsigned* wq = reinterpret_cast<unsigned*>(smem_raw + tile_smem2d(nx, rb)) + (threadIdx.x >> 5) * kQueuePerWarp;
    SiteAcc a{0.0, 0.0, 0.0f, 0.0f, 0, 0, 0, 0};
    tile2d<ITEMS, true, true>(T, k, rc, smem_raw, wq, a, err);
    block_reduce_and_finish(DiagAcc{a.sw, a.sr, a.nl, a.nw, a.nv0, a.nnf}, scr);
}

// ------------------------------------------------------------------ dispatch

static constexpr int kItems = 4;  // float4 per thread per plane: 4096 sites per plane tile

static size_t smem3d(int nx, int ty) { return tile_smem3d(nx, ty); }
static size_t smem2d(int nx, int rb) { return tile_smem2d(nx, rb); }

static constexpr size_t kFastSmemMax = 100 * 1024;
static constexpr size_t kMeasureSmemMax = kFastSmemMax + kQueueBytes;

bool fast_step_ok(const Geo& g, int precision)
{
    if (precision != PRS_FP32) return false;
    if (g.nx % 128 != 0 || g.nx > kItems * 1024 || (kItems * 1024) % g.nx != 0) return false;
    const int t = kItems * 1024 / g.nx;  // rows per plane tile (3D) or per band (2D)
    if (g.ny % t != 0) return false;
    return (g.dims == 3 ? smem3d(g.nx, t) : smem2d(g.nx, t)) <= kFastSmemMax;
}

// Shortest chunks the planner considers: 4 planes (3D), one band (2D).  A small box must be
// cut into enough chunks to occupy the GPU, or each pass is bound by the latency of a few CTAs
// marching long chunks (one step per pass, minimum 16 planes and 4 bands before: 128^3 22.1
// against 8.2 us per step, 256^2 8.2 against 4.2, 1024^2 8.2 against 6.2; large boxes pick
// long chunks either way).
constexpr int kMinPlanes = 4, kMinBands = 1;

// Number of z-chunks (3D) or row chunks (2D): balance whole waves of resident
// CTAs against the two halo planes each chunk re-reads.
static int pick_chunks(int tiles, int len, int min_len, int slots, long long max_blocks = 1ll << 40)
{
    int best = 1;
    double best_score = -1.0;
    for (int nc = 1; nc <= len / min_len || nc == 1; ++nc) {
        int c = (len + nc - 1) / nc;
        int n = (len + c - 1) / c;
        long long blocks = (long long)tiles * n;
        if (blocks > max_blocks && nc > 1) break;
        long long waves = (blocks + slots - 1) / slots;
        double fill = (double)blocks / (double)(waves * slots);
        double halo = (double)c / (double)(c + 2);
        double score = fill * halo * (waves >= 2 ? 1.0 : 0.9);
        if (score > best_score + 1e-9) {
            best_score = score;
            best = n;
        }
        if (nc > 4096) break;
    }
    return best;
}

cudaError_t launch_step_fast(const Geo& g, const float* in, float* out, const float* v, float* v_out,
                             KickF k, RunConst<float> rc, unsigned int* err, cudaStream_t st)
{
    static std::atomic<unsigned long long> attr3{0}, attr2{0};
    const int t = kItems * 1024 / g.nx;
    const int slots = 2 * sm_count_current();  // two resident CTAs per SM
    if (g.dims == 3) {
        const size_t sm = smem3d(g.nx, t);
        {
            const cudaError_t e = smem_limit_once(attr3, (const void*)k_step3d_f32<kItems>, (int)kFastSmemMax);
            if (e != cudaSuccess) return e;
        }
        if (sm > kFastSmemMax) return cudaErrorInvalidValue;
        const int ytiles = g.ny / t;
        int nchunks = pick_chunks(ytiles, g.nz, kMinPlanes, slots);
        const int cz = (g.nz + nchunks - 1) / nchunks;
        nchunks = (g.nz + cz - 1) / cz;
        k_step3d_f32<kItems><<<ytiles * nchunks, kFastThreads, sm, st>>>(in, out, v, v_out, g.nx, g.ny, g.nz, t, cz,
                                                                         k, rc, err);
        return cudaGetLastError();
    }
    const size_t sm = smem2d(g.nx, t);
    {
        const cudaError_t e = smem_limit_once(attr2, (const void*)k_step2d_f32<kItems>, (int)kFastSmemMax);
        if (e != cudaSuccess) return e;
    }
    if (sm > kFastSmemMax) return cudaErrorInvalidValue;
    const int bands = g.ny / t;
    int nchunks = pick_chunks(1, bands, kMinBands, slots);
    const int bpc = (bands + nchunks - 1) / nchunks;
    const int cy = bpc * t;
    nchunks = (g.ny + cy - 1) / cy;
    k_step2d_f32<kItems><<<nchunks, kFastThreads, sm, st>>>(in, out, v, v_out, g.nx, g.ny, t, cy, k, rc, err);
    return cudaGetLastError();
}

cudaError_t launch_measure_fast(const Geo& g, const float* phi, const float* v, RunConst<float> rc,
                                const DiagScratch& scr, unsigned int* err, cudaStream_t st)
{
    static std::atomic<unsigned long long> attr3{0}, attr2{0};
    const int t = kItems * 1024 / g.nx;
    const int slots = 2 * sm_count_current();
    if (g.dims == 3) {
        const size_t sm = smem3d(g.nx, t) + kQueueBytes;
        if (sm > kMeasureSmemMax) return cudaErrorNotSupported;
        {
            const cudaError_t e = smem_limit_once(attr3, (const void*)k_measure3d_f32<kItems>, (int)kMeasureSmemMax);
            if (e != cudaSuccess) return e;
        }
        const int ytiles = g.ny / t;
        if (ytiles > scr.max_blocks) return cudaErrorNotSupported;
        int nchunks = pick_chunks(ytiles, g.nz, kMinPlanes, slots, scr.max_blocks);
        const int cz = (g.nz + nchunks - 1) / nchunks;
        nchunks = (g.nz + cz - 1) / cz;
        if ((long long)ytiles * nchunks > scr.max_blocks) return cudaErrorNotSupported;
        k_measure3d_f32<kItems><<<ytiles * nchunks, kFastThreads, sm, st>>>(phi, v, g.nx, g.ny, g.nz, t, cz, rc, scr,
                                                                            err);
        return cudaGetLastError();
    }
    const size_t sm = smem2d(g.nx, t) + kQueueBytes;
    if (sm > kMeasureSmemMax) return cudaErrorNotSupported;
    {
        const cudaError_t e = smem_limit_once(attr2, (const void*)k_measure2d_f32<kItems>, (int)kMeasureSmemMax);
        if (e != cudaSuccess) return e;
    }
    const int bands = g.ny / t;
    int nchunks = pick_chunks(1, bands, kMinBands, slots, scr.max_blocks);
    const int bpc = (bands + nchunks - 1) / nchunks;
    const int cy = bpc * t;
    nchunks = (g.ny + cy - 1) / cy;
    if (nchunks > scr.max_blocks) return cudaErrorNotSupported;
    k_measure2d_f32<kItems><<<nchunks, kFastThreads, sm, st>>>(phi, v, g.nx, g.ny, t, cy, rc, scr, err);
    return cudaGetLastError();
}

cudaError_t launch_step_measure_fast(const Geo& g, const float* in, float* out, const float* v, float* v_out,
                                     KickF k, RunConst<float> rc, const DiagScratch& scr, unsigned int* err,
                                     cudaStream_t st)
{
    static std::atomic<unsigned long long> attr3{0}, attr2{0};
    const int t = kItems * 1024 / g.nx;
    const int slots = 2 * sm_count_current();
    if (g.dims == 3) {
        const size_t sm = smem3d(g.nx, t) + kQueueBytes;
        if (sm > kMeasureSmemMax) return cudaErrorNotSupported;
        {
            cudaError_t e = smem_limit_once(attr3, (const void*)k_step_measure3d_f32<kItems, 0>, (int)kMeasureSmemMax);
            static std::atomic<unsigned long long> attr31{0};
            if (e == cudaSuccess)
                e = smem_limit_once(attr31, (const void*)k_step_measure3d_f32<kItems, 1024>, (int)kMeasureSmemMax);
            if (e != cudaSuccess) return e;
        }
        const int ytiles = g.ny / t;
        if (ytiles > scr.max_blocks) return cudaErrorNotSupported;
        int nchunks = pick_chunks(ytiles, g.nz, kMinPlanes, slots, scr.max_blocks);
        const int cz = (g.nz + nchunks - 1) / nchunks;
        nchunks = (g.nz + cz - 1) / cz;
        if ((long long)ytiles * nchunks > scr.max_blocks) return cudaErrorNotSupported;
        if (g.nx == 1024)
            k_step_measure3d_f32<kItems, 1024><<<ytiles * nchunks, kFastThreads, sm, st>>>(
                in, out, v, v_out, g.nx, g.ny, g.nz, t, cz, k, rc, scr, err);
        else
            k_step_measure3d_f32<kItems, 0><<<ytiles * nchunks, kFastThreads, sm, st>>>(
                in, out, v, v_out, g.nx, g.ny, g.nz, t, cz, k, rc, scr, err);
        return cudaGetLastError();
    }
    const size_t sm = smem2d(g.nx, t) + kQueueBytes;
    if (sm > kMeasureSmemMax) return cudaErrorNotSupported;
    {
        const cudaError_t e = smem_limit_once(attr2, (const void*)k_step_measure2d_f32<kItems>, (int)kMeasureSmemMax);
        if (e != cudaSuccess) return e;
    }
    const int bands = g.ny / t;
    int nchunks = pick_chunks(1, bands, kMinBands, slots, scr.max_blocks);
    const int bpc = (bands + nchunks - 1) / nchunks;
    const int cy = bpc * t;
    nchunks = (g.ny + cy - 1) / cy;
    if (nchunks > scr.max_blocks) return cudaErrorNotSupported;
    k_step_measure2d_f32<kItems><<<nchunks, kFastThreads, sm, st>>>(in, out, v, v_out, g.nx, g.ny, t, cy, k, rc, scr,
                                                                    err);
    return cudaGetLastError();
}

}  // namespace prs

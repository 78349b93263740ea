// prs_noalloc.cu -- wall diagnostics for callers that must not allocate device memory.
//
// prs_measure allocates a little device scratch (one partial sum per block) when
// its run is created.  Some callers cannot allow that: a host application that
// owns every device allocation itself (its own caching pool, or a hard memory
// budget that a library must not go around), or a latency-critical loop where a
// cudaMalloc, which may synchronise the whole device, is not acceptable.  For
// them prs_measure_noalloc runs the same diagnostic kernel with its scratch in a
// fixed array compiled into this library, so the call itself allocates nothing.
//
// The array lives in device memory of every GPU that loads the library, for the
// life of the process: kNoAllocSlots partial slots of 48 bytes (3 MiB) plus the
// result and a completion counter.  One block handles kNoAllocSitesPerBlock
// sites, so the largest lattice is kNoAllocSlots * kNoAllocSitesPerBlock = 2^30
// sites (1024^3); larger lattices are rejected with PRS_EINVAL.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "prs.h"
#include "prs_internal.h"

namespace prs {

static const int kNoAllocSlots = 65536;
static const int64_t kNoAllocSitesPerBlock = 16384;
static const int64_t kNoAllocMaxSites = (int64_t)kNoAllocSlots * kNoAllocSitesPerBlock;

// [0, kNoAllocSlots): per-block partials; [kNoAllocSlots]: result; then the counter.
static const size_t kResultOffset = sizeof(DiagAcc) * kNoAllocSlots;
static const size_t kCounterOffset = kResultOffset + sizeof(DiagAcc);
static const size_t kScratchBytes = kCounterOffset + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

static const int64_t kMaxGridY = 65535;  // CUDA's limit on gridDim.y

static const int kMaxDevices = 64;
static std::mutex g_setup_mutex;
static void* g_scratch_addr[kMaxDevices];

// Device address of g_noalloc_scratch on the current device, looked up once per device.
static int scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        record_error(cudaGetErrorString(e));
        return PRS_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        record_error("prs_measure_noalloc: device ordinal out of range");
        return PRS_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[200];
            snprintf(msg, sizeof msg, "prs_measure_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            record_error(msg);
            return PRS_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PRS_OK;
}

}  // namespace prs

using namespace prs;

extern "C" int prs_measure_noalloc(const prs_params* p, const void* d_phi, const void* d_dphi, void* stream,
                                   prs_diag* out)
{
    if (!p || !out) return PRS_EINVAL;
    if ((p->dims != 2 && p->dims != 3) || (p->precision != PRS_FP32 && p->precision != PRS_FP64)) return PRS_EINVAL;
    int64_t nx = p->N, ny = p->Ny ? p->Ny : p->N, nz = p->dims == 3 ? (p->Nz ? p->Nz : p->N) : 1;
    if (nx < 3 || ny < 3 || (p->dims == 3 && nz < 3) || nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30))
        return PRS_EINVAL;
    if (!(p->dx > 0) || !(p->phi0 > 0) || !(p->W0 > 0)) return PRS_EINVAL;
    const int64_t S = nx * ny * nz;
    if (S > kNoAllocMaxSites) {
        char msg[200];
        snprintf(msg, sizeof msg, "prs_measure_noalloc: %lld sites exceed the static scratch limit of %lld sites",
                 (long long)S, (long long)kNoAllocMaxSites);
        record_error(msg);
        return PRS_EINVAL;
    }
    if (!d_phi || !d_dphi) return PRS_EINVAL;

    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    DiagScratch scr;
    scr.partials = (DiagAcc*)base;
    scr.result = (DiagAcc*)((char*)base + kResultOffset);
    scr.counter = (unsigned int*)((char*)base + kCounterOffset);
    scr.max_blocks = kNoAllocSlots;

    Geo g;
    g.dims = p->dims;
    g.nx = (int)nx;
    g.ny = (int)ny;
    g.nz = (int)nz;
    g.S = S;
    const double pi = 3.14159265358979323846;
    double rcd[6] = {p->deta, 1.0 / (p->dx * p->dx), 1.0 / (p->phi0 * p->phi0), (double)(2 * p->dims),
                     pi * pi / (2.0 * p->W0 * p->W0), p->phi0};
    cudaStream_t st = (cudaStream_t)stream;
    // one block per kNoAllocSitesPerBlock sites, striding over the rows along gridDim.y,
    // whose limit (65535) is one below the 65536 partial slots: at the 2^30-site limit the
    // blocks take a few more rows each
    int64_t want = (S + kNoAllocSitesPerBlock - 1) / kNoAllocSitesPerBlock;
    const int grid = (int)(want < kMaxGridY ? want : kMaxGridY);

    // the completion counter must start at zero; a previous call normally leaves it
    // there, but an interrupted one might not
    cudaError_t e = cudaMemsetAsync(scr.counter, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = launch_measure_on_grid(g, p->precision, d_phi, d_dphi, rcd, scr, grid, st);
    DiagAcc a;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&a, scr.result, sizeof(DiagAcc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof msg, "prs_measure_noalloc: %s", cudaGetErrorString(e));
        record_error(msg);
        return PRS_ECUDA;
    }
    out->sum_w = a.sum_w;
    out->sum_ratio = a.sum_ratio;
    out->n_links = a.n_links;
    out->n_wall = a.n_wall;
    out->n_vzero = a.n_vzero;
    out->n_nonfinite = a.n_nonfinite;
    out->area_per_volume = a.sum_w / ((double)S * p->dx);
    int64_t nw = a.n_wall - a.n_vzero;
    out->gamma_v = nw > 0 ? sqrt(a.sum_ratio / (2.0 * (double)nw)) : 0.0;
    out->step = -1;  // this entry point sees only the fields, not the run's step index
    out->eta = 0.0;
    return a.n_nonfinite ? PRS_ENONFINITE : PRS_OK;
}

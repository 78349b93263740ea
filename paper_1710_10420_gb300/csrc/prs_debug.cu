// prs_debug.cu -- the checks of a run created with PRS_DEBUG.
//
// There is no memory checker to run the library under, so a debug run checks what
// it can from inside, after every call that queues work:
//   * the run's stream is synchronised, so an asynchronous CUDA error is reported
//     by the call that caused it (PRS_ECUDA), not by a later one;
//   * a bounded device-side wait that gave up is reported at once (PRS_ETIMEOUT);
//   * the library-owned field buffers are allocated with 4 KiB guard bands before
//     and after each field, filled with a byte pattern at allocation; a kernel that
//     writes past either end of a field changes a band, and the call reports
//     PRS_ECUDA ("guard band ... overwritten");
//   * after a call that changes the state, phi^n and dphi are scanned for non-finite
//     values (PRS_ENONFINITE).
// Nothing here traps or stops the GPU: the scan kernel only reads and counts.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include "prs.h"
#include "prs_internal.h"
#include "prs_sim.h"

namespace prs {

namespace {

struct GuardSet {
    const unsigned char* band[6];  // before/after phi[0], phi[1], dphi (null: unchecked)
};

template <typename R>
__global__ void __launch_bounds__(256) k_debug_scan(GuardSet gs, const R* __restrict__ phi,
                                                    const R* __restrict__ dphi, int64_t S, DebugCheck* out)
{
    if (blockIdx.x == 0) {
        for (int b = 0; b < 6; ++b) {
            if (!gs.band[b]) continue;
            bool bad = false;
            for (size_t i = threadIdx.x; i < kGuardBytes; i += blockDim.x) bad |= gs.band[b][i] != kGuardByte;
            if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&out->bad_guard, 1u << b);
        }
    }
    if (!phi) return;
    unsigned long long n = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x)
        n += (!isfinite(phi[i])) + (!isfinite(dphi[i]));
    for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(&out->nonfinite, n);
}

}  // namespace

int debug_after(prs_sim* s, int rc, const char* where, bool scan_state)
{
    if (!s || !(s->p.flags & PRS_DEBUG)) return rc;
    if (rc != PRS_OK && rc != PRS_ENONFINITE) return rc;
    char msg[200];
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "%s (debug check)", where);
        return cuda_fail(e, msg);
    }
    unsigned int werr = 0;
    e = cudaMemcpy(&werr, &s->d_status->error, sizeof werr, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "debug check: error word");
    if (werr) {
        cudaMemset(&s->d_status->error, 0, sizeof werr);
        snprintf(msg, sizeof msg, "%s: device wait timed out (code %u)", where, werr);
        record_error(msg);
        return PRS_ETIMEOUT;
    }
    GuardSet gs{};
    if (s->owned && s->have_buffers) {
        const void* f[3] = {s->phi[0], s->phi[1], s->dphi};
        const size_t bytes = (size_t)s->g.S * s->elem;
        for (int i = 0; i < 3; ++i) {
            gs.band[2 * i] = (const unsigned char*)f[i] - kGuardBytes;
            gs.band[2 * i + 1] = (const unsigned char*)f[i] + bytes;
        }
    }
    const bool scan = scan_state && s->initialised && s->have_buffers;
    if ((e = cudaMemsetAsync(s->d_dbg, 0, sizeof(DebugCheck), s->stream)) != cudaSuccess)
        return cuda_fail(e, "debug check");
    const int64_t S = s->g.S;
    int grid = (int)((S + 255) / 256);
    if (grid > 4096) grid = 4096;
    if (grid < 1) grid = 1;
    if (s->p.precision == PRS_FP32)
        k_debug_scan<float><<<grid, 256, 0, s->stream>>>(gs, scan ? (const float*)s->phi[s->cur] : nullptr,
                                                         (const float*)s->dphi, S, s->d_dbg);
    else
        k_debug_scan<double><<<grid, 256, 0, s->stream>>>(gs, scan ? (const double*)s->phi[s->cur] : nullptr,
                                                          (const double*)s->dphi, S, s->d_dbg);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "debug check launch");
    DebugCheck h{};
    e = cudaMemcpyAsync(&h, s->d_dbg, sizeof h, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "debug check");
    if (h.bad_guard) {
        static const char* names[6] = {"before phi[0]", "after phi[0]", "before phi[1]",
                                       "after phi[1]",  "before dphi",  "after dphi"};
        int b = __builtin_ctz(h.bad_guard);
        snprintf(msg, sizeof msg, "%s: guard band %s overwritten", where, names[b]);
        record_error(msg);
        return PRS_ECUDA;
    }
    if (h.nonfinite) {
        snprintf(msg, sizeof msg, "%s: %llu non-finite values in phi and dphi", where, h.nonfinite);
        record_error(msg);
        return PRS_ENONFINITE;
    }
    return rc;
}

// Allocates one field of `bytes` with guard bands (PRS_DEBUG); *field is the usable
// part, *base what cudaFree takes.
int debug_alloc_field(size_t bytes, void** base, void** field)
{
    unsigned char* p = nullptr;
    if (cudaMalloc((void**)&p, bytes + 2 * kGuardBytes) != cudaSuccess) {
        cudaGetLastError();
        return PRS_ENOMEM;
    }
    if (cudaMemset(p, kGuardByte, kGuardBytes) != cudaSuccess ||
        cudaMemset(p + kGuardBytes + bytes, kGuardByte, kGuardBytes) != cudaSuccess) {
        cudaFree(p);
        return cuda_fail(cudaGetLastError(), "guard bands");
    }
    *base = p;
    *field = p + kGuardBytes;
    return PRS_OK;
}

}  // namespace prs

// prs_api.cu -- the C ABI of include/prs.h for single runs: parameter checks, the
// FP64 damping schedule (Eq. 6), buffer ownership, and the order of kernel launches.
// No exception crosses the ABI; every CUDA error becomes PRS_ECUDA.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "prs.h"
#include "prs_internal.h"
#include "prs_runs.h"
#include "prs_sim.h"

using namespace prs;



// ------------------------------------------------------------------ errors

static thread_local char g_last_error[256] = "";

int prs::cuda_fail(cudaError_t e, const char* what)
{
    snprintf(g_last_error, sizeof g_last_error, "%s: %s", what, cudaGetErrorString(e));
    return PRS_ECUDA;
}

#define PRS_CUDA(call)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

extern "C" const char* prs_strerror(int status)
{
    switch (status) {
        case PRS_OK: return "ok";
        case PRS_EINVAL: return "invalid argument";
        case PRS_ENOMEM: return "out of memory";
        case PRS_ECUDA: return "CUDA error";
        case PRS_ETIMEOUT: return "device wait timed out";
        case PRS_ENONFINITE: return "non-finite field value";
        case PRS_ESTATE: return "call out of order";
        default: return "unknown status";
    }
}

extern "C" const char* prs_last_error(void) { return g_last_error; }

namespace prs {
void record_error(const char* msg) { snprintf(g_last_error, sizeof g_last_error, "%s", msg); }
}  // namespace prs

// ------------------------------------------------------------- parameters

static const double kPi = 3.14159265358979323846;

static double potential_height(const prs_params& p) { return kPi * kPi / (2.0 * p.W0 * p.W0); }

// Eq. 6 and the force prefactor of Eq. 2 at step n, in FP64 on the host.
void prs::step_coefficients(const prs_params& p, int64_t n, double out[5])
{
    double eta = p.eta0 + (double)n * p.deta;  // computed from n, never accumulated
    double delta = 0.5 * p.alpha * p.deta * p.era_m / eta;
    double a_beta = 1.0;
    if (p.beta != 0.0) a_beta = pow(pow(eta, p.era_m), p.beta);  // a = eta^m, a(1) = 1
    out[0] = (1.0 - delta) / (1.0 + delta);
    out[1] = p.deta / (1.0 + delta);
    out[2] = 4.0 * potential_height(p) * a_beta / (p.phi0 * p.phi0);
    out[3] = delta;
    out[4] = 0.5 * p.deta * p.era_m / eta;
}

// Leapfrog stability of Eqs. 3-5 at step n: deta^2 (4D/dx^2 + max|V''|)/4 < 1,
// with max|V''| = 2 cV over |phi| <= phi0.
bool prs::cfl_ok(const prs_params& p, int64_t n)
{
    double c[5];
    step_coefficients(p, n, c);
    double lam = 4.0 * p.dims / (p.dx * p.dx) + 2.0 * c[2] * p.phi0 * p.phi0;
    return p.deta * p.deta * lam < 4.0;
}

static int check_params(const prs_params* pp, Geo* g)
{
    if (!pp) return PRS_EINVAL;
    const prs_params& p = *pp;
    if (p.dims != 2 && p.dims != 3) return PRS_EINVAL;
    if (p.precision != PRS_FP32 && p.precision != PRS_FP64) return PRS_EINVAL;
    if ((p.flags & ~(PRS_REPRO | PRS_FP32_CR | PRS_DEBUG)) != 0) return PRS_EINVAL;
    int64_t nx = p.N, ny = p.Ny ? p.Ny : p.N, nz = p.dims == 3 ? (p.Nz ? p.Nz : p.N) : 1;
    if (nx < 3 || ny < 3 || (p.dims == 3 && nz < 3)) return PRS_EINVAL;
    if (nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30)) return PRS_EINVAL;
    if (!(p.dx > 0) || !(p.deta > 0) || !(p.eta0 > 0) || !(p.phi0 > 0) || !(p.W0 > 0)) return PRS_EINVAL;
    if (!isfinite(p.dx) || !isfinite(p.deta) || !isfinite(p.eta0) || !isfinite(p.phi0)) return PRS_EINVAL;
    if (!isfinite(p.alpha) || !isfinite(p.beta) || !isfinite(p.era_m)) return PRS_EINVAL;
    if (p.tblock < 0 || p.tblock > 8) return PRS_EINVAL;
    if (!cfl_ok(p, 0)) return PRS_EINVAL;
    // delta must stay below 1 or (1-delta)/(1+delta) flips the velocity's sign
    double c[5];
    step_coefficients(p, 0, c);
    if (!(c[3] < 1.0)) return PRS_EINVAL;
    g->dims = p.dims;
    g->nx = (int)nx;
    g->ny = (int)ny;
    g->nz = (int)nz;
    g->S = nx * ny * nz;
    return PRS_OK;
}

extern "C" int prs_coefficients(const prs_params* params, int64_t n, double out[5])
{
    if (!params || !out || n < 0) return PRS_EINVAL;
    step_coefficients(*params, n, out);
    return PRS_OK;
}

// Largest stable time step at conformal time eta: deta^2 (4D/dx^2 + 2 cV(eta) phi0^2) < 4.
extern "C" int prs_stable_deta(const prs_params* params, double eta, double* deta_max)
{
    if (!params || !deta_max || !(eta > 0) || !isfinite(eta)) return PRS_EINVAL;
    prs_params q = *params;
    q.eta0 = eta;  // step 0 of q is at eta
    double c[5];
    step_coefficients(q, 0, c);
    const double lam = 4.0 * q.dims / (q.dx * q.dx) + 2.0 * c[2] * q.phi0 * q.phi0;
    if (!(lam > 0) || !isfinite(lam)) return PRS_EINVAL;
    *deta_max = 2.0 / sqrt(lam);
    return PRS_OK;
}

extern "C" int prs_default_tblock(const prs_params* params)
{
    Geo g;
    int rc = check_params(params, &g);
    if (rc) return rc;
    int t = default_fused_steps(g, params->precision, (params->flags & PRS_REPRO) != 0);
    return t < 1 ? 1 : t;
}

extern "C" int prs_max_tblock(const prs_params* params)
{
    Geo g;
    int rc = check_params(params, &g);
    if (rc) return rc;
    int t = max_fused_steps(g, params->precision, (params->flags & PRS_REPRO) != 0);
    return t < 1 ? 1 : t;
}

// -------------------------------------------------------------- lifecycle

static const int kMeasureBlocks = 8192;  // partial slots: the fast kernels use one per tile

extern "C" int prs_create(const prs_params* params, void* stream, prs_sim** out)
{
    if (!out) return PRS_EINVAL;
    Geo g;
    int rc = check_params(params, &g);
    if (rc) return rc;
    prs_sim* s = new (std::nothrow) prs_sim();
    if (!s) return PRS_ENOMEM;
    s->p = *params;
    s->g = g;
    s->elem = params->precision == PRS_FP32 ? sizeof(float) : sizeof(double);
    s->stream = (cudaStream_t)stream;
    s->rc[0] = params->deta;
    s->rc[1] = 1.0 / (params->dx * params->dx);
    s->rc[2] = 1.0 / (params->phi0 * params->phi0);
    s->rc[3] = (double)(2 * params->dims);
    s->rc[4] = potential_height(*params);
    s->rc[5] = params->phi0;
    s->scr.max_blocks = kMeasureBlocks;
    void* blob = nullptr;
    size_t bytes = sizeof(DiagAcc) * kMeasureBlocks + sizeof(DevStatus);
    if (cudaMalloc(&blob, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return PRS_ENOMEM;
    }
    s->scr.partials = (DiagAcc*)blob;
    s->d_status = (DevStatus*)(s->scr.partials + kMeasureBlocks);
    s->scr.result = &s->d_status->result;
    s->scr.counter = &s->d_status->counter;
    if (cudaMemset(blob, 0, bytes) != cudaSuccess ||
        cudaMallocHost((void**)&s->h_status, sizeof(DevStatus)) != cudaSuccess ||
        ((params->flags & PRS_DEBUG) && cudaMalloc((void**)&s->d_dbg, sizeof(DebugCheck)) != cudaSuccess)) {
        int r = cuda_fail(cudaGetLastError(), "prs_create");
        cudaFree(blob);
        cudaFreeHost(s->h_status);
        delete s;
        return r;
    }
    *out = s;
    return PRS_OK;
}

extern "C" int prs_bind(prs_sim* s, void* d_phi_a, void* d_phi_b, void* d_dphi)
{
    if (!s || !d_phi_a || !d_phi_b || !d_dphi || d_phi_a == d_phi_b) return PRS_EINVAL;
    if (((uintptr_t)d_phi_a | (uintptr_t)d_phi_b | (uintptr_t)d_dphi) & 15u) return PRS_EINVAL;
    if (s->have_buffers) return PRS_ESTATE;
    s->phi[0] = d_phi_a;
    s->phi[1] = d_phi_b;
    s->dphi = d_dphi;
    s->cur = 0;
    s->owned = false;
    s->have_buffers = true;
    return PRS_OK;
}

int prs::ensure_buffers(prs_sim* s)
{
    if (s->have_buffers) return PRS_OK;
    size_t bytes = (size_t)s->g.S * s->elem;
    if (s->p.flags & PRS_DEBUG) {
        void* f[3] = {nullptr, nullptr, nullptr};
        for (int i = 0; i < 3; ++i) {
            int rc = debug_alloc_field(bytes, &s->guard_base[i], &f[i]);
            if (rc) {
                for (int k = 0; k < i; ++k) cudaFree(s->guard_base[k]), s->guard_base[k] = nullptr;
                return rc;
            }
        }
        s->phi[0] = f[0];
        s->phi[1] = f[1];
        s->dphi = f[2];
        s->cur = 0;
        s->owned = true;
        s->have_buffers = true;
        return PRS_OK;
    }
    void *a = nullptr, *b = nullptr, *v = nullptr;
    if (cudaMalloc(&a, bytes) != cudaSuccess || cudaMalloc(&b, bytes) != cudaSuccess ||
        cudaMalloc(&v, bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(a);
        cudaFree(b);
        cudaFree(v);
        return PRS_ENOMEM;
    }
    s->phi[0] = a;
    s->phi[1] = b;
    s->dphi = v;
    s->cur = 0;
    s->owned = true;
    s->have_buffers = true;
    return PRS_OK;
}

extern "C" int prs_destroy(prs_sim* s)
{
    if (!s) return PRS_EINVAL;
    cudaStreamSynchronize(s->stream);
    if (s->owned && (s->p.flags & PRS_DEBUG)) {
        for (int i = 0; i < 3; ++i) cudaFree(s->guard_base[i]);
    } else if (s->owned) {
        cudaFree(s->phi[0]);
        cudaFree(s->phi[1]);
        cudaFree(s->dphi);
    }
    cudaFree(s->d_dbg);
    cudaFree(s->scr.partials);
    cudaFree(s->dphi_alt);
    cudaFree(s->adj_ws);
    for (cudaEvent_t e : s->adj_ev) cudaEventDestroy(e);
    cudaFreeHost(s->h_status);
    delete s;
    return PRS_OK;
}

// ------------------------------------------------------------------ state

// Steps per pass this run takes (params.tblock, or the library's choice, clamped).
static int run_tblock(const prs_sim* s)
{
    const bool repro = (s->p.flags & PRS_REPRO) != 0;
    int tmax = max_fused_steps(s->g, s->p.precision, repro);
    int tb = s->p.tblock > 0 ? s->p.tblock : default_fused_steps(s->g, s->p.precision, repro);
    if (tb > tmax) tb = tmax;
    return tb < 1 ? 1 : tb;
}

// The second dphi buffer of two-step passes, allocated with the fields (prs_init,
// prs_set_state) so that prs_step itself never allocates; if there is no room the run
// steps one step per pass.
static void ensure_dphi_alt(prs_sim* s)
{
    if (s->dphi_alt || run_tblock(s) < 2) return;
    if (cudaMalloc(&s->dphi_alt, (size_t)s->g.S * s->elem) != cudaSuccess) {
        cudaGetLastError();
        s->dphi_alt = nullptr;
    }
}


static int prs_init_impl(prs_sim* s, const void* h_phi, const void* h_dphi)
{
    if (!s) return PRS_EINVAL;
    int rc = ensure_buffers(s);
    if (rc) return rc;
    size_t bytes = (size_t)s->g.S * s->elem;
    s->cur = 0;
    if (h_phi) {
        PRS_CUDA(cudaMemcpyAsync(s->phi[0], h_phi, bytes, cudaMemcpyHostToDevice, s->stream));
        if (h_dphi)
            PRS_CUDA(cudaMemcpyAsync(s->dphi, h_dphi, bytes, cudaMemcpyHostToDevice, s->stream));
        else
            PRS_CUDA(cudaMemsetAsync(s->dphi, 0, bytes, s->stream));
    } else {
        PRS_CUDA(launch_init_random(s->g, s->p.precision, s->p.seed, s->phi[0], s->dphi, h_dphi == nullptr,
                                    s->stream));
        if (h_dphi) PRS_CUDA(cudaMemcpyAsync(s->dphi, h_dphi, bytes, cudaMemcpyHostToDevice, s->stream));
    }
    // host arrays may be pageable and reused by the caller right after return
    PRS_CUDA(cudaStreamSynchronize(s->stream));
    ensure_dphi_alt(s);
    s->n = 0;
    s->initialised = true;
    return PRS_OK;
}

static int set_state_queued(prs_sim* s, const void* h_phi, const void* h_dphi, int64_t n, bool wait)
{
    if (!s || !h_phi || !h_dphi || n < 0) return PRS_EINVAL;
    int rc = ensure_buffers(s);
    if (rc) return rc;
    size_t bytes = (size_t)s->g.S * s->elem;
    PRS_CUDA(cudaMemcpyAsync(s->phi[s->cur], h_phi, bytes, cudaMemcpyHostToDevice, s->stream));
    PRS_CUDA(cudaMemcpyAsync(s->dphi, h_dphi, bytes, cudaMemcpyHostToDevice, s->stream));
    if (wait) PRS_CUDA(cudaStreamSynchronize(s->stream));
    ensure_dphi_alt(s);
    s->n = n;
    s->initialised = true;
    return PRS_OK;
}

static int prs_set_state_impl(prs_sim* s, const void* h_phi, const void* h_dphi, int64_t n)
{
    return set_state_queued(s, h_phi, h_dphi, n, true);
}

extern "C" int prs_set_state_async(prs_sim* s, const void* h_phi, const void* h_dphi, int64_t n)
{
    return debug_after(s, set_state_queued(s, h_phi, h_dphi, n, false), "prs_set_state_async", true);
}

static int set_state_device(prs_sim* s, const void* d_phi, const void* d_dphi, int64_t n)
{
    if (!s || !d_phi || !d_dphi || n < 0) return PRS_EINVAL;
    int rc = ensure_buffers(s);
    if (rc) return rc;
    size_t bytes = (size_t)s->g.S * s->elem;
    if (d_phi != s->phi[s->cur])
        PRS_CUDA(cudaMemcpyAsync(s->phi[s->cur], d_phi, bytes, cudaMemcpyDeviceToDevice, s->stream));
    if (d_dphi != s->dphi) PRS_CUDA(cudaMemcpyAsync(s->dphi, d_dphi, bytes, cudaMemcpyDeviceToDevice, s->stream));
    ensure_dphi_alt(s);
    s->n = n;
    s->initialised = true;
    return PRS_OK;
}

extern "C" int prs_set_state_device(prs_sim* s, const void* d_phi, const void* d_dphi, int64_t n)
{
    return debug_after(s, set_state_device(s, d_phi, d_dphi, n), "prs_set_state_device", true);
}

extern "C" int prs_get_state(prs_sim* s, void* h_phi, void* h_dphi, int64_t* n)
{
    if (!s) return PRS_EINVAL;
    if (!s->initialised) return PRS_ESTATE;
    size_t bytes = (size_t)s->g.S * s->elem;
    if (h_phi) PRS_CUDA(cudaMemcpyAsync(h_phi, s->phi[s->cur], bytes, cudaMemcpyDeviceToHost, s->stream));
    if (h_dphi) PRS_CUDA(cudaMemcpyAsync(h_dphi, s->dphi, bytes, cudaMemcpyDeviceToHost, s->stream));
    PRS_CUDA(cudaStreamSynchronize(s->stream));
    if (n) *n = s->n;
    return PRS_OK;
}

extern "C" int prs_device_state(prs_sim* s, void** d_phi, void** d_dphi, int64_t* n)
{
    if (!s) return PRS_EINVAL;
    if (!s->initialised) return PRS_ESTATE;
    if (d_phi) *d_phi = s->phi[s->cur];
    if (d_dphi) *d_dphi = s->dphi;
    if (n) *n = s->n;
    return PRS_OK;
}

// From the next step on, steps of size deta: eta continues from the current time,
// eta_m = eta_n + (m - n) deta for the current step n (eta0 is re-based to eta_n - n deta).
static int set_deta(prs_sim* s, double deta)
{
    if (!s || !(deta > 0) || !isfinite(deta)) return PRS_EINVAL;
    prs_params q = s->p;
    const double eta_n = s->p.eta0 + (double)s->n * s->p.deta;
    q.eta0 = eta_n - (double)s->n * deta;
    q.deta = deta;
    double c[5];
    step_coefficients(q, s->n, c);
    if (!cfl_ok(q, s->n) || !(c[3] < 1.0)) return PRS_EINVAL;
    s->p = q;
    s->rc[0] = deta;
    return PRS_OK;
}

extern "C" int prs_set_deta(prs_sim* s, double deta) { return set_deta(s, deta); }

// ------------------------------------------------------ launcher setup

int prs::sm_count_current()
{
    static std::atomic<int> cache[64];
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 152;
    }
    if (dev >= 0 && dev < 64 && (n = cache[dev].load(std::memory_order_relaxed)) > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return 152;
    }
    if (dev >= 0 && dev < 64) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

cudaError_t prs::smem_limit_once(std::atomic<unsigned long long>& done, const void* func, int bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// ------------------------------------------------------------------- step

bool prs::cfl_ok_over(const prs_params& p, int64_t n, int64_t nsteps)
{
    return cfl_ok(p, n) && cfl_ok(p, n + nsteps - 1);
}

// The passes of a call of nsteps (>= 1): n3 of three steps, n2 of two, then n1 single steps.
static void step_plan(const prs_sim* s, int64_t nsteps, int64_t& n3, int64_t& n2, int64_t& n1)
{
    const bool repro = (s->p.flags & PRS_REPRO) != 0;
    const int tb = run_tblock(s);
    // Multi-step passes (two or three steps) read dphi across sites, so they write it to a
    // second buffer.  A call runs n3 passes of three steps, n2 of two, then n1 single steps:
    // with T = tblock = 3, nsteps / 3 triples and a pair or a single step for the remainder;
    // with T = 2, pairs, and for an odd count a single step, or, when the library chooses the
    // steps per pass (tblock = 0) and the box takes three-step passes, one triple instead of a
    // pair and a single step.  After an odd number of multi-step passes dphi sits in the
    // second buffer.  A run whose buffers the library owns (no PRS_DEBUG guard bands) then
    // swaps the roles of its two dphi buffers.  A run with bound buffers keeps dphi in the
    // bound buffer at the end of every call: the first single step after an odd number of
    // multi-step passes reads dphi in the second buffer and writes the bound one; with no
    // single step to do it, the triple of an odd T = 2 count runs as a pair and a single
    // step, else the last pair as two single steps, else the last triple as a pair and a
    // single step.  Single steps otherwise update dphi in place.
    const bool swap_ok = s->owned && (s->p.flags & PRS_DEBUG) == 0;
    n3 = 0, n2 = 0, n1 = nsteps;
    if (tb == 3) {
        n3 = nsteps / 3;
        n2 = nsteps - 3 * n3 == 2 ? 1 : 0;
        n1 = nsteps - 3 * n3 - 2 * n2;
    } else if (tb == 2) {
        n2 = nsteps / 2;
        n1 = nsteps - 2 * n2;
        if (n1 == 1 && n2 >= 1 && s->p.tblock == 0 && max_fused_steps(s->g, s->p.precision, repro) >= 3)
            n3 = 1, n2 -= 1, n1 = 0;
    }
    if (!s->dphi_alt) n3 = n2 = 0, n1 = nsteps;  // no second buffer (no room at prs_init)
    if (((n3 + n2) & 1) && n1 == 0 && !swap_ok) {
        if (tb == 2 && n3 == 1) n3 = 0, n2 += 1, n1 = 1;
        else if (n2 > 0) n2 -= 1, n1 += 2;
        else n3 -= 1, n2 += 1, n1 += 1;
    }
}

static int prs_step_impl(prs_sim* s, int64_t nsteps)
{
    if (!s || nsteps < 0) return PRS_EINVAL;
    if (!s->initialised) return PRS_ESTATE;
    if (nsteps == 0) return PRS_OK;
    if (!cfl_ok_over(s->p, s->n, nsteps)) return PRS_EINVAL;
    const bool repro = (s->p.flags & PRS_REPRO) != 0;
    int64_t n3, n2, n1;
    step_plan(s, nsteps, n3, n2, n1);
    unsigned int* err = &s->d_status->error;
    const RunConst<float> rcf{(float)s->rc[0], (float)s->rc[1], (float)s->rc[2],
                              (float)s->rc[3], (float)s->rc[4], (float)s->rc[5]};
    void* vbuf[2] = {s->dphi, s->dphi_alt};
    int vi = 0;  // vbuf[vi] holds dphi
    int64_t n = s->n;
    for (int64_t k = 0; k < n3 + n2; ++k) {
        const int t = k < n3 ? 3 : 2;
        double a[5], b[5], c[5];
        step_coefficients(s->p, n, a);
        step_coefficients(s->p, n + 1, b);
        cudaError_t e;
        if (t == 3) {
            step_coefficients(s->p, n + 2, c);
            e = launch_step_t3(s->g, (const float*)s->phi[s->cur], (float*)s->phi[1 - s->cur],
                               (const float*)vbuf[vi], (float*)vbuf[1 - vi], kick_f32(a, s->rc), kick_f32(b, s->rc),
                               kick_f32(c, s->rc), rcf, err, s->stream);
            if (e == cudaErrorNotSupported) {  // no tensor-map encoder: a pair, then a single step in place
                e = launch_step_t2(s->g, (const float*)s->phi[s->cur], (float*)s->phi[1 - s->cur],
                                   (const float*)vbuf[vi], (float*)vbuf[1 - vi], kick_f32(a, s->rc),
                                   kick_f32(b, s->rc), rcf, err, s->stream);
                if (e == cudaSuccess)
                    e = launch_step_io(s->g, s->p.precision, repro, s->phi[1 - s->cur], s->phi[s->cur],
                                       vbuf[1 - vi], vbuf[1 - vi], &c[0], &c[1], &c[2], 1, s->rc, err, s->stream);
                s->cur = 1 - s->cur;  // phi ends where it started; the common flip below undoes this
            }
        } else {
            e = launch_step_t2(s->g, (const float*)s->phi[s->cur], (float*)s->phi[1 - s->cur],
                               (const float*)vbuf[vi], (float*)vbuf[1 - vi], kick_f32(a, s->rc),
                               kick_f32(b, s->rc), rcf, err, s->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "prs_step launch");
        s->cur = 1 - s->cur;
        vi = 1 - vi;
        n += t;
    }
    for (int64_t k = 0; k < n1; ++k) {
        double c[5];
        step_coefficients(s->p, n + k, c);
        const void* v_in = vbuf[vi];  // the first single step brings dphi home
        cudaError_t e = launch_step_io(s->g, s->p.precision, repro, s->phi[s->cur], s->phi[1 - s->cur], v_in,
                                       s->dphi, &c[0], &c[1], &c[2], 1, s->rc, err, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "prs_step launch");
        s->cur = 1 - s->cur;
        vi = 0;
    }
    if (vi) {  // dphi now sits in the second buffer, which becomes the run's own (only when swap_ok)
        void* t = s->dphi;
        s->dphi = s->dphi_alt;
        s->dphi_alt = t;
    }
    s->n += nsteps;
    return PRS_OK;
}

// ---------------------------------------------------------------- measure

// After a synchronised read of h_status: a bounded device wait that gave up makes
// the state untrustworthy; report it once and clear the word.
int prs::check_device_error(prs_sim* s)
{
    if (s->h_status->error == 0) return PRS_OK;
    snprintf(g_last_error, sizeof g_last_error, "device wait timed out (code %u)", s->h_status->error);
    s->h_status->error = 0;
    cudaMemsetAsync(&s->d_status->error, 0, sizeof(unsigned int), s->stream);
    cudaStreamSynchronize(s->stream);
    return PRS_ETIMEOUT;
}

// The staged FP32 diagnostic kernels (alone or fused into a step) serve this run;
// PRS_FP32_CR asks for the generic kernel's correctly rounded division and sqrt.
static bool fast_diag_ok(const prs_sim* s)
{
    return fast_step_ok(s->g, s->p.precision) && (s->p.flags & PRS_FP32_CR) == 0;
}

static int measure_into(prs_sim* s, prs_diag* d)
{
    if (!s->initialised) return PRS_ESTATE;
    cudaError_t e = cudaErrorNotSupported;
    if (fast_diag_ok(s)) {
        RunConst<float> rc{(float)s->rc[0], (float)s->rc[1], (float)s->rc[2],
                           (float)s->rc[3], (float)s->rc[4], (float)s->rc[5]};
        e = launch_measure_fast(s->g, (const float*)s->phi[s->cur], (const float*)s->dphi, rc, s->scr,
                                &s->d_status->error, s->stream);
    }
    if (e == cudaErrorNotSupported)
        e = launch_measure(s->g, s->p.precision, s->phi[s->cur], s->dphi, s->rc, s->scr, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "prs_measure launch");
    PRS_CUDA(cudaMemcpyAsync(s->h_status, s->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s->stream));
    PRS_CUDA(cudaStreamSynchronize(s->stream));
    int err = check_device_error(s);
    if (err) return err;
    const DiagAcc& a = s->h_status->result;
    d->sum_w = a.sum_w;
    d->sum_ratio = a.sum_ratio;
    d->n_links = a.n_links;
    d->n_wall = a.n_wall;
    d->n_vzero = a.n_vzero;
    d->n_nonfinite = a.n_nonfinite;
    d->area_per_volume = a.sum_w / ((double)s->g.S * s->p.dx);  // dA/V = dx^(D-1)/(S dx^D)
    int64_t nw = a.n_wall - a.n_vzero;
    d->gamma_v = nw > 0 ? sqrt(a.sum_ratio / (2.0 * (double)nw)) : 0.0;
    d->step = s->n;
    d->eta = s->p.eta0 + (double)s->n * s->p.deta;
    return a.n_nonfinite ? PRS_ENONFINITE : PRS_OK;
}

// Fill a prs_diag from the device status copied to s->h_status (after a sync).
static void diag_from_status(const prs_sim* s, int64_t step, prs_diag* d)
{
    const DiagAcc& a = s->h_status->result;
    d->sum_w = a.sum_w;
    d->sum_ratio = a.sum_ratio;
    d->n_links = a.n_links;
    d->n_wall = a.n_wall;
    d->n_vzero = a.n_vzero;
    d->n_nonfinite = a.n_nonfinite;
    d->area_per_volume = a.sum_w / ((double)s->g.S * s->p.dx);
    int64_t nw = a.n_wall - a.n_vzero;
    d->gamma_v = nw > 0 ? sqrt(a.sum_ratio / (2.0 * (double)nw)) : 0.0;
    d->step = step;
    d->eta = s->p.eta0 + (double)step * s->p.deta;
}

static int prs_step_measure_impl(prs_sim* s, int64_t nsteps, prs_diag* out)
{
    if (!s || !out || nsteps < 0) return PRS_EINVAL;
    if (!s->initialised) return PRS_ESTATE;
    if (nsteps == 0) return measure_into(s, out);
    if (!cfl_ok_over(s->p, s->n, nsteps)) return PRS_EINVAL;
    const int64_t n0 = s->n;
    cudaError_t e = cudaErrorNotSupported;
    if (fast_diag_ok(s)) {
        double c[5];
        step_coefficients(s->p, n0, c);
        RunConst<float> rc{(float)s->rc[0], (float)s->rc[1], (float)s->rc[2],
                           (float)s->rc[3], (float)s->rc[4], (float)s->rc[5]};
        e = launch_step_measure_fast(s->g, (const float*)s->phi[s->cur], (float*)s->phi[1 - s->cur],
                                     (const float*)s->dphi, (float*)s->dphi,
                                     kick_f32(c, s->rc), rc, s->scr,
                                     &s->d_status->error, s->stream);
    }
    if (e == cudaErrorNotSupported) {
        // no fused kernel for this box: the diagnostics, then the steps
        int rc = measure_into(s, out);
        if (rc != PRS_OK && rc != PRS_ENONFINITE) return rc;
        int rs = prs_step(s, nsteps);
        if (rs) return rs;
        PRS_CUDA(cudaStreamSynchronize(s->stream));
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "prs_step_measure launch");
    s->cur = 1 - s->cur;
    s->n += 1;
    PRS_CUDA(cudaMemcpyAsync(s->h_status, s->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s->stream));
    int rs = prs_step(s, nsteps - 1);
    if (rs) return rs;
    PRS_CUDA(cudaStreamSynchronize(s->stream));
    int err = check_device_error(s);
    if (err) return err;
    diag_from_status(s, n0, out);
    return s->h_status->result.n_nonfinite ? PRS_ENONFINITE : PRS_OK;
}

int prs::step_runs(prs_sim* const* runs, int nruns, int64_t nsteps)
{
    if (nruns < 0 || nsteps < 0) return PRS_EINVAL;
    if (nruns == 0 || nsteps == 0) return PRS_OK;
    // the runs qualify when they share their box, stream and plan and the plan's triples are
    // 2D three-step passes; else each runs alone
    int64_t n3 = 0, n2 = 0, n1 = 0;
    bool together = nruns > 1 && nruns <= kT3MaxRuns;
    for (int r = 0; r < nruns && together; ++r) {
        const prs_sim* s = runs[r];
        if (!s) return PRS_EINVAL;
        if (!s->initialised) return PRS_ESTATE;
        if (!cfl_ok_over(s->p, s->n, nsteps)) return PRS_EINVAL;
        int64_t a3, a2, a1;
        step_plan(s, nsteps, a3, a2, a1);
        const Geo& g = s->g;
        const Geo& g0 = runs[0]->g;
        together = g.dims == 2 && g.nx == g0.nx && g.ny == g0.ny && s->stream == runs[0]->stream &&
                   s->p.precision == PRS_FP32 && (s->p.flags & PRS_REPRO) == 0 && run_tblock(s) == 3 &&
                   t3_2d_ok(g) && s->dphi_alt && (r == 0 || (a3 == n3 && a2 == n2 && a1 == n1));
        if (r == 0) n3 = a3, n2 = a2, n1 = a1;
    }
    if (!together || n3 == 0) {
        for (int r = 0; r < nruns; ++r) {
            const int rc = prs_step_impl(runs[r], nsteps);
            if (rc) return rc;
        }
        return PRS_OK;
    }
    // the passes of prs_step_impl, pass by pass across the runs: the triples as one launch
    std::vector<int> vi(nruns, 0);  // per run: its vbuf index that holds dphi
    std::vector<const float*> pin(nruns), vin(nruns);
    std::vector<float*> pout(nruns), vout(nruns);
    std::vector<KickF> kk(3 * (size_t)nruns);
    std::vector<RunConst<float>> rcs(nruns);
    for (int r = 0; r < nruns; ++r) {
        const prs_sim* s = runs[r];
        rcs[r] = RunConst<float>{(float)s->rc[0], (float)s->rc[1], (float)s->rc[2],
                                 (float)s->rc[3], (float)s->rc[4], (float)s->rc[5]};
    }
    auto vbuf = [&](int r, int i) { return i == 0 ? runs[r]->dphi : runs[r]->dphi_alt; };
    int64_t done = 0;
    for (int64_t k = 0; k < n3; ++k, done += 3) {
        for (int r = 0; r < nruns; ++r) {
            prs_sim* s = runs[r];
            for (int l = 0; l < 3; ++l) {
                double c[5];
                step_coefficients(s->p, s->n + done + l, c);
                kk[3 * (size_t)r + l] = kick_f32(c, s->rc);
            }
            pin[r] = (const float*)s->phi[s->cur];
            pout[r] = (float*)s->phi[1 - s->cur];
            vin[r] = (const float*)vbuf(r, vi[r]);
            vout[r] = (float*)vbuf(r, 1 - vi[r]);
        }
        const cudaError_t e = launch_step_t3_2d_runs(runs[0]->g, nruns, pin.data(), pout.data(), vin.data(),
                                                     vout.data(), kk.data(), rcs.data(),
                                                     &runs[0]->d_status->error, runs[0]->stream);
        if (e != cudaSuccess) return cuda_fail(e, "step_runs launch");
        for (int r = 0; r < nruns; ++r) runs[r]->cur = 1 - runs[r]->cur, vi[r] = 1 - vi[r];
    }
    for (int r = 0; r < nruns; ++r) {  // pairs, run by run
        prs_sim* s = runs[r];
        unsigned int* err = &s->d_status->error;
        int64_t n = s->n + done;
        for (int64_t k = 0; k < n2; ++k, n += 2) {
            double a[5], b[5];
            step_coefficients(s->p, n, a);
            step_coefficients(s->p, n + 1, b);
            const cudaError_t e =
                launch_step_t2(s->g, (const float*)s->phi[s->cur], (float*)s->phi[1 - s->cur],
                               (const float*)vbuf(r, vi[r]), (float*)vbuf(r, 1 - vi[r]), kick_f32(a, s->rc),
                               kick_f32(b, s->rc), rcs[r], err, s->stream);
            if (e != cudaSuccess) return cuda_fail(e, "step_runs launch");
            s->cur = 1 - s->cur;
            vi[r] = 1 - vi[r];
        }
    }
    done += 2 * n2;
    // single steps, each one launch over the runs (the first reads dphi where the multi-step
    // passes left it and writes the run's own buffer)
    std::vector<KickF> k1(nruns);
    for (int64_t k = 0; k < n1; ++k, ++done) {
        for (int r = 0; r < nruns; ++r) {
            prs_sim* s = runs[r];
            double c[5];
            step_coefficients(s->p, s->n + done, c);
            k1[r] = kick_f32(c, s->rc);
            pin[r] = (const float*)s->phi[s->cur];
            pout[r] = (float*)s->phi[1 - s->cur];
            vin[r] = (const float*)vbuf(r, vi[r]);
            vout[r] = (float*)s->dphi;
        }
        cudaError_t e = launch_step2d_runs(runs[0]->g, nruns, pin.data(), pout.data(), vin.data(), vout.data(),
                                           k1.data(), rcs.data(), nullptr, &runs[0]->d_status->error,
                                           runs[0]->stream);
        if (e == cudaErrorNotSupported) {  // no fast one-step pass for this box: run by run
            e = cudaSuccess;
            for (int r = 0; r < nruns && e == cudaSuccess; ++r) {
                prs_sim* s = runs[r];
                double c[5];
                step_coefficients(s->p, s->n + done, c);
                e = launch_step_io(s->g, s->p.precision, false, s->phi[s->cur], s->phi[1 - s->cur], vbuf(r, vi[r]),
                                   s->dphi, &c[0], &c[1], &c[2], 1, s->rc, &s->d_status->error, s->stream);
            }
        }
        if (e != cudaSuccess) return cuda_fail(e, "step_runs launch");
        for (int r = 0; r < nruns; ++r) runs[r]->cur = 1 - runs[r]->cur, vi[r] = 0;
    }
    for (int r = 0; r < nruns; ++r) {
        prs_sim* s = runs[r];
        if (vi[r]) {  // as prs_step_impl: only where the run may swap its dphi buffers
            void* t = s->dphi;
            s->dphi = s->dphi_alt;
            s->dphi_alt = t;
        }
        s->n += nsteps;
    }
    return PRS_OK;
}

int prs::step_measure_first(prs_sim* s, int64_t nsteps, DiagAcc* result, int64_t* taken)
{
    if (!s || !result || !taken || nsteps < 0) return PRS_EINVAL;
    if (!s->initialised) return PRS_ESTATE;
    if (nsteps > 0 && !cfl_ok_over(s->p, s->n, nsteps)) return PRS_EINVAL;
    *taken = 0;
    DiagScratch scr = s->scr;
    scr.result = result;
    const RunConst<float> rc{(float)s->rc[0], (float)s->rc[1], (float)s->rc[2],
                             (float)s->rc[3], (float)s->rc[4], (float)s->rc[5]};
    cudaError_t e = cudaErrorNotSupported;
    if (nsteps > 0 && fast_diag_ok(s)) {
        double c[5];
        step_coefficients(s->p, s->n, c);
        e = launch_step_measure_fast(s->g, (const float*)s->phi[s->cur], (float*)s->phi[1 - s->cur],
                                     (const float*)s->dphi, (float*)s->dphi, kick_f32(c, s->rc), rc, scr,
                                     &s->d_status->error, s->stream);
        if (e == cudaSuccess) {
            s->cur = 1 - s->cur;
            s->n += 1;
            *taken = 1;
            return PRS_OK;
        }
        if (e != cudaErrorNotSupported) return cuda_fail(e, "step_measure launch");
    }
    e = cudaErrorNotSupported;
    if (fast_diag_ok(s))
        e = launch_measure_fast(s->g, (const float*)s->phi[s->cur], (const float*)s->dphi, rc, scr,
                                &s->d_status->error, s->stream);
    if (e == cudaErrorNotSupported)
        e = launch_measure(s->g, s->p.precision, s->phi[s->cur], s->dphi, s->rc, scr, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step_measure launch");
    return PRS_OK;
}

int prs::step_measure_first_runs(prs_sim* const* runs, int nruns, int64_t nsteps, DiagAcc* const* results,
                                  int64_t* taken)
{
    if (nruns < 0 || nsteps < 0 || (nruns > 0 && (!runs || !results || !taken))) return PRS_EINVAL;
    bool together = nruns > 1 && nruns <= kT3MaxRuns && nsteps > 0;
    for (int r = 0; r < nruns && together; ++r) {
        const prs_sim* s = runs[r];
        together = s && results[r] && s->initialised && s->g.dims == 2 && s->g.nx == runs[0]->g.nx &&
                   s->g.ny == runs[0]->g.ny && s->stream == runs[0]->stream && fast_diag_ok(s) &&
                   cfl_ok_over(s->p, s->n, nsteps);
    }
    if (together) {  // one launch: each run's diagnostics fused into its first step
        std::vector<const float*> pin(nruns), vin(nruns);
        std::vector<float*> pout(nruns), vout(nruns);
        std::vector<KickF> kk(nruns);
        std::vector<RunConst<float>> rcs(nruns);
        std::vector<DiagScratch> scr(nruns);
        for (int r = 0; r < nruns; ++r) {
            const prs_sim* s = runs[r];
            double c[5];
            step_coefficients(s->p, s->n, c);
            kk[r] = kick_f32(c, s->rc);
            rcs[r] = RunConst<float>{(float)s->rc[0], (float)s->rc[1], (float)s->rc[2],
                                     (float)s->rc[3], (float)s->rc[4], (float)s->rc[5]};
            pin[r] = (const float*)s->phi[s->cur];
            pout[r] = (float*)s->phi[1 - s->cur];
            vin[r] = (const float*)s->dphi;
            vout[r] = (float*)s->dphi;
            scr[r] = s->scr;
            scr[r].result = results[r];
        }
        const cudaError_t e = launch_step2d_runs(runs[0]->g, nruns, pin.data(), pout.data(), vin.data(), vout.data(),
                                                 kk.data(), rcs.data(), scr.data(), &runs[0]->d_status->error,
                                                 runs[0]->stream);
        if (e == cudaSuccess) {
            for (int r = 0; r < nruns; ++r) {
                runs[r]->cur = 1 - runs[r]->cur;
                runs[r]->n += 1;
                taken[r] = 1;
            }
            return PRS_OK;
        }
        if (e != cudaErrorNotSupported) return cuda_fail(e, "step_measure launch");
    }
    for (int r = 0; r < nruns; ++r) {
        const int rc = step_measure_first(runs[r], nsteps, results[r], &taken[r]);
        if (rc) return rc;
    }
    return PRS_OK;
}

static int prs_measure_ex_impl(prs_sim* s, prs_diag* out)
{
    if (!s || !out) return PRS_EINVAL;
    return measure_into(s, out);
}

static int prs_measure_impl(prs_sim* s, double* area_per_volume, double* gamma_v, int64_t* n_links,
                           int64_t* n_wall_sites)
{
    if (!s) return PRS_EINVAL;
    prs_diag d;
    int rc = measure_into(s, &d);
    if (rc != PRS_OK && rc != PRS_ENONFINITE) return rc;
    if (area_per_volume) *area_per_volume = d.area_per_volume;
    if (gamma_v) *gamma_v = d.gamma_v;
    if (n_links) *n_links = d.n_links;
    if (n_wall_sites) *n_wall_sites = d.n_wall;
    return rc;
}

// ------------------------------------------------ entry points (PRS_DEBUG checks)

extern "C" int prs_init(prs_sim* s, const void* h_phi, const void* h_dphi)
{
    return debug_after(s, prs_init_impl(s, h_phi, h_dphi), "prs_init", true);
}

extern "C" int prs_set_state(prs_sim* s, const void* h_phi, const void* h_dphi, int64_t n)
{
    return debug_after(s, prs_set_state_impl(s, h_phi, h_dphi, n), "prs_set_state", true);
}

extern "C" int prs_step(prs_sim* s, int64_t nsteps)
{
    return debug_after(s, prs_step_impl(s, nsteps), "prs_step", true);
}

extern "C" int prs_step_measure(prs_sim* s, int64_t nsteps, prs_diag* out)
{
    return debug_after(s, prs_step_measure_impl(s, nsteps, out), "prs_step_measure", true);
}

extern "C" int prs_measure_ex(prs_sim* s, prs_diag* out)
{
    return debug_after(s, prs_measure_ex_impl(s, out), "prs_measure_ex", false);
}

extern "C" int prs_measure(prs_sim* s, double* area_per_volume, double* gamma_v, int64_t* n_links, int64_t* n_wall_sites)
{
    const int rc = prs_measure_impl(s, area_per_volume, gamma_v, n_links, n_wall_sites);
    return debug_after(s, rc, "prs_measure", false);
}

// prs_adjoint.cu -- reverse-time adjoint of the leapfrog step (Eqs. 3-6) and the
// two smooth observables it differentiates.  Not in the paper: the gradient of a
// smooth stand-in for the wall diagnostics with respect to the initial field and
// to alpha, by the transpose of the forward step written out by hand.
//
// Forward step n (coefficients c1, c2, cV of Eq. 4, 6 at eta_n):
//     v' = c1 v + c2 (L phi - f(phi)),   phi' = phi + deta v',   f = cV phi (phi^2/phi0^2 - 1)
// Its transpose, given the adjoints (lphi', lv') of (phi', v'):
//     lt   = lv' + deta lphi'
//     lphi = lphi' + c2 (L lt - f'(phi) lt),   f' = cV (3 phi^2/phi0^2 - 1)   (L is symmetric)
//     lv   = c1 lt
//     dJ/dalpha += sum_s lt_s (dc1/dalpha v_s + dc2/dalpha (L phi - f)_s)
// with d delta/d alpha = deta m/(2 eta_n), dc1/d delta = -2/(1+delta)^2,
// dc2/d delta = -deta/(1+delta)^2.
//
// The forward states come from checkpoints every K steps; each segment is
// recomputed into segment storage (the step kernel writes phi and dphi out of
// place), then walked backwards.  The state is never inverted algebraically:
// 1/c1 grows without bound as delta -> 1.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <new>
#include <vector>

#include "prs.h"
#include "prs_arith.cuh"
#include "prs_internal.h"
#include "prs_reduce.cuh"
#include "prs_sim.h"

namespace prs {

namespace {

// Neighbour indices of site (x, y, z) = s, periodic; x fastest.
struct Nbr {
    int64_t xp, xm, yp, ym, zp, zm;
};

__device__ __forceinline__ Nbr neighbours(const Geo& g, int64_t s, int x, int y, int z)
{
    const int64_t nx = g.nx, plane = nx * g.ny;
    Nbr n;
    n.xp = s - x + (x + 1 == g.nx ? 0 : x + 1);
    n.xm = s - x + (x == 0 ? g.nx - 1 : x - 1);
    n.yp = s + (int64_t)((y + 1 == g.ny ? 0 : y + 1) - y) * nx;
    n.ym = s + (int64_t)((y == 0 ? g.ny - 1 : y - 1) - y) * nx;
    n.zp = s + (int64_t)((z + 1 == g.nz ? 0 : z + 1) - z) * plane;
    n.zm = s + (int64_t)((z == 0 ? g.nz - 1 : z - 1) - z) * plane;
    return n;
}

// Sites visited row by row: block (bx, by) strides over rows by gridDim.y and
// over x by gridDim.x * blockDim.x; no division per site.
#define PRS_FOR_SITES(g, s, x, y, z)                                                          \
    for (int64_t row_ = blockIdx.y; row_ < (int64_t)(g).ny * (g).nz; row_ += gridDim.y)      \
        for (int x = blockIdx.x * blockDim.x + threadIdx.x, y = (int)(row_ % (g).ny),        \
                 z = (int)(row_ / (g).ny);                                                    \
             x < (g).nx; x += gridDim.x * blockDim.x)                                         \
            if (const int64_t s = row_ * (g).nx + x; true)

template <typename R, int D>
__device__ __forceinline__ R pair_sum(const R* f, const Nbr& n)
{
    R s2 = f[n.xp] + f[n.xm];
    s2 = s2 + (f[n.yp] + f[n.ym]);
    if (D == 3) s2 = s2 + (f[n.zp] + f[n.zm]);
    return s2;
}

struct AdjCoef {
    double c1, c2, cV, dc1, dc2;  // dc1, dc2: derivatives of c1, c2 with respect to alpha
};

// J contribution of the links (s, s+e_d) and dJ/dphi_s (written to grad).
template <typename R, int D>
__global__ void __launch_bounds__(256) k_observable(const R* __restrict__ phi, R* __restrict__ grad, Geo g, int obs,
                                                    double eps, double inv_dx2, double area_scale, DiagScratch scr)
{
    double J = 0.0;
    PRS_FOR_SITES(g, s, x, y, z)
    {
        const Nbr n = neighbours(g, s, x, y, z);
        const int64_t up[3] = {n.xp, n.yp, n.zp}, dn[3] = {n.xm, n.ym, n.zm};
        const double ps = (double)phi[s];
        double gr = 0.0;
        if (obs == PRS_OBS_GRAD_ENERGY) {
            for (int d = 0; d < D; ++d) {
                const double gd = (double)phi[up[d]] - ps;
                J += 0.5 * gd * gd * inv_dx2;
                gr += (2.0 * ps - (double)phi[up[d]] - (double)phi[dn[d]]) * inv_dx2;
            }
        } else {
            const double ss = tanh(ps / eps);
            double nb = 0.0;
            for (int d = 0; d < D; ++d) {
                const double su = tanh((double)phi[up[d]] / eps);
                J += 0.5 * (1.0 - ss * su) * area_scale;
                nb += su + tanh((double)phi[dn[d]] / eps);
            }
            gr = -0.5 * area_scale * (1.0 - ss * ss) / eps * nb;
        }
        grad[s] = (R)gr;
    }
    block_reduce_and_finish(DiagAcc{J, 0.0, 0, 0, 0, 0}, scr);
}

// One reverse step: (lphi_in, lv_in) at n+1 -> (lphi_out, lv_out) at n, using the
// forward state (phi, v) at n; the dJ/dalpha term of this step lands in *scr.result.
template <typename R, int D>
__global__ void __launch_bounds__(256)
    k_adjoint_step(const R* __restrict__ phi, const R* __restrict__ v, const R* __restrict__ lphi_in,
                   const R* __restrict__ lv_in, R* __restrict__ lphi_out, R* __restrict__ lv_out, Geo g, AdjCoef c,
                   RunConst<R> rc, DiagScratch scr)
{
    const R c1 = (R)c.c1, c2 = (R)c.c2, cV = (R)c.cV, deta = rc.deta;
    const R dc1 = (R)c.dc1, dc2 = (R)c.dc2;
    // per-thread sum of the dJ/dalpha terms in working precision, compensated
    // (Kahan): FP64 arithmetic per site would dominate the step on this GPU
    R da = 0, comp = 0;
    PRS_FOR_SITES(g, s, x, y, z)
    {
        const Nbr n = neighbours(g, s, x, y, z);
        auto lt = [&](int64_t q) { return lv_in[q] + deta * lphi_in[q]; };
        const R lts = lt(s);
        R s2 = lt(n.xp) + lt(n.xm);
        s2 = s2 + (lt(n.yp) + lt(n.ym));
        if (D == 3) s2 = s2 + (lt(n.zp) + lt(n.zm));
        const R Llt = (s2 - rc.twoD * lts) * rc.inv_dx2;
        const R p = phi[s];
        const R fprime = cV * ((R)3 * (p * p) * rc.inv_phi0sq - (R)1);
        lphi_out[s] = lphi_in[s] + c2 * (Llt - fprime * lts);
        lv_out[s] = c1 * lts;
        const R Lphi = (pair_sum<R, D>(phi, n) - rc.twoD * p) * rc.inv_dx2;
        const R f = (cV * p) * ((p * p) * rc.inv_phi0sq - (R)1);
        const R term = lts * (dc1 * v[s] + dc2 * (Lphi - f));
        const R yk = term - comp;
        const R t = da + yk;
        comp = (t - da) - yk;
        da = t;
    }
    block_reduce_and_finish(DiagAcc{(double)da, 0.0, 0, 0, 0, 0}, scr);
}

// Grid of the row-wise kernels: x blocks cover a row, y blocks stride over rows;
// at most 1216 blocks (one FP64 partial each).
dim3 grid_for(const Geo& g)
{
    const int gx = (g.nx + 255) / 256 < 4 ? (g.nx + 255) / 256 : 4;
    int64_t rows = (int64_t)g.ny * g.nz;
    int64_t gy = (152 * 8) / gx;
    if (gy > rows) gy = rows;
    return dim3((unsigned)gx, (unsigned)gy, 1);
}

template <typename R>
RunConst<R> run_const(const double* rcd)
{
    return RunConst<R>{(R)rcd[0], (R)rcd[1], (R)rcd[2], (R)rcd[3], (R)rcd[4], (R)rcd[5]};
}

cudaError_t launch_observable(const prs_sim* s, const void* phi, void* grad, int obs, double eps, DiagScratch scr)
{
    const double area_scale = 1.0 / ((double)s->g.S * s->p.dx);
    const dim3 grid = grid_for(s->g);
    if ((int)(grid.x * grid.y) > scr.max_blocks) return cudaErrorInvalidValue;
#define PRS_OBS_LAUNCH(R, D)                                                                                     \
    k_observable<R, D><<<grid, 256, 0, s->stream>>>((const R*)phi, (R*)grad, s->g, obs, eps, s->rc[1], area_scale, \
                                                    scr)
    if (s->p.precision == PRS_FP32) {
        if (s->g.dims == 3) PRS_OBS_LAUNCH(float, 3); else PRS_OBS_LAUNCH(float, 2);
    } else {
        if (s->g.dims == 3) PRS_OBS_LAUNCH(double, 3); else PRS_OBS_LAUNCH(double, 2);
    }
#undef PRS_OBS_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const prs_sim* s, const void* phi, const void* v, const void* lphi_in,
                                const void* lv_in, void* lphi_out, void* lv_out, const AdjCoef& c, DiagScratch scr)
{
    const dim3 grid = grid_for(s->g);
    if ((int)(grid.x * grid.y) > scr.max_blocks) return cudaErrorInvalidValue;
#define PRS_ADJ_LAUNCH(R, D)                                                                                         \
    k_adjoint_step<R, D><<<grid, 256, 0, s->stream>>>((const R*)phi, (const R*)v, (const R*)lphi_in, (const R*)lv_in, \
                                                      (R*)lphi_out, (R*)lv_out, s->g, c, run_const<R>(s->rc), scr)
    if (s->p.precision == PRS_FP32) {
        if (s->g.dims == 3) PRS_ADJ_LAUNCH(float, 3); else PRS_ADJ_LAUNCH(float, 2);
    } else {
        if (s->g.dims == 3) PRS_ADJ_LAUNCH(double, 3); else PRS_ADJ_LAUNCH(double, 2);
    }
#undef PRS_ADJ_LAUNCH
    return cudaGetLastError();
}

// Device memory owned by one prs_adjoint call, released on every path.
struct Scratch {
    std::vector<void*> blocks;
    ~Scratch()
    {
        for (void* p : blocks) cudaFree(p);
    }
    void* get(size_t bytes)
    {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        blocks.push_back(p);
        return p;
    }
};

}  // namespace

}  // namespace prs

using namespace prs;

extern "C" int prs_observable(prs_sim* s, int observable, double eps_smooth, double* J)
{
    if (!s || !J) return PRS_EINVAL;
    if (observable != PRS_OBS_GRAD_ENERGY && observable != PRS_OBS_SMOOTH_AREA) return PRS_EINVAL;
    if (observable == PRS_OBS_SMOOTH_AREA && !(eps_smooth > 0)) return PRS_EINVAL;
    if (!s->initialised) return PRS_ESTATE;
    Scratch mem;
    void* grad = mem.get((size_t)s->g.S * s->elem);
    if (!grad) return PRS_ENOMEM;
    DiagScratch scr = s->scr;
    cudaError_t e = launch_observable(s, s->phi[s->cur], grad, observable, eps_smooth, scr);
    if (e != cudaSuccess) return cuda_fail(e, "prs_observable launch");
    e = cudaMemcpyAsync(s->h_status, s->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "prs_observable");
    *J = s->h_status->result.sum_w;
    return PRS_OK;
}

extern "C" int prs_adjoint(prs_sim* s, int64_t nsteps, int observable, double eps_smooth, int64_t ckpt_every,
                           double* J, double* dJ_dalpha, void* d_dJ_dphi_init, void* d_dJ_dv_init)
{
    if (!s || nsteps < 0 || ckpt_every < 1) return PRS_EINVAL;
    if (observable != PRS_OBS_GRAD_ENERGY && observable != PRS_OBS_SMOOTH_AREA) return PRS_EINVAL;
    if (observable == PRS_OBS_SMOOTH_AREA && !(eps_smooth > 0)) return PRS_EINVAL;
    if (!s->initialised) return PRS_ESTATE;
    if (nsteps > 0 && !cfl_ok(s->p, s->n + nsteps - 1)) return PRS_EINVAL;
    const size_t fbytes = (size_t)s->g.S * s->elem;
    const int64_t n0 = s->n;
    const int64_t K = ckpt_every < nsteps ? ckpt_every : (nsteps > 0 ? nsteps : 1);
    const int64_t nseg = nsteps > 0 ? (nsteps + K - 1) / K : 0;
    const bool repro = (s->p.flags & PRS_REPRO) != 0;

    Scratch mem;
    char* ckpt = nseg ? (char*)mem.get(2 * fbytes * (size_t)nseg) : nullptr;  // (phi, v) at n0 + i K
    char* seg = K > 1 ? (char*)mem.get(2 * fbytes * (size_t)(K - 1)) : nullptr;  // states 1..K-1 of a segment
    char* adj = (char*)mem.get(4 * fbytes);                                        // lphi[2], lv[2]
    DiagAcc* dacc = (DiagAcc*)mem.get(sizeof(DiagAcc) * (size_t)(nsteps > 0 ? nsteps : 1));
    if ((nseg && !ckpt) || (K > 1 && !seg) || !adj || !dacc) return PRS_ENOMEM;
    std::vector<DiagAcc> hacc((size_t)(nsteps > 0 ? nsteps : 1));

    auto cphi = [&](int64_t i) { return ckpt + 2 * fbytes * (size_t)i; };
    auto sphi = [&](int64_t k, int64_t i) -> char* {  // state k (0..K-1) of segment i
        return k == 0 ? cphi(i) : seg + 2 * fbytes * (size_t)(k - 1);
    };
    auto sv = [&](int64_t k, int64_t i) -> char* { return sphi(k, i) + fbytes; };
    char* lphi[2] = {adj, adj + fbytes};
    char* lv[2] = {adj + 2 * fbytes, adj + 3 * fbytes};
    unsigned int* err = &s->d_status->error;
    cudaStream_t st = s->stream;
#define PRS_TRY(call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, "prs_adjoint"); \
    } while (0)

    // forward, keeping a checkpoint at the start of every segment
    for (int64_t i = 0; i < nseg; ++i) {
        PRS_TRY(cudaMemcpyAsync(cphi(i), s->phi[s->cur], fbytes, cudaMemcpyDeviceToDevice, st));
        PRS_TRY(cudaMemcpyAsync(cphi(i) + fbytes, s->dphi, fbytes, cudaMemcpyDeviceToDevice, st));
        const int64_t len = (i + 1) * K <= nsteps ? K : nsteps - i * K;
        int rc = prs_step(s, len);
        if (rc) return rc;
    }
    // J and dJ/dphi at the end; dJ/dv = 0 there
    DiagScratch scr = s->scr;
    PRS_TRY(launch_observable(s, s->phi[s->cur], lphi[0], observable, eps_smooth, scr));
    PRS_TRY(cudaMemcpyAsync(s->h_status, s->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    PRS_TRY(cudaMemsetAsync(lv[0], 0, fbytes, st));
    int cur = 0;
    // backward over segments
    for (int64_t i = nseg - 1; i >= 0; --i) {
        const int64_t a = n0 + i * K;
        const int64_t len = (i + 1) * K <= nsteps ? K : nsteps - i * K;
        for (int64_t k = 0; k + 1 < len; ++k) {  // recompute states a+1 .. a+len-1
            double c[5];
            step_coefficients(s->p, a + k, c);
            PRS_TRY(launch_step_io(s->g, s->p.precision, repro, sphi(k, i), sphi(k + 1, i), sv(k, i), sv(k + 1, i),
                                   &c[0], &c[1], &c[2], 1, s->rc, err, st));
        }
        for (int64_t k = len - 1; k >= 0; --k) {
            double c[5];
            step_coefficients(s->p, a + k, c);
            const double opd = 1.0 + c[3];
            AdjCoef ac{c[0], c[1], c[2], -2.0 / (opd * opd) * c[4], -s->p.deta / (opd * opd) * c[4]};
            DiagScratch sk = scr;
            sk.result = dacc + (a + k - n0);
            PRS_TRY(launch_adjoint_step(s, sphi(k, i), sv(k, i), lphi[cur], lv[cur], lphi[1 - cur], lv[1 - cur], ac,
                                        sk));
            cur = 1 - cur;
        }
    }
    if (d_dJ_dphi_init) PRS_TRY(cudaMemcpyAsync(d_dJ_dphi_init, lphi[cur], fbytes, cudaMemcpyDeviceToDevice, st));
    if (d_dJ_dv_init) PRS_TRY(cudaMemcpyAsync(d_dJ_dv_init, lv[cur], fbytes, cudaMemcpyDeviceToDevice, st));
    if (nsteps > 0)
        PRS_TRY(cudaMemcpyAsync(hacc.data(), dacc, sizeof(DiagAcc) * (size_t)nsteps, cudaMemcpyDeviceToHost, st));
    PRS_TRY(cudaStreamSynchronize(st));
    const double Jv = s->h_status->result.sum_w;
    // the bounded waits of the step kernels report through the error word
    PRS_TRY(cudaMemcpyAsync(&s->h_status->error, &s->d_status->error, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                            st));
    PRS_TRY(cudaStreamSynchronize(st));
#undef PRS_TRY
    int rc = check_device_error(s);
    if (rc) return rc;
    double da = 0.0;
    for (int64_t k = 0; k < nsteps; ++k) da += hacc[(size_t)k].sum_w;  // fixed order: step index
    if (J) *J = Jv;
    if (dJ_dalpha) *dJ_dalpha = da;
    return PRS_OK;
}

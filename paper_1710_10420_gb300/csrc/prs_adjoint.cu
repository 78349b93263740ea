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
// The sweep carries lphi (pointwise) and lt (the only adjoint field read across
// sites): step n reads lt_n with its neighbours and phi^n, dphi^n, lphi_{n+1} at
// the site, and writes
//     lphi_n = lphi_{n+1} + c2 (L lt_n - f'(phi^n) lt_n),  lt_{n-1} = c1 lt_n + deta lphi_n
// (at the first step of the run it writes lv_n0 = c1 lt_n0 instead): 24 bytes per
// site in FP32, one pass.  The L phi of dJ/dalpha becomes phi (L lt) in the sum over
// sites (L is symmetric), so phi is never read across sites in the FP32 kernels,
// which stage all four fields in shared memory with the TMA engine (prs_tile.cuh
// does the same for the forward step); the generic kernel keeps the form above.
//
// The forward states are either all kept (when they fit in device memory: GB300's
// HBM holds e.g. 1271 states of a 256^3 FP32 run) or checkpointed every K steps
// and each segment recomputed into segment storage (the step kernel writes phi
// and dphi out of place) before it is walked backwards.  The state is never
// inverted algebraically: 1/c1 grows without bound as delta -> 1.
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
#include "prs_tile.cuh"

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
__global__ void __launch_bounds__(256) k_observable(const R* __restrict__ phi, R* __restrict__ grad,
                                                    R* __restrict__ grad_deta, Geo g, int obs, double eps,
                                                    double inv_dx2, double area_scale, double deta, DiagScratch scr)
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
        if (grad_deta) grad_deta[s] = (R)gr * (R)deta;  // lt at the last step: lv = 0 there
    }
    block_reduce_and_finish(DiagAcc{J, 0.0, 0, 0, 0, 0}, scr);
}

// FP32 runs: the same observables with each site's terms in FP32, added to the
// thread's FP64 sum once per site (FP64 transcendental functions per link would
// make this pass cost as much as hundreds of steps on this GPU).  For the smooth
// area, 1 - t_s t_u of two same-sign values near the vacua cancels in FP32; with
// u = 1 - |tanh x| = 2/(e^{2|x|} + 1) it is u_s + u_u - u_s u_u, which does not, and
// 1 - t_s^2 = u_s (2 - u_s).
struct SmoothSign {
    float t, u;  // tanh(x) and 1 - |tanh(x)|
};

__device__ __forceinline__ SmoothSign smooth_sign(float x)
{
    const float ax = fabsf(x);
    const float u = ax > 0.5f ? 2.0f / (expf(2.0f * ax) + 1.0f) : 1.0f - tanhf(ax);
    const float t = ax > 0.5f ? 1.0f - u : tanhf(ax);
    return SmoothSign{copysignf(t, x), u};
}

__device__ __forceinline__ float one_minus_tt(const SmoothSign& a, const SmoothSign& b)
{
    if ((a.t < 0.0f) != (b.t < 0.0f)) return 1.0f + fabsf(a.t) * fabsf(b.t);
    return a.u + b.u - a.u * b.u;
}

template <int D>
__global__ void __launch_bounds__(256) k_observable_f32(const float* __restrict__ phi, float* __restrict__ grad,
                                                        float* __restrict__ grad_deta, Geo g, int obs, float inv_eps,
                                                        float inv_dx2, double jscale, float gscale, float deta,
                                                        DiagScratch scr)
{
    double J = 0.0;
    PRS_FOR_SITES(g, s, x, y, z)
    {
        const Nbr n = neighbours(g, s, x, y, z);
        const int64_t up[3] = {n.xp, n.yp, n.zp}, dn[3] = {n.xm, n.ym, n.zm};
        const float ps = phi[s];
        float js = 0.0f, gr = 0.0f;
        if (obs == PRS_OBS_GRAD_ENERGY) {
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float pu = phi[up[d]], pd = phi[dn[d]];
                const float gd = pu - ps;
                js += gd * gd;
                gr += (ps - pu) + (ps - pd);
            }
        } else {
            const SmoothSign ss = smooth_sign(ps * inv_eps);
            float nb = 0.0f;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const SmoothSign su = smooth_sign(phi[up[d]] * inv_eps);
                js += one_minus_tt(ss, su);
                nb += su.t + smooth_sign(phi[dn[d]] * inv_eps).t;
            }
            gr = -(ss.u * (2.0f - ss.u)) * nb;
        }
        gr *= gscale;
        J += (double)js;
        grad[s] = gr;
        if (grad_deta) grad_deta[s] = gr * deta;  // lt at the last step: lv = 0 there
    }
    block_reduce_and_finish(DiagAcc{J * jscale, 0.0, 0, 0, 0, 0}, scr);
}

// One reverse step n: lt_in = lt_n, lphi = lphi_{n+1} (updated in place to lphi_n),
// lt_out = lt_{n-1} (or lv_n at the run's first step, `last`), using the forward
// state (phi, v) at n; the dJ/dalpha term of this step lands in *scr.result.
template <typename R, int D>
__global__ void __launch_bounds__(256)
    k_adjoint_step(const R* __restrict__ phi, const R* __restrict__ v, const R* __restrict__ lt_in,
                   R* __restrict__ lphi, R* __restrict__ lt_out, Geo g, AdjCoef c, RunConst<R> rc, bool last,
                   DiagScratch scr)
{
    const R c1 = (R)c.c1, c2 = (R)c.c2, cV = (R)c.cV, deta = rc.deta;
    const R dc1 = (R)c.dc1, dc2 = (R)c.dc2;
    // per-thread sum of the dJ/dalpha terms in working precision, compensated
    // (Kahan): FP64 arithmetic per site would dominate the step on this GPU
    R da = 0, comp = 0;
    PRS_FOR_SITES(g, s, x, y, z)
    {
        const Nbr n = neighbours(g, s, x, y, z);
        const R lts = lt_in[s];
        const R Llt = (pair_sum<R, D>(lt_in, n) - rc.twoD * lts) * rc.inv_dx2;
        const R p = phi[s];
        const R fprime = cV * ((R)3 * (p * p) * rc.inv_phi0sq - (R)1);
        const R lp = lphi[s] + c2 * (Llt - fprime * lts);
        lphi[s] = lp;
        lt_out[s] = last ? c1 * lts : c1 * lts + deta * lp;
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

// ------------------------------------------------------- staged FP32 sweep

constexpr int kAdjItems = 2;  // float4 per thread per plane: 2048 sites per plane tile

struct AdjTile {
    const float* phi;    // phi^n (pointwise)
    const float* lt_in;  // lt_n (stencil)
    const float* v;      // dphi^n (pointwise)
    float* lphi;         // lphi_{n+1} -> lphi_n (pointwise, in place)
    float* lt_out;       // lt_{n-1}, or lv_n when last
    int nx, ny, nz, t;   // box; t = rows per plane tile (3D) or per band (2D)
    int y0, z0, len;     // first row, first plane (3D), planes (3D) or rows (2D)
};

struct AdjCoefF {
    float c1, c2, cV, dc1, dc2;
};

// 4 pair sums (x+ + x-) + (y+ + y-) [+ (z+ + z-)] of a float4 and its neighbours.
__device__ __forceinline__ float4 pairs4(float4 c, float left, float right, float4 yp, float4 ym, float4 zp, float4 zm,
                                         bool three_d)
{
    float4 r;
    r.x = (c.y + left) + (yp.x + ym.x);
    r.y = (c.z + c.x) + (yp.y + ym.y);
    r.z = (c.w + c.y) + (yp.z + ym.z);
    r.w = (right + c.z) + (yp.w + ym.w);
    if (three_d) {
        r.x = r.x + (zp.x + zm.x);
        r.y = r.y + (zp.y + zm.y);
        r.z = r.z + (zp.z + zm.z);
        r.w = r.w + (zp.w + zm.w);
    }
    return r;
}

struct AdjSum {  // per-thread compensated FP32 sum, folded into FP64 once per plane
    double tot;
    float s, comp;
    __device__ __forceinline__ void add(float term)
    {
        const float yk = term - comp;
        const float t = s + yk;
        comp = (t - s) - yk;
        s = t;
    }
    __device__ __forceinline__ void fold()
    {
        tot += (double)s;
        s = 0.0f;
        comp = 0.0f;
    }
};

// The pointwise part of one reverse step for 4 sites: p = phi^n, l = lt_n and sl its
// pair sums, vv = dphi^n, lp = lphi_{n+1} (becomes lphi_n), out = lt_{n-1} (lv_n when
// last).  The dJ/dalpha sum over sites of lt (dc1 v + dc2 (L phi - f)) is taken as
// the sum of lt (dc1 v - dc2 f) + dc2 phi (L lt): L is symmetric on the periodic
// lattice, so the totals are equal, and phi is then needed at the site only.
__device__ __forceinline__ void adj_update4(float4 p, float4 l, float4 sl, float4 vv, float4& lp, float4& out,
                                            const AdjCoefF& k, const RunConst<float>& rc, bool last, AdjSum& da)
{
    const float pc[4] = {p.x, p.y, p.z, p.w};
    const float lc[4] = {l.x, l.y, l.z, l.w}, slc[4] = {sl.x, sl.y, sl.z, sl.w};
    const float vc[4] = {vv.x, vv.y, vv.z, vv.w};
    float lpo[4] = {lp.x, lp.y, lp.z, lp.w}, o[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float q = pc[e], lt = lc[e];
        const float Llt = (slc[e] - rc.twoD * lt) * rc.inv_dx2;
        const float fprime = k.cV * (3.0f * (q * q) * rc.inv_phi0sq - 1.0f);
        const float lpn = lpo[e] + k.c2 * (Llt - fprime * lt);
        lpo[e] = lpn;
        o[e] = last ? k.c1 * lt : k.c1 * lt + rc.deta * lpn;
        const float f = (k.cV * q) * ((q * q) * rc.inv_phi0sq - 1.0f);
        da.add(lt * (k.dc1 * vc[e] - k.dc2 * f) + k.dc2 * (q * Llt));
    }
    lp = make_float4(lpo[0], lpo[1], lpo[2], lpo[3]);
    out = make_float4(o[0], o[1], o[2], o[3]);
}

// Shared memory of the staged sweep: the barriers, a 4-slot ring of lt (read with its
// neighbours: t+2 rows per 3D plane, t rows per 2D band) and a 2-slot ring holding
// phi^n, dphi^n and lphi_{n+1} of t rows each (read at the site only).
__host__ __device__ constexpr size_t adj_smem(int dims, int nx, int t)
{
    return 128 + 4 * (size_t)(dims == 3 ? t + 2 : t) * nx * 4 + 2 * 3 * (size_t)t * nx * 4;
}

// 3D: a tile of t rows x len planes.  Copy i (one mbarrier per lt slot) brings lt
// plane i of the tile (local: global z0-1+i) and, for i >= 2, the pointwise fields of
// local plane i-2, which iteration i-2 uses together with lt planes i-2 .. i.
template <int ITEMS>
__global__ void __launch_bounds__(kFastThreads, 2)
    k_adjoint3d_f32(AdjTile T, AdjCoefF k, RunConst<float> rc, bool last, DiagScratch scr, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    const int nx = T.nx, ny = T.ny, nz = T.nz, ty = T.t;
    const int tile = (ty + 2) * nx;  // floats per lt slot
    const int ptile = ty * nx;       // floats per pointwise field in a slot
    float* ringL = reinterpret_cast<float*>(smem_raw + 128);
    float* ringW = ringL + 4 * tile;  // [slot 0..1][phi, dphi, lphi][ptile]
    const int tid = threadIdx.x, lane = tid & 31;
    const int ytiles = ny / ty;
    const int y0 = (blockIdx.x % ytiles) * ty;
    const int z0 = (blockIdx.x / ytiles) * T.len;
    const int zn = min(T.len, nz - z0);
    const int nq = nx >> 2;
    const size_t plane = (size_t)nx * ny;
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
        mbar_fence_init();
        fence_proxy_async_global();
    }
    __syncthreads();
    const int ytop = (y0 == 0 ? ny : y0) - 1;
    const int ybot = (y0 + ty == ny) ? 0 : y0 + ty;
    const unsigned rowb = (unsigned)nx * 4u;
    const int nloc = zn + 2;
    auto issue = [&](int i) {
        int p = z0 - 1 + i;
        p = p < 0 ? p + nz : (p >= nz ? p - nz : p);
        uint64_t* b = &bar[i & 3];
        const bool pw = i >= 2;
        mbar_arrive_expect_tx(b, rowb * (unsigned)(ty + 2) + (pw ? 3u * rowb * (unsigned)ty : 0u));
        float* dst = ringL + (i & 3) * tile;
        const float* src = T.lt_in + (size_t)p * plane;
        bulk_g2s(dst, src + (size_t)ytop * nx, rowb, b);
        bulk_g2s(dst + nx, src + (size_t)y0 * nx, rowb * (unsigned)ty, b);
        bulk_g2s(dst + (size_t)(ty + 1) * nx, src + (size_t)ybot * nx, rowb, b);
        if (pw) {
            const size_t o = (size_t)(z0 + i - 2) * plane + (size_t)y0 * nx;
            float* w = ringW + ((i - 2) & 1) * 3 * ptile;
            bulk_g2s(w, T.phi + o, rowb * (unsigned)ty, b);
            bulk_g2s(w + ptile, T.v + o, rowb * (unsigned)ty, b);
            bulk_g2s(w + 2 * ptile, T.lphi + o, rowb * (unsigned)ty, b);
        }
    };
    int issued = -1;
    if (tid == 0)
        for (int i = 0; i < 3 && i < nloc; ++i) issue(i), issued = i;
    int row[ITEMS], col[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        int q = tid + kFastThreads * j;
        row[j] = q / nq;
        col[j] = q - row[j] * nq;
    }
    AdjSum da{0.0, 0.0f, 0.0f};
    for (int zi = 0; zi < zn; ++zi) {
        bool ok = true;
        if (zi == 0) ok = mbar_wait(&bar[0], 0, err) && mbar_wait(&bar[1], 0, err);
        ok = ok && mbar_wait(&bar[(zi + 2) & 3], ((zi + 2) >> 2) & 1, err);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain(bar, zi, issued, err);
            break;
        }
        if (tid == 0 && zi + 3 < nloc) issue(zi + 3), issued = zi + 3;
        const int sm = (zi & 3) * tile + nx, sc = ((zi + 1) & 3) * tile + nx, sp = ((zi + 2) & 3) * tile + nx;
        const float* w = ringW + (zi & 1) * 3 * ptile;
        const size_t bz = (size_t)(z0 + zi) * plane + (size_t)y0 * nx;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int off = row[j] * nx + 4 * col[j];
            const float4 c = lds4(ringL + sc + off);
            float left, right;
            x_halo(ringL + sc + row[j] * nx, col[j], nq, nx, lane, c, left, right);
            const float4 S = pairs4(c, left, right, lds4(ringL + sc + off + nx), lds4(ringL + sc + off - nx),
                                    lds4(ringL + sp + off), lds4(ringL + sm + off), true);
            float4 lp = lds4(w + 2 * ptile + off), out;
            adj_update4(lds4(w + off), c, S, lds4(w + ptile + off), lp, out, k, rc, last, da);
            stg4(T.lphi + bz + off, lp);
            stg4(T.lt_out + bz + off, out);
        }
        da.fold();
    }
    block_reduce_and_finish(DiagAcc{da.tot, 0.0, 0, 0, 0, 0}, scr);
}

// 2D: a tile of len rows in bands of t rows.  Local lt band 0 is the row above the
// tile, nb+1 the row below; copy i brings lt band i and, for i >= 2, the pointwise
// fields of band i-2 of the tile.
template <int ITEMS>
__global__ void __launch_bounds__(kFastThreads, 2)
    k_adjoint2d_f32(AdjTile T, AdjCoefF k, RunConst<float> rc, bool last, DiagScratch scr, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    const int nx = T.nx, ny = T.ny, rb = T.t;
    const int slot = rb * nx;  // floats per lt slot and per pointwise field in a slot
    float* ringL = reinterpret_cast<float*>(smem_raw + 128);
    float* ringW = ringL + 4 * slot;  // [slot 0..1][phi, dphi, lphi][slot]
    const int tid = threadIdx.x, lane = tid & 31;
    const int y0 = blockIdx.x * T.len;
    const int yn = min(T.len, ny - y0);
    const int nb = yn / rb;
    const int nq = nx >> 2;
    const int rmask = 4 * rb - 1;  // ring rows: a power of two (rb = 2048/nx, nx dividing 2048)
    const unsigned rowb = (unsigned)nx * 4u;
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
        mbar_fence_init();
        fence_proxy_async_global();
    }
    __syncthreads();
    const int nloc = nb + 2;
    auto issue = [&](int i) {
        uint64_t* b = &bar[i & 3];
        const bool pw = i >= 2;
        const unsigned pwb = pw ? 3u * rowb * (unsigned)rb : 0u;
        float* dst = ringL + (i & 3) * slot;
        if (i == 0 || i == nb + 1) {
            const int y = i == 0 ? (y0 == 0 ? ny : y0) - 1 : ((y0 + yn == ny) ? 0 : y0 + yn);
            const int r = i == 0 ? rb - 1 : 0;
            mbar_arrive_expect_tx(b, rowb + pwb);
            bulk_g2s(dst + (size_t)r * nx, T.lt_in + (size_t)y * nx, rowb, b);
        } else {
            mbar_arrive_expect_tx(b, rowb * (unsigned)rb + pwb);
            bulk_g2s(dst, T.lt_in + (size_t)(y0 + (i - 1) * rb) * nx, rowb * (unsigned)rb, b);
        }
        if (pw) {
            const size_t o = (size_t)(y0 + (i - 2) * rb) * nx;
            float* w = ringW + ((i - 2) & 1) * 3 * slot;
            bulk_g2s(w, T.phi + o, rowb * (unsigned)rb, b);
            bulk_g2s(w + slot, T.v + o, rowb * (unsigned)rb, b);
            bulk_g2s(w + 2 * slot, T.lphi + o, rowb * (unsigned)rb, b);
        }
    };
    int issued = -1;
    if (tid == 0)
        for (int i = 0; i < 3 && i < nloc; ++i) issue(i), issued = i;
    int row[ITEMS], col[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        int q = tid + kFastThreads * j;
        row[j] = q / nq;
        col[j] = q - row[j] * nq;
    }
    AdjSum da{0.0, 0.0f, 0.0f};
    for (int bi = 0; bi < nb; ++bi) {
        bool ok = true;
        if (bi == 0) ok = mbar_wait(&bar[0], 0, err) && mbar_wait(&bar[1], 0, err);
        ok = ok && mbar_wait(&bar[(bi + 2) & 3], ((bi + 2) >> 2) & 1, err);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain(bar, bi, issued, err);
            break;
        }
        if (tid == 0 && bi + 3 < nloc) issue(bi + 3), issued = bi + 3;
        const float* w = ringW + (bi & 1) * 3 * slot;
        const int yb = y0 + bi * rb;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int lr = (bi + 1) * rb + row[j];
            const int rc0 = (lr & rmask) * nx, ru = ((lr - 1) & rmask) * nx, rd = ((lr + 1) & rmask) * nx;
            const float4 c = lds4(ringL + rc0 + 4 * col[j]);
            float left, right;
            x_halo(ringL + rc0, col[j], nq, nx, lane, c, left, right);
            const float4 ym = lds4(ringL + ru + 4 * col[j]), yp = lds4(ringL + rd + 4 * col[j]);
            const float4 S = pairs4(c, left, right, yp, ym, ym, ym, false);
            const int off = row[j] * nx + 4 * col[j];
            float4 lp = lds4(w + 2 * slot + off), out;
            adj_update4(lds4(w + off), c, S, lds4(w + slot + off), lp, out, k, rc, last, da);
            const size_t o = (size_t)yb * nx + off;
            stg4(T.lphi + o, lp);
            stg4(T.lt_out + o, out);
        }
        da.fold();
    }
    block_reduce_and_finish(DiagAcc{da.tot, 0.0, 0, 0, 0, 0}, scr);
}

// FP32 boxes the staged sweep takes: x a multiple of 128 dividing 2048 (2D and 3D),
// y divisible by the rows of a tile, and the rings within 113 KB (two CTAs per SM).
bool adj_fast_ok(const Geo& g, int precision)
{
    if (precision != PRS_FP32) return false;
    if (g.nx % 128 != 0 || g.nx > kAdjItems * 1024 || (kAdjItems * 1024) % g.nx != 0) return false;
    const int t = kAdjItems * 1024 / g.nx;
    if (g.ny % t != 0) return false;
    return adj_smem(g.dims, g.nx, t) <= 113 * 1024;
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

cudaError_t launch_observable(const prs_sim* s, const void* phi, void* grad, void* grad_deta, int obs, double eps,
                              DiagScratch scr)
{
    const double area_scale = 1.0 / ((double)s->g.S * s->p.dx);
    const dim3 grid = grid_for(s->g);
    if ((int)(grid.x * grid.y) > scr.max_blocks) return cudaErrorInvalidValue;
#define PRS_OBS_LAUNCH(R, D)                                                                                     \
    k_observable<R, D><<<grid, 256, 0, s->stream>>>((const R*)phi, (R*)grad, (R*)grad_deta, s->g, obs, eps,       \
                                                    s->rc[1], area_scale, s->p.deta, scr)
    if (s->p.precision == PRS_FP32) {
        // J = jscale * sum of the per-site terms, dJ/dphi = gscale * per-site gradient term
        const bool area = obs == PRS_OBS_SMOOTH_AREA;
        const double jscale = area ? 0.5 * area_scale : 0.5 * s->rc[1];
        const float gscale = area ? (float)(0.5 * area_scale / eps) : (float)s->rc[1];
        const float inv_eps = area ? (float)(1.0 / eps) : 0.0f;
        if (s->g.dims == 3)
            k_observable_f32<3><<<grid, 256, 0, s->stream>>>((const float*)phi, (float*)grad, (float*)grad_deta,
                                                             s->g, obs, inv_eps, (float)s->rc[1], jscale, gscale,
                                                             (float)s->p.deta, scr);
        else
            k_observable_f32<2><<<grid, 256, 0, s->stream>>>((const float*)phi, (float*)grad, (float*)grad_deta,
                                                             s->g, obs, inv_eps, (float)s->rc[1], jscale, gscale,
                                                             (float)s->p.deta, scr);
    } else {
        if (s->g.dims == 3) PRS_OBS_LAUNCH(double, 3); else PRS_OBS_LAUNCH(double, 2);
    }
#undef PRS_OBS_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const prs_sim* s, const void* phi, const void* v, const void* lt_in, void* lphi,
                                void* lt_out, const AdjCoef& c, bool last, DiagScratch scr, unsigned int* err)
{
    const Geo& g = s->g;
    if (adj_fast_ok(g, s->p.precision)) {
        static std::atomic<unsigned long long> attr3{0}, attr2{0};
        const int t = kAdjItems * 1024 / g.nx;
        const int slots = 2 * sm_count_current();
        AdjTile T{(const float*)phi, (const float*)lt_in, (const float*)v, (float*)lphi, (float*)lt_out,
                  g.nx, g.ny, g.nz, t, 0, 0, 0};
        AdjCoefF k{(float)c.c1, (float)c.c2, (float)c.cV, (float)c.dc1, (float)c.dc2};
        RunConst<float> rc = run_const<float>(s->rc);
        if (g.dims == 3) {
            const size_t sm = adj_smem(3, g.nx, t);
            {
                const cudaError_t e = smem_limit_once(attr3, (const void*)k_adjoint3d_f32<kAdjItems>, 113 * 1024);
                if (e != cudaSuccess) return e;
            }
            const int ytiles = g.ny / t;
            // z-chunks: whole waves of resident CTAs, chunks of >= 8 planes, one partial per block
            int best = 1;
            double best_score = -1;
            for (int nc = 1; nc <= g.nz / 8 || nc == 1; ++nc) {
                const int cz = (g.nz + nc - 1) / nc, n = (g.nz + cz - 1) / cz;
                const long long blocks = (long long)ytiles * n;
                if (blocks > scr.max_blocks) break;
                const long long waves = (blocks + slots - 1) / slots;
                const double score = (double)blocks / (double)(waves * slots) * cz / (cz + 2.0);
                if (score > best_score + 1e-9) best_score = score, best = n;
            }
            T.len = (g.nz + best - 1) / best;
            const int blocks = ytiles * ((g.nz + T.len - 1) / T.len);
            k_adjoint3d_f32<kAdjItems><<<blocks, kFastThreads, sm, s->stream>>>(T, k, rc, last, scr, err);
            return cudaGetLastError();
        }
        const size_t sm = adj_smem(2, g.nx, t);
        {
            const cudaError_t e = smem_limit_once(attr2, (const void*)k_adjoint2d_f32<kAdjItems>, 113 * 1024);
            if (e != cudaSuccess) return e;
        }
        const int bands = g.ny / t;
        int nb = (bands + 4 * slots - 1) / (4 * slots);  // bands per tile: about four waves of tiles
        if (nb < 4) nb = 4;
        T.len = nb * t;
        int blocks = (g.ny + T.len - 1) / T.len;
        if (blocks > scr.max_blocks) {
            T.len = ((g.ny + scr.max_blocks - 1) / scr.max_blocks + t - 1) / t * t;
            blocks = (g.ny + T.len - 1) / T.len;
        }
        k_adjoint2d_f32<kAdjItems><<<blocks, kFastThreads, sm, s->stream>>>(T, k, rc, last, scr, err);
        return cudaGetLastError();
    }
    const dim3 grid = grid_for(g);
    if ((int)(grid.x * grid.y) > scr.max_blocks) return cudaErrorInvalidValue;
#define PRS_ADJ_LAUNCH(R, D)                                                                                  \
    k_adjoint_step<R, D><<<grid, 256, 0, s->stream>>>((const R*)phi, (const R*)v, (const R*)lt_in, (R*)lphi, \
                                                      (R*)lt_out, g, c, run_const<R>(s->rc), last, scr)
    if (s->p.precision == PRS_FP32) {
        if (g.dims == 3) PRS_ADJ_LAUNCH(float, 3); else PRS_ADJ_LAUNCH(float, 2);
    } else {
        if (g.dims == 3) PRS_ADJ_LAUNCH(double, 3); else PRS_ADJ_LAUNCH(double, 2);
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

static int prs_observable_impl(prs_sim* s, int observable, double eps_smooth, double* J)
{
    if (!s || !J) return PRS_EINVAL;
    if (observable != PRS_OBS_GRAD_ENERGY && observable != PRS_OBS_SMOOTH_AREA) return PRS_EINVAL;
    if (observable == PRS_OBS_SMOOTH_AREA && !(eps_smooth > 0)) return PRS_EINVAL;
    if (!s->initialised) return PRS_ESTATE;
    Scratch mem;
    void* grad = mem.get((size_t)s->g.S * s->elem);
    if (!grad) return PRS_ENOMEM;
    DiagScratch scr = s->scr;
    cudaError_t e = launch_observable(s, s->phi[s->cur], grad, nullptr, observable, eps_smooth, scr);
    if (e != cudaSuccess) return cuda_fail(e, "prs_observable launch");
    e = cudaMemcpyAsync(s->h_status, s->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "prs_observable");
    *J = s->h_status->result.sum_w;
    return PRS_OK;
}

static int prs_adjoint_impl(prs_sim* s, int64_t nsteps, int observable, double eps_smooth, int64_t ckpt_every,
                           double* J, double* dJ_dalpha, void* d_dJ_dphi_init, void* d_dJ_dv_init)
{
    if (!s || nsteps < 0 || ckpt_every < 0) return PRS_EINVAL;
    if (observable != PRS_OBS_GRAD_ENERGY && observable != PRS_OBS_SMOOTH_AREA) return PRS_EINVAL;
    if (observable == PRS_OBS_SMOOTH_AREA && !(eps_smooth > 0)) return PRS_EINVAL;
    if (!s->initialised) return PRS_ESTATE;
    if (nsteps > 0 && !cfl_ok_over(s->p, s->n, nsteps)) return PRS_EINVAL;
    const size_t fbytes = (size_t)s->g.S * s->elem;
    const int64_t n0 = s->n;
    const bool repro = (s->p.flags & PRS_REPRO) != 0;
    // every state kept (K = nsteps, no recomputation) when asked with ckpt_every = 0
    // and it fits in device memory with 2 GB to spare; else checkpoints every K
    int64_t K = ckpt_every;
    bool keep_all = false;
    if (ckpt_every == 0) {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const double need = 2.0 * (double)fbytes * (double)(nsteps + 1) + 3.0 * (double)fbytes + 2e9;
        keep_all = need <= (double)free_b + (double)s->adj_ws_bytes;  // the kept workspace is reusable
        K = keep_all ? (nsteps > 0 ? nsteps : 1) : 64;
    }
    if (K > nsteps) K = nsteps > 0 ? nsteps : 1;
    const int64_t nseg = nsteps > 0 ? (nsteps + K - 1) / K : 0;

    // one workspace, kept with the run for the next call: [states][lphi, lt[2]][dacc].
    // keep_all: states 0..nsteps back to back; else one checkpoint per segment plus
    // states 1..K-1 of the segment being swept
    // every array starts on a 256-byte boundary (odd boxes have sizes that are not)
    const size_t fs = (fbytes + 255) & ~(size_t)255;
    const size_t nstate = keep_all ? (size_t)(nsteps + 1) : (size_t)nseg + (size_t)(K > 1 ? K - 1 : 0);
    const size_t need = 2 * fs * nstate + 3 * fs + sizeof(DiagAcc) * (size_t)(nsteps > 0 ? nsteps : 1);
    if (s->adj_ws_bytes < need) {
        cudaFree(s->adj_ws);
        s->adj_ws = nullptr;
        s->adj_ws_bytes = 0;
        if (cudaMalloc(&s->adj_ws, need) != cudaSuccess) {
            cudaGetLastError();
            s->adj_ws = nullptr;
            return PRS_ENOMEM;
        }
        s->adj_ws_bytes = need;
    }
    char* ckpt = (char*)s->adj_ws;
    char* seg = keep_all ? nullptr : ckpt + 2 * fs * (size_t)nseg;
    char* adj = ckpt + 2 * fs * nstate;  // lphi, lt[2]
    DiagAcc* dacc = (DiagAcc*)(adj + 3 * fs);
    std::vector<DiagAcc> hacc((size_t)(nsteps > 0 ? nsteps : 1));

    auto state = [&](int64_t k, int64_t i) -> char* {  // phi of state k (0..K-1) of segment i; dphi at + fs
        if (keep_all) return ckpt + 2 * fs * (size_t)(i * K + k);
        return k == 0 ? ckpt + 2 * fs * (size_t)i : seg + 2 * fs * (size_t)(k - 1);
    };
    char* lphi = adj;
    char* lt[2] = {adj + fs, adj + 2 * fs};
    unsigned int* err = &s->d_status->error;
    cudaStream_t st = s->stream;
#define PRS_TRY(call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, "prs_adjoint"); \
    } while (0)

    DiagScratch scr = s->scr;
    // phase boundaries for prs_adjoint_timing: start, end of the forward (with J), then the
    // start of each segment's recomputation and of its reverse sweep, then the end
    const size_t nev = 3 + 2 * (size_t)nseg;
    while (s->adj_ev.size() < nev) {
        cudaEvent_t e;
        PRS_TRY(cudaEventCreate(&e));
        s->adj_ev.push_back(e);
    }
    s->adj_timed = false;
    PRS_TRY(cudaEventRecord(s->adj_ev[0], st));
    // Fill the states k_from+1 .. k_to (slot(k): phi of state k, dphi at + fs) from state
    // k_from, step n_first + k_from onwards: in pairs through the two-step pass, which
    // also stores the state between its two steps (FP32 3D boxes it takes, without
    // PRS_REPRO: 24 bytes a site per two states against 32), else one step at a time.
    const bool pairs_ok = s->p.precision == PRS_FP32 && !repro && s->g.dims == 3 && tblock_ok(s->g, PRS_FP32);
    const RunConst<float> rcf{(float)s->rc[0], (float)s->rc[1], (float)s->rc[2],
                              (float)s->rc[3], (float)s->rc[4], (float)s->rc[5]};
    auto fill = [&](auto slot, int64_t n_first, int64_t k_from, int64_t k_to) -> cudaError_t {
        for (int64_t k = k_from; k < k_to;) {
            double c0[5], c1[5];
            step_coefficients(s->p, n_first + k, c0);
            cudaError_t e;
            if (pairs_ok && k + 2 <= k_to) {
                step_coefficients(s->p, n_first + k + 1, c1);
                char* x = slot(k);
                char* y = slot(k + 1);
                char* z = slot(k + 2);
                e = launch_step_t2(s->g, (const float*)x, (float*)z, (const float*)(x + fs), (float*)(z + fs),
                                   kick_f32(c0, s->rc), kick_f32(c1, s->rc), rcf, err, st, (float*)y,
                                   (float*)(y + fs));
                k += 2;
            } else {
                char* x = slot(k);
                char* y = slot(k + 1);
                e = launch_step_io(s->g, s->p.precision, repro, x, y, x + fs, y + fs, &c0[0], &c0[1], &c0[2], 1,
                                   s->rc, err, st);
                k += 1;
            }
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    if (keep_all) {
        // forward, writing every state straight into its slot
        PRS_TRY(cudaMemcpyAsync(ckpt, s->phi[s->cur], fbytes, cudaMemcpyDeviceToDevice, st));
        PRS_TRY(cudaMemcpyAsync(ckpt + fs, s->dphi, fbytes, cudaMemcpyDeviceToDevice, st));
        PRS_TRY(fill([&](int64_t k) { return ckpt + 2 * fs * (size_t)k; }, n0, 0, nsteps));
        char* last = ckpt + 2 * fs * (size_t)nsteps;
        PRS_TRY(cudaMemcpyAsync(s->phi[s->cur], last, fbytes, cudaMemcpyDeviceToDevice, st));
        PRS_TRY(cudaMemcpyAsync(s->dphi, last + fs, fbytes, cudaMemcpyDeviceToDevice, st));
        s->n += nsteps;
    } else {
        // forward, keeping a checkpoint at the start of every segment
        for (int64_t i = 0; i < nseg; ++i) {
            PRS_TRY(cudaMemcpyAsync(state(0, i), s->phi[s->cur], fbytes, cudaMemcpyDeviceToDevice, st));
            PRS_TRY(cudaMemcpyAsync(state(0, i) + fs, s->dphi, fbytes, cudaMemcpyDeviceToDevice, st));
            const int64_t len = (i + 1) * K <= nsteps ? K : nsteps - i * K;
            int rc = prs_step(s, len);
            if (rc) return rc;
        }
    }
    // J and dJ/dphi at the end; lt = lv + deta lphi = deta dJ/dphi there (lv = 0)
    PRS_TRY(launch_observable(s, s->phi[s->cur], lphi, lt[0], observable, eps_smooth, scr));
    PRS_TRY(cudaMemcpyAsync(s->h_status, s->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    PRS_TRY(cudaEventRecord(s->adj_ev[1], st));
    int cur = 0;
    for (int64_t i = nseg - 1; i >= 0; --i) {
        const int64_t a = n0 + i * K;
        const int64_t len = (i + 1) * K <= nsteps ? K : nsteps - i * K;
        PRS_TRY(cudaEventRecord(s->adj_ev[2 + 2 * (size_t)(nseg - 1 - i)], st));
        if (!keep_all)  // recompute states a+1 .. a+len-1
            PRS_TRY(fill([&](int64_t k) { return state(k, i); }, a, 0, len - 1));
        PRS_TRY(cudaEventRecord(s->adj_ev[3 + 2 * (size_t)(nseg - 1 - i)], st));
        for (int64_t k = len - 1; k >= 0; --k) {
            double c[5];
            step_coefficients(s->p, a + k, c);
            const double opd = 1.0 + c[3];
            AdjCoef ac{c[0], c[1], c[2], -2.0 / (opd * opd) * c[4], -s->p.deta / (opd * opd) * c[4]};
            DiagScratch sk = scr;
            sk.result = dacc + (a + k - n0);
            PRS_TRY(launch_adjoint_step(s, state(k, i), state(k, i) + fs, lt[cur], lphi, lt[1 - cur], ac,
                                        a + k == n0, sk, err));
            cur = 1 - cur;
        }
    }
    PRS_TRY(cudaEventRecord(s->adj_ev[nev - 1], st));
    if (d_dJ_dphi_init) PRS_TRY(cudaMemcpyAsync(d_dJ_dphi_init, lphi, fbytes, cudaMemcpyDeviceToDevice, st));
    if (d_dJ_dv_init) {
        if (nsteps > 0)
            PRS_TRY(cudaMemcpyAsync(d_dJ_dv_init, lt[cur], fbytes, cudaMemcpyDeviceToDevice, st));
        else
            PRS_TRY(cudaMemsetAsync(d_dJ_dv_init, 0, fbytes, st));
    }
    if (nsteps > 0)
        PRS_TRY(cudaMemcpyAsync(hacc.data(), dacc, sizeof(DiagAcc) * (size_t)nsteps, cudaMemcpyDeviceToHost, st));
    PRS_TRY(cudaStreamSynchronize(st));
    const double Jv = s->h_status->result.sum_w;
    // the bounded waits of the step kernels report through the error word
    PRS_TRY(cudaMemcpyAsync(&s->h_status->error, &s->d_status->error, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                            st));
    PRS_TRY(cudaStreamSynchronize(st));
    {
        float f = 0.0f;
        double t[3] = {0.0, 0.0, 0.0};
        PRS_TRY(cudaEventElapsedTime(&f, s->adj_ev[0], s->adj_ev[1]));
        t[0] = f;
        for (int64_t r = 0; r < nseg; ++r) {
            PRS_TRY(cudaEventElapsedTime(&f, s->adj_ev[2 + 2 * r], s->adj_ev[3 + 2 * r]));
            t[1] += f;
            PRS_TRY(cudaEventElapsedTime(&f, s->adj_ev[3 + 2 * r], s->adj_ev[r + 1 < nseg ? 4 + 2 * r : nev - 1]));
            t[2] += f;
        }
        for (int q = 0; q < 3; ++q) s->adj_ms[q] = t[q];
        s->adj_timed = true;
    }
#undef PRS_TRY
    int rc = check_device_error(s);
    if (rc) return rc;
    double da = 0.0;
    for (int64_t k = 0; k < nsteps; ++k) da += hacc[(size_t)k].sum_w;  // fixed order: step index
    if (J) *J = Jv;
    if (dJ_dalpha) *dJ_dalpha = da;
    return PRS_OK;
}

extern "C" int prs_adjoint_timing(prs_sim* s, double ms[3])
{
    if (!s || !ms) return PRS_EINVAL;
    if (!s->adj_timed) return PRS_ESTATE;
    for (int q = 0; q < 3; ++q) ms[q] = s->adj_ms[q];
    return PRS_OK;
}

extern "C" int prs_observable(prs_sim* s, int observable, double eps_smooth, double* J)
{
    return debug_after(s, prs_observable_impl(s, observable, eps_smooth, J), "prs_observable", false);
}

extern "C" int prs_adjoint(prs_sim* s, int64_t nsteps, int observable, double eps_smooth, int64_t ckpt_every,
                           double* J, double* dJ_dalpha, void* d_dJ_dphi_init, void* d_dJ_dv_init)
{
    const int rc =
        prs_adjoint_impl(s, nsteps, observable, eps_smooth, ckpt_every, J, dJ_dalpha, d_dJ_dphi_init, d_dJ_dv_init);
    return debug_after(s, rc, "prs_adjoint", true);
}

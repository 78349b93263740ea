// prs_generic.cu -- initial conditions, the any-shape leapfrog step and the fused
// wall diagnostics with their FP64 reduction.
//
//   init     : SplitMix64 random field (Sec. III initial conditions), dphi = 0
//   step     : Eqs. 3-5 with the damping of Eq. 6, one thread per site, any box
//              side >= 3 (used for sides that are not a multiple of 4, for FP64 and
//              for the ragged cases the fast kernels do not take)
//   measure  : Eq. 7 (link sign-change area) and Eq. 8 (wall-weighted velocity)
//              in one pass, warp-shuffle + block reduction into per-block FP64
//              partials, then a fixed-order final reduction by the last block.
#include <cuda_runtime.h>

#include "prs_arith.cuh"
#include "prs_internal.h"
#include "prs_reduce.cuh"

namespace prs {

// ------------------------------------------------------------ initial field

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t idx)
{
    // Output number idx of SplitMix64 started at state `seed` (Steele, Lea & Flood 2014).
    uint64_t z = seed + (idx + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename R>
__global__ void k_init_random(R* __restrict__ phi, R* __restrict__ dphi, int64_t S, uint64_t seed, bool zero_dphi)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = splitmix64_at(seed, (uint64_t)s) >> 40;  // top 24 bits
        // (2k+1) 2^-24 - 1 is exact in both float and double
        double u = (double)(2ull * k + 1ull) * (1.0 / 16777216.0) - 1.0;
        phi[s] = (R)u;
        if (zero_dphi) dphi[s] = (R)0;
    }
}

static int grid_for(int64_t work, int block)
{
    int64_t b = (work + block - 1) / block;
    const int64_t cap = 152 * 64;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

cudaError_t launch_init_random(const Geo& g, int precision, uint64_t seed, void* phi, void* dphi, bool zero_dphi,
                               cudaStream_t st)
{
    const int block = 256;
    int grid = grid_for(g.S, block);
    if (precision == PRS_FP32)
        k_init_random<float><<<grid, block, 0, st>>>((float*)phi, (float*)dphi, g.S, seed, zero_dphi);
    else
        k_init_random<double><<<grid, block, 0, st>>>((double*)phi, (double*)dphi, g.S, seed, zero_dphi);
    return cudaGetLastError();
}

// Grid of the row-wise kernels: up to four x blocks per row, y blocks striding over the
// rows, at most cap blocks in all.
static dim3 rows_grid(const Geo& g, int cap)
{
    const int gx = (g.nx + 255) / 256 < 4 ? (g.nx + 255) / 256 : 4;
    int64_t gy = cap / gx;
    const int64_t rows = (int64_t)g.ny * g.nz;
    if (gy > rows) gy = rows;
    if (gy < 1) gy = 1;
    return dim3((unsigned)gx, (unsigned)gy, 1);
}

// --------------------------------------------------------- generic step

// One site of Eqs. 3-5 in the canonical evaluation order:
//   s2 = (x+ + x-) ; s2 += (y+ + y-) ; [s2 += (z+ + z-)]
//   lap = (s2 - 2D c) / dx^2 ; f = (cV c)(c c / phi0^2 - 1)
//   v' = c1 v + c2 (lap - f) ; phi' = c + deta v'
template <typename R, bool REPRO, int D>
__device__ __forceinline__ void site_update(R c, R xp, R xm, R yp, R ym, R zp, R zm, R& v, R& phi_new,
                                            const StepCoef<R>& k, const RunConst<R>& rc)
{
    using A = Arith<R, REPRO>;
    R s2 = A::add(xp, xm);
    s2 = A::add(s2, A::add(yp, ym));
    if (D == 3) s2 = A::add(s2, A::add(zp, zm));
    R lap = A::mul(A::sub(s2, A::mul(rc.twoD, c)), rc.inv_dx2);
    R f = A::mul(A::mul(k.cV, c), A::sub(A::mul(A::mul(c, c), rc.inv_phi0sq), (R)1));
    R vn = A::add(A::mul(k.c1, v), A::mul(k.c2, A::sub(lap, f)));
    v = vn;
    phi_new = A::add(c, A::mul(rc.deta, vn));
}

// The same step with the step's constants folded on the host (FP64 without PRS_REPRO):
//   v' = c1 v + g s2 + c (k1 - k2 c^2),  g = c2/dx^2, k1 = c2 cV - 2D g, k2 = c2 cV/phi0^2,
// which is Eq. 4 rearranged: 11 double operations a site instead of 15.  GB300 issues FP64
// at a small fraction of its FP32 rate and the generic step is bound by that rate, so the
// operation count sets its speed.  Every term is odd in phi, so Z2 symmetry stays exact.
template <int D>
__device__ __forceinline__ void site_update_folded(double c, double xp, double xm, double yp, double ym, double zp,
                                                   double zm, double& v, double& phi_new, const KickD& k, double deta)
{
    double s2 = xp + xm;
    s2 = s2 + (yp + ym);
    if (D == 3) s2 = s2 + (zp + zm);
    const double u = c * fma(-k.k2, c * c, k.k1);
    const double vn = fma(k.c1, v, fma(k.g, s2, u));
    v = vn;
    phi_new = fma(deta, vn, c);
}

template <typename R, bool REPRO, int D>
__global__ void k_step_generic(const R* __restrict__ phi, R* __restrict__ phi_out, const R* dphi, R* dphi_out,
                               Geo g, StepCoef<R> k, RunConst<R> rc, KickD kd)
{
    const int64_t nx = g.nx, ny = g.ny, nz = g.nz;
    const int64_t plane = nx * ny;
    // rows of x: y blocks stride over the rows (y, z decoded once per row), x threads over a row
    for (int64_t r = blockIdx.y; r < ny * nz; r += gridDim.y) {
        const int64_t y = r % ny, z = r / ny;
        const int64_t row = r * nx;
        const int64_t ypo = ((y + 1 == ny ? 0 : y + 1) - y) * nx, ymo = ((y == 0 ? ny - 1 : y - 1) - y) * nx;
        const int64_t zpo = ((z + 1 == nz ? 0 : z + 1) - z) * plane, zmo = ((z == 0 ? nz - 1 : z - 1) - z) * plane;
        for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nx; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = row + x;
        R c = phi[s];
        R xp = phi[row + (x + 1 == nx ? 0 : x + 1)];
        R xm = phi[row + (x == 0 ? nx - 1 : x - 1)];
        R yp = phi[s + ypo];
        R ym = phi[s + ymo];
        R zp = (R)0, zm = (R)0;
        if (D == 3) {
            zp = phi[s + zpo];
            zm = phi[s + zmo];
        }
        R v = dphi[s];
        R pn;
        if constexpr (sizeof(R) == 8 && !REPRO)
            site_update_folded<D>(c, xp, xm, yp, ym, zp, zm, v, pn, kd, rc.deta);
        else
            site_update<R, REPRO, D>(c, xp, xm, yp, ym, zp, zm, v, pn, k, rc);
        dphi_out[s] = v;
        phi_out[s] = pn;
        }
    }
}

template <typename R>
static RunConst<R> make_rc(const double rcd[6])
{
    return RunConst<R>{(R)rcd[0], (R)rcd[1], (R)rcd[2], (R)rcd[3], (R)rcd[4], (R)rcd[5]};
}

template <typename R, bool REPRO>
static cudaError_t step_generic_t(const Geo& g, const void* in, void* out, const void* dphi, void* dphi_out, double c1,
                                  double c2, double cV, const double rcd[6], cudaStream_t st)
{
    const int block = 256;
    const dim3 grid = rows_grid(g, 152 * 16);
    StepCoef<R> k{(R)c1, (R)c2, (R)cV};
    RunConst<R> rc = make_rc<R>(rcd);
    const double gq = c2 * rcd[1], h = c2 * cV;  // the folded kick (double): g, k1, k2
    const KickD kd{c1, gq, h - rcd[3] * gq, h * rcd[2]};
    if (g.dims == 3)
        k_step_generic<R, REPRO, 3><<<grid, block, 0, st>>>((const R*)in, (R*)out, (const R*)dphi, (R*)dphi_out, g, k,
                                                             rc, kd);
    else
        k_step_generic<R, REPRO, 2><<<grid, block, 0, st>>>((const R*)in, (R*)out, (const R*)dphi, (R*)dphi_out, g, k,
                                                             rc, kd);
    return cudaGetLastError();
}

cudaError_t launch_step_generic(const Geo& g, int precision, bool repro, const void* in, void* out, const void* dphi,
                                void* dphi_out, double c1, double c2, double cV, const double rcd[6], cudaStream_t st)
{
    if (precision == PRS_FP32) return step_generic_t<float, false>(g, in, out, dphi, dphi_out, c1, c2, cV, rcd, st);
    if (repro) return step_generic_t<double, true>(g, in, out, dphi, dphi_out, c1, c2, cV, rcd, st);
    return step_generic_t<double, false>(g, in, out, dphi, dphi_out, c1, c2, cV, rcd, st);
}

// ------------------------------------------------------------ diagnostics

template <typename R>
__device__ __forceinline__ R fetch(const R* __restrict__ phi, const Geo& g, int64_t x, int64_t y, int64_t z)
{
    x = x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
    y = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
    z = z < 0 ? z + g.nz : (z >= g.nz ? z - g.nz : z);
    return phi[x + (int64_t)g.nx * (y + (int64_t)g.ny * z)];
}

// Eq. 7 weight of the link from site (x,y,z) to its +1 neighbour along axis d:
// |g| / sum_i |g_i|, with g_d the one-sided difference along the link and the
// transverse components the centred differences averaged over the two ends.
template <typename R, int D>
__device__ R link_weight(const R* __restrict__ phi, const Geo& g, int64_t x, int64_t y, int64_t z, int d, R ps, R pt)
{
    using A = Arith<R, true>;
    int64_t tx = x + (d == 0), ty = y + (d == 1), tz = z + (d == 2);
    R num = (R)0, den = (R)0;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        R gg;
        if (e == d) {
            gg = A::sub(pt, ps);
        } else {
            int ex = (e == 0), ey = (e == 1), ez = (e == 2);
            R gs = A::sub(fetch(phi, g, x + ex, y + ey, z + ez), fetch(phi, g, x - ex, y - ey, z - ez));
            R gt = A::sub(fetch(phi, g, tx + ex, ty + ey, tz + ez), fetch(phi, g, tx - ex, ty - ey, tz - ez));
            gg = A::mul((R)0.25, A::add(gs, gt));
        }
        num = A::add(num, A::mul(gg, gg));
        den = A::add(den, fabs(gg));
    }
    // den > 0 (the link's own component is non-zero); if the squares underflow,
    // rescale the components by den first
    const R tiny = sizeof(R) == 4 ? (R)1e-30 : (R)1e-290;
    if (!(num >= tiny)) {
        R n2 = (R)0;
#pragma unroll
        for (int e = 0; e < D; ++e) {
            R gg;
            if (e == d) {
                gg = A::sub(pt, ps);
            } else {
                int ex = (e == 0), ey = (e == 1), ez = (e == 2);
                R gs = A::sub(fetch(phi, g, x + ex, y + ey, z + ez), fetch(phi, g, x - ex, y - ey, z - ez));
                R gt = A::sub(fetch(phi, g, tx + ex, ty + ey, tz + ez), fetch(phi, g, tx - ex, ty - ey, tz - ez));
                gg = A::mul((R)0.25, A::add(gs, gt));
            }
            const R r = A::div(gg, den);
            n2 = A::add(n2, A::mul(r, r));
        }
        return A::sqrt(n2);
    }
    return A::div(A::sqrt(num), den);
}

template <typename R, int D>
__global__ void __launch_bounds__(256) k_measure(const R* __restrict__ phi, const R* __restrict__ dphi, Geo g,
                                                 RunConst<R> rc, DiagScratch scr)
{
    using A = Arith<R, true>;
    DiagAcc a{0.0, 0.0, 0, 0, 0, 0};
    const int64_t rows = (int64_t)g.ny * g.nz;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const int64_t y = row % g.ny, z = row / g.ny;  // once per row
        for (int64_t x = blockIdx.x * blockDim.x + threadIdx.x; x < g.nx; x += gridDim.x * blockDim.x) {
            const int64_t s = row * g.nx + x;
            R ps = phi[s];
            R vs = dphi[s];
            bool neg = ps < (R)0;
            if (!isfinite(ps) || !isfinite(vs)) a.n_nonfinite++;
            bool wall = false;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                int ex = (d == 0), ey = (d == 1), ez = (d == 2);
                R pt = fetch(phi, g, x + ex, y + ey, z + ez);
                R pm = fetch(phi, g, x - ex, y - ey, z - ez);
                if ((pt < (R)0) != neg) {
                    a.n_links++;
                    a.sum_w += (double)link_weight<R, D>(phi, g, x, y, z, d, ps, pt);
                    wall = true;
                }
                if ((pm < (R)0) != neg) wall = true;
            }
            if (wall) {
                a.n_wall++;
                // u = phi^2/phi0^2 - 1.  FP64 keeps the order of Eq. 1; FP32 factors it as
                // (phi - phi0)(phi + phi0)/phi0^2, equal in exact arithmetic and free of
                // the cancellation of phi^2 - 1 next to the vacua.
                R u;
                if (sizeof(R) == 8)
                    u = A::sub(A::mul(A::mul(ps, ps), rc.inv_phi0sq), (R)1);
                else
                    u = A::mul(A::mul(A::sub(ps, rc.phi0), A::add(ps, rc.phi0)), rc.inv_phi0sq);
                R V = A::mul(A::mul(rc.V0, u), u);
                if (V > (R)0)
                    a.sum_ratio += (double)A::div(A::mul(vs, vs), V);
                else
                    a.n_vzero++;
            }
        }
    }
    block_reduce_and_finish(a, scr);
}

template <typename R>
static cudaError_t measure_t(const Geo& g, const void* phi, const void* dphi, const double rcd[6],
                             const DiagScratch& scr, cudaStream_t st)
{
    const dim3 grid = rows_grid(g, scr.max_blocks < 152 * 8 ? scr.max_blocks : 152 * 8);  // one partial per block
    RunConst<R> rc = make_rc<R>(rcd);
    if (g.dims == 3)
        k_measure<R, 3><<<grid, 256, 0, st>>>((const R*)phi, (const R*)dphi, g, rc, scr);
    else
        k_measure<R, 2><<<grid, 256, 0, st>>>((const R*)phi, (const R*)dphi, g, rc, scr);
    return cudaGetLastError();
}

cudaError_t launch_measure(const Geo& g, int precision, const void* phi, const void* dphi, const double rcd[6],
                           const DiagScratch& scr, cudaStream_t st)
{
    if (precision == PRS_FP32) return measure_t<float>(g, phi, dphi, rcd, scr, st);
    return measure_t<double>(g, phi, dphi, rcd, scr, st);
}

}  // namespace prs

namespace prs {

// The same diagnostic kernel on a caller-chosen grid (one partial slot per block in scr).
template <typename R>
static cudaError_t measure_grid_t(const Geo& g, const void* phi, const void* dphi, const double rcd[6],
                                  const DiagScratch& scr, int grid, cudaStream_t st)
{
    RunConst<R> rc = make_rc<R>(rcd);
    const dim3 g2(1, (unsigned)grid, 1);  // grid blocks striding over the rows
    if (g.dims == 3)
        k_measure<R, 3><<<g2, 256, 0, st>>>((const R*)phi, (const R*)dphi, g, rc, scr);
    else
        k_measure<R, 2><<<g2, 256, 0, st>>>((const R*)phi, (const R*)dphi, g, rc, scr);
    return cudaGetLastError();
}

cudaError_t launch_measure_on_grid(const Geo& g, int precision, const void* phi, const void* dphi,
                                   const double rcd[6], const DiagScratch& scr, int grid, cudaStream_t st)
{
    if (grid < 1 || grid > scr.max_blocks || grid > 65535) return cudaErrorInvalidValue;  // gridDim.y limit
    if (precision == PRS_FP32) return measure_grid_t<float>(g, phi, dphi, rcd, scr, grid, st);
    return measure_grid_t<double>(g, phi, dphi, rcd, scr, grid, st);
}

}  // namespace prs

// prs_tblock.cu -- two leapfrog steps (Eqs. 3-5) per pass over HBM, FP32 3D and 2D.
//
// One pass reads phi^n, dphi^{n-1/2} once and writes phi^{n+2}, dphi^{n+3/2} once:
// 16 bytes per two site-updates.  A CTA owns ty whole x-rows of y and a chunk of
// z-planes and marches along z through two levels:
//   level 1 (step n)   on ty+2 rows, from level-0 planes staged by the TMA engine
//                       (cp.async.bulk) in a 4-slot ring of ty+4 rows;
//   level 2 (step n+1) on the ty output rows, from level-1 planes kept in a second
//                       4-slot ring, two planes behind level 1, so each plane needs
//                       one barrier.
// dphi enters level 1 on ty+2 rows (its halo rows belong to neighbouring tiles), so
// it is read from one buffer and written to another; the level-1 dphi stays in the
// registers of the thread that owns its site until level 2 uses it.  The extra
// level-1 rows (2 per ty) are recomputed by both tiles that need them.
#include <cuda_runtime.h>

#include "prs_internal.h"
#include "prs_ptx.cuh"
#include "prs_tile.cuh"

namespace prs {

namespace {

constexpr int kTbThreads = 512;
constexpr int kTbItems = 3;  // float4 per thread per level-1 plane, at most

template <int ITEMS>
__global__ void __launch_bounds__(kTbThreads, 1)
    k_step3d_t2(const float* __restrict__ phi_in, float* __restrict__ phi_out, const float* __restrict__ v_in,
                float* __restrict__ v_out, int nx, int ny, int nz, int ty, int cz, StepCoef<float> k0,
                StepCoef<float> k1, RunConst<float> rc, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    const int r1 = ty + 2, r0 = ty + 4;       // rows of a level-1 and a level-0 plane tile
    const int t0 = r0 * nx, t1 = r1 * nx;      // floats per ring slot
    float* ring0 = reinterpret_cast<float*>(smem_raw + 128);
    float* ring1 = ring0 + 4 * t0;
    const int tid = threadIdx.x, lane = tid & 31;
    const int ytiles = ny / ty;
    const int y0 = (blockIdx.x % ytiles) * ty;
    const int z0 = (blockIdx.x / ytiles) * cz;
    const int zn = min(cz, nz - z0);
    const int nq = nx >> 2;
    const int total = r1 * nq;  // level-1 float4 items of a plane
    const size_t plane = (size_t)nx * ny;

    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto wy = [&](int y) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); };
    auto wz = [&](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };
    const unsigned rowb = (unsigned)nx * 4u;
    const int nload = zn + 4;  // level-0 local planes 0..zn+3 = global z0-2 .. z0+zn+1
    auto issue = [&](int i) {
        const float* src = phi_in + (size_t)wz(z0 - 2 + i) * plane;
        float* dst = ring0 + (i & 3) * t0;
        uint64_t* b = &bar[i & 3];
        mbar_arrive_expect_tx(b, rowb * (unsigned)r0);
        bulk_g2s(dst, src + (size_t)wy(y0 - 2) * nx, rowb, b);
        bulk_g2s(dst + nx, src + (size_t)wy(y0 - 1) * nx, rowb, b);
        bulk_g2s(dst + 2 * nx, src + (size_t)y0 * nx, rowb * (unsigned)ty, b);
        bulk_g2s(dst + (size_t)(ty + 2) * nx, src + (size_t)wy(y0 + ty) * nx, rowb, b);
        bulk_g2s(dst + (size_t)(ty + 3) * nx, src + (size_t)wy(y0 + ty + 1) * nx, rowb, b);
    };
    int issued = -1;
    if (tid == 0) issue(0), issued = 0;

    int row[ITEMS], col[ITEMS];
    bool on[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int q = tid + kTbThreads * j;
        on[j] = q < total;  // whole warps: nq and the block size are multiples of 32
        row[j] = on[j] ? q / nq : 0;
        col[j] = on[j] ? q - row[j] * nq : 0;
    }
    // dphi^{n-1/2} of the level-1 sites: the plane used now and the one loaded ahead
    float4 va[ITEMS], vb[ITEMS];
    // level-1 dphi^{n+1/2} of this thread's sites for the last three level-1 planes
    float4 w0[ITEMS], w1[ITEMS], w2[ITEMS];
    auto load_v = [&](int jl, float4* dst) {  // level-0 local plane jl, level-1 rows
        const float* vp = v_in + (size_t)wz(z0 - 2 + jl) * plane;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j)
            if (on[j]) dst[j] = ldg_stream4(vp + (size_t)wy(y0 - 1 + row[j]) * nx + 4 * col[j]);
    };

    for (int i = 0; i <= zn + 4; ++i) {
        bool ok = true;
        if (i < nload) ok = mbar_wait(&bar[i & 3], (i >> 2) & 1, err);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain(bar, i, issued, err);
            return;
        }
        if (tid == 0 && i + 1 < nload) issue(i + 1), issued = i + 1;
        const int j1 = i - 1;  // level-1 plane of this iteration
        const int k2 = i - 3;  // level-2 plane of this iteration
        const bool next_v = i >= 1 && i <= zn + 2;  // dphi of the next level-1 plane, one iteration ahead
        if (next_v) load_v(i, vb);
        if (j1 >= 1 && j1 <= zn + 2) {
            const float* pm = ring0 + ((j1 - 1) & 3) * t0;
            const float* pc = ring0 + (j1 & 3) * t0;
            const float* pp = ring0 + ((j1 + 1) & 3) * t0;
            float* l1 = ring1 + (j1 & 3) * t1;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if (!on[j]) continue;
                const int off = (row[j] + 1) * nx + 4 * col[j];  // level-0 row of this level-1 site
                const float4 c = lds4(pc + off);
                float left, right;
                x_halo(pc + (row[j] + 1) * nx, col[j], nq, nx, lane, c, left, right);
                float4 pn;
                float4 vv = va[j];
                update4(c, left, right, lds4(pc + off + nx), lds4(pc + off - nx), lds4(pp + off), lds4(pm + off), vv,
                        pn, k0, rc, true);
                *reinterpret_cast<float4*>(l1 + row[j] * nx + 4 * col[j]) = pn;
                w2[j] = vv;
            }
        }
        if (k2 >= 2 && k2 <= zn + 1) {
            const float* pm = ring1 + ((k2 - 1) & 3) * t1;
            const float* pc = ring1 + (k2 & 3) * t1;
            const float* pp = ring1 + ((k2 + 1) & 3) * t1;
            const size_t zo = (size_t)(z0 - 2 + k2) * plane;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if (!on[j] || row[j] < 1 || row[j] > ty) continue;  // warp-uniform: one row per warp
                const int off = row[j] * nx + 4 * col[j];
                const float4 c = lds4(pc + off);
                float left, right;
                x_halo(pc + row[j] * nx, col[j], nq, nx, lane, c, left, right);
                float4 pn;
                float4 vv = w0[j];
                update4(c, left, right, lds4(pc + off + nx), lds4(pc + off - nx), lds4(pp + off), lds4(pm + off), vv,
                        pn, k1, rc, true);
                const size_t go = zo + (size_t)(y0 + row[j] - 1) * nx + 4 * col[j];
                stg4(phi_out + go, pn);
                stg4(v_out + go, vv);
            }
        }
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            w0[j] = w1[j];
            w1[j] = w2[j];
            if (next_v) va[j] = vb[j];
        }
    }
}

// 2D: a CTA owns the rows [y0, y0+yn) of a chunk and marches along y through the same
// two levels on whole rows (x neighbours by shuffle, the periodic wrap by lanes 0/31):
//   level 1 (step n)   on rows y0-1 .. y0+yn, from level-0 rows y0-2 .. y0+yn+1 that the
//                       TMA engine stages in a ring of kR2Slots0 rows;
//   level 2 (step n+1) on rows y0 .. y0+yn-1, from level-1 rows kept in a ring of
//                       kR2Slots1 rows.
// Iteration t runs level 1 on local rows 2t-1, 2t and level 2 on rows 2t-4, 2t-3, whose
// level-1 rows (up to 2t-2) were written an iteration earlier: one barrier per two rows.
// y is the marching direction, so the only recomputed level-1 rows are the two outside
// the chunk.  As in 3D, dphi enters those rows from the neighbouring chunks, so it is read
// from one buffer and written to another; the level-1 dphi stays in the registers of the
// thread that owns its columns.
constexpr int kTb2Threads = 512;
constexpr int kR2Ahead = 1;                   // iterations of level-0 rows in flight
constexpr int kR2Slots0 = 4 + 2 * kR2Ahead;  // level-0 ring rows
constexpr int kR2Slots1 = 6;                 // level-1 ring rows

static __device__ __noinline__ void drain_rows(uint64_t* bar, int from, int issued, unsigned int* err)
{
    for (int i = from; i <= issued; ++i) mbar_wait(&bar[i % kR2Slots0], (i / kR2Slots0) & 1, err);
}

template <int ITEMS>
__global__ void __launch_bounds__(kTb2Threads, 1)
    k_step2d_t2(const float* __restrict__ phi_in, float* __restrict__ phi_out, const float* __restrict__ v_in,
                  float* __restrict__ v_out, int nx, int ny, int cy, StepCoef<float> k0, StepCoef<float> k1,
                  RunConst<float> rc, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    float* ring0 = reinterpret_cast<float*>(smem_raw + 128);
    float* ring1 = ring0 + kR2Slots0 * nx;
    const int tid = threadIdx.x, lane = tid & 31;
    const int y0 = blockIdx.x * cy;
    const int yn = min(cy, ny - y0);
    const int nq = nx >> 2;

    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < kR2Slots0; ++i) mbar_init(&bar[i], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto wy = [&](int y) {
        while (y < 0) y += ny;
        while (y >= ny) y -= ny;
        return y;
    };
    const unsigned rowb = (unsigned)nx * 4u;
    const int nload = yn + 4;  // level-0 local rows 0..yn+3 = global y0-2 .. y0+yn+1
    auto issue = [&](int i) {  // level-0 local row i
        uint64_t* b = &bar[i % kR2Slots0];
        mbar_arrive_expect_tx(b, rowb);
        bulk_g2s(ring0 + (i % kR2Slots0) * nx, phi_in + (size_t)wy(y0 - 2 + i) * nx, rowb, b);
    };
    // iteration t waits for rows 2t, 2t+1 and issues the two rows iteration t + kR2Ahead waits for
    int issued = -1;
    if (tid == 0)
        for (int i = 0; i < 2 * kR2Ahead && i < nload; ++i) issue(i), issued = i;

    int col[ITEMS];
    bool on[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int q = tid + kTb2Threads * j;
        on[j] = q < nq;
        col[j] = on[j] ? q : 0;
    }
    // dphi^{n-1/2} of level-1 rows 2t-1, 2t (a: now, b: loaded for the next iteration)
    float4 va0[ITEMS], va1[ITEMS], vb0[ITEMS], vb1[ITEMS];
    // level-1 dphi^{n+1/2}: even rows for two iterations, odd rows for one
    float4 e0[ITEMS], e1[ITEMS], o0[ITEMS];
    auto load_v = [&](int jl, float4* dst) {
        if (jl < 1 || jl > yn + 2) return;
        const float* vp = v_in + (size_t)wy(y0 - 2 + jl) * nx;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j)
            if (on[j]) dst[j] = ldg_stream4(vp + 4 * col[j]);
    };

    auto level1 = [&](int jr, const float4* vin, float4* vout) {
        if (jr < 1 || jr > yn + 2) return;
        const float* pm = ring0 + ((jr - 1) % kR2Slots0) * nx;
        const float* pc = ring0 + (jr % kR2Slots0) * nx;
        const float* pp = ring0 + ((jr + 1) % kR2Slots0) * nx;
        float* l1 = ring1 + (jr % kR2Slots1) * nx;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (!on[j]) continue;
            const float4 c = lds4(pc + 4 * col[j]);
            float left, right;
            x_halo(pc, col[j], nq, nx, lane, c, left, right);
            const float4 ym = lds4(pm + 4 * col[j]);
            float4 pn;
            float4 vv = vin[j];
            update4(c, left, right, lds4(pp + 4 * col[j]), ym, ym, ym, vv, pn, k0, rc, false);
            *reinterpret_cast<float4*>(l1 + 4 * col[j]) = pn;
            vout[j] = vv;
        }
    };
    auto level2 = [&](int kr, const float4* vin) {
        if (kr < 2 || kr > yn + 1) return;
        const float* pm = ring1 + ((kr - 1) % kR2Slots1) * nx;
        const float* pc = ring1 + (kr % kR2Slots1) * nx;
        const float* pp = ring1 + ((kr + 1) % kR2Slots1) * nx;
        const size_t ro = (size_t)(y0 - 2 + kr) * nx;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (!on[j]) continue;
            const float4 c = lds4(pc + 4 * col[j]);
            float left, right;
            x_halo(pc, col[j], nq, nx, lane, c, left, right);
            const float4 ym = lds4(pm + 4 * col[j]);
            float4 pn;
            float4 vv = vin[j];
            update4(c, left, right, lds4(pp + 4 * col[j]), ym, ym, ym, vv, pn, k1, rc, false);
            stg4(phi_out + ro + 4 * col[j], pn);
            stg4(v_out + ro + 4 * col[j], vv);
        }
    };

    const int tmax = (yn + 5) / 2;  // last iteration: level-2 row 2t-3 or 2t-4 reaches yn+1
    for (int t = 0; t <= tmax; ++t) {
        bool ok = true;
        for (int i = 2 * t; i <= 2 * t + 1; ++i)  // rows 2t, 2t+1 (rows below were waited earlier)
            if (i < nload) ok = ok && mbar_wait(&bar[i % kR2Slots0], (i / kR2Slots0) & 1, err);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain_rows(bar, 2 * t, issued, err);
            return;
        }
        // rows 2(t+kR2Ahead) and the next, into the slots of rows 2t-4 and 2t-3 (last read by
        // level 1 at iteration t-1; level 1 now reads rows 2t-2 .. 2t+1)
        if (tid == 0)
            for (int i = 2 * (t + kR2Ahead); i <= 2 * (t + kR2Ahead) + 1 && i < nload; ++i) issue(i), issued = i;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) va0[j] = vb0[j], va1[j] = vb1[j];
        load_v(2 * t + 1, vb0);  // for iteration t+1: rows 2t+1, 2t+2
        load_v(2 * t + 2, vb1);
        float4 no[ITEMS], ne[ITEMS];
        level1(2 * t - 1, va0, no);
        level1(2 * t, va1, ne);
        level2(2 * t - 4, e0);
        level2(2 * t - 3, o0);
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            e0[j] = e1[j];
            e1[j] = ne[j];
            o0[j] = no[j];
        }
    }
}

size_t smem2d_t2(int nx) { return 128 + (kR2Slots0 + kR2Slots1) * (size_t)nx * sizeof(float); }

size_t smem_t2(int nx, int ty) { return 128 + 4 * (size_t)(ty + 4) * nx * 4 + 4 * (size_t)(ty + 2) * nx * 4; }

constexpr size_t kTbSmemMax = 200 * 1024;

// Rows per tile: the largest power of two dividing ny whose rings fit and whose
// level-1 plane has at most kTbItems float4 per thread.
int pick_ty(const Geo& g)
{
    for (int ty = 32; ty >= 1; ty >>= 1) {
        if (g.ny % ty != 0 || ty > g.ny) continue;
        if (smem_t2(g.nx, ty) > kTbSmemMax) continue;
        if ((ty + 2) * (g.nx / 4) > kTbItems * kTbThreads) continue;
        return ty;
    }
    return 0;
}

}  // namespace


bool tblock_ok(const Geo& g, int precision)
{
    if (precision != PRS_FP32 || g.nx % 128 != 0) return false;
    if (g.dims == 2) return g.nx <= 2 * kTb2Threads * 4;  // at most two float4 per thread of a row
    return g.nx <= 1024 && g.nz >= 3 && pick_ty(g) > 0;
}

cudaError_t launch_step_t2(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out,
                           StepCoef<float> k0, StepCoef<float> k1, RunConst<float> rc, unsigned int* err,
                           cudaStream_t st)
{
    if (g.dims == 2) {
        static std::atomic<unsigned long long> attr1{0}, attr2{0};
        const size_t sm = smem2d_t2(g.nx);
        const int sms = sm_count_current();
        const int cy = (g.ny + sms - 1) / sms;
        const int blocks = (g.ny + cy - 1) / cy;
        if (g.nx / 4 > kTb2Threads) {
            const cudaError_t e =
                smem_limit_once(attr2, (const void*)k_step2d_t2<2>, (int)smem2d_t2(8 * kTb2Threads));
            if (e != cudaSuccess) return e;
            k_step2d_t2<2><<<blocks, kTb2Threads, sm, st>>>(phi_in, phi_out, v_in, v_out, g.nx, g.ny, cy, k0, k1,
                                                            rc, err);
        } else {
            const cudaError_t e =
                smem_limit_once(attr1, (const void*)k_step2d_t2<1>, (int)smem2d_t2(4 * kTb2Threads));
            if (e != cudaSuccess) return e;
            k_step2d_t2<1><<<blocks, kTb2Threads, sm, st>>>(phi_in, phi_out, v_in, v_out, g.nx, g.ny, cy, k0, k1,
                                                            rc, err);
        }
        return cudaGetLastError();
    }
    static std::atomic<unsigned long long> attr{0};
    {
        const cudaError_t e = smem_limit_once(attr, (const void*)k_step3d_t2<kTbItems>, (int)kTbSmemMax);
        if (e != cudaSuccess) return e;
    }
    const int ty = pick_ty(g);
    if (ty == 0) return cudaErrorInvalidValue;
    const int sms = sm_count_current();
    const int ytiles = g.ny / ty;
    // z-chunks: whole waves of one CTA per SM, balanced against the four halo planes
    int best = 1;
    double best_score = -1.0;
    for (int nc = 1; nc <= g.nz / 8 || nc == 1; ++nc) {
        const int c = (g.nz + nc - 1) / nc, n = (g.nz + c - 1) / c;
        const long long blocks = (long long)ytiles * n;
        const long long waves = (blocks + sms - 1) / sms;
        const double score = (double)blocks / (double)(waves * sms) * c / (c + 4.0) * (waves >= 2 ? 1.0 : 0.9);
        if (score > best_score + 1e-9) best_score = score, best = n;
        if (nc > 4096) break;
    }
    const int cz = (g.nz + best - 1) / best;
    const int blocks = ytiles * ((g.nz + cz - 1) / cz);
    k_step3d_t2<kTbItems><<<blocks, kTbThreads, smem_t2(g.nx, ty), st>>>(phi_in, phi_out, v_in, v_out, g.nx, g.ny,
                                                                         g.nz, ty, cz, k0, k1, rc, err);
    return cudaGetLastError();
}

}  // namespace prs

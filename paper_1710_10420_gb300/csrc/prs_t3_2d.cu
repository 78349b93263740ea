// prs_t3_2d.cu -- three leapfrog steps (Eqs. 3-5) per pass over HBM, FP32 2D, whole rows.
//
// A CTA owns the rows [y0, y0+yn) of a chunk (one chunk per SM) and marches along y, one row
// per iteration, through three levels on whole rows (x neighbours by warp shuffle, the
// periodic wrap by lanes 0/31):
//   level 1 (step n)   on rows y0-2 .. y0+yn+1, from level-0 rows y0-3 .. y0+yn+2 that the
//                       TMA engine stages into a ring, three rows ahead;
//   level 2 (step n+1) on rows y0-1 .. y0+yn, from the level-1 ring;
//   level 3 (step n+2) on the chunk's rows, from the level-2 ring, to HBM.
// Iteration i runs level 1 on local row i-1, level 2 on row i-3 and level 3 on row i-5: each
// level reads only rows that the level before it wrote in earlier iterations, so one barrier
// per row orders everything.  A thread owns the same columns of every row, so the dphi that
// level 1 hands to level 2 (and level 2 to level 3) stays in its registers, two rows deep.
// Only the rows outside the chunk (four at level 1, two at level 2) are computed twice.
// dphi enters those rows from the neighbouring chunks, so it is read from one buffer and
// written to another.  At one SM per chunk the two-step pass streams its rows at about the
// SM's share of the copy bandwidth, so the third level's gain is the bytes it saves.  One
// launch may also carry up to 16 runs of one box (launch_step_t3_2d_runs), each CTA a chunk
// of one run.
#include <cuda_runtime.h>

#include <atomic>
#include <type_traits>

#include "prs_internal.h"
#include "prs_runs.h"
#include "prs_ptx.cuh"
#include "prs_tile.cuh"

namespace prs {

namespace {

constexpr int kT3Threads = 512;
constexpr int kSlots1 = 4;  // level-1 ring rows: three read by level 2, one written
constexpr int kSlots2 = 4;  // level-2 ring rows: three read by level 3, one written

// A CTA's shape: THREADS threads, AHEAD level-0 rows in flight (the level-0 ring holds three
// read rows and AHEAD in flight), MINB CTAs per SM.  One 512-thread CTA per SM three rows ahead
// serves a run alone; two 256-thread CTAs per SM two rows ahead (13 rows of rings: 104 KB for
// 2048-wide rows) serve runs of up to 2048 columns grouped in one launch, whose chunks are long
// enough for twice as many CTAs, each hiding the other's row latency.
template <int THREADS, int AHEAD>
struct T3Shape {
    static constexpr int kThreads = THREADS, kAhead = AHEAD, kSlots0 = 3 + AHEAD;
    static constexpr int kMinBlocks = THREADS == kT3Threads ? 1 : 2;
};
using T3Alone = T3Shape<kT3Threads, 3>;
using T3Pair = T3Shape<256, 2>;

template <class SH>
size_t smem2d_t3(int nx)
{
    return 128 + (size_t)(SH::kSlots0 + kSlots1 + kSlots2) * nx * sizeof(float);
}

static __device__ __noinline__ void drain_rows3(uint64_t* bar, int from, int issued, int slots, unsigned int* err)
{
    for (int i = from; i <= issued; ++i) mbar_wait(&bar[i % slots], (unsigned)(i / slots) & 1u, err);
}

__device__ __forceinline__ int wrap_row(int y, int ny)
{
    while (y < 0) y += ny;
    while (y >= ny) y -= ny;
    return y;
}

// One level's update of a row from its ring rows below (m), at (c) and above (p): reads x
// neighbours by shuffle; vv is this thread's dphi (updated in place), pn the new phi.
template <int ITEMS>
__device__ __forceinline__ void row_update(const float* m, const float* c, const float* p, const int (&col)[ITEMS],
                                           const bool (&on)[ITEMS], int nq, int nx, int lane, float4 (&vv)[ITEMS],
                                           float4 (&pn)[ITEMS], const KickP& k)
{
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        if (!on[j]) continue;
        const float4 cc = lds4(c + 4 * col[j]);
        float left, right;
        x_halo(c, col[j], nq, nx, lane, cc, left, right);
        const float4 ym = lds4(m + 4 * col[j]);
        update4p<false>(cc, left, right, lds4(p + 4 * col[j]), ym, ym, ym, vv[j], pn[j], k);
    }
}

// The arguments of one run's pass.
struct T3One {
    const float* phi_in;
    float* phi_out;
    const float* v_in;
    float* v_out;
    KickP k[3];
};

// A: T3One (one run: CTA b takes the rows [b cy, (b+1) cy)) or T3Runs2D (several runs of one
// box in one launch: CTA b takes chunk b % bpr of run b / bpr, so that a box whose pass alone
// leaves each SM a short chunk, 2048^2: 14 rows with six of their twenty iterations filling and
// draining the levels, marches long chunks; chunk boundaries do not change the results, the
// rows outside a chunk are recomputed from the same inputs).  NX > 0: the row width as a
// compile-time constant (the 4096-wide production box).  (The body as a device function that
// both kinds of kernel call compiled to 114 instead of 98 registers for NX = 4096, and the
// pass ran 25.2 against 22.5 us per step.)
template <int ITEMS, int NX, class A, class SH = T3Alone>
__global__ void __launch_bounds__(SH::kThreads, SH::kMinBlocks)
    k_step2d_t3(const __grid_constant__ A a, int nx_, int ny, int cy, unsigned int* err)
{
    constexpr int kThreads = SH::kThreads, kAhead = SH::kAhead, kSlots0 = SH::kSlots0;
    constexpr bool kRuns = std::is_same<A, T3Runs2D>::value;
    int run = 0, blk = blockIdx.x;
    if constexpr (kRuns) {
        run = blockIdx.x / a.bpr;
        blk = blockIdx.x - run * a.bpr;
        if (blk * cy >= ny) return;  // the whole CTA, before any barrier
    }
    const float* __restrict__ phi_in;
    float* __restrict__ phi_out;
    const float* __restrict__ v_in;
    float* __restrict__ v_out;
    KickP k0, k1, k2;
    if constexpr (kRuns) {
        phi_in = a.phi_in[run], phi_out = a.phi_out[run], v_in = a.v_in[run], v_out = a.v_out[run];
        k0 = a.k[run][0], k1 = a.k[run][1], k2 = a.k[run][2];
    } else {
        phi_in = a.phi_in, phi_out = a.phi_out, v_in = a.v_in, v_out = a.v_out;
        k0 = a.k[0], k1 = a.k[1], k2 = a.k[2];
    }
    const int nx = NX > 0 ? NX : nx_;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    float* ring0 = reinterpret_cast<float*>(smem_raw + 128);
    float* ring1 = ring0 + kSlots0 * nx;
    float* ring2 = ring1 + kSlots1 * nx;
    const int tid = threadIdx.x, lane = tid & 31;
    const int y0 = blk * cy;
    const int yn = min(cy, ny - y0);
    const int nq = nx >> 2;
    const int nload = yn + 6;  // level-0 local rows 0 .. yn+5 = global y0-3 .. y0+yn+2

    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < kSlots0; ++i) mbar_init(&bar[i], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const unsigned rowb = (unsigned)nx * 4u;
    auto issue = [&](int i) {  // level-0 local row i into slot i mod kSlots0
        uint64_t* b = &bar[i % kSlots0];
        mbar_arrive_expect_tx(b, rowb);
        bulk_g2s(ring0 + (i % kSlots0) * nx, phi_in + (size_t)wrap_row(y0 - 3 + i, ny) * nx, rowb, b);
    };
    // row r may be staged once row r - kSlots0, last read by level 1 at iteration r - kSlots0 + 2,
    // is done with: at iteration r - kAhead
    int issued = -1;
    if (tid == 0)
        for (int i = 0; i < kAhead && i < nload; ++i) issue(i), issued = i;

    int col[ITEMS];
    bool on[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int q = tid + kThreads * j;
        on[j] = q < nq;
        col[j] = on[j] ? q : 0;
    }
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // vn: dphi^{n-1/2} of level-1 row j+1, loaded an iteration ahead; w1a/w1b: level-1 dphi
    // handed down one and two iterations ago; w2a/w2b: the same for level 2
    float4 vn[ITEMS], w1a[ITEMS], w1b[ITEMS], w2a[ITEMS], w2b[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) vn[j] = w1a[j] = w1b[j] = w2a[j] = w2b[j] = z4;
    auto load_v = [&](int jl) {  // dphi of level-1 local row jl (global y0-3+jl)
        if (jl < 1 || jl > yn + 4) return;
        const float* vp = v_in + (size_t)wrap_row(y0 - 3 + jl, ny) * nx;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j)
            if (on[j]) vn[j] = ldg_stream4(vp + 4 * col[j]);
    };
    load_v(1);

    const int iters = yn + 8;  // level 3 reaches local row yn+2 at iteration yn+7
    for (int i = 0; i < iters; ++i) {
        bool ok = true;
        if (i < nload) ok = mbar_wait(&bar[i % kSlots0], (unsigned)(i / kSlots0) & 1u, err);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain_rows3(bar, i, issued, kSlots0, err);
            return;
        }
        if (tid == 0 && i + kAhead < nload) issue(i + kAhead), issued = i + kAhead;
        const int ra = i - 1, rb = i - 3, rc = i - 5;  // local rows of levels 1, 2, 3
        float4 v1[ITEMS], v2[ITEMS];
        const bool do1 = ra >= 1 && ra <= yn + 4, do2 = rb >= 2 && rb <= yn + 3, do3 = rc >= 3 && rc <= yn + 2;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) v1[j] = vn[j];
        load_v(ra + 1);  // for the next iteration
        if (do1) {
            float4 pn[ITEMS];
            row_update(ring0 + ((ra + kSlots0 - 1) % kSlots0) * nx, ring0 + (ra % kSlots0) * nx,
                       ring0 + ((ra + 1) % kSlots0) * nx, col, on, nq, nx, lane, v1, pn, k0);
            float* l1 = ring1 + (ra % kSlots1) * nx;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (on[j]) *reinterpret_cast<float4*>(l1 + 4 * col[j]) = pn[j];
        }
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) v2[j] = w1b[j];
        if (do2) {
            float4 pn[ITEMS];
            row_update(ring1 + ((rb + kSlots1 - 1) % kSlots1) * nx, ring1 + (rb % kSlots1) * nx,
                       ring1 + ((rb + 1) % kSlots1) * nx, col, on, nq, nx, lane, v2, pn, k1);
            float* l2 = ring2 + (rb % kSlots2) * nx;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (on[j]) *reinterpret_cast<float4*>(l2 + 4 * col[j]) = pn[j];
        }
        if (do3) {
            float4 pn[ITEMS], v3[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) v3[j] = w2b[j];
            row_update(ring2 + ((rc + kSlots2 - 1) % kSlots2) * nx, ring2 + (rc % kSlots2) * nx,
                       ring2 + ((rc + 1) % kSlots2) * nx, col, on, nq, nx, lane, v3, pn, k2);
            const size_t ro = (size_t)(y0 - 3 + rc) * nx;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if (!on[j]) continue;
                stg4(phi_out + ro + 4 * col[j], pn[j]);
                stg4(v_out + ro + 4 * col[j], v3[j]);
            }
        }
        // the dphi each level hands down reaches the next level two iterations later
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            w1b[j] = w1a[j];
            w1a[j] = v1[j];
            w2b[j] = w2a[j];
            w2a[j] = v2[j];
        }
    }
}

}  // namespace

// The 2D three-step pass takes FP32 boxes with an x side that is a multiple of 128 up to
// 4096 (at most two float4 per thread of a 512-thread CTA, 14 rows of rings in shared memory).
bool t3_2d_ok(const Geo& g)
{
    return g.dims == 2 && g.nx % 128 == 0 && g.nx <= 2 * kT3Threads * 4 && g.ny >= 3;
}

// One launch of the pass for `a` (T3One or T3Runs2D) over `blocks` CTAs of cy rows.
template <class A>
static cudaError_t launch_t3_2d(const Geo& g, const A& a, int blocks, int cy, unsigned int* err, cudaStream_t st)
{
    static std::atomic<unsigned long long> attr1{0}, attr2{0}, attr4{0};
    const size_t sm = smem2d_t3<T3Alone>(g.nx);
    cudaError_t e;
    if (g.nx / 4 > kT3Threads) {
        e = smem_limit_once(attr2, (const void*)k_step2d_t3<2, 0, A>, (int)smem2d_t3<T3Alone>(8 * kT3Threads));
        if (e == cudaSuccess)
            e = smem_limit_once(attr4, (const void*)k_step2d_t3<2, 4096, A>, (int)smem2d_t3<T3Alone>(4096));
        if (e != cudaSuccess) return e;
        if (g.nx == 4096)
            k_step2d_t3<2, 4096, A><<<blocks, kT3Threads, sm, st>>>(a, g.nx, g.ny, cy, err);
        else
            k_step2d_t3<2, 0, A><<<blocks, kT3Threads, sm, st>>>(a, g.nx, g.ny, cy, err);
    } else {
        e = smem_limit_once(attr1, (const void*)k_step2d_t3<1, 0, A>, (int)smem2d_t3<T3Alone>(4 * kT3Threads));
        if (e != cudaSuccess) return e;
        k_step2d_t3<1, 0, A><<<blocks, kT3Threads, sm, st>>>(a, g.nx, g.ny, cy, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_step_t3_2d(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out,
                              KickF k0, KickF k1, KickF k2, RunConst<float> rc, unsigned int* err, cudaStream_t st)
{
    if (!t3_2d_ok(g)) return cudaErrorNotSupported;
    const T3One a{phi_in, phi_out, v_in, v_out,
                  {kick_packed(k0, rc.deta), kick_packed(k1, rc.deta), kick_packed(k2, rc.deta)}};
    const int sms = sm_count_current();
    const int cy = (g.ny + sms - 1) / sms;
    return launch_t3_2d(g, a, (g.ny + cy - 1) / cy, cy, err, st);
}

cudaError_t launch_step_t3_2d_runs(const Geo& g, int nruns, const float* const* phi_in, float* const* phi_out,
                                   const float* const* v_in, float* const* v_out, const KickF* k,
                                   const RunConst<float>* rc, unsigned int* err, cudaStream_t st)
{
    if (!t3_2d_ok(g) || nruns < 1 || nruns > kT3MaxRuns) return cudaErrorNotSupported;
    T3Runs2D R{};
    for (int r = 0; r < nruns; ++r) {
        R.phi_in[r] = phi_in[r];
        R.phi_out[r] = phi_out[r];
        R.v_in[r] = v_in[r];
        R.v_out[r] = v_out[r];
        for (int l = 0; l < 3; ++l) R.k[r][l] = kick_packed(k[3 * r + l], rc[r].deta);
    }
    const int sms = sm_count_current();
    if (g.nx > 8 * T3Pair::kThreads) {  // 4096-wide rows: one 512-thread CTA per SM
        R.bpr = sms / nruns > 0 ? sms / nruns : 1;
        const int cy = (g.ny + R.bpr - 1) / R.bpr;
        return launch_t3_2d(g, R, R.bpr * nruns, cy, err, st);
    }
    // up to 2048 columns: 256-thread CTAs, two per SM; the runs' chunks fill the CTA slots once
    const void* fn = g.nx > 4 * T3Pair::kThreads ? (const void*)k_step2d_t3<2, 0, T3Runs2D, T3Pair>
                                                 : (const void*)k_step2d_t3<1, 0, T3Runs2D, T3Pair>;
    static std::atomic<unsigned long long> attr_p1{0}, attr_p2{0};
    const size_t sm = smem2d_t3<T3Pair>(g.nx);
    cudaError_t e = smem_limit_once(g.nx > 4 * T3Pair::kThreads ? attr_p2 : attr_p1, fn,
                                    (int)smem2d_t3<T3Pair>(8 * T3Pair::kThreads));
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, T3Pair::kThreads, sm) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int slots = per_sm * sms;
    R.bpr = slots / nruns > 0 ? slots / nruns : 1;
    const int cy = (g.ny + R.bpr - 1) / R.bpr;
    if (g.nx > 4 * T3Pair::kThreads)
        k_step2d_t3<2, 0, T3Runs2D, T3Pair><<<R.bpr * nruns, T3Pair::kThreads, sm, st>>>(R, g.nx, g.ny, cy, err);
    else
        k_step2d_t3<1, 0, T3Runs2D, T3Pair><<<R.bpr * nruns, T3Pair::kThreads, sm, st>>>(R, g.nx, g.ny, cy, err);
    return cudaGetLastError();
}

}  // namespace prs

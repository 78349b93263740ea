// prs_batch.cu -- ensembles of independent PRS runs (mixed 2D/3D sizes, seeds and
// expansion eras) advanced by one persistent kernel.
//
// The paper motivates large sets of production runs (Sec. I, Sec. IV: calibrating
// the one-scale model needs many realisations); it runs them one at a time.  Here
// every run is cut into the tiles of prs_tile.cuh and the work items
// (run, tile, step n) are numbered in an order that is topological for the
// leapfrog (step-major within a group of runs), so a CTA that takes ticket t only
// ever waits for items with smaller tickets, already taken by running CTAs: the
// schedule cannot deadlock, whatever the number of resident CTAs.
//
//  * Dependencies: item (r, i, n) reads phi^n on tile i and its halo, written by
//    item n-1 of i and of its neighbour tiles, and writes phi^{n+1} over phi^{n-1},
//    which those neighbours read at their item n-1.  So it waits until the
//    progress counter of every neighbour (and of i) reaches n.  The waits are
//    acquire loads in a bounded, sleeping spin; the counters are released after a
//    tile's stores.  A wait that gives up sets an abort flag and an error code.
//  * Diagnostics every `measure_every` steps are fused into the step that reads the
//    same state (one pass over HBM for both); each tile writes its FP64 partial and
//    the last tile of a run's output adds them in tile order.
//  * Groups: runs are packed into groups whose fields fit a budget of L2 bytes, so
//    that small runs are stepped while they are resident in the 129 MB L2.
//  * The tile length and the group budget come from a short timed trial of
//    candidates at creation (the autotuner).  The persistent launch is captured
//    once into a CUDA graph and replayed while the step counts stay the same; the
//    counters are reset and the per-step coefficients uploaded before each replay.
//  * Runs stepped alone: a run whose box fills the GPU by itself (2^22 sites or more),
//    or a 2D run of 2^20 sites or more with 1024-column rows among at least 8 runs of
//    its box, that the library steps with multi-step passes stays out of the persistent
//    kernel.  It gains nothing from sharing the GPU, and its multi-step passes move a
//    half or a third of the bytes of one-step items (2048^2: 9.4 us per step with three
//    steps per pass against 11.4 us as one-step items).  Such a run gets a single-run
//    handle bound to its fields and is stepped after the persistent launch, on the same
//    stream, per output interval by the fused diagnostics pass and the library's passes,
//    its outputs written into the same result array: fields and outputs are those of the
//    run stepped alone through prs_step_measure (the sums to FP64 rounding).  Runs of one
//    2D box at the same step take their passes together, one launch for up to 16 runs
//    (step_measure_first_runs, step_runs), so that each SM marches a long chunk of rows
//    instead of a short chunk of one run.  A
//    fixed rule, not a timed choice, so that two ensembles of the same runs give the same
//    fields.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "prs.h"
#include "prs_internal.h"
#include "prs_runs.h"
#include "prs_reduce.cuh"
#include "prs_sim.h"
#include "prs_tile.cuh"

namespace prs {

namespace {

constexpr int kItems = 4;

struct BRun {
    int dims, nx, ny, nz;
    int t;        // rows per plane tile (3D) or per band (2D)
    int len;      // planes (3D) or rows (2D) per tile
    int ytiles;   // 3D: tiles across y; 2D: 1
    int ntiles;   // tiles per step
    int measure_every;
    int nout;     // outputs this call
    long long nitems;  // items per tile: steps + 1 (the last only measures)
    float* phi[2];     // phi[n & 1] holds phi^n (n counted from the start of the call)
    float* v;
    const float* coef;  // the FP32 kick (KickF) of local step n at coef[4n..4n+3]
    RunConst<float> rc;
    unsigned int* progress;  // per tile: items completed
    DiagAcc* partial;        // [output][tile]
    unsigned int* done;      // per output: tiles finished
    DiagAcc* result;         // per output
};

struct Seg {
    long long base;  // first ticket
    long long n_a;   // first local step
    long long tps;   // tickets per step
    int pos0, m;     // the group's sorted run positions [pos0, pos0+m) are active
};

struct BatchDev {
    const BRun* runs;
    const Seg* segs;
    int nseg;
    const int* pos_run;     // run index at each sorted position
    const int* pos_prefix;  // tiles before this position within its group
    long long total;
    unsigned long long* next;  // ticket counter
    unsigned int* abort_flag;
    unsigned int* err;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned int* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned int* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait until progress[j] >= n for every tile j next to tile i (and i).
__device__ bool wait_neighbours(const BatchDev& d, const BRun& R, int i, unsigned n)
{
    int nb[9];
    int cnt = 0;
    if (R.dims == 2) {
        const int T = R.ntiles;
        nb[cnt++] = i;
        nb[cnt++] = i == 0 ? T - 1 : i - 1;
        nb[cnt++] = i == T - 1 ? 0 : i + 1;
    } else {
        const int YT = R.ytiles, ZT = R.ntiles / R.ytiles;
        const int yt = i % YT, zt = i / YT;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy) {
                const int y = (yt + dy + YT) % YT, z = (zt + dz + ZT) % ZT;
                nb[cnt++] = z * YT + y;
            }
    }
    const unsigned long long t0 = global_ns();
    for (int q = 0; q < cnt; ++q) {
        unsigned sleep = 32;
        while (ld_acquire(R.progress + nb[q]) < n) {
            if (ld_acquire(d.abort_flag)) return false;
            if (global_ns() - t0 > kWaitLimitNs) {
                atomicOr(d.err, kErrWaitTimeout);
                atomicExch(d.abort_flag, 1u);
                return false;
            }
            __nanosleep(sleep);
            sleep = sleep < 1024 ? 2 * sleep : 1024;
        }
    }
    return true;
}

// Block sum of a DiagAcc into thread 0's return value (fixed order).
__device__ DiagAcc block_sum(DiagAcc a)
{
    __shared__ DiagAcc ws[32];
    acc_warp_reduce(a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) ws[wid] = a;
    __syncthreads();
    DiagAcc b{0.0, 0.0, 0, 0, 0, 0};
    if (wid == 0) {
        b = lane < nw ? ws[lane] : DiagAcc{0.0, 0.0, 0, 0, 0, 0};
        acc_warp_reduce(b);
    }
    __syncthreads();
    return b;
}

template <bool STEP, bool MEAS>
__device__ bool run_tile(const BRun& R, int i, long long n, unsigned char* smem, unsigned* wq, SiteAcc& a,
                         unsigned int* err)
{
    KickF k{};
    if (STEP) k = KickF{R.coef[4 * n], R.coef[4 * n + 1], R.coef[4 * n + 2], R.coef[4 * n + 3]};
    const float* pin = R.phi[n & 1];
    float* pout = R.phi[(n + 1) & 1];
    if (R.dims == 3) {
        const int yt = i % R.ytiles, zt = i / R.ytiles;
        Tile3D T{pin, pout, R.v, R.v, R.nx, R.ny, R.nz, R.t, yt * R.t, zt * R.len, 0};
        T.zn = min(R.len, R.nz - T.z0);
        return tile3d<kItems, STEP, MEAS>(T, k, R.rc, smem, wq, a, err);
    }
    Tile2D T{pin, pout, R.v, R.v, R.nx, R.ny, R.t, i * R.len, 0};
    T.yn = min(R.len, R.ny - T.y0);
    return tile2d<kItems, STEP, MEAS>(T, k, R.rc, smem, wq, a, err);
}

__global__ void __launch_bounds__(kFastThreads, 2) k_batch(BatchDev d, int queue_off)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ long long s_ticket;
    __shared__ int s_last;
    const int tid = threadIdx.x;
    unsigned* wq = reinterpret_cast<unsigned*>(smem + queue_off) + (tid >> 5) * kQueuePerWarp;
    for (;;) {
        if (tid == 0) s_ticket = (long long)atomicAdd(d.next, 1ull);
        __syncthreads();
        const long long t = s_ticket;
        if (t >= d.total) break;
        // decode the ticket: segment, local step, group position, tile
        int lo = 0, hi = d.nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (d.segs[mid].base <= t) lo = mid; else hi = mid - 1;
        }
        const Seg sg = d.segs[lo];
        const long long local = t - sg.base;
        const long long n = sg.n_a + local / sg.tps;
        const int rem = (int)(local % sg.tps);
        int a0 = sg.pos0, a1 = sg.pos0 + sg.m - 1;
        while (a0 < a1) {
            const int mid = (a0 + a1 + 1) >> 1;
            if (d.pos_prefix[mid] <= rem) a0 = mid; else a1 = mid - 1;
        }
        const int r = d.pos_run[a0];
        const int i = rem - d.pos_prefix[a0];
        const BRun& R = d.runs[r];

        bool ok = true;
        if (tid == 0) ok = wait_neighbours(d, R, i, (unsigned)n);
        if (__syncthreads_or(!ok)) break;

        const bool meas = R.measure_every > 0 && (n % R.measure_every) == 0;
        const bool step = n < R.nitems - 1;
        SiteAcc acc{0.0, 0.0, 0.0f, 0.0f, 0, 0, 0, 0};
        if (step && meas) ok = run_tile<true, true>(R, i, n, smem, wq, acc, d.err);
        else if (step) ok = run_tile<true, false>(R, i, n, smem, wq, acc, d.err);
        else if (meas) ok = run_tile<false, true>(R, i, n, smem, wq, acc, d.err);
        if (!ok) {
            if (tid == 0) atomicExch(d.abort_flag, 1u);
            break;
        }
        if (meas) {
            const DiagAcc b = block_sum(DiagAcc{acc.sw, acc.sr, acc.nl, acc.nw, acc.nv0, acc.nnf});
            const int k = (int)(n / R.measure_every);
            if (tid == 0) {
                R.partial[(size_t)k * R.ntiles + i] = b;
                __threadfence();
                s_last = atomicAdd(R.done + k, 1u) == (unsigned)R.ntiles - 1;
            }
            __syncthreads();
            if (s_last && tid < 32) {  // the run's last tile of this output adds the partials in tile order
                __threadfence();
                DiagAcc tot{0.0, 0.0, 0, 0, 0, 0};
                for (int j = tid; j < R.ntiles; j += 32) {
                    const DiagAcc* q = R.partial + (size_t)k * R.ntiles + j;
                    DiagAcc p{__ldcg(&q->sum_w), __ldcg(&q->sum_ratio), __ldcg(&q->n_links),
                              __ldcg(&q->n_wall), __ldcg(&q->n_vzero), __ldcg(&q->n_nonfinite)};
                    acc_add(tot, p);
                }
                acc_warp_reduce(tot);
                if (tid == 0) R.result[k] = tot;
            }
        }
        __syncthreads();  // every store of this item precedes the release below
        if (tid == 0) {
            __threadfence();
            st_release(R.progress + i, (unsigned)(n + 1));
        }
    }
}

}  // namespace

}  // namespace prs

using namespace prs;

struct prs_batch {
    std::vector<prs_params> p;
    std::vector<Geo> g;
    std::vector<int64_t> n;  // current step of each run
    std::vector<int> cur;    // which buffer holds phi^n
    std::vector<float*> phi0, phi1, v;
    std::vector<double> rc;  // 6 per run
    cudaStream_t stream;
    bool own_stream;
    char* fields;            // one allocation for every run's fields
    // tuned layout
    std::vector<int> len;     // tile length per run
    double group_budget;      // bytes of fields per group
    // device work buffers, sized by the last schedule
    void* work;
    size_t work_bytes;
    unsigned int* d_err;     // error word + abort flag + ticket counter live here
    unsigned int* h_err;
    std::vector<prs_sim*> solo;  // per run: its handle when stepped alone, else null
    cudaGraphExec_t graph;
    std::vector<int64_t> graph_nsteps;
    int64_t graph_measure;
    int smem;
    int grid;
};

static int batch_cuda(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return PRS_OK;
    char msg[256];
    snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    record_error(msg);
    return PRS_ECUDA;
}

static const int kTileLens[] = {4, 8, 16, 32};  // bands (2D) or planes (3D) per tile
static const int kNumTileLens = 4;

static int tile_rows(const Geo& g) { return kItems * 1024 / g.nx; }

// Builds the run descriptors and the ticket schedule for one call; returns the
// device-side BatchDev (pointers into b->work) and fills the host mirrors.
struct Schedule {
    std::vector<BRun> runs;
    std::vector<Seg> segs;
    std::vector<int> pos_run, pos_prefix;
    std::vector<float> coef;       // all runs' coefficient tables
    std::vector<size_t> coef_off;  // per run, in floats
    std::vector<size_t> prog_off, part_off, done_off, res_off;
    long long total = 0;
    size_t bytes = 0;
};

static int64_t align256(int64_t x) { return (x + 255) & ~(int64_t)255; }

static void plan(const prs_batch* b, const int64_t* nsteps, int64_t measure_every, double budget, Schedule& S)
{
    const int R = (int)b->p.size();
    S.runs.resize(R);
    S.coef_off.resize(R);
    S.prog_off.resize(R);
    S.part_off.resize(R);
    S.done_off.resize(R);
    S.res_off.resize(R);
    size_t off = 0;
    for (int r = 0; r < R; ++r) {
        const Geo& g = b->g[r];
        BRun& u = S.runs[r];
        u.dims = g.dims;
        u.nx = g.nx;
        u.ny = g.ny;
        u.nz = g.nz;
        u.t = tile_rows(g);
        if (g.dims == 3) {
            u.len = b->len[r];
            u.ytiles = g.ny / u.t;
            u.ntiles = u.ytiles * ((g.nz + u.len - 1) / u.len);
        } else {
            u.len = b->len[r] * u.t;
            u.ytiles = 1;
            u.ntiles = (g.ny + u.len - 1) / u.len;
        }
        u.measure_every = (int)measure_every;
        const bool alone = b->solo[r] != nullptr;  // no items in the persistent kernel
        u.nitems = alone ? 0 : nsteps[r] + 1;
        u.nout = measure_every > 0 ? (int)(nsteps[r] / measure_every) + 1 : 0;
        const double* rcd = &b->rc[6 * (size_t)r];
        u.rc = RunConst<float>{(float)rcd[0], (float)rcd[1], (float)rcd[2], (float)rcd[3], (float)rcd[4],
                               (float)rcd[5]};
        S.coef_off[r] = S.coef.size();
        for (int64_t k = 0; k < (alone ? 0 : nsteps[r]); ++k) {
            double c[5];
            step_coefficients(b->p[r], b->n[r] + k, c);
            const KickF kf = kick_f32(c, rcd);
            S.coef.push_back(kf.c1);
            S.coef.push_back(kf.g);
            S.coef.push_back(kf.k1);
            S.coef.push_back(kf.k2);
        }
        S.prog_off[r] = off;
        off += align256(sizeof(unsigned) * (size_t)u.ntiles);
        S.part_off[r] = off;
        off += align256(sizeof(DiagAcc) * (size_t)u.ntiles * (size_t)(u.nout > 0 ? u.nout : 1));
        S.done_off[r] = off;
        off += align256(sizeof(unsigned) * (size_t)(u.nout > 0 ? u.nout : 1));
        S.res_off[r] = off;
        off += align256(sizeof(DiagAcc) * (size_t)(u.nout > 0 ? u.nout : 1));
    }
    // groups: consecutive runs (in the caller's order) whose fields fit the budget
    std::vector<std::vector<int>> groups;
    double acc = 0.0;
    for (int r = 0; r < R; ++r) {
        if (b->solo[r]) continue;
        const double fb = 3.0 * (double)b->g[r].S * sizeof(float);
        if (groups.empty() || acc + fb > budget) {
            groups.emplace_back();
            acc = 0.0;
        }
        groups.back().push_back(r);
        acc += fb;
    }
    long long base = 0;
    for (auto& grp : groups) {
        std::vector<int> order(grp);
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return S.runs[x].nitems > S.runs[y].nitems; });
        const int pos0 = (int)S.pos_run.size();
        int pre = 0;
        for (int r : order) {
            S.pos_run.push_back(r);
            S.pos_prefix.push_back(pre);
            pre += S.runs[r].ntiles;
        }
        // active prefix shrinks as runs finish: one segment per distinct length
        long long n_a = 0;
        int m = (int)order.size();
        while (m > 0) {
            const long long n_b = S.runs[order[m - 1]].nitems;
            long long tps = 0;
            for (int q = 0; q < m; ++q) tps += S.runs[order[q]].ntiles;
            if (n_b > n_a) {
                S.segs.push_back(Seg{base, n_a, tps, pos0, m});
                base += (n_b - n_a) * tps;
                n_a = n_b;
            }
            --m;
        }
    }
    S.total = base;
    S.bytes = off;
}

extern "C" int prs_batch_destroy(prs_batch* b);

static int run_schedule(prs_batch* b, const int64_t* nsteps, int64_t measure_every, double budget, Schedule& S,
                        bool use_graph)
{
    plan(b, nsteps, measure_every, budget, S);
    const int R = (int)b->p.size();
    // device layout: [counters ...][runs][segs][pos_run][pos_prefix][coef]
    size_t o_runs = align256((int64_t)S.bytes);
    size_t o_segs = o_runs + align256(sizeof(BRun) * R);
    size_t o_pr = o_segs + align256(sizeof(Seg) * (S.segs.size() + 1));
    size_t o_pp = o_pr + align256(sizeof(int) * (S.pos_run.size() + 1));
    size_t o_coef = o_pp + align256(sizeof(int) * (S.pos_prefix.size() + 1));
    size_t total = o_coef + align256(sizeof(float) * (S.coef.size() + 1));
    if (total > b->work_bytes) {
        if (b->graph) cudaGraphExecDestroy(b->graph), b->graph = nullptr;
        cudaFree(b->work);
        b->work = nullptr;
        if (cudaMalloc(&b->work, total) != cudaSuccess) {
            cudaGetLastError();
            b->work_bytes = 0;
            return PRS_ENOMEM;
        }
        b->work_bytes = total;
    }
    char* w = (char*)b->work;
    for (int r = 0; r < R; ++r) {
        BRun& u = S.runs[r];
        u.phi[0] = b->cur[r] == 0 ? b->phi0[r] : b->phi1[r];
        u.phi[1] = b->cur[r] == 0 ? b->phi1[r] : b->phi0[r];
        u.v = b->v[r];
        u.coef = (const float*)(w + o_coef) + S.coef_off[r];
        u.progress = (unsigned*)(w + S.prog_off[r]);
        u.partial = (DiagAcc*)(w + S.part_off[r]);
        u.done = (unsigned*)(w + S.done_off[r]);
        u.result = (DiagAcc*)(w + S.res_off[r]);
    }
    BatchDev d;
    d.runs = (const BRun*)(w + o_runs);
    d.segs = (const Seg*)(w + o_segs);
    d.nseg = (int)S.segs.size();
    d.pos_run = (const int*)(w + o_pr);
    d.pos_prefix = (const int*)(w + o_pp);
    d.total = S.total;
    d.next = (unsigned long long*)(b->d_err + 2);
    d.abort_flag = b->d_err + 1;
    d.err = b->d_err;
    const int queue_off = b->smem - (int)kQueueBytes;
    cudaStream_t st = b->stream;
    int rc;
    if ((rc = batch_cuda(cudaMemsetAsync(w, 0, S.bytes, st), "batch reset"))) return rc;
    if ((rc = batch_cuda(cudaMemsetAsync(b->d_err + 1, 0, 3 * sizeof(unsigned), st), "batch reset"))) return rc;
    if ((rc = batch_cuda(cudaMemcpyAsync(w + o_runs, S.runs.data(), sizeof(BRun) * R, cudaMemcpyHostToDevice, st),
                         "batch upload")))
        return rc;
    if ((rc = batch_cuda(cudaMemcpyAsync(w + o_segs, S.segs.data(), sizeof(Seg) * S.segs.size(),
                                         cudaMemcpyHostToDevice, st), "batch upload")))
        return rc;
    if ((rc = batch_cuda(cudaMemcpyAsync(w + o_pr, S.pos_run.data(), sizeof(int) * S.pos_run.size(),
                                         cudaMemcpyHostToDevice, st), "batch upload")))
        return rc;
    if ((rc = batch_cuda(cudaMemcpyAsync(w + o_pp, S.pos_prefix.data(), sizeof(int) * S.pos_prefix.size(),
                                         cudaMemcpyHostToDevice, st), "batch upload")))
        return rc;
    if (!S.coef.empty() &&
        (rc = batch_cuda(cudaMemcpyAsync(w + o_coef, S.coef.data(), sizeof(float) * S.coef.size(),
                                         cudaMemcpyHostToDevice, st), "batch upload")))
        return rc;
    // the same launch every call with this schedule: replay it from a CUDA graph
    const bool same = use_graph && b->graph && b->graph_measure == measure_every &&
                      b->graph_nsteps == std::vector<int64_t>(nsteps, nsteps + R);
    if (same) return batch_cuda(cudaGraphLaunch(b->graph, st), "batch graph launch");
    if (use_graph) {
        if (b->graph) cudaGraphExecDestroy(b->graph), b->graph = nullptr;
        cudaGraph_t gr;
        if ((rc = batch_cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "batch capture")))
            return rc;
        k_batch<<<b->grid, kFastThreads, b->smem, st>>>(d, queue_off);
        cudaError_t e = cudaStreamEndCapture(st, &gr);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, gr, 0);
        if (e == cudaSuccess) cudaGraphDestroy(gr);
        if ((rc = batch_cuda(e, "batch graph"))) return rc;
        b->graph_nsteps.assign(nsteps, nsteps + R);
        b->graph_measure = measure_every;
        return batch_cuda(cudaGraphLaunch(b->graph, st), "batch graph launch");
    }
    k_batch<<<b->grid, kFastThreads, b->smem, st>>>(d, queue_off);
    return batch_cuda(cudaGetLastError(), "batch launch");
}

// Runs stepped alone, among those the library steps with multi-step passes (the ensemble's
// runs are FP32): boxes of 2^22 sites or more, which fill the GPU by themselves, and 2D boxes
// of 2^20 sites or more with rows of at least 1024 columns when the ensemble holds at least 8
// runs of that box, whose grouped three-step launches fill it together (16 x 1024^2 in the
// 64-run ensemble: 1.41 s against 1.47-1.60 s with them in the persistent kernel).
// class_runs: the runs of this box in the ensemble.
static bool steps_alone(const Geo& g, int class_runs)
{
    if (default_fused_steps(g, PRS_FP32, false) < 2) return false;
    if (g.S >= ((int64_t)1 << 22)) return true;
    return g.dims == 2 && g.nx >= 1024 && g.S >= ((int64_t)1 << 20) && class_runs >= 8;
}

// A run stepped alone: its handle follows the batch's view of the run (which field buffer
// holds phi^n, the step count) before it steps, and the batch takes the buffer back after.
static void solo_sync_in(prs_batch* b, int r)
{
    prs_sim* s = b->solo[r];
    s->cur = b->cur[r];
    s->n = b->n[r];
}

static int solo_make(prs_batch* b, int r)
{
    prs_sim* s = nullptr;
    int rc = prs_create(&b->p[r], b->stream, &s);
    if (!rc) rc = prs_bind(s, b->phi0[r], b->phi1[r], b->v[r]);
    if (!rc) {
        s->cur = b->cur[r];  // phi[0] = phi0, phi[1] = phi1: no copy below
        rc = prs_set_state_device(s, b->cur[r] == 0 ? b->phi0[r] : b->phi1[r], b->v[r], b->n[r]);
    }
    if (rc) {
        if (s) prs_destroy(s);
        return rc;
    }
    b->solo[r] = s;
    return PRS_OK;
}

// Queue the runs stepped alone, after the persistent launch, in groups of runs of one box
// at the same step with the same step count (at most kT3MaxRuns a group, which step_runs
// advances together, pass by pass): with outputs, per output the diagnostics of each run's
// state (into its result slot) fused into its first step, one launch for the group
// (step_measure_first_runs), then the steps up to the next output; else the steps.  Each run
// gets the passes prs_step_measure would give it alone (its fields bit for bit; its sums to
// FP64 rounding, their blocks grouped differently).
// Leaves b->cur to the caller (solo_take_back).
static int solo_queue(prs_batch* b, const int64_t* nsteps, int64_t measure_every, const Schedule& S)
{
    const int R = (int)b->p.size();
    std::vector<char> queued(R, 0);
    for (int r0 = 0; r0 < R; ++r0) {
        if (!b->solo[r0] || queued[r0]) continue;
        std::vector<int> grp;
        const Geo& a = b->g[r0];
        for (int r = r0; r < R && (int)grp.size() < kT3MaxRuns; ++r) {
            const Geo& g = b->g[r];
            if (b->solo[r] && !queued[r] && g.dims == a.dims && g.nx == a.nx && g.ny == a.ny && g.nz == a.nz &&
                b->n[r] == b->n[r0] && nsteps[r] == nsteps[r0])
                grp.push_back(r), queued[r] = 1;
        }
        std::vector<prs_sim*> sims;
        for (int r : grp) {
            solo_sync_in(b, r);
            sims.push_back(b->solo[r]);
        }
        const int m_runs = (int)sims.size();
        int rc = PRS_OK;
        if (measure_every > 0) {
            std::vector<int64_t> taken(m_runs, 0);
            for (int k = 0; k < S.runs[r0].nout && !rc; ++k) {
                const int64_t left = nsteps[r0] - (int64_t)k * measure_every;
                const int64_t m = left < measure_every ? left : measure_every;
                std::vector<DiagAcc*> res(m_runs);
                for (int q = 0; q < m_runs; ++q) res[q] = (DiagAcc*)((char*)b->work + S.res_off[grp[q]]) + k;
                rc = step_measure_first_runs(sims.data(), m_runs, m, res.data(), taken.data());
                bool same = true;
                for (int q = 0; q < m_runs; ++q) same = same && taken[q] == taken[0];
                if (!rc && same) rc = step_runs(sims.data(), m_runs, m - taken[0]);
                for (int q = 0; q < m_runs && !rc && !same; ++q) rc = step_runs(&sims[q], 1, m - taken[q]);
            }
        } else {
            rc = step_runs(sims.data(), m_runs, nsteps[r0]);
        }
        if (rc) return rc;
    }
    return PRS_OK;
}

static void solo_take_back(prs_batch* b)
{
    for (int r = 0; r < (int)b->p.size(); ++r)
        if (b->solo[r]) b->cur[r] = b->solo[r]->cur;
}

// Times one candidate layout on the batch's fields for a few steps.
static double trial(prs_batch* b, double budget, int steps)
{
    const int R = (int)b->p.size();
    std::vector<int64_t> ns(R, steps);
    Schedule S;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, b->stream);
    int rc = run_schedule(b, ns.data(), 0, budget, S, false);  // the runs stepped alone sit out
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 1e30f;
    if (rc == PRS_OK) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int r = 0; r < R; ++r)
        if ((steps & 1) && !b->solo[r]) b->cur[r] ^= 1;
    return rc == PRS_OK ? ms : 1e30;
}

// The autotuner: a tile length per geometry class (runs of equal dims and sides), by one
// sweep of coordinate descent from 16 — the layout that ran the 64-run mixed ensemble (16 each
// of 256^2, 1024^2, 2048^2, 128^3 to eta = N/2) fastest among those timed in full (2.21 s;
// 8 everywhere 2.33 s, 4 everywhere 2.63 s) — each class in turn tries every candidate (4 to 32)
// while the others keep theirs, timed as the difference of a 24-step and a 12-step trial of
// the whole ensemble (the steady-state cost of 12 steps: shorter trials, dominated by the
// pipeline's fill and drain, picked tiles too short for long runs), and takes one only when it
// is at least 3% faster (timing noise then rarely changes the choice) — then the group
// budget.  The fields do not depend on the choice; the diagnostic sums group per-tile
// partials, so they agree across choices to FP64 rounding.
static void autotune(prs_batch* b)
{
    const int R = (int)b->p.size();
    const int steps = 12;
    std::vector<int> cls(R, -1);  // class of each run
    std::vector<int> reps;        // first run of each class
    for (int r = 0; r < R; ++r) {
        for (size_t c = 0; c < reps.size() && cls[r] < 0; ++c) {
            const Geo& a = b->g[reps[c]];
            const Geo& g = b->g[r];
            if (a.dims == g.dims && a.nx == g.nx && a.ny == g.ny && a.nz == g.nz) cls[r] = (int)c;
        }
        if (cls[r] < 0) {
            cls[r] = (int)reps.size();
            reps.push_back(r);
        }
    }
    // the steady-state cost of a layout: a long trial minus a short one, so that the
    // pipeline's fill and drain (which long runs amortise) do not favour short tiles
    auto cost = [&](double budget) { return trial(b, budget, 2 * steps) - trial(b, budget, steps); };
    for (int r = 0; r < R; ++r) b->len[r] = 16;  // the best layout of full runs measured (see above)
    double best = cost(1e18);
    for (size_t c = 0; c < reps.size(); ++c) {
        if (b->solo[reps[c]]) continue;  // stepped alone: no tiles
        int best_len = b->len[reps[c]];
        for (int li = 0; li < kNumTileLens; ++li) {
            if (kTileLens[li] == best_len) continue;
            for (int r = 0; r < R; ++r)
                if (cls[r] == (int)c) b->len[r] = kTileLens[li];
            const double ms = cost(1e18);
            if (ms < 0.97 * best) best = ms, best_len = kTileLens[li];  // a clear gain only
        }
        for (int r = 0; r < R; ++r)
            if (cls[r] == (int)c) b->len[r] = best_len;
    }
    // then L2 groups, again only for a clear gain over one group (several groups run one
    // after the other, which starves the GPU once only a group's long runs are left)
    b->group_budget = 1e18;
    for (double bu : {64e6, 96e6}) {
        const double ms = cost(bu);
        if (ms < 0.97 * best) best = ms, b->group_budget = bu;
    }
}

extern "C" int prs_batch_create(const prs_params* runs, int nruns, void* stream, prs_batch** out)
{
    if (!runs || nruns < 1 || !out) return PRS_EINVAL;
    prs_batch* b = new (std::nothrow) prs_batch();
    if (!b) return PRS_ENOMEM;
    b->group_budget = 96e6;
    size_t total = 0;
    for (int r = 0; r < nruns; ++r) {
        // validate through a throwaway run description
        prs_sim* probe = nullptr;
        int rc = prs_create(&runs[r], nullptr, &probe);
        if (rc) {
            delete b;
            return rc;
        }
        Geo g = probe->g;
        double rcd[6];
        memcpy(rcd, probe->rc, sizeof rcd);
        prs_destroy(probe);
        if (!fast_step_ok(g, runs[r].precision) || (g.dims == 3 && g.nx > 1024) || runs[r].flags != 0) {
            record_error("prs_batch_create: runs must be FP32 with an x side that is a multiple of 128 and divides "
                         "4096 (3D: at most 1024), and 4096/nx dividing the y side");
            delete b;
            return PRS_EINVAL;
        }
        b->p.push_back(runs[r]);
        b->g.push_back(g);
        b->rc.insert(b->rc.end(), rcd, rcd + 6);
        total += 3 * (size_t)align256((int64_t)g.S * 4);
    }
    b->n.assign(nruns, 0);
    b->cur.assign(nruns, 0);
    b->len.assign(nruns, 16);
    b->solo.assign(nruns, nullptr);
    b->own_stream = stream == nullptr;
    int rc = PRS_OK;
    if (b->own_stream)
        rc = batch_cuda(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "prs_batch_create");
    else
        b->stream = (cudaStream_t)stream;
    if (rc) {
        delete b;
        return rc;
    }
    if (cudaMalloc((void**)&b->fields, total) != cudaSuccess ||
        cudaMalloc((void**)&b->d_err, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_err, 4 * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        prs_batch_destroy(b);
        return PRS_ENOMEM;
    }
    size_t off = 0;
    for (int r = 0; r < nruns; ++r) {
        const size_t fb = (size_t)align256(b->g[r].S * 4);
        b->phi0.push_back((float*)(b->fields + off));
        b->phi1.push_back((float*)(b->fields + off + fb));
        b->v.push_back((float*)(b->fields + off + 2 * fb));
        off += 3 * fb;
    }
    // shared memory: the largest tile plus the link queue; two CTAs per SM
    size_t sm = 0;
    for (int r = 0; r < nruns; ++r) {
        const Geo& g = b->g[r];
        sm = std::max(sm, (g.dims == 3 ? tile_smem3d(g.nx, tile_rows(g)) : tile_smem2d(g.nx, tile_rows(g))) +
                              kQueueBytes);
    }
    b->smem = (int)sm;
    rc = batch_cuda(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, b->smem),
                    "prs_batch_create");
    int per_sm = 0;
    if (!rc)
        rc = batch_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kFastThreads, b->smem),
                        "prs_batch_create");
    if (!rc && per_sm < 1) rc = PRS_EINVAL;
    if (rc) {
        prs_batch_destroy(b);
        return rc;
    }
    b->grid = per_sm * sm_count_current();
    // fields start from each run's seeded random initial condition; tune, then reset
    for (int r = 0; r < nruns && !rc; ++r)
        rc = batch_cuda(launch_init_random(b->g[r], PRS_FP32, runs[r].seed, b->phi0[r], b->v[r], true, b->stream),
                        "prs_batch_create");
    for (int r = 0; r < nruns && !rc; ++r) {
        int same = 0;
        for (const Geo& q : b->g)
            same += q.dims == b->g[r].dims && q.nx == b->g[r].nx && q.ny == b->g[r].ny && q.nz == b->g[r].nz;
        if (steps_alone(b->g[r], same)) rc = solo_make(b, r);
    }
    if (!rc) autotune(b);
    for (int r = 0; r < nruns && !rc; ++r) {
        rc = batch_cuda(launch_init_random(b->g[r], PRS_FP32, runs[r].seed, b->phi0[r], b->v[r], true, b->stream),
                        "prs_batch_create");
        b->cur[r] = 0;
        b->n[r] = 0;
    }
    if (!rc) rc = batch_cuda(cudaStreamSynchronize(b->stream), "prs_batch_create");
    if (rc) {
        prs_batch_destroy(b);
        return rc;
    }
    *out = b;
    return PRS_OK;
}

extern "C" int prs_batch_run(prs_batch* b, const int64_t* nsteps_per_run, int64_t measure_every, double* out_series,
                             int64_t out_capacity)
{
    if (!b || !nsteps_per_run || measure_every < 0) return PRS_EINVAL;
    const int R = (int)b->p.size();
    for (int r = 0; r < R; ++r) {
        if (nsteps_per_run[r] < 0) return PRS_EINVAL;
        if (nsteps_per_run[r] > 0 && !cfl_ok_over(b->p[r], b->n[r], nsteps_per_run[r])) return PRS_EINVAL;
        if (measure_every > 0 && (!out_series || nsteps_per_run[r] / measure_every + 1 > out_capacity))
            return PRS_EINVAL;
    }
    Schedule S;
    int rc = run_schedule(b, nsteps_per_run, measure_every, b->group_budget, S, true);
    if (rc) return rc;
    rc = solo_queue(b, nsteps_per_run, measure_every, S);
    solo_take_back(b);
    if (rc) return rc;
    std::vector<DiagAcc> res;
    if (measure_every > 0) {
        size_t nres = 0;
        for (int r = 0; r < R; ++r) nres += (size_t)S.runs[r].nout;
        res.resize(nres);
        size_t at = 0;
        for (int r = 0; r < R; ++r) {
            const int no = S.runs[r].nout;
            if ((rc = batch_cuda(cudaMemcpyAsync(res.data() + at, (char*)b->work + S.res_off[r], sizeof(DiagAcc) * no,
                                                 cudaMemcpyDeviceToHost, b->stream), "prs_batch_run")))
                return rc;
            at += no;
        }
    }
    if ((rc = batch_cuda(cudaMemcpyAsync(b->h_err, b->d_err, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream),
                         "prs_batch_run")))
        return rc;
    for (prs_sim* s : b->solo)  // the error words of the runs stepped alone
        if (s && (rc = batch_cuda(cudaMemcpyAsync(&s->h_status->error, &s->d_status->error, sizeof(unsigned),
                                                  cudaMemcpyDeviceToHost, b->stream), "prs_batch_run")))
            return rc;
    if ((rc = batch_cuda(cudaStreamSynchronize(b->stream), "prs_batch_run"))) return rc;
    if (b->h_err[0] || b->h_err[1]) {
        record_error("prs_batch_run: a bounded wait in the persistent kernel gave up");
        cudaMemsetAsync(b->d_err, 0, 2 * sizeof(unsigned), b->stream);
        cudaStreamSynchronize(b->stream);
        return PRS_ETIMEOUT;
    }
    for (prs_sim* s : b->solo)
        if (s && (rc = check_device_error(s))) return rc;
    size_t at = 0;
    for (int r = 0; r < R; ++r) {
        const int no = S.runs[r].nout;
        for (int k = 0; k < no; ++k) {
            const DiagAcc& a = res[at + k];
            double* o = out_series + ((size_t)r * out_capacity + k) * 4;
            const int64_t nw = a.n_wall - a.n_vzero;
            o[0] = (double)(b->n[r] + (int64_t)k * measure_every);
            o[1] = a.sum_w / ((double)b->g[r].S * b->p[r].dx);
            o[2] = nw > 0 ? sqrt(a.sum_ratio / (2.0 * (double)nw)) : 0.0;
            o[3] = (double)a.n_links;
        }
        at += no;
        b->n[r] += nsteps_per_run[r];
        if ((nsteps_per_run[r] & 1) && !b->solo[r]) b->cur[r] ^= 1;
    }
    return PRS_OK;
}

extern "C" int prs_batch_get_state(prs_batch* b, int run, void* h_phi, void* h_dphi, int64_t* n)
{
    if (!b || run < 0 || run >= (int)b->p.size()) return PRS_EINVAL;
    const size_t fb = (size_t)b->g[run].S * 4;
    const float* phi = b->cur[run] == 0 ? b->phi0[run] : b->phi1[run];
    int rc;
    if (h_phi && (rc = batch_cuda(cudaMemcpyAsync(h_phi, phi, fb, cudaMemcpyDeviceToHost, b->stream), "get_state")))
        return rc;
    if (h_dphi &&
        (rc = batch_cuda(cudaMemcpyAsync(h_dphi, b->v[run], fb, cudaMemcpyDeviceToHost, b->stream), "get_state")))
        return rc;
    if ((rc = batch_cuda(cudaStreamSynchronize(b->stream), "get_state"))) return rc;
    if (n) *n = b->n[run];
    return PRS_OK;
}

extern "C" int prs_batch_set_state(prs_batch* b, int run, const void* h_phi, const void* h_dphi, int64_t n)
{
    if (!b || run < 0 || run >= (int)b->p.size() || !h_phi || !h_dphi || n < 0) return PRS_EINVAL;
    const size_t fb = (size_t)b->g[run].S * 4;
    float* phi = b->cur[run] == 0 ? b->phi0[run] : b->phi1[run];
    int rc;
    if ((rc = batch_cuda(cudaMemcpyAsync(phi, h_phi, fb, cudaMemcpyHostToDevice, b->stream), "set_state"))) return rc;
    if ((rc = batch_cuda(cudaMemcpyAsync(b->v[run], h_dphi, fb, cudaMemcpyHostToDevice, b->stream), "set_state")))
        return rc;
    if ((rc = batch_cuda(cudaStreamSynchronize(b->stream), "set_state"))) return rc;
    b->n[run] = n;
    return PRS_OK;
}

extern "C" int prs_batch_tuning(prs_batch* b, int run, int* tile_len, double* group_bytes)
{
    if (!b || run < 0 || run >= (int)b->p.size()) return PRS_EINVAL;
    if (tile_len) *tile_len = b->solo[run] ? 0 : b->len[run];
    if (group_bytes) *group_bytes = b->group_budget;
    return PRS_OK;
}

extern "C" int prs_batch_destroy(prs_batch* b)
{
    if (!b) return PRS_EINVAL;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (prs_sim* s : b->solo)
        if (s) prs_destroy(s);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->work);
    cudaFree(b->fields);
    cudaFree(b->d_err);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return PRS_OK;
}

// prs_tblock.cu -- two leapfrog steps (Eqs. 3-5) per pass over HBM, FP32 3D and 2D.
//
// One pass reads phi^n, dphi^{n-1/2} once and writes phi^{n+2}, dphi^{n+3/2} once:
// 16 bytes per two site-updates.
//
// 3D: a CTA owns a tile of xw columns (the whole row, or a 128-multiple slice of it) by
// ty rows and a chunk of z-planes, and marches along z through two levels:
//   level 1 (step n)   on ty+2 rows, from level-0 phi planes of ty+4 rows in a 4-slot
//                       ring and dphi^{n-1/2} planes of ty+2 rows in a 3-slot ring;
//   level 2 (step n+1) on the ty output rows, one plane behind level 1, from level-1
//                       planes kept in a 2-slot ring.
// The TMA engine (cp.async.bulk) stages phi and dphi planes two iterations ahead, row
// by row, the copies spread over the warps.  Every staged row holds the columns
// [x0-4, x0+xw+4) (periodic in x), so a tile's edge columns find their x neighbours in
// the same shared-memory row: a warp covers 32 float4 of one row and takes its x
// neighbours by shuffle, lanes 0 and 31 from that row.  Shared memory serves only the x
// and y neighbours: each thread keeps the values of its own columns at planes z-1, z,
// z+1 in registers, for level 0 and for level 1, so one barrier per plane suffices.
// Level 1 also computes the two columns just outside a sliced tile (x0-1 and x0+xw,
// one thread of warp 0 per row and side), which level 2 needs as x neighbours; for
// whole rows those are the row's own wrapped end columns.  dphi enters level 1 on ty+2 rows (its halo
// rows belong to neighbouring tiles), so it is read from one buffer and written to
// another; the level-1 dphi stays in the registers of the thread that owns its site
// until level 2 uses it.
#include <cuda_runtime.h>

#include "prs_internal.h"
#include "prs_ptx.cuh"
#include "prs_tile.cuh"

namespace prs {

namespace {

constexpr int kTbThreads = 320;  // at most; a CTA has ceil((ty+2) * xw/4 / kTbItems) threads
constexpr int kTbItems = 2;      // level-1 float4 per thread per plane
constexpr int kTbMaxTy = 14;     // sliced tiles: 2 (ty+2) halo columns per plane, one lane each of warp 0

static __device__ __noinline__ void drain4(uint64_t* bar, int from, int issued, unsigned int* err)
{
    for (int i = from; i <= issued; ++i) mbar_wait(&bar[i & 3], (unsigned)(i >> 2) & 1u, err);
}

// MID: also store the state between the two steps (phi^{n+1}, dphi^{n+1/2}: level 1 at
// the output sites) into phi_mid, v_mid.
// The 128 x 8 tile (160 threads, 53 KB of shared memory) runs four CTAs per SM.
template <int ITEMS, int XW, int TY, bool MID>
__global__ void __launch_bounds__(XW == 128 && TY == 8 ? 160 : kTbThreads, XW == 128 && TY == 8 ? 4 : 2)
    k_step3d_t2(const float* __restrict__ phi_in, float* __restrict__ phi_out, const float* __restrict__ v_in,
                float* __restrict__ v_out, float* __restrict__ phi_mid, float* __restrict__ v_mid, int nx, int ny,
                int nz, int ty_, int cz, KickF k0, KickF k1, RunConst<float> rc, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    constexpr int xw = XW;
    constexpr int W = xw + 8;              // floats per staged row: columns x0-4 .. x0+xw+3
    const int ty = TY > 0 ? TY : ty_;
    const int r0 = ty + 4, r1 = ty + 2;    // rows of a level-0 and a level-1 plane tile
    const int s0 = r0 * W, s1 = r1 * W;    // floats per ring slot
    float* ring0 = reinterpret_cast<float*>(smem_raw + 128);  // phi^n: 4 slots
    float* ring1 = ring0 + 4 * s0;                            // level 1: 2 slots
    float* ringv = ring1 + 2 * s1;                            // dphi^{n-1/2}: 3 slots
    const int tid = threadIdx.x, lane = tid & 31;
    // the launch's thread count (plan3's formula), a constant for a fixed tile shape
    const int nthr = TY > 0 ? (((TY + 2) * (XW / 4) + ITEMS - 1) / ITEMS + 31) / 32 * 32 : (int)blockDim.x;
    const int nxt = nx / xw, ytiles = ny / ty;
    const int x0 = (blockIdx.x % nxt) * xw;
    const int y0 = (blockIdx.x / nxt % ytiles) * ty;
    const int z0 = blockIdx.x / nxt / ytiles * cz;
    const int zn = min(cz, nz - z0);
    const int nq = xw >> 2;
    const bool whole = xw == nx;
    const size_t plane = (size_t)nx * ny;
    const int nplanes = zn + 4;  // level-0 local planes 0..zn+3 = global z0-2 .. z0+zn+1

    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto wy = [&](int y) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); };
    auto wz = [&](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };
    // Iteration i stages phi plane i+2 and, for the level-1 planes 1..zn+2, dphi plane
    // i+1, both counted on bar[(i+2) % 4] (phi planes 0 and 1 go first, alone).  A staged
    // row is [x0-4, x0+xw+4) modulo nx: at most three runs, each a multiple of 4 floats
    // at a 16-byte boundary, at the same columns in every row.  Copy task c < 3 (r0 + r1)
    // is run c % 3 of staged row c / 3 (phi rows first, then dphi rows); thread
    // nthr-1-c owns it for the whole pass (the last warps, whose second item lies in the
    // level-1 halo row and has no level-2 work), so staging a plane costs each copying
    // thread one instruction sequence; thread 0 arms the barrier with the bytes (copies
    // landing before it leave the count negative, which holds the phase open).
    int cp_len = 0, cp_src = 0, cp_dst = 0;  // floats; source offset within a plane
    bool cp_v = false;
    {
        const int c = nthr - 1 - tid;
        const int r = c / 3, u = c - 3 * (c / 3);
        int x = x0 >= 4 ? x0 - 4 : x0 - 4 + nx, p = 0;
        for (int run = 0; run < u && p < W; ++run) {
            p += min(W - p, nx - x);
            x = 0;
        }
        if (r < r0 + r1 && p < W) {
            cp_len = min(W - p, nx - x);
            cp_v = r >= r0;
            cp_src = (cp_v ? wy(y0 - 1 + r - r0) : wy(y0 - 2 + r)) * nx + x;
            cp_dst = (cp_v ? r - r0 : r) * W + p;
        }
    }
    auto issue = [&](int pl, bool with_v) {
        uint64_t* b = &bar[pl & 3];
        if (tid == 0) mbar_arrive_expect_tx(b, (unsigned)(s0 + (with_v ? s1 : 0)) * 4u);
        if (cp_len == 0 || (cp_v && !with_v)) return;
        const float* src = cp_v ? v_in + (size_t)wz(z0 - 3 + pl) * plane : phi_in + (size_t)wz(z0 - 2 + pl) * plane;
        float* dst = cp_v ? ringv + ((pl - 1) % 3) * s1 : ring0 + (pl & 3) * s0;
        bulk_g2s(dst + cp_dst, src + cp_src, (unsigned)cp_len * 4u, b);
    };
    issue(0, false);
    issue(1, false);
    int issued = 1;
    // This thread's level-1 sites: float4 column col of level-1 row row (level-0 row
    // row+1, global row y0-1+row); whole warps share a row.
    int off[ITEMS], go[ITEMS];
    bool on[ITEMS], out[ITEMS], first[ITEMS], last[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int q = tid + nthr * j;
        on[j] = q < r1 * nq;
        const int row = on[j] ? q / nq : 0, col = on[j] ? q - row * nq : 0;
        out[j] = on[j] && row >= 1 && row <= ty;
        first[j] = col == 0;
        last[j] = col == nq - 1;
        off[j] = row * W + 4 + 4 * col;  // in a level-1 or dphi slot; +W in a level-0 slot
        go[j] = (y0 - 1 + row) * nx + x0 + 4 * col;  // in a plane, for the output rows
    }
    // Halo columns of a sliced tile: thread h < 2 r1 owns level-1 row h/2 at column
    // x0-1 (h even) or x0+xw (h odd).
    const bool hal = !whole && tid < 2 * r1;
    const int hoff = (tid >> 1) * W + ((tid & 1) ? xw + 4 : 3);  // in a level-1 or dphi slot

    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 f0m[ITEMS], f0c[ITEMS];  // level 0 at planes j-1, j of the level-1 plane j
    float4 f1m[ITEMS], f1c[ITEMS];  // level 1 at planes k-1, k of the level-2 plane k
    float4 w1[ITEMS];               // level-1 dphi^{n+1/2} at plane k
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) f0m[j] = f0c[j] = f1m[j] = f1c[j] = w1[j] = z4;
    float h0m = 0.f, h0c = 0.f;  // level 0 at planes j-1, j of a halo lane's column

    for (int i = 0; i < nplanes; ++i) {
        const bool ok = mbar_wait(&bar[i & 3], (unsigned)(i >> 2) & 1u, err);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain4(bar, i, issued, err);
            return;
        }
        if (i + 2 < nplanes) issue(i + 2, i + 1 >= 1 && i + 1 <= zn + 2), issued = i + 2;
        const int j = i - 1;  // level-1 plane of this iteration
        const int k = i - 2;  // level-2 plane of this iteration
        const float* Pn = ring0 + (i & 3) * s0 + W;        // level-0 plane j+1, from row 1
        const float* Pj = ring0 + ((i + 3) & 3) * s0 + W;  // level-0 plane j, from row 1
        float4 f0p[ITEMS], f1p[ITEMS], w1n[ITEMS];
#pragma unroll
        for (int q = 0; q < ITEMS; ++q) {
            f0p[q] = on[q] ? lds4(Pn + off[q]) : z4;
            f1p[q] = w1n[q] = z4;
        }
        const float h0p = hal ? Pn[hoff] : 0.f;
        if (j >= 1 && j <= zn + 2) {
            float* L1 = ring1 + (j & 1) * s1;
            const float* V = ringv + (j % 3) * s1;
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                if (!on[q]) continue;  // warp-uniform
                const float* c0 = Pj + off[q];
                const float4 c = f0c[q];
                float left = __shfl_up_sync(0xffffffffu, c.w, 1);
                float right = __shfl_down_sync(0xffffffffu, c.x, 1);
                if (lane == 0) left = c0[-1];
                if (lane == 31) right = c0[4];
                float4 pn;
                float4 vv = lds4(V + off[q]);
                update4(c, left, right, lds4(c0 + W), lds4(c0 - W), f0p[q], f0m[q], vv, pn, k0, rc, true);
                *reinterpret_cast<float4*>(L1 + off[q]) = pn;
                if (whole) {  // the wrapped end columns of the row, for level 2's x neighbours
                    if (first[q]) L1[off[q] + xw] = pn.x;
                    if (last[q]) L1[off[q] - xw + 3] = pn.w;
                }
                f1p[q] = pn;
                w1n[q] = vv;
            }
            if (hal) {
                const float* c0 = Pj + hoff;
                float vv = V[hoff];
                L1[hoff] = update1(h0c, c0[1], c0[-1], c0[W], c0[-W], h0p, h0m, vv, k0, rc, true);
            }
        }
        if (k >= 2 && k <= zn + 1) {
            const float* L1 = ring1 + (k & 1) * s1;
            const size_t zo = (size_t)(z0 - 2 + k) * plane;
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                if (!out[q]) continue;  // warp-uniform
                const float* c1p = L1 + off[q];
                const float4 c = f1c[q];
                float left = __shfl_up_sync(0xffffffffu, c.w, 1);
                float right = __shfl_down_sync(0xffffffffu, c.x, 1);
                if (lane == 0) left = c1p[-1];
                if (lane == 31) right = c1p[4];
                float4 pn;
                float4 vv = w1[q];
                if (MID) {
                    stg4(phi_mid + zo + go[q], c);
                    stg4(v_mid + zo + go[q], vv);
                }
                update4(c, left, right, lds4(c1p + W), lds4(c1p - W), f1p[q], f1m[q], vv, pn, k1, rc, true);
                stg4(phi_out + zo + go[q], pn);
                stg4(v_out + zo + go[q], vv);
            }
        }
#pragma unroll
        for (int q = 0; q < ITEMS; ++q) {
            f0m[q] = f0c[q];
            f0c[q] = f0p[q];
            f1m[q] = f1c[q];
            f1c[q] = f1p[q];
            w1[q] = w1n[q];
        }
        h0m = h0c;
        h0c = h0p;
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

// NX > 0: the row width as a compile-time constant (the 4096-wide production box).
template <int ITEMS, int NX>
__global__ void __launch_bounds__(kTb2Threads, 1)
    k_step2d_t2(const float* __restrict__ phi_in, float* __restrict__ phi_out, const float* __restrict__ v_in,
                  float* __restrict__ v_out, int nx_, int ny, int cy, KickP p0, KickP p1, unsigned int* err)
{
    const int nx = NX > 0 ? NX : nx_;
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
    // iteration t waits for rows 2t, 2t+1 and issues the two rows iteration t + kR2Ahead waits for;
    // before the first iteration every slot of the ring is free, so the rows of the first
    // iterations are all in flight at once instead of one iteration's latency apart
    int issued = -1;
    if (tid == 0)
        for (int i = 0; i < kR2Slots0 && i < nload; ++i) issue(i), issued = i;

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

    // ring slots by rotation: level-0 row r sits in slot r mod kR2Slots0, level-1 row r in slot
    // r mod kR2Slots1; an iteration advances every row index by two
    auto level1 = [&](int jr, int sm, const float4* vin, float4* vout) {  // sm = (jr - 1) mod kR2Slots0
        if (jr < 1 || jr > yn + 2) return;
        const int sc = sm + 1 == kR2Slots0 ? 0 : sm + 1, sp = sc + 1 == kR2Slots0 ? 0 : sc + 1;
        const float* pm = ring0 + sm * nx;
        const float* pc = ring0 + sc * nx;
        const float* pp = ring0 + sp * nx;
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
            update4p<false>(c, left, right, lds4(pp + 4 * col[j]), ym, ym, ym, vv, pn, p0);
            *reinterpret_cast<float4*>(l1 + 4 * col[j]) = pn;
            vout[j] = vv;
        }
    };
    auto level2 = [&](int kr, const float4* vin) {
        if (kr < 2 || kr > yn + 1) return;
        const int sc = kr % kR2Slots1, sm = sc == 0 ? kR2Slots1 - 1 : sc - 1, sp = sc + 1 == kR2Slots1 ? 0 : sc + 1;
        const float* pm = ring1 + sm * nx;
        const float* pc = ring1 + sc * nx;
        const float* pp = ring1 + sp * nx;
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
            update4p<false>(c, left, right, lds4(pp + 4 * col[j]), ym, ym, ym, vv, pn, p1);
            stg4(phi_out + ro + 4 * col[j], pn);
            stg4(v_out + ro + 4 * col[j], vv);
        }
    };

    const int tmax = (yn + 5) / 2;  // last iteration: level-2 row 2t-3 or 2t-4 reaches yn+1
    int s0 = kR2Slots0 - 2;         // (2t - 2) mod kR2Slots0: slot of level-1 row 2t-1's row below
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
            for (int i = max(issued + 1, 2 * (t + kR2Ahead)); i <= 2 * (t + kR2Ahead) + 1 && i < nload; ++i)
                issue(i), issued = i;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) va0[j] = vb0[j], va1[j] = vb1[j];
        load_v(2 * t + 1, vb0);  // for iteration t+1: rows 2t+1, 2t+2
        load_v(2 * t + 2, vb1);
        float4 no[ITEMS], ne[ITEMS];
        const int s1 = s0 + 1 == kR2Slots0 ? 0 : s0 + 1;  // (2t - 1) mod kR2Slots0
        level1(2 * t - 1, s0, va0, no);
        level1(2 * t, s1, va1, ne);
        level2(2 * t - 4, e0);
        level2(2 * t - 3, o0);
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            e0[j] = e1[j];
            e1[j] = ne[j];
            o0[j] = no[j];
        }
        s0 += 2;
        if (s0 >= kR2Slots0) s0 -= kR2Slots0;
    }
}

size_t smem2d_t2(int nx) { return 128 + (kR2Slots0 + kR2Slots1) * (size_t)nx * sizeof(float); }

constexpr size_t kTbSmemMax = 160 * 1024;

// Tile of a 3D two-step pass: xw columns (128 for x sides up to 256, four CTAs per SM;
// else the widest 128-multiple up to 256 that divides nx, two CTAs per SM: several CTAs
// per SM hide each other's barrier waits; measured 38.2 against 41.2 us per step at
// 256^3 for 128-column tiles, 1.72 against 1.67 ms at 1024^3) by ty rows (the largest divisor of ny whose level-1 plane takes at most
// kTbItems float4 per thread of a kTbThreads CTA; a sliced tile has one halo lane of
// warp 0 per level-1 row and side).
struct Tile3 {
    int xw, ty, threads;
    size_t smem;
};

bool plan3(const Geo& g, Tile3* t)
{
    if (g.nx % 128 != 0 || g.nz < 3) return false;
    int xw = 0;
    for (int w = g.nx <= 256 ? 128 : 256; w >= 128 && !xw; w -= 128)
        if (g.nx % w == 0) xw = w;
    const int nq = xw / 4;
    const int tymax = xw == g.nx ? 28 : kTbMaxTy;
    int ty = 0;
    for (int c = tymax < g.ny ? tymax : g.ny; c >= 1 && !ty; --c)
        if (g.ny % c == 0 && (c + 2) * nq <= kTbItems * kTbThreads) ty = c;
    if (!ty) return false;
    t->xw = xw;
    t->ty = ty;
    t->threads = (((ty + 2) * nq + kTbItems - 1) / kTbItems + 31) / 32 * 32;
    t->smem = 128 + (size_t)(4 * (ty + 4) + 5 * (ty + 2)) * (xw + 8) * sizeof(float);
    // one thread per copy task (3 runs of each of the 2 ty + 6 staged rows)
    return t->smem <= kTbSmemMax && t->threads >= 3 * (2 * ty + 6);
}

template <bool MID>
cudaError_t launch3(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out, float* phi_mid,
                    float* v_mid, KickF k0, KickF k1, RunConst<float> rc, unsigned int* err, cudaStream_t st)
{
    Tile3 t;
    if (!plan3(g, &t)) return cudaErrorInvalidValue;
    // the common tiles (256 x 8, 128 x 8) have their own instantiations with every size known
    const void* fn = t.xw == 256 ? (t.ty == 8 ? (const void*)k_step3d_t2<kTbItems, 256, 8, MID>
                                              : (const void*)k_step3d_t2<kTbItems, 256, 0, MID>)
                                 : (t.ty == 8 ? (const void*)k_step3d_t2<kTbItems, 128, 8, MID>
                                              : (const void*)k_step3d_t2<kTbItems, 128, 0, MID>);
    static std::atomic<unsigned long long> attr[4];
    {
        const int which = t.xw == 256 ? (t.ty == 8 ? 0 : 1) : (t.ty == 8 ? 3 : 2);
        const cudaError_t e = smem_limit_once(attr[which], fn, (int)kTbSmemMax);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, t.threads, t.smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int slots = per_sm * sm_count_current();
    const int tiles = (g.nx / t.xw) * (g.ny / t.ty);
    // z-chunks: whole waves of resident CTAs, balanced against the four halo planes per chunk
    int best = 1;
    double best_score = -1.0;
    for (int nc = 1; nc <= g.nz / 8 || nc == 1; ++nc) {
        const int c = (g.nz + nc - 1) / nc, n = (g.nz + c - 1) / c;
        const long long blocks = (long long)tiles * n;
        const long long waves = (blocks + slots - 1) / slots;
        const double score = (double)blocks / (double)(waves * slots) * c / (c + 4.0) * (waves >= 2 ? 1.0 : 0.9);
        if (score > best_score + 1e-9) best_score = score, best = n;
        if (nc > 4096) break;
    }
    const int cz = (g.nz + best - 1) / best;
    const long long blocks = (long long)tiles * ((g.nz + cz - 1) / cz);
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    if (t.xw == 256 && t.ty == 8)
        k_step3d_t2<kTbItems, 256, 8, MID><<<(unsigned)blocks, t.threads, t.smem, st>>>(
            phi_in, phi_out, v_in, v_out, phi_mid, v_mid, g.nx, g.ny, g.nz, t.ty, cz, k0, k1, rc, err);
    else if (t.xw == 256)
        k_step3d_t2<kTbItems, 256, 0, MID><<<(unsigned)blocks, t.threads, t.smem, st>>>(
            phi_in, phi_out, v_in, v_out, phi_mid, v_mid, g.nx, g.ny, g.nz, t.ty, cz, k0, k1, rc, err);
    else if (t.ty == 8)
        k_step3d_t2<kTbItems, 128, 8, MID><<<(unsigned)blocks, t.threads, t.smem, st>>>(
            phi_in, phi_out, v_in, v_out, phi_mid, v_mid, g.nx, g.ny, g.nz, t.ty, cz, k0, k1, rc, err);
    else
        k_step3d_t2<kTbItems, 128, 0, MID><<<(unsigned)blocks, t.threads, t.smem, st>>>(
            phi_in, phi_out, v_in, v_out, phi_mid, v_mid, g.nx, g.ny, g.nz, t.ty, cz, k0, k1, rc, err);
    return cudaGetLastError();
}

}  // namespace


bool tblock_ok(const Geo& g, int precision)
{
    if (precision != PRS_FP32 || g.nx % 128 != 0) return false;
    if (g.dims == 2) return g.nx <= 2 * kTb2Threads * 4;  // at most two float4 per thread of a row
    Tile3 t;
    return plan3(g, &t);
}

int tblock3_rows(const Geo& g)
{
    Tile3 t;
    return g.dims == 3 && plan3(g, &t) ? t.ty : 0;
}

cudaError_t launch_step_t2(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out,
                           KickF k0, KickF k1, RunConst<float> rc, unsigned int* err, cudaStream_t st,
                           float* phi_mid, float* v_mid)
{
    if (g.dims == 2) {
        if (phi_mid || v_mid) return cudaErrorNotSupported;
        const KickP p0 = kick_packed(k0, rc.deta), p1 = kick_packed(k1, rc.deta);
        static std::atomic<unsigned long long> attr1{0}, attr2{0};
        const size_t sm = smem2d_t2(g.nx);
        const int sms = sm_count_current();
        const int cy = (g.ny + sms - 1) / sms;
        const int blocks = (g.ny + cy - 1) / cy;
        if (g.nx / 4 > kTb2Threads) {
            const cudaError_t e =
                smem_limit_once(attr2, (const void*)k_step2d_t2<2, 0>, (int)smem2d_t2(8 * kTb2Threads));
            if (e != cudaSuccess) return e;
            static std::atomic<unsigned long long> attr4{0};
            const cudaError_t e4 = smem_limit_once(attr4, (const void*)k_step2d_t2<2, 4096>, (int)smem2d_t2(4096));
            if (e4 != cudaSuccess) return e4;
            if (g.nx == 4096)
                k_step2d_t2<2, 4096>
                    <<<blocks, kTb2Threads, sm, st>>>(phi_in, phi_out, v_in, v_out, g.nx, g.ny, cy, p0, p1, err);
            else
                k_step2d_t2<2, 0>
                    <<<blocks, kTb2Threads, sm, st>>>(phi_in, phi_out, v_in, v_out, g.nx, g.ny, cy, p0, p1, err);
        } else {
            const cudaError_t e =
                smem_limit_once(attr1, (const void*)k_step2d_t2<1, 0>, (int)smem2d_t2(4 * kTb2Threads));
            if (e != cudaSuccess) return e;
            k_step2d_t2<1, 0>
                <<<blocks, kTb2Threads, sm, st>>>(phi_in, phi_out, v_in, v_out, g.nx, g.ny, cy, p0, p1, err);
        }
        return cudaGetLastError();
    }
    if ((phi_mid == nullptr) != (v_mid == nullptr)) return cudaErrorInvalidValue;
    if (t2tma_ok(g)) {  // the production tile: planes staged by tensor copies
        const cudaError_t e = launch_step_t2_tma(g, phi_in, phi_out, v_in, v_out, k0, k1, rc, err, st, phi_mid, v_mid);
        if (e != cudaErrorNotSupported) return e;
    }
    if (phi_mid) return launch3<true>(g, phi_in, phi_out, v_in, v_out, phi_mid, v_mid, k0, k1, rc, err, st);
    return launch3<false>(g, phi_in, phi_out, v_in, v_out, nullptr, nullptr, k0, k1, rc, err, st);
}

}  // namespace prs

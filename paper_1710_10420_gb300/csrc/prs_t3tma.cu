// prs_t3tma.cu -- three leapfrog steps (Eqs. 3-5) per pass over HBM, FP32 3D, with the
// planes staged by TMA tensor copies.
//
// A CTA owns a tile of XW columns x 8 rows and a chunk of z-planes and marches along z
// through three levels, each one plane behind the one before:
//   level 1 (step n)   on 12 rows (y0-2 .. y0+9) and columns x0-2 .. x0+XW+1,
//   level 2 (step n+1) on 10 rows (y0-1 .. y0+8) and columns x0-1 .. x0+XW,
//   level 3 (step n+2) on the 8 output rows and XW columns,
// so a site of step n+2 depends only on staged sites of phi^n (a radius of three in x, y
// and z), and phi and dphi cross HBM once per three steps: 16 B per site per pass.
//
// Per plane one thread issues the tensor copies of phi^n on 14 rows (y0-3 .. y0+10) with
// its two 4-column x-halo boxes, and of dphi^{n-1/2} on level 1's 12 rows with their halo
// boxes, two planes ahead into a 4-slot and a 3-slot ring (one mbarrier per phi slot).
// Levels 1 and 2 write their planes into two-slot rings of rows XW+8 floats wide (columns
// x0-4 .. x0+XW+3); the next level reads x and y neighbours there.  A thread owns one
// float4 column of one level-1 row and the same float4 at levels 2 and 3 (rows are whole
// warps, so a level's participation is warp-uniform); in registers it keeps only what
// has left the rings: level 0 at plane j-1, level 1 at k-1, level 2 at l-1, and the dphi
// that level 1 and level 2 hand down to the next level at the same site.  The level-1 and
// level-2 columns outside the tile (two and one on each side) are single sites computed by
// 48 halo lanes on the two warps of rows that only run level 1.  One barrier per plane.
// dphi goes out of place (level 1 reads it on rows and planes of the neighbouring tiles).
//
// Instruction count is what bounds a pass that moves this few bytes per update, so the
// plane loop is specialised: the six iterations that fill the pipeline run with the later
// levels compiled out, and the steady-state body tests no plane ranges; the kick constants
// arrive packed as f32x2 operands; the copy context sits in shared memory (only thread 0
// reads it); x-edge values are loaded by the two lanes that use them.  At 512^3 that took
// the pass from 495 M to 387 M warp instructions (and shared-memory bank conflicts from
// 22.5 M to 9.3 M).
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>

#include "prs_internal.h"
#include "prs_ptx.cuh"
#include "prs_tile.cuh"
#include "prs_tmap.h"

namespace prs {

namespace {

constexpr int kTY = 8;
constexpr int kR0 = kTY + 6;  // staged phi^n rows: y0-3 .. y0+10
constexpr int kR1 = kTY + 4;  // level-1 rows (and staged dphi rows): y0-2 .. y0+9
constexpr int kHalo = 48;     // level-1 halo sites per plane: 12 rows x 4 columns

template <int XW>
struct T3 {
    static constexpr int F = XW / 4;            // float4 per row
    static constexpr int kThreads = kR1 * F;    // one level-1 float4 per thread
    static constexpr int kW = XW + 8;           // level-1/2 ring row: columns x0-4 .. x0+XW+3
    // phi slot (floats): main box [kR0][XW], left halo [kR0][4], right halo [kR0][4], each part
    // at a 128-byte boundary; dphi slot: main box [kR1][XW], halos [kR1][4]
    static constexpr int kHL0 = kR0 * XW, kHR0 = kHL0 + 64, kS0 = kHR0 + 64;
    static constexpr int kHLV = kR1 * XW, kHRV = kHLV + 64, kSV = kHRV + 64;
    static constexpr int kS1 = kR1 * kW;        // level-1 and level-2 slots (level 2 uses rows 1..10)
    static constexpr size_t kSmem = 128 + (size_t)(4 * kS0 + 3 * kSV + 4 * kS1) * sizeof(float);
    static constexpr unsigned kBytesPhi = (kR0 * XW + 2 * kR0 * 4) * 4u;
    static constexpr unsigned kBytesV = (kR1 * XW + 2 * kR1 * 4) * 4u;
    static constexpr int kMinBlocks = XW == 128 ? 2 : 1;
    static_assert(F % 32 == 0, "rows are whole warps");
    static_assert(kS0 % 32 == 0 && kSV % 32 == 0 && kHL0 % 32 == 0 && kHLV % 32 == 0 && kS1 % 4 == 0,
                  "128-byte aligned tensor-copy parts");
    static_assert(kThreads >= kHalo + 64, "halo lanes and the wrap tiles' row copies fit the CTA");
};

// Tensor maps of one pass (boxes one plane deep): phi^n XW x {14, 11, 3} and 4 x 14; dphi
// XW x {12, 10, 2} and 4 x 12.  The tiles at the ends of y split their boxes at the wrap.
struct T3Maps {
    CUtensorMap phi14, phi11, phi3, phih, v12, v10, v2, vh;
};

static __device__ __noinline__ void drain3(uint64_t* bar, int from, int issued, unsigned int* err)
{
    for (int i = from; i <= issued; ++i) mbar_wait(&bar[i & 3], (unsigned)(i >> 2) & 1u, err);
}

// What the copies of a plane need.  Only thread 0 (and, on the tiles at the ends of y, the
// last two warps) issue copies, so this lives in shared memory rather than in every thread's
// registers.
struct Ctx3 {
    const float* phi_in;
    const float* v_in;
    size_t plane;
    int nx, ny, nz, x0, y0, z0, zn, xl, xr, ywrap;  // ywrap: 0, -1 (top tile), +1 (bottom tile)
};

// The CTA's shared memory: mbarriers and the copy context, then the rings.
struct Smem3 {
    uint64_t bar[4];
    Ctx3 c;
};
static_assert(sizeof(Smem3) <= 128, "header fits the first 128 bytes");

extern __shared__ __align__(128) unsigned char t3_smem[];

__device__ __forceinline__ Smem3* hdr3() { return reinterpret_cast<Smem3*>(t3_smem); }

// ring0 (4 phi slots), ringv (3 dphi slots), ring1 and ring2 (2 slots each), after the header
template <int XW>
struct Rings3 {
    using S = T3<XW>;
    static __device__ __forceinline__ float* r0() { return reinterpret_cast<float*>(t3_smem + 128); }
    static __device__ __forceinline__ float* rv() { return r0() + 4 * S::kS0; }
    static __device__ __forceinline__ float* r1() { return rv() + 3 * S::kSV; }
    static __device__ __forceinline__ float* r2() { return r1() + 2 * S::kS1; }
};

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Stage level-0 plane pl (global z0-3+pl) and, with with_v, the dphi of level-1 plane pl-1
// into dphi slot vs = (pl-1) mod 3.  Called by every thread; thread 0 issues the tensor copies.
template <int XW>
__device__ __forceinline__ void issue3(const T3Maps& m, int tid, int pl, bool with_v, int vs)
{
    using S = T3<XW>;
    using R = Rings3<XW>;
    const Ctx3& c = hdr3()->c;
    uint64_t* b = &hdr3()->bar[pl & 3];
    if (tid == 0) {
        const int zg = wrapi(c.z0 - 3 + pl, c.nz), zvg = wrapi(c.z0 - 4 + pl, c.nz);
        float* d0 = R::r0() + (pl & 3) * S::kS0;
        float* dv = R::rv() + vs * S::kSV;
        mbar_arrive_expect_tx(b, S::kBytesPhi + (with_v ? S::kBytesV : 0u));
        if (c.ywrap == 0) {
            tma_load3(d0, &m.phi14, c.x0, c.y0 - 3, zg, b);
            tma_load3(d0 + S::kHL0, &m.phih, c.xl, c.y0 - 3, zg, b);
            tma_load3(d0 + S::kHR0, &m.phih, c.xr, c.y0 - 3, zg, b);
            if (with_v) {
                tma_load3(dv, &m.v12, c.x0, c.y0 - 2, zvg, b);
                tma_load3(dv + S::kHLV, &m.vh, c.xl, c.y0 - 2, zvg, b);
                tma_load3(dv + S::kHRV, &m.vh, c.xr, c.y0 - 2, zvg, b);
            }
        } else if (c.ywrap < 0) {  // y0 = 0: rows ny-3 .. ny-1, then 0 .. 10
            tma_load3(d0, &m.phi3, c.x0, c.ny - 3, zg, b);
            tma_load3(d0 + 3 * XW, &m.phi11, c.x0, 0, zg, b);
            if (with_v) {
                tma_load3(dv, &m.v2, c.x0, c.ny - 2, zvg, b);
                tma_load3(dv + 2 * XW, &m.v10, c.x0, 0, zvg, b);
            }
        } else {  // y0 = ny-8: rows ny-11 .. ny-1, then 0 .. 2
            tma_load3(d0, &m.phi11, c.x0, c.ny - 11, zg, b);
            tma_load3(d0 + 11 * XW, &m.phi3, c.x0, 0, zg, b);
            if (with_v) {
                tma_load3(dv, &m.v10, c.x0, c.ny - 10, zvg, b);
                tma_load3(dv + 10 * XW, &m.v2, c.x0, 0, zvg, b);
            }
        }
    }
    if (tid >= S::kThreads - 64 && c.ywrap != 0) {
        // the wrap tiles' halo columns row by row (16 bytes each) on the last two warps: task
        // t < 2 kR0 is phi row t/2, side t%2; then 2 kR1 dphi tasks
        const int zg = wrapi(c.z0 - 3 + pl, c.nz), zvg = wrapi(c.z0 - 4 + pl, c.nz);
        float* d0 = R::r0() + (pl & 3) * S::kS0;
        float* dv = R::rv() + vs * S::kSV;
        const int t = tid - (S::kThreads - 64);
        const bool isv = t >= 2 * kR0;
        if (t < 2 * (kR0 + kR1) && (!isv || with_v)) {
            const int tt = isv ? t - 2 * kR0 : t, r = tt >> 1, side = tt & 1;
            const int y = wrapi(isv ? c.y0 - 2 + r : c.y0 - 3 + r, c.ny);
            const float* src = (isv ? c.v_in + (size_t)zvg * c.plane : c.phi_in + (size_t)zg * c.plane) +
                               (size_t)y * c.nx + (side ? c.xr : c.xl);
            float* dst = (isv ? dv + (side ? S::kHRV : S::kHLV) : d0 + (side ? S::kHR0 : S::kHL0)) + 4 * r;
            bulk_g2s(dst, src, 16u, b);
        }
    }
}

__device__ __forceinline__ void xnb(float4 cc, float e, int lane, float& left, float& right)
{
    const float su = __shfl_up_sync(0xffffffffu, cc.w, 1), sd = __shfl_down_sync(0xffffffffu, cc.x, 1);
    left = lane == 0 ? e : su;
    right = lane == 31 ? e : sd;
}

// Per-thread offsets and roles.
struct Lane3 {
    int tid, lane, o0, o1, e0;
    bool edge, lv2, lv3, hal, hal2;
    unsigned hx;  // halo lane: its x neighbours' offsets in the phi slot, hxm | hxp << 16
    int hc, hv, ho;
};

// What a thread carries from plane to plane: level 0 at plane j-1 (am), level 1 at k-1 (bm),
// level 2 at l-1 (cm), the dphi level 1 and level 2 hand to the next level (w1, w2), and the
// halo lane's counterparts.  (Two sets alternating with the plane parity, so that a loop
// unrolled by two rotates them by renaming, need more than the 80 registers a thread of
// two 384-thread CTAs per SM has: they spilled and ran slower.)
struct Queue3 {
    float4 am, bm, cm, w1, w2;
    float hm, hb, hw;
};

// Plane iteration i with levels 1..LV active (LV = 3 in the steady state, whose loop body
// then tests no plane ranges; the first six iterations fill the pipeline).  vs = (i-1) mod 3,
// the dphi slot of level-1 plane j = i-1.  po, vo: the outputs at level-3 plane l = i-3, this
// thread's site.  Returns false when a wait gave up.
template <int XW, int LV>
__device__ __forceinline__ bool t3_iter(const T3Maps& m, const Lane3& t, int i, int nplanes, int vs, float* po,
                                        float* vo, const KickP& k0, const KickP& k1, const KickP& k2, Queue3& q,
                                        unsigned int* err)
{
    using S = T3<XW>;
    using R = Rings3<XW>;
    const int P = i & 1;
    const bool ok = mbar_wait(&hdr3()->bar[i & 3], (unsigned)(i >> 2) & 1u, err);
    if (__syncthreads_or(!ok)) {
        if (t.tid == 0) drain3(hdr3()->bar, i, min(i + 1, nplanes - 1), err);  // planes issued so far
        return false;
    }
    if (i + 2 < nplanes) issue3<XW>(m, t.tid, i + 2, true, vs == 0 ? 2 : vs - 1);
    const float* Ln = R::r0() + (i & 3) * S::kS0;        // level 0 at plane j+1
    const float* Lj = R::r0() + ((i + 3) & 3) * S::kS0;  // level 0 at plane j
    float4 pn, qn, w1n, w2n;
    float hpn = 0.f, hwn = 0.f;
    if (LV >= 1) {  // level 1 (step n) at plane j: level 0 at j-1 (am), j (ring), j+1 (ring)
        float* L1 = R::r1() + (P ^ 1) * S::kS1;
        const float* V = R::rv() + vs * S::kSV;
        const float4 a = lds4(Lj + t.o0);
        float e = 0.f, left, right;
        if (t.edge) e = Lj[t.e0];
        xnb(a, e, t.lane, left, right);
        float4 v = lds4(V + t.o0 - XW);
        update4p(a, left, right, lds4(Lj + t.o0 + XW), lds4(Lj + t.o0 - XW), lds4(Ln + t.o0), q.am, v, pn, k0);
        *reinterpret_cast<float4*>(L1 + t.o1) = pn;
        q.am = a;
        w1n = v;
        if (t.hal) {
            const float hcen = Lj[t.hc];
            float hv = V[t.hv];
            hpn = update1(hcen, Lj[t.hx >> 16], Lj[t.hx & 0xffffu], Lj[t.hc + 4], Lj[t.hc - 4], Ln[t.hc], q.hm, hv,
                          kick_scalar(k0), deta_only(k0), true);
            L1[t.ho] = hpn;
            q.hm = hcen;
            hwn = hv;
        }
    }
    if (LV >= 2) {  // level 2 (step n+1) at plane k: level 1 at k-1 (bm), k (ring), k+1 (pn)
        const float* L1k = R::r1() + P * S::kS1;
        float* L2 = R::r2() + P * S::kS1;
        if (t.lv2) {
            const float4 b = lds4(L1k + t.o1);
            float e = 0.f, left, right;
            if (t.edge) e = L1k[t.o1 + (t.lane == 0 ? -1 : 4)];
            xnb(b, e, t.lane, left, right);
            float4 v = q.w1;
            update4p(b, left, right, lds4(L1k + t.o1 + S::kW), lds4(L1k + t.o1 - S::kW), pn, q.bm, v, qn, k1);
            *reinterpret_cast<float4*>(L2 + t.o1) = qn;
            q.bm = b;
            w2n = v;
        }
        if (t.hal2) {
            const float hcen = L1k[t.ho];
            float hv = q.hw;
            L2[t.ho] = update1(hcen, L1k[t.ho + 1], L1k[t.ho - 1], L1k[t.ho + S::kW], L1k[t.ho - S::kW], hpn, q.hb,
                               hv, kick_scalar(k1), deta_only(k1), true);
            q.hb = hcen;
        }
    }
    if (LV >= 3 && t.lv3) {  // level 3 (step n+2) at plane l: level 2 at l-1 (cm), l (ring), l+1 (qn)
        const float* L2l = R::r2() + (P ^ 1) * S::kS1;
        const float4 d = lds4(L2l + t.o1);
        float e = 0.f, left, right;
        if (t.edge) e = L2l[t.o1 + (t.lane == 0 ? -1 : 4)];
        xnb(d, e, t.lane, left, right);
        float4 v = q.w2, out;
        update4p(d, left, right, lds4(L2l + t.o1 + S::kW), lds4(L2l + t.o1 - S::kW), qn, q.cm, v, out, k2);
        stg4(po, out);
        stg4(vo, v);
        q.cm = d;
    }
    // the dphi handed down reaches the next level in the next iteration
    if (LV >= 1) q.w1 = w1n;
    if (LV >= 1 && t.hal) q.hw = hwn;
    if (LV >= 2 && t.lv2) q.w2 = w2n;
    return true;
}

template <int XW>
__global__ void __launch_bounds__(T3<XW>::kThreads, T3<XW>::kMinBlocks)
    k_step3d_t3tma(const __grid_constant__ T3Maps maps, const float* __restrict__ phi_in,
                   float* __restrict__ phi_out, const float* __restrict__ v_in, float* __restrict__ v_out, int nx,
                   int ny, int nz, int cz, KickP k0, KickP k1, KickP k2, unsigned int* err)
{
    using S = T3<XW>;
    using R = Rings3<XW>;
    const int nxt = nx / XW, ytiles = ny / kTY;
    const int x0 = (blockIdx.x % nxt) * XW, y0 = (blockIdx.x / nxt % ytiles) * kTY, z0 = blockIdx.x / nxt / ytiles * cz;
    const int zn = min(cz, nz - z0);
    const int nplanes = zn + 6;  // level-0 local planes 0 .. zn+5 = global z0-3 .. z0+zn+2
    const size_t plane = (size_t)nx * ny;

    // this thread's float4: level-1 row r (global y0-2+r), column x0+4 col
    Lane3 t;
    t.tid = threadIdx.x;
    t.lane = t.tid & 31;
    const int r = t.tid / S::F, col = t.tid % S::F;
    t.o0 = (r + 1) * XW + 4 * col;   // phi slot (phi row r+1); dphi slot at o0 - XW
    t.o1 = r * S::kW + 4 + 4 * col;  // level-1/2 slots
    t.e0 = t.lane == 0 ? (col == 0 ? S::kHL0 + (r + 1) * 4 + 3 : t.o0 - 1)
                       : (col == S::F - 1 ? S::kHR0 + (r + 1) * 4 : t.o0 + 4);
    t.edge = t.lane == 0 || t.lane == 31;
    t.lv2 = r >= 1 && r <= kTY + 2;  // warp-uniform
    t.lv3 = r >= 2 && r <= kTY + 1;

    // halo lanes: the first warp (row 0) and the last 16 lanes of the last warp (row 11), both
    // level-1-only rows.  Halo site h: row h/4, column x0-2, x0-1, x0+XW, x0+XW+1 for h%4 = 0..3;
    // the two inner columns of rows 1..10 also run level 2.
    const int h = t.tid < 32 ? t.tid : (t.tid >= S::kThreads - (kHalo - 32) ? t.tid - (S::kThreads - kHalo) : -1);
    t.hal = h >= 0;
    t.hc = 0, t.hx = 0, t.hv = 0, t.ho = 4;
    t.hal2 = false;
    if (t.hal) {
        const int hr = h >> 2, w = h & 3;
        const int base = w < 2 ? S::kHL0 + (hr + 1) * 4 + 2 + w : S::kHR0 + (hr + 1) * 4 + (w - 2);
        t.hc = base;
        const unsigned hxm = w == 2 ? (hr + 1) * XW + XW - 1 : base - 1, hxp = w == 1 ? (hr + 1) * XW : base + 1;
        t.hx = hxm | hxp << 16;
        t.hv = w < 2 ? S::kHLV + hr * 4 + 2 + w : S::kHRV + hr * 4 + (w - 2);
        t.ho = hr * S::kW + (w < 2 ? 2 + w : XW + 4 + (w - 2));
        t.hal2 = (w == 1 || w == 2) && hr >= 1 && hr <= kTY + 2;
    }

    if (t.tid == 0) {
        Smem3* sm = hdr3();
        sm->c = Ctx3{phi_in, v_in, plane, nx, ny, nz, x0, y0, z0, zn, x0 >= 4 ? x0 - 4 : x0 - 4 + nx,
                     x0 + XW < nx ? x0 + XW : 0, y0 == 0 ? -1 : (y0 + kTY == ny ? 1 : 0)};
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(&sm->bar[i], 1);
        mbar_fence_init();
    }
    __syncthreads();
    issue3<XW>(maps, t.tid, 0, false, 0);
    issue3<XW>(maps, t.tid, 1, false, 0);

    Queue3 q;
    const size_t go = (size_t)z0 * plane + (size_t)(y0 - 2 + r) * nx + x0 + 4 * col;  // level-3 plane 3 = z0
    float* po = phi_out + go;
    float* vo = v_out + go;
    // pipeline fill: iterations 0, 1 only stage planes; level 1 starts at 2, level 2 at 4,
    // level 3 at 6; the queues' first planes are read where they are first needed
    if (!t3_iter<XW, 0>(maps, t, 0, nplanes, 2, po, vo, k0, k1, k2, q, err)) return;
    if (!t3_iter<XW, 0>(maps, t, 1, nplanes, 0, po, vo, k0, k1, k2, q, err)) return;
    q.am = lds4(R::r0() + t.o0);  // level 0 at plane 0 (slot 0)
    if (t.hal) q.hm = R::r0()[t.hc];
    if (!t3_iter<XW, 1>(maps, t, 2, nplanes, 1, po, vo, k0, k1, k2, q, err)) return;
    if (!t3_iter<XW, 1>(maps, t, 3, nplanes, 2, po, vo, k0, k1, k2, q, err)) return;
    if (t.lv2) q.bm = lds4(R::r1() + S::kS1 + t.o1);  // level 1 at plane 1 (slot 1)
    if (t.hal2) q.hb = R::r1()[S::kS1 + t.ho];
    if (!t3_iter<XW, 2>(maps, t, 4, nplanes, 0, po, vo, k0, k1, k2, q, err)) return;
    if (!t3_iter<XW, 2>(maps, t, 5, nplanes, 1, po, vo, k0, k1, k2, q, err)) return;
    if (t.lv3) q.cm = lds4(R::r2() + t.o1);  // level 2 at plane 2 (slot 0)
    int vs = 2;                                 // (i-1) mod 3 at i = 6
    for (int i = 6; i < nplanes; ++i) {
        if (!t3_iter<XW, 3>(maps, t, i, nplanes, vs, po, vo, k0, k1, k2, q, err)) return;
        po += plane;
        vo += plane;
        vs = vs == 2 ? 0 : vs + 1;
    }
}

template <int XW>
bool encode_maps(T3Maps& m, const float* phi_in, const float* v_in, const Geo& g)
{
    const EncodeTiled f = tmap_encoder();
    if (!f) return false;
    return tmap_encode(f, &m.phi14, phi_in, g, XW, kR0) && tmap_encode(f, &m.phi11, phi_in, g, XW, 11) &&
           tmap_encode(f, &m.phi3, phi_in, g, XW, 3) && tmap_encode(f, &m.phih, phi_in, g, 4, kR0) &&
           tmap_encode(f, &m.v12, v_in, g, XW, kR1) && tmap_encode(f, &m.v10, v_in, g, XW, 10) &&
           tmap_encode(f, &m.v2, v_in, g, XW, 2) && tmap_encode(f, &m.vh, v_in, g, 4, kR1);
}

template <int XW>
cudaError_t launch_xw(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out, KickP k0,
                      KickP k1, KickP k2, unsigned int* err, cudaStream_t st)
{
    using S = T3<XW>;
    T3Maps m;
    if (!encode_maps<XW>(m, phi_in, v_in, g)) return cudaErrorNotSupported;
    const void* fn = (const void*)k_step3d_t3tma<XW>;
    static std::atomic<unsigned long long> attr;
    cudaError_t e = smem_limit_once(attr, fn, (int)S::kSmem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, S::kThreads, S::kSmem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int slots = per_sm * sm_count_current();
    const int tiles = (g.nx / XW) * (g.ny / kTY);
    // z-chunks: whole waves of resident CTAs, balanced against the six halo planes per chunk
    int best = 1;
    double best_score = -1.0;
    for (int nc = 1; nc <= g.nz / 12 || nc == 1; ++nc) {
        const int cc = (g.nz + nc - 1) / nc, n = (g.nz + cc - 1) / cc;
        const long long blocks = (long long)tiles * n;
        const long long waves = (blocks + slots - 1) / slots;
        const double score = (double)blocks / (double)(waves * slots) * cc / (cc + 6.0) * (waves >= 2 ? 1.0 : 0.9);
        if (score > best_score + 1e-9) best_score = score, best = n;
        if (nc > 4096) break;
    }
    const int cz = (g.nz + best - 1) / best;
    const long long blocks = (long long)tiles * ((g.nz + cz - 1) / cz);
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    k_step3d_t3tma<XW><<<(unsigned)blocks, S::kThreads, S::kSmem, st>>>(m, phi_in, phi_out, v_in, v_out, g.nx, g.ny,
                                                                       g.nz, cz, k0, k1, k2, err);
    return cudaGetLastError();
}

// Tile width for this box: 128 columns (two 384-thread CTAs per SM) wherever the x side is a
// multiple of 128.  The 256-column tile (one 768-thread CTA per SM, the same redundancy in y,
// half the x-halo work) measured slower at 1024^3: 1.49 against 1.43 ms per step.
int t3_width(const Geo& g)
{
    if (g.dims != 3 || g.ny % kTY != 0 || g.ny < 2 * kTY || g.nz < 3) return 0;
    return g.nx % 128 == 0 ? 128 : 0;
}

}  // namespace

// The three-step pass applies to FP32 3D boxes with an x side that is a multiple of 128, a
// y side that is a multiple of 8 and at least 16, and a z side of at least 3.
bool t3tma_ok(const Geo& g) { return t3_width(g) != 0; }

cudaError_t launch_step_t3_tma(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out,
                               KickF k0, KickF k1, KickF k2, RunConst<float> rc, unsigned int* err, cudaStream_t st,
                               int width)
{
    const int xw = width ? width : t3_width(g);
    if (!t3tma_ok(g) || (xw != 128 && xw != 256) || g.nx % xw != 0) return cudaErrorNotSupported;
    if ((((uintptr_t)phi_in | (uintptr_t)v_in) & 15u) != 0) return cudaErrorNotSupported;
    const KickP p0 = kick_packed(k0, rc.deta), p1 = kick_packed(k1, rc.deta), p2 = kick_packed(k2, rc.deta);
    return xw == 256 ? launch_xw<256>(g, phi_in, phi_out, v_in, v_out, p0, p1, p2, err, st)
                     : launch_xw<128>(g, phi_in, phi_out, v_in, v_out, p0, p1, p2, err, st);
}

}  // namespace prs

// prs_t2tma.cu -- two leapfrog steps (Eqs. 3-5) per pass over HBM, FP32 3D, on the
// production tile of 256 columns x 8 rows, with the planes staged by TMA tensor copies.
//
// The pass is that of k_step3d_t2 (prs_tblock.cu): a CTA marches along z through its
// tile's chunk of planes; level 1 (step n) runs on the tile's 10 rows (8 output rows and
// the y halo rows) one plane ahead of level 2 (step n+1) on the 8 output rows; one
// barrier per plane.  What differs is how a plane arrives.  A tensor map describes each
// field as a 3D array (x, y, z), and one thread issues a handful of tensor copies per
// plane: the 256 x 12 box of phi^n (rows y0-2 .. y0+9), the 256 x 10 box of dphi^{n-1/2}
// (rows y0-1 .. y0+8), and for each the two 4-column x-halo boxes at columns x0-4 and
// x0+256 (taken modulo the x side, always a multiple of 4 floats: the 16-byte rule of
// tensor copies).  Only the tiles at the ends of y (periodic rows) split the main box at
// the wrap and fetch their halo columns row by row.  Issuing one copy per staged row from
// every lane, as the first version did, cost about a tenth of all instructions of the
// pass (each lane's copy is serialised through uniform registers).
//
// Only the planes that have left the shared-memory rings stay in registers (level 0 at plane
// j-1, level 1 at k-1, the level-1 dphi handed to level 2); the stencil reads the others in
// the rings, where it reads their neighbours anyway.  (Full register queues along z, rotated
// by moves or, with the plane loop unrolled three times, by renaming, spilled at the
// 96-register limit of two 320-thread CTAs per SM.)  The plane loop's steady-state body tests
// no plane ranges, the kick constants arrive packed as f32x2 operands, the copy context sits
// in shared memory and x-edge values are loaded by the two lanes that use them: together 22%
// fewer instructions than the plain loop, which leaves the pass waiting on its copies.
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>

#include "prs_internal.h"
#include "prs_ptx.cuh"
#include "prs_tile.cuh"
#include "prs_tmap.h"

namespace prs {

namespace {

constexpr int kXW = 256, kTY = 8;
constexpr int kR0 = kTY + 4, kR1 = kTY + 2;  // rows of a level-0 and a level-1 plane tile
constexpr int kThreads = 320;                // 640 level-1 float4 per plane, two per thread
constexpr int kW1 = kXW + 8;                 // level-1 ring row: columns x0-4 .. x0+xw+3
// level-0 slot (floats): main box [kR0][kXW], left halo [kR0][4], right halo [kR0][4], each
// part at a 128-byte boundary
constexpr int kHL0 = kR0 * kXW, kHR0 = kHL0 + 64, kS0 = kHR0 + 64;
// dphi slot: main box [kR1][kXW], halos [kR1][4]
constexpr int kHLV = kR1 * kXW, kHRV = kHLV + 64, kSV = kHRV + 64;
constexpr int kS1 = kR1 * kW1;  // level-1 slot
constexpr size_t kSmem = 128 + (size_t)(4 * kS0 + 2 * kS1 + 3 * kSV) * sizeof(float);
constexpr unsigned kBytesPhi = (kR0 * kXW + 2 * kR0 * 4) * 4u;
constexpr unsigned kBytesV = (kR1 * kXW + 2 * kR1 * 4) * 4u;
static_assert(kS0 % 32 == 0 && kSV % 32 == 0 && kHL0 % 32 == 0 && kHLV % 32 == 0, "128-byte aligned parts");

// Tensor maps of one pass: phi^n boxes 256 x {12, 10, 2} and 4 x 12, dphi boxes 256 x
// {10, 9, 1} and 4 x 10 (one plane deep).
struct T2Maps {
    CUtensorMap phi12, phi10, phi2, phih, v10, v9, v1, vh;
};

static __device__ __noinline__ void drain_planes(uint64_t* bar, int from, int issued, unsigned int* err)
{
    for (int i = from; i <= issued; ++i) mbar_wait(&bar[i & 3], (unsigned)(i >> 2) & 1u, err);
}

// What the copies of a plane need.  Only thread 0 (and, on the tiles at the ends of y, the
// last warp) issue copies, so this lives in shared memory rather than in every thread's
// registers.
struct Ctx2 {
    const float* phi_in;
    const float* v_in;
    size_t plane;
    int nx, ny, nz, x0, y0, z0, zn, xl, xr, ywrap;  // ywrap: 0, -1 (top tile), +1 (bottom tile)
};

// The CTA's shared memory: mbarriers and the copy context, then the rings.
struct Smem2 {
    uint64_t bar[4];
    Ctx2 c;
};
static_assert(sizeof(Smem2) <= 128, "header fits the first 128 bytes");

extern __shared__ __align__(128) unsigned char t2_smem[];

__device__ __forceinline__ Smem2* hdr2() { return reinterpret_cast<Smem2*>(t2_smem); }
// ring0 (4 phi slots), ring1 (2 level-1 slots), ringv (3 dphi slots), after the header
__device__ __forceinline__ float* ring0() { return reinterpret_cast<float*>(t2_smem + 128); }
__device__ __forceinline__ float* ring1() { return ring0() + 4 * kS0; }
__device__ __forceinline__ float* ringv() { return ring1() + 2 * kS1; }

__device__ __forceinline__ int wrap2(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Stage level-0 plane pl (global z0-2+pl) and, with with_v, the dphi of level-1 plane pl-1
// into dphi slot vs = (pl-1) mod 3.  Called by every thread; thread 0 issues the tensor copies.
__device__ __forceinline__ void issue_plane(const T2Maps& m, int tid, int pl, bool with_v, int vs)
{
    const Ctx2& c = hdr2()->c;
    uint64_t* b = &hdr2()->bar[pl & 3];
    if (tid == 0) {
        const int zg = wrap2(c.z0 - 2 + pl, c.nz), zvg = wrap2(c.z0 - 3 + pl, c.nz);
        float* d0 = ring0() + (pl & 3) * kS0;
        float* dv = ringv() + vs * kSV;
        mbar_arrive_expect_tx(b, kBytesPhi + (with_v ? kBytesV : 0u));
        if (c.ywrap == 0) {
            tma_load3(d0, &m.phi12, c.x0, c.y0 - 2, zg, b);
            tma_load3(d0 + kHL0, &m.phih, c.xl, c.y0 - 2, zg, b);
            tma_load3(d0 + kHR0, &m.phih, c.xr, c.y0 - 2, zg, b);
            if (with_v) {
                tma_load3(dv, &m.v10, c.x0, c.y0 - 1, zvg, b);
                tma_load3(dv + kHLV, &m.vh, c.xl, c.y0 - 1, zvg, b);
                tma_load3(dv + kHRV, &m.vh, c.xr, c.y0 - 1, zvg, b);
            }
        } else if (c.ywrap < 0) {  // y0 = 0: rows ny-2, ny-1, then 0 .. 9
            tma_load3(d0, &m.phi2, c.x0, c.ny - 2, zg, b);
            tma_load3(d0 + 2 * kXW, &m.phi10, c.x0, 0, zg, b);
            if (with_v) {
                tma_load3(dv, &m.v1, c.x0, c.ny - 1, zvg, b);
                tma_load3(dv + kXW, &m.v9, c.x0, 0, zvg, b);
            }
        } else {  // y0 = ny-8: rows ny-10 .. ny-1, then 0, 1
            tma_load3(d0, &m.phi10, c.x0, c.ny - 10, zg, b);
            tma_load3(d0 + 10 * kXW, &m.phi2, c.x0, 0, zg, b);
            if (with_v) {
                tma_load3(dv, &m.v9, c.x0, c.ny - 9, zvg, b);
                tma_load3(dv + 9 * kXW, &m.v1, c.x0, 0, zvg, b);
            }
        }
    }
    if (tid >= kThreads - 32 && c.ywrap != 0) {
        // the wrap tiles' halo columns row by row (16 bytes each) on the last warp: task
        // t = lane + 32 u; t < 2 kR0: phi row t/2, side t%2, then the dphi rows
        const int zg = wrap2(c.z0 - 2 + pl, c.nz), zvg = wrap2(c.z0 - 3 + pl, c.nz);
        float* d0 = ring0() + (pl & 3) * kS0;
        float* dv = ringv() + vs * kSV;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = (tid & 31) + 32 * u;
            const bool isv = t >= 2 * kR0;
            if (t >= 2 * (kR0 + kR1) || (isv && !with_v)) continue;
            const int tt = isv ? t - 2 * kR0 : t, r = tt >> 1, side = tt & 1;
            const int y = wrap2(isv ? c.y0 - 1 + r : c.y0 - 2 + r, c.ny);
            const float* src = (isv ? c.v_in + (size_t)zvg * c.plane : c.phi_in + (size_t)zg * c.plane) +
                               (size_t)y * c.nx + (side ? c.xr : c.xl);
            float* dst = (isv ? dv + (side ? kHRV : kHLV) : d0 + (side ? kHR0 : kHL0)) + 4 * r;
            bulk_g2s(dst, src, 16u, b);
        }
    }
}

// Per-thread offsets and roles.  Item h of a thread is level-1 float4 q = tid + 320 h: row
// q / 64 (item 1 sits 5 rows below item 0), column q % 64.
struct Lane2 {
    int tid, lane, o0, o1, e0[2];  // item 0's phi-slot and level-1-slot offsets; x-edge offsets
    bool edge, l2a, l2b, hal;      // l2a, l2b: item 0, 1 runs level 2 (warp-uniform)
    unsigned hx;                   // halo lane: x neighbours' offsets in the phi slot, hxm | hxp << 16
    int hc, hv, ho;
};
constexpr int kD0 = 5 * kXW, kD1 = 5 * kW1;  // item 1 - item 0 in the phi and level-1 slots

// What a thread carries from plane to plane: level 0 at plane j-1 (am), level 1 at k-1 (bm),
// the level-1 dphi^{n+1/2} at plane k (w1), and the halo lane's level 0 at j-1 (hm).
struct Queue2 {
    float4 am[2], bm[2], w1[2];
    float hm;
};

// Plane iteration i with levels 1..LV active (LV = 2 in the steady state, whose body tests
// no plane ranges; the first four iterations fill the pipeline).  Level 0 at planes j, j+1
// and level 1 at plane k are read from the rings (the stencil reads their x and y neighbours
// there anyway).  vs = (i-1) mod 3, the dphi slot of level-1 plane j = i-1.  off: the
// element offset of item 0's output at level-2 plane k = i-2.  Returns false when a wait
// gave up.
template <bool MID, int LV>
__device__ __forceinline__ bool t2_iter(const T2Maps& m, const Lane2& t, int i, int nplanes, int vs, size_t off,
                                        int nx5, const KickP& k0, const KickP& k1, Queue2& q, float* phi_out,
                                        float* v_out, float* phi_mid, float* v_mid, unsigned int* err)
{
    const bool ok = mbar_wait(&hdr2()->bar[i & 3], (unsigned)(i >> 2) & 1u, err);
    if (__syncthreads_or(!ok)) {
        if (t.tid == 0) drain_planes(hdr2()->bar, i, min(i + 1, nplanes - 1), err);  // planes issued so far
        return false;
    }
    if (i + 2 < nplanes) issue_plane(m, t.tid, i + 2, true, vs == 0 ? 2 : vs - 1);
    const int P = i & 1;
    const float* Ln = ring0() + (i & 3) * kS0;        // level 0 at plane j+1
    const float* Lj = ring0() + ((i + 3) & 3) * kS0;  // level 0 at plane j
    float4 pn[2], w1n[2];                             // level 1 at plane j of this thread's items
    if (LV >= 1) {  // level 1 (step n) at plane j: level 0 at j-1 (am), j, j+1 (ring)
        float* L1 = ring1() + (P ^ 1) * kS1;
        const float* V = ringv() + vs * kSV;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int o = t.o0 + h * kD0;
            const float4 a = lds4(Lj + o);
            float e = 0.f, left, right;
            if (t.edge) e = Lj[t.e0[h]];  // lane 0: the left neighbour, lane 31: the right one
            const float su = __shfl_up_sync(0xffffffffu, a.w, 1), sd = __shfl_down_sync(0xffffffffu, a.x, 1);
            left = t.lane == 0 ? e : su;
            right = t.lane == 31 ? e : sd;
            w1n[h] = lds4(V + o - kXW);  // dphi row = level-1 row
            update4p(a, left, right, lds4(Lj + o + kXW), lds4(Lj + o - kXW), lds4(Ln + o), q.am[h], w1n[h], pn[h],
                     k0);
            *reinterpret_cast<float4*>(L1 + t.o1 + h * kD1) = pn[h];
            q.am[h] = a;
        }
        if (t.hal) {
            const float hcen = Lj[t.hc];
            float vv = V[t.hv];
            L1[t.ho] = update1(hcen, Lj[t.hx >> 16], Lj[t.hx & 0xffffu], Lj[t.hc + 4], Lj[t.hc - 4], Ln[t.hc], q.hm,
                               vv, kick_scalar(k0), deta_only(k0), true);
            q.hm = hcen;
        }
    }
    if (LV >= 2) {  // level 2 (step n+1) at plane k: level 1 at k-1 (bm), k (ring), k+1 (pn)
        const float* L1 = ring1() + P * kS1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!(h == 0 ? t.l2a : t.l2b)) continue;  // the level-1 halo rows 0, 9
            const int o = t.o1 + h * kD1;
            const float4 b = lds4(L1 + o);
            float e = 0.f, left, right;
            if (t.edge) e = L1[o + (t.lane == 0 ? -1 : 4)];
            const float su = __shfl_up_sync(0xffffffffu, b.w, 1), sd = __shfl_down_sync(0xffffffffu, b.x, 1);
            left = t.lane == 0 ? e : su;
            right = t.lane == 31 ? e : sd;
            float4 vv = q.w1[h];
            const size_t go = off + (size_t)(h * nx5);
            if (MID) {
                stg4(phi_mid + go, b);
                stg4(v_mid + go, vv);
            }
            float4 out;
            update4p(b, left, right, lds4(L1 + o + kW1), lds4(L1 + o - kW1), pn[h], q.bm[h], vv, out, k1);
            stg4(phi_out + go, out);
            stg4(v_out + go, vv);
            q.bm[h] = b;
        }
    }
    if (LV >= 1) {
#pragma unroll
        for (int h = 0; h < 2; ++h) q.w1[h] = w1n[h];
    }
    return true;
}

template <bool MID>
__global__ void __launch_bounds__(kThreads, 2)
    k_step3d_t2tma(const __grid_constant__ T2Maps maps, const float* __restrict__ phi_in, float* __restrict__ phi_out,
                   const float* __restrict__ v_in, float* __restrict__ v_out, float* __restrict__ phi_mid,
                   float* __restrict__ v_mid, int nx, int ny, int nz, int cz, KickP k0, KickP k1, unsigned int* err)
{
    const int nxt = nx / kXW, ytiles = ny / kTY;
    const int x0 = (blockIdx.x % nxt) * kXW, y0 = (blockIdx.x / nxt % ytiles) * kTY, z0 = blockIdx.x / nxt / ytiles * cz;
    const int zn = min(cz, nz - z0);
    const int nplanes = zn + 4;  // level-0 local planes 0..zn+3 = global z0-2 .. z0+zn+1
    const size_t plane = (size_t)nx * ny;

    Lane2 t;
    t.tid = threadIdx.x;
    t.lane = t.tid & 31;
    const int row = t.tid >> 6, col = t.tid & 63;  // item 0; item 1 is row + 5
    t.o0 = (row + 1) * kXW + 4 * col;  // phi slot (phi row row+1); dphi slot at o0 - kXW
    t.o1 = row * kW1 + 4 + 4 * col;    // level-1 slot
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        // x neighbour beyond the warp's 32 float4: lane 0 reads the left one, lane 31 the right
        const int r = row + 5 * h, o = t.o0 + h * kD0;
        t.e0[h] = t.lane == 0 ? (col == 0 ? kHL0 + (r + 1) * 4 + 3 : o - 1) : (col == 63 ? kHR0 + (r + 1) * 4 : o + 4);
    }
    t.edge = t.lane == 0 || t.lane == 31;
    t.l2a = t.tid >= 64;   // item 0 on level-1 rows 1..4
    t.l2b = t.tid < 256;   // item 1 on level-1 rows 5..8
    // halo lanes: thread t < 2 kR1 computes level 1 at row t/2, column x0-1 (t even) or x0+256
    t.hal = t.tid < 2 * kR1;
    t.hc = 4, t.hx = 0, t.hv = 0, t.ho = 0;
    if (t.hal) {
        const int r = t.tid >> 1;
        if ((t.tid & 1) == 0) {
            t.hc = kHL0 + (r + 1) * 4 + 3;
            t.hx = (unsigned)(t.hc - 1) | (unsigned)((r + 1) * kXW) << 16;
            t.hv = kHLV + r * 4 + 3;
            t.ho = r * kW1 + 3;
        } else {
            t.hc = kHR0 + (r + 1) * 4;
            t.hx = (unsigned)((r + 1) * kXW + kXW - 1) | (unsigned)(t.hc + 1) << 16;
            t.hv = kHRV + r * 4;
            t.ho = r * kW1 + kXW + 4;
        }
    }
    if (t.tid == 0) {
        Smem2* sm = hdr2();
        sm->c = Ctx2{phi_in, v_in, plane, nx, ny, nz, x0, y0, z0, zn, x0 >= 4 ? x0 - 4 : x0 - 4 + nx,
                     x0 + kXW < nx ? x0 + kXW : 0, y0 == 0 ? -1 : (y0 + kTY == ny ? 1 : 0)};
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(&sm->bar[i], 1);
        mbar_fence_init();
    }
    __syncthreads();
    issue_plane(maps, t.tid, 0, false, 0);
    issue_plane(maps, t.tid, 1, false, 0);

    Queue2 q;
    const int nx5 = 5 * nx;
    size_t off = (size_t)z0 * plane + (size_t)(y0 - 1 + row) * nx + x0 + 4 * col;  // level-2 plane 2 = z0
    // pipeline fill: iterations 0, 1 only stage planes; level 1 starts at 2, level 2 at 4; the
    // queues' first planes are read where they are first needed
    if (!t2_iter<MID, 0>(maps, t, 0, nplanes, 2, off, nx5, k0, k1, q, phi_out, v_out, phi_mid, v_mid, err)) return;
    if (!t2_iter<MID, 0>(maps, t, 1, nplanes, 0, off, nx5, k0, k1, q, phi_out, v_out, phi_mid, v_mid, err)) return;
#pragma unroll
    for (int h = 0; h < 2; ++h) q.am[h] = lds4(ring0() + t.o0 + h * kD0);  // level 0 at plane 0 (slot 0)
    if (t.hal) q.hm = ring0()[t.hc];
    if (!t2_iter<MID, 1>(maps, t, 2, nplanes, 1, off, nx5, k0, k1, q, phi_out, v_out, phi_mid, v_mid, err)) return;
    if (!t2_iter<MID, 1>(maps, t, 3, nplanes, 2, off, nx5, k0, k1, q, phi_out, v_out, phi_mid, v_mid, err)) return;
#pragma unroll
    for (int h = 0; h < 2; ++h) q.bm[h] = lds4(ring1() + kS1 + t.o1 + h * kD1);  // level 1 at plane 1 (slot 1)
    int vs = 0;  // (i-1) mod 3 at i = 4
    for (int i = 4; i < nplanes; ++i) {
        if (!t2_iter<MID, 2>(maps, t, i, nplanes, vs, off, nx5, k0, k1, q, phi_out, v_out, phi_mid, v_mid, err))
            return;
        off += plane;
        vs = vs == 2 ? 0 : vs + 1;
    }
}

}  // namespace

EncodeTiled tmap_encoder()
{
    static std::atomic<EncodeTiled> fn{nullptr};
    EncodeTiled f = fn.load(std::memory_order_acquire);
    if (f) return f;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
        cudaGetLastError();
        return nullptr;
    }
    f = reinterpret_cast<EncodeTiled>(p);
    fn.store(f, std::memory_order_release);
    return f;
}

bool tmap_encode(EncodeTiled f, CUtensorMap* m, const float* base, const Geo& g, unsigned bw, unsigned bh)
{
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nx * g.ny * 4};
    const cuuint32_t box[3] = {bw, bh, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return f(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The tensor-copy pass applies to FP32 3D boxes tiled by 256 x 8 (x side a multiple of
// 256, y side a multiple of 8 and at least 16, z side at least 3).  With a 256-wide row the
// tile is the whole row: its halo boxes hold the row's own wrapped end columns, and the halo
// lanes compute two columns the row's float4 also compute (the same operations, so the same
// bits).
bool t2tma_ok(const Geo& g)
{
    return g.dims == 3 && g.nx % kXW == 0 && g.ny % kTY == 0 && g.ny >= 2 * kTY && g.nz >= 3;
}

cudaError_t launch_step_t2_tma(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out,
                               KickF k0, KickF k1, RunConst<float> rc, unsigned int* err, cudaStream_t st,
                               float* phi_mid, float* v_mid)
{
    if (!t2tma_ok(g)) return cudaErrorNotSupported;
    if ((((uintptr_t)phi_in | (uintptr_t)v_in) & 15u) != 0) return cudaErrorNotSupported;
    const EncodeTiled f = tmap_encoder();
    if (!f) return cudaErrorNotSupported;
    T2Maps m;
    if (!tmap_encode(f, &m.phi12, phi_in, g, kXW, kR0) || !tmap_encode(f, &m.phi10, phi_in, g, kXW, 10) ||
        !tmap_encode(f, &m.phi2, phi_in, g, kXW, 2) || !tmap_encode(f, &m.phih, phi_in, g, 4, kR0) ||
        !tmap_encode(f, &m.v10, v_in, g, kXW, kR1) || !tmap_encode(f, &m.v9, v_in, g, kXW, 9) ||
        !tmap_encode(f, &m.v1, v_in, g, kXW, 1) || !tmap_encode(f, &m.vh, v_in, g, 4, kR1))
        return cudaErrorNotSupported;
    const bool mid = phi_mid != nullptr;
    const KickP p0 = kick_packed(k0, rc.deta), p1 = kick_packed(k1, rc.deta);
    const void* fn = mid ? (const void*)k_step3d_t2tma<true> : (const void*)k_step3d_t2tma<false>;
    static std::atomic<unsigned long long> attr[2];
    cudaError_t e = smem_limit_once(attr[mid ? 1 : 0], fn, (int)kSmem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, kSmem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int slots = per_sm * sm_count_current();
    const int tiles = (g.nx / kXW) * (g.ny / kTY);
    // z-chunks: whole waves of resident CTAs, balanced against the four halo planes per chunk
    int best = 1;
    double best_score = -1.0;
    for (int nc = 1; nc <= g.nz / 8 || nc == 1; ++nc) {
        const int cc = (g.nz + nc - 1) / nc, n = (g.nz + cc - 1) / cc;
        const long long blocks = (long long)tiles * n;
        const long long waves = (blocks + slots - 1) / slots;
        const double score = (double)blocks / (double)(waves * slots) * cc / (cc + 4.0) * (waves >= 2 ? 1.0 : 0.9);
        if (score > best_score + 1e-9) best_score = score, best = n;
        if (nc > 4096) break;
    }
    const int cz = (g.nz + best - 1) / best;
    const long long blocks = (long long)tiles * ((g.nz + cz - 1) / cz);
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    if (mid)
        k_step3d_t2tma<true><<<(unsigned)blocks, kThreads, kSmem, st>>>(m, phi_in, phi_out, v_in, v_out, phi_mid, v_mid,
                                                                       g.nx, g.ny, g.nz, cz, p0, p1, err);
    else
        k_step3d_t2tma<false><<<(unsigned)blocks, kThreads, kSmem, st>>>(m, phi_in, phi_out, v_in, v_out, nullptr,
                                                                        nullptr, g.nx, g.ny, g.nz, cz, p0, p1, err);
    return cudaGetLastError();
}

}  // namespace prs

// prs_tile.cuh -- the FP32 tile routines shared by the single-run kernels
// (prs_fast.cu) and the persistent ensemble kernel (prs_batch.cu).
//
// A tile is a run of z-planes (3D: ty whole x-rows of y per plane) or of row bands
// (2D).  phi arrives through the TMA engine: cp.async.bulk copies of whole row runs
// into a 4-slot shared-memory ring, one mbarrier per slot; while plane z is used,
// planes z-1, z, z+1 are resident and z+2 is in flight.  x neighbours come from the
// neighbouring lane's float4 by warp shuffle (rows are whole, so the periodic wrap
// is a shared-memory read by lanes 0 and 31); y and z neighbours are 128-bit
// shared-memory reads; dphi is pointwise and loaded into registers one plane
// ahead.  A tile can apply one leapfrog step (Eqs. 3-5), accumulate the wall
// diagnostics (Eq. 7, Eq. 8) of the state it reads, or both from one read.
//
// Shared memory of a tile: [128 B: 4 mbarriers][4 ring slots][link queue, if
// measuring].  Every mbarrier wait is bounded; a tile that gives up returns false
// (the same value in every thread) after letting its issued copies land.
#pragma once

#include <cuda_runtime.h>

#include "prs_internal.h"
#include "prs_f32x2.cuh"
#include "prs_ptx.cuh"

namespace prs {

static constexpr int kFastThreads = 256;

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

__device__ __forceinline__ float4 ldg_stream4(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }

__device__ __forceinline__ void stg4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// Eqs. 3-5 at one site, FP32: x neighbours (xp, xm), y neighbours (a, b), z neighbours
// (e, f; 3D only).  Returns phi^{n+1}; vv becomes dphi^{n+1/2}.  The kick is KickF's
// folded form, 11 operations a site (the FP64 path keeps the canonical order of Eqs. 3-5
// as written); every term is odd in phi, so a negated field steps to the negated field
// exactly.  Each operation is pinned (round-to-nearest intrinsics, the three fused
// multiply-adds explicit), so update4's packed pairs give the same bits.
__device__ __forceinline__ float update1(float cc, float xp, float xm, float a, float b, float e, float f, float& vv,
                                         const KickF& k, const RunConst<float>& rc, bool three_d)
{
    float s2 = __fadd_rn(xp, xm);
    s2 = __fadd_rn(s2, __fadd_rn(a, b));
    if (three_d) s2 = __fadd_rn(s2, __fadd_rn(e, f));
    const float u = __fmul_rn(cc, __fmaf_rn(-k.k2, __fmul_rn(cc, cc), k.k1));
    const float vn = __fmaf_rn(k.c1, vv, __fmaf_rn(k.g, s2, u));
    vv = vn;
    return __fmaf_rn(rc.deta, vn, cc);
}

// Eqs. 3-5 for the four sites of one float4: update1's operations on two packed pairs
// of sites (x, y) and (z, w), one f32x2 instruction per pair and operation, except the
// x-neighbour sums, whose operands straddle the pairs.
__device__ __forceinline__ void update4(float4 c, float left, float right, float4 yp, float4 ym, float4 zp, float4 zm,
                                        float4& v, float4& pn, const KickF& k, const RunConst<float>& rc,
                                        bool three_d)
{
    const f2 kc1 = pk2(k.c1, k.c1), kg = pk2(k.g, k.g), kk1 = pk2(k.k1, k.k1), nk2 = pk2(-k.k2, -k.k2);
    const f2 dt = pk2(rc.deta, rc.deta);
    f2 s0 = pk2(__fadd_rn(c.y, left), __fadd_rn(c.z, c.x));
    f2 s1 = pk2(__fadd_rn(c.w, c.y), __fadd_rn(right, c.z));
    s0 = add2(s0, add2(pk2(yp.x, yp.y), pk2(ym.x, ym.y)));
    s1 = add2(s1, add2(pk2(yp.z, yp.w), pk2(ym.z, ym.w)));
    if (three_d) {
        s0 = add2(s0, add2(pk2(zp.x, zp.y), pk2(zm.x, zm.y)));
        s1 = add2(s1, add2(pk2(zp.z, zp.w), pk2(zm.z, zm.w)));
    }
    const f2 c0 = pk2(c.x, c.y), c1 = pk2(c.z, c.w);
    const f2 u0 = mul2(c0, fma2(nk2, mul2(c0, c0), kk1));
    const f2 u1 = mul2(c1, fma2(nk2, mul2(c1, c1), kk1));
    const f2 v0 = fma2(kc1, pk2(v.x, v.y), fma2(kg, s0, u0));
    const f2 v1 = fma2(kc1, pk2(v.z, v.w), fma2(kg, s1, u1));
    upk2(v0, v.x, v.y);
    upk2(v1, v.z, v.w);
    upk2(fma2(dt, v0, c0), pn.x, pn.y);
    upk2(fma2(dt, v1, c1), pn.z, pn.w);
}

// update4 with the constants already packed (KickP): the same operations in the same order,
// so the same bits.  THREE_D = false: the 2D update (zp, zm unused).
template <bool THREE_D = true>
__device__ __forceinline__ void update4p(float4 c, float left, float right, float4 yp, float4 ym, float4 zp,
                                         float4 zm, float4& v, float4& pn, const KickP& k)
{
    const f2 kc1{k.c1}, kg{k.g}, kk1{k.k1}, nk2{k.nk2}, dt{k.dt};
    f2 s0 = pk2(__fadd_rn(c.y, left), __fadd_rn(c.z, c.x));
    f2 s1 = pk2(__fadd_rn(c.w, c.y), __fadd_rn(right, c.z));
    s0 = add2(s0, add2(pk2(yp.x, yp.y), pk2(ym.x, ym.y)));
    s1 = add2(s1, add2(pk2(yp.z, yp.w), pk2(ym.z, ym.w)));
    if (THREE_D) {
        s0 = add2(s0, add2(pk2(zp.x, zp.y), pk2(zm.x, zm.y)));
        s1 = add2(s1, add2(pk2(zp.z, zp.w), pk2(zm.z, zm.w)));
    }
    const f2 c0 = pk2(c.x, c.y), c1 = pk2(c.z, c.w);
    const f2 u0 = mul2(c0, fma2(nk2, mul2(c0, c0), kk1));
    const f2 u1 = mul2(c1, fma2(nk2, mul2(c1, c1), kk1));
    const f2 v0 = fma2(kc1, pk2(v.x, v.y), fma2(kg, s0, u0));
    const f2 v1 = fma2(kc1, pk2(v.z, v.w), fma2(kg, s1, u1));
    upk2(v0, v.x, v.y);
    upk2(v1, v.z, v.w);
    upk2(fma2(dt, v0, c0), pn.x, pn.y);
    upk2(fma2(dt, v1, c1), pn.z, pn.w);
}

// The scalar kick constants and time step of a packed kick (the low halves), for update1.
__device__ __forceinline__ KickF kick_scalar(const KickP& k)
{
    return KickF{__uint_as_float((unsigned)k.c1), __uint_as_float((unsigned)k.g), __uint_as_float((unsigned)k.k1),
                 -__uint_as_float((unsigned)k.nk2)};
}

__device__ __forceinline__ RunConst<float> deta_only(const KickP& k)
{
    return RunConst<float>{__uint_as_float((unsigned)k.dt), 0.f, 0.f, 0.f, 0.f, 0.f};
}

// x-neighbours of a float4 at column `col` of a whole row in shared memory.
__device__ __forceinline__ void x_halo(const float* row, int col, int nq, int nx, int lane, float4 c, float& left,
                                       float& right)
{
    left = __shfl_up_sync(0xffffffffu, c.w, 1);
    right = __shfl_down_sync(0xffffffffu, c.x, 1);
    if (lane == 0) left = row[col == 0 ? nx - 1 : 4 * col - 1];
    if (lane == 31) right = row[col == nq - 1 ? 0 : 4 * col + 4];
}

// After a wait gave up: let the copies this CTA issued land (each wait again
// bounded) before the CTA exits and its shared memory is reused.  Slots are
// waited in issue order from local index `from`.
static __device__ __noinline__ void drain(uint64_t* bar, int from, int issued, unsigned int* err)
{
    for (int i = from; i <= issued; ++i) mbar_wait(&bar[i & 3], (i >> 2) & 1, err);
}


// --------------------------------------------------------------- diagnostics
//
// Eq. 7 and Eq. 8 on the same plane staging as the step: every site tests the
// signs of its 2D neighbours (one float4 of 4 sites at a time, x neighbours by
// shuffle); only sites with a crossing link (a few per cent) read the extra
// neighbours of the link-midpoint gradient from shared memory.  Each thread keeps
// its own FP64 sums and integer counts; prs_reduce.cuh finishes them in a fixed
// order.

// Per-thread sums.  The site terms of one plane (at most 16 sites x 3 links) are
// added in FP32 and folded into the FP64 totals once per plane: GB300 issues FP64
// at a small fraction of its FP32 rate, and a per-site FP64 add made the kernel
// arithmetic-bound.  The FP32 plane partial of <= 48 terms in [0, 1] (weights) or
// of the ratios keeps a relative error below 48 ulp.
struct SiteAcc {
    double sw, sr;
    float pw, pr;  // current plane's partial sums
    int nl, nw, nv0, nnf;
    // ratio_scale: the factor of the ratio partial (1/V0 for the (dphi/u)^2 form)
    __device__ __forceinline__ void fold(double ratio_scale)
    {
        sw += (double)pw;
        sr += (double)pr * ratio_scale;
        pw = 0.0f;
        pr = 0.0f;
    }
};

// |g| / sum_i |g_i| with the hardware reciprocal square root and reciprocal
// (a few ulp).  den > 0 because the link's own component is non-zero; when the
// squares underflow (|g| below ~1e-19) the components are first divided by den.
__device__ __forceinline__ float link_weight_from(float num, float den, float gx, float gy, float gz)
{
    if (num >= 1e-30f) return __fdividef(num * rsqrtf(num), den);
    const float a = gx / den, b = gy / den, c = gz / den;
    return sqrtf(a * a + b * b + c * c);
}

__device__ __forceinline__ float link_weight3(float gx, float gy, float gz)
{
    float num = gx * gx;
    num = num + gy * gy;
    num = num + gz * gz;
    float den = fabsf(gx);
    den = den + fabsf(gy);
    den = den + fabsf(gz);
    return link_weight_from(num, den, gx, gy, gz);
}

__device__ __forceinline__ float link_weight2(float gx, float gy)
{
    float num = gx * gx;
    num = num + gy * gy;
    float den = fabsf(gx);
    den = den + fabsf(gy);
    return link_weight_from(num, den, gx, gy, 0.0f);
}

// Bit e set when component e of the float4 is negative (the (phi < 0) rule; -0 is not).
__device__ __forceinline__ unsigned negmask4(float4 a)
{
    return (a.x < 0.0f ? 1u : 0u) | (a.y < 0.0f ? 2u : 0u) | (a.z < 0.0f ? 4u : 0u) | (a.w < 0.0f ? 8u : 0u);
}

// Eq. 8 terms of the wall sites among the four (bit e of `wall`), FP32 factored
// potential, hardware reciprocal; plus the exact count of non-finite values,
// screened by one sum (a non-finite value makes it non-finite).
__device__ __forceinline__ void wall_sites4(SiteAcc& a, unsigned wall, float4 c, float4 vv, const RunConst<float>& rc)
{
    const float cs[4] = {c.x, c.y, c.z, c.w};
    const float vs[4] = {vv.x, vv.y, vv.z, vv.w};
    const float screen = ((c.x + c.y) + (c.z + c.w)) + ((vv.x + vv.y) + (vv.z + vv.w));
    if (!isfinite(screen)) {
#pragma unroll
        for (int e = 0; e < 4; ++e) a.nnf += (!isfinite(cs[e]) || !isfinite(vs[e])) ? 1 : 0;
    }
    a.nw += __popc(wall);
    // dphi^2 / V = (dphi/u)^2 / V0 with u = phi^2/phi0^2 - 1: the per-site term is (dphi/u)^2,
    // and 1/V0 is applied once per plane when the FP32 partial is folded into FP64
    const bool v0pos = rc.V0 > 0.0f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float s = cs[e];
        const float u = ((s - rc.phi0) * (s + rc.phi0)) * rc.inv_phi0sq;
        const bool w = (wall >> e) & 1u;
        const bool pos = v0pos && u != 0.0f;
        const float q = __fdividef(vs[e], u);
        a.nv0 += (w && !pos) ? 1 : 0;
        a.pr += (w && pos) ? q * q : 0.0f;
    }
}

// Crossing links are compacted per warp: each lane appends its links (site e of
// its float4, axis d, item j of the lane's float4s in the plane) to the warp's queue
// in shared memory, and the warp takes them 32 at a time, so the link-midpoint
// gradients cost one pass instead of one divergent pass per site and axis.  Full
// rounds run as soon as 32 links are queued; fewer wait for the next float4, and the
// plane's remainder runs once at its end.  A queue holds the remainder (< 32) and one
// float4's links of the whole warp (32 lanes x 4 sites x 3 axes).
static constexpr int kQueuePerWarp = 32 + 32 * 12;
static constexpr size_t kQueueBytes = (kFastThreads / 32) * kQueuePerWarp * sizeof(unsigned);

// Appends this lane's set bits of `mask` (bit 4d+e: site e of the float4, axis d) of
// item j behind the qn pending entries of the warp queue; returns the new count.
__device__ __forceinline__ int enqueue_links(unsigned* wq, int qn, unsigned mask, int lane, int j)
{
    const int cnt = __popc(mask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int k = qn + incl - cnt;
    while (mask) {
        const int b = __ffs(mask) - 1;
        mask &= mask - 1;
        wq[k++] = ((unsigned)j << 9) | ((unsigned)lane << 4) | (unsigned)b;
    }
    __syncwarp();
    return qn + total;
}

// Runs the queued links 32 at a time: all of them when `flush`, else only full
// rounds, moving the rest to the front.  weight(ent) adds one link's weight.
// Returns the number of entries left.
template <typename W>
__device__ __forceinline__ int run_link_rounds(unsigned* wq, int qn, bool flush, int lane, W&& weight)
{
    const int done = flush ? qn : qn & ~31;
    for (int base = 0; base < done; base += 32)
        if (base + lane < done) weight(wq[base + lane]);
    const int rem = qn - done;
    unsigned keep = 0;
    if (lane < rem) keep = wq[done + lane];
    __syncwarp();
    if (lane < rem) wq[lane] = keep;
    __syncwarp();
    return rem;
}

// Eq. 7 weight of the link from site s = (x, row r) of plane Pc to its +1 neighbour t
// along axis d (3D).  One round of a warp's link queue holds links along mixed axes,
// so the axis selects offsets rather than code paths: t = s + o_d, and each transverse
// axis e adds ((phi(s+e) - phi(s-e)) + (phi(t+e) - phi(t-e)))/4, where t's transverse
// neighbours sit at the same offsets as s's (x is transverse only when the link is
// not along x, so s and t share their column).  The components reach link_weight3 in
// axis order (x, y, z).
__device__ __forceinline__ float weight3(const float* Pm, const float* Pc, const float* Pp, int r, int x, int d,
                                        int nx)
{
    const int px = (x + 1 == nx ? 0 : x + 1) - x, mx = (x == 0 ? nx - 1 : x - 1) - x;  // periodic in x
    const int pz = (int)(Pp - Pc), mz = (int)(Pm - Pc);                                 // ring slots
    const float* s = Pc + r * nx + x;
    const float* t = s + (d == 0 ? px : (d == 1 ? nx : pz));
    const int p1 = d == 0 ? nx : px, m1 = d == 0 ? -nx : mx;  // first transverse axis: y or x
    const int p2 = d == 2 ? nx : pz, m2 = d == 2 ? -nx : mz;  // second: z, or y for z-links
    const float gd = *t - *s;
    const float g1 = 0.25f * ((s[p1] - s[m1]) + (t[p1] - t[m1]));
    const float g2 = 0.25f * ((s[p2] - s[m2]) + (t[p2] - t[m2]));
    return link_weight3(d == 0 ? gd : g1, d == 0 ? g1 : (d == 1 ? gd : g2), d == 2 ? gd : g2);
}

// Eq. 7 weight of the link from x of row crow along axis d (2D); urow/drow are the
// rows above and below.  Branch-free over d as in weight3.
__device__ __forceinline__ float weight2(const float* urow, const float* crow, const float* drow, int x, int d, int nx)
{
    const int px = (x + 1 == nx ? 0 : x + 1) - x, mx = (x == 0 ? nx - 1 : x - 1) - x;
    const int pd = (int)(drow - crow), pu = (int)(urow - crow);
    const float* s = crow + x;
    const float* t = s + (d == 0 ? px : pd);
    const int p1 = d == 0 ? pd : px, m1 = d == 0 ? pu : mx;  // the transverse axis: y or x
    const float gd = *t - *s;
    const float g1 = 0.25f * ((s[p1] - s[m1]) + (t[p1] - t[m1]));
    return link_weight2(d == 0 ? gd : g1, d == 0 ? g1 : gd);
}


// Make generic-proxy writes by other CTAs (earlier tiles of a persistent kernel)
// visible to this CTA's bulk copies.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

struct Tile3D {
    const float* phi_in;
    float* phi_out;
    const float* v_in;
    float* v_out;
    int nx, ny, nz, ty;  // box; ty rows of y per plane in a tile
    int y0, z0, zn;      // first row, first plane, number of planes of this tile
};

struct Tile2D {
    const float* phi_in;
    float* phi_out;
    const float* v_in;
    float* v_out;
    int nx, ny, rb;  // box; rb rows per band
    int y0, yn;      // first row and number of rows (a multiple of rb)
};

__host__ __device__ constexpr size_t tile_smem3d(int nx, int ty) { return 128 + 4 * (size_t)(ty + 2) * nx * sizeof(float); }
__host__ __device__ constexpr size_t tile_smem2d(int nx, int rb) { return 128 + 4 * (size_t)rb * nx * sizeof(float); }

// One 3D tile: STEP applies Eqs. 3-5 (phi_in -> phi_out, v_in -> v_out); MEAS adds
// the Eq. 7/8 terms of (phi_in, v_in) to `a`.  wq: this warp's link queue (MEAS).
// NX > 0: the row width as a compile-time constant (then ty = ITEMS * 1024 / NX).
template <int ITEMS, bool STEP, bool MEAS, int NX = 0>
__device__ __forceinline__ bool tile3d(const Tile3D& T, const KickF& k, const RunConst<float>& rc,
                                       unsigned char* smem, unsigned* wq, SiteAcc& a, unsigned int* err)
{
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    float* ring = reinterpret_cast<float*>(smem + 128);
    const int tid = threadIdx.x, lane = tid & 31;
    const int nx = NX > 0 ? NX : T.nx, ty = NX > 0 ? ITEMS * 1024 / NX : T.ty;
    const int ny = T.ny, nz = T.nz, y0 = T.y0, z0 = T.z0, zn = T.zn;
    const int nq = nx >> 2;
    const double rscale = MEAS && rc.V0 > 0.0f ? 1.0 / (double)rc.V0 : 0.0;  // see wall_sites4
    const int tile = (ty + 2) * nx;
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
    const int nloc = zn + 2;  // local planes 0..zn+1 = global z0-1 .. z0+zn (periodic)
    auto issue = [&](int i) {
        int p = z0 - 1 + i;
        p = p < 0 ? p + nz : (p >= nz ? p - nz : p);
        float* dst = ring + (i & 3) * tile;
        const float* src = T.phi_in + (size_t)p * plane;
        uint64_t* b = &bar[i & 3];
        mbar_arrive_expect_tx(b, rowb * (unsigned)(ty + 2));
        bulk_g2s(dst, src + (size_t)ytop * nx, rowb, b);
        bulk_g2s(dst + nx, src + (size_t)y0 * nx, rowb * (unsigned)ty, b);
        bulk_g2s(dst + (size_t)(ty + 1) * nx, src + (size_t)ybot * nx, rowb, b);
    };
    int issued = -1;  // thread 0: highest local plane whose copy was issued
    if (tid == 0)
        for (int i = 0; i < 3 && i < nloc; ++i) issue(i), issued = i;

    int row[ITEMS], col[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        int q = tid + kFastThreads * j;
        row[j] = q / nq;
        col[j] = q - row[j] * nq;
    }
    // With whole 1024-wide rows and four items, a thread's items are the four rows of its
    // column: item j's +y and -y rows are items j+1 and j-1, and a plane's -z masks are the
    // previous plane's centre masks, whose own centre masks were its +z masks.  So a plane
    // computes 6 sign masks per thread (the +z plane's four and the two halo rows) instead of 20.
    constexpr bool kReuse = MEAS && NX == 1024 && ITEMS == 4;
    unsigned cmask[ITEMS], zmask[ITEMS];  // kReuse: this plane's and the previous plane's masks
    float4 vc[ITEMS];
    {
        const float* vb = T.v_in + (size_t)z0 * plane + (size_t)y0 * nx;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) vc[j] = ldg_stream4(vb + (size_t)row[j] * nx + 4 * col[j]);
    }

    for (int zi = 0; zi < zn; ++zi) {
        // local planes zi, zi+1, zi+2 (= z-1, z, z+1) must be resident
        bool ok = true;
        if (zi == 0) ok = mbar_wait(&bar[0], 0, err) && mbar_wait(&bar[1], 0, err);
        ok = ok && mbar_wait(&bar[(zi + 2) & 3], ((zi + 2) >> 2) & 1, err);
        // block-wide decision; also: every thread is done with the previous plane
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain(bar, zi, issued, err);
            __syncthreads();
            return false;
        }
        if (tid == 0 && zi + 3 < nloc) issue(zi + 3), issued = zi + 3;  // into the slot of plane z-2

        const int z = z0 + zi;
        float4 vn[ITEMS];
        if (zi + 1 < zn) {
            const float* vb = T.v_in + (size_t)(z + 1) * plane + (size_t)y0 * nx;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) vn[j] = ldg_stream4(vb + (size_t)row[j] * nx + 4 * col[j]);
        }
        const float* pm = ring + (zi & 3) * tile + nx;
        const float* pc = ring + ((zi + 1) & 3) * tile + nx;
        const float* pp = ring + ((zi + 2) & 3) * tile + nx;
        float* po = T.phi_out + (size_t)z * plane + (size_t)y0 * nx;
        float* vo = T.v_out + (size_t)z * plane + (size_t)y0 * nx;
        if (kReuse && zi == 0) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const int off = row[j] * nx + 4 * col[j];
                cmask[j] = negmask4(lds4(pc + off));
                zmask[j] = negmask4(lds4(pm + off));
            }
        }
        unsigned nmask[ITEMS];  // kReuse: the +z plane's masks, the next plane's centre masks
        int qn = 0;  // this warp's queued links (MEAS)
        // one queued link: item j's row and first column are the same in all lanes of
        // the warp (its 32 float4 are consecutive in one row)
        auto link3 = [&](unsigned ent) {
            const int jj = (int)(ent >> 9), b = ent & 15, e = b & 3, d = b >> 2;
            int r = row[0], cb = col[0];
#pragma unroll
            for (int i = 1; i < ITEMS; ++i)
                if (jj == i) r = row[i], cb = col[i];
            a.pw += weight3(pm, pc, pp, r, 4 * (cb - lane + (int)((ent >> 4) & 31)) + e, d, nx);
        };
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int r = row[j];
            const int off = r * nx + 4 * col[j];
            float4 c = lds4(pc + off);
            float4 ym = lds4(pc + off - nx);
            float4 yp = lds4(pc + off + nx);
            float4 zm = lds4(pm + off);
            float4 zp = lds4(pp + off);
            float left, right;
            x_halo(pc + r * nx, col[j], nq, nx, lane, c, left, right);
            if (MEAS) {
                unsigned sc, syp, sym, szp, szm;
                if (kReuse) {
                    sc = cmask[j];
                    sym = j > 0 ? cmask[j > 0 ? j - 1 : 0] : negmask4(ym);
                    syp = j < ITEMS - 1 ? cmask[j < ITEMS - 1 ? j + 1 : 0] : negmask4(yp);
                    szm = zmask[j];
                    szp = negmask4(zp);
                    nmask[j] = szp;
                } else {
                    sc = negmask4(c);
                    sym = negmask4(ym);
                    syp = negmask4(yp);
                    szm = negmask4(zm);
                    szp = negmask4(zp);
                }
                const unsigned sxp = (sc >> 1) | (right < 0.0f ? 8u : 0u);
                const unsigned sxm = ((sc << 1) & 15u) | (left < 0.0f ? 1u : 0u);
                const unsigned lx = sc ^ sxp, ly = sc ^ syp, lz = sc ^ szp;
                const unsigned wall = lx | ly | lz | (sc ^ sxm) | (sc ^ sym) | (sc ^ szm);
                wall_sites4(a, wall, c, vc[j], rc);
                // bit 4d+e: the link from site e along axis d crosses
                const unsigned lmask = lx | (ly << 4) | (lz << 8);
                a.nl += __popc(lmask);
                qn = enqueue_links(wq, qn, lmask, lane, j);
                qn = run_link_rounds(wq, qn, false, lane, link3);
            }
            if (STEP) {
                float4 pn;
                update4(c, left, right, yp, ym, zp, zm, vc[j], pn, k, rc, true);
                stg4(po + off, pn);
                stg4(vo + off, vc[j]);
            }
        }
        if (MEAS) {
            qn = run_link_rounds(wq, qn, true, lane, link3);
            a.fold(rscale);
        }
        if (kReuse) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) zmask[j] = cmask[j], cmask[j] = nmask[j];
        }
        if (zi + 1 < zn) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) vc[j] = vn[j];
        }
    }
    __syncthreads();  // the ring may be reused by the caller's next tile
    return true;
}

// One 2D tile of row bands (rb = ITEMS*1024/nx rows each); slot i&3 of the ring
// holds band i of the tile (band 0 = the row above it, band nb+1 = the row below).
template <int ITEMS, bool STEP, bool MEAS>
__device__ __forceinline__ bool tile2d(const Tile2D& T, const KickF& k, const RunConst<float>& rc,
                                       unsigned char* smem, unsigned* wq, SiteAcc& a, unsigned int* err)
{
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    float* ring = reinterpret_cast<float*>(smem + 128);
    const int tid = threadIdx.x, lane = tid & 31;
    const int nx = T.nx, ny = T.ny, rb = T.rb, y0 = T.y0, yn = T.yn;
    const int nb = yn / rb;
    const int nq = nx >> 2;
    const double rscale = MEAS && rc.V0 > 0.0f ? 1.0 / (double)rc.V0 : 0.0;  // see wall_sites4
    const int slot = rb * nx;
    const int ringrows = 4 * rb;  // a power of two: rb = 4096/nx rows, nx a multiple of 128 dividing 4096
    const int rmask = ringrows - 1;
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
        float* dst = ring + (i & 3) * slot;
        uint64_t* b = &bar[i & 3];
        if (i == 0) {  // the row above the tile, at the band's last row
            int y = (y0 == 0 ? ny : y0) - 1;
            mbar_arrive_expect_tx(b, rowb);
            bulk_g2s(dst + (size_t)(rb - 1) * nx, T.phi_in + (size_t)y * nx, rowb, b);
        } else if (i == nb + 1) {  // the row below the tile, at the band's first row
            int y = (y0 + yn == ny) ? 0 : y0 + yn;
            mbar_arrive_expect_tx(b, rowb);
            bulk_g2s(dst, T.phi_in + (size_t)y * nx, rowb, b);
        } else {
            int y = y0 + (i - 1) * rb;
            mbar_arrive_expect_tx(b, rowb * (unsigned)rb);
            bulk_g2s(dst, T.phi_in + (size_t)y * nx, rowb * (unsigned)rb, b);
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
    float4 vc[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) vc[j] = ldg_stream4(T.v_in + (size_t)(y0 + row[j]) * nx + 4 * col[j]);

    for (int bi = 0; bi < nb; ++bi) {
        bool ok = true;
        if (bi == 0) ok = mbar_wait(&bar[0], 0, err) && mbar_wait(&bar[1], 0, err);
        ok = ok && mbar_wait(&bar[(bi + 2) & 3], ((bi + 2) >> 2) & 1, err);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain(bar, bi, issued, err);
            __syncthreads();
            return false;
        }
        if (tid == 0 && bi + 3 < nloc) issue(bi + 3), issued = bi + 3;

        const int yb = y0 + bi * rb;  // first row of this band
        float4 vn[ITEMS];
        if (bi + 1 < nb) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                vn[j] = ldg_stream4(T.v_in + (size_t)(yb + rb + row[j]) * nx + 4 * col[j]);
        }
        int qn = 0;  // this warp's queued links (MEAS)
        auto link2 = [&](unsigned ent) {
            const int jj = (int)(ent >> 9), b = ent & 15, e = b & 3, d = b >> 2;
            int r = row[0], cb = col[0];
#pragma unroll
            for (int i = 1; i < ITEMS; ++i)
                if (jj == i) r = row[i], cb = col[i];
            const int lr = (bi + 1) * rb + r;
            a.pw += weight2(ring + (size_t)((lr - 1) & rmask) * nx, ring + (size_t)(lr & rmask) * nx,
                            ring + (size_t)((lr + 1) & rmask) * nx, 4 * (cb - lane + (int)((ent >> 4) & 31)) + e, d,
                            nx);
        };
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int lr = (bi + 1) * rb + row[j];  // local row of this site in ring order
            const float* crow = ring + (size_t)(lr & rmask) * nx;
            const float* urow = ring + (size_t)((lr - 1) & rmask) * nx;
            const float* drow = ring + (size_t)((lr + 1) & rmask) * nx;
            float4 c = lds4(crow + 4 * col[j]);
            float4 ym = lds4(urow + 4 * col[j]);
            float4 yp = lds4(drow + 4 * col[j]);
            float left, right;
            x_halo(crow, col[j], nq, nx, lane, c, left, right);
            if (MEAS) {
                const unsigned sc = negmask4(c);
                const unsigned sxp = (sc >> 1) | (right < 0.0f ? 8u : 0u);
                const unsigned sxm = ((sc << 1) & 15u) | (left < 0.0f ? 1u : 0u);
                const unsigned lx = sc ^ sxp, ly = sc ^ negmask4(yp);
                const unsigned wall = lx | ly | (sc ^ sxm) | (sc ^ negmask4(ym));
                wall_sites4(a, wall, c, vc[j], rc);
                const unsigned lmask = lx | (ly << 4);  // bit 4d+e
                a.nl += __popc(lmask);
                qn = enqueue_links(wq, qn, lmask, lane, j);
                qn = run_link_rounds(wq, qn, false, lane, link2);
            }
            if (STEP) {
                float4 pn;
                update4(c, left, right, yp, ym, ym, ym, vc[j], pn, k, rc, false);
                const size_t off = (size_t)(yb + row[j]) * nx + 4 * col[j];
                stg4(T.phi_out + off, pn);
                stg4(T.v_out + off, vc[j]);
            }
        }
        if (MEAS) {
            qn = run_link_rounds(wq, qn, true, lane, link2);
            a.fold(rscale);
        }
        if (bi + 1 < nb) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) vc[j] = vn[j];
        }
    }
    __syncthreads();
    return true;
}

}  // namespace prs

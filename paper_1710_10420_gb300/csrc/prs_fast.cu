// prs_fast.cu -- the FP32 leapfrog step (Eqs. 3-6) for boxes whose x side is a
// multiple of 128 and at most 4096: the path the benchmark times.
//
// Design (GB300-first; the paper's OpenCL code ran one kernel per Eq. 3, 4, 5 with
// no tiling): one kernel applies Eqs. 3-5 in a single pass over HBM, reading phi
// and dphi once and writing them once (16 B per site-update).
//
//  * A CTA owns full x-rows.  In 3D it owns `ty` rows of y and a chunk of z-planes
//    and marches along z; in 2D it owns a chunk of rows and marches along y.
//  * phi arrives through the TMA engine: cp.async.bulk copies of whole row runs
//    into a 4-slot shared-memory ring (3D: one slot = ty rows + the two y-halo
//    rows of one z-plane; 2D: one slot = one band of rows), completion tracked by
//    one mbarrier per slot.  While plane z is computed, planes z-1, z, z+1 are
//    resident and plane z+2 is in flight.
//  * x neighbours come from the neighbouring lane's float4 by warp shuffle (the
//    row is whole, so the periodic wrap is a shared-memory read by lanes 0/31);
//    y and z neighbours are 128-bit shared-memory reads.
//  * dphi is pointwise: each thread loads its float4 of the next plane into
//    registers one plane ahead, and writes it back in place.
//  * phi^{n+1} and dphi^{n+1/2} leave as coalesced 128-bit stores.
// Every mbarrier wait is bounded (prs_ptx.cuh) and the decision to give up is
// made block-wide, so a lost copy ends the kernel with an error code instead of
// a hang.
#include <cuda_runtime.h>

#include "prs_arith.cuh"
#include "prs_internal.h"
#include "prs_ptx.cuh"

namespace prs {

static constexpr int kFastThreads = 256;

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

__device__ __forceinline__ float4 ldg_stream4(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }

__device__ __forceinline__ void stg4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// Eqs. 3-5 for the four sites of one float4, in the canonical order of site_update.
__device__ __forceinline__ void update4(float4 c, float left, float right, float4 yp, float4 ym, float4 zp, float4 zm,
                                        float4& v, float4& pn, const StepCoef<float>& k, const RunConst<float>& rc,
                                        bool three_d)
{
    auto one = [&](float cc, float xp, float xm, float a, float b, float e, float f, float& vv) -> float {
        float s2 = xp + xm;
        s2 = s2 + (a + b);
        if (three_d) s2 = s2 + (e + f);
        float lap = (s2 - rc.twoD * cc) * rc.inv_dx2;
        float force = (k.cV * cc) * ((cc * cc) * rc.inv_phi0sq - 1.0f);
        float vn = k.c1 * vv + k.c2 * (lap - force);
        vv = vn;
        return cc + rc.deta * vn;
    };
    pn.x = one(c.x, c.y, left, yp.x, ym.x, zp.x, zm.x, v.x);
    pn.y = one(c.y, c.z, c.x, yp.y, ym.y, zp.y, zm.y, v.y);
    pn.z = one(c.z, c.w, c.y, yp.z, ym.z, zp.z, zm.z, v.z);
    pn.w = one(c.w, right, c.z, yp.w, ym.w, zp.w, zm.w, v.w);
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
__device__ __noinline__ void drain(uint64_t* bar, int from, int issued, unsigned int* err)
{
    for (int i = from; i <= issued; ++i) mbar_wait(&bar[i & 3], (i >> 2) & 1, err);
}

// ------------------------------------------------------------------------ 3D

template <int ITEMS>
__global__ void __launch_bounds__(kFastThreads, 2)
    k_step3d_f32(const float* __restrict__ phi_in, float* __restrict__ phi_out, float* __restrict__ v, int nx,
                 int ny, int nz, int ty, int cz, StepCoef<float> k, RunConst<float> rc, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    float* ring = reinterpret_cast<float*>(smem_raw + 128);
    const int tid = threadIdx.x, lane = tid & 31;
    const int ytiles = ny / ty;
    const int y0 = (blockIdx.x % ytiles) * ty;
    const int z0 = (blockIdx.x / ytiles) * cz;
    const int zn = min(cz, nz - z0);
    const int nq = nx >> 2;
    const int tile = (ty + 2) * nx;
    const size_t plane = (size_t)nx * ny;

    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
        mbar_fence_init();
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
        const float* src = phi_in + (size_t)p * plane;
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
    float4 vc[ITEMS];
    {
        const float* vb = v + (size_t)z0 * plane + (size_t)y0 * nx;
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
            return;
        }
        if (tid == 0 && zi + 3 < nloc) issue(zi + 3), issued = zi + 3;  // into the slot of plane z-2

        const int z = z0 + zi;
        float4 vn[ITEMS];
        if (zi + 1 < zn) {
            const float* vb = v + (size_t)(z + 1) * plane + (size_t)y0 * nx;
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) vn[j] = ldg_stream4(vb + (size_t)row[j] * nx + 4 * col[j]);
        }
        const float* pm = ring + (zi & 3) * tile + nx;
        const float* pc = ring + ((zi + 1) & 3) * tile + nx;
        const float* pp = ring + ((zi + 2) & 3) * tile + nx;
        float* po = phi_out + (size_t)z * plane + (size_t)y0 * nx;
        float* vo = v + (size_t)z * plane + (size_t)y0 * nx;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int off = row[j] * nx + 4 * col[j];
            const float* crow = pc + row[j] * nx;
            float4 c = lds4(pc + off);
            float4 ym = lds4(pc + off - nx);
            float4 yp = lds4(pc + off + nx);
            float4 zm = lds4(pm + off);
            float4 zp = lds4(pp + off);
            float left, right;
            x_halo(crow, col[j], nq, nx, lane, c, left, right);
            float4 pn;
            update4(c, left, right, yp, ym, zp, zm, vc[j], pn, k, rc, true);
            stg4(po + off, pn);
            stg4(vo + off, vc[j]);
        }
        if (zi + 1 < zn) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) vc[j] = vn[j];
        }
    }
}

// ------------------------------------------------------------------------ 2D

// Bands of rb = ITEMS*1024/nx rows; slot i&3 of the ring holds band i of the chunk
// (band 0 = the row above the chunk, band nb+1 = the row below it).
template <int ITEMS>
__global__ void __launch_bounds__(kFastThreads, 2)
    k_step2d_f32(const float* __restrict__ phi_in, float* __restrict__ phi_out, float* __restrict__ v, int nx,
                 int ny, int rb, int cy, StepCoef<float> k, RunConst<float> rc, unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    float* ring = reinterpret_cast<float*>(smem_raw + 128);
    const int tid = threadIdx.x, lane = tid & 31;
    const int y0 = blockIdx.x * cy;
    const int yn = min(cy, ny - y0);
    const int nb = yn / rb;
    const int nq = nx >> 2;
    const int slot = rb * nx;
    const int ringrows = 4 * rb;
    const unsigned rowb = (unsigned)nx * 4u;

    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
        mbar_fence_init();
    }
    __syncthreads();

    const int nloc = nb + 2;
    auto issue = [&](int i) {
        float* dst = ring + (i & 3) * slot;
        uint64_t* b = &bar[i & 3];
        if (i == 0) {  // the row above the chunk, at the band's last row
            int y = (y0 == 0 ? ny : y0) - 1;
            mbar_arrive_expect_tx(b, rowb);
            bulk_g2s(dst + (size_t)(rb - 1) * nx, phi_in + (size_t)y * nx, rowb, b);
        } else if (i == nb + 1) {  // the row below the chunk, at the band's first row
            int y = (y0 + yn == ny) ? 0 : y0 + yn;
            mbar_arrive_expect_tx(b, rowb);
            bulk_g2s(dst, phi_in + (size_t)y * nx, rowb, b);
        } else {
            int y = y0 + (i - 1) * rb;
            mbar_arrive_expect_tx(b, rowb * (unsigned)rb);
            bulk_g2s(dst, phi_in + (size_t)y * nx, rowb * (unsigned)rb, b);
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
    for (int j = 0; j < ITEMS; ++j) vc[j] = ldg_stream4(v + (size_t)(y0 + row[j]) * nx + 4 * col[j]);

    for (int bi = 0; bi < nb; ++bi) {
        bool ok = true;
        if (bi == 0) ok = mbar_wait(&bar[0], 0, err) && mbar_wait(&bar[1], 0, err);
        ok = ok && mbar_wait(&bar[(bi + 2) & 3], ((bi + 2) >> 2) & 1, err);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) drain(bar, bi, issued, err);
            return;
        }
        if (tid == 0 && bi + 3 < nloc) issue(bi + 3), issued = bi + 3;

        const int yb = y0 + bi * rb;  // first row of this band
        float4 vn[ITEMS];
        if (bi + 1 < nb) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) vn[j] = ldg_stream4(v + (size_t)(yb + rb + row[j]) * nx + 4 * col[j]);
        }
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int lr = (bi + 1) * rb + row[j];  // local row of this site in ring order
            const float* crow = ring + (size_t)(lr % ringrows) * nx;
            const float* urow = ring + (size_t)((lr + ringrows - 1) % ringrows) * nx;
            const float* drow = ring + (size_t)((lr + 1) % ringrows) * nx;
            float4 c = lds4(crow + 4 * col[j]);
            float4 ym = lds4(urow + 4 * col[j]);
            float4 yp = lds4(drow + 4 * col[j]);
            float left, right;
            x_halo(crow, col[j], nq, nx, lane, c, left, right);
            float4 pn;
            update4(c, left, right, yp, ym, ym, ym, vc[j], pn, k, rc, false);
            const size_t off = (size_t)(yb + row[j]) * nx + 4 * col[j];
            stg4(phi_out + off, pn);
            stg4(v + off, vc[j]);
        }
        if (bi + 1 < nb) {
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) vc[j] = vn[j];
        }
    }
}

// ------------------------------------------------------------------ dispatch

static constexpr int kItems = 4;  // float4 per thread per plane: 4096 sites per plane tile

static size_t smem3d(int nx, int ty) { return 128 + 4 * (size_t)(ty + 2) * nx * sizeof(float); }
static size_t smem2d(int nx, int rb) { return 128 + 4 * (size_t)rb * nx * sizeof(float); }

static constexpr size_t kFastSmemMax = 100 * 1024;

bool fast_step_ok(const Geo& g, int precision)
{
    if (precision != PRS_FP32) return false;
    if (g.nx % 128 != 0 || g.nx > kItems * 1024 || (kItems * 1024) % g.nx != 0) return false;
    const int t = kItems * 1024 / g.nx;  // rows per plane tile (3D) or per band (2D)
    if (g.ny % t != 0) return false;
    return (g.dims == 3 ? smem3d(g.nx, t) : smem2d(g.nx, t)) <= kFastSmemMax;
}

// Number of z-chunks (3D) or row chunks (2D): balance whole waves of resident
// CTAs against the two halo planes each chunk re-reads.
static int pick_chunks(int tiles, int len, int min_len, int slots)
{
    int best = 1;
    double best_score = -1.0;
    for (int nc = 1; nc <= len / min_len || nc == 1; ++nc) {
        int c = (len + nc - 1) / nc;
        int n = (len + c - 1) / c;
        long long blocks = (long long)tiles * n;
        long long waves = (blocks + slots - 1) / slots;
        double fill = (double)blocks / (double)(waves * slots);
        double halo = (double)c / (double)(c + 2);
        double score = fill * halo * (waves >= 2 ? 1.0 : 0.9);
        if (score > best_score + 1e-9) {
            best_score = score;
            best = n;
        }
        if (nc > 4096) break;
    }
    return best;
}

static int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 152;
    }
    return n;
}

cudaError_t launch_step_fast(const Geo& g, const float* in, float* out, float* v, StepCoef<float> k,
                             RunConst<float> rc, unsigned int* err, cudaStream_t st)
{
    static bool attr3 = false, attr2 = false;
    const int t = kItems * 1024 / g.nx;
    const int slots = 2 * sm_count();  // two resident CTAs per SM
    if (g.dims == 3) {
        const size_t sm = smem3d(g.nx, t);
        if (!attr3) {
            cudaError_t e = cudaFuncSetAttribute(k_step3d_f32<kItems>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kFastSmemMax);
            if (e != cudaSuccess) return e;
            attr3 = true;
        }
        if (sm > kFastSmemMax) return cudaErrorInvalidValue;
        const int ytiles = g.ny / t;
        int nchunks = pick_chunks(ytiles, g.nz, 16, slots);
        const int cz = (g.nz + nchunks - 1) / nchunks;
        nchunks = (g.nz + cz - 1) / cz;
        k_step3d_f32<kItems><<<ytiles * nchunks, kFastThreads, sm, st>>>(in, out, v, g.nx, g.ny, g.nz, t, cz, k, rc,
                                                                         err);
        return cudaGetLastError();
    }
    const size_t sm = smem2d(g.nx, t);
    if (!attr2) {
        cudaError_t e = cudaFuncSetAttribute(k_step2d_f32<kItems>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kFastSmemMax);
        if (e != cudaSuccess) return e;
        attr2 = true;
    }
    if (sm > kFastSmemMax) return cudaErrorInvalidValue;
    const int bands = g.ny / t;
    int nchunks = pick_chunks(1, bands, 4, slots);
    const int bpc = (bands + nchunks - 1) / nchunks;
    const int cy = bpc * t;
    nchunks = (g.ny + cy - 1) / cy;
    k_step2d_f32<kItems><<<nchunks, kFastThreads, sm, st>>>(in, out, v, g.nx, g.ny, t, cy, k, rc, err);
    return cudaGetLastError();
}

}  // namespace prs

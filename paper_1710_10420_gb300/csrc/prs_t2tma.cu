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
// The register queues along z (level 0 at planes j-1, j, j+1 and level 1 at k-1, k, k+1)
// rotate by moves: unrolling the plane loop three times, so that they rotate by renaming,
// spilled at the 96-register limit of two 320-thread CTAs per SM and measured slower
// (1.556 against 1.508 ms per step at 1024^3).
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

// Per-thread constants of the pass.
struct Ctx {
    const float* phi_in;
    const float* v_in;
    float* phi_out;
    float* v_out;
    float* phi_mid;
    float* v_mid;
    float *ring0, *ring1, *ringv;
    uint64_t* bar;
    unsigned int* err;
    size_t plane;
    int nx, ny, nz, x0, y0, z0, zn, nplanes, xl, xr, ywrap;  // ywrap: 0, -1 (top tile), +1 (bottom)
    int tid, lane;
    int o0[2], o1[2], e0[2], go[2];  // item offsets: level-0 slot, level-1 slot, x edge, plane
    bool hal;
    int hc, hxm, hxp, hv, ho;  // halo lane: offsets in level-0, dphi, level-1 slots
};

template <bool MID>
__device__ __forceinline__ void issue_plane(const Ctx& c, const T2Maps& m, int pl, bool with_v)
{
    uint64_t* b = &c.bar[pl & 3];
    const int zp = pl - 2 + c.z0, zv = pl - 3 + c.z0;  // global planes (before wrapping)
    const int zg = zp < 0 ? zp + c.nz : (zp >= c.nz ? zp - c.nz : zp);
    const int zvg = zv < 0 ? zv + c.nz : (zv >= c.nz ? zv - c.nz : zv);
    float* d0 = c.ring0 + (pl & 3) * kS0;
    float* dv = c.ringv + ((pl + 2) % 3) * kSV;  // slot of level-1 plane pl-1
    if (c.tid == 0) {
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
    if (c.ywrap != 0 && c.tid >= kThreads - 32) {
        // halo columns row by row (16 bytes each) on the last warp: task t = lane + 32 u;
        // t < 2 kR0: phi row t/2, side t%2, then the dphi rows
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int t = c.lane + 32 * u;
            const bool isv = t >= 2 * kR0;
            if (t >= 2 * (kR0 + kR1) || (isv && !with_v)) continue;
            const int tt = isv ? t - 2 * kR0 : t, r = tt >> 1, side = tt & 1;
            int y = isv ? c.y0 - 1 + r : c.y0 - 2 + r;
            y = y < 0 ? y + c.ny : (y >= c.ny ? y - c.ny : y);
            const float* src = (isv ? c.v_in + (size_t)zvg * c.plane : c.phi_in + (size_t)zg * c.plane) +
                               (size_t)y * c.nx + (side ? c.xr : c.xl);
            float* dst = (isv ? dv + (side ? kHRV : kHLV) : d0 + (side ? kHR0 : kHL0)) + 4 * r;
            bulk_g2s(dst, src, 16u, b);
        }
    }
}

// One plane iteration i of the march.  Level 0 at planes j, j+1 and level 1 at plane k are
// read from the rings (the stencil reads their x and y neighbours there anyway); only the
// planes that have left the rings stay in registers: am = level 0 at plane j-1, bm = level
// 1 at plane k-1, w1 = the level-1 dphi^{n+1/2} at plane k, and the halo lane's level 0 at
// planes j-1, j (hm, hc).  Returns false when a wait gave up.
template <bool MID>
__device__ __forceinline__ bool plane_iter(const Ctx& c, const T2Maps& m, int i, int& issued, const KickF& k0,
                                           const KickF& k1, const RunConst<float>& rc, float4 (&am)[2],
                                           float4 (&bm)[2], float4 (&w1)[2], float& hm, float& hc)
{
    const bool ok = mbar_wait(&c.bar[i & 3], (unsigned)(i >> 2) & 1u, c.err);
    if (__syncthreads_or(!ok)) {
        if (c.tid == 0) drain_planes(c.bar, i, issued, c.err);
        return false;
    }
    if (i + 2 < c.nplanes) {
        issue_plane<MID>(c, m, i + 2, i + 1 >= 1 && i + 1 <= c.zn + 2);
        issued = i + 2;
    }
    const int j = i - 1;  // level-1 plane of this iteration
    const int k = i - 2;  // level-2 plane of this iteration
    const float* Ln = c.ring0 + (i & 3) * kS0;        // level-0 plane j+1
    const float* Lj = c.ring0 + ((i + 3) & 3) * kS0;  // level-0 plane j
    const float hp = c.hal ? Ln[c.hc] : 0.f;
    float4 pn[2], w1n[2];  // level 1 at plane j (phi, dphi) of this thread's float4
    if (j >= 1 && j <= c.zn + 2) {
        float* L1 = c.ring1 + (j & 1) * kS1;
        const float* V = c.ringv + (j % 3) * kSV;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 cc = lds4(Lj + c.o0[h]);
            const float e = Lj[c.e0[h]];  // lane 0: the left neighbour, lane 31: the right one
            const float su = __shfl_up_sync(0xffffffffu, cc.w, 1), sd = __shfl_down_sync(0xffffffffu, cc.x, 1);
            const float left = c.lane == 0 ? e : su, right = c.lane == 31 ? e : sd;
            w1n[h] = lds4(V + c.o0[h] - kXW);  // dphi row = level-1 row
            update4(cc, left, right, lds4(Lj + c.o0[h] + kXW), lds4(Lj + c.o0[h] - kXW), lds4(Ln + c.o0[h]), am[h],
                    w1n[h], pn[h], k0, rc, true);
            *reinterpret_cast<float4*>(L1 + c.o1[h]) = pn[h];
            am[h] = cc;
        }
        if (c.hal) {
            float vv = V[c.hv];
            L1[c.ho] = update1(hc, Lj[c.hxp], Lj[c.hxm], Lj[c.hc + 4], Lj[c.hc - 4], hp, hm, vv, k0, rc, true);
        }
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) am[h] = lds4(Lj + c.o0[h]);
    }
    hm = hc;
    hc = hp;
    if (k >= 2 && k <= c.zn + 1) {
        const float* L1 = c.ring1 + (k & 1) * kS1;
        const size_t zo = (size_t)(c.z0 - 2 + k) * c.plane;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 0 ? c.tid < 64 : c.tid >= 256) continue;  // the level-1 halo rows 0, 9 (warp-uniform)
            const float4 cc = lds4(L1 + c.o1[h]);
            const float e = L1[c.o1[h] + (c.lane == 0 ? -1 : 4)];
            const float su = __shfl_up_sync(0xffffffffu, cc.w, 1), sd = __shfl_down_sync(0xffffffffu, cc.x, 1);
            const float left = c.lane == 0 ? e : su, right = c.lane == 31 ? e : sd;
            float4 vv = w1[h];
            if (MID) {
                stg4(c.phi_mid + zo + c.go[h], cc);
                stg4(c.v_mid + zo + c.go[h], vv);
            }
            float4 out;
            update4(cc, left, right, lds4(L1 + c.o1[h] + kW1), lds4(L1 + c.o1[h] - kW1), pn[h], bm[h], vv, out, k1, rc,
                    true);
            stg4(c.phi_out + zo + c.go[h], out);
            stg4(c.v_out + zo + c.go[h], vv);
            bm[h] = cc;
        }
    } else if (k == 1) {  // level 1 at plane 1, the first level-2 plane's z neighbour below
        const float* L1 = c.ring1 + kS1;
#pragma unroll
        for (int h = 0; h < 2; ++h) bm[h] = lds4(L1 + c.o1[h]);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) w1[h] = w1n[h];
    return true;
}

template <bool MID>
__global__ void __launch_bounds__(kThreads, 2)
    k_step3d_t2tma(const __grid_constant__ T2Maps maps, const float* __restrict__ phi_in, float* __restrict__ phi_out,
                   const float* __restrict__ v_in, float* __restrict__ v_out, float* __restrict__ phi_mid,
                   float* __restrict__ v_mid, int nx, int ny, int nz, int cz, KickF k0, KickF k1, RunConst<float> rc,
                   unsigned int* err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Ctx c;
    c.bar = reinterpret_cast<uint64_t*>(smem_raw);
    c.ring0 = reinterpret_cast<float*>(smem_raw + 128);
    c.ring1 = c.ring0 + 4 * kS0;
    c.ringv = c.ring1 + 2 * kS1;
    c.phi_in = phi_in;
    c.v_in = v_in;
    c.phi_out = phi_out;
    c.v_out = v_out;
    c.phi_mid = phi_mid;
    c.v_mid = v_mid;
    c.err = err;
    c.nx = nx;
    c.ny = ny;
    c.nz = nz;
    c.plane = (size_t)nx * ny;
    c.tid = threadIdx.x;
    c.lane = c.tid & 31;
    const int nxt = nx / kXW, ytiles = ny / kTY;
    c.x0 = (blockIdx.x % nxt) * kXW;
    c.y0 = (blockIdx.x / nxt % ytiles) * kTY;
    c.z0 = blockIdx.x / nxt / ytiles * cz;
    c.zn = min(cz, nz - c.z0);
    c.nplanes = c.zn + 4;  // level-0 local planes 0..zn+3 = global z0-2 .. z0+zn+1
    c.xl = c.x0 >= 4 ? c.x0 - 4 : c.x0 - 4 + nx;
    c.xr = c.x0 + kXW < nx ? c.x0 + kXW : 0;
    c.ywrap = c.y0 == 0 ? -1 : (c.y0 + kTY == ny ? 1 : 0);

    // this thread's level-1 float4: item h is q = tid + 320 h, level-1 row q / 64, column q % 64
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = c.tid + kThreads * h, row = q >> 6, col = q & 63;
        c.o0[h] = (row + 1) * kXW + 4 * col;      // level-0 slot (level-0 row row+1)
        c.o1[h] = row * kW1 + 4 + 4 * col;        // level-1 slot
        // x neighbour beyond the warp's 32 float4: lane 0 reads the left one, lane 31 the right
        const int el = col == 0 ? kHL0 + (row + 1) * 4 + 3 : c.o0[h] - 1;
        const int er = col == 63 ? kHR0 + (row + 1) * 4 : c.o0[h] + 4;
        c.e0[h] = c.lane == 0 ? el : er;
        c.go[h] = (c.y0 - 1 + row) * nx + c.x0 + 4 * col;
    }
    // halo lanes: thread t < 2 kR1 computes level 1 at row t/2, column x0-1 (t even) or x0+256
    c.hal = c.tid < 2 * kR1;
    {
        const int r = c.tid >> 1;
        if ((c.tid & 1) == 0) {
            c.hc = kHL0 + (r + 1) * 4 + 3;
            c.hxm = c.hc - 1;
            c.hxp = (r + 1) * kXW;
            c.hv = kHLV + r * 4 + 3;
            c.ho = r * kW1 + 3;
        } else {
            c.hc = kHR0 + (r + 1) * 4;
            c.hxm = (r + 1) * kXW + kXW - 1;
            c.hxp = c.hc + 1;
            c.hv = kHRV + r * 4;
            c.ho = r * kW1 + kXW + 4;
        }
        if (!c.hal) c.hc = 4, c.hxm = c.hxp = c.hv = c.ho = 0;
    }
    if (c.tid == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(&c.bar[i], 1);
        mbar_fence_init();
    }
    __syncthreads();
    issue_plane<MID>(c, maps, 0, false);
    issue_plane<MID>(c, maps, 1, false);
    int issued = 1;

    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 am[2] = {z4, z4}, bm[2] = {z4, z4}, w1[2] = {z4, z4};
    float hm = 0.f, hc = 0.f;
    for (int i = 0; i < c.nplanes; ++i)
        if (!plane_iter<MID>(c, maps, i, issued, k0, k1, rc, am, bm, w1, hm, hc)) return;
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
                                                                       g.nx, g.ny, g.nz, cz, k0, k1, rc, err);
    else
        k_step3d_t2tma<false><<<(unsigned)blocks, kThreads, kSmem, st>>>(m, phi_in, phi_out, v_in, v_out, nullptr,
                                                                        nullptr, g.nx, g.ny, g.nz, cz, k0, k1, rc, err);
    return cudaGetLastError();
}

}  // namespace prs

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

struct Ctx3 {
    const float* phi_in;
    const float* v_in;
    float *ring0, *ringv, *ring1, *ring2;
    uint64_t* bar;
    size_t plane;
    int nx, ny, nz, x0, y0, z0, zn, xl, xr, ywrap;  // ywrap: 0, -1 (top tile), +1 (bottom tile)
    int tid;
};

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Stage level-0 plane pl (global z0-3+pl) and, with with_v, the dphi of level-1 plane pl-1.
template <int XW>
__device__ __forceinline__ void issue3(const Ctx3& c, const T3Maps& m, int pl, bool with_v)
{
    using S = T3<XW>;
    uint64_t* b = &c.bar[pl & 3];
    const int zg = wrapi(c.z0 - 3 + pl, c.nz), zvg = wrapi(c.z0 - 4 + pl, c.nz);
    float* d0 = c.ring0 + (pl & 3) * S::kS0;
    float* dv = c.ringv + ((pl + 2) % 3) * S::kSV;  // slot of level-1 plane pl-1
    if (c.tid == 0) {
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
    if (c.ywrap != 0 && c.tid >= S::kThreads - 64) {
        // the wrap tiles' halo columns row by row (16 bytes each) on the last two warps: task
        // t < 2 kR0 is phi row t/2, side t%2; then 2 kR1 dphi tasks
        const int t = c.tid - (S::kThreads - 64);
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

template <int XW>
__global__ void __launch_bounds__(T3<XW>::kThreads, T3<XW>::kMinBlocks)
    k_step3d_t3tma(const __grid_constant__ T3Maps maps, const float* __restrict__ phi_in,
                   float* __restrict__ phi_out, const float* __restrict__ v_in, float* __restrict__ v_out, int nx,
                   int ny, int nz, int cz, KickF k0, KickF k1, KickF k2, RunConst<float> rc, unsigned int* err)
{
    using S = T3<XW>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Ctx3 c;
    c.bar = reinterpret_cast<uint64_t*>(smem_raw);
    c.ring0 = reinterpret_cast<float*>(smem_raw + 128);
    c.ringv = c.ring0 + 4 * S::kS0;
    c.ring1 = c.ringv + 3 * S::kSV;
    c.ring2 = c.ring1 + 2 * S::kS1;
    c.phi_in = phi_in;
    c.v_in = v_in;
    c.nx = nx;
    c.ny = ny;
    c.nz = nz;
    c.plane = (size_t)nx * ny;
    c.tid = threadIdx.x;
    const int lane = c.tid & 31;
    const int nxt = nx / XW, ytiles = ny / kTY;
    c.x0 = (blockIdx.x % nxt) * XW;
    c.y0 = (blockIdx.x / nxt % ytiles) * kTY;
    c.z0 = blockIdx.x / nxt / ytiles * cz;
    c.zn = min(cz, nz - c.z0);
    const int nplanes = c.zn + 6;  // level-0 local planes 0 .. zn+5 = global z0-3 .. z0+zn+2
    c.xl = c.x0 >= 4 ? c.x0 - 4 : c.x0 - 4 + nx;
    c.xr = c.x0 + XW < nx ? c.x0 + XW : 0;
    c.ywrap = c.y0 == 0 ? -1 : (c.y0 + kTY == ny ? 1 : 0);

    // this thread's float4: level-1 row r (global y0-2+r), column x0+4 col
    const int r = c.tid / S::F, col = c.tid % S::F;
    const int o0 = (r + 1) * XW + 4 * col;      // phi slot (phi row r+1); dphi slot at o0 - XW
    const int o1 = r * S::kW + 4 + 4 * col;     // level-1/2 slots
    const int e0 = lane == 0 ? (col == 0 ? S::kHL0 + (r + 1) * 4 + 3 : o0 - 1)
                             : (col == S::F - 1 ? S::kHR0 + (r + 1) * 4 : o0 + 4);
    const int e1 = o1 + (lane == 0 ? -1 : 4);  // the same neighbour in the level-1/2 slots
    const bool lv2 = r >= 1 && r <= kTY + 2, lv3 = r >= 2 && r <= kTY + 1;  // warp-uniform
    const int go = (c.y0 - 2 + r) * nx + c.x0 + 4 * col;

    // halo lanes: the first warp (row 0) and the last 16 lanes of the last warp (row 11), both
    // level-1-only rows.  Halo site h: row h/4, column x0-2, x0-1, x0+XW, x0+XW+1 for h%4 = 0..3;
    // the two inner columns of rows 1..10 also run level 2.
    const int h = c.tid < 32 ? c.tid : (c.tid >= S::kThreads - (kHalo - 32) ? c.tid - (S::kThreads - kHalo) : -1);
    const bool hal = h >= 0;
    int hc = 0, hxm = 0, hxp = 0, hv = 0, ho = 4;
    bool hal2 = false;
    if (hal) {
        const int hr = h >> 2, w = h & 3;
        const int base = w < 2 ? S::kHL0 + (hr + 1) * 4 + 2 + w : S::kHR0 + (hr + 1) * 4 + (w - 2);
        hc = base;
        hxm = w == 2 ? (hr + 1) * XW + XW - 1 : base - 1;
        hxp = w == 1 ? (hr + 1) * XW : base + 1;
        hv = w < 2 ? S::kHLV + hr * 4 + 2 + w : S::kHRV + hr * 4 + (w - 2);
        ho = hr * S::kW + (w < 2 ? 2 + w : XW + 4 + (w - 2));
        hal2 = (w == 1 || w == 2) && hr >= 1 && hr <= kTY + 2;
    }

    if (c.tid == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) mbar_init(&c.bar[i], 1);
        mbar_fence_init();
    }
    __syncthreads();
    issue3<XW>(c, maps, 0, false);
    issue3<XW>(c, maps, 1, false);
    int issued = 1;

    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 am = z4, bm = z4, cm = z4, w1 = z4, w2 = z4;
    float hm = 0.f, hb = 0.f, hw = 0.f;
    for (int i = 0; i < nplanes; ++i) {
        const bool ok = mbar_wait(&c.bar[i & 3], (unsigned)(i >> 2) & 1u, err);
        if (__syncthreads_or(!ok)) {
            if (c.tid == 0) drain3(c.bar, i, issued, err);
            return;
        }
        if (i + 2 < nplanes) {
            issue3<XW>(c, maps, i + 2, i + 1 >= 1 && i + 1 <= c.zn + 4);
            issued = i + 2;
        }
        const int j = i - 1, k = i - 2, l = i - 3;  // planes of levels 1, 2, 3
        const float* Ln = c.ring0 + (i & 3) * S::kS0;        // level 0 at plane j+1
        const float* Lj = c.ring0 + ((i + 3) & 3) * S::kS0;  // level 0 at plane j
        float4 pn = z4, w1n = z4, qn = z4, w2n = z4;
        float hpn = 0.f, hwn = 0.f;
        // level 1 (step n) at plane j
        if (j >= 1 && j <= c.zn + 4) {
            float* L1 = c.ring1 + (j & 1) * S::kS1;
            const float* V = c.ringv + (j % 3) * S::kSV;
            const float4 cc = lds4(Lj + o0);
            float left, right;
            xnb(cc, Lj[e0], lane, left, right);
            w1n = lds4(V + o0 - XW);
            update4(cc, left, right, lds4(Lj + o0 + XW), lds4(Lj + o0 - XW), lds4(Ln + o0), am, w1n, pn, k0, rc,
                    true);
            *reinterpret_cast<float4*>(L1 + o1) = pn;
            am = cc;
            if (hal) {
                const float hcen = Lj[hc];
                hwn = V[hv];
                hpn = update1(hcen, Lj[hxp], Lj[hxm], Lj[hc + 4], Lj[hc - 4], Ln[hc], hm, hwn, k0, rc, true);
                L1[ho] = hpn;
                hm = hcen;
            }
        } else {
            am = lds4(Lj + o0);
            if (hal) hm = Lj[hc];
        }
        // level 2 (step n+1) at plane k: level 1 at k-1 (bm), k (ring), k+1 (pn)
        if (k >= 2 && k <= c.zn + 3) {
            const float* L1 = c.ring1 + (k & 1) * S::kS1;
            float* L2 = c.ring2 + (k & 1) * S::kS1;
            if (lv2) {
                const float4 cc = lds4(L1 + o1);
                float left, right;
                xnb(cc, L1[e1], lane, left, right);
                w2n = w1;
                update4(cc, left, right, lds4(L1 + o1 + S::kW), lds4(L1 + o1 - S::kW), pn, bm, w2n, qn, k1, rc,
                        true);
                *reinterpret_cast<float4*>(L2 + o1) = qn;
                bm = cc;
            }
            if (hal2) {
                const float hcen = L1[ho];
                float vv = hw;
                L2[ho] = update1(hcen, L1[ho + 1], L1[ho - 1], L1[ho + S::kW], L1[ho - S::kW], hpn, hb, vv, k1, rc,
                                 true);
                hb = hcen;
            }
        } else if (k == 1) {  // level 1 at plane 1: the first level-2 plane's z neighbour below
            const float* L1 = c.ring1 + S::kS1;
            if (lv2) bm = lds4(L1 + o1);
            if (hal2) hb = L1[ho];
        }
        // level 3 (step n+2) at plane l: level 2 at l-1 (cm), l (ring), l+1 (qn); output
        if (l >= 3 && l <= c.zn + 2) {
            if (lv3) {
                const float* L2 = c.ring2 + (l & 1) * S::kS1;
                const float4 cc = lds4(L2 + o1);
                float left, right;
                xnb(cc, L2[e1], lane, left, right);
                float4 vv = w2, out;
                update4(cc, left, right, lds4(L2 + o1 + S::kW), lds4(L2 + o1 - S::kW), qn, cm, vv, out, k2, rc,
                        true);
                const size_t zo = (size_t)(c.z0 - 3 + l) * c.plane;
                stg4(phi_out + zo + go, out);
                stg4(v_out + zo + go, vv);
                cm = cc;
            }
        } else if (l == 2) {  // level 2 at plane 2 (ring slot 0): the first output plane's z neighbour below
            if (lv3) cm = lds4(c.ring2 + o1);
        }
        w1 = w1n;
        w2 = w2n;
        hw = hwn;
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
cudaError_t launch_xw(const Geo& g, const float* phi_in, float* phi_out, const float* v_in, float* v_out, KickF k0,
                      KickF k1, KickF k2, RunConst<float> rc, unsigned int* err, cudaStream_t st)
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
                                                                       g.nz, cz, k0, k1, k2, rc, err);
    return cudaGetLastError();
}

// Tile width for this box: 256 where it divides the x side (one 768-thread CTA per SM),
// else 128 (two 384-thread CTAs per SM); 0 when the pass does not apply.
int t3_width(const Geo& g)
{
    if (g.dims != 3 || g.ny % kTY != 0 || g.ny < 2 * kTY || g.nz < 3) return 0;
    if (g.nx % 256 == 0) return 256;
    if (g.nx % 128 == 0) return 128;
    return 0;
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
    return xw == 256 ? launch_xw<256>(g, phi_in, phi_out, v_in, v_out, k0, k1, k2, rc, err, st)
                     : launch_xw<128>(g, phi_in, phi_out, v_in, v_out, k0, k1, k2, rc, err, st);
}

}  // namespace prs

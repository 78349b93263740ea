// prs_reduce.cuh -- fixed-order reduction of the diagnostic sums (Eq. 7, Eq. 8):
// warp shuffles, then the warps of a block, then one partial per block; the last
// block to finish (an atomic completion counter, no waiting) adds the partials in
// index order.  Repeated launches on the same grid give bit-identical results.
#pragma once

#include <cuda_runtime.h>

#include "prs_internal.h"

namespace prs {

__device__ __forceinline__ void acc_add(DiagAcc& a, const DiagAcc& b)
{
    a.sum_w += b.sum_w;
    a.sum_ratio += b.sum_ratio;
    a.n_links += b.n_links;
    a.n_wall += b.n_wall;
    a.n_vzero += b.n_vzero;
    a.n_nonfinite += b.n_nonfinite;
}

__device__ __forceinline__ void acc_shfl_down(DiagAcc& a, int off)
{
    DiagAcc o;
    o.sum_w = __shfl_down_sync(0xffffffffu, a.sum_w, off);
    o.sum_ratio = __shfl_down_sync(0xffffffffu, a.sum_ratio, off);
    o.n_links = __shfl_down_sync(0xffffffffu, a.n_links, off);
    o.n_wall = __shfl_down_sync(0xffffffffu, a.n_wall, off);
    o.n_vzero = __shfl_down_sync(0xffffffffu, a.n_vzero, off);
    o.n_nonfinite = __shfl_down_sync(0xffffffffu, a.n_nonfinite, off);
    acc_add(a, o);
}

// Fixed-order warp reduction: lane 0 ends with the sum of the warp.
__device__ __forceinline__ void acc_warp_reduce(DiagAcc& a)
{
    for (int off = 16; off > 0; off >>= 1) acc_shfl_down(a, off);
}

// Every thread of the block calls this once with its own sums: block bid of the nblocks
// that reduce into scr; their total lands in *scr.result and the counter is reset for the
// next launch.
__device__ __forceinline__ void block_reduce_and_finish_at(DiagAcc a, const DiagScratch& scr, unsigned int bid,
                                                           unsigned int nblocks)
{
    __shared__ DiagAcc warp_sums[32];
    __shared__ bool is_last;
    acc_warp_reduce(a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) warp_sums[wid] = a;
    __syncthreads();
    if (wid == 0) {
        DiagAcc b = lane < nw ? warp_sums[lane] : DiagAcc{0.0, 0.0, 0, 0, 0, 0};
        acc_warp_reduce(b);
        if (lane == 0) {
            scr.partials[bid] = b;
            __threadfence();
            unsigned int done = atomicAdd(scr.counter, 1u);
            is_last = (done == nblocks - 1);
        }
    }
    __syncthreads();
    if (!is_last) return;
    // the last block to finish reduces every partial in a fixed order
    __threadfence();
    if (wid == 0) {
        DiagAcc t{0.0, 0.0, 0, 0, 0, 0};
        for (int i = lane; i < (int)nblocks; i += 32) {
            // other blocks wrote these: read through L2, not a possibly stale L1 line
            const DiagAcc* q = scr.partials + i;
            DiagAcc p{__ldcg(&q->sum_w), __ldcg(&q->sum_ratio), __ldcg(&q->n_links),
                      __ldcg(&q->n_wall), __ldcg(&q->n_vzero), __ldcg(&q->n_nonfinite)};
            acc_add(t, p);
        }
        acc_warp_reduce(t);
        if (lane == 0) {
            *scr.result = t;
            *scr.counter = 0u;  // ready for the next launch on this scratch
        }
    }
}

// The whole grid reduces into scr.
__device__ __forceinline__ void block_reduce_and_finish(DiagAcc a, const DiagScratch& scr)
{
    block_reduce_and_finish_at(a, scr, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                               gridDim.x * gridDim.y * gridDim.z);
}

}  // namespace prs

// prs_tmap.h -- TMA tensor maps of the FP32 3D fields and the tensor copy that reads them,
// shared by the multi-step passes (prs_t2tma.cu, prs_t3tma.cu).
//
// A field is described to the TMA engine as a 3D array (x, y, z) of floats, x fastest, with
// a box of bw x bh x 1 elements: one copy moves bh rows of bw columns of one plane.  The
// encoder is the driver's cuTensorMapEncodeTiled, looked up once through the runtime.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "prs_internal.h"
#include "prs_ptx.cuh"

namespace prs {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's encoder, or nullptr when the driver does not offer it.
EncodeTiled tmap_encoder();

// Encode `m` for the FP32 field at `base` (the box's geometry g) with a bw x bh box; false
// when the driver refuses (misaligned base, box too large).
bool tmap_encode(EncodeTiled f, CUtensorMap* m, const float* base, const Geo& g, unsigned bw, unsigned bh);

// One tensor copy of the box at (x, y, z) of `map` into shared memory at `dst` (128-byte
// aligned), counted on `bar` as transaction bytes.  x times 4 bytes must be a multiple of 16.
__device__ __forceinline__ void tma_load3(float* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace prs

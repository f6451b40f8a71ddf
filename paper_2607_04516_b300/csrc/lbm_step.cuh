// lbm_step.cuh -- the two step kernels of the in-place (AA) streaming scheme and their launch
// shapes.  Included by lbm_step_kern.cu, which is compiled once per storage type and forcing
// (LBM_INST_S, LBM_INST_FORCE), so that the instantiations build in parallel.
#pragma once

#include <cuda_runtime.h>

// resident 256-thread blocks per SM the step kernels are compiled for (caps registers at
// 65536 / (256 * blocks)); chosen by measurement on B300
#ifndef LBM_MIN_BLOCKS_LOCAL
#define LBM_MIN_BLOCKS_LOCAL 4
#endif
#ifndef LBM_MIN_BLOCKS_NEIGHBOR
#define LBM_MIN_BLOCKS_NEIGHBOR 4
#endif

#include "lbm_cell.cuh"
#include "lbm_internal.h"

namespace lbm {

// resident blocks per SM of the forced step kernels: the FP32 pair collision with the body force
// and the zone nudging spills heavily at 64 registers; at 80 (3 blocks) FP32 zones run 15% faster
// on the 400 x 400 x 80 city.  The 16-bit forced kernels spill too at 64 registers but still run
// faster at 4 blocks (zones 33.6 against 32.8 GLUPS at 3, same city)
#ifndef LBM_MIN_BLOCKS_FORCED32
#define LBM_MIN_BLOCKS_FORCED32 3
#endif
#ifndef LBM_MIN_BLOCKS_FORCED16
#define LBM_MIN_BLOCKS_FORCED16 4
#endif
template <int S, bool FORCE> constexpr int min_blocks(int unforced) {
    return !FORCE ? unforced : (S == LBM_F32 ? LBM_MIN_BLOCKS_FORCED32 : LBM_MIN_BLOCKS_FORCED16);
}

template <int S, bool FORCE, bool PACK, bool D32>
__global__ void __launch_bounds__(kBlock, min_blocks<S, FORCE>(LBM_MIN_BLOCKS_LOCAL)) k_step_local(StepArgs a) {
    local_block<S, FORCE, PACK, D32>(a, blockIdx.x);
}

// Blocks [0, face_blocks) update the face-layer cells (general boundary resolution, ALU heavy);
// the remaining blocks cover the lattice and update its interior cells.  Face blocks go first so
// that their arithmetic overlaps the memory traffic of the interior blocks, and no warp mixes the
// two paths.  The grid has one block per unit (units == gridDim.x); the 16-bit kernels are
// written as a loop over units all the same: on B300 that form of the code runs the 16-bit
// neighbour step 3-5% faster (0.310 against 0.326 ms on the 400 x 400 x 80 city) and the FP32 one
// 5% slower, so FP32 keeps the plain form.
template <int S, bool FORCE, bool PACK, bool D32>
__global__ void __launch_bounds__(kBlock, min_blocks<S, FORCE>(LBM_MIN_BLOCKS_NEIGHBOR)) k_step_neighbor(StepArgs a, unsigned face_blocks,
                                                                                 unsigned units) {
    if constexpr (S == LBM_F32) {
        neighbor_block<S, FORCE, PACK, D32>(a, blockIdx.x, face_blocks);
    } else {
        for (unsigned b = blockIdx.x; b < units; b += gridDim.x) neighbor_block<S, FORCE, PACK, D32>(a, b, face_blocks);
    }
}

template <int S, bool FORCE, bool PACK, bool D32>
void step_p(bool neighbor, const StepArgs &a, cudaStream_t s) {
    const unsigned lb = lattice_blocks<S, D32>(a.g.N);
    if (neighbor) {
        const unsigned fb = blocks_for(a.nface);
        k_step_neighbor<S, FORCE, PACK, D32><<<fb + lb, kBlock, 0, s>>>(a, fb, fb + lb);
    } else {
        k_step_local<S, FORCE, PACK, D32><<<lb, kBlock, 0, s>>>(a);
    }
}
// PACK (16-bit storage with N and nx even): adjacent cell pairs with 4-byte accesses.
// 16-bit storage: the local step uses adjacent packed pairs when the lattice allows it, the
// neighbour step the (n, n + 256) pairs (faster for its shifted accesses, measured on B300).
// FP32 storage: two cells per thread on lattices of at least kDual32MinCells cells.
template <int S, bool FORCE>
void step_t(bool neighbor, const StepArgs &a, cudaStream_t s) {
    if constexpr (S == LBM_F32) {
        if (a.g.N >= kDual32MinCells) step_p<S, FORCE, false, true>(neighbor, a, s);
        else step_p<S, FORCE, false, false>(neighbor, a, s);
    } else {
        if (a.pack16 && !neighbor) step_p<S, FORCE, true, false>(neighbor, a, s);
        else step_p<S, FORCE, false, false>(neighbor, a, s);
    }
}

}  // namespace lbm

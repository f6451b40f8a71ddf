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
// The unforced FP32 two-cell kernels (lattices of at least kDual32MinCells cells): 3 blocks per SM,
// whose 85 registers hold the pair collision with special-function reciprocals and square roots
// without spilling (400 x 400 x 80 city on B300: neighbour 0.385 -> 0.371 ms, local 0.322 -> 0.313
// ms against 4 blocks with the IEEE forms).
#ifndef LBM_MIN_BLOCKS_DUAL32
#define LBM_MIN_BLOCKS_DUAL32 3
#endif
template <int S, bool FORCE, bool D32 = false> constexpr int min_blocks(int unforced) {
    return FORCE ? (S == LBM_F32 ? LBM_MIN_BLOCKS_FORCED32 : LBM_MIN_BLOCKS_FORCED16)
                 : ((S == LBM_F32 && D32) ? LBM_MIN_BLOCKS_DUAL32 : unforced);
}

template <int S, bool FORCE, bool PACK, bool D32>
__global__ void __launch_bounds__(kBlock, min_blocks<S, FORCE, D32>(LBM_MIN_BLOCKS_LOCAL)) k_step_local(StepArgs a) {
    local_block<S, FORCE, PACK, D32>(a, blockIdx.x);
}

// face_blocks of the units update the face-layer cells (face tables or the general boundary
// resolution, latency and ALU heavy), placed among the lattice blocks as unit_of says; the
// remaining units cover the lattice and update its interior cells.  No warp mixes the two paths.  The grid has one block per unit (units == gridDim.x); the 16-bit kernels are
// written as a loop over units all the same: on B300 that form of the code runs the 16-bit
// neighbour step 3-5% faster (0.310 against 0.326 ms on the 400 x 400 x 80 city) and the FP32 one
// 5% slower, so FP32 keeps the plain form.
template <int S, bool FORCE, bool PACK, bool D32>
__global__ void __launch_bounds__(kBlock, min_blocks<S, FORCE, D32>(LBM_MIN_BLOCKS_NEIGHBOR)) k_step_neighbor(StepArgs a, unsigned face_blocks,
                                                                                 unsigned units, int pshift, unsigned lb0) {
    if constexpr (S == LBM_F32) {
        neighbor_block<S, FORCE, PACK, D32>(a, blockIdx.x, face_blocks, pshift, lb0);
    } else {
        for (unsigned b = blockIdx.x; b < units; b += gridDim.x) neighbor_block<S, FORCE, PACK, D32>(a, b, face_blocks, pshift, lb0);
    }
}

// The lattice blocks of the neighbour step that reach into the ground or top layer (zlat, two
// cells per thread): [0, g1) and [t0, ...) of the lattice blocks, one launch block each.
template <int S, bool FORCE, bool D32>
__global__ void __launch_bounds__(kBlock, min_blocks<S, FORCE, D32>(LBM_MIN_BLOCKS_NEIGHBOR)) k_step_layers(StepArgs a, unsigned g1,
                                                                               unsigned t0) {
    const unsigned lb = blockIdx.x < g1 ? blockIdx.x : t0 + (blockIdx.x - g1);
    constexpr long long span = (long long)cells_per_thread<S, D32>() * kBlock;
    prefetch_ahead<S, D32, true, kBlock>(a, lb, lattice_blocks<S, D32, kBlock>(a.g.N));
    neighbor_layer_unit<S, FORCE, D32, kBlock>(a, lb, block_layer_kind(a, lb, span), threadIdx.x);
}

template <int S, bool FORCE, bool PACK, bool D32>
void step_p(bool neighbor, const StepArgs &a, cudaStream_t s, const StepAux *aux) {
    const unsigned lb = lattice_blocks<S, D32>(a.g.N);
    if (neighbor) {
        const unsigned fb = blocks_for(step_face_cells(a));
        const LayerSplit ls = layer_split(a, (long long)cells_per_thread<S, D32>() * kBlock, lb);
        const unsigned nl = ls.t0 - ls.g1, nlay = ls.g1 + (lb - ls.t0);   // main / layer kernel lattice blocks
        // the layer kernel forked onto the domain's second stream when there is one (its launch
        // overlaps the main kernel instead of adding its ramp and tail), else in order
        const bool fork = nlay > 0 && fb + nl > 0 && aux && aux->stream &&
                          cudaEventRecord(aux->fork, s) == cudaSuccess && cudaStreamWaitEvent(aux->stream, aux->fork, 0) == cudaSuccess;
        if (nlay > 0) k_step_layers<S, FORCE, D32><<<nlay, kBlock, 0, fork ? aux->stream : s>>>(a, ls.g1, ls.t0);
        if (fork) cudaEventRecord(aux->join, aux->stream);
        if (fb + nl > 0)
            k_step_neighbor<S, FORCE, PACK, D32><<<fb + nl, kBlock, 0, s>>>(a, fb, fb + nl, face_period_shift(fb, fb + nl), ls.g1);
        if (fork) cudaStreamWaitEvent(s, aux->join, 0);
    } else {
        k_step_local<S, FORCE, PACK, D32><<<lb, kBlock, 0, s>>>(a);
    }
}
// PACK (16-bit storage with N and nx even): adjacent cell pairs with 4-byte accesses.
// 16-bit storage: the local step uses adjacent packed pairs when the lattice allows it, the
// neighbour step the (n, n + 256) pairs (faster for its shifted accesses, measured on B300).
// FP32 storage: two cells per thread on lattices of at least kDual32MinCells cells.
template <int S, bool FORCE>
void step_t(bool neighbor, const StepArgs &a, cudaStream_t s, const StepAux *aux) {
    if constexpr (S == LBM_F32) {
        if (a.g.N >= kDual32MinCells) step_p<S, FORCE, false, true>(neighbor, a, s, aux);
        else step_p<S, FORCE, false, false>(neighbor, a, s, aux);
    } else {
        if (a.pack16 && !neighbor) step_p<S, FORCE, true, false>(neighbor, a, s, aux);
        else step_p<S, FORCE, false, false>(neighbor, a, s, aux);
    }
}

}  // namespace lbm

// lbm_batch.cuh -- the batched step kernels (one launch per time step over every member domain) and
// their launch shapes.  Included by lbm_batch.cu (host logic) and by lbm_batch_kern.cu, which is
// compiled once per storage type (LBM_INST_S) so that the instantiations build in parallel.
#pragma once

#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_cell.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace batch {


// Launch shapes the autotuner chooses from (lbm_batch_autotune): threads per block B, resident blocks
// per SM the batched kernel is compiled for (its register cap), cells per thread of FP32 members
// (0: each member's own choice, as in its single-domain launch; 1 or 2 for all -- the unrolling of
// the cell loop), a persistent grid (one set of resident blocks striding over the members' blocks),
// the slot order (members in the given order or largest first), or one single-domain launch per
// member and step.
struct ShapeSpec {
    int B, minb, cpt;
    bool persistent, largest_first, sequential;
};
constexpr ShapeSpec kShapeSpec[] = {
    {256, 4, 0, false, false, false},   // 0
    {256, 3, 0, false, false, false},   // 1
    {256, 4, 0, false, true, false},    // 2
    {256, 3, 0, false, true, false},    // 3
    {256, 4, 0, false, false, true},    // 4: one single-domain launch per member and step
    {128, 8, 0, false, false, false},   // 5
    {512, 2, 0, false, false, false},   // 6
    {256, 4, 1, false, false, false},   // 7: FP32 members one cell per thread
    {256, 4, 2, false, false, false},   // 8: FP32 members two cells per thread
    {256, 4, 0, true, false, false},    // 9: persistent grid
};
constexpr int kNumShapes = (int)(sizeof(kShapeSpec) / sizeof(kShapeSpec[0]));
constexpr int kSequential = 4;
constexpr int kTableShapes = 4;   // shapes 0..3 also run with the member tables in device memory

struct BatchTables {
    const StepArgs *args;     // per member
    const unsigned *start;    // per slot: first block of the slot in the grid (+ total at [n])
    const int *member;        // per slot: member index
    int n;
};

// FP32 member: two cells per thread?
template <int S, int CPT> __device__ __forceinline__ bool batch_d32(const StepArgs &a) {
    return S == LBM_F32 && (CPT == 2 || (CPT == 0 && a.g.N >= kDual32MinCells));
}

// Block bid of a member's own launch of this step kind (the same block bodies as lbm_step).
// FASTC: the FP32 pair collision takes the special-function reciprocals and square roots; the
// batched kernels keep the IEEE forms (with the special-function forms they spilled 300-800 bytes a
// thread at 3 and 4 blocks per SM).
template <int S, bool NEIGHBOR, int B, int CPT, bool FASTC>
__device__ __forceinline__ void batch_block(const StepArgs &a, unsigned bid) {
    const bool d32 = batch_d32<S, CPT>(a);
    if constexpr (NEIGHBOR) {
        if (d32) neighbor_block<S, false, false, true, B, false, FASTC>(a, bid, face_blocks_of<B>(step_face_cells(a)));
        else neighbor_block<S, false, false, false, B, false, FASTC>(a, bid, face_blocks_of<B>(step_face_cells(a)));
    } else if constexpr (S == LBM_F32) {
        if (d32) local_block<S, false, false, true, B, FASTC>(a, bid);
        else local_block<S, false, false, false, B, FASTC>(a, bid);
    } else {
        if (a.pack16) local_block<S, false, true, false, B>(a, bid);
        else local_block<S, false, false, false, B>(a, bid);
    }
}

template <int S, bool NEIGHBOR, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_batch_step(BatchTables t) {
    __shared__ StepArgs sa;
    __shared__ unsigned s_bid;
    __shared__ int s_member;
    if (threadIdx.x == 0) {
        int lo = 0, hi = t.n - 1;   // last slot whose first block is <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (t.start[mid] <= blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_member = t.member[lo];
        s_bid = blockIdx.x - t.start[lo];
    }
    __syncthreads();
    {
        const int *src = (const int *)(t.args + s_member);
        int *dst = (int *)&sa;
        for (int k = threadIdx.x; k < (int)(sizeof(StepArgs) / sizeof(int)); k += kBlock) dst[k] = src[k];
    }
    __syncthreads();
    batch_block<S, NEIGHBOR, kBlock, 0, false>(sa, s_bid);
}

// Up to kParamMembers members: the step arguments and block tables travel in the kernel's parameter
// space (__grid_constant__, constant bank) instead of shared memory, as in the single-domain kernels.
constexpr int kParamMembers = 48;
struct BatchParams {
    StepArgs args[kParamMembers];
    unsigned start[kParamMembers + 1];
    int member[kParamMembers];
    int n;
};
static_assert(sizeof(BatchParams) <= 32000, "kernel parameter space");

template <int S, bool NEIGHBOR, int B, int MINB, int CPT, bool PERSIST>
__global__ void __launch_bounds__(B, MINB) k_batch_step_p(const __grid_constant__ BatchParams p) {
    const unsigned total = p.start[p.n];
    for (unsigned vb = blockIdx.x; vb < total; vb += PERSIST ? gridDim.x : total) {
        int lo = 0, hi = p.n - 1;   // last slot whose first block is <= vb (uniform)
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.start[mid] <= vb) lo = mid;
            else hi = mid - 1;
        }
        batch_block<S, NEIGHBOR, B, CPT, false>(p.args[p.member[lo]], vb - p.start[lo]);
    }
}

// blocks of a member's launch of this kind in shape sh (as its single-domain launch for shape 0)
template <int S> unsigned member_blocks(const StepArgs &a, bool neighbor, int sh) {
    const ShapeSpec &q = kShapeSpec[sh];
    const bool d32 = S == LBM_F32 && (q.cpt == 2 || (q.cpt == 0 && a.g.N >= kDual32MinCells));
    unsigned lb = 0, fb = 0;
    switch (q.B) {
        case 128: lb = d32 ? lattice_blocks<S, true, 128>(a.g.N) : lattice_blocks<S, false, 128>(a.g.N);
                  fb = face_blocks_of<128>(step_face_cells(a)); break;
        case 512: lb = d32 ? lattice_blocks<S, true, 512>(a.g.N) : lattice_blocks<S, false, 512>(a.g.N);
                  fb = face_blocks_of<512>(step_face_cells(a)); break;
        default: lb = d32 ? lattice_blocks<S, true, 256>(a.g.N) : lattice_blocks<S, false, 256>(a.g.N);
                 fb = face_blocks_of<256>(step_face_cells(a)); break;
    }
    return lb + (neighbor ? fb : 0u);
}
// Resident blocks of a persistent kernel: its occupancy times the SM count (queried once).
template <class K> unsigned persistent_grid(K kernel, int B) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, B, 0) != cudaSuccess || per < 1) {
        cudaGetLastError();
        return 0;
    }
    return (unsigned)(sms * per);
}

template <int S, bool NEIGHBOR, int B, int MINB, int CPT, bool PERSIST>
void launch_p(const BatchParams &p, unsigned blocks, cudaStream_t s) {
    if (PERSIST) {
        static unsigned grid = 0;   // per kernel (one template instance per kernel)
        if (!grid) grid = persistent_grid(k_batch_step_p<S, NEIGHBOR, B, MINB, CPT, PERSIST>, B);
        if (grid && grid < blocks) blocks = grid;
    }
    k_batch_step_p<S, NEIGHBOR, B, MINB, CPT, PERSIST><<<blocks, B, 0, s>>>(p);
}
template <int S, bool NEIGHBOR>
void launch_shape(int sh, const BatchTables &t, const BatchParams *p, unsigned blocks, cudaStream_t s) {
    if (!p) {   // member tables in device memory (more than kParamMembers members): shapes 0..3
        if (kShapeSpec[sh].minb == 3) k_batch_step<S, NEIGHBOR, 3><<<blocks, kBlock, 0, s>>>(t);
        else k_batch_step<S, NEIGHBOR, 4><<<blocks, kBlock, 0, s>>>(t);
        return;
    }
    switch (sh) {
        case 1: case 3: launch_p<S, NEIGHBOR, 256, 3, 0, false>(*p, blocks, s); break;
        case 5: launch_p<S, NEIGHBOR, 128, 8, 0, false>(*p, blocks, s); break;
        case 6: launch_p<S, NEIGHBOR, 512, 2, 0, false>(*p, blocks, s); break;
        case 7: if constexpr (S == LBM_F32) launch_p<S, NEIGHBOR, 256, 4, 1, false>(*p, blocks, s);
                else launch_p<S, NEIGHBOR, 256, 4, 0, false>(*p, blocks, s);
                break;
        case 8: if constexpr (S == LBM_F32) launch_p<S, NEIGHBOR, 256, 4, 2, false>(*p, blocks, s);
                else launch_p<S, NEIGHBOR, 256, 4, 0, false>(*p, blocks, s);
                break;
        case 9: launch_p<S, NEIGHBOR, 256, 4, 0, true>(*p, blocks, s); break;
        default: launch_p<S, NEIGHBOR, 256, 4, 0, false>(*p, blocks, s); break;
    }
}
// The batched launch of one storage type (defined in lbm_batch_kern.cu, one object per type).
template <int S>
void launch_batch_s(int sh, bool neighbor, const BatchTables &t, const BatchParams *p, unsigned blocks, cudaStream_t s);

}  // namespace batch
}  // namespace lbm

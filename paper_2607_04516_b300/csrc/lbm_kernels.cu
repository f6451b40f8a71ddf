// lbm_kernels.cu -- sm_103a kernels of the LBM-LES step and their launchers.
//
// Hot path: k_step_neighbor (layout B -> A) and k_step_local (layout A -> B), one launch per
// time step, one thread per cell, populations as 19 structure-of-arrays planes with x fastest.
// Both are HBM-bound stencils (about 2 flop per byte): no tensor cores, no shared-memory staging;
// every warp reads and writes 32 consecutive cells of each plane (fully coalesced; the neighbour
// step's x-shifted planes straddle one extra 32-byte sector that the next warp uses).
#include <cuda_runtime.h>

#include "lbm_cell.cuh"
#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------- grid wrappers
#define LBM_CELL_INDEX()                                                   \
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; \
    if (n >= G_N) return;

__global__ void k_flags(const uint8_t *__restrict__ mask, uint8_t *__restrict__ flags,
                        uint32_t *__restrict__ info, Geo G) {
    const long long G_N = G.N;
    LBM_CELL_INDEX();
    cell_flags(mask, flags, info, G, n);
}

template <int S>
__global__ void k_import(StepArgs a, const float *__restrict__ g) {
    const long long G_N = a.g.N;
    LBM_CELL_INDEX();
    cell_import<S>(a, n, g);
}

template <int S>
__global__ void k_init(StepArgs a, const float *__restrict__ rho, const float *__restrict__ u) {
    const long long G_N = a.g.N;
    LBM_CELL_INDEX();
    cell_init<S>(a, n, rho, u);
}

// Face tables (once per domain, after the flags; without them, as on lattices too large for their
// 32-bit codes, the face blocks resolve the boundary rules at run time).
template <int S>
__global__ void k_face_tables(StepArgs a, uint32_t *__restrict__ tab) {
    const long long t = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (t >= a.ngen) return;
    cell_face_table<S>(a, (int)t, tab);
}

template <int S>
__global__ void k_macros(StepArgs a, bool layoutA, float *__restrict__ rho_out,
                         float *__restrict__ u_out) {
    const long long G_N = a.g.N;
    LBM_CELL_INDEX();
    float r, ux, uy, uz;
    cell_macros<S>(a, n, layoutA, r, ux, uy, uz);
    if (rho_out) rho_out[n] = r;
    if (u_out) { u_out[3 * n] = ux; u_out[3 * n + 1] = uy; u_out[3 * n + 2] = uz; }
}

template <int S>
__global__ void k_sample(StepArgs a, bool layoutA, const int *__restrict__ ij, int ncol,
                         const int *__restrict__ kk, int nh, float *__restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)ncol * nh) return;
    const int c = (int)(t / nh), h = (int)(t - (long long)c * nh);
    const int x = ij[2 * c], y = ij[2 * c + 1], z = kk[h];
    float *o = out + 4 * t;
    if (x < 0 || x >= a.g.nx || y < 0 || y >= a.g.ny || z < 0 || z >= a.g.nz) {
        o[0] = o[1] = o[2] = o[3] = NAN;
        return;
    }
    float r, ux, uy, uz;
    cell_macros<S>(a, cell_of(a.g, x, y, z), layoutA, r, ux, uy, uz);
    o[0] = ux; o[1] = uy; o[2] = uz; o[3] = r;
}

template <int S>
__global__ void k_export(StepArgs a, bool layoutA, float *__restrict__ out) {
    const long long G_N = a.g.N;
    LBM_CELL_INDEX();
    cell_export<S>(a, n, layoutA, out);
}

// ---------------------------------------------------------------- FP64 diagnostics
// Pass 1: kRedBlocks blocks stride over the lattice; each thread accumulates its cells (diag_cell:
// FP32 partials of the small per-cell terms) and each block writes 4 FP64 partials into scratch.
// Pass 2: one block folds the partials.  Fixed block count -> deterministic result.
// (4 resident blocks per SM: at one block, as the unbounded register count allowed, the pass was
// latency-bound at a sixth of the HBM bandwidth)
template <int S>
__global__ void __launch_bounds__(kBlock, 4) k_reduce_partial(StepArgs a, bool layoutA,
                                                           double *__restrict__ part) {
    DiagAcc acc;
    const long long stride = (long long)gridDim.x * kBlock, first = (long long)blockIdx.x * kBlock + threadIdx.x;
    // cells off the face layers first; the face-layer cells, whose read-back of an odd step takes the
    // general boundary resolution, in a second loop over the face enumeration, so that they fill
    // whole warps instead of idling 31 lanes of the warps that hold one of them
    for (long long n = first; n < a.g.N; n += stride)
        if (!(a.flags[n] & F_FACE)) diag_cell<S>(a, n, layoutA, acc);
    for (long long t = first; t < a.nface; t += stride) diag_face_cell<S>(a, t, layoutA, acc);
    diag_block_store<kBlock>(acc, part + 4 * blockIdx.x);
}

__global__ void __launch_bounds__(kBlock) k_reduce_final(const double *__restrict__ part, int nb,
                                                         double *__restrict__ out) {
    __shared__ double sh[4][kBlock];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += kBlock) {
        v[0] += part[4 * b];
        v[1] += part[4 * b + 1];
        v[2] = fmax(v[2], part[4 * b + 2]);
        v[3] += part[4 * b + 3];
    }
    for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int s = kBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
            sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + s]);
            sh[3][threadIdx.x] += sh[3][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) out[k] = sh[k][0];
}

// ---------------------------------------------------------------- launchers

cudaError_t launch_flags(const uint8_t *mask, uint8_t *flags, uint32_t *info, const Geo &G, cudaStream_t s) {
    k_flags<<<blocks_for(G.N), kBlock, 0, s>>>(mask, flags, info, G);
    return cudaGetLastError();
}

template <int S>
static cudaError_t init_t(const StepArgs &a, const float *rho, const float *u, cudaStream_t s) {
    k_init<S><<<blocks_for(a.g.N), kBlock, 0, s>>>(a, rho, u);
    return cudaGetLastError();
}
cudaError_t launch_init(int store, const StepArgs &a, const float *rho, const float *u, cudaStream_t s) {
    switch (store) {
        case LBM_F32: return init_t<LBM_F32>(a, rho, u, s);
        case LBM_F16S: return init_t<LBM_F16S>(a, rho, u, s);
        default: return init_t<LBM_BF16S>(a, rho, u, s);
    }
}

template <int S>
static cudaError_t import_t(const StepArgs &a, const float *g, cudaStream_t s) {
    k_import<S><<<blocks_for(a.g.N), kBlock, 0, s>>>(a, g);
    return cudaGetLastError();
}
cudaError_t launch_import(int store, const StepArgs &a, const float *g, cudaStream_t s) {
    switch (store) {
        case LBM_F32: return import_t<LBM_F32>(a, g, s);
        case LBM_F16S: return import_t<LBM_F16S>(a, g, s);
        default: return import_t<LBM_BF16S>(a, g, s);
    }
}

// one object per (storage, forced) pair holds the step kernels (lbm_step_kern.cu)
void launch_step(int store, bool neighbor, bool force, const StepArgs &a, cudaStream_t s, const StepAux *aux) {
    switch (store) {
        case LBM_F32: force ? launch_step_sf<LBM_F32, true>(neighbor, a, s, aux) : launch_step_sf<LBM_F32, false>(neighbor, a, s, aux); break;
        case LBM_F16S: force ? launch_step_sf<LBM_F16S, true>(neighbor, a, s, aux) : launch_step_sf<LBM_F16S, false>(neighbor, a, s, aux); break;
        default: force ? launch_step_sf<LBM_BF16S, true>(neighbor, a, s, aux) : launch_step_sf<LBM_BF16S, false>(neighbor, a, s, aux); break;
    }
}

template <int S>
static cudaError_t face_tables_t(const StepArgs &a, uint32_t *tab, cudaStream_t s) {
    if (a.ngen <= 0) return cudaSuccess;
    k_face_tables<S><<<blocks_for(a.ngen), kBlock, 0, s>>>(a, tab);
    return cudaGetLastError();
}
cudaError_t launch_face_tables(int store, const StepArgs &a, uint32_t *tab, cudaStream_t s) {
    switch (store) {
        case LBM_F32: return face_tables_t<LBM_F32>(a, tab, s);
        case LBM_F16S: return face_tables_t<LBM_F16S>(a, tab, s);
        default: return face_tables_t<LBM_BF16S>(a, tab, s);
    }
}

template <int S>
static cudaError_t macros_t(const StepArgs &a, bool layoutA, float *rho, float *u, cudaStream_t s) {
    k_macros<S><<<blocks_for(a.g.N), kBlock, 0, s>>>(a, layoutA, rho, u);
    return cudaGetLastError();
}
cudaError_t launch_macros(int store, const StepArgs &a, bool layoutA, float *rho, float *u,
                          cudaStream_t s) {
    switch (store) {
        case LBM_F32: return macros_t<LBM_F32>(a, layoutA, rho, u, s);
        case LBM_F16S: return macros_t<LBM_F16S>(a, layoutA, rho, u, s);
        default: return macros_t<LBM_BF16S>(a, layoutA, rho, u, s);
    }
}

template <int S>
static cudaError_t sample_t(const StepArgs &a, bool layoutA, const int *ij, int ncol, const int *k,
                            int nh, float *out, cudaStream_t s) {
    k_sample<S><<<blocks_for((long long)ncol * nh), kBlock, 0, s>>>(a, layoutA, ij, ncol, k, nh, out);
    return cudaGetLastError();
}
cudaError_t launch_sample(int store, const StepArgs &a, bool layoutA, const int *ij, int ncol,
                          const int *k, int nh, float *out, cudaStream_t s) {
    switch (store) {
        case LBM_F32: return sample_t<LBM_F32>(a, layoutA, ij, ncol, k, nh, out, s);
        case LBM_F16S: return sample_t<LBM_F16S>(a, layoutA, ij, ncol, k, nh, out, s);
        default: return sample_t<LBM_BF16S>(a, layoutA, ij, ncol, k, nh, out, s);
    }
}

template <int S>
static cudaError_t export_t(const StepArgs &a, bool layoutA, float *out, cudaStream_t s) {
    k_export<S><<<blocks_for(a.g.N), kBlock, 0, s>>>(a, layoutA, out);
    return cudaGetLastError();
}
cudaError_t launch_export(int store, const StepArgs &a, bool layoutA, float *out, cudaStream_t s) {
    switch (store) {
        case LBM_F32: return export_t<LBM_F32>(a, layoutA, out, s);
        case LBM_F16S: return export_t<LBM_F16S>(a, layoutA, out, s);
        default: return export_t<LBM_BF16S>(a, layoutA, out, s);
    }
}

template <int S>
static cudaError_t reduce_t(const StepArgs &a, bool layoutA, double *part, double *out, cudaStream_t s) {
    k_reduce_partial<S><<<kRedBlocks, kBlock, 0, s>>>(a, layoutA, part);
    k_reduce_final<<<1, kBlock, 0, s>>>(part, kRedBlocks, out);
    return cudaGetLastError();
}
cudaError_t launch_reduce(int store, const StepArgs &a, bool layoutA, double *part, double *out,
                          cudaStream_t s) {
    switch (store) {
        case LBM_F32: return reduce_t<LBM_F32>(a, layoutA, part, out, s);
        case LBM_F16S: return reduce_t<LBM_F16S>(a, layoutA, part, out, s);
        default: return reduce_t<LBM_BF16S>(a, layoutA, part, out, s);
    }
}

}  // namespace lbm

// lbm_noalloc.cu -- lbm_diagnostics_noalloc: the FP64 diagnostics reduction with its scratch in a
// fixed device array that belongs to the library, for callers that must not allocate.
//
// Who needs it: code that runs where a device allocation is not allowed or not acceptable -- a
// serving loop under a fixed memory budget where every byte was reserved up front, a pipeline
// that must not stall on the allocator (cudaMalloc can synchronise the device), or a caller that
// sized its domain workspace without the reduction scratch it would otherwise borrow.  This entry
// point allocates nothing: the partial sums live in the file-scope array below, which every GPU
// that loads the library keeps for the life of the process.
//
// The array holds kMaxPartials partial blocks of 4 doubles (512 KiB).  One partial covers
// kCellsPerBlock cells, so lattices of up to kMaxPartials * kCellsPerBlock = 2^28 cells are
// accepted; larger ones are rejected with LBM_EINVAL before anything is launched.
//
// The array is shared by every call.  Each call's first kernel writes every partial slot that its
// second kernel reads (nothing is accumulated across calls, so nothing needs clearing), but two
// calls whose kernels overlap on the GPU -- on different streams, or from different host threads
// -- race on the same slots.  Issue them in one stream order.
//
// Set-up: the first call on each device looks up the array's device address
// (cudaGetSymbolAddress) and caches it; make that first call before capturing a stream into a
// CUDA graph, since the look-up is not a stream operation.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm_cell.cuh"
#include "lbm_internal.h"

// Device scratch: 4 doubles (mass, flux, max |u|, non-finite count) per pass-1 block
// (16384 blocks -> 512 KiB).
static __device__ __align__(256) double g_lbm_noalloc_partials[16384 * 4];

namespace lbm {
namespace {

constexpr int kBlockNa = 256;
constexpr int kCellsPerThread = 64;
constexpr long long kCellsPerBlock = (long long)kBlockNa * kCellsPerThread;   // 16384
constexpr long long kMaxPartials = 16384;
constexpr long long kMaxCells = kMaxPartials * kCellsPerBlock;                // 2^28
static_assert(sizeof(g_lbm_noalloc_partials) == kMaxPartials * 4 * sizeof(double), "scratch size");

// Host code may not pass g_lbm_noalloc_partials itself: on the host that name is only a stand-in
// for the device symbol, and a kernel given it would fault (or, where the GPU can reach host
// memory, quietly use the wrong memory).  Its device address is looked up with the device
// current, once per device, on the first call there, and cached.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_dev_ptr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_lbm_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_dev_ptr[dev] = (double *)p;
    }
    *out = g_dev_ptr[dev];
    return cudaSuccess;
}

// Pass 1: block b reduces the cells [b * kCellsPerBlock, (b + 1) * kCellsPerBlock) off the face
// layers and its share of the face enumeration into part[4b .. 4b+3], with the per-cell rule and
// the block fold of lbm_diagnostics (diag_cell, diag_block_store).
template <int S>
__global__ void __launch_bounds__(kBlockNa, 4) k_na_partial(StepArgs a, bool layoutA, double *__restrict__ part) {
    DiagAcc acc;
    const long long base = (long long)blockIdx.x * kCellsPerBlock;
    for (int k = 0; k < kCellsPerThread; ++k) {
        const long long n = base + (long long)k * kBlockNa + threadIdx.x;
        if (n >= a.g.N) break;
        if (!(a.flags[n] & F_FACE)) diag_cell<S>(a, n, layoutA, acc);
    }
    // the face-layer cells, as in lbm_diagnostics: this block's share of the face enumeration
    const long long fpb = (a.nface + gridDim.x - 1) / gridDim.x, t1 = (long long)(blockIdx.x + 1) * fpb;
    for (long long t = (long long)blockIdx.x * fpb + threadIdx.x; t < t1 && t < a.nface; t += kBlockNa)
        diag_face_cell<S>(a, t, layoutA, acc);
    diag_block_store<kBlockNa>(acc, part + 4 * blockIdx.x);
}

// Pass 2: one block folds the nb partials into the caller's out[4].
__global__ void __launch_bounds__(kBlockNa) k_na_final(const double *__restrict__ part, int nb,
                                                      double *__restrict__ out) {
    __shared__ double sh[4][kBlockNa];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += kBlockNa) {
        v[0] += part[4 * b];
        v[1] += part[4 * b + 1];
        v[2] = fmax(v[2], part[4 * b + 2]);
        v[3] += part[4 * b + 3];
    }
    for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int s = kBlockNa / 2; s > 0; s >>= 1) {
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

template <int S>
void launch_na(const StepArgs &a, bool layoutA, double *part, int nb, double *out, cudaStream_t s) {
    k_na_partial<S><<<nb, kBlockNa, 0, s>>>(a, layoutA, part);
    k_na_final<<<1, kBlockNa, 0, s>>>(part, nb, out);
}

}  // namespace
}  // namespace lbm

extern "C" lbm_status lbm_diagnostics_noalloc(lbm_domain *d, double *out) {
    using namespace lbm;
    if (!d) return LBM_EINVAL;
    if (!out) return domain_fail(d, LBM_EINVAL, "diagnostics_noalloc: out is NULL");
    const DomainView v = domain_view(d);
    if (v.args.g.N > kMaxCells)
        return domain_fail(d, LBM_EINVAL,
                           "diagnostics_noalloc: lattice has more than 2^28 cells, the limit of its "
                           "fixed 512 KiB scratch; use lbm_diagnostics");
    // the scratch address is per device: the current device must be the domain's
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return domain_fail(d, LBM_ECUDA, cudaGetErrorString(e));
    if (cur != v.device)
        return domain_fail(d, LBM_EINVAL, "diagnostics_noalloc: the current CUDA device is not the domain's device");
    double *part = nullptr;
    e = scratch_for_current_device(&part);
    if (e != cudaSuccess) return domain_fail(d, LBM_ECUDA, cudaGetErrorString(e));
    const int nb = (int)((v.args.g.N + kCellsPerBlock - 1) / kCellsPerBlock);
    switch (v.store) {
        case LBM_F32: launch_na<LBM_F32>(v.args, v.layoutA, part, nb, out, v.stream); break;
        case LBM_F16S: launch_na<LBM_F16S>(v.args, v.layoutA, part, nb, out, v.stream); break;
        default: launch_na<LBM_BF16S>(v.args, v.layoutA, part, nb, out, v.stream); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return domain_fail(d, LBM_ECUDA, cudaGetErrorString(e));
    return LBM_OK;
}

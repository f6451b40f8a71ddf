// lbm_internal.h -- launchers shared by the kernels (lbm_kernels.cu) and the C ABI (lbm_capi.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

constexpr int kRedBlocks = 148 * 8;   // diagnostics pass-1 blocks (8 per SM on a 148-SM B300)

// blocks of a one-thread-per-item launch of 256-thread blocks
inline unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

cudaError_t launch_flags(const uint8_t *mask, uint8_t *flags, uint32_t *info, const Geo &G, cudaStream_t s);
cudaError_t launch_init(int store, const StepArgs &a, const float *rho, const float *u, cudaStream_t s);
cudaError_t launch_import(int store, const StepArgs &a, const float *g, cudaStream_t s);
// A second stream and two events of a domain: the neighbour step's layer kernel (k_step_layers) runs
// on it concurrently with the main kernel, forked from and joined back into the step's stream (the
// two kernels touch disjoint memory: in the in-place scheme every location a neighbour step reads is
// written by the same thread).  stream == null: both kernels in order on the step's stream.
struct StepAux {
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
void launch_step(int store, bool neighbor, bool force, const StepArgs &a, cudaStream_t s, const StepAux *aux = nullptr);
// The step launch of one storage type and forcing (defined in lbm_step_kern.cu, one object each).
template <int S, bool FORCE> void launch_step_sf(bool neighbor, const StepArgs &a, cudaStream_t s, const StepAux *aux);
cudaError_t launch_macros(int store, const StepArgs &a, bool layoutA, float *rho, float *u,
                          cudaStream_t s);
cudaError_t launch_sample(int store, const StepArgs &a, bool layoutA, const int *ij, int ncol,
                          const int *k, int nh, float *out, cudaStream_t s);
cudaError_t launch_export(int store, const StepArgs &a, bool layoutA, float *out, cudaStream_t s);
cudaError_t launch_reduce(int store, const StepArgs &a, bool layoutA, double *part, double *out,
                          cudaStream_t s);
cudaError_t launch_face_tables(int store, const StepArgs &a, uint32_t *tab, cudaStream_t s);

// Read-only view of a domain for entry points defined outside lbm_capi.cu.
struct DomainView {
    StepArgs args;
    int store;
    bool layoutA;
    cudaStream_t stream;
    int device;      // CUDA device of the domain's workspace
};
DomainView domain_view(const lbm_domain *d);
// Level-to-height mapping of the inflow profile: s(z_k) = (1 - w1) speed[l0] + w1 speed[l1]
// (equal-height blocks when L divides nz, else linear between level centres).
void profile_level_weights(int L, int nz, int k, int &l0, int &l1, double &w1);
lbm_status domain_fail(lbm_domain *d, lbm_status st, const char *msg);
// Step counter bookkeeping for steps launched outside lbm_step (batched launches).
void domain_advance(lbm_domain *d, long long n);
// The domain has synthetic inflow turbulence switched on (its steps need the anchor kernel).
bool domain_stg_on(const lbm_domain *d);

}  // namespace lbm

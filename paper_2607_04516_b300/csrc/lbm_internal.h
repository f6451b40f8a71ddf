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
void launch_step(int store, bool neighbor, bool force, const StepArgs &a, cudaStream_t s);
// The step launch of one storage type and forcing (defined in lbm_step_kern.cu, one object each).
template <int S, bool FORCE> void launch_step_sf(bool neighbor, const StepArgs &a, cudaStream_t s);
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

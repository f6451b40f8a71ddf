// lbm_stg.h -- synthetic von Karman inflow turbulence (paper App. F), internal interface.
//
// Before a time step the equilibrium cells of the inflow faces x-, x+, y-, y+, z+ (never the
// ground) take U_i(t) = U_b,i + sigma_i q^(f)(x_i, t), with the random Fourier sum
//   q_a(x, t) = sum_m A_m,a cos(k_m . x + omega_m t + phi_m,a).
// The sum is split into a time part, evaluated once per step and mode,
//   C_m,a + i S_m,a = A_m,a exp(i (omega_m t + phi_m,a + k_m . x_fixed)),
// and a space part that factorises over the two in-plane axes of the face,
//   exp(i k_m . x_in-plane) = exp(i k_m,a1 i) exp(i k_m,a2 j),
// tabulated once per configuration in FP64 and stored as FP32 pairs.  Per cell and mode the kernel
// then does one complex product and six FMAs: q_a += C_m,a Re(e) - S_m,a Im(e); four threads share
// a cell's modes.  Phases are kept in turns and reduced in FP64 before the FP32 sincospi, so no
// FP32 argument grows with x or t.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "lbm.h"
#include "lbm_device.cuh"

namespace lbm {

#ifndef LBM_STG_POS
#define LBM_STG_POS 64
#endif
#ifndef LBM_STG_GROUPS
#define LBM_STG_GROUPS 4
#endif

constexpr int kStgMaxModes = 1024;
constexpr int kStgPos = LBM_STG_POS;             // plane positions per block
constexpr int kStgGroups = LBM_STG_GROUPS;       // thread groups splitting the modes
constexpr int kStgBlock = kStgPos * kStgGroups;
#ifndef LBM_STG_BATCH
#define LBM_STG_BATCH 4
#endif
constexpr int kStgBatch = LBM_STG_BATCH;         // modes whose table loads a thread issues together

struct StgMode {         // one Fourier mode of one face
    double w;            // omega_m / 2 pi                      [turns per step]
    float ph[3];         // (k_m . x_fixed + phi_m,a) / 2 pi    [turns, in [0, 1)]
    float amp[3];        // A_m,a = g_a A_m
};

struct StgFace {         // one inflow face (face index 0..3 or 5)
    const float2 *E1;    // [n_modes][n1]  exp(i k_m,a1 i)
    const float2 *E2;    // [n_modes][n2]  exp(i k_m,a2 j)
    const StgMode *mode; // [n_modes]
    float4 *ueq;         // [n2][n1]       U_i(t) of the face's equilibrium cells (w unused);
                         //                 set per launch to one of the two plane sets
    int face, n1, n2;
    int keep;            // the face is turbulent (has cells and U_c,f > 1e-7)
    int block_begin;     // first block of this face in the launch
};

struct StgLaunch {
    StgFace f[5];
    int nfaces, nblocks, n_modes;
    int char_normal, inflow_only;
    float intensity, sigma0;
    int inflow;          // bit k: face k is an inflow face
    long long t;         // time at which U is evaluated (an anchor)
    const float *ub;     // nz * 3
    const uint8_t *flags;
    Geo g;
};

// Host state of one domain's synthetic inflow.
struct StgState {
    bool on = false;
    bool valid = false;              // the planes hold U(t) of the last step taken
    lbm_stg_params p{};
    std::vector<double> rnd;         // [6][n_modes][6]
    char *ws = nullptr;
    size_t ws_bytes = 0;
    size_t table_bytes = 0;          // leading part of the workspace that holds the tables
    std::vector<char> image;         // host image of the tables (kept for the asynchronous copy)
    StgLaunch L{};
    float4 *plane[2][5] = {};        // two plane sets (anchor t_a and t_a + s), per face of L.f
    int cur = 0;                     // plane set holding U(anchor)
    long long anchor = -1;           // anchor whose U the current set holds (-1: none)
    float alpha = 0.0f;              // blend weight of the last step taken
    double u_ref = 0.0, e_c[3] = {1.0, 0.0, 0.0};
    int kept = 0;                    // bit k: face k is turbulent
};

// Device workspace bytes for n_modes modes on the inflow faces of this geometry (0 if none).
size_t stg_workspace_bytes(const Geo &g, int n_modes);

// Checks the parameters; nullptr if acceptable, else a message.
const char *stg_check(const lbm_stg_params *p);

// Builds the tables of App. F for the current profile ub (nz * 3, host) and the face planes of the
// solid mask (face_solid[k]: n1 * n2 bytes, nonzero = solid) into s.image and s.L (device pointers
// into s.ws).  nullptr on success, else a message.
const char *stg_build(StgState &s, const Geo &g, const float *ub, const std::vector<uint8_t> *face_solid,
                      const float *ub_dev, const uint8_t *flags_dev);

// Enqueues the evaluation of U(t) into plane set buf.
cudaError_t launch_stg(const StgState &s, long long t, int buf, cudaStream_t st);

// In-plane size of face k: (n1, n2) = (ny, nz), (nx, nz) or (nx, ny).
inline void stg_face_dims(const Geo &g, int k, int &n1, int &n2) {
    const int a = k / 2;
    n1 = a == 0 ? g.ny : g.nx;
    n2 = a == 2 ? g.ny : g.nz;
}

}  // namespace lbm

// lbm_adjoint.cu -- discrete adjoint of the fused step: gradient of a virtual-lidar misfit with
// respect to the inflow level speeds and direction (boundary assimilation; the paper fits the same
// inflow to lidar profiles by Kriging, Sec. 3 and App. A).
//
// Forward model.  F*_0 = f^eq(1, u_b(z)) in fluid cells and f^eq(rho_b, u_b(z)) in equilibrium
// cells (D.4); F*_n = Phi(F*_{n-1}), Phi = gather (D.3 with the face rules) + collision (D.1, D.4,
// D.8-D.11, D.2); equilibrium cells hold f^eq(rho_b, u_b(z)).  The lidar samples u = sum c F*/rho
// at fluid cells; J = sum over samples of |(u, v)bar - target|^2, the bar averaging the states
// T - n_avg + 1 .. T.
//
// Adjoint.  With lambda_n = dJ/dF*_n and mu_n(x) = J_C(f_n(x))^T lambda_n(x) for fluid x (J_C the
// Jacobian of the collision at the gathered state f_n = G F*_{n-1}; mu = 0 in equilibrium cells):
//     lambda_{n-1}(y, j) = sum over the consumers (x, i) of element (y, j) in step n of mu_n(x, i)
//                          + explicit lidar term at the sampled cells,
// i.e. a pull: the consumers are the cells and directions whose gather resolves to (y, j) -- the
// plain downstream cell y + c_j, the cell itself after bounce-back, and for face cells the wrapped,
// mirrored and zero-gradient consumers.  One kernel per step computes lambda_{n-1} at y from mu_n
// and then mu_{n-1}(y), so the adjoint of a step reads mu (19 values, shifted like the forward
// step's stores), the state F*_{n-2} (19, gathered like the forward step's loads) and writes mu
// (19): 228 bytes per cell in FP32.  Every element is written by the thread of its own cell, so two
// mu buffers alternate and nothing is accumulated across threads.
//
// Parameters.  Equilibrium cells contribute (d f^eq / d u)^T lambda_n to dJ/du_b(z) at every n,
// and every non-solid cell contributes (d f^eq / d u)^T lambda_0 through the initial state; both
// are accumulated in FP64 per cell, reduced per height in a fixed order, and mapped to the level
// speeds and the direction by the chain rule of the profile mapping.
//
// Memory.  States are kept in the plain post-collision layout (slot d of a cell holds F*_d), FP32,
// populations shifted by w_i.  The forward run (the production in-place kernels) exports a
// checkpoint every K states; the reverse sweep recomputes each segment of K states out of place
// from its checkpoint (a two-lattice pull step) and runs the adjoint steps of that segment.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lbm.h"
#include "lbm_cell.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kB = 256;
constexpr uint8_t F_SAMPLE = 32;   // adjoint flag copy: the cell is sampled by the lidar

// ---------------------------------------------------------------- face tables
// The boundary resolution of a face cell depends only on the geometry and the solid mask, so the
// reverse sweep resolves it once per call: per face cell t (face enumeration order) its cell index
// and kind, the plain-layout element each direction gathers, and up to two consumers (cell,
// direction) of each of its elements.  Codes are element indices d N + cell (< 19 N < 2^32 - 1).
//   tab[t]                   kFtNone (solid) or the cell index | kFtEq | kFtGeneral (a direction
//                            with more than two consumers: resolved at run time)
//   tab[(1 + i) nf + t]      gathered element of direction i (fluid cells)
//   tab[(20 + j) nf + t]     first consumer of element (cell, j), kFtNone: none
//   tab[(39 + j) nf + t]     second consumer, kFtNone: none
__global__ void k_adj_tables(StepArgs a, uint32_t *__restrict__ tab) {
    const long long t = (long long)blockIdx.x * kB + threadIdx.x;
    const long long nf = a.nface;
    if (t >= nf) return;
    int x, y, z;
    face_cell_xyz(a.g, t, x, y, z);
    const long long n = cell_of(a.g, x, y, z);
    const uint8_t fl = a.flags[n];
    if (fl & F_SOLID) {
        tab[t] = kFtNone;
        return;
    }
    const bool eq = (fl & F_EQ) != 0;
    uint32_t head = (uint32_t)n | (eq ? kFtEq : 0u);
    for (int i = 0; i < Q; ++i)
        tab[(1 + i) * nf + t] = eq ? kFtNone : (uint32_t)gather_elem_canon(a.g, a.flags, x, y, z, i);
    for (int j = 0; j < Q; ++j) {
        uint32_t v[2] = {kFtNone, kFtNone};
        int cnt = 0;
        scatter_targets(a.g, a.flags, x, y, z, j, !eq, [&](int kind, long long idx) {
            if (kind != 0) return;   // a population leaving the domain: no consumer
            if (cnt < 2) v[cnt] = (uint32_t)idx;
            ++cnt;
        });
        if (cnt > 2) head |= kFtGeneral;
        tab[(1 + Q + j) * nf + t] = v[0];
        tab[(1 + 2 * Q + j) * nf + t] = v[1];
    }
    tab[t] = head;
}

// ---------------------------------------------------------------- canonical forward step
// out = Phi(in), both in the plain post-collision layout.  Face blocks first (face cells, through
// the tables when given), then lattice blocks: interior cells pull from x - c_i (the
// solid-neighbour mask gives bounce-back).
__global__ void __launch_bounds__(kB) k_canon_step(StepArgs a, const uint32_t *__restrict__ tab,
                                                  unsigned face_blocks, const float *__restrict__ in,
                                                  float *__restrict__ out) {
    const long long N = a.g.N;
    float g[Q];
    long long n;
    if (blockIdx.x < face_blocks) {
        const long long t = (long long)blockIdx.x * kB + threadIdx.x;
        const long long nf = a.nface;
        if (t >= nf) return;
        int x, y, z;
        if (tab) {
            const uint32_t head = tab[t];
            if (head == kFtNone) return;
            n = head & kFtCell;
            if (head & kFtEq) {
                eq_cell_g(a, n, g);
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) g[i] = in[tab[(1 + i) * nf + t]];
                collide<false>(g, a);
            }
        } else {
            face_cell_xyz(a.g, t, x, y, z);
            n = cell_of(a.g, x, y, z);
            const uint8_t fl = a.flags[n];
            if (fl & F_SOLID) return;
            if (fl & F_EQ) {
                eq_cell_g(a, n, g);
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) g[i] = in[gather_elem_canon(a.g, a.flags, x, y, z, i)];
                collide<false>(g, a);
            }
        }
    } else {
        n = (long long)(blockIdx.x - face_blocks) * kB + threadIdx.x;
        if (n >= N) return;
        const uint8_t fl = a.flags[n];
        if (fl & (F_SOLID | F_FACE)) return;
        const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            g[i] = ((nb >> opp(i)) & 1u) ? in[(long long)opp(i) * N + n] : in[(long long)i * N + n - a.off[i]];
        collide<false>(g, a);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) out[(long long)i * N + n] = g[i];
}

// ---------------------------------------------------------------- collision adjoint
// lam (in): dJ/dg* of the post-collision populations; lam (out): dJ/dg of the pre-collision
// (gathered) populations g, i.e. J_C(g)^T lam, for the unforced collision of collide<false>:
//   g* = (1 - om) g + om g^eq(drho, u),  om = 1/tau_e,  tau_e = (tau + R)/2,
//   R = sqrt(tau^2 + 18 C^2 Q / rho),  Q = sqrt(2 Pi:Pi),  Pi = S - drho/3 I - j j^T / rho,
//   rho = 1 + drho,  drho = sum g,  j = sum c g,  u = j / rho,  S = sum c c g.
// Reverse mode of exactly these expressions; at Q = 0 the derivative of Q is taken as 0.
LBM_HD void collide_adjoint(const float (&g)[Q], float (&lam)[Q], const StepArgs &a) {
    float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
    float sxx = 0.0f, syy = 0.0f, szz = 0.0f, sxy = 0.0f, sxz = 0.0f, syz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += g[i];
        if (cx(i)) jx += cx(i) * g[i];
        if (cy(i)) jy += cy(i) * g[i];
        if (cz(i)) jz += cz(i) * g[i];
        if (cx(i)) sxx += g[i];
        if (cy(i)) syy += g[i];
        if (cz(i)) szz += g[i];
        if (cx(i) * cy(i)) sxy += cx(i) * cy(i) * g[i];
        if (cx(i) * cz(i)) sxz += cx(i) * cz(i) * g[i];
        if (cy(i) * cz(i)) syz += cy(i) * cz(i) * g[i];
    }
    const float rho = 1.0f + drho;
    const float ir = 1.0f / rho;
    const float ux = jx * ir, uy = jy * ir, uz = jz * ir;
    const float d3 = drho * (1.0f / 3.0f);
    const float pxx = sxx - d3 - jx * ux, pyy = syy - d3 - jy * uy, pzz = szz - d3 - jz * uz;
    const float pxy = sxy - jx * uy, pxz = sxz - jx * uz, pyz = syz - jy * uz;
    const float pp = pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (pxy * pxy + pxz * pxz + pyz * pyz);
    const float qn = sqrtf(2.0f * pp);
    const float R = sqrtf(a.tau * a.tau + a.c2x18 * qn * ir);
    const float om = 1.0f / (0.5f * (a.tau + R));
    const float u2 = ux * ux + uy * uy + uz * uz;
    // reverse through g* = g + om (g^eq - g) and g^eq_i = w_i (drho + rho E_i),
    // E_i = 3 cu + 4.5 cu^2 - 1.5 u.u
    float wbar = 0.0f, A0 = 0.0f, D = 0.0f;
    float Bx = 0.0f, By = 0.0f, Bz = 0.0f, Cx = 0.0f, Cy = 0.0f, Cz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        const float E = cu * (3.0f + 4.5f * cu) - 1.5f * u2;
        const float geq = wgt(i) * (drho + rho * E);
        wbar = fmaf(lam[i], geq - g[i], wbar);
        const float ge = om * lam[i] * wgt(i);     // dJ/dg^eq_i times w_i
        A0 = fmaf(ge, 1.0f + E, A0);
        D += ge;
        if (cx(i)) { Bx += cx(i) * ge; Cx += cx(i) * ge * cu; }
        if (cy(i)) { By += cy(i) * ge; Cy += cy(i) * ge * cu; }
        if (cz(i)) { Bz += cz(i) * ge; Cz += cz(i) * ge * cu; }
    }
    float ubx = rho * (3.0f * Bx + 9.0f * Cx - 3.0f * ux * D);
    float uby = rho * (3.0f * By + 9.0f * Cy - 3.0f * uy * D);
    float ubz = rho * (3.0f * Bz + 9.0f * Cz - 3.0f * uz * D);
    float drhobar = A0;
    // om = 1 / tau_e, tau_e = (tau + R)/2, R^2 = tau^2 + c2x18 X, X = Q / rho
    const float Rbar = 0.5f * (-om * om * wbar);
    const float Xbar = Rbar * a.c2x18 / (2.0f * R);
    const float qbar = Xbar * ir;
    float irbar = Xbar * qn;
    const float ppbar = qn > 0.0f ? qbar / qn : 0.0f;
    const float bxx = 2.0f * ppbar * pxx, byy = 2.0f * ppbar * pyy, bzz = 2.0f * ppbar * pzz;
    const float bxy = 2.0f * ppbar * pxy, bxz = 2.0f * ppbar * pxz, byz = 2.0f * ppbar * pyz;
    // Pi = S - drho/3 I - j j^T ir
    drhobar -= (bxx + byy + bzz) * (1.0f / 3.0f);
    float jbx = -2.0f * (bxx * ux + bxy * uy + bxz * uz);
    float jby = -2.0f * (bxy * ux + byy * uy + byz * uz);
    float jbz = -2.0f * (bxz * ux + byz * uy + bzz * uz);
    irbar -= bxx * jx * jx + byy * jy * jy + bzz * jz * jz + 2.0f * (bxy * jx * jy + bxz * jx * jz + byz * jy * jz);
    // u = j ir
    jbx += ubx * ir; jby += uby * ir; jbz += ubz * ir;
    irbar += ubx * jx + uby * jy + ubz * jz;
    // ir = 1 / rho, rho = 1 + drho
    drhobar += -ir * ir * irbar;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float sb = bxx * (cx(i) * cx(i)) + byy * (cy(i) * cy(i)) + bzz * (cz(i) * cz(i))
                       + 2.0f * (bxy * (cx(i) * cy(i)) + bxz * (cx(i) * cz(i)) + byz * (cy(i) * cz(i)));
        lam[i] = (1.0f - om) * lam[i] + drhobar + (cx(i) * jbx + cy(i) * jby + cz(i) * jbz) + sb;
    }
}

// (d g^eq / d u)^T lam at density rho and velocity u: d g^eq_i / d u_a = w_i rho (3 c_a + 9 (c.u) c_a
// - 3 u_a)
LBM_HD void feq_u_adjoint(const float (&lam)[Q], float rho, float ux, float uy, float uz, float &gx,
                          float &gy, float &gz) {
    float bx = 0.0f, by = 0.0f, bz = 0.0f, cxs = 0.0f, cys = 0.0f, czs = 0.0f, d = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        const float l = lam[i] * wgt(i);
        d += l;
        if (cx(i)) { bx += cx(i) * l; cxs += cx(i) * l * cu; }
        if (cy(i)) { by += cy(i) * l; cys += cy(i) * l * cu; }
        if (cz(i)) { bz += cz(i) * l; czs += cz(i) * l * cu; }
    }
    gx = rho * (3.0f * bx + 9.0f * cxs - 3.0f * ux * d);
    gy = rho * (3.0f * by + 9.0f * cys - 3.0f * uy * d);
    gz = rho * (3.0f * bz + 9.0f * czs - 3.0f * uz * d);
}

struct AdjArgs {
    const float *mu_in;      // mu_{m+1} (null when m = T)
    float *mu_out;           // mu_m (unused when m = 0)
    const float *Fprev;      // F*_{m-1} (unused when m = 0)
    const float *Fcur;       // F*_m (read at sampled cells)
    const uint8_t *aflags;   // cell flags | F_SAMPLE
    const long long *scell;  // sampled cell of each sample
    int ns;
    const double *resid;     // [ns][2] time-mean (u, v) minus target
    float escale;            // 2 / n_avg when state m is averaged, else 0
    double *gacc;            // [3][nface] per face cell: sum over m >= 1 of (d f^eq/du)^T lambda_m
    double *ic;              // m = 0: [3][N] per cell (d f^eq/du)^T lambda_0 (else null)
    const uint32_t *tab;     // face tables (null: face cells resolved at run time)
};

// lambda_m at cell n (direction by direction), then mu_m or the parameter terms.
LBM_HD void adj_cell(const StepArgs &a, const AdjArgs &b, long long n, long long t, bool face) {
    const long long N = a.g.N;
    const uint8_t fl = b.aflags[n];
    if (fl & F_SOLID) return;
    const bool eq = (fl & F_EQ) != 0;
    int x, y, z;
    cell_coords(a.g, n, x, y, z);
    float lam[Q];
    if (!b.mu_in) {
#pragma unroll
        for (int j = 0; j < Q; ++j) lam[j] = 0.0f;
    } else if (!face) {
        const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
#pragma unroll
        for (int j = 0; j < Q; ++j)
            lam[j] = ((nb >> j) & 1u) ? b.mu_in[(long long)opp(j) * N + n] : b.mu_in[(long long)j * N + n + a.off[j]];
    } else if (b.tab && !(b.tab[t] & kFtGeneral)) {
        const long long nf = a.nface;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const uint32_t c0 = b.tab[(1 + Q + j) * nf + t], c1 = b.tab[(1 + 2 * Q + j) * nf + t];
            lam[j] = (c0 != kFtNone ? b.mu_in[c0] : 0.0f) + (c1 != kFtNone ? b.mu_in[c1] : 0.0f);
        }
    } else {
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            float s = 0.0f;
            scatter_targets(a.g, a.flags, x, y, z, j, !eq, [&](int kind, long long idx) {
                if (kind == 0) s += b.mu_in[idx];
            });
            lam[j] = s;
        }
    }
    if ((fl & F_SAMPLE) && b.escale != 0.0f) {
        // explicit term: d ubar_a / d F*_i = (c_ia - u_a) / (rho n_avg)
        float r = 1.0f, jx = 0.0f, jy = 0.0f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float v = b.Fcur[(long long)i * N + n];
            r += v;
            jx += cx(i) * v;
            jy += cy(i) * v;
        }
        const float ux = jx / r, uy = jy / r;
        float rx = 0.0f, ry = 0.0f;
        for (int s = 0; s < b.ns; ++s)
            if (b.scell[s] == n) { rx += (float)b.resid[2 * s]; ry += (float)b.resid[2 * s + 1]; }
        const float kx = b.escale * rx / r, ky = b.escale * ry / r;
#pragma unroll
        for (int i = 0; i < Q; ++i) lam[i] += kx * (cx(i) - ux) + ky * (cy(i) - uy);
    }
    if (b.ic) {   // m = 0: the initial state f^eq(rho_0, u_b(z)) depends on the profile
        float ux, uy, uz;
        if (eq) eq_velocity(a, x, y, z, ux, uy, uz);
        else { ux = a.ub[3 * z]; uy = a.ub[3 * z + 1]; uz = a.ub[3 * z + 2]; }
        float gx, gy, gz;
        feq_u_adjoint(lam, eq ? a.rho_b : 1.0f, ux, uy, uz, gx, gy, gz);
        b.ic[n] = gx;
        b.ic[N + n] = gy;
        b.ic[2 * N + n] = gz;
        return;
    }
    if (eq) {
        float ux, uy, uz, gx, gy, gz;
        eq_velocity(a, x, y, z, ux, uy, uz);
        feq_u_adjoint(lam, a.rho_b, ux, uy, uz, gx, gy, gz);
        const long long nf = a.nface;
        b.gacc[t] += gx;
        b.gacc[nf + t] += gy;
        b.gacc[2 * nf + t] += gz;
        return;
    }
    float g[Q];
    if (!face) {
        const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
#pragma unroll
        for (int i = 0; i < Q; ++i)
            g[i] = ((nb >> opp(i)) & 1u) ? b.Fprev[(long long)opp(i) * N + n] : b.Fprev[(long long)i * N + n - a.off[i]];
    } else if (b.tab) {
        const long long nf = a.nface;
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = b.Fprev[b.tab[(1 + i) * nf + t]];
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = b.Fprev[gather_elem_canon(a.g, a.flags, x, y, z, i)];
    }
    collide_adjoint(g, lam, a);
#pragma unroll
    for (int i = 0; i < Q; ++i) b.mu_out[(long long)i * N + n] = lam[i];
}

// Face blocks first (face cells enumerated face by face, index t), then lattice blocks (cells on
// no face layer).
__global__ void __launch_bounds__(kB, 3) k_adj_step(StepArgs a, AdjArgs b, unsigned face_blocks) {
    if (blockIdx.x < face_blocks) {
        const long long t = (long long)blockIdx.x * kB + threadIdx.x;
        if (t >= a.nface) return;
        int x, y, z;
        face_cell_xyz(a.g, t, x, y, z);
        adj_cell(a, b, cell_of(a.g, x, y, z), t, true);
    } else {
        const long long n = (long long)(blockIdx.x - face_blocks) * kB + threadIdx.x;
        if (n >= a.g.N) return;
        if (a.flags[n] & F_FACE) return;
        adj_cell(a, b, n, -1, false);
    }
}

// ---------------------------------------------------------------- small kernels
// adjoint flags = cell flags | F_SAMPLE at the sampled cells; bad[0] counts samples on non-fluid
// cells
__global__ void k_adj_flags(const uint8_t *__restrict__ flags, uint8_t *__restrict__ aflags, long long N) {
    const long long n = (long long)blockIdx.x * kB + threadIdx.x;
    if (n < N) aflags[n] = flags[n];
}
__global__ void k_mark_samples(const long long *__restrict__ scell, int ns, const uint8_t *__restrict__ flags,
                               uint8_t *__restrict__ aflags, int *__restrict__ bad) {
    const int s = blockIdx.x * kB + threadIdx.x;
    if (s >= ns) return;
    const long long n = scell[s];
    if (flags[n] & (F_SOLID | F_EQ)) atomicAdd(bad, 1);
    aflags[n] = flags[n] | F_SAMPLE;
}

// acc[s] += (u, v, w, rho) of the current post-collision state (FP64)
__global__ void k_sample_acc(StepArgs a, bool layoutA, const long long *__restrict__ scell, int ns,
                             double *__restrict__ acc) {
    const int s = blockIdx.x * kB + threadIdx.x;
    if (s >= ns) return;
    float r, ux, uy, uz;
    cell_macros<LBM_F32>(a, scell[s], layoutA, r, ux, uy, uz);
    acc[4 * s] += ux;
    acc[4 * s + 1] += uy;
    acc[4 * s + 2] += uz;
    acc[4 * s + 3] += r;
}

// mean = acc / n_avg, resid = mean(u, v) - target, J = sum resid^2 (one block, fixed order)
__global__ void k_misfit(const double *__restrict__ acc, int ns, double inv_avg, const float *__restrict__ target,
                         double *__restrict__ resid, double *__restrict__ mean_out, double *__restrict__ J) {
    __shared__ double sh[kB];
    double part = 0.0;
    for (int s = threadIdx.x; s < ns; s += kB) {
        for (int c = 0; c < 4; ++c)
            if (mean_out) mean_out[4 * s + c] = acc[4 * s + c] * inv_avg;
        if (target) {
            const double rx = acc[4 * s] * inv_avg - (double)target[2 * s];
            const double ry = acc[4 * s + 1] * inv_avg - (double)target[2 * s + 1];
            if (resid) { resid[2 * s] = rx; resid[2 * s + 1] = ry; }
            part += rx * rx + ry * ry;
        }
    }
    sh[threadIdx.x] = part;
    __syncthreads();
    for (int w = kB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && J) *J = sh[0];
}

// g_ub[z][a] = sum over the cells of plane z of ic[a] + sum over the equilibrium face cells at
// height z of gacc[a] (one block per height, fixed order)
__global__ void k_reduce_height(StepArgs a, const double *__restrict__ ic, const double *__restrict__ gacc,
                                const uint8_t *__restrict__ flags, double *__restrict__ gub) {
    const int z = blockIdx.x;
    const long long plane = (long long)a.g.nx * a.g.ny, N = a.g.N, nf = a.nface;
    double v[3] = {0.0, 0.0, 0.0};
    for (long long r = threadIdx.x; r < plane; r += kB) {
        const long long n = (long long)z * plane + r;
        if (flags[n] & F_SOLID) continue;
        v[0] += ic[n]; v[1] += ic[N + n]; v[2] += ic[2 * N + n];
    }
    for (long long t = threadIdx.x; t < nf; t += kB) {
        int x, y, zz;
        face_cell_xyz(a.g, t, x, y, zz);
        if (zz != z) continue;
        if (!(flags[cell_of(a.g, x, y, zz)] & F_EQ)) continue;
        v[0] += gacc[t]; v[1] += gacc[nf + t]; v[2] += gacc[2 * nf + t];
    }
    __shared__ double sh[3][kB];
    for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int w = kB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) gub[3 * z + c] = sh[c][0];
}

// Chain rule of the profile mapping u_b(z) = s(z) (cos t, sin t, 0), s(z) = (1 - w) s_l0 + w s_l1:
// out[1 + l] = dJ/ds_l, out[1 + L] = dJ/dtheta (one block)
struct ChainRow {
    int l0, l1;
    double w1, s;
};
__global__ void k_chain(const double *__restrict__ gub, const ChainRow *__restrict__ tab, int nz, int L,
                        double ct, double st, double *__restrict__ out) {
    for (int l = threadIdx.x; l <= L; l += kB) {
        double v = 0.0;
        for (int z = 0; z < nz; ++z) {
            const double gx = gub[3 * z], gy = gub[3 * z + 1];
            if (l < L) {
                const double along = gx * ct + gy * st;
                if (tab[z].l0 == l) v += (1.0 - tab[z].w1) * along;
                if (tab[z].l1 == l) v += tab[z].w1 * along;
            } else {
                v += tab[z].s * (-gx * st + gy * ct);
            }
        }
        out[1 + l] = v;
    }
}

inline unsigned nblk(long long n) { return (unsigned)((n + kB - 1) / kB); }
inline size_t al(size_t v) { return (v + 255) / 256 * 256; }

struct AdjLayout {
    size_t ckpt, seg, mu, aflags, scell, acc, resid, gacc, gub, tab, bad, ftab, total;
    bool tables;
    int nseg, seglen;
};

AdjLayout adj_layout(long long N, int nz, long long nface, const lbm_adjoint_params *p, int ns, int grad) {
    AdjLayout L{};
    const size_t st = (size_t)Q * N * sizeof(float);
    size_t off = 0;
    L.scell = off; off = al(off + (size_t)ns * sizeof(long long));
    L.acc = off; off = al(off + (size_t)ns * 4 * sizeof(double));
    L.resid = off; off = al(off + (size_t)ns * 2 * sizeof(double));
    L.bad = off; off = al(off + sizeof(int));
    L.aflags = off; off = al(off + (size_t)N);
    if (grad) {
        L.seglen = p->checkpoint_every < p->n_steps ? p->checkpoint_every : p->n_steps;
        L.nseg = (p->n_steps + p->checkpoint_every - 1) / p->checkpoint_every;
        L.ckpt = off; off = al(off + (size_t)L.nseg * st);
        L.seg = off; off = al(off + (size_t)L.seglen * st);
        L.mu = off; off = al(off + 2 * st);
        L.gacc = off; off = al(off + (size_t)nface * 3 * sizeof(double));
        L.gub = off; off = al(off + (size_t)nz * 3 * sizeof(double));
        L.tab = off; off = al(off + (size_t)nz * sizeof(ChainRow));
        // face tables: element codes must fit 32 bits below the kFtNone marker, cell indices the
        // head's kFtCell bits
        L.tables = (long long)Q * N < (long long)kFtNone && N <= (long long)kFtCell;
        L.ftab = off;
        if (L.tables) off = al(off + (size_t)nface * kFtWords * sizeof(uint32_t));
    }
    L.total = off;
    return L;
}

const char *check_adj(const lbm_adjoint_params *p) {
    if (!p) return "adjoint params is NULL";
    if (p->n_steps < 1) return "n_steps must be >= 1";
    if (p->n_avg < 1 || p->n_avg > p->n_steps + 1) return "n_avg must be in [1, n_steps + 1]";
    if (p->checkpoint_every < 1) return "checkpoint_every must be >= 1";
    return nullptr;
}

lbm_status cu(lbm_domain *d, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LBM_OK;
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return domain_fail(d, LBM_ECUDA, buf);
}

// Shared by both entry points: checks, profile, initial state, forward run with lidar averaging
// (and checkpoints when ckpt != null), misfit.
lbm_status lidar_forward(lbm_domain *d, const lbm_adjoint_params *p, const float *speed, int L, float theta,
                         const int *ij, int ncol, const int *k, int nh, const float *target, char *ws,
                         size_t ws_bytes, double *out, double *mean, int grad, AdjLayout &AL) {
    if (const char *m = check_adj(p)) return domain_fail(d, LBM_EINVAL, m);
    const DomainView v0 = domain_view(d);
    const StepArgs &a0 = v0.args;
    if (v0.store != LBM_F32) return domain_fail(d, LBM_EINVAL, "lidar misfit: FP32 storage only");
    if (a0.fx != 0.0f || a0.fy != 0.0f || a0.fz != 0.0f || a0.ox != 0.0f || a0.oy != 0.0f || a0.oz != 0.0f)
        return domain_fail(d, LBM_EINVAL, "lidar misfit: body forces and rotation are not supported");
    for (int f = 0; f < 6; ++f)
        if (a0.ueq[f]) return domain_fail(d, LBM_EINVAL, "lidar misfit: switch the synthetic inflow off first");
    if (a0.sponge_top > 0 || a0.buffer_faces != 0 || a0.flux_balance)
        return domain_fail(d, LBM_EINVAL, "lidar misfit: relaxation zones and flux balancing are not supported");
    if (!ij || !k || ncol < 1 || nh < 1) return domain_fail(d, LBM_EINVAL, "lidar misfit: need >= 1 column and height");
    if ((long long)ncol * nh > (1 << 20)) return domain_fail(d, LBM_EINVAL, "lidar misfit: more than 2^20 samples");
    if (!ws || ((uintptr_t)ws % 256)) return domain_fail(d, LBM_EINVAL, "lidar misfit: workspace NULL or not 256-byte aligned");
    const int ns = ncol * nh;
    AL = adj_layout(a0.g.N, a0.g.nz, a0.nface, p, ns, grad);
    if (ws_bytes < AL.total) return domain_fail(d, LBM_ENOMEM, "lidar misfit: workspace too small");
    std::vector<long long> cells((size_t)ns);
    for (int c = 0; c < ncol; ++c)
        for (int h = 0; h < nh; ++h) {
            const int x = ij[2 * c], y = ij[2 * c + 1], z = k[h];
            if (x < 0 || x >= a0.g.nx || y < 0 || y >= a0.g.ny || z < 0 || z >= a0.g.nz)
                return domain_fail(d, LBM_EINVAL, "lidar misfit: sample outside the lattice");
            cells[(size_t)c * nh + h] = cell_of(a0.g, x, y, z);
        }
    lbm_status st = lbm_set_inflow_profile(d, speed, L, theta);
    if (st != LBM_OK) return st;
    st = lbm_init_fields(d, nullptr, nullptr);
    if (st != LBM_OK) return st;
    cudaStream_t s = v0.stream;
    long long *scell = (long long *)(ws + AL.scell);
    double *acc = (double *)(ws + AL.acc);
    int *bad = (int *)(ws + AL.bad);
    uint8_t *aflags = (uint8_t *)(ws + AL.aflags);
    if ((st = cu(d, cudaMemcpyAsync(scell, cells.data(), cells.size() * sizeof(long long), cudaMemcpyHostToDevice, s), "sample upload")) != LBM_OK) return st;
    if ((st = cu(d, cudaMemsetAsync(acc, 0, (size_t)ns * 4 * sizeof(double), s), "clear")) != LBM_OK) return st;
    if ((st = cu(d, cudaMemsetAsync(bad, 0, sizeof(int), s), "clear")) != LBM_OK) return st;
    k_adj_flags<<<nblk(a0.g.N), kB, 0, s>>>(a0.flags, aflags, a0.g.N);
    k_mark_samples<<<nblk(ns), kB, 0, s>>>(scell, ns, a0.flags, aflags, bad);
    int nbad = 0;
    if ((st = cu(d, cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s), "check copy")) != LBM_OK) return st;
    if ((st = cu(d, cudaStreamSynchronize(s), "check sync")) != LBM_OK) return st;
    if (nbad) return domain_fail(d, LBM_EINVAL, "lidar misfit: sampled cells must be fluid cells");

    const int T = p->n_steps, first = T - p->n_avg + 1;
    float *ckpt = grad ? (float *)(ws + AL.ckpt) : nullptr;
    const size_t st19 = (size_t)Q * a0.g.N;
    for (int n = 0; n <= T; ++n) {
        if (n > 0 && (st = lbm_step(d, 1)) != LBM_OK) return st;
        if (ckpt && n < T && n % p->checkpoint_every == 0)
            if ((st = lbm_export_populations(d, ckpt + (size_t)(n / p->checkpoint_every) * st19)) != LBM_OK) return st;
        if (n >= first) {
            const DomainView v = domain_view(d);
            k_sample_acc<<<nblk(ns), kB, 0, s>>>(v.args, v.layoutA, scell, ns, acc);
        }
    }
    k_misfit<<<1, kB, 0, s>>>(acc, ns, 1.0 / p->n_avg, target, (double *)(ws + AL.resid), mean,
                              out ? out : nullptr);
    return cu(d, cudaGetLastError(), "lidar forward kernels");
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" {

size_t lbm_adjoint_workspace_bytes(const lbm_domain *d, const lbm_adjoint_params *p, int ncol, int nh,
                                   int gradient) {
    if (!d || check_adj(p) || ncol < 1 || nh < 1) return 0;
    const DomainView v = domain_view(d);
    return adj_layout(v.args.g.N, v.args.g.nz, v.args.nface, p, ncol * nh, gradient).total;
}

lbm_status lbm_lidar_misfit(lbm_domain *d, const lbm_adjoint_params *p, const float *speed, int L, float theta,
                            const int *ij, int ncol, const int *k, int nh, const float *target, void *workspace,
                            size_t ws_bytes, double *out, double *mean) {
    if (!d) return LBM_EINVAL;
    AdjLayout AL;
    return lidar_forward(d, p, speed, L, theta, ij, ncol, k, nh, target, (char *)workspace, ws_bytes, out,
                         mean, 0, AL);
}

lbm_status lbm_lidar_misfit_grad(lbm_domain *d, const lbm_adjoint_params *p, const float *speed, int L,
                                 float theta, const int *ij, int ncol, const int *k, int nh,
                                 const float *target, void *workspace, size_t ws_bytes, double *out,
                                 double *mean) {
    if (!d) return LBM_EINVAL;
    if (!target || !out) return domain_fail(d, LBM_EINVAL, "lidar gradient: target and out are required");
    char *ws = (char *)workspace;
    AdjLayout AL;
    lbm_status st = lidar_forward(d, p, speed, L, theta, ij, ncol, k, nh, target, ws, ws_bytes, out, mean, 1, AL);
    if (st != LBM_OK) return st;
    const DomainView v = domain_view(d);
    const StepArgs &a = v.args;
    cudaStream_t s = v.stream;
    const long long N = a.g.N;
    const size_t st19 = (size_t)Q * N;
    const int T = p->n_steps, K = p->checkpoint_every, first = T - p->n_avg + 1;
    float *ckpt = (float *)(ws + AL.ckpt);
    float *seg = (float *)(ws + AL.seg);
    float *mu[2] = {(float *)(ws + AL.mu), (float *)(ws + AL.mu) + st19};
    double *gacc = (double *)(ws + AL.gacc);
    if ((st = cu(d, cudaMemsetAsync(mu[0], 0, 2 * st19 * sizeof(float), s), "clear")) != LBM_OK) return st;
    if ((st = cu(d, cudaMemsetAsync(gacc, 0, (size_t)a.nface * 3 * sizeof(double), s), "clear")) != LBM_OK) return st;
    uint32_t *ftab = AL.tables ? (uint32_t *)(ws + AL.ftab) : nullptr;
    const unsigned fb = nblk(a.nface), lb = nblk(N);
    if (ftab) k_adj_tables<<<fb, kB, 0, s>>>(a, ftab);
    AdjArgs b{};
    b.tab = ftab;
    b.aflags = (const uint8_t *)(ws + AL.aflags);
    b.scell = (const long long *)(ws + AL.scell);
    b.ns = ncol * nh;
    b.resid = (const double *)(ws + AL.resid);
    b.gacc = gacc;
    const float es = 2.0f / (float)p->n_avg;
    for (int c = AL.nseg - 1; c >= 0; --c) {
        const int base = c * K, len = (T - base) < K ? (T - base) : K;
        const auto state = [&](int kk) { return kk == 0 ? ckpt + (size_t)c * st19 : seg + (size_t)(kk - 1) * st19; };
        for (int kk = 1; kk <= len; ++kk) k_canon_step<<<fb + lb, kB, 0, s>>>(a, ftab, fb, state(kk - 1), state(kk));
        for (int m = base + len; m >= base + 1; --m) {
            const int kk = m - base;
            b.mu_in = m == T ? nullptr : mu[(m + 1) & 1];
            b.mu_out = mu[m & 1];
            b.Fprev = state(kk - 1);
            b.Fcur = state(kk);
            b.escale = m >= first ? es : 0.0f;
            b.ic = nullptr;
            k_adj_step<<<fb + lb, kB, 0, s>>>(a, b, fb);
        }
        if ((st = cu(d, cudaGetLastError(), "adjoint kernels")) != LBM_OK) return st;
    }
    // m = 0: lambda_0 and the initial-state terms (scratch: the free mu buffer, 3 N doubles)
    b.mu_in = mu[1];
    b.mu_out = nullptr;
    b.Fprev = nullptr;
    b.Fcur = ckpt;
    b.escale = 0 >= first ? es : 0.0f;
    b.ic = (double *)mu[0];
    k_adj_step<<<fb + lb, kB, 0, s>>>(a, b, fb);
    double *gub = (double *)(ws + AL.gub);
    k_reduce_height<<<a.g.nz, kB, 0, s>>>(a, b.ic, gacc, a.flags, gub);
    // chain rule to the level speeds and the direction (same mapping as lbm_set_inflow_profile)
    std::vector<ChainRow> tab((size_t)a.g.nz);
    for (int z = 0; z < a.g.nz; ++z) {
        int l0, l1;
        double w1;
        profile_level_weights(L, a.g.nz, z, l0, l1, w1);
        tab[z] = ChainRow{l0, l1, w1, (1.0 - w1) * (double)speed[l0] + w1 * (double)speed[l1]};
    }
    ChainRow *tab_dev = (ChainRow *)(ws + AL.tab);
    if ((st = cu(d, cudaMemcpyAsync(tab_dev, tab.data(), tab.size() * sizeof(ChainRow), cudaMemcpyHostToDevice, s), "table upload")) != LBM_OK) return st;
    k_chain<<<1, kB, 0, s>>>(gub, tab_dev, a.g.nz, L, std::cos((double)theta), std::sin((double)theta), out);
    return cu(d, cudaGetLastError(), "adjoint kernels");
}

}  // extern "C"

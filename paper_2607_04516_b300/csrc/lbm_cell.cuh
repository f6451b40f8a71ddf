// lbm_cell.cuh -- the per-cell bodies of every kernel (one call = the work of one thread).
// The kernels in lbm_kernels.cu are thin grid wrappers around these.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// ---------------------------------------------------------------- flags from the solid mask
LBM_HD void cell_flags(const uint8_t *__restrict__ mask, uint8_t *__restrict__ flags, const Geo &G,
                       long long n) {
    if (mask[n]) { flags[n] = F_SOLID; return; }
    int x, y, z;
    cell_coords(G, n, x, y, z);
    const bool lo[3] = {x == 0, y == 0, z == 0};
    const bool hi[3] = {x == G.nx - 1, y == G.ny - 1, z == G.nz - 1};
    bool eq = false, onface = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        onface |= lo[a] | hi[a];
        eq |= (lo[a] && G.face[2 * a] == LBM_FACE_INFLOW_EQ) ||
              (hi[a] && G.face[2 * a + 1] == LBM_FACE_INFLOW_EQ);
    }
    bool zgl = false;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        zgl |= (lo[a] && G.face[2 * a] == LBM_FACE_OUTFLOW_ZG) || (hi[a] && G.face[2 * a + 1] == LBM_FACE_OUTFLOW_ZG);
    uint8_t fl = zgl ? F_ZG : 0;
    if (onface) fl |= F_FACE;
    if (eq) {
        fl |= F_EQ;
    } else if (!onface) {   // interior cell: all 18 neighbours are in range
        bool near = false;
#pragma unroll
        for (int i = 1; i < Q; ++i) near |= mask[n + cx(i) + cy(i) * G.sy + cz(i) * G.sz] != 0;
        if (near) fl |= F_NEAR;
    }
    flags[n] = fl;
}

// ---------------------------------------------------------------- equilibrium initialisation
template <int S>
LBM_HD void cell_init(const StepArgs &a, long long n, const float *__restrict__ rho,
                      const float *__restrict__ u) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const uint8_t fl = a.flags[n];
    T *f = (T *)a.f;
    const long long N = a.g.N;
    if (fl & F_SOLID) {
#pragma unroll
        for (int i = 0; i < Q; ++i) f[(long long)i * N + n] = Cd::enc(0.0f);
        return;
    }
    const int z = (int)(n / a.g.sz);
    float drho, ux, uy, uz;
    if (fl & F_EQ) {
        drho = a.rho_b - 1.0f;
        ux = a.ub[3 * z]; uy = a.ub[3 * z + 1]; uz = a.ub[3 * z + 2];
    } else {
        drho = rho ? rho[n] - 1.0f : 0.0f;
        if (u) { ux = u[3 * n]; uy = u[3 * n + 1]; uz = u[3 * n + 2]; }
        else { ux = a.ub[3 * z]; uy = a.ub[3 * z + 1]; uz = a.ub[3 * z + 2]; }
    }
    float g[Q];
    equilibrium_shifted(drho, ux, uy, uz, g);
#pragma unroll
    for (int i = 0; i < Q; ++i) f[(long long)opp(i) * N + n] = Cd::enc(g[i]);   // layout B
    if (fl & F_ZG) {
        int x, y, zz;
        cell_coords(a.g, n, x, y, zz);
        store_side<T>(a.g, a.side, x, y, zz, g, [](float v) { return Cd::enc(v); });
    }
}

// ---------------------------------------------------------------- local step: A -> B
template <int S, bool FORCE>
LBM_HD void cell_local(const StepArgs &a, long long n) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const uint8_t fl = a.flags[n];
    if (fl & F_SOLID) return;
    T *__restrict__ f = (T *)a.f;
    const long long N = a.g.N;
    float g[Q];
    if (fl & F_EQ) {
        const int z = (int)(n / a.g.sz);
        equilibrium_shifted(a.rho_b - 1.0f, a.ub[3 * z], a.ub[3 * z + 1], a.ub[3 * z + 2], g);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = Cd::dec(f[(long long)i * N + n]);
        collide<FORCE>(g, a);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) f[(long long)opp(i) * N + n] = Cd::enc(g[i]);
    if (fl & F_ZG) {
        int x, y, z;
        cell_coords(a.g, n, x, y, z);
        store_side<T>(a.g, a.side, x, y, z, g, [](float v) { return Cd::enc(v); });
    }
}

// ---------------------------------------------------------------- neighbour step: B -> A
// Interior cell (on no face layer): pull from x - c_i and push to x + c_i; a solid neighbour turns
// the link into bounce-back (read / write the cell's own reversed slot).  The 18 neighbour flags
// are loaded only for cells marked F_NEAR.
template <int S, bool FORCE>
LBM_HD void cell_neighbor_interior(const StepArgs &a, long long n, uint8_t fl) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    T *__restrict__ f = (T *)a.f;
    const long long N = a.g.N;
    const long long sy = a.g.sy, sz = a.g.sz;
    unsigned nb = 0;   // bit i: the neighbour x + c_i is solid
    if (fl & F_NEAR) {
#pragma unroll
        for (int i = 1; i < Q; ++i)
            nb |= (unsigned)(a.flags[n + cx(i) + cy(i) * sy + cz(i) * sz] & F_SOLID) << i;
    }
    float g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const long long off = cx(i) + cy(i) * sy + cz(i) * sz;
        // source x - c_i = x + c_opp(i); bounce-back: f*_opp(i)(x) sits in slot i of x (layout B)
        const long long idx = ((nb >> opp(i)) & 1u) ? (long long)i * N + n : (long long)opp(i) * N + n - off;
        g[i] = Cd::dec(f[idx]);
    }
    collide<FORCE>(g, a);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const long long off = cx(i) + cy(i) * sy + cz(i) * sz;
        const long long idx = ((nb >> i) & 1u) ? (long long)opp(i) * N + n : (long long)i * N + n + off;
        f[idx] = Cd::enc(g[i]);
    }
}

// Face-layer cell: every boundary rule through the general gather / scatter resolution.
template <int S, bool FORCE>
LBM_HD void cell_neighbor_face(const StepArgs &a, uint8_t fl, int x, int y, int z) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    T *__restrict__ f = (T *)a.f;
    float g[Q];
    const bool fluid = !(fl & F_EQ);
    if (!fluid) {
        equilibrium_shifted(a.rho_b - 1.0f, a.ub[3 * z], a.ub[3 * z + 1], a.ub[3 * z + 2], g);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Loc l = gather_loc_B(a.g, a.flags, x, y, z, i);
            const T *base = l.kind == 0 ? f : (const T *)a.side[l.kind - 1];
            g[i] = Cd::dec(base[l.idx]);
        }
        collide<FORCE>(g, a);
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const T v = Cd::enc(g[j]);
        scatter_targets(a.g, a.flags, x, y, z, j, fluid, [&](int kind, long long idx) {
            T *base = kind == 0 ? f : (T *)a.side[kind - 1];
            base[idx] = v;
        });
    }
}

// ---------------------------------------------------------------- post-collision readback
// Shifted post-collision populations of a non-solid cell n in the current layout.
template <int S>
LBM_HD void read_post(const StepArgs &a, long long n, uint8_t fl, bool layoutA, float (&g)[Q]) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const T *f = (const T *)a.f;
    const long long N = a.g.N;
    int x, y, z;
    cell_coords(a.g, n, x, y, z);
    if (fl & F_EQ) {
        // the equilibrium populations as stored (and as consumed by the neighbours)
        equilibrium_shifted(a.rho_b - 1.0f, a.ub[3 * z], a.ub[3 * z + 1], a.ub[3 * z + 2], g);
#pragma unroll
        for (int j = 0; j < Q; ++j) g[j] = Cd::dec(Cd::enc(g[j]));
        return;
    }
    if (!layoutA) {
#pragma unroll
        for (int j = 0; j < Q; ++j) g[j] = Cd::dec(f[(long long)opp(j) * N + n]);
        return;
    }
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        float v = NAN;   // stays NaN only if no location held it (cannot happen for fluid cells)
        bool found = false;
        scatter_targets(a.g, a.flags, x, y, z, j, true, [&](int kind, long long idx) {
            if (found) return;
            const T *base = kind == 0 ? f : (const T *)a.side[kind - 1];
            v = Cd::dec(base[idx]);
            found = true;
        });
        g[j] = v;
    }
}

LBM_HD void macros_of(const StepArgs &a, const float (&g)[Q], float &rho, float &ux, float &uy,
                      float &uz) {
    float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += g[i];
        jx += cx(i) * g[i];
        jy += cy(i) * g[i];
        jz += cz(i) * g[i];
    }
    rho = 1.0f + drho;
    // after a Guo-forced collision sum c f* = rho u + F/2
    ux = (jx - 0.5f * a.fx) / rho;
    uy = (jy - 0.5f * a.fy) / rho;
    uz = (jz - 0.5f * a.fz) / rho;
}

// (rho, u) of the current post-collision state at cell n (equilibrium cells: rho_b, u_b;
// solid: zeros)
template <int S>
LBM_HD void cell_macros(const StepArgs &a, long long n, bool layoutA, float &r, float &ux, float &uy,
                        float &uz) {
    const uint8_t fl = a.flags[n];
    r = 0.0f; ux = 0.0f; uy = 0.0f; uz = 0.0f;
    if (fl & F_EQ) {
        const int z = (int)(n / a.g.sz);
        r = a.rho_b; ux = a.ub[3 * z]; uy = a.ub[3 * z + 1]; uz = a.ub[3 * z + 2];
    } else if (!(fl & F_SOLID)) {
        float g[Q];
        read_post<S>(a, n, fl, layoutA, g);
        macros_of(a, g, r, ux, uy, uz);
    }
}

template <int S>
LBM_HD void cell_export(const StepArgs &a, long long n, bool layoutA, float *__restrict__ out) {
    const uint8_t fl = a.flags[n];
    float g[Q];
    if (fl & F_SOLID) {
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = 0.0f;
    } else {
        read_post<S>(a, n, fl, layoutA, g);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) out[(long long)i * a.g.N + n] = g[i];
}

}  // namespace lbm

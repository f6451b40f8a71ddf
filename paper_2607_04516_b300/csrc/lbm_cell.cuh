// lbm_cell.cuh -- the per-cell bodies of every kernel (one call = the work of one thread).
// The kernels in lbm_kernels.cu are thin grid wrappers around these.
#pragma once

#include "lbm_device.cuh"

// 16-bit storage: evaluate the collision on opposite pairs (1) or direction by direction (0);
// chosen by measurement on B300
#ifndef LBM_PAIRS16
#define LBM_PAIRS16 1
#endif

namespace lbm {

constexpr bool kPairs16 = LBM_PAIRS16 != 0;

// Scale (log2) at which the 16-bit kernels hold populations in registers: the storage scale
// itself when the collision folds it in (unforced pair form), else 1 (plain g).
template <int S, bool FORCE> __host__ __device__ constexpr int reg_log2() {
    return (!FORCE && kPairs16) ? Codec<S>::kLog2 : 0;
}
// Shifted equilibrium of an equilibrium cell at register scale 2^L.
template <int L> LBM_HD void eq_cell_g_s(const StepArgs &a, long long n, float (&g)[Q]) {
    eq_cell_g(a, n, g);
    if (L != 0) {
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] *= (float)(1 << L);
    }
}

// ---------------------------------------------------------------- flags from the solid mask
// Cell kind bits and, for cells that use the store-side bounce-back convention (F_REDIR: interior
// cells, and cells of a no-slip / free-slip z layer with interior x and y, that have a solid
// neighbour), the mask of solid neighbours x + c_i.
LBM_HD void cell_flags(const uint8_t *__restrict__ mask, uint8_t *__restrict__ flags,
                       uint32_t *__restrict__ info, const Geo &G, long long n) {
    if (mask[n]) { flags[n] = F_SOLID; info[n] = F_SOLID; return; }
    int x, y, z;
    cell_coords(G, n, x, y, z);
    const bool lo[3] = {x == 0, y == 0, z == 0};
    const bool hi[3] = {x == G.nx - 1, y == G.ny - 1, z == G.nz - 1};
    bool eq = false, onface = false, zgl = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        onface |= lo[a] | hi[a];
        eq |= (lo[a] && G.face[2 * a] == LBM_FACE_INFLOW_EQ) || (hi[a] && G.face[2 * a + 1] == LBM_FACE_INFLOW_EQ);
        zgl |= (lo[a] && G.face[2 * a] == LBM_FACE_OUTFLOW_ZG) || (hi[a] && G.face[2 * a + 1] == LBM_FACE_OUTFLOW_ZG);
    }
    uint8_t fl = (zgl ? F_ZG : 0) | (onface ? F_FACE : 0) | (eq ? F_EQ : 0);
    const bool xy_interior = !lo[0] && !hi[0] && !lo[1] && !hi[1];
    const int zf = zfast_mask(G);
    const bool layer_path = xy_interior && ((lo[2] && (zf & 1)) || (hi[2] && (zf & 2))) && !(lo[2] && hi[2]);
    if (layer_path && zlat_of(G)) fl |= F_ZL;
    uint32_t nb = 0;
    if (!eq && ((!onface) || layer_path)) {
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int zz = z + cz(i);
            if (zz < 0 || zz >= G.nz) continue;   // beyond a z face: handled by the face rule
            nb |= (uint32_t)(mask[cell_of(G, x + cx(i), y + cy(i), zz)] != 0) << i;
        }
        if (nb) fl |= F_REDIR;
    }
    flags[n] = fl;
    info[n] = fl | (nb << 8);
}

// Store-side bounce-back: a post-collision population f*_k of a cell x whose neighbour x + c_k is
// solid is consumed by x itself, as f_opp(k), in the next neighbour step.  Instead of its own slot
// opp(k), an F_REDIR cell stores it into slot k of that solid neighbour (memory nobody else
// touches), so that the next neighbour step's gather of direction opp(k) is the plain pull from
// x - c_opp(k) = x + c_k.  Layout-B location of f*_k(x):
LBM_HD long long post_loc_B(const StepArgs &a, long long n, int k, unsigned nb) {
    return ((nb >> k) & 1u) ? (long long)k * a.g.N + n + a.off[k] : (long long)opp_rt(k) * a.g.N + n;
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
    // solid cells own no state: their slots only receive store-side bounce-back populations of
    // fluid neighbours (written below by those neighbours), so they are left alone here
    if (fl & F_SOLID) return;
    const int z = (int)(n / a.g.sz);
    float drho, ux, uy, uz;
    if (fl & F_EQ) {
        drho = a.rho_b - 1.0f;
        eq_velocity(a, n, ux, uy, uz);
    } else {
        drho = rho ? rho[n] - 1.0f : 0.0f;
        if (u) { ux = u[3 * n]; uy = u[3 * n + 1]; uz = u[3 * n + 2]; }
        else { ux = a.ub[3 * z]; uy = a.ub[3 * z + 1]; uz = a.ub[3 * z + 2]; }
    }
    float g[Q];
    equilibrium_shifted(drho, ux, uy, uz, g);
    const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
#pragma unroll
    for (int i = 0; i < Q; ++i)   // layout B
        f[((nb >> i) & 1u) ? (long long)i * N + n + a.off[i] : (long long)opp(i) * N + n] = Cd::enc(g[i]);
    if (fl & F_ZG) {
        int x, y, zz;
        cell_coords(a.g, n, x, y, zz);
        store_side<T>(a.g, a.side, x, y, zz, g, [](float v) { return Cd::enc(v); });
    }
}

// ---------------------------------------------------------------- state import (resume)
// Write the post-collision populations gin (shifted FP32, population-major, library direction
// order, as lbm_export_populations gives them) into layout B, the layout of an even step count:
// the same stores as cell_init (store-side bounce-back slots, outflow side buffers).
template <int S>
LBM_HD void cell_import(const StepArgs &a, long long n, const float *__restrict__ gin) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const uint8_t fl = a.flags[n];
    if (fl & F_SOLID) return;
    T *f = (T *)a.f;
    const long long N = a.g.N;
    float g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = gin[(long long)i * N + n];
    const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        f[((nb >> i) & 1u) ? (long long)i * N + n + a.off[i] : (long long)opp(i) * N + n] = Cd::enc(g[i]);
    if (fl & F_ZG) {
        int x, y, z;
        cell_coords(a.g, n, x, y, z);
        store_side<T>(a.g, a.side, x, y, z, g, [](float v) { return Cd::enc(v); });
    }
}

// ---------------------------------------------------------------- local step: A -> B
template <int S, bool FORCE>
LBM_HD void cell_local(const StepArgs &a, int n) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    T *const *P = (T *const *)a.plane;
    float g[Q];
    // the loads do not wait for the flag byte (values of solid / equilibrium cells are unused)
    static_assert(S == LBM_F32, "16-bit storage updates cells in pairs");
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = ld_early_f32((const float *)P[i] + n);
    const uint8_t fl = a.flags[n];
    if (fl & F_SOLID) return;
    if (fl & F_EQ) {
        eq_cell_g(a, n, g);
    } else {
        collide<FORCE>(g, a);
        if (FORCE) nudge(a, n, g);   // relaxation zones ride on the general (forced) path
    }
    if (fl & F_REDIR) {
        const unsigned nb = a.info[n] >> 8;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool bb = (nb >> i) & 1u;
            (bb ? P[i] : P[opp(i)])[bb ? n + a.off[i] : n] = Cd::enc(g[i]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) P[opp(i)][n] = Cd::enc(g[i]);
    }
    if (fl & F_ZG) {
        int x, y, z;
        cell_coords(a.g, n, x, y, z);
        store_side<T>(a.g, a.side, x, y, z, g, [](float v) { return Cd::enc(v); });
    }
}

// ---------------------------------------------------------------- neighbour step: B -> A
// Interior cell (on no face layer): pull from x - c_i and push to x + c_i.  A solid neighbour
// needs nothing on the gather side (store-side bounce-back, see post_loc_B); on the scatter side a
// population heading into a solid goes to the cell's own reversed slot.  No load depends on
// another load.
template <int S, bool FORCE>
LBM_HD void cell_neighbor_interior(const StepArgs &a, int n) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    T *const *P = (T *const *)a.plane;
    float g[Q];
    // the loads do not wait for the flag byte; for a solid or face cell they may fall outside its
    // neighbourhood but stay inside the workspace (guard after the planes), and are discarded
    static_assert(S == LBM_F32, "16-bit storage updates cells in pairs");
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = ld_early_f32((const float *)P[opp(i)] + n - a.off[i]);
    const uint8_t fl = a.flags[n];
    if (fl & (F_SOLID | F_FACE)) return;
    const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
    collide<FORCE>(g, a);
    if (FORCE) nudge(a, n, g);   // relaxation zones ride on the general (forced) path
    if (nb) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool bb = (nb >> i) & 1u;
            (bb ? P[opp(i)] : P[i])[bb ? n : n + a.off[i]] = Cd::enc(g[i]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) P[i][n + a.off[i]] = Cd::enc(g[i]);
    }
}

// Cell of the ground or top layer with interior x and y, when that z face is no-slip or
// free-slip: the interior rules plus, for the links crossing the face, bounce-back (no-slip) or
// specular reflection within the layer (free-slip).  Populations stored by such a cell toward the
// face stay in its own slots (no memory beyond the face), so those gathers read the cell itself.
template <int S, bool FORCE>
LBM_HD void cell_neighbor_zlayer(const StepArgs &a, int n, uint8_t fl, bool top) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    T *const *P = (T *const *)a.plane;
    const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
    const bool noslip = a.g.face[top ? 5 : 4] == LBM_FACE_NOSLIP;
    const int cout = top ? 1 : -1;        // c_z of the links leaving through this face
    float g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T *p;
        int idx;
        if (cz(i) == -cout) {             // the source x - c_i lies beyond the face
            if (noslip) {
                p = P[i]; idx = n;
            } else {
                // source (x - c_x, y - c_y) in this layer, mirrored direction; bounce-back if solid
                const int k = (cx(i) == 0 && cy(i) == 0) ? 0 : dir_c(-cx(i), -cy(i), 0);
                const int d = dir_c(cx(i), cy(i), -cz(i));
                const bool bb = k != 0 && ((nb >> k) & 1u);
                p = bb ? P[i] : P[opp(d)];
                idx = bb ? n : n + a.off[k];
            }
        } else {
            p = P[opp(i)]; idx = n - a.off[i];
        }
        g[i] = Cd::dec(p[idx]);
    }
    collide<FORCE>(g, a);
    if (FORCE) nudge(a, n, g);   // relaxation zones ride on the general (forced) path
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        T *p;
        int idx;
        if (cz(j) == cout) {              // the target x + c_j lies beyond the face
            if (noslip) {
                p = P[opp(j)]; idx = n;
            } else {
                const int k = (cx(j) == 0 && cy(j) == 0) ? 0 : dir_c(cx(j), cy(j), 0);
                const int m = dir_c(cx(j), cy(j), -cz(j));
                const bool bb = k != 0 && ((nb >> k) & 1u);
                p = bb ? P[opp(j)] : P[m];
                idx = bb ? n : n + a.off[k];
            }
        } else {
            const bool bb = (nb >> j) & 1u;
            p = bb ? P[opp(j)] : P[j];
            idx = bb ? n : n + a.off[j];
        }
        p[idx] = Cd::enc(g[j]);
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
        float ux, uy, uz;
        eq_velocity(a, x, y, z, ux, uy, uz);
        equilibrium_shifted(a.rho_b - 1.0f, ux, uy, uz, g);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Loc l = gather_loc_B(a.g, a.flags, x, y, z, i);
            const T *base = l.kind == 0 ? f : (const T *)a.side[l.kind - 1];
            g[i] = Cd::dec(base[l.idx]);
        }
        collide<FORCE>(g, a);
        if (FORCE) nudge(a, cell_of(a.g, x, y, z), g);   // relaxation zones ride on the general (forced) path
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

// ---------------------------------------------------------------- face tables
// The boundary resolution of a face cell depends only on the geometry and the solid mask, so it is
// done once, at domain creation, for the face cells [0, ngen) of the face enumeration: per cell its
// index and kind, per direction the storage element (offset from the population base, in storage
// elements; the side buffers lie after it in the workspace) its gather reads, and up to two
// elements its scatter writes.
//   tab[t]                         kFtNone for a solid cell, else the cell index | kFtEq for an
//                                  equilibrium cell | kFtGeneral when some direction has more
//                                  than two scatter targets (the cell keeps the general resolution)
//   tab[(1 + i) ngen + t]          gather element of direction i (fluid cells)
//   tab[(20 + j) ngen + t]         first scatter element of direction j (kFtNone: none)
//   tab[(39 + j) ngen + t]         second scatter element (kFtNone: none)
//   tab[58 ngen + t]               bit j: direction j scatters to its plain target alone (element
//                                  j N + n + c_j), so its two scatter words need not be read
//   tab[59 ngen + t]               bit j: direction j has a second scatter element

template <int S>
LBM_HD void cell_face_table(const StepArgs &a, int t, uint32_t *__restrict__ tab) {
    using T = typename Codec<S>::T;
    const long long ng = a.ngen;
    int x, y, z;
    face_cell_xyz(a.g, t, x, y, z);
    const long long n = cell_of(a.g, x, y, z);
    const uint8_t fl = a.flags[n];
    uint32_t head = (uint32_t)n | ((fl & F_EQ) ? kFtEq : 0u);
    long long sbase[6];
#pragma unroll
    for (int k = 0; k < 6; ++k)
        sbase[k] = a.side[k] ? (long long)(((const char *)a.side[k] - (const char *)a.f) / (long long)sizeof(T)) : 0;
    const auto code = [&](int kind, long long idx) -> uint32_t {
        return (uint32_t)(kind == 0 ? idx : sbase[kind - 1] + idx);
    };
    // a layer cell with solid neighbours follows the store-side bounce-back convention of the
    // lattice (its local step parks the reflected population in the solid neighbour's slot), so a
    // gather from a solid neighbour x - c_i is the plain pull from that neighbour
    const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
    for (int i = 0; i < Q; ++i) {
        uint32_t gv = kFtNone;
        if (!(fl & (F_SOLID | F_EQ))) {
            const Loc l = ((nb >> opp_rt(i)) & 1u) ? Loc{0, (long long)opp_rt(i) * a.g.N + n - a.off[i]}
                                                  : gather_loc_B(a.g, a.flags, x, y, z, i);
            gv = code(l.kind, l.idx);
        }
        tab[(1 + i) * ng + t] = gv;
    }
    const bool fluid = !(fl & F_EQ);
    uint32_t plain = 0, second = 0;
    for (int j = 0; j < Q; ++j) {
        uint32_t v[2] = {kFtNone, kFtNone};
        int cnt = 0;
        if (!(fl & F_SOLID))
            scatter_targets(a.g, a.flags, x, y, z, j, fluid, [&](int kind, long long idx) {
                // an equilibrium cell's stores into equilibrium cells are dropped: such a cell
                // ignores what it receives (its next local step writes its equilibrium over it, and
                // every read-back of it computes that equilibrium), and the equilibrium cell's own
                // read-back does not look for its populations either
                if (!fluid && kind == 0 && (a.flags[idx % a.g.N] & F_EQ)) return;
                if (cnt < 2) v[cnt] = code(kind, idx);
                ++cnt;
            });
        if (cnt > 2) head |= kFtGeneral;
        tab[(1 + Q + j) * ng + t] = v[0];
        tab[(1 + 2 * Q + j) * ng + t] = v[1];
        if (cnt == 1 && v[0] == code(0, (long long)j * a.g.N + n + a.off[j])) plain |= 1u << j;
        if (cnt >= 2) second |= 1u << j;
    }
    tab[(1 + 3 * Q) * ng + t] = plain;
    tab[(2 + 3 * Q) * ng + t] = second;
    tab[t] = (fl & F_SOLID) ? kFtNone : head;
}

// Face cell t of the tables: gathers and scatters through the precomputed elements.  The head and
// the gather elements are loaded together (they depend on t only), so a fluid cell waits for two
// memory round trips before its collision.  Returns false (nothing done) for a cell that keeps the
// general resolution.
template <int S, bool FORCE>
LBM_HD bool cell_neighbor_table(const StepArgs &a, int t) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    T *__restrict__ f = (T *)a.f;
    const uint32_t *__restrict__ tab = a.ftab;
    const long long ng = a.ngen;
    uint32_t e[Q];
    const uint32_t head = tab[t], plain = tab[(1 + 3 * Q) * ng + t], second = tab[(2 + 3 * Q) * ng + t];
#pragma unroll
    for (int i = 0; i < Q; ++i) e[i] = tab[(1 + i) * ng + t];
    if (head == kFtNone) return true;   // solid
    if (head & kFtGeneral) return false;
    float g[Q];
    if (head & kFtEq) {
        eq_cell_g(a, (long long)(head & kFtCell), g);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = Cd::dec(f[e[i]]);
        collide<FORCE>(g, a);
        if (FORCE) nudge(a, (long long)(head & kFtCell), g);   // relaxation zones ride on the general (forced) path
    }
    // plain directions store without reading their scatter words; the others read one or two
    const long long n = (long long)(head & kFtCell);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const T v = Cd::enc(g[j]);
        if ((plain >> j) & 1u) {
            ((T *)a.plane[j])[n + a.off[j]] = v;
            continue;
        }
        const uint32_t e0 = tab[(1 + Q + j) * ng + t];
        if (e0 != kFtNone) f[e0] = v;
        if ((second >> j) & 1u) f[tab[(1 + 2 * Q + j) * ng + t]] = v;
    }
    return true;
}

// ---------------------------------------------------------------- two cells per thread (16-bit)
// With 2-byte populations one cell per thread leaves too few bytes in flight; a thread updates
// the cells n0 and n1 = n0 + 256 (so every warp access stays 32 consecutive cells), issuing the
// loads of both before either collision and keeping the two 16-bit values of each direction in one
// register.  v0 / v1: the cell exists and takes this path.

template <int S, bool FORCE>
LBM_HD void store_local_one(const StepArgs &a, int n, uint8_t fl, const float (&g)[Q]) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    constexpr int LS = reg_log2<S, FORCE>();
    T *const *P = (T *const *)a.plane;
    if (fl & F_REDIR) {
        const unsigned nb = a.info[n] >> 8;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool bb = (nb >> i) & 1u;
            (bb ? P[i] : P[opp(i)])[bb ? n + a.off[i] : n] = Cd::template enc_s<LS>(g[i]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) P[opp(i)][n] = Cd::template enc_s<LS>(g[i]);
    }
    if (fl & F_ZG) {
        int x, y, z;
        cell_coords(a.g, n, x, y, z);
        store_side<T>(a.g, a.side, x, y, z, g, [](float v) { return Cd::template enc_s<LS>(v); });
    }
}

template <int S, bool FORCE>
LBM_HD void cell2_local(const StepArgs &a, int n0, int n1, bool v0, bool v1) {
    using Cd = Codec<S>;
    constexpr int LS = reg_log2<S, FORCE>();
    const unsigned short *const *P = (const unsigned short *const *)a.plane;
    uint32_t pk[Q];   // loaded before the flags are known (n1 may be past N: guard region)
#pragma unroll
    for (int i = 0; i < Q; ++i) pk[i] = ld_early_u16(P[i] + n0) | (ld_early_u16(P[i] + n1) << 16);
    const uint8_t f0 = v0 ? a.flags[n0] : F_SOLID, f1 = v1 ? a.flags[n1] : F_SOLID;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const uint8_t fl = c ? f1 : f0;
        if (fl & F_SOLID) continue;
        const int n = c ? n1 : n0;
        float g[Q];
        if (fl & F_EQ) {
            eq_cell_g_s<LS>(a, n, g);
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] = Cd::template dec_bits_s<LS>(c ? pk[i] >> 16 : pk[i] & 0xffffu);
            collide<FORCE, kPairs16, LS>(g, a);
            if (FORCE) nudge(a, n, g);   // relaxation zones ride on the general (forced) path
        }
        store_local_one<S, FORCE>(a, n, fl, g);
    }
}

template <int S, bool FORCE>
LBM_HD void cell2_neighbor_interior(const StepArgs &a, int n0, int n1, bool v0, bool v1) {
    using Cd = Codec<S>;
    constexpr int LS = reg_log2<S, FORCE>();
    unsigned short *const *P = (unsigned short *const *)a.plane;
    uint32_t pk[Q];   // loaded before the flags are known (guard region after the planes)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const unsigned short *p = P[opp(i)] - a.off[i];
        pk[i] = ld_early_u16(p + n0) | (ld_early_u16(p + n1) << 16);
    }
    const uint8_t f0 = v0 ? a.flags[n0] : F_SOLID, f1 = v1 ? a.flags[n1] : F_SOLID;
    const bool l0 = !(f0 & (F_SOLID | F_FACE)), l1 = !(f1 & (F_SOLID | F_FACE));
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!(c ? l1 : l0)) continue;
        const int n = c ? n1 : n0;
        const uint8_t fl = c ? f1 : f0;
        float g[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = Cd::template dec_bits_s<LS>(c ? pk[i] >> 16 : pk[i] & 0xffffu);
        collide<FORCE, kPairs16, LS>(g, a);
        if (FORCE) nudge(a, n, g);   // relaxation zones ride on the general (forced) path
        const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
        if (nb) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool bb = (nb >> i) & 1u;
                (bb ? P[opp(i)] : P[i])[bb ? n : n + a.off[i]] = Cd::template enc_bits_s<LS>(g[i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) P[i][n + a.off[i]] = Cd::template enc_bits_s<LS>(g[i]);
        }
    }
}

// Adjacent pairs (n0 = 2m, n0 + 1) with 4-byte accesses, for 16-bit storage when N and nx are
// even (plane bases and every c_x = 0 neighbour offset are then 4-byte aligned).  A warp load is
// 128 bytes, as in FP32 storage.  Pairs whose cells need individual handling (a solid cell, whose
// slots may be receiving a neighbour's bounce-back store, or a cell with redirected links) fall
// back to per-cell stores.

template <int S, bool FORCE>
LBM_HD void cellp_local(const StepArgs &a, int n0) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    constexpr int LS = reg_log2<S, FORCE>();
    const int m = n0 >> 1;
    uint32_t pk[Q];   // inputs; each half is replaced by its cell's encoded result once computed
#pragma unroll
    for (int i = 0; i < Q; ++i) pk[i] = ld_early_u32((const uint32_t *)a.plane[i] + m);   // before the flags
    const uint8_t f0 = a.flags[n0], f1 = a.flags[n0 + 1];
    if ((f0 & f1) & F_SOLID) return;
    // phase 1: both collisions, results packed into pk
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const uint8_t fl = c ? f1 : f0;
        if (fl & F_SOLID) continue;
        float g[Q];
        if (fl & F_EQ) {
            eq_cell_g_s<LS>(a, n0 + c, g);
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] = Cd::template dec_bits_s<LS>(c ? pk[i] >> 16 : pk[i] & 0xffffu);
            collide<FORCE, kPairs16, LS>(g, a);
            if (FORCE) nudge(a, n0 + c, g);   // relaxation zones ride on the general (forced) path
        }
        if (fl & F_ZG) {
            int x, y, z;
            cell_coords(a.g, n0 + c, x, y, z);
            store_side<T>(a.g, a.side, x, y, z, g, [](float v) { return Cd::template enc_s<LS>(v); });
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const uint32_t bits = Cd::template enc_bits_s<LS>(g[i]);
            pk[i] = c ? ((pk[i] & 0xffffu) | (bits << 16)) : ((pk[i] & 0xffff0000u) | bits);
        }
    }
    // phase 2: stores -- one 4-byte store per plane, unless a cell of the pair is solid (its
    // slots may be receiving a neighbour's bounce-back store) or redirects links
    if (!((f0 | f1) & (F_SOLID | F_REDIR))) {
#pragma unroll
        for (int i = 0; i < Q; ++i) ((uint32_t *)a.plane[opp(i)])[m] = pk[i];
        return;
    }
    unsigned short *const *P = (unsigned short *const *)a.plane;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const uint8_t fl = c ? f1 : f0;
        if (fl & F_SOLID) continue;
        const int n = n0 + c;
        const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool bb = (nb >> i) & 1u;
            (bb ? P[i] : P[opp(i)])[bb ? n + a.off[i] : n] = (unsigned short)(c ? pk[i] >> 16 : pk[i] & 0xffffu);
        }
    }
}

template <int S, bool FORCE>
LBM_HD void cellp_neighbor_interior(const StepArgs &a, int n0) {
    using Cd = Codec<S>;
    constexpr int LS = reg_log2<S, FORCE>();
    unsigned short *const *P = (unsigned short *const *)a.plane;
    const int n1 = n0 + 1;
    uint32_t pk[Q];   // loaded before the flags are known (guard region after the planes)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const unsigned short *p = P[opp(i)] - a.off[i];
        if (cx(i) == 0) pk[i] = ld_early_u32((const uint32_t *)(p + n0));   // adjacent, 4-byte aligned
        else pk[i] = ld_early_u16(p + n0) | (ld_early_u16(p + n1) << 16);
    }
    const uint8_t f0 = a.flags[n0], f1 = a.flags[n1];
    const bool l0 = !(f0 & (F_SOLID | F_FACE)), l1 = !(f1 & (F_SOLID | F_FACE));
    if (!l0 && !l1) return;
    // phase 1: both collisions, results packed into pk
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!(c ? l1 : l0)) continue;
        float g[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = Cd::template dec_bits_s<LS>(c ? pk[i] >> 16 : pk[i] & 0xffffu);
        collide<FORCE, kPairs16, LS>(g, a);
        if (FORCE) nudge(a, c ? n1 : n0, g);   // relaxation zones ride on the general (forced) path
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const uint32_t bits = Cd::template enc_bits_s<LS>(g[i]);
            pk[i] = c ? ((pk[i] & 0xffffu) | (bits << 16)) : ((pk[i] & 0xffff0000u) | bits);
        }
    }
    // phase 2: stores; the c_x = 0 targets of a plain pair are adjacent and 4-byte aligned
    const bool plain = l0 && l1 && !((f0 | f1) & F_REDIR);
    const unsigned nb0 = (l0 && (f0 & F_REDIR)) ? a.info[n0] >> 8 : 0u;
    const unsigned nb1 = (l1 && (f1 & F_REDIR)) ? a.info[n1] >> 8 : 0u;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (plain && cx(i) == 0) {
            *(uint32_t *)(P[i] + n0 + a.off[i]) = pk[i];
            continue;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (!(c ? l1 : l0)) continue;
            const int n = c ? n1 : n0;
            const bool bb = ((c ? nb1 : nb0) >> i) & 1u;
            (bb ? P[opp(i)] : P[i])[bb ? n : n + a.off[i]] = (unsigned short)(c ? pk[i] >> 16 : pk[i] & 0xffffu);
        }
    }
}

// ---------------------------------------------------------------- both cells in one collision
// Unforced 16-bit steps: the two cells of a thread go through collide2 together (FP32x2
// instructions), decoded from and encoded to one 32-bit word per direction.  A lane whose cell is
// solid computes on whatever the slots hold and is discarded; an equilibrium cell's lane is
// overwritten with its equilibrium before encoding.

// Overwrite the lanes of equilibrium cells with their equilibrium (register scale 2^L).
template <int L>
LBM_HD void eq_lanes(const StepArgs &a, long long n0, long long n1, uint8_t f0, uint8_t f1, float2 (&g)[Q]) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!((c ? f1 : f0) & F_EQ)) continue;
        float ge[Q];
        eq_cell_g_s<L>(a, c ? n1 : n0, ge);
#pragma unroll
        for (int i = 0; i < Q; ++i) (c ? g[i].y : g[i].x) = ge[i];
    }
}

// The same on packed words: the halves of equilibrium cells are replaced by their encoded
// equilibrium.
template <int S>
LBM_HD void eq_lanes_packed(const StepArgs &a, long long n0, long long n1, uint8_t f0, uint8_t f1,
                            uint32_t (&pk)[Q]) {
    using Cd = Codec<S>;
    constexpr int LS = Cd::kLog2;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!((c ? f1 : f0) & F_EQ)) continue;
        float ge[Q];
        eq_cell_g_s<LS>(a, c ? n1 : n0, ge);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const uint32_t b = Cd::template enc_bits_s<LS>(ge[i]);
            pk[i] = c ? (pk[i] & 0xffffu) | (b << 16) : (pk[i] & 0xffff0000u) | b;
        }
    }
}

// Forced collision of a 16-bit pair held as packed words n0, n1 (decoded to plain populations,
// through collide2_forced and nudge2, equilibrium lanes overwritten, encoded back).
template <int S>
LBM_HD void collide2_packed_forced(const StepArgs &a, int n0, int n1, uint8_t f0, uint8_t f1, uint32_t (&pk)[Q]) {
    using Cd = Codec<S>;
    float2 g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = Cd::template dec2<0>(pk[i]);
    const float2 drho = collide2_forced<0, 3>(g, a);
    nudge2(a, n0, n1, drho, g);
    if ((f0 | f1) & F_EQ) eq_lanes<0>(a, n0, n1, f0, f1, g);
#pragma unroll
    for (int i = 0; i < Q; ++i) pk[i] = Cd::template enc2<0>(g[i]);
}

// pk: the pair's 19 words (input), f0 / f1: its flags
template <int S, bool FORCE = false>
LBM_HD void cellp_local_dual_body(const StepArgs &a, int n0, uint32_t (&pk)[Q], uint8_t f0, uint8_t f1) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    constexpr int LS = Cd::kLog2;
    const int m = n0 >> 1;
    if ((f0 & f1) & F_SOLID) return;
    if constexpr (FORCE) {
        collide2_packed_forced<S>(a, n0, n0 + 1, f0, f1, pk);
    } else {
        collide2_packed<S>(pk, a);
        if ((f0 | f1) & F_EQ) eq_lanes_packed<S>(a, n0, n0 + 1, f0, f1, pk);
    }
    if ((f0 | f1) & F_ZG) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const uint8_t fl = c ? f1 : f0;
            if (!(fl & F_ZG) || (fl & F_SOLID)) continue;
            float gc[Q];   // the encoded values decode exactly, so the side copies keep their bits
#pragma unroll
            for (int i = 0; i < Q; ++i) gc[i] = Cd::template dec_bits_s<LS>(c ? pk[i] >> 16 : pk[i] & 0xffffu);
            int x, y, z;
            cell_coords(a.g, n0 + c, x, y, z);
            store_side<T>(a.g, a.side, x, y, z, gc, [](float v) { return Cd::template enc_s<LS>(v); });
        }
    }
    // one 4-byte store per plane, unless a cell of the pair is solid (its slots may be receiving a
    // neighbour's bounce-back store) or redirects links
    if (!((f0 | f1) & (F_SOLID | F_REDIR))) {
#pragma unroll
        for (int i = 0; i < Q; ++i) ((uint32_t *)a.plane[opp(i)])[m] = pk[i];
        return;
    }
    unsigned short *const *P = (unsigned short *const *)a.plane;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const uint8_t fl = c ? f1 : f0;
        if (fl & F_SOLID) continue;
        const int n = n0 + c;
        const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const bool bb = (nb >> i) & 1u;
            (bb ? P[i] : P[opp(i)])[bb ? n + a.off[i] : n] = (unsigned short)(c ? pk[i] >> 16 : pk[i] & 0xffffu);
        }
    }
}

// pk: the gathered pair (low half: cell n0), f0 / f1: flags (F_SOLID for a cell that does not exist)
template <int S, bool FORCE = false>
LBM_HD void cell2_neighbor_interior_dual_body(const StepArgs &a, int n0, int n1, uint32_t (&pk)[Q], uint8_t f0,
                                              uint8_t f1) {
    unsigned short *const *P = (unsigned short *const *)a.plane;
    const bool l0 = !(f0 & (F_SOLID | F_FACE)), l1 = !(f1 & (F_SOLID | F_FACE));
    if (!l0 && !l1) return;
    if constexpr (FORCE) collide2_packed_forced<S>(a, n0, n1, 0, 0, pk);   // interior cells: no equilibrium lanes
    else collide2_packed<S>(pk, a);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!(c ? l1 : l0)) continue;
        const int n = c ? n1 : n0;
        const uint8_t fl = c ? f1 : f0;
        const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
        if (nb) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool bb = (nb >> i) & 1u;
                (bb ? P[opp(i)] : P[i])[bb ? n : n + a.off[i]] = (unsigned short)(c ? pk[i] >> 16 : pk[i] & 0xffffu);
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) P[i][n + a.off[i]] = (unsigned short)(c ? pk[i] >> 16 : pk[i] & 0xffffu);
        }
    }
}

template <int S, bool FORCE = false>
LBM_HD void cellp_local_dual(const StepArgs &a, int n0) {
    const int m = n0 >> 1;
    uint32_t pk[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) pk[i] = ld_early_u32((const uint32_t *)a.plane[i] + m);   // before the flags
    cellp_local_dual_body<S, FORCE>(a, n0, pk, a.flags[n0], a.flags[n0 + 1]);
}

template <int S, bool FORCE = false>
LBM_HD void cell2_neighbor_interior_dual(const StepArgs &a, int n0, int n1, bool v0, bool v1) {
    const unsigned short *const *P = (const unsigned short *const *)a.plane;
    uint32_t pk[Q];   // loaded before the flags are known (guard region after the planes)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const unsigned short *p = P[opp(i)] - a.off[i];
        pk[i] = ld_early_u16(p + n0) | (ld_early_u16(p + n1) << 16);
    }
    cell2_neighbor_interior_dual_body<S, FORCE>(a, n0, n1, pk, v0 ? a.flags[n0] : F_SOLID, v1 ? a.flags[n1] : F_SOLID);
}

// ---------------------------------------------------------------- FP32 storage, two cells at once
// Unforced FP32 steps with two cells per thread (n0 and n0 + 256, so every warp access stays 32
// consecutive cells of a plane): both cells' loads are issued before either is computed, and both
// go through one collide2 (FP32x2 instructions).  Stores per cell, as in the one-cell kernels.

// Collision of the pair: unforced, or with the body force and the zone nudging (FORCE).
// FAST: special-function reciprocals and square roots in the collision (see rcp2, collide2_forced)
template <bool FORCE, bool FAST = true>
LBM_HD void collide2_f32(const StepArgs &a, int n0, int n1, float2 (&g)[Q]) {
    if constexpr (FORCE) {
        const float2 drho = collide2_forced<0, FAST ? 7 : 0>(g, a);
        nudge2(a, n0, n1, drho, g);
    } else {
        collide2<0, FAST>(g, a);
    }
}

// The local step's per-cell stores of a collided FP32 pair (solid lanes skipped, store-side
// bounce-back links, outflow side copies).  PLAIN: every link goes to the cell's own reversed slot
// and a link into a solid neighbour also goes to that neighbour's slot (the own slot of such a link
// is read by nobody: the only cell that would gather it is the solid neighbour); else a cell with
// solid neighbours selects one target per link.  The single-domain kernels take the first form, the
// batched ones (other register budgets, where it measured slower) the second.
template <bool PLAIN = true>
LBM_HD void cell2_local_store_f32(const StepArgs &a, int n0, int n1, uint8_t f0, uint8_t f1, const float2 (&g)[Q]) {
    float *const *P = (float *const *)a.plane;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const uint8_t fl = c ? f1 : f0;
        if (fl & F_SOLID) continue;
        const int n = c ? n1 : n0;
        if (PLAIN) {
#pragma unroll
            for (int i = 0; i < Q; ++i) P[opp(i)][n] = c ? g[i].y : g[i].x;
            if (fl & F_REDIR) {
                const unsigned nb = a.info[n] >> 8;
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    if ((nb >> i) & 1u) P[i][n + a.off[i]] = c ? g[i].y : g[i].x;
            }
        } else if (fl & F_REDIR) {
            const unsigned nb = a.info[n] >> 8;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool bb = (nb >> i) & 1u;
                (bb ? P[i] : P[opp(i)])[bb ? n + a.off[i] : n] = c ? g[i].y : g[i].x;
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) P[opp(i)][n] = c ? g[i].y : g[i].x;
        }
        if (fl & F_ZG) {
            float gc[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) gc[i] = c ? g[i].y : g[i].x;
            int x, y, z;
            cell_coords(a.g, n, x, y, z);
            store_side<float>(a.g, a.side, x, y, z, gc, [](float v) { return v; });
        }
    }
}

template <bool FORCE = false, bool FAST = true>
LBM_HD void cell2_local_dual_f32(const StepArgs &a, int n0, int n1, bool v0, bool v1) {
    float *const *P = (float *const *)a.plane;
    float2 g[Q];   // loaded before the flags are known (n1 may be past N: guard region)
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = make_float2(ld_early_f32(P[i] + n0), ld_early_f32(P[i] + n1));
    const uint8_t f0 = v0 ? a.flags[n0] : F_SOLID, f1 = v1 ? a.flags[n1] : F_SOLID;
    if ((f0 & f1) & F_SOLID) return;
    collide2_f32<FORCE, FAST>(a, n0, n1, g);
    if ((f0 | f1) & F_EQ) eq_lanes<0>(a, n0, n1, f0, f1, g);
    cell2_local_store_f32<FAST>(a, n0, n1, f0, f1, g);
}

// The neighbour step's per-cell scatter of a collided FP32 pair (l0 / l1: the lane takes this path;
// a population heading into a solid goes to the cell's own reversed slot).  PLAIN: every link is
// scattered downstream and a link into a solid neighbour also goes to the own reversed slot (its
// downstream store lands in the solid's slot that this same cell gathered its bounce-back from
// earlier in the step, which nothing else reads before the next local step rewrites it); else a
// cell with solid neighbours selects one target per link.
template <bool PLAIN = true>
LBM_HD void cell2_neighbor_store_f32(const StepArgs &a, int n0, int n1, bool l0, bool l1, uint8_t f0, uint8_t f1,
                                     const float2 (&g)[Q]) {
    float *const *P = (float *const *)a.plane;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!(c ? l1 : l0)) continue;
        const int n = c ? n1 : n0;
        const uint8_t fl = c ? f1 : f0;
        if (PLAIN) {
#pragma unroll
            for (int i = 0; i < Q; ++i) P[i][n + a.off[i]] = c ? g[i].y : g[i].x;
            if (fl & F_REDIR) {
                const unsigned nb = a.info[n] >> 8;
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    if ((nb >> i) & 1u) P[opp(i)][n] = c ? g[i].y : g[i].x;
            }
            continue;
        }
        const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
        if (nb) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool bb = (nb >> i) & 1u;
                (bb ? P[opp(i)] : P[i])[bb ? n : n + a.off[i]] = c ? g[i].y : g[i].x;
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) P[i][n + a.off[i]] = c ? g[i].y : g[i].x;
        }
    }
}

template <bool FORCE = false, bool FAST = true>
LBM_HD void cell2_neighbor_interior_dual_f32(const StepArgs &a, int n0, int n1, bool v0, bool v1) {
    float *const *P = (float *const *)a.plane;
    float2 g[Q];   // loaded before the flags are known (guard region after the planes)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float *p = P[opp(i)] - a.off[i];
        g[i] = make_float2(ld_early_f32(p + n0), ld_early_f32(p + n1));
    }
    const uint8_t f0 = v0 ? a.flags[n0] : F_SOLID, f1 = v1 ? a.flags[n1] : F_SOLID;
    const bool l0 = !(f0 & (F_SOLID | F_FACE)), l1 = !(f1 & (F_SOLID | F_FACE));
    if (!l0 && !l1) return;
    collide2_f32<FORCE, FAST>(a, n0, n1, g);
    cell2_neighbor_store_f32<FAST>(a, n0, n1, l0, l1, f0, f1, g);
}

// ---------------------------------------------------------------- ground and top layers in the lattice blocks
// With zlat the neighbour step updates the ground and top layer cells with interior x and y (F_ZL)
// in lattice blocks.  The per-cell form, cell2_neighbor_zl, serves the blocks that straddle a layer
// boundary (and free-slip layer cells next to a solid): both cells of each thread, interior cells
// as cell_neighbor_interior does, F_ZL cells with the rules of cell_neighbor_zlayer (the links
// crossing a no-slip face bounce back, those crossing a free-slip face reflect specularly within the
// layer; a solid mirrored source bounces back), both lanes through one paired collision.  The layer
// of a cell (1: ground, 2: top, 0: other) follows from its index, so every load is issued before the
// flags are known.  Blocks wholly in one layer take the static rules further below.

// Storage element that the neighbour step gathers direction i of cell n from (layer zl).
LBM_HD long long zl_gather_elem(const StepArgs &a, long long n, int zl, int i) {
    const int cross = cz(i) == 1 ? 1 : (cz(i) == -1 ? 2 : 0);   // the layer whose face the link crosses
    if (cross != 0 && zl == cross) {
        if (a.g.face[cross == 1 ? 4 : 5] == LBM_FACE_NOSLIP) return (long long)i * a.g.N + n;
        const int k = (cx(i) == 0 && cy(i) == 0) ? 0 : dir_c(-cx(i), -cy(i), 0);   // in-layer source
        const int d = dir_c(cx(i), cy(i), -cz(i));                                  // its direction
        return (long long)opp(d) * a.g.N + n + a.off[k];
    }
    return (long long)opp(i) * a.g.N + n - a.off[i];
}
// Storage element that the neighbour step scatters direction j of cell n to (layer zl, solid
// neighbour mask nb).
LBM_HD long long zl_scatter_elem(const StepArgs &a, long long n, int zl, unsigned nb, int j) {
    const int cross = cz(j) == -1 ? 1 : (cz(j) == 1 ? 2 : 0);   // target beyond the ground / top
    if (cross != 0 && zl == cross) {
        if (a.g.face[cross == 1 ? 4 : 5] == LBM_FACE_NOSLIP) return (long long)opp(j) * a.g.N + n;
        const int k = (cx(j) == 0 && cy(j) == 0) ? 0 : dir_c(cx(j), cy(j), 0);   // in-layer consumer
        const int m = dir_c(cx(j), cy(j), -cz(j));                                // reflected direction
        const bool bb = k != 0 && ((nb >> k) & 1u);
        return bb ? (long long)opp(j) * a.g.N + n : (long long)m * a.g.N + n + a.off[k];
    }
    return ((nb >> j) & 1u) ? (long long)opp(j) * a.g.N + n : (long long)j * a.g.N + n + a.off[j];
}

template <int S> LBM_HD float ld_early_dec(const void *base, long long e) {
    using Cd = Codec<S>;
    if constexpr (S == LBM_F32) return ld_early_f32((const float *)base + e);
    else return Cd::dec_bits(ld_early_u16((const unsigned short *)base + e));
}

// n1 (= n0 + the block size) exists when v1; both cells lie in the same lattice block.
template <int S, bool FORCE>
LBM_HD void cell2_neighbor_zl(const StepArgs &a, int n0, int n1, bool v1) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    T *const f = (T *)a.f;
    const long long A = a.g.sz, N = a.g.N;
    const int m1 = v1 ? n1 : n0;   // a missing second cell repeats the first, and is discarded
    const int zl0 = n0 < A ? 1 : (n0 >= N - A ? 2 : 0), zl1 = m1 < A ? 1 : (m1 >= N - A ? 2 : 0);
    float2 g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i)
        g[i] = make_float2(ld_early_dec<S>(f, zl_gather_elem(a, n0, zl0, i)), ld_early_dec<S>(f, zl_gather_elem(a, m1, zl1, i)));
    const uint8_t f0 = a.flags[n0], f1 = v1 ? a.flags[n1] : F_SOLID;
    const bool l0 = !(f0 & F_SOLID) && (!(f0 & F_FACE) || (f0 & F_ZL));
    const bool l1 = !(f1 & F_SOLID) && (!(f1 & F_FACE) || (f1 & F_ZL));
    if (!l0 && !l1) return;
    const unsigned nb0 = (l0 && (f0 & F_REDIR)) ? a.info[n0] >> 8 : 0u, nb1 = (l1 && (f1 & F_REDIR)) ? a.info[m1] >> 8 : 0u;
    // a free-slip face whose mirrored source in the layer is solid: bounce-back instead (own slot i)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int zl = c ? zl1 : zl0;
        const unsigned nb = c ? nb1 : nb0;
        if (zl == 0 || nb == 0 || a.g.face[zl == 1 ? 4 : 5] != LBM_FACE_FREESLIP) continue;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (cz(i) != (zl == 1 ? 1 : -1) || (cx(i) == 0 && cy(i) == 0)) continue;
            if ((nb >> dir_c(-cx(i), -cy(i), 0)) & 1u) (c ? g[i].y : g[i].x) = Cd::dec(f[(long long)i * N + (c ? m1 : n0)]);
        }
    }
    if constexpr (FORCE) {
        const float2 drho = collide2_forced<0>(g, a);
        nudge2(a, n0, m1, drho, g);
    } else {
        collide2<0>(g, a);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!(c ? l1 : l0)) continue;
        const int n = c ? n1 : n0, zl = c ? zl1 : zl0;
        const unsigned nb = c ? nb1 : nb0;
#pragma unroll
        for (int j = 0; j < Q; ++j) f[zl_scatter_elem(a, n, zl, nb, j)] = Cd::enc(c ? g[j].y : g[j].x);
    }
}

// Lattice blocks that lie wholly in the ground layer or wholly in the top layer (zlat) take the
// interior two-cell path with the rules of the crossing links fixed at compile time (ZK below): the
// gather of such a link reads the cell's own slot (no-slip: bounce-back) or the mirrored
// population of the in-layer source (free-slip), and its scatter writes the cell's own reversed
// slot or the mirrored slot of the in-layer consumer.  No tables and no per-lane selection, so
// these cells cost what interior cells cost.  Cells with solid neighbours on a free-slip layer
// (whose mirrored source may be solid) and blocks that straddle a layer boundary take
// cell2_neighbor_zl.
enum : int { ZK_INTERIOR = 0, ZK_GROUND_NOSLIP = 1, ZK_GROUND_FREESLIP = 2, ZK_TOP_NOSLIP = 3, ZK_TOP_FREESLIP = 4,
             ZK_MIXED = 5 };
__host__ __device__ constexpr bool zk_ground(int zk) { return zk == ZK_GROUND_NOSLIP || zk == ZK_GROUND_FREESLIP; }
__host__ __device__ constexpr bool zk_noslip(int zk) { return zk == ZK_GROUND_NOSLIP || zk == ZK_TOP_NOSLIP; }
// the gather of direction i crosses the layer's face
__host__ __device__ constexpr bool zk_cross_in(int zk, int i) { return zk_ground(zk) ? cz(i) == 1 : cz(i) == -1; }
// the scatter of direction j crosses the layer's face
__host__ __device__ constexpr bool zk_cross_out(int zk, int j) { return zk_ground(zk) ? cz(j) == -1 : cz(j) == 1; }

// Base of the gather of direction i (element at base + cell), and of the scatter of direction j.
template <class T, int ZK>
LBM_HD T *zk_gather_base(const StepArgs &a, int i) {
    T *const *P = (T *const *)a.plane;
    if (ZK != ZK_INTERIOR && zk_cross_in(ZK, i)) {
        if (zk_noslip(ZK)) return P[i];
        const int kk = (cx(i) == 0 && cy(i) == 0) ? 0 : dir_c(-cx(i), -cy(i), 0);   // in-layer source
        return P[opp(dir_c(cx(i), cy(i), -cz(i)))] + a.off[kk];
    }
    return P[opp(i)] - a.off[i];
}
template <class T, int ZK>
LBM_HD T *zk_scatter_base(const StepArgs &a, int j) {
    T *const *P = (T *const *)a.plane;
    if (ZK != ZK_INTERIOR && zk_cross_out(ZK, j)) {
        if (zk_noslip(ZK)) return P[opp(j)];
        const int kk = (cx(j) == 0 && cy(j) == 0) ? 0 : dir_c(cx(j), cy(j), 0);     // in-layer consumer
        return P[dir_c(cx(j), cy(j), -cz(j))] + a.off[kk];
    }
    return P[j] + a.off[j];
}

template <int S, bool FORCE> LBM_COLD_HD void neighbor_zl_cells(const StepArgs &a, int n0, int n1, bool v1);

// 16-bit storage, cells n0 and n0 + D of a ground or top block.
template <int S, bool FORCE, int ZK, int D>
LBM_HD void cell2_neighbor_layer_dual(const StepArgs &a, int n0, bool v1) {
    using T = unsigned short;
    const int n1 = n0 + D;
    uint32_t pk[Q];   // loaded before the flags are known (guard region after the planes)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T *p = zk_gather_base<T, ZK>(a, i);
        pk[i] = ld_early_u16(p + n0) | (ld_early_u16(p + n1) << 16);
    }
    const uint8_t f0 = a.flags[n0], f1 = v1 ? a.flags[n1] : F_SOLID;
    const bool l0 = !(f0 & F_SOLID) && (!(f0 & F_FACE) || (f0 & F_ZL));
    const bool l1 = !(f1 & F_SOLID) && (!(f1 & F_FACE) || (f1 & F_ZL));
    if (!l0 && !l1) return;
    if (!zk_noslip(ZK) && ((f0 | f1) & F_REDIR)) {   // a mirrored source may be solid
        neighbor_zl_cells<S, FORCE>(a, n0, n1, v1);
        return;
    }
    if constexpr (FORCE) collide2_packed_forced<S>(a, n0, n1, 0, 0, pk);
    else collide2_packed<S>(pk, a);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!(c ? l1 : l0)) continue;
        const int n = c ? n1 : n0;
        const unsigned nb = ((c ? f1 : f0) & F_REDIR) ? a.info[n] >> 8 : 0u;   // (no-slip layer: no crossing bits)
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const T v = (T)(c ? pk[j] >> 16 : pk[j] & 0xffffu);
            if (!zk_cross_out(ZK, j) && ((nb >> j) & 1u)) ((T *const *)a.plane)[opp(j)][n] = v;
            else zk_scatter_base<T, ZK>(a, j)[n] = v;
        }
    }
}

// FP32 storage, cells n0 and n0 + D of a ground or top block.
template <bool FORCE, int ZK, int D, bool FAST = true>
LBM_HD void cell2_neighbor_layer_dual_f32(const StepArgs &a, int n0, bool v1) {
    const int n1 = n0 + D;
    float2 g[Q];   // loaded before the flags are known (guard region after the planes)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float *p = zk_gather_base<float, ZK>(a, i);
        g[i] = make_float2(ld_early_f32(p + n0), ld_early_f32(p + n1));
    }
    const uint8_t f0 = a.flags[n0], f1 = v1 ? a.flags[n1] : F_SOLID;
    const bool l0 = !(f0 & F_SOLID) && (!(f0 & F_FACE) || (f0 & F_ZL));
    const bool l1 = !(f1 & F_SOLID) && (!(f1 & F_FACE) || (f1 & F_ZL));
    if (!l0 && !l1) return;
    if (!zk_noslip(ZK) && ((f0 | f1) & F_REDIR)) {   // a mirrored source may be solid
        neighbor_zl_cells<LBM_F32, FORCE>(a, n0, n1, v1);
        return;
    }
    collide2_f32<FORCE, FAST>(a, n0, n1, g);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!(c ? l1 : l0)) continue;
        const int n = c ? n1 : n0;
        const unsigned nb = ((c ? f1 : f0) & F_REDIR) ? a.info[n] >> 8 : 0u;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const float v = c ? g[j].y : g[j].x;
            if (!zk_cross_out(ZK, j) && ((nb >> j) & 1u)) ((float *const *)a.plane)[opp(j)][n] = v;
            else zk_scatter_base<float, ZK>(a, j)[n] = v;
        }
    }
}

// ---------------------------------------------------------------- post-collision readback
// Layout A, a cell on a face layer: each population from the first location its scatter wrote.
// A called function, so that the general resolution's registers do not weigh on the callers'
// common paths (the diagnostics kernel reads every cell through read_post).
template <int S>
LBM_COLD_HD void read_post_face(const StepArgs &a, long long n, float (&g)[Q]) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const T *f = (const T *)a.f;
    int x, y, z;
    cell_coords(a.g, n, x, y, z);
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

// Shifted post-collision populations of a non-solid cell n in the current layout.
template <int S>
LBM_HD void read_post(const StepArgs &a, long long n, uint8_t fl, bool layoutA, float (&g)[Q]) {
    using Cd = Codec<S>;
    using T = typename Cd::T;
    const T *f = (const T *)a.f;
    if (fl & F_EQ) {
        // the equilibrium populations as stored (and as consumed by the neighbours)
        int x, y, z;
        cell_coords(a.g, n, x, y, z);
        float ux, uy, uz;
        eq_velocity(a, x, y, z, ux, uy, uz);
        equilibrium_shifted(a.rho_b - 1.0f, ux, uy, uz, g);
#pragma unroll
        for (int j = 0; j < Q; ++j) g[j] = Cd::dec(Cd::enc(g[j]));
        return;
    }
    if (!layoutA) {
        const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
#pragma unroll
        for (int j = 0; j < Q; ++j) g[j] = Cd::dec(f[post_loc_B(a, n, j, nb)]);
        return;
    }
    if (!(fl & F_FACE)) {
        // a cell on no face layer: where the neighbour step stored it (plain downstream slot, or
        // its own reversed slot when the downstream cell is solid)
        const unsigned nb = (fl & F_REDIR) ? a.info[n] >> 8 : 0u;
#pragma unroll
        for (int j = 0; j < Q; ++j)
            g[j] = Cd::dec(f[((nb >> j) & 1u) ? (long long)opp(j) * a.g.N + n : (long long)j * a.g.N + n + a.off[j]]);
        return;
    }
    read_post_face<S>(a, n, g);
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
        r = a.rho_b;
        eq_velocity(a, n, ux, uy, uz);
    } else if (!(fl & F_SOLID)) {
        float g[Q];
        read_post<S>(a, n, fl, layoutA, g);
        macros_of(a, g, r, ux, uy, uz);
    }
}

// ---------------------------------------------------------------- diagnostics (one cell)
// Running diagnostics of one thread: fluid cells counted and their density deviations rho - 1
// summed in FP32 (the deviations are ~1e-3, so a thread's FP32 partial keeps ~1e-10 of the total
// mass; the totals are formed in FP64 across threads), the outward mass flux of the cells on open
// face layers in FP64 (few cells), the largest |u|^2 in FP32, and the fluid cells whose
// populations are not all finite.
struct DiagAcc {
    int cells = 0;
    float drho = 0.0f;
    double flux = 0.0;
    float u2max = 0.0f;
    int bad = 0;
};

// Add the non-solid cell n (equilibrium cells: flux only, at rho_b and their boundary velocity).
template <int S>
LBM_HD void diag_cell(const StepArgs &a, long long n, bool layoutA, DiagAcc &acc) {
    const uint8_t fl = a.flags[n];
    if (fl & F_SOLID) return;
    float r, ux, uy, uz;
    if (fl & F_EQ) {
        r = a.rho_b;
        eq_velocity(a, n, ux, uy, uz);
    } else {
        float g[Q];
        read_post<S>(a, n, fl, layoutA, g);
        float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
        bool finite = true;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            finite &= isfinite(g[i]);
            drho += g[i];
            jx += cx(i) * g[i];
            jy += cy(i) * g[i];
            jz += cz(i) * g[i];
        }
        if (!finite) { ++acc.bad; return; }
        r = 1.0f + drho;
        // after a Guo-forced collision sum c f* = rho u + F/2
        ux = (jx - 0.5f * a.fx) / r;
        uy = (jy - 0.5f * a.fy) / r;
        uz = (jz - 0.5f * a.fz) / r;
        ++acc.cells;
        acc.drho += drho;
        acc.u2max = fmaxf(acc.u2max, ux * ux + uy * uy + uz * uz);
    }
    if (!(fl & F_FACE)) return;   // only face-layer cells lie on an open face
    int x, y, z;
    cell_coords(a.g, n, x, y, z);
    const float uu[3] = {ux, uy, uz};
    const int p[3] = {x, y, z};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int f0 = a.g.face[2 * ax], f1 = a.g.face[2 * ax + 1];
        if ((f0 == LBM_FACE_INFLOW_EQ || f0 == LBM_FACE_OUTFLOW_ZG) && p[ax] == 0) acc.flux -= (double)r * uu[ax];
        if ((f1 == LBM_FACE_INFLOW_EQ || f1 == LBM_FACE_OUTFLOW_ZG) && p[ax] == dim(a.g, ax) - 1)
            acc.flux += (double)r * uu[ax];
    }
}

// Face cell t of the face enumeration (face_cell_xyz).
template <int S>
LBM_HD void diag_face_cell(const StepArgs &a, long long t, bool layoutA, DiagAcc &acc) {
    int x, y, z;
    face_cell_xyz(a.g, t, x, y, z);
    diag_cell<S>(a, cell_of(a.g, x, y, z), layoutA, acc);
}

// Fold the threads' diagnostics of one block (blockDim.x == B) into part[0..3] = (mass, net
// outward flux, max |u|, non-finite cells), in FP64 and in a fixed order (deterministic).
template <int B>
__device__ __forceinline__ void diag_block_store(const DiagAcc &acc, double *__restrict__ part) {
    __shared__ double sh[4][B];
    sh[0][threadIdx.x] = (double)acc.cells + (double)acc.drho;
    sh[1][threadIdx.x] = acc.flux;
    sh[2][threadIdx.x] = (double)sqrtf(acc.u2max);
    sh[3][threadIdx.x] = (double)acc.bad;
    __syncthreads();
    for (int s = B / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
            sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + s]);
            sh[3][threadIdx.x] += sh[3][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[k] = sh[k][0];
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

// ---------------------------------------------------------------- one block of a step kernel
// The work of block `bid` of a local or neighbour step launch over the lattice of `a` (256-thread
// blocks); shared by the single-domain kernels and the batched kernel, which places the blocks of
// several lattices in one grid.
constexpr int kBlock = 256;

// 16-bit storage, unforced steps: both cells of a thread in one FP32x2 collision (1), or one
// after the other (0); chosen by measurement on B300
#ifndef LBM_DUAL16
#define LBM_DUAL16 1
#endif
constexpr bool kDual16 = LBM_DUAL16 != 0;

// FP32 storage: lattices of at least this many cells take two cells per thread through collide2
// (FP32x2), smaller ones one cell per thread -- on B300 the two-cell kernels are 1.5-2% faster on
// the 12.8M-cell city and 19% slower on a 0.79M-cell lattice, where halving the blocks leaves a
// ragged last wave.  (Unforced steps; the general path runs its two cells one after the other.)
#ifndef LBM_DUAL32_MIN_CELLS
#define LBM_DUAL32_MIN_CELLS (1ll << 21)
#endif
constexpr long long kDual32MinCells = LBM_DUAL32_MIN_CELLS;

// cells per thread of the lattice blocks: two for 16-bit storage; for FP32 two when D32, else one
template <int S, bool D32 = false> __host__ __device__ constexpr int cells_per_thread() {
    return (S == LBM_F32 && !D32) ? 1 : 2;
}

// lattice blocks of a launch over N cells (blocks of B threads)
template <int S, bool D32 = false, int B = kBlock> __host__ __device__ inline unsigned lattice_blocks(long long N) {
    const long long cpt = cells_per_thread<S, D32>();
    return (unsigned)(((N + cpt - 1) / cpt + B - 1) / B);
}
template <int B = kBlock>
__host__ __device__ inline unsigned face_blocks_of(long long nface) { return (unsigned)((nface + B - 1) / B); }

// L2 prefetch ahead of the lattice blocks: block b asks the copy engine to bring the population
// tiles of a block about LBM_PF_BYTES of populations further on into L2 (one bulk prefetch per
// plane, no shared memory and no completion to wait for), so that block finds its loads in L2.
// 0 = off.  Measured on B300 (400 x 400 x 80 city): ~5.8 MB ahead is best for FP32 (148 blocks of
// 512 cells) and 16-bit storage (296 blocks) alike; FP32 +4.8%, FP16S +3.7% over no prefetch.
#ifndef LBM_PF_BYTES
#define LBM_PF_BYTES (148 * 512 * 76)
#endif

// Bring [lo, hi) of the population region [base, end) into L2: 16-byte aligned start and length
// (the rule of the bulk copy engine), clamped to the region.
__device__ __forceinline__ void prefetch_l2(const char *base, const char *end, const char *lo, const char *hi) {
    lo = lo < base ? base : lo;
    hi = hi > end ? end : hi;
    const uintptr_t a0 = (uintptr_t)lo & ~(uintptr_t)15, a1 = ((uintptr_t)hi + 15) & ~(uintptr_t)15;
    if (a1 <= a0 || (uintptr_t)end < a1) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((unsigned)(a1 - a0)) : "memory");
}

// The prefetch of lattice block lb + kPfDist (of `nlb`): threads 0..18 take one plane each, the
// cells of that block shifted by -off[i] in plane opp(i) (neighbour step) or in place (local step).
template <int S, bool D32, bool NEIGHBOR, int B = kBlock>
__device__ __forceinline__ void prefetch_ahead(const StepArgs &a, unsigned lb, unsigned nlb) {
    constexpr int sb = S == LBM_F32 ? 4 : 2;
    constexpr long long span = (long long)cells_per_thread<S, D32>() * B;
    constexpr unsigned kPfDist = (unsigned)((long long)LBM_PF_BYTES / (span * sb * Q));
    if constexpr (kPfDist == 0) return;
    if (threadIdx.x >= Q || lb + kPfDist >= nlb) return;
    const int i = threadIdx.x;
    const long long c0 = (long long)(lb + kPfDist) * span - (NEIGHBOR ? a.off[i] : 0);
    const char *base = (const char *)a.f, *end = base + (long long)Q * a.g.N * sb;
    const char *p = (const char *)a.plane[NEIGHBOR ? opp_rt(i) : i];
    prefetch_l2(base, end, p + c0 * sb, p + (c0 + span) * sb);
}

// B: threads per block (the kernels use kBlock; batched launches may choose another size).
// FASTC: the FP32 pair collision takes the special-function forms (kernels at <= 3 blocks per SM).
template <int S, bool FORCE, bool PACK, bool D32 = false, int B = kBlock, bool FASTC = true>
__device__ __forceinline__ void local_block(const StepArgs &a, unsigned bid) {
    prefetch_ahead<S, D32, false, B>(a, bid, lattice_blocks<S, D32, B>(a.g.N));
    if constexpr (S == LBM_F32 && cells_per_thread<S, D32>() == 2) {
        const int n0 = (int)(bid * 2 * B + threadIdx.x), n1 = n0 + B;
        if (n0 >= a.g.N) return;
        cell2_local_dual_f32<FORCE, FASTC>(a, n0, n1, true, n1 < a.g.N);
    } else if constexpr (cells_per_thread<S, D32>() == 1) {
        const int n = (int)(bid * B + threadIdx.x);
        if (n >= a.g.N) return;
        cell_local<S, FORCE>(a, n);
    } else if constexpr (PACK) {
        const int n0 = (int)(bid * 2 * B + 2 * threadIdx.x);
        if (n0 >= a.g.N) return;
        if constexpr (kDual16) cellp_local_dual<S, FORCE>(a, n0);
        else cellp_local<S, FORCE>(a, n0);
    } else {
        const int n0 = (int)(bid * 2 * B + threadIdx.x), n1 = n0 + B;
        if (n0 >= a.g.N) return;
        cell2_local<S, FORCE>(a, n0, n1, true, n1 < a.g.N);
    }
}

// The neighbour-step update of face cell t (face tables, or the general resolution).  With
// LBM_FACE_NOINLINE it is a called function, so that its registers (the table words and the
// populations of one cell) are allocated apart from the lattice path of the same kernel.
#ifndef LBM_FACE_NOINLINE
#define LBM_FACE_NOINLINE 1
#endif
#if LBM_FACE_NOINLINE
#define LBM_FACE_INLINE __noinline__
#else
#define LBM_FACE_INLINE __forceinline__
#endif
template <int S, bool FORCE>
__device__ LBM_FACE_INLINE void face_unit(const StepArgs &a, long long t) {
    int x, y, z;
    if (a.ftab) {   // tables cover every face cell
        if (cell_neighbor_table<S, FORCE>(a, (int)t)) return;
        const int n = (int)(a.ftab[t] & kFtCell);
        cell_coords(a.g, n, x, y, z);
        cell_neighbor_face<S, FORCE>(a, a.flags[n], x, y, z);
        return;
    }
    face_cell_xyz(a.g, t, x, y, z);
    const int n = (int)cell_of(a.g, x, y, z);
    const uint8_t fl = a.flags[n];
    if (fl & F_SOLID) return;
    if (t >= a.zface_begin && ((a.zfast >> (z == 0 ? 0 : 1)) & 1)) {
        cell_neighbor_zlayer<S, FORCE>(a, n, fl, z != 0);
        return;
    }
    cell_neighbor_face<S, FORCE>(a, fl, x, y, z);
}

// A lattice block lb of the neighbour step whose cells reach into the ground or top layer (zlat),
// of kind zk (block_layer_kind): the static layer path on two cells per thread, else (a block
// straddling a layer boundary, or one cell per thread) cell2_neighbor_zl.  The single-domain step
// runs these blocks in a kernel of their own (k_step_layers), so that their five variants do not
// weigh on the registers of the main kernel; the batched kernels take them inline.
// the per-cell layer form for the few blocks that straddle a layer boundary (a called function:
// its registers stay apart from the kernel's)
template <int S, bool FORCE>
LBM_COLD_HD void neighbor_zl_cells(const StepArgs &a, int n0, int n1, bool v1) {
    cell2_neighbor_zl<S, FORCE>(a, n0, n1, v1);
}

template <int S, bool FORCE, bool D32, int B>
LBM_HD void neighbor_layer_unit(const StepArgs &a, unsigned lb, int zk, unsigned tid) {
    constexpr long long cpt = cells_per_thread<S, D32>();
    const long long n0 = (long long)lb * cpt * B + tid, n1 = n0 + B;
    if (n0 >= a.g.N) return;
    const bool v1 = cpt == 2 && n1 < a.g.N;
    if constexpr (cpt == 2) {
#define LBM_LAYER_CASE(ZKV)                                                                                    \
        case ZKV:                                                                                              \
            if constexpr (S == LBM_F32) cell2_neighbor_layer_dual_f32<FORCE, ZKV, B>(a, (int)n0, v1);          \
            else cell2_neighbor_layer_dual<S, FORCE, ZKV, B>(a, (int)n0, v1);                                  \
            return;
        switch (zk) {
            LBM_LAYER_CASE(ZK_GROUND_NOSLIP)
            LBM_LAYER_CASE(ZK_GROUND_FREESLIP)
            LBM_LAYER_CASE(ZK_TOP_NOSLIP)
            LBM_LAYER_CASE(ZK_TOP_FREESLIP)
            default: break;
        }
#undef LBM_LAYER_CASE
    }
    neighbor_zl_cells<S, FORCE>(a, (int)n0, (int)n1, v1);
}

// The lattice blocks of the neighbour step take the ground and top layers (zlat): 1, or 0 to leave
// them to the face blocks (measured: the layer kernel is faster, see k_step_layers).
#ifndef LBM_ZLAT
#define LBM_ZLAT 1
#endif
// face cells the neighbour step's face blocks update
__host__ __device__ inline long long step_face_cells(const StepArgs &a) { return LBM_ZLAT ? a.nface_step : a.nface; }

// Lattice blocks (of span cells, nlb in all) that the single-domain neighbour step gives to
// k_step_layers: [0, g1) and [t0, nlb), the blocks that reach into the ground or top layer; the
// main kernel takes [g1, t0).  Without zlat: none (g1 = 0, t0 = nlb).
struct LayerSplit {
    unsigned g1, t0;
};
__host__ __device__ inline LayerSplit layer_split(const StepArgs &a, long long span, unsigned nlb) {
    if (!LBM_ZLAT || !a.zlat) return {0u, nlb};
    const long long A = a.g.sz;
    long long g1 = (A + span - 1) / span, t0 = (a.g.N - A) / span;
    if (g1 > (long long)nlb) g1 = nlb;
    if (t0 < g1) t0 = g1 = nlb;   // the layers reach every block: all in k_step_layers
    return {(unsigned)g1, (unsigned)t0};
}

// Kind of the lattice block lb (of span cells) with respect to the z layers (zlat).
LBM_HD int block_layer_kind(const StepArgs &a, unsigned lb, long long span) {
    const long long A = a.g.sz, c0 = (long long)lb * span;
    const long long c1 = c0 + span < a.g.N ? c0 + span : a.g.N;
    if (c0 >= A && c1 <= a.g.N - A) return ZK_INTERIOR;
    if (c1 <= A) return a.g.face[4] == LBM_FACE_NOSLIP ? ZK_GROUND_NOSLIP : ZK_GROUND_FREESLIP;
    if (c0 >= a.g.N - A) return a.g.face[5] == LBM_FACE_NOSLIP ? ZK_TOP_NOSLIP : ZK_TOP_FREESLIP;
    return ZK_MIXED;
}

// Position of the face blocks in the grid of a neighbour step.  The face blocks are latency-bound
// (table lookups, one cell per thread) and the lattice blocks bandwidth-bound; launched all first,
// the face blocks filled the GPU for their first waves with the DRAM half idle (about 55 us per
// step on the 400 x 400 x 80 city, for 16-bit and FP32 storage alike).  With pshift >= 0 the face
// blocks sit at every 2^pshift-th unit instead (from unit 0, while they last) and the lattice
// blocks fill the units between, in order, so that the face cells' latency hides under the lattice
// traffic.  pshift < 0: face blocks first.
#ifndef LBM_FACE_INTERLEAVE
#define LBM_FACE_INTERLEAVE 1
#endif
// Shift of the face-block period for fb face blocks among units units (-1: face blocks first): a
// quarter of the largest power of two 2^s with 2^s fb <= units, so that the face blocks, the
// slowest blocks of the launch, all start within the first quarter to half of the grid and none
// runs in the launch's tail (B300, 400 x 400 x 80 city: neighbour step FP32 0.353 -> 0.350 ms,
// FP16S 0.268 -> 0.266 ms against the period 2^s; 2^(s-1), 2^(s-3) and 2^(s-4) in between).
__host__ __device__ inline int face_period_shift(unsigned fb, unsigned units) {
    if (!LBM_FACE_INTERLEAVE || fb == 0) return -1;
    int s = 0;
    while ((2ull << s) * fb <= units) ++s;   // the largest power of two with 2^s fb <= units
    return s > 2 ? s - 2 : 0;
}
// unit u -> face block (*face = true) or lattice block, its index in its kind
__device__ __forceinline__ unsigned unit_of(unsigned u, unsigned fb, int pshift, bool &face) {
    if (pshift < 0) {
        face = u < fb;
        return face ? u : u - fb;
    }
    const unsigned q = u >> pshift;
    const bool at = (u & ((1u << pshift) - 1u)) == 0u;
    face = at && q < fb;
    if (face) return q;
    const unsigned before = q + (at ? 0u : 1u);   // face units at positions below u
    return u - (before < fb ? before : fb);
}

// unit: this block's place in the launch; the lattice blocks of the launch start at lattice block
// lb0.  LAYERS: the launch also covers the ground and top blocks (zlat), handled through
// neighbor_layer_unit, inline (the single-domain step gives them to k_step_layers instead).
template <int S, bool FORCE, bool PACK, bool D32 = false, int B = kBlock, bool LAYERS = false, bool FASTC = true>
__device__ __forceinline__ void neighbor_block(const StepArgs &a, unsigned unit, unsigned face_blocks, int pshift = -1,
                                               unsigned lb0 = 0) {
    bool face;
    const unsigned ub = unit_of(unit, face_blocks, pshift, face);
    // below, bid - face_blocks is the lattice block, bid the face block
    const unsigned bid = face ? ub : ub + face_blocks + lb0;
    if (!face) {
        prefetch_ahead<S, D32, true, B>(a, bid - face_blocks, lattice_blocks<S, D32, B>(a.g.N));
        if constexpr (LAYERS) {
            if (LBM_ZLAT && a.zlat) {
                const int zk = block_layer_kind(a, bid - face_blocks, (long long)cells_per_thread<S, D32>() * B);
                if (zk != ZK_INTERIOR) {
                    neighbor_layer_unit<S, FORCE, D32, B>(a, bid - face_blocks, zk, threadIdx.x);
                    return;
                }
            }
        }
        if constexpr (S == LBM_F32 && cells_per_thread<S, D32>() == 2) {
            const int n0 = (int)((bid - face_blocks) * 2 * B + threadIdx.x), n1 = n0 + B;
            if (n0 >= a.g.N) return;
            cell2_neighbor_interior_dual_f32<FORCE, FASTC>(a, n0, n1, true, n1 < a.g.N);
        } else if constexpr (cells_per_thread<S, D32>() == 1) {
            const int n = (int)((bid - face_blocks) * B + threadIdx.x);
            if (n >= a.g.N) return;
            cell_neighbor_interior<S, FORCE>(a, n);
        } else if constexpr (PACK) {
            const int n0 = (int)((bid - face_blocks) * 2 * B + 2 * threadIdx.x);
            if (n0 >= a.g.N) return;
            cellp_neighbor_interior<S, FORCE>(a, n0);
        } else {
            const int n0 = (int)((bid - face_blocks) * 2 * B + threadIdx.x), n1 = n0 + B;
            if (n0 >= a.g.N) return;
            if constexpr (kDual16) cell2_neighbor_interior_dual<S, FORCE>(a, n0, n1, true, n1 < a.g.N);
            else cell2_neighbor_interior<S, FORCE>(a, n0, n1, true, n1 < a.g.N);
        }
    } else {
        const long long t = (long long)bid * B + threadIdx.x;
        if (t >= step_face_cells(a)) return;
        face_unit<S, FORCE>(a, t);
    }
}

}  // namespace lbm

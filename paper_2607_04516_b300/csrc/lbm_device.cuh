// lbm_device.cuh -- device building blocks of the fused D3Q19 LBM-LES step (sm_103a).
//
// In-place streaming on ONE lattice, odd/even ("AA") pattern.  Two layouts alternate:
//   layout B (after a local step, or after lbm_init_fields):  slot opp(i) of cell x holds the
//            post-collision population f*_i(x) (not yet streamed);
//   layout A (after a neighbour step):  slot i of cell x holds f_i(x), the population that will
//            enter the next collision at x (already streamed).
// local step     (A -> B): read own slots, collide, write own slots in reversed order;
// neighbour step (B -> A): gather the upstream populations from layout B, collide, and scatter
//            each result into the layout-A slot of the cell that will consume it.
// Every memory location is read and written by the same thread within a step, so the update is
// race free in place.  All boundary rules live in the neighbour step (gather side and scatter
// side); the local step touches only its own cell.  The rules (App. D streaming + bounce-back,
// Sec. 3 boundary faces) are:
//   gather of population i at fluid x: s = x - c_i;  a NOSLIP face on any out-of-range axis, or a
//     solid resolved source, gives bounce-back f*_opp(i)(x);  otherwise each out-of-range axis is
//     resolved on its own: PERIODIC wraps, OUTFLOW_ZG clamps (zero gradient), FREESLIP clamps and
//     negates that velocity component; the result is f*_d(s) of the resolved source and direction.
//   scatter: exactly the set of (cell, slot) pairs whose gather resolves to (x, j) -- bounce-back
//     into the cell's own reversed slot, the plain downstream cell (wrapped / mirrored), and the
//     extra zero-gradient copies on an outflow layer -- plus, when none exists (a population
//     leaving through an outflow face), an exit slot that only the samplers read.
// Zero gradient gives one post-collision population two consumers (its plain downstream cell and
// the zero-gradient copy on the outflow layer), which an in-place lattice cannot serve: the plain
// consumer overwrites the slot.  So every outflow face owns a side buffer [19][face cells]: the
// local step (and the initialisation) also stores each layer cell's populations that point into
// the domain from that face there, and a gather that clamps on an outflow face reads them from
// the side buffer.  Its outward-direction slots hold the exits; the two sets never overlap.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include "lbm.h"

// every helper is usable from host code too, so the per-cell update can be exercised off-GPU
#define LBM_HD __host__ __device__ __forceinline__

namespace lbm {

constexpr int Q = 19;

// ---------------------------------------------------------------- lattice (library order)
// 0 rest; 1..6 = +x -x +y -y +z -z; 7..18 = (++0) (--0) (+0+) (-0-) (0++) (0--) (+-0) (-+0)
// (+0-) (-0+) (0+-) (0-+); opposite pairs (2k-1, 2k).
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 13 || i == 15) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 14 || i == 16) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 11 || i == 14 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 12 || i == 13 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
    return (i == 5 || i == 9 || i == 11 || i == 16 || i == 18) ? 1
         : (i == 6 || i == 10 || i == 12 || i == 15 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float wgt(int i) {
    return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr int cc(int i, int a) { return a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i)); }

// direction with the velocity component on axis a negated (runtime argument)
LBM_HD int mirror(int d, int a) {
    int c0 = 0, c1 = 0, c2 = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (i == d) { c0 = cx(i); c1 = cy(i); c2 = cz(i); }
    if (a == 0) c0 = -c0; else if (a == 1) c1 = -c1; else c2 = -c2;
    int r = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        if (cx(i) == c0 && cy(i) == c1 && cz(i) == c2) r = i;
    return r;
}

// ---------------------------------------------------------------- cell flags
enum : uint8_t {
    F_SOLID = 1,   // voxel solid: never updated, never read as a source
    F_EQ = 2,      // equilibrium boundary cell (on an INFLOW_EQ face layer)
    F_SLOW = 4,    // on a face layer or next to a solid: neighbour step takes the general path
    F_ZG = 8       // on an outflow face layer: also stores its inward populations to the side buffer
};

// ---------------------------------------------------------------- storage codecs
template <int S> struct Codec;
template <> struct Codec<LBM_F32> {
    using T = float;
    static LBM_HD float dec(T v) { return v; }
    static LBM_HD T enc(float g) { return g; }
};
template <> struct Codec<LBM_F16S> {
    using T = __half;
    static constexpr float kScale = 16384.0f;          // 2^14: keeps |g| ~ 1e-9 .. 4 normal
    static LBM_HD float dec(T v) { return __half2float(v) * (1.0f / kScale); }
    static LBM_HD T enc(float g) { return __float2half_rn(g * kScale); }
};
template <> struct Codec<LBM_BF16S> {
    using T = __nv_bfloat16;
    static LBM_HD float dec(T v) { return __bfloat162float(v); }
    static LBM_HD T enc(float g) { return __float2bfloat16_rn(g); }
};

// ---------------------------------------------------------------- kernel arguments
struct Geo {
    long long N;          // cells
    int nx, ny, nz;
    int face[6];
    long long sy, sz;     // strides of y and z in cells
};

struct StepArgs {
    void *f;                    // 19 * N populations (storage type)
    const uint8_t *flags;       // N
    const float *ub;            // nz * 3 inflow velocity per height
    void *side[6];              // per outflow face: 19 * (face cells) side/exit buffer, else null
    Geo g;
    float tau;
    float c2x18;                // 2 (C Delta)^2 / c_s^4 = 18 C^2
    float rho_b;
    float fx, fy, fz;           // body-force density (Guo)
};

// ---------------------------------------------------------------- physics (FP32)
// Equilibrium in shifted form: g^eq_i = f^eq_i - w_i = w_i (drho + rho (3 c.u + 4.5 (c.u)^2
// - 1.5 u.u))  (Eq. D.4 with c_s^2 = 1/3).
LBM_HD void equilibrium_shifted(float drho, float ux, float uy, float uz,
                                                    float (&g)[Q]) {
    const float rho = 1.0f + drho;
    const float u2 = 1.5f * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        g[i] = wgt(i) * (drho + rho * (cu * (3.0f + 4.5f * cu) - u2));
    }
}

// Moments (D.1), equilibrium (D.4), non-equilibrium flux (D.8), Q (D.10), tau_eff (D.11),
// BGK relaxation (D.2), optional Guo source.  g: shifted pre-collision populations in/out.
template <bool FORCE>
LBM_HD void collide(float (&g)[Q], const StepArgs &a) {
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
    const float irho = 1.0f / rho;
    if (FORCE) {
        jx += 0.5f * a.fx;
        jy += 0.5f * a.fy;
        jz += 0.5f * a.fz;
    }
    const float ux = jx * irho, uy = jy * irho, uz = jz * irho;
    // Pi^neq = sum c c g - drho/3 delta - rho u u   (since sum c c w = delta/3)
    const float d3 = drho * (1.0f / 3.0f);
    const float pxx = sxx - d3 - jx * ux, pyy = syy - d3 - jy * uy, pzz = szz - d3 - jz * uz;
    const float pxy = sxy - jx * uy, pxz = sxz - jx * uz, pyz = syz - jy * uz;
    const float pp = pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (pxy * pxy + pxz * pxz + pyz * pyz);
    const float qn = sqrtf(2.0f * pp);
    const float tau_e = 0.5f * (a.tau + sqrtf(a.tau * a.tau + a.c2x18 * qn * irho));
    const float om = 1.0f / tau_e;
    float geq[Q];
    equilibrium_shifted(drho, ux, uy, uz, geq);
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = fmaf(om, geq[i] - g[i], g[i]);
    if (FORCE) {
        const float pre = 1.0f - 0.5f * om;
        const float uf = ux * a.fx + uy * a.fy + uz * a.fz;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
            const float cf = cx(i) * a.fx + cy(i) * a.fy + cz(i) * a.fz;
            g[i] += pre * wgt(i) * (3.0f * (cf - uf) + 9.0f * cu * cf);
        }
    }
}

// ---------------------------------------------------------------- boundary resolution
LBM_HD long long cell_of(const Geo &G, int x, int y, int z) {
    return (long long)z * G.sz + (long long)y * G.sy + x;
}
LBM_HD int dim(const Geo &G, int a) { return a == 0 ? G.nx : (a == 1 ? G.ny : G.nz); }

// Number of cells of a face of axis a and the index of cell (x, y, z) within it.
LBM_HD long long face_cell(const Geo &G, int a, int x, int y, int z, long long &fcells) {
    if (a == 0) { fcells = (long long)G.ny * G.nz; return (long long)z * G.ny + y; }
    if (a == 1) { fcells = (long long)G.nx * G.nz; return (long long)z * G.nx + x; }
    fcells = (long long)G.nx * G.ny;
    return (long long)y * G.nx + x;
}

// Where the population entering fluid cell p in direction i sits in layout B: kind 0 = lattice
// element index; kind 1 + face = element index in that outflow face's side buffer.
struct Loc {
    int kind;
    long long idx;
};

LBM_HD Loc gather_loc_B(const Geo &G, const uint8_t *flags, int px, int py, int pz, int i) {
    int s[3] = {px - cx(i), py - cy(i), pz - cz(i)};
    const long long self = cell_of(G, px, py, pz);
    bool bb = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (s[a] < 0 && G.face[2 * a] == LBM_FACE_NOSLIP) bb = true;
        if (s[a] >= dim(G, a) && G.face[2 * a + 1] == LBM_FACE_NOSLIP) bb = true;
    }
    int d = i;
    int zg = -1;   // first outflow face the source was clamped onto
    if (!bb) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int n = dim(G, a);
            if (s[a] >= 0 && s[a] < n) continue;
            const int hi = s[a] >= n;
            const int k = G.face[2 * a + hi];
            if (k == LBM_FACE_PERIODIC) {
                s[a] = hi ? s[a] - n : s[a] + n;
            } else {
                s[a] = hi ? n - 1 : 0;
                if (k == LBM_FACE_FREESLIP) d = mirror(d, a);
                if (k == LBM_FACE_OUTFLOW_ZG && zg < 0) zg = 2 * a + hi;
            }
        }
        const long long src = cell_of(G, s[0], s[1], s[2]);
        if (flags[src] & F_SOLID) bb = true;
        else if (zg >= 0) {
            long long fcells;
            const long long fc = face_cell(G, zg >> 1, s[0], s[1], s[2], fcells);
            return Loc{1 + zg, (long long)d * fcells + fc};
        } else {
            return Loc{0, (long long)opp(d) * G.N + src};
        }
    }
    // bounce-back: f*_opp(i)(p) sits in slot i of p in layout B
    return Loc{0, (long long)i * G.N + self};
}

// Visit every layout-A location that must receive the post-collision population j of the
// non-solid cell p.  visit(ptr_kind, element_index): ptr_kind 0 = lattice, 1..6 = exit buffer of
// face (ptr_kind - 1).  Returns the number of visits.
template <class V>
LBM_HD int scatter_targets(const Geo &G, const uint8_t *flags, int px, int py,
                                               int pz, int j, bool fluid, V &&visit) {
    const int p[3] = {px, py, pz};
    int t[3] = {px + cx(j), py + cy(j), pz + cz(j)};
    int visits = 0;

    // (a) bounce-back into the cell's own reversed slot
    bool bb = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (t[a] < 0 && G.face[2 * a] == LBM_FACE_NOSLIP) bb = true;
        if (t[a] >= dim(G, a) && G.face[2 * a + 1] == LBM_FACE_NOSLIP) bb = true;
    }
    if (!bb) {
        int r[3] = {t[0], t[1], t[2]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int n = dim(G, a);
            if (r[a] >= 0 && r[a] < n) continue;
            const int hi = r[a] >= n;
            if (G.face[2 * a + hi] == LBM_FACE_PERIODIC) r[a] = hi ? r[a] - n : r[a] + n;
            else r[a] = hi ? n - 1 : 0;
        }
        if (flags[cell_of(G, r[0], r[1], r[2])] & F_SOLID) bb = true;
    }
    if (bb) {
        visit(0, (long long)opp(j) * G.N + cell_of(G, px, py, pz));
        ++visits;
    }

    // (b) cells whose gather resolves to (p, j): per axis up to two coordinates
    int opt[3][2], flip[3][2], nopt[3];
    int exit_axis = -1, exit_hi = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int n = dim(G, a);
        const int c = cc(j, a);
        nopt[a] = 0;
        if (c == 0) {
            opt[a][0] = p[a]; flip[a][0] = 0; nopt[a] = 1;
            continue;
        }
        if (t[a] >= 0 && t[a] < n) {
            opt[a][nopt[a]] = t[a]; flip[a][nopt[a]] = 0; ++nopt[a];
        } else {
            const int hi = t[a] >= n;
            const int k = G.face[2 * a + hi];
            if (k == LBM_FACE_PERIODIC) {
                opt[a][nopt[a]] = hi ? t[a] - n : t[a] + n; flip[a][nopt[a]] = 0; ++nopt[a];
            } else if (k == LBM_FACE_FREESLIP) {
                opt[a][nopt[a]] = p[a]; flip[a][nopt[a]] = 1; ++nopt[a];
            } else if (k == LBM_FACE_OUTFLOW_ZG && exit_axis < 0) {
                exit_axis = a; exit_hi = hi;
            }
        }
        // zero-gradient copy: p on an outflow layer and c_j pointing inward from that face
        if (c > 0 && p[a] == 0 && G.face[2 * a] == LBM_FACE_OUTFLOW_ZG) {
            opt[a][nopt[a]] = p[a]; flip[a][nopt[a]] = 0; ++nopt[a];
        }
        if (c < 0 && p[a] == n - 1 && G.face[2 * a + 1] == LBM_FACE_OUTFLOW_ZG) {
            opt[a][nopt[a]] = p[a]; flip[a][nopt[a]] = 0; ++nopt[a];
        }
    }
    int nb = 0;
    if (nopt[0] && nopt[1] && nopt[2]) {
        for (int ox = 0; ox < nopt[0]; ++ox)
            for (int oy = 0; oy < nopt[1]; ++oy)
                for (int oz = 0; oz < nopt[2]; ++oz) {
                    const long long y = cell_of(G, opt[0][ox], opt[1][oy], opt[2][oz]);
                    if (flags[y] & F_SOLID) continue;
                    int i = j;
                    if (flip[0][ox]) i = mirror(i, 0);
                    if (flip[1][oy]) i = mirror(i, 1);
                    if (flip[2][oz]) i = mirror(i, 2);
                    visit(0, (long long)i * G.N + y);
                    ++nb;
                }
    }
    visits += nb;

    // (c) nothing in the lattice consumes it: a population leaving through an outflow face
    if (visits == 0 && fluid && exit_axis >= 0) {
        long long fcells;
        const long long fc = face_cell(G, exit_axis, px, py, pz, fcells);
        visit(1 + 2 * exit_axis + exit_hi, (long long)j * fcells + fc);
        ++visits;
    }
    return visits;
}

LBM_HD void cell_coords(const Geo &G, long long n, int &x, int &y, int &z);

// Store the populations of an outflow-layer cell that point into the domain from each outflow
// face it lies on (its zero-gradient copies for the next neighbour step).
template <class T, class Enc>
LBM_HD void store_side(const Geo &G, void *const *side, int x, int y, int z, const float (&g)[Q],
                       Enc enc) {
    const int p[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int hi = 0; hi < 2; ++hi) {
            if (G.face[2 * a + hi] != LBM_FACE_OUTFLOW_ZG) continue;
            if (p[a] != (hi ? dim(G, a) - 1 : 0)) continue;
            long long fcells;
            const long long fc = face_cell(G, a, x, y, z, fcells);
            T *buf = (T *)side[2 * a + hi];
#pragma unroll
            for (int d = 0; d < Q; ++d) {
                const int c = cc(d, a);
                if ((hi && c < 0) || (!hi && c > 0)) buf[(long long)d * fcells + fc] = enc(g[d]);
            }
        }
    }
}

LBM_HD void cell_coords(const Geo &G, long long n, int &x, int &y, int &z) {
    z = (int)(n / G.sz);
    const long long r = n - (long long)z * G.sz;
    y = (int)(r / G.sy);
    x = (int)(r - (long long)y * G.sy);
}

}  // namespace lbm

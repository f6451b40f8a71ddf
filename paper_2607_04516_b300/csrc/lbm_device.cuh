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

// a rarely taken path kept out of line on the device (LBM_COLD_HD: callable from host builds too)
#ifdef __CUDA_ARCH__
#define LBM_COLD __noinline__
#else
#define LBM_COLD
#endif
#define LBM_COLD_HD __host__ __device__ __noinline__

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
// direction index of velocity (vx, vy, vz), -1 if not a D3Q19 velocity (a flat switch, so that the
// compiler folds it wherever the velocity is a constant, e.g. in unrolled direction loops)
__host__ __device__ constexpr int dir_c(int vx, int vy, int vz) {
    switch ((vx + 1) * 9 + (vy + 1) * 3 + (vz + 1)) {
        case 13: return 0;                        // (0, 0, 0)
        case 22: return 1;  case 4: return 2;     // (+1, 0, 0) (-1, 0, 0)
        case 16: return 3;  case 10: return 4;    // (0, +1, 0) (0, -1, 0)
        case 14: return 5;  case 12: return 6;    // (0, 0, +1) (0, 0, -1)
        case 25: return 7;  case 1: return 8;     // (+1, +1, 0) (-1, -1, 0)
        case 23: return 9;  case 3: return 10;    // (+1, 0, +1) (-1, 0, -1)
        case 17: return 11; case 9: return 12;    // (0, +1, +1) (0, -1, -1)
        case 19: return 13; case 7: return 14;    // (+1, -1, 0) (-1, +1, 0)
        case 21: return 15; case 5: return 16;    // (+1, 0, -1) (-1, 0, +1)
        case 15: return 17; case 11: return 18;   // (0, +1, -1) (0, -1, +1)
        default: return -1;
    }
}
constexpr bool dir_c_consistent(int i = 0) {
    return i == Q || (dir_c(cx(i), cy(i), cz(i)) == i && dir_c_consistent(i + 1));
}
static_assert(dir_c_consistent(), "dir_c must invert (cx, cy, cz)");

// Runtime (non-constant) direction arithmetic from packed constants.  Component a of c_d is
// ((PACK_a >> 2d) & 3) - 1; DIR_k holds, in 5-bit fields, the direction index of the velocity with
// key (cx+1)*9 + (cy+1)*3 + (cz+1) (31 where that velocity is not in D3Q19), 12 keys per word.
LBM_HD int crt(int d, int a) {
    const unsigned long long pack = a == 0 ? 0x1489489549ull : (a == 1 ? 0x960949495ull : 0x2214894955ull);
    return (int)((pack >> (2 * d)) & 3ull) - 1;
}
LBM_HD int dir_of(int vx, int vy, int vz) {
    const int k = (vx + 1) * 9 + (vy + 1) * 3 + (vz + 1);
    const unsigned long long w = k < 12 ? 0x9119f77e0257d1full : (k < 24 ? 0x485ff6fd6389406ull : 0x7cffull);
    return (int)((w >> (5 * (k % 12))) & 31ull);
}
// direction with the velocity component on axis a negated
LBM_HD int mirror(int d, int a) {
    const int vx = crt(d, 0), vy = crt(d, 1), vz = crt(d, 2);
    return dir_of(a == 0 ? -vx : vx, a == 1 ? -vy : vy, a == 2 ? -vz : vz);
}
LBM_HD int opp_rt(int d) { return d == 0 ? 0 : ((d & 1) ? d + 1 : d - 1); }

// ---------------------------------------------------------------- cell flags
enum : uint8_t {
    F_SOLID = 1,   // voxel solid: never updated, never read as a source
    F_EQ = 2,      // equilibrium boundary cell (on an INFLOW_EQ face layer)
    F_FACE = 4,    // on a face layer: the neighbour step handles it in the face blocks
    F_ZG = 8,      // on an outflow face layer: also stores its inward populations to the side buffer
    F_REDIR = 16,  // has a solid neighbour and stores bounce-back links into it (see cell_local)
    F_ZL = 32      // ground / top layer cell (interior x and y) that the neighbour step updates in the
                   // lattice blocks instead of the face blocks (both z faces no-slip or free-slip)
};

// ---------------------------------------------------------------- storage codecs
template <int S> struct Codec;
// kLog2: stored value = g * 2^kLog2.  dec_bits_s<L> / enc_bits_s<L> / enc_s<L> work on values
// scaled by 2^L (L = kLog2: the scale is folded into the collision, L = 0: plain g).
template <> struct Codec<LBM_F32> {
    using T = float;
    static constexpr int kLog2 = 0;
    static LBM_HD float dec(T v) { return v; }
    static LBM_HD T enc(float g) { return g; }
};
template <> struct Codec<LBM_F16S> {
    using T = __half;
    static constexpr float kScale = 16384.0f;          // 2^14: keeps |g| ~ 1e-9 .. 4 normal
    static LBM_HD float dec(T v) { return __half2float(v) * (1.0f / kScale); }
    static LBM_HD T enc(float g) { return __float2half_rn(g * kScale); }
    static constexpr int kLog2 = 14;
    static LBM_HD float dec_bits(unsigned b) { return dec(__ushort_as_half((unsigned short)b)); }
    static LBM_HD unsigned short enc_bits(float g) { return __half_as_ushort(enc(g)); }
    template <int L> static LBM_HD float dec_bits_s(unsigned b) {
        const float v = __half2float(__ushort_as_half((unsigned short)b));
        return L == kLog2 ? v : v * (1.0f / kScale);
    }
    template <int L> static LBM_HD T enc_s(float g) { return __float2half_rn(L == kLog2 ? g : g * kScale); }
    template <int L> static LBM_HD unsigned short enc_bits_s(float g) { return __half_as_ushort(enc_s<L>(g)); }
    // two cells in one 32-bit word (low half: first cell)
    template <int L> static LBM_HD float2 dec2(uint32_t u) {
        const float2 v = __half22float2(__halves2half2(__ushort_as_half((unsigned short)(u & 0xffffu)),
                                                       __ushort_as_half((unsigned short)(u >> 16))));
        return L == kLog2 ? v : make_float2(v.x * (1.0f / kScale), v.y * (1.0f / kScale));
    }
    template <int L> static LBM_HD uint32_t enc2(float2 g) {
        const __half2 h = __float22half2_rn(L == kLog2 ? g : make_float2(g.x * kScale, g.y * kScale));
        return (uint32_t)__half_as_ushort(__low2half(h)) | ((uint32_t)__half_as_ushort(__high2half(h)) << 16);
    }
};
template <> struct Codec<LBM_BF16S> {
    using T = __nv_bfloat16;
    static LBM_HD float dec(T v) { return __bfloat162float(v); }
    static LBM_HD T enc(float g) { return __float2bfloat16_rn(g); }
    static constexpr int kLog2 = 0;
    static LBM_HD float dec_bits(unsigned b) { return dec(__ushort_as_bfloat16((unsigned short)b)); }
    static LBM_HD unsigned short enc_bits(float g) { return __bfloat16_as_ushort(enc(g)); }
    template <int L> static LBM_HD float dec_bits_s(unsigned b) { return dec_bits(b); }
    template <int L> static LBM_HD T enc_s(float g) { return enc(g); }
    template <int L> static LBM_HD unsigned short enc_bits_s(float g) { return enc_bits(g); }
    template <int L> static LBM_HD float2 dec2(uint32_t u) {
        return __bfloat1622float2(__halves2bfloat162(__ushort_as_bfloat16((unsigned short)(u & 0xffffu)),
                                                     __ushort_as_bfloat16((unsigned short)(u >> 16))));
    }
    template <int L> static LBM_HD uint32_t enc2(float2 g) {
        const __nv_bfloat162 h = __float22bfloat162_rn(g);
        return (uint32_t)__bfloat16_as_ushort(__low2bfloat16(h)) |
               ((uint32_t)__bfloat16_as_ushort(__high2bfloat16(h)) << 16);
    }
};

// ---------------------------------------------------------------- early loads
// Population loads that must be issued before the cell's flag byte is examined (so that the
// flag load and the population loads overlap instead of costing two DRAM latencies).  Written as
// volatile PTX so the compiler cannot move them into the branch that uses them.  The addresses
// may belong to a neighbouring plane or the workspace guard when the cell turns out to be solid or
// on a face; such values are discarded.  (Host builds read through volatile for the same reason.)
LBM_HD float ld_early_f32(const float *p) {
#ifdef __CUDA_ARCH__
    float v;
    asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
#else
    return *(const volatile float *)p;
#endif
}
LBM_HD unsigned ld_early_u16(const unsigned short *p) {
#ifdef __CUDA_ARCH__
    unsigned short v;
    asm volatile("ld.global.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
#else
    return *(const volatile unsigned short *)p;
#endif
}
LBM_HD uint32_t ld_early_u32(const uint32_t *p) {
#ifdef __CUDA_ARCH__
    uint32_t v;
    asm volatile("ld.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
#else
    return *(const volatile uint32_t *)p;
#endif
}

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
    const uint32_t *info;       // N: flag byte | solid-neighbour mask << 8 (bit 8 + i: x + c_i solid)
                                //    (set for F_REDIR cells)
    const float *ub;            // nz * 3 inflow velocity per height
    void *side[6];              // per outflow face: 19 * (face cells) side/exit buffer, else null
    Geo g;
    float tau;
    float c2x18;                // 2 (C Delta)^2 / c_s^4 = 18 C^2
    float rho_b;
    float fx, fy, fz;           // uniform body-force density (Guo)
    float ox, oy, oz;           // Coriolis rotation vector Omega^lbm (force 2 rho Omega x u)
    long long nface;            // cells on face layers (enumerated by face_cell_xyz)
    void *plane[Q];             // base address of population plane i (= f + i * N elements)
    int off[Q];                 // cell offset of the neighbour x + c_i (c_x + c_y sy + c_z sz)
    int zwrap;                  // nz * sz: cell offset of a periodic wrap along z
    long long zface_begin;      // first face-enumeration index of the z faces (interior x, y)
    int zfast;                  // bit 0 / bit 1: the z- / z+ face cells take the layer path
    int zlat;                   // both z faces take the layer path, in the lattice blocks (F_ZL cells)
    long long nface_step;       // face cells the neighbour step's face blocks update: nface, or
                                // zface_begin when the lattice blocks take the z layers (zlat)
    int pack16;                 // 16-bit storage with N and nx even: lattice blocks update pairs of
                                // adjacent cells with 4-byte accesses
    const float4 *ueq[6];       // synthetic inflow turbulence (App. F): per inflow face x-, x+, y-,
                                // y+, z+ the velocity of its equilibrium cells at the current
                                // anchor, [n2][n1] in the face's plane (x+- : y + ny z;
                                // y+- : x + nx z; z+ : x + nx y); all null = u_b(z)
    const float4 *ueq_next[6];  // the same at the next anchor (used when ueq_alpha != 0)
    float ueq_alpha;            // U = (1 - alpha) ueq + alpha ueq_next
    const uint32_t *ftab;       // face tables of the first ngen face cells (null: every face cell
    int ngen;                   // takes the general resolution); layout in lbm_cell.cuh
    int sponge_top;             // relaxation zones (see nudge): top width, its rate,
    float sponge_sigma;
    int buffer_width;           // lateral width and rate, and the lateral faces that have a zone
    float buffer_sigma;         // (bit k: face k of x-, x+, y-, y+)
    int buffer_faces;
    float flux_shift;           // flux balancing: inward normal shift of equilibrium velocities
    int flux_balance;           // flux balancing on (the shift follows the profile)
    uint32_t div_nx, div_ny;    // multipliers for exact division by nx, ny (see set_divisors)
    int shr_nx, shr_ny;
};

// Division of a cell index 0 <= n < 2^31 by an invariant d >= 1 as floor(n m / 2^(31 + l)) with
// l = ceil(log2 d) and m = ceil(2^(31 + l) / d) < 2^32: exact because m d - 2^(31 + l) < d <= 2^l
// (Granlund and Montgomery, "Division by invariant integers using multiplication", 1994, Thm 4.2).
inline void divisor_of(int d, uint32_t &m, int &shr) {
    int l = 0;
    while ((1ll << l) < d) ++l;
    shr = 31 + l;
    m = (uint32_t)((((unsigned long long)1 << shr) + (unsigned long long)d - 1) / (unsigned long long)d);
}
inline void set_divisors(StepArgs &a) {
    divisor_of(a.g.nx, a.div_nx, a.shr_nx);
    divisor_of(a.g.ny, a.div_ny, a.shr_ny);
}
LBM_HD int div_by(int n, uint32_t m, int shr) { return (int)(((unsigned long long)(unsigned)n * m) >> shr); }

// Face tables (see cell_face_table): 32-bit storage-element codes per face cell
constexpr uint32_t kFtNone = 0xffffffffu;      // no element (head: a solid cell)
constexpr uint32_t kFtGeneral = 0x80000000u;   // head bit: the cell keeps the general resolution
constexpr uint32_t kFtEq = 0x40000000u;        // head bit: an equilibrium cell
constexpr uint32_t kFtCell = 0x3fffffffu;      // head bits of the cell index
constexpr int kFtWords = 3 + 3 * Q;            // words per face cell

// The z face layers whose cells (with interior x and y) take the layer path: no-slip or free-slip
// faces on a lattice at least 3 x 3 x 2.
LBM_HD int zfast_mask(const Geo &G) {
    if (G.nz < 2 || G.nx < 3 || G.ny < 3) return 0;
    const auto ok = [](int k) { return k == LBM_FACE_NOSLIP || k == LBM_FACE_FREESLIP; };
    return (ok(G.face[4]) ? 1 : 0) | (ok(G.face[5]) ? 2 : 0);
}
// The lattice blocks of the neighbour step take the ground and top layers (interior x and y) when
// both z faces take the layer path: then the face enumeration's z part is not visited by the face
// blocks, and those cells carry F_ZL.
LBM_HD bool zlat_of(const Geo &G) { return zfast_mask(G) == 3; }

// ---------------------------------------------------------------- special functions
// 1/x and square roots of the one-cell collision through the GPU's special-function unit
// (__fdividef, rsqrtf: relative error ~1e-7, inside the FP32 rounding the step accumulates anyway;
// measured faster than the IEEE forms in the FP32 step kernels); host builds take the exact forms.
LBM_HD float rcp_fast(float x) {
#ifdef __CUDA_ARCH__
    return __fdividef(1.0f, x);
#else
    return 1.0f / x;
#endif
}
LBM_HD float sqrt_pos_fast(float x) {   // x > 0
#ifdef __CUDA_ARCH__
    return x * rsqrtf(x);
#else
    return sqrtf(x);
#endif
}
LBM_HD float sqrt_nonneg_fast(float x) { return x > 0.0f ? sqrt_pos_fast(x) : 0.0f; }

// Reciprocals and square roots of the pair collisions.  FAST = true: single special-function-unit
// instructions (rcp.approx / sqrt.approx, relative error ~2^-22, far below the FP32 rounding a step
// accumulates anyway) with no slow-path branch; FAST = false: the IEEE forms.  The FP32-storage pair
// collision (collide2, kernels at 3 blocks per SM) takes the fast forms throughout; the 16-bit pair
// collision (collide2_moments, 4 blocks per SM) takes them for 1/rho and the two square roots and
// keeps the IEEE division of 2 / (tau + ...): with all three branch-free the compiler spilled 320
// bytes a thread (16-bit steps 37.6 GLUPS), with these two 53.9 against 52.2 for all-IEEE (400 x 400
// x 80 city, B300).  Host builds take the exact forms.  LBM_FAST2 = 0 / 1 forces one form everywhere
// (for measurements).
#ifndef LBM_FAST2
#define LBM_FAST2 -1
#endif
template <bool FAST> LBM_HD float rcp2_lane(float x) {
#ifdef __CUDA_ARCH__
    if ((LBM_FAST2 < 0 && FAST) || LBM_FAST2 == 1) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
#endif
    return 1.0f / x;
}
template <bool FAST> LBM_HD float sqrt2_lane(float x) {   // x >= 0
#ifdef __CUDA_ARCH__
    if ((LBM_FAST2 < 0 && FAST) || LBM_FAST2 == 1) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
#endif
    return sqrtf(x);
}
template <bool FAST> LBM_HD float2 rcp2(float2 x) { return make_float2(rcp2_lane<FAST>(x.x), rcp2_lane<FAST>(x.y)); }
template <bool FAST> LBM_HD float2 sqrt2(float2 x) { return make_float2(sqrt2_lane<FAST>(x.x), sqrt2_lane<FAST>(x.y)); }

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
//
// Two equivalent evaluation orders (chosen per storage kind by measurement on B300): direction by
// direction, or -- PAIRS, unforced only -- on opposite pairs (2k-1, 2k): s = g_i + g_opp(i) carries the even
// moments, d = g_i - g_opp(i) the odd ones, and the equilibrium of a pair splits into a shared
// even part w (drho + rho (4.5 (c.u)^2 - 1.5 u.u)) and an odd part +-3 w rho c.u, with the
// per-weight coefficients shared by the members of a pair.  Same arithmetic as D.2 / D.4, about
// half the operations of evaluating the 19 equilibria one by one.
// LOG2S (PAIRS only): g holds the populations scaled by 2^LOG2S on input and output (the storage
// scale of FP16 folded into the moments and the equilibrium coefficients; exact, a power of two).
template <bool FORCE, bool PAIRS = false, int LOG2S = 0>
LBM_HD void collide(float (&g)[Q], const StepArgs &a) {
    if (!FORCE && PAIRS) {
        constexpr float S = (float)(1 << LOG2S), iS = 1.0f / S;
        const float s1 = g[1] + g[2], d1 = g[1] - g[2];        // x
        const float s3 = g[3] + g[4], d3 = g[3] - g[4];        // y
        const float s5 = g[5] + g[6], d5 = g[5] - g[6];        // z
        const float s7 = g[7] + g[8], d7 = g[7] - g[8];        // +x+y
        const float s9 = g[9] + g[10], d9 = g[9] - g[10];      // +x+z
        const float s11 = g[11] + g[12], d11 = g[11] - g[12];  // +y+z
        const float s13 = g[13] + g[14], d13 = g[13] - g[14];  // +x-y
        const float s15 = g[15] + g[16], d15 = g[15] - g[16];  // +x-z
        const float s17 = g[17] + g[18], d17 = g[17] - g[18];  // +y-z
        const float drho = iS * (g[0] + (s1 + s3 + s5) + ((s7 + s9) + (s11 + s13)) + (s15 + s17));
        const float jx = iS * (d1 + d7 + d9 + d13 + d15);
        const float jy = iS * (d3 + d7 + d11 - d13 + d17);
        const float jz = iS * (d5 + d9 + d11 - d15 - d17);
        const float sxx = iS * (s1 + s7 + s9 + s13 + s15);
        const float syy = iS * (s3 + s7 + s11 + s13 + s17);
        const float szz = iS * (s5 + s9 + s11 + s15 + s17);
        const float sxy = iS * (s7 - s13), sxz = iS * (s9 - s15), syz = iS * (s11 - s17);
        const float rho = 1.0f + drho;
        const float irho = rcp_fast(rho);
        const float ux = jx * irho, uy = jy * irho, uz = jz * irho;
        const float d3r = drho * (1.0f / 3.0f);
        const float pxx = sxx - d3r - jx * ux, pyy = syy - d3r - jy * uy, pzz = szz - d3r - jz * uz;
        const float pxy = sxy - jx * uy, pxz = sxz - jx * uz, pyz = syz - jy * uz;
        const float pp = pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (pxy * pxy + pxz * pxz + pyz * pyz);
        const float qn = sqrt_nonneg_fast(2.0f * pp);
        const float om = 2.0f * rcp_fast(a.tau + sqrt_pos_fast(a.tau * a.tau + a.c2x18 * qn * irho));
        // per weight class w: even part  w (drho - 1.5 rho u.u) + w 4.5 rho (c.u)^2,
        //                     odd part   w 3 rho (c.u);   g* = g + om (g^eq - g)
        const float e = drho - 1.5f * rho * (ux * ux + uy * uy + uz * uz);
        const float e0 = (S / 3.0f) * e;
        const float e1 = (S / 18.0f) * e, q1 = (0.25f * S) * rho, a1 = rho * (S / 6.0f);
        const float e2 = (S / 36.0f) * e, q2 = (0.125f * S) * rho, a2 = rho * (S / 12.0f);
        g[0] = fmaf(om, e0 - g[0], g[0]);
#define LBM_PAIR(I, CU, E, Qc, Ac)                              \
        {                                                        \
            const float cu_ = (CU);                              \
            const float sym_ = fmaf(Qc * cu_, cu_, E);           \
            const float asym_ = Ac * cu_;                        \
            g[I] = fmaf(om, (sym_ + asym_) - g[I], g[I]);        \
            g[I + 1] = fmaf(om, (sym_ - asym_) - g[I + 1], g[I + 1]); \
        }
        LBM_PAIR(1, ux, e1, q1, a1)
        LBM_PAIR(3, uy, e1, q1, a1)
        LBM_PAIR(5, uz, e1, q1, a1)
        LBM_PAIR(7, ux + uy, e2, q2, a2)
        LBM_PAIR(9, ux + uz, e2, q2, a2)
        LBM_PAIR(11, uy + uz, e2, q2, a2)
        LBM_PAIR(13, ux - uy, e2, q2, a2)
        LBM_PAIR(15, ux - uz, e2, q2, a2)
        LBM_PAIR(17, uy - uz, e2, q2, a2)
#undef LBM_PAIR
        return;
    }
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
    const float irho = rcp_fast(rho);
    // body force of this cell: uniform part + Coriolis 2 rho Omega x (j / rho) = 2 Omega x j (App. E)
    const float Fx = FORCE ? a.fx + 2.0f * (a.oy * jz - a.oz * jy) : 0.0f;
    const float Fy = FORCE ? a.fy + 2.0f * (a.oz * jx - a.ox * jz) : 0.0f;
    const float Fz = FORCE ? a.fz + 2.0f * (a.ox * jy - a.oy * jx) : 0.0f;
    if (FORCE) {
        jx += 0.5f * Fx;
        jy += 0.5f * Fy;
        jz += 0.5f * Fz;
    }
    const float ux = jx * irho, uy = jy * irho, uz = jz * irho;
    // Pi^neq = sum c c g - drho/3 delta - rho u u   (since sum c c w = delta/3)
    const float d3 = drho * (1.0f / 3.0f);
    const float pxx = sxx - d3 - jx * ux, pyy = syy - d3 - jy * uy, pzz = szz - d3 - jz * uz;
    const float pxy = sxy - jx * uy, pxz = sxz - jx * uz, pyz = syz - jy * uz;
    const float pp = pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (pxy * pxy + pxz * pxz + pyz * pyz);
    const float qn = sqrt_nonneg_fast(2.0f * pp);
    const float om = 2.0f * rcp_fast(a.tau + sqrt_pos_fast(a.tau * a.tau + a.c2x18 * qn * irho));
    float geq[Q];
    equilibrium_shifted(drho, ux, uy, uz, geq);
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = fmaf(om, geq[i] - g[i], g[i]);
    if (!FORCE) return;
    const float pre = 1.0f - 0.5f * om;
    const float uf = ux * Fx + uy * Fy + uz * Fz;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        const float cf = cx(i) * Fx + cy(i) * Fy + cz(i) * Fz;
        g[i] += pre * wgt(i) * (3.0f * (cf - uf) + 9.0f * cu * cf);
    }
}

// ---------------------------------------------------------------- two cells at once
// Blackwell executes FP32 arithmetic on pairs of values (FADD2 / FMUL2 / FFMA2: one instruction for
// both lanes of a float2).  collide2 is the unforced pair form of collide<false, true, LOG2S>
// applied to two cells at once, lane x = first cell, lane y = second: the same arithmetic per lane
// (D.1, D.4, D.8-D.11, D.2), equal to the one-cell form up to the order of rounding.
LBM_HD float2 v2(float a) { return make_float2(a, a); }
LBM_HD float2 add2(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
LBM_HD float2 mul2(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    return __fmul2_rn(a, b);
#else
    return make_float2(a.x * b.x, a.y * b.y);
#endif
}
LBM_HD float2 fma2(float2 a, float2 b, float2 c) {
#ifdef __CUDA_ARCH__
    return __ffma2_rn(a, b, c);
#else
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}
LBM_HD float2 sub2(float2 a, float2 b) { return fma2(b, v2(-1.0f), a); }   // a - b, exact rounding
LBM_HD float2 fms2(float2 a, float2 b, float2 c) { return fma2(make_float2(-a.x, -a.y), b, c); }   // c - a b
// 2 / x (the relaxation rate from tau + sqrt(...)): one rounded division in the IEEE form
template <bool FAST> LBM_HD float2 two_over2(float2 x) {
    if ((LBM_FAST2 < 0 && FAST) || LBM_FAST2 == 1) return mul2(v2(2.0f), rcp2<FAST>(x));
    return make_float2(2.0f / x.x, 2.0f / x.y);
}

// The two-cell collision in two phases over an accessor get(i) -> float2 (the shifted populations
// of direction i, scaled by 2^LOG2S) and put(i, float2), for callers short of registers: the
// moments are accumulated pair by pair (s = g_i + g_i+1, d = g_i - g_i+1 of each opposite pair),
// so that besides the populations only the ten running moments are live; the relaxation then
// visits each direction once more.
// Relaxation coefficients of a pair of cells.  With LBM_RELAX_FOLD the rate om is folded into the
// equilibrium coefficients: g* = (1 - om) g + om g^eq, so that om1 = 1 - om and e*, q*, a* (and
// na* = -a*) already carry the factor om; otherwise g* = g + om (g^eq - g).  The two forms are the
// same arithmetic (Eq. D.2) up to FP32 rounding; the folded one takes 6 instead of 9 FP32x2
// instructions per opposite pair.
#ifndef LBM_RELAX_FOLD
#define LBM_RELAX_FOLD 1
#endif
struct Relax2 {
    float2 om, ux, uy, uz, e0, e1, q1, a1, e2, q2, a2, na1, na2;
};

template <int LOG2S, class Get>
LBM_HD Relax2 collide2_moments(Get get, const StepArgs &a) {
    constexpr float S = (float)(1 << LOG2S), iS = 1.0f / S;
    float2 m0 = get(0), jx, jy, jz, sxx, syy, szz, sxy, sxz, syz;
    {
        const float2 u = get(1), w = get(2), s_ = add2(u, w), d_ = sub2(u, w);
        m0 = add2(m0, s_); jx = d_; sxx = s_;
    }
    {
        const float2 u = get(3), w = get(4), s_ = add2(u, w), d_ = sub2(u, w);
        m0 = add2(m0, s_); jy = d_; syy = s_;
    }
    {
        const float2 u = get(5), w = get(6), s_ = add2(u, w), d_ = sub2(u, w);
        m0 = add2(m0, s_); jz = d_; szz = s_;
    }
    {   // (+x, +y)
        const float2 u = get(7), w = get(8), s_ = add2(u, w), d_ = sub2(u, w);
        m0 = add2(m0, s_); jx = add2(jx, d_); jy = add2(jy, d_); sxx = add2(sxx, s_); syy = add2(syy, s_); sxy = s_;
    }
    {   // (+x, +z)
        const float2 u = get(9), w = get(10), s_ = add2(u, w), d_ = sub2(u, w);
        m0 = add2(m0, s_); jx = add2(jx, d_); jz = add2(jz, d_); sxx = add2(sxx, s_); szz = add2(szz, s_); sxz = s_;
    }
    {   // (+y, +z)
        const float2 u = get(11), w = get(12), s_ = add2(u, w), d_ = sub2(u, w);
        m0 = add2(m0, s_); jy = add2(jy, d_); jz = add2(jz, d_); syy = add2(syy, s_); szz = add2(szz, s_); syz = s_;
    }
    {   // (+x, -y)
        const float2 u = get(13), w = get(14), s_ = add2(u, w), d_ = sub2(u, w);
        m0 = add2(m0, s_); jx = add2(jx, d_); jy = sub2(jy, d_); sxx = add2(sxx, s_); syy = add2(syy, s_); sxy = sub2(sxy, s_);
    }
    {   // (+x, -z)
        const float2 u = get(15), w = get(16), s_ = add2(u, w), d_ = sub2(u, w);
        m0 = add2(m0, s_); jx = add2(jx, d_); jz = sub2(jz, d_); sxx = add2(sxx, s_); szz = add2(szz, s_); sxz = sub2(sxz, s_);
    }
    {   // (+y, -z)
        const float2 u = get(17), w = get(18), s_ = add2(u, w), d_ = sub2(u, w);
        m0 = add2(m0, s_); jy = add2(jy, d_); jz = sub2(jz, d_); syy = add2(syy, s_); szz = add2(szz, s_); syz = sub2(syz, s_);
    }
    // the moments stay at the storage scale S: u = j (1/S) / rho, and the stress Pi carries the
    // factor S into Q, which the coefficient of Q under the square root takes back (S a power of 2)
    const float2 drho = LOG2S ? mul2(v2(iS), m0) : m0;
    const float2 rho = add2(v2(1.0f), drho);
    Relax2 r;
    const float2 irho = rcp2<true>(rho);
    const float2 irs = LOG2S ? mul2(v2(iS), irho) : irho;
    r.ux = mul2(jx, irs); r.uy = mul2(jy, irs); r.uz = mul2(jz, irs);
    const float2 d3r = mul2(m0, v2(1.0f / 3.0f));
    const float2 pxx = fms2(jx, r.ux, sub2(sxx, d3r)), pyy = fms2(jy, r.uy, sub2(syy, d3r)),
                 pzz = fms2(jz, r.uz, sub2(szz, d3r));
    const float2 pxy = fms2(jx, r.uy, sxy), pxz = fms2(jx, r.uz, sxz), pyz = fms2(jy, r.uz, syz);
    const float2 pd = fma2(pzz, pzz, fma2(pyy, pyy, mul2(pxx, pxx)));
    const float2 po = fma2(pyz, pyz, fma2(pxz, pxz, mul2(pxy, pxy)));
    const float2 pp2 = fma2(v2(4.0f), po, mul2(v2(2.0f), pd));   // 2 Pi:Pi (times S^2)
    const float2 arg = fma2(mul2(v2(a.c2x18 * iS), irho), sqrt2<true>(pp2), v2(a.tau * a.tau));
    const float2 om = two_over2<false>(add2(v2(a.tau), sqrt2<true>(arg)));
    const float2 uu = fma2(r.uz, r.uz, fma2(r.uy, r.uy, mul2(r.ux, r.ux)));
    const float2 e = fms2(mul2(v2(1.5f), rho), uu, drho);
    if (LBM_RELAX_FOLD) {
        r.om = sub2(v2(1.0f), om);   // 1 - om
        const float2 oe = mul2(om, e), orho = mul2(om, rho);
        r.e0 = mul2(v2(S / 3.0f), oe);
        r.e1 = mul2(v2(S / 18.0f), oe); r.q1 = mul2(v2(0.25f * S), orho); r.a1 = mul2(v2(S / 6.0f), orho);
        r.e2 = mul2(v2(S / 36.0f), oe); r.q2 = mul2(v2(0.125f * S), orho); r.a2 = mul2(v2(S / 12.0f), orho);
        r.na1 = mul2(v2(-S / 6.0f), orho); r.na2 = mul2(v2(-S / 12.0f), orho);
    } else {
        r.om = om;
        r.e0 = mul2(v2(S / 3.0f), e);
        r.e1 = mul2(v2(S / 18.0f), e); r.q1 = mul2(v2(0.25f * S), rho); r.a1 = mul2(v2(S / 6.0f), rho);
        r.e2 = mul2(v2(S / 36.0f), e); r.q2 = mul2(v2(0.125f * S), rho); r.a2 = mul2(v2(S / 12.0f), rho);
    }
    return r;
}

template <class Get, class Put>
LBM_HD void collide2_relax(const Relax2 &r, Get get, Put put) {
    if (LBM_RELAX_FOLD) {
        {
            const float2 g0 = get(0);
            put(0, fma2(r.om, g0, r.e0));
        }
#define LBM_PAIR2(I, CU, E, Qc, Ac, NAc)                             \
        {                                                           \
            const float2 cu_ = (CU);                                \
            const float2 sym_ = fma2(mul2(Qc, cu_), cu_, E);        \
            const float2 gi_ = get(I), gj_ = get(I + 1);            \
            put(I, fma2(r.om, gi_, fma2(Ac, cu_, sym_)));           \
            put(I + 1, fma2(r.om, gj_, fma2(NAc, cu_, sym_)));      \
        }
        LBM_PAIR2(1, r.ux, r.e1, r.q1, r.a1, r.na1)
        LBM_PAIR2(3, r.uy, r.e1, r.q1, r.a1, r.na1)
        LBM_PAIR2(5, r.uz, r.e1, r.q1, r.a1, r.na1)
        LBM_PAIR2(7, add2(r.ux, r.uy), r.e2, r.q2, r.a2, r.na2)
        LBM_PAIR2(9, add2(r.ux, r.uz), r.e2, r.q2, r.a2, r.na2)
        LBM_PAIR2(11, add2(r.uy, r.uz), r.e2, r.q2, r.a2, r.na2)
        LBM_PAIR2(13, sub2(r.ux, r.uy), r.e2, r.q2, r.a2, r.na2)
        LBM_PAIR2(15, sub2(r.ux, r.uz), r.e2, r.q2, r.a2, r.na2)
        LBM_PAIR2(17, sub2(r.uy, r.uz), r.e2, r.q2, r.a2, r.na2)
#undef LBM_PAIR2
        return;
    }
    {
        const float2 g0 = get(0);
        put(0, fma2(r.om, sub2(r.e0, g0), g0));
    }
#define LBM_PAIR2(I, CU, E, Qc, Ac)                                  \
    {                                                               \
        const float2 cu_ = (CU);                                    \
        const float2 sym_ = fma2(mul2(Qc, cu_), cu_, E);            \
        const float2 asym_ = mul2(Ac, cu_);                         \
        const float2 gi_ = get(I), gj_ = get(I + 1);                \
        put(I, fma2(r.om, sub2(add2(sym_, asym_), gi_), gi_));      \
        put(I + 1, fma2(r.om, sub2(sub2(sym_, asym_), gj_), gj_));  \
    }
    LBM_PAIR2(1, r.ux, r.e1, r.q1, r.a1)
    LBM_PAIR2(3, r.uy, r.e1, r.q1, r.a1)
    LBM_PAIR2(5, r.uz, r.e1, r.q1, r.a1)
    LBM_PAIR2(7, add2(r.ux, r.uy), r.e2, r.q2, r.a2)
    LBM_PAIR2(9, add2(r.ux, r.uz), r.e2, r.q2, r.a2)
    LBM_PAIR2(11, add2(r.uy, r.uz), r.e2, r.q2, r.a2)
    LBM_PAIR2(13, sub2(r.ux, r.uy), r.e2, r.q2, r.a2)
    LBM_PAIR2(15, sub2(r.ux, r.uz), r.e2, r.q2, r.a2)
    LBM_PAIR2(17, sub2(r.uy, r.uz), r.e2, r.q2, r.a2)
#undef LBM_PAIR2
}

// Two cells held as float pairs (FP32 storage): the moments as one balanced sum tree (more
// independent instructions in flight than the pair-by-pair accumulation, measured faster there).
template <int LOG2S, bool FAST = true>
LBM_HD void collide2(float2 (&g)[Q], const StepArgs &a) {
    constexpr float S = (float)(1 << LOG2S), iS = 1.0f / S;
    const float2 s1 = add2(g[1], g[2]), d1 = sub2(g[1], g[2]);
    const float2 s3 = add2(g[3], g[4]), d3 = sub2(g[3], g[4]);
    const float2 s5 = add2(g[5], g[6]), d5 = sub2(g[5], g[6]);
    const float2 s7 = add2(g[7], g[8]), d7 = sub2(g[7], g[8]);
    const float2 s9 = add2(g[9], g[10]), d9 = sub2(g[9], g[10]);
    const float2 s11 = add2(g[11], g[12]), d11 = sub2(g[11], g[12]);
    const float2 s13 = add2(g[13], g[14]), d13 = sub2(g[13], g[14]);
    const float2 s15 = add2(g[15], g[16]), d15 = sub2(g[15], g[16]);
    const float2 s17 = add2(g[17], g[18]), d17 = sub2(g[17], g[18]);
    const float2 m0 = add2(add2(add2(g[0], add2(add2(s1, s3), s5)), add2(add2(s7, s9), add2(s11, s13))),
                           add2(s15, s17));
    // moments at the storage scale S (see collide2_moments)
    const float2 jx = add2(add2(add2(add2(d1, d7), d9), d13), d15);
    const float2 jy = add2(sub2(add2(add2(d3, d7), d11), d13), d17);
    const float2 jz = sub2(sub2(add2(add2(d5, d9), d11), d15), d17);
    const float2 sxx = add2(add2(add2(add2(s1, s7), s9), s13), s15);
    const float2 syy = add2(add2(add2(add2(s3, s7), s11), s13), s17);
    const float2 szz = add2(add2(add2(add2(s5, s9), s11), s15), s17);
    const float2 sxy = sub2(s7, s13), sxz = sub2(s9, s15), syz = sub2(s11, s17);
    const float2 drho = LOG2S ? mul2(v2(iS), m0) : m0;
    const float2 rho = add2(v2(1.0f), drho);
    const float2 irho = rcp2<FAST>(rho);
    const float2 irs = LOG2S ? mul2(v2(iS), irho) : irho;
    const float2 ux = mul2(jx, irs), uy = mul2(jy, irs), uz = mul2(jz, irs);
    const float2 d3r = mul2(m0, v2(1.0f / 3.0f));
    const float2 pxx = fms2(jx, ux, sub2(sxx, d3r)), pyy = fms2(jy, uy, sub2(syy, d3r)),
                 pzz = fms2(jz, uz, sub2(szz, d3r));
    const float2 pxy = fms2(jx, uy, sxy), pxz = fms2(jx, uz, sxz), pyz = fms2(jy, uz, syz);
    const float2 pd = fma2(pzz, pzz, fma2(pyy, pyy, mul2(pxx, pxx)));
    const float2 po = fma2(pyz, pyz, fma2(pxz, pxz, mul2(pxy, pxy)));
    const float2 pp2 = fma2(v2(4.0f), po, mul2(v2(2.0f), pd));   // 2 Pi:Pi (times S^2)
    const float2 arg = fma2(mul2(v2(a.c2x18 * iS), irho), sqrt2<FAST>(pp2), v2(a.tau * a.tau));
    const float2 om = two_over2<FAST>(add2(v2(a.tau), sqrt2<FAST>(arg)));
    const float2 uu = fma2(uz, uz, fma2(uy, uy, mul2(ux, ux)));
    const float2 e = fms2(mul2(v2(1.5f), rho), uu, drho);
    if (LBM_RELAX_FOLD) {
        // g* = (1 - om) g + om g^eq with om folded into the equilibrium coefficients
        const float2 om1 = sub2(v2(1.0f), om);
        const float2 oe = mul2(om, e), orho = mul2(om, rho);
        const float2 e0 = mul2(v2(S / 3.0f), oe);
        const float2 e1 = mul2(v2(S / 18.0f), oe), q1 = mul2(v2(0.25f * S), orho), a1 = mul2(v2(S / 6.0f), orho),
                     na1 = mul2(v2(-S / 6.0f), orho);
        const float2 e2 = mul2(v2(S / 36.0f), oe), q2 = mul2(v2(0.125f * S), orho), a2 = mul2(v2(S / 12.0f), orho),
                     na2 = mul2(v2(-S / 12.0f), orho);
        g[0] = fma2(om1, g[0], e0);
#define LBM_PAIR2(I, CU, E, Qc, Ac, NAc)                                \
        {                                                               \
            const float2 cu_ = (CU);                                    \
            const float2 sym_ = fma2(mul2(Qc, cu_), cu_, E);            \
            g[I] = fma2(om1, g[I], fma2(Ac, cu_, sym_));                \
            g[I + 1] = fma2(om1, g[I + 1], fma2(NAc, cu_, sym_));       \
        }
        LBM_PAIR2(1, ux, e1, q1, a1, na1)
        LBM_PAIR2(3, uy, e1, q1, a1, na1)
        LBM_PAIR2(5, uz, e1, q1, a1, na1)
        LBM_PAIR2(7, add2(ux, uy), e2, q2, a2, na2)
        LBM_PAIR2(9, add2(ux, uz), e2, q2, a2, na2)
        LBM_PAIR2(11, add2(uy, uz), e2, q2, a2, na2)
        LBM_PAIR2(13, sub2(ux, uy), e2, q2, a2, na2)
        LBM_PAIR2(15, sub2(ux, uz), e2, q2, a2, na2)
        LBM_PAIR2(17, sub2(uy, uz), e2, q2, a2, na2)
#undef LBM_PAIR2
        return;
    }
    const float2 e0 = mul2(v2(S / 3.0f), e);
    const float2 e1 = mul2(v2(S / 18.0f), e), q1 = mul2(v2(0.25f * S), rho), a1 = mul2(v2(S / 6.0f), rho);
    const float2 e2 = mul2(v2(S / 36.0f), e), q2 = mul2(v2(0.125f * S), rho), a2 = mul2(v2(S / 12.0f), rho);
    g[0] = fma2(om, sub2(e0, g[0]), g[0]);
#define LBM_PAIR2(I, CU, E, Qc, Ac)                                        \
    {                                                                     \
        const float2 cu_ = (CU);                                          \
        const float2 sym_ = fma2(mul2(Qc, cu_), cu_, E);                  \
        const float2 asym_ = mul2(Ac, cu_);                               \
        g[I] = fma2(om, sub2(add2(sym_, asym_), g[I]), g[I]);             \
        g[I + 1] = fma2(om, sub2(sub2(sym_, asym_), g[I + 1]), g[I + 1]); \
    }
    LBM_PAIR2(1, ux, e1, q1, a1)
    LBM_PAIR2(3, uy, e1, q1, a1)
    LBM_PAIR2(5, uz, e1, q1, a1)
    LBM_PAIR2(7, add2(ux, uy), e2, q2, a2)
    LBM_PAIR2(9, add2(ux, uz), e2, q2, a2)
    LBM_PAIR2(11, add2(uy, uz), e2, q2, a2)
    LBM_PAIR2(13, sub2(ux, uy), e2, q2, a2)
    LBM_PAIR2(15, sub2(ux, uz), e2, q2, a2)
    LBM_PAIR2(17, sub2(uy, uz), e2, q2, a2)
#undef LBM_PAIR2
}

// Forced pair form of collide<true>: the body force F = f + 2 Omega x j of each lane (uniform part
// plus Coriolis, App. E), the half-force velocity u = (j + F/2) / rho in the equilibrium and the
// stress, and Guo's source (1 - om/2) w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)] added to the relaxed
// populations.  On an opposite pair (c_j = -c_i) the source splits like the equilibrium into a
// shared even part (1 - om/2) w (9 (c.u)(c.F) - 3 u.F) and an odd part +-(1 - om/2) 3 w c.F.  The
// same arithmetic per lane as the one-cell form up to the order of rounding.  Returns drho.
// FM: the special-function forms (see rcp2) for 1/rho (bit 0), the square roots (bit 1) and the
// division 2 / (tau + ...) (bit 2): all three for the FP32 two-cell kernels (3 blocks per SM), the
// first two for the 16-bit ones (4 blocks per SM: with all three the compiler spills); measured on
// B300, 400 x 400 x 80 city: FP32 zones 31.7 -> 33.1, FP16S with every physics term 33.6 -> 35.5 GLUPS.
template <int LOG2S, int FM = 0>
LBM_HD float2 collide2_forced(float2 (&g)[Q], const StepArgs &a) {
    constexpr float S = (float)(1 << LOG2S), iS = 1.0f / S;
    const float2 s1 = add2(g[1], g[2]), d1 = sub2(g[1], g[2]);
    const float2 s3 = add2(g[3], g[4]), d3 = sub2(g[3], g[4]);
    const float2 s5 = add2(g[5], g[6]), d5 = sub2(g[5], g[6]);
    const float2 s7 = add2(g[7], g[8]), d7 = sub2(g[7], g[8]);
    const float2 s9 = add2(g[9], g[10]), d9 = sub2(g[9], g[10]);
    const float2 s11 = add2(g[11], g[12]), d11 = sub2(g[11], g[12]);
    const float2 s13 = add2(g[13], g[14]), d13 = sub2(g[13], g[14]);
    const float2 s15 = add2(g[15], g[16]), d15 = sub2(g[15], g[16]);
    const float2 s17 = add2(g[17], g[18]), d17 = sub2(g[17], g[18]);
    const float2 is = v2(iS);
    const float2 drho = mul2(is, add2(add2(add2(g[0], add2(add2(s1, s3), s5)), add2(add2(s7, s9), add2(s11, s13))),
                                      add2(s15, s17)));
    float2 jx = mul2(is, add2(add2(add2(add2(d1, d7), d9), d13), d15));
    float2 jy = mul2(is, add2(sub2(add2(add2(d3, d7), d11), d13), d17));
    float2 jz = mul2(is, sub2(sub2(add2(add2(d5, d9), d11), d15), d17));
    const float2 sxx = mul2(is, add2(add2(add2(add2(s1, s7), s9), s13), s15));
    const float2 syy = mul2(is, add2(add2(add2(add2(s3, s7), s11), s13), s17));
    const float2 szz = mul2(is, add2(add2(add2(add2(s5, s9), s11), s15), s17));
    const float2 sxy = mul2(is, sub2(s7, s13)), sxz = mul2(is, sub2(s9, s15)), syz = mul2(is, sub2(s11, s17));
    const float2 rho = add2(v2(1.0f), drho);
    const float2 irho = rcp2<(FM & 1) != 0>(rho);
    // F = f + 2 Omega x j
    const float2 Fx = fma2(v2(2.0f), sub2(mul2(v2(a.oy), jz), mul2(v2(a.oz), jy)), v2(a.fx));
    const float2 Fy = fma2(v2(2.0f), sub2(mul2(v2(a.oz), jx), mul2(v2(a.ox), jz)), v2(a.fy));
    const float2 Fz = fma2(v2(2.0f), sub2(mul2(v2(a.ox), jy), mul2(v2(a.oy), jx)), v2(a.fz));
    jx = fma2(v2(0.5f), Fx, jx);
    jy = fma2(v2(0.5f), Fy, jy);
    jz = fma2(v2(0.5f), Fz, jz);
    const float2 ux = mul2(jx, irho), uy = mul2(jy, irho), uz = mul2(jz, irho);
    const float2 d3r = mul2(drho, v2(1.0f / 3.0f));
    const float2 pxx = fms2(jx, ux, sub2(sxx, d3r)), pyy = fms2(jy, uy, sub2(syy, d3r)),
                 pzz = fms2(jz, uz, sub2(szz, d3r));
    const float2 pxy = fms2(jx, uy, sxy), pxz = fms2(jx, uz, sxz), pyz = fms2(jy, uz, syz);
    const float2 pd = fma2(pzz, pzz, fma2(pyy, pyy, mul2(pxx, pxx)));
    const float2 po = fma2(pyz, pyz, fma2(pxz, pxz, mul2(pxy, pxy)));
    const float2 pp2 = fma2(v2(4.0f), po, mul2(v2(2.0f), pd));   // 2 Pi:Pi
    const float2 arg = fma2(mul2(v2(a.c2x18), irho), sqrt2<(FM & 2) != 0>(pp2), v2(a.tau * a.tau));
    const float2 om = two_over2<(FM & 4) != 0>(add2(v2(a.tau), sqrt2<(FM & 2) != 0>(arg)));
    const float2 uu = fma2(uz, uz, fma2(uy, uy, mul2(ux, ux)));
    const float2 e = fms2(mul2(v2(1.5f), rho), uu, drho);
    // source coefficients: pre = (1 - om/2) S, uf = u.F
    const float2 pre = mul2(v2(S), fma2(v2(-0.5f), om, v2(1.0f)));
    const float2 uf = fma2(uz, Fz, fma2(uy, Fy, mul2(ux, Fx)));
    const float2 u3 = mul2(v2(-3.0f), uf);
    g[0] = add2(fma2(om, sub2(mul2(v2(S / 3.0f), e), g[0]), g[0]), mul2(mul2(v2(1.0f / 3.0f), pre), u3));
    const float2 e1 = mul2(v2(S / 18.0f), e), q1 = mul2(v2(0.25f * S), rho), a1 = mul2(v2(S / 6.0f), rho);
    const float2 e2 = mul2(v2(S / 36.0f), e), q2 = mul2(v2(0.125f * S), rho), a2 = mul2(v2(S / 12.0f), rho);
    const float2 p1 = mul2(v2(1.0f / 18.0f), pre), p2 = mul2(v2(1.0f / 36.0f), pre);
#define LBM_PAIR2F(I, CU, CF, E, Qc, Ac, Pw)                                        \
    {                                                                                \
        const float2 cu_ = (CU), cf_ = (CF);                                         \
        const float2 sym_ = fma2(mul2(Qc, cu_), cu_, E);                             \
        const float2 asym_ = mul2(Ac, cu_);                                          \
        const float2 fs_ = mul2(Pw, fma2(mul2(v2(9.0f), cu_), cf_, u3));             \
        const float2 fa_ = mul2(mul2(v2(3.0f), Pw), cf_);                            \
        g[I] = add2(fma2(om, sub2(add2(sym_, asym_), g[I]), g[I]), add2(fs_, fa_));  \
        g[I + 1] = add2(fma2(om, sub2(sub2(sym_, asym_), g[I + 1]), g[I + 1]), sub2(fs_, fa_)); \
    }
    LBM_PAIR2F(1, ux, Fx, e1, q1, a1, p1)
    LBM_PAIR2F(3, uy, Fy, e1, q1, a1, p1)
    LBM_PAIR2F(5, uz, Fz, e1, q1, a1, p1)
    LBM_PAIR2F(7, add2(ux, uy), add2(Fx, Fy), e2, q2, a2, p2)
    LBM_PAIR2F(9, add2(ux, uz), add2(Fx, Fz), e2, q2, a2, p2)
    LBM_PAIR2F(11, add2(uy, uz), add2(Fy, Fz), e2, q2, a2, p2)
    LBM_PAIR2F(13, sub2(ux, uy), sub2(Fx, Fy), e2, q2, a2, p2)
    LBM_PAIR2F(15, sub2(ux, uz), sub2(Fx, Fz), e2, q2, a2, p2)
    LBM_PAIR2F(17, sub2(uy, uz), sub2(Fy, Fz), e2, q2, a2, p2)
#undef LBM_PAIR2F
    return drho;
}

// Two 16-bit cells held as their 19 packed storage words (low half: first cell): each direction
// is decoded where it is used, once for the moments and once for the relaxation, and the result
// is encoded in place, so that 19 registers instead of 38 carry the populations through the
// collision.  The empty asm statements between the phases keep the compiler from holding the
// first phase's decoded values live in place of the second decode.
template <int S>
LBM_HD void collide2_packed(uint32_t (&pk)[Q], const StepArgs &a) {
    using Cd = Codec<S>;
    constexpr int LS = Cd::kLog2;
    const Relax2 r = collide2_moments<LS>([&](int i) { return Cd::template dec2<LS>(pk[i]); }, a);
#ifdef __CUDA_ARCH__
#pragma unroll
    for (int i = 0; i < Q; ++i) asm volatile("" : "+r"(pk[i]));
#endif
    collide2_relax(r, [&](int i) { return Cd::template dec2<LS>(pk[i]); },
                   [&](int i, float2 v) { pk[i] = Cd::template enc2<LS>(v); });
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

// Source of population i entering fluid cell p: bounce-back (bb), or population d of cell src,
// with zg the first outflow face the source position was clamped onto (-1: none).
struct Src {
    bool bb;
    int d;
    int zg;
    int s[3];
    long long src;
};

LBM_HD Src resolve_source(const Geo &G, const uint8_t *flags, int px, int py, int pz, int i) {
    Src r{false, i, -1, {px - cx(i), py - cy(i), pz - cz(i)}, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (r.s[a] < 0 && G.face[2 * a] == LBM_FACE_NOSLIP) r.bb = true;
        if (r.s[a] >= dim(G, a) && G.face[2 * a + 1] == LBM_FACE_NOSLIP) r.bb = true;
    }
    if (r.bb) return r;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int n = dim(G, a);
        if (r.s[a] >= 0 && r.s[a] < n) continue;
        const int hi = r.s[a] >= n;
        const int k = G.face[2 * a + hi];
        if (k == LBM_FACE_PERIODIC) {
            r.s[a] = hi ? r.s[a] - n : r.s[a] + n;
        } else {
            r.s[a] = hi ? n - 1 : 0;
            if (k == LBM_FACE_FREESLIP) r.d = mirror(r.d, a);
            if (k == LBM_FACE_OUTFLOW_ZG && r.zg < 0) r.zg = 2 * a + hi;
        }
    }
    r.src = cell_of(G, r.s[0], r.s[1], r.s[2]);
    if (flags[r.src] & F_SOLID) r.bb = true;
    return r;
}

LBM_HD Loc gather_loc_B(const Geo &G, const uint8_t *flags, int px, int py, int pz, int i) {
    const Src r = resolve_source(G, flags, px, py, pz, i);
    if (!r.bb) {
        if (r.zg >= 0) {
            long long fcells;
            const long long fc = face_cell(G, r.zg >> 1, r.s[0], r.s[1], r.s[2], fcells);
            return Loc{1 + r.zg, (long long)r.d * fcells + fc};
        }
        return Loc{0, (long long)opp_rt(r.d) * G.N + r.src};
    }
    // bounce-back: f*_opp(i)(p) sits in slot i of p in layout B
    return Loc{0, (long long)i * G.N + cell_of(G, px, py, pz)};
}

// Element (d N + cell) of a population-major lattice holding the post-collision state F* in the
// plain (unstreamed) layout, F*_d(cell) in slot d, that the fluid cell p gathers as population i.
LBM_HD long long gather_elem_canon(const Geo &G, const uint8_t *flags, int px, int py, int pz, int i) {
    const Src r = resolve_source(G, flags, px, py, pz, i);
    if (r.bb) return (long long)opp_rt(i) * G.N + cell_of(G, px, py, pz);
    return (long long)r.d * G.N + r.src;
}

// Up to two coordinates on one axis at which a cell consumes population j of cell p (the plain
// downstream coordinate, or the clamped one of a free-slip reflection or a zero-gradient copy).
struct AxisOpt {
    int n;                 // 0, 1 or 2 options
    int c0, c1;            // coordinates
    bool f0, f1;           // negate this velocity component (free-slip reflection)
    bool exit_hi;          // n == 0 because the population leaves through this outflow face
    bool exit;
};

LBM_HD AxisOpt axis_options(const Geo &G, int a, int pa, int c) {
    AxisOpt o{0, 0, 0, false, false, false, false};
    const int n = dim(G, a);
    if (c == 0) { o.n = 1; o.c0 = pa; return o; }
    const int t = pa + c;
    if (t >= 0 && t < n) {
        o.n = 1; o.c0 = t;
    } else {
        const int hi = t >= n;
        const int k = G.face[2 * a + hi];
        if (k == LBM_FACE_PERIODIC) { o.n = 1; o.c0 = hi ? t - n : t + n; }
        else if (k == LBM_FACE_FREESLIP) { o.n = 1; o.c0 = pa; o.f0 = true; }
        else if (k == LBM_FACE_OUTFLOW_ZG) { o.exit = true; o.exit_hi = hi; }
    }
    // zero-gradient copy: p on an outflow layer and c pointing into the domain from that face
    const bool zg_lo = c > 0 && pa == 0 && G.face[2 * a] == LBM_FACE_OUTFLOW_ZG;
    const bool zg_hi = c < 0 && pa == n - 1 && G.face[2 * a + 1] == LBM_FACE_OUTFLOW_ZG;
    if (zg_lo || zg_hi) {
        if (o.n == 0) { o.c0 = pa; o.f0 = false; } else { o.c1 = pa; o.f1 = false; }
        ++o.n;
    }
    return o;
}

// Visit every layout-A location that must receive the post-collision population j of the
// non-solid cell p.  visit(kind, element_index): kind 0 = lattice, 1 + face = that outflow
// face's side buffer (exit slot).  Returns the number of visits.
template <class V>
LBM_HD int scatter_targets(const Geo &G, const uint8_t *flags, int px, int py, int pz, int j,
                           bool fluid, V &&visit) {
    const int cjx = crt(j, 0), cjy = crt(j, 1), cjz = crt(j, 2);
    const int t[3] = {px + cjx, py + cjy, pz + cjz};
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
        visit(0, (long long)opp_rt(j) * G.N + cell_of(G, px, py, pz));
        ++visits;
    }

    // (b) cells whose gather resolves to (p, j)
    const AxisOpt ox = axis_options(G, 0, px, cjx);
    const AxisOpt oy = axis_options(G, 1, py, cjy);
    const AxisOpt oz = axis_options(G, 2, pz, cjz);
#pragma unroll
    for (int kx = 0; kx < 2; ++kx) {
        if (kx >= ox.n) break;
#pragma unroll
        for (int ky = 0; ky < 2; ++ky) {
            if (ky >= oy.n) break;
#pragma unroll
            for (int kz = 0; kz < 2; ++kz) {
                if (kz >= oz.n) break;
                const long long y = cell_of(G, kx ? ox.c1 : ox.c0, ky ? oy.c1 : oy.c0, kz ? oz.c1 : oz.c0);
                if (flags[y] & F_SOLID) continue;
                const bool fx = kx ? ox.f1 : ox.f0, fy = ky ? oy.f1 : oy.f0, fz = kz ? oz.f1 : oz.f0;
                const int i = (fx || fy || fz) ? dir_of(fx ? -cjx : cjx, fy ? -cjy : cjy, fz ? -cjz : cjz) : j;
                visit(0, (long long)i * G.N + y);
                ++visits;
            }
        }
    }

    // (c) nothing in the lattice consumes it: a population leaving through an outflow face
    if (visits == 0 && fluid) {
        const int ea = ox.exit ? 0 : (oy.exit ? 1 : (oz.exit ? 2 : -1));
        if (ea >= 0) {
            const bool ehi = ea == 0 ? ox.exit_hi : (ea == 1 ? oy.exit_hi : oz.exit_hi);
            long long fcells;
            const long long fc = face_cell(G, ea, px, py, pz, fcells);
            visit(1 + 2 * ea + (ehi ? 1 : 0), (long long)j * fcells + fc);
            ++visits;
        }
    }
    return visits;
}

// The face-layer cells, enumerated face by face without repeats: the x faces whole, the y faces
// without their x-edges, the z faces without their x- and y-edges.
LBM_HD long long face_cell_count(const Geo &G) {
    const long long xs = G.nx == 1 ? 1 : 2, ys = G.ny == 1 ? 1 : 2, zs = G.nz == 1 ? 1 : 2;
    const long long ix = G.nx > 2 ? G.nx - 2 : 0, iy = G.ny > 2 ? G.ny - 2 : 0;
    return xs * G.ny * G.nz + ys * ix * G.nz + zs * ix * iy;
}
LBM_HD void face_cell_xyz(const Geo &G, long long t, int &x, int &y, int &z) {
    const long long xs = G.nx == 1 ? 1 : 2, ys = G.ny == 1 ? 1 : 2;
    const long long ix = G.nx > 2 ? G.nx - 2 : 0, iy = G.ny > 2 ? G.ny - 2 : 0;
    const long long nxf = (long long)G.ny * G.nz;
    if (t < xs * nxf) {
        const long long side = t / nxf, r = t - side * nxf;
        x = side ? G.nx - 1 : 0; y = (int)(r % G.ny); z = (int)(r / G.ny);
        return;
    }
    t -= xs * nxf;
    const long long nyf = ix * G.nz;
    if (t < ys * nyf) {
        const long long side = t / nyf, r = t - side * nyf;
        y = side ? G.ny - 1 : 0; x = 1 + (int)(r % ix); z = (int)(r / ix);
        return;
    }
    t -= ys * nyf;
    const long long nzf = ix * iy;
    const long long side = t / nzf, r = t - side * nzf;
    z = side ? G.nz - 1 : 0; x = 1 + (int)(r % ix); y = 1 + (int)(r / ix);
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
    if (G.N <= 0x7fffffffll) {   // 32-bit division (several times cheaper than 64-bit on the GPU)
        const unsigned un = (unsigned)n, sz = (unsigned)G.sz, sy = (unsigned)G.sy;
        const unsigned zz = un / sz, r = un - zz * sz, yy = r / sy;
        z = (int)zz; y = (int)yy; x = (int)(r - yy * sy);
        return;
    }
    z = (int)(n / G.sz);
    const long long r = n - (long long)z * G.sz;
    y = (int)(r / G.sy);
    x = (int)(r - (long long)y * G.sy);
}

// Inward unit normal of the face owning an equilibrium cell for the flux balancing: the first
// INFLOW_EQ face (x-, x+, y-, y+, z-, z+) whose layer holds the cell; -1 if none.
LBM_HD int flux_owner(const Geo &G, int x, int y, int z) {
    const int p[3] = {x, y, z};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int a = k >> 1;
        if (G.face[k] == LBM_FACE_INFLOW_EQ && p[a] == ((k & 1) ? dim(G, a) - 1 : 0)) return k;
    }
    return -1;
}
LBM_HD void add_flux_shift(const StepArgs &a, int x, int y, int z, float &ux, float &uy, float &uz) {
    if (a.flux_shift == 0.0f) return;
    const int k = flux_owner(a.g, x, y, z);
    if (k < 0) return;
    const float v = (k & 1) ? -a.flux_shift : a.flux_shift;
    if (k < 2) ux += v;
    else if (k < 4) uy += v;
    else uz += v;
}

// Velocity of the equilibrium cell (x, y, z).  With synthetic inflow turbulence on, a cell on an
// inflow face takes the value in the plane of the first inflow face holding it, in the order
// x-, x+, y-, y+, z+ (each boundary cell belongs to one face, App. F); a cell on none of them (an
// inflow ground) and every cell without turbulence take the profile u_b(z).
LBM_HD void eq_velocity(const StepArgs &a, int x, int y, int z, float &ux, float &uy, float &uz) {
    const Geo &G = a.g;
    int k = -1;
    long long idx = 0;
    if (a.ueq[0] && x == 0) { k = 0; idx = y + (long long)G.ny * z; }
    else if (a.ueq[1] && x == G.nx - 1) { k = 1; idx = y + (long long)G.ny * z; }
    else if (a.ueq[2] && y == 0) { k = 2; idx = x + (long long)G.nx * z; }
    else if (a.ueq[3] && y == G.ny - 1) { k = 3; idx = x + (long long)G.nx * z; }
    else if (a.ueq[5] && z == G.nz - 1) { k = 5; idx = x + (long long)G.nx * y; }
    if (k >= 0) {
        const float4 v = a.ueq[k][idx];
        ux = v.x; uy = v.y; uz = v.z;
        if (a.ueq_alpha != 0.0f) {   // linear in time between two anchors (App. F, stride s)
            const float4 w = a.ueq_next[k][idx];
            const float al = a.ueq_alpha;
            ux = (1.0f - al) * ux + al * w.x;
            uy = (1.0f - al) * uy + al * w.y;
            uz = (1.0f - al) * uz + al * w.z;
        }
    } else {
        ux = a.ub[3 * z]; uy = a.ub[3 * z + 1]; uz = a.ub[3 * z + 2];
    }
    add_flux_shift(a, x, y, z, ux, uy, uz);
}

LBM_HD void eq_velocity(const StepArgs &a, long long n, float &ux, float &uy, float &uz) {
    int x, y, z;
    cell_coords(a.g, n, x, y, z);
    eq_velocity(a, x, y, z, ux, uy, uz);
}

// Relaxation zones next to the top and the open lateral faces (Sec. 3): after its collision the fluid
// cell n relaxes toward f^eq(rho, u_b(z)) with the largest zone rate s = sigma ((w - d)/w)^2 over the
// zones whose face layer is d < w cells away.  g: shifted post-collision populations (in/out).
LBM_HD float zone_rate(const StepArgs &a, int x, int y, int z) {
    float s = 0.0f;
    if (a.sponge_top > 0) {
        const int d = a.g.nz - 1 - z;
        if (d < a.sponge_top) {
            const float r = (float)(a.sponge_top - d) / (float)a.sponge_top;
            s = fmaxf(s, a.sponge_sigma * r * r);
        }
    }
    if (a.buffer_faces) {
        const int dist[4] = {x, a.g.nx - 1 - x, y, a.g.ny - 1 - y};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!((a.buffer_faces >> k) & 1) || dist[k] >= a.buffer_width) continue;
            const float r = (float)(a.buffer_width - dist[k]) / (float)a.buffer_width;
            s = fmaxf(s, a.buffer_sigma * r * r);
        }
    }
    return s;
}

LBM_HD void nudge(const StepArgs &a, long long n, float (&g)[Q]) {
    if (a.sponge_top <= 0 && a.buffer_faces == 0) return;
    // coordinates by the precomputed divisors (cell indices stay below 2^31)
    const int r = div_by((int)n, a.div_nx, a.shr_nx), x = (int)n - r * a.g.nx;
    const int z = div_by(r, a.div_ny, a.shr_ny), y = r - z * a.g.ny;
    const float s = zone_rate(a, x, y, z);
    if (s <= 0.0f) return;
    float drho = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) drho += g[i];
    float geq[Q];
    equilibrium_shifted(drho, a.ub[3 * z], a.ub[3 * z + 1], a.ub[3 * z + 2], geq);
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = fmaf(-s, g[i] - geq[i], g[i]);
}

// The nudging of two cells n0, n1 (lanes x, y of g; 32-bit cell indices, n1 possibly past the
// lattice for a lane that is discarded), lane by lane as nudge(); a lane whose rate is 0 keeps its
// values exactly.
// drho: the pair's density deviation (the collision conserves it, so the pre-collision value
// serves; equal to the sum of the relaxed populations up to rounding).
LBM_HD void nudge2(const StepArgs &a, int n0, int n1, float2 drho, float2 (&g)[Q]) {
    if (a.sponge_top <= 0 && a.buffer_faces == 0) return;
    float s[2];
    int zc[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int n = c ? n1 : n0;
        const int r = div_by(n, a.div_nx, a.shr_nx), x = n - r * a.g.nx;
        const int z = div_by(r, a.div_ny, a.shr_ny), y = r - z * a.g.ny;
        zc[c] = z < a.g.nz ? z : a.g.nz - 1;
        s[c] = zone_rate(a, x, y, zc[c]);
    }
    if (s[0] <= 0.0f && s[1] <= 0.0f) return;
    const float2 ux = make_float2(a.ub[3 * zc[0]], a.ub[3 * zc[1]]);
    const float2 uy = make_float2(a.ub[3 * zc[0] + 1], a.ub[3 * zc[1] + 1]);
    const float2 uz = make_float2(a.ub[3 * zc[0] + 2], a.ub[3 * zc[1] + 2]);
    const float2 rho = add2(v2(1.0f), drho);
    const float2 ms = make_float2(-s[0], -s[1]);
    // direction by direction (fewer live registers than the opposite-pair form, measured faster)
    const float2 u2 = mul2(v2(1.5f), fma2(uz, uz, fma2(uy, uy, mul2(ux, ux))));
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float2 cu = fma2(v2((float)cz(i)), uz, fma2(v2((float)cy(i)), uy, mul2(v2((float)cx(i)), ux)));
        const float2 geq = mul2(v2(wgt(i)), fma2(rho, sub2(mul2(cu, fma2(v2(4.5f), cu, v2(3.0f))), u2), drho));
        g[i] = fma2(ms, sub2(g[i], geq), g[i]);
    }
}

// Shifted equilibrium of an equilibrium cell.
LBM_HD void eq_cell_g(const StepArgs &a, long long n, float (&g)[Q]) {
    float ux, uy, uz;
    eq_velocity(a, n, ux, uy, uz);
    equilibrium_shifted(a.rho_b - 1.0f, ux, uy, uz, g);
}

}  // namespace lbm

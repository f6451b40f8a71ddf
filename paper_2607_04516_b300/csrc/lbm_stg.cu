// lbm_stg.cu -- synthetic von Karman inflow turbulence (paper App. F): table construction on the
// host, one kernel per step that overwrites the velocity of the inflow faces' equilibrium cells.
#include <cmath>
#include <cstring>

#include "lbm_stg.h"

namespace lbm {

namespace {

constexpr size_t kAl = 256;
inline size_t al(size_t v) { return (v + kAl - 1) / kAl * kAl; }
constexpr int kOrder[5] = {0, 1, 2, 3, 5};   // x-, x+, y-, y+, z+ (never the ground)
constexpr double kPi = 3.14159265358979323846;

int inflow_mask(const Geo &g) {
    int m = 0;
    for (int k : kOrder)
        if (g.face[k] == LBM_FACE_INFLOW_EQ) m |= 1 << k;
    return m;
}

// (x, y, z) of position (i, j) in the plane of face k
LBM_HD void face_pos(const Geo &g, int k, int i, int j, int &x, int &y, int &z) {
    const int a = k / 2, hi = k & 1;
    if (a == 0) { x = hi ? g.nx - 1 : 0; y = i; z = j; }
    else if (a == 1) { x = i; y = hi ? g.ny - 1 : 0; z = j; }
    else { x = i; y = j; z = hi ? g.nz - 1 : 0; }
}

// First inflow face in the order x-, x+, y-, y+, z+ that holds (x, y, z), or -1.
LBM_HD int owner_face(int inflow, const Geo &g, int x, int y, int z) {
    if ((inflow & 1) && x == 0) return 0;
    if ((inflow & 2) && x == g.nx - 1) return 1;
    if ((inflow & 4) && y == 0) return 2;
    if ((inflow & 8) && y == g.ny - 1) return 3;
    if ((inflow & 32) && z == g.nz - 1) return 5;
    return -1;
}

// Time coefficients of mode m at the launch's time t: A_m,a (cos, sin) of the phases, stored as
// two float4 (C_x, C_y, C_z, S_x), (S_y, S_z, -, -).  omega_m t is reduced to turns in FP64 once per
// mode; the per-component phase offsets are added in FP32 within [0, 2).
LBM_HD void stg_coeff(const StgLaunch &L, const StgFace &F, float4 *cs, int m) {
    const StgMode &M = F.mode[m];
    double tw = M.w * (double)L.t;
    tw -= floor(tw);                                        // turns, in [0, 1)
    float C[3], S[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float th = (float)tw + M.ph[c];               // in [0, 2)
#ifdef __CUDA_ARCH__
        sincospif(2.0f * th, &S[c], &C[c]);
#else
        S[c] = (float)sin(2.0 * kPi * th); C[c] = (float)cos(2.0 * kPi * th);
#endif
    }
    cs[2 * m] = make_float4(M.amp[0] * C[0], M.amp[1] * C[1], M.amp[2] * C[2], M.amp[0] * S[0]);
    cs[2 * m + 1] = make_float4(M.amp[1] * S[1], M.amp[2] * S[2], 0.0f, 0.0f);
}

// Whether the position pos of face F is an equilibrium cell this face owns (else nothing is
// written there); if so its plane coordinates, u_b and, when it is turbulent, sigma_i.
LBM_HD bool stg_target(const StgLaunch &L, const StgFace &F, int pos, int &i, int &j, float4 &ub,
                       float &sigma, bool &turb) {
    j = pos / F.n1;
    i = pos - j * F.n1;
    turb = false;
    if (j >= F.n2) return false;
    int x, y, z;
    face_pos(L.g, F.face, i, j, x, y, z);
    if (owner_face(L.inflow, L.g, x, y, z) != F.face) return false;
    if (!(L.flags[cell_of(L.g, x, y, z)] & F_EQ)) return false;
    const float bx = L.ub[3 * z], by = L.ub[3 * z + 1], bz = L.ub[3 * z + 2];
    ub = make_float4(bx, by, bz, 0.0f);
    const int a = F.face / 2;
    const float ua = a == 0 ? bx : (a == 1 ? by : bz);
    const float un = (F.face & 1) ? -ua : ua;               // U_b . n_f, n_f the inward normal
    if (F.keep && !(L.inflow_only && !(un > 0.0f))) {
        turb = true;
        const float uchar = L.char_normal ? fabsf(un) : sqrtf(bx * bx + by * by + bz * bz);
        sigma = L.intensity > 0.0f ? L.intensity * uchar : L.sigma0;
    }
    return true;
}

#ifdef __CUDA_ARCH__
#define STG_LD(p) __ldg(p)
#else
#define STG_LD(p) (*(p))
#endif

// Partial mode sum over m = m0, m0 + dm, ... at plane position (i, j).  The table loads of
// kStgBatch modes are issued together (one memory round trip per batch: the tables are evicted
// from L2 by every lattice step, so each launch reads them from DRAM).
LBM_HD void stg_partial(const StgFace &F, const float4 *cs, int n_modes, int i, int j, int m0, int dm,
                        float &qx, float &qy, float &qz) {
    const float2 *__restrict__ e1 = F.E1 + i + m0 * F.n1;
    const float2 *__restrict__ e2 = F.E2 + j + m0 * F.n2;
    const int s1 = dm * F.n1, s2 = dm * F.n2;
    for (int mb = m0; mb < n_modes; mb += kStgBatch * dm) {
        float2 p[kStgBatch], q[kStgBatch];
#pragma unroll
        for (int u = 0; u < kStgBatch; ++u) {
            if (mb + u * dm < n_modes) {
                p[u] = STG_LD(e1 + u * s1);
                q[u] = STG_LD(e2 + u * s2);
            }
        }
#pragma unroll
        for (int u = 0; u < kStgBatch; ++u) {
            const int m = mb + u * dm;
            if (m < n_modes) {
                const float re = p[u].x * q[u].x - p[u].y * q[u].y;
                const float im = p[u].x * q[u].y + p[u].y * q[u].x;
                const float4 a = cs[2 * m], b = cs[2 * m + 1];
                qx += a.x * re - a.w * im;
                qy += a.y * re - b.x * im;
                qz += a.z * re - b.y * im;
            }
        }
        e1 += kStgBatch * s1;
        e2 += kStgBatch * s2;
    }
}

// A block updates kStgPos plane positions of one face; its kStgGroups thread groups split the
// modes (the faces hold only ~1e5 cells, so mode parallelism is what fills the GPU) and add their
// partial sums through shared memory.  The cell's flag and profile loads are issued before the
// time coefficients are computed, so both memory round trips overlap.
__global__ void __launch_bounds__(kStgBlock) k_stg(const StgLaunch L) {
    __shared__ float4 cs[kStgMaxModes * 2];
    __shared__ float red[kStgGroups - 1][3][kStgPos];
    int fi = 0;
    for (int k = 1; k < L.nfaces; ++k)
        if ((int)blockIdx.x >= L.f[k].block_begin) fi = k;
    const StgFace &F = L.f[fi];
    const int pl = threadIdx.x % kStgPos, grp = threadIdx.x / kStgPos;
    const int pos = ((int)blockIdx.x - F.block_begin) * kStgPos + pl;
    int i, j;
    float4 ub;
    float sigma = 0.0f;
    bool turb;
    const bool target = stg_target(L, F, pos, i, j, ub, sigma, turb);
    if (F.keep)
        for (int m = threadIdx.x; m < L.n_modes; m += kStgBlock) stg_coeff(L, F, cs, m);
    __syncthreads();
    float qx = 0.0f, qy = 0.0f, qz = 0.0f;
    if (target && turb) stg_partial(F, cs, L.n_modes, i, j, grp, kStgGroups, qx, qy, qz);
    if (grp > 0) {
        red[grp - 1][0][pl] = qx;
        red[grp - 1][1][pl] = qy;
        red[grp - 1][2][pl] = qz;
    }
    __syncthreads();
    if (grp == 0 && target) {
#pragma unroll
        for (int g = 0; g < kStgGroups - 1; ++g) {
            qx += red[g][0][pl];
            qy += red[g][1][pl];
            qz += red[g][2][pl];
        }
        if (turb) {
            ub.x += sigma * qx;
            ub.y += sigma * qy;
            ub.z += sigma * qz;
        }
        F.ueq[pos] = ub;
    }
}

}  // namespace

size_t stg_workspace_bytes(const Geo &g, int n_modes) {
    if (n_modes < 1 || n_modes > kStgMaxModes) return 0;
    const int inflow = inflow_mask(g);
    size_t tables = 0, planes = 0;
    for (int k : kOrder) {
        if (!(inflow & (1 << k))) continue;
        int n1, n2;
        stg_face_dims(g, k, n1, n2);
        tables += al((size_t)n_modes * n1 * sizeof(float2)) + al((size_t)n_modes * n2 * sizeof(float2)) +
                  al((size_t)n_modes * sizeof(StgMode));
        planes += al((size_t)n1 * n2 * sizeof(float4));
    }
    return tables + 2 * planes;
}

const char *stg_check(const lbm_stg_params *p) {
    if (!p) return "stg params is NULL";
    if (p->n_modes < 1 || p->n_modes > kStgMaxModes) return "stg: n_modes must be in 1..1024";
    if (!(p->length > 0.0f) || !std::isfinite(p->length)) return "stg: length must be finite and > 0";
    if (!std::isfinite(p->intensity) || !std::isfinite(p->sigma0)) return "stg: intensity / sigma0 not finite";
    if (p->intensity <= 0.0f && !(p->sigma0 >= 0.0f)) return "stg: sigma0 must be >= 0";
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->gain[a])) return "stg: gains must be finite";
    if (p->stride < 1) return "stg: stride must be >= 1";
    return nullptr;
}

const char *stg_build(StgState &s, const Geo &g, const float *ub, const std::vector<uint8_t> *face_solid,
                      const float *ub_dev, const uint8_t *flags_dev) {
    const int Nm = s.p.n_modes;
    const int inflow = inflow_mask(g);
    if (!inflow) return "stg: the domain has no inflow face among x-, x+, y-, y+, z+";
    if (s.rnd.size() != (size_t)6 * Nm * 6) return "stg: random draws have the wrong size";
    const bool cn = s.p.char_normal != 0, io = s.p.inflow_only != 0;

    // cells of each face: equilibrium (not solid), owned, through the optional inflow filter
    auto for_cells = [&](int k, auto &&fn) {
        int n1, n2;
        stg_face_dims(g, k, n1, n2);
        const int a = k / 2;
        const double sgn = (k & 1) ? -1.0 : 1.0;
        for (int j = 0; j < n2; ++j)
            for (int i = 0; i < n1; ++i) {
                if (face_solid[k][(size_t)i + (size_t)n1 * j]) continue;
                int x, y, z;
                face_pos(g, k, i, j, x, y, z);
                if (owner_face(inflow, g, x, y, z) != k) continue;
                const double U[3] = {ub[3 * z], ub[3 * z + 1], ub[3 * z + 2]};
                const double un = sgn * U[a];
                if (io && !(un > 0.0)) continue;
                fn(U, un);
            }
    };
    s.kept = 0;
    for (int k : kOrder) {
        if (!(inflow & (1 << k))) continue;
        long long cnt = 0;
        double sum[3] = {0.0, 0.0, 0.0};
        for_cells(k, [&](const double *U, double) {
            ++cnt;
            for (int c = 0; c < 3; ++c) sum[c] += U[c];
        });
        if (!cnt) continue;
        double mean[3];
        for (int c = 0; c < 3; ++c) mean[c] = sum[c] / (double)cnt;
        const double mn = (k & 1) ? -mean[k / 2] : mean[k / 2];
        const double Uc = cn ? std::fabs(mn) : std::sqrt(mean[0] * mean[0] + mean[1] * mean[1] + mean[2] * mean[2]);
        if (Uc > 1e-7) s.kept |= 1 << k;
    }
    double uref = 0.0, S[3] = {0.0, 0.0, 0.0};
    long long ntot = 0;
    for (int k : kOrder) {
        if (!(s.kept & (1 << k))) continue;
        for_cells(k, [&](const double *U, double) {
            uref += std::sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
            for (int c = 0; c < 3; ++c) S[c] += U[c];
            ++ntot;
        });
    }
    s.u_ref = ntot ? uref / (double)ntot : 0.0;
    const double Sn = std::sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    s.e_c[0] = 1.0; s.e_c[1] = 0.0; s.e_c[2] = 0.0;
    if (Sn > 0.0)
        for (int c = 0; c < 3; ++c) s.e_c[c] = S[c] / Sn;

    // workspace image: per inflow face E1, E2, modes; then the velocity planes
    size_t off = 0;
    struct Reg { size_t e1, e2, mode, plane[2]; int n1, n2; } reg[6] = {};
    for (int k : kOrder) {
        if (!(inflow & (1 << k))) continue;
        stg_face_dims(g, k, reg[k].n1, reg[k].n2);
        reg[k].e1 = off; off += al((size_t)Nm * reg[k].n1 * sizeof(float2));
        reg[k].e2 = off; off += al((size_t)Nm * reg[k].n2 * sizeof(float2));
        reg[k].mode = off; off += al((size_t)Nm * sizeof(StgMode));
    }
    s.table_bytes = off;
    for (int b = 0; b < 2; ++b)
        for (int k : kOrder) {
            if (!(inflow & (1 << k))) continue;
            reg[k].plane[b] = off; off += al((size_t)reg[k].n1 * reg[k].n2 * sizeof(float4));
        }
    if (off > s.ws_bytes) return "stg: workspace too small";
    s.image.assign(s.table_bytes, 0);

    double kmin = 2.0 * kPi / (10.0 * (double)s.p.length);
    const double kmax = kPi;
    if (kmin >= kmax) kmin = 0.1 * kmax;
    const double lkmin = std::log(kmin), lkmax = std::log(kmax);
    std::vector<double> kv((size_t)Nm * 3), amp(Nm);
    StgLaunch &L = s.L;
    L = StgLaunch{};
    L.nfaces = 0;
    int blocks = 0;
    for (int k : kOrder) {
        if (!(inflow & (1 << k))) continue;
        StgFace &F = L.f[L.nfaces++];
        F.face = k;
        F.n1 = reg[k].n1;
        F.n2 = reg[k].n2;
        F.keep = (s.kept >> k) & 1;
        F.E1 = (const float2 *)(s.ws + reg[k].e1);
        F.E2 = (const float2 *)(s.ws + reg[k].e2);
        F.mode = (const StgMode *)(s.ws + reg[k].mode);
        s.plane[0][L.nfaces - 1] = (float4 *)(s.ws + reg[k].plane[0]);
        s.plane[1][L.nfaces - 1] = (float4 *)(s.ws + reg[k].plane[1]);
        F.ueq = s.plane[0][L.nfaces - 1];
        F.block_begin = blocks;
        blocks += (int)(((long long)F.n1 * F.n2 + kStgPos - 1) / kStgPos);
        if (!F.keep) continue;
        // modes of this face: log-spaced band, isotropic directions, von Karman weights
        double suma2 = 0.0;
        for (int m = 0; m < Nm; ++m) {
            const double *R = &s.rnd[((size_t)k * Nm + m) * 6];
            const double xi = ((double)m + R[0]) / (double)Nm;
            const double km = std::exp(lkmin + xi * (lkmax - lkmin));
            const double mu = 2.0 * R[1] - 1.0, th = 2.0 * kPi * R[2];
            const double st = std::sqrt(std::fmax(0.0, 1.0 - mu * mu));
            kv[3 * m] = km * st * std::cos(th);
            kv[3 * m + 1] = km * st * std::sin(th);
            kv[3 * m + 2] = km * mu;
            const double kl = km * (double)s.p.length;
            const double W = std::pow(km, 4.0) / std::pow(1.0 + kl * kl, 17.0 / 6.0);
            amp[m] = std::sqrt(W);
            suma2 += W;
        }
        const double norm = std::sqrt(0.5 * suma2);
        const int a = k / 2, a1 = a == 0 ? 1 : 0, a2 = a == 2 ? 1 : 2;
        const double xf = (k & 1) ? (double)((a == 0 ? g.nx : (a == 1 ? g.ny : g.nz)) - 1) : 0.0;
        float2 *E1 = (float2 *)(s.image.data() + reg[k].e1);
        float2 *E2 = (float2 *)(s.image.data() + reg[k].e2);
        StgMode *M = (StgMode *)(s.image.data() + reg[k].mode);
        for (int m = 0; m < Nm; ++m) {
            const double *R = &s.rnd[((size_t)k * Nm + m) * 6];
            const double *kk = &kv[3 * m];
            const double omega = s.u_ref * (kk[0] * s.e_c[0] + kk[1] * s.e_c[1] + kk[2] * s.e_c[2]);
            M[m].w = omega / (2.0 * kPi);
            for (int c = 0; c < 3; ++c) {
                double ph = kk[a] * xf / (2.0 * kPi) + R[3 + c];
                ph -= std::floor(ph);
                M[m].ph[c] = (float)ph < 1.0f ? (float)ph : 0.0f;
                M[m].amp[c] = (float)(s.p.gain[c] * amp[m] / norm);
            }
            for (int i = 0; i < reg[k].n1; ++i) {
                const double p = kk[a1] * i;
                E1[(size_t)m * reg[k].n1 + i] = make_float2((float)std::cos(p), (float)std::sin(p));
            }
            for (int j = 0; j < reg[k].n2; ++j) {
                const double p = kk[a2] * j;
                E2[(size_t)m * reg[k].n2 + j] = make_float2((float)std::cos(p), (float)std::sin(p));
            }
        }
    }
    L.nblocks = blocks;
    L.n_modes = Nm;
    L.char_normal = cn ? 1 : 0;
    L.inflow_only = io ? 1 : 0;
    L.intensity = s.p.intensity;
    L.sigma0 = s.p.sigma0;
    L.inflow = inflow;
    L.ub = ub_dev;
    L.flags = flags_dev;
    L.g = g;
    return nullptr;
}

cudaError_t launch_stg(const StgState &s, long long t, int buf, cudaStream_t st) {
    StgLaunch L = s.L;
    L.t = t;
    for (int k = 0; k < L.nfaces; ++k) L.f[k].ueq = s.plane[buf][k];
    if (L.nblocks <= 0) return cudaSuccess;
    k_stg<<<L.nblocks, kStgBlock, 0, st>>>(L);
    return cudaGetLastError();
}

}  // namespace lbm

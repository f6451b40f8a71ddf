// lbm_capi.cu -- the C ABI declared in include/lbm.h: argument checks, workspace layout, launches.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_cell.cuh"
#include "lbm_internal.h"
#include "lbm_stg.h"

using namespace lbm;

// the neighbour step's layer kernel on a second stream of the domain (1), or in order (0)
#ifndef LBM_STEP_AUX
#define LBM_STEP_AUX 1
#endif

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t store_bytes(int store) { return store == LBM_F32 ? 4 : 2; }

// Regions of the caller's workspace, in bytes from its start.
struct Layout {
    size_t f, flags, info, ub, side[6], ftab, part, diag, total;
    long long side_cells[6];
    int ngen;   // face cells with precomputed tables (0: none)
};

bool valid_face(int k) { return k >= LBM_FACE_PERIODIC && k <= LBM_FACE_NOSLIP; }

// Returns nullptr when the arguments are acceptable, else a message.
const char *check_args(int nx, int ny, int nz, const lbm_params *p) {
    if (!p) return "params is NULL";
    if (nx < 1 || ny < 1 || nz < 1) return "lattice dimensions must be >= 1";
    const long long N = (long long)nx * ny * nz;
    // the step kernels index cells with 32-bit integers: a cell index, plus the 256-cell offset of
    // a thread's second cell, plus a neighbour offset (one z-plane and one row) must stay below 2^31
    if (N + 2 * ((long long)nx * ny + nx + 1) + 1024 > INT_MAX)
        return "lattice too large: nx*ny*nz + 2 (nx*ny + nx + 1) + 1024 must stay below 2^31";
    if (!(p->tau > 0.5f) || !std::isfinite(p->tau)) return "tau must be a finite value > 1/2";
    if (!(p->cs_smag >= 0.0f) || !std::isfinite(p->cs_smag)) return "cs_smag must be finite and >= 0";
    if (!(p->rho_b > 0.0f) || !std::isfinite(p->rho_b)) return "rho_b must be finite and > 0";
    if (p->store < LBM_F32 || p->store > LBM_BF16S) return "unknown storage kind";
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(p->force[k])) return "force must be finite";
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(p->coriolis[k])) return "coriolis must be finite";
    const int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        const int lo = p->face[2 * a], hi = p->face[2 * a + 1];
        if (!valid_face(lo) || !valid_face(hi)) return "unknown face kind";
        if ((lo == LBM_FACE_PERIODIC) != (hi == LBM_FACE_PERIODIC))
            return "a periodic face needs a periodic opposite face";
        if (lo != LBM_FACE_PERIODIC && n[a] < 2) return "non-periodic axes need at least 2 cells";
    }
    if (p->watchdog_every < 0) return "watchdog_every must be >= 0";
    if (p->sponge_top < 0 || p->buffer_width < 0) return "relaxation zone widths must be >= 0";
    if (!(p->sponge_sigma >= 0.0f && p->sponge_sigma <= 1.0f)) return "sponge_sigma must be in [0, 1]";
    if (!(p->buffer_sigma >= 0.0f && p->buffer_sigma <= 1.0f)) return "buffer_sigma must be in [0, 1]";
    if (p->flux_balance != 0 && p->flux_balance != 1) return "flux_balance must be 0 or 1";
    return nullptr;
}

Layout make_layout(int nx, int ny, int nz, const lbm_params *p) {
    Layout L{};
    const long long N = (long long)nx * ny * nz;
    const size_t sb = store_bytes(p->store);
    size_t off = 0;
    // populations between two guards of one z-plane + one row + 512 cells: the step kernels issue
    // their population loads before reading the cell flags, so a load for a cell that turns out to
    // be solid or on a face may reach up to that far before the first or past the last plane (its
    // value is discarded)
    const size_t guard = align_up(((size_t)nx * ny + nx + 512) * sb);
    L.f = guard; off = align_up(guard + (size_t)Q * N * sb + guard);
    L.flags = off; off = align_up(off + (size_t)N);
    L.info = off; off = align_up(off + (size_t)N * sizeof(uint32_t));
    L.ub = off; off = align_up(off + (size_t)nz * 3 * sizeof(float));
    const long long fc[3] = {(long long)ny * nz, (long long)nx * nz, (long long)nx * ny};
    for (int k = 0; k < 6; ++k) {
        L.side_cells[k] = 0;
        L.side[k] = 0;
        if (p->face[k] == LBM_FACE_OUTFLOW_ZG) {
            L.side_cells[k] = fc[k / 2];
            L.side[k] = off;
            off = align_up(off + (size_t)Q * fc[k / 2] * sb);
        }
    }
    // face tables of every face cell; their element codes are 32-bit offsets from the population
    // base and their heads hold 30-bit cell indices, so the populations and side buffers must span
    // fewer than 2^32 - 1 storage elements and the lattice fewer than 2^30 cells (else the face
    // blocks resolve every boundary rule at run time)
    Geo g{};
    g.N = N; g.nx = nx; g.ny = ny; g.nz = nz; g.sy = nx; g.sz = (long long)nx * ny;
    for (int k = 0; k < 6; ++k) g.face[k] = p->face[k];
    const long long ngen = face_cell_count(g);
    const bool fits = (off - L.f) / sb < (size_t)0xffffffffu && N <= (long long)kFtCell;
    L.ngen = fits ? (int)ngen : 0;
    L.ftab = off; off = align_up(off + (size_t)L.ngen * kFtWords * sizeof(uint32_t));
    L.part = off; off = align_up(off + (size_t)kRedBlocks * 4 * sizeof(double));
    L.diag = off; off = align_up(off + 4 * sizeof(double));
    L.total = off;
    return L;
}

}  // namespace

struct lbm_domain {
    int nx, ny, nz;
    int device;                  // CUDA device current at creation (the workspace's device)
    long long N;
    lbm_params p;
    cudaStream_t stream;
    char *ws;
    Layout L;
    long long t;                 // steps since init
    std::vector<float> ub_host;  // expanded profile staging
    std::vector<uint8_t> face_solid[6];   // solid mask on each face plane (n1 fastest)
    StgState stg;                // synthetic inflow turbulence (App. F)
    double flux_before, flux_after, flux_shift;   // flux balancing of the current profile
    bool flux_valid;             // the three above describe the current profile
    // pinned host staging of profile uploads (a ring, so that an upload never waits for the GPU);
    // null if pinned host memory was not available (then pageable copies)
    static constexpr int kStage = 4;
    float *ub_pinned = nullptr;
    cudaEvent_t ub_done[kStage];
    int ub_slot;
    StepAux aux;                 // second stream for the neighbour step's layer kernel (null: none)
    char err[512];
    ~lbm_domain() {
        if (ub_pinned) {
            for (int k = 0; k < kStage; ++k) cudaEventDestroy(ub_done[k]);
            cudaFreeHost(ub_pinned);
        }
        if (aux.stream) {
            cudaEventDestroy(aux.fork);
            cudaEventDestroy(aux.join);
            cudaStreamDestroy(aux.stream);
        }
    }
};

namespace {

lbm_status fail(lbm_domain *d, lbm_status st, const char *fmt, ...) {
    if (d) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(d->err, sizeof(d->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

lbm_status cuda_check(lbm_domain *d, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LBM_OK;
    return fail(d, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

StepArgs args_of(const lbm_domain *d) {
    StepArgs a{};
    a.f = d->ws + d->L.f;
    a.flags = (const uint8_t *)(d->ws + d->L.flags);
    a.info = (const uint32_t *)(d->ws + d->L.info);
    a.ub = (const float *)(d->ws + d->L.ub);
    for (int k = 0; k < 6; ++k) a.side[k] = d->L.side_cells[k] ? d->ws + d->L.side[k] : nullptr;
    a.g.N = d->N;
    a.g.nx = d->nx; a.g.ny = d->ny; a.g.nz = d->nz;
    for (int k = 0; k < 6; ++k) a.g.face[k] = d->p.face[k];
    a.g.sy = d->nx;
    a.g.sz = (long long)d->nx * d->ny;
    a.tau = d->p.tau;
    a.c2x18 = 18.0f * d->p.cs_smag * d->p.cs_smag;
    a.rho_b = d->p.rho_b;
    a.fx = d->p.force[0]; a.fy = d->p.force[1]; a.fz = d->p.force[2];
    a.ox = d->p.coriolis[0]; a.oy = d->p.coriolis[1]; a.oz = d->p.coriolis[2];
    a.nface = face_cell_count(a.g);
    const size_t sb = store_bytes(d->p.store);
    for (int i = 0; i < Q; ++i) {
        a.plane[i] = (char *)a.f + (size_t)i * (size_t)d->N * sb;
        a.off[i] = (int)(cx(i) + cy(i) * a.g.sy + cz(i) * a.g.sz);
    }
    a.zwrap = (int)(d->nz * a.g.sz);
    const long long xs = d->nx == 1 ? 1 : 2, ys = d->ny == 1 ? 1 : 2;
    const long long ix = d->nx > 2 ? d->nx - 2 : 0;
    a.zface_begin = xs * d->ny * d->nz + ys * ix * d->nz;
    a.zfast = zfast_mask(a.g);
    // (the lattice blocks take the z layers at the speed of interior cells on the two-cell paths:
    // 16-bit storage, and FP32 lattices of at least kDual32MinCells cells)
    a.zlat = (zlat_of(a.g) && (d->p.store != LBM_F32 || d->N >= kDual32MinCells)) ? 1 : 0;
    a.nface_step = a.zlat ? a.zface_begin : a.nface;
    a.pack16 = (d->p.store != LBM_F32 && d->N % 2 == 0 && d->nx % 2 == 0) ? 1 : 0;
    a.ftab = d->L.ngen ? (const uint32_t *)(d->ws + d->L.ftab) : nullptr;
    a.ngen = d->L.ngen;
    a.sponge_top = d->p.sponge_sigma > 0.0f ? d->p.sponge_top : 0;
    a.sponge_sigma = d->p.sponge_sigma;
    a.buffer_width = d->p.buffer_width;
    a.buffer_sigma = d->p.buffer_sigma;
    a.buffer_faces = 0;
    if (d->p.buffer_width > 0 && d->p.buffer_sigma > 0.0f)
        for (int k = 0; k < 4; ++k)
            if (d->p.face[k] == LBM_FACE_INFLOW_EQ || d->p.face[k] == LBM_FACE_OUTFLOW_ZG) a.buffer_faces |= 1 << k;
    a.flux_balance = d->p.flux_balance;
    set_divisors(a);
    a.flux_shift = d->p.flux_balance ? (float)d->flux_shift : 0.0f;
    if (d->stg.on && d->stg.valid) {
        const StgState &s = d->stg;
        for (int k = 0; k < s.L.nfaces; ++k) {
            a.ueq[s.L.f[k].face] = s.plane[s.cur][k];
            a.ueq_next[s.L.f[k].face] = s.plane[1 - s.cur][k];
        }
        a.ueq_alpha = s.alpha;
    }
    return a;
}

// Rebuild the synthetic-inflow tables for the current profile and upload them.
lbm_status stg_rebuild(lbm_domain *d) {
    const StepArgs a = args_of(d);
    const char *msg = stg_build(d->stg, a.g, d->ub_host.data(), d->face_solid, a.ub, a.flags);
    if (msg) return fail(d, LBM_EINVAL, "%s", msg);
    d->stg.valid = false;
    if (d->stg.table_bytes == 0) return LBM_OK;
    return cuda_check(d, cudaMemcpyAsync(d->stg.ws, d->stg.image.data(), d->stg.table_bytes,
                                         cudaMemcpyHostToDevice, d->stream), "stg table upload");
}

// The step needs the general (forced) kernels: a body force, rotation or relaxation zones.
bool has_force(const lbm_domain *d) {
    for (int k = 0; k < 3; ++k)
        if (d->p.force[k] != 0.0f || d->p.coriolis[k] != 0.0f) return true;
    const StepArgs a = args_of(d);
    return a.sponge_top > 0 || a.buffer_faces != 0;
}

// Flux balancing (Sec. 2.1): net volume inflow of the equilibrium cells of the profile, from the
// host copies of the profile and of the face planes' solid masks, and the uniform inward normal
// shift that cancels it (the least-squares smallest correction: the same on every cell).
void flux_balance_update(lbm_domain *d) {
    d->flux_before = d->flux_after = d->flux_shift = 0.0;
    const int n[3] = {d->nx, d->ny, d->nz};
    double phi = 0.0;
    long long cells = 0;
    for (int k = 0; k < 6; ++k) {
        if (d->p.face[k] != LBM_FACE_INFLOW_EQ) continue;
        const int a = k / 2, hi = k & 1;
        const int n1 = a == 0 ? n[1] : n[0], n2 = a == 2 ? n[1] : n[2];
        const double sgn = hi ? -1.0 : 1.0;
        for (int j = 0; j < n2; ++j)
            for (int i = 0; i < n1; ++i) {
                if (d->face_solid[k][(size_t)i + (size_t)n1 * j]) continue;
                const int p[3] = {a == 0 ? (hi ? n[0] - 1 : 0) : i, a == 1 ? (hi ? n[1] - 1 : 0) : (a == 0 ? i : j),
                                  a == 2 ? (hi ? n[2] - 1 : 0) : j};
                // owned by the first inflow face (x-, x+, y-, y+, z-, z+) holding the cell
                int owner = -1;
                for (int q = 0; q < 6 && owner < 0; ++q)
                    if (d->p.face[q] == LBM_FACE_INFLOW_EQ && p[q / 2] == ((q & 1) ? n[q / 2] - 1 : 0)) owner = q;
                if (owner != k) continue;
                phi += sgn * (double)d->ub_host[3 * p[2] + a];
                ++cells;
            }
    }
    d->flux_before = phi;
    if (!d->p.flux_balance || cells == 0) {
        d->flux_after = phi;
        return;
    }
    d->flux_shift = -phi / (double)cells;
    // what the kernels apply: the profile and the shift in FP32
    const float sh = (float)d->flux_shift;
    double after = 0.0;
    for (int k = 0; k < 6; ++k) {
        if (d->p.face[k] != LBM_FACE_INFLOW_EQ) continue;
        const int a = k / 2, hi = k & 1;
        const int n1 = a == 0 ? n[1] : n[0], n2 = a == 2 ? n[1] : n[2];
        const double sgn = hi ? -1.0 : 1.0;
        for (int j = 0; j < n2; ++j)
            for (int i = 0; i < n1; ++i) {
                if (d->face_solid[k][(size_t)i + (size_t)n1 * j]) continue;
                const int p[3] = {a == 0 ? (hi ? n[0] - 1 : 0) : i, a == 1 ? (hi ? n[1] - 1 : 0) : (a == 0 ? i : j),
                                  a == 2 ? (hi ? n[2] - 1 : 0) : j};
                int owner = -1;
                for (int q = 0; q < 6 && owner < 0; ++q)
                    if (d->p.face[q] == LBM_FACE_INFLOW_EQ && p[q / 2] == ((q & 1) ? n[q / 2] - 1 : 0)) owner = q;
                if (owner != k) continue;
                const float u = d->ub_host[3 * p[2] + a] + (float)(sgn * sh);
                after += sgn * (double)u;
            }
    }
    d->flux_after = after;
}

}  // namespace

namespace lbm {
void profile_level_weights(int L, int nz, int k, int &l0, int &l1, double &w1) {
    if (nz % L == 0) {   // equal-height blocks
        l0 = l1 = k / (nz / L);
        w1 = 0.0;
        return;
    }
    const double pos = (k + 0.5) * L / nz - 0.5;   // in units of level centres
    if (pos <= 0.0) { l0 = l1 = 0; w1 = 0.0; return; }
    if (pos >= L - 1) { l0 = l1 = L - 1; w1 = 0.0; return; }
    l0 = (int)pos;
    l1 = l0 + 1;
    w1 = pos - l0;
}
DomainView domain_view(const lbm_domain *d) {
    return DomainView{args_of(d), d->p.store, (d->t & 1) != 0, d->stream, d->device};
}
lbm_status domain_fail(lbm_domain *d, lbm_status st, const char *msg) { return fail(d, st, "%s", msg); }
void domain_advance(lbm_domain *d, long long n) { d->t += n; }
bool domain_stg_on(const lbm_domain *d) { return d->stg.on; }
}  // namespace lbm

extern "C" {

lbm_status lbm_params_default(lbm_params *p) {
    if (!p) return LBM_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->tau = 0.52f;
    p->cs_smag = 0.16f;
    p->rho_b = 1.0f;
    p->store = LBM_F32;
    const int f[6] = {LBM_FACE_INFLOW_EQ, LBM_FACE_OUTFLOW_ZG, LBM_FACE_PERIODIC,
                      LBM_FACE_PERIODIC, LBM_FACE_NOSLIP, LBM_FACE_FREESLIP};
    for (int k = 0; k < 6; ++k) p->face[k] = f[k];
    return LBM_OK;
}

lbm_status lbm_coriolis_omega(double lat_deg, double dt_si, float *out) {
    if (!out || !std::isfinite(lat_deg) || !std::isfinite(dt_si) || dt_si <= 0.0) return LBM_EINVAL;
    const double kOmega = 7.292115e-5;   // Earth's rotation rate [rad/s] (App. E)
    const double lat = lat_deg * 3.14159265358979323846 / 180.0;
    out[0] = 0.0f;
    out[1] = (float)(kOmega * dt_si * std::cos(lat));
    out[2] = (float)(kOmega * dt_si * std::sin(lat));
    return LBM_OK;
}

lbm_status lbm_lattice_units(double dx_si, double u_ref_si, double ma_lbm, double nu_si, double *out) {
    if (!out || !(dx_si > 0.0) || !(u_ref_si > 0.0) || !(ma_lbm > 0.0) || !(nu_si >= 0.0) || !std::isfinite(dx_si) ||
        !std::isfinite(u_ref_si) || !std::isfinite(ma_lbm) || !std::isfinite(nu_si))
        return LBM_EINVAL;
    const double cs = 1.0 / std::sqrt(3.0);
    const double u_lbm = ma_lbm * cs;
    const double dt = u_lbm * dx_si / u_ref_si;
    const double nu_lbm = nu_si * dt / (dx_si * dx_si);
    out[0] = dt;
    out[1] = u_lbm;
    out[2] = nu_lbm;
    out[3] = 3.0 * nu_lbm + 0.5;
    return LBM_OK;
}

lbm_status lbm_faces_for_direction(float theta, int *face) {
    if (!face || !std::isfinite(theta)) return LBM_EINVAL;
    const double c = std::cos((double)theta), s = std::sin((double)theta), eps = 1e-6;
    face[0] = c > eps ? LBM_FACE_INFLOW_EQ : LBM_FACE_OUTFLOW_ZG;
    face[1] = c < -eps ? LBM_FACE_INFLOW_EQ : LBM_FACE_OUTFLOW_ZG;
    face[2] = s > eps ? LBM_FACE_INFLOW_EQ : LBM_FACE_OUTFLOW_ZG;
    face[3] = s < -eps ? LBM_FACE_INFLOW_EQ : LBM_FACE_OUTFLOW_ZG;
    face[4] = LBM_FACE_NOSLIP;
    face[5] = LBM_FACE_FREESLIP;
    return LBM_OK;
}

size_t lbm_workspace_bytes(int nx, int ny, int nz, const lbm_params *p) {
    if (check_args(nx, ny, nz, p)) return 0;
    return make_layout(nx, ny, nz, p).total;
}

int lbm_direction_table(int *c, float *w) {
    for (int i = 0; i < Q; ++i) {
        if (c) { c[3 * i] = cx(i); c[3 * i + 1] = cy(i); c[3 * i + 2] = cz(i); }
        if (w) w[i] = wgt(i);
    }
    return Q;
}

lbm_status lbm_create_domain(const uint8_t *solid, int nx, int ny, int nz, const lbm_params *p,
                             void *workspace, size_t ws_bytes, void *stream, lbm_domain **out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!solid || !workspace) return LBM_EINVAL;
    if (check_args(nx, ny, nz, p)) return LBM_EINVAL;
    if ((uintptr_t)workspace % kAlign) return LBM_EINVAL;
    const Layout L = make_layout(nx, ny, nz, p);
    if (ws_bytes < L.total) return LBM_ENOMEM;
    lbm_domain *d = new (std::nothrow) lbm_domain();
    if (!d) return LBM_ENOMEM;
    d->nx = nx; d->ny = ny; d->nz = nz;
    d->device = 0;
    if (cudaGetDevice(&d->device) != cudaSuccess) {
        cudaGetLastError();
        delete d;
        return LBM_ECUDA;
    }
    d->N = (long long)nx * ny * nz;
    d->p = *p;
    d->stream = (cudaStream_t)stream;
    d->ws = (char *)workspace;
    d->L = L;
    d->t = 0;
    d->err[0] = 0;
    d->ub_host.assign((size_t)nz * 3, 0.0f);
    d->flux_before = d->flux_after = d->flux_shift = 0.0;
    d->flux_valid = true;
    d->ub_slot = 0;
    d->ub_pinned = nullptr;
    {
        float *pin = nullptr;
        if (cudaHostAlloc((void **)&pin, (size_t)lbm_domain::kStage * nz * 3 * sizeof(float), cudaHostAllocDefault) == cudaSuccess) {
            int k = 0;
            for (; k < lbm_domain::kStage; ++k)
                if (cudaEventCreateWithFlags(&d->ub_done[k], cudaEventDisableTiming) != cudaSuccess) break;
            if (k == lbm_domain::kStage) {
                d->ub_pinned = pin;
            } else {
                for (int j = 0; j < k; ++j) cudaEventDestroy(d->ub_done[j]);
                cudaFreeHost(pin);
            }
        }
        cudaGetLastError();   // a failed pinned allocation only means pageable uploads
    }
    {   // the layer kernel's stream (see StepAux); without it the step runs its kernels in order
        StepAux x;
        if (LBM_STEP_AUX && cudaStreamCreateWithFlags(&x.stream, cudaStreamNonBlocking) == cudaSuccess) {
            if (cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming) == cudaSuccess) {
                d->aux = x;
            } else {
                if (x.fork) cudaEventDestroy(x.fork);
                cudaStreamDestroy(x.stream);
            }
        }
        cudaGetLastError();
    }
    for (int k = 0; k < 6; ++k) {
        // face plane k: (y, z), (x, z) or (x, y), first index fastest
        const int a = k / 2, hi = k & 1;
        const int n1 = a == 0 ? ny : nx, n2 = a == 2 ? ny : nz;
        d->face_solid[k].assign((size_t)n1 * n2, 0);
        for (int j = 0; j < n2; ++j)
            for (int i = 0; i < n1; ++i) {
                const int x = a == 0 ? (hi ? nx - 1 : 0) : i;
                const int y = a == 1 ? (hi ? ny - 1 : 0) : (a == 0 ? i : j);
                const int z = a == 2 ? (hi ? nz - 1 : 0) : j;
                d->face_solid[k][(size_t)i + (size_t)n1 * j] =
                    solid[(size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z)] ? 1 : 0;
            }
    }

    StepArgs a = args_of(d);
    // the population region doubles as staging for the mask (it is initialised right after)
    uint8_t *mask_dev = (uint8_t *)(d->ws + L.f);
    lbm_status st = cuda_check(d, cudaMemcpyAsync(mask_dev, solid, (size_t)d->N, cudaMemcpyHostToDevice,
                                                  d->stream), "mask upload");
    if (st == LBM_OK) st = cuda_check(d, launch_flags(mask_dev, (uint8_t *)(d->ws + L.flags), (uint32_t *)(d->ws + L.info), a.g, d->stream), "flags kernel");
    if (st == LBM_OK) st = cuda_check(d, cudaMemsetAsync(d->ws + L.ub, 0, (size_t)nz * 3 * sizeof(float), d->stream), "profile clear");
    for (int k = 0; k < 6 && st == LBM_OK; ++k)
        if (L.side_cells[k])
            st = cuda_check(d, cudaMemsetAsync(d->ws + L.side[k], 0, (size_t)Q * L.side_cells[k] * store_bytes(p->store), d->stream), "side buffer clear");
    if (st == LBM_OK && L.ngen)
        st = cuda_check(d, launch_face_tables(p->store, a, (uint32_t *)(d->ws + L.ftab), d->stream), "face table kernel");
    if (st == LBM_OK) st = cuda_check(d, launch_init(p->store, a, nullptr, nullptr, d->stream), "init kernel");
    if (st != LBM_OK) {
        delete d;
        return st;
    }
    *out = d;
    return LBM_OK;
}

lbm_status lbm_set_stream(lbm_domain *d, void *stream) {
    if (!d) return LBM_EINVAL;
    d->stream = (cudaStream_t)stream;
    return LBM_OK;
}

lbm_status lbm_set_inflow_profile(lbm_domain *d, const float *speed, int L, float theta) {
    if (!d) return LBM_EINVAL;
    if (!speed || L < 1) return fail(d, LBM_EINVAL, "set_inflow_profile: need L >= 1 speeds");
    if (!std::isfinite(theta)) return fail(d, LBM_EINVAL, "set_inflow_profile: theta not finite");
    for (int l = 0; l < L; ++l)
        if (!std::isfinite(speed[l])) return fail(d, LBM_EINVAL, "set_inflow_profile: speed[%d] not finite", l);
    const int nz = d->nz;
    const double c = std::cos((double)theta), s = std::sin((double)theta);
    for (int k = 0; k < nz; ++k) {
        int l0, l1;
        double w1;
        profile_level_weights(L, nz, k, l0, l1, w1);
        const double v = (1.0 - w1) * (double)speed[l0] + w1 * (double)speed[l1];
        d->ub_host[3 * k] = (float)(v * c);
        d->ub_host[3 * k + 1] = (float)(v * s);
        d->ub_host[3 * k + 2] = 0.0f;
    }
    const size_t ub_bytes = (size_t)nz * 3 * sizeof(float);
    lbm_status st;
    if (d->ub_pinned) {
        const int k = d->ub_slot;
        d->ub_slot = (k + 1) % lbm_domain::kStage;
        float *stage = d->ub_pinned + (size_t)k * nz * 3;
        st = cuda_check(d, cudaEventSynchronize(d->ub_done[k]), "profile staging");   // its last copy ran
        if (st == LBM_OK) {
            std::memcpy(stage, d->ub_host.data(), ub_bytes);
            st = cuda_check(d, cudaMemcpyAsync(d->ws + d->L.ub, stage, ub_bytes, cudaMemcpyHostToDevice, d->stream),
                            "profile upload");
        }
        if (st == LBM_OK) st = cuda_check(d, cudaEventRecord(d->ub_done[k], d->stream), "profile staging");
    } else {
        st = cuda_check(d, cudaMemcpyAsync(d->ws + d->L.ub, d->ub_host.data(), ub_bytes, cudaMemcpyHostToDevice,
                                           d->stream), "profile upload");
    }
    d->flux_valid = false;
    if (d->p.flux_balance) {   // the shift is part of the step; otherwise computed on request
        flux_balance_update(d);
        d->flux_valid = true;
    }
    if (st == LBM_OK && d->stg.on) st = stg_rebuild(d);
    return st;
}

lbm_status lbm_init_fields(lbm_domain *d, const float *rho, const float *u) {
    if (!d) return LBM_EINVAL;
    d->stg.valid = false;   // equilibrium cells start from u_b
    const StepArgs a = args_of(d);
    lbm_status st = cuda_check(d, launch_init(d->p.store, a, rho, u, d->stream), "init kernel");
    if (st == LBM_OK) d->t = 0;
    return st;
}

lbm_status lbm_import_populations(lbm_domain *d, const float *g, long long step) {
    if (!d) return LBM_EINVAL;
    if (!g) return fail(d, LBM_EINVAL, "import: NULL pointer");
    if (step < 0 || (step & 1)) return fail(d, LBM_EINVAL, "import: step must be even and >= 0");
    d->stg.valid = false;   // synthetic inflow anchors are re-evaluated at the next step
    const StepArgs a = args_of(d);
    lbm_status st = cuda_check(d, launch_import(d->p.store, a, g, d->stream), "import kernel");
    if (st == LBM_OK) d->t = step;
    return st;
}

lbm_status lbm_diagnostics(lbm_domain *d, double *out) {
    if (!d || !out) return LBM_EINVAL;
    const StepArgs a = args_of(d);
    double *part = (double *)(d->ws + d->L.part);
    double *res = (double *)(d->ws + d->L.diag);
    lbm_status st = cuda_check(d, launch_reduce(d->p.store, a, (d->t & 1) != 0, part, res, d->stream), "reduce kernels");
    if (st != LBM_OK) return st;
    st = cuda_check(d, cudaMemcpyAsync(out, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, d->stream), "diagnostics copy");
    if (st != LBM_OK) return st;
    return cuda_check(d, cudaStreamSynchronize(d->stream), "diagnostics sync");
}

lbm_status lbm_step(lbm_domain *d, int n) {
    if (!d) return LBM_EINVAL;
    if (n < 0) return fail(d, LBM_EINVAL, "step: n must be >= 0");
    const bool force = has_force(d);
    for (int k = 0; k < n; ++k) {
        if (d->stg.on) {
            // U of the inflow faces, evaluated only at anchors t_a = floor(t/s) s: held, or (stride
            // > 1 with interpolation) kept for t_a and t_a + s and blended by the step itself
            StgState &s = d->stg;
            const long long t = d->t, sp = s.p.stride, ta = (t / sp) * sp;
            const bool interp = s.p.interpolate && sp > 1;
            if (!s.valid || s.anchor != ta) {
                cudaError_t e;
                if (interp && s.valid && s.anchor == ta - sp) {
                    s.cur ^= 1;                             // U(t_a) was the previous "next"
                    e = launch_stg(s, ta + sp, 1 - s.cur, d->stream);
                } else {
                    e = launch_stg(s, ta, s.cur, d->stream);
                    if (e == cudaSuccess && interp) e = launch_stg(s, ta + sp, 1 - s.cur, d->stream);
                }
                lbm_status st = cuda_check(d, e, "stg kernel launch");
                if (st != LBM_OK) return st;
                s.anchor = ta;
                s.valid = true;
            }
            s.alpha = interp ? (float)(t - ta) / (float)sp : 0.0f;
        }
        const StepArgs a = args_of(d);
        launch_step(d->p.store, (d->t & 1) == 0, force, a, d->stream, &d->aux);
        d->t += 1;
        if (d->p.watchdog_every > 0 && d->t % d->p.watchdog_every == 0) {
            double diag[4];
            lbm_status st = lbm_diagnostics(d, diag);
            if (st != LBM_OK) return st;
            if (diag[3] > 0.0)
                return fail(d, LBM_EUNSTABLE, "watchdog: %.0f fluid cells with non-finite populations at step %lld",
                            diag[3], d->t);
        }
    }
    return cuda_check(d, cudaGetLastError(), "step kernel launch");
}

long long lbm_steps_done(const lbm_domain *d) { return d ? d->t : -1; }

lbm_status lbm_flux_balance_info(const lbm_domain *d_, double *before, double *after, double *shift) {
    if (!d_) return LBM_EINVAL;
    lbm_domain *d = const_cast<lbm_domain *>(d_);   // lazily computed host-side bookkeeping
    if (!d->flux_valid) {
        flux_balance_update(d);
        d->flux_valid = true;
    }
    if (before) *before = d->flux_before;
    if (after) *after = d->flux_after;
    if (shift) *shift = d->p.flux_balance ? d->flux_shift : 0.0;
    return LBM_OK;
}

lbm_status lbm_sample_columns(lbm_domain *d, const int *ij, int ncol, const int *k, int nh, float *out) {
    if (!d) return LBM_EINVAL;
    if (ncol < 0 || nh < 0) return fail(d, LBM_EINVAL, "sample: negative counts");
    if ((long long)ncol * nh == 0) return LBM_OK;
    if (!ij || !k || !out) return fail(d, LBM_EINVAL, "sample: NULL pointer");
    const StepArgs a = args_of(d);
    return cuda_check(d, launch_sample(d->p.store, a, (d->t & 1) != 0, ij, ncol, k, nh, out, d->stream), "sample kernel");
}

lbm_status lbm_macroscopic(lbm_domain *d, float *rho, float *u) {
    if (!d) return LBM_EINVAL;
    if (!rho && !u) return LBM_OK;
    const StepArgs a = args_of(d);
    return cuda_check(d, launch_macros(d->p.store, a, (d->t & 1) != 0, rho, u, d->stream), "macroscopic kernel");
}

lbm_status lbm_export_populations(lbm_domain *d, float *g) {
    if (!d) return LBM_EINVAL;
    if (!g) return fail(d, LBM_EINVAL, "export: NULL pointer");
    const StepArgs a = args_of(d);
    return cuda_check(d, launch_export(d->p.store, a, (d->t & 1) != 0, g, d->stream), "export kernel");
}

lbm_status lbm_stg_params_default(lbm_stg_params *p) {
    if (!p) return LBM_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->n_modes = 64;
    p->length = 20.0f;
    p->intensity = 0.1f;
    p->sigma0 = 0.0f;
    p->gain[0] = p->gain[1] = p->gain[2] = 1.0f;
    p->stride = 1;
    p->interpolate = 1;
    return LBM_OK;
}

size_t lbm_stg_workspace_bytes(const lbm_domain *d, int n_modes) {
    if (!d) return 0;
    return stg_workspace_bytes(args_of(d).g, n_modes);
}

lbm_status lbm_stg_configure(lbm_domain *d, const lbm_stg_params *p, const double *uniforms,
                             void *workspace, size_t ws_bytes) {
    if (!d) return LBM_EINVAL;
    if (const char *msg = stg_check(p)) return fail(d, LBM_EINVAL, "%s", msg);
    if (!uniforms || !workspace) return fail(d, LBM_EINVAL, "stg: NULL uniforms or workspace");
    if ((uintptr_t)workspace % kAlign) return fail(d, LBM_EINVAL, "stg: workspace not 256-byte aligned");
    const size_t need = stg_workspace_bytes(args_of(d).g, p->n_modes);
    if (need == 0) return fail(d, LBM_EINVAL, "stg: the domain has no inflow face among x-, x+, y-, y+, z+");
    if (ws_bytes < need) return fail(d, LBM_ENOMEM, "stg: workspace has %zu bytes, needs %zu", ws_bytes, need);
    const size_t nr = (size_t)6 * p->n_modes * 6;
    for (size_t i = 0; i < nr; ++i)
        if (!(uniforms[i] >= 0.0 && uniforms[i] < 1.0)) return fail(d, LBM_EINVAL, "stg: uniforms[%zu] outside [0, 1)", i);
    StgState &s = d->stg;
    s.on = false;
    s.p = *p;
    s.rnd.assign(uniforms, uniforms + nr);
    s.ws = (char *)workspace;
    s.ws_bytes = ws_bytes;
    lbm_status st = stg_rebuild(d);
    if (st != LBM_OK) return st;
    s.on = true;
    s.valid = false;
    return LBM_OK;
}

lbm_status lbm_stg_disable(lbm_domain *d) {
    if (!d) return LBM_EINVAL;
    d->stg.on = false;
    d->stg.valid = false;
    return LBM_OK;
}

lbm_status lbm_stg_reference(const lbm_domain *d, double *u_ref, double *e_c, int *faces) {
    if (!d || !d->stg.on) return LBM_EINVAL;
    if (u_ref) *u_ref = d->stg.u_ref;
    if (e_c) for (int c = 0; c < 3; ++c) e_c[c] = d->stg.e_c[c];
    if (faces) *faces = d->stg.kept;
    return LBM_OK;
}

const char *lbm_last_error(const lbm_domain *d) { return d ? d->err : "no domain"; }

void lbm_destroy(lbm_domain *d) { delete d; }

}  // extern "C"

/*
 * lbm_oracle.c -- FP64 CPU oracle for one time step of the urban-wind LBM-LES solver.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct definition that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it; the product library never links, calls or falls back to it.  It
 * shares no code, header, table or constant with the CUDA sources.
 *
 * What it computes (paper App. D, equations numbered in order of appearance D.1 ... D.11):
 *   - D3Q19 lattice, c_s^2 = 1/3, weights fixed by 2nd/4th-order isotropy (App. D, text before D.1)
 *   - moments rho = sum f_i, rho u = sum c_i f_i                                   (D.1)
 *   - second-order Hermite equilibrium f_i^eq(rho, u)                              (D.4)
 *   - non-equilibrium flux Pi^(1) = sum c c (f - f^eq), Q = sqrt(2 Pi:Pi)          (D.8, D.10)
 *   - tau_eff = 1/2 [tau + sqrt(tau^2 + 2 (C Delta)^2 Q / (rho c_s^4))], Delta = 1  (D.11)
 *   - SRT-BGK collision f* = f - (f - f^eq)/tau_eff                                (D.2)
 *   - streaming f_i(x + c_i, t + 1) = f*_i(x, t)                                   (D.3)
 *   - halfway (mid-grid) bounce-back at solid cells and no-slip faces  (App. D, last paragraph)
 *   - equilibrium velocity boundary cells (Sec. 3, boundary-condition paragraph)
 *   - optional uniform body force and Coriolis force F_c = rho 2 Omega x u (App. E), both applied
 *     by Guo's forcing scheme
 *   - synthetic von Karman inflow turbulence on the equilibrium boundary cells (App. F), by direct
 *     summation of the Fourier modes (oracle_stg)
 *
 * The step is written as a two-lattice PULL: Fout(x) is computed from Fin (the post-collision
 * state of the previous step) by gathering each population from its upstream neighbour and then
 * colliding.  Observed state = post-collision populations F*.
 *
 * Readings where the paper is silent (each one is listed in the design notes of the repository):
 *   - lattice units, Delta t = Delta x = Delta = 1, so nu_0 = (tau - 1/2)/3;
 *   - Pi^(1) is taken from the pre-collision (post-stream) populations against f^eq of the same
 *     populations; Q sums all nine tensor components;
 *   - equilibrium boundary cells hold f^eq(rho_b, u_b(z)) and never gather;
 *   - outflow faces are zero-gradient: a population entering from outside the face is the
 *     same-direction population leaving the adjacent in-domain cell one step earlier;
 *   - free-slip faces reflect specularly (the normal velocity component is mirrored);
 *   - periodic faces wrap;
 *   - edges and corners: a source position outside the domain is resolved axis by axis
 *     (wrap / clamp / clamp + mirror); if any out-of-range axis is a no-slip face, or if the
 *     resolved source cell is solid, the population is bounced back from the cell itself.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORQ 19

/* face kinds, oracle-private numbering */
enum { OR_PERIODIC = 0, OR_INFLOW = 1, OR_OUTFLOW = 2, OR_FREESLIP = 3, OR_NOSLIP = 4 };
/* cell kinds */
enum { OR_FLUID = 0, OR_SOLID = 1, OR_EQ = 2 };

static int oc[ORQ][3];     /* lattice velocities */
static double ow[ORQ];     /* weights */
static int oopp[ORQ];      /* opposite direction */
static int omir[3][ORQ];   /* direction with component a negated */
static int otab_ready = 0;

/* D3Q19 = every c in {-1,0,1}^3 with |c|^2 <= 2; weight from |c|^2 alone (1/3, 1/18, 1/36).
 * These are the only weights that give sum w = 1, sum w c_a c_b = delta/3 and the 4th-order
 * isotropic tensor c_s^4 (dd + dd + dd) on this velocity set; the tests check exactly that. */
static void tables(void)
{
    if (otab_ready) return;
    int n = 0;
    for (int c2 = 0; c2 <= 2; ++c2)
        for (int z = -1; z <= 1; ++z)
            for (int y = -1; y <= 1; ++y)
                for (int x = -1; x <= 1; ++x)
                    if (x * x + y * y + z * z == c2) {
                        oc[n][0] = x; oc[n][1] = y; oc[n][2] = z;
                        ow[n] = (c2 == 0) ? 1.0 / 3.0 : (c2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
                        ++n;
                    }
    for (int i = 0; i < ORQ; ++i)
        for (int j = 0; j < ORQ; ++j) {
            if (oc[j][0] == -oc[i][0] && oc[j][1] == -oc[i][1] && oc[j][2] == -oc[i][2]) oopp[i] = j;
            for (int a = 0; a < 3; ++a) {
                int ok = 1;
                for (int b = 0; b < 3; ++b) ok &= (oc[j][b] == (b == a ? -oc[i][b] : oc[i][b]));
                if (ok) omir[a][i] = j;
            }
        }
    otab_ready = 1;
}

/* ---- exported lattice description (so the tests can pin it) ---- */
int oracle_lattice(int *c /* 19*3 */, double *w /* 19 */, int *opp /* 19 */)
{
    tables();
    for (int i = 0; i < ORQ; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = oc[i][a];
        w[i] = ow[i];
        opp[i] = oopp[i];
    }
    return ORQ;
}

/* ---- D.4: second-order Hermite equilibrium ---- */
void oracle_equilibrium(double rho, const double u[3], double feq[ORQ])
{
    tables();
    const double cs2 = 1.0 / 3.0;
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < ORQ; ++i) {
        const double cu = oc[i][0] * u[0] + oc[i][1] * u[1] + oc[i][2] * u[2];
        feq[i] = ow[i] * rho * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
    }
}

/* ---- D.11: closed-form effective relaxation time ---- */
double oracle_tau_eff(double tau, double C, double Q, double rho)
{
    const double cs2 = 1.0 / 3.0, Delta = 1.0;
    return 0.5 * (tau + sqrt(tau * tau + 2.0 * (C * Delta) * (C * Delta) * Q / (rho * cs2 * cs2)));
}

/* ---- one cell: moments, equilibrium, LES closure, BGK (+ Guo source) ----
 * f:     pre-collision populations (post-stream)
 * force: uniform body-force density (may be NULL)
 * omega: rotation vector Omega^lbm of the Coriolis force (may be NULL); App. E: once rho and u
 *        are recovered from the populations, F_c = rho 2 Omega^lbm x u joins the body force
 *        that Guo's scheme applies (u here = sum c f / rho, before any force correction)
 * out:   post-collision populations; q_out / tau_out optional diagnostics */
void oracle_collide_rot(const double f[ORQ], double tau, double C, const double *force,
                        const double *omega, double out[ORQ], double *q_out, double *tau_out)
{
    tables();
    const double cs2 = 1.0 / 3.0;
    double F[3] = {0.0, 0.0, 0.0};
    if (force) { F[0] = force[0]; F[1] = force[1]; F[2] = force[2]; }

    /* D.1 */
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < ORQ; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) m[a] += oc[i][a] * f[i];
    }
    if (omega) { /* App. E: F_c = rho 2 Omega x u with u = m / rho */
        const double v[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
        F[0] += rho * 2.0 * (omega[1] * v[2] - omega[2] * v[1]);
        F[1] += rho * 2.0 * (omega[2] * v[0] - omega[0] * v[2]);
        F[2] += rho * 2.0 * (omega[0] * v[1] - omega[1] * v[0]);
    }
    /* Guo: the velocity carries half the force impulse */
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * F[a]) / rho;

    double feq[ORQ];
    oracle_equilibrium(rho, u, feq);

    /* D.8: full 3x3 non-equilibrium momentum flux */
    double Pi[3][3] = {{0}};
    for (int i = 0; i < ORQ; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Pi[a][b] += oc[i][a] * oc[i][b] * (f[i] - feq[i]);
    /* D.10 */
    double PP = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) PP += Pi[a][b] * Pi[a][b];
    const double Q = sqrt(2.0 * PP);
    /* D.11 */
    const double te = oracle_tau_eff(tau, C, Q, rho);

    /* D.2 with Guo's source term S_i = (1 - 1/(2 tau)) w_i [(c - u)/c_s^2 + (c.u) c / c_s^4] . F */
    for (int i = 0; i < ORQ; ++i) {
        double cu = 0.0, cF = 0.0, uF = 0.0;
        for (int a = 0; a < 3; ++a) {
            cu += oc[i][a] * u[a];
            cF += oc[i][a] * F[a];
            uF += u[a] * F[a];
        }
        const double S = (1.0 - 0.5 / te) * ow[i] * ((cF - uF) / cs2 + cu * cF / (cs2 * cs2));
        out[i] = f[i] - (f[i] - feq[i]) / te + S;
    }
    if (q_out) *q_out = Q;
    if (tau_out) *tau_out = te;
}

void oracle_collide(const double f[ORQ], double tau, double C, const double *force, double out[ORQ],
                    double *q_out, double *tau_out)
{
    oracle_collide_rot(f, tau, C, force, NULL, out, q_out, tau_out);
}

/* ---- cell classification: solid mask wins, then equilibrium-face layers, else fluid ---- */
int oracle_classify(const uint8_t *solid, int nx, int ny, int nz, const int face[6], uint8_t *kind)
{
    const int n[3] = {nx, ny, nz};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t c = ((size_t)z * ny + y) * nx + x;
                const int p[3] = {x, y, z};
                uint8_t k = OR_FLUID;
                for (int a = 0; a < 3; ++a) {
                    if (p[a] == 0 && face[2 * a] == OR_INFLOW) k = OR_EQ;
                    if (p[a] == n[a] - 1 && face[2 * a + 1] == OR_INFLOW) k = OR_EQ;
                }
                if (solid[c]) k = OR_SOLID;
                kind[c] = k;
            }
    return 0;
}

/* ---- inflow profile: L level speeds -> per-cell-height velocity u_b[k][3] ----
 * L divides nz: equal-height blocks.  Otherwise: linear in height between level centres
 * (cell k sits at height k + 1/2 above the ground wall, level l is centred at (l + 1/2) nz / L),
 * held constant beyond the first and last centre.  Direction theta: 0 = +x, counter-clockwise. */
int oracle_expand_profile(const double *speed, int L, int nz, double theta, double *ub)
{
    if (L <= 0 || nz <= 0) return -1;
    for (int k = 0; k < nz; ++k) {
        double s;
        if (nz % L == 0) {
            s = speed[k / (nz / L)];
        } else {
            const double h = k + 0.5;
            const double pos = h * L / nz - 0.5; /* level-centre coordinate */
            if (pos <= 0.0) s = speed[0];
            else if (pos >= L - 1) s = speed[L - 1];
            else {
                const int l = (int)floor(pos);
                const double t = pos - l;
                s = (1.0 - t) * speed[l] + t * speed[l + 1];
            }
        }
        ub[3 * k + 0] = s * cos(theta);
        ub[3 * k + 1] = s * sin(theta);
        ub[3 * k + 2] = 0.0;
    }
    return 0;
}

/* ---- initial state: F = f^eq(rho, u) per cell ----
 * rho, u may be NULL (rho = 1, u = u_b(z)).  Equilibrium cells take f^eq(rho_b, u_b(z)); solid 0. */
int oracle_init(double *F, const uint8_t *kind, int nx, int ny, int nz, const double *rho,
                const double *u, const double *ub, double rho_b, const double *ueq)
{
    tables();
    const size_t N = (size_t)nx * ny * nz;
    for (size_t c = 0; c < N; ++c) {
        const int z = (int)(c / ((size_t)nx * ny));
        double feq[ORQ];
        if (kind[c] == OR_SOLID) {
            for (int i = 0; i < ORQ; ++i) F[i * N + c] = 0.0;
            continue;
        }
        if (kind[c] == OR_EQ) {
            oracle_equilibrium(rho_b, ueq ? ueq + 3 * c : ub + 3 * z, feq);
        } else {
            double uc[3];
            for (int a = 0; a < 3; ++a) uc[a] = u ? u[3 * c + a] : ub[3 * z + a];
            oracle_equilibrium(rho ? rho[c] : 1.0, uc, feq);
        }
        for (int i = 0; i < ORQ; ++i) F[i * N + c] = feq[i];
    }
    return 0;
}

/* ---- gather rule for the incoming population i of a fluid cell p (D.3 + boundary rules) ----
 * returns F*_d(s) from the previous post-collision state, or the bounced-back F*_opp(i)(p). */
static double gather(const double *Fin, const uint8_t *kind, const int n[3], size_t N,
                     const int face[6], const int p[3], int i)
{
    int s[3];
    int d = i;
    for (int a = 0; a < 3; ++a) s[a] = p[a] - oc[i][a];
    const size_t self = ((size_t)p[2] * n[1] + p[1]) * n[0] + p[0];

    /* a no-slip face on any out-of-range axis: halfway bounce-back from the cell itself */
    for (int a = 0; a < 3; ++a) {
        if (s[a] < 0 && face[2 * a] == OR_NOSLIP) return Fin[(size_t)oopp[i] * N + self];
        if (s[a] >= n[a] && face[2 * a + 1] == OR_NOSLIP) return Fin[(size_t)oopp[i] * N + self];
    }
    /* resolve the remaining out-of-range axes one at a time */
    for (int a = 0; a < 3; ++a) {
        if (s[a] >= 0 && s[a] < n[a]) continue;
        const int hi = s[a] >= n[a];
        const int kindf = face[2 * a + hi];
        if (kindf == OR_PERIODIC) {
            s[a] = hi ? s[a] - n[a] : s[a] + n[a];
        } else if (kindf == OR_FREESLIP) {
            s[a] = hi ? n[a] - 1 : 0;
            d = omir[a][d];
        } else { /* outflow (zero-gradient) and, unreachably for fluid cells, equilibrium faces */
            s[a] = hi ? n[a] - 1 : 0;
        }
    }
    const size_t src = ((size_t)s[2] * n[1] + s[1]) * n[0] + s[0];
    if (kind[src] == OR_SOLID) return Fin[(size_t)oopp[i] * N + self];
    return Fin[(size_t)d * N + src];
}

/* ---- one full time step over z-planes [z0, z1) (pass 0, nz for the whole lattice) ----
 * Fin:  post-collision state at step t (19 x N, population-major, x fastest)
 * Fout: post-collision state at step t+1
 * q_out, tau_out: optional per-cell Q and tau_eff of the step (fluid cells; NaN elsewhere)
 * omega: optional Coriolis rotation vector (lattice units)
 * ueq:   optional per-cell velocity of the equilibrium boundary cells (N x 3); NULL = u_b(z) */
int oracle_step(const double *Fin, double *Fout, const uint8_t *kind, int nx, int ny, int nz,
                const int face[6], const double *ub, double rho_b, double tau, double C,
                const double *force, int z0, int z1, double *q_out, double *tau_out,
                const double *omega, const double *ueq)
{
    tables();
    const int n[3] = {nx, ny, nz};
    const size_t N = (size_t)nx * ny * nz;
    if (z0 < 0) z0 = 0;
    if (z1 > nz) z1 = nz;
#pragma omp parallel for schedule(static)
    for (int z = z0; z < z1; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t c = ((size_t)z * ny + y) * nx + x;
                double f[ORQ], out[ORQ];
                double q = NAN, te = NAN;
                if (kind[c] == OR_SOLID) {
                    for (int i = 0; i < ORQ; ++i) out[i] = 0.0;
                } else if (kind[c] == OR_EQ) {
                    oracle_equilibrium(rho_b, ueq ? ueq + 3 * c : ub + 3 * z, out);
                } else {
                    const int p[3] = {x, y, z};
                    for (int i = 0; i < ORQ; ++i) f[i] = gather(Fin, kind, n, N, face, p, i);
                    oracle_collide_rot(f, tau, C, force, omega, out, &q, &te);
                }
                for (int i = 0; i < ORQ; ++i) Fout[(size_t)i * N + c] = out[i];
                if (q_out) q_out[c] = q;
                if (tau_out) tau_out[c] = te;
            }
    return 0;
}

/* ---- observed macroscopic fields of a post-collision state ----
 * fluid: rho = sum F*, u = (sum c F* - F/2) / rho (Guo: sum c F* = rho u + F/2 after collision)
 * equilibrium cells: (rho_b, u_b(z)); solid: rho = 0, u = 0. */
int oracle_macros(const double *F, const uint8_t *kind, int nx, int ny, int nz, const double *ub,
                  double rho_b, const double *force, double *rho, double *u, const double *ueq)
{
    tables();
    const size_t N = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (long long cc = 0; cc < (long long)N; ++cc) {
        const size_t c = (size_t)cc;
        const int z = (int)(c / ((size_t)nx * ny));
        if (kind[c] == OR_SOLID) {
            rho[c] = 0.0;
            u[3 * c] = u[3 * c + 1] = u[3 * c + 2] = 0.0;
            continue;
        }
        if (kind[c] == OR_EQ) {
            rho[c] = rho_b;
            for (int a = 0; a < 3; ++a) u[3 * c + a] = ueq ? ueq[3 * c + a] : ub[3 * z + a];
            continue;
        }
        double r = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < ORQ; ++i) {
            const double v = F[(size_t)i * N + c];
            r += v;
            for (int a = 0; a < 3; ++a) m[a] += oc[i][a] * v;
        }
        rho[c] = r;
        for (int a = 0; a < 3; ++a) u[3 * c + a] = (m[a] - 0.5 * (force ? force[a] : 0.0)) / r;
    }
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ======================================================================================
 * Synthetic von Karman inflow turbulence (paper App. F), evaluated by direct summation.
 *
 * Velocity of every equilibrium boundary cell at time step t:
 *   cell set Gamma_VK: equilibrium cells on the west, east, south, north and top faces (never the
 *   ground), each assigned to the first of those faces that contains it; optionally only cells
 *   with U_b . n_f > 0 (n_f the inward normal).  A face whose characteristic speed U_c,f (|mean
 *   U_b| or |mean U_b . n_f|) is <= 1e-7 is dropped.
 *   u_ref = mean |U_b| and e_c = sum U_b / |sum U_b| over the kept cells ((1,0,0) if the sum is 0).
 *   per face and mode m (m = 1..N_m): xi = (m - 1 + r)/N_m, k = exp(ln kmin + xi (ln kmax - ln kmin)),
 *     kmin = 2 pi/(10 L), kmax = pi (kmin -> 0.1 kmax if kmin >= kmax); k_vec = k (sqrt(1-mu^2) cos th,
 *     sqrt(1-mu^2) sin th, mu); W = k^4 / (1 + (k L)^2)^(17/6); A = sqrt(W) / sqrt(1/2 sum sqrt(W)^2);
 *     A_a = g_a A; omega = u_ref k_vec . e_c
 *   q_a(x, t) = sum_m A_a cos(k_vec . x + omega t + phi_a)   (x = integer cell indices)
 *   sigma = I u_char (I > 0) or sigma0; u_char = |U_b| or |U_b . n_f|
 *   temporal stride s: anchors t_a = floor(t/s) s; hold q(t_a) or interpolate linearly to t_a + s
 *   U = U_b + sigma q
 * Random inputs (readings: App. F states the distributions of r, mu, theta; phases uniform in
 * [0, 2 pi)): rnd[f][m][6] = uniforms in [0,1) giving r, (mu+1)/2, theta/(2 pi), phi_x/(2 pi),
 * phi_y/(2 pi), phi_z/(2 pi); f = face index 0..5 in the order x- x+ y- y+ z- z+ (z- unused).
 * Output ueq (N x 3): the velocity of every equilibrium cell (U_b where no turbulence applies).
 * ====================================================================================== */
typedef struct {
    int n_modes;
    double L;           /* integral length scale (lattice units) */
    double I;           /* turbulence intensity; <= 0 selects sigma0 */
    double sigma0;
    double gain[3];
    int char_normal;    /* 1: characteristic speeds use the face-normal component */
    int inflow_only;    /* 1: only cells with U_b . n_f > 0 */
    int stride;         /* >= 1 */
    int interpolate;    /* 1: linear between anchors, 0: hold */
} oracle_stg_params;

static const int stg_faces[5] = {0, 1, 2, 3, 5};   /* west, east, south, north, top */

static void face_normal_in(int f, double n[3])
{
    n[0] = n[1] = n[2] = 0.0;
    n[f / 2] = (f % 2 == 0) ? 1.0 : -1.0;
}

/* the STG face a cell belongs to (-1 if none) */
static int stg_face_of(int x, int y, int z, int nx, int ny, int nz, const int face[6])
{
    const int p[3] = {x, y, z}, n[3] = {nx, ny, nz};
    for (int k = 0; k < 5; ++k) {
        const int f = stg_faces[k], a = f / 2;
        if (face[f] != OR_INFLOW) continue;
        if ((f % 2 == 0 && p[a] == 0) || (f % 2 == 1 && p[a] == n[a] - 1)) return f;
    }
    return -1;
}

static void stg_q(const double *tab, int nm, const double x[3], double t, double q[3])
{
    /* tab per mode: kx ky kz omega Ax Ay Az phix phiy phiz */
    q[0] = q[1] = q[2] = 0.0;
    for (int m = 0; m < nm; ++m) {
        const double *T = tab + 10 * m;
        const double base = T[0] * x[0] + T[1] * x[1] + T[2] * x[2] + T[3] * t;
        for (int a = 0; a < 3; ++a) q[a] += T[4 + a] * cos(base + T[7 + a]);
    }
}

int oracle_stg(const uint8_t *kind, int nx, int ny, int nz, const int face[6], const double *ub,
               const oracle_stg_params *P, const double *rnd, long long t, double *ueq)
{
    const size_t N = (size_t)nx * ny * nz;
    const int nm = P->n_modes;
    if (nm < 1 || P->L <= 0.0 || P->stride < 1) return -1;
    /* 1. cell sets, face means, global u_ref and e_c */
    double sumU[6][3] = {{0}};
    long long cnt[6] = {0};
    for (size_t c = 0; c < N; ++c) {
        if (kind[c] != OR_EQ) continue;
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((size_t)nx * ny));
        const int f = stg_face_of(x, y, z, nx, ny, nz, face);
        if (f < 0) continue;
        double n[3];
        face_normal_in(f, n);
        const double *U = ub + 3 * z;
        if (P->inflow_only && U[0] * n[0] + U[1] * n[1] + U[2] * n[2] <= 0.0) continue;
        for (int a = 0; a < 3; ++a) sumU[f][a] += U[a];
        cnt[f]++;
    }
    int keep[6] = {0};
    for (int f = 0; f < 6; ++f) {
        if (!cnt[f]) continue;
        double mean[3], n[3];
        face_normal_in(f, n);
        for (int a = 0; a < 3; ++a) mean[a] = sumU[f][a] / cnt[f];
        const double Uc = P->char_normal ? fabs(mean[0] * n[0] + mean[1] * n[1] + mean[2] * n[2])
                                         : sqrt(mean[0] * mean[0] + mean[1] * mean[1] + mean[2] * mean[2]);
        keep[f] = Uc > 1e-7;
    }
    double uref = 0.0, S[3] = {0.0, 0.0, 0.0};
    long long ntot = 0;
    for (size_t c = 0; c < N; ++c) {
        if (kind[c] != OR_EQ) continue;
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((size_t)nx * ny));
        const int f = stg_face_of(x, y, z, nx, ny, nz, face);
        if (f < 0 || !keep[f]) continue;
        double n[3];
        face_normal_in(f, n);
        const double *U = ub + 3 * z;
        if (P->inflow_only && U[0] * n[0] + U[1] * n[1] + U[2] * n[2] <= 0.0) continue;
        uref += sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
        for (int a = 0; a < 3; ++a) S[a] += U[a];
        ntot++;
    }
    if (ntot) uref /= (double)ntot;
    double ec[3] = {1.0, 0.0, 0.0};
    const double Sn = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    if (Sn > 0.0) for (int a = 0; a < 3; ++a) ec[a] = S[a] / Sn;
    /* 2. mode tables */
    const double pi = 3.14159265358979323846;
    double kmin = 2.0 * pi / (10.0 * P->L), kmax = pi;
    if (kmin >= kmax) kmin = 0.1 * kmax;
    double *tab = (double *)calloc((size_t)6 * nm * 10, sizeof(double));
    if (!tab) return -2;
    for (int f = 0; f < 6; ++f) {
        if (!keep[f]) continue;
        double *T = tab + (size_t)f * nm * 10;
        double suma2 = 0.0;
        for (int m = 0; m < nm; ++m) {
            const double *R = rnd + ((size_t)f * nm + m) * 6;
            const double xi = (m + R[0]) / nm;
            const double k = exp(log(kmin) + xi * (log(kmax) - log(kmin)));
            const double mu = 2.0 * R[1] - 1.0, th = 2.0 * pi * R[2];
            const double s = sqrt(1.0 - mu * mu);
            T[10 * m + 0] = k * s * cos(th);
            T[10 * m + 1] = k * s * sin(th);
            T[10 * m + 2] = k * mu;
            T[10 * m + 3] = uref * (T[10 * m] * ec[0] + T[10 * m + 1] * ec[1] + T[10 * m + 2] * ec[2]);
            const double W = pow(k, 4) / pow(1.0 + (k * P->L) * (k * P->L), 17.0 / 6.0);
            T[10 * m + 4] = sqrt(W); /* raw amplitude, normalised below */
            suma2 += W;
            for (int a = 0; a < 3; ++a) T[10 * m + 7 + a] = 2.0 * pi * R[3 + a];
        }
        const double norm = sqrt(0.5 * suma2);
        for (int m = 0; m < nm; ++m) {
            const double A = T[10 * m + 4] / norm;
            for (int a = 0; a < 3; ++a) T[10 * m + 4 + a] = P->gain[a] * A;
        }
    }
    /* 3. boundary velocities */
    const long long ta = (t / P->stride) * P->stride;
    const double alpha = (double)(t - ta) / P->stride;
    for (size_t c = 0; c < N; ++c) {
        if (kind[c] != OR_EQ) { ueq[3 * c] = ueq[3 * c + 1] = ueq[3 * c + 2] = 0.0; continue; }
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((size_t)nx * ny));
        const double *U = ub + 3 * z;
        for (int a = 0; a < 3; ++a) ueq[3 * c + a] = U[a];
        const int f = stg_face_of(x, y, z, nx, ny, nz, face);
        if (f < 0 || !keep[f]) continue;
        double n[3];
        face_normal_in(f, n);
        const double Un = U[0] * n[0] + U[1] * n[1] + U[2] * n[2];
        if (P->inflow_only && Un <= 0.0) continue;
        const double uchar = P->char_normal ? fabs(Un) : sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
        const double sigma = P->I > 0.0 ? P->I * uchar : P->sigma0;
        const double X[3] = {(double)x, (double)y, (double)z};
        double q[3], q2[3];
        stg_q(tab + (size_t)f * nm * 10, nm, X, (double)ta, q);
        if (P->interpolate && alpha > 0.0) {
            stg_q(tab + (size_t)f * nm * 10, nm, X, (double)(ta + P->stride), q2);
            for (int a = 0; a < 3; ++a) q[a] = (1.0 - alpha) * q[a] + alpha * q2[a];
        }
        for (int a = 0; a < 3; ++a) ueq[3 * c + a] = U[a] + sigma * q[a];
    }
    free(tab);
    return 0;
}

// Host-side check of the neighbour step's face tables (cell_face_table) against the general
// boundary resolution they are built from (scatter_targets, the rules of App. D and Sec. 3 for
// every face kind).  For every face cell of small lattices with solids and every combination of
// inflow, outflow, periodic, no-slip and free-slip faces, and every direction j:
//   - a cell that is not an equilibrium cell keeps the resolver's targets, in its order;
//   - an equilibrium cell keeps the resolver's targets except those in equilibrium cells (such a
//     cell never reads what it receives: its local step writes its equilibrium over it, and every
//     read-back computes that equilibrium), and every dropped target is one;
//   - the plain bit is set exactly when the one kept target is the plain downstream slot.
// Compiled for the host only (the cell bodies are __host__ __device__); prints one line per lattice
// and exits non-zero on the first mismatch.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "lbm_cell.cuh"

using namespace lbm;

struct Visit {
    int kind;
    long long idx;
};

static long long dropped_total = 0;

static int check(int nx, int ny, int nz, const int face[6], unsigned seed) {
    using T = float;
    Geo G{};
    G.N = (long long)nx * ny * nz;
    G.nx = nx; G.ny = ny; G.nz = nz;
    for (int k = 0; k < 6; ++k) G.face[k] = face[k];
    G.sy = nx; G.sz = (long long)nx * ny;
    const long long N = G.N;
    std::vector<uint8_t> mask(N), flags(N);
    std::vector<uint32_t> info(N);
    srand(seed);
    for (long long n = 0; n < N; ++n) mask[n] = (rand() % 8) == 0;
    for (long long n = 0; n < N; ++n) cell_flags(mask.data(), flags.data(), info.data(), G, n);
    // populations and the six side buffers in one allocation (the tables code side-buffer
    // elements relative to the populations)
    const long long fc[3] = {(long long)ny * nz, (long long)nx * nz, (long long)nx * ny};
    std::vector<T> buf((size_t)(Q * N + 6 * Q * (fc[0] + fc[1] + fc[2])));
    StepArgs a{};
    a.g = G;
    a.flags = flags.data();
    a.info = info.data();
    a.f = buf.data();
    for (int i = 0; i < Q; ++i) {
        a.off[i] = (int)(cx(i) + cy(i) * G.sy + cz(i) * G.sz);
        a.plane[i] = (T *)a.f + (long long)i * N;
    }
    long long sbase[6];
    long long at = Q * N;
    for (int k = 0; k < 6; ++k) {
        sbase[k] = at;
        a.side[k] = (G.face[k] == LBM_FACE_OUTFLOW_ZG) ? (void *)(buf.data() + at) : nullptr;
        at += Q * fc[k / 2];
        if (!a.side[k]) sbase[k] = 0;
    }
    const long long ng = face_cell_count(G);
    a.ngen = (int)ng;
    std::vector<uint32_t> tab((size_t)((3 + 3 * Q) * ng));
    for (long long t = 0; t < ng; ++t) cell_face_table<LBM_F32>(a, (int)t, tab.data());
    long long cells = 0, dropped = 0;
    for (long long t = 0; t < ng; ++t) {
        int x, y, z;
        face_cell_xyz(G, t, x, y, z);
        const long long n = cell_of(G, x, y, z);
        const uint8_t fl = flags[n];
        if (fl & F_SOLID) {
            if (tab[t] != kFtNone) { printf("solid face cell %lld has a table\n", n); return 1; }
            continue;
        }
        if (tab[t] & kFtGeneral) continue;   // more than two targets somewhere: the general path
        ++cells;
        const bool eq = fl & F_EQ;
        const uint32_t plain = tab[(1 + 3 * Q) * ng + t], second = tab[(2 + 3 * Q) * ng + t];
        for (int j = 0; j < Q; ++j) {
            std::vector<Visit> all;
            scatter_targets(G, flags.data(), x, y, z, j, !eq, [&](int kind, long long idx) { all.push_back({kind, idx}); });
            std::vector<uint32_t> keep;
            for (const Visit &v : all) {
                const bool into_eq = v.kind == 0 && (flags[v.idx % N] & F_EQ);
                if (eq && into_eq) { ++dropped; continue; }
                keep.push_back((uint32_t)(v.kind == 0 ? v.idx : sbase[v.kind - 1] + v.idx));
            }
            const uint32_t w0 = tab[(1 + Q + j) * ng + t], w1 = tab[(1 + 2 * Q + j) * ng + t];
            const uint32_t k0 = keep.size() > 0 ? keep[0] : kFtNone, k1 = keep.size() > 1 ? keep[1] : kFtNone;
            if (w0 != k0 || w1 != k1 || (((second >> j) & 1u) != 0) != (keep.size() >= 2)) {
                printf("cell %lld (%d,%d,%d)%s j=%d: table %u %u (second %u), resolver keeps %zu: %u %u\n", n, x, y, z,
                       eq ? " eq" : "", j, w0, w1, (second >> j) & 1u, keep.size(), k0, k1);
                return 1;
            }
            const bool want_plain = keep.size() == 1 && k0 == (uint32_t)((long long)j * N + n + a.off[j]);
            if ((((plain >> j) & 1u) != 0) != want_plain) {
                printf("cell %lld j=%d: plain bit %u, expected %d\n", n, j, (plain >> j) & 1u, (int)want_plain);
                return 1;
            }
        }
    }
    dropped_total += dropped;
    printf("%dx%dx%d faces %d%d%d%d%d%d seed %u: %lld face cells, %lld dropped stores into equilibrium cells, "
           "tables match the resolution\n", nx, ny, nz, face[0], face[1], face[2], face[3], face[4], face[5], seed,
           cells, dropped);
    return 0;
}

int main() {
    const int P = LBM_FACE_PERIODIC, I = LBM_FACE_INFLOW_EQ, O = LBM_FACE_OUTFLOW_ZG, F = LBM_FACE_FREESLIP,
              W = LBM_FACE_NOSLIP;
    const int sets[][6] = {
        {I, O, I, O, W, F},   // the city's kind: inflow on two lateral faces, outflow on the others
        {O, I, O, I, W, F},
        {I, O, P, P, W, F},
        {I, I, O, O, F, W},   // inflow on both x faces: their edges meet other inflow cells
        {I, O, I, O, I, O},   // inflow and outflow on every axis
        {P, P, I, O, W, W},
        {O, O, I, I, W, I},
    };
    const int dims[][3] = {{9, 7, 6}, {12, 10, 5}, {6, 11, 8}};
    unsigned seed = 1;
    for (const auto &d : dims)
        for (const auto &f : sets)
            if (check(d[0], d[1], d[2], f, seed++)) return 1;
    if (dropped_total == 0) { printf("no store into an equilibrium cell was dropped\n"); return 1; }
    printf("all face-table checks passed\n");
    return 0;
}

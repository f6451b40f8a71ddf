// Host-side check of the neighbour step's ground / top layer path in the lattice blocks: for every
// F_ZL cell of small lattices with solids in and next to both layers, the storage elements its
// gathers read and its scatters write -- by the per-cell form (cell2_neighbor_zl) and by the static
// per-block rules (zk_gather_base / zk_scatter_base, where the kernel applies them) -- must equal
// those of the general boundary resolution (gather_loc_B / scatter_targets, the rules the face
// tables are built from), for no-slip and free-slip ground and top.  Also checks that cells of those lattices that
// are not F_ZL are either interior cells (plain pulls) or face cells the face blocks still visit.
// Compiled for the host only (the cell bodies are __host__ __device__); prints one line per lattice
// and exits non-zero on the first mismatch.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "lbm_cell.cuh"

using namespace lbm;

// collects the targets scatter_targets visits
struct Targets {
    long long t[4];
    int kinds[4];
    int cnt = 0;
    LBM_HD void operator()(int kind, long long idx) {
        if (cnt < 4) { kinds[cnt] = kind; t[cnt] = idx; }
        ++cnt;
    }
};

static int check(int nx, int ny, int nz, int zlo, int zhi, unsigned seed) {
    Geo G{};
    G.N = (long long)nx * ny * nz;
    G.nx = nx; G.ny = ny; G.nz = nz;
    const int lat[4] = {LBM_FACE_PERIODIC, LBM_FACE_PERIODIC, LBM_FACE_INFLOW_EQ, LBM_FACE_OUTFLOW_ZG};
    G.face[0] = lat[seed % 4]; G.face[1] = lat[(seed / 4) % 4];
    if ((G.face[0] == LBM_FACE_PERIODIC) != (G.face[1] == LBM_FACE_PERIODIC)) G.face[1] = G.face[0];
    G.face[2] = LBM_FACE_PERIODIC; G.face[3] = LBM_FACE_PERIODIC;
    G.face[4] = zlo; G.face[5] = zhi;
    G.sy = nx; G.sz = (long long)nx * ny;
    std::vector<uint8_t> mask(G.N), flags(G.N);
    std::vector<uint32_t> info(G.N);
    srand(seed);
    const int sparse = (seed % 2) ? 7 : 40;   // solids everywhere, both layers included (dense or sparse)
    for (long long n = 0; n < G.N; ++n) mask[n] = (rand() % sparse) == 0;
    for (long long n = 0; n < G.N; ++n) cell_flags(mask.data(), flags.data(), info.data(), G, n);
    StepArgs a{};
    a.g = G;
    a.flags = flags.data();
    a.info = info.data();
    std::vector<float> pop((size_t)(Q + 2) * G.N);   // 19 planes, with a plane of room on either side
    a.f = pop.data() + G.N;
    for (int i = 0; i < Q; ++i) {
        a.off[i] = (int)(cx(i) + cy(i) * G.sy + cz(i) * G.sz);
        a.plane[i] = (float *)a.f + (long long)i * G.N;
    }
    a.zlat = zlat_of(G) ? 1 : 0;
    int nzl = 0, nstatic = 0;
    for (long long n = 0; n < G.N; ++n) {
        const uint8_t fl = flags[n];
        if (!(fl & F_ZL)) continue;
        ++nzl;
        int x, y, z;
        cell_coords(G, n, x, y, z);
        const int zl = z == 0 ? 1 : 2;
        if (!a.zlat || (z != 0 && z != nz - 1) || x == 0 || y == 0 || x == nx - 1 || y == ny - 1 || (fl & (F_SOLID | F_EQ))) {
            printf("F_ZL on a cell that is not an interior-xy layer cell: n=%lld\n", n);
            return 1;
        }
        const unsigned nb = (fl & F_REDIR) ? info[n] >> 8 : 0u;
        for (int i = 0; i < Q; ++i) {
            // the resolution the face tables take (store-side bounce-back for solid neighbours)
            const Loc l = ((nb >> opp(i)) & 1u) ? Loc{0, (long long)opp(i) * G.N + n - a.off[i]}
                                                 : gather_loc_B(G, flags.data(), x, y, z, i);
            long long e = zl_gather_elem(a, n, zl, i);
            const int cross = zl == 1 ? 1 : -1;
            if (G.face[zl == 1 ? 4 : 5] == LBM_FACE_FREESLIP && cz(i) == cross && !(cx(i) == 0 && cy(i) == 0) &&
                ((nb >> dir_c(-cx(i), -cy(i), 0)) & 1u))
                e = (long long)i * G.N + n;   // the kernel's fix-up for a solid mirrored source
            if (l.kind != 0 || l.idx != e) {
                printf("gather mismatch n=%lld (%d,%d,%d) i=%d: resolver kind %d elem %lld, layer path %lld\n", n, x, y, z,
                       i, l.kind, l.idx, e);
                return 1;
            }
        }
        // the static per-block rules (a block wholly in this layer), as the kernel applies them:
        // free-slip layer cells with solid neighbours take the checked general form above
        const int zk = zl == 1 ? (zlo == LBM_FACE_NOSLIP ? ZK_GROUND_NOSLIP : ZK_GROUND_FREESLIP)
                               : (zhi == LBM_FACE_NOSLIP ? ZK_TOP_NOSLIP : ZK_TOP_FREESLIP);
        const bool static_ok = zk_noslip(zk) || !(fl & F_REDIR);
        if (static_ok) {
            for (int i = 0; i < Q; ++i) {
                long long e = 0;
                switch (zk) {
                    case ZK_GROUND_NOSLIP: e = zk_gather_base<float, ZK_GROUND_NOSLIP>(a, i) + n - (float *)a.f; break;
                    case ZK_GROUND_FREESLIP: e = zk_gather_base<float, ZK_GROUND_FREESLIP>(a, i) + n - (float *)a.f; break;
                    case ZK_TOP_NOSLIP: e = zk_gather_base<float, ZK_TOP_NOSLIP>(a, i) + n - (float *)a.f; break;
                    default: e = zk_gather_base<float, ZK_TOP_FREESLIP>(a, i) + n - (float *)a.f; break;
                }
                if (e != zl_gather_elem(a, n, zl, i)) {
                    printf("static gather mismatch n=%lld (%d,%d,%d) i=%d kind %d: %lld vs %lld\n", n, x, y, z, i, zk, e,
                           zl_gather_elem(a, n, zl, i));
                    return 1;
                }
            }
            for (int j = 0; j < Q; ++j) {
                long long e = 0;
                if (!zk_cross_out(zk, j) && ((nb >> j) & 1u)) {
                    e = (long long)opp(j) * G.N + n;
                } else {
                    switch (zk) {
                        case ZK_GROUND_NOSLIP: e = zk_scatter_base<float, ZK_GROUND_NOSLIP>(a, j) + n - (float *)a.f; break;
                        case ZK_GROUND_FREESLIP: e = zk_scatter_base<float, ZK_GROUND_FREESLIP>(a, j) + n - (float *)a.f; break;
                        case ZK_TOP_NOSLIP: e = zk_scatter_base<float, ZK_TOP_NOSLIP>(a, j) + n - (float *)a.f; break;
                        default: e = zk_scatter_base<float, ZK_TOP_FREESLIP>(a, j) + n - (float *)a.f; break;
                    }
                }
                if (e != zl_scatter_elem(a, n, zl, nb, j)) {
                    printf("static scatter mismatch n=%lld (%d,%d,%d) j=%d kind %d: %lld vs %lld\n", n, x, y, z, j, zk, e,
                           zl_scatter_elem(a, n, zl, nb, j));
                    return 1;
                }
            }
            ++nstatic;
        }
        for (int j = 0; j < Q; ++j) {
            Targets tg;
            scatter_targets(G, flags.data(), x, y, z, j, true, tg);
            const long long e = zl_scatter_elem(a, n, zl, nb, j);
            if (tg.cnt != 1 || tg.kinds[0] != 0 || tg.t[0] != e) {
                printf("scatter mismatch n=%lld (%d,%d,%d) j=%d: resolver %d target(s), first kind %d elem %lld, layer path %lld\n",
                       n, x, y, z, j, tg.cnt, tg.cnt ? tg.kinds[0] : -1, tg.cnt ? tg.t[0] : -1, e);
                return 1;
            }
        }
    }
    // every interior-xy layer cell that is not solid carries F_ZL when zlat holds
    if (a.zlat)
        for (long long n = 0; n < G.N; ++n) {
            int x, y, z;
            cell_coords(G, n, x, y, z);
            const bool layer = (z == 0 || z == nz - 1) && x > 0 && y > 0 && x < nx - 1 && y < ny - 1;
            if (layer && !(flags[n] & F_SOLID) && !(flags[n] & F_ZL)) {
                printf("layer cell without F_ZL: n=%lld\n", n);
                return 1;
            }
        }
    printf("%dx%dx%d z faces %d/%d lateral x %d/%d seed %u: %d layer cells (%d on the static rules) match the general resolution\n",
           nx, ny, nz, zlo, zhi, G.face[0], G.face[1], seed, nzl, nstatic);
    return 0;
}

int main() {
    const int kinds[2] = {LBM_FACE_NOSLIP, LBM_FACE_FREESLIP};
    const int dims[][3] = {{9, 7, 6}, {5, 4, 2}, {12, 3, 3}, {6, 6, 9}};
    unsigned seed = 1;
    for (const auto &d : dims)
        for (int lo = 0; lo < 2; ++lo)
            for (int hi = 0; hi < 2; ++hi)
                for (int r = 0; r < 4; ++r, ++seed)
                    if (check(d[0], d[1], d[2], kinds[lo], kinds[hi], seed)) return 1;
    printf("all layer-path checks passed\n");
    return 0;
}

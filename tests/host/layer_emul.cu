// Host emulation of the neighbour step's ground / top lattice blocks (the layer path of zlat): for
// lattices of uneven sizes with solids in both layers and every no-slip / free-slip combination of
// the z faces, every block that reaches into a layer runs the layer-path body of each of its
// threads (neighbor_layer_unit, 16-bit and FP32 storage, block sizes 128, 256 and 512 as the single
// and the batched launches use them) on a population buffer laid out as the device workspace
// (a guard of one z-plane, one row and 512 cells on either side of the 19 planes).  Built with
// AddressSanitizer by the test that runs it: any access outside the buffer aborts; writes into the
// guards are detected by canaries.  Prints one line per lattice, exits non-zero on a failure.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "lbm_cell.cuh"

using namespace lbm;

template <int S, int B>
static int run(int nx, int ny, int nz, const int face[6], unsigned seed) {
    using T = typename Codec<S>::T;
    Geo G{};
    G.N = (long long)nx * ny * nz;
    G.nx = nx; G.ny = ny; G.nz = nz;
    for (int k = 0; k < 6; ++k) G.face[k] = face[k];
    G.sy = nx; G.sz = (long long)nx * ny;
    const long long N = G.N;
    std::vector<uint8_t> mask(N), flags(N);
    std::vector<uint32_t> info(N);
    srand(seed);
    for (long long n = 0; n < N; ++n) mask[n] = (rand() % 9) == 0;
    for (long long n = 0; n < N; ++n) cell_flags(mask.data(), flags.data(), info.data(), G, n);
    const long long guard = (long long)nx * ny + nx + 512;
    std::vector<T> buf((size_t)(2 * guard + Q * N));
    T canary;
    memset(&canary, 0x5a, sizeof(T));
    for (auto &v : buf) v = canary;
    for (long long e = guard; e < guard + Q * N; ++e) buf[e] = Codec<S>::enc(0.001f * (float)((e * 7919) % 101 - 50) / 50.0f);
    StepArgs a{};
    a.g = G;
    a.f = buf.data() + guard;
    a.flags = flags.data();
    a.info = info.data();
    for (int i = 0; i < Q; ++i) {
        a.plane[i] = (T *)a.f + (long long)i * N;
        a.off[i] = (int)(cx(i) + cy(i) * G.sy + cz(i) * G.sz);
    }
    a.tau = 0.52f; a.c2x18 = 18.0f * 0.16f * 0.16f; a.rho_b = 1.0f;
    a.zlat = zlat_of(G) ? 1 : 0;
    if (!a.zlat) return 0;
    constexpr long long span = 2 * B;
    const unsigned nlb = (unsigned)((N + span - 1) / span);
    int blocks = 0;
    for (unsigned lb = 0; lb < nlb; ++lb) {
        const int zk = block_layer_kind(a, lb, span);
        if (zk == ZK_INTERIOR) continue;
        ++blocks;
        for (unsigned t = 0; t < (unsigned)B; ++t) neighbor_layer_unit<S, false, false, B>(a, lb, zk, t);
    }
    for (long long e = 0; e < guard; ++e)
        if (memcmp(&buf[e], &canary, sizeof(T)) || memcmp(&buf[guard + Q * N + e], &canary, sizeof(T))) {
            printf("write into a guard: element %lld\n", e);
            return 1;
        }
    printf("%dx%dx%d z %d/%d S=%d B=%d: %d layer blocks in bounds\n", nx, ny, nz, face[4], face[5], S, B, blocks);
    return 0;
}

int main() {
    const int dims[][3] = {{33, 26, 8}, {24, 20, 6}, {13, 7, 6}, {9, 7, 2}, {40, 30, 3}};
    const int lat[][4] = {{LBM_FACE_OUTFLOW_ZG, LBM_FACE_INFLOW_EQ, LBM_FACE_INFLOW_EQ, LBM_FACE_OUTFLOW_ZG},
                          {LBM_FACE_PERIODIC, LBM_FACE_PERIODIC, LBM_FACE_PERIODIC, LBM_FACE_PERIODIC}};
    const int zk[2] = {LBM_FACE_NOSLIP, LBM_FACE_FREESLIP};
    unsigned seed = 3;
    for (const auto &d : dims)
        for (const auto &l : lat)
            for (int lo = 0; lo < 2; ++lo)
                for (int hi = 0; hi < 2; ++hi, ++seed) {
                    const int face[6] = {l[0], l[1], l[2], l[3], zk[lo], zk[hi]};
                    if (run<LBM_F16S, 128>(d[0], d[1], d[2], face, seed) || run<LBM_F16S, 256>(d[0], d[1], d[2], face, seed) ||
                        run<LBM_F16S, 512>(d[0], d[1], d[2], face, seed) || run<LBM_F32, 256>(d[0], d[1], d[2], face, seed) ||
                        run<LBM_BF16S, 256>(d[0], d[1], d[2], face, seed))
                        return 1;
                }
    printf("all layer-block emulations in bounds\n");
    return 0;
}

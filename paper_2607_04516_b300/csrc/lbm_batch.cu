// lbm_batch.cu -- ensembles and uneven domains advanced together: one kernel launch per time step
// covers every cell of every member domain, optionally replayed from a CUDA graph, with the launch
// shape chosen by measurement (lbm_batch_autotune).
//
// The grid of a batched launch is the concatenation of the members' own grids (face blocks, then
// lattice blocks, exactly as a single-domain launch lays them out), in a slot order the autotuner
// may change.  A block finds its slot by binary search over the slots' first blocks, reads that
// member's step arguments (from the kernel's parameter space for up to 48 members, else from a copy
// in shared memory) and runs the same block body as the single-domain kernels (local_block /
// neighbor_block).  Members keep their own workspaces and
// state; the batch only adds a small table of step arguments and block offsets.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "lbm.h"
#include "lbm_cell.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace {

// Launch shapes the autotuner chooses from (lbm_batch_autotune): threads per block B, resident blocks
// per SM the batched kernel is compiled for (its register cap), cells per thread of FP32 members
// (0: each member's own choice, as in its single-domain launch; 1 or 2 for all -- the unrolling of
// the cell loop), a persistent grid (one set of resident blocks striding over the members' blocks),
// the slot order (members in the given order or largest first), or one single-domain launch per
// member and step.
struct ShapeSpec {
    int B, minb, cpt;
    bool persistent, largest_first, sequential;
};
constexpr ShapeSpec kShapeSpec[] = {
    {256, 4, 0, false, false, false},   // 0
    {256, 3, 0, false, false, false},   // 1
    {256, 4, 0, false, true, false},    // 2
    {256, 3, 0, false, true, false},    // 3
    {256, 4, 0, false, false, true},    // 4: one single-domain launch per member and step
    {128, 8, 0, false, false, false},   // 5
    {512, 2, 0, false, false, false},   // 6
    {256, 4, 1, false, false, false},   // 7: FP32 members one cell per thread
    {256, 4, 2, false, false, false},   // 8: FP32 members two cells per thread
    {256, 4, 0, true, false, false},    // 9: persistent grid
};
constexpr int kNumShapes = (int)(sizeof(kShapeSpec) / sizeof(kShapeSpec[0]));
constexpr int kSequential = 4;
constexpr int kTableShapes = 4;   // shapes 0..3 also run with the member tables in device memory

struct BatchTables {
    const StepArgs *args;     // per member
    const unsigned *start;    // per slot: first block of the slot in the grid (+ total at [n])
    const int *member;        // per slot: member index
    int n;
};

// FP32 member: two cells per thread?
template <int S, int CPT> __device__ __forceinline__ bool batch_d32(const StepArgs &a) {
    return S == LBM_F32 && (CPT == 2 || (CPT == 0 && a.g.N >= kDual32MinCells));
}

// Block bid of a member's own launch of this step kind (the same block bodies as lbm_step).
template <int S, bool NEIGHBOR, int B, int CPT>
__device__ __forceinline__ void batch_block(const StepArgs &a, unsigned bid) {
    const bool d32 = batch_d32<S, CPT>(a);
    if constexpr (NEIGHBOR) {
        if (d32) neighbor_block<S, false, false, true, B>(a, bid, face_blocks_of<B>(a.nface));
        else neighbor_block<S, false, false, false, B>(a, bid, face_blocks_of<B>(a.nface));
    } else if constexpr (S == LBM_F32) {
        if (d32) local_block<S, false, false, true, B>(a, bid);
        else local_block<S, false, false, false, B>(a, bid);
    } else {
        if (a.pack16) local_block<S, false, true, false, B>(a, bid);
        else local_block<S, false, false, false, B>(a, bid);
    }
}

template <int S, bool NEIGHBOR, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_batch_step(BatchTables t) {
    __shared__ StepArgs sa;
    __shared__ unsigned s_bid;
    __shared__ int s_member;
    if (threadIdx.x == 0) {
        int lo = 0, hi = t.n - 1;   // last slot whose first block is <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (t.start[mid] <= blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_member = t.member[lo];
        s_bid = blockIdx.x - t.start[lo];
    }
    __syncthreads();
    {
        const int *src = (const int *)(t.args + s_member);
        int *dst = (int *)&sa;
        for (int k = threadIdx.x; k < (int)(sizeof(StepArgs) / sizeof(int)); k += kBlock) dst[k] = src[k];
    }
    __syncthreads();
    batch_block<S, NEIGHBOR, kBlock, 0>(sa, s_bid);
}

// Up to kParamMembers members: the step arguments and block tables travel in the kernel's parameter
// space (__grid_constant__, constant bank) instead of shared memory, as in the single-domain kernels.
constexpr int kParamMembers = 48;
struct BatchParams {
    StepArgs args[kParamMembers];
    unsigned start[kParamMembers + 1];
    int member[kParamMembers];
    int n;
};
static_assert(sizeof(BatchParams) <= 32000, "kernel parameter space");

template <int S, bool NEIGHBOR, int B, int MINB, int CPT, bool PERSIST>
__global__ void __launch_bounds__(B, MINB) k_batch_step_p(const __grid_constant__ BatchParams p) {
    const unsigned total = p.start[p.n];
    for (unsigned vb = blockIdx.x; vb < total; vb += PERSIST ? gridDim.x : total) {
        int lo = 0, hi = p.n - 1;   // last slot whose first block is <= vb (uniform)
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.start[mid] <= vb) lo = mid;
            else hi = mid - 1;
        }
        batch_block<S, NEIGHBOR, B, CPT>(p.args[p.member[lo]], vb - p.start[lo]);
    }
}

// blocks of a member's launch of this kind in shape sh (as its single-domain launch for shape 0)
template <int S> unsigned member_blocks(const StepArgs &a, bool neighbor, int sh) {
    const ShapeSpec &q = kShapeSpec[sh];
    const bool d32 = S == LBM_F32 && (q.cpt == 2 || (q.cpt == 0 && a.g.N >= kDual32MinCells));
    unsigned lb = 0, fb = 0;
    switch (q.B) {
        case 128: lb = d32 ? lattice_blocks<S, true, 128>(a.g.N) : lattice_blocks<S, false, 128>(a.g.N);
                  fb = face_blocks_of<128>(a.nface); break;
        case 512: lb = d32 ? lattice_blocks<S, true, 512>(a.g.N) : lattice_blocks<S, false, 512>(a.g.N);
                  fb = face_blocks_of<512>(a.nface); break;
        default: lb = d32 ? lattice_blocks<S, true, 256>(a.g.N) : lattice_blocks<S, false, 256>(a.g.N);
                 fb = face_blocks_of<256>(a.nface); break;
    }
    return lb + (neighbor ? fb : 0u);
}
unsigned member_blocks(int store, const StepArgs &a, bool neighbor, int sh) {
    switch (store) {
        case LBM_F32: return member_blocks<LBM_F32>(a, neighbor, sh);
        case LBM_F16S: return member_blocks<LBM_F16S>(a, neighbor, sh);
        default: return member_blocks<LBM_BF16S>(a, neighbor, sh);
    }
}

// Resident blocks of a persistent kernel: its occupancy times the SM count (queried once).
template <class K> unsigned persistent_grid(K kernel, int B) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, B, 0) != cudaSuccess || per < 1) {
        cudaGetLastError();
        return 0;
    }
    return (unsigned)(sms * per);
}

template <int S, bool NEIGHBOR, int B, int MINB, int CPT, bool PERSIST>
void launch_p(const BatchParams &p, unsigned blocks, cudaStream_t s) {
    if (PERSIST) {
        static unsigned grid = 0;   // per kernel (one template instance per kernel)
        if (!grid) grid = persistent_grid(k_batch_step_p<S, NEIGHBOR, B, MINB, CPT, PERSIST>, B);
        if (grid && grid < blocks) blocks = grid;
    }
    k_batch_step_p<S, NEIGHBOR, B, MINB, CPT, PERSIST><<<blocks, B, 0, s>>>(p);
}
template <int S, bool NEIGHBOR>
void launch_shape(int sh, const BatchTables &t, const BatchParams *p, unsigned blocks, cudaStream_t s) {
    if (!p) {   // member tables in device memory (more than kParamMembers members): shapes 0..3
        if (kShapeSpec[sh].minb == 3) k_batch_step<S, NEIGHBOR, 3><<<blocks, kBlock, 0, s>>>(t);
        else k_batch_step<S, NEIGHBOR, 4><<<blocks, kBlock, 0, s>>>(t);
        return;
    }
    switch (sh) {
        case 1: case 3: launch_p<S, NEIGHBOR, 256, 3, 0, false>(*p, blocks, s); break;
        case 5: launch_p<S, NEIGHBOR, 128, 8, 0, false>(*p, blocks, s); break;
        case 6: launch_p<S, NEIGHBOR, 512, 2, 0, false>(*p, blocks, s); break;
        case 7: if constexpr (S == LBM_F32) launch_p<S, NEIGHBOR, 256, 4, 1, false>(*p, blocks, s);
                else launch_p<S, NEIGHBOR, 256, 4, 0, false>(*p, blocks, s);
                break;
        case 8: if constexpr (S == LBM_F32) launch_p<S, NEIGHBOR, 256, 4, 2, false>(*p, blocks, s);
                else launch_p<S, NEIGHBOR, 256, 4, 0, false>(*p, blocks, s);
                break;
        case 9: launch_p<S, NEIGHBOR, 256, 4, 0, true>(*p, blocks, s); break;
        default: launch_p<S, NEIGHBOR, 256, 4, 0, false>(*p, blocks, s); break;
    }
}
void launch_batch(int store, int sh, bool neighbor, const BatchTables &t, const BatchParams *p, unsigned blocks,
                  cudaStream_t s) {
    switch (store) {
        case LBM_F32:
            if (neighbor) launch_shape<LBM_F32, true>(sh, t, p, blocks, s);
            else launch_shape<LBM_F32, false>(sh, t, p, blocks, s);
            break;
        case LBM_F16S:
            if (neighbor) launch_shape<LBM_F16S, true>(sh, t, p, blocks, s);
            else launch_shape<LBM_F16S, false>(sh, t, p, blocks, s);
            break;
        default:
            if (neighbor) launch_shape<LBM_BF16S, true>(sh, t, p, blocks, s);
            else launch_shape<LBM_BF16S, false>(sh, t, p, blocks, s);
            break;
    }
}

inline size_t al256(size_t v) { return (v + 255) / 256 * 256; }

struct BatchLayout {
    size_t args, start_nb, start_lc, member, total;
};
BatchLayout batch_layout(int n) {
    BatchLayout L{};
    size_t off = 0;
    L.args = off; off = al256(off + (size_t)n * sizeof(StepArgs));
    L.start_nb = off; off = al256(off + (size_t)(n + 1) * sizeof(unsigned));
    L.start_lc = off; off = al256(off + (size_t)(n + 1) * sizeof(unsigned));
    L.member = off; off = al256(off + (size_t)n * sizeof(int));
    L.total = off;
    return L;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_batch {
    std::vector<lbm_domain *> dom;
    std::vector<StepArgs> args;
    int store;
    cudaStream_t stream;
    char *ws;
    BatchLayout L;
    int shape;                     // index into kShapeSpec
    unsigned total_nb, total_lc;   // grid sizes of the two step kinds
    BatchParams *params[2];        // parameter-space tables (neighbour, local); null above kParamMembers
    cudaGraphExec_t graph;
    int graph_steps;
    int graph_parity;
    char err[512];
};

namespace {

lbm_status bfail(lbm_batch *b, lbm_status st, const char *fmt, ...) {
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

lbm_status bcuda(lbm_batch *b, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LBM_OK;
    return bfail(b, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Upload the step arguments and the block tables of the current shape.
lbm_status batch_upload(lbm_batch *b) {
    const int n = (int)b->dom.size();
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    if (kShapeSpec[b->shape].largest_first)   // largest member first: its blocks start earliest
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return b->args[x].g.N > b->args[y].g.N; });
    std::vector<unsigned> snb(n + 1), slc(n + 1);
    snb[0] = slc[0] = 0;
    for (int k = 0; k < n; ++k) {
        const StepArgs &a = b->args[order[k]];
        snb[k + 1] = snb[k] + member_blocks(b->store, a, true, b->shape);
        slc[k + 1] = slc[k] + member_blocks(b->store, a, false, b->shape);
    }
    b->total_nb = snb[n];
    b->total_lc = slc[n];
    if (b->params[0]) {
        for (int kind = 0; kind < 2; ++kind) {
            BatchParams &P = *b->params[kind];
            std::memset(&P, 0, sizeof(P));
            P.n = n;
            for (int m = 0; m < n; ++m) P.args[m] = b->args[m];
            for (int k = 0; k <= n; ++k) P.start[k] = kind == 0 ? snb[k] : slc[k];
            for (int k = 0; k < n; ++k) P.member[k] = order[k];
        }
    }
    const cudaStream_t s = b->stream;
    lbm_status st = bcuda(b, cudaMemcpyAsync(b->ws + b->L.args, b->args.data(), n * sizeof(StepArgs), cudaMemcpyHostToDevice, s), "batch upload");
    if (st == LBM_OK) st = bcuda(b, cudaMemcpyAsync(b->ws + b->L.start_nb, snb.data(), (n + 1) * sizeof(unsigned), cudaMemcpyHostToDevice, s), "batch upload");
    if (st == LBM_OK) st = bcuda(b, cudaMemcpyAsync(b->ws + b->L.start_lc, slc.data(), (n + 1) * sizeof(unsigned), cudaMemcpyHostToDevice, s), "batch upload");
    if (st == LBM_OK) st = bcuda(b, cudaMemcpyAsync(b->ws + b->L.member, order.data(), n * sizeof(int), cudaMemcpyHostToDevice, s), "batch upload");
    if (st == LBM_OK) st = bcuda(b, cudaStreamSynchronize(s), "batch upload sync");   // host vectors go out of scope
    return st;
}

// All members at the same step parity (they advance in lockstep); returns the parity or -1.
int batch_parity(const lbm_batch *b) {
    const long long t0 = lbm_steps_done(b->dom[0]);
    for (lbm_domain *d : b->dom)
        if ((lbm_steps_done(d) & 1) != (t0 & 1)) return -1;
    return (int)(t0 & 1);
}

// Enqueue nsteps batched steps starting at parity p (no bookkeeping).
void batch_enqueue(lbm_batch *b, int nsteps, int p) {
    const int n = (int)b->dom.size();
    if (b->shape == kSequential) {
        for (int k = 0; k < nsteps; ++k)
            for (int m = 0; m < n; ++m) launch_step(b->store, ((p + k) & 1) == 0, false, b->args[m], b->stream);
        return;
    }
    for (int k = 0; k < nsteps; ++k) {
        const bool neighbor = ((p + k) & 1) == 0;
        BatchTables t{(const StepArgs *)(b->ws + b->L.args),
                      (const unsigned *)(b->ws + (neighbor ? b->L.start_nb : b->L.start_lc)),
                      (const int *)(b->ws + b->L.member), n};
        launch_batch(b->store, b->shape, neighbor, t, b->params[neighbor ? 0 : 1], neighbor ? b->total_nb : b->total_lc,
                     b->stream);
    }
}

void batch_advance(lbm_batch *b, int nsteps) {
    for (lbm_domain *d : b->dom) domain_advance(d, nsteps);
}

void free_batch(lbm_batch *b) {
    delete b->params[0];
    delete b->params[1];
    delete b;
}

void drop_graph(lbm_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_steps = 0;
}

// Shapes 5..9 keep the member tables in the kernel's parameter space only (at most kParamMembers
// members); FP32 cells-per-thread shapes are the same as shape 0 for 16-bit storage.
bool shape_available(const lbm_batch *b, int shape) {
    if (shape >= kTableShapes && shape != kSequential && !b->params[0]) return false;
    if (b->store != LBM_F32 && kShapeSpec[shape].cpt != 0) return false;
    return true;
}

}  // namespace

extern "C" {

size_t lbm_batch_workspace_bytes(int n) {
    if (n < 1 || n > 4096) return 0;
    return batch_layout(n).total;
}

lbm_status lbm_batch_create(lbm_domain *const *domains, int n, void *workspace, size_t ws_bytes, void *stream,
                            lbm_batch **out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!domains || n < 1 || n > 4096 || !workspace || ((uintptr_t)workspace % 256)) return LBM_EINVAL;
    const BatchLayout L = batch_layout(n);
    if (ws_bytes < L.total) return LBM_ENOMEM;
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ENOMEM;
    b->err[0] = 0;
    b->stream = (cudaStream_t)stream;
    b->ws = (char *)workspace;
    b->L = L;
    b->shape = 0;
    b->graph = nullptr;
    b->graph_steps = 0;
    b->graph_parity = 0;
    b->params[0] = b->params[1] = nullptr;
    if (n <= kParamMembers) {
        b->params[0] = new (std::nothrow) BatchParams();
        b->params[1] = new (std::nothrow) BatchParams();
        if (!b->params[0] || !b->params[1]) {
            free_batch(b);
            return LBM_ENOMEM;
        }
    }
    for (int m = 0; m < n; ++m) {
        lbm_domain *d = domains[m];
        if (!d) { free_batch(b); return LBM_EINVAL; }
        const DomainView v = domain_view(d);
        const StepArgs &a = v.args;
        if (m == 0) b->store = v.store;
        bool bad = v.store != b->store || domain_stg_on(d);
        bad |= a.fx != 0.0f || a.fy != 0.0f || a.fz != 0.0f || a.ox != 0.0f || a.oy != 0.0f || a.oz != 0.0f;
        bad |= a.sponge_top > 0 || a.buffer_faces != 0;
        for (lbm_domain *e : b->dom) bad |= e == d;
        if (bad) {
            free_batch(b);
            return LBM_EINVAL;   // mixed storage, forced, turbulent-inflow or repeated members
        }
        b->dom.push_back(d);
        b->args.push_back(a);
    }
    if (batch_parity(b) < 0) {
        free_batch(b);
        return LBM_ESTATE;   // members must have taken steps of the same parity
    }
    const lbm_status st = batch_upload(b);
    if (st != LBM_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch *b, int nsteps) {
    if (!b) return LBM_EINVAL;
    if (nsteps < 0) return bfail(b, LBM_EINVAL, "batch step: nsteps must be >= 0");
    const int p = batch_parity(b);
    if (p < 0) return bfail(b, LBM_ESTATE, "batch step: members are at steps of different parity");
    batch_enqueue(b, nsteps, p);
    const lbm_status st = bcuda(b, cudaGetLastError(), "batch step launch");
    if (st == LBM_OK) batch_advance(b, nsteps);
    return st;
}

lbm_status lbm_batch_capture(lbm_batch *b, int nsteps) {
    if (!b) return LBM_EINVAL;
    if (nsteps < 2 || (nsteps & 1)) return bfail(b, LBM_EINVAL, "batch capture: nsteps must be even and >= 2");
    if (!b->stream) return bfail(b, LBM_EINVAL, "batch capture: needs a non-default stream");
    const int p = batch_parity(b);
    if (p < 0) return bfail(b, LBM_ESTATE, "batch capture: members are at steps of different parity");
    drop_graph(b);
    cudaGraph_t g = nullptr;
    lbm_status st = bcuda(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (st != LBM_OK) return st;
    batch_enqueue(b, nsteps, p);
    const cudaError_t le = cudaGetLastError();
    st = bcuda(b, cudaStreamEndCapture(b->stream, &g), "end capture");
    if (st == LBM_OK) st = bcuda(b, le, "captured launch");
    if (st == LBM_OK) st = bcuda(b, cudaGraphInstantiate(&b->graph, g, 0), "graph instantiate");
    if (g) cudaGraphDestroy(g);
    if (st != LBM_OK) {
        b->graph = nullptr;
        return st;
    }
    b->graph_steps = nsteps;
    b->graph_parity = p;
    return LBM_OK;
}

lbm_status lbm_batch_launch(lbm_batch *b) {
    if (!b) return LBM_EINVAL;
    if (!b->graph) return bfail(b, LBM_ESTATE, "batch launch: nothing captured");
    if (batch_parity(b) != b->graph_parity)
        return bfail(b, LBM_ESTATE, "batch launch: members are not at the parity the graph was captured at");
    const lbm_status st = bcuda(b, cudaGraphLaunch(b->graph, b->stream), "graph launch");
    if (st == LBM_OK) batch_advance(b, b->graph_steps);
    return st;
}

lbm_status lbm_batch_autotune(lbm_batch *b, int trial_steps, int *choice, float *ms_per_step) {
    if (!b) return LBM_EINVAL;
    if (trial_steps < 2 || (trial_steps & 1)) return bfail(b, LBM_EINVAL, "autotune: trial_steps must be even and >= 2");
    const int p = batch_parity(b);
    if (p < 0) return bfail(b, LBM_ESTATE, "autotune: members are at steps of different parity");
    drop_graph(b);
    cudaEvent_t e0, e1;
    lbm_status st = bcuda(b, cudaEventCreate(&e0), "event");
    if (st != LBM_OK) return st;
    st = bcuda(b, cudaEventCreate(&e1), "event");
    if (st != LBM_OK) { cudaEventDestroy(e0); return st; }
    float best = 0.0f;
    int best_shape = kSequential;
    bool any = false;
    for (int shape = 0; shape < kNumShapes && st == LBM_OK; ++shape) {
        if (ms_per_step) ms_per_step[shape] = -1.0f;
        if (!shape_available(b, shape)) continue;
        b->shape = shape;
        st = batch_upload(b);
        if (st != LBM_OK) break;
        batch_enqueue(b, 2, p);                      // warm-up (even: parity kept)
        st = bcuda(b, cudaEventRecord(e0, b->stream), "event");
        if (st != LBM_OK) break;
        batch_enqueue(b, trial_steps, p);
        st = bcuda(b, cudaEventRecord(e1, b->stream), "event");
        if (st == LBM_OK) st = bcuda(b, cudaEventSynchronize(e1), "event sync");
        if (st == LBM_OK) st = bcuda(b, cudaGetLastError(), "autotune launch");
        if (st != LBM_OK) break;
        batch_advance(b, 2 + trial_steps);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)trial_steps;
        if (ms_per_step) ms_per_step[shape] = ms;
        if (!any || ms < best) { best = ms; best_shape = shape; }
        any = true;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LBM_OK) return st;
    b->shape = best_shape;
    if (choice) *choice = best_shape;
    return batch_upload(b);
}

lbm_status lbm_batch_set_shape(lbm_batch *b, int shape) {
    if (!b) return LBM_EINVAL;
    if (shape < 0 || shape >= kNumShapes) return bfail(b, LBM_EINVAL, "batch shape out of range");
    if (!shape_available(b, shape))
        return bfail(b, LBM_EINVAL, "batch shape %d needs at most %d members", shape, kParamMembers);
    drop_graph(b);
    b->shape = shape;
    return batch_upload(b);
}

int lbm_batch_shape(const lbm_batch *b) { return b ? b->shape : -1; }

int lbm_batch_shape_count(void) { return kNumShapes; }

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->err : "no batch"; }

void lbm_batch_destroy(lbm_batch *b) {
    if (!b) return;
    drop_graph(b);
    free_batch(b);
}

}  // extern "C"

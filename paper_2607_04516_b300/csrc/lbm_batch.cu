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

#include "lbm_batch.cuh"

namespace lbm {
namespace {

using namespace lbm::batch;

unsigned member_blocks(int store, const StepArgs &a, bool neighbor, int sh) {
    switch (store) {
        case LBM_F32: return batch::member_blocks<LBM_F32>(a, neighbor, sh);
        case LBM_F16S: return batch::member_blocks<LBM_F16S>(a, neighbor, sh);
        default: return batch::member_blocks<LBM_BF16S>(a, neighbor, sh);
    }
}

void launch_batch(int store, int sh, bool neighbor, const BatchTables &t, const BatchParams *p, unsigned blocks,
                  cudaStream_t s) {
    switch (store) {
        case LBM_F32: launch_batch_s<LBM_F32>(sh, neighbor, t, p, blocks, s); break;
        case LBM_F16S: launch_batch_s<LBM_F16S>(sh, neighbor, t, p, blocks, s); break;
        default: launch_batch_s<LBM_BF16S>(sh, neighbor, t, p, blocks, s); break;
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
        // batched launches take the ground and top layers through the face blocks, as the
        // single-domain step does without zlat: the layer blocks' own kernel (k_step_layers) has no
        // batched form, and inlined into the batched kernels its variants cost their registers
        // (every batched shape ran at half speed)
        StepArgs ab = a;
        ab.zlat = 0;
        ab.nface_step = ab.nface;
        b->args.push_back(ab);
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

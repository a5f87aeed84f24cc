// Engine: context, model intake, device-resident products, the solve
// phases (each a CUDA graph whose while node runs sweep bodies until the
// device work list empties), Algorithm 2 and Algorithm 1, and the C-ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace morap {

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

#define CK(call)                                                                                         \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return ::morap::fail(MORAP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

#define CKL(expr)                                                                                        \
    do {                                                                                                 \
        int e_ = (expr);                                                                                 \
        if (e_ != 0)                                                                                     \
            return ::morap::fail(MORAP_ECUDA,                                                            \
                                 std::string(#expr) + ": " + cudaGetErrorString((cudaError_t)e_));       \
    } while (0)

#define CKR(expr)               \
    do {                        \
        int r_ = (expr);        \
        if (r_ != MORAP_OK)     \
            return r_;          \
    } while (0)

static inline int next_pow2(int k) {
    int p = 1;
    while (p < k) p <<= 1;
    return p;
}

}  // namespace morap

using namespace morap;

// ------------------------------------------------------------- the context
struct DevAlloc {
    void *ptr;
    size_t bytes;
};

struct LoopGraph {
    cudaGraphExec_t exec = nullptr;
    int grid = 0;
    int variant = -1;  // kernel shape of the sweeps (chosen before the graph is built)
    unsigned int tail = 0;  // work-list length at which k_sweep_tail takes the rest (0: none)
    int tail_grid = 0;      // its cooperative grid
};

struct morap_ctx {
    morap_config cfg{};
    int sm_count = 0;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev[8] = {};
    std::vector<HostAgent> agents;
    std::vector<HostTask> tasks;
    bool built = false;
    bool all_free_action = true;
    size_t device_bytes = 0;
    std::vector<DevAlloc> allocs;

    // products
    int P = 0, nI = 0, nJ = 0;
    // morap_select_pairs: the (agent, task) of each product to build, in
    // order; empty = every agent x task pair, product p = i * |J| + j
    std::vector<int32_t> sel_agent, sel_task;
    uint32_t TS = 0, TSA = 0, TT = 0;
    std::vector<ProdDesc> h_prods;      // with the merged transition offsets (tr_off, n_tr)
    std::vector<ProdDesc> h_prods_key;  // as computed from the models alone (the layout's identity)
    uint32_t *row_cnt = nullptr;        // [SA] merged transitions per product row (construction scratch)
    uint32_t *prod_tr = nullptr;        // [P] merged transitions per product (first build)
    std::vector<int4> h_chunks;
    int32_t *in_items = nullptr;  // [items][kInItems] input items of each sweep work item
    uint2 *item_w = nullptr;      // [items] (transitions, rows) of each work item
    uint8_t *chg[3] = {};         // per item: changed in sweep n % 3
    ProdDesc *d_prods = nullptr;
    AgentDesc *d_agents = nullptr;
    TaskDesc *d_tasks = nullptr;
    int4 *d_chunks = nullptr;
    uint4 *d_chunk_u = nullptr;  // per item: global state range and the product's first pre-sink state
    uint32_t *state_sa = nullptr, *state_tr = nullptr, *sa_tr = nullptr;
    int32_t *col = nullptr;
    int2 *cp32 = nullptr;
    float2 *pdf = nullptr, *costdf = nullptr;
    float *cost32 = nullptr;
    double *p64 = nullptr, *cost64 = nullptr;
    std::vector<void *> build_allocs;
    int64_t csr_bytes = 0;
    // resident model arrays (inputs of the product construction)
    AgentDesc *d_ad = nullptr;
    TaskDesc *d_td = nullptr;
    int32_t *d_sp = nullptr, *d_sap = nullptr, *d_succ = nullptr, *d_lp = nullptr, *d_la = nullptr, *d_ap = nullptr;
    double *d_prob = nullptr, *d_cost = nullptr;
    int16_t *d_nd = nullptr;
    uint8_t *d_letters = nullptr;
    uint32_t max_S = 1, max_work = 1, max_rows = 1;
    int max_row = 1;  // longest action row (successors) of any agent
    std::vector<size_t> layout_sig;
    int64_t last_h2d_bytes = 0;

    // solve buffers for Kp
    int Kp = 0;
    std::vector<void *> solve_allocs;
    void *V32[2] = {}, *V64[2] = {};
    uint8_t *a_rec = nullptr, *policy = nullptr, *frozen = nullptr;
    float2 *w32 = nullptr;
    double2 *w64 = nullptr;
    float4 *wdf = nullptr;
    double *thr32 = nullptr, *thr64 = nullptr, *d_W = nullptr, *d_c = nullptr;
    int32_t *d_status = nullptr, *sweeps_pair = nullptr;
    unsigned long long *res[3] = {};
    unsigned int *list[3] = {};
    LoopCtl *ctl = nullptr;  // [3]: FP32, FP64, evaluation
    LoopGraph g32[7], g64[7];  // per Kp = 1, 2, 4, ..., 64 (log2 index); g64: the polish phase
    int polish = kSweepDF;     // the polish kind of the current buffers (kSweepDF or kSweepDelta)
    void *Vd[2] = {};          // residual-correction polish: the correction, double buffered
    float *G = nullptr;        // residual-correction polish: [state-action][Kp] table
    SweepArgs argsd{};
    int Kcap = 0;              // weights per product the solve buffers hold
    double ms_tune = 0.0;      // host time spent choosing kernel shapes (cumulative)
    SweepArgs args32{}, args64{};

    // evaluation buffers (capacity-based)
    std::vector<void *> eval_allocs;
    size_t eval_cap_pairs = 0, eval_cap_chunks = 0, eval_cap_states = 0;
    float4 *E[2] = {};
    int4 *d_epairs = nullptr, *d_echunks = nullptr;
    int *d_ebpairs = nullptr;  // pairs evaluated one block each (k_eval_block)
    bool eval_block_ready = false;
    unsigned long long *eres[3] = {};
    unsigned int *elist[3] = {};
    int32_t *esweeps = nullptr;
    uint8_t *efrozen = nullptr;
    uint32_t *item_tmu = nullptr, *pair_tmu = nullptr;  // scheduler transitions per eval item / pair
    double *d_rc = nullptr, *d_rp = nullptr;
    int32_t *ecol = nullptr;
    float2 *ep = nullptr, *ecost = nullptr;
    LoopGraph geval[24];  // per grid bucket: min(full grid, 2^b) blocks
    int eval_full_grid = 0;
    bool eval_ready = false;
    EvalArgs eargs{};

    // pinned host staging
    LoopCtl *h_ctl = nullptr;
    double *h_stage = nullptr;
    size_t h_stage_bytes = 0;

    morap_solve_stats stats{};
    std::vector<int> last_assign;  // [K][nJ] of the last supporting-point call
    int last_K = 0;                // weights whose schedulers the last optimisation left on the device
};

namespace {

void dev_free_list(morap_ctx *c, std::vector<void *> &lst) {
    for (void *p : lst) {
        for (size_t i = 0; i < c->allocs.size(); ++i)
            if (c->allocs[i].ptr == p) {
                if (c->cfg.free)
                    c->cfg.free(p, c->allocs[i].bytes, c->cfg.alloc_user);
                else
                    cudaFree(p);
                c->device_bytes -= c->allocs[i].bytes;
                c->allocs.erase(c->allocs.begin() + i);
                break;
            }
    }
    lst.clear();
}

// Allocate `bytes` of device memory into *out, tracked in `lst`.  Refuses
// (ENOMEM) before allocating when the budget would be exceeded.
template <typename T>
int dev_alloc(morap_ctx *c, std::vector<void *> &lst, T **out, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    if (c->cfg.hbm_budget && c->device_bytes + bytes > c->cfg.hbm_budget)
        return fail(MORAP_ENOMEM, "HBM budget exceeded: need " + std::to_string(c->device_bytes + bytes) +
                                      " bytes, budget " + std::to_string(c->cfg.hbm_budget));
    void *p = nullptr;
    if (c->cfg.alloc) {
        p = c->cfg.alloc(bytes, c->cfg.alloc_user);
        if (!p) return fail(MORAP_ENOMEM, "allocator callback failed for " + std::to_string(bytes) + " bytes");
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(MORAP_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
    }
    c->allocs.push_back({p, bytes});
    c->device_bytes += bytes;
    lst.push_back(p);
    *out = static_cast<T *>(p);
    return MORAP_OK;
}

int stage_ctl(morap_ctx *c) {
    if (!c->h_ctl) CK(cudaMallocHost((void **)&c->h_ctl, sizeof(LoopCtl)));
    return MORAP_OK;
}

int stage(morap_ctx *c, size_t bytes) {
    if (bytes <= c->h_stage_bytes) return MORAP_OK;
    if (c->h_stage) cudaFreeHost(c->h_stage);
    c->h_stage = nullptr;
    c->h_stage_bytes = 0;
    CK(cudaMallocHost((void **)&c->h_stage, bytes));
    c->h_stage_bytes = bytes;
    return MORAP_OK;
}

void destroy_graph(LoopGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
}

void free_solve(morap_ctx *c) {
    for (int i = 0; i < 7; ++i) {
        destroy_graph(c->g32[i]);
        destroy_graph(c->g64[i]);
        c->g32[i].grid = c->g64[i].grid = 0;
        c->g32[i].variant = c->g64[i].variant = -1;
    }
    c->Vd[0] = c->Vd[1] = nullptr;
    c->G = nullptr;
    dev_free_list(c, c->solve_allocs);
    c->Kp = 0;
    c->Kcap = 0;
    c->last_K = 0;  // the schedulers of the last solve are gone
}

int log2_of(int Kp) {
    int l = 0;
    while ((1 << l) < Kp) ++l;
    return l;
}

void free_eval(morap_ctx *c) {
    for (auto &g : c->geval) {
        destroy_graph(g);
        g.grid = 0;
    }
    c->eval_ready = false;
    dev_free_list(c, c->eval_allocs);
    c->eval_cap_pairs = c->eval_cap_chunks = c->eval_cap_states = 0;
}

// Grid of a persistent sweep launch: every co-resident block, no more (the
// blocks pull work items until the sweep's list is exhausted).
int sweep_grid(morap_ctx *c, int blocks_per_sm) { return c->sm_count * std::max(1, blocks_per_sm); }

int no_tail(cudaStream_t) { return 0; }

// Build one device loop: a graph whose while node repeats a body of six
// sweep launches and one control launch until the control kernel clears the
// condition (work list down to g.tail items, or empty, or sweep cap), then,
// with g.tail > 0, one tail launch that runs the remaining sweeps.
template <typename F, typename T>
int build_loop_graph(morap_ctx *c, LoopGraph &g, LoopCtl *ctl, F &&launch_sweep_at, T &&launch_tail) {
    destroy_graph(g);
    cudaGraph_t graph = nullptr;
    CK(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    CK(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int rc = 0;
    for (int pos = 0; pos < 6 && rc == 0; ++pos) rc = launch_sweep_at(pos, c->cap_stream);
    if (rc == 0) rc = launch_loop_control(ctl, (unsigned long long)handle, 0, c->cap_stream);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &captured);
    if (rc != 0) {
        cudaGraphDestroy(graph);
        return fail(MORAP_ECUDA, std::string("capturing a sweep body: ") + cudaGetErrorString((cudaError_t)rc));
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(MORAP_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    }
    if (g.tail > 0) {  // the tail launch, after the while node
        e = cudaStreamBeginCaptureToGraph(c->cap_stream, graph, &node, nullptr, 1, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = launch_tail(c->cap_stream);
            captured = nullptr;
            e = cudaStreamEndCapture(c->cap_stream, &captured);
        }
        if (rc != 0 || e != cudaSuccess) {
            cudaGraphDestroy(graph);
            return fail(MORAP_ECUDA, std::string("capturing a tail launch: ") +
                                         cudaGetErrorString(rc != 0 ? (cudaError_t)rc : e));
        }
    }
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(MORAP_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    return MORAP_OK;
}

// Run one sweep loop: the captured graph (launch_mode 0), or the same
// kernels body by body from the host, reading the work list in between.
template <typename F, typename T>
int run_loop(morap_ctx *c, LoopGraph &g, LoopCtl *ctl, cudaStream_t s, F &&launch_sweep_at, T &&launch_tail) {
    if (c->cfg.launch_mode == 0) {
        CK(cudaGraphLaunch(g.exec, s));
        return MORAP_OK;
    }
    CKR(stage_ctl(c));
    for (;;) {
        for (int pos = 0; pos < 6; ++pos) CKL(launch_sweep_at(pos, s));
        CKL(launch_loop_control_host(ctl, 0, s));
        CK(cudaMemcpyAsync(c->h_ctl, ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (c->h_ctl->cnt[0] <= g.tail || c->h_ctl->sweep_base >= c->h_ctl->cap) break;
    }
    if (g.tail > 0) CKL(launch_tail(s));
    return MORAP_OK;
}

// Blocks of a sweep launch with kernel shape v: every co-resident block, but
// no more than one warp per work item needs.
int sweep_launch_grid(morap_ctx *c, int kind, int Kp, int v) {
    const size_t useful = (c->h_chunks.size() + kThreads / 32 - 1) / (kThreads / 32);
    return std::max(1, (int)std::min<size_t>((size_t)sweep_grid(c, sweep_blocks_per_sm(kind, Kp, v)), useful));
}

// Build the loop graph of one phase for kernel shape v.
// The arguments of a sweep kind (the polish kinds share the phase-2 control block).
const SweepArgs &args_of(morap_ctx *c, int kind) {
    return kind == kSweepF32 ? c->args32 : kind == kSweepDF ? c->args64 : c->argsd;
}

// The tail of a phase's loop (config tail_items): the cooperative grid is
// every block that can be resident (no more than one warp per work item
// needs), and the loop hands over once its list has at most tail_items
// items, and never more than that grid has warps.  -1: a quarter of its
// warps, the longest list at which every item is split over two or more
// warps (a warp's share of 32 states or fewer, one staged batch that the
// warp keeps for the rest of the launch).
void setup_tail(morap_ctx *c, LoopGraph &G, int kind, int Kp) {
    G.tail = 0;
    G.tail_grid = 0;
    if (c->cfg.tail_items == 0) return;
    const int bps = sweep_tail_blocks_per_sm(kind, Kp);
    if (bps <= 0) return;  // no occupancy figure: the loop runs to the end one launch per sweep
    const size_t useful = (c->h_chunks.size() + kThreads / 32 - 1) / (kThreads / 32);
    G.tail_grid = (int)std::max<size_t>(1, std::min<size_t>((size_t)c->sm_count * bps, useful));
    // the tail launch deals its first list to its warps, one item per warp at most
    const unsigned int warps = (unsigned int)G.tail_grid * (unsigned int)(kThreads / 32);
    G.tail = c->cfg.tail_items > 0 ? std::min((unsigned int)c->cfg.tail_items, warps) : std::max(1u, warps / 4);
}

int build_phase_graph(morap_ctx *c, LoopGraph &G, int kind, int Kp, int v) {
    destroy_graph(G);
    G.variant = v;
    G.grid = sweep_launch_grid(c, kind, Kp, v);
    setup_tail(c, G, kind, Kp);
    if (c->cfg.launch_mode != 0) return MORAP_OK;
    const SweepArgs a = args_of(c, kind);
    const int grid = G.grid, tgrid = G.tail_grid;
    return build_loop_graph(
        c, G, a.ctl, [&](int pos, cudaStream_t st) { return launch_sweep(kind, Kp, v, a, pos, grid, st); },
        [&](cudaStream_t st) { return launch_sweep_tail(kind, Kp, a, tgrid, st); });
}

// The tuner.  The first solve of a phase at a given Kp runs its loop from the
// host, body by body (six sweeps and the control kernel), rotating the kernel
// shape from one body to the next, and times each body with CUDA events
// against the algorithmic bytes it moved; the shape with the most bytes per
// millisecond over the whole loop is kept and the phase's graph is built with
// it.  Every shape does the same arithmetic, so the solve's results are those
// of any single shape; only the first solve pays for the host round trips.
int run_loop_tuning(morap_ctx *c, LoopGraph &G, int kind, int Kp, cudaStream_t s) {
    const SweepArgs a = args_of(c, kind);
    const int nvar = sweep_variant_count(kind);
    std::vector<double> ms(nvar, 0.0), bytes(nvar, 0.0);
    CKR(stage_ctl(c));
    unsigned long long prev_bytes = 0;
    for (int body = 0;; ++body) {
        const int v = body % nvar;
        const int grid = sweep_launch_grid(c, kind, Kp, v);
        CK(cudaEventRecord(c->ev[7], s));
        for (int pos = 0; pos < 6; ++pos) CKL(launch_sweep(kind, Kp, v, a, pos, grid, s));
        CK(cudaEventRecord(c->ev[5], s));
        CKL(launch_loop_control_host(a.ctl, 0, s));
        CK(cudaMemcpyAsync(c->h_ctl, a.ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, c->ev[7], c->ev[5]));
        ms[v] += t;
        bytes[v] += (double)(c->h_ctl->bytes - prev_bytes);
        prev_bytes = c->h_ctl->bytes;
        if (c->h_ctl->cnt[0] == 0 || c->h_ctl->sweep_base >= c->h_ctl->cap) break;
    }
    int best = 0;
    double best_rate = -1.0;
    for (int v = 0; v < nvar; ++v)
        if (ms[v] > 0.0 && bytes[v] / ms[v] > best_rate) {
            best_rate = bytes[v] / ms[v];
            best = v;
        }
    return build_phase_graph(c, G, kind, Kp, best);
}

// Make the loop of one phase ready for Kp: the shape forced by the config,
// shape 0 for instances whose sweeps are too short for the shape to matter,
// otherwise (first solve at this Kp) the tuner decides inside the solve.
// Returns through `tune` whether this solve must run the tuning loop.
int prepare_phase(morap_ctx *c, int kind, int Kp, bool &tune) {
    LoopGraph &G = kind == kSweepF32 ? c->g32[log2_of(Kp)] : c->g64[log2_of(Kp)];
    tune = false;
    if (G.variant >= 0) return MORAP_OK;
    CKL(sweep_setup_attributes());
    const int forced = kind == kSweepF32 ? c->cfg.sweep_variant_fp32 : c->cfg.sweep_variant_fp64;
    const bool worth = (double)c->TT * (double)Kp >= (double)(1u << 24);
    if (forced >= sweep_variant_count(kind))
        return fail(MORAP_EINVAL, "config: sweep_variant_fp64 is not a shape of this polish form");
    if (forced >= 0) return build_phase_graph(c, G, kind, Kp, forced);
    if (!worth) return build_phase_graph(c, G, kind, Kp, 0);
    tune = true;
    return MORAP_OK;
}

// Solve buffers are sized for the largest Kp seen so far (a [state][Kp]
// layout for a smaller Kp fits inside), so batches of varying size do not
// reallocate; the loop graphs are kept per Kp.
int ensure_solve(morap_ctx *c, int Kp) {
    if (Kp <= c->Kcap) {
        c->Kp = Kp;
        return MORAP_OK;
    }
    free_solve(c);
    const size_t TS = c->TS, P = c->P;
    const size_t np = P * Kp;
    auto &L = c->solve_allocs;
    if (c->all_free_action && c->cfg.precision == MORAP_PREC_MIXED) {
        CKR(dev_alloc(c, L, (float **)&c->V32[0], TS * Kp * sizeof(float)));
        CKR(dev_alloc(c, L, (float **)&c->V32[1], TS * Kp * sizeof(float)));
    }
    CKR(dev_alloc(c, L, (double **)&c->V64[0], TS * Kp * sizeof(double)));
    CKR(dev_alloc(c, L, (double **)&c->V64[1], TS * Kp * sizeof(double)));
    c->polish = kSweepDF;
    if (c->V32[0] && c->cfg.polish == 0) {
        c->polish = kSweepDelta;
        CKR(dev_alloc(c, L, (float **)&c->Vd[0], TS * Kp * sizeof(float)));
        CKR(dev_alloc(c, L, (float **)&c->Vd[1], TS * Kp * sizeof(float)));
        CKR(dev_alloc(c, L, &c->G, std::max<size_t>(c->TSA, 1) * Kp * sizeof(float)));
    }
    CKR(dev_alloc(c, L, &c->a_rec, TS * Kp));
    CKR(dev_alloc(c, L, &c->policy, TS * Kp));
    CKR(dev_alloc(c, L, &c->frozen, np));
    CKR(dev_alloc(c, L, &c->w32, np * sizeof(float2)));
    CKR(dev_alloc(c, L, &c->w64, np * sizeof(double2)));
    CKR(dev_alloc(c, L, &c->wdf, np * sizeof(float4)));
    CKR(dev_alloc(c, L, &c->thr32, np * sizeof(double)));
    CKR(dev_alloc(c, L, &c->thr64, np * sizeof(double)));
    CKR(dev_alloc(c, L, &c->d_W, (size_t)Kp * (c->nI + c->nJ) * sizeof(double)));
    CKR(dev_alloc(c, L, &c->d_c, np * sizeof(double)));
    CKR(dev_alloc(c, L, &c->d_status, np * sizeof(int32_t)));
    CKR(dev_alloc(c, L, &c->sweeps_pair, np * sizeof(int32_t)));
    for (int i = 0; i < 3; ++i) {
        CKR(dev_alloc(c, L, &c->res[i], np * sizeof(unsigned long long)));
        CKR(dev_alloc(c, L, &c->list[i], c->h_chunks.size() * sizeof(unsigned int)));
    }
    CKR(dev_alloc(c, L, &c->ctl, 3 * sizeof(LoopCtl)));
    c->Kp = Kp;
    c->Kcap = Kp;

    SweepArgs a{};
    a.state_sa = c->state_sa;
    a.state_tr = c->state_tr;
    a.sa_tr = c->sa_tr;
    a.col = c->col;
    a.cp32 = c->cp32;
    a.pdf = c->pdf;
    a.costdf = c->costdf;
    a.wdf = c->wdf;
    a.p64 = c->p64;
    a.cost32 = c->cost32;
    a.cost64 = c->cost64;
    a.chunks = c->d_chunks;
    a.chunk_u = c->d_chunk_u;
    a.prods = c->d_prods;
    a.w32 = c->w32;
    a.w64 = c->w64;
    for (int i = 0; i < 3; ++i) {
        a.res[i] = c->res[i];
        a.list[i] = c->list[i];
    }
    a.sweeps_pair = c->sweeps_pair;
    a.frozen = c->frozen;
    a.a_rec = c->a_rec;
    a.in_items = c->in_items;
    a.item_w = c->item_w;
    a.skip = c->cfg.skip_unchanged ? 1 : 0;
    // instances with many more work items than resident warps keep their
    // lists in order (their values do not fit in L2; see k_sweep)
    a.keep_batch = c->h_chunks.size() >= (size_t)16 * 16 * std::max(1, c->sm_count) ? 1 : 4;
    for (int q = 0; q < 3; ++q) a.chg[q] = c->chg[q];
    a.eps1 = c->cfg.eps_vi;
    a.eps1f = (float)c->cfg.eps_vi;
    a.gmax = c->cfg.item_warps_max > 0 ? c->cfg.item_warps_max : 8;
    a.P = c->P;
    SweepArgs a32 = a, a64 = a;
    a32.thr = c->thr32;
    a32.ctl = c->ctl + 0;
    a32.V[0] = c->V32[0];
    a32.V[1] = c->V32[1];
    a64.thr = c->thr64;
    a64.ctl = c->ctl + 1;
    a64.V[0] = c->V64[0];
    a64.V[1] = c->V64[1];
    c->args32 = a32;
    c->args64 = a64;
    SweepArgs ad = a64;  // the residual correction iterates d with the phase-2 control block
    ad.V[0] = c->Vd[0];
    ad.V[1] = c->Vd[1];
    ad.G = c->G;
    c->argsd = ad;
    if (c->cfg.in_place) {  // one value array per phase: a sweep reads what it has already written
        c->args32.V[1] = c->args32.V[0];
        c->args64.V[1] = c->args64.V[0];
        c->argsd.V[1] = c->argsd.V[0];
    }
    return MORAP_OK;
}

int ensure_eval(morap_ctx *c, size_t n_pairs, size_t n_chunks, size_t n_states) {
    if (n_pairs <= c->eval_cap_pairs && n_chunks <= c->eval_cap_chunks && n_states <= c->eval_cap_states &&
        c->eval_ready && c->eargs.policy == c->policy)
        return MORAP_OK;
    free_eval(c);
    n_pairs = std::max<size_t>(n_pairs, 1);
    n_chunks = std::max<size_t>(n_chunks, 1);
    n_states = std::max<size_t>(n_states, 1);
    auto &L = c->eval_allocs;
    CKR(dev_alloc(c, L, &c->E[0], n_states * sizeof(float4)));
    CKR(dev_alloc(c, L, &c->E[1], n_states * sizeof(float4)));
    CKR(dev_alloc(c, L, &c->d_epairs, n_pairs * sizeof(int4)));
    CKR(dev_alloc(c, L, &c->d_echunks, n_chunks * sizeof(int4)));
    CKR(dev_alloc(c, L, &c->d_ebpairs, n_pairs * sizeof(int)));
    for (int i = 0; i < 3; ++i) {
        CKR(dev_alloc(c, L, &c->eres[i], n_pairs * sizeof(unsigned long long)));
        CKR(dev_alloc(c, L, &c->elist[i], n_chunks * sizeof(unsigned int)));
    }
    CKR(dev_alloc(c, L, &c->esweeps, n_pairs * sizeof(int32_t)));
    CKR(dev_alloc(c, L, &c->efrozen, n_pairs));
    CKR(dev_alloc(c, L, &c->d_rc, n_pairs * sizeof(double)));
    CKR(dev_alloc(c, L, &c->d_rp, n_pairs * sizeof(double)));
    CKR(dev_alloc(c, L, &c->ecol, n_states * (size_t)c->max_row * sizeof(int32_t)));
    CKR(dev_alloc(c, L, &c->ep, n_states * (size_t)c->max_row * sizeof(float2)));
    CKR(dev_alloc(c, L, &c->ecost, n_states * sizeof(float2)));
    CKR(dev_alloc(c, L, &c->item_tmu, n_chunks * sizeof(uint32_t)));
    CKR(dev_alloc(c, L, &c->pair_tmu, n_pairs * sizeof(uint32_t)));
    c->eval_cap_pairs = n_pairs;
    c->eval_cap_chunks = n_chunks;
    c->eval_cap_states = n_states;
    EvalArgs e{};
    e.state_sa = c->state_sa;
    e.sa_tr = c->sa_tr;
    e.col = c->col;
    e.pdf = c->pdf;
    e.costdf = c->costdf;
    e.prods = c->d_prods;
    e.policy = c->policy;
    e.Kp = c->Kp;
    e.chunks = c->d_echunks;
    e.pairs = c->d_epairs;
    e.thr = c->cfg.eps_eval;
    for (int i = 0; i < 3; ++i) {
        e.res[i] = c->eres[i];
        e.list[i] = c->elist[i];
    }
    e.sweeps_pair = c->esweeps;
    e.frozen = c->efrozen;
    e.item_tmu = c->item_tmu;
    e.pair_tmu = c->pair_tmu;
    e.ctl = c->ctl + 2;
    e.E[0] = c->E[0];
    e.E[1] = c->E[1];
    e.ecol = c->ecol;
    e.ep = c->ep;
    e.ecost = c->ecost;
    e.stride = c->max_row;
    c->eargs = e;
    c->eval_full_grid = sweep_grid(c, eval_blocks_per_sm());
    c->eval_ready = true;
    return MORAP_OK;
}

// The evaluation loop for n_chunks work items (one block each): a graph per
// power-of-two grid bucket, so small evaluations do not occupy every SM.
LoopGraph *eval_graph(morap_ctx *c, size_t n_chunks, int &rc) {
    int b = 0;
    while (((size_t)1 << b) < n_chunks && b < 23) ++b;
    LoopGraph &g = c->geval[b];
    rc = MORAP_OK;
    if (g.grid) return &g;
    g.grid = std::max(1, (int)std::min<size_t>((size_t)c->eval_full_grid, (size_t)1 << b));
    if (c->cfg.launch_mode == 0) {
        const EvalArgs e = c->eargs;
        const int grid = g.grid;
        rc = build_loop_graph(
            c, g, e.ctl, [&](int pos, cudaStream_t s) { return launch_eval_sweep(e, pos, grid, s); }, no_tail);
    }
    return &g;
}

double ms_between(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return (double)ms;
}

int check_weights(morap_ctx *c, int K, const double *W) {
    const int n = c->nI + c->nJ;
    for (int k = 0; k < K; ++k)
        for (int i = 0; i < n; ++i) {
            const double w = W[(size_t)k * n + i];
            if (!(w >= 0.0) || !std::isfinite(w))
                return fail(MORAP_EINVAL, "weight vectors need finite entries >= 0 (row " + std::to_string(k) + ")");
        }
    return MORAP_OK;
}

// Algorithm 2 loop 1 (Algorithm 3 for all products and K <= 64 weights):
// leaves the scheduler in c->policy and c_ij in h_c[p*Kp + k]; per-pair
// status in h_status.
int run_optimisation(morap_ctx *c, int K, const double *W, cudaStream_t s, std::vector<double> &h_c,
                     std::vector<int32_t> &h_status) {
    const int Kp = next_pow2(K);
    c->last_K = 0;
    CKR(ensure_solve(c, Kp));
    const size_t np = (size_t)c->P * Kp;
    const size_t nW = (size_t)K * (c->nI + c->nJ);
    CKR(stage(c, std::max(nW * sizeof(double), np * (sizeof(double) + sizeof(int32_t)) + 3 * sizeof(LoopCtl))));
    std::memcpy(c->h_stage, W, nW * sizeof(double));
    CK(cudaMemcpyAsync(c->d_W, c->h_stage, nW * sizeof(double), cudaMemcpyHostToDevice, s));
    CKL(launch_setup_weights(c->d_prods, c->P, c->nI, c->nJ, K, Kp, c->d_W, c->w32, c->w64, c->wdf, c->thr32,
                             c->thr64, c->cfg.eps_vi, c->V32[0] != nullptr, s));
    const size_t nv = (size_t)c->TS * Kp;
    const unsigned int cap = (unsigned int)std::max(1, c->cfg.max_sweeps);
    const unsigned int n_items = (unsigned int)c->h_chunks.size();
    int launches = 1;  // setup_weights
    CK(cudaMemsetAsync(c->a_rec, 0, nv, s));
    const bool mixed = c->V32[0] != nullptr;
    if (mixed) {
        CK(cudaMemsetAsync(c->V32[0], 0, nv * sizeof(float), s));
        CK(cudaMemsetAsync(c->V32[1], 0, nv * sizeof(float), s));
        bool tune = false;
        CKR(prepare_phase(c, kSweepF32, Kp, tune));
        LoopGraph &G32 = c->g32[log2_of(Kp)];
        CKL(launch_loop_init(c->ctl + 0, c->list[0], n_items, c->res, np, c->sweeps_pair, c->frozen, cap, s,
                             c->chg[2], c->w64, tune ? 0u : G32.tail));
        const auto t0 = std::chrono::steady_clock::now();
        CK(cudaEventRecord(c->ev[0], s));
        if (tune) {
            CKR(run_loop_tuning(c, G32, kSweepF32, Kp, s));
        } else {
            const SweepArgs a32 = c->args32;
            const int grid = G32.grid, v = G32.variant, tgrid = G32.tail_grid;
            CKR(run_loop(
                c, G32, c->ctl + 0, s,
                [&](int pos, cudaStream_t st) { return launch_sweep(kSweepF32, Kp, v, a32, pos, grid, st); },
                [&](cudaStream_t st) { return launch_sweep_tail(kSweepF32, Kp, a32, tgrid, st); }));
        }
        CK(cudaEventRecord(c->ev[1], s));
        if (tune) c->ms_tune += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (c->polish == kSweepDelta) {
            // the residual correction starts from d = 0 on the table of the FP32 result
            CKL(launch_delta_table(Kp, c->args64, (int)n_items, (const float *)c->V32[0], c->G, s));
            CK(cudaMemsetAsync(c->Vd[0], 0, nv * sizeof(float), s));
            CK(cudaMemsetAsync(c->Vd[1], 0, nv * sizeof(float), s));
        } else {
            CKL(launch_convert((const float *)c->V32[0], (float2 *)c->V64[0], (float2 *)c->V64[1], nv, s));
        }
        launches += 2;
    } else {
        CK(cudaMemsetAsync(c->V64[0], 0, nv * sizeof(double), s));
        CK(cudaMemsetAsync(c->V64[1], 0, nv * sizeof(double), s));
    }
    const int pk = mixed ? c->polish : kSweepDF;  // the polish kind of this solve
    bool tune64 = false;
    CKR(prepare_phase(c, pk, Kp, tune64));
    LoopGraph &G64 = c->g64[log2_of(Kp)];
    CKL(launch_loop_init(c->ctl + 1, c->list[0], n_items, c->res, np, c->sweeps_pair, c->frozen, cap, s,
                         c->chg[2], c->w64, tune64 ? 0u : G64.tail));
    const auto t64 = std::chrono::steady_clock::now();
    CK(cudaEventRecord(c->ev[6], s));
    if (tune64) {
        CKR(run_loop_tuning(c, G64, pk, Kp, s));
    } else {
        const SweepArgs a2 = args_of(c, pk);
        const int grid = G64.grid, v = G64.variant, tgrid = G64.tail_grid;
        CKR(run_loop(
            c, G64, c->ctl + 1, s,
            [&](int pos, cudaStream_t st) { return launch_sweep(pk, Kp, v, a2, pos, grid, st); },
            [&](cudaStream_t st) { return launch_sweep_tail(pk, Kp, a2, tgrid, st); }));
    }
    CK(cudaEventRecord(c->ev[2], s));
    if (tune64) c->ms_tune += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t64).count();
    if (pk == kSweepDelta) {  // V = B + d, exactly, in double-float
        CKL(launch_delta_combine((const float *)c->V32[0], (const float *)c->Vd[0], (float2 *)c->V64[0], nv, s));
        launches += 1;
    }
    CKL(launch_finalize(Kp, c->args64, (int)n_items, c->cfg.tau_policy, c->policy, s));
    CKL(launch_gather_c(Kp, c->d_prods, c->P, (const float2 *)c->V64[0], c->frozen, c->d_c, c->d_status, s));
    CK(cudaEventRecord(c->ev[3], s));
    launches += 3;
    double *hc = c->h_stage;
    int32_t *hs = (int32_t *)(hc + np);
    LoopCtl *hctl = (LoopCtl *)(hs + np + (np & 1));
    CK(cudaMemcpyAsync(hc, c->d_c, np * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hs, c->d_status, np * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hctl, c->ctl, 2 * sizeof(LoopCtl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if ((mixed && hctl[0].bar_err) || hctl[1].bar_err)
        return fail(MORAP_ECUDA, "a sweep loop's tail launch gave up waiting at a grid barrier (1 s)");
    // The scheduler's anchoring rounds, only when some recorded action was
    // not kept (rare: its value drifted by steps below eps1 after the record).
    for (int round = 1, pending = (int)hctl[1].undecided; pending > 0 && round <= kAnchorRounds; ++round) {
        CK(cudaMemsetAsync(&c->ctl[1].decided, 0, sizeof(unsigned int), s));
        CKL(launch_anchor(Kp, c->args64, (int)n_items, c->cfg.tau_policy, c->policy, round, s));
        CK(cudaMemcpyAsync(&hctl[1].decided, &c->ctl[1].decided, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        ++launches;
        if (hctl[1].decided == 0) break;
        pending -= (int)hctl[1].decided;
    }
    h_c.assign(hc, hc + np);
    h_status.assign(hs, hs + np);
    morap_solve_stats &st = c->stats;
    st = morap_solve_stats{};
    st.K = K;
    if (mixed) {
        st.fp32_sweeps = (int32_t)hctl[0].sweep_base;
        st.skipped_fp32 = (int64_t)hctl[0].skipped;
        st.computed_fp32 = (int64_t)hctl[0].computed;
        st.updates_fp32 = (int64_t)hctl[0].updates;
        st.bytes_fp32 = (int64_t)hctl[0].bytes;
        st.ms_fp32 = ms_between(c->ev[0], c->ev[1]);
    }
    st.fp64_sweeps = (int32_t)hctl[1].sweep_base;
    st.skipped_fp64 = (int64_t)hctl[1].skipped;
    st.computed_fp64 = (int64_t)hctl[1].computed;
    st.anchored_states = (int64_t)hctl[1].undecided;
    st.work_items = (int64_t)n_items;
    st.updates_fp64 = (int64_t)hctl[1].updates;
    st.bytes_fp64 = (int64_t)hctl[1].bytes;
    st.ms_fp64 = ms_between(c->ev[6], c->ev[2]);
    st.ms_finalise = ms_between(c->ev[2], c->ev[3]);
    st.h2d_bytes = (int64_t)(nW * sizeof(double));
    st.d2h_bytes = (int64_t)(np * (sizeof(double) + sizeof(int32_t)) + 2 * sizeof(LoopCtl));
    // one launch per sweep and one control launch per body of six, except
    // the sweeps of a tail launch (one launch, which a loop with a tail
    // threshold makes even when no sweep is left for it)
    if (mixed) {
        st.tail_sweeps_fp32 = (int32_t)hctl[0].tail_sweeps;
        const int n = st.fp32_sweeps - st.tail_sweeps_fp32;
        launches += n + n / 6 + (hctl[0].tail > 0 ? 1 : 0);
    }
    st.tail_sweeps_fp64 = (int32_t)hctl[1].tail_sweeps;
    const int n64 = st.fp64_sweeps - st.tail_sweeps_fp64;
    launches += n64 + n64 / 6 + (hctl[1].tail > 0 ? 1 : 0);
    st.kernel_launches = launches;
    st.variant_fp32 = mixed ? c->g32[log2_of(Kp)].variant : -1;
    st.variant_fp64 = c->g64[log2_of(Kp)].variant;
    st.polish = pk == kSweepDelta ? 0 : 1;
    st.ms_tune = c->ms_tune;
    int bad = 0;
    for (int p = 0; p < c->P; ++p)
        for (int k = 0; k < K; ++k) bad += h_status[(size_t)p * Kp + k] != MORAP_OK;
    st.pairs_not_converged = bad;
    c->last_K = K;
    return MORAP_OK;
}

// Algorithm 4 for a list of (product, weight) pairs under the scheduler in
// c->policy; returns r_cost and r_prob per pair.
int run_evaluation_group(morap_ctx *c, const std::vector<int4> &pairs_in, cudaStream_t s, std::vector<double> &rc,
                         std::vector<double> &rp, int &not_conv) {
    std::vector<int4> pairs = pairs_in;
    // Pairs small enough for one block run all their sweeps in k_eval_block;
    // the others go through the multi-launch loop over kEvalChunk-state
    // items.  The loop's items come first in `chunks`, then those of the
    // block pairs (every pair's rows are compacted).
    std::vector<int4> chunks, bchunks;
    std::vector<int> bpairs;
    uint32_t bmax = 0;
    size_t off = 0;
    for (size_t e = 0; e < pairs.size(); ++e) {
        const ProdDesc &pd = c->h_prods[pairs[e].x];
        pairs[e].z = (int)off;
        off += pd.n_nd + 1;
        const bool block = c->cfg.eval_block && pd.n_nd + 1 <= kEvalBlockStates;
        if (block) {
            bpairs.push_back((int)e);
            bmax = std::max(bmax, pd.n_nd + 1);
        }
        for (uint32_t b = 0; b < pd.n_nd; b += kEvalChunk)
            (block ? bchunks : chunks)
                .push_back(make_int4((int)e, (int)b, (int)std::min<uint32_t>(pd.n_nd, b + kEvalChunk), b == 0));
    }
    const size_t n_loop = chunks.size();
    chunks.insert(chunks.end(), bchunks.begin(), bchunks.end());
    // largest pairs first: blocks start in index order, so the long ones do
    // not end up in the last wave
    std::stable_sort(bpairs.begin(), bpairs.end(), [&](int x, int y) {
        return c->h_prods[pairs[x].x].n_nd > c->h_prods[pairs[y].x].n_nd;
    });
    if (off > 0x7fffffffull) return fail(MORAP_ENOMEM, "evaluation batch too large");
    CKR(ensure_eval(c, pairs.size(), chunks.size(), off));
    const size_t npair = pairs.size(), nb = bpairs.size();
    const size_t up = npair * sizeof(int4) + chunks.size() * sizeof(int4) + nb * sizeof(int);
    CKR(stage(c, std::max(up, 2 * npair * sizeof(double) + npair * 4 + sizeof(LoopCtl) + 64)));
    if (npair) {
        char *h = (char *)c->h_stage;
        std::memcpy(h, pairs.data(), npair * sizeof(int4));
        std::memcpy(h + npair * sizeof(int4), chunks.data(), chunks.size() * sizeof(int4));
        std::memcpy(h + (npair + chunks.size()) * sizeof(int4), bpairs.data(), nb * sizeof(int));
        CK(cudaMemcpyAsync(c->d_epairs, h, npair * sizeof(int4), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(c->d_echunks, h + npair * sizeof(int4), chunks.size() * sizeof(int4),
                           cudaMemcpyHostToDevice, s));
        if (nb)
            CK(cudaMemcpyAsync(c->d_ebpairs, h + (npair + chunks.size()) * sizeof(int4), nb * sizeof(int),
                               cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemsetAsync(c->E[0], 0, off * sizeof(float4), s));
    CK(cudaMemsetAsync(c->E[1], 0, off * sizeof(float4), s));
    CK(cudaMemsetAsync(c->item_tmu, 0, chunks.size() * sizeof(uint32_t), s));
    CK(cudaMemsetAsync(c->pair_tmu, 0, std::max<size_t>(npair, 1) * sizeof(uint32_t), s));
    {
        EvalArgs ea = c->eargs;  // the scheduler layout of the last solve
        ea.Kp = c->Kp;
        CKL(launch_eval_compact(ea, (int)chunks.size(), s));
    }
    const unsigned int cap = (unsigned int)std::max(1, c->cfg.max_sweeps);
    CKL(launch_loop_init(c->ctl + 2, c->elist[0], (unsigned int)n_loop, c->eres, npair, c->esweeps, c->efrozen, cap,
                         s));
    CK(cudaEventRecord(c->ev[4], s));
    int launches = 3;
    if (nb) {
        // the loop checks its cap after every body of six sweeps
        if (!c->eval_block_ready) {
            CKL(eval_block_setup());
            c->eval_block_ready = true;
        }
        CKL(launch_eval_block(c->eargs, c->d_ebpairs, (int)nb, bmax, (cap + 5) / 6 * 6, s));
        launches += 1;
    }
    if (n_loop) {
        const EvalArgs ea = c->eargs;
        int rc = MORAP_OK;
        LoopGraph *ge = eval_graph(c, n_loop, rc);
        CKR(rc);
        const int grid = ge->grid;
        CKR(run_loop(
            c, *ge, c->ctl + 2, s, [&](int pos, cudaStream_t st) { return launch_eval_sweep(ea, pos, grid, st); },
            no_tail));
    }
    CK(cudaEventRecord(c->ev[5], s));
    CKL(launch_gather_eval(c->d_epairs, (int)npair, c->d_prods, c->E[0], c->d_rc, c->d_rp, s));
    // the D2H copies below land in the staging buffer the H2D copies above
    // read from; both are ordered on the same stream
    double *h = c->h_stage;
    uint8_t *hf = (uint8_t *)(h + 2 * npair);
    LoopCtl *hctl = (LoopCtl *)(((uintptr_t)(hf + npair) + 15) & ~uintptr_t(15));
    if (npair) {
        CK(cudaMemcpyAsync(h, c->d_rc, npair * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h + npair, c->d_rp, npair * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hf, c->efrozen, npair, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaMemcpyAsync(hctl, c->ctl + 2, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    rc.assign(h, h + npair);
    rp.assign(h + npair, h + 2 * npair);
    not_conv = 0;
    // a product without non-done states (every location of its task is
    // done) has nothing to evaluate (its values are 0): nothing can fail to
    // converge there
    for (size_t e = 0; e < npair; ++e) not_conv += hf[e] == 0 && c->h_prods[pairs[e].x].n_nd > 0;
    c->stats.eval_sweeps = (int32_t)std::max(n_loop ? hctl->sweep_base : 0u, hctl->block_sweeps);
    c->stats.updates_eval = (int64_t)hctl->updates;
    c->stats.bytes_eval = (int64_t)hctl->bytes;
    c->stats.ms_eval = ms_between(c->ev[4], c->ev[5]);
    c->stats.eval_pairs = (int32_t)npair;
    c->stats.h2d_bytes += (int64_t)((npair + chunks.size()) * sizeof(int4));
    c->stats.d2h_bytes += (int64_t)(npair * (2 * sizeof(double) + 1) + sizeof(LoopCtl));
    if (n_loop) launches += (int)hctl->sweep_base + (int)hctl->sweep_base / 6;
    c->stats.kernel_launches += launches;
    return MORAP_OK;
}

// Algorithm 4 for a list of (product, weight) pairs, in groups of at most
// kEvalStates value slots (one device loop per group), so the device buffers
// of an evaluation stay bounded however many pairs are asked for.
constexpr size_t kEvalStates = size_t(1) << 27;

int run_evaluation(morap_ctx *c, const std::vector<int4> &pairs, cudaStream_t s, std::vector<double> &rc,
                   std::vector<double> &rp, int &not_conv) {
    rc.clear();
    rp.clear();
    not_conv = 0;
    int32_t sweeps = 0, npairs = 0;
    int64_t updates = 0, bytes = 0;
    double ms = 0.0;
    size_t e0 = 0;
    do {
        size_t e1 = e0, states = 0;
        while (e1 < pairs.size() && (e1 == e0 || states + c->h_prods[pairs[e1].x].n_nd + 1 <= kEvalStates))
            states += c->h_prods[pairs[e1++].x].n_nd + 1;
        std::vector<int4> group(pairs.begin() + e0, pairs.begin() + e1);
        std::vector<double> grc, grp;
        int nc = 0;
        CKR(run_evaluation_group(c, group, s, grc, grp, nc));
        rc.insert(rc.end(), grc.begin(), grc.end());
        rp.insert(rp.end(), grp.begin(), grp.end());
        not_conv += nc;
        sweeps = std::max(sweeps, c->stats.eval_sweeps);
        updates += c->stats.updates_eval;
        bytes += c->stats.bytes_eval;
        ms += c->stats.ms_eval;
        npairs += c->stats.eval_pairs;
        e0 = e1;
    } while (e0 < pairs.size());
    c->stats.eval_sweeps = sweeps;
    c->stats.updates_eval = updates;
    c->stats.bytes_eval = bytes;
    c->stats.ms_eval = ms;
    c->stats.eval_pairs = npairs;
    return MORAP_OK;
}

}  // namespace

// Allocate, once, everything a batch of up to K weights needs (solve buffers,
// evaluation buffers for K x |J| assigned pairs of the largest products) and
// the loop graphs of every padded size up to K whose kernel shape needs no
// tuning, so that later batches of varying size neither allocate nor free
// (a device free synchronises the whole device).
// A context holding the products of several built contexts: every agent and
// task of each, and the pair list of each one's agent x task products (in
// order: context q's product a * |J_q| + t is product pair_off[q] + a * |J_q| + t).
// Built on the first context's device and configuration.
int morap::ctx_merge(morap_ctx *const *ctxs, int n, morap_ctx **out, std::vector<int32_t> &agent_off,
                     std::vector<int32_t> &task_off, std::vector<int32_t> &pair_off) {
    if (n < 1) return fail(MORAP_EINVAL, "merge: no context");
    morap_config cfg = ctxs[0]->cfg;
    cfg.alloc = nullptr;
    cfg.free = nullptr;
    cfg.alloc_user = nullptr;
    cfg.hbm_budget = 0;
    morap_ctx *m = nullptr;
    int rc = morap_ctx_create(&cfg, &m);
    if (rc != MORAP_OK) return rc;
    agent_off.assign(n, 0);
    task_off.assign(n, 0);
    pair_off.assign(n, 0);
    for (int q = 0; q < n; ++q) {
        const morap_ctx *c = ctxs[q];
        if (!c->sel_agent.empty()) {
            morap_ctx_destroy(m);
            return fail(MORAP_EINVAL, "merge: a context with a pair list");
        }
        agent_off[q] = (int32_t)m->agents.size();
        task_off[q] = (int32_t)m->tasks.size();
        pair_off[q] = (int32_t)m->sel_agent.size();
        for (size_t a = 0; a < c->agents.size(); ++a)
            for (size_t t = 0; t < c->tasks.size(); ++t) {
                m->sel_agent.push_back(agent_off[q] + (int32_t)a);
                m->sel_task.push_back(task_off[q] + (int32_t)t);
            }
        m->agents.insert(m->agents.end(), c->agents.begin(), c->agents.end());
        m->tasks.insert(m->tasks.end(), c->tasks.begin(), c->tasks.end());
    }
    if ((rc = morap_build(m, nullptr, nullptr)) != MORAP_OK) {
        morap_ctx_destroy(m);
        return rc;
    }
    *out = m;
    return MORAP_OK;
}

// The serving workers run several sweep loops on one GPU at once, where the
// cooperative tail launches of two loops could each hold part of the GPU
// while waiting for the rest: their contexts run every sweep as its own
// launch.  Graphs built with a tail are rebuilt without it.
int morap::ctx_no_tail(morap_ctx *c) {
    c->cfg.tail_items = 0;
    for (int i = 0; i < 7; ++i) {
        if (c->g32[i].variant >= 0 && c->g32[i].tail > 0)
            CKR(build_phase_graph(c, c->g32[i], kSweepF32, 1 << i, c->g32[i].variant));
        if (c->g64[i].variant >= 0 && c->g64[i].tail > 0)
            CKR(build_phase_graph(c, c->g64[i], c->polish, 1 << i, c->g64[i].variant));
    }
    return MORAP_OK;
}

// What decides a context's arithmetic (precision path and stopping rules):
// contexts with equal keys give the same results for the same product.
std::string morap::ctx_arith_key(const morap_ctx *c) {
    const morap_config &f = c->cfg;
    const bool fp32 = c->all_free_action && f.precision == MORAP_PREC_MIXED;
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%d/%d/%a/%a/%a/%d/%d/%d/%d", fp32 ? 1 : 0, f.polish, f.eps_vi, f.eps_eval,
                  f.tau_policy, f.max_sweeps, f.in_place, f.eval_block, f.device);
    return buf;
}

// The largest product (states, done slot included) of a built context.
int64_t morap::ctx_max_states(const morap_ctx *c) {
    int64_t m = 0;
    for (const ProdDesc &pd : c->h_prods) m = std::max<int64_t>(m, (int64_t)pd.n_nd + 1);
    return m;
}

int morap::ctx_reserve(morap_ctx *c, int K) {
    if (!c->built) return fail(MORAP_ESTATE, "reserve before build");
    CK(cudaSetDevice(c->cfg.device));
    const int Kp = next_pow2(std::max(1, std::min(K, 64)));
    const int old_Kp = c->Kp;
    const bool grow = Kp > c->Kcap;
    CKR(ensure_solve(c, Kp));
    size_t states = 0, chunks = 0;
    // the evaluation buffers are sized for one assignment per weight; a
    // context with a pair list has no fixed assignment shape (they grow on demand)
    for (int j = 0; j < c->nJ && c->sel_agent.empty(); ++j) {
        uint32_t mx = 0;
        for (int i = 0; i < c->nI; ++i) mx = std::max(mx, c->h_prods[(size_t)i * c->nJ + j].n_nd);
        states += mx + 1;
        chunks += (mx + kEvalChunk - 1) / kEvalChunk;
    }
    if (c->sel_agent.empty())
        CKR(ensure_eval(c, (size_t)Kp * c->nJ, (size_t)Kp * chunks, (size_t)Kp * std::min<size_t>(states, kEvalStates)));
    for (int kp = 1; kp <= Kp; kp *= 2)
        for (int f = 0; f < 2; ++f) {
            if (f == 0 && !c->V32[0]) continue;
            bool tune = false;
            CKR(prepare_phase(c, f == 1 ? (c->V32[0] ? c->polish : kSweepDF) : kSweepF32, kp, tune));  // shapes that
            // need tuning are left to the first solve
        }
    if (!grow) c->Kp = old_Kp;
    return MORAP_OK;
}

namespace {

int supporting_batch(morap_ctx *c, int K, const double *W, cudaStream_t s, double *r_out, int32_t *assign_out,
                     double *c_out) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    std::vector<double> hc;
    std::vector<int32_t> hs;
    CKR(run_optimisation(c, K, W, s, hc, hs));
    const auto t1 = clk::now();
    const int Kp = c->Kp, nI = c->nI, nJ = c->nJ;
    std::vector<double> Cm((size_t)nI * nJ);
    std::vector<int4> pairs;
    std::vector<int> assign((size_t)K * nJ, -1);
    for (int k = 0; k < K; ++k) {
        for (int p = 0; p < nI * nJ; ++p) Cm[p] = hc[(size_t)p * Kp + k];
        assign_tasks(nI, nJ, Cm.data(), assign.data() + (size_t)k * nJ);
        for (int j = 0; j < nJ; ++j) {
            const int i = assign[(size_t)k * nJ + j];
            if (i >= 0) pairs.push_back(make_int4(i * nJ + j, k, 0, 0));
        }
    }
    const auto t2 = clk::now();
    std::vector<double> rc, rp;
    int nc = 0;
    CKR(run_evaluation(c, pairs, s, rc, rp, nc));
    const auto t3 = clk::now();
    const int nobj = nI + nJ;
    for (int k = 0; k < K; ++k)
        for (int i = 0; i < nobj; ++i) r_out[(size_t)k * nobj + i] = 0.0;
    for (size_t e = 0; e < pairs.size(); ++e) {
        const int p = pairs[e].x, k = pairs[e].y, i = p / nJ, j = p % nJ;
        r_out[(size_t)k * nobj + i] = rc[e];
        r_out[(size_t)k * nobj + nI + j] = rp[e];
    }
    if (assign_out) std::copy(assign.begin(), assign.end(), assign_out);
    if (c_out)
        for (int k = 0; k < K; ++k)
            for (int p = 0; p < c->P; ++p) c_out[(size_t)k * c->P + p] = hc[(size_t)p * Kp + k];
    c->last_assign = assign;
    auto ms = [](clk::duration d) { return std::chrono::duration<double, std::milli>(d).count(); };
    c->stats.ms_host = ms(t2 - t1);
    c->stats.ms_total = ms(t3 - t0);
    c->stats.pairs_not_converged += nc;
    for (int32_t st : hs)
        if (st != MORAP_OK) return fail(MORAP_ENOTCONV, "a (product, weight) pair reached the sweep cap");
    if (nc) return fail(MORAP_ENOTCONV, "an evaluation reached the sweep cap");
    return MORAP_OK;
}

int validate_agent(int32_t n, int32_t s0, const int32_t *state_ptr, const int32_t *sa_ptr, const int32_t *succ,
                   const double *prob, const double *cost, const int32_t *label_ptr, const int32_t *label_ap,
                   HostAgent &A) {
    if (n < 1) return fail(MORAP_EINVAL, "agent: n_states must be >= 1");
    if (s0 < 0 || s0 >= n) return fail(MORAP_EINVAL, "agent: s0 out of range");
    if (!state_ptr || !sa_ptr || !succ || !prob || !cost || !label_ptr)
        return fail(MORAP_EINVAL, "agent: null array");
    if (state_ptr[0] != 0) return fail(MORAP_EINVAL, "agent: state_ptr[0] must be 0");
    for (int s = 0; s < n; ++s)
        if (state_ptr[s + 1] <= state_ptr[s])
            return fail(MORAP_EINVAL, "agent: state " + std::to_string(s) + " has no enabled action");
    const int32_t SA = state_ptr[n];
    if (SA > 255 * n) return fail(MORAP_EINVAL, "agent: at most 255 actions per state");
    for (int s = 0; s < n; ++s)
        if (state_ptr[s + 1] - state_ptr[s] > 255)
            return fail(MORAP_EINVAL, "agent: state " + std::to_string(s) + " has more than 255 actions");
    if (sa_ptr[0] != 0) return fail(MORAP_EINVAL, "agent: sa_ptr[0] must be 0");
    A = HostAgent();
    A.n_states = n;
    A.s0 = s0;
    A.state_ptr.assign(state_ptr, state_ptr + n + 1);
    A.sa_ptr.push_back(0);
    A.free_action_everywhere = true;
    std::vector<std::pair<int32_t, double>> row;
    for (int s = 0; s < n; ++s) {
        bool free_here = false;
        for (int32_t a = state_ptr[s]; a < state_ptr[s + 1]; ++a) {
            if (sa_ptr[a + 1] < sa_ptr[a])
                return fail(MORAP_EINVAL, "agent: sa_ptr not monotone at row " + std::to_string(a));
            if (!std::isfinite(cost[a]) || cost[a] < 0.0)
                return fail(MORAP_EINVAL, "agent: cost of row " + std::to_string(a) + " must be finite and >= 0");
            row.clear();
            double sum = 0.0;
            for (int32_t t = sa_ptr[a]; t < sa_ptr[a + 1]; ++t) {
                if (succ[t] < 0 || succ[t] >= n)
                    return fail(MORAP_EINVAL, "agent: successor out of range in row " + std::to_string(a));
                if (!(prob[t] >= 0.0) || !std::isfinite(prob[t]))
                    return fail(MORAP_EINVAL, "agent: probability out of range in row " + std::to_string(a));
                sum += prob[t];
                if (prob[t] > 0.0) row.emplace_back(succ[t], prob[t]);
            }
            if (std::fabs(sum - 1.0) > 1e-9)
                return fail(MORAP_EINVAL, "agent: row " + std::to_string(a) + " sums to " + std::to_string(sum) +
                                              " (actions must be enabled, Sec. 2)");
            std::sort(row.begin(), row.end());
            for (size_t k = 0; k < row.size(); ++k) {
                if (k > 0 && row[k].first == A.succ.back()) {
                    A.prob.back() += row[k].second;
                } else {
                    A.succ.push_back(row[k].first);
                    A.prob.push_back(row[k].second);
                }
            }
            A.sa_ptr.push_back((int32_t)A.succ.size());
            A.cost.push_back(cost[a]);
            if (cost[a] == 0.0) free_here = true;
        }
        if (!free_here) A.free_action_everywhere = false;
    }
    if (label_ptr[0] != 0) return fail(MORAP_EINVAL, "agent: label_ptr[0] must be 0");
    for (int s = 0; s < n; ++s)
        if (label_ptr[s + 1] < label_ptr[s]) return fail(MORAP_EINVAL, "agent: label_ptr not monotone");
    if (label_ptr[n] > 0 && !label_ap) return fail(MORAP_EINVAL, "agent: null label_ap");
    A.label_ptr.assign(label_ptr, label_ptr + n + 1);
    if (label_ptr[n] > 0) A.label_ap.assign(label_ap, label_ap + label_ptr[n]);
    return MORAP_OK;
}

// Product construction K-B0 from the resident model arrays: letters, the
// merged row counts, the rows' transition offsets, then the CSR itself.
int run_construction(morap_ctx *c, cudaStream_t s, bool letters_and_counts = true) {
    if (letters_and_counts) {
        CKL(launch_letters(c->d_prods, c->P, c->d_ad, c->d_td, c->d_lp, c->d_la, c->d_ap, c->d_letters, c->max_S,
                           s));
        CKL(launch_row_count(c->d_prods, c->P, c->d_ad, c->d_td, c->d_sap, c->d_succ, c->d_letters, c->d_nd,
                             c->row_cnt, nullptr, c->max_rows, s));
    }
    CKL(launch_row_offsets(c->d_prods, c->P, c->row_cnt, c->sa_tr, s));
    CKL(launch_build(c->d_prods, c->P, c->d_ad, c->d_td, c->d_sp, c->d_sap, c->d_succ, c->d_prob, c->d_cost,
                     c->d_letters, c->d_nd, c->state_sa, c->state_tr, c->sa_tr, c->col, c->cp32, c->p64, c->pdf,
                     c->cost32, c->cost64, c->costdf, c->TS, c->TSA, c->TT, c->max_work, s));
    CKL(launch_item_inputs(c->d_chunks, (int)c->h_chunks.size(), c->d_prods, c->state_tr, c->col, c->in_items, c->item_w,
                                c->state_sa, s));
    return MORAP_OK;
}

// The FP64 probabilities and costs of the product CSRs, which only the plain
// baseline and morap_product_download read: allocated and filled by a
// construction pass on first use, then kept up to date by every rebuild.
int ensure_fp64_csr(morap_ctx *c, cudaStream_t s) {
    if (c->p64) return MORAP_OK;
    auto &L = c->build_allocs;
    CKR(dev_alloc(c, L, &c->p64, std::max<uint64_t>(c->TT, 1) * 8));
    CKR(dev_alloc(c, L, &c->cost64, std::max<uint64_t>(c->TSA, 1) * 8));
    c->csr_bytes += (int64_t)8 * c->TT + (int64_t)8 * c->TSA;
    CKR(run_construction(c, s, false));
    CK(cudaStreamSynchronize(s));
    return MORAP_OK;
}

int do_build(morap_ctx *c, cudaStream_t s, morap_footprint *fp) {
    if (c->agents.empty() || c->tasks.empty()) return fail(MORAP_ESTATE, "build: add at least one agent and one task");
    const int nI = (int)c->agents.size(), nJ = (int)c->tasks.size();
    const bool selected = !c->sel_agent.empty();
    const int P = selected ? (int)c->sel_agent.size() : nI * nJ;
    for (size_t e = 0; e < c->sel_agent.size(); ++e)
        if (c->sel_agent[e] >= nI || c->sel_task[e] >= nJ)
            return fail(MORAP_EINVAL, "build: selected pair " + std::to_string(e) + " names an agent or task not added");
    // host-side descriptors
    std::vector<AgentDesc> ad(nI);
    std::vector<int32_t> a_sp, a_sap, a_succ, a_lp, a_la;
    std::vector<double> a_prob, a_cost;
    uint32_t max_S = 1;
    int max_row_new = 1;
    bool all_free = true;
    for (int i = 0; i < nI; ++i) {
        const HostAgent &A = c->agents[i];
        AgentDesc &d = ad[i];
        d.sp_off = (uint32_t)a_sp.size();
        d.sap_off = (uint32_t)a_sap.size();
        d.cost_off = (uint32_t)a_cost.size();
        d.tr_off = (uint32_t)a_succ.size();
        d.lp_off = (uint32_t)a_lp.size();
        d.la_off = (uint32_t)a_la.size();
        d.S = (uint32_t)A.n_states;
        d.SA = (uint32_t)A.cost.size();
        d.T = (uint32_t)A.succ.size();
        d.s0 = A.s0;
        a_sp.insert(a_sp.end(), A.state_ptr.begin(), A.state_ptr.end());
        a_sap.insert(a_sap.end(), A.sa_ptr.begin(), A.sa_ptr.end());
        a_cost.insert(a_cost.end(), A.cost.begin(), A.cost.end());
        a_succ.insert(a_succ.end(), A.succ.begin(), A.succ.end());
        a_prob.insert(a_prob.end(), A.prob.begin(), A.prob.end());
        a_lp.insert(a_lp.end(), A.label_ptr.begin(), A.label_ptr.end());
        a_la.insert(a_la.end(), A.label_ap.begin(), A.label_ap.end());
        max_S = std::max(max_S, d.S);
        all_free = all_free && A.free_action_everywhere;
        for (size_t r = 0; r + 1 < A.sa_ptr.size(); ++r) max_row_new = std::max(max_row_new, A.sa_ptr[r + 1] - A.sa_ptr[r]);
    }
    std::vector<TaskDesc> td(nJ);
    std::vector<int16_t> nd_delta;
    std::vector<int32_t> ap_ids;
    for (int j = 0; j < nJ; ++j) {
        const HostTask &T = c->tasks[j];
        TaskDesc &d = td[j];
        d.delta_off = (uint32_t)nd_delta.size();
        d.ap_off = (uint32_t)ap_ids.size();
        d.n_ap = T.n_ap;
        d.n_letters = T.n_letters;
        d.Qn = T.n_nd;
        d.n_pre = T.n_pre;
        d.q0_ploc = T.ploc[T.q0];
        nd_delta.insert(nd_delta.end(), T.nd_delta.begin(), T.nd_delta.end());
        ap_ids.insert(ap_ids.end(), T.ap_ids.begin(), T.ap_ids.end());
    }
    if (ap_ids.empty()) ap_ids.push_back(0);
    if (nd_delta.empty()) nd_delta.push_back(-1);
    if (a_la.empty()) a_la.push_back(0);
    std::vector<ProdDesc> prods(P);
    std::vector<int4> chunks;
    uint64_t TS = 0, TSA = 0, TT = 0, letters = 0, max_work = 1, max_rows = 1;
    for (int p = 0; p < P; ++p) {
            const int i = selected ? c->sel_agent[p] : p / nJ, j = selected ? c->sel_task[p] : p % nJ;
            ProdDesc &pd = prods[p];
            const AgentDesc &a = ad[i];
            const TaskDesc &t = td[j];
            pd.agent = i;
            pd.task = j;
            pd.S = a.S;
            pd.SA = a.SA;
            pd.T = a.T;
            pd.Qn = t.Qn;
            pd.n_nd = (uint32_t)t.Qn * a.S;
            pd.pre_begin = (uint32_t)(t.Qn - t.n_pre) * a.S;
            pd.init_local = t.q0_ploc >= 0 ? t.q0_ploc * (int32_t)a.S + a.s0 : (int32_t)pd.n_nd;
            pd.state_off = (uint32_t)TS;
            pd.sa_off = (uint32_t)TSA;
            pd.tr_off = (uint32_t)TT;
            pd.letter_off = (uint32_t)letters;
            pd.item_off = (uint32_t)chunks.size();
            TS += (uint64_t)pd.n_nd + 1;
            TSA += (uint64_t)t.Qn * a.SA;
            TT += (uint64_t)t.Qn * a.T;
            letters += a.S;
            max_work = std::max<uint64_t>(max_work, (uint64_t)t.Qn * a.T + 1);
            max_rows = std::max<uint64_t>(max_rows, (uint64_t)t.Qn * a.SA);
            if (TS >= 0x7fffffffull || TSA >= 0xffffffffull || TT >= 0xffffffffull)
                return fail(MORAP_ENOMEM, "products exceed the 32-bit index range of one context");
            for (uint32_t b = 0; b < pd.n_nd; b += kChunk)
                chunks.push_back(make_int4(p, (int)b, (int)std::min<uint32_t>(pd.n_nd, b + kChunk), b == 0));
        }
    // Same layout as the resident one: refill in place and keep the solve
    // buffers and their graphs.
    std::vector<size_t> sig = {(size_t)nI, (size_t)nJ, (size_t)TS, (size_t)TSA, (size_t)TT, a_sp.size(),
                               a_sap.size(), a_succ.size(), a_lp.size(), a_la.size(), ap_ids.size(),
                               nd_delta.size(), (size_t)letters, chunks.size(), (size_t)all_free,
                               (size_t)max_row_new};
    const bool reuse = c->built && sig == c->layout_sig &&
                       std::memcmp(prods.data(), c->h_prods_key.data(), P * sizeof(ProdDesc)) == 0;
    if (!reuse) {
        free_eval(c);
        free_solve(c);
        dev_free_list(c, c->build_allocs);
        c->built = false;
        c->nI = nI;
        c->nJ = nJ;
        c->P = P;
        c->h_prods = prods;
        c->h_prods_key = prods;
        c->h_chunks = chunks;
        c->TS = (uint32_t)TS;
        c->TSA = (uint32_t)TSA;
        c->TT = (uint32_t)TT;  // the unmerged count until the row counts are in
        c->max_S = max_S;
        c->max_work = (uint32_t)std::min<uint64_t>(max_work, 0xffffffffull);
        c->max_rows = (uint32_t)std::min<uint64_t>(max_rows, 0xffffffffull);
        c->all_free_action = all_free;
        c->max_row = max_row_new;
        auto &L = c->build_allocs;
        CKR(dev_alloc(c, L, &c->state_sa, (TS + 1) * 4));
        CKR(dev_alloc(c, L, &c->state_tr, (TS + 1) * 4));
        CKR(dev_alloc(c, L, &c->sa_tr, (TSA + 1) * 4));
        CKR(dev_alloc(c, L, &c->row_cnt, std::max<uint64_t>(TSA, 1) * 4));
        CKR(dev_alloc(c, L, &c->prod_tr, (size_t)P * 4));
        CKR(dev_alloc(c, L, &c->costdf, std::max<uint64_t>(TSA, 1) * 8));
        CKR(dev_alloc(c, L, &c->cost32, std::max<uint64_t>(TSA, 1) * 4));
        c->cost64 = nullptr;  // FP64 copies (plain baseline, downloads) on first use: ensure_fp64_csr
        c->p64 = nullptr;
        CKR(dev_alloc(c, L, &c->d_prods, P * sizeof(ProdDesc)));
        CKR(dev_alloc(c, L, &c->d_chunks, std::max<size_t>(chunks.size(), 1) * sizeof(int4)));
        CKR(dev_alloc(c, L, &c->d_chunk_u, std::max<size_t>(chunks.size(), 1) * sizeof(uint4)));
        CKR(dev_alloc(c, L, &c->in_items, std::max<size_t>(chunks.size(), 1) * kInItems * sizeof(int32_t)));
        CKR(dev_alloc(c, L, &c->item_w, std::max<size_t>(chunks.size(), 1) * sizeof(uint2)));
        for (int q = 0; q < 3; ++q) CKR(dev_alloc(c, L, &c->chg[q], std::max<size_t>(chunks.size(), 1)));
        CKR(dev_alloc(c, L, &c->d_ad, nI * sizeof(AgentDesc)));
        CKR(dev_alloc(c, L, &c->d_td, nJ * sizeof(TaskDesc)));
        CKR(dev_alloc(c, L, &c->d_sp, a_sp.size() * 4));
        CKR(dev_alloc(c, L, &c->d_sap, a_sap.size() * 4));
        CKR(dev_alloc(c, L, &c->d_succ, std::max<size_t>(a_succ.size(), 1) * 4));
        CKR(dev_alloc(c, L, &c->d_prob, std::max<size_t>(a_prob.size(), 1) * 8));
        CKR(dev_alloc(c, L, &c->d_cost, std::max<size_t>(a_cost.size(), 1) * 8));
        CKR(dev_alloc(c, L, &c->d_lp, a_lp.size() * 4));
        CKR(dev_alloc(c, L, &c->d_la, a_la.size() * 4));
        CKR(dev_alloc(c, L, &c->d_ap, ap_ids.size() * 4));
        CKR(dev_alloc(c, L, &c->d_nd, nd_delta.size() * 2));
        CKR(dev_alloc(c, L, &c->d_letters, std::max<uint64_t>(letters, 1)));
    }
    auto up = [&](void *dst, const void *src, size_t bytes) -> int {
        if (bytes) CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
        return MORAP_OK;
    };
    size_t h2d = 0;
    auto upc = [&](void *dst, const void *src, size_t bytes) -> int {
        h2d += bytes;
        return up(dst, src, bytes);
    };
    CKR(upc(c->d_prods, prods.data(), P * sizeof(ProdDesc)));
    CKR(upc(c->d_chunks, chunks.data(), chunks.size() * sizeof(int4)));
    {
        std::vector<uint4> cu(chunks.size());
        for (size_t q = 0; q < chunks.size(); ++q) {
            const ProdDesc &pd = prods[chunks[q].x];
            cu[q] = make_uint4(pd.state_off + (uint32_t)chunks[q].y, pd.state_off + (uint32_t)chunks[q].z,
                               pd.state_off + pd.pre_begin, 0u);
        }
        CKR(upc(c->d_chunk_u, cu.data(), cu.size() * sizeof(uint4)));
    }
    CKR(upc(c->d_ad, ad.data(), nI * sizeof(AgentDesc)));
    CKR(upc(c->d_td, td.data(), nJ * sizeof(TaskDesc)));
    CKR(upc(c->d_sp, a_sp.data(), a_sp.size() * 4));
    CKR(upc(c->d_sap, a_sap.data(), a_sap.size() * 4));
    CKR(upc(c->d_succ, a_succ.data(), a_succ.size() * 4));
    CKR(upc(c->d_prob, a_prob.data(), a_prob.size() * 8));
    CKR(upc(c->d_cost, a_cost.data(), a_cost.size() * 8));
    CKR(upc(c->d_lp, a_lp.data(), a_lp.size() * 4));
    CKR(upc(c->d_la, a_la.data(), a_la.size() * 4));
    CKR(upc(c->d_ap, ap_ids.data(), ap_ids.size() * 4));
    CKR(upc(c->d_nd, nd_delta.data(), nd_delta.size() * 2));
    // first pass: the merged transition count of every row and product, then
    // each product's transition offset and the total (one read-back)
    CKL(launch_letters(c->d_prods, c->P, c->d_ad, c->d_td, c->d_lp, c->d_la, c->d_ap, c->d_letters, c->max_S, s));
    CK(cudaMemsetAsync(c->prod_tr, 0, (size_t)P * 4, s));
    CKL(launch_row_count(c->d_prods, c->P, c->d_ad, c->d_td, c->d_sap, c->d_succ, c->d_letters, c->d_nd, c->row_cnt,
                         c->prod_tr, c->max_rows, s));
    std::vector<uint32_t> ptr_count(P);
    CK(cudaMemcpyAsync(ptr_count.data(), c->prod_tr, (size_t)P * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    uint64_t TTm = 0;
    std::vector<ProdDesc> merged = prods;
    for (int p = 0; p < P; ++p) {
        merged[p].tr_off = (uint32_t)TTm;
        merged[p].n_tr = ptr_count[p];
        TTm += ptr_count[p];
    }
    if (reuse && TTm != c->TT) return fail(MORAP_ECUDA, "build: the merged transition count changed on a rebuild");
    if (!reuse) {
        auto &L = c->build_allocs;
        c->TT = (uint32_t)TTm;
        CKR(dev_alloc(c, L, &c->col, std::max<uint64_t>(TTm, 1) * 4));
        CKR(dev_alloc(c, L, &c->cp32, std::max<uint64_t>(TTm, 1) * 8));
        CKR(dev_alloc(c, L, &c->pdf, std::max<uint64_t>(TTm, 1) * 8));
        // state starts (x2), row starts, col, cp32, pdf; cost32, costdf
        c->csr_bytes = (int64_t)(8 * (TS + 1) + 4 * (TSA + 1) + 4 * TTm + 8 * TTm + 8 * TTm + 4 * TSA + 8 * TSA);
        c->layout_sig = sig;
    }
    c->h_prods = merged;
    CKR(upc(c->d_prods, merged.data(), P * sizeof(ProdDesc)));
    CKR(run_construction(c, s, false));
    CK(cudaStreamSynchronize(s));  // the host vectors above go out of scope
    TT = c->TT;
    c->built = true;
    c->last_h2d_bytes = (int64_t)h2d;
    if (fp) {
        fp->n_products = P;
        fp->n_states = (int64_t)TS;
        fp->n_sa = (int64_t)TSA;
        fp->n_trans = (int64_t)TT;
        fp->csr_bytes = c->csr_bytes;
        fp->device_bytes = (int64_t)c->device_bytes;
        fp->h2d_bytes = (int64_t)h2d;
    }
    return MORAP_OK;
}


}  // namespace

// =================================================================== C-ABI

#define API_BEGIN try {
#define API_END                                                          \
    }                                                                    \
    catch (const std::bad_alloc &) {                                     \
        return fail(MORAP_ENOMEM, "host allocation failed");             \
    }                                                                    \
    catch (const std::exception &ex) {                                   \
        return fail(MORAP_EINVAL, std::string("internal: ") + ex.what()); \
    }

extern "C" {

void morap_config_default(morap_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->eps_vi = 1e-8;
    cfg->eps_eval = 1e-11;
    cfg->tau_policy = 1e-9;
    cfg->max_sweeps = 100000;
    cfg->precision = MORAP_PREC_MIXED;
    cfg->device = 0;
    cfg->sweep_variant_fp32 = -1;
    cfg->sweep_variant_fp64 = -1;
    cfg->skip_unchanged = 1;
    cfg->polish = 0;
    cfg->eval_block = 1;
    cfg->in_place = 0;
    cfg->item_warps_max = 0;
    cfg->tail_items = -1;
}

const char *morap_last_error(void) { return g_last_error.c_str(); }

int morap_barrier_selfcheck(int32_t device, int32_t *timed_out, double *ms) {
    API_BEGIN
    if (!timed_out || !ms) return fail(MORAP_EINVAL, "barrier selfcheck: NULL output");
    CK(cudaSetDevice(device));
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    LoopCtl *d = nullptr;
    CK(cudaMalloc(&d, sizeof(LoopCtl)));
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(LoopCtl), s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = (cudaError_t)launch_barrier_selfcheck(d, std::max(2, sms), s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    LoopCtl h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(d);
    if (e != cudaSuccess) return fail(MORAP_ECUDA, std::string("barrier selfcheck: ") + cudaGetErrorString(e));
    *timed_out = h.bar_err ? 1 : 0;
    *ms = (double)t;
    return MORAP_OK;
    API_END
}

int morap_ctx_create(const morap_config *cfg, morap_ctx **out) {
    API_BEGIN
    if (!out) return fail(MORAP_EINVAL, "out is NULL");
    *out = nullptr;
    morap_config c;
    if (cfg)
        c = *cfg;
    else
        morap_config_default(&c);
    if (!(c.eps_vi > 0) || !(c.eps_eval > 0) || !(c.tau_policy >= 0) || c.max_sweeps < 1)
        return fail(MORAP_EINVAL, "config: eps_vi, eps_eval > 0, tau_policy >= 0, max_sweeps >= 1 required");
    if (c.precision != MORAP_PREC_MIXED && c.precision != MORAP_PREC_FP64)
        return fail(MORAP_EINVAL, "config: unknown precision mode");
    if (c.launch_mode != 0 && c.launch_mode != 1) return fail(MORAP_EINVAL, "config: unknown launch mode");
    if ((c.alloc == nullptr) != (c.free == nullptr)) return fail(MORAP_EINVAL, "config: alloc and free go together");
    if (c.sweep_variant_fp32 < -1 || c.sweep_variant_fp32 >= sweep_variant_count(kSweepF32) ||
        c.sweep_variant_fp64 < -1 ||
        c.sweep_variant_fp64 >= std::max(sweep_variant_count(kSweepDF), sweep_variant_count(kSweepDelta)))
        return fail(MORAP_EINVAL, "config: sweep_variant_* must be -1 (tuned) or a shape index");
    if (c.polish != 0 && c.polish != 1) return fail(MORAP_EINVAL, "config: polish must be 0 or 1");
    if (c.eval_block != 0 && c.eval_block != 1) return fail(MORAP_EINVAL, "config: eval_block must be 0 or 1");
    if (c.in_place != 0 && c.in_place != 1) return fail(MORAP_EINVAL, "config: in_place must be 0 or 1");
    if (c.item_warps_max != 0 && c.item_warps_max != 1 && c.item_warps_max != 2 && c.item_warps_max != 4 &&
        c.item_warps_max != 8)
        return fail(MORAP_EINVAL, "config: item_warps_max must be 0, 1, 2, 4 or 8");
    if (c.skip_unchanged != 0 && c.skip_unchanged != 1)
        return fail(MORAP_EINVAL, "config: skip_unchanged must be 0 or 1");
    if (c.tail_items < -1) return fail(MORAP_EINVAL, "config: tail_items must be -1 (automatic), 0 (off) or > 0");
    CK(cudaSetDevice(c.device));
    morap_ctx *ctx = new morap_ctx();
    ctx->cfg = c;
    cudaError_t e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, c.device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
    if (e != cudaSuccess) {
        morap_ctx_destroy(ctx);
        return fail(MORAP_ECUDA, std::string("context setup: ") + cudaGetErrorString(e));
    }
    *out = ctx;
    return MORAP_OK;
    API_END
}

int morap_ctx_destroy(morap_ctx *ctx) {
    if (!ctx) return MORAP_OK;
    cudaSetDevice(ctx->cfg.device);
    cudaDeviceSynchronize();
    free_eval(ctx);
    free_solve(ctx);
    dev_free_list(ctx, ctx->build_allocs);
    for (auto &a : ctx->allocs) {
        if (ctx->cfg.free)
            ctx->cfg.free(a.ptr, a.bytes, ctx->cfg.alloc_user);
        else
            cudaFree(a.ptr);
    }
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
    return MORAP_OK;
}

int morap_add_agent(morap_ctx *ctx, int32_t n_states, int32_t s0, const int32_t *state_ptr, const int32_t *sa_ptr,
                    const int32_t *succ, const double *prob, const double *cost, const int32_t *label_ptr,
                    const int32_t *label_ap, int32_t *agent_id) {
    API_BEGIN
    if (!ctx) return fail(MORAP_EINVAL, "ctx is NULL");
    if (ctx->built) return fail(MORAP_ESTATE, "add_agent after build");
    HostAgent A;
    CKR(validate_agent(n_states, s0, state_ptr, sa_ptr, succ, prob, cost, label_ptr, label_ap, A));
    ctx->agents.push_back(std::move(A));
    if (agent_id) *agent_id = (int32_t)ctx->agents.size() - 1;
    return MORAP_OK;
    API_END
}

int morap_add_task(morap_ctx *ctx, int32_t n_locs, int32_t q0, int32_t n_ap, const int32_t *ap_ids,
                   const int32_t *delta, const uint8_t *accepting, int32_t *task_id) {
    API_BEGIN
    if (!ctx) return fail(MORAP_EINVAL, "ctx is NULL");
    if (ctx->built) return fail(MORAP_ESTATE, "add_task after build");
    HostTask T;
    CKR(preprocess_task(n_locs, q0, n_ap, ap_ids, delta, accepting, T));
    ctx->tasks.push_back(std::move(T));
    if (task_id) *task_id = (int32_t)ctx->tasks.size() - 1;
    return MORAP_OK;
    API_END
}

int morap_select_pairs(morap_ctx *ctx, int32_t n_pairs, const int32_t *agent, const int32_t *task) {
    API_BEGIN
    if (!ctx) return fail(MORAP_EINVAL, "ctx is NULL");
    if (ctx->built) return fail(MORAP_ESTATE, "select_pairs after build");
    if (n_pairs < 0 || (n_pairs > 0 && (!agent || !task))) return fail(MORAP_EINVAL, "bad argument");
    std::vector<int64_t> keys((size_t)n_pairs);
    for (int e = 0; e < n_pairs; ++e) {
        if (agent[e] < 0 || task[e] < 0) return fail(MORAP_EINVAL, "negative agent or task index");
        keys[e] = ((int64_t)agent[e] << 32) | (int64_t)task[e];
    }
    std::sort(keys.begin(), keys.end());
    if (std::adjacent_find(keys.begin(), keys.end()) != keys.end()) return fail(MORAP_EINVAL, "a pair is listed twice");
    ctx->sel_agent.assign(agent, agent + n_pairs);
    ctx->sel_task.assign(task, task + n_pairs);
    return MORAP_OK;
    API_END
}

int morap_build(morap_ctx *ctx, void *stream, morap_footprint *fp) {
    API_BEGIN
    if (!ctx) return fail(MORAP_EINVAL, "ctx is NULL");
    CK(cudaSetDevice(ctx->cfg.device));
    return do_build(ctx, (cudaStream_t)stream, fp);
    API_END
}

int morap_rebuild(morap_ctx *ctx, void *stream) {
    API_BEGIN
    if (!ctx) return fail(MORAP_EINVAL, "ctx is NULL");
    if (!ctx->built) return fail(MORAP_ESTATE, "rebuild before build");
    CK(cudaSetDevice(ctx->cfg.device));
    CKR(run_construction(ctx, (cudaStream_t)stream));
    return MORAP_OK;
    API_END
}

int morap_solve(morap_ctx *ctx, int32_t K, const double *W, void *stream, double *c_out, double *rcost_out,
                double *rprob_out, int32_t *status_out) {
    API_BEGIN
    if (!ctx || !W || !c_out) return fail(MORAP_EINVAL, "null argument");
    if (!ctx->built) return fail(MORAP_ESTATE, "solve before build");
    if (K < 1) return fail(MORAP_EINVAL, "K must be >= 1");
    CK(cudaSetDevice(ctx->cfg.device));
    CKR(check_weights(ctx, K, W));
    cudaStream_t s = (cudaStream_t)stream;
    const int nobj = ctx->nI + ctx->nJ;
    bool any_bad = false;
    for (int k0 = 0; k0 < K; k0 += 64) {
        const int kb = std::min(64, K - k0);
        std::vector<double> hc;
        std::vector<int32_t> hs;
        CKR(run_optimisation(ctx, kb, W + (size_t)k0 * nobj, s, hc, hs));
        const int Kp = ctx->Kp;
        for (int k = 0; k < kb; ++k)
            for (int p = 0; p < ctx->P; ++p) {
                c_out[(size_t)(k0 + k) * ctx->P + p] = hc[(size_t)p * Kp + k];
                if (status_out) status_out[(size_t)(k0 + k) * ctx->P + p] = hs[(size_t)p * Kp + k];
                any_bad = any_bad || hs[(size_t)p * Kp + k] != MORAP_OK;
            }
        if (rcost_out || rprob_out) {
            std::vector<int4> pairs;
            for (int k = 0; k < kb; ++k)
                for (int p = 0; p < ctx->P; ++p) pairs.push_back(make_int4(p, k, 0, 0));
            std::vector<double> rc, rp;
            int nc = 0;
            CKR(run_evaluation(ctx, pairs, s, rc, rp, nc));
            for (size_t e = 0; e < pairs.size(); ++e) {
                const size_t o = (size_t)(k0 + pairs[e].y) * ctx->P + pairs[e].x;
                if (rcost_out) rcost_out[o] = rc[e];
                if (rprob_out) rprob_out[o] = rp[e];
            }
            any_bad = any_bad || nc > 0;
        }
    }
    if (any_bad) return fail(MORAP_ENOTCONV, "a pair reached the sweep cap");
    return MORAP_OK;
    API_END
}

int morap_evaluate(morap_ctx *ctx, int32_t n_pairs, const int32_t *pair_product, const int32_t *pair_weight,
                   void *stream, double *rcost_out, double *rprob_out) {
    API_BEGIN
    if (!ctx || n_pairs < 0 || (n_pairs > 0 && (!pair_product || !pair_weight || !rcost_out || !rprob_out)))
        return fail(MORAP_EINVAL, "null argument");
    if (!ctx->built || ctx->last_K == 0) return fail(MORAP_ESTATE, "evaluate before a solve");
    std::vector<int4> pairs((size_t)n_pairs);
    for (int e = 0; e < n_pairs; ++e) {
        if (pair_product[e] < 0 || pair_product[e] >= ctx->P) return fail(MORAP_EINVAL, "product index out of range");
        if (pair_weight[e] < 0 || pair_weight[e] >= ctx->last_K)
            return fail(MORAP_EINVAL, "weight index out of range of the last solve");
        pairs[e] = make_int4(pair_product[e], pair_weight[e], 0, 0);
    }
    if (n_pairs == 0) return MORAP_OK;
    CK(cudaSetDevice(ctx->cfg.device));
    std::vector<double> rc, rp;
    int nc = 0;
    CKR(run_evaluation(ctx, pairs, (cudaStream_t)stream, rc, rp, nc));
    std::copy(rc.begin(), rc.end(), rcost_out);
    std::copy(rp.begin(), rp.end(), rprob_out);
    if (nc) return fail(MORAP_ENOTCONV, "an evaluation reached the sweep cap");
    return MORAP_OK;
    API_END
}

int morap_supporting_points(morap_ctx *ctx, int32_t K, const double *W, void *stream, double *r_out,
                            int32_t *assign_out, double *c_out) {
    API_BEGIN
    if (!ctx || !W || !r_out) return fail(MORAP_EINVAL, "null argument");
    if (!ctx->built) return fail(MORAP_ESTATE, "supporting_points before build");
    if (!ctx->sel_agent.empty())
        return fail(MORAP_ESTATE, "supporting_points needs every agent x task product (the context has a pair list)");
    if (K < 1) return fail(MORAP_EINVAL, "K must be >= 1");
    CK(cudaSetDevice(ctx->cfg.device));
    CKR(check_weights(ctx, K, W));
    const int nobj = ctx->nI + ctx->nJ;
    int status = MORAP_OK;
    for (int k0 = 0; k0 < K; k0 += 64) {
        const int kb = std::min(64, K - k0);
        const int rc = supporting_batch(ctx, kb, W + (size_t)k0 * nobj, (cudaStream_t)stream, r_out + (size_t)k0 * nobj,
                                        assign_out ? assign_out + (size_t)k0 * ctx->nJ : nullptr,
                                        c_out ? c_out + (size_t)k0 * ctx->P : nullptr);
        if (rc == MORAP_ENOTCONV)
            status = rc;
        else if (rc != MORAP_OK)
            return rc;
    }
    return status;
    API_END
}

int morap_last_solve_stats(const morap_ctx *ctx, morap_solve_stats *out) {
    if (!ctx || !out) return fail(MORAP_EINVAL, "null argument");
    *out = ctx->stats;
    return MORAP_OK;
}

namespace {
int run_query(morap_ctx *ctx, const double *t, const double *M, double eps, int32_t max_iter, void *stream,
              morap_point_result *res, bool verify_only) {
    if (!ctx || !t || !res) return fail(MORAP_EINVAL, "null argument");
    if (!ctx->built) return fail(MORAP_ESTATE, "query before build");
    if (!(eps >= 0) || max_iter < 1) return fail(MORAP_EINVAL, "eps >= 0 and max_iter >= 1 required");
    const int n = ctx->nI + ctx->nJ;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(t[i])) return fail(MORAP_EINVAL, "threshold entries must be finite");
    Alg1 q;
    q.init(n, t, M, eps, max_iter, verify_only);
    std::vector<double> r(n);
    std::vector<int32_t> f(ctx->nJ);
    while (!q.done) {
        const int rc = morap_supporting_points(ctx, 1, q.w.data(), stream, r.data(), f.data(), nullptr);
        if (rc == MORAP_ENOTCONV)
            q.status = rc;
        else if (rc != MORAP_OK)
            return rc;
        q.step(r.data(), f.data(), ctx->nJ);
    }
    const int status = alg1_result(q, res);
    if (status != MORAP_OK) return fail(status, "query stopped before ||t_down - t_up|| <= eps");
    return MORAP_OK;
}
}  // namespace

int morap_query(morap_ctx *ctx, const double *t, const double *M, double eps, int32_t max_iter, void *stream,
                morap_point_result *res) {
    API_BEGIN
    return run_query(ctx, t, M, eps, max_iter, stream, res, false);
    API_END
}

int morap_verify(morap_ctx *ctx, const double *t, const double *M, double eps, int32_t max_iter, void *stream,
                 morap_point_result *res) {
    API_BEGIN
    return run_query(ctx, t, M, eps, max_iter, stream, res, true);
    API_END
}

struct morap_pareto {
    Alg1 q;
};

int morap_pareto_create_mode(int32_t n, const double *t, const double *M, double eps, int32_t max_iter,
                             int32_t mode, morap_pareto **out) {
    API_BEGIN
    if (mode != MORAP_PARETO_SYNTHESIS && mode != MORAP_PARETO_VERIFY)
        return fail(MORAP_EINVAL, "pareto_create: unknown mode");
    if (!t || !out || n < 1) return fail(MORAP_EINVAL, "pareto_create: n >= 1, t and out required");
    if (!(eps >= 0) || max_iter < 1) return fail(MORAP_EINVAL, "eps >= 0 and max_iter >= 1 required");
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(t[i])) return fail(MORAP_EINVAL, "threshold entries must be finite");
    auto *ps = new morap_pareto();
    ps->q.init(n, t, M, eps, max_iter, mode == MORAP_PARETO_VERIFY);
    *out = ps;
    return MORAP_OK;
    API_END
}

int morap_pareto_create(int32_t n, const double *t, const double *M, double eps, int32_t max_iter,
                        morap_pareto **out) {
    return morap_pareto_create_mode(n, t, M, eps, max_iter, MORAP_PARETO_SYNTHESIS, out);
}

int morap_pareto_next(const morap_pareto *ps, double *w_out, int32_t *done) {
    if (!ps || !done) return fail(MORAP_EINVAL, "pareto_next: null argument");
    *done = ps->q.done ? 1 : 0;
    if (!ps->q.done) {
        if (!w_out) return fail(MORAP_EINVAL, "pareto_next: w_out required");
        std::copy(ps->q.w.begin(), ps->q.w.end(), w_out);
    }
    return MORAP_OK;
}

int morap_pareto_step(morap_pareto *ps, const double *r, int32_t solve_status) {
    API_BEGIN
    if (!ps || !r) return fail(MORAP_EINVAL, "pareto_step: null argument");
    if (ps->q.done) return fail(MORAP_ESTATE, "pareto_step: the loop already stopped");
    if (solve_status != MORAP_OK && solve_status != MORAP_ENOTCONV)
        return fail(MORAP_EINVAL, "pareto_step: solve_status must be MORAP_OK or MORAP_ENOTCONV");
    for (int i = 0; i < ps->q.n; ++i)
        if (!std::isfinite(r[i])) return fail(MORAP_EINVAL, "supporting point entries must be finite");
    if (solve_status == MORAP_ENOTCONV && ps->q.status == MORAP_OK) ps->q.status = MORAP_ENOTCONV;
    ps->q.step(r);
    return MORAP_OK;
    API_END
}

int morap_pareto_result(const morap_pareto *ps, morap_point_result *res) {
    if (!ps || !res) return fail(MORAP_EINVAL, "pareto_result: null argument");
    const int st = alg1_result(ps->q, res);
    if (st != MORAP_OK) return fail(st, "loop stopped before ||t_down - t_up|| <= eps");
    return MORAP_OK;
}

void morap_pareto_destroy(morap_pareto *ps) { delete ps; }

int morap_solve_plain(morap_ctx *ctx, int32_t n_pairs, const int32_t *pair_product, const double *pair_w,
                      void *stream, double *c_out, double *rcost_out, double *rprob_out, double *stats_out) {
    API_BEGIN
    if (!ctx || (n_pairs > 0 && (!pair_product || !pair_w || !c_out))) return fail(MORAP_EINVAL, "null argument");
    if (!ctx->built) return fail(MORAP_ESTATE, "solve_plain before build");
    CK(cudaSetDevice(ctx->cfg.device));
    cudaStream_t s = (cudaStream_t)stream;
    CKR(ensure_fp64_csr(ctx, s));
    uint32_t max_n = 1, max_sa = 1;
    for (int e = 0; e < n_pairs; ++e) {
        if (pair_product[e] < 0 || pair_product[e] >= ctx->P) return fail(MORAP_EINVAL, "product index out of range");
        const ProdDesc &pd = ctx->h_prods[pair_product[e]];
        max_n = std::max(max_n, pd.n_nd + 1);
        max_sa = std::max(max_sa, (uint32_t)pd.Qn * pd.SA);
    }
    std::vector<void *> L;
    double *x, *y, *q;
    int32_t *a_rec, *mu;
    unsigned long long *dres;
    int rc = MORAP_OK;
    auto cleanup = [&]() { dev_free_list(ctx, L); };
    if ((rc = dev_alloc(ctx, L, &x, (size_t)max_n * 8)) || (rc = dev_alloc(ctx, L, &y, (size_t)max_n * 8)) ||
        (rc = dev_alloc(ctx, L, &q, (size_t)max_sa * 8)) || (rc = dev_alloc(ctx, L, &a_rec, (size_t)max_n * 4)) ||
        (rc = dev_alloc(ctx, L, &mu, (size_t)max_n * 4)) || (rc = dev_alloc(ctx, L, &dres, 64))) {
        cleanup();
        return rc;
    }
    unsigned long long *h_res = nullptr;
    if (cudaMallocHost((void **)&h_res, 64) != cudaSuccess) {
        cleanup();
        return fail(MORAP_ECUDA, "cudaMallocHost");
    }
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    double sweeps_vi = 0, sweeps_eval = 0, updates = 0;
    bool capped = false;
    auto run = [&]() -> int {
        for (int e = 0; e < n_pairs; ++e) {
            const ProdDesc &pd = ctx->h_prods[pair_product[e]];
            const uint32_t n = pd.n_nd, n_sa = (uint32_t)pd.Qn * pd.SA;
            const uint32_t pre_sa = (uint32_t)(pd.pre_begin / std::max<uint32_t>(pd.S, 1)) * pd.SA;
            const uint32_t n_tr = pd.n_tr;
            const double wi = pair_w[2 * e], wp = pair_w[2 * e + 1];
            CK(cudaMemsetAsync(x, 0, (size_t)(n + 1) * 8, s));
            CK(cudaMemsetAsync(y, 0, (size_t)(n + 1) * 8, s));
            CK(cudaMemsetAsync(a_rec, 0, (size_t)(n + 1) * 4, s));
            double *xc = x, *yc = y;
            int sw = 0;
            for (;;) {
                CK(cudaMemsetAsync(dres, 0, 8, s));
                CKL(launch_plain_spmv(ctx->sa_tr, ctx->col, ctx->p64, ctx->cost64, pd.sa_off, n_sa, wi, wp, pre_sa,
                                      pd.state_off, xc, q, s));
                CKL(launch_plain_reduce(ctx->state_sa, pd.state_off, n, pd.sa_off, q, xc, yc, a_rec,
                                        ctx->cfg.eps_vi, dres, s));
                CK(cudaMemcpyAsync(h_res, dres, 8, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                std::swap(xc, yc);
                ++sw;
                updates += n_tr;
                double r;
                std::memcpy(&r, h_res, 8);
                if (r <= ctx->cfg.eps_vi) break;
                if (sw >= ctx->cfg.max_sweeps) {
                    capped = true;
                    break;
                }
            }
            sweeps_vi += sw;
            CKL(launch_plain_spmv(ctx->sa_tr, ctx->col, ctx->p64, ctx->cost64, pd.sa_off, n_sa, wi, wp, pre_sa,
                                  pd.state_off, xc, q, s));
            CKL(plain_finalize(ctx->state_sa, ctx->sa_tr, ctx->col, ctx->p64, pd.state_off, n, pd.sa_off, q, a_rec,
                               ctx->cfg.tau_policy, mu, dres + 1, s));
            double cval = 0.0;
            if ((uint32_t)pd.init_local < n) CK(cudaMemcpyAsync(&cval, xc + pd.init_local, 8, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            c_out[e] = cval;
            for (int obj = 0; obj < 2; ++obj) {
                double *out = obj == 0 ? rcost_out : rprob_out;
                if (!out) continue;
                CK(cudaMemsetAsync(x, 0, (size_t)(n + 1) * 8, s));
                CK(cudaMemsetAsync(y, 0, (size_t)(n + 1) * 8, s));
                double *xe = x, *ye = y;
                int se = 0;
                for (;;) {
                    CK(cudaMemsetAsync(dres, 0, 8, s));
                    CKL(launch_plain_eval(ctx->state_sa, ctx->sa_tr, ctx->col, ctx->p64, ctx->cost64, pd.state_off, n,
                                          pd.pre_begin, mu, obj, xe, ye, dres, s));
                    CK(cudaMemcpyAsync(h_res, dres, 8, cudaMemcpyDeviceToHost, s));
                    CK(cudaStreamSynchronize(s));
                    std::swap(xe, ye);
                    ++se;
                    double r;
                    std::memcpy(&r, h_res, 8);
                    if (r <= ctx->cfg.eps_eval) break;
                    if (se >= ctx->cfg.max_sweeps) {
                        capped = true;
                        break;
                    }
                }
                sweeps_eval += se;
                double v = 0.0;
                if ((uint32_t)pd.init_local < n) CK(cudaMemcpyAsync(&v, xe + pd.init_local, 8, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                out[e] = v;
            }
        }
        return MORAP_OK;
    };
    rc = run();
    const double ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    cudaFreeHost(h_res);
    cleanup();
    if (rc != MORAP_OK) return rc;
    if (stats_out) {
        stats_out[0] = sweeps_vi;
        stats_out[1] = sweeps_eval;
        stats_out[2] = updates;
        stats_out[3] = ms;
    }
    if (capped) return fail(MORAP_ENOTCONV, "plain VI reached the sweep cap");
    return MORAP_OK;
    API_END
}

int morap_assign_max(int32_t n, const double *C, int32_t *f_out) {
    API_BEGIN
    if (n < 0 || (n > 0 && (!C || !f_out))) return fail(MORAP_EINVAL, "bad argument");
    std::vector<int> f(n);
    if (n) hungarian_max(n, C, f.data());
    for (int j = 0; j < n; ++j) f_out[j] = f[j];
    return MORAP_OK;
    API_END
}

int morap_assign_tasks(int32_t n_agents, int32_t n_tasks, int32_t K, const double *c, int32_t *assign_out) {
    API_BEGIN
    if (n_agents < 0 || n_tasks < 0 || K < 0) return fail(MORAP_EINVAL, "negative size");
    if ((size_t)n_agents * n_tasks * K > 0 && (!c || !assign_out)) return fail(MORAP_EINVAL, "null argument");
    for (int k = 0; k < K; ++k)
        assign_tasks(n_agents, n_tasks, c + (size_t)k * n_agents * n_tasks, assign_out + (size_t)k * n_tasks);
    return MORAP_OK;
    API_END
}

int morap_random_assignment(int32_t n_points, int32_t n_agents, int32_t n_tasks, const double *lambda,
                            const int32_t *assign_hist, double *P_out) {
    API_BEGIN
    if (n_points < 0 || n_agents < 0 || n_tasks < 0) return fail(MORAP_EINVAL, "negative size");
    if ((size_t)n_agents * n_tasks > 0 && !P_out) return fail(MORAP_EINVAL, "null argument");
    if (n_points > 0 && n_tasks > 0 && (!lambda || !assign_hist)) return fail(MORAP_EINVAL, "null argument");
    for (int l = 0; l < n_points; ++l) {
        if (!(lambda[l] >= 0.0) || !std::isfinite(lambda[l]))
            return fail(MORAP_EINVAL, "lambda[" + std::to_string(l) + "] is not a finite weight >= 0");
        for (int j = 0; j < n_tasks; ++j) {
            const int32_t i = assign_hist[(size_t)l * n_tasks + j];
            if (i < -1 || i >= n_agents)
                return fail(MORAP_EINVAL, "assign_hist[" + std::to_string(l) + "][" + std::to_string(j) +
                                              "] is not an agent index or -1");
        }
    }
    std::fill(P_out, P_out + (size_t)n_agents * n_tasks, 0.0);
    for (int l = 0; l < n_points; ++l)
        for (int j = 0; j < n_tasks; ++j) {
            const int32_t i = assign_hist[(size_t)l * n_tasks + j];
            if (i >= 0) P_out[(size_t)i * n_tasks + j] += lambda[l];
        }
    return MORAP_OK;
    API_END
}

int morap_project_halfspaces(int32_t n, int32_t m, const double *t, const double *A, const double *b,
                             const double *M, double *z_out) {
    API_BEGIN
    if (n < 1 || m < 0 || !t || !z_out || (m > 0 && (!A || !b))) return fail(MORAP_EINVAL, "bad argument");
    const int rc = project_halfspaces(n, m, t, A, b, M, z_out);
    if (rc > 1) return fail(MORAP_ENOTCONV, "QP factorisation failed");
    return MORAP_OK;
    API_END
}

int morap_project_down_hull(int32_t n, int32_t m, const double *t, const double *Phi, const double *M,
                            double *x_out) {
    API_BEGIN
    if (n < 1 || m < 1 || !t || !Phi || !x_out) return fail(MORAP_EINVAL, "bad argument");
    const int rc = project_down_hull(n, m, t, Phi, M, x_out);
    if (rc > 1) return fail(MORAP_ENOTCONV, "QP factorisation failed");
    return MORAP_OK;
    API_END
}

int morap_task_preprocess(int32_t n_locs, int32_t q0, int32_t n_ap, const int32_t *delta, const uint8_t *accepting,
                          int32_t *n_locs_out, uint8_t *flags_out) {
    API_BEGIN
    std::vector<int32_t> ids(std::max(n_ap, 0));
    for (int b = 0; b < n_ap; ++b) ids[b] = b;
    HostTask T;
    CKR(preprocess_task(n_locs, q0, n_ap, ids.data(), delta, accepting, T));
    if (n_locs_out) *n_locs_out = T.n_locs;
    if (flags_out)
        for (int q = 0; q < T.n_locs; ++q) flags_out[q] = T.flags[q];
    return MORAP_OK;
    API_END
}

int morap_product_info(const morap_ctx *ctx, int32_t p, int64_t *info) {
    if (!ctx || !info) return fail(MORAP_EINVAL, "null argument");
    if (!ctx->built) return fail(MORAP_ESTATE, "not built");
    if (p < 0 || p >= ctx->P) return fail(MORAP_EINVAL, "product index out of range");
    const ProdDesc &pd = ctx->h_prods[p];
    info[0] = pd.S;
    info[1] = pd.Qn;
    info[2] = (int64_t)pd.n_nd + 1;
    info[3] = (int64_t)pd.Qn * pd.SA;
    info[4] = (int64_t)pd.n_tr;
    info[5] = pd.init_local;
    info[6] = pd.state_off;
    info[7] = pd.pre_begin;
    info[8] = pd.agent;
    info[9] = pd.task;
    return MORAP_OK;
}

int morap_product_download(morap_ctx *ctx, int32_t p, int64_t *state_sa, int64_t *sa_tr, int32_t *col,
                           double *prob, double *cost, int32_t *loc_out) {
    API_BEGIN
    if (!ctx) return fail(MORAP_EINVAL, "null argument");
    if (!ctx->built) return fail(MORAP_ESTATE, "not built");
    if (p < 0 || p >= ctx->P) return fail(MORAP_EINVAL, "product index out of range");
    CK(cudaSetDevice(ctx->cfg.device));
    if (prob || cost) CKR(ensure_fp64_csr(ctx, nullptr));
    const ProdDesc &pd = ctx->h_prods[p];
    const size_t ns = pd.n_nd + 1, nsa = (size_t)pd.Qn * pd.SA, nt = pd.n_tr;
    std::vector<uint32_t> tmp;
    if (state_sa) {
        tmp.resize(ns + 1);
        CK(cudaMemcpy(tmp.data(), ctx->state_sa + pd.state_off, (ns + 1) * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i <= ns; ++i) state_sa[i] = (int64_t)tmp[i] - pd.sa_off;
    }
    if (sa_tr) {
        tmp.resize(nsa + 1);
        CK(cudaMemcpy(tmp.data(), ctx->sa_tr + pd.sa_off, (nsa + 1) * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i <= nsa; ++i) sa_tr[i] = (int64_t)tmp[i] - pd.tr_off;
    }
    if (col && nt) {
        CK(cudaMemcpy(col, ctx->col + pd.tr_off, nt * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < nt; ++i) col[i] -= (int32_t)pd.state_off;
    }
    if (prob && nt) CK(cudaMemcpy(prob, ctx->p64 + pd.tr_off, nt * 8, cudaMemcpyDeviceToHost));
    if (cost && nsa) CK(cudaMemcpy(cost, ctx->cost64 + pd.sa_off, nsa * 8, cudaMemcpyDeviceToHost));
    if (loc_out) {
        const HostTask &T = ctx->tasks[pd.task];
        for (int k = 0; k < T.n_nd; ++k) loc_out[k] = T.loc_of[k];
    }
    return MORAP_OK;
    API_END
}

int morap_last_policy(morap_ctx *ctx, int32_t k, int32_t p, uint8_t *mu_out, double *values_out) {
    API_BEGIN
    if (!ctx) return fail(MORAP_EINVAL, "null argument");
    if (!ctx->Kp) return fail(MORAP_ESTATE, "no solve yet");
    if (p < 0 || p >= ctx->P || k < 0 || k >= ctx->Kp) return fail(MORAP_EINVAL, "index out of range");
    CK(cudaSetDevice(ctx->cfg.device));
    const ProdDesc &pd = ctx->h_prods[p];
    const size_t n = pd.n_nd + 1, Kp = ctx->Kp;
    if (mu_out) {
        std::vector<uint8_t> buf(n * Kp);
        CK(cudaMemcpy(buf.data(), ctx->policy + (size_t)pd.state_off * Kp, n * Kp, cudaMemcpyDeviceToHost));
        for (size_t u = 0; u < n; ++u) mu_out[u] = buf[u * Kp + k];
    }
    if (values_out) {
        std::vector<float2> buf(n * Kp);
        CK(cudaMemcpy(buf.data(), (float2 *)ctx->V64[0] + (size_t)pd.state_off * Kp, n * Kp * 8,
                      cudaMemcpyDeviceToHost));
        for (size_t u = 0; u < n; ++u) values_out[u] = (double)buf[u * Kp + k].x + (double)buf[u * Kp + k].y;
    }
    return MORAP_OK;
    API_END
}

}  // extern "C"

// Internal declarations shared by the engine's translation units.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <vector_types.h>

#include "../../include/morap.h"

namespace morap {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

// ------------------------------------------------------------- host models
struct HostAgent {
    int32_t n_states = 0, s0 = 0;
    std::vector<int32_t> state_ptr, sa_ptr, succ;
    std::vector<double> prob, cost;
    std::vector<int32_t> label_ptr, label_ap;
    bool free_action_everywhere = false;  // every state has a zero-cost action
};

// A task after preprocessing.  Product locations are the non-done
// locations, numbered with the pre-sinks last so that "pre-sink" is a
// single threshold on the product-local state index.
struct HostTask {
    int32_t n_locs = 0;  // after pre-sink insertion
    int32_t q0 = 0;
    int32_t n_ap = 0, n_letters = 1;
    std::vector<int32_t> ap_ids;
    std::vector<int32_t> delta;   // [n_locs][n_letters]
    std::vector<uint8_t> flags;   // bit0 accepting, bit1 trap, bit2 pre-sink, bit3 done
    std::vector<int32_t> ploc;    // product location index of each location, -1 if done
    std::vector<int32_t> loc_of;  // location of each product location index
    int32_t n_nd = 0, n_pre = 0;
    // nd_delta[pl * n_letters + letter] = product location index of the
    // successor location, or -1 when it is done.
    std::vector<int16_t> nd_delta;
};

int preprocess_task(int32_t n_locs, int32_t q0, int32_t n_ap, const int32_t *ap_ids, const int32_t *delta,
                    const uint8_t *accepting, HostTask &out);

// --------------------------------------------------------- host algorithms
// Square assignment maximising sum_j C[f(j)][j]; C row-major [n][n].
void hungarian_max(int n, const double *C, int *f);
// Rectangular assignment of Algorithm 2 (C row-major [nI][nJ]): assign[j] =
// agent of task j, -1 for none.
void assign_tasks(int nI, int nJ, const double *C, int32_t *assign);

// Dense convex QP: min 1/2 x'Gx + c'x  s.t.  A x <= b (m rows), E x = d (p rows).
// Mehrotra predictor-corrector primal-dual interior point.  Returns 0 on
// convergence.
int qp_solve(int n, const double *G, const double *c, int m, const double *A, const double *b, int p,
             const double *E, const double *d, double *x, double tol = 1e-13, int max_iter = 200);

int project_halfspaces(int n, int m, const double *t, const double *A, const double *b, const double *M,
                       double *z);
// lambda (nullable, [m]): convex weights of the points with x <= sum lambda_l Phi_l
int project_down_hull(int n, int m, const double *t, const double *Phi, const double *M, double *x,
                      double *lambda = nullptr);

// ||v||_M = sqrt(v' M v); M row-major [n][n], NULL = identity.
double mnorm(int n, const double *v, const double *M);

// Algorithm 1 advanced one supporting point at a time: `w` is the direction
// whose supporting point step() expects next, until `done`.
struct Alg1 {
    int n = 0, it = 0, max_iter = 64, status = 0;
    double eps = 1e-6, dist = HUGE_VAL;
    bool moved = false, done = false;
    // verification only (Sec. 5, Exp. 2): the first supporting hyperplane
    // that separates t ends the loop with the verdict "not achievable"
    bool verify_only = false, decided = false;
    std::vector<double> t, M, w, t_dn, t_up, Phi, A, b, w_hist, r_hist;
    std::vector<double> lambda;  // convex weights of the points behind t_up (last projection)
    std::vector<int32_t> f_hist;  // assignment of each point, [it][f_tasks], when the caller gives it
    int f_tasks = 0;
    void init(int n_obj, const double *t_in, const double *M_in, double eps_in, int max_iter_in,
              bool verify_only_in = false);
    void step(const double *r, const int32_t *assign = nullptr, int n_tasks = 0);
};
// Fill *res from a finished run; returns its status (ENOTCONV when it
// stopped with ||t_down - t_up|| > eps).
int alg1_result(const Alg1 &q, morap_point_result *res);

// ------------------------------------------------------ device layout
struct ProdDesc {
    uint32_t state_off;  // global index of the product's first state
    uint32_t n_nd;       // non-done states (Qn * S); the done slot is state_off + n_nd
    uint32_t pre_begin;  // local states >= pre_begin sit at a pre-sink location
    int32_t init_local;  // local index of (s0, q0), == n_nd when q0 is done
    uint32_t sa_off, tr_off;
    int32_t agent, task;
    uint32_t S, SA, T;   // agent sizes
    int32_t Qn;
    uint32_t letter_off; // offset of this product's letter table (per agent state)
    uint32_t item_off;   // index of the product's first sweep work item
    uint32_t n_tr;       // product transitions (successors into the done slot merged per row)
};

struct AgentDesc {
    uint32_t sp_off;    // into the concatenated state_ptr arrays (S+1 each)
    uint32_t sap_off;   // into the concatenated sa_ptr arrays (SA+1 each)
    uint32_t cost_off;  // into the concatenated cost arrays (SA each)
    uint32_t tr_off;    // into the concatenated succ/prob arrays (T each)
    uint32_t lp_off;    // into the concatenated label_ptr arrays (S+1 each)
    uint32_t la_off;    // into the concatenated label_ap arrays
    uint32_t S, SA, T;
    int32_t s0;
};

struct TaskDesc {
    uint32_t delta_off;  // into nd_delta
    uint32_t ap_off;     // into ap_ids
    int32_t n_ap, n_letters, Qn, n_pre;
    int32_t q0_ploc;     // product location index of q0, -1 if done
};

// Loop control block for one device-side sweep loop (see sweep.cu).
struct LoopCtl {
    unsigned int cnt[3];   // length of work list L[n % 3]
    unsigned int next[3];  // dynamic scheduling cursor of sweep n into L[n % 3]
    unsigned int sweep_base;
    unsigned int hit_cap;
    unsigned int cap;
    unsigned int skipped;  // work items a sweep skipped because none of their inputs changed
    unsigned int block_sweeps;  // most sweeps of a pair evaluated by one block (k_eval_block)
    unsigned long long updates;
    unsigned long long bytes;
    unsigned int undecided;  // scheduler states whose recorded action is not kept (k_finalize)
    unsigned int decided;    // states one anchoring round decided (k_anchor)
    unsigned int computed;   // work items a sweep computed (not skipped)
    unsigned int tail;       // the graph's while loop stops once the work list has <= tail items
                             // (0: runs to the end; otherwise k_sweep_tail runs the rest)
    unsigned int bar;        // k_sweep_tail's grid-barrier arrivals
    unsigned int bar_err;    // 1: a grid-barrier wait of k_sweep_tail ran out
    unsigned int tail_sweeps;  // sweeps k_sweep_tail ran
};

#ifndef MORAP_CHUNK
#define MORAP_CHUNK 64
#endif
constexpr int kChunk = MORAP_CHUNK;  // states per (warp) work item of the optimisation sweeps
constexpr int kEvalChunk = 256;  // states per work item of the evaluation sweeps
// Pairs whose n + 1 values fit twice in kEvalBlockSmem bytes are evaluated by
// one block each, all sweeps in one launch (k_eval_block).
constexpr int kEvalBlockThreads = 1024;
constexpr int kEvalBlockSmem = 224 * 1024;
constexpr uint32_t kEvalBlockStates = kEvalBlockSmem / (2 * 16);
constexpr int kThreads = 256;
// Rounds of the scheduler's anchoring step (a state decided in round r is
// stamped r + 1 in a byte): states still undecided after them keep the
// lowest-index near-maximiser that is not a self-loop.
constexpr int kAnchorRounds = 254;
constexpr int kInItems = 16;     // input items recorded per work item (more: always recomputed)
int sweep_smem_bytes(int kind);
int sweep_setup_attributes();

struct SweepArgs {
    const uint32_t *state_sa;
    const uint32_t *state_tr;  // first transition of each state (= sa_tr[state_sa[u]])
    const uint32_t *sa_tr;
    const int32_t *col;
    const int2 *cp32;     // per transition {col, p rounded down as float bits}
    const double *p64;
    const float *cost32;
    const double *cost64;
    const int4 *chunks;   // {product, begin, end, first}
    const uint4 *chunk_u; // per item {first state, end state, product's first pre-sink state, 0}, global indices
    const ProdDesc *prods;
    const float2 *pdf;    // per transition: p as a double-float (hi, lo)
    const float2 *costdf; // per state-action: cost as a double-float
    const float2 *w32;    // per pair (p*Kp + k): (-(w_i rounded up), w_p rounded down)
    const double2 *w64;   // per pair: (w_i, w_p)
    const float4 *wdf;    // per pair: (w_i.hi, w_i.lo, w_p.hi, w_p.lo)
    const double *thr;    // per pair freeze threshold of this phase
    unsigned long long *res[3];  // per pair residual of sweep n % 3 (double bits)
    int32_t *sweeps_pair;
    uint8_t *frozen;      // per pair: 1 once its residual fell to the threshold
    unsigned int *list[3];
    LoopCtl *ctl;
    void *V[2];
    uint8_t *a_rec;
    // Exact skipping: a work item whose states and successors all kept their
    // values in the previous sweep would reproduce its values bit for bit,
    // so it is not recomputed.  in_items[item][kInItems]: the other items
    // holding successors of its states (-1 none, -2 too many: always
    // recompute); chg[n % 3][item]: some value of the item changed in sweep n.
    const int32_t *in_items;
    const uint2 *item_w;  // (transitions, state-action rows) of each item, for the statistics
    uint8_t *chg[3];
    int skip;  // 0: recompute every item (skipping disabled)
    int keep_batch;  // kept items appended per atomic (1 keeps the list's order; 1..32)
    const float *G;  // residual-correction polish: [state-action][Kp] table (see ArithDelta)
    double eps1;
    float eps1f;  // eps1 rounded to FP32 (record tests in the kernels)
    int P;
    int gmax;     // most warps per work item (1, 2, 4 or 8)
};

struct EvalArgs {
    const uint32_t *state_sa;
    const uint32_t *sa_tr;
    const int32_t *col;
    const float2 *pdf;      // double-float probability per transition
    const float2 *costdf;   // double-float cost per state-action
    const ProdDesc *prods;
    const uint8_t *policy;  // [state][Kp]
    int Kp;
    const int4 *chunks;     // {eval pair, begin, end, first}
    const int4 *pairs;      // {product, k, value offset, 0}
    double thr;
    unsigned long long *res[3];
    int32_t *sweeps_pair;
    uint8_t *frozen;
    unsigned int *list[3];
    LoopCtl *ctl;
    float4 *E[2];    // (cost.h, cost.l, prob.h, prob.l) double-float values
    // compact scheduler rows of the evaluated pairs (built once per call):
    // for pair e with value offset off and n + 1 states (done slot n), slot j
    // of state s is at off * stride + j * (n + 1) + s
    int32_t *ecol;   // local successor (n = done slot for padding)
    float2 *ep;      // double-float probability (0 for padding)
    float2 *ecost;   // double-float cost of the scheduler's action, at off + s
    int stride;      // slots per state: the longest action row of any agent
    // transitions of the scheduler's rows (padding excluded) per evaluation
    // work item and per pair, summed by k_eval_compact (zeroed before it)
    uint32_t *item_tmu;
    uint32_t *pair_tmu;
};

// Engine helpers the serving layer uses (engine.cu).
int ctx_reserve(morap_ctx *c, int K);
int ctx_merge(morap_ctx *const *ctxs, int n, morap_ctx **out, std::vector<int32_t> &agent_off,
              std::vector<int32_t> &task_off, std::vector<int32_t> &pair_off);
std::string ctx_arith_key(const morap_ctx *c);
int64_t ctx_max_states(const morap_ctx *c);
int ctx_no_tail(morap_ctx *c);  // every sweep of the context's loops its own launch (tail_items = 0)

// ---------------------------------------------------------- kernel launchers
// (defined in the .cu files; every launcher enqueues on `s` and returns the
// cudaError_t of the launch as an int)
int launch_letters(const ProdDesc *prods, int P, const AgentDesc *agents, const TaskDesc *tasks,
                   const int32_t *label_ptr, const int32_t *label_ap, const int32_t *ap_ids, uint8_t *letters,
                   uint32_t max_S, void *s);
// Product construction, first pass: the number of transitions of every
// product row after merging its successors into the done slot (row_cnt[row]),
// and, when prod_tr is not NULL, their sum per product (added to prod_tr[p]).
int launch_row_count(const ProdDesc *prods, int P, const AgentDesc *agents, const TaskDesc *tasks,
                     const int32_t *a_sa_ptr, const int32_t *a_succ, const uint8_t *letters,
                     const int16_t *nd_delta, uint32_t *row_cnt, uint32_t *prod_tr, uint32_t max_rows, void *s);
// Second pass: sa_tr[row] = the product's tr_off + the exclusive prefix sum
// of row_cnt over the product's rows (one block per product).
int launch_row_offsets(const ProdDesc *prods, int P, const uint32_t *row_cnt, uint32_t *sa_tr, void *s);
int launch_build(const ProdDesc *prods, int P, const AgentDesc *agents, const TaskDesc *tasks,
                 const int32_t *a_state_ptr, const int32_t *a_sa_ptr, const int32_t *a_succ, const double *a_prob,
                 const double *a_cost, const uint8_t *letters, const int16_t *nd_delta, uint32_t *state_sa,
                 uint32_t *state_tr, uint32_t *sa_tr, int32_t *col, int2 *cp32, double *p64, float2 *pdf,
                 float *cost32, double *cost64, float2 *costdf, uint32_t total_states, uint32_t total_sa,
                 uint32_t total_tr, uint32_t max_work, void *s);

int launch_setup_weights(const ProdDesc *prods, int P, int nI, int nJ, int K, int Kp, const double *W,
                         float2 *w32, double2 *w64, float4 *wdf, double *thr32, double *thr64, double eps1,
                         bool after_fp32, void *s);
int launch_item_inputs(const int4 *chunks, int n_items, const ProdDesc *prods, const uint32_t *state_tr,
                       const int32_t *col, int32_t *in_items, uint2 *item_w, const uint32_t *state_sa,
                       void *s);
// chg_prev (nullable, [n_items]): set to 1 so that the first sweep recomputes every item;
// w_pair (nullable, [n_pairs]): pairs whose two weights are both 0 start frozen
int launch_loop_init(LoopCtl *ctl, unsigned int *list0, unsigned int n_items, unsigned long long *res[3],
                     size_t n_pairs, int32_t *sweeps_pair, uint8_t *frozen, unsigned int cap, void *s,
                     uint8_t *chg_prev = nullptr, const double2 *w_pair = nullptr, unsigned int tail = 0);
// Sweep kinds: the FP32 round-down phase, the double-float polish, and the
// polish as an FP32 residual correction on a double-float table.
enum { kSweepF32 = 0, kSweepDF = 1, kSweepDelta = 2 };
// One sweep with kernel shape `variant` (0 .. sweep_variant_count - 1; all
// shapes give bit-identical results, they differ only in speed).
int launch_sweep(int kind, int Kp, int variant, const SweepArgs &a, int pos, int grid, void *s);
int sweep_blocks_per_sm(int kind, int Kp, int variant);
// The rest of a loop whose work list has fallen to ctl->tail items, in one
// cooperative launch of `grid` blocks (at most sweep_tail_blocks_per_sm per
// SM; 0 there: the occupancy query failed).  Same results as the sweeps one
// launch each.  A grid-barrier wait that runs out sets ctl->bar_err.
int launch_sweep_tail(int kind, int Kp, const SweepArgs &a, int grid, void *s);
int sweep_tail_blocks_per_sm(int kind, int Kp);
// A cooperative launch of the tail's grid barrier in which one block never
// arrives (the others' bounded waits run out; ctl->bar_err is set).
int launch_barrier_selfcheck(LoopCtl *ctl, int grid, void *s);
int sweep_variant_count(int kind);

int eval_blocks_per_sm();
int launch_loop_control(LoopCtl *ctl, unsigned long long handle, int next_idx, void *s);
int launch_loop_control_host(LoopCtl *ctl, int next_idx, void *s);
// The residual-correction table G[sa][k] = r_a + sum p B(s') - B(s) (+ the
// pre-sink weight) in double-float from the FP32 values B, rounded to FP32.
int launch_delta_table(int Kp, const SweepArgs &a, int n_chunks, const float *B, float *G, void *s);
// V = B + d as an exact double-float sum.
int launch_delta_combine(const float *B, const float *d, float2 *V, size_t n, void *s);
int launch_convert(const float *v32, float2 *vda, float2 *vdb, size_t n, void *s);
// The returned scheduler (a.a_rec is consumed: it becomes the anchoring
// flags; a.ctl->undecided counts the states the anchoring rounds decide).
int launch_finalize(int Kp, const SweepArgs &a, int n_chunks, double tau, uint8_t *policy, void *s);
// One anchoring round over every undecided (state, weight); a.ctl->decided
// counts the states it decided.
int launch_anchor(int Kp, const SweepArgs &a, int n_chunks, double tau, uint8_t *policy, int round, void *s);
int launch_gather_c(int Kp, const ProdDesc *prods, int P, const float2 *V64, const uint8_t *frozen, double *c_out,
                    int32_t *status_out, void *s);
int eval_block_setup();  // once per device: k_eval_block's shared-memory limit
// Algorithm 4 for n_bpairs pairs (indices into a.pairs), one block each,
// every sweep in one launch; max_states bounds their n + 1 values.
int launch_eval_block(const EvalArgs &a, const int *bpairs, int n_bpairs, uint32_t max_states, unsigned int cap,
                      void *s);
int launch_eval_sweep(const EvalArgs &a, int pos, int grid, void *s);
int launch_eval_compact(const EvalArgs &a, int n_chunks, void *s);
int launch_gather_eval(const int4 *pairs, int n_pairs, const ProdDesc *prods, const float4 *E, double *rc,
                       double *rp, void *s);
// plain baseline
int launch_plain_spmv(const uint32_t *sa_tr, const int32_t *col, const double *p64, const double *cost64,
                      uint32_t sa_begin, uint32_t n_sa, double wi, double wp, uint32_t pre_sa_begin,
                      uint32_t state_off, const double *x, double *q, void *s);
int launch_plain_reduce(const uint32_t *state_sa, uint32_t state_off, uint32_t n_states, uint32_t sa_begin,
                        const double *q, const double *x, double *y, int32_t *a_rec, double eps,
                        unsigned long long *res, void *s);
// The returned scheduler of the plain path from the Q values q of the final
// iterate: kept recorded actions, then the anchoring rounds (at most
// kAnchorRounds).  a_rec is consumed (it becomes the anchor flags); counter
// is one device word of scratch.  Synchronises the stream.
int plain_finalize(const uint32_t *state_sa, const uint32_t *sa_tr, const int32_t *col, const double *p64,
                   uint32_t state_off, uint32_t n_states, uint32_t sa_begin, const double *q, int32_t *a_rec,
                   double tau, int32_t *mu, unsigned long long *counter, void *s);
int launch_plain_eval(const uint32_t *state_sa, const uint32_t *sa_tr, const int32_t *col, const double *p64,
                      const double *cost64, uint32_t state_off, uint32_t n_states, uint32_t pre_begin,
                      const int32_t *mu, int objective, const double *x, double *y, unsigned long long *res,
                      void *s);

}  // namespace morap

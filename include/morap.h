/*
 * morap.h -- C-ABI of the GB300 engine for multi-objective random task
 * assignment and planning (MORAP, arxiv 2305.04397).
 *
 * The engine solves, for every agent x task product MDP M_i (x) A_j
 * (Sec. 2 "Product MDP", Sec. 3.1), the weighted-sum value iteration of
 * Algorithm 3, evaluates the cost and probability objectives of the
 * returned scheduler with Algorithm 4 (Appendix A.4), chooses the task
 * assignment of Algorithm 2 (Sec. 3.3), and answers threshold-point queries
 * with the point-oriented Pareto loop of Algorithm 1 (Sec. 3.3, Thm 3).
 *
 * Conventions
 *  - Every call returns an int status (MORAP_OK = 0).  On failure the
 *    message of the calling thread's last error is available from
 *    morap_last_error(); no call aborts the process.
 *  - Inputs are caller-owned and are copied (or fully consumed) during the
 *    call.  Outputs go to caller-allocated HOST arrays whose sizes are given
 *    per call.  Handles are opaque and destroyed explicitly (the paper's
 *    models are owned by exactly one owner, Sec. 4 "Programming").
 *  - Objectives are maximised.  Costs enter as negative rewards (Sec. 3.1):
 *    "expected cost <= 8" is the threshold c_i = -8.  The objective vector
 *    has |I| + |J| entries: k = i for agent i's cost, k = |I| + j for task j's
 *    probability (Def. 1, Algorithm 1 input t = (c, p)).
 *  - "stream" arguments are cudaStream_t values passed as void*; NULL means
 *    the legacy default stream.
 *  - A context is not thread-safe: one host thread drives it at a time.
 *  - No call of this library waits on the device without a bound: every
 *    device loop has a sweep cap (MORAP_ENOTCONV when it is reached).
 */
#ifndef MORAP_H
#define MORAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
enum {
    MORAP_OK = 0,
    MORAP_EINVAL = 1,   /* malformed argument or model (message says which)   */
    MORAP_ENOMEM = 2,   /* HBM budget or device allocation refused            */
    MORAP_ENOTCONV = 3, /* a sweep cap was reached; outputs hold the last iterate */
    MORAP_ECUDA = 4,    /* a CUDA runtime call failed (message has the error) */
    MORAP_EBUSY = 5,    /* serving: the query is still in flight              */
    MORAP_ESTATE = 6    /* call order violated (e.g. solve before build)      */
};

/* Precision modes for the optimisation sweeps (Algorithm 3). */
enum {
    /* FP32 sweeps with every operation rounded toward -inf (a certified lower
     * bound of the FP64 iterate), then FP64-accurate sweeps from that bound
     * (see morap_config.polish) until their residual is <= eps_vi / 8: the
     * bound lies below the iterate by FP32 roundings that add up along each
     * path while each one is below eps_vi, which a test at eps_vi itself
     * would leave in place.  Used for products whose agent has a zero-cost
     * action in every state; other products run MORAP_PREC_FP64. */
    MORAP_PREC_MIXED = 0,
    /* FP64 sweeps from 0, as printed. */
    MORAP_PREC_FP64 = 1
};

/* Optional device allocator.  alloc returns a device pointer (or NULL on
 * failure) valid on the context's device; free releases it.  When both are
 * NULL the library uses cudaMalloc / cudaFree. */
typedef void *(*morap_alloc_fn)(size_t bytes, void *user);
typedef void (*morap_free_fn)(void *ptr, size_t bytes, void *user);

typedef struct morap_config {
    double eps_vi;      /* epsilon_1 of Algorithm 3 (stop when max|y - x| <= eps_vi; eps_vi / 8 for the
                           phase that follows an FP32 phase, see MORAP_PREC_MIXED); default 1e-8      */
    double eps_eval;    /* epsilon_2 of Algorithm 4; default 1e-11 (its stop error grows with the
                           expected number of steps, so it is kept below the 1e-6 value tolerance)   */
    double tau_policy;  /* tie tolerance of the returned scheduler, see morap_solve; default 1e-9     */
    int32_t max_sweeps; /* cap on sweeps per phase (FP32, FP64, evaluation); default 100000         */
    int32_t precision;  /* MORAP_PREC_MIXED (default) or MORAP_PREC_FP64                            */
    int32_t device;     /* CUDA device ordinal; default 0                                            */
    int32_t launch_mode;/* 0 (default): each sweep loop is one CUDA graph whose while node runs
                           bodies of six sweeps until the device work list is empty or short
                           enough for the tail launch (tail_items) that ends the graph; 1: the
                           host launches the same kernels body by body and reads the work list
                           between bodies (same results; for profilers that cannot enter
                           conditional graphs)                                                     */
    size_t hbm_budget;  /* admission limit in bytes for all device memory of the context; 0 = none  */
    morap_alloc_fn alloc;
    morap_free_fn free;
    void *alloc_user;
    int32_t sweep_variant_fp32; /* kernel shape of the FP32 / double-float sweeps: -1 (default) =   */
    int32_t sweep_variant_fp64; /* tuned: the first solve at a given padded batch size runs each
                                   phase's loop from the host with the shapes rotated body by body
                                   and keeps the one that moved the most bytes per ms (instances
                                   with fewer than 2^24 transition-weights per sweep use shape 0);
                                   >= 0 forces one (0 .. 3).  Every shape gives bit-identical
                                   results.                                                         */
    int32_t skip_unchanged;     /* 1 (default): a sweep does not recompute a work item none of whose
                                   inputs changed in the previous sweep (the values it would write
                                   are the ones already there, so results are bit-identical);
                                   0: every sweep recomputes every item of an active product      */
    int32_t polish;             /* the second phase of a mixed-precision solve: 0 (default) = FP32
                                   residual correction on a double-float table (V = B + d with B
                                   the FP32 phase's values, d iterated in FP32); 1 = the sweeps in
                                   double-float on V itself.  0 holds one more value array in FP32
                                   and a [state-action][Kp] FP32 table on the device.             */
    int32_t eval_block;         /* 1 (default): Algorithm 4 evaluates each pair whose values fit in
                                   one block's shared memory (n + 1 <= 7168 states) with one block
                                   running all its sweeps in one launch; larger pairs, or all pairs
                                   with 0, run the multi-launch sweep loop.  Same results.         */
    int32_t in_place;           /* 0 (default): Algorithm 3's sweeps are synchronous (Jacobi: each
                                   sweep reads the previous sweep's values only), so results do not
                                   depend on scheduling, kernel shape or batch; 1: values are
                                   updated in place, as the paper's printed loop does (a sweep may
                                   read values already updated in the same sweep, in an order set
                                   by the GPU's scheduling).  Same fixed point and stopping rule;
                                   usually fewer sweeps; results reproducible only to the
                                   tolerance.  Algorithm 4 stays synchronous.                       */
    int32_t item_warps_max;     /* most warps that share one sweep work item: a sweep whose work list is
                                   short (the late sweeps of a loop) splits each item's states over up
                                   to this many warps, 1, 2, 4 or 8; 0 (default) = 8 (capped at what
                                   one item fills).  Same results for every value.               */
    int32_t tail_items;         /* the end of each Algorithm 3 sweep loop: once the loop's work list
                                   holds at most this many work items, its remaining sweeps run in
                                   one cooperative launch (every block resident; a grid-wide barrier
                                   between sweeps instead of a launch per sweep) in which each warp
                                   group keeps one item, with its staged rows, for the rest of the
                                   loop.  -1 (default): a quarter of that launch's warps (every
                                   item then split over two or more warps, each warp's share one
                                   staged batch); 0: no such launch (one launch per sweep to the
                                   end); > 0: this many, at most one item per warp of the launch.
                                   Same results for every value.  Each barrier wait is bounded
                                   (1 s): a wait that runs out ends the launch and the call returns
                                   MORAP_ECUDA.  The cooperative launch needs the whole GPU's
                                   resident blocks, so the serving workers (several loops at once on
                                   one GPU) run without it; contexts that solve at the same time on
                                   one GPU (several streams or threads) should set 0 as well.      */
} morap_config;

typedef struct morap_ctx morap_ctx;

/* Fill *cfg with the defaults listed above. */
void morap_config_default(morap_config *cfg);

/* Create a context on cfg->device (cfg may be NULL for the defaults).
 * Errors: EINVAL (bad config), ECUDA. */
int morap_ctx_create(const morap_config *cfg, morap_ctx **out);

/* Release every device and host resource of the context.  NULL is a no-op. */
int morap_ctx_destroy(morap_ctx *ctx);

/* Message of the calling thread's most recent failed call ("" if none).
 * The pointer stays valid until the thread's next failing call. */
const char *morap_last_error(void);

/* Self-check of the bounded wait in the grid barrier that separates the
 * sweeps of a tail launch (config tail_items): one cooperative launch of that
 * barrier on `device` in which one block never arrives, so every other
 * block's wait runs out (after 1 s) and the kernel ends by itself.
 * *timed_out = 1 when the waits ran out and reported it, *ms = the launch's
 * device time.  Synchronous; allocates and frees one small device buffer; no
 * context needed.  Errors: EINVAL (NULL output), ECUDA. */
int morap_barrier_selfcheck(int32_t device, int32_t *timed_out, double *ms);

/* ---------------------------------------------------------------- models */

/* Add agent i (a labelled MDP with a cost per action, Sec. 2 "Markov
 * Decision Process"; its reward structure rho_i(s, a) = -cost(s, a)).
 *   n_states        |S|, >= 1;  s0 the initial state
 *   state_ptr[n+1]  actions of state s are rows state_ptr[s] .. state_ptr[s+1]-1
 *                   (every state needs >= 1 enabled action); the local index of
 *                   an action is its position in that range
 *   sa_ptr[SA+1]    successors of row a are sa_ptr[a] .. sa_ptr[a+1]-1
 *   succ[T], prob[T] successor states and probabilities; each row must sum to
 *                   1 within 1e-9 (enabled actions, Sec. 2); duplicates are
 *                   merged and zero entries dropped
 *   cost[SA]        finite, >= 0
 *   label_ptr[n+1], label_ap[]  L(s): the atomic propositions (any int32 ids)
 *                   holding in state s
 * *agent_id receives the agent's index (0, 1, ... in call order).
 * Errors: EINVAL (message names the offending row), ESTATE after build. */
int morap_add_agent(morap_ctx *ctx, int32_t n_states, int32_t s0, const int32_t *state_ptr,
                    const int32_t *sa_ptr, const int32_t *succ, const double *prob, const double *cost,
                    const int32_t *label_ptr, const int32_t *label_ap, int32_t *agent_id);

/* Add task j, a DFA (Q, q0, Q_F, 2^AP, delta) whose accepting locations are
 * sinks (Sec. 2 "Deterministic Finite Automata").
 *   n_ap in 0..8    letters are 0 .. 2^n_ap - 1, bit b set iff ap_ids[b] in L(s)
 *   delta[n_locs * 2^n_ap]  delta[q * 2^n_ap + letter]
 *   accepting[n_locs]       1 for accepting locations
 * The library computes the traps Q_R (no run reaches Q_F), done_j = Q_F u Q_R,
 * and the pre-sinks carrying rho_{j+|I|} (Sec. 3.1).  Every transition into
 * Q_F that does not leave from a pre-sink is redirected through one added
 * pre-sink location, so the one-off reward counts every accomplishment.
 * Errors: EINVAL (accepting location not a sink, target out of range),
 * ESTATE after build. */
int morap_add_task(morap_ctx *ctx, int32_t n_locs, int32_t q0, int32_t n_ap, const int32_t *ap_ids,
                   const int32_t *delta, const uint8_t *accepting, int32_t *task_id);

/* Restrict the context to a list of products (before morap_build): only
 * M_{agent[e]} (x) A_{task[e]} for e = 0 .. n_pairs-1 is built, and product p
 * of the context is the p-th pair of the list (without a list, product p is
 * i * |J| + j for every agent i and task j).  For drivers that spread the
 * independent products of one instance over several devices (Sec. 3.2: the
 * products share nothing until the assignment), one device's share per
 * context.  A context with a list answers morap_solve (c_out[K][n_pairs],
 * the list's order) and morap_evaluate; morap_supporting_points and
 * morap_query need every pair (ESTATE).
 * Errors: EINVAL (negative index, a pair listed twice; an agent or task not
 * added is reported by morap_build), ESTATE after build. */
int morap_select_pairs(morap_ctx *ctx, int32_t n_pairs, const int32_t *agent, const int32_t *task);

typedef struct morap_footprint {
    int64_t n_products;   /* |I| * |J|                                        */
    int64_t n_states;     /* product states over all products (done slots included) */
    int64_t n_sa;         /* state-action rows                                 */
    int64_t n_trans;      /* transitions                                       */
    int64_t csr_bytes;    /* device bytes of the product CSRs                  */
    int64_t device_bytes; /* all device bytes the context holds now            */
    int64_t h2d_bytes;    /* host->device bytes this build copied              */
} morap_footprint;

/* Upload the agents and tasks and build all |I| x |J| product MDPs on the
 * device (Sec. 2 "Product MDP": P'((s,q),a,(s',q')) = P(s,a,s') iff
 * q' = delta(q, L(s')); product states whose location is in done_j are one
 * absorbing slot of value 0).  Device-resident until the context is
 * destroyed; calling it again rebuilds in place.  fp may be NULL.
 * Errors: ESTATE (no agent or task), ENOMEM (hbm_budget), ECUDA. */
int morap_build(morap_ctx *ctx, void *stream, morap_footprint *fp);

/* Re-run the product construction on the device from the agent and task
 * arrays already resident since the last morap_build (no host transfer).
 * Enqueued on `stream`; returns once the launches are queued.
 * Errors: ESTATE (no build yet), ECUDA. */
int morap_rebuild(morap_ctx *ctx, void *stream);

/* ------------------------------------------------------------ the solver */

/* Algorithm 2, loop 1 for K weight vectors at once, plus Algorithm 4 for the
 * cost and probability of EVERY product under its returned scheduler.
 *   W[K][|I|+|J|]           weight vectors (entries >= 0)
 *   c_out[K][|I|][|J|]      c_ij = optimal scalarised value at (s_i0, q_j0)
 *                           ([K][n_pairs] in list order for a context with
 *                           morap_select_pairs)
 *   rcost_out, rprob_out    same layout: E[rho_i] and E[rho_{|I|+j}] under
 *                           the returned scheduler (may be NULL to skip
 *                           Algorithm 4)
 *   status_out[K][|I|][|J|] may be NULL; MORAP_OK or MORAP_ENOTCONV per pair
 * The returned scheduler mu keeps, in each state, the action Algorithm 3 last
 * recorded when its Q-value on the final values is within tau_policy of the
 * maximum, and otherwise the lowest-index maximiser.
 * Returns ENOTCONV if any pair hit the sweep cap (outputs still written). */
int morap_solve(morap_ctx *ctx, int32_t K, const double *W, void *stream, double *c_out, double *rcost_out,
                double *rprob_out, int32_t *status_out);

/* Algorithm 4 (both objectives) for chosen (product, weight) pairs under
 * the schedulers of the last morap_solve / morap_supporting_points batch on
 * this context (its last block of at most 64 weights): pair e is product
 * pair_product[e] (= i * |J| + j) under weight pair_weight[e] (index within
 * that block).  rcost_out[e] = E[rho_i], rprob_out[e] = E[rho_{|I|+j}].
 * This is loop 2 of Algorithm 2 run separately, for drivers that choose the
 * assignment themselves (e.g. from c values gathered across devices).
 * Errors: EINVAL (index out of range), ESTATE (no solve since the build),
 * ENOTCONV (a pair reached the sweep cap; outputs still written), ECUDA. */
int morap_evaluate(morap_ctx *ctx, int32_t n_pairs, const int32_t *pair_product, const int32_t *pair_weight,
                   void *stream, double *rcost_out, double *rprob_out);

/* Algorithm 2 in full for K weight vectors in one batch: loop 1 over all
 * products, the assignment f maximising sum_j c_{f(j), j} (Hungarian;
 * |I| != |J| is padded with zero-valued dummy agents or tasks), and loop 2
 * (Algorithm 4) on the assigned products only.
 *   r_out[K][|I|+|J|]   the supporting point r for each w (agents without a
 *                       real task and tasks without a real agent get 0)
 *   assign_out[K][|J|]  f(j) (an agent index, or -1 for a dummy agent); may be NULL
 *   c_out[K][|I|][|J|]  may be NULL
 * Errors as morap_solve. */
int morap_supporting_points(morap_ctx *ctx, int32_t K, const double *W, void *stream, double *r_out,
                            int32_t *assign_out, double *c_out);

/* Statistics of the last morap_solve / morap_supporting_points call. */
typedef struct morap_solve_stats {
    int32_t K;                /* weights in the batch                              */
    int32_t fp32_sweeps;      /* sweeps of the FP32 phase (0 if unused), counted in bodies of six */
    int32_t fp64_sweeps;      /* sweeps of the second (polish) phase                 */
    int32_t eval_sweeps;      /* sweep launches of the evaluation phase             */
    int64_t updates_fp32;     /* transition-updates executed: one (s,a,s') term for one weight in one
                                 sweep (work items skipped exactly are not counted)   */
    int64_t updates_fp64;
    int64_t updates_eval;     /* one (s, mu(s), s') term for one objective (cost or probability) */
    int64_t bytes_fp32;       /* algorithmic bytes the sweeps had to move           */
    int64_t bytes_fp64;
    int64_t bytes_eval;
    double ms_fp32;           /* device time of each phase's sweep loop (CUDA events on the
                                 launching stream around the loop's graph launch)       */
    double ms_fp64;
    double ms_finalise;
    double ms_eval;
    double ms_host;           /* host assignment and bookkeeping inside the call    */
    double ms_total;          /* whole call, host wall clock                        */
    int32_t pairs_not_converged;
    int32_t eval_pairs;
    int64_t h2d_bytes;        /* host->device bytes the call copied                  */
    int64_t d2h_bytes;        /* device->host bytes the call copied                  */
    int32_t kernel_launches;  /* kernels of this library the call launched          */
    int32_t variant_fp32;     /* kernel shapes the sweeps used (-1: phase not run)  */
    int32_t variant_fp64;
    int32_t polish;           /* the second phase's form: 0 = FP32 residual correction,
                                 1 = double-float sweeps (always 1 without an FP32 phase) */
    double ms_tune;           /* host time the context has spent tuning shapes      */
    int64_t skipped_fp32;     /* work-item sweeps skipped exactly (nothing they read had
                                 changed; their values are reproduced bit for bit)     */
    int64_t skipped_fp64;
    int64_t work_items;       /* work items (64 states of one product) per full sweep  */
    int64_t computed_fp32;    /* work-item sweeps computed (skipped ones excluded)   */
    int64_t computed_fp64;
    int64_t anchored_states;  /* (state, weight) entries whose recorded action was not kept and
                                 that the scheduler's anchoring rounds decided          */
    int32_t tail_sweeps_fp32; /* of fp32_sweeps / fp64_sweeps: the sweeps the loop's tail launch
                                 ran (config tail_items)                                */
    int32_t tail_sweeps_fp64;
} morap_solve_stats;

int morap_last_solve_stats(const morap_ctx *ctx, morap_solve_stats *out);

/* The plain one-model-at-a-time FP64 GPU value iteration (the baseline the
 * paper's GPU path uses: per model and weight, a CSR SpMV kernel, a segmented
 * max/argmax kernel with the residual, and a host convergence check after
 * every sweep; then Algorithm 4 the same way).
 *   n_pairs, pair_product[n]  product index p = i*|J| + j
 *   pair_w[n][2]              (w_i, w_{|I|+j}) for each pair
 *   c_out, rcost_out, rprob_out [n]
 * stats_out may be NULL: {sweeps_vi, sweeps_eval, updates, milliseconds}. */
int morap_solve_plain(morap_ctx *ctx, int32_t n_pairs, const int32_t *pair_product, const double *pair_w,
                      void *stream, double *c_out, double *rcost_out, double *rprob_out, double *stats_out);

/* Allocation-free plain value iteration for one product and one weight
 * vector (the paper has no counterpart: this is an interface for callers).
 * Some callers may not allocate device memory: hosts that hand every byte
 * of the GPU to their own memory pool and treat any outside cudaMalloc as a
 * leak or a deadlock risk, and real-time loops that forbid allocation after
 * start-up.  This call allocates nothing (no cudaMalloc, cudaFree, pinned
 * host memory or allocating library routine): the caller passes the inputs
 * and outputs, and the scratch it needs (second value buffer, state-action
 * values, recorded actions, residual and round words) lives in one static
 * device array of about 6.3 MB that every GPU which loads this library
 * holds until the process exits.
 *   Limits: n_states <= 131071 (plus the done slot) and n_sa <= 655360;
 *   larger products are rejected with MORAP_EINVAL.
 *   Inputs (device memory, the product's CSR with local indices, e.g. as
 *   morap_product_download returns it): state_sa[n_states + 1] and
 *   sa_tr[n_sa + 1] (uint32), col[] (int32; n_states is the absorbing done
 *   slot), prob[] and cost[] (double); pre_begin = first state at a pre-sink
 *   location; init_state = the state whose value is returned in *c_out.
 *   Outputs: values[n_states + 1] (device, double; the final iterate with
 *   values[n_states] = 0), policy[n_states] (device, int32: the returned
 *   scheduler), *c_out and *sweeps_out (host, either may be NULL).
 *   The computation is morap_solve_plain's: Algorithm 3 in FP64 from 0 with
 *   a host convergence check after every sweep, then the scheduler reading.
 * The call is synchronous: it waits on `stream` after every sweep and reads
 * the residual on the host, so it cannot run inside a stream capture (a
 * capturing stream is refused with MORAP_EINVAL before anything is
 * enqueued).  The stream and every buffer must belong to the current
 * device (MORAP_EINVAL otherwise), because the scratch used is the current
 * device's copy of the array.  The first call on each device looks up that
 * copy's address (cudaGetSymbolAddress) with the device current.  Every
 * call on a device shares the one array and clears what must start at
 * zero; calls that overlap on the GPU (other threads or streams) race on it.
 * Errors: EINVAL (sizes over the limits, bad arguments, wrong device,
 * capturing stream), ENOTCONV (sweep cap reached; outputs hold the last
 * iterate), ECUDA. */
int morap_plain_vi_noalloc(int32_t n_states, int32_t n_sa, const uint32_t *state_sa, const uint32_t *sa_tr,
                           const int32_t *col, const double *prob, const double *cost, int32_t pre_begin,
                           int32_t init_state, double w_cost, double w_prob, double eps, double tau,
                           int32_t max_sweeps, void *stream, double *values, int32_t *policy, double *c_out,
                           int32_t *sweeps_out);

/* ------------------------------------------------------ point queries */

typedef struct morap_point_result {
    int32_t feasible;     /* 1 iff t_down == t when the loop stopped (Cor. (ii))      */
    int32_t iterations;   /* supporting points computed                               */
    int32_t converged;    /* 1 iff ||t_down - t_up|| <= eps when it stopped           */
    int32_t status;       /* MORAP_OK or the first failing status                     */
    double distance;      /* ||t_down - t_up||                                         */
    double *t_up;         /* caller-provided [|I|+|J|] or NULL                          */
    double *t_down;       /* caller-provided [|I|+|J|] or NULL                          */
    double *w_hist;       /* caller-provided [max_iter][|I|+|J|] or NULL                */
    double *r_hist;       /* caller-provided [max_iter][|I|+|J|] or NULL                */
    double *lambda;       /* caller-provided [max_iter] or NULL: the synthesis — convex
                             weights over the supporting points r_hist with
                             sum_l lambda_l r_l >= t_up (>= t when feasible).  Running
                             point l's assignment and schedulers with probability
                             lambda_l achieves that vector in expectation (Sec. 3.3)  */
    int32_t *assign_hist; /* caller-provided [max_iter][|J|] or NULL: the task
                             assignment of each point (agent of task j, -1 for none);
                             morap_query only.  A point's schedulers are those of
                             morap_solve for its weight vector w_hist[l] (results are
                             deterministic)                                          */
} morap_point_result;

/* Algorithm 1 for threshold t = (c, p) with norm ||v|| = sqrt(v^T M v)
 * (M symmetric positive definite, [n][n] row-major, NULL = identity) and
 * tolerance eps.  The first direction is e_1; after each supporting point
 * the outer bound t_down (projection of t onto {z : w'.z <= w'.r'}) is
 * updated when w.r < w.t_down, the inner bound t_up (projection onto
 * down(conv Phi)) is refreshed, and the loop stops when
 * ||t_down - t_up|| <= eps or after max_iter points.
 * Errors: EINVAL, ENOTCONV (max_iter reached or a sweep cap), ECUDA. */
int morap_query(morap_ctx *ctx, const double *t, const double *M, double eps, int32_t max_iter, void *stream,
                morap_point_result *res);

/* Algorithm 1 in the verification-only setting (Sec. 5, Experiment 2): the
 * outer-bound projection is replaced by a stop, so the loop ends with
 * feasible = 0 at the first supporting point with w.r < w.t (t is separated
 * from the achievable set by that hyperplane), or with feasible = 1 once
 * ||t - t_up|| <= eps.  It runs the same directions and points as
 * morap_query up to that point (t_down stays t), so the verdict is
 * morap_query's and it never needs more iterations.  converged = 1 when
 * the verdict is final.  Same arguments and errors as morap_query. */
int morap_verify(morap_ctx *ctx, const double *t, const double *M, double eps, int32_t max_iter, void *stream,
                 morap_point_result *res);

/* Algorithm 1 with the supporting points supplied by the caller, one at a
 * time: for drivers that compute them elsewhere (products sharded over
 * several devices or processes, another solver).  morap_query is this loop
 * fed by morap_supporting_points on one context.  Host-only; the handle is
 * owned by the caller and not thread-safe.
 *   morap_pareto_create: n objectives, t[n], M as for morap_query (copied),
 *     eps >= 0, max_iter >= 1.  Errors: EINVAL.
 *   morap_pareto_next: *done = 1 once the loop stopped; otherwise w_out[n]
 *     receives the direction whose supporting point the next step needs
 *     (e_1 first).
 *   morap_pareto_step: r[n] = the supporting point for that direction (the
 *     r of Algorithm 2); solve_status = the status of the call that computed
 *     it (MORAP_OK or MORAP_ENOTCONV, which is carried into the result).
 *     Errors: EINVAL (null, non-finite r), ESTATE (the loop already stopped).
 *   morap_pareto_result: fills *res as morap_query does; returns its status.
 */
typedef struct morap_pareto morap_pareto;
int morap_pareto_create(int32_t n, const double *t, const double *M, double eps, int32_t max_iter,
                        morap_pareto **out);
/* As morap_pareto_create with a mode: MORAP_PARETO_SYNTHESIS (Algorithm 1,
 * what morap_pareto_create makes) or MORAP_PARETO_VERIFY (the
 * verification-only loop of morap_verify).  Errors: EINVAL. */
#define MORAP_PARETO_SYNTHESIS 0
#define MORAP_PARETO_VERIFY 1
int morap_pareto_create_mode(int32_t n, const double *t, const double *M, double eps, int32_t max_iter,
                             int32_t mode, morap_pareto **out);
int morap_pareto_next(const morap_pareto *ps, double *w_out, int32_t *done);
int morap_pareto_step(morap_pareto *ps, const double *r, int32_t solve_status);
int morap_pareto_result(const morap_pareto *ps, morap_point_result *res);
void morap_pareto_destroy(morap_pareto *ps);

/* ------------------------------------------------------------- serving
 * Continuous batching of threshold-point queries (Algorithm 1) over several
 * resident instances (built contexts).  Each query runs Algorithm 1 with
 * M = I and the server's eps / max_iter.  A query waiting for its next
 * supporting point joins the next device round: an idle instance takes its
 * own waiting queries as one morap_supporting_points batch on its own
 * stream, or, with merge_instances, one round serves the waiting queries of
 * every instance of a group as the weight columns of one batch (a query's
 * column weighs only its instance's products).
 * Admission: queries are admitted in arrival order while the device bytes of
 * their weight slots (26 bytes per product state of the instance) fit
 * hbm_budget (0 = no limit); at least one query is always admitted.
 * A query's result does not depend on the batch it rides in.
 * The instances must outlive the server and must not be used by the caller
 * while the server runs. */
typedef struct morap_server morap_server;

typedef struct morap_server_config {
    size_t hbm_budget;  /* admission budget in bytes, 0 = none                   */
    int32_t max_batch;  /* queries per device batch, 1..64 (default 64)          */
    int32_t n_workers;  /* host threads (default 8): Algorithm 1 steps, or the
                           instances' batches without merge_instances          */
    double eps;         /* Algorithm 1 tolerance of every query (default 1e-6)   */
    int32_t max_iter;   /* supporting points per query (default 64)              */
    int32_t merge_instances; /* 0 (default): each instance batches its own queries on
                           its own stream; 1: one device round takes the waiting
                           queries of every instance of a group (instances with
                           the same arithmetic and a similar size), on a context
                           holding the group's products (built at server
                           creation; the instances' own contexts are left
                           untouched).  A merged round computes every weight
                           column of every product it touches: lower latency at
                           light load, lower saturation throughput           */
} morap_server_config;

typedef struct morap_serving_stats {
    int64_t submitted, completed, batches;
    double mean_batch;     /* queries per batch                                    */
    double p50_ms, p99_ms; /* submit-to-completion latency percentiles             */
    double queries_per_s;  /* completed / (last completion - first submit)         */
    double wall_s;
    int64_t bytes_in_use;  /* admitted weight-slot bytes                            */
} morap_serving_stats;

void morap_server_config_default(morap_server_config *cfg);
int morap_server_create(morap_ctx *const *instances, int32_t n_instances, const morap_server_config *cfg,
                        morap_server **out);
/* Stops the threads (queries still in flight are abandoned) and frees the server. */
int morap_server_destroy(morap_server *server);
/* Non-blocking.  t has |I| + |J| entries of that instance.  Errors: EINVAL. */
int morap_submit(morap_server *server, int32_t instance, const double *t, int64_t *ticket_out);
/* MORAP_EBUSY while the query runs; then fills *res as morap_query does
 * (w_hist / r_hist, when given, need iterations x (|I|+|J|) entries). */
int morap_poll(morap_server *server, int64_t ticket, morap_point_result *res);
/* Block until every submitted query completed or timeout_s passed (EBUSY). */
int morap_server_wait(morap_server *server, double timeout_s);
int morap_server_stats(morap_server *server, morap_serving_stats *stats);

/* ------------------------------------------------ host-side building blocks
 * These run on the CPU only (no device needed) and are what morap_query and
 * morap_supporting_points use. */

/* The synthesised random assignment (Sec. 3.3, the synthesis after
 * Algorithm 1; Lemma 2): running point l's deterministic assignment f_l with
 * probability lambda_l assigns agent i to task j with probability
 *   P_out[i][j] = sum_l lambda_l [f_l(j) = i]      ([n_agents][n_tasks]).
 * lambda[n_points] and assign_hist[n_points][n_tasks] are what
 * morap_query returns in morap_point_result (lambda, assign_hist; -1 marks
 * a task no agent does).  With the lambda of a query (sum 1) P is doubly
 * substochastic.  Host-only.  Errors: EINVAL (null pointer, negative or
 * non-finite lambda, agent index out of range). */
int morap_random_assignment(int32_t n_points, int32_t n_agents, int32_t n_tasks, const double *lambda,
                            const int32_t *assign_hist, double *P_out);

/* Hungarian assignment: f_out[j] = the row assigned to column j maximising
 * sum_j C[f(j)][j] for a square C [n][n] (row-major, rows = agents). */
int morap_assign_max(int32_t n, const double *C, int32_t *f_out);

/* Algorithm 2's assignment for each of K value matrices c[K][|I|][|J|]
 * (c_ij = optimal scalarised value of agent i on task j): with |I| != |J|
 * the matrix is padded with zero rows or columns to a square one (a padded
 * agent does nothing, a padded task is not done); assign_out[K][|J|] = the
 * agent given task j, or -1 when no agent is.  The same routine the
 * supporting-point calls use. */
int morap_assign_tasks(int32_t n_agents, int32_t n_tasks, int32_t K, const double *c, int32_t *assign_out);

/* argmin_z ||t - z||_M subject to A z <= b; A is [m][n] row-major. */
int morap_project_halfspaces(int32_t n, int32_t m, const double *t, const double *A, const double *b,
                             const double *M, double *z_out);

/* argmin_x ||t - x||_M over x in down(conv{Phi_0..Phi_{m-1}}); Phi is [m][n]. */
int morap_project_down_hull(int32_t n, int32_t m, const double *t, const double *Phi, const double *M,
                            double *x_out);

/* Task preprocessing as morap_add_task does it, exposed for checking:
 * n_locs_out = locations after the optional pre-sink insertion (<= n_locs+1),
 * flags_out[n_locs+1]: bit0 accepting, bit1 trap, bit2 pre-sink, bit3 done. */
int morap_task_preprocess(int32_t n_locs, int32_t q0, int32_t n_ap, const int32_t *delta,
                          const uint8_t *accepting, int32_t *n_locs_out, uint8_t *flags_out);

/* ------------------------------------------------------ introspection */

/* info_out[10] for product p = i*|J| + j: {S_agent, n_nondone_locations,
 * n_states (incl. the done slot), n_sa, n_trans, init_local (local index of
 * (s_i0, q_j0); the done slot when q_j0 is done), state_offset, pre_begin
 * (first local state whose location is a pre-sink), agent i, task j}. */
int morap_product_info(const morap_ctx *ctx, int32_t p, int64_t *info_out);

/* Copy product p's CSR to host arrays sized from morap_product_info:
 * state_sa[n_states+1], sa_tr[n_sa+1] (both rebased to 0), col[n_trans]
 * (local state index; n_states-1 is the done slot), prob[n_trans],
 * cost[n_sa], loc_out[n_nondone_locations] (the DFA location, after
 * preprocessing, of each product location index).  Any pointer may be NULL. */
int morap_product_download(morap_ctx *ctx, int32_t p, int64_t *state_sa, int64_t *sa_tr, int32_t *col,
                           double *prob, double *cost, int32_t *loc_out);

/* After morap_solve: the returned scheduler (local action index) and the final
 * FP64 values of weight k on product p, over its local states. */
int morap_last_policy(morap_ctx *ctx, int32_t k, int32_t p, uint8_t *mu_out, double *values_out);

#ifdef __cplusplus
}
#endif

#endif /* MORAP_H */

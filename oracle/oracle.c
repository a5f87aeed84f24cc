/*
 * Plain FP64 CPU oracle for the per-product computations of the method.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into oracle/liboracle.so
 * and may be loaded only by the tests, by __graft_entry__.smoke() and by the
 * CPU-baseline leg of bench.py.  The CUDA engine never links, loads or calls
 * it, and it shares no code with the engine.
 *
 * Everything here is written for readability, one state at a time, in the
 * order the paper states it:
 *   - orc_build_product  : the product MDP M (x) A (Sec. 2 "Product MDP",
 *                          Sec. 3.1 agent-task products with done_j)
 *   - orc_alg3           : value iteration for the scalarised reward with the
 *                          policy record of Algorithm 3 (Appendix A.4)
 *   - orc_finalise_policy: the reading used for which recorded action is the
 *                          returned scheduler when actions tie
 *   - orc_alg4           : fixed-policy value iteration of Algorithm 4
 *
 * Conventions shared with the Python side (oracle/core.py):
 *   product state u = k*S + s for the k-th non-done DFA location and agent
 *   state s; one extra absorbing state DONE = n_nd*S with no actions and
 *   value 0 collects every successor whose location is accepting or a trap.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Product construction.  P'((s,q), a, (s',q')) = P(s,a,s') when
 * q' = delta(q, L(s')) (labels are read on the successor), and 0 otherwise.
 * Successors whose location is done map to DONE; duplicates are merged by
 * summing their probabilities.  The caller sizes the outputs for the worst
 * case: state_ptr[n_nd*S+2], sa_ptr[n_nd*SA+1], col/prob[n_nd*T],
 * sa_cost[n_nd*SA].  Returns the number of transitions written. */
long orc_build_product(int S, const int *a_state_ptr, const int *a_sa_ptr, const int *a_succ,
                       const double *a_prob, const double *a_cost, const int *letter, int n_nd,
                       const int *nd_loc, const int *nd_pos, const int *delta, int n_letters,
                       int *state_ptr, int *sa_ptr, int *col, double *prob, double *sa_cost)
{
    const int done = n_nd * S;
    long n_tr = 0;
    int n_sa = 0;
    for (int k = 0; k < n_nd; ++k) {
        const int q = nd_loc[k];
        for (int s = 0; s < S; ++s) {
            const int u = k * S + s;
            state_ptr[u] = n_sa;
            for (int a = a_state_ptr[s]; a < a_state_ptr[s + 1]; ++a) {
                sa_ptr[n_sa] = (int)n_tr;
                sa_cost[n_sa] = a_cost[a];
                const long row_begin = n_tr;
                for (int t = a_sa_ptr[a]; t < a_sa_ptr[a + 1]; ++t) {
                    const int s2 = a_succ[t];
                    const int q2 = delta[q * n_letters + letter[s2]];
                    const int u2 = nd_pos[q2] < 0 ? done : nd_pos[q2] * S + s2;
                    long found = -1;
                    for (long r = row_begin; r < n_tr; ++r)
                        if (col[r] == u2) found = r;
                    if (found >= 0) {
                        prob[found] += a_prob[t];
                    } else {
                        col[n_tr] = u2;
                        prob[n_tr] = a_prob[t];
                        ++n_tr;
                    }
                }
                ++n_sa;
            }
        }
    }
    state_ptr[done] = n_sa;     /* DONE has no actions */
    state_ptr[done + 1] = n_sa;
    sa_ptr[n_sa] = (int)n_tr;
    return n_tr;
}

/* Q(u, a) = rew[a] + sum_{u'} P(u, a, u') x[u'] for one state-action row. */
static double q_value(int a, const int *sa_ptr, const int *col, const double *prob, const double *rew,
                      const double *x)
{
    double acc = rew[a];
    for (int t = sa_ptr[a]; t < sa_ptr[a + 1]; ++t)
        acc += prob[t] * x[col[t]];
    return acc;
}

/* Algorithm 3.  x holds the start vector on entry (zero for the paper's
 * algorithm) and the last sweep's values on exit.  Sweeps are synchronous
 * (every y is computed from the previous sweep's x), and the loop is read as
 * do { ... } while (!stable) with `stable` reset at the top of each sweep.
 * When |y_u - x_u| > eps the maximising action (the lowest local index among
 * equal maxima) is recorded in a_rec[u]; a_rec keeps its initial contents
 * elsewhere.  Returns 0 on convergence, 1 when max_sweeps was reached. */
int orc_alg3(int n, const int *state_ptr, const int *sa_ptr, const int *col, const double *prob,
             const double *rew, double eps, int max_sweeps, double *x, int *a_rec, int *sweeps_out)
{
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    int sweeps = 0, stable = 0;
    while (!stable && sweeps < max_sweeps) {
        stable = 1;
        for (int u = 0; u < n; ++u) {
            const int a0 = state_ptr[u], a1 = state_ptr[u + 1];
            if (a0 == a1) {            /* DONE: absorbing, value 0 */
                y[u] = x[u];
                continue;
            }
            double best = q_value(a0, sa_ptr, col, prob, rew, x);
            int best_a = 0;
            for (int a = a0 + 1; a < a1; ++a) {
                const double qa = q_value(a, sa_ptr, col, prob, rew, x);
                if (qa > best) {
                    best = qa;
                    best_a = a - a0;
                }
            }
            y[u] = best;
            if (fabs(best - x[u]) > eps) {
                stable = 0;
                a_rec[u] = best_a;
            }
        }
        memcpy(x, y, sizeof(double) * (size_t)n);
        ++sweeps;
    }
    free(y);
    *sweeps_out = sweeps;
    return stable ? 0 : 1;
}

/* The scheduler returned for Algorithm 3.  On the final values x, keep the
 * recorded action when its Q-value is within tau of the maximum; such
 * states, and the absorbing DONE state, are "anchored".  A state whose
 * recorded action fell more than tau behind (its value kept drifting by
 * steps below eps after the last record) takes an action within tau of the
 * maximum that is not a self-loop (an action whose only successor is u
 * itself) and reaches, with positive probability, a state other than u that
 * is already anchored: in rounds, each round deciding every remaining state
 * from the anchors of the rounds before it (lowest-index such action), and
 * anchoring the states it decided.  The levels so formed lead every decided
 * state to an anchor with probability one, so two states that tie can never
 * send the run back and forth between themselves forever (with a zero
 * weight on the cost every move is free, and "go to the neighbour" ties
 * with the maximum in a region of equal values).  States no round decides
 * take the lowest-index non-self-loop action within tau of the maximum, and
 * a self-loop only when nothing else is within tau.  (At a fixed point a
 * zero-reward self-loop always ties with the maximum, so preferring it would
 * return "stay forever" in states where the value came from moving.) */
static int is_self_loop(int u, int a, const int *sa_ptr, const int *col)
{
    return sa_ptr[a + 1] - sa_ptr[a] == 1 && col[sa_ptr[a]] == u;
}

static double max_q(int u, const int *state_ptr, const int *sa_ptr, const int *col, const double *prob,
                    const double *rew, const double *x)
{
    double best = q_value(state_ptr[u], sa_ptr, col, prob, rew, x);
    for (int a = state_ptr[u] + 1; a < state_ptr[u + 1]; ++a) {
        const double qa = q_value(a, sa_ptr, col, prob, rew, x);
        if (qa > best)
            best = qa;
    }
    return best;
}

void orc_finalise_policy(int n, const int *state_ptr, const int *sa_ptr, const int *col, const double *prob,
                         const double *rew, const double *x, const int *a_rec, double tau, int *mu)
{
    /* anchored[u]: 1 from the start, r + 1 once decided in round r, 0 while undecided */
    int *anchored = (int *)calloc((size_t)n, sizeof(int));
    int undecided = 0;
    for (int u = 0; u < n; ++u) {
        const int a0 = state_ptr[u], a1 = state_ptr[u + 1];
        mu[u] = 0;
        if (a0 == a1) {
            anchored[u] = 1;
            continue;
        }
        const double best = max_q(u, state_ptr, sa_ptr, col, prob, rew, x);
        if (q_value(a0 + a_rec[u], sa_ptr, col, prob, rew, x) >= best - tau) {
            mu[u] = a_rec[u];
            anchored[u] = 1;
        } else {
            ++undecided;
        }
    }
    /* at most 254 rounds: the engine stamps the round in a byte; states still
     * undecided after them take the plain fallback below */
    for (int round = 1; undecided > 0 && round <= 254; ++round) {
        int decided = 0;
        for (int u = 0; u < n; ++u) {
            if (anchored[u])
                continue;
            const int a0 = state_ptr[u], a1 = state_ptr[u + 1];
            const double best = max_q(u, state_ptr, sa_ptr, col, prob, rew, x);
            for (int a = a0; a < a1 && !anchored[u]; ++a) {
                if (q_value(a, sa_ptr, col, prob, rew, x) < best - tau || is_self_loop(u, a, sa_ptr, col))
                    continue;
                for (int t = sa_ptr[a]; t < sa_ptr[a + 1]; ++t) {
                    const int v = col[t];
                    /* anchored before this round: 1 (from the start) or decided in an earlier round */
                    if (prob[t] > 0.0 && v != u && anchored[v] >= 1 && anchored[v] <= round) {
                        mu[u] = a - a0;
                        anchored[u] = round + 1;
                        ++decided;
                        break;
                    }
                }
            }
        }
        undecided -= decided;
        if (decided == 0)
            break;
    }
    for (int u = 0; u < n && undecided > 0; ++u) {
        if (anchored[u])
            continue;
        const int a0 = state_ptr[u], a1 = state_ptr[u + 1];
        const double best = max_q(u, state_ptr, sa_ptr, col, prob, rew, x);
        int pick = -1, pick_loop = -1;
        for (int a = a0; a < a1; ++a) {
            if (q_value(a, sa_ptr, col, prob, rew, x) < best - tau)
                continue;
            if (is_self_loop(u, a, sa_ptr, col)) {
                if (pick_loop < 0)
                    pick_loop = a - a0;
            } else if (pick < 0) {
                pick = a - a0;
            }
        }
        mu[u] = pick >= 0 ? pick : pick_loop;
    }
    free(anchored);
}

/* Algorithm 4: y_u = rew(u, mu(u)) + sum P(u, mu(u), u') x_u' from x = 0
 * (or the given start), synchronous sweeps, until max |y - x| <= eps.
 * Returns 0 on convergence, 1 when max_sweeps was reached. */
int orc_alg4(int n, const int *state_ptr, const int *sa_ptr, const int *col, const double *prob,
             const double *rew, const int *mu, double eps, int max_sweeps, double *x, int *sweeps_out)
{
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    int sweeps = 0, stable = 0;
    while (!stable && sweeps < max_sweeps) {
        stable = 1;
        for (int u = 0; u < n; ++u) {
            const int a0 = state_ptr[u], a1 = state_ptr[u + 1];
            if (a0 == a1) {
                y[u] = x[u];
                continue;
            }
            y[u] = q_value(a0 + mu[u], sa_ptr, col, prob, rew, x);
            if (fabs(y[u] - x[u]) > eps)
                stable = 0;
        }
        memcpy(x, y, sizeof(double) * (size_t)n);
        ++sweeps;
    }
    free(y);
    *sweeps_out = sweeps;
    return stable ? 0 : 1;
}

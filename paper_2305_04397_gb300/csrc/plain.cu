// The plain per-model FP64 value iteration the engine is measured against:
// one product and one weight at a time, a CSR SpMV kernel that forms every
// state-action value, a second kernel that takes the max/argmax over each
// state's actions together with the residual, and a host-side convergence
// check after every sweep (the design of the paper's GPU path: a sparse
// matrix-vector product plus one reduction kernel per iteration, with
// convergence decided on the host).
#include <cuda_runtime.h>
#include <math_constants.h>

#include "internal.h"

namespace morap {

namespace {

__global__ void k_plain_spmv(const uint32_t *sa_tr, const int32_t *col, const double *p64, const double *cost64,
                             uint32_t sa_begin, uint32_t n_sa, double wi, double wp, uint32_t pre_sa_begin,
                             uint32_t state_off, const double *x, double *q) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n_sa; v += gridDim.x * blockDim.x) {
        const uint32_t sa = sa_begin + v;
        double acc = (v >= pre_sa_begin ? wp : 0.0) - wi * cost64[sa];
        for (uint32_t t = sa_tr[sa]; t < sa_tr[sa + 1]; ++t) acc = fma(p64[t], x[(uint32_t)col[t] - state_off], acc);
        q[v] = acc;
    }
}

__device__ __forceinline__ void block_max_atomic(double r, unsigned long long *res) {
    __shared__ double s[32];
    for (int off = 16; off > 0; off >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, off));
    if ((threadIdx.x & 31) == 0) s[threadIdx.x / 32] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) m = fmax(m, s[w]);
        if (m > 0.0) atomicMax(res, (unsigned long long)__double_as_longlong(m));
    }
}

__global__ void k_plain_reduce(const uint32_t *state_sa, uint32_t state_off, uint32_t n_states, uint32_t sa_begin,
                               const double *q, const double *x, double *y, int32_t *a_rec, double eps,
                               unsigned long long *res) {
    double r = 0.0;
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n_states) {
        const uint32_t a0 = state_sa[state_off + u] - sa_begin, a1 = state_sa[state_off + u + 1] - sa_begin;
        double best = -CUDART_INF;
        int32_t ba = 0;
        for (uint32_t a = a0; a < a1; ++a)
            if (q[a] > best) {
                best = q[a];
                ba = (int32_t)(a - a0);
            }
        y[u] = best;
        r = fabs(best - x[u]);
        if (r > eps) a_rec[u] = ba;
    }
    block_max_atomic(r, res);
}

// The returned scheduler (the reading of the oracle and the batched
// finaliser): keep the recorded action when its Q is within tau of the
// maximum (the state is then "anchored", and a_rec[u] becomes the flag 1);
// otherwise the lowest-index near-maximiser that is not a self-loop (or a
// self-loop when nothing else is within tau) as a provisional choice, flag
// 0, counted in *undecided.  k_plain_anchor then decides those states in
// rounds (see there).
__global__ void k_plain_finalize(const uint32_t *state_sa, const uint32_t *sa_tr, const int32_t *col,
                                 uint32_t state_off, uint32_t n_states, uint32_t sa_begin, const double *q,
                                 int32_t *a_rec, double tau, int32_t *mu, unsigned long long *undecided) {
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_states) return;
    const uint32_t a0 = state_sa[state_off + u] - sa_begin, a1 = state_sa[state_off + u + 1] - sa_begin;
    double best = -CUDART_INF;
    for (uint32_t a = a0; a < a1; ++a) best = fmax(best, q[a]);
    if (q[a0 + a_rec[u]] >= best - tau) {
        mu[u] = a_rec[u];
        a_rec[u] = 1;
        return;
    }
    int32_t pick = -1, pick_loop = -1;
    for (uint32_t a = a0; a < a1; ++a) {
        if (q[a] < best - tau) continue;
        const uint32_t sa = sa_begin + a;
        const bool self_loop = sa_tr[sa + 1] - sa_tr[sa] == 1 && (uint32_t)col[sa_tr[sa]] == state_off + u;
        if (self_loop) {
            if (pick_loop < 0) pick_loop = (int32_t)(a - a0);
        } else if (pick < 0) {
            pick = (int32_t)(a - a0);
        }
    }
    mu[u] = pick >= 0 ? pick : pick_loop;
    a_rec[u] = 0;
    atomicAdd(undecided, 1ull);
}

// One round of the anchoring: an undecided state takes the lowest-index
// action within tau of the maximum that is not a self-loop and reaches, with
// positive probability, another state anchored before this round (flag 1,
// or decided in an earlier round: flag r + 1 for round r; the done slot is
// always anchored).  States decided now get flag round + 1, which this
// round's readers treat as not yet anchored, so the result does not depend
// on the order in which threads run.
__global__ void k_plain_anchor(const uint32_t *state_sa, const uint32_t *sa_tr, const int32_t *col, const double *p64,
                               uint32_t state_off, uint32_t n_states, uint32_t sa_begin, const double *q, double tau,
                               int round, int32_t *flag, int32_t *mu, unsigned long long *decided) {
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_states || flag[u] != 0) return;
    const uint32_t a0 = state_sa[state_off + u] - sa_begin, a1 = state_sa[state_off + u + 1] - sa_begin;
    double best = -CUDART_INF;
    for (uint32_t a = a0; a < a1; ++a) best = fmax(best, q[a]);
    for (uint32_t a = a0; a < a1; ++a) {
        if (q[a] < best - tau) continue;
        const uint32_t sa = sa_begin + a;
        const uint32_t t0 = sa_tr[sa], t1 = sa_tr[sa + 1];
        if (t1 - t0 == 1 && (uint32_t)col[t0] == state_off + u) continue;  // self-loop
        for (uint32_t t = t0; t < t1; ++t) {
            const uint32_t v = (uint32_t)col[t] - state_off;
            if (!(p64[t] > 0.0) || v == u) continue;
            const int32_t f = v < n_states ? flag[v] : 1;
            if (f >= 1 && f <= round) {
                mu[u] = (int32_t)(a - a0);
                flag[u] = round + 1;
                atomicAdd(decided, 1ull);
                return;
            }
        }
    }
}

__global__ void k_plain_eval(const uint32_t *state_sa, const uint32_t *sa_tr, const int32_t *col, const double *p64,
                             const double *cost64, uint32_t state_off, uint32_t n_states, uint32_t pre_begin,
                             const int32_t *mu, int objective, const double *x, double *y, unsigned long long *res) {
    double r = 0.0;
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n_states) {
        const uint32_t sa = state_sa[state_off + u] + (uint32_t)mu[u];
        double acc = objective == 0 ? -cost64[sa] : (u >= pre_begin ? 1.0 : 0.0);
        for (uint32_t t = sa_tr[sa]; t < sa_tr[sa + 1]; ++t) acc = fma(p64[t], x[(uint32_t)col[t] - state_off], acc);
        y[u] = acc;
        r = fabs(acc - x[u]);
    }
    block_max_atomic(r, res);
}

}  // namespace

int launch_plain_spmv(const uint32_t *sa_tr, const int32_t *col, const double *p64, const double *cost64,
                      uint32_t sa_begin, uint32_t n_sa, double wi, double wp, uint32_t pre_sa_begin,
                      uint32_t state_off, const double *x, double *q, void *s) {
    if (n_sa == 0) return 0;
    const int grid = (int)((n_sa + 255) / 256);
    k_plain_spmv<<<grid, 256, 0, (cudaStream_t)s>>>(sa_tr, col, p64, cost64, sa_begin, n_sa, wi, wp, pre_sa_begin,
                                                    state_off, x, q);
    return (int)cudaGetLastError();
}

int launch_plain_reduce(const uint32_t *state_sa, uint32_t state_off, uint32_t n_states, uint32_t sa_begin,
                        const double *q, const double *x, double *y, int32_t *a_rec, double eps,
                        unsigned long long *res, void *s) {
    if (n_states == 0) return 0;
    k_plain_reduce<<<(n_states + 255) / 256, 256, 0, (cudaStream_t)s>>>(state_sa, state_off, n_states, sa_begin, q,
                                                                       x, y, a_rec, eps, res);
    return (int)cudaGetLastError();
}

int plain_finalize(const uint32_t *state_sa, const uint32_t *sa_tr, const int32_t *col, const double *p64,
                   uint32_t state_off, uint32_t n_states, uint32_t sa_begin, const double *q, int32_t *a_rec,
                   double tau, int32_t *mu, unsigned long long *counter, void *sv) {
    if (n_states == 0) return 0;
    cudaStream_t s = (cudaStream_t)sv;
    const int grid = (int)((n_states + 255) / 256);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return (int)e;
    k_plain_finalize<<<grid, 256, 0, s>>>(state_sa, sa_tr, col, state_off, n_states, sa_begin, q, a_rec, tau, mu,
                                          counter);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    unsigned long long pending = 0;
    if ((e = cudaMemcpyAsync(&pending, counter, sizeof(pending), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return (int)e;
    for (int round = 1; pending > 0 && round <= kAnchorRounds; ++round) {
        unsigned long long decided = 0;
        if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s)) != cudaSuccess) return (int)e;
        k_plain_anchor<<<grid, 256, 0, s>>>(state_sa, sa_tr, col, p64, state_off, n_states, sa_begin, q, tau, round,
                                            a_rec, mu, counter);
        if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
        if ((e = cudaMemcpyAsync(&decided, counter, sizeof(decided), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return (int)e;
        if (decided == 0) break;
        pending -= decided;
    }
    return 0;
}

int launch_plain_eval(const uint32_t *state_sa, const uint32_t *sa_tr, const int32_t *col, const double *p64,
                      const double *cost64, uint32_t state_off, uint32_t n_states, uint32_t pre_begin,
                      const int32_t *mu, int objective, const double *x, double *y, unsigned long long *res,
                      void *s) {
    if (n_states == 0) return 0;
    k_plain_eval<<<(n_states + 255) / 256, 256, 0, (cudaStream_t)s>>>(state_sa, sa_tr, col, p64, cost64, state_off,
                                                                     n_states, pre_begin, mu, objective, x, y, res);
    return (int)cudaGetLastError();
}

}  // namespace morap

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

__global__ void k_plain_finalize(const uint32_t *state_sa, const uint32_t *sa_tr, const int32_t *col,
                                 uint32_t state_off, uint32_t n_states, uint32_t sa_begin, const double *q,
                                 const int32_t *a_rec, double tau, int32_t *mu) {
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_states) return;
    const uint32_t a0 = state_sa[state_off + u] - sa_begin, a1 = state_sa[state_off + u + 1] - sa_begin;
    double best = -CUDART_INF;
    for (uint32_t a = a0; a < a1; ++a) best = fmax(best, q[a]);
    if (q[a0 + a_rec[u]] >= best - tau) {
        mu[u] = a_rec[u];
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

int launch_plain_finalize(const uint32_t *state_sa, const uint32_t *sa_tr, const int32_t *col, uint32_t state_off,
                          uint32_t n_states, uint32_t sa_begin, const double *q, const int32_t *a_rec, double tau,
                          int32_t *mu, void *s) {
    if (n_states == 0) return 0;
    k_plain_finalize<<<(n_states + 255) / 256, 256, 0, (cudaStream_t)s>>>(state_sa, sa_tr, col, state_off, n_states,
                                                                         sa_begin, q, a_rec, tau, mu);
    return (int)cudaGetLastError();
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

// Product construction on the device (Sec. 2 "Product MDP", Sec. 3.1).
//
// The product of agent i and task j keeps the agent's state and action
// shape once per non-done DFA location: product state (pl, s) has the
// actions of agent state s, and each agent transition (s, a, s', p) becomes
// ((pl, s), a, (pl', s'), p) with pl' = delta(pl, L(s')) -- the label is
// read on the successor.  Successors whose location is done (accepting or
// trap) all go to the product's single absorbing done slot (value 0) and are
// merged into one transition of the row, whose probability is their sum (in
// the agent's order), at the position of the first of them.  States and
// rows are in closed form (local state u = pl*S + s, local row v = pl*SA +
// a); the rows' transition offsets come from a count pass and a per-product
// prefix sum.
#include <cuda_runtime.h>

#include "internal.h"

namespace morap {

namespace {

// a double as an unevaluated sum hi + lo of two floats
__device__ __forceinline__ float2 to_df(double d) {
    const float h = __double2float_rn(d);
    return make_float2(h, __double2float_rn(d - (double)h));
}

// letter of task j on every agent state s: bit b set iff ap_ids[b] in L(s)
__global__ void k_letters(const ProdDesc *prods, int P, const AgentDesc *agents, const TaskDesc *tasks,
                          const int32_t *label_ptr, const int32_t *label_ap, const int32_t *ap_ids,
                          uint8_t *letters) {
    for (int p = blockIdx.y; p < P; p += gridDim.y) {
        const ProdDesc pd = prods[p];
        const AgentDesc ad = agents[pd.agent];
        const TaskDesc td = tasks[pd.task];
        for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ad.S; s += gridDim.x * blockDim.x) {
            const int32_t l0 = label_ptr[ad.lp_off + s], l1 = label_ptr[ad.lp_off + s + 1];
            unsigned int letter = 0;
            for (int32_t k = l0; k < l1; ++k) {
                const int32_t ap = label_ap[ad.la_off + k];
                for (int b = 0; b < td.n_ap; ++b)
                    if (ap_ids[td.ap_off + b] == ap) letter |= 1u << b;
            }
            letters[pd.letter_off + s] = (uint8_t)letter;
        }
    }
}

// First pass: merged transition count of every row (and per product).
__global__ void k_row_count(const ProdDesc *prods, int P, const AgentDesc *agents, const TaskDesc *tasks,
                            const int32_t *a_sa_ptr, const int32_t *a_succ, const uint8_t *letters,
                            const int16_t *nd_delta, uint32_t *row_cnt, uint32_t *prod_tr) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int p = blockIdx.y; p < P; p += gridDim.y) {
        const ProdDesc pd = prods[p];
        const AgentDesc ad = agents[pd.agent];
        const TaskDesc td = tasks[pd.task];
        const uint32_t SA = ad.SA, n_sa = (uint32_t)td.Qn * SA;
        unsigned int total = 0;
        for (uint32_t v = tid; v < n_sa; v += stride) {
            const uint32_t pl = v / SA, a = v - pl * SA;
            const int32_t e0 = a_sa_ptr[ad.sap_off + a], e1 = a_sa_ptr[ad.sap_off + a + 1];
            uint32_t n = 0;
            bool done_seen = false;
            for (int32_t e = e0; e < e1; ++e) {
                const int32_t s2 = a_succ[ad.tr_off + e];
                const uint32_t letter = letters[pd.letter_off + (uint32_t)s2];
                const bool done = nd_delta[td.delta_off + pl * (uint32_t)td.n_letters + letter] < 0;
                n += done && done_seen ? 0u : 1u;
                done_seen = done_seen || done;
            }
            row_cnt[pd.sa_off + v] = n;
            total += n;
        }
        if (prod_tr) {
            total = __reduce_add_sync(0xffffffffu, total);
            if ((threadIdx.x & 31) == 0 && total) atomicAdd(prod_tr + p, total);
        }
    }
}

// Second pass: per product, sa_tr = tr_off + exclusive prefix sum of the
// row counts, in tiles of the block's size with a running carry.
__global__ void __launch_bounds__(1024) k_row_offsets(const ProdDesc *prods, int P, const uint32_t *row_cnt,
                                                      uint32_t *sa_tr) {
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int p = blockIdx.x; p < P; p += gridDim.x) {
        const ProdDesc pd = prods[p];
        const uint32_t n_sa = (uint32_t)pd.Qn * pd.SA;
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (uint32_t base = 0; base < n_sa; base += blockDim.x) {
            const uint32_t v = base + threadIdx.x;
            const uint32_t x = v < n_sa ? row_cnt[pd.sa_off + v] : 0u;
            uint32_t incl = x;  // inclusive scan within the warp
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) warp_sum[w] = incl;
            __syncthreads();
            if (w == 0) {
                const uint32_t ws = lane < (int)(blockDim.x >> 5) ? warp_sum[lane] : 0u;
                uint32_t wi = ws;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
                    if (lane >= o) wi += y;
                }
                warp_sum[lane] = wi - ws;  // exclusive prefix of the warp sums
            }
            __syncthreads();
            const uint32_t c0 = carry;
            if (v < n_sa) sa_tr[pd.sa_off + v] = pd.tr_off + c0 + warp_sum[w] + incl - x;
            __syncthreads();
            if (threadIdx.x == blockDim.x - 1) carry = c0 + warp_sum[w] + incl;
            __syncthreads();
        }
    }
}

__global__ void k_build(const ProdDesc *prods, int P, const AgentDesc *agents, const TaskDesc *tasks,
                        const int32_t *a_state_ptr, const int32_t *a_sa_ptr, const int32_t *a_succ,
                        const double *a_prob, const double *a_cost, const uint8_t *letters, const int16_t *nd_delta,
                        uint32_t *state_sa, uint32_t *state_tr, uint32_t *sa_tr, int32_t *col, int2 *cp32,
                        double *p64, float2 *pdf, float *cost32, double *cost64, float2 *costdf,
                        uint32_t total_states, uint32_t total_sa, uint32_t total_tr) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    if (blockIdx.y == 0 && tid == 0) {
        state_sa[total_states] = total_sa;
        state_tr[total_states] = total_tr;
        sa_tr[total_sa] = total_tr;
    }
    for (int p = blockIdx.y; p < P; p += gridDim.y) {
        const ProdDesc pd = prods[p];
        const AgentDesc ad = agents[pd.agent];
        const TaskDesc td = tasks[pd.task];
        const uint32_t S = ad.S, SA = ad.SA, T = ad.T;
        // states (the done slot u == n_nd has an empty action range)
        for (uint32_t u = tid; u <= pd.n_nd; u += stride) {
            uint32_t v;
            if (u < pd.n_nd) {
                const uint32_t pl = u / S, s = u - pl * S;
                v = pl * SA + (uint32_t)a_state_ptr[ad.sp_off + s];
            } else {
                v = (uint32_t)td.Qn * SA;
            }
            state_sa[pd.state_off + u] = pd.sa_off + v;
            // the first transition of the state's first row (k_row_offsets
            // ran before); the done slot: the end of the product's transitions
            state_tr[pd.state_off + u] = u < pd.n_nd ? sa_tr[pd.sa_off + v] : pd.tr_off + pd.n_tr;
        }
        // state-action rows (their costs) and their transitions
        const uint32_t n_sa = (uint32_t)td.Qn * SA;
        const uint32_t done = pd.state_off + pd.n_nd;
        for (uint32_t v = tid; v < n_sa; v += stride) {
            const uint32_t pl = v / SA, a = v - pl * SA;
            const double c = a_cost[ad.cost_off + a];
            if (cost64) cost64[pd.sa_off + v] = c;  // the FP64 copies only once a caller needs them
            cost32[pd.sa_off + v] = __double2float_ru(c);
            costdf[pd.sa_off + v] = to_df(c);
            const int32_t e0 = a_sa_ptr[ad.sap_off + a], e1 = a_sa_ptr[ad.sap_off + a + 1];
            uint32_t t = sa_tr[pd.sa_off + v];
            uint32_t t_done = 0xffffffffu;  // position of the merged done transition
            double p_done = 0.0;
            for (int32_t e = e0; e < e1; ++e) {
                const int32_t s2 = a_succ[ad.tr_off + e];
                const uint32_t letter = letters[pd.letter_off + (uint32_t)s2];
                const int32_t pl2 = nd_delta[td.delta_off + pl * (uint32_t)td.n_letters + letter];
                const double pr = a_prob[ad.tr_off + e];
                if (pl2 < 0) {
                    if (t_done == 0xffffffffu) t_done = t++;
                    p_done += pr;
                    continue;
                }
                const int32_t cg = (int32_t)(pd.state_off + (uint32_t)pl2 * S + (uint32_t)s2);
                col[t] = cg;
                if (p64) p64[t] = pr;
                pdf[t] = to_df(pr);
                cp32[t] = make_int2(cg, __float_as_int(__double2float_rd(pr)));
                ++t;
            }
            if (t_done != 0xffffffffu) {
                col[t_done] = (int32_t)done;
                if (p64) p64[t_done] = p_done;
                pdf[t_done] = to_df(p_done);
                cp32[t_done] = make_int2((int32_t)done, __float_as_int(__double2float_rd(p_done)));
            }
        }
    }
}

}  // namespace

int launch_letters(const ProdDesc *prods, int P, const AgentDesc *agents, const TaskDesc *tasks,
                   const int32_t *label_ptr, const int32_t *label_ap, const int32_t *ap_ids, uint8_t *letters,
                   uint32_t max_S, void *s) {
    dim3 grid((max_S + 255) / 256 < 64 ? (max_S + 255) / 256 : 64, P < 65535 ? P : 65535);
    if (grid.x == 0) grid.x = 1;
    k_letters<<<grid, 256, 0, (cudaStream_t)s>>>(prods, P, agents, tasks, label_ptr, label_ap, ap_ids, letters);
    return (int)cudaGetLastError();
}

int launch_row_count(const ProdDesc *prods, int P, const AgentDesc *agents, const TaskDesc *tasks,
                     const int32_t *a_sa_ptr, const int32_t *a_succ, const uint8_t *letters,
                     const int16_t *nd_delta, uint32_t *row_cnt, uint32_t *prod_tr, uint32_t max_rows, void *s) {
    dim3 grid((max_rows + 255) / 256 < 64 ? (max_rows + 255) / 256 : 64, P < 65535 ? P : 65535);
    if (grid.x == 0) grid.x = 1;
    k_row_count<<<grid, 256, 0, (cudaStream_t)s>>>(prods, P, agents, tasks, a_sa_ptr, a_succ, letters, nd_delta,
                                                    row_cnt, prod_tr);
    return (int)cudaGetLastError();
}

int launch_row_offsets(const ProdDesc *prods, int P, const uint32_t *row_cnt, uint32_t *sa_tr, void *s) {
    if (P <= 0) return 0;
    k_row_offsets<<<P < 4096 ? P : 4096, 1024, 0, (cudaStream_t)s>>>(prods, P, row_cnt, sa_tr);
    return (int)cudaGetLastError();
}

int launch_build(const ProdDesc *prods, int P, const AgentDesc *agents, const TaskDesc *tasks,
                 const int32_t *a_state_ptr, const int32_t *a_sa_ptr, const int32_t *a_succ, const double *a_prob,
                 const double *a_cost, const uint8_t *letters, const int16_t *nd_delta, uint32_t *state_sa,
                 uint32_t *state_tr, uint32_t *sa_tr, int32_t *col, int2 *cp32, double *p64, float2 *pdf,
                 float *cost32, double *cost64, float2 *costdf, uint32_t total_states, uint32_t total_sa,
                 uint32_t total_tr, uint32_t max_work, void *s) {
    dim3 grid((max_work + 255) / 256 < 64 ? (max_work + 255) / 256 : 64, P < 65535 ? P : 65535);
    if (grid.x == 0) grid.x = 1;
    k_build<<<grid, 256, 0, (cudaStream_t)s>>>(prods, P, agents, tasks, a_state_ptr, a_sa_ptr, a_succ, a_prob, a_cost,
                                                letters, nd_delta, state_sa, state_tr, sa_tr, col, cp32, p64, pdf,
                                                cost32, cost64, costdf, total_states, total_sa, total_tr);
    return (int)cudaGetLastError();
}

}  // namespace morap

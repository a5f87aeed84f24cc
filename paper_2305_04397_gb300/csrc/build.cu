// Product construction on the device (Sec. 2 "Product MDP", Sec. 3.1).
//
// The product of agent i and task j keeps the agent's CSR shape once per
// non-done DFA location: product state (pl, s) has the actions of agent
// state s, and each agent transition (s, a, s', p) becomes ((pl, s), a,
// (pl', s'), p) with pl' = delta(pl, L(s')) -- the label is read on the
// successor.  A successor whose location is done (accepting or trap) goes to
// the product's single absorbing done slot (value 0).  Because the shape is a
// replication, every offset is known in closed form and the build is one
// pass with no scan: local state u = pl*S + s, local row v = pl*SA + a, local
// transition t = pl*T + e.
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
            uint32_t t0;
            if (u < pd.n_nd) {
                const uint32_t pl = u / S, s = u - pl * S;
                t0 = pl * T + (uint32_t)a_sa_ptr[ad.sap_off + a_state_ptr[ad.sp_off + s]];
            } else {
                t0 = (uint32_t)td.Qn * T;
            }
            state_tr[pd.state_off + u] = pd.tr_off + t0;
        }
        // state-action rows
        const uint32_t n_sa = (uint32_t)td.Qn * SA;
        for (uint32_t v = tid; v < n_sa; v += stride) {
            const uint32_t pl = v / SA, a = v - pl * SA;
            sa_tr[pd.sa_off + v] = pd.tr_off + pl * T + (uint32_t)a_sa_ptr[ad.sap_off + a];
            const double c = a_cost[ad.cost_off + a];
            cost64[pd.sa_off + v] = c;
            cost32[pd.sa_off + v] = __double2float_ru(c);
            costdf[pd.sa_off + v] = to_df(c);
        }
        // transitions
        const uint32_t n_tr = (uint32_t)td.Qn * T;
        const uint32_t done = pd.state_off + pd.n_nd;
        for (uint32_t t = tid; t < n_tr; t += stride) {
            const uint32_t pl = t / T, e = t - pl * T;
            const int32_t s2 = a_succ[ad.tr_off + e];
            const uint32_t letter = letters[pd.letter_off + (uint32_t)s2];
            const int32_t pl2 = nd_delta[td.delta_off + pl * (uint32_t)td.n_letters + letter];
            const int32_t cg = pl2 < 0 ? (int32_t)done : (int32_t)(pd.state_off + (uint32_t)pl2 * S + (uint32_t)s2);
            const double pr = a_prob[ad.tr_off + e];
            col[pd.tr_off + t] = cg;
            p64[pd.tr_off + t] = pr;
            pdf[pd.tr_off + t] = to_df(pr);
            cp32[pd.tr_off + t] = make_int2(cg, __float_as_int(__double2float_rd(pr)));
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

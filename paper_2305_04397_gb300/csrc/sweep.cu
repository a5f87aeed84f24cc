// Batched Bellman sweeps of Algorithm 3 and Algorithm 4 over all products
// and all weights of a batch, with the per-(product, weight) residual
// reduction, the device work lists and the loop control that a CUDA-graph
// while node evaluates between bodies.
//
// Data layout (HBM):
//   values  V[state][Kp]   (Kp = weights padded to a power of two), double
//                          buffered; a sweep reads V[n % 2] and writes
//                          V[(n + 1) % 2] (synchronous sweeps, as the oracle)
//   a_rec   [state][Kp]    uint8 local action recorded by Algorithm 3
//   CSR     state_sa[state+1] -> sa_tr[sa+1] -> col[t], p[t]
//
// Thread mapping: LPS = Kp / VEC lanes share one state, lane l owns weights
// [l*VEC, l*VEC+VEC) and loads them as one vector, so the value row of a
// successor is one coalesced Kp-wide read and the CSR stream is read once for
// all Kp weights.  A 256-thread block takes 512-state work items of one
// product from the sweep's work list (dynamic scheduling); the item's
// residuals are reduced with warp shuffles, then across warps in shared
// memory, then with one 64-bit atomicMax per weight.
//
// Work lists: L[n % 3] holds the items of sweep n.  An item is re-queued for
// sweep n+1 when its product still had an active weight in sweep n.  Weight k
// of product p is active in sweep n iff its residual of sweep n-1 exceeded the
// phase threshold; an inactive weight copies its value (y = x), so both value
// buffers agree once it freezes, and a product whose residuals were all
// exactly 0 is dropped.  Each pair therefore runs exactly the sweeps it would
// run alone (results do not depend on the batch).
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cstdint>

#include "internal.h"

namespace morap {

namespace {

template <typename T>
struct Arith;

// FP32 with every rounding toward -inf: with V >= 0, p rounded down and the
// reward rounded down, each computed Q is <= the exact Q of the same iterate,
// so every FP32 iterate is a lower bound of the exact one (and of the fixed
// point reached from 0).
template <>
struct Arith<float> {
    using W = float2;
    static __device__ __forceinline__ float reward(float2 w, float cost, bool pre) {
        return __fsub_rd(pre ? w.y : 0.0f, __fmul_ru(w.x, cost));
    }
    static __device__ __forceinline__ float mac(float p, float v, float acc) { return __fmaf_rd(p, v, acc); }
    // Algorithm 3 records the maximiser when the value moves by more than
    // eps1.  In FP32 a move of a few ulps is rounding, not propagation, so the
    // FP32 phase records only moves above 64 ulps of the new value (the FP64
    // phase that follows records with eps1 itself).
    static __device__ __forceinline__ double record_threshold(float y, double eps1) {
        const double rel = (double)y * 7.62939453125e-06; /* 2^-17 */
        return rel > eps1 ? rel : eps1;
    }
    static __device__ __forceinline__ float cost(const SweepArgs &a, uint32_t sa) { return __ldg(a.cost32 + sa); }
    static __device__ __forceinline__ void edge(const SweepArgs &a, uint32_t t, int32_t &c, float &p) {
        const int2 e = __ldg(a.cp32 + t);
        c = e.x;
        p = __int_as_float(e.y);
    }
    static __device__ __forceinline__ float2 weight(const SweepArgs &a, size_t pair) { return a.w32[pair]; }
};

template <>
struct Arith<double> {
    using W = double2;
    static __device__ __forceinline__ double reward(double2 w, double cost, bool pre) {
        return (pre ? w.y : 0.0) - w.x * cost;
    }
    static __device__ __forceinline__ double mac(double p, double v, double acc) { return fma(p, v, acc); }
    static __device__ __forceinline__ double record_threshold(double, double eps1) { return eps1; }
    static __device__ __forceinline__ double cost(const SweepArgs &a, uint32_t sa) { return __ldg(a.cost64 + sa); }
    static __device__ __forceinline__ void edge(const SweepArgs &a, uint32_t t, int32_t &c, double &p) {
        c = __ldg(a.col + t);
        p = __ldg(a.p64 + t);
    }
    static __device__ __forceinline__ double2 weight(const SweepArgs &a, size_t pair) { return a.w64[pair]; }
};

template <typename T, int VEC>
struct Vec {
    T v[VEC];
};

template <typename T, int VEC>
__device__ __forceinline__ Vec<T, VEC> vload(const T *p) {
    Vec<T, VEC> r;
    if constexpr (sizeof(T) * VEC == 16) {
        if constexpr (sizeof(T) == 4) {
            const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
            r.v[0] = q.x, r.v[1] = q.y, r.v[2] = q.z, r.v[3] = q.w;
        } else {
            const double2 q = __ldg(reinterpret_cast<const double2 *>(p));
            r.v[0] = q.x, r.v[1] = q.y;
        }
    } else if constexpr (sizeof(T) * VEC == 8) {
        if constexpr (sizeof(T) == 4) {
            const float2 q = __ldg(reinterpret_cast<const float2 *>(p));
            r.v[0] = q.x, r.v[1] = q.y;
        } else {
            r.v[0] = __ldg(p);
        }
    } else {
        r.v[0] = __ldg(p);
    }
    return r;
}

template <typename T, int VEC>
__device__ __forceinline__ void vstore(T *p, const Vec<T, VEC> &x) {
    if constexpr (sizeof(T) * VEC == 16) {
        if constexpr (sizeof(T) == 4)
            *reinterpret_cast<float4 *>(p) = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
        else
            *reinterpret_cast<double2 *>(p) = make_double2(x.v[0], x.v[1]);
    } else if constexpr (sizeof(T) * VEC == 8) {
        if constexpr (sizeof(T) == 4)
            *reinterpret_cast<float2 *>(p) = make_float2(x.v[0], x.v[1]);
        else
            p[0] = x.v[0];
    } else {
        p[0] = x.v[0];
    }
}

template <typename T, int KP>
struct Layout {
    static constexpr int VEC = (16 / sizeof(T)) < KP ? (16 / (int)sizeof(T)) : KP;
    static constexpr int LPS = KP / VEC;               // lanes per state
    static constexpr int SPR = kThreads / LPS;         // states per block round
    static constexpr int WARPS = kThreads / 32;
};

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double as_double(unsigned long long b) { return __longlong_as_double((long long)b); }

// ------------------------------------------------------------- the sweep
template <typename T, int KP>
__global__ void __launch_bounds__(kThreads, 3) k_sweep(SweepArgs a, int pos) {
    using L = Layout<T, KP>;
    using Ar = Arith<T>;
    constexpr int VEC = L::VEC, LPS = L::LPS, SPR = L::SPR;
    constexpr int D = kGatherBatch;
    const int cur = pos % 3, nxt = (pos + 1) % 3, far = (pos + 2) % 3;
    const T *__restrict__ Vold = static_cast<const T *>(a.V[pos & 1]);
    T *__restrict__ Vnew = static_cast<T *>(a.V[(pos + 1) & 1]);
    const unsigned long long *res_prev = a.res[far];
    unsigned long long *res_cur = a.res[cur];
    unsigned long long *res_next = a.res[nxt];
    LoopCtl *ctl = a.ctl;

    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->cnt[far] = 0;
        ctl->next[far] = 0;
    }
    const unsigned int n_items = ctl->cnt[cur];
    const unsigned int sweep = ctl->sweep_base + pos;

    __shared__ unsigned int s_item;
    __shared__ int s_active[KP];
    __shared__ int s_any_active, s_any_nonzero;
    __shared__ double s_red[L::WARPS][KP];

    const int lane_in_state = threadIdx.x % LPS;
    const int slot = threadIdx.x / LPS;
    const int k0 = lane_in_state * VEC;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    for (;;) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(&ctl->next[cur], 1u);
            s_any_active = 0;
            s_any_nonzero = 0;
        }
        __syncthreads();
        const unsigned int it = s_item;
        if (it >= n_items) break;
        const unsigned int item = a.list[cur][it];
        const int4 ch = a.chunks[item];
        const int p = ch.x;
        const size_t pair0 = (size_t)p * KP;
        if (threadIdx.x < KP) {
            const double prev = as_double(res_prev[pair0 + threadIdx.x]);
            const int act = prev > a.thr[pair0 + threadIdx.x];
            s_active[threadIdx.x] = act;
            if (act) atomicOr(&s_any_active, 1);
            if (prev > 0.0) atomicOr(&s_any_nonzero, 1);
        }
        __syncthreads();
        const bool any_active = s_any_active != 0;
        if (s_any_nonzero == 0) {  // converged earlier and already copied: drop
            if (ch.w && threadIdx.x < KP) a.frozen[pair0 + threadIdx.x] = 1;
            __syncthreads();
            continue;
        }
        const ProdDesc pd = a.prods[p];
        if (threadIdx.x == 0 && any_active) {
            const unsigned int at = atomicAdd(&ctl->cnt[nxt], 1u);
            a.list[nxt][at] = item;
        }
        if (ch.w && threadIdx.x < KP) {
            res_next[pair0 + threadIdx.x] = 0ull;
            if (s_active[threadIdx.x])
                a.sweeps_pair[pair0 + threadIdx.x] = (int32_t)(sweep + 1);
            else
                a.frozen[pair0 + threadIdx.x] = 1;
        }
        bool act[VEC];
        typename Ar::W w[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            act[v] = s_active[k0 + v] != 0;
            w[v] = Ar::weight(a, pair0 + k0 + v);
        }
        T rmax[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) rmax[v] = T(0);

        for (int s = ch.y + slot; s < ch.z; s += SPR) {
            const uint32_t u = pd.state_off + (uint32_t)s;
            const size_t row = (size_t)u * KP + k0;
            const Vec<T, VEC> x = vload<T, VEC>(Vold + row);
            Vec<T, VEC> y = x;
            if (any_active) {
                const bool pre = (uint32_t)s >= pd.pre_begin;
                const uint32_t a0 = __ldg(a.state_sa + u), a1 = __ldg(a.state_sa + u + 1);
                const uint32_t te = __ldg(a.sa_tr + a1);
                T best[VEC], acc[VEC];
                uint32_t best_a[VEC];
                uint32_t sa = a0, bound = __ldg(a.sa_tr + a0 + 1);
                {
                    const T c0 = Ar::cost(a, a0);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        best[v] = -CUDART_INF;
                        best_a[v] = 0;
                        acc[v] = Ar::reward(w[v], c0, pre);
                    }
                }
                // The state's transitions form one stream over its actions;
                // D gathers are issued back to back before they are consumed.
                for (uint32_t base = __ldg(a.sa_tr + a0); base < te; base += D) {
                    int32_t cl[D];
                    T pr[D];
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        const uint32_t t = base + i;
                        if (t < te) {
                            Ar::edge(a, t, cl[i], pr[i]);
                        } else {
                            cl[i] = -1;
                            pr[i] = T(0);
                        }
                    }
                    Vec<T, VEC> xv[D];
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        if (cl[i] >= 0) {
                            xv[i] = vload<T, VEC>(Vold + (size_t)cl[i] * KP + k0);
                        } else {
#pragma unroll
                            for (int v = 0; v < VEC; ++v) xv[i].v[v] = T(0);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < D; ++i) {
                        if (cl[i] < 0) continue;
                        while (base + i >= bound) {  // close action sa, open the next one
#pragma unroll
                            for (int v = 0; v < VEC; ++v)
                                if (acc[v] > best[v]) {
                                    best[v] = acc[v];
                                    best_a[v] = sa - a0;
                                }
                            ++sa;
                            bound = __ldg(a.sa_tr + sa + 1);
                            const T cs = Ar::cost(a, sa);
#pragma unroll
                            for (int v = 0; v < VEC; ++v) acc[v] = Ar::reward(w[v], cs, pre);
                        }
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[v] = Ar::mac(pr[i], xv[i].v[v], acc[v]);
                    }
                }
#pragma unroll
                for (int v = 0; v < VEC; ++v)
                    if (acc[v] > best[v]) {
                        best[v] = acc[v];
                        best_a[v] = sa - a0;
                    }
                uint32_t rec_mask = 0;
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    if (!act[v]) continue;
                    y.v[v] = best[v];
                    const T d = fabs(best[v] - x.v[v]);
                    rmax[v] = d > rmax[v] ? d : rmax[v];
                    if ((double)d > Ar::record_threshold(best[v], a.eps1)) rec_mask |= 1u << v;
                }
                if (rec_mask) {
                    if constexpr (VEC == 4) {
                        if (rec_mask == 0xFu) {
                            *reinterpret_cast<uint32_t *>(a.a_rec + row) =
                                best_a[0] | (best_a[1] << 8) | (best_a[2] << 16) | (best_a[3] << 24);
                        } else {
#pragma unroll
                            for (int v = 0; v < VEC; ++v)
                                if (rec_mask & (1u << v)) a.a_rec[row + v] = (uint8_t)best_a[v];
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            if (rec_mask & (1u << v)) a.a_rec[row + v] = (uint8_t)best_a[v];
                    }
                }
            }
            vstore<T, VEC>(Vnew + row, y);
        }
        // residual reduction: lanes with the same lane_in_state share weights
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            T r = rmax[v];
#pragma unroll
            for (int off = LPS; off < 32; off <<= 1) {
                const T o = __shfl_xor_sync(0xffffffffu, r, off);
                r = o > r ? o : r;
            }
            if (lane < LPS) s_red[warp][lane * VEC + v] = (double)r;
        }
        __syncthreads();
        if (any_active && threadIdx.x < KP) {
            double r = 0.0;
#pragma unroll
            for (int wi = 0; wi < L::WARPS; ++wi) r = s_red[wi][threadIdx.x] > r ? s_red[wi][threadIdx.x] : r;
            if (r > 0.0) atomic_max_nonneg(res_cur + pair0 + threadIdx.x, r);
        }
        if (threadIdx.x == 0) {
            const uint32_t n_s = (uint32_t)(ch.z - ch.y);
            const uint32_t u0 = pd.state_off + ch.y, u1 = pd.state_off + ch.z;
            unsigned long long bytes = 2ull * n_s * KP * sizeof(T);
            if (any_active) {
                const uint32_t sa0 = a.state_sa[u0], sa1 = a.state_sa[u1];
                const uint32_t tr0 = a.sa_tr[sa0], tr1 = a.sa_tr[sa1];
                int n_act = 0;
                for (int k = 0; k < KP; ++k) n_act += s_active[k];
                atomicAdd(&ctl->updates, (unsigned long long)(tr1 - tr0) * (unsigned long long)n_act);
                bytes += 4ull * (n_s + 1) + 4ull * (sa1 - sa0 + 1) + (unsigned long long)(sa1 - sa0) * sizeof(T) +
                         (unsigned long long)(tr1 - tr0) * (4 + sizeof(T));  // col + p per transition
            }
            atomicAdd(&ctl->bytes, bytes);
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------- finalise
// The returned scheduler: keep the recorded action when its Q-value on the
// final FP64 values is within tau of the maximum; otherwise the lowest-index
// action within tau of the maximum that is not a self-loop (a zero-reward
// self-loop ties with the maximum at any fixed point), and only if every
// such action is a self-loop the lowest-index one.
template <int KP>
__global__ void __launch_bounds__(kThreads) k_finalize(SweepArgs a, int n_chunks, double tau, uint8_t *policy) {
    using L = Layout<double, KP>;
    constexpr int VEC = L::VEC, LPS = L::LPS, SPR = L::SPR;
    constexpr int MAXA = 32;  // actions scanned twice per state: first for the max, then for the choice
    const double *__restrict__ V = static_cast<const double *>(a.V[0]);
    const int k0 = (threadIdx.x % LPS) * VEC, slot = threadIdx.x / LPS;
    for (int item = blockIdx.x; item < n_chunks; item += gridDim.x) {
        const int4 ch = a.chunks[item];
        const int p = ch.x;
        const ProdDesc pd = a.prods[p];
        double2 w[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) w[v] = a.w64[(size_t)p * KP + k0 + v];
        for (int s = ch.y + slot; s < ch.z; s += SPR) {
            const uint32_t u = pd.state_off + (uint32_t)s;
            const size_t row = (size_t)u * KP + k0;
            const bool pre = (uint32_t)s >= pd.pre_begin;
            const uint32_t a0 = a.state_sa[u], a1 = a.state_sa[u + 1];
            double best[VEC], qrec[VEC];
            uint8_t rec[VEC], pick[VEC], pick_loop[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                best[v] = -CUDART_INF;
                rec[v] = a.a_rec[row + v];
                qrec[v] = -CUDART_INF;
                pick[v] = 0xFF;
                pick_loop[v] = 0xFF;
            }
            for (int pass = 0; pass < 2; ++pass) {
                for (uint32_t sa = a0; sa < a1; ++sa) {
                    const double c = a.cost64[sa];
                    double acc[VEC];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[v] = (pre ? w[v].y : 0.0) - w[v].x * c;
                    const uint32_t t0 = a.sa_tr[sa], t1 = a.sa_tr[sa + 1];
                    bool self_loop = (t1 - t0 == 1) && ((uint32_t)a.col[t0] == u);
                    for (uint32_t t = t0; t < t1; ++t) {
                        const int32_t cl = a.col[t];
                        const double pr = a.p64[t];
                        const Vec<double, VEC> xv = vload<double, VEC>(V + (size_t)cl * KP + k0);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[v] = fma(pr, xv.v[v], acc[v]);
                    }
                    const uint8_t la = (uint8_t)(sa - a0);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        if (pass == 0) {
                            best[v] = acc[v] > best[v] ? acc[v] : best[v];
                            if (la == rec[v]) qrec[v] = acc[v];
                        } else if (acc[v] >= best[v] - tau) {
                            if (self_loop) {
                                if (pick_loop[v] == 0xFF) pick_loop[v] = la;
                            } else if (pick[v] == 0xFF) {
                                pick[v] = la;
                            }
                        }
                    }
                }
                bool all_kept = true;
#pragma unroll
                for (int v = 0; v < VEC; ++v) all_kept = all_kept && (qrec[v] >= best[v] - tau);
                if (all_kept) break;  // the second pass is only needed for a fallback
            }
#pragma unroll
            for (int v = 0; v < VEC; ++v)
                policy[row + v] = (qrec[v] >= best[v] - tau) ? rec[v] : (pick[v] != 0xFF ? pick[v] : pick_loop[v]);
        }
    }
    (void)MAXA;
}

// ------------------------------------------------------------- evaluation
// Algorithm 4 for both objectives of a pair at once: E[u] = (cost, prob)
// with y = (-cost(u, mu(u)), pre(u)) + sum p E[u'].
__global__ void __launch_bounds__(kThreads) k_eval_sweep(EvalArgs a, int pos) {
    const int cur = pos % 3, nxt = (pos + 1) % 3, far = (pos + 2) % 3;
    const double2 *__restrict__ Eold = a.E[pos & 1];
    double2 *__restrict__ Enew = a.E[(pos + 1) & 1];
    LoopCtl *ctl = a.ctl;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->cnt[far] = 0;
        ctl->next[far] = 0;
    }
    const unsigned int n_items = ctl->cnt[cur];
    const unsigned int sweep = ctl->sweep_base + pos;
    __shared__ unsigned int s_item;
    __shared__ double s_red[kThreads / 32];
    __shared__ unsigned int s_nt[kThreads / 32];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctl->next[cur], 1u);
        __syncthreads();
        const unsigned int it = s_item;
        if (it >= n_items) break;
        const unsigned int item = a.list[cur][it];
        const int4 ch = a.chunks[item];
        const int e = ch.x;
        const double prev = as_double(a.res[far][e]);
        const bool active = prev > a.thr;
        if (prev == 0.0) {
            if (ch.w && threadIdx.x == 0) a.frozen[e] = 1;
            __syncthreads();
            continue;
        }
        const int4 pr = a.pairs[e];
        const ProdDesc pd = a.prods[pr.x];
        if (threadIdx.x == 0 && active) {
            const unsigned int at = atomicAdd(&ctl->cnt[nxt], 1u);
            a.list[nxt][at] = item;
        }
        if (ch.w && threadIdx.x == 0) {
            a.res[nxt][e] = 0ull;
            if (active)
                a.sweeps_pair[e] = (int32_t)(sweep + 1);
            else
                a.frozen[e] = 1;
        }
        double r = 0.0;
        unsigned int n_t = 0;
        const int s = ch.y + threadIdx.x;
        if (s < ch.z) {
            const size_t off = (size_t)pr.z;
            const double2 x = Eold[off + s];
            double2 y = x;
            if (active) {
                const uint32_t u = pd.state_off + (uint32_t)s;
                const uint32_t sa = a.state_sa[u] + a.policy[(size_t)u * a.Kp + pr.y];
                double yc = -a.cost64[sa];
                double yp = ((uint32_t)s >= pd.pre_begin) ? 1.0 : 0.0;
                const uint32_t t0 = a.sa_tr[sa], t1 = a.sa_tr[sa + 1];
                n_t = t1 - t0;
                for (uint32_t t = t0; t < t1; ++t) {
                    const uint32_t loc = (uint32_t)a.col[t] - pd.state_off;
                    const double p = a.p64[t];
                    const double2 xv = Eold[off + loc];
                    yc = fma(p, xv.x, yc);
                    yp = fma(p, xv.y, yp);
                }
                y = make_double2(yc, yp);
                r = fmax(fabs(yc - x.x), fabs(yp - x.y));
            }
            Enew[off + s] = y;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            r = fmax(r, __shfl_xor_sync(0xffffffffu, r, off));
            n_t += __shfl_xor_sync(0xffffffffu, n_t, off);
        }
        if ((threadIdx.x & 31) == 0) {
            s_red[threadIdx.x / 32] = r;
            s_nt[threadIdx.x / 32] = n_t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0.0;
            unsigned long long nt = 0;
            for (int wi = 0; wi < kThreads / 32; ++wi) {
                m = fmax(m, s_red[wi]);
                nt += s_nt[wi];
            }
            if (active && m > 0.0) atomic_max_nonneg(a.res[cur] + e, m);
            const unsigned long long n_s = (unsigned long long)(ch.z - ch.y);
            // values: read + write 16 B per state; when computing also the
            // policy byte, state_sa and sa_tr (4 + 8), the cost (8) and the
            // policy row's transitions (col 4 + p 8 each)
            unsigned long long bytes = n_s * 32ull;
            if (active) {
                bytes += n_s * (1 + 4 + 8 + 8) + nt * 12ull;
                atomicAdd(&ctl->updates, nt * 2ull);
            }
            atomicAdd(&ctl->bytes, bytes);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- small kernels

__global__ void k_setup_weights(const ProdDesc *prods, int P, int nI, int nJ, int K, int Kp, const double *W,
                                float2 *w32, double2 *w64, double *thr32, double *thr64, double eps1) {
    const size_t n = (size_t)P * Kp;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(idx / Kp), k = (int)(idx % Kp);
        const ProdDesc pd = prods[p];
        double wi = 0.0, wp = 0.0;
        if (k < K) {
            wi = W[(size_t)k * (nI + nJ) + pd.agent];
            wp = W[(size_t)k * (nI + nJ) + nI + pd.task];
        }
        w64[idx] = make_double2(wi, wp);
        w32[idx] = make_float2(__double2float_ru(wi), __double2float_rd(wp));
        // FP32 phase: stop once the residual is within a few ulps of the
        // largest possible value (values lie in [0, w_p]); FP64 phase: eps1.
        thr32[idx] = fmax(eps1, wp * 9.5367431640625e-07 /* 2^-20 */);
        thr64[idx] = eps1;
    }
}

__global__ void k_loop_init(LoopCtl *ctl, unsigned int *list0, unsigned int n_items, unsigned long long *r0,
                            unsigned long long *r1, unsigned long long *r2, size_t n_pairs, int32_t *sweeps_pair,
                            uint8_t *frozen, unsigned int cap) {
    const size_t gid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = gid; i < n_items; i += stride) list0[i] = (unsigned int)i;
    const unsigned long long inf_bits = (unsigned long long)__double_as_longlong(CUDART_INF);
    for (size_t i = gid; i < n_pairs; i += stride) {
        r0[i] = 0ull;
        r1[i] = 0ull;
        r2[i] = inf_bits;  // "previous" residual of sweep 0: everything active
        sweeps_pair[i] = 0;
        frozen[i] = 0;
    }
    if (gid == 0) {
        ctl->cnt[0] = n_items;
        ctl->cnt[1] = ctl->cnt[2] = 0;
        ctl->next[0] = ctl->next[1] = ctl->next[2] = 0;
        ctl->sweep_base = 0;
        ctl->hit_cap = 0;
        ctl->cap = cap;
        ctl->updates = 0;
        ctl->bytes = 0;
    }
}

// Evaluated after each body of 6 sweeps: continue while the work list of
// the next sweep is non-empty and the sweep cap is not reached.
__global__ void k_loop_control(LoopCtl *ctl, cudaGraphConditionalHandle handle, int next_idx) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    ctl->sweep_base += 6;
    const bool more = ctl->cnt[next_idx] > 0;
    const bool go = more && ctl->sweep_base < ctl->cap;
    if (more && !go) ctl->hit_cap = 1;
    cudaGraphSetConditional(handle, go ? 1u : 0u);
}

// Host-driven variant of the control step (launch_mode 1).
__global__ void k_loop_control_host(LoopCtl *ctl, int next_idx) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    ctl->sweep_base += 6;
    if (ctl->cnt[next_idx] > 0 && ctl->sweep_base >= ctl->cap) ctl->hit_cap = 1;
}

__global__ void k_convert(const float *v32, double *a, double *b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double v = (double)v32[i];
        a[i] = v;
        b[i] = v;
    }
}

// c_ij = V(s0, q0) for every (product, weight); a pair that never froze
// stopped at the sweep cap.
__global__ void k_gather_c(int Kp, const ProdDesc *prods, int P, const double *V, const uint8_t *frozen,
                           double *c_out, int32_t *status_out) {
    const size_t n = (size_t)P * Kp;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(idx / Kp), k = (int)(idx % Kp);
        const ProdDesc pd = prods[p];
        const double v = (uint32_t)pd.init_local >= pd.n_nd ? 0.0 : V[(size_t)(pd.state_off + pd.init_local) * Kp + k];
        c_out[idx] = v;
        status_out[idx] = frozen[idx] ? MORAP_OK : MORAP_ENOTCONV;
    }
}

__global__ void k_gather_eval(const int4 *pairs, int n_pairs, const ProdDesc *prods, const double2 *E, double *rc,
                              double *rp) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_pairs; e += gridDim.x * blockDim.x) {
        const int4 pr = pairs[e];
        const ProdDesc pd = prods[pr.x];
        if ((uint32_t)pd.init_local >= pd.n_nd) {
            rc[e] = 0.0;
            rp[e] = 0.0;
        } else {
            const double2 v = E[(size_t)pr.z + pd.init_local];
            rc[e] = v.x;
            rp[e] = v.y;
        }
    }
}

template <typename T>
int launch_sweep_t(int Kp, const SweepArgs &a, int pos, int grid, cudaStream_t s) {
    switch (Kp) {
    case 1: k_sweep<T, 1><<<grid, kThreads, 0, s>>>(a, pos); break;
    case 2: k_sweep<T, 2><<<grid, kThreads, 0, s>>>(a, pos); break;
    case 4: k_sweep<T, 4><<<grid, kThreads, 0, s>>>(a, pos); break;
    case 8: k_sweep<T, 8><<<grid, kThreads, 0, s>>>(a, pos); break;
    case 16: k_sweep<T, 16><<<grid, kThreads, 0, s>>>(a, pos); break;
    case 32: k_sweep<T, 32><<<grid, kThreads, 0, s>>>(a, pos); break;
    case 64: k_sweep<T, 64><<<grid, kThreads, 0, s>>>(a, pos); break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

}  // namespace

template <typename T>
int blocks_per_sm_t(int Kp) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (Kp) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<T, 1>, kThreads, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<T, 2>, kThreads, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<T, 4>, kThreads, 0); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<T, 8>, kThreads, 0); break;
    case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<T, 16>, kThreads, 0); break;
    case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<T, 32>, kThreads, 0); break;
    case 64: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<T, 64>, kThreads, 0); break;
    default: break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

int sweep_blocks_per_sm(bool fp64, int Kp) { return fp64 ? blocks_per_sm_t<double>(Kp) : blocks_per_sm_t<float>(Kp); }

int eval_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_eval_sweep, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

int launch_sweep(bool fp64, int Kp, const SweepArgs &a, int pos, int grid, void *s) {
    return fp64 ? launch_sweep_t<double>(Kp, a, pos, grid, (cudaStream_t)s)
                : launch_sweep_t<float>(Kp, a, pos, grid, (cudaStream_t)s);
}

int launch_finalize(int Kp, const SweepArgs &a, int n_chunks, double tau, uint8_t *policy, void *sv) {
    cudaStream_t s = (cudaStream_t)sv;
    const int grid = n_chunks < 8192 ? n_chunks : 8192;
    if (grid <= 0) return 0;
    switch (Kp) {
    case 1: k_finalize<1><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy); break;
    case 2: k_finalize<2><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy); break;
    case 4: k_finalize<4><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy); break;
    case 8: k_finalize<8><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy); break;
    case 16: k_finalize<16><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy); break;
    case 32: k_finalize<32><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy); break;
    case 64: k_finalize<64><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy); break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

int launch_eval_sweep(const EvalArgs &a, int pos, int grid, void *s) {
    k_eval_sweep<<<grid, kThreads, 0, (cudaStream_t)s>>>(a, pos);
    return (int)cudaGetLastError();
}

int launch_setup_weights(const ProdDesc *prods, int P, int nI, int nJ, int K, int Kp, const double *W, float2 *w32,
                         double2 *w64, double *thr32, double *thr64, double eps1, void *s) {
    const size_t n = (size_t)P * Kp;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_setup_weights<<<grid > 0 ? grid : 1, 256, 0, (cudaStream_t)s>>>(prods, P, nI, nJ, K, Kp, W, w32, w64, thr32,
                                                                     thr64, eps1);
    return (int)cudaGetLastError();
}

int launch_loop_init(LoopCtl *ctl, unsigned int *list0, unsigned int n_items, unsigned long long *res[3],
                     size_t n_pairs, int32_t *sweeps_pair, uint8_t *frozen, unsigned int cap, void *s) {
    const size_t n = n_items > n_pairs ? n_items : n_pairs;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_loop_init<<<grid > 0 ? grid : 1, 256, 0, (cudaStream_t)s>>>(ctl, list0, n_items, res[0], res[1], res[2],
                                                                 n_pairs, sweeps_pair, frozen, cap);
    return (int)cudaGetLastError();
}

int launch_loop_control(LoopCtl *ctl, unsigned long long handle, int next_idx, void *s) {
    k_loop_control<<<1, 32, 0, (cudaStream_t)s>>>(ctl, (cudaGraphConditionalHandle)handle, next_idx);
    return (int)cudaGetLastError();
}

int launch_loop_control_host(LoopCtl *ctl, int next_idx, void *s) {
    k_loop_control_host<<<1, 32, 0, (cudaStream_t)s>>>(ctl, next_idx);
    return (int)cudaGetLastError();
}

int launch_convert(const float *v32, double *v64a, double *v64b, size_t n, void *s) {
    const int grid = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
    k_convert<<<grid > 0 ? grid : 1, 256, 0, (cudaStream_t)s>>>(v32, v64a, v64b, n);
    return (int)cudaGetLastError();
}

int launch_gather_c(int Kp, const ProdDesc *prods, int P, const double *V64, const uint8_t *frozen, double *c_out,
                    int32_t *status_out, void *s) {
    const size_t n = (size_t)P * Kp;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_gather_c<<<grid > 0 ? grid : 1, 256, 0, (cudaStream_t)s>>>(Kp, prods, P, V64, frozen, c_out, status_out);
    return (int)cudaGetLastError();
}

int launch_gather_eval(const int4 *pairs, int n_pairs, const ProdDesc *prods, const double2 *E, double *rc,
                       double *rp, void *s) {
    const int grid = (n_pairs + 255) / 256;
    if (grid == 0) return 0;
    k_gather_eval<<<grid, 256, 0, (cudaStream_t)s>>>(pairs, n_pairs, prods, E, rc, rp);
    return (int)cudaGetLastError();
}

}  // namespace morap

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

// ------------------------------------------------------------ arithmetic
//
// Two value formats run the same sweep code:
//  * FP32 with every rounding toward -inf (phase 1).  With V >= 0, the
//    probabilities rounded down and the rewards rounded down, each computed
//    Q is <= the exact Q of the same iterate, so every iterate is a lower
//    bound of the exact one and of the fixed point reached from 0.
//  * double-float (phase 2): a value is an unevaluated sum hi + lo of two
//    FP32 numbers (about 48 significant bits).  Sums use Knuth's two-sum,
//    products Dekker's two-product through an FMA; GB300's FP64 units run at
//    a small fraction of the FP32 rate, so this is the fast way to carry the
//    precision the stopping rule eps1 = 1e-8 needs.

struct DF {
    float h, l;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    const float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
    return {s, e};
}

__device__ __forceinline__ DF fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fadd_rn(b, -__fadd_rn(s, -a))};
}

__device__ __forceinline__ DF df_norm(DF x) { return fast_two_sum(x.h, x.l); }

__device__ __forceinline__ DF df_add(DF x, DF y) {
    DF s = two_sum(x.h, y.h);
    s.l = __fadd_rn(s.l, __fadd_rn(x.l, y.l));
    return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ DF df_mul(DF x, DF y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ bool df_gt(DF a, DF b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }

struct ArithF32 {
    using Val = float;
    using W = float2;    // (w_i rounded up, w_p rounded down)
    using Cost = float;  // rounded up
    using Prob = float;  // rounded down
    static constexpr int WORDS = 1;
    static __device__ __forceinline__ W weight(const SweepArgs &a, size_t pair) { return a.w32[pair]; }
    static __device__ __forceinline__ Cost cost(const SweepArgs &a, uint32_t sa) { return __ldg(a.cost32 + sa); }
    static __device__ __forceinline__ void edge(const SweepArgs &a, uint32_t t, int32_t &c, Prob &p) {
        const int2 e = __ldg(a.cp32 + t);
        c = e.x;
        p = __int_as_float(e.y);
    }
    static __device__ __forceinline__ Val reward(W w, Cost c, bool pre) {
        return __fsub_rd(pre ? w.y : 0.0f, __fmul_ru(w.x, c));
    }
    static __device__ __forceinline__ void mac(Val &acc, Prob p, Val v) { acc = __fmaf_rd(p, v, acc); }
    static __device__ __forceinline__ void close(Val &) {}
    static __device__ __forceinline__ bool gt(Val a, Val b) { return a > b; }
    static __device__ __forceinline__ Val neg_inf() { return -CUDART_INF_F; }
    static __device__ __forceinline__ Val zero() { return 0.0f; }
    static __device__ __forceinline__ float diff(Val y, Val x) { return fabsf(y - x); }
    static __device__ __forceinline__ Val from_words(const float *w) { return w[0]; }
    static __device__ __forceinline__ void to_words(Val v, float *w) { w[0] = v; }
    // Algorithm 3 records the maximiser when the value moves by more than
    // eps1.  In FP32 a move of a few ulps is rounding, not propagation, so
    // this phase records only moves above 64 ulps of the new value (the
    // double-float phase that follows records with eps1 itself).
    static __device__ __forceinline__ float record_threshold(Val y, double eps1) {
        const float rel = y * 7.62939453125e-06f; /* 2^-17 */
        return rel > (float)eps1 ? rel : (float)eps1;
    }
};

struct ArithDF {
    using Val = DF;
    using W = float4;    // (w_i.h, w_i.l, w_p.h, w_p.l)
    using Cost = DF;
    using Prob = DF;
    static constexpr int WORDS = 2;
    static __device__ __forceinline__ W weight(const SweepArgs &a, size_t pair) { return a.wdf[pair]; }
    static __device__ __forceinline__ Cost cost(const SweepArgs &a, uint32_t sa) {
        const float2 c = __ldg(a.costdf + sa);
        return {c.x, c.y};
    }
    static __device__ __forceinline__ void edge(const SweepArgs &a, uint32_t t, int32_t &c, Prob &p) {
        c = __ldg(a.col + t);
        const float2 q = __ldg(a.pdf + t);
        p = {q.x, q.y};
    }
    static __device__ __forceinline__ Val reward(W w, Cost c, bool pre) {
        const DF m = df_mul({w.x, w.y}, c);
        const DF base = pre ? DF{w.z, w.w} : DF{0.0f, 0.0f};
        return df_add(base, {-m.h, -m.l});
    }
    // acc += p * v with the sum left unnormalised until the action closes
    static __device__ __forceinline__ void mac(Val &acc, Prob p, Val v) {
        const float ph = __fmul_rn(p.h, v.h);
        float pe = __fmaf_rn(p.h, v.h, -ph);
        pe = __fmaf_rn(p.h, v.l, pe);
        pe = __fmaf_rn(p.l, v.h, pe);
        const DF s = two_sum(acc.h, ph);
        acc.h = s.h;
        acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, pe));
    }
    static __device__ __forceinline__ void close(Val &v) { v = df_norm(v); }
    static __device__ __forceinline__ bool gt(Val a, Val b) { return df_gt(a, b); }
    static __device__ __forceinline__ Val neg_inf() { return {-CUDART_INF_F, 0.0f}; }
    static __device__ __forceinline__ Val zero() { return {0.0f, 0.0f}; }
    static __device__ __forceinline__ float diff(Val y, Val x) {
        return fabsf(__fadd_rn(__fadd_rn(y.h, -x.h), __fadd_rn(y.l, -x.l)));
    }
    static __device__ __forceinline__ Val from_words(const float *w) { return {w[0], w[1]}; }
    static __device__ __forceinline__ void to_words(Val v, float *w) {
        w[0] = v.h;
        w[1] = v.l;
    }
    static __device__ __forceinline__ float record_threshold(Val, double eps1) { return (float)eps1; }
};

// Load / store NW consecutive 32-bit words with the widest aligned accesses.
template <int NW>
__device__ __forceinline__ void load_words(const float *p, float (&w)[NW]) {
    if constexpr (NW >= 4) {
#pragma unroll
        for (int i = 0; i < NW / 4; ++i) {
            const float4 q = __ldg(reinterpret_cast<const float4 *>(p) + i);
            w[4 * i] = q.x, w[4 * i + 1] = q.y, w[4 * i + 2] = q.z, w[4 * i + 3] = q.w;
        }
    } else if constexpr (NW == 2) {
        const float2 q = __ldg(reinterpret_cast<const float2 *>(p));
        w[0] = q.x, w[1] = q.y;
    } else {
        w[0] = __ldg(p);
    }
}

template <int NW>
__device__ __forceinline__ void store_words(float *p, const float (&w)[NW]) {
    if constexpr (NW >= 4) {
#pragma unroll
        for (int i = 0; i < NW / 4; ++i)
            reinterpret_cast<float4 *>(p)[i] = make_float4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
    } else if constexpr (NW == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(w[0], w[1]);
    } else {
        p[0] = w[0];
    }
}

// Lanes per state and weights per lane for each (format, Kp).
template <class Ar, int KP>
struct Shape {
    static constexpr int VMAX = Ar::WORDS == 1 ? 8 : 4;  // weights per lane
    static constexpr int VEC = KP < VMAX ? KP : VMAX;
    static constexpr int LPS = KP / VEC;                  // lanes per state (<= 32)
    static constexpr int SPW = 32 / LPS;                  // states per warp round
};

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double as_double(unsigned long long b) { return __longlong_as_double((long long)b); }

template <typename T, int VEC>
struct Vec {
    T v[VEC];
};

template <typename T, int VEC>
__device__ __forceinline__ Vec<T, VEC> vload(const T *p) {
    Vec<T, VEC> r;
    if constexpr (sizeof(T) * VEC == 16) {
        const double2 q = __ldg(reinterpret_cast<const double2 *>(p));
        r.v[0] = q.x, r.v[1] = q.y;
    } else {
        r.v[0] = __ldg(p);
    }
    return r;
}

// ------------------------------------------------------------- the sweep
//
// Work items are 128-state ranges of one product taken by whole warps
// (dynamic scheduling, no block barriers).  Inside a warp, LPS lanes share a
// state and each lane owns VEC of the Kp weights, so a successor's value row
// is read once, coalesced, for all weights.  Each lane consumes its state's
// transitions as one stream across the actions, issuing kGatherBatch
// independent gathers before it consumes them.
template <class Ar, int KP>
__global__ void __launch_bounds__(kThreads, 3) k_sweep(SweepArgs a, int pos) {
    using Val = typename Ar::Val;
    using SH = Shape<Ar, KP>;
    constexpr int VEC = SH::VEC, LPS = SH::LPS, SPW = SH::SPW;
    constexpr int NW = VEC * Ar::WORDS;      // 32-bit words a lane moves per state row
    constexpr int D = NW >= 8 ? kGatherBatch / 2 : kGatherBatch;  // keep the batch within registers
    constexpr int ROW = KP * Ar::WORDS;      // words per state row
    const int cur = pos % 3, nxt = (pos + 1) % 3, far = (pos + 2) % 3;
    const float *__restrict__ Vold = static_cast<const float *>(a.V[pos & 1]);
    float *__restrict__ Vnew = static_cast<float *>(a.V[(pos + 1) & 1]);
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
    const int lane = threadIdx.x & 31;
    const int grp = lane / LPS, li = lane % LPS, k0 = li * VEC;

    for (;;) {
        unsigned int it = 0;
        if (lane == 0) it = atomicAdd(&ctl->next[cur], 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const unsigned int item = a.list[cur][it];
        const int4 ch = a.chunks[item];
        const int p = ch.x;
        const size_t pair0 = (size_t)p * KP;
        // activity of the product's weights from the previous sweep's residuals
        unsigned int act_w[2] = {0u, 0u}, nz_w[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < (KP + 31) / 32; ++h) {
            const int k = lane + 32 * h;
            bool act = false, nz = false;
            if (k < KP) {
                const double prev = as_double(res_prev[pair0 + k]);
                act = prev > a.thr[pair0 + k];
                nz = prev > 0.0;
            }
            act_w[h] = __ballot_sync(0xffffffffu, act);
            nz_w[h] = __ballot_sync(0xffffffffu, nz);
        }
        const bool any_active = (act_w[0] | act_w[1]) != 0u;
        if ((nz_w[0] | nz_w[1]) == 0u) {  // converged earlier and already copied: drop
            if (ch.w)
                for (int k = lane; k < KP; k += 32) a.frozen[pair0 + k] = 1;
            continue;
        }
        const ProdDesc pd = a.prods[p];
        if (lane == 0 && any_active) {
            const unsigned int at = atomicAdd(&ctl->cnt[nxt], 1u);
            a.list[nxt][at] = item;
        }
        if (ch.w)
            for (int k = lane; k < KP; k += 32) {
                res_next[pair0 + k] = 0ull;
                if ((act_w[k >> 5] >> (k & 31)) & 1u)
                    a.sweeps_pair[pair0 + k] = (int32_t)(sweep + 1);
                else
                    a.frozen[pair0 + k] = 1;
            }
        bool act[VEC];
        typename Ar::W w[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int k = k0 + v;
            act[v] = ((act_w[k >> 5] >> (k & 31)) & 1u) != 0u;
            w[v] = Ar::weight(a, pair0 + k);
        }
        float rmax[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) rmax[v] = 0.0f;

        for (int s = ch.y + grp; s < ch.z; s += SPW) {
            const uint32_t u = pd.state_off + (uint32_t)s;
            const size_t row = (size_t)u * ROW + (size_t)k0 * Ar::WORDS;
            float yw[NW];
            if (!any_active) {  // every weight of the product froze: copy the row
                load_words<NW>(Vold + row, yw);
                store_words<NW>(Vnew + row, yw);
                continue;
            }
            const bool pre = (uint32_t)s >= pd.pre_begin;
            const uint32_t a0 = __ldg(a.state_sa + u), a1 = __ldg(a.state_sa + u + 1);
            const uint32_t te = __ldg(a.sa_tr + a1);
            Val best[VEC], acc[VEC];
            uint32_t best_a[(VEC + 3) / 4];  // recorded-action candidates, 8 bits per weight
            uint32_t sa = a0, bound = __ldg(a.sa_tr + a0 + 1);
            {
                const typename Ar::Cost c0 = Ar::cost(a, a0);
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    best[v] = Ar::neg_inf();
                    acc[v] = Ar::reward(w[v], c0, pre);
                }
#pragma unroll
                for (int i = 0; i < (VEC + 3) / 4; ++i) best_a[i] = 0u;
            }
            for (uint32_t base = __ldg(a.sa_tr + a0); base < te; base += D) {
                int32_t cl[D];
                typename Ar::Prob pr[D];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    if (base + i < te) {
                        Ar::edge(a, base + i, cl[i], pr[i]);
                    } else {
                        cl[i] = -1;
                    }
                }
                float gw[D][NW];
#pragma unroll
                for (int i = 0; i < D; ++i)
                    if (cl[i] >= 0) load_words<NW>(Vold + (size_t)cl[i] * ROW + (size_t)k0 * Ar::WORDS, gw[i]);
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    if (cl[i] < 0) continue;
                    while (base + i >= bound) {  // close action sa, open the next one
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            Ar::close(acc[v]);
                            if (Ar::gt(acc[v], best[v])) {
                                best[v] = acc[v];
                                best_a[v / 4] = (best_a[v / 4] & ~(0xFFu << (8 * (v % 4)))) | ((sa - a0) << (8 * (v % 4)));
                            }
                        }
                        ++sa;
                        bound = __ldg(a.sa_tr + sa + 1);
                        const typename Ar::Cost cs = Ar::cost(a, sa);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[v] = Ar::reward(w[v], cs, pre);
                    }
#pragma unroll
                    for (int v = 0; v < VEC; ++v) Ar::mac(acc[v], pr[i], Ar::from_words(&gw[i][v * Ar::WORDS]));
                }
            }
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                Ar::close(acc[v]);
                if (Ar::gt(acc[v], best[v])) {
                    best[v] = acc[v];
                    best_a[v / 4] = (best_a[v / 4] & ~(0xFFu << (8 * (v % 4)))) | ((sa - a0) << (8 * (v % 4)));
                }
            }
            load_words<NW>(Vold + row, yw);  // x; replaced below by y for the active weights
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                if (!act[v]) continue;
                const float d = Ar::diff(best[v], Ar::from_words(&yw[v * Ar::WORDS]));
                rmax[v] = d > rmax[v] ? d : rmax[v];
                if (d > Ar::record_threshold(best[v], a.eps1))
                    a.a_rec[(size_t)u * KP + k0 + v] = (uint8_t)(best_a[v / 4] >> (8 * (v % 4)));
                Ar::to_words(best[v], &yw[v * Ar::WORDS]);
            }
            store_words<NW>(Vnew + row, yw);
        }
        // residual: lanes with the same li share weights
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            float r = rmax[v];
#pragma unroll
            for (int off = LPS; off < 32; off <<= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, off));
            if (grp == 0 && any_active && r > 0.0f) atomic_max_nonneg(res_cur + pair0 + k0 + v, (double)r);
        }
        if (lane == 0) {
            const uint32_t n_s = (uint32_t)(ch.z - ch.y);
            const uint32_t u0 = pd.state_off + ch.y, u1 = pd.state_off + ch.z;
            unsigned long long bytes = 2ull * n_s * ROW * 4;
            if (any_active) {
                const uint32_t sa0 = a.state_sa[u0], sa1 = a.state_sa[u1];
                const uint32_t tr0 = a.sa_tr[sa0], tr1 = a.sa_tr[sa1];
                const int n_act = __popc(act_w[0]) + __popc(act_w[1]);
                atomicAdd(&ctl->updates, (unsigned long long)(tr1 - tr0) * (unsigned long long)n_act);
                // state_sa, sa_tr, cost and (col, p) per transition, 4 bytes per word
                bytes += 4ull * (n_s + 1) + 4ull * (sa1 - sa0 + 1) + 4ull * Ar::WORDS * (sa1 - sa0) +
                         4ull * (1 + Ar::WORDS) * (tr1 - tr0);
            }
            atomicAdd(&ctl->bytes, bytes);
        }
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
    constexpr int VEC = KP < 2 ? KP : 2, LPS = KP / VEC, SPR = kThreads / LPS;
    constexpr int MAXA = 32;  // actions scanned twice per state: first for the max, then for the choice
    const float2 *__restrict__ V = static_cast<const float2 *>(a.V[0]);  // double-float values
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
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            const float2 xv = V[(size_t)cl * KP + k0 + v];
                            acc[v] = fma(pr, (double)xv.x + (double)xv.y, acc[v]);
                        }
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

__device__ __forceinline__ float2 to_df(double d) {
    const float h = __double2float_rn(d);
    return make_float2(h, __double2float_rn(d - (double)h));
}

__global__ void k_setup_weights(const ProdDesc *prods, int P, int nI, int nJ, int K, int Kp, const double *W,
                                float2 *w32, double2 *w64, float4 *wdf, double *thr32, double *thr64, double eps1) {
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
        const float2 a = to_df(wi), b = to_df(wp);
        wdf[idx] = make_float4(a.x, a.y, b.x, b.y);
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

__global__ void k_convert(const float *v32, float2 *a, float2 *b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 v = make_float2(v32[i], 0.0f);
        a[i] = v;
        b[i] = v;
    }
}

// c_ij = V(s0, q0) for every (product, weight); a pair that never froze
// stopped at the sweep cap.
__global__ void k_gather_c(int Kp, const ProdDesc *prods, int P, const float2 *V, const uint8_t *frozen,
                           double *c_out, int32_t *status_out) {
    const size_t n = (size_t)P * Kp;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(idx / Kp), k = (int)(idx % Kp);
        const ProdDesc pd = prods[p];
        double v = 0.0;
        if ((uint32_t)pd.init_local < pd.n_nd) {
            const float2 x = V[(size_t)(pd.state_off + pd.init_local) * Kp + k];
            v = (double)x.x + (double)x.y;
        }
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

template <class Ar>
int launch_sweep_t(int Kp, const SweepArgs &a, int pos, int grid, cudaStream_t s) {
    switch (Kp) {
    case 1: k_sweep<Ar, 1><<<grid, kThreads, 0, s>>>(a, pos); break;
    case 2: k_sweep<Ar, 2><<<grid, kThreads, 0, s>>>(a, pos); break;
    case 4: k_sweep<Ar, 4><<<grid, kThreads, 0, s>>>(a, pos); break;
    case 8: k_sweep<Ar, 8><<<grid, kThreads, 0, s>>>(a, pos); break;
    case 16: k_sweep<Ar, 16><<<grid, kThreads, 0, s>>>(a, pos); break;
    case 32: k_sweep<Ar, 32><<<grid, kThreads, 0, s>>>(a, pos); break;
    case 64: k_sweep<Ar, 64><<<grid, kThreads, 0, s>>>(a, pos); break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

}  // namespace

template <class Ar>
int blocks_per_sm_t(int Kp) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (Kp) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<Ar, 1>, kThreads, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<Ar, 2>, kThreads, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<Ar, 4>, kThreads, 0); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<Ar, 8>, kThreads, 0); break;
    case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<Ar, 16>, kThreads, 0); break;
    case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<Ar, 32>, kThreads, 0); break;
    case 64: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<Ar, 64>, kThreads, 0); break;
    default: break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

int sweep_blocks_per_sm(bool fp64, int Kp) { return fp64 ? blocks_per_sm_t<ArithDF>(Kp) : blocks_per_sm_t<ArithF32>(Kp); }

int eval_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_eval_sweep, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

int launch_sweep(bool fp64, int Kp, const SweepArgs &a, int pos, int grid, void *s) {
    return fp64 ? launch_sweep_t<ArithDF>(Kp, a, pos, grid, (cudaStream_t)s)
                : launch_sweep_t<ArithF32>(Kp, a, pos, grid, (cudaStream_t)s);
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
                         double2 *w64, float4 *wdf, double *thr32, double *thr64, double eps1, void *s) {
    const size_t n = (size_t)P * Kp;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_setup_weights<<<grid > 0 ? grid : 1, 256, 0, (cudaStream_t)s>>>(prods, P, nI, nJ, K, Kp, W, w32, w64, wdf,
                                                                     thr32, thr64, eps1);
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

int launch_convert(const float *v32, float2 *vda, float2 *vdb, size_t n, void *s) {
    const int grid = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
    k_convert<<<grid > 0 ? grid : 1, 256, 0, (cudaStream_t)s>>>(v32, vda, vdb, n);
    return (int)cudaGetLastError();
}

int launch_gather_c(int Kp, const ProdDesc *prods, int P, const float2 *V64, const uint8_t *frozen, double *c_out,
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

// Batched Bellman sweeps of Algorithm 3 and Algorithm 4 over all products
// and all weights of a batch, with the per-(product, weight) residual
// reduction, the device work lists and the loop control that a CUDA-graph
// while node evaluates between bodies.
//
// Data layout (HBM):
//   values  V[state][Kp]   (Kp = weights padded to a power of two), double
//                          buffered; a sweep reads V[n % 2] and writes
//                          V[(n + 1) % 2] (synchronous sweeps, as the oracle;
//                          with in-place sweeps both are one array)
//   a_rec   [state][Kp]    uint8 local action recorded by Algorithm 3
//   CSR     state_sa[state+1] -> sa_tr[sa+1] -> col[t], p[t]
//
// Thread mapping: LPS = Kp / VEC lanes share one state, lane l owns weights
// [l*VEC, l*VEC+VEC) and loads them as one vector, so the value row of a
// successor is one coalesced Kp-wide read and the CSR stream is read once for
// all Kp weights.  Each warp takes kChunk-state work items of one product
// from the sweep's work list (its first without an atomic, then one item per
// atomic); an item's residuals are reduced with warp shuffles and one 64-bit
// atomicMax per weight.  Items none of whose inputs changed in the previous sweep are
// skipped exactly (see SweepArgs::in_items).
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

#include <array>
#include <cstdint>
#include <type_traits>
#include <utility>

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

__device__ __forceinline__ bool df_gt(DF a, DF b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }

__device__ __forceinline__ void cp_async4(void *smem, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(g));
}
__device__ __forceinline__ void cp_async8(void *smem, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(g));
}
// Ask L2 to fetch a contiguous range of global memory (a hint with no
// completion and no effect on results).  Start and size must be multiples of
// 16 bytes, and the range must lie inside one allocation.
__device__ __forceinline__ void prefetch_l2(const void *g, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(g), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Per-warp staging capacity: up to kStageStates states whose rows and
// transitions fit AMAX / EMAX entries are copied to shared memory per batch.
constexpr int kStageStates = 32;  // states per batch (at most; fewer when the rows do not fit)

struct ArithF32 {
    using Val = float;
    static constexpr int AMAX = 192, EMAX = 448;
    // ssa[kStageStates + 1] | str[AM + 1] | cost[AM] | edge[EM] (int2)
    template <int AM, int EM>
    struct Lay {
        static constexpr int STR = 136, COST = STR + 4 * (AM + 2), EDGE = COST + 4 * AM, BYTES = EDGE + 8 * EM;
    };
    static constexpr int STAGE_BYTES = Lay<AMAX, EMAX>::BYTES;
    struct View {
        const uint32_t *str;
        const float *cost;
        const int2 *edge;
    };
    template <int AM = AMAX, int EM = EMAX>
    static __device__ __forceinline__ View smem_view(unsigned char *b) {
        using L = Lay<AM, EM>;
        return {reinterpret_cast<const uint32_t *>(b + L::STR), reinterpret_cast<const float *>(b + L::COST),
                reinterpret_cast<const int2 *>(b + L::EDGE)};
    }
    static __device__ __forceinline__ View global_view(const SweepArgs &a, uint32_t A0, uint32_t T0) {
        return {a.sa_tr + A0, a.cost32 + A0, a.cp32 + T0};
    }
    template <int AM = AMAX, int EM = EMAX>
    static __device__ __forceinline__ void stage(const SweepArgs &a, unsigned char *b, uint32_t A0, uint32_t nA,
                                                 uint32_t T0, uint32_t nT, int lane) {
        using L = Lay<AM, EM>;
        uint32_t *str = reinterpret_cast<uint32_t *>(b + L::STR);
        float *cost = reinterpret_cast<float *>(b + L::COST);
        int2 *edge = reinterpret_cast<int2 *>(b + L::EDGE);
        for (uint32_t i = lane; i <= nA; i += 32) cp_async4(str + i, a.sa_tr + A0 + i);
        for (uint32_t i = lane; i < nA; i += 32) cp_async4(cost + i, a.cost32 + A0 + i);
        for (uint32_t i = lane; i < nT; i += 32) cp_async8(edge + i, a.cp32 + T0 + i);
    }
    using W = float2;    // (-w_i rounded away from zero, w_p rounded down)
    using Cost = float;  // rounded up
    using Prob = float;  // rounded down
    static constexpr int WORDS = 1;
    static __device__ __forceinline__ W weight(const SweepArgs &a, size_t pair) { return a.w32[pair]; }
    static __device__ __forceinline__ Cost cost(const View &v, uint32_t la) { return v.cost[la]; }
    static __device__ __forceinline__ void edge(const View &v, uint32_t lt, int32_t &c, Prob &p) {
        const int2 e = v.edge[lt];
        c = e.x;
        p = __int_as_float(e.y);
    }
    // rd(-w_i' c) with w_i' >= w_i and c rounded up: a lower bound of the
    // action's reward; the pre-sink weight (the same for every action of a
    // state) is added once, after the maximum, by add_base
    using CW = float;  // the part of W the reward needs
    static __device__ __forceinline__ CW cost_weight(W w) { return w.x; }
    static __device__ __forceinline__ Val reward_cw(CW w, Cost c) { return __fmul_rd(w, c); }
    static __device__ __forceinline__ Val reward(W w, Cost c) { return reward_cw(cost_weight(w), c); }
    static __device__ __forceinline__ Val add_base(Val v, W w, bool pre) { return pre ? __fadd_rd(v, w.y) : v; }
    static __device__ __forceinline__ void mac(Val &acc, Prob p, Val v) { acc = __fmaf_rd(p, v, acc); }
    static __device__ __forceinline__ void close(Val &) {}
    static __device__ __forceinline__ bool gt(Val a, Val b) { return a > b; }
    static __device__ __forceinline__ Val neg_inf() { return -CUDART_INF_F; }
    static __device__ __forceinline__ float diff(Val y, Val x) { return fabsf(y - x); }
    static __device__ __forceinline__ Val from_words(const float *w) { return w[0]; }
    static __device__ __forceinline__ void to_words(Val v, float *w) { w[0] = v; }
    // Algorithm 3 records the maximiser when the value moves by more than
    // eps1.  In FP32 a move of a few ulps is rounding, not propagation, so
    // this phase records only moves above 64 ulps of the new value (the
    // double-float phase that follows records with eps1 itself).
    static __device__ __forceinline__ float record_threshold(Val y, float eps1) {
        const float rel = y * 7.62939453125e-06f; /* 2^-17 */
        return rel > eps1 ? rel : eps1;
    }
};

struct ArithDF {
    using Val = DF;
    static constexpr int AMAX = 192, EMAX = 448;
    // ssa | str[AM + 1] | cost[AM] (float2) | col[EM] | p[EM] (float2)
    template <int AM, int EM>
    struct Lay {
        static constexpr int STR = 136, COST = STR + 4 * (AM + 2), COL = COST + 8 * AM, P = COL + 4 * EM,
                             BYTES = P + 8 * EM;
    };
    static constexpr int STAGE_BYTES = Lay<AMAX, EMAX>::BYTES;
    struct View {
        const uint32_t *str;
        const float2 *cost;
        const int32_t *col;
        const float2 *p;
    };
    template <int AM = AMAX, int EM = EMAX>
    static __device__ __forceinline__ View smem_view(unsigned char *b) {
        using L = Lay<AM, EM>;
        return {reinterpret_cast<const uint32_t *>(b + L::STR), reinterpret_cast<const float2 *>(b + L::COST),
                reinterpret_cast<const int32_t *>(b + L::COL), reinterpret_cast<const float2 *>(b + L::P)};
    }
    static __device__ __forceinline__ View global_view(const SweepArgs &a, uint32_t A0, uint32_t T0) {
        return {a.sa_tr + A0, a.costdf + A0, a.col + T0, a.pdf + T0};
    }
    template <int AM = AMAX, int EM = EMAX>
    static __device__ __forceinline__ void stage(const SweepArgs &a, unsigned char *b, uint32_t A0, uint32_t nA,
                                                 uint32_t T0, uint32_t nT, int lane) {
        using L = Lay<AM, EM>;
        uint32_t *str = reinterpret_cast<uint32_t *>(b + L::STR);
        float2 *cost = reinterpret_cast<float2 *>(b + L::COST);
        int32_t *col = reinterpret_cast<int32_t *>(b + L::COL);
        float2 *p = reinterpret_cast<float2 *>(b + L::P);
        for (uint32_t i = lane; i <= nA; i += 32) cp_async4(str + i, a.sa_tr + A0 + i);
        for (uint32_t i = lane; i < nA; i += 32) cp_async8(cost + i, a.costdf + A0 + i);
        for (uint32_t i = lane; i < nT; i += 32) {
            cp_async4(col + i, a.col + T0 + i);
            cp_async8(p + i, a.pdf + T0 + i);
        }
    }
    using W = float4;    // (w_i.h, w_i.l, w_p.h, w_p.l)
    using Cost = DF;
    using Prob = DF;
    static constexpr int WORDS = 2;
    static __device__ __forceinline__ W weight(const SweepArgs &a, size_t pair) { return a.wdf[pair]; }
    static __device__ __forceinline__ Cost cost(const View &v, uint32_t la) {
        const float2 c = v.cost[la];
        return {c.x, c.y};
    }
    static __device__ __forceinline__ void edge(const View &v, uint32_t lt, int32_t &c, Prob &p) {
        c = v.col[lt];
        const float2 q = v.p[lt];
        p = {q.x, q.y};
    }
    // -w_i c, left unnormalised (the accumulation that follows tolerates
    // it); the pre-sink weight is added once per state by add_base
    using CW = float2;  // w_i as (hi, lo)
    static __device__ __forceinline__ CW cost_weight(W w) { return make_float2(w.x, w.y); }
    static __device__ __forceinline__ Val reward_cw(CW w, Cost c) {
        const float m = __fmul_rn(w.x, c.h);
        float e = __fmaf_rn(w.x, c.h, -m);
        e = __fmaf_rn(w.x, c.l, e);
        e = __fmaf_rn(w.y, c.h, e);
        return {-m, -e};
    }
    static __device__ __forceinline__ Val reward(W w, Cost c) { return reward_cw(cost_weight(w), c); }
    static __device__ __forceinline__ Val add_base(Val v, W w, bool pre) { return pre ? df_add({w.z, w.w}, v) : v; }
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
    static __device__ __forceinline__ float diff(Val y, Val x) {
        return fabsf(__fadd_rn(__fadd_rn(y.h, -x.h), __fadd_rn(y.l, -x.l)));
    }
    static __device__ __forceinline__ Val from_words(const float *w) { return {w[0], w[1]}; }
    static __device__ __forceinline__ void to_words(Val v, float *w) {
        w[0] = v.h;
        w[1] = v.l;
    }
    static __device__ __forceinline__ float record_threshold(Val, float eps1) { return eps1; }
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

// Value loads of the sweeps.  One launch per sweep reads values no kernel of
// the launch writes (the read-only path); a launch that runs several sweeps
// (COH) reads values other blocks wrote in its previous sweep, so it loads
// them from L2 (ld.global.cg), never from an SM's non-coherent cache.
template <int NW, bool COH>
__device__ __forceinline__ void load_vals(const float *p, float (&w)[NW]) {
    if constexpr (!COH) {
        load_words<NW>(p, w);
    } else if constexpr (NW >= 4) {
#pragma unroll
        for (int i = 0; i < NW / 4; ++i) {
            const float4 q = __ldcg(reinterpret_cast<const float4 *>(p) + i);
            w[4 * i] = q.x, w[4 * i + 1] = q.y, w[4 * i + 2] = q.z, w[4 * i + 3] = q.w;
        }
    } else if constexpr (NW == 2) {
        const float2 q = __ldcg(reinterpret_cast<const float2 *>(p));
        w[0] = q.x, w[1] = q.y;
    } else {
        w[0] = __ldcg(p);
    }
}

// A load of loop state written during the launch (residuals, change flags,
// work lists, counters): from L2 when the launch runs several sweeps.
template <bool COH, typename T>
__device__ __forceinline__ T ld_loop(const T *p) {
    if constexpr (COH)
        return __ldcg(p);
    else
        return *p;
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

// The polish phase as a residual correction (the default after an FP32
// phase).  With B the certified FP32 lower bound the FP32 phase ends on and
// V = B + d, the Bellman update of state s reads
//   y(s) - B(s) = max_a [ G_a(s) + sum_s' p d(s') ],
//   G_a(s)      = r_a(s) + sum_s' p B(s') - B(s),
// so once G (one value per state-action row and weight) has been formed in
// double-float from B and rounded to FP32, the correction d is iterated in
// plain FP32 with one fused multiply-add per transition and weight.  d is of
// the size of B's remaining error (about 1e-5 of the values), so FP32
// carries it to about 1e-12; the winning G_a are of the same size.  d
// starts at 0, the sweeps, freezes and records follow the paper's rule on d
// (y - x is the same quantity in V and in d), and V = B + d is formed
// exactly in double-float at the end.
struct ArithDelta : ArithF32 {
    using Prob = float;
    // the rows' costs are inside G: only the row starts and the transitions are staged
    template <int AM = AMAX, int EM = EMAX>
    static __device__ __forceinline__ void stage(const SweepArgs &a, unsigned char *b, uint32_t A0, uint32_t nA,
                                                 uint32_t T0, uint32_t nT, int lane) {
        using L = Lay<AM, EM>;
        uint32_t *str = reinterpret_cast<uint32_t *>(b + L::STR);
        int2 *edge = reinterpret_cast<int2 *>(b + L::EDGE);
        for (uint32_t i = lane; i <= nA; i += 32) cp_async4(str + i, a.sa_tr + A0 + i);
        for (uint32_t i = lane; i < nT; i += 32) cp_async8(edge + i, a.cp32 + T0 + i);
    }
    static __device__ __forceinline__ Val add_base(Val v, W, bool) { return v; }  // inside G
    static __device__ __forceinline__ void mac(Val &acc, Prob p, Val v) { acc = __fmaf_rn(p, v, acc); }
    static __device__ __forceinline__ float record_threshold(Val, float eps1) { return eps1; }
};

// The value of action row la before its transitions are added: the
// scalarised reward, or for the residual correction the row of G.
template <class Ar, int KP, int VEC>
__device__ __forceinline__ void init_action(const SweepArgs &a, const typename Ar::View &vw, uint32_t A0,
                                            uint32_t la, int k0, const typename Ar::W *__restrict__ sw,
                                            typename Ar::Val (&acc)[VEC]) {
    if constexpr (std::is_same<Ar, ArithDelta>::value) {
        float g[VEC];
        load_words<VEC>(a.G + (size_t)(A0 + la) * KP + k0, g);
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = g[v];
    } else {
        const typename Ar::Cost c = Ar::cost(vw, la);
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = Ar::reward(sw[v], c);
    }
}

// Kernel shapes the tuner chooses from, per value format: VMAX weights per
// lane (a lane owns VEC = min(Kp, VMAX) consecutive weights of a state), D
// successor gathers in flight per action, and MINB resident blocks per SM
// the register allocation is sized for.  Entry 0 is the default.  Every
// shape performs the same operations in the same order per (state, weight),
// so all of them give bit-identical results.
template <class Ar>
struct Variants;
template <>
struct Variants<ArithF32> {
    static constexpr int N = 4;
    static constexpr int vmax[N] = {8, 8, 4, 8};
    static constexpr int d[N] = {3, 4, 2, 2};  // shape 2: D = 2 keeps 3 blocks per SM free of spills
    static constexpr int minb[N] = {2, 2, 3, 2};
    static constexpr int pipe[N] = {0, 0, 0, 1};  // actions software-pipelined
};
template <>
struct Variants<ArithDelta> : Variants<ArithF32> {};
template <>
struct Variants<ArithDF> {
    static constexpr int N = 4;
    static constexpr int vmax[N] = {4, 4, 2, 4};
    static constexpr int d[N] = {3, 4, 2, 2};
    static constexpr int minb[N] = {2, 2, 3, 2};
    static constexpr int pipe[N] = {0, 0, 0, 1};
};

// Lanes per state and weights per lane for each (format, Kp, VMAX).
template <class Ar, int KP, int VMAX>
struct Shape {
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
// Work items are kChunk-state ranges of one product taken by whole warps
// (dynamic scheduling, no block barriers).  A warp walks its item in
// batches: it copies the batch's state starts, action-row starts, costs and
// (successor, probability) stream into its own shared-memory buffer with
// cp.async (one coalesced round trip per batch instead of one per
// transition), then computes.  Inside the batch, LPS lanes share a state and
// each lane owns VEC of the Kp weights, so a successor's value row is read
// once, coalesced, for all weights.  Actions are the outer loop; within an
// action a lane issues D independent value gathers before it consumes them.
template <class Ar, int KP, int VMAX, int D, bool COH>
__device__ __forceinline__ void process_state(const SweepArgs &a, const typename Ar::View &vw, const uint32_t *ssa,
                                              uint32_t A0, uint32_t T0, int i, uint32_t u, bool pre,
                                              const typename Ar::W *__restrict__ sw, const unsigned int act_bits,
                                              const float *__restrict__ Vold, float *__restrict__ Vnew, int k0,
                                              float (&rmax)[Shape<Ar, KP, VMAX>::VEC], bool &changed) {
    using Val = typename Ar::Val;
    using SH = Shape<Ar, KP, VMAX>;
    constexpr int VEC = SH::VEC;
    constexpr int NW = VEC * Ar::WORDS;
    constexpr int ROW = KP * Ar::WORDS;
    const size_t row = (size_t)u * ROW + (size_t)k0 * Ar::WORDS;
    const uint32_t la0 = ssa[i] - A0, la1 = ssa[i + 1] - A0;
    Val best[VEC];
    // the maximising actions; one byte per weight for Kp >= 32, where the
    // registers it saves avoid spills (smaller Kp run faster unpacked)
    constexpr int PACK = KP >= 32 ? 4 : 1;
    uint32_t best_a[(VEC + PACK - 1) / PACK];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
        best[v] = Ar::neg_inf();
        if (v % PACK == 0) best_a[v / PACK] = 0u;
    }
    uint32_t t0 = vw.str[la0] - T0;
    // Actions are the outer loop: every lane closes an action at the same
    // point of the instruction stream, whatever its transition counts.
    for (uint32_t la = la0; la < la1; ++la) {
        const uint32_t t1 = vw.str[la + 1] - T0;
        Val acc[VEC];
        init_action<Ar, KP, VEC>(a, vw, A0, la, k0, sw, acc);
        for (uint32_t base = t0; base < t1; base += D) {
            int32_t cl[D];
            typename Ar::Prob pr[D];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                if (base + j < t1) {
                    Ar::edge(vw, base + j, cl[j], pr[j]);
                } else {
                    cl[j] = -1;
                }
            }
            float gw[D][NW];
#pragma unroll
            for (int j = 0; j < D; ++j)
                if (cl[j] >= 0) load_vals<NW, COH>(Vold + (size_t)cl[j] * ROW + (size_t)k0 * Ar::WORDS, gw[j]);
#pragma unroll
            for (int j = 0; j < D; ++j) {
                if (cl[j] < 0) continue;
#pragma unroll
                for (int v = 0; v < VEC; ++v) Ar::mac(acc[v], pr[j], Ar::from_words(&gw[j][v * Ar::WORDS]));
            }
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            Ar::close(acc[v]);
            const bool better = Ar::gt(acc[v], best[v]);
            best[v] = better ? acc[v] : best[v];
            if constexpr (PACK == 1) {
                best_a[v] = better ? la - la0 : best_a[v];
            } else if (better) {
                const int sh = 8 * (v % PACK);
                best_a[v / PACK] = (best_a[v / PACK] & ~(0xFFu << sh)) | ((la - la0) << sh);
            }
        }
        t0 = t1;
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v) best[v] = Ar::add_base(best[v], sw[v], pre);
    float yw[NW];
    load_vals<NW, COH>(Vold + row, yw);  // x; replaced below by y for the active weights
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
        if (!((act_bits >> v) & 1u)) continue;
        const float d = Ar::diff(best[v], Ar::from_words(&yw[v * Ar::WORDS]));
        rmax[v] = d > rmax[v] ? d : rmax[v];
        if (d > Ar::record_threshold(best[v], a.eps1f)) a.a_rec[(size_t)u * KP + k0 + v] = (uint8_t)(best_a[v / PACK] >> (8 * (v % PACK)));
        float before[Ar::WORDS];
#pragma unroll
        for (int q = 0; q < Ar::WORDS; ++q) before[q] = yw[v * Ar::WORDS + q];
        Ar::to_words(best[v], &yw[v * Ar::WORDS]);
#pragma unroll
        for (int q = 0; q < Ar::WORDS; ++q)
            changed = changed || __float_as_uint(before[q]) != __float_as_uint(yw[v * Ar::WORDS + q]);
    }
    store_words<NW>(Vnew + row, yw);
}

// The same per-state computation with the actions software-pipelined: the
// (successor, probability) slots of action a + 1 are read and their value
// gathers issued before action a is reduced, so one gather round trip is
// exposed per state instead of one per action.  Actions with more than D
// transitions finish their remaining slots unpipelined.  Same operations in
// the same order per (state, weight) as process_state.
template <class Ar, int KP, int VMAX, int D, bool COH>
__device__ __forceinline__ void process_state_pipe(const SweepArgs &a, const typename Ar::View &vw,
                                                   const uint32_t *ssa, uint32_t A0, uint32_t T0, int i, uint32_t u,
                                                   bool pre, const typename Ar::W *__restrict__ sw,
                                                   const unsigned int act_bits, const float *__restrict__ Vold,
                                                   float *__restrict__ Vnew, int k0,
                                                   float (&rmax)[Shape<Ar, KP, VMAX>::VEC], bool &changed) {
    using Val = typename Ar::Val;
    using Prob = typename Ar::Prob;
    using SH = Shape<Ar, KP, VMAX>;
    constexpr int VEC = SH::VEC;
    constexpr int NW = VEC * Ar::WORDS;
    constexpr int ROW = KP * Ar::WORDS;
    const float *__restrict__ vbase = Vold + (size_t)k0 * Ar::WORDS;
    const size_t row = (size_t)u * ROW + (size_t)k0 * Ar::WORDS;
    const uint32_t la0 = ssa[i] - A0, la1 = ssa[i + 1] - A0;
    Val best[VEC];
    // the maximising actions; one byte per weight for Kp >= 32, where the
    // registers it saves avoid spills (smaller Kp run faster unpacked)
    constexpr int PACK = KP >= 32 ? 4 : 1;
    uint32_t best_a[(VEC + PACK - 1) / PACK];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
        best[v] = Ar::neg_inf();
        if (v % PACK == 0) best_a[v / PACK] = 0u;
    }
    struct Slots {
        int32_t cl[D];
        Prob pr[D];
        float gw[D][NW];
        uint32_t t0, t1;
    };
    // read slots t0 .. t0 + D - 1 of the current row and issue their gathers
    auto fill = [&](Slots &S) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (S.t0 + j < S.t1) {
                Ar::edge(vw, S.t0 + j, S.cl[j], S.pr[j]);
            } else {
                S.cl[j] = -1;
            }
        }
#pragma unroll
        for (int j = 0; j < D; ++j)
            if (S.cl[j] >= 0) load_vals<NW, COH>(vbase + (size_t)S.cl[j] * ROW, S.gw[j]);
    };
    auto fetch = [&](uint32_t la, Slots &S) {
        S.t0 = vw.str[la] - T0;
        S.t1 = vw.str[la + 1] - T0;
        fill(S);
    };
    auto reduce = [&](uint32_t la, Slots &S) {
        Val acc[VEC];
        init_action<Ar, KP, VEC>(a, vw, A0, la, k0, sw, acc);
        for (;;) {
#pragma unroll
            for (int j = 0; j < D; ++j) {
                if (S.cl[j] < 0) continue;
#pragma unroll
                for (int v = 0; v < VEC; ++v) Ar::mac(acc[v], S.pr[j], Ar::from_words(&S.gw[j][v * Ar::WORDS]));
            }
            if (S.t0 + D >= S.t1) break;
            S.t0 += D;  // rows longer than D: the next slots, unpipelined
            fill(S);
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            Ar::close(acc[v]);
            const bool better = Ar::gt(acc[v], best[v]);
            best[v] = better ? acc[v] : best[v];
            if constexpr (PACK == 1) {
                best_a[v] = better ? la - la0 : best_a[v];
            } else if (better) {
                const int sh = 8 * (v % PACK);
                best_a[v / PACK] = (best_a[v / PACK] & ~(0xFFu << sh)) | ((la - la0) << sh);
            }
        }
    };
    Slots A, B;
    fetch(la0, A);
    for (uint32_t la = la0;;) {
        const bool more = la + 1 < la1;
        if (more) fetch(la + 1, B);
        reduce(la, A);
        if (!more) break;
        ++la;
        const bool more2 = la + 1 < la1;
        if (more2) fetch(la + 1, A);
        reduce(la, B);
        if (!more2) break;
        ++la;
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v) best[v] = Ar::add_base(best[v], sw[v], pre);
    float yw[NW];
    load_vals<NW, COH>(Vold + row, yw);  // x; replaced below by y for the active weights
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
        if (!((act_bits >> v) & 1u)) continue;
        const float d = Ar::diff(best[v], Ar::from_words(&yw[v * Ar::WORDS]));
        rmax[v] = d > rmax[v] ? d : rmax[v];
        if (d > Ar::record_threshold(best[v], a.eps1f)) a.a_rec[(size_t)u * KP + k0 + v] = (uint8_t)(best_a[v / PACK] >> (8 * (v % PACK)));
        float before[Ar::WORDS];
#pragma unroll
        for (int q = 0; q < Ar::WORDS; ++q) before[q] = yw[v * Ar::WORDS + q];
        Ar::to_words(best[v], &yw[v * Ar::WORDS]);
#pragma unroll
        for (int q = 0; q < Ar::WORDS; ++q)
            changed = changed || __float_as_uint(before[q]) != __float_as_uint(yw[v * Ar::WORDS + q]);
    }
    store_words<NW>(Vnew + row, yw);
}

// Named barrier of the G warps (G * 32 threads) of a work group; id >= 1
// (0 is __syncthreads).
__device__ __forceinline__ void group_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

// Work items are kChunk-state ranges of one product taken by groups of G
// warps (dynamic scheduling), walked in batches of up to 32 states: a warp
// copies the batch's state starts, action-row starts, costs and (successor,
// probability) stream into its own shared-memory buffer with cp.async, then
// computes.  Inside a batch, LPS lanes share a state and each lane owns VEC
// of the Kp weights, so a successor's value row is read once, coalesced, for
// all weights.
//
// G is 1 (one warp per item, no barriers) while the sweep's work list holds
// at least half as many items as the grid has warps; shorter lists (the late
// sweeps of a loop) split each item's states over G = 2, 4 or 8 warps of a
// block, so the item's chain of dependent loads is walked G times faster.
// Every warp of a group reads the item's bookkeeping (activity, exact-skip
// inputs) itself and takes the same decisions; the group's first warp does
// the item's writes (work list, freezes, change flag, residuals, counters)
// after a barrier that combines the warps' change flags and residuals.  The
// per-(state, weight) arithmetic does not depend on G, so neither do the
// results.
// Per-thread running sums of a launch's statistics (kept by the group
// leaders' lane 0), added to the loop's counters once per launch.
struct PassStats {
    unsigned long long updates, bytes;
    unsigned int skipped, computed;
};

// One sweep (pos = sweep mod 6: value buffer pos & 1, work list pos % 3).
// COH: the launch runs several sweeps, so everything the previous sweep wrote
// (values, residuals, change flags, lists, counters) is read from L2.
template <class Ar, int KP, int VMAX, int D, int PIPE, bool COH>
__device__ __forceinline__ void sweep_pass(const SweepArgs &a, int pos, unsigned int sweep, PassStats &ps) {
    using SH = Shape<Ar, KP, VMAX>;
    constexpr int VEC = SH::VEC, LPS = SH::LPS, SPW = SH::SPW;
    constexpr int NW = VEC * Ar::WORDS;
    constexpr int ROW = KP * Ar::WORDS;
    constexpr int WPB = kThreads / 32;  // warps per block
    constexpr int GMAX = (kChunk / SPW) < WPB ? (kChunk / SPW) : WPB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
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
    // group exchange: the item of the next two rounds (double buffered), each
    // warp's change flag and per-weight residuals
    __shared__ unsigned int g_it[2][WPB];
    __shared__ unsigned char g_chg[WPB];
    __shared__ float g_res[WPB][KP];
    const unsigned int n_items = ld_loop<COH>(&ctl->cnt[cur]);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;  // warp in block
    const int grp = lane / LPS, li = lane % LPS, k0 = li * VEC;
    unsigned char *warp_buf = smem_raw + wib * (Ar::STAGE_BYTES + KP * (int)sizeof(typename Ar::W));
    unsigned char *stage_buf = warp_buf;
    uint32_t *ssa = reinterpret_cast<uint32_t *>(stage_buf);
    typename Ar::W *wsm = reinterpret_cast<typename Ar::W *>(warp_buf + Ar::STAGE_BYTES);  // the item's weights

    const unsigned int n_warps = gridDim.x * WPB;
    int G = 1;  // warps per item, the same in every block
    const int gcap = a.gmax < GMAX ? a.gmax : GMAX;
    while (G < gcap && (unsigned long long)(2 * G) * n_items <= n_warps) G *= 2;
    const int gib = wib / G;           // group in block
    const int g = wib % G;             // warp in group
    const bool leader = g == 0;
    const int bar_id = 1 + gib, bar_threads = 32 * G;
    const unsigned int n_groups = n_warps / G;
    const unsigned int group_id = blockIdx.x * (WPB / G) + gib;

    // The shared counters see few atomics: the statistics are summed per warp
    // and per block, and items that stay in the work list are collected per
    // group leader (lane i holds the i-th) and appended a.keep_batch at a
    // time.  Large instances append each item at once instead (keep_batch =
    // 1): then the next list keeps the order of this one (neighbouring items
    // stay neighbours), which keeps the value gathers of concurrent warps
    // close together when the values do not fit in L2; batches would
    // interleave the warps' items from one sweep to the next.
    unsigned int kept = 0u;
    int n_kept = 0;  // warp-uniform
    auto flush_kept = [&]() {
        unsigned int at = 0;
        if (lane == 0) at = atomicAdd(&ctl->cnt[nxt], (unsigned int)n_kept);
        at = __shfl_sync(0xffffffffu, at, 0);
        if (lane < n_kept) a.list[nxt][at + lane] = kept;
        n_kept = 0;
    };
    // Group g of the grid takes list entry g without an atomic; later items
    // are taken one at a time from a shared cursor that starts after those.
    const int keep_batch = a.keep_batch;
    bool first = true;
    for (int round = 0;; ++round) {
        unsigned int it = group_id;
        if (!first) {
            if (leader && lane == 0) it = n_groups + atomicAdd(&ctl->next[cur], 1u);
        }
        first = false;
        if (G == 1) {
            it = __shfl_sync(0xffffffffu, it, 0);
        } else {
            if (leader && lane == 0) g_it[round & 1][gib] = it;
            group_sync(bar_id, bar_threads);
            it = g_it[round & 1][gib];
        }
        if (it >= n_items) break;
        const unsigned int item = ld_loop<COH>(&a.list[cur][it]);
        // the exact-skip test's inputs (see below) depend only on the
        // item: load them now, alongside the item's descriptor
        bool in_chg = false;
        uint2 iw = make_uint2(0u, 0u);  // lane 0: (transitions, rows) of the item
        if (lane == 0) iw = __ldg(a.item_w + item);
        if (a.skip) {
            const int32_t in = lane < kInItems ? __ldg(a.in_items + (size_t)item * kInItems + lane) : -1;
            in_chg = (lane == 0 && ld_loop<COH>(&a.chg[far][item])) || in == -2 ||
                     (in >= 0 && ld_loop<COH>(&a.chg[far][in]));
        }
        const int4 ch = a.chunks[item];
        const uint4 cu = a.chunk_u[item];  // the item's global state range and its product's first pre-sink state
        const int p = ch.x;
        const size_t pair0 = (size_t)p * KP;
        // activity of the product's weights from the previous sweep's residuals
        unsigned int act_w[2] = {0u, 0u}, nz_w[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < (KP + 31) / 32; ++h) {
            const int k = lane + 32 * h;
            bool act = false, nz = false;
            if (k < KP) {
                const double prev = as_double(ld_loop<COH>(&res_prev[pair0 + k]));
                act = prev > a.thr[pair0 + k];
                nz = prev > 0.0;
            }
            act_w[h] = __ballot_sync(0xffffffffu, act);
            nz_w[h] = __ballot_sync(0xffffffffu, nz);
        }
        const bool any_active = (act_w[0] | act_w[1]) != 0u;
        if ((nz_w[0] | nz_w[1]) == 0u) {  // converged earlier and already copied: drop
            if (ch.w && leader)
                for (int k = lane; k < KP; k += 32) a.frozen[pair0 + k] = 1;
            continue;
        }
        if (any_active && leader) {
            if (lane == n_kept) kept = item;
            if (++n_kept == keep_batch) flush_kept();
        }
        if (ch.w && leader)
            for (int k = lane; k < KP; k += 32) {
                res_next[pair0 + k] = 0ull;
                if ((act_w[k >> 5] >> (k & 31)) & 1u)
                    a.sweeps_pair[pair0 + k] = (int32_t)(sweep + 1);
                else
                    a.frozen[pair0 + k] = 1;
            }
        if (any_active && a.skip) {
            // exact skipping: nothing this item reads changed in the previous
            // sweep, so it would reproduce its values bit for bit (and both
            // value buffers already hold them)
            if (!__any_sync(0xffffffffu, in_chg)) {
                if (leader && lane == 0) {  // no update executed and no byte moved
                    a.chg[cur][item] = 0;
                    ++ps.skipped;
                }
                continue;
            }
        }
        bool changed = false;
        unsigned int act_bits = 0u;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int k = k0 + v;
            act_bits |= ((act_w[k >> 5] >> (k & 31)) & 1u) << v;
        }
        for (int k = lane; k < KP; k += 32) wsm[k] = Ar::weight(a, pair0 + k);
        __syncwarp();
        float rmax[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) rmax[v] = 0.0f;
        // this warp's share of the item's states (global state indices)
        const int span = ((int)(cu.y - cu.x) + G - 1) / G;
        const int s_begin = min((int)cu.y, (int)cu.x + g * span), s_end = min((int)cu.y, s_begin + span);

        if (!any_active) {  // every weight of the product froze: copy its rows once
            for (int s = s_begin + grp; s < s_end; s += SPW) {
                const size_t row = (size_t)(uint32_t)s * ROW + (size_t)k0 * Ar::WORDS;
                float yw[NW];
                load_vals<NW, COH>(Vold + row, yw);
                store_words<NW>(Vnew + row, yw);
            }
        } else if (s_begin < s_end) {
            // a batch's state boundaries are loaded while the previous
            // batch is staged and computed
            uint32_t nx_sa = 0, nx_tr = 0;
            if (lane <= min(kStageStates, s_end - s_begin)) {
                nx_sa = __ldg(a.state_sa + (uint32_t)s_begin + lane);
                nx_tr = __ldg(a.state_tr + (uint32_t)s_begin + lane);
            }
            for (int s0 = s_begin; s0 < s_end;) {
                const int m_max = min(kStageStates, s_end - s0);
                const uint32_t u0 = (uint32_t)s0;
                const uint32_t my_sa = nx_sa, my_tr = nx_tr;
                const uint32_t A0 = __shfl_sync(0xffffffffu, my_sa, 0);
                const uint32_t T0 = __shfl_sync(0xffffffffu, my_tr, 0);
                const bool fits =
                    lane <= m_max && my_sa - A0 <= (uint32_t)Ar::AMAX && my_tr - T0 <= (uint32_t)Ar::EMAX;
                int m = __popc(__ballot_sync(0xffffffffu, fits)) - 1;  // boundaries 0..m fit
                const bool staged = m >= 1;
                if (!staged) m = 1;  // one state too large for the buffer: read it from global memory
                const uint32_t A1 = __shfl_sync(0xffffffffu, my_sa, m);
                const uint32_t T1 = __shfl_sync(0xffffffffu, my_tr, m);
                if (lane <= m) ssa[lane] = my_sa;
                if (s0 + m < s_end && lane <= min(kStageStates, s_end - (s0 + m))) {
                    nx_sa = __ldg(a.state_sa + u0 + (uint32_t)m + lane);
                    nx_tr = __ldg(a.state_tr + u0 + (uint32_t)m + lane);
                }
                typename Ar::View vw;
                // the batch's rows of G (residual correction) are one
                // contiguous range: start it towards L2 before staging
                if constexpr (std::is_same<Ar, ArithDelta>::value && KP % 4 == 0)
                    if (lane == 0 && A1 > A0) prefetch_l2(a.G + (size_t)A0 * KP, (A1 - A0) * (uint32_t)(KP * 4));
                if (staged) {
                    Ar::stage(a, stage_buf, A0, A1 - A0, T0, T1 - T0, lane);
                    cp_async_wait_all();
                    vw = Ar::smem_view(stage_buf);
                } else {
                    vw = Ar::global_view(a, A0, T0);
                }
                __syncwarp();
                for (int i = grp; i < m; i += SPW)
                    if constexpr (PIPE)
                        process_state_pipe<Ar, KP, VMAX, D, COH>(a, vw, ssa, A0, T0, i, u0 + (uint32_t)i,
                                                            u0 + (uint32_t)i >= cu.z, wsm + k0, act_bits, Vold,
                                                            Vnew, k0, rmax, changed);
                    else
                        process_state<Ar, KP, VMAX, D, COH>(a, vw, ssa, A0, T0, i, u0 + (uint32_t)i,
                                                       u0 + (uint32_t)i >= cu.z, wsm + k0, act_bits, Vold, Vnew, k0,
                                                       rmax, changed);
                __syncwarp();  // the next batch reuses the buffer
                s0 += m;
            }
        }
        // residual: lanes with the same li share weights
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            float r = rmax[v];
#pragma unroll
            for (int off = LPS; off < 32; off <<= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, off));
            rmax[v] = r;
        }
        bool any_chg = __any_sync(0xffffffffu, changed);
        if (G > 1) {  // combine the group's warps in shared memory
            if (grp == 0)
#pragma unroll
                for (int v = 0; v < VEC; ++v) g_res[wib][k0 + v] = rmax[v];
            if (lane == 0) g_chg[wib] = any_chg ? 1 : 0;
            group_sync(bar_id, bar_threads);
            if (leader) {
                for (int q = 1; q < G; ++q) {
                    any_chg = any_chg || g_chg[wib + q] != 0;
#pragma unroll
                    for (int v = 0; v < VEC; ++v) rmax[v] = fmaxf(rmax[v], g_res[wib + q][k0 + v]);
                }
            }
        }
        if (leader) {
            if (lane == 0) a.chg[cur][item] = any_chg ? 1 : 0;
#pragma unroll
            for (int v = 0; v < VEC; ++v)
                if (grp == 0 && any_active && rmax[v] > 0.0f) atomic_max_nonneg(res_cur + pair0 + k0 + v, (double)rmax[v]);
            if (lane == 0) {
                const uint32_t n_s = cu.y - cu.x;
                ps.bytes += 2ull * n_s * ROW * 4;
                if (any_active) {
                    const int n_act = __popc(act_w[0]) + __popc(act_w[1]);
                    ++ps.computed;
                    ps.updates += (unsigned long long)iw.x * (unsigned long long)n_act;
                    // state_sa + state_tr, sa_tr, cost and (col, p) per transition, 4 bytes per word
                    ps.bytes += 8ull * (n_s + 1) + 4ull * (iw.y + 1) + 4ull * (1 + Ar::WORDS) * iw.x;
                    // per row: its cost, or for the residual correction its row of G
                    ps.bytes += (std::is_same<Ar, ArithDelta>::value ? 4ull * KP : 4ull * Ar::WORDS) * iw.y;
                }
            }
        }
    }
    if (leader && n_kept) flush_kept();
}

// A launch's statistics: per block in shared memory, then one global atomic each.
__device__ __forceinline__ void flush_stats(LoopCtl *ctl, const PassStats &ps) {
    __shared__ PassStats b;
    if (threadIdx.x == 0) b = PassStats{0ull, 0ull, 0u, 0u};
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        if (ps.updates) atomicAdd(&b.updates, ps.updates);
        if (ps.bytes) atomicAdd(&b.bytes, ps.bytes);
        if (ps.skipped) atomicAdd(&b.skipped, ps.skipped);
        if (ps.computed) atomicAdd(&b.computed, ps.computed);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (b.updates) atomicAdd(&ctl->updates, b.updates);
        if (b.bytes) atomicAdd(&ctl->bytes, b.bytes);
        if (b.skipped) atomicAdd(&ctl->skipped, b.skipped);
        if (b.computed) atomicAdd(&ctl->computed, b.computed);
    }
}

// One sweep per launch: the loop's graph (or the host) launches it six times
// per body, then the control kernel.
template <class Ar, int KP, int VMAX, int D, int MINB, int PIPE>
__global__ void __launch_bounds__(kThreads, MINB) k_sweep(SweepArgs a, int pos) {
    PassStats ps = {0ull, 0ull, 0u, 0u};
    sweep_pass<Ar, KP, VMAX, D, PIPE, false>(a, pos, a.ctl->sweep_base + pos, ps);
    flush_stats(a.ctl, ps);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier of all blocks of a cooperative launch (every block is resident):
// a block arrives by one atomic on ctl->bar and waits until all gridDim.x
// arrivals of this round are in.  The wait is bounded: after kBarrierNs of
// wall-clock time (or kBarrierSpins polls), or once another block has given
// up (ctl->bar_err), the block sets ctl->bar_err and the call returns false;
// the kernel then ends and the host reports the error.
constexpr unsigned long long kBarrierNs = 1000000000ull;  // 1 s
constexpr unsigned int kBarrierSpins = 1u << 24;
__device__ __forceinline__ bool grid_barrier(LoopCtl *ctl, unsigned int &target) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        __threadfence();  // this block's writes of the sweep before its arrival
        atomicAdd(&ctl->bar, 1u);
        int ok = 1;
        const unsigned long long t0 = global_ns();
        for (unsigned int n = 0; ld_acquire_gpu(&ctl->bar) < target; ++n) {
            if ((n & 31u) == 31u &&
                (ld_acquire_gpu(&ctl->bar_err) != 0u || n >= kBarrierSpins || global_ns() - t0 > kBarrierNs)) {
                atomicExch(&ctl->bar_err, 1u);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Self-check of grid_barrier's bounded wait: the last block never arrives,
// so every other block's wait runs out and the kernel ends on its own with
// ctl->bar_err set.
__global__ void k_barrier_selfcheck(LoopCtl *ctl) {
    if (blockIdx.x == gridDim.x - 1) return;
    unsigned int target = 0u;
    grid_barrier(ctl, target);
}

// The rest of a loop in one cooperative launch (the loop's "tail": its work
// list has fallen to ctl->tail items or fewer, at most one per warp of the
// launch).  Sweep n of the launch is the loop's sweep sweep_base + n; a grid
// barrier separates consecutive sweeps.  An item only ever leaves the work
// list, so the launch deals the items of its first list to warp groups once
// (group g keeps entry g): a group keeps its item's descriptor, weights and,
// when a warp's share of the item fits one staged batch, that batch in
// shared memory, and rereads per sweep only what the sweep decides on
// (residuals, change flags) and the values it gathers (from L2: other
// blocks wrote them in the previous sweep).  Each state is computed as in
// sweep_pass, and the item set of each sweep is the one the launch-per-sweep
// loop would have, so the results are bit for bit the same.  The launch ends
// when the work list is empty (the sweep count rounded up to a body of six,
// as the launch-per-sweep loop counts it) or at the cap.
template <class Ar, int KP, int VMAX, int D, int MINB, int PIPE>
__global__ void __launch_bounds__(kThreads, MINB) k_sweep_tail(SweepArgs a) {
    using SH = Shape<Ar, KP, VMAX>;
    constexpr int VEC = SH::VEC, LPS = SH::LPS, SPW = SH::SPW;
    constexpr int NW = VEC * Ar::WORDS;
    constexpr int ROW = KP * Ar::WORDS;
    constexpr int WPB = kThreads / 32;
    constexpr int GMAX = (kChunk / SPW) < WPB ? (kChunk / SPW) : WPB;
    constexpr unsigned int NONE = 0xFFFFFFFFu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned char g_chg[WPB];
    __shared__ float g_res[WPB][KP];
    LoopCtl *ctl = a.ctl;
    // sweep_base is rewritten below only by block 0, after a barrier that
    // every block reaches after this read, or with the value read here
    const unsigned int base = ctl->sweep_base, cap = ctl->cap;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / LPS, li = lane % LPS, k0 = li * VEC;
    unsigned char *stage_buf = smem_raw + wib * (Ar::STAGE_BYTES + KP * (int)sizeof(typename Ar::W));
    uint32_t *ssa = reinterpret_cast<uint32_t *>(stage_buf);
    typename Ar::W *wsm = reinterpret_cast<typename Ar::W *>(stage_buf + Ar::STAGE_BYTES);

    // warp groups, fixed for the launch from its first list (sweep position 0)
    const unsigned int n0 = ld_loop<true>(&ctl->cnt[0]);
    const unsigned int n_warps = gridDim.x * WPB;
    int G = 1;
    const int gcap = a.gmax < GMAX ? a.gmax : GMAX;
    while (G < gcap && (unsigned long long)(2 * G) * n0 <= n_warps) G *= 2;
    const int gib = wib / G, g = wib % G;
    const bool leader = g == 0;
    const int bar_id = 1 + gib, bar_threads = 32 * G;
    const unsigned int n_groups = n_warps / G;
    if (n0 > n_groups) {  // more items than groups: the host sizes the tail so that this cannot be
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&ctl->bar_err, 1u);
        return;
    }
    const unsigned int group_id = blockIdx.x * (WPB / G) + gib;

    // the group's item and what the launch keeps of it
    unsigned int item = group_id < n0 ? ld_loop<true>(&a.list[0][group_id]) : NONE;
    int4 ch = make_int4(0, 0, 0, 0);
    uint4 cu = make_uint4(0u, 0u, 0u, 0u);
    uint2 iw = make_uint2(0u, 0u);  // lane 0: (transitions, rows) of the item
    int32_t in = -1;                // lanes < kInItems: an input item of the item
    size_t pair0 = 0;
    double thr_w[2] = {0.0, 0.0};   // freeze thresholds of weights lane and lane + 32
    int s_begin = 0, s_end = 0;     // this warp's share of the item's states
    if (item != NONE) {
        ch = a.chunks[item];
        cu = a.chunk_u[item];
        if (lane == 0) iw = __ldg(a.item_w + item);
        if (a.skip && lane < kInItems) in = __ldg(a.in_items + (size_t)item * kInItems + lane);
        pair0 = (size_t)ch.x * KP;
#pragma unroll
        for (int h = 0; h < (KP + 31) / 32; ++h)
            if (lane + 32 * h < KP) thr_w[h] = a.thr[pair0 + lane + 32 * h];
        const int span = ((int)(cu.y - cu.x) + G - 1) / G;
        s_begin = min((int)cu.y, (int)cu.x + g * span);
        s_end = min((int)cu.y, s_begin + span);
    }
    bool have_w = false;  // the item's weights are in wsm
    bool kept_batch = false;  // the warp's whole share is the batch staged in its buffer
    uint32_t kA0 = 0u, kT0 = 0u;
    int km = 0;

    PassStats ps = {0ull, 0ull, 0u, 0u};
    unsigned int target = 0u, n = 0u;
    for (;; ++n) {
        if (ld_loop<true>(&ctl->cnt[n % 3]) == 0u) {
            n = (n + 5u) / 6u * 6u;
            break;
        }
        if (n % 6u == 0u && base + n >= cap) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->hit_cap = 1;
            break;
        }
        const int pos = (int)(n % 6u);
        const int cur = pos % 3, nxt = (pos + 1) % 3, far = (pos + 2) % 3;
        const float *__restrict__ Vold = static_cast<const float *>(a.V[pos & 1]);
        float *__restrict__ Vnew = static_cast<float *>(a.V[(pos + 1) & 1]);
        const unsigned long long *res_prev = a.res[far];
        unsigned long long *res_cur = a.res[cur];
        unsigned long long *res_next = a.res[nxt];
        const unsigned int sweep = base + n;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctl->cnt[far] = 0;
            ctl->next[far] = 0;
        }
        if (item != NONE) {
            bool in_chg = false;
            if (a.skip)
                in_chg = (lane == 0 && ld_loop<true>(&a.chg[far][item])) || in == -2 ||
                         (in >= 0 && ld_loop<true>(&a.chg[far][in]));
            unsigned int act_w[2] = {0u, 0u}, nz_w[2] = {0u, 0u};
#pragma unroll
            for (int h = 0; h < (KP + 31) / 32; ++h) {
                const int k = lane + 32 * h;
                bool act = false, nz = false;
                if (k < KP) {
                    const double prev = as_double(ld_loop<true>(&res_prev[pair0 + k]));
                    act = prev > thr_w[h];
                    nz = prev > 0.0;
                }
                act_w[h] = __ballot_sync(0xffffffffu, act);
                nz_w[h] = __ballot_sync(0xffffffffu, nz);
            }
            const bool any_active = (act_w[0] | act_w[1]) != 0u;
            if ((nz_w[0] | nz_w[1]) == 0u) {  // converged earlier and already copied: the item leaves
                if (ch.w && leader)
                    for (int k = lane; k < KP; k += 32) a.frozen[pair0 + k] = 1;
                item = NONE;
            } else {
                if (any_active && leader && lane == 0) atomicAdd(&ctl->cnt[nxt], 1u);  // stays in the list
                if (ch.w && leader)
                    for (int k = lane; k < KP; k += 32) {
                        res_next[pair0 + k] = 0ull;
                        if ((act_w[k >> 5] >> (k & 31)) & 1u)
                            a.sweeps_pair[pair0 + k] = (int32_t)(sweep + 1);
                        else
                            a.frozen[pair0 + k] = 1;
                    }
                const bool skipped = any_active && a.skip && !__any_sync(0xffffffffu, in_chg);
                if (skipped) {  // exact skipping, as in sweep_pass
                    if (leader && lane == 0) {
                        a.chg[cur][item] = 0;
                        ++ps.skipped;
                    }
                } else {
                    bool changed = false;
                    unsigned int act_bits = 0u;
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        const int k = k0 + v;
                        act_bits |= ((act_w[k >> 5] >> (k & 31)) & 1u) << v;
                    }
                    if (!have_w) {
                        for (int k = lane; k < KP; k += 32) wsm[k] = Ar::weight(a, pair0 + k);
                        __syncwarp();
                        have_w = true;
                    }
                    float rmax[VEC];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) rmax[v] = 0.0f;
                    if (!any_active) {  // every weight of the product froze: copy its rows once
                        for (int s = s_begin + grp; s < s_end; s += SPW) {
                            const size_t row = (size_t)(uint32_t)s * ROW + (size_t)k0 * Ar::WORDS;
                            float yw[NW];
                            load_vals<NW, true>(Vold + row, yw);
                            store_words<NW>(Vnew + row, yw);
                        }
                    } else if (kept_batch) {
                        const typename Ar::View vw = Ar::smem_view(stage_buf);
                        const uint32_t u0 = (uint32_t)s_begin;
                        for (int i = grp; i < km; i += SPW)
                            if constexpr (PIPE)
                                process_state_pipe<Ar, KP, VMAX, D, true>(a, vw, ssa, kA0, kT0, i, u0 + (uint32_t)i,
                                                                          u0 + (uint32_t)i >= cu.z, wsm + k0, act_bits,
                                                                          Vold, Vnew, k0, rmax, changed);
                            else
                                process_state<Ar, KP, VMAX, D, true>(a, vw, ssa, kA0, kT0, i, u0 + (uint32_t)i,
                                                                     u0 + (uint32_t)i >= cu.z, wsm + k0, act_bits,
                                                                     Vold, Vnew, k0, rmax, changed);
                        __syncwarp();
                    } else if (s_begin < s_end) {
                        uint32_t nx_sa = 0, nx_tr = 0;
                        if (lane <= min(kStageStates, s_end - s_begin)) {
                            nx_sa = __ldg(a.state_sa + (uint32_t)s_begin + lane);
                            nx_tr = __ldg(a.state_tr + (uint32_t)s_begin + lane);
                        }
                        for (int s0 = s_begin; s0 < s_end;) {
                            const int m_max = min(kStageStates, s_end - s0);
                            const uint32_t u0 = (uint32_t)s0;
                            const uint32_t my_sa = nx_sa, my_tr = nx_tr;
                            const uint32_t A0 = __shfl_sync(0xffffffffu, my_sa, 0);
                            const uint32_t T0 = __shfl_sync(0xffffffffu, my_tr, 0);
                            const bool fits = lane <= m_max && my_sa - A0 <= (uint32_t)Ar::AMAX &&
                                              my_tr - T0 <= (uint32_t)Ar::EMAX;
                            int m = __popc(__ballot_sync(0xffffffffu, fits)) - 1;
                            const bool staged = m >= 1;
                            if (!staged) m = 1;
                            const uint32_t A1 = __shfl_sync(0xffffffffu, my_sa, m);
                            const uint32_t T1 = __shfl_sync(0xffffffffu, my_tr, m);
                            if (lane <= m) ssa[lane] = my_sa;
                            if (s0 + m < s_end && lane <= min(kStageStates, s_end - (s0 + m))) {
                                nx_sa = __ldg(a.state_sa + u0 + (uint32_t)m + lane);
                                nx_tr = __ldg(a.state_tr + u0 + (uint32_t)m + lane);
                            }
                            typename Ar::View vw;
                            if (staged) {
                                Ar::stage(a, stage_buf, A0, A1 - A0, T0, T1 - T0, lane);
                                cp_async_wait_all();
                                vw = Ar::smem_view(stage_buf);
                            } else {
                                vw = Ar::global_view(a, A0, T0);
                            }
                            __syncwarp();
                            for (int i = grp; i < m; i += SPW)
                                if constexpr (PIPE)
                                    process_state_pipe<Ar, KP, VMAX, D, true>(a, vw, ssa, A0, T0, i, u0 + (uint32_t)i,
                                                                              u0 + (uint32_t)i >= cu.z, wsm + k0,
                                                                              act_bits, Vold, Vnew, k0, rmax, changed);
                                else
                                    process_state<Ar, KP, VMAX, D, true>(a, vw, ssa, A0, T0, i, u0 + (uint32_t)i,
                                                                         u0 + (uint32_t)i >= cu.z, wsm + k0, act_bits,
                                                                         Vold, Vnew, k0, rmax, changed);
                            __syncwarp();
                            if (staged && s0 == s_begin && m == s_end - s_begin) {  // the whole share: keep it
                                kept_batch = true;
                                kA0 = A0;
                                kT0 = T0;
                                km = m;
                            }
                            s0 += m;
                        }
                    }
                    // residual: lanes with the same li share weights
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        float r = rmax[v];
#pragma unroll
                        for (int off = LPS; off < 32; off <<= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, off));
                        rmax[v] = r;
                    }
                    bool any_chg = __any_sync(0xffffffffu, changed);
                    if (G > 1) {
                        if (grp == 0)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) g_res[wib][k0 + v] = rmax[v];
                        if (lane == 0) g_chg[wib] = any_chg ? 1 : 0;
                        group_sync(bar_id, bar_threads);
                        if (leader) {
                            for (int q = 1; q < G; ++q) {
                                any_chg = any_chg || g_chg[wib + q] != 0;
#pragma unroll
                                for (int v = 0; v < VEC; ++v) rmax[v] = fmaxf(rmax[v], g_res[wib + q][k0 + v]);
                            }
                        }
                    }
                    if (leader) {
                        if (lane == 0) a.chg[cur][item] = any_chg ? 1 : 0;
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            if (grp == 0 && any_active && rmax[v] > 0.0f)
                                atomic_max_nonneg(res_cur + pair0 + k0 + v, (double)rmax[v]);
                        if (lane == 0) {
                            const uint32_t n_s = cu.y - cu.x;
                            ps.bytes += 2ull * n_s * ROW * 4;
                            if (any_active) {
                                const int n_act = __popc(act_w[0]) + __popc(act_w[1]);
                                ++ps.computed;
                                ps.updates += (unsigned long long)iw.x * (unsigned long long)n_act;
                                ps.bytes += 8ull * (n_s + 1) + 4ull * (iw.y + 1) + 4ull * (1 + Ar::WORDS) * iw.x;
                                ps.bytes +=
                                    (std::is_same<Ar, ArithDelta>::value ? 4ull * KP : 4ull * Ar::WORDS) * iw.y;
                            }
                        }
                    }
                }
                if (!any_active) item = NONE;  // copied once; not in the next list
            }
        }
        if (!grid_barrier(ctl, target)) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->sweep_base = base + n;
        ctl->tail_sweeps = n;
    }
    flush_stats(ctl, ps);
}

// -------------------------------------------------------------- finalise
// The returned scheduler: keep the recorded action when its Q-value on the
// final FP64 values is within tau of the maximum (the state is "anchored");
// otherwise, provisionally, the lowest-index action within tau of the
// maximum that is not a self-loop (a zero-reward self-loop ties with the
// maximum at any fixed point), and only if every such action is a self-loop
// the lowest-index one.  a_rec is consumed: it becomes the anchoring flag
// (1 anchored, 0 undecided), and the undecided (state, weight) entries are
// counted in ctl->undecided for the anchoring rounds (k_anchor).
template <int KP>
__global__ void __launch_bounds__(kThreads) k_finalize(SweepArgs a, int n_chunks, double tau, uint8_t *policy) {
    constexpr int VEC = KP < 2 ? KP : 2, LPS = KP / VEC, SPR = kThreads / LPS;
    const float2 *__restrict__ V = static_cast<const float2 *>(a.V[0]);  // double-float values
    const int k0 = (threadIdx.x % LPS) * VEC, slot = threadIdx.x / LPS;
    const float ftau = (float)tau;
    for (int item = blockIdx.x; item < n_chunks; item += gridDim.x) {
        const int4 ch = a.chunks[item];
        const int p = ch.x;
        const ProdDesc pd = a.prods[p];
        ArithDF::W w[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) w[v] = a.wdf[(size_t)p * KP + k0 + v];
        for (int s = ch.y + slot; s < ch.z; s += SPR) {
            const uint32_t u = pd.state_off + (uint32_t)s;
            const size_t row = (size_t)u * KP + k0;
            const uint32_t a0 = a.state_sa[u], a1 = a.state_sa[u + 1];
            // Q without the state's pre-sink weight, which is the same for
            // every action and cancels in every comparison below
            DF best[VEC], qrec[VEC];
            uint8_t rec[VEC], pick[VEC], pick_loop[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                best[v] = ArithDF::neg_inf();
                rec[v] = a.a_rec[row + v];
                qrec[v] = ArithDF::neg_inf();
                pick[v] = 0xFF;
                pick_loop[v] = 0xFF;
            }
            // Q within tau of the maximum, on the double-float values
            auto near_max = [&](const DF &q, const DF &m) {
                return __fadd_rn(__fadd_rn(q.h, -m.h), __fadd_rn(q.l, -m.l)) >= -ftau;
            };
            for (int pass = 0; pass < 2; ++pass) {
                for (uint32_t sa = a0; sa < a1; ++sa) {
                    const float2 cd = a.costdf[sa];
                    DF acc[VEC];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[v] = ArithDF::reward(w[v], {cd.x, cd.y});
                    const uint32_t t0 = a.sa_tr[sa], t1 = a.sa_tr[sa + 1];
                    const bool self_loop = (t1 - t0 == 1) && ((uint32_t)a.col[t0] == u);
                    for (uint32_t t = t0; t < t1; ++t) {
                        const int32_t cl = a.col[t];
                        const float2 pr = a.pdf[t];
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            const float2 xv = V[(size_t)cl * KP + k0 + v];
                            ArithDF::mac(acc[v], {pr.x, pr.y}, {xv.x, xv.y});
                        }
                    }
                    const uint8_t la = (uint8_t)(sa - a0);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        acc[v] = df_norm(acc[v]);
                        if (pass == 0) {
                            best[v] = df_gt(acc[v], best[v]) ? acc[v] : best[v];
                            if (la == rec[v]) qrec[v] = acc[v];
                        } else if (near_max(acc[v], best[v])) {
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
                for (int v = 0; v < VEC; ++v) all_kept = all_kept && near_max(qrec[v], best[v]);
                if (all_kept) break;  // the second pass is only needed for a fallback
            }
            unsigned int undecided = 0;
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                const bool kept = near_max(qrec[v], best[v]);
                policy[row + v] = kept ? rec[v] : (pick[v] != 0xFF ? pick[v] : pick_loop[v]);
                a.a_rec[row + v] = kept ? 1 : 0;
                undecided += kept ? 0u : 1u;
            }
            if (undecided) atomicAdd(&a.ctl->undecided, undecided);
        }
    }
}

// One anchoring round of the returned scheduler.  With a zero weight on the
// cost every move is free, so in a region of equal values "go to the
// neighbour" ties with the maximum and two undecided neighbours could send
// the run between them forever.  An undecided (state, weight) therefore
// takes the lowest-index action within tau of the maximum that is not a
// self-loop and reaches, with positive probability, another state anchored
// before this round: flag 1, or decided in an earlier round r' (flag
// r' + 1); the done slot is always anchored.  Decided entries get flag
// round + 1, which this round's readers treat as not yet anchored, so the
// result does not depend on the order in which threads run.  Each decided
// state reaches an anchor with positive probability through states of
// lower rounds, so the scheduler reaches the kept recorded actions (or the
// done slot) with probability one.  One thread per (state, weight).
template <int KP>
__global__ void __launch_bounds__(kThreads) k_anchor(SweepArgs a, int n_chunks, double tau, uint8_t *policy,
                                                      int round) {
    constexpr int SPR = kThreads / KP;
    const float2 *__restrict__ V = static_cast<const float2 *>(a.V[0]);  // double-float values
    const int k = threadIdx.x % KP, slot = threadIdx.x / KP;
    const float ftau = (float)tau;
    unsigned int decided = 0;
    for (int item = blockIdx.x; item < n_chunks; item += gridDim.x) {
        const int4 ch = a.chunks[item];
        const ProdDesc pd = a.prods[ch.x];
        const uint32_t done_slot = pd.state_off + pd.n_nd;
        const ArithDF::W w = a.wdf[(size_t)ch.x * KP + k];
        for (int s = ch.y + slot; s < ch.z; s += SPR) {
            const uint32_t u = pd.state_off + (uint32_t)s;
            const size_t row = (size_t)u * KP + k;
            if (a.a_rec[row] != 0) continue;
            const uint32_t a0 = a.state_sa[u], a1 = a.state_sa[u + 1];
            auto q_of = [&](uint32_t sa) {
                const float2 cd = a.costdf[sa];
                DF acc = ArithDF::reward(w, {cd.x, cd.y});
                for (uint32_t t = a.sa_tr[sa]; t < a.sa_tr[sa + 1]; ++t) {
                    const float2 pr = a.pdf[t];
                    const float2 xv = V[(size_t)a.col[t] * KP + k];
                    ArithDF::mac(acc, {pr.x, pr.y}, {xv.x, xv.y});
                }
                return df_norm(acc);
            };
            DF best = ArithDF::neg_inf();
            for (uint32_t sa = a0; sa < a1; ++sa) {
                const DF q = q_of(sa);
                best = df_gt(q, best) ? q : best;
            }
            for (uint32_t sa = a0; sa < a1; ++sa) {
                const uint32_t t0 = a.sa_tr[sa], t1 = a.sa_tr[sa + 1];
                if (t1 - t0 == 1 && (uint32_t)a.col[t0] == u) continue;  // self-loop
                const DF q = q_of(sa);
                if (!(__fadd_rn(__fadd_rn(q.h, -best.h), __fadd_rn(q.l, -best.l)) >= -ftau)) continue;
                bool hit = false;
                for (uint32_t t = t0; t < t1 && !hit; ++t) {
                    const uint32_t v = (uint32_t)a.col[t];
                    if (!(a.pdf[t].x > 0.0f) || v == u) continue;
                    const int f = v == done_slot ? 1 : (int)a.a_rec[(size_t)v * KP + k];
                    hit = f >= 1 && f <= round;
                }
                if (hit) {
                    policy[row] = (uint8_t)(sa - a0);
                    a.a_rec[row] = (uint8_t)(round + 1);
                    ++decided;
                    break;
                }
            }
        }
    }
    if (decided) atomicAdd(&a.ctl->decided, decided);
}

// ------------------------------------------------------------- evaluation
// Algorithm 4 for both objectives of a pair at once: E[u] = (cost, prob)
// with y = (-cost(u, mu(u)), pre(u)) + sum p E[u'].  The scheduler's rows
// are first gathered into a compact structure-of-arrays layout with a fixed
// number of slots per state, so a sweep reads independent coalesced words
// instead of chasing scheduler -> state -> row -> transition pointers.
__global__ void __launch_bounds__(kThreads) k_eval_compact(EvalArgs a, int n_chunks) {
    for (int item = blockIdx.x; item < n_chunks; item += gridDim.x) {
        const int4 ch = a.chunks[item];
        const int4 pr = a.pairs[ch.x];
        const ProdDesc pd = a.prods[pr.x];
        const uint32_t n1 = pd.n_nd + 1;
        const size_t off = (size_t)pr.z;
        const int s = ch.y + threadIdx.x;
        if (s >= ch.z) continue;
        const uint32_t u = pd.state_off + (uint32_t)s;
        const uint32_t sa = a.state_sa[u] + a.policy[(size_t)u * a.Kp + pr.y];
        const uint32_t t0 = a.sa_tr[sa], t1 = a.sa_tr[sa + 1];
        atomicAdd(&a.item_tmu[item], t1 - t0);  // the scheduler's transitions, for the statistics
        atomicAdd(&a.pair_tmu[ch.x], t1 - t0);
        a.ecost[off + s] = a.costdf[sa];
        for (int j = 0; j < a.stride; ++j) {
            const size_t at = off * a.stride + (size_t)j * n1 + s;
            if (t0 + j < t1) {
                a.ecol[at] = a.col[t0 + j] - (int32_t)pd.state_off;
                a.ep[at] = a.pdf[t0 + j];
            } else {
                a.ecol[at] = (int32_t)pd.n_nd;
                a.ep[at] = make_float2(0.0f, 0.0f);
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_eval_sweep(EvalArgs a, int pos) {
    const int cur = pos % 3, nxt = (pos + 1) % 3, far = (pos + 2) % 3;
    const float4 *__restrict__ Eold = a.E[pos & 1];
    float4 *__restrict__ Enew = a.E[(pos + 1) & 1];
    LoopCtl *ctl = a.ctl;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->cnt[far] = 0;
        ctl->next[far] = 0;
    }
    const unsigned int n_items = ctl->cnt[cur];
    const unsigned int sweep = ctl->sweep_base + pos;
    __shared__ unsigned int s_item;
    __shared__ float s_red[kThreads / 32];
    const int stride = a.stride;
    // Moves below this fraction of a value are double-float rounding, not
    // propagation: each of the stride + 1 accumulations adds at most a few
    // units of 2^-48 relative error, so they are not counted as residual.
    const float noise = (float)(stride + 1) * 2.8421709430404007e-14f; /* 2^-45 */
    // Few atomics on the shared counters: block b takes list entry b first
    // and later ones from a cursor that starts after gridDim.x; items that
    // stay in the list are appended up to 32 at a time; the statistics are
    // summed per block (thread 0's registers).
    __shared__ unsigned int s_kept[32];
    __shared__ int s_n_kept;
    if (threadIdx.x == 0) s_n_kept = 0;
    auto flush_kept = [&]() {  // thread 0
        const unsigned int at = atomicAdd(&ctl->cnt[nxt], (unsigned int)s_n_kept);
        for (int q = 0; q < s_n_kept; ++q) a.list[nxt][at + q] = s_kept[q];
        s_n_kept = 0;
    };
    unsigned long long b_updates = 0, b_bytes = 0;
    bool first = true;
    for (;;) {
        if (threadIdx.x == 0) s_item = first ? blockIdx.x : gridDim.x + atomicAdd(&ctl->next[cur], 1u);
        first = false;
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
            s_kept[s_n_kept++] = item;
            if (s_n_kept == 32) flush_kept();
        }
        if (ch.w && threadIdx.x == 0) {
            a.res[nxt][e] = 0ull;
            if (active)
                a.sweeps_pair[e] = (int32_t)(sweep + 1);
            else
                a.frozen[e] = 1;
        }
        float r = 0.0f;
        const int s = ch.y + threadIdx.x;
        const size_t off = (size_t)pr.z;
        const uint32_t n1 = pd.n_nd + 1;
        if (s < ch.z) {
            const float4 x = Eold[off + s];
            float4 y = x;
            if (active) {
                const float2 cc = a.ecost[off + s];
                DF yc = {-cc.x, -cc.y};
                DF yp = {((uint32_t)s >= pd.pre_begin) ? 1.0f : 0.0f, 0.0f};
                const size_t base = off * stride + s;
                int j = 0;
                for (; j + 4 <= stride; j += 4) {
                    int32_t c[4];
                    float2 p[4];
                    float4 v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        c[q] = a.ecol[base + (size_t)(j + q) * n1];
                        p[q] = a.ep[base + (size_t)(j + q) * n1];
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] = Eold[off + c[q]];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        ArithDF::mac(yc, {p[q].x, p[q].y}, {v[q].x, v[q].y});
                        ArithDF::mac(yp, {p[q].x, p[q].y}, {v[q].z, v[q].w});
                    }
                }
                for (; j < stride; ++j) {
                    const int32_t c = a.ecol[base + (size_t)j * n1];
                    const float2 p = a.ep[base + (size_t)j * n1];
                    const float4 v = Eold[off + c];
                    ArithDF::mac(yc, {p.x, p.y}, {v.x, v.y});
                    ArithDF::mac(yp, {p.x, p.y}, {v.z, v.w});
                }
                yc = df_norm(yc);
                yp = df_norm(yp);
                y = make_float4(yc.h, yc.l, yp.h, yp.l);
                float dc = ArithDF::diff(yc, {x.x, x.y}), dp = ArithDF::diff(yp, {x.z, x.w});
                dc = dc > noise * fabsf(yc.h) ? dc : 0.0f;
                dp = dp > noise * fabsf(yp.h) ? dp : 0.0f;
                r = fmaxf(dc, dp);
            }
            Enew[off + s] = y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x / 32] = r;
        __syncthreads();
        if (threadIdx.x == 0) {
            float mx = 0.0f;
            for (int wi = 0; wi < kThreads / 32; ++wi) mx = fmaxf(mx, s_red[wi]);
            if (active && mx > 0.0f) atomic_max_nonneg(a.res[cur] + e, (double)mx);
            const unsigned long long n_s = (unsigned long long)(ch.z - ch.y);
            // values read + written (16 B each); when computing also the cost
            // (8) and the successor and probability (4 + 8) of each of the
            // scheduler's transitions (padding slots are not algorithmic);
            // updates: one term per transition and objective
            b_bytes += n_s * 32ull;
            if (active) {
                const unsigned long long tm = a.item_tmu[item];
                b_bytes += n_s * 8ull + 12ull * tm;
                b_updates += tm * 2ull;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (s_n_kept) flush_kept();
        if (b_updates) atomicAdd(&ctl->updates, b_updates);
        if (b_bytes) atomicAdd(&ctl->bytes, b_bytes);
    }
}

// Algorithm 4 for one pair per block, every sweep inside one launch, as an
// FP32 iteration followed by an FP32 residual correction on a double-float
// table (the same scheme as the optimisation's polish, for a fixed
// scheduler, where it is exact algebra: E = B + d with d = G + P d):
//   A. E <- r + P E from 0 in FP32 (round to nearest) until, for both
//      objectives, the sweep's largest move is at most 2^-18 of its largest
//      value; B = the result;
//   B. G = r + P B - B per state in double-float, rounded to FP32;
//   C. d <- G + P d from 0 in FP32 until the sweep's largest move is at most
//      thr (moves below (slots + 1) * 2^-23 |y| are FP32 rounding noise and
//      count as 0, the analogue of k_eval_sweep's double-float floor);
//   D. E = B + d, exactly, as a double-float pair.
// The values live in shared memory (four float2 arrays: A's two buffers,
// of which the unused one holds G, and C's two), one block barrier
// separates sweeps.  A sweep costs two FP32 multiply-adds per slot instead
// of two double-float ones; the result agrees with the double-float loop
// to ~1e-9 (FP32 carries d, which is ~2^-18 of the values, to ~2^-24 of
// itself per sweep).  The final values go to E[0], where the gather reads
// them.  MS > 0: rows of at most MS slots, U states per thread loaded
// together so that their loads overlap; MS = 0: any row length.
template <int MS, int U>
__global__ void __launch_bounds__(kEvalBlockThreads, 1) k_eval_block(EvalArgs a, const int *bpairs, unsigned int cap) {
    constexpr int NWARP = kEvalBlockThreads / 32;
    extern __shared__ __align__(16) float2 sX[];
    __shared__ float s_red[2][4][NWARP];
    const int e = bpairs[blockIdx.x];
    const int4 pr = a.pairs[e];
    const ProdDesc pd = a.prods[pr.x];
    const uint32_t n = pd.n_nd, n1 = n + 1;
    const size_t off = (size_t)pr.z;
    const int stride = a.stride;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // X(q): phase A's buffers (q = 0, 1); D(q): phase C's
    auto X = [&](unsigned int q) { return sX + (q & 1u) * n1; };
    auto D = [&](unsigned int q) { return sX + (2u + (q & 1u)) * n1; };
    for (uint32_t s = threadIdx.x; s < 4 * n1; s += kEvalBlockThreads) sX[s] = make_float2(0.f, 0.f);
    __syncthreads();
    const float noise = (float)(stride + 1) * 1.1920928955078125e-07f; /* 2^-23 */
    const float thr_f = __double2float_rd(a.thr);  // float r > thr_f exactly when (double)r > thr
    // block-wide maxima of up to four quantities; every warp reduces the
    // per-warp values itself, so one barrier per sweep suffices
    // (the correction stage's test reads only the two moves: NQ = 2 there)
    auto block_max = [&](float (&v)[4], int parity, auto nq) {
        constexpr int NQ = decltype(nq)::value;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[q] = fmaxf(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
            if (lane == 0) s_red[parity][q][warp] = v[q];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float m = lane < NWARP ? s_red[parity][q][lane] : 0.0f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            v[q] = m;
        }
    };
    // One FP32 sweep over the block's states: y = base(s) + sum_j p_j x(c_j)
    // with base = (-cost, pre) (phase A, Gt == nullptr) or G(s) (phase C);
    // m[0..1] = largest move per objective (phase C: beyond the noise
    // floor), m[2..3] = largest |y| per objective.
    auto sweep = [&](const float2 *Xo, float2 *Xn, const float2 *Gt, float (&m)[4]) {
        m[0] = m[1] = m[2] = m[3] = 0.0f;
        constexpr int MSX = MS > 0 ? MS : 1;
        auto one = [&](uint32_t s, float2 base, const int32_t (&c)[MSX], const float2 (&p)[MSX]) {
            float yc = base.x, yp = base.y;
#pragma unroll
            for (int j = 0; j < MSX; ++j) {
                if (j >= stride) break;
                const float2 v = Xo[c[j]];
                yc = __fmaf_rn(p[j].x, v.x, yc);
                yp = __fmaf_rn(p[j].x, v.y, yp);
            }
            const float2 x = Xo[s];
            Xn[s] = make_float2(yc, yp);
            float dc = fabsf(yc - x.x), dp = fabsf(yp - x.y);
            if (Gt) {
                dc = dc > noise * fabsf(yc) ? dc : 0.0f;
                dp = dp > noise * fabsf(yp) ? dp : 0.0f;
            }
            m[0] = fmaxf(m[0], dc);
            m[1] = fmaxf(m[1], dp);
            m[2] = fmaxf(m[2], fabsf(yc));
            m[3] = fmaxf(m[3], fabsf(yp));
        };
        if constexpr (MS > 0) {
            for (uint32_t s0 = threadIdx.x; s0 < n; s0 += U * kEvalBlockThreads) {
                float2 base[U];
                int32_t c[U][MSX];
                float2 p[U][MSX];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t s = s0 + u * kEvalBlockThreads;
                    if (s < n) {
                        if (Gt) {
                            base[u] = Gt[s];
                        } else {
                            base[u] = make_float2(-a.ecost[off + s].x, s >= pd.pre_begin ? 1.0f : 0.0f);
                        }
                        const size_t b0 = off * stride + s;
#pragma unroll
                        for (int j = 0; j < MS; ++j)
                            if (j < stride) {
                                c[u][j] = a.ecol[b0 + (size_t)j * n1];
                                p[u][j] = a.ep[b0 + (size_t)j * n1];
                            }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t s = s0 + u * kEvalBlockThreads;
                    if (s < n) one(s, base[u], c[u], p[u]);
                }
            }
        } else {
            for (uint32_t s = threadIdx.x; s < n; s += kEvalBlockThreads) {
                const float2 base =
                    Gt ? Gt[s] : make_float2(-a.ecost[off + s].x, s >= pd.pre_begin ? 1.0f : 0.0f);
                const size_t b0 = off * stride + s;
                float yc = base.x, yp = base.y;
                for (int j = 0; j < stride; ++j) {
                    const int32_t c = a.ecol[b0 + (size_t)j * n1];
                    const float px = a.ep[b0 + (size_t)j * n1].x;
                    const float2 v = Xo[c];
                    yc = __fmaf_rn(px, v.x, yc);
                    yp = __fmaf_rn(px, v.y, yp);
                }
                const float2 x = Xo[s];
                Xn[s] = make_float2(yc, yp);
                float dc = fabsf(yc - x.x), dp = fabsf(yp - x.y);
                if (Gt) {
                    dc = dc > noise * fabsf(yc) ? dc : 0.0f;
                    dp = dp > noise * fabsf(yp) ? dp : 0.0f;
                }
                m[0] = fmaxf(m[0], dc);
                m[1] = fmaxf(m[1], dp);
                m[2] = fmaxf(m[2], fabsf(yc));
                m[3] = fmaxf(m[3], fabsf(yp));
            }
        }
    };
    unsigned int sweeps = 0, sweeps_a = 0;
    bool converged = false;
    // A
    for (;;) {
        if (sweeps >= cap) break;
        float m[4];
        sweep(X(sweeps), X(sweeps + 1), nullptr, m);
        block_max(m, sweeps & 1, std::integral_constant<int, 4>{});
        ++sweeps;
        const float f = 3.814697265625e-06f; /* 2^-18 */
        if (m[0] <= f * m[2] && m[1] <= f * m[3]) break;
    }
    sweeps_a = sweeps;
    const float2 *B = X(sweeps);
    float2 *G = X(sweeps + 1);
    if (sweeps < cap) {
        // B: the table in double-float
        for (uint32_t s = threadIdx.x; s < n; s += kEvalBlockThreads) {
            const float2 cc = a.ecost[off + s];
            DF gc = {-cc.x, -cc.y};
            DF gp = {s >= pd.pre_begin ? 1.0f : 0.0f, 0.0f};
            const size_t b0 = off * stride + s;
            for (int j = 0; j < stride; ++j) {
                const int32_t c = a.ecol[b0 + (size_t)j * n1];
                const float2 p = a.ep[b0 + (size_t)j * n1];
                const float2 v = B[c];
                ArithDF::mac(gc, {p.x, p.y}, {v.x, 0.0f});
                ArithDF::mac(gp, {p.x, p.y}, {v.y, 0.0f});
            }
            const float2 b = B[s];
            gc = df_add(df_norm(gc), {-b.x, 0.0f});
            gp = df_add(df_norm(gp), {-b.y, 0.0f});
            G[s] = make_float2(__fadd_rn(gc.h, gc.l), __fadd_rn(gp.h, gp.l));
        }
        __syncthreads();
        // C
        unsigned int k = 0;
        while (sweeps < cap) {
            float m[4];
            sweep(D(k), D(k + 1), G, m);
            block_max(m, sweeps & 1, std::integral_constant<int, 2>{});
            ++sweeps;
            ++k;
            if (!(fmaxf(m[0], m[1]) > thr_f)) {
                converged = true;
                break;
            }
        }
        // D: E = B + d
        const float2 *d = D(k);
        for (uint32_t s = threadIdx.x; s < n; s += kEvalBlockThreads) {
            const float2 b = B[s], v = d[s];
            const DF ec = two_sum(b.x, v.x), ep = two_sum(b.y, v.y);
            a.E[0][off + s] = make_float4(ec.h, ec.l, ep.h, ep.l);
        }
    } else {
        for (uint32_t s = threadIdx.x; s < n; s += kEvalBlockThreads) {
            const float2 b = B[s];
            a.E[0][off + s] = make_float4(b.x, 0.0f, b.y, 0.0f);
        }
    }
    if (threadIdx.x == 0) {
        a.frozen[e] = converged ? 1 : 0;
        a.sweeps_pair[e] = (int32_t)sweeps;
        // per sweep the scheduler's transitions and costs are read once (the
        // table pass reads them once more); the values stay in shared memory.
        // Padding slots count neither as bytes nor as updates.
        const unsigned long long tm = a.pair_tmu[e];
        const unsigned long long per = (unsigned long long)n * 8ull + 12ull * tm;
        atomicAdd(&a.ctl->updates, (unsigned long long)sweeps * tm * 2ull);
        atomicAdd(&a.ctl->bytes, (unsigned long long)(sweeps + (sweeps > sweeps_a ? 1 : 0)) * per + 16ull * n);
        atomicMax(&a.ctl->block_sweeps, sweeps);
    }
}

// ------------------------------------------------------------- small kernels

// The FP32 phase hands over to the polish phase once a pair's residual is
// at most 2^-MORAP_THR32_SHIFT of its largest possible value.  Its
// round-down iterates increase monotonically to a fixed point of the rounded
// operator, where the residual is exactly 0, so any shift terminates.  The
// residual correction that follows needs a late hand-over: its table G is
// rounded to FP32 once, so G must be small (the hand-over values close to
// the fixed point).  The polish then stops 2^-MORAP_POLISH_SHIFT below eps1
// (see launch_setup_weights).
#ifndef MORAP_POLISH_SHIFT
#define MORAP_POLISH_SHIFT 3
#endif
#ifndef MORAP_THR32_SHIFT
#define MORAP_THR32_SHIFT 16
#endif

__device__ __forceinline__ float2 to_df(double d) {
    const float h = __double2float_rn(d);
    return make_float2(h, __double2float_rn(d - (double)h));
}

__global__ void k_setup_weights(const ProdDesc *prods, int P, int nI, int nJ, int K, int Kp, const double *W,
                                float2 *w32, double2 *w64, float4 *wdf, double *thr32, double *thr64, double eps1,
                                double eps_polish) {
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
        w32[idx] = make_float2(-__double2float_ru(wi), __double2float_rd(wp));
        const float2 a = to_df(wi), b = to_df(wp);
        wdf[idx] = make_float4(a.x, a.y, b.x, b.y);
        // FP32 phase: stop once the residual is within a few ulps of the
        // largest possible value (values lie in [0, w_p]); polish phase:
        // eps_polish (see launch_setup_weights).
        thr32[idx] = fmax(eps1, ldexp(wp, -MORAP_THR32_SHIFT));
        thr64[idx] = eps_polish;
    }
}

// w_pair (nullable): per (product, weight) pair its two weights; a pair with
// both 0 has every value 0 at every sweep (each Q is 0), so it starts frozen
// ("previous" residual 0) instead of being swept once to find that out.
__global__ void k_loop_init(LoopCtl *ctl, unsigned int *list0, unsigned int n_items, unsigned long long *r0,
                            unsigned long long *r1, unsigned long long *r2, size_t n_pairs, int32_t *sweeps_pair,
                            uint8_t *frozen, unsigned int cap, uint8_t *chg_prev, const double2 *w_pair,
                            unsigned int tail) {
    const size_t gid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = gid; i < n_items; i += stride) {
        list0[i] = (unsigned int)i;
        if (chg_prev) chg_prev[i] = 1;
    }
    const unsigned long long inf_bits = (unsigned long long)__double_as_longlong(CUDART_INF);
    for (size_t i = gid; i < n_pairs; i += stride) {
        r0[i] = 0ull;
        r1[i] = 0ull;
        // "previous" residual of sweep 0: everything active, except pairs with no weight
        const bool idle = w_pair && w_pair[i].x == 0.0 && w_pair[i].y == 0.0;
        r2[i] = idle ? 0ull : inf_bits;
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
        ctl->skipped = 0;
        ctl->block_sweeps = 0;
        ctl->updates = 0;
        ctl->bytes = 0;
        ctl->undecided = 0;
        ctl->decided = 0;
        ctl->computed = 0;
        ctl->tail = tail;
        ctl->bar = 0;
        ctl->bar_err = 0;
        ctl->tail_sweeps = 0;
    }
}

// Evaluated after each body of 6 sweeps: continue while the work list of
// the next sweep is longer than ctl->tail (non-empty without a tail launch)
// and the sweep cap is not reached.
__global__ void k_loop_control(LoopCtl *ctl, cudaGraphConditionalHandle handle, int next_idx) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    ctl->sweep_base += 6;
    const bool more = ctl->cnt[next_idx] > ctl->tail;
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

// The residual-correction table: G[sa][k] = -w_i c(sa) + sum_t p_t B(s'_t)
// - B(s) (+ w_p at a pre-sink state) for every action row of every state,
// formed in double-float from the FP32 values B and rounded once to FP32.
// One thread per (state, weight); the threads of a state write its rows'
// Kp weights as consecutive words.
template <int KP>
__global__ void __launch_bounds__(kThreads) k_delta_table(SweepArgs a, int n_chunks, const float *B, float *G) {
    constexpr int SPR = kThreads / KP > 0 ? kThreads / KP : 1;
    const int k = threadIdx.x % KP, slot = threadIdx.x / KP;
    if (slot >= SPR) return;
    for (int item = blockIdx.x; item < n_chunks; item += gridDim.x) {
        const int4 ch = a.chunks[item];
        const ProdDesc pd = a.prods[ch.x];
        const ArithDF::W w = a.wdf[(size_t)ch.x * KP + k];
        for (int s = ch.y + slot; s < ch.z; s += SPR) {
            const uint32_t u = pd.state_off + (uint32_t)s;
            const bool pre = (uint32_t)s >= pd.pre_begin;
            const float bs = B[(size_t)u * KP + k];
            const uint32_t a0 = a.state_sa[u], a1 = a.state_sa[u + 1];
            for (uint32_t sa = a0; sa < a1; ++sa) {
                const float2 cd = a.costdf[sa];
                DF acc = ArithDF::reward(w, {cd.x, cd.y});
                for (uint32_t t = a.sa_tr[sa], t1 = a.sa_tr[sa + 1]; t < t1; ++t) {
                    const float2 pr = a.pdf[t];
                    ArithDF::mac(acc, {pr.x, pr.y}, {B[(size_t)a.col[t] * KP + k], 0.0f});
                }
                acc = ArithDF::add_base(df_norm(acc), w, pre);
                acc = df_add(acc, {-bs, 0.0f});
                G[(size_t)sa * KP + k] = __fadd_rn(acc.h, acc.l);
            }
        }
    }
}

// V = B + d as an unevaluated double-float sum (two_sum is exact).
__global__ void k_delta_combine(const float *B, const float *d, float2 *V, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const DF v = two_sum(B[i], d[i]);
        V[i] = make_float2(v.h, v.l);
    }
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
        // a product without non-done states has nothing to iterate (its
        // values are 0): converged
        status_out[idx] = (frozen[idx] || pd.n_nd == 0) ? MORAP_OK : MORAP_ENOTCONV;
    }
}

__global__ void k_gather_eval(const int4 *pairs, int n_pairs, const ProdDesc *prods, const float4 *E, double *rc,
                              double *rp) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_pairs; e += gridDim.x * blockDim.x) {
        const int4 pr = pairs[e];
        const ProdDesc pd = prods[pr.x];
        if ((uint32_t)pd.init_local >= pd.n_nd) {
            rc[e] = 0.0;
            rp[e] = 0.0;
        } else {
            const float4 v = E[(size_t)pr.z + pd.init_local];
            rc[e] = (double)v.x + (double)v.y;
            rp[e] = (double)v.z + (double)v.w;
        }
    }
}

template <class Ar>
constexpr int smem_of() {
    return (kThreads / 32) * (Ar::STAGE_BYTES + 64 * (int)sizeof(typename Ar::W));  // sized for the largest Kp
}

using SweepFn = void (*)(SweepArgs, int);

struct SweepKernel {
    SweepFn f;
    int smem;  // dynamic shared memory per block
};

template <class Ar, int KP, int V>
SweepKernel sweep_kernel() {
    using VA = Variants<Ar>;
    return {&k_sweep<Ar, KP, VA::vmax[V], VA::d[V], VA::minb[V], VA::pipe[V]>, smem_of<Ar>()};
}

template <class Ar, int KP, int... V>
std::array<SweepKernel, Variants<Ar>::N> sweep_row(std::integer_sequence<int, V...>) {
    return {sweep_kernel<Ar, KP, V>()...};
}

// sweep_fn<Ar>(log2 Kp, variant)
template <class Ar>
const SweepKernel *sweep_fn(int lg, int v) {
    using Seq = std::make_integer_sequence<int, Variants<Ar>::N>;
    static const std::array<std::array<SweepKernel, Variants<Ar>::N>, 7> table = {
        sweep_row<Ar, 1>(Seq{}),  sweep_row<Ar, 2>(Seq{}),  sweep_row<Ar, 4>(Seq{}), sweep_row<Ar, 8>(Seq{}),
        sweep_row<Ar, 16>(Seq{}), sweep_row<Ar, 32>(Seq{}), sweep_row<Ar, 64>(Seq{})};
    if (lg < 0 || lg > 6 || v < 0 || v >= Variants<Ar>::N) return nullptr;
    return &table[lg][v];
}

struct TailKernel {
    void (*f)(SweepArgs);
    int smem;
};

// k_sweep_tail in one kernel shape per format (MORAP_TAIL_SHAPE, 0 by
// default), per log2 Kp.
#ifndef MORAP_TAIL_SHAPE
#define MORAP_TAIL_SHAPE 0
#endif
// Blocks per SM the tail kernel's registers are sized for: it keeps each
// warp's item across sweeps, which at two blocks per SM spills.
#ifndef MORAP_TAIL_MINB
#define MORAP_TAIL_MINB 1
#endif
template <class Ar, int KP>
TailKernel tail_kernel() {
    using VA = Variants<Ar>;
    constexpr int V = MORAP_TAIL_SHAPE;
    return {&k_sweep_tail<Ar, KP, VA::vmax[V], VA::d[V], MORAP_TAIL_MINB, VA::pipe[V]>, smem_of<Ar>()};
}

template <class Ar>
const TailKernel *tail_fn(int lg) {
    static const std::array<TailKernel, 7> table = {tail_kernel<Ar, 1>(),  tail_kernel<Ar, 2>(),
                                                     tail_kernel<Ar, 4>(),  tail_kernel<Ar, 8>(),
                                                     tail_kernel<Ar, 16>(), tail_kernel<Ar, 32>(),
                                                     tail_kernel<Ar, 64>()};
    if (lg < 0 || lg > 6) return nullptr;
    return &table[lg];
}

int log2_kp(int Kp) {
    int l = 0;
    while ((1 << l) < Kp) ++l;
    return (1 << l) == Kp ? l : -1;
}

template <class Ar>
int launch_sweep_t(int Kp, int variant, const SweepArgs &a, int pos, int grid, cudaStream_t s) {
    const SweepKernel *k = sweep_fn<Ar>(log2_kp(Kp), variant);
    if (!k) return (int)cudaErrorInvalidValue;
    k->f<<<grid, kThreads, k->smem, s>>>(a, pos);
    return (int)cudaGetLastError();
}

// A cooperative launch (every block resident at once, which the grid
// barriers of k_sweep_tail need); the runtime refuses a grid that does not fit.
template <class Ar>
int launch_sweep_tail_t(int Kp, const SweepArgs &a, int grid, cudaStream_t s) {
    const TailKernel *k = tail_fn<Ar>(log2_kp(Kp));
    if (!k || grid <= 0) return (int)cudaErrorInvalidValue;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned int)grid);
    lc.blockDim = dim3(kThreads);
    lc.dynamicSmemBytes = (size_t)k->smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    void *args[] = {const_cast<SweepArgs *>(&a)};
    return (int)cudaLaunchKernelExC(&lc, reinterpret_cast<const void *>(k->f), args);
}

template <class Ar>
cudaError_t set_attr_t() {
    for (int lg = 0; lg < 7; ++lg) {
        for (int v = 0; v < Variants<Ar>::N; ++v) {
            const SweepKernel *k = sweep_fn<Ar>(lg, v);
            const cudaError_t e = cudaFuncSetAttribute(k->f, cudaFuncAttributeMaxDynamicSharedMemorySize, k->smem);
            if (e != cudaSuccess) return e;
        }
        const TailKernel *t = tail_fn<Ar>(lg);
        const cudaError_t e = cudaFuncSetAttribute(t->f, cudaFuncAttributeMaxDynamicSharedMemorySize, t->smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

template <class Ar>
int blocks_per_sm_t(int Kp, int variant) {
    const SweepKernel *k = sweep_fn<Ar>(log2_kp(Kp), variant);
    int n = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k->f, kThreads, k->smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

int sweep_setup_attributes() {
    cudaError_t e = set_attr_t<ArithF32>();
    if (e == cudaSuccess) e = set_attr_t<ArithDF>();
    if (e == cudaSuccess) e = set_attr_t<ArithDelta>();
    return (int)e;
}

int eval_block_setup() {
    cudaError_t e = cudaFuncSetAttribute(k_eval_block<4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kEvalBlockSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_eval_block<8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEvalBlockSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_eval_block<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEvalBlockSmem);
    return (int)e;
}

int launch_eval_block(const EvalArgs &a, const int *bpairs, int n_bpairs, uint32_t max_states, unsigned int cap,
                      void *s) {
    if (n_bpairs <= 0) return 0;
    const size_t smem = 2ull * max_states * sizeof(float4);
    if (smem > (size_t)kEvalBlockSmem) return (int)cudaErrorInvalidValue;
    if (a.stride <= 4)
        k_eval_block<4, 2><<<n_bpairs, kEvalBlockThreads, smem, (cudaStream_t)s>>>(a, bpairs, cap);
    else if (a.stride <= 8)
        k_eval_block<8, 1><<<n_bpairs, kEvalBlockThreads, smem, (cudaStream_t)s>>>(a, bpairs, cap);
    else
        k_eval_block<0, 1><<<n_bpairs, kEvalBlockThreads, smem, (cudaStream_t)s>>>(a, bpairs, cap);
    return (int)cudaGetLastError();
}

int sweep_smem_bytes(int kind) {
    return kind == kSweepDF ? smem_of<ArithDF>() : kind == kSweepDelta ? smem_of<ArithDelta>() : smem_of<ArithF32>();
}

int sweep_blocks_per_sm(int kind, int Kp, int variant) {
    return kind == kSweepDF      ? blocks_per_sm_t<ArithDF>(Kp, variant)
           : kind == kSweepDelta ? blocks_per_sm_t<ArithDelta>(Kp, variant)
                                 : blocks_per_sm_t<ArithF32>(Kp, variant);
}

int sweep_variant_count(int kind) {
    return kind == kSweepDF ? Variants<ArithDF>::N : kind == kSweepDelta ? Variants<ArithDelta>::N : Variants<ArithF32>::N;
}





int eval_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_eval_sweep, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

int launch_sweep(int kind, int Kp, int variant, const SweepArgs &a, int pos, int grid, void *s) {
    return kind == kSweepDF      ? launch_sweep_t<ArithDF>(Kp, variant, a, pos, grid, (cudaStream_t)s)
           : kind == kSweepDelta ? launch_sweep_t<ArithDelta>(Kp, variant, a, pos, grid, (cudaStream_t)s)
                                 : launch_sweep_t<ArithF32>(Kp, variant, a, pos, grid, (cudaStream_t)s);
}

int launch_sweep_tail(int kind, int Kp, const SweepArgs &a, int grid, void *s) {
    return kind == kSweepDF      ? launch_sweep_tail_t<ArithDF>(Kp, a, grid, (cudaStream_t)s)
           : kind == kSweepDelta ? launch_sweep_tail_t<ArithDelta>(Kp, a, grid, (cudaStream_t)s)
                                 : launch_sweep_tail_t<ArithF32>(Kp, a, grid, (cudaStream_t)s);
}

int launch_barrier_selfcheck(LoopCtl *ctl, int grid, void *s) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned int)grid);
    lc.blockDim = dim3(kThreads);
    lc.stream = (cudaStream_t)s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    void *args[] = {&ctl};
    return (int)cudaLaunchKernelExC(&lc, reinterpret_cast<const void *>(&k_barrier_selfcheck), args);
}

template <class Ar>
int tail_blocks_per_sm_t(int Kp) {
    const TailKernel *k = tail_fn<Ar>(log2_kp(Kp));
    int n = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k->f, kThreads, k->smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int sweep_tail_blocks_per_sm(int kind, int Kp) {
    return kind == kSweepDF      ? tail_blocks_per_sm_t<ArithDF>(Kp)
           : kind == kSweepDelta ? tail_blocks_per_sm_t<ArithDelta>(Kp)
                                 : tail_blocks_per_sm_t<ArithF32>(Kp);
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

int launch_anchor(int Kp, const SweepArgs &a, int n_chunks, double tau, uint8_t *policy, int round, void *sv) {
    cudaStream_t s = (cudaStream_t)sv;
    const int grid = n_chunks < 8192 ? n_chunks : 8192;
    if (grid <= 0) return 0;
    switch (Kp) {
    case 1: k_anchor<1><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy, round); break;
    case 2: k_anchor<2><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy, round); break;
    case 4: k_anchor<4><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy, round); break;
    case 8: k_anchor<8><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy, round); break;
    case 16: k_anchor<16><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy, round); break;
    case 32: k_anchor<32><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy, round); break;
    case 64: k_anchor<64><<<grid, kThreads, 0, s>>>(a, n_chunks, tau, policy, round); break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

int launch_eval_compact(const EvalArgs &a, int n_chunks, void *s) {
    if (n_chunks <= 0) return 0;
    k_eval_compact<<<n_chunks < 65535 ? n_chunks : 65535, kThreads, 0, (cudaStream_t)s>>>(a, n_chunks);
    return (int)cudaGetLastError();
}

int launch_eval_sweep(const EvalArgs &a, int pos, int grid, void *s) {
    k_eval_sweep<<<grid, kThreads, 0, (cudaStream_t)s>>>(a, pos);
    return (int)cudaGetLastError();
}

int launch_setup_weights(const ProdDesc *prods, int P, int nI, int nJ, int K, int Kp, const double *W, float2 *w32,
                         double2 *w64, float4 *wdf, double *thr32, double *thr64, double eps1, bool after_fp32,
                         void *s) {
    const size_t n = (size_t)P * Kp;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    // A phase that starts from the FP32 phase's values stops at a residual
    // 2^-MORAP_POLISH_SHIFT below eps1: those values lie below the exact
    // iterate by the FP32 roundings of the last sweeps, which add up along
    // every path (to 1e-6 on paths of hundreds of steps) while each is
    // smaller than eps1, so a residual test at eps1 stops before the
    // deficit has been propagated away (c 2.3e-6 below the fixed point on
    // the 128x128 batch; 2e-7 at eps1 / 8).  A phase that starts from 0
    // stops at eps1, as Algorithm 3 does.
    const double eps_polish = after_fp32 ? ldexp(eps1, -MORAP_POLISH_SHIFT) : eps1;
    k_setup_weights<<<grid > 0 ? grid : 1, 256, 0, (cudaStream_t)s>>>(prods, P, nI, nJ, K, Kp, W, w32, w64, wdf,
                                                                     thr32, thr64, eps1, eps_polish);
    return (int)cudaGetLastError();
}

int launch_loop_init(LoopCtl *ctl, unsigned int *list0, unsigned int n_items, unsigned long long *res[3],
                     size_t n_pairs, int32_t *sweeps_pair, uint8_t *frozen, unsigned int cap, void *s,
                     uint8_t *chg_prev, const double2 *w_pair, unsigned int tail) {
    const size_t n = n_items > n_pairs ? n_items : n_pairs;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_loop_init<<<grid > 0 ? grid : 1, 256, 0, (cudaStream_t)s>>>(ctl, list0, n_items, res[0], res[1], res[2],
                                                                 n_pairs, sweeps_pair, frozen, cap, chg_prev,
                                                                 w_pair, tail);
    return (int)cudaGetLastError();
}

// The input items of every work item: the items (of the same product) that
// hold successors of its states.  One warp per item; duplicates are removed
// with warp matching; more than kInItems distinct inputs mark the item as
// always recomputed.
__global__ void k_item_inputs(const int4 *chunks, int n_items, const ProdDesc *prods, const uint32_t *state_tr,
                              const int32_t *col, int32_t *in_items, uint2 *item_w, const uint32_t *state_sa) {
    __shared__ int32_t set[kThreads / 32][kInItems];
    __shared__ int cnt[kThreads / 32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int item = blockIdx.x * (kThreads / 32) + w; item < n_items; item += gridDim.x * (kThreads / 32)) {
        const int4 ch = chunks[item];
        const ProdDesc pd = prods[ch.x];
        if (lane == 0) cnt[w] = 0;
        __syncwarp();
        const uint32_t t0 = state_tr[pd.state_off + ch.y], t1 = state_tr[pd.state_off + ch.z];
        if (lane == 0) item_w[item] = make_uint2(t1 - t0, state_sa[pd.state_off + ch.z] - state_sa[pd.state_off + ch.y]);
        for (uint32_t base = t0; base < t1; base += 32) {
            // the set as the previous batches left it (they are complete: __syncwarp
            // below); values inserted by this batch are distinct from each other
            const int n_before = min(cnt[w], kInItems);
            const uint32_t t = base + lane;
            int v = -1;
            if (t < t1) {
                const uint32_t cl = (uint32_t)col[t] - pd.state_off;
                if (cl < pd.n_nd) {
                    const int it = (int)(pd.item_off + cl / kChunk);
                    if (it != item) v = it;
                }
            }
            const unsigned int same = __match_any_sync(0xffffffffu, v);
            if (v >= 0 && (__ffs(same) - 1) == lane) {  // one lane per distinct value of this batch
                bool present = false;
                for (int q = 0; q < n_before; ++q) present = present || set[w][q] == v;
                if (!present) {
                    const int at = atomicAdd(&cnt[w], 1);
                    if (at < kInItems) set[w][at] = v;
                }
            }
            __syncwarp();
        }
        const int n = cnt[w];
        if (lane < kInItems)
            in_items[(size_t)item * kInItems + lane] = n > kInItems ? -2 : (lane < n ? set[w][lane] : -1);
        __syncwarp();
    }
}

int launch_item_inputs(const int4 *chunks, int n_items, const ProdDesc *prods, const uint32_t *state_tr,
                       const int32_t *col, int32_t *in_items, uint2 *item_w, const uint32_t *state_sa, void *s) {
    if (n_items <= 0) return 0;
    const int grid = (n_items + kThreads / 32 - 1) / (kThreads / 32);
    k_item_inputs<<<grid < 65535 ? grid : 65535, kThreads, 0, (cudaStream_t)s>>>(chunks, n_items, prods, state_tr, col,
                                                                              in_items, item_w, state_sa);
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

int launch_delta_table(int Kp, const SweepArgs &a, int n_chunks, const float *B, float *G, void *sv) {
    cudaStream_t s = (cudaStream_t)sv;
    const int grid = n_chunks < 8192 ? n_chunks : 8192;
    if (grid <= 0) return 0;
    switch (Kp) {
    case 1: k_delta_table<1><<<grid, kThreads, 0, s>>>(a, n_chunks, B, G); break;
    case 2: k_delta_table<2><<<grid, kThreads, 0, s>>>(a, n_chunks, B, G); break;
    case 4: k_delta_table<4><<<grid, kThreads, 0, s>>>(a, n_chunks, B, G); break;
    case 8: k_delta_table<8><<<grid, kThreads, 0, s>>>(a, n_chunks, B, G); break;
    case 16: k_delta_table<16><<<grid, kThreads, 0, s>>>(a, n_chunks, B, G); break;
    case 32: k_delta_table<32><<<grid, kThreads, 0, s>>>(a, n_chunks, B, G); break;
    case 64: k_delta_table<64><<<grid, kThreads, 0, s>>>(a, n_chunks, B, G); break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

int launch_delta_combine(const float *B, const float *d, float2 *V, size_t n, void *s) {
    const int grid = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
    k_delta_combine<<<grid > 0 ? grid : 1, 256, 0, (cudaStream_t)s>>>(B, d, V, n);
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

int launch_gather_eval(const int4 *pairs, int n_pairs, const ProdDesc *prods, const float4 *E, double *rc,
                       double *rp, void *s) {
    const int grid = (n_pairs + 255) / 256;
    if (grid == 0) return 0;
    k_gather_eval<<<grid, 256, 0, (cudaStream_t)s>>>(pairs, n_pairs, prods, E, rc, rp);
    return (int)cudaGetLastError();
}

}  // namespace morap

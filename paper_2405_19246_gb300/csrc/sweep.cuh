// Sweep kernels: the marginal product M_j of l-marginal Sinkhorn with L1 cost
// (arXiv 2405.19246, Sec. 3 and Sec. 4.2) as scans over tiles of the merged
// support order.
//
// What is computed.  For target j and every subset S of R = [l]\{j}:
//   F_S(x) = sum over placements of one point of each marginal of S, all
//            before x in the merged order, of prod phi * exp(-cost integral)
//   (the cost integral grows at rate w_s = |S|(l-|S|), Sec. 4.2 cost).
// In the "cumulative frame" of a tile, F~_S(t) = F_S(t) exp(w_s pos_t),
// pos_t = (x_t - x_base)/eps, the decay disappears and a point of marginal m
// only injects
//     F~_T += phi_m exp((w_s - w_{s-1}) pos_t) F~_{T\m}   for every T containing m,
// which is the paper's recurrences J = lambda^2 J + psi P (Algorithm 2) with the
// multipliers moved into the frame.
//
// Block engine (Engine, one tile per CTA, each thread a contiguous chunk of
// points).  Level s = |T| depends on level s-1 at the same point, so a tile
// runs level by level: walk the points recomputing levels 1..s from the final
// lower-level values, block-scan the level-s chunk totals, take the level's
// carries, then give every state of the level its own scale (the largest
// tile-end value of the state becomes 1).  Values inside a tile are FP32 (or
// FP64) "f-representations" F~_S exp(-sum_{m in S} beta_m) / scale_S with
// per-tile FP64 baselines beta_m (the re-centring of Algorithm 5).  Carries
// between tiles are scaled floats (mantissa, binary exponent).
//
// This engine serves the objective sweeps over all 2^l subsets
// (objective.cuh): tile operators (k_tileop) and the multi-block carry scan
// (k_carry) for l <= 4, the look-back scan (lookback, k_bwd) for l = 5..7.
// The carry scan also serves the marginal products of l <= 5, whose tile
// kernels are in tile.cuh; the products of l >= 6 run in warp.cuh with the
// level scans (k_lscan) defined here.
#pragma once
#include <limits>
#include <climits>
#include <cstddef>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include <cuda_pipeline.h>

#include "mmot_internal.cuh"

namespace mmot {

__host__ __device__ constexpr int popc_c(int x)
{
    int c = 0;
    while (x) {
        c += x & 1;
        x >>= 1;
    }
    return c;
}

template <typename V>
__device__ __forceinline__ V vexp(V x);
template <>
__device__ __forceinline__ float vexp<float>(float x) { return __expf(x); }
template <>
__device__ __forceinline__ double vexp<double>(double x) { return exp(x); }
template <typename V>
__device__ __forceinline__ V vlog(V x);
template <>
__device__ __forceinline__ float vlog<float>(float x) { return logf(x); }
template <>
__device__ __forceinline__ double vlog<double>(double x) { return log(x); }

// exp of an FP64 argument to the accuracy of V (FP32: exp2f of the
// fractional part of x*log2(e), the integer part scales the exponent)
template <typename V>
__device__ __forceinline__ double exp_acc(double x);
template <>
__device__ __forceinline__ double exp_acc<double>(double x) { return exp(x); }
template <>
__device__ __forceinline__ double exp_acc<float>(double x)
{
    if (!(x > -1.0e300)) return 0.0;
    const double y = x * 1.4426950408889634074;
    if (y > 1.0e4) return INFINITY;
    if (y < -1.0e4) return 0.0;
    const double n = floor(y);
    return ldexp((double)exp2f((float)(y - n)), (int)n);
}

constexpr double kLog2e = 1.4426950408889634074;  // log2(e)
constexpr double kLn2 = 0.69314718055994530942;    // ln(2)

template <typename V>
__device__ __forceinline__ V vexp2(V x);
template <>
__device__ __forceinline__ float vexp2<float>(float x) { return exp2f(x); }
template <>
__device__ __forceinline__ double vexp2<double>(double x) { return exp2(x); }
template <typename V>
__device__ __forceinline__ V vldexp(V x, int e);
template <>
__device__ __forceinline__ float vldexp<float>(float x, int e) { return ldexpf(x, e); }
template <>
__device__ __forceinline__ double vldexp<double>(double x, int e) { return ldexp(x, e); }
template <typename V>
__device__ __forceinline__ V vfrexp(V x, int *e);
template <>
__device__ __forceinline__ float vfrexp<float>(float x, int *e) { return frexpf(x, e); }
template <>
__device__ __forceinline__ double vfrexp<double>(double x, int *e) { return frexp(x, e); }

// Scaled float: value = m * 2^k with m = 0 or 0.5 <= m < 1.  Carries between
// tiles span far more than the FP32 (or FP64) exponent range; keeping the
// binary exponent as an integer makes products with exp(x) for a large FP64 x
// cost one exp2 of the fractional part of x*log2(e) and no FP64
// transcendental.
template <typename V>
struct Sf {
    V m;
    int k;
};

template <typename V>
__device__ __forceinline__ Sf<V> sf_zero() { return Sf<V>{V(0), 0}; }

// x = m 2^k with 0.5 <= m < 1 (x >= 0).  FP32: read and set the exponent
// field directly; subnormal x (far below every value that matters next to
// the O(1) mantissas used here) is flushed to 0.
template <typename V>
__device__ __forceinline__ Sf<V> sf_make(V x);
template <>
__device__ __forceinline__ Sf<float> sf_make<float>(float x)
{
    const int bits = __float_as_int(x);
    const int ef = (bits >> 23) & 0xff;
    Sf<float> r;
    if (ef == 0) {
        r.m = 0.f;
        r.k = 0;
    } else {
        r.m = __int_as_float((bits & 0x807fffff) | (126 << 23));
        r.k = ef - 126;
    }
    return r;
}
template <>
__device__ __forceinline__ Sf<double> sf_make<double>(double x)
{
    Sf<double> r;
    if (x == 0.0) {
        r.m = 0.0;
        r.k = 0;
    } else {
        r.m = frexp(x, &r.k);
    }
    return r;
}

// 2^d for d <= 0 (FP32: built from the exponent field; 0 below 2^-126)
template <typename V>
__device__ __forceinline__ V pow2neg(int d);
template <>
__device__ __forceinline__ float pow2neg<float>(int d)
{
    return (d < -126) ? 0.f : __int_as_float((d + 127) << 23);
}
template <>
__device__ __forceinline__ double pow2neg<double>(int d)
{
    return (d < -1022) ? 0.0 : __longlong_as_double((long long)(d + 1023) << 52);
}

// a * exp(x) for an FP64 exponent x (x = -inf gives 0)
template <typename V>
__device__ __forceinline__ Sf<V> sf_scale_exp(Sf<V> a, double x)
{
    if (a.m == V(0) || !(x > -1.0e300)) return sf_zero<V>();
    const double y = fmin(x * kLog2e, 1.0e9);
    if (y < -1.0e9) return sf_zero<V>();
    const double n = floor(y);
    Sf<V> r = sf_make<V>(a.m * vexp2<V>((V)(y - n)));
    r.k += a.k + (int)n;
    return r;
}

// A tile constant x as x log2(e) in fixed point: int64 with 32 fractional
// bits.  Sums of such values are exact, so the scale of a state,
// exp(sum_{m in T} beta_m + gamma_|T|), costs integer adds and one FP32 exp2
// instead of FP64 arithmetic per state (one FP64 warp instruction occupies the
// FP64 pipe of a sub-partition for about 64 cycles on this GPU).  Each term
// is rounded to 2^-32, far below the FP32 mantissa.  (FP32 path only: the
// FP64 path keeps FP64 exponents.)
__device__ __forceinline__ long long fx_log2(double x)
{
    const double y = fmin(fmax(x * (kLog2e * 4294967296.0), -4.0e18), 4.0e18);
    return __double2ll_rn(y);
}

// a * 2^(X / 2^32)
template <typename V>
__device__ __forceinline__ Sf<V> sf_scale_fx(Sf<V> a, long long X)
{
    if (a.m == V(0)) return a;
    const int n = (int)(X >> 32);   // floor
    const float fr = (float)(unsigned)(X & 0xffffffffll) * 2.3283064365386963e-10f;
    Sf<V> r = sf_make<V>(a.m * (V)exp2f(fr));
    r.k += a.k + n;
    return r;
}

template <typename V>
__device__ __forceinline__ Sf<V> sf_add(Sf<V> a, Sf<V> b)
{
    if (a.m == V(0)) return b;
    if (b.m == V(0)) return a;
    Sf<V> r;
    if (a.k >= b.k) {
        r = sf_make<V>(a.m + b.m * pow2neg<V>(b.k - a.k));
        r.k += a.k;
    } else {
        r = sf_make<V>(b.m + a.m * pow2neg<V>(a.k - b.k));
        r.k += b.k;
    }
    return r;
}

// value * 2^(-shift)
template <typename V>
__device__ __forceinline__ V sf_value(Sf<V> a, int shift)
{
    if (a.m == V(0)) return V(0);
    const int d = a.k - shift;
    return (d <= 0) ? a.m * pow2neg<V>(d) : vldexp<V>(a.m, d);
}

// sum over the 32 lanes; every lane receives lane 0's result
template <typename V>
__device__ __forceinline__ Sf<V> sf_warp_sum(Sf<V> a)
{
    constexpr unsigned FULL = 0xffffffffu;
    int kmax = (a.m == V(0)) ? INT_MIN : a.k;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(FULL, kmax, o));
    if (kmax == INT_MIN) return sf_zero<V>();
    V m = (a.m == V(0)) ? V(0) : a.m * pow2neg<V>(a.k - kmax);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const V y = __shfl_down_sync(FULL, m, o);
        if ((threadIdx.x & 31) + o < 32) m += y;
    }
    m = __shfl_sync(FULL, m, 0);
    Sf<V> r = sf_make<V>(m);
    r.k += kmax;
    return r;
}

// sf_warp_sum with rolled shuffle rounds: for code that runs once per warp,
// where fetching the instructions costs more than the loop overhead
template <typename V>
__device__ __forceinline__ Sf<V> sf_warp_sum_rolled(Sf<V> a)
{
    constexpr unsigned FULL = 0xffffffffu;
    int kmax = (a.m == V(0)) ? INT_MIN : a.k;
#pragma unroll 1
    for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(FULL, kmax, o));
    if (kmax == INT_MIN) return sf_zero<V>();
    V m = (a.m == V(0)) ? V(0) : a.m * pow2neg<V>(a.k - kmax);
#pragma unroll 1
    for (int o = 1; o < 32; o <<= 1) {
        const V y = __shfl_down_sync(FULL, m, o);
        if ((threadIdx.x & 31) + o < 32) m += y;
    }
    m = __shfl_sync(FULL, m, 0);
    Sf<V> r = sf_make<V>(m);
    r.k += kmax;
    return r;
}

// storage form of a scaled float
template <typename V>
struct SfSt;
template <>
struct SfSt<float> {
    using T = float2;
};
template <>
struct SfSt<double> {
    using T = double2;
};
template <typename V>
using SfT = typename SfSt<V>::T;

__device__ __forceinline__ float2 sf_store(Sf<float> a) { return make_float2(a.m, __int_as_float(a.k)); }
__device__ __forceinline__ double2 sf_store(Sf<double> a) { return make_double2(a.m, (double)a.k); }
template <typename V>
__device__ __forceinline__ Sf<V> sf_load(SfT<V> d);
template <>
__device__ __forceinline__ Sf<float> sf_load<float>(float2 d) { return Sf<float>{d.x, __float_as_int(d.y)}; }
template <>
__device__ __forceinline__ Sf<double> sf_load<double>(double2 d) { return Sf<double>{d.x, (int)d.y}; }
template <typename V>
__device__ __forceinline__ SfT<V> *sfp(void *p) { return static_cast<SfT<V> *>(p); }
template <typename V>
__device__ __forceinline__ const SfT<V> *sfp(const void *p) { return static_cast<const SfT<V> *>(p); }
template <typename V>
__device__ __forceinline__ SfT<V> sf_one_st() { return sf_store(Sf<V>{V(0.5), 1}); }

// a * b
template <typename V>
__device__ __forceinline__ Sf<V> sf_mul(Sf<V> a, Sf<V> b)
{
    if (a.m == V(0) || b.m == V(0)) return sf_zero<V>();
    Sf<V> r = sf_make<V>(a.m * b.m);
    r.k += a.k + b.k;
    return r;
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait on a flag: returns the nonzero flag, or -1 when the poll limit
// is reached or another tile has already reported an error.
__device__ __forceinline__ int wait_flag(const int *flag, const int *err, int limit)
{
    int f = ld_acquire(flag);
    int it = 0;
    while (f == 0) {
        if (++it > limit) return -1;
        if ((it & 63) == 0 && *(volatile const int *)err != 0) return -1;
        __nanosleep(32);
        f = ld_acquire(flag);
    }
    return f;
}

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

template <int NB, typename V, int NT, int C, int JCAP, bool WITH_G>
struct SweepSmem {
    static constexpr int NS = 1 << NB;
    static constexpr int K = NT * C;
    static constexpr int NW = NT / 32;
    Sf<V> E[NS];           // carry of each state at the tile base (absolute)
    Sf<V> Eh[NS];          // the same times exp(-sum_{m in S} beta_m)
    Sf<V> Gs[NS];          // scale of each state (provisional while its level runs)
    Sf<V> GsG[NS];         // final scales of the backward pass (combine)
    V rr[NS][NB];          // injection ratio into state T at a point of bit k
    V rhoS[NS];            // provisional-to-final rescale of each state of the level
    int eS[NS];            // combine: binary exponent of scale(F_S) * scale(G_{R\S})
    double beta[NB];       // baselines of the marginals mapped to bits
    double dred[NW];       // FP64 reduction scratch
    V scan[NW][NS];        // warp totals / warp prefixes
    V tot[NS];             // block totals of the current level
    V tc[NS];              // tile carries in f-representation
    V D[NB];               // provisional level shifts
    V fred[NW][NB];        // reduction scratch
    int ired[NW];
    int ntarget;
    int bits;              // bits (marginals other than the target) present in the tile
    V pos[K];
    V lphi[K];
    int16_t slot[K];
    uint8_t mid[K];
    // backward states at target points; also the scratch of the tile-operator
    // composition (NB x NS x NT values)
    static constexpr int OPSZ = (NB <= kMaxOpBits) ? NB * NS * (NT / 32) : 0;
    static constexpr int GSZ = (NS * JCAP > OPSZ) ? NS * JCAP : OPSZ;
    // 16-byte aligned: the epilogue keeps FP64 values in this space
    alignas(16) V G[WITH_G ? GSZ : 1];
    double lmu[WITH_G ? JCAP : 1];   // ln mu of the tile's target points (prefetched)
};

// Per-thread engine: a contiguous chunk of C points of the tile, in the
// processing order of the pass (forward: increasing x, backward: decreasing).
// NB state bits; L marginals in the cost (L = NB + 1 for a marginal product,
// L = NB for the all-subset sweeps of the objective).
template <int NB, typename V, int NT, int C, int JCAP, bool WITH_G, int L = NB + 1>
struct Engine {
    static constexpr int NS = 1 << NB;
    static constexpr int K = NT * C;
    static constexpr int NW = NT / 32;
    static constexpr unsigned FULL = 0xffffffffu;
    // Full unrolling keeps the state vectors in registers; beyond 32 states
    // the loops stay rolled (state vectors in local memory) to bound code size.
    static constexpr int UNR = (NB <= 5) ? NS : 1;
    using Sm = SweepSmem<NB, V, NT, C, JCAP, WITH_G>;

    int bit[C];     // bit of the point's marginal; -1 target; -2 padding
    int idx[C];     // index within the tile (forward order)
    V pp[C];        // position in the pass frame (units of eps)
    V fac[C][NB];   // injection factor per level (before the per-state ratios)
    V carry[NS];    // thread carries (f-representation), final levels only
    V run[NS];      // running local sums of the current walk
    const V *rrp;   // the tile's injection ratios (shared memory, [NS][NB])
    // for few states the ratios of a walk are held in registers
    static constexpr bool RREG = (NB <= 3);
    V rrr[RREG ? NS : 1][RREG ? NB : 1];

    __device__ __forceinline__ void load_ratios()
    {
        if constexpr (RREG) {
#pragma unroll
            for (int T = 0; T < NS; ++T)
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if ((T >> k) & 1) rrr[T][k] = rrp[T * NB + k];
        }
    }

    template <int T, int KB>
    __device__ __forceinline__ V ratio() const
    {
        if constexpr (RREG)
            return rrr[T][KB];
        else
            return rrp[T * NB + KB];
    }

    // rate w_s = s(l - s) with l = NB + 1
    __device__ static constexpr V rate(int s) { return (V)(s * (L - s)); }
    // provisional level shift of level s in a tile of the given span
    __device__ static V dshift(int s, V span)
    {
        const V as = rate(s) - rate(s - 1);
        return (as > V(0)) ? as * span : V(0);
    }

    __device__ void setup(Sm &sm, int n, V span, bool fwd, int j)
    {
        const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
        V lph[C];
        V dl[NB];
#pragma unroll
        for (int s = 0; s < NB; ++s) dl[s] = -INFINITY;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int r = tid * C + c;
            bit[c] = -2;
            idx[c] = 0;
            pp[c] = V(0);
            lph[c] = V(-INFINITY);
            if (r < n) {
                const int id = fwd ? r : n - 1 - r;
                const int m = sm.mid[id];
                idx[c] = id;
                bit[c] = (m == j) ? -1 : (m < j ? m : m - 1);
                pp[c] = fwd ? sm.pos[id] : span - sm.pos[id];
                lph[c] = sm.lphi[id];

            }
        }
        int msk = 0;
#pragma unroll
        for (int c = 0; c < C; ++c)
            if (bit[c] >= 0) msk |= 1 << bit[c];
        msk = __reduce_or_sync(FULL, msk);
        if (lane == 0 && msk) atomicOr(&sm.bits, msk);
        // Level shift D_s = max(0, a_s span): ln phi <= 0 inside a tile (the
        // baselines are the per-tile maxima) and 0 <= p <= span, so every
        // injection factor exp(ln phi + a_s p - D_s) is at most 1.
        (void)dl;
        (void)w;
        if (tid < NB) sm.D[tid] = Engine::dshift(tid + 1, span);
#pragma unroll
        for (int c = 0; c < C; ++c) {
#pragma unroll
            for (int s = 1; s <= NB; ++s) {
                const V ex = lph[c] + (rate(s) - rate(s - 1)) * pp[c] - dshift(s, span);
                fac[c][s - 1] = (bit[c] >= 0) ? vexp<V>(ex) : V(0);
            }
        }
#pragma unroll(UNR)
        for (int S = 0; S < NS; ++S) carry[S] = V(0);
        rrp = &sm.rr[0][0];
    }

    // F_T += phi * F_{T\k} at a point of bit k, in the f-representation of
    // each state: the factor is the point's level factor times the tile's
    // ratio of the two states' scales
    template <int SMAX, int KB>
    __device__ __forceinline__ void inject(int c)
    {
        if constexpr (RREG) {
            static_for<0, NS>([&](auto tc) {
                constexpr int T = decltype(tc)::value;
                if constexpr (((T >> KB) & 1) && popc_c(T) <= SMAX) {
                    constexpr int U = T ^ (1 << KB);
                    const V fu = (U == 0) ? V(1) : (carry[U] + run[U]);
                    run[T] = fma(fac[c][popc_c(T) - 1] * ratio<T, KB>(), fu, run[T]);
                }
            });
        } else {
#pragma unroll(UNR)
            for (int T = 0; T < NS; ++T) {
                if (((T >> KB) & 1) && popc_c(T) <= SMAX) {
                    const int U = T ^ (1 << KB);
                    const V fu = (U == 0) ? V(1) : (carry[U] + run[U]);
                    run[T] = fma(fac[c][popc_c(T) - 1] * rrp[T * NB + KB], fu, run[T]);
                }
            }
        }
    }

    template <int SMAX, int KB = 0>
    __device__ __forceinline__ void inject_dispatch(int k, int c)
    {
        if constexpr (KB < NB) {
            if (k == KB)
                inject<SMAX, KB>(c);
            else
                inject_dispatch<SMAX, KB + 1>(k, c);
        }
    }

    // Branch-free injection of point c (few states): every state T takes the
    // value of T\k for the point's bit k through a select, so the lanes of a
    // warp, whose points belong to different marginals, do not diverge.  A
    // state not containing k selects 0; T\k never contains k, so it is not
    // changed by this point and the in-place update is exact.
    template <int SMAX>
    __device__ __forceinline__ void inject_select(int c, int k)
    {
        V fu[NS];
        fu[0] = V(1);
        static_for<1, NS>([&](auto uc) {
            constexpr int U = decltype(uc)::value;
            if constexpr (popc_c(U) < SMAX) fu[U] = carry[U] + run[U];
        });
        static_for<1, NS>([&](auto tc) {
            constexpr int T = decltype(tc)::value;
            if constexpr (popc_c(T) <= SMAX) {
                V src = V(0);
                static_for<0, NB>([&](auto kc) {
                    constexpr int KB = decltype(kc)::value;
                    if constexpr ((T >> KB) & 1) {
                        constexpr int U = T ^ (1 << KB);
                        src = (k == KB) ? fu[U] * ratio<T, KB>() : src;
                    }
                });
                run[T] = fma(fac[c][popc_c(T) - 1], src, run[T]);
            }
        });
    }

    // Walk the chunk, recomputing levels 1..SMAX; on_target(c) is called at
    // target points with run[] holding the local sums before the point.
    template <int SMAX, typename OnT>
    __device__ __forceinline__ void walk(OnT &&on_target)
    {
        load_ratios();
#pragma unroll(UNR)
        for (int S = 0; S < NS; ++S) run[S] = V(0);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int k = bit[c];
            if constexpr (RREG) {
                inject_select<SMAX>(c, k);
                if (k == -1) on_target(c);
            } else {
                if (k >= 0)
                    inject_dispatch<SMAX>(k, c);
                else if (k == -1)
                    on_target(c);
            }
        }
    }

    // Walk the chunk calling on_point(c) at every injected point, before (PRE)
    // or after its injection.
    template <bool PRE, typename OnP>
    __device__ __forceinline__ void walk_each(OnP &&on_point)
    {
        load_ratios();
#pragma unroll(UNR)
        for (int S = 0; S < NS; ++S) run[S] = V(0);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int k = bit[c];
            if (k >= 0) {
                if constexpr (PRE) on_point(c);
                inject_dispatch<NB>(k, c);
                if constexpr (!PRE) on_point(c);
            }
        }
    }

    __device__ static double sum_beta(const Sm &sm, int S)
    {
        double b = 0.0;
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if ((S >> k) & 1) b += sm.beta[k];
        return b;
    }

    // Exclusive block scan of the level-s chunk totals (run[] after a walk);
    // block totals land in sm.tot.
    template <int s>
    __device__ void block_scan_level(Sm &sm, V (&excl)[NS])
    {
        const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
        for (int S = 0; S < NS; ++S) {
            if (popc_c(S) == s) {
                V incl = run[S];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const V y = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += y;
                }
                V ex = __shfl_up_sync(FULL, incl, 1);
                excl[S] = (lane == 0) ? V(0) : ex;
                if (lane == 31) sm.scan[w][S] = incl;
            }
        }
        __syncthreads();
        if (w == 0) {
#pragma unroll
            for (int S = 0; S < NS; ++S) {
                if (popc_c(S) == s) {
                    const V x = (lane < NW) ? sm.scan[lane][S] : V(0);
                    V incl = x;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const V y = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o) incl += y;
                    }
                    V ex = __shfl_up_sync(FULL, incl, 1);
                    if (lane == 0) ex = V(0);
                    if (lane < NW) sm.scan[lane][S] = ex;
                    if (lane == NW - 1) sm.tot[S] = incl;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int S = 0; S < NS; ++S)
            if (popc_c(S) == s) excl[S] += sm.scan[w][S];
    }

    // Look-back for level s (warp 0): publish the tile aggregate, combine the
    // predecessors' aggregates / inclusive prefixes into sm.E, publish the
    // inclusive prefix.  The 32 lanes inspect a window of 32 predecessors at
    // once; the window moves back until it holds an inclusive prefix.
    template <int s>
    __device__ void lookback(Sm &sm, const SweepArgs &a, int v, int b, bool fwd)
    {
        const int lane = threadIdx.x & 31;
        constexpr int NQ = (NS + 31) / 32;
        const double ws = (double)s * (double)(L - s);
        Sf<V> own[NQ], acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int S = lane + 32 * q;
            own[q] = sf_zero<V>();
            acc[q] = sf_zero<V>();
            if (S < NS && popc_c(S) == s) {
                own[q] = sf_scale_exp(sf_mul(sf_make<V>(sm.tot[S]), sm.Gs[S]), sum_beta(sm, S));
                sfp<V>(a.agg)[(size_t)v * NS + S] = sf_store(own[q]);
            }
        }
        int *myflag = a.flags + (size_t)v * (NB + 1) + s;
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(myflag, 1);
        bool fail = false;
        const double ub = fwd ? a.ulb[b] : a.urb[b];
        // lane i inspects predecessor base - i (flag and decay); the terms are
        // then gathered state-parallel: for each predecessor in the window every
        // lane adds the values of its own states (S = lane + 32q), so no
        // reduction across lanes is needed
        const int myseg = a.seg ? a.seg[b] : 0;
        int base = v - 1;
        while (base >= 0) {
            const int p = base - lane;
            // a predecessor of another instance contributes nothing and ends the window
            const bool other = (p >= 0) && a.seg && a.seg[fwd ? p : a.nt - 1 - p] != myseg;
            int f = (p >= 0 && !other) ? ld_acquire(a.flags + (size_t)p * (NB + 1) + s) : 2;
            unsigned incl;
            int it = 0;
            while (true) {
                incl = __ballot_sync(FULL, f >= 2);
                const int first = incl ? (__ffs(incl) - 1) : 31;
                const bool mine = lane <= first;
                if (!__ballot_sync(FULL, mine && f == 0)) break;
                if (++it > a.spin_limit || ((it & 63) == 0 && *(volatile const int *)a.err != 0)) {
                    fail = true;
                    break;
                }
                __nanosleep(32);
                if (mine && f == 0) f = ld_acquire(a.flags + (size_t)p * (NB + 1) + s);
            }
            if (fail) break;
            const int first = incl ? (__ffs(incl) - 1) : 31;
            if (__ballot_sync(FULL, lane <= first && f == 3)) {
                fail = true;
                break;
            }
            // decay exp(-w_s d) of this lane's predecessor as (fraction, power of two)
            V dm = V(0);
            int dk = INT_MIN / 2;
            if (p >= 0 && !other) {
                const int bp = fwd ? p : a.nt - 1 - p;
                const double d = fwd ? (ub - a.ulb[bp]) : (a.urb[bp] - ub);
                const double y = -ws * d * kLog2e;
                if (y >= -1.0e9) {
                    const double n = floor(y);
                    dm = vexp2<V>((V)(y - n));
                    dk = (int)n;
                }
            }
            for (int i = 0; i <= first; ++i) {
                const int pi = __shfl_sync(FULL, p, i);
                const int fi = __shfl_sync(FULL, f, i);
                const V dmi = __shfl_sync(FULL, dm, i);
                const int dki = __shfl_sync(FULL, dk, i);
                if (pi < 0 || dmi == V(0)) continue;   // none, another instance or no decay left
                const SfT<V> *src = sfp<V>((fi == 2) ? a.inc : a.agg) + (size_t)pi * NS;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const int S = lane + 32 * q;
                    if (S < NS && popc_c(S) == s) {
                        const Sf<V> raw = sf_load<V>(__ldcg(src + S));
                        if (raw.m != V(0)) {
                            Sf<V> t = sf_make<V>(raw.m * dmi);
                            t.k += raw.k + dki;
                            acc[q] = sf_add(acc[q], t);
                        }
                    }
                }
            }
            if (incl) break;
            base -= 32;
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int S = lane + 32 * q;
            if (S < NS && popc_c(S) == s) {
                sm.E[S] = acc[q];
                sm.Eh[S] = sf_scale_exp(acc[q], -sum_beta(sm, S));
                sfp<V>(a.inc)[(size_t)v * NS + S] = sf_store(sf_add(acc[q], own[q]));
            }
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            st_release(myflag, fail ? 3 : 2);
            if (fail) atomicOr(a.err, ERR_TIMEOUT);
        }
    }

    // Provisional scales of the states of level s (warp 0): the largest scale
    // of the states it is injected from, times exp(D_s), so every injection
    // ratio rr[T][k] = scale(T\k) exp(D_s) / scale(T) is at most 1.
    template <int s>
    __device__ void prepare(Sm &sm)
    {
        const int lane = threadIdx.x & 31;
        const Sf<V> eD = sf_make<V>(vexp<V>(sm.D[s - 1]));
        for (int T = lane; T < NS; T += 32) {
            if (popc_c(T) != s) continue;
            // only sources that inject in this tile (a point of bit k present)
            // choose the scale: the others would only push the real
            // contributions out of range
            Sf<V> mx = sf_zero<V>();
            for (int k = 0; k < NB; ++k) {
                if (!((T >> k) & 1) || !((sm.bits >> k) & 1)) continue;
                const Sf<V> u = sm.Gs[T ^ (1 << k)];
                if (mx.m == V(0) || u.k > mx.k || (u.k == mx.k && u.m > mx.m)) mx = u;
            }
            if (mx.m == V(0)) mx = Sf<V>{V(0.5), 1};   // no in-tile injection into T
            const Sf<V> GP = sf_mul(mx, eD);
            sm.Gs[T] = GP;
            for (int k = 0; k < NB; ++k) {
                V r = V(0);
                if (((T >> k) & 1) && ((sm.bits >> k) & 1)) {
                    const Sf<V> a = sf_mul(sm.Gs[T ^ (1 << k)], eD);
                    r = (a.m / GP.m) * pow2neg<V>(a.k - GP.k);
                }
                sm.rr[T][k] = r;
            }
        }
    }

    // Final scale of each state of level s (warp 0): the tile-end value
    // relative to exp(sum_{m in S} beta_m) is R_S = Eh_S + A_S scale_S, and the
    // new scale is 2^k with k its binary exponent, so every value of the state
    // becomes at most 1.  The carry turns into f-representation and the
    // injection ratios into the state follow the rescale.  Each state has its
    // own scale: states of one level may differ by far more than the FP32
    // range (sparse supports at small eps).
    template <int s>
    __device__ void normalise(Sm &sm)
    {
        const int lane = threadIdx.x & 31;
        for (int S = lane; S < NS; S += 32) {
            if (popc_c(S) != s) continue;
            const Sf<V> G = sm.Gs[S];
            const Sf<V> A = sf_make<V>(sm.tot[S]);
            const Sf<V> R = sf_add(sm.Eh[S], sf_mul(A, G));
            V tc = V(0), rho = V(0);
            if (R.m != V(0)) {
                tc = sf_value(sm.Eh[S], R.k);
                rho = (A.m == V(0)) ? V(0) : sf_value(G, R.k);
                if (!(rho <= std::numeric_limits<V>::max())) rho = V(0);
                sm.Gs[S] = Sf<V>{V(0.5), R.k + 1};
            }
            sm.tc[S] = tc;
            sm.rhoS[S] = rho;
            for (int k = 0; k < NB; ++k) sm.rr[S][k] *= rho;
        }
        if constexpr (s < NB) {
            __syncwarp();
            prepare<s + 1>(sm);
        }
    }

    // One level of the pass.  MAIN: carries by look-back; otherwise sm.E of
    // level s must already hold the known carries.
    template <int s, bool MAIN>
    __device__ void level(Sm &sm, const SweepArgs &a, int v, int b, bool fwd)
    {
        walk<s>([](int) {});
        V excl[NS];
        block_scan_level<s>(sm, excl);
        if (threadIdx.x < 32) {
            if constexpr (MAIN) lookback<s>(sm, a, v, b, fwd);
            __syncwarp();
            normalise<s>(sm);
        }
        __syncthreads();
#pragma unroll
        for (int S = 0; S < NS; ++S)
            if (popc_c(S) == s) carry[S] = sm.tc[S] + sm.rhoS[S] * excl[S];
    }

    // ---- carry-free transfer operator of the chunk ------------------------
    // op[s][U] (U non-empty, s + |U| <= NB): weight with which a state of
    // level s at the chunk start reaches the state with the marginals U added
    // at the chunk end, in the cumulative frame and f-representation of the
    // tile.  op[0][U] is the chunk's own contribution (from the empty state).
    // These are the paper's per-class nested sums (Sec. 4.2, J^{(l)} recursion)
    // grouped by starting level, so a tile can be summarised without its carry.
    __device__ static constexpr bool op_valid(int s, int U) { return U != 0 && s < NB && s + popc_c(U) <= NB; }

    template <int KB>
    __device__ __forceinline__ void op_inject(V (&op)[NB][NS], int c)
    {
#pragma unroll
        for (int s = 0; s < NB; ++s) {
#pragma unroll
            for (int U = 1; U < NS; ++U) {
                if (((U >> KB) & 1) && s + popc_c(U) <= NB) {
                    const int W = U ^ (1 << KB);
                    const V prev = (W == 0) ? V(1) : op[s][W];
                    op[s][U] = fma(fac[c][s + popc_c(U) - 1], prev, op[s][U]);
                }
            }
        }
    }

    template <int KB = 0>
    __device__ __forceinline__ void op_dispatch(V (&op)[NB][NS], int k, int c)
    {
        if constexpr (KB < NB) {
            if (k == KB)
                op_inject<KB>(op, c);
            else
                op_dispatch<KB + 1>(op, k, c);
        }
    }

    __device__ void op_walk(V (&op)[NB][NS])
    {
#pragma unroll
        for (int s = 0; s < NB; ++s)
#pragma unroll
            for (int U = 0; U < NS; ++U) op[s][U] = V(0);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int k = bit[c];
            if (k >= 0) op_dispatch(op, k, c);
        }
    }

    // R = X then Y (both in the same frame and representation)
    __device__ static void op_compose(const V (&X)[NB][NS], const V (&Y)[NB][NS], V (&R)[NB][NS])
    {
#pragma unroll
        for (int s = 0; s < NB; ++s) {
#pragma unroll
            for (int U = 1; U < NS; ++U) {
                if (s + popc_c(U) <= NB) {
                    V r = X[s][U] + Y[s][U];
#pragma unroll
                    for (int Vv = 1; Vv < NS; ++Vv) {
                        if ((Vv & ~U) == 0 && Vv != U) r = fma(X[s][Vv], Y[s + popc_c(Vv)][U ^ Vv], r);
                    }
                    R[s][U] = r;
                } else {
                    R[s][U] = V(0);
                }
            }
            R[s][0] = V(0);
        }
    }

    template <bool MAIN>
    __device__ void all_levels(Sm &sm, const SweepArgs &a, int v, int b, bool fwd)
    {
        __syncthreads();   // sm.bits complete (Engine::setup)
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) sm.Gs[0] = Sf<V>{V(0.5), 1};
            __syncwarp();
            prepare<1>(sm);
        }
        __syncthreads();
        static_for<1, NB + 1>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            level<s, MAIN>(sm, a, v, b, fwd);
        });
    }
};

// baselines of the marginals mapped to bits for target j
template <int NB, typename V, int NT, int C, int JCAP, bool WITH_G>
__device__ void load_betas(SweepSmem<NB, V, NT, C, JCAP, WITH_G> &sm, const SweepArgs &a, int b, int j)
{
    if (threadIdx.x < NB) {
        const int k = threadIdx.x;
        const int m = (k < j) ? k : k + 1;
        const int rt = __ldg(a.reftile + (size_t)b * a.l + m);
        sm.beta[k] = *(volatile const double *)(a.beta + (size_t)rt * a.l + m);
    }
}

template <int NB, typename V, int NT, int C, int JCAP, bool WITH_G>
__device__ void load_tile(SweepSmem<NB, V, NT, C, JCAP, WITH_G> &sm, const SweepArgs &a, int b,
                          int n, uint32_t t0, int j)
{
    const V *pos = static_cast<const V *>(a.pos);
    const V *lphi = static_cast<const V *>(a.lphi);
    for (int i = threadIdx.x; i < n; i += NT) {
        sm.pos[i] = __ldg(pos + t0 + i);
        sm.lphi[i] = lphi[t0 + i];
        sm.mid[i] = __ldg(a.mid + t0 + i);
    }
    load_betas(sm, a, b, j);
    if (threadIdx.x == 0) sm.bits = 0;
    __syncthreads();
}

// Tiles of a frozen (converged) instance of a batch do no update or residual
// work; their residual term is 0.
__device__ __forceinline__ bool skip_tile(const SweepArgs &a, int b)
{
    if (!a.frozen || (a.mode != MODE_UPDATE && a.mode != MODE_RESIDUAL)) return false;
    if (!a.frozen[a.seg[b]]) return false;
    if (a.mode == MODE_RESIDUAL && threadIdx.x == 0) a.partial[b] = 0.0;
    return true;
}

template <int NB, typename V, int NT, int C, int JCAP, int L = NB + 1>
__global__ void __launch_bounds__(NT, 3) k_bwd(SweepArgs a)
{
    using Sm = SweepSmem<NB, V, NT, C, JCAP, false>;
    using En = Engine<NB, V, NT, C, JCAP, false, L>;
    constexpr int NS = 1 << NB;
    extern __shared__ __align__(16) unsigned char smraw[];
    Sm &sm = *reinterpret_cast<Sm *>(smraw);
    __shared__ int s_v;
    if (threadIdx.x == 0) s_v = atomicAdd(a.counter, 1);
    __syncthreads();
    const int v = s_v;
    if (v >= a.nt) return;
    const int b = a.nt - 1 - v;
    if (skip_tile(a, b)) return;
    const uint32_t t0 = a.tstart[b];
    const int n = (int)(a.tstart[b + 1] - t0);
    load_tile<NB, V, NT, C, JCAP, false>(sm, a, b, n, t0, a.j);
    En e;
    e.setup(sm, n, (V)a.span[b], false, a.j);
    e.template all_levels<true>(sm, a, v, b, false);
    for (int S = threadIdx.x; S < NS; S += NT)
        sfp<V>(a.bcarry)[(size_t)b * NS + S] = (S == 0) ? sf_one_st<V>() : sf_store(sm.E[S]);
}

// Carry-free transfer operator of tile b for target j in one direction,
// stored as scaled floats with the decay to the next tile base (processing
// order) included:
//   op[b][s][U] = T_b[s][U] exp(sum_{m in U} beta_m + gamma_{s+|U|} - gamma_s - w_{s+|U|} d)
// where T_b is the composition of the thread operators (tile frame and
// f-representation, provisional level scales gamma) and d the distance from
// this tile's base to the next one, in units of eps.
template <int NB, typename V, int NT, int C, int JCAP, int L = NB + 1>
__device__ void tile_operator(SweepSmem<NB, V, NT, C, JCAP, true> &sm, const SweepArgs &a, int b, int n,
                              int j, bool fwd)
{
    using En = Engine<NB, V, NT, C, JCAP, true, L>;
    constexpr int NS = 1 << NB;
    static_assert(NB * NS * (NT / 32) <= SweepSmem<NB, V, NT, C, JCAP, true>::GSZ, "operator scratch");
    const int tid = threadIdx.x;
    En e;
    e.setup(sm, n, (V)a.span[b], fwd, j);
    V op[NB][NS];
    e.op_walk(op);
    // composition in processing order (thread order is processing order in
    // both directions, see Engine::setup): a shuffle tree inside each warp,
    // then the warp results in order by warp 0
    constexpr int NW = NT / 32;
    const int lane = tid & 31, w = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        V Y[NB][NS], R[NB][NS];
#pragma unroll
        for (int s = 0; s < NB; ++s)
#pragma unroll
            for (int U = 0; U < NS; ++U)
                Y[s][U] = En::op_valid(s, U) ? __shfl_down_sync(0xffffffffu, op[s][U], o) : V(0);
        En::op_compose(op, Y, R);
        if ((lane & (2 * o - 1)) == 0) {
#pragma unroll
            for (int s = 0; s < NB; ++s)
#pragma unroll
                for (int U = 0; U < NS; ++U) op[s][U] = R[s][U];
        }
    }
    V *scr = sm.G;   // [NW][NB][NS]
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < NB; ++s)
#pragma unroll
            for (int U = 0; U < NS; ++U) scr[(w * NB + s) * NS + U] = op[s][U];
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NB; ++s)
#pragma unroll
            for (int U = 0; U < NS; ++U) op[s][U] = scr[s * NS + U];
        for (int q = 1; q < NW; ++q) {
            V Y[NB][NS], R[NB][NS];
#pragma unroll
            for (int s = 0; s < NB; ++s)
#pragma unroll
                for (int U = 0; U < NS; ++U) Y[s][U] = scr[(q * NB + s) * NS + U];
            En::op_compose(op, Y, R);
#pragma unroll
            for (int s = 0; s < NB; ++s)
#pragma unroll
                for (int U = 0; U < NS; ++U) op[s][U] = R[s][U];
        }
#pragma unroll
        for (int s = 0; s < NB; ++s)
#pragma unroll
            for (int U = 0; U < NS; ++U) scr[s * NS + U] = op[s][U];
    }
    __syncthreads();
    // absolute scaled floats with the decay to the next base
    double d = 0.0;
    bool cut = false;   // the next tile belongs to another instance of a batch
    if (fwd) {
        if (b + 1 < a.nt) {
            d = a.ulb[b + 1] - a.ulb[b];
            cut = a.seg && a.seg[b + 1] != a.seg[b];
        }
    } else {
        if (b >= 1) {
            d = a.urb[b] - a.urb[b - 1];
            cut = a.seg && a.seg[b - 1] != a.seg[b];
        }
    }
    SfT<V> *dst = sfp<V>(fwd ? a.opF : a.opB) + (size_t)b * NB * NS;
    for (int idx = tid; idx < NB * NS; idx += NT) {
        const int s = idx / NS, U = idx % NS;
        if (!En::op_valid(s, U)) continue;
        const int su = s + popc_c(U);
        double gs = 0.0, gsu = 0.0, bu = 0.0;
        for (int q = 0; q < su; ++q) {
            if (q < s) gs += (double)sm.D[q];
            gsu += (double)sm.D[q];
        }
        for (int k = 0; k < NB; ++k)
            if ((U >> k) & 1) bu += sm.beta[k];
        const double wsu = (double)su * (double)(L - su);
        const V val = scr[s * NS + U];
        dst[idx] = cut ? sf_store(sf_zero<V>()) : sf_store(sf_scale_exp(sf_make<V>(val), bu + gsu - gs - wsu * d));
    }
    __syncthreads();
}

template <int NB, typename V, int NT, int C, int JCAP, int L = NB + 1>
__global__ void __launch_bounds__(NT, 3) k_tileop(SweepArgs a)
{
    using Sm = SweepSmem<NB, V, NT, C, JCAP, true>;
    extern __shared__ __align__(16) unsigned char smraw[];
    Sm &sm = *reinterpret_cast<Sm *>(smraw);
    const int b = blockIdx.x;
    const uint32_t t0 = a.tstart[b];
    const int n = (int)(a.tstart[b + 1] - t0);
    load_tile<NB, V, NT, C, JCAP, true>(sm, a, b, n, t0, a.j);
    tile_operator<NB, V, NT, C, JCAP, L>(sm, a, b, n, a.j, true);
    tile_operator<NB, V, NT, C, JCAP, L>(sm, a, b, n, a.j, false);
}

// ---- level passes (many state bits) -----------------------------------------
// For l >= 6 the carries of level s are computed in one pass per level and
// direction: every tile evaluates its own contribution to the states of level
// s at its base, given the (already known) carries of the lower levels
// (k_wpass, warp.cuh), and one scalar affine scan per state over the tiles
// turns those contributions into every tile's carry (k_lscan):
//   E_T(next base) = exp(-w_s d) (E_T + own_T).
// No tile waits on another tile; the scans wait only on earlier chunks.
// Scalar carry scan of one state of level SL over the tiles (processing
// order): blockIdx.y picks the state, blockIdx.x the chunk of tiles.  Each
// thread composes the maps x -> dec (x + own) of its tiles, the block scans
// them, the chunk publishes its contribution at the next chunk's base and
// adds those of the earlier chunks (same instance only; bounded waits).
template <int NB, typename V, int LM = NB + 1>
__global__ void __launch_bounds__(256) k_lscan(SweepArgs a, int SL, int fwd_i)
{
    constexpr int NS = 1 << NB;
    constexpr int NTB = 256;
    constexpr int NWB = NTB / 32;
    constexpr unsigned FULL = 0xffffffffu;
    const bool fwd = (fwd_i != 0);
    const int G = gridDim.x, c = blockIdx.x;
    // the state of level SL this block scans
    int T = 0;
    for (int S = 1, q = 0; S < NS; ++S) {
        if (popc_c(S) != SL) continue;
        if (q == (int)blockIdx.y) {
            T = S;
            break;
        }
        ++q;
    }
    const SfT<V> *own = sfp<V>(a.agg);   // written in pass 1 of a two-level scan
    const SfT<V> *__restrict__ pdec = sfp<V>(fwd ? a.pdecF : a.pdecB);
    SfT<V> *E = sfp<V>(fwd ? a.fcarry : a.bcarry);
    const int slot = ((fwd ? 0 : 1) * NS + T) * 32;
    SfT<V> *cagg = sfp<V>(a.cagg) + slot;
    int *cflag = a.cflags + slot;
    const int nt = a.nt, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int Rc = (nt + G - 1) / G;
    const int cv0 = min(nt, c * Rc), cv1 = min(nt, cv0 + Rc);
    const int R = (cv1 - cv0 + NTB - 1) / NTB;
    const int v0 = min(cv1, cv0 + tid * R), v1 = min(cv1, v0 + R);
    auto tile_of = [&](int v) { return fwd ? v : nt - 1 - v; };
    auto chunk_base = [&](int q) -> double {
        const int v = min(nt - 1, q * Rc);
        return fwd ? a.ulb[tile_of(v)] : a.urb[tile_of(v)];
    };
    __shared__ V s_am[NWB], s_bm[NWB];
    __shared__ int s_ak[NWB], s_bk[NWB];
    __shared__ V s_em;
    __shared__ int s_ek;
    // pass 1: this thread's map x -> am x + bb (the second level of a
    // two-level pass first adds the share of the previous level's carries,
    // E[T \ m] coef[m], to the stored contribution)
    Sf<V> am = Sf<V>{V(0.5), 1}, bb = sf_zero<V>();
    for (int v = v0; v < v1; ++v) {
        const int b = tile_of(v);
        const Sf<V> dec = sf_load<V>(__ldg(pdec + (size_t)b * (NB + 1) + SL));
        Sf<V> o = sf_load<V>(__ldcg(own + (size_t)b * NS + T));
        if (a.pair) {
#pragma unroll
            for (int m = 0; m < NB; ++m) {
                if (!((T >> m) & 1)) continue;
                const Sf<V> eu = sf_load<V>(__ldcg(E + (size_t)b * NS + (T ^ (1 << m))));
                if (eu.m != V(0)) o = sf_add(o, sf_mul(eu, sf_load<V>(__ldcg(sfp<V>(a.coef) + (size_t)b * NB + m))));
            }
            sfp<V>(a.agg)[(size_t)b * NS + T] = sf_store(o);   // read again by pass 2
        }
        bb = sf_mul(sf_add(bb, o), dec);
        am = sf_mul(am, dec);
    }
    // inclusive scan of the maps across the warp, then across warps
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Sf<V> oa, ob;
        oa.m = __shfl_up_sync(FULL, am.m, o);
        oa.k = __shfl_up_sync(FULL, am.k, o);
        ob.m = __shfl_up_sync(FULL, bb.m, o);
        ob.k = __shfl_up_sync(FULL, bb.k, o);
        if (lane >= o) {
            bb = sf_add(sf_mul(ob, am), bb);
            am = sf_mul(oa, am);
        }
    }
    if (lane == 31) {
        s_am[w] = am.m;
        s_ak[w] = am.k;
        s_bm[w] = bb.m;
        s_bk[w] = bb.k;
    }
    Sf<V> exa, exb;
    exa.m = __shfl_up_sync(FULL, am.m, 1);
    exa.k = __shfl_up_sync(FULL, am.k, 1);
    exb.m = __shfl_up_sync(FULL, bb.m, 1);
    exb.k = __shfl_up_sync(FULL, bb.k, 1);
    if (lane == 0) {
        exa = Sf<V>{V(0.5), 1};
        exb = sf_zero<V>();
    }
    __syncthreads();
    if (w == 0) {
        Sf<V> wa = (lane < NWB) ? Sf<V>{s_am[lane], s_ak[lane]} : Sf<V>{V(0.5), 1};
        Sf<V> wb = (lane < NWB) ? Sf<V>{s_bm[lane], s_bk[lane]} : sf_zero<V>();
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Sf<V> oa, ob;
            oa.m = __shfl_up_sync(FULL, wa.m, o);
            oa.k = __shfl_up_sync(FULL, wa.k, o);
            ob.m = __shfl_up_sync(FULL, wb.m, o);
            ob.k = __shfl_up_sync(FULL, wb.k, o);
            if (lane >= o) {
                wb = sf_add(sf_mul(ob, wa), wb);
                wa = sf_mul(oa, wa);
            }
        }
        Sf<V> tot;
        tot.m = __shfl_sync(FULL, wb.m, NWB - 1);
        tot.k = __shfl_sync(FULL, wb.k, NWB - 1);
        if (lane == 0) cagg[c] = sf_store(tot);
        // exclusive warp prefixes (maps of the warps before)
        Sf<V> pa, pb;
        pa.m = __shfl_up_sync(FULL, wa.m, 1);
        pa.k = __shfl_up_sync(FULL, wa.k, 1);
        pb.m = __shfl_up_sync(FULL, wb.m, 1);
        pb.k = __shfl_up_sync(FULL, wb.k, 1);
        if (lane == 0) {
            pa = Sf<V>{V(0.5), 1};
            pb = sf_zero<V>();
        }
        __syncwarp();
        if (lane < NWB) {
            s_am[lane] = pa.m;
            s_ak[lane] = pa.k;
            s_bm[lane] = pb.m;
            s_bk[lane] = pb.k;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0 && !(a.hold && c == 0)) st_release(cflag + c, 1);
        // carry into this chunk: contributions of the earlier chunks of the same instance
        const double ws = (double)(SL * (LM - SL));
        const double ub = chunk_base(c);
        Sf<V> part = sf_zero<V>();
        bool fail = false;
        for (int p = lane; p < c; p += 32) {
            const bool same = !a.seg || a.seg[tile_of(min(nt - 1, (p + 1) * Rc))] == a.seg[tile_of(min(nt - 1, c * Rc))];
            if (!same) continue;
            const int f = wait_flag(cflag + p, a.err, a.spin_limit);
            if (f < 0) {
                fail = true;
                continue;
            }
            const double d = fabs(ub - chunk_base(p + 1));
            part = sf_add(part, sf_scale_exp(sf_load<V>(__ldcg(cagg + p)), -ws * d));
        }
        if (__ballot_sync(FULL, fail) && lane == 0) atomicOr(a.err, ERR_TIMEOUT);
        const Sf<V> t = sf_warp_sum(part);
        if (lane == 0) {
            s_em = t.m;
            s_ek = t.k;
        }
    }
    __syncthreads();
    // this thread's incoming carry: chunk carry through the maps before it
    const Sf<V> wpa = Sf<V>{s_am[w], s_ak[w]}, wpb = Sf<V>{s_bm[w], s_bk[w]};
    const Sf<V> chunkin = Sf<V>{s_em, s_ek};
    Sf<V> cur = sf_add(sf_mul(sf_add(sf_mul(wpa, chunkin), wpb), exa), exb);
    // pass 2: apply
    for (int v = v0; v < v1; ++v) {
        const int b = tile_of(v);
        E[(size_t)b * NS + T] = sf_store(cur);
        const Sf<V> dec = sf_load<V>(__ldg(pdec + (size_t)b * (NB + 1) + SL));
        const Sf<V> o = sf_load<V>(__ldcg(own + (size_t)b * NS + T));
        cur = sf_mul(sf_add(cur, o), dec);
    }
}

// Exclusive carries of every tile from the tile operators.  For level s each
// state is an affine recurrence over the tiles in processing order,
//   E_T(next) = exp(-w_s d) E_T + sum_{S strictly inside T} E_S op[|S|][T\S]
// (E_empty = 1).  Grid: G co-resident blocks per direction (blockIdx.y), each
// owning a contiguous chunk of tiles; per level a block composes its chunk's
// maps (block scan), publishes the chunk's contribution at the next chunk's
// base, adds the contributions of all earlier chunks (at most 31, one warp
// window, decays from the tile positions) and applies the result to its
// tiles.  Waits are bounded; on timeout the error word is set.
template <int NB, typename V, int RM, int L = NB + 1>
__global__ void __launch_bounds__(256) k_carry(SweepArgs a)
{
    constexpr int NS = 1 << NB;
    constexpr int NTB = 256;
    constexpr int NWB = NTB / 32;
    constexpr unsigned FULL = 0xffffffffu;
    const bool fwd = (blockIdx.y == 0);
    const int G = gridDim.x, c = blockIdx.x;
    const SfT<V> *__restrict__ op = sfp<V>(fwd ? a.opF : a.opB);
    const SfT<V> *__restrict__ pdec = sfp<V>(fwd ? a.pdecF : a.pdecB);
    SfT<V> *E = sfp<V>(fwd ? a.fcarry : a.bcarry);
    SfT<V> *cagg = sfp<V>(a.cagg) + (size_t)blockIdx.y * G * NS;
    int *cflag = a.cflags + (size_t)blockIdx.y * G * (NB + 1);
    const int nt = a.nt, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int Rc = (nt + G - 1) / G;                  // tiles per chunk
    const int cv0 = min(nt, c * Rc), cv1 = min(nt, cv0 + Rc);
    const int R = (cv1 - cv0 + NTB - 1) / NTB;        // tiles per thread (<= RM)
    const int v0 = min(cv1, cv0 + tid * R), v1 = min(cv1, v0 + R);
    auto tile_of = [&](int v) { return fwd ? v : nt - 1 - v; };
    // base position of chunk q in processing order (units of eps)
    auto chunk_base = [&](int q) -> double {
        const int v = min(nt - 1, q * Rc);
        return fwd ? a.ulb[tile_of(v)] : a.urb[tile_of(v)];
    };
    __shared__ V s_am[NWB];
    __shared__ int s_ak[NWB];
    __shared__ V s_m[NWB][NS];
    __shared__ int s_k[NWB][NS];
    __shared__ V s_em[NS];
    __shared__ int s_ek[NS];
    for (int v = v0; v < v1; ++v) E[(size_t)tile_of(v) * NS] = sf_one_st<V>();
    static_for<1, NB + 1>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        __syncthreads();
        // pass 1: offsets and decays of this thread's tiles (loads only)
        Sf<V> off[RM][NS];
        Sf<V> dec[RM];
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            const int v = v0 + r;
            const bool ok = v < v1;
            const int b = ok ? tile_of(v) : 0;
            dec[r] = ok ? sf_load<V>(__ldg(pdec + (size_t)b * (NB + 1) + s)) : sf_zero<V>();
            Sf<V> Elow[NS];
#pragma unroll
            for (int S = 1; S < NS; ++S)
                Elow[S] = (ok && popc_c(S) < s) ? sf_load<V>(__ldcg(E + (size_t)b * NS + S)) : sf_zero<V>();
#pragma unroll
            for (int T = 1; T < NS; ++T) {
                if (popc_c(T) == s) {
                    Sf<V> acc = ok ? sf_load<V>(__ldg(op + ((size_t)b * NB + 0) * NS + T)) : sf_zero<V>();
#pragma unroll
                    for (int S = 1; S < NS; ++S) {
                        if ((S & ~T) == 0 && S != T) {
                            const Sf<V> o = ok ? sf_load<V>(__ldg(op + ((size_t)b * NB + popc_c(S)) * NS + (T ^ S)))
                                               : sf_zero<V>();
                            acc = sf_add(acc, sf_mul(Elow[S], o));
                        }
                    }
                    off[r][T] = acc;
                }
            }
        }
        // composition of the thread's maps: x -> am x + bb
        Sf<V> am = Sf<V>{V(0.5), 1};
        Sf<V> bb[NS];
#pragma unroll
        for (int T = 0; T < NS; ++T) bb[T] = sf_zero<V>();
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            if (v0 + r < v1) {
#pragma unroll
                for (int T = 1; T < NS; ++T)
                    if (popc_c(T) == s) bb[T] = sf_add(sf_mul(bb[T], dec[r]), off[r][T]);
                am = sf_mul(am, dec[r]);
            }
        }
        // block scan of the maps (inclusive in the warp, then across warps)
#pragma unroll 1
        for (int o = 1; o < 32; o <<= 1) {
            Sf<V> oa;
            oa.m = __shfl_up_sync(FULL, am.m, o);
            oa.k = __shfl_up_sync(FULL, am.k, o);
#pragma unroll
            for (int T = 1; T < NS; ++T) {
                if (popc_c(T) == s) {
                    Sf<V> ob;
                    ob.m = __shfl_up_sync(FULL, bb[T].m, o);
                    ob.k = __shfl_up_sync(FULL, bb[T].k, o);
                    if (lane >= o) bb[T] = sf_add(sf_mul(ob, am), bb[T]);
                }
            }
            if (lane >= o) am = sf_mul(oa, am);
        }
        if (lane == 31) {
            s_am[w] = am.m;
            s_ak[w] = am.k;
#pragma unroll
            for (int T = 1; T < NS; ++T)
                if (popc_c(T) == s) {
                    s_m[w][T] = bb[T].m;
                    s_k[w][T] = bb[T].k;
                }
        }
        Sf<V> exa;
        exa.m = __shfl_up_sync(FULL, am.m, 1);
        exa.k = __shfl_up_sync(FULL, am.k, 1);
        if (lane == 0) exa = Sf<V>{V(0.5), 1};
        Sf<V> exb[NS];
#pragma unroll
        for (int T = 1; T < NS; ++T) {
            if (popc_c(T) == s) {
                exb[T].m = __shfl_up_sync(FULL, bb[T].m, 1);
                exb[T].k = __shfl_up_sync(FULL, bb[T].k, 1);
                if (lane == 0) exb[T] = sf_zero<V>();
            }
        }
        __syncthreads();
        if (w == 0) {
            // warp prefixes (lanes < NWB) and the chunk total
            Sf<V> wa = (lane < NWB) ? Sf<V>{s_am[lane], s_ak[lane]} : Sf<V>{V(0.5), 1};
            Sf<V> wb[NS];
#pragma unroll
            for (int T = 1; T < NS; ++T)
                if (popc_c(T) == s) wb[T] = (lane < NWB) ? Sf<V>{s_m[lane][T], s_k[lane][T]} : sf_zero<V>();
#pragma unroll 1
            for (int o = 1; o < 32; o <<= 1) {
                Sf<V> oa;
                oa.m = __shfl_up_sync(FULL, wa.m, o);
                oa.k = __shfl_up_sync(FULL, wa.k, o);
#pragma unroll
                for (int T = 1; T < NS; ++T) {
                    if (popc_c(T) == s) {
                        Sf<V> ob;
                        ob.m = __shfl_up_sync(FULL, wb[T].m, o);
                        ob.k = __shfl_up_sync(FULL, wb[T].k, o);
                        if (lane >= o) wb[T] = sf_add(sf_mul(ob, wa), wb[T]);
                    }
                }
                if (lane >= o) wa = sf_mul(oa, wa);
            }
            // publish the chunk's contribution at the next chunk's base
            int *myflag = cflag + (size_t)c * (NB + 1) + s;
#pragma unroll
            for (int T = 1; T < NS; ++T) {
                if (popc_c(T) == s) {
                    Sf<V> tot;
                    tot.m = __shfl_sync(FULL, wb[T].m, NWB - 1);
                    tot.k = __shfl_sync(FULL, wb[T].k, NWB - 1);
                    if (lane == 0) cagg[(size_t)c * NS + T] = sf_store(tot);
                    Sf<V> pb;
                    pb.m = __shfl_up_sync(FULL, wb[T].m, 1);
                    pb.k = __shfl_up_sync(FULL, wb[T].k, 1);
                    if (lane == 0) pb = sf_zero<V>();
                    if (lane < NWB) {
                        s_m[lane][T] = pb.m;
                        s_k[lane][T] = pb.k;
                    }
                }
            }
            __threadfence();
            __syncwarp();
            if (lane == 0 && !(a.hold && c == 0)) st_release(myflag, 1);
            // carry into this chunk: contributions of all earlier chunks
            const double ws = (double)(s * (L - s));
            const double ub = chunk_base(c);
            bool fail = false;
            Sf<V> part[NS];
#pragma unroll
            for (int T = 0; T < NS; ++T) part[T] = sf_zero<V>();
            // chunk p's contribution reaches this chunk only inside one instance
            const bool same = !a.seg || a.seg[tile_of(min(nt - 1, (lane + 1) * Rc))] == a.seg[tile_of(min(nt - 1, c * Rc))];
            if (lane < c && same) {
                const int p = lane;
                const int f = wait_flag(cflag + (size_t)p * (NB + 1) + s, a.err, a.spin_limit);
                if (f < 0) {
                    fail = true;
                } else {
                    const double d = fabs(ub - chunk_base(p + 1));
#pragma unroll
                    for (int T = 1; T < NS; ++T)
                        if (popc_c(T) == s)
                            part[T] = sf_scale_exp(sf_load<V>(__ldcg(cagg + (size_t)p * NS + T)), -ws * d);
                }
            }
            if (__ballot_sync(FULL, fail)) {
                if (lane == 0) atomicOr(a.err, ERR_TIMEOUT);
            }
            // states entering the range (shards): at the first tile's base
            if (a.inflow && lane == 0) {
                const double d0 = fabs(ub - chunk_base(0));
#pragma unroll
                for (int T = 1; T < NS; ++T)
                    if (popc_c(T) == s)
                        part[T] = sf_add(part[T], sf_scale_exp(sf_load<V>(sfp<V>(a.inflow)[(fwd ? 0 : 1) * NS + T]),
                                                               -ws * d0));
            }
#pragma unroll
            for (int T = 1; T < NS; ++T) {
                if (popc_c(T) == s) {
                    const Sf<V> t = sf_warp_sum_rolled(part[T]);
                    if (lane == 0) {
                        s_em[T] = t.m;
                        s_ek[T] = t.k;
                    }
                }
            }
        }
        __syncthreads();
        // this thread's carry: chunk carry through the warp prefix and the lane prefix
        Sf<V> cur[NS];
#pragma unroll
        for (int T = 1; T < NS; ++T) {
            if (popc_c(T) == s) {
                // maps before this thread: warp prefix (s_am of warps before, stored as
                // exclusive offsets in s_m/s_k) and the in-warp exclusive (exa, exb)
                Sf<V> m = Sf<V>{V(0.5), 1};
                for (int q = 0; q < w; ++q) m = sf_mul(m, Sf<V>{s_am[q], s_ak[q]});
                const Sf<V> chunkin = sf_mul(Sf<V>{s_em[T], s_ek[T]}, sf_mul(m, exa));
                const Sf<V> pre = sf_add(sf_mul(Sf<V>{s_m[w][T], s_k[w][T]}, exa), exb[T]);
                cur[T] = sf_add(chunkin, pre);
            }
        }
        // pass 2: apply (stores only)
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            const int v = v0 + r;
            if (v < v1) {
                const int b = tile_of(v);
#pragma unroll
                for (int T = 1; T < NS; ++T) {
                    if (popc_c(T) == s) {
                        E[(size_t)b * NS + T] = sf_store(cur[T]);
                        cur[T] = sf_add(sf_mul(cur[T], dec[r]), off[r][T]);
                    }
                }
            }
        }
        __threadfence_block();
    });
}

template <int NB, typename V, int NT, int C, int JCAP, int L = NB + 1>
cudaError_t launch_tileop_impl(const SweepArgs &a, cudaStream_t st)
{
    using Sm = SweepSmem<NB, V, NT, C, JCAP, true>;
    auto kern = k_tileop<NB, V, NT, C, JCAP, L>;
    const size_t sz = sizeof(Sm);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz);
    if (e != cudaSuccess) return e;
    kern<<<a.nt, NT, sz, st>>>(a);
    return cudaGetLastError();
}

// chunks per direction (co-resident: 2 * G blocks)
inline int carry_chunks(int nt) { return nt < 32 ? (nt > 0 ? nt : 1) : 32; }

template <int NB, typename V, int L = NB + 1>
cudaError_t launch_carry_impl(const SweepArgs &a, cudaStream_t st)
{
    const int G = carry_chunks(a.nt);
    const int Rc = (a.nt + G - 1) / G;
    const int R = (Rc + 255) / 256;
    const dim3 grid(G, 2);
    if (R <= 1)
        k_carry<NB, V, 1, L><<<grid, 256, 0, st>>>(a);
    else if (R <= 2)
        k_carry<NB, V, 2, L><<<grid, 256, 0, st>>>(a);
    else if (R <= 4)
        k_carry<NB, V, 4, L><<<grid, 256, 0, st>>>(a);
    else if (R <= 8)
        k_carry<NB, V, 8, L><<<grid, 256, 0, st>>>(a);
    else
        return cudaErrorInvalidConfiguration;   // more than 65536 tiles
    return cudaGetLastError();
}

// chunks of a level scan: at most 256 co-resident blocks over the level's states
inline int lscan_chunks(int nt, int nstates)
{
    int G = 256 / (nstates > 0 ? nstates : 1);
    G = G < 1 ? 1 : (G > 32 ? 32 : G);
    return nt < G ? (nt > 0 ? nt : 1) : G;
}

template <int NB, typename V>
cudaError_t launch_lscan_impl(const SweepArgs &a, cudaStream_t st, int SL, int fwd)
{
    int nst = 0;
    for (int S = 1; S < (1 << NB); ++S)
        if (popc_c(S) == SL) ++nst;
    const dim3 grid(lscan_chunks(a.nt, nst), nst);
    k_lscan<NB, V><<<grid, 256, 0, st>>>(a, SL, fwd);
    return cudaGetLastError();
}

template <int NB, typename V, int NT, int C, int JCAP, int L = NB + 1>
cudaError_t launch_bwd_impl(const SweepArgs &a, cudaStream_t st)
{
    using Sm = SweepSmem<NB, V, NT, C, JCAP, false>;
    auto kern = k_bwd<NB, V, NT, C, JCAP, L>;
    const size_t sz = sizeof(Sm);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz);
    if (e != cudaSuccess) return e;
    kern<<<a.nt, NT, sz, st>>>(a);
    return cudaGetLastError();
}



}  // namespace mmot

// Sweep kernels: the marginal product M_j of l-marginal Sinkhorn with L1 cost
// (arXiv 2405.19246, Sec. 3 and Sec. 4.2) as a level-pipelined, decoupled
// look-back scan over tiles of the merged support order.
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
// multipliers moved into the frame.  Level s = |T| depends on level s-1 at the
// same point, so the scan runs level by level: for s = 1..l-1 each tile
//   1. walks its points (each thread a contiguous chunk) recomputing levels
//      1..s from the final lower-level carries,
//   2. block-scans the level-s chunk totals,
//   3. publishes its level-s aggregate (FP64 log domain) and looks back over
//      the preceding tiles for its exclusive carry (decoupled look-back over
//      the associative pairs (decay, offset); the decay of level s over a
//      distance d is exp(-w_s d/eps), the same for every state of the level),
//   4. renormalises level s so that its largest tile-end value is 1.
// Values inside a tile are FP32 (or FP64) "f-representations"
//     f_S = F~_S exp(-sum_{m in S} beta_m - gamma_{|S|})
// with per-tile FP64 baselines beta_m (from the potentials; the re-centring of
// Algorithm 5) and per-level scales gamma_s.  Carries between tiles are FP64
// logarithms.
//
// The backward states G are the mirror image.  k_bwd runs the backward scan
// and stores each tile's backward carry; k_fwd recomputes the tile's backward
// states from that carry (no look-back), keeps them at the target points in
// shared memory, runs the forward scan with look-back and combines
//     M_j(i) = sum_S F_S(x_i^-) G_{R\S}(x_i^+)
// at the target points, then applies the FP64 epilogue (potential update
// g_j = eps (ln mu_j - ln M_j), or an output mode).
#pragma once
#include <cmath>
#include <cstdint>
#include <type_traits>

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

__device__ __forceinline__ double lae(double a, double b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    const double m = fmax(a, b);
    return m + log1p(exp(fmin(a, b) - m));
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
    double E[NS];          // FP64 log carry of each state at the tile base
    double gam[NB + 1];    // level scales of the current pass
    double gamG[NB + 1];   // level scales of the backward pass (k_fwd)
    double beta[NB];       // baselines of the marginals mapped to bits
    double dred[NW];       // FP64 reduction scratch
    V scan[NW][NS];        // warp totals / warp prefixes
    V tot[NS];             // block totals of the current level
    V tc[NS];              // tile carries in f-representation
    V rho;                 // rescale factor of the current level
    V D[NB];               // provisional level scales
    V fred[NW][NB];        // reduction scratch
    int ired[NW];
    int ntarget;
    V pos[K];
    V lphi[K];
    int16_t slot[K];
    uint8_t mid[K];
    V G[WITH_G ? NS * JCAP : 1];  // backward states at target points
};

// Per-thread engine: a contiguous chunk of C points of the tile, in the
// processing order of the pass (forward: increasing x, backward: decreasing).
template <int NB, typename V, int NT, int C, int JCAP, bool WITH_G>
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
    V fac[C][NB];   // injection factor per level
    V carry[NS];    // thread carries (f-representation), final levels only
    V run[NS];      // running local sums of the current walk

    // rate w_s = s(l - s) with l = NB + 1
    __device__ static constexpr V rate(int s) { return (V)(s * (NB + 1 - s)); }

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
                if (bit[c] >= 0) {
#pragma unroll
                    for (int s = 1; s <= NB; ++s)
                        dl[s - 1] = fmax(dl[s - 1], lph[c] + (rate(s) - rate(s - 1)) * pp[c]);
                }
            }
        }
        // block max of the injection exponents per level
#pragma unroll
        for (int s = 0; s < NB; ++s) {
            V x = dl[s];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(FULL, x, o));
            if (lane == 0) sm.fred[w][s] = x;
        }
        __syncthreads();
        if (tid < NB) {
            V x = V(-INFINITY);
            for (int q = 0; q < NW; ++q) x = fmax(x, sm.fred[q][tid]);
            sm.D[tid] = (x == V(-INFINITY)) ? V(0) : x;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < C; ++c) {
#pragma unroll
            for (int s = 1; s <= NB; ++s) {
                const V ex = lph[c] + (rate(s) - rate(s - 1)) * pp[c] - sm.D[s - 1];
                fac[c][s - 1] = (bit[c] >= 0) ? vexp<V>(ex) : V(0);
            }
        }
#pragma unroll(UNR)
        for (int S = 0; S < NS; ++S) carry[S] = V(0);
    }

    template <int SMAX, int KB>
    __device__ __forceinline__ void inject(int c)
    {
#pragma unroll(UNR)
        for (int T = 0; T < NS; ++T) {
            if (((T >> KB) & 1) && popc_c(T) <= SMAX) {
                const int U = T ^ (1 << KB);
                const V fu = (U == 0) ? V(1) : (carry[U] + run[U]);
                run[T] = fma(fac[c][popc_c(T) - 1], fu, run[T]);
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

    // Walk the chunk, recomputing levels 1..SMAX; on_target(c) is called at
    // target points with run[] holding the local sums before the point.
    template <int SMAX, typename OnT>
    __device__ __forceinline__ void walk(OnT &&on_target)
    {
#pragma unroll(UNR)
        for (int S = 0; S < NS; ++S) run[S] = V(0);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int k = bit[c];
            if (k >= 0)
                inject_dispatch<SMAX>(k, c);
            else if (k == -1)
                on_target(c);
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
    // inclusive prefix.
    template <int s>
    __device__ void lookback(Sm &sm, const SweepArgs &a, int v, int b, bool fwd)
    {
        const int lane = threadIdx.x & 31;
        constexpr int NQ = (NS + 31) / 32;
        const double ws = (double)s * (double)(NB + 1 - s);
        double aggv[NQ], acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int S = lane + 32 * q;
            aggv[q] = -INFINITY;
            acc[q] = -INFINITY;
            if (S < NS && popc_c(S) == s) {
                const double A = (double)sm.tot[S];
                aggv[q] = (A > 0.0) ? log(A) + sum_beta(sm, S) + sm.gam[s] : -INFINITY;
                a.agg[(size_t)v * NS + S] = aggv[q];
            }
        }
        int *myflag = a.flags + (size_t)v * (NB + 1) + s;
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(myflag, 1);
        bool fail = false;
        const double xb = fwd ? a.xlb[b] : a.xrb[b];
        int p = v - 1;
        while (p >= 0) {
            const int f = wait_flag(a.flags + (size_t)p * (NB + 1) + s, a.err, a.spin_limit);
            if (f < 0 || f == 3) {
                fail = true;
                break;
            }
            const int bp = fwd ? p : a.nt - 1 - p;
            const double d = (fwd ? (xb - a.xlb[bp]) : (a.xrb[bp] - xb)) / a.eps;
            const double *src = (f == 2) ? a.inc : a.agg;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int S = lane + 32 * q;
                if (S < NS && popc_c(S) == s)
                    acc[q] = lae(acc[q], __ldcg(src + (size_t)p * NS + S) - ws * d);
            }
            if (f == 2) break;
            --p;
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int S = lane + 32 * q;
            if (S < NS && popc_c(S) == s) {
                sm.E[S] = acc[q];
                a.inc[(size_t)v * NS + S] = lae(acc[q], aggv[q]);
            }
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            st_release(myflag, fail ? 3 : 2);
            if (fail) atomicOr(a.err, ERR_TIMEOUT);
        }
    }

    // Choose the final scale of level s from the tile-end values and turn the
    // tile carry into f-representation (warp 0).
    template <int s>
    __device__ void normalise(Sm &sm)
    {
        const int lane = threadIdx.x & 31;
        constexpr int NQ = (NS + 31) / 32;
        const double gs = sm.gam[s];
        double L[NQ];
        double gmax = -INFINITY;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int S = lane + 32 * q;
            L[q] = -INFINITY;
            if (S < NS && popc_c(S) == s) {
                const double A = (double)sm.tot[S];
                L[q] = lae(sm.E[S] - sum_beta(sm, S), A > 0.0 ? log(A) + gs : -INFINITY);
                gmax = fmax(gmax, L[q]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(FULL, gmax, o));
        const double gnew = (gmax == -INFINITY) ? gs : gmax;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int S = lane + 32 * q;
            if (S < NS && popc_c(S) == s) sm.tc[S] = (V)exp(sm.E[S] - sum_beta(sm, S) - gnew);
        }
        if (lane == 0) {
            sm.rho = (V)exp(gs - gnew);
            sm.gam[s] = gnew;
            if (s < NB) sm.gam[s + 1] = gnew + (double)sm.D[s];
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
        const V rho = sm.rho;
#pragma unroll
        for (int S = 0; S < NS; ++S)
            if (popc_c(S) == s) carry[S] = sm.tc[S] + rho * excl[S];
#pragma unroll
        for (int c = 0; c < C; ++c) fac[c][s - 1] *= rho;
        __syncthreads();
    }

    template <bool MAIN>
    __device__ void all_levels(Sm &sm, const SweepArgs &a, int v, int b, bool fwd)
    {
        if (threadIdx.x == 0) {
            sm.gam[0] = 0.0;
            sm.gam[1] = (double)sm.D[0];
        }
        __syncthreads();
        static_for<1, NB + 1>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            level<s, MAIN>(sm, a, v, b, fwd);
        });
    }
};

template <int NB, typename V, int NT, int C, int JCAP, bool WITH_G>
__device__ void load_tile(SweepSmem<NB, V, NT, C, JCAP, WITH_G> &sm, const SweepArgs &a, int b,
                          int n, uint32_t t0)
{
    const V *pos = static_cast<const V *>(a.pos);
    const V *lphi = static_cast<const V *>(a.lphi);
    for (int i = threadIdx.x; i < n; i += NT) {
        sm.pos[i] = __ldg(pos + t0 + i);
        sm.lphi[i] = __ldg(lphi + t0 + i);
        sm.mid[i] = __ldg(a.mid + t0 + i);
    }
    if (threadIdx.x < NB) {
        const int k = threadIdx.x;
        const int m = (k < a.j) ? k : k + 1;
        const int rt = __ldg(a.reftile + (size_t)b * a.l + m);
        sm.beta[k] = a.beta[(size_t)rt * a.l + m];
    }
    __syncthreads();
}

template <int NB, typename V, int NT, int C, int JCAP>
__global__ void __launch_bounds__(NT) k_bwd(SweepArgs a)
{
    using Sm = SweepSmem<NB, V, NT, C, JCAP, false>;
    using En = Engine<NB, V, NT, C, JCAP, false>;
    constexpr int NS = 1 << NB;
    extern __shared__ __align__(16) unsigned char smraw[];
    Sm &sm = *reinterpret_cast<Sm *>(smraw);
    __shared__ int s_v;
    if (threadIdx.x == 0) s_v = atomicAdd(a.counter, 1);
    __syncthreads();
    const int v = s_v;
    if (v >= a.nt) return;
    const int b = a.nt - 1 - v;
    const uint32_t t0 = a.tstart[b];
    const int n = (int)(a.tstart[b + 1] - t0);
    load_tile<NB, V, NT, C, JCAP, false>(sm, a, b, n, t0);
    En e;
    e.setup(sm, n, (V)a.span[b], false, a.j);
    e.template all_levels<true>(sm, a, v, b, false);
    for (int S = threadIdx.x; S < NS; S += NT) a.bcarry[(size_t)b * NS + S] = (S == 0) ? 0.0 : sm.E[S];
}

template <int NB, typename V, int NT, int C, int JCAP>
__global__ void __launch_bounds__(NT) k_fwd(SweepArgs a)
{
    using Sm = SweepSmem<NB, V, NT, C, JCAP, true>;
    using En = Engine<NB, V, NT, C, JCAP, true>;
    constexpr int NS = 1 << NB;
    constexpr int FULLS = NS - 1;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smraw[];
    Sm &sm = *reinterpret_cast<Sm *>(smraw);
    __shared__ int s_v;
    if (threadIdx.x == 0) s_v = atomicAdd(a.counter, 1);
    __syncthreads();
    const int v = s_v;
    if (v >= a.nt) return;
    const int b = v;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t t0 = a.tstart[b];
    const int n = (int)(a.tstart[b + 1] - t0);
    const V span = (V)a.span[b];
    load_tile<NB, V, NT, C, JCAP, true>(sm, a, b, n, t0);

    // ranks of the target points (forward order)
    {
        int cntt = 0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int r = tid * C + c;
            if (r < n && sm.mid[r] == a.j) ++cntt;
        }
        int incl = cntt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) sm.ired[w] = incl;
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int q = 0; q < NW; ++q) {
                const int t = sm.ired[q];
                sm.ired[q] = acc;
                acc += t;
            }
            sm.ntarget = acc;
        }
        __syncthreads();
        int rank = sm.ired[w] + incl - cntt;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int r = tid * C + c;
            if (r < n && sm.mid[r] == a.j) sm.slot[r] = (int16_t)(rank++);
        }
        __syncthreads();
    }
    if (sm.ntarget > JCAP) {
        if (tid == 0) atomicOr(a.err, ERR_RANGE);
    }

    En e;
    // ---- backward states inside the tile from the stored carry -------------
    e.setup(sm, n, span, false, a.j);
    for (int S = tid; S < NS; S += NT) sm.E[S] = (S == 0) ? 0.0 : a.bcarry[(size_t)b * NS + S];
    __syncthreads();
    e.template all_levels<false>(sm, a, v, b, false);
    e.template walk<NB>([&](int c) {
        const int sl = sm.slot[e.idx[c]];
        if (sl < JCAP) {
#pragma unroll
            for (int U = 0; U < NS; ++U) sm.G[U * JCAP + sl] = (U == 0) ? V(1) : (e.carry[U] + e.run[U]);
        }
    });
    if (tid <= NB) sm.gamG[tid] = sm.gam[tid];
    __syncthreads();

    // ---- forward scan with look-back, then combine ---------------------------
    e.setup(sm, n, span, true, a.j);
    e.template all_levels<true>(sm, a, v, b, true);

    // per-tile constants of the combine
    __shared__ double s_base;
    __shared__ V s_dG[NB + 1];
    if (tid == 0) {
        double gmx = -INFINITY;
        for (int s = 0; s <= NB; ++s) gmx = fmax(gmx, sm.gam[s] + sm.gamG[NB - s]);
        if (gmx == -INFINITY) gmx = 0.0;
        double sb = 0.0;
        for (int k = 0; k < NB; ++k) sb += sm.beta[k];
        s_base = sb + gmx;
        for (int s = 0; s <= NB; ++s) {
            const double d = sm.gam[s] + sm.gamG[NB - s] - gmx;
            s_dG[s] = (d < -1e30) ? V(-1e30) : (V)d;
        }
    }
    __syncthreads();
    double lnM[C];
#pragma unroll
    for (int c = 0; c < C; ++c) lnM[c] = 0.0;
    const double base = s_base;
    e.template walk<NB>([&](int c) {
        const int sl = sm.slot[e.idx[c]];
        V X[NB + 1];
#pragma unroll
        for (int s = 0; s <= NB; ++s) X[s] = V(0);
        if (sl < JCAP) {
#pragma unroll
            for (int S = 0; S < NS; ++S) {
                const V fS = (S == 0) ? V(1) : (e.carry[S] + e.run[S]);
                X[popc_c(S)] += fS * sm.G[(FULLS ^ S) * JCAP + sl];
            }
        }
        const V pF = e.pp[c];
        const V pG = span - pF;
        V ev[NB + 1];
        V emax = V(-INFINITY);
#pragma unroll
        for (int s = 0; s <= NB; ++s) {
            ev[s] = s_dG[s] - En::rate(s) * pF - En::rate(NB - s) * pG;
            if (X[s] > V(0)) emax = (ev[s] > emax) ? ev[s] : emax;
        }
        V sum = V(0);
#pragma unroll
        for (int s = 0; s <= NB; ++s)
            if (X[s] > V(0)) sum += vexp<V>(ev[s] - emax) * X[s];
        lnM[c] = (sum > V(0)) ? base + (double)emax + log((double)sum) : -INFINITY;
    });

    // ---- FP64 epilogue ------------------------------------------------------
    const int32_t off = a.cnt[(size_t)b * a.l + a.j];
    if (a.mode == MODE_UPDATE) {
        double gv[C];
        double gmax = -INFINITY;
        bool bad = false;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            gv[c] = -INFINITY;
            if (e.bit[c] == -1) {
                const int i = off + sm.slot[e.idx[c]];
                const double lm = a.lnmuj[i];
                if (lm > -INFINITY) {
                    gv[c] = a.eps * (lm - lnM[c]);
                    if (!isfinite(gv[c])) bad = true;
                    gmax = fmax(gmax, gv[c] / a.eps);
                }
            }
        }
        if (bad) atomicOr(a.err, ERR_NONFINITE);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(FULL, gmax, o));
        if (lane == 0) sm.dred[w] = gmax;
        __syncthreads();
        if (tid == 0) {
            double x = -INFINITY;
            for (int q = 0; q < NW; ++q) x = fmax(x, sm.dred[q]);
            if (!isfinite(x)) x = 0.0;
            sm.dred[0] = x;
            if (sm.ntarget > 0) a.beta[(size_t)b * a.l + a.j] = x;
        }
        __syncthreads();
        const double bnew = sm.dred[0];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            if (e.bit[c] == -1) {
                const int i = off + sm.slot[e.idx[c]];
                a.gj[i] = gv[c];
                static_cast<V *>(a.lphi)[t0 + e.idx[c]] = (V)(gv[c] / a.eps - bnew);
            }
        }
    } else if (a.mode == MODE_RESIDUAL) {
        double acc = 0.0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            if (e.bit[c] == -1) {
                const int i = off + sm.slot[e.idx[c]];
                const double gg = a.gj[i];
                const double marg = (gg == -INFINITY || lnM[c] == -INFINITY) ? 0.0 : exp(gg / a.eps + lnM[c]);
                acc += fabs(marg - a.muj[i]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (lane == 0) sm.dred[w] = acc;
        __syncthreads();
        if (tid == 0) {
            double x = 0.0;
            for (int q = 0; q < NW; ++q) x += sm.dred[q];
            a.partial[b] = x;
        }
    } else {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            if (e.bit[c] == -1) {
                const int i = off + sm.slot[e.idx[c]];
                double r;
                if (a.mode == MODE_OUT_M)
                    r = exp(lnM[c]);
                else if (a.mode == MODE_OUT_PLAN)
                    r = (a.gj[i] == -INFINITY) ? 0.0 : exp(a.gj[i] / a.eps + lnM[c]);
                else
                    r = lnM[c];
                a.out[i] = r;
            }
        }
    }
}

template <int NB, typename V, int NT, int C, int JCAP>
cudaError_t launch_bwd_impl(const SweepArgs &a, cudaStream_t st)
{
    using Sm = SweepSmem<NB, V, NT, C, JCAP, false>;
    auto kern = k_bwd<NB, V, NT, C, JCAP>;
    const size_t sz = sizeof(Sm);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz);
    if (e != cudaSuccess) return e;
    kern<<<a.nt, NT, sz, st>>>(a);
    return cudaGetLastError();
}

template <int NB, typename V, int NT, int C, int JCAP>
cudaError_t launch_fwd_impl(const SweepArgs &a, cudaStream_t st)
{
    using Sm = SweepSmem<NB, V, NT, C, JCAP, true>;
    auto kern = k_fwd<NB, V, NT, C, JCAP>;
    const size_t sz = sizeof(Sm);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz);
    if (e != cudaSuccess) return e;
    kern<<<a.nt, NT, sz, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mmot

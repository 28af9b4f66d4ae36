// Transport cost W = <C, T> of the current plan (Eq. k-mmot distance).
//
// Gap formula: between consecutive points of the merged order every tuple
// whose set S of marginals lies left of the gap pays |S|(l - |S|) per unit
// length (for a tuple, sum_{i<k} |x_i - x_k| is the integral over y of
// n(y)(l - n(y)), n(y) the number of its points left of y), so
//   W = sum_t (x_t - x_{t-1}) sum_S w_|S| F_S(x_t^-) G_{S^c}(x_t, incl. t)
// over all 2^l subsets S of the l marginals, F the forward states (Sec. 4.2
// class sums grouped by subset) before point t and G the backward states
// including it.  The sweeps are the ones of the marginal product with l state
// bits and no target marginal; the rate of a state is again w_s = s(l - s).
//
// In the tile frame F_S G_{S^c} at any position carries exp(-w_s span), the
// same for every point of the tile, so each tile yields, in FP64,
//   partial[b] = eps * W_b / Z_b,  out[b] = ln Z
// with W_b the tile's gap sum and Z_b = sum_S F_S G_{S^c} at the first gap of
// the tile (Z_b is the total mass Z in the tile's scale; the ratio is W_b / Z).
#pragma once
#include "shapes.cuh"
#include "sweep.cuh"

namespace mmot {

template <int NB, typename V, int NT, int C, int JCAP, bool LOOKBACK>
__global__ void __launch_bounds__(NT) k_objective(SweepArgs a)
{
    using Sm = SweepSmem<NB, V, NT, C, JCAP, true>;
    using En = Engine<NB, V, NT, C, JCAP, true, NB>;
    constexpr int NS = 1 << NB;
    constexpr int FULLS = NS - 1;
    constexpr int K = NT * C;
    constexpr int NW = NT / 32;
    static_assert(JCAP == K, "the objective keeps the backward states of every point");
    extern __shared__ __align__(16) unsigned char smraw[];
    Sm &sm = *reinterpret_cast<Sm *>(smraw);
    __shared__ int s_v;
    __shared__ double s_base;
    __shared__ V s_wm[NW];
    __shared__ int s_wk[NW];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int v, b;
    if constexpr (LOOKBACK) {
        if (tid == 0) s_v = atomicAdd(a.counter, 1);
        __syncthreads();
        v = s_v;
        if (v >= a.nt) return;
        b = v;
    } else {
        b = v = blockIdx.x;
    }
    const uint32_t t0 = a.tstart[b];
    const int n = (int)(a.tstart[b + 1] - t0);
    const V span = (V)a.span[b];
    load_tile<NB, V, NT, C, JCAP, true>(sm, a, b, n, t0, a.j);

    // ---- backward states including each point, kept for every point --------
    En e;
    e.setup(sm, n, span, false, a.j);
    for (int S = tid; S < NS; S += NT) {
        sm.E[S] = sf_load<V>(sfp<V>(a.bcarry)[(size_t)b * NS + S]);
        sm.Eh[S] = sf_scale_exp(sm.E[S], -En::sum_beta(sm, S));
    }
    __syncthreads();
    e.template all_levels<false>(sm, a, v, b, false);
    e.template walk_each<false>([&](int c) {
        const int id = e.idx[c];
#pragma unroll(En::UNR)
        for (int U = 0; U < NS; ++U) sm.G[U * K + id] = (U == 0) ? V(1) : (e.carry[U] + e.run[U]);
    });
    for (int S = tid; S < NS; S += NT) sm.GsG[S] = sm.Gs[S];
    __syncthreads();

    // ---- forward states --------------------------------------------------------
    e.setup(sm, n, span, true, a.j);
    if constexpr (LOOKBACK) {
        e.template all_levels<true>(sm, a, v, b, true);
    } else {
        for (int S = tid; S < NS; S += NT) {
            sm.E[S] = sf_load<V>(sfp<V>(a.fcarry)[(size_t)b * NS + S]);
            sm.Eh[S] = sf_scale_exp(sm.E[S], -En::sum_beta(sm, S));
        }
        __syncthreads();
        e.template all_levels<false>(sm, a, v, b, true);
    }
    // binary exponent of the product of the two states' scales, and the FP64
    // base; the factor exp(-w_s span) is the same at every point of the tile
    for (int S = tid; S < NS; S += NT) sm.eS[S] = (sm.Gs[S].k - 1) + (sm.GsG[FULLS ^ S].k - 1);
    if (tid == 0) {
        double sb = 0.0;
        for (int k = 0; k < NB; ++k) sb += sm.beta[k];
        s_base = sb;
    }
    __syncthreads();
    V q[NB + 1];
#pragma unroll
    for (int s = 0; s <= NB; ++s) q[s] = vexp<V>(-En::rate(s) * span);
    // gap before the tile's first point (none at the start of an instance)
    const bool first = (b == 0) || (a.seg && a.seg[b - 1] != a.seg[b]);
    const V gap0 = first ? V(0) : (V)(a.ulb[b] - a.urb[b - 1]);
    Sf<V> accW = sf_zero<V>(), accZ = sf_zero<V>();
    e.template walk_each<true>([&](int c) {
        const int id = e.idx[c];
        // sum over S of w_S F_S G_{S^c} (and without weights for Z), as
        // mantissa x 2^exponent with a running maximum exponent
        int Emax = INT_MIN / 2;
        V sw = V(0), sz = V(0);
#pragma unroll(En::UNR)
        for (int S = 0; S < NS; ++S) {
            const V fS = (S == 0) ? V(1) : (e.carry[S] + e.run[S]);
            const Sf<V> fm = sf_make<V>(fS);
            const Sf<V> gm = sf_make<V>(sm.G[(FULLS ^ S) * K + id]);
            if (fm.m != V(0) && gm.m != V(0)) {
                const int s = popc_c(S);
                const V z = fm.m * gm.m * q[s];
                const int E = fm.k + gm.k + sm.eS[S];
                if (E > Emax) {
                    const V r = pow2neg<V>(Emax - E);
                    sw = fma(sw, r, En::rate(s) * z);
                    sz = fma(sz, r, z);
                    Emax = E;
                } else {
                    const V r = pow2neg<V>(E - Emax);
                    sw = fma(En::rate(s) * z, r, sw);
                    sz = fma(z, r, sz);
                }
            }
        }
        if (!(sz > V(0))) return;
        const V dx = (id > 0) ? sm.pos[id] - sm.pos[id - 1] : gap0;
        Sf<V> t = sf_make<V>(dx * sw);
        t.k += Emax;
        if (t.m != V(0)) accW = sf_add(accW, t);
        if (id == 0) {
            accZ = sf_make<V>(sz);
            accZ.k += Emax;
        }
    });
    const Sf<V> ws = sf_warp_sum(accW);
    if (lane == 0) {
        s_wm[w] = ws.m;
        s_wk[w] = ws.k;
    }
    __syncthreads();
    if (tid == 0) {
        Sf<V> tot = sf_zero<V>();
        for (int q = 0; q < NW; ++q) tot = sf_add(tot, Sf<V>{s_wm[q], s_wk[q]});
        // thread 0 holds the first point of the tile (forward order)
        if (accZ.m == V(0)) {
            a.partial[b] = 0.0;
            a.out[b] = -INFINITY;
        } else {
            const double r = (tot.m == V(0)) ? 0.0 : ldexp((double)tot.m / (double)accZ.m, tot.k - accZ.k);
            a.partial[b] = tile_eps(a, b) * r;
            a.out[b] = log((double)accZ.m) + (double)accZ.k * kLn2 + s_base;
        }
    }
}

template <int NB, typename V, int NT, int C, bool LOOKBACK>
cudaError_t launch_objective_kernel(const SweepArgs &a, cudaStream_t st)
{
    constexpr int K = NT * C;
    using Sm = SweepSmem<NB, V, NT, C, K, true>;
    auto kern = k_objective<NB, V, NT, C, K, LOOKBACK>;
    const size_t sz = sizeof(Sm);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz);
    if (e != cudaSuccess) return e;
    kern<<<a.nt, NT, sz, st>>>(a);
    return cudaGetLastError();
}

// Objective kernels of l marginals on the tiling of the marginal product
// (tile shape of l - 1 bits).  kind: 0 backward look-back sweep, 2 tile
// operators, 3 carry scan, 5 objective (three-phase carries for l <= 4,
// forward look-back otherwise).
template <int Lm, typename V>
cudaError_t launch_objective_impl(const SweepArgs &a, cudaStream_t st, int kind)
{
    using S = Shape<Lm - 1, V>;
    constexpr bool THREE = (Lm <= kMaxOpBits);
    if (kind == 5) return launch_objective_kernel<Lm, V, S::NT, S::C, !THREE>(a, st);
    if constexpr (THREE) {
        if (kind == 2) return launch_tileop_impl<Lm, V, S::NT, S::C, S::JCAP, Lm>(a, st);
        if (kind == 3) return launch_carry_impl<Lm, V, Lm>(a, st);
    } else {
        if (kind == 0) return launch_bwd_impl<Lm, V, S::NT, S::C, S::JCAP, Lm>(a, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace mmot

#define MMOT_INSTANTIATE_OBJECTIVE(L_)                                                  \
    namespace mmot {                                                                   \
    template <>                                                                        \
    cudaError_t launch_objective<L_, float>(const SweepArgs &a, cudaStream_t s, int k) \
    {                                                                                  \
        return launch_objective_impl<L_, float>(a, s, k);                              \
    }                                                                                  \
    template <>                                                                        \
    cudaError_t launch_objective<L_, double>(const SweepArgs &a, cudaStream_t s, int k)\
    {                                                                                  \
        return launch_objective_impl<L_, double>(a, s, k);                             \
    }                                                                                  \
    }

// Warp-per-tile marginal products for many state bits (l >= 6, NB >= 5).
//
// With 2^{l-1} >= 32 states a tile is processed by one warp: lane L holds the
// states T = L + 32 q (q < NS/32) as scaled floats (mantissa, binary
// exponent), and the warp walks the tile's points in order.  At a point of
// bit k every state T containing k gains phi * F_{T\k} (Sec. 4.2 recurrences
// grouped by subset); F_{T\k} sits in lane L ^ 2^k for k < 5 and in the same
// lane's register q ^ 2^{k-5} otherwise, so one xor-shuffle or a register
// select fetches it.  Every state keeps its own exponent, so states of one
// level may differ by any factor.  Values are kept in the tile's cumulative
// frame relative to exp(sum_{m in T} beta_m + gamma_{|T|}) (gamma_s =
// D_1 + ... + D_s, D_r = max(0, a_r span)), as in the block engine.
//
// Carries: level passes (k_wpass) give each tile's own contribution to the
// states of one level from the known lower-level carries; the scalar scans
// of k_lscan turn them into carries.  The final kernel (k_wprod) runs the
// backward pass of the tile from its backward carries (states at the target
// points kept in shared memory), then the forward pass with the combine
// M_j = sum_S F_S(x^-) G_{R\S}(x^+) and the FP64 epilogue.
#pragma once
#include "shapes.cuh"
#include "sweep.cuh"

namespace mmot {

// NB state bits; LM marginals in the cost (NB + 1 for a marginal product, NB
// for the all-subset sweeps of the objective).
template <int NB, typename V, int LM = NB + 1>
struct WarpRun {
    static_assert(NB + 1 <= 16, "a row of the factor buffer holds levels 0..NB");
    static constexpr int NS = 1 << NB;
    static constexpr int NQ = NS / 32;
    static constexpr int L = LM;
    static constexpr unsigned FULL = 0xffffffffu;
    Sf<V> f[NQ];
    V D[NB + 1];         // D[s] = max(0, a_s span), s = 1..NB
    double gam[NB + 1];  // gamma_s = D_1 + ... + D_s
    V span;
    int lane;
    int coef_level = 0;   // > 0: lane m sums the level-coef_level factors of the points of bit m
    V coef_acc = V(0);
    // FP32 path: this warp's fixed-point table in shared memory, [0, NB) the
    // baselines beta_k, [NB, 2 NB] gamma_s (fx_log2)
    long long *fx = nullptr;

    __device__ static constexpr int rate(int s) { return s * (L - s); }

    __device__ void init(const SweepArgs &a, int b)
    {
        lane = threadIdx.x & 31;
        span = (V)a.span[b];
        gam[0] = 0.0;
        D[0] = V(0);
#pragma unroll
        for (int s = 1; s <= NB; ++s) {
            const V as = (V)(rate(s) - rate(s - 1));
            D[s] = (as > V(0)) ? as * span : V(0);
            if constexpr (sizeof(V) == 8) gam[s] = gam[s - 1] + (double)D[s];
        }
    }

    // sum of the baselines of the marginals in T (bits mapped around the target)
    __device__ static double sum_beta(const double *beta, int T)
    {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if ((T >> k) & 1) s += beta[k];
        return s;
    }

    // gamma_s for a runtime level (selected from registers: no local memory)
    __device__ double gam_at(int s) const
    {
        double g = 0.0;
#pragma unroll
        for (int q = 0; q <= NB; ++q)
            if (q == s) g = gam[q];
        return g;
    }

    // FP32 path: the fixed-point table of the tile (lane k: beta_k; lanes
    // 1..NB: D_s, then a prefix sum over the lanes for gamma_s)
    __device__ void setup_fx(const double *beta, long long *table)
    {
        fx = table;
        if constexpr (sizeof(V) == 4) {
            double bk = 0.0;
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (k == lane) bk = beta[k];
            if (lane < NB) fx[lane] = fx_log2(bk);
            V d = V(0);
#pragma unroll
            for (int s = 1; s <= NB; ++s)
                if (s == lane) d = D[s];
            long long g = (lane >= 1 && lane <= NB) ? fx_log2((double)d) : 0ll;
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) {
                const long long y = __shfl_up_sync(FULL, g, o);
                if (lane >= o) g += y;
            }
            if (lane <= NB) fx[NB + lane] = g;
            __syncwarp();
        }
    }

    // a * exp(sign (sum_{k in T} beta_k + gamma_s))
    __device__ __forceinline__ Sf<V> scale_state(Sf<V> a, int T, int s, bool neg, const double *beta) const
    {
        if constexpr (sizeof(V) == 4) {
            long long X = 0;
#pragma unroll
            for (int q = 0; q <= NB; ++q)
                if (q == s) X = fx[NB + q];
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if ((T >> k) & 1) X += fx[k];
            return sf_scale_fx(a, neg ? -X : X);
        } else {
            const double x = sum_beta(beta, T) + gam_at(s);
            return sf_scale_exp(a, neg ? -x : x);
        }
    }

    // states from absolute carries (levels below maxlev; the rest 0; the
    // empty state 1, the source of the level-1 injections)
    __device__ void load_carries(const SfT<V> *carry, int b, const double *beta, int maxlev)
    {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int T = lane + 32 * q;
            const int s = __popc(T);
            f[q] = (T == 0) ? Sf<V>{V(0.5), 1} : sf_zero<V>();
            if (T != 0 && s < maxlev) f[q] = scale_state(sf_load<V>(carry[(size_t)b * NS + T]), T, s, true, beta);
        }
    }

    // Injection factors of the chunk's points, one point per lane, all levels:
    // fb[lane][s] = exp(ln phi + a_s p - D_s), a_s = w_s - w_{s-1}
    __device__ void chunk_facs(V lp, V pp, bool inj, V (*fb)[16]) const
    {
        if (inj) {
            static_for<1, NB + 1>([&](auto sc) {
                constexpr int s = decltype(sc)::value;
                fb[lane][s] = vexp<V>(lp + (V)(rate(s) - rate(s - 1)) * pp - D[s]);
            });
        }
        __syncwarp();
    }

    // F_T += phi F_{T\k} for every state T containing k, factors fr[s] of the
    // point (F_{T\k} sits in lane ^ 2^k for k < 5, in register q ^ 2^{k-5}
    // otherwise; the empty state is 1)
    __device__ __forceinline__ void inject(int k, const V *fr)
    {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int T = lane + 32 * q;
            Sf<V> src;
            if (k < 5) {
                src.m = __shfl_xor_sync(FULL, f[q].m, 1 << k);
                src.k = __shfl_xor_sync(FULL, f[q].k, 1 << k);
            } else {
                src = f[0];
#pragma unroll
                for (int q2 = 0; q2 < NQ; ++q2)
                    if (q2 == (q ^ (1 << (k - 5)))) src = f[q2];
            }
            if ((T >> k) & 1) {
                if ((T ^ (1 << k)) == 0) src = Sf<V>{V(0.5), 1};
                if (src.m != V(0)) {
                    Sf<V> t = sf_make<V>(src.m * fr[__popc(T)]);
                    t.k += src.k;
                    if (t.m != V(0)) f[q] = sf_add(f[q], t);
                }
            }
        }
    }

    // ---- chunk frame (fast path) ---------------------------------------------
    // Over a chunk of 32 points every state T is kept as an FP32/FP64 value v
    // relative to a fixed power of two 2^E_T: E_T bounds what T can reach in
    // the chunk, the largest own exponent of the states U inside T from which
    // the chunk's marginals (cbits) lead to T, plus 5 bits per level of growth
    // (32 injections at most, each factor <= 1).  An injection is then one
    // FMA with the precomputed ratio 2^{E_{T\k} - E_T}.  A chunk in which some
    // state's own value would sit more than 2^-90 below its frame (sources
    // far larger than the state itself, sparse supports at small eps) runs
    // with exact scaled floats instead.
    static constexpr int kHead = 5 * NB + 2;

    __device__ __forceinline__ bool chunk_frame(int cbits, int (&E)[NQ], V (&v)[NQ], V (&rt)[NQ][NB])
    {
        int e[NQ], m[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            e[q] = (f[q].m == V(0)) ? INT_MIN / 2 : f[q].k;
            m[q] = e[q];
        }
        // max over the subsets reachable through the chunk's marginals
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            if ((cbits >> b) & 1) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    int src;
                    if constexpr (b < 5) {
                        src = __shfl_xor_sync(FULL, m[q], 1 << b);
                    } else {
                        src = m[0];
#pragma unroll
                        for (int q2 = 0; q2 < NQ; ++q2)
                            if (q2 == (q ^ (1 << (b - 5)))) src = m[q2];
                    }
                    if (((lane + 32 * q) >> b) & 1) m[q] = max(m[q], src);
                }
            }
        });
        bool bad = false;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            E[q] = m[q] + kHead;
            if (f[q].m != V(0) && E[q] - e[q] > 90) bad = true;
        }
        if (__any_sync(FULL, bad)) return false;
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = (f[q].m == V(0)) ? V(0) : f[q].m * pow2neg<V>(e[q] - E[q]);
        // ratios of the injections 2^{E_{T\k} - E_T}
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                int es;
                if constexpr (b < 5) {
                    es = __shfl_xor_sync(FULL, E[q], 1 << b);
                } else {
                    es = E[0];
#pragma unroll
                    for (int q2 = 0; q2 < NQ; ++q2)
                        if (q2 == (q ^ (1 << (b - 5)))) es = E[q2];
                }
                const int d = es - E[q];
                rt[q][b] = (((lane + 32 * q) >> b) & 1) ? ((d <= 0) ? pow2neg<V>(d) : vldexp<V>(V(1), d)) : V(0);
            }
        });
        return true;
    }

    // one injection of bit K in the chunk frame
    template <int K>
    __device__ __forceinline__ void inject_frame(V (&v)[NQ], const V (&rt)[NQ][NB], const V *fr)
    {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            V src;
            if constexpr (K < 5) {
                src = __shfl_xor_sync(FULL, v[q], 1 << K);
            } else {
                src = v[0];
#pragma unroll
                for (int q2 = 0; q2 < NQ; ++q2)
                    if (q2 == (q ^ (1 << (K - 5)))) src = v[q2];
            }
            if (((lane + 32 * q) >> K) & 1) v[q] = fma(fr[__popc(lane + 32 * q)] * rt[q][K], src, v[q]);
        }
    }

    template <int K = 0>
    __device__ __forceinline__ void inject_frame_dispatch(int k, V (&v)[NQ], const V (&rt)[NQ][NB], const V *fr)
    {
        if constexpr (K < NB) {
            if (k == K)
                inject_frame<K>(v, rt, fr);
            else
                inject_frame_dispatch<K + 1>(k, v, rt, fr);
        }
    }

    __device__ __forceinline__ void frame_out(const int (&E)[NQ], const V (&v)[NQ])
    {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            Sf<V> t = sf_make<V>(v[q]);
            if (t.m != V(0)) t.k += E[q];
            f[q] = t;
        }
    }

    // Walk the tile's n points in processing order; on_target(slot, p) at the
    // target points with the states before the point.  bits of the marginals:
    // m < j -> m, m > j -> m - 1, target j -> -1.  fb: this warp's 32 x 16
    // buffer of injection factors (shared memory).
    template <typename OnT>
    __device__ void run(const SweepArgs &a, uint32_t t0, int n, int j, bool fwd, int ntarget, V (*fb)[16],
                        OnT &&on_target)
    {
        const V *pos = static_cast<const V *>(a.pos);
        const V *lphi = static_cast<const V *>(a.lphi);
        int seen = 0;   // targets passed so far
        for (int c0 = 0; c0 < n; c0 += 32) {
            const int r = c0 + lane;
            V pp = V(0), lp = V(0);
            int bit = -2;
            if (r < n) {
                const int id = fwd ? r : n - 1 - r;
                const int m = a.mid[t0 + id];
                bit = (m == j) ? -1 : (m < j ? m : m - 1);
                const V x = pos[t0 + id];
                pp = fwd ? x : span - x;
                lp = lphi[t0 + id];
            }
            chunk_facs(lp, pp, bit >= 0, fb);
            const int cnt = min(32, n - c0);
            const int cbits = __reduce_or_sync(FULL, bit >= 0 ? (1 << bit) : 0);
            int E[NQ];
            V v[NQ];
            V rt[NQ][NB];
            if (chunk_frame(cbits, E, v, rt)) {
                for (int i = 0; i < cnt; ++i) {
                    const int k = __shfl_sync(FULL, bit, i);
                    if (k == -1) {
                        frame_out(E, v);
                        const V p = __shfl_sync(FULL, pp, i);
                        const int slot = fwd ? seen : ntarget - 1 - seen;
                        on_target(slot, p);
                        ++seen;
                        continue;
                    }
                    if (coef_level && lane == k) coef_acc += fb[i][coef_level];
                    inject_frame_dispatch(k, v, rt, fb[i]);
                }
                frame_out(E, v);
            } else {
                for (int i = 0; i < cnt; ++i) {
                    const int k = __shfl_sync(FULL, bit, i);
                    if (k == -1) {
                        const V p = __shfl_sync(FULL, pp, i);
                        const int slot = fwd ? seen : ntarget - 1 - seen;
                        on_target(slot, p);
                        ++seen;
                        continue;
                    }
                    if (coef_level && lane == k) coef_acc += fb[i][coef_level];
                    inject(k, fb[i]);
                }
            }
            __syncwarp();   // the next chunk overwrites fb
        }
    }
};

// Objective walk: every point injects (no target); on_point(id, p) is called
// before (PRE) or after the point's injection with the tile-local index.
// Only the points at processing positions [r0, r1) of the n-point tile are
// walked (position = index forward, n - 1 - index backward).
template <int NB, typename V, int LM, bool PRE, typename OnP>
__device__ void warp_run_each(WarpRun<NB, V, LM> &r, const SweepArgs &a, uint32_t t0, int n, bool fwd,
                              int r0, int r1, V (*fb)[16], OnP &&on_point)
{
    constexpr unsigned FULL = 0xffffffffu;
    const V *pos = static_cast<const V *>(a.pos);
    const V *lphi = static_cast<const V *>(a.lphi);
    const int lane = r.lane;
    for (int c0 = r0; c0 < r1; c0 += 32) {
        const int rr = c0 + lane;
        V pp = V(0), lp = V(0);
        int bit = -2, idl = 0;
        if (rr < r1) {
            idl = fwd ? rr : n - 1 - rr;
            bit = a.mid[t0 + idl];
            const V x = pos[t0 + idl];
            pp = fwd ? x : r.span - x;
            lp = lphi[t0 + idl];
        }
        r.chunk_facs(lp, pp, bit >= 0, fb);
        const int cnt = min(32, r1 - c0);
        for (int i = 0; i < cnt; ++i) {
            const int k = __shfl_sync(FULL, bit, i);
            const V p = __shfl_sync(FULL, pp, i);
            const int id = __shfl_sync(FULL, idl, i);
            if constexpr (PRE) on_point(id, p);
            r.inject(k, fb[i]);
            if constexpr (!PRE) on_point(id, p);
        }
        __syncwarp();
    }
}

// number of target points of the tile
__device__ __forceinline__ int warp_count_targets(const SweepArgs &a, uint32_t t0, int n, int j)
{
    int c = 0;
    for (int r = threadIdx.x & 31; r < n; r += 32) c += (a.mid[t0 + r] == j);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    return c;
}

template <int NB>
__device__ __forceinline__ void warp_betas(const SweepArgs &a, int b, int j, double *beta)
{
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        const int m = (k < j) ? k : k + 1;
        const int rt = __ldg(a.reftile + (size_t)b * a.l + m);
        beta[k] = *(volatile const double *)(a.beta + (size_t)rt * a.l + m);
    }
}

// Level pass: the tile's own contribution to the states of level SL at its
// base, from the carries of the lower levels.  4 warps per block, one tile
// per warp.
template <int NB, typename V, int LM = NB + 1>
__global__ void __launch_bounds__(128) k_wpass(SweepArgs a, int SL, int fwd_i)
{
    constexpr int NS = 1 << NB;
    const int b = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (b >= a.nt) return;
    if (a.frozen && (a.mode == MODE_UPDATE || a.mode == MODE_RESIDUAL) && a.frozen[a.seg[b]]) return;
    const bool fwd = (fwd_i != 0);
    const uint32_t t0 = a.tstart[b];
    const int n = (int)(a.tstart[b + 1] - t0);
    double beta[NB];
    warp_betas<NB>(a, b, a.j, beta);
    __shared__ V fbuf[4][32][16];
    __shared__ long long fxt[4][2 * NB + 1];
    WarpRun<NB, V, LM> r;
    r.init(a, b);
    r.setup_fx(beta, fxt[threadIdx.x >> 5]);
    r.load_carries(sfp<V>(fwd ? a.fcarry : a.bcarry), b, beta, SL);
    const bool pair = a.pair && SL < NB;
    r.coef_level = pair ? SL + 1 : 0;
    r.run(a, t0, n, a.j, fwd, 0, fbuf[threadIdx.x >> 5], [](int, V) {});
#pragma unroll
    for (int q = 0; q < WarpRun<NB, V, LM>::NQ; ++q) {
        const int T = r.lane + 32 * q;
        const int s = popc_c(T);
        if (s == SL || (pair && s == SL + 1))
            sfp<V>(a.agg)[(size_t)b * NS + T] = sf_store(r.scale_state(r.f[q], T, s, false, beta));
    }
    if (pair && r.lane < NB) {
        // a level-SL carry U reaches U + {m} with exp(beta_m + D_{SL+1}) times
        // the sum of the level-(SL+1) factors of the points of marginal m
        V dn = V(0);
#pragma unroll
        for (int s = 1; s <= NB; ++s)
            if (s == SL + 1) dn = r.D[s];
        double bm = 0.0;
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if (k == r.lane) bm = beta[k];
        sfp<V>(a.coef)[(size_t)b * NB + r.lane] = sf_store(sf_scale_exp(sf_make<V>(r.coef_acc), bm + (double)dn));
    }
}

// Backward walk of a marginal product (backward carries known): the states at
// every target point of the tile go to a.gtarg, [target][2^NB] scaled floats
// (the target's local index), read by k_wprod.  4 warps per block, one tile
// per warp.
template <int NB, typename V>
__global__ void __launch_bounds__(128) k_wbwd(SweepArgs a)
{
    using R = WarpRun<NB, V>;
    constexpr int NS = 1 << NB;
    constexpr int NQ = R::NQ;
    const int b = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (b >= a.nt) return;
    if (a.frozen && (a.mode == MODE_UPDATE || a.mode == MODE_RESIDUAL) && a.frozen[a.seg[b]]) return;
    __shared__ V fbuf[4][32][16];
    __shared__ long long fxt[4][2 * NB + 1];
    const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
    const uint32_t t0 = a.tstart[b];
    const int n = (int)(a.tstart[b + 1] - t0);
    const int nt = warp_count_targets(a, t0, n, a.j);
    double beta[NB];
    warp_betas<NB>(a, b, a.j, beta);
    SfT<V> *G = sfp<V>(a.gtarg) + (size_t)a.cnt[(size_t)b * a.l + a.j] * NS;
    R rb;
    rb.init(a, b);
    rb.setup_fx(beta, fxt[wv]);
    rb.load_carries(sfp<V>(a.bcarry), b, beta, NB + 1);
    rb.run(a, t0, n, a.j, false, nt, fbuf[wv], [&](int slot, V) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) G[(size_t)slot * NS + lane + 32 * q] = sf_store(rb.f[q]);
    });
}

// One tile of a marginal product (both carries known; the backward states at
// the targets from k_wbwd): forward pass with the combine, FP64 epilogue.
// One warp per block.  The combine keeps each target's sum as an FP32
// mantissa and a binary exponent; the FP64 work (ln M, the potential update,
// residual and objective terms) runs afterwards with one target per lane.
template <int NB, typename V>
__global__ void __launch_bounds__(32) k_wprod(SweepArgs a)
{
    using R = WarpRun<NB, V>;
    constexpr int NS = 1 << NB;
    constexpr int NQ = R::NQ;
    constexpr int JCAP = WShape<NB, V>::JCAP;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ V tsw[JCAP];      // per target: sum mantissa (0: M = 0)
    __shared__ int tew[JCAP];    // per target: binary exponent of the sum
    __shared__ double gq[JCAP];  // per target: new g/eps (update)
    __shared__ V fbuf[32][16];
    __shared__ long long fxt[2 * NB + 1];
    const int b = blockIdx.x;
    if (a.frozen && (a.mode == MODE_UPDATE || a.mode == MODE_RESIDUAL) && a.frozen[a.seg[b]]) {
        if (a.mode == MODE_RESIDUAL && threadIdx.x == 0) a.partial[b] = 0.0;
        return;
    }
    const int lane = threadIdx.x & 31;
    const uint32_t t0 = a.tstart[b];
    const int n = (int)(a.tstart[b + 1] - t0);
    const int nt = warp_count_targets(a, t0, n, a.j);
    if (nt > JCAP) {
        if (lane == 0) atomicOr(a.err, ERR_RANGE);
        return;
    }
    double beta[NB];
    warp_betas<NB>(a, b, a.j, beta);
    double sb = 0.0;
#pragma unroll
    for (int k = 0; k < NB; ++k) sb += beta[k];
    const double eps_b = tile_eps(a, b);
    const double inv_eps_b = a.teps ? 1.0 / eps_b : a.inv_eps;

    // the backward states at the target points (k_wbwd)
    const SfT<V> *Gt = sfp<V>(a.gtarg) + (size_t)a.cnt[(size_t)b * a.l + a.j] * NS;
    R rb;
    rb.init(a, b);
    rb.setup_fx(beta, fxt);

    // Per-level factor of the combine, exp(gamma_s + gamma_{NB-s} - w_s pF -
    // w_{NB-s} pG) with pG = span - pF:  exp(K_s - a_s pF), K_s = gamma_s +
    // gamma_{NB-s} - w_{NB-s} span, a_s = w_s - w_{NB-s}.  Lane s keeps K_s
    // (fixed point on the FP32 path, FP64 otherwise); per target it forms
    // a_s pF log2(e) as an exact FP32 product plus a rounded remainder.
    const int sl_ = (lane <= NB) ? lane : 0;
    const int as_ = R::rate(sl_) - R::rate(NB - sl_);
    long long Kx = 0;
    double Kd = 0.0;
    if constexpr (sizeof(V) == 4) {
        long long g1 = 0, g2 = 0;
#pragma unroll
        for (int q = 0; q <= NB; ++q) {
            if (q == sl_) g1 = fxt[NB + q];
            if (q == NB - sl_) g2 = fxt[NB + q];
        }
        Kx = g1 + g2 - fx_log2((double)R::rate(NB - sl_) * (double)rb.span);
    } else {
        Kd = (rb.gam_at(sl_) + rb.gam_at(NB - sl_) - (double)R::rate(NB - sl_) * (double)rb.span) * kLog2e;
    }

    // forward pass and combine, per target: sum_S F_S G_{R\S} factor_|S| as
    // mantissa x 2^exponent into tsw / tew
    R rf;
    rf.init(a, b);
    rf.fx = fxt;
    rf.load_carries(sfp<V>(a.fcarry), b, beta, NB + 1);
    rf.run(a, t0, n, a.j, true, nt, fbuf, [&](int slot, V pF) {
        int en = 0;
        V em = V(0);
        if (lane <= NB) {
            if constexpr (sizeof(V) == 4) {
                constexpr float L2h = 1.44269502162933349609375f;   // log2(e) rounded to FP32
                constexpr float L2l = 1.925963033500011e-08f;       // log2(e) - L2h
                const float af = (float)as_;
                const float ph = af * pF;
                const float pl = fmaf(af, pF, -ph);                 // a pF = ph + pl exactly
                const float th = ph * L2h;
                const float tl = fmaf(ph, L2h, -th) + fmaf(ph, L2l, pl * L2h);
                const float nth = floorf(th);
                const float fy = (th - nth) + tl;                  // a pF log2(e) = nth + fy
                const int nK = (int)(Kx >> 32);
                const float fK = (float)(unsigned)(Kx & 0xffffffffll) * 2.3283064365386963e-10f;
                const float cf = fK - fy;
                const float fl = floorf(cf);
                en = nK - (int)nth + (int)fl;
                em = exp2f(cf - fl);
            } else {
                const double c = Kd - (double)as_ * (double)pF * kLog2e;
                const double fl = floor(c);
                en = (int)fl;
                em = vexp2<V>((V)(c - fl));
            }
        }
        int Emax = INT_MIN / 2;
        V sum = V(0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int S = lane + 32 * q;
            const int s = popc_c(S);
            const int ens = __shfl_sync(FULL, en, s);
            const V ems = __shfl_sync(FULL, em, s);
            const Sf<V> fS = (S == 0) ? Sf<V>{V(0.5), 1} : rf.f[q];
            const int U = (NS - 1) ^ S;
            const Sf<V> gU = (U == 0) ? Sf<V>{V(0.5), 1} : sf_load<V>(__ldcg(Gt + (size_t)slot * NS + U));
            if (fS.m != V(0) && gU.m != V(0)) {
                const Sf<V> z = sf_make<V>(fS.m * gU.m * ems);
                const int E = z.k + fS.k + gU.k + ens;
                if (E > Emax) {
                    sum = fma(sum, pow2neg<V>(Emax - E), z.m);
                    Emax = E;
                } else {
                    sum = fma(z.m, pow2neg<V>(E - Emax), sum);
                }
            }
        }
        // across the warp
        int Ew = Emax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) Ew = max(Ew, __shfl_xor_sync(FULL, Ew, o));
        V sw = (sum > V(0)) ? sum * pow2neg<V>(Emax - Ew) : V(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sw += __shfl_xor_sync(FULL, sw, o);
        if (lane == 0) {
            tsw[slot] = sw;
            tew[slot] = Ew;
        }
    });
    __syncwarp();

    // FP64 epilogue, one target per lane: ln M = sum of the baselines +
    // Ew ln 2 + ln(sw)
    const int32_t off = a.cnt[(size_t)b * a.l + a.j];
    double qmax = -INFINITY;
    bool bad = false;
    double racc = 0.0;
    double oacc[4] = {0.0, 0.0, 0.0, 0.0};   // MODE_OBJ: mass, L1 error, g marg, g mu
    for (int slot = lane; slot < nt; slot += 32) {
        const V sw = tsw[slot];
        const double lnM = (sw > V(0)) ? sb + (double)tew[slot] * kLn2 + (double)vlog<V>(sw) : -INFINITY;
        const int i = off + slot;
        if (a.mode == MODE_UPDATE) {
            const double lm = a.lnmuj[i];
            double g = -INFINITY;
            if (lm > -INFINITY) {
                g = lm - lnM;
                if (!isfinite(g)) bad = true;
                qmax = fmax(qmax, (double)(V)g);
            }
            gq[slot] = g;
        } else if (a.mode == MODE_RESIDUAL) {
            const double gg = a.gj[i];
            const double marg = (gg == -INFINITY || lnM == -INFINITY) ? 0.0 : exp(gg * inv_eps_b + lnM);
            racc += fabs(marg - a.muj[i]);
        } else if (a.mode == MODE_OBJ) {
            const double gg = a.gj[i];
            const double mu = a.muj[i];
            const double marg = (gg == -INFINITY || lnM == -INFINITY) ? 0.0 : exp(gg * inv_eps_b + lnM);
            oacc[0] += marg;
            oacc[1] += fabs(marg - mu);
            if (gg != -INFINITY) {
                oacc[2] += gg * marg;
                oacc[3] += gg * mu;
            }
        } else if (a.mode == MODE_OUT_M) {
            a.out[i] = (lnM == -INFINITY) ? 0.0 : exp(lnM);
        } else if (a.mode == MODE_OUT_PLAN) {
            a.out[i] = (a.gj[i] == -INFINITY || lnM == -INFINITY) ? 0.0 : exp(a.gj[i] * inv_eps_b + lnM);
        } else {
            a.out[i] = lnM;
        }
    }
    if (a.mode == MODE_UPDATE) {
        // new potentials and ln phi relative to the new baseline, by lane
        // (each lane its points; the slot is the rank among the targets)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qmax = fmax(qmax, __shfl_xor_sync(FULL, qmax, o));
        bad = __any_sync(FULL, bad);
        const double bx = isfinite(qmax) ? qmax : 0.0;
        if (lane == 0) {
            if (bad) atomicOr(a.err, ERR_NONFINITE);
            if (nt > 0) a.beta[(size_t)b * a.l + a.j] = bx;
        }
        __syncwarp();
        V *lph = static_cast<V *>(a.lphi);
        int base = 0;
        for (int c0 = 0; c0 < n; c0 += 32) {
            const int r = c0 + lane;
            const bool tg = (r < n) && (a.mid[t0 + r] == a.j);
            const unsigned mask = __ballot_sync(FULL, tg);
            if (tg) {
                const int slot = base + __popc(mask & ((1u << lane) - 1u));
                const double g = gq[slot];
                a.gj[off + slot] = eps_b * g;
                lph[t0 + r] = (V)(g - bx);
            }
            base += __popc(mask);
        }
    } else if (a.mode == MODE_RESIDUAL) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) racc += __shfl_xor_sync(FULL, racc, o);
        if (lane == 0) a.partial[b] = racc;
    } else if (a.mode == MODE_OBJ) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) oacc[q] += __shfl_xor_sync(FULL, oacc[q], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) a.part4[(size_t)b * 4 + q] = oacc[q];
        }
    }
}

template <int NB, typename V>
cudaError_t launch_wpass_impl(const SweepArgs &a, cudaStream_t st, int SL, int fwd)
{
    k_wpass<NB, V><<<(a.nt + 3) / 4, 128, 0, st>>>(a, SL, fwd);
    return cudaGetLastError();
}

// Objective of l = NB marginals on warp tiles (all 2^l subsets, no target):
// W = <C, T> by the gap formula, as in objective.cuh.  The tile is taken in
// chunks of CH points: a backward walk from the tile's end keeps the
// backward states including each point of the chunk in shared memory, then
// the forward walk over the chunk adds, before each point's injection,
// (x_t - x_{t-1}) sum_S w_|S| F_S G_{S^c} with F_S G_{S^c} formed as
// mantissa x 2^exponent.  Per tile: partial[b] = eps W_b / Z_b, out[b] = ln Z.
template <int NB, typename V, int CH>
__global__ void __launch_bounds__(32) k_wobj(SweepArgs a)
{
    using R = WarpRun<NB, V, NB>;
    constexpr int NS = 1 << NB;
    constexpr int NQ = R::NQ;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char wsm[];
    SfT<V> *Gall = reinterpret_cast<SfT<V> *>(wsm);
    __shared__ V fbuf[32][16];
    __shared__ long long fxt[2 * NB + 1];
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const uint32_t t0 = a.tstart[b];
    const int n = (int)(a.tstart[b + 1] - t0);
    double beta[NB];
    warp_betas<NB>(a, b, a.j, beta);
    double sb = 0.0;
#pragma unroll
    for (int k = 0; k < NB; ++k) sb += beta[k];

    R rb;
    rb.init(a, b);
    rb.setup_fx(beta, fxt);
    R rf;
    rf.init(a, b);
    rf.fx = fxt;
    rf.load_carries(sfp<V>(a.fcarry), b, beta, NB + 1);
    // exp(gamma^F_s + gamma^G_{l-s} - w_s span) = mu_s 2^(n_s), by lane s
    int en = 0;
    V em = V(0);
    if (lane <= NB) {
        const int s = lane;
        if constexpr (sizeof(V) == 4) {
            long long g1 = 0, g2 = 0;
#pragma unroll
            for (int q = 0; q <= NB; ++q) {
                if (q == s) g1 = fxt[NB + q];
                if (q == NB - s) g2 = fxt[NB + q];
            }
            const long long X = g1 + g2 - fx_log2((double)R::rate(s) * (double)rf.span);
            en = (int)(X >> 32);
            em = exp2f((float)(unsigned)(X & 0xffffffffll) * 2.3283064365386963e-10f);
        } else {
            const double c = (rf.gam_at(s) + rb.gam_at(NB - s) - (double)R::rate(s) * (double)rf.span) * kLog2e;
            const double fl = floor(c);
            en = (int)fl;
            em = vexp2<V>((V)(c - fl));
        }
    }
    const bool first = (b == 0) || (a.seg && a.seg[b - 1] != a.seg[b]);
    const V gap0 = first ? V(0) : (V)(a.ulb[b] - a.urb[b - 1]);
    const V *pos = static_cast<const V *>(a.pos);
    Sf<V> accW = sf_zero<V>(), accZ = sf_zero<V>();
    for (int c0 = 0; c0 < n; c0 += CH) {
    const int c1 = min(n, c0 + CH);
    // backward states including each point of [c0, c1)
    rb.load_carries(sfp<V>(a.bcarry), b, beta, NB + 1);
    __syncwarp();
    warp_run_each<NB, V, NB, false>(rb, a, t0, n, false, 0, n - c0, fbuf, [&](int id, V) {
        if (id < c1) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) Gall[(size_t)(id - c0) * NS + lane + 32 * q] = sf_store(rb.f[q]);
        }
    });
    __syncwarp();
    warp_run_each<NB, V, NB, true>(rf, a, t0, n, true, c0, c1, fbuf, [&](int id, V) {
        int Emax = INT_MIN / 2;
        V sw = V(0), sz = V(0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int S = lane + 32 * q;
            const int s = popc_c(S);
            const int ens = __shfl_sync(FULL, en, s);
            const V ems = __shfl_sync(FULL, em, s);
            const Sf<V> fS = (S == 0) ? Sf<V>{V(0.5), 1} : rf.f[q];
            const int U = (NS - 1) ^ S;
            const Sf<V> gU = (U == 0) ? Sf<V>{V(0.5), 1} : sf_load<V>(Gall[(size_t)(id - c0) * NS + U]);
            if (fS.m != V(0) && gU.m != V(0)) {
                const Sf<V> z = sf_make<V>(fS.m * gU.m * ems);
                const int E = z.k + fS.k + gU.k + ens;
                const V wz = (V)R::rate(s) * z.m;
                if (E > Emax) {
                    const V r = pow2neg<V>(Emax - E);
                    sw = fma(sw, r, wz);
                    sz = fma(sz, r, z.m);
                    Emax = E;
                } else {
                    const V r = pow2neg<V>(E - Emax);
                    sw = fma(wz, r, sw);
                    sz = fma(z.m, r, sz);
                }
            }
        }
        int Ew = Emax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) Ew = max(Ew, __shfl_xor_sync(FULL, Ew, o));
        const V r = (sz > V(0)) ? pow2neg<V>(Emax - Ew) : V(0);
        V tw = sw * r, tz = sz * r;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tw += __shfl_xor_sync(FULL, tw, o);
            tz += __shfl_xor_sync(FULL, tz, o);
        }
        if (tz > V(0)) {
            const V dx = (id > 0) ? pos[t0 + id] - pos[t0 + id - 1] : gap0;
            Sf<V> t = sf_make<V>(dx * tw);
            t.k += Ew;
            if (t.m != V(0)) accW = sf_add(accW, t);
            if (id == 0) {
                accZ = sf_make<V>(tz);
                accZ.k += Ew;
            }
        }
    });
    }
    if (lane == 0) {
        if (accZ.m == V(0)) {
            a.partial[b] = 0.0;
            a.out[b] = -INFINITY;
        } else {
            const double rr = (accW.m == V(0)) ? 0.0 : ldexp((double)accW.m / (double)accZ.m, accW.k - accZ.k);
            a.partial[b] = tile_eps(a, b) * rr;
            a.out[b] = log((double)accZ.m) + (double)accZ.k * kLn2 + sb;
        }
    }
}

// objective launches for l = NB marginals on warp tiles of K points:
// kind 5 level pass, 6 level scan, 7 objective kernel
template <int NB, typename V, int K>
cudaError_t launch_wobj_impl(const SweepArgs &a, cudaStream_t st, int kind, int SL, int fwd)
{
    if (kind == 5) {
        k_wpass<NB, V, NB><<<(a.nt + 3) / 4, 128, 0, st>>>(a, SL, fwd);
        return cudaGetLastError();
    }
    if (kind == 6) {
        int nst = 0;
        for (int S = 1; S < (1 << NB); ++S)
            if (popc_c(S) == SL) ++nst;
        const dim3 grid(lscan_chunks(a.nt, nst), nst);
        k_lscan<NB, V, NB><<<grid, 256, 0, st>>>(a, SL, fwd);
        return cudaGetLastError();
    }
    if (kind == 7) {
        constexpr int CH = 16;   // points whose backward states are kept at once
        const size_t sz = (size_t)CH * (1 << NB) * sizeof(SfT<V>);
        auto kern = k_wobj<NB, V, CH>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz);
        if (e != cudaSuccess) return e;
        kern<<<a.nt, 32, sz, st>>>(a);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

template <int NB, typename V>
cudaError_t launch_wprod_impl(const SweepArgs &a, cudaStream_t st)
{
    k_wprod<NB, V><<<a.nt, 32, 0, st>>>(a);
    return cudaGetLastError();
}

template <int NB, typename V>
cudaError_t launch_wbwd_impl(const SweepArgs &a, cudaStream_t st)
{
    k_wbwd<NB, V><<<(a.nt + 3) / 4, 128, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mmot

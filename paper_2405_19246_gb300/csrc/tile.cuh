// Tile kernels of the three-phase marginal product for l <= 5 marginals
// (NB = l - 1 <= 4 state bits): the known-carry tile products with the FP64
// potential update (k_tile) and the carry-free tile transfer operators
// (k_tops).  The carries between tiles come from the carry scan (k_carry in
// sweep.cuh) over the operators these kernels store.
//
// What is computed (arXiv 2405.19246, Sec. 3 and Sec. 4.2).  For target j and
// every subset S of R = [l] \ {j} the forward state F_S(x) sums, over
// placements of one point of each marginal of S left of x, the product of
// their scalings times exp(-cost so far); between merged points every state
// with |S| = s decays at rate w_s = s(l - s), and a point of marginal m adds
// phi_m F_{S\m} to every S containing m (the class recurrences of Sec. 4.2
// with shared prefixes; Algorithm 2's lambda^2 multiplier is the l = 3 case).
// The backward states G are the mirror image, and
//     M_j(i) = sum_S F_S(x_i^-) G_{R\S}(x_i^+)        (Eq. Jk k margin).
//
// Layout of one tile (one CTA): NT threads (NW = NT / 32 warps), each lane
// owns C consecutive points of the merged order, kept in registers:
//   ph = phi_m e^{-beta_m}   (beta_m the tile maximum of g_m/eps; <= 1),
//   pe = e^{pos}, pm = e^{-pos}   (pos = (x - x_first_of_tile)/eps),
//   the marginal of the point.
// The stream is stored this way (exponentials, padded so that every tile
// starts on a 16-element boundary), so a point costs no transcendental and
// the injection factors keep FP32 relative accuracy: in the cumulative frame
// of the tile (no decay between points) the factor of a level-s injection is
//     fac_s = ph * e^{a_s p} * e^{-max(0, a_s span)},   a_s = w_s - w_{s-1},
// with p = pos forward and span - pos backward, and it is at most 1.
//
// One pass (backward or forward) over the tile with known tile carries:
//  1. every lane computes its chunk's transfer operator op[s][V] (unit state
//     of level s at the chunk start reaching level s + |V| with the marginals
//     V added), one walk;
//  2. level by level, every state T of level s gets its chunk-local value
//     from the operator and the chunk-start values of the lower levels, a
//     warp scan plus one cross-warp step gives each lane its chunk-start
//     value, and the tile-end value fixes the state's power-of-two scale (each
//     state its own scale: states of one level may differ by more than the
//     FP32 range on sparse supports at small eps);
//  3. a second walk with the chunk-start values produces the states at every
//     point: the backward pass keeps G at the target points in shared memory,
//     the forward pass combines with them.
// Then the FP64 epilogue (potential update, residual or output) and, after an
// update, the transfer operators of the next target from the new potentials
// (one walk computing the forward and the backward operator, composed over
// the lanes and warps), stored for the next carry scan.
#pragma once
#include "shapes.cuh"
#include "sweep.cuh"

namespace mmot {

// ---- double-FP32 (hi + lo) arithmetic ------------------------------------------
// Used where an FP32 value must carry more than 24 bits (ln mu minus a large
// baseline, the exponent of a new scaling) without FP64 instructions, whose
// rate on this GPU is a small fraction of FP32.
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 f2_fast_two_sum(float a, float b)
{
    const float s = a + b;
    return F2{s, b - (s - a)};
}
__device__ __forceinline__ F2 f2_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return F2{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    const F2 s = f2_two_sum(a.hi, b.hi);
    return f2_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ F2 f2_neg(F2 a) { return F2{-a.hi, -a.lo}; }
__device__ __forceinline__ F2 f2_from_double(double x)
{
    const float h = (float)x;
    return F2{h, (float)(x - (double)h)};
}

// ln 2 split so that k * kLn2Hi is exact for |k| < 2^12, and log2(e) as hi + lo
constexpr float kLn2Hi = 0.693115234375f;   // 2839 / 4096
constexpr float kLn2Lo = (float)(0.69314718055994530942 - 0.693115234375);
constexpr float kLog2eHi = (float)1.4426950408889634074;
constexpr float kLog2eLo = (float)(1.4426950408889634074 - (double)(float)1.4426950408889634074);

// e^x for x = hi + lo given as double-FP32, to FP32 accuracy for any |x| the
// FP32 range allows: exp2 of the rounded x log2(e) times a first-order
// correction for the rest.
__device__ __forceinline__ float f2_exp(F2 x)
{
    const float y = x.hi * kLog2eHi;
    const float ye = fmaf(x.hi, kLog2eHi, -y) + fmaf(x.hi, kLog2eLo, x.lo * kLog2eHi);
    return exp2f(y) * fmaf(ye, 0.69314718f, 1.0f);
}

// 2^d as V for an integer d (0 below the normal range, the largest finite
// power of two above it)
template <typename V>
__device__ __forceinline__ V pow2i(int d);
template <>
__device__ __forceinline__ float pow2i<float>(int d)
{
    d = max(-127, min(127, d));
    return (d == -127) ? 0.f : __int_as_float((d + 127) << 23);
}
template <>
__device__ __forceinline__ double pow2i<double>(int d)
{
    d = max(-1023, min(1023, d));
    return (d == -1023) ? 0.0 : __longlong_as_double((long long)(d + 1023) << 52);
}

// ---- compile-time subset bookkeeping -------------------------------------------
// op[s][V] is valid for V != 0 and s + |V| <= NB (s < NB).
template <int NB>
__host__ __device__ constexpr bool op_ok(int s, int V)
{
    return V != 0 && s < NB && s + popc_c(V) <= NB;
}

// Forward operator, one point of bit k (runtime) appended on the right:
//   F[s][V] += [k in V] fac[s + |V|] F[s][V \ k]   (F[s][0] = 1).
// k < 0 (target, padding) leaves F unchanged.  Branch-free: the lanes of a
// warp hold points of different marginals.
template <int NB, typename V>
__device__ __forceinline__ void op_push_right(V (&op)[NB][1 << NB], int k, const V (&fac)[NB + 1])
{
    constexpr int NS = 1 << NB;
    static_for<0, NB>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        static_for<1, NS>([&](auto vc) {
            constexpr int Vv = decltype(vc)::value;
            if constexpr (op_ok<NB>(s, Vv)) {
                V src = V(0);
                static_for<0, NB>([&](auto kc) {
                    constexpr int kb = decltype(kc)::value;
                    if constexpr ((Vv >> kb) & 1) {
                        constexpr int W = Vv ^ (1 << kb);
                        if constexpr (W == 0)
                            src = (k == kb) ? V(1) : src;
                        else
                            src = (k == kb) ? op[s][W] : src;
                    }
                });
                op[s][Vv] = fma(fac[s + popc_c(Vv)], src, op[s][Vv]);
            }
        });
    });
}

// Backward operator built in forward point order: the new point is the first
// one the backward pass meets, so it is composed on the left:
//   B[s][V] += [k in V] fac[s + 1] B[s + 1][V \ k]   (B[.][0] = 1).
template <int NB, typename V>
__device__ __forceinline__ void op_push_left(V (&op)[NB][1 << NB], int k, const V (&fac)[NB + 1])
{
    constexpr int NS = 1 << NB;
    static_for<0, NB>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        static_for<1, NS>([&](auto vc) {
            constexpr int Vv = decltype(vc)::value;
            if constexpr (op_ok<NB>(s, Vv)) {
                V src = V(0);
                static_for<0, NB>([&](auto kc) {
                    constexpr int kb = decltype(kc)::value;
                    if constexpr ((Vv >> kb) & 1) {
                        constexpr int W = Vv ^ (1 << kb);
                        if constexpr (W == 0)
                            src = (k == kb) ? V(1) : src;
                        else
                            src = (k == kb) ? op[s + 1][W] : src;
                    }
                });
                op[s][Vv] = fma(fac[s + 1], src, op[s][Vv]);
            }
        });
    });
}

// R = X then Y (X applied first)
template <int NB, typename V>
__device__ __forceinline__ void op_compose(const V (&X)[NB][1 << NB], const V (&Y)[NB][1 << NB], V (&R)[NB][1 << NB])
{
    constexpr int NS = 1 << NB;
    static_for<0, NB>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        static_for<1, NS>([&](auto vc) {
            constexpr int Vv = decltype(vc)::value;
            if constexpr (op_ok<NB>(s, Vv)) {
                V r = X[s][Vv] + Y[s][Vv];
                static_for<1, NS>([&](auto wc) {
                    constexpr int W1 = decltype(wc)::value;
                    if constexpr ((W1 & ~Vv) == 0 && W1 != Vv) r = fma(X[s][W1], Y[s + popc_c(W1)][Vv ^ W1], r);
                });
                R[s][Vv] = r;
            }
        });
    });
}

template <int NB, typename V>
__device__ __forceinline__ void op_zero(V (&op)[NB][1 << NB])
{
#pragma unroll
    for (int s = 0; s < NB; ++s)
#pragma unroll
        for (int U = 0; U < (1 << NB); ++U) op[s][U] = V(0);
}

template <int NB, typename V>
__device__ __forceinline__ void op_shfl_xor(const V (&X)[NB][1 << NB], V (&Y)[NB][1 << NB], int o)
{
    static_for<0, NB>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        static_for<1, (1 << NB)>([&](auto vc) {
            constexpr int Vv = decltype(vc)::value;
            if constexpr (op_ok<NB>(s, Vv)) Y[s][Vv] = __shfl_xor_sync(0xffffffffu, X[s][Vv], o);
        });
    });
}

// Butterfly over the lanes of a warp: every lane ends with the composition of
// the warp's operators in lane order (fwd: lane 0 first; otherwise lane 31
// first, the order of the backward pass).  At each step the pair's operators
// X (this lane's) and Y (the partner's) are composed with the lower-ordered
// one first; the operand selection is folded into the terms.
template <int NB, typename V>
__device__ __forceinline__ void op_warp_reduce(V (&op)[NB][1 << NB], bool lane_order)
{
    constexpr int NS = 1 << NB;
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int o = 1; o < 32; o <<= 1) {
        V Y[NB][NS];
        op_shfl_xor<NB, V>(op, Y, o);
        const bool first = (((lane & o) == 0) == lane_order);   // this lane's operator is applied first
        V R[NB][NS];
        static_for<0, NB>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            static_for<1, NS>([&](auto vc) {
                constexpr int Vv = decltype(vc)::value;
                if constexpr (op_ok<NB>(s, Vv)) {
                    V r = op[s][Vv] + Y[s][Vv];
                    static_for<1, NS>([&](auto wc) {
                        constexpr int W1 = decltype(wc)::value;
                        if constexpr ((W1 & ~Vv) == 0 && W1 != Vv) {
                            constexpr int s2 = s + popc_c(W1);
                            const V a1 = first ? op[s][W1] : Y[s][W1];
                            const V b1 = first ? Y[s2][Vv ^ W1] : op[s2][Vv ^ W1];
                            r = fma(a1, b1, r);
                        }
                    });
                    R[s][Vv] = r;
                }
            });
        });
        static_for<0, NB>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            static_for<1, NS>([&](auto vc) {
                constexpr int Vv = decltype(vc)::value;
                if constexpr (op_ok<NB>(s, Vv)) op[s][Vv] = R[s][Vv];
            });
        });
    }
}

// number of valid operator entries
template <int NB>
__host__ __device__ constexpr int op_count()
{
    int c = 0;
    for (int s = 0; s < NB; ++s)
        for (int U = 1; U < (1 << NB); ++U)
            if (op_ok<NB>(s, U)) ++c;
    return c;
}

template <int NB, typename V, int NT, int JCAP>
struct TileSm {
    static constexpr int NS = 1 << NB;
    static constexpr int NW = NT / 32;
    static constexpr int NOP = op_count<NB>();
    V wsum[NW][NS];       // warp totals of a level scan
    int wcnt[NW];         // target points per warp
    int wbits[NW];        // marginals (as bits of the target's mapping) present per warp
    float wmax[NW];       // warp maxima of the new g/eps
    double dred[NW];      // FP64 reduction scratch
    int eB[NS];           // scales of the backward states
    V csc[NS];            // combine: kappa_|S| 2^{E_S - Emax} of every term
    int esx[NS];          // combine: E_S - Emax
    V kap[NB + 1];        // combine: mantissas of kappa_s
    int emax;             // combine: largest term exponent
    int fast;             // combine: every term within 2^60 of the largest
    // per target slot: ln M as mantissa (lmx) and binary exponent (lme) after
    // the combine; the new scaled phi and ln phi after the update
    alignas(16) V lmx[JCAP];
    int lme[JCAP];
    // backward states at the target slots (state U at row U - 1); after the
    // combine, the warps' transfer operators
    static constexpr int GSZ = (NS - 1) * JCAP;
    static constexpr int OSZ = NW * 2 * NB * NS;
    alignas(16) V buf[GSZ > OSZ ? GSZ : OSZ];
    // forward states (state S at row S - 1) and e^{pos} at the target slots:
    // the combine runs by slot after the forward walk, so a warp does not
    // run it at every chunk position where one of its lanes has a target
    alignas(16) V fst[(NS - 1) * JCAP];
    V tpe[JCAP];
};

// Per-tile constants of one pass, identical in every lane.
template <int NB, typename V>
struct PassC {
    V cf[NB + 1];      // e^{-max(0, a_s span)} forward / e^{min(0, a_s span)} backward, s = 1..NB
    int e[1 << NB];    // final binary scale of every state (e[0] = 0)
};

template <int NB, typename V, int NT, int C, int JCAP, bool WITH_NEXT>
struct TileRun {
    static constexpr int NS = 1 << NB;
    static constexpr int NW = NT / 32;
    static constexpr int L = NB + 1;
    static constexpr int K = NT * C;
    static constexpr unsigned FULL = 0xffffffffu;
    using Sm = TileSm<NB, V, NT, JCAP>;

    int lane, w, tid;
    int n;            // points in the tile
    V span;
    V ph[C], pe[C], pm[C];
    unsigned mdw[(C + 3) / 4];   // marginal of each point, 4 per word (0xff: padding)
    int bt[C];        // bit of the point for the current target (-1 target, -2 none)

    __device__ static constexpr int rate(int s) { return s * (L - s); }

    // the lane's C points: e^{pos}, e^{-pos}, scaled phi and marginal, and the
    // bit of each point for target j
    __device__ __forceinline__ void load(const SweepArgs &a, int b, uint32_t t0, int i0, int j)
    {
        const V *epos = static_cast<const V *>(a.epos);
        const V *ephi = static_cast<const V *>(a.ephi);
        if (i0 < n) {
            constexpr int PV = 16 / sizeof(V);   // values per 16-byte load
            static_assert(C % PV == 0 || C < PV, "chunk of whole 16-byte pieces");
            if constexpr (C >= PV) {
#pragma unroll
                for (int q = 0; q < C / PV; ++q) {
                    const uint4 u = __ldg(reinterpret_cast<const uint4 *>(epos + t0 + i0) + q);
                    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(ephi + t0 + i0) + q);
                    memcpy(&pe[q * PV], &u, 16);
                    memcpy(&ph[q * PV], &v, 16);
                }
            } else {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    pe[c] = epos[t0 + i0 + c];
                    ph[c] = ephi[t0 + i0 + c];
                }
            }
            if constexpr (C == 16) {
                const uint4 u = __ldg(reinterpret_cast<const uint4 *>(a.emid + t0 + i0));
                mdw[0] = u.x;
                mdw[1] = u.y;
                mdw[2] = u.z;
                mdw[3] = u.w;
            } else if constexpr (C == 8) {
                const uint2 u = __ldg(reinterpret_cast<const uint2 *>(a.emid + t0 + i0));
                mdw[0] = u.x;
                mdw[1] = u.y;
            } else if constexpr (C == 4) {
                mdw[0] = __ldg(reinterpret_cast<const unsigned *>(a.emid + t0 + i0));
            } else {
                unsigned w0 = 0xffffffffu;
#pragma unroll
                for (int c = 0; c < C; ++c) w0 = (w0 & ~(0xffu << (8 * c))) | ((unsigned)a.emid[t0 + i0 + c] << (8 * c));
                mdw[0] = w0;
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                pe[c] = V(1);
                ph[c] = V(0);
            }
#pragma unroll
            for (int q = 0; q < (C + 3) / 4; ++q) mdw[q] = 0xffffffffu;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            pm[c] = V(1) / pe[c];
            bt[c] = bit_of(mid_of(c), j);
        }
    }

    __device__ __forceinline__ int mid_of(int c) const { return (mdw[c >> 2] >> (8 * (c & 3))) & 0xff; }

    __device__ __forceinline__ static int bit_of(int m, int j) { return (m == 0xff) ? -2 : (m == j ? -1 : (m < j ? m : m - 1)); }
    __device__ static constexpr int arate(int s) { return rate(s) - rate(s - 1); }   // L + 1 - 2s

    // e^{a p} for the point in the pass frame: forward p = pos (pe^a),
    // backward p = span - pos (e^{a span} pm^a; the e^{a span} is in cf)
    template <bool FWD>
    __device__ __forceinline__ void facs(int c, const PassC<NB, V> &P, V (&f)[NB + 1]) const
    {
        const V up = FWD ? pe[c] : pm[c];
        const V dn = FWD ? pm[c] : pe[c];
        // a_s = L + 1 - 2 s = NB + 2 - 2 s: NB, NB - 2, ..., 2 - NB
        const V up2 = up * up, dn2 = dn * dn;
        V pw[NB + 1];
        static_for<1, NB + 1>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            constexpr int a = arate(s);
            V x;
            if constexpr (a == 0) x = V(1);
            else if constexpr (a == 1) x = up;
            else if constexpr (a == 2) x = up2;
            else if constexpr (a == 3) x = up2 * up;
            else if constexpr (a == 4) x = up2 * up2;
            else if constexpr (a == -1) x = dn;
            else if constexpr (a == -2) x = dn2;
            else if constexpr (a == -3) x = dn2 * dn;
            else x = dn2 * dn2;
            pw[s] = x;
        });
        f[0] = V(0);
        static_for<1, NB + 1>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            f[s] = (ph[c] * P.cf[s]) * pw[s];
        });
    }

    __device__ __forceinline__ void setup_consts(PassC<NB, V> &P, bool fwd) const
    {
        P.cf[0] = V(1);
#pragma unroll
        for (int s = 1; s <= NB; ++s) {
            const V as = (V)arate(s) * span;
            P.cf[s] = fwd ? vexp<V>(-(as > V(0) ? as : V(0))) : vexp<V>(as < V(0) ? as : V(0));
        }
#pragma unroll
        for (int S = 0; S < NS; ++S) P.e[S] = 0;
    }

    // Steps 1-2 of a pass: chunk-start values x[] (final per-state scales in
    // P.e) from the tile carries.  cu: on lane T < NS, the carry of state T in
    // the unscaled tile frame (carry e^{-(sum beta_T + Gamma_|T|)}).
    // Provisional scale of state T: the largest final scale among the lower
    // states U that can reach T inside this tile (every marginal of T \ U
    // has points in the tile: bits), plus headroom for the in-tile sums.  A
    // source that cannot inject must not set the scale: its size would push
    // the real contributions out of range (sparse supports at small eps).
    __device__ __forceinline__ static int prov_scale(int T, const int (&e)[NS], int bits)
    {
        int m = INT_MIN;
#pragma unroll
        for (int U = 0; U < NS; ++U)
            if ((U & ~T) == 0 && U != T && ((T ^ U) & ~bits) == 0) m = max(m, e[U]);
        return (m == INT_MIN) ? 0 : m + 32;
    }

    template <bool FWD>
    __device__ __forceinline__ void chunk_starts(Sm &sm, PassC<NB, V> &P, const Sf<V> cu, V (&x)[NS], int bits)
    {
        __syncthreads();   // the previous pass has finished reading sm.wsum
        // 1. chunk operator
        V op[NB][NS];
        op_zero<NB, V>(op);
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const int c = FWD ? i : C - 1 - i;
            V f[NB + 1];
            facs<FWD>(c, P, f);
            op_push_right<NB, V>(op, bt[c], f);
        }
        x[0] = V(1);
        // 2. level by level
        static_for<1, NB + 1>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            // provisional scale of each state of the level: the largest final
            // scale of its lower states plus headroom for the in-tile sums
            int pi[NS];
            V loc[NS];
            static_for<1, NS>([&](auto tc) {
                constexpr int T = decltype(tc)::value;
                if constexpr (popc_c(T) == s) {
                    pi[T] = prov_scale(T, P.e, bits);
                    V acc = op[0][T] * pow2i<V>(-pi[T]);
                    static_for<1, NS>([&](auto uc) {
                        constexpr int U = decltype(uc)::value;
                        if constexpr ((U & ~T) == 0 && U != T)
                            acc = fma(x[U] * pow2i<V>(P.e[U] - pi[T]), op[popc_c(U)][T ^ U], acc);
                    });
                    loc[T] = acc;
                }
            });
            // warp scan (inclusive, in pass order: ascending lanes forward,
            // descending backward) and warp totals
            V ex[NS];
            static_for<1, NS>([&](auto tc) {
                constexpr int T = decltype(tc)::value;
                if constexpr (popc_c(T) == s) {
                    V incl = loc[T];
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        if constexpr (FWD) {
                            const V y = __shfl_up_sync(FULL, incl, o);
                            if (lane >= o) incl += y;
                        } else {
                            const V y = __shfl_down_sync(FULL, incl, o);
                            if (lane + o < 32) incl += y;
                        }
                    }
                    // exclusive prefix by a shift, not incl - loc: the
                    // difference would lose a small prefix next to a large
                    // own value (sparse supports)
                    if constexpr (FWD) {
                        const V y = __shfl_up_sync(FULL, incl, 1);
                        ex[T] = (lane == 0) ? V(0) : y;
                    } else {
                        const V y = __shfl_down_sync(FULL, incl, 1);
                        ex[T] = (lane == 31) ? V(0) : y;
                    }
                    if (lane == (FWD ? 31 : 0)) sm.wsum[w][T] = incl;
                }
            });
            __syncthreads();
            // carry of each state of the level in its provisional frame, the
            // tile-end value and the final scale: lane T computes state T
            int eT = 0;
            Sf<V> cp = sf_zero<V>();
            if (lane < NS && popc_c(lane) == s) {
                const int T = lane;
                int piT = 0;
#pragma unroll
                for (int T2 = 1; T2 < NS; ++T2)
                    if (T2 == T) piT = prov_scale(T2, P.e, bits);
                cp = cu;
                if (cp.m != V(0)) cp.k -= piT;
                V Z = V(0);
#pragma unroll
                for (int q = 0; q < NW; ++q) Z += sm.wsum[q][T];
                const Sf<V> R = sf_add(cp, sf_make<V>(Z));
                eT = (R.m == V(0)) ? piT : piT + R.k;
            }
            static_for<1, NS>([&](auto tc) {
                constexpr int T = decltype(tc)::value;
                if constexpr (popc_c(T) == s) {
                    P.e[T] = __shfl_sync(FULL, eT, T);
                    Sf<V> c;
                    c.m = __shfl_sync(FULL, cp.m, T);
                    c.k = __shfl_sync(FULL, cp.k, T);
                    V wp = V(0);
#pragma unroll
                    for (int q = 0; q < NW; ++q)
                        if (FWD ? (q < w) : (q > w)) wp += sm.wsum[q][T];
                    const Sf<V> v = sf_add(c, sf_make<V>(wp + ex[T]));
                    x[T] = sf_value(v, P.e[T] - pi[T]);
                }
            });
        });
    }
};


// ---- transfer operators of one target ----------------------------------------
// Forward and backward operators of tile b for target jn from the points in
// the lanes' registers (one walk; the backward operator is built in forward
// order by composing on the left), composed over the lanes and warps, turned
// into absolute scaled floats with the decay to the next tile base (processing
// order) and stored for the carry scan:
//   op[b][s][U] = T_b[s][U] exp(sum_{m in U} beta_m + Gamma_{s+|U|} - Gamma_s - w_{s+|U|} d)
// (T_b in the unscaled tile frame; d the distance to the next base).
template <int NB, typename V, int NT, int C, int JCAP>
__device__ __forceinline__ void tile_ops_body(TileRun<NB, V, NT, C, JCAP, true> &r, TileSm<NB, V, NT, JCAP> &sm, const SweepArgs &a,
                              int b, int jn)
{
    using R = TileRun<NB, V, NT, C, JCAP, true>;
    constexpr int NS = 1 << NB;
    constexpr int NW = NT / 32;
    constexpr int L = NB + 1;
    const int lane = r.lane, w = r.w;
    PassC<NB, V> PF, PB;
    r.setup_consts(PF, true);
    r.setup_consts(PB, false);
    V opf[NB][NS], opb[NB][NS];
    op_zero<NB, V>(opf);
    op_zero<NB, V>(opb);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int k = R::bit_of(r.mid_of(c), jn);
        V ff[NB + 1], fb[NB + 1];
        r.template facs<true>(c, PF, ff);
        r.template facs<false>(c, PB, fb);
        op_push_right<NB, V>(opf, k, ff);
        op_push_left<NB, V>(opb, k, fb);
    }
    op_warp_reduce<NB, V>(opf, true);
    op_warp_reduce<NB, V>(opb, false);
    V *sc = sm.buf;   // [NW][2][NB][NS]
    if (lane == 0) {
        static_for<0, NB>([&](auto scc) {
            constexpr int s = decltype(scc)::value;
            static_for<1, NS>([&](auto vc) {
                constexpr int U = decltype(vc)::value;
                if constexpr (op_ok<NB>(s, U)) {
                    sc[((w * 2 + 0) * NB + s) * NS + U] = opf[s][U];
                    sc[((w * 2 + 1) * NB + s) * NS + U] = opb[s][U];
                }
            });
        });
    }
    __syncthreads();
    if (w != 0) return;
    static_for<0, NB>([&](auto scc) {
        constexpr int s = decltype(scc)::value;
        static_for<1, NS>([&](auto vc) {
            constexpr int U = decltype(vc)::value;
            if constexpr (op_ok<NB>(s, U)) {
                opf[s][U] = (lane < NW) ? sc[((lane * 2 + 0) * NB + s) * NS + U] : V(0);
                opb[s][U] = (lane < NW) ? sc[((lane * 2 + 1) * NB + s) * NS + U] : V(0);
            }
        });
    });
    op_warp_reduce<NB, V>(opf, true);
    op_warp_reduce<NB, V>(opb, false);
    // baselines of target jn's bits (beta of the current target just written
    // by this block is visible after the barrier above)
    const int l = a.l;
    double beta[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        const int m = (k < jn) ? k : k + 1;
        const int rt = __ldg(a.reftile + (size_t)b * l + m);
        beta[k] = *(volatile const double *)(a.beta + (size_t)rt * l + m);
    }
    double Gam[NB + 1];
    Gam[0] = 0.0;
#pragma unroll
    for (int s = 1; s <= NB; ++s) {
        const V as = (V)R::arate(s) * r.span;
        Gam[s] = Gam[s - 1] + (double)(as > V(0) ? as : V(0));
    }
    double dF = 0.0, dB = 0.0;
    bool cutF = true, cutB = true;
    if (b + 1 < a.nt) {
        dF = a.ulb[b + 1] - a.ulb[b];
        cutF = a.seg && a.seg[b + 1] != a.seg[b];
    }
    if (b >= 1) {
        dB = a.urb[b] - a.urb[b - 1];
        cutB = a.seg && a.seg[b - 1] != a.seg[b];
    }
    // entries are spread over the lanes: entry e (both directions, [dir][s][U])
    // goes to lane e % 32
    constexpr int NE = 2 * NB * NS;
    constexpr int PER = (NE + 31) / 32;
    V val[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) val[q] = V(0);
    static_for<0, NB>([&](auto scc) {
        constexpr int s = decltype(scc)::value;
        static_for<1, NS>([&](auto vc) {
            constexpr int U = decltype(vc)::value;
            if constexpr (op_ok<NB>(s, U)) {
                constexpr int eF = (0 * NB + s) * NS + U, eB = (1 * NB + s) * NS + U;
                if (lane == eF % 32) val[eF / 32] = opf[s][U];
                if (lane == eB % 32) val[eB / 32] = opb[s][U];
            }
        });
    });
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = q * 32 + lane;
        if (e >= NE) continue;
        const int dir = e / (NB * NS), s = (e / NS) % NB, U = e % NS;
        if (U == 0 || s + __popc(U) > NB) continue;
        const int su = s + __popc(U);
        double bu = 0.0;
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if ((U >> k) & 1) bu += beta[k];
        const double d = dir ? dB : dF;
        const bool cut = dir ? cutB : cutF;
        const double wsu = (double)su * (double)(L - su);
        double gsu = 0.0, gs = 0.0;
#pragma unroll
        for (int t = 0; t <= NB; ++t) {
            if (t == su) gsu = Gam[t];
            if (t == s) gs = Gam[t];
        }
        const Sf<V> o = cut ? sf_zero<V>() : sf_scale_exp(sf_make<V>(val[q]), bu + gsu - gs - wsu * d);
        sfp<V>(dir ? a.opB : a.opF)[((size_t)b * NB + s) * NS + U] = sf_store(o);
    }
}

// Transfer operators of every tile for target a.j (when the stored ones
// belong to another target).
template <int NB, typename V, int NT, int C, int JCAP>
__global__ void __launch_bounds__(NT, sizeof(V) == 4 ? 2 : 1) k_tops(SweepArgs a)
{
    using R = TileRun<NB, V, NT, C, JCAP, true>;
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    TileSm<NB, V, NT, JCAP> &sm = *reinterpret_cast<TileSm<NB, V, NT, JCAP> *>(tsm_raw);
    const int b = blockIdx.x;
    R r;
    r.tid = threadIdx.x;
    r.lane = r.tid & 31;
    r.w = r.tid >> 5;
    r.n = (int)(a.tstart[b + 1] - a.tstart[b]);
    r.span = (V)a.span[b];
    r.load(a, b, a.toff[b], r.tid * C, a.j);
    tile_ops_body<NB, V, NT, C, JCAP>(r, sm, a, b, a.j);
}

// ---- the tile product ------------------------------------------------------------

template <int NB, typename V, int NT, int C, int JCAP>
__global__ void __launch_bounds__(NT, sizeof(V) == 4 ? 2 : 1) k_tile(SweepArgs a)
{
    using R = TileRun<NB, V, NT, C, JCAP, true>;
    using Sm = typename R::Sm;
    constexpr int NS = 1 << NB;
    constexpr int FULLS = NS - 1;
    constexpr int NW = NT / 32;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    Sm &sm = *reinterpret_cast<Sm *>(tsm_raw);
    const int b = blockIdx.x;
    if (skip_tile(a, b)) return;
    R r;
    r.tid = threadIdx.x;
    r.lane = r.tid & 31;
    r.w = r.tid >> 5;
    const int tid = r.tid, lane = r.lane, w = r.w;
    const uint32_t ts = a.tstart[b];
    r.n = (int)(a.tstart[b + 1] - ts);
    r.span = (V)a.span[b];
    const uint32_t t0 = a.toff[b];
    const int i0 = tid * C;   // first tile-local index of this lane's chunk
    const int j = a.j;
    const int l = a.l;

    r.load(a, b, t0, i0, j);

    // ---- target slots (rank among the tile's targets, forward order) -------
    int tcount = 0;
#pragma unroll
    for (int c = 0; c < C; ++c) tcount += (r.bt[c] == -1);
    int tincl = tcount;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, tincl, o);
        if (lane >= o) tincl += y;
    }
    if (lane == 31) sm.wcnt[w] = tincl;
    int lbits = 0;
#pragma unroll
    for (int c = 0; c < C; ++c)
        if (r.bt[c] >= 0) lbits |= 1 << r.bt[c];
    lbits = __reduce_or_sync(FULL, lbits);
    if (lane == 0) sm.wbits[w] = lbits;
    // per-tile FP64 constants: baselines of the marginals mapped to bits
    double beta[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        const int m = (k < j) ? k : k + 1;
        const int rt = __ldg(a.reftile + (size_t)b * l + m);
        beta[k] = *(volatile const double *)(a.beta + (size_t)rt * l + m);
    }
    __syncthreads();
    int slot0 = tincl - tcount;   // first slot of this lane's targets
    int ntarget = 0;
    int bits = 0;                 // marginals (as bits) with points in the tile
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        const int cq = sm.wcnt[q];
        if (q < w) slot0 += cq;
        ntarget += cq;
        bits |= sm.wbits[q];
    }
    if (ntarget > JCAP) {
        if (tid == 0) atomicOr(a.err, ERR_RANGE);
        return;
    }
    // Gamma_s = D_1 + ... + D_s, D_s = max(0, a_s span)
    double Gam[NB + 1];
    Gam[0] = 0.0;
#pragma unroll
    for (int s = 1; s <= NB; ++s) {
        const V as = (V)R::arate(s) * r.span;
        Gam[s] = Gam[s - 1] + (double)(as > V(0) ? as : V(0));
    }
    auto gam_at = [&](int S) {
        double g = 0.0;
        const int ps = __popc(S);
#pragma unroll
        for (int q = 0; q <= NB; ++q)
            if (q == ps) g = Gam[q];
        return g;
    };
    auto sum_beta = [&](int S) {
        double x = 0.0;
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if ((S >> k) & 1) x += beta[k];
        return x;
    };

    // ---- backward pass: G at the target points -------------------------------
    PassC<NB, V> PB;
    r.setup_consts(PB, false);
    V x[NS];
    {
        Sf<V> cu = sf_zero<V>();
        if (lane < NS && lane > 0) {
            cu = sf_load<V>(sfp<V>(a.bcarry)[(size_t)b * NS + lane]);
            cu = sf_scale_exp(cu, -(sum_beta(lane) + gam_at(lane)));
        }
        r.template chunk_starts<false>(sm, PB, cu, x, bits);
    }
    {
        // ratios 2^{e_{T\k} - e_T} of the injections
        V rr[NS][NB];
        static_for<1, NS>([&](auto tc) {
            constexpr int T = decltype(tc)::value;
            static_for<0, NB>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                if constexpr ((T >> k) & 1) rr[T][k] = pow2i<V>(PB.e[T ^ (1 << k)] - PB.e[T]);
            });
        });
        V f[NS];
#pragma unroll
        for (int S = 0; S < NS; ++S) f[S] = x[S];
        int slot = slot0 + tcount - 1;
#pragma unroll
        for (int i = 0; i < C; ++i) {
            const int c = C - 1 - i;
            const int k = r.bt[c];
            if (k == -1) {
                if (slot < JCAP) {
#pragma unroll
                    for (int U = 1; U < NS; ++U) sm.buf[(U - 1) * JCAP + slot] = f[U];
                }
                --slot;
            }
            V fc[NB + 1];
            r.template facs<false>(c, PB, fc);
            static_for<1, NS>([&](auto tc) {
                constexpr int T = decltype(tc)::value;
                V src = V(0), rat = V(0);
                static_for<0, NB>([&](auto kc) {
                    constexpr int kb = decltype(kc)::value;
                    if constexpr ((T >> kb) & 1) {
                        src = (k == kb) ? f[T ^ (1 << kb)] : src;
                        rat = (k == kb) ? rr[T][kb] : rat;
                    }
                });
                f[T] = fma(fc[popc_c(T)] * rat, src, f[T]);
            });
        }
#pragma unroll
        for (int S = 0; S < NS; ++S)
            if (tid == S) sm.eB[S] = PB.e[S];   // (a runtime index would put PB in local memory)
    }
    // (the chunk_starts barriers of the forward pass order these writes
    // before the combine reads them)

    // ---- forward pass and combine ------------------------------------------------
    PassC<NB, V> PF;
    r.setup_consts(PF, true);
    {
        Sf<V> cu = sf_zero<V>();
        if (lane < NS && lane > 0) {
            cu = sf_load<V>(sfp<V>(a.fcarry)[(size_t)b * NS + lane]);
            cu = sf_scale_exp(cu, -(sum_beta(lane) + gam_at(lane)));
        }
        r.template chunk_starts<true>(sm, PF, cu, x, bits);
    }
    // Per term S: F_S G_{R\S} = f g 2^{eF_S + eB_{R\S}} e^{sum beta_R} kappa_s e^{-(2s - NB) pos},
    // kappa_s = e^{Gamma_s + Gamma_{NB-s} - w_{NB-s} span}.  Terms in units of
    // 2^Emax, Emax the largest exponent over S (warp 0 computes the tile
    // constants; the barrier also orders the backward states before the
    // combine reads them).
    if (w == 0) {
        int kapk = 0;
        V kapm = V(0);
        if (lane <= NB) {
            const int s = lane;
            double g1 = 0.0, g2 = 0.0;
#pragma unroll
            for (int q = 0; q <= NB; ++q) {
                if (q == s) g1 = Gam[q];
                if (q == NB - s) g2 = Gam[q];
            }
            const double lk = g1 + g2 - (double)((NB - s) * (R::L - (NB - s))) * (double)r.span;
            const Sf<V> kk = sf_scale_exp(Sf<V>{V(0.5), 1}, lk);
            kapm = kk.m;
            kapk = kk.k;
            sm.kap[s] = kk.m;
        }
        const int src = (lane < NS) ? __popc(lane) : 0;
        const int kk = __shfl_sync(FULL, kapk, src);
        const V km = __shfl_sync(FULL, kapm, src);
        int eF = 0;
#pragma unroll
        for (int S = 0; S < NS; ++S)
            if (lane == S) eF = PF.e[S];
        const int Es = (lane < NS) ? eF + sm.eB[(NS - 1) ^ (lane & (NS - 1))] + kk : INT_MIN / 2;
        int em = Es;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(FULL, em, o));
        int en = (lane < NS) ? Es : INT_MAX / 2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) en = min(en, __shfl_xor_sync(FULL, en, o));
        if (lane < NS) {
            sm.esx[lane] = Es - em;
            sm.csc[lane] = km * pow2i<V>(Es - em);
        }
        if (lane == 0) {
            sm.emax = em;
            sm.fast = (em - en <= 60) ? 1 : 0;
        }
    }
    __syncthreads();
    const int Emax = sm.emax;
    const bool fast = (sm.fast != 0);
    double base = 0.0;
#pragma unroll
    for (int k = 0; k < NB; ++k) base += beta[k];
    {
        V rr[NS][NB];
        static_for<1, NS>([&](auto tc) {
            constexpr int T = decltype(tc)::value;
            static_for<0, NB>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                if constexpr ((T >> k) & 1) rr[T][k] = pow2i<V>(PF.e[T ^ (1 << k)] - PF.e[T]);
            });
        });
        V f[NS];
#pragma unroll
        for (int S = 0; S < NS; ++S) f[S] = x[S];
        int slot = slot0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int k = r.bt[c];
            if (k == -1) {
                if (slot < JCAP) {
#pragma unroll
                    for (int S = 1; S < NS; ++S) sm.fst[(S - 1) * JCAP + slot] = f[S];
                    sm.tpe[slot] = r.pe[c];
                }
                ++slot;
            }
            V fc[NB + 1];
            r.template facs<true>(c, PF, fc);
            static_for<1, NS>([&](auto tc) {
                constexpr int T = decltype(tc)::value;
                V src = V(0), rat = V(0);
                static_for<0, NB>([&](auto kc) {
                    constexpr int kb = decltype(kc)::value;
                    if constexpr ((T >> kb) & 1) {
                        src = (k == kb) ? f[T ^ (1 << kb)] : src;
                        rat = (k == kb) ? rr[T][kb] : rat;
                    }
                });
                f[T] = fma(fc[popc_c(T)] * rat, src, f[T]);
            });
        }
    }
    __syncthreads();   // forward states of every target slot in sm.fst / sm.tpe
    // ---- combine, by target slot ---------------------------------------------
    for (int sl = tid; sl < min(ntarget, JCAP); sl += NT) {
        // e^{-(2s - NB) pos} = pe^{NB - 2s}
        V q[NB + 1];
        {
            const V p1 = sm.tpe[sl], m1 = V(1) / p1;
            static_for<0, NB + 1>([&](auto sc) {
                constexpr int s = decltype(sc)::value;
                constexpr int e = NB - 2 * s;
                V v = V(1);
                if constexpr (e > 0) {
#pragma unroll
                    for (int t = 0; t < e; ++t) v *= p1;
                } else if constexpr (e < 0) {
#pragma unroll
                    for (int t = 0; t < -e; ++t) v *= m1;
                }
                q[s] = v;
            });
        }
        V sum = V(0);
        int E = 0;
        if (fast) {
#pragma unroll
            for (int S = 0; S < NS; ++S) {
                const V fS = (S == 0) ? V(1) : sm.fst[(S - 1) * JCAP + sl];
                const V gS = (S == FULLS) ? V(1) : sm.buf[((FULLS ^ S) - 1) * JCAP + sl];
                sum = fma(fS * gS, sm.csc[S] * q[popc_c(S)], sum);
            }
            if (!(sum >= pow2neg<V>(-100))) sum = V(0);
        }
        if (sum == V(0)) {
            // exact: every term as mantissa x 2^exponent
            int Em = INT_MIN / 2;
#pragma unroll
            for (int S = 0; S < NS; ++S) {
                const V fS = (S == 0) ? V(1) : sm.fst[(S - 1) * JCAP + sl];
                const V gS = (S == FULLS) ? V(1) : sm.buf[((FULLS ^ S) - 1) * JCAP + sl];
                const Sf<V> fm = sf_make<V>(fS);
                const Sf<V> gm = sf_make<V>(gS);
                if (fm.m != V(0) && gm.m != V(0)) {
                    const V z = fm.m * gm.m * sm.kap[popc_c(S)] * q[popc_c(S)];
                    const int Ez = fm.k + gm.k + sm.esx[S];
                    if (Ez > Em) {
                        sum = fma(sum, pow2neg<V>(Em - Ez), z);
                        Em = Ez;
                    } else {
                        sum = fma(z, pow2neg<V>(Ez - Em), sum);
                    }
                }
            }
            E = (sum > V(0)) ? Em : 0;
        }
        // ln M = base + (Emax + lme) ln 2 + ln(lmx), lmx in [0.5, 1) (0: M = 0);
        // the binary exponent is split off so that the logarithm is taken of
        // a mantissa
        V mx = V(0);
        int me = 0;
        if (sum > V(0)) {
            const Sf<V> sm2 = sf_make<V>(sum);
            mx = sm2.m;
            me = E + sm2.k;
        }
        sm.lmx[sl] = mx;
        sm.lme[sl] = me;
    }
    __syncthreads();   // ln M of every target slot in sm.lmx / sm.lme

    // ---- epilogue, by target slot (coalesced over the target's local indices)
    const int ntg = min(ntarget, JCAP);
    const double eps_b = tile_eps(a, b);
    const double inv_eps_b = a.teps ? 1.0 / eps_b : a.inv_eps;
    const int32_t off = a.cnt[(size_t)b * l + j];   // local index of the tile's first target
    const double base2 = base + (double)Emax * kLn2;
    if (a.mode == MODE_UPDATE) {
        // g/eps = ln mu - ln M = (ln mu - base2) - lme ln 2 - ln lmx: in
        // double-FP32 on the FP32 path (then stored as FP64), in FP64 on the
        // FP64 path
        float qmax = -INFINITY;
        bool bad = false;
        const F2 nb2 = f2_neg(f2_from_double(base2));
        for (int sl = tid; sl < ntg; sl += NT) {
            const int i = off + sl;
            const V mx = sm.lmx[sl];
            const int me = sm.lme[sl];
            double gd = -INFINITY;
            F2 gq{-INFINITY, 0.f};
            if (mx > V(0)) {
                if constexpr (sizeof(V) == 4) {
                    const float2 lm = __ldg(a.lnmuj_ff + i);
                    if (lm.x > -INFINITY) {
                        F2 t = f2_add(F2{lm.x, lm.y}, nb2);
                        t = f2_add(t, F2{-(float)me * kLn2Hi, -(float)me * kLn2Lo});
                        t = f2_add(t, F2{-logf((float)mx), 0.f});
                        gq = t;
                        gd = (double)t.hi + (double)t.lo;
                    }
                } else {
                    const double lm = __ldg(a.lnmuj + i);
                    if (lm > -INFINITY) gd = ((lm - base2) - (double)me * kLn2) - (double)vlog<V>(mx);
                    gq = f2_from_double(gd);
                }
                if (!(gq.hi < INFINITY) && gq.hi != -INFINITY) bad = true;
            } else if (__ldg(a.lnmuj + i) > -INFINITY) {
                gd = INFINITY;   // M = 0 at a point with mass: infinite potential
                bad = true;
            }
            a.gj[i] = eps_b * gd;
            if (gq.hi > -INFINITY && gq.hi < INFINITY) qmax = fmaxf(qmax, gq.hi);
            // keep g/eps for the new scaling (double-FP32 in the slot's space)
            if constexpr (sizeof(V) == 4) {
                sm.lmx[sl] = gq.hi;
                sm.lme[sl] = __float_as_int(gq.lo);
            } else {
                sm.lmx[sl] = gd;
            }
        }
        if (bad) atomicOr(a.err, ERR_NONFINITE);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qmax = fmaxf(qmax, __shfl_xor_sync(FULL, qmax, o));
        if (lane == 0) sm.wmax[w] = qmax;
        __syncthreads();
        float bx = -INFINITY;
#pragma unroll
        for (int q = 0; q < NW; ++q) bx = fmaxf(bx, sm.wmax[q]);
        if (!(bx > -INFINITY && bx < INFINITY)) bx = 0.f;
        if (tid == 0 && ntarget > 0) a.beta[(size_t)b * l + j] = (double)bx;
        // new scaled phi e^{g/eps - bx} and ln phi - bx, by slot
        for (int sl = tid; sl < ntg; sl += NT) {
            V e, lp;
            if constexpr (sizeof(V) == 4) {
                const F2 d = f2_add(F2{sm.lmx[sl], __int_as_float(sm.lme[sl])}, F2{-bx, 0.f});
                e = (d.hi == -INFINITY) ? 0.f : f2_exp(d);
                lp = d.hi + d.lo;
            } else {
                const double d = sm.lmx[sl] - (double)bx;
                e = exp(d);
                lp = d;
            }
            sm.lmx[sl] = e;
            if constexpr (sizeof(V) == 4)
                sm.lme[sl] = __float_as_int(lp);
            else
                sm.buf[sl] = lp;   // the backward states are no longer read
        }
        __syncthreads();
        // into the lanes' registers (next target's operators) and the streams
        V *ephi = static_cast<V *>(a.ephi);
        V *lphi = static_cast<V *>(a.lphi);
        int slot = slot0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            if (r.bt[c] == -1) {
                if (slot < JCAP) {
                    const V e = sm.lmx[slot];
                    V lp;
                    if constexpr (sizeof(V) == 4)
                        lp = __int_as_float(sm.lme[slot]);
                    else
                        lp = sm.buf[slot];
                    r.ph[c] = e;
                    ephi[t0 + i0 + c] = e;
                    lphi[ts + i0 + c] = lp;
                }
                ++slot;
            }
        }
    } else if (a.mode == MODE_RESIDUAL) {
        double acc = 0.0;
        for (int sl = tid; sl < ntg; sl += NT) {
            const int i = off + sl;
            const double gg = a.gj[i];
            const V mx = sm.lmx[sl];
            double marg = 0.0;
            if (gg != -INFINITY && mx > V(0))
                marg = exp_acc<V>(gg * inv_eps_b + (base2 + (double)sm.lme[sl] * kLn2 + (double)vlog<V>(mx)));
            acc += fabs(marg - a.muj[i]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (lane == 0) sm.dred[w] = acc;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < NW; ++q) t += sm.dred[q];
            a.partial[b] = t;
        }
    } else {
        for (int sl = tid; sl < ntg; sl += NT) {
            const int i = off + sl;
            const V mx = sm.lmx[sl];
            const double lnMc = (mx > V(0)) ? base2 + (double)sm.lme[sl] * kLn2 + (double)vlog<V>(mx) : -INFINITY;
            double o;
            if (a.mode == MODE_OUT_M)
                o = exp_acc<V>(lnMc);
            else if (a.mode == MODE_OUT_PLAN)
                o = (a.gj[i] == -INFINITY) ? 0.0 : exp_acc<V>(a.gj[i] * inv_eps_b + lnMc);
            else
                o = lnMc;
            a.out[i] = o;
        }
    }

    // ---- operators of the next target from the new potentials --------------
    if (a.mode == MODE_UPDATE && a.jnext >= 0) {
        __syncthreads();   // the combine no longer reads sm.buf; new beta_j written
        tile_ops_body<NB, V, NT, C, JCAP>(r, sm, a, b, a.jnext);
    }
}


template <int NB, typename V, int NT, int C, int JCAP>
cudaError_t launch_tile_impl(const SweepArgs &a, cudaStream_t st)
{
    auto kern = k_tile<NB, V, NT, C, JCAP>;
    const size_t sz = sizeof(TileSm<NB, V, NT, JCAP>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz);
    if (e != cudaSuccess) return e;
    kern<<<a.nt, NT, sz, st>>>(a);
    return cudaGetLastError();
}

template <int NB, typename V, int NT, int C, int JCAP>
cudaError_t launch_tops_impl(const SweepArgs &a, cudaStream_t st)
{
    auto kern = k_tops<NB, V, NT, C, JCAP>;
    const size_t sz = sizeof(TileSm<NB, V, NT, JCAP>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz);
    if (e != cudaSuccess) return e;
    kern<<<a.nt, NT, sz, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mmot

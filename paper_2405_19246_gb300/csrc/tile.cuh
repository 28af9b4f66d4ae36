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

// 1/x rounded to nearest (the same value as V(1) / x, without the general
// division sequence)
template <typename V>
__device__ __forceinline__ V vrcp(V x);
template <>
__device__ __forceinline__ float vrcp<float>(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <>
__device__ __forceinline__ double vrcp<double>(double x) { return __drcp_rn(x); }

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

// One-hot factors of a point: fe[s][k] = fac[s] if the point's bit is k,
// else 0 (k < 0: target or padding, all 0).  The injections below then need
// no per-lane selection of their source: the lanes of a warp hold points of
// different marginals, and every term is an FMA with a zero factor except
// the one of the point's marginal.
template <int NB, typename V>
__device__ __forceinline__ void onehot(int k, const V (&fac)[NB + 1], V (&fe)[NB + 1][NB])
{
    static_for<1, NB + 1>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        static_for<0, NB>([&](auto kc) {
            constexpr int kb = decltype(kc)::value;
            fe[s][kb] = (k == kb) ? fac[s] : V(0);
        });
    });
}

// Forward operator, one point appended on the right:
//   F[s][V] += fac[s + |V|] F[s][V \ k]  for the point's bit k in V (F[s][0] = 1).
// (A term of another bit has a zero factor, so the order of the in-place
// updates does not matter.)
template <int NB, typename V>
__device__ __forceinline__ void op_push_right(V (&op)[NB][1 << NB], const V (&fe)[NB + 1][NB])
{
    constexpr int NS = 1 << NB;
    static_for<0, NB>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        static_for<1, NS>([&](auto vc) {
            constexpr int Vv = decltype(vc)::value;
            if constexpr (op_ok<NB>(s, Vv)) {
                V acc = op[s][Vv];
                static_for<0, NB>([&](auto kc) {
                    constexpr int kb = decltype(kc)::value;
                    if constexpr ((Vv >> kb) & 1) {
                        constexpr int W = Vv ^ (1 << kb);
                        if constexpr (W == 0)
                            acc += fe[s + 1][kb];
                        else
                            acc = fma(fe[s + popc_c(Vv)][kb], op[s][W], acc);
                    }
                });
                op[s][Vv] = acc;
            }
        });
    });
}

// Backward operator built in forward point order: the new point is the first
// one the backward pass meets, so it is composed on the left:
//   B[s][V] += fac[s + 1] B[s + 1][V \ k]   (B[.][0] = 1).
template <int NB, typename V>
__device__ __forceinline__ void op_push_left(V (&op)[NB][1 << NB], const V (&fe)[NB + 1][NB])
{
    constexpr int NS = 1 << NB;
    static_for<0, NB>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        static_for<1, NS>([&](auto vc) {
            constexpr int Vv = decltype(vc)::value;
            if constexpr (op_ok<NB>(s, Vv)) {
                V acc = op[s][Vv];
                static_for<0, NB>([&](auto kc) {
                    constexpr int kb = decltype(kc)::value;
                    if constexpr ((Vv >> kb) & 1) {
                        constexpr int W = Vv ^ (1 << kb);
                        if constexpr (W == 0)
                            acc += fe[s + 1][kb];
                        else
                            acc = fma(fe[s + 1][kb], op[s + 1][W], acc);
                    }
                });
                op[s][Vv] = acc;
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

// index of entry (s, U) among the valid entries (s-major, then U)
template <int NB>
__host__ __device__ constexpr int op_index(int s, int U)
{
    int c = 0;
    for (int s2 = 0; s2 < NB; ++s2)
        for (int U2 = 1; U2 < (1 << NB); ++U2)
            if (op_ok<NB>(s2, U2)) {
                if (s2 == s && U2 == U) return c;
                ++c;
            }
    return -1;
}

// resident blocks per SM the register allocation is sized for (FP32: four
// tiles of up to 128 threads, whose shared memory also fits four to an SM, or
// two 256-thread tiles; FP64: the registers it needs)
template <typename V, int NT>
struct TileMinBlocks {
    static constexpr int value = (sizeof(V) == 4) ? (NT >= 256 ? 2 : 4) : 1;
};

template <int NB, typename V, int NT, int C, int JCAP>
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
    long long fxb[NB];    // FP32 path: baselines beta_k of the bits, fixed point (fx_log2)
    long long fxg[NB + 1];  // FP32 path: Gamma_s, fixed point
    int emax;             // combine: largest term exponent
    int fast;             // combine: every term within 2^60 of the largest
    // per target slot: ln M as mantissa (lmx) and binary exponent (lme) after
    // the combine; the new scaled phi and ln phi after the update; e^{pos}
    alignas(16) V lmx[JCAP];
    int lme[JCAP];
    V tpe[JCAP];
    // backward states (state U at row U - 1) then forward states at the
    // target slots; afterwards the lanes' transfer operators of the next
    // target ([dir][entry][lane])
    static constexpr int GSZ = (NS - 1) * JCAP;
    static constexpr int OSZ = 2 * NOP * NT;
    alignas(16) V area[2 * GSZ > OSZ ? 2 * GSZ : OSZ];
    // the lanes' points, [c][lane] (each lane reads only its own points, in
    // rolled loops: registers would need fully unrolled walks, whose code
    // does not fit the instruction cache)
    alignas(16) V pph[C * NT];   // scaled phi
    V ppe[C * NT];               // e^{pos}
    uint8_t pmd[C * NT];         // marginal (0xff: padding)
    __device__ V *gst() { return area; }
    __device__ V *fst() { return area + GSZ; }
};

// Per-tile constants of one pass, identical in every lane.
template <int NB, typename V>
struct PassC {
    V cf[NB + 1];      // e^{-max(0, a_s span)} forward / e^{min(0, a_s span)} backward, s = 1..NB
    int e[1 << NB];    // final binary scale of every state (e[0] = 0)
};

template <int NB, typename V, int NT, int C, int JCAP>
struct TileRun {
    static constexpr int NS = 1 << NB;
    static constexpr int NW = NT / 32;
    static constexpr int L = NB + 1;
    static constexpr int K = NT * C;
    static constexpr unsigned FULL = 0xffffffffu;
    using Sm = TileSm<NB, V, NT, C, JCAP>;

    int lane, w, tid;
    int n;            // points in the tile
    uint32_t ts;      // merged index of the tile's first point
    int jcur;         // target whose bit mapping bt() uses
    V span;
    Sm *sp;           // the block's shared memory (per-point arrays)

    __device__ static constexpr int rate(int s) { return s * (L - s); }
    __device__ static constexpr int arate(int s) { return rate(s) - rate(s - 1); }   // L + 1 - 2s

    __device__ __forceinline__ V ph(int c) const { return sp->pph[c * NT + tid]; }
    __device__ __forceinline__ V pe(int c) const { return sp->ppe[c * NT + tid]; }
    __device__ __forceinline__ void set_ph(int c, V v) { sp->pph[c * NT + tid] = v; }
    __device__ __forceinline__ int mid_of(int c) const { return sp->pmd[c * NT + tid]; }
    __device__ __forceinline__ static int bit_of(int m, int j) { return (m == 0xff) ? -2 : (m == j ? -1 : (m < j ? m : m - 1)); }
    // bit of point c for the current target: 0..NB-1, -1 target, -2 padding
    __device__ __forceinline__ int bt(int c) const { return bit_of(mid_of(c), jcur); }
    __device__ __forceinline__ void set_bits(int j) { jcur = j; }

    // FP32 path: the fixed-point table of the baselines of the bits (beta, per
    // thread in registers) and of Gamma_s, by threads 0..2 NB; the caller
    // passes a barrier before reading it
    __device__ __forceinline__ void fill_fx(const double (&beta)[NB]) const
    {
        if constexpr (sizeof(V) == 4) {
            if (tid < NB) {
                double bk = 0.0;
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if (k == tid) bk = beta[k];
                sp->fxb[tid] = fx_log2(bk);
            } else if (tid <= 2 * NB) {
                const int s = tid - NB;
                double g = 0.0;
#pragma unroll
                for (int q = 1; q <= NB; ++q) {
                    const V as = (V)arate(q) * span;
                    if (q <= s) g += (double)(as > V(0) ? as : V(0));
                }
                sp->fxg[s] = fx_log2(g);
            }
        }
    }

    // FP32 path: a * exp(-(sum_{k in T} beta_k + Gamma_|T|)) from the table
    __device__ __forceinline__ Sf<V> unscale_fx(Sf<V> a, int T) const
    {
        long long X = sp->fxg[__popc(T)];
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if ((T >> k) & 1) X += sp->fxb[k];
        return sf_scale_fx(a, -X);
    }

    // the lane's C points (e^{pos}, scaled phi, marginal) into shared memory
    __device__ __forceinline__ void load(const SweepArgs &a, uint32_t t0, int i0)
    {
        const V *epos = static_cast<const V *>(a.epos);
        const V *ephi = static_cast<const V *>(a.ephi);
        constexpr int PV = 16 / sizeof(V);   // values per 16-byte load
        static_assert(C % PV == 0 && C % 4 == 0, "chunk of whole 16-byte pieces");
        if (a.ugrid && i0 < n) {
            // uniform grid: e^{pos} from the table by grid steps, the marginal
            // from the merged index (l = NB + 1 points per grid point)
            const V *E = static_cast<const V *>(a.ugrid);
            const uint32_t g0 = ts / (uint32_t)L;
#pragma unroll
            for (int q = 0; q < C / PV; ++q) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(ephi + t0 + i0) + q);
                V pv[PV];
                memcpy(pv, &v, 16);
#pragma unroll
                for (int e = 0; e < PV; ++e) {
                    const int r = i0 + q * PV + e;
                    const uint32_t t = ts + (uint32_t)r;
                    const bool in = r < n;
                    sp->ppe[(q * PV + e) * NT + tid] = in ? __ldg(E + (t / (uint32_t)L - g0)) : V(1);
                    sp->pph[(q * PV + e) * NT + tid] = pv[e];
                    sp->pmd[(q * PV + e) * NT + tid] = in ? (uint8_t)(t % (uint32_t)L) : (uint8_t)0xff;
                }
            }
        } else if (i0 < n) {
#pragma unroll
            for (int q = 0; q < C / PV; ++q) {
                const uint4 u = __ldg(reinterpret_cast<const uint4 *>(epos + t0 + i0) + q);
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(ephi + t0 + i0) + q);
                V pu[PV], pv[PV];
                memcpy(pu, &u, 16);
                memcpy(pv, &v, 16);
#pragma unroll
                for (int e = 0; e < PV; ++e) {
                    sp->ppe[(q * PV + e) * NT + tid] = pu[e];
                    sp->pph[(q * PV + e) * NT + tid] = pv[e];
                }
            }
#pragma unroll
            for (int q = 0; q < C / 4; ++q) {
                const unsigned u = __ldg(reinterpret_cast<const unsigned *>(a.emid + t0 + i0) + q);
#pragma unroll
                for (int e = 0; e < 4; ++e) sp->pmd[(q * 4 + e) * NT + tid] = (uint8_t)(u >> (8 * e));
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                sp->ppe[c * NT + tid] = V(1);
                sp->pph[c * NT + tid] = V(0);
                sp->pmd[c * NT + tid] = 0xff;
            }
        }
    }

    // injection factors of point c in the pass frame, levels 1..NB:
    // forward p = pos (pe^a), backward p = span - pos (e^{a span} pe^{-a};
    // the e^{a span} is in cf)
    template <bool FWD>
    __device__ __forceinline__ void facs(int c, const PassC<NB, V> &P, V (&f)[NB + 1]) const
    {
        const V pc = pe(c);
        const V pinv = vrcp<V>(pc);
        const V up = FWD ? pc : pinv;
        const V dn = FWD ? pinv : pc;
        const V up2 = up * up, dn2 = dn * dn;
        const V phc = ph(c);
        f[0] = V(0);
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
            f[s] = (phc * P.cf[s]) * x;
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

    // Steps 1-2 of a pass: chunk-start values x[] (final per-state scales in
    // P.e) from the tile carries.  cu: on lane T < NS, the carry of state T in
    // the unscaled tile frame (carry e^{-(sum beta_T + Gamma_|T|)}).
    template <bool FWD>
    __device__ __forceinline__ void chunk_starts(Sm &sm, PassC<NB, V> &P, const Sf<V> cu, V (&x)[NS], int bits,
                                                 const V *lop)
    {
        __syncthreads();   // the previous pass has finished reading sm.wsum
        // 1. chunk operator: stored by the walk that computed the tile
        // operators of this target (lop: [entry][lane]), else one walk
        V op[NB][NS];
        op_zero<NB, V>(op);
        if (lop) {
            static_for<0, NB>([&](auto scc) {
                constexpr int s = decltype(scc)::value;
                static_for<1, NS>([&](auto vc) {
                    constexpr int U = decltype(vc)::value;
                    if constexpr (op_ok<NB>(s, U)) op[s][U] = lop[op_index<NB>(s, U) * NT + tid];
                });
            });
        } else {
#pragma unroll 4
            for (int i = 0; i < C; ++i) {
                const int c = FWD ? i : C - 1 - i;
                V f[NB + 1], fe[NB + 1][NB];
                facs<FWD>(c, P, f);
                onehot<NB, V>(bt(c), f, fe);
                op_push_right<NB, V>(op, fe);
            }
        }
        x[0] = V(1);
        // 2. level by level
        static_for<1, NB + 1>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
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
            // descending backward), exclusive by a lane shift (not incl - loc:
            // the difference would lose a small prefix next to a large own
            // value), warp totals
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
            // Lane T (state T of the level): the carry in the provisional
            // frame, the tile-end value R = carry + tile total, the final scale
            // 2^{e_T} (e_T = pi_T + exponent of R) and, in the final frame, the
            // carry's share cpf and the factor 2^{-exponent of R} (as two
            // powers of two) for the in-tile prefixes.
            int eT = 0;
            V cpf = V(0), ra = V(0), rb = V(0);
            if (lane < NS && popc_c(lane) == s) {
                const int T = lane;
                int piT = 0;
#pragma unroll
                for (int T2 = 1; T2 < NS; ++T2)
                    if (T2 == T) piT = prov_scale(T2, P.e, bits);
                Sf<V> cp = cu;
                if (cp.m != V(0)) cp.k -= piT;
                V Z = V(0);
#pragma unroll
                for (int q = 0; q < NW; ++q) Z += sm.wsum[q][T];
                const Sf<V> Rv = sf_add(cp, sf_make<V>(Z));
                if (Rv.m == V(0)) {
                    eT = piT;
                } else {
                    eT = piT + Rv.k;
                    cpf = sf_value(cp, Rv.k);
                    const int h = -(Rv.k >> 1);
                    ra = pow2i<V>(h);
                    rb = pow2i<V>(-Rv.k - h);
                }
            }
            static_for<1, NS>([&](auto tc) {
                constexpr int T = decltype(tc)::value;
                if constexpr (popc_c(T) == s) {
                    P.e[T] = __shfl_sync(FULL, eT, T);
                    const V c0 = __shfl_sync(FULL, cpf, T);
                    const V r1 = __shfl_sync(FULL, ra, T);
                    const V r2 = __shfl_sync(FULL, rb, T);
                    V wp = V(0);
#pragma unroll
                    for (int q = 0; q < NW; ++q)
                        if (FWD ? (q < w) : (q > w)) wp += sm.wsum[q][T];
                    x[T] = fma((wp + ex[T]) * r1, r2, c0);
                }
            });
        });
    }

    // ratios 2^{e_{T\k} - e_T} of the injections of a pass
    __device__ __forceinline__ static void ratios(const PassC<NB, V> &P, V (&rr)[NS][NB])
    {
        static_for<1, NS>([&](auto tc) {
            constexpr int T = decltype(tc)::value;
            static_for<0, NB>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                if constexpr ((T >> k) & 1) rr[T][k] = pow2i<V>(P.e[T ^ (1 << k)] - P.e[T]);
            });
        });
    }

    // state walk step: F_T += phi F_{T\k} for every T containing the point's
    // bit k, in each state's own scale (one-hot factors, no selection)
    __device__ __forceinline__ static void inject(V (&f)[NS], const V (&fe)[NB + 1][NB], const V (&rr)[NS][NB])
    {
        static_for<1, NS>([&](auto tc) {
            constexpr int T = NS - decltype(tc)::value;
            V acc = f[T];
            static_for<0, NB>([&](auto kc) {
                constexpr int kb = decltype(kc)::value;
                if constexpr ((T >> kb) & 1) {
                    constexpr int W = T ^ (1 << kb);
                    const V g = fe[popc_c(T)][kb] * rr[T][kb];
                    if constexpr (W == 0)
                        acc += g;
                    else
                        acc = fma(g, f[W], acc);
                }
            });
            f[T] = acc;
        });
    }
};

// ---- transfer operators of one target ----------------------------------------
// Forward and backward operators of tile b for target jn from the points in
// the lanes' registers (one walk; the backward operator is built in forward
// order by composing on the left), composed over the lanes by a tree in
// shared memory, turned into absolute scaled floats with the decay to the next
// tile base (processing order) and stored for the carry scan:
//   op[b][s][U] = T_b[s][U] exp(sum_{m in U} beta_m + Gamma_{s+|U|} - Gamma_s - w_{s+|U|} d)
// (T_b in the unscaled tile frame; d the distance to the next base).
// Expects the caller to have passed a barrier after the last use of sm.area.
template <int NB, typename V, int NT, int C, int JCAP>
__device__ __forceinline__ void tile_ops_body(TileRun<NB, V, NT, C, JCAP> &r, TileSm<NB, V, NT, C, JCAP> &sm,
                                              const SweepArgs &a, int b, int jn)
{
    using R = TileRun<NB, V, NT, C, JCAP>;
    constexpr int NS = 1 << NB;
    constexpr int L = NB + 1;
    constexpr int NOP = op_count<NB>();
    const int tid = r.tid;
    PassC<NB, V> PF, PB;
    r.setup_consts(PF, true);
    r.setup_consts(PB, false);
    {
        V opf[NB][NS], opb[NB][NS];
        op_zero<NB, V>(opf);
        op_zero<NB, V>(opb);
#pragma unroll 2
        for (int c = 0; c < C; ++c) {
            const int k = R::bit_of(r.mid_of(c), jn);
            V ff[NB + 1], fb[NB + 1], fe[NB + 1][NB];
            r.template facs<true>(c, PF, ff);
            r.template facs<false>(c, PB, fb);
            onehot<NB, V>(k, ff, fe);
            op_push_right<NB, V>(opf, fe);
            onehot<NB, V>(k, fb, fe);
            op_push_left<NB, V>(opb, fe);
        }
        V *sc = sm.area;   // [2][NOP][NT]
        // the lanes' operators also go out for the next product of target jn
        // (its chunk starts need no walk): [tile][dir][entry][lane]
        V *lo = a.lops ? static_cast<V *>(a.lops) + (size_t)b * 2 * NOP * NT : nullptr;
        static_for<0, NB>([&](auto scc) {
            constexpr int s = decltype(scc)::value;
            static_for<1, NS>([&](auto vc) {
                constexpr int U = decltype(vc)::value;
                if constexpr (op_ok<NB>(s, U)) {
                    constexpr int e = op_index<NB>(s, U);
                    sc[(0 * NOP + e) * NT + tid] = opf[s][U];
                    sc[(1 * NOP + e) * NT + tid] = opb[s][U];
                    if (lo) {
                        lo[(0 * NOP + e) * NT + tid] = opf[s][U];
                        lo[(1 * NOP + e) * NT + tid] = opb[s][U];
                    }
                }
            });
        });
    }
    // tree over the lanes' operators (positions in point order): forward, the
    // left one first; backward, the right one first
#pragma unroll 1
    for (int st = 1; st < NT; st <<= 1) {
        __syncthreads();
        if (tid < NT / st) {
            const int d = tid & 1, p = tid >> 1;
            const int i0 = 2 * p * st, i1 = i0 + st;
            V *sc = sm.area + (size_t)d * NOP * NT;
            V A[NB][NS], B[NB][NS], Rr[NB][NS];
            static_for<0, NB>([&](auto scc) {
                constexpr int s = decltype(scc)::value;
                static_for<1, NS>([&](auto vc) {
                    constexpr int U = decltype(vc)::value;
                    if constexpr (op_ok<NB>(s, U)) {
                        constexpr int e = op_index<NB>(s, U);
                        const V x0 = sc[e * NT + i0], x1 = sc[e * NT + i1];
                        A[s][U] = d ? x1 : x0;
                        B[s][U] = d ? x0 : x1;
                    }
                });
            });
            op_compose<NB, V>(A, B, Rr);
            static_for<0, NB>([&](auto scc) {
                constexpr int s = decltype(scc)::value;
                static_for<1, NS>([&](auto vc) {
                    constexpr int U = decltype(vc)::value;
                    if constexpr (op_ok<NB>(s, U)) sc[op_index<NB>(s, U) * NT + i0] = Rr[s][U];
                });
            });
        }
    }
    __syncthreads();
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
    if constexpr (sizeof(V) == 4) {
        r.fill_fx(beta);   // target jn's bits
        __syncthreads();
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
    } else if (a.shard_end) {
        dF = a.urb[b] - a.ulb[b];   // to the range's right end
        cutF = false;
    }
    if (b >= 1) {
        dB = a.urb[b] - a.urb[b - 1];
        cutB = a.seg && a.seg[b - 1] != a.seg[b];
    } else if (a.shard_end) {
        dB = a.urb[0] - a.ulb[0];   // to the range's left end
        cutB = false;
    }
    for (int t = tid; t < 2 * NOP; t += NT) {
        const int dir = t / NOP, e = t % NOP;
        int s = 0, U = 0;
        static_for<0, NB>([&](auto scc) {
            constexpr int s2 = decltype(scc)::value;
            static_for<1, NS>([&](auto vc) {
                constexpr int U2 = decltype(vc)::value;
                if constexpr (op_ok<NB>(s2, U2)) {
                    if (e == op_index<NB>(s2, U2)) {
                        s = s2;
                        U = U2;
                    }
                }
            });
        });
        const V val = sm.area[((size_t)dir * NOP + e) * NT];
        const int su = s + __popc(U);
        const double d = dir ? dB : dF;
        const bool cut = dir ? cutB : cutF;
        const double wsu = (double)su * (double)(L - su);
        Sf<V> o = sf_zero<V>();
        if (!cut) {
            if constexpr (sizeof(V) == 4) {
                long long X = sm.fxg[su] - sm.fxg[s] - fx_log2(wsu * d);
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if ((U >> k) & 1) X += sm.fxb[k];
                o = sf_scale_fx(sf_make<V>(val), X);
            } else {
                double bu = 0.0;
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    if ((U >> k) & 1) bu += beta[k];
                double gsu = 0.0, gs = 0.0;
#pragma unroll
                for (int q = 0; q <= NB; ++q) {
                    if (q == su) gsu = Gam[q];
                    if (q == s) gs = Gam[q];
                }
                o = sf_scale_exp(sf_make<V>(val), bu + gsu - gs - wsu * d);
            }
        }
        sfp<V>(dir ? a.opB : a.opF)[((size_t)b * NB + s) * NS + U] = sf_store(o);
    }
}

// Transfer operators of every tile for target a.j (when the stored ones
// belong to another target).
template <int NB, typename V, int NT, int C, int JCAP>
__global__ void __launch_bounds__(NT, TileMinBlocks<V, NT>::value) k_tops(SweepArgs a)
{
    using R = TileRun<NB, V, NT, C, JCAP>;
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    TileSm<NB, V, NT, C, JCAP> &sm = *reinterpret_cast<TileSm<NB, V, NT, C, JCAP> *>(tsm_raw);
    const int b = blockIdx.x;
    R r;
    r.tid = threadIdx.x;
    r.lane = r.tid & 31;
    r.w = r.tid >> 5;
    r.n = (int)(a.tstart[b + 1] - a.tstart[b]);
    r.span = (V)a.span[b];
    r.sp = &sm;
    r.ts = a.tstart[b];
    r.load(a, a.toff[b], r.tid * C);
    tile_ops_body<NB, V, NT, C, JCAP>(r, sm, a, b, a.j);
}

// ---- the tile product ------------------------------------------------------------

template <int NB, typename V, int NT, int C, int JCAP>
__global__ void __launch_bounds__(NT, TileMinBlocks<V, NT>::value) k_tile(SweepArgs a)
{
    using R = TileRun<NB, V, NT, C, JCAP>;
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

    r.sp = &sm;
    r.ts = ts;
    r.load(a, t0, i0);
    r.set_bits(j);
    // this tile's stored lane operators of target j (forward, then backward)
    constexpr int NOPL = op_count<NB>();
    const V *lops = a.lops ? static_cast<const V *>(a.lops) + (size_t)b * 2 * NOPL * NT : nullptr;

    // ---- target slots (rank among the tile's targets, forward order) -------
    int tcount = 0, lbits = 0;
#pragma unroll 4
    for (int c = 0; c < C; ++c) {
        const int k = r.bt(c);
        tcount += (k == -1);
        if (k >= 0) lbits |= 1 << k;
    }
    int tincl = tcount;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, tincl, o);
        if (lane >= o) tincl += y;
    }
    if (lane == 31) sm.wcnt[w] = tincl;
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
    r.fill_fx(beta);
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
            if constexpr (sizeof(V) == 4)
                cu = r.unscale_fx(cu, lane);
            else
                cu = sf_scale_exp(cu, -(sum_beta(lane) + gam_at(lane)));
        }
        r.template chunk_starts<false>(sm, PB, cu, x, bits, lops ? lops + NOPL * NT : nullptr);
    }
    {
        V rr[NS][NB];
        R::ratios(PB, rr);
        V f[NS];
#pragma unroll
        for (int S = 0; S < NS; ++S) f[S] = x[S];
        int slot = slot0 + tcount - 1;
        V *G = sm.gst();
#pragma unroll 4
        for (int i = 0; i < C; ++i) {
            const int c = C - 1 - i;
            const int k = r.bt(c);
            if (k == -1) {
                if (slot < JCAP) {
#pragma unroll
                    for (int U = 1; U < NS; ++U) G[(U - 1) * JCAP + slot] = f[U];
                }
                --slot;
            }
            V fc[NB + 1], fe[NB + 1][NB];
            r.template facs<false>(c, PB, fc);
            onehot<NB, V>(k, fc, fe);
            R::inject(f, fe, rr);
        }
#pragma unroll
        for (int S = 0; S < NS; ++S)
            if (tid == S) sm.eB[S] = PB.e[S];   // (a runtime index would put PB in local memory)
    }

    // ---- forward pass --------------------------------------------------------
    PassC<NB, V> PF;
    r.setup_consts(PF, true);
    {
        Sf<V> cu = sf_zero<V>();
        if (lane < NS && lane > 0) {
            cu = sf_load<V>(sfp<V>(a.fcarry)[(size_t)b * NS + lane]);
            if constexpr (sizeof(V) == 4)
                cu = r.unscale_fx(cu, lane);
            else
                cu = sf_scale_exp(cu, -(sum_beta(lane) + gam_at(lane)));
        }
        r.template chunk_starts<true>(sm, PF, cu, x, bits, lops);
    }
    // Per term S: F_S G_{R\S} = f g 2^{eF_S + eB_{R\S}} e^{sum beta_R} kappa_s e^{-(2s - NB) pos},
    // kappa_s = e^{Gamma_s + Gamma_{NB-s} - w_{NB-s} span}.  Terms in units of
    // 2^Emax, Emax the largest exponent over S (warp 0 computes the tile
    // constants; later barriers order them before the combine).
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
    double base = 0.0;
#pragma unroll
    for (int k = 0; k < NB; ++k) base += beta[k];
    {
        V rr[NS][NB];
        R::ratios(PF, rr);
        V f[NS];
#pragma unroll
        for (int S = 0; S < NS; ++S) f[S] = x[S];
        int slot = slot0;
        V *F = sm.fst();
#pragma unroll 4
        for (int c = 0; c < C; ++c) {
            const int k = r.bt(c);
            if (k == -1) {
                if (slot < JCAP) {
#pragma unroll
                    for (int S = 1; S < NS; ++S) F[(S - 1) * JCAP + slot] = f[S];
                    sm.tpe[slot] = r.pe(c);
                }
                ++slot;
            }
            V fc[NB + 1], fe[NB + 1][NB];
            r.template facs<true>(c, PF, fc);
            onehot<NB, V>(k, fc, fe);
            R::inject(f, fe, rr);
        }
    }
    __syncthreads();   // forward and backward states of every target slot in shared memory
    const int Emax = sm.emax;
    const bool fast = (sm.fast != 0);
    // ---- combine, by target slot ---------------------------------------------
    {
        const V *G = sm.gst();
        const V *F = sm.fst();
        for (int sl = tid; sl < min(ntarget, JCAP); sl += NT) {
            // e^{-(2s - NB) pos} = pe^{NB - 2s}
            V q[NB + 1];
            {
                const V p1 = sm.tpe[sl], m1 = vrcp<V>(p1);
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
                    const V fS = (S == 0) ? V(1) : F[(S - 1) * JCAP + sl];
                    const V gS = (S == FULLS) ? V(1) : G[((FULLS ^ S) - 1) * JCAP + sl];
                    sum = fma(fS * gS, sm.csc[S] * q[popc_c(S)], sum);
                }
                if (!(sum >= pow2neg<V>(-100))) sum = V(0);
            }
            if (sum == V(0)) {
                // exact: every term as mantissa x 2^exponent
                int Em = INT_MIN / 2;
#pragma unroll
                for (int S = 0; S < NS; ++S) {
                    const V fS = (S == 0) ? V(1) : F[(S - 1) * JCAP + sl];
                    const V gS = (S == FULLS) ? V(1) : G[((FULLS ^ S) - 1) * JCAP + sl];
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
                sm.area[sl] = lp;   // the backward states are no longer read
        }
        __syncthreads();
        // into the lanes' points (next target's operators) and the streams
        V *ephi = static_cast<V *>(a.ephi);
        V *lphi = static_cast<V *>(a.lphi);
        int slot = slot0;
#pragma unroll 4
        for (int c = 0; c < C; ++c) {
            if (r.bt(c) == -1) {
                if (slot < JCAP) {
                    const V e = sm.lmx[slot];
                    V lp;
                    if constexpr (sizeof(V) == 4)
                        lp = __int_as_float(sm.lme[slot]);
                    else
                        lp = sm.area[slot];
                    r.set_ph(c, e);
                    ephi[t0 + i0 + c] = e;
                    lphi[ts + i0 + c] = lp;
                }
                ++slot;
            }
        }
    } else if (a.mode == MODE_OBJ) {
        // the plan marginal marg = phi_j M_j and the tile's sums of the
        // objective terms (Eq. k-mmot distance): mass, L1 error, g marg, g mu
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int sl = tid; sl < ntg; sl += NT) {
            const int i = off + sl;
            const double gg = a.gj[i];
            const double mu = a.muj[i];
            const V mx = sm.lmx[sl];
            double marg = 0.0;
            if (gg != -INFINITY && mx > V(0))
                marg = exp_acc<V>(gg * inv_eps_b + (base2 + (double)sm.lme[sl] * kLn2 + (double)vlog<V>(mx)));
            acc[0] += marg;
            acc[1] += fabs(marg - mu);
            if (gg != -INFINITY) {
                acc[2] += gg * marg;
                acc[3] += gg * mu;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(FULL, acc[q], o);
        }
        __syncthreads();   // sm.area is free
        double *red = reinterpret_cast<double *>(sm.area);   // [4][NW]
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) red[q * NW + w] = acc[q];
        }
        __syncthreads();
        if (tid < 4) {
            double t = 0.0;
            for (int q = 0; q < NW; ++q) t += red[tid * NW + q];
            a.part4[(size_t)b * 4 + tid] = t;
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
        __syncthreads();   // the epilogue no longer reads sm.area; new beta_j written
        tile_ops_body<NB, V, NT, C, JCAP>(r, sm, a, b, a.jnext);
    }
}


template <int NB, typename V>
cudaError_t launch_tile_impl(const SweepArgs &a, cudaStream_t st)
{
    using TS = TShape<NB, V>;
    auto kern = k_tile<NB, V, TS::NT, TS::C, TS::JCAP>;
    const size_t sz = sizeof(TileSm<NB, V, TS::NT, TS::C, TS::JCAP>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz);
    if (e != cudaSuccess) return e;
    kern<<<a.nt, TS::NT, sz, st>>>(a);
    return cudaGetLastError();
}

template <int NB, typename V>
cudaError_t launch_tops_impl(const SweepArgs &a, cudaStream_t st)
{
    using TS = TShape<NB, V>;
    auto kern = k_tops<NB, V, TS::NT, TS::C, TS::JCAP>;
    const size_t sz = sizeof(TileSm<NB, V, TS::NT, TS::C, TS::JCAP>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz);
    if (e != cudaSuccess) return e;
    kern<<<a.nt, TS::NT, sz, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mmot

// Transfer operator of a whole shard (a contiguous range of the merged order
// held by one plan), for the exchange between shards of one instance.
//
// The forward states of Sec. 4.2 are linear in the states entering a range:
// a state S of level s at the left end x_L (before the range's first point)
// reaches S + U at the right end x_R (after its last point) with a factor
// that depends only on s and on the marginals U it picks up inside the range
// (the rates w_{s+|V|} of the levels it passes and the injections of U's
// points), and stays S with the decay exp(-w_s (x_R - x_L)/eps).  The tile
// operators op[b][s][U] (tile b's base to the next base, decay included) and
// the tile decays compose to that operator in processing order:
//     (X then Y)[s][U] = sum_{V subset U} X[s][V] Y[s + |V|][U \ V]
// (entry [s][0] the decay of level s).  The backward operator is the mirror
// image (right end to left end).  The last tile in processing order carries
// the decay to the range's own end (x_R forward, x_L backward).
//
// One block per direction; each thread composes a contiguous run of tiles
// in shared memory, then a tree over the threads.  The result goes out as
// FP64 natural logarithms (-inf for 0): lnop[dir][s][U], s = 0..NB.
#pragma once
#include "sweep.cuh"

namespace mmot {

// X <- X then Y, in place.  X and Y: [NB + 1][NS] scaled floats ([s][0] the
// decay of level s); entries with s + |U| > NB stay 0.  U runs by decreasing
// size so that every X[s][V], V inside U, is still the old value.
template <int NB, typename V, typename GetY>
__device__ void sf_op_then(SfT<V> *X, GetY &&Y)
{
    constexpr int NS = 1 << NB;
    for (int s = 0; s <= NB; ++s) {
        for (int sz = NB - s; sz >= 1; --sz) {
            for (int U = 1; U < NS; ++U) {
                if (__popc(U) != sz) continue;
                Sf<V> acc = sf_zero<V>();
                // V = 0: X[s][0] Y[s][U];  V = U: X[s][U] Y[s + |U|][0]
                for (int Vs = U;; Vs = (Vs - 1) & U) {
                    const Sf<V> x = sf_load<V>(X[s * NS + Vs]);
                    if (x.m != V(0)) acc = sf_add(acc, sf_mul(x, Y(s + __popc(Vs), U ^ Vs)));
                    if (Vs == 0) break;
                }
                X[s * NS + U] = sf_store(acc);
            }
        }
        X[s * NS] = sf_store(sf_mul(sf_load<V>(X[s * NS]), Y(s, 0)));
    }
}

template <int NB, typename V>
__global__ void __launch_bounds__(64) k_opcompose(SweepArgs a, double *lnop)
{
    constexpr int NS = 1 << NB;
    constexpr int NE = (NB + 1) * NS;
    constexpr int NTH = 64;
    extern __shared__ __align__(16) unsigned char k_opcompose_sm[];
    SfT<V> *acc = reinterpret_cast<SfT<V> *>(k_opcompose_sm);   // [NTH][NE]
    const bool fwd = (blockIdx.x == 0);
    const SfT<V> *op = sfp<V>(fwd ? a.opF : a.opB);
    const SfT<V> *dec = sfp<V>(fwd ? a.pdecF : a.pdecB);
    const int nt = a.nt, tid = threadIdx.x;
    const int R = (nt + NTH - 1) / NTH;
    const int v0 = min(nt, tid * R), v1 = min(nt, v0 + R);
    SfT<V> *X = acc + (size_t)tid * NE;
    for (int e = 0; e < NE; ++e) X[e] = (e % NS == 0) ? sf_one_st<V>() : sf_store(sf_zero<V>());
    for (int v = v0; v < v1; ++v) {
        const int b = fwd ? v : nt - 1 - v;
        sf_op_then<NB, V>(X, [&](int t, int W) -> Sf<V> {
            if (W == 0) return sf_load<V>(__ldg(dec + (size_t)b * (NB + 1) + t));
            if (t >= NB || t + __popc(W) > NB) return sf_zero<V>();
            return sf_load<V>(__ldg(op + ((size_t)b * NB + t) * NS + W));
        });
    }
    __syncthreads();
    for (int st = 1; st < NTH; st <<= 1) {
        if (tid % (2 * st) == 0 && tid + st < NTH) {
            const SfT<V> *Yp = acc + (size_t)(tid + st) * NE;
            sf_op_then<NB, V>(X, [&](int t, int W) -> Sf<V> {
                if (t + __popc(W) > NB) return sf_zero<V>();
                return sf_load<V>(Yp[t * NS + W]);
            });
        }
        __syncthreads();
    }
    for (int e = tid; e < NE; e += NTH) {
        const Sf<V> x = sf_load<V>(acc[e]);
        const int s = e / NS, U = e % NS;
        double y = -INFINITY;
        if (x.m != V(0) && s + __popc(U) <= NB) y = log((double)x.m) + (double)x.k * kLn2;
        lnop[(size_t)(fwd ? 0 : 1) * NE + e] = y;
    }
}

template <int NB, typename V>
cudaError_t launch_opcompose_impl(const SweepArgs &a, cudaStream_t st, double *lnop)
{
    constexpr int NE = (NB + 1) * (1 << NB);
    const size_t smem = (size_t)64 * NE * sizeof(SfT<V>);
    auto kern = k_opcompose<NB, V>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<2, 64, smem, st>>>(a, lnop);
    return cudaGetLastError();
}

}  // namespace mmot

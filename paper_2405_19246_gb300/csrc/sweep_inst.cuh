// Explicit instantiation of the sweep launchers for one bit count NB.
#pragma once
#include "shapes.cuh"
#include "sweep.cuh"
#include "warp.cuh"
#include "tile.cuh"
#include "shard.cuh"

// launchers of the three-phase design, defined for NB <= kMaxOpBits
#define MMOT_INSTANTIATE_OPS(NB_, V_)                                                  \
    namespace mmot {                                                                   \
    template <>                                                                        \
    cudaError_t launch_tileop<NB_, V_>(const SweepArgs &a, cudaStream_t s)             \
    {                                                                                  \
        return launch_tops_impl<NB_, V_>(a, s);                                        \
    }                                                                                  \
    template <>                                                                        \
    cudaError_t launch_prod<NB_, V_>(const SweepArgs &a, cudaStream_t s)               \
    {                                                                                  \
        return launch_tile_impl<NB_, V_>(a, s);                                        \
    }                                                                                  \
    template <>                                                                        \
    cudaError_t launch_carry<NB_, V_>(const SweepArgs &a, cudaStream_t s)              \
    {                                                                                  \
        return launch_carry_impl<NB_, V_>(a, s);                                       \
    }                                                                                  \
    template <>                                                                        \
    cudaError_t launch_opcompose<NB_, V_>(const SweepArgs &a, cudaStream_t s, double *o)\
    {                                                                                  \
        return launch_opcompose_impl<NB_, V_>(a, s, o);                                \
    }                                                                                  \
    }

// launchers of the level passes and warp-tile products (l >= 6, warp.cuh)
#define MMOT_INSTANTIATE_LEVELS(NB_, V_)                                               \
    namespace mmot {                                                                   \
    template <>                                                                        \
    cudaError_t launch_lagg<NB_, V_>(const SweepArgs &a, cudaStream_t s, int L, int f) \
    {                                                                                  \
        return launch_wpass_impl<NB_, V_>(a, s, L, f);                                 \
    }                                                                                  \
    template <>                                                                        \
    cudaError_t launch_lscan<NB_, V_>(const SweepArgs &a, cudaStream_t s, int L, int f)\
    {                                                                                  \
        return launch_lscan_impl<NB_, V_>(a, s, L, f);                                 \
    }                                                                                  \
    template <>                                                                        \
    cudaError_t launch_prod<NB_, V_>(const SweepArgs &a, cudaStream_t s)               \
    {                                                                                  \
        return launch_wprod_impl<NB_, V_>(a, s);                                       \
    }                                                                                  \
    template <>                                                                        \
    cudaError_t launch_wbwd<NB_, V_>(const SweepArgs &a, cudaStream_t s)               \
    {                                                                                  \
        return launch_wbwd_impl<NB_, V_>(a, s);                                        \
    }                                                                                  \
    }

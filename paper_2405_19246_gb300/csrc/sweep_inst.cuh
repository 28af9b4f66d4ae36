// Explicit instantiation of the sweep launchers for one bit count NB.
#pragma once
#include "shapes.cuh"
#include "sweep.cuh"

#define MMOT_INSTANTIATE(NB_)                                                          \
    namespace mmot {                                                                   \
    template <>                                                                        \
    cudaError_t launch_bwd<NB_, float>(const SweepArgs &a, cudaStream_t s)             \
    {                                                                                  \
        using S = Shape<NB_, float>;                                                   \
        return launch_bwd_impl<NB_, float, S::NT, S::C, S::JCAP>(a, s);                \
    }                                                                                  \
    template <>                                                                        \
    cudaError_t launch_fwd<NB_, float>(const SweepArgs &a, cudaStream_t s)             \
    {                                                                                  \
        using S = Shape<NB_, float>;                                                   \
        return launch_fwd_impl<NB_, float, S::NT, S::C, S::JCAP>(a, s);                \
    }                                                                                  \
    template <>                                                                        \
    cudaError_t launch_bwd<NB_, double>(const SweepArgs &a, cudaStream_t s)            \
    {                                                                                  \
        using S = Shape<NB_, double>;                                                  \
        return launch_bwd_impl<NB_, double, S::NT, S::C, S::JCAP>(a, s);               \
    }                                                                                  \
    template <>                                                                        \
    cudaError_t launch_fwd<NB_, double>(const SweepArgs &a, cudaStream_t s)            \
    {                                                                                  \
        using S = Shape<NB_, double>;                                                  \
        return launch_fwd_impl<NB_, double, S::NT, S::C, S::JCAP>(a, s);               \
    }                                                                                  \
    }

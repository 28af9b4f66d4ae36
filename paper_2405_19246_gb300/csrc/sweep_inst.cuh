// Explicit instantiation of the sweep launchers for one bit count NB.
#pragma once
#include "shapes.cuh"
#include "sweep.cuh"

// launchers of the three-phase design, defined for NB <= kMaxOpBits
#define MMOT_INSTANTIATE_OPS(NB_, V_)                                                  \
    namespace mmot {                                                                   \
    template <>                                                                        \
    cudaError_t launch_tileop<NB_, V_>(const SweepArgs &a, cudaStream_t s)             \
    {                                                                                  \
        using S = Shape<NB_, V_>;                                                      \
        return launch_tileop_impl<NB_, V_, S::NT, S::C, S::JCAP>(a, s);                \
    }                                                                                  \
    template <>                                                                        \
    cudaError_t launch_prod<NB_, V_>(const SweepArgs &a, cudaStream_t s)               \
    {                                                                                  \
        using S = Shape<NB_, V_>;                                                      \
        return launch_prod_impl<NB_, V_, S::NT, S::C, S::JCAP>(a, s);                  \
    }                                                                                  \
    template <>                                                                        \
    cudaError_t launch_carry<NB_, V_>(const SweepArgs &a, cudaStream_t s)              \
    {                                                                                  \
        return launch_carry_impl<NB_, V_>(a, s);                                       \
    }                                                                                  \
    }

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

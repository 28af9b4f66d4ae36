// Tile shapes per bit count NB (= l - 1) and precision.
//
// K = NT * C points per tile, one chunk of C consecutive points per thread.
// The backward states of a tile are kept at its target points in shared memory
// (NS x JCAP values), so K shrinks as the state count NS = 2^NB grows.
// span_limit bounds max_s w_s * (x_last - x_first)/eps inside a tile, which
// keeps every in-tile exponent small enough for the precision: the rounding
// of a position enters an exponent as about u * span_limit (FP32: 6e-8 * 24;
// FP64: 1.1e-16 * 50, so ln M keeps its 1e-12 bound).
#pragma once
#include "mmot_internal.cuh"

namespace mmot {

template <int NB, typename V>
struct Shape;

// JCAP: at most this many points of one marginal in a tile (the tiling cuts a
// tile early otherwise); half the tile for l >= 3.
#define MMOT_SHAPE(NB_, V_, NT_, C_)                             \
    template <>                                                  \
    struct Shape<NB_, V_> {                                      \
        static constexpr int NT = NT_;                           \
        static constexpr int C = C_;                             \
        static constexpr int K = NT_ * C_;                       \
        static constexpr int JCAP = (NB_ >= 2) ? NT_ * C_ / 2 : NT_ * C_; \
    };

MMOT_SHAPE(1, float, 256, 16)
MMOT_SHAPE(2, float, 256, 16)
MMOT_SHAPE(3, float, 256, 8)
MMOT_SHAPE(4, float, 256, 4)
MMOT_SHAPE(5, float, 128, 4)
MMOT_SHAPE(6, float, 128, 2)
MMOT_SHAPE(7, float, 128, 1)
MMOT_SHAPE(1, double, 256, 8)
MMOT_SHAPE(2, double, 256, 8)
MMOT_SHAPE(3, double, 256, 4)
MMOT_SHAPE(4, double, 256, 2)
MMOT_SHAPE(5, double, 128, 2)
MMOT_SHAPE(6, double, 128, 1)
MMOT_SHAPE(7, double, 64, 1)
#undef MMOT_SHAPE

// points per warp tile of the products with l >= 6 (warp.cuh; the plan's
// tiling uses at most this many, a quarter of them of one marginal: with
// l >= 6 marginals a tile holds about K/l points of each, and the backward
// states kept per target (2^{l-1} scaled floats) set the shared memory)
template <int NB, typename V>
struct WShape {
    static constexpr int K = (sizeof(V) == 4) ? (NB <= 5 ? 128 : 64) : (NB <= 5 ? 64 : 32);
    static constexpr int JCAP = K / 4;
};

// Lanes per tile and points per lane of the tile kernels of l <= 5
// (tile.cuh), NT * C = Shape<NB, V>::K.  JCAP: the most points of one
// marginal a tile may hold (the tiling cuts a tile earlier otherwise): the
// share 1/l of a tile plus 32, a multiple of 32; the tile
// kernels keep the forward and backward states of every target point in
// shared memory, so the bound sets their shared memory.
template <int NB, typename V>
struct TShape {
    static constexpr int C = (sizeof(V) == 4) ? 16 : 8;
    static constexpr int K = Shape<NB, V>::K;
    static constexpr int NT = K / C;
    static constexpr int JCAP = ((K / (NB + 1) + 32) + 31) / 32 * 32;
    static_assert(NT % 32 == 0 && NT * C == K, "tile of whole warps");
};

constexpr double kSpanLimitF32 = 24.0;
constexpr double kSpanLimitF64 = 50.0;

}  // namespace mmot

// Level-pass and warp-tile kernels for l = 6 marginals (5 state bits).
#include "sweep_inst.cuh"
MMOT_INSTANTIATE_LEVELS(5, float)
MMOT_INSTANTIATE_LEVELS(5, double)

// Level-pass and warp-tile kernels for l = 7 marginals (6 state bits).
#include "sweep_inst.cuh"
MMOT_INSTANTIATE_LEVELS(6, float)
MMOT_INSTANTIATE_LEVELS(6, double)

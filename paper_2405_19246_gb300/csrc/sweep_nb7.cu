// Level-pass and warp-tile kernels for l = 8 marginals (7 state bits).
#include "sweep_inst.cuh"
MMOT_INSTANTIATE_LEVELS(7, float)
MMOT_INSTANTIATE_LEVELS(7, double)

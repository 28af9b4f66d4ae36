// Sweep kernels for l = 2 marginals (1 state bits).
#include "sweep_inst.cuh"
MMOT_INSTANTIATE_OPS(1, float)
MMOT_INSTANTIATE_OPS(1, double)

// Sweep kernels for l = 3 marginals (2 state bits).
#include "sweep_inst.cuh"
MMOT_INSTANTIATE_OPS(2, float)
MMOT_INSTANTIATE_OPS(2, double)

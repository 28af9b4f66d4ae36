// Sweep kernels for l = 4 marginals (3 state bits).
#include "sweep_inst.cuh"
MMOT_INSTANTIATE_OPS(3, float)
MMOT_INSTANTIATE_OPS(3, double)

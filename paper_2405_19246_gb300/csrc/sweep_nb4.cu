// Sweep kernels for l = 5 marginals (4 state bits).
#include "sweep_inst.cuh"
MMOT_INSTANTIATE_OPS(4, float)
MMOT_INSTANTIATE_OPS(4, double)

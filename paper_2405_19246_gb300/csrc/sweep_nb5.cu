// Sweep kernels for l = 6 marginals (5 state bits).
#include "sweep_inst.cuh"
MMOT_INSTANTIATE(5)

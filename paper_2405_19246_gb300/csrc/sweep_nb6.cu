// Sweep kernels for l = 7 marginals (6 state bits).
#include "sweep_inst.cuh"
MMOT_INSTANTIATE(6)

// Sweep kernels for l = 8 marginals (7 state bits).
#include "sweep_inst.cuh"
MMOT_INSTANTIATE(7)

// Objective kernels for l = 6 marginals.
#include "objective.cuh"
MMOT_INSTANTIATE_OBJECTIVE(6)

// Objective kernels for l = 2 marginals.
#include "objective.cuh"
MMOT_INSTANTIATE_OBJECTIVE(2)

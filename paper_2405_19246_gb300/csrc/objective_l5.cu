// Objective kernels for l = 5 marginals.
#include "objective.cuh"
MMOT_INSTANTIATE_OBJECTIVE(5)
